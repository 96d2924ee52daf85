"""FP64 CPU oracle of the Asp-Clean2016 minor cycle -- TEST INFRASTRUCTURE.

This package is the plain, slow, obviously-correct statement of what the
CUDA path computes.  It exists to check that path and nothing else: only the
test suite, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference
arm of ``bench.py`` may import it.  The product library never calls it and
shares no code with it (the only common dependency is the ``synth`` input
generator, which holds none of the method's arithmetic).

Everything is NumPy in float64, vectorised over pixels only where the
definition is an independent per-pixel formula or a plain sum; loops follow
the order of the algorithm in the paper (Sect. 2 steps 1-4, Sect. 3 Eqs. 6-8,
and the initial-value heuristic of Sect. 3).

Parity pins (what fixes each function independently of itself) live in
``tests/test_oracle_*.py``.  Functions whose behaviour is a reading of a gap
in the paper (active-set rule, LM constants, fit window, switch heuristic
details) are pinned only to the paper's degenerate cases and to invariants;
they carry a "reading" note in their docstrings.
"""
from .asp_oracle import *  # noqa: F401,F403
from . import mlp_oracle  # noqa: F401,E402  (learned initial values: MLP, loss, optimiser)
from . import elliptical  # noqa: F401,E402  (elliptical beam and components)
from . import multichannel  # noqa: F401,E402  (joint multi-channel fits)
