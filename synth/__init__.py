"""Seeded synthetic inputs for the Asp-Clean2016 minor cycle.

This module produces data only: sky models, point spread functions, dirty
images and noise, drawn from ``numpy.random.default_rng`` seeded with
``SeedSequence([config_id, seed])``.  It holds none of the deconvolution
method's arithmetic (no Gaussian fitting, no deconvolution, no subtraction);
both the FP64 oracle and the CUDA path consume what it writes.

The paper's own data (the simulated EVLA L-band observation of M31, Sect. 4)
is not available, so these generators stand in for it with the shapes and
value ranges of the five workload configurations:

* ``config1``: 256x256, 5 points + 3 Gaussians, analytic PSF (Gaussian main
  lobe sigma 1.5 px plus a 2 % ring at 12 px), noise 1e-3.
* ``config2``: 1024x1024, 50 power-law points, 20 Gaussians, one k^-3
  Gaussian-random-field patch, PSF = FFT of a seeded uv mask, noise 1e-4.
* ``config3``: 4096x4096 scaled-up config 1 (400 points, 150 Gaussians,
  4 GRF patches, PSF main lobe 2.5 px, ring at 20 px).
* ``config4``: 64 config-1-style images of uneven sizes.
"""
from .sky import (  # noqa: F401
    SynthImage,
    analytic_psf,
    config1,
    config2,
    config3,
    config4,
    small_case,
    gaussian_psf,
    elliptical_psf,
    elliptical_field,
    rng_for,
)
from .mlp_init import mlp_init  # noqa: F401,E402  (initial weights of the learned-init network)
