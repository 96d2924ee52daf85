"""Pins of the oracle's damped solve, cholesky_solve_damped (Marquardt's
damping A + lam diag(A), LM reading 9), against what the mathematics fixes
rather than a retyped formula:

* a diagonal A gives delta_i = g_i / (A_ii (1 + lam)) in closed form;
* lam = 0 is the Gauss-Newton step: A delta = g;
* lam -> infinity tends to lam delta = diag(A)^-1 g, the diagonally scaled
  gradient step;
* a parameter the data does not constrain (a zero row and column) is damped
  with 1: delta_i = g_i / lam;
* rescaling the parameters (A -> S A S, g -> S g) rescales the step
  (delta -> S^-1 delta), Marquardt's reason for damping with diag(A);
* the step is a descent direction (g . delta > 0) and shrinks as lam grows.

Planted mistakes at the end check that these pins catch damping with lam I
and damping with lam diag(A)^2."""
import numpy as np
import pytest

import oracle as O
import oracle.asp_oracle as OA


def _spd(n, seed, spread=1.0):
    rng = np.random.default_rng(seed)
    M = rng.normal(size=(n, n))
    s = np.exp(rng.uniform(-spread, spread, n))          # parameters on different scales
    return (s[:, None] * (M @ M.T + 0.5 * np.eye(n))) * s[None, :], rng.normal(size=n)


def test_diagonal_matrix_closed_form():
    A = np.diag([4.0, 0.25, 9.0, 1e-3])
    g = np.array([1.0, -2.0, 0.5, 3.0])
    for lam in (0.0, 1e-3, 0.37, 10.0):
        want = g / (np.diag(A) * (1.0 + lam))
        np.testing.assert_allclose(O.cholesky_solve_damped(A, g, lam), want, rtol=1e-14)


def test_undamped_step_solves_the_normal_equations():
    A, g = _spd(7, 1)
    d = O.cholesky_solve_damped(A, g, 0.0)
    assert np.max(np.abs(A @ d - g)) < 1e-12 * np.max(np.abs(g)) * np.linalg.cond(A)


def test_large_lambda_tends_to_the_scaled_gradient_step():
    A, g = _spd(6, 2, spread=2.0)
    for lam in (1e6, 1e9):
        d = O.cholesky_solve_damped(A, g, lam)
        # (A + lam D) d = g  =>  lam d = D^-1 g - D^-1 A d, and |d| = O(1/lam)
        np.testing.assert_allclose(lam * d, g / np.diag(A), rtol=50.0 / lam * np.linalg.norm(A, 2)
                                   / np.min(np.diag(A)))


def test_unconstrained_parameter_is_damped_with_one():
    A, g = _spd(5, 3)
    A[2, :] = 0.0
    A[:, 2] = 0.0
    lam = 0.25
    d = O.cholesky_solve_damped(A, g, lam)
    assert d[2] == pytest.approx(g[2] / lam, rel=1e-14)
    # the other four unknowns are those of the system with parameter 2 removed
    keep = [0, 1, 3, 4]
    Ak = A[np.ix_(keep, keep)]
    dk = O.cholesky_solve_damped(Ak, g[keep], lam)
    np.testing.assert_allclose(d[keep], dk, rtol=1e-12)
    assert O.cholesky_solve_damped(A, g, 0.0) is None      # singular without damping


def test_step_is_invariant_under_parameter_rescaling():
    A, g = _spd(6, 4)
    s = np.array([1e-3, 0.5, 2.0, 10.0, 1.0, 300.0])
    for lam in (1e-3, 0.1, 10.0):
        d = O.cholesky_solve_damped(A, g, lam)
        ds = O.cholesky_solve_damped(s[:, None] * A * s[None, :], s * g, lam)
        np.testing.assert_allclose(ds, d / s, rtol=1e-10)


def test_step_is_descent_and_shrinks_with_lambda():
    A, g = _spd(8, 5, spread=1.5)
    norms = []
    for lam in (0.0, 1e-2, 1.0, 1e2, 1e4):
        d = O.cholesky_solve_damped(A, g, lam)
        assert g @ d > 0.0
        norms.append(np.sqrt(d @ (np.diag(A) * d)))          # the step in the scaled metric
    assert all(b < a for a, b in zip(norms, norms[1:]))


def test_not_positive_definite_is_reported():
    A, g = _spd(4, 6)
    assert O.cholesky_solve_damped(-A, g, 0.0) is None
    B = A.copy()
    B[0, 1] = B[1, 0] = 10.0 * np.sqrt(A[0, 0] * A[1, 1])   # indefinite 2 x 2 block
    assert O.cholesky_solve_damped(B, g, 0.0) is None


# ---------------------------------------------------------------- planted mistakes

def _plant(monkeypatch, fn):
    monkeypatch.setattr(OA, "cholesky_solve_damped", fn)
    monkeypatch.setattr(O, "cholesky_solve_damped", fn)


def test_damping_with_identity_is_caught(monkeypatch):
    def bad(A, g, lam):                       # Levenberg's lam I, not Marquardt's lam diag(A)
        return np.linalg.solve(A + lam * np.eye(len(g)), g)

    _plant(monkeypatch, bad)
    with pytest.raises(AssertionError):
        test_diagonal_matrix_closed_form()
    with pytest.raises(AssertionError):
        test_step_is_invariant_under_parameter_rescaling()


def test_damping_with_squared_diagonal_is_caught(monkeypatch):
    def bad(A, g, lam):
        return np.linalg.solve(A + lam * np.diag(np.diag(A) ** 2), g)

    _plant(monkeypatch, bad)
    with pytest.raises(AssertionError):
        test_diagonal_matrix_closed_form()
    with pytest.raises(AssertionError):
        test_large_lambda_tends_to_the_scaled_gradient_step()
