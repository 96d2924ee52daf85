"""FP32 error bounds of the GPU's LM arithmetic, derived from its operations.

The CUDA path evaluates the Eq. 6 model, residual and Jacobian per pixel in
FP32, sums [J | r]^T [J | r] with compensated FP32 leaves and error-free
pair trees, and solves the damped normal equations (A + lambda D) delta = g
with an FP32 Cholesky factor of the scaled matrix (refined in FP64 when a
pivot is small).  The bounds below follow those operations; the oracle's
FP64 values are treated as exact.

u32 = 2^-24 (unit roundoff of FP32).

* Jacobian entry of member k at a pixel: relative error (8 + 2 |arg_k|) u32,
  arg_k = r^2 / (2 w_k^2) (the exponent argument's rounding grows with it,
  plus ex2 and the products).
* Residual: 8 u32 (|T| + sum_k |g_k|) -- the target's staging (R plus the
  added-back members) and the model sum -- plus each member's own
  evaluation error.
* Sums: (64 + log2 n + 16) u32 of sum |terms| (leaf of <= 64 pixels, Kahan
  across leaves, pair trees; 16 for the final roundings), plus an absolute
  floor for FP32 underflow of the products.
* Damped solve (Higham, Accuracy and Stability of Numerical Algorithms,
  Thm 10.3 and 8.5): the scaled matrix S (A + lambda D) S has a unit
  diagonal, so its Cholesky factor's rows have unit norm and the backward
  error of factor + two triangular solves is at most (3P + 6) u32 per entry
  of the scaled matrix, i.e. (3P + 6) u32 sqrt(M_ii M_jj) of M = A + lambda
  D; the FP32 copies of A, g and lambda add u32 |A|, u32 |g|, u32 lambda D.
  The step error then is, to first order, |M^-1| (dg + dM |delta|).
"""
from __future__ import annotations

import numpy as np

import oracle as O

U32 = 2.0 ** -24


def pass_bounds(T, xs, ys, theta, extra_scale=None):
    """Oracle normal equations at theta and the FP32 bounds of the GPU's
    pixel pass.  Returns dict(A, g, chi2, bA, bg, bc, r).  ``extra_scale``:
    per-pixel magnitudes that entered the GPU's FP32 target beyond |T|
    (e.g. sum of |g| of the added-back members)."""
    theta = np.asarray(theta, dtype=np.float64).ravel()
    xs = np.asarray(xs, dtype=np.float64).ravel()
    ys = np.asarray(ys, dtype=np.float64).ravel()
    T = np.asarray(T, dtype=np.float64).ravel()
    model, J = O.model_and_jacobian(theta, xs, ys)
    r = T - model
    n = xs.size
    th = theta.reshape(-1, 4)
    eps = np.stack([(8 + 2 * ((xs - x0) ** 2 + (ys - y0) ** 2) / (2 * w * w)) * U32 for _, x0, y0, w in th], 1)
    aJ = np.abs(J)
    EJ = np.repeat(eps, 4, axis=1) * aJ
    scale_r = np.abs(T) + O.gauss_model(np.abs(theta), xs, ys)
    if extra_scale is not None:
        scale_r = scale_r + np.asarray(extra_scale, dtype=np.float64).ravel()
    Er = 8 * U32 * scale_r + (aJ[:, 0::4] * eps * np.abs(th[:, 0])).sum(1)
    c = 64 + np.log2(max(n, 2)) + 16
    tiny = 4 * n * 2.0 ** -149
    A = J.T @ J
    g = J.T @ r
    chi2 = float(r @ r)
    bA = EJ.T @ aJ + aJ.T @ EJ + c * U32 * (aJ.T @ aJ) + tiny
    bg = EJ.T @ np.abs(r) + aJ.T @ Er + c * U32 * (aJ.T @ np.abs(r)) + tiny
    bc = 2 * float(np.abs(r) @ Er) + c * U32 * chi2 + tiny
    return dict(A=A, g=g, chi2=chi2, bA=bA, bg=bg, bc=bc, r=r)


def marquardt_diag(A):
    d = np.diag(A).copy()
    d[~(d > 0)] = 1.0
    return d


def step_bound(A, g, lam, bA, bg, delta):
    """First-order bound of |delta_gpu - delta| for the damped step delta =
    M^-1 g, M = A + lam D, from the FP32 errors bA, bg of the normal
    equations and the FP32 solve.  Returns (bound, kappa) with kappa =
    max row sum of |M^-1| dM on the scaled system S M S, S = diag(M)^-1/2
    (the first-order bound is meaningful while kappa is well below 1)."""
    P = A.shape[0]
    d = marquardt_diag(A)
    M = A + lam * np.diag(d)
    Mi = np.linalg.inv(M)
    dm = np.sqrt(np.abs(np.diag(M)))
    dM = bA + U32 * np.abs(A) + (3 * P + 6) * U32 * np.outer(dm, dm)
    dM = dM + np.diag(lam * (np.diag(bA) + 2 * U32 * d))
    dg = bg + U32 * np.abs(g)
    aMi = np.abs(Mi)
    bound = aMi @ (dg + dM @ np.abs(delta))
    # validity of the first-order bound, measured on the diagonally scaled
    # system the solver factors (invariant to the parameters' units)
    sc = 1.0 / dm
    kappa = float(np.max(((np.abs(Mi) * np.outer(1 / sc, 1 / sc)) @ (dM * np.outer(sc, sc))).sum(1)))
    return bound, kappa


def step_backward(A, g, lam, bA, bg, delta):
    """Componentwise backward error of a computed damped step: the residual
    |M delta - g| of the FP64 system and the part of it the FP32 errors
    allow, dg + dM |delta| (same dM, dg as step_bound)."""
    P = A.shape[0]
    d = marquardt_diag(A)
    M = A + lam * np.diag(d)
    dm = np.sqrt(np.abs(np.diag(M)))
    dM = bA + U32 * np.abs(A) + (3 * P + 6) * U32 * np.outer(dm, dm) + np.diag(lam * (np.diag(bA) + 2 * U32 * d))
    dg = bg + U32 * np.abs(g)
    return np.abs(M @ delta - g), dg + dM @ np.abs(delta)


def param_scale(theta):
    """Per-parameter scale of the parity bar: |a| for amplitudes, max(1, w)
    for centres, w for widths."""
    th = np.asarray(theta, dtype=np.float64).reshape(-1, 4)
    s = np.empty_like(th)
    s[:, 0] = np.abs(th[:, 0])
    s[:, 1] = np.maximum(1.0, th[:, 3])
    s[:, 2] = np.maximum(1.0, th[:, 3])
    s[:, 3] = th[:, 3]
    return s.ravel()


def optimum_floor(A, bg):
    """First-order distance between the FP64 optimum and a point where the
    GPU's FP32 gradient vanishes: |A^-1| bg (the FP32 error of g = J^T r
    moves the stationary point by A^-1 dg)."""
    return np.abs(np.linalg.pinv(A)) @ bg


def chi2_valley(A, bc):
    """Extent of the chi^2 valley at the FP32 chi^2 error: parameter i can
    move by sqrt(2 bc (A^-1)_ii) (the others re-optimised) before chi^2
    rises by 2 bc, the error of two FP32 chi^2 evaluations.  Marquardt's
    accept test compares two such values, so LM run in FP32 cannot tell
    points inside this valley apart and may stop anywhere in it.  bc is
    dominated by 2 u32 sum |r| (|T| + sum |g|): at high signal to noise
    the residual is a small difference of large FP32 numbers."""
    return np.sqrt(2.0 * bc * np.maximum(np.diag(np.linalg.pinv(A)), 0.0))
