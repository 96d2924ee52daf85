"""The FP32 error model of tests/fp32_bounds.py against an FP32 evaluation
of the same pixel pass (NumPy float32, on the CPU).

The GPU's parity tests accept its normal equations and chi^2 within the
bounds pass_bounds derives from the pass's operations.  Here those bounds
are checked against an independent FP32 evaluation of the pass, in the
GPU's order of operations: member frames rounded from FP64 (integer centre
plus fractional offset, exponent constant 0.5 log2(e) / w^2, 1 / w^2,
1 / w^3), per-pixel exp2 of the negated argument, the J row and residual in
FP32, sums of J^T J, J^T r and r^2 in FP32 leaves of at most 64 pixels
with compensated (Kahan) accumulation across leaves.  Every entry must lie
within its bound, and the bounds must not be loose by orders of magnitude
(a bound far above every error would pass any GPU result)."""
import math

import numpy as np
import pytest

import oracle as O
from tests.fp32_bounds import pass_bounds

F = np.float32
LOG2E = 1.4426950408889634


def _fp32_pass(T, xs, ys, theta):
    """FP32 J rows and residuals, then FP32-leaf / Kahan sums."""
    th = np.asarray(theta, dtype=np.float64).reshape(-1, 4)
    px = xs.astype(np.int64)
    py = ys.astype(np.int64)
    n, K = xs.size, th.shape[0]
    J = np.zeros((n, 4 * K), dtype=F)
    model = np.zeros(n, dtype=F)
    for k, (a, x, y, w) in enumerate(th):
        cx, cy = math.floor(x + 0.5), math.floor(y + 0.5)
        fx, fy = F(x - cx), F(y - cy)
        iw = 1.0 / w
        c, iw2, iw3 = F(0.5 * LOG2E * iw * iw), F(iw * iw), F(iw * iw * iw)
        dx = (px - cx).astype(F) - fx
        dy = (py - cy).astype(F) - fy
        q = dx * dx + dy * dy
        e = np.exp2(-(c * q)).astype(F)
        gk = F(a) * e
        J[:, 4 * k] = e
        J[:, 4 * k + 1] = gk * dx * iw2
        J[:, 4 * k + 2] = gk * dy * iw2
        J[:, 4 * k + 3] = gk * q * iw3
        model = model + gk
    r = T.astype(F) - model
    Jr = np.concatenate([J, r[:, None]], axis=1)
    P1 = Jr.shape[1]
    tot = np.zeros((P1, P1), dtype=F)
    comp = np.zeros((P1, P1), dtype=F)
    for s in range(0, n, 64):
        blk = Jr[s: s + 64]
        leaf = np.zeros((P1, P1), dtype=F)
        for row in blk:                                  # FP32 products summed in FP32
            leaf = leaf + np.outer(row, row).astype(F)
        y = leaf - comp                                  # Kahan across leaves
        t = tot + y
        comp = (t - tot) - y
        tot = t
    S = tot.astype(np.float64)
    return S[:-1, :-1], S[:-1, -1], float(S[-1, -1])


def _case(seed, K, n_side):
    rng = np.random.default_rng(seed)
    ys, xs = np.mgrid[0:n_side, 0:n_side].astype(np.float64)
    xs, ys = xs.ravel(), ys.ravel()
    truth = np.column_stack([rng.uniform(0.1, 1.0, K), rng.uniform(5, n_side - 5, K),
                             rng.uniform(5, n_side - 5, K), rng.uniform(1.2, 6.0, K)]).ravel()
    T = O.gauss_model(truth, xs, ys) + rng.normal(0, 1e-3, xs.size)
    T = T.astype(F).astype(np.float64)                   # the GPU's target is FP32
    theta = truth * np.tile([1.05, 1.0, 1.0, 0.95], K) + np.tile([0.0, 0.3, -0.2, 0.0], K)
    return T, xs, ys, theta


@pytest.mark.parametrize("seed,K,n_side", [(0, 1, 24), (1, 3, 32), (2, 6, 40), (3, 10, 48)])
def test_fp32_pass_within_its_error_bounds(seed, K, n_side):
    T, xs, ys, theta = _case(seed, K, n_side)
    b = pass_bounds(T, xs, ys, theta)
    A32, g32, c32 = _fp32_pass(T, xs, ys, theta)
    iu = np.triu_indices(A32.shape[0])
    errA, errg, errc = np.abs(A32 - b["A"])[iu], np.abs(g32 - b["g"]), abs(c32 - b["chi2"])
    assert np.all(errA <= b["bA"][iu]), np.max(errA / b["bA"][iu])
    assert np.all(errg <= b["bg"]), np.max(errg / b["bg"])
    assert errc <= b["bc"], errc / b["bc"]
    # not vacuous: the largest error reaches a visible fraction of its bound
    ratio = max(np.max(errA / b["bA"][iu]), np.max(errg / b["bg"]), errc / b["bc"])
    assert ratio > 1e-3, ratio


def test_bounds_catch_a_real_fp32_mistake():
    """The same FP32 pass evaluated at widths off by 2^-9 relative (about
    what an 8-bit mantissa would keep) must leave the bounds: they are tight
    enough to see an error that a correct FP32 evaluation does not make."""
    T, xs, ys, theta = _case(4, 3, 32)
    b = pass_bounds(T, xs, ys, theta)
    th = np.asarray(theta, float).reshape(-1, 4).copy()
    th[:, 3] *= 1.0 + 2.0 ** -9                          # a width off by 2^-9 relative
    A32, g32, c32 = _fp32_pass(T, xs, ys, th.ravel())
    iu = np.triu_indices(A32.shape[0])
    assert np.any(np.abs(A32 - b["A"])[iu] > b["bA"][iu]) or np.any(np.abs(g32 - b["g"]) > b["bg"])


def _fp32_damped_solve(A, g, lam):
    """The kernel's solve in FP32: FP32 copies of A and g, the scaled matrix
    S (A + lam D) S with S = diag(A + lam D)^-1/2 (unit diagonal), its FP32
    Cholesky factor and the two FP32 triangular solves, then delta = S x."""
    import scipy.linalg
    A32, g32 = A.astype(F), g.astype(F)
    d = np.diag(A32).copy()
    d[~(d > 0)] = F(1)
    M = A32 + F(lam) * np.diag(d).astype(F)
    s = (F(1) / np.sqrt(np.diag(M))).astype(F)
    Ms = (s[:, None] * M * s[None, :]).astype(F)
    L = scipy.linalg.cholesky(Ms, lower=True)
    assert L.dtype == F
    y = scipy.linalg.solve_triangular(L, (s * g32).astype(F), lower=True)
    x = scipy.linalg.solve_triangular(L.T, y, lower=False)
    assert x.dtype == F
    return (s * x).astype(np.float64)


@pytest.mark.parametrize("seed,K", [(5, 2), (6, 5), (7, 9)])
def test_fp32_damped_solve_within_the_step_bound(seed, K):
    from tests.fp32_bounds import marquardt_diag, step_backward, step_bound
    T, xs, ys, theta = _case(seed, K, 40)
    b = pass_bounds(T, xs, ys, theta)
    A32, g32, _ = _fp32_pass(T, xs, ys, theta)              # the FP32 sums the solve starts from
    for lam in (1e-6, 1e-3, 1.0):
        M = b["A"] + lam * np.diag(marquardt_diag(b["A"]))
        delta = np.linalg.solve(M, b["g"])
        got = _fp32_damped_solve(A32, g32, lam)
        bound, kappa = step_bound(b["A"], b["g"], lam, b["bA"], b["bg"], delta)
        if kappa < 0.5:                                      # the first-order bound is meaningful
            assert np.all(np.abs(got - delta) <= bound), np.max(np.abs(got - delta) / bound)
        resid, allowed = step_backward(b["A"], b["g"], lam, b["bA"], b["bg"], got)
        assert np.all(resid <= allowed), np.max(resid / allowed)


# ---------------------------------------------------------------- image passes

def _fp32_smooth(R, s):
    """Both separable passes in FP32, taps rounded from FP64 and applied in
    index order with fused multiply-adds rounded once each (the kernel's
    fmaf chain, emulated as an FP64 product and sum rounded to FP32)."""
    k = O.smoothing_kernel_1d(s).astype(F)
    m = (len(k) - 1) // 2

    def rows(X):
        Hh, Ww = X.shape
        pad = np.zeros((Hh, Ww + 2 * m), dtype=F)
        pad[:, m: m + Ww] = X
        out = np.zeros((Hh, Ww), dtype=F)
        for i in range(len(k)):
            out = (out.astype(np.float64) + np.float64(k[i]) * pad[:, i: i + Ww].astype(np.float64)).astype(F)
        return out

    return rows(rows(R.astype(F)).T).T.astype(np.float64)


@pytest.mark.parametrize("s", [2.0, 8.0, 32.0])
def test_fp32_smoothing_within_the_parity_tolerance(s):
    """The smoothing parity bar is 1e-5 relative L2 against the FP64 oracle;
    an FP32 evaluation of the two passes in the kernel's order lands
    within it by more than an order of magnitude, up to 257 taps."""
    import synth
    case = synth.small_case(256, 256, seed=5, n_gauss=2, sigma_range=(3, 8))
    ref = O.smooth_separable(case.dirty, s)
    got = _fp32_smooth(case.dirty, s)
    rel = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    assert rel < 1e-6, rel


def test_fp32_fft_update_within_the_parity_tolerance():
    """The FFT residual update in FP32 (the change image on the zero-padded
    2H x 2W grid, single-precision real transforms, the product with the
    PSF's single-precision transform, R -= conv / 4HW in FP32) against the
    oracle's direct subtraction: the change it makes is within 1e-6
    relative L2, an order inside the 1e-5 bar, for the update sizes and
    term widths of the teacher-forced tests."""
    import scipy.fft
    import synth
    H, W = 96, 104
    case = synth.small_case(H, W, seed=7)
    rng = np.random.default_rng(7)
    terms = []
    for w in (0.0, 0.3, 1.4, 4.7, 9.0, 2.2):
        t = O.component_terms(rng.normal(), rng.uniform(0, W - 1), rng.uniform(0, H - 1), w, w == 0.0, H, W)
        if t is not None:
            terms.append(t)
    R0 = case.dirty.astype(F).astype(np.float64)
    ref = O.subtract_terms(R0, case.psf, terms) - R0
    pad = np.zeros((2 * H, 2 * W), dtype=F)
    pad[:H, :W] = O.terms_to_image(terms, H, W).astype(F)
    bhat = scipy.fft.rfft2(case.psf.astype(F))
    conv = scipy.fft.irfft2(scipy.fft.rfft2(pad) * bhat, s=(2 * H, 2 * W))   # normalised by 1 / 4HW
    assert conv.dtype == F
    new = (R0.astype(F) - conv[H:, W:]).astype(np.float64)
    rel = float(np.linalg.norm((new - R0) - ref) / np.linalg.norm(ref))
    assert rel < 1e-6, rel
