"""Asp-Clean2016 minor cycle in plain FP64 NumPy -- TEST INFRASTRUCTURE ONLY.

Notation follows the paper (Zhang, Bhatnagar, Rau & Zhang 2016):

* residual image ``R`` (``I^residual``), PSF ``B`` with its single-Gaussian
  approximation ``(alpha_b, omega_b)`` (Sect. 3);
* a fitted (PSF-convolved) Gaussian ``g(p; a_ic, x_ic, y_ic, omega_ic)``
  (Eq. 6), deconvolved by Eq. 7 (width) and Eq. 8 (amplitude);
* the loop gain applied to a new component before it enters the model
  (Sect. 3, after Eq. 8).

Readings of points the paper leaves open are marked "Reading:" in the
docstrings; they are the ones the CUDA path implements as well.

Parity pins (tests/test_oracle_*.py): Eq. 7-8 against numerical 2-D
Gaussian convolution; the Jacobian against central finite differences; LM
against exact recovery of noiseless Gaussians and against MINPACK's
Levenberg-Marquardt (scipy.optimize.least_squares); subtraction and
smoothing against brute-force 2-D direct sums; the argmax against a
pure-Python scan.  Parity unpinned beyond invariants: the active-set
selection and retention rule, the init-mode switch and the fit-window size
(readings with no printed values to check against).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np
import scipy.linalg

__all__ = [
    "LMParams", "AspParams", "FitResult", "Component", "lm_exact",
    "LM_CONVERGED", "LM_CAP", "LM_STALLED", "MODE_SIMPLE", "MODE_SMOOTH",
    "round_half_up", "gauss_model", "model_and_jacobian", "normal_equations", "lm_fit",
    "cholesky_solve_damped", "psf_convolve", "model_jac_2004", "lm_fit_2004",
    "halfmax_width", "beam_fit", "peak_simple", "smoothing_scales", "smoothing_kernel_1d",
    "smooth_separable", "smooth_definition", "peak_smooth",
    "deconvolve", "gauss_approx", "component_terms", "terms_to_image",
    "subtract_terms", "subtract_definition", "beam_image_box", "subtract_beam_images",
    "member_box", "boxes_overlap", "MinorCycle", "mad_sigma",
]

SQRT_PI = math.sqrt(math.pi)

# LM status codes (shared meaning with the C-ABI's asp_fit_info.status)
LM_CONVERGED, LM_CAP, LM_STALLED = 0, 1, 2
# init modes
MODE_SIMPLE, MODE_SMOOTH = 0, 1


@dataclasses.dataclass
class LMParams:
    """Levenberg-Marquardt constants (Marquardt 1963; the paper gives none).

    Reading: Marquardt-scaled damping ``A + lambda diag(A)`` with lambda0 =
    1e-3, /10 on an accepted step (floor 1e-12), x10 on a rejected one, stop
    as "stalled" above 1e12; at most ``max_iter`` solves.  Convergence: the
    predicted decrease of a proposed step, or the actual relative decrease
    of an accepted one, is below ``rtol``; or an accepted step moves every
    parameter by less than ``xtol`` of its scale (|a| for amplitude, omega
    for centre and width).
    """

    lambda0: float = 1e-3
    lambda_up: float = 10.0
    lambda_down: float = 10.0
    lambda_min: float = 1e-12
    lambda_max: float = 1e12
    max_iter: int = 50
    rtol: float = 1e-7
    xtol: float = 1e-7


def lm_exact() -> LMParams:
    """Tight settings that drive the oracle to the optimum itself (used to
    compare converged fits independently of the iteration schedule)."""
    return LMParams(max_iter=500, rtol=1e-15, xtol=1e-13)


@dataclasses.dataclass
class AspParams:
    """Minor-cycle parameters (loop gain 0.35: Sect. 4; 5 % area switch:
    Sect. 3; stopping rule: Sect. 2 step 4)."""

    gain: float = 0.35
    k_max: int = 5
    noise_sigma: float = 0.0        # <= 0: estimate 1.4826 MAD of the dirty image
    stop_ksigma: float = 3.0
    n_scales: int = 6
    area_frac: float = 0.05
    init_mode: str = "auto"          # auto | simple | smooth
    tau: float = 1e-3                # active-set retention threshold
    retained_cap_factor: int = 8     # retained list capped at factor * k_max
    major_every: int = 0             # 0: full-PSF subtraction every iteration; n: minor/major split
    lm: LMParams = dataclasses.field(default_factory=LMParams)


@dataclasses.dataclass
class FitResult:
    theta: np.ndarray
    chi2_init: float
    chi2: float
    iters: int
    passes: int
    lam: float
    status: int
    pixel_evals: int
    # the last proposed point theta + delta (None if no solve succeeded) and
    # chi^2 of the last pixel pass (at that point when it was evaluated)
    trial: Optional[np.ndarray] = None
    chi2_trial: float = float("nan")


@dataclasses.dataclass
class Component:
    """A deconvolved model component (Eq. 2 term): flux F, amplitude alpha,
    centre, width omega_i (0 for a point)."""

    flux: float
    amp: float
    x: float
    y: float
    width: float
    is_point: bool


def round_half_up(v):
    """Nearest integer, halves rounded up (floor(v + 0.5))."""
    return np.floor(np.asarray(v, dtype=np.float64) + 0.5).astype(np.int64)


# --------------------------------------------------------------------------
# Eq. 6: the fitted Gaussian and its analytic Jacobian

def gauss_model(theta, xs, ys):
    """Sum over members of ``a exp(-((x-x0)^2 + (y-y0)^2) / (2 omega^2))``
    (the model of Sect. 2 step 2, one term per active-set member), with
    ``theta = [a_0, x_0, y_0, omega_0, a_1, ...]``."""
    theta = np.asarray(theta, dtype=np.float64)
    out = np.zeros(np.broadcast(xs, ys).shape)
    for k in range(len(theta) // 4):
        a, x0, y0, w = theta[4 * k: 4 * k + 4]
        out += a * np.exp(-((xs - x0) ** 2 + (ys - y0) ** 2) / (2.0 * w * w))
    return out


def model_and_jacobian(theta, xs, ys):
    """Model and its Jacobian with respect to ``theta`` (columns a, x, y,
    omega per member): d/da = E, d/dx0 = g dx / omega^2, d/dy0 = g dy /
    omega^2, d/domega = g r^2 / omega^3, with E the unit-amplitude
    Gaussian and g = a E."""
    theta = np.asarray(theta, dtype=np.float64)
    K = len(theta) // 4
    xs = np.asarray(xs, dtype=np.float64).ravel()
    ys = np.asarray(ys, dtype=np.float64).ravel()
    n = xs.size
    J = np.empty((n, 4 * K))
    model = np.zeros(n)
    for k in range(K):
        a, x0, y0, w = theta[4 * k: 4 * k + 4]
        dx = xs - x0
        dy = ys - y0
        r2 = dx * dx + dy * dy
        e = np.exp(-r2 / (2.0 * w * w))
        g = a * e
        J[:, 4 * k] = e
        J[:, 4 * k + 1] = g * dx / (w * w)
        J[:, 4 * k + 2] = g * dy / (w * w)
        J[:, 4 * k + 3] = g * r2 / (w * w * w)
        model += g
    return model, J


def normal_equations(T, xs, ys, theta):
    """The LM pixel pass: ``A = J^T J``, ``g = J^T r``, ``chi2 = r^T r`` with
    ``r = T - model`` over the given pixels (Eq. 6 objective)."""
    model, J = model_and_jacobian(theta, xs, ys)
    r = np.asarray(T, dtype=np.float64).ravel() - model
    return J.T @ J, J.T @ r, float(r @ r)


def cholesky_solve_damped(A, g, lam):
    """Solve ``(A + lam diag(d)) delta = g`` by Cholesky, ``d_i = A_ii`` (1
    where A_ii is 0, i.e. a parameter the data does not constrain).
    Returns None when the matrix is not positive definite."""
    d = np.diag(A).copy()
    d[~(d > 0)] = 1.0
    M = A + lam * np.diag(d)
    try:
        c = scipy.linalg.cho_factor(M, lower=True, check_finite=True)
    except (np.linalg.LinAlgError, ValueError):
        return None
    delta = scipy.linalg.cho_solve(c, g)
    if not np.all(np.isfinite(delta)):
        return None
    return delta


def _valid(theta, box, omega_min):
    """Reading (the fit is local, Sect. 2): a trial point is usable when every
    value is finite, every centre lies in the window and every width is in
    (omega_min, window extent]; a Gaussian wider than its window is not
    constrained by the data (it degenerates into a pedestal of unbounded
    flux)."""
    if not np.all(np.isfinite(theta)):
        return False
    x0b, x1b, y0b, y1b = box
    omega_max = max(x1b - x0b + 1, y1b - y0b + 1)
    for k in range(len(theta) // 4):
        _, x, y, w = theta[4 * k: 4 * k + 4]
        if not (w > omega_min) or w > omega_max:
            return False
        if x < x0b or x > x1b or y < y0b or y > y1b:
            return False
    return True


def _step_scale(theta):
    """Per-parameter scale of the xtol test: |a| (1 where a = 0) for the
    amplitude, omega for centre and width."""
    scale = np.empty_like(theta)
    scale[0::4] = np.abs(theta[0::4])
    scale[0::4][scale[0::4] == 0] = 1.0
    scale[1::4] = theta[3::4]
    scale[2::4] = theta[3::4]
    scale[3::4] = theta[3::4]
    return scale


def lm_fit(T, xs, ys, theta0, box, omega_min, lm: Optional[LMParams] = None, model_jac=None, valid=None,
           step_scale=None) -> FitResult:
    """Levenberg-Marquardt minimisation of the Eq. 6 objective.

    ``T`` are the target values at pixel coordinates ``(xs, ys)``; ``box =
    (x0, x1, y0, y1)`` the window (a trial centre outside it, a width
    ``<= omega_min`` or a non-finite value is rejected like a step that
    raised chi^2).  Steps (Marquardt 1963):

    1. evaluate A, g, chi^2 at the current point;
    2. solve the damped normal equations (one iteration per solve);
    3. stop as converged if the predicted decrease ``2 d.g - d.A.d`` (=
       ``d.g + lambda d.D.d`` for the damped step) is below ``rtol * chi^2``;
    4. evaluate chi^2 (with A, g) at the trial point; accept iff chi^2
       strictly decreases (lambda /= 10), else lambda *= 10;
    5. on an accepted step stop if the relative decrease is below rtol or
       every |delta_i| is below xtol of its scale; on a reject stop if
       lambda exceeds lambda_max; stop after max_iter solves.

    ``model_jac(theta) -> (model, J)`` replaces the Eq. 6 model and Jacobian
    (e.g. the Eq. 3 objective of :func:`model_jac_2004`); xs and ys then
    only size the data.  ``valid(theta) -> bool`` and ``step_scale(theta)
    -> scales`` replace the trial-point test and the xtol scales of the
    four-parameter members (the elliptical members of
    ``oracle.elliptical``).
    """
    lm = lm or LMParams()
    T = np.asarray(T, dtype=np.float64).ravel()
    xs = np.asarray(xs, dtype=np.float64).ravel()
    ys = np.asarray(ys, dtype=np.float64).ravel()
    theta = np.array(theta0, dtype=np.float64)
    n = T.size
    if model_jac is None:
        ne = lambda th: normal_equations(T, xs, ys, th)   # noqa: E731
    else:
        def ne(th):
            m, J = model_jac(th)
            r = T - m
            return J.T @ J, J.T @ r, float(r @ r)
    A, g, chi2 = ne(theta)
    chi2_init = chi2
    passes, iters, lam = 1, 0, lm.lambda0
    status = LM_CAP
    last_trial, last_pass_chi2 = None, chi2
    while True:
        if iters >= lm.max_iter:
            status = LM_CAP
            break
        delta = cholesky_solve_damped(A, g, lam)
        iters += 1
        if delta is None:
            lam *= lm.lambda_up
            if lam > lm.lambda_max:
                status = LM_STALLED
                break
            continue
        last_trial = theta + delta
        # predicted decrease 2 d.g - d.A.d of the linearised model; by the
        # damped normal equations (A + lam D) d = g it equals d.g + lam d.D.d
        dd = np.diag(A).copy()
        dd[~(dd > 0)] = 1.0
        pred = float(delta @ g) + lam * float(delta @ (dd * delta))
        if pred <= lm.rtol * chi2:
            status = LM_CONVERGED
            break
        trial = last_trial
        if not (_valid(trial, box, omega_min) if valid is None else valid(trial)):
            lam *= lm.lambda_up
            if lam > lm.lambda_max:
                status = LM_STALLED
                break
            continue
        A2, g2, chi2_t = ne(trial)
        passes += 1
        last_pass_chi2 = chi2_t
        if chi2_t < chi2:
            rel = (chi2 - chi2_t) / chi2 if chi2 > 0 else 0.0
            scale = _step_scale(theta) if step_scale is None else step_scale(theta)
            small = float(np.max(np.abs(delta) / scale)) < lm.xtol
            theta, A, g, chi2 = trial, A2, g2, chi2_t
            lam = max(lam / lm.lambda_down, lm.lambda_min)
            if rel < lm.rtol or small:
                status = LM_CONVERGED
                break
        else:
            lam *= lm.lambda_up
            if lam > lm.lambda_max:
                status = LM_STALLED
                break
    return FitResult(theta, chi2_init, chi2, iters, passes, lam, status, passes * n, last_trial, last_pass_chi2)


# --------------------------------------------------------------------------
# Asp-Clean2004's objective (Sect. 2, Eq. 3): the full PSF inside chi^2

def psf_convolve(B, img):
    """``(B * img)(p) = sum_q B(p - q + (H, W)) img(q)`` for H x W images
    with the 2H x 2W PSF (zero lag at [H, W]), as an FP64 FFT product on
    the 2H x 2W grid (no wrap-around: p - q + H lies in [1, 2H - 1])."""
    B = np.asarray(B, dtype=np.float64)
    img = np.asarray(img, dtype=np.float64)
    H, W = img.shape
    pad = np.zeros((2 * H, 2 * W))
    pad[:H, :W] = img
    out = np.fft.irfft2(np.fft.rfft2(pad) * np.fft.rfft2(B), s=(2 * H, 2 * W))
    return out[H: 2 * H, W: 2 * W]


def model_jac_2004(B, theta, H, W):
    """The Eq. 3 model B * sum_k g_k over the whole image and its
    Jacobian: g_k the *unconvolved* component a exp(-r^2 / 2 omega^2)
    sampled at the pixel centres; each column is the PSF convolution of the
    component's derivative image (Sect. 2: one FFT convolution per
    evaluation).  Returns (model (N,), J (N, 4K))."""
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    m, Jimg = model_and_jacobian(theta, xs.ravel(), ys.ravel())
    model = psf_convolve(B, m.reshape(H, W)).ravel()
    J = np.stack([psf_convolve(B, Jimg[:, j].reshape(H, W)).ravel() for j in range(Jimg.shape[1])], 1)
    return model, J


def lm_fit_2004(T_img, B, theta0, omega_min, lm: Optional[LMParams] = None) -> FitResult:
    """Levenberg-Marquardt on the Eq. 3 objective chi^2 = || T - B * sum_k
    g_k ||^2 over the whole image (T: the residual with the fitted members'
    previous contributions added back through B), with the same LM rules
    as :func:`lm_fit`; trial centres must stay in the image."""
    T_img = np.asarray(T_img, dtype=np.float64)
    H, W = T_img.shape
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    return lm_fit(T_img.ravel(), xs.ravel(), ys.ravel(), theta0, (0, W - 1, 0, H - 1), omega_min, lm,
                  model_jac=lambda th: model_jac_2004(B, th, H, W))


# --------------------------------------------------------------------------
# Beam: the PSF approximated as a single Gaussian (Sect. 3, Eqs. 7-8)

def halfmax_width(B):
    """Initial beam width from the PSF's half-maximum crossings.

    Reading (the paper says only that the PSF is approximated by a single
    Gaussian): the zero-lag value ``B[H, W]`` is the peak; along the four
    axis directions the first sample below half of it is found and the
    crossing radius is linearly interpolated; the mean radius divided by
    ``sqrt(2 ln 2)`` is the Gaussian sigma."""
    B = np.asarray(B, dtype=np.float64)
    H, W = B.shape[0] // 2, B.shape[1] // 2
    peak = B[H, W]
    half = 0.5 * peak
    radii = []
    for dy, dx in ((0, 1), (0, -1), (1, 0), (-1, 0)):
        prev = peak
        rad = float(min(H, W) - 1)
        for s in range(1, min(H, W)):
            v = B[H + dy * s, W + dx * s]
            if v < half:
                rad = (s - 1) + (prev - half) / (prev - v)
                break
            prev = v
        radii.append(rad)
    return (sum(radii) / 4.0) / math.sqrt(2.0 * math.log(2.0))


def beam_fit(B, lm: Optional[LMParams] = None):
    """Fit ``(alpha_b, omega_b)`` to the PSF main lobe (Sect. 3).

    Reading: an Eq.-6 LM fit of one circular Gaussian (amplitude, centre,
    width free) to the pixels within radius ``ceil(3 omega_init)`` of the
    zero lag, started from ``(B[H, W], W, H, omega_init)`` with omega_init
    from :func:`halfmax_width`; trial widths must stay above ``0.25
    omega_init``.  Returns ``(alpha_b, omega_b, fit)``."""
    B = np.asarray(B, dtype=np.float64)
    H, W = B.shape[0] // 2, B.shape[1] // 2
    w0 = halfmax_width(B)
    r = int(math.ceil(3.0 * w0))
    ys, xs = np.mgrid[H - r: H + r + 1, W - r: W + r + 1]
    inside = (xs - W) ** 2 + (ys - H) ** 2 <= r * r
    xs = xs[inside].astype(np.float64)
    ys = ys[inside].astype(np.float64)
    T = B[ys.astype(np.int64), xs.astype(np.int64)]
    theta0 = np.array([B[H, W], float(W), float(H), w0])
    fit = lm_fit(T, xs, ys, theta0, (W - r, W + r, H - r, H + r), 0.25 * w0, lm)
    return float(fit.theta[0]), float(fit.theta[3]), fit


# --------------------------------------------------------------------------
# Initial values (Sect. 2 step 1; Sect. 3 "simple method")

def peak_simple(R):
    """``argmax_p |R(p)|``, lowest row-major index on ties.  Returns
    ``(index, R[index])``."""
    flat = np.asarray(R).ravel()
    idx = int(np.argmax(np.abs(flat)))
    return idx, float(flat[idx])


def smoothing_scales(omega_b, n_scales, H, W):
    """Reading: s_j = omega_b 2^j, j = 0..n_scales-1, keeping s_j <= min(H,
    W)/8 (j = 0 always kept)."""
    out = []
    for j in range(n_scales):
        s = omega_b * (2.0 ** j)
        if j == 0 or s <= min(H, W) / 8.0:
            out.append(s)
    return out


def smoothing_kernel_1d(s):
    """1-D factor of the unit-L2 Gaussian smoothing kernel: exp(-u^2/2s^2)
    for |u| <= ceil(4s), divided by sqrt(sum of squares) so the separable
    2-D kernel has unit L2 norm (reading: a matched filter, whose response
    to a Gaussian of width omega peaks at s = omega)."""
    m = int(math.ceil(4.0 * s))
    u = np.arange(-m, m + 1, dtype=np.float64)
    e = np.exp(-u * u / (2.0 * s * s))
    return e / math.sqrt(float(e @ e))


def _correlate_rows(X, k):
    """out[y, x] = sum_u k[u] X[y, x + u - m], zero outside (k odd length)."""
    m = (len(k) - 1) // 2
    Hh, Ww = X.shape
    pad = np.zeros((Hh, Ww + 2 * m))
    pad[:, m: m + Ww] = X
    out = np.zeros((Hh, Ww))
    for i in range(len(k)):
        out += k[i] * pad[:, i: i + Ww]
    return out


def smooth_separable(R, s):
    """``S = R * k_s`` with the unit-L2 kernel, zero-padded edges, as a row
    pass then a column pass (the kernel is separable and symmetric)."""
    k = smoothing_kernel_1d(s)
    S1 = _correlate_rows(np.asarray(R, dtype=np.float64), k)
    return _correlate_rows(S1.T, k).T


def smooth_definition(R, s):
    """Brute-force 2-D direct form of :func:`smooth_separable`:
    ``S(p) = sum_q k(q) R(p + q)`` over the full square support."""
    R = np.asarray(R, dtype=np.float64)
    k1 = smoothing_kernel_1d(s)
    m = (len(k1) - 1) // 2
    Hh, Ww = R.shape
    pad = np.zeros((Hh + 2 * m, Ww + 2 * m))
    pad[m: m + Hh, m: m + Ww] = R
    out = np.zeros((Hh, Ww))
    for qy in range(-m, m + 1):
        for qx in range(-m, m + 1):
            out += k1[qy + m] * k1[qx + m] * pad[m + qy: m + qy + Hh, m + qx: m + qx + Ww]
    return out


def peak_smooth(R, omega_b, n_scales):
    """Multi-scale smoothing init (Sect. 2 step 1, Sect. 3): the global peak of
    |S_j| over all scales and pixels (ties: lower j, then lower index).

    Returns ``dict(scale_index, s, index, value, a0, x0, y0, w0)`` with
    ``w0 = max(s_j, omega_b)`` and ``a0 = S_j(p*) / (sqrt(pi) s_j)`` (the
    amplitude of a Gaussian of width s_j whose unit-L2 matched-filter
    response is S_j(p*))."""
    R = np.asarray(R, dtype=np.float64)
    Hh, Ww = R.shape
    best = None
    for j, s in enumerate(smoothing_scales(omega_b, n_scales, Hh, Ww)):
        S = smooth_separable(R, s)
        idx = int(np.argmax(np.abs(S).ravel()))
        v = float(S.ravel()[idx])
        if best is None or abs(v) > abs(best[3]):
            best = (j, s, idx, v)
    j, s, idx, v = best
    return dict(scale_index=j, s=s, index=idx, value=v, a0=v / (SQRT_PI * s),
                x0=float(idx % Ww), y0=float(idx // Ww), w0=max(s, omega_b))


# --------------------------------------------------------------------------
# Eqs. 7-8: analytic deconvolution of the fitted Gaussian

def deconvolve(a_ic, w_ic, alpha_b, omega_b):
    """Eq. 7 (``omega_i = sqrt(omega_ic^2 - omega_b^2)``) and Eq. 8
    (``alpha_i = alpha_ic omega_ic^2 / (2 pi alpha_b omega_b^2 omega_i^2)``).

    Written through the flux ``F = 2 pi alpha_i omega_i^2 = alpha_ic
    omega_ic^2 / (alpha_b omega_b^2)`` (Eq. 8 times 2 pi omega_i^2), which
    stays finite as omega_i -> 0.  Reading (Eq. 7 is imaginary for
    omega_ic <= omega_b): if ``omega_ic^2 <= omega_b^2 (1 + 1e-3)`` the
    component is a point of flux F.  Returns ``(F, alpha_i, omega_i,
    is_point)`` (alpha_i = F for a point)."""
    F = a_ic * w_ic * w_ic / (alpha_b * omega_b * omega_b)
    if w_ic * w_ic > omega_b * omega_b * (1.0 + 1e-3):
        wi = math.sqrt(w_ic * w_ic - omega_b * omega_b)
        return F, F / (2.0 * math.pi * wi * wi), wi, False
    return F, F, 0.0, True


def gauss_approx(F, w_i, alpha_b, omega_b):
    """The single-Gaussian-beam image of a component (inverse of Eqs. 7-8):
    ``(a_ic, omega_ic)`` with ``omega_ic^2 = omega_i^2 + omega_b^2`` and
    ``a_ic = alpha_b omega_b^2 F / omega_ic^2``."""
    w_ic = math.sqrt(w_i * w_i + omega_b * omega_b)
    return alpha_b * omega_b * omega_b * F / (w_ic * w_ic), w_ic


# --------------------------------------------------------------------------
# Component images and subtraction (Sect. 2 step 3, with the full PSF B)

def component_terms(F, x, y, w, is_point, H, W):
    """A component sampled on the image grid as one separable term
    ``(qx0, wx, qy0, wy, F)``: image value ``F wx[i] wy[j]`` at ``(qx0 + i,
    qy0 + j)``.

    Reading: extended (omega_i >= 0.5 px) -> the sampled Gaussian on the box
    ``|q - centre|_inf <= ceil(5 omega_i) + 1``, each axis factor normalised
    to unit sum over the whole box so the component's discrete flux is F;
    otherwise a bilinear deposit of F on the 4 pixels around the centre.
    Pixels outside the image are dropped (no renormalisation).  Returns None
    when nothing falls inside the image."""
    if is_point or w < 0.5:
        fx0, fy0 = math.floor(x), math.floor(y)
        fx, fy = x - fx0, y - fy0
        cols = np.array([fx0, fx0 + 1], dtype=np.int64)
        rows = np.array([fy0, fy0 + 1], dtype=np.int64)
        wx = np.array([1.0 - fx, fx])
        wy = np.array([1.0 - fy, fy])
    else:
        h = math.ceil(5.0 * w) + 1
        cols = np.arange(math.ceil(x - h), math.floor(x + h) + 1, dtype=np.int64)
        rows = np.arange(math.ceil(y - h), math.floor(y + h) + 1, dtype=np.int64)
        wx = np.exp(-((cols - x) ** 2) / (2.0 * w * w))
        wy = np.exp(-((rows - y) ** 2) / (2.0 * w * w))
        wx = wx / wx.sum()
        wy = wy / wy.sum()
    kx = (cols >= 0) & (cols < W)
    ky = (rows >= 0) & (rows < H)
    if not kx.any() or not ky.any():
        return None
    return (int(cols[kx][0]), wx[kx], int(rows[ky][0]), wy[ky], float(F))


def terms_to_image(terms, H, W):
    """Sum of separable terms as a dense H x W image (for definition mode)."""
    img = np.zeros((H, W))
    for qx0, wx, qy0, wy, s in terms:
        img[qy0: qy0 + len(wy), qx0: qx0 + len(wx)] += s * np.outer(wy, wx)
    return img


def subtract_terms(R, B, terms):
    """``R(p) -= sum_t s_t sum_j wy_t[j] sum_i wx_t[i] B(p - q_ij + (H, W))``
    with the full PSF (no truncation), term by term as a horizontal pass
    over B's rows followed by a vertical pass.  Returns the new image."""
    R = np.array(R, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    H, W = R.shape
    for qx0, wx, qy0, wy, s in terms:
        ny = len(wy)
        # rows of B needed: py - qy + H for py in [0,H), qy in [qy0, qy0+ny)
        r0 = H - qy0 - ny + 1
        nrows = H + ny - 1
        T1 = np.zeros((nrows, W))
        for i in range(len(wx)):
            c0 = W - qx0 - i
            T1 += wx[i] * B[r0: r0 + nrows, c0: c0 + W]
        out = np.zeros((H, W))
        for j in range(ny):
            # B row for (py, qy0 + j) is py - qy0 - j + H = r0 + (py + ny - 1 - j)
            out += wy[j] * T1[ny - 1 - j: ny - 1 - j + H, :]
        R -= s * out
    return R


def beam_image_box(x, y, w, alpha_b, omega_b, H, W):
    """Reading of the minor cycle's approximate subtraction (the Clark-style
    split): a component of flux 1 and width w through the single-Gaussian
    beam is the Gaussian (a_ic, w_ic) of :func:`gauss_approx`, evaluated on
    the box |q - centre|_inf <= ceil(5 w_ic) + 1 (clipped to the image).
    Returns (qx0, qy0, image) or None."""
    a_ic, w_ic = gauss_approx(1.0, w, alpha_b, omega_b)
    h = math.ceil(5.0 * w_ic) + 1
    x0, x1 = max(math.ceil(x - h), 0), min(math.floor(x + h), W - 1)
    y0, y1 = max(math.ceil(y - h), 0), min(math.floor(y + h), H - 1)
    if x0 > x1 or y0 > y1:
        return None
    ys, xs = np.mgrid[y0: y1 + 1, x0: x1 + 1].astype(np.float64)
    return x0, y0, a_ic * np.exp(-((xs - x) ** 2 + (ys - y) ** 2) / (2.0 * w_ic * w_ic))


def subtract_beam_images(R, items, alpha_b, omega_b):
    """``R -= sum_i F_i * beam image of component i`` for items (F, x, y,
    w): the minor cycle's update with the PSF approximated by its fitted
    Gaussian.  Returns the new image."""
    R = np.array(R, dtype=np.float64)
    H, W = R.shape
    for F, x, y, w in items:
        b = beam_image_box(x, y, w, alpha_b, omega_b, H, W)
        if b is None:
            continue
        x0, y0, img = b
        R[y0: y0 + img.shape[0], x0: x0 + img.shape[1]] -= F * img
    return R


def subtract_definition(R, B, dC):
    """Brute-force 2-D direct form: ``R(p) -= sum_q dC(q) B(p - q + (H, W))``
    over every nonzero model pixel q and every image pixel p."""
    R = np.array(R, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    H, W = R.shape
    for qy, qx in zip(*np.nonzero(dC)):
        R -= dC[qy, qx] * B[H - qy: 2 * H - qy, W - qx: 2 * W - qx]
    return R


# --------------------------------------------------------------------------
# Active set and fit window (Sect. 1: heuristics limit the set of scales
# fitted in an iteration; Sect. 2 step 2 fits the data locally)

def member_box(x, y, w):
    """Reading: the fit window of one member is the square of half-width
    ``h = max(5, ceil(4 omega))`` around its rounded centre.  Returns
    ``(x0, x1, y0, y1)`` (inclusive, unclipped)."""
    h = max(5, int(math.ceil(4.0 * w)))
    rx, ry = int(round_half_up(x)), int(round_half_up(y))
    return (rx - h, rx + h, ry - h, ry + h)


def boxes_overlap(a, b):
    return a[0] <= b[1] and b[0] <= a[1] and a[2] <= b[3] and b[2] <= a[3]


def mad_sigma(img):
    """1.4826 x median absolute deviation (noise estimate when none is given)."""
    v = np.asarray(img, dtype=np.float64).ravel()
    med = np.median(v)
    return 1.4826 * float(np.median(np.abs(v - med)))


class MinorCycle:
    """The Asp-Clean2016 minor cycle (Sect. 2 steps 1-4 with the Sect. 3
    objective, deconvolution and initial-value switch).

    State: residual R (FP64), PSF B, beam (alpha_b, omega_b), the component
    list, the retained (active) list, the iteration counter and the last
    iteration's (omega_i, omega_0) for the switch heuristic.

    Per iteration (reading of the loop for the joint active-set fit):

    1. peak of |R|; stop if it is below ``stop_ksigma * noise_sigma``;
    2. init mode: SIMPLE iff t > 0 and ``omega_i(t-1)^2 < area_frac *
       omega_0(t-1)^2`` (area of the optimal component vs area of the initial
       guess, both from the last iteration), else SMOOTH;
    3. initial values (a0, x0, y0, omega0) by that mode;
    4. active set: the new member plus retained members (most recent first)
       whose boxes overlap the new member's box and whose centres are not
       co-located with the new one, at most k_max in total;
       the joint window is the bounding box of their boxes clipped to the
       image; the target is ``T = R + sum_old g(G_k)`` over the window, with
       G_k the single-Gaussian image of old member k;
    5. LM fit of all members jointly (Eq. 6);
    6. deconvolution (Eqs. 7-8); the new component's flux is multiplied by the
       loop gain; old members are replaced by their refit values;
    7. ``R -= B * dC`` with dC = gain c_new + sum_old (c'_k - c_k);
    8. retention: an old member stays retained iff its fit moved some
       parameter by more than tau (relative: |da|/|a|, |dx|/omega,
       |dy|/omega, |domega|/omega); the new member is always retained; the
       list is capped at retained_cap_factor * k_max (oldest dropped).
    """

    def __init__(self, dirty, psf, params: AspParams, beam=None, mlp=None):
        self.mlp = mlp   # learned initial values (mlp_oracle.MLPWeights) or None
        self.R = np.array(dirty, dtype=np.float64)
        self.B = np.asarray(psf, dtype=np.float64)
        self.H, self.W = self.R.shape
        assert self.B.shape == (2 * self.H, 2 * self.W)
        self.p = params
        if beam is None:
            ab, wb, _ = beam_fit(self.B)
        else:
            ab, wb = beam
        self.alpha_b, self.omega_b = float(ab), float(wb)
        self.noise = params.noise_sigma if params.noise_sigma > 0 else mad_sigma(self.R)
        self.D = self.R.copy()          # the dirty image (the major cycle's start)
        self.since_major = 0
        self.comps: list[Component] = []
        self.retained: list[int] = []
        self.t = 0
        self.last_wi = 0.0
        self.last_w0 = 0.0
        self.stopped = False
        self.history: list[dict] = []

    # -- helpers
    def G(self, k):
        c = self.comps[k]
        a, w = gauss_approx(c.flux, c.width, self.alpha_b, self.omega_b)
        return np.array([a, c.x, c.y, w])

    def _component_from_fit(self, a, x, y, w, gain=1.0):
        F, amp, wi, pt = deconvolve(a, w, self.alpha_b, self.omega_b)
        F *= gain
        amp *= gain
        return Component(F, amp, float(x), float(y), wi, pt)

    def choose_mode(self):
        m = self.p.init_mode
        if m == "simple":
            return MODE_SIMPLE
        if m == "smooth":
            return MODE_SMOOTH
        if self.t > 0 and self.last_wi ** 2 < self.p.area_frac * self.last_w0 ** 2:
            return MODE_SIMPLE
        return MODE_SMOOTH

    def initial_values(self, mode):
        if mode == MODE_SIMPLE:
            idx, v = peak_simple(self.R)
            return dict(a0=v, x0=float(idx % self.W), y0=float(idx // self.W), w0=self.omega_b,
                        index=idx, scale_index=-1)
        return peak_smooth(self.R, self.omega_b, self.p.n_scales)

    def select(self, init):
        """Active set: retained members (most recent first) whose boxes overlap
        the new member's box and whose centres are not co-located with it
        (squared distance > max(omega0, omega_ic,k)^2; co-located members
        leave only the sum of their amplitudes determined), at most
        k_max - 1 of them."""
        new_box = member_box(init["x0"], init["y0"], init["w0"])
        chosen = []
        for k in self.retained:
            if len(chosen) >= self.p.k_max - 1:
                break
            G = self.G(k)
            if boxes_overlap(member_box(G[1], G[2], G[3]), new_box):
                dx, dy = G[1] - init["x0"], G[2] - init["y0"]
                m = max(init["w0"], G[3])
                if dx * dx + dy * dy > m * m:
                    chosen.append(k)
        boxes = [new_box] + [member_box(*self.G(k)[1:4]) for k in chosen]
        x0 = max(0, min(b[0] for b in boxes))
        x1 = min(self.W - 1, max(b[1] for b in boxes))
        y0 = max(0, min(b[2] for b in boxes))
        y1 = min(self.H - 1, max(b[3] for b in boxes))
        return chosen, (x0, x1, y0, y1)

    # -- one iteration
    def prepare(self):
        """Steps 1-4 of an iteration without changing the state: the stopping
        test, the init mode, the initial values, the active set, the window
        and the fit's target T and start theta0.  None when the noise
        threshold stops the cycle."""
        pidx, pval = peak_simple(self.R)
        if abs(pval) < self.p.stop_ksigma * self.noise:
            return None
        mode = self.choose_mode()
        init = self.initial_values(mode)
        chosen, win = self.select(init)
        x0, x1, y0, y1 = win
        ys, xs = np.mgrid[y0: y1 + 1, x0: x1 + 1]
        xs = xs.astype(np.float64).ravel()
        ys = ys.astype(np.float64).ravel()
        T = self.R[y0: y1 + 1, x0: x1 + 1].ravel().copy()
        theta0 = [init["a0"], init["x0"], init["y0"], init["w0"]]
        for k in chosen:
            G = self.G(k)
            T += gauss_model(G, xs, ys)
            theta0 += list(G)
        return dict(peak_index=pidx, peak_value=pval, mode=mode, init=init, chosen=chosen, window=win,
                    xs=xs, ys=ys, T=T, theta0=np.array(theta0))

    def step(self):
        if self.stopped:
            return None
        prep = self.prepare()
        if prep is None:
            self.stopped = True
            return None
        pidx, pval, mode, init = prep["peak_index"], prep["peak_value"], prep["mode"], prep["init"]
        chosen, win, xs, ys, T, theta0 = (prep[k] for k in ("chosen", "window", "xs", "ys", "T", "theta0"))
        learned = None
        if self.mlp is not None:
            fit, learned = self._learned_fit(T, xs, ys, theta0, win, init)
        else:
            fit = lm_fit(T, xs, ys, theta0, win, 0.25 * self.omega_b, self.p.lm)
        th = fit.theta
        terms = []
        new = self._component_from_fit(*th[0:4], gain=self.p.gain)
        self.comps.append(new)
        new_index = len(self.comps) - 1
        t = component_terms(new.flux, new.x, new.y, new.width, new.is_point, self.H, self.W)
        if t is not None:
            terms.append(t)
        still = []
        old_comps = {}
        for m, k in enumerate(chosen, start=1):
            old = self.comps[k]
            old_comps[m] = old
            G0 = theta0[4 * m: 4 * m + 4]
            a, x, y, w = th[4 * m: 4 * m + 4]
            tau = self.p.tau
            moved = (abs(a - G0[0]) > tau * abs(G0[0]) or abs(x - G0[1]) > tau * G0[3]
                     or abs(y - G0[2]) > tau * G0[3] or abs(w - G0[3]) > tau * G0[3])
            nc = self._component_from_fit(a, x, y, w)
            t_new = component_terms(nc.flux, nc.x, nc.y, nc.width, nc.is_point, self.H, self.W)
            t_old = component_terms(old.flux, old.x, old.y, old.width, old.is_point, self.H, self.W)
            if t_new is not None:
                terms.append(t_new)
            if t_old is not None:
                terms.append(t_old[:4] + (-t_old[4],))
            self.comps[k] = nc
            if moved:
                still.append(k)
        dropped = set(chosen) - set(still)
        self.retained = [new_index] + [k for k in self.retained if k not in dropped]
        cap = self.p.retained_cap_factor * self.p.k_max
        self.retained = self.retained[:cap]
        if self.p.major_every > 0:
            # minor/major split: each term's single-Gaussian-beam image
            items = [(new.flux, new.x, new.y, new.width)]
            for m, k in enumerate(chosen, start=1):
                nc = self.comps[k]
                items.append((nc.flux, nc.x, nc.y, nc.width))
                items.append((-old_comps[m].flux, old_comps[m].x, old_comps[m].y, old_comps[m].width))
            self.R = subtract_beam_images(self.R, items, self.alpha_b, self.omega_b)
            self.since_major += 1
        else:
            self.R = subtract_terms(self.R, self.B, terms)
        self.last_wi = new.width
        self.last_w0 = init["w0"]
        rec = dict(t=self.t, mode=mode, peak_index=pidx, peak_value=pval, init=init,
                   members=[new_index] + chosen, window=win, fit=fit, n_terms=len(terms), learned=learned,
                   T=T, xs=xs, ys=ys, theta0=theta0)
        self.history.append(rec)
        self.t += 1
        return rec

    def _learned_fit(self, T, xs, ys, theta0, win, init):
        """Learned initial values (reading of the fallback rule: the plain
        start stays as fallback whenever LM from the learned start converges
        to a worse chi^2 than LM from the plain start): the plain method
        fixed p*, the members and the window; the network proposes the new
        member's start from the 32 x 32 patch at p* (BF16 operands as on the
        GPU).  A proposal that is not finite, has a zero amplitude, or lies
        outside the window or the width bounds is not used (the plain fit
        alone).  Otherwise LM runs from both starts and the learned start's
        result is kept when it is finite, above the width bound and its
        chi^2 is not above the plain start's fit's."""
        from . import mlp_oracle as Mo
        omega_min = 0.25 * self.omega_b
        px, py = int(init["x0"]), int(init["y0"])
        rp = float(self.R[py, px])
        patch = Mo.extract_patch(self.R, px, py)
        out, _ = Mo.forward(self.mlp, patch[None, :], round_bf16=True)
        prop = Mo.init_from_output(out[0], rp, px, py, self.omega_b) if rp != 0 else np.full(4, np.nan)
        x0b, x1b, y0b, y1b = win
        omega_max = max(x1b - x0b + 1, y1b - y0b + 1)
        ok = (np.all(np.isfinite(prop)) and prop[0] != 0 and prop[3] > omega_min and not prop[3] > omega_max
              and x0b <= prop[1] <= x1b and y0b <= prop[2] <= y1b)
        info = dict(used=bool(ok), refit=False, kept=False, proposal=prop, chi2_learned=None, chi2_plain=None)
        if not ok:
            return lm_fit(T, xs, ys, theta0, win, omega_min, self.p.lm), info
        th_l = theta0.copy()
        th_l[0:4] = prop
        fit_l = lm_fit(T, xs, ys, th_l, win, omega_min, self.p.lm)
        fit_p = lm_fit(T, xs, ys, theta0, win, omega_min, self.p.lm)
        info["chi2_learned"], info["chi2_plain"] = fit_l.chi2, fit_p.chi2
        good = np.isfinite(fit_l.chi2) and fit_l.theta[3] > omega_min and fit_l.chi2 <= fit_p.chi2
        if good:
            info["kept"] = True
            return fit_l, info
        info["refit"] = True
        return fit_p, info

    def major(self):
        """The major cycle of the minor/major split: the exact residual
        ``R = D - B * M`` (Sect. 2 step 3 with the full PSF) of the whole
        component list, each component sampled as in the per-iteration
        subtraction."""
        terms = []
        for c in self.comps:
            t = component_terms(c.flux, c.x, c.y, c.width, c.is_point, self.H, self.W)
            if t is not None:
                terms.append(t)
        self.R = subtract_terms(self.D, self.B, terms)
        self.since_major = 0

    def run(self, n_iter):
        """Up to n_iter iterations; with the minor/major split a major cycle
        follows every major_every iterations and ends the run."""
        for _ in range(n_iter):
            rec = self.step()
            if rec is None:
                break
            if self.p.major_every > 0 and self.since_major >= self.p.major_every:
                self.major()
        if self.p.major_every > 0 and self.since_major > 0:
            self.major()
        return self

    # -- state exchange (teacher forcing)
    def get_state(self):
        return dict(R=self.R.copy(), comps=[dataclasses.replace(c) for c in self.comps],
                    retained=list(self.retained), t=self.t, last_wi=self.last_wi,
                    last_w0=self.last_w0)

    def set_state(self, R, comps, retained, t, last_wi, last_w0):
        self.R = np.array(R, dtype=np.float64)
        self.comps = [dataclasses.replace(c) for c in comps]
        self.retained = list(retained)
        self.t = int(t)
        self.last_wi = float(last_wi)
        self.last_w0 = float(last_w0)
        self.stopped = False

    def stats(self):
        fl = np.array([c.flux for c in self.comps]) if self.comps else np.zeros(0)
        return dict(iterations=self.t, components=len(self.comps),
                    model_flux=float(fl.sum()), residual_rms=float(np.sqrt(np.mean(self.R ** 2))),
                    residual_max=float(np.abs(self.R).max()),
                    pixel_evals=int(sum(h["fit"].pixel_evals for h in self.history)))
