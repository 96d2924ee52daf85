"""Pins of the FP64 oracle against closed forms and independent definitions.

Every check here compares the oracle with something that does not come from
the oracle itself: numerical integration, finite differences, pure-Python
loops, MINPACK's Levenberg-Marquardt, or a closed form of the mathematics.
"""
import math

import numpy as np
import pytest
from scipy.optimize import least_squares
from scipy.signal import fftconvolve

import oracle as O
import synth

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


# ----------------------------------------------------------------- Eq. 7-8

def _numeric_gauss_conv(alpha_i, w_i, alpha_b, w_b, step=0.05, span=7.0):
    """Continuous 2-D convolution of two centred circular Gaussians by
    direct numerical integration on a fine grid; returns (peak, width from
    the second moment, integral)."""
    n = int(round(span * max(w_i, w_b) * 1.5 / step))
    u = (np.arange(2 * n + 1) - n) * step      # odd length: zero lag on a sample
    X, Y = np.meshgrid(u, u)
    r2 = X * X + Y * Y
    f1 = alpha_i * np.exp(-r2 / (2 * w_i * w_i))
    f2 = alpha_b * np.exp(-r2 / (2 * w_b * w_b))
    conv = fftconvolve(f1, f2, mode="same") * step * step
    c = len(u) // 2
    peak = conv[c, c]
    integ = conv.sum() * step * step
    m2 = (conv * r2).sum() * step * step / integ
    return peak, math.sqrt(m2 / 2.0), integ


@pytest.mark.parametrize("alpha_i,w_i,alpha_b,w_b", [
    (0.3, 2.0, 1.0, 1.5), (1.7, 4.5, 0.9, 2.0), (-0.2, 1.1, 1.2, 1.3)])
def test_eq7_eq8_against_numerical_convolution(alpha_i, w_i, alpha_b, w_b):
    peak, w_ic, integ = _numeric_gauss_conv(alpha_i, w_i, alpha_b, w_b)
    F, alpha, wi, is_point = O.deconvolve(peak, w_ic, alpha_b, w_b)
    assert not is_point
    assert wi == pytest.approx(w_i, rel=2e-5)
    assert alpha == pytest.approx(alpha_i, rel=2e-4)
    # flux of the component = integral of the convolution / integral of the beam
    assert F == pytest.approx(integ / (2 * math.pi * alpha_b * w_b * w_b), rel=2e-4)
    assert F == pytest.approx(2 * math.pi * alpha_i * w_i * w_i, rel=2e-4)


def test_eq8_literal_and_widths_in_quadrature():
    a_ic, w_ic, ab, wb = 0.8, 3.0, 1.1, 1.7
    F, alpha, wi, _ = O.deconvolve(a_ic, w_ic, ab, wb)
    assert wi == pytest.approx(math.sqrt(w_ic ** 2 - wb ** 2), rel=1e-15)      # Eq. 7
    assert alpha == pytest.approx(a_ic * w_ic ** 2 / (2 * math.pi * ab * wb ** 2 * wi ** 2),
                                  rel=1e-14)                                    # Eq. 8
    a2, w2 = O.gauss_approx(F, wi, ab, wb)
    assert a2 == pytest.approx(a_ic, rel=1e-14) and w2 == pytest.approx(w_ic, rel=1e-14)


def test_point_rule_conserves_flux():
    ab, wb = 0.95, 1.5
    F, alpha, wi, is_point = O.deconvolve(0.5, 1.5, ab, wb)
    assert is_point and wi == 0.0
    assert F == pytest.approx(0.5 / ab)        # point source: a_ic = alpha_b F
    F2, _, _, p2 = O.deconvolve(0.5, 1.4, ab, wb)
    assert p2 and F2 == pytest.approx(0.5 * 1.4 ** 2 / (ab * wb ** 2))


# ----------------------------------------------------------------- Eq. 6 model

def test_model_against_python_loop():
    rng = np.random.default_rng(1)
    theta = [0.7, 3.2, 4.9, 1.3, -0.4, 5.5, 2.1, 2.7]
    xs = rng.uniform(0, 8, 13)
    ys = rng.uniform(0, 8, 13)
    m = O.gauss_model(theta, xs, ys)
    for i in range(13):
        v = 0.0
        for k in range(2):
            a, x0, y0, w = theta[4 * k: 4 * k + 4]
            v += a * math.exp(-((xs[i] - x0) ** 2 + (ys[i] - y0) ** 2) / (2 * w * w))
        assert m[i] == pytest.approx(v, rel=1e-15, abs=1e-300)


def test_jacobian_against_central_differences():
    rng = np.random.default_rng(2)
    theta = np.array([0.9, 10.3, 9.7, 2.2, -0.35, 12.1, 11.4, 3.1, 0.2, 8.0, 13.0, 1.6])
    ys, xs = np.mgrid[0:22, 0:20]
    xs = xs.ravel().astype(float)
    ys = ys.ravel().astype(float)
    _, J = O.model_and_jacobian(theta, xs, ys)
    for i in range(theta.size):
        h = 1e-5 * max(1.0, abs(theta[i]))
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (O.gauss_model(tp, xs, ys) - O.gauss_model(tm, xs, ys)) / (2 * h)
        err = np.max(np.abs(fd - J[:, i])) / np.max(np.abs(J[:, i]))
        assert err < 1e-7, (i, err)
    del rng


def test_normal_equations_against_python_sums():
    theta = [1.2, 2.4, 3.1, 1.7, 0.3, 4.0, 2.0, 2.5]
    pts = [(x, y) for y in range(6) for x in range(5)]
    T = [math.sin(0.3 * x + 0.7 * y) for x, y in pts]
    xs = np.array([p[0] for p in pts], float)
    ys = np.array([p[1] for p in pts], float)
    A, g, chi2 = O.normal_equations(T, xs, ys, theta)
    P = len(theta)
    A2 = [[0.0] * P for _ in range(P)]
    g2 = [0.0] * P
    c2 = 0.0
    for (x, y), t in zip(pts, T):
        row = []
        model = 0.0
        for k in range(2):
            a, x0, y0, w = theta[4 * k: 4 * k + 4]
            e = math.exp(-((x - x0) ** 2 + (y - y0) ** 2) / (2 * w * w))
            gk = a * e
            model += gk
            row += [e, gk * (x - x0) / w ** 2, gk * (y - y0) / w ** 2,
                    gk * ((x - x0) ** 2 + (y - y0) ** 2) / w ** 3]
        r = t - model
        c2 += r * r
        for i in range(P):
            g2[i] += row[i] * r
            for j in range(P):
                A2[i][j] += row[i] * row[j]
    np.testing.assert_allclose(A, np.array(A2), rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(g, np.array(g2), rtol=1e-13, atol=1e-15)
    assert chi2 == pytest.approx(c2, rel=1e-13)


# ----------------------------------------------------------------- LM

def _grid(nx, ny):
    ys, xs = np.mgrid[0:ny, 0:nx]
    return xs.ravel().astype(float), ys.ravel().astype(float)


def test_lm_recovers_noiseless_single_gaussian():
    xs, ys = _grid(31, 29)
    truth = np.array([0.83, 15.37, 13.81, 2.9])
    T = O.gauss_model(truth, xs, ys)
    fit = O.lm_fit(T, xs, ys, [0.5, 15.0, 14.0, 1.5], (0, 30, 0, 28), 0.3, O.lm_exact())
    np.testing.assert_allclose(fit.theta, truth, rtol=1e-9)
    assert fit.chi2 < 1e-20


def test_lm_recovers_noiseless_overlapping_gaussians():
    xs, ys = _grid(40, 36)
    truth = np.array([1.0, 15.2, 17.9, 2.4, 0.6, 21.3, 18.6, 3.3, -0.25, 18.1, 12.4, 1.9])
    T = O.gauss_model(truth, xs, ys)
    start = truth * np.array([0.8, 1, 1, 1.2, 1.2, 1, 1, 0.85, 0.7, 1, 1, 1.1]) + \
        np.array([0, 0.4, -0.3, 0, 0, -0.5, 0.3, 0, 0, 0.2, 0.4, 0])
    fit = O.lm_fit(T, xs, ys, start, (0, 39, 0, 35), 0.3, O.lm_exact())
    np.testing.assert_allclose(fit.theta, truth, rtol=1e-9, atol=1e-11)


@pytest.mark.parametrize("K", [1, 2])
def test_lm_matches_minpack_on_noisy_data(K):
    rng = np.random.default_rng(10 + K)
    xs, ys = _grid(26, 24)
    truth = np.array([0.9, 12.3, 11.7, 2.3, 0.4, 14.6, 12.9, 3.0])[: 4 * K]
    T = O.gauss_model(truth, xs, ys) + rng.normal(0, 0.01, xs.size)
    start = truth + np.tile([0.1, 0.3, -0.2, 0.4], K)
    fit = O.lm_fit(T, xs, ys, start, (0, 25, 0, 23), 0.3, O.lm_exact())
    ref = least_squares(lambda th: O.gauss_model(th, xs, ys) - T, start, method="lm",
                        xtol=1e-15, ftol=1e-15, gtol=1e-15, max_nfev=20000)
    # both stop where FP64 chi^2 can no longer resolve a step (~1e-8 here)
    np.testing.assert_allclose(fit.theta, ref.x, rtol=1e-7, atol=1e-9)
    assert fit.chi2 <= float(ref.fun @ ref.fun) * (1 + 1e-12)
    A, g, _ = O.normal_equations(T, xs, ys, fit.theta)       # stationarity
    assert np.max(np.abs(np.linalg.solve(A, g))) < 1e-7


def test_damped_solve_matches_direct():
    rng = np.random.default_rng(3)
    M = rng.normal(size=(8, 8))
    A = M @ M.T + 0.1 * np.eye(8)
    g = rng.normal(size=8)
    lam = 0.37
    d = np.linalg.solve(A + lam * np.diag(np.diag(A)), g)
    np.testing.assert_allclose(O.cholesky_solve_damped(A, g, lam), d, rtol=1e-12)
    assert O.cholesky_solve_damped(-A, g, 0.0) is None


# ----------------------------------------------------------------- beam

def test_beam_fit_config1_psf():
    c = synth.config1(0)
    ab, wb, fit = O.beam_fit(c.psf, O.lm_exact())
    assert ab == pytest.approx(1.0, abs=1e-6)
    assert wb == pytest.approx(1.5, abs=1e-6)


@pytest.mark.parametrize("sigma,amp", [(2.3, 0.7), (1.2, 1.0), (3.0, 2.5)])
def test_beam_fit_pure_gaussian(sigma, amp):
    psf = synth.gaussian_psf(32, 40, sigma, amp)
    ab, wb, fit = O.beam_fit(psf, O.lm_exact())
    assert ab == pytest.approx(amp, rel=1e-10)
    assert wb == pytest.approx(sigma, rel=1e-10)
    assert fit.theta[1] == pytest.approx(40.0, abs=1e-9) and fit.theta[2] == pytest.approx(32.0, abs=1e-9)


# ----------------------------------------------------------------- peak search

def test_argmax_against_python_scan_with_ties():
    rng = np.random.default_rng(4)
    for trial in range(20):
        h, w = rng.integers(1, 9, 2)
        R = rng.integers(-3, 4, (h, w)).astype(np.float32)
        idx, v = O.peak_simple(R)
        best, bi = -1.0, -1
        flat = R.ravel().tolist()
        for i, val in enumerate(flat):
            if abs(val) > best:
                best, bi = abs(val), i
        assert idx == bi and v == flat[bi]


def test_smoothing_kernel_unit_l2_and_scales():
    for s in (1.5, 3.0, 7.7):
        k = O.smoothing_kernel_1d(s)
        assert np.sum(np.outer(k, k) ** 2) == pytest.approx(1.0, rel=1e-14)
        assert len(k) == 2 * math.ceil(4 * s) + 1
    assert O.smoothing_scales(1.5, 6, 256, 256) == [1.5, 3.0, 6.0, 12.0, 24.0]
    assert O.smoothing_scales(40.0, 6, 64, 64) == [40.0]


@pytest.mark.parametrize("shape,s", [((17, 23), 1.5), ((20, 13), 3.0)])
def test_smoothing_separable_against_definition(shape, s):
    rng = np.random.default_rng(5)
    R = rng.normal(size=shape)
    np.testing.assert_allclose(O.smooth_separable(R, s), O.smooth_definition(R, s),
                               rtol=1e-12, atol=1e-13)


def test_smoothing_pure_python_corner():
    rng = np.random.default_rng(6)
    R = rng.normal(size=(9, 7))
    s = 1.2
    k = O.smoothing_kernel_1d(s)
    m = (len(k) - 1) // 2
    S = O.smooth_separable(R, s)
    for (py, px) in [(0, 0), (4, 3), (8, 6), (2, 5)]:
        v = 0.0
        for qy in range(-m, m + 1):
            for qx in range(-m, m + 1):
                y, x = py + qy, px + qx
                if 0 <= y < 9 and 0 <= x < 7:
                    v += k[qy + m] * k[qx + m] * R[y, x]
        assert S[py, px] == pytest.approx(v, rel=1e-12, abs=1e-14)


def test_smoothing_init_recovers_gaussian_scale_and_amplitude():
    wb = 1.5
    H = W = 96
    for j, A in [(1, 0.8), (2, -1.3)]:
        s = wb * 2 ** j
        ys, xs = np.mgrid[0:H, 0:W]
        R = A * np.exp(-((xs - 47) ** 2 + (ys - 50) ** 2) / (2 * s * s))
        init = O.peak_smooth(R, wb, 6)
        assert init["scale_index"] == j
        assert (init["x0"], init["y0"]) == (47.0, 50.0)
        assert init["a0"] == pytest.approx(A, rel=1e-7)
        assert init["w0"] == s


# ----------------------------------------------------------------- subtraction

def _random_terms(rng, H, W, n):
    terms = []
    for i in range(n):
        x, y = rng.uniform(-2, W + 1), rng.uniform(-2, H + 1)
        w = [0.0, 0.3, 0.8, 1.7][i % 4]
        t = O.component_terms(rng.normal(), x, y, w, w == 0.0, H, W)
        if t is not None:
            terms.append(t)
    return terms


@pytest.mark.parametrize("H,W", [(9, 11), (16, 13), (1, 5)])
def test_subtraction_separable_against_definition(H, W):
    rng = np.random.default_rng(H * 100 + W)
    R = rng.normal(size=(H, W))
    B = rng.normal(size=(2 * H, 2 * W))
    terms = _random_terms(rng, H, W, 8)
    a = O.subtract_terms(R, B, terms)
    b = O.subtract_definition(R, B, O.terms_to_image(terms, H, W))
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12)


def test_subtraction_pure_python_quadruple_loop():
    rng = np.random.default_rng(7)
    H, W = 5, 6
    R = rng.normal(size=(H, W))
    B = rng.normal(size=(2 * H, 2 * W))
    terms = _random_terms(rng, H, W, 4)
    dC = O.terms_to_image(terms, H, W)
    out = O.subtract_terms(R, B, terms)
    for py in range(H):
        for px in range(W):
            v = R[py, px]
            for qy in range(H):
                for qx in range(W):
                    v -= dC[qy, qx] * B[py - qy + H, px - qx + W]
            assert out[py, px] == pytest.approx(v, rel=1e-12, abs=1e-12)


def test_component_terms_flux_and_bilinear():
    H, W = 40, 50
    t = O.component_terms(2.5, 20.3, 18.6, 3.2, False, H, W)
    assert O.terms_to_image([t], H, W).sum() == pytest.approx(2.5, rel=1e-14)
    p = O.component_terms(1.0, 10.25, 7.5, 0.0, True, H, W)
    img = O.terms_to_image([p], H, W)
    assert img[7, 10] == pytest.approx(0.75 * 0.5) and img[8, 11] == pytest.approx(0.25 * 0.5)
    # centroid of a bilinear deposit is the component position
    ys, xs = np.mgrid[0:H, 0:W]
    assert (img * xs).sum() == pytest.approx(10.25) and (img * ys).sum() == pytest.approx(7.5)


def test_subtracting_gaussian_through_gaussian_psf_matches_closed_form():
    """A10: Gaussian (x) Gaussian is the Gaussian of Eqs. 7-8."""
    H, W = 64, 64
    ab, wb = 0.9, 1.6
    B = synth.gaussian_psf(H, W, wb, ab)
    F, wi, x, y = 3.0, 2.5, 31.4, 30.7
    t = O.component_terms(F, x, y, wi, False, H, W)
    out = -O.subtract_terms(np.zeros((H, W)), B, [t])
    a_ic, w_ic = O.gauss_approx(F, wi, ab, wb)
    ys, xs = np.mgrid[0:H, 0:W]
    expect = a_ic * np.exp(-((xs - x) ** 2 + (ys - y) ** 2) / (2 * w_ic ** 2))
    assert np.max(np.abs(out - expect)) < 1e-4 * abs(a_ic)


# ----------------------------------------------------------------- minor cycle

def test_first_iteration_on_point_source_gaussian_psf():
    """Noiseless point source through a Gaussian PSF: the first fit finds
    (alpha_b F, omega_b) exactly, the component is a point with gain*F, and
    the residual is (1 - gain) * dirty."""
    H, W = 48, 52
    ab, wb = 1.0, 1.7
    B = synth.gaussian_psf(H, W, wb, ab)
    sky = np.zeros((H, W))
    sky[20, 27] = 0.8
    dirty = O.subtract_definition(np.zeros((H, W)), B, -sky)
    p = O.AspParams(k_max=1, noise_sigma=1e-6, init_mode="simple", lm=O.lm_exact())
    mc = O.MinorCycle(dirty, B, p)
    assert mc.alpha_b == pytest.approx(ab, rel=1e-10) and mc.omega_b == pytest.approx(wb, rel=1e-10)
    mc.step()
    c = mc.comps[0]
    assert c.is_point and c.flux == pytest.approx(0.35 * 0.8, rel=1e-8)
    assert (c.x, c.y) == (pytest.approx(27.0, abs=1e-8), pytest.approx(20.0, abs=1e-8))
    np.testing.assert_allclose(mc.R, 0.65 * dirty, atol=1e-9)


def test_kmax1_fit_is_eq6_least_squares():
    """With an active set of one the fit is exactly Eq. 6 on the window."""
    c = synth.small_case(40, 44, seed=3, n_points=1, n_gauss=1)
    p = O.AspParams(k_max=1, noise_sigma=1e-3, init_mode="smooth", lm=O.lm_exact())
    mc = O.MinorCycle(c.dirty, c.psf, p)
    R0 = mc.R.copy()
    rec = mc.step()
    x0, x1, y0, y1 = rec["window"]
    ys, xs = np.mgrid[y0:y1 + 1, x0:x1 + 1]
    xs, ys = xs.ravel().astype(float), ys.ravel().astype(float)
    T = R0[y0:y1 + 1, x0:x1 + 1].ravel()
    init = rec["init"]
    start = [init["a0"], init["x0"], init["y0"], init["w0"]]
    ref = least_squares(lambda th: O.gauss_model(th, xs, ys) - T, start, method="lm",
                        xtol=1e-15, ftol=1e-15, gtol=1e-15, max_nfev=20000)
    np.testing.assert_allclose(rec["fit"].theta, ref.x, rtol=1e-7, atol=1e-9)


def test_minor_cycle_reduces_residual_and_recovers_flux():
    H, W = 48, 48
    ab, wb = 1.0, 1.5
    B = synth.gaussian_psf(H, W, wb, ab)
    sky = np.zeros((H, W))
    sky[12, 30] = 1.0
    sky[33, 15] = -0.5
    dirty = O.subtract_definition(np.zeros((H, W)), B, -sky)
    p = O.AspParams(k_max=3, noise_sigma=1e-4)
    mc = O.MinorCycle(dirty, B, p).run(60)
    st = mc.stats()
    assert st["residual_max"] < 2e-3
    assert st["model_flux"] == pytest.approx(0.5, abs=5e-3)


# ----------------------------------------------------------------- active set and width bound (readings)

def test_active_set_excludes_colocated_members():
    c = synth.small_case(64, 64, seed=1, n_points=1, n_gauss=0)
    mc = O.MinorCycle(c.dirty, c.psf, O.AspParams(k_max=4, noise_sigma=1e-3))
    wb = mc.omega_b
    mc.comps = [O.Component(1.0, 1.0, 30.0, 30.0, 0.0, True),      # co-located with the new member
                O.Component(1.0, 1.0, 34.5, 30.0, 0.0, True),      # overlapping, 4.5 px away
                O.Component(1.0, 1.0, 60.0, 60.0, 0.0, True)]      # no overlap
    mc.retained = [0, 1, 2]
    chosen, win = mc.select(dict(a0=1.0, x0=30.2, y0=29.9, w0=wb))
    assert chosen == [1]
    b_new, b_1 = O.member_box(30.2, 29.9, wb), O.member_box(34.5, 30.0, mc.G(1)[3])
    assert win == (min(b_new[0], b_1[0]), max(b_new[1], b_1[1]), min(b_new[2], b_1[2]), max(b_new[3], b_1[3]))


def test_trial_widths_bounded_by_window():
    xs, ys = _grid(15, 15)
    T = 0.01 + 0.001 * xs          # a pedestal: an unbounded width would fit it best
    fit = O.lm_fit(T, xs, ys, [0.5, 7.0, 7.0, 3.0], (0, 14, 0, 14), 0.3, O.lm_exact())
    assert 0.3 < fit.theta[3] <= 15.0


def test_minor_cycle_recovers_total_flux_and_reaches_noise():
    """The paper's quality observables (Table 1: total model flux close to the
    original's; Table 2 / Fig. 4: residual at the noise level), on a field
    whose true sky is known."""
    case = synth.small_case(72, 80, seed=21, n_points=3, n_gauss=1, sigma_range=(2.0, 3.0), noise_sigma=1e-3)
    mc = O.MinorCycle(case.dirty, case.psf, O.AspParams(k_max=3, noise_sigma=case.noise_sigma)).run(400)
    st = mc.stats()
    assert mc.stopped                                     # stopped by the noise threshold
    assert st["residual_max"] < 3 * case.noise_sigma
    assert st["model_flux"] == pytest.approx(case.sky.sum(), rel=0.01)
    assert st["residual_rms"] == pytest.approx(case.noise_sigma, rel=0.1)


# ----------------------------------------------------------------- noise level, init switch, boxes (readings)

def test_mad_sigma_hand_computed_and_normal_consistency():
    """1.4826 x MAD: hand-computed medians on small arrays (odd and even
    length, an outlier), and the estimator's defining property -- on a
    normal sample it estimates the standard deviation, since the median of
    |N(0, s^2)| is s times the 0.75 quantile of N(0, 1), 0.674490 (so
    1.4826 = 1 / 0.674490 to five digits)."""
    assert O.mad_sigma([1.0, 2.0, 3.0, 4.0, 100.0]) == pytest.approx(1.4826, rel=1e-15)   # med 3, |dev| med 1
    assert O.mad_sigma([1.0, 2.0, 3.0, 4.0]) == pytest.approx(1.4826, rel=1e-15)          # med 2.5, |dev| med 1
    assert O.mad_sigma([[5.0, 5.0], [5.0, 9.0]]) == 0.0                                     # med 5, |dev| med 0
    assert O.mad_sigma([-2.0, 0.0, 0.0, 0.0, 6.0]) == 0.0
    assert 1.0 / 1.4826 == pytest.approx(0.6744897501960817, rel=1e-4)                      # Phi^-1(3/4)
    rng = np.random.default_rng(12)
    for s in (1e-3, 2.5):
        x = rng.normal(0.7, s, 1_000_000)
        assert O.mad_sigma(x) == pytest.approx(s, rel=0.01)


def _mc_with_last(t, last_wi, last_w0, area_frac=0.05, init_mode="auto"):
    c = synth.small_case(24, 24, seed=0, n_points=1, n_gauss=0)
    mc = O.MinorCycle(c.dirty, c.psf, O.AspParams(area_frac=area_frac, init_mode=init_mode, noise_sigma=1e-3),
                      beam=(1.0, 1.5))
    mc.t, mc.last_wi, mc.last_w0 = t, last_wi, last_w0
    return mc


def test_choose_mode_five_percent_area_rule():
    """Sect. 3: the simple method iff the area of the last optimal component
    is below 5 % of the area of the last initial guess (area ~ width^2).
    Constructed cases: the first iteration has no history (smoothing); a
    point component (omega_i = 0) means the simple method; areas just below
    and above 5 %; a width ratio of 0.1 is an area ratio of 0.01; exact
    equality is not 'below' (area_frac 1/4 and widths 1 and 2 make it exact
    in binary)."""
    assert _mc_with_last(0, 0.0, 1.5).choose_mode() == O.MODE_SMOOTH
    assert _mc_with_last(3, 0.0, 1.5).choose_mode() == O.MODE_SIMPLE
    assert _mc_with_last(3, 0.2236, 1.0).choose_mode() == O.MODE_SIMPLE      # area ratio 0.049997
    assert _mc_with_last(3, 0.2237, 1.0).choose_mode() == O.MODE_SMOOTH      # area ratio 0.050042
    assert _mc_with_last(3, 0.1, 1.0).choose_mode() == O.MODE_SIMPLE
    assert _mc_with_last(3, 1.0, 2.0, area_frac=0.25).choose_mode() == O.MODE_SMOOTH
    assert _mc_with_last(3, 0.999, 2.0, area_frac=0.25).choose_mode() == O.MODE_SIMPLE
    assert _mc_with_last(3, 5.0, 1.0, init_mode="simple").choose_mode() == O.MODE_SIMPLE
    assert _mc_with_last(3, 0.0, 1.0, init_mode="smooth").choose_mode() == O.MODE_SMOOTH


def test_member_box_half_width_and_rounding():
    """Member box: half-width max(5, ceil(4 omega)) around the centre
    rounded half up; values worked by hand."""
    assert O.member_box(10.0, 20.0, 1.0) == (5, 15, 15, 25)          # 4 omega = 4 < 5
    assert O.member_box(10.0, 20.0, 1.25) == (5, 15, 15, 25)         # ceil(5.0) = 5
    assert O.member_box(10.0, 20.0, 1.26) == (4, 16, 14, 26)         # ceil(5.04) = 6
    assert O.member_box(2.5, 3.49, 2.0) == (-5, 11, -5, 11)          # 2.5 -> 3, 3.49 -> 3, h = 8
    assert O.member_box(-0.5, -1.5, 0.5) == (-5, 5, -6, 4)           # -0.5 -> 0, -1.5 -> -1
    assert O.member_box(7.5, 8.5, 30.0) == (-112, 128, -111, 129)    # h = 120


def test_window_is_clipped_bounding_box_of_member_boxes():
    """The joint window: bounding box of the members' boxes clipped to the
    image, worked by hand for a new member at a corner and one retained
    member reaching past the opposite edge."""
    c = synth.small_case(40, 50, seed=0, n_points=1, n_gauss=0)
    mc = O.MinorCycle(c.dirty, c.psf, O.AspParams(k_max=3, noise_sigma=1e-3), beam=(1.0, 1.5))
    # retained member: flux 1, width 3 -> omega_ic = sqrt(9 + 2.25) = 3.354, h = ceil(13.42) = 14
    mc.comps = [O.Component(1.0, 1.0 / (2 * math.pi * 9.0), 8.4, 33.2, 3.0, False)]
    mc.retained = [0]
    chosen, win = mc.select(dict(a0=1.0, x0=2.0, y0=37.0, w0=1.5))   # new box: h = 6, (-4, 8, 31, 43)
    assert chosen == [0]                                              # 6.4^2 + 3.8^2 > 3.354^2
    assert win == (0, 22, 19, 39)                                     # (-6, 22, 19, 47) clipped to 50 x 40
    chosen, win = mc.select(dict(a0=1.0, x0=49.0, y0=0.0, w0=1.5))   # far corner: no overlap
    assert chosen == [] and win == (43, 49, 0, 6)


# ----------------------------------------------------------------- minor/major split (reading of the Clark comparison)

@pytest.mark.parametrize("F,x,y,w", [(1.3, 20.4, 18.7, 2.5), (-0.6, 15.0, 22.0, 0.0), (0.8, 21.6, 19.1, 4.0)])
def test_beam_image_is_full_psf_subtraction_through_a_gaussian_psf(F, x, y, w):
    """Through a PSF that is itself the Gaussian (alpha_b, omega_b), the
    minor cycle's beam image of a component is the exact subtraction of its
    sampled image (Sect. 3: Gaussian * Gaussian is the Gaussian with widths
    in quadrature and the amplitude of Eq. 8) -- up to the discrete
    sampling's aliasing and the 5 omega_ic box; a point component (w = 0)
    on a pixel is the beam itself (off a pixel the exact path deposits it
    bilinearly, a reading of its own)."""
    H, W = 40, 44
    ab, wb = 0.9, 1.8
    B = synth.gaussian_psf(H, W, wb, ab)
    t = O.component_terms(F, x, y, w, w == 0.0, H, W)
    exact = -O.subtract_terms(np.zeros((H, W)), B, [t])
    approx = -O.subtract_beam_images(np.zeros((H, W)), [(F, x, y, w)], ab, wb)
    scale = np.abs(exact).max()
    assert np.abs(exact - approx).max() <= 2e-5 * scale


def test_major_cycle_is_the_brute_force_exact_residual():
    c = synth.small_case(24, 28, seed=4, n_points=1, n_gauss=1, sigma_range=(2.0, 3.0))
    mc = O.MinorCycle(c.dirty, c.psf, O.AspParams(k_max=2, noise_sigma=c.noise_sigma, major_every=3))
    for _ in range(2):
        mc.step()
    mc.major()
    dC = O.terms_to_image([O.component_terms(k.flux, k.x, k.y, k.width, k.is_point, 24, 28) for k in mc.comps], 24, 28)
    ref = O.subtract_definition(c.dirty, c.psf, dC)
    np.testing.assert_allclose(mc.R, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_major_every_iteration_reproduces_the_exact_cycle():
    """With a major cycle after every minor iteration the residual is exact
    at every peak search: the run takes the exact cycle's decisions and ends
    with its components."""
    c = synth.small_case(48, 52, seed=6, n_points=2, n_gauss=1, sigma_range=(2.0, 4.0))
    a = O.MinorCycle(c.dirty, c.psf, O.AspParams(k_max=3, noise_sigma=c.noise_sigma)).run(12)
    b = O.MinorCycle(c.dirty, c.psf, O.AspParams(k_max=3, noise_sigma=c.noise_sigma, major_every=1)).run(12)
    assert [h["window"] for h in a.history] == [h["window"] for h in b.history]
    fa = np.array([[k.flux, k.x, k.y, k.width] for k in a.comps])
    fb = np.array([[k.flux, k.x, k.y, k.width] for k in b.comps])
    np.testing.assert_allclose(fa, fb, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(a.R, b.R, rtol=0, atol=1e-10)


# ----------------------------------------------------------------- Asp-Clean2004 objective (Eq. 3)

@pytest.mark.parametrize("H,W", [(9, 11), (16, 13)])
def test_psf_convolve_is_the_direct_convolution(H, W):
    rng = np.random.default_rng(H * W)
    B = rng.normal(size=(2 * H, 2 * W))
    img = rng.normal(size=(H, W))
    np.testing.assert_allclose(O.psf_convolve(B, img), -O.subtract_definition(np.zeros((H, W)), B, img),
                               rtol=0, atol=1e-12)


def test_2004_jacobian_against_central_differences():
    H, W = 20, 22
    B = synth.small_case(H, W, seed=2).psf.astype(np.float64)
    theta = np.array([0.8, 9.3, 10.6, 2.1, -0.4, 12.2, 8.8, 1.4])
    _, J = O.model_jac_2004(B, theta, H, W)
    for j in range(theta.size):
        h = 1e-6 * max(1.0, abs(theta[j]))
        tp, tm = theta.copy(), theta.copy()
        tp[j] += h
        tm[j] -= h
        fd = (O.model_jac_2004(B, tp, H, W)[0] - O.model_jac_2004(B, tm, H, W)[0]) / (2 * h)
        assert np.max(np.abs(fd - J[:, j])) <= 1e-6 * max(np.max(np.abs(J[:, j])), 1e-12), j


def test_eq3_optimum_maps_to_eq6_optimum_through_eqs7_8():
    """Sect. 3's premise, made exact by a Gaussian PSF: fitting the
    unconvolved component through B (Eq. 3) and fitting the convolved
    Gaussian directly (Eq. 6) reach the same optimum, related by Eq. 7
    (omega_ic^2 = omega_i^2 + omega_b^2) and Eq. 8 (alpha_ic = 2 pi alpha_i
    alpha_b omega_i^2 omega_b^2 / omega_ic^2), with equal centres."""
    H, W = 40, 44
    ab, wb = 0.9, 1.8
    B = synth.gaussian_psf(H, W, wb, ab)
    truth = np.array([0.7, 21.3, 19.6, 2.6])
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    D = O.psf_convolve(B, O.gauss_model(truth, xs, ys)) + np.random.default_rng(1).normal(0, 1e-4, (H, W))
    f3 = O.lm_fit_2004(D, B, truth * [1.1, 1, 1, 0.9] + [0, 0.2, -0.2, 0], 0.3, O.lm_exact())
    f6 = O.lm_fit(D.ravel(), xs.ravel(), ys.ravel(), [1.0, 21.0, 20.0, 3.0], (0, W - 1, 0, H - 1), 0.3,
                  O.lm_exact())
    a, x, y, w = f3.theta
    a_ic, x_ic, y_ic, w_ic = f6.theta
    assert w_ic ** 2 == pytest.approx(w * w + wb * wb, rel=1e-9)
    assert a_ic == pytest.approx(2 * math.pi * a * ab * w * w * wb * wb / w_ic ** 2, rel=1e-9)
    assert x == pytest.approx(x_ic, abs=1e-9) and y == pytest.approx(y_ic, abs=1e-9)
    assert f3.chi2 == pytest.approx(f6.chi2, rel=1e-9)
