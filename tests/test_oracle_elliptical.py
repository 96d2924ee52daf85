"""Pins of the elliptical oracle (oracle/elliptical.py) to things other than
itself: the paper's circular case term by term, central finite
differences, exact recovery of noiseless rotated ellipses, MINPACK on the
same objective, the continuous convolution identity against a numerical
2-D convolution of sampled Gaussians, and planted mistakes each pin must
catch."""
import math

import numpy as np
import pytest
import scipy.optimize
import scipy.signal

import oracle as O
import oracle.elliptical as E


def _grid(H, W):
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    return xs.ravel(), ys.ravel()


def _circ_to_ell(theta4):
    out = []
    for a, x, y, w in np.asarray(theta4, float).reshape(-1, 4):
        out += [a, x, y, 1.0 / (w * w), 0.0, 1.0 / (w * w)]
    return np.array(out)


def test_circular_case_is_the_papers_model_and_jacobian():
    """With A = C = 1/omega^2 and B = 0 the model is Eq. 6's Gaussian, the
    a, x0, y0 columns are the circular ones and the chain rule through
    dA/domega = dC/domega = -2/omega^3 gives the omega column."""
    xs, ys = _grid(23, 27)
    th4 = np.array([1.3, 11.2, 12.7, 2.3, -0.4, 15.1, 8.9, 3.4])
    m4, J4 = O.model_and_jacobian(th4, xs, ys)
    m6, J6 = E.ell_model_and_jacobian(_circ_to_ell(th4), xs, ys)
    np.testing.assert_allclose(m6, m4, rtol=1e-12, atol=1e-300)
    for k in range(2):
        w = th4[4 * k + 3]
        np.testing.assert_allclose(J6[:, 6 * k: 6 * k + 3], J4[:, 4 * k: 4 * k + 3], rtol=1e-13, atol=1e-300)
        dw = (J6[:, 6 * k + 3] + J6[:, 6 * k + 5]) * (-2.0 / w ** 3)
        np.testing.assert_allclose(dw, J4[:, 4 * k + 3], rtol=1e-12, atol=1e-15)


def test_model_against_python_loop():
    th = np.array([0.9, 4.3, 5.1] + list(E.precision_from_axes(2.5, 1.2, 0.7)))
    for x, y in ((0, 0), (4, 5), (7, 2), (3, 9)):
        A, B, C = th[3:]
        dx, dy = x - th[1], y - th[2]
        expect = th[0] * math.exp(-0.5 * (A * dx * dx + 2 * B * dx * dy + C * dy * dy))
        assert E.ell_model(th, np.float64(x), np.float64(y)) == pytest.approx(expect, rel=1e-14)


def test_jacobian_against_central_differences():
    xs, ys = _grid(19, 21)
    th = np.array([1.1, 9.3, 10.2] + list(E.precision_from_axes(3.1, 1.4, 0.45)) +
                  [-0.6, 6.7, 8.8] + list(E.precision_from_axes(2.0, 1.7, -1.1)))
    _, J = E.ell_model_and_jacobian(th, xs, ys)
    for i in range(th.size):
        h = 1e-6 * max(1.0, abs(th[i]))
        tp, tm = th.copy(), th.copy()
        tp[i] += h
        tm[i] -= h
        fd = (E.ell_model(tp, xs, ys) - E.ell_model(tm, xs, ys)) / (2 * h)
        np.testing.assert_allclose(J[:, i], fd, rtol=1e-6, atol=1e-8 * np.max(np.abs(fd)) + 1e-12)


def test_axes_round_trip():
    for smaj, smin, phi in ((3.0, 1.0, 0.3), (2.0, 1.9, -1.2), (5.0, 0.8, 1.5)):
        A, B, C = E.precision_from_axes(smaj, smin, phi)
        a2, b2, p2 = E.axes_from_precision(A, B, C)
        assert a2 == pytest.approx(smaj, rel=1e-12) and b2 == pytest.approx(smin, rel=1e-12)
        assert p2 == pytest.approx(phi, abs=1e-10)


@pytest.mark.parametrize("truth", [
    [(1.0, 16.3, 15.6, 4.0, 1.5, 0.6)],
    [(0.8, 12.2, 14.1, 3.0, 1.8, -0.4), (-0.5, 20.7, 17.3, 2.4, 2.0, 1.1)],
    [(0.7, 10.5, 10.4, 2.8, 1.3, 0.2), (0.6, 19.3, 12.2, 2.2, 1.6, 1.3), (0.4, 14.6, 21.1, 3.4, 2.9, -0.9)],
])
def test_lm_recovers_noiseless_rotated_ellipses(truth):
    H, W = 32, 32
    xs, ys = _grid(H, W)
    th = np.concatenate([[a, x, y, *E.precision_from_axes(s1, s2, p)] for a, x, y, s1, s2, p in truth])
    T = E.ell_model(th, xs, ys)
    start = th.copy()
    for k in range(len(truth)):
        start[6 * k] *= 0.9
        start[6 * k + 1] += 0.3
        start[6 * k + 2] -= 0.2
        start[6 * k + 3: 6 * k + 6] *= np.array([1.15, 0.8, 0.9])
    fit = E.ell_lm_fit(T, xs, ys, start, (0, W - 1, 0, H - 1), 0.3, O.lm_exact())
    assert fit.status == O.LM_CONVERGED
    np.testing.assert_allclose(fit.theta, th, rtol=1e-8, atol=1e-9)


def test_lm_matches_minpack_on_noisy_data():
    H, W = 30, 34
    xs, ys = _grid(H, W)
    th = np.array([1.0, 15.2, 14.4, *E.precision_from_axes(3.5, 1.6, 0.8),
                   0.5, 21.3, 17.8, *E.precision_from_axes(2.2, 1.9, -0.3)])
    T = E.ell_model(th, xs, ys) + np.random.default_rng(3).normal(0, 0.02, xs.size)
    start = th * np.array([0.9, 1.01, 0.99, 1.1, 0.9, 1.05] * 2)
    fit = E.ell_lm_fit(T, xs, ys, start, (0, W - 1, 0, H - 1), 0.3, O.lm_exact())
    ref = scipy.optimize.least_squares(lambda p: E.ell_model(p, xs, ys) - T, start,
                                       jac=lambda p: E.ell_model_and_jacobian(p, xs, ys)[1],
                                       method="lm", xtol=1e-15, ftol=1e-15, gtol=1e-15, max_nfev=20000)
    np.testing.assert_allclose(fit.theta, ref.x, rtol=1e-7, atol=1e-9)


def test_circular_data_fits_to_a_circle_with_the_circular_optimum():
    H, W = 28, 30
    xs, ys = _grid(H, W)
    th4 = np.array([0.9, 14.3, 13.6, 2.7])
    T = O.gauss_model(th4, xs, ys) + np.random.default_rng(5).normal(0, 0.01, xs.size)
    c = O.lm_fit(T, xs, ys, th4 * [0.9, 1.0, 1.0, 1.1], (0, W - 1, 0, H - 1), 0.3, O.lm_exact())
    e = E.ell_lm_fit(T, xs, ys, _circ_to_ell(th4 * [0.9, 1.0, 1.0, 1.1]), (0, W - 1, 0, H - 1), 0.3, O.lm_exact())
    # the elliptical optimum has at least the circular fit's quality, and
    # on data that is a circle plus noise it stays close to that circle
    assert e.chi2 <= c.chi2 * (1 + 1e-12)
    a, x, y, A, B, C = e.theta
    w = c.theta[3]
    assert abs(B) < 0.02 / w ** 2 and A == pytest.approx(1 / w ** 2, rel=0.02) and C == pytest.approx(1 / w ** 2, rel=0.02)
    assert x == pytest.approx(c.theta[1], abs=0.01) and y == pytest.approx(c.theta[2], abs=0.01)


def _sampled(a, P, h, n):
    u = (np.arange(n) - n // 2) * h
    X, Y = np.meshgrid(u, u)
    A, B, C = P[0][0], P[0][1], P[1][1]
    return a * np.exp(-0.5 * (A * X * X + 2 * B * X * Y + C * Y * Y)), X, Y


@pytest.mark.parametrize("comp,beam", [
    ((0.7, 2.6, 1.1, 0.4), (1.2, 1.8, 1.3, -0.7)),
    ((1.5, 1.4, 1.4, 0.0), (0.9, 2.1, 2.1, 0.0)),
    ((0.3, 3.3, 0.9, 1.2), (1.0, 1.5, 1.2, 0.2)),
])
def test_convolution_identity_against_numerical_convolution(comp, beam):
    """Sigma_ic = Sigma_i + Sigma_b and flux_ic = flux_i flux_b, checked
    against the 2-D convolution of the two sampled Gaussians (grid step
    h, sum times h^2), then inverted by ell_deconvolve."""
    a_i, s1, s2, p = comp
    a_b, t1, t2, q = beam
    P_i = np.array(E.precision_from_axes(s1, s2, p))
    P_b = np.array(E.precision_from_axes(t1, t2, q))
    Pm = lambda v: np.array([[v[0], v[1]], [v[1], v[2]]])
    h, n = 0.125, 257
    gi, _, _ = _sampled(a_i, Pm(P_i), h, n)
    gb, _, _ = _sampled(a_b, Pm(P_b), h, n)
    conv = scipy.signal.fftconvolve(gi, gb, mode="same") * h * h
    a_ic, P_ic = E.ell_convolve_shape(a_i, Pm(P_i), a_b, Pm(P_b))
    ref, _, _ = _sampled(a_ic, P_ic, h, n)
    c = n // 2
    sl = slice(c - 60, c + 61)
    np.testing.assert_allclose(conv[sl, sl], ref[sl, sl], rtol=1e-6, atol=1e-9 * a_ic)
    F, a_back, S_i, is_point = E.ell_deconvolve(a_ic, P_ic, a_b, Pm(P_b))
    assert not is_point
    assert F == pytest.approx(2 * math.pi * a_i / math.sqrt(np.linalg.det(Pm(P_i))), rel=1e-12)
    assert a_back == pytest.approx(a_i, rel=1e-12)
    np.testing.assert_allclose(S_i, np.linalg.inv(Pm(P_i)), rtol=1e-12, atol=1e-12)


def test_deconvolve_circular_case_is_eqs_7_8():
    """For circular shapes the elliptical rule is Eqs. 7-8 (asp_oracle.deconvolve),
    the point case included."""
    ab, wb = 0.8, 1.7
    Pb = np.eye(2) / wb ** 2
    for a_ic, w_ic in ((1.3, 2.9), (0.4, 1.7 * math.sqrt(1.0005)), (2.0, 1.6)):
        F, a_i, S_i, pt = E.ell_deconvolve(a_ic, np.eye(2) / w_ic ** 2, ab, Pb)
        Fc, ac, wc, ptc = O.deconvolve(a_ic, w_ic, ab, wb)
        assert pt == ptc and F == pytest.approx(Fc, rel=1e-12) and a_i == pytest.approx(ac, rel=1e-12)
        assert math.sqrt(S_i[0, 0]) == pytest.approx(wc, rel=1e-12, abs=1e-12)


def test_beam_fit_recovers_an_elliptical_gaussian_psf():
    H, W = 40, 44
    P = E.precision_from_axes(2.6, 1.5, 0.5)
    ys, xs = np.mgrid[0:2 * H, 0:2 * W].astype(np.float64)
    B = E.ell_model(np.array([1.0, W, H, *P]), xs, ys)
    th, fit = E.ell_beam_fit(B, O.lm_exact())
    np.testing.assert_allclose(th, [1.0, W, H, *P], rtol=1e-8, atol=1e-9)


def test_valid_rejects_non_positive_definite_and_out_of_range_widths():
    box = (0, 20, 0, 20)
    ok = np.array([1.0, 10.0, 10.0, *E.precision_from_axes(3.0, 1.0, 0.3)])
    assert E.ell_valid(ok, box, 0.5)
    bad_pd = ok.copy()
    bad_pd[4] = math.sqrt(ok[3] * ok[5]) * 1.01      # B^2 > A C
    assert not E.ell_valid(bad_pd, box, 0.5)
    assert not E.ell_valid(ok, box, 1.01)              # sigma_min = 1 <= omega_min
    wide = np.array([1.0, 10.0, 10.0, *E.precision_from_axes(21.5, 2.0, 0.0)])
    assert not E.ell_valid(wide, box, 0.5)             # sigma_max above the window extent
    off = ok.copy()
    off[1] = 20.5
    assert not E.ell_valid(off, box, 0.5)


# ---------------------------------------------------------------- planted mistakes

def _patch(monkeypatch, name, fn):
    monkeypatch.setattr(E, name, fn)


def test_planted_cross_term_sign_is_caught(monkeypatch):
    orig = E.ell_model_and_jacobian

    def bad(theta, xs, ys):
        m, J = orig(theta, xs, ys)
        J = J.copy()
        J[:, 4::6] *= -1.0          # d/dB with the wrong sign
        return m, J

    _patch(monkeypatch, "ell_model_and_jacobian", bad)
    with pytest.raises(AssertionError):
        test_jacobian_against_central_differences()


def test_planted_missing_cross_factor_two_is_caught(monkeypatch):
    def bad(theta, xs, ys):
        theta = np.asarray(theta, float)
        out = np.zeros(np.broadcast(xs, ys).shape)
        for k in range(len(theta) // 6):
            a, x0, y0, A, B, C = theta[6 * k: 6 * k + 6]
            dx, dy = xs - x0, ys - y0
            out += a * np.exp(-0.5 * (A * dx * dx + B * dx * dy + C * dy * dy))
        return out

    _patch(monkeypatch, "ell_model", bad)
    with pytest.raises(AssertionError):
        test_model_against_python_loop()


def test_planted_precisions_added_instead_of_covariances_is_caught(monkeypatch):
    def bad(a_i, P_i, alpha_b, P_b):
        Si, Sb = np.linalg.inv(P_i), np.linalg.inv(P_b)
        P_ic = np.asarray(P_i) + np.asarray(P_b)                # precisions added
        a_ic = a_i * alpha_b * 2 * math.pi * math.sqrt(np.linalg.det(Si) * np.linalg.det(Sb) * np.linalg.det(P_ic))
        return a_ic, P_ic

    _patch(monkeypatch, "ell_convolve_shape", bad)
    with pytest.raises(AssertionError):
        test_convolution_identity_against_numerical_convolution((0.7, 2.6, 1.1, 0.4), (1.2, 1.8, 1.3, -0.7))


def test_planted_deconvolution_without_the_beam_determinant_is_caught(monkeypatch):
    def bad(a_ic, P_ic, alpha_b, P_b):
        Sic, Sb = np.linalg.inv(P_ic), np.linalg.inv(P_b)
        F = a_ic * math.sqrt(np.linalg.det(Sic)) / alpha_b      # det Sigma_b dropped
        Si = Sic - Sb
        return F, F / (2 * math.pi * math.sqrt(np.linalg.det(Si))), Si, False

    _patch(monkeypatch, "ell_deconvolve", bad)
    with pytest.raises(AssertionError):
        test_deconvolve_circular_case_is_eqs_7_8()


def test_planted_validity_without_positive_definiteness_is_caught(monkeypatch):
    def bad(theta, box, omega_min):
        return bool(np.all(np.isfinite(theta)))

    _patch(monkeypatch, "ell_valid", bad)
    with pytest.raises(AssertionError):
        test_valid_rejects_non_positive_definite_and_out_of_range_widths()


def test_precision_form_equals_the_rotated_axes_form():
    """The precision-matrix model against the generator's independent
    rotated-axes formula u^2/s1^2 + v^2/s2^2."""
    import synth
    src = [(1.0, 10.3, 9.7, 3.0, 1.5, 0.6), (-0.4, 5.2, 14.1, 2.2, 2.0, -1.3)]
    img = synth.elliptical_field(20, 22, src, 0.0, 0)
    ys, xs = np.mgrid[0:20, 0:22].astype(float)
    th = np.concatenate([[a, x, y, *E.precision_from_axes(s1, s2, p)] for a, x, y, s1, s2, p in src])
    np.testing.assert_allclose(E.ell_model(th, xs, ys), img, rtol=1e-12, atol=1e-15)


# ---------------------------------------------------------------- member box and xtol scales

def test_member_box_of_a_circle_is_the_circular_box():
    for x, y, w in ((10.2, 7.5, 1.3), (40.5, 3.49, 2.6), (-3.5, 12.0, 0.7)):
        assert E.ell_member_box(x, y, 1 / w ** 2, 0.0, 1 / w ** 2) == O.member_box(x, y, w)


def test_member_box_follows_the_major_width():
    A, B, C = E.precision_from_axes(3.2, 0.9, 0.6)
    h = max(math.ceil(4 * 3.2), 5)                              # 13
    assert E.ell_member_box(20.4, 30.6, A, B, C) == (20 - h, 20 + h, 31 - h, 31 + h)


def test_xtol_scales_hand_values():
    A, B, C = 1 / 9, 0.0, 1.0                                   # major width 3 along x, minor 1
    sc = E.ell_step_scale(np.array([-0.4, 5.0, 6.0, A, B, C, 0.0, 1.0, 2.0, 0.25, 0.0, 0.25]))
    np.testing.assert_allclose(sc, [0.4, 3.0, 3.0, 5 / 9, 5 / 9, 5 / 9, 1.0, 2.0, 2.0, 0.25, 0.25, 0.25],
                               rtol=1e-14)
