"""Pins of the joint multi-channel oracle (oracle/multichannel.py): for one
channel it is the paper's Eq. 6 fit reparameterised by Eq. 7; central
finite differences; exact recovery across channels with different beams;
MINPACK; Eq. 8 per channel; planted mistakes each pin must catch."""
import math

import numpy as np
import pytest
import scipy.optimize

import oracle as O
import oracle.multichannel as M


def _grid(H, W):
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    return xs.ravel(), ys.ravel()


def test_one_channel_is_eq6_reparameterised_by_eq7():
    """C = 1: the joint fit's optimum (x, y, s, a) is the circular fit's
    (a, x, y, omega_ic) with omega_ic^2 = s^2 + omega_b^2, and its model
    and Jacobian are the circular ones through that map."""
    H, W = 30, 32
    xs, ys = _grid(H, W)
    wb = 1.7
    truth = np.array([0.8, 15.3, 14.6, math.sqrt(2.4 ** 2 + wb ** 2)])
    T = O.gauss_model(truth, xs, ys) + np.random.default_rng(2).normal(0, 0.01, xs.size)
    start4 = truth * [0.9, 1.0, 1.0, 1.1]
    c = O.lm_fit(T, xs, ys, start4, (0, W - 1, 0, H - 1), 0.3, O.lm_exact())
    s0 = math.sqrt(start4[3] ** 2 - wb ** 2)
    m = M.mc_lm_fit(T, xs, ys, np.zeros(xs.size, int), [start4[1], start4[2], s0, start4[0]], (0, W - 1, 0, H - 1),
                    [wb * wb], O.lm_exact())
    x, y, s, a = m.theta
    assert a == pytest.approx(c.theta[0], rel=1e-8)
    assert x == pytest.approx(c.theta[1], abs=1e-8) and y == pytest.approx(c.theta[2], abs=1e-8)
    assert math.sqrt(s * s + wb * wb) == pytest.approx(c.theta[3], rel=1e-8)
    assert m.chi2 == pytest.approx(c.chi2, rel=1e-10)
    # model and Jacobian through the map
    th4 = np.array([a, x, y, math.sqrt(s * s + wb * wb)])
    m4, J4 = O.model_and_jacobian(th4, xs, ys)
    m1, J1 = M.mc_model_and_jacobian(m.theta, xs, ys, np.zeros(xs.size, int), [wb * wb])
    np.testing.assert_allclose(m1, m4, rtol=1e-12, atol=1e-300)
    np.testing.assert_allclose(J1[:, 3], J4[:, 0], rtol=1e-12, atol=1e-300)
    np.testing.assert_allclose(J1[:, 0], J4[:, 1], rtol=1e-12, atol=1e-300)
    np.testing.assert_allclose(J1[:, 2], J4[:, 3] * s / th4[3], rtol=1e-12, atol=1e-300)


def _stacked(C, H=24, W=26):
    xs, ys = _grid(H, W)
    return (np.concatenate([xs] * C), np.concatenate([ys] * C), np.repeat(np.arange(C), xs.size))


def test_jacobian_against_central_differences():
    wb2 = np.array([1.4, 1.9, 2.6]) ** 2
    X, Y, Ch = _stacked(3)
    th = np.array([11.3, 12.1, 2.2, 0.9, 0.7, 0.5,
                   14.6, 9.4, 0.8, -0.4, -0.3, -0.2])
    _, J = M.mc_model_and_jacobian(th, X, Y, Ch, wb2)
    for i in range(th.size):
        h = 1e-6 * max(1.0, abs(th[i]))
        tp, tm = th.copy(), th.copy()
        tp[i] += h
        tm[i] -= h
        fd = (M.mc_model(tp, X, Y, Ch, wb2) - M.mc_model(tm, X, Y, Ch, wb2)) / (2 * h)
        np.testing.assert_allclose(J[:, i], fd, rtol=1e-6, atol=1e-8 * np.max(np.abs(fd)) + 1e-12)


def _spectral(C, a0, alpha):
    nu = np.linspace(1.0, 2.0, C)
    return a0 * nu ** alpha


def test_lm_recovers_noiseless_members_across_channels():
    """Two members over four channels whose beams narrow with frequency and
    whose amplitudes follow power laws."""
    C = 4
    wb2 = (1.5 * 1.0 / np.linspace(1.0, 2.0, C) * 1.6) ** 2
    X, Y, Ch = _stacked(C, 30, 32)
    th = np.concatenate([[13.2, 14.7, 2.1, *_spectral(C, 0.9, -0.7)], [19.6, 16.3, 0.9, *_spectral(C, 0.5, 0.4)]])
    # the data channel by channel from the paper's circular model (Eq. 6
    # with the Eq. 7 width), independently of mc_model
    xs, ys = _grid(30, 32)
    T = np.concatenate([O.gauss_model(np.concatenate([[m[3 + c], m[0], m[1], math.sqrt(m[2] ** 2 + wb2[c])]
                                                      for m in th.reshape(2, -1)]), xs, ys) for c in range(C)])
    start = th.copy().reshape(2, -1)
    start[:, 0] += 0.3
    start[:, 1] -= 0.2
    start[:, 2] *= 1.2
    start[:, 3:] *= 0.9
    fit = M.mc_lm_fit(T, X, Y, Ch, start.ravel(), (0, 31, 0, 29), wb2, O.lm_exact())
    assert fit.status == O.LM_CONVERGED
    got = fit.theta.reshape(2, -1)
    got[:, 2] = np.abs(got[:, 2])   # s enters squared
    np.testing.assert_allclose(got.ravel(), th, rtol=1e-8, atol=1e-9)


def test_lm_matches_minpack_on_noisy_data():
    C = 3
    wb2 = np.array([1.8, 1.5, 1.3]) ** 2
    X, Y, Ch = _stacked(C, 28, 30)
    th = np.concatenate([[13.2, 12.7, 2.4, 0.8, 0.7, 0.6], [17.9, 15.8, 1.5, 0.4, 0.5, 0.6]])
    T = M.mc_model(th, X, Y, Ch, wb2) + np.random.default_rng(9).normal(0, 0.02, X.size)
    start = th * np.array([1.01, 0.99, 1.2, 0.9, 0.9, 0.9] * 2)
    fit = M.mc_lm_fit(T, X, Y, Ch, start, (0, 29, 0, 27), wb2, O.lm_exact())
    ref = scipy.optimize.least_squares(lambda p: M.mc_model(p, X, Y, Ch, wb2) - T, start,
                                       jac=lambda p: M.mc_model_and_jacobian(p, X, Y, Ch, wb2)[1],
                                       method="lm", xtol=1e-15, ftol=1e-15, gtol=1e-15, max_nfev=20000)
    got, want = fit.theta.reshape(2, -1).copy(), ref.x.reshape(2, -1).copy()
    got[:, 2], want[:, 2] = np.abs(got[:, 2]), np.abs(want[:, 2])
    np.testing.assert_allclose(got, want, rtol=1e-7, atol=1e-9)


def test_flux_per_channel_is_eq8():
    wb = np.array([1.6, 1.3])
    ab = np.array([0.9, 1.1])
    th = np.array([10.0, 11.0, 2.0, 0.8, 0.6])
    F, pt = M.mc_flux(th, ab, wb ** 2)
    for c in range(2):
        w_ic = math.sqrt(4.0 + wb[c] ** 2)
        Fc, _, wi, ptc = O.deconvolve(th[3 + c], w_ic, ab[c], wb[c])
        assert F[0, c] == pytest.approx(Fc, rel=1e-13) and wi == pytest.approx(2.0, rel=1e-12) and not ptc
    assert not pt[0]
    F, pt = M.mc_flux(np.array([10.0, 11.0, 0.01, 0.8, 0.6]), ab, wb ** 2)
    assert pt[0]


def test_window_and_stack():
    wb2 = np.array([1.5, 2.0]) ** 2
    th = np.array([10.2, 12.7, 1.0, 1.0, 1.0])
    box = M.mc_window(th, wb2, 40, 40)
    h = max(math.ceil(4 * math.sqrt(1.0 + 4.0)), 5)
    assert box == (10 - h, 10 + h, 13 - h, 13 + h)
    imgs = [np.arange(1600.0).reshape(40, 40), -np.arange(1600.0).reshape(40, 40)]
    T, X, Y, Ch = M.mc_stack(imgs, (2, 4, 5, 6))
    assert T.size == 2 * 6 and list(Ch) == [0] * 6 + [1] * 6
    assert T[0] == 5 * 40 + 2 and T[6] == -(5 * 40 + 2) and X[2] == 4 and Y[3] == 6


# ---------------------------------------------------------------- planted mistakes

def test_planted_linear_width_sum_is_caught(monkeypatch):
    orig = M.mc_model_and_jacobian

    def bad(theta, xs, ys, chan, wb2):
        # omega = s + omega_b instead of the quadrature sum of Eq. 7
        th = np.asarray(theta, float).reshape(-1, 3 + len(wb2)).copy()
        wb = np.sqrt(np.asarray(wb2, float))
        s_eff = th[:, 2:3] + wb[None, :]
        # the same model evaluated with omega^2 = (s + omega_b)^2 per channel
        out, J = orig(theta, xs, ys, chan, wb2)
        m = np.zeros(np.asarray(xs).size)
        ch = np.asarray(chan).ravel()
        for k in range(th.shape[0]):
            w2 = s_eff[k, ch] ** 2
            r2 = (np.asarray(xs).ravel() - th[k, 0]) ** 2 + (np.asarray(ys).ravel() - th[k, 1]) ** 2
            m += th[k, 3:][ch] * np.exp(-r2 / (2 * w2))
        return m, J

    monkeypatch.setattr(M, "mc_model_and_jacobian", bad)
    with pytest.raises(AssertionError):
        test_one_channel_is_eq6_reparameterised_by_eq7()


def test_planted_width_derivative_without_s_is_caught(monkeypatch):
    orig = M.mc_model_and_jacobian

    def bad(theta, xs, ys, chan, wb2):
        m, J = orig(theta, xs, ys, chan, wb2)
        th = np.asarray(theta, float).reshape(-1, 3 + len(wb2))
        J = J.copy()
        for k in range(th.shape[0]):
            J[:, (3 + len(wb2)) * k + 2] /= th[k, 2]      # dropped the factor s
        return m, J

    monkeypatch.setattr(M, "mc_model_and_jacobian", bad)
    with pytest.raises(AssertionError):
        test_jacobian_against_central_differences()


def test_planted_amplitudes_in_the_wrong_channel_are_caught(monkeypatch):
    orig = M.mc_model_and_jacobian

    def bad(theta, xs, ys, chan, wb2):
        C = len(wb2)
        return orig(theta, xs, ys, (np.asarray(chan) + 1) % C, wb2)

    monkeypatch.setattr(M, "mc_model_and_jacobian", bad)
    with pytest.raises(AssertionError):
        test_lm_recovers_noiseless_members_across_channels()


# ---------------------------------------------------------------- trial test and xtol scales

def test_trial_test_hand_cases():
    wb2 = np.array([1.5, 2.0]) ** 2            # widest beam 2.0
    box = (10, 29, 5, 20)                      # extent max(20, 16) = 20
    ok = np.array([15.0, 12.0, 1.0, 0.5, 0.4])
    assert M.mc_valid(ok, box, wb2)
    assert M.mc_valid(np.array([15.0, 12.0, 0.0, 0.5, 0.4]), box, wb2)          # a point (s = 0)
    assert M.mc_valid(np.array([10.0, 20.0, 1.0, 0.5, 0.4]), box, wb2)          # centre on the box edge
    assert not M.mc_valid(np.array([9.99, 12.0, 1.0, 0.5, 0.4]), box, wb2)      # centre outside
    assert not M.mc_valid(np.array([15.0, 20.01, 1.0, 0.5, 0.4]), box, wb2)
    s_edge = math.sqrt(20.0 ** 2 - 4.0)                                          # s^2 + 4 = 20^2
    assert M.mc_valid(np.array([15.0, 12.0, s_edge, 0.5, 0.4]), box, wb2)
    assert not M.mc_valid(np.array([15.0, 12.0, s_edge * (1 + 1e-9), 0.5, 0.4]), box, wb2)
    assert not M.mc_valid(np.array([15.0, 12.0, np.nan, 0.5, 0.4]), box, wb2)


def test_xtol_scales_hand_values():
    wb2 = np.array([1.5, 2.0]) ** 2
    th = np.array([15.0, 12.0, 1.5, -0.5, 0.0])
    w = math.sqrt(1.5 ** 2 + 4.0)
    np.testing.assert_allclose(M.mc_step_scale(th, wb2), [w, w, w, 0.5, 1.0], rtol=1e-15)
