"""Joint wide-band fit over a batch's images as channels (asp_batch_fit_joint;
oracle/multichannel.py states the reading) against the FP64 oracle:
converged fits within 1e-4 of each parameter's scale, Eq. 8 per channel,
and the one-channel case against the paper's Eq. 6 fit through Eq. 7."""
import math

import numpy as np
import pytest

import oracle as O
import oracle.multichannel as M
import synth

pytestmark = pytest.mark.gpu

TIGHT = dict(lm_max_iter=300, lm_rtol=1e-12, lm_xtol=1e-10)


def _channels(H, W, members, sigmas, noise, seed):
    """Dirty images of one field in len(sigmas) channels: member (x, y, s,
    a_1 .. a_C) is the Gaussian of width sqrt(s^2 + sigma_c^2) in channel c
    (a Gaussian PSF of width sigma_c), plus noise."""
    dirty, psf = [], []
    for c, sg in enumerate(sigmas):
        src = [(m[3 + c], m[0], m[1], math.hypot(m[2], sg), math.hypot(m[2], sg), 0.0) for m in members]
        dirty.append(synth.elliptical_field(H, W, src, noise, seed + c).astype(np.float32))
        psf.append(synth.gaussian_psf(H, W, sg).astype(np.float32))
    return dirty, psf


def _oracle(b, dirty, init, n_old=0):
    beams = [b.image(c).beam for c in range(b.n)]
    wb2 = np.array([bm[1] ** 2 for bm in beams])
    ab = np.array([bm[0] for bm in beams])
    H, W = dirty[0].shape
    box = M.mc_window(np.asarray(init, float).ravel(), wb2, H, W)
    T, xs, ys, ch = M.mc_stack([d.astype(np.float64) for d in dirty], box)
    if n_old:
        T = T + M.mc_model(np.asarray(init[-n_old:], float).ravel(), xs, ys, ch, wb2)
    fit = M.mc_lm_fit(T, xs, ys, ch, np.asarray(init, float).ravel(), box, wb2, O.lm_exact())
    return fit, box, wb2, ab


def _close(g, o, wb2, rtol=1e-4):
    g, o = np.asarray(g, float).reshape(-1, 3 + wb2.size).copy(), np.asarray(o, float).reshape(-1, 3 + wb2.size).copy()
    g[:, 2], o[:, 2] = np.abs(g[:, 2]), np.abs(o[:, 2])   # s enters squared
    err = np.abs(g - o).ravel() / M.mc_step_scale(o.ravel(), wb2)
    assert np.all(err <= rtol), (err.max(), g, o)


@pytest.mark.parametrize("C,members,n_old", [
    (4, [[38.3, 41.6, 2.2, 0.9, 0.8, 0.7, 0.6]], 0),
    (4, [[36.2, 40.1, 1.4, 0.8, 0.85, 0.9, 0.95], [44.7, 43.3, 2.6, -0.5, -0.45, -0.4, -0.35]], 0),
    (3, [[35.5, 38.4, 1.8, 0.7, 0.6, 0.5], [43.3, 45.2, 0.6, 0.4, 0.5, 0.6]], 1),
])
def test_joint_fit_matches_oracle(asp, C, members, n_old):
    H, W = 80, 88
    sigmas = 1.6 / np.linspace(1.0, 1.6, C)
    dirty, psf = _channels(H, W, members, sigmas, 5e-3, 3)
    b = asp.Batch(dirty, psf, noise_sigma=5e-3, k_max=5, **TIGHT)
    init = np.array(members, float)
    init[:, 0] += 0.4
    init[:, 1] -= 0.3
    init[:, 2] *= 1.2
    init[:, 3:] *= 0.9
    out, flux, pt, info = b.fit_joint(init, n_old)
    ref, box, wb2, ab = _oracle(b, dirty, init, n_old)
    assert info["status"] != O.LM_CAP and ref.status != O.LM_CAP
    assert (info["x0"], info["x1"], info["y0"], info["y1"]) == box
    _close(out, ref.theta, wb2)
    assert info["chi2_final"] == pytest.approx(ref.chi2, rel=1e-4)
    F, P = M.mc_flux(out.ravel(), ab, wb2)
    np.testing.assert_allclose(flux, F, rtol=1e-12)
    assert list(pt) == list(P)
    b.close()


def test_one_channel_joint_fit_is_the_circular_fit_through_eq7(asp):
    H, W = 64, 72
    dirty, psf = _channels(H, W, [[33.4, 30.8, 2.3, 0.8]], [1.7], 5e-3, 8)
    b = asp.Batch(dirty, psf, noise_sigma=5e-3, k_max=3, **TIGHT)
    ab, wb, _, _ = b.image(0).beam
    out, flux, pt, info = b.fit_joint([[33.0, 31.0, 2.0, 0.7]], 0)
    (a, x, y, w), = b.image(0).fit([[0.7, 33.0, 31.0, math.hypot(2.0, wb)]], 0)[0]
    xj, yj, sj, aj = out[0]
    assert aj == pytest.approx(a, rel=1e-4)
    assert abs(xj - x) < 1e-4 * w and abs(yj - y) < 1e-4 * w
    assert math.hypot(sj, wb) == pytest.approx(w, rel=1e-4)
    Fc, _, wi, _ = O.deconvolve(a, w, ab, wb)
    assert flux[0, 0] == pytest.approx(Fc, rel=1e-4)
    b.close()


def test_joint_fit_over_sixteen_channels_spans_several_ctas(asp):
    H, W = 128, 136
    C = 16
    rng = np.random.default_rng(6)
    members = [[rng.uniform(45, 90), rng.uniform(45, 85), rng.uniform(1.0, 3.0),
                *(rng.uniform(0.4, 1.0) * np.linspace(1.0, 2.0, C) ** rng.uniform(-1, 1))] for _ in range(3)]
    sigmas = 1.8 / np.linspace(1.0, 1.8, C)
    dirty, psf = _channels(H, W, members, sigmas, 5e-3, 21)
    b = asp.Batch(dirty, psf, noise_sigma=5e-3, k_max=5, **TIGHT)
    init = np.array(members, float) * np.array([1.0, 1.0, 1.15] + [0.92] * C)
    out, flux, pt, info = b.fit_joint(init, 0)
    ref, box, wb2, ab = _oracle(b, dirty, init)
    assert info["status"] != O.LM_CAP and ref.status != O.LM_CAP
    _close(out, ref.theta, wb2)
    b.close()


def test_joint_fit_arguments_checked(asp):
    d1, p1 = _channels(40, 40, [[20.0, 20.0, 1.0, 0.5]], [1.5], 1e-3, 0)
    d2, p2 = _channels(40, 44, [[20.0, 20.0, 1.0, 0.5]], [1.5], 1e-3, 1)
    b = asp.Batch(d1 + d2, p1 + p2, noise_sigma=1e-3, k_max=3)
    with pytest.raises(asp.AspError) as e:
        b.fit_joint([[20.0, 20.0, 1.0, 0.5, 0.5]], 0)     # channels of different sizes
    assert e.value.status == 8
    b.close()
    dirty, psf = _channels(40, 40, [[20.0, 20.0, 1.0] + [0.5] * 8], [1.5] * 8, 1e-3, 0)
    b = asp.Batch(dirty, psf, noise_sigma=1e-3, k_max=3)
    with pytest.raises(asp.AspError) as e:
        b.fit_joint([[20.0, 20.0, 1.0] + [0.5] * 8] * 19, 0)   # 19 x 11 > 200 parameters
    assert e.value.status == 8
    b.close()
