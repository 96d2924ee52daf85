"""Asp-Clean2004's objective (Sect. 2, Eq. 3: the full PSF inside chi^2,
applied by an FFT convolution in every evaluation) on the GPU
(asp_fit_2004) against the FP64 oracle (lm_fit_2004), and the identity that
makes the paper's Eq. 6 possible: with a Gaussian PSF the Eq. 3 optimum maps
to the Eq. 6 optimum through Eqs. 7-8."""
import math

import numpy as np
import pytest

import oracle as O
import synth

pytestmark = pytest.mark.gpu

TIGHT = dict(lm_max_iter=300, lm_rtol=1e-12, lm_xtol=1e-10)


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _close(g, o, rtol=1e-4):
    for gi, oi in zip(np.asarray(g).reshape(-1, 4), np.asarray(o).reshape(-1, 4)):
        a, x, y, w = oi
        assert abs(gi[0] - a) <= rtol * abs(a), (gi, oi)
        assert abs(gi[1] - x) <= rtol * max(1.0, w), (gi, oi)
        assert abs(gi[2] - y) <= rtol * max(1.0, w), (gi, oi)
        assert abs(gi[3] - w) <= rtol * w, (gi, oi)


def _field(H, W, truth, noise, seed, psf):
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    img = O.gauss_model(np.asarray(truth, float).ravel(), xs, ys)
    return (O.psf_convolve(psf, img) + np.random.default_rng(seed).normal(0, noise, (H, W))).astype(np.float32)


@pytest.mark.parametrize("truth,start,n_old", [
    ([[0.6, 24.3, 21.7, 2.5]], [[0.5, 24.0, 22.0, 3.0]], 0),
    ([[0.5, 20.3, 22.1, 2.0], [-0.3, 27.6, 19.4, 3.2]], [[0.45, 20.0, 22.5, 2.3], [-0.3, 27.6, 19.4, 3.2]], 1),
])
def test_fit_2004_matches_oracle(asp, truth, start, n_old):
    H, W = 44, 48
    psf = synth.small_case(H, W, seed=7, psf_sigma=1.6).psf.astype(np.float64)
    dirty = _field(H, W, truth, 2e-2, 3, psf)
    ctx = asp.Context(_t(dirty), _t(psf), noise_sigma=2e-2, k_max=4, **TIGHT)
    start = np.asarray(start, float)
    out, info = ctx.fit_2004(start, n_old, 0.1)
    # the oracle: T = R + B * (the added-back members' start components)
    T = dirty.astype(np.float64)
    if n_old:
        ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
        T = T + O.psf_convolve(psf, O.gauss_model(start[-n_old:].ravel(), xs, ys))
    ref = O.lm_fit_2004(T, psf, start.ravel(), 0.1, O.lm_exact())
    assert info["status"] != O.LM_CAP and ref.status != O.LM_CAP
    _close(out, ref.theta)
    assert info["chi2_final"] == pytest.approx(ref.chi2, rel=1e-4)
    assert info["pixel_evals"] == info["passes"] * H * W
    ctx.close()


def test_eq3_optimum_maps_to_eq6_optimum_on_the_gpu(asp):
    """The GPU's Eq. 3 fit through a Gaussian PSF and its Eq. 6 fit of the
    same data obey Eq. 7 and Eq. 8 (the Sect. 3 closed form)."""
    H, W = 48, 52
    ab, wb = 0.9, 1.8
    psf = synth.gaussian_psf(H, W, wb, ab)
    # near-noiseless: the Eq. 6 fit sees its member window, the Eq. 3 fit the
    # whole image, so only the noise-free optimum is the same point
    dirty = _field(H, W, [[0.7, 25.3, 23.6, 2.6]], 1e-6, 5, psf)
    ctx = asp.Context(_t(dirty), _t(psf), noise_sigma=1e-6, k_max=2, **TIGHT)
    (a, x, y, w), = ctx.fit_2004([[0.6, 25.0, 24.0, 3.0]], 0, 0.1)[0]
    (a_ic, x_ic, y_ic, w_ic), = ctx.fit([[6.0, 25.0, 24.0, 3.3]], 0)[0]
    assert w_ic ** 2 == pytest.approx(w * w + wb * wb, rel=1e-4)
    assert a_ic == pytest.approx(2 * math.pi * a * ab * w * w * wb * wb / (w * w + wb * wb), rel=1e-4)
    assert abs(x - x_ic) < 1e-4 * w_ic and abs(y - y_ic) < 1e-4 * w_ic
    ctx.close()


def test_fit_2004_rejects_large_active_sets(asp):
    case = synth.small_case(32, 32, seed=0)
    ctx = asp.Context(_t(case.dirty), _t(case.psf), noise_sigma=1e-3, k_max=12)
    with pytest.raises(asp.AspError) as e:
        ctx.fit_2004([[0.1, 10.0 + k, 12.0, 2.0] for k in range(9)], 0)
    assert e.value.status == 8
    ctx.close()
