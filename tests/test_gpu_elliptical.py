"""The elliptical variant (the paper's circular Gaussians of Sect. 3 with a
2 x 2 shape; oracle/elliptical.py states the readings) on the GPU against
the FP64 oracle: converged fits within 1e-4 of each parameter's scale, the
elliptical beam, Eqs. 7-8 for ellipses, and the circular case."""
import math

import numpy as np
import pytest

import oracle as O
import oracle.elliptical as E
import synth

pytestmark = pytest.mark.gpu

TIGHT = dict(lm_max_iter=300, lm_rtol=1e-12, lm_xtol=1e-10)


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _rows(src):
    return np.array([[a, x, y, *E.precision_from_axes(s1, s2, p)] for a, x, y, s1, s2, p in src])


def _scales(th):
    return E.ell_step_scale(np.asarray(th, float).ravel())


def _close(g, o, rtol=1e-4):
    g, o = np.asarray(g, float).ravel(), np.asarray(o, float).ravel()
    err = np.abs(g - o) / _scales(o)
    assert np.all(err <= rtol), (err.max(), g, o)


def _window(init, H, W):
    b = np.array([E.ell_member_box(r[1], r[2], r[3], r[4], r[5]) for r in init])
    return max(b[:, 0].min(), 0), min(b[:, 1].max(), W - 1), max(b[:, 2].min(), 0), min(b[:, 3].max(), H - 1)


def _oracle_fit(dirty, init, n_old, wb):
    H, W = dirty.shape
    x0, x1, y0, y1 = _window(init, H, W)
    ys, xs = np.mgrid[y0:y1 + 1, x0:x1 + 1].astype(np.float64)
    T = dirty[y0:y1 + 1, x0:x1 + 1].astype(np.float64)
    if n_old:
        T = T + E.ell_model(np.asarray(init[-n_old:], float).ravel(), xs, ys)
    return E.ell_lm_fit(T.ravel(), xs.ravel(), ys.ravel(), np.asarray(init, float).ravel(), (x0, x1, y0, y1),
                        0.25 * wb, O.lm_exact())


CASES = [
    ([(0.9, 30.3, 27.6, 4.0, 1.8, 0.5)], 0),
    ([(0.8, 26.2, 28.1, 3.0, 1.8, -0.4), (-0.5, 33.7, 31.3, 2.6, 2.0, 1.1)], 0),
    ([(0.7, 24.5, 24.4, 2.8, 1.6, 0.2), (0.6, 33.3, 26.2, 2.4, 1.7, 1.3), (0.4, 28.6, 35.1, 3.4, 2.9, -0.9)], 1),
]


@pytest.mark.parametrize("src,n_old", CASES)
def test_fit_elliptical_matches_oracle(asp, src, n_old):
    H, W = 60, 64
    case = synth.small_case(H, W, seed=2)
    dirty = synth.elliptical_field(H, W, src, 1e-2, 7).astype(np.float32)
    ctx = asp.Context(_t(dirty), _t(case.psf), noise_sigma=1e-2, k_max=5, **TIGHT)
    _, wb, _, _ = ctx.beam
    truth = _rows(src)
    init = truth * np.array([0.9, 1.0, 1.0, 1.1, 0.85, 0.9])
    init[:, 1] += 0.4
    init[:, 2] -= 0.3
    out, info = ctx.fit_elliptical(init, n_old)
    ref = _oracle_fit(dirty, init, n_old, wb)
    assert info["status"] != O.LM_CAP and ref.status != O.LM_CAP
    _close(out, ref.theta)
    assert info["chi2_final"] == pytest.approx(ref.chi2, rel=1e-4)
    assert (info["x0"], info["x1"], info["y0"], info["y1"]) == _window(init, H, W)
    ctx.close()


def test_elliptical_fit_of_a_circle_is_the_circular_fit(asp):
    H, W = 56, 60
    case = synth.small_case(H, W, seed=3)
    dirty = synth.elliptical_field(H, W, [(0.8, 28.3, 27.6, 2.7, 2.7, 0.0)], 5e-3, 9).astype(np.float32)
    ctx = asp.Context(_t(dirty), _t(case.psf), noise_sigma=5e-3, k_max=3, **TIGHT)
    (a, x, y, w), = ctx.fit([[0.7, 28.0, 28.0, 3.0]], 0)[0]
    (ea, ex, ey, A, B, C), = ctx.fit_elliptical([[0.7, 28.0, 28.0, 1 / 9.0, 0.0, 1 / 9.0]], 0)[0]
    assert abs(B) < 0.02 / w ** 2
    assert A == pytest.approx(1 / w ** 2, rel=0.02) and C == pytest.approx(1 / w ** 2, rel=0.02)
    assert ex == pytest.approx(x, abs=0.01) and ey == pytest.approx(y, abs=0.01)
    ctx.close()


def test_large_window_elliptical_fit_spans_several_ctas(asp):
    """12 members (72 parameters) over a window of several CTAs."""
    H, W = 160, 168
    rng = np.random.default_rng(4)
    src = [(rng.uniform(0.3, 1.0) * rng.choice([-1, 1]), rng.uniform(30, 138), rng.uniform(30, 130),
            rng.uniform(3.0, 6.0), rng.uniform(1.5, 2.9), rng.uniform(-1.5, 1.5)) for _ in range(12)]
    case = synth.small_case(H, W, seed=5)
    dirty = synth.elliptical_field(H, W, src, 1e-2, 11).astype(np.float32)
    ctx = asp.Context(_t(dirty), _t(case.psf), noise_sigma=1e-2, k_max=20, **TIGHT)
    _, wb, _, _ = ctx.beam
    init = _rows(src) * np.array([0.95, 1.0, 1.0, 1.05, 0.95, 0.95])
    out, info = ctx.fit_elliptical(init, 0)
    ref = _oracle_fit(dirty, init, 0, wb)
    assert info["status"] != O.LM_CAP and ref.status != O.LM_CAP
    _close(out, ref.theta)
    ctx.close()


@pytest.mark.parametrize("psf_kind", ["gaussian", "ringed"])
def test_elliptical_beam_matches_oracle(asp, psf_kind):
    H, W = 48, 52
    ring = 12.0 if psf_kind == "ringed" else None
    psf = synth.elliptical_psf(H, W, 2.6, 1.5, 0.5, 1.0, ring)
    dirty = np.random.default_rng(1).normal(0, 1e-3, (H, W))
    ctx = asp.Context(_t(dirty), _t(psf), noise_sigma=1e-3, k_max=2, **TIGHT)
    b = ctx.beam_elliptical()
    ref, fit = E.ell_beam_fit(psf.astype(np.float32).astype(np.float64), O.lm_exact())
    _close(b, ref)
    if psf_kind == "gaussian":
        _close(b, [1.0, W, H, *E.precision_from_axes(2.6, 1.5, 0.5)])
    ctx.close()


def test_deconvolve_elliptical_matches_oracle(asp):
    case = synth.small_case(32, 32, seed=0)
    ctx = asp.Context(_t(case.dirty), _t(case.psf), noise_sigma=1e-3)
    beam = np.array([0.9, 32.0, 32.0, *E.precision_from_axes(2.1, 1.4, 0.3)])
    Pb = np.array([[beam[3], beam[4]], [beam[4], beam[5]]])
    rows = []
    for a_i, s1, s2, p in ((0.7, 2.6, 1.1, 0.4), (1.5, 1.4, 1.3, -0.2), (0.3, 3.3, 0.9, 1.2)):
        P_i = np.array(E.precision_from_axes(s1, s2, p))
        a_ic, P_ic = E.ell_convolve_shape(a_i, np.array([[P_i[0], P_i[1]], [P_i[1], P_i[2]]]), beam[0], Pb)
        rows.append([a_ic, 10.0, 11.0, P_ic[0, 0], P_ic[0, 1], P_ic[1, 1]])
    rows.append([0.5, 3.0, 4.0, beam[3], beam[4], beam[5]])          # the beam itself: a point
    out = ctx.deconvolve_elliptical(rows, beam)
    for r, o in zip(rows, out):
        F, a_i, S_i, pt = E.ell_deconvolve(r[0], np.array([[r[3], r[4]], [r[4], r[5]]]), beam[0], Pb)
        assert bool(o[7]) == pt
        assert o[0] == pytest.approx(F, rel=1e-10) and o[1] == pytest.approx(a_i, rel=1e-10)
        np.testing.assert_allclose(o[4:7], [S_i[0, 0], S_i[0, 1], S_i[1, 1]], rtol=1e-9, atol=1e-12)
    ctx.close()


def test_elliptical_arguments_checked(asp):
    case = synth.small_case(32, 32, seed=0)
    ctx = asp.Context(_t(case.dirty), _t(case.psf), noise_sigma=1e-3, k_max=5)
    with pytest.raises(asp.AspError) as e:
        ctx.fit_elliptical([[1.0, 16.0, 16.0, 0.1, 0.2, 0.1]], 0)   # B^2 > A C
    assert e.value.status == 1
    with pytest.raises(asp.AspError) as e:
        ctx.fit_elliptical([[0.1, 16.0, 16.0, 0.2, 0.0, 0.2]] * (asp.ASP_ELL_KMAX + 1), 0)
    assert e.value.status == 8
    ctx.close()
