"""The minor/major split (asp_params.major_every > 0, in the manner of Clark
CLEAN: the paper's Sect. 1 and Sect. 3 comparison) against the FP64 oracle.

* the minor cycle's beam-image subtraction (asp_subtract_beam) equals the
  oracle's, 1e-5 relative L2;
* every major cycle makes the residual exact: after a call, R - D equals the
  oracle's full-PSF subtraction of the GPU's own component list, 1e-5
  relative L2 (FFT convolution on the GPU, separable direct sums in FP64);
* the runs: with a major cycle after every iteration the split takes the
  exact cycle's decisions; a split run to the noise threshold reaches the
  oracle split run's residual RMS and model flux.
"""
import numpy as np
import pytest

import oracle as O
import synth
from tests import teacher

pytestmark = pytest.mark.gpu


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, float) - np.asarray(b, float)) / max(np.linalg.norm(b), 1e-300))


def _terms(comps, H, W):
    ts = [O.component_terms(c[0], c[2], c[3], c[4], bool(c[5]), H, W) for c in comps]
    return [t for t in ts if t is not None]


@pytest.mark.parametrize("H,W", [(64, 72), (257, 240)])
def test_beam_subtraction_matches_oracle(asp, H, W):
    case = synth.small_case(H, W, seed=3)
    ctx = asp.Context(_t(case.dirty), _t(case.psf), noise_sigma=case.noise_sigma, k_max=4, major_every=5)
    ab, wb, _, _ = ctx.beam
    rng = np.random.default_rng(H)
    comps = []
    for w in (0.0, 0.3, 1.7, 5.2, 11.0):
        comps.append([rng.normal(), 0.0, rng.uniform(2, W - 3), rng.uniform(2, H - 3), w, int(w == 0.0)])
    gain = 0.6
    ctx.subtract_beam(comps, gain)
    ref = O.subtract_beam_images(case.dirty, [(gain * c[0], c[2], c[3], c[4]) for c in comps], ab, wb)
    d_gpu = ctx.residual().astype(np.float64) - case.dirty
    assert _rel_l2(d_gpu, ref - case.dirty) < 1e-5
    pk = ctx.find_peak(asp.ASP_PEAK_SIMPLE)
    assert pk["index"] == O.peak_simple(ctx.residual())[0]
    ctx.close()


def test_major_cycle_makes_the_residual_exact(asp):
    case = synth.small_case(96, 104, seed=11, n_points=3, n_gauss=2, sigma_range=(2.5, 6))
    ctx = asp.Context(_t(case.dirty), _t(case.psf), noise_sigma=case.noise_sigma, k_max=3, major_every=4)
    for calls in (4, 6, 1):                      # a full block, a block and a half, a single iteration
        ctx.minor_cycle(calls)
        comps = ctx.components()
        ref = O.subtract_terms(case.dirty, case.psf, _terms(comps, case.H, case.W))
        R = ctx.residual().astype(np.float64)
        assert _rel_l2(R - case.dirty, ref - case.dirty) < 1e-5
    st = ctx.stats()
    assert st["iterations"] == 11
    ctx.close()


def test_major_cycle_exact_at_full_size(asp):
    """The 1024^2 workload: after 40 iterations with a major cycle every 20
    the residual matches the brute-force direct subtraction of the GPU's
    components at sampled pixels."""
    case = synth.config2(0)
    ctx = asp.Context(_t(case.dirty), _t(case.psf), noise_sigma=case.noise_sigma, k_max=case.k_max,
                      major_every=20)
    ctx.minor_cycle(40)
    comps = ctx.components()
    terms = _terms(comps, case.H, case.W)
    rng = np.random.default_rng(9)
    py = np.concatenate([rng.integers(0, case.H, 200), comps[:20, 3].round().astype(int).clip(0, case.H - 1)])
    px = np.concatenate([rng.integers(0, case.W, 200), comps[:20, 2].round().astype(int).clip(0, case.W - 1)])
    d_ref = -teacher.subtraction_at(case.psf.astype(np.float64), terms, case.H, case.W, py, px)
    d_gpu = ctx.residual().astype(np.float64)[py, px] - case.dirty[py, px]
    assert _rel_l2(d_gpu, d_ref) < 1e-5
    ctx.close()


def test_major_every_iteration_takes_the_exact_cycles_decisions(asp):
    case = synth.small_case(96, 104, seed=12, n_points=3, n_gauss=2, sigma_range=(2.5, 6))
    kw = dict(noise_sigma=case.noise_sigma, k_max=3)
    a = asp.Context(_t(case.dirty), _t(case.psf), **kw)
    b = asp.Context(_t(case.dirty), _t(case.psf), major_every=1, **kw)
    a.minor_cycle(10)
    b.minor_cycle(10)
    ha, hb = a.history(), b.history()
    for x, y in zip(ha, hb):
        assert (x["mode"], x["k"], x["x0"], x["x1"], x["y0"], x["y1"]) == \
               (y["mode"], y["k"], y["x0"], y["x1"], y["y0"], y["y1"])
    np.testing.assert_allclose(a.components()[:, 0], b.components()[:, 0], rtol=1e-4)
    a.close()
    b.close()


def test_split_run_to_noise_matches_oracle(asp):
    case = synth.small_case(72, 80, seed=21, n_points=3, n_gauss=1, sigma_range=(2.0, 3.0), noise_sigma=1e-3)
    ctx = asp.Context(_t(case.dirty), _t(case.psf), noise_sigma=case.noise_sigma, k_max=3, major_every=5)
    st = ctx.minor_cycle(400)
    ab, wb, _, _ = ctx.beam
    mc = O.MinorCycle(case.dirty, case.psf, O.AspParams(k_max=3, noise_sigma=case.noise_sigma, major_every=5),
                      beam=(ab, wb)).run(400)
    R = ctx.residual().astype(np.float64)
    assert st["stop_reason"] == asp.ASP_STOP_NOISE and mc.stopped
    assert np.sqrt(np.mean(R ** 2)) == pytest.approx(np.sqrt(np.mean(mc.R ** 2)), rel=0.05)
    assert ctx.components()[:, 0].sum() == pytest.approx(mc.stats()["model_flux"], rel=0.01)
    assert ctx.components()[:, 0].sum() == pytest.approx(case.sky.sum(), rel=0.05)
    ctx.close()


def test_batches_reject_the_split(asp):
    c = synth.config4(1, sizes=(64,))
    with pytest.raises(asp.AspError) as e:
        asp.Batch([c.dirty], [c.psf], major_every=3)
    assert e.value.status == 8
