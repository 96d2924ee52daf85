"""Parity of the CUDA path (through the C-ABI) with the FP64 oracle.

Tolerances (spec bar): model/residual images 1e-5 relative L2 (of the
subtracted or smoothed part, which is stricter than of the whole image);
fitted amplitude, centre and width 1e-4 relative (centres |dx| <= 1e-4
max(1, w)); peak indices bit-exact on identical FP32 input.  Normal-equation
sums are held to the FP32 summation bound (64 + log2 Wn + 16) u32 sum|terms|.
"""
import numpy as np
import pytest

import oracle as O
import synth
from tests import fp32_bounds as FB
from tests import teacher

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _ctx(asp, case, **kw):
    kw.setdefault("noise_sigma", case.noise_sigma)
    kw.setdefault("k_max", case.k_max)
    return asp.Context(_t(case.dirty), _t(case.psf), **kw)


def _rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, float) - np.asarray(b, float)) / max(np.linalg.norm(b), 1e-300))


def _param_close(g, o, rtol=1e-4):
    a, x, y, w = o
    assert abs(g[0] - a) <= rtol * abs(a), (g, o)
    assert abs(g[1] - x) <= rtol * max(1.0, w), (g, o)
    assert abs(g[2] - y) <= rtol * max(1.0, w), (g, o)
    assert abs(g[3] - w) <= rtol * w, (g, o)


# ----------------------------------------------------------------- beam (a1)

@pytest.mark.parametrize("maker", ["config1", "small_gauss", "config2_small"])
def test_beam_fit_matches_oracle(asp, maker):
    if maker == "config1":
        case = synth.config1(0)
    elif maker == "small_gauss":
        case = synth.small_case(40, 48, seed=2, psf_sigma=2.3, ring=False)
    else:
        case = synth.config2(0, size=256)
    ctx = _ctx(asp, case)
    ab, wb, xb, yb = ctx.beam
    oab, owb, fit = O.beam_fit(case.psf, O.lm_exact())     # the optimum itself
    _param_close([ab, xb, yb, wb], [oab, fit.theta[1], fit.theta[2], owb])
    if maker == "config1":
        assert ab == pytest.approx(1.0, abs=2e-6) and wb == pytest.approx(1.5, abs=2e-6)
    ctx.close()


# ----------------------------------------------------------------- peak (a2)

@pytest.mark.parametrize("H,W", [(3, 5), (17, 13), (64, 64), (131, 257), (512, 640)])
def test_argmax_bit_exact(asp, H, W):
    rng = np.random.default_rng(H * 1000 + W)
    psf = synth.gaussian_psf(H, W, 1.5)
    ctx = asp.Context(_t(rng.normal(size=(H, W))), _t(psf), noise_sigma=1.0)
    for trial in range(4):
        if trial == 0:
            R = rng.normal(size=(H, W)).astype(np.float32)
        elif trial == 1:
            R = rng.integers(-3, 4, size=(H, W)).astype(np.float32)     # many ties, +/- equal |v|
        elif trial == 2:
            R = np.zeros((H, W), np.float32)
            R.flat[rng.integers(0, H * W, 3)] = -2.5
        else:
            R = np.zeros((H, W), np.float32)                              # all equal: index 0
        ctx.set_residual(_t(R))
        pk = ctx.find_peak(asp.ASP_PEAK_SIMPLE)
        idx, val = O.peak_simple(R)
        assert pk["index"] == idx and pk["value"] == np.float32(val)
        assert (pk["x"], pk["y"]) == (idx % W, idx // W)
    ctx.close()


def test_degenerate_one_pixel_image_is_an_error(asp):
    """A 1x1 image has no PSF main lobe to fit: the beam fit reports it."""
    with pytest.raises(asp.AspError):
        asp.Context(_t(np.ones((1, 1))), _t(synth.gaussian_psf(1, 1, 1.5)), noise_sigma=1.0)


# ----------------------------------------------------------------- subtraction (a9)

@pytest.mark.parametrize("sub_mode", ["direct", "fft"])
@pytest.mark.parametrize("H,W,seed", [(48, 40, 0), (97, 131, 1), (256, 256, 2)])
def test_subtraction_matches_oracle(asp, H, W, seed, sub_mode):
    """Both forms of the residual update (direct separable passes; one FFT
    product of the change image) against the oracle's direct sums.  A
    second update elsewhere checks that the FFT form's change image holds
    only the current terms (the previous box is cleared)."""
    case = synth.small_case(H, W, seed=seed)
    rng = np.random.default_rng(seed)
    mode = asp.ASP_SUB_FFT if sub_mode == "fft" else asp.ASP_SUB_DIRECT
    ctx = _ctx(asp, case, k_max=k_max, sub_mode=mode)
    R0 = case.dirty.astype(np.float64)
    for rnd in range(2):
        comps = []
        for i in range(6):
            w = [0.0, 0.3, 1.4, 4.7, 9.0, 0.8][(i + 3 * rnd) % 6]
            comps.append([rng.normal(), 0.0, rng.uniform(-3, W + 2), rng.uniform(-3, H + 2), w, int(w == 0.0)])
        gain = 0.7
        ctx.subtract(comps, gain)
        R = ctx.residual().astype(np.float64)
        terms = [O.component_terms(gain * c[0], c[2], c[3], c[4], bool(c[5]), H, W) for c in comps]
        ref = O.subtract_terms(R0, case.psf, [t for t in terms if t is not None])
        d_gpu, d_ref = R - R0, ref - R0
        assert _rel_l2(d_gpu, d_ref) < 1e-5, rnd
        assert _rel_l2(R, ref) < 1e-5, rnd
        pk = ctx.find_peak(asp.ASP_PEAK_SIMPLE)
        idx, _ = O.peak_simple(ctx.residual())
        assert pk["index"] == idx
        R0 = R
    ctx.close()


def test_fft_update_is_the_default_from_its_size(asp):
    """sub_mode AUTO takes the FFT form from ASP_SUB_FFT_MIN_PIXELS pixels:
    a run's launches show which form ran."""
    for H, W, fft in ((256, 256, False), (512, 512, True)):
        case = synth.small_case(H, W, seed=4)
        ctx = _ctx(asp, case, k_max=3)
        ctx.set_profiling(True)
        ctx.minor_cycle(2)
        prof = {k["name"]: k for k in ctx.kernel_times()}
        assert (prof["subtraction (FFT)"]["launches"] > 0) == fft
        assert (prof["k_sub_v_argmax"]["launches"] > 0) == (not fft)
        ctx.close()


def test_subtraction_gaussian_psf_closed_form(asp):
    H = W = 64
    ab, wb = 0.9, 1.6
    psf = synth.gaussian_psf(H, W, wb, ab)
    ctx = asp.Context(_t(np.zeros((H, W))), _t(psf), noise_sigma=1e-3)
    F, wi, x, y = 3.0, 2.5, 31.4, 30.7
    ctx.subtract([[F, 0.0, x, y, wi, 0]], 1.0)
    out = -ctx.residual().astype(np.float64)
    a_ic, w_ic = O.gauss_approx(F, wi, ab, wb)
    ys, xs = np.mgrid[0:H, 0:W]
    expect = a_ic * np.exp(-((xs - x) ** 2 + (ys - y) ** 2) / (2 * w_ic ** 2))
    assert np.max(np.abs(out - expect)) < 1e-4 * abs(a_ic)
    ctx.close()


# ----------------------------------------------------------------- smoothing (a3)

@pytest.mark.parametrize("H,W", [(64, 80), (256, 256), (61, 75), (97, 130)])
def test_smoothing_images_and_peak(asp, H, W):
    """Even W takes the paired column pass, odd W the single one; odd H
    leaves the paired row pass a last pair with one live row."""
    case = synth.small_case(H, W, seed=5, n_gauss=2, sigma_range=(3, 8))
    ctx = _ctx(asp, case)
    _, wb, _, _ = ctx.beam
    scales = ctx.scales()
    assert np.allclose(scales, O.smoothing_scales(wb, 6, H, W), rtol=1e-12)
    for j, s in enumerate(scales):
        S = ctx.smooth(j).cpu().numpy().astype(np.float64)
        ref = O.smooth_separable(case.dirty, s)
        assert _rel_l2(S, ref) < 1e-5, (j, s)
    pk = ctx.find_peak(asp.ASP_PEAK_SMOOTH)
    init = O.peak_smooth(case.dirty.astype(np.float64), wb, 6)
    # the GPU's winner is a maximum of |S| within FP32 rounding of the oracle's
    Sj = O.smooth_separable(case.dirty, scales[pk["scale_index"]])
    assert abs(Sj.ravel()[pk["index"]]) >= abs(init["value"]) * (1 - 1e-5)
    if (pk["scale_index"], pk["index"]) == (init["scale_index"], init["index"]):
        assert pk["a0"] == pytest.approx(init["a0"], rel=1e-5)
        assert pk["w0"] == pytest.approx(init["w0"], rel=1e-12)
    ctx.close()


# ----------------------------------------------------------------- LM pixel pass (a6)

@pytest.mark.parametrize("K,n_old", [(1, 0), (3, 2), (6, 3), (12, 0), (21, 5)])
def test_normal_equations_within_fp32_bound(asp, K, n_old):
    rng = np.random.default_rng(K)
    H, W = 120, 136
    case = synth.small_case(H, W, seed=K, n_points=3, n_gauss=2)
    ctx = _ctx(asp, case, k_max=max(K, 1))
    theta = np.column_stack([rng.uniform(-1, 1, K), rng.uniform(30, 100, K), rng.uniform(30, 90, K),
                             rng.uniform(1.2, 6, K)])
    win = (11, 124, 7, 118)
    A, g, chi2 = ctx.normal_equations(theta, n_old, win)
    x0, x1, y0, y1 = win
    ys, xs = np.mgrid[y0:y1 + 1, x0:x1 + 1]
    xs, ys = xs.ravel().astype(float), ys.ravel().astype(float)
    T = case.dirty[y0:y1 + 1, x0:x1 + 1].ravel().astype(np.float64)
    old = theta[K - n_old:].ravel()
    if n_old:
        T = T + O.gauss_model(old, xs, ys)
    # the FP32 error model of the pass (tests/fp32_bounds.py): Jacobian
    # entries (8 + 2 |arg_k|) u32 relative, residual 8 u32 (|T| + sum |g_k|)
    # plus the members' evaluation errors, sums (64 + log2 n + 16) u32 of
    # sum |terms|; the oracle's FP64 sums are the reference
    pb = FB.pass_bounds(T, xs, ys, theta.ravel())
    Ao, go, co = pb["A"], pb["g"], pb["chi2"]
    bA, bg, bc = pb["bA"], pb["bg"], pb["bc"]
    assert np.all(np.abs(A - Ao) <= bA + 1e-300), np.max(np.abs(A - Ao) / (bA + 1e-300))
    assert np.all(np.abs(g - go) <= bg + 1e-300), np.max(np.abs(g - go) / (bg + 1e-300))
    assert abs(chi2 - co) <= bc, (chi2, co, bc)
    ctx.close()


# ----------------------------------------------------------------- LM fit (a6 + a7)

@pytest.mark.parametrize("seed,K", [(0, 1), (1, 1), (2, 2), (3, 3), (4, 5)])
def test_fit_converges_to_oracle_optimum(asp, seed, K):
    rng = np.random.default_rng(100 + seed)
    H, W = 80, 88
    truth = []
    for k in range(K):
        truth.append([rng.uniform(0.5, 1.5) * rng.choice([-1, 1]), rng.uniform(34, 50), rng.uniform(30, 46),
                      rng.uniform(1.6, 4.0)])
    truth = np.array(truth)
    ys, xs = np.mgrid[0:H, 0:W]
    img = O.gauss_model(truth.ravel(), xs.astype(float), ys.astype(float)) + rng.normal(0, 1e-3, (H, W))
    psf = synth.gaussian_psf(H, W, 1.5)
    ctx = asp.Context(_t(img), _t(psf), k_max=K, noise_sigma=1e-3, lm_max_iter=200, lm_rtol=1e-9, lm_xtol=1e-9)
    start = truth * [1.15, 1, 1, 0.9] + [0, 0.3, -0.2, 0]
    out, info = ctx.fit(start, 0)
    x0, x1, y0, y1 = info["x0"], info["x1"], info["y0"], info["y1"]
    yy, xx = np.mgrid[y0:y1 + 1, x0:x1 + 1]
    T = img.astype(np.float32)[y0:y1 + 1, x0:x1 + 1].astype(np.float64).ravel()
    ref = O.lm_fit(T, xx.ravel().astype(float), yy.ravel().astype(float), start.ravel(), (x0, x1, y0, y1),
                   0.25 * 1.5, O.lm_exact())
    for k in range(K):
        _param_close(out[k], ref.theta[4 * k: 4 * k + 4])
    assert info["chi2_final"] == pytest.approx(ref.chi2, rel=1e-4)
    assert info["pixel_evals"] == info["passes"] * (x1 - x0 + 1) * (y1 - y0 + 1)
    ctx.close()


def test_large_window_multi_cta_fit(asp):
    """A window big enough to use many CTAs and the grid barriers."""
    rng = np.random.default_rng(7)
    H = W = 600
    truth = np.array([[0.8, 301.3, 297.6, 40.0], [-0.3, 280.2, 320.4, 25.0]])
    ys, xs = np.mgrid[0:H, 0:W]
    img = O.gauss_model(truth.ravel(), xs.astype(float), ys.astype(float)) + rng.normal(0, 1e-3, (H, W))
    psf = synth.gaussian_psf(H, W, 2.0)
    ctx = asp.Context(_t(img), _t(psf), k_max=2, noise_sigma=1e-3, lm_max_iter=100, lm_rtol=1e-10, lm_xtol=1e-9)
    start = truth * [0.9, 1, 1, 1.1] + [0, 0.5, -0.5, 0]
    out, info = ctx.fit(start, 0)
    x0, x1, y0, y1 = info["x0"], info["x1"], info["y0"], info["y1"]
    assert (x1 - x0 + 1) * (y1 - y0 + 1) > 100000
    yy, xx = np.mgrid[y0:y1 + 1, x0:x1 + 1]
    T = img.astype(np.float32)[y0:y1 + 1, x0:x1 + 1].astype(np.float64).ravel()
    ref = O.lm_fit(T, xx.ravel().astype(float), yy.ravel().astype(float), start.ravel(), (x0, x1, y0, y1),
                   0.5, O.lm_exact())
    for k in range(2):
        _param_close(out[k], ref.theta[4 * k: 4 * k + 4])
    ctx.close()


# ----------------------------------------------------------------- minor cycle (a2-a10)

def _oracle_from_gpu_state(ctx, case, p, beam):
    return teacher.oracle_from_state(ctx, case, p, beam)[0]


TIGHT = dict(lm_max_iter=300, lm_rtol=1e-12, lm_xtol=1e-10)


@pytest.mark.parametrize("k_max,sub_mode", [(1, "direct"), (3, "direct"), (5, "direct"), (5, "fft")])
def test_teacher_forced_minor_cycle_steps(asp, k_max, sub_mode, capsys):
    """Each iteration starts both sides from the GPU's state (tests/teacher.py):
    the discrete decisions agree exactly; the GPU's residual update is the
    oracle's subtraction of the GPU's fitted components within 1e-5
    relative L2; where the fits converged, every parameter is within 1e-4
    of its scale of the oracle's optimum, or within twice the first-order
    FP32 floor |A^-1| dg where that is larger.  Both sides run LM to the
    optimum (tight tolerances; the GPU ends at its FP32 floor)."""
    case = synth.small_case(96, 104, seed=11, n_points=3, n_gauss=2, sigma_range=(2.5, 6))
    mode = asp.ASP_SUB_FFT if sub_mode == "fft" else asp.ASP_SUB_DIRECT
    ctx = _ctx(asp, case, k_max=k_max, sub_mode=mode, **TIGHT)
    ab, wb, _, _ = ctx.beam
    p = O.AspParams(k_max=k_max, noise_sigma=case.noise_sigma, lm=O.lm_exact())
    stats = teacher.Stats()
    for it in range(12):
        mc, st = teacher.oracle_from_state(ctx, case, p, (ab, wb))
        R_before = mc.R.copy()
        rec = mc.step()
        if rec is None:
            break
        ctx.minor_cycle(1)
        teacher.check_iteration(ctx, case, rec, R_before, st, stats)
    assert stats.fits >= 3 and stats.updates >= 10
    with capsys.disabled():
        print(f"\nk_max {k_max} ({sub_mode} update): {stats.fits} converged fits, {stats.params_beyond_1e4}/{stats.params} parameters "
              f"beyond 1e-4 (within the FP32 floor), max |dtheta|/scale {stats.max_rel_param:.2e}; "
              f"residual updates max rel L2 {stats.max_rel_update:.2e}")
    ctx.close()


def test_teacher_forced_default_tolerances_decisions(asp):
    """With the default LM settings the discrete decisions of every
    iteration still agree when both sides start from the same state."""
    case = synth.config1(0)
    ctx = _ctx(asp, case)
    ab, wb, _, _ = ctx.beam
    p = O.AspParams(k_max=case.k_max, noise_sigma=case.noise_sigma)
    for it in range(10):
        mc = _oracle_from_gpu_state(ctx, case, p, (ab, wb))
        rec = mc.step()
        ctx.minor_cycle(1)
        h = ctx.history()[-1]
        assert h["mode"] == rec["mode"]
        assert (h["x0"], h["x1"], h["y0"], h["y1"]) == tuple(rec["window"])
        assert h["k"] == len(rec["members"])
    ctx.close()


def test_minor_cycle_to_noise_matches_oracle(asp):
    """A run to the noise threshold: final residual RMS and recovered model
    flux agree with the oracle's own run (the paper's quality observables,
    Tables 1-2)."""
    case = synth.small_case(72, 80, seed=21, n_points=3, n_gauss=1, sigma_range=(2.0, 3.0), noise_sigma=1e-3)
    ctx = _ctx(asp, case, k_max=3)
    st = ctx.minor_cycle(400)
    ab, wb, _, _ = ctx.beam
    mc = O.MinorCycle(case.dirty, case.psf, O.AspParams(k_max=3, noise_sigma=case.noise_sigma),
                      beam=(ab, wb)).run(400)
    R = ctx.residual().astype(np.float64)
    rms_g, rms_o = np.sqrt(np.mean(R ** 2)), np.sqrt(np.mean(mc.R ** 2))
    assert st["stop_reason"] == asp.ASP_STOP_NOISE and mc.stopped
    assert rms_g == pytest.approx(rms_o, rel=0.05)
    assert ctx.components()[:, 0].sum() == pytest.approx(mc.stats()["model_flux"], rel=0.01)
    assert ctx.components()[:, 0].sum() == pytest.approx(case.sky.sum(), rel=0.05)
    ctx.close()


def test_noise_stop_and_mad_estimate(asp):
    case = synth.small_case(64, 64, seed=3, n_points=1, n_gauss=0, noise_sigma=1e-3)
    ctx = asp.Context(_t(case.dirty), _t(case.psf), noise_sigma=0.0, k_max=2)
    st = ctx.minor_cycle(500)
    assert st["stop_reason"] == asp.ASP_STOP_NOISE
    assert st["peak_abs"] < 3 * O.mad_sigma(case.dirty) * (1 + 1e-6)
    ctx.close()


def test_state_save_load_round_trip(asp, tmp_path):
    case = synth.small_case(80, 80, seed=4, n_points=2, n_gauss=1)
    a = _ctx(asp, case, k_max=3)
    a.minor_cycle(5)
    path = str(tmp_path / "state.bin")
    from paper_1606_07872_gb300 import asp_save_state, asp_load_state
    asp_save_state(a.h, path)
    a.minor_cycle(5)
    b = _ctx(asp, case, k_max=3)
    asp_load_state(b.h, path)
    b.minor_cycle(5)
    np.testing.assert_array_equal(a.residual(), b.residual())
    np.testing.assert_array_equal(a.components(), b.components())
    a.close()
    b.close()


def test_nonfinite_input_rejected(asp):
    case = synth.small_case(32, 32, seed=0)
    d = case.dirty.copy()
    d[3, 4] = np.nan
    with pytest.raises(asp.AspError) as e:
        asp.Context(_t(d), _t(case.psf), noise_sigma=1e-3)
    assert e.value.status == 4


def test_invalid_arguments(asp):
    case = synth.small_case(32, 32, seed=0)
    ctx = _ctx(asp, case, k_max=2)
    with pytest.raises(asp.AspError):
        ctx.fit([[1, 5, 5, 1.5]] * 3, 0)          # more members than k_max
    with pytest.raises(asp.AspError):
        ctx.fit([[1, 5, 5, -1.0]], 0)             # negative width
    with pytest.raises(asp.AspError):
        ctx.subtract([[1, 0, 5, 5, np.nan, 0]])
    ctx.close()
    with pytest.raises(asp.AspError) as e:
        _ctx(asp, case, fit_px_per_cta=-1)        # negative fit tile
    assert e.value.status == 1


@pytest.mark.parametrize("px", [32, 200, 5000])
def test_fit_tile_changes_only_rounding(asp, px):
    """The fit's launch shape (window pixels per CTA) decides how many CTAs
    share the accumulation, hence only the FP32 summation order: a joint fit
    of three overlapping Gaussians from a fixed start converges to the
    default shape's optimum within the parity bound (1e-4 per parameter)."""
    rng = np.random.default_rng(40 + px)
    H = W = 96
    truth = np.array([[0.8, 40.3, 47.1, 2.6], [-0.4, 52.2, 50.6, 3.1], [0.3, 47.0, 38.5, 2.2]])
    ys, xs = np.mgrid[0:H, 0:W]
    img = O.gauss_model(truth.ravel(), xs.astype(float), ys.astype(float)) + rng.normal(0, 1e-3, (H, W))
    psf = synth.gaussian_psf(H, W, 1.5)
    start = truth * [1.1, 1, 1, 0.9] + [0, 0.3, -0.2, 0]
    fits = []
    for kw in ({}, dict(fit_px_per_cta=px)):
        ctx = asp.Context(_t(img), _t(psf), k_max=5, noise_sigma=1e-3, lm_max_iter=300, lm_rtol=1e-12,
                          lm_xtol=1e-10, **kw)
        out, info = ctx.fit(start, 0)
        fits.append((np.asarray(out, float), info))
        ctx.close()
    (a, ia), (b, ib) = fits
    assert ia["status"] == ib["status"] == O.LM_CONVERGED
    assert np.all(np.abs(a - b) <= 1e-4 * np.maximum(np.abs(a), 1.0)), (a, b)
    assert ia["chi2_final"] == pytest.approx(ib["chi2_final"], rel=1e-5)


def test_config2_full_size_sampled(asp):
    case = synth.config2(0)
    ctx = _ctx(asp, case)
    ab, wb, xb, yb = ctx.beam
    oab, owb, fit = O.beam_fit(case.psf, O.lm_exact())
    _param_close([ab, xb, yb, wb], [oab, fit.theta[1], fit.theta[2], owb])
    st = ctx.minor_cycle(20)
    assert st["iterations"] == 20
    R = ctx.residual()
    pk = ctx.find_peak(asp.ASP_PEAK_SIMPLE)
    idx, val = O.peak_simple(R)
    assert pk["index"] == idx
    # teacher-forced iterations at full size (tests/teacher.py), with the
    # run's own LM settings: decisions, the residual update (1e-5), and the
    # parameters of converged fits (1e-4 or the FP32 floor)
    p = O.AspParams(k_max=case.k_max, noise_sigma=case.noise_sigma)
    stats = teacher.Stats()
    for it in range(3):
        mc, st = teacher.oracle_from_state(ctx, case, p, (ab, wb))
        R_before = mc.R.copy()
        rec = mc.step()
        ctx.minor_cycle(1)
        teacher.check_iteration(ctx, case, rec, R_before, st, stats)
    assert stats.updates == 3
    ctx.close()
