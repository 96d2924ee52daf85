"""Large active sets (more than 32 members: the fit variant that keeps A in
L2 and accumulates the normal equations in tile rounds) and the 4096x4096
workload (config 3) at full size."""
import numpy as np
import pytest

import oracle as O
import synth
from tests import teacher

pytestmark = pytest.mark.gpu


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _param_close(g, o, rtol=1e-4):
    a, x, y, w = o
    assert abs(g[0] - a) <= rtol * abs(a), (g, o)
    assert abs(g[1] - x) <= rtol * max(1.0, w), (g, o)
    assert abs(g[2] - y) <= rtol * max(1.0, w), (g, o)
    assert abs(g[3] - w) <= rtol * w, (g, o)


@pytest.mark.parametrize("K", [36, 48])
def test_large_active_set_fit_matches_oracle(asp, K):
    """A joint fit of K overlapping Gaussians (P = 4K > 128 parameters; 48
    needs two rounds of accumulator tiles) reaches the FP64 oracle's
    optimum: every parameter within 1e-4, chi^2 within 1e-4 relative."""
    rng = np.random.default_rng(7 + K)
    H = W = 128
    side = int(np.ceil(np.sqrt(K)))
    truth = []
    for k in range(K):
        gx, gy = k % side, k // side
        truth.append([rng.uniform(0.5, 1.5) * rng.choice([-1, 1]), 34 + 9.0 * gx + rng.uniform(-1, 1),
                      34 + 9.0 * gy + rng.uniform(-1, 1), rng.uniform(2.0, 3.5)])
    truth = np.array(truth)
    ys, xs = np.mgrid[0:H, 0:W]
    img = O.gauss_model(truth.ravel(), xs.astype(float), ys.astype(float)) + rng.normal(0, 1e-3, (H, W))
    psf = synth.gaussian_psf(H, W, 1.5)
    ctx = asp.Context(_t(img), _t(psf), k_max=50, noise_sigma=1e-3, lm_max_iter=300, lm_rtol=1e-10,
                      lm_xtol=1e-10)
    start = truth * [1.1, 1, 1, 0.92] + [0, 0.25, -0.2, 0]
    out, info = ctx.fit(start, 0)
    x0, x1, y0, y1 = info["x0"], info["x1"], info["y0"], info["y1"]
    yy, xx = np.mgrid[y0:y1 + 1, x0:x1 + 1]
    T = img.astype(np.float32)[y0:y1 + 1, x0:x1 + 1].astype(np.float64).ravel()
    ref = O.lm_fit(T, xx.ravel().astype(float), yy.ravel().astype(float), start.ravel(), (x0, x1, y0, y1),
                   0.25 * 1.5, O.lm_exact())
    assert ref.status == O.LM_CONVERGED
    for k in range(K):
        _param_close(out[k], ref.theta[4 * k: 4 * k + 4])
    assert info["chi2_final"] == pytest.approx(ref.chi2, rel=1e-4)
    ctx.close()


def test_config3_full_size_first_iterations(asp, capsys):
    """The 4096x4096 workload (k_max 50) at full size: starting each
    iteration from the GPU's state, the first iterations take the oracle's
    decisions (peak, window, active set), reach its fit (1e-4 of each
    parameter's scale, or the FP32 floor) and update the residual as the
    oracle's brute-force direct subtraction of the fitted components does
    (1e-5 relative L2 at 512 random pixels and around each term;
    tests/teacher.py)."""
    case = synth.config3(0)
    ctx = asp.Context(_t(case.dirty), _t(case.psf), k_max=case.k_max, noise_sigma=case.noise_sigma, init_mode=1,
                      lm_max_iter=300, lm_rtol=1e-12, lm_xtol=1e-10)
    ab, wb, _, _ = ctx.beam
    p = O.AspParams(k_max=case.k_max, noise_sigma=case.noise_sigma, init_mode="simple", lm=O.lm_exact())
    rng = np.random.default_rng(3)
    stats = teacher.Stats()
    for it in range(3):
        mc, st = teacher.oracle_from_state(ctx, case, p, (ab, wb))
        rec = teacher.oracle_iteration(mc)
        R0 = mc.R.copy()
        ctx.minor_cycle(1)
        teacher.check_iteration(ctx, case, rec, R0, st, stats, sample_px=512, rng=rng)
    assert stats.updates == 3
    with capsys.disabled():
        print(f"\nconfig 3: {stats.updates} updates (max rel L2 {stats.max_rel_update:.2e}), {stats.fits} converged "
              f"fits, max |dtheta|/scale {stats.max_rel_param:.2e}")
    ctx.close()
