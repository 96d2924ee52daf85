"""Step-by-step parity of Levenberg-Marquardt (Marquardt 1963, the minimiser
of the Eq. 6 objective) on the fits of the 1024 x 1024 workload, at full
size, fits that hit the 50-solve cap included.

Each checked minor-cycle iteration starts both sides from the GPU's own
state: the oracle prepares the iteration (mode, initial values, active set,
window, target T = R + sum of the added-back members) and the decisions
must match the GPU's.  The GPU then runs that fit's LM for m damped solves
(m = 0 ... 49) and stops; from each snapshot (theta_m, lambda_m) BOTH sides
take one Marquardt step (asp_fit_lm with max_iter = 1; the oracle's lm_fit
with the same start and damping):

* the step delta element by element: within 1e-4 of the parameter's scale
  (|a|; max(1, w) for centres; w for widths), or within twice the derived
  first-order bound of the FP32 normal equations through the damped solve
  where that bound is larger (flat directions at small damping) -- wherever
  that bound is valid (the scaled damped system is conditioned well enough
  for the FP32 errors: kappa < 0.5); and always, componentwise backward
  error: the GPU's step solves the damped normal equations within twice
  their FP32 error bounds (where kappa >= 0.5 the step is not unique at
  FP32 precision and this is what identifies a correct one);
* chi^2 at theta and at the GPU's trial point within the FP32 bound of the
  pixel pass;
* the validity test of the trial point exactly, and the accept bit exactly
  wherever the oracle's chi^2 margin exceeds the two chi^2 bounds (else
  either decision is a correct LM step);
* the damping update exactly (lambda / 10 floored at 1e-12, or 10 lambda).

The residual update of the iteration itself is checked against the
oracle's subtraction of the GPU's fitted components (1e-5 relative L2).
"""
import numpy as np
import pytest

import oracle as O
import oracle.asp_oracle as OA
import synth
from tests import fp32_bounds as FB
from tests import teacher

pytestmark = pytest.mark.gpu

SNAPSHOTS = (0, 1, 4, 12, 25, 40, 49)
# iterations of the 1024^2 workload checked (the state is advanced on the
# GPU between them): the first ones, and fits that hit the 50-solve cap,
# found in a first run of the same (deterministic) cycle
FIRST = (0, 1, 40)
N_CAPPED = 4
SCAN = 600


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, float) - np.asarray(b, float)) / max(np.linalg.norm(b), 1e-300))


class Tally:
    def __init__(self):
        self.steps = 0
        self.forward = 0
        self.entries = 0
        self.needed_bound = 0
        self.max_rel = 0.0
        self.accept_checked = 0
        self.accept_ambiguous = 0
        self.capped_fits = 0
        self.fits = 0


def _one_step(ctx, prep, n_old, theta, lam, omega_min, extra, tally):
    xs, ys, T, win = prep["xs"], prep["ys"], prep["T"], prep["window"]
    rows = np.asarray(theta).reshape(-1, 4)
    # the fit is the iteration's own (window, target with the members added
    # back at their initial values); LM restarts at (theta, lam)
    out, info, trial_g, chi2_last = ctx.fit_lm(prep["theta0"].reshape(-1, 4), n_old, lam, 1, start=rows)
    theta = np.asarray(theta, dtype=np.float64).ravel()
    trial_g = trial_g.ravel()
    lm1 = O.LMParams(lambda0=lam, max_iter=1)
    ref = O.lm_fit(T, xs, ys, theta, win, omega_min, lm1)
    pb = FB.pass_bounds(T, xs, ys, theta, extra)
    # chi^2 at the start point
    assert abs(info["chi2_init"] - pb["chi2"]) <= pb["bc"], (info["chi2_init"], pb["chi2"], pb["bc"])
    assert info["iters"] == 1
    if ref.trial is None:
        # the FP64 damped matrix is not positive definite: LM raises lambda
        assert info["passes"] == 1 and info["lambda"] == lam * 10.0
        return
    d_o = ref.trial - theta
    d_g = trial_g - theta
    bound, kappa = FB.step_bound(pb["A"], pb["g"], lam, pb["bA"], pb["bg"], d_o)
    scale = FB.param_scale(theta)
    err = np.abs(d_g - d_o)
    # backward error, always: the GPU's step solves the damped system within
    # the FP32 errors of its normal equations and solve
    resid, allowed = FB.step_backward(pb["A"], pb["g"], lam, pb["bA"], pb["bg"], d_g)
    assert np.all(resid <= 2.0 * allowed), np.max(resid / allowed)
    tally.steps += 1
    if kappa < 0.5:
        # forward error: the first-order bound holds (scaled system well
        # enough conditioned for the FP32 errors), so delta is unique to it
        tol = np.maximum(1e-4 * scale, 2.0 * bound)
        assert np.all(err <= tol), (np.max(err / tol), d_g, d_o, bound)
        tally.forward += 1
        tally.entries += err.size
        tally.needed_bound += int(np.sum(err > 1e-4 * scale))
        tally.max_rel = max(tally.max_rel, float(np.max(err / scale)))
    # the predicted-decrease convergence test (2 d.g - d.A.d = d.g + lam d.D.d)
    d = FB.marquardt_diag(pb["A"])
    pred = lambda dd: float(dd @ pb["g"]) + lam * float(dd @ (d * dd))   # noqa: E731
    thr = 1e-7 * pb["chi2"]
    p_err = abs(pred(d_g) - pred(d_o)) + float(np.abs(d_o) @ (pb["bg"] + FB.U32 * np.abs(pb["g"]))) + \
        1e-7 * pb["bc"] + 4 * len(d_o) * FB.U32 * (abs(pred(d_o)) + 1e-300)
    conv_o = pred(d_o) <= thr
    conv_g = info["passes"] == 1 and info["status"] == O.LM_CONVERGED
    if abs(pred(d_o) - thr) > p_err:
        assert conv_g == conv_o, (pred(d_o), thr, p_err, info)
    if conv_g:
        return
    # validity of the GPU's own trial point: a deterministic FP64 test
    valid = OA._valid(trial_g, win, omega_min)
    assert (info["passes"] == 2) == valid, (info, trial_g)
    if not valid:
        assert info["lambda"] == lam * 10.0
        return
    pt = FB.pass_bounds(T, xs, ys, trial_g, extra)
    assert abs(chi2_last - pt["chi2"]) <= pt["bc"], (chi2_last, pt["chi2"], pt["bc"])
    accepted = bool(np.any(out.ravel() != theta))
    if accepted:
        np.testing.assert_array_equal(out.ravel(), trial_g)
        assert info["lambda"] == max(lam / 10.0, 1e-12)
    else:
        assert info["lambda"] == lam * 10.0
    margin = pt["chi2"] - pb["chi2"]
    if abs(margin) > pt["bc"] + pb["bc"]:
        assert accepted == (margin < 0), (margin, pt["bc"], pb["bc"])
        tally.accept_checked += 1
    else:
        tally.accept_ambiguous += 1


def test_lm_steps_match_oracle_at_full_size(asp, capsys):
    case = synth.config2(0)
    ctx = asp.Context(_t(case.dirty), _t(case.psf), k_max=case.k_max, noise_sigma=case.noise_sigma,
                      gain=case.gain, lm_max_iter=case.lm_max_iter)
    ab, wb, _, _ = ctx.beam
    omega_min = 0.25 * wb
    p = O.AspParams(k_max=case.k_max, noise_sigma=case.noise_sigma, gain=case.gain)
    tally = Tally()
    residual_checks = 0
    ctx.minor_cycle(SCAN)
    capped = [h["t"] for h in ctx.history() if h["status"] == O.LM_CAP and h["t"] > FIRST[-1]]
    assert len(capped) >= N_CAPPED, len(capped)
    # twice as many candidates as needed, spread over the scan: a fit that
    # capped in the scan run can converge when fitted again (its start comes
    # back through the host's FP64 state, and the trajectory is chaotic in
    # the last bits), so candidates are examined until N_CAPPED capped
    n_cand = min(len(capped), 2 * N_CAPPED)
    picks = [capped[(i * (len(capped) - 1)) // (n_cand - 1)] for i in range(n_cand)]
    iterations = sorted(set(FIRST) | set(picks))
    ctx.close()
    ctx = asp.Context(_t(case.dirty), _t(case.psf), k_max=case.k_max, noise_sigma=case.noise_sigma,
                      gain=case.gain, lm_max_iter=case.lm_max_iter)
    t = 0
    for it in iterations:
        if it not in FIRST and tally.capped_fits >= N_CAPPED:
            break
        if it > t:
            ctx.minor_cycle(it - t)
            t = it
        mc, st_before = teacher.oracle_from_state(ctx, case, p, (ab, wb))
        prep = mc.prepare()
        assert prep is not None
        theta0 = prep["theta0"]
        K = len(theta0) // 4
        n_old = K - 1
        extra = O.gauss_model(np.abs(theta0[4:]), prep["xs"], prep["ys"]) if K > 1 else None
        full, full_info = ctx.fit_lm(theta0.reshape(-1, 4), n_old, 1e-3, case.lm_max_iter)[:2]
        tally.fits += 1
        tally.capped_fits += int(full_info["status"] == O.LM_CAP)
        for m in SNAPSHOTS:
            snap, sinfo = ctx.fit_lm(theta0.reshape(-1, 4), n_old, 1e-3, m)[:2]
            _one_step(ctx, prep, n_old, snap.ravel(), sinfo["lambda"], omega_min, extra, tally)
        # the iteration itself on the GPU: same decisions, and its residual
        # update is the oracle's subtraction of the GPU's fitted components
        R_before = ctx.residual().astype(np.float64)
        ctx.minor_cycle(1)
        t += 1
        h = ctx.history()[-1]
        assert h["mode"] == prep["mode"]
        assert (h["x0"], h["x1"], h["y0"], h["y1"]) == tuple(prep["window"])
        assert h["k"] == K
        if residual_checks < 3:
            terms = teacher.update_terms(st_before["comps"], ctx.state()["comps"], prep["chosen"], case.H, case.W)
            R_ref = O.subtract_terms(R_before, case.psf, terms)
            R_gpu = ctx.residual().astype(np.float64)
            assert _rel_l2(R_gpu - R_before, R_ref - R_before) < 1e-5
            residual_checks += 1
    ctx.close()
    assert tally.capped_fits >= N_CAPPED, "the capped fits of the first run did not recur"
    assert tally.steps >= 30
    with capsys.disabled():
        print(f"\nLM steps: {tally.steps} from {tally.fits} fits ({tally.capped_fits} capped), forward-checked "
              f"{tally.forward}; "
              f"{tally.needed_bound}/{tally.entries} step entries beyond 1e-4 of their scale (within the FP32 "
              f"bound); max |d_gpu - d_oracle| / scale = {tally.max_rel:.2e}; accept bits compared "
              f"{tally.accept_checked}, within the chi^2 bounds {tally.accept_ambiguous}")
