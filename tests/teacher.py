"""Teacher-forced checks of one minor-cycle iteration (Sect. 2 steps 1-4
with the Sect. 3 objective): both sides start from the GPU's state, then

* the discrete decisions (init mode, window, active-set size) are equal;
* the residual update R_after - R_before of the GPU equals the oracle's
  subtraction (Sect. 2 step 3, full PSF) of the components the GPU's fit
  produced -- new component with the loop gain, refit members replacing
  their old values -- within 1e-5 relative L2 (the subtraction is checked
  on its own, given the fit);
* where neither fit stopped at the iteration cap, every fitted parameter agrees with the FP64
  oracle's optimum within 1e-4 of its scale (|a|; max(1, w) for centres; w
  for widths), or, where it is larger, within twice the FP32 floor of the
  optimum: the larger of the gradient floor |A^-1| dg (the GPU's FP32 J^T r
  moves the stationary point by A^-1 dg) and the chi^2 valley at the FP32
  chi^2 error, sqrt(2 bc (A^-1)_ii) (Marquardt's accept test compares two
  FP32 chi^2 values, so LM cannot tell apart points whose chi^2 differ by
  less than 2 bc) -- both wide only along the flat directions of joint fits
  (tests/fp32_bounds.py);
* chi^2 of the GPU's parameters (evaluated in FP64 on the oracle's target)
  is the optimum's within four FP32 chi^2 bounds.
"""
from __future__ import annotations

import numpy as np

import oracle as O
from tests import fp32_bounds as FB


class Stats:
    def __init__(self):
        self.fits = 0
        self.params = 0
        self.params_beyond_1e4 = 0
        self.max_rel_param = 0.0
        self.max_rel_update = 0.0
        self.updates = 0
        self.max_over_valley = 0.0


def oracle_from_state(view, case, p, beam):
    st = view.state()
    mc = O.MinorCycle(case.dirty, case.psf, p, beam=beam)
    comps = [O.Component(q[0], q[1], q[2], q[3], q[4], bool(q[5])) for q in st["comps"]]
    mc.set_state(view.residual().astype(np.float64), comps, st["retained"], st["t"], st["last_wi"], st["last_w0"])
    return mc, st


def oracle_iteration(mc):
    """The oracle's record of one iteration from its current state without
    applying it (steps 1-5: decisions, target and the LM fit; no
    subtraction), for checks on large images where a second full-image
    subtraction would dominate the test's time."""
    prep = mc.prepare()
    if prep is None:
        return None
    fit = O.lm_fit(prep["T"], prep["xs"], prep["ys"], prep["theta0"], prep["window"], 0.25 * mc.omega_b, mc.p.lm)
    return dict(mode=prep["mode"], window=prep["window"], members=[len(mc.comps)] + list(prep["chosen"]),
                fit=fit, T=prep["T"], xs=prep["xs"], ys=prep["ys"], theta0=prep["theta0"])


def update_terms(comps_before, comps_after, chosen, H, W):
    """Separable terms of the GPU's iteration: the new component (last in
    comps_after) plus (refit - old) for each retained member it refitted."""
    terms = []
    new = comps_after[len(comps_before)]
    terms.append(O.component_terms(new[0], new[2], new[3], new[4], bool(new[5]), H, W))
    for k in chosen:
        c1, c0 = comps_after[k], comps_before[k]
        terms.append(O.component_terms(c1[0], c1[2], c1[3], c1[4], bool(c1[5]), H, W))
        t0 = O.component_terms(c0[0], c0[2], c0[3], c0[4], bool(c0[5]), H, W)
        if t0 is not None:
            terms.append(t0[:4] + (-t0[4],))
    return [t for t in terms if t is not None]


def subtraction_at(B, terms, H, W, py, px):
    """Brute-force 2-D direct form of the subtraction at given pixels:
    sum over each term's support q of s wx wy B(p - q + (H, W))."""
    out = np.zeros(len(py))
    for qx0, wx, qy0, wy, s in terms:
        jy = np.arange(len(wy))
        ix = np.arange(len(wx))
        for n, (y, x) in enumerate(zip(py, px)):
            Bsub = B[np.ix_(y - qy0 - jy + H, x - qx0 - ix + W)]
            out[n] += s * float(wy @ Bsub @ wx)
    return out


def check_iteration(view, case, rec, R_before, st_before, stats: Stats, sample_px=None, rng=None):
    """The checks listed in the module docstring for one iteration the GPU
    has just run (view.history()[-1]) and the oracle's record ``rec`` of
    the same iteration from the same state."""
    h = view.history()[-1]
    assert h["mode"] == rec["mode"]
    assert (h["x0"], h["x1"], h["y0"], h["y1"]) == tuple(rec["window"])
    assert h["k"] == len(rec["members"])
    H, W = case.H, case.W
    st_after = view.state()
    terms = update_terms(st_before["comps"], st_after["comps"], rec["members"][1:], H, W)
    R = view.residual().astype(np.float64)
    if sample_px is None:
        ref = O.subtract_terms(R_before, case.psf, terms)
        d_gpu, d_ref = R - R_before, ref - R_before
    else:
        # random pixels plus a 5 x 5 lattice around each term's centre
        pts = [(int(rng.integers(0, H)), int(rng.integers(0, W))) for _ in range(sample_px)]
        for qx0, wx, qy0, wy, _ in terms:
            cy, cx = qy0 + len(wy) // 2, qx0 + len(wx) // 2
            for dy in (-8, -2, 0, 2, 8):
                for dx in (-8, -2, 0, 2, 8):
                    pts.append((min(max(cy + dy, 0), H - 1), min(max(cx + dx, 0), W - 1)))
        py = np.array([q[0] for q in pts])
        px = np.array([q[1] for q in pts])
        d_ref = -subtraction_at(np.asarray(case.psf, np.float64), terms, H, W, py, px)
        d_gpu = R[py, px] - R_before[py, px]
    rel = float(np.linalg.norm(d_gpu - d_ref) / max(np.linalg.norm(d_ref), 1e-300))
    assert rel < 1e-5, rel
    stats.updates += 1
    stats.max_rel_update = max(stats.max_rel_update, rel)
    fit = rec["fit"]
    # the oracle's fit reached its optimum (converged, or stalled at its own
    # FP64 resolution under the tight tolerances) and the GPU's did not stop
    # at the iteration cap
    if fit.status == O.LM_CAP or h["status"] == O.LM_CAP:
        return False
    th_gpu, _ = view.last_fit()
    th_gpu = th_gpu.ravel()
    T, xs, ys = rec["T"], rec["xs"], rec["ys"]
    theta0 = rec["theta0"]
    extra = O.gauss_model(np.abs(theta0[4:]), xs, ys) if len(theta0) > 4 else None
    chi2_gpu = float(np.sum((T - O.gauss_model(th_gpu, xs, ys)) ** 2))
    pb = FB.pass_bounds(T, xs, ys, fit.theta, extra)
    assert chi2_gpu <= fit.chi2 + 4.0 * pb["bc"], (chi2_gpu, fit.chi2, pb["bc"])
    floor = np.maximum(FB.optimum_floor(pb["A"], pb["bg"]), FB.chi2_valley(pb["A"], pb["bc"]))
    scale = FB.param_scale(fit.theta)
    err = np.abs(th_gpu - fit.theta)
    tol = np.maximum(1e-4 * scale, 2.0 * floor)
    assert np.all(err <= tol), (np.max(err / tol), th_gpu, fit.theta, floor)
    stats.max_over_valley = max(stats.max_over_valley, float(np.max(err / np.maximum(floor, 1e-300))))
    stats.fits += 1
    stats.params += err.size
    stats.params_beyond_1e4 += int(np.sum(err > 1e-4 * scale))
    stats.max_rel_param = max(stats.max_rel_param, float(np.max(err / scale)))
    return True
