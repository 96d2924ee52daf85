#!/usr/bin/env python
"""Benchmark of the Asp-Clean2016 minor cycle on one GB300 (or N replicas).

Workload (default): the 1024x1024 configuration -- 50 power-law points, 20
Gaussians (sigma 2-60 px), one k^-3 GRF patch, uv-mask PSF with a ~2 px main
lobe, noise 1e-4, active set <= 20, 2000 minor-cycle iterations, loop gain
0.35, LM cap 50.  Synthetic, seeded (synth.config2).

One step = one whole pass of the hot path over the image: asp_reset with the
dirty image and the PSF (beam fit, first peak) then asp_minor_cycle for the
configuration's 2000 iterations (peak search, active set, LM fits,
deconvolution, subtraction, stopping tests).  Inputs are resident in HBM when
the timed region starts; L2 is flushed (256 MB write) between steps, outside
the timed region.  The metric is minor-cycle iterations per second (whole job);
LM pixel evaluations per second are reported beside it.

Under torchrun (N > 1) every rank runs its own replica of the workload with
its own seed (independent images, no collective): weak scaling.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

UNIT = "iterations/s"


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--iters", type=int, default=0, help="minor-cycle iterations per step (0: the workload's 2000)")
    ap.add_argument("--size", type=int, default=0, help="image side (0: the workload's own)")
    ap.add_argument("--config", type=int, choices=[2, 3], default=2,
                    help="workload of the main line: 2 (1024^2, k_max 20) or 3 (4096^2, k_max 50)")
    ap.add_argument("--no-config3", action="store_true", help="skip the 4096^2 measurement beside config 2")
    ap.add_argument("--config3-iters", type=int, default=300,
                    help="iterations per 4096^2 step beside config 2 (its first 300 of 5000; 0: all 5000)")
    ap.add_argument("--config3-steps", type=int, default=1)
    ap.add_argument("--config3-warmup", type=int, default=1)
    ap.add_argument("--split-config3", action="store_true", help="also measure the split on the 4096^2 workload")
    ap.add_argument("--fit-px", type=int, default=0, help="LM fit tile: window pixels per CTA (0: library default)")
    ap.add_argument("--no-split", action="store_true", help="skip the minor/major split comparison")
    ap.add_argument("--no-elliptical", action="store_true", help="skip the elliptical-variant comparison")
    ap.add_argument("--no-joint", action="store_true", help="skip the joint wide-band fit comparison")
    ap.add_argument("--large-fit", type=int, default=0,
                    help="only run one LM step of this many members over a ~950^2 window of a 2048^2 image "
                         "(k_max 50: the large fit variant), for profiling, and print its outcome")
    ap.add_argument("--sub", choices=["auto", "direct", "fft"], default="auto",
                    help="residual update form of the measured runs (auto: FFT from 512x512 pixels)")
    ap.add_argument("--no-sub-forms", action="store_true",
                    help="skip the comparison with the direct residual update")
    ap.add_argument("--no-2004", action="store_true", help="skip the Eq. 3 vs Eq. 6 per-iteration comparison")
    ap.add_argument("--split-every", type=int, default=50, help="minor iterations per major cycle in the split")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=20.0, help="seconds of oracle work for cpu_baseline")
    ap.add_argument("--no-batched", action="store_true", help="skip the 64-image batch comparison")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-initial-value comparison")
    ap.add_argument("--batch-images", type=int, default=64)
    ap.add_argument("--learned-train-images", type=int, default=120, help="config-1 images harvested for training")
    return ap.parse_args()


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    smax.append(float(f[2]))
                except ValueError:
                    continue
                for n, v in zip(names, f[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
            os.unlink(self.path)
        except OSError:
            pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- helpers

def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def _traffic_record():
    """Per-launch DRAM bytes of the dominant kernel from a committed ncu
    summary, if the kernel source has not changed since it was taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path))
    except (OSError, ValueError):
        return {}
    import hashlib
    out = {}
    for name, r in rec.items():
        src = os.path.join(ROOT, r.get("source", ""))
        try:
            h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        except OSError:
            continue
        if h == r.get("source_sha256_16"):
            out[name] = r
    return out


def _fit_phases(st) -> dict:
    """The fit kernel's own phase clocks (CTA 0 of every fit, %globaltimer)
    over the profiled step, per damped solve (LM iteration)."""
    li = max(int(st["lm_iters"]), 1)
    us = lambda k: 1e3 * float(st[k]) / li   # noqa: E731
    return {"lm_iters": int(st["lm_iters"]), "passes": int(st["lm_passes"]),
            "refinements": int(st["fit_refinements"]), "fp64_fallbacks": int(st["fit_fallbacks"]),
            "us_per_lm_iter": {"pixel_pass": us("fit_pass_ms"), "chi2_decision_reduction": us("fit_reduce_ms"),
                               "solve_total": us("fit_solve_ms"), "damped_solve": us("fit_factor_ms"),
                               "post_solve_checks": us("fit_subst_ms")}}


def _nvtx(push: bool):
    """NVTX range 'asp_timed' around the timed steps, so that a profiler can
    select exactly their launches (ncu --nvtx --nvtx-include asp_timed/)."""
    try:
        import torch
        if push:
            torch.cuda.nvtx.range_push("asp_timed")
        else:
            torch.cuda.nvtx.range_pop()
    except Exception:
        pass


def _workload(config: int, size: int, seed: int):
    import synth
    if config == 3:
        return synth.config3(seed, size=size or 4096)
    return synth.config2(seed, size=size or 1024)


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def aggregate(t_ms: float, iters: int, pevals: int, device) -> tuple:
    """Whole-job totals over the replicas: the slowest rank's time and the
    sum of every rank's work (identity on one process)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return t_ms, iters, pevals
    tt = torch.tensor([t_ms, float(iters), float(pevals)], dtype=torch.float64, device=device)
    mx = tt.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(tt, op=dist.ReduceOp.SUM)
    return float(mx[0]), int(tt[1]), int(tt[2])


# ---------------------------------------------------------------- cpu baseline (oracle)

def _oracle_sample(config: int, size: int, budget_s: float, seed: int = 0, resume=None):
    """Run the FP64 oracle's minor cycle on the same workload until budget_s
    has been spent (at least one iteration).  Returns (iterations, seconds,
    pixel_evals, state)."""
    import oracle as O
    case = _workload(config, size, seed)
    if resume is None:
        mc = O.MinorCycle(case.dirty, case.psf, O.AspParams(k_max=case.k_max, noise_sigma=case.noise_sigma,
                                                            gain=case.gain))
    else:
        mc = resume
    n0, pe0 = mc.t, sum(h["fit"].pixel_evals for h in mc.history)
    t0 = time.perf_counter()
    while True:
        if mc.step() is None:
            break
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    pe = sum(h["fit"].pixel_evals for h in mc.history) - pe0
    return mc.t - n0, dt, pe, mc


def _cpu_threads_env():
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[k] = "1"
    return env


def snapshot_states(asp, case, n_iter: int, n_snap: int, path: str):
    """States of the workload's run at n_snap iterations spread uniformly
    over [0, n_iter) (the GPU runs the cycle; each state is the residual,
    the component list, the retained list, t and the switch statistics), so
    that the oracle can be timed on iterations from the whole run."""
    import numpy as np
    import torch
    ctx = asp.Context(torch.from_numpy(case.dirty).cuda(), torch.from_numpy(case.psf).cuda(), k_max=case.k_max,
                      noise_sigma=case.noise_sigma, gain=case.gain, lm_max_iter=case.lm_max_iter)
    ab, wb, _, _ = ctx.beam
    data, t = {"beam": np.array([ab, wb])}, 0
    for i in range(n_snap):
        want = (i * n_iter) // n_snap
        if want > t:
            ctx.minor_cycle(want - t)
            t = want
        st = ctx.state()
        data[f"R{i}"] = ctx.residual()
        data[f"comps{i}"] = st["comps"]
        data[f"ret{i}"] = np.asarray(st["retained"], dtype=np.int64)
        data[f"meta{i}"] = np.array([st["t"], st["last_wi"], st["last_w0"]])
    ctx.close()
    np.savez(path, n=n_snap, **data)


def _oracle_on_snapshots(config: int, size: int, path: str, idx, budget_s: float):
    """Time the oracle's next iteration from each snapshot in idx (one
    iteration each, in order, until budget_s is spent; at least one).
    Returns (iterations, seconds, pixel_evals)."""
    import numpy as np
    import oracle as O
    case = _workload(config, size, 0)
    z = np.load(path)
    ab, wb = z["beam"]
    p = O.AspParams(k_max=case.k_max, noise_sigma=case.noise_sigma, gain=case.gain)
    n, dt, pe = 0, 0.0, 0
    for i in idx:
        mc = O.MinorCycle(case.dirty, case.psf, p, beam=(ab, wb))
        comps = [O.Component(c[0], c[1], c[2], c[3], c[4], bool(c[5])) for c in z[f"comps{i}"]]
        t, wi, w0 = z[f"meta{i}"]
        mc.set_state(z[f"R{i}"].astype(np.float64), comps, list(z[f"ret{i}"]), int(t), wi, w0)
        t0 = time.perf_counter()
        rec = mc.step()
        dt += time.perf_counter() - t0
        if rec is not None:
            n += 1
            pe += rec["fit"].pixel_evals
        if dt >= budget_s:
            break
    return n, dt, pe


def cpu_baseline(asp, config: int, case, n_iter: int, budget: float) -> dict:
    """The oracle as it stands, timed on iterations spread uniformly over the
    workload's run (each restarted from the GPU's state at that point):
    single-threaded until ``budget`` seconds, and on every host core at once
    (one single-threaded process per core, each on its own snapshots)."""
    n_cores = os.cpu_count() or 1
    n_snap = max(16, n_cores)
    fd, path = tempfile.mkstemp(suffix=".npz")
    os.close(fd)
    try:
        snapshot_states(asp, case, n_iter, n_snap, path)
        size = case.H

        def child(idx, b):
            code = ("import json,sys; sys.path.insert(0, %r); import bench; "
                    "print(json.dumps(bench._oracle_on_snapshots(%d, %d, %r, %r, %f)))"
                    % (ROOT, config, size, path, list(idx), b))
            return subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, text=True,
                                    env=_cpu_threads_env())

        # one thread: snapshots in an interleaved order (early and late
        # iterations alike) until the budget
        order = [i for k in range(4) for i in range(k, n_snap, 4)]
        pr = child(order, budget)
        out, _ = pr.communicate(timeout=budget * 30 + 900)
        n1, dt1, pe1 = json.loads(out.strip().splitlines()[-1])
        # all cores: every snapshot once, spread over the processes
        t0 = time.perf_counter()
        procs = [child(range(j, n_snap, n_cores), 1e9) for j in range(n_cores)]
        res = [json.loads(q.communicate(timeout=budget * 60 + 1800)[0].strip().splitlines()[-1]) for q in procs]
        wall = time.perf_counter() - t0
        nA = sum(r[0] for r in res)
        peA = sum(r[2] for r in res)
    finally:
        os.unlink(path)
    return {"value": n1 / dt1, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{n1} minor-cycle iterations of the {case.H}x{case.W} workload, each restarted from the GPU "
                      f"run's state at one of {n_snap} points spread uniformly over its {n_iter} iterations (FP64 "
                      f"NumPy oracle, 1 thread, {dt1:.1f} s)",
            "pixel_evals_per_s": pe1 / dt1,
            "all_cores": {"value": nA / wall, "unit": UNIT, "cores": n_cores,
                          "sample": f"all {n_snap} snapshot iterations, {n_cores} single-threaded processes, "
                                    f"{wall:.1f} s wall", "pixel_evals_per_s": peA / wall}}


# ---------------------------------------------------------------- reference arm

def run_reference(a):
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle as O  # noqa: F401  (the reference arm is the oracle itself)
    n_total, t_total, pe_total = 0, 0.0, 0
    state = None
    budget = max(2.0, min(a.cpu_budget, 15.0))
    # warm-up steps continue the same run (each step a bounded sample)
    for i in range(a.warmup + a.steps):
        n, dt, pe, state = _oracle_sample(a.config, a.size, budget, resume=state)
        if i >= a.warmup:
            n_total += n
            t_total += dt
            pe_total += pe
    value = n_total / t_total if t_total > 0 else 0.0
    case = _workload(a.config, a.size, 0)
    line = {"metric": _metric(case, a.config), "value": value, "unit": UNIT, "impl": "reference", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * t_total / max(a.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _config(case, a.config, a.iters or case.n_iter, world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{n_total} consecutive minor-cycle iterations after {a.warmup} warm-up "
                                       f"samples, {budget:.0f} s per step, 1 thread"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "pixel_evals_per_s": pe_total / t_total if t_total else 0.0}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- batched and learned comparisons

def batched_comparison(asp, n_images: int, seed0: int = 0, weights=None) -> dict:
    """The 64-image workload: config-1-style images of sizes drawn from
    {256, 512, 1024, 2048}^2, each with its own PSF and seed, 200 iterations.
    The batch (autotuned window tile, one launch per kernel, all fits in one
    cooperative launch) against the same images' own contexts run one after
    another; both from the dirty images, device-synchronised wall time.
    With trained weights the batch also runs with learned initial values
    (batched + learned against the same sequential plain runs)."""
    import numpy as np
    import synth
    cases = [synth.config4(seed0 + i) for i in range(n_images)]
    n_iter = cases[0].n_iter
    b = asp.Batch([c.dirty for c in cases], [c.psf for c in cases], noise_sigma=cases[0].noise_sigma,
                  k_max=cases[0].k_max)
    # the tile is chosen on the first eighth of the run: on the first 8
    # iterations alone (their large windows) it picked tiles that lost
    # over the whole run (1.06x instead of 1.41x the sequential runs)
    tune = b.autotune(max(8, n_iter // 8))
    # sequential: each image's own context (graph captured before the clock)
    b.reset()
    views = [b.image(i) for i in range(n_images)]
    for v in views:
        v.minor_cycle(0)
    t0 = time.perf_counter()
    seq = [v.minor_cycle(n_iter) for v in views]
    t_seq = time.perf_counter() - t0
    seq_rms = [float(np.sqrt(np.mean(v.residual().astype(np.float64) ** 2))) for v in views]
    b.reset()
    b.minor_cycle(0)
    l0 = b.launches()
    t0 = time.perf_counter()
    bat = b.minor_cycle(n_iter)
    t_bat = time.perf_counter() - t0
    launches = b.launches() - l0
    bat_rms = [float(np.sqrt(np.mean(b.image(i).residual().astype(np.float64) ** 2))) for i in range(n_images)]
    it_seq = sum(s["iterations"] for s in seq)
    it_bat = sum(s["iterations"] for s in bat)
    out = {"workload": f"config4: {n_images} images, sizes {{256,512,1024,2048}}^2, PSF sigma U[1.2,3], "
                       f"k_max {cases[0].k_max}, {n_iter} iterations each",
           "sizes": [int(c.H) for c in cases],
           "iterations_per_s": it_bat / t_bat, "sequential_iterations_per_s": it_seq / t_seq,
           "speedup": (it_bat / t_bat) / (it_seq / t_seq),
           "pixel_evals_per_s": sum(s["pixel_evals"] for s in bat) / t_bat,
           "sequential_pixel_evals_per_s": sum(s["pixel_evals"] for s in seq) / t_seq,
           "max_rms_ratio_batch_vs_sequential": max(x / y for x, y in zip(bat_rms, seq_rms)),
           "mean_rms_ratio_batch_vs_sequential": float(np.mean([x / y for x, y in zip(bat_rms, seq_rms)])),
           "gpu_launches": launches, "autotune": tune}
    # the work queue: every image's own minor cycle, images on CUDA streams
    queue = []
    for lanes, px in ((4, 0), (8, 0), (16, 0), (8, 768), (16, 768)):
        b.reset()
        b.run_queue(0, n_lanes=lanes, px_per_cta=px)          # graphs for this lane count and tile
        t0 = time.perf_counter()
        q = b.run_queue(n_iter, n_lanes=lanes, px_per_cta=px)
        t_q = time.perf_counter() - t0
        q_rms = [float(np.sqrt(np.mean(b.image(i).residual().astype(np.float64) ** 2))) for i in range(n_images)]
        it_q = sum(x["iterations"] for x in q)
        queue.append({"lanes": lanes, "px_per_cta": px, "iterations_per_s": it_q / t_q,
                      "speedup_vs_sequential": (it_q / t_q) / (it_seq / t_seq),
                      "mean_rms_ratio_vs_sequential": float(np.mean([x / y for x, y in zip(q_rms, seq_rms)])),
                      "max_rms_ratio_vs_sequential": max(x / y for x, y in zip(q_rms, seq_rms))})
    out["queue"] = {"runs": queue, "best": max(queue, key=lambda r: r["iterations_per_s"])}
    b.run_queue(0, n_lanes=1, px_per_cta=0)                   # the images' uncapped defaults back
    if weights is not None:
        b.set_mlp(weights)
        b.reset()
        b.minor_cycle(0)
        t0 = time.perf_counter()
        lrn = b.minor_cycle(n_iter)
        t_l = time.perf_counter() - t0
        l_rms = [float(np.sqrt(np.mean(b.image(i).residual().astype(np.float64) ** 2))) for i in range(n_images)]
        it_l = sum(x["iterations"] for x in lrn)
        out["learned"] = {"iterations_per_s": it_l / t_l, "speedup_vs_sequential_plain": (it_l / t_l) / (it_seq / t_seq),
                          "pixel_evals_per_s": sum(x["pixel_evals"] for x in lrn) / t_l,
                          "mean_rms_ratio_vs_plain": float(np.mean([x / y for x, y in zip(l_rms, seq_rms)])),
                          "lm_iters_per_fit": sum(x["lm_iters"] for x in lrn) / max(it_l, 1),
                          "plain_lm_iters_per_fit": sum(x["lm_iters"] for x in seq) / max(it_seq, 1),
                          "learned_fits": sum(x["learned_fits"] for x in lrn),
                          "learned_refits": sum(x["learned_refits"] for x in lrn)}
    b.close()
    return out


def elliptical_comparison(asp, reps: int = 20) -> dict:
    """The elliptical variant against the circular fit on one window of the
    1024x1024 workload's size: 12 rotated elliptical sources (widths 3-6 by
    1.5-2.9 px) over a ~150 px region, noise 1e-2; the same 12 members
    fitted as ellipses (6 parameters each) and as circles (4 each) from the
    same circular starts, each fit
    repeated ``reps`` times through the C ABI (per call: the launch, the
    device synchronisation and the result copy)."""
    import numpy as np
    import torch
    import synth
    H = W = 1024
    rng = np.random.default_rng(4)
    src = [(rng.uniform(0.3, 1.0) * rng.choice([-1, 1]), rng.uniform(450, 560), rng.uniform(450, 560),
            rng.uniform(3.0, 6.0), rng.uniform(1.5, 2.9), rng.uniform(-1.5, 1.5)) for _ in range(12)]
    dirty = synth.elliptical_field(H, W, src, 1e-2, 11).astype(np.float32)
    psf = synth.small_case(H, W, seed=5).psf
    ctx = asp.Context(torch.from_numpy(dirty).cuda(), torch.from_numpy(psf).cuda(), noise_sigma=1e-2, k_max=20)
    # both fits start from the same circles (what the peak search
    # proposes): width sqrt(s_major s_minor), so the ellipse fit has to find
    # each shape and orientation
    ell_init, circ_init = [], []
    for a, x, y, s1, s2, phi in src:
        w2 = s1 * s2
        ell_init.append([a, x, y, 1.0 / w2, 0.0, 1.0 / w2])
        circ_init.append([a, x, y, math.sqrt(w2)])
    out = {}
    for name, call, init, npm in (("elliptical", ctx.fit_elliptical, ell_init, 6), ("circular", ctx.fit, circ_init, 4)):
        call(init, 0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        infos = [call(init, 0)[1] for _ in range(reps)]
        t = (time.perf_counter() - t0) / reps
        it = infos[-1]["iters"]
        P = npm * len(init)
        pe = infos[-1]["pixel_evals"]
        flops = pe * ((P + 1) * (P + 2) + 20.0 * len(init))
        out[name] = {"ms_per_fit": t * 1e3, "lm_iters": it, "passes": infos[-1]["passes"], "pixel_evals": pe,
                     "us_per_lm_iter": t * 1e6 / max(it, 1), "status": infos[-1]["status"],
                     "chi2_final": infos[-1]["chi2_final"], "fp32_tflops": flops / t / 1e12,
                     "window": [infos[-1]["x0"], infos[-1]["x1"], infos[-1]["y0"], infos[-1]["y1"]]}
    ctx.close()
    out["members"] = 12
    out["us_per_lm_iter_ratio_ell_over_circ"] = out["elliptical"]["us_per_lm_iter"] / out["circular"]["us_per_lm_iter"]
    out["chi2_ratio_ell_over_circ"] = out["elliptical"]["chi2_final"] / out["circular"]["chi2_final"]
    out["note"] = ("fp32_tflops counts (P+1)(P+2) + 20 K flops per pixel evaluation (the SYRK's upper triangle as "
                   "FMAs plus the members' model and Jacobian), P = 6K or 4K")
    return out


def joint_comparison(asp, C: int = 32, reps: int = 10) -> dict:
    """The joint wide-band fit against per-channel fits: one field observed
    in C = 32 channels (the paper's data has 32) of 256x256, each channel's
    Gaussian PSF narrowing with frequency (sigma 2.0 .. 1.0 px), three
    members with power-law spectra (index -1 .. 1), noise 5e-3.  Joint: one
    fit of 3 (3 + C) parameters over all channels' windows.  Per channel:
    C independent circular fits of the same members (4 parameters each).
    Both from the same starts, each repeated ``reps`` times through the C
    ABI; reported: time per fit, LM iterations, and the spread of the
    members' fitted centres across channels (the joint fit shares one)."""
    import numpy as np
    import synth
    H = W = 256
    rng = np.random.default_rng(12)
    nu = np.linspace(1.0, 2.0, C)
    sig = 2.0 / nu
    members = [[rng.uniform(110, 146), rng.uniform(110, 146), rng.uniform(1.0, 3.0),
                *(rng.uniform(0.3, 1.0) * nu ** rng.uniform(-1, 1))] for _ in range(3)]
    dirty, psf = [], []
    for c in range(C):
        src = [(m[3 + c], m[0], m[1], math.hypot(m[2], sig[c]), math.hypot(m[2], sig[c]), 0.0) for m in members]
        dirty.append(synth.elliptical_field(H, W, src, 5e-3, 100 + c).astype(np.float32))
        psf.append(synth.gaussian_psf(H, W, sig[c]).astype(np.float32))
    b = asp.Batch(dirty, psf, noise_sigma=5e-3, k_max=5)
    init = np.array(members, float)
    init[:, 0] += 0.3
    init[:, 1] -= 0.2
    init[:, 2] *= 1.2
    init[:, 3:] *= 0.9
    b.fit_joint(init, 0)
    t0 = time.perf_counter()
    for _ in range(reps):
        out, flux, pt, info = b.fit_joint(init, 0)
    t_joint = (time.perf_counter() - t0) / reps
    views = [b.image(c) for c in range(C)]
    starts = [[[m[3 + c], m[0], m[1], math.hypot(m[2], sig[c])] for m in init] for c in range(C)]
    for c in range(C):
        views[c].fit(starts[c], 0)
    t0 = time.perf_counter()
    for _ in range(reps):
        per = [views[c].fit(starts[c], 0) for c in range(C)]
    t_per = (time.perf_counter() - t0) / reps
    xs = np.array([[r[1] for r in p[0]] for p in per])        # [C, K] centres of the per-channel fits
    b.close()
    return {"channels": C, "image": f"{H}x{W}", "members": len(members),
            "joint": {"ms": t_joint * 1e3, "lm_iters": info["iters"], "parameters": int(init.size),
                      "pixel_evals": info["pixel_evals"], "status": info["status"],
                      "us_per_lm_iter": t_joint * 1e6 / max(info["iters"], 1)},
            "per_channel": {"ms": t_per * 1e3, "fits": C, "lm_iters": int(sum(p[1]["iters"] for p in per)),
                            "centre_spread_px": float(np.max(xs.std(axis=0)))},
            "time_ratio_per_channel_over_joint": t_per / t_joint,
            "true_centres_x": [float(m[0]) for m in members], "joint_centres_x": [float(r[0]) for r in out]}


def learned_comparison(asp, n_train_images: int, seed: int = 0):
    """Learned initial values: harvest (patch, converged fit) pairs from
    GPU runs of config-1 and config-2-style images (seeds >= 10000), train
    the network on the GPU, then the equal-RMS protocol on the 1024x1024
    workload (plain for 2000 iterations gives RMS_p; learned until RMS <=
    1.01 RMS_p or 3000 iterations)."""
    from paper_1606_07872_gb300 import learned as L
    import synth
    t0 = time.perf_counter()
    X, T = L.harvest(L.default_training_cases(n_train_images, 2))
    t_h = time.perf_counter() - t0
    w = L.train(X, T, L.weight_init(seed), epochs=200, batch=1024, lr=1e-3)
    t_t = time.perf_counter() - t0 - t_h
    res = L.compare_equal_rms(synth.config2(0), w)
    p, q = res["plain"], res["learned"]
    return {"training_pairs": int(X.shape[0]), "harvest_s": t_h, "train_s": t_t,
            "plain": {k: p[k] for k in ("iterations", "seconds", "rms", "lm_iters_per_fit", "pixel_evals")},
            "learned": {k: q[k] for k in ("iterations", "seconds", "rms", "lm_iters_per_fit", "pixel_evals",
                                          "learned_fits", "learned_refits", "learned_kept")},
            "reached_equal_rms": bool(res["reached"]),
            "time_to_rms_ratio_plain_over_learned": res["time_ratio"],
            "lm_iters_per_fit_ratio_plain_over_learned": res["lm_iters_ratio"]}, w


# ---------------------------------------------------------------- our arm

def measure_workload(asp, case, n_iter, steps, warmup, local, world, flush, fit_px=0, major_every=0,
                     sub_mode=0) -> dict:
    """Device-timed steps (inputs resident in HBM), end-to-end steps through
    the C-ABI with host buffers, and one profiled step (CUDA events around
    every launch) of one workload on this rank."""
    import ctypes as C
    import torch
    dirty = torch.from_numpy(case.dirty).cuda()
    psf = torch.from_numpy(case.psf).cuda()
    stream = torch.cuda.Stream()
    params = asp.default_params(k_max=case.k_max, noise_sigma=case.noise_sigma, gain=case.gain,
                                lm_max_iter=case.lm_max_iter, fit_px_per_cta=fit_px, major_every=major_every,
                                sub_mode=sub_mode)
    with torch.cuda.stream(stream):
        ctx = asp.Context(dirty, psf, params=params, stream=stream)
    L = asp.lib()

    def reset(d_ptr, on_host, p_ptr=None, p_host=0):
        asp._check(L.asp_reset(ctx.h, d_ptr, on_host, p_ptr, p_host), "asp_reset", ctx.h)

    def step_device():
        reset(dirty.data_ptr(), 0, psf.data_ptr(), 0)
        return asp.asp_minor_cycle(ctx.h, n_iter)

    def launches():
        n = C.c_int64()
        L.asp_launch_count(ctx.h, C.byref(n))
        return n.value

    for _ in range(warmup):
        step_device()
    torch.cuda.synchronize()
    # ---- timed region (device-resident inputs)
    times, iters, pevals, fit_flops = [], 0, 0, 0.0
    l0 = launches()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    _nvtx(True)
    with ClockSampler(local) as clk:
        for _ in range(steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = step_device()
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            iters += st["iterations"]
            pevals += st["pixel_evals"]
            fit_flops += st["fit_flops"]
    torch.cuda.synchronize()
    _nvtx(False)
    n_launch = launches() - l0
    t_ms, iters, pevals = aggregate(sum(times), iters, pevals, "cuda")
    # ---- end to end through the C-ABI with host buffers
    dirty_h = torch.from_numpy(case.dirty).pin_memory()
    psf_h = torch.from_numpy(case.psf).pin_memory()
    res_h = torch.empty((case.H, case.W), dtype=torch.float32).pin_memory()
    e2e_ms, e2e_iters, comps_bytes = 0.0, 0, 0
    for _ in range(steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        reset(dirty_h.data_ptr(), 1, psf_h.data_ptr(), 1)
        st = asp.asp_minor_cycle(ctx.h, n_iter)
        asp.asp_copy_residual(ctx.h, res_h.numpy())
        comps = asp.asp_get_components(ctx.h)
        e1.record(stream)
        e1.synchronize()
        e2e_ms += e0.elapsed_time(e1)
        e2e_iters += st["iterations"]
        comps_bytes = comps.shape[0] * C.sizeof(asp.asp_component)
    e2e = {"value": e2e_iters / (e2e_ms / 1e3), "unit": UNIT,
           "h2d_bytes_per_step": int(case.dirty.nbytes + case.psf.nbytes),
           "d2h_bytes_per_step": int(res_h.numel() * 4 + comps_bytes)}
    # the run's outcome (the trajectory of discrete decisions depends on the
    # FP32 summation order, so the work per iteration is reported with it)
    import numpy as np
    res = res_h.numpy().astype(np.float64)
    outcome = {"final_residual_rms": float(np.sqrt(np.mean(res ** 2))), "components": int(comps.shape[0]),
               "model_flux": float(comps[:, 0].sum()) if comps.shape[0] else 0.0,
               "lm_iters_per_step": int(st["lm_iters"]), "pixel_evals_per_step": int(st["pixel_evals"])}
    # ---- per-kernel times (events around every launch, direct launches)
    L.asp_set_profiling(ctx.h, 1)
    step_device()
    kt = (asp._lib.asp_kernel_time * 32)()
    nk = C.c_int()
    L.asp_get_kernel_times(ctx.h, kt, 32, C.byref(nk))
    prof_stats = asp.asp_get_stats(ctx.h)
    L.asp_set_profiling(ctx.h, 0)
    ctx.close()
    kernels = {k.name.decode(): {"launches": k.launches, "total_ms": k.total_ms} for k in kt[: nk.value]}
    return {"t_ms": t_ms, "iters": iters, "pevals": pevals, "fit_flops": fit_flops, "n_launch": n_launch,
            "e2e": e2e, "outcome": outcome, "kernels": kernels, "prof": prof_stats, "clocks": clk.summary(),
            "n_iter": n_iter,
            "steps": steps, "N": case.H * case.W}


def rooflines(m: dict, peaks: dict, alu: dict) -> dict:
    """Achieved rate of each kernel class against its bound, from the
    profiled step: the method's algorithmic work (flops, exponentials,
    bytes) over the class's event-timed launch time."""
    k, st = m["kernels"], m["prof"]
    hbm = float(peaks["hbm_gbs"])
    fma = max(alu["fp32_fma_tflops"], alu["fp32_fma2_tflops"])
    ex2 = alu["ex2_gops"]
    out = {}
    if "k_lm_fit" in k:
        s = k["k_lm_fit"]["total_ms"] / 1e3
        pass_s = st["fit_pass_ms"] / 1e3
        out["k_lm_fit"] = {
            "bound": "alu", "unit": "TFLOP/s", "peak": fma,
            "achieved": st["fit_flops"] / s / 1e12, "frac": st["fit_flops"] / s / 1e12 / fma,
            "pixel_pass_only": {"achieved": st["fit_flops"] / pass_s / 1e12 if pass_s else None,
                                "frac": st["fit_flops"] / pass_s / 1e12 / fma if pass_s else None,
                                "note": "pixel-pass phase clocks of the fit kernel's first CTA"},
            "ex2": {"achieved_gops": st["fit_ex2"] / s / 1e9, "peak_gops": ex2, "frac": st["fit_ex2"] / s / 1e9 / ex2},
            "avg_launch_ms": k["k_lm_fit"]["total_ms"] / max(k["k_lm_fit"]["launches"], 1)}
    if k.get("k_sub_h", {}).get("launches") and k.get("k_sub_v_argmax", {}).get("launches"):
        s = (k["k_sub_h"]["total_ms"] + k["k_sub_v_argmax"]["total_ms"]) / 1e3
        out["k_sub_h+k_sub_v_argmax"] = {
            "bound": "hbm", "unit": "GB/s", "peak": hbm, "achieved": st["sub_bytes"] / s / 1e9,
            "frac": st["sub_bytes"] / s / 1e9 / hbm, "fp32_tflops": st["sub_flops"] / s / 1e12,
            "fp32_frac": st["sub_flops"] / s / 1e12 / fma,
            "bytes_note": "PSF regions read once + residual read and written once per iteration"}
    if k.get("subtraction (FFT)", {}).get("launches"):
        # one update: the forward transform's input (4N floats) and output
        # (2H (W+1) complex ~ 4N floats) once, the product's three complex
        # streams, the inverse transform's input and output once, R read and
        # written and the convolution's image quarter read: 124 N bytes
        kk = k["subtraction (FFT)"]
        s = kk["total_ms"] / 1e3
        by = 124.0 * m["N"] * kk["launches"]
        out["subtraction (FFT)"] = {"bound": "hbm", "unit": "GB/s", "peak": hbm, "achieved": by / s / 1e9,
                                    "frac": by / s / 1e9 / hbm, "us_per_update": kk["total_ms"] * 1e3 / kk["launches"],
                                    "bytes_note": "124 N bytes per update: each transform's input and output once, "
                                                  "the product's three streams, R read and written, the "
                                                  "convolution's image quarter read (cuFFT kernels included)"}
    if k.get("k_smooth_h", {}).get("launches") and k.get("k_smooth_v_argmax", {}).get("launches"):
        s = (k["k_smooth_h"]["total_ms"] + k["k_smooth_v_argmax"]["total_ms"]) / 1e3
        by = 4.0 * m["N"] * st["smooth_iters"]
        out["k_smooth_h+k_smooth_v_argmax"] = {
            "bound": "alu", "unit": "TFLOP/s", "peak": fma, "achieved": st["smooth_flops"] / s / 1e12,
            "frac": st["smooth_flops"] / s / 1e12 / fma, "hbm_gbs": by / s / 1e9, "hbm_frac": by / s / 1e9 / hbm,
            "bytes_note": "residual read once per smoothing iteration", "smoothing_iterations": st["smooth_iters"]}
    if "k_argmax_abs" in k and k["k_argmax_abs"]["launches"]:
        s = k["k_argmax_abs"]["total_ms"] / 1e3
        by = 4.0 * m["N"] * k["k_argmax_abs"]["launches"]
        out["k_argmax_abs"] = {"bound": "hbm", "unit": "GB/s", "peak": hbm, "achieved": by / s / 1e9,
                               "frac": by / s / 1e9 / hbm, "bytes_note": "residual read once per launch"}
    return out


def _metric(case, config: int) -> str:
    return f"minor-cycle iterations/s (Asp-Clean2016, {case.H}x{case.W}, active set <= {case.k_max})"


def _config(case, config: int, n_iter: int, world: int, sub: int = 0) -> dict:
    """The workload's config block; `residual_update` names the update form
    a default context of this size takes (the same in both arms, so that
    their configs compare equal)."""
    form = "fft" if (sub == 2 or (sub == 0 and case.H * case.W >= 512 * 512)) else "direct"
    return {"workload": f"config{config} {case.H}x{case.W} Asp-Clean2016 minor cycle, k_max {case.k_max}, "
                        f"{n_iter} iterations/step, gain {case.gain}",
            "global_batch": world, "seq_len": None, "parallelism": f"replicas x{world}",
            "l2": "flushed (256 MB write) between steps, outside timing", "residual_update": form}


def workload_line(a, m: dict, case, world: int, peaks: dict, peak_kind: str, alu: dict, name: str) -> dict:
    t_ms, iters = m["t_ms"], m["iters"]
    k = m["kernels"]
    dominant = max(k, key=lambda n: k[n]["total_ms"])
    roofs = rooflines(m, peaks, alu)
    traffic = _traffic_record()
    if dominant in ("k_sub_h", "k_sub_v_argmax"):
        key = "k_sub_h+k_sub_v_argmax"
    elif dominant in ("k_smooth_h", "k_smooth_v_argmax"):
        key = "k_smooth_h+k_smooth_v_argmax"
    else:
        key = dominant
    r = roofs.get(key, {})
    roof = {"bound": r.get("bound"), "achieved": r.get("achieved"), "peak": r.get("peak"), "unit": r.get("unit"),
            "frac": r.get("frac"), "kernel": key,
            "traffic": traffic.get(key, {}).get("bytes_per_launch"),
            "peak_source": ("measured by this run's own FP32 FMA microbenchmark (asp_measure_alu_peaks; the larger "
                            "of scalar and packed two-lane FMA)") if r.get("unit") == "TFLOP/s" else
                           f"{peak_kind}: MEASURED_PEAKS.json hbm_gbs (copy bandwidth)"}
    if key == "k_lm_fit":
        roof["pixel_pass_only"] = r["pixel_pass_only"]
        roof["ex2"] = r["ex2"]
        roof["avg_launch_ms"] = r["avg_launch_ms"]
    return {"metric": _metric(case, int(name[-1])),
            "value": iters / (t_ms / 1e3), "unit": UNIT, "n_gpus": world, "steps": m["steps"],
            "ms_per_step": t_ms / m["steps"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": _config(case, int(name[-1]), m["n_iter"], world),
            "pixel_evals_per_s": m["pevals"] / (t_ms / 1e3), "fit_tflops": m["fit_flops"] / (t_ms / 1e3) / 1e12,
            "e2e": m["e2e"], "outcome": m["outcome"], "gpu_launches": m["n_launch"], "roofline": roof,
            "kernel_rooflines": roofs,
            "kernels": k, "fit_phases": _fit_phases(m["prof"]), "clocks": m["clocks"]}


def asp2004_comparison(asp) -> dict:
    """The paper's Table 3 per-iteration comparison, on this GPU: one LM fit
    of the first component of a workload with Asp-Clean2004's objective
    (Eq. 3: the full PSF applied by FFT in every evaluation, whole image)
    and with Asp-Clean2016's (Eq. 6: the fitted Gaussian directly, local
    window), from the same smoothed-peak start; wall time per LM iteration
    (device-synchronised C-ABI calls, best of 3)."""
    import math
    import torch
    import synth
    out = {"paper_table3_per_iteration_ratio": {"uniform": 61.11, "natural": 101.21, "robust": 41.66,
                                                "note": "Python + CASA on a CPU, M31 256x256 (context)"}}
    for name, case in (("256x256 (config1)", synth.config1(0)), ("1024x1024 (config2)", synth.config2(0))):
        ctx = asp.Context(torch.from_numpy(case.dirty).cuda(), torch.from_numpy(case.psf).cuda(), k_max=case.k_max,
                          noise_sigma=case.noise_sigma)
        ab, wb, _, _ = ctx.beam
        pk = ctx.find_peak(asp.ASP_PEAK_SMOOTH)
        init6 = [[pk["a0"], pk["x0"], pk["y0"], pk["w0"]]]
        wi = math.sqrt(max(pk["w0"] ** 2 - wb * wb, 0.25))
        init3 = [[pk["a0"] * pk["w0"] ** 2 / (2 * math.pi * ab * wb * wb * wi * wi), pk["x0"], pk["y0"], wi]]
        res = {}
        for kind, call in (("eq6", lambda: ctx.fit(init6, 0)), ("eq3", lambda: ctx.fit_2004(init3, 0, 0.1))):
            best, info = None, None
            for _ in range(3):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                _, info = call()
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                best = dt if best is None else min(best, dt)
            res[kind] = {"seconds": best, "lm_iters": info["iters"], "passes": info["passes"],
                         "ms_per_lm_iter": 1e3 * best / max(info["iters"], 1)}
        res["per_iteration_ratio_eq3_over_eq6"] = res["eq3"]["ms_per_lm_iter"] / res["eq6"]["ms_per_lm_iter"]
        out[name] = res
        ctx.close()
    return out


SUB_MODES = {"auto": 0, "direct": 1, "fft": 2}


def sub_form_summary(m: dict, line: dict) -> dict:
    """The same workload with the direct residual update (separable passes)
    beside the measured line's form: rate, final RMS, the update's time."""
    t = m["t_ms"]
    k = m["kernels"]
    upd = lambda kk: sum(kk.get(n, {}).get("total_ms", 0.0) for n in ("k_sub_h", "k_sub_v_argmax", "subtraction (FFT)"))
    return {"value": m["iters"] / (t / 1e3), "unit": UNIT,
            "speedup_of_measured_form": line["value"] / (m["iters"] / (t / 1e3)),
            "rms_ratio_measured_over_direct": line["outcome"]["final_residual_rms"] / m["outcome"]["final_residual_rms"],
            "update_ms_per_step": {"direct": upd(k), "measured": upd(line.get("kernels", {}))},
            "outcome": m["outcome"]}


def split_summary(m: dict, exact_line: dict) -> dict:
    """The minor/major split against the exact-subtraction run of the same
    workload: rate, the final (exact) residual RMS and the kernel times."""
    t = m["t_ms"]
    return {"value": m["iters"] / (t / 1e3), "unit": UNIT, "e2e": m["e2e"], "outcome": m["outcome"],
            "speedup_vs_exact": (m["iters"] / (t / 1e3)) / exact_line["value"],
            "rms_ratio_vs_exact": m["outcome"]["final_residual_rms"] / exact_line["outcome"]["final_residual_rms"],
            "kernels": m["kernels"], "clocks": m["clocks"]}


def _sub_form(asp, case, sub: int) -> str:
    """The residual update form a context of this size takes."""
    if sub == SUB_MODES["auto"]:
        return "fft" if case.H * case.W >= asp.ASP_SUB_FFT_MIN_PIXELS else "direct"
    return "fft" if sub == SUB_MODES["fft"] else "direct"


def run_ours(a):
    import torch
    import paper_1606_07872_gb300 as asp
    from paper_1606_07872_gb300 import build as _b

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    _b.build()
    peaks, peak_kind = _peaks()
    alu = asp.asp_measure_alu_peaks()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    main_cfg = a.config
    case = _workload(main_cfg, a.size, rank)
    n_iter = a.iters or case.n_iter
    sub = SUB_MODES[a.sub]
    m = measure_workload(asp, case, n_iter, a.steps, a.warmup, local, world, flush, a.fit_px, 0, sub)
    line = workload_line(a, m, case, world, peaks, peak_kind, alu, f"config{main_cfg}")
    line["config"]["residual_update"] = _sub_form(asp, case, sub)
    line["warmup"] = a.warmup
    line["alu_peaks"] = dict(alu, note="own microbenchmark on this device, this run: one full wave of "
                                       "independent FMA / ex2.approx chains, CUDA-event timed")
    weights = None
    if main_cfg == 2 and not a.no_config3:
        try:
            c3 = _workload(3, 4096, rank)
            m3 = measure_workload(asp, c3, a.config3_iters or c3.n_iter, a.config3_steps, a.config3_warmup,
                                  local, world, flush, 0, 0, sub)
            line["config3"] = workload_line(a, m3, c3, world, peaks, peak_kind, alu, "config3")
            line["config3"]["warmup"] = a.config3_warmup
            line["config3"]["config"]["residual_update"] = _sub_form(asp, c3, sub)
            if not a.no_sub_forms and _sub_form(asp, c3, sub) == "fft":
                md = measure_workload(asp, c3, a.config3_iters or c3.n_iter, 1, 1, local, world, flush, 0, 0,
                                      SUB_MODES["direct"])
                line["config3"]["direct_update"] = sub_form_summary(md, line["config3"])
            del c3
        except Exception as e:   # report, never hide, a failed measurement
            line["config3"] = {"error": repr(e)[:300]}
    if not a.no_sub_forms and line["config"]["residual_update"] == "fft":
        try:
            md = measure_workload(asp, case, n_iter, a.steps, a.warmup, local, world, flush, a.fit_px, 0,
                                  SUB_MODES["direct"])
            line["direct_update"] = sub_form_summary(md, line)
        except Exception as e:   # report, never hide, a failed measurement
            line["direct_update"] = {"error": repr(e)[:300]}
    if main_cfg == 2 and not a.no_split:
        try:
            ms = measure_workload(asp, case, n_iter, a.steps, a.warmup, local, world, flush, a.fit_px, a.split_every)
            line["split"] = {"major_every": a.split_every, "config2": split_summary(ms, line)}
            if a.split_config3 and isinstance(line.get("config3"), dict) and "value" in line["config3"]:
                c3 = _workload(3, 4096, rank)
                m3 = measure_workload(asp, c3, a.config3_iters or c3.n_iter, a.config3_steps, a.config3_warmup,
                                      local, world, flush, 0, a.split_every)
                line["split"]["config3"] = split_summary(m3, line["config3"])
                del c3
        except Exception as e:   # report, never hide, a failed measurement
            line["split"] = {"error": repr(e)[:300]}
    if rank == 0 and main_cfg == 2 and not a.no_2004:
        try:
            line["asp2004"] = asp2004_comparison(asp)
        except Exception as e:   # report, never hide, a failed comparison
            line["asp2004"] = {"error": repr(e)[:300]}
    if rank == 0 and main_cfg == 2 and not a.no_elliptical:
        try:
            line["elliptical"] = elliptical_comparison(asp)
        except Exception as e:   # report, never hide, a failed comparison
            line["elliptical"] = {"error": repr(e)[:300]}
    if rank == 0 and main_cfg == 2 and not a.no_joint:
        try:
            line["joint"] = joint_comparison(asp)
        except Exception as e:   # report, never hide, a failed comparison
            line["joint"] = {"error": repr(e)[:300]}
    if rank == 0 and main_cfg == 2 and not a.no_learned:
        try:
            line["learned"], weights = learned_comparison(asp, a.learned_train_images)
        except Exception as e:   # report, never hide, a failed comparison
            line["learned"] = {"error": repr(e)[:300]}
    if rank == 0 and main_cfg == 2 and not a.no_batched:
        try:
            line["batched"] = batched_comparison(asp, a.batch_images, seed0=1000 * rank, weights=weights)
        except Exception as e:
            line["batched"] = {"error": repr(e)[:300]}
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        try:
            line["cpu_baseline"] = cpu_baseline(asp, main_cfg, case, n_iter, a.cpu_budget)
        except Exception as e:  # report, never hide, a failed baseline
            line["cpu_baseline"] = {"value": None, "error": repr(e)[:200]}
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line))
    return 0


def large_fit_probe(K: int) -> dict:
    """One LM step (the start's pass, one damped solve, the trial's pass) of
    K members over a ~950^2 window, timed as the mean of 5 calls after one
    (the first of the 6 is the one a profiler capturing launch 2 sees: the
    beam fit is launch 1): K circular sources of width 40 px
    (synth.elliptical_field, seed 0, noise 1e-2) on a 2048^2 image with a
    Gaussian PSF of width 2, context k_max 50; the start has the sources'
    amplitudes x 0.9, centres shifted by half a pixel and width 42."""
    import numpy as np
    import torch
    import paper_1606_07872_gb300 as asp
    import synth
    H = W = 2048
    rng = np.random.default_rng(0)
    src = [(rng.uniform(0.3, 1.0), rng.uniform(700, 1350), rng.uniform(700, 1350), 40.0, 40.0, 0.0)
           for _ in range(K)]
    dirty = synth.elliptical_field(H, W, src, 1e-2, 3).astype(np.float32)
    psf = synth.gaussian_psf(H, W, 2.0).astype(np.float32)
    ctx = asp.Context(torch.from_numpy(dirty).cuda(), torch.from_numpy(psf).cuda(), noise_sigma=1e-2, k_max=50)
    init = [[a * 0.9, x + 0.5, y - 0.5, 42.0] for a, x, y, *_ in src]
    _, info = ctx.fit_lm(init, 0, 1e-3, 1)[:2]
    torch.cuda.synchronize()
    reps = 5
    t0 = time.perf_counter()
    for _ in range(reps):
        _, info = ctx.fit_lm(init, 0, 1e-3, 1)[:2]
    t = (time.perf_counter() - t0) / reps
    ctx.close()
    P = 4 * K
    return {"members": K, "ms": t * 1e3, "info": info,
            "tflops": info["pixel_evals"] * (15 * K + 1 + (P + 1) * (P + 2)) / t / 1e12}


def main():
    a = _args()
    if a.large_fit:
        from paper_1606_07872_gb300 import build as _b
        _b.build()
        print(json.dumps(large_fit_probe(a.large_fit)))
        return 0
    if a.impl == "reference":
        return run_reference(a)
    return run_ours(a)


if __name__ == "__main__":
    sys.exit(main())
