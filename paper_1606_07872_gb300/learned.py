"""Learned initial values: harvest training pairs from GPU minor cycles,
train the network on the GPU, and compare learned against plain starts at
equal final residual RMS.

Everything here is orchestration of library calls (contexts, the harvest
hook, the asp_mlp trainer); every step of the method and of the network runs
in the library's kernels.
"""
from __future__ import annotations

import time
from typing import Iterable, Optional, Sequence

import numpy as np

from . import ASP_STOP_ITER, Context, MLP


def harvest(cases: Iterable, n_iter: Optional[int] = None, converged_only: bool = True, params: Optional[dict] = None):
    """Run each synthetic case's minor cycle on the GPU (plain initial
    values) and collect (patch, target) pairs of its fits.  Returns X (n x
    1024) and T (n x 4), float32."""
    import torch
    Xs, Ts = [], []
    for case in cases:
        n = int(n_iter or case.n_iter)
        kw = dict(noise_sigma=case.noise_sigma, k_max=case.k_max)
        kw.update(params or {})
        ctx = Context(case.dirty, case.psf, **kw)
        P = torch.zeros((n, 1024), dtype=torch.float32, device="cuda")
        T = torch.zeros((n, 8), dtype=torch.float32, device="cuda")
        ctx.set_harvest(P, T)
        st = ctx.minor_cycle(n)
        m = int(st["iterations"])
        rec = T[:m].cpu().numpy()
        X = P[:m].cpu().numpy()
        keep = np.all(np.isfinite(rec[:, :4]), axis=1) & np.all(np.isfinite(X), axis=1)
        if converged_only:
            keep &= rec[:, 7] == 0
        # drop the tails: joint refits where the new member's amplitude or
        # position says little about the patch (ratio outside [-1, 4], more
        # than 8 px away, width beyond e^+-3 of the beam)
        keep &= (rec[:, 0] > -1.0) & (rec[:, 0] < 4.0) & (np.abs(rec[:, 1]) < 3.0)
        keep &= (np.abs(rec[:, 2]) < 8.0) & (np.abs(rec[:, 3]) < 8.0)
        Xs.append(X[keep])
        Ts.append(rec[keep, :4])
        ctx.close()
    return np.concatenate(Xs), np.concatenate(Ts)


def train(X, T, init: dict, epochs: int = 20, batch: int = 1024, lr: float = 1e-3, seed: int = 0,
          log=None) -> dict:
    """Adam on the GPU trainer over shuffled mini-batches.  The targets are
    standardised per output for training (mean mu, std sigma) and the
    standardisation is folded back into the output layer afterwards
    (W3 <- sigma W3, b3 <- sigma b3 + mu), so the returned FP32 weights map a
    patch to the targets themselves.  The learning rate decays linearly to
    a tenth over the epochs."""
    rng = np.random.default_rng(seed)
    T = np.asarray(T, dtype=np.float64)
    mu, sd = T.mean(axis=0), T.std(axis=0) + 1e-6
    net = MLP(init, max_batch=batch)
    net.set_data(X, (T - mu) / sd)
    n = X.shape[0]
    b = min(batch, n)
    for ep in range(epochs):
        perm = rng.permutation(n)
        losses = []
        lr_e = lr * (1.0 - 0.9 * ep / max(epochs - 1, 1))
        for i in range(0, n - b + 1, b):
            losses.append(net.step(perm[i:i + b], lr=lr_e, update=True))
        if log is not None:
            log(ep, float(np.mean(losses)))
    w = net.params()
    net.close()
    w["W3"] = (w["W3"] * sd[:, None]).astype(np.float32)
    w["b3"] = (w["b3"] * sd + mu).astype(np.float32)
    return w


def rms(ctx) -> float:
    R = ctx.residual().astype(np.float64)
    return float(np.sqrt(np.mean(R * R)))


def run_to_rms(case, weights: Optional[dict], target_rms: Optional[float], cap: int, chunk: int = 50,
               params: Optional[dict] = None):
    """Minor cycle (learned starts if weights) until the residual RMS reaches
    target_rms (checked every chunk iterations) or cap iterations.  Returns
    a dict: iterations, seconds (device-synchronised wall time of the
    minor-cycle calls), rms, lm_iters, pixel_evals, fits, learned counters."""
    kw = dict(noise_sigma=case.noise_sigma, k_max=case.k_max)
    kw.update(params or {})
    ctx = Context(case.dirty, case.psf, **kw)
    if weights is not None:
        ctx.set_mlp(weights)
    ctx.minor_cycle(0)                     # capture the graph outside the clock
    secs = 0.0
    st = ctx.stats()
    while st["iterations"] < cap:
        n = min(chunk, cap - st["iterations"])
        t0 = time.perf_counter()
        st = ctx.minor_cycle(n)
        secs += time.perf_counter() - t0
        if st["stop_reason"] not in (0, ASP_STOP_ITER) and st["iterations"] < cap:
            break                              # the noise test (or capacity) ended the run
        if target_rms is not None and rms(ctx) <= target_rms:
            break
    out = dict(iterations=int(st["iterations"]), seconds=secs, rms=rms(ctx), lm_iters=int(st["lm_iters"]),
               pixel_evals=int(st["pixel_evals"]), learned_fits=int(st["learned_fits"]),
               learned_refits=int(st["learned_refits"]), learned_kept=int(st["learned_kept"]))
    out["lm_iters_per_fit"] = out["lm_iters"] / max(out["iterations"], 1)
    ctx.close()
    return out


def compare_equal_rms(case, weights: dict, cap: Optional[int] = None, chunk: int = 50,
                      learned_cap_factor: float = 1.5) -> dict:
    """The equal-RMS protocol: plain for the cap gives RMS_p; the learned run
    goes until RMS <= 1.01 RMS_p, or learned_cap_factor times the cap (a
    learned run that needs more iterations than plain still gets its time to
    equal RMS measured, and loses on it)."""
    cap = int(cap or case.n_iter)
    plain = run_to_rms(case, None, None, cap, chunk)
    learned = run_to_rms(case, weights, 1.01 * plain["rms"], int(learned_cap_factor * cap), chunk)
    return dict(plain=plain, learned=learned,
                reached=learned["rms"] <= 1.01 * plain["rms"],
                time_ratio=plain["seconds"] / max(learned["seconds"], 1e-12),
                lm_iters_ratio=plain["lm_iters_per_fit"] / max(learned["lm_iters_per_fit"], 1e-12))


def default_training_cases(n_config1: int = 300, n_config2: int = 6, size2: int = 512, seed0: int = 10000):
    """Training images: config-1 and (smaller) config-2 style, seeds >= 10000
    (disjoint from the evaluation seeds)."""
    import synth
    cases = [synth.config1(seed0 + i) for i in range(n_config1)]
    cases += [synth.config2(seed0 + 500 + i, size=size2) for i in range(n_config2)]
    return cases


def weight_init(seed: int = 0) -> dict:
    import synth
    return {k: np.asarray(v, dtype=np.float32) for k, v in synth.mlp_init(seed).items()}


def summarize(res: dict) -> str:
    p, q = res["plain"], res["learned"]
    return (f"plain: {p['iterations']} it in {p['seconds']:.2f} s, rms {p['rms']:.4g}, "
            f"{p['lm_iters_per_fit']:.1f} LM it/fit | learned: {q['iterations']} it in {q['seconds']:.2f} s, "
            f"rms {q['rms']:.4g}, {q['lm_iters_per_fit']:.1f} LM it/fit, fits {q['learned_fits']} "
            f"refits {q['learned_refits']} | time ratio {res['time_ratio']:.2f}")


__all__: Sequence[str] = ("harvest", "train", "run_to_rms", "compare_equal_rms", "default_training_cases",
                          "weight_init", "summarize")
