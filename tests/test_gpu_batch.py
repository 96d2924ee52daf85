"""Batched minor cycles (many independent images, one launch per kernel and
one cooperative launch for all LM fits) against single contexts and the
FP64 oracle."""
import numpy as np
import pytest

import oracle as O
import synth
from tests import teacher

pytestmark = pytest.mark.gpu

TIGHT = dict(lm_max_iter=300, lm_rtol=1e-12, lm_xtol=1e-10)


def _cases(seeds, sizes):
    return [synth.config4(s, sizes=sizes) for s in seeds]


def _batch(asp, cases, **kw):
    kw.setdefault("noise_sigma", cases[0].noise_sigma)
    kw.setdefault("k_max", cases[0].k_max)
    return asp.Batch([c.dirty for c in cases], [c.psf for c in cases], **kw)


def _rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, float) - np.asarray(b, float)) / max(np.linalg.norm(b), 1e-300))


# 768 window pixels per CTA: a 128 x 128 window takes 22 CTAs, below the
# equal share of 3 images, so batch and single contexts use the same grids
SAME_GRID = dict(fit_px_per_cta=768)


def test_batch_equals_single_contexts_bit_exact(asp):
    """With fit groups at least as large as a single context's fit grid,
    every batch image computes exactly what its own context computes: same
    kernels, same buffers, same reduction order."""
    cases = _cases([1, 2, 3], sizes=(64, 96, 128))
    b = _batch(asp, cases, **SAME_GRID)
    stats = b.minor_cycle(25)
    for i, c in enumerate(cases):
        ctx = asp.Context(c.dirty, c.psf, noise_sigma=c.noise_sigma, k_max=c.k_max, **SAME_GRID)
        st = ctx.minor_cycle(25)
        img = b.image(i)
        assert stats[i]["iterations"] == st["iterations"]
        assert stats[i]["pixel_evals"] == st["pixel_evals"]
        np.testing.assert_array_equal(img.residual(), ctx.residual())
        np.testing.assert_array_equal(img.components(), ctx.components())
        ctx.close()
    b.close()


def test_batch_teacher_forced_per_image(asp):
    """Every image of a batch, started each iteration from the GPU's own
    state on both sides, takes the oracle's discrete decisions, its
    residual update is the oracle's subtraction of its fitted components
    (1e-5 relative L2) and its converged fits sit at the oracle's optimum
    (1e-4, or the FP32 floor; tests/teacher.py)."""
    cases = _cases([11, 12, 13, 14], sizes=(64, 80, 96, 112))
    b = _batch(asp, cases, **TIGHT)
    stats = _teacher_forced(b, cases, 6, tight=True)
    assert stats.fits >= 8 and stats.updates >= 20
    b.close()


def _teacher_forced(b, cases, n_iter, tight, sample_px=None, step=None):
    """Per-image teacher-forced checks of n_iter batch iterations (see
    tests/teacher.py; step() advances every image by one, by default one
    lock-step batch iteration); returns the statistics."""
    views = [b.image(i) for i in range(len(cases))]
    lm = O.lm_exact() if tight else O.LMParams()
    ps = [O.AspParams(k_max=c.k_max, noise_sigma=c.noise_sigma, lm=lm) for c in cases]
    stats = teacher.Stats()
    rng = np.random.default_rng(5)
    for it in range(n_iter):
        recs = []
        for v, c, p in zip(views, cases, ps):
            ab, wb, _, _ = v.beam
            mc, st = teacher.oracle_from_state(v, c, p, (ab, wb))
            recs.append((teacher.oracle_iteration(mc), mc.R.copy(), st))
        if step is None:
            b.minor_cycle(1)
        else:
            step()
        for v, c, (rec, R0, st) in zip(views, cases, recs):
            if rec is None:
                continue
            big = c.H * c.W > 512 * 512
            teacher.check_iteration(v, c, rec, R0, st, stats, sample_px=(sample_px if big else None), rng=rng)
    return stats


def test_batch_teacher_forced_large_images(asp, capsys):
    """A batch holding one 1024^2 and one 2048^2 image of the 64-image
    workload's kind beside two small ones, default LM settings: each image's
    iterations are checked as in test_batch_teacher_forced_per_image (the
    large images' residual updates at sampled pixels against the
    brute-force 2-D direct subtraction), with the CTA groups the on-demand
    policy sizes from 2048^2 windows."""
    cases = [synth.config4(s, sizes=(n,)) for s, n in ((51, 1024), (52, 2048), (53, 128), (54, 256))]
    b = _batch(asp, cases)
    b.autotune(2)
    stats = _teacher_forced(b, cases, 3, tight=False, sample_px=256)
    assert stats.updates >= 10
    with capsys.disabled():
        print(f"\nbatch with 1024^2 and 2048^2 images: {stats.updates} updates (max rel L2 "
              f"{stats.max_rel_update:.2e}), {stats.fits} converged fits")
    b.close()


def test_batch_autotune_then_parity(asp):
    """The autotuner picks a window tile (pixels per CTA) and CTA-group
    policy by timing trial iterations from a reset; it changes only how
    the fits are spread over CTAs, so after it every image still takes the
    oracle's decisions step by step."""
    cases = _cases([21, 22, 23], sizes=(64, 96, 128))
    b = _batch(asp, cases, **TIGHT)
    t = b.autotune(4)
    assert t["n_candidates"] == 18 and t["best_ms"] > 0 and t["default_ms"] > 0
    assert t["px_per_cta"] in (0, 48, 192, 384, 768, 1536) and t["share_policy"] in (0, 1, 2)
    assert b.minor_cycle(0)[0]["iterations"] == 0          # the tuner leaves the batch reset
    assert _teacher_forced(b, cases, 4, tight=True).fits >= 4
    assert b.launches() > 0
    b.close()


def test_batch_images_stop_independently(asp):
    """An image that runs out of signal above the 3 sigma threshold stops on
    its own noise test while the other continues; each keeps its own
    iteration count."""
    quiet = synth.small_case(48, 48, seed=5, n_points=1, n_gauss=0, noise_sigma=1e-5)
    busy = synth.config4(31, sizes=(96,))
    b = asp.Batch([quiet.dirty, busy.dirty], [quiet.psf, busy.psf], noise_sigma=1e-3, k_max=5)
    st = b.minor_cycle(40)
    assert st[0]["stop_reason"] == asp.ASP_STOP_NOISE and st[0]["iterations"] < 40
    assert st[1]["iterations"] == 40
    b.close()


def test_batch_invalid_arguments(asp):
    c = synth.config4(1, sizes=(64,))
    with pytest.raises(ValueError):
        asp.Batch([c.dirty], [])
    with pytest.raises(ValueError):
        asp.Batch([c.dirty], [c.psf[:10, :10]])          # PSF must be 2H x 2W


def test_batch_learned_equals_single_contexts(asp):
    """Learned initial values in a batch (one network pass for all images
    per iteration) give every image exactly what its own context with the
    same network computes."""
    cases = _cases([41, 42, 43], sizes=(64, 96, 128))
    w = {k: np.asarray(v, dtype=np.float32) for k, v in synth.mlp_init(2).items()}
    b = _batch(asp, cases, **SAME_GRID)
    b.set_mlp(w)
    stats = b.minor_cycle(12)
    assert all(s["learned_fits"] > 0 for s in stats)
    for i, c in enumerate(cases):
        ctx = asp.Context(c.dirty, c.psf, noise_sigma=c.noise_sigma, k_max=c.k_max, **SAME_GRID)
        ctx.set_mlp(w)
        st = ctx.minor_cycle(12)
        for k in ("iterations", "learned_fits", "learned_refits", "learned_kept", "pixel_evals"):
            assert stats[i][k] == st[k], k
        np.testing.assert_array_equal(b.image(i).residual(), ctx.residual())
        ctx.close()
    b.close()


def test_work_queue_equals_each_images_own_run(asp):
    """The work queue (images on 4 CUDA streams, each running its own minor
    cycle) computes exactly what each image's context computes alone with
    the same fit grid cap and window tile: the lanes share no state."""
    cases = _cases([21, 22, 23, 24, 25, 26], sizes=(64, 96, 128, 256))
    b = _batch(asp, cases)
    stats = b.run_queue(30, n_lanes=4, px_per_cta=768)
    res = [b.image(i).residual() for i in range(len(cases))]
    comps = [b.image(i).components() for i in range(len(cases))]
    b.reset()
    for i in range(len(cases)):
        st = b.image(i).minor_cycle(30)        # the image's own context, one after another
        assert st["iterations"] == stats[i]["iterations"] and st["pixel_evals"] == stats[i]["pixel_evals"]
        np.testing.assert_array_equal(b.image(i).residual(), res[i])
        np.testing.assert_array_equal(b.image(i).components(), comps[i])
    b.close()


def test_work_queue_teacher_forced_large_images(asp):
    """Queue mode at config-4 sizes (a 1024^2 and a 2048^2 image beside two
    small ones, default LM settings): every image's iterations,
    teacher-forced, agree with the oracle -- decisions exactly, residual
    updates within 1e-5 relative L2 (the large images' at sampled pixels
    against the brute-force direct subtraction)."""
    cases = [synth.config4(s, sizes=(z,)) for s, z in ((31, 256), (32, 1024), (33, 2048), (34, 512))]
    b = _batch(asp, cases)
    b.run_queue(3, n_lanes=3)
    stats = _teacher_forced(b, cases, 2, tight=False, sample_px=256, step=lambda: b.run_queue(1, n_lanes=3))
    assert stats.updates >= 6
    b.close()
