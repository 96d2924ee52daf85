"""Batched minor cycles (many independent images, one launch per kernel and
one cooperative launch for all LM fits) against single contexts and the
FP64 oracle."""
import numpy as np
import pytest

import oracle as O
import synth

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
    state on both sides, takes the oracle's discrete decisions and its
    residual update follows the oracle's (3e-4 relative L2 for a single
    member, 1e-2 for joint fits that may sit elsewhere in a flat valley)."""
    cases = _cases([11, 12, 13, 14], sizes=(64, 80, 96, 112))
    b = _batch(asp, cases, **TIGHT)
    views = [b.image(i) for i in range(len(cases))]
    ps = [O.AspParams(k_max=c.k_max, noise_sigma=c.noise_sigma, lm=O.lm_exact()) for c in cases]
    checked = 0
    for it in range(6):
        recs, befores = [], []
        for v, c, p in zip(views, cases, ps):
            ab, wb, _, _ = v.beam
            st = v.state()
            mc = O.MinorCycle(c.dirty, c.psf, p, beam=(ab, wb))
            comps = [O.Component(q[0], q[1], q[2], q[3], q[4], bool(q[5])) for q in st["comps"]]
            mc.set_state(v.residual().astype(np.float64), comps, st["retained"], st["t"], st["last_wi"],
                         st["last_w0"])
            befores.append(mc.R.copy())
            recs.append((mc, mc.step()))
        b.minor_cycle(1)
        for v, (mc, rec), R0 in zip(views, recs, befores):
            if rec is None:
                continue
            h = v.history()[-1]
            assert h["mode"] == rec["mode"]
            assert (h["x0"], h["x1"], h["y0"], h["y1"]) == tuple(rec["window"])
            assert h["k"] == len(rec["members"])
            if rec["fit"].status != O.LM_CONVERGED or h["status"] == O.LM_CAP:
                continue
            R = v.residual().astype(np.float64)
            assert _rel_l2(R - R0, mc.R - R0) < (3e-4 if len(rec["members"]) == 1 else 1e-2)
            checked += 1
    assert checked >= 8
    b.close()


def _teacher_forced(b, cases, n_iter, tight):
    """Per-image teacher-forced check (see test_batch_teacher_forced_per_image);
    returns the number of converged steps compared."""
    views = [b.image(i) for i in range(len(cases))]
    lm = O.lm_exact() if tight else O.LMParams()
    ps = [O.AspParams(k_max=c.k_max, noise_sigma=c.noise_sigma, lm=lm) for c in cases]
    checked = 0
    for it in range(n_iter):
        recs, befores = [], []
        for v, c, p in zip(views, cases, ps):
            ab, wb, _, _ = v.beam
            st = v.state()
            mc = O.MinorCycle(c.dirty, c.psf, p, beam=(ab, wb))
            comps = [O.Component(q[0], q[1], q[2], q[3], q[4], bool(q[5])) for q in st["comps"]]
            mc.set_state(v.residual().astype(np.float64), comps, st["retained"], st["t"], st["last_wi"],
                         st["last_w0"])
            befores.append(mc.R.copy())
            recs.append((mc, mc.step()))
        b.minor_cycle(1)
        for v, (mc, rec), R0 in zip(views, recs, befores):
            if rec is None:
                continue
            h = v.history()[-1]
            assert h["mode"] == rec["mode"]
            assert (h["x0"], h["x1"], h["y0"], h["y1"]) == tuple(rec["window"])
            assert h["k"] == len(rec["members"])
            if not tight or rec["fit"].status != O.LM_CONVERGED or h["status"] == O.LM_CAP:
                continue
            R = v.residual().astype(np.float64)
            assert _rel_l2(R - R0, mc.R - R0) < (3e-4 if len(rec["members"]) == 1 else 1e-2)
            checked += 1
    return checked


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
    assert _teacher_forced(b, cases, 4, tight=True) >= 4
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
