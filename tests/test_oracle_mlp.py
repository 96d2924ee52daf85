"""Pins of the learned-initial-value oracle (oracle/mlp_oracle.py) to things
other than itself: closed forms, finite differences, exhaustive rounding
properties."""
import math

import numpy as np
import pytest
import scipy.stats

from oracle import mlp_oracle as M


def _weights(seed=0, scale=1.0):
    rng = np.random.default_rng(seed)
    return M.MLPWeights(rng.normal(0, 0.03 * scale, (256, 1024)), rng.normal(0, 0.1, 256),
                        rng.normal(0, 0.06 * scale, (256, 256)), rng.normal(0, 0.1, 256),
                        rng.normal(0, 0.06 * scale, (4, 256)), rng.normal(0, 0.1, 4))


def test_gelu_closed_forms():
    z = np.array([-3.0, -1.0, -0.5, 0.0, 0.5, 1.0, 3.0])
    np.testing.assert_allclose(M.gelu(z), z * scipy.stats.norm.cdf(z), rtol=1e-15, atol=1e-16)
    assert M.gelu(0.0) == 0.0
    assert M.gelu(1.0) == pytest.approx(0.8413447460685429, abs=1e-15)
    # GELU(z) - GELU(-z) = z because Phi(z) + Phi(-z) = 1
    zz = np.linspace(-6, 6, 101)
    np.testing.assert_allclose(M.gelu(zz) - M.gelu(-zz), zz, atol=1e-14)


def test_gelu_grad_is_the_derivative():
    z = np.linspace(-5, 5, 41)
    h = 1e-6
    fd = (M.gelu(z + h) - M.gelu(z - h)) / (2 * h)
    np.testing.assert_allclose(M.gelu_grad(z), fd, rtol=1e-8, atol=1e-9)


@pytest.mark.parametrize("rounded", [False, True])
def test_backward_matches_finite_differences(rounded):
    """Every weight block's gradient agrees with central differences of the
    loss (FP64, no rounding: the chain rule itself).  With BF16 rounding the
    loss is piecewise constant in everything upstream of a rounded operand
    (W1, b1, W2 through the rounded x0, h1, W2), so that case is checked on
    the continuous part: b2 and the FP32 output layer."""
    w = _weights(1)
    rng = np.random.default_rng(2)
    X = rng.normal(0, 1, (6, 1024))
    T = rng.normal(0, 1, (6, 4))
    Y, c = M.forward(w, X, round_bf16=rounded)
    _, dY = M.mse(Y, T)
    g = M.backward(w, c, dY)
    picks = [("b2", (200,)), ("W3", (1, 30)), ("b3", (3,))]
    if not rounded:
        picks += [("b1", (5,)), ("W1", (3, 17)), ("W1", (255, 1023)), ("W2", (7, 9)), ("W2", (0, 255))]
    for name, idx in picks:
        p = getattr(w, name)
        old = p[idx]
        h = 1e-6 * max(1.0, abs(old))
        p[idx] = old + h
        lp = M.mse(M.forward(w, X, round_bf16=rounded)[0], T)[0]
        p[idx] = old - h
        lm = M.mse(M.forward(w, X, round_bf16=rounded)[0], T)[0]
        p[idx] = old
        fd = (lp - lm) / (2 * h)
        assert getattr(g, name)[idx] == pytest.approx(fd, rel=1e-5, abs=1e-11), (name, idx)


def test_mse_gradient():
    Y = np.array([[1.0, 2.0], [3.0, 5.0]])
    T = np.array([[0.0, 2.0], [3.0, 1.0]])
    L, d = M.mse(Y, T)
    assert L == pytest.approx((1 + 16) / 4)
    np.testing.assert_allclose(d, 2 * (Y - T) / 4)


def test_bf16_rounding_properties():
    rng = np.random.default_rng(3)
    x = rng.normal(0, 1, 20000) * np.exp(rng.uniform(-20, 20, 20000))
    r = M.bf16(x)
    np.testing.assert_array_equal(M.bf16(r), r)                       # idempotent
    rel = np.abs(r - x.astype(np.float32)) / np.abs(x.astype(np.float32))
    assert rel.max() <= 2.0 ** -8 * (1 + 1e-7)                         # unit roundoff of an 8-bit significand
    s = np.sort(x)
    assert np.all(np.diff(M.bf16(s)) >= 0)                             # monotone
    # every BF16 value is exact (top 16 bits of a float32, low 16 zero)
    bits = (rng.integers(0, 2 ** 16, 5000, dtype=np.uint64) << 16).astype(np.uint32)
    v = bits.view(np.float32).astype(np.float64)
    v = v[np.isfinite(v)]
    np.testing.assert_array_equal(M.bf16(v), v)
    # ties go to the even significand
    assert M.bf16(1.0 + 2.0 ** -8) == 1.0
    assert M.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6
    assert M.bf16(-(1.0 + 2.0 ** -8)) == -1.0


def test_adam_first_step_closed_form():
    """From zero moments the bias-corrected first step is lr g / (|g| + eps):
    every weight with a non-zero gradient moves by lr against its sign."""
    w = _weights(4)
    w0 = w.copy()
    rng = np.random.default_rng(5)
    g = M.MLPWeights(*(rng.normal(0, 1, getattr(w, n).shape) for n in w.names()))
    st = M.adam_init(w)
    M.adam_step(w, g, st, lr=1e-3)
    for n in w.names():
        d = getattr(w, n) - getattr(w0, n)
        gn = getattr(g, n)
        np.testing.assert_allclose(d, -1e-3 * gn / (np.abs(gn) + 1e-8), rtol=1e-12)


def test_patch_padding_and_scale():
    R = np.arange(40 * 50, dtype=float).reshape(40, 50) - 1000.0
    p = M.extract_patch(R, 3, 2).reshape(32, 32)
    assert p[16, 16] == pytest.approx(R[2, 3] / abs(R[2, 3]))
    assert np.all(p[:14, :] == 0) and np.all(p[:, :13] == 0)          # rows < 0 and columns < 0
    np.testing.assert_allclose(p[14:, 13:], R[0:18, 0:19] / abs(R[2, 3]))
    q = M.extract_patch(R, 49, 39).reshape(32, 32)
    assert np.all(q[24:, :] == 0) and np.all(q[:, 17:] == 0)          # beyond the last row / column


def test_target_and_init_are_inverse():
    theta = np.array([0.37, 101.25, 55.5, 3.2])
    t = M.fit_target(theta, 0.5, 100, 56, 2.0)
    np.testing.assert_allclose(t, [0.74, math.log(1.6), 1.25, -0.5])
    np.testing.assert_allclose(M.init_from_output(t, 0.5, 100, 56, 2.0), theta)


# ---------------------------------------------------------------- the learned step of the minor cycle

def _const_net(b3):
    """A network whose output is the constant b3 (zero weights)."""
    return M.MLPWeights(np.zeros((256, 1024)), np.zeros(256), np.zeros((256, 256)), np.zeros(256),
                        np.zeros((4, 256)), np.asarray(b3, dtype=np.float64))


def _run(case, mlp, n=5, mode="simple"):
    import oracle as O
    mc = O.MinorCycle(case.dirty, case.psf, O.AspParams(k_max=3, noise_sigma=case.noise_sigma, init_mode=mode),
                      mlp=mlp)
    recs = [mc.step() for _ in range(n)]
    return mc, recs


def test_learned_step_reproducing_the_plain_start_changes_nothing():
    """A network that proposes exactly the simple method's start (a0 = R(p*),
    omega0 = omega_b, the peak pixel) gives the plain run, fit for fit."""
    import synth
    case = synth.small_case(64, 72, seed=4)
    plain, rp = _run(case, None)
    learn, rl = _run(case, _const_net([1.0, 0.0, 0.0, 0.0]))
    for a, b in zip(rp, rl):
        assert b["learned"]["used"] and b["learned"]["kept"]
        np.testing.assert_allclose(a["fit"].theta, b["fit"].theta, rtol=0, atol=0)
    np.testing.assert_array_equal(plain.R, learn.R)


def test_learned_proposal_outside_the_window_is_not_used():
    import synth
    case = synth.small_case(64, 72, seed=4)
    _, rp = _run(case, None)
    _, rl = _run(case, _const_net([1.0, 0.0, 1e6, 0.0]))
    for a, b in zip(rp, rl):
        assert not b["learned"]["used"]
        np.testing.assert_array_equal(a["fit"].theta, b["fit"].theta)


def test_learned_fallback_keeps_the_better_fit():
    """A start far from the source (wrong sign, 6 px off, 5x too wide) ends in
    a worse minimum or at the cap: the plain start is refitted and the lower
    chi^2 kept, so the result is never worse than the plain fit."""
    import synth
    case = synth.small_case(64, 72, seed=4)
    _, rp = _run(case, None, n=3)
    _, rl = _run(case, _const_net([-3.0, np.log(5.0), 6.0, -6.0]), n=3)
    assert any(b["learned"]["refit"] for b in rl)
    for a, b in zip(rp, rl):
        assert b["fit"].chi2 <= a["fit"].chi2 * (1 + 1e-9)
