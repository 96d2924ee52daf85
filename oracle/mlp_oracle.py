"""Learned initial values for the minor cycle -- FP64 NumPy oracle, TEST
INFRASTRUCTURE ONLY (imported by tests/, __graft_entry__.smoke() and
bench.py's baseline legs; never by the library).

The paper's initial values for a new component come from the residual's
peak (simple method) or from the peak of smoothed residuals (Sect. 2 step 1,
Sect. 3).  This module states the learned alternative that the CUDA path
implements next to them:

* input: the 32 x 32 patch of the residual centred on the peak p* of the
  plain method (rows y*-16 .. y*+15, columns x*-16 .. x*+15, zero outside
  the image), divided by |R(p*)|;
* network: x -> GELU(W1 x + b1) -> GELU(W2 h1 + b2) -> W3 h2 + b3 with
  1024 -> 256 -> 256 -> 4 units, GELU the exact erf form
  GELU(z) = z Phi(z) = z (1 + erf(z / sqrt 2)) / 2;
* output (the training target of a fit): (a / R(p*), log(omega / omega_b),
  x - x*, y - y*) for the converged new member (a, x, y, omega) of the
  active-set fit (Eq. 6);
* loss: mean squared error over the batch and the four outputs;
* optimiser: Adam (Kingma & Ba 2015) on FP32 master weights.

The GPU trains with BF16 tensor-core products for the two wide layers
(operands rounded to BF16, FP32 accumulation) and FP32 for the 256 -> 4
output layer.  ``bf16`` states that rounding (round to nearest, ties to
even) and ``forward``/``backward`` with round_bf16=True round exactly the
operands the GPU rounds, so the gradient check compares like with like.

Parity pins (tests/test_oracle_mlp.py): GELU against its closed-form values
and scipy's normal CDF; every gradient against central finite differences;
Adam's first step against its closed form (|step| = lr for every weight
with a non-zero gradient); bf16 rounding against exhaustive properties
(idempotent, monotone, ties to even, exact on BF16 values).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.special

PATCH = 32
N_IN, N_H1, N_H2, N_OUT = PATCH * PATCH, 256, 256, 4

__all__ = ["PATCH", "N_IN", "N_H1", "N_H2", "N_OUT", "MLPWeights", "gelu", "gelu_grad", "bf16", "forward",
           "backward", "mse", "adam_init", "adam_step", "extract_patch", "fit_target", "init_from_output"]


@dataclasses.dataclass
class MLPWeights:
    W1: np.ndarray   # (256, 1024)
    b1: np.ndarray   # (256,)
    W2: np.ndarray   # (256, 256)
    b2: np.ndarray   # (256,)
    W3: np.ndarray   # (4, 256)
    b3: np.ndarray   # (4,)

    def names(self):
        return ("W1", "b1", "W2", "b2", "W3", "b3")

    def copy(self) -> "MLPWeights":
        return MLPWeights(*(getattr(self, n).copy() for n in self.names()))


def gelu(z):
    """GELU(z) = z Phi(z), Phi the standard normal CDF (exact erf form)."""
    z = np.asarray(z, dtype=np.float64)
    return 0.5 * z * (1.0 + scipy.special.erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    """d GELU / dz = Phi(z) + z phi(z)."""
    z = np.asarray(z, dtype=np.float64)
    return 0.5 * (1.0 + scipy.special.erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def bf16(x):
    """Round to the nearest BF16 value (8-bit significand), ties to even,
    returned as float64.  Non-finite values pass through."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    return np.where(np.isfinite(f), out, f.astype(np.float64))


def forward(w: MLPWeights, X, round_bf16: bool = False):
    """Batch forward pass; X is (n, 1024).  With round_bf16 the operands of
    the two wide products (inputs, W1, h1, W2) are first rounded to BF16, as
    on the GPU; the output layer and all sums are exact.  Returns (Y, cache)."""
    r = bf16 if round_bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    X = np.asarray(X, dtype=np.float64)
    x0 = r(X)
    z1 = x0 @ r(w.W1).T + w.b1
    h1 = gelu(z1)
    z2 = r(h1) @ r(w.W2).T + w.b2
    h2 = gelu(z2)
    y = h2 @ w.W3.T + w.b3
    return y, dict(x0=x0, z1=z1, h1=r(h1), z2=z2, h2=h2, r=r)


def mse(Y, T):
    """Mean squared error over all entries and its gradient dL/dY."""
    Y = np.asarray(Y, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    d = Y - T
    return float(np.mean(d * d)), 2.0 * d / d.size


def backward(w: MLPWeights, cache, dY):
    """Gradients of the loss (given dL/dY) with respect to every weight
    (chain rule through the layers in reverse order).  With the forward's
    BF16 rounding, the wide products of the backward pass round their
    operands the same way (dz2, W2, dz1; the stored h1 and x0 are already
    rounded); the GELU derivative is taken at the unrounded z."""
    r = cache["r"]
    dY = np.asarray(dY, dtype=np.float64)
    g = {}
    g["W3"] = dY.T @ cache["h2"]
    g["b3"] = dY.sum(axis=0)
    dh2 = dY @ w.W3
    dz2 = dh2 * gelu_grad(cache["z2"])
    g["W2"] = r(dz2).T @ cache["h1"]
    g["b2"] = dz2.sum(axis=0)
    dh1 = r(dz2) @ r(w.W2)
    dz1 = dh1 * gelu_grad(cache["z1"])
    g["W1"] = r(dz1).T @ cache["x0"]
    g["b1"] = dz1.sum(axis=0)
    return MLPWeights(g["W1"], g["b1"], g["W2"], g["b2"], g["W3"], g["b3"])


def adam_init(w: MLPWeights):
    z = lambda a: np.zeros_like(a, dtype=np.float64)  # noqa: E731
    return dict(t=0, m=MLPWeights(*(z(getattr(w, n)) for n in w.names())),
                v=MLPWeights(*(z(getattr(w, n)) for n in w.names())))


def adam_step(w: MLPWeights, g: MLPWeights, state, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update in place: m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2,
    w <- w - lr m_hat / (sqrt(v_hat) + eps) with bias-corrected m_hat, v_hat."""
    state["t"] += 1
    t = state["t"]
    for n in w.names():
        m = getattr(state["m"], n)
        v = getattr(state["v"], n)
        gn = getattr(g, n)
        m[...] = beta1 * m + (1 - beta1) * gn
        v[...] = beta2 * v + (1 - beta2) * gn * gn
        mh = m / (1 - beta1 ** t)
        vh = v / (1 - beta2 ** t)
        p = getattr(w, n)
        p[...] = p - lr * mh / (np.sqrt(vh) + eps)


def extract_patch(R, px: int, py: int):
    """The 32 x 32 input patch at peak (px, py): rows py-16..py+15, columns
    px-16..px+15 of R, zero outside the image, divided by |R(py, px)|
    (row-major, length 1024)."""
    R = np.asarray(R, dtype=np.float64)
    H, W = R.shape
    out = np.zeros((PATCH, PATCH))
    y0, x0 = py - PATCH // 2, px - PATCH // 2
    ys, ye = max(0, y0), min(H, y0 + PATCH)
    xs, xe = max(0, x0), min(W, x0 + PATCH)
    out[ys - y0:ye - y0, xs - x0:xe - x0] = R[ys:ye, xs:xe]
    s = abs(R[py, px])
    return (out / s if s > 0 else out).reshape(-1)


def fit_target(theta_new, peak_value: float, px: int, py: int, omega_b: float):
    """Training target from the converged new member (a, x, y, omega)."""
    a, x, y, w = (float(v) for v in theta_new)
    return np.array([a / peak_value, math.log(w / omega_b), x - px, y - py])


def init_from_output(out, peak_value: float, px: int, py: int, omega_b: float):
    """Initial values (a0, x0, y0, omega0) from a network output."""
    o = np.asarray(out, dtype=np.float64)
    return np.array([o[0] * peak_value, px + o[2], py + o[3], omega_b * math.exp(o[1])])
