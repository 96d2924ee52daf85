"""Joint multi-channel (wide-band) fits -- TEST INFRASTRUCTURE ONLY (FP64).

The paper's data has many frequency channels (Sect. 4) and its motivation
is wide-band imaging (Sect. 1), but its fits are per image.  A joint fit
over C channels shares what the sky shares and lets the rest vary.  Reading
(not in the paper; the natural combination of Eq. 6 and Eqs. 7-8 over
channels, stated once here and implemented the same way by the CUDA path):

* every channel c has its own residual image R_c and PSF with circular beam
  (alpha_b_c, omega_b_c) (Sect. 3 per channel);
* a joint member k has a centre (x_k, y_k) and an intrinsic width s_k
  shared by all channels, and an image-plane amplitude a_kc per channel;
  in channel c it is the PSF-convolved Gaussian of Eq. 6,
  ``a_kc exp(-r^2 / (2 omega_kc^2))`` with ``omega_kc^2 = s_k^2 +
  omega_b_c^2`` (Eq. 7 solved for the convolved width);
* chi^2 is the sum over channels of Eq. 6's sum over the shared window
  (the union of the members' boxes of their widest convolved width);
* parameters per member (x, y, s, a_1 ... a_C); LM with the circular fit's
  rules; a trial point is usable when it is finite, the centres lie in the
  window and every convolved width is at most the window extent (s may
  reach 0: a point source); xtol scales: the widest convolved width for x,
  y and s, |a_kc| (1 where 0) for the amplitudes;
* per-channel flux by Eq. 8: ``F_kc = a_kc omega_kc^2 / (alpha_b_c
  omega_b_c^2)``; the member is a point when ``s_k^2 <= 1e-3 min_c
  omega_b_c^2`` (the circular point rule of the narrowest beam).

For C = 1 the joint fit is the paper's Eq. 6 fit reparameterised by Eq. 7
(omega_ic^2 = s^2 + omega_b^2): both reach the same optimum, the pin that
ties this module to the paper (tests/test_oracle_multichannel.py).
"""
from __future__ import annotations

from typing import Optional

import numpy as np

from .asp_oracle import FitResult, LMParams, lm_fit

__all__ = ["mc_model_and_jacobian", "mc_model", "mc_valid", "mc_step_scale", "mc_lm_fit", "mc_flux",
           "mc_window", "mc_stack"]


def _unpack(theta, C):
    th = np.asarray(theta, dtype=np.float64).reshape(-1, 3 + C)
    return th[:, 0], th[:, 1], th[:, 2], th[:, 3:]


def mc_model_and_jacobian(theta, xs, ys, chan, wb2):
    """Model and Jacobian over a stacked pixel list (xs, ys, chan: the
    channel of each pixel); wb2[c] = omega_b_c^2.  Columns per member:
    d/dx = g dx / omega^2, d/dy = g dy / omega^2, d/ds = g r^2 s / omega^4,
    d/da_kc = E on channel c's pixels (0 elsewhere)."""
    wb2 = np.asarray(wb2, dtype=np.float64)
    C = wb2.size
    x0, y0, s, a = _unpack(theta, C)
    K = x0.size
    xs = np.asarray(xs, dtype=np.float64).ravel()
    ys = np.asarray(ys, dtype=np.float64).ravel()
    chan = np.asarray(chan).ravel()
    NPM = 3 + C
    J = np.zeros((xs.size, NPM * K))
    model = np.zeros(xs.size)
    rows = np.arange(xs.size)
    for k in range(K):
        w2 = s[k] * s[k] + wb2[chan]
        dx = xs - x0[k]
        dy = ys - y0[k]
        r2 = dx * dx + dy * dy
        e = np.exp(-r2 / (2.0 * w2))
        g = a[k, chan] * e
        model += g
        J[:, NPM * k] = g * dx / w2
        J[:, NPM * k + 1] = g * dy / w2
        J[:, NPM * k + 2] = g * r2 * s[k] / (w2 * w2)
        J[rows, NPM * k + 3 + chan] = e
    return model, J


def mc_model(theta, xs, ys, chan, wb2):
    return mc_model_and_jacobian(theta, xs, ys, chan, wb2)[0]


def mc_valid(theta, box, wb2):
    """Trial-point test (module reading)."""
    if not np.all(np.isfinite(theta)):
        return False
    wb2 = np.asarray(wb2, dtype=np.float64)
    x0, y0, s, _ = _unpack(theta, wb2.size)
    x0b, x1b, y0b, y1b = box
    omega_max = max(x1b - x0b + 1, y1b - y0b + 1)
    for k in range(x0.size):
        if x0[k] < x0b or x0[k] > x1b or y0[k] < y0b or y0[k] > y1b:
            return False
        if s[k] * s[k] + wb2.max() > omega_max * omega_max:
            return False
    return True


def mc_step_scale(theta, wb2):
    """xtol scales (module reading): the widest convolved width for x, y and
    s; |a_kc| (1 where 0) for the amplitudes."""
    wb2 = np.asarray(wb2, dtype=np.float64)
    C = wb2.size
    th = np.asarray(theta, dtype=np.float64).reshape(-1, 3 + C)
    sc = np.empty_like(th)
    sc[:, :3] = np.sqrt(th[:, 2:3] ** 2 + wb2.max())
    a = np.abs(th[:, 3:])
    a[a == 0] = 1.0
    sc[:, 3:] = a
    return sc.ravel()


def mc_window(theta, wb2, H, W):
    """The shared fit window: the union of the circular member boxes
    (half-size max(ceil(4 omega), 5) around the rounded centre) of each
    member's widest convolved width, clipped to the image."""
    wb2 = np.asarray(wb2, dtype=np.float64)
    x0, y0, s, _ = _unpack(theta, wb2.size)
    b = []
    for k in range(x0.size):
        h = max(int(np.ceil(4.0 * np.sqrt(s[k] ** 2 + wb2.max()))), 5)
        rx, ry = int(np.floor(x0[k] + 0.5)), int(np.floor(y0[k] + 0.5))
        b.append((rx - h, rx + h, ry - h, ry + h))
    b = np.array(b)
    return max(b[:, 0].min(), 0), min(b[:, 1].max(), W - 1), max(b[:, 2].min(), 0), min(b[:, 3].max(), H - 1)


def mc_stack(images, box):
    """The window's pixels of every channel, stacked channel by channel
    (row-major within a channel): (T, xs, ys, chan)."""
    x0, x1, y0, y1 = box
    ys, xs = np.mgrid[y0:y1 + 1, x0:x1 + 1].astype(np.float64)
    T, X, Y, Cc = [], [], [], []
    for c, img in enumerate(images):
        T.append(np.asarray(img, dtype=np.float64)[y0:y1 + 1, x0:x1 + 1].ravel())
        X.append(xs.ravel())
        Y.append(ys.ravel())
        Cc.append(np.full(xs.size, c))
    return np.concatenate(T), np.concatenate(X), np.concatenate(Y), np.concatenate(Cc)


def mc_lm_fit(T, xs, ys, chan, theta0, box, wb2, lm: Optional[LMParams] = None) -> FitResult:
    """The joint fit: asp_oracle.lm_fit's Marquardt steps with the joint
    model, test and scales."""
    xs = np.asarray(xs, dtype=np.float64).ravel()
    ys = np.asarray(ys, dtype=np.float64).ravel()
    return lm_fit(T, xs, ys, theta0, box, 0.0, lm,
                  model_jac=lambda th: mc_model_and_jacobian(th, xs, ys, chan, wb2),
                  valid=lambda th: mc_valid(th, box, wb2), step_scale=lambda th: mc_step_scale(th, wb2))


def mc_flux(theta, alpha_b, wb2):
    """Eq. 8 per channel: F_kc = a_kc omega_kc^2 / (alpha_b_c omega_b_c^2),
    and the point flag s^2 <= 1e-3 min_c omega_b_c^2.  Returns (F [K, C],
    is_point [K])."""
    wb2 = np.asarray(wb2, dtype=np.float64)
    alpha_b = np.asarray(alpha_b, dtype=np.float64)
    _, _, s, a = _unpack(theta, wb2.size)
    w2 = s[:, None] ** 2 + wb2[None, :]
    F = a * w2 / (alpha_b[None, :] * wb2[None, :])
    return F, s * s <= 1e-3 * wb2.min()
