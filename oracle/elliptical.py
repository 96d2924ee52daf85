"""Elliptical beam and components -- TEST INFRASTRUCTURE ONLY (FP64 NumPy).

The paper writes every Gaussian as circular: width omega for the
components and the beam (Sect. 3, Eqs. 6-8).  Real beams are elliptical, and
the same method carries over with a 2 x 2 shape per Gaussian.  Reading (the
paper has no elliptical form; these are the natural generalisations, stated
once here and implemented the same way by the CUDA path):

* a member is ``a exp(-q / 2)``, ``q = A dx^2 + 2 B dx dy + C dy^2`` with
  ``(dx, dy)`` the offset from the centre ``(x0, y0)`` and ``P = [[A, B],
  [B, C]]`` the precision matrix (inverse covariance ``Sigma = P^-1``).
  Parameters per member: ``(a, x0, y0, A, B, C)``.  The exponent is linear
  in (A, B, C), so the Jacobian has no singular column where the ellipse
  becomes a circle (an angle parameter would);
* the objective is Eq. 6 with this model, minimised by the same
  Levenberg-Marquardt steps as the circular fit (``asp_oracle.lm_fit``);
* a trial point is usable when every value is finite, every centre lies in
  the window and P is positive definite with principal widths ``sigma =
  1 / sqrt(mu)`` (mu the eigenvalues of P) in (omega_min, window extent];
* the xtol scale is |a| (1 where a = 0) for the amplitude, the major
  width sigma_max for the centre and the mean diagonal precision (A + C) / 2
  for A, B and C;
* Eq. 7 becomes ``Sigma_i = Sigma_ic - Sigma_b`` (covariances add under
  convolution) and Eq. 8 flux conservation, ``F = a_ic sqrt(det Sigma_ic) /
  (alpha_b sqrt(det Sigma_b))``, ``a_i = F / (2 pi sqrt(det Sigma_i))``;
  the component is a point when the smaller eigenvalue of Sigma_ic -
  Sigma_b is at most 1e-3 times the smaller eigenvalue of Sigma_b (for a
  circular beam exactly the circular rule ``omega_ic^2 <= omega_b^2 (1 +
  1e-3)``);
* the beam: the circular beam fit of ``asp_oracle.beam_fit``, then the
  elliptical fit of the same main-lobe pixels started from it
  (``A = C = 1 / omega_b^2``, ``B = 0``).

Pins (tests/test_oracle_elliptical.py): the circular case term by term,
central finite differences of the Jacobian, exact recovery of noiseless
rotated ellipses, MINPACK on the same objective, and the convolution
identity against numerical 2-D convolution of sampled ellipses.
"""
from __future__ import annotations

import math
from typing import Optional

import numpy as np

from .asp_oracle import FitResult, LMParams, beam_fit, lm_fit

__all__ = ["NPM", "ell_model", "ell_model_and_jacobian", "ell_valid", "ell_step_scale", "ell_lm_fit",
           "ell_beam_fit", "ell_deconvolve", "ell_convolve_shape", "precision_from_axes", "axes_from_precision",
           "sigma_max", "ell_member_box"]

NPM = 6   # parameters per elliptical member: a, x0, y0, A, B, C


def precision_from_axes(s_major, s_minor, phi):
    """(A, B, C) of an ellipse with principal widths s_major >= s_minor and
    the major axis at angle phi from +x: Sigma = R diag(s_major^2,
    s_minor^2) R^T, P = Sigma^-1."""
    c, s = math.cos(phi), math.sin(phi)
    i1, i2 = 1.0 / (s_major * s_major), 1.0 / (s_minor * s_minor)
    return c * c * i1 + s * s * i2, c * s * (i1 - i2), s * s * i1 + c * c * i2


def axes_from_precision(A, B, C):
    """Inverse of :func:`precision_from_axes`: (s_major, s_minor, phi) with
    phi in (-pi/2, pi/2]."""
    mu, V = np.linalg.eigh(np.array([[A, B], [B, C]], dtype=np.float64))
    # the smaller precision eigenvalue belongs to the major axis
    v = V[:, 0]
    phi = math.atan2(v[1], v[0])
    if phi <= -math.pi / 2:
        phi += math.pi
    elif phi > math.pi / 2:
        phi -= math.pi
    return 1.0 / math.sqrt(mu[0]), 1.0 / math.sqrt(mu[1]), phi


def _mu(A, B, C):
    """Eigenvalues (mu_minus, mu_plus) of the precision matrix."""
    h = 0.5 * (A + C)
    r = math.hypot(0.5 * (A - C), B)
    return h - r, h + r


def sigma_max(A, B, C):
    """Major principal width 1 / sqrt(mu_minus) (inf if P is not positive
    definite)."""
    mm, _ = _mu(A, B, C)
    return 1.0 / math.sqrt(mm) if mm > 0 else math.inf


def ell_member_box(x, y, A, B, C):
    """The circular member box (asp_oracle.member_box) of the major width:
    half-size max(ceil(4 sigma_max), 5) around the rounded centre."""
    h = max(int(math.ceil(4.0 * sigma_max(A, B, C))), 5)
    rx, ry = int(math.floor(x + 0.5)), int(math.floor(y + 0.5))
    return rx - h, rx + h, ry - h, ry + h


def ell_model(theta, xs, ys):
    """Sum over members of ``a exp(-(A dx^2 + 2 B dx dy + C dy^2) / 2)``."""
    theta = np.asarray(theta, dtype=np.float64)
    out = np.zeros(np.broadcast(xs, ys).shape)
    for k in range(len(theta) // NPM):
        a, x0, y0, A, B, C = theta[NPM * k: NPM * k + NPM]
        dx = xs - x0
        dy = ys - y0
        out += a * np.exp(-0.5 * (A * dx * dx + 2.0 * B * dx * dy + C * dy * dy))
    return out


def ell_model_and_jacobian(theta, xs, ys):
    """Model and Jacobian (columns a, x0, y0, A, B, C per member):
    d/da = E, d/dx0 = g (A dx + B dy), d/dy0 = g (B dx + C dy),
    d/dA = -g dx^2 / 2, d/dB = -g dx dy, d/dC = -g dy^2 / 2, with E the
    unit-amplitude Gaussian and g = a E."""
    theta = np.asarray(theta, dtype=np.float64)
    K = len(theta) // NPM
    xs = np.asarray(xs, dtype=np.float64).ravel()
    ys = np.asarray(ys, dtype=np.float64).ravel()
    J = np.empty((xs.size, NPM * K))
    model = np.zeros(xs.size)
    for k in range(K):
        a, x0, y0, A, B, C = theta[NPM * k: NPM * k + NPM]
        dx = xs - x0
        dy = ys - y0
        e = np.exp(-0.5 * (A * dx * dx + 2.0 * B * dx * dy + C * dy * dy))
        g = a * e
        J[:, NPM * k] = e
        J[:, NPM * k + 1] = g * (A * dx + B * dy)
        J[:, NPM * k + 2] = g * (B * dx + C * dy)
        J[:, NPM * k + 3] = -0.5 * g * dx * dx
        J[:, NPM * k + 4] = -g * dx * dy
        J[:, NPM * k + 5] = -0.5 * g * dy * dy
        model += g
    return model, J


def ell_valid(theta, box, omega_min):
    """Trial-point test (module reading): finite, centres in the window,
    P positive definite with principal widths in (omega_min, extent]."""
    if not np.all(np.isfinite(theta)):
        return False
    x0b, x1b, y0b, y1b = box
    omega_max = max(x1b - x0b + 1, y1b - y0b + 1)
    for k in range(len(theta) // NPM):
        _, x, y, A, B, C = theta[NPM * k: NPM * k + NPM]
        if x < x0b or x > x1b or y < y0b or y > y1b:
            return False
        mm, mp = _mu(A, B, C)
        if not (mm > 0):
            return False
        # sigma_min > omega_min  <=>  mu_plus < 1 / omega_min^2;
        # sigma_max <= omega_max <=>  mu_minus >= 1 / omega_max^2
        if not (mp < 1.0 / (omega_min * omega_min)) or not (mm >= 1.0 / (omega_max * omega_max)):
            return False
    return True


def ell_step_scale(theta):
    """xtol scales (module reading): |a| (1 where 0), sigma_max for the
    centre, (A + C) / 2 for A, B and C."""
    theta = np.asarray(theta, dtype=np.float64)
    sc = np.empty_like(theta)
    for k in range(len(theta) // NPM):
        a, _, _, A, B, C = theta[NPM * k: NPM * k + NPM]
        sc[NPM * k] = abs(a) if a != 0 else 1.0
        smax = sigma_max(A, B, C)
        sc[NPM * k + 1] = smax
        sc[NPM * k + 2] = smax
        sc[NPM * k + 3: NPM * k + 6] = 0.5 * (A + C)
    return sc


def ell_lm_fit(T, xs, ys, theta0, box, omega_min, lm: Optional[LMParams] = None) -> FitResult:
    """Eq. 6 with elliptical members, the Levenberg-Marquardt steps of
    asp_oracle.lm_fit (Marquardt damping, accept on a chi^2 decrease, the
    same stopping rules) with the elliptical model, test and scales."""
    xs = np.asarray(xs, dtype=np.float64).ravel()
    ys = np.asarray(ys, dtype=np.float64).ravel()
    return lm_fit(T, xs, ys, theta0, box, omega_min, lm,
                  model_jac=lambda th: ell_model_and_jacobian(th, xs, ys),
                  valid=lambda th: ell_valid(th, box, omega_min), step_scale=ell_step_scale)


def ell_beam_fit(B, lm: Optional[LMParams] = None):
    """The elliptical beam (module reading): the circular beam fit, then the
    elliptical fit of the same main-lobe pixels (radius ceil(3 omega_init)
    around the zero lag, omega_init the half-maximum width) from
    (alpha_b, x_b, y_b, 1/omega_b^2, 0, 1/omega_b^2), trial widths above
    0.25 omega_init.  Returns (theta6, fit)."""
    from .asp_oracle import halfmax_width
    B = np.asarray(B, dtype=np.float64)
    H, W = B.shape[0] // 2, B.shape[1] // 2
    _, _, cfit = beam_fit(B, lm)
    w0 = halfmax_width(B)
    r = int(math.ceil(3.0 * w0))
    ys, xs = np.mgrid[H - r: H + r + 1, W - r: W + r + 1]
    inside = (xs - W) ** 2 + (ys - H) ** 2 <= r * r
    xs = xs[inside].astype(np.float64)
    ys = ys[inside].astype(np.float64)
    T = B[ys.astype(np.int64), xs.astype(np.int64)]
    a, x, y, w = cfit.theta
    theta0 = np.array([a, x, y, 1.0 / (w * w), 0.0, 1.0 / (w * w)])
    fit = ell_lm_fit(T, xs, ys, theta0, (W - r, W + r, H - r, H + r), 0.25 * w0, lm)
    return fit.theta.copy(), fit


def ell_convolve_shape(a_i, P_i, alpha_b, P_b):
    """The Gaussian (a_ic, P_ic) that a component (a_i, P_i) becomes when
    convolved with the beam (alpha_b, P_b) in the continuum: Sigma_ic =
    Sigma_i + Sigma_b and a_ic = a_i alpha_b 2 pi sqrt(det Sigma_i det
    Sigma_b / det Sigma_ic) (flux_ic = flux_i flux_b)."""
    Si = np.linalg.inv(np.asarray(P_i, dtype=np.float64))
    Sb = np.linalg.inv(np.asarray(P_b, dtype=np.float64))
    Sic = Si + Sb
    a_ic = a_i * alpha_b * 2.0 * math.pi * math.sqrt(np.linalg.det(Si) * np.linalg.det(Sb) / np.linalg.det(Sic))
    return a_ic, np.linalg.inv(Sic)


def ell_deconvolve(a_ic, P_ic, alpha_b, P_b):
    """Eqs. 7-8 for ellipses (module reading).  Returns (F, a_i, Sigma_i,
    is_point): Sigma_i = Sigma_ic - Sigma_b, F = a_ic sqrt(det Sigma_ic) /
    (alpha_b sqrt(det Sigma_b)), a_i = F / (2 pi sqrt(det Sigma_i)); a point
    (Sigma_i = 0, a_i = F) when the smaller eigenvalue of Sigma_ic - Sigma_b
    is at most 1e-3 times the smaller eigenvalue of Sigma_b."""
    Sic = np.linalg.inv(np.asarray(P_ic, dtype=np.float64))
    Sb = np.linalg.inv(np.asarray(P_b, dtype=np.float64))
    F = a_ic * math.sqrt(np.linalg.det(Sic)) / (alpha_b * math.sqrt(np.linalg.det(Sb)))
    Si = Sic - Sb
    if np.linalg.eigvalsh(Si)[0] <= 1e-3 * np.linalg.eigvalsh(Sb)[0]:
        return F, F, np.zeros((2, 2)), True
    return F, F / (2.0 * math.pi * math.sqrt(np.linalg.det(Si))), Si, False
