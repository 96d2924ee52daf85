"""Seeded sky models, PSFs and dirty images (data only, no method arithmetic).

Conventions shared by every consumer:

* images are ``H x W`` arrays indexed ``[y, x]`` (row-major, y slow), pixel
  centres at integer coordinates;
* the PSF ``B`` is a ``2H x 2W`` array whose centre (zero lag) sits at index
  ``[H, W]``, so ``B[p - q + (H, W)]`` exists for every pair of pixels p, q of
  the image;
* the dirty image is the linear (zero-padded) convolution of the sky with the
  PSF plus white Gaussian noise (imaging model, Sect. 2, Eq. 1), computed in
  FP64 and stored as FP32.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np
from scipy.signal import fftconvolve


def rng_for(config_id: int, seed: int) -> np.random.Generator:
    """The generator every synthetic input of (config_id, seed) draws from."""
    return np.random.default_rng(np.random.SeedSequence([int(config_id), int(seed)]))


@dataclasses.dataclass
class SynthImage:
    """One synthetic observation plus the run parameters of its workload."""

    name: str
    dirty: np.ndarray          # float32 (H, W)
    psf: np.ndarray            # float32 (2H, 2W), zero lag at [H, W]
    sky: np.ndarray            # float64 (H, W) true sky
    noise_sigma: float
    k_max: int
    n_iter: int
    gain: float = 0.35
    lm_max_iter: int = 50
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def H(self) -> int:
        return self.dirty.shape[0]

    @property
    def W(self) -> int:
        return self.dirty.shape[1]


# ----------------------------------------------------------------- PSFs

def analytic_psf(H: int, W: int, sigma: float, ring_radius: Optional[float],
                 ring_level: float = 0.02) -> np.ndarray:
    """Unit-peak Gaussian main lobe plus an optional ring sidelobe.

    ``B(r) = exp(-r^2 / 2 sigma^2) + ring_level * exp(-(r - R)^2 / 2 sigma^2)``
    on a ``2H x 2W`` grid centred at ``[H, W]`` (the ring's radial width is the
    main-lobe sigma).
    """
    y = np.arange(2 * H, dtype=np.float64)[:, None] - H
    x = np.arange(2 * W, dtype=np.float64)[None, :] - W
    r2 = x * x + y * y
    b = np.exp(-r2 / (2.0 * sigma * sigma))
    if ring_radius is not None and ring_level != 0.0:
        r = np.sqrt(r2)
        b = b + ring_level * np.exp(-((r - ring_radius) ** 2) / (2.0 * sigma * sigma))
    return b


def gaussian_psf(H: int, W: int, sigma: float, amp: float = 1.0) -> np.ndarray:
    """Pure circular Gaussian PSF ``amp * exp(-r^2 / 2 sigma^2)`` (2H x 2W)."""
    return amp * analytic_psf(H, W, sigma, None)


def _rotated_gaussian(xs, ys, a, x0, y0, s_major, s_minor, phi):
    """``a exp(-(u^2 / s_major^2 + v^2 / s_minor^2) / 2)`` with (u, v) the
    offset from (x0, y0) rotated by -phi (major axis at angle phi from +x)."""
    c, s = np.cos(phi), np.sin(phi)
    dx, dy = xs - x0, ys - y0
    u = c * dx + s * dy
    v = -s * dx + c * dy
    return a * np.exp(-0.5 * (u * u / (s_major * s_major) + v * v / (s_minor * s_minor)))


def elliptical_psf(H: int, W: int, s_major: float, s_minor: float, phi: float, amp: float = 1.0,
                   ring_radius: Optional[float] = None, ring_level: float = 0.02) -> np.ndarray:
    """Elliptical Gaussian main lobe (widths s_major, s_minor, major axis at
    phi) plus an optional circular ring sidelobe, 2H x 2W, zero lag at
    [H, W]."""
    y = np.arange(2 * H, dtype=np.float64)[:, None]
    x = np.arange(2 * W, dtype=np.float64)[None, :]
    b = _rotated_gaussian(x, y, amp, float(W), float(H), s_major, s_minor, phi)
    if ring_radius is not None and ring_level != 0.0:
        r = np.sqrt((x - W) ** 2 + (y - H) ** 2)
        b = b + amp * ring_level * np.exp(-((r - ring_radius) ** 2) / (2.0 * s_minor * s_minor))
    return b


def elliptical_field(H: int, W: int, sources, noise_sigma: float, seed: int) -> np.ndarray:
    """Sum of rotated elliptical Gaussians (rows a, x0, y0, s_major,
    s_minor, phi) on the H x W pixel grid plus seeded white noise, FP64."""
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    img = np.zeros((H, W))
    for a, x0, y0, s1, s2, phi in sources:
        img += _rotated_gaussian(xs, ys, a, x0, y0, s1, s2, phi)
    return img + rng_for(200, seed).normal(0.0, noise_sigma, (H, W))


def _halfmax_sigma(psf: np.ndarray) -> float:
    """Main-lobe width of a generated PSF from the area above half maximum.

    Generator-side size control only (used to tune the uv taper): the number
    of pixels of the central 129x129 region at or above half the zero-lag
    value is taken as the area of a disc of radius sigma sqrt(2 ln 2).
    """
    H2, W2 = psf.shape
    cy, cx = H2 // 2, W2 // 2
    r = min(64, cy, cx)
    core = psf[cy - r: cy + r + 1, cx - r: cx + r + 1]
    area = float(np.count_nonzero(core >= 0.5 * psf[cy, cx]))
    return float(np.sqrt(area / np.pi) / np.sqrt(2.0 * np.log(2.0)))


def uv_mask_psf(H: int, W: int, rng: np.random.Generator, fill: float = 0.05,
                k0: float = 0.08, target_sigma: float = 2.0) -> tuple[np.ndarray, float]:
    """FFT of a seeded, radially denser random uv mask with a Gaussian taper.

    The mask is Bernoulli with ``p(k) = min(1, c exp(-|k| / k0))`` (``c`` set
    so the mean fill is ``fill``), made Hermitian-symmetric, multiplied by a
    Gaussian taper ``exp(-|k|^2 / 2 s_t^2)``; the PSF is its inverse FFT
    (real, because the weights are Hermitian-symmetric), shifted to
    ``[H, W]`` and normalised to unit peak, so it has negative sidelobes like
    an interferometer's PSF.  (Taking the modulus instead rectifies the
    sidelobes into a positive floor holding ~150x the main lobe's integral,
    under which a main-lobe Gaussian approximation of the PSF over-subtracts
    without bound.)  ``s_t`` is bisected until the half-maximum width lies
    within 2.5 % of ``target_sigma``.  Returns ``(psf, s_t)``.
    """
    H2, W2 = 2 * H, 2 * W
    ky = np.fft.fftfreq(H2)[:, None]
    kx = np.fft.fftfreq(W2)[None, :]
    k = np.sqrt(kx * kx + ky * ky)
    base = np.exp(-k / k0)
    lo_c, hi_c = 0.0, 1.0 / base.mean() * 4.0
    for _ in range(60):
        c = 0.5 * (lo_c + hi_c)
        if np.minimum(1.0, c * base).mean() < fill:
            lo_c = c
        else:
            hi_c = c
    prob = np.minimum(1.0, c * base)
    mask = rng.random((H2, W2)) < prob
    # Hermitian symmetry: sample (ky, kx) <-> (-ky, -kx)
    flip = np.roll(mask[::-1, ::-1], (1, 1), axis=(0, 1))
    mask = mask | flip
    mask[0, 0] = True

    def make(s_t: float) -> np.ndarray:
        w = mask * np.exp(-(k * k) / (2.0 * s_t * s_t))
        img = np.real(np.fft.ifft2(w))
        img = np.fft.fftshift(img)
        return img / img[H, W]

    # wider taper in uv -> narrower main lobe; bisect on log s_t
    lo, hi = np.log(0.01), np.log(0.5)
    psf = make(np.exp(0.5 * (lo + hi)))
    for _ in range(40):
        mid = 0.5 * (lo + hi)
        psf = make(np.exp(mid))
        s = _halfmax_sigma(psf)
        if abs(s - target_sigma) <= 0.025 * target_sigma:
            break
        if s > target_sigma:
            lo = mid
        else:
            hi = mid
    return psf, float(np.exp(mid))


# ----------------------------------------------------------------- sky parts

def _gaussian_blob(H: int, W: int, cx: float, cy: float, sigma: float, peak: float) -> np.ndarray:
    y = np.arange(H, dtype=np.float64)[:, None]
    x = np.arange(W, dtype=np.float64)[None, :]
    # evaluate only inside 8 sigma: exp(-32) ~ 1e-14 relative beyond
    r = int(np.ceil(8.0 * sigma))
    out = np.zeros((H, W))
    x0, x1 = max(0, int(np.floor(cx)) - r), min(W, int(np.floor(cx)) + r + 1)
    y0, y1 = max(0, int(np.floor(cy)) - r), min(H, int(np.floor(cy)) + r + 1)
    if x0 < x1 and y0 < y1:
        dx = x[:, x0:x1] - cx
        dy = y[y0:y1, :] - cy
        out[y0:y1, x0:x1] = peak * np.exp(-(dx * dx + dy * dy) / (2.0 * sigma * sigma))
    return out


def grf_patch(n: int, rng: np.random.Generator, rms: float) -> np.ndarray:
    """Gaussian random field with power spectrum k^-3, unit std scaled to
    ``rms``, then multiplied by a 2-D Hann taper."""
    white = rng.standard_normal((n, n))
    f = np.fft.fft2(white)
    ky = np.fft.fftfreq(n)[:, None]
    kx = np.fft.fftfreq(n)[None, :]
    k = np.sqrt(kx * kx + ky * ky)
    amp = np.zeros_like(k)
    amp[k > 0] = k[k > 0] ** -1.5
    field = np.real(np.fft.ifft2(f * amp))
    field = field / field.std() * rms
    hann = np.hanning(n)
    return field * np.outer(hann, hann)


def _powerlaw_fluxes(rng: np.random.Generator, n: int, smin: float, smax: float,
                     index: float = -1.5) -> np.ndarray:
    """Inverse-CDF draws from dN/dS proportional to S^index on [smin, smax]."""
    g = index + 1.0
    u = rng.random(n)
    return (smin ** g + u * (smax ** g - smin ** g)) ** (1.0 / g)


def _crop_psf(psf: np.ndarray, rel: float = 1e-30) -> np.ndarray:
    """Smallest centred crop outside which |psf| < rel * max (convolution
    speed-up for analytic PSFs whose far field underflows)."""
    H2, W2 = psf.shape
    cy, cx = H2 // 2, W2 // 2
    thr = rel * np.abs(psf).max()
    big = np.abs(psf) >= thr
    ys = np.nonzero(big.any(axis=1))[0]
    xs = np.nonzero(big.any(axis=0))[0]
    ry = int(max(cy - ys.min(), ys.max() - cy))
    rx = int(max(cx - xs.min(), xs.max() - cx))
    ry, rx = min(ry, cy - 1), min(rx, cx - 1)
    return psf[cy - ry: cy + ry + 1, cx - rx: cx + rx + 1]


def dirty_from_sky(sky: np.ndarray, psf: np.ndarray, noise: np.ndarray) -> np.ndarray:
    """``D(p) = sum_q sky(q) B(p - q + (H, W)) + noise(p)`` in FP64 (Eq. 1)."""
    H, W = sky.shape
    crop = _crop_psf(psf)
    ch, cw = crop.shape
    full = fftconvolve(sky, crop, mode="full")
    oy, ox = ch // 2, cw // 2
    return full[oy: oy + H, ox: ox + W] + noise


# ----------------------------------------------------------------- configs

def _config1_style(name: str, H: int, W: int, rng: np.random.Generator, n_points: int,
                   n_gauss: int, sigma_range, psf_sigma: float, ring_radius: float,
                   noise_sigma: float, log_sigma: bool = False, n_grf: int = 0,
                   grf_size: int = 0, grf_rms: float = 0.01, k_max: int = 5,
                   n_iter: int = 200) -> SynthImage:
    sky = np.zeros((H, W))
    px = rng.integers(0, W, n_points)
    py = rng.integers(0, H, n_points)
    pf = rng.uniform(0.1, 1.0, n_points)
    for x, y, f in zip(px, py, pf):
        sky[y, x] += f
    gx = rng.uniform(0, W - 1, n_gauss)
    gy = rng.uniform(0, H - 1, n_gauss)
    if log_sigma:
        gs = np.exp(rng.uniform(np.log(sigma_range[0]), np.log(sigma_range[1]), n_gauss))
    else:
        gs = rng.uniform(sigma_range[0], sigma_range[1], n_gauss)
    gp = rng.uniform(0.05, 0.5, n_gauss)
    for x, y, s, p in zip(gx, gy, gs, gp):
        sky += _gaussian_blob(H, W, x, y, s, p)
    for _ in range(n_grf):
        patch = grf_patch(grf_size, rng, grf_rms)
        ox = int(rng.integers(0, W - grf_size + 1))
        oy = int(rng.integers(0, H - grf_size + 1))
        sky[oy: oy + grf_size, ox: ox + grf_size] += patch
    psf = analytic_psf(H, W, psf_sigma, ring_radius)
    noise = rng.standard_normal((H, W)) * noise_sigma
    dirty = dirty_from_sky(sky, psf, noise)
    meta = dict(points=np.stack([px, py, pf], 1), gaussians=np.stack([gx, gy, gs, gp], 1),
                psf_sigma=psf_sigma, true_flux=float(sky.sum()))
    return SynthImage(name, dirty.astype(np.float32), psf.astype(np.float32), sky, noise_sigma,
                      k_max=k_max, n_iter=n_iter, meta=meta)


def config1(seed: int = 0) -> SynthImage:
    """256x256: 5 points (U[0.1,1] at integer pixels), 3 Gaussians (sigma
    U[2,20], peak U[0.05,0.5]); PSF sigma 1.5 with a 2 % ring at 12 px;
    noise 1e-3; active set <= 5, 200 iterations."""
    return _config1_style("config1_256", 256, 256, rng_for(1, seed), 5, 3, (2.0, 20.0), 1.5,
                          12.0, 1e-3, k_max=5, n_iter=200)


def config2(seed: int = 0, size: int = 1024) -> SynthImage:
    """1024x1024: 50 power-law points (index -1.5 on [1e-3, 1]), 20 Gaussians
    (sigma log-uniform [2,60], peak U[0.05,0.5]), one 300x300 k^-3 GRF patch of
    RMS 0.01; PSF = FFT of a seeded uv mask (main lobe ~2 px); noise 1e-4;
    active set <= 20, 2000 iterations."""
    rng = rng_for(2, seed)
    H = W = int(size)
    sky = np.zeros((H, W))
    n_points, n_gauss = 50, 20
    px = rng.integers(0, W, n_points)
    py = rng.integers(0, H, n_points)
    pf = _powerlaw_fluxes(rng, n_points, 1e-3, 1.0)
    for x, y, f in zip(px, py, pf):
        sky[y, x] += f
    gx = rng.uniform(0, W - 1, n_gauss)
    gy = rng.uniform(0, H - 1, n_gauss)
    gs = np.exp(rng.uniform(np.log(2.0), np.log(60.0), n_gauss))
    gp = rng.uniform(0.05, 0.5, n_gauss)
    for x, y, s, p in zip(gx, gy, gs, gp):
        sky += _gaussian_blob(H, W, x, y, s, p)
    gsize = min(300, H // 2)
    patch = grf_patch(gsize, rng, 0.01)
    ox = int(rng.integers(0, W - gsize + 1))
    oy = int(rng.integers(0, H - gsize + 1))
    sky[oy: oy + gsize, ox: ox + gsize] += patch
    psf, s_t = uv_mask_psf(H, W, rng)
    noise = rng.standard_normal((H, W)) * 1e-4
    dirty = dirty_from_sky(sky, psf, noise)
    meta = dict(points=np.stack([px, py, pf], 1), gaussians=np.stack([gx, gy, gs, gp], 1),
                uv_taper=s_t, true_flux=float(sky.sum()), grf_origin=(ox, oy, gsize))
    return SynthImage(f"config2_{H}", dirty.astype(np.float32), psf.astype(np.float32), sky, 1e-4,
                      k_max=20, n_iter=2000, meta=meta)


def config3(seed: int = 0, size: int = 4096) -> SynthImage:
    """4096x4096 scaled-up config 1: 400 points, 150 Gaussians (sigma
    log-uniform [2,200]), 4 GRF patches of 600x600; PSF sigma 2.5 with a 2 %
    ring at 20 px; noise 1e-3; active set <= 50, 5000 iterations."""
    scale = size / 4096.0
    return _config1_style(f"config3_{size}", size, size, rng_for(3, seed),
                          max(1, int(round(400 * scale * scale))),
                          max(1, int(round(150 * scale * scale))), (2.0, 200.0 * max(scale, 0.1)),
                          2.5, 20.0, 1e-3, log_sigma=True, n_grf=4 if size >= 1200 else 0,
                          grf_size=600, k_max=50, n_iter=5000)


def config4(seed: int, sizes=(256, 512, 1024, 2048)) -> SynthImage:
    """One image of the 64-image batch: size drawn from ``sizes`` (square),
    PSF sigma U[1.2, 3] with the config-1 ring scaled to 8 sigma, config-1
    source counts and ranges, 200 iterations, active set <= 5."""
    rng = rng_for(4, seed)
    n = int(rng.choice(np.asarray(sizes)))
    psf_sigma = float(rng.uniform(1.2, 3.0))
    return _config1_style(f"config4_s{seed}_{n}", n, n, rng, 5, 3, (2.0, 20.0), psf_sigma,
                          8.0 * psf_sigma, 1e-3, k_max=5, n_iter=200)


def small_case(H: int, W: int, seed: int = 0, psf_sigma: float = 1.5, n_points: int = 2,
               n_gauss: int = 1, sigma_range=(2.0, 5.0), noise_sigma: float = 1e-3,
               ring: bool = True, k_max: int = 5, n_iter: int = 20) -> SynthImage:
    """A tiny config-1-style image for tests (arbitrary, possibly ragged, size)."""
    return _config1_style(f"small_{H}x{W}_s{seed}", H, W, rng_for(100, seed), n_points, n_gauss,
                          sigma_range, psf_sigma, 8.0 * psf_sigma if ring else None, noise_sigma,
                          k_max=k_max, n_iter=n_iter)
