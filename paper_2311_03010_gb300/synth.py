"""Seeded synthetic workloads for EECMG image restoration.

The restoration method is tested on synthetic stand-ins for the paper's test
image, which is not published: piecewise-constant rectangles and ellipses on
the [0, 255] grey scale, a linear gradient and (for the larger cases) a
sinusoidal texture band.  Degradation follows the model of Section 1 (Eqs. 1
and 8): a point-spread-function blur with zero boundary plus Gaussian noise
scaled to a relative level v (Section 5, noise levels).

This module only *makes inputs*.  It holds none of the restoration method's
arithmetic: the blur that simulates the degradation is scipy's FFT
convolution (a library routine), and both the CPU oracle and the CUDA path
receive its output, rounded to FP32, as their input.

PSF shapes:
  * Gaussian (Section 5): 1-D h(i) = exp(-i^2 / (2 sigma^2)) for |i| <= band,
    normalised to sum 1; the 2-D PSF is the outer product h h^T (H = h (x) h).
  * Linear motion blur (not in the paper): a segment of length ``length``
    centred at the origin, at ``angle_deg`` from the +x axis with y pointing
    up, sampled at 8*length+1 points and splatted bilinearly into an odd
    square support of side 2*ceil(length/2)+1; symmetrised so that
    K(p, q) = K(-p, -q) exactly, then normalised to sum 1.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "synthetic_image",
    "gaussian_psf",
    "motion_psf",
    "degrade",
    "Problem",
    "make_problem",
    "batch_specs",
    "arrival_trace",
    "synthetic_volume",
    "gaussian_psf3",
    "make_volume_problem",
]


def _paint_rect(img, yy0, xx0, cy, cx, hy, hx, val):
    h, w = img.shape
    y0 = max(0, int(math.floor(cy - hy)))
    y1 = min(h, int(math.ceil(cy + hy)) + 1)
    x0 = max(0, int(math.floor(cx - hx)))
    x1 = min(w, int(math.ceil(cx + hx)) + 1)
    if y0 >= y1 or x0 >= x1:
        return
    ys = yy0[y0:y1, None]
    xs = xx0[None, x0:x1]
    m = (np.abs(ys - cy) <= hy) & (np.abs(xs - cx) <= hx)
    img[y0:y1, x0:x1][m] = val


def _paint_ellipse(img, yy0, xx0, cy, cx, a, b, ang, val):
    h, w = img.shape
    r = max(a, b)
    y0 = max(0, int(math.floor(cy - r)))
    y1 = min(h, int(math.ceil(cy + r)) + 1)
    x0 = max(0, int(math.floor(cx - r)))
    x1 = min(w, int(math.ceil(cx + r)) + 1)
    if y0 >= y1 or x0 >= x1:
        return
    dy = yy0[y0:y1, None] - cy
    dx = xx0[None, x0:x1] - cx
    ca, sa = math.cos(ang), math.sin(ang)
    xr = dx * ca + dy * sa
    yr = -dx * sa + dy * ca
    m = (xr / a) ** 2 + (yr / b) ** 2 <= 1.0
    img[y0:y1, x0:x1][m] = val


def synthetic_image(h: int, w: int, seed: int, texture: bool = True) -> np.ndarray:
    """A seeded FP64 test image of shape (h, w) with values in [0, 255].

    Constant background, n_rect rectangles and n_ell ellipses (centres
    uniform, extents 5-40 % of the side, ellipse angle uniform in [0, pi),
    intensity uniform in [0, 255], painted in order), plus a linear gradient
    with a total swing uniform in [20, 60] grey levels, plus (``texture``) a
    horizontal band of 20 % of the height carrying A*sin(2*pi*(x cos(phi) +
    y sin(phi))/T), A in [10, 30], T in [6, 16] pixels.  Clipped to [0, 255].
    n_rect = 4 + area/2^16 and n_ell = 3 + area/2^16, each capped at 64.
    """
    rng = np.random.default_rng(seed)
    img = np.full((h, w), rng.uniform(0.0, 255.0), dtype=np.float64)
    area = h * w
    n_rect = min(64, 4 + area // 65536)
    n_ell = min(64, 3 + area // 65536)
    yy0 = np.arange(h, dtype=np.float64)
    xx0 = np.arange(w, dtype=np.float64)
    for _ in range(n_rect):
        cy, cx = rng.uniform(0, h), rng.uniform(0, w)
        hy = 0.5 * rng.uniform(0.05, 0.40) * h
        hx = 0.5 * rng.uniform(0.05, 0.40) * w
        _paint_rect(img, yy0, xx0, cy, cx, hy, hx, rng.uniform(0.0, 255.0))
    side = min(h, w)
    for _ in range(n_ell):
        cy, cx = rng.uniform(0, h), rng.uniform(0, w)
        a = max(0.5, 0.5 * rng.uniform(0.05, 0.40) * side)
        b = max(0.5, 0.5 * rng.uniform(0.05, 0.40) * side)
        ang = rng.uniform(0.0, math.pi)
        _paint_ellipse(img, yy0, xx0, cy, cx, a, b, ang, rng.uniform(0.0, 255.0))
    # linear gradient, zero mean, total swing in [20, 60]
    swing = rng.uniform(20.0, 60.0)
    phi = rng.uniform(0.0, 2.0 * math.pi)
    ga, gb = math.cos(phi), math.sin(phi)
    span = abs(ga) * max(w - 1, 1) + abs(gb) * max(h - 1, 1)
    grad = (ga * xx0[None, :] + gb * yy0[:, None]) * (swing / span)
    img += grad - grad.mean()
    if texture:
        bh = max(1, int(round(0.2 * h)))
        y0 = int(rng.integers(0, max(1, h - bh + 1)))
        amp = rng.uniform(10.0, 30.0)
        per = rng.uniform(6.0, 16.0)
        th = rng.uniform(0.0, math.pi)
        ys = yy0[y0:y0 + bh, None]
        img[y0:y0 + bh, :] += amp * np.sin(
            2.0 * math.pi * (xx0[None, :] * math.cos(th) + ys * math.sin(th)) / per)
    np.clip(img, 0.0, 255.0, out=img)
    return img


def gaussian_psf(sigma: float, band: int) -> np.ndarray:
    """Separable Gaussian PSF of size (2*band+1)^2, FP64, sum 1 (Section 5)."""
    i = np.arange(-band, band + 1, dtype=np.float64)
    h = np.exp(-(i * i) / (2.0 * sigma * sigma))
    h /= h.sum()
    return np.outer(h, h)


def motion_psf(length: float, angle_deg: float) -> np.ndarray:
    """Centrosymmetric linear-motion PSF, odd square support, FP64, sum 1."""
    r = int(math.ceil(length / 2.0))
    n = 2 * r + 1
    k = np.zeros((n, n), dtype=np.float64)
    th = math.radians(angle_deg)
    c, s = math.cos(th), math.sin(th)
    npts = int(round(8 * length)) + 1
    half = (npts - 1) / 2.0
    for i in range(npts):
        t = (i - half) / 8.0            # exact multiples of 1/8: symmetric in t
        col = r + t * c
        row = r - t * s                 # y points up
        c0, r0 = math.floor(col), math.floor(row)
        fc, fr = col - c0, row - r0
        for (rr, cc, wt) in ((r0, c0, (1 - fr) * (1 - fc)), (r0, c0 + 1, (1 - fr) * fc),
                             (r0 + 1, c0, fr * (1 - fc)), (r0 + 1, c0 + 1, fr * fc)):
            if 0 <= rr < n and 0 <= cc < n:
                k[rr, cc] += wt
    k = 0.5 * (k + k[::-1, ::-1])
    k /= k.sum()
    return k


def degrade(u: np.ndarray, psf: np.ndarray, v: float, noise_seed: int):
    """g_delta = h * u + e (Eqs. 1, 8), zero boundary, ||e|| / ||u|| = v.

    e = v * ||u|| * e_hat / ||e_hat|| with e_hat iid N(0, 1) drawn from
    ``default_rng(noise_seed)``.  Returns (g_delta as FP32, delta) where
    delta = ||e||_RMS (Eq. 10).
    """
    from scipy.signal import fftconvolve

    g = fftconvolve(u, psf, mode="same")
    rng = np.random.default_rng(noise_seed)
    e_hat = rng.standard_normal(u.shape)
    e = (v * np.linalg.norm(u) / np.linalg.norm(e_hat)) * e_hat
    gd = (g + e).astype(np.float32)
    delta = float(np.sqrt(np.mean(e * e)))
    return gd, delta


@dataclass
class Problem:
    """One restoration problem: clean image, PSF, degraded data (FP32)."""

    u: np.ndarray          # clean image, FP64
    psf: np.ndarray        # FP64, odd sizes, centred
    g: np.ndarray          # degraded data, FP32
    delta: float           # ||e||_RMS
    v: float               # relative noise level
    meta: dict = field(default_factory=dict)


def make_problem(h, w, seed, psf, v, noise_seed=None, texture=True) -> Problem:
    u = synthetic_image(h, w, seed, texture=texture)
    ns = seed + 1 if noise_seed is None else noise_seed
    g, delta = degrade(u, psf, v, ns)
    return Problem(u=u, psf=psf, g=g, delta=delta, v=v,
                   meta={"h": h, "w": w, "seed": seed, "noise_seed": ns})


def batch_specs(n: int, seed: int, smin: int = 128, smax: int = 1536):
    """Uneven batch: sizes, PSFs and noise levels, seeded.

    Side s uniform in {smin..smax}; square or 3:4 (long side s, short side
    round(0.75 s), orientation random) with probability 1/2 each.  PSF:
    Gaussian sigma ~ U[1, 4] (band ceil(3 sigma)) or motion length ~
    U{5..21}, angle ~ U[0, 180), probability 1/2 each.  v ~ U[0.5 %, 5 %].
    """
    rng = np.random.default_rng(seed)
    specs = []
    for i in range(n):
        s = int(rng.integers(smin, smax + 1))
        if rng.uniform() < 0.5:
            h = w = s
        else:
            short = int(round(0.75 * s))
            h, w = (s, short) if rng.uniform() < 0.5 else (short, s)
        if rng.uniform() < 0.5:
            sig = float(rng.uniform(1.0, 4.0))
            psf = ("gauss", sig, int(math.ceil(3 * sig)))
        else:
            psf = ("motion", int(rng.integers(5, 22)), float(rng.uniform(0.0, 180.0)))
        v = float(rng.uniform(0.005, 0.05))
        specs.append({"h": h, "w": w, "psf": psf, "v": v, "seed": seed + i})
    return specs


def psf_from_spec(spec) -> np.ndarray:
    kind = spec[0]
    if kind == "gauss":
        return gaussian_psf(spec[1], spec[2])
    return motion_psf(spec[1], spec[2])


def arrival_trace(n: int, rate: float, seed: int, smin: int = 256, smax: int = 4096,
                  vmin: float = 0.01, vmax: float = 0.05):
    """Poisson arrivals (rate per second) with log-uniform pixel counts.

    Returns a list of dicts with arrival time t (s), size (h, w), PSF spec and
    noise level.  Pixel count is log-uniform in [smin^2, smax^2]; the side is
    its square root rounded to a multiple of 8.  PSF mix as ``batch_specs``.
    """
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=n))
    out = []
    lo, hi = math.log(smin * smin), math.log(smax * smax)
    for i in range(n):
        px = math.exp(rng.uniform(lo, hi))
        s = max(smin, min(smax, int(round(math.sqrt(px) / 8.0)) * 8))
        if rng.uniform() < 0.5:
            sig = float(rng.uniform(1.0, 4.0))
            psf = ("gauss", sig, int(math.ceil(3 * sig)))
        else:
            psf = ("motion", int(rng.integers(5, 22)), float(rng.uniform(0.0, 180.0)))
        out.append({"t": float(t[i]), "h": s, "w": s, "psf": psf,
                    "v": float(rng.uniform(vmin, vmax)), "seed": seed + i})
    return out


# ---------------------------------------------------------------- volumes


def synthetic_volume(d: int, h: int, w: int, seed: int) -> np.ndarray:
    """A seeded FP64 test volume of shape (d, h, w) with values in [0, 255].

    The 3-D counterpart of ``synthetic_image``: constant background, n_box
    axis-aligned boxes and n_ell ellipsoids (centres uniform, semi-axes 2.5-20
    % of each side, intensity uniform in [0, 255], painted in order), plus a
    linear gradient along a random direction with a total swing uniform in
    [20, 60] grey levels.  Clipped to [0, 255].  n_box = 4 + voxels/2^21 and
    n_ell = 3 + voxels/2^21, each capped at 64.
    """
    rng = np.random.default_rng(seed)
    vol = np.full((d, h, w), rng.uniform(0.0, 255.0), dtype=np.float64)
    nvox = d * h * w
    n_box = min(64, 4 + nvox // (1 << 21))
    n_ell = min(64, 3 + nvox // (1 << 21))
    zz = np.arange(d, dtype=np.float64)[:, None, None]
    yy = np.arange(h, dtype=np.float64)[None, :, None]
    xx = np.arange(w, dtype=np.float64)[None, None, :]
    for _ in range(n_box):
        c = [rng.uniform(0, n) for n in (d, h, w)]
        r = [0.5 * rng.uniform(0.05, 0.40) * n for n in (d, h, w)]
        val = rng.uniform(0.0, 255.0)
        m = (np.abs(zz - c[0]) <= r[0]) & (np.abs(yy - c[1]) <= r[1]) & (np.abs(xx - c[2]) <= r[2])
        vol[m] = val
    for _ in range(n_ell):
        c = [rng.uniform(0, n) for n in (d, h, w)]
        r = [max(0.5, 0.5 * rng.uniform(0.05, 0.40) * n) for n in (d, h, w)]
        val = rng.uniform(0.0, 255.0)
        m = ((zz - c[0]) / r[0]) ** 2 + ((yy - c[1]) / r[1]) ** 2 + ((xx - c[2]) / r[2]) ** 2 <= 1.0
        vol[m] = val
    swing = rng.uniform(20.0, 60.0)
    dirn = rng.standard_normal(3)
    dirn /= np.linalg.norm(dirn)
    span = sum(abs(dirn[i]) * max(n - 1, 1) for i, n in enumerate((d, h, w)))
    grad = (dirn[0] * zz + dirn[1] * yy + dirn[2] * xx) * (swing / span)
    vol += grad - grad.mean()
    np.clip(vol, 0.0, 255.0, out=vol)
    return vol


def gaussian_psf3(sigma: float, band: int) -> np.ndarray:
    """Separable 3-D Gaussian PSF of size (2*band+1)^3, FP64, sum 1 (h (x) h (x) h)."""
    i = np.arange(-band, band + 1, dtype=np.float64)
    h = np.exp(-(i * i) / (2.0 * sigma * sigma))
    h /= h.sum()
    return h[:, None, None] * h[None, :, None] * h[None, None, :]


def make_volume_problem(d, h, w, seed, psf, v, noise_seed=None) -> Problem:
    """A volume restoration problem: ``synthetic_volume`` degraded by ``degrade``."""
    u = synthetic_volume(d, h, w, seed)
    ns = seed + 1 if noise_seed is None else noise_seed
    g, delta = degrade(u, psf, v, ns)
    return Problem(u=u, psf=psf, g=g, delta=delta, v=v,
                   meta={"d": d, "h": h, "w": w, "seed": seed, "noise_seed": ns})
