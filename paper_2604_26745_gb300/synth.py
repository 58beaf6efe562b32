"""Seeded synthetic inputs: fuel-assembly phantoms, Poisson noise, request streams.

This module holds none of the reconstruction arithmetic (no ray sums, derivatives or
solver steps).  It only draws phantoms and noise, so the CUDA path and the CPU oracle
can be fed identical inputs.  Every random draw comes from numpy's
``Generator(PCG64(seed))``.

Phantoms follow the synthetic assemblies of Sec. 3.3 of the paper (a square lattice
of fuel rods, each with its own emission and attenuation value, some rods
non-emitting; water has attenuation but no emission), in pixel units:
rods are disks rasterised by area fraction with ``supersample`` x ``supersample``
points per pixel.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _disk_fraction(n: int, cx: float, cy: float, radius: float, ss: int) -> tuple:
    """Area fraction of a disk (centred coordinates, pixel units) in each pixel of its
    bounding box; returns (iy0, ix0, frac[h, w])."""
    c = 0.5 * (n - 1)
    ix0 = max(0, int(math.floor(cx + c - radius - 1)))
    ix1 = min(n - 1, int(math.ceil(cx + c + radius + 1)))
    iy0 = max(0, int(math.floor(cy + c - radius - 1)))
    iy1 = min(n - 1, int(math.ceil(cy + c + radius + 1)))
    if ix1 < ix0 or iy1 < iy0:
        return iy0, ix0, np.zeros((0, 0))
    off = (np.arange(ss) + 0.5) / ss - 0.5
    xs = (np.arange(ix0, ix1 + 1) - c)[None, :, None, None] + off[None, None, None, :]
    ys = (np.arange(iy0, iy1 + 1) - c)[:, None, None, None] + off[None, None, :, None]
    inside = (xs - cx) ** 2 + (ys - cy) ** 2 <= radius * radius
    return iy0, ix0, inside.mean(axis=(2, 3))


@dataclass
class Phantom:
    lam: np.ndarray
    mu: np.ndarray
    rod_lambda: np.ndarray = field(default=None)
    rod_mu: np.ndarray = field(default=None)


def lattice_phantom(n: int, n_lat: int, radius: float | None = None, seed: int = 0,
                    lam_range=(0.5, 1.5), zero_frac: float = 0.1, mu_rod=0.08,
                    mu_bg: float = 0.01, pitch: int | None = None, supersample: int = 8,
                    jitter: float = 0.0) -> Phantom:
    """n x n phantom with an n_lat x n_lat rod lattice at pitch floor(n / n_lat).

    Rod emission ~ U(lam_range); floor(zero_frac * n_lat^2) rods, chosen without
    replacement, are non-emitting (attenuation kept).  Rod attenuation is ``mu_rod``
    or, if a (lo, hi) pair, ~ U(lo, hi) per rod.  Background (water): attenuation
    ``mu_bg``, no emission.  ``jitter`` > 0 perturbs rod centres by U(-jitter, jitter)
    pixels, like the perturbed positions of the paper's training data.
    """
    g = rng(seed)
    P = pitch if pitch is not None else n // n_lat
    r = radius if radius is not None else float(round(0.35 * P))
    nrod = n_lat * n_lat
    lam_rod = g.uniform(lam_range[0], lam_range[1], size=nrod)
    nz = int(math.floor(zero_frac * nrod))
    if nz > 0:
        lam_rod[g.choice(nrod, size=nz, replace=False)] = 0.0
    if isinstance(mu_rod, (tuple, list)):
        mu_r = g.uniform(mu_rod[0], mu_rod[1], size=nrod)
    else:
        mu_r = np.full(nrod, float(mu_rod))
    jit = g.uniform(-jitter, jitter, size=(nrod, 2)) if jitter > 0 else np.zeros((nrod, 2))
    lam = np.zeros((n, n))
    frac_mu = np.zeros((n, n))
    for i in range(n_lat):
        for j in range(n_lat):
            k = i * n_lat + j
            cx = (j - 0.5 * (n_lat - 1)) * P + jit[k, 0]
            cy = (i - 0.5 * (n_lat - 1)) * P + jit[k, 1]
            iy0, ix0, fr = _disk_fraction(n, cx, cy, r, supersample)
            if fr.size == 0:
                continue
            h, w = fr.shape
            lam[iy0:iy0 + h, ix0:ix0 + w] += fr * lam_rod[k]
            frac_mu[iy0:iy0 + h, ix0:ix0 + w] += fr * (mu_r[k] - mu_bg)
    mu = mu_bg + frac_mu
    return Phantom(lam=lam, mu=mu, rod_lambda=lam_rod, rod_mu=mu_r)


def disk_image(n: int, radius: float, value: float, supersample: int = 8,
               center=(0.0, 0.0)) -> np.ndarray:
    """A single disk rasterised by area fraction (supersample = 1: point-evaluated)."""
    img = np.zeros((n, n))
    iy0, ix0, fr = _disk_fraction(n, center[0], center[1], radius, supersample)
    if fr.size:
        h, w = fr.shape
        img[iy0:iy0 + h, ix0:ix0 + w] = fr * value
    return img


def poisson_noise(y_clean: np.ndarray, counts: float, seed: int) -> np.ndarray:
    """y = Poisson(C y_clean / max y_clean) * max y_clean / C (C counts in the max bin)."""
    g = rng(seed)
    y_clean = np.asarray(y_clean, dtype=np.float64)
    ymax = float(y_clean.max())
    if ymax <= 0:
        return y_clean.copy()
    lam = np.clip(counts * y_clean / ymax, 0.0, None)
    return g.poisson(lam).astype(np.float64) * ymax / counts


def random_direction(shape, seed: int) -> np.ndarray:
    """Standard-normal array (directions for derivative checks)."""
    return rng(seed).standard_normal(shape)


@dataclass
class Request:
    """One reconstruction request of the serving stream (sizes and seeds only)."""
    rid: int
    arrival_s: float
    n: int
    n_lat: int
    n_angles: int
    n_det: int
    n_sub: int
    counts: float
    phantom_seed: int
    noise_seed: int


def serving_stream(n_requests: int = 256, rate_hz: float = 50.0, seed: int = 4242,
                   sizes=(96, 128, 192, 256), lattices=(9, 10, 17), angles=(180, 360),
                   subs=(3, 4, 5, 6, 7), n_det: int = 182) -> list:
    """Poisson arrivals (exponential gaps of mean 1/rate) with per-request sizes drawn
    uniformly from the given sets and counts C = 10^U(4, 6)."""
    g = rng(seed)
    t = 0.0
    out = []
    for i in range(n_requests):
        t += g.exponential(1.0 / rate_hz)
        out.append(Request(
            rid=i, arrival_s=t, n=int(g.choice(sizes)), n_lat=int(g.choice(lattices)),
            n_angles=int(g.choice(angles)), n_det=n_det, n_sub=int(g.choice(subs)),
            counts=float(10 ** g.uniform(4, 6)), phantom_seed=int(10000 + i),
            noise_seed=int(20000 + i)))
    return out
