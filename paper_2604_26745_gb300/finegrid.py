"""Data from a twice finer grid (the paper generates its phantoms at twice the spatial
resolution and projects them from there, to avoid the inverse crime; Sec. 4).

A problem on an n x n grid (pixel size 1) is projected from a 2n x 2n grid of pixel size
1/2.  In fine-pixel units every length doubles: the field-of-view radius and the
detector pitch are twice the coarse ones, while the sample step stays one (fine) pixel, so
the ray sums are also sampled twice as densely.  An attenuation of mu per coarse pixel is
mu / 2 per fine pixel, and a ray sum measured in fine-pixel lengths is twice the same sum
in coarse-pixel lengths:

    y_coarse = 1/2 * A_fine(lambda_fine, mu_fine / 2)

with lambda_fine, mu_fine the fine images in the coarse problem's units.  The detector
layout (angles, banks, detectors, sub-rays) is unchanged, so y_coarse is data for the
coarse reconstruction.
"""
from __future__ import annotations

import math

import torch

from . import pget as P
from . import synth


def fine_geometry(g: P.pget_geometry) -> P.pget_geometry:
    """The geometry of the same scanner on the 2n x 2n grid of half-size pixels."""
    n = g.n
    r = g.fov_radius if g.fov_radius > 0 else n / math.sqrt(2.0)
    nbk = g.n_banks if g.n_banks > 0 else (2 if g.n_det == 182 else 1)
    p = g.det_pitch if g.det_pitch > 0 else 2.0 * r / (g.n_det // nbk)
    h = g.step if g.step > 0 else 1.0
    return P.geometry(2 * n, g.n_angles, g.n_det, n_sub=g.n_sub, collimator=g.collimator, n_banks=nbk,
                      step=h, fov_radius=2.0 * r, det_pitch=2.0 * p)


def fine_lattice_phantom(n: int, n_lat: int, radius: float | None = None, seed: int = 0, **kw) -> synth.Phantom:
    """The rod lattice of synth.lattice_phantom(n, ...) rasterised on the 2n grid: same
    rods (positions, radii and values drawn from the same seed), twice the resolution.
    Values stay in the coarse problem's units."""
    pitch = n // n_lat
    r = radius if radius is not None else float(round(0.35 * pitch))
    if kw.get("jitter"):
        kw["jitter"] = 2.0 * kw["jitter"]  # the same displacements, in fine pixels
    return synth.lattice_phantom(2 * n, n_lat, radius=2.0 * r, seed=seed, pitch=2 * pitch, **kw)


def project_fine(ctx: P.Context, g: P.pget_geometry, precision: int, lam_fine: torch.Tensor,
                 mu_fine: torch.Tensor) -> torch.Tensor:
    """y for the coarse problem g from fine images (2n x 2n, coarse units)."""
    y = P.pget_forward(ctx, fine_geometry(g), precision, lam_fine.contiguous(), (0.5 * mu_fine).contiguous())
    return 0.5 * y
