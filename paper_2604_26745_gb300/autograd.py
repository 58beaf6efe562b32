"""torch.autograd wrappers of the attenuated ray transform (Sec. 2.1, Eq. (1)) and its
derivatives (Eq. (2)), computed by the library's CUDA kernels.

``project(lam, mu, geometry)`` returns y = A(lam, mu) for one image pair [n, n] or a batch
[..., n, n]; reverse mode (``.backward()``) runs the adjoint kernel (pget_vjp) and forward
mode (dual tensors of ``torch.autograd.forward_ad``) runs the Jacobian-vector kernel
(pget_jvp).  A batch runs through the batched calls (pget_forward_batch, pget_jvp_batch,
pget_vjp_batch): one walk launch covers the views of many pairs, with every pair's result
equal to its single-pair call's bitwise.  Only lam and mu are
kept for the backward pass: the attenuation prefixes along every ray are recomputed by
the kernels rather than stored (storing the per-sample factors exp(-E_j) and prefix sums
would take 8 bytes per ray sample, ~1 GB per 256 x 256 image at 360 x 182 x 5 rays).
"""
from __future__ import annotations

import threading

import torch

from . import pget as P

_ctx_lock = threading.Lock()
_contexts = {}


def context(device: int) -> P.Context:
    """The library context used by the autograd wrappers on one device (created once)."""
    with _ctx_lock:
        c = _contexts.get(device)
        if c is None:
            c = _contexts[device] = P.Context(device)
        return c


def _prec_of(dtype: torch.dtype, precision):
    if precision is not None:
        return precision
    return P.PGET_F64 if dtype == torch.float64 else P.PGET_F32_KAHAN


class AttenuatedRayTransform(torch.autograd.Function):
    """y = A(lam, mu) for image pairs [B, n, n] (B >= 1) on one CUDA device."""

    @staticmethod
    def forward(lam, mu, geometry, precision):
        ctx_ = context(lam.device.index or 0)
        return P.pget_forward_batch(ctx_, geometry, precision, lam.contiguous(), mu.contiguous())

    @staticmethod
    def setup_context(ctx, inputs, output):
        lam, mu, geometry, precision = inputs
        ctx.save_for_backward(lam, mu)
        ctx.save_for_forward(lam, mu)
        ctx.geometry = geometry
        ctx.precision = precision

    @staticmethod
    def backward(ctx, grad_y):
        lam, mu = ctx.saved_tensors
        c = context(lam.device.index or 0)
        gl, gm = P.pget_vjp_batch(c, ctx.geometry, ctx.precision, lam.contiguous(), mu.contiguous(),
                                  grad_y.contiguous())
        return gl, gm, None, None

    @staticmethod
    def jvp(ctx, dlam, dmu, _g, _p):
        lam, mu = ctx.saved_tensors
        c = context(lam.device.index or 0)
        dlam = torch.zeros_like(lam) if dlam is None else dlam.contiguous()
        dmu = torch.zeros_like(mu) if dmu is None else dmu.contiguous()
        return P.pget_jvp_batch(c, ctx.geometry, ctx.precision, lam.contiguous(), mu.contiguous(), dlam, dmu)


def project(lam: torch.Tensor, mu: torch.Tensor, geometry: P.pget_geometry, precision=None) -> torch.Tensor:
    """Differentiable forward model for [n, n] or batched [..., n, n] CUDA tensors."""
    if lam.shape != mu.shape or lam.dim() < 2 or not lam.is_cuda:
        raise ValueError("lam and mu must be CUDA tensors of the same shape [..., n, n]")
    prec = _prec_of(lam.dtype, precision)
    if P.dtype_of(prec) != lam.dtype:
        raise ValueError("tensor dtype does not match the precision")
    lead = lam.shape[:-2]
    ls = lam.reshape(-1, *lam.shape[-2:])
    ms = mu.reshape(-1, *mu.shape[-2:])
    y = AttenuatedRayTransform.apply(ls, ms, geometry, prec)
    return y.reshape(*lead, geometry.n_angles, geometry.n_det)


def data_loss(lam, mu, y, geometry, precision=None) -> torch.Tensor:
    """1/2 |A(lam, mu) - y|^2 summed over the batch (the data term of Eq. (6))."""
    r = project(lam, mu, geometry, precision) - y
    return 0.5 * (r * r).sum()
