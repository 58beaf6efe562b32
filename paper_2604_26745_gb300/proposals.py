"""Learned proposal operator of Sec. 3.3 for the accelerated scheme (Alg. 2).

The convolutional encoder-decoder of the paper's figure maps the iterate u and the LM step
s (both stacked [2, n, n]: emission, attenuation) to a proposal u~ = G(u, s):

    e = E_u(u) + E_s(s)          two encoders, each three convolutions with a ReLU,
                                 channels 2 -> 8 -> 16 -> 32; their outputs are summed
    d = D(e)                     decoder: convolution + ReLU 32 -> 32 (from the sum), then
                                 32 -> 16 -> 8 with a ReLU each, then a convolution 8 -> 2
                                 without activation
    u~ = ReLU(u + L(s) * d)      d multiplied pixelwise by L(s), L a 5 x 5 convolution
                                 2 -> 2 without bias or activation (the L of Prop.
                                 conv_check, G = u + L(s) . g(u, s)), added to u by the skip
                                 connection and projected to non-negative values

Readings (the paper's figure is a simplified picture and the text gives one kernel size):
L is 5 x 5 without bias as the text states; the ten other convolutions are 3 x 3 with
bias, keeping the image size.  This gives 27 198 parameters.  The paper reports 28 104;
no choice of uniform kernel sizes (1 to 7 px) and biases for the figure's wiring, with or
without the 32 -> 32 layer or with shared encoders, reproduces that count, and 5 x 5
kernels throughout would give 75 070, so the figure's channel widths and wiring are kept
and the count differs by 3 %.  As in Sec. 4, the inputs are scaled by the box bounds
(lambda / lambda_max, mu / mu_max) and the correction is scaled back.  No trained weights
ship with the library (the paper's training data are not available): the module is the
architecture, to be trained by the caller or loaded from a state dict, and Alg. 2's
safeguard keeps any proposal from harming the iteration.  Its convolutions run in the
framework's convolution library.
"""
from __future__ import annotations

import torch
from torch import nn

KERNEL = 3        # the ten convolutions of the encoders and the decoder
L_KERNEL = 5      # the linear operator L on s (no bias)


def _conv(cin: int, cout: int, k: int = KERNEL, bias: bool = True) -> nn.Conv2d:
    return nn.Conv2d(cin, cout, kernel_size=k, padding=k // 2, bias=bias)


class ConvProposal(nn.Module):
    """u~ = ReLU(u + L(s) * D(E_u(u) + E_s(s))) on images scaled by the box bounds."""

    WIDTHS = (2, 8, 16, 32)

    def __init__(self, lambda_max: float = 2.0, mu_max: float = 0.2):
        super().__init__()
        w = self.WIDTHS
        enc = lambda: nn.Sequential(*[m for a, b in zip(w[:-1], w[1:]) for m in (_conv(a, b), nn.ReLU())])
        self.enc_u = enc()
        self.enc_s = enc()
        r = (w[-1],) + w[::-1]  # 32 -> 32 -> 16 -> 8 with ReLU, then 8 -> 2 without activation
        layers = [m for a, b in zip(r[:-2], r[1:-1]) for m in (_conv(a, b), nn.ReLU())]
        self.dec = nn.Sequential(*layers, _conv(r[-2], r[-1]))
        self.L = _conv(2, 2, L_KERNEL, bias=False)
        self.register_buffer("scale", torch.tensor([lambda_max, mu_max]).view(1, 2, 1, 1))

    def forward(self, u: torch.Tensor, s: torch.Tensor) -> torch.Tensor:
        """u, s: [B, 2, n, n] (or [2, n, n]) in physical units; returns u~ of the same shape."""
        squeeze = u.dim() == 3
        if squeeze:
            u, s = u.unsqueeze(0), s.unsqueeze(0)
        sc = self.scale.to(dtype=u.dtype)
        un, sn = u / sc, s / sc
        d = self.dec(self.enc_u(un) + self.enc_s(sn))
        # ReLU(u / sc + L(s) d) sc with the scale applied to the correction only (sc > 0):
        # the same map, and exactly u where the correction vanishes
        out = torch.relu(u + sc * (self.L(sn) * d))
        return out.squeeze(0) if squeeze else out


def as_proposal(model: nn.Module):
    """The G(u, s, k) callable of accelerated_solve for a module taking (u, s)."""

    @torch.no_grad()
    def G(u: torch.Tensor, s: torch.Tensor, k: int) -> torch.Tensor:
        p = next(model.parameters())
        return model(u.to(p.dtype), s.to(p.dtype)).to(u.dtype)

    return G
