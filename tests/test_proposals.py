"""The convolutional proposal operator of Sec. 3.3 (architecture only; no trained weights):
the wiring and channel widths of the paper's figure (two encoders 2 -> 8 -> 16 -> 32 summed,
a decoder 32 -> 32 -> 16 -> 8 -> 2, the product with L(s) and the skip connection), ten
3 x 3 convolutions with bias and L a 5 x 5 convolution 2 -> 2 without bias (as the paper
states), 27 198 parameters; it keeps the image size (odd n too), returns non-negative
images, and with all weights zero reduces to its skip connection (u~ = u for feasible u)."""
import pytest

torch = pytest.importorskip("torch")

from paper_2604_26745_gb300.proposals import ConvProposal, as_proposal  # noqa: E402


def test_architecture():
    m = ConvProposal()
    convs = [x for x in m.modules() if isinstance(x, torch.nn.Conv2d)]
    assert len(convs) == 11
    net, L = convs[:10], m.L
    assert all(c.kernel_size == (3, 3) and c.padding == (1, 1) and c.bias is not None for c in net)
    assert L.kernel_size == (5, 5) and L.padding == (2, 2) and L.bias is None  # L: no bias
    chans = [(c.in_channels, c.out_channels) for c in net]
    assert chans == [(2, 8), (8, 16), (16, 32), (2, 8), (8, 16), (16, 32), (32, 32), (32, 16), (16, 8), (8, 2)]
    assert (L.in_channels, L.out_channels) == (2, 2)
    # count written out: encoders 2 x (2*8*9+8 + 8*16*9+16 + 16*32*9+32), decoder
    # 32*32*9+32 + 32*16*9+16 + 16*8*9+8 + 8*2*9+2, L 2*2*25
    assert sum(p.numel() for p in m.parameters()) == 2 * 5960 + 15178 + 100 == 27198


@pytest.mark.parametrize("n", [16, 27])
def test_shape_and_sign(n):
    torch.manual_seed(0)
    m = ConvProposal().double()
    u = torch.rand(2, n, n, dtype=torch.float64) * torch.tensor([2.0, 0.2], dtype=torch.float64).view(2, 1, 1)
    s = 0.1 * torch.randn(2, n, n, dtype=torch.float64)
    out = m(u, s)
    assert out.shape == (2, n, n) and (out >= 0).all()
    assert m(u[None], s[None]).shape == (1, 2, n, n)


def test_zero_weights_is_the_skip_connection():
    m = ConvProposal().double()
    for p in m.parameters():
        torch.nn.init.zeros_(p)
    u = torch.rand(2, 20, 20, dtype=torch.float64)
    s = torch.randn(2, 20, 20, dtype=torch.float64)
    assert torch.equal(m(u, s), u)
    G = as_proposal(m)
    assert torch.equal(G(u, s, 0), u)
