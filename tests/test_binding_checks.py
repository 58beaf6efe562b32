"""The binding's argument checks, on the CPU (no compute call is made).

A raw pointer cannot say where it points, how wide its elements are or how many there
are. So the binding checks each array argument before the C call:
- a CUDA tensor for the device entry points, a CPU tensor for the host-buffer solve;
- contiguity;
- the precision's element size;
- at least the elements the geometry needs.

A mismatch raises ValueError (TypeError for a non-tensor) and the library is never
called with it.
"""
import pytest
import torch

from paper_2604_26745_gb300 import pget as P


class _Ctx:
    h = None  # the library is never reached: the checks raise first
    device = 0


G = P.geometry(16, 8, 91)
NN, M = 16 * 16, 8 * 91


def test_device_entry_points_refuse_host_tensors():
    x = torch.zeros((16, 16), dtype=torch.float32)
    r = torch.zeros((8, 91), dtype=torch.float32)
    p = P.default_params(precision=P.PGET_F32)
    calls = [
        lambda: P.pget_forward(_Ctx, G, P.PGET_F32, x, x),
        lambda: P.pget_jvp(_Ctx, G, P.PGET_F32, x, x, x, x),
        lambda: P.pget_vjp(_Ctx, G, P.PGET_F32, x, x, r),
        lambda: P.pget_reg_apply(_Ctx, 16, P.PGET_F32, 0.1, 1e-3, x, x),
        lambda: P.pget_lm_solve(_Ctx, G, p, r, x, x),
        lambda: P.pget_lm_trial(_Ctx, G, p, r, x, x),
        lambda: P.pget_project(_Ctx, p, x, x),
        lambda: P.pget_submit(_Ctx, G, p, r),
        lambda: P.pget_forward_noalloc(G, P.PGET_F32, x, x, r),
    ]
    for call in calls:
        with pytest.raises(ValueError, match="CUDA tensor"):
            call()


@pytest.mark.parametrize("prec,dt", [(P.PGET_F64, torch.float32), (P.PGET_F32, torch.float64),
                                     (P.PGET_F32_KAHAN, torch.float16), (P.PGET_F32, torch.int32)])
def test_host_solve_refuses_the_wrong_element_type(prec, dt):
    p = P.default_params(precision=prec)
    y = torch.zeros((8, 91), dtype=dt)
    x = torch.zeros((16, 16), dtype=dt)
    with pytest.raises(ValueError, match="precision"):
        P.pget_lm_solve_host(_Ctx, G, p, y, x, x)


def test_host_solve_refuses_short_and_strided_arrays():
    p = P.default_params(precision=P.PGET_F32)
    y = torch.zeros((8, 91))
    x = torch.zeros((16, 16))
    with pytest.raises(ValueError, match="elements"):
        P.pget_lm_solve_host(_Ctx, G, p, y[:, :90].contiguous(), x, x)
    with pytest.raises(ValueError, match="elements"):
        P.pget_lm_solve_host(_Ctx, G, p, y, x[:15].contiguous(), x)
    with pytest.raises(ValueError, match="contiguous"):
        P.pget_lm_solve_host(_Ctx, G, p, y, torch.zeros((16, 32))[:, ::2], x)
    with pytest.raises(TypeError):
        P.pget_lm_solve_host(_Ctx, G, p, y, x, x.numpy())  # not a tensor


def test_sizes_come_from_the_geometry():
    """An array larger than needed is accepted (a prefix is read), exactly the size too."""
    a = torch.zeros(NN + 5)
    assert P._arr(a, P.PGET_F32, NN, None, "a", host=True) == a.data_ptr()
    assert P._arr(a[:NN], P.PGET_F32, NN, None, "a", host=True) == a.data_ptr()
    assert P._arr(None, P.PGET_F32, NN, None, "a") is None  # optional arguments stay NULL
