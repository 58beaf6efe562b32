"""The library's host-side geometry against exact arithmetic, on the CPU.

Sub-rays of neighbouring detectors can lie on the same line. The library traces such
lines once, as slots of a lattice: per bank, from the smallest to the largest sub-ray
offset, with the greatest common spacing of all offsets. Here the offsets are rebuilt
as exact rationals from the detector and sub-ray definitions:
- detector d of bank b at (d − (nb − 1)/2 + b/2)·p;
- triangular sub-rays at (k − (S − 1)/2)·2p/(S + 1), box sub-rays at (k − (S − 1)/2)·p/S.

The slot count of the widest bank must equal the library's max_slots. The GPU parity
tests then show that tracing slots instead of sub-rays changes no result.
"""
from fractions import Fraction
from functools import reduce
from math import gcd

import pytest

from paper_2604_26745_gb300 import pget as P


def _offsets(nb, S, collimator, bank):
    out = set()
    for d in range(nb):
        centre = Fraction(2 * d - (nb - 1) + bank, 2)
        for k in range(S):
            u = Fraction(2 * k - (S - 1), S + 1) if collimator == 1 else Fraction(2 * k - (S - 1), 2 * S)
            out.add(centre + u)
    return sorted(out)


def _slots(offsets):
    den = reduce(lambda a, x: a * x.denominator // gcd(a, x.denominator), offsets, 1)
    ints = [int(x * den) for x in offsets]
    step = reduce(gcd, (v - ints[0] for v in ints[1:]), 0) or 1
    return (ints[-1] - ints[0]) // step + 1


@pytest.mark.parametrize("n_det,S,collimator", [(182, 5, 1), (91, 5, 1), (182, 4, 0), (91, 3, 1), (182, 10, 1),
                                                (182, 1, 1), (91, 7, 0), (182, 2, 1), (90, 6, 0)])
def test_slot_lattice_matches_exact_offsets(n_det, S, collimator):
    banks = 2 if n_det == 182 else 1
    nb = n_det // banks
    per_bank = [_offsets(nb, S, collimator, b) for b in range(banks)]
    want = max(_slots(o) for o in per_bank)
    info = P.geometry_info(P.geometry(64, 8, n_det, n_sub=S, collimator=collimator))
    assert info["max_slots"] == want
    assert info["max_slots"] >= max(len(o) for o in per_bank)  # every sub-ray has a slot


def test_benchmark_geometry_counts():
    """The counts quoted for the single-request geometry: 455 sub-rays of a bank on 275
    distinct lines; at S = 10, 1009 slots of which 910 carry a sub-ray."""
    o5 = _offsets(91, 5, 1, 0)
    assert len(o5) == 275 and _slots(o5) == 275
    o10 = _offsets(91, 10, 1, 0)
    assert len(o10) == 910 and _slots(o10) == 1009


def test_allocation_free_path_refuses_before_any_work():
    """pget_forward_noalloc validates its geometry on the host like the context path.

    Oversized detector counts are refused at once (PGET_EINVAL), not walked. Without a GPU
    a valid geometry ends in PGET_ECUDA at the first CUDA call. The array arguments are
    placeholders that the host code never reads. This test runs only where there is no
    GPU, so they can never reach a kernel."""
    import ctypes
    import time

    import torch
    if torch.cuda.is_available():
        pytest.skip("placeholder pointers are for machines without a GPU")
    L = P.load()
    fake = ctypes.c_void_p(256)
    t0 = time.perf_counter()
    for n_det, want in ((2 ** 31 - 1, P.PGET_EINVAL), (1025, P.PGET_EINVAL), (182, P.PGET_ECUDA)):
        g = P.geometry(16, 8, n_det, n_sub=64 if n_det != 182 else 5)
        assert L.pget_forward_noalloc(ctypes.byref(g), P.PGET_F32, fake, fake, fake, None) == want
    assert time.perf_counter() - t0 < 5.0
