"""Random geometries through the host-side validation, on the CPU.

Any pget_geometry, including negative, huge and non-finite fields, must come back from
pget_geometry_info either as sizes inside the documented limits or as a refusal
(ValueError for PGET_EINVAL, PgetError otherwise). It must never crash the process, hang
or allocate without bound. Sizes are drawn so that a valid geometry stays small in host
memory; the limits themselves are checked in tests/test_abi.py.
"""
import math

import pytest

hyp = pytest.importorskip("hypothesis")
st = pytest.importorskip("hypothesis.strategies")

from paper_2604_26745_gb300 import pget as P  # noqa: E402

ints = lambda lo, hi, extra: st.one_of(st.integers(lo, hi), st.sampled_from(extra))
floats = st.one_of(st.floats(allow_nan=True, allow_infinity=True, width=64),
                   st.sampled_from([0.0, -1.0, 1e-300, 1e300, 0.5, 2.0]))


@hyp.settings(max_examples=400, deadline=None, derandomize=True)
@hyp.given(n=ints(-4, 300, [0, 1, 2, 16384, 16385, -(2 ** 31)]),
           n_angles=ints(-4, 64, [0, 1, (1 << 20) + 1, 2 ** 31 - 1, -(2 ** 31)]),
           n_det=ints(-4, 400, [0, 1, 91, 182, 2 ** 31 - 1]),
           n_sub=ints(-2, 70, [0, 1, 64, 65]),
           collimator=ints(-2, 3, [0, 1]),
           n_banks=ints(-2, 4, [0, 1, 2]),
           step=floats, fov_radius=floats, det_pitch=floats)
def test_geometry_validation_never_crashes(n, n_angles, n_det, n_sub, collimator, n_banks, step, fov_radius,
                                           det_pitch):
    g = P.pget_geometry(n=n, n_angles=n_angles, n_det=n_det, n_banks=n_banks, n_sub=n_sub, collimator=collimator,
                        step=step, fov_radius=fov_radius, det_pitch=det_pitch)
    try:
        info = P.geometry_info(g)
    except (ValueError, P.PgetError):
        return
    assert 2 <= n <= 16384 and 1 <= n_angles <= (1 << 20) and 1 <= n_sub <= 64 and collimator in (0, 1)
    assert info["n_banks"] in (1, 2) and n_det % info["n_banks"] == 0
    assert 1 <= info["n_samples"] <= (1 << 20) and 1 <= info["max_slots"] <= 1024
    for k in ("fov_radius", "det_pitch"):
        assert math.isfinite(info[k])
