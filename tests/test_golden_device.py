"""The detector geometry against the device the paper describes (Sec. 2; the numbers are
in tests/golden/pget_device.txt).

The line of every detector is recovered from the oracle's own readings. With μ = 0, a
constant emission map and the row-index ramp are both reproduced exactly by bilinear
sampling, so for a ray at height c + s the ratio of the two readings is c + s. At φ = 0,
bank A looks along +x and bank B along -x. Checks:
- the 2 × 91 heights of one angle are distinct and evenly spaced by the effective spacing;
- each bank alone is spaced by twice that (the detector pitch of the half-pitch
  interleave);
- bank A is centred on the grid, and bank B's lines fall midway between bank A's;
- the pitch holds an element;
- the library picks the same two banks for 2 × 91 detectors.
"""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "pget_device.txt")


def _device():
    d = {}
    for line in open(GOLDEN):
        line = line.split("#")[0].strip()
        if line:
            k, v = (x.strip() for x in line.split("="))
            d[k] = float(v)
    return d


def test_detector_lines_interleave_to_the_effective_spacing(O):
    dev = _device()
    nb, per = int(dev["banks"]), int(dev["detectors_per_bank"])
    pitch = 2.0 * dev["effective_spacing_mm"]  # one pixel = 1 mm
    assert pitch >= dev["element_width_mm"]
    n = 384  # every detector line crosses the grid's interior rows: |s| <= 182 < (n - 1) / 2
    g = O.geom(n, 1, nb * per, n_sub=1, det_pitch=pitch, step=1.0)
    assert O.geom_info(g)["n_banks"] == nb and O.geom_info(g)["pitch"] == pitch
    zero = np.zeros((n, n))
    ones = np.ones((n, n))
    ramp = np.repeat(np.arange(n, dtype=float)[:, None], n, axis=1)  # value = row index
    y1 = O.forward(g, ones, zero)[0]
    y2 = O.forward(g, ramp, zero)[0]
    assert np.all(y1 > 0)
    heights = y2 / y1
    a, b = np.sort(heights[:per]), np.sort(heights[per:])
    np.testing.assert_allclose(np.diff(a), pitch, rtol=0, atol=1e-9)
    np.testing.assert_allclose(np.diff(b), pitch, rtol=0, atol=1e-9)
    both = np.sort(heights)
    np.testing.assert_allclose(np.diff(both), dev["effective_spacing_mm"], rtol=0, atol=1e-9)
    # bank A is centred on the grid and bank B's lines fall midway between bank A's
    assert abs(a.mean() - 0.5 * (n - 1)) <= 1e-9
    np.testing.assert_allclose(np.mod(b - a[0], pitch), 0.5 * pitch, rtol=0, atol=1e-9)


def test_library_takes_two_banks_for_the_device():
    from paper_2604_26745_gb300 import pget
    dev = _device()
    nb, per = int(dev["banks"]), int(dev["detectors_per_bank"])
    info = pget.geometry_info(pget.geometry(128, 360, nb * per, n_sub=5))
    assert info["n_banks"] == nb
