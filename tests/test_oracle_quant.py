"""Pins for the oracle's storage-format rounding (CPU only).

Edge values come from the IEEE binary16 and OCP FP8 definitions.  The FP8
rounders are also checked against every finite value decoded from the 256
bit patterns of each format: each must round to itself, and a dense sweep
must never produce a value outside that set.
"""

import numpy as np
import pytest

from oracle import quant as Q


def test_binary16_edges():
    v = np.array([65504.0, 65519.99, 65520.0, 1e6, -65520.0,
                  1 + 2.0 ** -11, 1 + 3 * 2.0 ** -11, 2.0 ** -24, 2.0 ** -25, 1.5 * 2.0 ** -24])
    r = Q.round_binary16(v)
    assert r[0] == 65504.0 and r[1] == 65504.0
    assert np.isinf(r[2]) and np.isinf(r[3]) and r[4] == -np.inf
    assert r[5] == 1.0                       # tie to even (down)
    assert r[6] == 1 + 2.0 ** -9             # tie to even (up)
    assert r[7] == 2.0 ** -24                # smallest subnormal
    assert r[8] == 0.0                       # tie to even -> 0
    assert r[9] == 2.0 ** -23


def _decode(bits, fmt):
    """Value of an FP8 bit pattern from the format definition."""
    ebits, mbits, bias = {"e4m3": (4, 3, 7), "e5m2": (5, 2, 15)}[fmt]
    s = (bits >> 7) & 1
    e = (bits >> mbits) & ((1 << ebits) - 1)
    m = bits & ((1 << mbits) - 1)
    if fmt == "e4m3" and e == 15 and m == 7:
        return np.nan
    if fmt == "e5m2" and e == 31:
        return np.nan if m else (-np.inf if s else np.inf)
    if e == 0:
        mag = m * 2.0 ** (1 - bias - mbits)
    else:
        mag = (1 + m / 2.0 ** mbits) * 2.0 ** (e - bias)
    return -mag if s else mag


@pytest.mark.parametrize("fmt,vmax", [("e4m3", 448.0), ("e5m2", 57344.0)])
def test_fp8_grid_fixed_points(fmt, vmax):
    vals = np.array([_decode(b, fmt) for b in range(256)])
    finite = vals[np.isfinite(vals)]
    assert np.max(finite) == vmax
    assert np.array_equal(Q.round_fp8(finite, fmt), finite)
    sweep = np.concatenate([np.linspace(-vmax * 1.5, vmax * 1.5, 200001),
                            np.geomspace(1e-8, vmax * 2, 50001)])
    out = Q.round_fp8(sweep, fmt)
    assert np.all(np.isin(out, finite))
    # nearest: no finite grid value is strictly closer than the chosen one
    inside = np.abs(sweep) <= vmax
    grid = np.sort(np.unique(finite))
    pos = np.clip(np.searchsorted(grid, sweep[inside]), 1, grid.size - 1)
    best = np.minimum(np.abs(grid[pos] - sweep[inside]), np.abs(grid[pos - 1] - sweep[inside]))
    assert np.all(np.abs(out[inside] - sweep[inside]) <= best + 1e-300)


def test_fp8_edges():
    e4 = Q.round_fp8(np.array([464.0, 1e6, -1e6, 2.0 ** -9, 2.0 ** -10, 1.0625, 1.1875, np.nan]), "e4m3")
    assert e4[0] == 448.0 and e4[1] == 448.0 and e4[2] == -448.0
    assert e4[3] == 2.0 ** -9 and e4[4] == 0.0
    assert e4[5] == 1.0 and e4[6] == 1.25
    assert np.isnan(e4[7])
    e5 = Q.round_fp8(np.array([1e9, 2.0 ** -16, 1.125, 1.375, -3.0]), "e5m2")
    assert e5[0] == 57344.0 and e5[1] == 2.0 ** -16
    assert e5[2] == 1.0 and e5[3] == 1.5 and e5[4] == -3.0


def test_complex_rounding_is_componentwise():
    z = np.array([1.0625 + 464j])
    assert Q.round_fp8(z, "e4m3")[0] == 1.0 + 448j
