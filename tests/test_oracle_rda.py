"""Pins for the range-Doppler oracle with range-cell migration correction (CPU only).

Closed forms used:
* the hyperbolic range history: the range-compressed echo of pulse eta peaks
  at r_k + (sqrt(R^2 + (v t)^2) - R) / range_cell, t = (eta - eta_k) / PRF;
* stationary phase: in the range-Doppler domain the target sits at
  r_k + dR(f) / range_cell, dR(f) = R (1 / D(f) - 1), and its small-f form
  lambda^2 R f^2 / (8 v^2);
* after RCMC and the matched azimuth filter a noise-free unit target peaks at
  M L_a (unnormalised filters), with PSLR -13.26 dB and 3 dB widths of
  0.886 fs / B = 1.063 range cells and 0.886 / 0.8 = 1.108 azimuth cells;
* band-limited shifts: integer shifts are rotations, and a sampled cosine
  shifted by half a sample is the cosine at the half-sample points.
"""

import math

import numpy as np
import pytest

from oracle import fft as F
from oracle import metrics, rda, sar
from paper_2605_28451_gb300 import synth

pytestmark = pytest.mark.slow

N_AZ, N_RG, LA = 2048, 1024, synth.AZIMUTH_APERTURE
M = synth.range_chirp_params()[0]
GEO = synth.radar_geometry()


def _subcell_peak(row: np.ndarray, factor: int = 32) -> float:
    """Position of the largest |.| of a band-limited row, interpolated by zero-padding its DFT."""
    n = row.shape[0]
    spec = F.fft(row)
    big = np.zeros(n * factor, dtype=np.complex128)
    big[: n // 2] = spec[: n // 2]
    big[-n // 2:] = spec[-n // 2:]
    up = F.ifft(big)
    return float(np.argmax(np.abs(up))) / factor


@pytest.fixture(scope="module")
def centre():
    sc = synth.migrating_scene(N_AZ, N_RG, [(1024, 512, 1.0)])
    hr = sar.matched_filter(sc.ref_range, False)
    rc = sar.range_compress(sc.raw, hr)
    return {
        "hr": hr, "rc": rc, "rd": rda.range_doppler(rc),
        "img": rda.image(sc.raw, hr, GEO, LA),
        "img_no_rcmc": rda.image(sc.raw, hr, GEO, LA, correct_migration=False),
    }


@pytest.fixture(scope="module")
def edge():
    sc = synth.migrating_scene(N_AZ, N_RG, [(1024, 272, 1.0)])
    hr = sar.matched_filter(sc.ref_range, False)
    return {
        "img": rda.image(sc.raw, hr, GEO, LA),
        "img_fixed_rate": rda.image(sc.raw, hr, GEO, LA, range_dependent=False),
    }


def test_geometry_closed_forms():
    assert GEO.range_cell_m == pytest.approx(synth.SPEED_OF_LIGHT_MPS / 240e6)
    ka = 2 * 100.0 ** 2 / (0.03 * 20e3)                         # 33.3 Hz/s at R0
    assert ka / GEO.prf_hz ** 2 == pytest.approx(0.8 / LA)      # same k_a as the migration-free scene
    assert float(rda.azimuth_rate(20e3, GEO)) == pytest.approx(0.8 / LA)
    t_edge = (LA / 2) / GEO.prf_hz
    rcm_cells = (math.hypot(20e3, 100.0 * t_edge) - 20e3) / GEO.range_cell_m
    assert rcm_cells == pytest.approx(1.23, abs=0.01)           # about 1.2 range cells at the aperture edge
    # the Doppler-domain migration at the edge's Doppler frequency agrees to second order
    f_edge = ka * t_edge
    assert float(rda.migration_m(f_edge, 20e3, 0.03, 100.0)) / GEO.range_cell_m == pytest.approx(rcm_cells, rel=0.01)
    f = np.array([0.0, 1.0, 10.0, 50.0])
    small = 0.03 ** 2 * 20e3 * f ** 2 / (8 * 100.0 ** 2)
    assert np.allclose(rda.migration_m(f, 20e3, 0.03, 100.0), small, rtol=2e-3, atol=0)


def test_doppler_bins_are_signed():
    f = rda.doppler_frequencies(8, 80.0)
    assert f.tolist() == [0.0, 10.0, 20.0, 30.0, -40.0, -30.0, -20.0, -10.0]


def test_band_limited_shift():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((3, 64)) + 1j * rng.standard_normal((3, 64))
    assert np.allclose(rda.shift_rows(x, np.array([0.0, 1.0, -5.0])),
                       np.stack([x[0], np.roll(x[1], 1), np.roll(x[2], -5)]), atol=1e-12)
    n = 64
    r = np.arange(n)
    c = np.cos(2 * np.pi * 5 * r / n)[None, :]
    got = rda.shift_rows(c, np.array([0.5]))
    assert np.allclose(got, np.cos(2 * np.pi * 5 * (r - 0.5) / n), atol=1e-12)
    nyq = np.cos(np.pi * r)[None, :]                              # the Nyquist row stays real
    assert np.max(np.abs(rda.shift_rows(nyq, np.array([0.25])).imag)) < 1e-12


@pytest.mark.parametrize("offset", [-512, -384, -256, 0, 128, 300, 511])
def test_echo_follows_the_hyperbolic_range_history(centre, offset):
    t = offset / GEO.prf_hz
    r_k = 20e3                                                    # target at the scene-centre cell
    want = 512 + (math.hypot(r_k, 100.0 * t) - r_k) / GEO.range_cell_m
    assert _subcell_peak(centre["rc"][1024 + offset]) == pytest.approx(want, abs=0.04)


def test_rcmc_removes_the_doppler_dependent_migration(centre):
    rd = centre["rd"]
    f = rda.doppler_frequencies(N_AZ, GEO.prf_hz)
    bins = [k for k in range(0, N_AZ, 61) if abs(f[k]) <= 0.35 * GEO.prf_hz]
    straight = rda.rcmc(rd, GEO, N_RG)
    for k in bins:
        migr = float(rda.migration_m(f[k], 20e3, GEO.wavelength_m, GEO.speed_mps)) / GEO.range_cell_m
        assert _subcell_peak(rd[k]) == pytest.approx(512 + migr, abs=0.05), k
        assert _subcell_peak(straight[k]) == pytest.approx(512, abs=0.05), k
    assert max(abs(f[k]) for k in bins) > 0.3 * GEO.prf_hz      # reaches migrations of about a cell


def test_rcmc_focuses_the_target(centre):
    img, raw_img = np.abs(centre["img"]), np.abs(centre["img_no_rcmc"])
    assert np.unravel_index(np.argmax(img), img.shape) == (1024, 512)
    assert img.max() >= 0.99 * M * LA
    assert raw_img.max() <= 0.8 * M * LA                          # uncorrected: energy split over range cells


def test_focused_response_closed_forms(centre):
    (m,) = metrics.point_target_metrics(centre["img"], [(1024, 512, 1.0)])
    assert m["pslr_range_db"] == pytest.approx(-13.26, abs=0.3)
    assert m["pslr_azimuth_db"] == pytest.approx(-13.26, abs=0.3)
    assert m["width_range_cells"] == pytest.approx(0.886 * 120e6 / 100e6, rel=0.02)
    assert m["width_azimuth_cells"] == pytest.approx(0.886 / 0.8, rel=0.02)


def test_azimuth_filter_must_follow_the_range(edge):
    """300 m from the scene centre the FM rate differs by 1.5 %: ten radians
    at the aperture edge, enough to defocus a filter built for R0."""
    img, fixed = np.abs(edge["img"]), np.abs(edge["img_fixed_rate"])
    assert np.unravel_index(np.argmax(img), img.shape) == (1024, 272)
    assert img.max() >= 0.99 * M * LA
    assert fixed.max() <= 0.5 * M * LA
