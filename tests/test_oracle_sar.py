"""Pins for the oracle's SAR compression and point-target metrics (CPU only).

Closed forms used (noise-free, unit-modulus chirps, integer target cells):

* range matched-filter peak = sum |s_r|^2 = M = 480 at the target cell;
* with both filters unnormalised the image peak is M * L_a;
* an unweighted band-limited response has PSLR -13.26 dB and a 3 dB width
  of 0.886 / (band fraction) cells: 0.886 * fs / B = 1.063 range cells and
  0.886 / 0.8 = 1.108 azimuth cells;
* matched-filter SNR gain: image SNR = M L_a a^2 / sigma^2 (76.9 dB at a = 1).

The metric code is pinned separately on an analytic separable Dirichlet
response, which involves no SAR code at all.
"""

import numpy as np
import pytest

from oracle import fft as F
from oracle import metrics, sar
from paper_2605_28451_gb300 import synth

M = synth.range_chirp_params()[0]
LA = synth.AZIMUTH_APERTURE


def test_chirp_constants():
    m, k, fs = synth.range_chirp_params()
    assert m == 480 and k == pytest.approx(2.5e13) and fs == 120e6


@pytest.fixture(scope="module")
def clean_scene():
    t = [(1024, 1024, 1.0)]
    sc = synth.point_target_scene(2048, 2048, noise=False, targets=t)
    return sc, t


def test_range_peak_is_pulse_energy(clean_scene):
    sc, t = clean_scene
    hr = sar.matched_filter(sc.ref_range, False)
    rc = sar.range_compress(sc.raw[1000:1040], hr)
    peak = np.abs(rc[:, 1024])
    assert np.allclose(peak, M, rtol=1e-12)
    assert np.all(np.argmax(np.abs(rc), axis=1) == 1024)


def test_image_peak_unnormalised_filters(clean_scene):
    sc, t = clean_scene
    hr = sar.matched_filter(sc.ref_range, False)
    ha = sar.matched_filter(sc.ref_azimuth, False)
    img = sar.range_doppler_image(sc.raw, hr, ha)
    assert np.unravel_index(np.argmax(np.abs(img)), img.shape) == (1024, 1024)
    assert abs(img[1024, 1024]) == pytest.approx(M * LA, rel=1e-12)


def test_peak_normalised_azimuth_filter_bounded(clean_scene):
    sc, _ = clean_scene
    ha = sar.matched_filter(sc.ref_azimuth, True)
    assert np.max(np.abs(ha)) == pytest.approx(1.0, rel=1e-15)


def test_point_target_closed_forms(clean_scene):
    sc, t = clean_scene
    hr = sar.matched_filter(sc.ref_range, False)
    ha = sar.matched_filter(sc.ref_azimuth, True)
    img = sar.range_doppler_image(sc.raw, hr, ha)
    m = metrics.point_target_metrics(img, t)[0]
    assert m["peak_cell"] == (1024, 1024)
    assert m["pslr_range_db"] == pytest.approx(-13.26, abs=0.2)
    assert m["pslr_azimuth_db"] == pytest.approx(-13.26, abs=0.2)
    assert m["width_range_cells"] == pytest.approx(0.886 * 120e6 / 100e6, rel=0.02)
    assert m["width_azimuth_cells"] == pytest.approx(0.886 / 0.8, rel=0.02)
    assert -10.3 <= m["islr_range_db"] <= -9.4
    assert -10.3 <= m["islr_azimuth_db"] <= -9.4


def _dirichlet(n, frac, x0):
    """Band-limited unit response: inverse DFT of a flat band of width frac*n centred at 0."""
    k = np.fft.fftfreq(n) * n
    band = (np.abs(k) <= frac * n / 2).astype(float)
    spec = band * np.exp(-2j * np.pi * k * x0 / n)
    return F.ifft(spec)


def test_metric_code_on_analytic_response():
    n = 512
    r = _dirichlet(n, 0.8, 200.3)
    a = _dirichlet(n, 0.5, 300.0)
    img = np.outer(a, r)
    m = metrics.point_target_metrics(img, [(300, 200, 1.0)], guard=8)[0]
    assert m["pslr_range_db"] == pytest.approx(-13.26, abs=0.15)
    assert m["pslr_azimuth_db"] == pytest.approx(-13.26, abs=0.15)
    assert m["width_range_cells"] == pytest.approx(0.886 / 0.8, rel=0.01)
    assert m["width_azimuth_cells"] == pytest.approx(0.886 / 0.5, rel=0.01)


def test_sqnr_alignment_and_cap():
    rng = np.random.default_rng(0)
    y = rng.standard_normal(1000) + 1j * rng.standard_normal(1000)
    e = 1e-3 * (rng.standard_normal(1000) + 1j * rng.standard_normal(1000))
    base = metrics.sqnr_db(y, y + e)
    assert metrics.sqnr_db(y, 0.25 * (y + e)) == pytest.approx(base, abs=1e-6)
    assert metrics.sqnr_db(y, 0.25 * (y + e), align=False) < 3.0
    assert metrics.sqnr_db(y, y) == metrics.SQNR_CAP_DB
    assert base == pytest.approx(10 * np.log10(np.sum(np.abs(y) ** 2) / np.sum(np.abs(e) ** 2)), abs=0.01)


def test_naive_schedule_overflows_fp16_and_bfp_does_not(clean_scene):
    sc, _ = clean_scene
    hr = sar.matched_filter(sc.ref_range, False)
    m = sar.stage_maxima(sc.raw[1024:1025], hr)
    assert m["naive_out"] > 65520.0 * 10
    for key in ("spectrum", "bfp_pre", "bfp_out"):
        assert m[key] < 65504.0 / 2
    rc = sar.range_compress(sc.raw, hr)
    ha = sar.matched_filter(sc.ref_azimuth, True)
    ma = sar.stage_maxima(rc, ha, axis=0)
    for key in ("spectrum", "bfp_pre", "bfp_out"):
        assert ma[key] < 65504.0 / 2
    assert ma["naive_out"] > 65520.0


@pytest.mark.slow
def test_target_snr_closed_form():
    sc = synth.point_target_scene(2048, 2048)
    hr = sar.matched_filter(sc.ref_range, False)
    ha = sar.matched_filter(sc.ref_azimuth, True)
    img = sar.range_doppler_image(sc.raw, hr, ha)
    ms = metrics.point_target_metrics(img, sc.targets)
    for m in ms[:4]:
        expect = 10 * np.log10(M * LA / synth.NOISE_VARIANCE) + 20 * np.log10(m["amplitude"])
        assert m["snr_db"] == pytest.approx(expect, abs=0.6)
