"""Planted mistakes in the SAR, autofocus, convolution and block-exponent oracles (CPU only).

Each test plants one plausible mistake in an oracle module (a dropped
conjugate, a wrong axis, a flipped sign, an off-by-one exponent) and checks
that the quantity the module's pins test moves far outside its tolerance.
The mistakes are planted by swapping the module's reference to numpy (or to
a helper) for a proxy, so the oracle's own code runs unchanged around them.
"""

import numpy as np
import pytest

from oracle import autofocus as AF
from oracle import bfp, conv, sar
from oracle import metrics
from paper_2605_28451_gb300 import synth


class _Proxy:
    """A module stand-in: the given attributes, everything else from ``base``."""

    def __init__(self, base, **over):
        self._base = base
        self.__dict__.update(over)

    def __getattr__(self, name):
        return getattr(self._base, name)


M = synth.range_chirp_params()[0]


@pytest.fixture(scope="module")
def clean_scene():
    return synth.point_target_scene(512, 1024, noise=False, aperture=128, targets=[(256, 512, 1.0)])


def _range_peak_error(sc):
    """The range pin: |rc| at the target cell equals M on every line of the aperture."""
    hr = sar.matched_filter(sc.ref_range, False)
    rc = sar.range_compress(sc.raw[250:262], hr)
    return float(np.max(np.abs(np.abs(rc[:, 512]) - M)) / M)


def test_matched_filter_without_conjugate_is_caught(clean_scene, monkeypatch):
    assert _range_peak_error(clean_scene) <= 1e-12
    monkeypatch.setattr(sar, "np", _Proxy(np, conj=lambda a: a))
    assert _range_peak_error(clean_scene) > 0.5


def _image_peak(sc):
    """The image pin: with both filters unnormalised the peak is M L_a at the target cell."""
    hr = sar.matched_filter(sc.ref_range, False)
    ha = sar.matched_filter(sc.ref_azimuth, False)
    img = sar.range_doppler_image(sc.raw, hr, ha)
    return np.unravel_index(np.argmax(np.abs(img)), img.shape), float(np.max(np.abs(img)))


def test_azimuth_compression_along_range_is_caught(monkeypatch):
    """A square scene, so that compressing the wrong axis still runs."""
    sc = synth.point_target_scene(512, 512, noise=False, aperture=128, targets=[(256, 256, 1.0)])
    cell, peak = _image_peak(sc)
    assert cell == (256, 256) and peak == pytest.approx(M * 128, rel=1e-12)
    real_compress = sar.compress
    monkeypatch.setattr(sar, "compress", lambda x, h, axis: real_compress(x, h, -1))
    cell, peak = _image_peak(sc)
    assert cell != (256, 256) or abs(peak - M * 128) > 0.1 * M * 128


@pytest.fixture(scope="module")
def af_case():
    n_az, n_rg, ap = 128, 32, 64
    sc = synth.point_target_scene(n_az, n_rg, aperture=ap, targets=[(64, 10, 1.0), (40, 22, 0.5)])
    hr = sar.matched_filter(synth.centred_reference(synth.range_chirp()[:20], n_rg), False)
    ha = sar.matched_filter(sc.ref_azimuth, True)
    rc = sar.range_compress(sc.raw, hr)
    u = rc * np.exp(1j * synth.phase_error(n_az, quad_rad=2.0))[:, None]
    return u, ha


def _fd_mismatch(u, ha):
    """The gradient pin: analytic gradient against FP64 central differences."""
    phi = np.zeros(u.shape[0])
    _, g = AF.entropy_and_grad(u, phi, ha)
    pulses = np.arange(0, u.shape[0], 16)
    fd = AF.central_difference(u, phi, ha, pulses, h=1e-4)
    return float(np.linalg.norm(g[pulses] - fd) / np.linalg.norm(fd))


@pytest.mark.parametrize("kind", ["adjoint_without_conjugate", "gradient_sign", "dropped_entropy_term"])
def test_autofocus_adjoint_mistakes_are_caught(af_case, monkeypatch, kind):
    u, ha = af_case
    assert _fd_mismatch(u, ha) <= 1e-6
    if kind == "adjoint_without_conjugate":
        real_az = AF._sar.azimuth_compress
        calls = {"n": 0}

        def az(x, h):
            calls["n"] += 1
            # entropy_and_grad calls it twice: forward, then the adjoint with conj(Ha)
            return real_az(x, np.conj(h) if calls["n"] % 2 == 0 else h)
        monkeypatch.setattr(AF, "_sar", _Proxy(sar, azimuth_compress=az))
        _, g = AF.entropy_and_grad(u, np.zeros(u.shape[0]), ha)
        monkeypatch.undo()
        pulses = np.arange(0, u.shape[0], 16)
        fd = AF.central_difference(u, np.zeros(u.shape[0]), ha, pulses, h=1e-4)
        assert np.linalg.norm(g[pulses] - fd) > 1e-3 * np.linalg.norm(fd)
        return
    if kind == "gradient_sign":
        monkeypatch.setattr(AF, "np", _Proxy(np, imag=lambda a: -np.imag(a)))
    else:
        real_where = np.where

        def where(cond, a, b):
            # G = -(ln p + E) / S * I  becomes  -(ln p) / S * I
            if isinstance(a, np.ndarray) and a.dtype == np.float64:
                return real_where(cond, a - where.e_term, b)
            return real_where(cond, a, b)
        # -(ln p + E)/S  minus  (-E/S)  =  -(ln p)/S
        e, _ = AF.entropy_and_grad(u, np.zeros(u.shape[0]), ha)
        where.e_term = -e / float(np.sum(np.abs(AF.image(u, np.zeros(u.shape[0]), ha)) ** 2))
        monkeypatch.setattr(AF, "np", _Proxy(np, where=where))
    _, g = AF.entropy_and_grad(u, np.zeros(u.shape[0]), ha)
    monkeypatch.undo()
    pulses = np.arange(0, u.shape[0], 16)
    fd = AF.central_difference(u, np.zeros(u.shape[0]), ha, pulses, h=1e-4)
    assert np.linalg.norm(g[pulses] - fd) > 1e-3 * np.linalg.norm(fd)


def test_correlation_without_conjugate_is_caught(monkeypatch):
    x = synth.complex_gaussian(2, 64, seed=1)
    g = synth.complex_gaussian(1, 64, seed=2)[0]
    direct = conv.correlate_direct(x, g)
    assert metrics.rel_l2(direct, conv.spectral(x, conv.correlation_filter(g))) <= 1e-12
    monkeypatch.setattr(conv, "np", _Proxy(np, conj=lambda a: a))
    assert metrics.rel_l2(direct, conv.spectral(x, conv.correlation_filter(g))) > 0.5


def test_block_exponent_off_by_one_is_caught(monkeypatch):
    rng = np.random.default_rng(3)
    v = (rng.standard_normal((50, 8)) + 1j * rng.standard_normal((50, 8))) * 10.0 ** rng.integers(-9, 9, (50, 1))
    m = bfp.block_max(v)

    def smallest(mi):
        return min(e for e in range(-80, 81) if mi * 2.0 ** -e <= bfp.DEFAULT_LIMIT)
    want = np.array([smallest(mi) for mi in m])
    assert np.array_equal(bfp.block_exponent(v), want)
    real_ceil = np.ceil
    monkeypatch.setattr(bfp, "np", _Proxy(np, ceil=lambda a: real_ceil(a) + 1,
                                          where=lambda c, a, b: b))      # skip the exactness corrections
    assert not np.array_equal(bfp.block_exponent(v), want)


def test_rcmc_in_the_wrong_direction_is_caught(monkeypatch):
    """RCMC that moves each Doppler row the wrong way doubles the migration
    instead of removing it; the straightened-peak pin sees about a cell."""
    from oracle import rda
    geo = synth.radar_geometry()
    sc = synth.migrating_scene(2048, 1024, [(1024, 512, 1.0)])
    rd = rda.range_doppler(sar.range_compress(sc.raw, sar.matched_filter(sc.ref_range, False)))
    f = rda.doppler_frequencies(2048, geo.prf_hz)
    k = int(np.argmin(np.abs(f - 0.33 * geo.prf_hz)))

    def peak(row):
        up = np.abs(np.fft.ifft(np.concatenate([np.fft.fft(row)[:512], np.zeros(31 * 1024),
                                                np.fft.fft(row)[512:]])))
        return float(np.argmax(up)) / 32

    assert abs(peak(rda.rcmc(rd, geo, 1024)[k]) - 512) <= 0.05
    real_shift = rda.shift_rows
    monkeypatch.setattr(rda, "shift_rows", lambda x, cells: real_shift(x, -np.asarray(cells)))
    assert abs(peak(rda.rcmc(rd, geo, 1024)[k]) - 512) > 0.5
