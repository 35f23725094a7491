"""The seeded input recipe (the synthetic stand-ins for the paper's workloads).

The paper leaves the SAR scene and the mixed-length batch underspecified; the
generators complete them.  These tests pin that completion:
- the LFM pulse's time-bandwidth product and sample count;
- the azimuth chirp's Doppler sweep;
- the target amplitudes and spacing;
- the noise level;
- the phase-error model;
- the uneven length distribution and its total of about 2^28 points.
None of the method's arithmetic is involved.
"""

import math

import numpy as np
import pytest

from paper_2605_28451_gb300 import synth


def test_complex_gaussian_is_seeded_standard_normal():
    a = synth.complex_gaussian(64, 1024, seed=7)
    assert np.array_equal(a, synth.complex_gaussian(64, 1024, seed=7))
    assert not np.array_equal(a, synth.complex_gaussian(64, 1024, seed=8))
    for part in (a.real, a.imag):
        assert abs(part.mean()) < 0.01
        assert abs(part.var() - 1.0) < 0.02


def test_range_chirp_matches_the_completed_radar_parameters():
    m, k, fs = synth.range_chirp_params()
    assert (m, fs) == (480, 120e6)                          # Tp = 4 us at 120 MHz
    assert k == pytest.approx(2.5e13)                       # B / Tp = 100 MHz / 4 us
    assert k * (m / fs) ** 2 == pytest.approx(400.0)        # time-bandwidth product
    s = synth.range_chirp()
    assert s.shape == (480,)
    assert np.allclose(np.abs(s), 1.0)
    # instantaneous frequency K t spans the 100 MHz bandwidth across the pulse
    dphase = np.diff(np.unwrap(np.angle(s))) * fs / (2 * math.pi)
    assert dphase.max() - dphase.min() == pytest.approx(100e6, rel=0.01)


def test_azimuth_chirp_sweeps_the_doppler_fraction_of_the_prf():
    s = synth.azimuth_chirp()
    assert s.shape == (1024,)
    assert np.allclose(np.abs(s), 1.0)
    f = np.diff(np.unwrap(np.angle(s))) / (2 * math.pi)     # cycles per pulse (PRF = 1)
    assert f.max() - f.min() == pytest.approx(0.8, rel=0.01)


def test_centred_reference_puts_the_pulse_centre_at_index_zero():
    pulse = np.arange(1, 11, dtype=np.complex128)           # M = 10
    ref = synth.centred_reference(pulse, 64)
    assert ref[0] == pulse[5]                               # sample M/2 at index 0
    assert ref[64 - 5] == pulse[0]                          # sample 0 at -M/2 mod n
    assert np.count_nonzero(ref) == 10


@pytest.mark.parametrize("n_az,n_rg", [(4096, 4096), (1024, 4096)])
def test_target_layout_amplitudes_positions_and_spacing(n_az, n_rg):
    t = synth.target_layout(n_az, n_rg, synth.AZIMUTH_APERTURE)
    assert len(t) == 8
    assert [a for _, _, a in t] == pytest.approx([10.0 ** (-k / 7.0) for k in range(8)])
    assert t[0][2] == 1.0 and t[-1][2] == pytest.approx(0.1)
    full = n_az // 2 > synth.AZIMUTH_APERTURE // 2 + 64
    lo_a, hi_a = (512 + 64, n_az - 512 - 64) if full else (64, n_az - 64)
    for i, (eta, r, _) in enumerate(t):
        assert lo_a <= eta <= hi_a and 256 <= r <= n_rg - 256
        for eta2, r2, _ in t[:i]:
            assert abs(eta - eta2) >= 128 or abs(r - r2) >= 128


def test_scene_noise_is_20_db_below_a_unit_target_per_sample():
    sc = synth.point_target_scene(512, 1024, targets=[])
    assert sc.raw.real.var() == pytest.approx(0.005, rel=0.03)
    assert sc.raw.imag.var() == pytest.approx(0.005, rel=0.03)
    assert np.mean(np.abs(sc.raw) ** 2) == pytest.approx(0.01, rel=0.03)


def test_scene_echo_is_the_outer_product_of_the_two_chirps():
    sc = synth.point_target_scene(2048, 2048, noise=False, targets=[(1000, 900, 0.5)])
    sr, sa = synth.range_chirp(), synth.azimuth_chirp()
    block = sc.raw[1000 - 512:1000 + 512, 900 - 240:900 + 240]
    assert np.allclose(block, 0.5 * np.outer(sa, sr))
    assert np.count_nonzero(sc.raw) == 1024 * 480


def test_phase_error_model():
    n = 4096
    quad = synth.phase_error(n, noise_rad=0.0)
    assert quad[0] == pytest.approx(4 * math.pi)             # 4 pi at the aperture edge
    assert quad[n // 2] == pytest.approx(0.0)                # 0 at the centre
    noise = synth.phase_error(n) - quad
    assert noise.std() == pytest.approx(0.3, rel=0.05)
    assert np.array_equal(synth.phase_error(n), synth.phase_error(n))


def test_uneven_lengths_follow_the_zipf_weights_and_total_about_2_to_28():
    lengths = synth.uneven_lengths(20000, seed=3)
    assert set(np.unique(lengths)) <= set(synth.UNEVEN_LENGTHS)
    assert int(lengths.sum()) == 251873792                   # 2^27.9, the workload's point count
    w = np.array([(i + 1.0) ** -0.5 for i in range(5)])
    w /= w.sum()
    counts = np.array([(lengths == n).sum() for n in synth.UNEVEN_LENGTHS])
    assert np.allclose(counts / 20000, w, atol=0.01)


def test_uneven_batch_packs_transforms_contiguously():
    lengths = np.array([256, 16, 4096])
    data, offsets = synth.uneven_batch(lengths, seed=1)
    assert data.shape == (256 + 16 + 4096,)
    assert offsets.tolist() == [0, 256, 272]


def test_migrating_scene_support_and_phase():
    """Each pulse of the aperture carries one unit-modulus pulse of M samples
    (give or take one where the fractional delay moves the window), and the
    pulse at the aperture centre has no migration: it equals the
    migration-free echo there."""
    m = synth.range_chirp_params()[0]
    sc = synth.migrating_scene(2048, 1024, [(1024, 512, 1.0)])
    rows = np.count_nonzero(sc.raw, axis=1)
    assert np.all((rows[512:1536] >= m - 1) & (rows[512:1536] <= m + 1))
    assert rows[:512].sum() == 0 and rows[1536:].sum() == 0
    assert np.allclose(np.abs(sc.raw[sc.raw != 0]), 1.0)
    flat = synth.point_target_scene(2048, 1024, noise=False, targets=[(1024, 512, 1.0)])
    assert np.allclose(sc.raw[1024], flat.raw[1024], atol=1e-9)
