"""Seeded synthetic inputs shared by the CUDA path, its tests and the FP64 oracle.

This module holds no arithmetic of the method itself (no transform, no filter
spectrum, no block shift, no metric).  It only draws the numbers that both
sides receive, so that each side can compute its own answer from identical
inputs.  Every generator is deterministic given its seed.

Workload shapes follow the paper's experiments:

* Section V (Table II): batched complex transforms of length 4096, batch 256,
  with re, im ~ N(0, 1).
* Section VI: a point-target SAR scene (X band, B = 100 MHz, v = 100 m/s,
  R0 = 20 km, 20 dB additive noise).  The paper leaves the sample rate,
  pulse length, aperture length and target layout open; the completion used
  here is: fs = 120 MHz, time-bandwidth product 400 (Tp = 4 us, M = 480
  samples, K = B / Tp), an azimuth chirp of L_a = 1024 pulses with a Doppler
  bandwidth of 0.8 PRF (normalised rate k_a = 0.8 / L_a), 8 targets with
  amplitudes 10^(-k/7), and complex AWGN of variance 0.01 (20 dB below the
  unit-amplitude target per sample).  Range-cell migration is neglected in
  point_target_scene; migrating_scene adds it (wavelength 0.03 m, exact
  hyperbolic range history) for the range-cell-migration correction.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Scene constants (Section VI completion, see module docstring).
RANGE_BANDWIDTH_HZ = 100e6
RANGE_SAMPLE_RATE_HZ = 120e6
RANGE_TBP = 400
AZIMUTH_APERTURE = 1024
AZIMUTH_DOPPLER_FRACTION = 0.8
NOISE_VARIANCE = 0.01
N_TARGETS = 8
MIN_TARGET_SEPARATION = 128

# Geometry of the scene with range-cell migration (Section VI gives X band,
# v = 100 m/s and R0 = 20 km; the completion adds a wavelength of 0.03 m and
# a PRF chosen so that the azimuth FM rate at R0 gives the same normalised
# rate k_a = 0.8 / L_a as the migration-free scene).
WAVELENGTH_M = 0.03
PLATFORM_SPEED_MPS = 100.0
SCENE_CENTRE_RANGE_M = 20e3
SPEED_OF_LIGHT_MPS = 299792458.0

# Uneven-batch lengths (mixed-length workload, Zipf-like weights).
UNEVEN_LENGTHS = (256, 1024, 4096, 16384, 65536)
UNEVEN_ZIPF_EXPONENT = 0.5


def complex_gaussian(batch: int, n: int, seed: int = 0) -> np.ndarray:
    """[batch][n] complex128 with re, im ~ N(0, 1) i.i.d. (Table II workload)."""
    rng = np.random.default_rng(seed)
    re = rng.standard_normal((batch, n))
    im = rng.standard_normal((batch, n))
    return re + 1j * im


def range_chirp_params():
    """(M, K, fs): pulse samples, FM rate (Hz/s), sample rate for the range chirp."""
    tp = RANGE_TBP / RANGE_BANDWIDTH_HZ
    m = int(round(tp * RANGE_SAMPLE_RATE_HZ))
    k = RANGE_BANDWIDTH_HZ / tp
    return m, k, RANGE_SAMPLE_RATE_HZ


def range_chirp() -> np.ndarray:
    """Unit-modulus LFM pulse s_r[m] = exp(j pi K t_m^2), t_m = (m - M/2) / fs."""
    m, k, fs = range_chirp_params()
    t = (np.arange(m) - m / 2) / fs
    return np.exp(1j * np.pi * k * t * t)


def azimuth_chirp(aperture: int = AZIMUTH_APERTURE,
                  doppler_fraction: float = AZIMUTH_DOPPLER_FRACTION) -> np.ndarray:
    """Unit-modulus azimuth chirp s_a[n] = exp(-j pi k_a n'^2), n' = n - L_a/2.

    k_a = doppler_fraction / L_a (cycles per pulse^2 with PRF normalised to 1),
    so the chirp sweeps doppler_fraction * PRF over the aperture.
    """
    ka = doppler_fraction / aperture
    n = np.arange(aperture) - aperture / 2
    return np.exp(-1j * np.pi * ka * n * n)


def centred_reference(pulse: np.ndarray, n: int) -> np.ndarray:
    """Place a length-M pulse circularly centred at index 0 of a length-n line.

    Sample m goes to index (m - M/2) mod n, so that a matched filter built from
    this line puts each compressed target at its centre index.
    """
    m = pulse.shape[0]
    out = np.zeros(n, dtype=np.complex128)
    idx = (np.arange(m) - m // 2) % n
    out[idx] = pulse
    return out


@dataclass
class Scene:
    raw: np.ndarray               # [n_az][n_rg] complex128 echo
    ref_range: np.ndarray         # [n_rg] complex128, range pulse centred at 0
    ref_azimuth: np.ndarray       # [n_az] complex128, azimuth chirp centred at 0
    targets: list = field(default_factory=list)   # (eta, r, amplitude)
    noise_variance: float = NOISE_VARIANCE


def target_layout(n_az: int, n_rg: int, aperture: int, seed: int = 1,
                  count: int = N_TARGETS):
    """Integer target positions (eta, r) and amplitudes a_k = 10^(-k/7).

    Range positions are drawn from [256, n_rg - 256].  Azimuth positions are
    drawn from [L_a/2 + 64, n_az - L_a/2 - 64] when the scene is long enough
    to hold a whole aperture around each target, else from [64, n_az - 64]
    (apertures clipped at the scene edge).  Any two targets are at least
    MIN_TARGET_SEPARATION cells apart in range or in azimuth; a draw that
    breaks this is redrawn.
    """
    rng = np.random.default_rng(seed)
    lo_a, hi_a = aperture // 2 + 64, n_az - aperture // 2 - 64
    if hi_a <= lo_a:
        lo_a, hi_a = 64, n_az - 64
    lo_r, hi_r = 256, n_rg - 256
    pos = []
    while len(pos) < count:
        eta = int(rng.integers(lo_a, hi_a + 1))
        r = int(rng.integers(lo_r, hi_r + 1))
        ok = all(abs(eta - e) >= MIN_TARGET_SEPARATION or abs(r - q) >= MIN_TARGET_SEPARATION
                 for e, q in pos)
        if ok:
            pos.append((eta, r))
    return [(eta, r, 10.0 ** (-k / 7.0)) for k, (eta, r) in enumerate(pos)]


def point_target_scene(n_az: int, n_rg: int, aperture: int = AZIMUTH_APERTURE,
                       noise: bool = True, targets=None, target_seed: int = 1,
                       noise_seed: int = 2) -> Scene:
    """Raw echo raw[eta][r] = sum_k a_k s_r[r - r_k + M/2] s_a[eta - eta_k + L_a/2] + noise.

    Each echo is zero outside its pulse and aperture support.  Noise is complex
    AWGN of total variance NOISE_VARIANCE split equally between re and im.
    """
    sr = range_chirp()
    sa = azimuth_chirp(aperture)
    m = sr.shape[0]
    if targets is None:
        targets = target_layout(n_az, n_rg, aperture, seed=target_seed)
    raw = np.zeros((n_az, n_rg), dtype=np.complex128)
    for eta, r, a in targets:
        r0 = r - m // 2
        e0 = eta - aperture // 2
        rs, re_ = max(r0, 0), min(r0 + m, n_rg)
        es, ee = max(e0, 0), min(e0 + aperture, n_az)
        raw[es:ee, rs:re_] += a * np.outer(sa[es - e0:ee - e0], sr[rs - r0:re_ - r0])
    if noise:
        rng = np.random.default_rng(noise_seed)
        s = math.sqrt(NOISE_VARIANCE / 2.0)
        raw += s * rng.standard_normal((n_az, n_rg))
        raw += 1j * s * rng.standard_normal((n_az, n_rg))
    return Scene(raw=raw,
                 ref_range=centred_reference(sr, n_rg),
                 ref_azimuth=centred_reference(sa[: min(aperture, n_az)], n_az),
                 targets=list(targets))


@dataclass
class Geometry:
    range_cell_m: float           # slant-range sample spacing c / (2 fs)
    prf_hz: float                 # pulse repetition frequency
    wavelength_m: float
    speed_mps: float
    centre_range_m: float         # slant range of range cell n_rg / 2


def radar_geometry(aperture: int = AZIMUTH_APERTURE,
                   doppler_fraction: float = AZIMUTH_DOPPLER_FRACTION) -> Geometry:
    """Scene geometry: the PRF makes Ka(R0) / PRF^2 = doppler_fraction / aperture,
    with Ka(R) = 2 v^2 / (lambda R) the azimuth FM rate in Hz/s."""
    ka_hz = 2.0 * PLATFORM_SPEED_MPS ** 2 / (WAVELENGTH_M * SCENE_CENTRE_RANGE_M)
    prf = math.sqrt(ka_hz * aperture / doppler_fraction)
    return Geometry(range_cell_m=SPEED_OF_LIGHT_MPS / (2.0 * RANGE_SAMPLE_RATE_HZ), prf_hz=prf,
                    wavelength_m=WAVELENGTH_M, speed_mps=PLATFORM_SPEED_MPS,
                    centre_range_m=SCENE_CENTRE_RANGE_M)


def slant_range_m(r_cell, n_rg: int, geo: Geometry):
    """Slant range of range cell r (cell n_rg / 2 is at the scene-centre range)."""
    return geo.centre_range_m + (np.asarray(r_cell, dtype=np.float64) - n_rg / 2) * geo.range_cell_m


def migrating_scene(n_az: int, n_rg: int, targets, aperture: int = AZIMUTH_APERTURE,
                    noise: bool = False, noise_seed: int = 2) -> Scene:
    """Raw echo with range-cell migration and the exact hyperbolic range history.

    Target (eta_k, r_k, a_k) at slant range R_k = slant_range_m(r_k) is seen
    over the pulses |eta - eta_k| < L_a / 2 at range
        R_k(eta) = sqrt(R_k^2 + (v (eta - eta_k) / PRF)^2),
    so its echo is
        a_k chirp((r - r_k - d) / fs) exp(-j 4 pi (R_k(eta) - R_k) / lambda),
        d = (R_k(eta) - R_k) / range_cell,
    with chirp(tau) = exp(j pi K tau^2) for -Tp/2 <= tau < Tp/2 (the pulse of
    range_chirp, evaluated at the delayed sample times).  With d = 0 and the
    phase expanded to second order this is point_target_scene's echo.
    Noise, when asked for, is as in point_target_scene.
    """
    m, k, fs = range_chirp_params()
    geo = radar_geometry(aperture)
    tp = m / fs
    raw = np.zeros((n_az, n_rg), dtype=np.complex128)
    rr = np.arange(n_rg)
    for eta, r, a in targets:
        r_k = float(slant_range_m(r, n_rg, geo))
        for e in range(max(eta - aperture // 2, 0), min(eta - aperture // 2 + aperture, n_az)):
            t = (e - eta) / geo.prf_hz
            r_e = math.sqrt(r_k * r_k + (geo.speed_mps * t) ** 2)
            d = (r_e - r_k) / geo.range_cell_m
            tau = (rr - r - d) / fs
            inside = (tau >= -tp / 2) & (tau < tp / 2)
            phase = np.pi * k * tau * tau - 4.0 * np.pi * (r_e - r_k) / geo.wavelength_m
            raw[e] += np.where(inside, a * np.exp(1j * phase), 0.0)
    if noise:
        rng = np.random.default_rng(noise_seed)
        s = math.sqrt(NOISE_VARIANCE / 2.0)
        raw += s * rng.standard_normal((n_az, n_rg))
        raw += 1j * s * rng.standard_normal((n_az, n_rg))
    return Scene(raw=raw, ref_range=centred_reference(range_chirp(), n_rg),
                 ref_azimuth=centred_reference(azimuth_chirp(aperture)[: min(aperture, n_az)], n_az),
                 targets=list(targets))


def phase_error(n_az: int, seed: int = 5, quad_rad: float = 4 * math.pi,
                noise_rad: float = 0.3) -> np.ndarray:
    """Per-pulse phase error: quad_rad * (2n/n_az - 1)^2 + N(0, noise_rad^2)."""
    rng = np.random.default_rng(seed)
    u = 2.0 * np.arange(n_az) / n_az - 1.0
    return quad_rad * u * u + noise_rad * rng.standard_normal(n_az)


def uneven_lengths(count: int = 20000, seed: int = 3,
                   lengths=UNEVEN_LENGTHS, exponent: float = UNEVEN_ZIPF_EXPONENT) -> np.ndarray:
    """Transform lengths drawn with P(lengths[i]) proportional to (i + 1)^-exponent."""
    rng = np.random.default_rng(seed)
    w = np.array([(i + 1.0) ** -exponent for i in range(len(lengths))])
    w /= w.sum()
    return np.asarray(lengths, dtype=np.int64)[rng.choice(len(lengths), size=count, p=w)]


def uneven_batch(lengths: np.ndarray, seed: int = 30):
    """Pack transforms of the given lengths contiguously; returns (data, offsets).

    data is complex128 of total length sum(lengths) with re, im ~ N(0, 1);
    offsets[i] is the first point of transform i.
    """
    lengths = np.asarray(lengths, dtype=np.int64)
    offsets = np.zeros(lengths.shape[0], dtype=np.int64)
    if lengths.shape[0] > 1:
        offsets[1:] = np.cumsum(lengths)[:-1]
    total = int(lengths.sum())
    rng = np.random.default_rng(seed)
    data = rng.standard_normal(total) + 1j * rng.standard_normal(total)
    return data, offsets


def range_compressed_scene(n_az: int, n_rg: int, aperture: int, targets, noise_std: float = 0.05,
                           seed: int = 2) -> np.ndarray:
    """Ideally range-compressed echoes [n_az][n_rg]: target (eta, r, a) puts
    a * s_a[eta' - eta + L_a/2] into range bin r over its aperture, plus complex
    AWGN of standard deviation noise_std per component."""
    sa = azimuth_chirp(aperture)
    rc = np.zeros((n_az, n_rg), dtype=np.complex128)
    for eta, r, a in targets:
        e0 = eta - aperture // 2
        es, ee = max(e0, 0), min(e0 + aperture, n_az)
        rc[es:ee, r] += a * sa[es - e0:ee - e0]
    rng = np.random.default_rng(seed)
    rc += noise_std * (rng.standard_normal((n_az, n_rg)) + 1j * rng.standard_normal((n_az, n_rg)))
    return rc
