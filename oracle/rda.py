"""Range-Doppler processing with range-cell migration correction, in FP64 (oracle; test infrastructure only).

Section VI names range-cell-migration correction (RCMC) as a stage of the
paper's range-Doppler pipeline and leaves it in FP32; the migration-free
scene of ``oracle.sar`` does not need it.  For a scene with the hyperbolic
range history R(t) = sqrt(R^2 + v^2 t^2), the textbook range-Doppler
algorithm is, in the order it runs:

1. range compression per azimuth line (``oracle.sar.range_compress``);
2. azimuth DFT per range column, into the range-Doppler domain;
3. RCMC: at Doppler frequency f a target sits at range R + dR(f), with
       dR(f) = R (1 / D(f) - 1),   D(f) = sqrt(1 - (lambda f / (2 v))^2)
   (stationary phase on the hyperbolic history); each Doppler row is moved
   back by dR(f) / range_cell cells;
4. azimuth matched filter per range column, built from that column's FM
   rate Ka(R) = 2 v^2 / (lambda R), then the inverse azimuth DFT.

Readings:
* RCMC is the bulk correction: dR(f) is evaluated at the scene-centre range
  R0 for every column, and the shift is the exact band-limited one (a
  linear phase across the row's range DFT).  The range dependence of dR is
  (R - R0) / R0 of the migration, under 0.04 cells across the 1024-cell
  swaths used here, and is neglected.
* The azimuth filter of column r is conj(DFT(ref_r)) with ref_r the chirp
  exp(-j pi k_a(R_r) n^2), n in [-L_a/2, L_a/2), k_a(R) = Ka(R) / PRF^2,
  circularly centred at index 0; unnormalised, or divided by its largest
  magnitude as in ``oracle.sar``.  Unlike the migration-free path, k_a
  changes with range: across a 1.3 km swath at 20 km it moves by 3 %, which
  is tens of radians of phase at the aperture's edge.
"""

from __future__ import annotations

import numpy as np

from . import fft as _fft
from . import sar as _sar


def doppler_frequencies(n_az: int, prf_hz: float) -> np.ndarray:
    """Signed frequency (Hz) of each azimuth DFT bin: k / n_az * PRF, k folded into [-n_az/2, n_az/2)."""
    k = np.arange(n_az)
    k = np.where(k >= n_az // 2, k - n_az, k)
    return k * prf_hz / n_az


def migration_m(f_hz: np.ndarray, range_m, wavelength_m: float, speed_mps: float) -> np.ndarray:
    """dR(f) = R (1 / sqrt(1 - (lambda f / (2 v))^2) - 1)."""
    d = np.sqrt(1.0 - (wavelength_m * np.asarray(f_hz) / (2.0 * speed_mps)) ** 2)
    return np.asarray(range_m) * (1.0 / d - 1.0)


def shift_rows(x: np.ndarray, cells: np.ndarray) -> np.ndarray:
    """Band-limited circular shift of each row by cells[i] (positive: towards larger index).

    y(r) = x(r - s): the row's DFT times exp(-2 pi i q s / N) with q the signed
    frequency index; the Nyquist bin takes cos(pi s), the even part of its
    two signed forms, so that a real row stays real.
    """
    x = np.asarray(x, dtype=np.complex128)
    n = x.shape[-1]
    q = np.arange(n)
    q = np.where(q > n // 2, q - n, q).astype(np.float64)
    s = np.asarray(cells, dtype=np.float64)[:, None]
    ramp = np.exp(-2j * np.pi * q[None, :] * s / n)
    if n % 2 == 0:
        ramp[:, n // 2] = np.cos(np.pi * s[:, 0])
    return _fft.ifft(_fft.fft(x) * ramp)


def range_doppler(rc: np.ndarray) -> np.ndarray:
    """Azimuth DFT of each range column: [n_az][n_rg] -> [Doppler][n_rg]."""
    return _fft.fft_axis(rc, axis=0)


def rcmc(s_rd: np.ndarray, geo, n_rg: int) -> np.ndarray:
    """Bulk RCMC: every Doppler row moved back by dR(f, R0) / range_cell cells."""
    f = doppler_frequencies(s_rd.shape[0], geo.prf_hz)
    cells = migration_m(f, geo.centre_range_m, geo.wavelength_m, geo.speed_mps) / geo.range_cell_m
    return shift_rows(s_rd, -cells)


def azimuth_rate(range_m, geo) -> np.ndarray:
    """k_a(R) = 2 v^2 / (lambda R PRF^2), cycles per pulse^2."""
    return 2.0 * geo.speed_mps ** 2 / (geo.wavelength_m * np.asarray(range_m) * geo.prf_hz ** 2)


def azimuth_filters(n_az: int, n_rg: int, aperture: int, geo, peak_normalise: bool,
                    range_dependent: bool = True) -> np.ndarray:
    """[n_az][n_rg]: column r holds conj(DFT(ref_r)), ref_r the centred chirp of rate k_a(R_r)."""
    r_m = geo.centre_range_m + (np.arange(n_rg) - n_rg / 2) * geo.range_cell_m   # cell n_rg / 2 at R0
    if not range_dependent:
        r_m = np.full(n_rg, geo.centre_range_m)
    ka = azimuth_rate(r_m, geo)
    n = np.arange(aperture) - aperture / 2
    idx = (np.arange(aperture) - aperture // 2) % n_az
    refs = np.zeros((n_rg, n_az), dtype=np.complex128)
    refs[:, idx] = np.exp(-1j * np.pi * ka[:, None] * n[None, :] ** 2)
    h = np.conj(_fft.fft(refs))                       # [n_rg][n_az]
    if peak_normalise:
        h = h / np.max(np.abs(h), axis=1, keepdims=True)
    return h.T


def image(raw: np.ndarray, hr: np.ndarray, geo, aperture: int, correct_migration: bool = True,
          range_dependent: bool = True, peak_normalise: bool = False) -> np.ndarray:
    """Range compression, azimuth DFT, RCMC, per-column azimuth filter, inverse azimuth DFT."""
    n_az, n_rg = raw.shape
    s_rd = range_doppler(_sar.range_compress(raw, hr))
    if correct_migration:
        s_rd = rcmc(s_rd, geo, n_rg)
    ha = azimuth_filters(n_az, n_rg, aperture, geo, peak_normalise, range_dependent)
    return _fft.fft_axis(s_rd * ha, axis=0, inverse=True)
