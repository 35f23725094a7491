"""FP64 range-Doppler SAR compression (oracle; test infrastructure only).

Matched-filter compression (Section III-B):  y = IDFT(DFT(x) . H), with the
normalised inverse of ``oracle.fft``.  Range compression applies it to every
azimuth line (last axis), azimuth compression to every range column of the
range-compressed data (first axis), as in Fig. 1.

Filters (a reading of Section III-B, which allows both |H| <= 1 and an
unnormalised filter):

* range:   Hr = conj(DFT(ref_r))                          (unnormalised)
* azimuth: Ha = conj(DFT(ref_a)) / max_k |DFT(ref_a)[k]|  (|Ha| <= 1)

where ref is the transmitted chirp placed circularly centred at index 0, so a
compressed target lands on its centre cell.

``stage_maxima`` reports the largest magnitude at every storage point of the
pipeline in FP64, once with the fixed 1/N block shift of Eq. 1 and once
without it (the naive schedule of Section III-B whose unnormalised inverse
reaches O(N^2) before the final 1/N).
"""

from __future__ import annotations

import numpy as np

from . import fft as _fft


def matched_filter(ref: np.ndarray, peak_normalise: bool) -> np.ndarray:
    """conj(DFT(ref)), optionally divided by its largest magnitude."""
    h = np.conj(_fft.fft(np.asarray(ref, dtype=np.complex128)))
    if peak_normalise:
        h = h / np.max(np.abs(h))
    return h


def compress(x: np.ndarray, h: np.ndarray, axis: int) -> np.ndarray:
    """IDFT(DFT(x) . H) along ``axis``; H broadcasts along that axis."""
    x = np.moveaxis(np.asarray(x, dtype=np.complex128), axis, -1)
    y = _fft.ifft(_fft.fft(x) * np.asarray(h, dtype=np.complex128))
    return np.moveaxis(y, -1, axis)


def range_compress(raw: np.ndarray, hr: np.ndarray) -> np.ndarray:
    """Per azimuth line: IDFT(DFT(raw[eta, :]) . Hr).  raw is [n_az][n_rg]."""
    return compress(raw, hr, axis=-1)


def azimuth_compress(rc: np.ndarray, ha: np.ndarray) -> np.ndarray:
    """Per range column: IDFT(DFT(rc[:, r]) . Ha).  rc is [n_az][n_rg]."""
    return compress(rc, ha, axis=0)


def range_doppler_image(raw: np.ndarray, hr: np.ndarray, ha: np.ndarray) -> np.ndarray:
    return azimuth_compress(range_compress(raw, hr), ha)


def stage_maxima(x: np.ndarray, h: np.ndarray, axis: int = -1) -> dict:
    """Largest |.| at each storage point of one compression, with and without the shift.

    Returns a dict with keys
      'spectrum'      max |DFT(x)|                               (both schedules)
      'product'       max |DFT(x) . H|                           (both schedules)
      'bfp_pre'       max |conj(DFT(x) . H) / N|    input of the shifted inverse
      'bfp_out'       max |y|                       shifted inverse output
      'naive_out'     max |N y|                     unshifted inverse output
    """
    xm = np.moveaxis(np.asarray(x, dtype=np.complex128), axis, -1)
    n = xm.shape[-1]
    spec = _fft.fft(xm)
    prod = spec * h
    y = _fft.ifft(prod)
    return {
        "spectrum": float(np.max(np.abs(spec))),
        "product": float(np.max(np.abs(prod))),
        "bfp_pre": float(np.max(np.abs(prod))) / n,
        "bfp_out": float(np.max(np.abs(y))),
        "naive_out": float(np.max(np.abs(_fft.ifft_unnormalised(prod)))),
    }
