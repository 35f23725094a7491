"""FP64 quality metrics (oracle; test infrastructure only).

* SQNR with optimal real-scale alignment (Section IV-B, Section VI): the test
  signal is scaled by the real alpha that minimises ||ref - alpha * test||,
  alpha = Re<test, ref> / ||test||^2, then SQNR = 10 log10(||ref||^2 /
  ||ref - alpha test||^2).  The unaligned figure uses alpha = 1.
* Point-target metrics (Section VI, Table III).  The paper names PSLR, ISLR,
  target SNR and 3 dB resolution but does not define windows; the reading
  used here:
    - peak: argmax |I| within +-4 cells of the target's nominal cell;
    - a 64 x 64 window around that peak is interpolated x16 by zero-padding
      its 2-D DFT; 1-D cuts through the interpolated maximum along range
      (axis 1) and azimuth (axis 0);
    - mainlobe: from the peak out to the first local minimum on each side;
    - PSLR = 20 log10(max sidelobe / peak), ISLR = 10 log10(sidelobe energy
      / mainlobe energy), both over the cut;
    - 3 dB width: distance between the half-power crossings (linear
      interpolation), in original cells;
    - SNR = 10 log10(|peak|^2 / mean |I|^2 over the noise region), the noise
      region being every cell at least 96 cells from every target in both
      range and azimuth.
"""

from __future__ import annotations

import numpy as np

from . import fft as _fft

SQNR_CAP_DB = 300.0


def sqnr_db(ref: np.ndarray, test: np.ndarray, align: bool = True) -> float:
    ref = np.asarray(ref, dtype=np.complex128).ravel()
    test = np.asarray(test, dtype=np.complex128).ravel()
    alpha = 1.0
    if align:
        tt = float(np.vdot(test, test).real)
        if tt > 0:
            alpha = float(np.vdot(test, ref).real) / tt
    err = float(np.sum(np.abs(ref - alpha * test) ** 2))
    sig = float(np.sum(np.abs(ref) ** 2))
    if err == 0.0:
        return SQNR_CAP_DB
    return min(SQNR_CAP_DB, 10.0 * np.log10(sig / err))


def rel_l2(ref: np.ndarray, test: np.ndarray) -> float:
    ref = np.asarray(ref, dtype=np.complex128).ravel()
    test = np.asarray(test, dtype=np.complex128).ravel()
    return float(np.linalg.norm(ref - test) / np.linalg.norm(ref))


def upsample2d(win: np.ndarray, factor: int) -> np.ndarray:
    """Band-limited interpolation of a square window by zero-padding its 2-D DFT."""
    w = win.shape[0]
    spec = _fft.fft_axis(_fft.fft_axis(win, 0), 1)
    big = w * factor
    pad = np.zeros((big, big), dtype=np.complex128)
    h = w // 2
    pad[:h, :h] = spec[:h, :h]
    pad[:h, big - h:] = spec[:h, h:]
    pad[big - h:, :h] = spec[h:, :h]
    pad[big - h:, big - h:] = spec[h:, h:]
    out = _fft.fft_axis(_fft.fft_axis(pad, 0, inverse=True), 1, inverse=True)
    return out * (factor * factor)


def cut_metrics(cut: np.ndarray, factor: int) -> dict:
    """PSLR / ISLR / 3 dB width of a 1-D interpolated magnitude cut."""
    mag = np.abs(np.asarray(cut))
    p = int(np.argmax(mag))
    lo = p
    while lo > 0 and mag[lo - 1] < mag[lo]:
        lo -= 1
    hi = p
    while hi < mag.shape[0] - 1 and mag[hi + 1] < mag[hi]:
        hi += 1
    peak = mag[p]
    side = np.concatenate((mag[:lo], mag[hi + 1:]))
    main = mag[lo:hi + 1]
    pslr = 20.0 * np.log10(np.max(side) / peak) if side.size else -np.inf
    islr = 10.0 * np.log10(np.sum(side ** 2) / np.sum(main ** 2)) if side.size else -np.inf
    pw = mag ** 2
    half = 0.5 * pw[p]
    i = p
    while i > lo and pw[i - 1] >= half:
        i -= 1
    left = i - (pw[i] - half) / (pw[i] - pw[i - 1]) if i > 0 and pw[i - 1] < half else float(i)
    j = p
    while j < hi and pw[j + 1] >= half:
        j += 1
    right = j + (pw[j] - half) / (pw[j] - pw[j + 1]) if j < mag.shape[0] - 1 and pw[j + 1] < half else float(j)
    return {"pslr_db": float(pslr), "islr_db": float(islr), "width_cells": float((right - left) / factor)}


def noise_mask(shape, targets, guard: int = 96) -> np.ndarray:
    n_az, n_rg = shape
    keep_a = np.ones(n_az, dtype=bool)
    keep_r = np.ones(n_rg, dtype=bool)
    for eta, r, _ in targets:
        keep_a[max(0, eta - guard + 1):eta + guard] = False
        keep_r[max(0, r - guard + 1):r + guard] = False
    return np.outer(keep_a, keep_r)


def point_target_metrics(img: np.ndarray, targets, window: int = 64, factor: int = 16,
                         search: int = 4, guard: int = 96) -> list:
    """Per-target PSLR / ISLR / 3 dB widths / SNR of an image [n_az][n_rg]."""
    img = np.asarray(img, dtype=np.complex128)
    n_az, n_rg = img.shape
    mask = noise_mask(img.shape, targets, guard)
    noise_power = float(np.mean(np.abs(img[mask]) ** 2)) if mask.any() else float("nan")
    out = []
    for eta, r, amp in targets:
        rows = np.arange(eta - search, eta + search + 1) % n_az
        cols = np.arange(r - search, r + search + 1) % n_rg
        sub = np.abs(img[np.ix_(rows, cols)])
        ia, ir = np.unravel_index(int(np.argmax(sub)), sub.shape)
        pa, pr = int(rows[ia]), int(cols[ir])
        h = window // 2
        wr = np.arange(pa - h, pa + h) % n_az
        wc = np.arange(pr - h, pr + h) % n_rg
        up = upsample2d(img[np.ix_(wr, wc)], factor)
        ua, ur = np.unravel_index(int(np.argmax(np.abs(up))), up.shape)
        rng_cut = cut_metrics(up[ua, :], factor)
        az_cut = cut_metrics(up[:, ur], factor)
        peak = float(np.abs(up[ua, ur]))
        out.append({
            "eta": int(eta), "r": int(r), "amplitude": float(amp),
            "peak_cell": (pa, pr), "peak": peak,
            "pslr_range_db": rng_cut["pslr_db"], "pslr_azimuth_db": az_cut["pslr_db"],
            "pslr_db": max(rng_cut["pslr_db"], az_cut["pslr_db"]),
            "islr_range_db": rng_cut["islr_db"], "islr_azimuth_db": az_cut["islr_db"],
            "width_range_cells": rng_cut["width_cells"],
            "width_azimuth_cells": az_cut["width_cells"],
            "snr_db": 10.0 * np.log10(peak * peak / noise_power),
        })
    return out
