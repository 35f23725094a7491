"""Circular convolution and correlation, in FP64 (oracle; test infrastructure only).

Section VIII (Generality) applies the fixed 1/N shift to any
forward-multiply-inverse pipeline with known growth: convolution,
correlation and spectral layers, not only matched filtering.  The oracle
states the two classic ones by their defining sums, over the last axis with
indices mod N:

    convolution   (x * g)[n]  = sum_m x[m] g[(n - m) mod N]
    correlation   (x ** g)[n] = sum_m x[(m + n) mod N] conj(g[m])

and the pipeline that computes them, y = IDFT(DFT(x) . H), with
H = DFT(g) for the convolution and H = conj(DFT(g)) for the correlation
(the matched filter of ``oracle.sar`` is the correlation with the pulse).

The defining sums are evaluated directly, O(N^2) per line, for checking;
``spectral`` is the pipeline in FP64.
"""

from __future__ import annotations

import numpy as np

from . import fft as _fft


def _lag_matrix(n: int) -> np.ndarray:
    """L[n, m] = (n - m) mod N."""
    idx = np.arange(n)
    return (idx[:, None] - idx[None, :]) % n


def convolve_direct(x: np.ndarray, g: np.ndarray) -> np.ndarray:
    """sum_m x[m] g[(n - m) mod N] along the last axis (g broadcasts over leading axes)."""
    x = np.asarray(x, dtype=np.complex128)
    g = np.asarray(g, dtype=np.complex128)
    n = x.shape[-1]
    gm = g[..., _lag_matrix(n)]                       # gm[..., n, m] = g[(n - m) mod N]
    return np.einsum("...m,...nm->...n", x, gm)


def correlate_direct(x: np.ndarray, g: np.ndarray) -> np.ndarray:
    """sum_m x[(m + n) mod N] conj(g[m]) along the last axis."""
    x = np.asarray(x, dtype=np.complex128)
    g = np.asarray(g, dtype=np.complex128)
    n = x.shape[-1]
    idx = np.arange(n)
    xm = x[..., (idx[:, None] + idx[None, :]) % n]   # xm[..., n, m] = x[(m + n) mod N]
    return np.einsum("...nm,...m->...n", xm, np.conj(g))


def spectral(x: np.ndarray, h: np.ndarray) -> np.ndarray:
    """IDFT(DFT(x) . H) along the last axis: the forward-multiply-inverse pipeline."""
    return _fft.ifft(_fft.fft(x) * np.asarray(h, dtype=np.complex128))


def convolution_filter(g: np.ndarray) -> np.ndarray:
    """H with spectral(x, H) = x * g."""
    return _fft.fft(g)


def correlation_filter(g: np.ndarray) -> np.ndarray:
    """H with spectral(x, H) = x ** g."""
    return np.conj(_fft.fft(g))
