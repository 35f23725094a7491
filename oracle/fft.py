"""FP64 discrete Fourier transforms (oracle; test infrastructure only).

Definitions (Section III-B of the paper, and the standard DFT):

    forward   X[k] = sum_{n<N} x[n] exp(-2 pi i n k / N)          (unnormalised)
    inverse   x[n] = (1/N) sum_{k<N} X[k] exp(+2 pi i n k / N)     (normalised)

The paper realises the inverse as conj(FFT(conj z)) / N and moves the 1/N in
front of the transform (Eq. 1); both are identities of the definition above,
so the oracle computes the definition itself and the tests check the
identities against it.

``fft`` is a plain iterative radix-2 decimation-in-time FFT (bit-reversal
permutation, then log2 N butterfly stages), vectorised over leading axes.
``dft_bruteforce`` evaluates the defining sum as a matrix product, for
checking ``fft`` on small N.
"""

from __future__ import annotations

import numpy as np


def _check_pow2(n: int) -> int:
    if n < 1 or (n & (n - 1)) != 0:
        raise ValueError(f"length {n} is not a power of two")
    return n.bit_length() - 1


def _bit_reverse_indices(n: int) -> np.ndarray:
    bits = _check_pow2(n)
    idx = np.arange(n)
    rev = np.zeros(n, dtype=np.int64)
    for b in range(bits):
        rev |= ((idx >> b) & 1) << (bits - 1 - b)
    return rev


def _radix2(x: np.ndarray, sign: int) -> np.ndarray:
    """Unnormalised sum_n x[n] exp(sign * 2 pi i n k / N) along the last axis."""
    x = np.asarray(x, dtype=np.complex128)
    n = x.shape[-1]
    lead = x.shape[:-1]
    a = x[..., _bit_reverse_indices(n)].copy()
    half = 1
    while half < n:
        # Blocks of length 2*half: first half holds the transform of the even
        # samples, second half that of the odd samples (after bit reversal).
        w = np.exp(sign * 2j * np.pi * np.arange(half) / (2 * half))
        blocks = a.reshape(lead + (n // (2 * half), 2, half))
        even = blocks[..., 0, :]
        odd = blocks[..., 1, :] * w
        a = np.stack((even + odd, even - odd), axis=-2).reshape(lead + (n,))
        half *= 2
    return a


def fft(x: np.ndarray) -> np.ndarray:
    """Forward unnormalised DFT along the last axis."""
    return _radix2(x, -1)


def ifft(x: np.ndarray) -> np.ndarray:
    """Normalised inverse DFT along the last axis: (1/N) sum_k X[k] e^{+2 pi i nk/N}."""
    n = np.asarray(x).shape[-1]
    return _radix2(x, +1) / n


def ifft_unnormalised(x: np.ndarray) -> np.ndarray:
    """Inverse DFT without the 1/N (the quantity that overflows FP16, Section III-B)."""
    return _radix2(x, +1)


def dft_bruteforce(x: np.ndarray, sign: int = -1) -> np.ndarray:
    """O(N^2) evaluation of sum_n x[n] exp(sign 2 pi i n k / N) along the last axis."""
    x = np.asarray(x, dtype=np.complex128)
    n = x.shape[-1]
    nk = np.outer(np.arange(n), np.arange(n)) % n       # exact integer phase index
    mat = np.exp(sign * 2j * np.pi * nk / n)
    return x @ mat


def fft_axis(x: np.ndarray, axis: int, inverse: bool = False) -> np.ndarray:
    """Forward (or normalised inverse) DFT along a chosen axis."""
    moved = np.moveaxis(np.asarray(x, dtype=np.complex128), axis, -1)
    out = ifft(moved) if inverse else fft(moved)
    return np.moveaxis(out, -1, axis)
