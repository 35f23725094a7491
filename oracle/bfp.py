"""Adaptive per-block exponents, in FP64 (oracle; test infrastructure only).

The paper's block schedule is fixed: one 1/N shift per transform, because
the growth of a matched filter is known (Section IV-A, Eq. 1).  Its
limitations paragraph (Section VIII) names the alternative: an exponent per
block, found by a reduction over the block, that keeps pathological inputs
in range.  Reading (nothing more is specified):

* a block is one transform line (the last axis);
* its exponent e is the smallest integer with m 2^-e <= limit, where m is
  the largest |real| or |imaginary| component in the block; an all-zero
  block takes e = 0;
* the stored block is round(v 2^-e) in the storage format, with e beside
  it; its value is mantissa * 2^e;
* limit defaults to 2^14: the stored components stay within (2^13, 2^14],
  leaving a factor of four below FP16's 65504 for the growth of one
  radix-2 stage and the rounding that follows it.

``adaptive_spectral`` applies it at the one storage point of a
forward-multiply-inverse line: y = IDFT(DFT(x) . H) in FP64, then one
exponent per line.  A scene of any amplitude then stores without overflow,
and its mantissas do not depend on the amplitude's power-of-two part.
"""

from __future__ import annotations

import numpy as np

from . import conv as _conv
from . import quant as _quant

DEFAULT_LIMIT = 2.0 ** 14


def block_max(v: np.ndarray) -> np.ndarray:
    """Largest |real| or |imaginary| component of each block (last axis)."""
    v = np.asarray(v, dtype=np.complex128)
    return np.maximum(np.abs(v.real), np.abs(v.imag)).max(axis=-1)


def block_exponent(v: np.ndarray, limit: float = DEFAULT_LIMIT) -> np.ndarray:
    """Smallest integer e per block with block_max(v) 2^-e <= limit (0 for a zero block)."""
    m = block_max(v)
    e = np.zeros(m.shape, dtype=np.int64)
    nz = m > 0
    # ceil(log2(m / limit)), corrected so that the inequality holds exactly
    est = np.ceil(np.log2(m[nz] / limit)).astype(np.int64)
    est = np.where(np.ldexp(m[nz], -est) > limit, est + 1, est)
    est = np.where(np.ldexp(m[nz], -(est - 1)) <= limit, est - 1, est)
    e[nz] = est
    return e


def quantize(v: np.ndarray, limit: float = DEFAULT_LIMIT, round_fn=_quant.round_binary16):
    """(mantissas, exponents): round(v 2^-e) per block, and e per block."""
    v = np.asarray(v, dtype=np.complex128)
    e = block_exponent(v, limit)
    scaled = np.ldexp(v.real, -e[..., None]) + 1j * np.ldexp(v.imag, -e[..., None])
    return round_fn(scaled), e


def value(mantissas: np.ndarray, exponents: np.ndarray) -> np.ndarray:
    """The values a block-floating-point array represents: mantissa * 2^e."""
    m = np.asarray(mantissas, dtype=np.complex128)
    e = np.asarray(exponents)[..., None]
    return np.ldexp(m.real, e) + 1j * np.ldexp(m.imag, e)


def adaptive_spectral(x: np.ndarray, h: np.ndarray, limit: float = DEFAULT_LIMIT,
                      round_fn=_quant.round_binary16):
    """IDFT(DFT(x) . H) per line, stored with one adaptive exponent per line."""
    return quantize(_conv.spectral(x, h), limit, round_fn)
