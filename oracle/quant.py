"""Storage-format rounding, written from the formats' definitions (oracle).

TEST INFRASTRUCTURE ONLY.

* binary16 (IEEE 754 half): 1 sign, 5 exponent (bias 15), 10 fraction bits;
  largest finite 65504; values at or beyond 65520 round to infinity.
* OCP FP8 E4M3: 1 sign, 4 exponent (bias 7), 3 mantissa bits; no infinity,
  largest finite 448, smallest subnormal 2^-9.
* OCP FP8 E5M2: 1 sign, 5 exponent (bias 15), 2 mantissa bits; largest finite
  57344, smallest subnormal 2^-16.
* bfloat16: 1 sign, 8 exponent (bias 127), 7 fraction bits; the range of
  binary32 with 8 significant bits (Section IV-C compares it with FP16:
  range traded for mantissa).  Largest finite (2 - 2^-7) 2^127; values at or
  beyond (2 - 2^-8) 2^127 round to infinity, as in binary16.

All conversions round to nearest, ties to even.  The FP8 conversions are
"satfinite": a finite value beyond the largest finite magnitude becomes that
magnitude with its sign, and NaN stays NaN (Section VII: FP8 storage, FP32
or wider compute).

``round_binary16`` uses numpy's float16 cast, which is IEEE round-to-nearest-
even; the tests pin it against hand-checked edge values (65504, 65519.99,
65520, subnormals, ties).  The FP8 and bfloat16 rounders are written out
from the definition: pick the binade of |x| (never below the smallest normal
binade), round |x| / quantum to the nearest even integer, scale back, then
clamp (FP8) or overflow to infinity (bfloat16).
"""

from __future__ import annotations

import numpy as np


def round_binary16(x: np.ndarray) -> np.ndarray:
    """Round real or complex values to binary16 and return them as float64/complex128."""
    x = np.asarray(x)
    with np.errstate(over="ignore"):
        if np.iscomplexobj(x):
            return (x.real.astype(np.float16).astype(np.float64)
                    + 1j * x.imag.astype(np.float16).astype(np.float64))
        return x.astype(np.float16).astype(np.float64)


def round_binary32(x: np.ndarray) -> np.ndarray:
    x = np.asarray(x)
    if np.iscomplexobj(x):
        return (x.real.astype(np.float32).astype(np.float64)
                + 1j * x.imag.astype(np.float32).astype(np.float64))
    return x.astype(np.float32).astype(np.float64)


FP8_FORMATS = {
    # name: (mantissa bits, minimum normal exponent, largest finite)
    "e4m3": (3, -6, 448.0),
    "e5m2": (2, -14, 57344.0),
}


def _round_fp8_real(x: np.ndarray, fmt: str) -> np.ndarray:
    mbits, emin, vmax = FP8_FORMATS[fmt]
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    nan = np.isnan(x)
    a = np.abs(np.where(nan, 0.0, x))
    with np.errstate(divide="ignore"):
        e = np.floor(np.log2(np.where(a > 0, a, 1.0)))
    e = np.maximum(e, emin)
    quantum = np.exp2(e - mbits)
    q = np.round(a / quantum) * quantum          # np.round is ties-to-even
    q = np.minimum(q, vmax)                       # satfinite
    out[:] = np.copysign(q, x)
    out[nan] = np.nan
    return out


def round_fp8(x: np.ndarray, fmt: str) -> np.ndarray:
    """Round to OCP FP8 ('e4m3' or 'e5m2'), RN-even, satfinite; returns float64/complex128."""
    x = np.asarray(x)
    if np.iscomplexobj(x):
        return _round_fp8_real(x.real, fmt) + 1j * _round_fp8_real(x.imag, fmt)
    return _round_fp8_real(x, fmt)


BF16_FRACTION_BITS = 7
BF16_MIN_NORMAL_EXP = -126
BF16_MAX = (2.0 - 2.0 ** -7) * 2.0 ** 127


def _round_bf16_real(x: np.ndarray) -> np.ndarray:
    x = np.asarray(x, dtype=np.float64)
    nan = np.isnan(x)
    a = np.abs(np.where(nan, 0.0, x))
    with np.errstate(divide="ignore", invalid="ignore"):
        e = np.floor(np.log2(np.where((a > 0) & np.isfinite(a), a, 1.0)))
    e = np.maximum(e, BF16_MIN_NORMAL_EXP)
    quantum = np.exp2(e - BF16_FRACTION_BITS)
    with np.errstate(invalid="ignore", over="ignore"):
        q = np.round(a / quantum) * quantum       # ties to even
    q = np.where(q > BF16_MAX, np.inf, q)        # round-to-nearest overflows to infinity
    q = np.where(np.isinf(a), np.inf, q)
    return np.where(nan, np.nan, np.copysign(q, x))


def round_bfloat16(x: np.ndarray) -> np.ndarray:
    """Round to bfloat16, RN-even, overflow to infinity; returns float64/complex128."""
    x = np.asarray(x)
    if np.iscomplexobj(x):
        return _round_bf16_real(x.real) + 1j * _round_bf16_real(x.imag)
    return _round_bf16_real(x)
