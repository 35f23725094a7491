"""Rounding emulation of FFT precision modes (oracle; test infrastructure only).

The paper measures FFT quality in several precision modes:
- pure FP16 arithmetic with FP16 twiddle tables (Section III-A, Table I);
- FP16 storage with wider compute, and the same with OCP FP8 storage
  (Section VII, Table V);
- FP32, pure FP16, FP16 storage / FP32 compute and FP16 multiply / FP32
  accumulate, for the SAR chain (Section VI);
- bfloat16, as the range-for-mantissa alternative (Section IV-C).

``fft_rounded`` restates one radix-2 decimation-in-time FFT (bit reversal,
then log2 N butterfly stages: t = w * odd, then even + t and even - t) with
three rounding hooks:

    store(v)  applied to the input and to each stage's output (storage points;
              every stage unless ``store_stages`` names a subset)
    mul(v)    applied to each real product of the twiddle multiply
    add(v)    applied to each real sum or difference, and to the twiddle
              table entries (the table is built in the arithmetic format)

The twiddle multiply takes four real products and two real sums, and the
butterfly four real sums, so one complex butterfly is the ten-operation
"standard" butterfly of Table I.  A hook left as None is exact FP64.

The pure-Python structure mirrors ``oracle.fft``'s radix-2 transform, so with
every hook None it is the exact DFT up to FP64 rounding.  Nothing in it is
tuned to the paper's printed numbers; the CPU tests compare its SQNR with
Tables I and V, and with the mantissa-width and storage-count rules that
follow from the rounding error model.

``count_storage_points`` and ``predict_sqnr_db`` give the error model itself:
each storage point of a format with p fraction bits adds noise of relative
power c * 2^(-2p), independent of scale, so K points give
SQNR = -10 log10(K c 2^(-2p)).
"""

from __future__ import annotations

from typing import Callable, Optional

import numpy as np

from . import quant
from .fft import _bit_reverse_indices

Hook = Optional[Callable[[np.ndarray], np.ndarray]]


def _apply(hook: Hook, v: np.ndarray) -> np.ndarray:
    return v if hook is None else hook(v)


def _complex(hook: Hook, z: np.ndarray) -> np.ndarray:
    if hook is None:
        return z
    return hook(z.real) + 1j * hook(z.imag)


def fft_rounded(x: np.ndarray, store: Hook = None, mul: Hook = None, add: Hook = None,
                sign: int = -1, store_stages=None, store_input: bool = True) -> np.ndarray:
    """sum_n x[n] exp(sign 2 pi i n k / N) along the last axis, rounding at the hooks.

    ``store_stages`` lists the stages (1 .. log2 N) after which ``store``
    applies; None means every stage.  Stages 4, 8, 12 of N = 4096 are the
    pass boundaries of a radix-16 schedule, and {log2 N} alone is a
    transform that stores only its output.  ``store_input`` rounds the
    input as well.
    """
    x = np.asarray(x, dtype=np.complex128)
    n = x.shape[-1]
    lead = x.shape[:-1]
    a = x[..., _bit_reverse_indices(n)]
    if store_input:
        a = _complex(store, a)
    re, im = a.real.copy(), a.imag.copy()
    half, stage = 1, 0
    while half < n:
        stage += 1
        w = np.exp(sign * 2j * np.pi * np.arange(half) / (2 * half))
        wr, wi = _apply(add, w.real), _apply(add, w.imag)
        br = re.reshape(lead + (n // (2 * half), 2, half))
        bi = im.reshape(lead + (n // (2 * half), 2, half))
        er, ei = br[..., 0, :], bi[..., 0, :]
        orr, oi = br[..., 1, :], bi[..., 1, :]
        # t = w * odd: four products, two sums
        tr = _apply(add, _apply(mul, orr * wr) - _apply(mul, oi * wi))
        ti = _apply(add, _apply(mul, orr * wi) + _apply(mul, oi * wr))
        # even +- t: four sums
        re = np.stack((_apply(add, er + tr), _apply(add, er - tr)), axis=-2).reshape(lead + (n,))
        im = np.stack((_apply(add, ei + ti), _apply(add, ei - ti)), axis=-2).reshape(lead + (n,))
        if store_stages is None or stage in store_stages:
            re, im = _apply(store, re), _apply(store, im)
        half *= 2
    return re + 1j * im


# The precision modes, as (store, mul, add) hooks.
MODES = {
    "fp64": (None, None, None),
    "fp32": (quant.round_binary32, quant.round_binary32, quant.round_binary32),
    "pure_fp16": (quant.round_binary16, quant.round_binary16, quant.round_binary16),
    "fp16_storage_fp32_compute": (quant.round_binary16, quant.round_binary32, quant.round_binary32),
    "fp16_mul_fp32_acc": (quant.round_binary16, quant.round_binary16, quant.round_binary32),
    "pure_bf16": (quant.round_bfloat16, quant.round_bfloat16, quant.round_bfloat16),
    "fp16_storage_fp64_compute": (quant.round_binary16, None, None),
    "e4m3_storage_fp64_compute": (lambda v: quant.round_fp8(v, "e4m3"), None, None),
    "e5m2_storage_fp64_compute": (lambda v: quant.round_fp8(v, "e5m2"), None, None),
}


def fft_mode(x: np.ndarray, mode: str, sign: int = -1) -> np.ndarray:
    store, mul, add = MODES[mode]
    return fft_rounded(x, store=store, mul=mul, add=add, sign=sign)


def count_storage_points(n: int, store_stages=None, store_input: bool = True) -> int:
    """Storage points of ``fft_rounded`` with a store hook (the input, then the stored stages)."""
    stages = (n.bit_length() - 1) if store_stages is None else len(store_stages)
    return stages + (1 if store_input else 0)


def predict_sqnr_db(points: int, fraction_bits: int, c: float) -> float:
    """SQNR of ``points`` independent roundings of relative noise power c 2^(-2p) each."""
    return -10.0 * np.log10(points * c * 2.0 ** (-2 * fraction_bits))
