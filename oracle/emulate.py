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


# ---- radix-16 schedule with every operation rounded -------------------------
#
# The same precision mode ("pure FP16": every add and multiply in the storage
# format) on a radix-16 Stockham schedule instead of radix 2: each pass
# multiplies point r of butterfly j by W_{16 Ns}^{(j mod Ns) r}, runs a 16-point
# DFT as two layers of 4-point DFTs around the internal twiddles W16^{r1 k2},
# and writes point r to (j / Ns) 16 Ns + (j mod Ns) + r Ns.  The complex
# product by a stored twiddle w = (c, s) takes two rounded steps,
#     t = rn(a.re * (c, s)),   a w = rn(a.im * (-s, c) + t)   (fused),
# and the products by W16^2, W16^6 and -i are a rounded sum and a rounded
# product by the stored sqrt(1/2), and an exact swap.  Twiddles are rounded
# once from their exact values.  With op = None it is the exact DFT.


def _r(op, v):
    return v if op is None else op(v)


def _cmul16(op, ar, ai, wr, wi):
    tr, ti = _r(op, ar * wr), _r(op, ar * wi)
    return _r(op, ai * (-wi) + tr), _r(op, ai * wr + ti)


def _dft4_16(op, a):
    (r0, i0), (r1, i1), (r2, i2), (r3, i3) = a
    t0 = (_r(op, r0 + r2), _r(op, i0 + i2))
    t1 = (_r(op, r0 - r2), _r(op, i0 - i2))
    t2 = (_r(op, r1 + r3), _r(op, i1 + i3))
    e = (_r(op, i1 - i3), -_r(op, r1 - r3))              # -i (a1 - a3), rounded once
    return [(_r(op, t0[0] + t2[0]), _r(op, t0[1] + t2[1])),
            (_r(op, t1[0] + e[0]), _r(op, t1[1] + e[1])),
            (_r(op, t0[0] - t2[0]), _r(op, t0[1] - t2[1])),
            (_r(op, t1[0] - e[0]), _r(op, t1[1] - e[1]))]


def _dft16_rounded(op, v):
    v = list(v)
    for r1 in range(4):
        v[r1], v[r1 + 4], v[r1 + 8], v[r1 + 12] = _dft4_16(op, [v[r1], v[r1 + 4], v[r1 + 8], v[r1 + 12]])
    c1, s1, h = _r(op, np.cos(np.pi / 8)), _r(op, np.sin(np.pi / 8)), _r(op, np.sqrt(0.5))

    def w2(a):
        return _r(op, _r(op, a[0] + a[1]) * h), _r(op, _r(op, a[1] - a[0]) * h)

    def w6(a):
        return _r(op, _r(op, a[1] - a[0]) * h), _r(op, _r(op, -a[0] - a[1]) * h)

    v[5] = _cmul16(op, *v[5], c1, -s1)
    v[9] = w2(v[9])
    v[13] = _cmul16(op, *v[13], s1, -c1)
    v[6] = w2(v[6])
    v[10] = (v[10][1], -v[10][0])
    v[14] = w6(v[14])
    v[7] = _cmul16(op, *v[7], s1, -c1)
    v[11] = w6(v[11])
    v[15] = _cmul16(op, *v[15], -c1, s1)
    out = [None] * 16
    for k2 in range(4):
        a = _dft4_16(op, [v[4 * k2], v[4 * k2 + 1], v[4 * k2 + 2], v[4 * k2 + 3]])
        for k1 in range(4):
            out[k2 + 4 * k1] = a[k1]
    return out


def fft_radix16_rounded(x: np.ndarray, op: Hook = None) -> np.ndarray:
    """Forward DFT along the last axis (N a power of 16) on the radix-16 schedule, rounding every operation."""
    x = np.asarray(x, dtype=np.complex128)
    n = x.shape[-1]
    if n < 16 or 16 ** round(np.log(n) / np.log(16)) != n:
        raise ValueError(f"length {n} is not a power of 16")
    re, im = _r(op, x.real.copy()), _r(op, x.imag.copy())
    q = n // 16
    j = np.arange(q)
    ns = 1
    while ns < n:
        k = j % ns
        u = [(re[..., j + q * r], im[..., j + q * r]) for r in range(16)]
        if ns > 1:
            for r in range(1, 16):
                w = np.exp(-2j * np.pi * k * r / (16 * ns))
                u[r] = _cmul16(op, *u[r], _r(op, w.real), _r(op, w.imag))
        o = _dft16_rounded(op, u)
        nre, nim = np.empty_like(re), np.empty_like(im)
        base = (j // ns) * ns * 16 + k
        for r in range(16):
            nre[..., base + r * ns], nim[..., base + r * ns] = o[r]
        re, im = nre, nim
        ns *= 16
    return re + 1j * im


# ---- radix-16 schedule with FP16 operands and FP32 accumulation ---------------
#
# Section VI lists an "FP16 multiply / FP32 accumulate" mode.  On a radix-16
# Stockham schedule whose 16-point DFT blocks are dense 16 x 16 products, the
# mode reads: every pass takes its 16 inputs as FP16 operands, multiplies them
# by the DFT-16 coefficients W16^(q r) held in FP16, and sums the (exact)
# products in FP32; the pass twiddles W_{16 Ns}^{k r} multiply the FP32 sums
# in FP32 (the two products and the fused sum of a complex multiply, each
# rounded), and only the next pass's operand rounding returns them to FP16.
# The output is stored in FP16.  Hooks: ``operand`` (pass inputs), ``coeff``
# (the DFT-16 coefficients), ``acc`` (the dot-product sums, the twiddle
# products and the twiddle table), ``store`` (the output).  All None gives
# the exact DFT.  The order of the FP32 additions inside a dot product is not
# modelled: the exact sum is rounded once.


def fft_radix16_mma(x: np.ndarray, operand: Hook = quant.round_binary16, coeff: Hook = quant.round_binary16,
                    acc: Hook = quant.round_binary32, store: Hook = quant.round_binary16) -> np.ndarray:
    """Forward DFT along the last axis (N a power of 16) with FP16 operands and FP32 accumulation."""
    x = np.asarray(x, dtype=np.complex128)
    n = x.shape[-1]
    if n < 16 or 16 ** round(np.log(n) / np.log(16)) != n:
        raise ValueError(f"length {n} is not a power of 16")
    qr = np.outer(np.arange(16), np.arange(16)) % 16
    w16 = np.exp(-2j * np.pi * qr / 16)
    w16 = _r(coeff, w16.real) + 1j * _r(coeff, w16.imag)
    vals = x.copy()
    q = n // 16
    j = np.arange(q)
    ns = 1
    while ns < n:
        k = j % ns
        u = np.stack([vals[..., j + q * r] for r in range(16)], axis=-2)      # [..., 16, q]
        if ns > 1:
            r = np.arange(16)[:, None]
            w = np.exp(-2j * np.pi * k[None, :] * r / (16 * ns))
            wr, wi = _r(acc, w.real), _r(acc, w.imag)
            ur, ui = u.real, u.imag
            # fmaf(a.re, w.re, -rn(a.im w.im)), fmaf(a.re, w.im, rn(a.im w.re))
            u = _r(acc, ur * wr - _r(acc, ui * wi)) + 1j * _r(acc, ur * wi + _r(acc, ui * wr))
        a = _r(operand, u.real) + 1j * _r(operand, u.imag)
        y = np.einsum("qr,...rj->...qj", w16, a)
        y = _r(acc, y.real) + 1j * _r(acc, y.imag)
        out = np.empty_like(vals)
        base = (j // ns) * ns * 16 + k
        for r in range(16):
            out[..., base + r * ns] = y[..., r, :]
        vals = out
        ns *= 16
    return _r(store, vals.real) + 1j * _r(store, vals.imag)
