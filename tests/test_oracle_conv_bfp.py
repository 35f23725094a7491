"""Pins for the convolution / correlation oracle and the adaptive block exponents (CPU only).

Convolution and correlation: the direct sums against the shift and
constant-kernel closed forms, symmetry, numpy's linear convolution on
zero-padded inputs, and the convolution and correlation theorems (the
spectral pipeline against the direct sums).  Adaptive exponents: a plain
search over integers for the smallest admissible exponent, exact
power-of-two covariance, the mantissa range, the storage error bound and
inputs whose fixed-shift output would overflow FP16.
"""

import numpy as np
import pytest

from oracle import bfp, conv
from oracle import fft as F
from oracle import metrics, quant
from paper_2605_28451_gb300 import synth


@pytest.mark.parametrize("shift", [0, 1, 5, 31])
def test_convolution_with_shifted_impulse_is_a_rotation(shift):
    x = synth.complex_gaussian(3, 32, seed=shift)
    g = np.zeros(32, dtype=np.complex128)
    g[shift] = 1.0
    assert np.allclose(conv.convolve_direct(x, g), np.roll(x, shift, axis=-1), atol=1e-14)
    assert np.allclose(conv.correlate_direct(x, g), np.roll(x, -shift, axis=-1), atol=1e-14)


def test_convolution_with_constant_kernel_sums_the_line():
    x = synth.complex_gaussian(2, 16, seed=1)
    y = conv.convolve_direct(x, np.ones(16))
    assert np.allclose(y, x.sum(axis=-1, keepdims=True) * np.ones(16), atol=1e-12)


def test_convolution_commutes_and_correlation_is_conjugate_symmetric():
    x = synth.complex_gaussian(1, 24, seed=2)[0]
    g = synth.complex_gaussian(1, 24, seed=3)[0]
    assert np.allclose(conv.convolve_direct(x, g), conv.convolve_direct(g, x), atol=1e-12)
    c_xg = conv.correlate_direct(x, g)
    c_gx = conv.correlate_direct(g, x)
    lag = (-np.arange(24)) % 24
    assert np.allclose(c_xg, np.conj(c_gx[lag]), atol=1e-12)
    assert conv.correlate_direct(x, x)[0] == pytest.approx(np.vdot(x, x))     # energy at lag 0


def test_circular_convolution_of_zero_padded_lines_is_linear_convolution():
    rng = np.random.default_rng(4)
    a = rng.standard_normal(20) + 1j * rng.standard_normal(20)
    b = rng.standard_normal(12) + 1j * rng.standard_normal(12)
    n = 32                                                      # >= 20 + 12 - 1
    pa = np.zeros(n, complex)
    pa[:20] = a
    pb = np.zeros(n, complex)
    pb[:12] = b
    assert np.allclose(conv.convolve_direct(pa, pb)[:31], np.convolve(a, b), atol=1e-12)


@pytest.mark.parametrize("n", [16, 64, 256])
def test_convolution_and_correlation_theorems(n):
    x = synth.complex_gaussian(4, n, seed=n)
    g = synth.complex_gaussian(1, n, seed=n + 1)[0]
    conv_direct = conv.convolve_direct(x, g)
    corr_direct = conv.correlate_direct(x, g)
    assert metrics.rel_l2(conv_direct, conv.spectral(x, conv.convolution_filter(g))) <= 1e-12
    assert metrics.rel_l2(corr_direct, conv.spectral(x, conv.correlation_filter(g))) <= 1e-12


def test_fixed_shift_bounds_the_inverse_by_the_spectrum():
    """Section VIII: with the 1/N shift, the inverse is an average of the
    products, so its magnitude never exceeds the largest product; the
    unnormalised inverse is N times larger."""
    x = synth.complex_gaussian(8, 512, seed=5)
    h = conv.correlation_filter(synth.complex_gaussian(1, 512, seed=6)[0])
    prod = F.fft(x) * h
    y = conv.spectral(x, h)
    assert np.all(np.abs(y).max(axis=-1) <= np.abs(prod).max(axis=-1) * (1 + 1e-12))
    assert np.allclose(F.ifft_unnormalised(prod), 512 * y, rtol=1e-12, atol=1e-9)


def _exponent_by_search(m, limit):
    for e in range(-80, 81):
        if m * 2.0 ** -e <= limit:
            return e
    raise AssertionError


@pytest.mark.parametrize("limit", [2.0 ** 14, 448.0, 1000.0])
def test_block_exponent_is_the_smallest_admissible(limit):
    rng = np.random.default_rng(9)
    v = (rng.standard_normal((200, 8)) + 1j * rng.standard_normal((200, 8))) * 10.0 ** rng.integers(-20, 20, (200, 1))
    v[3] = 0.0
    v[4, 0] = limit                                             # exactly at the limit: e = 0
    v[4, 1:] = 0.0
    v[5, 0] = 2 * limit                                         # a power of two above it: e = 1
    v[5, 1:] = 0.0
    e = bfp.block_exponent(v, limit)
    m = np.maximum(np.abs(v.real), np.abs(v.imag)).max(axis=-1)
    for i in range(200):
        assert e[i] == (0 if m[i] == 0 else _exponent_by_search(m[i], limit)), i
    assert e[4] == 0 and e[5] == 1


@pytest.mark.parametrize("k", [-40, -7, 0, 3, 60])
def test_power_of_two_scaling_moves_only_the_exponent(k):
    x = synth.complex_gaussian(16, 256, seed=10)
    m0, e0 = bfp.quantize(x)
    m1, e1 = bfp.quantize(x * 2.0 ** k)
    assert np.array_equal(m0, m1)
    assert np.array_equal(e1, e0 + k)


def test_mantissa_range_and_storage_error():
    x = synth.complex_gaussian(64, 1024, seed=11) * 10.0 ** np.random.default_rng(12).uniform(-8, 8, (64, 1))
    m, e = bfp.quantize(x)
    peak = bfp.block_max(m)
    assert np.all(peak <= bfp.DEFAULT_LIMIT) and np.all(peak > bfp.DEFAULT_LIMIT / 2)
    err = bfp.value(m, e) - x
    scale = np.ldexp(1.0, e)[:, None]
    # half an FP16 ulp of each component, or half the smallest subnormal step, in block units
    for part_err, part in ((err.real, x.real), (err.imag, x.imag)):
        assert np.all(np.abs(part_err) <= 2.0 ** -11 * np.abs(part) + 2.0 ** -25 * scale)


def test_pathological_amplitudes_store_without_overflow():
    """A line that the fixed 1/N schedule would store far beyond 65504 (a
    flat spectrum of magnitude N times a large amplitude) keeps a finite
    mantissa, and the value matches the FP64 result to FP16 precision."""
    n = 1024
    pulse = np.exp(1j * np.pi * np.arange(n) ** 2 / n)           # unit-modulus spectrum magnitude sqrt(n)
    x = np.stack([pulse * 1e6, pulse, pulse * 1e-6])
    h = conv.correlation_filter(pulse)
    y = conv.spectral(x, h)
    assert np.abs(y[0]).max() > 1e8                              # n * 1e6 at lag 0
    assert np.isinf(quant.round_binary16(y[0])).any()           # fixed schedule: overflow
    m, e = bfp.adaptive_spectral(x, h)
    assert np.all(np.isfinite(m))
    for i in range(3):
        assert metrics.rel_l2(y[i], bfp.value(m[i], e[i])) <= 2.0 ** -10


def test_zero_block():
    m, e = bfp.quantize(np.zeros((2, 8), complex))
    assert np.all(m == 0) and np.all(e == 0)
