"""GPU parity of the general forward-multiply-inverse pipeline (Section VIII, Generality).

Circular convolution and correlation of batched dense lines, y =
IDFT(DFT(x) . H) with the 1/N shift before the inverse, run through
sar_range_compress with transpose_out = 0 (the range matched filter is the
correlation case) and through the dedicated entry bfp_spectral_filter: one
filter for every line, or one per line (a spectral layer's per-channel
weights, truncated to the lowest modes), in each arithmetic mode.  The inputs
are not a radar scene: x and the kernel g are seeded complex Gaussians, H =
DFT(g) or conj(DFT(g)) rounded to complex64.

Bars as for range compression: FP32 output to relative L2 <= 1e-6 of the
FP64 pipeline on the same H; FP16 output per element within half an FP16 ulp
plus the FP32 arithmetic error.  For short lines the oracle's defining sums
(no FFT) are checked as well.
"""

import numpy as np
import pytest

from oracle import conv, metrics
from paper_2605_28451_gb300 import bfpfft as B
from paper_2605_28451_gb300 import build, synth

from _helpers import empty_like_storage, fp16_elementwise_ok, from_device, storage_round, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib(cuda_ready):
    build.build()
    B.lib()


def gpu_spectral_filter(x_stored, in_dtype, out_dtype, h64):
    import torch
    batch, n = x_stored.shape
    x = to_device(x_stored, in_dtype)
    h = to_device(h64, B.F32)
    out = empty_like_storage((batch, n), out_dtype)
    B.sar_range_compress(x, in_dtype, out, out_dtype, h, batch, n, False)
    torch.cuda.synchronize()
    assert B.bfpfft_device_status() == B.OK
    return from_device(out, out_dtype)


@pytest.mark.parametrize("n", [256, 1024, 4096, 16384])
@pytest.mark.parametrize("kind", ["convolution", "correlation"])
@pytest.mark.parametrize("in_dtype,out_dtype", [(B.F32, B.F32), (B.F16_BFP, B.F16_BFP), (B.F32, B.F16_BFP)])
def test_convolution_and_correlation(n, kind, in_dtype, out_dtype):
    batch = 7
    x = storage_round(synth.complex_gaussian(batch, n, seed=n + 1), in_dtype)
    g = synth.complex_gaussian(1, n, seed=n + 2)[0] / np.sqrt(n)     # |y| of order one
    spec = np.fft.fft(g)
    h = storage_round(spec if kind == "convolution" else np.conj(spec), B.F32)
    got = gpu_spectral_filter(x, in_dtype, out_dtype, h)
    expect = conv.spectral(x, h)
    if out_dtype == B.F32:
        assert metrics.rel_l2(expect, got) <= 1e-6
    else:
        ok, worst = fp16_elementwise_ok(got, expect)
        assert ok, worst
    if n <= 1024:
        direct = conv.convolve_direct(x, g) if kind == "convolution" else conv.correlate_direct(x, g)
        assert metrics.rel_l2(direct, got) <= (1e-6 if out_dtype == B.F32 else 1e-3)


def spectral_entry(x_stored, in_dtype, out_dtype, h64, h_stride, arith):
    import torch
    batch, n = x_stored.shape
    x = to_device(x_stored, in_dtype)
    h = to_device(h64, B.F32)
    out = empty_like_storage((batch, n), out_dtype)
    B.bfp_spectral_filter(x, in_dtype, h, h_stride, out, out_dtype, n, batch, arith)
    torch.cuda.synchronize()
    assert B.bfpfft_device_status() == B.OK
    return from_device(out, out_dtype)


# (arith, in, out, SQNR floor against FP64 for FP16 outputs)
MODES = [(B.ARITH_F32, B.F32, B.F32, None), (B.ARITH_F32, B.F16_BFP, B.F16_BFP, None),
         (B.ARITH_F16, B.F32, B.F16_BFP, 50.0), (B.ARITH_F16_MUL_F32_ACC, B.F32, B.F16_BFP, 55.0),
         (B.ARITH_F16_MUL_F32_ACC, B.F16_BFP, B.F16_BFP, 55.0)]


def _check_mode(got, expect, out_dtype, floor):
    if out_dtype == B.F32:
        assert metrics.rel_l2(expect, got) <= 1e-6
    elif floor is None:
        ok, worst = fp16_elementwise_ok(got, expect)
        assert ok, worst
    else:
        assert metrics.sqnr_db(expect, got) >= floor


@pytest.mark.parametrize("arith,in_dtype,out_dtype,floor", MODES)
@pytest.mark.parametrize("kind", ["convolution", "correlation"])
def test_spectral_entry_one_filter(arith, in_dtype, out_dtype, floor, kind):
    """bfp_spectral_filter with h_stride = 0 (one filter for every line) at
    N = 4096, which every mode supports: the FP64 pipeline of the same H, and
    the defining sums."""
    n, batch = 4096, 9
    x = storage_round(synth.complex_gaussian(batch, n, seed=5), in_dtype)
    g = synth.complex_gaussian(1, n, seed=6)[0] / np.sqrt(n)
    h = storage_round(conv.convolution_filter(g) if kind == "convolution" else conv.correlation_filter(g), B.F32)
    got = spectral_entry(x, in_dtype, out_dtype, h, 0, arith)
    _check_mode(got, conv.spectral(x, h), out_dtype, floor)
    direct = conv.convolve_direct(x[:2], g) if kind == "convolution" else conv.correlate_direct(x[:2], g)
    if out_dtype == B.F32:
        assert metrics.rel_l2(direct, got[:2]) <= 1e-6
    else:
        assert metrics.sqnr_db(direct, got[:2]) >= (floor if floor is not None else 60.0) - 1.0


@pytest.mark.parametrize("arith,in_dtype,out_dtype,floor", MODES)
@pytest.mark.parametrize("batch", [3, 1300])
def test_spectral_entry_per_line_filters(arith, in_dtype, out_dtype, floor, batch):
    """h_stride = n: every line has its own filter -- a spectral layer's
    per-channel weights, nonzero only on the 24 lowest modes of each sign
    (the truncation of a Fourier neural operator layer).  Each line against
    the FP64 pipeline with its own weights; a line filtered with another
    line's weights would miss by far more than the bars.  1300 lines make
    every kernel's CTAs take more than one line or group."""
    n, modes = 4096, 24
    rng = np.random.default_rng(batch)
    x = storage_round(synth.complex_gaussian(batch, n, seed=batch + 1), in_dtype)
    w = np.zeros((batch, n), dtype=complex)
    keep = np.r_[np.arange(modes), np.arange(n - modes, n)]
    w[:, keep] = (rng.standard_normal((batch, keep.size)) + 1j * rng.standard_normal((batch, keep.size))) * 4.0
    h = storage_round(w, B.F32)
    got = spectral_entry(x, in_dtype, out_dtype, h, n, arith)
    expect = conv.spectral(x, h)
    _check_mode(got, expect, out_dtype, floor)
    rows = [0, batch // 2, batch - 1]
    for r in rows:
        assert metrics.sqnr_db(expect[r], got[r]) >= (100.0 if out_dtype == B.F32 else 45.0)
        if batch > 1:
            other = conv.spectral(x[r], h[(r + 1) % batch])
            assert metrics.sqnr_db(other, got[r]) < 10.0


@pytest.mark.parametrize("n", [256, 16384])
def test_spectral_entry_per_line_filters_other_lengths(n):
    """Per-line filters at the shortest and longest line lengths (FP32 mode,
    FP16 storage): the one-CTA and the cluster row kernels."""
    batch = 37
    rng = np.random.default_rng(n)
    x = storage_round(synth.complex_gaussian(batch, n, seed=n), B.F16_BFP)
    h = storage_round((rng.standard_normal((batch, n)) + 1j * rng.standard_normal((batch, n))) / np.sqrt(2), B.F32)
    got = spectral_entry(x, B.F16_BFP, B.F16_BFP, h, n, B.ARITH_F32)
    ok, worst = fp16_elementwise_ok(got, conv.spectral(x, h))
    assert ok, worst


@pytest.mark.parametrize("arith,in_dtype,out_dtype,floor", MODES)
def test_spectral_entry_in_place(arith, in_dtype, out_dtype, floor):
    """x and out the same buffer (same storage type): the bits of the out-of-place call."""
    import torch
    if in_dtype != out_dtype:
        pytest.skip("in place needs one storage type")
    n, batch = 4096, 300
    x = storage_round(synth.complex_gaussian(batch, n, seed=31), in_dtype)
    h = storage_round(conv.correlation_filter(synth.complex_gaussian(1, n, seed=32)[0] / np.sqrt(n)), B.F32)
    hd = to_device(h, B.F32)
    src = to_device(x, in_dtype)
    ref = torch.empty_like(src)
    B.bfp_spectral_filter(src, in_dtype, hd, 0, ref, out_dtype, n, batch, arith)
    buf = src.clone()
    B.bfp_spectral_filter(buf, in_dtype, hd, 0, buf, out_dtype, n, batch, arith)
    torch.cuda.synchronize()
    assert torch.equal(buf, ref)
