"""GPU parity of the general forward-multiply-inverse pipeline (Section VIII, Generality).

Circular convolution and correlation of batched dense lines, y =
IDFT(DFT(x) . H) with the 1/N shift before the inverse, run through
sar_range_compress with transpose_out = 0 (the range matched filter is the
correlation case).  The inputs are not a radar scene: x and the kernel g are
seeded complex Gaussians, H = DFT(g) or conj(DFT(g)) rounded to complex64.

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
