"""GPU parity of the batched FFT (bfpfft_plan_create / bfpfft_exec) against the FP64 oracle.

Tolerances, stated against FP64 on the exact values the GPU receives:
* FP32 storage: relative L2 error <= 1e-6 (and per element <= 1e-5 of the rms).
* FP16 storage (block-floating-point): every element within half an FP16 ulp
  of the oracle plus the FP32 arithmetic error (tests/_helpers.py), and
  SQNR >= 55 dB at N = 4096 (Section III-A, Table II), within 1.5 dB of the
  oracle emulator's prediction for the same storage schedule.
* FP8 storage: every element equal to the oracle's rounding of the same
  value, or one FP8 step away where FP32 arithmetic puts the value within
  1e-5 (relative) of a rounding boundary.
"""

import numpy as np
import pytest

from oracle import fft as F
from oracle import emulate, metrics, quant
from paper_2605_28451_gb300 import bfpfft as B
from paper_2605_28451_gb300 import build, synth

from _helpers import empty_like_storage, fp8_close, fp16_elementwise_ok, from_device, storage_round, to_device

pytestmark = pytest.mark.gpu

SIZES = [16, 32, 64, 128, 256, 512, 1024, 2048, 4096, 8192, 16384, 32768, 65536]


@pytest.fixture(scope="module", autouse=True)
def _lib(cuda_ready):
    build.build()
    B.lib()


def run_fft(x_stored: np.ndarray, dtype: int, direction: int, inplace=False):
    import torch
    batch, n = x_stored.shape
    plan = B.bfpfft_plan_create(n, batch, dtype, direction)
    xin = to_device(x_stored, dtype)
    out = xin if inplace else empty_like_storage((batch, n), dtype)
    B.bfpfft_exec(plan, xin, out)
    torch.cuda.synchronize()
    return from_device(out, dtype)


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("batch", [1, 7])
def test_f32_forward_and_inverse(n, batch, rows_variant):
    x = storage_round(synth.complex_gaussian(batch, n, seed=n + batch), B.F32)
    got = run_fft(x, B.F32, B.FORWARD)
    ref = F.fft(x)
    assert metrics.rel_l2(ref, got) <= 1e-6
    assert np.max(np.abs(got - ref)) <= 1e-5 * np.sqrt(np.mean(np.abs(ref) ** 2))
    y = storage_round(ref, B.F32)
    got_i = run_fft(y, B.F32, B.INVERSE)
    ref_i = F.ifft(y)
    assert metrics.rel_l2(ref_i, got_i) <= 1e-6


ROW_VARIANTS = ["tma", "plain", "pp", "h16", "h16pp", "tma_pp", "tma_h16", "tma_h16pp", "tc", "plain4", "plain_l2",
                "plain4_l2", "h16_l2", "h16_4_l2", "h16s_4_l2", "twopass"]


@pytest.fixture(params=ROW_VARIANTS)
def rows_variant(request, monkeypatch):
    """Every row-kernel variant (BFPFFT_ROWS): pipelined persistent or plain,
    FP32 or FP16 shared-memory exchange, one buffer or two."""
    monkeypatch.setenv("BFPFFT_ROWS", request.param)
    yield request.param
    assert B.bfpfft_device_status() == B.OK


def f16_check(got, ref, variant, n):
    """FP16-storage parity.  With an FP32 exchange every output is the RN
    rounding of an FP32 result (tests/_helpers.py).  With an FP16 exchange
    (variants h16*), and between the two passes of the two-pass long lines,
    each inter-pass exchange is an FP16 storage point as well;
    its rounding errors (<= 2^-12 of the intermediate) spread through the
    remaining passes like noise of rms about 2^-11 rms(y), so every element
    must lie within 2^-11 |y| + 6 * 2^-11 rms(y) (a 6-sigma bound) and the
    SQNR must reach 55 dB (the benchmark spec's FP16-BFP bar)."""
    fp16_inside = (("h16" in variant and n > 16) or (variant == "tc" and n == 4096)
                   or (variant == "twopass" and n >= 32768))
    if fp16_inside:
        # The tensor-core variant (tc, N = 4096) also rounds the DFT-16
        # coefficients to FP16: two error sources of rms 2^-11/sqrt(3) per pass,
        # about 1.1 * 2^-11 rms per component in all; 8 * 2^-11 rms is > 7 sigma.
        rms = np.sqrt(np.mean(np.abs(ref) ** 2))
        k = 8.0 if variant == "tc" else 6.0
        bound = 2.0 ** -11 * (np.abs(ref) + k * rms)
        assert np.all(np.abs(got.real - ref.real) <= bound) and np.all(np.abs(got.imag - ref.imag) <= bound)
        assert metrics.sqnr_db(ref, got) >= 55.0
    else:
        ok, worst = fp16_elementwise_ok(got, ref)
        assert ok, worst


@pytest.mark.parametrize("n,batch", [(n, b) for n in SIZES for b in (3, 33) if n * b <= (1 << 21)] +
                         [(256, 20000), (4096, 1000), (65536, 5)])
def test_f16_bfp_forward_and_inverse(n, batch, rows_variant):
    """Ragged batches; the last two cases make every persistent CTA of the
    pipelined kernel walk several groups and end on a partial group."""
    x = storage_round(synth.complex_gaussian(batch, n, seed=100 + n + batch), B.F16_BFP)
    got = run_fft(x, B.F16_BFP, B.FORWARD)
    ref = F.fft(x)
    f16_check(got, ref, rows_variant, n)
    spec = storage_round(ref, B.F16_BFP)
    got_i = run_fft(spec, B.F16_BFP, B.INVERSE)
    ref_i = F.ifft(spec)
    f16_check(got_i, ref_i, rows_variant, n)


def test_f16_bfp_sqnr_at_4096_batch_256():
    """The Table II workload: N = 4096, batch 256, re, im ~ N(0, 1), seed 0."""
    x64 = synth.complex_gaussian(256, 4096, seed=0)
    x = storage_round(x64, B.F16_BFP)
    X = run_fft(x, B.F16_BFP, B.FORWARD)
    ref = F.fft(x)
    s_fwd = metrics.sqnr_db(ref, X)
    assert s_fwd >= 55.0, s_fwd
    # The default path computes in FP32 and stores FP16 only at the output (the
    # input is FP16 already).  The oracle's emulator of that storage schedule
    # predicts the SQNR, and the GPU must land within 1.5 dB of it.
    schedule = dict(store=quant.round_binary16, mul=quant.round_binary32, add=quant.round_binary32,
                    store_stages={12}, store_input=False)
    pred_fwd = metrics.sqnr_db(ref, emulate.fft_rounded(x, **schedule))
    assert abs(s_fwd - pred_fwd) <= 1.5, (s_fwd, pred_fwd)
    y = run_fft(X, B.F16_BFP, B.INVERSE)
    s_inv = metrics.sqnr_db(F.ifft(X), y)
    assert s_inv >= 55.0, s_inv
    pred_inv = metrics.sqnr_db(F.ifft(X), emulate.fft_rounded(X / 4096, sign=+1, **schedule))
    assert abs(s_inv - pred_inv) <= 1.5, (s_inv, pred_inv)
    assert metrics.rel_l2(x, y) <= 3e-3            # round trip
    assert metrics.sqnr_db(x64, y) >= 50.0         # against the unrounded input too
    X32 = run_fft(storage_round(x64, B.F32), B.F32, B.FORWARD)
    assert metrics.rel_l2(F.fft(storage_round(x64, B.F32)), X32) <= 1e-6


def test_naive_inverse_overflows_and_bfp_does_not():
    """Section III-B: a flat spectrum of magnitude N (the matched product of a
    discrete chirp with its unnormalised filter) has an unnormalised inverse of
    N^2 ~ 1.7e7 at n = 0; stored to FP16 it is Inf.  With the 1/N shift the
    same input gives N = 4096, finite."""
    n = 4096
    spec = np.full((2, n), float(n), dtype=complex)
    naive = run_fft(spec, B.F16_NAIVE, B.INVERSE)
    assert np.isinf(naive.real[:, 0]).all()
    bfp = run_fft(spec, B.F16_BFP, B.INVERSE)
    assert np.all(np.isfinite(bfp))
    ok, worst = fp16_elementwise_ok(bfp, F.ifft(spec))
    assert ok, worst


def test_naive_inverse_matches_bfp_when_in_range():
    x = storage_round(0.01 * synth.complex_gaussian(4, 1024, seed=7), B.F16_BFP)
    naive = run_fft(x, B.F16_NAIVE, B.INVERSE)
    ref = F.ifft(x)
    assert np.all(np.isfinite(naive))
    assert metrics.sqnr_db(ref, naive) >= 50.0


def test_in_place_and_empty_batch():
    import torch
    x = storage_round(synth.complex_gaussian(5, 2048, seed=3), B.F16_BFP)
    got = run_fft(x, B.F16_BFP, B.FORWARD, inplace=True)
    ok, _ = fp16_elementwise_ok(got, F.fft(x))
    assert ok
    plan = B.bfpfft_plan_create(2048, 0, B.F16_BFP, B.FORWARD)
    B.bfpfft_exec(plan, None, None)       # batch 0: a no-op, NULL buffers accepted
    torch.cuda.synchronize()


def test_misaligned_pointer_rejected():
    import torch
    buf = torch.zeros(4096 * 2 + 8, dtype=torch.float16, device="cuda:0")
    plan = B.bfpfft_plan_create(4096, 1, B.F16_BFP, B.FORWARD)
    with pytest.raises(B.BfpfftError) as e:
        B.bfpfft_exec(plan, buf.data_ptr() + 4, buf.data_ptr() + 4)
    assert e.value.status == B.ERR_MISALIGNED


def test_large_batch_sampled_lines():
    """The benchmark's launch configuration (N = 4096, batch 65536, FP16): the
    oracle checks 8 sampled lines of the full-size output."""
    import torch
    n, batch = 4096, 65536
    g = torch.Generator(device="cuda:0").manual_seed(0)
    xin = torch.randn((batch, n, 2), device="cuda:0", generator=g).to(torch.float16)
    out = torch.empty_like(xin)
    plan = B.bfpfft_plan_create(n, batch, B.F16_BFP, B.FORWARD)
    B.bfpfft_exec(plan, xin, out)
    torch.cuda.synchronize()
    rows = [0, 1, 4095, 4096, 30001, 65534, 65535, 12345]
    xs = from_device(xin[rows], B.F16_BFP)
    got = from_device(out[rows], B.F16_BFP)
    ok, worst = fp16_elementwise_ok(got, F.fft(xs))
    assert ok, worst


@pytest.mark.parametrize("dtype,fmt", [(B.E4M3_BFP, "e4m3"), (B.E5M2_BFP, "e5m2")])
@pytest.mark.parametrize("n", [256, 4096, 32768, 65536])
def test_fp8_storage_matches_oracle_rounding(dtype, fmt, n, rows_variant):
    """FP8 storage against the oracle's rounding of the exact scaled values;
    lines of 32768 / 65536 points run four-step (their outputs exchanged as
    rounded FP8 pairs) or as two passes."""
    batch = 16 if n <= 4096 else 3
    x = quant.round_fp8(synth.complex_gaussian(batch, n, seed=n), fmt)
    plan = B.bfpfft_plan_create(n, batch, dtype, B.FORWARD)
    in_exp, out_exp = B.bfpfft_plan_scale_exp(plan)
    assert in_exp == 0 and out_exp == (int(np.log2(n)) + 1) // 2
    got = run_fft(x, dtype, B.FORWARD)                   # stored = true * 2^-out_exp
    exact = F.fft(x) * 2.0 ** -out_exp
    fp8_close(got, exact, fmt)
    # inverse of the stored spectrum back to the input scale
    got_i = run_fft(got, dtype, B.INVERSE)
    exact_i = F.ifft(got * 2.0 ** out_exp)
    fp8_close(got_i, exact_i, fmt)


@pytest.mark.parametrize("variant", ["plain_l2", "plain4_l2"])
@pytest.mark.parametrize("n,batch", [(4096, 1999), (256, 16 * 977 + 5)])
def test_prefetching_variants_over_many_waves(variant, n, batch, monkeypatch):
    """Variants whose CTAs prefetch into L2 the lines of the CTA one resident
    wave later: batches several waves deep with a ragged tail (the last
    prefetches are clipped to the array), sampled lines (all of them at
    N = 256) against the oracle, forward and inverse."""
    import torch
    monkeypatch.setenv("BFPFFT_ROWS", variant)
    x = storage_round(synth.complex_gaussian(batch, n, seed=batch), B.F16_BFP)
    rows = np.arange(batch) if n <= 256 else np.unique(
        np.r_[0, 1, 455, 456, 457, 607, 608, batch // 2, batch - 2, batch - 1,
              np.random.default_rng(5).integers(0, batch, 8)])
    for direction, ref_fn in ((B.FORWARD, F.fft), (B.INVERSE, F.ifft)):
        plan = B.bfpfft_plan_create(n, batch, B.F16_BFP, direction)
        xin = to_device(x, B.F16_BFP)
        out = torch.empty_like(xin)
        B.bfpfft_exec(plan, xin, out)
        torch.cuda.synchronize()
        assert B.bfpfft_device_status() == B.OK
        got = from_device(out[torch.as_tensor(rows, device=out.device)], B.F16_BFP)
        ok, worst = fp16_elementwise_ok(got, ref_fn(x[rows]))
        assert ok, (variant, n, direction, worst)


@pytest.mark.parametrize("variant", [None, "tma"])
@pytest.mark.parametrize("n,batch", [(4096, 300), (65536, 12)])
def test_exec_reads_and_writes_pinned_host_buffers(n, batch, variant, monkeypatch):
    """Pinned host buffers passed straight to bfpfft_exec: the kernels read
    and write them in place over the CPU-GPU link (no staging copies, no L2
    prefetch and no bulk copies from host memory: a bulk-copy variant falls
    back to plain loads); results are bit-identical to device buffers."""
    import torch
    if variant is None:
        monkeypatch.delenv("BFPFFT_ROWS", raising=False)
    else:
        monkeypatch.setenv("BFPFFT_ROWS", variant)
    x = storage_round(synth.complex_gaussian(batch, n, seed=n + 1), B.F16_BFP)
    dev_in = to_device(x, B.F16_BFP)
    host_in = torch.empty(dev_in.shape, dtype=dev_in.dtype, pin_memory=True)
    host_in.copy_(dev_in)
    host_out = torch.empty_like(host_in, pin_memory=True)
    mid = torch.empty_like(dev_in)
    ref_mid, ref_out = torch.empty_like(dev_in), torch.empty_like(dev_in)
    fwd = B.bfpfft_plan_create(n, batch, B.F16_BFP, B.FORWARD)
    inv = B.bfpfft_plan_create(n, batch, B.F16_BFP, B.INVERSE)
    B.bfpfft_exec(fwd, host_in, mid)
    B.bfpfft_exec(inv, mid, host_out)
    B.bfpfft_exec(fwd, dev_in, ref_mid)
    B.bfpfft_exec(inv, ref_mid, ref_out)
    torch.cuda.synchronize()
    assert B.bfpfft_device_status() == B.OK
    assert torch.equal(mid, ref_mid)
    assert torch.equal(host_out.to(dev_in.device), ref_out)
    ok, worst = fp16_elementwise_ok(from_device(mid[:4], B.F16_BFP), F.fft(x[:4]))
    assert ok, worst
