"""Precision modes on the GPU (Section VI's mode list, Table I's pure FP16,
Section IV-C's bfloat16) against the oracle's rounding schedules.

- Pure FP16 and bfloat16 (bfpfft_plan_set_arith): every operation of the
  kernel rounds in the order of oracle.emulate.fft_radix16_rounded, so on
  lengths that are powers of 16 the GPU output equals the emulator's value
  by value (allowed: 1 ulp on 1 in 1000 components, where the emulator's
  FP64 evaluation of a fused multiply-add rounds twice), and the SQNR
  against FP64 equals the emulator's within 0.1 dB -- within the +-1.5 dB
  band of the prediction (60.4 dB pure FP16 at N = 4096).  Other lengths:
  SQNR against FP64 above the mode's floor.
- FP16 operands / FP32 accumulation (the tensor-core DFT blocks): against
  oracle.emulate.fft_radix16_mma, which the GPU matches far more closely
  (>= 6 dB) than either matches the exact DFT.
- The same tensor-core rows with FP8 storage: every stored value is the FP8
  rounding of a value within the tensor-core bound of the exact scaled
  transform, and the SQNR equals the FP32-arithmetic FP8 path's.
"""

import numpy as np
import pytest

from oracle import emulate as E
from oracle import fft as F
from oracle import metrics
from oracle import quant as Q
from paper_2605_28451_gb300 import bfpfft as B
from paper_2605_28451_gb300 import build, synth

from _helpers import fp8_within, from_device, storage_round, to_device

pytestmark = pytest.mark.gpu

ROUND = {B.F16_BFP: Q.round_binary16, B.BF16: Q.round_bfloat16}
ULP_BITS = {B.F16_BFP: 10, B.BF16: 7}


@pytest.fixture(scope="module", autouse=True)
def _lib(cuda_ready):
    build.build()
    B.lib()


def gpu_run(x, n, dtype, direction, arith):
    import torch
    p = B.bfpfft_plan_create(n, x.shape[0], dtype, direction)
    B.bfpfft_plan_set_arith(p, arith)
    xin = to_device(x, dtype)
    out = torch.empty_like(xin)
    B.bfpfft_exec(p, xin, out)
    torch.cuda.synchronize()
    assert B.bfpfft_plan_status(p) == B.OK
    return from_device(out, dtype)


def emulate_rounded(x, dtype, direction):
    """The kernel's schedule: forward, or conj(forward(rn(conj(z) / N))) for the inverse."""
    op = ROUND[dtype]
    if direction == B.FORWARD:
        return E.fft_radix16_rounded(x, op)
    n = x.shape[-1]
    return np.conj(E.fft_radix16_rounded(op(np.conj(x) / n), op))


def assert_same_values(got, emu, fraction_bits, min_equal=0.999):
    for g, e in ((got.real, emu.real), (got.imag, emu.imag)):
        diff = g != e
        assert diff.mean() <= 1.0 - min_equal, diff.mean()
        ulp = np.exp2(np.floor(np.log2(np.maximum(np.abs(e[diff]), 2.0 ** -14))) - fraction_bits)
        assert np.all(np.abs(g[diff] - e[diff]) <= ulp), np.max(np.abs(g[diff] - e[diff]) / ulp)


@pytest.mark.parametrize("dtype,arith", [(B.F16_BFP, B.ARITH_F16), (B.BF16, B.ARITH_BF16)])
@pytest.mark.parametrize("n", [256, 4096])
@pytest.mark.parametrize("direction", [B.FORWARD, B.INVERSE])
def test_16bit_arithmetic_equals_the_rounded_schedule(dtype, arith, n, direction):
    batch = 64 if n == 4096 else 256
    x = storage_round(synth.complex_gaussian(batch, n, seed=0), dtype)
    if direction == B.INVERSE:
        x = storage_round(F.fft(x), dtype)            # a spectrum of the right scale
    got = gpu_run(x, n, dtype, direction, arith)
    emu = emulate_rounded(x, dtype, direction)
    assert_same_values(got, emu, ULP_BITS[dtype])
    exact = F.fft(x) if direction == B.FORWARD else F.ifft(x)
    s_gpu, s_emu = metrics.sqnr_db(exact, got), metrics.sqnr_db(exact, emu)
    assert abs(s_gpu - s_emu) <= 0.1, (s_gpu, s_emu)
    if dtype == B.F16_BFP and n == 4096 and direction == B.FORWARD:
        assert abs(s_gpu - 60.4) <= 1.5        # the emulator's prediction for pure FP16 at 4096
        assert s_gpu >= 55.0


@pytest.mark.parametrize("n", [16, 32, 64, 128, 512, 1024, 2048, 8192, 16384])
@pytest.mark.parametrize("dtype,arith,floor_db", [(B.F16_BFP, B.ARITH_F16, 55.0), (B.BF16, B.ARITH_BF16, 35.0)])
def test_16bit_arithmetic_other_lengths(n, dtype, arith, floor_db):
    batch = max(2, (1 << 18) // n)
    x = storage_round(synth.complex_gaussian(batch, n, seed=1), dtype)
    fwd = gpu_run(x, n, dtype, B.FORWARD, arith)
    assert metrics.sqnr_db(F.fft(x), fwd) >= floor_db
    spec = storage_round(F.fft(x), dtype)
    inv = gpu_run(spec, n, dtype, B.INVERSE, arith)
    assert metrics.sqnr_db(F.ifft(spec), inv) >= floor_db


@pytest.mark.parametrize("direction", [B.FORWARD, B.INVERSE])
def test_fp16_operands_fp32_accumulation_follow_the_mma_schedule(direction):
    n, batch = 4096, 64
    x = storage_round(synth.complex_gaussian(batch, n, seed=2), B.F16_BFP)
    if direction == B.INVERSE:
        x = storage_round(F.fft(x), B.F16_BFP)
    got = gpu_run(x, n, B.F16_BFP, direction, B.ARITH_F16_MUL_F32_ACC)
    if direction == B.FORWARD:
        emu = E.fft_radix16_mma(x)
        exact = F.fft(x)
    else:
        emu = np.conj(E.fft_radix16_mma(np.conj(x) / n))
        exact = F.ifft(x)
    s_emu = metrics.sqnr_db(exact, emu)
    assert metrics.sqnr_db(emu, got) >= s_emu + 6.0
    assert abs(metrics.sqnr_db(exact, got) - s_emu) <= 0.5
    assert metrics.sqnr_db(exact, got) >= 55.0


def test_pure_fp16_naive_inverse_overflows_and_the_shift_does_not():
    n, batch = 4096, 4
    spec = np.full((batch, n), 100.0 + 0.0j)
    naive = gpu_run(spec, n, B.F16_NAIVE, B.INVERSE, B.ARITH_F16)
    assert not np.all(np.isfinite(naive))
    bfp = gpu_run(spec, n, B.F16_BFP, B.INVERSE, B.ARITH_F16)
    assert np.all(np.isfinite(bfp))
    assert metrics.sqnr_db(F.ifft(spec), bfp) >= 50.0


def test_set_arith_combinations():
    def status(n, dtype, arith, direction=B.FORWARD):
        p = B.bfpfft_plan_create(n, 2, dtype, direction)
        try:
            B.bfpfft_plan_set_arith(p, arith)
        except B.BfpfftError as e:
            return e.status
        return B.OK
    assert status(4096, B.F16_BFP, B.ARITH_F16) == B.OK
    assert status(16384, B.F16_NAIVE, B.ARITH_F16) == B.OK
    assert status(32768, B.F16_BFP, B.ARITH_F16) == B.ERR_UNSUPPORTED
    assert status(4096, B.F32, B.ARITH_F16) == B.ERR_UNSUPPORTED
    assert status(4096, B.E4M3_BFP, B.ARITH_F16) == B.ERR_UNSUPPORTED
    assert status(4096, B.F16_BFP, B.ARITH_F16_MUL_F32_ACC) == B.OK
    assert status(8192, B.F16_BFP, B.ARITH_F16_MUL_F32_ACC) == B.ERR_UNSUPPORTED
    assert status(4096, B.E4M3_BFP, B.ARITH_F16_MUL_F32_ACC) == B.OK
    assert status(4096, B.E5M2_BFP, B.ARITH_F16_MUL_F32_ACC, B.INVERSE) == B.OK
    assert status(1024, B.E4M3_BFP, B.ARITH_F16_MUL_F32_ACC) == B.ERR_UNSUPPORTED
    assert status(4096, B.F32, B.ARITH_F16_MUL_F32_ACC) == B.ERR_UNSUPPORTED
    assert status(4096, B.BF16, B.ARITH_F32) == B.ERR_UNSUPPORTED
    assert status(4096, B.F16_BFP, B.ARITH_BF16) == B.ERR_UNSUPPORTED
    assert status(4096, B.F16_BFP, 9) == B.ERR_INVALID_ARG
    u = B.bfpfft_plan_create_many([256, 4096], [0, 256], B.F16_BFP, B.FORWARD)
    with pytest.raises(B.BfpfftError) as e:
        B.bfpfft_plan_set_arith(u, B.ARITH_F16)
    assert e.value.status == B.ERR_UNSUPPORTED


def _tc_plan(n, batch, direction):
    p = B.bfpfft_plan_create(n, batch, B.F16_BFP, direction)
    B.bfpfft_plan_set_arith(p, B.ARITH_F16_MUL_F32_ACC)
    return p


def _mma_inverse(x):
    return np.conj(E.fft_radix16_mma(np.conj(x) / x.shape[-1]))


@pytest.mark.parametrize("batch,rows", [
    (65536, [0, 1, 1215, 1216, 2431, 30001, 65534, 65535]),   # the benchmark's launch: 53-54 lines per CTA
    (2 * 1216 + 7, [0, 6, 7, 1215, 1216, 1222, 2431, 2438]),  # ragged: CTAs take 2 or 3 lines
])
def test_tensor_core_rows_at_the_benchmark_configuration(batch, rows):
    """The benchmark's timed step (N = 4096, FP16 operands, FP32 accumulation
    on the tensor cores, persistent CTAs walking many lines): sampled lines of
    the forward output and of the shifted inverse of that output against the
    FP64 oracle (SQNR >= 55 dB) and against oracle.emulate.fft_radix16_mma,
    which the GPU matches far more closely than either matches the exact
    transform."""
    import torch
    n = 4096
    g = torch.Generator(device="cuda:0").manual_seed(7)
    xin = torch.randn((batch, n, 2), device="cuda:0", generator=g).to(torch.float16)
    y = torch.empty_like(xin)
    z = torch.empty_like(xin)
    fwd, inv = _tc_plan(n, batch, B.FORWARD), _tc_plan(n, batch, B.INVERSE)
    B.bfpfft_exec(fwd, xin, y)
    B.bfpfft_exec(inv, y, z)
    torch.cuda.synchronize()
    assert B.bfpfft_plan_status(fwd) == B.OK and B.bfpfft_plan_status(inv) == B.OK
    x = from_device(xin[rows], B.F16_BFP)
    got_f = from_device(y[rows], B.F16_BFP)
    got_i = from_device(z[rows], B.F16_BFP)
    for got, exact, emu in ((got_f, F.fft(x), E.fft_radix16_mma(x)),
                            (got_i, F.ifft(got_f), _mma_inverse(got_f))):
        s_emu = metrics.sqnr_db(exact, emu)
        assert metrics.sqnr_db(exact, got) >= 55.0
        assert abs(metrics.sqnr_db(exact, got) - s_emu) <= 0.5
        assert metrics.sqnr_db(emu, got) >= s_emu + 6.0
        for line in range(len(rows)):            # no line left behind by the persistent loop
            assert metrics.sqnr_db(exact[line], got[line]) >= 55.0, rows[line]


def test_tensor_core_rows_host_buffers_and_in_place():
    """Pinned host input (no L2 prefetch of host memory) and in-place calls
    give the same bits as device buffers out of place."""
    import torch
    n, batch = 4096, 1300
    x = storage_round(synth.complex_gaussian(batch, n, seed=11), B.F16_BFP)
    dev_in = to_device(x, B.F16_BFP)
    host_in = torch.empty(dev_in.shape, dtype=dev_in.dtype, pin_memory=True)
    host_in.copy_(dev_in)
    fwd, inv = _tc_plan(n, batch, B.FORWARD), _tc_plan(n, batch, B.INVERSE)
    ref_y, ref_z = torch.empty_like(dev_in), torch.empty_like(dev_in)
    B.bfpfft_exec(fwd, dev_in, ref_y)
    B.bfpfft_exec(inv, ref_y, ref_z)
    host_y = torch.empty_like(dev_in)
    B.bfpfft_exec(fwd, host_in, host_y)
    inplace = dev_in.clone()
    B.bfpfft_exec(fwd, inplace, inplace)
    B.bfpfft_exec(inv, inplace, inplace)
    torch.cuda.synchronize()
    assert B.bfpfft_plan_status(fwd) == B.OK and B.bfpfft_plan_status(inv) == B.OK
    assert torch.equal(host_y, ref_y)
    assert torch.equal(inplace, ref_z)


def test_tensor_core_rows_graph_replay():
    """A tensor-core plan replayed through its CUDA graph gives the bits of a
    direct call, on the first replay and after the input changes."""
    import torch
    n, batch = 4096, 700
    fwd = _tc_plan(n, batch, B.FORWARD)
    x = to_device(storage_round(synth.complex_gaussian(batch, n, seed=21), B.F16_BFP), B.F16_BFP)
    direct, graphed = torch.empty_like(x), torch.empty_like(x)
    B.bfpfft_exec(fwd, x, direct)
    B.bfpfft_exec_graph(fwd, x, graphed)
    torch.cuda.synchronize()
    assert torch.equal(direct, graphed)
    x.copy_(to_device(storage_round(synth.complex_gaussian(batch, n, seed=22), B.F16_BFP), B.F16_BFP))
    B.bfpfft_exec(fwd, x, direct)
    B.bfpfft_exec_graph(fwd, x, graphed)
    torch.cuda.synchronize()
    assert torch.equal(direct, graphed)
    assert B.bfpfft_plan_status(fwd) == B.OK


# Error of the tensor-core rows before their final rounding: FP16 rounding of
# the operands at each of the three passes (and of the DFT-16 coefficients),
# noise of rms about 1.1 * 2^-11 rms(y) per component; 8 * 2^-11 rms(y) is
# more than 7 sigma (the FP16-row bound without its final FP16 rounding).
TC_RMS_BOUND = 8 * 2.0 ** -11


@pytest.mark.parametrize("dtype,fmt", [(B.E4M3_BFP, "e4m3"), (B.E5M2_BFP, "e5m2")])
@pytest.mark.parametrize("batch", [1, 7, 2 * 1216 + 7])
def test_fp8_storage_on_the_tensor_cores(dtype, fmt, batch):
    """FP8 storage (Section VII) with FP16 operands and FP32 accumulation on
    the tensor cores, N = 4096, forward and the inverse of the stored
    spectrum; the stored scale is the FP8 plan's (2^-6 forward, 2^6 back)."""
    n = 4096
    x = Q.round_fp8(synth.complex_gaussian(batch, n, seed=40 + batch), fmt)
    p = B.bfpfft_plan_create(n, batch, dtype, B.FORWARD)
    _, s = B.bfpfft_plan_scale_exp(p)
    assert s == 6
    got = gpu_run(x, n, dtype, B.FORWARD, B.ARITH_F16_MUL_F32_ACC)
    ref = gpu_run(x, n, dtype, B.FORWARD, B.ARITH_F32)
    exact = F.fft(x) * 2.0 ** -s
    assert fp8_within(got, exact, fmt, 1e-5, TC_RMS_BOUND) <= 0.05
    assert abs(metrics.sqnr_db(exact, got) - metrics.sqnr_db(exact, ref)) <= 0.05
    got_i = gpu_run(got, n, dtype, B.INVERSE, B.ARITH_F16_MUL_F32_ACC)
    ref_i = gpu_run(got, n, dtype, B.INVERSE, B.ARITH_F32)
    exact_i = F.ifft(got * 2.0 ** s)
    assert fp8_within(got_i, exact_i, fmt, 1e-5, TC_RMS_BOUND) <= 0.05
    assert abs(metrics.sqnr_db(exact_i, got_i) - metrics.sqnr_db(exact_i, ref_i)) <= 0.05


def test_fp8_tensor_core_rows_host_buffers_and_in_place():
    """FP8 tensor-core rows from pinned host memory and in place give the bits
    of device buffers out of place."""
    import torch
    n, batch = 4096, 1300
    x = Q.round_fp8(synth.complex_gaussian(batch, n, seed=12), "e4m3")
    dev_in = to_device(x, B.E4M3_BFP)
    host_in = torch.empty(dev_in.shape, dtype=dev_in.dtype, pin_memory=True)
    host_in.copy_(dev_in)
    fwd = B.bfpfft_plan_create(n, batch, B.E4M3_BFP, B.FORWARD)
    B.bfpfft_plan_set_arith(fwd, B.ARITH_F16_MUL_F32_ACC)
    ref, from_host = torch.empty_like(dev_in), torch.empty_like(dev_in)
    B.bfpfft_exec(fwd, dev_in, ref)
    B.bfpfft_exec(fwd, host_in, from_host)
    inplace = dev_in.clone()
    B.bfpfft_exec(fwd, inplace, inplace)
    torch.cuda.synchronize()
    assert B.bfpfft_plan_status(fwd) == B.OK
    assert torch.equal(from_host, ref) and torch.equal(inplace, ref)
