"""Adaptive per-line block exponents on the GPU (Section VIII) against the FP64 oracle.

Bars: every line's exponent equals oracle.bfp.block_exponent of the exact
result (the smallest e with max |Re|, |Im| * 2^-e <= 2^14), except where the
exact maximum lies within FP32 rounding of an exponent boundary (there the
GPU decides in FP32 and one step either way is allowed); mantissas within
half an FP16 ulp of the exact scaled result plus the FP32 arithmetic error;
the stored block maximum in (2^13, 2^14].  Scaling a line by 2^k moves only
its exponent: mantissas bit-identical, exponent + k.  Amplitudes 2^-20 ..
2^20, where the fixed 1/N shift of Eq. 1 overflows FP16, store finite.
"""

import numpy as np
import pytest

from oracle import bfp, metrics, sar
from oracle import fft as F
from paper_2605_28451_gb300 import bfpfft as B
from paper_2605_28451_gb300 import build, synth

from _helpers import fp16_elementwise_ok, from_device, storage_round, to_device

pytestmark = pytest.mark.gpu

AMPS = (-20, -7, 0, 3, 9, 20, -13, 14)


@pytest.fixture(scope="module", autouse=True)
def _lib(cuda_ready):
    build.build()
    B.lib()


def _exps(e):
    import torch
    return torch.from_numpy(np.ascontiguousarray(np.asarray(e, dtype=np.int32))).cuda()


def _near_boundary(y: np.ndarray) -> np.ndarray:
    """Lines whose exact block maximum is within FP32 reach of a power of two,
    where the GPU's FP32 maximum may fall on the other side."""
    m = bfp.block_max(y)
    with np.errstate(divide="ignore"):
        l2 = np.log2(np.where(m > 0, m, 1.0))
    return np.abs(l2 - np.round(l2)) < 1e-5


def check_adaptive(m_gpu, e_gpu, y):
    """The GPU's (mantissas, exponents) against the exact result y [lines][n]."""
    e_ref = bfp.block_exponent(y)
    near = _near_boundary(y)
    assert np.array_equal(e_gpu[~near], e_ref[~near]), (e_gpu[~near], e_ref[~near])
    assert np.all(np.abs(e_gpu[near] - e_ref[near]) <= 1)
    scaled = np.ldexp(y.real, -e_gpu[:, None]) + 1j * np.ldexp(y.imag, -e_gpu[:, None])
    ok, worst = fp16_elementwise_ok(m_gpu, scaled)
    assert ok, worst
    peak = bfp.block_max(m_gpu)
    live = bfp.block_max(y) > 0
    assert np.all(peak[live] <= bfp.DEFAULT_LIMIT)
    # RN can land a maximum just above 2^13 on 2^13 itself (FP16 spacing 8 there)
    assert np.all(peak[live & ~near] >= bfp.DEFAULT_LIMIT / 2)
    assert np.all(e_gpu[~live] == 0) and np.all(peak[~live] == 0)


def amplitude_lines(n, seed=0):
    """N(0, 1) lines scaled by 2^a for a in AMPS, plus one zero line."""
    x = synth.complex_gaussian(len(AMPS), n, seed=seed) * np.exp2(np.array(AMPS, dtype=float))[:, None]
    return np.concatenate([x, np.zeros((1, n), complex)])


@pytest.mark.parametrize("n", [16, 64, 256, 512, 1024, 4096, 16384])
@pytest.mark.parametrize("direction", [B.FORWARD, B.INVERSE])
def test_adaptive_transform(n, direction):
    import torch
    m_in, e_in = bfp.quantize(amplitude_lines(n, seed=n))
    lines = m_in.shape[0]
    p = B.bfpfft_plan_create(n, lines, B.F16_ADAPTIVE, direction)
    x = to_device(m_in, B.F16_BFP)
    out = torch.empty_like(x)
    e_out = _exps(np.zeros(lines))
    B.bfpfft_exec_adaptive(p, x, _exps(e_in), out, e_out)
    torch.cuda.synchronize()
    v = bfp.value(m_in, e_in)
    y = F.fft(v) if direction == B.FORWARD else F.ifft(v)
    check_adaptive(from_device(out, B.F16_BFP), e_out.cpu().numpy().astype(np.int64), y)
    assert B.bfpfft_plan_status(p) == B.OK


@pytest.mark.parametrize("n", [256, 4096])
def test_power_of_two_scaling_moves_only_the_exponent(n):
    """FP32 arithmetic on values scaled by an exact power of two is scaled
    exactly: the mantissas are bit-identical and the exponent moves by k."""
    import torch
    m_in, e_in = bfp.quantize(synth.complex_gaussian(6, n, seed=7))
    x = to_device(m_in, B.F16_BFP)
    p = B.bfpfft_plan_create(n, 6, B.F16_ADAPTIVE, B.FORWARD)
    base_out = torch.empty_like(x)
    base_e = _exps(np.zeros(6))
    B.bfpfft_exec_adaptive(p, x, _exps(e_in), base_out, base_e)
    for k in (-20, -1, 1, 20):
        out = torch.empty_like(x)
        e = _exps(np.zeros(6))
        B.bfpfft_exec_adaptive(p, x, _exps(e_in + k), out, e)
        torch.cuda.synchronize()
        assert torch.equal(out, base_out)
        assert np.array_equal(e.cpu().numpy(), base_e.cpu().numpy() + k)


@pytest.mark.parametrize("amp_log2", [-20, 0, 20])
@pytest.mark.parametrize("n_rg", [256, 4096, 16384])
def test_spectral_adaptive_range_lines(amp_log2, n_rg):
    """Range compression of point-target echoes at amplitude 2^a: the adaptive
    form matches the oracle's adaptive_spectral; the fixed-shift FP16 form
    overflows to Inf at 2^20 (its output peaks at 480 * 2^20)."""
    import torch
    n_az = 12
    sc = synth.point_target_scene(n_az, n_rg, aperture=8, targets=[(6, n_rg // 2, 1.0), (3, n_rg // 4, 0.4)])
    raw = storage_round(sc.raw * 2.0 ** amp_log2, B.F32)
    ref = synth.centred_reference(synth.range_chirp()[: min(480, n_rg // 2)], n_rg)
    h64 = storage_round(sar.matched_filter(storage_round(ref, B.F32), False), B.F32)
    h = to_device(h64, B.F32)
    x = to_device(raw, B.F32)
    out = torch.empty((n_az, n_rg, 2), dtype=torch.float16, device="cuda:0")
    e_out = _exps(np.zeros(n_az))
    B.bfp_spectral_adaptive(x, B.F32, None, h, out, e_out, n_rg, n_az)
    torch.cuda.synchronize()
    m_gpu = from_device(out, B.F16_BFP)
    e_gpu = e_out.cpu().numpy().astype(np.int64)
    y = sar.range_compress(raw, h64)
    check_adaptive(m_gpu, e_gpu, y)
    m_ref, e_ref = bfp.adaptive_spectral(raw, h64)
    assert metrics.sqnr_db(bfp.value(m_ref, e_ref), bfp.value(m_gpu, e_gpu)) >= 55.0
    fixed = torch.empty_like(out)
    B.sar_range_compress(x, B.F32, fixed, B.F16_BFP, h, n_az, n_rg, False)
    torch.cuda.synchronize()
    fixed_finite = bool(torch.isfinite(fixed).all().item())
    assert fixed_finite == (amp_log2 < 20)
    assert np.all(np.isfinite(m_gpu))


def test_chained_spectral_from_adaptive_input():
    """A second forward-multiply-inverse stage fed with the first stage's
    mantissas and exponents (no rescaling in between)."""
    import torch
    n, lines = 1024, len(AMPS) + 1
    x = amplitude_lines(n, seed=3)
    g = synth.complex_gaussian(1, n, seed=4)[0]
    h64 = storage_round(F.fft(g), B.F32)
    h = to_device(h64, B.F32)
    xin = to_device(storage_round(x, B.F32), B.F32)
    mid = torch.empty((lines, n, 2), dtype=torch.float16, device="cuda:0")
    e_mid = _exps(np.zeros(lines))
    B.bfp_spectral_adaptive(xin, B.F32, None, h, mid, e_mid, n, lines)
    out = torch.empty_like(mid)
    e_out = _exps(np.zeros(lines))
    B.bfp_spectral_adaptive(mid, B.F16_ADAPTIVE, e_mid, h, out, e_out, n, lines)
    torch.cuda.synchronize()
    v_mid = bfp.value(from_device(mid, B.F16_BFP), e_mid.cpu().numpy().astype(np.int64))
    y = sar.compress(v_mid, h64, axis=-1)
    check_adaptive(from_device(out, B.F16_BFP), e_out.cpu().numpy().astype(np.int64), y)


def test_plain_exec_rejects_adaptive_plans():
    import torch
    p = B.bfpfft_plan_create(256, 2, B.F16_ADAPTIVE, B.FORWARD)
    x = torch.zeros((2, 256, 2), dtype=torch.float16, device="cuda:0")
    with pytest.raises(B.BfpfftError) as e:
        B.bfpfft_exec(p, x, x)
    assert e.value.status == B.ERR_INVALID_ARG
    q = B.bfpfft_plan_create(256, 2, B.F16_BFP, B.FORWARD)
    with pytest.raises(B.BfpfftError) as e:
        B.bfpfft_exec_adaptive(q, x, None, x, _exps([0, 0]))
    assert e.value.status == B.ERR_INVALID_ARG
