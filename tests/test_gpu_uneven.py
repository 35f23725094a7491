"""GPU parity of the uneven-batch persistent launch (bfpfft_plan_create_many).

Every line of a small mixed batch is checked against the FP64 oracle with the
same bars as the uniform transforms (FP32: relative L2 <= 1e-6; FP16-BFP:
half an FP16 ulp plus the FP32 arithmetic; FP8: the oracle's rounding of the
same value up to a rounding-boundary tie).  The config-4 workload (20,000
transforms, lengths 256 ... 65536 with Zipf weights, about 2^28 points) runs
at full size and the oracle checks sampled lines of every length.  Graph
replays must reproduce the direct launch bit for bit.
"""

import numpy as np
import pytest

from oracle import fft as F
from oracle import metrics, quant
from paper_2605_28451_gb300 import bfpfft as B
from paper_2605_28451_gb300 import build, synth

from _helpers import fp8_close, fp16_elementwise_ok, from_device, storage_round, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib(cuda_ready):
    build.build()
    B.lib()


def packed(lengths, dtype, seed):
    data, offsets = synth.uneven_batch(lengths, seed=seed)
    if dtype in (B.E4M3_BFP, B.E5M2_BFP):
        data = quant.round_fp8(data, "e4m3" if dtype == B.E4M3_BFP else "e5m2")
    return storage_round(data, dtype), offsets


# Schedule flags the long_lines fixture applies to every uneven plan a test makes.
SCHEDULE = {"flags": 0}


def create_many(lengths, offsets, dtype, direction):
    plan = B.bfpfft_plan_create_many(lengths, offsets, dtype, direction)
    flags = SCHEDULE["flags"]
    if flags:
        if dtype != B.F16_BFP:
            flags &= ~B.MANY_FP16_ROWS
        B.bfpfft_plan_set_many_schedule(plan, 0, flags)
    return plan


def run_many(data, lengths, offsets, dtype, direction, graph=False, reps=1):
    import torch
    plan = create_many(lengths, offsets, dtype, direction)
    x = to_device(data, dtype)
    y = torch.empty_like(x)
    for _ in range(reps):
        (B.bfpfft_exec_graph if graph else B.bfpfft_exec)(plan, x, y)
    torch.cuda.synchronize()
    assert B.bfpfft_device_status() == B.OK
    return from_device(y, dtype), plan


MIXED = [65536, 16, 4096, 256, 16384, 1024, 8192, 32, 4096, 32768, 512, 2048, 64, 128, 65536, 256, 4096] * 2


@pytest.fixture(params=["fourstep", "twopass", "fourstep_h16", "per_length", "per_length_h16"])
def long_lines(request, monkeypatch):
    """Lines of 32768 / 65536 points inside the persistent kernel (four-step) or
    split off to the two-pass kernels (BFPFFT_ROWS=twopass forces the split);
    fourstep_h16: four-step lines with their row exchange in FP16 words
    (BFPFFT_ROWS naming an FP16-exchange variant forces it); per_length: one
    dense-row launch per length over its listed lines (schedule flag), with
    FP32 or FP16 (per_length_h16) four-step row exchanges."""
    monkeypatch.delenv("BFPFFT_ROWS", raising=False)
    if request.param == "twopass":
        monkeypatch.setenv("BFPFFT_ROWS", "twopass")
    elif request.param == "fourstep_h16":
        monkeypatch.setenv("BFPFFT_ROWS", "h16_l2")
    elif request.param == "per_length":
        monkeypatch.setitem(SCHEDULE, "flags", B.MANY_PER_LENGTH)
    elif request.param == "per_length_h16":
        monkeypatch.setitem(SCHEDULE, "flags", B.MANY_PER_LENGTH | B.MANY_FP16_ROWS)
    return request.param


def fp16_line_ok(g, ref, n, long_lines):
    """FP16 parity of one line.  The two-pass intermediate (lines of 32768
    points or more) and the FP16 row exchange of four-step lines (8192 points
    or more) are one more FP16 storage point: the FP16-exchange bound of the
    uniform row tests.  One launch per length runs lines of 8192 and 16384
    points on one CTA (FP32 exchanges), so there only lines of 32768 points or
    more carry the FP16 row exchange."""
    if ((long_lines == "twopass" and n >= 32768) or (long_lines == "fourstep_h16" and n >= 8192)
            or (long_lines == "per_length_h16" and n >= 32768)):
        rms = np.sqrt(np.mean(np.abs(ref) ** 2))
        bound = 2.0 ** -11 * (np.abs(ref) + 6.0 * rms)
        return (np.all(np.abs(g.real - ref.real) <= bound) and np.all(np.abs(g.imag - ref.imag) <= bound)
                and metrics.sqnr_db(ref, g) >= 55.0), None
    return fp16_elementwise_ok(g, ref)


@pytest.mark.parametrize("direction", [B.FORWARD, B.INVERSE])
@pytest.mark.parametrize("dtype", [B.F32, B.F16_BFP])
def test_mixed_lengths_every_line(dtype, direction, long_lines):
    lengths = np.array(MIXED)
    data, offsets = packed(lengths, dtype, seed=31)
    got, plan = run_many(data, lengths, offsets, dtype, direction)
    tasks, clusters = B.bfpfft_plan_info(plan)
    assert tasks > 0 and clusters > 0
    for n, o in zip(lengths, offsets):
        x = data[o:o + n]
        ref = F.fft(x) if direction == B.FORWARD else F.ifft(x)
        g = got[o:o + n]
        if dtype == B.F32:
            assert metrics.rel_l2(ref, g) <= 1e-6, n
        else:
            ok, worst = fp16_line_ok(g, ref, n, long_lines)
            assert ok, (n, worst)


@pytest.mark.parametrize("dtype,fmt", [(B.E4M3_BFP, "e4m3"), (B.E5M2_BFP, "e5m2")])
def test_fp8_mixed_lengths(dtype, fmt, long_lines):
    lengths = np.array([4096, 256, 65536, 1024, 16384, 4096])
    data, offsets = packed(lengths, dtype, seed=32)
    got, _ = run_many(data, lengths, offsets, dtype, B.FORWARD)
    for n, o in zip(lengths, offsets):
        s = (int(np.log2(n)) + 1) // 2
        exact = F.fft(data[o:o + n]) * 2.0 ** -s
        fp8_close(got[o:o + n], exact, fmt)


def test_graph_replay_matches_direct_launch(long_lines):
    lengths = np.array(MIXED)
    data, offsets = packed(lengths, B.F16_BFP, seed=33)
    direct, _ = run_many(data, lengths, offsets, B.F16_BFP, B.FORWARD)
    replay, _ = run_many(data, lengths, offsets, B.F16_BFP, B.FORWARD, graph=True, reps=3)
    assert np.array_equal(direct.view(np.float64), replay.view(np.float64))


def test_empty_uneven_plan():
    plan = B.bfpfft_plan_create_many([], [], B.F16_BFP, B.FORWARD)
    B.bfpfft_exec(plan, None, None)


def test_uneven_plan_rejects_bad_lengths():
    with pytest.raises(B.BfpfftError) as e:
        B.bfpfft_plan_create_many([4096, 100], [0, 4096], B.F16_BFP, B.FORWARD)
    assert e.value.status == B.ERR_UNSUPPORTED
    with pytest.raises(B.BfpfftError) as e:
        B.bfpfft_plan_create_many([4096], [0], B.F16_NAIVE, B.FORWARD)
    assert e.value.status == B.ERR_UNSUPPORTED


def test_config4_full_size_sampled_lines(long_lines):
    """20,000 transforms, lengths from {256, 1024, 4096, 16384, 65536} with Zipf
    weights (seed 3), FP16-BFP, one persistent launch through a CUDA graph (with
    the two-pass split: the two-pass kernels, then the persistent launch)."""
    import torch
    lengths = synth.uneven_lengths(20000, seed=3)
    offsets = np.zeros_like(lengths)
    offsets[1:] = np.cumsum(lengths)[:-1]
    total = int(lengths.sum())
    assert 2 ** 27 < total < 2 ** 29
    g = torch.Generator(device="cuda:0").manual_seed(3)
    x = torch.randn((total, 2), device="cuda:0", generator=g).to(torch.float16)
    y = torch.empty_like(x)
    plan = create_many(lengths, offsets, B.F16_BFP, B.FORWARD)
    B.bfpfft_exec_graph(plan, x, y)
    torch.cuda.synchronize()
    assert B.bfpfft_device_status() == B.OK
    rng = np.random.default_rng(7)
    for n in (256, 1024, 4096, 16384, 65536):
        idx = np.flatnonzero(lengths == n)
        for i in rng.choice(idx, 2, replace=False):
            o = int(offsets[i])
            xs = from_device(x[o:o + n], B.F16_BFP)
            ys = from_device(y[o:o + n], B.F16_BFP)
            ok, worst = fp16_line_ok(ys, F.fft(xs), n, long_lines)
            assert ok, (n, worst)


def test_tuner_uniform_and_uneven(tmp_path, monkeypatch):
    """bfpfft_plan_tune picks a candidate, stores it in the cache file, and a
    plan created with BFPFFT_TUNE=cached reuses it; results stay within the
    usual parity bars whichever candidate wins."""
    import torch
    monkeypatch.setenv("BFPFFT_TUNE_CACHE", str(tmp_path / "tune.txt"))
    monkeypatch.delenv("BFPFFT_ROWS", raising=False)
    plan = B.bfpfft_plan_create(4096, 512, B.F16_BFP, B.FORWARD)
    chosen, ms = B.bfpfft_plan_tune(plan, allow_fp16_exchange=False)
    assert chosen in (0, 1, 2, 5, 9, 10, 11) and ms > 0
    text = (tmp_path / "tune.txt").read_text()
    assert "/n4096/" in text and f" {chosen} " in text
    x = storage_round(synth.complex_gaussian(512, 4096, seed=9), B.F16_BFP)
    xin = to_device(x, B.F16_BFP)
    y = torch.empty_like(xin)
    B.bfpfft_exec(plan, xin, y)
    torch.cuda.synchronize()
    ok, worst = fp16_elementwise_ok(from_device(y, B.F16_BFP)[:8], F.fft(x[:8]))
    assert ok, worst
    lengths = np.array(MIXED)
    data, offsets = packed(lengths, B.F16_BFP, seed=34)
    many = B.bfpfft_plan_create_many(lengths, offsets, B.F16_BFP, B.FORWARD)
    code, _ = B.bfpfft_plan_tune(many)          # clusters + 65536 * (two-pass long lines, or 4: per length)
    assert 1 <= (code & 0xffff) <= B.bfpfft_plan_info(many)[1] and (code >> 16) in (0, 1, 4)
    got, _ = run_many(data, lengths, offsets, B.F16_BFP, B.FORWARD)
    tuned = B.bfpfft_plan_create_many(lengths, offsets, B.F16_BFP, B.FORWARD)
    code_t, _ = B.bfpfft_plan_tune(tuned)
    x_many = to_device(data, B.F16_BFP)
    y_many = torch.empty_like(x_many)
    B.bfpfft_exec(tuned, x_many, y_many)
    torch.cuda.synchronize()
    out = from_device(y_many, B.F16_BFP)
    for n, o in zip(lengths, offsets):
        ok, worst = fp16_line_ok(out[o:o + n], F.fft(data[o:o + n]), n,
                                 "twopass" if (code_t >> 16) & 1 else "fourstep")
        assert ok, (n, worst)
    long_plan = B.bfpfft_plan_create(65536, 8, B.F16_BFP, B.FORWARD)
    chosen_long, _ = B.bfpfft_plan_tune(long_plan)
    assert chosen_long in (11, 15)                # the four-step kernel or the two-pass kernels
    monkeypatch.setenv("BFPFFT_TUNE", "cached")
    again = B.bfpfft_plan_create(4096, 512, B.F16_BFP, B.FORWARD)
    B.bfpfft_exec(again, xin, y)
    torch.cuda.synchronize()
    ok, worst = fp16_elementwise_ok(from_device(y, B.F16_BFP)[:8], F.fft(x[:8]))
    assert ok, worst


def test_tuner_with_fp16_exchanges_allowed(tmp_path, monkeypatch):
    """With allow_fp16_exchange the tuner also times the FP16-exchange and
    tensor-core variants; whichever wins, the plan's results stay within the
    FP16 budget (SQNR against the FP64 oracle well above the 55 dB bar)."""
    import torch
    monkeypatch.setenv("BFPFFT_TUNE_CACHE", str(tmp_path / "tune.txt"))
    monkeypatch.delenv("BFPFFT_ROWS", raising=False)
    plan = B.bfpfft_plan_create(4096, 512, B.F16_BFP, B.FORWARD)
    chosen, ms = B.bfpfft_plan_tune(plan, allow_fp16_exchange=True)
    assert chosen in (0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12) and ms > 0
    x = storage_round(synth.complex_gaussian(512, 4096, seed=10), B.F16_BFP)
    xin = to_device(x, B.F16_BFP)
    y = torch.empty_like(xin)
    B.bfpfft_exec(plan, xin, y)
    torch.cuda.synchronize()
    assert B.bfpfft_device_status() == B.OK
    got = from_device(y, B.F16_BFP)[:16]
    assert metrics.sqnr_db(F.fft(x[:16]), got) >= 60.0, chosen
    # Uneven plan: the FP16 row exchange of four-step lines is a candidate too
    # (code bit 17); every line stays within the FP16 budget of its mode.
    lengths = np.array(MIXED)
    data, offsets = packed(lengths, B.F16_BFP, seed=35)
    many = B.bfpfft_plan_create_many(lengths, offsets, B.F16_BFP, B.FORWARD)
    code, _ = B.bfpfft_plan_tune(many, allow_fp16_exchange=True)
    assert 1 <= (code & 0xffff) <= B.bfpfft_plan_info(many)[1] and (code >> 16) in (0, 1, 2, 3, 4, 6)
    x_many = to_device(data, B.F16_BFP)
    y_many = torch.empty_like(x_many)
    B.bfpfft_exec(many, x_many, y_many)
    torch.cuda.synchronize()
    assert B.bfpfft_device_status() == B.OK
    out = from_device(y_many, B.F16_BFP)
    flags = code >> 16
    mode = {0: "fourstep", 1: "twopass", 2: "fourstep_h16", 3: "fourstep_h16", 4: "per_length",
            6: "per_length_h16"}[flags]
    for n, o in zip(lengths, offsets):
        ok, worst = fp16_line_ok(out[o:o + n], F.fft(data[o:o + n]), n, mode)
        assert ok, (n, code, worst)
    # Uniform lines of 65536 points: four-step (FP32 or FP16 row exchange) or two-pass.
    long_plan = B.bfpfft_plan_create(65536, 8, B.F16_BFP, B.FORWARD)
    chosen_long, _ = B.bfpfft_plan_tune(long_plan, allow_fp16_exchange=True)
    assert chosen_long in (11, 12, 15)
    xl = storage_round(synth.complex_gaussian(8, 65536, seed=11), B.F16_BFP)
    xl_d = to_device(xl, B.F16_BFP)
    yl = torch.empty_like(xl_d)
    B.bfpfft_exec(long_plan, xl_d, yl)
    torch.cuda.synchronize()
    assert B.bfpfft_device_status() == B.OK
    gl = from_device(yl, B.F16_BFP)
    for i in range(8):
        ok, worst = fp16_line_ok(gl[i], F.fft(xl[i]), 65536, "fourstep" if chosen_long == 11 else "fourstep_h16")
        assert ok, (chosen_long, worst)
