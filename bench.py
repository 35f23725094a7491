#!/usr/bin/env python3
"""Benchmark: batched FP16 block-floating-point FFT GFLOPS and HBM roofline on GB300.

Workload (the Table II transform widened past L2): complex transforms of
length 4096, FP16-BFP storage (half2), batch 65536 (1 GiB in, 1 GiB out, so
no L2 flush is needed between steps).  One step = forward FFT + inverse FFT
with the 1/N block shift (two launches of the row kernel), GFLOPS =
2 * 5 N log2 N * batch / t (Section V's convention).

Beside the headline line the JSON carries: the same workload in FP32
storage, the exact Table II size (batch 256, L2 flushed between steps), SAR
range compression (1024 x 4096) and the full 4096 x 4096 range-Doppler image,
the FP16 SQNR against the FP32 path, the roofline of the dominant kernel,
the oracle timed on the host cores, an end-to-end number through the C ABI
with host buffers, and the SM clocks sampled during the timed region.

--impl reference times the FP64 oracle (test infrastructure) on the host
cores on a bounded sample of the same workload and prints the same line.

Multi-GPU: one process per GPU (torchrun); every rank runs the same batch
(weak scaling, replicas: the transforms are independent, no collective).
"""

from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N = 4096
BATCH = 65536
LOG2N = 12
FLOPS_PER_TRANSFORM = 5 * N * LOG2N
FALLBACK_HBM_GBS = 6800.0


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _max_over_ranks(value: float, dist, device) -> float:
    """The largest value over all ranks (for times: the slowest rank's), or
    the value itself when no process group is running."""
    import torch
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _job_value(world: int, flops_per_rank_step: float, t_ms: float) -> float:
    """Whole-job GFLOPS: every rank runs its own replica of the workload (no
    data-path collective), so the job does `world` times one rank's work in
    the slowest rank's time."""
    return world * flops_per_rank_step / (t_ms * 1e-3) / 1e9


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


# Sources of the headline row kernel: its DRAM traffic in profiles/ is valid
# only while these are unchanged.
KERNEL_SOURCES = ("fft_rows.cuh", "complex_ops.cuh", "storage.cuh", "async_copy.cuh", "rows_f16.cu", "tc_fft.cuh")


def _kernel_source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2605_28451_gb300", "csrc")
    for f in KERNEL_SOURCES:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def _profiled_traffic(kernel_tag: str):
    """DRAM bytes per launch recorded by an ncu capture in profiles/, or None
    when no capture exists or the kernel sources changed since it was taken."""
    p = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(p):
        return None
    want = _kernel_source_hash()
    for line in open(p):
        parts = line.split()
        if len(parts) >= 4 and parts[0] == kernel_tag and parts[1] == want:
            return float(parts[3])
    return None


class ClockSampler:
    """nvidia-smi samples (SM clock, throttle reasons) during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                     timeout=5).stdout.strip()
                if out:
                    self.samples.append([x.strip() for x in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.1)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[2 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def _events_time(fn, steps, stream, per_launch=None):
    """Run fn() `steps` times between events; returns total ms."""
    import torch
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for _ in range(steps):
        fn()
    end.record(stream)
    end.synchronize()
    return start.elapsed_time(end)


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2605_28451_gb300 import bfpfft as B
    from paper_2605_28451_gb300 import build as _b

    world, rank, local = _dist()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    _b.build()
    B.lib()
    stream = torch.cuda.current_stream()
    batch = args.batch

    # ---- inputs resident in HBM (seeded, synthetic: re, im ~ N(0, 1)) -------------
    g = torch.Generator(device=dev).manual_seed(1000 + rank)
    x16 = torch.randn((batch, N, 2), device=dev, generator=g).to(torch.float16)
    y16 = torch.empty_like(x16)
    z16 = torch.empty_like(x16)
    fwd16 = _tc_plan(B, batch, B.FORWARD)
    inv16 = _tc_plan(B, batch, B.INVERSE)

    def step16(evs=None):
        if evs is not None:
            evs[0].record(stream)
        B.bfpfft_exec(fwd16, x16, y16, stream)
        if evs is not None:
            evs[1].record(stream)
        B.bfpfft_exec(inv16, y16, z16, stream)
        if evs is not None:
            evs[2].record(stream)

    events = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    with ClockSampler(local) as clocks:
        for _ in range(args.warmup):
            step16()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for i in range(args.steps):
            step16(events[i])
        t_end.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
    fwd_ms = [e[0].elapsed_time(e[1]) for e in events]
    inv_ms = [e[1].elapsed_time(e[2]) for e in events]
    step_ms = [e[0].elapsed_time(e[2]) for e in events]
    t_ms = _max_over_ranks(t_start.elapsed_time(t_end) / args.steps, dist, dev)
    flops_step = 2.0 * FLOPS_PER_TRANSFORM * batch
    value = _job_value(world, flops_step, t_ms)

    # ---- SQNR of the FP16 path against the FP32 path on the same input ----------
    x32 = torch.view_as_complex(x16[:256].float().contiguous())
    y32 = torch.empty_like(x32)
    p32 = B.bfpfft_plan_create(N, 256, B.F32, B.FORWARD)
    B.bfpfft_exec(p32, x32, y32, stream)
    y16c = torch.view_as_complex(y16[:256].float().contiguous()).to(torch.complex128)
    r = y32.to(torch.complex128)
    alpha = (torch.vdot(y16c.flatten(), r.flatten()).real / torch.vdot(y16c.flatten(), y16c.flatten()).real)
    sqnr16 = float(10 * torch.log10((r.abs() ** 2).sum() / ((r - alpha * y16c).abs() ** 2).sum()))

    # ---- FP32 storage on the same workload ---------------------------------------
    xf = torch.view_as_complex(x16.float().contiguous())
    del x32, y32
    yf = torch.empty_like(xf)
    zf = torch.empty_like(xf)
    fwd32 = B.bfpfft_plan_create(N, batch, B.F32, B.FORWARD)
    inv32 = B.bfpfft_plan_create(N, batch, B.F32, B.INVERSE)

    def step32():
        B.bfpfft_exec(fwd32, xf, yf, stream)
        B.bfpfft_exec(inv32, yf, zf, stream)

    for _ in range(3):
        step32()
    k32 = max(3, args.steps // 2)
    t32 = _events_time(step32, k32, stream) / k32
    gflops32 = flops_step / (t32 * 1e-3) / 1e9
    del xf, yf, zf

    # ---- FP8 (E4M3) storage on the same workload ------------------------------------
    x8 = x16.to(torch.float8_e4m3fn).view(torch.uint8)
    y8, z8 = torch.empty_like(x8), torch.empty_like(x8)
    fwd8 = B.bfpfft_plan_create(N, batch, B.E4M3_BFP, B.FORWARD)
    inv8 = B.bfpfft_plan_create(N, batch, B.E4M3_BFP, B.INVERSE)

    def step8():
        B.bfpfft_exec(fwd8, x8, y8, stream)
        B.bfpfft_exec(inv8, y8, z8, stream)

    for _ in range(3):
        step8()
    t8 = _events_time(step8, k32, stream) / k32
    fp8_entry = {"gflops": round(flops_step / (t8 * 1e-3) / 1e9, 1), "ms_per_step": round(t8, 4),
                 "alg_gbs": round(2 * 4.0 * N * batch / (t8 * 1e-3) / 1e9, 1),
                 "dtype": "E4M3 storage (4 B per point), f32 arithmetic"}
    # The same FP8 storage with FP16 operands and FP32 accumulation on the tensor cores.
    for p8 in (fwd8, inv8):
        B.bfpfft_plan_set_arith(p8, B.ARITH_F16_MUL_F32_ACC)
    for _ in range(3):
        step8()
    t8t = _events_time(step8, k32, stream) / k32
    fp8_tc_entry = {"gflops": round(flops_step / (t8t * 1e-3) / 1e9, 1), "ms_per_step": round(t8t, 4),
                    "alg_gbs": round(2 * 4.0 * N * batch / (t8t * 1e-3) / 1e9, 1),
                    "dtype": "E4M3 storage (4 B per point), FP16 operands / FP32 accumulation (tensor cores)"}
    del x8, y8, z8

    # ---- Table II size exactly: N = 4096, batch 256, L2 flushed between steps ------
    small_x = x16[:256].contiguous()
    small_y = torch.empty_like(small_x)
    small_z = torch.empty_like(small_x)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def small_batch(pf, pi):
        small = []
        for i in range(30 + 5):
            flush.fill_(i & 0xFF)
            e0.record(stream)
            B.bfpfft_exec(pf, small_x, small_y, stream)
            B.bfpfft_exec(pi, small_y, small_z, stream)
            e1.record(stream)
            e1.synchronize()
            if i >= 5:
                small.append(e0.elapsed_time(e1))
        return statistics.median(small)

    t_small = small_batch(_tc_plan(B, 256, B.FORWARD), _tc_plan(B, 256, B.INVERSE))
    gflops_small = 2.0 * FLOPS_PER_TRANSFORM * 256 / (t_small * 1e-3) / 1e9
    # the FP32-arithmetic kernel (one 256-thread CTA per line) has the shorter per-line chain
    t_small32 = small_batch(B.bfpfft_plan_create(N, 256, B.F16_BFP, B.FORWARD),
                            B.bfpfft_plan_create(N, 256, B.F16_BFP, B.INVERSE))
    gflops_small32 = 2.0 * FLOPS_PER_TRANSFORM * 256 / (t_small32 * 1e-3) / 1e9
    del flush

    # ---- precision modes and adaptive exponents on the same workload ------------------
    modes = _bench_precision_modes(B, torch, dev, stream, x16, flops_step, k32)

    # ---- batch sweep of the FP16-BFP transform (Table II's batch 256 up to 2 GiB) -----
    sweep = _bench_batch_sweep(B, torch, dev, stream)

    # ---- SAR: range compression 1024 x 4096 and the 4096 x 4096 image ---------------
    sar = _bench_sar(B, torch, dev, stream)

    # ---- autofocus: entropy + adjoint gradient on a 4096 x 4096 FP16 scene -----------
    autofocus = _bench_autofocus(B, torch, dev, stream)

    # ---- uneven batch: 20,000 transforms, lengths 256..65536, one persistent launch ---
    uneven = _bench_uneven(B, torch, dev, stream)

    # ---- end to end through the C ABI with host buffers ---------------------------
    e2e = _bench_e2e(B, torch, dev, stream, x16, fwd16, inv16, flops_step, args)

    # ---- roofline of the dominant kernel (forward FP16 rows) -------------------------
    peak, peak_kind = _peaks()
    alg_bytes = 8.0 * N * batch                          # one FP16 read + one FP16 write per point
    fwd_avg = sum(fwd_ms) / len(fwd_ms)
    inv_avg = sum(inv_ms) / len(inv_ms)
    achieved = alg_bytes / (fwd_avg * 1e-3) / 1e9
    traffic = _profiled_traffic("fft_tc_f16_fwd_4096")

    if rank == 0:
        cpu = _cpu_baseline(seconds=args.cpu_seconds) if world == 1 else None
        line = {
            "metric": "batched FFT GFLOPS (5 N log2 N per transform), FP16-BFP storage, N=4096",
            "value": round(value, 1),
            "unit": "GFLOPS",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": round(t_ms, 4),
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f16 storage; f16 operands, f32 accumulation (tcgen05 DFT-16 blocks)",
            "data": "synthetic (re, im ~ N(0,1), seeded)",
            "config": _config(batch, world),
            "roofline": {
                "bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic,
                "kernel": "fft_tc_kernel<forward> (radix-16 passes as tcgen05.mma kind::f16, FP32 accumulators "
                          "in TMEM, 8 persistent CTAs/SM, L2 prefetch of each CTA's next line)",
                "kernel_source_hash": _kernel_source_hash(),
                "bytes_per_launch": alg_bytes, "launch_ms": round(fwd_avg, 5), "peak_source": peak_kind,
                "frac_of_8tbs_nominal": round(achieved / 8000.0, 4),
            },
            "fp16_sqnr_vs_fp32_db": round(sqnr16, 2),
            "fp32_storage_gflops": round(gflops32, 1),
            "fp8_e4m3_storage": fp8_entry,
            "fp8_e4m3_storage_tensor_cores": fp8_tc_entry,
            "fp16_over_fp32": round(value / world / gflops32, 3),
            "inverse_launch_ms": round(inv_avg, 5),
            "table2_batch256_l2_flushed": {"gflops": round(gflops_small, 1), "ms_median": round(t_small, 5),
                                           "fp32_arithmetic_gflops": round(gflops_small32, 1),
                                           "fp32_arithmetic_ms_median": round(t_small32, 5)},
            "precision_modes": modes,
            "batch_sweep": sweep,
            "ms_per_step_median": round(statistics.median(step_ms), 4),
            "gflops_at_median_step": round(_job_value(world, flops_step, statistics.median(step_ms)), 1),
            "sar": sar,
            "autofocus_4096x4096": autofocus,
            "uneven_20000": uneven,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "clocks": clocks.summary(),
            "gpu_launches": 2 * args.steps,
        }
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def _tc_plan(B, batch: int, direction: int):
    """The headline plan: N = 4096 FP16-BFP storage with FP16 operands and
    FP32 accumulation, the radix-16 DFT blocks on the tensor cores."""
    p = B.bfpfft_plan_create(N, batch, B.F16_BFP, direction)
    B.bfpfft_plan_set_arith(p, B.ARITH_F16_MUL_F32_ACC)
    return p


def _bench_batch_sweep(B, torch, dev, stream, batches=(256, 4096, 32768, 131072), steps: int = 30):
    """FP16-BFP forward + shifted inverse at N = 4096 for several batches:
    median of `steps` steps after 5 warm-ups, L2 flushed between steps when
    the input is smaller than 512 MiB (the largest batch moves 2 GiB each way)."""
    peak, _ = _peaks()
    out = {}
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    for batch in batches:
        g = torch.Generator(device=dev).manual_seed(batch)
        x = torch.randn((batch, N, 2), device=dev, generator=g).to(torch.float16)
        y, z = torch.empty_like(x), torch.empty_like(x)
        pf = _tc_plan(B, batch, B.FORWARD)
        pi = _tc_plan(B, batch, B.INVERSE)
        small = x.numel() * x.element_size() < 512 * 1024 * 1024
        fw, tot = [], []
        for i in range(steps + 5):
            if small:
                flush.fill_(i & 0xFF)
            e[0].record(stream)
            B.bfpfft_exec(pf, x, y, stream)
            e[1].record(stream)
            B.bfpfft_exec(pi, y, z, stream)
            e[2].record(stream)
            e[2].synchronize()
            if i >= 5:
                fw.append(e[0].elapsed_time(e[1]))
                tot.append(e[0].elapsed_time(e[2]))
        t, t_f = statistics.median(tot), statistics.median(fw)
        gbs = 8.0 * N * batch / (t_f * 1e-3) / 1e9
        out[str(batch)] = {"gflops": round(2.0 * FLOPS_PER_TRANSFORM * batch / (t * 1e-3) / 1e9, 1),
                           "ms_median": round(t, 5), "forward_gbs": round(gbs, 1),
                           "forward_frac_of_measured_hbm": round(gbs / peak, 4), "l2_flushed": small}
        del x, y, z, pf, pi
    del flush
    return out


def _sqnr_vs(B, torch, ref_c64, test, test_dtype, count, stream):
    """Aligned SQNR (dB) of `test` against a complex64 reference, by the library's FP64 sums."""
    ws_bytes = B.bfp_sqnr_workspace_bytes()
    ws = torch.empty(ws_bytes // 8, dtype=torch.float64, device=ref_c64.device)
    sums = torch.empty(8, dtype=torch.float64, device=ref_c64.device)
    B.bfp_sqnr_sums(ref_c64, B.F32, test, test_dtype, count, sums, ws, ws_bytes, stream)
    return round(B.sqnr_from_sums(sums[:5].cpu().tolist())["aligned_db"], 2)


def _bench_precision_modes(B, torch, dev, stream, x16, flops_step, steps):
    """The paper's other precision modes on the headline workload (N = 4096,
    batch of x16, forward + shifted inverse; the headline itself is FP16
    operands with FP32 accumulation on the tensor cores): FP16 storage with
    FP32 arithmetic throughout, pure FP16 arithmetic, bfloat16, and FP16 with
    adaptive per-line exponents.  Each: GFLOPS, the forward launch's GB/s and
    fraction of the measured HBM copy bandwidth, and the forward output's
    SQNR against the FP32-storage path on the first 256 lines."""
    batch = x16.shape[0]
    peak, _ = _peaks()
    ref_x = torch.view_as_complex(x16[:256].float().contiguous())
    ref_y = torch.empty_like(ref_x)
    B.bfpfft_exec(B.bfpfft_plan_create(N, 256, B.F32, B.FORWARD), ref_x, ref_y, stream)
    out = {}

    def timed(run_fwd, run_inv):
        for _ in range(3):
            run_fwd()
            run_inv()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        fw, tot = [], []
        for _ in range(steps):
            e[0].record(stream)
            run_fwd()
            e[1].record(stream)
            run_inv()
            e[2].record(stream)
            e[2].synchronize()
            fw.append(e[0].elapsed_time(e[1]))
            tot.append(e[0].elapsed_time(e[2]))
        return statistics.median(fw), statistics.median(tot)

    cases = (("fp16_storage_fp32_arithmetic", B.F16_BFP, B.ARITH_F32, x16),
             ("pure_fp16", B.F16_BFP, B.ARITH_F16, x16),
             ("bf16", B.BF16, B.ARITH_BF16, None))
    for name, dtype, arith, xin in cases:
        if xin is None:
            xin = x16.to(torch.bfloat16)
        y, z = torch.empty_like(xin), torch.empty_like(xin)
        pf = B.bfpfft_plan_create(N, batch, dtype, B.FORWARD)
        pi = B.bfpfft_plan_create(N, batch, dtype, B.INVERSE)
        B.bfpfft_plan_set_arith(pf, arith)
        B.bfpfft_plan_set_arith(pi, arith)
        t_f, t = timed(lambda: B.bfpfft_exec(pf, xin, y, stream), lambda: B.bfpfft_exec(pi, y, z, stream))
        gbs = 8.0 * N * batch / (t_f * 1e-3) / 1e9
        y32 = torch.view_as_complex(y[:256].float().contiguous())
        out[name] = {"gflops": round(flops_step / (t * 1e-3) / 1e9, 1), "ms_per_step": round(t, 4),
                     "forward_launch_ms": round(t_f, 5), "forward_gbs": round(gbs, 1),
                     "forward_frac_of_measured_hbm": round(gbs / peak, 4),
                     "sqnr_vs_fp32_db": _sqnr_vs(B, torch, ref_y, y32, B.F32, 256 * N, stream)}
        del y, z
    # adaptive exponents: the same input, and the same input scaled by 2^20
    e_in = torch.zeros(batch, dtype=torch.int32, device=dev)
    e_mid = torch.empty_like(e_in)
    e_out = torch.empty_like(e_in)
    y, z = torch.empty_like(x16), torch.empty_like(x16)
    pf = B.bfpfft_plan_create(N, batch, B.F16_ADAPTIVE, B.FORWARD)
    pi = B.bfpfft_plan_create(N, batch, B.F16_ADAPTIVE, B.INVERSE)
    t_f, t = timed(lambda: B.bfpfft_exec_adaptive(pf, x16, e_in, y, e_mid, stream),
                   lambda: B.bfpfft_exec_adaptive(pi, y, e_mid, z, e_out, stream))
    gbs = 8.0 * N * batch / (t_f * 1e-3) / 1e9
    e20 = torch.full_like(e_in, 20)
    B.bfpfft_exec_adaptive(pf, x16, e20, y, e_mid, stream)
    vals = (torch.view_as_complex(y[:256].float().contiguous())
            * torch.pow(2.0, e_mid[:256].float() - 20.0)[:, None])
    out["adaptive_exponents_fp16"] = {
        "gflops": round(flops_step / (t * 1e-3) / 1e9, 1), "ms_per_step": round(t, 4),
        "forward_launch_ms": round(t_f, 5), "forward_gbs": round(gbs, 1),
        "forward_frac_of_measured_hbm": round(gbs / peak, 4),
        "input_scaled_2^20_finite": bool(torch.isfinite(y).all().item()),
        "sqnr_vs_fp32_db_input_scaled_2^20": _sqnr_vs(B, torch, ref_y, vals.to(torch.complex64), B.F32, 256 * N,
                                                       stream)}
    return out


def _bench_sar(B, torch, dev, stream):
    from paper_2605_28451_gb300 import synth
    out = {}
    for name, n_az, n_rg in (("range_compress_1024x4096", 1024, 4096), ("image_4096x4096", 4096, 4096)):
        sc = synth.point_target_scene(n_az, n_rg)
        raw = torch.from_numpy(sc.raw.astype("complex64")).to(dev)
        hr = torch.empty(n_rg, dtype=torch.complex64, device=dev)
        ha = torch.empty(n_az, dtype=torch.complex64, device=dev)
        B.sar_make_filter(torch.from_numpy(sc.ref_range.astype("complex64")).to(dev), n_rg, False, hr, stream)
        B.sar_make_filter(torch.from_numpy(sc.ref_azimuth.astype("complex64")).to(dev), n_az, True, ha, stream)
        rc = torch.empty((n_rg, n_az, 2), dtype=torch.float16, device=dev)
        img = torch.empty((n_az, n_rg, 2), dtype=torch.float16, device=dev)
        flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
        full = name.startswith("image")

        def step():
            B.sar_range_compress(raw, B.F32, rc, B.F16_BFP, hr, n_az, n_rg, True, stream)
            if full:
                B.sar_azimuth_compress(rc, B.F16_BFP, 1, img, B.F16_BFP, ha, n_az, n_rg, stream)

        for _ in range(3):
            step()
        ts = []
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for i in range(20):
            flush.fill_(i & 0xFF)
            e0.record(stream)
            step()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        t = statistics.median(ts)
        transforms = 2 * n_az + (2 * n_rg if full else 0)
        flops = transforms * 5 * 4096 * 12
        bytes_ = n_az * n_rg * (12 + (8 if full else 0))
        out[name] = {"ms_median_l2_flushed": round(t, 4), "gflops": round(flops / (t * 1e-3) / 1e9, 1),
                     "alg_gbs": round(bytes_ / (t * 1e-3) / 1e9, 1), "dtype": "complex64 in, FP16-BFP out",
                     "naive_has_nonfinite": None}
        if full:
            out[name].update(_image_quality(B, torch, dev, stream, raw, hr, ha, img, sc.targets, n_az, n_rg))
            out["table4_modes_4096x4096"] = _bench_sar_modes(B, torch, dev, stream, raw, hr, ha, sc.targets,
                                                             n_az, n_rg, flush)
        if not full:
            # the same call in Table IV's 16-bit modes (FP16 out, corner-turned)
            for mname, marith in (("pure_fp16", B.ARITH_F16), ("fp16_mul_fp32_acc_tensor_cores",
                                                                   B.ARITH_F16_MUL_F32_ACC)):
                tm = []
                for i in range(23):
                    flush.fill_(i & 0xFF)
                    e0.record(stream)
                    B.sar_range_compress_arith(raw, B.F32, rc, B.F16_BFP, hr, n_az, n_rg, True, marith, stream)
                    e1.record(stream)
                    e1.synchronize()
                    if i >= 3:
                        tm.append(e0.elapsed_time(e1))
                out[name][mname + "_ms_median_l2_flushed"] = round(statistics.median(tm), 4)
            naive = torch.empty((n_az, n_rg, 2), dtype=torch.float16, device=dev)
            B.sar_range_compress(raw, B.F32, naive, B.F16_NAIVE, hr, n_az, n_rg, False, stream)
            torch.cuda.synchronize()
            out[name]["naive_has_nonfinite"] = bool((~torch.isfinite(naive)).any().item())
        del raw, rc, img, flush
    return out


def _bench_sar_modes(B, torch, dev, stream, raw, hr, ha, targets, n_az, n_rg, flush):
    """Table IV's four precision modes of the range-Doppler image on the same
    scene: time (median of 20, L2 flushed), SQNR against the GPU FP32 image and
    point-target deltas against the FP64 oracle's stored metrics."""
    modes = (("fp32", B.F32, B.ARITH_F32), ("fp16_mul_fp32_acc_tensor_cores", B.F16_BFP, B.ARITH_F16_MUL_F32_ACC),
             ("fp16_storage_fp32_compute", B.F16_BFP, B.ARITH_F32), ("pure_fp16", B.F16_BFP, B.ARITH_F16))
    imgs, out = {}, {}
    for name, dt, arith in modes:
        shape = (n_rg, n_az) if dt == B.F32 else (n_rg, n_az, 2)
        tdt = torch.complex64 if dt == B.F32 else torch.float16
        rc = torch.empty(shape, dtype=tdt, device=dev)
        img = torch.empty((n_az, n_rg) if dt == B.F32 else (n_az, n_rg, 2), dtype=tdt, device=dev)

        def step():
            B.sar_range_compress_arith(raw, B.F32, rc, dt, hr, n_az, n_rg, True, arith, stream)
            B.sar_azimuth_compress_arith(rc, dt, 1, img, dt, ha, n_az, n_rg, arith, stream)

        for _ in range(3):
            step()
        ts = []
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for i in range(20):
            flush.fill_(i & 0xFF)
            e0.record(stream)
            step()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        imgs[name] = (img, dt)
        out[name] = {"ms_median_l2_flushed": round(statistics.median(ts), 4)}
        del rc
    ref = imgs["fp32"][0]
    ws_bytes = B.bfp_sqnr_workspace_bytes()
    ws = torch.empty(ws_bytes // 8, dtype=torch.float64, device=dev)
    sums = torch.empty(8, dtype=torch.float64, device=dev)
    t = torch.tensor([[e, r] for e, r, _ in targets], dtype=torch.int32, device=dev)
    pw = B.sar_point_target_workspace_bytes(n_az, n_rg)
    pws = torch.empty(pw, dtype=torch.uint8, device=dev)
    m = torch.empty((len(targets), 12), dtype=torch.float64, device=dev)
    for name, (img, dt) in imgs.items():
        if name != "fp32":
            B.bfp_sqnr_sums(ref, B.F32, img, dt, n_az * n_rg, sums, ws, ws_bytes, stream)
            out[name]["sqnr_vs_fp32_db"] = round(B.sqnr_from_sums(sums[:5].cpu().tolist())["aligned_db"], 2)
        B.sar_point_target_metrics(img, dt, n_az, n_rg, t, len(targets), 96, m, pws, pw, stream)
        torch.cuda.synchronize()
        out[name]["vs_fp64_oracle"] = _golden_deltas(m.cpu().numpy(), targets, n_az, n_rg)
    return out


def _image_quality(B, torch, dev, stream, raw, hr, ha, img16, targets, n_az, n_rg):
    """FP16-BFP image vs the FP32 image of the same scene, both on the GPU:
    end-to-end SQNR (FP64 reduction) and the point-target metrics (FP64 kernel);
    and the FP16 image's metrics against the FP64 oracle's stored values."""
    rc32 = torch.empty((n_rg, n_az), dtype=torch.complex64, device=dev)
    img32 = torch.empty((n_az, n_rg), dtype=torch.complex64, device=dev)
    B.sar_range_compress(raw, B.F32, rc32, B.F32, hr, n_az, n_rg, True, stream)
    B.sar_azimuth_compress(rc32, B.F32, 1, img32, B.F32, ha, n_az, n_rg, stream)
    ws_bytes = B.bfp_sqnr_workspace_bytes()
    ws = torch.empty(ws_bytes // 8, dtype=torch.float64, device=dev)
    sums = torch.empty(8, dtype=torch.float64, device=dev)
    B.bfp_sqnr_sums(img32, B.F32, img16, B.F16_BFP, n_az * n_rg, sums, ws, ws_bytes, stream)
    sq = B.sqnr_from_sums(sums[:5].cpu().tolist())
    t = torch.tensor([[e, r] for e, r, _ in targets], dtype=torch.int32, device=dev)
    pw = B.sar_point_target_workspace_bytes(n_az, n_rg)
    pws = torch.empty(pw, dtype=torch.uint8, device=dev)
    m16 = torch.empty((len(targets), 12), dtype=torch.float64, device=dev)
    m32 = torch.empty_like(m16)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    B.sar_point_target_metrics(img16, B.F16_BFP, n_az, n_rg, t, len(targets), 96, m16, pws, pw, stream)
    e1.record(stream)
    B.sar_point_target_metrics(img32, B.F32, n_az, n_rg, t, len(targets), 96, m32, pws, pw, stream)
    torch.cuda.synchronize()
    a, b = m16.cpu().numpy(), m32.cpu().numpy()
    d = abs(a - b)
    out = {"sqnr_fp16_vs_fp32_db": round(sq["aligned_db"], 2), "nonfinite": sq["nonfinite"],
           "max_abs_delta_db": {"pslr": float(d[:, 0:2].max()), "islr": float(d[:, 2:4].max()),
                                "snr": float(d[:, 7].max())},
           "max_abs_delta_width_cells": float(d[:, 4:6].max()),
           "pslr_db_fp16": [round(float(x), 2) for x in a[:, 0:2].max(axis=1)],
           "snr_db_fp16": [round(float(x), 2) for x in a[:, 7]],
           "metrics_kernel_ms": round(e0.elapsed_time(e1), 3)}
    out["fp16_vs_fp64_oracle"] = _golden_deltas(a, targets, n_az, n_rg)
    return out


def _golden_deltas(m16, targets, n_az, n_rg):
    """The FP16 image's point-target metrics against the FP64 oracle's, stored
    for the 4096 x 4096 scene in tests/golden (written by an oracle-only
    script); None for other scenes."""
    p = os.path.join(ROOT, "tests", "golden", "sar_4096_image_metrics.json")
    if not os.path.exists(p):
        return None
    gold = json.load(open(p))
    if (n_az, n_rg) != (4096, 4096) or gold["targets"] != [[int(e), int(r)] for e, r, _ in targets]:
        return None
    keys = ("pslr_range_db", "pslr_azimuth_db", "islr_range_db", "islr_azimuth_db", "width_range_cells",
            "width_azimuth_cells", "peak", "snr_db")
    ref = [[g[k] for k in keys] for g in gold["metrics"]]
    dd = [[abs(float(m16[i][c]) - ref[i][c]) for c in range(8)] for i in range(len(ref))]
    return {"max_abs_delta_db": {"pslr": max(max(r[0:2]) for r in dd), "islr": max(max(r[2:4]) for r in dd),
                                 "snr": max(r[7] for r in dd)},
            "max_abs_delta_width_cells": max(max(r[4:6]) for r in dd),
            "bar": "0.1 dB, 0.1 cell", "source": "tests/golden/sar_4096_image_metrics.json"}


def _bench_autofocus(B, torch, dev, stream):
    """One autofocus gradient step (entropy pass + adjoint pass) on 4096 range
    bins x 4096 pulses of FP16 range-compressed data."""
    from paper_2605_28451_gb300 import autofocus as GA
    from paper_2605_28451_gb300 import synth
    n = 4096
    g = torch.Generator(device=dev).manual_seed(5)
    rc = torch.randn((n, n, 2), device=dev, generator=g).to(torch.float16)
    ref = synth.centred_reference(synth.azimuth_chirp(1024), n)
    ha = torch.empty(n, dtype=torch.complex64, device=dev)
    B.sar_make_filter(torch.from_numpy(ref.astype("complex64")).to(dev), n, True, ha, stream)
    phi = torch.from_numpy(synth.phase_error(n).astype("float32")).to(dev)
    grad = torch.empty(n, dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    out = {}
    ref_grad = None
    for name, arith in (("fp32_arithmetic", B.ARITH_F32), ("tensor_cores", B.ARITH_F16_MUL_F32_ACC)):
        ws = GA.Workspace(n, dev, arith)

        def step():
            B.sar_autofocus_grad(rc, B.F16_BFP, phi, ha, n, n, grad, ws.stats, ws.buf, ws.bytes, stream, arith)

        for _ in range(3):
            step()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ts = []
        for i in range(10):
            flush.fill_(i & 0xFF)
            e0.record(stream)
            step()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        t = statistics.median(ts)
        # entropy pass: 2 transforms per range bin; gradient pass: 4 (recomputed forward + adjoint)
        flops = 6 * n * 5 * n * 12
        out[name] = {"ms_median_l2_flushed": round(t, 4), "gflops": round(flops / (t * 1e-3) / 1e9, 1),
                     "alg_gbs": round(3 * 4 * n * n / (t * 1e-3) / 1e9, 1)}
        g = grad.double()
        if ref_grad is None:
            ref_grad = g.clone()
        else:                             # the tensor-core gradient against the FP32-arithmetic one
            out[name]["grad_rel_l2_vs_fp32_arithmetic"] = round(float((g - ref_grad).norm() / ref_grad.norm()), 6)
    out["fp32_arithmetic"]["dtype"] = "FP16-BFP rc, FP32 arithmetic"
    out["tensor_cores"]["dtype"] = "FP16-BFP rc, FP16 operands / FP32 accumulation"
    out.update(out["fp32_arithmetic"])          # the step's headline figures stay at the top level
    return out


def _bench_uneven(B, torch, dev, stream):
    """20,000 transforms with lengths drawn from {256, 1024, 4096, 16384, 65536}
    (Zipf weights, seed 3), forward, in FP16-BFP, FP32, E4M3 and E5M2 storage,
    each plan on the schedule the tuner picks (the persistent launch, or one
    launch per length) and replayed through a CUDA graph; the SQNR of each
    against the FP32 path by the library's FP64 reduction."""
    import numpy as np

    from paper_2605_28451_gb300 import synth
    lengths = synth.uneven_lengths(20000, seed=3)
    offsets = np.zeros_like(lengths)
    offsets[1:] = np.cumsum(lengths)[:-1]
    total = int(lengths.sum())
    flops = float(np.sum(5.0 * lengths * np.log2(lengths)))
    g = torch.Generator(device=dev).manual_seed(3)
    x32 = torch.randn((total, 2), device=dev, generator=g)
    y32 = torch.empty_like(x32)
    out = {"transforms": 20000, "points": total}
    ws_bytes = B.bfp_sqnr_workspace_bytes()
    ws = torch.empty(ws_bytes // 8, dtype=torch.float64, device=dev)
    sums = torch.empty(8, dtype=torch.float64, device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    scale = None
    for name, dtype in (("f32", B.F32), ("f16_bfp", B.F16_BFP), ("f16_bfp_persistent_kernel", B.F16_BFP),
                        ("f16_bfp_tuned_fp16_exchange", B.F16_BFP), ("e4m3", B.E4M3_BFP), ("e5m2", B.E5M2_BFP)):
        if dtype == B.F32:
            xin = x32
        elif dtype == B.F16_BFP:
            xin = x32.to(torch.float16)
        else:
            f8 = torch.float8_e4m3fn if dtype == B.E4M3_BFP else torch.float8_e5m2
            xin = x32.to(f8).view(torch.uint8)
        yout = y32 if dtype == B.F32 else torch.empty_like(xin)
        plan = B.bfpfft_plan_create_many(lengths, offsets, dtype, B.FORWARD)
        # The tuner's pick among cluster counts, two-pass long lines, one launch
        # per length and (FP16 exchanges allowed) the FP16 row exchange of
        # four-step lines; one FP16 plan keeps the untuned persistent kernel.
        if name == "f16_bfp_persistent_kernel":
            code = 0
        else:
            code, _ = B.bfpfft_plan_tune(plan, allow_fp16_exchange=name == "f16_bfp_tuned_fp16_exchange")
        for _ in range(3):
            B.bfpfft_exec_graph(plan, xin, yout, stream)
        ts = []
        for _ in range(10):
            e0.record(stream)
            B.bfpfft_exec_graph(plan, xin, yout, stream)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        t = statistics.median(ts)
        entry = {"ms_median": round(t, 4), "gflops": round(flops / (t * 1e-3) / 1e9, 1),
                 "alg_gbs": round(total * 2 * xin.element_size() * xin.shape[-1] / (t * 1e-3) / 1e9, 1)}
        if code:
            entry["tuned"] = {"clusters": code & 0xffff, "two_pass_long_lines": bool((code >> 16) & 1),
                              "fp16_row_exchange": bool((code >> 17) & 1),
                              "one_launch_per_length": bool((code >> 18) & 1)}
        if dtype == B.F16_BFP:
            B.bfp_sqnr_sums(torch.view_as_complex(y32), B.F32, yout, B.F16_BFP, total, sums, ws, ws_bytes, stream)
            entry["sqnr_vs_f32_db"] = round(B.sqnr_from_sums(sums[:5].cpu().tolist())["aligned_db"], 2)
        elif dtype != B.F32:
            if scale is None:
                s = np.repeat(np.exp2(-((np.log2(lengths).astype(np.int64) + 1) // 2)), lengths).astype(np.float32)
                scale = torch.from_numpy(s).to(dev)
            f8 = torch.float8_e4m3fn if dtype == B.E4M3_BFP else torch.float8_e5m2
            y8 = yout.view(f8).float()
            ref_scaled = (torch.view_as_real(torch.view_as_complex(y32)) * scale[:, None]).contiguous()
            B.bfp_sqnr_sums(torch.view_as_complex(ref_scaled), B.F32, torch.view_as_complex(y8.contiguous()), B.F32,
                            total, sums, ws, ws_bytes, stream)
            entry["sqnr_vs_f32_db"] = round(B.sqnr_from_sums(sums[:5].cpu().tolist())["aligned_db"], 2)
            del y8, ref_scaled
        out[name] = entry
        del plan
    return out


def _bench_e2e(B, torch, dev, stream, x16, fwd, inv, flops_step, args, chunks: int = 8):
    """Same metric through the C ABI with pinned host input and output buffers;
    every step copies its whole input host->device and its whole result
    device->host inside the timed region.  The batch is pipelined in `chunks`
    slices over three streams (copy in, transform, copy out), so the two copy
    directions and the transforms overlap as a serving loop would run them."""
    batch = x16.shape[0]
    assert batch % chunks == 0
    per = batch // chunks
    host_in = torch.empty(x16.shape, dtype=x16.dtype, pin_memory=True)
    host_in.copy_(x16)
    host_out = torch.empty_like(host_in, pin_memory=True)
    d_in = torch.empty_like(x16)
    d_mid = torch.empty_like(x16)
    d_out = torch.empty_like(x16)
    fwd_c = _tc_plan(B, per, B.FORWARD)
    inv_c = _tc_plan(B, per, B.INVERSE)
    s_in, s_fft, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    ev_in = [torch.cuda.Event() for _ in range(chunks)]
    ev_fft = [torch.cuda.Event() for _ in range(chunks)]
    ev_out = [torch.cuda.Event() for _ in range(chunks)]
    started = [False]

    def step():
        for c in range(chunks):
            sl = slice(c * per, (c + 1) * per)
            with torch.cuda.stream(s_in):
                if started[0]:
                    s_in.wait_event(ev_fft[c])          # previous step's transform read d_in[c]
                d_in[sl].copy_(host_in[sl], non_blocking=True)
                ev_in[c].record(s_in)
            s_fft.wait_event(ev_in[c])
            if started[0]:
                s_fft.wait_event(ev_out[c])             # previous step's copy-out read d_out[c]
            B.bfpfft_exec(fwd_c, d_in[sl], d_mid[sl], s_fft)
            B.bfpfft_exec(inv_c, d_mid[sl], d_out[sl], s_fft)
            ev_fft[c].record(s_fft)
            with torch.cuda.stream(s_out):
                s_out.wait_event(ev_fft[c])
                host_out[sl].copy_(d_out[sl], non_blocking=True)
                ev_out[c].record(s_out)
        started[0] = True

    for _ in range(2):
        step()
    torch.cuda.synchronize()
    k = max(3, args.steps // 2)
    t0 = time.perf_counter()
    for _ in range(k):
        step()
    torch.cuda.synchronize()
    t = (time.perf_counter() - t0) / k
    nbytes = x16.numel() * x16.element_size()
    assert torch.equal(host_out[:2].to(dev), d_out[:2])
    return {"value": round(flops_step / t / 1e9, 1), "unit": "GFLOPS", "h2d_bytes_per_step": nbytes,
            "d2h_bytes_per_step": nbytes, "ms_per_step": round(t * 1e3, 3),
            "pipeline": f"{chunks} chunks over copy-in / transform / copy-out streams"}


# The oracle's timing sample: lines of N = 4096 (the headline line length),
# forward + inverse, the same per-line work as one GPU step.
ORACLE_LINES = 64


def _cpu_model() -> str:
    """The host CPU's model name (x86 'model name', Arm 'CPU part' / lscpu)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine()


def _oracle_lines(lines: int, seed: int = 0) -> float:
    """Time one forward + inverse of `lines` oracle lines (seconds).  Runs in
    a worker process of the spawned pool, or in the caller."""
    from oracle import fft as F
    from paper_2605_28451_gb300 import synth
    x = synth.complex_gaussian(lines, N, seed=seed)
    t0 = time.perf_counter()
    F.ifft(F.fft(x))
    return time.perf_counter() - t0


class OraclePool:
    """The FP64 oracle on every host core: one spawned worker per core, each
    transforming its own ORACLE_LINES lines (the oracle itself is single-
    threaded numpy; spawned, not forked, so no CUDA state is inherited)."""

    def __init__(self):
        import multiprocessing as mp
        self.cores = os.cpu_count() or 1
        self.pool = mp.get_context("spawn").Pool(self.cores)
        self.pool.map(_oracle_lines, [1] * self.cores)          # imports done in every worker

    def step(self) -> float:
        """Wall time (s) of one step: every core runs ORACLE_LINES lines."""
        t0 = time.perf_counter()
        self.pool.map(_oracle_lines, [ORACLE_LINES] * self.cores)
        return time.perf_counter() - t0

    def close(self):
        self.pool.close()
        self.pool.join()


def _cpu_baseline(seconds: float = 10.0):
    """The FP64 oracle as it stands, on a bounded sample of the workload:
    ORACLE_LINES lines of N = 4096 forward + inverse per core, repeated for
    about `seconds` on one core and then on all cores at once."""
    flops_line = 2.0 * FLOPS_PER_TRANSFORM
    _oracle_lines(ORACLE_LINES)                                   # warm-up
    reps, t1, t_end = 0, 0.0, time.perf_counter() + seconds / 2
    while reps < 2 or time.perf_counter() < t_end:
        t1 += _oracle_lines(ORACLE_LINES)
        reps += 1
    one_core = flops_line * ORACLE_LINES * reps / t1 / 1e9
    pool = OraclePool()
    try:
        ts, t_end = [], time.perf_counter() + seconds / 2
        while len(ts) < 2 or time.perf_counter() < t_end:
            ts.append(pool.step())
    finally:
        pool.close()
    all_cores = flops_line * ORACLE_LINES * pool.cores / statistics.median(ts) / 1e9
    return {"value": round(all_cores, 3), "unit": "GFLOPS", "cores": pool.cores, "kind": "oracle",
            "sample": f"{ORACLE_LINES} lines of N={N} per core, forward + inverse, FP64 numpy radix-2; "
                      f"{len(ts)} all-core steps (median), {reps} single-core reps",
            "single_core_value": round(one_core, 3), "cpu_model": _cpu_model()}


def _config(batch: int, world: int) -> dict:
    """The workload both arms report (the reference arm times a bounded
    sample of it, described in its cpu_baseline)."""
    return {"workload": f"forward + 1/N-shifted inverse FFT, N={N}, batch {batch} per GPU, FP16-BFP (half2)",
            "l2": "inputs 1 GiB > L2, no flush needed", "parallelism": f"replicas x{world}"}


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return
    pool = OraclePool()
    try:
        for _ in range(args.warmup):
            pool.step()
        ts = [pool.step() for _ in range(args.steps)]
    finally:
        pool.close()
    t = sum(ts) / len(ts)
    value = 2.0 * FLOPS_PER_TRANSFORM * ORACLE_LINES * pool.cores / t / 1e9
    sample = (f"{ORACLE_LINES} lines of N={N} per core per step on {pool.cores} cores (of the {args.batch}-line "
              f"workload), forward + inverse, FP64 numpy radix-2")
    print(json.dumps({
        "impl": "reference",
        "metric": "batched FFT GFLOPS (5 N log2 N per transform), FP16-BFP storage, N=4096",
        "value": round(value, 4), "unit": "GFLOPS", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(t * 1e3, 3), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic (re, im ~ N(0,1), seeded)",
        "config": _config(args.batch, world),
        "sample": sample,
        "cpu_baseline": {"value": round(value, 4), "unit": "GFLOPS", "cores": pool.cores, "kind": "oracle",
                         "sample": sample, "cpu_model": _cpu_model()},
        "e2e": {"value": round(value, 4), "unit": "GFLOPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch", type=int, default=BATCH)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
