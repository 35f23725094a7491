"""Run one hot-path case a few times, for profiling under ncu.

    python -m paper_2605_28451_gb300.profile_cases <case> [--batch B] [--reps R]

Cases (FP16-BFP unless named otherwise, N = 4096 lines):
  fft16_fwd, fft16_inv   batched transform, batch B (default 16384: 256 MiB in); --arith f16 | f16mul | bf16
                         selects pure FP16, FP16 operands / FP32 accumulation (tensor cores) or bfloat16
  fft32_fwd              the same in FP32 storage
  fft8_fwd               the same in E4M3 storage (--arith f16mul: on the tensor cores)
  adaptive16_fwd         FP16 with adaptive per-line exponents, batch B
  rda16                  range-Doppler image with RCMC and range-dependent filters, 4096 x 4096, FP16
  range16                range compression of a 1024 x 4096 complex64 scene to FP16, corner-turned
  image16                range + azimuth compression of a 4096 x 4096 scene to an FP16 image
                         (range16, image16: --arith f16 | f16mul for Table IV's pure-FP16 and tensor-core modes)
  autofocus16            one autofocus gradient step on 4096 x 4096 FP16 range-compressed data (--arith
                         f16mul: the transforms on the tensor cores)
  uneven16               a persistent uneven batch of B transforms (default 2000; lengths 256 .. 65536,
                         Zipf weights, seed 3), FP16, forward; --many-flags 4: one launch per length
                         (| 2: FP16 four-step row exchanges)
Inputs are seeded and synthetic.  Nothing is checked here; the tests do that.
"""

from __future__ import annotations

import argparse

import torch

from . import bfpfft as B
from . import build, synth


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("case")
    ap.add_argument("--batch", type=int, default=16384)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--n", type=int, default=4096, help="transform length of the fft* cases")
    ap.add_argument("--time", action="store_true", help="print the median ms per rep (CUDA events)")
    ap.add_argument("--arith", default="f32", choices=["f32", "f16", "f16mul", "bf16"])
    ap.add_argument("--many-flags", type=int, default=0, help="uneven16: schedule flags (MANY_*)")
    args = ap.parse_args()
    times = []
    build.build()
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream()
    n = args.n if args.case.startswith("fft") else 4096
    g = torch.Generator(device=dev).manual_seed(0)
    if args.case in ("fft16_fwd", "fft16_inv", "fft32_fwd", "fft8_fwd"):
        dtype = B.F32 if args.case == "fft32_fwd" else (B.BF16 if args.arith == "bf16" else B.F16_BFP)
        dtype = B.E4M3_BFP if args.case == "fft8_fwd" else dtype
        direction = B.INVERSE if args.case == "fft16_inv" else B.FORWARD
        x = torch.randn((args.batch, n, 2), device=dev, generator=g)
        if dtype == B.E4M3_BFP:
            x = x.to(torch.float8_e4m3fn).view(torch.uint8)
        elif dtype != B.F32:
            x = x.to(torch.bfloat16 if dtype == B.BF16 else torch.float16)
        y = torch.empty_like(x)
        plan = B.bfpfft_plan_create(n, args.batch, dtype, direction)
        arith = {"f32": None, "f16": B.ARITH_F16, "f16mul": B.ARITH_F16_MUL_F32_ACC, "bf16": None}[args.arith]
        if arith is not None:
            B.bfpfft_plan_set_arith(plan, arith)
        for _ in range(args.reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            B.bfpfft_exec(plan, x, y, stream)
            e1.record(stream)
            times.append((e0, e1))
        bytes_per_rep = args.batch * n * {B.F32: 16, B.E4M3_BFP: 4}.get(dtype, 8)
    elif args.case == "adaptive16_fwd":
        x = torch.randn((args.batch, n, 2), device=dev, generator=g).to(torch.float16)
        y = torch.empty_like(x)
        e_in = torch.zeros(args.batch, dtype=torch.int32, device=dev)
        e_out = torch.empty_like(e_in)
        plan = B.bfpfft_plan_create(n, args.batch, B.F16_ADAPTIVE, B.FORWARD)
        for _ in range(args.reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            B.bfpfft_exec_adaptive(plan, x, e_in, y, e_out, stream)
            e1.record(stream)
            times.append((e0, e1))
        bytes_per_rep = args.batch * n * 8
    elif args.case == "rda16":
        geo = synth.radar_geometry(1024)
        sc = synth.point_target_scene(n, n)
        raw = torch.from_numpy(sc.raw.astype("complex64")).to(dev)
        hr = torch.empty(n, dtype=torch.complex64, device=dev)
        B.sar_make_filter(torch.from_numpy(sc.ref_range.astype("complex64")).to(dev), n, False, hr, stream)
        img = torch.empty((n, n, 2), dtype=torch.float16, device=dev)
        g5 = (geo.range_cell_m, geo.prf_hz, geo.wavelength_m, geo.speed_mps, geo.centre_range_m)
        flags = B.RDA_RCMC | B.RDA_RANGE_DEPENDENT | B.RDA_PEAK_NORMALISE
        for _ in range(args.reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            B.sar_rda_image(raw, B.F32, img, B.F16_BFP, hr, n, n, g5, 1024, flags, stream)
            e1.record(stream)
            times.append((e0, e1))
        bytes_per_rep = n * n * 20
    elif args.case in ("range16", "image16"):
        n_az = 1024 if args.case == "range16" else n
        sc = synth.point_target_scene(n_az, n)
        raw = torch.from_numpy(sc.raw.astype("complex64")).to(dev)
        hr = torch.empty(n, dtype=torch.complex64, device=dev)
        ha = torch.empty(n_az, dtype=torch.complex64, device=dev)
        B.sar_make_filter(torch.from_numpy(sc.ref_range.astype("complex64")).to(dev), n, False, hr, stream)
        B.sar_make_filter(torch.from_numpy(sc.ref_azimuth.astype("complex64")).to(dev), n_az, True, ha, stream)
        rc = torch.empty((n, n_az, 2), dtype=torch.float16, device=dev)
        img = torch.empty((n_az, n, 2), dtype=torch.float16, device=dev)
        sar_arith = {"f32": B.ARITH_F32, "f16": B.ARITH_F16, "f16mul": B.ARITH_F16_MUL_F32_ACC}[args.arith]
        for _ in range(args.reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            B.sar_range_compress_arith(raw, B.F32, rc, B.F16_BFP, hr, n_az, n, True, sar_arith, stream)
            if args.case == "image16":
                B.sar_azimuth_compress_arith(rc, B.F16_BFP, 1, img, B.F16_BFP, ha, n_az, n, sar_arith, stream)
            e1.record(stream)
            times.append((e0, e1))
        bytes_per_rep = n_az * n * (12 if args.case == "range16" else 20)
    elif args.case == "autofocus16":
        from . import autofocus as GA
        rc = torch.randn((n, n, 2), device=dev, generator=g).to(torch.float16)
        ha = torch.empty(n, dtype=torch.complex64, device=dev)
        B.sar_make_filter(torch.from_numpy(synth.centred_reference(synth.azimuth_chirp(1024), n)
                                           .astype("complex64")).to(dev), n, True, ha, stream)
        phi = torch.from_numpy(synth.phase_error(n).astype("float32")).to(dev)
        af_arith = B.ARITH_F16_MUL_F32_ACC if args.arith == "f16mul" else B.ARITH_F32
        ws = GA.Workspace(n, dev, af_arith)
        grad = torch.empty(n, dtype=torch.float32, device=dev)
        stats = torch.empty(4, dtype=torch.float64, device=dev)
        for _ in range(args.reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            B.sar_autofocus_grad(rc, B.F16_BFP, phi, ha, n, n, grad, stats, ws.buf, ws.bytes, stream, af_arith)
            e1.record(stream)
            times.append((e0, e1))
        bytes_per_rep = n * n * 12
    elif args.case == "uneven16":
        import numpy as np
        count = args.batch if args.batch != 16384 else 2000
        lengths = synth.uneven_lengths(count, seed=3)
        offsets = np.zeros_like(lengths)
        offsets[1:] = np.cumsum(lengths)[:-1]
        total = int(lengths.sum())
        x = torch.randn((total, 2), device=dev, generator=g).to(torch.float16)
        y = torch.empty_like(x)
        plan = B.bfpfft_plan_create_many(lengths, offsets, B.F16_BFP, B.FORWARD)
        if args.many_flags:
            B.bfpfft_plan_set_many_schedule(plan, 0, args.many_flags)
        for _ in range(args.reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            B.bfpfft_exec(plan, x, y, stream)
            e1.record(stream)
            times.append((e0, e1))
        bytes_per_rep = total * 8
    else:
        raise SystemExit(f"unknown case {args.case}")
    torch.cuda.synchronize()
    if args.time and times:
        import os
        import statistics
        ms = statistics.median(a.elapsed_time(b) for a, b in times[1:] or times)
        print(f"{args.case} arith={args.arith} variant={os.environ.get('BFPFFT_ROWS', 'default')} ms={ms:.5f} "
              f"alg_GBps={bytes_per_rep / (ms * 1e-3) / 1e9:.1f}")
    status = B.bfpfft_device_status()
    if status != B.OK:
        raise SystemExit(f"device status {status}")


if __name__ == "__main__":
    main()
