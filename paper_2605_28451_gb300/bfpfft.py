"""Thin ctypes binding of include/bfpfft.h.

Argument marshalling only: every function here converts torch tensors to raw
device pointers and the current CUDA stream, calls the C entry point of the
same name, and turns a non-zero status into ``BfpfftError``.  There is no
fallback: if the compiled library is missing, the first call raises.
"""

from __future__ import annotations

import ctypes
import os

from . import build as _build

# Status codes (enum bfpfft_status).
OK = 0
ERR_INVALID_ARG = 1
ERR_UNSUPPORTED = 2
ERR_CUDA = 3
ERR_OOM = 4
ERR_TIMEOUT = 5
ERR_NONFINITE = 6
ERR_MISALIGNED = 7

# Storage dtypes (enum bfpfft_dtype).
F32 = 0
F16_BFP = 1
F16_NAIVE = 2
E4M3_BFP = 3
E5M2_BFP = 4
F16_ADAPTIVE = 5
BF16 = 6

# Arithmetic modes (enum bfpfft_arith).
ARITH_F32 = 0
ARITH_F16 = 1
ARITH_F16_MUL_F32_ACC = 2
ARITH_BF16 = 3

FORWARD = -1
INVERSE = +1

CHECK_FINITE = 1   # plan flag (enum bfpfft_flags)

# Uneven-plan schedule flags (enum bfpfft_many_schedule).
MANY_TWO_PASS = 1
MANY_FP16_ROWS = 2
MANY_PER_LENGTH = 4

BYTES_PER_POINT = {F32: 8, F16_BFP: 4, F16_NAIVE: 4, E4M3_BFP: 2, E5M2_BFP: 2, F16_ADAPTIVE: 4, BF16: 4}

_c_int64 = ctypes.c_int64
_vp = ctypes.c_void_p

# name -> (restype, argtypes); every exported symbol of include/bfpfft.h.
SIGNATURES = {
    "bfpfft_version": (ctypes.c_int, []),
    "bfpfft_error_string": (ctypes.c_char_p, [ctypes.c_int]),
    "bfpfft_plan_create": (ctypes.c_int, [ctypes.POINTER(_vp), _c_int64, _c_int64, ctypes.c_int, ctypes.c_int]),
    "bfpfft_exec": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "bfpfft_plan_create_many": (ctypes.c_int, [ctypes.POINTER(_vp), _c_int64, _vp, _vp, ctypes.c_int, ctypes.c_int]),
    "bfpfft_plan_info": (ctypes.c_int, [_vp, ctypes.POINTER(_c_int64), ctypes.POINTER(_c_int64)]),
    "bfpfft_exec_graph": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "bfpfft_plan_tune": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float)]),
    "bfpfft_plan_destroy": (ctypes.c_int, [_vp]),
    "bfpfft_plan_scale_exp": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "bfpfft_device_status": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int)]),
    "bfpfft_plan_status": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int)]),
    "bfpfft_plan_set_flags": (ctypes.c_int, [_vp, ctypes.c_int]),
    "bfpfft_plan_set_many_schedule": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int]),
    "bfpfft_plan_selftest_wait": (ctypes.c_int, [_vp, _vp]),
    "bfpfft_plan_set_arith": (ctypes.c_int, [_vp, ctypes.c_int]),
    "bfpfft_exec_adaptive": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "bfp_spectral_adaptive": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _vp, _vp, _c_int64, _c_int64, _vp]),
    "bfp_spectral_filter": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _c_int64, _vp, ctypes.c_int, _c_int64, _c_int64,
                                           ctypes.c_int, _vp]),
    "sar_make_filter": (ctypes.c_int, [_vp, _c_int64, ctypes.c_int, _vp, _vp]),
    "sar_range_compress": (ctypes.c_int, [_vp, ctypes.c_int, _vp, ctypes.c_int, _vp, _c_int64, _c_int64,
                                          ctypes.c_int, _vp]),
    "sar_azimuth_compress": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_int, _vp, _c_int64,
                                            _c_int64, _vp]),
    "sar_range_compress_arith": (ctypes.c_int, [_vp, ctypes.c_int, _vp, ctypes.c_int, _vp, _c_int64, _c_int64,
                                                ctypes.c_int, ctypes.c_int, _vp]),
    "sar_azimuth_compress_arith": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_int, _vp, _c_int64,
                                                  _c_int64, ctypes.c_int, _vp]),
    "sar_rda_image": (ctypes.c_int, [_vp, ctypes.c_int, _vp, ctypes.c_int, _vp, _c_int64, _c_int64, _vp, _c_int64,
                                     ctypes.c_int, _vp]),
    "sar_autofocus_workspace_bytes": (ctypes.c_size_t, [_c_int64]),
    "sar_autofocus_entropy": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _c_int64, _c_int64, _vp, _vp,
                                             ctypes.c_size_t, _vp]),
    "sar_autofocus_grad": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _c_int64, _c_int64, _vp, _vp, _vp,
                                          ctypes.c_size_t, _vp]),
    "sar_autofocus_entropy_arith": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _c_int64, _c_int64, _vp, _vp,
                                                   ctypes.c_size_t, ctypes.c_int, _vp]),
    "sar_autofocus_grad_arith": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _c_int64, _c_int64, _vp, _vp, _vp,
                                                ctypes.c_size_t, ctypes.c_int, _vp]),
    "sar_point_target_workspace_bytes": (ctypes.c_size_t, [_c_int64, _c_int64]),
    "sar_point_target_metrics": (ctypes.c_int, [_vp, ctypes.c_int, _c_int64, _c_int64, _vp, _c_int64, ctypes.c_int,
                                                _vp, _vp, ctypes.c_size_t, _vp]),
    "bfp_sqnr_workspace_bytes": (ctypes.c_size_t, []),
    "bfp_sqnr_sums_noalloc_max_count": (ctypes.c_longlong, []),
    "bfp_sqnr_sums_noalloc": (ctypes.c_int, [_vp, ctypes.c_int, _vp, ctypes.c_int, _c_int64, _vp, _vp]),
    "bfp_sqnr_sums": (ctypes.c_int, [_vp, ctypes.c_int, _vp, ctypes.c_int, _c_int64, _vp, _vp, ctypes.c_size_t,
                                     _vp]),
}

_lib = None


class BfpfftError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: status {status} ({error_string(status)})")


def library_path() -> str:
    return _build.LIB_PATH


def lib():
    """Load libbfpfft.so (built in-tree by build.build()); raise if it is missing."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with paper_2605_28451_gb300.build.build(); "
                               "there is no CPU fallback")
        handle = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _lib = handle
    return _lib


def error_string(status: int) -> str:
    try:
        return lib().bfpfft_error_string(int(status)).decode()
    except Exception:  # library not loadable: still give a readable message
        return "unknown"


def _check(status: int, where: str):
    if status != OK:
        raise BfpfftError(status, where)


def _ptr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def bfpfft_version() -> int:
    return lib().bfpfft_version()


class Plan:
    """Owning handle of a bfpfft_plan (destroyed with the object)."""

    def __init__(self, handle: int, n: int, batch: int, dtype: int, direction: int):
        self.handle, self.n, self.batch, self.dtype, self.direction = handle, n, batch, dtype, direction

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and _lib is not None:
            _lib.bfpfft_plan_destroy(h)
            self.handle = None


def bfpfft_plan_create(n: int, batch: int, dtype: int, direction: int) -> Plan:
    h = _vp()
    _check(lib().bfpfft_plan_create(ctypes.byref(h), int(n), int(batch), int(dtype), int(direction)),
           "bfpfft_plan_create")
    return Plan(h.value, n, batch, dtype, direction)


def bfpfft_exec(plan: Plan, inp, out, stream=None):
    _check(lib().bfpfft_exec(plan.handle, _ptr(inp), _ptr(out), _stream(stream)), "bfpfft_exec")


def bfpfft_plan_create_many(n, offset_pts, dtype: int, direction: int) -> Plan:
    """Uneven plan; n and offset_pts are sequences of ints (host)."""
    import numpy as np
    n_arr = np.ascontiguousarray(np.asarray(n, dtype=np.int64))
    o_arr = np.ascontiguousarray(np.asarray(offset_pts, dtype=np.int64))
    if n_arr.shape != o_arr.shape:
        raise ValueError("n and offset_pts differ in length")
    h = _vp()
    _check(lib().bfpfft_plan_create_many(ctypes.byref(h), int(n_arr.size), n_arr.ctypes.data if n_arr.size else None,
                                         o_arr.ctypes.data if o_arr.size else None, int(dtype), int(direction)),
           "bfpfft_plan_create_many")
    return Plan(h.value, 0, int(n_arr.size), dtype, direction)


def bfpfft_plan_info(plan: Plan):
    t, c = _c_int64(), _c_int64()
    _check(lib().bfpfft_plan_info(plan.handle, ctypes.byref(t), ctypes.byref(c)), "bfpfft_plan_info")
    return t.value, c.value


def bfpfft_plan_tune(plan: Plan, allow_fp16_exchange: bool = False):
    """Tune the plan on its own shape; returns (chosen variant or cluster count, median ms)."""
    c, ms = ctypes.c_int(), ctypes.c_float()
    _check(lib().bfpfft_plan_tune(plan.handle, int(bool(allow_fp16_exchange)), ctypes.byref(c), ctypes.byref(ms)),
           "bfpfft_plan_tune")
    return c.value, ms.value


def bfpfft_exec_graph(plan: Plan, inp, out, stream=None):
    _check(lib().bfpfft_exec_graph(plan.handle, _ptr(inp), _ptr(out), _stream(stream)), "bfpfft_exec_graph")


def bfpfft_plan_destroy(plan: Plan):
    if plan.handle:
        _check(lib().bfpfft_plan_destroy(plan.handle), "bfpfft_plan_destroy")
        plan.handle = None


def bfpfft_plan_scale_exp(plan: Plan):
    a, b = ctypes.c_int(), ctypes.c_int()
    _check(lib().bfpfft_plan_scale_exp(plan.handle, ctypes.byref(a), ctypes.byref(b)), "bfpfft_plan_scale_exp")
    return a.value, b.value


def bfpfft_device_status() -> int:
    """Synchronise the device, then read and clear its status word."""
    st = ctypes.c_int()
    _check(lib().bfpfft_device_status(ctypes.byref(st)), "bfpfft_device_status")
    return st.value


def bfpfft_plan_status(plan: Plan) -> int:
    """Synchronise the device, then read and clear the plan's status word."""
    st = ctypes.c_int()
    _check(lib().bfpfft_plan_status(plan.handle, ctypes.byref(st)), "bfpfft_plan_status")
    return st.value


def bfpfft_plan_set_flags(plan: Plan, flags: int):
    _check(lib().bfpfft_plan_set_flags(plan.handle, int(flags)), "bfpfft_plan_set_flags")


def bfpfft_plan_set_many_schedule(plan: Plan, clusters: int = 0, flags: int = 0):
    """Uneven plan: persistent clusters (0: all resident) and MANY_* flags."""
    _check(lib().bfpfft_plan_set_many_schedule(plan.handle, int(clusters), int(flags)),
           "bfpfft_plan_set_many_schedule")


def bfpfft_plan_set_arith(plan: Plan, arith: int):
    _check(lib().bfpfft_plan_set_arith(plan.handle, int(arith)), "bfpfft_plan_set_arith")


def bfpfft_plan_selftest_wait(plan: Plan, stream=None):
    _check(lib().bfpfft_plan_selftest_wait(plan.handle, _stream(stream)), "bfpfft_plan_selftest_wait")


def bfpfft_exec_adaptive(plan: Plan, inp, in_exp, out, out_exp, stream=None):
    """FP16 mantissas + int32 per-line exponents in and out (in_exp may be None)."""
    _check(lib().bfpfft_exec_adaptive(plan.handle, _ptr(inp), _ptr(in_exp), _ptr(out), _ptr(out_exp),
                                      _stream(stream)), "bfpfft_exec_adaptive")


def bfp_spectral_filter(x, x_dtype: int, h, h_stride: int, out, out_dtype: int, n: int, lines: int,
                        arith: int = ARITH_F32, stream=None):
    _check(lib().bfp_spectral_filter(_ptr(x), int(x_dtype), _ptr(h), int(h_stride), _ptr(out), int(out_dtype), int(n),
                                     int(lines), int(arith), _stream(stream)), "bfp_spectral_filter")


def bfp_spectral_adaptive(x, x_dtype: int, x_exp, h, out, out_exp, n: int, lines: int, stream=None):
    _check(lib().bfp_spectral_adaptive(_ptr(x), int(x_dtype), _ptr(x_exp), _ptr(h), _ptr(out), _ptr(out_exp),
                                       int(n), int(lines), _stream(stream)), "bfp_spectral_adaptive")


def sar_make_filter(ref, n: int, peak_normalise: bool, h_out, stream=None):
    _check(lib().sar_make_filter(_ptr(ref), int(n), int(bool(peak_normalise)), _ptr(h_out), _stream(stream)),
           "sar_make_filter")


def sar_range_compress(raw, raw_dtype: int, out, out_dtype: int, hr, n_az: int, n_rg: int,
                       transpose_out: bool = False, stream=None):
    _check(lib().sar_range_compress(_ptr(raw), int(raw_dtype), _ptr(out), int(out_dtype), _ptr(hr), int(n_az),
                                    int(n_rg), int(bool(transpose_out)), _stream(stream)), "sar_range_compress")


def sar_azimuth_compress(rc, rc_dtype: int, rc_layout: int, img, img_dtype: int, ha, n_az: int, n_rg: int,
                         stream=None):
    _check(lib().sar_azimuth_compress(_ptr(rc), int(rc_dtype), int(rc_layout), _ptr(img), int(img_dtype), _ptr(ha),
                                      int(n_az), int(n_rg), _stream(stream)), "sar_azimuth_compress")


def sar_range_compress_arith(raw, raw_dtype: int, out, out_dtype: int, hr, n_az: int, n_rg: int,
                             transpose_out: bool, arith: int, stream=None):
    _check(lib().sar_range_compress_arith(_ptr(raw), int(raw_dtype), _ptr(out), int(out_dtype), _ptr(hr), int(n_az),
                                          int(n_rg), int(bool(transpose_out)), int(arith), _stream(stream)),
           "sar_range_compress_arith")


def sar_azimuth_compress_arith(rc, rc_dtype: int, rc_layout: int, img, img_dtype: int, ha, n_az: int, n_rg: int,
                               arith: int, stream=None):
    _check(lib().sar_azimuth_compress_arith(_ptr(rc), int(rc_dtype), int(rc_layout), _ptr(img), int(img_dtype),
                                            _ptr(ha), int(n_az), int(n_rg), int(arith), _stream(stream)),
           "sar_azimuth_compress_arith")


RDA_RCMC = 1
RDA_RANGE_DEPENDENT = 2
RDA_PEAK_NORMALISE = 4


def sar_rda_image(raw, raw_dtype: int, img, img_dtype: int, hr, n_az: int, n_rg: int, geometry, aperture: int,
                  flags: int, stream=None):
    """geometry: (range cell m, PRF Hz, wavelength m, speed m/s, centre slant range m)."""
    g = (ctypes.c_double * 5)(*[float(v) for v in geometry])
    _check(lib().sar_rda_image(_ptr(raw), int(raw_dtype), _ptr(img), int(img_dtype), _ptr(hr), int(n_az), int(n_rg),
                               ctypes.cast(g, _vp), int(aperture), int(flags), _stream(stream)), "sar_rda_image")


def bfp_sqnr_workspace_bytes() -> int:
    return int(lib().bfp_sqnr_workspace_bytes())


def bfp_sqnr_sums(ref, ref_dtype: int, test, test_dtype: int, count: int, sums_out, workspace, ws_bytes: int,
                  stream=None):
    _check(lib().bfp_sqnr_sums(_ptr(ref), int(ref_dtype), _ptr(test), int(test_dtype), int(count), _ptr(sums_out),
                               _ptr(workspace), int(ws_bytes), _stream(stream)), "bfp_sqnr_sums")


def sqnr_from_sums(s) -> dict:
    """Aligned / unaligned SQNR in dB from the five sums of bfp_sqnr_sums (host arithmetic on 5 numbers)."""
    import math
    s0, s1, s2, s3, bad = (float(v) for v in s)
    err_aligned = s0 - s2 * s2 / s1 if s1 > 0 else s0
    cap = 300.0

    def db(num, den):
        return cap if den <= 0 else min(cap, 10.0 * math.log10(num / den))
    return {"aligned_db": db(s0, err_aligned), "unaligned_db": db(s0, s3), "nonfinite": int(bad),
            "alpha": s2 / s1 if s1 > 0 else float("nan")}


def sar_autofocus_workspace_bytes(n_az: int) -> int:
    return int(lib().sar_autofocus_workspace_bytes(int(n_az)))


def sar_autofocus_entropy(rc, rc_dtype: int, phi, ha, n_az: int, n_rg: int, stats_out, workspace, ws_bytes: int,
                          stream=None, arith: int = ARITH_F32):
    _check(lib().sar_autofocus_entropy_arith(_ptr(rc), int(rc_dtype), _ptr(phi), _ptr(ha), int(n_az), int(n_rg),
                                             _ptr(stats_out), _ptr(workspace), int(ws_bytes), int(arith),
                                             _stream(stream)), "sar_autofocus_entropy")


def sar_autofocus_grad(rc, rc_dtype: int, phi, ha, n_az: int, n_rg: int, grad_out, stats_out, workspace,
                       ws_bytes: int, stream=None, arith: int = ARITH_F32):
    _check(lib().sar_autofocus_grad_arith(_ptr(rc), int(rc_dtype), _ptr(phi), _ptr(ha), int(n_az), int(n_rg),
                                          _ptr(grad_out), _ptr(stats_out), _ptr(workspace), int(ws_bytes),
                                          int(arith), _stream(stream)), "sar_autofocus_grad")


def bfp_sqnr_sums_noalloc_max_count() -> int:
    return int(lib().bfp_sqnr_sums_noalloc_max_count())


def bfp_sqnr_sums_noalloc(ref, ref_dtype: int, test, test_dtype: int, count: int, sums_out, stream=None):
    """bfp_sqnr_sums with the library's built-in scratch: no workspace, no allocation."""
    _check(lib().bfp_sqnr_sums_noalloc(_ptr(ref), int(ref_dtype), _ptr(test), int(test_dtype), int(count),
                                       _ptr(sums_out), _stream(stream)), "bfp_sqnr_sums_noalloc")


PT_FIELDS = ("pslr_range_db", "pslr_azimuth_db", "islr_range_db", "islr_azimuth_db", "width_range_cells",
             "width_azimuth_cells", "peak", "snr_db", "noise_power", "peak_eta", "peak_r", "reserved")


def sar_point_target_workspace_bytes(n_az: int, n_rg: int) -> int:
    return int(lib().sar_point_target_workspace_bytes(int(n_az), int(n_rg)))


def sar_point_target_metrics(img, img_dtype: int, n_az: int, n_rg: int, targets, k: int, guard: int, out, workspace,
                             ws_bytes: int, stream=None):
    _check(lib().sar_point_target_metrics(_ptr(img), int(img_dtype), int(n_az), int(n_rg), _ptr(targets), int(k),
                                          int(guard), _ptr(out), _ptr(workspace), int(ws_bytes), _stream(stream)),
           "sar_point_target_metrics")
