"""The C-ABI library builds, loads and exports every symbol of include/*.h;
host-side argument checks and fault injection return the documented status
codes without touching a GPU (CPU only)."""

import glob
import os
import re

import pytest

from paper_2605_28451_gb300 import bfpfft as B
from paper_2605_28451_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:[A-Za-z_]\w*[\s\*]+)+(\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return B.lib()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 9
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(B.SIGNATURES), "binding misses a declared function"


def test_version_and_error_strings(lib):
    assert B.bfpfft_version() >= 100
    for st in range(8):
        assert B.error_string(st) not in ("", "unknown status")
    assert B.error_string(99) == "unknown status"


@pytest.mark.parametrize("n", [0, 8, 12, 100, 131072, 1 << 20])
def test_unsupported_lengths(lib, n):
    with pytest.raises(B.BfpfftError) as e:
        B.bfpfft_plan_create(n, 4, B.F16_BFP, B.FORWARD)
    assert e.value.status == B.ERR_UNSUPPORTED


@pytest.mark.parametrize("batch,dtype,direction", [(-1, B.F32, B.FORWARD), (4, 9, B.FORWARD),
                                                   (4, B.F32, 0), (4, -1, B.INVERSE)])
def test_invalid_plan_args(lib, batch, dtype, direction):
    with pytest.raises(B.BfpfftError) as e:
        B.bfpfft_plan_create(4096, batch, dtype, direction)
    assert e.value.status == B.ERR_INVALID_ARG


def test_null_plan_and_buffers(lib):
    assert lib.bfpfft_exec(None, None, None, None) == B.ERR_INVALID_ARG
    assert lib.bfpfft_plan_destroy(None) == B.OK
    assert lib.bfpfft_plan_create(None, 4096, 1, 0, -1) == B.ERR_INVALID_ARG


def test_sar_argument_checks(lib):
    assert lib.sar_range_compress(16, 0, 16, 1, 16, -1, 4096, 0, None) == B.ERR_INVALID_ARG
    assert lib.sar_range_compress(16, 0, 16, 1, 16, 8, 4095, 0, None) == B.ERR_UNSUPPORTED
    assert lib.sar_range_compress(16, 0, 16, 1, 16, 8, 128, 0, None) == B.ERR_UNSUPPORTED
    assert lib.sar_range_compress(16, 0, 16, 1, 16, 0, 4096, 0, None) == B.OK   # empty
    assert lib.sar_range_compress(None, 0, 16, 1, 16, 8, 4096, 0, None) == B.ERR_INVALID_ARG
    assert lib.sar_range_compress(17, 0, 16, 1, 16, 8, 4096, 0, None) == B.ERR_MISALIGNED
    assert lib.sar_range_compress(16, 7, 16, 1, 16, 8, 4096, 0, None) == B.ERR_UNSUPPORTED
    assert lib.sar_range_compress(16, 0, 16, 1, 16, 8, 4096, 2, None) == B.ERR_INVALID_ARG
    assert lib.sar_azimuth_compress(16, 0, 3, 16, 1, 16, 4096, 8, None) == B.ERR_INVALID_ARG
    assert lib.sar_azimuth_compress(16, 0, 0, 16, 1, 16, 4096, 0, None) == B.OK
    assert lib.sar_make_filter(16, 100, 1, 16, None) == B.ERR_UNSUPPORTED
    assert lib.sar_make_filter(16, 64, 1, 18, None) == B.ERR_MISALIGNED


def test_fault_injection_plan(lib, monkeypatch):
    monkeypatch.setenv("BFPFFT_FAULT", "plan")
    with pytest.raises(B.BfpfftError) as e:
        B.bfpfft_plan_create(4096, 4, B.F16_BFP, B.FORWARD)
    assert e.value.status == B.ERR_CUDA


def test_fault_injection_alloc(lib, monkeypatch):
    """BFPFFT_FAULT=alloc: plan creation reports OOM before touching a GPU."""
    import numpy as np
    monkeypatch.setenv("BFPFFT_FAULT", "alloc")
    with pytest.raises(B.BfpfftError) as e:
        B.bfpfft_plan_create(4096, 4, B.F16_BFP, B.FORWARD)
    assert e.value.status == B.ERR_OOM
    with pytest.raises(B.BfpfftError) as e:
        B.bfpfft_plan_create_many(np.array([256, 4096]), np.array([0, 256]), B.F16_BFP, B.FORWARD)
    assert e.value.status == B.ERR_OOM


def test_uneven_offsets_must_be_multiples_of_16(lib):
    """Uneven plans refuse a line offset that is not a multiple of 16 points
    (the kernels' bulk L2 prefetches need 16-byte-aligned lines) before any
    device work."""
    import numpy as np
    with pytest.raises(B.BfpfftError) as e:
        B.bfpfft_plan_create_many(np.array([256, 4096]), np.array([0, 264]), B.F16_BFP, B.FORWARD)
    assert e.value.status == B.ERR_INVALID_ARG


def test_fault_injection_launch(lib, monkeypatch):
    """BFPFFT_FAULT=launch: every plan-less call fails its launch with ERR_CUDA after
    checking its arguments and before any device work (addresses 16 are fake)."""
    monkeypatch.setenv("BFPFFT_FAULT", "launch")
    assert lib.sar_range_compress(16, 0, 16, 1, 16, 8, 4096, 0, None) == B.ERR_CUDA
    assert lib.sar_range_compress(16, 0, 16, 1, 16, 8, 4096, 1, None) == B.ERR_CUDA
    assert lib.sar_azimuth_compress(16, 1, 1, 16, 1, 16, 4096, 8, None) == B.ERR_CUDA
    assert lib.sar_make_filter(16, 4096, 1, 32, None) == B.ERR_CUDA
    ws = 1 << 26
    assert lib.sar_autofocus_grad(16, 1, 16, 16, 4096, 8, 16, 16, 16, ws, None) == B.ERR_CUDA
    assert lib.sar_point_target_metrics(16, 1, 64, 64, 16, 1, 8, 16, 16, 1 << 30, None) == B.ERR_CUDA
    assert lib.bfp_sqnr_sums(16, 0, 16, 1, 100, 16, 16, 1 << 20, None) == B.ERR_CUDA
    # argument errors still come first
    assert lib.sar_range_compress(None, 0, 16, 1, 16, 8, 4096, 0, None) == B.ERR_INVALID_ARG
    assert lib.sar_range_compress(16, 0, 16, 1, 16, 8, 4095, 0, None) == B.ERR_UNSUPPORTED


def test_status_and_flag_argument_checks(lib):
    import ctypes
    st = ctypes.c_int(-1)
    assert lib.bfpfft_plan_status(None, ctypes.byref(st)) == B.ERR_INVALID_ARG
    assert lib.bfpfft_plan_set_flags(None, B.CHECK_FINITE) == B.ERR_INVALID_ARG
    assert lib.bfpfft_plan_set_many_schedule(None, 0, B.MANY_PER_LENGTH) == B.ERR_INVALID_ARG
    assert lib.bfpfft_plan_selftest_wait(None, None) == B.ERR_INVALID_ARG
    assert lib.bfpfft_device_status(None) == B.ERR_INVALID_ARG


def test_adaptive_argument_checks(lib):
    """Adaptive exponents: lengths above 16384 and bad dtypes are refused before any device work."""
    with pytest.raises(B.BfpfftError) as e:
        B.bfpfft_plan_create(32768, 4, B.F16_ADAPTIVE, B.FORWARD)
    assert e.value.status == B.ERR_UNSUPPORTED
    sf = lib.bfp_spectral_filter
    assert sf(16, B.F32, 16, 0, 16, B.F32, 4096, 0, B.ARITH_F32, None) == B.OK                 # no lines
    assert sf(16, B.F32, 16, 0, 16, B.F32, 4096, -1, B.ARITH_F32, None) == B.ERR_INVALID_ARG
    assert sf(16, B.F32, 16, 7, 16, B.F32, 4096, 4, B.ARITH_F32, None) == B.ERR_INVALID_ARG    # stride not 0 or n
    assert sf(16, B.F32, 16, 4096, 16, B.F32, 4096, 4, 9, None) == B.ERR_INVALID_ARG            # unknown arith
    assert sf(16, B.F32, 16, 0, 16, B.F32, 128, 4, B.ARITH_F32, None) == B.ERR_UNSUPPORTED      # n below 256
    assert sf(16, B.E4M3_BFP, 16, 0, 16, B.F32, 4096, 4, B.ARITH_F32, None) == B.ERR_UNSUPPORTED
    assert sf(16, B.F32, 16, 0, 16, B.F32, 4096, 4, B.ARITH_F16, None) == B.ERR_UNSUPPORTED     # FP16 mode, FP32 out
    assert sf(16, B.F32, 16, 0, 16, B.F16_BFP, 2048, 4, B.ARITH_F16_MUL_F32_ACC, None) == B.ERR_UNSUPPORTED
    assert sf(None, B.F32, 16, 0, 16, B.F32, 4096, 4, B.ARITH_F32, None) == B.ERR_INVALID_ARG
    assert sf(17, B.F32, 16, 0, 16, B.F32, 4096, 4, B.ARITH_F32, None) == B.ERR_MISALIGNED
    assert lib.bfp_spectral_adaptive(16, B.F32, None, 16, 16, 16, 32768, 4, None) == B.ERR_UNSUPPORTED
    assert lib.bfp_spectral_adaptive(16, B.E4M3_BFP, None, 16, 16, 16, 4096, 4, None) == B.ERR_UNSUPPORTED
    assert lib.bfp_spectral_adaptive(16, B.F32, 16, 16, 16, 16, 4096, 4, None) == B.ERR_INVALID_ARG
    assert lib.bfp_spectral_adaptive(16, B.F32, None, 16, 16, 16, 4096, 0, None) == B.OK
    assert lib.bfp_spectral_adaptive(16, B.F32, None, 16, 16, None, 4096, 4, None) == B.ERR_INVALID_ARG
    assert lib.bfp_spectral_adaptive(17, B.F32, None, 16, 16, 16, 4096, 4, None) == B.ERR_MISALIGNED
    assert lib.bfpfft_exec_adaptive(None, 16, None, 16, 16, None) == B.ERR_INVALID_ARG
