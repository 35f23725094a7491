"""GPU FP64 metric reductions (bfp_sqnr_sums) against the oracle's SQNR (Section IV-B)."""

import numpy as np
import pytest

from oracle import metrics
from paper_2605_28451_gb300 import bfpfft as B
from paper_2605_28451_gb300 import build

from _helpers import storage_round, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib(cuda_ready):
    build.build()
    B.lib()


def gpu_sums(ref, ref_dtype, test, test_dtype):
    import torch
    r = to_device(ref, ref_dtype)
    t = to_device(test, test_dtype)
    ws_bytes = B.bfp_sqnr_workspace_bytes()
    ws = torch.empty(ws_bytes // 8, dtype=torch.float64, device="cuda:0")
    out = torch.empty(8, dtype=torch.float64, device="cuda:0")
    B.bfp_sqnr_sums(r, ref_dtype, t, test_dtype, ref.size, out, ws, ws_bytes)
    torch.cuda.synchronize()
    return out[:5].cpu().numpy()


@pytest.mark.parametrize("count", [1, 1000, 4096 * 33 + 7, 1 << 22])
@pytest.mark.parametrize("ref_dtype,test_dtype", [(B.F32, B.F16_BFP), (B.F16_BFP, B.F16_BFP), (B.F32, B.F32)])
def test_sums_match_oracle(count, ref_dtype, test_dtype):
    rng = np.random.default_rng(count)
    y = rng.standard_normal(count) + 1j * rng.standard_normal(count)
    ref = storage_round(y, ref_dtype)
    test = storage_round(0.7 * y + 1e-3 * (rng.standard_normal(count) + 1j * rng.standard_normal(count)), test_dtype)
    s = gpu_sums(ref, ref_dtype, test, test_dtype)
    exact = [np.sum(np.abs(ref) ** 2), np.sum(np.abs(test) ** 2), np.vdot(test, ref).real,
             np.sum(np.abs(ref - test) ** 2), 0.0]
    assert np.allclose(s, exact, rtol=1e-10, atol=0)
    q = B.sqnr_from_sums(s)
    assert q["aligned_db"] == pytest.approx(metrics.sqnr_db(ref, test), abs=1e-6)
    assert q["unaligned_db"] == pytest.approx(metrics.sqnr_db(ref, test, align=False), abs=1e-6)


def test_nonfinite_counted_and_excluded():
    ref = np.ones(100, complex)
    test = np.ones(100, complex)
    test[[3, 50]] = np.inf
    test[7] = np.nan
    s = gpu_sums(ref, B.F32, test, B.F16_NAIVE)
    assert s[4] == 3
    assert s[0] == 97 and s[3] == 0


def test_empty_count_writes_zeros():
    import torch
    ws = torch.empty(B.bfp_sqnr_workspace_bytes() // 8, dtype=torch.float64, device="cuda:0")
    out = torch.full((8,), 7.0, dtype=torch.float64, device="cuda:0")
    buf = torch.zeros(16, dtype=torch.complex64, device="cuda:0")
    B.bfp_sqnr_sums(buf, B.F32, buf, B.F32, 0, out, ws, B.bfp_sqnr_workspace_bytes())
    torch.cuda.synchronize()
    assert out[:5].abs().sum().item() == 0.0


def test_reproducible():
    rng = np.random.default_rng(1)
    y = rng.standard_normal(1 << 20) + 1j * rng.standard_normal(1 << 20)
    a = gpu_sums(y, B.F32, y * 0.9, B.F16_BFP)
    b = gpu_sums(y, B.F32, y * 0.9, B.F16_BFP)
    assert np.array_equal(a, b)
