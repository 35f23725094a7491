"""Failure detection on the GPU: plan-owned status words, the non-finite output
check of BFPFFT_CHECK_FINITE, a bounded device wait driven to expiry, and the
host-injected faults of BFPFFT_FAULT on a live device.

Nothing here faults or hangs the GPU: the expired wait is the library's own
one-second bound on a barrier no copy will complete (the kernel records the
timeout and returns), and the other failures are made on the host.
"""

import numpy as np
import pytest

from oracle import fft as F
from oracle import metrics
from paper_2605_28451_gb300 import bfpfft as B
from paper_2605_28451_gb300 import build, synth

from _helpers import empty_like_storage, from_device, storage_round, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib(cuda_ready):
    build.build()
    B.lib()


def _run(plan, x, dtype):
    import torch
    out = torch.empty_like(x)
    B.bfpfft_exec(plan, x, out)
    torch.cuda.synchronize()
    return from_device(out, dtype)


def test_clean_exec_reports_ok():
    n, batch = 4096, 8
    x = to_device(storage_round(synth.complex_gaussian(batch, n, seed=0), B.F16_BFP), B.F16_BFP)
    p = B.bfpfft_plan_create(n, batch, B.F16_BFP, B.FORWARD)
    B.bfpfft_plan_set_flags(p, B.CHECK_FINITE)
    _run(p, x, B.F16_BFP)
    assert B.bfpfft_plan_status(p) == B.OK


@pytest.mark.parametrize("n", [256, 4096, 16384])
def test_naive_inverse_reports_nonfinite_bfp_does_not(n):
    """A flat spectrum of height 100: the unnormalised inverse peaks at 100 N
    (>= 65520 for N >= 1024, and 25600 at N = 256), the shifted inverse at 100."""
    batch = 4
    spec = np.full((batch, n), 100.0 + 0.0j)
    x = to_device(spec, B.F16_BFP)
    naive = B.bfpfft_plan_create(n, batch, B.F16_NAIVE, B.INVERSE)
    bfp = B.bfpfft_plan_create(n, batch, B.F16_BFP, B.INVERSE)
    for p in (naive, bfp):
        B.bfpfft_plan_set_flags(p, B.CHECK_FINITE)
    y_naive = _run(naive, x, B.F16_NAIVE)
    y_bfp = _run(bfp, x, B.F16_BFP)
    overflow = 100.0 * n >= 65520
    assert (B.bfpfft_plan_status(naive) == B.ERR_NONFINITE) == overflow
    assert (not np.all(np.isfinite(y_naive))) == overflow
    assert B.bfpfft_plan_status(bfp) == B.OK
    expect = F.ifft(spec)
    assert metrics.sqnr_db(expect, y_bfp) >= 55.0


def test_check_is_off_without_the_flag():
    n, batch = 4096, 2
    x = to_device(np.full((batch, n), 100.0 + 0.0j), B.F16_BFP)
    p = B.bfpfft_plan_create(n, batch, B.F16_NAIVE, B.INVERSE)
    y = _run(p, x, B.F16_NAIVE)
    assert not np.all(np.isfinite(y))
    assert B.bfpfft_plan_status(p) == B.OK
    B.bfpfft_plan_set_flags(p, B.CHECK_FINITE)
    _run(p, x, B.F16_NAIVE)
    assert B.bfpfft_plan_status(p) == B.ERR_NONFINITE
    assert B.bfpfft_plan_status(p) == B.OK        # read and cleared


@pytest.mark.parametrize("n", [32768, 65536])
def test_fourstep_overflow_reported(n):
    """FP16 forward of a constant line of 1.5: X[0] = 1.5 n, which reaches 65520
    at n = 65536 only (four-step kernel with the output exchange)."""
    batch = 2
    x = to_device(np.full((batch, n), 1.5 + 0.0j), B.F16_BFP)
    p = B.bfpfft_plan_create(n, batch, B.F16_BFP, B.FORWARD)
    B.bfpfft_plan_set_flags(p, B.CHECK_FINITE)
    y = _run(p, x, B.F16_BFP)
    overflow = 1.5 * n >= 65520
    assert (B.bfpfft_plan_status(p) == B.ERR_NONFINITE) == overflow
    assert (not np.all(np.isfinite(y))) == overflow


@pytest.mark.parametrize("line", [1, 2])
def test_uneven_plan_reports_nonfinite(line):
    """Uneven batch: a constant line of 60 makes the DC bin 60 n >= 65520 -- in
    the 16384-point line (four-step, direct strided store) or in a 4096-point
    line (CTA-local); every other line stays finite."""
    import torch
    lengths = [65536, 16384, 4096, 256, 4096]
    offs = np.concatenate([[0], np.cumsum(lengths)[:-1]]).astype(np.int64)
    total = int(sum(lengths))
    data = storage_round(synth.complex_gaussian(1, total, seed=30)[0], B.F16_BFP)
    p = B.bfpfft_plan_create_many(lengths, offs, B.F16_BFP, B.FORWARD)
    B.bfpfft_plan_set_flags(p, B.CHECK_FINITE)
    x = to_device(data, B.F16_BFP)
    out = torch.empty_like(x)
    B.bfpfft_exec(p, x, out)
    assert B.bfpfft_plan_status(p) == B.OK
    big = data.copy()
    big[offs[line]:offs[line] + lengths[line]] = 60.0
    B.bfpfft_exec(p, to_device(big, B.F16_BFP), out)
    assert B.bfpfft_plan_status(p) == B.ERR_NONFINITE
    got = from_device(out, B.F16_BFP)
    assert not np.isfinite(got[offs[line]])
    assert np.all(np.isfinite(np.delete(got, offs[line])))


def test_bounded_wait_expires_and_context_survives():
    """The self-test arms a barrier for a copy that is never issued; the bounded
    wait expires after about a second, the plan reads TIMEOUT, a second plan
    stays clean, and the context still computes correct transforms."""
    import time

    import torch
    n, batch = 4096, 4
    a = B.bfpfft_plan_create(n, batch, B.F16_BFP, B.FORWARD)
    b = B.bfpfft_plan_create(n, batch, B.F16_BFP, B.FORWARD)
    t0 = time.time()
    B.bfpfft_plan_selftest_wait(a)
    torch.cuda.synchronize()
    waited = time.time() - t0
    assert B.bfpfft_plan_status(a) == B.ERR_TIMEOUT
    assert B.bfpfft_plan_status(b) == B.OK
    assert B.bfpfft_plan_status(a) == B.OK        # read and cleared
    assert 0.5 <= waited <= 30.0
    xs = storage_round(synth.complex_gaussian(batch, n, seed=1), B.F16_BFP)
    y = _run(a, to_device(xs, B.F16_BFP), B.F16_BFP)
    assert metrics.sqnr_db(F.fft(xs), y) >= 55.0
    assert B.bfpfft_plan_status(a) == B.OK


def test_injected_launch_and_alloc_faults_leave_the_library_usable(monkeypatch):
    import torch
    n, batch = 4096, 4
    xs = storage_round(synth.complex_gaussian(batch, n, seed=2), B.F16_BFP)
    x = to_device(xs, B.F16_BFP)
    p = B.bfpfft_plan_create(n, batch, B.F16_BFP, B.FORWARD)
    out = torch.empty_like(x)
    monkeypatch.setenv("BFPFFT_FAULT", "launch")
    with pytest.raises(B.BfpfftError) as e:
        B.bfpfft_exec(p, x, out)
    assert e.value.status == B.ERR_CUDA
    monkeypatch.setenv("BFPFFT_FAULT", "alloc")
    # the split corner turn draws scratch from the library's pool: injected OOM
    raw = to_device(np.ones((8, n)), B.F32)
    hr = to_device(np.ones(n), B.F32)
    rc = empty_like_storage((n, 8), B.F16_BFP)
    with pytest.raises(B.BfpfftError) as e:
        B.sar_range_compress(raw, B.F32, rc, B.F16_BFP, hr, 8, n, True)
    assert e.value.status == B.ERR_OOM
    with pytest.raises(B.BfpfftError) as e:
        B.bfpfft_plan_create(n, batch, B.F16_BFP, B.INVERSE)
    assert e.value.status == B.ERR_OOM
    monkeypatch.delenv("BFPFFT_FAULT")
    B.bfpfft_exec(p, x, out)
    torch.cuda.synchronize()
    assert metrics.sqnr_db(F.fft(xs), from_device(out, B.F16_BFP)) >= 55.0
    B.sar_range_compress(raw, B.F32, rc, B.F16_BFP, hr, 8, n, True)
    torch.cuda.synchronize()
    assert B.bfpfft_plan_status(p) == B.OK
    assert B.bfpfft_device_status() == B.OK
