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


def gpu_point_metrics(img, dtype, targets, guard=96):
    import torch
    n_az, n_rg = img.shape
    d = to_device(img, dtype)
    t = torch.tensor([[e, r] for e, r, _ in targets], dtype=torch.int32, device="cuda:0")
    out = torch.empty((len(targets), 12), dtype=torch.float64, device="cuda:0")
    wsb = B.sar_point_target_workspace_bytes(n_az, n_rg)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda:0")
    B.sar_point_target_metrics(d, dtype, n_az, n_rg, t, len(targets), guard, out, ws, wsb)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("dtype", [B.F32, B.F16_BFP])
def test_point_target_metrics_match_oracle(dtype):
    """Section VI metrics computed on the GPU in FP64 equal the oracle's
    (same definitions, FP64 on both sides) to 1e-6 dB / 1e-6 cell."""
    from oracle import sar
    from paper_2605_28451_gb300 import synth
    sc = synth.point_target_scene(1024, 2048, aperture=512)
    hr = sar.matched_filter(sc.ref_range, False)
    ha = sar.matched_filter(sc.ref_azimuth, True)
    img = storage_round(sar.range_doppler_image(sc.raw, hr, ha), dtype)
    ref = metrics.point_target_metrics(img, sc.targets)
    got = gpu_point_metrics(img, dtype, sc.targets)
    for m, g in zip(ref, got):
        assert (int(g[9]), int(g[10])) == m["peak_cell"]
        for i, key in enumerate(("pslr_range_db", "pslr_azimuth_db", "islr_range_db", "islr_azimuth_db",
                                 "width_range_cells", "width_azimuth_cells")):
            assert g[i] == pytest.approx(m[key], abs=1e-6), key
        assert g[6] == pytest.approx(m["peak"], rel=1e-9)
        assert g[7] == pytest.approx(m["snr_db"], abs=1e-6)


def test_point_target_metrics_closed_form():
    """Noise-free single target: PSLR -13.26 dB and the unweighted 3 dB widths
    (0.886 fs/B range cells, 0.886/0.8 azimuth cells), on the GPU."""
    from oracle import sar
    from paper_2605_28451_gb300 import synth
    t = [(512, 1024, 1.0)]
    sc = synth.point_target_scene(1024, 2048, aperture=512, noise=False, targets=t)
    hr = sar.matched_filter(sc.ref_range, False)
    ha = sar.matched_filter(sc.ref_azimuth, True)
    img = sar.range_doppler_image(sc.raw, hr, ha)
    g = gpu_point_metrics(img, B.F32, t)[0]
    assert g[0] == pytest.approx(-13.26, abs=0.2) and g[1] == pytest.approx(-13.26, abs=0.2)
    assert g[4] == pytest.approx(0.886 * 1.2, rel=0.02) and g[5] == pytest.approx(0.886 / 0.8, rel=0.02)
