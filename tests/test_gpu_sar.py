"""GPU parity of the SAR range-Doppler compression against the FP64 oracle.

Stated against FP64: FP32 paths to relative L2 <= 1e-6; FP16-BFP outputs per
element within half an FP16 ulp plus the FP32 arithmetic error; end-to-end
FP16 image SQNR >= 40 dB; PSLR / ISLR / SNR within 0.1 dB and 3 dB widths
within 0.1 cell of the oracle's image (Section VI, Table III).  The naive
unshifted FP16 path must produce Inf or NaN (Section III-B).
"""

import numpy as np
import pytest

from oracle import metrics, sar
from paper_2605_28451_gb300 import bfpfft as B
from paper_2605_28451_gb300 import build, synth

from _helpers import empty_like_storage, fp16_elementwise_ok, from_device, storage_round, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib(cuda_ready):
    build.build()
    B.lib()


@pytest.fixture(params=["split", "fused"])
def sar_turn(request, monkeypatch):
    """Both corner-turn forms: dense rows plus a tiled transpose through
    scratch, or the on-chip turn through cluster shared memory."""
    monkeypatch.setenv("BFPFFT_SAR_TURN", request.param)
    yield request.param
    assert B.bfpfft_device_status() == B.OK


def gpu_filter(ref: np.ndarray, peak_normalise: bool):
    """sar_make_filter on the GPU (checked against the oracle by test_make_filter)."""
    import torch
    n = ref.shape[0]
    r = to_device(ref, B.F32)
    h = torch.empty(n, dtype=torch.complex64, device="cuda:0")
    B.sar_make_filter(r, n, peak_normalise, h)
    torch.cuda.synchronize()
    return h


def oracle_filter(ref: np.ndarray, peak_normalise: bool):
    """The filter spectrum both sides receive: the oracle's FP64 matched filter
    rounded once to FP32.  Returns (device complex64 tensor, the same values in
    complex128 for the oracle), so no oracle input comes from the GPU."""
    h64 = storage_round(sar.matched_filter(storage_round(ref, B.F32), peak_normalise), B.F32)
    return to_device(h64, B.F32), h64


def gpu_range(raw_stored, raw_dtype, out_dtype, hr, transpose=False):
    import torch
    n_az, n_rg = raw_stored.shape
    x = to_device(raw_stored, raw_dtype)
    out = empty_like_storage((n_rg, n_az) if transpose else (n_az, n_rg), out_dtype)
    B.sar_range_compress(x, raw_dtype, out, out_dtype, hr, n_az, n_rg, transpose)
    torch.cuda.synchronize()
    return from_device(out, out_dtype)


def gpu_azimuth(rc_stored, rc_dtype, layout, img_dtype, ha, n_az, n_rg):
    import torch
    x = to_device(rc_stored, rc_dtype)
    img = empty_like_storage((n_az, n_rg), img_dtype)
    B.sar_azimuth_compress(x, rc_dtype, layout, img, img_dtype, ha, n_az, n_rg)
    torch.cuda.synchronize()
    return from_device(img, img_dtype)


@pytest.mark.parametrize("n", [256, 4096, 16384])
@pytest.mark.parametrize("norm", [False, True])
def test_make_filter(n, norm):
    ref = synth.centred_reference(synth.range_chirp()[: min(480, n // 2)], n)
    h = gpu_filter(ref, norm).cpu().numpy().astype(np.complex128)
    expect = sar.matched_filter(storage_round(ref, B.F32), norm)
    assert metrics.rel_l2(expect, h) <= 1e-6


@pytest.mark.parametrize("n_az", [8, 45])
@pytest.mark.parametrize("n_rg", [256, 512, 1024, 2048, 4096, 8192, 16384])
@pytest.mark.parametrize("transpose", [False, True])
@pytest.mark.parametrize("raw_dtype,out_dtype", [(B.F32, B.F32), (B.F32, B.F16_BFP), (B.F16_BFP, B.F16_BFP),
                                                 (B.F16_BFP, B.F32)])
def test_range_compress(n_az, n_rg, transpose, raw_dtype, out_dtype, sar_turn):
    sc = synth.point_target_scene(n_az, n_rg, aperture=16, targets=[(n_az // 2, n_rg // 2, 1.0)],
                                  noise_seed=n_az + n_rg)
    ref_r = synth.centred_reference(synth.range_chirp()[: min(480, n_rg // 2)], n_rg)
    hr, hr64 = oracle_filter(ref_r, False)
    raw = storage_round(sc.raw, raw_dtype)
    got = gpu_range(raw, raw_dtype, out_dtype, hr, transpose)
    if transpose:
        got = got.T
    expect = sar.range_compress(raw, hr64)
    if out_dtype == B.F32:
        assert metrics.rel_l2(expect, got) <= 1e-6
    else:
        ok, worst = fp16_elementwise_ok(got, expect)
        assert ok, worst


@pytest.mark.parametrize("n_az", [256, 1024, 4096, 16384])
@pytest.mark.parametrize("n_rg", [8, 45])
@pytest.mark.parametrize("layout", [0, 1])
@pytest.mark.parametrize("rc_dtype,img_dtype", [(B.F32, B.F32), (B.F16_BFP, B.F16_BFP), (B.F16_BFP, B.F32)])
def test_azimuth_compress(n_az, n_rg, layout, rc_dtype, img_dtype, sar_turn):
    rng = np.random.default_rng(n_az + n_rg)
    rc = rng.standard_normal((n_az, n_rg)) + 1j * rng.standard_normal((n_az, n_rg))
    rc = storage_round(rc, rc_dtype)
    ref_a = synth.centred_reference(synth.azimuth_chirp(min(1024, n_az // 2)), n_az)
    ha, ha64 = oracle_filter(ref_a, True)
    stored = rc if layout == 0 else np.ascontiguousarray(rc.T)
    got = gpu_azimuth(stored, rc_dtype, layout, img_dtype, ha, n_az, n_rg)
    expect = sar.azimuth_compress(rc, ha64)
    if img_dtype == B.F32:
        assert metrics.rel_l2(expect, got) <= 1e-6
    else:
        ok, worst = fp16_elementwise_ok(got, expect)
        assert ok, worst


def _pipeline(raw_c64, hr, ha, n_az, n_rg, dtype):
    """GPU range compression (corner-turned store) then azimuth compression."""
    import torch
    raw = to_device(raw_c64, B.F32)
    rc = empty_like_storage((n_rg, n_az), dtype)
    img = empty_like_storage((n_az, n_rg), dtype)
    B.sar_range_compress(raw, B.F32, rc, dtype, hr, n_az, n_rg, True)
    B.sar_azimuth_compress(rc, B.F16_BFP if dtype != B.F32 else B.F32, 1, img, dtype, ha, n_az, n_rg)
    torch.cuda.synchronize()
    return from_device(img, dtype)


@pytest.fixture(scope="module")
def small_scene():
    n_az, n_rg, ap = 1024, 2048, 512
    sc = synth.point_target_scene(n_az, n_rg, aperture=ap)
    raw = storage_round(sc.raw, B.F32)
    hr, hr64 = oracle_filter(sc.ref_range, False)
    ha, ha64 = oracle_filter(sc.ref_azimuth, True)
    img_ref = sar.range_doppler_image(raw, hr64, ha64)
    return sc, raw, hr, ha, img_ref


def test_end_to_end_fp16_image_quality(small_scene):
    sc, raw, hr, ha, img_ref = small_scene
    n_az, n_rg = raw.shape
    img16 = _pipeline(raw, hr, ha, n_az, n_rg, B.F16_BFP)
    img32 = _pipeline(raw, hr, ha, n_az, n_rg, B.F32)
    assert np.all(np.isfinite(img16))
    assert metrics.sqnr_db(img_ref, img16) >= 40.0
    assert metrics.rel_l2(img_ref, img32) <= 1e-6
    m_ref = metrics.point_target_metrics(img_ref, sc.targets)
    m16 = metrics.point_target_metrics(img16, sc.targets)
    for a, b in zip(m_ref, m16):
        assert a["peak_cell"] == b["peak_cell"]
        for k in ("pslr_range_db", "pslr_azimuth_db", "islr_range_db", "islr_azimuth_db", "snr_db"):
            assert abs(a[k] - b[k]) <= 0.1, (k, a[k], b[k])
        for k in ("width_range_cells", "width_azimuth_cells"):
            assert abs(a[k] - b[k]) <= 0.1, (k, a[k], b[k])


def test_naive_fp16_range_compression_overflows():
    """Config 2 shape: 1024 azimuth lines x 4096 range samples.  The
    unnormalised range inverse peaks at N * M = 1.97e6 > 65504 (Section III-B)."""
    sc = synth.point_target_scene(1024, 4096)
    raw = storage_round(sc.raw, B.F32)
    hr, hr64 = oracle_filter(sc.ref_range, False)
    naive = gpu_range(raw, B.F32, B.F16_NAIVE, hr)
    assert (~np.isfinite(naive)).any()
    m = sar.stage_maxima(raw[sc.targets[0][0]:sc.targets[0][0] + 1], hr64)
    assert m["naive_out"] > 65520.0 and m["bfp_out"] < 65504.0 / 2
    bfp = gpu_range(raw, B.F32, B.F16_BFP, hr)
    assert np.all(np.isfinite(bfp))
    rows = [t[0] for t in sc.targets[:4]]
    expect = sar.range_compress(raw[rows], hr64)
    ok, worst = fp16_elementwise_ok(bfp[rows], expect)
    assert ok, worst


@pytest.fixture(scope="module")
def config3_reference():
    """Config 3 at full size: the 4096 x 4096 point-target scene, its FP32 raw
    echo (what the GPU receives), the FP32-rounded filters, and the oracle's
    FP64 image and point-target metrics of the same inputs."""
    n = 4096
    sc = synth.point_target_scene(n, n)
    raw = storage_round(sc.raw, B.F32)
    hr, hr64 = oracle_filter(sc.ref_range, False)
    ha, ha64 = oracle_filter(sc.ref_azimuth, True)
    img_ref = sar.range_doppler_image(raw, hr64, ha64)
    m_ref = metrics.point_target_metrics(img_ref, sc.targets)
    return sc, raw, hr, ha, img_ref, m_ref


def test_config3_golden_metrics_match_the_oracle(config3_reference):
    """tests/golden/sar_4096_image_metrics.json (which bench.py reports deltas
    against) holds exactly what the oracle computes for the config-3 scene."""
    import json
    import os
    sc, _, _, _, _, m_ref = config3_reference
    with open(os.path.join(os.path.dirname(__file__), "golden", "sar_4096_image_metrics.json")) as f:
        gold = json.load(f)
    assert [tuple(t) for t in gold["targets"]] == [(e, r) for e, r, _ in sc.targets]
    for g, m in zip(gold["metrics"], m_ref):
        for k, v in g.items():
            assert v == pytest.approx(m[k], abs=1e-6), k


@pytest.mark.parametrize("dtype", [B.F16_BFP, B.F32])
def test_config3_full_size_image_against_fp64(config3_reference, dtype, sar_turn):
    """Config 3 at full size, both corner-turn forms: the GPU image against the
    FP64 image of the same inputs -- end-to-end SQNR >= 40 dB over the whole
    image (FP32: relative L2 <= 1e-6), and per target |dPSLR|, |dISLR|, |dSNR|
    <= 0.1 dB, |d3 dB width| <= 0.1 cell, same peak cell."""
    sc, raw, hr, ha, img_ref, m_ref = config3_reference
    n = raw.shape[0]
    img = _pipeline(raw, hr, ha, n, n, dtype)
    assert np.all(np.isfinite(img))
    if dtype == B.F32:
        assert metrics.rel_l2(img_ref, img) <= 1e-6
    assert metrics.sqnr_db(img_ref, img) >= 40.0
    m_gpu = metrics.point_target_metrics(img, sc.targets)
    for a, b in zip(m_ref, m_gpu):
        assert a["peak_cell"] == b["peak_cell"]
        for k in ("pslr_range_db", "pslr_azimuth_db", "islr_range_db", "islr_azimuth_db", "snr_db"):
            assert abs(a[k] - b[k]) <= 0.1, (k, a[k], b[k])
        for k in ("width_range_cells", "width_azimuth_cells"):
            assert abs(a[k] - b[k]) <= 0.1, (k, a[k], b[k])


@pytest.mark.parametrize("n_rg", [256, 4096, 16384])
@pytest.mark.parametrize("transpose", [False, True])
@pytest.mark.parametrize("raw_dtype", [B.F32, B.F16_BFP])
def test_pure_fp16_range_compression(n_rg, transpose, raw_dtype):
    """Section VI's pure FP16 mode (sar_range_compress_arith, BFPFFT_ARITH_F16):
    every transform and the filter product in FP16 arithmetic; SQNR against the
    FP64 oracle of the same stored inputs >= 50 dB per call (two transforms and
    a product, each rounding every operation to FP16)."""
    import torch
    n_az = 45
    sc = synth.point_target_scene(n_az, n_rg, aperture=16, targets=[(n_az // 2, n_rg // 2, 1.0)],
                                  noise_seed=n_az + n_rg)
    ref_r = synth.centred_reference(synth.range_chirp()[: min(480, n_rg // 2)], n_rg)
    hr, hr64 = oracle_filter(ref_r, False)
    raw = storage_round(sc.raw, raw_dtype)
    out = empty_like_storage((n_rg, n_az) if transpose else (n_az, n_rg), B.F16_BFP)
    B.sar_range_compress_arith(to_device(raw, raw_dtype), raw_dtype, out, B.F16_BFP, hr, n_az, n_rg, transpose,
                               B.ARITH_F16)
    torch.cuda.synchronize()
    got = from_device(out, B.F16_BFP)
    if transpose:
        got = got.T
    # the kernel rounds a complex64 echo to FP16 on load: the oracle takes the same values
    expect = sar.range_compress(storage_round(raw, B.F16_BFP), hr64)
    assert metrics.sqnr_db(expect, got) >= 50.0


def test_pure_fp16_naive_range_compression_overflows():
    sc = synth.point_target_scene(1024, 4096)
    raw = storage_round(sc.raw, B.F32)
    hr, _ = oracle_filter(sc.ref_range, False)
    import torch
    out = empty_like_storage((1024, 4096), B.F16_BFP)
    B.sar_range_compress_arith(to_device(raw, B.F32), B.F32, out, B.F16_NAIVE, hr, 1024, 4096, False, B.ARITH_F16)
    torch.cuda.synchronize()
    assert not np.all(np.isfinite(from_device(out, B.F16_BFP)))


def test_config3_pure_fp16_image_against_fp64(config3_reference):
    """Config 3 at full size in the pure FP16 mode (Table III: the paper's pure
    FP16 image keeps PSLR / SNR within 0.1 dB of FP32): SQNR >= 40 dB over the
    whole image, per target |dPSLR|, |dISLR|, |dSNR| <= 0.1 dB, |dwidth| <= 0.1
    cell against the FP64 image, same peak cell."""
    import torch
    sc, raw, hr, ha, img_ref, m_ref = config3_reference
    n = raw.shape[0]
    rc = empty_like_storage((n, n), B.F16_BFP)
    img = empty_like_storage((n, n), B.F16_BFP)
    B.sar_range_compress_arith(to_device(raw, B.F32), B.F32, rc, B.F16_BFP, hr, n, n, True, B.ARITH_F16)
    B.sar_azimuth_compress_arith(rc, B.F16_BFP, 1, img, B.F16_BFP, ha, n, n, B.ARITH_F16)
    torch.cuda.synchronize()
    got = from_device(img, B.F16_BFP)
    assert np.all(np.isfinite(got))
    assert metrics.sqnr_db(img_ref, got) >= 40.0
    m16 = metrics.point_target_metrics(got, sc.targets)
    for a, b in zip(m_ref, m16):
        assert a["peak_cell"] == b["peak_cell"]
        for k in ("pslr_range_db", "pslr_azimuth_db", "islr_range_db", "islr_azimuth_db", "snr_db"):
            assert abs(a[k] - b[k]) <= 0.1, (k, a[k], b[k])
        for k in ("width_range_cells", "width_azimuth_cells"):
            assert abs(a[k] - b[k]) <= 0.1, (k, a[k], b[k])


def test_arith_argument_checks():
    import torch
    x = torch.zeros((8, 4096), dtype=torch.complex64, device="cuda:0")
    h = torch.zeros(4096, dtype=torch.complex64, device="cuda:0")
    with pytest.raises(B.BfpfftError) as e:
        B.sar_range_compress_arith(x, B.F32, x, B.F32, h, 8, 4096, False, B.ARITH_F16)   # FP32 out
    assert e.value.status == B.ERR_UNSUPPORTED
    with pytest.raises(B.BfpfftError) as e:
        B.sar_range_compress_arith(x, B.F32, x, B.F16_BFP, h, 8, 4096, False, 7)
    assert e.value.status == B.ERR_INVALID_ARG
    with pytest.raises(B.BfpfftError) as e:
        B.sar_azimuth_compress_arith(x, B.F32, 1, x, B.F16_BFP, h, 4096, 8, B.ARITH_F16)   # FP32 rc
    assert e.value.status == B.ERR_UNSUPPORTED


def _tc_compress_emulated(x, h64):
    """The tensor-core compression schedule (oracle.emulate.fft_radix16_mma):
    FP16 operands at every pass of the forward transform, its FP32 spectrum
    times the FP32 filter, conj(.) / N rounded to the inverse's FP16 operands,
    the inverse's passes, FP16 output."""
    from oracle import emulate as E
    from oracle import quant as Q
    n = x.shape[-1]
    X = E.fft_radix16_mma(x, store=Q.round_binary32)
    Y = Q.round_binary32(X.real * h64.real - X.imag * h64.imag) + \
        1j * Q.round_binary32(X.real * h64.imag + X.imag * h64.real)
    return np.conj(E.fft_radix16_mma(np.conj(Y) / n))


@pytest.mark.parametrize("transpose", [False, True])
@pytest.mark.parametrize("raw_dtype", [B.F32, B.F16_BFP])
def test_tensor_core_range_compression(transpose, raw_dtype):
    """Table IV's FP16-multiply / FP32-accumulate mode (sar_range_compress_arith
    with BFPFFT_ARITH_F16_MUL_F32_ACC): both transforms on the tensor cores and
    the filter product in FP32 between them.  1300 lines, so persistent CTAs
    take one or two.  Against the FP64 oracle of the stored echo: SQNR >= 55 dB;
    on sampled lines the GPU follows the emulated schedule far more closely
    (>= 6 dB) than the schedule follows the exact result, and lands within
    0.5 dB of its SQNR."""
    import torch
    n_az, n_rg = 1300, 4096
    sc = synth.point_target_scene(n_az, n_rg, aperture=16, targets=[(n_az // 2, n_rg // 2, 1.0)],
                                  noise_seed=7)
    hr, hr64 = oracle_filter(synth.centred_reference(synth.range_chirp()[:480], n_rg), False)
    raw = storage_round(sc.raw, raw_dtype)
    out = empty_like_storage((n_rg, n_az) if transpose else (n_az, n_rg), B.F16_BFP)
    B.sar_range_compress_arith(to_device(raw, raw_dtype), raw_dtype, out, B.F16_BFP, hr, n_az, n_rg, transpose,
                               B.ARITH_F16_MUL_F32_ACC)
    torch.cuda.synchronize()
    assert B.bfpfft_device_status() == B.OK
    got = from_device(out, B.F16_BFP)
    if transpose:
        got = got.T
    expect = sar.range_compress(raw, hr64)
    assert np.all(np.isfinite(got))
    assert metrics.sqnr_db(expect, got) >= 55.0
    rows = [0, 1, 649, 650, 1215, 1216, 1298, 1299]
    emu = _tc_compress_emulated(raw[rows], hr64)
    s_emu = metrics.sqnr_db(expect[rows], emu)
    assert metrics.sqnr_db(emu, got[rows]) >= s_emu + 6.0
    assert abs(metrics.sqnr_db(expect[rows], got[rows]) - s_emu) <= 0.5


@pytest.mark.parametrize("layout", [0, 1])
@pytest.mark.parametrize("rc_dtype", [B.F32, B.F16_BFP])
def test_tensor_core_azimuth_compression(layout, rc_dtype):
    """Azimuth lines of 4096 pulses on the tensor cores, both rc layouts and
    both rc storage types: SQNR >= 55 dB against the FP64 oracle."""
    n_az, n_rg = 4096, 45
    rng = np.random.default_rng(3)
    rc = storage_round(rng.standard_normal((n_az, n_rg)) + 1j * rng.standard_normal((n_az, n_rg)), rc_dtype)
    ha, ha64 = oracle_filter(synth.centred_reference(synth.azimuth_chirp(1024), n_az), True)
    import torch
    x = to_device(rc if layout == 0 else np.ascontiguousarray(rc.T), rc_dtype)
    img = empty_like_storage((n_az, n_rg), B.F16_BFP)
    B.sar_azimuth_compress_arith(x, rc_dtype, layout, img, B.F16_BFP, ha, n_az, n_rg, B.ARITH_F16_MUL_F32_ACC)
    torch.cuda.synchronize()
    got = from_device(img, B.F16_BFP)
    assert metrics.sqnr_db(sar.azimuth_compress(rc, ha64), got) >= 55.0


def test_config3_tensor_core_image_against_fp64(config3_reference):
    """Config 3 at full size in the tensor-core mode: SQNR >= 40 dB over the
    whole image, per target |dPSLR|, |dISLR|, |dSNR| <= 0.1 dB, |dwidth| <= 0.1
    cell against the FP64 image, same peak cell."""
    import torch
    sc, raw, hr, ha, img_ref, m_ref = config3_reference
    n = raw.shape[0]
    rc = empty_like_storage((n, n), B.F16_BFP)
    img = empty_like_storage((n, n), B.F16_BFP)
    mode = B.ARITH_F16_MUL_F32_ACC
    B.sar_range_compress_arith(to_device(raw, B.F32), B.F32, rc, B.F16_BFP, hr, n, n, True, mode)
    B.sar_azimuth_compress_arith(rc, B.F16_BFP, 1, img, B.F16_BFP, ha, n, n, mode)
    torch.cuda.synchronize()
    got = from_device(img, B.F16_BFP)
    assert np.all(np.isfinite(got))
    assert metrics.sqnr_db(img_ref, got) >= 40.0
    m_tc = metrics.point_target_metrics(got, sc.targets)
    for a, b in zip(m_ref, m_tc):
        assert a["peak_cell"] == b["peak_cell"]
        for k in ("pslr_range_db", "pslr_azimuth_db", "islr_range_db", "islr_azimuth_db", "snr_db"):
            assert abs(a[k] - b[k]) <= 0.1, (k, a[k], b[k])
        for k in ("width_range_cells", "width_azimuth_cells"):
            assert abs(a[k] - b[k]) <= 0.1, (k, a[k], b[k])


def test_tensor_core_arith_argument_checks():
    import torch
    x = torch.zeros((8, 4096), dtype=torch.complex64, device="cuda:0")
    h = torch.zeros(4096, dtype=torch.complex64, device="cuda:0")
    mode = B.ARITH_F16_MUL_F32_ACC
    for out_dtype in (B.F32, B.F16_NAIVE):
        with pytest.raises(B.BfpfftError) as e:
            B.sar_range_compress_arith(x, B.F32, x, out_dtype, h, 8, 4096, False, mode)
        assert e.value.status == B.ERR_UNSUPPORTED
    y = torch.zeros((16, 2048), dtype=torch.complex64, device="cuda:0")
    with pytest.raises(B.BfpfftError) as e:
        B.sar_range_compress_arith(y, B.F32, y, B.F16_BFP, h, 16, 2048, False, mode)    # N = 2048
    assert e.value.status == B.ERR_UNSUPPORTED
    with pytest.raises(B.BfpfftError) as e:
        B.sar_azimuth_compress_arith(y, B.F32, 1, y, B.F16_BFP, h, 2048, 16, mode)
    assert e.value.status == B.ERR_UNSUPPORTED


def test_tensor_core_range_compression_from_pinned_host_memory():
    """A pinned host echo read in place by the tensor-core lines (no L2
    prefetch of host memory): the bits of the device-memory call."""
    import torch
    n_az, n_rg = 300, 4096
    sc = synth.point_target_scene(n_az, n_rg, aperture=16, targets=[(n_az // 2, n_rg // 2, 1.0)], noise_seed=9)
    hr, _ = oracle_filter(synth.centred_reference(synth.range_chirp()[:480], n_rg), False)
    dev_raw = to_device(storage_round(sc.raw, B.F32), B.F32)
    host_raw = torch.empty(dev_raw.shape, dtype=dev_raw.dtype, pin_memory=True)
    host_raw.copy_(dev_raw)
    ref = empty_like_storage((n_az, n_rg), B.F16_BFP)
    got = empty_like_storage((n_az, n_rg), B.F16_BFP)
    mode = B.ARITH_F16_MUL_F32_ACC
    B.sar_range_compress_arith(dev_raw, B.F32, ref, B.F16_BFP, hr, n_az, n_rg, False, mode)
    B.sar_range_compress_arith(host_raw, B.F32, got, B.F16_BFP, hr, n_az, n_rg, False, mode)
    torch.cuda.synchronize()
    assert B.bfpfft_device_status() == B.OK
    assert torch.equal(got, ref)
