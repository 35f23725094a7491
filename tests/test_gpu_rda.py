"""Range-Doppler imaging with RCMC and range-dependent azimuth filters on the
GPU (sar_rda_image; Section VI's RCMC stage) against the FP64 oracle
(oracle.rda.image) on the migrating scene (exact hyperbolic range history).

Bars: FP32 storage relative L2 <= 1e-5 against FP64 (the filters and the
RCMC phase ramp are generated on the GPU from FP32-evaluated phases after an
FP64 reduction, about 1e-6 of each term); FP16-BFP image SQNR >= 40 dB and
point-target PSLR / ISLR / SNR within 0.1 dB, 3 dB widths within 0.1 cell;
every combination of the RCMC and range-dependent-filter switches matches
the oracle with the same switches.
"""

import numpy as np
import pytest

from oracle import metrics, rda, sar
from paper_2605_28451_gb300 import bfpfft as B
from paper_2605_28451_gb300 import build, synth

from _helpers import empty_like_storage, from_device, storage_round, to_device

pytestmark = pytest.mark.gpu

APERTURE = 1024


@pytest.fixture(scope="module", autouse=True)
def _lib(cuda_ready):
    build.build()
    B.lib()


def geometry_tuple(geo):
    return (geo.range_cell_m, geo.prf_hz, geo.wavelength_m, geo.speed_mps, geo.centre_range_m)


def scene(n_az, n_rg, noise):
    targets = [(n_az // 2, n_rg // 4, 1.0), (n_az // 2 - 300, (3 * n_rg) // 4, 0.5), (n_az // 2 + 350, n_rg // 2, 0.3)]
    sc = synth.migrating_scene(n_az, n_rg, targets, aperture=APERTURE, noise=noise)
    raw = storage_round(sc.raw, B.F32)
    hr64 = storage_round(sar.matched_filter(storage_round(sc.ref_range, B.F32), False), B.F32)
    return sc, raw, hr64, synth.radar_geometry(APERTURE)


def gpu_image(raw, hr64, geo, dtype, flags):
    import torch
    n_az, n_rg = raw.shape
    img = empty_like_storage((n_az, n_rg), dtype)
    B.sar_rda_image(to_device(raw, B.F32), B.F32, img, dtype, to_device(hr64, B.F32), n_az, n_rg, geometry_tuple(geo),
                    APERTURE, flags)
    torch.cuda.synchronize()
    assert B.bfpfft_device_status() == B.OK
    return from_device(img, dtype)


@pytest.fixture(scope="module")
def small():
    return scene(2048, 1024, noise=False)


@pytest.mark.parametrize("rcmc", [False, True])
@pytest.mark.parametrize("range_dependent", [False, True])
@pytest.mark.parametrize("peak_normalise", [False, True])
def test_fp32_image_matches_the_oracle(small, rcmc, range_dependent, peak_normalise):
    sc, raw, hr64, geo = small
    flags = (B.RDA_RCMC if rcmc else 0) | (B.RDA_RANGE_DEPENDENT if range_dependent else 0) | \
            (B.RDA_PEAK_NORMALISE if peak_normalise else 0)
    got = gpu_image(raw, hr64, geo, B.F32, flags)
    expect = rda.image(raw, hr64, geo, APERTURE, correct_migration=rcmc, range_dependent=range_dependent,
                       peak_normalise=peak_normalise)
    assert metrics.rel_l2(expect, got) <= 1e-5


@pytest.mark.parametrize("n_az,n_rg", [(2048, 1024), (4096, 4096)])
def test_fp16_image_quality_against_fp64(n_az, n_rg):
    sc, raw, hr64, geo = scene(n_az, n_rg, noise=True)
    flags = B.RDA_RCMC | B.RDA_RANGE_DEPENDENT | B.RDA_PEAK_NORMALISE
    got = gpu_image(raw, hr64, geo, B.F16_BFP, flags)
    assert np.all(np.isfinite(got))
    expect = rda.image(raw, hr64, geo, APERTURE, peak_normalise=True)
    assert metrics.sqnr_db(expect, got) >= 40.0
    m_ref = metrics.point_target_metrics(expect, sc.targets)
    m16 = metrics.point_target_metrics(got, sc.targets)
    for a, b in zip(m_ref, m16):
        assert a["peak_cell"] == b["peak_cell"]
        for k in ("pslr_range_db", "pslr_azimuth_db", "islr_range_db", "islr_azimuth_db", "snr_db"):
            assert abs(a[k] - b[k]) <= 0.1, (k, a[k], b[k])
        for k in ("width_range_cells", "width_azimuth_cells"):
            assert abs(a[k] - b[k]) <= 0.1, (k, a[k], b[k])


def test_migration_correction_focuses_where_the_plain_chain_does_not(small):
    """The off-centre targets' peaks: with RCMC and range-dependent filters the
    GPU image reaches the oracle's focused peaks; the migration-free chain
    (sar_range_compress + sar_azimuth_compress with the centre-range filter)
    stays below them."""
    import torch
    sc, raw, hr64, geo = small
    n_az, n_rg = raw.shape
    focused = gpu_image(raw, hr64, geo, B.F32, B.RDA_RCMC | B.RDA_RANGE_DEPENDENT | B.RDA_PEAK_NORMALISE)
    ha64 = storage_round(rda.azimuth_filters(n_az, 1, APERTURE, geo, True, range_dependent=False)[:, 0], B.F32)
    rc = empty_like_storage((n_rg, n_az), B.F32)
    img = empty_like_storage((n_az, n_rg), B.F32)
    B.sar_range_compress(to_device(raw, B.F32), B.F32, rc, B.F32, to_device(hr64, B.F32), n_az, n_rg, True)
    B.sar_azimuth_compress(rc, B.F32, 1, img, B.F32, to_device(ha64, B.F32), n_az, n_rg)
    torch.cuda.synchronize()
    plain = from_device(img, B.F32)
    m_f = metrics.point_target_metrics(focused, sc.targets, guard=8)
    m_p = metrics.point_target_metrics(plain, sc.targets, guard=8)
    assert m_f[1]["peak"] > 1.2 * m_p[1]["peak"]      # 3/4 of the swath out: k_a is off by 2 %


def test_argument_checks():
    import torch
    x = torch.zeros((256, 256), dtype=torch.complex64, device="cuda:0")
    h = torch.zeros(256, dtype=torch.complex64, device="cuda:0")
    geo = geometry_tuple(synth.radar_geometry(APERTURE))
    with pytest.raises(B.BfpfftError) as e:
        B.sar_rda_image(x, B.F32, x, B.F16_BFP, h, 256, 256, geo, 128, B.RDA_RCMC)   # FP16 needs peak normalise
    assert e.value.status == B.ERR_UNSUPPORTED
    with pytest.raises(B.BfpfftError) as e:
        B.sar_rda_image(x, B.F32, x, B.F32, h, 256, 256, geo, 512, 0)                 # aperture > n_az
    assert e.value.status == B.ERR_INVALID_ARG
    with pytest.raises(B.BfpfftError) as e:
        B.sar_rda_image(x, B.F32, x, B.F32, h, 256, 128, geo, 128, 0)
    assert e.value.status == B.ERR_UNSUPPORTED
    bad = (geo[0], 1e9, geo[2], geo[3], geo[4])                                          # lambda PRF / 4v >= 1
    with pytest.raises(B.BfpfftError) as e:
        B.sar_rda_image(x, B.F32, x, B.F32, h, 256, 256, bad, 128, 0)
    assert e.value.status == B.ERR_INVALID_ARG
