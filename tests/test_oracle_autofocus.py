"""Pins for the oracle's entropy autofocus and analytic adjoint (CPU only).

* The analytic gradient matches FP64 central finite differences of the
  entropy (which needs no adjoint at all) on sampled pulses.
* A constant phase does not change |I|, so the gradient sums to zero.
* Entropy closed forms: one bright pixel gives 0, K equal pixels give ln K.
* The injected error is the one the gradient corrects: entropy at phi = eps
  is lower than at phi = 0.
"""

import numpy as np
import pytest

from oracle import autofocus as AF
from oracle import sar
from paper_2605_28451_gb300 import synth


@pytest.fixture(scope="module")
def small_case():
    n_az, n_rg, ap = 256, 64, 128
    t = [(128, 20, 1.0), (100, 45, 0.5)]
    sc = synth.point_target_scene(n_az, n_rg, aperture=ap, targets=t)
    ref_r = synth.centred_reference(synth.range_chirp()[:40], n_rg)
    hr = sar.matched_filter(ref_r, False)
    ha = sar.matched_filter(sc.ref_azimuth, True)
    rc = sar.range_compress(sc.raw, hr)
    eps = synth.phase_error(n_az, quad_rad=2.0)
    u = rc * np.exp(1j * eps)[:, None]
    return u, ha, eps


def test_entropy_closed_forms():
    img = np.zeros((8, 8), complex)
    img[3, 4] = 2.0 - 1j
    assert AF.entropy_of(img) == pytest.approx(0.0, abs=1e-15)
    img[:] = 0
    img.flat[:5] = 3.0
    assert AF.entropy_of(img) == pytest.approx(np.log(5.0), rel=1e-14)


def test_gradient_matches_finite_differences(small_case):
    u, ha, _ = small_case
    phi = np.zeros(u.shape[0])
    _, g = AF.entropy_and_grad(u, phi, ha)
    pulses = np.random.default_rng(4).choice(u.shape[0], 16, replace=False)
    fd = AF.central_difference(u, phi, ha, pulses, h=1e-4)
    assert np.linalg.norm(g[pulses] - fd) <= 1e-6 * np.linalg.norm(fd)


def test_gradient_sums_to_zero(small_case):
    u, ha, _ = small_case
    _, g = AF.entropy_and_grad(u, 0.1 * np.arange(u.shape[0]) ** 1.5 / 100, ha)
    assert abs(np.sum(g)) <= 1e-9 * np.linalg.norm(g)


def test_entropy_value_consistent(small_case):
    u, ha, _ = small_case
    phi = np.linspace(0, 1, u.shape[0])
    e, _ = AF.entropy_and_grad(u, phi, ha)
    assert e == pytest.approx(AF.entropy(u, phi, ha), rel=1e-13)


def test_true_phase_focuses(small_case):
    u, ha, eps = small_case
    assert AF.entropy(u, eps, ha) < AF.entropy(u, np.zeros_like(eps), ha)
