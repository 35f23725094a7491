"""Pins for the FP64 oracle FFT (CPU only).

Each check is fixed by the mathematics of the DFT, not by the oracle itself:
the defining sum evaluated directly, Parseval, impulse and constant spectra,
the shift theorem, the inverse round trip, an independent library FFT, and
the identities the paper relies on (conj-FFT-conj inverse, Section III-B;
the 1/N shift moved in front of the inverse, Eq. 1).  A final group plants
plausible mistakes in a copy of the oracle and checks a pin catches each.
"""

import json
import os

import numpy as np
import pytest

from oracle import fft as F
from paper_2605_28451_gb300 import synth

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _rand(batch, n, seed=11):
    return synth.complex_gaussian(batch, n, seed)


@pytest.mark.parametrize("n", [1, 2, 4, 8, 16, 32, 64, 256])
def test_fft_matches_defining_sum(n):
    x = _rand(3, n)
    ref = F.dft_bruteforce(x, -1)
    assert np.linalg.norm(F.fft(x) - ref) <= 1e-12 * max(1.0, np.linalg.norm(ref))


@pytest.mark.parametrize("n", [2, 16, 64, 128])
def test_inverse_matches_defining_sum(n):
    x = _rand(2, n, 12)
    ref = F.dft_bruteforce(x, +1) / n
    assert np.linalg.norm(F.ifft(x) - ref) <= 1e-12 * np.linalg.norm(ref)


@pytest.mark.parametrize("n", [16, 512, 4096])
def test_parseval(n):
    x = _rand(4, n, 13)
    X = F.fft(x)
    lhs = np.sum(np.abs(X) ** 2, axis=-1)
    rhs = n * np.sum(np.abs(x) ** 2, axis=-1)
    assert np.allclose(lhs, rhs, rtol=1e-12)


@pytest.mark.parametrize("n0", [0, 1, 5, 1000])
def test_impulse_gives_flat_spectrum(n0):
    n = 4096
    x = np.zeros(n, complex)
    x[n0] = 1.0
    X = F.fft(x)
    assert np.allclose(np.abs(X), 1.0, atol=1e-12)
    k = np.arange(n)
    assert np.allclose(X, np.exp(-2j * np.pi * ((n0 * k) % n) / n), atol=1e-12)


def test_constant_gives_scaled_impulse():
    n = 4096
    X = F.fft(np.full(n, 2.5 - 1j))
    expect = np.zeros(n, complex)
    expect[0] = n * (2.5 - 1j)
    assert np.max(np.abs(X - expect)) <= 1e-9


@pytest.mark.parametrize("n", [64, 4096])
def test_round_trip(n):
    x = _rand(3, n, 14)
    assert np.max(np.abs(F.ifft(F.fft(x)) - x)) <= 1e-13


@pytest.mark.parametrize("shift", [1, 7, 300])
def test_shift_theorem(shift):
    n = 1024
    x = _rand(1, n, 15)[0]
    k = np.arange(n)
    lhs = F.fft(np.roll(x, shift))
    rhs = np.exp(-2j * np.pi * ((shift * k) % n) / n) * F.fft(x)
    assert np.max(np.abs(lhs - rhs)) <= 1e-10


def test_linearity():
    x, y = _rand(1, 256, 16)[0], _rand(1, 256, 17)[0]
    a, b = 0.3 - 2j, -1.7 + 0.5j
    assert np.allclose(F.fft(a * x + b * y), a * F.fft(x) + b * F.fft(y), atol=1e-11)


@pytest.mark.parametrize("n", [16, 4096, 65536])
def test_against_independent_library_fft(n):
    x = _rand(2, n, 18)
    ref = np.fft.fft(x)
    assert np.linalg.norm(F.fft(x) - ref) <= 1e-13 * np.linalg.norm(ref) * np.log2(n)
    assert np.linalg.norm(F.ifft(x) - np.fft.ifft(x)) <= 1e-13 * np.linalg.norm(np.fft.ifft(x)) * np.log2(n)


def test_conj_fft_conj_is_inverse():
    """Section III-B: IFFT(z) = conj(FFT(conj z)), normalised by 1/N."""
    z = _rand(2, 4096, 19)
    assert np.max(np.abs(np.conj(F.fft(np.conj(z))) / 4096 - F.ifft(z))) <= 1e-13


def test_prescaled_inverse_equals_output_scaling():
    """Eq. 1: conj(z) * (1/N) before the transform equals 1/N after it."""
    z = _rand(2, 4096, 20) * 1000.0
    pre = np.conj(F.fft(np.conj(z) * (1.0 / 4096)))
    assert np.max(np.abs(pre - F.ifft(z))) <= 1e-12 * np.max(np.abs(z))


def test_paper_magnitude_growth_worked_example():
    """Section III-B magnitudes for unit-modulus input at N = 4096.

    A constant line drives one forward bin to N = 4096 (the O(N) bound).  The
    discrete chirp x[n] = exp(j pi n^2 / N) has a flat spectrum |X| = sqrt(N);
    its unnormalised matched filter H = conj(X) gives X H = N in every bin, so
    the unnormalised inverse reaches N^2 ~ 1.7e7 (far above 65504), while with
    the 1/N shift in front of the inverse (Eq. 1) the input of the inverse is 1
    and its output N <= 4096 (Fig. 1)."""
    from oracle import sar
    n = GOLDEN["naive_inverse_order_n2"]["n"]
    m = sar.stage_maxima(np.ones(n, complex), np.ones(n, complex))
    assert m["spectrum"] == pytest.approx(GOLDEN["forward_bins_order_n"]["value"], rel=1e-12)
    chirp = np.exp(1j * np.pi * np.arange(n) ** 2 / n)
    spec = F.fft(chirp)
    assert np.allclose(np.abs(spec), np.sqrt(n), rtol=1e-9)
    m = sar.stage_maxima(chirp, np.conj(spec))
    assert m["naive_out"] == pytest.approx(GOLDEN["naive_inverse_order_n2"]["value"],
                                           rel=GOLDEN["naive_inverse_order_n2"]["rel_tol"])
    assert m["naive_out"] > GOLDEN["fp16_max_finite"]["value"]
    assert m["bfp_pre"] == pytest.approx(1.0, rel=1e-9)
    assert m["bfp_out"] == pytest.approx(n, rel=1e-9)
    assert max(m["bfp_pre"], m["bfp_out"]) <= GOLDEN["bfp_bound"]["value"]


def test_non_power_of_two_rejected():
    with pytest.raises(ValueError):
        F.fft(np.ones(12, complex))


# ---- planted mistakes: each must be caught by one of the pins above --------

def _planted(monkeypatch, kind):
    if kind == "no_bit_reversal":
        monkeypatch.setattr(F, "_bit_reverse_indices", lambda n: np.arange(n))
    elif kind == "twiddle_sign":
        orig = F._radix2
        monkeypatch.setattr(F, "_radix2", lambda x, sign: orig(x, -sign))
    elif kind == "dropped_odd_term":
        real_stack = np.stack

        def bad_stack(arrs, axis=0):
            even, odd = arrs
            return real_stack((even + 0.999999 * odd, even - odd), axis=axis)
        monkeypatch.setattr(F.np, "stack", bad_stack)


@pytest.mark.parametrize("kind", ["no_bit_reversal", "twiddle_sign", "dropped_odd_term"])
def test_planted_mistake_is_caught(monkeypatch, kind):
    x = _rand(1, 64, 21)
    ref = F.dft_bruteforce(x, -1)          # computed before the mistake is planted
    _planted(monkeypatch, kind)
    err = np.linalg.norm(F.fft(x) - ref) / np.linalg.norm(ref)
    assert err > 1e-9
