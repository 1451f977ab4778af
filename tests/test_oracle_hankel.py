"""Pins for the oracle's Hankel values H0^(1), H1^(1) (std::cyl_bessel_jl / cyl_neumannl).

Checked against an independent arbitrary-precision library (mpmath, 40 digits) and against
the Wronskian J1 Y0 - J0 Y1 = 2/(pi z) (a weak check: it holds even when values are off).
"""
import numpy as np
import pytest

import oracle

# Accuracy the long-double libstdc++ functions reach, per range of z (relative, |H|).
BOUNDS = [(1e-4, 1.0, 1e-15), (1.0, 10.0, 1e-15), (10.0, 100.0, 2e-15),
          (100.0, 1e3, 2e-14), (1e3, 1e4, 1e-13), (1e4, 1e5, 1e-12)]


@pytest.mark.parametrize("lo,hi,tol", BOUNDS)
def test_hankel_vs_mpmath(lo, hi, tol):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    rng = np.random.default_rng(int(lo * 1000) % 1000 + 7)
    z = np.exp(rng.uniform(np.log(lo), np.log(hi), 25))
    h0, h1 = oracle.hankel01(z)
    for zi, a, b in zip(z, h0, h1):
        m0 = complex(mpmath.hankel1(0, mpmath.mpf(float(zi))))
        m1 = complex(mpmath.hankel1(1, mpmath.mpf(float(zi))))
        assert abs(a - m0) <= tol * abs(m0), (zi, a, m0)
        assert abs(b - m1) <= tol * abs(m1), (zi, b, m1)


def test_hankel_vs_scipy_midrange():
    sp = pytest.importorskip("scipy.special")
    z = np.linspace(0.05, 60.0, 997)
    h0, h1 = oracle.hankel01(z)
    assert np.max(np.abs(h0 - sp.hankel1(0, z)) / np.abs(h0)) < 1e-13
    assert np.max(np.abs(h1 - sp.hankel1(1, z)) / np.abs(h1)) < 1e-13


def test_wronskian():
    z = np.exp(np.linspace(np.log(1e-3), np.log(9e4), 2001))
    h0, h1 = oracle.hankel01(z)
    w = h1.real * h0.imag - h0.real * h1.imag
    assert np.max(np.abs(w * (np.pi * z / 2) - 1.0)) < 1e-12


def test_small_argument_limits():
    # H0 ~ 1 + (2i/pi)(ln(z/2) + gamma),  H1 ~ z/2 - 2i/(pi z)  as z -> 0  (A&S 9.1.7-9.1.9)
    z = np.array([1e-6, 1e-5])
    h0, h1 = oracle.hankel01(z)
    g = oracle.EULER_GAMMA
    assert np.allclose(h0, 1 + 2j / np.pi * (np.log(z / 2) + g), rtol=1e-9)
    assert np.allclose(h1, z / 2 - 2j / (np.pi * z), rtol=1e-9)


def test_f1_pole_free():
    # F1(z) = H1(z)/z + 2i/(pi z^2) -> 1/2 + (i/pi)(ln(z/2) + gamma - 1/2)  as z -> 0
    z = np.array([1e-4, 1e-3])
    f = oracle.f1(z)
    g = oracle.EULER_GAMMA
    ref = 0.5 + 1j / np.pi * (np.log(z / 2) + g - 0.5)
    assert np.allclose(f, ref, rtol=1e-6)
    # and equals the plain definition where no cancellation occurs
    z = np.array([3.0, 17.0, 250.0])
    h0, h1 = oracle.hankel01(z)
    assert np.allclose(f := oracle.f1(z), h1 / z + 2j / (np.pi * z * z), rtol=1e-14, atol=0)
