"""Geometry generator checks (inputs shared by the oracle and the CUDA path)."""
import numpy as np
import pytest

from paper_2607_00790_gb300 import inputs


def test_disk_geometry():
    c = inputs.disk(64, R=1.7)
    assert abs(c["perimeter"] - 2 * np.pi * 1.7) < 1e-13
    assert np.allclose(c["kappa"], 1 / 1.7)
    assert np.allclose(c["nx"], c["x"] / 1.7) and np.allclose(c["ny"], c["y"] / 1.7)


def test_star_geometry():
    integrate = pytest.importorskip("scipy.integrate")
    c = inputs.star(4096)
    f = lambda t: np.hypot(-1.5 * np.sin(5 * t) * np.cos(t) - (1 + 0.3 * np.cos(5 * t)) * np.sin(t),
                           -1.5 * np.sin(5 * t) * np.sin(t) + (1 + 0.3 * np.cos(5 * t)) * np.cos(t))
    L, _ = integrate.quad(f, 0, 2 * np.pi, limit=400, epsabs=1e-13)
    assert abs(c["perimeter"] - L) < 1e-11
    assert abs(np.hypot(c["nx"], c["ny"]) - 1).max() < 1e-14
    # normal orthogonal to the chord of neighbouring nodes (to O(h^2))
    tx = np.roll(c["x"], -1) - np.roll(c["x"], 1)
    ty = np.roll(c["y"], -1) - np.roll(c["y"], 1)
    assert np.max(np.abs(tx * c["nx"] + ty * c["ny"]) / np.hypot(tx, ty)) < 1e-3
    # total curvature of a simple closed curve is 2 pi
    assert abs(np.sum(c["kappa"] * c["w"]) - 2 * np.pi) < 1e-10


def test_density_wavenumber():
    c = inputs.star(16384)
    assert abs(inputs.k0_for_density(c) - 761.09) < 0.01


def test_ellipse_and_fourier():
    e = inputs.ellipse(512, 1.2, 0.7)
    assert abs(np.sum(e["kappa"] * e["w"]) - 2 * np.pi) < 1e-10
    a, b = inputs.shape_coefficients(1)
    f = inputs.fourier(1024, a, b)
    assert abs(np.sum(f["kappa"] * f["w"]) - 2 * np.pi) < 1e-8


def test_batched_manifest_seeded():
    m1 = inputs.batched_manifest(0)
    m2 = inputs.batched_manifest(0)
    assert m1 == m2 and len(m1) == 64
    assert all(2048 <= s["N"] <= 32768 and 1.2 <= s["n"] <= 2.0 for s in m1)
