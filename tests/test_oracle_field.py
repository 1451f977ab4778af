"""Pins of the oracle's field evaluation off the curve (integral representations): with the
exact Mie boundary values of the disk as densities, the represented field must equal the Mie
series field inside and outside (spectral accuracy away from the curve), and a planted sign
error in the exterior representation is caught."""
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from oracle.build import HERE
from paper_2607_00790_gb300 import inputs


def field_error(N=256, R=1.0):
    c = inputs.disk(N, R)
    ph = oracle.Physics(2 * np.pi, n=1.5)
    u, q = oracle.mie_boundary(R, ph, c["t"])
    rng = np.random.default_rng(1)
    rr = np.concatenate([rng.uniform(0.1, 0.8, 20), rng.uniform(1.2, 3.0, 20)])
    tt = rng.uniform(0, 2 * np.pi, 40)
    px, py = rr * np.cos(tt), rr * np.sin(tt)
    val, inside = oracle.field(c, ph, u, q, px, py)
    ex = oracle.mie_field(R, ph, px, py)
    return np.max(np.abs(val[:, 0] - ex)) / np.max(np.abs(ex)), np.all(inside == (rr < R))


def test_field_matches_mie_series():
    err, sides = field_error()
    assert sides
    assert err < 1e-12, err


def test_field_of_the_dense_solution_converges():
    """Densities from the dense Nystrom solve: the field error follows the O(h^3) density error."""
    errs = []
    for N in (64, 128, 256):
        c = inputs.disk(N)
        ph = oracle.Physics(2 * np.pi, n=1.5)
        x = oracle.dense_solve(oracle.wsbm_dense(c, ph), oracle.rhs_planewave(c, ph, [0.0]))
        u, q = oracle.split_uq(x)
        px = np.array([0.3, -0.5, 2.0, 0.0])
        py = np.array([0.2, 0.1, 1.0, -2.5])
        val, _ = oracle.field(c, ph, u, q, px, py)
        ex = oracle.mie_field(1.0, ph, px, py)
        errs.append(np.max(np.abs(val[:, 0] - ex)) / np.max(np.abs(ex)))
    assert errs[1] / errs[2] > 6.0 and errs[0] / errs[1] > 6.0, errs


def test_planted_representation_sign_is_caught():
    src = open(os.path.join(HERE, "wsbm_oracle.cpp")).read()
    old = "          acc += w[j] * (Dy * uj - eps0 * G * qj);"
    assert src.count(old) == 1
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "m.cpp")
        open(path, "w").write(src.replace(old, "          acc += w[j] * (-Dy * uj - eps0 * G * qj);"))
        so = os.path.join(d, "libm.so")
        subprocess.run(["g++", "-std=c++17", "-O1", "-fPIC", "-shared", "-fopenmp",
                        "-ffp-contract=off", "-o", so, path], check=True)
        with oracle.use_library(so):
            err, _ = field_error()
            assert err > 1e-6
