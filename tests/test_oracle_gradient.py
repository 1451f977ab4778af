"""Pins of the oracle's shape-gradient part against finite differences.

* The tangent of the Fourier curve's node arrays against central differences of the input
  generator itself.
* The dual-number derivative of lam^T A x (every input kind: positions, normals, weights,
  curvatures, k1, eps1) against central differences of the dense assembly.
* The dense adjoint gradient of the far-field intensity misfit with respect to all 32 shape
  coefficients and the refractive index against central differences (step 1e-6) of the
  dense loss.
Plus two planted mistakes in a private copy of the oracle's dual arithmetic, each caught.
"""
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from oracle.build import HERE
from paper_2607_00790_gb300 import inputs

KEYS = ("x", "y", "nx", "ny", "w", "kappa")
H = 1e-6


def shape_case(N):
    a, b = inputs.shape_coefficients(1)
    c = inputs.fourier(N, a, b)
    return a, b, c, inputs.k0_for_density(c)


def test_fourier_tangents_match_differences():
    N = 64
    a, b, c, _ = shape_case(N)
    T = oracle.fourier_tangents(N, a, b)
    assert T.shape == (32, 6, N)
    for k in range(32):
        ap, am, bp, bm = a.copy(), a.copy(), b.copy(), b.copy()
        if k < 16:
            ap[k] += H
            am[k] -= H
        else:
            bp[k - 16] += H
            bm[k - 16] -= H
        cp, cm = inputs.fourier(N, ap, bp), inputs.fourier(N, am, bm)
        for q, key in enumerate(KEYS):
            fd = (cp[key] - cm[key]) / (2 * H)
            scale = max(np.max(np.abs(fd)), 1e-3)
            assert np.max(np.abs(fd - T[k, q])) / scale < 1e-7, (k, key)


def bilinear_cases(N, seed=5):
    a, b, c, k0 = shape_case(N)
    ph = oracle.Physics(k0, n=1.5)
    rng = np.random.default_rng(seed)
    lam = rng.normal(size=2 * N) + 1j * rng.normal(size=2 * N)
    xv = rng.normal(size=2 * N) + 1j * rng.normal(size=2 * N)
    tans = [rng.normal(size=(6, N))]
    for q, i in [(0, 3), (1, 7), (2, 10), (3, 20), (4, 33), (5, 40)]:
        t = np.zeros((6, N))
        t[q, i] = 1.0
        tans.append(t)
    tans += [np.zeros((6, N)), np.zeros((6, N))]
    tk1 = np.zeros(len(tans))
    te = np.zeros(len(tans))
    tk1[-2] = 1.0
    te[-1] = 1.0
    return c, ph, lam, xv, np.array(tans), tk1, te


def bilinear_errors(N=64):
    c, ph, lam, xv, tans, tk1, te = bilinear_cases(N)
    an = oracle.wsbm_bilinear_tangent(c, ph, lam, xv, tans, tk1, te)
    errs = []
    for t in range(len(tans)):
        vals = []
        for sgn in (1, -1):
            cc = dict(c)
            for q, k in enumerate(KEYS):
                cc[k] = c[k] + sgn * H * tans[t][q]
            pp = oracle.Physics(ph.k0, eps0=ph.eps0, eps1=ph.eps1 + sgn * H * te[t])
            pp.k1 = ph.k1 + sgn * H * tk1[t]
            vals.append(lam @ oracle.wsbm_dense(cc, pp) @ xv)
        fd = (vals[0] - vals[1]) / (2 * H)
        errs.append(abs(fd - an[t]) / abs(an[t]))
    return np.array(errs)


def test_bilinear_tangent_matches_differences():
    errs = bilinear_errors()
    assert np.all(errs < 1e-6), errs


def gradient_case(N=96):
    a, b, c, k0 = shape_case(N)
    at, bt = inputs.shape_coefficients(2)
    n = 1.5
    ph = oracle.Physics(k0, n=n)
    angles = 2 * np.pi * np.arange(64) / 64
    target = np.abs(oracle.gradient._forward(inputs.fourier(N, at, bt), ph, 0.0, angles)[3]) ** 2
    return a, b, n, k0, angles, target


def test_shape_gradient_matches_differences():
    N = 96
    a, b, n, k0, angles, target = gradient_case(N)
    c = inputs.fourier(N, a, b)
    tan = np.concatenate([oracle.fourier_tangents(N, a, b), np.zeros((1, 6, N))])
    tk1 = np.zeros(33)
    te = np.zeros(33)
    tk1[-1] = k0
    te[-1] = 2 * n
    L, g, _ = oracle.shape_loss_grad_dense(c, oracle.Physics(k0, n=n), 0.0, angles, target,
                                           tan, tk1, te)
    assert L > 0
    for k in range(33):
        vals = []
        for sgn in (1, -1):
            aa, bb, nn = a.copy(), b.copy(), n
            if k < 16:
                aa[k] += sgn * H
            elif k < 32:
                bb[k - 16] += sgn * H
            else:
                nn += sgn * H
            vals.append(oracle.shape_loss_dense(inputs.fourier(N, aa, bb),
                                                oracle.Physics(k0, n=nn), 0.0, angles, target))
        fd = (vals[0] - vals[1]) / (2 * H)
        assert abs(fd - g[k]) <= 1e-6 * np.max(np.abs(g)), (k, fd, g[k])


DUAL_MUTANTS = {
    # derivative of H1 with the wrong sign of its 1/z term
    "h1_derivative": ("o.h1 = cd{h.h1, (h.h0 - h.h1 / z.v) * z.t};",
                      "o.h1 = cd{h.h1, (h.h0 + h.h1 / z.v) * z.t};"),
    # weight derivative dropped from the off-diagonal blocks
    "weight_tangent": ("rd wj{g.w[j], g.tw[j]};", "rd wj{g.w[j], 0.0};"),
}


@pytest.mark.parametrize("name", sorted(DUAL_MUTANTS))
def test_planted_derivative_mistake_is_caught(name):
    old, new = DUAL_MUTANTS[name]
    src = open(os.path.join(HERE, "wsbm_oracle.cpp")).read()
    assert src.count(old) == 1
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "m.cpp")
        open(path, "w").write(src.replace(old, new))
        so = os.path.join(d, "libm.so")
        subprocess.run(["g++", "-std=c++17", "-O1", "-fPIC", "-shared", "-fopenmp",
                        "-ffp-contract=off", "-o", so, path], check=True)
        with oracle.use_library(so):
            assert not np.all(bilinear_errors() < 1e-6)
