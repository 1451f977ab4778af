"""Seeded synthetic inputs: closed curves sampled at equispaced parameter values.

This module holds no arithmetic of the solver itself.  It turns an analytic parametric
curve gamma(t), t in [0, 2 pi), into the arrays the solver takes as input (node positions,
outward unit normals, trapezoidal weights w_j = (2 pi/N)|gamma'(t_j)|, curvature), and draws
the random scatterer parameters of the batched and shape-gradient workloads from fixed
seeds.  Both the CUDA path and the CPU oracle are fed from here.

Curves (the paper's Fig. "mesh" shows a circle and a smooth star; its star parameters are
not printed):
  disk       gamma = R (cos t, sin t)
  star       r(t) = 1 + a cos(m t)            (a = 0.3, m = 5 unless stated)
  ellipse    gamma = (a cos t, b sin t)
  fourier    r(t) = 1 + sum_j a_j cos(j t) + b_j sin(j t)
"""
from __future__ import annotations

import numpy as np


def _polar(N, r, rp, rpp):
    """Arrays for the polar curve gamma(t) = r(t)(cos t, sin t); r, rp, rpp are callables."""
    t = 2.0 * np.pi * np.arange(N) / N
    c, s = np.cos(t), np.sin(t)
    rr, r1, r2 = r(t), rp(t), rpp(t)
    x, y = rr * c, rr * s
    xp, yp = r1 * c - rr * s, r1 * s + rr * c
    xpp = r2 * c - 2.0 * r1 * s - rr * c
    ypp = r2 * s + 2.0 * r1 * c - rr * s
    return _finish(N, t, x, y, xp, yp, xpp, ypp)


def _finish(N, t, x, y, xp, yp, xpp, ypp):
    sp = np.sqrt(xp * xp + yp * yp)
    curve = {
        "t": t,
        "x": x,
        "y": y,
        "nx": yp / sp,  # outward for a counter-clockwise curve
        "ny": -xp / sp,
        "w": (2.0 * np.pi / N) * sp,
        "kappa": (xp * ypp - yp * xpp) / sp**3,
    }
    curve["perimeter"] = float(np.sum(curve["w"]))
    return {k: (np.ascontiguousarray(v) if isinstance(v, np.ndarray) else v)
            for k, v in curve.items()}


def disk(N, R=1.0):
    return _polar(N, lambda t: R + 0 * t, lambda t: 0 * t, lambda t: 0 * t)


def star(N, a=0.3, m=5):
    return _polar(N, lambda t: 1.0 + a * np.cos(m * t),
                  lambda t: -a * m * np.sin(m * t),
                  lambda t: -a * m * m * np.cos(m * t))


def ellipse(N, a, b):
    t = 2.0 * np.pi * np.arange(N) / N
    c, s = np.cos(t), np.sin(t)
    return _finish(N, t, a * c, b * s, -a * s, b * c, -a * c, -b * s)


def fourier(N, acoef, bcoef):
    acoef = np.asarray(acoef, dtype=np.float64)
    bcoef = np.asarray(bcoef, dtype=np.float64)
    j = np.arange(1, acoef.size + 1)

    def r(t):
        return 1.0 + np.cos(np.outer(t, j)) @ acoef + np.sin(np.outer(t, j)) @ bcoef

    def rp(t):
        return (-np.sin(np.outer(t, j)) * j) @ acoef + (np.cos(np.outer(t, j)) * j) @ bcoef

    def rpp(t):
        return (-np.cos(np.outer(t, j)) * j * j) @ acoef + (-np.sin(np.outer(t, j)) * j * j) @ bcoef

    return _polar(N, r, rp, rpp)


def k0_for_density(curve, nodes_per_wavelength=15.0):
    """Exterior wavenumber giving the stated number of nodes per exterior wavelength:
    k0 = 2 pi N / (npw * perimeter)."""
    N = curve["x"].size
    return 2.0 * np.pi * N / (nodes_per_wavelength * curve["perimeter"])


# ------------------------------------------------------------------ named workloads ----
def workload(name, N=None):
    """The named synthetic workloads.  Returns (curve, dict of physical/solver parameters)."""
    if name == "disk":
        N = N or 256
        c = disk(N)
        return c, dict(k0=2.0 * np.pi, n=1.5, leaf=64, nproxy=64, tol=1e-10,
                       angles=[0.0], nfar=360)
    if name == "paper_table":
        # Table "para": eps0 = 1, eps1 = 5, mu = 1, omega = 10  =>  k0 = 10, k1 = 10 sqrt 5
        N = N or 256
        c = star(N)
        return c, dict(k0=10.0, n=float(np.sqrt(5.0)), leaf=128, nproxy=128, tol=1e-8,
                       angles=[0.0], nfar=360)
    if name == "star":
        N = N or 16384
        c = star(N)
        return c, dict(k0=k0_for_density(c), n=1.5, leaf=128, nproxy=128, tol=1e-8,
                       angles=list(2 * np.pi * np.arange(8) / 8), nfar=360)
    if name == "mixed":
        N = N or 262144
        c = star(N)
        return c, dict(k0=k0_for_density(c), n=1.5, leaf=128, nproxy=128, tol=1e-6,
                       angles=list(2 * np.pi * np.arange(8) / 8), nfar=360)
    raise KeyError(name)


def batched_manifest(seed=0, count=64):
    """Scatterer parameters of the batched workload: kind ellipse/star 50/50, ellipse axes
    U[0.5, 1.5], star a ~ U[0.1, 0.3], m ~ U{3..7}, N ~ U{2048..32768}, n ~ U[1.2, 2.0]."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        kind = "ellipse" if rng.random() < 0.5 else "star"
        if kind == "ellipse":
            geo = dict(a=float(rng.uniform(0.5, 1.5)), b=float(rng.uniform(0.5, 1.5)))
        else:
            geo = dict(a=float(rng.uniform(0.1, 0.3)), m=int(rng.integers(3, 8)))
        out.append(dict(kind=kind, geo=geo, N=int(rng.integers(2048, 32769)),
                        n=float(rng.uniform(1.2, 2.0))))
    return out


def shape_coefficients(seed, count=16, sigma=0.02):
    """Fourier shape coefficients a_j, b_j ~ N(0, sigma^2) of the shape-gradient workload."""
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, sigma, count), rng.normal(0.0, sigma, count)
