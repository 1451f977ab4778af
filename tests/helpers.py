"""Shared helpers for the parity tests: device geometry and per-entry error scales.

The scale M of an entry is the sum of the magnitudes of the terms the entry adds up
(eq. weakly_bm), built from the oracle's Hankel values; parity is |a_gpu - a_oracle| <= tol * M.
This guards the comparison against cancellation between terms (d.n near the diagonal, the
N_k0 - N_k1 difference) without weakening it where no cancellation occurs.
"""
import numpy as np

import oracle


def entry_scale(curve, ph, rows, cols):
    """Per-entry magnitude scale M for A[rows, cols] (paper order)."""
    rows = np.asarray(rows)
    cols = np.asarray(cols)
    N = curve["x"].size
    # node-pair quantities on the grid of distinct row and column nodes, then gathered
    ui, ri = np.unique(rows % N, return_inverse=True)
    uj, cj = np.unique(cols % N, return_inverse=True)
    Mn = _node_scale(curve, ph, ui, uj)
    a = (rows // N)[:, None]
    b = (cols // N)[None, :]
    return Mn[a, b, ri[:, None], cj[None, :]]


def _node_scale(curve, ph, ui, uj):
    """M[a, b, i, j]: scale of entry (a, b) of the 2x2 block of nodes ui[i], uj[j]."""
    i = ui[:, None]
    j = uj[None, :]
    x, y, nx, ny, w = (np.asarray(curve[k]) for k in ("x", "y", "nx", "ny", "w"))
    dx = x[i] - x[j]
    dy = y[i] - y[j]
    r = np.hypot(dx, dy)
    diag = r == 0
    r = np.where(diag, 1.0, r)
    dny = np.abs(dx * nx[j] + dy * ny[j]) / r
    dnx = np.abs(dx * nx[i] + dy * ny[i]) / r
    z0, z1 = ph.k0 * r, ph.k1 * r
    h0a, h1a = oracle.hankel01(z0.ravel())
    h0b, h1b = oracle.hankel01(z1.ravel())
    f1a = oracle.f1(z0.ravel())
    f1b = oracle.f1(z1.ravel())
    sh = r.shape
    H0a, H1a, H0b, H1b, F1a, F1b = (np.abs(v).reshape(sh) for v in (h0a, h1a, h0b, h1b, f1a, f1b))
    k0, k1, e0, e1 = ph.k0, ph.k1, ph.eps0, ph.eps1
    c = dnx * dny
    nn = np.abs(nx[i] * nx[j] + ny[i] * ny[j]) + 2 * c
    dN = 0.25 * ((k0**2 * H0a + k1**2 * H0b) * c + (k0**2 * F1a + k1**2 * F1b) * nn)
    wj = w[j]
    M = np.empty((2, 2) + sh)
    M[0, 0] = wj * 0.25 * k1 * H1b * dny
    M[0, 1] = wj * 0.25 * e1 * H0b
    M[1, 0] = wj * (0.25 * k0 * H1a * dny + dN / k0)
    M[1, 1] = wj * (0.25 * e0 * H0a + dnx / (4 * k0) * (e0 * k0 * H1a + e1 * k1 * H1b))
    # diagonal blocks: scale 1 (the identity terms dominate)
    M[:, :, diag] = 1.0
    return M


def device_geom(curve):
    from paper_2607_00790_gb300 import binding
    return binding.make_geom(curve)
