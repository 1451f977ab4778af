"""Pins for the oracle's proxy-circle blocks (proxy-surface method, Sec. III).

The proxy blocks are correct when they span what they stand in for:
* every far column of the box's row block A(I_box, far) lies in the range of the proxy row
  block (far sources act on the box equations only through fields the proxy sources
  reproduce);
* every far row of A(far, I_box) lies in the row space of the proxy column block.
A wrong sign, a dropped term or a swapped wavenumber in either block breaks the span.
"""
import numpy as np
import pytest

import oracle
from paper_2607_00790_gb300 import inputs


def setup_box(N=1024, lo=128, hi=256, npw=15.0, P=200):
    c = inputs.star(N)
    ph = oracle.Physics(inputs.k0_for_density(c, npw), n=1.5)
    nodes = np.arange(lo, hi)
    circ = oracle.proxy_circle(c, nodes)
    cx, cy, rho = circ
    d = np.hypot(c["x"] - cx, c["y"] - cy)
    far = np.array([j for j in range(N) if (j < lo or j >= hi) and d[j] > rho])
    box_unk = np.concatenate([nodes, nodes + N])
    far_unk = np.concatenate([far, far + N])
    return c, ph, circ, box_unk, far_unk, P


def residual_in_range(B, Y, cut=1e-12):
    U, s, _ = np.linalg.svd(B, full_matrices=False)
    U = U[:, s > cut * s[0]]
    R = Y - U @ (U.conj().T @ Y)
    return np.linalg.norm(R) / np.linalg.norm(Y)


def row_and_col_residuals():
    c, ph, circ, box, far, P = setup_box()
    Prow = oracle.proxy_row_block(c, ph, box, circ, P)
    Pcol = oracle.proxy_col_block(c, ph, box, circ, P)
    Afar_cols = oracle.wsbm_entries(c, ph, box, far)   # box equations x far unknowns
    Afar_rows = oracle.wsbm_entries(c, ph, far, box)   # far equations x box unknowns
    r1 = residual_in_range(Prow, Afar_cols)
    r2 = residual_in_range(Pcol.conj().T, Afar_rows.conj().T)
    # the test has teeth only if the proxy blocks are numerically rank deficient
    s = np.linalg.svd(Pcol, compute_uv=False)
    assert np.sum(s > 1e-12 * s[0]) < 0.6 * box.size
    return r1, r2


def test_proxy_blocks_span_far_interactions():
    r1, r2 = row_and_col_residuals()
    assert r1 < 1e-9, r1
    assert r2 < 1e-9, r2


def test_proxy_block_shapes_and_circle():
    c, ph, circ, box, far, P = setup_box()
    cx, cy, rho = circ
    nodes = box[: box.size // 2]
    R = np.max(np.hypot(c["x"][nodes] - cx, c["y"][nodes] - cy))
    assert abs(rho - 1.5 * R) < 1e-15
    assert oracle.proxy_row_block(c, ph, box, circ, P).shape == (box.size, 2 * P)
    assert oracle.proxy_col_block(c, ph, box, circ, P).shape == (2 * P, box.size)
    # the k0 proxy source never drives the first (k1-only) equation
    Prow = oracle.proxy_row_block(c, ph, box, circ, P)
    assert np.all(Prow[: nodes.size, P:] == 0)
