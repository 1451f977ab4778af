"""Parity of the device WSBM entries (eq. weakly_bm, one-point corrected diagonal) and the
proxy-circle blocks with the oracle, on the same seeded inputs, element by element."""
import numpy as np
import pytest

import oracle
from helpers import entry_scale
from paper_2607_00790_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-12


def gpu_entries(curve, ph, rows, cols, precision=0):
    import torch
    from paper_2607_00790_gb300 import binding
    g, keep = binding.make_geom(curve)
    p = binding.make_params(ph.k0, ph.k1 / ph.k0, ph.eps0, ph.eps1, precision=precision)
    r = torch.tensor(np.asarray(rows, dtype=np.int64), device="cuda")
    c = torch.tensor(np.asarray(cols, dtype=np.int64), device="cuda")
    out = binding.wsbm_entries_raw(g, p, r, c)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def check(curve, ph, rows, cols, tol=TOL):
    ref = oracle.wsbm_entries(curve, ph, rows, cols)
    got = gpu_entries(curve, ph, rows, cols)
    M = entry_scale(curve, ph, rows, cols)
    err = np.abs(got - ref) / M
    assert np.all(np.isfinite(got))
    assert err.max() <= tol, (err.max(), np.unravel_index(np.argmax(err), err.shape))
    fro = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert fro <= tol, fro
    return err.max()


def test_disk_full_matrix():
    c, prm = inputs.workload("disk")
    ph = oracle.Physics(prm["k0"], n=prm["n"])
    idx = np.arange(2 * c["x"].size)
    A = oracle.wsbm_dense(c, ph)
    got = gpu_entries(c, ph, idx, idx)
    M = entry_scale(c, ph, idx, idx)
    assert (np.abs(got - A) / M).max() <= TOL
    assert np.linalg.norm(got - A) / np.linalg.norm(A) <= TOL


def test_star_ragged_block():
    c = inputs.star(1000)
    ph = oracle.Physics(inputs.k0_for_density(c), n=1.5)
    rng = np.random.default_rng(5)
    rows = rng.choice(2000, 301, replace=False)
    cols = rng.choice(2000, 173, replace=False)
    check(c, ph, rows, cols)


def test_star_16384_samples():
    c, prm = inputs.workload("star")
    ph = oracle.Physics(prm["k0"], n=prm["n"])
    rng = np.random.default_rng(6)
    # a contiguous leaf-sized band (near field) and scattered far samples
    band = np.arange(5000, 5128)
    rows = np.concatenate([band, band + 16384])
    cols = np.concatenate([band[::3], band[::5] + 16384, rng.integers(0, 32768, 40)])
    check(c, ph, rows, cols)


def test_star_2p18_samples():
    c, prm = inputs.workload("mixed")
    ph = oracle.Physics(prm["k0"], n=prm["n"])
    rng = np.random.default_rng(7)
    N = c["x"].size
    rows = np.concatenate([rng.integers(0, 2 * N, 48), np.arange(1000, 1024), np.arange(1000, 1024) + N])
    cols = np.concatenate([rng.integers(0, 2 * N, 48), np.arange(990, 1040), np.arange(990, 1040) + N])
    check(c, ph, rows, cols)


def test_paper_table_parameters():
    c = inputs.star(600)
    ph = oracle.Physics(10.0, eps0=1.0, eps1=5.0)
    idx = np.arange(0, 1200, 7)
    check(c, ph, idx, idx)


def test_edge_cases():
    c = inputs.disk(2)
    ph = oracle.Physics(1.0, n=1.5)
    idx = np.arange(4)
    check(c, ph, idx, idx)
    c = inputs.star(64)
    ph = oracle.Physics(3.0, n=2.0)
    check(c, ph, [5], [5])                       # one diagonal entry
    check(c, ph, [7, 7, 71, 7], [3, 67, 3, 3])   # repeated indices
    assert gpu_entries(c, ph, [], [1, 2]).shape == (0, 2)


def test_deterministic():
    c = inputs.star(512)
    ph = oracle.Physics(inputs.k0_for_density(c), n=1.5)
    idx = np.arange(0, 1024, 3)
    a = gpu_entries(c, ph, idx, idx)
    b = gpu_entries(c, ph, idx, idx)
    assert np.array_equal(a, b)


def test_invalid_arguments():
    import torch
    from paper_2607_00790_gb300 import binding
    c = inputs.disk(16)
    g, keep = binding.make_geom(c)
    p = binding.make_params(-1.0, 1.5)
    r = torch.arange(4, device="cuda")
    with pytest.raises(binding.WsbmError):
        binding.wsbm_entries_raw(g, p, r, r)


# ------------------------------------------------------------------------ proxy blocks ----
def gpu_proxy(curve, ph, side, idx, circle, P, precision=0):
    import torch
    from paper_2607_00790_gb300 import binding
    g, keep = binding.make_geom(curve)
    p = binding.make_params(ph.k0, ph.k1 / ph.k0, ph.eps0, ph.eps1, precision=precision)
    t = torch.tensor(np.asarray(idx, dtype=np.int64), device="cuda")
    out = binding.wsbm_proxy_block(g, p, side, t, circle, P)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("N,lo,hi,P", [(1024, 128, 256, 200), (16384, 4096, 4224, 128),
                                       (262144, 100000, 100128, 160)])
def test_proxy_blocks_match_oracle(N, lo, hi, P):
    c = inputs.star(N)
    ph = oracle.Physics(inputs.k0_for_density(c), n=1.5)
    nodes = np.arange(lo, hi)
    circ = oracle.proxy_circle(c, nodes)
    box = np.concatenate([nodes, nodes + N])
    for side in (0, 1):
        ref = (oracle.proxy_row_block(c, ph, box, circ, P) if side == 0
               else oracle.proxy_col_block(c, ph, box, circ, P))
        got = gpu_proxy(c, ph, side, box, circ, P)
        assert got.shape == ref.shape
        # per column scale: the largest entry magnitude in that column of the block
        scale = np.maximum(np.abs(ref).max(axis=0, keepdims=True), 1e-300)
        err = np.abs(got - ref) / scale
        assert err.max() <= TOL, (side, err.max())
        mixed = gpu_proxy(c, ph, side, box, circ, P, precision=1)
        rel = np.linalg.norm(mixed - ref) / np.linalg.norm(ref)
        assert rel < 1e-6, (side, rel)
        fine = gpu_proxy(c, ph, side, box, circ, P, precision=2)
        rel = np.linalg.norm(fine - ref) / np.linalg.norm(ref)
        assert rel < 5e-8, (side, rel)


def test_proxy_blocks_on_an_upper_level_circle():
    """Proxy blocks on the circle of a level-3 box of the 2^18 star (32768 nodes, radius ~0.8),
    where the arguments k r reach ~3e4: 128 of the box's nodes against 1024 proxy points.
    Per-entry bound: the magnitude of the terms the entry adds up (the combined-field source
    cancels to leading order when d.nu/r ~ -1, as it does from the far side of this circle), in
    the large-argument form |H0|, |H1| <= sqrt(2/(pi z)), times 1e-12 plus the phase change of
    one-ulp differences in the proxy points (sincospi on the GPU, std::cos/std::sin in the
    oracle) and in z, |dz| <= 8 z eps."""
    N = 262144
    c = inputs.star(N)
    ph = oracle.Physics(inputs.k0_for_density(c), n=1.5)
    lo, hi = 3 * 32768, 4 * 32768
    circ = oracle.proxy_circle(c, np.arange(lo, hi))
    nodes = np.arange(lo + 5000, lo + 5128)
    box = np.concatenate([nodes, nodes + N])
    P = 1024
    t = 2 * np.pi * np.arange(P) / P
    px, py = circ[0] + circ[2] * np.cos(t), circ[1] + circ[2] * np.sin(t)
    r = np.hypot(c["x"][box % N][:, None] - px[None, :], c["y"][box % N][:, None] - py[None, :])
    pw = 2 * np.pi * circ[2] / P
    eps = 2.0 ** -53
    for side in (0, 1):
        ref = (oracle.proxy_row_block(c, ph, box, circ, P) if side == 0
               else oracle.proxy_col_block(c, ph, box, circ, P))
        got = gpu_proxy(c, ph, side, box, circ, P)
        err = np.abs(got - ref)
        for s_, k in ((0, ph.k1), (1, ph.k0)):
            z = k * r
            amp = np.sqrt(2.0 / (np.pi * z))
            assert z.min() > 20.0
            if side == 0:   # rows: box equations, columns: sources s_ (P each)
                M = pw * (k / 4) * amp * 2 * (1 + k / ph.k0)
                e = err[:, s_ * P:(s_ + 1) * P]
            else:           # rows: fields s_ at the proxy points, columns: box unknowns
                w = c["w"][box % N][:, None]
                M = (w * (k / 4 + np.maximum(ph.eps0, ph.eps1) / 4) * amp).T
                z = z.T
                e = err[s_ * P:(s_ + 1) * P, :]
            bound = M * (TOL + 8 * z * eps)
            assert np.all(e <= bound), (side, s_, float((e / bound).max()))
