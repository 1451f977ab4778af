"""HSS build, factor, solve and far field on the GPU against the dense oracle (densities and
far field within 10x the ID tolerance) and against the Mie series on the disk."""
import numpy as np
import pytest

import oracle
from paper_2607_00790_gb300 import inputs

pytestmark = pytest.mark.gpu


def gpu_solver(curve, prm, precision=0, leaf=None, tol=None, nproxy=None, id_method=0):
    from paper_2607_00790_gb300 import binding
    g, keep = binding.make_geom(curve)
    p = binding.make_params(prm["k0"], prm["n"], leaf=leaf or prm["leaf"],
                            nproxy=nproxy or prm["nproxy"], id_tol=tol or prm["tol"],
                            precision=precision, id_method=id_method)
    s = binding.Solver(g, p)
    s._keep = keep
    return s


def solve_gpu(s, angles):
    import torch
    ang = torch.tensor(np.asarray(angles, dtype=np.float64), device="cuda")
    s.factor()
    rhs = s.rhs_planewave(ang)
    u, q = s.solve(rhs)
    torch.cuda.synchronize()
    return rhs.cpu().numpy(), u.cpu().numpy(), q.cpu().numpy()


def farfield_gpu(s, u, q, angles):
    import torch
    uu = torch.tensor(u, device="cuda")
    qq = torch.tensor(q, device="cuda")
    a = torch.tensor(np.asarray(angles, dtype=np.float64), device="cuda")
    return s.farfield(uu, qq, a).cpu().numpy()


def dense_reference(curve, ph, angles):
    A = oracle.wsbm_dense(curve, ph)
    b = oracle.rhs_planewave(curve, ph, angles)
    x = oracle.dense_solve(A, b)
    u, q = oracle.split_uq(x)
    return b, u, q


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_disk_config_vs_dense_and_mie():
    c, prm = inputs.workload("disk")
    ph = oracle.Physics(prm["k0"], n=prm["n"])
    s = gpu_solver(c, prm)
    rhs, u, q = solve_gpu(s, [0.0])
    b, ud, qd = dense_reference(c, ph, [0.0])
    assert rel(rhs, b) < 1e-14
    tol = prm["tol"]
    assert rel(u, ud) < 10 * tol, rel(u, ud)
    assert rel(q, qd) < 10 * tol, rel(q, qd)
    ang = 2 * np.pi * np.arange(360) / 360
    ff = farfield_gpu(s, u, q, ang)
    ffd = oracle.farfield(c, ph, ud, qd, ang)
    assert rel(ff, ffd) < 10 * tol, rel(ff, ffd)
    # Mie: the HSS solution carries the O(h^3) discretisation error of the dense system
    ue, _ = oracle.mie_boundary(1.0, ph, c["t"])
    err = np.linalg.norm(u[:, 0].real - ue.real) / np.linalg.norm(ue.real)
    assert abs(err - 7.74e-5) < 1e-6, err
    st = s.stats()
    assert st["levels"] == 2 and st["root_size"] > 0 and st["entries_generated"] > 0


@pytest.mark.parametrize("N,leaf", [(1024, 64), (1536, 128)])
def test_star_15_nodes_per_wavelength_vs_dense(N, leaf):
    c = inputs.star(N)
    prm = dict(k0=inputs.k0_for_density(c), n=1.5, leaf=leaf, nproxy=64, tol=1e-8)
    ph = oracle.Physics(prm["k0"], n=prm["n"])
    angles = 2 * np.pi * np.arange(8) / 8
    s = gpu_solver(c, prm)
    rhs, u, q = solve_gpu(s, angles)
    b, ud, qd = dense_reference(c, ph, angles)
    assert rel(u, ud) < 10 * prm["tol"], rel(u, ud)
    assert rel(q, qd) < 10 * prm["tol"], rel(q, qd)
    ang = 2 * np.pi * np.arange(360) / 360
    ff = farfield_gpu(s, u, q, ang)
    ffd = oracle.farfield(c, ph, ud, qd, ang)
    assert rel(ff, ffd) < 10 * prm["tol"], rel(ff, ffd)


def test_mixed_precision_vs_fp64_path():
    c = inputs.star(1024)
    prm = dict(k0=inputs.k0_for_density(c), n=1.5, leaf=64, nproxy=64, tol=1e-6)
    ang = 2 * np.pi * np.arange(360) / 360
    s64 = gpu_solver(c, prm, precision=0)
    _, u64, q64 = solve_gpu(s64, [0.0, 1.0])
    f64 = farfield_gpu(s64, u64, q64, ang)
    smx = gpu_solver(c, prm, precision=1)
    _, umx, qmx = solve_gpu(smx, [0.0, 1.0])
    fmx = farfield_gpu(smx, umx, qmx, ang)
    assert rel(fmx, f64) < 1e-5, rel(fmx, f64)


def test_mixed_fine_reaches_fp64_accuracy_at_tight_tolerance():
    """Amplitude-only mixed precision at ID tol 1e-7: far field within 10x tol of the dense
    oracle (the FP32 noise of WSBM_MIXED, ~1e-7, would not allow it)."""
    c = inputs.star(1536)
    prm = dict(k0=inputs.k0_for_density(c), n=1.5, leaf=64, nproxy=64, tol=1e-7)
    ph = oracle.Physics(prm["k0"], n=prm["n"])
    ang = 2 * np.pi * np.arange(360) / 360
    s = gpu_solver(c, prm, precision=2)
    _, u, q = solve_gpu(s, [0.0, 1.0])
    ff = farfield_gpu(s, u, q, ang)
    _, ud, qd = dense_reference(c, ph, [0.0, 1.0])
    ffd = oracle.farfield(c, ph, ud, qd, ang)
    assert rel(ff, ffd) < 10 * prm["tol"], rel(ff, ffd)


@pytest.mark.parametrize("id_method", [0, 1])
def test_id_methods_match_dense(id_method):
    """Randomized leaf IDs (sketch, default) and the full column-pivoted QR everywhere: both
    within 10x the ID tolerance of the dense oracle; the sketch is used only by the first."""
    c = inputs.star(1536)
    prm = dict(k0=inputs.k0_for_density(c), n=1.5, leaf=128, nproxy=128, tol=1e-8)
    ph = oracle.Physics(prm["k0"], n=prm["n"])
    ang = 2 * np.pi * np.arange(90) / 90
    s = gpu_solver(c, prm, id_method=id_method)
    _, u, q = solve_gpu(s, [0.0, 2.5])
    st = s.stats()
    assert (st["sketch_matrices"] > 0) == (id_method == 0)
    _, ud, qd = dense_reference(c, ph, [0.0, 2.5])
    assert rel(u, ud) < 10 * prm["tol"] and rel(q, qd) < 10 * prm["tol"], (rel(u, ud), rel(q, qd))
    ff = farfield_gpu(s, u, q, ang)
    assert rel(ff, oracle.farfield(c, ph, ud, qd, ang)) < 10 * prm["tol"]
    s.close()


def test_sketch_fallback_keeps_accuracy():
    """Leaf boxes of 64 nodes at tol 1e-10: the ranks come within 16 rows of the 64-row sketches,
    so those sides are redone on the full ID matrices; the result stays within 10x tol."""
    c = inputs.star(2048)
    prm = dict(k0=inputs.k0_for_density(c), n=1.5, leaf=64, nproxy=64, tol=1e-10)
    ph = oracle.Physics(prm["k0"], n=prm["n"])
    s = gpu_solver(c, prm)
    _, u, q = solve_gpu(s, [0.7])
    st = s.stats()
    assert st["sketch_matrices"] > 0 and st["sketch_fallbacks"] > 0, st
    _, ud, qd = dense_reference(c, ph, [0.7])
    assert rel(u, ud) < 10 * prm["tol"] and rel(q, qd) < 10 * prm["tol"], (rel(u, ud), rel(q, qd))
    s.close()


def test_leaf_boxes_beyond_fused_lu_limit():
    """Two leaf boxes of 520 nodes (1040 unknowns, above the fused LU + solve kernel's 1024)
    take the blocked LU and triangular solves; the result stays within 10x tol of the dense
    oracle, and the memory pool can be trimmed after."""
    from paper_2607_00790_gb300 import binding
    c = inputs.star(1040)
    prm = dict(k0=inputs.k0_for_density(c), n=1.5, leaf=520, nproxy=64, tol=1e-8)
    ph = oracle.Physics(prm["k0"], n=prm["n"])
    s = gpu_solver(c, prm)
    _, u, q = solve_gpu(s, [0.3])
    st = s.stats()
    assert st["levels"] >= 1 and st["rank_per_level"][st["levels"]] > 0 and st["lu_matrices"] == 0, st
    _, ud, qd = dense_reference(c, ph, [0.3])
    assert rel(u, ud) < 10 * prm["tol"] and rel(q, qd) < 10 * prm["tol"], (rel(u, ud), rel(q, qd))
    s.close()
    binding.trim_memory()


def test_single_box_tree():
    c = inputs.star(48)
    prm = dict(k0=3.0, n=1.5, leaf=64, nproxy=16, tol=1e-10)
    ph = oracle.Physics(prm["k0"], n=prm["n"])
    s = gpu_solver(c, prm)
    _, u, q = solve_gpu(s, [0.3])
    _, ud, qd = dense_reference(c, ph, [0.3])
    assert rel(u, ud) < 1e-12 and rel(q, qd) < 1e-12
    assert s.stats()["levels"] == 0


def test_paper_table_parameters_star():
    c = inputs.star(1024)
    prm = dict(k0=10.0, n=float(np.sqrt(5.0)), leaf=64, nproxy=64, tol=1e-10)
    ph = oracle.Physics(10.0, eps0=1.0, eps1=5.0)
    s = gpu_solver(c, prm)
    _, u, q = solve_gpu(s, [0.0])
    _, ud, qd = dense_reference(c, ph, [0.0])
    assert rel(u, ud) < 1e-9 and rel(q, qd) < 1e-9


def test_solve_before_factor_and_bad_args():
    import torch
    from paper_2607_00790_gb300 import binding
    c = inputs.disk(128)
    g, keep = binding.make_geom(c)
    s = binding.Solver(g, binding.make_params(2 * np.pi, 1.5, leaf=32, nproxy=32, id_tol=1e-8))
    rhs = torch.zeros((256, 1), dtype=torch.complex128, device="cuda")
    with pytest.raises(binding.WsbmError) as e:
        s.solve(rhs)
    assert e.value.code == -6
    with pytest.raises(binding.WsbmError):
        binding.Solver(g, binding.make_params(2 * np.pi, 1.5, leaf=2))
    bad = dict(c)
    bad["w"] = c["w"].copy()
    bad["w"][3] = np.nan
    gb, kb = binding.make_geom(bad)
    with pytest.raises(binding.WsbmError):
        binding.Solver(gb, binding.make_params(2 * np.pi, 1.5))


def test_box_info_matches_oracle_circle():
    c, prm = inputs.workload("star", N=4096)
    s = gpu_solver(c, prm)
    for level, box in [(5, 0), (5, 17), (3, 5), (1, 1)]:
        circ, rng = s.box_info(level, box)
        cx, cy, rho = oracle.proxy_circle(c, np.arange(rng[0], rng[1]))
        assert (circ[0], circ[1], circ[3]) == (cx, cy, rho)


def test_factor_solve_deterministic():
    c = inputs.star(768)
    prm = dict(k0=inputs.k0_for_density(c), n=1.5, leaf=64, nproxy=64, tol=1e-8)
    s = gpu_solver(c, prm)
    _, u1, q1 = solve_gpu(s, [0.0])
    _, u2, q2 = solve_gpu(s, [0.0])
    assert np.array_equal(u1, u2) and np.array_equal(q1, q2)


def test_full_size_leaf_skeletons_span_far_field():
    """At the bench size (N = 2^18, 15 nodes per wavelength, leaf-level build): the row
    skeleton of a box must reproduce the box's far-field rows, and the column skeleton its
    far-field columns, to the ID tolerance; far entries are sampled from the oracle."""
    from paper_2607_00790_gb300 import binding
    c, prm = inputs.workload("mixed")  # star, N = 262144, 15 nodes per wavelength
    N = c["x"].size
    tol = 1e-8
    g, keep = binding.make_geom(c)
    p = binding.make_params(prm["k0"], prm["n"], leaf=128, nproxy=128, id_tol=tol, max_levels=1)
    s = binding.Solver(g, p)
    s._keep = keep
    s.factor()
    ph = oracle.Physics(prm["k0"], n=prm["n"])
    L = s.stats()["levels"]
    rng = np.random.default_rng(31)
    for box in (3, 1000):
        circ, (lo, hi) = s.box_info(L, box)
        nodes = np.arange(lo, hi)
        unk = np.concatenate([nodes, nodes + N])
        jr, jc = s.skeletons(L, box)
        assert 0 < jr.size < unk.size
        d = np.hypot(c["x"] - circ[0], c["y"] - circ[1])
        far_nodes = rng.choice(np.nonzero(d > circ[3])[0], 600, replace=False)
        far = np.concatenate([far_nodes, far_nodes + N])
        for rows_side in (True, False):
            A = oracle.wsbm_entries(c, ph, unk, far) if rows_side else oracle.wsbm_entries(c, ph, far, unk).T
            sk = jr if rows_side else jc
            pos = np.searchsorted(unk, sk)
            Q, _ = np.linalg.qr(A[pos].T)           # span of the skeleton rows
            R = A.T - Q @ (Q.conj().T @ A.T)
            rel = np.linalg.norm(R) / np.linalg.norm(A)
            assert rel < 10 * tol, (box, rows_side, rel)
    s.close()


def test_leaf_level_of_65536_boxes():
    """A tree level of 65536 boxes (N = 2^20, leaf 16): every batched launch over the boxes of a
    level runs in chunks of at most 65535 along the grid's y dimension. The skeletons of a box
    in the first chunk and of the last box (the second chunk) must reproduce their far-field
    rows and columns to the ID tolerance (far entries from the oracle)."""
    from paper_2607_00790_gb300 import binding
    N = 1 << 20
    c = inputs.star(N)
    k0 = float(inputs.k0_for_density(c)) / 4.0  # 60 nodes per wavelength: small box ranks
    # QR cutoff id_tol / (4 sqrt(65536)) = 2.5e-7 relative to each ID matrix's largest column
    tol = 2.5e-7 * 4 * 256
    cut = tol / (4 * 256)
    g, keep = binding.make_geom(c)
    p = binding.make_params(k0, 1.5, leaf=16, nproxy=32, id_tol=tol, max_levels=1)
    s = binding.Solver(g, p)
    s._keep = keep
    s.factor()
    st = s.stats()
    L = st["levels"]
    assert st["nboxes_leaf"] == 65536, st["nboxes_leaf"]
    ph = oracle.Physics(k0, n=1.5)
    rng = np.random.default_rng(7)
    for box in (3, 65535):
        circ, (lo, hi) = s.box_info(L, box)
        nodes = np.arange(lo, hi)
        unk = np.concatenate([nodes, nodes + N])
        jr, jc = s.skeletons(L, box)
        assert 0 < jr.size < unk.size
        d = np.hypot(c["x"] - circ[0], c["y"] - circ[1])
        far_nodes = rng.choice(np.nonzero(d > circ[3])[0], 400, replace=False)
        far = np.concatenate([far_nodes, far_nodes + N])
        for rows_side in (True, False):
            A = oracle.wsbm_entries(c, ph, unk, far) if rows_side else oracle.wsbm_entries(c, ph, far, unk).T
            sk = jr if rows_side else jc
            pos = np.searchsorted(unk, sk)
            Q, _ = np.linalg.qr(A[pos].T)
            R = A.T - Q @ (Q.conj().T @ A.T)
            rel = np.linalg.norm(R) / np.linalg.norm(A)
            assert rel < 40 * cut, (box, rows_side, rel)
    s.close()


def test_torch_allocator_supplies_the_factors():
    """With PyTorch's caching allocator plugged in (wsbm_set_allocator), the factors and the
    build's work space come from PyTorch: the memory it reports grows by at least the factor
    bytes, the solution is unchanged, and closing the handle returns the factors to it."""
    import torch
    from paper_2607_00790_gb300 import binding
    c, prm = inputs.workload("disk")
    ph = oracle.Physics(prm["k0"], n=prm["n"])
    g, keep = binding.make_geom(c)
    p = binding.make_params(prm["k0"], prm["n"], leaf=prm["leaf"], nproxy=prm["nproxy"],
                            id_tol=prm["tol"])
    binding.use_torch_allocator(True)
    try:
        torch.cuda.synchronize()
        m0 = torch.cuda.memory_allocated()
        s = binding.Solver(g, p)
        s.factor()
        torch.cuda.synchronize()
        m1 = torch.cuda.memory_allocated()
        fb = s.stats()["factor_bytes"]
        assert fb > 0 and m1 - m0 >= fb, (m0, m1, fb)
        ang = torch.tensor([0.0], dtype=torch.float64, device="cuda")
        u, q = s.solve(s.rhs_planewave(ang))
        _, ud, qd = dense_reference(c, ph, [0.0])
        assert rel(u.cpu().numpy(), ud) < 10 * prm["tol"]
        del u, q
        torch.cuda.synchronize()
        m2 = torch.cuda.memory_allocated()
        s.close()
        torch.cuda.synchronize()
        assert m2 - torch.cuda.memory_allocated() >= fb
    finally:
        binding.use_torch_allocator(False)
