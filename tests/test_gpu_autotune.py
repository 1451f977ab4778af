"""Autotuners of the launch shapes: they pick among the documented candidates, the choice
sticks for later calls on the device, and every shape they can pick gives a correct product,
factor and solve.  Shapes that only reorder independent work (the raster group of the GEMM's
tile order, the tile shape and grid of the entry kernels) change no bit of any result."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

EPS = 2.0 ** -53


@pytest.fixture
def restore_tuning():
    from paper_2607_00790_gb300 import binding
    saved = binding.wsbm_tuning()
    yield saved
    binding.wsbm_tuning_set(**saved)


def test_autotune_picks_candidates_and_keeps_them(restore_tuning):
    from paper_2607_00790_gb300 import binding
    choice, ms = binding.wsbm_autotune(n_box=128, nbox=64, nrhs_box=48, n_root=2048)
    assert choice["tc_group"] in (4, 8, 16)
    assert choice["box_nb"] in (32, 64)
    assert choice["root_nb_mid"] in (128, 256)
    assert choice["root_nb_large"] == restore_tuning["root_nb_large"]  # class not timed: kept
    assert choice["cpqr_cb"] in (2, 4, 8)
    assert len(ms) == 10 and all(t > 0 for t in ms)
    # the fastest candidate of each group is the one kept
    assert ms[[4, 8, 16].index(choice["tc_group"])] == min(ms[0:3])
    assert ms[3 + [32, 64].index(choice["box_nb"])] == min(ms[3:5])
    assert ms[5 + [128, 256].index(choice["root_nb_mid"])] == min(ms[5:7])
    assert ms[7 + [2, 4, 8].index(choice["cpqr_cb"])] == min(ms[7:10])
    now = binding.wsbm_tuning()
    assert now["tuned"] and all(now[k] == choice[k] for k in binding.TUNE_KEYS)
    # the build shapes are untouched
    assert all(now[k] == restore_tuning[k] for k in binding.TUNE_BUILD_KEYS)


def test_tuning_rejects_bad_shapes_and_sizes(restore_tuning):
    from paper_2607_00790_gb300 import binding
    for bad in [dict(tc_group=0), dict(box_nb=12), dict(box_nb=72), dict(root_nb_mid=192),
                dict(root_nb_large=512), dict(cpqr_cb=3), dict(pair_tf=8), dict(proxy_tf=128),
                dict(pair_ctas=0), dict(proxy_ctas=65), dict(cpqr_threads=64), dict(solve_tc_min=0)]:
        with pytest.raises(binding.WsbmError):
            binding.wsbm_tuning_set(**bad)
    assert binding.wsbm_tuning() == restore_tuning
    with pytest.raises(binding.WsbmError):
        binding.wsbm_autotune(n_box=32, nbox=4, nrhs_box=4, n_root=1024)
    with pytest.raises(binding.WsbmError):
        binding.wsbm_autotune(n_box=128, nbox=4, nrhs_box=4, n_root=65536)


def test_raster_group_changes_no_bit(restore_tuning):
    import torch
    from paper_2607_00790_gb300 import binding
    rng = np.random.default_rng(21)
    m, n, k = 1500, 1300, 300
    A = torch.as_tensor(rng.normal(size=(m, k)) + 1j * rng.normal(size=(m, k)), device="cuda")
    B = torch.as_tensor(rng.normal(size=(k, n)) + 1j * rng.normal(size=(k, n)), device="cuda")
    outs = []
    for g in (1, 4, 8, 16, 64):
        binding.wsbm_tuning_set(tc_group=g)
        outs.append(np.ascontiguousarray(binding.wsbm_zgemm(A, B).cpu().numpy()))
    for o in outs[1:]:
        assert o.tobytes() == outs[0].tobytes()
    ref = A.cpu().numpy() @ B.cpu().numpy()
    assert np.linalg.norm(outs[0] - ref) <= 2e-15 * np.linalg.norm(ref)


@pytest.mark.parametrize("nb", [128, 256])
def test_root_lu_panel_widths(nb, restore_tuning):
    """wsbm_lu_dense (n = 2600, several outer panels and a ragged last one) with either outer
    panel width: P A = L U to rounding."""
    import torch
    from paper_2607_00790_gb300 import binding
    n = 2600
    rng = np.random.default_rng(nb)
    A = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n)) + 4.0 * np.eye(n)
    binding.wsbm_tuning_set(root_nb_mid=nb, root_nb_large=nb)
    LU, piv = binding.wsbm_lu_dense(torch.as_tensor(A, device="cuda"))
    torch.cuda.synchronize()
    LU = LU.cpu().numpy()
    piv = piv.cpu().numpy()
    L = np.tril(LU, -1) + np.eye(n)
    U = np.triu(LU)
    PA = A.copy()
    for j in range(n):
        if piv[j] != j:
            PA[[j, piv[j]]] = PA[[piv[j], j]]
    assert np.linalg.norm(PA - L @ U) / np.linalg.norm(A) < 50 * n * EPS


_DENSE = {}


def _star_dense():
    """Dense oracle solution of the 2048-node star (15 nodes per wavelength), computed once."""
    import oracle
    from paper_2607_00790_gb300 import inputs
    if not _DENSE:
        c = inputs.star(2048)
        k0 = inputs.k0_for_density(c)
        ph = oracle.Physics(k0, n=1.5)
        A = oracle.wsbm_dense(c, ph)
        b = oracle.rhs_planewave(c, ph, [0.3])
        _DENSE.update(curve=c, k0=k0, x=oracle.dense_solve(A, b)[:, 0])
    return _DENSE


def _star_solve(tol=1e-10):
    import torch
    from paper_2607_00790_gb300 import binding
    d = _star_dense()
    g, keep = binding.make_geom(d["curve"])
    p = binding.make_params(d["k0"], 1.5, leaf=128, nproxy=128, id_tol=tol)
    s = binding.Solver(g, p)
    s.factor()
    st = s.stats()
    u, q = s.solve(s.rhs_planewave(torch.tensor([0.3], dtype=torch.float64, device="cuda")))
    torch.cuda.synchronize()
    x = np.concatenate([u.cpu().numpy()[:, 0], q.cpu().numpy()[:, 0]])
    s.close()
    return x, st


@pytest.mark.parametrize("box_nb", [16, 32, 64])
def test_box_panel_widths_give_the_same_solver(box_nb, restore_tuning):
    """HSS build of the 2048-node star with leaves of 128 nodes (256 unknowns per box: the
    tensor-core box LU) at each box panel width: the solution is within 10x the ID tolerance of
    the dense oracle solve."""
    from paper_2607_00790_gb300 import binding
    binding.wsbm_tuning_set(box_nb=box_nb)
    x, st = _star_solve()
    assert st["lu_tc_matrices"] > 0
    d = _star_dense()
    err = np.linalg.norm(x - d["x"]) / np.linalg.norm(d["x"])
    assert err < 10 * 1e-10, err


def test_entry_shapes_change_no_bit(restore_tuning):
    """Every tile width and grid of the entry kernels gives the same solution bit for bit (the
    shapes only reorder independent entries)."""
    from paper_2607_00790_gb300 import binding
    ref, _ = _star_solve()
    for tf, ctas in [(16, 8), (64, 32), (16, 32), (64, 8)]:
        binding.wsbm_tuning_set(pair_tf=tf, pair_ctas=ctas, proxy_tf=80 - tf, proxy_ctas=40 - ctas)
        x, _ = _star_solve()
        assert x.tobytes() == ref.tobytes(), (tf, ctas)


@pytest.mark.parametrize("threads", [128, 256])
def test_qr_block_sizes_solve_to_tolerance(threads, restore_tuning):
    """The thread-per-column QR with 128 or 256 threads (its norm sums round differently): the
    solution stays within 10x the ID tolerance of the dense oracle solve."""
    from paper_2607_00790_gb300 import binding
    binding.wsbm_tuning_set(cpqr_threads=threads)
    x, _ = _star_solve()
    d = _star_dense()
    err = np.linalg.norm(x - d["x"]) / np.linalg.norm(d["x"])
    assert err < 10 * 1e-10, err


def test_autotune_build_picks_candidates(restore_tuning):
    from paper_2607_00790_gb300 import binding
    d = _star_dense()
    g, keep = binding.make_geom(d["curve"])
    p = binding.make_params(d["k0"], 1.5, leaf=128, nproxy=128, id_tol=1e-10)
    choice, ms = binding.wsbm_autotune_build(g, p)
    assert choice["pair_tf"] in (16, 32, 64) and choice["proxy_tf"] in (16, 32, 64)
    assert choice["pair_ctas"] in (8, 16, 32) and choice["proxy_ctas"] in (8, 16, 32)
    assert choice["cpqr_threads"] in (128, 256)
    assert len(ms) == 20 and all(t > 0 for t in ms)
    cand = [(tf, c) for tf in (16, 32, 64) for c in (8, 16, 32)]
    assert ms[cand.index((choice["pair_tf"], choice["pair_ctas"]))] == min(ms[0:9])
    assert ms[9 + cand.index((choice["proxy_tf"], choice["proxy_ctas"]))] == min(ms[9:18])
    assert ms[18 + [128, 256].index(choice["cpqr_threads"])] == min(ms[18:20])
    now = binding.wsbm_tuning()
    assert now["tuned_build"] and all(now[k] == choice[k] for k in binding.TUNE_BUILD_KEYS)
    # a build with the tuned shapes still solves to the ID accuracy
    x, _ = _star_solve()
    err = np.linalg.norm(x - d["x"]) / np.linalg.norm(d["x"])
    assert err < 10 * 1e-10, err
