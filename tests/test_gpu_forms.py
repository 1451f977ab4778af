"""The comparison formulations on the GPU (eqs. bm and pmchwt, Sec. II): entries and proxy row
blocks element by element against the oracle, the HSS solution against the oracle's dense
solve of the same formulation, and the calls that implement eq. (weakly_bm) only refusing them."""
import numpy as np
import pytest

import oracle
from paper_2607_00790_gb300 import inputs

pytestmark = pytest.mark.gpu

FORMS = [1, 2]  # WSBM_FORM_BM, WSBM_FORM_PMCHWT


def _params(ph, form, **kw):
    from paper_2607_00790_gb300 import binding
    return binding.make_params(ph.k0, ph.k1 / ph.k0, ph.eps0, ph.eps1, formulation=form, **kw)


def _entries(curve, ph, form, rows, cols):
    import torch
    from paper_2607_00790_gb300 import binding
    g, keep = binding.make_geom(curve)
    r = torch.tensor(np.asarray(rows, dtype=np.int64), device="cuda")
    c = torch.tensor(np.asarray(cols, dtype=np.int64), device="cuda")
    out = binding.wsbm_entries_raw(g, _params(ph, form), r, c)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _compare(got, ref):
    assert np.all(np.isfinite(got))
    row_scale = np.abs(ref).max(axis=1, keepdims=True)
    err = np.abs(got - ref) / row_scale
    assert err.max() <= 1e-11, (err.max(), np.unravel_index(np.argmax(err), err.shape))
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-12


@pytest.mark.parametrize("form", FORMS)
def test_disk_full_matrix(form):
    c, prm = inputs.workload("disk")
    ph = oracle.Physics(prm["k0"], n=prm["n"])
    idx = np.arange(2 * c["x"].size)
    _compare(_entries(c, ph, form, idx, idx), oracle.form_dense(c, ph, form))


@pytest.mark.parametrize("form", FORMS)
def test_star_ragged_block_with_diagonal(form):
    c = inputs.star(700)
    ph = oracle.Physics(inputs.k0_for_density(c), n=1.5)
    A = oracle.form_dense(c, ph, form)
    rng = np.random.default_rng(11)
    rows = np.concatenate([np.arange(40, 77), rng.choice(1400, 150, replace=False)])
    cols = np.concatenate([np.arange(60, 101), rng.choice(1400, 93, replace=False)])
    _compare(_entries(c, ph, form, rows, cols), A[np.ix_(rows, cols)])


@pytest.mark.parametrize("form", FORMS)
def test_proxy_row_blocks(form):
    import torch
    from paper_2607_00790_gb300 import binding
    c = inputs.star(1024)
    ph = oracle.Physics(inputs.k0_for_density(c), n=1.5)
    nodes = np.arange(128, 256)
    box = np.concatenate([nodes, nodes + 1024])
    circ = oracle.proxy_circle(c, nodes)
    P = 200
    ref = oracle.proxy_row_block_form(c, ph, box, circ, P, form)
    g, keep = binding.make_geom(c)
    idx = torch.tensor(box, device="cuda")
    got = binding.wsbm_proxy_block(g, _params(ph, form), 0, idx, circ, P).cpu().numpy()
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= 1e-12 * scale
    # the column block is shared by the formulations
    col_f = binding.wsbm_proxy_block(g, _params(ph, form), 1, idx, circ, P).cpu().numpy()
    col_w = binding.wsbm_proxy_block(g, _params(ph, 0), 1, idx, circ, P).cpu().numpy()
    assert np.array_equal(col_f, col_w)


@pytest.mark.parametrize("form", FORMS)
def test_hss_solve_vs_dense(form):
    import torch
    from paper_2607_00790_gb300 import binding
    N = 1024
    c = inputs.star(N)
    ph = oracle.Physics(inputs.k0_for_density(c), n=1.5)
    tol = 1e-8
    angles = [0.0, 2.0]
    g, keep = binding.make_geom(c)
    s = binding.Solver(g, _params(ph, form, leaf=64, nproxy=64, id_tol=tol))
    s._keep = keep
    s.factor()
    ang = torch.tensor(angles, dtype=torch.float64, device="cuda")
    rhs = s.rhs_planewave(ang)
    u, q = s.solve(rhs)
    b = oracle.form_rhs(c, ph, angles, form)
    # the phase k0 d.x reaches about 62: one-ulp differences of the plane wave are about 1e-14
    assert np.linalg.norm(rhs.cpu().numpy() - b) <= 1e-12 * np.linalg.norm(b)
    A = oracle.form_dense(c, ph, form)
    x = oracle.dense_solve(A, b)
    ud, qd = x[:N], x[N:]
    rel = lambda a, r: np.linalg.norm(a - r) / np.linalg.norm(r)  # noqa: E731
    xh = np.concatenate([u.cpu().numpy(), q.cpu().numpy()])
    obs = torch.tensor(2 * np.pi * np.arange(90) / 90, device="cuda")
    ff = s.farfield(u, q, obs).cpu().numpy()
    ffd = oracle.farfield(c, ph, ud, qd, obs.cpu().numpy())
    if form == 1:  # second kind like eq. (weakly_bm): condition number 1.1e3 here
        assert rel(xh[:N], ud) < 10 * tol and rel(xh[N:], qd) < 10 * tol
        assert rel(ff, ffd) < 10 * tol
    else:
        # eq. (pmchwt) is of the first kind in q (S_k in one block, the hypersingular N_k in
        # the other): condition number 8.2e4 against 4.8e2 for eq. (weakly_bm) on this curve.
        # The compression is checked by the residual r = A xh - b; the densities and the far
        # field are then held to what that residual allows, xh - x = A^-1 r:
        #   |xh - x| <= |A^-1|_2 |r|,   |F xh - F x| <= |F|_2 |A^-1|_2 |r|
        # (F: the far-field map of (u, q), built column by column from the oracle).
        r = A @ xh - b
        assert np.linalg.norm(r) / np.linalg.norm(b) < 10 * tol, np.linalg.norm(r) / np.linalg.norm(b)
        inv_norm = 1.0 / np.linalg.svd(A, compute_uv=False)[-1]
        bound_x = inv_norm * np.linalg.norm(r)
        assert np.linalg.norm(xh - x) <= bound_x * (1 + 1e-6), (np.linalg.norm(xh - x), bound_x)
        eye = np.eye(2 * N, dtype=np.complex128)
        F = oracle.farfield(c, ph, eye[:N], eye[N:], obs.cpu().numpy())
        bound_f = np.linalg.norm(F, 2) * bound_x
        assert np.linalg.norm(ff - ffd) <= bound_f * (1 + 1e-6), (np.linalg.norm(ff - ffd), bound_f)
    assert s.stats()["max_rank"] > 0
    s.close()


def test_calls_of_eq_weakly_bm_only_refuse_the_other_forms():
    import torch
    from paper_2607_00790_gb300 import binding
    c = inputs.star(256)
    ph = oracle.Physics(inputs.k0_for_density(c), n=1.5)
    g, keep = binding.make_geom(c)
    x = torch.zeros(512, 1, dtype=torch.complex128, device="cuda")
    with pytest.raises(binding.WsbmError):
        binding.wsbm_matvec(g, _params(ph, 1), x)
    with pytest.raises(binding.WsbmError):
        binding.Solver(g, _params(ph, 2, precision=binding.WSBM_MIXED))
    with pytest.raises(binding.WsbmError):
        binding.Solver(g, _params(ph, 3))
