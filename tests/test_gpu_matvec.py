"""Matrix-free dense product on the GPU: against the oracle's product, and as the residual of
HSS solutions (within the ID tolerance, and driven to rounding level by iterative
refinement with the HSS factor as preconditioner)."""
import numpy as np
import pytest

import oracle
from paper_2607_00790_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_matvec_matches_oracle():
    import torch
    from paper_2607_00790_gb300 import binding
    c, prm = inputs.workload("star", N=700)  # ragged against the 128-node tiles
    N = 700
    ph = oracle.Physics(prm["k0"], n=prm["n"])
    rng = np.random.default_rng(2)
    x = rng.normal(size=(2 * N, 2)) + 1j * rng.normal(size=(2 * N, 2))
    g, keep = binding.make_geom(c)
    p = binding.make_params(prm["k0"], prm["n"])
    y = binding.wsbm_matvec(g, p, torch.as_tensor(x, device="cuda")).cpu().numpy()
    ref = oracle.wsbm_matvec(c, ph, x)
    assert np.linalg.norm(y - ref) <= 1e-12 * np.linalg.norm(ref)


def test_hss_residual_and_refinement():
    import torch
    from paper_2607_00790_gb300 import binding
    c, prm = inputs.workload("star", N=4096)
    tol = 1e-8
    g, keep = binding.make_geom(c)
    p = binding.make_params(prm["k0"], prm["n"], leaf=128, nproxy=128, id_tol=tol)
    s = binding.Solver(g, p)
    s.factor()
    rhs = s.rhs_planewave(torch.tensor([0.0, 2.0], dtype=torch.float64, device="cuda"))
    u, q = s.solve(rhs)
    u, q, res = s.refine(g, p, rhs, u, q, iters=3)
    assert res[0] < 10 * tol, res
    assert res[-1] < 1e-13, res
    s.close()


def test_transposed_matvec_and_adjoint_refinement():
    import torch
    from paper_2607_00790_gb300 import binding
    c, prm = inputs.workload("star", N=700)
    N = 700
    ph = oracle.Physics(prm["k0"], n=prm["n"])
    rng = np.random.default_rng(4)
    x = rng.normal(size=(2 * N, 2)) + 1j * rng.normal(size=(2 * N, 2))
    g, keep = binding.make_geom(c)
    p = binding.make_params(prm["k0"], prm["n"], leaf=64, nproxy=64, id_tol=1e-6)
    y = binding.wsbm_matvec(g, p, torch.as_tensor(x, device="cuda"), trans=True).cpu().numpy()
    A = oracle.wsbm_dense(c, ph)
    ref = A.T @ x
    assert np.linalg.norm(y - ref) <= 1e-12 * np.linalg.norm(ref)
    # adjoint solve at a loose ID tolerance, refined to rounding level
    s = binding.Solver(g, p)
    s.factor()
    v = torch.as_tensor(x[:, :1], device="cuda")
    l1, l2 = s.solve_transposed(v)
    l1, l2, res = s.refine(g, p, v, l1, l2, iters=4, trans=True)
    assert res[0] > 1e-9 and res[-1] < 1e-13, res
    lam = np.concatenate([l1.cpu().numpy(), l2.cpu().numpy()])
    exact = np.linalg.solve(A.T, x[:, :1])
    assert np.linalg.norm(lam - exact) <= 1e-11 * np.linalg.norm(exact)
    s.close()
