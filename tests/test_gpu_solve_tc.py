"""Solves with many right-hand sides on the tensor cores: with 16 or more right-hand sides the
products of the up and down sweeps run on the tensor cores, and so do the LU solves of box
factors of 128 or more unknowns (block solves with inverted diagonal blocks); dense roots of at
least `solve_tc_min` unknowns take the block solve from 4 right-hand sides on.  Checked against
the FP64 solves of the same factors (2 right-hand sides per call), against the dense oracle, with
the root forced onto the tensor cores (solve_tc_min = 1), on a tree-less curve whose root is the
whole matrix, and batched against one-by-one."""
import numpy as np
import pytest

import oracle
from paper_2607_00790_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture
def restore_tuning():
    from paper_2607_00790_gb300 import binding
    saved = binding.wsbm_tuning()
    yield saved
    binding.wsbm_tuning_set(**saved)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _solve(s, angles):
    import torch
    u, q = s.solve(s.rhs_planewave(torch.tensor(angles, dtype=torch.float64, device="cuda")))
    torch.cuda.synchronize()
    return np.concatenate([u.cpu().numpy(), q.cpu().numpy()])


def test_tc_solve_matches_fp64_and_oracle(restore_tuning):
    """2048-node star at 15 nodes per wavelength, ID tolerance 1e-10, 16 plane waves solved at
    once (tensor cores, root included) and in calls of 2 (FP64 throughout): they agree far below
    the tolerance, and both are within 10x the tolerance of the dense oracle solve."""
    from paper_2607_00790_gb300 import binding
    c = inputs.star(2048)
    k0 = inputs.k0_for_density(c)
    angles = list(2 * np.pi * np.arange(16) / 16)
    g, keep = binding.make_geom(c)
    p = binding.make_params(k0, 1.5, leaf=128, nproxy=128, id_tol=1e-10)
    binding.wsbm_tuning_set(solve_tc_min=1)
    s = binding.Solver(g, p)
    s.factor()
    root = s.stats()["root_size"]
    assert root > 2 * 256  # several diagonal blocks of the root's block solve
    xtc = _solve(s, angles)
    x64 = np.concatenate([_solve(s, angles[i:i + 2]) for i in range(0, 16, 2)], axis=1)
    s.close()
    assert xtc.tobytes() != x64.tobytes()  # a different arithmetic path ran
    assert rel(xtc, x64) < 1e-11, rel(xtc, x64)
    ph = oracle.Physics(k0, n=1.5)
    xd = oracle.dense_solve(oracle.wsbm_dense(c, ph), oracle.rhs_planewave(c, ph, angles))
    assert rel(xtc, xd) < 10 * 1e-10, rel(xtc, xd)
    assert rel(x64, xd) < 10 * 1e-10, rel(x64, xd)


def test_root_only_curve_tc_solve_matches_oracle(restore_tuning):
    """A curve with no tree (leaf size above N: the root is the whole 2N x 2N matrix, its
    right-hand sides in the interleaved solve vector): the tensor-core solve is the dense solve
    to rounding (relative error below 1e-11; two diagonal blocks of 256 rows)."""
    from paper_2607_00790_gb300 import binding
    c = inputs.disk(256)
    angles = list(np.linspace(0.0, 3.0, 20))
    g, keep = binding.make_geom(c)
    p = binding.make_params(2 * np.pi, 1.5, leaf=512, nproxy=64, id_tol=1e-10)
    binding.wsbm_tuning_set(solve_tc_min=1)
    s = binding.Solver(g, p)
    s.factor()
    st = s.stats()
    assert st["levels"] == 0 and st["root_size"] == 512
    x = _solve(s, angles)
    s.close()
    ph = oracle.Physics(2 * np.pi, n=1.5)
    xd = oracle.dense_solve(oracle.wsbm_dense(c, ph), oracle.rhs_planewave(c, ph, angles))
    assert rel(x, xd) < 1e-11, rel(x, xd)


def test_batched_tc_solve_equals_individual(restore_tuning):
    """Three curves of different sizes and depths, 24 random right-hand sides each, boxes and
    roots on the tensor-core solves: the batched solve (one plan, one product launch per panel
    step over all curves) equals the one-curve solves bit for bit, also on a second call (graph
    replay)."""
    import torch
    from paper_2607_00790_gb300 import binding
    binding.wsbm_tuning_set(solve_tc_min=1)
    curves = [inputs.star(1024), inputs.ellipse(1536, 1.3, 0.8), inputs.star(300, a=0.2, m=3)]
    geoms = [binding.make_geom(c) for c in curves]
    ps = [binding.make_params(inputs.k0_for_density(c), 1.5, leaf=64, nproxy=64, id_tol=1e-8)
          for c in curves]
    b = binding.Batch([g for g, _ in geoms], ps)
    b.factor()
    rng = np.random.default_rng(13)
    for call in range(2):
        rhs = [torch.as_tensor(rng.normal(size=(2 * g.n, 24)) + 1j * rng.normal(size=(2 * g.n, 24)),
                               device="cuda") for g, _ in geoms]
        got = b.solve(rhs)
        for i in range(len(curves)):
            u, q = b.solver(i).solve(rhs[i])
            assert torch.equal(got[i][0], u) and torch.equal(got[i][1], q), (call, i)
    b.close()
