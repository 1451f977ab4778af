"""Batched builds: several scatterers (different sizes, depths, physics and precision) built
and factored with shared launches per tree level must give exactly the results of factoring
each alone; one member is also checked against the dense oracle."""
import numpy as np
import pytest

import oracle
from paper_2607_00790_gb300 import inputs

pytestmark = pytest.mark.gpu


def members():
    out = []
    c, prm = inputs.workload("disk")
    out.append((c, dict(k0=prm["k0"], n=1.5, leaf=64, nproxy=64, tol=1e-10, precision=0)))
    c = inputs.star(1024)
    out.append((c, dict(k0=inputs.k0_for_density(c), n=1.5, leaf=64, nproxy=64, tol=1e-8, precision=0)))
    c = inputs.ellipse(768, 1.3, 0.8)
    out.append((c, dict(k0=inputs.k0_for_density(c), n=1.3, leaf=64, nproxy=64, tol=1e-8, precision=0)))
    c = inputs.star(48)
    out.append((c, dict(k0=3.0, n=1.5, leaf=64, nproxy=16, tol=1e-10, precision=0)))
    c = inputs.star(512)
    out.append((c, dict(k0=10.0, n=float(np.sqrt(5.0)), eps1=5.0, leaf=64, nproxy=64, tol=1e-10, precision=0)))
    c = inputs.star(768, a=0.2, m=3)
    out.append((c, dict(k0=inputs.k0_for_density(c), n=1.7, leaf=64, nproxy=64, tol=1e-6, precision=1)))
    return out


def params(binding, d):
    return binding.make_params(d["k0"], d["n"], eps1=d.get("eps1", 0.0), leaf=d["leaf"],
                               nproxy=d["nproxy"], id_tol=d["tol"], precision=d["precision"])


def solve(s, angles, obs):
    import torch
    u, q = s.solve(s.rhs_planewave(torch.tensor(angles, device="cuda")))
    ff = s.farfield(u, q, torch.tensor(obs, device="cuda"))
    torch.cuda.synchronize()
    return u.cpu().numpy(), q.cpu().numpy(), ff.cpu().numpy()


def test_batch_equals_individual_and_dense():
    from paper_2607_00790_gb300 import binding
    ms = members()
    geoms = [binding.make_geom(c) for c, _ in ms]
    angles = np.array([0.3, 2.0])
    obs = 2 * np.pi * np.arange(90) / 90
    b = binding.Batch([g for g, _ in geoms], [params(binding, d) for _, d in ms])
    b.factor()
    batched = [solve(b.solver(i), angles, obs) for i in range(len(ms))]
    st = b.stats()
    assert st["launches"] > 0 and st["entries_generated"] > 0
    for i, (c, d) in enumerate(ms):
        s = binding.Solver(geoms[i][0], params(binding, d))
        s.factor()
        alone = solve(s, angles, obs)
        s.close()
        for a, x in zip(batched[i], alone):
            assert np.array_equal(a, x), i
    # member 1 (star, 15 nodes per wavelength) against the dense oracle
    c, d = ms[1]
    ph = oracle.Physics(d["k0"], n=d["n"])
    x = oracle.dense_solve(oracle.wsbm_dense(c, ph), oracle.rhs_planewave(c, ph, angles))
    ud, qd = oracle.split_uq(x)
    u, q, ff = batched[1]
    assert np.linalg.norm(u - ud) / np.linalg.norm(ud) < 10 * d["tol"]
    ffd = oracle.farfield(c, ph, ud, qd, obs)
    assert np.linalg.norm(ff - ffd) / np.linalg.norm(ffd) < 10 * d["tol"]
    b.close()


def test_batch_solve_equals_individual_solves_and_replays():
    """wsbm_batch_solve (one plan, shared launches per tree step, captured CUDA graph) gives
    exactly the per-curve solves, also on a second call (graph replay) with new right-hand
    sides; curves of different depth, including a root-only one, are mixed."""
    import torch
    from paper_2607_00790_gb300 import binding
    ms = members()
    geoms = [binding.make_geom(c) for c, _ in ms]
    b = binding.Batch([g for g, _ in geoms], [params(binding, d) for _, d in ms])
    b.factor()
    rng = np.random.default_rng(5)
    for call in range(2):
        rhs = [torch.as_tensor(rng.normal(size=(2 * g.n, 3)) + 1j * rng.normal(size=(2 * g.n, 3)),
                               device="cuda") for g, _ in geoms]
        got = b.solve(rhs)
        for i in range(len(ms)):
            u, q = b.solver(i).solve(rhs[i])
            assert torch.equal(got[i][0], u) and torch.equal(got[i][1], q), (call, i)
    b.close()


def test_batch_solve_after_member_refactor():
    """Re-factoring one member of a batch on its own (wsbm_factor on the handle the batch hands
    out) releases the factors that the batch's cached solve plan points into; the next batch
    solve must build a new plan and still equal the per-curve solves."""
    import torch
    from paper_2607_00790_gb300 import binding
    ms = members()[:3]
    geoms = [binding.make_geom(c) for c, _ in ms]
    b = binding.Batch([g for g, _ in geoms], [params(binding, d) for _, d in ms])
    b.factor()
    rng = np.random.default_rng(9)
    rhs = [torch.as_tensor(rng.normal(size=(2 * g.n, 2)) + 1j * rng.normal(size=(2 * g.n, 2)),
                           device="cuda") for g, _ in geoms]
    first = b.solve(rhs)
    b.solver(1).factor()
    torch.cuda.synchronize()
    again = b.solve(rhs)
    for i in range(len(ms)):
        u, q = b.solver(i).solve(rhs[i])
        assert torch.equal(again[i][0], u) and torch.equal(again[i][1], q), i
        assert torch.equal(again[i][0], first[i][0]), i
    b.close()
