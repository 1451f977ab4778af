"""Field off the curve on the GPU: against the oracle's representation sums on a star with
random densities (several right-hand sides, ragged target count), against the Mie series field
of the disk from its exact boundary values, and the inside/outside decision."""
import numpy as np
import pytest

import oracle
from paper_2607_00790_gb300 import inputs

pytestmark = pytest.mark.gpu


def _t(a, dt=None):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt or torch.float64, device="cuda")


def star_points(nin, nout, seed=0):
    rng = np.random.default_rng(seed)
    t = rng.uniform(0, 2 * np.pi, nin + nout)
    r = 1.0 + 0.3 * np.cos(5 * t)
    s = np.concatenate([rng.uniform(0.2, 0.7, nin), rng.uniform(1.3, 3.0, nout)])
    return s * r * np.cos(t), s * r * np.sin(t), np.arange(nin + nout) < nin


def test_field_matches_oracle_on_star():
    import torch
    from paper_2607_00790_gb300 import binding
    N = 1500
    c = inputs.star(N)
    k0 = float(inputs.k0_for_density(c))
    ph = oracle.Physics(k0, n=1.5)
    rng = np.random.default_rng(3)
    u = rng.normal(size=(N, 6)) + 1j * rng.normal(size=(N, 6))
    q = rng.normal(size=(N, 6)) + 1j * rng.normal(size=(N, 6))
    px, py, ins = star_points(77, 100)
    g, keep = binding.make_geom(c)
    p = binding.make_params(k0, 1.5)
    val, inside = binding.field(g, p, _t(u, torch.complex128), _t(q, torch.complex128), _t(px), _t(py))
    val, inside = val.cpu().numpy(), inside.cpu().numpy()
    ref, ref_in = oracle.field(c, ph, u, q, px, py)
    assert np.array_equal(inside, ins) and np.array_equal(ref_in, ins)
    err = np.abs(val - ref) / np.max(np.abs(ref), axis=0)
    assert np.max(err) < 1e-12, np.max(err)


def test_field_matches_mie_on_disk():
    import torch
    from paper_2607_00790_gb300 import binding
    N, R = 256, 1.0
    c = inputs.disk(N, R)
    ph = oracle.Physics(2 * np.pi, n=1.5)
    u, q = oracle.mie_boundary(R, ph, c["t"])
    rng = np.random.default_rng(4)
    rr = np.concatenate([rng.uniform(0.1, 0.8, 30), rng.uniform(1.2, 3.0, 30)])
    tt = rng.uniform(0, 2 * np.pi, 60)
    px, py = rr * np.cos(tt), rr * np.sin(tt)
    g, keep = binding.make_geom(c)
    p = binding.make_params(2 * np.pi, 1.5)
    val, inside = binding.field(g, p, _t(u[:, None], torch.complex128), _t(q[:, None], torch.complex128),
                                _t(px), _t(py))
    ex = oracle.mie_field(R, ph, px, py)
    assert np.array_equal(inside.cpu().numpy(), rr < R)
    assert np.max(np.abs(val.cpu().numpy()[:, 0] - ex)) / np.max(np.abs(ex)) < 1e-12
