"""Gradient path on the GPU against the oracle: the Fourier curve and its reverse map, the
pairwise backward kernel of the Nystrom matrix (against the oracle's dual-number derivatives),
the right-hand-side and far-field reverse maps, the transposed HSS solve (against a dense LU of
A^T) and the whole shape / refractive-index gradient (against the oracle's dense adjoint)."""
import numpy as np
import pytest

import oracle
from paper_2607_00790_gb300 import inputs

pytestmark = pytest.mark.gpu

KEYS = ("x", "y", "nx", "ny", "w", "kappa")


def _t(a, dt=None):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt or torch.float64, device="cuda")


def fourier_case(N):
    a, b = inputs.shape_coefficients(1)
    c = inputs.fourier(N, a, b)
    return a, b, c, inputs.k0_for_density(c)


def test_curve_fourier_matches_inputs():
    from paper_2607_00790_gb300 import binding
    for N in (64, 1000):
        a, b, c, _ = fourier_case(N)
        out = binding.curve_fourier(_t(a), _t(b), N).cpu().numpy()
        for q, k in enumerate(KEYS):
            err = np.max(np.abs(out[q] - c[k])) / np.max(np.abs(c[k]))
            assert err < 1e-13, (N, k, err)


def test_curve_fourier_vjp_matches_oracle_tangents():
    from paper_2607_00790_gb300 import binding
    N = 200
    a, b, _, _ = fourier_case(N)
    rng = np.random.default_rng(3)
    g = rng.normal(size=(6, N))
    gc = binding.curve_fourier_vjp(_t(a), _t(b), N, _t(g)).cpu().numpy()
    ref = np.einsum("kqi,qi->k", oracle.fourier_tangents(N, a, b), g)
    assert np.max(np.abs(gc - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_entries_vjp_matches_oracle_dual_numbers():
    import torch
    from paper_2607_00790_gb300 import binding
    N = 256
    a, b, c, k0 = fourier_case(N)
    ph = oracle.Physics(k0, n=1.5)
    rng = np.random.default_rng(7)
    lam = rng.normal(size=2 * N) + 1j * rng.normal(size=2 * N)
    xv = rng.normal(size=2 * N) + 1j * rng.normal(size=2 * N)
    g, keep = binding.make_geom(c)
    p = binding.make_params(k0, 1.5)
    grad, gphys = binding.entries_vjp(g, p, _t(lam, torch.complex128), _t(xv, torch.complex128))
    grad = grad.cpu().numpy()
    gphys = gphys.cpu().numpy()
    # unit tangents at sampled nodes (first, last, interior) for every input kind, k1, eps1,
    # and one random direction of all node inputs at once
    nodes = [0, 1, 77, 128, 200, N - 1]
    tans, want = [], []
    for q in range(6):
        for i in nodes:
            t = np.zeros((6, N))
            t[q, i] = 1.0
            tans.append(t)
            want.append(grad[q, i])
    rnd = rng.normal(size=(6, N))
    tans += [np.zeros((6, N)), np.zeros((6, N)), rnd]
    want += [gphys[0], gphys[1], np.sum(grad * rnd)]
    tk1 = np.zeros(len(tans))
    te = np.zeros(len(tans))
    tk1[-3] = 1.0
    te[-2] = 1.0
    ref = oracle.wsbm_bilinear_tangent(c, ph, lam, xv, np.array(tans), tk1, te).real
    want = np.array(want)
    scale = np.max(np.abs(ref[:-3]))
    assert np.max(np.abs(want[:-3] - ref[:-3])) <= 1e-10 * scale
    for t in (-3, -2, -1):
        assert abs(want[t] - ref[t]) <= 1e-10 * abs(ref[t]), (t, want[t], ref[t])


def test_rhs_and_farfield_vjp_match_oracle():
    import torch
    from paper_2607_00790_gb300 import binding
    N = 300
    a, b, c, k0 = fourier_case(N)
    ph = oracle.Physics(k0, n=1.5)
    rng = np.random.default_rng(9)
    g, keep = binding.make_geom(c)
    p = binding.make_params(k0, 1.5)
    inc = np.array([0.0, 1.1])
    lam = rng.normal(size=(2 * N, 2)) + 1j * rng.normal(size=(2 * N, 2))
    gr = binding.rhs_planewave_vjp(g, p, _t(inc), _t(lam, torch.complex128)).cpu().numpy()
    T = rng.normal(size=(3, 6, N))
    for t in range(3):
        ref = sum(np.real(oracle.rhs_tangent(c, ph, th, T[t])[0] @ lam[:, a_])
                  for a_, th in enumerate(inc))
        assert abs(np.sum(gr * T[t]) - ref) <= 1e-11 * abs(ref)
    obs = 2 * np.pi * np.arange(64) / 64
    u = rng.normal(size=(N, 2)) + 1j * rng.normal(size=(N, 2))
    q = rng.normal(size=(N, 2)) + 1j * rng.normal(size=(N, 2))
    gF = rng.normal(size=(64, 2)) + 1j * rng.normal(size=(64, 2))
    v, gf = binding.farfield_vjp(g, p, _t(u, torch.complex128), _t(q, torch.complex128), _t(obs),
                                 _t(gF, torch.complex128))
    v, gf = v.cpu().numpy(), gf.cpu().numpy()
    C = oracle.farfield_matrix(c, ph, obs)
    vref = C.T @ np.conj(gF)
    assert np.max(np.abs(v - vref)) <= 1e-12 * np.max(np.abs(vref))
    for t in range(3):
        ref = sum(np.real(oracle.farfield_tangent(c, ph, u[:, r], q[:, r], obs, T[t])[0] @ np.conj(gF[:, r]))
                  for r in range(2))
        assert abs(np.sum(gf * T[t]) - ref) <= 1e-11 * abs(ref)


@pytest.mark.parametrize("name", ["disk", "star"])
def test_transposed_solve_matches_dense(name):
    import torch
    from paper_2607_00790_gb300 import binding
    if name == "disk":
        c, prm = inputs.workload("disk")
    else:
        c, prm = inputs.workload("star", N=1024)
        prm = dict(prm, leaf=64, nproxy=64, tol=1e-10)
    N = c["x"].size
    ph = oracle.Physics(prm["k0"], n=prm["n"])
    g, keep = binding.make_geom(c)
    p = binding.make_params(prm["k0"], prm["n"], leaf=prm["leaf"], nproxy=prm["nproxy"],
                            id_tol=prm["tol"])
    s = binding.Solver(g, p)
    s.factor()
    rng = np.random.default_rng(11)
    v = rng.normal(size=(2 * N, 3)) + 1j * rng.normal(size=(2 * N, 3))
    l1, l2 = s.solve_transposed(_t(v, torch.complex128))
    lam = np.concatenate([l1.cpu().numpy(), l2.cpu().numpy()])
    A = oracle.wsbm_dense(c, ph)
    ref = np.linalg.solve(A.T, v)
    err = np.linalg.norm(lam - ref) / np.linalg.norm(ref)
    assert err < 100 * prm["tol"], err  # random right-hand sides: 100x the ID tolerance
    s.close()


def test_shape_gradient_matches_dense_adjoint():
    """N = 512: loss and gradient in all 32 Fourier coefficients and n through the autograd
    Functions (HSS at ID tol 1e-12) against the oracle's dense adjoint gradient."""
    import torch
    from paper_2607_00790_gb300 import autograd as ag
    N = 512
    a, b, c, k0 = fourier_case(N)
    n = 1.5
    at, bt = inputs.shape_coefficients(2)
    obs = 2 * np.pi * np.arange(64) / 64
    ph = oracle.Physics(k0, n=n)
    target = np.abs(oracle.gradient._forward(inputs.fourier(N, at, bt), ph, 0.0, obs)[3]) ** 2
    ta = _t(a).requires_grad_(True)
    tb = _t(b).requires_grad_(True)
    tn = torch.tensor(n, dtype=torch.float64, device="cuda", requires_grad=True)
    curve = ag.fourier_curve(ta, tb, N)
    F = ag.farfield(curve, tn, k0, _t([0.0]), _t(obs), leaf=64, nproxy=64, tol=1e-12)
    L = torch.sum((F[:, 0].abs() ** 2 - _t(target)) ** 2)
    L.backward()
    g_gpu = np.concatenate([ta.grad.cpu().numpy(), tb.grad.cpu().numpy(), [tn.grad.item()]])
    tan = np.concatenate([oracle.fourier_tangents(N, a, b), np.zeros((1, 6, N))])
    tk1 = np.zeros(33)
    te = np.zeros(33)
    tk1[-1] = k0
    te[-1] = 2 * n
    L_ref, g_ref, _ = oracle.shape_loss_grad_dense(c, ph, 0.0, obs, target, tan, tk1, te)
    assert abs(L.item() - L_ref) <= 1e-8 * L_ref
    assert np.max(np.abs(g_gpu - g_ref)) <= 1e-7 * np.max(np.abs(g_ref)), (g_gpu, g_ref)
