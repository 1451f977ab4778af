"""torch.autograd.Function wrappers for shape and refractive-index gradients.

``FourierCurve``: Fourier coefficients (a_j, b_j) -> node arrays of the curve
r(t) = 1 + sum_j a_j cos(jt) + b_j sin(jt)  (kernels wsbm_curve_fourier / _vjp).

``FarField``: node arrays and refractive index n -> far field u_inf(obs) of the plane waves
at the incident angles.  Forward: HSS build + factor, right-hand sides, solve, far field.
Backward (the adjoint method for A(p) x = b(p), F = C(p) x):
    v = C^T conj(gF),  A^T lam = v  (transposed solve with the same HSS factors),
    dL/ds = Re(conj(gF) dF/ds) + Re(lam^T db/ds) - Re(lam^T (dA/ds) x),
    dL/dn = -(k0 Re(lam^T dA/dk1 x) + 2 n eps0 Re(lam^T dA/deps1 x))   (k1 = n k0, eps1 = n^2 eps0).
Every step runs in the library's kernels; PyTorch only holds the tensors.
"""
from __future__ import annotations

import torch

from . import binding


class FourierCurve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, a, b, N):
        a = a.detach().contiguous()
        b = b.detach().contiguous()
        out = binding.curve_fourier(a, b, N)
        ctx.save_for_backward(a, b)
        ctx.N = N
        return tuple(out[k] for k in range(6))

    @staticmethod
    def backward(ctx, *grads):
        a, b = ctx.saved_tensors
        N = ctx.N
        g = torch.stack([gk if gk is not None else torch.zeros(N, dtype=torch.float64, device=a.device)
                         for gk in grads])
        gc = binding.curve_fourier_vjp(a, b, N, g)
        M = a.numel()
        return gc[:M], gc[M:], None


def fourier_curve(a, b, N):
    """(x, y, nx, ny, w, kappa) of the Fourier curve, differentiable in a and b."""
    return FourierCurve.apply(a, b, N)


class FarField(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, y, nx, ny, w, kappa, n, k0, inc, obs, leaf, nproxy, tol, precision,
                refine):
        geom, keep = binding.geom_from_tensors(x.detach(), y.detach(), nx.detach(), ny.detach(),
                                               w.detach(), kappa.detach())
        nval = float(n.detach())
        params = binding.make_params(k0, nval, leaf=leaf, nproxy=nproxy, id_tol=tol,
                                     precision=precision)
        s = binding.Solver(geom, params, device=x.device)
        s.factor()
        rhs = s.rhs_planewave(inc)
        u, q = s.solve(rhs)
        if refine:
            u, q, _ = s.refine(geom, params, rhs, u, q, iters=refine)
        F = s.farfield(u, q, obs)
        ctx.solver = s
        ctx.refine = refine
        ctx.geom, ctx.params, ctx.keep = geom, params, keep
        ctx.k0, ctx.n = k0, nval
        ctx.save_for_backward(u, q, inc, obs)
        return F

    @staticmethod
    def backward(ctx, gF):
        u, q, inc, obs = ctx.saved_tensors
        geom, params, s = ctx.geom, ctx.params, ctx.solver
        v, g_ff = binding.farfield_vjp(geom, params, u, q, obs, gF.contiguous())
        l1, l2 = s.solve_transposed(v)
        if ctx.refine:
            l1, l2, _ = s.refine(geom, params, v, l1, l2, iters=ctx.refine, trans=True)
        lam = torch.cat([l1, l2], dim=0)
        g_rhs = binding.rhs_planewave_vjp(geom, params, inc, lam)
        sol = torch.cat([u, q], dim=0)
        g_a = torch.zeros_like(g_ff)
        gphys = torch.zeros(2, dtype=torch.float64, device=u.device)
        for c in range(u.shape[1]):
            ga, gp = binding.entries_vjp(geom, params, lam[:, c].contiguous(), sol[:, c].contiguous())
            g_a += ga
            gphys += gp
        g = g_ff + g_rhs - g_a
        gn = -(gphys[0] * ctx.k0 + gphys[1] * 2.0 * ctx.n * params.eps0)
        s.close()
        ctx.solver = None
        return (g[0], g[1], g[2], g[3], g[4], g[5], gn.reshape(()), None, None, None, None,
                None, None, None, None)


def farfield(curve, n, k0, inc, obs, leaf=64, nproxy=64, tol=1e-10, precision=0, refine=0):
    """Far field (nobs x ninc) of the node arrays `curve` = (x, y, nx, ny, w, kappa) with
    refractive index n (a 0-d tensor), differentiable in the node arrays and n.  refine > 0
    adds that many refinement steps against the dense matrix-free product to the solution and
    to the adjoint multipliers (HSS factor as preconditioner; O(N^2) per step)."""
    x, y, nx, ny, w, kappa = curve
    return FarField.apply(x, y, nx, ny, w, kappa, n, float(k0), inc, obs, int(leaf), int(nproxy),
                          float(tol), int(precision), int(refine))
