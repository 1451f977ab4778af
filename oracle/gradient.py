"""Shape and refractive-index gradient of a far-field misfit, dense and plain (oracle part).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The loss is the squared far-field intensity misfit
    L(a, b, n) = sum_m (|u_inf(theta_m)|^2 - t_m)^2
for one incident plane wave, with the scatterer boundary r(t) = 1 + sum_j a_j cos(jt) +
b_j sin(jt) and refractive index n (k1 = n k0, eps1 = n^2 eps0; k0 held fixed).  The paper
does not differentiate its solver; the adjoint reading used here is the textbook one for a
linear system A(p) x = b(p) with an output F(p, x):
    dL/dp = Re(conj(g) . dF/dp|_x) + Re(lam^T (db/dp - dA/dp x)),   A^T lam = C^T conj(g),
with g = dL/dRe F + i dL/dIm F = 4 (|F|^2 - t) F and C = dF/dx.  Every matrix here is dense:
A from the oracle's Nystrom assembly, dA/dp from its dual-number evaluation of the same
blocks (``wsbm_bilinear_tangent``), solves by numpy's LU.
"""
from __future__ import annotations

import numpy as np


def fourier_tangents(N, acoef, bcoef):
    """Derivatives of the node arrays (x, y, nx, ny, w, kappa) of the curve
    r(t) = 1 + sum_j a_j cos(jt) + b_j sin(jt), gamma = r (cos t, sin t), t_i = 2 pi i/N,
    with respect to a_1..a_M, b_1..b_M.  Returns (2M, 6, N)."""
    acoef = np.asarray(acoef, dtype=np.float64)
    bcoef = np.asarray(bcoef, dtype=np.float64)
    M = acoef.size
    t = 2.0 * np.pi * np.arange(N) / N
    c, s = np.cos(t), np.sin(t)
    r = np.ones(N)
    r1 = np.zeros(N)
    r2 = np.zeros(N)
    for j in range(1, M + 1):
        cj, sj = np.cos(j * t), np.sin(j * t)
        r += acoef[j - 1] * cj + bcoef[j - 1] * sj
        r1 += j * (-acoef[j - 1] * sj + bcoef[j - 1] * cj)
        r2 += -j * j * (acoef[j - 1] * cj + bcoef[j - 1] * sj)
    xp, yp = r1 * c - r * s, r1 * s + r * c
    xpp = r2 * c - 2.0 * r1 * s - r * c
    ypp = r2 * s + 2.0 * r1 * c - r * s
    sp = np.sqrt(xp * xp + yp * yp)
    kap = (xp * ypp - yp * xpp) / sp**3
    out = np.zeros((2 * M, 6, N))
    for k in range(2 * M):
        j = k % M + 1
        if k < M:  # d/da_j
            dr, dr1, dr2 = np.cos(j * t), -j * np.sin(j * t), -j * j * np.cos(j * t)
        else:  # d/db_j
            dr, dr1, dr2 = np.sin(j * t), j * np.cos(j * t), -j * j * np.sin(j * t)
        dxp, dyp = dr1 * c - dr * s, dr1 * s + dr * c
        dxpp = dr2 * c - 2.0 * dr1 * s - dr * c
        dypp = dr2 * s + 2.0 * dr1 * c - dr * s
        dsp = (xp * dxp + yp * dyp) / sp
        out[k, 0] = dr * c
        out[k, 1] = dr * s
        out[k, 2] = dyp / sp - yp * dsp / sp**2
        out[k, 3] = -dxp / sp + xp * dsp / sp**2
        out[k, 4] = (2.0 * np.pi / N) * dsp
        out[k, 5] = (dxp * ypp + xp * dypp - dyp * xpp - yp * dxpp) / sp**3 - 3.0 * kap * dsp / sp
    return out


def rhs_tangent(curve, phys, theta, tan):
    """Derivative of the right-hand side [0 ; -u_in - alpha du_in/dn] (plane wave at angle
    theta) along each tangent (ntan, 6, N).  Returns (ntan, 2N)."""
    x, y, nx, ny = (np.asarray(curve[k]) for k in ("x", "y", "nx", "ny"))
    N = x.size
    tan = np.asarray(tan).reshape(-1, 6, N)
    dx, dy = np.cos(theta), np.sin(theta)
    k0 = phys.k0
    uin = np.exp(1j * k0 * (dx * x + dy * y))
    dn = dx * nx + dy * ny
    out = np.zeros((tan.shape[0], 2 * N), dtype=np.complex128)
    for t in range(tan.shape[0]):
        duin = 1j * k0 * (dx * tan[t, 0] + dy * tan[t, 1]) * uin
        ddn = dx * tan[t, 2] + dy * tan[t, 3]
        dnu = 1j * k0 * (ddn * uin + dn * duin)  # d of du_in/dn = i k0 (d.n) u_in
        out[t, N:] = -duin - phys.alpha * dnu
    return out


def farfield_matrix(curve, phys, angles):
    """C with u_inf = C [u; q] (the far-field formula of ``oracle.farfield``): (nang, 2N)."""
    x, y, nx, ny, w = (np.asarray(curve[k]) for k in ("x", "y", "nx", "ny", "w"))
    k0 = phys.k0
    pref = np.exp(1j * np.pi / 4) / np.sqrt(8 * np.pi * k0)
    th = np.asarray(angles, dtype=np.float64)[:, None]
    ph = np.exp(-1j * k0 * (np.cos(th) * x + np.sin(th) * y))
    xn = np.cos(th) * nx + np.sin(th) * ny
    return np.concatenate([pref * w * (-1j * k0 * xn) * ph, pref * w * (-phys.eps0) * ph], axis=1)


def farfield_tangent(curve, phys, u, q, angles, tan):
    """Derivative of u_inf(angles) along each tangent with the densities u, q held fixed.
    Returns (ntan, nang)."""
    x, y, nx, ny, w = (np.asarray(curve[k]) for k in ("x", "y", "nx", "ny", "w"))
    N = x.size
    tan = np.asarray(tan).reshape(-1, 6, N)
    k0 = phys.k0
    pref = np.exp(1j * np.pi / 4) / np.sqrt(8 * np.pi * k0)
    out = np.zeros((tan.shape[0], len(angles)), dtype=np.complex128)
    for a, th in enumerate(angles):
        cx, cy = np.cos(th), np.sin(th)
        ph = np.exp(-1j * k0 * (cx * x + cy * y))
        xn = cx * nx + cy * ny
        body = -1j * k0 * xn * u - phys.eps0 * q
        for t in range(tan.shape[0]):
            dph = -1j * k0 * (cx * tan[t, 0] + cy * tan[t, 1]) * ph
            dbody = -1j * k0 * (cx * tan[t, 2] + cy * tan[t, 3]) * u
            out[t, a] = pref * np.sum(tan[t, 4] * body * ph + w * dbody * ph + w * body * dph)
    return out


def _forward(curve, phys, theta_inc, angles):
    from . import farfield, rhs_planewave, wsbm_dense

    A = wsbm_dense(curve, phys)
    b = rhs_planewave(curve, phys, [theta_inc])[:, 0]
    sol = np.linalg.solve(A, b)
    N = curve["x"].size
    F = farfield(curve, phys, sol[:N], sol[N:], angles)[:, 0]
    return A, b, sol, F


def shape_loss_dense(curve, phys, theta_inc, angles, target):
    """L = sum_m (|u_inf(theta_m)|^2 - t_m)^2 from the dense Nystrom solve."""
    _, _, _, F = _forward(curve, phys, theta_inc, angles)
    return float(np.sum((np.abs(F) ** 2 - target) ** 2))


def shape_loss_grad_dense(curve, phys, theta_inc, angles, target, tan, tk1, teps1):
    """Loss and its derivative along each tangent (ntan, 6, N) + (tk1, teps1), by the dense
    adjoint.  For the Fourier shape parameters pass ``fourier_tangents``; for the refractive
    index n pass a zero node tangent with tk1 = k0 and teps1 = 2 n eps0."""
    from . import wsbm_bilinear_tangent

    A, b, sol, F = _forward(curve, phys, theta_inc, angles)
    N = curve["x"].size
    loss = float(np.sum((np.abs(F) ** 2 - target) ** 2))
    g = 4.0 * (np.abs(F) ** 2 - target) * F
    Cm = farfield_matrix(curve, phys, angles)
    v = Cm.T @ np.conj(g)
    lam = np.linalg.solve(A.T, v)
    tan = np.asarray(tan).reshape(-1, 6, N)
    dF = farfield_tangent(curve, phys, sol[:N], sol[N:], angles, tan)
    db = rhs_tangent(curve, phys, theta_inc, tan)
    dAx = wsbm_bilinear_tangent(curve, phys, lam, sol, tan, tk1, teps1)
    grad = np.real(dF @ np.conj(g)) + np.real(db @ lam) - np.real(dAx)
    return loss, grad, dict(F=F, g=g, lam=lam, sol=sol, v=v)
