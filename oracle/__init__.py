"""CPU oracle for the weakly singular Burton-Miller (WSBM) Nystrom system.

TEST INFRASTRUCTURE ONLY.  The product library never imports, links or calls this package;
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` do.
It shares no code with the CUDA path.

Two parts (paper: Matsumoto & Yokota, TE-mode transmission, Secs. II-IV):

* O-dense: the Nystrom matrix of eq. (weakly_bm) assembled entry by entry in C++17
  (``wsbm_oracle.cpp``; Hankel values from ``std::cyl_bessel_jl`` / ``std::cyl_neumannl``),
  followed by a dense LU solve (``numpy.linalg.solve``).  The HSS solver approximates this
  system to the interpolative-decomposition tolerance.
* O-phys: the Mie series for a disk (Sec. IV compares against the closed-form solution of
  the disk), which fixes the discretisation and the paper's O(h^3) claim.

* Shape gradients (``gradient.py``): the dense adjoint of a far-field intensity misfit,
  with matrix derivatives from a dual-number evaluation of the same blocks.

Every public function states the passage it follows.  Nothing here is tuned for speed.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import build as _build, library_path

_LIB = None

_d = ctypes.c_double
_i64 = ctypes.c_int64
_pd = ctypes.POINTER(ctypes.c_double)
_pi64 = ctypes.POINTER(ctypes.c_int64)

EULER_GAMMA = 0.57721566490153286060651209008240243


def _lib():
    global _LIB
    if _LIB is None:
        path = library_path()
        if not os.path.exists(path):
            _build()
        lib = ctypes.CDLL(path)
        lib.orc_hankel01.argtypes = [_pd, _i64, _pd]
        lib.orc_f1.argtypes = [_pd, _i64, _pd]
        geo = [_i64, _pd, _pd, _pd, _pd, _pd, _pd, _d, _d, _d, _d]
        lib.orc_wsbm_entries.argtypes = geo + [_pi64, _i64, _pi64, _i64, _pd]
        lib.orc_wsbm_dense.argtypes = geo + [_pd]
        lib.orc_wsbm_matvec.argtypes = geo + [_pd, _i64, _pd]
        lib.orc_proxy_circle.argtypes = [_pd, _pd, _pi64, _i64, _d, _pd]
        lib.orc_proxy_row_block.argtypes = geo + [_pi64, _i64, _d, _d, _d, _i64, _pd]
        lib.orc_proxy_col_block.argtypes = geo + [_pi64, _i64, _d, _d, _d, _i64, _pd]
        lib.orc_wsbm_bilinear_tangent.argtypes = geo + [_pd, _pd, _i64, _pd, _pd, _pd, _pd]
        lib.orc_field.argtypes = geo + [_pd, _pd, _i64, _pd, _pd, _i64, _pd,
                                        ctypes.POINTER(ctypes.c_int32)]
        lib.orc_field.restype = ctypes.c_int
        lib.orc_form_dense.argtypes = geo + [ctypes.c_int32, _pd]
        lib.orc_form_dense.restype = ctypes.c_int
        lib.orc_layer_ops.argtypes = geo[:9] + [_pd]
        lib.orc_layer_ops.restype = ctypes.c_int
        lib.orc_proxy_row_block_form.argtypes = geo + [ctypes.c_int32, _pi64, _i64, _d, _d, _d, _i64, _pd]
        lib.orc_proxy_row_block_form.restype = ctypes.c_int
        for f in (lib.orc_hankel01, lib.orc_f1, lib.orc_wsbm_entries, lib.orc_wsbm_dense,
                  lib.orc_wsbm_matvec, lib.orc_proxy_circle, lib.orc_proxy_row_block,
                  lib.orc_proxy_col_block, lib.orc_wsbm_bilinear_tangent):
            f.restype = ctypes.c_int
        _LIB = lib
    return _LIB


class use_library:
    """Temporarily point the oracle at another build of ``wsbm_oracle.cpp`` (used by the test
    that plants mistakes in a copy of the oracle to show the pins catch them)."""

    def __init__(self, path):
        self.path = path

    def __enter__(self):
        global _LIB
        self.saved = _LIB
        _LIB = None
        saved_path = library_path
        globals()["library_path"] = lambda: self.path
        try:
            _lib()
        finally:
            globals()["library_path"] = saved_path
        return self

    def __exit__(self, *exc):
        global _LIB
        _LIB = self.saved
        return False


def _p(a):
    return a.ctypes.data_as(_pd)


def _pi(a):
    return a.ctypes.data_as(_pi64)


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Physics:
    """Material and wave parameters of eq. (weakly_bm).

    k_j = omega sqrt(eps_j mu_j) with mu_0 = mu_1 = 1 (Sec. II; Table para), so for a
    refractive index n: eps1 = n^2 eps0 and k1 = n k0.  alpha = i/k0 (Sec. II).
    """

    def __init__(self, k0, n=None, eps0=1.0, eps1=None):
        if eps1 is None:
            eps1 = n * n * eps0
        self.k0 = float(k0)
        self.eps0 = float(eps0)
        self.eps1 = float(eps1)
        self.k1 = float(k0) * float(np.sqrt(self.eps1 / self.eps0))
        self.alpha = 1j / self.k0

    def args(self):
        return (self.k0, self.k1, self.eps0, self.eps1)


def _geo(curve):
    arrs = [_c64(curve[k]) for k in ("x", "y", "nx", "ny", "w", "kappa")]
    return arrs


# ----------------------------------------------------------------------------- Hankel ----
def hankel01(z):
    """H0^(1)(z), H1^(1)(z) from libstdc++'s long-double Bessel functions, rounded to double."""
    z = _c64(np.atleast_1d(z))
    out = np.empty(4 * z.size)
    rc = _lib().orc_hankel01(_p(z), z.size, _p(out))
    assert rc == 0
    o = out.reshape(-1, 4)
    return o[:, 0] + 1j * o[:, 1], o[:, 2] + 1j * o[:, 3]


def f1(z):
    """F1(z) = H1(z)/z + 2i/(pi z^2), formed in long double."""
    z = _c64(np.atleast_1d(z))
    out = np.empty(2 * z.size)
    _lib().orc_f1(_p(z), z.size, _p(out))
    o = out.reshape(-1, 2)
    return o[:, 0] + 1j * o[:, 1]


# ---------------------------------------------------------------------------- entries ----
def wsbm_entries(curve, phys, rows, cols):
    """Entries A[rows, cols] of the WSBM Nystrom matrix, eq. (weakly_bm), paper order [u; q]."""
    g = _geo(curve)
    n = g[0].size
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    cols = np.ascontiguousarray(cols, dtype=np.int64)
    out = np.empty(2 * rows.size * cols.size)
    rc = _lib().orc_wsbm_entries(n, *[_p(a) for a in g], *phys.args(), _pi(rows), rows.size,
                                 _pi(cols), cols.size, _p(out))
    if rc != 0:
        raise ValueError("index out of range")
    return out.view(np.complex128).reshape(cols.size, rows.size).T


def wsbm_dense(curve, phys):
    """The dense 2N x 2N WSBM matrix (paper order), eq. (weakly_bm) with the one-point
    corrected diagonal."""
    g = _geo(curve)
    n = g[0].size
    out = np.empty(2 * (2 * n) * (2 * n))
    _lib().orc_wsbm_dense(n, *[_p(a) for a in g], *phys.args(), _p(out))
    return out.view(np.complex128).reshape(2 * n, 2 * n).T


def wsbm_matvec(curve, phys, xvec):
    """y = A x without storing A (paper order); xvec: (2N,) or (2N, nrhs) complex."""
    g = _geo(curve)
    n = g[0].size
    xv = np.asarray(xvec, dtype=np.complex128)
    one = xv.ndim == 1
    xm = np.asfortranarray(xv.reshape(2 * n, -1))
    nrhs = xm.shape[1]
    xin = np.ascontiguousarray(xm.T).view(np.float64).ravel()
    out = np.empty(2 * 2 * n * nrhs)
    _lib().orc_wsbm_matvec(n, *[_p(a) for a in g], *phys.args(), _p(xin), nrhs, _p(out))
    y = out.view(np.complex128).reshape(nrhs, 2 * n).T
    return y[:, 0] if one else y


# ------------------------------------------------------------------------------ proxy ----
def proxy_circle(curve, nodes, ratio=1.5):
    """Proxy circle of a box (proxy-surface method, Sec. III): centre = bounding-box midpoint
    of the nodes, radius = ratio * (largest node distance from the centre)."""
    nodes = np.ascontiguousarray(nodes, dtype=np.int64)
    out = np.empty(4)
    rc = _lib().orc_proxy_circle(_p(_c64(curve["x"])), _p(_c64(curve["y"])), _pi(nodes),
                                 nodes.size, float(ratio), _p(out))
    assert rc == 0
    return out[0], out[1], out[3]


def proxy_row_block(curve, phys, rows, circle, P):
    """Box equations x 2P combined-field proxy sources (k1 sources, then k0 sources)."""
    g = _geo(curve)
    n = g[0].size
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    out = np.empty(2 * rows.size * 2 * P)
    cx, cy, rho = circle
    _lib().orc_proxy_row_block(n, *[_p(a) for a in g], *phys.args(), _pi(rows), rows.size,
                               cx, cy, rho, int(P), _p(out))
    return out.view(np.complex128).reshape(2 * P, rows.size).T


def proxy_row_block_form(curve, phys, rows, circle, P, form):
    """Proxy row block of form 0 (eq. weakly_bm), 1 (eq. bm) or 2 (eq. pmchwt): box equations x
    2P combined-field proxy sources (k1 sources, then k0 sources)."""
    g = _geo(curve)
    n = g[0].size
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    out = np.empty(2 * rows.size * 2 * P)
    cx, cy, rho = circle
    rc = _lib().orc_proxy_row_block_form(n, *[_p(a) for a in g], *phys.args(), int(form), _pi(rows),
                                         rows.size, cx, cy, rho, int(P), _p(out))
    if rc:
        raise ValueError(f"form {form}")
    return out.view(np.complex128).reshape(2 * P, rows.size).T


def proxy_col_block(curve, phys, cols, circle, P):
    """2P proxy evaluations (psi1 then psi0 at the proxy points) x box unknowns."""
    g = _geo(curve)
    n = g[0].size
    cols = np.ascontiguousarray(cols, dtype=np.int64)
    out = np.empty(2 * 2 * P * cols.size)
    cx, cy, rho = circle
    _lib().orc_proxy_col_block(n, *[_p(a) for a in g], *phys.args(), _pi(cols), cols.size,
                               cx, cy, rho, int(P), _p(out))
    return out.view(np.complex128).reshape(cols.size, 2 * P).T


# ------------------------------------------------------------------ right-hand side ----
def rhs_planewave(curve, phys, angles):
    """Right-hand side of eq. (weakly_bm): [0 ; -u_in - alpha du_in/dn] for plane waves
    u_in = exp(i k0 d.x), d = (cos theta, sin theta).  Returns (2N, nang)."""
    angles = np.atleast_1d(np.asarray(angles, dtype=np.float64))
    x, y, nx, ny = (np.asarray(curve[k]) for k in ("x", "y", "nx", "ny"))
    n = x.size
    b = np.zeros((2 * n, angles.size), dtype=np.complex128)
    for a, th in enumerate(angles):
        dx, dy = np.cos(th), np.sin(th)
        uin = np.exp(1j * phys.k0 * (dx * x + dy * y))
        duin = 1j * phys.k0 * (dx * nx + dy * ny) * uin
        b[n:, a] = -uin - phys.alpha * duin
    return b


# --------------------------------------------- the comparison formulations (eqs. bm, pmchwt) ----
FORM_WSBM, FORM_BM, FORM_PMCHWT = 0, 1, 2


def form_dense(curve, phys, form):
    """Dense 2N x 2N matrix, unknowns [u ; q]: form 0 eq. (weakly_bm), 1 eq. (bm), 2 eq.
    (pmchwt) with its columns in the order (u, q).  N_k alone (forms 1, 2) takes the one-point
    correction -pi/(6 w_i) of its 1/r^2 part plus the log correction; its O(1) diagonal term
    is left out, so both converge at first order (Sec. II, after eq. (bm))."""
    g = _geo(curve)
    n = g[0].size
    out = np.empty(2 * (2 * n) * (2 * n))
    rc = _lib().orc_form_dense(n, *[_p(a) for a in g], *phys.args(), int(form), _p(out))
    if rc:
        raise ValueError(f"form {form}")
    return out.view(np.complex128).reshape(2 * n, 2 * n).T


def form_rhs(curve, phys, angles, form):
    """Right-hand sides for plane waves: forms 0 and 1 [0 ; -u_in - alpha du_in/dn] (eqs.
    weakly_bm, bm), form 2 [-u_in ; -eps0^-1 du_in/dn] (eq. pmchwt)."""
    if form in (FORM_WSBM, FORM_BM):
        return rhs_planewave(curve, phys, angles)
    angles = np.atleast_1d(np.asarray(angles, dtype=np.float64))
    x, y, nx, ny = (np.asarray(curve[k]) for k in ("x", "y", "nx", "ny"))
    n = x.size
    b = np.zeros((2 * n, angles.size), dtype=np.complex128)
    for a, th in enumerate(angles):
        dx, dy = np.cos(th), np.sin(th)
        uin = np.exp(1j * phys.k0 * (dx * x + dy * y))
        b[:n, a] = -uin
        b[n:, a] = -(1j * phys.k0 * (dx * nx + dy * ny) * uin) / phys.eps0
    return b


def layer_ops(curve, k0, k1):
    """The discretized S, D, D*, N at k0 and k1 (one-point corrected diagonals, weights folded
    in) as a dict of N x N complex matrices: S0, S1, D0, D1, Ds0, Ds1, N0, N1."""
    g = _geo(curve)
    n = g[0].size
    out = np.empty(2 * 8 * n * n)
    _lib().orc_layer_ops(n, *[_p(a) for a in g], float(k0), float(k1), _p(out))
    m = out.view(np.complex128).reshape(8, n, n)
    names = ("S0", "S1", "D0", "D1", "Ds0", "Ds1", "N0", "N1")
    return {nm: m[t].T.copy() for t, nm in enumerate(names)}


def dense_solve(A, b):
    """Dense LU with partial pivoting (LAPACK through numpy) of the Nystrom system."""
    return np.linalg.solve(A, b)


def split_uq(sol):
    n = sol.shape[0] // 2
    return sol[:n], sol[n:]


def farfield(curve, phys, u, q, angles):
    """Far-field pattern of the scattered field,
    u_inf(theta) = e^{i pi/4}/sqrt(8 pi k0) sum_j w_j [-i k0 (xh.n_j) u_j - eps0 q_j] e^{-i k0 xh.y_j},
    from the exterior Green representation u_sc = D_k0[u] - S_k0[eps0 q] (q = eps0^-1 du/dn,
    Sec. II) and the large-argument form of H0.  The paper does not print it."""
    angles = np.atleast_1d(np.asarray(angles, dtype=np.float64))
    x, y, nx, ny, w = (np.asarray(curve[k]) for k in ("x", "y", "nx", "ny", "w"))
    u = np.asarray(u).reshape(x.size, -1)
    q = np.asarray(q).reshape(x.size, -1)
    k0 = phys.k0
    out = np.zeros((angles.size, u.shape[1]), dtype=np.complex128)
    pref = np.exp(1j * np.pi / 4) / np.sqrt(8 * np.pi * k0)
    for a, th in enumerate(angles):
        cx, cy = np.cos(th), np.sin(th)
        ph = np.exp(-1j * k0 * (cx * x + cy * y))
        xn = cx * nx + cy * ny
        for c in range(u.shape[1]):
            out[a, c] = pref * np.sum(w * (-1j * k0 * xn * u[:, c] - phys.eps0 * q[:, c]) * ph)
    return out


def field(curve, phys, u, q, tx, ty):
    """Field at points off the curve from the densities (integral representations; Sec. II
    notes the domain solution follows from u and q): scattered field D_k0[u] - eps0 S_k0[q] at
    exterior points, total field eps1 S_k1[q] - D_k1[u] at interior points (side by the
    crossing-number test).  u, q: (N,) or (N, nrhs).  Returns (values (nt, nrhs), inside)."""
    g = _geo(curve)
    n = g[0].size
    U = np.asarray(u, dtype=np.complex128).reshape(n, -1)
    Q = np.asarray(q, dtype=np.complex128).reshape(n, -1)
    nrhs = U.shape[1]
    uu = np.ascontiguousarray(U.T).view(np.float64).ravel()
    qq = np.ascontiguousarray(Q.T).view(np.float64).ravel()
    tx = _c64(np.atleast_1d(tx))
    ty = _c64(np.atleast_1d(ty))
    out = np.empty(2 * tx.size * nrhs)
    inside = np.empty(tx.size, dtype=np.int32)
    _lib().orc_field(n, *[_p(a) for a in g], *phys.args(), _p(uu), _p(qq), nrhs, _p(tx), _p(ty),
                     tx.size, _p(out), inside.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    return out.view(np.complex128).reshape(nrhs, tx.size).T, inside.astype(bool)


# -------------------------------------------------------------------------------- Mie ----
def mie_disk(R, phys, theta_inc=0.0, mmax=None):
    """Mie-series coefficients for TE transmission by a disk of radius R centred at 0.

    Transmission conditions u0 = u1 and eps0^-1 du0/dn = eps1^-1 du1/dn on r = R (Sec. II,
    q = scaled normal derivative).  Incident e^{i k0 x.d} = sum_m i^m J_m(k0 r) e^{im(t - t_inc)};
    scattered sum a_m H_m(k0 r) e^{im(t - t_inc)};  interior sum b_m J_m(k1 r) e^{im(t - t_inc)}.
    Returns (m, a_m, b_m).
    """
    from scipy.special import hankel1, h1vp, jv, jvp

    k0, k1 = phys.k0, phys.k1
    if mmax is None:
        mmax = int(np.ceil(k1 * R + 40))
    m = np.arange(-mmax, mmax + 1)
    beta = k1 * phys.eps0 / (k0 * phys.eps1)
    J0 = jv(m, k0 * R)
    J0p = jvp(m, k0 * R)
    J1 = jv(m, k1 * R)
    J1p = jvp(m, k1 * R)
    H0 = hankel1(m, k0 * R)
    H0p = h1vp(m, k0 * R)
    im = (1j) ** (m % 4)
    a = im * (beta * J0 * J1p - J0p * J1) / (H0p * J1 - beta * H0 * J1p)
    b = (im * J0 + a * H0) / J1
    return m, a, b


def mie_boundary(R, phys, theta, theta_inc=0.0):
    """Exact boundary values u and q = eps1^-1 du1/dn at polar angles theta on the disk."""
    from scipy.special import jv, jvp

    m, a, b = mie_disk(R, phys, theta_inc)
    e = np.exp(1j * np.outer(np.asarray(theta) - theta_inc, m))
    u = e @ (b * jv(m, phys.k1 * R))
    q = (phys.k1 / phys.eps1) * (e @ (b * jvp(m, phys.k1 * R)))
    return u, q


def mie_field(R, phys, px, py, theta_inc=0.0):
    """Exact field of the disk at points: scattered sum a_m H_m(k0 r) e^{im(t - t_inc)} outside,
    total sum b_m J_m(k1 r) e^{im(t - t_inc)} inside (the split returned by ``field``)."""
    from scipy.special import hankel1, jv

    m, a, b = mie_disk(R, phys, theta_inc)
    px, py = np.atleast_1d(px), np.atleast_1d(py)
    r, t = np.hypot(px, py), np.arctan2(py, px)
    e = np.exp(1j * np.outer(t - theta_inc, m))
    out = np.where(r > R, np.sum(e * a * hankel1(m, phys.k0 * r[:, None]), axis=1),
                   np.sum(e * b * jv(m, phys.k1 * r[:, None]), axis=1))
    return out


def mie_farfield(R, phys, angles, theta_inc=0.0):
    """u_inf(theta) = sqrt(2/(pi k0)) e^{-i pi/4} sum_m a_m (-i)^m e^{im(theta - theta_inc)}."""
    m, a, _ = mie_disk(R, phys, theta_inc)
    e = np.exp(1j * np.outer(np.asarray(angles) - theta_inc, m))
    mi = (-1j) ** (m % 4)
    return np.sqrt(2 / (np.pi * phys.k0)) * np.exp(-1j * np.pi / 4) * (e @ (a * mi))


# ----------------------------------------------------- circle operator eigenvalues ----
def circle_eigenvalues(k, R, m):
    """Eigenvalues of S_k, D_k, D*_k, N_k on a circle of radius R for e^{im theta}
    (separation of variables with the Graf addition theorem; derived, not in the paper):
      S: (i pi R/2) J_m H_m,  D = D*: (i pi k R/4)(J_m' H_m + J_m H_m'),  N: (i pi k^2 R/2) J_m' H_m'
    all at k R."""
    from scipy.special import hankel1, h1vp, jv, jvp

    z = k * R
    J, Jp, H, Hp = jv(m, z), jvp(m, z), hankel1(m, z), h1vp(m, z)
    S = 1j * np.pi * R / 2 * J * H
    D = 1j * np.pi * k * R / 4 * (Jp * H + J * Hp)
    N = 1j * np.pi * k * k * R / 2 * Jp * Hp
    return S, D, N


# ------------------------------------------------------- derivatives (shape gradient) ----
def wsbm_bilinear_tangent(curve, phys, lam, xv, tan, tk1, teps1):
    """Directional derivatives d/ds (lam^T A x) of the Nystrom matrix of eq. (weakly_bm) with
    the one-point corrected diagonal, by forward-mode (dual-number) evaluation of the same
    block definitions.  lam, xv: (2N,) complex, paper order; tan: (ntan, 6, N) tangents of
    (x, y, nx, ny, w, kappa); tk1, teps1: (ntan,) tangents of k1 and eps1.  Returns (ntan,)."""
    g = _geo(curve)
    n = g[0].size
    tan = _c64(np.asarray(tan, dtype=np.float64).reshape(-1, 6, n))
    ntan = tan.shape[0]
    tk1 = _c64(np.broadcast_to(np.asarray(tk1, dtype=np.float64), (ntan,)))
    teps1 = _c64(np.broadcast_to(np.asarray(teps1, dtype=np.float64), (ntan,)))
    lam = np.ascontiguousarray(lam, dtype=np.complex128).view(np.float64)
    xv = np.ascontiguousarray(xv, dtype=np.complex128).view(np.float64)
    out = np.empty(2 * ntan)
    _lib().orc_wsbm_bilinear_tangent(n, *[_p(a) for a in g], *phys.args(), _p(lam), _p(xv),
                                     ntan, _p(tan), _p(tk1), _p(teps1), _p(out))
    return out.view(np.complex128)


from .gradient import (farfield_matrix, farfield_tangent, fourier_tangents,  # noqa: E402
                       rhs_tangent, shape_loss_dense, shape_loss_grad_dense)
