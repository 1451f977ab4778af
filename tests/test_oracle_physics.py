"""Pins for the oracle's WSBM Nystrom system (eq. weakly_bm, one-point corrected diagonal).

* On a circle every block of the system is diagonalised by e^{im theta}; the discrete
  operator must reproduce the closed-form symbol with an O(h^3) error (the paper's claim).
* The dense solve must reproduce the Mie series for a disk with slope ~3 (Sec. IV,
  Fig. error_circle: WSBM converges at O(h^3) in the relative 2-norm error of Re(u)).
* The far field must match the Mie far field.
"""
import numpy as np
import pytest

import oracle
from paper_2607_00790_gb300 import inputs


def wsbm_symbol(ph, R, m):
    S0, D0, N0 = oracle.circle_eigenvalues(ph.k0, R, m)
    S1, D1, N1 = oracle.circle_eigenvalues(ph.k1, R, m)
    al, e0, e1 = ph.alpha, ph.eps0, ph.eps1
    return np.array([[D1 + 0.5, -e1 * S1],
                     [D0 - 0.5 + al * (N0 - N1), -e0 * S0 - al * (e0 * D0 - e1 * D1) - al * (e0 + e1) / 2]])


def symbol_errors(ph, R, m, N):
    c = inputs.disk(N, R)
    A = oracle.wsbm_dense(c, ph)
    e = np.exp(1j * m * c["t"])
    sym = wsbm_symbol(ph, R, m)
    err = np.zeros((2, 2))
    for b in range(2):
        v = np.zeros(2 * N, complex)
        v[b * N:(b + 1) * N] = e
        y = A @ v
        for a in range(2):
            err[a, b] = np.max(np.abs(y[a * N:(a + 1) * N] - sym[a, b] * e)) / abs(sym[a, b])
    return err


@pytest.mark.parametrize("m", [0, 3, 7])
def test_circle_symbol_third_order(m):
    ph = oracle.Physics(2 * np.pi, n=1.5)
    e64 = symbol_errors(ph, 1.3, m, 64)
    e128 = symbol_errors(ph, 1.3, m, 128)
    e256 = symbol_errors(ph, 1.3, m, 256)
    assert np.all(e256 < 2e-4)
    # third order: the error drops ~8x per halving of h in every block
    assert np.all(e64 / e128 > 6.5) and np.all(e128 / e256 > 6.5), (e64, e128, e256)


def test_circle_symbol_paper_table():
    # Table para: eps0 = 1, eps1 = 5, omega = 10 (k0 = 10, k1 = 10 sqrt 5)
    ph = oracle.Physics(10.0, eps0=1.0, eps1=5.0)
    e128 = symbol_errors(ph, 1.0, 2, 128)
    e256 = symbol_errors(ph, 1.0, 2, 256)
    assert np.all(e128 / e256 > 6.0), (e128, e256)


def mie_errors(N, ph, R=1.0):
    c = inputs.disk(N, R)
    A = oracle.wsbm_dense(c, ph)
    b = oracle.rhs_planewave(c, ph, [0.0])
    u, q = oracle.split_uq(oracle.dense_solve(A, b))
    ue, qe = oracle.mie_boundary(R, ph, c["t"])
    ang = 2 * np.pi * np.arange(360) / 360
    ff = oracle.farfield(c, ph, u, q, ang)[:, 0]
    ffe = oracle.mie_farfield(R, ph, ang)
    return (np.linalg.norm(u[:, 0].real - ue.real) / np.linalg.norm(ue.real),
            np.linalg.norm(q[:, 0] - qe) / np.linalg.norm(qe),
            np.linalg.norm(ff - ffe) / np.linalg.norm(ffe))


def test_mie_disk_third_order():
    ph = oracle.Physics(2 * np.pi, n=1.5)
    errs = [mie_errors(N, ph) for N in (64, 128, 256, 512)]
    eu = np.array([e[0] for e in errs])
    slopes = np.log2(eu[:-1] / eu[1:])
    assert np.all(slopes > 2.9), slopes
    assert abs(slopes[-1] - 3.0) < 0.1
    assert eu[2] < 1e-4 and errs[2][1] < 3e-5 and errs[2][2] < 1e-4


def test_mie_paper_table_parameters():
    ph = oracle.Physics(10.0, eps0=1.0, eps1=5.0)
    e1 = mie_errors(256, ph)[0]
    e2 = mie_errors(512, ph)[0]
    assert np.log2(e1 / e2) > 2.8, (e1, e2)


def test_one_point_log_correction_constant():
    # The one-point rule  h sum_{j != 0} ln|jh| f(jh) + h ln(h/2pi) f(0)  integrates
    # ln|x| e^{-x^2} to O(h^3); exact value -(sqrt(pi)/2)(gamma + 2 ln 2).
    exact = -(np.sqrt(np.pi) / 2) * (oracle.EULER_GAMMA + 2 * np.log(2))
    errs = []
    for h in (0.4, 0.2, 0.1, 0.05):
        j = np.arange(1, int(12 / h))
        x = j * h
        approx = 2 * h * np.sum(np.log(x) * np.exp(-x * x)) + h * np.log(h / (2 * np.pi))
        errs.append(abs(approx - exact))
    errs = np.array(errs)
    assert np.all(np.log2(errs[:-1] / errs[1:]) > 2.8), errs


def test_entries_gather_matches_dense():
    c = inputs.star(96)
    ph = oracle.Physics(7.0, n=1.5)
    A = oracle.wsbm_dense(c, ph)
    rng = np.random.default_rng(3)
    rows = rng.integers(0, 192, 40)
    cols = rng.integers(0, 192, 33)
    assert np.array_equal(oracle.wsbm_entries(c, ph, rows, cols), A[np.ix_(rows, cols)])


def test_matvec_matches_dense():
    c = inputs.star(80)
    ph = oracle.Physics(5.0, n=1.3)
    A = oracle.wsbm_dense(c, ph)
    rng = np.random.default_rng(4)
    x = rng.normal(size=(160, 3)) + 1j * rng.normal(size=(160, 3))
    assert np.allclose(oracle.wsbm_matvec(c, ph, x), A @ x, rtol=1e-13, atol=1e-13)
