"""Plant plausible mistakes in a private copy of the oracle and show a pin catches each.

Each mutant is compiled from ``oracle/wsbm_oracle.cpp`` with one textual change; the
committed oracle is never modified.
"""
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from oracle.build import HERE

from test_oracle_physics import mie_errors, symbol_errors
from test_oracle_proxy import row_and_col_residuals

MUTANTS = {
    # D kernel differentiates the wrong point (transposed operand)
    "d_kernel_wrong_normal": ("cplx Dy0 = 0.25 * I1 * p.k0 * ha.h1 * (dny / r);",
                              "cplx Dy0 = 0.25 * I1 * p.k0 * ha.h1 * (dnx / r);"),
    # one-point log correction dropped from S
    "no_log_correction": ("(EULER_GAMMA + std::log(k * wi / (4.0 * PI))) / (2.0 * PI)",
                          "(EULER_GAMMA + std::log(k / 2.0)) / (2.0 * PI)"),
    # curvature limit of D, D* dropped
    "no_curvature_term": ("double Dd = -wi * kap / (4.0 * PI);", "double Dd = 0.0;"),
    # wrong sign of the Burton-Miller coupling constant in the off-diagonal entries
    "alpha_sign": ("cplx alpha = I1 / p.k0;\n  double wj", "cplx alpha = -I1 / p.k0;\n  double wj"),
    # wavenumbers swapped in the N_k0 - N_k1 difference
    "dN_swapped": ("(q0 * ha.f1 - q1 * hb.f1)", "(q0 * hb.f1 - q1 * ha.f1)"),
    # sign error in the proxy row block
    "proxy_row_sign": ("out[1][0] = pw * (-alpha * dphi[0]);", "out[1][0] = pw * (alpha * dphi[0]);"),
    # one-point correction of the hypersingular part of N_k dropped (eqs. bm, pmchwt)
    "no_hypersingular_correction": (" - PI / (6.0 * wi);", ";"),
    # sign error in the proxy column block
    "proxy_col_sign": ("out[s][1] = -eps * wj * (0.25 * I1 * h.h0);",
                       "out[s][1] = eps * wj * (0.25 * I1 * h.h0);"),
}


def build_mutant(name, tmpdir):
    old, new = MUTANTS[name]
    src = open(os.path.join(HERE, "wsbm_oracle.cpp")).read()
    assert src.count(old) == 1, name
    path = os.path.join(tmpdir, f"{name}.cpp")
    open(path, "w").write(src.replace(old, new))
    so = os.path.join(tmpdir, f"lib{name}.so")
    subprocess.run(["g++", "-std=c++17", "-O1", "-fPIC", "-shared", "-fopenmp",
                    "-ffp-contract=off", "-o", so, path], check=True)
    return so


def form_pin_ok():
    """Standard BM on the disk (N = 256): first-order accurate against the Mie series."""
    from paper_2607_00790_gb300 import inputs
    c, prm = inputs.workload("disk", N=256)
    ph = oracle.Physics(prm["k0"], n=prm["n"])
    x = oracle.dense_solve(oracle.form_dense(c, ph, oracle.FORM_BM), oracle.form_rhs(c, ph, [0.0], 1))
    th = np.arctan2(np.asarray(c["y"]), np.asarray(c["x"]))
    ue, _ = oracle.mie_boundary(1.0, ph, th)
    return np.linalg.norm(x[:256, 0].real - ue.real) / np.linalg.norm(ue.real) < 0.03


def pins_pass():
    ph = oracle.Physics(2 * np.pi, n=1.5)
    e128 = symbol_errors(ph, 1.3, 3, 128)
    e256 = symbol_errors(ph, 1.3, 3, 256)
    sym_ok = np.all(e256 < 2e-4) and np.all(e128 / e256 > 6.5)
    mie_ok = mie_errors(256, ph)[0] < 1e-4
    r1, r2 = row_and_col_residuals()
    return sym_ok and mie_ok and r1 < 1e-9 and r2 < 1e-9 and form_pin_ok()


def test_pins_pass_on_committed_oracle():
    assert pins_pass()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name):
    with tempfile.TemporaryDirectory() as d:
        so = build_mutant(name, d)
        with oracle.use_library(so):
            assert not pins_pass(), f"mutant {name} passed every pin"
