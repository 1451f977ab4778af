"""Parity of the device Hankel evaluator with the oracle at identical arguments."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

# Break points of the device evaluator (series / fitted intervals / asymptotic term counts).
BREAKS = [1.5, 2.0, 3.0, 4.0, 5.5, 8.0, 12.0, 20.0, 100.0, 1000.0]


def sample_z(seed=0):
    rng = np.random.default_rng(seed)
    z = np.exp(rng.uniform(np.log(1e-3), np.log(6e4), 4000))
    edges = []
    for b in BREAKS:
        edges += [np.nextafter(b, 0), b, np.nextafter(b, np.inf)]
    return np.concatenate([z, np.array(edges), np.linspace(0.05, 120.0, 2400)])


def device_hankel(z, precision):
    import torch
    from paper_2607_00790_gb300 import binding
    out = binding.wsbm_hankel01(torch.tensor(z, device="cuda"), precision).cpu().numpy()
    return out[:, 0] + 1j * out[:, 1], out[:, 2] + 1j * out[:, 3], out[:, 4] + 1j * out[:, 5]


def test_fp64_hankel_matches_oracle():
    from paper_2607_00790_gb300 import binding
    z = sample_z()
    h0, h1, f1 = device_hankel(z, binding.WSBM_FP64)
    r0, r1 = oracle.hankel01(z)
    rf = oracle.f1(z)
    tol = np.where(z < 1e3, 3e-15, np.where(z < 1e4, 2e-14, 1e-13))
    e0 = np.abs(h0 - r0) / np.abs(r0)
    e1 = np.abs(h1 - r1) / np.abs(r1)
    ef = np.abs(f1 - rf) / np.abs(rf)
    assert np.all(e0 <= tol), (z[np.argmax(e0 / tol)], e0.max())
    assert np.all(e1 <= tol), (z[np.argmax(e1 / tol)], e1.max())
    assert np.all(ef <= tol), (z[np.argmax(ef / tol)], ef.max())


def test_mixed_hankel_within_fp32_bound():
    from paper_2607_00790_gb300 import binding
    z = sample_z(1)
    h0, h1, _ = device_hankel(z, binding.WSBM_MIXED)
    r0, r1 = oracle.hankel01(z)
    e = np.maximum(np.abs(h0 - r0) / np.abs(r0), np.abs(h1 - r1) / np.abs(r1))
    assert e.max() < 1e-6, (z[np.argmax(e)], e.max())


def test_mixed_fine_hankel_within_fp32_table_bound():
    """Amplitude-only mixed evaluation: FP32 P - 1, Q (fits to 2.1e-8 absolute), everything else
    FP64; the series region (z < 1.5) is the FP64 evaluator unchanged."""
    from paper_2607_00790_gb300 import binding
    z = sample_z(3)
    h0, h1, f1 = device_hankel(z, binding.WSBM_MIXED_FINE)
    r0, r1 = oracle.hankel01(z)
    e = np.maximum(np.abs(h0 - r0) / np.abs(r0), np.abs(h1 - r1) / np.abs(r1))
    big = z >= 1.5
    assert e[big].max() < 5e-8, (z[big][np.argmax(e[big])], e[big].max())
    assert e[~big].max() < 3e-15
    rf = oracle.f1(z)
    ef = np.abs(f1 - rf) / np.abs(rf)
    assert ef[big].max() < 2e-7 and ef[~big].max() < 3e-15


def test_hankel_empty_and_deterministic():
    import torch
    from paper_2607_00790_gb300 import binding
    z = torch.tensor(sample_z(2)[:777], device="cuda")
    a = binding.wsbm_hankel01(z)
    b = binding.wsbm_hankel01(z)
    assert torch.equal(a, b)
    e = binding.wsbm_hankel01(torch.empty(0, dtype=torch.float64, device="cuda"))
    assert e.shape == (0, 6)
