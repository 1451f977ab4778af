"""Tensor-core row sketch Y = Omega A: against numpy's Omega @ A with the same Rademacher
matrix (the counter-based hash written out below), on a tall ID-shaped matrix and on ragged
shapes; the error must stay within 4 m 2^-53 of each column's scale (the 56-bit digits of A,
exact products and sums, and numpy's own FP64 sum)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

M32 = np.uint64(0xFFFFFFFF)


def omega(l, m, seed):
    r = np.arange(l, dtype=np.uint64)[:, None]
    c = np.arange(m, dtype=np.uint64)[None, :]
    h = ((r * np.uint64(0x9E3779B1)) & M32) ^ ((c * np.uint64(0x85EBCA77) + np.uint64(seed)) & M32)
    h ^= h >> np.uint64(16)
    h = (h * np.uint64(0x7FEB352D)) & M32
    h ^= h >> np.uint64(15)
    h = (h * np.uint64(0x846CA68B)) & M32
    h ^= h >> np.uint64(16)
    return np.where(h & np.uint64(1), -1.0, 1.0)


@pytest.mark.parametrize("m,n,l,seed", [(382, 256, 160, 0), (37, 13, 16, 7), (1000, 9, 48, 3), (500, 40, 192, 9),
                                        (16, 8, 16, 1)])
def test_sketch_matches_numpy(m, n, l, seed):
    import torch
    from paper_2607_00790_gb300 import binding
    rng = np.random.default_rng(m + n)
    A = rng.normal(size=(m, n)) + 1j * rng.normal(size=(m, n))
    A[:, 0] *= 1e-7  # columns of very different scales
    if n > 3:
        A[:, 3] *= 1e5
    Y = binding.wsbm_sketch(torch.as_tensor(A, device="cuda"), l, seed).cpu().numpy()
    ref = omega(l, m, seed) @ A
    colmax = np.maximum(np.abs(A.real).max(axis=0), np.abs(A.imag).max(axis=0))
    err = np.abs(Y - ref).max(axis=0)
    assert np.all(err <= 4 * m * 2.0 ** -53 * colmax), (err / colmax).max()
