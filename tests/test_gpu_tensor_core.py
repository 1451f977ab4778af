"""Tensor-core complex GEMM (exact 8-bit digit planes, tcgen05) and the dense LU built on it,
against numpy's FP64 BLAS/LAPACK products.

The split-precision product keeps each entry within about 2^-53 * 2k * max|A_i.| * max|B_.j|
of the exact product (the bound of an FP64 GEMM); the tests hold it to that bound with a factor
of 4, on ragged sizes (tiles of 128 rows and 32 complex columns, K chunks of 64 complex
values), several K chunks, more tiles than SMs, rows and columns of very different scales, zero
rows and columns, and integer inputs whose product is exact."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

EPS = 2.0 ** -53


def rand_c(rng, shape):
    return rng.normal(size=shape) + 1j * rng.normal(size=shape)


def tc_product(A, B, C=None, alpha=1.0, beta=0.0):
    import torch
    from paper_2607_00790_gb300 import binding
    tA = torch.as_tensor(A, device="cuda")
    tB = torch.as_tensor(B, device="cuda")
    tC = None if C is None else torch.as_tensor(C, device="cuda")
    out = binding.wsbm_zgemm(tA, tB, tC, alpha=alpha, beta=beta)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def check_bound(got, ref, A, B, factor=4.0):
    k = A.shape[1]
    ra = np.maximum(np.abs(A.real), np.abs(A.imag)).max(axis=1)
    cb = np.maximum(np.abs(B.real), np.abs(B.imag)).max(axis=0)
    bound = factor * EPS * 2 * k * ra[:, None] * cb[None, :] + 4 * EPS * np.abs(ref)
    err = np.abs(got - ref)
    assert np.all(err <= bound), float((err / np.maximum(bound, 1e-300)).max())


@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (200, 70, 45), (129, 33, 64), (700, 300, 500),
                                   (2000, 1000, 96)])
def test_zgemm_matches_fp64_product(m, n, k):
    rng = np.random.default_rng(m + 7 * n + 31 * k)
    A = rand_c(rng, (m, k)) * 10.0 ** rng.uniform(-3, 3, size=(m, 1))
    B = rand_c(rng, (k, n)) * 10.0 ** rng.uniform(-3, 3, size=(1, n))
    got = tc_product(A, B)
    ref = A @ B
    check_bound(got, ref, A, B)
    assert np.linalg.norm(got - ref) <= 2e-15 * np.linalg.norm(ref)


def test_zgemm_alpha_beta_and_zero_lines():
    rng = np.random.default_rng(3)
    m, n, k = 300, 90, 130
    A = rand_c(rng, (m, k))
    B = rand_c(rng, (k, n))
    A[17] = 0.0
    B[:, 5] = 0.0
    C = rand_c(rng, (m, n))
    alpha, beta = 0.5 - 2.0j, -1.25 + 0.75j
    got = tc_product(A, B, C, alpha=alpha, beta=beta)
    ref = alpha * (A @ B) + beta * C
    ra = np.maximum(np.abs(A.real), np.abs(A.imag)).max(axis=1)
    cb = np.maximum(np.abs(B.real), np.abs(B.imag)).max(axis=0)
    bound = 8 * EPS * (2 * k * abs(alpha) * ra[:, None] * cb[None, :] + np.abs(ref) + np.abs(beta * C))
    assert np.all(np.abs(got - ref) <= bound)
    # a zero row of A or column of B leaves beta C (to the rounding of the complex multiply)
    assert np.allclose(got[17], beta * C[17], rtol=4 * EPS, atol=0)
    assert np.allclose(got[:, 5], beta * C[:, 5], rtol=4 * EPS, atol=0)


def test_zgemm_exact_on_integers():
    """Small integers: every digit product and sum is exact, so the result is the exact
    product, bit for bit."""
    rng = np.random.default_rng(5)
    m, n, k = 257, 65, 300
    A = rng.integers(-1000, 1000, size=(m, k)) + 1j * rng.integers(-1000, 1000, size=(m, k))
    B = rng.integers(-1000, 1000, size=(k, n)) + 1j * rng.integers(-1000, 1000, size=(k, n))
    got = tc_product(A.astype(np.complex128), B.astype(np.complex128))
    assert np.array_equal(got, (A @ B).astype(np.complex128))


def test_zgemm_rejects_bad_sizes():
    import torch
    from paper_2607_00790_gb300 import binding
    A = torch.zeros((4, 0), dtype=torch.complex128, device="cuda")
    B = torch.zeros((0, 4), dtype=torch.complex128, device="cuda")
    with pytest.raises(binding.WsbmError):
        binding.wsbm_zgemm(A, B)


@pytest.mark.parametrize("n", [300, 1000, 2100])
def test_lu_dense_factors_and_solves(n):
    """P A = L U to rounding, and the factors solve A x = b like LAPACK's."""
    import torch
    from paper_2607_00790_gb300 import binding
    rng = np.random.default_rng(n)
    A = rand_c(rng, (n, n)) + 5.0 * np.eye(n)
    LU, piv = binding.wsbm_lu_dense(torch.as_tensor(A, device="cuda"))
    torch.cuda.synchronize()
    LU = LU.cpu().numpy()
    piv = piv.cpu().numpy()
    L = np.tril(LU, -1) + np.eye(n)
    U = np.triu(LU)
    PA = A.copy()
    for j in range(n):
        p = piv[j]
        assert j <= p < n
        if p != j:
            PA[[j, p]] = PA[[p, j]]
    # pivot by max(|Re|, |Im|) to within 2^-20: |l| <= sqrt(2) (1 + 2^-20)
    assert np.abs(L).max() <= 1.4143, np.abs(L).max()
    res = np.linalg.norm(PA - L @ U) / np.linalg.norm(A)
    assert res < 50 * n * EPS, res
    b = rand_c(rng, (n, 3))
    Pb = b.copy()
    for j in range(n):
        if piv[j] != j:
            Pb[[j, piv[j]]] = Pb[[piv[j], j]]
    x = np.linalg.solve(U, np.linalg.solve(L, Pb))
    ref = np.linalg.solve(A, b)
    assert np.linalg.norm(x - ref) <= 1e-11 * np.linalg.norm(ref)


def test_zgemm_batched_items_of_different_sizes():
    """One launch over 37 products of different shapes (empty ones, ragged edges, k from 1 to
    200 padded to the largest, leading dimensions above the row counts): each C_i against
    numpy's FP64 product at the same bound."""
    import torch
    from paper_2607_00790_gb300 import binding
    rng = np.random.default_rng(11)
    As, Bs, Cs, refs, hostA, hostB = [], [], [], [], [], []
    for i in range(37):
        m = int(rng.integers(0, 300)) if i % 9 else 0
        n = int(rng.integers(1, 100)) if i % 11 else 0
        k = int(rng.integers(1, 200))
        A = rand_c(rng, (m, k)) * 10.0 ** rng.uniform(-2, 2, size=(m, 1))
        B = rand_c(rng, (k, n)) * 10.0 ** rng.uniform(-2, 2, size=(1, n))
        C0 = rand_c(rng, (m, n))
        lda, ldc = m + 3, m + 5
        tA = torch.zeros((k, lda), dtype=torch.complex128, device="cuda").T[:m]
        tA.copy_(torch.as_tensor(A))
        tB = torch.as_tensor(B, device="cuda").T.contiguous().T
        tC = torch.zeros((n, ldc), dtype=torch.complex128, device="cuda").T[:m]
        tC.copy_(torch.as_tensor(C0))
        As.append(tA)
        Bs.append(tB)
        Cs.append(tC)
        refs.append(C0 - A @ B)
        hostA.append(A)
        hostB.append(B)
    binding.wsbm_zgemm_batched(As, Bs, Cs, alpha=-1.0, beta=1.0)
    torch.cuda.synchronize()
    for i in range(37):
        got = Cs[i].cpu().numpy()
        if got.size == 0:
            continue
        A, B = hostA[i], hostB[i]
        k = A.shape[1]
        ra = np.maximum(np.abs(A.real), np.abs(A.imag)).max(axis=1)
        cb = np.maximum(np.abs(B.real), np.abs(B.imag)).max(axis=0)
        bound = 4 * EPS * 2 * k * ra[:, None] * cb[None, :] + 8 * EPS * np.abs(refs[i])
        assert np.all(np.abs(got - refs[i]) <= bound), i
