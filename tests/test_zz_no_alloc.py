"""wsbm_entries_raw_noalloc: the allocation-free variant of wsbm_entries_raw, for callers that
cannot allocate device memory (their framework's allocator owns the GPU, a fixed memory
budget, or a path that must not pay for cudaMalloc/cudaFree).  It must give the same entries
as wsbm_entries_raw, call after call, although every call reuses one library-owned scratch
array.  This file is collected last so that a failure here stops a -x run only after every
other test has run."""
import ctypes

import numpy as np
import pytest

import oracle
from helpers import entry_scale
from paper_2607_00790_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-12


def noalloc_entries(g, p, rows, cols):
    import torch
    from paper_2607_00790_gb300 import binding
    lib = binding.lib()
    f = lib.wsbm_entries_raw_noalloc
    f.argtypes = [ctypes.POINTER(binding.Geom), ctypes.POINTER(binding.Params), ctypes.c_void_p,
                  ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    out = torch.empty((cols.numel(), rows.numel()), dtype=torch.complex128, device="cuda")
    rc = f(ctypes.byref(g), ctypes.byref(p), ctypes.c_void_p(rows.data_ptr()), rows.numel(),
           ctypes.c_void_p(cols.data_ptr()), cols.numel(), ctypes.c_void_p(out.data_ptr()),
           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, out.T


def test_noalloc_matches_allocating_entry_point_twice():
    import torch
    from paper_2607_00790_gb300 import binding
    c = inputs.star(2000)
    ph = oracle.Physics(inputs.k0_for_density(c), n=1.5)
    g, keep = binding.make_geom(c)
    p = binding.make_params(ph.k0, 1.5)
    rng = np.random.default_rng(21)
    cases = [(rng.choice(4000, 300, replace=False), rng.choice(4000, 177, replace=False)),
             (np.arange(1000, 1100), np.concatenate([np.arange(950, 1150), [3999, 0]]))]
    for rows, cols in cases:  # two calls in a row, different sizes, same scratch array
        r = torch.tensor(rows, device="cuda")
        cl = torch.tensor(cols, device="cuda")
        rc, got = noalloc_entries(g, p, r, cl)
        assert rc == 0
        ref = binding.wsbm_entries_raw(g, p, r, cl)
        torch.cuda.synchronize()
        got, ref = got.cpu().numpy(), ref.cpu().numpy()
        M = entry_scale(c, ph, rows, cols)
        assert (np.abs(got - ref) / M).max() <= TOL
        assert np.linalg.norm(got - ref) <= TOL * np.linalg.norm(ref)


def test_noalloc_rejects_oversized_request():
    import torch
    from paper_2607_00790_gb300 import binding
    c = inputs.disk(64)
    g, keep = binding.make_geom(c)
    p = binding.make_params(2.0, 1.5)
    big = torch.zeros(65536, dtype=torch.int64, device="cuda")
    one = torch.zeros(1, dtype=torch.int64, device="cuda")
    rc, _ = noalloc_entries(g, p, big, one)
    assert rc == -1


def test_noalloc_at_the_scratch_limit():
    """nr + nc equal to WSBM_NOALLOC_MAX_INDICES (65536), split unevenly (65000 rows, 536
    columns), fills the scratch array to its end: the row and column slot lists must not overlap
    and must match wsbm_entries_raw; one index more is refused with INVALID_ARG."""
    import torch
    from paper_2607_00790_gb300 import binding
    c = inputs.star(40000)
    ph = oracle.Physics(inputs.k0_for_density(c), n=1.5)
    g, keep = binding.make_geom(c)
    p = binding.make_params(ph.k0, 1.5)
    rng = np.random.default_rng(23)
    rows = torch.tensor(rng.choice(80000, 65000, replace=False), device="cuda")
    cols = torch.tensor(rng.choice(80000, 536, replace=False), device="cuda")
    for _ in range(2):
        rc, got = noalloc_entries(g, p, rows, cols)
        assert rc == 0
        ref = binding.wsbm_entries_raw(g, p, rows, cols)
        torch.cuda.synchronize()
        assert torch.linalg.norm(got - ref).item() <= TOL * torch.linalg.norm(ref).item()
        assert (got - ref).abs().max().item() <= TOL * ref.abs().max().item()
    rc, _ = noalloc_entries(g, p, rows, torch.cat([cols, cols[:1]]))
    assert rc == -1
