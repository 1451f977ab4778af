"""Thin ctypes binding of ``libwsbm_hss.so`` (declared in include/wsbm_hss.h).

Argument marshalling only: every computation runs in the library's CUDA kernels.  PyTorch
supplies device memory and the stream (the current torch stream of the tensors' device).
The binding refuses to run when the library is missing or a tensor is not on a CUDA device.
"""
from __future__ import annotations

import ctypes
import os

import torch

from .build import LIB as LIB_PATH

_LIB = None

WSBM_OK = 0
WSBM_FP64 = 0
WSBM_MIXED = 1
WSBM_MIXED_FINE = 2
ERRORS = {0: "ok", -1: "invalid argument", -2: "out of memory", -3: "CUDA error",
          -4: "rank overflow", -5: "timeout", -6: "not factored", -7: "no device"}


class WsbmError(RuntimeError):
    def __init__(self, code, where):
        super().__init__(f"{where}: {ERRORS.get(code, code)} ({code})")
        self.code = code


class Geom(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("x", ctypes.c_void_p), ("y", ctypes.c_void_p),
                ("nx", ctypes.c_void_p), ("ny", ctypes.c_void_p), ("w", ctypes.c_void_p),
                ("kappa", ctypes.c_void_p)]


class Params(ctypes.Structure):
    _fields_ = [("k0", ctypes.c_double), ("refr_index", ctypes.c_double),
                ("eps0", ctypes.c_double), ("eps1", ctypes.c_double),
                ("leaf", ctypes.c_int32), ("nproxy", ctypes.c_int32),
                ("id_tol", ctypes.c_double), ("precision", ctypes.c_int32),
                ("proxy_ratio", ctypes.c_double), ("max_levels", ctypes.c_int32),
                ("root_cap", ctypes.c_int32), ("id_method", ctypes.c_int32), ("formulation", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int32), ("nboxes_leaf", ctypes.c_int32),
                ("entries_generated", ctypes.c_int64), ("pairs_evaluated", ctypes.c_int64),
                ("ms_entries", ctypes.c_double), ("ms_id", ctypes.c_double),
                ("ms_factor", ctypes.c_double), ("ms_total_factor", ctypes.c_double),
                ("max_rank", ctypes.c_int32), ("root_size", ctypes.c_int32),
                ("rank_per_level", ctypes.c_int32 * 32), ("factor_bytes", ctypes.c_int64),
                ("entries_proxy", ctypes.c_int64), ("pairs_proxy", ctypes.c_int64),
                ("ms_proxy", ctypes.c_double), ("entries_pairs", ctypes.c_int64),
                ("pairs_pairs", ctypes.c_int64), ("ms_pairs", ctypes.c_double),
                ("launches", ctypes.c_int64), ("ms_cpqr", ctypes.c_double),
                ("cpqr_matrices", ctypes.c_int64), ("cpqr_flops", ctypes.c_double),
                ("sketch_matrices", ctypes.c_int64), ("sketch_fallbacks", ctypes.c_int64),
                ("ms_sketch", ctypes.c_double), ("ms_lu", ctypes.c_double),
                ("lu_flops", ctypes.c_double), ("lu_matrices", ctypes.c_int64),
                ("lu_tc_matrices", ctypes.c_int64)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "rank_per_level"}
        d["rank_per_level"] = list(self.rank_per_level)[: self.levels + 1]
        return d


def lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_2607_00790_gb300.build.build() first")
        L = ctypes.CDLL(LIB_PATH)
        vp, i64, i32, d = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
        L.wsbm_hankel01.argtypes = [vp, i64, vp, i32, vp]
        L.wsbm_entries_raw.argtypes = [ctypes.POINTER(Geom), ctypes.POINTER(Params), vp, i64, vp,
                                       i64, vp, vp]
        L.wsbm_proxy_block.argtypes = [ctypes.POINTER(Geom), ctypes.POINTER(Params), i32, vp, i64,
                                       d, d, d, i32, vp, vp]
        L.wsbm_create.argtypes = [ctypes.POINTER(Geom), ctypes.POINTER(Params), vp,
                                  ctypes.POINTER(vp)]
        L.wsbm_factor.argtypes = [vp]
        L.wsbm_rhs_planewave.argtypes = [vp, vp, i32, vp]
        L.wsbm_solve.argtypes = [vp, vp, i32, vp, vp]
        L.wsbm_farfield.argtypes = [vp, vp, vp, i32, vp, i32, vp]
        L.wsbm_entries.argtypes = [vp, vp, i64, vp, i64, vp]
        L.wsbm_box_info.argtypes = [vp, i32, i32, ctypes.POINTER(d), ctypes.POINTER(i64)]
        L.wsbm_stats.argtypes = [vp, ctypes.POINTER(Stats)]
        L.wsbm_box_skeletons.argtypes = [vp, i32, i32, vp, vp, i32, ctypes.POINTER(i32)]
        L.wsbm_box_skeletons.restype = ctypes.c_int
        L.wsbm_destroy.argtypes = [vp]
        L.wsbm_destroy.restype = None
        L.wsbm_batch_create.argtypes = [ctypes.POINTER(Geom), ctypes.POINTER(Params), i32, vp,
                                        ctypes.POINTER(vp)]
        L.wsbm_batch_factor.argtypes = [vp]
        L.wsbm_batch_handle.argtypes = [vp, i32, ctypes.POINTER(vp)]
        L.wsbm_batch_stats.argtypes = [vp, ctypes.POINTER(Stats)]
        L.wsbm_batch_solve.argtypes = [vp, ctypes.POINTER(vp), i32, ctypes.POINTER(vp),
                                       ctypes.POINTER(vp)]
        L.wsbm_batch_solve.restype = ctypes.c_int
        L.wsbm_batch_destroy.argtypes = [vp]
        L.wsbm_batch_destroy.restype = None
        G, P = ctypes.POINTER(Geom), ctypes.POINTER(Params)
        L.wsbm_solve_transposed.argtypes = [vp, vp, i32, vp, vp]
        L.wsbm_refine.argtypes = [vp, i32, vp, i32, vp, vp, i32, ctypes.POINTER(d)]
        L.wsbm_zgemm.argtypes = [i32, i32, i32, ctypes.POINTER(d), vp, i64, vp, i64,
                                 ctypes.POINTER(d), vp, i64, vp]
        L.wsbm_zgemm.restype = ctypes.c_int
        L.wsbm_zgemm_batched.argtypes = [i32, vp, ctypes.POINTER(d), ctypes.POINTER(d), vp]
        L.wsbm_zgemm_batched.restype = ctypes.c_int
        L.wsbm_lu_dense.argtypes = [vp, i64, i32, vp, vp]
        L.wsbm_lu_dense.restype = ctypes.c_int
        L.wsbm_autotune.argtypes = [i32, i32, i32, i32, vp, vp, vp]
        L.wsbm_autotune.restype = ctypes.c_int
        L.wsbm_autotune_build.argtypes = [ctypes.POINTER(Geom), ctypes.POINTER(Params), vp, vp, vp]
        L.wsbm_autotune_build.restype = ctypes.c_int
        L.wsbm_tuning.argtypes = [vp]
        L.wsbm_tuning.restype = ctypes.c_int
        L.wsbm_tuning_set.argtypes = [vp]
        L.wsbm_tuning_set.restype = ctypes.c_int
        L.wsbm_refine.restype = ctypes.c_int
        L.wsbm_matvec.argtypes = [G, P, i32, vp, i32, vp, vp]
        L.wsbm_matvec.restype = ctypes.c_int
        L.wsbm_field.argtypes = [G, P, vp, vp, i32, vp, vp, i64, vp, vp, vp]
        L.wsbm_sketch.argtypes = [vp, i64, i32, i32, i32, vp, i64, ctypes.c_uint32, vp]
        L.wsbm_sketch.restype = ctypes.c_int
        L.wsbm_field.restype = ctypes.c_int
        L.wsbm_entries_vjp.argtypes = [G, P, vp, vp, vp, vp, vp]
        L.wsbm_rhs_planewave_vjp.argtypes = [G, P, vp, i32, vp, vp, vp]
        L.wsbm_farfield_vjp.argtypes = [G, P, vp, vp, i32, vp, i32, vp, vp, vp, vp]
        L.wsbm_curve_fourier.argtypes = [i32, i64, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        L.wsbm_curve_fourier_vjp.argtypes = [i32, i64, vp, vp, vp, vp, vp]
        for f in ("wsbm_solve_transposed", "wsbm_entries_vjp", "wsbm_rhs_planewave_vjp",
                  "wsbm_farfield_vjp", "wsbm_curve_fourier", "wsbm_curve_fourier_vjp"):
            getattr(L, f).restype = ctypes.c_int
        L.wsbm_strerror.argtypes = [ctypes.c_int]
        L.wsbm_strerror.restype = ctypes.c_char_p
        L.wsbm_trim_memory.argtypes = []
        L.wsbm_trim_memory.restype = ctypes.c_int
        L.wsbm_set_allocator.argtypes = [_ALLOC_FN, _FREE_FN, ctypes.c_void_p]
        L.wsbm_set_allocator.restype = ctypes.c_int
        for f in ("wsbm_hankel01", "wsbm_entries_raw", "wsbm_proxy_block", "wsbm_create",
                  "wsbm_factor", "wsbm_rhs_planewave", "wsbm_solve", "wsbm_farfield",
                  "wsbm_entries", "wsbm_box_info", "wsbm_stats", "wsbm_batch_create",
                  "wsbm_batch_factor", "wsbm_batch_handle", "wsbm_batch_stats"):
            getattr(L, f).restype = ctypes.c_int
        _LIB = L
    return _LIB


def _check(rc, where):
    if rc != WSBM_OK:
        raise WsbmError(rc, where)


def _dev(t, dtype):
    if not isinstance(t, torch.Tensor) or t.device.type != "cuda":
        raise ValueError("expected a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"expected a contiguous {dtype} tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(device=None):
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def trim_memory():
    """Return the library's cached work-space memory to the device."""
    _check(lib().wsbm_trim_memory(), "wsbm_trim_memory")


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)
_TORCH_CB = None  # created once and never released: handles keep calling them until destroyed


def _torch_alloc(nbytes, stream, ctx):
    import torch
    try:
        return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
    except Exception:  # out of memory: the library reports WSBM_ERR_OOM
        return None


def _torch_free(ptr, stream, ctx):
    import torch
    torch.cuda.caching_allocator_delete(int(ptr))


def use_torch_allocator(enable=True):
    """Let PyTorch's caching allocator supply the factors and work space of the handles created
    from now on (enable=False: the library's own pool again)."""
    global _TORCH_CB
    if enable:
        if _TORCH_CB is None:
            _TORCH_CB = (_ALLOC_FN(_torch_alloc), _FREE_FN(_torch_free))
        _check(lib().wsbm_set_allocator(_TORCH_CB[0], _TORCH_CB[1], None), "wsbm_set_allocator")
    else:
        _check(lib().wsbm_set_allocator(_ALLOC_FN(), _FREE_FN(), None), "wsbm_set_allocator")


def make_geom(curve, device="cuda"):
    """Device copies of a curve's arrays (x, y, nx, ny, w, kappa) and the ABI struct."""
    t = {k: torch.as_tensor(curve[k], dtype=torch.float64).to(device).contiguous()
         for k in ("x", "y", "nx", "ny", "w", "kappa")}
    g = Geom(t["x"].numel(), *[t[k].data_ptr() for k in ("x", "y", "nx", "ny", "w", "kappa")])
    return g, t


WSBM_ID_SKETCH = 0
WSBM_ID_FULL = 1


WSBM_FORM_WSBM, WSBM_FORM_BM, WSBM_FORM_PMCHWT = 0, 1, 2


def make_params(k0, n, eps0=1.0, eps1=0.0, leaf=64, nproxy=64, id_tol=1e-10,
                precision=WSBM_FP64, proxy_ratio=1.5, max_levels=0, root_cap=0,
                id_method=WSBM_ID_SKETCH, formulation=WSBM_FORM_WSBM):
    return Params(k0, n, eps0, eps1, leaf, nproxy, id_tol, precision, proxy_ratio, max_levels,
                  root_cap, id_method, formulation)


# ---------------------------------------------------------------- stateless calls ----
def wsbm_hankel01(z, precision=WSBM_FP64):
    out = torch.empty((z.numel(), 6), dtype=torch.float64, device=z.device)
    _check(lib().wsbm_hankel01(_dev(z, torch.float64), z.numel(), _dev(out, torch.float64),
                               precision, _stream(z.device)), "wsbm_hankel01")
    return out


def wsbm_entries_raw(geom, params, rows, cols):
    dev = rows.device
    out = torch.empty((cols.numel(), rows.numel()), dtype=torch.complex128, device=dev)
    _check(lib().wsbm_entries_raw(ctypes.byref(geom), ctypes.byref(params), _dev(rows, torch.int64),
                                  rows.numel(), _dev(cols, torch.int64), cols.numel(),
                                  _dev(out, torch.complex128), _stream(dev)), "wsbm_entries_raw")
    return out.T


def wsbm_proxy_block(geom, params, side, idx, circle, P):
    dev = idx.device
    cx, cy, rho = circle
    shape = (2 * P, idx.numel()) if side == 0 else (idx.numel(), 2 * P)
    out = torch.empty(shape, dtype=torch.complex128, device=dev)
    _check(lib().wsbm_proxy_block(ctypes.byref(geom), ctypes.byref(params), side,
                                  _dev(idx, torch.int64), idx.numel(), cx, cy, rho, P,
                                  _dev(out, torch.complex128), _stream(dev)), "wsbm_proxy_block")
    return out.T


def wsbm_matvec(geom, params, x, trans=False):
    """y = A x, or A^T x with trans (dense, matrix-free); x: 2N x nrhs (or 2N) complex128,
    paper order."""
    dev = x.device
    one = x.dim() == 1
    xm = x.reshape(x.shape[0], -1)
    xc = xm.T.contiguous()
    y = torch.empty_like(xc)
    _check(lib().wsbm_matvec(ctypes.byref(geom), ctypes.byref(params), int(bool(trans)),
                             _dev(xc, torch.complex128), xc.shape[0], _dev(y, torch.complex128),
                             _stream(dev)), "wsbm_matvec")
    return y[0] if one else y.T


def wsbm_zgemm(A, B, C=None, alpha=1.0, beta=0.0):
    """C = beta C + alpha A B (complex128 device tensors) on the tensor cores (exact digits)."""
    m, k = A.shape
    n = B.shape[1]
    Af = A.T.contiguous()  # column-major storage: the transpose's rows
    Bf = B.T.contiguous()
    Cf = (C.T.contiguous() if C is not None
          else torch.zeros((n, m), dtype=torch.complex128, device=A.device))
    al = (ctypes.c_double * 2)(complex(alpha).real, complex(alpha).imag)
    be = (ctypes.c_double * 2)(complex(beta).real, complex(beta).imag)
    _check(lib().wsbm_zgemm(m, n, k, al, _dev(Af, torch.complex128), m, _dev(Bf, torch.complex128), k,
                            be, _dev(Cf, torch.complex128), m, _stream(A.device)), "wsbm_zgemm")
    return Cf.T


class GemmItem(ctypes.Structure):
    _fields_ = [("A", ctypes.c_void_p), ("lda", ctypes.c_int64), ("B", ctypes.c_void_p),
                ("ldb", ctypes.c_int64), ("C", ctypes.c_void_p), ("ldc", ctypes.c_int64),
                ("m", ctypes.c_int32), ("n", ctypes.c_int32), ("k", ctypes.c_int32),
                ("pad", ctypes.c_int32)]


def _ld(t):
    """Leading dimension of a column-major (stride-1 rows) tensor; a single column's stride is
    arbitrary in torch, so it counts as the row count."""
    if t.shape[1] <= 1:
        return max(int(t.shape[0]), 1)
    if t.shape[0] > 1 and t.stride(0) != 1:
        raise ValueError("expected column-major storage (stride 1 along the rows)")
    return int(t.stride(1))


def wsbm_zgemm_batched(As, Bs, Cs, alpha=1.0, beta=0.0):
    """C_i = beta C_i + alpha A_i B_i for lists of complex128 device tensors stored column-major
    (pass the transposes' storage: tensors whose .T is contiguous), in one tensor-core launch."""
    n = len(As)
    items = (GemmItem * n)()
    keep = []
    for i, (A, B, C) in enumerate(zip(As, Bs, Cs)):
        m, k = A.shape
        nn = B.shape[1]
        items[i] = GemmItem(A.data_ptr(), _ld(A), B.data_ptr(), _ld(B), C.data_ptr(), _ld(C), m, nn, k, 0)
        keep.append((A, B, C))
    al = (ctypes.c_double * 2)(complex(alpha).real, complex(alpha).imag)
    be = (ctypes.c_double * 2)(complex(beta).real, complex(beta).imag)
    _check(lib().wsbm_zgemm_batched(n, ctypes.cast(items, ctypes.c_void_p), al, be,
                                    _stream(As[0].device)), "wsbm_zgemm_batched")


def wsbm_lu_dense(A):
    """LU with partial pivoting of a square complex128 device matrix: returns (LU, piv) with LU
    column-major-equivalent (L unit lower, U upper) as a torch tensor and piv (int32)."""
    n = A.shape[0]
    Af = A.T.contiguous()
    piv = torch.empty(n, dtype=torch.int32, device=A.device)
    _check(lib().wsbm_lu_dense(_dev(Af, torch.complex128), n, n, _dev(piv, torch.int32),
                               _stream(A.device)), "wsbm_lu_dense")
    return Af.T, piv


TUNE_KEYS = ("tc_group", "box_nb", "root_nb_mid", "root_nb_large", "cpqr_cb")
TUNE_BUILD_KEYS = ("pair_tf", "pair_ctas", "proxy_tf", "proxy_ctas", "cpqr_threads")


def wsbm_autotune(n_box=256, nbox=512, nrhs_box=160, n_root=16384, device=None):
    """Time the candidate shapes of the tensor-core paths and of the warp QR on the current
    device and keep the fastest (see wsbm_autotune in the C header).  Returns (choices dict,
    candidate times in ms: raster groups 4/8/16, box panel widths 32/64, root panel widths
    128/256, QR columns per pass 2/4/8)."""
    out = (ctypes.c_int32 * 5)()
    ms = (ctypes.c_double * 10)()
    _check(lib().wsbm_autotune(n_box, nbox, nrhs_box, n_root, out, ms, _stream(device)), "wsbm_autotune")
    return dict(zip(TUNE_KEYS, list(out))), list(ms)


def wsbm_autotune_build(geom, params, device=None):
    """Time the entry-kernel tile shapes and grids and the QR block size on leaf-level builds of
    the given problem (see wsbm_autotune_build in the C header).  Returns (choices dict, times
    in ms: 9 pair-kernel and 9 proxy-kernel times over (tile width 16/32/64) x (8/16/32 CTAs
    per SM), then the ID-phase times for 128 / 256 QR threads)."""
    out = (ctypes.c_int32 * 5)()
    ms = (ctypes.c_double * 20)()
    _check(lib().wsbm_autotune_build(ctypes.byref(geom), ctypes.byref(params), out, ms, _stream(device)),
           "wsbm_autotune_build")
    return dict(zip(TUNE_BUILD_KEYS, list(out))), list(ms)


def wsbm_tuning():
    """The launch shapes in use on the current device, with "tuned" / "tuned_build" = True once
    the respective autotuner ran there, and "solve_tc_min" (the smallest root order whose solves
    with 4 or more right-hand sides use the tensor cores)."""
    out = (ctypes.c_int32 * 13)()
    _check(lib().wsbm_tuning(out), "wsbm_tuning")
    v = list(out)
    d = dict(zip(TUNE_KEYS + TUNE_BUILD_KEYS, v[:10]))
    d["tuned"] = bool(v[10])
    d["tuned_build"] = bool(v[11])
    d["solve_tc_min"] = v[12]
    return d


def wsbm_tuning_set(**shapes):
    """Set launch shapes of the current device without timing; keys as wsbm_tuning() returns
    them (the ones not given keep their current value)."""
    cur = wsbm_tuning()
    for k in shapes:
        if k not in cur:
            raise KeyError(k)
    cur.update(shapes)
    arr = (ctypes.c_int32 * 13)(*[int(cur[k]) for k in TUNE_KEYS + TUNE_BUILD_KEYS],
                                int(bool(cur["tuned"])), int(bool(cur["tuned_build"])),
                                int(cur["solve_tc_min"]))
    _check(lib().wsbm_tuning_set(arr), "wsbm_tuning_set")


def wsbm_sketch(A, l, seed=0):
    """Y = Omega A (l x n) for a complex128 matrix A (m x n), Omega Rademacher +-1."""
    dev = A.device
    Ac = A.T.contiguous()  # column-major storage of A
    m, n = A.shape
    Y = torch.empty((n, l), dtype=torch.complex128, device=dev)
    _check(lib().wsbm_sketch(_dev(Ac, torch.complex128), m, m, n, l, _dev(Y, torch.complex128), l,
                             seed, _stream(dev)), "wsbm_sketch")
    return Y.T


def field(geom, params, u, q, tx, ty):
    """Field at points (tx, ty) off the curve from densities u, q (N x nrhs complex128):
    scattered field outside, total field inside.  Returns (values nt x nrhs, inside bool)."""
    dev = u.device
    uc, qc = u.T.contiguous(), q.T.contiguous()
    nrhs = uc.shape[0]
    nt = tx.numel()
    out = torch.empty((nrhs, nt), dtype=torch.complex128, device=dev)
    inside = torch.empty(nt, dtype=torch.int8, device=dev)
    _check(lib().wsbm_field(ctypes.byref(geom), ctypes.byref(params), _dev(uc, torch.complex128),
                            _dev(qc, torch.complex128), nrhs, _dev(tx, torch.float64),
                            _dev(ty, torch.float64), nt, _dev(out, torch.complex128),
                            _dev(inside, torch.int8), _stream(dev)), "wsbm_field")
    return out.T, inside.bool()


# ------------------------------------------------------------------- gradients ----
def entries_vjp(geom, params, lam, x):
    """(Re(lam^T dA/ds x) for the six node arrays as a (6, N) tensor, [d/dk1, d/deps1]);
    lam, x: complex128 vectors of length 2N (paper order)."""
    dev = lam.device
    N = geom.n
    grad = torch.empty((6, N), dtype=torch.float64, device=dev)
    gphys = torch.empty(2, dtype=torch.float64, device=dev)
    _check(lib().wsbm_entries_vjp(ctypes.byref(geom), ctypes.byref(params),
                                  _dev(lam, torch.complex128), _dev(x, torch.complex128),
                                  _dev(grad, torch.float64), _dev(gphys, torch.float64),
                                  _stream(dev)), "wsbm_entries_vjp")
    return grad, gphys


def rhs_planewave_vjp(geom, params, angles, lam):
    """Re(sum_a lam_a^T db_a/ds) as (6, N); lam: 2N x nang complex128."""
    dev = lam.device
    lc = lam.T.contiguous()
    grad = torch.empty((6, geom.n), dtype=torch.float64, device=dev)
    _check(lib().wsbm_rhs_planewave_vjp(ctypes.byref(geom), ctypes.byref(params),
                                        _dev(angles, torch.float64), angles.numel(),
                                        _dev(lc, torch.complex128), _dev(grad, torch.float64),
                                        _stream(dev)), "wsbm_rhs_planewave_vjp")
    return grad


def farfield_vjp(geom, params, u, q, angles, gF):
    """(v = C^T conj(gF) as 2N x nrhs, explicit node gradient (6, N)); u, q: N x nrhs,
    gF: nang x nrhs (complex128)."""
    dev = u.device
    nrhs = u.shape[1]
    uc, qc, gc = u.T.contiguous(), q.T.contiguous(), gF.T.contiguous()
    v = torch.empty((nrhs, 2 * geom.n), dtype=torch.complex128, device=dev)
    grad = torch.empty((6, geom.n), dtype=torch.float64, device=dev)
    _check(lib().wsbm_farfield_vjp(ctypes.byref(geom), ctypes.byref(params),
                                   _dev(uc, torch.complex128), _dev(qc, torch.complex128), nrhs,
                                   _dev(angles, torch.float64), angles.numel(),
                                   _dev(gc, torch.complex128), _dev(v, torch.complex128),
                                   _dev(grad, torch.float64), _stream(dev)), "wsbm_farfield_vjp")
    return v.T, grad


def curve_fourier(a, b, N):
    """Node arrays (x, y, nx, ny, w, kappa) of r(t) = 1 + sum a_j cos jt + b_j sin jt."""
    dev = a.device
    out = torch.empty((6, N), dtype=torch.float64, device=dev)
    ptrs = [ctypes.c_void_p(out[k].data_ptr()) for k in range(6)]
    _check(lib().wsbm_curve_fourier(a.numel(), N, _dev(a, torch.float64), _dev(b, torch.float64),
                                    *ptrs, _stream(dev)), "wsbm_curve_fourier")
    return out


def curve_fourier_vjp(a, b, N, grad):
    """Coefficient gradient (a_1..a_M, b_1..b_M) from a (6, N) node gradient."""
    dev = a.device
    out = torch.empty(2 * a.numel(), dtype=torch.float64, device=dev)
    g = grad.contiguous()
    _check(lib().wsbm_curve_fourier_vjp(a.numel(), N, _dev(a, torch.float64),
                                        _dev(b, torch.float64), _dev(g, torch.float64),
                                        _dev(out, torch.float64), _stream(dev)),
           "wsbm_curve_fourier_vjp")
    return out


def geom_from_tensors(x, y, nx, ny, w, kappa):
    ts = [t.contiguous() for t in (x, y, nx, ny, w, kappa)]
    for t in ts:
        _dev(t, torch.float64)
    return Geom(ts[0].numel(), *[t.data_ptr() for t in ts]), ts


# --------------------------------------------------------------------- HSS handle ----
class Solver:
    """wsbm_create / wsbm_factor / wsbm_solve / wsbm_farfield on one handle."""

    def __init__(self, geom, params, device="cuda", _handle=None):
        self.device = torch.device(device)
        self.n = geom.n
        self.owned = _handle is None
        if _handle is not None:
            self.h = _handle
            return
        h = ctypes.c_void_p()
        _check(lib().wsbm_create(ctypes.byref(geom), ctypes.byref(params), _stream(self.device),
                                 ctypes.byref(h)), "wsbm_create")
        self.h = h

    def factor(self):
        _check(lib().wsbm_factor(self.h), "wsbm_factor")

    def rhs_planewave(self, angles):
        out = torch.empty((angles.numel(), 2 * self.n), dtype=torch.complex128, device=self.device)
        _check(lib().wsbm_rhs_planewave(self.h, _dev(angles, torch.float64), angles.numel(),
                                        _dev(out, torch.complex128)), "wsbm_rhs_planewave")
        return out.T

    def solve(self, rhs):
        rhs_c = rhs.T.contiguous() if not rhs.T.is_contiguous() else rhs.T
        nrhs = rhs.shape[1]
        u = torch.empty((nrhs, self.n), dtype=torch.complex128, device=self.device)
        q = torch.empty((nrhs, self.n), dtype=torch.complex128, device=self.device)
        _check(lib().wsbm_solve(self.h, _dev(rhs_c, torch.complex128), nrhs,
                                _dev(u, torch.complex128), _dev(q, torch.complex128)), "wsbm_solve")
        return u.T, q.T

    def solve_transposed(self, v):
        """A^T lam = v (v: 2N x nrhs indexed like the unknowns); returns the multipliers of
        the first and second equations, N x nrhs each."""
        vc = v.T.contiguous()
        nrhs = v.shape[1]
        l1 = torch.empty((nrhs, self.n), dtype=torch.complex128, device=self.device)
        l2 = torch.empty((nrhs, self.n), dtype=torch.complex128, device=self.device)
        _check(lib().wsbm_solve_transposed(self.h, _dev(vc, torch.complex128), nrhs,
                                           _dev(l1, torch.complex128), _dev(l2, torch.complex128)),
               "wsbm_solve_transposed")
        return l1.T, l2.T

    def refine(self, geom, params, rhs, u, q, iters=3, trans=False):
        """wsbm_refine: iterative refinement against the dense matrix-free product (with trans:
        the adjoint system A^T lam = b, lam = (u, q) the multipliers of the two equations).
        geom and params are the handle's (kept for the callers' convenience).  Returns
        (u, q, relative residual before each step and after the last)."""
        rc_ = rhs.T.contiguous()
        nrhs = rhs.shape[1]
        uc = u.T.contiguous().clone()  # refined in place: never the caller's storage
        qc = q.T.contiguous().clone()
        res = (ctypes.c_double * (iters + 1))()
        _check(lib().wsbm_refine(self.h, 1 if trans else 0, _dev(rc_, torch.complex128), nrhs,
                                 _dev(uc, torch.complex128), _dev(qc, torch.complex128), iters, res),
               "wsbm_refine")
        return uc.T, qc.T, list(res)

    def farfield(self, u, q, angles):
        uc, qc = u.T.contiguous(), q.T.contiguous()
        nrhs = u.shape[1]
        out = torch.empty((nrhs, angles.numel()), dtype=torch.complex128, device=self.device)
        _check(lib().wsbm_farfield(self.h, _dev(uc, torch.complex128), _dev(qc, torch.complex128),
                                   nrhs, _dev(angles, torch.float64), angles.numel(),
                                   _dev(out, torch.complex128)), "wsbm_farfield")
        return out.T

    def entries(self, rows, cols):
        out = torch.empty((cols.numel(), rows.numel()), dtype=torch.complex128, device=self.device)
        _check(lib().wsbm_entries(self.h, _dev(rows, torch.int64), rows.numel(),
                                  _dev(cols, torch.int64), cols.numel(),
                                  _dev(out, torch.complex128)), "wsbm_entries")
        return out.T

    def box_info(self, level, box):
        out = (ctypes.c_double * 4)()
        rng = (ctypes.c_int64 * 2)()
        _check(lib().wsbm_box_info(self.h, level, box, out, rng), "wsbm_box_info")
        return tuple(out), tuple(rng)

    def stats(self):
        s = Stats()
        _check(lib().wsbm_stats(self.h, ctypes.byref(s)), "wsbm_stats")
        return s.as_dict()

    def skeletons(self, level, box, cap=4096):
        """Row and column skeleton indices (paper order) of a compressed box."""
        import numpy as np
        jr = np.empty(cap, dtype=np.int64)
        jc = np.empty(cap, dtype=np.int64)
        k = ctypes.c_int32()
        _check(lib().wsbm_box_skeletons(self.h, level, box, ctypes.c_void_p(jr.ctypes.data),
                                        ctypes.c_void_p(jc.ctypes.data), cap, ctypes.byref(k)),
               "wsbm_box_skeletons")
        return jr[: k.value].copy(), jc[: k.value].copy()

    def close(self):
        if self.h and self.owned:
            lib().wsbm_destroy(self.h)
        self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """wsbm_batch_*: many curves built and factored with shared launches per tree level."""

    def __init__(self, geoms, params, device="cuda"):
        self.device = torch.device(device)
        n = len(geoms)
        G = (Geom * n)(*geoms)
        P = (Params * n)(*params)
        h = ctypes.c_void_p()
        _check(lib().wsbm_batch_create(G, P, n, _stream(self.device), ctypes.byref(h)),
               "wsbm_batch_create")
        self.h = h
        self.sizes = [g.n for g in geoms]

    def factor(self):
        _check(lib().wsbm_batch_factor(self.h), "wsbm_batch_factor")

    def solver(self, i):
        hh = ctypes.c_void_p()
        _check(lib().wsbm_batch_handle(self.h, i, ctypes.byref(hh)), "wsbm_batch_handle")
        g = Geom(self.sizes[i])
        return Solver(g, None, self.device, _handle=hh)

    def stats(self):
        s = Stats()
        _check(lib().wsbm_batch_stats(self.h, ctypes.byref(s)), "wsbm_batch_stats")
        return s.as_dict()

    def solve(self, rhs_list):
        """Solve every curve at once; rhs_list[i]: 2N_i x nrhs complex128.  Returns [(u, q)]."""
        n = len(self.sizes)
        nrhs = rhs_list[0].shape[1]
        rc = [r.T.contiguous() for r in rhs_list]
        us = [torch.empty((nrhs, N), dtype=torch.complex128, device=self.device) for N in self.sizes]
        qs = [torch.empty((nrhs, N), dtype=torch.complex128, device=self.device) for N in self.sizes]
        arr = lambda ts: (ctypes.c_void_p * n)(*[t.data_ptr() for t in ts])
        _check(lib().wsbm_batch_solve(self.h, arr(rc), nrhs, arr(us), arr(qs)), "wsbm_batch_solve")
        return [(u.T, q.T) for u, q in zip(us, qs)]

    def close(self):
        if self.h:
            lib().wsbm_batch_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
