// Descriptors and host entry points of the batched dense complex128 kernels (dense.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#define WSBM_NB 32  // panel / block width of the blocked LU and triangular solves

// Kernel-launch counter of the library (every launch site calls wsbm_count_launch()).
void wsbm_count_launch();
void wsbm_count_launches(int64_t n);  // launches replayed from a captured CUDA graph
int64_t wsbm_launch_count();
// Stream-ordered allocation from the library's memory pool of device dev (see capi.cu).
cudaError_t wsbm_malloc_async(void** p, size_t bytes, int dev, cudaStream_t st);
// Number of SMs of the current device (cached per device, thread safe).
int wsbm_sm_count();
// Opt a kernel in to `bytes` of dynamic shared memory on the current device (remembered per
// device and kernel, thread safe).  Returns cudaSuccess or the error of the attribute call.
cudaError_t wsbm_smem_optin(const void* kernel, size_t bytes);

// autotune.cu: launch shapes, per device (defaults until an autotune call or wsbm_tuning_set):
// rows per raster group of the GEMM's tile order, panel width of the batched box LU (<= 64),
// outer panel width of the root LU below and from wsbm_lu_big_large_n() unknowns (128 or 256);
// tile width (16, 32, 64) and CTAs per SM of the node-pair and proxy entry kernels; threads per
// CTA of the thread-per-column QR (128 or 256) and columns per warp pass of the warp QR (2, 4
// or 8); the smallest root order whose solves with many right-hand sides use the tensor cores.
struct WsbmTune {
  int tc_group, box_nb, root_nb_mid, root_nb_large, tuned;
  int pair_tf, pair_ctas, proxy_tf, proxy_ctas, cpqr_threads, cpqr_cb, tuned_build;
  int solve_tc_min;
};
WsbmTune wsbm_tune_current();

// tc_gemm.cu: C (m x n) = beta C + alpha A (m x k) B (k x n), complex128 column-major, on the
// tensor cores from exact 8-bit digit planes (FP64-level accuracy).  ws: 256-byte aligned
// device work space of wsbm_zgemm_tc_ws_bytes(m, n, k) bytes.  1 <= k <= 32768.  Returns 0,
// -1 (bad arguments) or -3 (launch / tensor-map error); enqueues only.
int wsbm_zgemm_tc(int m, int n, int k, double2 alpha, const double2* A, int64_t lda, const double2* B,
                  int64_t ldb, double2 beta, double2* C, int64_t ldc, void* ws, cudaStream_t st);
size_t wsbm_zgemm_tc_ws_bytes(int m, int n, int k);
// Many products in one launch: C_i = beta C_i + alpha A_i B_i (sizes per item; K padded with
// zeros to the largest k).  ws: 256-byte aligned, wsbm_zgemm_tc_batched_ws_bytes(p, n) bytes.
// At most 65535 items.  Returns 0, -1 or -3; enqueues only (the item table is copied to ws).
struct TcProduct {
  const double2* A;
  int64_t lda;
  const double2* B;
  int64_t ldb;
  double2* C;
  int64_t ldc;
  int m, n, k, pad;
};
int wsbm_zgemm_tc_batched(const TcProduct* p, int nitems, double2 alpha, double2 beta, void* ws,
                          cudaStream_t st);
size_t wsbm_zgemm_tc_batched_ws_bytes(const TcProduct* p, int nitems);
// The same with an explicit raster group (rows of tiles per group, 1..64).
int wsbm_zgemm_tc_batched_g(const TcProduct* p, int nitems, double2 alpha, double2 beta, void* ws,
                            cudaStream_t st, int group);
// The same split into a host-side plan (item tables and work-space layout, built once) and a
// launch sequence that reads the item tables from a device copy of `tab` made by the caller:
// no host memory is read at launch, so the launches can be captured into a CUDA graph.
// ws: 256-byte aligned, ws_bytes (the item-table region at off_tab is not used by _run).
struct TcPlan {
  int nitems = 0, tiles = 0, kmax = 0, maxm = 0, maxn = 0;
  int64_t ra = 0, rb = 0;
  size_t off_exp = 0, off_tab = 0, ws_bytes = 0;
  std::vector<unsigned char> tab;
};
int wsbm_zgemm_tc_plan(const TcProduct* p, int nitems, TcPlan* out);
int wsbm_zgemm_tc_run(const TcPlan& pl, const void* dtab, double2 alpha, double2 beta, void* ws,
                      cudaStream_t st, int group);
// Randomized row sketches Y_i = Omega[:m_i, :k_i] B_i on the tensor cores (Omega: +-1 from the
// sketch hash of (row, column, seed), shared by all items; B_i: k_i x n_i complex, C_i = Y_i:
// m_i x n_i, A ignored).  ws: 256-byte aligned, wsbm_sketch_tc_ws_bytes(p, n) bytes.  At most
// 65535 items, k_i <= 65536.  Returns 0, -1 or -3; enqueues only.
size_t wsbm_sketch_tc_ws_bytes(const TcProduct* p, int nitems);
int wsbm_sketch_tc(const TcProduct* p, int nitems, uint32_t seed, void* ws, cudaStream_t st);
// Synchronizes the stream and returns -5 (and clears the flag) if a bounded wait of the GEMM
// kernel ran out since the last call, else 0 (-3 on a CUDA error).
int wsbm_zgemm_tc_status(cudaStream_t st);

// C = alpha * op(A) * B + beta * C  (column-major, op(A) m x k, B k x n, C m x n);
// op(A) = A (ta = 0, A stored m x k) or A^T (ta = 1, A stored k x m).
struct GemmDesc {
  const double2* A;
  const double2* B;
  double2* C;
  int64_t lda, ldb, ldc;
  int32_t m, n, k, ta;
  double2 alpha, beta;
};

// In-place LU with partial pivoting of an n x n matrix; piv[j] = row swapped with row j.
struct LuDesc {
  double2* A;
  int64_t lda;
  int32_t* piv;
  int32_t n, pad;
};

// B (n x nrhs) <- op(T)^-1 B with T n x n holding an LU factor (unit lower L below the
// diagonal, non-unit upper U on and above it); piv: the LU row interchanges.  trans = 0 solves
// with L (forward) and U (backward); trans = 1 with U^T (forward) and L^T (backward).
struct TrsmDesc {
  const double2* T;
  int64_t ldt;
  double2* B;
  int64_t ldb;
  const int32_t* piv;
  int32_t n, nrhs;
  int32_t trans, pad;
};

// Column-pivoted QR state of an m x n matrix.  state[0] = next step (0 for a fresh matrix),
// state[1] = rank reached; perm[t] = original column at position t; norm2 = remaining squared
// column norms; tauv, betav = reflector scalars and R diagonal; rdiag0 = |R_00|.
struct QrDesc {
  double2* A;
  int64_t lda;
  int32_t m, n;
  int32_t kt;  // mode 1 target rank
  int32_t pad;
  double tol;
  int32_t* perm;
  int32_t* state;
  double* norm2;
  double* nref;  // remaining squared norm at its last exact computation
  double* tauv;
  double2* betav;
  double* rdiag0;
};

// Fused LU with partial pivoting and solve of [A | B]: A (n x n, column-major, in place) <- its
// LU factor (the LuDesc layout, piv[j] = row swapped with row j), B (n x nrhs) <- A^-1 B.
// S: scratch of n x wsbm_lu_solve_ldr(n, nrhs) elements (the row-major working copy).
struct LuSolveDesc {
  double2* A;
  int64_t lda;
  int32_t* piv;
  double2* B;
  int64_t ldb;
  double2* S;
  int32_t n, nrhs;
};
#define WSBM_LUS_MAXN 1024  // largest n of the fused kernel (its panel sits in shared memory)
int64_t wsbm_lu_solve_ldr(int n, int nrhs);
// Returns -1 (nothing launched) when max_n exceeds WSBM_LUS_MAXN.
int wsbm_lu_solve_fused_batched(const LuSolveDesc* d_desc, int nbatch, int max_n, int max_nc,
                                cudaStream_t st);
// The same factorization and solve with the products on the tensor cores (tc_gemm.cu):
// h: host copy of the descriptors (S unused), d: device copy, d_lu: device LuDesc {A, lda, piv, n}
// per item.  ws: 256-byte aligned, wsbm_lu_solve_tc_ws_bytes(h, nbatch) bytes.  Enqueues only.
int wsbm_lu_solve_tc_batched(const LuSolveDesc* h, const LuSolveDesc* d, int nbatch, const LuDesc* d_lu,
                             void* ws, cudaStream_t st);
// The same with an explicit panel width nb (8 <= nb <= 64, a multiple of 8).
int wsbm_lu_solve_tc_batched_nb(const LuSolveDesc* h, const LuSolveDesc* d, int nbatch, const LuDesc* d_lu,
                                void* ws, cudaStream_t st, int nb);
size_t wsbm_lu_solve_tc_ws_bytes(const LuSolveDesc* h, int nbatch);

// Inverses of the nb x nb diagonal blocks (nb <= 256, per item) of LU factors A (n x n, unit
// lower L and upper U): block p of L into Linv + p nb^2, of U into Uinv + p nb^2 (leading
// dimension nb).  max_blocks: the largest ceil(n / nb), max_nb the largest nb of the batch.
// Enqueues only; returns 0, -1 or -3.
struct DinvDesc {
  const double2* A;
  int64_t lda;
  double2* Linv;
  double2* Uinv;
  int32_t n, nb;
};
int wsbm_lu_dinv_batched(const DinvDesc* d_desc, int nitems, int max_blocks, int max_nb, cudaStream_t st);
// The row permutation of LU row interchanges: perm (device int32 n) with (P b)[r] = b[perm[r]].
struct PermDesc {
  const int32_t* piv;
  int32_t* perm;
  int32_t n, pad;
};
int wsbm_piv_perm_batched(const PermDesc* d_desc, int nitems, cudaStream_t st);

int wsbm_gemm_batched(const GemmDesc* d_desc, int nbatch, int max_m, int max_n, cudaStream_t st);
int wsbm_lu_batched(const LuDesc* d_desc, int nbatch, int max_n, int* d_info, cudaStream_t st);
// LU with partial pivoting of one large n x n matrix (same factor layout and piv as
// wsbm_lu_batched), trailing updates on the tensor cores.  ws: 256-byte aligned device work
// space of wsbm_lu_big_ws_bytes(n) bytes; d_info (device int, may be NULL) receives j + 1 when
// pivot j is exactly zero.  Enqueues only; returns 0, -1 or -3.
int wsbm_lu_big(double2* A, int64_t lda, int n, int* piv, int* d_info, void* ws, cudaStream_t st);
// The same with an explicit outer panel width nb (128 or 256).
int wsbm_lu_big_nb(double2* A, int64_t lda, int n, int* piv, int* d_info, void* ws, cudaStream_t st, int nb);
int wsbm_lu_big_large_n();  // n from which the root LU takes the large-class panel width
size_t wsbm_lu_big_ws_bytes(int n);
int wsbm_trsm_batched(const TrsmDesc* d_desc, int nbatch, int max_n, int max_nrhs, int lower,
                      cudaStream_t st);
int wsbm_lu_solve_batched(const TrsmDesc* d_desc_lower, const TrsmDesc* d_desc_upper, int nbatch,
                          int max_n, int max_nrhs, cudaStream_t st);
// B <- D^-T B for LU-factored D (descriptors with trans = 1): U^T, then L^T, then the row
// interchanges undone in reverse order.
int wsbm_lu_solve_t_batched(const TrsmDesc* d_desc, int nbatch, int max_n, int max_nrhs,
                            cudaStream_t st);
// max_m: the largest m of the batch (selects the thread-per-column kernel when it fits)
int wsbm_cpqr_batched(const QrDesc* d_desc, int nbatch, int mode, int max_m, cudaStream_t st);
int wsbm_cpqr_finish(const QrDesc* d_desc, int nbatch, cudaStream_t st);
