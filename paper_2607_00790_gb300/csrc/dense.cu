// Batched dense complex128 linear algebra for the HSS factor (Martinsson-Rokhlin solver,
// Sec. III): blocked LU with partial pivoting, blocked triangular solves, complex GEMM and a
// column-pivoted Householder QR for the interpolative decompositions.
//
// Every routine works on a batch of column-major matrices of different sizes described by
// device arrays.  Blocked algorithms step through panels of WSBM_NB columns on the host; each
// step launches one kernel over the whole batch (matrices that are already finished skip).
// The O(n^3) work is in the GEMM kernel, which tiles every matrix of the batch over many CTAs.
#include <math.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "dense.h"

#define GT 32  // GEMM tile (GT x GT outputs per CTA)
#define GK 16  // GEMM k-chunk

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {  // a*b + c
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
__device__ __forceinline__ double2 cfms(double2 a, double2 b, double2 c) {  // c - a*b
  return make_double2(fma(-a.x, b.x, fma(a.y, b.y, c.x)), fma(-a.x, b.y, fma(-a.y, b.x, c.y)));
}
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  double s = 1.0 / (b.x * b.x + b.y * b.y);
  return make_double2((a.x * b.x + a.y * b.y) * s, (a.y * b.x - a.x * b.y) * s);
}
__device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }

// --------------------------------------------------------------------------- GEMM ----
// C[m x n] = alpha * A[m x k] * B[k x n] + beta * C, one GT x GT tile of C.
template <bool TA>
__device__ void gemm_tile(int m, int n, int k, const double2* __restrict__ A, int64_t lda,
                          const double2* __restrict__ B, int64_t ldb, double2* C, int64_t ldc,
                          double2 alpha, double2 beta, int tm, int tn) {
  __shared__ double2 sA[GK][GT + 1];
  __shared__ double2 sB[GK][GT + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;  // 256 threads: 16 x 16, 2x2 each
  const int i0 = tm * GT, j0 = tn * GT;
  double2 acc[2][2];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) acc[a][b] = make_double2(0.0, 0.0);
  for (int kk = 0; kk < k; kk += GK) {
    __syncthreads();
    for (int t = threadIdx.x; t < GK * GT; t += blockDim.x) {
      int r = t % GT, c = t / GT;  // A: row r of the tile, k index c
      int gi = i0 + r, gk = kk + c;
      sA[c][r] = (gi < m && gk < k) ? A[TA ? gk + (int64_t)gi * lda : gi + (int64_t)gk * lda]
                                    : make_double2(0.0, 0.0);
      int br = t % GK, bc = t / GK;  // B: k index br, column bc
      int gk2 = kk + br, gj = j0 + bc;
      sB[br][bc] = (gk2 < k && gj < n) ? B[gk2 + (int64_t)gj * ldb] : make_double2(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll 4
    for (int c = 0; c < GK; ++c) {
      double2 a0 = sA[c][tx], a1 = sA[c][tx + 16];
      double2 b0 = sB[c][ty], b1 = sB[c][ty + 16];
      acc[0][0] = cfma(a0, b0, acc[0][0]);
      acc[1][0] = cfma(a1, b0, acc[1][0]);
      acc[0][1] = cfma(a0, b1, acc[0][1]);
      acc[1][1] = cfma(a1, b1, acc[1][1]);
    }
  }
  const bool beta0 = beta.x == 0.0 && beta.y == 0.0;
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      int gi = i0 + tx + 16 * a, gj = j0 + ty + 16 * b;
      if (gi < m && gj < n) {
        double2* p = C + gi + (int64_t)gj * ldc;
        double2 v = cmul(alpha, acc[a][b]);
        *p = beta0 ? v : cfma(beta, *p, v);
      }
    }
}

__global__ void __launch_bounds__(256) k_gemm(const GemmDesc* __restrict__ d, int nbatch) {
  const GemmDesc g = d[blockIdx.y];
  int ntm = (g.m + GT - 1) / GT, ntn = (g.n + GT - 1) / GT;
  for (int t = blockIdx.x; t < ntm * ntn; t += gridDim.x) {
    if (g.ta)
      gemm_tile<true>(g.m, g.n, g.k, g.A, g.lda, g.B, g.ldb, g.C, g.ldc, g.alpha, g.beta, t % ntm, t / ntm);
    else
      gemm_tile<false>(g.m, g.n, g.k, g.A, g.lda, g.B, g.ldb, g.C, g.ldc, g.alpha, g.beta, t % ntm, t / ntm);
  }
}

// LU trailing update at panel j0 (width jb): A22 -= A21 * A12.
__global__ void __launch_bounds__(256) k_lu_update(const LuDesc* __restrict__ d, int j0, int jb) {
  const LuDesc q = d[blockIdx.y];
  int e = j0 + jb;
  if (e >= q.n) return;
  int m = q.n - e;
  int nt = (m + GT - 1) / GT;
  const double2 one = make_double2(1.0, 0.0), mone = make_double2(-1.0, 0.0);
  int kb = min(jb, q.n - j0);
  for (int t = blockIdx.x; t < nt * nt; t += gridDim.x)
    gemm_tile<false>(m, m, kb, q.A + e + (int64_t)j0 * q.lda, q.lda, q.A + j0 + (int64_t)e * q.lda, q.lda,
              q.A + e + (int64_t)e * q.lda, q.lda, mone, one, t % nt, t / nt);
}

// ------------------------------------------------------------------- LU panel ----
// Factor columns [j0, j0+jb) of rows [j0, n) in place with partial pivoting; row swaps are
// applied inside the panel only (k_laswp applies them elsewhere).  One CTA per matrix.
__global__ void __launch_bounds__(256) k_lu_panel(const LuDesc* __restrict__ d, int j0, int jb,
                                                  int* __restrict__ info) {
  const LuDesc q = d[blockIdx.x];
  if (j0 >= q.n) return;
  const int n = q.n;
  const int je = min(j0 + jb, n);
  double2* A = q.A;
  const int64_t lda = q.lda;
  __shared__ double sval[256];
  __shared__ int sidx[256];
  __shared__ int spiv;
  for (int j = j0; j < je; ++j) {
    // pivot search over rows j..n-1 of column j
    double best = -1.0;
    int bi = j;
    for (int i = j + threadIdx.x; i < n; i += blockDim.x) {
      double v = cabs2(A[i + (int64_t)j * lda]);
      if (v > best) {
        best = v;
        bi = i;
      }
    }
    sval[threadIdx.x] = best;
    sidx[threadIdx.x] = bi;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) {
        double o = sval[threadIdx.x + s];
        int oi = sidx[threadIdx.x + s];
        if (o > sval[threadIdx.x] || (o == sval[threadIdx.x] && oi < sidx[threadIdx.x])) {
          sval[threadIdx.x] = o;
          sidx[threadIdx.x] = oi;
        }
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      spiv = sidx[0];
      q.piv[j] = sidx[0];
      if (sval[0] == 0.0 && info) info[blockIdx.x] = j + 1;  // exactly singular
    }
    __syncthreads();
    const int p = spiv;
    if (p != j) {
      for (int c = j0 + threadIdx.x; c < je; c += blockDim.x) {
        double2 t = A[j + (int64_t)c * lda];
        A[j + (int64_t)c * lda] = A[p + (int64_t)c * lda];
        A[p + (int64_t)c * lda] = t;
      }
    }
    __syncthreads();
    double2 piv = A[j + (int64_t)j * lda];
    double2 inv = (piv.x == 0.0 && piv.y == 0.0) ? make_double2(0.0, 0.0)
                                                   : cdiv(make_double2(1.0, 0.0), piv);
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x)
      A[i + (int64_t)j * lda] = cmul(A[i + (int64_t)j * lda], inv);
    __syncthreads();
    // rank-1 update of the remaining panel columns
    for (int c = j + 1; c < je; ++c) {
      double2 u = A[j + (int64_t)c * lda];
      for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x)
        A[i + (int64_t)c * lda] = cfms(A[i + (int64_t)j * lda], u, A[i + (int64_t)c * lda]);
    }
    __syncthreads();
  }
}

// Apply the row interchanges of panel [j0, j0+jb) to the columns outside the panel.
__global__ void k_laswp(const LuDesc* __restrict__ d, int j0, int jb) {
  const LuDesc q = d[blockIdx.y];
  if (j0 >= q.n) return;
  const int je = min(j0 + jb, q.n);
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < q.n; c += gridDim.x * blockDim.x) {
    if (c >= j0 && c < je) continue;
    double2* col = q.A + (int64_t)c * q.lda;
    for (int j = j0; j < je; ++j) {
      int p = q.piv[j];
      if (p != j) {
        double2 t = col[j];
        col[j] = col[p];
        col[p] = t;
      }
    }
  }
}

// A12 = L11^-1 A12 for the block row of panel [j0, j0+jb) (unit lower L11), columns >= j0+jb.
__global__ void k_lu_trsm_row(const LuDesc* __restrict__ d, int j0, int jb) {
  const LuDesc q = d[blockIdx.y];
  const int je = min(j0 + jb, q.n);
  if (je >= q.n) return;
  for (int c = je + blockIdx.x * blockDim.x + threadIdx.x; c < q.n; c += gridDim.x * blockDim.x) {
    double2* col = q.A + (int64_t)c * q.lda;
    for (int i = j0 + 1; i < je; ++i) {
      double2 s = col[i];
      for (int t = j0; t < i; ++t) s = cfms(q.A[i + (int64_t)t * q.lda], col[t], s);
      col[i] = s;
    }
  }
}

// ------------------------------------------------------------- triangular solves ----
// B <- op(T)^-1 B for a diagonal block [j0, j0+jb) of T (lower unit or upper non-unit),
// RHS columns in parallel.
__global__ void k_trsm_diag(const TrsmDesc* __restrict__ d, int j0, int jb, int fwd) {
  const TrsmDesc q = d[blockIdx.y];
  if (j0 >= q.n) return;
  const int je = min(j0 + jb, q.n);
  const bool unit = (fwd != 0) != (q.trans != 0);  // L and L^T have a unit diagonal
  const int64_t si = q.trans ? q.ldt : 1, st = q.trans ? 1 : q.ldt;  // op(T)(i,t) = T[i*si + t*st]
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < q.nrhs; c += gridDim.x * blockDim.x) {
    double2* col = q.B + (int64_t)c * q.ldb;
    if (fwd) {
      for (int i = j0; i < je; ++i) {
        double2 s = col[i];
        for (int t = j0; t < i; ++t) s = cfms(q.T[i * si + t * st], col[t], s);
        col[i] = unit ? s : cdiv(s, q.T[i * si + i * st]);
      }
    } else {
      for (int i = je - 1; i >= j0; --i) {
        double2 s = col[i];
        for (int t = i + 1; t < je; ++t) s = cfms(q.T[i * si + t * st], col[t], s);
        col[i] = unit ? s : cdiv(s, q.T[i * si + i * st]);
      }
    }
  }
}

// Update after a solved diagonal block: lower: B[je:n] -= T[je:n, j0:je] B[j0:je];
// upper: B[0:j0] -= T[0:j0, j0:je] B[j0:je].
__global__ void __launch_bounds__(256) k_trsm_update(const TrsmDesc* __restrict__ d, int j0, int jb,
                                                     int lower) {
  const TrsmDesc q = d[blockIdx.y];
  if (j0 >= q.n) return;
  const int je = min(j0 + jb, q.n);
  int m = lower ? q.n - je : j0;
  if (m <= 0 || q.nrhs <= 0) return;
  int r0 = lower ? je : 0;
  int ntm = (m + GT - 1) / GT, ntn = (q.nrhs + GT - 1) / GT;
  const double2 one = make_double2(1.0, 0.0), mone = make_double2(-1.0, 0.0);
  for (int t = blockIdx.x; t < ntm * ntn; t += gridDim.x) {
    if (q.trans)  // op(T)[r0.., j0..je) = (T[j0..je, r0..])^T
      gemm_tile<true>(m, q.nrhs, je - j0, q.T + j0 + (int64_t)r0 * q.ldt, q.ldt, q.B + j0, q.ldb,
                      q.B + r0, q.ldb, mone, one, t % ntm, t / ntm);
    else
      gemm_tile<false>(m, q.nrhs, je - j0, q.T + r0 + (int64_t)j0 * q.ldt, q.ldt, q.B + j0, q.ldb,
                       q.B + r0, q.ldb, mone, one, t % ntm, t / ntm);
  }
}

// Apply the LU row interchanges to B (forward order).
__global__ void k_apply_piv(const TrsmDesc* __restrict__ d) {
  const TrsmDesc q = d[blockIdx.y];
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < q.nrhs; c += gridDim.x * blockDim.x) {
    double2* col = q.B + (int64_t)c * q.ldb;
    for (int j = 0; j < q.n; ++j) {
      int p = q.piv[j];
      if (p != j) {
        double2 t = col[j];
        col[j] = col[p];
        col[p] = t;
      }
    }
  }
}

// Undo the LU row interchanges (reverse order): B <- P^T B.
__global__ void k_apply_piv_inv(const TrsmDesc* __restrict__ d) {
  const TrsmDesc q = d[blockIdx.y];
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < q.nrhs; c += gridDim.x * blockDim.x) {
    double2* col = q.B + (int64_t)c * q.ldb;
    for (int j = q.n - 1; j >= 0; --j) {
      int p = q.piv[j];
      if (p != j) {
        double2 t = col[j];
        col[j] = col[p];
        col[p] = t;
      }
    }
  }
}

// --------------------------------------------------------- fused LU + solve ----
// One CTA per matrix on a row-major working copy S of [A | B], so that a row of the trailing
// matrix is one coalesced access per warp.  Blocked right-looking LU with panels of LUS_B
// columns: the panel (rows j0..n-1) is staged in shared memory and factored by one warp with
// partial pivoting; then every thread takes one column c >= j0 + LUS_B at a time, applies the
// panel's row interchanges, solves the unit-lower L11 for its LUS_B rows of U12 and updates its
// trailing column with the rank-LUS_B product L21 U12 (one load and store per LUS_B complex
// FMAs).  Columns left of the panel only take the interchanges.  Back substitution with U on
// the B columns runs in the same blocks from the bottom, the U block column staged in shared
// memory.  Pivot choice: largest max(|re|, |im|) (integer compare of the bit patterns), first
// row on ties.
#define LUS_T 256
#define LUS_B 8

__device__ __forceinline__ unsigned long long lus_key(double2 v) {
  const unsigned long long m = 0x7fffffffffffffffull;
  const unsigned long long a = (unsigned long long)__double_as_longlong(v.x) & m;
  const unsigned long long b = (unsigned long long)__double_as_longlong(v.y) & m;
  return a > b ? a : b;
}

__device__ __forceinline__ double2* lus_col(const LuSolveDesc& q, int c) {
  return c < q.n ? q.A + (int64_t)c * q.lda : q.B + (int64_t)(c - q.n) * q.ldb;
}

// column-major [A | B] <-> row-major S through a 32 x 33 shared tile (8 warps, 4 rows each)
__device__ void lus_transpose(const LuSolveDesc& q, double2* S, int64_t ldr, double2* tile,
                              bool to_rows) {
  const int n = q.n, nc = q.n + q.nrhs;
  const int ntr = (n + 31) / 32, ntc = (nc + 31) / 32;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int t = 0; t < ntr * ntc; ++t) {
    const int r0 = (t % ntr) * 32, c0 = (t / ntr) * 32;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int a = w + 8 * s;
      if (to_rows) {
        const int c = c0 + a, r = r0 + lane;
        if (r < n && c < nc) tile[a * 33 + lane] = lus_col(q, c)[r];
      } else {
        const int r = r0 + a, c = c0 + lane;
        if (r < n && c < nc) tile[lane * 33 + a] = S[(int64_t)r * ldr + c];
      }
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int a = w + 8 * s;
      if (to_rows) {
        const int r = r0 + a, c = c0 + lane;
        if (r < n && c < nc) S[(int64_t)r * ldr + c] = tile[lane * 33 + a];
      } else {
        const int c = c0 + a, r = r0 + lane;
        if (r < n && c < nc) lus_col(q, c)[r] = tile[a * 33 + lane];
      }
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(LUS_T) k_lu_solve_fused(const LuSolveDesc* __restrict__ d) {
  const LuSolveDesc q = d[blockIdx.x];
  const int n = q.n, nr = q.nrhs, nc = n + nr;
  if (n <= 0) return;
  const int64_t ldr = ((int64_t)nc + 7) & ~(int64_t)7;  // = wsbm_lu_solve_ldr(n, nrhs)
  double2* __restrict__ S = q.S;
  extern __shared__ double2 lus_sm[];
  double2* sinv = lus_sm;    // n pivot reciprocals
  double2* sp = lus_sm + n;  // panel / U block: LUS_B columns of stride m + 1; transpose tile
  __shared__ int spiv[LUS_B];
  const int tid = threadIdx.x, lane = tid & 31;

  lus_transpose(q, S, ldr, sp, true);
  for (int j0 = 0; j0 < n; j0 += LUS_B) {
    const int bb = min(LUS_B, n - j0), m = n - j0, ld = m + 1;
    __syncthreads();  // trailing updates of the previous panel done
    for (int e = tid; e < m * bb; e += LUS_T) {
      const int r = e / bb, t = e - r * bb;
      sp[t * ld + r] = S[(int64_t)(j0 + r) * ldr + j0 + t];
    }
    __syncthreads();
    if (tid < 32) {  // panel factorization, one warp
      for (int jj = 0; jj < bb; ++jj) {
        double2* col = sp + jj * ld;
        unsigned long long best = 0;
        int bi = 0x7fffffff;
        for (int r = jj + lane; r < m; r += 32) {
          const unsigned long long k = lus_key(col[r]);
          if (k > best || bi == 0x7fffffff) {
            best = k;
            bi = r;
          }
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
          const unsigned long long ob = __shfl_xor_sync(0xffffffffu, best, o);
          const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
          if (ob > best || (ob == best && oi < bi)) {
            best = ob;
            bi = oi;
          }
        }
        const int p = bi;
        if (p != jj && lane < bb) {
          double2* a = sp + lane * ld;
          const double2 x = a[jj];
          a[jj] = a[p];
          a[p] = x;
        }
        __syncwarp();
        const double2 pv = col[jj];
        const double2 inv =
            (pv.x == 0.0 && pv.y == 0.0) ? make_double2(0.0, 0.0) : cdiv(make_double2(1.0, 0.0), pv);
        if (lane == 0) {
          spiv[jj] = j0 + p;
          q.piv[j0 + jj] = j0 + p;
          sinv[j0 + jj] = inv;
        }
        for (int r = jj + 1 + lane; r < m; r += 32) col[r] = cmul(col[r], inv);
        __syncwarp();
        for (int t = jj + 1; t < bb; ++t) {
          double2* ct = sp + t * ld;
          const double2 u = ct[jj];
          for (int r = jj + 1 + lane; r < m; r += 32) ct[r] = cfms(col[r], u, ct[r]);
        }
        __syncwarp();
      }
    }
    __syncthreads();
    for (int e = tid; e < m * bb; e += LUS_T) {
      const int r = e / bb, t = e - r * bb;
      S[(int64_t)(j0 + r) * ldr + j0 + t] = sp[t * ld + r];
    }
    for (int c = tid; c < j0; c += LUS_T)  // columns of L: interchanges only
      for (int jj = 0; jj < bb; ++jj) {
        const int p = spiv[jj];
        if (p != j0 + jj) {
          double2* a = S + (int64_t)(j0 + jj) * ldr + c;
          double2* b = S + (int64_t)p * ldr + c;
          const double2 x = *a;
          *a = *b;
          *b = x;
        }
      }
    for (int c = j0 + bb + tid; c < nc; c += LUS_T) {
      double2 u[LUS_B];
#pragma unroll
      for (int jj = 0; jj < LUS_B; ++jj)
        if (jj < bb) {
          const int p = spiv[jj];
          double2* a = S + (int64_t)(j0 + jj) * ldr + c;
          if (p != j0 + jj) {
            double2* b = S + (int64_t)p * ldr + c;
            const double2 x = *a;
            *a = *b;
            *b = x;
          }
        }
#pragma unroll
      for (int t = 0; t < LUS_B; ++t)
        if (t < bb) {
          double2 v = S[(int64_t)(j0 + t) * ldr + c];
#pragma unroll
          for (int s2 = 0; s2 < t; ++s2) v = cfms(sp[s2 * ld + t], u[s2], v);
          u[t] = v;
          S[(int64_t)(j0 + t) * ldr + c] = v;
        }
      int r = bb;
      for (; r + 1 < m; r += 2) {
        double2* e0 = S + (int64_t)(j0 + r) * ldr + c;
        double2* e1 = e0 + ldr;
        double2 a0 = *e0, a1 = *e1;
#pragma unroll
        for (int t = 0; t < LUS_B; ++t)
          if (t < bb) {
            a0 = cfms(sp[t * ld + r], u[t], a0);
            a1 = cfms(sp[t * ld + r + 1], u[t], a1);
          }
        *e0 = a0;
        *e1 = a1;
      }
      if (r < m) {
        double2* e0 = S + (int64_t)(j0 + r) * ldr + c;
        double2 a0 = *e0;
#pragma unroll
        for (int t = 0; t < LUS_B; ++t)
          if (t < bb) a0 = cfms(sp[t * ld + r], u[t], a0);
        *e0 = a0;
      }
    }
  }
  // back substitution U X = Y on the B columns, block rows from the bottom
  for (int j0 = ((n - 1) / LUS_B) * LUS_B; j0 >= 0; j0 -= LUS_B) {
    const int bb = min(LUS_B, n - j0), m = j0 + bb, ld = m + 1;
    __syncthreads();
    for (int e = tid; e < m * bb; e += LUS_T) {
      const int r = e / bb, t = e - r * bb;
      sp[t * ld + r] = S[(int64_t)r * ldr + j0 + t];
    }
    __syncthreads();
    for (int c = n + tid; c < nc; c += LUS_T) {
      double2 x[LUS_B];
#pragma unroll
      for (int t = 0; t < LUS_B; ++t) x[t] = t < bb ? S[(int64_t)(j0 + t) * ldr + c] : make_double2(0.0, 0.0);
#pragma unroll
      for (int t = LUS_B - 1; t >= 0; --t)
        if (t < bb) {
          x[t] = cmul(x[t], sinv[j0 + t]);
#pragma unroll
          for (int s2 = 0; s2 < t; ++s2) x[s2] = cfms(sp[t * ld + j0 + s2], x[t], x[s2]);
        }
#pragma unroll
      for (int t = 0; t < LUS_B; ++t)
        if (t < bb) S[(int64_t)(j0 + t) * ldr + c] = x[t];
      int i = 0;
      for (; i + 1 < j0; i += 2) {
        double2* e0 = S + (int64_t)i * ldr + c;
        double2* e1 = e0 + ldr;
        double2 a0 = *e0, a1 = *e1;
#pragma unroll
        for (int t = 0; t < LUS_B; ++t)
          if (t < bb) {
            a0 = cfms(sp[t * ld + i], x[t], a0);
            a1 = cfms(sp[t * ld + i + 1], x[t], a1);
          }
        *e0 = a0;
        *e1 = a1;
      }
      if (i < j0) {
        double2* e0 = S + (int64_t)i * ldr + c;
        double2 a0 = *e0;
#pragma unroll
        for (int t = 0; t < LUS_B; ++t)
          if (t < bb) a0 = cfms(sp[t * ld + i], x[t], a0);
        *e0 = a0;
      }
    }
  }
  __syncthreads();
  lus_transpose(q, S, ldr, sp, false);
}

// ------------------------------------------------- column-pivoted Householder QR ----
// One CTA per matrix M (m x n, in place).  Step j: pivot the column of largest remaining norm
// to position j, reflect rows j..m-1 with P = I - tau u u^H (Hermitian, tau real,
// u = x - beta e1, beta = -(x0/|x0|)|x|), so P x = beta e1.  Mode 0 stops at the first j with
// |beta_j| <= tol |beta_0| (rank k = j); mode 1 runs until step kt.  The state (reflected
// matrix, exact remaining column norms, permutation) lets a later call resume.  On return
// the R factor sits in rows 0..k-1 (diagonal included; below it, reflector data).
#ifndef CPQR_CB
#define CPQR_CB 4  // default trailing columns per warp pass of the warp variant (2, 4 or 8)
#endif
#ifndef CPQR_MINB
#define CPQR_MINB 4  // minimum resident CTAs per SM asked of the register allocator (measured best)
#endif
// TPC (thread per column): each thread updates whole trailing columns against the reflector
// staged in shared memory (no warp reductions; the strided column loads stay in L1, and on
// GB300 a warp-wide DFMA takes 16 clocks, which hides them).  Used when the reflector fits the
// shared memory budget (m <= CPQR_TPC_MAXM).
#ifndef CPQR_TPC_MAXM
#define CPQR_TPC_MAXM 2048
#endif
// Warp variant: CB trailing columns per warp per pass (2*CB partial sums, a power of two <= 16).
template <bool TPC, int CB>
__global__ void __launch_bounds__(256, CPQR_MINB) k_cpqr(const QrDesc* __restrict__ d, int mode) {
  // 5 - log2(2*CB): the lane holding reduced value t is t << SH
  constexpr int SH = CB == 1 ? 4 : CB == 2 ? 3 : CB == 4 ? 2 : CB == 8 ? 1 : 0;
  extern __shared__ double2 su[];  // TPC: the reflector u = M[j:m, j]
  const QrDesc q = d[blockIdx.x];
  const int m = q.m, n = q.n;
  double2* M = q.A;
  const int64_t ld = q.lda;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __shared__ double sval[256];
  __shared__ int sidx[256];
  __shared__ double s_tau;
  __shared__ double2 s_beta;
  __shared__ int s_stop;
  const int kmax = min(m, n);
  int j = q.state[0];  // resume point
  if (j == 0 && threadIdx.x == 0) q.state[1] = 0;
  // initial exact norms
  if (j == 0) {
    for (int c = warp; c < n; c += nw) {
      double s = 0.0;
      for (int i = lane; i < m; i += 32) s += cabs2(M[i + (int64_t)c * ld]);
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) {
        q.norm2[c] = s;
        q.nref[c] = s;
      }
    }
    for (int c = threadIdx.x; c < n; c += blockDim.x) q.perm[c] = c;
  }
  __syncthreads();
  const int kt = mode == 1 ? min(q.kt, kmax) : kmax;
  for (; j < kt; ++j) {
    // pivot: largest remaining norm (lowest index on ties)
    double best = -1.0;
    int bi = j;
    for (int c = j + threadIdx.x; c < n; c += blockDim.x) {
      double v = q.norm2[c];
      if (v > best) {
        best = v;
        bi = c;
      }
    }
    sval[threadIdx.x] = best;
    sidx[threadIdx.x] = bi;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) {
        double o = sval[threadIdx.x + s];
        int oi = sidx[threadIdx.x + s];
        if (o > sval[threadIdx.x] || (o == sval[threadIdx.x] && oi < sidx[threadIdx.x])) {
          sval[threadIdx.x] = o;
          sidx[threadIdx.x] = oi;
        }
      }
      __syncthreads();
    }
    const int p = sidx[0];
    const double nrm = sqrt(fmax(sval[0], 0.0));
    if (threadIdx.x == 0) {
      int stop = 0;
      if (j == 0) q.rdiag0[0] = nrm;
      if (mode == 0 && (nrm <= q.tol * q.rdiag0[0] || nrm == 0.0)) stop = 1;
      s_stop = stop;
    }
    __syncthreads();
    if (s_stop) break;
    if (p != j) {  // swap whole columns j <-> p
      for (int i = threadIdx.x; i < m; i += blockDim.x) {
        double2 t = M[i + (int64_t)j * ld];
        M[i + (int64_t)j * ld] = M[i + (int64_t)p * ld];
        M[i + (int64_t)p * ld] = t;
      }
      if (threadIdx.x == 0) {
        double t = q.norm2[j];
        q.norm2[j] = q.norm2[p];
        q.norm2[p] = t;
        t = q.nref[j];
        q.nref[j] = q.nref[p];
        q.nref[p] = t;
        int ti = q.perm[j];
        q.perm[j] = q.perm[p];
        q.perm[p] = ti;
      }
    }
    __syncthreads();
    // reflector from x = M[j:m, j]; |x| recomputed exactly
    double s = 0.0;
    for (int i = j + threadIdx.x; i < m; i += blockDim.x) s += cabs2(M[i + (int64_t)j * ld]);
    sval[threadIdx.x] = s;
    __syncthreads();
    for (int t = blockDim.x / 2; t > 0; t >>= 1) {
      if (threadIdx.x < t) sval[threadIdx.x] += sval[threadIdx.x + t];
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      double xn = sqrt(sval[0]);
      double2 x0 = M[j + (int64_t)j * ld];
      double a0 = sqrt(cabs2(x0));
      double2 beta = a0 > 0.0 ? make_double2(-x0.x / a0 * xn, -x0.y / a0 * xn) : make_double2(-xn, 0.0);
      double2 u0 = make_double2(x0.x - beta.x, x0.y - beta.y);
      // u^H u = 2 |x| (|x| + |x0|)
      double uu = 2.0 * xn * (xn + a0);
      s_tau = uu > 0.0 ? 2.0 / uu : 0.0;
      s_beta = beta;
      M[j + (int64_t)j * ld] = u0;
    }
    __syncthreads();
    const double tau = s_tau;
    if (TPC) {
      const int mm = m - j;
      for (int i = threadIdx.x; i < mm; i += blockDim.x) su[i] = M[j + i + (int64_t)j * ld];
      __syncthreads();
      for (int c = j + 1 + threadIdx.x; c < n; c += blockDim.x) {
        double2* col = M + (int64_t)c * ld + j;
        double wr0 = 0.0, wi0 = 0.0, wr1 = 0.0, wi1 = 0.0;  // w = u^H col, two chains
        int i = 0;
        for (; i + 1 < mm; i += 2) {
          const double2 u0 = su[i], c0 = col[i], u1 = su[i + 1], c1 = col[i + 1];
          wr0 = fma(u0.x, c0.x, fma(u0.y, c0.y, wr0));
          wi0 = fma(u0.x, c0.y, fma(-u0.y, c0.x, wi0));
          wr1 = fma(u1.x, c1.x, fma(u1.y, c1.y, wr1));
          wi1 = fma(u1.x, c1.y, fma(-u1.y, c1.x, wi1));
        }
        if (i < mm) {
          const double2 u0 = su[i], c0 = col[i];
          wr0 = fma(u0.x, c0.x, fma(u0.y, c0.y, wr0));
          wi0 = fma(u0.x, c0.y, fma(-u0.y, c0.x, wi0));
        }
        const double2 w = make_double2(tau * (wr0 + wr1), tau * (wi0 + wi1));
        for (i = 0; i < mm; ++i) col[i] = cfms(su[i], w, col[i]);
        // remaining norm: downdate by the new row-j entry, recompute once cancellation has
        // eaten half its digits
        double nv = q.norm2[c] - cabs2(col[0]);
        if (nv <= 1e-8 * q.nref[c]) {
          double ns = 0.0;
          for (i = 1; i < mm; ++i) ns += cabs2(col[i]);
          nv = ns;
          q.nref[c] = ns;
        }
        q.norm2[c] = fmax(nv, 0.0);
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        q.tauv[j] = tau;
        q.betav[j] = s_beta;
      }
      __syncthreads();
      continue;
    }
    // apply P to the trailing columns: a warp takes CB columns at a time, so each element
    // of u is loaded once for all of them and the 2*CB partial dot products are summed
    // across the warp by recursive halving (each level hands half of the values to the partner
    // lane; 2*CB - 1 + (5 - log2(2*CB)) adds per lane instead of 10 per column).  The remaining
    // norm is downdated by the new row-j entry and recomputed exactly once cancellation has
    // eaten half its digits (remaining norm below 1e-8 of the last exact one).
    const double2* u = M + (int64_t)j * ld;
    for (int c0 = j + 1 + warp * CB; c0 < n; c0 += nw * CB) {
      const int nc = min(CB, n - c0);
      double acc[2 * CB];  // re of the nc columns, then im
#pragma unroll
      for (int v = 0; v < 2 * CB; ++v) acc[v] = 0.0;
      for (int i = j + lane; i < m; i += 32) {  // w = u^H col, as fused multiply-adds
        const double2 ui = u[i];
#pragma unroll
        for (int v = 0; v < CB; ++v) {
          if (v < nc) {
            const double2 ci = M[i + (int64_t)(c0 + v) * ld];
            acc[v] = fma(ui.x, ci.x, fma(ui.y, ci.y, acc[v]));
            acc[CB + v] = fma(ui.x, ci.y, fma(-ui.y, ci.x, acc[CB + v]));
          }
        }
      }
      int cur = 2 * CB;
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) {
        if (cur > 1) {
          const int h = cur >> 1;
          const bool up = (lane & o) != 0;
#pragma unroll
          for (int v = 0; v < CB; ++v) {
            if (v < h) {
              const double send = up ? acc[v] : acc[v + h];
              const double keep = up ? acc[v + h] : acc[v];
              acc[v] = keep + __shfl_xor_sync(0xffffffffu, send, o);
            }
          }
          cur = h;
        } else {
          acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], o);
        }
      }
      // value t (re of column t for t < CB, im of column t - CB otherwise) sits in lane t << SH
      double2 w[CB];
#pragma unroll
      for (int v = 0; v < CB; ++v) {
        w[v].x = tau * __shfl_sync(0xffffffffu, acc[0], v << SH);
        w[v].y = tau * __shfl_sync(0xffffffffu, acc[0], (CB + v) << SH);
      }
      for (int i = j + lane; i < m; i += 32) {
        const double2 ui = u[i];
#pragma unroll
        for (int v = 0; v < CB; ++v) {
          if (v < nc) {
            double2* pc = M + i + (int64_t)(c0 + v) * ld;
            *pc = cfms(ui, w[v], *pc);
          }
        }
      }
      __syncwarp();
      for (int v = 0; v < nc; ++v) {
        const int c = c0 + v;
        const double2* col = M + (int64_t)c * ld;
        const double rj = cabs2(col[j]);  // the new row-j entry (written by lane 0)
        double nv = q.norm2[c] - rj;
        if (nv <= 1e-8 * q.nref[c]) {
          double ns = 0.0;
          for (int i = j + 1 + lane; i < m; i += 32) ns += cabs2(col[i]);
          for (int o = 16; o > 0; o >>= 1) ns += __shfl_xor_sync(0xffffffffu, ns, o);
          nv = ns;
          __syncwarp();
          if (lane == 0) q.nref[c] = ns;
        }
        __syncwarp();
        if (lane == 0) q.norm2[c] = fmax(nv, 0.0);
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      q.tauv[j] = tau;
      q.betav[j] = s_beta;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    q.state[0] = j;
    q.state[1] = j;  // rank reached
  }
}

// After the QR: put the diagonal of R back (the reflectors are no longer needed) and zero
// the part of column t below the diagonal within the first k rows (none: R11 is k x k).
__global__ void k_cpqr_finish(const QrDesc* __restrict__ d) {
  const QrDesc q = d[blockIdx.x];
  int k = q.state[1];
  for (int t = threadIdx.x; t < k; t += blockDim.x) q.A[t + (int64_t)t * q.lda] = q.betav[t];
}

// ------------------------------------------------------------------ host drivers ----
static int grid_cap() { return wsbm_sm_count() * 8; }

static int tiles_x(int64_t tiles) {
  int cap = grid_cap();
  return (int)(tiles < 1 ? 1 : (tiles < cap ? tiles : cap));
}

// The batched kernels below index their descriptor by blockIdx.y; a batch of more than
// LAUNCH_MAX_Y matrices runs as consecutive chunks (the matrices are independent).
#define LAUNCH_MAX_Y 65535

int wsbm_gemm_batched(const GemmDesc* d_desc, int nbatch, int max_m, int max_n, cudaStream_t st) {
  if (nbatch <= 0) return 0;
  if (nbatch > LAUNCH_MAX_Y) {
    for (int c = 0; c < nbatch; c += LAUNCH_MAX_Y)
      if (int rc = wsbm_gemm_batched(d_desc + c, std::min(LAUNCH_MAX_Y, nbatch - c), max_m, max_n, st))
        return rc;
    return 0;
  }
  int64_t t = (int64_t)((max_m + GT - 1) / GT) * ((max_n + GT - 1) / GT);
  dim3 grid(tiles_x(t), nbatch);
  k_gemm<<<grid, 256, 0, st>>>(d_desc, nbatch);
  wsbm_count_launch();
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int wsbm_lu_batched(const LuDesc* d_desc, int nbatch, int max_n, int* d_info, cudaStream_t st) {
  if (nbatch <= 0) return 0;
  if (nbatch > LAUNCH_MAX_Y) {
    for (int c = 0; c < nbatch; c += LAUNCH_MAX_Y)
      if (int rc = wsbm_lu_batched(d_desc + c, std::min(LAUNCH_MAX_Y, nbatch - c), max_n,
                                   d_info ? d_info + c : nullptr, st))
        return rc;
    return 0;
  }
  for (int j0 = 0; j0 < max_n; j0 += WSBM_NB) {
    k_lu_panel<<<nbatch, 256, 0, st>>>(d_desc, j0, WSBM_NB, d_info);
    wsbm_count_launch();
    dim3 gs(tiles_x((max_n + 127) / 128), nbatch);
    k_laswp<<<gs, 128, 0, st>>>(d_desc, j0, WSBM_NB);
    wsbm_count_launch();
    k_lu_trsm_row<<<gs, 128, 0, st>>>(d_desc, j0, WSBM_NB);
    wsbm_count_launch();
    int m = max_n - j0 - WSBM_NB;
    if (m > 0) {
      int64_t t = (int64_t)((m + GT - 1) / GT) * ((m + GT - 1) / GT);
      dim3 gg(tiles_x(t), nbatch);
      k_lu_update<<<gg, 256, 0, st>>>(d_desc, j0, WSBM_NB);
      wsbm_count_launch();
    }
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

// Triangular solves T^-1 B (lower unit: forward; upper non-unit: backward), blocked.
int wsbm_trsm_batched(const TrsmDesc* d_desc, int nbatch, int max_n, int max_nrhs, int lower,
                      cudaStream_t st) {
  if (nbatch <= 0 || max_n <= 0 || max_nrhs <= 0) return 0;
  if (nbatch > LAUNCH_MAX_Y) {
    for (int c = 0; c < nbatch; c += LAUNCH_MAX_Y)
      if (int rc = wsbm_trsm_batched(d_desc + c, std::min(LAUNCH_MAX_Y, nbatch - c), max_n, max_nrhs,
                                     lower, st))
        return rc;
    return 0;
  }
  dim3 gd(tiles_x((max_nrhs + 127) / 128), nbatch);
  if (lower) {
    for (int j0 = 0; j0 < max_n; j0 += WSBM_NB) {
      k_trsm_diag<<<gd, 128, 0, st>>>(d_desc, j0, WSBM_NB, 1);
      wsbm_count_launch();
      int m = max_n - j0 - WSBM_NB;
      if (m > 0) {
        int64_t t = (int64_t)((m + GT - 1) / GT) * ((max_nrhs + GT - 1) / GT);
        k_trsm_update<<<dim3(tiles_x(t), nbatch), 256, 0, st>>>(d_desc, j0, WSBM_NB, 1);
        wsbm_count_launch();
      }
    }
  } else {
    int last = ((max_n - 1) / WSBM_NB) * WSBM_NB;
    for (int j0 = last; j0 >= 0; j0 -= WSBM_NB) {
      k_trsm_diag<<<gd, 128, 0, st>>>(d_desc, j0, WSBM_NB, 0);
      wsbm_count_launch();
      if (j0 > 0) {
        int64_t t = (int64_t)((j0 + GT - 1) / GT) * ((max_nrhs + GT - 1) / GT);
        k_trsm_update<<<dim3(tiles_x(t), nbatch), 256, 0, st>>>(d_desc, j0, WSBM_NB, 0);
        wsbm_count_launch();
      }
    }
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

// Upper-triangular backward solves must start at each matrix's own last block; the blocked
// loop above runs from the batch maximum, and blocks with j0 >= n skip, so a smaller matrix
// simply starts later.  (Each k_trsm_diag / k_trsm_update guards j0 >= n.)

int wsbm_lu_solve_batched(const TrsmDesc* d_desc_lower, const TrsmDesc* d_desc_upper, int nbatch,
                          int max_n, int max_nrhs, cudaStream_t st) {
  if (nbatch <= 0) return 0;
  if (nbatch > LAUNCH_MAX_Y) {
    for (int c = 0; c < nbatch; c += LAUNCH_MAX_Y)
      if (int rc = wsbm_lu_solve_batched(d_desc_lower + c, d_desc_upper + c,
                                         std::min(LAUNCH_MAX_Y, nbatch - c), max_n, max_nrhs, st))
        return rc;
    return 0;
  }
  dim3 gd(tiles_x((max_nrhs + 127) / 128), nbatch);
  k_apply_piv<<<gd, 128, 0, st>>>(d_desc_lower);
  wsbm_count_launch();
  int rc = wsbm_trsm_batched(d_desc_lower, nbatch, max_n, max_nrhs, 1, st);
  if (rc) return rc;
  return wsbm_trsm_batched(d_desc_upper, nbatch, max_n, max_nrhs, 0, st);
}

int64_t wsbm_lu_solve_ldr(int n, int nrhs) { return ((int64_t)n + nrhs + 7) & ~(int64_t)7; }

int wsbm_lu_solve_fused_batched(const LuSolveDesc* d_desc, int nbatch, int max_n, int max_nc,
                                cudaStream_t st) {
  if (nbatch <= 0) return 0;
  if (max_n > WSBM_LUS_MAXN || max_n > max_nc) return -1;
  const size_t tile = 32 * 33, panel = (size_t)(max_n + 1) * LUS_B;
  const size_t sm = ((size_t)max_n + (panel > tile ? panel : tile)) * sizeof(double2);
  // the opt-in above 48 KB is a per-device attribute of the kernel
  if (wsbm_smem_optin((const void*)k_lu_solve_fused, sm) != cudaSuccess) return -3;
  k_lu_solve_fused<<<nbatch, LUS_T, sm, st>>>(d_desc);
  wsbm_count_launch();
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int wsbm_cpqr_batched(const QrDesc* d_desc, int nbatch, int mode, int max_m, cudaStream_t st) {
  if (nbatch <= 0) return 0;
  const WsbmTune tu = wsbm_tune_current();
  if (max_m <= CPQR_TPC_MAXM) {
    const int thr = tu.cpqr_threads == 128 ? 128 : 256;
    k_cpqr<true, CPQR_CB><<<nbatch, thr, (size_t)max_m * sizeof(double2), st>>>(d_desc, mode);
  } else if (tu.cpqr_cb == 2) {
    k_cpqr<false, 2><<<nbatch, 256, 0, st>>>(d_desc, mode);
  } else if (tu.cpqr_cb == 8) {
    k_cpqr<false, 8><<<nbatch, 256, 0, st>>>(d_desc, mode);
  } else {
    k_cpqr<false, 4><<<nbatch, 256, 0, st>>>(d_desc, mode);
  }
  wsbm_count_launch();
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int wsbm_cpqr_finish(const QrDesc* d_desc, int nbatch, cudaStream_t st) {
  if (nbatch <= 0) return 0;
  k_cpqr_finish<<<nbatch, 128, 0, st>>>(d_desc);
  wsbm_count_launch();
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int wsbm_lu_solve_t_batched(const TrsmDesc* d_desc, int nbatch, int max_n, int max_nrhs,
                            cudaStream_t st) {
  if (nbatch <= 0) return 0;
  if (nbatch > LAUNCH_MAX_Y) {
    for (int c = 0; c < nbatch; c += LAUNCH_MAX_Y)
      if (int rc = wsbm_lu_solve_t_batched(d_desc + c, std::min(LAUNCH_MAX_Y, nbatch - c), max_n,
                                           max_nrhs, st))
        return rc;
    return 0;
  }
  int rc = wsbm_trsm_batched(d_desc, nbatch, max_n, max_nrhs, 1, st);  // U^T, forward
  if (rc) return rc;
  rc = wsbm_trsm_batched(d_desc, nbatch, max_n, max_nrhs, 0, st);  // L^T, backward
  if (rc) return rc;
  dim3 gd(tiles_x((max_nrhs + 127) / 128), nbatch);
  k_apply_piv_inv<<<gd, 128, 0, st>>>(d_desc);
  wsbm_count_launch();
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

// ------------------------------------------------------------- LU of one large matrix ----
// Right-looking blocked LU with partial pivoting for a single large matrix (the dense root of
// a full build): outer panels of LUB_NB columns (LUB_NB_BIG for large n, where the deeper
// tensor-core products pay for the longer panels).  Each panel is factored recursively (halves,
// down to blocks of LUB_WB columns done column by column), with every column operation spread
// over the whole GPU: the pivot search is one launch whose CTAs combine their candidates with
// atomicMax on a 64-bit key, the row swap one small launch, the scaling and rank-1 update of
// the block (with the search of the next column fused in) one launch.  The panel's row swaps
// are applied to the other columns (k_laswp), U12 = L11^-1 A12 (k_lu_trsm_row) and the trailing
// update A22 -= L21 U12 runs on the tensor cores (wsbm_zgemm_tc).  Factors and piv as for
// wsbm_lu_batched.  Pivot: the row of largest max(|re|, |im|) compared on the upper 32 bits of
// its bit pattern (within 2^-20 of the largest), first row on ties.
#ifndef LUB_NB
#define LUB_NB 128      // outer panel width
#endif
#ifndef LUB_NB_BIG
#define LUB_NB_BIG 256  // outer panel width from LUB_BIG_N on: deeper tensor-core products
#endif
#ifndef LUB_BIG_N
#define LUB_BIG_N 12288
#endif
#define LUB_WB 8    // column-by-column block width
#define LUB_TC_K 32 // panel updates of at least this depth run on the tensor cores

__device__ __forceinline__ unsigned long long lub_key(double2 v, int row) {
  const unsigned long long m = 0x7fffffffffffffffull;
  const unsigned long long a = (unsigned long long)__double_as_longlong(v.x) & m;
  const unsigned long long b = (unsigned long long)__double_as_longlong(v.y) & m;
  const unsigned long long hi = (a > b ? a : b) >> 32;
  return (hi << 32) | (unsigned long long)(0xFFFFFFFFu - (unsigned)row);
}

__device__ __forceinline__ void lub_block_max(unsigned long long best, unsigned long long* key) {
  __shared__ unsigned long long red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long x = __shfl_xor_sync(0xFFFFFFFFu, best, o);
    best = x > best ? x : best;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x < 32) {
    best = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long x = __shfl_xor_sync(0xFFFFFFFFu, best, o);
      best = x > best ? x : best;
    }
    if (threadIdx.x == 0 && best) atomicMax(key, best);
  }
}

// key = max over rows [c, n) of column c (the key must be 0 on entry).
__global__ void __launch_bounds__(256) k_lub_search(const double2* __restrict__ A, int64_t lda, int n, int c,
                                                   unsigned long long* __restrict__ key) {
  unsigned long long best = 0;
  const double2* col = A + (int64_t)c * lda;
  for (int i = c + blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const unsigned long long k = lub_key(col[i], i);
    best = k > best ? k : best;
  }
  lub_block_max(best, key);
}

// Pivot of column c from its key: piv[c] = p, swap rows c and p over the panel columns
// [cs, ce), store 1/pivot; clear the key of column c + 1.
__global__ void k_lub_swap(double2* __restrict__ A, int64_t lda, int c, int cs, int ce,
                           const unsigned long long* __restrict__ key, int* __restrict__ piv,
                           double2* __restrict__ inv, unsigned long long* __restrict__ key_next,
                           int* __restrict__ info) {
  const unsigned long long k = key[0];
  const int p = k ? (int)(0xFFFFFFFFu - (unsigned)(k & 0xFFFFFFFFull)) : c;
  __shared__ double2 spv;
  if (threadIdx.x == 0) spv = A[p + (int64_t)c * lda];  // the value that lands on the diagonal
  __syncthreads();
  if (p != c) {
    for (int cc = cs + threadIdx.x; cc < ce; cc += blockDim.x) {
      double2* col = A + (int64_t)cc * lda;
      const double2 t = col[c];
      col[c] = col[p];
      col[p] = t;
    }
  }
  if (threadIdx.x == 0) {
    const double2 pv = spv;
    piv[c] = p;
    key_next[0] = 0ull;
    inv[0] = (pv.x == 0.0 && pv.y == 0.0) ? make_double2(0.0, 0.0) : cdiv(make_double2(1.0, 0.0), pv);
    if (pv.x == 0.0 && pv.y == 0.0 && info) info[0] = c + 1;
  }
}

// Rows (c, n): l = A[i,c] / pivot, A[i,c] = l, A[i,cc] -= l A[c,cc] for cc in (c, ce);
// then, when c + 1 < ce, the candidates of column c + 1 into key_next.
__global__ void __launch_bounds__(256) k_lub_update(double2* __restrict__ A, int64_t lda, int n, int c, int ce,
                                                   const double2* __restrict__ inv,
                                                   unsigned long long* __restrict__ key_next) {
  const double2 iv = inv[0];
  double2 u[LUB_WB];
  const int w = ce - c - 1;
#pragma unroll
  for (int t = 0; t < LUB_WB - 1; ++t) u[t] = t < w ? A[c + (int64_t)(c + 1 + t) * lda] : make_double2(0.0, 0.0);
  unsigned long long best = 0;
  for (int i = c + 1 + blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double2* a = A + i + (int64_t)c * lda;
    const double2 l = cmul(*a, iv);
    *a = l;
#pragma unroll
    for (int t = 0; t < LUB_WB - 1; ++t) {
      if (t < w) {
        double2* b = a + (int64_t)(1 + t) * lda;
        const double2 v = cfms(l, u[t], *b);
        *b = v;
        if (t == 0) {
          const unsigned long long k = lub_key(v, i);
          best = k > best ? k : best;
        }
      }
    }
  }
  if (w > 0) lub_block_max(best, key_next);
}

// B[r0 : r0+nb, cols] <- L^-1 B with L = the unit lower triangle of A[r0 : r0+nb, r0 : r0+nb];
// one thread per column of [c0, c1).
__global__ void k_lub_trsm(double2* __restrict__ A, int64_t lda, int r0, int nb, int c0, int c1) {
  const int c = c0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= c1) return;
  double2* col = A + (int64_t)c * lda;
  for (int i = r0 + 1; i < r0 + nb; ++i) {
    double2 s = col[i];
    for (int t = r0; t < i; ++t) s = cfms(A[i + (int64_t)t * lda], col[t], s);
    col[i] = s;
  }
}

// X = L^-1 for the unit lower triangle L of A[r0 : r0+nb, r0 : r0+nb] (X nb x nb, ldx = nb):
// one thread per column j, x_ij = -sum_{j<=t<i} l_it x_tj.
__global__ void k_lub_trinv(const double2* __restrict__ A, int64_t lda, int r0, int nb, double2* __restrict__ X) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nb) return;
  double2* x = X + (int64_t)j * nb;
  for (int i = 0; i < j; ++i) x[i] = make_double2(0.0, 0.0);
  x[j] = make_double2(1.0, 0.0);
  for (int i = j + 1; i < nb; ++i) {
    double2 s = make_double2(0.0, 0.0);
    const double2* li = A + (r0 + i) + (int64_t)r0 * lda;
    for (int t = j; t < i; ++t) s = cfms(li[(int64_t)t * lda], x[t], s);
    x[i] = s;
  }
}

// C[m x nc] -= A[m x k] B[k x nc] (the updates inside a panel), FP64 tiles.
__global__ void __launch_bounds__(256) k_lub_gemm(int m, int nc, int k, const double2* __restrict__ A,
                                                  int64_t lda, const double2* __restrict__ B, int64_t ldb,
                                                  double2* C, int64_t ldc) {
  const int ntm = (m + GT - 1) / GT, ntn = (nc + GT - 1) / GT;
  const double2 one = make_double2(1.0, 0.0), mone = make_double2(-1.0, 0.0);
  for (int t = blockIdx.x; t < ntm * ntn; t += gridDim.x)
    gemm_tile<false>(m, nc, k, A, lda, B, ldb, C, ldc, mone, one, t % ntm, t / ntm);
}

namespace {
struct LubCtx {
  double2* A;
  int64_t lda;
  int n;
  int* piv;
  unsigned long long* key;  // n + 1 keys
  double2* inv;
  int* info;
  cudaStream_t st;
  int cs, ce;   // current outer panel
  void* tcws;   // work space of the tensor-core products
};

int lub_grid(int64_t rows) {
  const int64_t b = (rows + 255) / 256, cap = (int64_t)wsbm_sm_count() * 4;
  return (int)(b < 1 ? 1 : (b < cap ? b : cap));
}

// factor columns [c0, c1) of rows [c0, n); row swaps across the whole outer panel
void lub_rec(const LubCtx& x, int c0, int c1) {
  const int w = c1 - c0;
  if (w <= LUB_WB) {
    k_lub_search<<<lub_grid(x.n - c0), 256, 0, x.st>>>(x.A, x.lda, x.n, c0, x.key + c0);
    wsbm_count_launch();
    for (int c = c0; c < c1; ++c) {
      k_lub_swap<<<1, 128, 0, x.st>>>(x.A, x.lda, c, x.cs, x.ce, x.key + c, x.piv, x.inv, x.key + c + 1, x.info);
      k_lub_update<<<lub_grid(x.n - c - 1), 256, 0, x.st>>>(x.A, x.lda, x.n, c, c1, x.inv, x.key + c + 1);
      wsbm_count_launches(2);
    }
    return;
  }
  const int mid = c0 + ((w / 2 + LUB_WB - 1) / LUB_WB) * LUB_WB;
  lub_rec(x, c0, mid);
  // A[c0:mid, mid:c1] = L11^-1 A[c0:mid, mid:c1];  A[mid:n, mid:c1] -= A[mid:n, c0:mid] A[c0:mid, mid:c1]
  k_lub_trsm<<<(c1 - mid + 63) / 64, 64, 0, x.st>>>(x.A, x.lda, c0, mid - c0, mid, c1);
  wsbm_count_launch();
  const int m = x.n - mid;
  if (mid - c0 >= LUB_TC_K && m >= 2 * LUB_NB) {
    // the wide updates of the panel on the tensor cores
    const double2 mone = make_double2(-1.0, 0.0), one = make_double2(1.0, 0.0);
    wsbm_zgemm_tc(m, c1 - mid, mid - c0, mone, x.A + mid + (int64_t)c0 * x.lda, x.lda,
                  x.A + c0 + (int64_t)mid * x.lda, x.lda, one, x.A + mid + (int64_t)mid * x.lda, x.lda,
                  x.tcws, x.st);
  } else {
    const int64_t tiles = (int64_t)((m + GT - 1) / GT) * ((c1 - mid + GT - 1) / GT);
    k_lub_gemm<<<tiles_x(tiles), 256, 0, x.st>>>(m, c1 - mid, mid - c0, x.A + mid + (int64_t)c0 * x.lda, x.lda,
                                               x.A + c0 + (int64_t)mid * x.lda, x.lda,
                                               x.A + mid + (int64_t)mid * x.lda, x.lda);
    wsbm_count_launch();
  }
  // the key of column mid is set by the first search of the right half
  lub_rec(x, mid, c1);
}
}  // namespace

int wsbm_lu_big_large_n() { return LUB_BIG_N; }

// outer panel width: the tuned one of n's size class (LUB_NB / LUB_NB_BIG by default)
static int lub_nb(int n) {
  const WsbmTune t = wsbm_tune_current();
  return n >= LUB_BIG_N ? t.root_nb_large : t.root_nb_mid;
}

size_t wsbm_lu_big_ws_bytes(int n) {
  size_t b = wsbm_zgemm_tc_ws_bytes(n, n, LUB_NB_BIG);  // either panel width fits
  b = (b + 255) & ~(size_t)255;
  b += ((size_t)n + 8) * sizeof(unsigned long long) + 256 + sizeof(LuDesc) + 256;
  b += (size_t)LUB_NB_BIG * LUB_NB_BIG * sizeof(double2) + 256;  // L11^-1
  return b;
}

int wsbm_lu_big(double2* A, int64_t lda, int n, int* piv, int* d_info, void* ws, cudaStream_t st) {
  return wsbm_lu_big_nb(A, lda, n, piv, d_info, ws, st, lub_nb(n));
}

int wsbm_lu_big_nb(double2* A, int64_t lda, int n, int* piv, int* d_info, void* ws, cudaStream_t st, int nb) {
  if (n <= 0) return 0;
  if (!A || !piv || !ws || lda < n || ((uintptr_t)ws & 255)) return -1;
  if (nb != LUB_NB && nb != LUB_NB_BIG) return -1;
  size_t off = (wsbm_zgemm_tc_ws_bytes(n, n, LUB_NB_BIG) + 255) & ~(size_t)255;
  unsigned long long* key = (unsigned long long*)((char*)ws + off);
  off += ((size_t)n + 8) * sizeof(unsigned long long);
  off = (off + 255) & ~(size_t)255;
  double2* inv = (double2*)((char*)ws + off);
  LuDesc* dd = (LuDesc*)((char*)ws + off + 256);
  double2* Linv = (double2*)((char*)ws + ((off + 256 + sizeof(LuDesc) + 255) & ~(size_t)255));
  LuDesc h;
  h.A = A;
  h.lda = lda;
  h.piv = piv;
  h.n = n;
  h.pad = 0;
  if (cudaMemcpyAsync(dd, &h, sizeof(h), cudaMemcpyHostToDevice, st) != cudaSuccess) return -3;
  if (cudaMemsetAsync(key, 0, ((size_t)n + 8) * sizeof(unsigned long long), st) != cudaSuccess) return -3;
  LubCtx x;
  x.A = A;
  x.lda = lda;
  x.n = n;
  x.piv = piv;
  x.key = key;
  x.inv = inv;
  x.info = d_info;
  x.st = st;
  x.tcws = ws;
  const double2 mone = make_double2(-1.0, 0.0), one = make_double2(1.0, 0.0);
  for (int j0 = 0; j0 < n; j0 += nb) {
    const int jb = std::min(nb, n - j0), je = j0 + jb;
    x.cs = j0;
    x.ce = je;
    lub_rec(x, j0, je);
    dim3 gs(tiles_x((n + 127) / 128), 1);
    k_laswp<<<gs, 128, 0, st>>>(dd, j0, jb);
    wsbm_count_launch();
    if (je < n) {
      const int m = n - je;
      if (m >= 2 * LUB_NB) {
        // U12 = L11^-1 A12 as a tensor-core product with the explicit inverse of the unit lower
        // L11 (the digit planes of A12 are formed before A12 is overwritten)
        k_lub_trinv<<<(jb + 63) / 64, 64, 0, st>>>(A, lda, j0, jb, Linv);
        wsbm_count_launch();
        const double2 zero = make_double2(0.0, 0.0);
        int rc = wsbm_zgemm_tc(jb, m, jb, one, Linv, jb, A + j0 + (int64_t)je * lda, lda, zero,
                               A + j0 + (int64_t)je * lda, lda, ws, st);
        if (rc) return rc;
      } else {
        k_lu_trsm_row<<<gs, 128, 0, st>>>(dd, j0, jb);
        wsbm_count_launch();
      }
      int rc = wsbm_zgemm_tc(m, m, jb, mone, A + je + (int64_t)j0 * lda, lda, A + j0 + (int64_t)je * lda, lda,
                             one, A + je + (int64_t)je * lda, lda, ws, st);
      if (rc) return rc;
    }
  }
  // (the tensor-core kernel's timeout flag is read by the caller through wsbm_zgemm_tc_status)
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

// ----------------------------------------------- batched LU + solve on the tensor cores ----
// The box factors of a level (LU(D) with D^-1 L, and Dhat = M^-1) as a blocked right-looking LU
// with LUT_NB-column panels over every box of the batch at once: per panel, the panel is
// factored with partial pivoting on the FP64 pipe (k_lu_panel, one CTA per matrix), its row
// swaps are applied to the rest of A and to B, U12 = L11^-1 A12 (and L11^-1 B12) and the
// trailing update A22 -= L21 U12 (B22 likewise) run as batched products on the tensor cores
// (wsbm_zgemm_tc_batched, two items per box: the A part and the B part), with L11^-1 formed
// explicitly per box.  The back substitution X = U^-1 B runs by panels from the bottom:
// X_p = U_pp^-1 X_p and X_{<p} -= U_{<p,p} X_p, again as batched tensor-core products.
// Same factors (L unit lower, U, piv[j] = the row swapped with row j) and solution as
// k_lu_solve_fused, to rounding; pivoting by |a|^2 (k_lu_panel).
#define LUT_NB 64

// Apply the swaps piv[j0 .. je) to the columns of A outside [j0, je) and to every column of B.
__global__ void k_lut_swap(const LuSolveDesc* __restrict__ d, int j0, int jb) {
  const LuSolveDesc q = d[blockIdx.y];
  if (j0 >= q.n) return;
  const int je = min(j0 + jb, q.n), nc = q.n + q.nrhs;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
    if (c >= j0 && c < je) continue;
    double2* col = c < q.n ? q.A + (int64_t)c * q.lda : q.B + (int64_t)(c - q.n) * q.ldb;
    for (int j = j0; j < je; ++j) {
      const int p = q.piv[j];
      if (p != j) {
        const double2 t = col[j];
        col[j] = col[p];
        col[p] = t;
      }
    }
  }
}

// X = inverse of the unit lower (upper = 0) or of the upper (upper = 1, non-unit) triangle of
// the diagonal block A[j0 : j0+jb, j0 : j0+jb] of item blockIdx.y; X: jb x jb (ld jb) at
// X + blockIdx.y * ldx_item.  One thread per column j: x_ij from the rows before (lower) or
// after (upper) it.
__global__ void k_lut_trinv(const LuSolveDesc* __restrict__ d, int j0, int jb, int upper,
                            double2* __restrict__ Xall, int64_t ldx_item) {
  const LuSolveDesc q = d[blockIdx.y];
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j0 >= q.n) return;
  const int b = min(jb, q.n - j0);
  if (j >= b) return;
  double2* x = Xall + blockIdx.y * ldx_item + (int64_t)j * b;
  const double2* T = q.A + j0 + (int64_t)j0 * q.lda;
  const double2 one = make_double2(1.0, 0.0), zero = make_double2(0.0, 0.0);
  if (!upper) {
    for (int i = 0; i < j; ++i) x[i] = zero;
    x[j] = one;
    for (int i = j + 1; i < b; ++i) {
      double2 s = zero;
      for (int t = j; t < i; ++t) s = cfms(T[i + (int64_t)t * q.lda], x[t], s);
      x[i] = s;
    }
  } else {
    for (int i = j + 1; i < b; ++i) x[i] = zero;
    const double2 djj = T[j + (int64_t)j * q.lda];
    x[j] = (djj.x == 0.0 && djj.y == 0.0) ? zero : cdiv(one, djj);
    for (int i = j - 1; i >= 0; --i) {
      double2 s = zero;
      for (int t = i + 1; t <= j; ++t) s = cfms(T[i + (int64_t)t * q.lda], x[t], s);
      const double2 dii = T[i + (int64_t)i * q.lda];
      x[i] = (dii.x == 0.0 && dii.y == 0.0) ? zero : cdiv(s, dii);
    }
  }
}

// Inverses of the diagonal blocks of LU factors (unit lower L, upper U), for block triangular
// solves whose products run on the tensor cores.  Item blockIdx.y with block width nb = q.nb,
// block p = blockIdx.x (rows and columns p nb .. min(n, (p + 1) nb)), blockIdx.z = 0: L_pp^-1
// into Linv + p nb^2, 1: U_pp^-1 into Uinv + p nb^2 (column-major, leading dimension nb; the
// part outside a ragged last block is not written).  Thread j forms column j by substitution.
// A zero diagonal entry of U leaves a zero row in U_pp^-1.
__global__ void k_lu_dinv(const DinvDesc* __restrict__ d) {
  const DinvDesc q = d[blockIdx.y];
  const int nb = q.nb, p = blockIdx.x, j0 = p * nb;
  if (j0 >= q.n) return;
  const int b = min(nb, q.n - j0), j = threadIdx.x;
  if (j >= b) return;
  const bool upper = blockIdx.z != 0;
  double2* x = (upper ? q.Uinv : q.Linv) + (int64_t)p * nb * nb + (int64_t)j * nb;
  const double2* T = q.A + j0 + (int64_t)j0 * q.lda;
  const double2 one = make_double2(1.0, 0.0), zero = make_double2(0.0, 0.0);
  if (!upper) {
    for (int i = 0; i < j; ++i) x[i] = zero;
    x[j] = one;
    for (int i = j + 1; i < b; ++i) {
      double2 s = zero;
      for (int t = j; t < i; ++t) s = cfms(T[i + (int64_t)t * q.lda], x[t], s);
      x[i] = s;
    }
  } else {
    for (int i = j + 1; i < b; ++i) x[i] = zero;
    const double2 djj = T[j + (int64_t)j * q.lda];
    x[j] = (djj.x == 0.0 && djj.y == 0.0) ? zero : cdiv(one, djj);
    for (int i = j - 1; i >= 0; --i) {
      double2 s = zero;
      for (int t = i + 1; t <= j; ++t) s = cfms(T[i + (int64_t)t * q.lda], x[t], s);
      const double2 dii = T[i + (int64_t)i * q.lda];
      x[i] = (dii.x == 0.0 && dii.y == 0.0) ? zero : cdiv(s, dii);
    }
  }
}

int wsbm_lu_dinv_batched(const DinvDesc* d_desc, int nitems, int max_blocks, int max_nb, cudaStream_t st) {
  if (nitems <= 0 || max_blocks <= 0) return 0;
  if (max_nb < 1 || max_nb > 256) return -1;
  for (int c = 0; c < nitems; c += LAUNCH_MAX_Y) {
    const int n = std::min(LAUNCH_MAX_Y, nitems - c);
    k_lu_dinv<<<dim3(max_blocks, n, 2), max_nb, 0, st>>>(d_desc + c);
    wsbm_count_launch();
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

// perm of the row interchanges piv (piv[j]: the row swapped with row j at step j, j = 0..n-1):
// (P b)[r] = b[perm[r]].  One thread per item (the swaps are sequential).
__global__ void k_piv_perm(const PermDesc* __restrict__ d, int nitems) {
  const int it = blockIdx.x * blockDim.x + threadIdx.x;
  if (it >= nitems) return;
  const PermDesc q = d[it];
  for (int r = 0; r < q.n; ++r) q.perm[r] = r;
  for (int j = 0; j < q.n; ++j) {
    const int p = q.piv[j];
    if (p > j && p < q.n) {
      const int t = q.perm[j];
      q.perm[j] = q.perm[p];
      q.perm[p] = t;
    }
  }
}

int wsbm_piv_perm_batched(const PermDesc* d_desc, int nitems, cudaStream_t st) {
  if (nitems <= 0) return 0;
  k_piv_perm<<<(nitems + 63) / 64, 64, 0, st>>>(d_desc, nitems);
  wsbm_count_launch();
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

size_t wsbm_lu_solve_tc_ws_bytes(const LuSolveDesc* h, int nbatch) {
  // the largest product step: two items per box (A part and B part) of the first panel
  std::vector<TcProduct> p;
  p.reserve(2 * (size_t)nbatch);
  int maxn = 0;
  for (int i = 0; i < nbatch; ++i) {
    TcProduct a;
    memset(&a, 0, sizeof(a));
    a.m = h[i].n;
    a.n = h[i].n;
    a.k = LUT_NB;
    p.push_back(a);
    a.n = h[i].nrhs > 0 ? h[i].nrhs : 1;
    p.push_back(a);
    maxn = std::max(maxn, h[i].n);
  }
  size_t b = wsbm_zgemm_tc_batched_ws_bytes(p.data(), (int)p.size());
  b = (b + 255) & ~(size_t)255;
  b += (size_t)nbatch * LUT_NB * LUT_NB * sizeof(double2) + 256;  // diagonal-block inverses
  return b;
}

int wsbm_lu_solve_tc_batched(const LuSolveDesc* h, const LuSolveDesc* d, int nbatch, const LuDesc* d_lu,
                             void* ws, cudaStream_t st) {
  return wsbm_lu_solve_tc_batched_nb(h, d, nbatch, d_lu, ws, st, wsbm_tune_current().box_nb);
}

int wsbm_lu_solve_tc_batched_nb(const LuSolveDesc* h, const LuSolveDesc* d, int nbatch, const LuDesc* d_lu,
                                void* ws, cudaStream_t st, int nb) {
  if (nbatch <= 0) return 0;
  if (nb < 8 || nb > LUT_NB || nb % 8) return -1;
  if (nbatch > 32767 || !h || !d || !d_lu || !ws) return -1;
  int maxn = 0, maxnc = 0;
  for (int i = 0; i < nbatch; ++i) {
    maxn = std::max(maxn, h[i].n);
    maxnc = std::max(maxnc, h[i].n + h[i].nrhs);
  }
  size_t off = wsbm_zgemm_tc_ws_bytes(1, 1, 1);  // recomputed below for the actual products
  {
    std::vector<TcProduct> p(2 * (size_t)nbatch);
    for (int i = 0; i < nbatch; ++i) {
      memset(&p[2 * i], 0, 2 * sizeof(TcProduct));
      p[2 * i].m = p[2 * i + 1].m = h[i].n;
      p[2 * i].n = h[i].n;
      p[2 * i + 1].n = h[i].nrhs > 0 ? h[i].nrhs : 1;
      p[2 * i].k = p[2 * i + 1].k = LUT_NB;
    }
    off = (wsbm_zgemm_tc_batched_ws_bytes(p.data(), (int)p.size()) + 255) & ~(size_t)255;
  }
  double2* X = (double2*)((char*)ws + off);  // LUT_NB x LUT_NB per box
  const int64_t ldx = (int64_t)LUT_NB * LUT_NB;
  const double2 one = make_double2(1.0, 0.0), mone = make_double2(-1.0, 0.0), zero = make_double2(0.0, 0.0);
  std::vector<TcProduct> items;
  items.reserve(2 * (size_t)nbatch);
  auto run = [&](double2 alpha, double2 beta) -> int {
    if (items.empty()) return 0;
    int rc = wsbm_zgemm_tc_batched(items.data(), (int)items.size(), alpha, beta, ws, st);
    items.clear();
    return rc;
  };
  auto add = [&](const double2* A, int64_t lda, const double2* B, int64_t ldb, double2* C, int64_t ldc, int m,
                 int n, int k) {
    if (m <= 0 || n <= 0 || k <= 0) return;
    TcProduct t;
    t.A = A;
    t.lda = lda;
    t.B = B;
    t.ldb = ldb;
    t.C = C;
    t.ldc = ldc;
    t.m = m;
    t.n = n;
    t.k = k;
    t.pad = 0;
    items.push_back(t);
  };
  // ---- factorization
  for (int j0 = 0; j0 < maxn; j0 += nb) {
    k_lu_panel<<<nbatch, 256, 0, st>>>(d_lu, j0, nb, nullptr);
    k_lut_swap<<<dim3(tiles_x((maxnc + 127) / 128), nbatch), 128, 0, st>>>(d, j0, nb);
    k_lut_trinv<<<dim3(1, nbatch), nb, 0, st>>>(d, j0, nb, 0, X, ldx);
    wsbm_count_launches(3);
    // U12 = L11^-1 [A12 | B1]  (in place: the digit planes are formed before C is written)
    for (int i = 0; i < nbatch; ++i) {
      const LuSolveDesc& q = h[i];
      if (j0 >= q.n) continue;
      const int jb = std::min(nb, q.n - j0), je = j0 + jb;
      const double2* Li = X + i * ldx;
      add(Li, jb, q.A + j0 + (int64_t)je * q.lda, q.lda, q.A + j0 + (int64_t)je * q.lda, q.lda, jb, q.n - je, jb);
      add(Li, jb, q.B + j0, q.ldb, q.B + j0, q.ldb, jb, q.nrhs, jb);
    }
    if (int rc = run(one, zero)) return rc;
    // A22 -= L21 U12, B2 -= L21 U12_B
    for (int i = 0; i < nbatch; ++i) {
      const LuSolveDesc& q = h[i];
      if (j0 >= q.n) continue;
      const int jb = std::min(nb, q.n - j0), je = j0 + jb;
      const double2* L21 = q.A + je + (int64_t)j0 * q.lda;
      add(L21, q.lda, q.A + j0 + (int64_t)je * q.lda, q.lda, q.A + je + (int64_t)je * q.lda, q.lda, q.n - je,
          q.n - je, jb);
      add(L21, q.lda, q.B + j0, q.ldb, q.B + je, q.ldb, q.n - je, q.nrhs, jb);
    }
    if (int rc = run(mone, one)) return rc;
  }
  // ---- back substitution X = U^-1 (L^-1 P B), panels from the bottom
  for (int j0 = ((maxn - 1) / nb) * nb; j0 >= 0; j0 -= nb) {
    k_lut_trinv<<<dim3(1, nbatch), nb, 0, st>>>(d, j0, nb, 1, X, ldx);
    wsbm_count_launch();
    for (int i = 0; i < nbatch; ++i) {
      const LuSolveDesc& q = h[i];
      if (j0 >= q.n) continue;
      const int jb = std::min(nb, q.n - j0);
      add(X + i * ldx, jb, q.B + j0, q.ldb, q.B + j0, q.ldb, jb, q.nrhs, jb);
    }
    if (int rc = run(one, zero)) return rc;
    for (int i = 0; i < nbatch; ++i) {
      const LuSolveDesc& q = h[i];
      if (j0 >= q.n || j0 == 0) continue;
      const int jb = std::min(nb, q.n - j0);
      add(q.A + (int64_t)j0 * q.lda, q.lda, q.B + j0, q.ldb, q.B, q.ldb, j0, q.nrhs, jb);
    }
    if (int rc = run(mone, one)) return rc;
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}
