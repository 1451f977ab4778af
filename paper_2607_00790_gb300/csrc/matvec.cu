// Matrix-free products with the full WSBM Nystrom matrix (no storage): y = A x and y = A^T x.
#include <math.h>

#include "entry_blocks.cuh"

// Matrix-free product y = A x (TRANS: y = A^T x) over every node pair (dense, O(N^2) pair
// evaluations; used for residuals and iterative refinement of HSS and adjoint solutions).
// Thread = output node i; CTA row blockIdx.y covers the other nodes [j0, j1); per-split
// partial sums, reduced in a fixed order by k_matvec_reduce.  Vectors in paper order.
#define MV_THREADS 128
#define MV_RHS 4  // right-hand sides sharing each pair's Hankel evaluations
struct MvSlot {
  double x, y, nx, ny, w, kap;
  double2 u[MV_RHS], q[MV_RHS];
};

// nr <= MV_RHS columns c0 .. c0 + nr - 1 of x (column stride 2N); partial sums of column r of
// split s at part[(s * MV_RHS + r) * 2N + row].
template <bool TRANS>
__global__ void __launch_bounds__(MV_THREADS)
    k_matvec(DevGeom g, Phys ph, const double2* __restrict__ xin, int nr, int64_t jspan,
             double2* __restrict__ part) {
  __shared__ HkTables T;
  __shared__ MvSlot sj[MV_THREADS];
  hk_stage_tables(&T);
  const int64_t N = g.n;
  const int64_t i = (int64_t)blockIdx.x * MV_THREADS + threadIdx.x;
  const int64_t j0 = (int64_t)blockIdx.y * jspan;
  const int64_t j1 = min(N, j0 + jspan);
  const bool valid = i < N;
  double xi = 0, yi = 0, nxi = 0, nyi = 0, wi = 0, ki = 0;
  if (valid) {
    xi = g.x[i];
    yi = g.y[i];
    nxi = g.nx[i];
    nyi = g.ny[i];
    wi = g.w[i];
    ki = g.kappa[i];
  }
  double2 a0[MV_RHS], a1[MV_RHS];
#pragma unroll
  for (int r = 0; r < MV_RHS; ++r) a0[r] = a1[r] = make_double2(0.0, 0.0);
  for (int64_t jc = j0; jc < j1; jc += MV_THREADS) {
    __syncthreads();
    {
      int64_t j = jc + threadIdx.x;
      if (j < j1) {
        MvSlot& s = sj[threadIdx.x];
        s.x = g.x[j];
        s.y = g.y[j];
        s.nx = g.nx[j];
        s.ny = g.ny[j];
        s.w = g.w[j];
        s.kap = g.kappa[j];
#pragma unroll
        for (int r = 0; r < MV_RHS; ++r) {
          const bool on = r < nr;
          s.u[r] = on ? xin[(int64_t)r * 2 * N + j] : make_double2(0.0, 0.0);
          s.q[r] = on ? xin[(int64_t)r * 2 * N + N + j] : make_double2(0.0, 0.0);
        }
      }
    }
    __syncthreads();
    if (!valid) continue;
    const int nj = (int)min((int64_t)MV_THREADS, j1 - jc);
#pragma unroll 1
    for (int jj = 0; jj < nj; ++jj) {
      // keep the Hankel tables in shared memory: no hoisting of their loads out of the loop
      asm volatile("" ::: "memory");
      const MvSlot& s = sj[jj];
      double2 e[2][2];
      if (jc + jj == i) {
        block_diag(ph, wi, ki, e);
      } else if (!TRANS) {  // block (i, j): row node i, column node j
        PairGeom G;
        pair_geom(xi, yi, nxi, nyi, s.x, s.y, s.nx, s.ny, ph, G);
        block_offdiag(T, ph, G, s.w, e);
      } else {  // block (j, i), applied transposed
        PairGeom G;
        pair_geom(s.x, s.y, s.nx, s.ny, xi, yi, nxi, nyi, ph, G);
        block_offdiag(T, ph, G, wi, e);
      }
      if (TRANS) {
        double2 t = e[0][1];
        e[0][1] = e[1][0];
        e[1][0] = t;
      }
#pragma unroll
      for (int r = 0; r < MV_RHS; ++r) {
        if (r >= nr) break;
        const double2 u = s.u[r], q = s.q[r];
        a0[r].x += e[0][0].x * u.x - e[0][0].y * u.y + e[0][1].x * q.x - e[0][1].y * q.y;
        a0[r].y += e[0][0].x * u.y + e[0][0].y * u.x + e[0][1].x * q.y + e[0][1].y * q.x;
        a1[r].x += e[1][0].x * u.x - e[1][0].y * u.y + e[1][1].x * q.x - e[1][1].y * q.y;
        a1[r].y += e[1][0].x * u.y + e[1][0].y * u.x + e[1][1].x * q.y + e[1][1].y * q.x;
      }
    }
  }
  if (valid) {
#pragma unroll
    for (int r = 0; r < MV_RHS; ++r) {
      if (r >= nr) break;
      double2* pr = part + ((int64_t)blockIdx.y * MV_RHS + r) * 2 * N;
      pr[i] = a0[r];
      pr[N + i] = a1[r];
    }
  }
}

// y[:, r] = sum over the splits, in split order, for the nr columns of one launch.
__global__ void k_matvec_reduce(int64_t N, int nsplit, int nr, const double2* __restrict__ part,
                                double2* __restrict__ y) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < 2 * N * nr;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / (2 * N), row = e % (2 * N);
    double2 s = make_double2(0.0, 0.0);
    for (int t = 0; t < nsplit; ++t) {
      double2 v = part[((int64_t)t * MV_RHS + r) * 2 * N + row];
      s.x += v.x;
      s.y += v.y;
    }
    y[r * 2 * N + row] = s;
  }
}

static int grid_for(int64_t blocks) {
  const int64_t cap = (int64_t)wsbm_sm_count() * 16;
  return (int)(blocks < 1 ? 1 : (blocks < cap ? blocks : cap));
}

int wsbm_phys_from_params(const wsbm_params* p, Phys* ph);
int wsbm_geom_check(const wsbm_geom* g);
DevGeom wsbm_devgeom(const wsbm_geom* g);

extern "C" int wsbm_matvec(const wsbm_geom* g, const wsbm_params* p, int32_t trans, const void* x,
                           int32_t nrhs, void* y, void* stream) {
  int rc = wsbm_geom_check(g);
  if (rc) return rc;
  Phys ph;
  if ((rc = wsbm_phys_from_params(p, &ph))) return rc;
  if (p->formulation != WSBM_FORM_WSBM) return WSBM_ERR_INVALID_ARG;  // eq. (weakly_bm) only
  if ((trans != 0 && trans != 1) || nrhs < 0 || (nrhs > 0 && (!x || !y))) return WSBM_ERR_INVALID_ARG;
  if (nrhs == 0) return WSBM_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t N = g->n;
  const int64_t nti = (N + MV_THREADS - 1) / MV_THREADS;
  int nsm = wsbm_sm_count(), per_sm = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_matvec<false>, MV_THREADS, 0) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  int64_t want = (int64_t)nsm * per_sm * 8;  // about eight waves
  int64_t nsplit = (want + nti - 1) / nti;
  if (nsplit < 1) nsplit = 1;
  if (nsplit > nti) nsplit = nti;
  const int64_t jspan = (N + nsplit - 1) / nsplit;
  nsplit = (N + jspan - 1) / jspan;
  WsbmScratch scr(st);
  double2* part = nullptr;
  if ((rc = scr.get((size_t)nsplit * MV_RHS * 2 * N * sizeof(double2), (void**)&part))) return rc;
  DevGeom dg = wsbm_devgeom(g);
  for (int c = 0; c < nrhs && rc == WSBM_OK; c += MV_RHS) {
    const int nr = nrhs - c < MV_RHS ? nrhs - c : MV_RHS;
    const double2* xc = (const double2*)x + (int64_t)c * 2 * N;
    if (trans)
      k_matvec<true><<<dim3((unsigned)nti, (unsigned)nsplit), MV_THREADS, 0, st>>>(dg, ph, xc, nr, jspan, part);
    else
      k_matvec<false><<<dim3((unsigned)nti, (unsigned)nsplit), MV_THREADS, 0, st>>>(dg, ph, xc, nr, jspan, part);
    wsbm_count_launch();
    int64_t blocks = (2 * N * nr + 255) / 256;
    k_matvec_reduce<<<grid_for(blocks), 256, 0, st>>>(N, (int)nsplit, nr, part,
                                                     (double2*)y + (int64_t)c * 2 * N);
    wsbm_count_launch();
    if (cudaGetLastError() != cudaSuccess) rc = WSBM_ERR_CUDA;
  }
  return rc;
}
