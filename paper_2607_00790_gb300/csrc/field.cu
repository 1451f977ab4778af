// Field off the curve from the boundary densities by the integral representations (Sec. II:
// once u and q are known on the curve, the solution in each domain follows from them):
//   exterior x:  u_sc(x) = D_k0[u](x) - eps0 S_k0[q](x)      (scattered part)
//   interior x:  u(x)    = eps1 S_k1[q](x) - D_k1[u](x)      (total field)
// S_k[f](x) = sum_j w_j (i/4) H0(k r) f_j,  D_k[f](x) = sum_j w_j (ik/4) H1(k r) (d.n_j)/r f_j,
// d = x - y_j.  The side of x comes from the Laplace double layer of the unit density (Gauss:
// -sum_j w_j (d.n_j)/(2 pi r^2) is 1 inside, 0 outside, up to the quadrature error near the
// curve).  The trapezoidal sums are accurate a few node spacings away from the curve; closer
// targets need a near-singular quadrature, which the paper does not describe.
#include <math.h>

#include <algorithm>

#include "hankel.cuh"
#include "wsbm_internal.h"

namespace {

#define FLD_THREADS 128
#define FLD_RHS 4  // right-hand sides per launch (Hankel values shared by all of them)

struct FldSlot {
  double x, y, nx, ny, w, pad;
};

// side[t] = 1 inside, 0 outside (one thread per target, all sources)
__global__ void k_field_side(DevGeom g, const double* __restrict__ tx, const double* __restrict__ ty,
                             int64_t nt, int8_t* __restrict__ side) {
  __shared__ FldSlot sj[FLD_THREADS];
  const int64_t t = (int64_t)blockIdx.x * FLD_THREADS + threadIdx.x;
  const double px = t < nt ? tx[t] : 0.0, py = t < nt ? ty[t] : 0.0;
  double acc = 0.0;
  for (int64_t jc = 0; jc < g.n; jc += FLD_THREADS) {
    __syncthreads();
    int64_t j = jc + threadIdx.x;
    if (j < g.n) {
      sj[threadIdx.x].x = g.x[j];
      sj[threadIdx.x].y = g.y[j];
      sj[threadIdx.x].nx = g.nx[j];
      sj[threadIdx.x].ny = g.ny[j];
      sj[threadIdx.x].w = g.w[j];
    }
    __syncthreads();
    const int nj = (int)min((int64_t)FLD_THREADS, g.n - jc);
    for (int jj = 0; jj < nj; ++jj) {
      const FldSlot& s = sj[jj];
      const double dx = px - s.x, dy = py - s.y;
      const double r2 = dx * dx + dy * dy;
      if (r2 > 0.0) acc += s.w * (dx * s.nx + dy * s.ny) / r2;
    }
  }
  if (t < nt) side[t] = (-acc / (2.0 * WSBM_PI)) > 0.5 ? 1 : 0;
}

// Partial sums over the sources [j0, j1) of CTA row blockIdx.y, for FLD_RHS right-hand sides
// starting at column c0.  part: nsplit x nt x FLD_RHS complex128.
__global__ void __launch_bounds__(FLD_THREADS)
    k_field(DevGeom g, Phys ph, const double2* __restrict__ u, const double2* __restrict__ q, int nrhs,
            int c0, const double* __restrict__ tx, const double* __restrict__ ty, int64_t nt,
            const int8_t* __restrict__ side, int64_t jspan, double2* __restrict__ part) {
  __shared__ HkTables T;
  __shared__ FldSlot sj[FLD_THREADS];
  __shared__ double2 su[FLD_RHS][FLD_THREADS], sq[FLD_RHS][FLD_THREADS];
  hk_stage_tables(&T);
  const int64_t N = g.n;
  const int64_t t = (int64_t)blockIdx.x * FLD_THREADS + threadIdx.x;
  const int64_t j0 = (int64_t)blockIdx.y * jspan, j1 = min(N, j0 + jspan);
  const bool valid = t < nt;
  const double px = valid ? tx[t] : 0.0, py = valid ? ty[t] : 0.0;
  const bool in = valid && side[t] != 0;
  const double k = in ? ph.k1 : ph.k0;
  const int nc = min(FLD_RHS, nrhs - c0);
  double2 acc[FLD_RHS];
#pragma unroll
  for (int c = 0; c < FLD_RHS; ++c) acc[c] = make_double2(0.0, 0.0);
  for (int64_t jc = j0; jc < j1; jc += FLD_THREADS) {
    __syncthreads();
    {
      int64_t j = jc + threadIdx.x;
      if (j < j1) {
        FldSlot& s = sj[threadIdx.x];
        s.x = g.x[j];
        s.y = g.y[j];
        s.nx = g.nx[j];
        s.ny = g.ny[j];
        s.w = g.w[j];
#pragma unroll
        for (int c = 0; c < FLD_RHS; ++c) {
          su[c][threadIdx.x] = c < nc ? u[(int64_t)(c0 + c) * N + j] : make_double2(0.0, 0.0);
          sq[c][threadIdx.x] = c < nc ? q[(int64_t)(c0 + c) * N + j] : make_double2(0.0, 0.0);
        }
      }
    }
    __syncthreads();
    if (!valid) continue;
    const int nj = (int)min((int64_t)FLD_THREADS, j1 - jc);
#pragma unroll 1
    for (int jj = 0; jj < nj; ++jj) {
      // keep the Hankel tables in shared memory: no hoisting of their loads out of the loop
      asm volatile("" ::: "memory");
      const FldSlot& s = sj[jj];
      const double dx = px - s.x, dy = py - s.y;
      const double r2 = fma(dx, dx, dy * dy);
      if (r2 == 0.0) continue;
      const double rs = rsqrt(r2);  // 1/r
      const double r = r2 * rs;
      const double z = k * r;
      Hk h;
      hankel_fp64_rs<false>(T, z, rsqrt(z), h);
      // w G = (i w/4) H0;  w dG/dn_y = (i k w/4) H1 (d.n)/r
      const double sg = 0.25 * s.w, sd = 0.25 * s.w * k * (dx * s.nx + dy * s.ny) * rs;
      const double2 G = make_double2(-sg * h.h0i, sg * h.h0r);
      const double2 D = make_double2(-sd * h.h1i, sd * h.h1r);
      const double ea = in ? ph.eps1 : -ph.eps0;  // coefficient of S[q]
      const double eb = in ? -1.0 : 1.0;          // coefficient of D[u]
#pragma unroll
      for (int c = 0; c < FLD_RHS; ++c) {
        const double2 uu = su[c][jj], qq = sq[c][jj];
        acc[c].x += ea * (G.x * qq.x - G.y * qq.y) + eb * (D.x * uu.x - D.y * uu.y);
        acc[c].y += ea * (G.x * qq.y + G.y * qq.x) + eb * (D.x * uu.y + D.y * uu.x);
      }
    }
  }
  if (valid) {
#pragma unroll
    for (int c = 0; c < FLD_RHS; ++c)
      part[((int64_t)blockIdx.y * nt + t) * FLD_RHS + c] = acc[c];
  }
}

__global__ void k_field_reduce(int64_t nt, int nsplit, int nrhs, int c0,
                               const double2* __restrict__ part, double2* __restrict__ out) {
  const int nc = min(FLD_RHS, nrhs - c0);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nt * nc;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = e / nc;
    const int c = (int)(e % nc);
    double2 s = make_double2(0.0, 0.0);
    for (int p = 0; p < nsplit; ++p) {
      double2 v = part[((int64_t)p * nt + t) * FLD_RHS + c];
      s.x += v.x;
      s.y += v.y;
    }
    out[(int64_t)(c0 + c) * nt + t] = s;
  }
}

int grid_cap(int64_t blocks) {
  const int64_t cap = (int64_t)wsbm_sm_count() * 16;
  return (int)(blocks < 1 ? 1 : (blocks < cap ? blocks : cap));
}

}  // namespace

int wsbm_phys_from_params(const wsbm_params* p, Phys* ph);
int wsbm_geom_check(const wsbm_geom* g);
DevGeom wsbm_devgeom(const wsbm_geom* g);

extern "C" int wsbm_field(const wsbm_geom* g, const wsbm_params* p, const void* u, const void* q,
                          int32_t nrhs, const double* tx, const double* ty, int64_t nt, void* out,
                          int8_t* inside, void* stream) {
  int rc = wsbm_geom_check(g);
  if (rc) return rc;
  Phys ph;
  if ((rc = wsbm_phys_from_params(p, &ph))) return rc;
  if (nrhs < 1 || nt < 0 || !u || !q || (nt > 0 && (!tx || !ty || !out || !inside)))
    return WSBM_ERR_INVALID_ARG;
  if (nt == 0) return WSBM_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t N = g->n;
  const int64_t nti = (nt + FLD_THREADS - 1) / FLD_THREADS;
  int nsm = wsbm_sm_count(), per_sm = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_field, FLD_THREADS, 0) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  int64_t want = (int64_t)nsm * per_sm * 8;  // about eight waves, at least 128 sources a CTA
  int64_t nsplit = std::max<int64_t>(1, std::min<int64_t>((want + nti - 1) / nti, (N + 127) / 128));
  const int64_t jspan = (N + nsplit - 1) / nsplit;
  nsplit = (N + jspan - 1) / jspan;
  WsbmScratch scr(st);
  double2* part = nullptr;
  if ((rc = scr.get((size_t)nsplit * nt * FLD_RHS * sizeof(double2), (void**)&part))) return rc;
  DevGeom dg = wsbm_devgeom(g);
  k_field_side<<<(unsigned)nti, FLD_THREADS, 0, st>>>(dg, tx, ty, nt, inside);
  wsbm_count_launch();
  for (int c0 = 0; c0 < nrhs; c0 += FLD_RHS) {
    k_field<<<dim3((unsigned)nti, (unsigned)nsplit), FLD_THREADS, 0, st>>>(
        dg, ph, (const double2*)u, (const double2*)q, nrhs, c0, tx, ty, nt, inside, jspan, part);
    wsbm_count_launch();
    k_field_reduce<<<grid_cap((nt * FLD_RHS + 255) / 256), 256, 0, st>>>(nt, (int)nsplit, nrhs, c0,
                                                                         part, (double2*)out);
    wsbm_count_launch();
  }
  rc = cudaGetLastError() == cudaSuccess ? WSBM_OK : WSBM_ERR_CUDA;
  return rc;
}
