// Entries of the two formulations the paper compares the WSBM equation with (Sec. II): the
// standard Burton-Miller equation (eq. bm) and the PMCHWT equation (eq. pmchwt, stored with its
// columns in the order (u, q) like the other two), for the same node-pair and proxy tasks as
// the WSBM kernels.  Both contain the hypersingular N_k alone:
//   N_k = (i k^2/4)[H0(kr) c + F1(kr)(n_x.n_y - 2c)] + (n_x.n_y - 2c)/(2 pi r^2),
// with F1(z) = H1(z)/z + 2i/(pi z^2) from the Hankel evaluator and the k-independent
// 1/r^2 part written out.  Its one-point corrected diagonal adds -pi/(6 w_i) for the 1/r^2
// part to the log correction of the k-dependent part; the O(1) curvature term is left out, so
// these formulations converge at first order, as the paper reports.
//
// The kernels here are plain (one pair per thread over the same 32 x 4 tiles, no grouping by
// evaluation path): the formulations are the paper's comparison, the tuned kernels serve the
// WSBM system.
#include <math.h>

#include "entry_blocks.cuh"

namespace {

struct FSlot {
  double x, y, nx, ny, w, kap;
  int32_t node, p0, p1;
};

__device__ __forceinline__ int form_find_task(const int32_t* tile0s, int stride, int ntasks,
                                              int64_t tile) {
  int lo = 0, hi = ntasks - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if ((int64_t)tile0s[(int64_t)mid * stride] <= tile)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ void form_load(const DevGeom& g, const int32_t* nodes, const int32_t* pos,
                                          int t, FSlot& s) {
  const int32_t nd = nodes[t];
  s.node = nd;
  s.x = g.x[nd];
  s.y = g.y[nd];
  s.nx = g.nx[nd];
  s.ny = g.ny[nd];
  s.w = g.w[nd];
  s.kap = g.kappa[nd];
  s.p0 = pos[2 * t];
  s.p1 = pos[2 * t + 1];
}

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cscale(double s, double2 a) { return make_double2(s * a.x, s * a.y); }
// (i/k0) a
__device__ __forceinline__ double2 times_alpha(double inv_k0, double2 a) {
  return make_double2(-a.y * inv_k0, a.x * inv_k0);
}

// The four layer operators at one wavenumber for an off-diagonal pair, weight w_j folded in.
struct Ops1 {
  double2 S, D, Dx, N;
};

__device__ __forceinline__ void ops_offdiag(const Hk& h, double k, const PairGeom& G, double wj,
                                            Ops1& o) {
  const double q = 0.25 * wj;
  o.S = make_double2(-q * h.h0i, q * h.h0r);                 // (i/4) H0
  const double a = q * k * G.dny * G.ir;                     // D: (ik/4) H1 (d.n_y)/r
  o.D = make_double2(-a * h.h1i, a * h.h1r);
  const double b = -q * k * G.dnx * G.ir;                    // D*: -(ik/4) H1 (d.n_x)/r
  o.Dx = make_double2(-b * h.h1i, b * h.h1r);
  const double m2c = G.nn - 2.0 * G.c;
  const double Xr = h.h0r * G.c + h.f1r * m2c, Xi = h.h0i * G.c + h.f1i * m2c;
  const double q2 = q * k * k;                               // (i k^2/4) X
  const double lap = wj * m2c * (G.ir * G.ir) / (2.0 * WSBM_PI);
  o.N = make_double2(-q2 * Xi + lap, q2 * Xr);
}

// The same on the diagonal (one-point corrected).
__device__ __forceinline__ void ops_diag(double k, double wi, double kap, Ops1& o) {
  const double L = log(k * wi / (4.0 * WSBM_PI));
  o.S = make_double2(-wi * (WSBM_EULER + L) / (2.0 * WSBM_PI), 0.25 * wi);
  const double Dd = -wi * kap / (4.0 * WSBM_PI);
  o.D = make_double2(Dd, 0.0);
  o.Dx = o.D;
  const double f = k * k * (L + WSBM_EULER - 0.5);
  o.N = make_double2(-wi * f / (4.0 * WSBM_PI) - WSBM_PI / (6.0 * wi), wi * k * k / 8.0);
}

// 2x2 block of form 1 (eq. bm) or 2 (eq. pmchwt) from the operators at k0 (o0) and k1 (o1);
// id = 1/2 on the diagonal (the jump terms of eq. bm), 0 off it.
__device__ __forceinline__ void form_block(int form, const Phys& ph, const Ops1& o0, const Ops1& o1,
                                           double id, double2 e[2][2]) {
  if (form == 1) {
    e[0][0] = make_double2(o1.D.x + id, o1.D.y);
    e[0][1] = cscale(-ph.eps1, o1.S);
    const double2 aN = times_alpha(ph.inv_k0, o0.N);
    e[1][0] = make_double2(o0.D.x - id + aN.x, o0.D.y + aN.y);
    const double2 aD = times_alpha(ph.inv_k0, make_double2(o0.Dx.x + id, o0.Dx.y));
    e[1][1] = cscale(-ph.eps0, cadd(o0.S, aD));
  } else {
    e[0][0] = cadd(o0.D, o1.D);
    e[0][1] = cadd(cscale(-ph.eps0, o0.S), cscale(-ph.eps1, o1.S));
    e[1][0] = cadd(cscale(1.0 / ph.eps0, o0.N), cscale(1.0 / ph.eps1, o1.N));
    e[1][1] = cscale(-1.0, cadd(o0.Dx, o1.Dx));
  }
}

__global__ void __launch_bounds__(WSBM_PAIR_THREADS)
    k_pairs_form(int form, DevGeom g0, Phys ph0, const PairTask* __restrict__ tasks, int ntasks,
                 int64_t ntiles, const DevGeom* __restrict__ geos, const Phys* __restrict__ phys) {
  __shared__ HkTables T;
  __shared__ FSlot sf[WSBM_TILE_F];
  __shared__ FSlot ss[WSBM_TILE_S];
  hk_stage_tables(&T);
  const int tx = threadIdx.x & (WSBM_TILE_F - 1);
  const int ty = threadIdx.x / WSBM_TILE_F;
  const int stride = sizeof(PairTask) / sizeof(int32_t);
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int ti = form_find_task(&tasks[0].tile0, stride, ntasks, tile);
    const PairTask tk = tasks[ti];
    const DevGeom g = geos ? geos[tk.inst] : g0;
    const Phys ph = phys ? phys[tk.inst] : ph0;
    const bool fc = tk.fastc != 0;
    const int nf = fc ? tk.nc : tk.nr;
    const int ns = fc ? tk.nr : tk.nc;
    const int nft = (nf + WSBM_TILE_F - 1) / WSBM_TILE_F;
    const int64_t lt = tile - tk.tile0;
    const int f0 = (int)(lt % nft) * WSBM_TILE_F;
    const int s0 = (int)(lt / nft) * WSBM_TILE_S;
    __syncthreads();  // previous tile done with the staged slots (and tables staged)
    if (threadIdx.x < WSBM_TILE_F) {
      const int f = f0 + threadIdx.x;
      if (f < nf) {
        if (fc)
          form_load(g, tk.cnode, tk.cpos, f, sf[threadIdx.x]);
        else
          form_load(g, tk.rnode, tk.rpos, f, sf[threadIdx.x]);
      }
    } else if (threadIdx.x < WSBM_TILE_F + WSBM_TILE_S) {
      const int k = threadIdx.x - WSBM_TILE_F;
      const int s = s0 + k;
      if (s < ns) {
        if (fc)
          form_load(g, tk.rnode, tk.rpos, s, ss[k]);
        else
          form_load(g, tk.cnode, tk.cpos, s, ss[k]);
      }
    }
    __syncthreads();
    const int f = f0 + tx, s = s0 + ty;
    if (f < nf && s < ns) {
      const FSlot& R = fc ? ss[ty] : sf[tx];
      const FSlot& C = fc ? sf[tx] : ss[ty];
      Ops1 o0, o1;
      double id = 0.0;
      if (R.node == C.node) {
        ops_diag(ph.k0, R.w, R.kap, o0);
        ops_diag(ph.k1, R.w, R.kap, o1);
        id = 0.5;
      } else {
        PairGeom G;
        pair_geom(R.x, R.y, R.nx, R.ny, C.x, C.y, C.nx, C.ny, ph, G);
        Hk a, b;
        hankel_fp64_rs<true>(T, G.z0, G.rs0, a);
        hankel_fp64_rs<true>(T, G.z1, G.rs1, b);
        ops_offdiag(a, ph.k0, G, C.w, o0);
        ops_offdiag(b, ph.k1, G, C.w, o1);
      }
      double2 e[2][2];
      form_block(form, ph, o0, o1, id, e);
      const int rp[2] = {R.p0, R.p1};
      const int cp[2] = {C.p0, C.p1};
#pragma unroll
      for (int bb = 0; bb < 2; ++bb)
#pragma unroll
        for (int aa = 0; aa < 2; ++aa)
          if (rp[aa] >= 0 && cp[bb] >= 0) {
            const int64_t off = tk.trans ? ((int64_t)cp[bb] + (int64_t)rp[aa] * tk.ld)
                                         : ((int64_t)rp[aa] + (int64_t)cp[bb] * tk.ld);
            tk.out[off] = e[aa][bb];
          }
    }
  }
}

// Proxy row block (sources on the proxy circle acting on a box's equations), FP64.  With the
// combined-field source Phi_k = dG/dnu_p - i k G and dPhi_k its n_x-derivative:
//   form 1 (eq. bm):     k1 source [Phi1 ; 0],                 k0 source [0 ; Phi0 + alpha dPhi0]
//   form 2 (eq. pmchwt): k1 source [Phi1 ; dPhi1 / eps1],      k0 source [Phi0 ; dPhi0 / eps0]
// Column blocks (the box unknowns' potentials at the proxy points) are the same for every
// formulation and come from the WSBM proxy kernel.
__global__ void __launch_bounds__(WSBM_PAIR_THREADS)
    k_proxy_rows_form(int form, DevGeom g0, Phys ph0, const ProxyTask* __restrict__ tasks,
                      int ntasks, int64_t ntiles, const DevGeom* __restrict__ geos,
                      const Phys* __restrict__ phys) {
  __shared__ HkTables T;
  __shared__ double spx[WSBM_TILE_F], spy[WSBM_TILE_F], snx[WSBM_TILE_F], sny[WSBM_TILE_F];
  __shared__ FSlot ss[WSBM_TILE_S];
  hk_stage_tables(&T);
  const int tx = threadIdx.x & (WSBM_TILE_F - 1);
  const int ty = threadIdx.x / WSBM_TILE_F;
  const int stride = sizeof(ProxyTask) / sizeof(int32_t);
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int ti = form_find_task(&tasks[0].tile0, stride, ntasks, tile);
    const ProxyTask tk = tasks[ti];
    const DevGeom g = geos ? geos[tk.inst] : g0;
    const Phys ph = phys ? phys[tk.inst] : ph0;
    const int nft = (tk.P + WSBM_TILE_F - 1) / WSBM_TILE_F;
    const int64_t lt = tile - tk.tile0;
    const int m0 = (int)(lt % nft) * WSBM_TILE_F;
    const int s0 = (int)(lt / nft) * WSBM_TILE_S;
    __syncthreads();
    if (threadIdx.x < WSBM_TILE_F) {
      const int m = m0 + threadIdx.x;
      if (m < tk.P) {
        double sn, cs;
        sincospi(2.0 * (double)m / (double)tk.P, &sn, &cs);
        snx[threadIdx.x] = cs;
        sny[threadIdx.x] = sn;
        spx[threadIdx.x] = tk.cx + tk.rho * cs;
        spy[threadIdx.x] = tk.cy + tk.rho * sn;
      }
    } else if (threadIdx.x < WSBM_TILE_F + WSBM_TILE_S) {
      const int k = threadIdx.x - WSBM_TILE_F;
      if (s0 + k < tk.nn) form_load(g, tk.node, tk.pos, s0 + k, ss[k]);
    }
    __syncthreads();
    const int m = m0 + tx, s = s0 + ty;
    if (m < tk.P && s < tk.nn) {
      const FSlot& X = ss[ty];
      const double pw = 2.0 * WSBM_PI * tk.rho / (double)tk.P;
      const double dx = X.x - spx[tx], dy = X.y - spy[tx];
      const double r = sqrt(dx * dx + dy * dy);
      const double ir = 1.0 / r;
      const double dnu = (dx * snx[tx] + dy * sny[tx]) * ir;  // (d . nu_p) / r
      const double dnx = (dx * X.nx + dy * X.ny) * ir;        // (d . n_x) / r
      const double nn = X.nx * snx[tx] + X.ny * sny[tx];
      const double c = dnx * dnu;
      double2 phi[2], dphi[2];  // 0: k1, 1: k0
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        const double k = t == 0 ? ph.k1 : ph.k0;
        const double z = k * r;
        Hk h;
        hankel_fp64_rs<false>(T, z, rsqrt(z), h);
        // Phi = (ik/4) H1 dnu - i k (i/4) H0 = (ik/4) H1 dnu + (k/4) H0
        const double q = 0.25 * k;
        phi[t] = make_double2(q * (-h.h1i * dnu + h.h0r), q * (h.h1r * dnu + h.h0i));
        // dPhi = N_k(x, p) - i k dG/dn_x,  dG/dn_x = -(ik/4) H1 dnx
        //      = (i k^2/4)[H0 c + (H1/z)(nn - 2c)] - (k^2/4) H1 dnx
        const double q2 = 0.25 * k * k;
        const double m2c = nn - 2.0 * c;
        const double iz = 1.0 / z;
        const double Xr = h.h0r * c + h.h1r * iz * m2c, Xi = h.h0i * c + h.h1i * iz * m2c;
        dphi[t] = make_double2(q2 * (-Xi - h.h1r * dnx), q2 * (Xr - h.h1i * dnx));
      }
      double2 o[2][2];  // o[s][a]: source s (0: k1, 1: k0), equation a
      if (form == 1) {
        o[0][0] = cscale(pw, phi[0]);
        o[0][1] = make_double2(0.0, 0.0);
        o[1][0] = make_double2(0.0, 0.0);
        o[1][1] = cscale(pw, cadd(phi[1], times_alpha(ph.inv_k0, dphi[1])));
      } else {
        o[0][0] = cscale(pw, phi[0]);
        o[0][1] = cscale(pw / ph.eps1, dphi[0]);
        o[1][0] = cscale(pw, phi[1]);
        o[1][1] = cscale(pw / ph.eps0, dphi[1]);
      }
      const int bp[2] = {X.p0, X.p1};
#pragma unroll
      for (int sg = 0; sg < 2; ++sg) {
        const int64_t prow = (int64_t)tk.off + (int64_t)sg * tk.P + m;
#pragma unroll
        for (int a = 0; a < 2; ++a)
          if (bp[a] >= 0) {
            const int64_t off = tk.tr ? ((int64_t)bp[a] + prow * tk.ld) : (prow + (int64_t)bp[a] * tk.ld);
            tk.out[off] = o[sg][a];
          }
      }
    }
  }
}

int form_grid(int64_t ntiles) {
  const int64_t cap = (int64_t)wsbm_sm_count() * 16;
  return (int)(ntiles < cap ? ntiles : cap);
}

}  // namespace

int wsbm_launch_pairs_form(int form, const DevGeom& g, const Phys& ph, const PairTask* d_tasks,
                           int ntasks, int64_t ntiles, cudaStream_t st, const DevGeom* geos,
                           const Phys* phys) {
  if (form != 1 && form != 2) return WSBM_ERR_INVALID_ARG;
  if (ntiles <= 0) return WSBM_OK;
  k_pairs_form<<<form_grid(ntiles), WSBM_PAIR_THREADS, 0, st>>>(form, g, ph, d_tasks, ntasks, ntiles,
                                                                 geos, phys);
  wsbm_count_launch();
  return cudaGetLastError() == cudaSuccess ? WSBM_OK : WSBM_ERR_CUDA;
}

int wsbm_launch_proxy_rows_form(int form, const DevGeom& g, const Phys& ph, const ProxyTask* d_tasks,
                                int ntasks, int64_t ntiles, cudaStream_t st, const DevGeom* geos,
                                const Phys* phys) {
  if (form != 1 && form != 2) return WSBM_ERR_INVALID_ARG;
  if (ntiles <= 0) return WSBM_OK;
  k_proxy_rows_form<<<form_grid(ntiles), WSBM_PAIR_THREADS, 0, st>>>(form, g, ph, d_tasks, ntasks,
                                                                      ntiles, geos, phys);
  wsbm_count_launch();
  return cudaGetLastError() == cudaSuccess ? WSBM_OK : WSBM_ERR_CUDA;
}
