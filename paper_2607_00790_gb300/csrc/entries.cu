// Entry generation for the WSBM Nystrom matrix (eq. weakly_bm; block form A_ij of Sec. III)
// and for the proxy-circle blocks of the proxy-surface method (Sec. III).
//
// Work unit: one node pair (or node / proxy-point pair).  It evaluates H0, H1 at z0 = k0 r and
// z1 = k1 r once and writes all entries of its 2x2 block, so every unit costs the same (the
// paper balances threads the same way: each block A_ij carries the same seven layer-potential
// terms).  A CTA stages the node data of a 32 x 4 tile in shared memory; the 32 slots of the
// fast dimension normally map to consecutive output rows, so a warp's complex128 stores are
// contiguous; for short-by-long blocks the longer list takes the fast dimension instead (the
// kernels are FP64-bound, so fewer idle lanes beat coalesced stores).
// Launches are grid-stride over a flat tile list spanning many blocks (all boxes of a tree
// level in one launch).
#include <math.h>

#include "entry_blocks.cuh"

struct SlotData {
  double x, y, nx, ny, w, kap;
  float fnx, fny, fw;  // FP32 copies for the mixed-precision algebra
  int32_t node, p0, p1;
};

__device__ __forceinline__ int find_task_by_tile(const int32_t* tile0s, int stride, int ntasks,
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

__device__ __forceinline__ void load_slot(const DevGeom& g, const int32_t* nodes,
                                          const int32_t* pos, int t, SlotData& s) {
  int32_t nd = nodes[t];
  s.node = nd;
  s.x = g.x[nd];
  s.y = g.y[nd];
  s.nx = g.nx[nd];
  s.ny = g.ny[nd];
  s.w = g.w[nd];
  s.kap = g.kappa[nd];
  s.fnx = (float)s.nx;
  s.fny = (float)s.ny;
  s.fw = (float)s.w;
  s.p0 = pos[2 * t];
  s.p1 = pos[2 * t + 1];
}

// TF slots along the fast (contiguous-output) dimension x TS = WSBM_PAIR_THREADS / TF along the
// other (TF a power of two, 16..64).
template <int TF>
__global__ void __launch_bounds__(WSBM_PAIR_THREADS)
    k_pairs(DevGeom g0, Phys ph0, const PairTask* __restrict__ tasks, int ntasks, int64_t ntiles,
            const DevGeom* __restrict__ geos, const Phys* __restrict__ phys) {
  constexpr int TS = WSBM_PAIR_THREADS / TF;
  __shared__ HkTables T;
  __shared__ SlotData sf[TF];
  __shared__ SlotData ss[TS];
  __shared__ int s_cnt[WSBM_PAIR_THREADS / 32][3];
  __shared__ int16_t s_list[WSBM_PAIR_THREADS];
  __shared__ int s_ntot;
  hk_stage_tables(&T);
  const int tx = threadIdx.x & (TF - 1);
  const int ty = threadIdx.x / TF;
  const int stride = sizeof(PairTask) / sizeof(int32_t);
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    int ti = find_task_by_tile(&tasks[0].tile0, stride, ntasks, tile);
    const PairTask tk = tasks[ti];
    const DevGeom g = geos ? geos[tk.inst] : g0;
    const Phys ph = phys ? phys[tk.inst] : ph0;
    const bool fc = tk.fastc != 0;
    const int nf = fc ? tk.nc : tk.nr;
    const int ns = fc ? tk.nr : tk.nc;
    const int nft = (nf + TF - 1) / TF;
    const int64_t lt = tile - tk.tile0;
    const int f0 = (int)(lt % nft) * TF;
    const int s0 = (int)(lt / nft) * TS;
    __syncthreads();  // previous tile done with the staged slots (and tables staged)
    if (threadIdx.x < TF) {
      int f = f0 + threadIdx.x;
      if (f < nf) {
        if (fc)
          load_slot(g, tk.cnode, tk.cpos, f, sf[threadIdx.x]);
        else
          load_slot(g, tk.rnode, tk.rpos, f, sf[threadIdx.x]);
      }
    } else if (threadIdx.x < TF + TS) {
      int k = threadIdx.x - TF;
      int s = s0 + k;
      if (s < ns) {
        if (fc)
          load_slot(g, tk.rnode, tk.rpos, s, ss[k]);
        else
          load_slot(g, tk.cnode, tk.cpos, s, ss[k]);
      }
    }
    __syncthreads();
    // Group the tile's pairs by evaluation path before evaluating them: far pairs (both
    // Hankel arguments on the large-argument branch), near pairs (at least one ascending
    // series) and diagonal pairs (one-point correction).  Threads then take pairs from the
    // grouped list, so a warp mixes paths only at a group boundary instead of wherever the
    // diagonal band crosses the tile.  (The grouping only orders work; any pair may be
    // evaluated by any thread.)
    int cls = 3;  // 3: outside the task
    {
      const int f = f0 + tx, s = s0 + ty;
      if (f < nf && s < ns) {
        const SlotData& R = fc ? ss[ty] : sf[tx];
        const SlotData& C = fc ? sf[tx] : ss[ty];
        if (R.node == C.node) {
          cls = 2;
        } else {
          // near: min(k0, k1) r < HK_Z_SERIES, compared on r^2 (no square root)
          const double dx = R.x - C.x, dy = R.y - C.y;
          const double rz = HK_Z_SERIES * fmax(ph.inv_k0, ph.inv_k1);
          cls = fma(dx, dx, dy * dy) < rz * rz ? 1 : 0;
        }
      }
    }
    {
      const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
      const unsigned lt = (1u << lane) - 1u;
      unsigned bal[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        bal[c] = __ballot_sync(0xffffffffu, cls == c);
        if (lane == 0) s_cnt[warp][c] = __popc(bal[c]);
      }
      __syncthreads();
      int base = 0, pos = -1;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        int before = 0, total = 0;
#pragma unroll
        for (int w = 0; w < WSBM_PAIR_THREADS / 32; ++w) {
          total += s_cnt[w][c];
          if (w < warp) before += s_cnt[w][c];
        }
        if (cls == c) pos = base + before + __popc(bal[c] & lt);
        base += total;
      }
      if (pos >= 0) s_list[pos] = (int16_t)threadIdx.x;
      if (threadIdx.x == 0) s_ntot = base;
    }
    __syncthreads();
    if ((int)threadIdx.x < s_ntot) {
      const int me = s_list[threadIdx.x];
      const int mx = me & (TF - 1), my = me / TF;
      const SlotData& R = fc ? ss[my] : sf[mx];
      const SlotData& C = fc ? sf[mx] : ss[my];
      double2 e[2][2];
      if (R.node == C.node) {
        block_diag(ph, R.w, R.kap, e);
      } else {
        PairGeom G;
        pair_geom(R.x, R.y, R.nx, R.ny, C.x, C.y, C.nx, C.ny, ph, G);
        block_offdiag(T, ph, G, C.w, e);
      }
      const int rp[2] = {R.p0, R.p1};
      const int cp[2] = {C.p0, C.p1};
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int a = 0; a < 2; ++a) {
          if (rp[a] >= 0 && cp[b] >= 0) {
            int64_t off = tk.trans ? ((int64_t)cp[b] + (int64_t)rp[a] * tk.ld)
                                   : ((int64_t)rp[a] + (int64_t)cp[b] * tk.ld);
            tk.out[off] = e[a][b];
          }
        }
    }
  }
}

// --------------------------------------------------------------------- proxy blocks ----
struct ProxyPt {
  double px, py, pnx, pny;
  float fpnx, fpny;
};

// Sources on the proxy circle acting on equations at node x (row side).  Combined-field
// source Phi_k = dG/dnu_p - i k G;  out[s][a]: source s (0: k1, 1: k0), equation a.
//   s = k1: [Phi1 ; -alpha d_nx Phi1]     s = k0: [0 ; Phi0 + alpha d_nx Phi0]
template <bool PQ32>
__device__ __forceinline__ void proxy_row_fp64(const HkTables& T, const Phys& ph, const SlotData& X,
                                               const ProxyPt& p, double pw, double2 o[2][2]) {
  double dx = X.x - p.px, dy = X.y - p.py;
  double r2 = dx * dx + dy * dy;
  double r = sqrt(r2);
  double z1 = ph.k1 * r;
  double rs1 = rsqrt(z1);
  double ir = ph.k1 * (rs1 * rs1);
  double dnu = (dx * p.pnx + dy * p.pny) * ir;
  double dnx = (dx * X.nx + dy * X.ny) * ir;
  double nn = X.nx * p.pnx + X.ny * p.pny;
  double c = dnx * dnu;
  double inv_k0 = ph.inv_k0;
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    double k = s == 0 ? ph.k1 : ph.k0;
    double ik = s == 0 ? ph.inv_k1 : ph.inv_k0;
    Hk h;
    if (s == 0)
      hankel_fp64_rs<false, PQ32>(T, z1, rs1, h);
    else
      hankel_fp64_rs<false, PQ32>(T, ph.k0 * r, rs1 * ph.s10, h);
    // phi = (ik/4) H1 dnu + (k/4) H0
    double q = 0.25 * k;
    double phr = q * (-h.h1i * dnu + h.h0r), phi = q * (h.h1r * dnu + h.h0i);
    // dphi = N_k - (k^2/4) H1 dnx,  N_k = (i k^2/4)[H0 c + H1/(kr) (nn - 2c)]
    double q2 = 0.25 * k * k;
    double izr = ir * ik;
    double m2c = nn - 2.0 * c;
    double Xr = h.h0r * c + h.h1r * izr * m2c, Xi = h.h0i * c + h.h1i * izr * m2c;
    double dpr = q2 * (-Xi - h.h1r * dnx), dpi = q2 * (Xr - h.h1i * dnx);
    // alpha * dphi = (i/k0)(dpr + i dpi) = (-dpi/k0, dpr/k0)
    double adr = -dpi * inv_k0, adi = dpr * inv_k0;
    if (s == 0) {
      o[0][0] = make_double2(pw * phr, pw * phi);
      o[0][1] = make_double2(-pw * adr, -pw * adi);
    } else {
      o[1][0] = make_double2(0.0, 0.0);
      o[1][1] = make_double2(pw * (phr + adr), pw * (phi + adi));
    }
  }
}

// Fields of the box unknowns at a proxy point (column side).  out[s][b]: field s (0: psi1,
// 1: psi0), unknown b:  u_j -> w_j (ik/4) H1 (d.n_y)/r,  q_j -> -eps_s w_j (i/4) H0.
template <bool PQ32>
__device__ __forceinline__ void proxy_col_fp64(const HkTables& T, const Phys& ph, const SlotData& Y,
                                               const ProxyPt& p, double2 o[2][2]) {
  double dx = p.px - Y.x, dy = p.py - Y.y;
  double r2 = dx * dx + dy * dy;
  double r = sqrt(r2);
  double z1 = ph.k1 * r;
  double rs1 = rsqrt(z1);
  double dny = (dx * Y.nx + dy * Y.ny) * (ph.k1 * (rs1 * rs1));
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    double k = s == 0 ? ph.k1 : ph.k0;
    double eps = s == 0 ? ph.eps1 : ph.eps0;
    Hk h;
    if (s == 0)
      hankel_fp64_rs<false, PQ32>(T, z1, rs1, h);
    else
      hankel_fp64_rs<false, PQ32>(T, ph.k0 * r, rs1 * ph.s10, h);
    double a = 0.25 * Y.w * k * dny;
    o[s][0] = make_double2(-a * h.h1i, a * h.h1r);
    double bq = -0.25 * eps * Y.w;
    o[s][1] = make_double2(-bq * h.h0i, bq * h.h0r);
  }
}

// Mixed precision versions: z = k r formed in FP64 and reduced mod 2 pi in FP64; amplitude and
// entry algebra in FP32.
// sqrt of r2 > 0 for the mixed path: FP64 reciprocal-square-root seed and one Newton step
// (relative error ~1e-13, far below the FP32 amplitude; no IEEE rounding needed there).
__device__ __forceinline__ double sqrt_mixed(double r2) {
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(r2));
  double h = 0.5 * r2;
  y = fma(y, fma(-h * y, y, 0.5), y);
  return r2 * y;
}

__device__ __forceinline__ void hankel_mixed(const HkTables& T, double z, float rsz, HkF& o) {
  if (__double2hiint(z) >= HK_SERIES_HI) {
    hankel_mixed_large(T, z, rsz, o);
  } else {
    Hk h;
    hankel_fp64(T, z, h);
    o.h0r = (float)h.h0r;
    o.h0i = (float)h.h0i;
    o.h1r = (float)h.h1r;
    o.h1i = (float)h.h1i;
  }
}

// Row side in mixed precision.  With H1 = -i H0 + D (D = H1 + i H0, small for large z) and
// 1 + d.nu/r = |d x nu|^2 / (r (r - d.nu)), the combined-field source and its normal
// derivative are written without the leading-order cancellation:
//   (4/k) Phi     = H0 (1 + dnu) + i dnu D
//   (4/k^2) dPhi  = dnx (i H0 (1 + dnu) - D) + i (H1/z)(n_x.nu - 2 dnx dnu)
// (dnu = d.nu/r, dnx = d.n_x/r).  d.nu and d x nu are formed in FP64.
__device__ __forceinline__ void proxy_row_mixed(const HkTables& T, const Phys& ph, const SlotData& X,
                                                const ProxyPt& p, double pw, double2 o[2][2]) {
  double dx = X.x - p.px, dy = X.y - p.py;
  double r = sqrt_mixed(fma(dx, dx, dy * dy));
  // directions in FP32 from the FP64 difference vector (d.nu and d x nu keep relative accuracy)
  float fdx = (float)dx, fdy = (float)dy, fr = (float)r;
  float ir = 1.0f / fr;
  float pnx = p.fpnx, pny = p.fpny;
  float dnu = (fdx * pnx + fdy * pny) * ir;
  float cr = (fdx * pny - fdy * pnx) * ir;
  float opd = cr * cr / (1.0f - dnu);  // 1 + dnu
  float dnx = (fdx * X.fnx + fdy * X.fny) * ir;
  float nn = X.fnx * pnx + X.fny * pny;
  float m2c = nn - 2.0f * dnx * dnu;
  float inv_k0 = ph.finv_k0;
  float fpw = (float)pw;
  float rsr = rsqrtf(fr);
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    double kd = s == 0 ? ph.k1 : ph.k0;
    float k = s == 0 ? ph.fk1 : ph.fk0;
    double z = kd * r;
    float rsz = rsr * (s == 0 ? ph.frk1 : ph.frk0);
    HkF h;
    float Dr, Di;
    if (__double2hiint(z) >= HK_SERIES_HI) {
      hankel_mixed_large(T, z, rsz, h, &Dr, &Di);
    } else {
      Hk hd;
      hankel_fp64(T, z, hd);
      h.h0r = (float)hd.h0r;
      h.h0i = (float)hd.h0i;
      h.h1r = (float)hd.h1r;
      h.h1i = (float)hd.h1i;
      Dr = (float)(hd.h1r - hd.h0i);
      Di = (float)(hd.h1i + hd.h0r);
    }
    float q = 0.25f * k;
    // (4/k) Phi = H0 opd + i dnu D
    float phr = q * (h.h0r * opd - dnu * Di), phi = q * (h.h0i * opd + dnu * Dr);
    // (4/k^2) dPhi = dnx (i H0 opd - D) + i (H1/z) m2c
    float izr = ir / k;
    float Br = -h.h0i * opd - Dr, Bi = h.h0r * opd - Di;
    float q2 = 0.25f * k * k;
    float dpr = q2 * (dnx * Br - h.h1i * izr * m2c), dpi = q2 * (dnx * Bi + h.h1r * izr * m2c);
    float adr = -dpi * inv_k0, adi = dpr * inv_k0;
    if (s == 0) {
      o[0][0] = make_double2(fpw * phr, fpw * phi);
      o[0][1] = make_double2(-fpw * adr, -fpw * adi);
    } else {
      o[1][0] = make_double2(0.0, 0.0);
      o[1][1] = make_double2(fpw * (phr + adr), fpw * (phi + adi));
    }
  }
}

__device__ __forceinline__ void proxy_col_mixed(const HkTables& T, const Phys& ph, const SlotData& Y,
                                                const ProxyPt& p, double2 o[2][2]) {
  double dx = p.px - Y.x, dy = p.py - Y.y;
  double r = sqrt_mixed(fma(dx, dx, dy * dy));
  float fr = (float)r;
  float dny = ((float)dx * Y.fnx + (float)dy * Y.fny) / fr;
  float w = Y.fw;
  float rsr = rsqrtf(fr);
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    double kd = s == 0 ? ph.k1 : ph.k0;
    float k = s == 0 ? ph.fk1 : ph.fk0;
    float eps = s == 0 ? ph.feps1 : ph.feps0;
    HkF h;
    hankel_mixed(T, kd * r, rsr * (s == 0 ? ph.frk1 : ph.frk0), h);
    float a = 0.25f * w * k * dny;
    o[s][0] = make_double2(-a * h.h1i, a * h.h1r);
    float bq = -0.25f * eps * w;
    o[s][1] = make_double2(-bq * h.h0i, bq * h.h0r);
  }
}

// MODE: WSBM_FP64, WSBM_MIXED or WSBM_MIXED_FINE
template <int MODE, int TF>
__global__ void __launch_bounds__(WSBM_PAIR_THREADS)
    k_proxy(DevGeom g0, Phys ph0, const ProxyTask* __restrict__ tasks, int ntasks, int64_t ntiles,
            const DevGeom* __restrict__ geos, const Phys* __restrict__ phys) {
  constexpr int TS = WSBM_PAIR_THREADS / TF;
  __shared__ HkTables T;
  __shared__ ProxyPt sp[TF];
  __shared__ SlotData ss[TS];
  hk_stage_tables(&T);
  const int tx = threadIdx.x & (TF - 1);
  const int ty = threadIdx.x / TF;
  const int stride = sizeof(ProxyTask) / sizeof(int32_t);
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    int ti = find_task_by_tile(&tasks[0].tile0, stride, ntasks, tile);
    const ProxyTask tk = tasks[ti];
    const DevGeom g = geos ? geos[tk.inst] : g0;
    const Phys ph = phys ? phys[tk.inst] : ph0;
    const int nft = (tk.P + TF - 1) / TF;
    const int64_t lt = tile - tk.tile0;
    const int m0 = (int)(lt % nft) * TF;
    const int s0 = (int)(lt / nft) * TS;
    __syncthreads();
    if (threadIdx.x < TF) {
      int m = m0 + threadIdx.x;
      if (m < tk.P) {
        double sn, cs;
        sincospi(2.0 * (double)m / (double)tk.P, &sn, &cs);
        sp[threadIdx.x].pnx = cs;
        sp[threadIdx.x].pny = sn;
        sp[threadIdx.x].fpnx = (float)cs;
        sp[threadIdx.x].fpny = (float)sn;
        sp[threadIdx.x].px = tk.cx + tk.rho * cs;
        sp[threadIdx.x].py = tk.cy + tk.rho * sn;
      }
    } else if (threadIdx.x < TF + TS) {
      int k = threadIdx.x - TF;
      if (s0 + k < tk.nn) load_slot(g, tk.node, tk.pos, s0 + k, ss[k]);
    }
    __syncthreads();
    const int m = m0 + tx, s = s0 + ty;
    if (m < tk.P && s < tk.nn) {
      double2 o[2][2];
      const SlotData& X = ss[ty];
      if (tk.side == 0) {
        double pw = 2.0 * WSBM_PI * tk.rho / (double)tk.P;
        if (MODE == WSBM_MIXED)
          proxy_row_mixed(T, ph, X, sp[tx], pw, o);
        else
          proxy_row_fp64<MODE == WSBM_MIXED_FINE>(T, ph, X, sp[tx], pw, o);
      } else {
        if (MODE == WSBM_MIXED)
          proxy_col_mixed(T, ph, X, sp[tx], o);
        else
          proxy_col_fp64<MODE == WSBM_MIXED_FINE>(T, ph, X, sp[tx], o);
      }
      const int bp[2] = {X.p0, X.p1};
#pragma unroll
      for (int sgn = 0; sgn < 2; ++sgn) {
        int64_t prow = (int64_t)tk.off + (int64_t)sgn * tk.P + m;
#pragma unroll
        for (int a = 0; a < 2; ++a) {
          if (bp[a] >= 0) {
            int64_t off = tk.tr ? ((int64_t)bp[a] + prow * tk.ld) : (prow + (int64_t)bp[a] * tk.ld);
            tk.out[off] = o[sgn][a];
          }
        }
      }
    }
  }
}

// -------------------------------------------------------------- Hankel test kernel ----
__global__ void k_hankel(const double* __restrict__ z, int64_t n, double* __restrict__ out,
                         int mixed) {
  __shared__ HkTables T;
  hk_stage_tables(&T);
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double zi = z[i];
    double* o = out + 6 * i;
    if (mixed == WSBM_MIXED_FINE) {
      Hk h;
      hankel_fp64_rs<true, true>(T, zi, rsqrt(zi), h);
      o[0] = h.h0r;
      o[1] = h.h0i;
      o[2] = h.h1r;
      o[3] = h.h1i;
      o[4] = h.f1r;
      o[5] = h.f1i;
    } else if (mixed) {
      HkF h;
      hankel_mixed(T, zi, rsqrtf((float)zi), h);
      o[0] = h.h0r;
      o[1] = h.h0i;
      o[2] = h.h1r;
      o[3] = h.h1i;
      o[4] = 0.0;
      o[5] = 0.0;
    } else {
      Hk h;
      hankel_fp64(T, zi, h);
      o[0] = h.h0r;
      o[1] = h.h0i;
      o[2] = h.h1r;
      o[3] = h.h1i;
      o[4] = h.f1r;
      o[5] = h.f1i;
    }
  }
}

__global__ void k_unknowns_to_slots(const int64_t* __restrict__ idx, int64_t n, int64_t N,
                                    int32_t* __restrict__ node, int32_t* __restrict__ pos) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    int64_t u = idx[t];
    int comp = u >= N ? 1 : 0;
    node[t] = (int32_t)(u - comp * N);
    pos[2 * t + comp] = (int32_t)t;
    pos[2 * t + 1 - comp] = -1;
  }
}

// ------------------------------------------------------------------- host helpers ----
static int grid_for(int64_t ntiles, int ctas = WSBM_ENTRY_CTAS) {
  const int64_t cap = (int64_t)wsbm_sm_count() * ctas;
  return (int)(ntiles < cap ? ntiles : cap);
}

static bool tile_ok(int tf, int ctas) { return (tf == 16 || tf == 32 || tf == 64) && ctas >= 1 && ctas <= 64; }

int64_t wsbm_pair_tiles(int32_t nr, int32_t nc, int32_t fastc, int tf) {
  int32_t nf = fastc ? nc : nr, ns = fastc ? nr : nc;
  if (nf <= 0 || ns <= 0) return 0;
  const int ts = WSBM_PAIR_THREADS / tf;
  return (int64_t)((nf + tf - 1) / tf) * ((ns + ts - 1) / ts);
}

int64_t wsbm_proxy_tiles(int32_t nn, int32_t P, int tf) {
  if (nn <= 0 || P <= 0) return 0;
  const int ts = WSBM_PAIR_THREADS / tf;
  return (int64_t)((P + tf - 1) / tf) * ((nn + ts - 1) / ts);
}

int wsbm_launch_pairs(const DevGeom& g, const Phys& ph, const PairTask* d_tasks, int ntasks,
                      int64_t ntiles, cudaStream_t st, const DevGeom* geos, const Phys* phys, int tf,
                      int ctas) {
  if (ntiles <= 0) return WSBM_OK;
  if (!tile_ok(tf, ctas)) return WSBM_ERR_INVALID_ARG;
  const int gr = grid_for(ntiles, ctas);
  if (tf == 16)
    k_pairs<16><<<gr, WSBM_PAIR_THREADS, 0, st>>>(g, ph, d_tasks, ntasks, ntiles, geos, phys);
  else if (tf == 64)
    k_pairs<64><<<gr, WSBM_PAIR_THREADS, 0, st>>>(g, ph, d_tasks, ntasks, ntiles, geos, phys);
  else
    k_pairs<32><<<gr, WSBM_PAIR_THREADS, 0, st>>>(g, ph, d_tasks, ntasks, ntiles, geos, phys);
  wsbm_count_launch();
  return cudaGetLastError() == cudaSuccess ? WSBM_OK : WSBM_ERR_CUDA;
}

template <int MODE>
static void launch_proxy_mode(int tf, int gr, cudaStream_t st, const DevGeom& g, const Phys& ph,
                              const ProxyTask* d_tasks, int ntasks, int64_t ntiles, const DevGeom* geos,
                              const Phys* phys) {
  if (tf == 16)
    k_proxy<MODE, 16><<<gr, WSBM_PAIR_THREADS, 0, st>>>(g, ph, d_tasks, ntasks, ntiles, geos, phys);
  else if (tf == 64)
    k_proxy<MODE, 64><<<gr, WSBM_PAIR_THREADS, 0, st>>>(g, ph, d_tasks, ntasks, ntiles, geos, phys);
  else
    k_proxy<MODE, 32><<<gr, WSBM_PAIR_THREADS, 0, st>>>(g, ph, d_tasks, ntasks, ntiles, geos, phys);
}

int wsbm_launch_proxy(const DevGeom& g, const Phys& ph, const ProxyTask* d_tasks, int ntasks,
                      int64_t ntiles, int mixed, cudaStream_t st, const DevGeom* geos,
                      const Phys* phys, int tf, int ctas) {
  if (ntiles <= 0) return WSBM_OK;
  if (!tile_ok(tf, ctas)) return WSBM_ERR_INVALID_ARG;
  const int gr = grid_for(ntiles, ctas);
  if (mixed == WSBM_MIXED)
    launch_proxy_mode<WSBM_MIXED>(tf, gr, st, g, ph, d_tasks, ntasks, ntiles, geos, phys);
  else if (mixed == WSBM_MIXED_FINE)
    launch_proxy_mode<WSBM_MIXED_FINE>(tf, gr, st, g, ph, d_tasks, ntasks, ntiles, geos, phys);
  else
    launch_proxy_mode<WSBM_FP64>(tf, gr, st, g, ph, d_tasks, ntasks, ntiles, geos, phys);
  wsbm_count_launch();
  return cudaGetLastError() == cudaSuccess ? WSBM_OK : WSBM_ERR_CUDA;
}

int wsbm_launch_hankel(const double* z, int64_t n, double* out, int mixed, cudaStream_t st) {
  if (n <= 0) return WSBM_OK;
  int64_t blocks = (n + 255) / 256;
  k_hankel<<<grid_for(blocks), 256, 0, st>>>(z, n, out, mixed);
  wsbm_count_launch();
  return cudaGetLastError() == cudaSuccess ? WSBM_OK : WSBM_ERR_CUDA;
}

int wsbm_launch_unknowns_to_slots(const int64_t* idx, int64_t n, int64_t N, int32_t* node,
                                  int32_t* pos, cudaStream_t st) {
  if (n <= 0) return WSBM_OK;
  int64_t blocks = (n + 255) / 256;
  k_unknowns_to_slots<<<grid_for(blocks), 256, 0, st>>>(idx, n, N, node, pos);
  wsbm_count_launch();
  return cudaGetLastError() == cudaSuccess ? WSBM_OK : WSBM_ERR_CUDA;
}
