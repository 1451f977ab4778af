// Reverse-mode (adjoint) kernels for shape and refractive-index gradients.
//
// The paper does not differentiate its solver.  For a far-field output F of the solution of
// A(p) x = b(p) the gradient of a real loss needs, besides the transposed solve A^T lam = v,
//   * the contraction Re(lam^T (dA/ds) x) for every node input s (position, normal, weight,
//     curvature) and for k1 and eps1:  k_entries_vjp, a dense node-pair reduction over the
//     same 2x2 blocks of eq. (weakly_bm) that the entry generator writes;
//   * Re(lam^T db/ds) for the plane-wave right-hand side:  k_rhs_planewave_vjp;
//   * the adjoint source v = C^T conj(g) and the explicit far-field derivative:  k_farfield_vjp;
//   * the Fourier curve r(t) = 1 + sum_j a_j cos(jt) + b_j sin(jt) and its reverse map from
//     node gradients to coefficient gradients:  k_curve_fourier / k_curve_fourier_vjp.
//
// Kernel algebra of the pair reduction.  With d = x_t - x_s (target minus source),
// a = d.n_t, b = d.n_s, nn = n_t.n_s and per wavenumber k
//   S_k = (i/4) H0(kr),  D_k = G_k b,  D*_k = -G_k a,  N_k = H_k a b + G_k nn,
//   G_k = (ik/4) H1(kr)/r,  H_k = (dG_k/dr)/r,
// and N_k0 - N_k1 is formed from the pole-free parts (the k-independent 1/(2 pi r^2) of G_k and
// -1/(pi r^4) of H_k cancel):  G^_k = (ik^2/4) F1(kr),  dG^_k/dr = (ik^2/4)(H0 - 2 F1)/r,
//   H^_k = (dG^_k/dr)/r,  dH^_k/dr = (ik^2/4)(-k H1/r^2 - 4 (H0 - 2 F1)/r^3),
// using H0' = -H1, H1' = H0 - H1/z, F1' = (H0 - 2 F1)/z.  Each block is a function of
// (r, a, b, nn) and the source weight; the chain rule to positions and normals is
//   d/dx_t = f_r d/r + f_a n_t + f_b n_s,  d/dx_s = -d/dx_t,  d/dn_t = f_a d + f_nn n_s,
//   d/dn_s = f_b d + f_nn n_t.
// Wavenumber derivatives: dS_k/dk = -(ir/4) H1, dD_k/dk = (ik/4) H0 b, dD*_k/dk = -(ik/4) H0 a,
//   dN_k/dk = (ik/4)(H0 nn - k H1 a b / r).
#include <math.h>
#include <string.h>

#include <algorithm>

#include "hankel.cuh"
#include "wsbm_internal.h"

namespace {

struct cx {
  double r, i;
};
__device__ __forceinline__ cx operator+(cx a, cx b) { return cx{a.r + b.r, a.i + b.i}; }
__device__ __forceinline__ cx operator-(cx a, cx b) { return cx{a.r - b.r, a.i - b.i}; }
__device__ __forceinline__ cx operator-(cx a) { return cx{-a.r, -a.i}; }
__device__ __forceinline__ cx operator*(cx a, cx b) {
  return cx{fma(a.r, b.r, -a.i * b.i), fma(a.r, b.i, a.i * b.r)};
}
__device__ __forceinline__ cx operator*(double s, cx a) { return cx{s * a.r, s * a.i}; }
__device__ __forceinline__ cx ti(cx a) { return cx{-a.i, a.r}; }  // i a
__device__ __forceinline__ double re_mul(cx a, cx b) { return fma(a.r, b.r, -a.i * b.i); }
__device__ __forceinline__ cx ld2(const double2* p, int64_t k) {
  double2 v = p[k];
  return cx{v.x, v.y};
}

#define VJP_THREADS 128

// Kernel values of one wavenumber k at distance r (see the header comment): S_k, dS_k/dr,
// G_k, dG_k/dr and the pole-free G^_k, dG^_k/dr, H^_k, dH^_k/dr.
struct KVals {
  cx S, Sr, G, Gr, Gh, Ghr, Hh, Hhr;
};

__device__ __forceinline__ void kvals(const Hk& h, double k, double ir, KVals& K) {
  const cx H0{h.h0r, h.h0i}, H1{h.h1r, h.h1i}, F1{h.f1r, h.f1i};
  K.S = 0.25 * ti(H0);
  K.Sr = (-0.25 * k) * ti(H1);
  K.G = (0.25 * k * ir) * ti(H1);
  K.Gr = (0.25 * k * ir) * ti(k * H0 - (2.0 * ir) * H1);
  const cx X = H0 - 2.0 * F1;
  const double q = 0.25 * k * k;
  K.Gh = q * ti(F1);
  K.Ghr = (q * ir) * ti(X);
  K.Hh = ir * K.Ghr;
  K.Hhr = (q * ir * ir) * ti((-k) * H1 - (4.0 * ir) * X);
}

// Products of one orientation of a pair: target multipliers (l0, l1) times source unknowns.
struct RoleProd {
  cx l0u, l1u, l0q, l1q;
};
__device__ __forceinline__ RoleProd role_prod(cx l0, cx l1, cx u, cx q) {
  return RoleProd{l0 * u, l1 * u, l0 * q, l1 * q};
}

struct RoleAcc {
  double val, dr, da, db, dnn;
};

// Adds wavenumber K's share (K0: k = k0, sign +1 in N_k0 - N_k1; K1: k = k1, sign -1) of
// lam_t^T A_ts x_s / w_s and of its derivatives in (r, a, b, nn).  In terms of the products:
//   D_k1 <- l0 u,  D_k0 <- l1 u,  alpha (N_k0 - N_k1) <- l1 u,  -eps1 S_k1 <- l0 q,
//   -eps0 S_k0 <- l1 q,  -alpha eps0 D*_k0 <- l1 q,  +alpha eps1 D*_k1 <- l1 q.
template <int KI>
__device__ __forceinline__ void role_add(const KVals& K, const Phys& ph, const RoleProd& P,
                                         double a, double b, double nn, RoleAcc& o) {
  const cx gb = KI == 0 ? P.l1u : P.l0u;                                  // D_k = G_k b
  const cx ga = ti((KI == 0 ? -ph.eps0 : ph.eps1) * ph.inv_k0 * P.l1q);   // D*_k terms: -ga G_k a
  const cx sv = KI == 0 ? ph.eps0 * P.l1q : ph.eps1 * P.l0q;              // -eps_k S_k
  const cx cN = ti((KI == 0 ? ph.inv_k0 : -ph.inv_k0) * P.l1u);           // +-alpha l1 u
  const double ab = a * b;
  const double gbG = re_mul(gb, K.G), gaG = re_mul(ga, K.G);
  o.val += b * gbG - a * gaG - re_mul(sv, K.S) + re_mul(cN, ab * K.Hh + nn * K.Gh);
  o.dr += b * re_mul(gb, K.Gr) - a * re_mul(ga, K.Gr) - re_mul(sv, K.Sr) +
          re_mul(cN, ab * K.Hhr + nn * K.Ghr);
  const double cNH = re_mul(cN, K.Hh);
  o.da += b * cNH - gaG;
  o.db += gbG + a * cNH;
  o.dnn += re_mul(cN, K.Gh);
}

// d/dk1 and d/deps1 of lam_t^T A_ts x_s / w_s (target orientation only), from the k1 values:
//   dS/dk = -(ir/4) H1, dD/dk = (ik/4) H0 b, dD*/dk = -(ik/4) H0 a,
//   dN/dk = (ik/4)(H0 nn - k H1 a b / r).
__device__ __forceinline__ void phys_add(const Hk& h, const KVals& K, const Phys& ph,
                                         const RoleProd& P, double r, double ir, double a,
                                         double b, double nn, double* pk1, double* pe1) {
  const double k1 = ph.k1;
  const cx H0{h.h0r, h.h0i}, H1{h.h1r, h.h1i};
  const cx KS = (-0.25 * r) * ti(H1);
  const cx KG = (0.25 * k1) * ti(H0);
  const cx KN = (0.25 * k1) * ti(nn * H0 - (k1 * a * b * ir) * H1);
  const cx cDs1 = ti((ph.eps1 * ph.inv_k0) * P.l1q);  // alpha eps1 l1 q
  const cx cN = ti(ph.inv_k0 * P.l1u);                // alpha l1 u
  *pk1 += re_mul(KG, b * P.l0u - a * cDs1) - ph.eps1 * re_mul(P.l0q, KS) - re_mul(cN, KN);
  *pe1 += -re_mul(P.l0q, K.S) - a * re_mul(ti(ph.inv_k0 * P.l1q), K.G);
}

// Diagonal block (one-point corrected rule): derivatives in w_i, kappa_i, k1, eps1.
__device__ __forceinline__ void vjp_diag(const Phys& ph, double wi, double kap, cx l0, cx l1, cx u,
                                         cx q, double* gw, double* gk, double* pk1, double* pe1) {
  const double k0 = ph.k0, k1 = ph.k1, e0 = ph.eps0, e1 = ph.eps1;
  const double inv2pi = 1.0 / (2.0 * WSBM_PI), inv4pi = 1.0 / (4.0 * WSBM_PI);
  const double L0 = log(k0 * wi * inv4pi), L1 = log(k1 * wi * inv4pi);
  const double Dd = -wi * kap * inv4pi, Dd_w = -kap * inv4pi, Dd_k = -wi * inv4pi;
  const cx S0w{-(WSBM_EULER + L0 + 1.0) * inv2pi, 0.25};
  const cx S1w{-(WSBM_EULER + L1 + 1.0) * inv2pi, 0.25};
  const cx S1d = wi * cx{-(WSBM_EULER + L1) * inv2pi, 0.25};
  const double f0 = k0 * k0 * (L0 + WSBM_EULER - 0.5), f1 = k1 * k1 * (L1 + WSBM_EULER - 0.5);
  const cx dNw{-(f0 - f1) * inv4pi - (k0 * k0 - k1 * k1) * inv4pi, (k0 * k0 - k1 * k1) * 0.125};
  const cx dNk1 = wi * cx{2.0 * k1 * (L1 + WSBM_EULER) * inv4pi, -0.25 * k1};
  const cx alpha{0.0, ph.inv_k0};
  const cx l0u = l0 * u, l1u = l1 * u, l0q = l0 * q, l1q = l1 * q;
  // dB/dw = l0 u Dd_w - eps1 l0 q S1_w + l1 u (Dd_w + alpha dN_w) + l1 q (-eps0 S0_w - alpha (eps0-eps1) Dd_w)
  cx t = Dd_w * l0u - e1 * (l0q * S1w) + (Dd_w * l1u + l1u * (alpha * dNw)) -
         l1q * (e0 * S0w + ((e0 - e1) * Dd_w) * alpha);
  *gw += t.r;
  cx tk = Dd_k * (l0u + l1u) - ((e0 - e1) * Dd_k) * (alpha * l1q);
  *gk += tk.r;
  // d/dk1: -eps1 l0 q dS1/dk1 + alpha l1 u dN/dk1,  dS1/dk1 = -w/(2 pi k1)
  cx tk1 = (e1 * wi * inv2pi / k1) * l0q + l1u * (alpha * dNk1);
  *pk1 += tk1.r;
  // d/deps1: -l0 q S1 + l1 q alpha (Dd - 1/2)
  cx te1 = -(l0q * S1d) + (Dd - 0.5) * (alpha * l1q);
  *pe1 += te1.r;
}

struct VjpSlot {
  double x, y, nx, ny, w, pad;
  cx l0, l1, u, q;
};

// grid (ceil(N/128), nsplit): thread = target node i; the CTA covers sources [j0, j1).
// part: nsplit x 6 x N partial node gradients; pphys: (gridDim.x * gridDim.y) x 2.
__global__ void __launch_bounds__(VJP_THREADS)
    k_entries_vjp(DevGeom g, Phys ph, const double2* __restrict__ lam, const double2* __restrict__ xv,
                  int64_t jspan, double* __restrict__ part, double* __restrict__ pphys) {
  __shared__ HkTables T;
  __shared__ VjpSlot sj[VJP_THREADS];
  __shared__ double red[2][VJP_THREADS];
  hk_stage_tables(&T);
  const int64_t N = g.n;
  const int64_t i = (int64_t)blockIdx.x * VJP_THREADS + threadIdx.x;
  const int64_t j0 = (int64_t)blockIdx.y * jspan;
  const int64_t j1 = min(N, j0 + jspan);
  const bool valid = i < N;
  double xi = 0, yi = 0, nxi = 0, nyi = 0, wi = 0, kap = 0;
  cx l0i{0, 0}, l1i{0, 0}, ui{0, 0}, qi{0, 0};
  if (valid) {
    xi = g.x[i];
    yi = g.y[i];
    nxi = g.nx[i];
    nyi = g.ny[i];
    wi = g.w[i];
    kap = g.kappa[i];
    l0i = ld2(lam, i);
    l1i = ld2(lam, N + i);
    ui = ld2(xv, i);
    qi = ld2(xv, N + i);
  }
  double gx = 0, gy = 0, gnx = 0, gny = 0, gw = 0, gk = 0, pk1 = 0, pe1 = 0;
  if (valid && i >= j0 && i < j1) vjp_diag(ph, wi, kap, l0i, l1i, ui, qi, &gw, &gk, &pk1, &pe1);
  for (int64_t jc = j0; jc < j1; jc += VJP_THREADS) {
    __syncthreads();
    {
      int64_t j = jc + threadIdx.x;
      if (j < j1) {
        VjpSlot& s = sj[threadIdx.x];
        s.x = g.x[j];
        s.y = g.y[j];
        s.nx = g.nx[j];
        s.ny = g.ny[j];
        s.w = g.w[j];
        s.l0 = ld2(lam, j);
        s.l1 = ld2(lam, N + j);
        s.u = ld2(xv, j);
        s.q = ld2(xv, N + j);
      }
    }
    __syncthreads();
    if (!valid) continue;
    const int nj = (int)min((int64_t)VJP_THREADS, j1 - jc);
#pragma unroll 1
    for (int jj = 0; jj < nj; ++jj) {
      // keep the Hankel tables in shared memory: no hoisting of their loads out of the loop
      asm volatile("" ::: "memory");
      if (jc + jj == i) continue;
      const VjpSlot& s = sj[jj];
      const double dx = xi - s.x, dy = yi - s.y;
      const double r = sqrt(fma(dx, dx, dy * dy));
      const double ir = 1.0 / r;
      const double z0 = ph.k0 * r, z1 = ph.k1 * r;
      const double rs0 = rsqrt(z0), rs1 = rs0 * ph.s01;
      const double a = fma(dx, nxi, dy * nyi);
      const double b = fma(dx, s.nx, dy * s.ny);
      const double nn = fma(nxi, s.nx, nyi * s.ny);
      const double rhx = dx * ir, rhy = dy * ir;
      // orientation T: node i is the target of pair (i, j);  orientation S: node i is the
      // source of pair (j, i), where d' = -d, a' = d'.n_j = -b, b' = d'.n_i = -a
      const RoleProd PT = role_prod(l0i, l1i, s.u, s.q);
      const RoleProd PS = role_prod(s.l0, s.l1, ui, qi);
      RoleAcc oT{0, 0, 0, 0, 0}, oS{0, 0, 0, 0, 0};
      {
        Hk h;
        hankel_fp64_rs<true>(T, z0, rs0, h);
        KVals K;
        kvals(h, ph.k0, ir, K);
        role_add<0>(K, ph, PT, a, b, nn, oT);
        role_add<0>(K, ph, PS, -b, -a, nn, oS);
      }
      {
        Hk h;
        hankel_fp64_rs<true>(T, z1, rs1, h);
        KVals K;
        kvals(h, ph.k1, ir, K);
        role_add<1>(K, ph, PT, a, b, nn, oT);
        role_add<1>(K, ph, PS, -b, -a, nn, oS);
        double tk1 = 0.0, te1 = 0.0;
        phys_add(h, K, ph, PT, r, ir, a, b, nn, &tk1, &te1);
        pk1 += s.w * tk1;
        pe1 += s.w * te1;
      }
      gx += s.w * (oT.dr * rhx + oT.da * nxi + oT.db * s.nx);
      gy += s.w * (oT.dr * rhy + oT.da * nyi + oT.db * s.ny);
      gnx += s.w * (oT.da * dx + oT.dnn * s.nx);
      gny += s.w * (oT.da * dy + oT.dnn * s.ny);
      gx += wi * (oS.dr * rhx - oS.da * s.nx - oS.db * nxi);
      gy += wi * (oS.dr * rhy - oS.da * s.ny - oS.db * nyi);
      gnx += wi * (oS.dnn * s.nx - oS.db * dx);
      gny += wi * (oS.dnn * s.ny - oS.db * dy);
      gw += oS.val;
    }
  }
  if (valid) {
    double* o = part + (int64_t)blockIdx.y * 6 * N;
    o[i] = gx;
    o[N + i] = gy;
    o[2 * N + i] = gnx;
    o[3 * N + i] = gny;
    o[4 * N + i] = gw;
    o[5 * N + i] = gk;
  }
  red[0][threadIdx.x] = pk1;
  red[1][threadIdx.x] = pe1;
  __syncthreads();
  for (int s = VJP_THREADS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      red[0][threadIdx.x] += red[0][threadIdx.x + s];
      red[1][threadIdx.x] += red[1][threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    int64_t b = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
    pphys[2 * b] = red[0][0];
    pphys[2 * b + 1] = red[1][0];
  }
}

// grad[q N + i] = sum over splits (fixed order); block 0 also sums the per-CTA k1 / eps1 parts.
__global__ void k_vjp_reduce(int64_t N, int nsplit, const double* __restrict__ part,
                             int64_t nblk, const double* __restrict__ pphys, double* __restrict__ grad,
                             double* __restrict__ gphys) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < 6 * N;
       e += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int t = 0; t < nsplit; ++t) s += part[(int64_t)t * 6 * N + e];
    grad[e] = s;
  }
  if (blockIdx.x == 0) {
    __shared__ double red[2][256];
    double a = 0.0, b = 0.0;
    for (int64_t t = threadIdx.x; t < nblk; t += blockDim.x) {
      a += pphys[2 * t];
      b += pphys[2 * t + 1];
    }
    red[0][threadIdx.x] = a;
    red[1][threadIdx.x] = b;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) {
        red[0][threadIdx.x] += red[0][threadIdx.x + s];
        red[1][threadIdx.x] += red[1][threadIdx.x + s];
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      gphys[0] = red[0][0];
      gphys[1] = red[1][0];
    }
  }
}

// Re(lam^T db/ds) for plane-wave right-hand sides b = [0; (d.n - 1) u_in], u_in = e^{i k0 d.x}:
// db/dx = (d.n - 1) i k0 d u_in,  db/dn = d u_in.  lam: 2N x nang (paper order).
__global__ void k_rhs_planewave_vjp(DevGeom g, double k0, const double* __restrict__ ang, int nang,
                                    const double2* __restrict__ lam, double* __restrict__ grad) {
  const int64_t N = g.n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double x = g.x[i], y = g.y[i], nx = g.nx[i], ny = g.ny[i];
    double gx = 0, gy = 0, gnx = 0, gny = 0;
    for (int a = 0; a < nang; ++a) {
      double sa, ca;
      sincos(ang[a], &sa, &ca);
      double sp, cp;
      sincos(k0 * (ca * x + sa * y), &sp, &cp);
      const cx uin{cp, sp};
      const cx l1 = ld2(lam, (int64_t)a * 2 * N + N + i);
      const cx lu = l1 * uin;
      const double sdn = ca * nx + sa * ny - 1.0;
      const double t = -sdn * k0 * lu.i;  // Re(l1 (s-1) i k0 u_in) = -(s-1) k0 Im(l1 u_in)
      gx += t * ca;
      gy += t * sa;
      gnx += ca * lu.r;
      gny += sa * lu.r;
    }
    grad[i] = gx;
    grad[N + i] = gy;
    grad[2 * N + i] = gnx;
    grad[3 * N + i] = gny;
    grad[4 * N + i] = 0.0;
    grad[5 * N + i] = 0.0;
  }
}

// Far field F_mc = c0 sum_j w_j [-i k0 (xh_m.n_j) u_jc - eps0 q_jc] e^{-i k0 xh_m.x_j},
// c0 = e^{i pi/4}/sqrt(8 pi k0).  Given gF (nang x nrhs, the loss gradient dL/dReF + i dL/dImF)
// it writes v = C^T conj(gF) (2N x nrhs, paper order) and the explicit node gradient
// Re(sum conj(gF) dF/ds) at fixed densities.
__global__ void k_farfield_vjp(DevGeom g, double k0, double eps0, const double2* __restrict__ u,
                               const double2* __restrict__ q, int nrhs, const double* __restrict__ ang,
                               int nang, const double2* __restrict__ gF, double2* __restrict__ v,
                               double* __restrict__ grad) {
  const int64_t N = g.n;
  const double pr = 1.0 / sqrt(8.0 * WSBM_PI * k0) * 0.70710678118654752440;
  const cx c0{pr, pr};
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < N;
       j += (int64_t)gridDim.x * blockDim.x) {
    const double x = g.x[j], y = g.y[j], nx = g.nx[j], ny = g.ny[j], w = g.w[j];
    double gx = 0, gy = 0, gnx = 0, gny = 0, gw = 0;
    for (int c = 0; c < nrhs; ++c) {
      const cx uj = ld2(u, (int64_t)c * N + j), qj = ld2(q, (int64_t)c * N + j);
      cx vu{0, 0}, vq{0, 0};
      for (int m = 0; m < nang; ++m) {
        double sa, ca;
        sincos(ang[m], &sa, &ca);
        double sp, cp;
        sincos(k0 * (ca * x + sa * y), &sp, &cp);
        const cx E{cp, -sp};
        const cx gm = ld2(gF, (int64_t)c * nang + m);
        const cx cg = cx{gm.r, -gm.i} * c0 * E;  // conj(g) c0 E
        const double xn = ca * nx + sa * ny;
        const cx Tm = (-k0 * xn) * ti(uj) - eps0 * qj;
        const cx cgT = cg * Tm;
        vu = vu + (-k0 * xn * w) * ti(cg);
        vq = vq + (-eps0 * w) * cg;
        // d/dx: w T (-i k0 ca) ;  d/dn: w (-i k0 ca u)
        const double ph = k0 * w * cgT.i;  // Re(-i k0 w cgT) = k0 w Im(cgT)
        gx += ph * ca;
        gy += ph * sa;
        const cx cgu = cg * uj;
        gnx += k0 * w * cgu.i * ca;
        gny += k0 * w * cgu.i * sa;
        gw += cgT.r;
      }
      v[(int64_t)c * 2 * N + j] = make_double2(vu.r, vu.i);
      v[(int64_t)c * 2 * N + N + j] = make_double2(vq.r, vq.i);
    }
    grad[j] = gx;
    grad[N + j] = gy;
    grad[2 * N + j] = gnx;
    grad[3 * N + j] = gny;
    grad[4 * N + j] = gw;
    grad[5 * N + j] = 0.0;
  }
}

// r, r', r'' of r(t) = 1 + sum_{j=1..M} a_j cos(jt) + b_j sin(jt)
__device__ __forceinline__ void fourier_r(int M, const double* __restrict__ a,
                                          const double* __restrict__ b, double t, double* r,
                                          double* r1, double* r2) {
  double s0 = 1.0, s1 = 0.0, s2 = 0.0;
  for (int j = 1; j <= M; ++j) {
    double sj, cj;
    sincos(j * t, &sj, &cj);
    const double aj = a[j - 1], bj = b[j - 1];
    s0 += aj * cj + bj * sj;
    s1 += j * (bj * cj - aj * sj);
    s2 -= (double)j * j * (aj * cj + bj * sj);
  }
  *r = s0;
  *r1 = s1;
  *r2 = s2;
}

__global__ void k_curve_fourier(int M, int64_t N, const double* __restrict__ a,
                                const double* __restrict__ b, double* x, double* y, double* nx,
                                double* ny, double* w, double* kappa) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double t = 2.0 * WSBM_PI * (double)i / (double)N;
    double r, r1, r2;
    fourier_r(M, a, b, t, &r, &r1, &r2);
    double s, c;
    sincos(t, &s, &c);
    const double xp = r1 * c - r * s, yp = r1 * s + r * c;
    const double xpp = r2 * c - 2.0 * r1 * s - r * c, ypp = r2 * s + 2.0 * r1 * c - r * s;
    const double sp = sqrt(xp * xp + yp * yp);
    x[i] = r * c;
    y[i] = r * s;
    nx[i] = yp / sp;
    ny[i] = -xp / sp;
    w[i] = (2.0 * WSBM_PI / (double)N) * sp;
    kappa[i] = (xp * ypp - yp * xpp) / (sp * sp * sp);
  }
}

// One CTA per coefficient (blockIdx.x < M: a_{j}, else b_{j}); the node loop reverses
// the geometry map to (dL/dr, dL/dr', dL/dr'') and contracts with the basis function.
__global__ void k_curve_fourier_vjp(int M, int64_t N, const double* __restrict__ a,
                                    const double* __restrict__ b, const double* __restrict__ grad,
                                    double* __restrict__ gcoef) {
  __shared__ double red[256];
  const int kk = blockIdx.x;
  const int j = kk % M + 1;
  const bool isb = kk >= M;
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
    const double t = 2.0 * WSBM_PI * (double)i / (double)N;
    double r, r1, r2;
    fourier_r(M, a, b, t, &r, &r1, &r2);
    double s, c;
    sincos(t, &s, &c);
    const double xp = r1 * c - r * s, yp = r1 * s + r * c;
    const double xpp = r2 * c - 2.0 * r1 * s - r * c, ypp = r2 * s + 2.0 * r1 * c - r * s;
    const double sp = sqrt(xp * xp + yp * yp);
    const double kap = (xp * ypp - yp * xpp) / (sp * sp * sp);
    const double gX = grad[i], gY = grad[N + i], gNx = grad[2 * N + i], gNy = grad[3 * N + i];
    const double gW = grad[4 * N + i], gK = grad[5 * N + i];
    double g_xp = -gNy / sp, g_yp = gNx / sp;
    double g_sp = (-gNx * yp + gNy * xp) / (sp * sp) + gW * (2.0 * WSBM_PI / (double)N) -
                  3.0 * gK * kap / sp;
    const double gC = gK / (sp * sp * sp);
    g_xp += gC * ypp;
    g_yp -= gC * xpp;
    const double g_xpp = -gC * yp, g_ypp = gC * xp;
    g_xp += g_sp * xp / sp;
    g_yp += g_sp * yp / sp;
    const double g_r = gX * c + gY * s - g_xp * s + g_yp * c - g_xpp * c - g_ypp * s;
    const double g_r1 = g_xp * c + g_yp * s - 2.0 * g_xpp * s + 2.0 * g_ypp * c;
    const double g_r2 = g_xpp * c + g_ypp * s;
    double sj, cj;
    sincos(j * t, &sj, &cj);
    if (!isb)
      acc += g_r * cj - g_r1 * j * sj - g_r2 * (double)j * j * cj;
    else
      acc += g_r * sj + g_r1 * j * cj - g_r2 * (double)j * j * sj;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) gcoef[kk] = red[0];
}

int grid_for(int64_t work, int per) {
  int64_t b = (work + per - 1) / per;
  if (b < 1) b = 1;
  const int64_t cap = (int64_t)wsbm_sm_count() * 16;
  if (b > cap) b = cap;
  return (int)b;
}

}  // namespace

int wsbm_phys_from_params(const wsbm_params* p, Phys* ph);
int wsbm_geom_check(const wsbm_geom* g);
DevGeom wsbm_devgeom(const wsbm_geom* g);

extern "C" int wsbm_entries_vjp(const wsbm_geom* g, const wsbm_params* p, const void* lam,
                                const void* x, double* grad, double* gphys, void* stream) {
  int rc = wsbm_geom_check(g);
  if (rc) return rc;
  Phys ph;
  if ((rc = wsbm_phys_from_params(p, &ph))) return rc;
  if (p->formulation != WSBM_FORM_WSBM) return WSBM_ERR_INVALID_ARG;  // eq. (weakly_bm) only
  if (!lam || !x || !grad || !gphys) return WSBM_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t N = g->n;
  const int64_t nti = (N + VJP_THREADS - 1) / VJP_THREADS;
  int nsm = wsbm_sm_count(), per_sm = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_entries_vjp, VJP_THREADS, 0) !=
          cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  // about eight waves of CTAs, each covering at least 128 sources
  int64_t want = (int64_t)nsm * per_sm * 8;
  int64_t nsplit = (want + nti - 1) / nti;
  nsplit = std::max<int64_t>(1, std::min<int64_t>(nsplit, nti));
  const int64_t jspan = (N + nsplit - 1) / nsplit;
  nsplit = (N + jspan - 1) / jspan;
  const int64_t nblk = nti * nsplit;
  WsbmScratch scr(st);
  double* part = nullptr;
  double* pphys = nullptr;
  if ((rc = scr.get((size_t)nsplit * 6 * N * sizeof(double), (void**)&part))) return rc;
  if ((rc = scr.get((size_t)nblk * 2 * sizeof(double), (void**)&pphys))) return rc;
  DevGeom dg = wsbm_devgeom(g);
  k_entries_vjp<<<dim3((unsigned)nti, (unsigned)nsplit), VJP_THREADS, 0, st>>>(
      dg, ph, (const double2*)lam, (const double2*)x, jspan, part, pphys);
  wsbm_count_launch();
  k_vjp_reduce<<<grid_for(6 * N, 256), 256, 0, st>>>(N, (int)nsplit, part, nblk, pphys, grad, gphys);
  wsbm_count_launch();
  rc = cudaGetLastError() == cudaSuccess ? WSBM_OK : WSBM_ERR_CUDA;
  return rc;
}

extern "C" int wsbm_rhs_planewave_vjp(const wsbm_geom* g, const wsbm_params* p,
                                      const double* angles, int32_t nang, const void* lam,
                                      double* grad, void* stream) {
  int rc = wsbm_geom_check(g);
  if (rc) return rc;
  if (!p || !(p->k0 > 0.0) || nang < 0 || !grad || (nang > 0 && (!angles || !lam)))
    return WSBM_ERR_INVALID_ARG;
  if (p->formulation != WSBM_FORM_WSBM) return WSBM_ERR_INVALID_ARG;  // eq. (weakly_bm) only
  cudaStream_t st = (cudaStream_t)stream;
  k_rhs_planewave_vjp<<<grid_for(g->n, 256), 256, 0, st>>>(wsbm_devgeom(g), p->k0, angles, nang,
                                                           (const double2*)lam, grad);
  wsbm_count_launch();
  return cudaGetLastError() == cudaSuccess ? WSBM_OK : WSBM_ERR_CUDA;
}

extern "C" int wsbm_farfield_vjp(const wsbm_geom* g, const wsbm_params* p, const void* u,
                                 const void* q, int32_t nrhs, const double* angles, int32_t nang,
                                 const void* gF, void* v, double* grad, void* stream) {
  int rc = wsbm_geom_check(g);
  if (rc) return rc;
  Phys ph;
  if ((rc = wsbm_phys_from_params(p, &ph))) return rc;
  if (p->formulation != WSBM_FORM_WSBM) return WSBM_ERR_INVALID_ARG;  // eq. (weakly_bm) only
  if (nrhs < 1 || nang < 0 || !u || !q || !v || !grad || (nang > 0 && (!angles || !gF)))
    return WSBM_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  k_farfield_vjp<<<grid_for(g->n, 128), 128, 0, st>>>(wsbm_devgeom(g), ph.k0, ph.eps0,
                                                      (const double2*)u, (const double2*)q, nrhs,
                                                      angles, nang, (const double2*)gF,
                                                      (double2*)v, grad);
  wsbm_count_launch();
  return cudaGetLastError() == cudaSuccess ? WSBM_OK : WSBM_ERR_CUDA;
}

extern "C" int wsbm_curve_fourier(int32_t M, int64_t N, const double* a, const double* b,
                                  double* x, double* y, double* nx, double* ny, double* w,
                                  double* kappa, void* stream) {
  if (M < 0 || N < 3 || (M > 0 && (!a || !b)) || !x || !y || !nx || !ny || !w || !kappa)
    return WSBM_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  k_curve_fourier<<<grid_for(N, 256), 256, 0, st>>>(M, N, a, b, x, y, nx, ny, w, kappa);
  wsbm_count_launch();
  return cudaGetLastError() == cudaSuccess ? WSBM_OK : WSBM_ERR_CUDA;
}

extern "C" int wsbm_curve_fourier_vjp(int32_t M, int64_t N, const double* a, const double* b,
                                      const double* grad, double* gcoef, void* stream) {
  if (M < 1 || N < 3 || !a || !b || !grad || !gcoef) return WSBM_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  k_curve_fourier_vjp<<<2 * M, 256, 0, st>>>(M, N, a, b, grad, gcoef);
  wsbm_count_launch();
  return cudaGetLastError() == cudaSuccess ? WSBM_OK : WSBM_ERR_CUDA;
}
