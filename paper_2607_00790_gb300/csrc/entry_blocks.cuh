// Device functions of one WSBM node-pair block (eq. weakly_bm; block form A_ij of Sec. III),
// shared by the entry generator and the matrix-free product.
#pragma once
#include "hankel.cuh"
#include "wsbm_internal.h"

#define WSBM_4PI 12.566370614359172954

// Geometric quantities of a pair with the operation order fixed (no contraction): r and the
// arguments z = k r are reproducible bit for bit by any IEEE double implementation.
struct PairGeom {
  double r, ir, z0, z1, dnx, dny, nn, c, rs0, rs1;
};

__device__ __forceinline__ void pair_geom(double xi, double yi, double nxi, double nyi, double xj,
                                          double yj, double nxj, double nyj, const Phys& ph,
                                          PairGeom& G) {
  double dx = __dsub_rn(xi, xj);
  double dy = __dsub_rn(yi, yj);
  double r2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
  double r = __dsqrt_rn(r2);
  G.r = r;
  G.z0 = __dmul_rn(ph.k0, r);
  G.z1 = __dmul_rn(ph.k1, r);
  G.dny = __dadd_rn(__dmul_rn(dx, nxj), __dmul_rn(dy, nyj));
  G.dnx = __dadd_rn(__dmul_rn(dx, nxi), __dmul_rn(dy, nyi));
  G.nn = __dadd_rn(__dmul_rn(nxi, nxj), __dmul_rn(nyi, nyj));
  // one reciprocal square root serves both wavenumbers and 1/r
  G.rs0 = rsqrt(G.z0);
  G.rs1 = G.rs0 * ph.s01;
  G.ir = ph.k0 * (G.rs0 * G.rs0);
  G.c = G.dnx * G.dny * (G.ir * G.ir);
}

// Off-diagonal 2x2 block, weight w_j folded in (kernels: G_k = (i/4) H0(kr);
// D: (ik/4) H1 (d.n_y)/r;  D*: -(ik/4) H1 (d.n_x)/r;
// N_k0 - N_k1 = (i/4)[(k0^2 H0(z0) - k1^2 H0(z1)) c + (k0^2 F1(z0) - k1^2 F1(z1))(n_x.n_y - 2c)]).
__device__ __forceinline__ void block_offdiag(const HkTables& T, const Phys& ph, const PairGeom& G,
                                              double wj, double2 e[2][2]) {
  Hk a, b;
  hankel_fp64_rs<true>(T, G.z0, G.rs0, a);
  hankel_fp64_rs<true>(T, G.z1, G.rs1, b);
  const double k0 = ph.k0, k1 = ph.k1;
  double s11 = 0.25 * wj * k1 * G.dny * G.ir;  // A11 = i s11 H1(z1)
  e[0][0] = make_double2(-s11 * b.h1i, s11 * b.h1r);
  double s12 = -0.25 * ph.eps1 * wj;  // A12 = i s12 H0(z1)
  e[0][1] = make_double2(-s12 * b.h0i, s12 * b.h0r);
  double q0 = k0 * k0, q1 = k1 * k1;
  double m2c = G.nn - 2.0 * G.c;
  double gr = (q0 * a.h0r - q1 * b.h0r) * G.c + (q0 * a.f1r - q1 * b.f1r) * m2c;
  double gi = (q0 * a.h0i - q1 * b.h0i) * G.c + (q0 * a.f1i - q1 * b.f1i) * m2c;
  double inv4k0 = 0.25 * ph.inv_k0;
  double t1 = 0.25 * k0 * G.dny * G.ir;
  // A21 = w [ i t1 H1(z0) + alpha dN ],  alpha dN = -(1/(4 k0)) (gr + i gi)
  e[1][0] = make_double2(wj * (-t1 * a.h1i - inv4k0 * gr), wj * (t1 * a.h1r - inv4k0 * gi));
  // A22 = w [ -i (eps0/4) H0(z0) - (d.n_x/(4 k0 r)) (eps0 k0 H1(z0) - eps1 k1 H1(z1)) ]
  double u = G.dnx * G.ir * inv4k0;
  double vr = ph.eps0 * k0 * a.h1r - ph.eps1 * k1 * b.h1r;
  double vi = ph.eps0 * k0 * a.h1i - ph.eps1 * k1 * b.h1i;
  e[1][1] = make_double2(wj * (0.25 * ph.eps0 * a.h0i - u * vr),
                         wj * (-0.25 * ph.eps0 * a.h0r - u * vi));
}

// Diagonal 2x2 block: one-point corrected trapezoidal rule.  A kernel a ln|x-y| + b gets the
// weight w_i [a ln(w_i/2pi) + b(x_i, x_i)]; D and D* tend to -kappa/(4 pi).
__device__ __forceinline__ void block_diag(const Phys& ph, double wi, double kap, double2 e[2][2]) {
  const double k0 = ph.k0, k1 = ph.k1;
  double L0 = log(k0 * wi / WSBM_4PI);
  double L1 = log(k1 * wi / WSBM_4PI);
  double S0r = -wi * (WSBM_EULER + L0) / (2.0 * WSBM_PI), Si = 0.25 * wi;
  double S1r = -wi * (WSBM_EULER + L1) / (2.0 * WSBM_PI);
  double Dd = -wi * kap / WSBM_4PI;
  double f0 = k0 * k0 * (L0 + WSBM_EULER - 0.5);
  double f1 = k1 * k1 * (L1 + WSBM_EULER - 0.5);
  double dNr = -wi * (f0 - f1) / WSBM_4PI;
  double dNi = wi * (k0 * k0 - k1 * k1) / 8.0;
  e[0][0] = make_double2(Dd + 0.5, 0.0);
  e[0][1] = make_double2(-ph.eps1 * S1r, -ph.eps1 * Si);
  e[1][0] = make_double2(Dd - 0.5 - dNi / k0, dNr / k0);
  e[1][1] = make_double2(-ph.eps0 * S0r,
                         -ph.eps0 * Si - ((ph.eps0 - ph.eps1) * Dd + 0.5 * (ph.eps0 + ph.eps1)) / k0);
}
