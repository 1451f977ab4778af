// Plain, slow CPU oracle for the weakly singular Burton-Miller (WSBM) Nystrom system.
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or calls this file;
// only the test suite, the smoke check and the CPU-baseline leg of the benchmark do.  It
// shares no code, header or constant table with the CUDA path.
//
// What it computes (paper: Matsumoto & Yokota, "Proxy-surface-based fast direct solver for
// TE-mode scattering problems on distributed memory systems"):
//   * Hankel values H0^(1)(z), H1^(1)(z) from the C++17 special functions
//     std::cyl_bessel_jl / std::cyl_neumannl, evaluated in long double and rounded to double.
//   * The 2x2 WSBM block of eq. (weakly_bm) for a node pair (Sec. II; the block form A_ij of
//     Sec. III), with the kernels of S_k, D_k, D*_k and N_k of the 2-D Helmholtz fundamental
//     solution G_k = (i/4) H0^(1)(k r).  The paper names these operators but does not print
//     G; the reading (radiating H^(1), D differentiates in y, D* in x) is the one consistent
//     with the jump terms +-I/2 of eqs. (bm) and (weakly_bm).
//   * The one-point corrected diagonal (Sec. I/II: a local correction of the diagonal terms
//     alone, zeta-corrected trapezoidal rule).  The paper prints no formula; the reading
//     is the one-point log correction w_i*ln(w_i/2pi) applied to each log-singular kernel
//     and the smooth limits of D and D* (curvature term).
//   * Proxy-circle blocks used by the proxy-surface interpolative decomposition (Sec. III,
//     proxy-surface low-rank approximation).
//   * The standard Burton-Miller (eq. bm) and PMCHWT (eq. pmchwt) matrices, with a one-point
//     correction of the hypersingular N_k (first-order accurate, as the paper reports).
//   * Directional derivatives of lam^T A x along tangents of the node data, k1 and eps1, by
//     evaluating the same block definitions in dual-number arithmetic (forward mode).  The
//     paper does not differentiate its solver; this serves the shape-gradient tests.
//
// Floating point: compile with -ffp-contract=off so that the geometric quantities
// (d, r, k*r, d.n) follow exactly the operation order written below.
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <vector>

typedef std::complex<double> cplx;
typedef long double ld;

static const double PI = 3.14159265358979323846264338327950288;
static const double EULER_GAMMA = 0.57721566490153286060651209008240243;
static const ld PI_L = 3.14159265358979323846264338327950288L;

// ---------------------------------------------------------------------------------------
// Hankel functions of the first kind, orders 0 and 1, and the pole-free combination
//   F1(z) = H1(z)/z + 2i/(pi z^2)
// (the k-independent 1/r^2 pole of N_k cancels in N_k0 - N_k1; the paper notes that this
// difference is only weakly singular, Sec. II after eq. (weakly_bm)).
// ---------------------------------------------------------------------------------------
struct Hank {
  cplx h0, h1, f1;
};

static Hank hankel_eval(double z) {
  ld zl = (ld)z;
  ld j0 = std::cyl_bessel_jl(0.0L, zl);
  ld j1 = std::cyl_bessel_jl(1.0L, zl);
  ld y0 = std::cyl_neumannl(0.0L, zl);
  ld y1 = std::cyl_neumannl(1.0L, zl);
  Hank h;
  h.h0 = cplx((double)j0, (double)y0);
  h.h1 = cplx((double)j1, (double)y1);
  ld f1re = j1 / zl;
  ld f1im = y1 / zl + 2.0L / (PI_L * zl * zl);
  h.f1 = cplx((double)f1re, (double)f1im);
  return h;
}

struct Params {
  double k0, k1, eps0, eps1;
};

// ---------------------------------------------------------------------------------------
// Off-diagonal 2x2 WSBM block for row node i (target x), column node j (source y), with the
// quadrature weight w_j folded in.  Eq. (weakly_bm):
//   [ D_k1 + I/2                          , -eps1 S_k1                                  ]
//   [ D_k0 - I/2 + alpha (N_k0 - N_k1)    , -eps0 S_k0 - alpha(eps0 D*_k0 - eps1 D*_k1) ]
//       - alpha (eps0+eps1) I/2 on the diagonal;  alpha = i/k0 (Sec. II, after eq. (bm)).
// Kernels (d = x - y, r = |d|):
//   G_k   = (i/4) H0(k r)
//   dG/dn_y = (i k/4) H1(k r) (d.n_y)/r                         (kernel of D_k)
//   dG/dn_x = -(i k/4) H1(k r) (d.n_x)/r                        (kernel of D*_k)
//   N_k   = (i k^2/4) [ H0(kr) c + H1(kr)/(kr) (n_x.n_y - 2c) ],  c = (d.n_x)(d.n_y)/r^2
// ---------------------------------------------------------------------------------------
struct Geom {
  int64_t n;
  const double *x, *y, *nx, *ny, *w, *kappa;
};

static void pair_block_offdiag(const Geom& g, const Params& p, int64_t i, int64_t j, cplx a[2][2]) {
  const cplx I1(0.0, 1.0);
  double dx = g.x[i] - g.x[j];
  double dy = g.y[i] - g.y[j];
  double r2 = dx * dx + dy * dy;
  double r = std::sqrt(r2);
  double z0 = p.k0 * r;
  double z1 = p.k1 * r;
  double dny = dx * g.nx[j] + dy * g.ny[j];
  double dnx = dx * g.nx[i] + dy * g.ny[i];
  double nn = g.nx[i] * g.nx[j] + g.ny[i] * g.ny[j];
  double c = (dnx * dny) / r2;
  Hank ha = hankel_eval(z0);
  Hank hb = hankel_eval(z1);
  cplx G0 = 0.25 * I1 * ha.h0;
  cplx G1 = 0.25 * I1 * hb.h0;
  cplx Dy0 = 0.25 * I1 * p.k0 * ha.h1 * (dny / r);
  cplx Dy1 = 0.25 * I1 * p.k1 * hb.h1 * (dny / r);
  cplx Dx0 = -0.25 * I1 * p.k0 * ha.h1 * (dnx / r);
  cplx Dx1 = -0.25 * I1 * p.k1 * hb.h1 * (dnx / r);
  double q0 = p.k0 * p.k0, q1 = p.k1 * p.k1;
  cplx dN = 0.25 * I1 * ((q0 * ha.h0 - q1 * hb.h0) * c + (q0 * ha.f1 - q1 * hb.f1) * (nn - 2.0 * c));
  cplx alpha = I1 / p.k0;
  double wj = g.w[j];
  a[0][0] = wj * Dy1;
  a[0][1] = -p.eps1 * wj * G1;
  a[1][0] = wj * (Dy0 + alpha * dN);
  a[1][1] = wj * (-p.eps0 * G0 - alpha * (p.eps0 * Dx0 - p.eps1 * Dx1));
}

// Diagonal 2x2 block: one-point corrected trapezoidal rule.  A kernel a(x,y) ln|x-y| + b(x,y)
// gets the diagonal weight w_i [a ln(w_i/2pi) + b(x_i,x_i)].  Applied to
//   S_k:   a = -1/(2pi),            b = i/4 - (ln(k/2) + gamma)/(2pi)
//   D, D*: a = 0,                   b = -kappa/(4pi)          (smooth limit, outward normal)
//   N_k0 - N_k1: a = -(k0^2-k1^2)/(4pi),
//                b = i(k0^2-k1^2)/8 - [k0^2(ln(k0/2)+gamma-1/2) - k1^2(ln(k1/2)+gamma-1/2)]/(4pi)
// plus the identity terms of eq. (weakly_bm).
// corrected diagonal of S_k, and the k-dependent log and smooth parts of N_k (times 4 pi / w_i)
static cplx s_diag(double k, double wi) {
  const cplx I1(0.0, 1.0);
  return wi * (0.25 * I1 - (EULER_GAMMA + std::log(k * wi / (4.0 * PI))) / (2.0 * PI));
}
static double n_log_part(double k, double wi) {
  return k * k * (std::log(k * wi / (4.0 * PI)) + EULER_GAMMA - 0.5);
}

static void pair_block_diag(const Geom& g, const Params& p, int64_t i, cplx a[2][2]) {
  const cplx I1(0.0, 1.0);
  double wi = g.w[i];
  double kap = g.kappa[i];
  auto S = [&](double k) { return s_diag(k, wi); };
  auto f = [&](double k) { return n_log_part(k, wi); };
  double Dd = -wi * kap / (4.0 * PI);
  cplx dN = wi * (I1 * (p.k0 * p.k0 - p.k1 * p.k1) / 8.0 - (f(p.k0) - f(p.k1)) / (4.0 * PI));
  cplx alpha = I1 / p.k0;
  a[0][0] = Dd + 0.5;
  a[0][1] = -p.eps1 * S(p.k1);
  a[1][0] = Dd - 0.5 + alpha * dN;
  a[1][1] = -p.eps0 * S(p.k0) - alpha * (p.eps0 - p.eps1) * Dd - alpha * (p.eps0 + p.eps1) * 0.5;
}

static void pair_block(const Geom& g, const Params& p, int64_t i, int64_t j, cplx a[2][2]) {
  if (i == j)
    pair_block_diag(g, p, i, a);
  else
    pair_block_offdiag(g, p, i, j, a);
}

// ---------------------------------------------------------------------------------------
// The two formulations the paper sets against eq. (weakly_bm) (Sec. II): the PMCHWT equation
// (eq. pmchwt) and the standard Burton-Miller equation (eq. bm).  Both contain N_k alone, whose
// kernel is hypersingular: near the diagonal, in the curve parameter t with trapezoidal step h
// and speed |x'|,  N_k(x(s), x(t)) |x'(t)| = 1/(2 pi |x'| (t-s)^2) + O(1/(t-s))
// - (k^2/4pi) |x'| ln|t-s| + O(1).  One-point correction of the diagonal (reading of the
// zeta-corrected rule for the hypersingular operator; the paper does not print it):
//   * the 1/(t-s)^2 part: the punctured sum h sum_{j!=0} g(jh)/(jh)^2 exceeds the finite-part
//     integral by 2 zeta(2) g(0)/h, so the diagonal weight is -(pi^2/3h) / (2 pi |x'|)
//     = -pi / (6 w_i)  (w_i = h |x'_i|);
//   * the log part: the weight w_i [a ln(w_i/2pi) + b] as for S_k, with a = -k^2/(4pi) and
//     b = i k^2/8 - k^2 (ln(k/2) + gamma - 1/2)/(4pi) (the k-dependent smooth limit);
//   * the O(1) term of the expansion (a curvature term of the Laplace hypersingular kernel)
//     is not corrected: it leaves an O(h) error, the first-order convergence the paper
//     reports for both formulations.
// In N_k0 - N_k1 the -pi/(6 w_i) weights cancel and the rest reproduces the diagonal of
// eq. (weakly_bm) above.
// ---------------------------------------------------------------------------------------
struct Ops {
  cplx S[2], D[2], Dx[2], N[2];  // index 0: k0, 1: k1; quadrature weight w_j folded in
};

static void pair_ops_offdiag(const Geom& g, const Params& p, int64_t i, int64_t j, Ops& o) {
  const cplx I1(0.0, 1.0);
  double dx = g.x[i] - g.x[j];
  double dy = g.y[i] - g.y[j];
  double r2 = dx * dx + dy * dy;
  double r = std::sqrt(r2);
  double dny = dx * g.nx[j] + dy * g.ny[j];
  double dnx = dx * g.nx[i] + dy * g.ny[i];
  double nn = g.nx[i] * g.nx[j] + g.ny[i] * g.ny[j];
  double c = (dnx * dny) / r2;
  double wj = g.w[j];
  const double ks[2] = {p.k0, p.k1};
  for (int t = 0; t < 2; ++t) {
    const double k = ks[t];
    Hank h = hankel_eval(k * r);
    o.S[t] = wj * 0.25 * I1 * h.h0;
    o.D[t] = wj * 0.25 * I1 * k * h.h1 * (dny / r);
    o.Dx[t] = -wj * 0.25 * I1 * k * h.h1 * (dnx / r);
    // N_k = (i k^2/4) [H0 c + H1/(kr) (nn - 2c)]
    o.N[t] = wj * 0.25 * I1 * k * k * (h.h0 * c + h.h1 / (k * r) * (nn - 2.0 * c));
  }
}

static void pair_ops_diag(const Geom& g, const Params& p, int64_t i, Ops& o) {
  const cplx I1(0.0, 1.0);
  double wi = g.w[i];
  double kap = g.kappa[i];
  const double ks[2] = {p.k0, p.k1};
  for (int t = 0; t < 2; ++t) {
    const double k = ks[t];
    o.S[t] = s_diag(k, wi);
    o.D[t] = -wi * kap / (4.0 * PI);
    o.Dx[t] = o.D[t];
    o.N[t] = wi * (I1 * k * k / 8.0 - n_log_part(k, wi) / (4.0 * PI)) - PI / (6.0 * wi);
  }
}

// 2x2 block of a formulation, unknowns (u, q) in this order for all three:
//   form 1, eq. (bm):     [ D_k1 + I/2,          -eps1 S_k1                  ]
//                          [ D_k0 - I/2 + a N_k0, -eps0 (S_k0 + a (D*_k0 + I/2)) ]
//   form 2, eq. (pmchwt), its columns in the order (u, q):
//                          [ D_k0 + D_k1,              -(eps0 S_k0 + eps1 S_k1) ]
//                          [ N_k0/eps0 + N_k1/eps1,    -(D*_k0 + D*_k1)          ]
static void form_block(const Geom& g, const Params& p, int form, int64_t i, int64_t j, cplx a[2][2]) {
  const cplx I1(0.0, 1.0);
  Ops o;
  if (i == j)
    pair_ops_diag(g, p, i, o);
  else
    pair_ops_offdiag(g, p, i, j, o);
  const double id = (i == j) ? 0.5 : 0.0;
  const cplx alpha = I1 / p.k0;
  if (form == 1) {
    a[0][0] = o.D[1] + id;
    a[0][1] = -p.eps1 * o.S[1];
    a[1][0] = o.D[0] - id + alpha * o.N[0];
    a[1][1] = -p.eps0 * (o.S[0] + alpha * (o.Dx[0] + id));
  } else {
    a[0][0] = o.D[0] + o.D[1];
    a[0][1] = -(p.eps0 * o.S[0] + p.eps1 * o.S[1]);
    a[1][0] = o.N[0] / p.eps0 + o.N[1] / p.eps1;
    a[1][1] = -(o.Dx[0] + o.Dx[1]);
  }
}

// ---------------------------------------------------------------------------------------
// Proxy-circle entries (proxy-surface method, Sec. III).  A proxy point p with outward unit
// normal nu carries a combined-field source Phi_k(x,p) = dG_k(x,p)/dnu_p - i eta G_k(x,p),
// eta = k (the combined field avoids interior resonances of the proxy disk).
//
// Row block (the equations of a box, used to pick row skeletons).  In eq. (weakly_bm) the
// equations at a target x read, for far sources,
//   eq1(x) = psi1(x),     eq2(x) = psi0(x) + alpha d_n psi0(x) - alpha d_n psi1(x)
// with psi_k the k-field of the sources.  Column m (0 <= m < P) is the k1 proxy source
// [Phi1 ; -alpha d_nx Phi1], column P+m the k0 proxy source [0 ; Phi0 + alpha d_nx Phi0].
//
// Column block (the unknowns of a box, used to pick column skeletons).  Far equations depend
// on the box's unknowns only through psi1 and psi0 outside the proxy circle, which the
// exterior Dirichlet data on the circle fixes.  Row m is psi1 at p_m, row P+m is psi0 at p_m:
//   u_j -> w_j dG_k(p,y_j)/dn_y,   q_j -> -eps_k w_j G_k(p,y_j).
// ---------------------------------------------------------------------------------------
static void proxy_row_entries(const Geom& g, const Params& p, int64_t i, double px, double py,
                              double pnx, double pny, double pw, cplx out[2][2], int form = 0) {
  const cplx I1(0.0, 1.0);
  double dx = g.x[i] - px;
  double dy = g.y[i] - py;
  double r2 = dx * dx + dy * dy;
  double r = std::sqrt(r2);
  double dnu = dx * pnx + dy * pny;       // d . nu_p
  double dnx = dx * g.nx[i] + dy * g.ny[i];  // d . n_x
  double nn = g.nx[i] * pnx + g.ny[i] * pny;
  double c = (dnx * dnu) / r2;
  cplx alpha = I1 / p.k0;
  cplx phi[2], dphi[2];
  for (int s = 0; s < 2; ++s) {
    double k = (s == 0) ? p.k1 : p.k0;
    double z = k * r;
    Hank h = hankel_eval(z);
    cplx G = 0.25 * I1 * h.h0;
    cplx dGdnu = 0.25 * I1 * k * h.h1 * (dnu / r);
    cplx dGdnx = -0.25 * I1 * k * h.h1 * (dnx / r);
    cplx Nk = 0.25 * I1 * k * k * (h.h0 * c + (h.h1 / z) * (nn - 2.0 * c));
    double eta = k;
    phi[s] = dGdnu - I1 * eta * G;
    dphi[s] = Nk - I1 * eta * dGdnx;
  }
  // out[a][s]: equation a of node i, source s (0 = k1 source, 1 = k0 source)
  if (form == 1) {  // eq. (bm): eq1 = psi1, eq2 = psi0 + alpha d_n psi0
    out[0][0] = pw * phi[0];
    out[1][0] = cplx(0.0, 0.0);
    out[0][1] = cplx(0.0, 0.0);
    out[1][1] = pw * (phi[1] + alpha * dphi[1]);
    return;
  }
  if (form == 2) {  // eq. (pmchwt): eq1 = psi0 + psi1, eq2 = d_n psi0 / eps0 + d_n psi1 / eps1
    out[0][0] = pw * phi[0];
    out[1][0] = pw * dphi[0] / p.eps1;
    out[0][1] = pw * phi[1];
    out[1][1] = pw * dphi[1] / p.eps0;
    return;
  }
  out[0][0] = pw * phi[0];
  out[1][0] = pw * (-alpha * dphi[0]);
  out[0][1] = cplx(0.0, 0.0);
  out[1][1] = pw * (phi[1] + alpha * dphi[1]);
}

static void proxy_col_entries(const Geom& g, const Params& p, int64_t j, double px, double py,
                              cplx out[2][2]) {
  const cplx I1(0.0, 1.0);
  double dx = px - g.x[j];
  double dy = py - g.y[j];
  double r2 = dx * dx + dy * dy;
  double r = std::sqrt(r2);
  double dny = dx * g.nx[j] + dy * g.ny[j];
  double wj = g.w[j];
  // out[s][b]: field s (0 = psi1, 1 = psi0) from unknown b (0 = u_j, 1 = q_j)
  for (int s = 0; s < 2; ++s) {
    double k = (s == 0) ? p.k1 : p.k0;
    double eps = (s == 0) ? p.eps1 : p.eps0;
    Hank h = hankel_eval(k * r);
    out[s][0] = wj * (0.25 * I1 * k * h.h1 * (dny / r));
    out[s][1] = -eps * wj * (0.25 * I1 * h.h0);
  }
}

// ---------------------------------------------------------------------------------------
// Forward-mode derivatives (shape and refractive-index gradients).  A dual number carries a
// value and its derivative along one tangent direction of the inputs (node positions,
// normals, weights, curvatures, k1, eps1).  The blocks below are the blocks above evaluated
// in dual arithmetic, so their derivative parts are the exact directional derivatives of
// the same definitions.  Hankel derivatives: H0' = -H1, H1' = H0 - H1/z, and for
// F1 = H1/z + 2i/(pi z^2):  F1' = (H0 - 2 F1)/z.
// ---------------------------------------------------------------------------------------
struct rd {
  double v, t;
};
struct cd {
  cplx v, t;
};
static inline rd R(double v) { return rd{v, 0.0}; }
static inline rd operator+(rd a, rd b) { return rd{a.v + b.v, a.t + b.t}; }
static inline rd operator-(rd a, rd b) { return rd{a.v - b.v, a.t - b.t}; }
static inline rd operator*(rd a, rd b) { return rd{a.v * b.v, a.t * b.v + a.v * b.t}; }
static inline rd operator*(double s, rd a) { return rd{s * a.v, s * a.t}; }
static inline rd operator/(rd a, rd b) { return rd{a.v / b.v, (a.t * b.v - a.v * b.t) / (b.v * b.v)}; }
static inline rd operator/(rd a, double s) { return rd{a.v / s, a.t / s}; }
static inline rd dsqrt(rd a) {
  double q = std::sqrt(a.v);
  return rd{q, a.t / (2.0 * q)};
}
static inline rd dlog(rd a) { return rd{std::log(a.v), a.t / a.v}; }
static inline cd C(cplx v) { return cd{v, cplx(0.0, 0.0)}; }
static inline cd operator+(cd a, cd b) { return cd{a.v + b.v, a.t + b.t}; }
static inline cd operator-(cd a, cd b) { return cd{a.v - b.v, a.t - b.t}; }
static inline cd operator-(cd a) { return cd{-a.v, -a.t}; }
static inline cd operator*(cd a, cd b) { return cd{a.v * b.v, a.t * b.v + a.v * b.t}; }
static inline cd operator*(cd a, rd b) { return cd{a.v * b.v, a.t * b.v + a.v * b.t}; }
static inline cd operator*(rd b, cd a) { return a * b; }
static inline cd operator*(cplx s, cd a) { return cd{s * a.v, s * a.t}; }
static inline cd operator*(double s, cd a) { return cd{s * a.v, s * a.t}; }
static inline cd operator/(cd a, double s) { return cd{a.v / s, a.t / s}; }
static inline cd operator+(cd a, rd b) { return cd{a.v + b.v, a.t + b.t}; }
static inline cd operator-(cd a, rd b) { return cd{a.v - b.v, a.t - b.t}; }
static inline cd operator+(rd b, cd a) { return a + b; }

struct HankD {
  cd h0, h1, f1;
};
static HankD hankel_dual(const Hank& h, rd z) {
  HankD o;
  o.h0 = cd{h.h0, -h.h1 * z.t};
  o.h1 = cd{h.h1, (h.h0 - h.h1 / z.v) * z.t};
  o.f1 = cd{h.f1, (h.h0 - 2.0 * h.f1) / z.v * z.t};
  return o;
}

struct GeomT {  // node arrays and one tangent direction of them
  const double *x, *y, *nx, *ny, *w, *kappa;
  const double *tx, *ty, *tnx, *tny, *tw, *tkappa;
};
struct ParamsT {
  double k0;
  rd k1;
  double eps0;
  rd eps1;
};

static void pair_block_offdiag_dual(const GeomT& g, const ParamsT& p, int64_t i, int64_t j,
                                    const Hank& ha, const Hank& hb, cd a[2][2]) {
  const cplx I1(0.0, 1.0);
  rd dx = rd{g.x[i], g.tx[i]} - rd{g.x[j], g.tx[j]};
  rd dy = rd{g.y[i], g.ty[i]} - rd{g.y[j], g.ty[j]};
  rd nxi{g.nx[i], g.tnx[i]}, nyi{g.ny[i], g.tny[i]}, nxj{g.nx[j], g.tnx[j]}, nyj{g.ny[j], g.tny[j]};
  rd r2 = dx * dx + dy * dy;
  rd r = dsqrt(r2);
  rd z0 = p.k0 * r;
  rd z1 = p.k1 * r;
  rd dny = dx * nxj + dy * nyj;
  rd dnx = dx * nxi + dy * nyi;
  rd nn = nxi * nxj + nyi * nyj;
  rd c = (dnx * dny) / r2;
  HankD A = hankel_dual(ha, z0);
  HankD B = hankel_dual(hb, z1);
  cd G0 = (0.25 * I1) * A.h0;
  cd G1 = (0.25 * I1) * B.h0;
  cd Dy0 = (0.25 * I1 * p.k0) * (A.h1 * (dny / r));
  cd Dy1 = (0.25 * I1) * (p.k1 * (B.h1 * (dny / r)));
  cd Dx0 = (-0.25 * I1 * p.k0) * (A.h1 * (dnx / r));
  cd Dx1 = (-0.25 * I1) * (p.k1 * (B.h1 * (dnx / r)));
  double q0 = p.k0 * p.k0;
  rd q1 = p.k1 * p.k1;
  rd m2c = nn - 2.0 * c;
  cd dN = (0.25 * I1) * ((q0 * A.h0 - q1 * B.h0) * c + (q0 * A.f1 - q1 * B.f1) * m2c);
  cplx alpha = I1 / p.k0;
  rd wj{g.w[j], g.tw[j]};
  a[0][0] = wj * Dy1;
  a[0][1] = -(p.eps1 * (wj * G1));
  a[1][0] = wj * (Dy0 + alpha * dN);
  a[1][1] = wj * ((-p.eps0) * G0 - alpha * (p.eps0 * Dx0 - p.eps1 * Dx1));
}

static void pair_block_diag_dual(const GeomT& g, const ParamsT& p, int64_t i, cd a[2][2]) {
  const cplx I1(0.0, 1.0);
  rd wi{g.w[i], g.tw[i]};
  rd kap{g.kappa[i], g.tkappa[i]};
  auto S = [&](rd k) {
    return wi * (C(0.25 * I1) - (R(EULER_GAMMA) + dlog(k * wi / (4.0 * PI))) / (2.0 * PI));
  };
  auto f = [&](rd k) { return k * k * (dlog(k * wi / (4.0 * PI)) + R(EULER_GAMMA - 0.5)); };
  rd k0 = R(p.k0);
  rd Dd = -1.0 * (wi * kap) / (4.0 * PI);
  cd dN = wi * (C(I1 / 8.0) * (k0 * k0 - p.k1 * p.k1) - C(cplx(1.0, 0.0)) * ((f(k0) - f(p.k1)) / (4.0 * PI)));
  cplx alpha = I1 / p.k0;
  a[0][0] = C(cplx(0.5, 0.0)) + Dd;
  a[0][1] = -(p.eps1 * S(p.k1));
  a[1][0] = C(cplx(-0.5, 0.0)) + Dd + alpha * dN;
  a[1][1] = (-p.eps0) * S(k0) - alpha * (C(cplx(1.0, 0.0)) * ((R(p.eps0) - p.eps1) * Dd)) -
            alpha * (C(cplx(0.5, 0.0)) * (R(p.eps0) + p.eps1));
}

extern "C" {

// H0, H1 at n arguments; out[4t..4t+3] = Re H0, Im H0, Re H1, Im H1.
int orc_hankel01(const double* z, int64_t n, double* out) {
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t t = 0; t < n; ++t) {
    Hank h = hankel_eval(z[t]);
    out[4 * t + 0] = h.h0.real();
    out[4 * t + 1] = h.h0.imag();
    out[4 * t + 2] = h.h1.real();
    out[4 * t + 3] = h.h1.imag();
  }
  return 0;
}

// F1(z) = H1(z)/z + 2i/(pi z^2); out[2t], out[2t+1] = Re, Im.
int orc_f1(const double* z, int64_t n, double* out) {
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t t = 0; t < n; ++t) {
    Hank h = hankel_eval(z[t]);
    out[2 * t] = h.f1.real();
    out[2 * t + 1] = h.f1.imag();
  }
  return 0;
}

// Entries A[rows, cols] of the 2N x 2N WSBM matrix, unknowns in the paper's block order
// [u ; q] (index r < N: u_r / first equation at node r;  r >= N: q_{r-N} / second equation).
// out: column-major nr x nc complex128 (interleaved re, im), leading dimension nr.
int orc_wsbm_entries(int64_t n, const double* x, const double* y, const double* nx,
                     const double* ny, const double* w, const double* kappa, double k0,
                     double k1, double eps0, double eps1, const int64_t* rows, int64_t nr,
                     const int64_t* cols, int64_t nc, double* out) {
  Geom g{n, x, y, nx, ny, w, kappa};
  Params p{k0, k1, eps0, eps1};
  for (int64_t t = 0; t < nr; ++t)
    if (rows[t] < 0 || rows[t] >= 2 * n) return -1;
  for (int64_t t = 0; t < nc; ++t)
    if (cols[t] < 0 || cols[t] >= 2 * n) return -1;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t cc = 0; cc < nc; ++cc) {
    int64_t j = cols[cc] % n, b = cols[cc] / n;
    for (int64_t rr = 0; rr < nr; ++rr) {
      int64_t i = rows[rr] % n, a = rows[rr] / n;
      cplx blk[2][2];
      pair_block(g, p, i, j, blk);
      cplx v = blk[a][b];
      out[2 * (cc * nr + rr)] = v.real();
      out[2 * (cc * nr + rr) + 1] = v.imag();
    }
  }
  return 0;
}

// The full dense 2N x 2N matrix, paper order, column-major complex128.
int orc_wsbm_dense(int64_t n, const double* x, const double* y, const double* nx, const double* ny,
                   const double* w, const double* kappa, double k0, double k1, double eps0,
                   double eps1, double* out) {
  Geom g{n, x, y, nx, ny, w, kappa};
  Params p{k0, k1, eps0, eps1};
  int64_t ld2 = 2 * n;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t j = 0; j < n; ++j) {
    for (int64_t i = 0; i < n; ++i) {
      cplx blk[2][2];
      pair_block(g, p, i, j, blk);
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
          int64_t r = a * n + i, c = b * n + j;
          out[2 * (c * ld2 + r)] = blk[a][b].real();
          out[2 * (c * ld2 + r) + 1] = blk[a][b].imag();
        }
    }
  }
  return 0;
}

// Dense 2N x 2N matrix of form 1 (eq. bm) or 2 (eq. pmchwt, columns (u, q)), paper order
// [u ; q] columns and [eq1 ; eq2] rows as orc_wsbm_dense; form 0 is eq. (weakly_bm).
int orc_form_dense(int64_t n, const double* x, const double* y, const double* nx, const double* ny,
                   const double* w, const double* kappa, double k0, double k1, double eps0,
                   double eps1, int32_t form, double* out) {
  if (form < 0 || form > 2) return -1;
  Geom g{n, x, y, nx, ny, w, kappa};
  Params p{k0, k1, eps0, eps1};
  int64_t ld2 = 2 * n;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t j = 0; j < n; ++j) {
    for (int64_t i = 0; i < n; ++i) {
      cplx blk[2][2];
      if (form == 0)
        pair_block(g, p, i, j, blk);
      else
        form_block(g, p, form, i, j, blk);
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
          int64_t r = a * n + i, c = b * n + j;
          out[2 * (c * ld2 + r)] = blk[a][b].real();
          out[2 * (c * ld2 + r) + 1] = blk[a][b].imag();
        }
    }
  }
  return 0;
}

// The four layer operators at k0 and k1 as dense N x N matrices (one-point corrected
// diagonal as above, weights folded in): out = [S0, S1, D0, D1, D*0, D*1, N0, N1], each N x N
// column-major complex128.
int orc_layer_ops(int64_t n, const double* x, const double* y, const double* nx, const double* ny,
                  const double* w, const double* kappa, double k0, double k1, double* out) {
  Geom g{n, x, y, nx, ny, w, kappa};
  Params p{k0, k1, 1.0, 1.0};
  const int64_t nn = n * n;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i) {
      Ops o;
      if (i == j)
        pair_ops_diag(g, p, i, o);
      else
        pair_ops_offdiag(g, p, i, j, o);
      const cplx v[8] = {o.S[0], o.S[1], o.D[0], o.D[1], o.Dx[0], o.Dx[1], o.N[0], o.N[1]};
      for (int t = 0; t < 8; ++t) {
        out[2 * (t * nn + j * n + i)] = v[t].real();
        out[2 * (t * nn + j * n + i) + 1] = v[t].imag();
      }
    }
  return 0;
}

// Matrix-free product y = A x for the dense system (paper order), x, y complex128 of length
// 2N, nrhs columns (column-major, leading dimension 2N).
int orc_wsbm_matvec(int64_t n, const double* x, const double* y, const double* nx, const double* ny,
                    const double* w, const double* kappa, double k0, double k1, double eps0,
                    double eps1, const double* xin, int64_t nrhs, double* yout) {
  Geom g{n, x, y, nx, ny, w, kappa};
  Params p{k0, k1, eps0, eps1};
  const cplx* X = reinterpret_cast<const cplx*>(xin);
  cplx* Y = reinterpret_cast<cplx*>(yout);
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t i = 0; i < n; ++i) {
    std::vector<cplx> acc(2 * nrhs, cplx(0.0, 0.0));
    for (int64_t j = 0; j < n; ++j) {
      cplx blk[2][2];
      pair_block(g, p, i, j, blk);
      for (int64_t c = 0; c < nrhs; ++c) {
        const cplx* xc = X + c * 2 * n;
        acc[2 * c] += blk[0][0] * xc[j] + blk[0][1] * xc[n + j];
        acc[2 * c + 1] += blk[1][0] * xc[j] + blk[1][1] * xc[n + j];
      }
    }
    for (int64_t c = 0; c < nrhs; ++c) {
      Y[c * 2 * n + i] = acc[2 * c];
      Y[c * 2 * n + n + i] = acc[2 * c + 1];
    }
  }
  return 0;
}

// Proxy circle of a set of nodes: centre = midpoint of the bounding box, R = largest distance
// from the centre to a node, proxy radius rho = ratio * R.  out: cx, cy, R, rho.
int orc_proxy_circle(const double* x, const double* y, const int64_t* nodes, int64_t m,
                     double ratio, double* out) {
  if (m <= 0) return -1;
  double xmin = x[nodes[0]], xmax = xmin, ymin = y[nodes[0]], ymax = ymin;
  for (int64_t t = 1; t < m; ++t) {
    double a = x[nodes[t]], b = y[nodes[t]];
    if (a < xmin) xmin = a;
    if (a > xmax) xmax = a;
    if (b < ymin) ymin = b;
    if (b > ymax) ymax = b;
  }
  double cx = 0.5 * (xmin + xmax), cy = 0.5 * (ymin + ymax);
  double R = 0.0;
  for (int64_t t = 0; t < m; ++t) {
    double dx = x[nodes[t]] - cx, dy = y[nodes[t]] - cy;
    double d = std::sqrt(dx * dx + dy * dy);
    if (d > R) R = d;
  }
  out[0] = cx;
  out[1] = cy;
  out[2] = R;
  out[3] = ratio * R;
  return 0;
}

// Proxy points p_m = c + rho (cos t_m, sin t_m), t_m = 2 pi m / P, outward normals.
static void proxy_point(double cx, double cy, double rho, int64_t P, int64_t m, double* px,
                        double* py, double* pnx, double* pny) {
  double t = 2.0 * PI * (double)m / (double)P;
  double ct = std::cos(t), st = std::sin(t);
  *pnx = ct;
  *pny = st;
  *px = cx + rho * ct;
  *py = cy + rho * st;
}

// Row proxy block: rows = equation indices (paper order) of a box, columns = 2P proxy
// sources (k1 sources first, then k0 sources), each scaled by the proxy weight 2 pi rho / P.
// out: column-major nr x 2P complex128.
// The same for the equations of form 1 (eq. bm) or 2 (eq. pmchwt); form 0 is the block above.
// The column block is the same for all three: their far interactions depend on a box's
// unknowns only through the k0 and k1 potentials psi0, psi1.
int orc_proxy_row_block_form(int64_t n, const double* x, const double* y, const double* nx,
                             const double* ny, const double* w, const double* kappa, double k0,
                             double k1, double eps0, double eps1, int32_t form, const int64_t* rows,
                             int64_t nr, double cx, double cy, double rho, int64_t P, double* out) {
  if (form < 0 || form > 2) return -1;
  Geom g{n, x, y, nx, ny, w, kappa};
  Params p{k0, k1, eps0, eps1};
  double pw = 2.0 * PI * rho / (double)P;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t m = 0; m < P; ++m) {
    double px, py, pnx, pny;
    proxy_point(cx, cy, rho, P, m, &px, &py, &pnx, &pny);
    for (int64_t rr = 0; rr < nr; ++rr) {
      int64_t i = rows[rr] % n, a = rows[rr] / n;
      cplx e[2][2];
      proxy_row_entries(g, p, i, px, py, pnx, pny, pw, e, form);
      for (int s = 0; s < 2; ++s) {
        int64_t cc = s * P + m;
        out[2 * (cc * nr + rr)] = e[a][s].real();
        out[2 * (cc * nr + rr) + 1] = e[a][s].imag();
      }
    }
  }
  return 0;
}

int orc_proxy_row_block(int64_t n, const double* x, const double* y, const double* nx,
                        const double* ny, const double* w, const double* kappa, double k0,
                        double k1, double eps0, double eps1, const int64_t* rows, int64_t nr,
                        double cx, double cy, double rho, int64_t P, double* out) {
  Geom g{n, x, y, nx, ny, w, kappa};
  Params p{k0, k1, eps0, eps1};
  double pw = 2.0 * PI * rho / (double)P;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t m = 0; m < P; ++m) {
    double px, py, pnx, pny;
    proxy_point(cx, cy, rho, P, m, &px, &py, &pnx, &pny);
    for (int64_t rr = 0; rr < nr; ++rr) {
      int64_t i = rows[rr] % n, a = rows[rr] / n;
      cplx e[2][2];
      proxy_row_entries(g, p, i, px, py, pnx, pny, pw, e);
      for (int s = 0; s < 2; ++s) {
        int64_t cc = s * P + m;
        out[2 * (cc * nr + rr)] = e[a][s].real();
        out[2 * (cc * nr + rr) + 1] = e[a][s].imag();
      }
    }
  }
  return 0;
}

// Column proxy block: rows = 2P proxy evaluations (psi1 at the P points, then psi0), columns =
// unknown indices (paper order) of a box.  out: column-major 2P x nc complex128.
int orc_proxy_col_block(int64_t n, const double* x, const double* y, const double* nx,
                        const double* ny, const double* w, const double* kappa, double k0,
                        double k1, double eps0, double eps1, const int64_t* cols, int64_t nc,
                        double cx, double cy, double rho, int64_t P, double* out) {
  Geom g{n, x, y, nx, ny, w, kappa};
  Params p{k0, k1, eps0, eps1};
  int64_t ldo = 2 * P;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t cc = 0; cc < nc; ++cc) {
    int64_t j = cols[cc] % n, b = cols[cc] / n;
    for (int64_t m = 0; m < P; ++m) {
      double px, py, pnx, pny;
      proxy_point(cx, cy, rho, P, m, &px, &py, &pnx, &pny);
      cplx e[2][2];
      proxy_col_entries(g, p, j, px, py, e);
      for (int s = 0; s < 2; ++s) {
        int64_t rr = s * P + m;
        out[2 * (cc * ldo + rr)] = e[s][b].real();
        out[2 * (cc * ldo + rr) + 1] = e[s][b].imag();
      }
    }
  }
  return 0;
}


// Directional derivatives of the bilinear form lam^T A x along ntan tangent directions of the
// inputs: out[t] = sum_{r,c} lam_r (dA_rc / ds_t) x_c (complex), paper order for lam (equation
// index) and x (unknown index), both complex128 of length 2N.  tan: ntan x 6 x N doubles, the
// tangent of (x, y, nx, ny, w, kappa); tk1, teps1: ntan tangents of k1 and eps1.
int orc_wsbm_bilinear_tangent(int64_t n, const double* x, const double* y, const double* nx,
                              const double* ny, const double* w, const double* kappa, double k0,
                              double k1, double eps0, double eps1, const double* lam,
                              const double* xv, int64_t ntan, const double* tan,
                              const double* tk1, const double* teps1, double* out) {
  const cplx* L = reinterpret_cast<const cplx*>(lam);
  const cplx* X = reinterpret_cast<const cplx*>(xv);
  std::vector<cplx> acc((size_t)ntan, cplx(0.0, 0.0));
#pragma omp parallel
  {
    std::vector<cplx> mine((size_t)ntan, cplx(0.0, 0.0));
#pragma omp for schedule(dynamic, 1)
    for (int64_t i = 0; i < n; ++i) {
      for (int64_t j = 0; j < n; ++j) {
        Hank ha{}, hb{};
        if (i != j) {
          double dx = x[i] - x[j], dy = y[i] - y[j];
          double r = std::sqrt(dx * dx + dy * dy);
          ha = hankel_eval(k0 * r);
          hb = hankel_eval(k1 * r);
        }
        for (int64_t t = 0; t < ntan; ++t) {
          const double* tv = tan + t * 6 * n;
          GeomT g{x, y, nx, ny, w, kappa, tv, tv + n, tv + 2 * n, tv + 3 * n, tv + 4 * n, tv + 5 * n};
          ParamsT p{k0, rd{k1, tk1[t]}, eps0, rd{eps1, teps1[t]}};
          cd blk[2][2];
          if (i == j)
            pair_block_diag_dual(g, p, i, blk);
          else
            pair_block_offdiag_dual(g, p, i, j, ha, hb, blk);
          cplx s(0.0, 0.0);
          for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) s += L[a * n + i] * blk[a][b].t * X[b * n + j];
          mine[t] += s;
        }
      }
    }
#pragma omp critical
    for (int64_t t = 0; t < ntan; ++t) acc[t] += mine[t];
  }
  for (int64_t t = 0; t < ntan; ++t) {
    out[2 * t] = acc[t].real();
    out[2 * t + 1] = acc[t].imag();
  }
  return 0;
}


// Field off the curve from the boundary densities by the integral representations (the paper
// notes that u and q on the curve give the solution in the domains through them):
//   exterior x:  u_sc(x) = D_k0[u](x) - eps0 S_k0[q](x)   (scattered part; total = u_in + u_sc)
//   interior x:  u(x)    = eps1 S_k1[q](x) - D_k1[u](x)
// with S_k[f](x) = sum_j w_j G_k(x, y_j) f_j, D_k[f](x) = sum_j w_j dG_k(x, y_j)/dn_y f_j.
// The side of x is decided by the crossing-number test of the closed polygon through the nodes.
// u, q: N x nrhs complex128 (column-major); out: nt x nrhs complex128; inside: nt int32.
int orc_field(int64_t n, const double* x, const double* y, const double* nx, const double* ny,
              const double* w, const double* kappa, double k0, double k1, double eps0,
              double eps1, const double* u, const double* q, int64_t nrhs, const double* tx,
              const double* ty, int64_t nt, double* out, int32_t* inside) {
  (void)kappa;
  const cplx* U = reinterpret_cast<const cplx*>(u);
  const cplx* Q = reinterpret_cast<const cplx*>(q);
  cplx* O = reinterpret_cast<cplx*>(out);
  const cplx I1(0.0, 1.0);
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t t = 0; t < nt; ++t) {
    // crossing number of the ray from (tx, ty) towards +x
    int cross = 0;
    for (int64_t j = 0; j < n; ++j) {
      int64_t k = (j + 1) % n;
      bool a = y[j] > ty[t], b = y[k] > ty[t];
      if (a != b) {
        double xc = x[j] + (ty[t] - y[j]) * (x[k] - x[j]) / (y[k] - y[j]);
        if (xc > tx[t]) cross ^= 1;
      }
    }
    inside[t] = cross;
    const double k = cross ? k1 : k0;
    for (int64_t c = 0; c < nrhs; ++c) {
      cplx acc(0.0, 0.0);
      for (int64_t j = 0; j < n; ++j) {
        double dx = tx[t] - x[j], dy = ty[t] - y[j];
        double r = std::sqrt(dx * dx + dy * dy);
        Hank h = hankel_eval(k * r);
        cplx G = 0.25 * I1 * h.h0;
        cplx Dy = 0.25 * I1 * k * h.h1 * ((dx * nx[j] + dy * ny[j]) / r);
        cplx uj = U[c * n + j], qj = Q[c * n + j];
        if (cross)
          acc += w[j] * (eps1 * G * qj - Dy * uj);
        else
          acc += w[j] * (Dy * uj - eps0 * G * qj);
      }
      O[c * nt + t] = acc;
    }
  }
  return 0;
}

}  // extern "C"
