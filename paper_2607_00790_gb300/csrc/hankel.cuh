// Device evaluation of the Hankel functions H0^(1), H1^(1) (the kernels of every layer
// potential in eq. (weakly_bm): G_k = (i/4) H0^(1)(k r) and its normal derivatives).
//
// GB300 executes FP64 at 1/64 of the FP32 rate, so the evaluator is built to spend few FP64
// instructions per argument:
//   z < 1.5     ascending series in z^2/4 (A&S 9.1.10, 9.1.11, 9.1.13); the 1/z pole of Y1 is kept
//               apart so F1 = H1/z + 2i/(pi z^2) is formed without cancellation;
//   z >= 1.5    H_nu = sqrt(2/(pi z)) (P_nu + i Q_nu) e^{i(z - pi/4 - nu pi/2)};
//               P_nu - 1, Q_nu are degree-10 polynomials in u = 1/z on seven intervals up to
//               z = 20 (the functions are smooth in 1/z), and degree-6 polynomials in 1/z^2
//               beyond (P_nu - 1 and z Q_nu), evaluated there in two-float (hi + lo FP32)
//               arithmetic on the FP32 pipe: they are small corrections, so 48 significant
//               bits give them an absolute error below 1e-17;
//   phase       z - pi/4 is reduced by multiples of pi/2 (Cody-Waite with a two-part pi/2 and
//               fused multiply-adds) and sin/cos of the remainder |w| <= pi/4 come from fitted
//               polynomials, so no rounding of z - pi/4 enters the phase.
// The interval is chosen by comparing the high 32-bit word of z as an integer (integer pipe).
// All coefficients are fitted by gen_hankel_coeffs.py (50-digit arithmetic) and checked there.
//
// Mixed evaluator (WSBM_MIXED): the phase is reduced in FP64 (z - 2 pi n, two-part 2 pi), then
// sin/cos of the remainder (rounded to FP32: phase error <= 2e-7), sqrt(2/(pi z)) and P, Q
// (degree-4 fits in 1/z, degree-2 in 1/z^2) are FP32.  Arguments below 1.5 fall back to the FP64
// evaluator.  Amplitude-only mixed evaluator (WSBM_MIXED_FINE): the FP64 evaluator with only
// P - 1 and Q from the FP32 tables (relative error of H ~ 2e-8).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "hankel_coeffs.inc"

#define WSBM_PI 3.14159265358979323846
#define WSBM_2_OVER_PI 0.63661977236758134308
#define WSBM_SQRT_2_OVER_PI 0.79788456080286535588
#define WSBM_INV_SQRT2 0.70710678118654752440
#define WSBM_EULER 0.57721566490153286061

struct Hk {
  double h0r, h0i, h1r, h1i, f1r, f1i;
};

struct HkF {
  float h0r, h0i, h1r, h1i;
};

// Coefficient tables staged in shared memory by every kernel that evaluates Hankel values
// (divergent interval indices within a warp would serialise constant-bank reads).
struct HkTables {
  double iv[HK_NIV][2];
  double fit[HK_NIV][4][HK_DEG + 1];
  double asy[4][HK_DEG_T + 1];
  double ser[4][HK_NSER];
  double sn[HK_DEG_SC + 1];
  double cs[HK_DEG_SC + 1];
  float ivf[HK_NIV][2];
  float fitf[HK_NIV][4][HKF_DEG + 1];
  float asyf[4][HKF_DEG_T + 1];
  float asyh[4][HK_DEG_T + 1], asyl[4][HK_DEG_T + 1];  // hk_asy as two-float sums (hi + lo)
};

template <class T>
__device__ __forceinline__ void hk_copy(T* dst, const T* src, int n) {
  for (int k = threadIdx.x; k < n; k += blockDim.x) dst[k] = src[k];
}

__device__ __forceinline__ void hk_stage_tables(HkTables* t) {
  hk_copy(&t->iv[0][0], &hk_iv[0][0], HK_NIV * 2);
  hk_copy(&t->fit[0][0][0], &hk_fit[0][0][0], HK_NIV * 4 * (HK_DEG + 1));
  hk_copy(&t->asy[0][0], &hk_asy[0][0], 4 * (HK_DEG_T + 1));
  hk_copy(&t->ser[0][0], &hk_ser[0][0], 4 * HK_NSER);
  hk_copy(t->sn, hk_sin, HK_DEG_SC + 1);
  hk_copy(t->cs, hk_cos, HK_DEG_SC + 1);
  hk_copy(&t->fitf[0][0][0], &hkf_fit[0][0][0], HK_NIV * 4 * (HKF_DEG + 1));
  hk_copy(&t->asyf[0][0], &hkf_asy[0][0], 4 * (HKF_DEG_T + 1));
  for (int k = threadIdx.x; k < HK_NIV * 2; k += blockDim.x)
    (&t->ivf[0][0])[k] = (float)(&hk_iv[0][0])[k];
  for (int k = threadIdx.x; k < 4 * (HK_DEG_T + 1); k += blockDim.x) {
    const double c = (&hk_asy[0][0])[k];
    const float h = __double2float_rn(c);
    (&t->asyh[0][0])[k] = h;
    (&t->asyl[0][0])[k] = __double2float_rn(c - (double)h);
  }
}

// Exact widening of a normal FP32 value (or zero) to FP64 by integer operations (rebias the
// exponent, shift the fraction), which keeps the conversion off the FP64 pipe.
__device__ __forceinline__ double f2d_exact(float f) {
  const unsigned int b = __float_as_uint(f);
  const unsigned int e = (b >> 23) & 0xFFu;
  if (e == 0u) return 0.0;  // zero (the two-float parts here are never subnormal)
  const unsigned long long d = ((unsigned long long)(b & 0x80000000u) << 32) |
                               ((unsigned long long)(e + 896u) << 52) |
                               ((unsigned long long)(b & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)d);
}

// Two-float (hi + lo, about 48 significant bits) Horner step r <- r s + c on the FP32 pipe:
// exact product hi part by FMA, Knuth two-sum with the coefficient, renormalisation.
__device__ __forceinline__ void ff_step(float& rh, float& rl, float sh, float sl, float ch, float cl) {
  const float ph = rh * sh;
  float pl = fmaf(rh, sh, -ph);
  pl = fmaf(rh, sl, pl);
  pl = fmaf(rl, sh, pl);
  const float th = ph + ch;
  const float bb = th - ph;
  float tl = (ph - (th - bb)) + (ch - bb);
  tl = tl + (pl + cl);
  rh = th + tl;
  rl = tl - (rh - th);
}

// sum_k c_k s^k of an asymptotic table row: degrees 4.. in FP32 (they carry below 1e-7 of the
// leading term), degrees 3 to 0 in two-float arithmetic.
__device__ __forceinline__ void hk_asy_ff(const HkTables& T, int row, float sh, float sl, float* rh,
                                          float* rl) {
  float t = T.asyh[row][HK_DEG_T];
#pragma unroll
  for (int k = HK_DEG_T - 1; k >= 4; --k) t = fmaf(t, sh, T.asyh[row][k]);
  float h = t, l = 0.0f;
#pragma unroll
  for (int k = 3; k >= 0; --k) ff_step(h, l, sh, sl, T.asyh[row][k], T.asyl[row][k]);
  *rh = h;
  *rl = l;
}

template <int N>
__device__ __forceinline__ double hk_horner(const double* c, double s) {
  double r = c[N - 1];
#pragma unroll
  for (int k = N - 2; k >= 0; --k) r = fma(r, s, c[k]);
  return r;
}

template <int N>
__device__ __forceinline__ float hk_hornerf(const float* c, float s) {
  float r = c[N - 1];
#pragma unroll
  for (int k = N - 2; k >= 0; --k) r = fmaf(r, s, c[k]);
  return r;
}

// Interval index for HK_Z_SERIES <= z < HK_Z_ASYM from the high word of z (integer compares:
// the bounds have zero low words, and positive doubles order like their bit patterns).
__device__ __forceinline__ int hk_interval_hi(int hi) {
  const int lim[HK_NIV - 1] = HK_IV_HI;
  int iv = 0;
#pragma unroll
  for (int k = 0; k < HK_NIV - 1; ++k) iv += (hi >= lim[k]) ? 1 : 0;
  return iv;
}
__device__ __forceinline__ int hk_interval(double z) { return hk_interval_hi(__double2hiint(z)); }

// e^{i(z - pi/4)} = E + iF.  z - pi/4 = w + k pi/2 with |w| <= pi/4: k = rint(2z/pi - 1/2),
// w = z - (k + 1/2) pi/2 by two fused multiply-adds with a two-part pi/2, then
// e^{i(w + k pi/2)} = i^k (cos w + i sin w).
__device__ __forceinline__ void hk_phase(const HkTables& T, double z, double* E, double* F) {
  const double MAGIC = 6755399441055744.0;  // 1.5 * 2^52: adding it rounds to an integer
  double t = fma(z, HK_2_OVER_PI, -0.5);
  double tm = __dadd_rn(t, MAGIC);
  int q = __double2loint(tm);
  double k = __dsub_rn(tm, MAGIC);
  double m = k + 0.5;
  double w = fma(-m, HK_PIO2_HI, z);
  w = fma(-m, HK_PIO2_LO, w);
  double v = w * w;
  double s = fma(w * v, hk_horner<HK_DEG_SC + 1>(T.sn, v), w);
  double c = fma(v, fma(v, hk_horner<HK_DEG_SC + 1>(T.cs, v), -0.5), 1.0);
  double a = (q & 1) ? s : c;
  double b = (q & 1) ? c : s;
  *E = ((q + 1) & 2) ? -a : a;  // negative for k = 1, 2 (mod 4)
  *F = (q & 2) ? -b : b;        // negative for k = 2, 3
}

// Small argument: ascending series (u_in = 1/z).
__device__ __forceinline__ void hk_series(const HkTables& T, double z, double iz, Hk& o) {
  double u = 0.25 * z * z;
  double j0 = hk_horner<HK_NSER>(T.ser[0], u);
  double j1 = 0.5 * z * hk_horner<HK_NSER>(T.ser[1], u);
  double s0 = hk_horner<HK_NSER>(T.ser[2], u);
  double s1 = hk_horner<HK_NSER>(T.ser[3], u);
  double L = log(0.5 * z);
  double y0 = WSBM_2_OVER_PI * (fma(L + WSBM_EULER, j0, s0));
  // Y1 + 2/(pi z): pole-free part
  double y1h = WSBM_2_OVER_PI * L * j1 - (0.5 / WSBM_PI) * z * s1;
  o.h0r = j0;
  o.h0i = y0;
  o.h1r = j1;
  o.h1i = y1h - WSBM_2_OVER_PI * iz;
  o.f1r = j1 * iz;
  o.f1i = y1h * iz;
}

// P_nu - 1 (pm0, pm1) and Q_nu for z >= HK_Z_SERIES, u = 1/z.
__device__ __forceinline__ void hk_pq(const HkTables& T, int zhi, double u, double* pm0,
                                      double* Q0, double* pm1, double* Q1) {
  if (zhi < HK_ASYM_HI) {
    int iv = hk_interval_hi(zhi);
    double s = (u - T.iv[iv][0]) * T.iv[iv][1];
    *pm0 = hk_horner<HK_DEG + 1>(T.fit[iv][0], s);
    *Q0 = hk_horner<HK_DEG + 1>(T.fit[iv][1], s);
    *pm1 = hk_horner<HK_DEG + 1>(T.fit[iv][2], s);
    *Q1 = hk_horner<HK_DEG + 1>(T.fit[iv][3], s);
  } else {
    // z >= 20: P - 1 (|.| < 4e-4) and z Q in two-float arithmetic on the FP32 pipe; the
    // absolute error of P and Q stays below 1e-17
    const double s = (u * u - HK_T_C) * HK_T_IH;
    const float sh = __double2float_rn(s), sl = __double2float_rn(s - f2d_exact(sh));
    float h, l;
    hk_asy_ff(T, 0, sh, sl, &h, &l);
    *pm0 = f2d_exact(h) + f2d_exact(l);
    hk_asy_ff(T, 1, sh, sl, &h, &l);
    *Q0 = u * (f2d_exact(h) + f2d_exact(l));
    hk_asy_ff(T, 2, sh, sl, &h, &l);
    *pm1 = f2d_exact(h) + f2d_exact(l);
    hk_asy_ff(T, 3, sh, sl, &h, &l);
    *Q1 = u * (f2d_exact(h) + f2d_exact(l));
  }
}

// P_nu - 1 and Q_nu from the FP32 tables (amplitude-only mixed precision, WSBM_MIXED_FINE):
// the values are small corrections (|P - 1| ~ 1/(8z)^2, |Q| ~ 1/(8z)), so FP32 rounding of them
// and the 2e-8 absolute error of the FP32 fits set the relative error of H; the phase factor
// and everything after stay FP64.
__device__ __forceinline__ void hk_pq_f32(const HkTables& T, int zhi, double u, double* pm0,
                                          double* Q0, double* pm1, double* Q1) {
  const float uf = (float)u;
  float a, b, c, d;
  if (zhi < HK_ASYM_HI) {
    int iv = hk_interval_hi(zhi);
    float s = (uf - T.ivf[iv][0]) * T.ivf[iv][1];
    a = hk_hornerf<HKF_DEG + 1>(T.fitf[iv][0], s);
    b = hk_hornerf<HKF_DEG + 1>(T.fitf[iv][1], s);
    c = hk_hornerf<HKF_DEG + 1>(T.fitf[iv][2], s);
    d = hk_hornerf<HKF_DEG + 1>(T.fitf[iv][3], s);
  } else {
    float s = (uf * uf - (float)HK_T_C) * (float)HK_T_IH;
    a = hk_hornerf<HKF_DEG_T + 1>(T.asyf[0], s);
    b = uf * hk_hornerf<HKF_DEG_T + 1>(T.asyf[1], s);
    c = hk_hornerf<HKF_DEG_T + 1>(T.asyf[2], s);
    d = uf * hk_hornerf<HKF_DEG_T + 1>(T.asyf[3], s);
  }
  *pm0 = (double)a;
  *Q0 = (double)b;
  *pm1 = (double)c;
  *Q1 = (double)d;
}

// FP64 H0, H1 and (WITH_F1) F1 = H1/z + 2i/(pi z^2) at z > 0, given rs ~ 1/sqrt(z) to a few
// ulp (callers derive it for both wavenumbers from one reciprocal square root).  PQ32: the
// amplitude corrections P - 1, Q come from the FP32 tables (hk_pq_f32) for z >= 1.5.
template <bool WITH_F1 = true, bool PQ32 = false>
__device__ __forceinline__ void hankel_fp64_rs(const HkTables& T, double z, double rs, Hk& o) {
  double u = rs * rs;
  const int zhi = __double2hiint(z);
  if (zhi < HK_SERIES_HI) {
    hk_series(T, z, u, o);
    return;
  }
  double A = WSBM_SQRT_2_OVER_PI * rs;
  double E, F;
  hk_phase(T, z, &E, &F);
  double pm0, Q0, pm1, Q1;
  if (PQ32)
    hk_pq_f32(T, zhi, u, &pm0, &Q0, &pm1, &Q1);
  else
    hk_pq(T, zhi, u, &pm0, &Q0, &pm1, &Q1);
  double P0 = fma(A, pm0, A), AQ0 = A * Q0;
  double P1 = fma(A, pm1, A), AQ1 = A * Q1;
  o.h0r = fma(P0, E, -AQ0 * F);
  o.h0i = fma(P0, F, AQ0 * E);
  // e^{i(z - 3pi/4)} = -i (E + iF) = F - iE
  o.h1r = fma(P1, F, AQ1 * E);
  o.h1i = fma(AQ1, F, -P1 * E);
  if (WITH_F1) {
    o.f1r = o.h1r * u;
    o.f1i = fma(WSBM_2_OVER_PI * u, u, o.h1i * u);
  }
}

__device__ __forceinline__ void hankel_fp64(const HkTables& T, double z, Hk& o) {
  hankel_fp64_rs<true>(T, z, rsqrt(z), o);
}

// Mixed: FP64 phase reduction, FP32 amplitude.  Valid for z >= HK_Z_SERIES.  Also returns
// D = H1 + i H0 = sqrt(2/(pi z)) e^{i(z - pi/4)} [(Q1 - Q0) + i(P0 - P1)], formed from the small
// differences of P and Q so that it keeps its relative accuracy (H1 ~ -i H0 for large z, and
// combined-field sources cancel to leading order).
// rsz: 1/sqrt(z) in FP32 (callers derive it from one FP32 reciprocal square root per pair).
__device__ __forceinline__ void hankel_mixed_large(const HkTables& T, double z, float rsz, HkF& o,
                                                   float* Dr = nullptr, float* Di = nullptr) {
  // z - 2 pi n with 2 pi split into a short head (n * head exact) and a tail
  double n = rint(z * (0.5 / WSBM_PI));
  double y = fma(-n, HK_TWO_PI_HI, z);
  y = fma(-n, HK_TWO_PI_LO, y);
  float yf = (float)y;
  float sn, cs;
  sincosf(yf, &sn, &cs);
  float rs = rsz;
  float u = rs * rs;
  float A = (float)WSBM_SQRT_2_OVER_PI * rs;
  float E = (cs + sn) * (float)WSBM_INV_SQRT2;
  float F = (sn - cs) * (float)WSBM_INV_SQRT2;
  float P0, Q0, P1, Q1;  // P0, P1 hold P - 1 until D is formed
  const int zhi = __double2hiint(z);
  if (zhi < HK_ASYM_HI) {
    int iv = hk_interval_hi(zhi);
    float s = (u - T.ivf[iv][0]) * T.ivf[iv][1];
    P0 = hk_hornerf<HKF_DEG + 1>(T.fitf[iv][0], s);
    Q0 = hk_hornerf<HKF_DEG + 1>(T.fitf[iv][1], s);
    P1 = hk_hornerf<HKF_DEG + 1>(T.fitf[iv][2], s);
    Q1 = hk_hornerf<HKF_DEG + 1>(T.fitf[iv][3], s);
  } else {
    float s = (u * u - (float)HK_T_C) * (float)HK_T_IH;
    P0 = hk_hornerf<HKF_DEG_T + 1>(T.asyf[0], s);
    Q0 = u * hk_hornerf<HKF_DEG_T + 1>(T.asyf[1], s);
    P1 = hk_hornerf<HKF_DEG_T + 1>(T.asyf[2], s);
    Q1 = u * hk_hornerf<HKF_DEG_T + 1>(T.asyf[3], s);
  }
  if (Dr) {
    float dr = Q1 - Q0, di = P0 - P1;
    *Dr = A * (E * dr - F * di);
    *Di = A * (E * di + F * dr);
  }
  P0 += 1.0f;
  P1 += 1.0f;
  o.h0r = A * (P0 * E - Q0 * F);
  o.h0i = A * (P0 * F + Q0 * E);
  o.h1r = A * (P1 * F + Q1 * E);
  o.h1i = A * (Q1 * F - P1 * E);
}
