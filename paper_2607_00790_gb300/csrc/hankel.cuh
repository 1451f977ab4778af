// Device evaluation of the Hankel functions H0^(1), H1^(1) (the kernels of every layer
// potential in eq. (weakly_bm): G_k = (i/4) H0^(1)(k r) and its normal derivatives).
//
// FP64 evaluator, three regimes:
//   z <  3    ascending series in u = z^2/4 (A&S 9.1.10, 9.1.11, 9.1.13); the 1/z pole of Y1
//             is kept apart so F1 = H1/z + 2i/(pi z^2) is formed without cancellation;
//   3 <= z < 20   H_nu = sqrt(2/(pi z)) (P_nu + i Q_nu) e^{i(z - pi/4 - nu pi/2)} with P_nu - 1
//             and Q_nu from piecewise polynomial fits (degree 16 on [a, 1.5a] intervals);
//   z >= 20   the same form with P, Q from the Hankel asymptotic expansion (A&S 9.2.5-9.2.10);
//             the number of terms falls as z grows.
// The phase factor e^{iz} comes from sincos(z) of the exact double z, and e^{-i pi/4} is
// applied as a constant rotation, so no rounding of z - pi/4 enters the phase (one ulp of a
// z near 5e4 would otherwise cost ~4e-12 relative).
//
// Mixed evaluator (WSBM_MIXED): the phase is reduced in FP64 (z - 2 pi n, two-part constant),
// then sin/cos of the reduced phase, the amplitude sqrt(2/(pi z)) and P, Q are FP32 (fits of
// degree 6, three asymptotic terms).  Arguments below 3 fall back to the FP64 evaluator.
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
// (divergent interval indices within a warp make constant-bank reads serialise).
struct HkTables {
  double iv[HK_NIV][4];
  double fit[HK_NIV][4][HK_DEG + 1];
  double asy[4][HK_NASY];
  double ser[4][HK_NSER];
  float fitf[HK_NIV][4][HKF_DEG + 1];
  float asyf[4][3];
};

__device__ __forceinline__ void hk_stage_tables(HkTables* t) {
  const double* src[4] = {&hk_iv[0][0], &hk_fit[0][0][0], &hk_asy[0][0], &hk_ser[0][0]};
  double* dst[4] = {&t->iv[0][0], &t->fit[0][0][0], &t->asy[0][0], &t->ser[0][0]};
  const int cnt[4] = {HK_NIV * 4, HK_NIV * 4 * (HK_DEG + 1), 4 * HK_NASY, 4 * HK_NSER};
  for (int a = 0; a < 4; ++a)
    for (int k = threadIdx.x; k < cnt[a]; k += blockDim.x) dst[a][k] = src[a][k];
  for (int k = threadIdx.x; k < HK_NIV * 4 * (HKF_DEG + 1); k += blockDim.x)
    (&t->fitf[0][0][0])[k] = (&hkf_fit[0][0][0])[k];
  for (int k = threadIdx.x; k < 12; k += blockDim.x) t->asyf[k / 3][k % 3] = (float)hk_asy[k / 3][k % 3];
}

template <int N>
__device__ __forceinline__ double hk_horner(const double* c, double s) {
  double r = c[N - 1];
#pragma unroll
  for (int k = N - 2; k >= 0; --k) r = fma(r, s, c[k]);
  return r;
}

__device__ __forceinline__ double hk_horner_n(const double* c, int n, double s) {
  double r = c[n - 1];
  for (int k = n - 2; k >= 0; --k) r = fma(r, s, c[k]);
  return r;
}

template <int N>
__device__ __forceinline__ float hk_hornerf(const float* c, float s) {
  float r = c[N - 1];
#pragma unroll
  for (int k = N - 2; k >= 0; --k) r = fmaf(r, s, c[k]);
  return r;
}

__device__ __forceinline__ int hk_interval(double z) {
  int iv = 0;
#pragma unroll
  for (int k = 1; k < HK_NIV; ++k) iv += (z >= 0.0 + hk_iv_lo(k)) ? 1 : 0;
  return iv;
}

// Small argument: ascending series.
__device__ __forceinline__ void hk_series(const HkTables& T, double z, Hk& o) {
  double u = 0.25 * z * z;
  double j0 = hk_horner<HK_NSER>(T.ser[0], u);
  double j1 = 0.5 * z * hk_horner<HK_NSER>(T.ser[1], u);
  double s0 = hk_horner<HK_NSER>(T.ser[2], u);
  double s1 = hk_horner<HK_NSER>(T.ser[3], u);
  double L = log(0.5 * z);
  double iz = 1.0 / z;
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

// P_nu, Q_nu for z >= HK_Z_SERIES.
__device__ __forceinline__ void hk_pq(const HkTables& T, double z, double iz, double* P0,
                                      double* Q0, double* P1, double* Q1) {
  if (z < HK_Z_ASYM) {
    int iv = hk_interval(z);
    double s = (z - T.iv[iv][2]) * T.iv[iv][3];
    *P0 = 1.0 + hk_horner<HK_DEG + 1>(T.fit[iv][0], s);
    *Q0 = hk_horner<HK_DEG + 1>(T.fit[iv][1], s);
    *P1 = 1.0 + hk_horner<HK_DEG + 1>(T.fit[iv][2], s);
    *Q1 = hk_horner<HK_DEG + 1>(T.fit[iv][3], s);
  } else {
    double t = iz * iz;
    int n = (z < 40.0) ? HK_NASY : (z < 100.0) ? 7 : (z < 1000.0) ? 5 : 3;
    *P0 = hk_horner_n(T.asy[0], n, t);
    *Q0 = iz * hk_horner_n(T.asy[1], n, t);
    *P1 = hk_horner_n(T.asy[2], n, t);
    *Q1 = iz * hk_horner_n(T.asy[3], n, t);
  }
}

// FP64 H0, H1 and F1 = H1/z + 2i/(pi z^2) at z > 0.
__device__ __forceinline__ void hankel_fp64(const HkTables& T, double z, Hk& o) {
  if (z < HK_Z_SERIES) {
    hk_series(T, z, o);
    return;
  }
  double rs = rsqrt(z);
  double iz = rs * rs;
  double A = WSBM_SQRT_2_OVER_PI * rs;
  double sn, cs;
  sincos(z, &sn, &cs);
  double E = (cs + sn) * WSBM_INV_SQRT2;  // e^{i(z - pi/4)} = E + iF
  double F = (sn - cs) * WSBM_INV_SQRT2;
  double P0, Q0, P1, Q1;
  hk_pq(T, z, iz, &P0, &Q0, &P1, &Q1);
  o.h0r = A * (P0 * E - Q0 * F);
  o.h0i = A * (P0 * F + Q0 * E);
  // e^{i(z - 3pi/4)} = -i (E + iF) = F - iE
  o.h1r = A * (P1 * F + Q1 * E);
  o.h1i = A * (Q1 * F - P1 * E);
  o.f1r = o.h1r * iz;
  o.f1i = fma(WSBM_2_OVER_PI * iz, iz, o.h1i * iz);
}

// Mixed: FP64 phase reduction, FP32 amplitude.  Valid for z >= HK_Z_SERIES.  Also returns
// D = H1 + i H0 = sqrt(2/(pi z)) e^{i(z - pi/4)} [(Q1 - Q0) + i(P0 - P1)], formed from the small
// differences of P and Q so that it keeps its relative accuracy (H1 ~ -i H0 for large z, and
// combined-field sources cancel to leading order).
__device__ __forceinline__ void hankel_mixed_large(const HkTables& T, double z, HkF& o,
                                                   float* Dr = nullptr, float* Di = nullptr) {
  // z - 2 pi n with 2 pi split into a short head (n * head exact) and a tail
  double n = rint(z * (0.5 / WSBM_PI));
  double y = fma(-n, HK_TWO_PI_HI, z);
  y = fma(-n, HK_TWO_PI_LO, y);
  float yf = (float)y;
  float sn, cs;
  sincosf(yf, &sn, &cs);
  float zf = (float)z;
  float rs = rsqrtf(zf);
  float A = (float)WSBM_SQRT_2_OVER_PI * rs;
  float E = (cs + sn) * (float)WSBM_INV_SQRT2;
  float F = (sn - cs) * (float)WSBM_INV_SQRT2;
  float P0, Q0, P1, Q1;
  if (z < HK_Z_ASYM) {
    int iv = hk_interval(z);
    float s = (float)((z - T.iv[iv][2]) * T.iv[iv][3]);
    P0 = hk_hornerf<HKF_DEG + 1>(T.fitf[iv][0], s);  // P0 - 1
    Q0 = hk_hornerf<HKF_DEG + 1>(T.fitf[iv][1], s);
    P1 = hk_hornerf<HKF_DEG + 1>(T.fitf[iv][2], s);  // P1 - 1
    Q1 = hk_hornerf<HKF_DEG + 1>(T.fitf[iv][3], s);
  } else {
    float iz = rs * rs;
    float t = iz * iz;
    P0 = t * fmaf(T.asyf[0][2], t, T.asyf[0][1]);  // P0 - 1
    Q0 = iz * fmaf(fmaf(T.asyf[1][2], t, T.asyf[1][1]), t, T.asyf[1][0]);
    P1 = t * fmaf(T.asyf[2][2], t, T.asyf[2][1]);  // P1 - 1
    Q1 = iz * fmaf(fmaf(T.asyf[3][2], t, T.asyf[3][1]), t, T.asyf[3][0]);
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
