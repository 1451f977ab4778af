"""Generate the coefficient tables of the device Hankel evaluator (writes hankel_coeffs.inc).

The evaluator writes, for z >= Z_SERIES,
    H_nu(z) = sqrt(2/(pi z)) (P_nu(z) + i Q_nu(z)) exp(i (z - pi/4 - nu pi/2)),   nu = 0, 1,
which defines the real functions P_nu, Q_nu exactly (P -> 1, Q -> 0 as z -> infinity).

* Z_SERIES <= z < Z_ASYM: P_nu - 1 and Q_nu on the intervals BOUNDS are polynomials of degree
  DEG in s = (u - c)/h, u = 1/z (c, h: centre and half-width of the interval in u), obtained by
  interpolation at Chebyshev points in 50-digit arithmetic (mpmath).  In u the functions are far
  smoother than in z (degree 10 instead of 16 for the same accuracy).
* z >= Z_ASYM: P_nu - 1 and z Q_nu as polynomials of degree DEG_T in s = (t - c)/h, t = 1/z^2 on
  [0, 1/Z_ASYM^2], interpolated the same way (their values at t = 0 follow the Hankel asymptotic
  expansion, A&S 9.2.5-9.2.10: P -> 1, z Q -> (4 nu^2 - 1)/8).
* z < Z_SERIES: ascending series (A&S 9.1.10, 9.1.11, 9.1.13 with psi(k+1) = H_k - gamma) in
  u = z^2/4:
    J0 = sum (-u)^k/(k!)^2,          J1 = (z/2) sum (-u)^k/(k!(k+1)!),
    Y0 = (2/pi)(ln(z/2) + gamma) J0 + (2/pi) sum_{k>=1} (-1)^{k+1} H_k u^k/(k!)^2,
    Y1 = -2/(pi z) + (2/pi) ln(z/2) J1 - (z/(2 pi)) sum (-1)^k (H_k + H_{k+1} - 2 gamma) u^k/(k!(k+1)!).
* sin and cos on |w| <= pi/4 (after a Cody-Waite reduction of z - pi/4 by multiples of pi/2):
    sin w = w + w^3 S(w^2),   cos w = 1 - w^2/2 + w^4 C(w^2),
  S and C of degree DEG_SC in v = w^2, least-squares fits at Chebyshev points of [0, VMAX].
* FP32 tables for the mixed-precision evaluator: the same intervals with degree DEG_F in s, and
  degree DEG_TF in t for z >= Z_ASYM.

Every table is checked here by evaluating it the way the device does (float64 / float32 Horner
with numpy) against mpmath; the script fails if a bound is missed.

Run:  python gen_hankel_coeffs.py   (needs mpmath; the generated file is committed)
"""
import os

import mpmath as mp
import numpy as np

mp.mp.dps = 50

# interval bounds in z: dyadic values, so the device can compare the high word of z as an integer
BOUNDS = [1.5, 2.0, 3.0, 4.0, 5.5, 8.0, 12.0, 20.0]
Z_SERIES = BOUNDS[0]
Z_ASYM = BOUNDS[-1]
DEG = 10
DEG_T = 6
N_SERIES = 12
DEG_SC = 6
VMAX = 0.66   # (pi/4 + slack)^2
DEG_F = 4
DEG_TF = 2
TWO_PI_HEAD_BITS = 33   # 2 pi head for the mixed evaluator: n * head is exact for n < 2^20


def PQ(nu, z):
    z = mp.mpf(z)
    h = mp.hankel1(nu, z)
    v = mp.sqrt(mp.pi * z / 2) * h * mp.exp(-1j * (z - mp.pi / 4 - nu * mp.pi / 2))
    return mp.re(v), mp.im(v)


def cheb_interp(f, lo, hi, deg):
    """Monomial coefficients in s = (x - c)/h of the degree-deg interpolant at Chebyshev points."""
    lo, hi = mp.mpf(lo), mp.mpf(hi)
    c, h = (lo + hi) / 2, (hi - lo) / 2
    n = deg + 1
    s = [mp.cos(mp.pi * (2 * j + 1) / (2 * n)) for j in range(n)]
    V = mp.matrix(n, n)
    for i in range(n):
        for j in range(n):
            V[i, j] = s[i] ** j
    coef = mp.lu_solve(V, mp.matrix([f(c + h * sj) for sj in s]))
    return [coef[j] for j in range(n)], c, h


def horner(cf, x, dt):
    r = dt(cf[-1])
    for v in reversed(cf[:-1]):
        r = dt(r * x + dt(v)) if dt is np.float32 else r * x + v
    return r


def fit_tables():
    mids, fits, fitsf = [], [], []
    for a, b in zip(BOUNDS[:-1], BOUNDS[1:]):
        lo, hi = mp.mpf(1) / b, mp.mpf(1) / a          # u-interval
        row, rowf = [], []
        for nu in (0, 1):
            for which in (0, 1):
                f = lambda u, nu=nu, which=which: PQ(nu, 1 / u)[which] - (1 if which == 0 else 0)
                cf, c, h = cheb_interp(f, lo, hi, DEG)
                cff, _, _ = cheb_interp(f, lo, hi, DEG_F)
                row.append(cf)
                rowf.append(cff)
        mids.append((a, b, c, 1 / h))
        fits.append(row)
        fitsf.append(rowf)
    return mids, fits, fitsf


def asym_tables():
    T = 1 / mp.mpf(Z_ASYM) ** 2
    out, outf = [], []
    for nu in (0, 1):
        fP = lambda t, nu=nu: (PQ(nu, 1 / mp.sqrt(t))[0] - 1) if t > 0 else mp.mpf(0)
        fQ = lambda t, nu=nu: (PQ(nu, 1 / mp.sqrt(t))[1] / mp.sqrt(t)) if t > 0 else (4 * mp.mpf(nu) ** 2 - 1) / 8
        for f in (fP, fQ):
            cf, c, h = cheb_interp(f, mp.mpf(0), T, DEG_T)
            cff, _, _ = cheb_interp(f, mp.mpf(0), T, DEG_TF)
            out.append(cf)
            outf.append(cff)
    return out, outf, c, 1 / h


def series_coeffs():
    H = [mp.mpf(0)]
    for k in range(1, N_SERIES + 2):
        H.append(H[-1] + mp.mpf(1) / k)
    g = mp.euler
    j0 = [(-1) ** k / mp.factorial(k) ** 2 for k in range(N_SERIES)]
    j1 = [(-1) ** k / (mp.factorial(k) * mp.factorial(k + 1)) for k in range(N_SERIES)]
    y0 = [mp.mpf(0)] + [(-1) ** (k + 1) * H[k] / mp.factorial(k) ** 2 for k in range(1, N_SERIES)]
    y1 = [(-1) ** k * (H[k] + H[k + 1] - 2 * g) / (mp.factorial(k) * mp.factorial(k + 1))
          for k in range(N_SERIES)]
    return j0, j1, y0, y1


def lsq_fit(f, vmax, deg, npts=200):
    """Least-squares monomial fit in v on [0, vmax] at Chebyshev points (50-digit)."""
    pts = [vmax * (1 + mp.cos(mp.pi * (2 * j + 1) / (2 * npts))) / 2 for j in range(npts)]
    A = mp.matrix(npts, deg + 1)
    y = mp.matrix(npts, 1)
    for i, v in enumerate(pts):
        for j in range(deg + 1):
            A[i, j] = v ** j
        y[i] = f(v)
    coef = mp.qr_solve(A, y)[0]
    return [coef[j] for j in range(deg + 1)]


def sincos_tables():
    fs = lambda v: (mp.sin(mp.sqrt(v)) - mp.sqrt(v)) / (mp.sqrt(v) ** 3) if v > 0 else -mp.mpf(1) / 6
    fc = lambda v: (mp.cos(mp.sqrt(v)) - 1 + v / 2) / (v * v) if v > 0 else mp.mpf(1) / 24
    return lsq_fit(fs, mp.mpf(VMAX), DEG_SC), lsq_fit(fc, mp.mpf(VMAX), DEG_SC)


# ---------------------------------------------------------------- device emulation ----
def pq_eval64(z, mids, fits, asy, tc, tih):
    if z < Z_ASYM:
        iv = sum(1 for b in BOUNDS[1:-1] if z >= b)
        a, b, c, ih = mids[iv]
        s = (1.0 / z - float(c)) * float(ih)
        r = [horner([float(v) for v in cf], s, float) for cf in fits[iv]]
        return 1 + r[0], r[1], 1 + r[2], r[3]
    u = 1.0 / z
    s = (u * u - float(tc)) * float(tih)
    r = [horner([float(v) for v in cf], s, float) for cf in asy]
    return 1 + r[0], u * r[1], 1 + r[2], u * r[3]


def check(mids, fits, fitsf, asy, asyf, tc, tih, S, C):
    rng = np.random.default_rng(0)
    zs = np.concatenate([rng.uniform(Z_SERIES, Z_ASYM, 3000), np.geomspace(Z_ASYM, 1e6, 600),
                         np.array(BOUNDS), np.nextafter(np.array(BOUNDS), 0)])
    worst = 0.0
    for z in zs:
        if z < Z_SERIES:
            continue
        p0, q0, p1, q1 = pq_eval64(float(z), mids, fits, asy, tc, tih)
        r0, r1 = PQ(0, z), PQ(1, z)
        worst = max(worst, abs(p0 - float(r0[0])), abs(q0 - float(r0[1])),
                    abs(p1 - float(r1[0])), abs(q1 - float(r1[1])))
    assert worst < 3.5e-16, ("FP64 P/Q fit error", worst)
    # FP32 tables
    worstf = 0.0
    for z in zs[::7]:
        if z < Z_SERIES:
            continue
        if z < Z_ASYM:
            iv = sum(1 for b in BOUNDS[1:-1] if z >= b)
            a, b, c, ih = mids[iv]
            s = np.float32((1.0 / z - float(c)) * float(ih))
            r = [float(horner([np.float32(float(v)) for v in cf], s, np.float32)) for cf in fitsf[iv]]
            vals = (r[0], r[1], r[2], r[3])
        else:
            u = 1.0 / z
            s = np.float32((u * u - float(tc)) * float(tih))
            r = [float(horner([np.float32(float(v)) for v in cf], s, np.float32)) for cf in asyf]
            vals = (r[0], u * r[1], r[2], u * r[3])
        r0, r1 = PQ(0, z), PQ(1, z)
        worstf = max(worstf, abs(vals[0] - float(r0[0] - 1)), abs(vals[1] - float(r0[1])),
                     abs(vals[2] - float(r1[0] - 1)), abs(vals[3] - float(r1[1])))
    assert worstf < 1.5e-7, ("FP32 P/Q fit error", worstf)
    # sin / cos
    ws = np.linspace(-np.pi / 4 - 1e-3, np.pi / 4 + 1e-3, 20001)
    Sf = [float(v) for v in S]
    Cf = [float(v) for v in C]
    es = ec = 0.0
    for w in ws[::5]:
        v = w * w
        s = w + (w * v) * horner(Sf, v, float)
        c = 1.0 + v * (-0.5 + v * horner(Cf, v, float))
        es = max(es, abs(s - float(mp.sin(w))))
        ec = max(ec, abs(c - float(mp.cos(w))))
    assert es < 2.3e-16 and ec < 2.3e-16, ("sincos error", es, ec)
    return worst, worstf, es, ec


def fmt(v):
    return repr(float(v))


def main():
    mids, fits, fitsf = fit_tables()
    asy, asyf, tc, tih = asym_tables()
    S, C = sincos_tables()
    errs = check(mids, fits, fitsf, asy, asyf, tc, tih, S, C)
    nv = len(mids)
    L = ["// Generated by gen_hankel_coeffs.py -- do not edit.",
         f"// max abs error (emulated): P,Q FP64 {errs[0]:.2e}, FP32 {errs[1]:.2e}; sin {errs[2]:.2e}, cos {errs[3]:.2e}",
         f"#define HK_Z_SERIES {Z_SERIES!r}", f"#define HK_Z_ASYM {Z_ASYM!r}", f"#define HK_NIV {nv}",
         f"#define HK_DEG {DEG}", f"#define HK_DEG_T {DEG_T}", f"#define HK_NSER {N_SERIES}",
         f"#define HK_DEG_SC {DEG_SC}", f"#define HKF_DEG {DEG_F}", f"#define HKF_DEG_T {DEG_TF}", ""]
    # interval i covers [BOUNDS[i], BOUNDS[i+1]); high 32-bit words of the inner bounds
    import struct
    his = [struct.unpack("<II", struct.pack("<d", b))[1] for b in BOUNDS[1:-1]]
    los = [struct.unpack("<II", struct.pack("<d", b))[0] for b in BOUNDS]
    assert all(l == 0 for l in los), "bounds must have a zero low word"
    L.append("// high 32-bit words of the inner interval bounds (their low words are zero)")
    L.append("#define HK_IV_HI {" + ", ".join(str(h) for h in his) + "}")
    L.append(f"#define HK_SERIES_HI {struct.unpack('<II', struct.pack('<d', BOUNDS[0]))[1]}")
    L.append(f"#define HK_ASYM_HI {struct.unpack('<II', struct.pack('<d', BOUNDS[-1]))[1]}")
    L.append("// per interval: centre and 1/half-width in u = 1/z")
    L.append("static __device__ const double hk_iv[HK_NIV][2] = {")
    for (a, b, c, ih) in mids:
        L.append(f"  {{{fmt(c)}, {fmt(ih)}}},  // z in [{a}, {b})")
    L.append("};")
    L.append("// fits[iv][fn][k], fn = P0-1, Q0, P1-1, Q1")
    L.append("static __device__ const double hk_fit[HK_NIV][4][HK_DEG + 1] = {")
    for row in fits:
        L.append("  {")
        for cf in row:
            L.append("    {" + ", ".join(fmt(v) for v in cf) + "},")
        L.append("  },")
    L.append("};")
    L.append(f"#define HK_T_C {fmt(tc)}")
    L.append(f"#define HK_T_IH {fmt(tih)}")
    L.append("// z >= HK_Z_ASYM, in t = 1/z^2: fn = P0-1, z Q0, P1-1, z Q1")
    L.append("static __device__ const double hk_asy[4][HK_DEG_T + 1] = {")
    for cf in asy:
        L.append("  {" + ", ".join(fmt(v) for v in cf) + "},")
    L.append("};")
    j0, j1, y0, y1 = series_coeffs()
    L.append("static __device__ const double hk_ser[4][HK_NSER] = {")
    for arr in (j0, j1, y0, y1):
        L.append("  {" + ", ".join(fmt(v) for v in arr) + "},")
    L.append("};")
    L.append("// sin w = w + w^3 S(w^2), cos w = 1 - w^2/2 + w^4 C(w^2), |w| <= pi/4")
    L.append("static __device__ const double hk_sin[HK_DEG_SC + 1] = {" + ", ".join(fmt(v) for v in S) + "};")
    L.append("static __device__ const double hk_cos[HK_DEG_SC + 1] = {" + ", ".join(fmt(v) for v in C) + "};")
    half_pi = mp.pi / 2
    c1 = mp.mpf(float(half_pi))
    L.append(f"#define HK_PIO2_HI {fmt(c1)}")
    L.append(f"#define HK_PIO2_LO {fmt(half_pi - c1)}")
    L.append(f"#define HK_2_OVER_PI {fmt(2 / mp.pi)}")
    L.append("static __device__ const float hkf_fit[HK_NIV][4][HKF_DEG + 1] = {")
    for row in fitsf:
        L.append("  {")
        for cf in row:
            L.append("    {" + ", ".join(fmt(v) + "f" for v in cf) + "},")
        L.append("  },")
    L.append("};")
    L.append("static __device__ const float hkf_asy[4][HKF_DEG_T + 1] = {")
    for cf in asyf:
        L.append("  {" + ", ".join(fmt(v) + "f" for v in cf) + "},")
    L.append("};")
    two_pi = 2 * mp.pi
    e = int(mp.floor(mp.log(two_pi, 2)))
    scale = mp.mpf(2) ** (TWO_PI_HEAD_BITS - 1 - e)
    head = mp.floor(two_pi * scale) / scale
    L.append(f"#define HK_TWO_PI_HI {fmt(head)}")
    L.append(f"#define HK_TWO_PI_LO {fmt(two_pi - head)}")
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "hankel_coeffs.inc")
    open(out, "w").write("\n".join(L) + "\n")
    print("wrote", out, "errors", errs)


if __name__ == "__main__":
    main()
