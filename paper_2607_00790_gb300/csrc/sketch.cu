// Randomized row sketch of the ID matrices on the tensor cores: Y = Omega M, with Omega an
// l x m Rademacher matrix (entries +-1 from a counter-based hash of (row, column, seed)) and M
// an m x n complex128 matrix.  The column-pivoted QR of Y (l rows) then picks the skeleton and
// the interpolation coefficients of M (randomized interpolative decomposition: the column
// space geometry of M survives the sketch for ranks well below l).
//
// Exact FP64 products from BF16 tensor cores: every column of M is scaled by a power of two so
// that its entries lie in (-1, 1), and each real and imaginary part is rounded to a 40-bit
// integer and split into S = 5 balanced base-256 digits, v = sum_p b_p 2^(-8p) + r with integers
// |b_p| <= 256 (exact in BF16) and |r| <= 2^-41.  Omega (+-1) is exact in BF16 too, so every product is exact and each slice's
// sum over m <= 65536 rows is exact in the FP32 accumulator (|sum| <= 256 m < 2^24).  The
// slices are combined in FP64: Y carries a relative error of about 2^-41 of its column scale.
//
// Layout: one CTA per (descriptor, strip of 16 columns), one warp per 16 rows of Y, warp-level
// mma.sync m16n8k16 (BF16 in, FP32 accumulate); each 32 x 16 chunk of M is split once into
// shared memory (one FP64 multiply and one integer conversion per value, then integer digits)
// and read by every warp.
#include <cuda_bf16.h>
#include <math.h>

#include "wsbm_internal.h"

namespace {

#define SK_S 5         // slices of 8 bits
#define SK_NT 2        // mma n-tiles (8 columns each) per warp
#define SK_COLS (8 * SK_NT)  // columns per CTA
#define SK_K 32        // rows of M per shared-memory stage
#define SK_MAX_WARPS 12  // l <= 192 (keeps the 80 accumulators of a warp in registers)

struct SketchDesc {
  const double2* A;
  int64_t lda;
  double2* Y;
  int64_t ldy;
  int32_t m, n, l, pad;
};

__device__ __forceinline__ uint32_t sk_hash(uint32_t r, uint32_t c, uint32_t seed) {
  uint32_t h = r * 0x9E3779B1u ^ (c * 0x85EBCA77u + seed);
  h ^= h >> 16;
  h *= 0x7FEB352Du;
  h ^= h >> 15;
  h *= 0x846CA68Bu;
  h ^= h >> 16;
  return h;
}

// BF16 bit patterns of +1 and -1
__device__ __forceinline__ uint32_t sk_sign16(uint32_t r, uint32_t c, uint32_t seed) {
  return (sk_hash(r, c, seed) & 1u) ? 0xBF80u : 0x3F80u;
}

__device__ __forceinline__ void sk_mma(float d[4], const uint32_t a[4], const uint32_t b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint16_t sk_bf16_bits(float v) {
  __nv_bfloat16 h = __float2bfloat16_rn(v);  // exact: integers of at most 9 bits
  return *reinterpret_cast<uint16_t*>(&h);
}

// Balanced base-256 digits of X (|X| < 2^40): X = sum_{p=1..5} b_p 2^(8(5-p)), b_p in [-128, 128].
__device__ __forceinline__ void sk_digits(long long X, float b[SK_S]) {
#pragma unroll
  for (int p = SK_S - 1; p >= 0; --p) {
    const long long d = ((X + 128) & 255) - 128;
    b[p] = (float)(int)d;
    X = (X - d) >> 8;
  }
  b[0] += (float)(int)(X << 8);  // the carry out of the top digit (|X| < 2^40 leaves b_1 <= 256)
}

__global__ void __launch_bounds__(SK_MAX_WARPS * 32)
    k_sketch(const SketchDesc* __restrict__ d, uint32_t seed) {
  const SketchDesc q = d[blockIdx.y];
  const int c0 = blockIdx.x * SK_COLS;
  if (c0 >= q.n) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  __shared__ int s_exp[SK_COLS];                                  // 40 - e: scale 2^(40 - e)
  __shared__ double s_sc[SK_COLS], s_inv[SK_COLS];                // 2^(40 - e), 2^e
  __shared__ uint16_t sB[SK_S][2][SK_K][SK_COLS];                 // [slice][re/im][k][column]
  // column maxima of |Re|, |Im| by integer compares of the bit patterns (non-negative doubles
  // order like their bits), then the exponent e with max < 2^e
  for (int cc = warp; cc < SK_COLS; cc += nwarps) {
    const int c = c0 + cc;
    unsigned long long mx = 0;
    if (c < q.n)
      for (int i = lane; i < q.m; i += 32) {
        const double2 v = q.A[i + (int64_t)c * q.lda];
        const unsigned long long a = (unsigned long long)__double_as_longlong(v.x) & 0x7FFFFFFFFFFFFFFFull;
        const unsigned long long b = (unsigned long long)__double_as_longlong(v.y) & 0x7FFFFFFFFFFFFFFFull;
        mx = max(mx, max(a, b));
      }
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) {
      const int E = (int)(mx >> 52);       // biased exponent of the largest magnitude
      const int se = mx ? 40 - (E - 1022) : 0;  // max < 2^(E - 1022); zero columns: any scale
      s_exp[cc] = se > 1000 ? 1000 : se;        // columns below 2^-960 sketch as zero
      s_sc[cc] = ldexp(1.0, s_exp[cc]);
      s_inv[cc] = ldexp(1.0, 40 - s_exp[cc]);
    }
  }
  __syncthreads();
  const int gid = lane >> 2, tig = lane & 3;
  const int row0 = warp * 16;
  const bool active = row0 < q.l;
  float acc[SK_S][2][SK_NT][4];
#pragma unroll
  for (int p = 0; p < SK_S; ++p)
#pragma unroll
    for (int t = 0; t < 2; ++t)
#pragma unroll
      for (int nt = 0; nt < SK_NT; ++nt)
#pragma unroll
        for (int z = 0; z < 4; ++z) acc[p][t][nt][z] = 0.0f;
  for (int i0 = 0; i0 < q.m; i0 += SK_K) {
    // split the SK_K x SK_COLS chunk of M into 8-bit slices: one FP64 multiply (exact power-of-
    // two scale) and one conversion to a 40-bit integer per value, then integer digits
    for (int e = threadIdx.x; e < SK_K * SK_COLS; e += blockDim.x) {
      const int kk = e % SK_K, cc = e / SK_K;
      const int i = i0 + kk, c = c0 + cc;
      double2 v = make_double2(0.0, 0.0);
      if (i < q.m && c < q.n) v = q.A[i + (int64_t)c * q.lda];
      const double sc = s_sc[cc];
      float b[SK_S];
      sk_digits(__double2ll_rn(v.x * sc), b);
#pragma unroll
      for (int p = 0; p < SK_S; ++p) sB[p][0][kk][cc] = sk_bf16_bits(b[p]);
      sk_digits(__double2ll_rn(v.y * sc), b);
#pragma unroll
      for (int p = 0; p < SK_S; ++p) sB[p][1][kk][cc] = sk_bf16_bits(b[p]);
    }
    __syncthreads();
    if (active) {
#pragma unroll
      for (int ks = 0; ks < SK_K / 16; ++ks) {
        // A fragment: Omega rows row0 + {gid, gid+8}, columns i0 + 16 ks + tig*2 + {0, 1, 8, 9}
        const uint32_t ra = row0 + gid, rb = row0 + gid + 8;
        const uint32_t k0 = i0 + 16 * ks + tig * 2;
        uint32_t a[4];
        a[0] = sk_sign16(ra, k0, seed) | (sk_sign16(ra, k0 + 1, seed) << 16);
        a[1] = sk_sign16(rb, k0, seed) | (sk_sign16(rb, k0 + 1, seed) << 16);
        a[2] = sk_sign16(ra, k0 + 8, seed) | (sk_sign16(ra, k0 + 9, seed) << 16);
        a[3] = sk_sign16(rb, k0 + 8, seed) | (sk_sign16(rb, k0 + 9, seed) << 16);
        const int kb = 16 * ks + tig * 2;
#pragma unroll
        for (int nt = 0; nt < SK_NT; ++nt) {
          const int col = nt * 8 + gid;
#pragma unroll
          for (int p = 0; p < SK_S; ++p)
#pragma unroll
            for (int part = 0; part < 2; ++part) {
              uint32_t b[2];
              b[0] = (uint32_t)sB[p][part][kb][col] | ((uint32_t)sB[p][part][kb + 1][col] << 16);
              b[1] = (uint32_t)sB[p][part][kb + 8][col] | ((uint32_t)sB[p][part][kb + 9][col] << 16);
              sk_mma(acc[p][part][nt], a, b);
            }
        }
      }
    }
    __syncthreads();
  }
  if (!active) return;
  // combine the slices in FP64 (slice p carries 2^(8(5-p)) / 2^40 = 2^(-8p)) and undo the scale
#pragma unroll
  for (int nt = 0; nt < SK_NT; ++nt)
#pragma unroll
    for (int z = 0; z < 4; ++z) {
      const int r = row0 + gid + ((z & 2) ? 8 : 0);
      const int cc = nt * 8 + tig * 2 + (z & 1);
      const int c = c0 + cc;
      if (r >= q.l || c >= q.n) continue;
      double re = 0.0, im = 0.0, w = 1.0 / 256.0;
#pragma unroll
      for (int p = 0; p < SK_S; ++p) {
        re = fma((double)acc[p][0][nt][z], w, re);
        im = fma((double)acc[p][1][nt][z], w, im);
        w *= 1.0 / 256.0;
      }
      const double inv = s_inv[cc];  // 2^e
      q.Y[r + (int64_t)c * q.ldy] = make_double2(re * inv, im * inv);
    }
}

}  // namespace

// Batched sketch launch: d_desc device array of n descriptors, max_n / max_l their largest n, l.
int wsbm_sketch_batched(const void* d_desc, int ndesc, int max_n, int max_l, uint32_t seed,
                        cudaStream_t st) {
  if (ndesc <= 0) return WSBM_OK;
  if (max_l < 16 || max_l > 16 * SK_MAX_WARPS || max_l % 16) return WSBM_ERR_INVALID_ARG;
  const SketchDesc* d = (const SketchDesc*)d_desc;
  for (int off = 0; off < ndesc; off += 65535) {
    const int cnt = ndesc - off < 65535 ? ndesc - off : 65535;
    dim3 grid((unsigned)((max_n + SK_COLS - 1) / SK_COLS), (unsigned)cnt);
    k_sketch<<<grid, (max_l / 16) * 32, 0, st>>>(d + off, seed);
    wsbm_count_launch();
  }
  return cudaGetLastError() == cudaSuccess ? WSBM_OK : WSBM_ERR_CUDA;
}

size_t wsbm_sketch_desc_size() { return sizeof(SketchDesc); }

void wsbm_sketch_desc_fill(void* slot, const void* A, int64_t lda, void* Y, int64_t ldy, int32_t m,
                           int32_t n, int32_t l) {
  SketchDesc* s = (SketchDesc*)slot;
  s->A = (const double2*)A;
  s->lda = lda;
  s->Y = (double2*)Y;
  s->ldy = ldy;
  s->m = m;
  s->n = n;
  s->l = l;
  s->pad = 0;
}

extern "C" int wsbm_sketch(const void* A, int64_t lda, int32_t m, int32_t n, int32_t l, void* Y,
                           int64_t ldy, uint32_t seed, void* stream) {
  if (m < 1 || n < 1 || l < 16 || l > 16 * SK_MAX_WARPS || l % 16 || m > 65536 || !A || !Y ||
      lda < m || ldy < l)
    return WSBM_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  SketchDesc h;
  wsbm_sketch_desc_fill(&h, A, lda, Y, ldy, m, n, l);
  WsbmScratch scr(st);
  SketchDesc* d = nullptr;
  int rc = scr.get(sizeof(h), (void**)&d);
  if (rc) return rc;
  if (cudaMemcpyAsync(d, &h, sizeof(h), cudaMemcpyHostToDevice, st) != cudaSuccess) rc = WSBM_ERR_CUDA;
  if (!rc) rc = wsbm_sketch_batched(d, 1, n, l, seed, st);
  if (!rc && cudaStreamSynchronize(st) != cudaSuccess) rc = WSBM_ERR_CUDA;  // h is on this frame
  return rc;
}
