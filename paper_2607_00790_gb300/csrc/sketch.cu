// Randomized row sketch of the ID matrices on the tensor cores: Y = Omega M, with Omega an
// l x m Rademacher matrix (entries +-1 from a counter-based hash of (row, column, seed)) and M
// an m x n complex128 matrix.  The column-pivoted QR of Y (l rows) then picks the skeleton and
// the interpolation coefficients of M (randomized interpolative decomposition: the column
// space geometry of M survives the sketch for ranks well below l).
//
// Exact FP64 products from BF16 tensor cores: every column of M is scaled by a power of two so
// that its entries lie in [-1, 1], and each real and imaginary part is split into S = 5 slices
// of 8 bits, v = sum_p b_p 2^(-8p) + r with integers |b_p| <= 256 (exact in BF16) and
// |r| <= 2^-41.  Omega (+-1) is exact in BF16 too, so every product is exact and each slice's
// sum over m <= 65536 rows is exact in the FP32 accumulator (|sum| <= 256 m < 2^24).  The
// slices are combined in FP64: Y carries a relative error of about 2^-41 of its column scale.
//
// Layout: one CTA per (descriptor, strip of 8 columns), one warp per 16 rows of Y, warp-level
// mma.sync m16n8k16 (BF16 in, FP32 accumulate); the 16 x 8 chunk of M of each K step is split
// once into shared memory and read by every warp.
#include <cuda_bf16.h>
#include <math.h>

#include "wsbm_internal.h"

namespace {

#define SK_S 5         // slices of 8 bits
#define SK_COLS 8      // columns per CTA (the mma N)
#define SK_MAX_WARPS 16  // l <= 256 (keeps the 40 accumulators in registers)

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

__global__ void __launch_bounds__(SK_MAX_WARPS * 32)
    k_sketch(const SketchDesc* __restrict__ d, uint32_t seed) {
  const SketchDesc q = d[blockIdx.y];
  const int c0 = blockIdx.x * SK_COLS;
  if (c0 >= q.n) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  __shared__ double s_scale[SK_COLS];
  __shared__ uint16_t sB[SK_S][2][16][SK_COLS];  // [slice][re/im][k][column]
  // column maxima of |Re|, |Im| -> power-of-two scales
  for (int cc = warp; cc < SK_COLS; cc += nwarps) {
    const int c = c0 + cc;
    double mx = 0.0;
    if (c < q.n)
      for (int i = lane; i < q.m; i += 32) {
        const double2 v = q.A[i + (int64_t)c * q.lda];
        mx = fmax(mx, fmax(fabs(v.x), fabs(v.y)));
      }
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) {
      int e = 0;
      if (mx > 0.0) frexp(mx, &e);  // mx < 2^e
      s_scale[cc] = ldexp(1.0, -e);
    }
  }
  __syncthreads();
  const int gid = lane >> 2, tig = lane & 3;
  const int row0 = warp * 16;  // rows of Y of this warp
  const bool active = row0 < q.l;
  float acc[SK_S][2][4];
#pragma unroll
  for (int p = 0; p < SK_S; ++p)
#pragma unroll
    for (int t = 0; t < 2; ++t)
#pragma unroll
      for (int z = 0; z < 4; ++z) acc[p][t][z] = 0.0f;
  for (int i0 = 0; i0 < q.m; i0 += 16) {
    // split the 16 x 8 chunk of M into slices
    for (int e = threadIdx.x; e < 16 * SK_COLS; e += blockDim.x) {
      const int kk = e & 15, cc = e >> 4;
      const int i = i0 + kk, c = c0 + cc;
      double2 v = make_double2(0.0, 0.0);
      if (i < q.m && c < q.n) v = q.A[i + (int64_t)c * q.lda];
      double t[2] = {v.x * s_scale[cc] * 256.0, v.y * s_scale[cc] * 256.0};
#pragma unroll
      for (int part = 0; part < 2; ++part) {
        double x = t[part];
#pragma unroll
        for (int p = 0; p < SK_S; ++p) {
          const double b = rint(x);
          sB[p][part][kk][cc] = sk_bf16_bits((float)b);
          x = (x - b) * 256.0;
        }
      }
    }
    __syncthreads();
    if (active) {
      // A fragment: Omega rows row0 + {gid, gid+8}, columns i0 + tig*2 + {0, 1, 8, 9}
      const uint32_t ra = row0 + gid, rb = row0 + gid + 8;
      const uint32_t k0 = i0 + tig * 2;
      uint32_t a[4];
      a[0] = sk_sign16(ra, k0, seed) | (sk_sign16(ra, k0 + 1, seed) << 16);
      a[1] = sk_sign16(rb, k0, seed) | (sk_sign16(rb, k0 + 1, seed) << 16);
      a[2] = sk_sign16(ra, k0 + 8, seed) | (sk_sign16(ra, k0 + 9, seed) << 16);
      a[3] = sk_sign16(rb, k0 + 8, seed) | (sk_sign16(rb, k0 + 9, seed) << 16);
#pragma unroll
      for (int p = 0; p < SK_S; ++p)
#pragma unroll
        for (int part = 0; part < 2; ++part) {
          uint32_t b[2];
          b[0] = (uint32_t)sB[p][part][tig * 2][gid] | ((uint32_t)sB[p][part][tig * 2 + 1][gid] << 16);
          b[1] = (uint32_t)sB[p][part][tig * 2 + 8][gid] | ((uint32_t)sB[p][part][tig * 2 + 9][gid] << 16);
          sk_mma(acc[p][part], a, b);
        }
    }
    __syncthreads();
  }
  if (!active) return;
  // combine the slices in FP64 and undo the column scale
#pragma unroll
  for (int z = 0; z < 4; ++z) {
    const int r = row0 + gid + ((z & 2) ? 8 : 0);
    const int cc = tig * 2 + (z & 1);
    const int c = c0 + cc;
    if (r >= q.l || c >= q.n) continue;
    double re = 0.0, im = 0.0, w = 1.0 / 256.0;
#pragma unroll
    for (int p = 0; p < SK_S; ++p) {
      re = fma((double)acc[p][0][z], w, re);
      im = fma((double)acc[p][1][z], w, im);
      w *= 1.0 / 256.0;
    }
    const double inv = 1.0 / s_scale[cc];
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
  SketchDesc* d = nullptr;
  if (cudaMallocAsync((void**)&d, sizeof(h), st) != cudaSuccess) return WSBM_ERR_OOM;
  int rc = WSBM_OK;
  if (cudaMemcpyAsync(d, &h, sizeof(h), cudaMemcpyHostToDevice, st) != cudaSuccess) rc = WSBM_ERR_CUDA;
  if (!rc) rc = wsbm_sketch_batched(d, 1, n, l, seed, st);
  if (!rc && cudaStreamSynchronize(st) != cudaSuccess) rc = WSBM_ERR_CUDA;  // h is on this frame
  cudaFreeAsync(d, st);
  return rc;
}
