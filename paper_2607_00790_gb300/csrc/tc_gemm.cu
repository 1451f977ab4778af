// Complex128 GEMM on the tensor cores with exact split precision (tcgen05 + TMA + TMEM).
//
//   C (m x n) = beta C + alpha A (m x k) B (k x n),   complex128, column-major.
//
// GB300 runs FP64 at 2 DFMA/clk/SM against 4096 BF16 multiply-adds/clk/SM on the tensor
// cores, so the dense contractions of the factorization (trailing updates of the blocked LU of
// large boxes and of the dense root) are formed from exact 8-bit pieces:
//
//  1. Scaling.  Row i of A gets a power of two 2^e_i with |Re A_il|, |Im A_il| < 2^(e_i - 1);
//     column j of B likewise 2^f_j.  The scaled values x (|x| < 1/2) are written as the 56-bit
//     integer X = x 2^56 (rounded when x has bits below 2^-56), and X as seven balanced base-256
//     digits d_0..d_6 in [-128, 128] (x = sum_t d_t 2^-8(t+1)), each exact in BF16.
//  2. Real form of the complex product.  Row i of A becomes the real row (Re A_i0, Im A_i0,
//     Re A_i1, Im A_i1, ...); column j of C becomes two real columns: 2j = Re C_j with B entries
//     (Re B_lj, -Im B_lj), 2j+1 = Im C_j with (Im B_lj, Re B_lj).  K_real = 2k.
//  3. Digit products on the tensor cores.  For every digit diagonal d = t + u <= 7 the FP32
//     accumulator acc_d (in TMEM) collects sum A_t B_u over a chunk of 256 real K values.  Every
//     product is an integer of magnitude <= 2^14, so the sums of diagonals 0..3 (at most 4 * 256
//     products) are exact integers of magnitude <= 2^24; diagonals 4..7 (weight 2^-48 and below
//     against 2^-16 for diagonal 0) may round, by less than 2^-53.7 of the chunk's largest
//     possible leading term.  Pairs with t + u >= 8 are left out: their weight is below 2^-63 of
//     the leading term.
//  4. Recombination without FP64 arithmetic.  After each chunk the accumulators are drained
//     into a fixed-point sum of 2^-64 resolution: a 64-bit integer T of unit 2^-48 (digit
//     diagonals 0..4 and the high part of 5) and a 16-bit fraction F of unit 2^-64 (the rest of
//     5, diagonal 6, and diagonal 7 rounded), whose carries move into T after every chunk
//     (integer and FP32 pipes only).  At the end of the K loop,
//     C_ij = beta C_ij + alpha (T + F 2^-16) 2^(e_i + f_j - 48).
//
// Error: the rounding of X to 56 bits (relative to the row or column maximum) and the pairs
// left out keep each entry of A B within about 2^-53 * 2k * max|A_i.| * max|B_.j| of the exact
// product, the bound of an FP64 product.
//
// Kernel: one CTA per SM, persistent over 128 x 64 (real) output tiles.  Warp 0 issues the TMA
// loads of the 14 digit planes of a 16-wide K block (a 4-stage ring in shared memory, 32-byte
// swizzled rows), warp 1 allocates TMEM (8 accumulators x 64 columns) and issues the MMAs
// (one thread), warps 2-9 drain the accumulators (two threads per TMEM lane = output row, each
// with 32 of the 64 columns) and write C.  Every wait on a barrier is bounded in time; a wait that runs out sets an error
// flag read by the host, and all roles then leave their loops.
#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "dense.h"

#define TC_BM 128                       // output rows per tile (= TMEM lanes)
#define TC_BN 64                        // real output columns per tile (32 complex)
#ifndef TC_BK
#define TC_BK 16                        // real K values per pipeline stage (32-byte rows)
#endif
#define TC_S 7                          // digits per operand
#define TC_ND 8                         // digit diagonals kept (t + u <= 7)
#define TC_STAGES (64 / TC_BK)          // 4 stages of 16 K values (2 of 32): about 168 KB in flight
#define TC_KC 256                       // real K values per accumulation chunk (drain period)
#define TC_A_TILE (TC_BM * TC_BK * 2)   // bytes of one A digit plane tile (4 KB)
#define TC_B_TILE (TC_BN * TC_BK * 2)   // bytes of one B digit plane tile (2 KB)
#define TC_STAGE_BYTES (TC_S * (TC_A_TILE + TC_B_TILE))
#define TC_FRAC_BYTES (TC_BN * TC_BM * 4)  // fraction words F of a tile (int32, column-major)
#define TC_SMEM (TC_STAGES * TC_STAGE_BYTES + TC_FRAC_BYTES + 256 + 1024)
#define TC_THREADS 320                  // producer, MMA, 8 epilogue warps
#define TC_EPI 256                      // epilogue threads (two per TMEM lane)
#define TC_TMEM_COLS 512
#define TC_WAIT_NS 2000000000ull        // bound of every barrier wait (2 s)

static_assert(TC_STAGE_BYTES % 1024 == 0, "stage alignment");
static_assert(TC_KC % TC_BK == 0, "chunk of whole stages");
static_assert(TC_BK == 16 || TC_BK == 32, "rows of 32 bytes (32-byte swizzle) or 64 (64-byte swizzle)");

static __device__ int g_tc_error;  // set when a bounded wait ran out

// ----------------------------------------------------------------- PTX helpers ----
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase of parity `parity` of barrier `bar`, at most TC_WAIT_NS.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255) == 0) {
      if (*(volatile int*)&g_tc_error) return false;
      if (globaltimer() - t0 > TC_WAIT_NS) {
        atomicExch(&g_tc_error, 1);
        return false;
      }
    }
  }
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int c0,
                                            int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(dst),
      "l"((uint64_t)map), "r"(bar), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory operand descriptor: K-major tile of TC_BK * 2-byte rows swizzled over the row
// width (atoms of 8 rows, 8 * 2 TC_BK bytes apart), descriptor version 1; swizzle code 6 for
// 32-byte rows, 4 for 64-byte rows.
__device__ __forceinline__ uint64_t sdesc_sw(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);               // start address
  d |= (uint64_t)1 << 16;                              // leading byte offset (unused for this layout)
  d |= (uint64_t)((8 * 2 * TC_BK) >> 4) << 32;         // stride byte offset: 8-row groups
  d |= (uint64_t)1 << 46;                              // version
  d |= (uint64_t)(TC_BK == 16 ? 6 : 4) << 61;          // layout: 32- or 64-byte swizzle
  return d;
}
// Instruction descriptor: BF16 x BF16 -> FP32, both operands K-major, M = 128, N = n (a
// multiple of 16, at most 256).
__host__ __device__ constexpr uint32_t tc_idesc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TC_BM >> 4) << 24);
}
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accum));
}

// The 34 digit pairs (t, u), t + u <= 7, as 11 MMAs: A digit t against the B digits u0 ..
// u0 + cnt - 1, which sit one after another in shared memory (one tile of 64 * cnt rows) and
// whose diagonals t + u0 .. t + u0 + cnt - 1 are adjacent accumulators in TMEM (N = 64 cnt).
// The first two MMAs of a chunk start diagonals 4..7 and 0..3 from zero; every later one adds.
__device__ __forceinline__ void tc_sched(int e, int& t, int& u0, int& cnt) {
  switch (e) {
    case 0: t = 1, u0 = 3, cnt = 4; break;
    case 1: t = 0, u0 = 0, cnt = 4; break;
    case 2: t = 0, u0 = 4, cnt = 3; break;
    case 3: t = 1, u0 = 0, cnt = 3; break;
    case 4: t = 2, u0 = 0, cnt = 4; break;
    case 5: t = 2, u0 = 4, cnt = 2; break;
    case 6: t = 3, u0 = 0, cnt = 4; break;
    case 7: t = 3, u0 = 4, cnt = 1; break;
    case 8: t = 4, u0 = 0, cnt = 4; break;
    case 9: t = 5, u0 = 0, cnt = 3; break;
    default: t = 6, u0 = 0, cnt = 2; break;
  }
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// x 2^ex: exponent-field addition when x and the result are normal, else ldexp.
__device__ __forceinline__ double scale2(double x, int ex) {
  const long long b = __double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FF);
  if (e > 0 && e + ex >= 1 && e + ex <= 2046) return __longlong_as_double(b + ((long long)ex << 52));
  return ldexp(x, ex);
}

// (T + F 2^-16) 2^ex (F in [0, 2^16)) as the correctly rounded double (to nearest, ties to
// even), formed with integer operations only: the 80-bit fixed-point value T 2^16 + F is
// normalized by a leading-zero count, rounded to 53 bits and given its exponent field, so the
// FP64 pipe (2 operations per clock per SM on this GPU) does not convert the accumulated sums.
// Returns false (and leaves x) when the result would leave the normal range.
__device__ __forceinline__ bool fixed_to_double(long long T, int F, int ex, double& x) {
  uint64_t lo = ((uint64_t)T << 16) | (uint64_t)(uint32_t)F;
  uint64_t hi = (uint64_t)(T >> 48);  // sign extension of T's top 16 bits
  const bool neg = T < 0;
  if (neg) {  // magnitude of the 128-bit two's-complement value
    lo = ~lo + 1;
    hi = ~hi + (lo == 0 ? 1 : 0);
  }
  if ((hi | lo) == 0) {
    x = 0.0;
    return true;
  }
  int p;          // bit index of the leading one
  uint64_t m;     // the 64 bits from the leading one down, left aligned
  uint64_t below; // the bits below those 64 (nonzero: part of the sticky bit)
  if (hi) {
    const int z = __clzll((long long)hi);
    p = 127 - z;
    m = z ? (hi << z) | (lo >> (64 - z)) : hi;
    below = z ? (lo << z) : lo;
  } else {
    const int z = __clzll((long long)lo);
    p = 63 - z;
    m = lo << z;
    below = 0;
  }
  uint64_t mant = m >> 11;  // 53 significant bits
  if (((m >> 10) & 1) && ((m & 0x3FF) | below | (mant & 1))) {
    ++mant;
    if (mant >> 53) {
      mant >>= 1;
      ++p;
    }
  }
  const int E = p - 16 + ex + 1023;
  if (E <= 0 || E >= 2047) return false;
  x = __longlong_as_double((long long)(((uint64_t)neg << 63) | ((uint64_t)E << 52) | (mant & 0xFFFFFFFFFFFFFull)));
  return true;
}

// --------------------------------------------------------------- digit planes ----
// Exponent e with |v| < 2^(e-1) for every |Re|, |Im| of the row/column maximum `mx` (as raw
// bits of a non-negative double); 0 for an all-zero row.
__device__ __forceinline__ int scale_exp(uint64_t mxbits) {
  if (mxbits == 0) return 0;
  const int E = (int)(mxbits >> 52);
  return (E > 0 ? E : 1) - 1021;
}
__device__ __forceinline__ uint64_t abs_bits(double v) {
  return (uint64_t)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
}
// The seven balanced base-256 digits of X = v 2^(56 - e) (|v| < 2^(e-1)), most significant first.
__device__ __forceinline__ void digits7(double v, int e, int* d) {
  const uint64_t b = (uint64_t)__double_as_longlong(v);
  const int E = (int)((b >> 52) & 0x7FF);
  uint64_t mant = b & 0xFFFFFFFFFFFFFull;
  if (E) mant |= 1ull << 52;
  const int sh = (E > 0 ? E : 1) - 1075 + 56 - e;
  int64_t X;
  if (mant == 0 || sh <= -64) {
    X = 0;
  } else if (sh >= 0) {
    X = (int64_t)(mant << sh);  // sh <= 2: |X| < 2^55
  } else {
    X = (int64_t)((mant + (1ull << (-sh - 1))) >> (-sh));  // round half up
  }
  if (b >> 63) X = -X;
#pragma unroll
  for (int t = TC_S - 1; t >= 1; --t) {
    const int dt = (int)((X + 128) & 255) - 128;
    d[t] = dt;
    X = (X - dt) >> 8;
  }
  d[0] = (int)X;
}

// One operand of a batched call, as the split kernels see it: source matrix, its sizes, its
// first row in the plane tensor and the offset of its exponents.
struct TcSrc {
  const double2* M;
  int64_t ld;
  int rows, k;  // A: m x k (rows = m); B: k x n (rows = n columns of B)
  int prow;     // first plane row (A: row offset; B': 2 x column offset)
  int eoff;     // first exponent
};

// Row exponents of A (m x k): one thread per row (coalesced along the column); item blockIdx.y.
__global__ void k_tc_row_exp(const TcSrc* __restrict__ src, int* __restrict__ rexp) {
  const TcSrc q = src[blockIdx.y];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= q.rows) return;
  uint64_t mx = 0;
  for (int l = 0; l < q.k; ++l) {
    const double2 v = q.M[i + (int64_t)l * q.ld];
    mx = max(mx, max(abs_bits(v.x), abs_bits(v.y)));
  }
  rexp[q.eoff + i] = scale_exp(mx);
}

// Digit planes of A: PA[t][row][2l + c] (c = 0: Re, 1: Im), rows of Ka BF16 values (zero
// beyond 2k).  Block: 32 rows x 32 complex columns of item blockIdx.z, staged through shared
// memory so that both the reads (along a column) and the writes (along a row) are contiguous.
__global__ void __launch_bounds__(256) k_tc_split_a(const TcSrc* __restrict__ src, const int* __restrict__ rexp,
                                                    __nv_bfloat16* __restrict__ PA, int64_t plane, int64_t Ka) {
  __shared__ __nv_bfloat16 s[TC_S][32][64 + 2];
  const TcSrc q = src[blockIdx.z];
  const int i0 = blockIdx.x * 32, l0 = blockIdx.y * 32;
  if (i0 >= q.rows) return;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  for (int ll = ty; ll < 32; ll += 8) {
    const int i = i0 + tx, l = l0 + ll;
    int dr[TC_S], di[TC_S];
    if (i < q.rows && l < q.k) {
      const double2 v = q.M[i + (int64_t)l * q.ld];
      const int e = rexp[q.eoff + i];
      digits7(v.x, e, dr);
      digits7(v.y, e, di);
    } else {
#pragma unroll
      for (int t = 0; t < TC_S; ++t) dr[t] = di[t] = 0;
    }
#pragma unroll
    for (int t = 0; t < TC_S; ++t) {
      s[t][tx][2 * ll] = __float2bfloat16_rn((float)dr[t]);
      s[t][tx][2 * ll + 1] = __float2bfloat16_rn((float)di[t]);
    }
  }
  __syncthreads();
  // write: for each plane and row, 64 consecutive BF16 values (columns 2 l0 .. 2 l0 + 63)
  for (int w = threadIdx.x; w < TC_S * 32 * 32; w += blockDim.x) {
    const int t = w / (32 * 32), r = (w / 32) % 32, c2 = w % 32;  // c2: pair of BF16 values
    const int i = i0 + r, kk = 2 * l0 + 2 * c2;
    if (i >= q.rows || kk >= Ka) continue;
    __nv_bfloat162 p;
    p.x = s[t][r][2 * c2];
    p.y = s[t][r][2 * c2 + 1];
    *reinterpret_cast<__nv_bfloat162*>(PA + t * plane + (int64_t)(q.prow + i) * Ka + kk) = p;
  }
}

// Column exponents of B (k x n): one warp per column; item blockIdx.y.
__global__ void k_tc_col_exp(const TcSrc* __restrict__ src, int* __restrict__ cexp) {
  const TcSrc q = src[blockIdx.y];
  const int j = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x & 31;
  if (j >= q.rows) return;
  uint64_t mx = 0;
  for (int l = lane; l < q.k; l += 32) {
    const double2 v = q.M[l + (int64_t)j * q.ld];
    mx = max(mx, max(abs_bits(v.x), abs_bits(v.y)));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long other = __shfl_xor_sync(0xFFFFFFFFu, (unsigned long long)mx, o);
    mx = max(mx, (uint64_t)other);
  }
  if (lane == 0) cexp[q.eoff + j] = scale_exp(mx);
}

// Digit planes of the real form of B: PB[u][2j][2l] = Re B_lj, PB[u][2j][2l+1] = -Im B_lj,
// PB[u][2j+1][2l] = Im B_lj, PB[u][2j+1][2l+1] = Re B_lj (digits of; zero beyond 2k).
// One thread per (l, j): reads along the column, writes along the rows.  Column blockIdx.x of
// item blockIdx.z.
__global__ void __launch_bounds__(256) k_tc_split_b(const TcSrc* __restrict__ src, const int* __restrict__ cexp,
                                                    __nv_bfloat16* __restrict__ PB, int64_t plane, int64_t Ka) {
  const TcSrc q = src[blockIdx.z];
  const int j = blockIdx.x;
  if (j >= q.rows) return;
  const int e = cexp[q.eoff + j];
  for (int l = blockIdx.y * blockDim.x + threadIdx.x; 2 * l < Ka; l += gridDim.y * blockDim.x) {
    int dr[TC_S], di[TC_S];
    if (l < q.k) {
      const double2 v = q.M[l + (int64_t)j * q.ld];
      digits7(v.x, e, dr);
      digits7(v.y, e, di);
    } else {
#pragma unroll
      for (int t = 0; t < TC_S; ++t) dr[t] = di[t] = 0;
    }
#pragma unroll
    for (int u = 0; u < TC_S; ++u) {
      __nv_bfloat162 re, im;
      re.x = __float2bfloat16_rn((float)dr[u]);
      re.y = __float2bfloat16_rn((float)-di[u]);
      im.x = __float2bfloat16_rn((float)di[u]);
      im.y = __float2bfloat16_rn((float)dr[u]);
      __nv_bfloat16* row = PB + u * plane + (int64_t)(q.prow + 2 * j) * Ka + 2 * l;
      *reinterpret_cast<__nv_bfloat162*>(row) = re;
      *reinterpret_cast<__nv_bfloat162*>(row + Ka) = im;
    }
  }
}

// ------------------------------------------------------------------ the GEMM ----
// One product of a batched call (C_i = beta C_i + alpha A_i B_i), as the GEMM kernel sees it.
struct TcItem {
  double2* C;
  int64_t ldc;
  int m, n;              // complex sizes of C_i
  int arow, brow;        // first plane row of A_i's digits and of B_i's (2 x column offset)
  int eoff_r, eoff_c;    // first row / column exponent
  int tiles_m, tiles_n;  // its 128-row and 64-real-column tiles
  int tile0;             // index of its first tile in the launch
  int pad;
};

struct TcArgs {
  int nitems, ntiles;
  int nkb;              // K blocks of TC_BK real values (common to all items)
  double2 alpha, beta;
  int sub;              // alpha = -1, beta = 1 (C -= A B): two FP64 additions per entry
  int group;            // row tiles per raster group of the tile order
  const TcItem* items;
  const int* rexp;
  const int* cexp;
};

// Item of launch tile t (binary search over the items' first tiles).
__device__ __forceinline__ int find_item(const TcArgs& a, int t) {
  int lo = 0, hi = a.nitems - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (a.items[mid].tile0 <= t) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Tile r of an item -> (tm, tn): groups of G row tiles, so that the CTAs running at the same
// time share their A and B digit planes in L2.
__device__ __forceinline__ void tile_coords(const TcItem& it, int r, int G, int& tm, int& tn) {
  const int per_group = G * it.tiles_n;
  const int g = r / per_group, q = r % per_group;
  const int gm = min(G, it.tiles_m - g * G);
  tm = g * G + q % gm;
  tn = q / gm;
}

// A1: A is one digit plane of a real matrix (the sketches: Omega = +-1, row scale 2^8).
template <bool A1>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_zgemm_tc(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, const TcArgs a) {
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* gbase = smem_raw + (base - raw);
  int* frac = reinterpret_cast<int*>(gbase + TC_STAGES * TC_STAGE_BYTES);  // F[col][row]
  const uint32_t bars = base + TC_STAGES * TC_STAGE_BYTES + TC_FRAC_BYTES;  // full[S], empty[S], tfull, tempty
  const uint32_t full0 = bars, empty0 = bars + 8 * TC_STAGES, tfull = bars + 16 * TC_STAGES,
                 tempty = tfull + 8;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(gbase + TC_STAGES * TC_STAGE_BYTES + TC_FRAC_BYTES + 128);
  const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
  const int ntiles = a.ntiles;
  const int nchunk_kb = TC_KC / TC_BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(tfull, 1);
    mbar_init(tempty, TC_EPI);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TC_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ---------------------------------------------------------------- TMA producer
    if (lane == 0) {
      uint32_t it = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const TcItem item = a.items[find_item(a, t)];
        int tm, tn;
        tile_coords(item, t - item.tile0, a.group, tm, tn);
        for (int kb = 0; kb < a.nkb && ok; ++kb, ++it) {
          const uint32_t s = it % TC_STAGES, ph = (it / TC_STAGES) & 1;
          if (!(ok = mbar_wait(empty0 + 8 * s, ph ^ 1))) break;
          const uint32_t full = full0 + 8 * s;
          mbar_expect_tx(full, A1 ? TC_A_TILE + TC_S * TC_B_TILE : TC_STAGE_BYTES);
          const uint32_t sa = base + s * TC_STAGE_BYTES, sb = sa + TC_S * TC_A_TILE;
#pragma unroll
          for (int p = 0; p < TC_S; ++p) {
            if (p == 0 || !A1) tma_load_3d(sa + p * TC_A_TILE, &mapA, full, kb * TC_BK, item.arow + tm * TC_BM, p);
            tma_load_3d(sb + p * TC_B_TILE, &mapB, full, kb * TC_BK, item.brow + tn * TC_BN, p);
          }
        }
      }
      // every load issued must have landed before the CTA can leave: wait (bounded) for the
      // last fill of each stage (no later phase of that barrier exists)
      for (uint32_t s = 0; s < TC_STAGES; ++s) {
        if (it <= s) continue;
        const uint32_t last = s + ((it - 1 - s) / TC_STAGES) * TC_STAGES;
        mbar_wait(full0 + 8 * s, (last / TC_STAGES) & 1);
      }
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      uint32_t it = 0, chunk = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        for (int kb0 = 0; kb0 < a.nkb && ok; kb0 += nchunk_kb, ++chunk) {
          if (!(ok = mbar_wait(tempty, (chunk & 1) ^ 1))) break;
          tc_fence_after();
          const int kb1 = min(a.nkb, kb0 + nchunk_kb);
          for (int kb = kb0; kb < kb1; ++kb, ++it) {
            const uint32_t s = it % TC_STAGES, ph = (it / TC_STAGES) & 1;
            if (!(ok = mbar_wait(full0 + 8 * s, ph))) break;
            tc_fence_after();
            const uint32_t sa = base + s * TC_STAGE_BYTES, sb = sa + TC_S * TC_A_TILE;
#pragma unroll
            for (int kk = 0; kk < TC_BK / 16; ++kk) {
#pragma unroll
              for (int e = 0; e < 11; ++e) {
                // one-digit A: only A digit 0 (entries 1 and 2: diagonals 0..3 and 4..6, both
                // started from zero; diagonal 7 stays unused)
                if (A1 && e != 1 && e != 2) continue;
                int tt, u0, cnt;
                tc_sched(e, tt, u0, cnt);
                const uint64_t da = sdesc_sw(sa + tt * TC_A_TILE);
                const uint64_t db = sdesc_sw(sb + u0 * TC_B_TILE);
                const uint32_t acc = (kb > kb0 || kk > 0 || (e >= 2 && !A1)) ? 1u : 0u;
                // K step of 16 BF16 values = 32 bytes = 2 units of the start address
                tc_mma(tmem + (tt + u0) * TC_BN, da + 2 * kk, db + 2 * kk, tc_idesc(cnt * TC_BN), acc);
              }
            }
            tc_commit(empty0 + 8 * s);  // the stage is free once these MMAs have read it
          }
          if (ok) tc_commit(tfull);  // the chunk's accumulators are complete
        }
      }
    }
  } else {
    // ---------------------------------------------------------------- epilogue (warps 2-9)
    const int q = warp & 3;              // TMEM lane quadrant of this warp
    const int half = (warp - 2) / 4;     // which 32 of the tile's 64 real columns
    const int row = q * 32 + lane;       // output row within the tile
    const uint32_t tq = tmem + ((uint32_t)(q * 32) << 16) + half * (TC_BN / 2);
    uint32_t chunk = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      const TcItem item = a.items[find_item(a, t)];
      int tm, tn;
      tile_coords(item, t - item.tile0, a.group, tm, tn);
      long long T[TC_BN / 2];
#pragma unroll
      for (int c = 0; c < TC_BN / 2; ++c) {
        T[c] = 0;
        frac[(half * (TC_BN / 2) + c) * TC_BM + row] = 0;
      }
      for (int kb0 = 0; kb0 < a.nkb; kb0 += nchunk_kb, ++chunk) {
        if (!(ok = mbar_wait(tfull, chunk & 1))) break;
        tc_fence_after();
#pragma unroll
        for (int g = 0; g < TC_BN / 16; ++g) {
          // diagonals in pairs, converted as they arrive (fewer live registers)
          float v0[8], v1[8];
          int p1[8], p3[8], f5[8];
          long long p2[8];
          tmem_ld8(tq + 0 * TC_BN + g * 8, v0);
          tmem_ld8(tq + 1 * TC_BN + g * 8, v1);
          tmem_ld_wait();
#pragma unroll
          for (int c = 0; c < 8; ++c) p1[c] = __float2int_rn(v0[c]) * 256 + __float2int_rn(v1[c]);  // < 2^31
          tmem_ld8(tq + 2 * TC_BN + g * 8, v0);
          tmem_ld8(tq + 3 * TC_BN + g * 8, v1);
          tmem_ld_wait();
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            p2[c] = ((long long)__float2int_rn(v0[c]) << 8) + __float2int_rn(v1[c]);  // up to 2^32
          }
          tmem_ld8(tq + 4 * TC_BN + g * 8, v0);
          tmem_ld8(tq + 5 * TC_BN + g * 8, v1);
          tmem_ld_wait();
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const int i5 = __float2int_rn(v1[c]);
            p3[c] = __float2int_rn(v0[c]) + (i5 >> 8);  // unit 2^-48
            f5[c] = (i5 & 255) << 8;                     // unit 2^-64
          }
          tmem_ld8(tq + 6 * TC_BN + g * 8, v0);
          tmem_ld8(tq + 7 * TC_BN + g * 8, v1);
          tmem_ld_wait();
          if (A1) {
#pragma unroll
            for (int c = 0; c < 8; ++c) v1[c] = 0.0f;
          }
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const int col = half * (TC_BN / 2) + g * 8 + c;
            int* fp = frac + col * TC_BM + row;
            const int fn = *fp + f5[c] + __float2int_rn(v0[c]) + __float2int_rn(v1[c] * (1.0f / 256.0f));
            *fp = fn & 0xFFFF;
            T[g * 8 + c] += ((long long)p1[c] << 24) + (p2[c] << 8) + (long long)p3[c] + (fn >> 16);
          }
        }
        tc_fence_before();
        mbar_arrive(tempty);
      }
      if (!ok) break;
      // C = beta C + alpha (T + F 2^-16) 2^(e_i + f_j - 48); the power of two enters through
      // the exponent field (integer pipe), so C -= A B costs one FMA and one add per value
      const int i = tm * TC_BM + row;
      if (i < item.m) {
        const int ei = a.rexp[item.eoff_r + i];
#pragma unroll
        for (int c = 0; c < TC_BN / 4; ++c) {
          const int j = tn * (TC_BN / 2) + half * (TC_BN / 4) + c;
          if (j >= item.n) continue;
          const int ex = ei + a.cexp[item.eoff_c + j] - 48;
          const int* fp = frac + (half * (TC_BN / 2) + 2 * c) * TC_BM + row;
          double2* p = item.C + i + (int64_t)j * item.ldc;
          if (A1) {
            // the sketch's tiles (one A digit) are short next to their epilogue: the sums become
            // doubles by integer operations (off the FP64 pipe) and are stored (C = A B)
            double xr, xi;
            if (!fixed_to_double(T[2 * c], fp[0], ex, xr))
              xr = scale2(fma((double)fp[0], 1.0 / 65536.0, (double)T[2 * c]), ex);
            if (!fixed_to_double(T[2 * c + 1], fp[TC_BM], ex, xi))
              xi = scale2(fma((double)fp[TC_BM], 1.0 / 65536.0, (double)T[2 * c + 1]), ex);
            *p = make_double2(xr, xi);
            continue;
          }
          const double xr = scale2(fma((double)fp[0], 1.0 / 65536.0, (double)T[2 * c]), ex);
          const double xi = scale2(fma((double)fp[TC_BM], 1.0 / 65536.0, (double)T[2 * c + 1]), ex);
          if (a.sub) {
            const double2 o = *p;
            *p = make_double2(o.x - xr, o.y - xi);
          } else {
            double2 r = make_double2(a.alpha.x * xr - a.alpha.y * xi, a.alpha.x * xi + a.alpha.y * xr);
            if (a.beta.x != 0.0 || a.beta.y != 0.0) {
              const double2 o = *p;
              r.x += a.beta.x * o.x - a.beta.y * o.y;
              r.y += a.beta.x * o.y + a.beta.y * o.x;
            }
            *p = r;
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS));
  }
}

// -------------------------------------------------------------------- host side ----
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static std::once_flag once;
  static EncodeTiledFn fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  });
  return fn;
}

static int64_t tc_ka(int k) { return ((int64_t)2 * k + TC_BK - 1) / TC_BK * TC_BK; }

// Work space of a batched call: digit planes (rows of A and B' of all items, padded each to a
// multiple of 16 rows), exponents, and the three item tables.
static size_t tc_ws_layout(const TcProduct* p, int nitems, int kmax, int64_t* arows, int64_t* brows,
                           size_t* off_exp, size_t* off_tab) {
  int64_t ra = 0, rb = 0, ne = 0;
  for (int i = 0; i < nitems; ++i) {
    ra += (p[i].m + 15) / 16 * 16;
    rb += (2 * (int64_t)p[i].n + 15) / 16 * 16;
    ne += p[i].m + p[i].n;
  }
  const int64_t Ka = tc_ka(kmax);
  size_t b = (size_t)TC_S * (size_t)(ra + rb) * (size_t)Ka * 2;
  b = (b + 255) & ~(size_t)255;
  *off_exp = b;
  b += (size_t)ne * sizeof(int);
  b = (b + 255) & ~(size_t)255;
  *off_tab = b;
  b += (size_t)nitems * (sizeof(TcItem) + 2 * sizeof(TcSrc)) + 256;
  *arows = ra;
  *brows = rb;
  return b;
}

size_t wsbm_zgemm_tc_batched_ws_bytes(const TcProduct* p, int nitems) {
  int kmax = 1;
  for (int i = 0; i < nitems; ++i) kmax = p[i].k > kmax ? p[i].k : kmax;
  int64_t ra, rb;
  size_t oe, ot;
  return tc_ws_layout(p, nitems, kmax, &ra, &rb, &oe, &ot);
}

size_t wsbm_zgemm_tc_ws_bytes(int m, int n, int k) {
  TcProduct p;
  memset(&p, 0, sizeof(p));
  p.m = m;
  p.n = n;
  p.k = k;
  return wsbm_zgemm_tc_batched_ws_bytes(&p, 1);
}

// 3-D map over the digit planes [TC_S][rows][Ka] with boxes of TC_BK x box_rows x 1.
static int make_map(CUtensorMap* map, void* planes, int64_t rows, int64_t Ka, int box_rows, int nplanes = TC_S) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return -3;
  cuuint64_t dims[3] = {(cuuint64_t)Ka, (cuuint64_t)rows, (cuuint64_t)nplanes};
  cuuint64_t strides[2] = {(cuuint64_t)Ka * 2, (cuuint64_t)rows * Ka * 2};
  cuuint32_t box[3] = {TC_BK, (cuuint32_t)box_rows, 1};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, planes, dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, TC_BK == 16 ? CU_TENSOR_MAP_SWIZZLE_32B : CU_TENSOR_MAP_SWIZZLE_64B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : -3;
}

int wsbm_zgemm_tc_plan(const TcProduct* p, int nitems, TcPlan* out) {
  if (!out) return -1;
  out->nitems = 0;
  out->tiles = 0;
  out->ws_bytes = 0;
  out->tab.clear();
  if (nitems <= 0) return 0;
  if (!p || nitems > 65535) return -1;
  int kmax = 1, maxm = 0, maxn = 0;
  for (int i = 0; i < nitems; ++i) {
    const TcProduct& q = p[i];
    if (q.m < 0 || q.n < 0 || q.k < 1 || q.k > 32768) return -1;
    if (q.m > 0 && q.n > 0 && (!q.A || !q.B || !q.C || q.lda < q.m || q.ldb < q.k || q.ldc < q.m)) return -1;
    kmax = q.k > kmax ? q.k : kmax;
    maxm = q.m > maxm ? q.m : maxm;
    maxn = q.n > maxn ? q.n : maxn;
  }
  int64_t ra, rb;
  size_t off_exp, off_tab;
  out->ws_bytes = tc_ws_layout(p, nitems, kmax, &ra, &rb, &off_exp, &off_tab);
  if (ra >= INT32_MAX || rb >= INT32_MAX) return -1;
  // item tables
  out->tab.assign((size_t)nitems * (sizeof(TcItem) + 2 * sizeof(TcSrc)), 0);
  TcItem* items = (TcItem*)out->tab.data();
  TcSrc* sa = (TcSrc*)(out->tab.data() + (size_t)nitems * sizeof(TcItem));
  TcSrc* sb = sa + nitems;
  int64_t arow = 0, brow = 0, eo = 0, tiles = 0;
  for (int i = 0; i < nitems; ++i) {
    const TcProduct& q = p[i];
    TcItem& it = items[i];
    it.C = q.C;
    it.ldc = q.ldc;
    it.m = q.m;
    it.n = q.n;
    it.arow = (int)arow;
    it.brow = (int)brow;
    it.eoff_r = (int)eo;
    it.eoff_c = (int)(eo + q.m);
    it.tiles_m = (q.m + TC_BM - 1) / TC_BM;
    it.tiles_n = (2 * q.n + TC_BN - 1) / TC_BN;
    if (q.m == 0 || q.n == 0) it.tiles_m = it.tiles_n = 0;
    it.tile0 = (int)tiles;
    it.pad = 0;
    tiles += (int64_t)it.tiles_m * it.tiles_n;
    sa[i] = {q.A, q.lda, q.m, q.k, (int)arow, (int)eo};
    sb[i] = {q.B, q.ldb, q.n, q.k, (int)brow, (int)(eo + q.m)};
    arow += (q.m + 15) / 16 * 16;
    brow += (2 * (int64_t)q.n + 15) / 16 * 16;
    eo += q.m + q.n;
  }
  if (tiles >= INT32_MAX) return -1;
  out->nitems = nitems;
  out->tiles = (int)tiles;
  out->kmax = kmax;
  out->maxm = maxm;
  out->maxn = maxn;
  out->ra = ra;
  out->rb = rb;
  out->off_exp = off_exp;
  out->off_tab = off_tab;
  return 0;
}

int wsbm_zgemm_tc_run(const TcPlan& pl, const void* dtab_v, double2 alpha, double2 beta, void* ws,
                      cudaStream_t st, int group) {
  if (pl.nitems <= 0 || pl.tiles == 0) return 0;
  if (group < 1 || group > 64) return -1;
  if (!dtab_v || !ws || ((uintptr_t)ws & 255) != 0) return -1;
  const int nitems = pl.nitems;
  const int64_t Ka = tc_ka(pl.kmax), ra = pl.ra, rb = pl.rb;
  __nv_bfloat16* PA = (__nv_bfloat16*)ws;
  __nv_bfloat16* PB = PA + (size_t)TC_S * ra * Ka;
  int* exps = (int*)((char*)ws + pl.off_exp);
  const unsigned char* dtab = (const unsigned char*)dtab_v;
  const TcItem* ditems = (const TcItem*)dtab;
  const TcSrc* dsa = (const TcSrc*)(dtab + (size_t)nitems * sizeof(TcItem));
  const TcSrc* dsb = dsa + nitems;
  // digit planes (the padding rows between items are never read into a stored output)
  k_tc_row_exp<<<dim3((pl.maxm + 127) / 128, nitems), 128, 0, st>>>(dsa, exps);
  k_tc_split_a<<<dim3((pl.maxm + 31) / 32, (unsigned)((Ka / 2 + 31) / 32), nitems), 256, 0, st>>>(
      dsa, exps, PA, (int64_t)ra * Ka, Ka);
  k_tc_col_exp<<<dim3((pl.maxn + 7) / 8, nitems), 256, 0, st>>>(dsb, exps);
  k_tc_split_b<<<dim3(pl.maxn, (unsigned)((Ka / 2 + 255) / 256), nitems), 256, 0, st>>>(
      dsb, exps, PB, (int64_t)rb * Ka, Ka);
  wsbm_count_launches(4);
  CUtensorMap ma, mb;
  if (make_map(&ma, PA, ra, Ka, TC_BM) || make_map(&mb, PB, rb, Ka, TC_BN)) return -3;
  TcArgs a;
  a.nitems = nitems;
  a.ntiles = pl.tiles;
  a.nkb = (int)(Ka / TC_BK);
  a.alpha = alpha;
  a.beta = beta;
  a.sub = alpha.x == -1.0 && alpha.y == 0.0 && beta.x == 1.0 && beta.y == 0.0;
  a.group = group;
  a.items = ditems;
  a.rexp = exps;
  a.cexp = exps;
  if (wsbm_smem_optin((const void*)k_zgemm_tc<false>, TC_SMEM) != cudaSuccess) return -3;
  const int grid = pl.tiles < wsbm_sm_count() ? pl.tiles : wsbm_sm_count();
  k_zgemm_tc<false><<<grid, TC_THREADS, TC_SMEM, st>>>(ma, mb, a);
  wsbm_count_launch();
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int wsbm_zgemm_tc_batched_g(const TcProduct* p, int nitems, double2 alpha, double2 beta, void* ws,
                            cudaStream_t st, int group) {
  if (nitems <= 0) return 0;
  if (group < 1 || group > 64) return -1;
  if (!p || !ws || ((uintptr_t)ws & 255) != 0) return -1;
  TcPlan pl;
  if (int rc = wsbm_zgemm_tc_plan(p, nitems, &pl)) return rc;
  if (pl.tiles == 0) return 0;
  // the item tables sit at the end of the work space, copied in stream order before the
  // launches that read them
  unsigned char* dtab = (unsigned char*)ws + pl.off_tab;
  if (cudaMemcpyAsync(dtab, pl.tab.data(), pl.tab.size(), cudaMemcpyHostToDevice, st) != cudaSuccess) return -3;
  return wsbm_zgemm_tc_run(pl, dtab, alpha, beta, ws, st, group);
}

int wsbm_zgemm_tc_batched(const TcProduct* p, int nitems, double2 alpha, double2 beta, void* ws, cudaStream_t st) {
  return wsbm_zgemm_tc_batched_g(p, nitems, alpha, beta, ws, st, wsbm_tune_current().tc_group);
}

int wsbm_zgemm_tc(int m, int n, int k, double2 alpha, const double2* A, int64_t lda, const double2* B,
                  int64_t ldb, double2 beta, double2* C, int64_t ldc, void* ws, cudaStream_t st) {
  if (m < 0 || n < 0 || k < 0) return -1;
  if (m == 0 || n == 0) return 0;
  if (k < 1 || k > 32768) return -1;  // the 64-bit recombination is sized for K_real <= 65536
  TcProduct p;
  p.A = A;
  p.lda = lda;
  p.B = B;
  p.ldb = ldb;
  p.C = C;
  p.ldc = ldc;
  p.m = m;
  p.n = n;
  p.k = k;
  p.pad = 0;
  return wsbm_zgemm_tc_batched(&p, 1, alpha, beta, ws, st);
}

// Error flag of the bounded waits: returns it and clears it (synchronizes the stream).
int wsbm_zgemm_tc_status(cudaStream_t st) {
  if (cudaStreamSynchronize(st) != cudaSuccess) return -3;
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_tc_error, sizeof(int)) != cudaSuccess) return -3;
  if (v) {
    const int zero = 0;
    cudaMemcpyToSymbol(g_tc_error, &zero, sizeof(int));
    return -5;
  }
  return 0;
}

// ------------------------------------------------ sketches Y = Omega M (Omega = +-1) ----
// Y_i (l_i x n_i) = Omega[:l_i, :m_i] M_i (m_i x n_i complex) with Omega_rc = -1 when bit 0 of
// the sketch hash of (r, c, seed) is set, else +1, shared by every item.  Omega is exact in BF16
// (one digit plane, row scale 2^8: the value +-1 is the digit +-1 of weight 2^-8), so each
// real-form column of M (Re and Im separately: Omega is real) meets one A digit: 7 digit pairs
// per product, every FP32 sum exact (|sum| <= 256 * 128 per chunk), and Y carries only the
// 56-bit rounding of M relative to its column maximum.
__device__ __forceinline__ uint32_t tc_sk_hash(uint32_t r, uint32_t c, uint32_t seed) {
  uint32_t h = r * 0x9E3779B1u ^ (c * 0x85EBCA77u + seed);
  h ^= h >> 16;
  h *= 0x7FEB352Du;
  h ^= h >> 15;
  h *= 0x846CA68Bu;
  h ^= h >> 16;
  return h;
}

// Omega into the A plane (rows x Ka BF16) and the row exponents (8) of its rows.
__global__ void k_tc_omega(__nv_bfloat16* __restrict__ PA, int rows, int64_t Ka, uint32_t seed,
                           int* __restrict__ rexp) {
  const int64_t tot = (int64_t)rows * Ka;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / Ka), c = (int)(e % Ka);
    PA[e] = __float2bfloat16_rn((tc_sk_hash((uint32_t)r, (uint32_t)c, seed) & 1u) ? -1.0f : 1.0f);
    if (c == 0) rexp[r] = 8;
  }
}

// Digit planes of the real-form columns of M for a real A: PB[u][2j][l] = digit u of Re M_lj,
// PB[u][2j+1][l] = digit u of Im M_lj (zero beyond k).  Column blockIdx.x of item blockIdx.z.
__global__ void __launch_bounds__(256) k_tc_split_b_real(const TcSrc* __restrict__ src, const int* __restrict__ cexp,
                                                         __nv_bfloat16* __restrict__ PB, int64_t plane, int64_t Ka) {
  const TcSrc q = src[blockIdx.z];
  const int j = blockIdx.x;
  if (j >= q.rows) return;
  const int e = cexp[q.eoff + j];
  for (int l = blockIdx.y * blockDim.x + threadIdx.x; l < Ka; l += gridDim.y * blockDim.x) {
    int dr[TC_S], di[TC_S];
    if (l < q.k) {
      const double2 v = q.M[l + (int64_t)j * q.ld];
      digits7(v.x, e, dr);
      digits7(v.y, e, di);
    } else {
#pragma unroll
      for (int t = 0; t < TC_S; ++t) dr[t] = di[t] = 0;
    }
#pragma unroll
    for (int u = 0; u < TC_S; ++u) {
      __nv_bfloat16* row = PB + u * plane + (int64_t)(q.prow + 2 * j) * Ka + l;
      row[0] = __float2bfloat16_rn((float)dr[u]);
      row[Ka] = __float2bfloat16_rn((float)di[u]);
    }
  }
}

static int64_t tc_ka_real(int k) { return ((int64_t)k + TC_BK - 1) / TC_BK * TC_BK; }

// Work space of one sketch launch over items p[0..n) (p[i].m = l_i rows of Y, k = m_i rows of
// M, n = n_i columns): Omega plane, B digit planes, exponents, item tables.
static size_t sk_layout(const TcProduct* p, int n, int64_t* la, int64_t* rb, int64_t* Ka, size_t* off_b,
                        size_t* off_exp, size_t* off_tab) {
  int lmax = 0, kmax = 1;
  int64_t r = 0, ne = 0;
  for (int i = 0; i < n; ++i) {
    lmax = std::max(lmax, p[i].m);
    kmax = std::max(kmax, p[i].k);
    r += (2 * (int64_t)p[i].n + 15) / 16 * 16;
    ne += p[i].n;
  }
  *la = ((int64_t)lmax + 15) / 16 * 16;
  *Ka = tc_ka_real(kmax);
  *rb = r;
  size_t b = (size_t)(*la) * (*Ka) * 2;
  b = (b + 255) & ~(size_t)255;
  *off_b = b;
  b += (size_t)TC_S * r * (*Ka) * 2;
  b = (b + 255) & ~(size_t)255;
  *off_exp = b;
  b += ((size_t)(*la) + ne) * sizeof(int);
  b = (b + 255) & ~(size_t)255;
  *off_tab = b;
  b += (size_t)n * (sizeof(TcItem) + sizeof(TcSrc)) + 256;
  return b;
}

size_t wsbm_sketch_tc_ws_bytes(const TcProduct* p, int nitems) {
  int64_t la, rb, Ka;
  size_t ob, oe, ot;
  return sk_layout(p, nitems, &la, &rb, &Ka, &ob, &oe, &ot);
}

int wsbm_sketch_tc(const TcProduct* p, int nitems, uint32_t seed, void* ws, cudaStream_t st) {
  if (nitems <= 0) return 0;
  if (!p || !ws || ((uintptr_t)ws & 255) != 0 || nitems > 65535) return -1;
  for (int i = 0; i < nitems; ++i) {
    const TcProduct& q = p[i];
    if (q.m < 1 || q.n < 0 || q.k < 1 || q.k > 65536 || !q.B || !q.C || q.ldb < q.k || q.ldc < q.m) return -1;
  }
  int64_t la, rb, Ka;
  size_t off_b, off_exp, off_tab;
  sk_layout(p, nitems, &la, &rb, &Ka, &off_b, &off_exp, &off_tab);
  if (rb >= INT32_MAX || la > 65536) return -1;
  __nv_bfloat16* PA = (__nv_bfloat16*)ws;
  __nv_bfloat16* PB = (__nv_bfloat16*)((char*)ws + off_b);
  int* exps = (int*)((char*)ws + off_exp);
  std::vector<unsigned char> tab((size_t)nitems * (sizeof(TcItem) + sizeof(TcSrc)));
  TcItem* items = (TcItem*)tab.data();
  TcSrc* sb = (TcSrc*)(tab.data() + (size_t)nitems * sizeof(TcItem));
  int64_t brow = 0, eo = la, tiles = 0;
  int maxn = 0;
  for (int i = 0; i < nitems; ++i) {
    const TcProduct& q = p[i];
    TcItem& it = items[i];
    it.C = q.C;
    it.ldc = q.ldc;
    it.m = q.m;
    it.n = q.n;
    it.arow = 0;  // Omega is shared
    it.brow = (int)brow;
    it.eoff_r = 0;
    it.eoff_c = (int)eo;
    it.tiles_m = (q.m + TC_BM - 1) / TC_BM;
    it.tiles_n = (2 * q.n + TC_BN - 1) / TC_BN;
    if (q.n == 0) it.tiles_m = it.tiles_n = 0;
    it.tile0 = (int)tiles;
    it.pad = 0;
    tiles += (int64_t)it.tiles_m * it.tiles_n;
    sb[i] = {q.B, q.ldb, q.n, q.k, (int)brow, (int)eo};
    brow += (2 * (int64_t)q.n + 15) / 16 * 16;
    eo += q.n;
    maxn = std::max(maxn, q.n);
  }
  if (tiles == 0) return 0;
  if (tiles >= INT32_MAX) return -1;
  unsigned char* dtab = (unsigned char*)ws + off_tab;
  if (cudaMemcpyAsync(dtab, tab.data(), tab.size(), cudaMemcpyHostToDevice, st) != cudaSuccess) return -3;
  const TcItem* ditems = (const TcItem*)dtab;
  const TcSrc* dsb = (const TcSrc*)(dtab + (size_t)nitems * sizeof(TcItem));
  {
    const int64_t tot = la * Ka;
    const int g = (int)std::min<int64_t>((tot + 255) / 256, (int64_t)wsbm_sm_count() * 8);
    k_tc_omega<<<g, 256, 0, st>>>(PA, (int)la, Ka, seed, exps);
  }
  k_tc_col_exp<<<dim3((maxn + 7) / 8, nitems), 256, 0, st>>>(dsb, exps);
  k_tc_split_b_real<<<dim3(std::max(maxn, 1), (unsigned)((Ka + 255) / 256), nitems), 256, 0, st>>>(
      dsb, exps, PB, (int64_t)rb * Ka, Ka);
  wsbm_count_launches(3);
  CUtensorMap ma, mb;
  if (make_map(&ma, PA, la, Ka, TC_BM, 1) || make_map(&mb, PB, rb, Ka, TC_BN)) return -3;
  TcArgs a;
  a.nitems = nitems;
  a.ntiles = (int)tiles;
  a.nkb = (int)(Ka / TC_BK);
  a.alpha = make_double2(1.0, 0.0);
  a.beta = make_double2(0.0, 0.0);
  a.sub = 0;
  a.group = wsbm_tune_current().tc_group;
  a.items = ditems;
  a.rexp = exps;
  a.cexp = exps;
  if (wsbm_smem_optin((const void*)k_zgemm_tc<true>, TC_SMEM) != cudaSuccess) return -3;
  const int grid = a.ntiles < wsbm_sm_count() ? a.ntiles : wsbm_sm_count();
  k_zgemm_tc<true><<<grid, TC_THREADS, TC_SMEM, st>>>(ma, mb, a);
  wsbm_count_launch();
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}
