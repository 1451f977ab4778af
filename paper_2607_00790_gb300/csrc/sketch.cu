// Randomized row sketch of the ID matrices: Y = Omega M, with Omega an l x m Rademacher matrix
// (entries +-1 from a counter-based hash of (row, column, seed)) and M an m x n complex128
// matrix.  The column-pivoted QR of Y (l rows) then picks the skeleton and the interpolation
// coefficients of M (randomized interpolative decomposition: the column space geometry of M
// survives the sketch for ranks well below l).
//
// The products run on the tensor cores (tcgen05, tc_gemm.cu, wsbm_sketch_tc): Omega is one
// exact BF16 digit plane shared by every matrix of a launch, each column of M is scaled by a
// power of two and written as seven exact 8-bit digits (56 bits), every FP32 sum is exact, and Y
// carries only the 56-bit rounding of M relative to its column maximum.  The matrices of a batch
// go through in launches whose work space (digit planes) stays within a caller's budget.
#include <algorithm>
#include <vector>

#include "wsbm_internal.h"

namespace {

struct SketchDesc {
  const double2* A;
  int64_t lda;
  double2* Y;
  int64_t ldy;
  int32_t m, n, l, pad;
};

TcProduct sk_item(const SketchDesc& d) {
  TcProduct t;
  t.A = nullptr;
  t.lda = 0;
  t.B = d.A;
  t.ldb = d.lda;
  t.C = d.Y;
  t.ldc = d.ldy;
  t.m = d.l;
  t.n = d.n;
  t.k = d.m;
  t.pad = 0;
  return t;
}

// Launch boundaries: consecutive runs of descriptors whose work space fits `cap` (a single
// descriptor always forms a run), at most 65535 per run.
std::vector<std::pair<int, int>> sk_runs(const std::vector<TcProduct>& p, size_t cap, size_t* max_bytes) {
  std::vector<std::pair<int, int>> runs;
  *max_bytes = 0;
  const int n = (int)p.size();
  int i = 0;
  while (i < n) {
    int cnt = std::min(n - i, 65535);
    size_t b = wsbm_sketch_tc_ws_bytes(p.data() + i, cnt);
    while (cnt > 1 && b > cap) {
      cnt = (cnt + 1) / 2;
      b = wsbm_sketch_tc_ws_bytes(p.data() + i, cnt);
    }
    runs.push_back({i, cnt});
    *max_bytes = std::max(*max_bytes, b);
    i += cnt;
  }
  return runs;
}

std::vector<TcProduct> sk_items(const void* h_desc, int ndesc) {
  const SketchDesc* d = (const SketchDesc*)h_desc;
  std::vector<TcProduct> p;
  p.reserve(ndesc);
  for (int i = 0; i < ndesc; ++i) p.push_back(sk_item(d[i]));
  return p;
}

}  // namespace

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

size_t wsbm_sketch_ws_bytes(const void* h_desc, int ndesc, size_t cap) {
  if (ndesc <= 0) return 0;
  size_t mx = 0;
  sk_runs(sk_items(h_desc, ndesc), cap, &mx);
  return mx;
}

int wsbm_sketch_batched(const void* h_desc, int ndesc, uint32_t seed, void* ws, size_t cap, cudaStream_t st) {
  if (ndesc <= 0) return WSBM_OK;
  const std::vector<TcProduct> p = sk_items(h_desc, ndesc);
  size_t mx = 0;
  for (const auto& r : sk_runs(p, cap, &mx)) {
    const int rc = wsbm_sketch_tc(p.data() + r.first, r.second, seed, ws, st);
    if (rc) return rc == -1 ? WSBM_ERR_INVALID_ARG : WSBM_ERR_CUDA;
  }
  return WSBM_OK;
}

extern "C" int wsbm_sketch(const void* A, int64_t lda, int32_t m, int32_t n, int32_t l, void* Y,
                           int64_t ldy, uint32_t seed, void* stream) {
  if (m < 1 || n < 1 || l < 16 || l > 192 || l % 16 || m > 65536 || !A || !Y || lda < m || ldy < l)
    return WSBM_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  SketchDesc h;
  wsbm_sketch_desc_fill(&h, A, lda, Y, ldy, m, n, l);
  WsbmScratch scr(st);
  const size_t need = wsbm_sketch_ws_bytes(&h, 1, 0);
  void* ws = nullptr;
  int rc = scr.get(need, &ws);
  if (!rc) rc = wsbm_sketch_batched(&h, 1, seed, ws, need, st);
  if (!rc && cudaStreamSynchronize(st) != cudaSuccess) rc = WSBM_ERR_CUDA;
  if (!rc && wsbm_zgemm_tc_status(st) == -5) rc = WSBM_ERR_TIMEOUT;
  return rc;
}
