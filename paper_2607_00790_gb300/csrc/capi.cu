// C ABI: argument checking, scratch management and launches of the stateless calls.
#include <math.h>
#include <string.h>

#include <atomic>
#include <map>
#include <mutex>
#include <utility>

#include "wsbm_internal.h"

static std::atomic<int64_t> g_launches{0};
void wsbm_count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void wsbm_count_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
int64_t wsbm_launch_count() { return g_launches.load(std::memory_order_relaxed); }

// One memory pool per device for the work space of the factor and solve.  The default pool
// unmaps freed memory at every synchronization, so each tree level would map its gigabytes of
// ID matrices again; this pool keeps up to a quarter of the device memory (at most 48 GB)
// mapped between calls.  wsbm_trim_memory() hands the cached part back.
static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[64];

static cudaMemPool_t lib_pool(int dev) {
  if (dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_pool[dev]) {
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    cudaDeviceProp prop;
    uint64_t thr = 0;
    if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) thr = prop.totalGlobalMem / 4;
    if (thr > (48ull << 30)) thr = 48ull << 30;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    g_pool[dev] = pool;
  }
  return g_pool[dev];
}

cudaError_t wsbm_malloc_async(void** p, size_t bytes, int dev, cudaStream_t st) {
  cudaMemPool_t pool = lib_pool(dev);
  if (!pool) return cudaMallocAsync(p, bytes, st);
  return cudaMallocFromPoolAsync(p, bytes, pool, st);
}

// Caller-supplied allocator (wsbm_set_allocator).
static std::mutex g_alloc_mu;
static WsbmAllocator g_alloc;

extern "C" int wsbm_set_allocator(wsbm_alloc_fn alloc, wsbm_free_fn release, void* ctx) {
  if ((alloc == nullptr) != (release == nullptr)) return WSBM_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  g_alloc.alloc = alloc;
  g_alloc.release = release;
  g_alloc.ctx = alloc ? ctx : nullptr;
  return WSBM_OK;
}

WsbmAllocator wsbm_current_allocator() {
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  return g_alloc;
}

int wsbm_dev_alloc(const WsbmAllocator& a, size_t bytes, cudaStream_t st, void** p) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  if (a.alloc) {
    *p = a.alloc(bytes, (void*)st, a.ctx);
    return *p ? WSBM_OK : WSBM_ERR_OOM;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return WSBM_ERR_CUDA;
  if (wsbm_malloc_async(p, bytes, dev, st) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return WSBM_ERR_OOM;
  }
  return WSBM_OK;
}

void wsbm_dev_free(const WsbmAllocator& a, void* p, cudaStream_t st) {
  if (!p) return;
  if (a.alloc)
    a.release(p, (void*)st, a.ctx);
  else
    cudaFreeAsync(p, st);
}

// SM count and shared-memory opt-ins, per device.
static std::mutex g_dev_mu;
static int g_nsm[64];
static std::map<std::pair<int, const void*>, size_t> g_optin;

int wsbm_sm_count() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  std::lock_guard<std::mutex> lk(g_dev_mu);
  if (g_nsm[dev] <= 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
    g_nsm[dev] = n;
  }
  return g_nsm[dev];
}

cudaError_t wsbm_smem_optin(const void* kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_dev_mu);
  size_t& done = g_optin[std::make_pair(dev, kernel)];
  if (bytes <= done) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) done = bytes;
  return e;
}

extern "C" int wsbm_trim_memory(void) {
  std::lock_guard<std::mutex> lk(g_pool_mu);
  for (int d = 0; d < 64; ++d)
    if (g_pool[d] && cudaMemPoolTrimTo(g_pool[d], 0) != cudaSuccess) return WSBM_ERR_CUDA;
  return WSBM_OK;
}

extern "C" const char* wsbm_strerror(int code) {
  switch (code) {
    case WSBM_OK: return "ok";
    case WSBM_ERR_INVALID_ARG: return "invalid argument";
    case WSBM_ERR_OOM: return "out of memory";
    case WSBM_ERR_CUDA: return "CUDA error";
    case WSBM_ERR_RANK_OVERFLOW: return "interpolative decomposition rank above its cap";
    case WSBM_ERR_TIMEOUT: return "bounded device wait timed out";
    case WSBM_ERR_NOT_FACTORED: return "handle not factored";
    case WSBM_ERR_NO_DEVICE: return "no usable CUDA device";
    default: return "unknown error";
  }
}

// Physics of eq. (weakly_bm) from the parameters: k1 = n k0 (mu0 = mu1 = 1), eps1 defaults to
// n^2 eps0, eps0 to 1.
int wsbm_phys_from_params(const wsbm_params* p, Phys* ph) {
  if (!p || !ph) return WSBM_ERR_INVALID_ARG;
  if (!(p->k0 > 0.0) || !(p->refr_index > 0.0) || !isfinite(p->k0) || !isfinite(p->refr_index))
    return WSBM_ERR_INVALID_ARG;
  double eps0 = p->eps0 > 0.0 ? p->eps0 : 1.0;
  double eps1 = p->eps1 > 0.0 ? p->eps1 : p->refr_index * p->refr_index * eps0;
  if (!isfinite(eps0) || !isfinite(eps1)) return WSBM_ERR_INVALID_ARG;
  if (p->formulation < WSBM_FORM_WSBM || p->formulation > WSBM_FORM_PMCHWT) return WSBM_ERR_INVALID_ARG;
  ph->k0 = p->k0;
  ph->k1 = p->refr_index * p->k0;
  ph->eps0 = eps0;
  ph->eps1 = eps1;
  ph->inv_k0 = 1.0 / ph->k0;
  ph->inv_k1 = 1.0 / ph->k1;
  ph->s01 = sqrt(ph->k0 / ph->k1);
  ph->s10 = sqrt(ph->k1 / ph->k0);
  ph->fk0 = (float)ph->k0;
  ph->fk1 = (float)ph->k1;
  ph->frk0 = (float)(1.0 / sqrt(ph->k0));
  ph->frk1 = (float)(1.0 / sqrt(ph->k1));
  ph->finv_k0 = (float)ph->inv_k0;
  ph->feps0 = (float)ph->eps0;
  ph->feps1 = (float)ph->eps1;
  ph->fpad = 0.0f;
  return WSBM_OK;
}

int wsbm_geom_check(const wsbm_geom* g) {
  if (!g || g->n < 2 || g->n > (int64_t)1 << 30) return WSBM_ERR_INVALID_ARG;
  if (!g->x || !g->y || !g->nx || !g->ny || !g->w || !g->kappa) return WSBM_ERR_INVALID_ARG;
  return WSBM_OK;
}

DevGeom wsbm_devgeom(const wsbm_geom* g) {
  DevGeom d;
  d.x = g->x;
  d.y = g->y;
  d.nx = g->nx;
  d.ny = g->ny;
  d.w = g->w;
  d.kappa = g->kappa;
  d.n = g->n;
  return d;
}

#define CK(call)                                  \
  do {                                            \
    if ((call) != cudaSuccess) {                  \
      rc = WSBM_ERR_CUDA;                         \
      goto done;                                  \
    }                                             \
  } while (0)

extern "C" int wsbm_hankel01(const double* z, int64_t n, double* out, int32_t precision,
                             void* stream) {
  if (n < 0 || (n > 0 && (!z || !out))) return WSBM_ERR_INVALID_ARG;
  if (precision != WSBM_FP64 && precision != WSBM_MIXED && precision != WSBM_MIXED_FINE)
    return WSBM_ERR_INVALID_ARG;
  return wsbm_launch_hankel(z, n, out, precision, (cudaStream_t)stream);
}

extern "C" int wsbm_entries_raw(const wsbm_geom* g, const wsbm_params* p, const int64_t* rows,
                                int64_t nr, const int64_t* cols, int64_t nc, void* out,
                                void* stream) {
  int rc = wsbm_geom_check(g);
  if (rc) return rc;
  Phys ph;
  if ((rc = wsbm_phys_from_params(p, &ph))) return rc;
  if (nr < 0 || nc < 0 || nr > INT32_MAX / 2 || nc > INT32_MAX / 2) return WSBM_ERR_INVALID_ARG;
  if (nr == 0 || nc == 0) return WSBM_OK;
  if (!rows || !cols || !out) return WSBM_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  WsbmScratch scr(st);
  int32_t* buf = nullptr;
  PairTask* dtask = nullptr;
  size_t nint = (size_t)3 * nr + 3 * nc;
  if ((rc = scr.get(nint * sizeof(int32_t), (void**)&buf))) return rc;
  if ((rc = scr.get(sizeof(PairTask), (void**)&dtask))) return rc;
  {
    int32_t* rnode = buf;
    int32_t* rpos = rnode + nr;
    int32_t* cnode = rpos + 2 * nr;
    int32_t* cpos = cnode + nc;
    PairTask t;
    memset(&t, 0, sizeof(t));
    t.rnode = rnode;
    t.rpos = rpos;
    t.cnode = cnode;
    t.cpos = cpos;
    t.out = (double2*)out;
    t.ld = nr;
    t.nr = (int32_t)nr;
    t.nc = (int32_t)nc;
    t.trans = 0;
    t.tile0 = 0;
    t.fastc = 0;
    DevGeom dg = wsbm_devgeom(g);
    if ((rc = wsbm_launch_unknowns_to_slots(rows, nr, g->n, rnode, rpos, st))) goto done;
    if ((rc = wsbm_launch_unknowns_to_slots(cols, nc, g->n, cnode, cpos, st))) goto done;
    CK(cudaMemcpyAsync(dtask, &t, sizeof(t), cudaMemcpyHostToDevice, st));
    if (p->formulation == WSBM_FORM_WSBM)
      rc = wsbm_launch_pairs(dg, ph, dtask, 1, wsbm_pair_tiles(t.nr, t.nc, 0), st);
    else
      rc = wsbm_launch_pairs_form(p->formulation, dg, ph, dtask, 1, wsbm_pair_tiles(t.nr, t.nc, 0), st);
    // the task struct lives on this stack frame: wait for the copy before returning
    CK(cudaStreamSynchronize(st));
  }
done:
  return rc;
}

extern "C" int wsbm_proxy_block(const wsbm_geom* g, const wsbm_params* p, int32_t side,
                                const int64_t* idx, int64_t nidx, double cx, double cy, double rho,
                                int32_t P, void* out, void* stream) {
  int rc = wsbm_geom_check(g);
  if (rc) return rc;
  Phys ph;
  if ((rc = wsbm_phys_from_params(p, &ph))) return rc;
  if ((side != 0 && side != 1) || P < 1 || nidx < 0 || nidx > INT32_MAX / 2) return WSBM_ERR_INVALID_ARG;
  if (!(rho > 0.0) || !isfinite(cx) || !isfinite(cy) || !isfinite(rho)) return WSBM_ERR_INVALID_ARG;
  if (p->precision != WSBM_FP64 && p->precision != WSBM_MIXED && p->precision != WSBM_MIXED_FINE)
    return WSBM_ERR_INVALID_ARG;
  // the comparison formulations have FP64 row blocks only (the column block is shared)
  if (p->formulation != WSBM_FORM_WSBM && side == 0 && p->precision != WSBM_FP64)
    return WSBM_ERR_INVALID_ARG;
  if (nidx == 0) return WSBM_OK;
  if (!idx || !out) return WSBM_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  WsbmScratch scr(st);
  int32_t* buf = nullptr;
  ProxyTask* dtask = nullptr;
  if ((rc = scr.get((size_t)3 * nidx * sizeof(int32_t), (void**)&buf))) return rc;
  if ((rc = scr.get(sizeof(ProxyTask), (void**)&dtask))) return rc;
  {
    ProxyTask t;
    memset(&t, 0, sizeof(t));
    t.node = buf;
    t.pos = buf + nidx;
    t.out = (double2*)out;
    t.cx = cx;
    t.cy = cy;
    t.rho = rho;
    t.nn = (int32_t)nidx;
    t.P = P;
    t.side = side;
    t.tr = side == 0 ? 1 : 0;  // row block: box equations are the rows of the output
    t.ld = side == 0 ? nidx : 2 * (int64_t)P;
    t.off = 0;
    t.tile0 = 0;
    DevGeom dg = wsbm_devgeom(g);
    if ((rc = wsbm_launch_unknowns_to_slots(idx, nidx, g->n, buf, buf + nidx, st))) goto done;
    CK(cudaMemcpyAsync(dtask, &t, sizeof(t), cudaMemcpyHostToDevice, st));
    if (side == 0 && p->formulation != WSBM_FORM_WSBM)
      rc = wsbm_launch_proxy_rows_form(p->formulation, dg, ph, dtask, 1, wsbm_proxy_tiles(t.nn, P), st);
    else
      rc = wsbm_launch_proxy(dg, ph, dtask, 1, wsbm_proxy_tiles(t.nn, P), p->precision, st);
    CK(cudaStreamSynchronize(st));
  }
done:
  return rc;
}

extern "C" int wsbm_zgemm(int32_t m, int32_t n, int32_t k, const double* alpha, const void* A, int64_t lda,
                          const void* B, int64_t ldb, const double* beta, void* C, int64_t ldc,
                          void* stream) {
  if (m < 0 || n < 0 || k < 1 || k > 32768 || !alpha || !beta) return WSBM_ERR_INVALID_ARG;
  if (m == 0 || n == 0) return WSBM_OK;
  if (!A || !B || !C || lda < m || ldb < k || ldc < m) return WSBM_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  WsbmScratch scr(st);
  void* ws = nullptr;
  int rc = scr.get(wsbm_zgemm_tc_ws_bytes(m, n, k), &ws);
  if (rc) return rc;
  rc = wsbm_zgemm_tc(m, n, k, make_double2(alpha[0], alpha[1]), (const double2*)A, lda, (const double2*)B, ldb,
                     make_double2(beta[0], beta[1]), (double2*)C, ldc, ws, st);
  if (rc == -1) return WSBM_ERR_INVALID_ARG;
  if (rc) return WSBM_ERR_CUDA;
  rc = wsbm_zgemm_tc_status(st);
  return rc == 0 ? WSBM_OK : (rc == -5 ? WSBM_ERR_TIMEOUT : WSBM_ERR_CUDA);
}

extern "C" int wsbm_lu_dense(void* A, int64_t lda, int32_t n, int32_t* piv, void* stream) {
  if (n < 0 || (n > 0 && (!A || !piv || lda < n))) return WSBM_ERR_INVALID_ARG;
  if (n == 0) return WSBM_OK;
  cudaStream_t st = (cudaStream_t)stream;
  WsbmScratch scr(st);
  void* ws = nullptr;
  int rc = scr.get(wsbm_lu_big_ws_bytes(n), &ws);
  if (rc) return rc;
  rc = wsbm_lu_big((double2*)A, lda, n, piv, nullptr, ws, st);
  if (rc == -1) return WSBM_ERR_INVALID_ARG;
  if (rc) return WSBM_ERR_CUDA;
  rc = wsbm_zgemm_tc_status(st);
  return rc == 0 ? WSBM_OK : (rc == -5 ? WSBM_ERR_TIMEOUT : WSBM_ERR_CUDA);
}

extern "C" int wsbm_zgemm_batched(int32_t count, const wsbm_gemm_item* items, const double* alpha,
                                  const double* beta, void* stream) {
  if (count < 0 || count > 65535 || (count > 0 && !items) || !alpha || !beta) return WSBM_ERR_INVALID_ARG;
  if (count == 0) return WSBM_OK;
  static_assert(sizeof(wsbm_gemm_item) == sizeof(TcProduct), "item layout");
  const TcProduct* p = reinterpret_cast<const TcProduct*>(items);
  for (int i = 0; i < count; ++i)
    if (p[i].k < 1 || p[i].k > 32768 || p[i].m < 0 || p[i].n < 0) return WSBM_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  WsbmScratch scr(st);
  void* ws = nullptr;
  int rc = scr.get(wsbm_zgemm_tc_batched_ws_bytes(p, count), &ws);
  if (rc) return rc;
  rc = wsbm_zgemm_tc_batched(p, count, make_double2(alpha[0], alpha[1]), make_double2(beta[0], beta[1]), ws, st);
  if (rc == -1) return WSBM_ERR_INVALID_ARG;
  if (rc) return WSBM_ERR_CUDA;
  rc = wsbm_zgemm_tc_status(st);
  return rc == 0 ? WSBM_OK : (rc == -5 ? WSBM_ERR_TIMEOUT : WSBM_ERR_CUDA);
}
