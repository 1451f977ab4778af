// Autotuners of the launch shapes (per device, for the rest of the process).
//
// wsbm_autotune (synthetic data of the caller's sizes):
//   tc_group      rows of 128-row tiles per raster group of the GEMM's tile order (how much of
//                 A and B the CTAs running at the same time share in L2): 4, 8 or 16;
//   box_nb        panel width of the batched box LU (FP64 panel vs tensor-core product work):
//                 32 or 64;
//   root_nb_*     outer panel width of the root LU below / from wsbm_lu_big_large_n() unknowns:
//                 128 or 256;
//   cpqr_cb       trailing columns per warp pass of the warp QR (ID matrices of more than 2048
//                 rows): 2, 4 or 8.
// wsbm_autotune_build (leaf-level builds of the caller's problem):
//   pair_tf, pair_ctas    tile width (16, 32, 64; 128 / width rows) and CTAs per SM (8, 16, 32)
//                         of the node-pair entry kernel;
//   proxy_tf, proxy_ctas  the same for the proxy-block kernel;
//   cpqr_threads          threads per CTA of the thread-per-column QR: 128 or 256.
// Every candidate is timed with CUDA events (the library's own per-kernel events for the build
// shapes) after a warm-up call; the fastest is kept.  Without a call the defaults below hold.
#include <math.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "wsbm_internal.h"

static std::mutex g_tune_mu;
static WsbmTune g_tune[64];
static bool g_tune_init = false;

static WsbmTune tune_default() {
  WsbmTune t;
  t.tc_group = 8;
  t.box_nb = 64;
  t.root_nb_mid = 128;
  t.root_nb_large = 256;
  t.tuned = 0;
  t.pair_tf = WSBM_TILE_F;
  t.pair_ctas = WSBM_ENTRY_CTAS;
  t.proxy_tf = WSBM_TILE_F;
  t.proxy_ctas = WSBM_ENTRY_CTAS;
  t.cpqr_threads = 256;
  t.cpqr_cb = 4;
  t.tuned_build = 0;
  t.solve_tc_min = 1024;
  return t;
}

WsbmTune wsbm_tune_current() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return tune_default();
  std::lock_guard<std::mutex> lk(g_tune_mu);
  if (!g_tune_init) {
    for (auto& t : g_tune) t = tune_default();
    g_tune_init = true;
  }
  return g_tune[dev];
}

static void tune_store(const WsbmTune& t) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  if (!g_tune_init) {
    for (auto& x : g_tune) x = tune_default();
    g_tune_init = true;
  }
  g_tune[dev] = t;
}

// a[i + j ld] = hash-based value in [-1, 1) + i [-1, 1), plus `diag` where j % cper == i (the
// diagonal of each square block when the columns come in groups of cper; cper = 0: none).
__global__ void k_tune_fill(double2* a, int64_t rows, int64_t cols, int64_t ld, uint32_t seed, double diag,
                            int64_t cper) {
  const int64_t tot = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % rows, j = e / rows;
    uint32_t h = (uint32_t)(e * 2654435761u) ^ seed;
    h ^= h >> 15;
    h *= 2246822519u;
    h ^= h >> 13;
    h *= 3266489917u;
    h ^= h >> 16;
    const double re = (double)(h & 0xFFFF) / 32768.0 - 1.0, im = (double)(h >> 16) / 32768.0 - 1.0;
    double2 v = make_double2(re, im);
    if (cper > 0 && j % cper == i) v.x += diag;
    a[i + j * ld] = v;
  }
}

namespace {
struct Timer {
  cudaEvent_t a = nullptr, b = nullptr;
  Timer() {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
  }
  ~Timer() {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
};

int fill(double2* p, int64_t rows, int64_t cols, uint32_t seed, double diag, int64_t cper, cudaStream_t st) {
  const int64_t tot = rows * cols;
  const int g = (int)std::min<int64_t>((tot + 255) / 256, (int64_t)wsbm_sm_count() * 8);
  k_tune_fill<<<g < 1 ? 1 : g, 256, 0, st>>>(p, rows, cols, rows, seed, diag, cper);
  wsbm_count_launch();
  return cudaGetLastError() == cudaSuccess ? WSBM_OK : WSBM_ERR_CUDA;
}
}  // namespace

extern "C" int wsbm_autotune(int32_t n_box, int32_t nbox, int32_t nrhs_box, int32_t n_root, int32_t* out,
                             double* ms, void* stream) {
  // at most 8 GiB per copy of the boxes and 16 GiB per copy of the root matrix
  if (n_box < 64 || n_box > 4096 || nbox < 1 || nbox > 32767 || nrhs_box < 1 || nrhs_box > 4096 || n_root < 256 ||
      n_root > 32768 || (double)nbox * n_box * (n_box + nrhs_box) * 16.0 > 8.0 * (1ull << 30))
    return WSBM_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  WsbmScratch scr(st);
  const WsbmTune t0 = wsbm_tune_current();
  WsbmTune t = t0;
  Timer tm;
  double times[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  auto best_of = [&](auto&& f, double* out_ms) -> int {
    int rc = f();  // warm-up
    if (rc) return rc;
    float best = 1e30f;
    for (int r = 0; r < 3; ++r) {
      cudaEventRecord(tm.a, st);
      if ((rc = f())) return rc;
      cudaEventRecord(tm.b, st);
      if (cudaEventSynchronize(tm.b) != cudaSuccess) return WSBM_ERR_CUDA;
      float v = 0.f;
      cudaEventElapsedTime(&v, tm.a, tm.b);
      best = v < best ? v : best;
    }
    if (wsbm_zgemm_tc_status(st) != 0) return WSBM_ERR_TIMEOUT;
    *out_ms = best;
    return WSBM_OK;
  };
  int rc = WSBM_OK;
  // 1. GEMM raster group: C -= A B, 8192 x 8192 x 256
  {
    const int m = 8192, n = 8192, k = 256;
    double2 *A, *B, *C;
    void* ws;
    if ((rc = scr.get((size_t)m * k * 16, (void**)&A)) || (rc = scr.get((size_t)k * n * 16, (void**)&B)) ||
        (rc = scr.get((size_t)m * n * 16, (void**)&C)) || (rc = scr.get(wsbm_zgemm_tc_ws_bytes(m, n, k), &ws)))
      return rc;
    if ((rc = fill(A, m, k, 1u, 0.0, 0, st)) || (rc = fill(B, k, n, 2u, 0.0, 0, st)) ||
        (rc = fill(C, m, n, 3u, 0.0, 0, st)))
      return rc;
    TcProduct p;
    p.A = A;
    p.lda = m;
    p.B = B;
    p.ldb = k;
    p.C = C;
    p.ldc = m;
    p.m = m;
    p.n = n;
    p.k = k;
    p.pad = 0;
    const int cand[3] = {4, 8, 16};
    double bestv = 1e30;
    for (int c = 0; c < 3; ++c) {
      rc = best_of(
          [&] {
            return wsbm_zgemm_tc_batched_g(&p, 1, make_double2(-1.0, 0.0), make_double2(1.0, 0.0), ws, st, cand[c])
                       ? WSBM_ERR_CUDA
                       : WSBM_OK;
          },
          &times[c]);
      if (rc) return rc;
      if (times[c] < bestv) {
        bestv = times[c];
        t.tc_group = cand[c];
      }
    }
  }
  // 2. box LU panel width: nbox boxes of n_box unknowns with nrhs_box right-hand sides
  {
    const int64_t per = (int64_t)n_box * (n_box + nrhs_box);
    double2 *W0, *W;
    int32_t* piv;
    if ((rc = scr.get((size_t)nbox * per * 16, (void**)&W0)) || (rc = scr.get((size_t)nbox * per * 16, (void**)&W)) ||
        (rc = scr.get((size_t)nbox * n_box * 4, (void**)&piv)))
      return rc;
    // each box: [A | B] with A diagonally dominant
    if ((rc = fill(W0, n_box, (int64_t)nbox * (n_box + nrhs_box), 4u, 2.0 * n_box, n_box + nrhs_box, st))) return rc;
    std::vector<LuSolveDesc> h(nbox);
    std::vector<LuDesc> l(nbox);
    for (int b = 0; b < nbox; ++b) {
      double2* base = W + b * per;
      h[b] = {base, n_box, piv + (int64_t)b * n_box, base + (int64_t)n_box * n_box, n_box, nullptr, n_box, nrhs_box};
      l[b] = {base, n_box, piv + (int64_t)b * n_box, n_box, 0};
    }
    LuSolveDesc* dh;
    LuDesc* dl;
    void* ws;
    if ((rc = scr.get(h.size() * sizeof(LuSolveDesc), (void**)&dh)) ||
        (rc = scr.get(l.size() * sizeof(LuDesc), (void**)&dl)) ||
        (rc = scr.get(wsbm_lu_solve_tc_ws_bytes(h.data(), nbox), &ws)))
      return rc;
    if (cudaMemcpyAsync(dh, h.data(), h.size() * sizeof(LuSolveDesc), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(dl, l.data(), l.size() * sizeof(LuDesc), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return WSBM_ERR_CUDA;
    const int cand[2] = {32, 64};
    double bestv = 1e30;
    for (int c = 0; c < 2; ++c) {
      rc = best_of(
          [&] {
            // a fresh copy each time (the LU works in place), timed alike for every candidate
            if (cudaMemcpyAsync(W, W0, (size_t)nbox * per * 16, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
              return WSBM_ERR_CUDA;
            return wsbm_lu_solve_tc_batched_nb(h.data(), dh, nbox, dl, ws, st, cand[c]) ? WSBM_ERR_CUDA : WSBM_OK;
          },
          &times[3 + c]);
      if (rc) return rc;
      if (times[3 + c] < bestv) {
        bestv = times[3 + c];
        t.box_nb = cand[c];
      }
    }
  }
  // 3. root LU panel width at n_root (the size class of n_root)
  {
    const int64_t n = n_root;
    double2 *A0, *A;
    int32_t* piv;
    void* ws;
    if ((rc = scr.get((size_t)n * n * 16, (void**)&A0)) || (rc = scr.get((size_t)n * n * 16, (void**)&A)) ||
        (rc = scr.get((size_t)n * 4, (void**)&piv)) || (rc = scr.get(wsbm_lu_big_ws_bytes((int)n), &ws)))
      return rc;
    if ((rc = fill(A0, n, n, 5u, 2.0 * sqrt((double)n), n, st))) return rc;
    const int cand[2] = {128, 256};
    double bestv = 1e30;
    int pick = 0;
    for (int c = 0; c < 2; ++c) {
      rc = best_of(
          [&] {
            if (cudaMemcpyAsync(A, A0, (size_t)n * n * 16, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
              return WSBM_ERR_CUDA;
            return wsbm_lu_big_nb(A, n, (int)n, piv, nullptr, ws, st, cand[c]) ? WSBM_ERR_CUDA : WSBM_OK;
          },
          &times[5 + c]);
      if (rc) return rc;
      if (times[5 + c] < bestv) {
        bestv = times[5 + c];
        pick = cand[c];
      }
    }
    if (n_root >= wsbm_lu_big_large_n())
      t.root_nb_large = pick;
    else
      t.root_nb_mid = pick;
  }
  // 4. warp QR columns per pass: 152 ID-shaped matrices of 2560 x 128 (more rows than the
  // thread-per-column variant takes), full QR (128 steps)
  {
    const int m = 2560, n = 128, nb = 152;
    // per matrix: perm (n int), state (2 int, padded), norm2 / nref / tauv (n double each),
    // rdiag0 (1 double, padded to n), betav (n double2)
    const size_t per_state = (size_t)n * 4 + (size_t)n * 4 + (size_t)4 * n * 8 + (size_t)n * 16 + 64;
    double2 *M0, *M;
    char* sw;
    if ((rc = scr.get((size_t)nb * m * n * 16, (void**)&M0)) || (rc = scr.get((size_t)nb * m * n * 16, (void**)&M)) ||
        (rc = scr.get((size_t)nb * per_state, (void**)&sw)))
      return rc;
    if ((rc = fill(M0, m, (int64_t)nb * n, 6u, 0.0, 0, st))) return rc;
    std::vector<QrDesc> q(nb);
    for (int b = 0; b < nb; ++b) {
      char* w = sw + (size_t)b * per_state;
      QrDesc& d = q[b];
      memset(&d, 0, sizeof(d));
      d.A = M + (size_t)b * m * n;
      d.lda = m;
      d.m = m;
      d.n = n;
      d.kt = n;
      d.tol = 0.0;
      d.perm = (int32_t*)w;
      d.state = (int32_t*)(w + (size_t)n * 4);
      d.norm2 = (double*)(w + (size_t)n * 8);
      d.nref = d.norm2 + n;
      d.tauv = d.nref + n;
      d.rdiag0 = d.tauv + n;
      d.betav = (double2*)(d.rdiag0 + n);
    }
    QrDesc* dq;
    if ((rc = scr.get(q.size() * sizeof(QrDesc), (void**)&dq))) return rc;
    if (cudaMemcpyAsync(dq, q.data(), q.size() * sizeof(QrDesc), cudaMemcpyHostToDevice, st) != cudaSuccess)
      return WSBM_ERR_CUDA;
    const int cand[3] = {2, 4, 8};
    double bestv = 1e30;
    int pick = t.cpqr_cb;
    for (int c = 0; c < 3; ++c) {
      WsbmTune tc = t0;
      tc.cpqr_cb = cand[c];
      tune_store(tc);  // wsbm_cpqr_batched reads the table
      rc = best_of(
          [&] {
            if (cudaMemcpyAsync(M, M0, (size_t)nb * m * n * 16, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
                cudaMemsetAsync(sw, 0, (size_t)nb * per_state, st) != cudaSuccess)
              return WSBM_ERR_CUDA;
            return wsbm_cpqr_batched(dq, nb, 1, m, st) ? WSBM_ERR_CUDA : WSBM_OK;
          },
          &times[7 + c]);
      if (rc) {
        tune_store(t0);
        return rc;
      }
      if (times[7 + c] < bestv) {
        bestv = times[7 + c];
        pick = cand[c];
      }
    }
    t.cpqr_cb = pick;
  }
  t.tuned = 1;
  tune_store(t);
  if (out) {
    out[0] = t.tc_group;
    out[1] = t.box_nb;
    out[2] = t.root_nb_mid;
    out[3] = t.root_nb_large;
    out[4] = t.cpqr_cb;
  }
  if (ms)
    for (int i = 0; i < 10; ++i) ms[i] = times[i];
  return WSBM_OK;
}

// Leaf-level builds (max_levels = 1) of the caller's problem with each entry-kernel shape and
// QR block size; the library's per-kernel device times decide (the ID phase's for the QR).
extern "C" int wsbm_autotune_build(const wsbm_geom* g, const wsbm_params* p, int32_t* out, double* ms,
                                   void* stream) {
  if (!g || !p) return WSBM_ERR_INVALID_ARG;
  wsbm_params q = *p;
  q.max_levels = 1;
  const WsbmTune t0 = wsbm_tune_current();
  WsbmTune t = t0;
  double tm_pairs[9], tm_proxy[9], tm_qr[2];
  auto build = [&](const WsbmTune& cand, wsbm_stats_t* so) -> int {
    tune_store(cand);
    wsbm_hss_t h = nullptr;
    int rc = wsbm_create(g, &q, stream, &h);
    if (rc == WSBM_OK) rc = wsbm_factor(h);
    if (rc == WSBM_OK) rc = wsbm_stats(h, so);
    if (h) wsbm_destroy(h);
    return rc;
  };
  wsbm_stats_t so;
  int rc = build(t0, &so);  // warm-up
  const int tfs[3] = {16, 32, 64}, ctas[3] = {8, 16, 32};
  double bp = 1e30, bx = 1e30;
  for (int a = 0; a < 3 && rc == WSBM_OK; ++a)
    for (int b = 0; b < 3 && rc == WSBM_OK; ++b) {
      WsbmTune c = t0;
      c.pair_tf = c.proxy_tf = tfs[a];
      c.pair_ctas = c.proxy_ctas = ctas[b];
      rc = build(c, &so);
      if (rc) break;
      tm_pairs[3 * a + b] = so.ms_pairs;
      tm_proxy[3 * a + b] = so.ms_proxy;
      if (so.ms_pairs < bp) {
        bp = so.ms_pairs;
        t.pair_tf = tfs[a];
        t.pair_ctas = ctas[b];
      }
      if (so.ms_proxy < bx) {
        bx = so.ms_proxy;
        t.proxy_tf = tfs[a];
        t.proxy_ctas = ctas[b];
      }
    }
  const int thr[2] = {128, 256};
  double bq = 1e30;
  for (int a = 0; a < 2 && rc == WSBM_OK; ++a) {
    WsbmTune c = t;
    c.cpqr_threads = thr[a];
    rc = build(c, &so);
    if (rc) break;
    tm_qr[a] = so.ms_id;  // every QR launch of the level (sketch IDs, redone sides, completion)
    if (so.ms_id < bq) {
      bq = so.ms_id;
      t.cpqr_threads = thr[a];
    }
  }
  if (rc) {
    tune_store(t0);
    return rc;
  }
  t.tuned_build = 1;
  tune_store(t);
  if (out) {
    out[0] = t.pair_tf;
    out[1] = t.pair_ctas;
    out[2] = t.proxy_tf;
    out[3] = t.proxy_ctas;
    out[4] = t.cpqr_threads;
  }
  if (ms) {
    for (int i = 0; i < 9; ++i) {
      ms[i] = tm_pairs[i];
      ms[9 + i] = tm_proxy[i];
    }
    ms[18] = tm_qr[0];
    ms[19] = tm_qr[1];
  }
  return WSBM_OK;
}

extern "C" int wsbm_tuning(int32_t* out) {
  if (!out) return WSBM_ERR_INVALID_ARG;
  const WsbmTune t = wsbm_tune_current();
  const int32_t v[13] = {t.tc_group, t.box_nb,     t.root_nb_mid, t.root_nb_large, t.cpqr_cb,
                         t.pair_tf,  t.pair_ctas,  t.proxy_tf,    t.proxy_ctas,    t.cpqr_threads,
                         t.tuned,    t.tuned_build, t.solve_tc_min};
  memcpy(out, v, sizeof(v));
  return WSBM_OK;
}

extern "C" int wsbm_tuning_set(const int32_t* in) {
  if (!in) return WSBM_ERR_INVALID_ARG;
  auto tf_ok = [](int v) { return v == 16 || v == 32 || v == 64; };
  auto ctas_ok = [](int v) { return v >= 1 && v <= 64; };
  if (in[0] < 1 || in[0] > 64 || in[1] < 8 || in[1] > 64 || in[1] % 8 || (in[2] != 128 && in[2] != 256) ||
      (in[3] != 128 && in[3] != 256) || (in[4] != 2 && in[4] != 4 && in[4] != 8) || !tf_ok(in[5]) ||
      !ctas_ok(in[6]) || !tf_ok(in[7]) || !ctas_ok(in[8]) || (in[9] != 128 && in[9] != 256) ||
      (in[10] != 0 && in[10] != 1) || (in[11] != 0 && in[11] != 1) || in[12] < 1)
    return WSBM_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return WSBM_ERR_CUDA;
  if (dev < 0 || dev >= 64) return WSBM_ERR_INVALID_ARG;
  WsbmTune t;
  t.tc_group = in[0];
  t.box_nb = in[1];
  t.root_nb_mid = in[2];
  t.root_nb_large = in[3];
  t.cpqr_cb = in[4];
  t.pair_tf = in[5];
  t.pair_ctas = in[6];
  t.proxy_tf = in[7];
  t.proxy_ctas = in[8];
  t.cpqr_threads = in[9];
  t.tuned = in[10];
  t.tuned_build = in[11];
  t.solve_tc_min = in[12];
  tune_store(t);
  return WSBM_OK;
}
