// HSS direct solver for the WSBM system (Sec. III): perfect binary tree over the curve-ordered
// nodes, proxy-surface interpolative decompositions, Martinsson-Rokhlin compressed factor,
// solve, plane-wave right-hand sides and far field.
//
// Unknowns are interleaved inside the library (unknown 2i+c: c = 0 for u_i / the first
// equation at node i, c = 1 for q_i / the second), so every box owns a contiguous range; the
// ABI converts from and to the paper's block order [u; q].
//
// Per tree level, leaves to root, the host builds flat task lists for all boxes of the level
// and each phase is one batched launch (the GPU analogue of the paper's one-block-per-thread
// load balance): entries of the diagonal blocks, sibling blocks and near-field blocks (one
// node-pair kernel), proxy blocks (one proxy kernel), column-pivoted QR of every box's row and
// column ID matrices, LU of the diagonal blocks, D^-1 L, R D^-1 L and its inverse.  Between
// levels the host reads the ranks and skeleton indices (the paper's halo exchange of skeleton
// indices between neighbouring subtrees becomes this read-back).
//
// For box tau with candidate rows I_r and columns I_c (leaf: its unknowns; otherwise the
// children's skeletons), the row ID gives L (A(I_r, far) ~ L A(J_r, far)), the column ID R
// (A(far, I_c) ~ A(far, J_c) R), and the compressed factor stores
//   LU(D), Z = D^-1 L, Dhat = (R D^-1 L)^-1, the column-ID coefficients and permutation.
// Solve:  up   xh = D^-1 b, bt = Dhat R xh;  root: dense LU solve of the merged skeleton system;
//         down x = xh - Z (bt - Dhat y).
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <functional>
#include <memory>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "dense.h"
#include "wsbm_internal.h"

// Randomized leaf IDs: sketch rows l = 16 ceil((n/2 + PAD)/16) and the QR cutoff on a sketch
// relative to that of a full QR (a sketch's trailing singular values are distorted, so its QR
// stops with a slightly tighter cutoff).
#ifndef WSBM_SKETCH_PAD
#define WSBM_SKETCH_PAD 0
#endif
// Boxes of at least this many unknowns (and at most WSBM_LUS_MAXN) are factored by the batched
// LU whose products run on the tensor cores; smaller ones by the fused FP64 kernel.
#ifndef WSBM_LU_TC_MIN
#define WSBM_LU_TC_MIN 128
#endif
// Dense roots of at least this order are factored by the LU whose trailing updates run on
// the tensor cores (wsbm_lu_big); smaller ones by the batched FP64 blocked LU.
// Solves with at least WSBM_TCSOLVE_RHS right-hand sides run their products on the tensor
// cores, and their LU solves of box factors of at least WSBM_LU_TC_MIN unknowns as block solves
// there (WSBM_TCSOLVE_NB rows per block); the LU solves of dense roots of at least
// wsbm_tune_current().solve_tc_min unknowns (1024 unless set) take the block solve from
// WSBM_TCSOLVE_RHS_ROOT right-hand sides on (a large root is read once per solve either way,
// and its FP64 triangular solve is bound by the FP64 pipe already at a few right-hand sides).
// The other LU solves stay FP64 triangular solves.
#ifndef WSBM_TCSOLVE_RHS_ROOT
#define WSBM_TCSOLVE_RHS_ROOT 4
#endif
#ifndef WSBM_TCSOLVE_RHS
#define WSBM_TCSOLVE_RHS 16
#endif
#ifndef WSBM_TCSOLVE_NB
#define WSBM_TCSOLVE_NB 256
#endif
#ifndef WSBM_TCSOLVE_WS
#define WSBM_TCSOLVE_WS ((size_t)4 << 30)  // digit-plane work space of one solve product launch
#endif
#ifndef WSBM_BIGLU_MIN
#define WSBM_BIGLU_MIN 2048
#endif
#ifndef WSBM_SKETCH_CUT
#define WSBM_SKETCH_CUT 0.25  // measured: far-field error 3.6-5.8x tol, as with the full QR
#endif

int wsbm_phys_from_params(const wsbm_params* p, Phys* ph);
int wsbm_geom_check(const wsbm_geom* g);

#define HK(call)                               \
  do {                                         \
    int _rc = (call);                          \
    if (_rc != WSBM_OK) return _rc;            \
  } while (0)
#define HC(call)                                 \
  do {                                           \
    if ((call) != cudaSuccess) return WSBM_ERR_CUDA; \
  } while (0)

struct Box {
  int64_t lo, hi;
  double cx, cy, R, rho;
  int P;
  std::vector<int32_t> cr, cc;  // candidate rows / columns (interleaved unknown ids)
  int n = 0, k = 0;
  std::vector<int32_t> Jr, Jc;
  std::vector<int> near;
  // factor storage (device)
  double2* D = nullptr;   // LU of D, n x n
  int32_t* piv = nullptr;
  double2* Z = nullptr;   // n x k
  double2* Dc = nullptr;  // k x k
  double2* Tc = nullptr;  // k x (n - k)
  int32_t* pc = nullptr;  // n
};

struct Level {
  std::vector<Box> box;
  bool compressed = false;
};

struct wsbm_hss {
  int dev = 0;
  cudaStream_t st = nullptr;
  // allocator of the geometry copy, factors and work space, fixed at creation (null
  // callbacks: the library's pool)
  WsbmAllocator alloc;
  int64_t N = 0;
  double *x = nullptr, *y = nullptr, *nx = nullptr, *ny = nullptr, *w = nullptr, *kappa = nullptr;
  std::vector<double> hx, hy, hw;
  std::vector<int32_t> slot_scratch;  // per-node scratch of make_slots (all -1 between uses)
  DevGeom g;
  Phys ph;
  wsbm_params prm;
  double cut = 0.0;  // CPQR cutoff
  int L = 0, top = 0;
  std::vector<Level> lv;
  double2* root = nullptr;
  int32_t* root_piv = nullptr;
  int root_n = 0;
  bool factored = false;
  uint64_t generation = 0;   // bumped whenever the factors are released (see plan_get)
  std::vector<void*> owned;  // factor allocations
  std::vector<void*> geo;    // the geometry copy
  wsbm_stats_t stats;
  cudaEvent_t ev[14];
  std::shared_ptr<struct SolvePlan> plan;  // solve plan of the last nrhs (see wsbm_solve)
};

// ---------------------------------------------------------------- small kernels ----
__global__ void k_fill_identity(double2* A, int64_t lda, int n) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)n * n;
       t += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(t % n), j = (int)(t / n);
    A[i + (int64_t)j * lda] = make_double2(i == j ? 1.0 : 0.0, 0.0);
  }
}

// Identity into each dst (m x n, leading dimension ldd); batched over blockIdx.y.
struct CopyDesc;
__global__ void k_fill_identity_batched(const CopyDesc* __restrict__ d);

// L (n x k): L[perm[t], t] = 1 for t < k; L[perm[k+s], t] = T[t + s*ldt]  (T: k x (n-k)).
struct BuildLDesc {
  double2* L;
  const double2* T;
  const int32_t* perm;
  int64_t ldt;
  int32_t n, k;
};
__global__ void k_build_L(const BuildLDesc* __restrict__ d) {
  const BuildLDesc q = d[blockIdx.y];
  int64_t tot = (int64_t)q.n * q.k;
  // written by permuted position, so no inverse permutation is needed
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    int pos = (int)(e % q.n), t = (int)(e / q.n);
    double2 v;
    if (pos < q.k)
      v = make_double2(pos == t ? 1.0 : 0.0, 0.0);
    else
      v = q.T[t + (int64_t)(pos - q.k) * q.ldt];
    q.L[q.perm[pos] + (int64_t)t * q.n] = v;
  }
}

// out[t, c] = in[perm[t], c]  (rows gathered; n x ncol)
struct GatherDesc {
  double2* out;
  const double2* in;
  const int32_t* perm;
  int64_t ldo, ldi;
  int32_t n, ncol;
};
__global__ void k_gather_rows(const GatherDesc* __restrict__ d) {
  const GatherDesc q = d[blockIdx.y];
  int64_t tot = (int64_t)q.n * q.ncol;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    int t = (int)(e % q.n), c = (int)(e / q.n);
    q.out[t + (int64_t)c * q.ldo] = q.in[q.perm[t] + (int64_t)c * q.ldi];
  }
}

// out[perm[t], c] -= in[t, c]: applies R^T = Pi^T [I; Tc^T] after its dense part (the
// column-ID permutation is a bijection, so no two threads touch the same row).
__global__ void k_scatter_sub_rows(const GatherDesc* __restrict__ d) {
  const GatherDesc q = d[blockIdx.y];
  int64_t tot = (int64_t)q.n * q.ncol;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    int t = (int)(e % q.n), c = (int)(e / q.n);
    double2* o = q.out + q.perm[t] + (int64_t)c * q.ldo;
    double2 v = q.in[t + (int64_t)c * q.ldi];
    *o = make_double2(o->x - v.x, o->y - v.y);
  }
}

// 2D copy (n rows, ncol columns) between strided matrices, batched.
struct CopyDesc {
  double2* dst;
  const double2* src;
  int64_t ldd, lds;
  int32_t m, n;
};
__global__ void k_fill_identity_batched(const CopyDesc* __restrict__ d) {
  const CopyDesc q = d[blockIdx.y];
  int64_t tot = (int64_t)q.m * q.n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(e % q.m), j = (int)(e / q.m);
    q.dst[i + (int64_t)j * q.ldd] = make_double2(i == j ? 1.0 : 0.0, 0.0);
  }
}

// int32 vector copies, one descriptor per block row of the grid
struct CopyIntDesc {
  int32_t* dst;
  const int32_t* src;
  int64_t n;
};
__global__ void k_copy_int(const CopyIntDesc* __restrict__ d) {
  const CopyIntDesc q = d[blockIdx.y];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < q.n; e += (int64_t)gridDim.x * blockDim.x)
    q.dst[e] = q.src[e];
}

__global__ void k_copy2d(const CopyDesc* __restrict__ d) {
  const CopyDesc q = d[blockIdx.y];
  int64_t tot = (int64_t)q.m * q.n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(e % q.m), j = (int)(e / q.m);
    q.dst[i + (int64_t)j * q.ldd] = q.src[i + (int64_t)j * q.lds];
  }
}

// Plane-wave right-hand side, interleaved: b[2i] = 0, b[2i+1] = -u_in - alpha du_in/dn
//   = (d.n - 1) u_in  (alpha = i/k0, du_in/dn = i k0 (d.n) u_in).  Output in paper order.
// form 2 (eq. pmchwt): b = [-u_in ; -eps0^-1 du_in/dn] = [-u_in ; -(i k0 d.n / eps0) u_in].
__global__ void k_rhs_planewave(DevGeom g, double k0, const double* __restrict__ ang, int nang,
                                double2* __restrict__ rhs, int form, double eps0) {
  int64_t N = g.n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N * nang;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e % N;
    int a = (int)(e / N);
    double ca, sa;
    sincos(ang[a], &sa, &ca);
    double ph = k0 * (ca * g.x[i] + sa * g.y[i]);
    double s, c;
    sincos(ph, &s, &c);
    double dn = ca * g.nx[i] + sa * g.ny[i];
    double2* col = rhs + (int64_t)a * 2 * N;
    if (form == WSBM_FORM_PMCHWT) {
      const double t = k0 * dn / eps0;
      col[i] = make_double2(-c, -s);
      col[N + i] = make_double2(t * s, -t * c);
    } else {
      col[i] = make_double2(0.0, 0.0);
      col[N + i] = make_double2((dn - 1.0) * c, (dn - 1.0) * s);
    }
  }
}

// paper order (2N x nrhs, ld 2N) -> interleaved (2N x nrhs)
__global__ void k_to_interleaved(const double2* __restrict__ in, double2* __restrict__ out, int64_t N,
                                 int nrhs) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < 2 * N * nrhs;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = e % (2 * N), c = e / (2 * N);
    int64_t node = r % N, comp = r / N;
    out[2 * node + comp + c * 2 * N] = in[e];
  }
}

// interleaved x (2N x nrhs) -> u, q (N x nrhs each)
__global__ void k_split_uq(const double2* __restrict__ x, double2* __restrict__ u,
                           double2* __restrict__ q, int64_t N, int nrhs) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N * nrhs;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e % N, c = e / N;
    u[e] = x[2 * i + c * 2 * N];
    q[e] = x[2 * i + 1 + c * 2 * N];
  }
}

// Far field: one CTA per observation angle, all right-hand sides, reduction over nodes.
//   u_inf = e^{i pi/4}/sqrt(8 pi k0) sum_j w_j [-i k0 (xh.n_j) u_j - eps0 q_j] e^{-i k0 xh.x_j}
#define FF_CHUNK 8
__global__ void __launch_bounds__(256) k_farfield(DevGeom g, double k0, double eps0,
                                                  const double2* __restrict__ u,
                                                  const double2* __restrict__ q, int nrhs,
                                                  const double* __restrict__ ang, int nang,
                                                  double2* __restrict__ out) {
  __shared__ double2 red[FF_CHUNK][256 / 32];
  const int a = blockIdx.x;
  double ca, sa;
  sincos(ang[a], &sa, &ca);
  const int64_t N = g.n;
  const double pr = 1.0 / sqrt(8.0 * 3.14159265358979323846 * k0);
  const double2 pref = make_double2(pr * 0.70710678118654752440, pr * 0.70710678118654752440);
  for (int c0 = 0; c0 < nrhs; c0 += FF_CHUNK) {
    double2 acc[FF_CHUNK];
#pragma unroll
    for (int c = 0; c < FF_CHUNK; ++c) acc[c] = make_double2(0.0, 0.0);
    for (int64_t j = threadIdx.x; j < N; j += blockDim.x) {
      double s, cph;
      sincos(k0 * (ca * g.x[j] + sa * g.y[j]), &s, &cph);
      double2 e = make_double2(cph, -s);  // e^{-i k0 xh.x_j}
      double xn = k0 * (ca * g.nx[j] + sa * g.ny[j]);
      double wj = g.w[j];
#pragma unroll
      for (int c = 0; c < FF_CHUNK; ++c) {
        if (c0 + c < nrhs) {
          double2 uj = u[j + (int64_t)(c0 + c) * N], qj = q[j + (int64_t)(c0 + c) * N];
          // -i xn u - eps0 q
          double2 t = make_double2(xn * uj.y - eps0 * qj.x, -xn * uj.x - eps0 * qj.y);
          acc[c].x += wj * (t.x * e.x - t.y * e.y);
          acc[c].y += wj * (t.x * e.y + t.y * e.x);
        }
      }
    }
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < FF_CHUNK; ++c) {
      double2 v = acc[c];
      for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
      }
      if (lane == 0) red[c][wp] = v;
    }
    __syncthreads();
    if (threadIdx.x < FF_CHUNK && c0 + threadIdx.x < nrhs) {
      double2 v = make_double2(0.0, 0.0);
      for (int k = 0; k < 256 / 32; ++k) {
        v.x += red[threadIdx.x][k].x;
        v.y += red[threadIdx.x][k].y;
      }
      out[a + (int64_t)(c0 + threadIdx.x) * nang] =
          make_double2(pref.x * v.x - pref.y * v.y, pref.x * v.y + pref.y * v.x);
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ host helpers ----
// Launch a kernel whose blockIdx.y indexes a descriptor array d[0..n), in chunks of at most
// 65535 descriptors (the grid's y limit), 256 threads a block.
template <class D, class... KA, class... A>
static void launch_y(void (*kern)(const D*, KA...), unsigned gx, int64_t n, const D* d,
                     cudaStream_t st, A... args) {
  for (int64_t y0 = 0; y0 < n; y0 += 65535) {
    const unsigned gy = (unsigned)std::min<int64_t>(65535, n - y0);
    kern<<<dim3(gx, gy), 256, 0, st>>>(d + y0, args...);
    wsbm_count_launch();
  }
}

static int gridfor(int64_t work, int per = 256) {
  int64_t b = (work + per - 1) / per;
  if (b < 1) b = 1;
  if (b > 152 * 16) b = 152 * 16;
  return (int)b;
}

// Pinned staging for host <-> device copies, one buffer per stream: copies from pageable memory
// are staged by the driver at a few GB/s.  The buffer is handed out bump-allocated and reset
// only at the start of a call that ends with its stream synchronized (the build of one tree
// level, the roots, a transposed solve, a create), so nothing staged earlier is still being
// copied; a reset grows it to the previous call's peak.  When it is full, copies fall back to
// pageable memory.
struct PinPool {
  unsigned char* p = nullptr;
  size_t cap = 0, off = 0, peak = 0;
  int users = 0;  // handles created on this stream; the buffer is freed with the last one
};
static std::mutex g_pin_mu;
static std::unordered_map<cudaStream_t, PinPool> g_pin;

static void pin_acquire(cudaStream_t st) {
  std::lock_guard<std::mutex> lk(g_pin_mu);
  ++g_pin[st].users;
}

static void pin_release(cudaStream_t st) {
  std::lock_guard<std::mutex> lk(g_pin_mu);
  auto it = g_pin.find(st);
  if (it == g_pin.end() || --it->second.users > 0) return;
  if (it->second.p) cudaFreeHost(it->second.p);
  g_pin.erase(it);
}

static void pin_reset(cudaStream_t st) {
  // a call that returned early on an error may have left copies queued; an idle stream returns
  // at once
  cudaStreamSynchronize(st);
  std::lock_guard<std::mutex> lk(g_pin_mu);
  PinPool& P = g_pin[st];
  if (P.peak > P.cap) {
    if (P.p) cudaFreeHost(P.p);
    P.p = nullptr;
    P.cap = 0;
    const size_t want = P.peak + P.peak / 4;
    if (cudaMallocHost((void**)&P.p, want) == cudaSuccess) P.cap = want;
    else cudaGetLastError();
  }
  P.off = 0;
  P.peak = 0;
}

static void* pin_take(cudaStream_t st, size_t bytes) {
  std::lock_guard<std::mutex> lk(g_pin_mu);
  PinPool& P = g_pin[st];
  // the offset also advances past requests that did not fit, so the peak is what the whole
  // call needed
  const size_t a = (P.off + 255) & ~(size_t)255;
  P.off = a + bytes;
  P.peak = std::max(P.peak, P.off);
  return (P.p && P.off <= P.cap) ? P.p + a : nullptr;
}

// device memory of a handle, stream ordered on its stream, from the allocator the handle
// captured at creation
static int halloc(wsbm_hss* h, size_t bytes, void** p) {
  return wsbm_dev_alloc(h->alloc, bytes, h->st, p);
}

template <class T>
static int upload(wsbm_hss* h, const std::vector<T>& v, T** d, std::vector<void*>& tmp) {
  *d = nullptr;
  if (v.empty()) return WSBM_OK;
  const size_t bytes = v.size() * sizeof(T);
  HK(halloc(h, bytes, (void**)d));
  tmp.push_back(*d);
  const void* src = v.data();
  if (void* stage = pin_take(h->st, bytes)) {
    memcpy(stage, v.data(), bytes);
    src = stage;
  }
  if (cudaMemcpyAsync(*d, src, bytes, cudaMemcpyHostToDevice, h->st) != cudaSuccess)
    return WSBM_ERR_CUDA;
  return WSBM_OK;
}

static int dalloc(wsbm_hss* h, size_t bytes, void** p, std::vector<void*>& list) {
  if (bytes == 0) bytes = 16;
  HK(halloc(h, bytes, p));
  list.push_back(*p);
  return WSBM_OK;
}

static void free_list(wsbm_hss* h, std::vector<void*>& list) {
  for (void* p : list) wsbm_dev_free(h->alloc, p, h->st);
  list.clear();
}

// Work space of one call: released in stream order when the call returns, also on an early
// error return (free_list empties the list, so an explicit release before is harmless).
struct TmpMem {
  wsbm_hss* h;
  std::vector<void*> v;
  explicit TmpMem(wsbm_hss* hh) : h(hh) {}
  ~TmpMem() { free_list(h, v); }
};

// Slots (node, two output positions) for a list of interleaved unknowns placed at output
// positions base + t.  `at` is a per-node scratch array holding -1 on entry and on exit.
// Per-thread node scratch for make_slots in parallel host loops (holds -1 between uses).
static std::vector<int32_t>& thread_slot_scratch(int64_t n) {
  static thread_local std::vector<int32_t> at;
  if ((int64_t)at.size() < n) at.assign((size_t)n, -1);
  return at;
}

// Slots of one unknown list (node ids and the positions of their two components).
struct Slots {
  std::vector<int32_t> nodes, pos;
};

static void make_slots(const std::vector<int32_t>& U, int base, std::vector<int32_t>& nodes,
                       std::vector<int32_t>& pos, std::vector<int32_t>& at) {
  for (size_t t = 0; t < U.size(); ++t) {
    int32_t node = U[t] >> 1, comp = U[t] & 1;
    int32_t s = at[node];
    if (s < 0) {
      s = (int32_t)nodes.size();
      at[node] = s;
      nodes.push_back(node);
      pos.push_back(-1);
      pos.push_back(-1);
    }
    pos[2 * (size_t)s + comp] = base + (int32_t)t;
  }
  for (int32_t nd : nodes) at[nd] = -1;
}

// A flat list of pair tasks for one launch (possibly over several curves: `inst` selects the
// curve's geometry and physics); slot arrays are concatenated and uploaded once.
struct PairBatch {
  std::vector<PairTask> tasks;
  PairTask* dtasks = nullptr;
  std::vector<int32_t> ints;  // slot data
  struct Ref {
    int64_t rn, rp, cn, cp;
  };
  std::vector<Ref> refs;
  int64_t tiles = 0, entries = 0, pairs = 0;
  int tf = WSBM_TILE_F, ctas = WSBM_ENTRY_CTAS;  // tile shape and grid, fixed in prepare()

  // entries of the block (rowU x colU) of curve `inst`; `at` is that curve's slot scratch
  int64_t add(int inst, std::vector<int32_t>& at, const std::vector<int32_t>& rowU, int rbase,
              const std::vector<int32_t>& colU, int cbase, double2* out, int64_t ld, int trans) {
    if (rowU.empty() || colU.empty()) return 0;
    Slots R, C;
    make_slots(rowU, rbase, R.nodes, R.pos, at);
    make_slots(colU, cbase, C.nodes, C.pos, at);
    return add_slots(inst, R, C, (int64_t)rowU.size() * colU.size(), out, ld, trans);
  }

  // the same with the slots already made (entries = |rowU| |colU|)
  int64_t add_slots(int inst, const Slots& R, const Slots& C, int64_t e, double2* out, int64_t ld,
                    int trans) {
    if (e == 0) return 0;
    const std::vector<int32_t>&rn = R.nodes, &rp = R.pos, &cn = C.nodes, &cp = C.pos;
    Ref r;
    r.rn = (int64_t)ints.size();
    ints.insert(ints.end(), rn.begin(), rn.end());
    r.rp = (int64_t)ints.size();
    ints.insert(ints.end(), rp.begin(), rp.end());
    r.cn = (int64_t)ints.size();
    ints.insert(ints.end(), cn.begin(), cn.end());
    r.cp = (int64_t)ints.size();
    ints.insert(ints.end(), cp.begin(), cp.end());
    refs.push_back(r);
    PairTask t;
    memset(&t, 0, sizeof(t));
    t.out = out;
    t.ld = ld;
    t.nr = (int32_t)rn.size();
    t.nc = (int32_t)cn.size();
    t.trans = trans;
    t.tile0 = 0;  // counted in prepare() for the launch's tile shape
    t.inst = inst;
    // the longer slot list runs along the fast tile dimension (fewer idle lanes); for equal
    // lengths the one that gives contiguous stores
    t.fastc = t.nc > t.nr ? 1 : (t.nc < t.nr ? 0 : trans);
    entries += e;
    pairs += (int64_t)rn.size() * cn.size();
    tasks.push_back(t);
    return e;
  }

  // tile shape (the tuned one for eq. (weakly_bm), the default for the comparison
  // formulations) and tile numbering, then upload of slot data and task list (before any
  // timed region)
  int prepare(wsbm_hss* h, std::vector<void*>& tmp) {
    if (tasks.empty()) return WSBM_OK;
    if (h->prm.formulation == WSBM_FORM_WSBM) {
      const WsbmTune tu = wsbm_tune_current();
      tf = tu.pair_tf;
      ctas = tu.pair_ctas;
    }
    tiles = 0;
    for (auto& t : tasks) {
      t.tile0 = (int32_t)tiles;
      tiles += wsbm_pair_tiles(t.nr, t.nc, t.fastc, tf);
    }
    if (tiles > INT32_MAX) return WSBM_ERR_INVALID_ARG;
    int32_t* dints = nullptr;
    HK(upload(h, ints, &dints, tmp));
    for (size_t i = 0; i < tasks.size(); ++i) {
      tasks[i].rnode = dints + refs[i].rn;
      tasks[i].rpos = dints + refs[i].rp;
      tasks[i].cnode = dints + refs[i].cn;
      tasks[i].cpos = dints + refs[i].cp;
    }
    return upload(h, tasks, &dtasks, tmp);
  }
  // the formulation is the same for every curve of a launch (checked at batch creation)
  int run(wsbm_hss* h, const DevGeom* geos, const Phys* phys) {
    if (tasks.empty()) return WSBM_OK;
    if (h->prm.formulation != WSBM_FORM_WSBM)
      return wsbm_launch_pairs_form(h->prm.formulation, h->g, h->ph, dtasks, (int)tasks.size(), tiles,
                                    h->st, geos, phys);
    return wsbm_launch_pairs(h->g, h->ph, dtasks, (int)tasks.size(), tiles, h->st, geos, phys, tf, ctas);
  }
};

struct ProxyBatch {
  std::vector<ProxyTask> tasks;
  ProxyTask* dtasks = nullptr;
  std::vector<int32_t> ints;
  std::vector<std::pair<int64_t, int64_t>> refs;
  int64_t tiles = 0, entries = 0, pairs = 0;
  int tf = WSBM_TILE_F, ctas = WSBM_ENTRY_CTAS;  // tile shape and grid, fixed in prepare()

  int64_t add(int inst, std::vector<int32_t>& at, const std::vector<int32_t>& U, const Box& b,
              int side, double2* out, int64_t ld) {
    Slots S;
    make_slots(U, 0, S.nodes, S.pos, at);
    return add_slots(inst, S, (int64_t)U.size(), b, side, out, ld);
  }

  int64_t add_slots(int inst, const Slots& S, int64_t nU, const Box& b, int side, double2* out,
                    int64_t ld) {
    const std::vector<int32_t>&nn = S.nodes, &pp = S.pos;
    refs.push_back({(int64_t)ints.size(), (int64_t)ints.size() + (int64_t)nn.size()});
    ints.insert(ints.end(), nn.begin(), nn.end());
    ints.insert(ints.end(), pp.begin(), pp.end());
    ProxyTask t;
    memset(&t, 0, sizeof(t));
    t.out = out;
    t.ld = ld;
    t.cx = b.cx;
    t.cy = b.cy;
    t.rho = b.rho;
    t.nn = (int32_t)nn.size();
    t.P = b.P;
    t.side = side;
    t.tr = 0;
    t.off = 0;
    t.tile0 = 0;  // counted in prepare()
    t.inst = inst;
    int64_t e = nU * 2 * b.P;
    entries += e;
    pairs += (int64_t)nn.size() * b.P;
    tasks.push_back(t);
    return e;
  }

  // forms: row blocks of a comparison formulation (default tile shape)
  int prepare(wsbm_hss* h, std::vector<void*>& tmp, bool forms = false) {
    if (tasks.empty()) return WSBM_OK;
    if (!forms) {
      const WsbmTune tu = wsbm_tune_current();
      tf = tu.proxy_tf;
      ctas = tu.proxy_ctas;
    }
    tiles = 0;
    for (auto& t : tasks) {
      t.tile0 = (int32_t)tiles;
      tiles += wsbm_proxy_tiles(t.nn, t.P, tf);
    }
    if (tiles > INT32_MAX) return WSBM_ERR_INVALID_ARG;
    int32_t* dints = nullptr;
    HK(upload(h, ints, &dints, tmp));
    for (size_t i = 0; i < tasks.size(); ++i) {
      tasks[i].node = dints + refs[i].first;
      tasks[i].pos = dints + refs[i].second;
    }
    return upload(h, tasks, &dtasks, tmp);
  }
  int run(wsbm_hss* h, int mixed, const DevGeom* geos, const Phys* phys) {
    if (tasks.empty()) return WSBM_OK;
    return wsbm_launch_proxy(h->g, h->ph, dtasks, (int)tasks.size(), tiles, mixed, h->st, geos, phys, tf,
                             ctas);
  }
};

static void box_circle(const wsbm_hss* h, Box& b) {
  double xmin = h->hx[b.lo], xmax = xmin, ymin = h->hy[b.lo], ymax = ymin;
  for (int64_t i = b.lo + 1; i < b.hi; ++i) {
    double a = h->hx[i], c = h->hy[i];
    if (a < xmin) xmin = a;
    if (a > xmax) xmax = a;
    if (c < ymin) ymin = c;
    if (c > ymax) ymax = c;
  }
  b.cx = 0.5 * (xmin + xmax);
  b.cy = 0.5 * (ymin + ymax);
  double R = 0.0;
  for (int64_t i = b.lo; i < b.hi; ++i) {
    double dx = h->hx[i] - b.cx, dy = h->hy[i] - b.cy;
    double d = sqrt(dx * dx + dy * dy);
    if (d > R) R = d;
  }
  b.R = R;
  b.rho = h->prm.proxy_ratio * R;
  // proxy count: the leaf value, grown with the circle so it carries the k1 rho propagating
  // modes plus the evanescent ones down to the cutoff (they decay like (R/rho)^m)
  double need = h->ph.k1 * b.rho + log(1.0 / h->cut) / log(h->prm.proxy_ratio);
  int P = (int)ceil(need);
  if (P < h->prm.nproxy) P = h->prm.nproxy;
  P = (P + 7) / 8 * 8;
  b.P = P;
}

static double elapsed(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  return ms;
}

// -------------------------------------------------------------------------- create ----
extern "C" int wsbm_create(const wsbm_geom* g, const wsbm_params* p, void* stream, wsbm_hss_t* out) {
  if (!out) return WSBM_ERR_INVALID_ARG;
  *out = nullptr;
  int rc = wsbm_geom_check(g);
  if (rc) return rc;
  Phys ph;
  if ((rc = wsbm_phys_from_params(p, &ph))) return rc;
  if (p->leaf < 4 || p->nproxy < 8 || !(p->id_tol > 0.0) || !(p->id_tol < 1.0)) return WSBM_ERR_INVALID_ARG;
  if (p->precision != WSBM_FP64 && p->precision != WSBM_MIXED && p->precision != WSBM_MIXED_FINE)
    return WSBM_ERR_INVALID_ARG;
  if (p->id_method != WSBM_ID_SKETCH && p->id_method != WSBM_ID_FULL) return WSBM_ERR_INVALID_ARG;
  if (p->formulation != WSBM_FORM_WSBM && p->precision != WSBM_FP64) return WSBM_ERR_INVALID_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) return WSBM_ERR_NO_DEVICE;
  wsbm_hss* h = new wsbm_hss();
  cudaGetDevice(&h->dev);
  h->st = (cudaStream_t)stream;
  h->alloc = wsbm_current_allocator();
  pin_acquire(h->st);
  h->N = g->n;
  h->ph = ph;
  h->prm = *p;
  if (!(h->prm.proxy_ratio > 1.0)) h->prm.proxy_ratio = 1.5;
  memset(&h->stats, 0, sizeof(h->stats));
  for (int i = 0; i < 14; ++i) cudaEventCreate(&h->ev[i]);
  size_t bytes = (size_t)h->N * sizeof(double);
  double** dst[6] = {&h->x, &h->y, &h->nx, &h->ny, &h->w, &h->kappa};
  const double* src[6] = {g->x, g->y, g->nx, g->ny, g->w, g->kappa};
  for (int a = 0; a < 6; ++a) {
    if (dalloc(h, bytes, (void**)dst[a], h->geo) != WSBM_OK) {
      wsbm_destroy(h);
      return WSBM_ERR_OOM;
    }
    if (cudaMemcpyAsync(*dst[a], src[a], bytes, cudaMemcpyDeviceToDevice, h->st) != cudaSuccess) {
      wsbm_destroy(h);
      return WSBM_ERR_CUDA;
    }
  }
  h->hx.resize(h->N);
  h->hy.resize(h->N);
  h->slot_scratch.assign(h->N, -1);
  h->hw.resize(h->N);
  std::vector<double> hk(h->N), hnx(h->N), hny(h->N);
  {
    // read the geometry back through the stream's pinned staging buffer when it is large enough
    // (create ends with the stream synchronized, like the calls that reset the buffer)
    pin_reset(h->st);
    std::vector<double>* dsth[6] = {&h->hx, &h->hy, &h->hw, &hnx, &hny, &hk};
    const double* srch[6] = {g->x, g->y, g->w, g->nx, g->ny, g->kappa};
    void* stage[6];
    for (int a = 0; a < 6; ++a) {
      stage[a] = pin_take(h->st, bytes);
      cudaMemcpyAsync(stage[a] ? stage[a] : (void*)dsth[a]->data(), srch[a], bytes,
                      cudaMemcpyDeviceToHost, h->st);
    }
    if (cudaStreamSynchronize(h->st) != cudaSuccess) {
      wsbm_destroy(h);
      return WSBM_ERR_CUDA;
    }
    for (int a = 0; a < 6; ++a)
      if (stage[a]) memcpy(dsth[a]->data(), stage[a], bytes);
  }
  for (int64_t i = 0; i < h->N; ++i) {
    if (!isfinite(h->hx[i]) || !isfinite(h->hy[i]) || !isfinite(h->hw[i]) || !isfinite(hk[i]) ||
        !isfinite(hnx[i]) || !isfinite(hny[i]) || !(h->hw[i] > 0.0)) {
      wsbm_destroy(h);
      return WSBM_ERR_INVALID_ARG;
    }
  }
  h->g.x = h->x;
  h->g.y = h->y;
  h->g.nx = h->nx;
  h->g.ny = h->ny;
  h->g.w = h->w;
  h->g.kappa = h->kappa;
  h->g.n = h->N;
  // tree: perfect binary tree over contiguous node ranges
  int L = 0;
  while (((h->N) >> L) > p->leaf && L < 24) ++L;
  if (L > 0 && (h->N >> L) < 2) --L;
  h->L = L;
  // CPQR cutoff: the errors of the 2^L leaf-box IDs (and of the levels above) add up in the
  // solution roughly incoherently, so the cutoff shrinks with the square root of the number of
  // leaf boxes; the factor 4 keeps densities and far field within a few id_tol of the dense
  // solution on 15-node-per-wavelength curves up to N = 32768
  h->cut = p->id_tol / (4.0 * sqrt((double)((int64_t)1 << L)));
  h->lv.resize(L + 1);
  for (int l = 0; l <= L; ++l) {
    int nb = 1 << l;
    h->lv[l].box.resize(nb);
    for (int b = 0; b < nb; ++b) {
      Box& bx = h->lv[l].box[b];
      bx.lo = (int64_t)((__int128)b * h->N / nb);
      bx.hi = (int64_t)((__int128)(b + 1) * h->N / nb);
      box_circle(h, bx);
    }
  }
  h->stats.levels = L;
  h->stats.nboxes_leaf = 1 << L;
  *out = h;
  return WSBM_OK;
}

static void release_factors(wsbm_hss* h) {
  h->plan.reset();  // a solve plan refers to the factors
  ++h->generation;  // and so does any batch plan that includes this handle
  free_list(h, h->owned);
  for (auto& l : h->lv) l.compressed = false;
  for (auto& l : h->lv)
    for (auto& b : l.box) {
      b.D = b.Z = b.Dc = b.Tc = nullptr;
      b.piv = b.pc = nullptr;
      b.k = b.n = 0;
      b.cr.clear();
      b.cc.clear();
      b.Jr.clear();
      b.Jc.clear();
      b.near.clear();
    }
  h->root = nullptr;
  h->root_piv = nullptr;
  h->root_n = 0;
  h->factored = false;
}

extern "C" void wsbm_destroy(wsbm_hss_t h) {
  if (!h) return;
  release_factors(h);
  free_list(h, h->geo);
  cudaStreamSynchronize(h->st);
  pin_release(h->st);
  for (int i = 0; i < 14; ++i)
    if (h->ev[i]) cudaEventDestroy(h->ev[i]);
  delete h;
}

// ---------------------------------------------------------------------- one level ----
// A box of one tree level of one curve, as seen by a (possibly batched) level build.
struct BoxRef {
  wsbm_hss* h;
  int inst;  // index of h in the batch (selects geometry and physics in the kernels)
  int l, b;
  Box& box() const { return h->lv[l].box[b]; }
};

// Per-launch device copies of the curves' geometry and physics, indexed by instance.
struct InstArrays {
  DevGeom* geos = nullptr;
  Phys* phys = nullptr;
};
static int upload_instances(wsbm_hss* h0, const std::vector<wsbm_hss*>& hs, InstArrays* ia,
                            std::vector<void*>& tmp) {
  std::vector<DevGeom> g;
  std::vector<Phys> p;
  for (auto* h : hs) {
    g.push_back(h->g);
    p.push_back(h->ph);
  }
  HK(upload(h0, g, &ia->geos, tmp));
  return upload(h0, p, &ia->phys, tmp);
}

// Compress and factor one tree level of each item (a curve and its level): every phase is one
// launch over all boxes of all items (entries, proxy blocks, IDs, LU, D^-1 L, Dhat).  All
// handles share one stream.  Candidates (cr, cc) of every box must be set.
// Algorithmic flops of the fused LU + solve of an n x n matrix with nrhs right-hand sides:
// multipliers (one complex multiply, 6 flops) and trailing updates (one complex FMA, 8 flops) of
// the LU, the forward and backward substitutions, and the pivot scalings of the back solve.
static double lu_solve_flops(double n, double nrhs) {
  const double a = n * (n - 1) / 2, b = (n - 1) * n * (2 * n - 1) / 6;
  return 6 * a + 8 * b + 16 * a * nrhs + 6 * n * nrhs;
}

static int factor_levels(const std::vector<wsbm_hss*>& hs, const std::vector<int>& levels,
                         double ms_out[5], int64_t* cpqr_mats, double* cpqr_flops,
                         int64_t sketch_out[2], double* sketch_ms, double lu_out[4]) {
  wsbm_hss* h0 = hs[0];
  cudaStream_t st = h0->st;
  pin_reset(st);  // the previous level ended with the stream synchronized
  TmpMem tmpm(h0);
  std::vector<void*>& tmp = tmpm.v;
  std::vector<BoxRef> R;
  for (size_t i = 0; i < hs.size(); ++i) {
    if (levels[i] < 1) continue;
    int nb = (int)hs[i]->lv[levels[i]].box.size();
    for (int b = 0; b < nb; ++b) R.push_back({hs[i], (int)i, levels[i], b});
  }
  const int NB = (int)R.size();
  if (NB == 0) return WSBM_OK;
  InstArrays ia;
  HK(upload_instances(h0, hs, &ia, tmp));
  // ---- near candidates: the candidate rows / columns of the other boxes of the same level
  // whose nodes lie inside the proxy circle.  Everything outside the circle is represented by
  // the proxy sources, whatever box it belongs to.  Only boxes whose bounding circle meets the
  // proxy circle are scanned.
  std::vector<std::vector<int32_t>> NR(NB), NC(NB);
#pragma omp parallel for schedule(dynamic, 16)
  for (int r = 0; r < NB; ++r) {
    wsbm_hss* h = R[r].h;
    Level& LV = h->lv[R[r].l];
    const int nb = (int)LV.box.size();
    Box& B = R[r].box();
    B.near.clear();
    const double r2 = B.rho * B.rho;
    for (int s2 = 0; s2 < nb; ++s2) {
      if (s2 == R[r].b) continue;
      const Box& S = LV.box[s2];
      double cdx = S.cx - B.cx, cdy = S.cy - B.cy;
      double reach = B.rho + S.R;
      if (cdx * cdx + cdy * cdy >= reach * reach) continue;
      size_t nr0 = NR[r].size(), nc0 = NC[r].size();
      for (int32_t u : S.cr) {
        double dx = h->hx[u >> 1] - B.cx, dy = h->hy[u >> 1] - B.cy;
        if (dx * dx + dy * dy < r2) NR[r].push_back(u);
      }
      for (int32_t u : S.cc) {
        double dx = h->hx[u >> 1] - B.cx, dy = h->hy[u >> 1] - B.cy;
        if (dx * dx + dy * dy < r2) NC[r].push_back(u);
      }
      if (NR[r].size() > nr0 || NC[r].size() > nc0) B.near.push_back(s2);
    }
  }
  // ---- storage: D and its pivots (kept, per curve), ID matrices (temporary)
  std::vector<int64_t> mr(NB), mc(NB);
  std::vector<size_t> Dtot(hs.size(), 0), ntot_h(hs.size(), 0);
  size_t Mtot = 0, ntot = 0;
  int maxn = 0;
  for (int r = 0; r < NB; ++r) {
    Box& B = R[r].box();
    B.n = (int)B.cr.size();
    mr[r] = 2 * (int64_t)B.P + (int64_t)NC[r].size();
    mc[r] = 2 * (int64_t)B.P + (int64_t)NR[r].size();
    Dtot[R[r].inst] += (size_t)B.n * B.n;
    ntot_h[R[r].inst] += B.n;
    Mtot += (size_t)(mr[r] + mc[r]) * B.n;
    ntot += B.n;
    maxn = std::max(maxn, B.n);
  }
  std::vector<double2*> Dall(hs.size(), nullptr);
  std::vector<int32_t*> pivall(hs.size(), nullptr);
  for (size_t i = 0; i < hs.size(); ++i) {
    if (!Dtot[i]) continue;
    HK(dalloc(hs[i], Dtot[i] * sizeof(double2), (void**)&Dall[i], hs[i]->owned));
    HK(dalloc(hs[i], ntot_h[i] * sizeof(int32_t), (void**)&pivall[i], hs[i]->owned));
  }
  double2* Mall = nullptr;
  HK(dalloc(h0, Mtot * sizeof(double2), (void**)&Mall, tmp));
  std::vector<double2*> Mr(NB), Mc(NB);
  {
    std::vector<size_t> oD(hs.size(), 0), oN(hs.size(), 0);
    size_t oM = 0;
    for (int r = 0; r < NB; ++r) {
      Box& B = R[r].box();
      int i = R[r].inst;
      B.D = Dall[i] + oD[i];
      B.piv = pivall[i] + oN[i];
      oD[i] += (size_t)B.n * B.n;
      oN[i] += B.n;
      Mr[r] = Mall + oM;
      oM += (size_t)mr[r] * B.n;
      Mc[r] = Mall + oM;
      oM += (size_t)mc[r] * B.n;
    }
  }
  // ---- entries: diagonal blocks (leaf) or sibling blocks (upper), near blocks, proxy blocks
  PairBatch pb;
  ProxyBatch xbp[3];  // per precision mode of the curves (one proxy launch each)
  ProxyBatch xbf;     // row blocks of the comparison formulations (eqs. bm, pmchwt), FP64
  std::vector<CopyDesc> copies;
  std::vector<int64_t> e_pairs(hs.size(), 0), e_proxy(hs.size(), 0);
  // slots of every box's lists in parallel (per-thread scratch), then the batches in box order
  // (the task order, and so every result, is that of a serial build)
  struct BoxSlots {
    Slots cr, cc, nc, nr, s1r, s1c, s2r, s2c;
  };
  std::vector<BoxSlots> bs(NB);
#pragma omp parallel for schedule(dynamic, 16)
  for (int r = 0; r < NB; ++r) {
    wsbm_hss* h = R[r].h;
    const int l = R[r].l;
    Box& B = R[r].box();
    std::vector<int32_t>& at = thread_slot_scratch(h->N);
    BoxSlots& S = bs[r];
    make_slots(B.cr, 0, S.cr.nodes, S.cr.pos, at);
    make_slots(B.cc, 0, S.cc.nodes, S.cc.pos, at);
    make_slots(NC[r], 2 * B.P, S.nc.nodes, S.nc.pos, at);
    make_slots(NR[r], 2 * B.P, S.nr.nodes, S.nr.pos, at);
    if (l != h->L) {
      Box& A1 = h->lv[l + 1].box[2 * R[r].b];
      Box& A2 = h->lv[l + 1].box[2 * R[r].b + 1];
      make_slots(A1.Jr, 0, S.s1r.nodes, S.s1r.pos, at);
      make_slots(A2.Jc, A1.k, S.s1c.nodes, S.s1c.pos, at);
      make_slots(A2.Jr, A1.k, S.s2r.nodes, S.s2r.pos, at);
      make_slots(A1.Jc, 0, S.s2c.nodes, S.s2c.pos, at);
    }
  }
  for (int r = 0; r < NB; ++r) {
    wsbm_hss* h = R[r].h;
    const int i = R[r].inst, l = R[r].l;
    Box& B = R[r].box();
    const BoxSlots& S = bs[r];
    if (l == h->L) {
      e_pairs[i] += pb.add_slots(i, S.cr, S.cc, (int64_t)B.cr.size() * B.cc.size(), B.D, B.n, 0);
    } else {
      Box& A1 = h->lv[l + 1].box[2 * R[r].b];
      Box& A2 = h->lv[l + 1].box[2 * R[r].b + 1];
      int ka = A1.k, kb = A2.k;
      e_pairs[i] += pb.add_slots(i, S.s1r, S.s1c, (int64_t)A1.Jr.size() * A2.Jc.size(), B.D, B.n, 0);
      e_pairs[i] += pb.add_slots(i, S.s2r, S.s2c, (int64_t)A2.Jr.size() * A1.Jc.size(), B.D, B.n, 0);
      copies.push_back({B.D, A1.Dc, B.n, ka, ka, ka});
      copies.push_back({B.D + ka + (int64_t)ka * B.n, A2.Dc, B.n, kb, kb, kb});
    }
    // row ID matrix (stored transposed: rows = near columns) and column ID matrix
    e_pairs[i] += pb.add_slots(i, S.cr, S.nc, (int64_t)B.cr.size() * NC[r].size(), Mr[r], mr[r], 1);
    e_pairs[i] += pb.add_slots(i, S.nr, S.cc, (int64_t)NR[r].size() * B.cc.size(), Mc[r], mc[r], 0);
    ProxyBatch& xb = xbp[h->prm.precision];
    ProxyBatch& xr = h->prm.formulation != WSBM_FORM_WSBM ? xbf : xb;
    e_proxy[i] += xr.add_slots(i, S.cr, (int64_t)B.cr.size(), B, 0, Mr[r], mr[r]);
    e_proxy[i] += xb.add_slots(i, S.cc, (int64_t)B.cc.size(), B, 1, Mc[r], mc[r]);
  }
  if (!copies.empty()) {
    CopyDesc* dc = nullptr;
    HK(upload(h0, copies, &dc, tmp));
    int64_t mx = 0;
    for (auto& c : copies) mx = std::max(mx, (int64_t)c.m * c.n);
    launch_y(k_copy2d, gridfor(mx), (int64_t)copies.size(), dc, st);
  }
  HK(pb.prepare(h0, tmp));
  for (auto& xb : xbp) HK(xb.prepare(h0, tmp));
  HK(xbf.prepare(h0, tmp, true));
  // timed: the entry kernels only
  HC(cudaEventRecord(h0->ev[0], st));
  HK(pb.run(h0, ia.geos, ia.phys));
  HC(cudaEventRecord(h0->ev[4], st));
  for (int m = 0; m < 3; ++m) HK(xbp[m].run(h0, m, ia.geos, ia.phys));
  if (!xbf.tasks.empty())
    HK(wsbm_launch_proxy_rows_form(h0->prm.formulation, h0->g, h0->ph, xbf.dtasks, (int)xbf.tasks.size(),
                                   xbf.tiles, st, ia.geos, ia.phys));
  HC(cudaEventRecord(h0->ev[1], st));
  for (size_t i = 0; i < hs.size(); ++i) {
    hs[i]->stats.entries_generated += e_pairs[i] + e_proxy[i];
    hs[i]->stats.entries_pairs += e_pairs[i];
    hs[i]->stats.entries_proxy += e_proxy[i];
  }
  // pair counts are kept per launch; a single curve owns them all
  if (hs.size() == 1) {
    h0->stats.pairs_evaluated += pb.pairs + xbp[0].pairs + xbp[1].pairs + xbp[2].pairs + xbf.pairs;
    h0->stats.pairs_pairs += pb.pairs;
    h0->stats.pairs_proxy += xbp[0].pairs + xbp[1].pairs + xbp[2].pairs + xbf.pairs;
  }
  // ---- randomized sketches of the leaf-level ID matrices (tensor cores): Y = Omega M with
  // l = max(32, 16 ceil((n/2 + WSBM_SKETCH_PAD)/16)) rows, where M has at least 1.5 l rows;
  // their QR stops at WSBM_SKETCH_CUT times the cutoff of a full QR
  std::vector<int> lsk(2 * NB, 0);
  std::vector<double2*> Ysk(2 * NB, nullptr);
  bool sketched = false;
  {
    size_t Ytot = 0;
    for (int r = 0; r < NB; ++r) {
      wsbm_hss* h = R[r].h;
      Box& B = R[r].box();
      if (h->prm.id_method != WSBM_ID_SKETCH || R[r].l != h->L || B.n < 64) continue;
      const int l = std::max(32, 16 * ((B.n / 2 + WSBM_SKETCH_PAD + 15) / 16));
      for (int s2 = 0; s2 < 2; ++s2) {
        const int64_t m = s2 == 0 ? mr[r] : mc[r];
        if (l > 192 || m < (3 * (int64_t)l) / 2 || m > 65536) continue;
        lsk[2 * r + s2] = l;
        Ytot += (size_t)l * B.n;
      }
    }
    if (Ytot) {
      double2* Yall = nullptr;
      HK(dalloc(h0, Ytot * sizeof(double2), (void**)&Yall, tmp));
      const size_t dsz = wsbm_sketch_desc_size();
      std::vector<unsigned char> sd;
      size_t oY = 0;
      int nsk = 0;
      for (int r = 0; r < NB; ++r)
        for (int s2 = 0; s2 < 2; ++s2) {
          const int l = lsk[2 * r + s2];
          if (!l) continue;
          Box& B = R[r].box();
          Ysk[2 * r + s2] = Yall + oY;
          oY += (size_t)l * B.n;
          sd.resize(sd.size() + dsz);
          const int64_t m = s2 == 0 ? mr[r] : mc[r];
          wsbm_sketch_desc_fill(sd.data() + (size_t)nsk * dsz, s2 == 0 ? Mr[r] : Mc[r], m,
                                Ysk[2 * r + s2], l, (int32_t)m, B.n, l);
          ++nsk;
        }
      // digit-plane work space of the tensor-core sketches: at most 4 GiB per launch
      const size_t cap = (size_t)4 << 30;
      void* skws = nullptr;
      HK(dalloc(h0, wsbm_sketch_ws_bytes(sd.data(), nsk, cap), &skws, tmp));
      HC(cudaEventRecord(h0->ev[12], st));
      HK(wsbm_sketch_batched(sd.data(), nsk, 0x5eed1234u, skws, cap, st));
      HC(cudaEventRecord(h0->ev[13], st));
      sketch_out[0] += nsk;
      sketched = true;  // timed after the next synchronization
    }
  }
  // ---- interpolative decompositions: CPQR of Mr (row ID) and Mc (column ID) of every box
  // (or of their sketches)
  std::vector<QrDesc> qd(2 * NB);
  int32_t *perm = nullptr, *state = nullptr;
  double *norm2 = nullptr, *nref = nullptr, *tauv = nullptr, *rd0 = nullptr;
  double2* betav = nullptr;
  HK(dalloc(h0, 2 * ntot * sizeof(double), (void**)&nref, tmp));
  HK(dalloc(h0, 2 * ntot * sizeof(int32_t), (void**)&perm, tmp));
  HK(dalloc(h0, 2 * NB * 2 * sizeof(int32_t), (void**)&state, tmp));
  HK(dalloc(h0, 2 * ntot * sizeof(double), (void**)&norm2, tmp));
  HK(dalloc(h0, 2 * ntot * sizeof(double), (void**)&tauv, tmp));
  HK(dalloc(h0, 2 * ntot * sizeof(double2), (void**)&betav, tmp));
  HK(dalloc(h0, 2 * NB * sizeof(double), (void**)&rd0, tmp));
  HC(cudaMemsetAsync(state, 0, 2 * NB * 2 * sizeof(int32_t), st));
  {
    size_t on = 0;
    for (int r = 0; r < NB; ++r)
      for (int s = 0; s < 2; ++s) {
        QrDesc& q = qd[2 * r + s];
        memset(&q, 0, sizeof(q));
        if (lsk[2 * r + s]) {
          q.A = Ysk[2 * r + s];
          q.lda = lsk[2 * r + s];
        } else {
          q.A = s == 0 ? Mr[r] : Mc[r];
          q.lda = s == 0 ? mr[r] : mc[r];
        }
        q.m = (int32_t)q.lda;
        q.n = R[r].box().n;
        q.tol = R[r].h->cut * (lsk[2 * r + s] ? WSBM_SKETCH_CUT : 1.0);
        q.perm = perm + on;
        q.norm2 = norm2 + on;
        q.nref = nref + on;
        q.tauv = tauv + on;
        q.betav = betav + on;
        q.state = state + 2 * (2 * r + s);
        q.rdiag0 = rd0 + (2 * r + s);
        on += q.n;
      }
  }
  // launch order: largest matrices first, so that the last wave holds the short ones
  std::vector<QrDesc> qs(qd);
  std::stable_sort(qs.begin(), qs.end(), [](const QrDesc& x, const QrDesc& y) {
    return (int64_t)x.m * x.n > (int64_t)y.m * y.n;
  });
  QrDesc* dq = nullptr;
  HK(upload(h0, qs, &dq, tmp));
  HC(cudaEventRecord(h0->ev[5], st));
  int qmax_m = 0;
  for (auto& q : qd) qmax_m = std::max(qmax_m, q.m);
  HK(wsbm_cpqr_batched(dq, 2 * NB, 0, qmax_m, st));
  HC(cudaEventRecord(h0->ev[6], st));
  *cpqr_mats = 2 * (int64_t)NB;
  std::vector<int32_t> hstate(4 * NB);
  HC(cudaMemcpyAsync(hstate.data(), state, hstate.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  HC(cudaStreamSynchronize(st));
  if (sketched) sketch_ms[0] += elapsed(h0->ev[12], h0->ev[13]);
  // algorithmic flops of that launch: 16 per element per reflection step (complex dot and
  // update of the trailing columns) plus the initial column norms
  for (int r = 0; r < NB; ++r)
    for (int s = 0; s < 2; ++s) {
      const QrDesc& q = qd[2 * r + s];
      const int k = hstate[4 * r + 2 * s + 1];
      double f = 4.0 * q.m * q.n;
      for (int j = 0; j < k; ++j) f += 16.0 * (double)(q.m - j) * (double)(q.n - j - 1);
      cpqr_flops[0] += f;
    }
  // a sketched side must leave room for the rank of both sides (the row and column IDs share
  // k): redo it on the full matrix when its rank, or the box's rank, comes within 16 of l
  for (int pass = 0; pass < 2; ++pass) {
    std::vector<QrDesc> redo;
    std::vector<int> which;
    for (int r = 0; r < NB; ++r) {
      const int k = std::max(hstate[4 * r + 1], hstate[4 * r + 3]);
      for (int s = 0; s < 2; ++s) {
        const int l = lsk[2 * r + s];
        if (!l || k + 16 <= l) continue;
        QrDesc& q = qd[2 * r + s];
        q.A = s == 0 ? Mr[r] : Mc[r];
        q.lda = s == 0 ? mr[r] : mc[r];
        q.m = (int32_t)q.lda;
        q.tol = R[r].h->cut;
        lsk[2 * r + s] = 0;
        redo.push_back(q);
        which.push_back(2 * r + s);
      }
    }
    if (redo.empty()) break;
    sketch_out[1] += (int64_t)redo.size();
    for (int w : which)  // restart these QRs from step 0 (the others keep their resume state)
      HC(cudaMemsetAsync(state + 2 * w, 0, 2 * sizeof(int32_t), st));
    QrDesc* dr = nullptr;
    HK(upload(h0, redo, &dr, tmp));
    int rmax = 0;
    for (auto& q : redo) rmax = std::max(rmax, q.m);
    HK(wsbm_cpqr_batched(dr, (int)redo.size(), 0, rmax, st));
    std::vector<int32_t> hs2(4 * NB);
    HC(cudaMemcpyAsync(hs2.data(), state, hs2.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    HC(cudaStreamSynchronize(st));
    for (int w : which) {
      hstate[2 * w] = hs2[2 * w];
      hstate[2 * w + 1] = hs2[2 * w + 1];
    }
  }
  std::vector<QrDesc> more;
  for (int r = 0; r < NB; ++r) {
    Box& B = R[r].box();
    int kr = hstate[4 * r + 1], kc = hstate[4 * r + 3];
    int k = std::max(std::max(kr, kc), 1);
    k = std::min(k, B.n);
    B.k = k;
    for (int s = 0; s < 2; ++s) {
      int ks = s == 0 ? kr : kc;
      if (ks < k) {
        QrDesc q = qd[2 * r + s];
        q.kt = k;
        more.push_back(q);
      }
    }
  }
  if (!more.empty()) {
    QrDesc* dm = nullptr;
    HK(upload(h0, more, &dm, tmp));
    int mmax = 0;
    for (auto& q : more) mmax = std::max(mmax, q.m);
    HK(wsbm_cpqr_batched(dm, (int)more.size(), 1, mmax, st));
  }
  {
    QrDesc* dfin = nullptr;  // the final descriptors (sketched sides may have been redone on M)
    HK(upload(h0, qd, &dfin, tmp));
    HK(wsbm_cpqr_finish(dfin, 2 * NB, st));
  }
  // T = R11^-1 R12 in place (both sides)
  {
    std::vector<TrsmDesc> td;
    int mk = 0, mrhs = 0;
    for (int r = 0; r < NB; ++r)
      for (int s = 0; s < 2; ++s) {
        Box& B = R[r].box();
        TrsmDesc t;
        memset(&t, 0, sizeof(t));
        t.T = qd[2 * r + s].A;
        t.ldt = qd[2 * r + s].lda;
        t.B = qd[2 * r + s].A + (int64_t)B.k * t.ldt;
        t.ldb = t.ldt;
        t.n = B.k;
        t.nrhs = B.n - B.k;
        mk = std::max(mk, t.n);
        mrhs = std::max(mrhs, t.nrhs);
        td.push_back(t);
      }
    TrsmDesc* dtd = nullptr;
    HK(upload(h0, td, &dtd, tmp));
    HK(wsbm_trsm_batched(dtd, (int)td.size(), mk, mrhs, 0, st));
  }
  // the permutations are read on the host after the final synchronization of this call; a
  // pageable read-back here would hold the host until the queue drains
  std::vector<int32_t> hperm(2 * ntot);
  void* perm_stage = pin_take(st, hperm.size() * sizeof(int32_t));
  HC(cudaMemcpyAsync(perm_stage ? perm_stage : (void*)hperm.data(), perm, hperm.size() * sizeof(int32_t),
                     cudaMemcpyDeviceToHost, st));
  HC(cudaEventRecord(h0->ev[2], st));
  // ---- factor: LU(D), Z = D^-1 L, M = R Z, Dhat = M^-1
  std::vector<size_t> Ztot(hs.size(), 0), Ktot(hs.size(), 0), Ttot(hs.size(), 0);
  size_t Zsum = 0, Ksum = 0;
  int maxk = 0;
  for (int r = 0; r < NB; ++r) {
    Box& B = R[r].box();
    int i = R[r].inst;
    Ztot[i] += (size_t)B.n * B.k;
    Ktot[i] += (size_t)B.k * B.k;
    Ttot[i] += (size_t)B.k * (B.n - B.k);
    Zsum += (size_t)B.n * B.k;
    Ksum += (size_t)B.k * B.k;
    maxk = std::max(maxk, B.k);
  }
  std::vector<double2*> Zall(hs.size(), nullptr), Dcall(hs.size(), nullptr), Tcall(hs.size(), nullptr);
  std::vector<int32_t*> pcall(hs.size(), nullptr);
  for (size_t i = 0; i < hs.size(); ++i) {
    if (!ntot_h[i]) continue;
    HK(dalloc(hs[i], Ztot[i] * sizeof(double2), (void**)&Zall[i], hs[i]->owned));
    HK(dalloc(hs[i], Ktot[i] * sizeof(double2), (void**)&Dcall[i], hs[i]->owned));
    HK(dalloc(hs[i], Ttot[i] * sizeof(double2), (void**)&Tcall[i], hs[i]->owned));
    HK(dalloc(hs[i], ntot_h[i] * sizeof(int32_t), (void**)&pcall[i], hs[i]->owned));
  }
  double2 *Mall2 = nullptr, *Zp = nullptr;
  int32_t* pivM = nullptr;
  HK(dalloc(h0, Ksum * sizeof(double2), (void**)&Mall2, tmp));
  HK(dalloc(h0, Zsum * sizeof(double2), (void**)&Zp, tmp));
  HK(dalloc(h0, ntot * sizeof(int32_t), (void**)&pivM, tmp));
  std::vector<LuDesc> luD, luM;
  std::vector<BuildLDesc> bl;
  std::vector<TrsmDesc> zl, ml;
  std::vector<GatherDesc> gz;
  std::vector<GemmDesc> gm;
  std::vector<int> gm_box;  // box of each gm entry
  std::vector<CopyDesc> tcc, pcopy, idd;
  {
    std::vector<size_t> oz(hs.size(), 0), ok(hs.size(), 0), ot(hs.size(), 0), on(hs.size(), 0);
    size_t gz_o = 0, gk_o = 0, gn_o = 0;
    for (int r = 0; r < NB; ++r) {
      Box& B = R[r].box();
      const int i = R[r].inst;
      const int n = B.n, k = B.k;
      B.Z = Zall[i] + oz[i];
      B.Dc = Dcall[i] + ok[i];
      B.Tc = Tcall[i] + ot[i];
      B.pc = pcall[i] + on[i];
      oz[i] += (size_t)n * k;
      ok[i] += (size_t)k * k;
      ot[i] += (size_t)k * (n - k);
      on[i] += n;
      double2* M = Mall2 + gk_o;
      double2* Zg = Zp + gz_o;
      int32_t* pM = pivM + gn_o;
      gz_o += (size_t)n * k;
      gk_o += (size_t)k * k;
      gn_o += n;
      luD.push_back({B.D, n, B.piv, n, 0});
      const QrDesc& qr = qd[2 * r];
      const QrDesc& qc = qd[2 * r + 1];
      bl.push_back({B.Z, qr.A + (int64_t)k * qr.lda, qr.perm, qr.lda, n, k});
      TrsmDesc t;
      memset(&t, 0, sizeof(t));
      t.T = B.D;
      t.ldt = n;
      t.B = B.Z;
      t.ldb = n;
      t.piv = B.piv;
      t.n = n;
      t.nrhs = k;
      zl.push_back(t);
      // Zg = Z[pc, :];  M = Zg[0:k, :] + Tc Zg[k:n, :]
      gz.push_back({Zg, B.Z, qc.perm, n, n, n, k});
      pcopy.push_back({M, Zg, k, n, k, k});
      if (n > k) {
        GemmDesc gd;
        memset(&gd, 0, sizeof(gd));
        gd.A = qc.A + (int64_t)k * qc.lda;
        gd.lda = qc.lda;
        gd.B = Zg + k;
        gd.ldb = n;
        gd.C = M;
        gd.ldc = k;
        gd.m = k;
        gd.n = k;
        gd.k = n - k;
        gd.alpha = make_double2(1.0, 0.0);
        gd.beta = make_double2(1.0, 0.0);
        gm.push_back(gd);
        gm_box.push_back(r);
        tcc.push_back({B.Tc, qc.A + (int64_t)k * qc.lda, k, qc.lda, k, n - k});
      }
      luM.push_back({M, k, pM, k, 0});
      TrsmDesc tm;
      memset(&tm, 0, sizeof(tm));
      tm.T = M;
      tm.ldt = k;
      tm.B = B.Dc;
      tm.ldb = k;
      tm.piv = pM;
      tm.n = k;
      tm.nrhs = k;
      ml.push_back(tm);
      idd.push_back({B.Dc, nullptr, k, 0, k, k});
    }
  }
  LuDesc *dluD = nullptr, *dluM = nullptr;
  BuildLDesc* dbl = nullptr;
  TrsmDesc *dzl = nullptr, *dml = nullptr;
  GatherDesc* dgz = nullptr;
  CopyDesc *dtcc = nullptr, *dpc = nullptr, *didd = nullptr;
  HK(upload(h0, luD, &dluD, tmp));
  HK(upload(h0, luM, &dluM, tmp));
  HK(upload(h0, bl, &dbl, tmp));
  HK(upload(h0, zl, &dzl, tmp));
  HK(upload(h0, ml, &dml, tmp));
  HK(upload(h0, gz, &dgz, tmp));
  HK(upload(h0, tcc, &dtcc, tmp));
  HK(upload(h0, pcopy, &dpc, tmp));
  HK(upload(h0, idd, &didd, tmp));
  int64_t maxnk = 0;
  for (int r = 0; r < NB; ++r) maxnk = std::max(maxnk, (int64_t)R[r].box().n * R[r].box().k);
  // LU(D) with Z = D^-1 L, and LU(M) with Dhat = M^-1 (and M += Tc Zg[k:n] before it), chosen
  // per box so that a box's factors do not depend on the other boxes of the launch: boxes of
  // WSBM_LU_TC_MIN unknowns or more by the batched LU whose products run on the tensor cores,
  // the others in the fused FP64 kernel; when a box exceeds the fused kernel, every box of the
  // launch by the blocked LU and triangular solves
  const bool fits = maxn <= WSBM_LUS_MAXN;
  std::vector<int> itc, ifu;
  for (int r = 0; r < NB; ++r) (fits && R[r].box().n >= WSBM_LU_TC_MIN ? itc : ifu).push_back(r);
  if (itc.size() > 32767) {  // beyond one batched launch: the fused kernel for all
    ifu.insert(ifu.end(), itc.begin(), itc.end());
    std::sort(ifu.begin(), ifu.end());
    itc.clear();
  }
  std::vector<char> on_tc(NB, 0);
  for (int r : itc) on_tc[r] = 1;
  const bool lu_tc = !itc.empty();
  LuSolveDesc *dfz = nullptr, *dfm = nullptr, *dfz_t = nullptr, *dfm_t = nullptr;
  LuDesc *dluD_t = nullptr, *dluM_t = nullptr;
  std::vector<LuSolveDesc> fz_t, fm_t;
  std::vector<TcProduct> gm_t;
  std::vector<GemmDesc> gm_f;
  GemmDesc* dgm_f = nullptr;
  int maxn_f = 0, maxk_f = 0;
  void* wstc = nullptr;
  for (size_t g = 0; g < gm.size(); ++g) {
    if (on_tc[gm_box[g]])
      gm_t.push_back({gm[g].A, gm[g].lda, gm[g].B, gm[g].ldb, gm[g].C, gm[g].ldc, gm[g].m, gm[g].n, gm[g].k, 0});
    else
      gm_f.push_back(gm[g]);
  }
  if (!gm_f.empty()) HK(upload(h0, gm_f, &dgm_f, tmp));
  if (fits) {
    // fused kernel: its row-major scratch for the boxes it takes (one scratch serves both launches)
    size_t sz = 0, sm = 0;
    for (int r : ifu) {
      const Box& B = R[r].box();
      sz += (size_t)B.n * wsbm_lu_solve_ldr(B.n, B.k);
      sm += (size_t)B.k * wsbm_lu_solve_ldr(B.k, B.k);
      maxn_f = std::max(maxn_f, B.n);
      maxk_f = std::max(maxk_f, B.k);
    }
    if (!ifu.empty()) {
      double2* Sc = nullptr;
      HK(dalloc(h0, std::max(sz, sm) * sizeof(double2), (void**)&Sc, tmp));
      std::vector<LuSolveDesc> fz(ifu.size()), fm(ifu.size());
      size_t oz = 0, om = 0;
      for (size_t t = 0; t < ifu.size(); ++t) {
        const int r = ifu[t];
        const Box& B = R[r].box();
        fz[t] = {B.D, B.n, B.piv, B.Z, B.n, Sc + oz, B.n, B.k};
        fm[t] = {luM[r].A, B.k, luM[r].piv, B.Dc, B.k, Sc + om, B.k, B.k};
        oz += (size_t)B.n * wsbm_lu_solve_ldr(B.n, B.k);
        om += (size_t)B.k * wsbm_lu_solve_ldr(B.k, B.k);
      }
      HK(upload(h0, fz, &dfz, tmp));
      HK(upload(h0, fm, &dfm, tmp));
    }
    if (lu_tc) {
      std::vector<LuDesc> ld_t, lm_t;
      for (int r : itc) {
        const Box& B = R[r].box();
        fz_t.push_back({B.D, B.n, B.piv, B.Z, B.n, nullptr, B.n, B.k});
        fm_t.push_back({luM[r].A, B.k, luM[r].piv, B.Dc, B.k, nullptr, B.k, B.k});
        ld_t.push_back(luD[r]);
        lm_t.push_back(luM[r]);
      }
      HK(upload(h0, fz_t, &dfz_t, tmp));
      HK(upload(h0, fm_t, &dfm_t, tmp));
      HK(upload(h0, ld_t, &dluD_t, tmp));
      HK(upload(h0, lm_t, &dluM_t, tmp));
      size_t wb = std::max(wsbm_lu_solve_tc_ws_bytes(fz_t.data(), (int)itc.size()),
                           wsbm_lu_solve_tc_ws_bytes(fm_t.data(), (int)itc.size()));
      if (!gm_t.empty()) wb = std::max(wb, wsbm_zgemm_tc_batched_ws_bytes(gm_t.data(), (int)gm_t.size()));
      HK(dalloc(h0, wb, &wstc, tmp));
    }
  }
  launch_y(k_build_L, gridfor(maxnk), NB, dbl, st);
  if (fits) {
    HC(cudaEventRecord(h0->ev[8], st));
    if (dfz) HK(wsbm_lu_solve_fused_batched(dfz, (int)ifu.size(), maxn_f, maxn_f + maxk_f, st));
    if (lu_tc && wsbm_lu_solve_tc_batched(fz_t.data(), dfz_t, (int)itc.size(), dluD_t, wstc, st))
      return WSBM_ERR_CUDA;
    HC(cudaEventRecord(h0->ev[9], st));
  } else {
    HK(wsbm_lu_batched(dluD, NB, maxn, nullptr, st));
    HK(wsbm_lu_solve_batched(dzl, dzl, NB, maxn, maxk, st));
  }
  launch_y(k_gather_rows, gridfor(maxnk), NB, dgz, st);
  launch_y(k_copy2d, gridfor((int64_t)maxk * maxk), NB, dpc, st);
  // M += Tc Zg[k:n]
  if (!gm_t.empty() && wsbm_zgemm_tc_batched(gm_t.data(), (int)gm_t.size(), make_double2(1.0, 0.0),
                                             make_double2(1.0, 0.0), wstc, st))
    return WSBM_ERR_CUDA;
  if (!gm_f.empty()) HK(wsbm_gemm_batched(dgm_f, (int)gm_f.size(), maxk, maxk, st));
  if (!tcc.empty()) {
    launch_y(k_copy2d, gridfor(maxnk), (int64_t)tcc.size(), dtcc, st);
  }
  launch_y(k_fill_identity_batched, gridfor((int64_t)maxk * maxk), NB, didd, st);
  if (fits) {
    HC(cudaEventRecord(h0->ev[10], st));
    if (dfm) HK(wsbm_lu_solve_fused_batched(dfm, (int)ifu.size(), maxk_f, 2 * maxk_f, st));
    if (lu_tc && wsbm_lu_solve_tc_batched(fm_t.data(), dfm_t, (int)itc.size(), dluM_t, wstc, st))
      return WSBM_ERR_CUDA;
    HC(cudaEventRecord(h0->ev[11], st));
  } else {
    HK(wsbm_lu_batched(dluM, NB, maxk, nullptr, st));
    HK(wsbm_lu_solve_batched(dml, dml, NB, maxk, maxk, st));
  }
  HC(cudaGetLastError());
  // column permutations (kept for the solve): one launch copies them out of the QR state
  {
    std::vector<CopyIntDesc> pcd(NB);
    int64_t maxpn = 1;
    size_t on = 0;
    for (int r = 0; r < NB; ++r) {
      const Box& B = R[r].box();
      pcd[r] = {B.pc, perm + on + B.n, B.n};  // column side of box r
      on += 2 * (size_t)B.n;
      maxpn = std::max(maxpn, (int64_t)B.n);
    }
    CopyIntDesc* dpcd = nullptr;
    HK(upload(h0, pcd, &dpcd, tmp));
    launch_y(k_copy_int, gridfor(maxpn), NB, dpcd, st);
  }
  HC(cudaEventRecord(h0->ev[3], st));
  HC(cudaStreamSynchronize(st));
  if (perm_stage) memcpy(hperm.data(), perm_stage, hperm.size() * sizeof(int32_t));
  if (fits) {  // device time, flops and matrices of the box factors' LU + solve launches
    lu_out[0] += elapsed(h0->ev[8], h0->ev[9]) + elapsed(h0->ev[10], h0->ev[11]);
    for (int r = 0; r < NB; ++r) {
      const Box& B = R[r].box();
      lu_out[1] += lu_solve_flops(B.n, B.k) + lu_solve_flops(B.k, B.k);
    }
    lu_out[2] += 2.0 * NB;
    lu_out[3] += 2.0 * (double)itc.size();
  }
  ms_out[0] = elapsed(h0->ev[0], h0->ev[1]);
  ms_out[1] = elapsed(h0->ev[0], h0->ev[4]);
  ms_out[2] = elapsed(h0->ev[1], h0->ev[2]);
  ms_out[3] = elapsed(h0->ev[2], h0->ev[3]);
  ms_out[4] = elapsed(h0->ev[5], h0->ev[6]);
  // skeletons
  {
    size_t on = 0;
    for (int r = 0; r < NB; ++r) {
      Box& B = R[r].box();
      const int32_t* pr = hperm.data() + on;
      on += B.n;
      const int32_t* pcp = hperm.data() + on;
      on += B.n;
      B.Jr.resize(B.k);
      B.Jc.resize(B.k);
      for (int t = 0; t < B.k; ++t) {
        B.Jr[t] = B.cr[pr[t]];
        B.Jc[t] = B.cc[pcp[t]];
      }
      wsbm_hss* h = R[r].h;
      h->stats.rank_per_level[R[r].l] = std::max(h->stats.rank_per_level[R[r].l], B.k);
      h->stats.max_rank = std::max(h->stats.max_rank, B.k);
    }
  }
  for (size_t i = 0; i < hs.size(); ++i)
    if (levels[i] >= 1) hs[i]->lv[levels[i]].compressed = true;
  free_list(h0, tmp);
  return WSBM_OK;
}

// Dense roots: for each curve, merge the skeletons of every box of its top level (all of A when
// its tree has a single box); entries in one launch, LU in one batched call.
static int factor_roots(const std::vector<wsbm_hss*>& hs, double ms_out[2]) {
  wsbm_hss* h0 = hs[0];
  cudaStream_t st = h0->st;
  pin_reset(st);  // the levels ended with the stream synchronized
  TmpMem tmpm(h0);
  std::vector<void*>& tmp = tmpm.v;
  InstArrays ia;
  HK(upload_instances(h0, hs, &ia, tmp));
  PairBatch pb;
  std::vector<CopyDesc> copies;
  std::vector<LuDesc> lus;
  std::vector<int64_t> e_pairs(hs.size(), 0);
  int maxn = 0;
  {
    // a large root needs its memory in one piece: hand the pool's cached work space of the
    // levels back first (the levels ended with the stream synchronized)
    size_t rb = 0;
    for (auto* h : hs) {
      int64_t S = 0;
      if (h->L == 0) S = 2 * h->N;
      else for (auto& b : h->lv[h->top].box) S += b.k;
      rb += (size_t)S * S * sizeof(double2);
    }
    if (rb > ((size_t)4 << 30)) wsbm_trim_memory();
  }
  for (size_t i = 0; i < hs.size(); ++i) {
    wsbm_hss* h = hs[i];
    std::vector<int32_t> Rr, Rc;
    std::vector<int> off;
    if (h->L == 0) {
      for (int64_t u = 0; u < 2 * h->N; ++u) {
        Rr.push_back((int32_t)u);
        Rc.push_back((int32_t)u);
      }
    } else {
      for (auto& b : h->lv[h->top].box) {
        off.push_back((int)Rr.size());
        Rr.insert(Rr.end(), b.Jr.begin(), b.Jr.end());
        Rc.insert(Rc.end(), b.Jc.begin(), b.Jc.end());
      }
    }
    const int n = (int)Rr.size();
    h->root_n = n;
    h->stats.root_size = n;
    maxn = std::max(maxn, n);
    HK(dalloc(h, (size_t)n * n * sizeof(double2), (void**)&h->root, h->owned));
    HK(dalloc(h, (size_t)n * sizeof(int32_t), (void**)&h->root_piv, h->owned));
    if (h->L == 0) {
      e_pairs[i] += pb.add((int)i, h->slot_scratch, Rr, 0, Rc, 0, h->root, n, 0);
    } else {
      Level& T = h->lv[h->top];
      int nb = (int)T.box.size();
      for (int a = 0; a < nb; ++a) {
        Box& A = T.box[a];
        copies.push_back({h->root + off[a] + (int64_t)off[a] * n, A.Dc, n, A.k, A.k, A.k});
        for (int b = 0; b < nb; ++b) {
          if (a == b) continue;
          e_pairs[i] += pb.add((int)i, h->slot_scratch, A.Jr, off[a], T.box[b].Jc, off[b], h->root, n, 0);
        }
      }
    }
    lus.push_back({h->root, n, h->root_piv, n, 0});
  }
  if (!copies.empty()) {
    CopyDesc* dc = nullptr;
    HK(upload(h0, copies, &dc, tmp));
    int64_t mx = 0;
    for (auto& c : copies) mx = std::max(mx, (int64_t)c.m * c.n);
    launch_y(k_copy2d, gridfor(mx), (int64_t)copies.size(), dc, st);
  }
  HK(pb.prepare(h0, tmp));
  HC(cudaEventRecord(h0->ev[0], st));
  HK(pb.run(h0, ia.geos, ia.phys));
  HC(cudaEventRecord(h0->ev[1], st));
  for (size_t i = 0; i < hs.size(); ++i) {
    hs[i]->stats.entries_generated += e_pairs[i];
    hs[i]->stats.entries_pairs += e_pairs[i];
  }
  if (hs.size() == 1) {
    h0->stats.pairs_evaluated += pb.pairs;
    h0->stats.pairs_pairs += pb.pairs;
  }
  // large roots: one at a time through the LU whose trailing updates run on the tensor cores;
  // the others in one batched blocked LU
  {
    std::vector<LuDesc> small;
    int maxs = 0;
    size_t wsb = 0;
    for (auto& l : lus)
      if (l.n >= WSBM_BIGLU_MIN) wsb = std::max(wsb, wsbm_lu_big_ws_bytes(l.n));
    void* ws = nullptr;
    if (wsb) HK(dalloc(h0, wsb, &ws, tmp));
    for (auto& l : lus) {
      if (l.n >= WSBM_BIGLU_MIN) {
        if (wsbm_lu_big(l.A, l.lda, l.n, l.piv, nullptr, ws, st)) return WSBM_ERR_CUDA;
      } else {
        small.push_back(l);
        maxs = std::max(maxs, l.n);
      }
    }
    if (!small.empty()) {
      LuDesc* ds = nullptr;
      HK(upload(h0, small, &ds, tmp));
      HK(wsbm_lu_batched(ds, (int)small.size(), maxs, nullptr, st));
    }
    if (wsb && wsbm_zgemm_tc_status(st) != 0) return WSBM_ERR_TIMEOUT;
  }
  HC(cudaEventRecord(h0->ev[2], st));
  HC(cudaStreamSynchronize(st));
  ms_out[0] = elapsed(h0->ev[0], h0->ev[1]);
  ms_out[1] = elapsed(h0->ev[1], h0->ev[2]);
  free_list(h0, tmp);
  return WSBM_OK;
}

// Build and factor every handle of `hs` (sharing one stream): level by level from the leaves,
// each round batching the current level of every curve that is still compressing (curves of
// different depth are aligned at their leaves), then all dense roots at once.
// bstats (optional) receives the timings of the shared launches.
static int factor_all(const std::vector<wsbm_hss*>& hs, wsbm_stats_t* bstats) {
  wsbm_hss* h0 = hs[0];
  cudaEvent_t t0, t1;
  cudaEventCreate(&t0);
  cudaEventCreate(&t1);
  cudaEventRecord(t0, h0->st);
  const int64_t launches0 = wsbm_launch_count();
  double ms[5] = {0, 0, 0, 0, 0};  // entries, pair kernel, IDs, factor, CPQR
  int64_t cpqr_mats = 0;
  double cpqr_flops = 0.0, ms_sketch = 0.0;
  double lu_acc[4] = {0.0, 0.0, 0.0, 0.0};  // box LU + solve: device ms, flops, matrices, on TC
  int64_t sketch_cnt[2] = {0, 0};  // sketched ID matrices, redone on the full matrix
  std::vector<int> level(hs.size(), 0), done(hs.size(), 0);
  std::vector<char> partial(hs.size(), 0);
  int rc = WSBM_OK;
  // largest dense root that fits in three quarters of the device memory (complex128)
  int64_t mem_cap = INT32_MAX;
  {
    size_t fb = 0, tb = 0;
    if (cudaMemGetInfo(&fb, &tb) == cudaSuccess && tb > 0)
      mem_cap = (int64_t)sqrt(0.75 * (double)tb / (double)sizeof(double2));
  }
  for (size_t i = 0; i < hs.size(); ++i) {
    wsbm_hss* h = hs[i];
    release_factors(h);
    int32_t lev = h->stats.levels, nbl = h->stats.nboxes_leaf;
    memset(&h->stats, 0, sizeof(h->stats));
    h->stats.levels = lev;
    h->stats.nboxes_leaf = nbl;
    h->top = h->L;
    level[i] = h->L;  // 0: nothing to compress
    partial[i] = h->L > 0 && h->prm.max_levels > 0;
    if (h->L > 0) {
      for (auto& b : h->lv[h->L].box) {
        for (int64_t n = b.lo; n < b.hi; ++n) {
          b.cr.push_back((int32_t)(2 * n));
          b.cr.push_back((int32_t)(2 * n + 1));
        }
        b.cc = b.cr;
      }
    }
  }
  for (;;) {
    bool any = false;
    for (int l : level) any = any || l >= 1;
    if (!any) break;
    double m4[5];
    int64_t nq = 0;
    rc = factor_levels(hs, level, m4, &nq, &cpqr_flops, sketch_cnt, &ms_sketch, lu_acc);
    if (rc) break;
    for (int a = 0; a < 5; ++a) ms[a] += m4[a];
    cpqr_mats += nq;
    for (size_t i = 0; i < hs.size(); ++i) {
      if (level[i] < 1) continue;
      wsbm_hss* h = hs[i];
      const int l = level[i];
      h->top = l;
      ++done[i];
      int next = 0;
      if (l > 1 && !(h->prm.max_levels > 0 && done[i] >= h->prm.max_levels)) {
        const int64_t root_cap = std::min<int64_t>(h->prm.root_cap > 0 ? h->prm.root_cap : 40000, mem_cap);
        int64_t Scur = 0, Snext = 0;
        int nmax = 0;
        for (auto& b : h->lv[l].box) {
          Scur += b.n;
          Snext += b.k;
        }
        for (int p = 0; p < (1 << (l - 1)); ++p) {
          Box& P = h->lv[l - 1].box[p];
          Box& A = h->lv[l].box[2 * p];
          Box& B = h->lv[l].box[2 * p + 1];
          P.cr = A.Jr;
          P.cr.insert(P.cr.end(), B.Jr.begin(), B.Jr.end());
          P.cc = A.Jc;
          P.cc.insert(P.cc.end(), B.Jc.begin(), B.Jc.end());
          nmax = std::max(nmax, (int)P.cr.size());
        }
        // stop compressing when it no longer pays (high-frequency boxes keep most unknowns)
        // and the merged system fits the root (root_cap, and three quarters of the device
        // memory), or when the next level's boxes would be too large for one-CTA
        // column-pivoted QR
        bool stop = (Snext > 0.8 * (double)Scur && Snext <= root_cap) || nmax > 3072;
        if (!stop) next = l - 1;
      }
      level[i] = next;
    }
  }
  std::vector<wsbm_hss*> roots;
  if (!rc) {
    for (size_t i = 0; i < hs.size(); ++i) {
      wsbm_hss* h = hs[i];
      if (h->L > 0 && !partial[i]) {
        const int root_cap = h->prm.root_cap > 0 ? h->prm.root_cap : 40000;
        int64_t S = 0;
        for (auto& b : h->lv[h->top].box) S += b.k;
        if (S > root_cap) rc = WSBM_ERR_RANK_OVERFLOW;
      }
      if (!partial[i]) roots.push_back(h);
    }
  }
  double mr2[2] = {0, 0};
  if (!rc && !roots.empty()) rc = factor_roots(roots, mr2);
  cudaEventRecord(t1, h0->st);
  cudaEventSynchronize(t1);
  const double total = elapsed(t0, t1);
  const int64_t launches = wsbm_launch_count() - launches0;
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  for (size_t i = 0; i < hs.size(); ++i) {
    wsbm_hss* h = hs[i];
    if (rc) {
      int32_t keep[32];
      memcpy(keep, h->stats.rank_per_level, sizeof(keep));
      release_factors(h);
      memcpy(h->stats.rank_per_level, keep, sizeof(keep));  // kept for diagnosis
      continue;
    }
    // a single curve owns the shared launches; in a batch they are reported by the batch
    if (hs.size() == 1) {
      h->stats.ms_entries = ms[0] + mr2[0];
      h->stats.ms_pairs = ms[1] + mr2[0];
      h->stats.ms_proxy = ms[0] - ms[1];
      h->stats.ms_id = ms[2];
      h->stats.ms_factor = ms[3] + mr2[1];
      h->stats.ms_total_factor = total;
      h->stats.launches = launches;
      h->stats.ms_cpqr = ms[4];
      h->stats.cpqr_matrices = cpqr_mats;
      h->stats.cpqr_flops = cpqr_flops;
      h->stats.sketch_matrices = sketch_cnt[0];
      h->stats.sketch_fallbacks = sketch_cnt[1];
      h->stats.ms_sketch = ms_sketch;
      h->stats.ms_lu = lu_acc[0];
      h->stats.lu_flops = lu_acc[1];
      h->stats.lu_matrices = (int64_t)lu_acc[2];
      h->stats.lu_tc_matrices = (int64_t)lu_acc[3];
    }
    size_t bytes = 0;
    for (int l = h->top; l <= h->L && h->L > 0; ++l)
      for (auto& b : h->lv[l].box)
        bytes += ((size_t)b.n * b.n + (size_t)b.n * b.k + (size_t)b.k * b.k + (size_t)b.k * (b.n - b.k)) *
                 sizeof(double2);
    bytes += (size_t)h->root_n * h->root_n * sizeof(double2);
    h->stats.factor_bytes = (int64_t)bytes;
    h->factored = !partial[i];
  }
  if (bstats) {
    memset(bstats, 0, sizeof(*bstats));
    for (auto* h : hs) {
      bstats->entries_generated += h->stats.entries_generated;
      bstats->entries_pairs += h->stats.entries_pairs;
      bstats->entries_proxy += h->stats.entries_proxy;
      bstats->max_rank = std::max(bstats->max_rank, h->stats.max_rank);
      bstats->root_size = std::max(bstats->root_size, h->stats.root_size);
      bstats->factor_bytes += h->stats.factor_bytes;
      bstats->levels = std::max(bstats->levels, h->stats.levels);
      bstats->nboxes_leaf += h->stats.nboxes_leaf;
    }
    bstats->ms_entries = ms[0] + mr2[0];
    bstats->ms_pairs = ms[1] + mr2[0];
    bstats->ms_proxy = ms[0] - ms[1];
    bstats->ms_id = ms[2];
    bstats->ms_factor = ms[3] + mr2[1];
    bstats->ms_total_factor = total;
    bstats->launches = launches;
    bstats->ms_cpqr = ms[4];
    bstats->cpqr_matrices = cpqr_mats;
    bstats->cpqr_flops = cpqr_flops;
    bstats->sketch_matrices = sketch_cnt[0];
    bstats->sketch_fallbacks = sketch_cnt[1];
    bstats->ms_sketch = ms_sketch;
    bstats->ms_lu = lu_acc[0];
    bstats->lu_flops = lu_acc[1];
    bstats->lu_matrices = (int64_t)lu_acc[2];
    bstats->lu_tc_matrices = (int64_t)lu_acc[3];
  }
  return rc;
}

extern "C" int wsbm_factor(wsbm_hss_t h) {
  if (!h) return WSBM_ERR_INVALID_ARG;
  std::vector<wsbm_hss*> hs(1, h);
  return factor_all(hs, nullptr);
}

// ------------------------------------------------------------------------ batches ----
struct wsbm_batch {
  std::vector<wsbm_hss*> hs;
  wsbm_stats_t stats;
  std::shared_ptr<struct SolvePlan> plan;
};

extern "C" int wsbm_batch_create(const wsbm_geom* g, const wsbm_params* p, int32_t count,
                                 void* stream, wsbm_batch_t* out) {
  if (!out || !g || !p || count < 1) return WSBM_ERR_INVALID_ARG;
  *out = nullptr;
  for (int i = 1; i < count; ++i)  // one launch per phase serves every curve: one formulation
    if (p[i].formulation != p[0].formulation) return WSBM_ERR_INVALID_ARG;
  wsbm_batch* b = new wsbm_batch();
  memset(&b->stats, 0, sizeof(b->stats));
  for (int i = 0; i < count; ++i) {
    wsbm_hss_t h = nullptr;
    int rc = wsbm_create(&g[i], &p[i], stream, &h);
    if (rc) {
      wsbm_batch_destroy(b);
      return rc;
    }
    b->hs.push_back(h);
  }
  *out = b;
  return WSBM_OK;
}

extern "C" int wsbm_batch_factor(wsbm_batch_t b) {
  if (!b || b->hs.empty()) return WSBM_ERR_INVALID_ARG;
  b->plan.reset();
  return factor_all(b->hs, &b->stats);
}

extern "C" int wsbm_batch_handle(wsbm_batch_t b, int32_t i, wsbm_hss_t* out) {
  if (!b || !out || i < 0 || i >= (int32_t)b->hs.size()) return WSBM_ERR_INVALID_ARG;
  *out = b->hs[i];
  return WSBM_OK;
}

extern "C" int wsbm_batch_stats(wsbm_batch_t b, wsbm_stats_t* s) {
  if (!b || !s) return WSBM_ERR_INVALID_ARG;
  *s = b->stats;
  return WSBM_OK;
}

extern "C" void wsbm_batch_destroy(wsbm_batch_t b) {
  if (!b) return;
  b->plan.reset();
  for (auto* h : b->hs) wsbm_destroy(h);
  delete b;
}

// ----------------------------------------------------------------------- solve ----
// Batched layout conversions (one CTA row per handle).
struct ConvDesc {
  const double2* in;
  double2 *out, *out2;
  int64_t N;
};
__global__ void k_to_interleaved_batched(const ConvDesc* __restrict__ d, int nrhs) {
  const ConvDesc c = d[blockIdx.y];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < 2 * c.N * nrhs;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = e % (2 * c.N), col = e / (2 * c.N);
    int64_t node = r % c.N, comp = r / c.N;
    c.out[2 * node + comp + col * 2 * c.N] = c.in[e];
  }
}
__global__ void k_split_uq_batched(const ConvDesc* __restrict__ d, int nrhs) {
  const ConvDesc c = d[blockIdx.y];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < c.N * nrhs;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e % c.N, col = e / c.N;
    c.out[e] = c.in[2 * i + col * 2 * c.N];
    c.out2[e] = c.in[2 * i + 1 + col * 2 * c.N];
  }
}

// A solve plan: for a set of factored handles (one stream) and a number of right-hand sides,
// every work buffer and descriptor array of the Martinsson-Rokhlin solve is allocated and
// uploaded once, and the launches are recorded as a list of operations:
//   up sweep    xh = D^-1 b, g = xh[pc], r = g[0:k] + Tc g[k:n], bt = Dhat r
//   roots       dense LU solves of the merged skeleton systems (one batched launch)
//   down sweep  x = xh - Z (bt - Dhat y)
// Tree levels of different handles are aligned at their leaves (as in the batched factor), so
// each phase of a tree step is one launch over every box of every handle.  On its first run the
// list is captured into a CUDA graph; later runs replay the graph.  Right-hand sides enter and
// solutions leave through the plan's own buffers (rin, uo, qo).
struct SolvePlan {
  std::vector<wsbm_hss*> hs;
  std::vector<uint64_t> gen;  // factor generation of each handle when the plan was built
  WsbmAllocator alloc;        // the first handle's allocator (buffers and descriptors)
  int nrhs = 0;
  cudaStream_t st = nullptr;  // the handles' stream (buffers are allocated in its order)
  cudaStream_t cs = nullptr;  // the plan's own stream: capture and replay (a graph cannot be
                              // captured on the legacy default stream)
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  std::vector<void*> mem;
  std::vector<double2*> rin, uo, qo;
  std::vector<std::function<int(cudaStream_t)>> ops;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t launches = 0;
  bool graph_ok = true;
  void* tcws = nullptr;  // work space of the tensor-core products (shared by their operations)
  size_t tcws_bytes = 0;
  bool uses_tc = false;
  ~SolvePlan() {
    if (cs) cudaStreamSynchronize(cs);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    for (void* p : mem) wsbm_dev_free(alloc, p, st);
    cudaStreamSynchronize(st);
    if (ev_in) cudaEventDestroy(ev_in);
    if (ev_out) cudaEventDestroy(ev_out);
    if (cs) cudaStreamDestroy(cs);
  }
};

template <class T>
static int plan_upload(SolvePlan& P, const std::vector<T>& v, T** d) {
  *d = nullptr;
  if (v.empty()) return WSBM_OK;
  HK(wsbm_dev_alloc(P.alloc, v.size() * sizeof(T), P.st, (void**)d));
  P.mem.push_back(*d);
  if (cudaMemcpyAsync(*d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, P.st) != cudaSuccess)
    return WSBM_ERR_CUDA;
  return WSBM_OK;
}
static int plan_alloc(SolvePlan& P, size_t bytes, double2** p) {
  HK(wsbm_dev_alloc(P.alloc, bytes, P.st, (void**)p));
  P.mem.push_back(*p);
  return WSBM_OK;
}

static int plan_copies(SolvePlan& P, const std::vector<CopyDesc>& c) {
  if (c.empty()) return WSBM_OK;
  CopyDesc* d = nullptr;
  HK(plan_upload(P, c, &d));
  int64_t mx = 0;
  for (auto& x : c) mx = std::max(mx, (int64_t)x.m * x.n);
  const unsigned nb = (unsigned)c.size();
  P.ops.push_back([d, mx, nb](cudaStream_t st) {
    launch_y(k_copy2d, gridfor(mx), nb, d, st);
    return WSBM_OK;
  });
  return WSBM_OK;
}
static int plan_gemms(SolvePlan& P, const std::vector<GemmDesc>& g) {
  if (g.empty()) return WSBM_OK;
  GemmDesc* d = nullptr;
  HK(plan_upload(P, g, &d));
  int mm = 0, mn = 0;
  for (auto& x : g) {
    mm = std::max(mm, x.m);
    mn = std::max(mn, x.n);
  }
  const int nb = (int)g.size();
  P.ops.push_back([d, nb, mm, mn](cudaStream_t st) { return wsbm_gemm_batched(d, nb, mm, mn, st); });
  return WSBM_OK;
}
static int plan_lu_solves(SolvePlan& P, const std::vector<TrsmDesc>& t) {
  if (t.empty()) return WSBM_OK;
  TrsmDesc* d = nullptr;
  HK(plan_upload(P, t, &d));
  int mn = 0, mr = 0;
  for (auto& x : t) {
    mn = std::max(mn, x.n);
    mr = std::max(mr, x.nrhs);
  }
  const int nb = (int)t.size();
  P.ops.push_back([d, nb, mn, mr](cudaStream_t st) { return wsbm_lu_solve_batched(d, d, nb, mn, mr, st); });
  return WSBM_OK;
}
static int plan_gathers(SolvePlan& P, const std::vector<GatherDesc>& g) {
  if (g.empty()) return WSBM_OK;
  GatherDesc* d = nullptr;
  HK(plan_upload(P, g, &d));
  int64_t mx = 0;
  for (auto& x : g) mx = std::max(mx, (int64_t)x.n * x.ncol);
  const unsigned nb = (unsigned)g.size();
  P.ops.push_back([d, mx, nb](cudaStream_t st) {
    launch_y(k_gather_rows, gridfor(mx), nb, d, st);
    return WSBM_OK;
  });
  return WSBM_OK;
}
// One launch sequence of the tensor-core product over `items` (C = beta C + alpha A B each; C
// may be B itself: B's digit planes are formed before C is written): the item tables are built
// and uploaded now; the work space is shared by every such operation of the plan and allocated
// once all are known (plan_tc_finish).
static int plan_tc(SolvePlan& P, const std::vector<TcProduct>& items, double2 alpha, double2 beta) {
  // launches of at most 65535 items whose digit planes take at most WSBM_TCSOLVE_WS bytes (one
  // item always forms a launch): the shared work space stays small next to the factors
  for (size_t c0 = 0; c0 < items.size();) {
    int n = (int)std::min<size_t>(65535, items.size() - c0);
    while (n > 1 && wsbm_zgemm_tc_batched_ws_bytes(items.data() + c0, n) > WSBM_TCSOLVE_WS) n = (n + 1) / 2;
    auto pl = std::make_shared<TcPlan>();
    const size_t i0 = c0;
    c0 += n;
    if (wsbm_zgemm_tc_plan(items.data() + i0, n, pl.get())) return WSBM_ERR_INVALID_ARG;
    if (pl->tiles == 0) continue;
    unsigned char* dtab = nullptr;
    HK(plan_upload(P, pl->tab, &dtab));
    P.tcws_bytes = std::max(P.tcws_bytes, pl->ws_bytes);
    P.uses_tc = true;
    const int group = wsbm_tune_current().tc_group;
    SolvePlan* pp = &P;
    P.ops.push_back([pl, dtab, alpha, beta, pp, group](cudaStream_t st) {
      return wsbm_zgemm_tc_run(*pl, dtab, alpha, beta, pp->tcws, st, group) ? WSBM_ERR_CUDA : WSBM_OK;
    });
  }
  return WSBM_OK;
}
static int plan_tc_finish(SolvePlan& P) {
  if (!P.tcws_bytes) return WSBM_OK;
  HK(wsbm_dev_alloc(P.alloc, P.tcws_bytes, P.st, &P.tcws));
  P.mem.push_back(P.tcws);
  return WSBM_OK;
}
static TcProduct tc_item(const double2* A, int64_t lda, const double2* B, int64_t ldb, double2* C, int64_t ldc,
                         int m, int n, int k) {
  TcProduct t;
  t.A = A;
  t.lda = lda;
  t.B = B;
  t.ldb = ldb;
  t.C = C;
  t.ldc = ldc;
  t.m = m;
  t.n = n;
  t.k = k;
  t.pad = 0;
  return t;
}

// LU solves A x = y with many right-hand sides on the tensor cores, batched over matrices of
// different orders (box factors D of a tree step, dense roots).  Item: t.T = LU of A (t.n x t.n,
// leading dimension t.ldt), t.piv its row interchanges, y = t.B (leading dimension t.ldb, the
// plan's nrhs columns), overwritten by x.  Blocked by nb = min(n, WSBM_TCSOLVE_NB) rows: y is
// permuted into a working copy W; then, panel by panel, W_p <- L_pp^-1 W_p and
// W_below -= L_below,p W_p (forward), W_p <- U_pp^-1 W_p and W_above -= U_above,p W_p
// (backward), with the inverses of the diagonal blocks and the permutation formed once per plan
// and every product on the tensor cores (one launch sequence per panel step over all items);
// W is copied back to y.
static int plan_lu_tc(SolvePlan& P, const std::vector<TrsmDesc>& items) {
  if (items.empty()) return WSBM_OK;
  const int nrhs = P.nrhs;
  const double2 one = make_double2(1.0, 0.0), zero = make_double2(0.0, 0.0), mone = make_double2(-1.0, 0.0);
  struct R {
    const double2* LU;
    int64_t ld;
    int n, nb, np;
    double2 *Li, *Ui, *W;
  };
  size_t tot_inv = 0, tot_w = 0, tot_perm = 0;
  for (const TrsmDesc& t : items) {
    const int nb = std::min(t.n, WSBM_TCSOLVE_NB), np = (t.n + nb - 1) / nb;
    tot_inv += (size_t)np * nb * nb;
    tot_w += (size_t)t.n * nrhs;
    tot_perm += ((size_t)t.n + 63) / 64 * 64;
  }
  // one allocation per kind: inverses, working copies, permutations
  double2 *Li, *Ui, *W;
  int32_t* perm;
  HK(plan_alloc(P, tot_inv * sizeof(double2), &Li));
  HK(plan_alloc(P, tot_inv * sizeof(double2), &Ui));
  HK(plan_alloc(P, tot_w * sizeof(double2), &W));
  HK(wsbm_dev_alloc(P.alloc, tot_perm * sizeof(int32_t), P.st, (void**)&perm));
  P.mem.push_back(perm);
  std::vector<R> rr;
  std::vector<DinvDesc> dd;
  std::vector<PermDesc> pd;
  std::vector<GatherDesc> g0;
  std::vector<CopyDesc> cfin;
  int maxp = 0, maxnb = 0;
  size_t oi = 0, ow = 0, op = 0;
  for (const TrsmDesc& t : items) {
    R r;
    r.LU = t.T;
    r.ld = t.ldt;
    r.n = t.n;
    r.nb = std::min(t.n, WSBM_TCSOLVE_NB);
    r.np = (t.n + r.nb - 1) / r.nb;
    r.Li = Li + oi;
    r.Ui = Ui + oi;
    r.W = W + ow;
    oi += (size_t)r.np * r.nb * r.nb;
    ow += (size_t)t.n * nrhs;
    int32_t* pm = perm + op;
    op += ((size_t)t.n + 63) / 64 * 64;
    dd.push_back({t.T, t.ldt, r.Li, r.Ui, t.n, r.nb});
    pd.push_back({t.piv, pm, t.n, 0});
    g0.push_back({r.W, t.B, pm, t.n, t.ldb, t.n, nrhs});
    cfin.push_back({t.B, r.W, t.ldb, t.n, t.n, nrhs});
    maxp = std::max(maxp, r.np);
    maxnb = std::max(maxnb, r.nb);
    rr.push_back(r);
  }
  // inverses of the diagonal blocks and the permutations: once, now (not recorded operations)
  {
    DinvDesc* d = nullptr;
    PermDesc* q = nullptr;
    HK(plan_upload(P, dd, &d));
    HK(plan_upload(P, pd, &q));
    if (wsbm_lu_dinv_batched(d, (int)dd.size(), maxp, maxnb, P.st)) return WSBM_ERR_CUDA;
    if (wsbm_piv_perm_batched(q, (int)pd.size(), P.st)) return WSBM_ERR_CUDA;
  }
  HK(plan_gathers(P, g0));
  std::vector<TcProduct> i1, i2;
  for (int q = 0; q < maxp; ++q) {  // forward: unit lower L
    i1.clear();
    i2.clear();
    for (const R& r : rr) {
      if (q >= r.np) continue;
      const int j0 = q * r.nb, jb = std::min(r.nb, r.n - j0), je = j0 + jb;
      i1.push_back(tc_item(r.Li + (int64_t)q * r.nb * r.nb, r.nb, r.W + j0, r.n, r.W + j0, r.n, jb, nrhs, jb));
      if (je < r.n)
        i2.push_back(tc_item(r.LU + je + (int64_t)j0 * r.ld, r.ld, r.W + j0, r.n, r.W + je, r.n, r.n - je, nrhs, jb));
    }
    HK(plan_tc(P, i1, one, zero));
    HK(plan_tc(P, i2, mone, one));
  }
  for (int q = 0; q < maxp; ++q) {  // backward: U, from each matrix's last panel
    i1.clear();
    i2.clear();
    for (const R& r : rr) {
      const int p = r.np - 1 - q;
      if (p < 0) continue;
      const int j0 = p * r.nb, jb = std::min(r.nb, r.n - j0);
      i1.push_back(tc_item(r.Ui + (int64_t)p * r.nb * r.nb, r.nb, r.W + j0, r.n, r.W + j0, r.n, jb, nrhs, jb));
      if (j0 > 0) i2.push_back(tc_item(r.LU + (int64_t)j0 * r.ld, r.ld, r.W + j0, r.n, r.W, r.n, j0, nrhs, jb));
    }
    HK(plan_tc(P, i1, one, zero));
    HK(plan_tc(P, i2, mone, one));
  }
  return plan_copies(P, cfin);
}

// LU solves of a plan step: with min_rhs or more right-hand sides, the matrices of at least
// min_n unknowns on the tensor cores (plan_lu_tc), the rest as FP64 triangular solves.
static int plan_lu_solves_auto(SolvePlan& P, const std::vector<TrsmDesc>& t, int min_n, int min_rhs) {
  if (P.nrhs < min_rhs) return plan_lu_solves(P, t);
  std::vector<TrsmDesc> tc, fp;
  for (const TrsmDesc& x : t) (x.n >= min_n ? tc : fp).push_back(x);
  HK(plan_lu_solves(P, fp));
  return plan_lu_tc(P, tc);
}

// Products of a plan step: on the tensor cores with WSBM_TCSOLVE_RHS or more right-hand sides
// (when the items share alpha and beta and none is transposed), else the FP64 kernel.
static int plan_gemms_auto(SolvePlan& P, const std::vector<GemmDesc>& g) {
  if (g.empty()) return WSBM_OK;
  bool tc = P.nrhs >= WSBM_TCSOLVE_RHS;
  for (const GemmDesc& x : g)
    if (x.ta || x.alpha.x != g[0].alpha.x || x.alpha.y != g[0].alpha.y || x.beta.x != g[0].beta.x ||
        x.beta.y != g[0].beta.y || x.k > 32768)
      tc = false;
  if (!tc) return plan_gemms(P, g);
  std::vector<TcProduct> it;
  it.reserve(g.size());
  for (const GemmDesc& x : g)
    if (x.m > 0 && x.n > 0 && x.k > 0) it.push_back(tc_item(x.A, x.lda, x.B, x.ldb, x.C, x.ldc, x.m, x.n, x.k));
  return plan_tc(P, it, g[0].alpha, g[0].beta);
}

static TrsmDesc lu_desc(const double2* T, int64_t ldt, double2* B, int64_t ldb, const int32_t* piv,
                        int n, int nrhs) {
  TrsmDesc t;
  memset(&t, 0, sizeof(t));
  t.T = T;
  t.ldt = ldt;
  t.B = B;
  t.ldb = ldb;
  t.piv = piv;
  t.n = n;
  t.nrhs = nrhs;
  return t;
}
static GemmDesc gemm_n(const double2* A, int64_t lda, const double2* B, int64_t ldb, double2* C,
                       int64_t ldc, int m, int n, int k, double alpha, double beta) {
  GemmDesc g;
  memset(&g, 0, sizeof(g));
  g.A = A;
  g.lda = lda;
  g.B = B;
  g.ldb = ldb;
  g.C = C;
  g.ldc = ldc;
  g.m = m;
  g.n = n;
  g.k = k;
  g.alpha = make_double2(alpha, 0.0);
  g.beta = make_double2(beta, 0.0);
  return g;
}

static int plan_build(SolvePlan& P) {
  const int nrhs = P.nrhs;
  const size_t NH = P.hs.size();
  P.rin.resize(NH);
  P.uo.resize(NH);
  P.qo.resize(NH);
  std::vector<double2*> bint(NH);
  // per handle, per level: xh (n x nrhs), g (n x nrhs), bt (k x nrhs), r / t (k x nrhs)
  std::vector<std::vector<std::vector<double2*>>> XH(NH), G(NH), BT(NH), RT(NH);
  std::vector<double2*> Y(NH, nullptr);
  int T = 0;
  for (size_t i = 0; i < NH; ++i) {
    wsbm_hss* h = P.hs[i];
    const int64_t N = h->N;
    HK(plan_alloc(P, (size_t)2 * N * nrhs * sizeof(double2), &P.rin[i]));
    HK(plan_alloc(P, (size_t)N * nrhs * sizeof(double2), &P.uo[i]));
    HK(plan_alloc(P, (size_t)N * nrhs * sizeof(double2), &P.qo[i]));
    HK(plan_alloc(P, (size_t)2 * N * nrhs * sizeof(double2), &bint[i]));
    if (h->L == 0) continue;
    T = std::max(T, h->L - h->top + 1);
    XH[i].resize(h->L + 1);
    G[i].resize(h->L + 1);
    BT[i].resize(h->L + 1);
    RT[i].resize(h->L + 1);
    for (int l = h->L; l >= h->top; --l) {
      Level& LV = h->lv[l];
      size_t tn = 0, tk = 0;
      for (auto& b : LV.box) {
        tn += b.n;
        tk += b.k;
      }
      double2 *xh, *g, *bt, *rt;
      HK(plan_alloc(P, tn * nrhs * sizeof(double2), &xh));
      HK(plan_alloc(P, tn * nrhs * sizeof(double2), &g));
      HK(plan_alloc(P, tk * nrhs * sizeof(double2), &bt));
      HK(plan_alloc(P, tk * nrhs * sizeof(double2), &rt));
      size_t on = 0, ok = 0;
      for (auto& b : LV.box) {
        XH[i][l].push_back(xh + on * nrhs);
        G[i][l].push_back(g + on * nrhs);
        BT[i][l].push_back(bt + ok * nrhs);
        RT[i][l].push_back(rt + ok * nrhs);
        on += b.n;
        ok += b.k;
      }
    }
    HK(plan_alloc(P, (size_t)h->root_n * nrhs * sizeof(double2), &Y[i]));
  }
  // paper order -> interleaved
  {
    std::vector<ConvDesc> cv;
    int64_t mx = 0;
    for (size_t i = 0; i < NH; ++i) {
      cv.push_back({P.rin[i], bint[i], nullptr, P.hs[i]->N});
      mx = std::max(mx, 2 * P.hs[i]->N * nrhs);
    }
    ConvDesc* d = nullptr;
    HK(plan_upload(P, cv, &d));
    const unsigned nb = (unsigned)cv.size();
    P.ops.push_back([d, mx, nb, nrhs](cudaStream_t st) {
      launch_y(k_to_interleaved_batched, gridfor(mx), nb, d, st, nrhs);
      return WSBM_OK;
    });
  }
  // ---- up sweep, tree step t = 0 at the leaves of every handle
  for (int t = 0; t < T; ++t) {
    std::vector<CopyDesc> c1, rc0;
    std::vector<TrsmDesc> sd;
    std::vector<GatherDesc> gd;
    std::vector<GemmDesc> g1, g2;
    for (size_t i = 0; i < NH; ++i) {
      wsbm_hss* h = P.hs[i];
      if (h->L == 0) continue;
      const int l = h->L - t;
      if (l < h->top) continue;
      Level& LV = h->lv[l];
      for (int b = 0; b < (int)LV.box.size(); ++b) {
        Box& B = LV.box[b];
        double2* xh = XH[i][l][b];
        if (l == h->L) {
          c1.push_back({xh, bint[i] + 2 * B.lo, B.n, 2 * h->N, B.n, nrhs});
        } else {
          Box& A1 = h->lv[l + 1].box[2 * b];
          Box& A2 = h->lv[l + 1].box[2 * b + 1];
          c1.push_back({xh, BT[i][l + 1][2 * b], B.n, A1.k, A1.k, nrhs});
          c1.push_back({xh + A1.k, BT[i][l + 1][2 * b + 1], B.n, A2.k, A2.k, nrhs});
        }
        sd.push_back(lu_desc(B.D, B.n, xh, B.n, B.piv, B.n, nrhs));
        double2* gb = G[i][l][b];
        double2* rb = RT[i][l][b];
        gd.push_back({gb, xh, B.pc, B.n, B.n, B.n, nrhs});
        rc0.push_back({rb, gb, B.k, B.n, B.k, nrhs});
        if (B.n > B.k) g1.push_back(gemm_n(B.Tc, B.k, gb + B.k, B.n, rb, B.k, B.k, nrhs, B.n - B.k, 1.0, 1.0));
        g2.push_back(gemm_n(B.Dc, B.k, rb, B.k, BT[i][l][b], B.k, B.k, nrhs, B.k, 1.0, 0.0));
      }
    }
    HK(plan_copies(P, c1));
    HK(plan_lu_solves_auto(P, sd, WSBM_LU_TC_MIN, WSBM_TCSOLVE_RHS));
    HK(plan_gathers(P, gd));
    HK(plan_copies(P, rc0));
    HK(plan_gemms_auto(P, g1));
    HK(plan_gemms_auto(P, g2));
  }
  // ---- roots
  {
    std::vector<CopyDesc> c;
    std::vector<TrsmDesc> rs;
    for (size_t i = 0; i < NH; ++i) {
      wsbm_hss* h = P.hs[i];
      if (h->L == 0) {
        rs.push_back(lu_desc(h->root, h->root_n, bint[i], 2 * h->N, h->root_piv, h->root_n, nrhs));
        continue;
      }
      Level& TL = h->lv[h->top];
      int off = 0;
      for (int b = 0; b < (int)TL.box.size(); ++b) {
        c.push_back({Y[i] + off, BT[i][h->top][b], h->root_n, TL.box[b].k, TL.box[b].k, nrhs});
        off += TL.box[b].k;
      }
      rs.push_back(lu_desc(h->root, h->root_n, Y[i], h->root_n, h->root_piv, h->root_n, nrhs));
    }
    HK(plan_copies(P, c));
    HK(plan_lu_solves_auto(P, rs, wsbm_tune_current().solve_tc_min, WSBM_TCSOLVE_RHS_ROOT));
  }
  // ---- down sweep: t = bt - Dhat y (in RT), xh -= Z t; y of a box = its slice of the parent's x
  for (int t = T - 1; t >= 0; --t) {
    std::vector<CopyDesc> cb;
    std::vector<GemmDesc> g1, g2;
    for (size_t i = 0; i < NH; ++i) {
      wsbm_hss* h = P.hs[i];
      if (h->L == 0) continue;
      const int l = h->L - t;
      if (l < h->top) continue;
      Level& LV = h->lv[l];
      int yoff = 0;
      for (int b = 0; b < (int)LV.box.size(); ++b) {
        Box& B = LV.box[b];
        const double2* yb;
        int64_t ldy;
        if (l == h->top) {
          yb = Y[i] + yoff;
          ldy = h->root_n;
          yoff += B.k;
        } else {
          Box& Pb = h->lv[l - 1].box[b / 2];
          yb = XH[i][l - 1][b / 2] + ((b % 2) ? LV.box[b - 1].k : 0);
          ldy = Pb.n;
        }
        double2* tt = RT[i][l][b];
        cb.push_back({tt, BT[i][l][b], B.k, B.k, B.k, nrhs});
        g1.push_back(gemm_n(B.Dc, B.k, yb, ldy, tt, B.k, B.k, nrhs, B.k, -1.0, 1.0));
        g2.push_back(gemm_n(B.Z, B.n, tt, B.k, XH[i][l][b], B.n, B.n, nrhs, B.k, -1.0, 1.0));
      }
    }
    HK(plan_copies(P, cb));
    HK(plan_gemms_auto(P, g1));
    HK(plan_gemms_auto(P, g2));
  }
  // ---- leaves back to the interleaved vector, then u, q
  {
    std::vector<CopyDesc> c;
    std::vector<ConvDesc> cv;
    int64_t mx = 0;
    for (size_t i = 0; i < NH; ++i) {
      wsbm_hss* h = P.hs[i];
      if (h->L > 0) {
        Level& LV = h->lv[h->L];
        for (int b = 0; b < (int)LV.box.size(); ++b)
          c.push_back({bint[i] + 2 * LV.box[b].lo, XH[i][h->L][b], 2 * h->N, LV.box[b].n, LV.box[b].n, nrhs});
      }
      cv.push_back({bint[i], P.uo[i], P.qo[i], h->N});
      mx = std::max(mx, h->N * nrhs);
    }
    HK(plan_copies(P, c));
    ConvDesc* d = nullptr;
    HK(plan_upload(P, cv, &d));
    const unsigned nb = (unsigned)cv.size();
    P.ops.push_back([d, mx, nb, nrhs](cudaStream_t st) {
      launch_y(k_split_uq_batched, gridfor(mx), nb, d, st, nrhs);
      return WSBM_OK;
    });
  }
  HK(plan_tc_finish(P));
  return cudaGetLastError() == cudaSuccess ? WSBM_OK : WSBM_ERR_CUDA;
}

static int plan_exec(SolvePlan& P) {
  cudaStream_t st = P.cs;
  if (P.graph_ok && !P.exec) {
    const int64_t c0 = wsbm_launch_count();
    bool ok = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    int rc = WSBM_OK;
    if (ok)
      for (auto& op : P.ops)
        if ((rc = op(st)) != WSBM_OK) break;
    cudaGraph_t g = nullptr;
    if (ok) ok = cudaStreamEndCapture(st, &g) == cudaSuccess && rc == WSBM_OK && g != nullptr;
    if (ok) ok = cudaGraphInstantiate(&P.exec, g, 0) == cudaSuccess;
    P.launches = wsbm_launch_count() - c0;
    if (ok) {
      P.graph = g;
    } else {
      if (g) cudaGraphDestroy(g);
      P.exec = nullptr;
      P.graph_ok = false;
      cudaGetLastError();  // clear a capture error; run the operations directly instead
    }
    wsbm_count_launches(-P.launches);  // counted again when they run
  }
  if (P.exec) {
    HC(cudaGraphLaunch(P.exec, st));
    wsbm_count_launches(P.launches);
    return WSBM_OK;
  }
  for (auto& op : P.ops) HK(op(st));
  return cudaGetLastError() == cudaSuccess ? WSBM_OK : WSBM_ERR_CUDA;
}

// Run the plan on its own stream, ordered after everything already queued on the handles'
// stream and before anything queued there later: capture its operations into a CUDA graph on
// the first run, replay the graph after (or run the operations directly if capture failed).
static int plan_run(SolvePlan& P) {
  HC(cudaEventRecord(P.ev_in, P.st));
  HC(cudaStreamWaitEvent(P.cs, P.ev_in, 0));
  HK(plan_exec(P));
  HC(cudaEventRecord(P.ev_out, P.cs));
  HC(cudaStreamWaitEvent(P.st, P.ev_out, 0));
  return WSBM_OK;
}

// A plan holds device pointers into its handles' factors, so it is reused only while every
// handle still has the factors it was built from (a member of a batch may have been
// re-factored on its own since).
static int plan_get(std::shared_ptr<SolvePlan>& slot, const std::vector<wsbm_hss*>& hs, int nrhs) {
  std::vector<uint64_t> gen(hs.size());
  for (size_t i = 0; i < hs.size(); ++i) gen[i] = hs[i]->generation;
  if (slot && slot->nrhs == nrhs && slot->hs == hs && slot->gen == gen) return WSBM_OK;
  slot.reset();
  auto P = std::make_shared<SolvePlan>();
  P->hs = hs;
  P->gen = gen;
  P->alloc = hs[0]->alloc;
  P->nrhs = nrhs;
  P->st = hs[0]->st;
  if (cudaStreamCreateWithFlags(&P->cs, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&P->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&P->ev_out, cudaEventDisableTiming) != cudaSuccess)
    return WSBM_ERR_CUDA;
  int rc = plan_build(*P);
  if (rc != WSBM_OK) return rc;
  slot = P;
  return WSBM_OK;
}

// Solves of several handles (paper-order right-hand sides in, u and q out) with one plan.
static int solve_set(std::shared_ptr<SolvePlan>& slot, const std::vector<wsbm_hss*>& hs,
                     const void* const* rhs, int32_t nrhs, void* const* u, void* const* q) {
  HK(plan_get(slot, hs, nrhs));
  SolvePlan& P = *slot;
  cudaStream_t st = P.st;
  for (size_t i = 0; i < hs.size(); ++i)
    HC(cudaMemcpyAsync(P.rin[i], rhs[i], (size_t)2 * hs[i]->N * nrhs * sizeof(double2),
                       cudaMemcpyDeviceToDevice, st));
  HK(plan_run(P));
  for (size_t i = 0; i < hs.size(); ++i) {
    const size_t bytes = (size_t)hs[i]->N * nrhs * sizeof(double2);
    HC(cudaMemcpyAsync(u[i], P.uo[i], bytes, cudaMemcpyDeviceToDevice, st));
    HC(cudaMemcpyAsync(q[i], P.qo[i], bytes, cudaMemcpyDeviceToDevice, st));
  }
  HC(cudaStreamSynchronize(st));
  if (P.uses_tc) {  // a bounded wait of the tensor-core kernel that ran out
    const int t = wsbm_zgemm_tc_status(st);
    if (t == -5) return WSBM_ERR_TIMEOUT;
    if (t) return WSBM_ERR_CUDA;
  }
  return WSBM_OK;
}

extern "C" int wsbm_solve(wsbm_hss_t h, const void* rhs, int32_t nrhs, void* u, void* q) {
  if (!h) return WSBM_ERR_INVALID_ARG;
  if (!h->factored) return WSBM_ERR_NOT_FACTORED;
  if (nrhs < 0 || (nrhs > 0 && (!rhs || !u || !q))) return WSBM_ERR_INVALID_ARG;
  if (nrhs == 0) return WSBM_OK;
  std::vector<wsbm_hss*> hs(1, h);
  return solve_set(h->plan, hs, &rhs, nrhs, &u, &q);
}

extern "C" int wsbm_batch_solve(wsbm_batch_t b, const void* const* rhs, int32_t nrhs,
                                void* const* u, void* const* q) {
  if (!b || b->hs.empty()) return WSBM_ERR_INVALID_ARG;
  for (auto* h : b->hs)
    if (!h->factored) return WSBM_ERR_NOT_FACTORED;
  if (nrhs < 0 || (nrhs > 0 && (!rhs || !u || !q))) return WSBM_ERR_INVALID_ARG;
  if (nrhs == 0) return WSBM_OK;
  for (size_t i = 0; i < b->hs.size(); ++i)
    if (!rhs[i] || !u[i] || !q[i]) return WSBM_ERR_INVALID_ARG;
  return solve_set(b->plan, b->hs, rhs, nrhs, u, q);
}

// Transposed solve A^T lam = v with the same factors.  For A ~ D + L A~ R (per level) the
// transpose has the same form with L <-> R^T, so with Z = D^-1 L and Dhat = (R D^-1 L)^-1:
//   up    s = Z^T v (= L^T D^-T v),  bt = Dhat^T s;   root: transposed LU solve;
//   down  lam = D^-T (v - R^T (bt - Dhat^T y)),  R^T = Pi^T [I; Tc^T].
static GemmDesc gemm_t(const double2* A, int64_t lda, const double2* B, int64_t ldb, double2* C,
                       int64_t ldc, int m, int n, int k, double alpha, double beta) {
  GemmDesc g;
  memset(&g, 0, sizeof(g));
  g.A = A;
  g.lda = lda;
  g.B = B;
  g.ldb = ldb;
  g.C = C;
  g.ldc = ldc;
  g.m = m;
  g.n = n;
  g.k = k;
  g.ta = 1;
  g.alpha = make_double2(alpha, 0.0);
  g.beta = make_double2(beta, 0.0);
  return g;
}

static TrsmDesc lu_t(const double2* T, int64_t ldt, double2* B, int64_t ldb, const int32_t* piv,
                     int n, int nrhs) {
  TrsmDesc t;
  memset(&t, 0, sizeof(t));
  t.T = T;
  t.ldt = ldt;
  t.B = B;
  t.ldb = ldb;
  t.piv = piv;
  t.n = n;
  t.nrhs = nrhs;
  t.trans = 1;
  return t;
}

extern "C" int wsbm_solve_transposed(wsbm_hss_t h, const void* rhs, int32_t nrhs, void* lam1,
                                     void* lam2) {
  if (!h) return WSBM_ERR_INVALID_ARG;
  if (!h->factored) return WSBM_ERR_NOT_FACTORED;
  if (nrhs < 0 || (nrhs > 0 && (!rhs || !lam1 || !lam2))) return WSBM_ERR_INVALID_ARG;
  if (nrhs == 0) return WSBM_OK;
  cudaStream_t st = h->st;
  pin_reset(st);
  TmpMem tmpm(h);
  std::vector<void*>& tmp = tmpm.v;
  const int64_t N = h->N;
  double2* bint = nullptr;
  HK(dalloc(h, (size_t)2 * N * nrhs * sizeof(double2), (void**)&bint, tmp));
  k_to_interleaved<<<gridfor(2 * N * nrhs), 256, 0, st>>>((const double2*)rhs, bint, N, nrhs);
  wsbm_count_launch();
  if (h->L == 0) {
    std::vector<TrsmDesc> v(1, lu_t(h->root, h->root_n, bint, 2 * N, h->root_piv, h->root_n, nrhs));
    TrsmDesc* dt = nullptr;
    HK(upload(h, v, &dt, tmp));
    HK(wsbm_lu_solve_t_batched(dt, 1, h->root_n, nrhs, st));
    k_split_uq<<<gridfor(N * nrhs), 256, 0, st>>>(bint, (double2*)lam1, (double2*)lam2, N, nrhs);
    wsbm_count_launch();
    HC(cudaStreamSynchronize(st));
    free_list(h, tmp);
    return WSBM_OK;
  }
  const int L = h->L, top = h->top;
  std::vector<std::vector<double2*>> V(L + 1), BT(L + 1);
  int maxn = 0, maxk = 0;
  for (int l = L; l >= top; --l) {
    Level& LV = h->lv[l];
    int nb = (int)LV.box.size();
    V[l].resize(nb);
    BT[l].resize(nb);
    size_t tn = 0, tk = 0;
    for (auto& b : LV.box) {
      tn += b.n;
      tk += b.k;
      maxn = std::max(maxn, b.n);
      maxk = std::max(maxk, b.k);
    }
    double2 *v = nullptr, *bt = nullptr;
    HK(dalloc(h, tn * nrhs * sizeof(double2), (void**)&v, tmp));
    HK(dalloc(h, tk * nrhs * sizeof(double2), (void**)&bt, tmp));
    size_t on = 0, ok = 0;
    for (int b = 0; b < nb; ++b) {
      V[l][b] = v + on * nrhs;
      BT[l][b] = bt + ok * nrhs;
      on += LV.box[b].n;
      ok += LV.box[b].k;
    }
  }
  // ---- upward sweep: v = leaf rows or the children's bt;  s = Z^T v;  bt = Dhat^T s
  for (int l = L; l >= top; --l) {
    Level& LV = h->lv[l];
    int nb = (int)LV.box.size();
    std::vector<CopyDesc> c1;
    std::vector<GemmDesc> g1, g2;
    size_t tk = 0;
    int lk = 0;
    for (auto& b : LV.box) {
      tk += b.k;
      lk = std::max(lk, b.k);
    }
    double2* sbuf = nullptr;
    HK(dalloc(h, tk * nrhs * sizeof(double2), (void**)&sbuf, tmp));
    size_t ok = 0;
    for (int b = 0; b < nb; ++b) {
      Box& B = LV.box[b];
      if (l == L) {
        c1.push_back({V[l][b], bint + 2 * B.lo, B.n, 2 * N, B.n, nrhs});
      } else {
        Box& A1 = h->lv[l + 1].box[2 * b];
        Box& A2 = h->lv[l + 1].box[2 * b + 1];
        c1.push_back({V[l][b], BT[l + 1][2 * b], B.n, A1.k, A1.k, nrhs});
        c1.push_back({V[l][b] + A1.k, BT[l + 1][2 * b + 1], B.n, A2.k, A2.k, nrhs});
      }
      double2* sb = sbuf + ok * nrhs;
      ok += B.k;
      g1.push_back(gemm_t(B.Z, B.n, V[l][b], B.n, sb, B.k, B.k, nrhs, B.n, 1.0, 0.0));
      g2.push_back(gemm_t(B.Dc, B.k, sb, B.k, BT[l][b], B.k, B.k, nrhs, B.k, 1.0, 0.0));
    }
    CopyDesc* d1 = nullptr;
    GemmDesc *dg1 = nullptr, *dg2 = nullptr;
    HK(upload(h, c1, &d1, tmp));
    HK(upload(h, g1, &dg1, tmp));
    HK(upload(h, g2, &dg2, tmp));
    launch_y(k_copy2d, gridfor((int64_t)maxn * nrhs), (int64_t)c1.size(), d1, st);
    HK(wsbm_gemm_batched(dg1, nb, lk, nrhs, st));
    HK(wsbm_gemm_batched(dg2, nb, lk, nrhs, st));
  }
  // ---- root: transposed LU solve of the merged skeleton system
  double2* y = nullptr;
  HK(dalloc(h, (size_t)h->root_n * nrhs * sizeof(double2), (void**)&y, tmp));
  {
    Level& T = h->lv[top];
    std::vector<CopyDesc> c;
    int off = 0;
    for (int b = 0; b < (int)T.box.size(); ++b) {
      c.push_back({y + off, BT[top][b], h->root_n, T.box[b].k, T.box[b].k, nrhs});
      off += T.box[b].k;
    }
    CopyDesc* dc = nullptr;
    HK(upload(h, c, &dc, tmp));
    launch_y(k_copy2d, gridfor((int64_t)maxk * nrhs), (int64_t)c.size(), dc, st);
    std::vector<TrsmDesc> v(1, lu_t(h->root, h->root_n, y, h->root_n, h->root_piv, h->root_n, nrhs));
    TrsmDesc* dt = nullptr;
    HK(upload(h, v, &dt, tmp));
    HK(wsbm_lu_solve_t_batched(dt, 1, h->root_n, nrhs, st));
  }
  // ---- downward sweep: t = bt - Dhat^T y;  v -= R^T t;  lam = D^-T v  (in place in V)
  for (int l = top; l <= L; ++l) {
    Level& LV = h->lv[l];
    int nb = (int)LV.box.size();
    size_t tk = 0, tn = 0;
    int lk = 0, ln = 0, lr = 0;
    for (auto& b : LV.box) {
      tk += b.k;
      tn += b.n;
      lk = std::max(lk, b.k);
      ln = std::max(ln, b.n);
      lr = std::max(lr, b.n - b.k);
    }
    double2 *tb = nullptr, *ub = nullptr;
    HK(dalloc(h, tk * nrhs * sizeof(double2), (void**)&tb, tmp));
    HK(dalloc(h, tn * nrhs * sizeof(double2), (void**)&ub, tmp));
    std::vector<CopyDesc> cb, cu;
    std::vector<GemmDesc> g1, g2;
    std::vector<GatherDesc> sc;
    std::vector<TrsmDesc> sd;
    size_t ok = 0, on = 0;
    int yoff = 0;
    for (int b = 0; b < nb; ++b) {
      Box& B = LV.box[b];
      const double2* yb;
      int64_t ldy;
      if (l == top) {
        yb = y + yoff;
        ldy = h->root_n;
        yoff += B.k;
      } else {
        Box& P = h->lv[l - 1].box[b / 2];
        yb = V[l - 1][b / 2] + ((b % 2) ? h->lv[l].box[b - 1].k : 0);
        ldy = P.n;
      }
      double2* t = tb + ok * nrhs;
      double2* u = ub + on * nrhs;
      ok += B.k;
      on += B.n;
      cb.push_back({t, BT[l][b], B.k, B.k, B.k, nrhs});
      g1.push_back(gemm_t(B.Dc, B.k, yb, ldy, t, B.k, B.k, nrhs, B.k, -1.0, 1.0));
      cu.push_back({u, t, B.n, B.k, B.k, nrhs});
      if (B.n > B.k)
        g2.push_back(gemm_t(B.Tc, B.k, t, B.k, u + B.k, B.n, B.n - B.k, nrhs, B.k, 1.0, 0.0));
      sc.push_back({V[l][b], u, B.pc, B.n, B.n, B.n, nrhs});
      sd.push_back(lu_t(B.D, B.n, V[l][b], B.n, B.piv, B.n, nrhs));
    }
    CopyDesc *dcb = nullptr, *dcu = nullptr;
    GemmDesc *dg1 = nullptr, *dg2 = nullptr;
    GatherDesc* dsc = nullptr;
    TrsmDesc* dsd = nullptr;
    HK(upload(h, cb, &dcb, tmp));
    HK(upload(h, cu, &dcu, tmp));
    HK(upload(h, g1, &dg1, tmp));
    HK(upload(h, g2, &dg2, tmp));
    HK(upload(h, sc, &dsc, tmp));
    HK(upload(h, sd, &dsd, tmp));
    launch_y(k_copy2d, gridfor((int64_t)lk * nrhs), nb, dcb, st);
    HK(wsbm_gemm_batched(dg1, nb, lk, nrhs, st));
    launch_y(k_copy2d, gridfor((int64_t)lk * nrhs), nb, dcu, st);
    if (!g2.empty()) HK(wsbm_gemm_batched(dg2, (int)g2.size(), lr, nrhs, st));
    launch_y(k_scatter_sub_rows, gridfor((int64_t)ln * nrhs), nb, dsc, st);
    HK(wsbm_lu_solve_t_batched(dsd, nb, ln, nrhs, st));
  }
  {
    Level& LV = h->lv[L];
    std::vector<CopyDesc> c;
    for (int b = 0; b < (int)LV.box.size(); ++b) {
      Box& B = LV.box[b];
      c.push_back({bint + 2 * B.lo, V[L][b], 2 * N, B.n, B.n, nrhs});
    }
    CopyDesc* dc = nullptr;
    HK(upload(h, c, &dc, tmp));
    launch_y(k_copy2d, gridfor((int64_t)maxn * nrhs), (int64_t)c.size(), dc, st);
    k_split_uq<<<gridfor(N * nrhs), 256, 0, st>>>(bint, (double2*)lam1, (double2*)lam2, N, nrhs);
    wsbm_count_launch();
  }
  HC(cudaGetLastError());
  HC(cudaStreamSynchronize(st));
  free_list(h, tmp);
  return WSBM_OK;
}

extern "C" int wsbm_rhs_planewave(wsbm_hss_t h, const double* angles, int32_t nang, void* rhs) {
  if (!h || nang < 0 || (nang > 0 && (!angles || !rhs))) return WSBM_ERR_INVALID_ARG;
  if (nang == 0) return WSBM_OK;
  k_rhs_planewave<<<gridfor(h->N * nang), 256, 0, h->st>>>(h->g, h->ph.k0, angles, nang, (double2*)rhs,
                                                         h->prm.formulation, h->ph.eps0);
  wsbm_count_launch();
  return cudaGetLastError() == cudaSuccess ? WSBM_OK : WSBM_ERR_CUDA;
}

extern "C" int wsbm_farfield(wsbm_hss_t h, const void* u, const void* q, int32_t nrhs,
                             const double* angles, int32_t nang, void* out) {
  if (!h || nrhs < 0 || nang < 0) return WSBM_ERR_INVALID_ARG;
  if (nrhs == 0 || nang == 0) return WSBM_OK;
  if (!u || !q || !angles || !out) return WSBM_ERR_INVALID_ARG;
  k_farfield<<<nang, 256, 0, h->st>>>(h->g, h->ph.k0, h->ph.eps0, (const double2*)u, (const double2*)q, nrhs, angles, nang, (double2*)out);
  wsbm_count_launch();
  return cudaGetLastError() == cudaSuccess ? WSBM_OK : WSBM_ERR_CUDA;
}

extern "C" int wsbm_entries(wsbm_hss_t h, const int64_t* rows, int64_t nr, const int64_t* cols,
                            int64_t nc, void* out) {
  if (!h) return WSBM_ERR_INVALID_ARG;
  wsbm_geom g = {h->N, h->x, h->y, h->nx, h->ny, h->w, h->kappa};
  return wsbm_entries_raw(&g, &h->prm, rows, nr, cols, nc, out, h->st);
}

extern "C" int wsbm_box_info(wsbm_hss_t h, int32_t level, int32_t box, double* out4, int64_t* range2) {
  if (!h || level < 0 || level > h->L || box < 0 || box >= (1 << level) || !out4 || !range2)
    return WSBM_ERR_INVALID_ARG;
  const Box& b = h->lv[level].box[box];
  out4[0] = b.cx;
  out4[1] = b.cy;
  out4[2] = b.R;
  out4[3] = b.rho;
  range2[0] = b.lo;
  range2[1] = b.hi;
  return WSBM_OK;
}

extern "C" int wsbm_box_skeletons(wsbm_hss_t h, int32_t level, int32_t box, int64_t* jr,
                                  int64_t* jc, int32_t cap, int32_t* k) {
  if (!h || !k || level < 1 || level > h->L || box < 0 || box >= (1 << level))
    return WSBM_ERR_INVALID_ARG;
  const Level& LV = h->lv[level];
  if (!LV.compressed) return WSBM_ERR_INVALID_ARG;
  const Box& b = LV.box[box];
  *k = b.k;
  if (cap < b.k || !jr || !jc) return WSBM_ERR_INVALID_ARG;
  // interleaved 2i + c  ->  paper order c N + i
  for (int t = 0; t < b.k; ++t) {
    jr[t] = (int64_t)(b.Jr[t] & 1) * h->N + (b.Jr[t] >> 1);
    jc[t] = (int64_t)(b.Jc[t] & 1) * h->N + (b.Jc[t] >> 1);
  }
  return WSBM_OK;
}

extern "C" int wsbm_stats(wsbm_hss_t h, wsbm_stats_t* s) {
  if (!h || !s) return WSBM_ERR_INVALID_ARG;
  *s = h->stats;
  return WSBM_OK;
}

// ----------------------------------------------------------------- refinement ----
// Iterative refinement with the dense matrix-free product: r = b - A x, x += HSS^-1 r.
// x is kept in paper order [u; q] (one column of 2N per right-hand side).

// r = b - y, with per-block partial sums of |b|^2 and |r|^2 (blocks of one column each).
__global__ void __launch_bounds__(256) k_residual(const double2* __restrict__ b,
                                                  const double2* __restrict__ y,
                                                  double2* __restrict__ r, int64_t len,
                                                  double* __restrict__ part) {
  const int c = blockIdx.y;
  const double2* bc = b + (int64_t)c * len;
  const double2* yc = y + (int64_t)c * len;
  double2* rc = r + (int64_t)c * len;
  double sb = 0.0, sr = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x) {
    double2 bv = bc[i], yv = yc[i];
    double2 rv = make_double2(bv.x - yv.x, bv.y - yv.y);
    rc[i] = rv;
    sb += bv.x * bv.x + bv.y * bv.y;
    sr += rv.x * rv.x + rv.y * rv.y;
  }
  __shared__ double s1[256], s2[256];
  s1[threadIdx.x] = sb;
  s2[threadIdx.x] = sr;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      s1[threadIdx.x] += s1[threadIdx.x + s];
      s2[threadIdx.x] += s2[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * ((int64_t)c * gridDim.x + blockIdx.x)] = s1[0];
    part[2 * ((int64_t)c * gridDim.x + blockIdx.x) + 1] = s2[0];
  }
}

// x[:, c] = [u[:, c]; q[:, c]] (mode 0), or u += x[0:N], q += x[N:2N] (mode 1).
__global__ void k_uq_pack(double2* __restrict__ x, double2* __restrict__ u, double2* __restrict__ q,
                          int64_t N, int nrhs, int mode) {
  const int64_t tot = 2 * N * nrhs;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / (2 * N), i = e % (2 * N);
    double2* d = i < N ? u + c * N + i : q + c * N + (i - N);
    if (mode == 0) {
      x[e] = *d;
    } else {
      double2 v = *d, a = x[e];
      *d = make_double2(v.x + a.x, v.y + a.y);
    }
  }
}

extern "C" int wsbm_refine(wsbm_hss_t h, int32_t trans, const void* rhs, int32_t nrhs, void* u,
                           void* q, int32_t iters, double* res) {
  if (!h || (trans != 0 && trans != 1) || nrhs < 0 || iters < 0) return WSBM_ERR_INVALID_ARG;
  if (!h->factored) return WSBM_ERR_NOT_FACTORED;
  if (h->prm.formulation != WSBM_FORM_WSBM) return WSBM_ERR_INVALID_ARG;  // matvec: eq. (weakly_bm)
  if (nrhs == 0) return WSBM_OK;
  if (!rhs || !u || !q) return WSBM_ERR_INVALID_ARG;
  cudaStream_t st = h->st;
  TmpMem tmpm(h);
  std::vector<void*>& tmp = tmpm.v;
  const int64_t N = h->N, len = 2 * N;
  double2 *x = nullptr, *y = nullptr, *r = nullptr, *du = nullptr, *dq = nullptr;
  double* part = nullptr;
  const int gx = 64;
  HK(dalloc(h, (size_t)len * nrhs * sizeof(double2), (void**)&x, tmp));
  HK(dalloc(h, (size_t)len * nrhs * sizeof(double2), (void**)&y, tmp));
  HK(dalloc(h, (size_t)len * nrhs * sizeof(double2), (void**)&r, tmp));
  HK(dalloc(h, (size_t)N * nrhs * sizeof(double2), (void**)&du, tmp));
  HK(dalloc(h, (size_t)N * nrhs * sizeof(double2), (void**)&dq, tmp));
  HK(dalloc(h, (size_t)2 * gx * nrhs * sizeof(double), (void**)&part, tmp));
  wsbm_geom g;
  g.n = N;
  g.x = h->x;
  g.y = h->y;
  g.nx = h->nx;
  g.ny = h->ny;
  g.w = h->w;
  g.kappa = h->kappa;
  std::vector<double> hp((size_t)2 * gx * nrhs);
  for (int it = 0; it <= iters; ++it) {
    k_uq_pack<<<gridfor(len * nrhs), 256, 0, st>>>(x, (double2*)u, (double2*)q, N, nrhs, 0);
    wsbm_count_launch();
    HK(wsbm_matvec(&g, &h->prm, trans, x, nrhs, y, (void*)st));
    k_residual<<<dim3(gx, nrhs), 256, 0, st>>>((const double2*)rhs, y, r, len, part);
    wsbm_count_launch();
    HC(cudaGetLastError());
    if (res) {
      HC(cudaMemcpyAsync(hp.data(), part, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
      HC(cudaStreamSynchronize(st));
      double sb = 0.0, sr = 0.0;
      for (size_t i = 0; i < hp.size(); i += 2) {
        sb += hp[i];
        sr += hp[i + 1];
      }
      res[it] = sb > 0.0 ? sqrt(sr / sb) : sqrt(sr);
    }
    if (it == iters) break;
    HK(trans ? wsbm_solve_transposed(h, r, nrhs, du, dq) : wsbm_solve(h, r, nrhs, du, dq));
    // x = [du; dq] then u += du, q += dq
    HC(cudaMemcpy2DAsync(r, len * sizeof(double2), du, N * sizeof(double2), N * sizeof(double2), nrhs,
                         cudaMemcpyDeviceToDevice, st));
    HC(cudaMemcpy2DAsync(r + N, len * sizeof(double2), dq, N * sizeof(double2), N * sizeof(double2),
                         nrhs, cudaMemcpyDeviceToDevice, st));
    k_uq_pack<<<gridfor(len * nrhs), 256, 0, st>>>(r, (double2*)u, (double2*)q, N, nrhs, 1);
    wsbm_count_launch();
  }
  HC(cudaStreamSynchronize(st));
  return WSBM_OK;
}
