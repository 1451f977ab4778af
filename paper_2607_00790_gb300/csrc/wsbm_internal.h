// Internal types shared by the CUDA translation units of the library (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/wsbm_hss.h"
#include "dense.h"

struct DevGeom {
  const double *x, *y, *nx, *ny, *w, *kappa;
  int64_t n;
};

struct Phys {
  double k0, k1, eps0, eps1;
  double inv_k0, inv_k1;  // 1/k0, 1/k1
  double s01, s10;        // sqrt(k0/k1), sqrt(k1/k0): 1/sqrt(k1 r) = s01/sqrt(k0 r)
  // FP32 copies for the mixed-precision kernels
  float fk0, fk1, frk0, frk1, finv_k0, feps0, feps1, fpad;  // frk = 1/sqrt(k)
};

// One output block of node-pair entries of the WSBM matrix.  A row "slot" t names row node
// rnode[t]; its equation a (0: first row of eq. (weakly_bm), 1: second row) goes to output
// row rpos[2t+a] (-1: not requested).  Columns likewise with the unknowns u (b = 0), q (b = 1).
// trans = 0: entry (row, col) is stored at out[row + col*ld]; trans = 1: at out[col + row*ld].
struct PairTask {
  const int32_t* rnode;
  const int32_t* rpos;
  const int32_t* cnode;
  const int32_t* cpos;
  double2* out;
  int64_t ld;
  int32_t nr, nc;
  int32_t trans;  // output layout (see above)
  int32_t tile0;  // index of this task's first tile in the launch
  int32_t fastc;  // 1: column slots run along the 32-wide fast tile dimension, 0: row slots
  int32_t inst;   // instance (curve) of a batched launch; 0 otherwise
};

// One proxy-circle block (proxy-surface method).  Box slot t names node node[t]; its
// component a goes to box column pos[2t+a] (-1: absent).  Proxy row index = off + s*P + m,
// s = 0 for the k1 source / field, s = 1 for k0.
// side = 0: sources acting on the box equations;  side = 1: box unknowns' fields at p_m.
// tr = 0: out[proxyrow + boxcol*ld];  tr = 1: out[boxcol + proxyrow*ld].
struct ProxyTask {
  const int32_t* node;
  const int32_t* pos;
  double2* out;
  int64_t ld;
  double cx, cy, rho;
  int32_t nn, P;
  int32_t side, tr;
  int32_t off;
  int32_t tile0;
  int32_t inst;  // instance (curve) of a batched launch; 0 otherwise
  int32_t pad;
};

// Tiles: TILE_F slots along the fast (contiguous-output) dimension x TILE_S along the other
// (the default shape; the entry kernels of eq. (weakly_bm) also take TF = 16 or 64 with
// TS = 128 / TF, the comparison formulations' kernels this shape only).
#define WSBM_TILE_F 32
#define WSBM_TILE_S 4
#define WSBM_PAIR_THREADS 128
#define WSBM_ENTRY_CTAS 16  // default grid of the persistent entry kernels, CTAs per SM

// entries.cu
// Launch the entry kernels.  geos / phys: optional device arrays indexed by the tasks' `inst`
// (batched launches over several curves); when NULL every task uses g / ph.  tf: tile width
// (16, 32 or 64) that the tasks' tile0 and ntiles were counted with (wsbm_pair_tiles /
// wsbm_proxy_tiles with the same tf); ctas: grid size in CTAs per SM (1..64).
int wsbm_launch_pairs(const DevGeom& g, const Phys& ph, const PairTask* d_tasks, int ntasks,
                      int64_t ntiles, cudaStream_t st, const DevGeom* geos = nullptr,
                      const Phys* phys = nullptr, int tf = WSBM_TILE_F, int ctas = WSBM_ENTRY_CTAS);
int wsbm_launch_proxy(const DevGeom& g, const Phys& ph, const ProxyTask* d_tasks, int ntasks,
                      int64_t ntiles, int mixed, cudaStream_t st, const DevGeom* geos = nullptr,
                      const Phys* phys = nullptr, int tf = WSBM_TILE_F, int ctas = WSBM_ENTRY_CTAS);
// forms.cu: the same tasks for the comparison formulations (form 1: eq. bm, 2: eq. pmchwt);
// the proxy launch takes row-side tasks only (the column side is formulation independent).
int wsbm_launch_pairs_form(int form, const DevGeom& g, const Phys& ph, const PairTask* d_tasks,
                           int ntasks, int64_t ntiles, cudaStream_t st, const DevGeom* geos = nullptr,
                           const Phys* phys = nullptr);
int wsbm_launch_proxy_rows_form(int form, const DevGeom& g, const Phys& ph, const ProxyTask* d_tasks,
                                int ntasks, int64_t ntiles, cudaStream_t st,
                                const DevGeom* geos = nullptr, const Phys* phys = nullptr);
int64_t wsbm_pair_tiles(int32_t nr, int32_t nc, int32_t fastc, int tf = WSBM_TILE_F);
int64_t wsbm_proxy_tiles(int32_t nn, int32_t P, int tf = WSBM_TILE_F);
int wsbm_launch_hankel(const double* z, int64_t n, double* out, int mixed, cudaStream_t st);
int wsbm_launch_unknowns_to_slots(const int64_t* idx, int64_t n, int64_t N, int32_t* node,
                                  int32_t* pos, cudaStream_t st);

// sketch.cu: randomized row sketches Y = Omega M of ID matrices on the tensor cores.  h_desc:
// host array of ndesc descriptors (wsbm_sketch_desc_fill); the matrices go through in launches
// whose work space stays within `cap` bytes (one matrix always fits: wsbm_sketch_ws_bytes gives
// the work space the same split needs).  Enqueues only.
size_t wsbm_sketch_ws_bytes(const void* h_desc, int ndesc, size_t cap);
int wsbm_sketch_batched(const void* h_desc, int ndesc, uint32_t seed, void* ws, size_t cap, cudaStream_t st);
size_t wsbm_sketch_desc_size();
void wsbm_sketch_desc_fill(void* slot, const void* A, int64_t lda, void* Y, int64_t ldy, int32_t m,
                           int32_t n, int32_t l);

// capi.cu: device memory of the library.  Every allocation goes through the allocator set by
// wsbm_set_allocator (a handle captures it at creation; the stateless calls read it at each
// call), else through the library's memory pool of the current device.  Both are stream
// ordered on the call's stream.
struct WsbmAllocator {
  wsbm_alloc_fn alloc = nullptr;
  wsbm_free_fn release = nullptr;
  void* ctx = nullptr;
};
WsbmAllocator wsbm_current_allocator();
int wsbm_dev_alloc(const WsbmAllocator& a, size_t bytes, cudaStream_t st, void** p);
void wsbm_dev_free(const WsbmAllocator& a, void* p, cudaStream_t st);

// Work space of one stateless call, released in stream order when it goes out of scope (also
// on an early error return).
struct WsbmScratch {
  WsbmAllocator a;
  cudaStream_t st;
  std::vector<void*> v;
  explicit WsbmScratch(cudaStream_t s) : a(wsbm_current_allocator()), st(s) {}
  ~WsbmScratch() {
    for (void* p : v) wsbm_dev_free(a, p, st);
  }
  int get(size_t bytes, void** p) {
    int rc = wsbm_dev_alloc(a, bytes, st, p);
    if (rc == WSBM_OK) v.push_back(*p);
    return rc;
  }
};
