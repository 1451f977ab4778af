// wsbm_entries_raw_noalloc: the entries of wsbm_entries_raw without any device allocation.
//
// Its scratch (the row / column slot lists and the task descriptor) lives in one file-scope
// device array of fixed size.  Every GPU that loads the library holds this array until the
// process exits.  In host code the array's name stands for a host-side shadow, not a device
// address, so the host looks the address up with cudaGetSymbolAddress once per device (on the
// first call made on that device, with that device current) and passes it to the kernels.
#include <string.h>

#include <mutex>

#include "wsbm_internal.h"

int wsbm_phys_from_params(const wsbm_params* p, Phys* ph);
int wsbm_geom_check(const wsbm_geom* g);
DevGeom wsbm_devgeom(const wsbm_geom* g);

// Bytes: one 256-byte slot for the task descriptor, then 3 int32 per row index (node, two
// positions) and 3 per column index.
#define WSBM_NOALLOC_BYTES (256 + (size_t)6 * WSBM_NOALLOC_MAX_INDICES * sizeof(int32_t))

static __device__ __align__(256) unsigned char g_noalloc_scratch[WSBM_NOALLOC_BYTES];

#define WSBM_NOALLOC_MAX_DEVICES 64
static void* g_scratch_addr[WSBM_NOALLOC_MAX_DEVICES];
static std::mutex g_scratch_mutex;

// Device address of the scratch array on the current device (looked up once per device).
static int scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return WSBM_ERR_CUDA;
  if (dev < 0 || dev >= WSBM_NOALLOC_MAX_DEVICES) return WSBM_ERR_NO_DEVICE;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return WSBM_ERR_CUDA;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return WSBM_OK;
}

// The task descriptor is written on the device from a by-value kernel argument, so no host
// buffer has to outlive the call.
__global__ void k_store_task(PairTask* dst, PairTask t) { *dst = t; }

extern "C" int wsbm_entries_raw_noalloc(const wsbm_geom* g, const wsbm_params* p,
                                        const int64_t* rows, int64_t nr, const int64_t* cols,
                                        int64_t nc, void* out, void* stream) {
  int rc = wsbm_geom_check(g);
  if (rc) return rc;
  Phys ph;
  if ((rc = wsbm_phys_from_params(p, &ph))) return rc;
  if (p->formulation != WSBM_FORM_WSBM) return WSBM_ERR_INVALID_ARG;  // eq. (weakly_bm) only
  if (nr < 0 || nc < 0 || nr + nc > WSBM_NOALLOC_MAX_INDICES) return WSBM_ERR_INVALID_ARG;
  if (nr == 0 || nc == 0) return WSBM_OK;
  if (!rows || !cols || !out) return WSBM_ERR_INVALID_ARG;
  void* base = nullptr;
  if ((rc = scratch_address(&base))) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  PairTask* dtask = (PairTask*)base;
  int32_t* rnode = (int32_t*)((unsigned char*)base + 256);
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
  // every slot entry is written by the two kernels below, so nothing needs clearing
  if ((rc = wsbm_launch_unknowns_to_slots(rows, nr, g->n, rnode, rpos, st))) return rc;
  if ((rc = wsbm_launch_unknowns_to_slots(cols, nc, g->n, cnode, cpos, st))) return rc;
  k_store_task<<<1, 1, 0, st>>>(dtask, t);
  wsbm_count_launch();
  if (cudaGetLastError() != cudaSuccess) return WSBM_ERR_CUDA;
  return wsbm_launch_pairs(wsbm_devgeom(g), ph, dtask, 1, wsbm_pair_tiles(t.nr, t.nc, 0), st);
}
