/*
 * wsbm_hss.h -- C ABI of the GB300 (sm_103a) entry generator and HSS direct solver for the
 * weakly singular Burton-Miller (WSBM) boundary integral equation of 2-D TE-mode transmission
 * scattering (Matsumoto & Yokota, "Proxy-surface-based fast direct solver for TE-mode
 * scattering problems on distributed memory systems"), and of the standard Burton-Miller and
 * PMCHWT equations the paper compares it with (wsbm_params.formulation).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Return value: WSBM_OK (0) on success, a negative WSBM_ERR_* code otherwise; no C++
 *    exception crosses this boundary.  wsbm_strerror() names a code.
 *  - Pointers documented as "device" are CUDA device pointers of the current device; they are
 *    owned by the caller and only read (inputs) or written (outputs) during the call, in
 *    stream order on `stream` (a cudaStream_t passed as void*; NULL = the legacy default
 *    stream).  Calls return after enqueueing unless stated otherwise.
 *  - Complex numbers are interleaved (re, im) pairs of doubles (complex128).
 *  - Matrices are column-major.
 *  - Unknown indices follow the paper's block order [u ; q] (eq. weakly_bm): for a curve of N
 *    nodes, index r < N is u at node r (and, as a row, the first equation at node r);
 *    index r >= N is q at node r - N (the second equation).
 *  - Geometry: N nodes in counter-clockwise order along a closed smooth curve, outward unit
 *    normals, trapezoidal weights w_j (= h |gamma'(t_j)| for equispaced t_j) and curvature
 *    kappa_j (needed by the one-point corrected diagonal of D and D*).
 */
#ifndef WSBM_HSS_H
#define WSBM_HSS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  WSBM_OK = 0,
  WSBM_ERR_INVALID_ARG = -1,   /* bad size, NULL pointer, non-finite or inconsistent input */
  WSBM_ERR_OOM = -2,           /* a device or host allocation failed                        */
  WSBM_ERR_CUDA = -3,          /* a CUDA runtime call or kernel launch failed               */
  WSBM_ERR_RANK_OVERFLOW = -4, /* an interpolative decomposition needed more than its cap   */
  WSBM_ERR_TIMEOUT = -5,       /* a bounded device wait gave up                             */
  WSBM_ERR_NOT_FACTORED = -6,  /* solve/farfield before a successful wsbm_factor            */
  WSBM_ERR_NO_DEVICE = -7      /* no usable sm_103 device                                   */
};

enum { WSBM_FP64 = 0, WSBM_MIXED = 1, WSBM_MIXED_FINE = 2 };

/* Curve data, all device pointers to n doubles, caller-owned. */
typedef struct {
  int64_t n;
  const double *x, *y;   /* node positions                    */
  const double *nx, *ny; /* outward unit normals              */
  const double *w;       /* quadrature weights                */
  const double *kappa;   /* signed curvature (circle: 1/R)    */
} wsbm_geom;

/* Physical and solver parameters.
 *  k0          exterior wavenumber (> 0)
 *  refr_index  n = k1/k0 (> 0); with mu0 = mu1 = 1, eps1 = n^2 eps0 (Sec. II, k_j = omega sqrt(eps_j mu_j))
 *  eps0, eps1  permittivities; eps1 <= 0 selects eps1 = n^2 eps0; eps0 <= 0 selects 1
 *  leaf        target leaf size in nodes (>= 4); the tree is a perfect binary tree of depth
 *              L = ceil(log2(n/leaf)) over contiguous node ranges (Sec. III, Fig. tree)
 *  nproxy      proxy points on each leaf's proxy circle (>= 8; grown on upper levels)
 *  id_tol      accuracy target of the HSS solution (0 < id_tol < 1): the column-pivoted QRs of
 *              the interpolative decompositions stop at |R_kk| <= id_tol / (4 sqrt(2^L)) |R_00|
 *              (L the tree depth: the errors of the 2^L leaf boxes add up in the solution), which
 *              keeps densities and far field within a few id_tol of the dense solution
 *  precision   WSBM_FP64; WSBM_MIXED: proxy blocks evaluated with an FP32 amplitude and phase
 *              factor after an FP64 phase reduction (entries to ~1e-7); WSBM_MIXED_FINE: proxy
 *              blocks with only the amplitude corrections P - 1, Q of the Hankel functions in
 *              FP32 (entries to ~2e-8).  Every other entry, the ID and the factor stay FP64
 *  proxy_ratio proxy radius / box radius (<= 1 selects 1.5)
 *  max_levels  0: build and factor the whole tree.  m > 0: compress only the m lowest tree
 *              levels and stop before the dense root (a partial build for measuring the build
 *              phase on problems whose root system would not fit); solve then fails with
 *              WSBM_ERR_NOT_FACTORED
 *  root_cap    largest dense root order accepted (0 selects 40000); a factorization whose
 *              merged skeleton system would be larger fails with WSBM_ERR_RANK_OVERFLOW.
 *              Compression goes on past the levels that save under 20 % until the merged
 *              system fits both root_cap and three quarters of the device memory
 *  id_method   WSBM_ID_SKETCH (0): leaf-level IDs from the column-pivoted QR of a tensor-core
 *              sketch Omega M of the ID matrix (l = 16 ceil(n/32) rows, used when M has at
 *              least 1.5 l rows; the QR of a sketch stops at a quarter of the usual cutoff; a
 *              side whose rank, or the box's, comes within 16 of l is redone on M);
 *              WSBM_ID_FULL (1): column-pivoted QR of the full ID matrices everywhere
 *  formulation WSBM_FORM_WSBM (0): eq. (weakly_bm), third order; WSBM_FORM_BM (1): the
 *              standard Burton-Miller equation, eq. (bm); WSBM_FORM_PMCHWT (2): eq. (pmchwt),
 *              unknowns still (u, q), right-hand side [-u_in ; -eps0^-1 du_in/dn].  Forms 1 and
 *              2 hold the hypersingular N_k, whose one-point correction leaves them first order
 *              (the paper's comparison, Sec. II); they need precision WSBM_FP64 and are
 *              refused (INVALID_ARG) by the matrix-free product, the no-allocation entries and
 *              the gradient calls, which implement eq. (weakly_bm) only
 */
enum { WSBM_ID_SKETCH = 0, WSBM_ID_FULL = 1 };
enum { WSBM_FORM_WSBM = 0, WSBM_FORM_BM = 1, WSBM_FORM_PMCHWT = 2 };
typedef struct {
  double k0, refr_index, eps0, eps1;
  int32_t leaf, nproxy;
  double id_tol;
  int32_t precision;
  double proxy_ratio;
  int32_t max_levels, root_cap;
  int32_t id_method, formulation;
} wsbm_params;

/* Counters of a handle. */
typedef struct {
  int32_t levels;              /* tree depth L                                        */
  int32_t nboxes_leaf;
  int64_t entries_generated;   /* complex entries written by the entry kernels         */
  int64_t pairs_evaluated;     /* node-node and node-proxy pairs evaluated             */
  double ms_entries;           /* summed device time of the entry kernels             */
  double ms_id;                /* interpolative decompositions                        */
  double ms_factor;            /* LU, R D^-1 L, root                                  */
  double ms_total_factor;      /* wsbm_factor wall time on the stream (events)        */
  int32_t max_rank;            /* largest skeleton size                               */
  int32_t root_size;           /* order of the dense root system                      */
  int32_t rank_per_level[32];  /* largest skeleton size on each level (index = level) */
  int64_t factor_bytes;        /* device memory held by the factors                   */
  int64_t entries_proxy;       /* entries written by the proxy-block kernel            */
  int64_t pairs_proxy;         /* node / proxy-point pairs it evaluated                */
  double ms_proxy;             /* its summed device time                              */
  int64_t entries_pairs;       /* entries written by the node-pair kernel              */
  int64_t pairs_pairs;         /* node pairs it evaluated                              */
  double ms_pairs;             /* its summed device time                              */
  int64_t launches;            /* kernels launched by the last wsbm_factor            */
  double ms_cpqr;              /* device time of the first column-pivoted QR launch   */
  int64_t cpqr_matrices;       /* ID matrices it factored (sketches or full matrices) */
  double cpqr_flops;           /* its algorithmic FP64 flops: 16 per element per step */
  int64_t sketch_matrices;     /* ID matrices replaced by their sketch                */
  int64_t sketch_fallbacks;    /* sketched sides redone on the full matrix            */
  double ms_sketch;            /* device time of the sketch launches                  */
  double ms_lu;                /* device time of the box factors' LU + solve launches
                                  (LU with D^-1 L, and Dhat), summed over the levels   */
  double lu_flops;             /* their algorithmic FP64 flops                        */
  int64_t lu_matrices;         /* matrices they factored                              */
  int64_t lu_tc_matrices;      /* of these, factored by the batched LU whose products
                                  run on the tensor cores (the rest: fused FP64 kernel) */
} wsbm_stats_t;

typedef struct wsbm_hss* wsbm_hss_t;

/* Device memory of the library: a handle's geometry copy, factors, work space and solve plans,
 * and the work space of the stateless calls (wsbm_entries_raw, wsbm_proxy_block, wsbm_matvec,
 * wsbm_field, wsbm_sketch, wsbm_entries_vjp).  No call allocates device memory any other way
 * (wsbm_entries_raw_noalloc allocates none).
 * alloc(bytes, stream, ctx): device memory of at least `bytes` bytes usable in stream order on
 * `stream` (the handle's stream), or NULL (the call then fails with WSBM_ERR_OOM).
 * release(ptr, stream, ctx): returns a block in stream order: work queued on `stream` before
 * the call may still read or write it.  Both are called from the calling host thread only.
 * The default is a library memory pool per device (see wsbm_trim_memory); a framework's
 * caching allocator can be plugged in instead, so that it supplies the memory. */
typedef void* (*wsbm_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*wsbm_free_fn)(void* ptr, void* stream, void* ctx);

/* Allocator of the handles created after this call (a handle keeps the one it was created
 * with, for all its allocations and releases) and of the stateless calls made after it (each
 * call takes and returns its work space through the allocator current at its start).  alloc = release = NULL restores the library
 * pool.  Errors: INVALID_ARG when exactly one of the two is NULL.  No device is touched. */
int wsbm_set_allocator(wsbm_alloc_fn alloc, wsbm_free_fn release, void* ctx);

/* ---------------------------------------------------------------- stateless kernels ---- */

/* Hankel functions H0^(1)(z), H1^(1)(z) at n arguments z > 0 (the kernel of every layer
 * potential of eq. weakly_bm; G_k = (i/4) H0^(1)(k r)).
 *   z    device, n doubles
 *   out  device, 6n doubles: per argument Re H0, Im H0, Re H1, Im H1, Re F1, Im F1 where
 *        F1(z) = H1(z)/z + 2i/(pi z^2) (pole-free part used by N_k0 - N_k1)
 *   precision  WSBM_FP64, WSBM_MIXED (FP32 amplitude and phase factor after an FP64 phase
 *              reduction; F1 not computed, zeros) or WSBM_MIXED_FINE (FP32 P - 1 and Q only)
 * Errors: INVALID_ARG (n < 0, NULL with n > 0), CUDA. */
int wsbm_hankel01(const double* z, int64_t n, double* out, int32_t precision, void* stream);

/* Entries A[rows, cols] of the 2N x 2N Nystrom matrix of eq. (weakly_bm) (block form A_ij of
 * Sec. III) with the one-point corrected diagonal.
 *   rows, cols  device int64 unknown indices in [0, 2N), paper order
 *   out         device complex128, column-major nr x nc (leading dimension nr)
 * Errors: INVALID_ARG (bad sizes, NULL pointers, parameters out of range), OOM, CUDA.
 * Indices out of range are not checked on the device; they must lie in [0, 2N). */
int wsbm_entries_raw(const wsbm_geom* g, const wsbm_params* p, const int64_t* rows, int64_t nr,
                     const int64_t* cols, int64_t nc, void* out, void* stream);

/* Largest nr + nc accepted by wsbm_entries_raw_noalloc. */
#define WSBM_NOALLOC_MAX_INDICES 65536

/* Same entries as wsbm_entries_raw, computed without allocating any device memory.  The paper
 * has no counterpart to this call: it exists for callers that cannot allocate, for example a
 * framework whose caching allocator already owns the GPU's memory, code that runs under a fixed
 * device-memory budget, or a latency-critical path that must not pay for cudaMalloc/cudaFree
 * (which can synchronise with the device).
 * Scratch: a library-owned device array of 256 + 24 * WSBM_NOALLOC_MAX_INDICES bytes (about
 * 1.5 MB), held by every GPU that loads the library until the process exits.  The first call on
 * a device looks up that array's device address (cudaGetSymbolAddress, with that device
 * current); make that first call before any stream capture.  The array is shared by every
 * call and keeps the last call's contents: calls whose work overlaps on the GPU (different
 * streams, or different host threads on one device) race and must be ordered by the caller.
 * Arguments, layout and ownership as for wsbm_entries_raw; the call only enqueues work.
 * Errors: INVALID_ARG (also when nr + nc > WSBM_NOALLOC_MAX_INDICES), CUDA, NO_DEVICE. */
int wsbm_entries_raw_noalloc(const wsbm_geom* g, const wsbm_params* p, const int64_t* rows,
                             int64_t nr, const int64_t* cols, int64_t nc, void* out, void* stream);

/* Proxy-circle blocks of the proxy-surface method (Sec. III) for one box, the inputs of its
 * interpolative decompositions.  The circle has centre (cx, cy), radius rho and P equispaced
 * points p_m = c + rho (cos 2 pi m/P, sin 2 pi m/P) with outward normals.
 * Row block (side = 0): rows = the box equations `idx` (paper order), 2P columns: column m is
 *   the k1 combined-field source (d/dnu - i k1) G_k1 at p_m entering [eq1 ; -alpha d/dn_x],
 *   column P+m the k0 source entering [0 ; 1 + alpha d/dn_x]; scaled by 2 pi rho / P.
 *   out: complex128 nidx x 2P, column-major.
 * Column block (side = 1): 2P rows (the k1 field, then the k0 field, of the box unknowns at
 *   the proxy points), columns = the box unknowns `idx`.  out: complex128 2P x nidx.
 * precision WSBM_MIXED / WSBM_MIXED_FINE evaluate these blocks as described for wsbm_params.
 * Errors: INVALID_ARG, OOM, CUDA. */
int wsbm_proxy_block(const wsbm_geom* g, const wsbm_params* p, int32_t side, const int64_t* idx,
                     int64_t nidx, double cx, double cy, double rho, int32_t P, void* out,
                     void* stream);

/* -------------------------------------------------------------------- HSS solver ---- */

/* Create a solver handle for a curve (copies nothing but the pointers' data it needs: the
 * geometry is copied into library-owned device memory, so the caller may free g afterwards).
 * The handle uses `stream` for all its work.  Errors: INVALID_ARG (n < 2*leaf... see leaf,
 * non-finite geometry), OOM, CUDA, NO_DEVICE. */
int wsbm_create(const wsbm_geom* g, const wsbm_params* p, void* stream, wsbm_hss_t* out);

/* Build and factor the HSS approximation of the WSBM matrix: per tree level, leaf to root,
 * generate the dense diagonal blocks, the proxy and near-field blocks, compute row and column
 * interpolative decompositions (column-pivoted QR with relative tolerance id_tol), form the
 * sibling skeleton blocks and the compressed Martinsson-Rokhlin factors; LU of the dense
 * root.  Synchronous (returns when the factor is complete).  Errors: OOM, CUDA,
 * RANK_OVERFLOW. */
int wsbm_factor(wsbm_hss_t h);

/* Right-hand sides of eq. (weakly_bm) for plane waves exp(i k0 (cos a, sin a).x):
 * [0 ; -u_in - alpha du_in/dn].  angles: device, nang doubles; rhs: device complex128,
 * 2N x nang column-major, paper order. */
int wsbm_rhs_planewave(wsbm_hss_t h, const double* angles, int32_t nang, void* rhs);

/* Solve A [u; q] = rhs with the factors.  rhs: device complex128 2N x nrhs (paper order);
 * u, q: device complex128 N x nrhs each.  The first call with a given nrhs builds a solve plan
 * (work buffers, descriptors) and captures its launches into a CUDA graph; later calls with the
 * same nrhs replay it.  Synchronous.  Errors: NOT_FACTORED, OOM, CUDA. */
int wsbm_solve(wsbm_hss_t h, const void* rhs, int32_t nrhs, void* u, void* q);

/* Transposed solve A^T lam = rhs with the same factors (the adjoint solve of a gradient).
 * rhs: device complex128 2N x nrhs indexed like the unknowns [u; q] (paper order); lam1, lam2:
 * device complex128 N x nrhs each, the multipliers of the first and second equations.
 * The paper has no counterpart (it does not differentiate its solver).  Errors: as
 * wsbm_solve. */
int wsbm_solve_transposed(wsbm_hss_t h, const void* rhs, int32_t nrhs, void* lam1, void* lam2);

/* Iterative refinement of a solution against the dense Nystrom matrix of eq. (weakly_bm):
 * r = rhs - A x, x += HSS^-1 r (trans = 0; x = [u; q]), or, for the adjoint system
 * A^T lam = rhs, r = rhs - A^T lam, lam += HSS^-T r (trans = 1; u, q then hold the multipliers
 * lam1, lam2 of the first and second equations).  The products are the matrix-free ones of
 * wsbm_matvec (every node pair, O(N^2) work each), the corrections come from the handle's
 * factors (wsbm_solve / wsbm_solve_transposed), so each step gains about the accuracy of the
 * HSS solve.  The paper has no counterpart (its solutions are the HSS ones).
 *   rhs   device complex128 2N x nrhs (paper order, as for wsbm_solve)
 *   u, q  device complex128 N x nrhs each: the solution on entry, the refined one on exit
 *   iters refinement steps (>= 0)
 *   res   host, iters + 1 doubles, or NULL: |r| / |rhs| (Frobenius over all right-hand sides)
 *         before each step and after the last
 * Work space from the handle's allocator.  Synchronous.  Errors: INVALID_ARG (also for the
 * formulations other than eq. weakly_bm), NOT_FACTORED, OOM, CUDA. */
int wsbm_refine(wsbm_hss_t h, int32_t trans, const void* rhs, int32_t nrhs, void* u, void* q,
                int32_t iters, double* res);

/* Far-field pattern of the scattered field at nang observation angles:
 * u_inf(a) = e^{i pi/4}/sqrt(8 pi k0) sum_j w_j [-i k0 (xh.n_j) u_j - eps0 q_j] e^{-i k0 xh.x_j}.
 * u, q: device complex128 N x nrhs; angles: device doubles; out: device complex128
 * nang x nrhs. */
int wsbm_farfield(wsbm_hss_t h, const void* u, const void* q, int32_t nrhs, const double* angles,
                  int32_t nang, void* out);

/* Entries of the handle's matrix (same as wsbm_entries_raw with the handle's geometry). */
int wsbm_entries(wsbm_hss_t h, const int64_t* rows, int64_t nr, const int64_t* cols, int64_t nc,
                 void* out);

/* Proxy circle the handle uses for box `box` (0-based, left to right) on tree level `level`
 * (0 = root, L = leaves), and the node range [first, last) of that box.
 * out4 (host): cx, cy, R, rho; range2 (host): first, last. */
int wsbm_box_info(wsbm_hss_t h, int32_t level, int32_t box, double* out4, int64_t* range2);

/* Skeletons of box `box` on level `level` after wsbm_factor (also after a partial build):
 * k (host) receives the skeleton size; jr, jc (host, capacity cap each) receive the row and
 * column skeleton indices in the paper's unknown order.  Errors: INVALID_ARG (level not
 * compressed, cap < k). */
int wsbm_box_skeletons(wsbm_hss_t h, int32_t level, int32_t box, int64_t* jr, int64_t* jc,
                       int32_t cap, int32_t* k);

/* Counters and timings (host struct). */
int wsbm_stats(wsbm_hss_t h, wsbm_stats_t* s);

/* Release every device buffer of the handle. */
void wsbm_destroy(wsbm_hss_t h);

/* ------------------------------------------------------------------ batched builds ---- */

/* Batches of independent scatterers (each curve with its own physics and parameters, all
 * sharing one stream).  wsbm_batch_factor builds and factors every curve with one launch per
 * phase per tree level over all curves (curves of different depth are aligned at their leaves,
 * each stops compressing by its own rule), then all dense roots in one batched LU: the paper's
 * equal-cost-per-block load balance carried across many scatterers.
 * Results are identical to factoring each curve alone. */
typedef struct wsbm_batch* wsbm_batch_t;

/* g[0..count), p[0..count): as for wsbm_create (geometry copied).  Errors as wsbm_create. */
int wsbm_batch_create(const wsbm_geom* g, const wsbm_params* p, int32_t count, void* stream,
                      wsbm_batch_t* out);

/* Synchronous.  Errors: OOM, CUDA, RANK_OVERFLOW (any curve). */
int wsbm_batch_factor(wsbm_batch_t b);

/* Handle of curve i (owned by the batch: use it for rhs / solve / far field / stats, do not
 * destroy it). */
int wsbm_batch_handle(wsbm_batch_t b, int32_t i, wsbm_hss_t* out);

/* Solve every curve of a factored batch: rhs[i] (device complex128 2N_i x nrhs, paper order),
 * u[i], q[i] (device complex128 N_i x nrhs); rhs, u, q are host arrays of `count` device
 * pointers.  All curves go through one solve plan: each phase of a tree step is one launch over
 * the boxes of every curve (levels aligned at the leaves), the roots are one batched LU solve,
 * and the whole launch sequence is captured into a CUDA graph on the first call with a given
 * nrhs and replayed by later calls (wsbm_solve uses the same plan machinery for one curve).
 * The plan's buffers and descriptors stay allocated until the next factorization, a call with
 * another nrhs, or destruction.  Synchronous.  Errors: NOT_FACTORED, INVALID_ARG, OOM, CUDA. */
int wsbm_batch_solve(wsbm_batch_t b, const void* const* rhs, int32_t nrhs, void* const* u,
                     void* const* q);

/* Timings of the shared launches and summed counters of the last wsbm_batch_factor. */
int wsbm_batch_stats(wsbm_batch_t b, wsbm_stats_t* s);

void wsbm_batch_destroy(wsbm_batch_t b);

/* Matrix-free product y = A x (trans = 0) or y = A^T x (trans = 1) with the full Nystrom
 * matrix of eq. (weakly_bm) (every node pair, O(N^2) work, nothing stored): residuals and
 * iterative refinement of HSS and adjoint solutions.  x, y: device complex128 2N x nrhs in
 * paper order (for trans = 0, x by unknown and y by equation; the reverse for trans = 1).
 * The Hankel values of each node pair are evaluated once for up to four right-hand sides.
 * Scratch: 4 x 2N x (eight waves of CTAs / ceil(N/128)) complex128 from the library's
 * allocator (wsbm_set_allocator) on `stream`.  Asynchronous.  Errors: INVALID_ARG, OOM, CUDA. */
int wsbm_matvec(const wsbm_geom* g, const wsbm_params* p, int32_t trans, const void* x,
                int32_t nrhs, void* y, void* stream);

/* Field at nt points off the curve from densities u, q (device complex128 N x nrhs), by the
 * integral representations (Sec. II: the domain solution follows from the boundary values):
 * exterior points get the scattered field D_k0[u] - eps0 S_k0[q] (add the incident wave for
 * the total field), interior points the total field eps1 S_k1[q] - D_k1[u].  tx, ty: device
 * doubles; out: device complex128 nt x nrhs; inside: device int8 nt, 1 for interior points
 * (Gauss test of the Laplace double layer).  The trapezoidal sums are accurate a few node
 * spacings away from the curve; no near-singular quadrature is applied.  Scratch from the
 * library's allocator (wsbm_set_allocator) on `stream`; asynchronous.  Errors: INVALID_ARG, OOM, CUDA. */
int wsbm_field(const wsbm_geom* g, const wsbm_params* p, const void* u, const void* q,
               int32_t nrhs, const double* tx, const double* ty, int64_t nt, void* out,
               int8_t* inside, void* stream);

/* Randomized row sketch Y = Omega A on the tensor cores: A device complex128 m x n (column-
 * major, lda >= m), Omega the l x m Rademacher matrix with entries +-1 (bit 0 of a counter-based
 * hash of (row, column, seed)), Y device complex128 l x n (ldy >= l).  Products are formed
 * exactly from seven 8-bit digits of the power-of-two scaled columns of A (tcgen05 BF16 MMAs
 * with exact FP32 sums), so Y carries a relative error of about 2^-56 of its column scale.  The HSS
 * build uses it for the interpolative decompositions of the leaf level (no counterpart in the
 * paper, which does not say how its IDs are computed).  l: multiple of 16 in [16, 192];
 * m <= 65536.  Synchronous.  Errors: INVALID_ARG, OOM, CUDA. */
int wsbm_sketch(const void* A, int64_t lda, int32_t m, int32_t n, int32_t l, void* Y, int64_t ldy,
                uint32_t seed, void* stream);

/* Complex GEMM C = beta C + alpha A B on the tensor cores, the dense contraction of the
 * blocked LU factorizations of large boxes and of the dense root (the paper factors with FP64
 * CPU arithmetic; GB300's FP64 pipe runs at 1/64 of its FP32 rate and far below its tensor
 * cores).  Rows of A and columns of B are scaled by powers of two and cut into seven exact
 * 8-bit digits; BF16 tensor-core products of the digits accumulate in FP32 (exactly for the
 * leading digit diagonals) and are recombined in 64-bit integers with a 2^-64 fraction, so each
 * entry of A B carries an error below about 2^-53 * 2k * max_l |A_il| * max_l |B_lj| (the
 * order of an FP64 product).
 *   A  device complex128 m x k (lda >= m); B: k x n (ldb >= k); C: m x n (ldc >= m); all
 *      column-major; alpha, beta: host, 2 doubles (re, im) each
 *   1 <= k <= 32768
 * Work space (7 (m + 2n) 2k BF16 values, rounded up) from the library's allocator.
 * Synchronous.  Errors: INVALID_ARG, OOM, CUDA, TIMEOUT (a bounded wait inside the kernel ran
 * out; the result is then incomplete). */
int wsbm_zgemm(int32_t m, int32_t n, int32_t k, const double* alpha, const void* A, int64_t lda,
               const void* B, int64_t ldb, const double* beta, void* C, int64_t ldc, void* stream);

/* Many independent products C_i = beta C_i + alpha A_i B_i in one launch of the same
 * tensor-core kernel (the batched trailing updates of the box factors): items[i] gives device
 * pointers and sizes of product i (layout and error bound as for wsbm_zgemm; k_i >= 1, the
 * shorter products are padded with zeros to the largest k).  count <= 65535; alpha, beta: host,
 * 2 doubles each, common to all items.  Synchronous.  Errors: as wsbm_zgemm. */
typedef struct {
  const void* A;
  int64_t lda;
  const void* B;
  int64_t ldb;
  void* C;
  int64_t ldc;
  int32_t m, n, k, pad;
} wsbm_gemm_item;
int wsbm_zgemm_batched(int32_t count, const wsbm_gemm_item* items, const double* alpha,
                       const double* beta, void* stream);

/* LU factorization with partial pivoting of one dense complex matrix (the dense root of the
 * Martinsson-Rokhlin factor, Sec. III, at the sizes of full builds): right-looking, panels of
 * 128 columns factored on the whole GPU, trailing updates through the tensor-core product of
 * wsbm_zgemm.  A: device complex128 n x n (lda >= n), overwritten by L (unit lower, below the
 * diagonal) and U; piv: device int32 n, piv[j] = the row swapped with row j at step j.  The
 * pivot is the row of largest max(|Re|, |Im|) to within 2^-20 (first row on ties).  A zero
 * pivot leaves a zero multiplier column (no error).  Work space (about 10.8 KB per row) from
 * the library's allocator.  Synchronous.  Errors: INVALID_ARG, OOM, CUDA, TIMEOUT. */
int wsbm_lu_dense(void* A, int64_t lda, int32_t n, int32_t* piv, void* stream);

/* Autotuners of the launch shapes (no counterpart in the paper).  Each times its candidates
 * with CUDA events on `stream`, keeps the fastest for every later call on the current device
 * (builds, solves, wsbm_zgemm*, wsbm_lu_dense) for the rest of the process, and leaves the
 * other shapes as they were.  Every shape gives the same accuracy; the GEMM raster group and
 * the entry-kernel shapes change no bit of any result (the panel widths and QR block sizes
 * change the rounding order).  While an autotuner runs it switches the device's shapes between
 * candidates: other calls on the same device must not run at the same time.
 *
 * wsbm_autotune: synthetic complex data of the given sizes, best of three after one warm-up:
 *   out[0]  rows of 128-row tiles per raster group of the tensor-core GEMM's tile order, of
 *           {4, 8, 16} (one 8192 x 8192 x 256 product);
 *   out[1]  panel width of the batched box LU, of {32, 64} (nbox boxes of n_box unknowns with
 *           nrhs_box right-hand sides each: the leaf level of a build);
 *   out[2], out[3]  outer panel width of the root LU, of {128, 256}, for roots below and from
 *           12288 unknowns; only the class of n_root is timed, the other keeps its value;
 *   out[4]  columns per warp pass of the column-pivoted QR of ID matrices of more than 2048
 *           rows, of {2, 4, 8} (152 matrices of 2560 x 128).
 * ms: host, 10 doubles or NULL: the candidates' times in that order.  Work space (two copies of
 * the boxes, two n_root x n_root matrices, about 1.2 GiB for the product and 1.5 GiB for the
 * QRs) from the library's allocator.  Sizes: 64 <= n_box <= 4096, 1 <= nbox <= 32767, 1 <= nrhs_box <= 4096,
 * at most 8 GiB of boxes, 256 <= n_root <= 32768.  Defaults without a call: 8, 64, 128, 256, 4.
 * Synchronous.  Errors: INVALID_ARG, OOM, CUDA, TIMEOUT. */
int wsbm_autotune(int32_t n_box, int32_t nbox, int32_t nrhs_box, int32_t n_root, int32_t* out,
                  double* ms, void* stream);
/* wsbm_autotune_build: leaf-level builds (p->max_levels taken as 1) of the given problem, one
 * per candidate after one warm-up build, timed by the library's per-kernel device times
 * (wsbm_stats_t ms_pairs, ms_proxy, and ms_id for the QR):
 *   out[0], out[1]  tile width (16, 32 or 64 nodes along the contiguous output dimension,
 *           128 / width along the other) and grid (8, 16 or 32 CTAs per SM) of the node-pair
 *           entry kernel of eq. (weakly_bm) (the comparison formulations keep 32 and 16);
 *   out[2], out[3]  the same for the proxy-block kernel;
 *   out[4]  threads per CTA (128 or 256) of the thread-per-column QR of the ID matrices.
 * ms: host, 20 doubles or NULL: pair-kernel times of the 9 (width, grid) pairs in row-major
 * order of {16, 32, 64} x {8, 16, 32}, then the proxy-kernel times in the same order, then the
 * ID-phase times for 128 and 256 QR threads.  Defaults without a call: 32, 16, 32, 16, 256.
 * Synchronous.  Errors: those of wsbm_create / wsbm_factor (the shapes are then unchanged). */
int wsbm_autotune_build(const wsbm_geom* g, const wsbm_params* p, int32_t* out, double* ms,
                        void* stream);
/* The shapes in use on the current device: out[0..4] as wsbm_autotune's, out[5..9] as
 * wsbm_autotune_build's, out[10] = 1 once wsbm_autotune ran on this device, out[11] = 1 once
 * wsbm_autotune_build did (or the flags last given to wsbm_tuning_set), out[12] the smallest
 * dense root order whose solves with 4 or more right-hand sides run as block solves on the
 * tensor cores (default 1024).  out: 13 int32.  Errors: INVALID_ARG (out NULL). */
int wsbm_tuning(int32_t* out);
/* Sets the shapes of the current device without timing (e.g. the result of an earlier
 * autotune): in[0..12] in the order of wsbm_tuning, each among its documented candidates
 * (raster group 1..64; box panel width 8..64, a multiple of 8; grids 1..64 CTAs per SM; flags
 * 0 or 1; root order >= 1).  A solve plan already built keeps the shapes it was built with.
 * Errors: INVALID_ARG, CUDA (no device). */
int wsbm_tuning_set(const int32_t* in);

/* ---------------------------------------------------------------- gradients ----
 * Reverse-mode building blocks of shape and refractive-index gradients of a far-field loss
 * (no counterpart in the paper, which does not differentiate its solver).  With the solution x
 * of A x = b and multipliers lam of A^T lam = v:
 *   dL/ds = Re(conj(gF) . dF/ds) + Re(lam^T db/ds) - Re(lam^T (dA/ds) x)
 * for every input s.  Node gradients are device doubles laid out as six N-blocks
 * [x | y | nx | ny | w | kappa]; outputs are overwritten; all calls are asynchronous on
 * `stream` (a cudaStream_t, NULL = default stream).  Errors: INVALID_ARG, OOM, CUDA. */

/* grad = Re(lam^T (dA/ds) x) for every node input s of the Nystrom matrix of eq. (weakly_bm)
 * (dense: every node pair, O(N^2) work), gphys[0] = Re(lam^T (dA/dk1) x),
 * gphys[1] = Re(lam^T (dA/deps1) x).  lam, x: device complex128 2N (paper order: lam by
 * equation, x by unknown).  Scratch: about 6 N x (2 .. 8 waves of CTAs) doubles from the
 * library's allocator (wsbm_set_allocator) on `stream`. */
int wsbm_entries_vjp(const wsbm_geom* g, const wsbm_params* p, const void* lam, const void* x,
                     double* grad, double* gphys, void* stream);

/* grad = Re(sum_a lam_a^T db_a/ds) for plane-wave right-hand sides at nang angles (device
 * doubles); lam: device complex128 2N x nang (paper order).  Only x, y, nx, ny are nonzero. */
int wsbm_rhs_planewave_vjp(const wsbm_geom* g, const wsbm_params* p, const double* angles,
                           int32_t nang, const void* lam, double* grad, void* stream);

/* For far fields F = C [u; q] (the formula of wsbm_farfield) and gF = dL/dRe F + i dL/dIm F
 * (device complex128 nang x nrhs): v = C^T conj(gF) (device complex128 2N x nrhs, paper order)
 * and grad = Re(sum conj(gF) dF/ds) at fixed u, q (device complex128 N x nrhs each). */
int wsbm_farfield_vjp(const wsbm_geom* g, const wsbm_params* p, const void* u, const void* q,
                      int32_t nrhs, const double* angles, int32_t nang, const void* gF, void* v,
                      double* grad, void* stream);

/* Nodes of the curve r(t) = 1 + sum_{j=1..M} a_j cos(jt) + b_j sin(jt), gamma = r (cos t, sin t),
 * at t_i = 2 pi i / N: positions, outward unit normals, trapezoidal weights (2 pi/N)|gamma'|
 * and curvature.  a, b: device M doubles; outputs: device N doubles each. */
int wsbm_curve_fourier(int32_t M, int64_t N, const double* a, const double* b, double* x,
                       double* y, double* nx, double* ny, double* w, double* kappa, void* stream);

/* gcoef (device, 2M doubles: a_1..a_M, b_1..b_M) = the coefficient gradient of a loss whose
 * node gradient (six N-blocks as above) is grad. */
int wsbm_curve_fourier_vjp(int32_t M, int64_t N, const double* a, const double* b,
                           const double* grad, double* gcoef, void* stream);

/* Static name of an error code. */
const char* wsbm_strerror(int code);

/* The work space of wsbm_factor, wsbm_batch_factor and the transposed solve comes from a
 * memory pool per device that keeps up to a quarter of the device memory (at most 48 GB)
 * mapped between calls, so that repeated builds do not map it again.  This call returns every
 * cached, unused byte of those pools to the device.  WSBM_OK or WSBM_ERR_CUDA. */
int wsbm_trim_memory(void);

#ifdef __cplusplus
}
#endif
#endif /* WSBM_HSS_H */
