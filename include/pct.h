/*
 * pct.h -- C ABI of the GB300 proton-CT reconstruction library (libpct.so).
 *
 * The library computes the hot path of arXiv 1707.05014: for every proton
 * history it estimates the most-likely path (MLP) from the measured entry and
 * exit position and direction (Sec. 2), turns it into the sparse row a_i of
 * A x = b (voxel indices and chord lengths, Sec. 2), and runs the DROP
 * block-iterative row-projection solve over the relative stopping power x
 * (Sec. 2.1, Fig. 1). Rows are recomputed on the GPU in every sweep and never
 * stored.
 *
 * Conventions (all calls):
 *   - Every function returns a pct_status (PCT_OK = 0, errors < 0); no C++
 *     exception crosses the ABI. pct_last_error() returns a thread-local text
 *     for the last failing call of the calling thread.
 *   - Geometry: the grid is centred at the origin, voxel j = ix + nx*(iy +
 *     ny*iz). The gantry angle phi rotates about z: beam direction
 *     d = (cos phi, sin phi, 0), lateral axis e_t = (-sin phi, cos phi, 0),
 *     vertical e_v = (0, 0, 1). Measurement planes at depth u = -R and +R,
 *     R = min(nx*hx, ny*hy)/2. Lengths in mm, slopes dimensionless.
 *   - Device work is queued on the context's stream (pct_set_stream); calls
 *     return before it finishes unless stated. Errors raised by a kernel
 *     surface on the next synchronising call (pct_sync, pct_get_rsp to host).
 *   - The context owns every device buffer it allocates (cudaMalloc on the
 *     context's device); pct_destroy frees them.
 */
#ifndef PCT_H
#define PCT_H

#include <stdint.h>

#if defined(__GNUC__)
#define PCT_API __attribute__((visibility("default")))
#else
#define PCT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef int pct_status;
#define PCT_OK 0
#define PCT_ERR_INVALID_ARG (-1)  /* bad pointer, size or option                 */
#define PCT_ERR_INVALID_DATA (-2) /* a history record failed validation          */
#define PCT_ERR_NO_MEMORY (-3)    /* device or host allocation failed            */
#define PCT_ERR_CUDA (-4)         /* a CUDA runtime call or kernel failed        */
#define PCT_ERR_CAPACITY (-5)     /* caller buffer too small (see *needed)      */
#define PCT_ERR_TIMEOUT (-6)      /* a bounded device-side wait ran out          */
#define PCT_ERR_STATE (-7)        /* call out of order (e.g. iterate before load) */

/* Voxel grid: nx*ny*nz voxels of hx*hy*hz mm (Sec. 2: the RSP is sought on a
 * box of M voxels). Each of nx, ny, nz must lie in [1, 512]. */
typedef struct pct_grid {
  int32_t nx, ny, nz;
  double hx, hy, hz;
} pct_grid;

/* Solver options (Sec. 2.1: user-determined number of blocks; the number of
 * iterations is passed to pct_iterate). */
typedef struct pct_config {
  int32_t n_blocks;         /* DROP blocks B >= 1; block b holds histories
                               [b*N/B, (b+1)*N/B) in load order               */
  float lambda;             /* relaxation, 0 < lambda < 2 (default 1)         */
  double node_step_mm;      /* MLP node spacing request; <= 0: min(h)/2        */
  int32_t flags;            /* PCT_FLAG_*                                      */
  float clamp_min;          /* lower clamp of x after each block (with flag)   */
  int32_t threads_per_proton; /* lanes per history in the fused kernel and the
                               row export: 1 (0 = 1) or 2, 4, 8, 16, 32 (the group
                               walk: the lanes split the history's MLP
                               segments; same runs, in the same order). With an
                               object hull the one-lane kernels run.          */
  int32_t cta_threads;      /* threads per CTA of the load-time count kernel;
                             * 0 = 128 (the fused kernel always runs 128)    */
  /* Total-variation superiorization (Sec. 4.2), off when tvs_beta0 <= 0:
   * before every DROP block (with PCT_FLAG_CARP: before every CARP iteration)
   * x is perturbed once along -grad TV_eps(x) / rms, with step
   * tvs_beta0 * tvs_alpha^l (l counts every trial of the run), keeping the
   * first of up to tvs_tries trials that does not raise TV_eps. TV_eps sums
   * sqrt(dx^2 + dy^2 + dz^2 + eps^2) over forward differences. */
  float tvs_beta0;          /* step in RSP units, e.g. 0.02                     */
  float tvs_alpha;          /* step decay per trial; <= 0: 0.99                 */
  float tvs_eps;            /* TV smoothing; <= 0: 1e-4                         */
  int32_t tvs_tries;        /* trials per perturbation; <= 0: 4                 */
  int32_t carp_strings;     /* PCT_FLAG_CARP: number of strings S; string s holds
                               blocks [s B/S, (s+1) B/S); <= 0 or > B: one block
                               per string                                      */
} pct_config;

#define PCT_FLAG_CLAMP 1    /* x_j = max(x_j, clamp_min) after each block      */
#define PCT_FLAG_NO_KAHAN 2 /* plain instead of compensated a_i.x (precision study) */
#define PCT_FLAG_PROFILE 4  /* record CUDA events around every fused launch
                               (read with pct_last_sweep_times)               */
#define PCT_FLAG_CARP 16    /* pct_iterate runs CARP (Sec. 2.2, Fig. 2) instead of
                               DROP: carp_strings strings of consecutive blocks;
                               every string sweeps its blocks with the DROP
                               block update on a copy of the same starting x
                               (the blocked form of a string's row sweep), and
                               x becomes the component average of the string
                               results over the strings touching each voxel.
                               Not accepted by pct_batch_create.             */
#define PCT_FLAG_NO_SORT 8  /* keep each block in load order (default: each
                               block is stored ordered by gantry angle and by
                               the lateral position of the history's MLP at the
                               quarter points of the slab, which keeps the
                               lanes of a warp on nearly the same path;
                               membership of the blocks, and so the result, is
                               unchanged up to floating-point summation order) */

/* One history per index: entry state at u = -R, exit state at u = +R, the
 * WEPL b_i (mm) and the gantry angle as cos/sin (Sec. 2: each proton is
 * measured by its position and direction before and after the object, and
 * by its WEPL). Eleven float arrays of n elements each (structure of
 * arrays). */
typedef struct pct_histories {
  int64_t n;
  const float *t0, *v0, *st0, *sv0; /* lateral / vertical position and slope at u = -R */
  const float *t2, *v2, *st2, *sv2; /* the same at u = +R                            */
  const float *wepl;                /* water-equivalent path length, mm              */
  const float *cphi, *sphi;         /* cos and sin of the gantry angle               */
} pct_histories;

/* pct_load_histories flags */
#define PCT_LOAD_HOST 0          /* arrays are host memory; copied to the device   */
#define PCT_LOAD_DEVICE_COPY 1   /* device arrays; copied into context storage     */
#define PCT_LOAD_DEVICE_BORROW 2 /* device arrays used in place; the caller keeps
                                    them alive and unchanged until pct_destroy or
                                    the next load                                 */

typedef struct pct_ctx pct_ctx;

/* Create a context for one grid on CUDA device `device`. Builds the FP64 MLP
 * coefficient table on the GPU (Sec. 2, MLP of Schulte et al. 2008: first rows
 * of (S1^-1 + R1^T S2^-1 R1)^-1 S1^-1 R0 and ... R1^T S2^-1 per node).
 * *out receives the context; on error *out is NULL. */
PCT_API pct_status pct_create(pct_ctx **out, const pct_grid *grid, const pct_config *cfg, int device);

/* Free all device buffers, graphs and the stream owned by ctx. NULL is a no-op. */
PCT_API pct_status pct_destroy(pct_ctx *ctx);

/* Use `stream` (a cudaStream_t, or the special handles cudaStreamLegacy /
 * cudaStreamPerThread; NULL = the context's own non-blocking stream) for all
 * later device work of ctx. The caller keeps the stream alive. Switching to a
 * different stream first waits for the work queued on the current one. */
PCT_API pct_status pct_set_stream(pct_ctx *ctx, void *stream);

/* Derived geometry: plane half-distance R (mm), node spacing du (mm),
 * interior node count K+1 (nodes k = 0..K at u = -R + k du), extension nodes
 * per side E, voxel count M. Any pointer may be NULL. */
PCT_API pct_status pct_geometry(const pct_ctx *ctx, double *R, double *du, int32_t *K, int32_t *E, int64_t *M);

/* Copy the FP64 MLP table, (K+1) x 4 doubles (c1, c2 [mm], c3, c4 [mm]; node
 * k lateral position t_k = c1 t0 + c2 st0 + c3 t2 + c4 st2), to `out` (host
 * memory if to_device == 0, else device memory). Synchronises on host copies. */
PCT_API pct_status pct_mlp_table(pct_ctx *ctx, double *out, int to_device);

/* Load N histories (Sec. 2). Validates every record on the GPU: finite
 * values, |slope| < 0.5, |t|,|v| within the position limit (half the grid's
 * 3-D diagonal plus R), wepl >= 0, |cos^2 + sin^2 - 1| < 1e-3. On failure
 * returns PCT_ERR_INVALID_DATA and the first bad index in *first_bad (may be
 * NULL; -1 when all are valid). The records are copied into context storage
 * (ordered within each block unless PCT_FLAG_NO_SORT; PCT_LOAD_DEVICE_BORROW
 * avoids the copy only with PCT_FLAG_NO_SORT). Resets x to 0. Each block's
 * run counts s_j (DROP's diagonal weights) are formed by the first
 * pct_iterate sweep after the load, which counts each block's runs as it
 * updates it (pct_batch_create counts them itself if no sweep has). The
 * context keeps its record buffers across loads and grows them when a load
 * needs more. Host records (PCT_LOAD_HOST) pass through two staging slots of
 * the largest block's 44 bytes per history, the next block's copy overlapping
 * the current block's ordering; every copy has finished when the call
 * returns, also on error, so the caller may free the host arrays then. Each
 * block must hold fewer than 2^32 histories. Synchronises. */
PCT_API pct_status pct_load_histories(pct_ctx *ctx, const pct_histories *h, int flags, int64_t *first_bad);

/* Rows a_i of histories [first, first+count) of the loaded set (indices in
 * load order), in CSR form,
 * all DEVICE pointers: row_ptr (count+1 int64), vox (cap int32 voxel
 * indices), len (cap float chord lengths in mm, in path order; a run is a
 * maximal stretch in one voxel, zero-length runs never appear). `nodes`
 * (optional, may be NULL) receives count x (K+1) x 3 int32: the path's nodes
 * k = 0..K between the planes (the MLP nodes; with a hull, the ray nodes
 * outside it) in Q20 fixed point grid units. *needed receives the total number of
 * runs; if it exceeds cap, returns PCT_ERR_CAPACITY and writes no runs.
 * Synchronises. */
PCT_API pct_status pct_mlp_rows(pct_ctx *ctx, int64_t first, int64_t count, int64_t *row_ptr, int32_t *vox, float *len,
                        int64_t cap, int32_t *nodes, int64_t *needed);

/* Object hull of the MLP. Sec. 2 cites the MLP of Schulte et al. 2008, which
 * estimates the path inside the object and takes it straight outside. With a
 * hull set, history i's path is its entry ray up to node iin, the MLP of the
 * water layer between nodes iin and iout, then its exit ray. The layer has
 * n = iout - iin node intervals; its FP64 table is built on the GPU for every
 * n and rounded to FP32. The MLP starts from the ray positions at the hull
 * and the measured slopes. iin is the first node k in [0, K] whose entry-ray
 * point (t0 + st0 k du, at depth u_k) lies in a hull voxel; iout is the last
 * node whose exit-ray point (t2 + st2 (k - K) du) does. A history with no such
 * pair (iout <= iin) keeps the plane-to-plane MLP, like every history without
 * a hull. The same fixed single-precision operation order as without a hull
 * defines the rows bit for bit.
 *
 * pct_set_hull: mask = M bytes, nonzero = inside the object (device memory
 * if on_device, else host); NULL removes the hull. Recomputes the ranges of
 * loaded histories (their block weights are recounted by the next sweep);
 * later loads use the hull too. Synchronises. Contexts with a hull are not
 * accepted by pct_batch_create. */
PCT_API pct_status pct_set_hull(pct_ctx *ctx, const uint8_t *mask, int on_device);

/* Space-carved hull from the loaded histories: every voxel on the
 * plane-to-plane row of a history with wepl <= wepl_max crossed only air and
 * is outside; the hull is every other voxel, grown by `dilate` steps of the
 * 6-neighbourhood (dilate >= 0; 1 restores boundary voxels that grazing
 * histories carved). Then as pct_set_hull. Allocates 2 M bytes of scratch
 * for the call. Synchronises. */
PCT_API pct_status pct_carve_hull(pct_ctx *ctx, float wepl_max, int32_t dilate);

/* Copy the current hull mask (M bytes) to host `out`. PCT_ERR_STATE without
 * a hull. Synchronises. */
PCT_API pct_status pct_get_hull(pct_ctx *ctx, uint8_t *out);

/* Hull nodes (iin, iout) of histories [first, first+count) in load order,
 * to host `out` (2 x count int32). PCT_ERR_STATE without a hull or
 * histories. Synchronises. */
PCT_API pct_status pct_hull_ranges(pct_ctx *ctx, int64_t first, int64_t count, int32_t *out);

/* FP64 MLP table of a layer of n node intervals (1 <= n <= K; n = K is the
 * slab between the planes, equal to pct_mlp_table), (n+1) x 4 doubles for
 * nodes m = 0..n from the layer entry, computed on the GPU, to host `out`.
 * Synchronises. */
PCT_API pct_status pct_mlp_table_n(pct_ctx *ctx, int32_t n, double *out);

/* Forward projection y[p] = a_i.x for histories i = first+p (load order) of
 * the loaded set, with the current x and the fused kernel's arithmetic
 * (compensated unless PCT_FLAG_NO_KAHAN). y: DEVICE, count floats.
 * Asynchronous. (Sec. 2: a_i.x is the model WEPL of history i.) */
PCT_API pct_status pct_project(pct_ctx *ctx, int64_t first, int64_t count, float *y);

/* Data residual sum_i (b_i - a_i.x)^2 with the current x over every
 * stride-th stored history (stride 1: all of them; a larger stride gives an
 * unbiased sample, since every block spans all angles), accumulated in
 * double; written to host *sum_sq. Synchronises. */
PCT_API pct_status pct_residual(pct_ctx *ctx, int64_t stride, double *sum_sq);

/* Run counts s_j of DROP block `block` as float (exact integers), M values,
 * written to DEVICE memory `out`. */
PCT_API pct_status pct_block_counts(pct_ctx *ctx, int32_t block, float *out);

/* Form the DROP weights S_b^-1 = diag(1/s_j) of every block of the loaded
 * histories now (Sec. 2.1: the update of block b divides by its run counts).
 * Otherwise the first pct_iterate after a load forms them while it sweeps
 * (cheaper: the counting rides on the sweep's own walk, where this call walks
 * every history once more); a caller that times sweeps separately from this
 * set-up calls it first. No-op
 * if they are formed already. PCT_ERR_STATE without loaded histories.
 * Synchronises. */
PCT_API pct_status pct_block_weights(pct_ctx *ctx);

/* Set the initial image x0 (M floats; device memory if on_device, else host).
 * Does not reset the TVS trial counter (pct_load_histories does). */
PCT_API pct_status pct_set_x0(pct_ctx *ctx, const float *x0, int on_device);

/* Run n_sweeps DROP iterations (Sec. 2.1, Fig. 1): for each block b in
 * order, every history i of b contributes lambda (b_i - a_i.x)/|a_i|^2 a_i
 * (a_i recomputed from the MLP, a_i.x compensated), then
 * x_j += delta_j / s_j. Asynchronous on the context stream; one CUDA graph
 * per sweep. The first sweep after a load also forms the block weights
 * unless pct_block_weights did: with one lane per history and no hull, CARP
 * or TVS it adds each run's update and count as one float pair; it then waits
 * for that sweep, and if a voxel collected 2^24 or more runs of one block
 * (where a float count is no longer exact) it undoes the sweep, forms the
 * weights with integer counts and sweeps again. It allocates 12 bytes per
 * voxel for this on its first use. */
PCT_API pct_status pct_iterate(pct_ctx *ctx, int32_t n_sweeps);

/* ---- A DROP block shared by several processes (Sec. 1 and Sec. 3.1: the
 * histories are distributed over processors, each of which works on its own
 * part). Each rank's context holds its share of the histories, B blocks over
 * them, so that global block b is the union of the ranks' blocks b. One block
 * update is then
 *   pct_block_partial on every rank -> all-reduce(sum) of delta and counts
 *   -> pct_block_apply with the sums on every rank,
 * which gives every rank the x of one DROP block over the union (Sec. 2.1),
 * up to floating-point summation order. The run counts of a block do not
 * change between sweeps, so their sum can be reduced once and kept. ---- */

/* This rank's part of block `block` with the context's current x:
 * delta_out[j] = lambda sum_i a_ij (b_i - a_i.x) / |a_i|^2 over the block's
 * histories in this context (DEVICE, M floats, overwritten), and, if
 * counts_out is not NULL, the block's run counts s_j as float (DEVICE, M
 * floats, overwritten). x is not changed. Asynchronous. */
PCT_API pct_status pct_block_partial(pct_ctx *ctx, int32_t block, float *delta_out, float *counts_out);

/* x_j += delta_j / counts_j where counts_j > 0 (voxels no rank's histories
 * touch are unchanged), then the PCT_FLAG_CLAMP clamp if set: the DROP block
 * update from the sums of every rank's pct_block_partial output (DEVICE
 * arrays of M floats, read only). Asynchronous. */
PCT_API pct_status pct_block_apply(pct_ctx *ctx, const float *delta, const float *counts);

/* Testing hook (process-wide): with k >= 1, the k-th device allocation that a
 * context makes from now on fails as if the device had no memory left (the
 * call reports PCT_ERR_NO_MEMORY); later allocations succeed again. k <= 0
 * disarms it. */
PCT_API void pct_debug_fail_alloc(int64_t k);

/* With PCT_FLAG_PROFILE: wait for the queued work, then write the device
 * time (ms) of each block's fused MLP + projection kernel and of each block's
 * apply kernel in the most recent sweep to fused_ms[b] and apply_ms[b]
 * (n_blocks entries each, host memory; either may be NULL). Returns
 * PCT_ERR_STATE without the flag or before the first sweep. */
PCT_API pct_status pct_last_sweep_times(pct_ctx *ctx, float *fused_ms, float *apply_ms);

/* Copy x (M floats) to `out` (host memory if to_device == 0, else device).
 * Synchronises for host copies and reports device-side errors. */
PCT_API pct_status pct_get_rsp(pct_ctx *ctx, float *out, int to_device);

/* Wait for all queued work of ctx; report device-side errors. */
PCT_API pct_status pct_sync(pct_ctx *ctx);

/* Kernel launches queued by this context since creation (for accounting). */
PCT_API int64_t pct_launch_count(const pct_ctx *ctx);

/* ---- Batched reconstructions (no counterpart in the paper: a system
 * feature). Several loaded contexts on one device, of uneven size, advance
 * together. Two modes, chosen by pct_batch_autotune (or set in the config):
 * PCT_BATCH_PERSISTENT -- ONE persistent launch per call: CTAs take work items
 * (a chunk of one block's histories, or a voxel tile of one block update) from
 * a fixed block-major queue over all reconstructions; per-reconstruction
 * counters with bounded waits keep each reconstruction's DROP stages in order
 * (Sec. 2.1, Fig. 1: block b starts from the result of block b-1).
 * PCT_BATCH_GRAPH_BRANCHES -- each reconstruction's stages as a chain of the
 * per-block kernels; the chains run as parallel branches of one CUDA graph.
 * Either way each reconstruction's result equals its own pct_iterate up to
 * floating-point summation order. ---- */

typedef struct pct_batch pct_batch;

#define PCT_BATCH_PERSISTENT 1     /* one persistent launch per call (work queue)      */
#define PCT_BATCH_GRAPH_BRANCHES 2 /* each reconstruction a chain of per-block kernels;
                                      the chains are parallel branches of one graph    */

typedef struct pct_batch_config {
  int32_t mode;                   /* PCT_BATCH_*; other values: PCT_BATCH_GRAPH_BRANCHES */
  int32_t branches;               /* graph-branch mode: concurrent branches (1..8);
                                     <= 0: min(8, n)                                    */
  int32_t chunk;                  /* histories per work item; <= 0: 4096                   */
  int32_t ctas_per_sm;            /* resident CTAs per SM; <= 0 or above the occupancy
                                     limit: the occupancy limit                            */
  int32_t apply_tiles;            /* voxel tiles per block update; <= 0: one per 32768
                                     voxels, at most 64                                    */
  double wait_limit_s;            /* bound on every wait inside the launch; <= 0: 2 s       */
  int32_t debug_unreachable_wait; /* test hook: non-zero makes every block-update wait
                                     unreachable, so the bound runs out and the call
                                     reports PCT_ERR_TIMEOUT (the GPU stays usable)        */
  int32_t lanes;                  /* graph-branch mode: lanes per history of the fused
                                     kernels (1, 2, 4, 8, 16 or 32, as threads_per_proton);
                                     <= 0: each context's own threads_per_proton. The
                                     persistent kernel always takes one lane per history  */
} pct_batch_config;

/* Group n loaded contexts (same device) for batched sweeps. cfg may be NULL
 * (defaults). The contexts must outlive the batch and must not be reloaded
 * or given a hull while it exists (pct_batch_iterate and pct_batch_autotune
 * then return PCT_ERR_STATE). DROP contexts without TVS only. */
PCT_API pct_status pct_batch_create(pct_batch **out, pct_ctx *const *ctxs, int32_t n, const pct_batch_config *cfg);
PCT_API pct_status pct_batch_destroy(pct_batch *batch);

/* n_sweeps DROP sweeps of every reconstruction in one persistent launch
 * (captured once per n_sweeps as a CUDA graph), queued on `stream` (a
 * cudaStream_t; NULL = the batch's own stream). Asynchronous; first waits
 * on the host for the work of any context whose stream is not `stream`. */
PCT_API pct_status pct_batch_iterate(pct_batch *batch, int32_t n_sweeps, void *stream);

/* Wait for the batch's work on `stream` (NULL = own stream); returns
 * PCT_ERR_TIMEOUT if a bounded wait ran out: the blocks not applied in that
 * call are dropped (update buffers cleared), x stays finite and the contexts
 * stay usable. */
PCT_API pct_status pct_batch_sync(pct_batch *batch, void *stream);

/* Time one sweep for each candidate -- graph branches with 1, 4 or 8
 * branches; persistent with chunk in {2048, 4096, 8192} and CTAs per SM in
 * {occupancy limit, limit - 1, limit / 2} -- keep the fastest, and restore
 * every reconstruction's x. Writes the chosen configuration and its sweep
 * time (ms). */
PCT_API pct_status pct_batch_autotune(pct_batch *batch, pct_batch_config *chosen, float *best_ms);

/* Kernel launches made by the batch (for accounting). */
PCT_API int64_t pct_batch_launch_count(const pct_batch *batch);

/* ---- Learned warm start (no counterpart in the paper: a system feature).
 * A 3-D U-Net f (4 levels, 16/32/64/128 channels, 3x3x3 convolutions,
 * stride-2 down, nearest-x2-up + conv, additive skips, ReLU) maps the image
 * x1 after the first DROP sweep to x0 = x1 + f(x1), a starting image closer to
 * the converged reconstruction. BF16 weights and activations, FP32
 * accumulation on the tensor cores, FP32 master weights and Adam. Volumes are
 * nz x ny x nx floats in the reconstruction's voxel order (x fastest); each
 * dimension a multiple of 8. ---- */
typedef struct pct_net pct_net;

/* Create a network for nz x ny x nx volumes; He-normal weights from `seed`. */
PCT_API pct_status pct_net_create(pct_net **out, int32_t nz, int32_t ny, int32_t nx, uint64_t seed, int device);
PCT_API pct_status pct_net_destroy(pct_net *net);

/* Number of FP32 parameters (15 layers: 27*Cin*Cout weights [tap][ci][co]
 * then Cout biases each; channel counts padded to >= 16). */
PCT_API int64_t pct_net_param_count(const pct_net *net);
/* Copy the FP32 master parameters to / from HOST memory. */
PCT_API pct_status pct_net_get_params(pct_net *net, float *out);
PCT_API pct_status pct_net_set_params(pct_net *net, const float *in);

/* x0 = x1 + f(x1); x1, x0 DEVICE arrays. Asynchronous on `stream` (NULL =
 * the network's own stream). */
PCT_API pct_status pct_net_forward(pct_net *net, const float *x1, float *x0, void *stream);

/* Forward + backward of the L1 loss mean|x1 + f(x1) - target| without an
 * update: writes the loss (host *loss) and dLoss/dparams (HOST grads, may be
 * NULL). x0_scratch: DEVICE array of one volume. Synchronises. */
PCT_API pct_status pct_net_gradients(pct_net *net, const float *x1, const float *target, float *x0_scratch,
                                     float *grads, double *loss);

/* One Adam step (beta 0.9 / 0.999, eps 1e-8) on the L1 loss of one pair.
 * loss may be NULL (then no synchronisation). */
PCT_API pct_status pct_net_train_step(pct_net *net, const float *x1, const float *target, float *x0_scratch,
                                      float lr, double *loss, void *stream);

/* One layer of the network on the caller's DEVICE data, through the same
 * kernels as pct_net_forward / pct_net_gradients (for checking them layer by
 * layer). Layer l (0..14) has Cin, Cout channels and input / output grids at
 * the levels of the topology above (level 0: nz x ny x nx, each further level
 * halves every dimension); activations and gradients are BF16 (uint16 bit
 * patterns), channels last: [voxel][channel]. Weights and biases are the
 * net's current parameters.
 *   PCT_NET_FORWARD (l = 0..13): out[vox_out][Cout] = bf16(relu(conv(in) +
 *     bias + skip)); skip is the [vox_out][Cout] input of the additive skip of
 *     layers 8, 10 and 12, NULL for the others.
 *   PCT_NET_DATA_GRAD (l = 1..14): out[vox_in][Cin] = bf16((conv^T(dy) + add)
 *     * [mask > 0]); dy: [vox_out][Cout] gradient of layer l's pre-activation;
 *     mask: layer l-1's stored activation; add: the skip gradient into layer
 *     l-1's output (may be NULL; must be NULL for the up-convolutions 8, 10, 12).
 *   PCT_NET_WEIGHT_GRAD (l = 0..14): out = float[27*Cin*Cout + Cout], dW
 *     [tap][ci][co] then db, from the layer's input `in` and `dy` (zeroed
 *     first).
 * Asynchronous on `stream` (NULL = the network's own stream). */
/* Channels (padded) and grid levels of layer l's input and output. */
PCT_API pct_status pct_net_layer_shape(const pct_net *net, int32_t layer, int32_t *cin, int32_t *cout,
                                       int32_t *in_level, int32_t *out_level);
#define PCT_NET_FORWARD 0
#define PCT_NET_DATA_GRAD 1
#define PCT_NET_WEIGHT_GRAD 2
PCT_API pct_status pct_net_layer(pct_net *net, int32_t layer, int32_t op, const void *in, const void *skip,
                                 const void *dy, const void *mask, const void *add, void *out, void *stream);

/* One DROP block update that allocates no device or host memory, for callers
 * that cannot allocate once they run (services that reserve all GPU memory
 * at start-up for a fixed plan, plugins whose host application owns every
 * device allocation). The paper has no counterpart; it is the same update as
 * one block of pct_iterate without a context.
 *
 * h: the histories of ONE block, DEVICE pointers, used in place in the given
 * order. x: DEVICE array of nx*ny*nz floats, read and updated in place:
 * x_j += lambda/s_j * sum_i a_ij (b_i - a_i.x)/|a_i|^2. cfg: lambda,
 * node_step_mm, flags (PCT_FLAG_CLAMP, PCT_FLAG_NO_KAHAN) and clamp_min are
 * used; n_blocks, threads_per_proton, cta_threads and the TVS fields are
 * ignored. stream: a
 * cudaStream_t (NULL = the legacy default stream).
 *
 * Scratch: a fixed 16.1 MiB device array inside the library (its update
 * accumulator, run counts and MLP table) that every GPU loading the library
 * holds until exit. Grids above 2,097,152 voxels return PCT_ERR_CAPACITY.
 * Every call looks up that array's device address in the context current on
 * the calling thread (the current device's), so the call follows a reset or
 * a change of context. Every call on a device uses the same array and clears
 * what must start at zero, so calls that overlap on the GPU (different
 * streams or threads, same device) race.
 * Validates the records (as pct_load_histories does) and synchronises the
 * stream once to report PCT_ERR_INVALID_DATA; the update itself is queued
 * asynchronously. No cudaMalloc, cudaFree or other allocating call is made. */
PCT_API pct_status pct_drop_block_noalloc(const pct_grid *grid, const pct_config *cfg, const pct_histories *h,
                                          float *x, void *stream);

/* Text for the last error of the calling thread ("" if none). */
PCT_API const char *pct_last_error(void);

/* Measured roofs of the resources the fused kernel uses (Sec. 2 / 2.1 give no
 * hardware model; these are this library's own microbenchmarks). Each rate is
 * the best of five timed launches (CUDA events) after a warm-up, with
 * 8 CTAs of 256 threads per SM:
 *   l2_red_per_s          float atomicAdd at random addresses of an
 *                         array_bytes array (default 8 MB, L2-resident);
 *   l2_red_coherent_per_s the same with the 32 lanes of a warp on one
 *                         128-byte line per step;
 *   l2_gather_per_s       random 4-byte loads from the same array;
 *   alu_ops_per_s         integer shift/xor/add chains (4 source operations
 *                         per step, 8 independent chains per thread);
 *   fma_ops_per_s         FP32 FMA chains (8 independent chains per thread).
 * l2_bytes and sms come from cudaDeviceProp. Allocates array_bytes (rounded
 * down to a power of two, 4 KB .. 8 GB; <= 0: 8 MB) for the call, on
 * `device`. Synchronises. */
typedef struct pct_roofs {
  double l2_red_per_s, l2_red_coherent_per_s, l2_gather_per_s, alu_ops_per_s, fma_ops_per_s;
  int64_t array_bytes, l2_bytes;
  int32_t sms;
} pct_roofs;
PCT_API pct_status pct_measure_roofs(int device, int64_t array_bytes, pct_roofs *out);

#ifdef __cplusplus
}
#endif

#endif /* PCT_H */
