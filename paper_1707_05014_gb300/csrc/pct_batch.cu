// Batched persistent DROP: several independent reconstructions of uneven size
// in one launch per call (pct_batch_*, declared in include/pct.h).
//
// Each reconstruction r runs the DROP stages of Sec. 2.1 / Fig. 1 in order:
// for every sweep and block b, the block's histories contribute to delta_r,
// then x_r += delta_r / s_r. Here a fixed queue of work items, block-major
// across reconstructions, feeds a persistent grid:
//   chunk item (r, b, c)  : `chunk` histories of block b of reconstruction r
//   apply item (r, b, t)  : voxel tile t of the block update of (r, b)
// A chunk of stage (sweep, b) waits until every apply tile of the previous
// stage of r has finished; an apply tile waits until every chunk of its stage
// has finished. Both waits read monotonic per-reconstruction counters, so an
// item only ever waits for items dequeued before it, which are running on
// resident CTAs: the launch cannot deadlock. Every wait is bounded; when a
// bound runs out the kernel records PCT_ERR_TIMEOUT in a status word, every
// CTA stops taking work, and the host reports the status.
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <string>
#include <vector>

#include "pct_ctx.h"
#include "pct_drop.cuh"
#include "pct_trace.h"

namespace {

using pct::Geo;
using pct::Rec;

struct ReconDesc {
  Geo g;
  Rec rec;
  const float4* tab;
  float* x;
  float* delta;
  const float* inv_s;
  int64_t M;
  float lambda;
  int flags;
  int clamp;
  float clamp_min;
};

struct Item {
  int32_t r;      // reconstruction
  int32_t kind;   // 0 = chunk of histories, 1 = voxel tile of a block update
  int32_t block;  // DROP block
  uint32_t wait;  // counter value (within one sweep) this item waits for
  int64_t first;  // first history (chunk) or voxel (tile)
  int64_t count;
};

constexpr int kThreads = 128;

// Record pointers of a reconstruction, re-read for every history (volatile
// loads cannot be hoisted): keeping eleven pointers live across the walk
// would cost 22 registers.
__device__ __forceinline__ Rec load_rec_ptrs(const ReconDesc* R) {
  const unsigned long long* p = reinterpret_cast<const unsigned long long*>(&R->rec);
  unsigned long long v[11];
#pragma unroll
  for (int f = 0; f < 11; ++f) asm volatile("ld.global.u64 %0, [%1];" : "=l"(v[f]) : "l"(p + f));
  return Rec{(const float*)v[0], (const float*)v[1], (const float*)v[2], (const float*)v[3], (const float*)v[4],
             (const float*)v[5], (const float*)v[6], (const float*)v[7], (const float*)v[8], (const float*)v[9],
             (const float*)v[10]};
}

// The histories of one chunk item (kept out of line so that the walk gets the
// same registers as in the per-block kernel).
__device__ __noinline__ void run_chunk(const ReconDesc* __restrict__ R, int64_t first, int64_t count, float4* tab) {
  const Geo g = R->g;
  for (int k = threadIdx.x; k <= g.K; k += kThreads) tab[k] = R->tab[k];
  __syncthreads();
  float* x = R->x;
  float* delta = R->delta;
  const float lambda = R->lambda;
  const int flags = R->flags;
  if (flags & 2) {
    for (int64_t p = threadIdx.x; p < count; p += kThreads)
      pct::drop_history<true, true>(g, tab, load_rec_ptrs(R), first + p, x, delta, lambda);
  } else {
    for (int64_t p = threadIdx.x; p < count; p += kThreads)
      pct::drop_history<true, false>(g, tab, load_rec_ptrs(R), first + p, x, delta, lambda);
  }
}

__global__ void __launch_bounds__(kThreads, 6) batch_kernel(const ReconDesc* __restrict__ recs,
                                                          const Item* __restrict__ items, int64_t per_sweep,
                                                          int n_sweeps, const uint2* __restrict__ sweep_counts,
                                                          unsigned* chunk_done, unsigned* apply_done,
                                                          unsigned long long* head, int* status,
                                                          long long spin_limit, unsigned debug_extra) {
  extern __shared__ float4 tab[];
  __shared__ long long s_item;
  __shared__ int s_go;
  const long long total = per_sweep * (long long)n_sweeps;
  for (;;) {
    if (threadIdx.x == 0) {
      const long long i = (long long)atomicAdd(head, 1ull);
      int go = i < total && *(volatile int*)status == 0;
      if (go) {
        const int sweep = (int)(i / per_sweep);
        const Item it = items[i % per_sweep];
        const uint2 sc = sweep_counts[it.r];  // x: apply tiles per sweep, y: chunks per sweep
        const unsigned target = (unsigned)sweep * (it.kind == 0 ? sc.x : sc.y) + it.wait + (it.kind ? debug_extra : 0u);
        volatile unsigned* ctr = it.kind == 0 ? apply_done + it.r : chunk_done + it.r;
        long long spins = 0;
        while (*ctr < target) {
          if (*(volatile int*)status != 0) {
            go = 0;
            break;
          }
          if (++spins > spin_limit) {
            atomicCAS(status, 0, -PCT_ERR_TIMEOUT);
            go = 0;
            break;
          }
          __nanosleep(256);
        }
        __threadfence();  // acquire: the work behind the counter is visible below
      }
      s_item = i;
      s_go = go;
    }
    __syncthreads();
    const long long i = s_item;
    const int go = s_go;
    __syncthreads();  // both read before thread 0 overwrites them
    if (!go) break;
    const Item it = items[i % per_sweep];
    const ReconDesc& R = recs[it.r];
    if (it.kind == 0) {
      run_chunk(&R, it.first, it.count, tab);
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();  // release the delta contributions
        atomicAdd(chunk_done + it.r, 1u);
      }
    } else {
      const float* inv = R.inv_s + (size_t)it.block * R.M;
      for (int64_t j = it.first + threadIdx.x; j < it.first + it.count; j += kThreads)
        pct::apply_voxel<true>(R.x, R.delta, inv, j, R.clamp, R.clamp_min);
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();  // release the updated x
        atomicAdd(apply_done + it.r, 1u);
      }
    }
  }
}

}  // namespace

struct pct_batch {
  int device = 0;
  std::vector<pct_ctx*> ctx;
  std::vector<uint64_t> gen;  // each context's generation when the batch was made
  pct_batch_config cfg{};
  int n_sms = 0;
  int max_ctas_per_sm = 0;
  int max_nodes = 0;
  cudaStream_t own_stream = nullptr;
  ReconDesc* d_recs = nullptr;
  Item* d_items = nullptr;
  uint2* d_sweep_counts = nullptr;
  unsigned* d_counters = nullptr;  // chunk_done[n], apply_done[n], head (2 words), status
  int64_t per_sweep = 0;
  cudaGraphExec_t graph = nullptr;
  int graph_sweeps = -1;
  int64_t graph_launches = 0;
  float* x_save = nullptr;  // autotuning restores every x afterwards
  int64_t x_total = 0;
  int64_t launches = 0;
  std::vector<cudaStream_t> branch;  // graph-branch mode: one stream per branch
  std::vector<cudaEvent_t> join;     // [0] fork, [1..] joins
};

namespace {

#define PCT_BCK(call)                                                                     \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) return bfail(PCT_ERR_CUDA, #call, cudaGetErrorString(e_));     \
  } while (0)

pct_status bfail(pct_status code, const char* what, const char* detail = "") {
  std::string m = std::string(what) + (detail[0] ? ": " : "") + detail;
  pct::set_error_text(m.c_str());
  return code;
}

void free_plan(pct_batch* b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
  b->graph_sweeps = -1;
  cudaFree(b->d_items);
  b->d_items = nullptr;
}

// Build the work queue of one sweep for the current chunk / tile sizes.
pct_status build_plan(pct_batch* b) {
  free_plan(b);
  const int n = (int)b->ctx.size();
  const int64_t chunk = b->cfg.chunk;
  int maxB = 0;
  for (auto* c : b->ctx) maxB = std::max(maxB, c->cfg.n_blocks);
  std::vector<Item> items;
  std::vector<uint2> counts(n, make_uint2(0, 0));  // x: apply tiles, y: chunks (per sweep)
  std::vector<uint32_t> chunks_so_far(n, 0), tiles_so_far(n, 0);
  std::vector<int> tiles(n);
  for (int r = 0; r < n; ++r) {
    const int64_t M = b->ctx[r]->M;
    int t = b->cfg.apply_tiles > 0 ? b->cfg.apply_tiles : (int)std::min<int64_t>(64, (M + 32767) / 32768);
    tiles[r] = std::max(1, t);
  }
  for (int blk = 0; blk < maxB; ++blk) {
    for (int r = 0; r < n; ++r) {
      pct_ctx* c = b->ctx[r];
      if (blk >= c->cfg.n_blocks) continue;
      const int64_t lo = pct::block_first(c, blk), hi = pct::block_first(c, blk + 1);
      for (int64_t f = lo; f < hi; f += chunk) {
        Item it{r, 0, blk, tiles_so_far[r], f, std::min(chunk, hi - f)};
        items.push_back(it);
        ++chunks_so_far[r];
      }
    }
    for (int r = 0; r < n; ++r) {
      pct_ctx* c = b->ctx[r];
      if (blk >= c->cfg.n_blocks) continue;
      const int64_t M = c->M, per = (M + tiles[r] - 1) / tiles[r];
      for (int t = 0; t < tiles[r]; ++t) {
        const int64_t f = t * per;
        if (f >= M) break;
        Item it{r, 1, blk, chunks_so_far[r], f, std::min(per, M - f)};
        items.push_back(it);
        ++tiles_so_far[r];
      }
    }
  }
  for (int r = 0; r < n; ++r) counts[r] = make_uint2(tiles_so_far[r], chunks_so_far[r]);
  b->per_sweep = (int64_t)items.size();
  PCT_BCK(cudaMalloc((void**)&b->d_items, items.size() * sizeof(Item)));
  PCT_BCK(cudaMemcpy(b->d_items, items.data(), items.size() * sizeof(Item), cudaMemcpyHostToDevice));
  PCT_BCK(cudaMemcpy(b->d_sweep_counts, counts.data(), n * sizeof(uint2), cudaMemcpyHostToDevice));
  return PCT_OK;
}

pct_status enqueue(pct_batch* b, int n_sweeps, cudaStream_t s, long long spin_limit) {
  const int n = (int)b->ctx.size();
  unsigned* chunk_done = b->d_counters;
  unsigned* apply_done = b->d_counters + n;
  unsigned long long* head = (unsigned long long*)(b->d_counters + 2 * n);  // 8-byte aligned: 2n words
  int* status = (int*)(head + 1);
  const size_t words = 2 * n + 3;
  PCT_BCK(cudaMemsetAsync(b->d_counters, 0, words * sizeof(unsigned), s));
  const int ctas = b->n_sms * b->cfg.ctas_per_sm;
  const size_t smem = (size_t)b->max_nodes * sizeof(float4);
  batch_kernel<<<ctas, kThreads, smem, s>>>(b->d_recs, b->d_items, b->per_sweep, n_sweeps, b->d_sweep_counts,
                                            chunk_done, apply_done, head, status, spin_limit,
                                            b->cfg.debug_unreachable_wait ? 1u : 0u);
  PCT_BCK(cudaGetLastError());
  b->launches += 1;
  return PCT_OK;
}

// Lanes per history of a context's fused kernels in graph-branch mode.
int lanes_of(const pct_batch* b, const pct_ctx* c) { return b->cfg.lanes > 0 ? b->cfg.lanes : c->cfg.threads_per_proton; }

// The group kernels' shared-memory limit for every context's table, set
// outside stream capture.
pct_status prepare_lanes(pct_batch* b) {
  for (auto* c : b->ctx) {
    const int T = lanes_of(b, c);
    if (T > 1) PCT_BCK(pct::prepare_drop_group(T, c->K));
  }
  return PCT_OK;
}

// Graph-branch mode: each reconstruction's stages as a chain of the per-block
// kernels (fused, then apply, per block), chains spread over branch streams
// that fork from and join into s, so that independent chains overlap.
pct_status enqueue_branches(pct_batch* b, int n_sweeps, cudaStream_t s) {
  const int nb = std::max(1, std::min((int)b->branch.size(), b->cfg.branches > 0 ? b->cfg.branches : 8));
  PCT_BCK(cudaEventRecord(b->join[0], s));
  for (int k = 0; k < nb; ++k) PCT_BCK(cudaStreamWaitEvent(b->branch[k], b->join[0], 0));
  for (size_t r = 0; r < b->ctx.size(); ++r) {
    pct_ctx* c = b->ctx[r];
    cudaStream_t bs = b->branch[r % nb];
    const int clamp = (c->cfg.flags & PCT_FLAG_CLAMP) != 0;
    for (int sw = 0; sw < n_sweeps; ++sw)
      for (int blk = 0; blk < c->cfg.n_blocks; ++blk) {
        const int64_t lo = pct::block_first(c, blk), hi = pct::block_first(c, blk + 1);
        PCT_BCK(pct::launch_drop_fused(c->geo, c->rec, c->tab32, pct::Hull{}, lo, hi - lo, c->x, c->delta,
                                       c->cfg.lambda, c->cfg.flags, lanes_of(b, c), bs));
        PCT_BCK(pct::launch_drop_apply(c->x, c->delta, c->inv_s + (size_t)blk * c->M, c->M, clamp,
                                       c->cfg.clamp_min, bs));
        b->launches += 2;
      }
  }
  for (int k = 0; k < nb; ++k) {
    PCT_BCK(cudaEventRecord(b->join[1 + k], b->branch[k]));
    PCT_BCK(cudaStreamWaitEvent(s, b->join[1 + k], 0));
  }
  return PCT_OK;
}

pct_status enqueue_any(pct_batch* b, int n_sweeps, cudaStream_t s, long long spin_limit);

// The descriptors and the plan hold each context's record pointers, block
// ranges and weights as they were at pct_batch_create: refuse to run on a
// context reloaded or given a hull since.
pct_status check_contexts(const pct_batch* b) {
  for (size_t r = 0; r < b->ctx.size(); ++r)
    if (!b->ctx[r]->loaded || b->ctx[r]->generation != b->gen[r])
      return bfail(PCT_ERR_STATE, "a context was reloaded or given a hull after pct_batch_create",
                   "create the batch again");
  return PCT_OK;
}

long long spin_limit_of(const pct_batch* b) {
  const double lim = b->cfg.wait_limit_s > 0 ? b->cfg.wait_limit_s : 2.0;
  return (long long)(lim / 300e-9) + 1;  // ~300 ns per polling round (256 ns sleep + read)
}

pct_status enqueue_any(pct_batch* b, int n_sweeps, cudaStream_t s, long long spin_limit) {
  if (b->cfg.mode == PCT_BATCH_GRAPH_BRANCHES) return enqueue_branches(b, n_sweeps, s);
  return enqueue(b, n_sweeps, s, spin_limit);
}

pct_status read_status(pct_batch* b, cudaStream_t s) {
  if (b->cfg.mode == PCT_BATCH_GRAPH_BRANCHES) {
    PCT_BCK(cudaStreamSynchronize(s));
    return PCT_OK;
  }
  const int n = (int)b->ctx.size();
  unsigned long long* head = (unsigned long long*)(b->d_counters + 2 * n);
  int st = 0;
  PCT_BCK(cudaMemcpyAsync(&st, (int*)(head + 1), sizeof st, cudaMemcpyDeviceToHost, s));
  PCT_BCK(cudaStreamSynchronize(s));
  if (st != 0) {
    // leave every context consistent: drop partial block contributions
    for (auto* c : b->ctx) PCT_BCK(cudaMemsetAsync(c->delta, 0, c->M * sizeof(float), s));
    PCT_BCK(cudaStreamSynchronize(s));
    return bfail(PCT_ERR_TIMEOUT,
                 "batched launch: a bounded wait ran out (blocks not applied in this call are lost; x stays finite)");
  }
  return PCT_OK;
}

}  // namespace

extern "C" {

pct_status pct_batch_create(pct_batch** out, pct_ctx* const* ctxs, int32_t n, const pct_batch_config* cfg) {
  if (!out) return bfail(PCT_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!ctxs || n < 1) return bfail(PCT_ERR_INVALID_ARG, "need at least one context");
  for (int r = 0; r < n; ++r) {
    if (!ctxs[r]) return bfail(PCT_ERR_INVALID_ARG, "context is NULL");
    if (!ctxs[r]->loaded) return bfail(PCT_ERR_STATE, "every context must have histories loaded");
    if (ctxs[r]->device != ctxs[0]->device) return bfail(PCT_ERR_INVALID_ARG, "contexts on different devices");
    if (ctxs[r]->cfg.flags & PCT_FLAG_CARP) return bfail(PCT_ERR_INVALID_ARG, "CARP contexts are not batched");
    if (ctxs[r]->cfg.tvs_beta0 > 0.f) return bfail(PCT_ERR_INVALID_ARG, "TVS contexts are not batched");
    if (ctxs[r]->hull_mask) return bfail(PCT_ERR_INVALID_ARG, "contexts with an object hull are not batched");
    if (pct::ensure_block_weights(ctxs[r]) != PCT_OK) return bfail(PCT_ERR_CUDA, "block weights", pct_last_error());
  }
  pct_batch* b = new pct_batch();
  b->device = ctxs[0]->device;
  b->ctx.assign(ctxs, ctxs + n);
  for (int r = 0; r < n; ++r) b->gen.push_back(ctxs[r]->generation);
  if (cfg) b->cfg = *cfg;
  pct::DeviceGuard device_guard_;
  pct_status st = PCT_OK;
  do {
    cudaError_t e = cudaSetDevice(b->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->n_sms, cudaDevAttrMultiProcessorCount, b->device);
    for (auto* c : b->ctx) b->max_nodes = std::max(b->max_nodes, c->K + 1);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b->max_ctas_per_sm, batch_kernel, kThreads,
                                                        (size_t)b->max_nodes * sizeof(float4));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->own_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      st = bfail(PCT_ERR_CUDA, "batch set-up", cudaGetErrorString(e));
      break;
    }
    if (b->cfg.chunk <= 0) b->cfg.chunk = 4096;
    if (b->cfg.mode != PCT_BATCH_PERSISTENT && b->cfg.mode != PCT_BATCH_GRAPH_BRANCHES)
      b->cfg.mode = PCT_BATCH_GRAPH_BRANCHES;
    if (b->cfg.branches <= 0) b->cfg.branches = std::min(8, n);
    b->branch.assign(std::max(1, std::min(8, n)), nullptr);
    for (auto& bs : b->branch)
      if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking);
    b->join.assign(b->branch.size() + 1, nullptr);
    for (auto& ev : b->join)
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      st = bfail(PCT_ERR_CUDA, "batch streams", cudaGetErrorString(e));
      break;
    }
    if (b->cfg.ctas_per_sm <= 0 || b->cfg.ctas_per_sm > b->max_ctas_per_sm) b->cfg.ctas_per_sm = b->max_ctas_per_sm;
    if (b->cfg.lanes < 0) b->cfg.lanes = 0;
    if (b->cfg.lanes > 1 && !pct::group_lanes_supported(b->cfg.lanes)) {
      st = bfail(PCT_ERR_INVALID_ARG, "lanes must be 1, 2, 4, 8, 16 or 32");
      break;
    }
    std::vector<ReconDesc> rd(n);
    for (int r = 0; r < n; ++r) {
      pct_ctx* c = b->ctx[r];
      rd[r] = ReconDesc{c->geo,  c->rec,        c->tab32,    c->x, c->delta, c->inv_s, c->M, c->cfg.lambda,
                        c->cfg.flags, (c->cfg.flags & PCT_FLAG_CLAMP) != 0, c->cfg.clamp_min};
      b->x_total += c->M;
    }
    const size_t words = 2 * n + 1 + 3;
    if (cudaMalloc((void**)&b->d_recs, n * sizeof(ReconDesc)) != cudaSuccess ||
        cudaMalloc((void**)&b->d_sweep_counts, n * sizeof(uint2)) != cudaSuccess ||
        cudaMalloc((void**)&b->d_counters, words * sizeof(unsigned)) != cudaSuccess ||
        cudaMalloc((void**)&b->x_save, b->x_total * sizeof(float)) != cudaSuccess) {
      (void)cudaGetLastError();
      st = bfail(PCT_ERR_NO_MEMORY, "batch allocation failed");
      break;
    }
    if ((e = cudaMemcpy(b->d_recs, rd.data(), n * sizeof(ReconDesc), cudaMemcpyHostToDevice)) != cudaSuccess) {
      st = bfail(PCT_ERR_CUDA, "batch descriptors", cudaGetErrorString(e));
      break;
    }
    st = build_plan(b);
  } while (0);
  if (st != PCT_OK) {
    pct_batch_destroy(b);
    return st;
  }
  *out = b;
  return PCT_OK;
}

pct_status pct_batch_destroy(pct_batch* b) {
  if (!b) return PCT_OK;
  pct::DeviceGuard device_guard_;
  cudaSetDevice(b->device);
  if (b->own_stream) cudaStreamSynchronize(b->own_stream);
  free_plan(b);
  cudaFree(b->d_recs);
  cudaFree(b->d_sweep_counts);
  cudaFree(b->d_counters);
  cudaFree(b->x_save);
  for (auto bs : b->branch)
    if (bs) cudaStreamDestroy(bs);
  for (auto ev : b->join)
    if (ev) cudaEventDestroy(ev);
  if (b->own_stream) cudaStreamDestroy(b->own_stream);
  delete b;
  return PCT_OK;
}

pct_status pct_batch_iterate(pct_batch* b, int32_t n_sweeps, void* stream) {
  pct::TraceRange trace_("pct_batch_iterate");
  if (!b) return bfail(PCT_ERR_INVALID_ARG, "batch is NULL");
  if (n_sweeps < 0) return bfail(PCT_ERR_INVALID_ARG, "n_sweeps < 0");
  pct_status cs = check_contexts(b);
  if (cs != PCT_OK) return cs;
  if (n_sweeps == 0) return PCT_OK;
  pct::DeviceGuard device_guard_;
  PCT_BCK(cudaSetDevice(b->device));
  cudaStream_t s = stream ? (cudaStream_t)stream : b->own_stream;
  // work a context queued on its own stream (a load's counting sweep, its own
  // sweeps) finishes before the batch reads and writes its image
  for (auto* c : b->ctx)
    if (c->stream != s) PCT_BCK(cudaStreamSynchronize(c->stream));
  if (b->cfg.debug_unreachable_wait) return enqueue(b, n_sweeps, s, spin_limit_of(b));  // persistent only
  if (!b->graph || b->graph_sweeps != n_sweeps) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    cudaGraph_t g = nullptr;
    PCT_BCK(cudaStreamSynchronize(s));
    if (b->cfg.mode != PCT_BATCH_PERSISTENT) {
      const pct_status ps = prepare_lanes(b);
      if (ps != PCT_OK) return ps;
    }
    PCT_BCK(cudaStreamBeginCapture(b->own_stream, cudaStreamCaptureModeThreadLocal));
    const int64_t l0 = b->launches;
    pct_status st = enqueue_any(b, n_sweeps, b->own_stream, spin_limit_of(b));
    cudaError_t e = cudaStreamEndCapture(b->own_stream, &g);
    if (st != PCT_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (e != cudaSuccess) return bfail(PCT_ERR_CUDA, "batch capture", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      b->graph = nullptr;
      return bfail(PCT_ERR_CUDA, "batch graph instantiate", cudaGetErrorString(e));
    }
    b->graph_sweeps = n_sweeps;
    b->graph_launches = b->launches - l0;  // kernels per graph run
    b->launches = l0;                      // counted when the graph runs
  }
  PCT_BCK(cudaGraphLaunch(b->graph, s));
  b->launches += b->graph_launches;
  return PCT_OK;
}

pct_status pct_batch_sync(pct_batch* b, void* stream) {
  if (!b) return bfail(PCT_ERR_INVALID_ARG, "batch is NULL");
  pct::DeviceGuard device_guard_;
  PCT_BCK(cudaSetDevice(b->device));
  cudaStream_t s = stream ? (cudaStream_t)stream : b->own_stream;
  PCT_BCK(cudaStreamSynchronize(s));
  PCT_BCK(cudaGetLastError());
  return read_status(b, s);
}

pct_status pct_batch_autotune(pct_batch* b, pct_batch_config* chosen, float* best_ms) {
  pct::TraceRange trace_("pct_batch_autotune");
  if (!b) return bfail(PCT_ERR_INVALID_ARG, "batch is NULL");
  pct_status cs = check_contexts(b);
  if (cs != PCT_OK) return cs;
  pct::DeviceGuard device_guard_;
  PCT_BCK(cudaSetDevice(b->device));
  cudaStream_t s = b->own_stream;
  for (auto* c : b->ctx) PCT_BCK(cudaStreamSynchronize(c->stream));  // the contexts' queued work first
  // save every x: the trial sweeps change them
  int64_t off = 0;
  for (auto* c : b->ctx) {
    PCT_BCK(cudaMemcpyAsync(b->x_save + off, c->x, c->M * sizeof(float), cudaMemcpyDeviceToDevice, s));
    off += c->M;
  }
  struct Cand {
    int mode, chunk, ctas, branches, lanes;
  };
  std::vector<Cand> cands;
  for (int lanes : {1, 16, 32})
    for (int nb : {1, 4, 8})
      if (nb <= (int)b->branch.size() && (nb == 1 || nb <= (int)b->ctx.size()))
        cands.push_back({PCT_BATCH_GRAPH_BRANCHES, b->cfg.chunk, b->cfg.ctas_per_sm, nb, lanes});
  for (int ch : {2048, 4096, 8192})
    for (int v : {b->max_ctas_per_sm, b->max_ctas_per_sm - 1, b->max_ctas_per_sm / 2})
      if (v >= 1) cands.push_back({PCT_BATCH_PERSISTENT, ch, v, b->cfg.branches, 1});
  cudaEvent_t e0, e1;
  PCT_BCK(cudaEventCreate(&e0));
  PCT_BCK(cudaEventCreate(&e1));
  pct_batch_config best = b->cfg;
  float best_t = INFINITY;
  pct_status st = PCT_OK;
  for (const Cand& cd : cands) {
    b->cfg.mode = cd.mode;
    b->cfg.chunk = cd.chunk;
    b->cfg.ctas_per_sm = cd.ctas;
    b->cfg.branches = cd.branches;
    b->cfg.lanes = cd.lanes;
    if ((st = build_plan(b)) != PCT_OK) break;
    if (cd.mode != PCT_BATCH_PERSISTENT && (st = prepare_lanes(b)) != PCT_OK) break;
    float t = 0.f;
    if (cudaEventRecord(e0, s) != cudaSuccess || (st = enqueue_any(b, 1, s, spin_limit_of(b))) != PCT_OK ||
        cudaEventRecord(e1, s) != cudaSuccess || (st = read_status(b, s)) != PCT_OK ||
        cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) {
      if (st == PCT_OK) st = bfail(PCT_ERR_CUDA, "autotune timing");
      break;
    }
    if (t < best_t) {
      best_t = t;
      best = b->cfg;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != PCT_OK) return st;
  b->cfg = best;
  if ((st = build_plan(b)) != PCT_OK) return st;
  off = 0;
  for (auto* c : b->ctx) {
    PCT_BCK(cudaMemcpyAsync(c->x, b->x_save + off, c->M * sizeof(float), cudaMemcpyDeviceToDevice, s));
    PCT_BCK(cudaMemsetAsync(c->delta, 0, c->M * sizeof(float), s));
    off += c->M;
  }
  PCT_BCK(cudaStreamSynchronize(s));
  if (chosen) *chosen = best;
  if (best_ms) *best_ms = best_t;
  return PCT_OK;
}

int64_t pct_batch_launch_count(const pct_batch* b) { return b ? b->launches : 0; }

}  // extern "C"
