// C ABI of libpct (declared in include/pct.h): context, buffers, loading,
// row export and the DROP iteration loop under a captured CUDA graph.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/pct.h"
#include "pct_ctx.h"
#include "pct_trace.h"

using pct::Geo;
using pct::Rec;


namespace {

thread_local std::string g_err;

pct_status fail(pct_status code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define PCT_CK(call)                                                                          \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) return fail(PCT_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

// Failure injection for tests (pct_debug_fail_alloc): when armed with k, the
// k-th device allocation made through dev_alloc from then on fails as if the
// device had no memory left; each later allocation succeeds again.
std::atomic<int64_t> g_fail_alloc_countdown{0};

cudaError_t dev_alloc(void** p, size_t bytes) {
  int64_t k = g_fail_alloc_countdown.load();
  while (k > 0 && !g_fail_alloc_countdown.compare_exchange_weak(k, k - 1)) {
  }
  if (k == 1) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(p, bytes);
}

#define PCT_ALLOC(ptr, bytes)                                                                         \
  do {                                                                                                \
    cudaError_t e_ = dev_alloc((void**)&(ptr), (bytes));                                              \
    if (e_ != cudaSuccess) {                                                                          \
      (void)cudaGetLastError();                                                                       \
      return fail(PCT_ERR_NO_MEMORY, "cudaMalloc(%lld bytes): %s", (long long)(bytes), cudaGetErrorString(e_)); \
    }                                                                                                 \
  } while (0)

void drop_graphs(pct_ctx* c) {
  if (c->sweep) cudaGraphExecDestroy(c->sweep);
  c->sweep = nullptr;
  if (c->sweep_count) cudaGraphExecDestroy(c->sweep_count);
  c->sweep_count = nullptr;
  c->graph_n = -1;
}

// Forget the loaded set (its buffers, and the sweep graphs, stay for the
// next load; pct_load_histories drops the graphs if what they captured
// changes).
void reset_records(pct_ctx* c) {
  c->swept = false;
  c->where = nullptr;
  c->rec = Rec{};
  c->n = 0;
  c->loaded = false;
  c->weights_ready = false;
}

void free_records(pct_ctx* c) {
  drop_graphs(c);
  reset_records(c);
  cudaFree(c->rec_store);
  cudaFree(c->inv_s);
  cudaFree(c->where_buf);
  cudaFree(c->hull_range);
  cudaFree(c->staging);
  cudaFree(c->sort_key);
  cudaFree(c->sort_order);
  cudaFree(c->sort_hist);
  c->rec_store = nullptr;
  c->inv_s = nullptr;
  c->where_buf = nullptr;
  c->hull_range = nullptr;
  c->staging = nullptr;
  c->sort_key = c->sort_order = c->sort_hist = nullptr;
  c->rec_cap = c->where_cap = c->range_cap = c->staging_cap = c->key_cap = c->order_cap = c->hist_cap = 0;
}

// Make `p` hold at least `need` elements (contents not kept when it grows).
template <class T>
pct_status grow(T*& p, int64_t& cap, int64_t need) {
  if (p && cap >= need) return PCT_OK;
  cudaFree(p);
  p = nullptr;
  cap = 0;
  cudaError_t e = dev_alloc((void**)&p, (size_t)need * sizeof(T));
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    p = nullptr;
    return fail(PCT_ERR_NO_MEMORY, "cudaMalloc(%lld bytes): %s", (long long)(need * (int64_t)sizeof(T)),
                cudaGetErrorString(e));
  }
  cap = need;
  return PCT_OK;
}

#define PCT_GROW(ptr, cap, need)                   \
  do {                                             \
    pct_status s_ = grow((ptr), (cap), (need));    \
    if (s_ != PCT_OK) return s_;                   \
  } while (0)

int64_t block_lo(const pct_ctx* c, int b) { return (int64_t)b * c->n / c->cfg.n_blocks; }

pct_status sync_and_check(pct_ctx* c) {
  PCT_CK(cudaStreamSynchronize(c->stream));
  PCT_CK(cudaGetLastError());
  return PCT_OK;
}

// DROP block weights (Sec. 2.1): s_j = runs of block b in voxel j; inv_s
// holds 1/s_j (0 where the block does not touch voxel j).
pct_status block_weights(pct_ctx* c) {
  for (int b = 0; b < c->cfg.n_blocks; ++b) {
    const int64_t lo = block_lo(c, b), hi = block_lo(c, b + 1);
    PCT_CK(cudaMemsetAsync(c->cnt, 0, (size_t)c->M * sizeof(unsigned int), c->stream));
    PCT_CK(pct::launch_count(c->geo, c->rec, c->tab32, pct::hull_view(c), lo, hi - lo, c->cnt, c->cfg.cta_threads,
                             c->stream));
    PCT_CK(pct::launch_inv_counts(c->cnt, c->inv_s + (size_t)b * c->M, c->M, c->stream));
    c->launches += 2;
  }
  c->weights_ready = true;
  return PCT_OK;
}

}  // namespace

void pct::set_error_text(const char* msg) { g_err = msg; }

pct_status pct::ensure_block_weights(pct_ctx* c) {
  if (c->weights_ready || !c->loaded) return PCT_OK;
  pct::DeviceGuard device_guard_;
  PCT_CK(cudaSetDevice(c->device));
  pct_status st = block_weights(c);
  if (st != PCT_OK) return st;
  return sync_and_check(c);
}

extern "C" {

const char* pct_last_error(void) { return g_err.c_str(); }

void pct_debug_fail_alloc(int64_t k) { g_fail_alloc_countdown.store(k > 0 ? k : 0); }

pct_status pct_create(pct_ctx** out, const pct_grid* grid, const pct_config* cfg, int device) {
  if (!out) return fail(PCT_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!grid || !cfg) return fail(PCT_ERR_INVALID_ARG, "grid or cfg is NULL");
  const pct_grid& g = *grid;
  if (g.nx < 1 || g.ny < 1 || g.nz < 1 || g.nx > pct::kMaxDim || g.ny > pct::kMaxDim || g.nz > pct::kMaxDim)
    return fail(PCT_ERR_INVALID_ARG, "grid dims must be in [1, %d]", pct::kMaxDim);
  if (!(g.hx > 0 && g.hy > 0 && g.hz > 0) || !isfinite(g.hx) || !isfinite(g.hy) || !isfinite(g.hz))
    return fail(PCT_ERR_INVALID_ARG, "voxel sizes must be finite and > 0");
  if (cfg->n_blocks < 1) return fail(PCT_ERR_INVALID_ARG, "n_blocks must be >= 1");
  if (!(cfg->lambda > 0.f && cfg->lambda < 2.f)) return fail(PCT_ERR_INVALID_ARG, "lambda must be in (0, 2)");
  if (cfg->threads_per_proton != 0 && cfg->threads_per_proton != 1 && !pct::group_lanes_supported(cfg->threads_per_proton))
    return fail(PCT_ERR_INVALID_ARG, "threads_per_proton must be 1, 2, 4, 8, 16 or 32");

  pct_ctx* c = new pct_ctx();
  c->device = device;
  c->grid = g;
  c->cfg = *cfg;
  if (c->cfg.cta_threads <= 0) c->cfg.cta_threads = 128;
  if (c->cfg.threads_per_proton <= 0) c->cfg.threads_per_proton = 1;
  if (c->cfg.tvs_alpha <= 0.f) c->cfg.tvs_alpha = 0.99f;
  if (c->cfg.tvs_eps <= 0.f) c->cfg.tvs_eps = 1e-4f;
  if (c->cfg.tvs_tries <= 0) c->cfg.tvs_tries = 4;
  if (c->cfg.carp_strings <= 0 || c->cfg.carp_strings > c->cfg.n_blocks) c->cfg.carp_strings = c->cfg.n_blocks;
  if (!(c->cfg.tvs_beta0 >= 0.f) || c->cfg.tvs_alpha > 1.f) {
    delete c;
    return fail(PCT_ERR_INVALID_ARG, "TVS needs beta0 >= 0 and 0 < alpha <= 1");
  }

  // Geometry in FP64, then rounded once to FP32 for the kernels.
  const double X = g.nx * g.hx, Y = g.ny * g.hy, Z = g.nz * g.hz;
  const double hmin = fmin(g.hx, fmin(g.hy, g.hz));
  const double step = cfg->node_step_mm > 0 ? cfg->node_step_mm : 0.5 * hmin;
  c->R = 0.5 * fmin(X, Y);
  c->K = (int)ceil(2.0 * c->R / step - 1e-9);
  if (c->K < 2 || c->K + 1 > pct::kMaxNodes) {
    delete c;
    return fail(PCT_ERR_INVALID_ARG, "node count K+1 = %d outside [3, %d]", c->K + 1, pct::kMaxNodes);
  }
  c->du = 2.0 * c->R / c->K;
  const double hd_xy = 0.5 * sqrt(X * X + Y * Y);
  c->E = (int)ceil((hd_xy - c->R) / c->du) + 2;
  c->M = (int64_t)g.nx * g.ny * g.nz;
  c->pos_limit = (float)(0.5 * sqrt(X * X + Y * Y + Z * Z) + c->R);
  {
    // worst-case node distance from the grid centre, in voxels: must stay
    // inside the +-1000 voxel quantisation range for every valid record
    const double umax = c->R + (c->E + 1) * c->du;
    const double tmax = c->pos_limit + 0.5 * (2.0 * c->R + c->E * c->du);
    const double qmax = (umax + tmax) / hmin + 0.5 * fmax((double)g.nx, fmax((double)g.ny, (double)g.nz));
    if (qmax >= pct::kQClamp) {
      delete c;
      return fail(PCT_ERR_INVALID_ARG, "grid too large for the fixed-point node range (%.0f voxels)", qmax);
    }
  }
  c->geo = pct::make_geo(g.nx, g.ny, g.nz, g.hx, g.hy, g.hz, c->R, c->du, c->K, c->E);

  pct::DeviceGuard device_guard_;
  pct_status st = PCT_OK;
  do {
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) {
      st = fail(PCT_ERR_CUDA, "cudaSetDevice(%d): %s", device, cudaGetErrorString(e));
      break;
    }
    e = cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      st = fail(PCT_ERR_CUDA, "cudaStreamCreate: %s", cudaGetErrorString(e));
      break;
    }
    c->stream = c->own_stream;
    size_t M = (size_t)c->M;
    if (dev_alloc((void**)&c->tab64, (c->K + 1) * 4 * sizeof(double)) != cudaSuccess ||
        dev_alloc((void**)&c->tab32, (c->K + 1) * sizeof(float4)) != cudaSuccess ||
        dev_alloc((void**)&c->x, M * sizeof(float)) != cudaSuccess ||
        dev_alloc((void**)&c->delta, M * sizeof(float)) != cudaSuccess ||
        dev_alloc((void**)&c->cnt, M * sizeof(unsigned int)) != cudaSuccess ||
        dev_alloc((void**)&c->first_bad, sizeof(unsigned long long)) != cudaSuccess ||
        dev_alloc((void**)&c->acc, sizeof(double)) != cudaSuccess) {
      (void)cudaGetLastError();
      st = fail(PCT_ERR_NO_MEMORY, "device allocation failed for a %lld-voxel grid", (long long)c->M);
      break;
    }
    if ((e = cudaMemsetAsync(c->x, 0, M * sizeof(float), c->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(c->delta, 0, M * sizeof(float), c->stream)) != cudaSuccess ||
        (e = pct::launch_mlp_table(c->R, c->du, c->K, c->tab64, c->tab32, c->stream)) != cudaSuccess ||
        (c->cfg.threads_per_proton > 1 && (e = pct::prepare_drop_group(c->cfg.threads_per_proton, c->K)) != cudaSuccess) ||
        (e = cudaStreamSynchronize(c->stream)) != cudaSuccess) {
      st = fail(PCT_ERR_CUDA, "context set-up: %s", cudaGetErrorString(e));
      break;
    }
    {
      // the table's largest node-to-node step bounds every MLP segment (the
      // walk's per-history choice between its two forms)
      std::vector<float4> th((size_t)c->K + 1);
      if ((e = cudaMemcpy(th.data(), c->tab32, th.size() * sizeof(float4), cudaMemcpyDeviceToHost)) != cudaSuccess) {
        st = fail(PCT_ERR_CUDA, "table read-back: %s", cudaGetErrorString(e));
        break;
      }
      pct::set_table_bound(c->geo, th.data(), c->K);
    }
    c->launches += 1;
    if (c->cfg.flags & PCT_FLAG_CARP) {
      if (dev_alloc((void**)&c->carp_sum, M * sizeof(float)) != cudaSuccess ||
          dev_alloc((void**)&c->carp_touch, M * sizeof(float)) != cudaSuccess ||
          dev_alloc((void**)&c->carp_x0, M * sizeof(float)) != cudaSuccess) {
        (void)cudaGetLastError();
        st = fail(PCT_ERR_NO_MEMORY, "CARP buffers");
        break;
      }
      if ((e = cudaMemsetAsync(c->carp_sum, 0, M * sizeof(float), c->stream)) != cudaSuccess ||
          (e = cudaMemsetAsync(c->carp_touch, 0, M * sizeof(float), c->stream)) != cudaSuccess ||
          (e = cudaStreamSynchronize(c->stream)) != cudaSuccess) {
        st = fail(PCT_ERR_CUDA, "CARP buffers: %s", cudaGetErrorString(e));
        break;
      }
    }
    if (c->cfg.tvs_beta0 > 0.f) {
      if (dev_alloc((void**)&c->tv_g, M * sizeof(float)) != cudaSuccess ||
          dev_alloc((void**)&c->tv_xp, M * sizeof(float)) != cudaSuccess ||
          dev_alloc((void**)&c->tv_acc, 3 * sizeof(double)) != cudaSuccess ||
          dev_alloc((void**)&c->tv_state, sizeof(pct::TvState)) != cudaSuccess) {
        (void)cudaGetLastError();
        st = fail(PCT_ERR_NO_MEMORY, "TVS buffers");
        break;
      }
      if ((e = cudaMemsetAsync(c->tv_acc, 0, 3 * sizeof(double), c->stream)) != cudaSuccess ||
          (e = cudaMemsetAsync(c->tv_state, 0, sizeof(pct::TvState), c->stream)) != cudaSuccess ||
          (e = cudaStreamSynchronize(c->stream)) != cudaSuccess) {
        st = fail(PCT_ERR_CUDA, "TVS buffers: %s", cudaGetErrorString(e));
        break;
      }
    }
    if (c->cfg.flags & PCT_FLAG_PROFILE) {
      c->ev = new cudaEvent_t[3 * c->cfg.n_blocks]();
      for (int i = 0; i < 3 * c->cfg.n_blocks && e == cudaSuccess; ++i) e = cudaEventCreate(&c->ev[i]);
      if (e != cudaSuccess) {
        st = fail(PCT_ERR_CUDA, "cudaEventCreate: %s", cudaGetErrorString(e));
        break;
      }
    }
  } while (0);
  if (st != PCT_OK) {
    pct_destroy(c);
    return st;
  }
  *out = c;
  return PCT_OK;
}

pct_status pct_destroy(pct_ctx* c) {
  if (!c) return PCT_OK;
  pct::DeviceGuard device_guard_;
  cudaSetDevice(c->device);
  if (c->own_stream) cudaStreamSynchronize(c->own_stream);
  if (c->stream && c->stream != c->own_stream) cudaStreamSynchronize(c->stream);
  if (c->copy_stream) cudaStreamSynchronize(c->copy_stream);
  free_records(c);
  cudaFree(c->tab64);
  cudaFree(c->tab32);
  cudaFree(c->x);
  cudaFree(c->delta);
  cudaFree(c->cnt);
  cudaFree(c->pair);
  cudaFree(c->pair_overflow);
  cudaFree(c->x_save);
  cudaFree(c->first_bad);
  cudaFree(c->acc);
  cudaFree(c->carp_sum);
  cudaFree(c->carp_touch);
  cudaFree(c->carp_x0);
  cudaFree(c->tv_g);
  cudaFree(c->tv_xp);
  cudaFree(c->tv_acc);
  cudaFree(c->tv_state);
  cudaFree(c->hull_mask);
  cudaFree(c->fam32);
  if (c->ev) {
    for (int i = 0; i < 3 * c->cfg.n_blocks; ++i) cudaEventDestroy(c->ev[i]);
    delete[] c->ev;
  }
  for (int i = 0; i < 4; ++i)
    if (c->load_ev[i]) cudaEventDestroy(c->load_ev[i]);
  if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
  if (c->own_stream) cudaStreamDestroy(c->own_stream);
  delete c;
  return PCT_OK;
}

pct_status pct_set_stream(pct_ctx* c, void* stream) {
  if (!c) return fail(PCT_ERR_INVALID_ARG, "ctx is NULL");
  cudaStream_t next = stream ? (cudaStream_t)stream : c->own_stream;
  pct::DeviceGuard device_guard_;
  if (next != c->stream) {
    // work queued on the old stream finishes before any on the new one starts
    PCT_CK(cudaSetDevice(c->device));
    PCT_CK(cudaStreamSynchronize(c->stream));
  }
  c->stream = next;
  return PCT_OK;
}

pct_status pct_geometry(const pct_ctx* c, double* R, double* du, int32_t* K, int32_t* E, int64_t* M) {
  if (!c) return fail(PCT_ERR_INVALID_ARG, "ctx is NULL");
  if (R) *R = c->R;
  if (du) *du = c->du;
  if (K) *K = c->K;
  if (E) *E = c->E;
  if (M) *M = c->M;
  return PCT_OK;
}

pct_status pct_mlp_table(pct_ctx* c, double* out, int to_device) {
  if (!c || !out) return fail(PCT_ERR_INVALID_ARG, "ctx or out is NULL");
  pct::DeviceGuard device_guard_;
  PCT_CK(cudaSetDevice(c->device));
  size_t bytes = (size_t)(c->K + 1) * 4 * sizeof(double);
  PCT_CK(cudaMemcpyAsync(out, c->tab64, bytes, to_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                         c->stream));
  if (!to_device) return sync_and_check(c);
  return PCT_OK;
}

namespace {

Rec rec_at(float* base, int64_t stride) {
  const float* f[11];
  for (int i = 0; i < 11; ++i) f[i] = base + (size_t)i * stride;
  return Rec{f[0], f[1], f[2], f[3], f[4], f[5], f[6], f[7], f[8], f[9], f[10]};
}

Rec rec_offset(const float* const* src, int64_t lo) {
  return Rec{src[0] + lo, src[1] + lo, src[2] + lo, src[3] + lo, src[4] + lo, src[5] + lo,
             src[6] + lo, src[7] + lo, src[8] + lo, src[9] + lo, src[10] + lo};
}



// Bring block b's records to the device, validate them and store them ordered
// (or copied) into the context's record arrays, all queued on the context's
// stream; host records go through staging slot b & 1 on the copy stream.
pct_status load_block(pct_ctx* c, const float* const src[11], int flags, int b, int64_t max_blk, bool sort,
                      bool in_place) {
  const int64_t lo = block_lo(c, b), cnt = block_lo(c, b + 1) - lo;
  Rec blk;
  if (flags == PCT_LOAD_HOST) {
    const int slot = b & 1;
    float* dst = c->staging + (size_t)slot * 11 * max_blk;
    if (b >= 2) PCT_CK(cudaStreamWaitEvent(c->copy_stream, c->load_ev[2 + slot], 0));  // block b - 2 consumed
    for (int f = 0; f < 11; ++f)
      PCT_CK(cudaMemcpyAsync(dst + (size_t)f * max_blk, src[f] + lo, (size_t)cnt * sizeof(float),
                             cudaMemcpyHostToDevice, c->copy_stream));
    PCT_CK(cudaEventRecord(c->load_ev[slot], c->copy_stream));
    PCT_CK(cudaStreamWaitEvent(c->stream, c->load_ev[slot], 0));
    blk = rec_at(dst, max_blk);
  } else {
    blk = rec_offset(src, lo);
  }
  PCT_CK(pct::launch_validate(blk, cnt, lo, c->pos_limit, c->first_bad, c->stream));
  c->launches += 1;
  if (sort) {
    PCT_CK(pct::launch_sort_block(blk, cnt, lo, c->pos_limit, c->tab32, c->K, c->rec, c->where, c->sort_key, c->sort_hist, c->sort_order,
                                  c->stream));
    c->launches += 5;
  } else if (!in_place) {
    PCT_CK(pct::launch_copy_block(blk, cnt, lo, c->rec, c->stream));
    c->launches += 1;
  }
  if (flags == PCT_LOAD_HOST) PCT_CK(cudaEventRecord(c->load_ev[2 + (b & 1)], c->stream));
  return PCT_OK;
}

}  // namespace

pct_status pct_load_histories(pct_ctx* c, const pct_histories* h, int flags, int64_t* first_bad) {
  pct::TraceRange trace_("pct_load_histories");
  if (first_bad) *first_bad = -1;
  if (!c || !h) return fail(PCT_ERR_INVALID_ARG, "ctx or histories is NULL");
  if (h->n < 1) return fail(PCT_ERR_INVALID_ARG, "n must be >= 1");
  if (h->n < c->cfg.n_blocks) return fail(PCT_ERR_INVALID_ARG, "n (%lld) < n_blocks (%d)", (long long)h->n,
                                          c->cfg.n_blocks);
  if (h->n >= ((int64_t)1 << 32) * c->cfg.n_blocks) return fail(PCT_ERR_INVALID_ARG, "blocks of >= 2^32 histories");
  const float* src[11] = {h->t0, h->v0, h->st0, h->sv0, h->t2, h->v2, h->st2, h->sv2, h->wepl, h->cphi, h->sphi};
  for (int f = 0; f < 11; ++f)
    if (!src[f]) return fail(PCT_ERR_INVALID_ARG, "history array %d is NULL", f);
  if (flags != PCT_LOAD_HOST && flags != PCT_LOAD_DEVICE_COPY && flags != PCT_LOAD_DEVICE_BORROW)
    return fail(PCT_ERR_INVALID_ARG, "unknown load flags %d", flags);
  pct::DeviceGuard device_guard_;
  PCT_CK(cudaSetDevice(c->device));
  PCT_CK(cudaStreamSynchronize(c->stream));
  if (c->copy_stream) PCT_CK(cudaStreamSynchronize(c->copy_stream));  // copies left by a failed load
  reset_records(c);
  ++c->generation;
  const int64_t n = h->n;
  c->n = n;
  const int B = c->cfg.n_blocks;
  const bool sort = !(c->cfg.flags & PCT_FLAG_NO_SORT);
  const bool in_place = flags == PCT_LOAD_DEVICE_BORROW && !sort;
  int64_t max_blk = 0;
  for (int b = 0; b < B; ++b) max_blk = block_lo(c, b + 1) - block_lo(c, b) > max_blk ? block_lo(c, b + 1) - block_lo(c, b) : max_blk;

  if (in_place) {
    c->rec = rec_offset(src, 0);
  } else {
    PCT_GROW(c->rec_store, c->rec_cap, n * 11);
    c->rec = rec_at(c->rec_store, n);
  }
  if (sort) {
    PCT_GROW(c->where_buf, c->where_cap, n);
    c->where = c->where_buf;
    PCT_GROW(c->sort_key, c->key_cap, max_blk);
    PCT_GROW(c->sort_order, c->order_cap, max_blk);
    PCT_GROW(c->sort_hist, c->hist_cap, pct::kSortHistEntries);
  }
  if (flags == PCT_LOAD_HOST) {
    PCT_GROW(c->staging, c->staging_cap, 2 * max_blk * 11);
    if (!c->copy_stream) PCT_CK(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
    for (int i = 0; i < 4; ++i)
      if (!c->load_ev[i]) PCT_CK(cudaEventCreateWithFlags(&c->load_ev[i], cudaEventDisableTiming));
  }

  // per block: bring the records to the device, validate, order (or copy).
  // Host records go through two staging slots: block b + 1 is copied on the
  // copy stream while block b is validated and ordered on the context's stream.
  PCT_CK(cudaMemsetAsync(c->first_bad, 0xff, sizeof(unsigned long long), c->stream));
  {
    pct_status lst = PCT_OK;
    for (int b = 0; b < B && lst == PCT_OK; ++b) lst = load_block(c, src, flags, b, max_blk, sort, in_place);
    if (flags == PCT_LOAD_HOST) {
      // no copy outlives the call: the caller may free its host arrays on return
      const cudaError_t e = cudaStreamSynchronize(c->copy_stream);
      if (lst == PCT_OK && e != cudaSuccess) lst = fail(PCT_ERR_CUDA, "host copies: %s", cudaGetErrorString(e));
    }
    if (lst != PCT_OK) return lst;
  }
  unsigned long long fb = 0;
  PCT_CK(cudaMemcpyAsync(&fb, c->first_bad, sizeof fb, cudaMemcpyDeviceToHost, c->stream));
  PCT_CK(cudaStreamSynchronize(c->stream));
  if (fb != ~0ull) {
    if (first_bad) *first_bad = (int64_t)fb;
    reset_records(c);
    return fail(PCT_ERR_INVALID_DATA, "history %lld failed validation", (long long)fb);
  }

  // hull ranges of the stored histories, then the DROP block weights
  if (c->hull_mask) {
    PCT_GROW(c->hull_range, c->range_cap, n);
    PCT_CK(pct::launch_hull_ranges(c->geo, c->rec, n, c->hull_mask, c->hull_range, c->stream));
    c->launches += 1;
  }
  // the sweep graphs captured the record pointers, the block ranges (from n)
  // and the hull ranges: keep them only if none of these changed
  if (c->graph_n != n || memcmp(&c->graph_rec, &c->rec, sizeof(Rec)) != 0 ||
      c->graph_range != pct::hull_view(c).range)
    drop_graphs(c);
  // the block weights are counted by the first sweep (pct_iterate), or on
  // demand (pct::ensure_block_weights)
  if (!c->inv_s) PCT_ALLOC(c->inv_s, (size_t)B * c->M * sizeof(float));
  c->weights_ready = false;
  PCT_CK(cudaMemsetAsync(c->x, 0, (size_t)c->M * sizeof(float), c->stream));
  PCT_CK(cudaMemsetAsync(c->delta, 0, (size_t)c->M * sizeof(float), c->stream));
  if (c->tv_state) PCT_CK(cudaMemsetAsync(c->tv_state, 0, sizeof(pct::TvState), c->stream));
  pct_status st = sync_and_check(c);
  if (st != PCT_OK) return st;
  c->loaded = true;
  return PCT_OK;
}

pct_status pct_set_hull(pct_ctx* c, const uint8_t* mask, int on_device) {
  if (!c) return fail(PCT_ERR_INVALID_ARG, "ctx is NULL");
  pct::DeviceGuard device_guard_;
  PCT_CK(cudaSetDevice(c->device));
  PCT_CK(cudaStreamSynchronize(c->stream));
  drop_graphs(c);  // the sweep's kernels change
  ++c->generation;
  if (!mask) {
    cudaFree(c->hull_mask);
    cudaFree(c->hull_range);
    c->hull_mask = nullptr;
    c->hull_range = nullptr;
    c->range_cap = 0;
  } else {
    if (!c->hull_mask) PCT_ALLOC(c->hull_mask, (size_t)c->M);
    if (!c->fam32) {
      PCT_ALLOC(c->fam32, (size_t)pct::family_offset(c->K + 1) * sizeof(float4));
      PCT_CK(pct::launch_mlp_family(c->R, c->du, c->K, c->fam32, 0, nullptr, c->stream));
      c->launches += 1;
    }
    PCT_CK(cudaMemcpyAsync(c->hull_mask, mask, (size_t)c->M,
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
    if (c->loaded) {
      PCT_GROW(c->hull_range, c->range_cap, c->n);
      PCT_CK(pct::launch_hull_ranges(c->geo, c->rec, c->n, c->hull_mask, c->hull_range, c->stream));
      c->launches += 1;
    }
  }
  c->weights_ready = false;  // the rows changed: the next sweep recounts
  return sync_and_check(c);
}

pct_status pct_carve_hull(pct_ctx* c, float wepl_max, int32_t dilate) {
  if (!c) return fail(PCT_ERR_INVALID_ARG, "ctx is NULL");
  if (!c->loaded) return fail(PCT_ERR_STATE, "no histories loaded");
  if (dilate < 0) return fail(PCT_ERR_INVALID_ARG, "dilate must be >= 0");
  pct::DeviceGuard device_guard_;
  PCT_CK(cudaSetDevice(c->device));
  uint8_t *out = nullptr, *tmp = nullptr;
  cudaError_t e = dev_alloc((void**)&out, (size_t)c->M);
  if (e == cudaSuccess) e = dev_alloc((void**)&tmp, (size_t)c->M);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    cudaFree(out);
    return fail(PCT_ERR_NO_MEMORY, "carving scratch (%lld bytes)", (long long)c->M);
  }
  e = pct::launch_carve_hull(c->geo, c->rec, c->tab32, c->n, wepl_max, dilate, out, tmp, c->stream);
  c->launches += 1 + dilate;
  pct_status st = e == cudaSuccess ? pct_set_hull(c, out, 1) : fail(PCT_ERR_CUDA, "carving: %s", cudaGetErrorString(e));
  cudaStreamSynchronize(c->stream);
  cudaFree(out);
  cudaFree(tmp);
  return st;
}

pct_status pct_get_hull(pct_ctx* c, uint8_t* out) {
  if (!c || !out) return fail(PCT_ERR_INVALID_ARG, "ctx or out is NULL");
  if (!c->hull_mask) return fail(PCT_ERR_STATE, "no hull set");
  pct::DeviceGuard device_guard_;
  PCT_CK(cudaSetDevice(c->device));
  PCT_CK(cudaMemcpyAsync(out, c->hull_mask, (size_t)c->M, cudaMemcpyDeviceToHost, c->stream));
  return sync_and_check(c);
}

pct_status pct_hull_ranges(pct_ctx* c, int64_t first, int64_t count, int32_t* out) {
  if (!c || (count > 0 && !out)) return fail(PCT_ERR_INVALID_ARG, "ctx or out is NULL");
  if (!c->loaded) return fail(PCT_ERR_STATE, "no histories loaded");
  if (!c->hull_mask) return fail(PCT_ERR_STATE, "no hull set");
  if (first < 0 || count < 0 || first + count > c->n) return fail(PCT_ERR_INVALID_ARG, "range outside [0, n)");
  pct::DeviceGuard device_guard_;
  PCT_CK(cudaSetDevice(c->device));
  if (count == 0) return PCT_OK;
  int32_t* d = nullptr;
  PCT_ALLOC(d, (size_t)count * 2 * sizeof(int32_t));
  cudaError_t e = pct::launch_gather_ranges(c->hull_range, c->where, first, count, d, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out, d, (size_t)count * 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cudaFree(d);
  c->launches += 1;
  if (e != cudaSuccess) return fail(PCT_ERR_CUDA, "hull ranges: %s", cudaGetErrorString(e));
  return PCT_OK;
}

pct_status pct_mlp_table_n(pct_ctx* c, int32_t n, double* out) {
  if (!c || !out) return fail(PCT_ERR_INVALID_ARG, "ctx or out is NULL");
  if (n < 1 || n > c->K) return fail(PCT_ERR_INVALID_ARG, "n must be in [1, K]");
  pct::DeviceGuard device_guard_;
  PCT_CK(cudaSetDevice(c->device));
  double* d = nullptr;
  PCT_ALLOC(d, (size_t)(n + 1) * 4 * sizeof(double));
  cudaError_t e = pct::launch_mlp_family(c->R, c->du, c->K, nullptr, n, d, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, d, (size_t)(n + 1) * 4 * sizeof(double), cudaMemcpyDeviceToHost,
                                            c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cudaFree(d);
  c->launches += 1;
  if (e != cudaSuccess) return fail(PCT_ERR_CUDA, "layer table: %s", cudaGetErrorString(e));
  return PCT_OK;
}

pct_status pct_mlp_rows(pct_ctx* c, int64_t first, int64_t count, int64_t* row_ptr, int32_t* vox, float* len,
                        int64_t cap, int32_t* nodes, int64_t* needed) {
  if (needed) *needed = 0;
  if (!c || !row_ptr) return fail(PCT_ERR_INVALID_ARG, "ctx or row_ptr is NULL");
  if (!c->loaded) return fail(PCT_ERR_STATE, "no histories loaded");
  if (first < 0 || count < 0 || first + count > c->n) return fail(PCT_ERR_INVALID_ARG, "range outside [0, n)");
  if (cap < 0 || (cap > 0 && (!vox || !len))) return fail(PCT_ERR_INVALID_ARG, "bad row buffers");
  pct::DeviceGuard device_guard_;
  PCT_CK(cudaSetDevice(c->device));
  PCT_CK(pct::launch_row_counts(c->geo, c->rec, c->tab32, pct::hull_view(c), first, count, c->where, row_ptr,
                                c->cfg.threads_per_proton, c->stream));
  PCT_CK(pct::launch_scan_rows(row_ptr, count, c->stream));
  c->launches += 2;
  int64_t total = 0;
  PCT_CK(cudaMemcpyAsync(&total, row_ptr + count, sizeof total, cudaMemcpyDeviceToHost, c->stream));
  PCT_CK(cudaStreamSynchronize(c->stream));
  if (needed) *needed = total;
  if (total > cap) return fail(PCT_ERR_CAPACITY, "rows need %lld runs, capacity %lld", (long long)total,
                               (long long)cap);
  PCT_CK(pct::launch_row_fill(c->geo, c->rec, c->tab32, pct::hull_view(c), first, count, c->where, row_ptr, vox,
                              len, nodes, c->cfg.threads_per_proton, c->stream));
  c->launches += 1;
  return sync_and_check(c);
}

pct_status pct_project(pct_ctx* c, int64_t first, int64_t count, float* y) {
  if (!c || (count > 0 && !y)) return fail(PCT_ERR_INVALID_ARG, "ctx or y is NULL");
  if (!c->loaded) return fail(PCT_ERR_STATE, "no histories loaded");
  if (first < 0 || count < 0 || first + count > c->n) return fail(PCT_ERR_INVALID_ARG, "range outside [0, n)");
  pct::DeviceGuard device_guard_;
  PCT_CK(cudaSetDevice(c->device));
  PCT_CK(pct::launch_project(c->geo, c->rec, c->tab32, pct::hull_view(c), first, count, c->where, c->x, c->cfg.flags,
                             y, c->stream));
  c->launches += 1;
  return PCT_OK;
}

pct_status pct_residual(pct_ctx* c, int64_t stride, double* sum_sq) {
  if (!c || !sum_sq) return fail(PCT_ERR_INVALID_ARG, "ctx or sum_sq is NULL");
  if (stride < 1) return fail(PCT_ERR_INVALID_ARG, "stride must be >= 1");
  if (!c->loaded) return fail(PCT_ERR_STATE, "no histories loaded");
  pct::DeviceGuard device_guard_;
  PCT_CK(cudaSetDevice(c->device));
  PCT_CK(cudaMemsetAsync(c->acc, 0, sizeof(double), c->stream));
  PCT_CK(pct::launch_residual(c->geo, c->rec, c->tab32, pct::hull_view(c), c->n, stride, c->x, c->cfg.flags, c->acc,
                              c->stream));
  c->launches += 1;
  PCT_CK(cudaMemcpyAsync(sum_sq, c->acc, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  return sync_and_check(c);
}

pct_status pct_block_counts(pct_ctx* c, int32_t block, float* out) {
  if (!c || !out) return fail(PCT_ERR_INVALID_ARG, "ctx or out is NULL");
  if (!c->loaded) return fail(PCT_ERR_STATE, "no histories loaded");
  if (block < 0 || block >= c->cfg.n_blocks) return fail(PCT_ERR_INVALID_ARG, "block out of range");
  pct::DeviceGuard device_guard_;
  PCT_CK(cudaSetDevice(c->device));
  const int64_t lo = block_lo(c, block), hi = block_lo(c, block + 1);
  PCT_CK(cudaMemsetAsync(c->cnt, 0, (size_t)c->M * sizeof(unsigned int), c->stream));
  PCT_CK(pct::launch_count(c->geo, c->rec, c->tab32, pct::hull_view(c), lo, hi - lo, c->cnt, c->cfg.cta_threads,
                           c->stream));
  PCT_CK(pct::launch_counts_to_float(c->cnt, out, c->M, c->stream));
  c->launches += 2;
  return PCT_OK;
}

pct_status pct_block_weights(pct_ctx* c) {
  pct::TraceRange trace_("pct_block_weights");
  if (!c) return fail(PCT_ERR_INVALID_ARG, "ctx is NULL");
  if (!c->loaded) return fail(PCT_ERR_STATE, "no histories loaded");
  return pct::ensure_block_weights(c);
}

pct_status pct_set_x0(pct_ctx* c, const float* x0, int on_device) {
  if (!c || !x0) return fail(PCT_ERR_INVALID_ARG, "ctx or x0 is NULL");
  pct::DeviceGuard device_guard_;
  PCT_CK(cudaSetDevice(c->device));
  PCT_CK(cudaMemcpyAsync(c->x, x0, (size_t)c->M * sizeof(float),
                         on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
  if (!on_device) return sync_and_check(c);
  return PCT_OK;
}

// The first sweep after a load adds each run's update and count by one vector
// reduction (pct::launch_drop_fused_pair) for one lane per history without a
// hull, CARP or TVS; the others count with integer atomics beside the update.
static bool paired_counting(const pct_ctx* c) {
  return c->cfg.threads_per_proton <= 1 && !c->hull_mask && !(c->cfg.flags & PCT_FLAG_CARP) &&
         !(c->cfg.tvs_beta0 > 0.f);
}

// One sweep as a CUDA graph. counting: the first sweep after a load also
// counts each block's runs (cnt) and forms its weights inv_s just before the
// block's update, in place of a separate counting pass.
static pct_status build_sweep_graph(pct_ctx* c, bool counting, cudaGraphExec_t* out) {
  cudaGraph_t graph = nullptr;
  cudaStream_t s = c->own_stream;
  PCT_CK(cudaStreamSynchronize(s));
  PCT_CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  cudaError_t err = cudaSuccess;
  const int B = c->cfg.n_blocks;
  const int clamp = (c->cfg.flags & PCT_FLAG_CLAMP) != 0;
  const bool carp = (c->cfg.flags & PCT_FLAG_CARP) != 0;
  const bool tvs = c->cfg.tvs_beta0 > 0.f;
  const pct::TvsParams tp{c->cfg.tvs_beta0, c->cfg.tvs_alpha, c->cfg.tvs_eps, c->cfg.tvs_tries};
  const size_t xbytes = (size_t)c->M * sizeof(float);
  if (tvs && carp)
    err = pct::launch_tvs(c->x, c->grid.nx, c->grid.ny, c->grid.nz, tp, c->tv_g, c->tv_xp, c->tv_acc, c->tv_state, s);
  if (carp && err == cudaSuccess) err = cudaMemcpyAsync(c->carp_x0, c->x, xbytes, cudaMemcpyDeviceToDevice, s);
  const bool pair = counting && paired_counting(c);
  if (pair) {
    // the image before the sweep (kept to redo it with integer counts), a clean
    // update-and-count array and overflow flag
    err = cudaMemcpyAsync(c->x_save, c->x, xbytes, cudaMemcpyDeviceToDevice, s);
    if (err == cudaSuccess) err = cudaMemsetAsync(c->pair, 0, (size_t)c->M * sizeof(float2), s);
    if (err == cudaSuccess) err = cudaMemsetAsync(c->pair_overflow, 0, sizeof(int), s);
  }
  const int S = carp ? c->cfg.carp_strings : 1;
  for (int st = 0; st < S && err == cudaSuccess; ++st) {
    // CARP: string st sweeps blocks [st B/S, (st+1) B/S) on a copy of the
    // iteration's starting image; DROP: one "string" of all blocks on x
    const int b0 = carp ? (int)((int64_t)st * B / S) : 0, b1 = carp ? (int)((int64_t)(st + 1) * B / S) : B;
    if (carp && st > 0) err = cudaMemcpyAsync(c->x, c->carp_x0, xbytes, cudaMemcpyDeviceToDevice, s);
    for (int b = b0; b < b1 && err == cudaSuccess; ++b) {
      const int64_t lo = block_lo(c, b), hi = block_lo(c, b + 1);
      if (tvs && !carp)
        err = pct::launch_tvs(c->x, c->grid.nx, c->grid.ny, c->grid.nz, tp, c->tv_g, c->tv_xp, c->tv_acc,
                              c->tv_state, s);
      if (pair) {
        if (err == cudaSuccess && c->ev) err = cudaEventRecordWithFlags(c->ev[3 * b], s, cudaEventRecordExternal);
        if (err == cudaSuccess)
          err = pct::launch_drop_fused_pair(c->geo, c->rec, c->tab32, lo, hi - lo, c->x, c->pair, c->cfg.lambda,
                                            c->cfg.flags, s);
        if (err == cudaSuccess && c->ev) err = cudaEventRecordWithFlags(c->ev[3 * b + 1], s, cudaEventRecordExternal);
        if (err == cudaSuccess)
          err = pct::launch_drop_apply_pair(c->x, c->pair, c->inv_s + (size_t)b * c->M, c->M, clamp, c->cfg.clamp_min,
                                            c->pair_overflow, s);
        if (err == cudaSuccess && c->ev) err = cudaEventRecordWithFlags(c->ev[3 * b + 2], s, cudaEventRecordExternal);
        continue;
      }
      if (err == cudaSuccess && counting) err = cudaMemsetAsync(c->cnt, 0, (size_t)c->M * sizeof(unsigned int), s);
      if (err == cudaSuccess && c->ev) err = cudaEventRecordWithFlags(c->ev[3 * b], s, cudaEventRecordExternal);
      if (err == cudaSuccess)
        err = pct::launch_drop_fused(c->geo, c->rec, c->tab32, pct::hull_view(c), lo, hi - lo, c->x, c->delta,
                                     c->cfg.lambda, c->cfg.flags, c->cfg.threads_per_proton, s, counting ? c->cnt : nullptr);
      if (err == cudaSuccess && c->ev) err = cudaEventRecordWithFlags(c->ev[3 * b + 1], s, cudaEventRecordExternal);
      if (err == cudaSuccess && counting) err = pct::launch_inv_counts(c->cnt, c->inv_s + (size_t)b * c->M, c->M, s);
      if (err == cudaSuccess)
        err = pct::launch_drop_apply(c->x, c->delta, c->inv_s + (size_t)b * c->M, c->M, carp ? 0 : clamp,
                                     c->cfg.clamp_min, s);
      if (err == cudaSuccess && c->ev) err = cudaEventRecordWithFlags(c->ev[3 * b + 2], s, cudaEventRecordExternal);
    }
    if (carp && err == cudaSuccess)
      err = pct::launch_carp_collect(c->x, c->inv_s + (size_t)b0 * c->M, b1 - b0, c->M, c->carp_sum, c->carp_touch, s);
  }
  if (carp && err == cudaSuccess)
    err = pct::launch_carp_finish(c->x, c->carp_x0, c->carp_sum, c->carp_touch, c->M, clamp, c->cfg.clamp_min, s);
  cudaError_t e2 = cudaStreamEndCapture(s, &graph);
  if (err != cudaSuccess || e2 != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    (void)cudaGetLastError();
    return fail(PCT_ERR_CUDA, "sweep capture: %s", cudaGetErrorString(err != cudaSuccess ? err : e2));
  }
  cudaError_t e3 = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  if (e3 != cudaSuccess) {
    *out = nullptr;
    return fail(PCT_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e3));
  }
  c->graph_n = c->n;
  c->graph_rec = c->rec;
  c->graph_range = pct::hull_view(c).range;
  return PCT_OK;
}

pct_status pct_iterate(pct_ctx* c, int32_t n_sweeps) {
  pct::TraceRange trace_("pct_iterate");
  if (!c) return fail(PCT_ERR_INVALID_ARG, "ctx is NULL");
  if (!c->loaded) return fail(PCT_ERR_STATE, "no histories loaded");
  if (n_sweeps < 0) return fail(PCT_ERR_INVALID_ARG, "n_sweeps < 0");
  pct::DeviceGuard device_guard_;
  PCT_CK(cudaSetDevice(c->device));
  if (n_sweeps == 0) return PCT_OK;
  // the capture stream must not have pending work from another stream
  if ((!c->sweep || !c->weights_ready) && c->stream != c->own_stream) PCT_CK(cudaStreamSynchronize(c->stream));
  const int64_t per_sweep = 2 * c->cfg.n_blocks + ((c->cfg.flags & PCT_FLAG_CARP) ? c->cfg.carp_strings + 1 : 0);
  if (!c->weights_ready) {
    // first sweep after a load: counts the block weights as it goes
    const bool pair = paired_counting(c);
    if (pair) {
      if (!c->pair) PCT_ALLOC(c->pair, (size_t)c->M * sizeof(float2));
      if (!c->pair_overflow) PCT_ALLOC(c->pair_overflow, sizeof(int));
      if (!c->x_save) PCT_ALLOC(c->x_save, (size_t)c->M * sizeof(float));
    }
    if (!c->sweep_count) {
      pct_status st = build_sweep_graph(c, true, &c->sweep_count);
      if (st != PCT_OK) return st;
    }
    PCT_CK(cudaGraphLaunch(c->sweep_count, c->stream));
    c->launches += pair ? per_sweep : per_sweep + c->cfg.n_blocks;
    bool redo = false;
    if (pair) {
      // a float count that reached 2^24 may have lost runs: undo the sweep,
      // form the weights with integer counts and sweep again
      int overflow = 0;
      PCT_CK(cudaMemcpyAsync(&overflow, c->pair_overflow, sizeof overflow, cudaMemcpyDeviceToHost, c->stream));
      PCT_CK(cudaStreamSynchronize(c->stream));
      if (overflow) {
        PCT_CK(cudaMemcpyAsync(c->x, c->x_save, (size_t)c->M * sizeof(float), cudaMemcpyDeviceToDevice, c->stream));
        pct_status st = block_weights(c);
        if (st != PCT_OK) return st;
        redo = true;
      }
    }
    c->weights_ready = true;
    c->swept = true;
    if (!redo) --n_sweeps;
  }
  if (n_sweeps > 0 && !c->sweep) {
    pct_status st = build_sweep_graph(c, false, &c->sweep);
    if (st != PCT_OK) return st;
  }
  for (int s = 0; s < n_sweeps; ++s) PCT_CK(cudaGraphLaunch(c->sweep, c->stream));
  c->launches += (int64_t)n_sweeps * per_sweep;
  if (n_sweeps > 0) c->swept = true;
  return PCT_OK;
}

pct_status pct_block_partial(pct_ctx* c, int32_t block, float* delta_out, float* counts_out) {
  if (!c || !delta_out) return fail(PCT_ERR_INVALID_ARG, "ctx or delta_out is NULL");
  if (!c->loaded) return fail(PCT_ERR_STATE, "no histories loaded");
  if (block < 0 || block >= c->cfg.n_blocks) return fail(PCT_ERR_INVALID_ARG, "block out of range");
  pct::DeviceGuard device_guard_;
  PCT_CK(cudaSetDevice(c->device));
  const int64_t lo = block_lo(c, block), hi = block_lo(c, block + 1);
  const size_t bytes = (size_t)c->M * sizeof(float);
  PCT_CK(cudaMemsetAsync(delta_out, 0, bytes, c->stream));
  if (counts_out) PCT_CK(cudaMemsetAsync(c->cnt, 0, (size_t)c->M * sizeof(unsigned int), c->stream));
  PCT_CK(pct::launch_drop_fused(c->geo, c->rec, c->tab32, pct::hull_view(c), lo, hi - lo, c->x, delta_out,
                                c->cfg.lambda, c->cfg.flags, c->cfg.threads_per_proton, c->stream,
                                counts_out ? c->cnt : nullptr));
  c->launches += 1;
  if (counts_out) {
    PCT_CK(pct::launch_counts_to_float(c->cnt, counts_out, c->M, c->stream));
    c->launches += 1;
  }
  return PCT_OK;
}

pct_status pct_block_apply(pct_ctx* c, const float* delta, const float* counts) {
  if (!c || !delta || !counts) return fail(PCT_ERR_INVALID_ARG, "ctx, delta or counts is NULL");
  pct::DeviceGuard device_guard_;
  PCT_CK(cudaSetDevice(c->device));
  PCT_CK(pct::launch_apply_reduced(c->x, delta, counts, c->M, (c->cfg.flags & PCT_FLAG_CLAMP) != 0, c->cfg.clamp_min,
                                   c->stream));
  c->launches += 1;
  return PCT_OK;
}

pct_status pct_last_sweep_times(pct_ctx* c, float* fused_ms, float* apply_ms) {
  if (!c) return fail(PCT_ERR_INVALID_ARG, "ctx is NULL");
  if (!c->ev || !c->swept) return fail(PCT_ERR_STATE, "profiling off or no sweep run yet");
  pct::DeviceGuard device_guard_;
  PCT_CK(cudaSetDevice(c->device));
  pct_status st = sync_and_check(c);
  if (st != PCT_OK) return st;
  for (int b = 0; b < c->cfg.n_blocks; ++b) {
    float f = 0.f, a = 0.f;
    PCT_CK(cudaEventElapsedTime(&f, c->ev[3 * b], c->ev[3 * b + 1]));
    PCT_CK(cudaEventElapsedTime(&a, c->ev[3 * b + 1], c->ev[3 * b + 2]));
    if (fused_ms) fused_ms[b] = f;
    if (apply_ms) apply_ms[b] = a;
  }
  return PCT_OK;
}

pct_status pct_get_rsp(pct_ctx* c, float* out, int to_device) {
  if (!c || !out) return fail(PCT_ERR_INVALID_ARG, "ctx or out is NULL");
  pct::DeviceGuard device_guard_;
  PCT_CK(cudaSetDevice(c->device));
  if (to_device) {
    PCT_CK(cudaMemcpyAsync(out, c->x, (size_t)c->M * sizeof(float), cudaMemcpyDeviceToDevice, c->stream));
    return PCT_OK;
  }
  // Wait for the queued sweeps first, then copy: a copy to pageable host
  // memory queued behind a long run of sweeps finished measurably later
  // (about 0.19 s after 10 sweeps of 50M histories) than this order.
  pct_status st = sync_and_check(c);
  if (st != PCT_OK) return st;
  PCT_CK(cudaMemcpyAsync(out, c->x, (size_t)c->M * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
  return sync_and_check(c);
}

pct_status pct_sync(pct_ctx* c) {
  if (!c) return fail(PCT_ERR_INVALID_ARG, "ctx is NULL");
  pct::DeviceGuard device_guard_;
  PCT_CK(cudaSetDevice(c->device));
  return sync_and_check(c);
}

int64_t pct_launch_count(const pct_ctx* c) { return c ? c->launches : 0; }

}  // extern "C"
