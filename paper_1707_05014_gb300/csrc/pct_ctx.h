// Context object behind the C ABI's pct_ctx handle (shared by the library's
// translation units; not part of the ABI).
#pragma once

#include <stdint.h>

#include "../../include/pct.h"
#include "pct_internal.h"

struct pct_ctx {
  int device = 0;
  pct_grid grid{};
  pct_config cfg{};
  pct::Geo geo{};
  double R = 0, du = 0;
  int K = 0, E = 0;
  int64_t M = 0;
  float pos_limit = 0;
  cudaStream_t own_stream = nullptr;  // created by the context; also the capture stream
  cudaStream_t stream = nullptr;      // where work is queued
  double* tab64 = nullptr;
  float4* tab32 = nullptr;
  int64_t n = 0;
  float* rec_store = nullptr;  // owned copy of the 11 record arrays (null when borrowed)
  pct::Rec rec{};
  int64_t* where = nullptr;    // load index -> stored position (null: stored in load order)
  // Buffers of the loaded set, kept across loads and grown when a load needs
  // more (freed by pct_destroy): records, the load-order map, hull ranges,
  // and the load's scratch (host staging, sort keys, order, bins).
  int64_t rec_cap = 0, where_cap = 0, range_cap = 0, staging_cap = 0, key_cap = 0, order_cap = 0, hist_cap = 0;
  int64_t* where_buf = nullptr;
  float* staging = nullptr;   // two slots of the largest block's 11 arrays (host loads)
  // Host loads: the next block's copy (copy_stream) overlaps the current
  // block's validation and ordering (stream). load_ev[s]: slot s copied;
  // load_ev[2 + s]: slot s consumed. Created by the first host load.
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t load_ev[4] = {};
  unsigned* sort_key = nullptr;
  unsigned* sort_order = nullptr;
  unsigned* sort_hist = nullptr;
  float* x = nullptr;
  float* delta = nullptr;
  float* inv_s = nullptr;  // B x M
  unsigned int* cnt = nullptr;
  // The first sweep after a load without a hull, CARP or TVS: the block's
  // update and run counts side by side (M float2), a flag set where a float
  // count reached 2^24, and the image before that sweep (to redo it with exact
  // integer counts if the flag is set). Allocated by the first such sweep.
  float2* pair = nullptr;
  int* pair_overflow = nullptr;
  float* x_save = nullptr;
  unsigned long long* first_bad = nullptr;
  double* acc = nullptr;  // residual accumulator
  float* carp_sum = nullptr;    // CARP: sum of string estimates per voxel
  float* carp_touch = nullptr;  // CARP: number of strings touching each voxel
  float* carp_x0 = nullptr;     // CARP: the iteration's starting image
  float* tv_g = nullptr;        // TVS: gradient
  float* tv_xp = nullptr;       // TVS: trial image
  double* tv_acc = nullptr;     // TVS: |g|^2, TV(x), TV(x')
  pct::TvState* tv_state = nullptr;
  uint8_t* hull_mask = nullptr;   // object hull, M bytes (null: no hull)
  int32_t* hull_range = nullptr;  // per stored history: iin | iout << 16 (with a hull and histories)
  float4* fam32 = nullptr;        // MLP tables of every hull thickness (with a hull)
  bool weights_ready = false;  // inv_s holds the block weights of the loaded histories
  cudaGraphExec_t sweep = nullptr;
  cudaGraphExec_t sweep_count = nullptr;  // first sweep after a load (counts the block weights)
  // What the two sweep graphs captured: a reload with the same history count,
  // record storage and hull keeps them (no destroy and rebuild per load).
  int64_t graph_n = -1;
  pct::Rec graph_rec{};  // all eleven record pointers (a borrowed load may move any of them)
  const int32_t* graph_range = nullptr;
  cudaEvent_t* ev = nullptr;  // 3 per block (profiling): fused start, fused end, apply end
  bool swept = false;
  int64_t launches = 0;
  bool loaded = false;
  uint64_t generation = 0;  // bumped by every load and hull change (a batch checks it)
};

namespace pct {
// The hull as the kernels see it (range null: no hull).
inline Hull hull_view(const pct_ctx* c) { return Hull{c->hull_mask ? c->hull_range : nullptr, c->fam32}; }
// Compute the DROP block weights now if the first sweep has not done it yet
// (callers that read inv_s outside pct_iterate). Synchronises.
pct_status ensure_block_weights(pct_ctx* c);
// First history of DROP block b: b * n / B (blocks are contiguous ranges).
inline int64_t block_first(const pct_ctx* c, int b) { return (int64_t)b * c->n / c->cfg.n_blocks; }
}  // namespace pct
