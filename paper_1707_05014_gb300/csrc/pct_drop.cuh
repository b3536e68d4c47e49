// Per-history DROP contribution (arXiv 1707.05014 Sec. 2.1, Fig. 1):
//   r_i = lambda (b_i - a_i.x) / |a_i|^2,   delta_j += r_i a_ij
// with a_i the MLP row (Sec. 2) walked on the fly. Shared by the per-block
// kernel and the batched persistent kernel.
#pragma once

#include "pct_walk.cuh"

namespace pct {

// Plain (weak) global load, cached in L1. Written as PTX so the compiler
// cannot turn it into a read-only (non-coherent) load: under the PTX memory
// model a weak load ordered after an acquire (counter read + fence) and a CTA
// barrier observes every write released before that counter was set.
__device__ __forceinline__ float ld_weak(const float* p) {
  float v;
  asm("ld.global.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}

// pair[0] += u, pair[1] += 1 in one vector reduction (sm_90 and later).
__device__ __forceinline__ void red_add_pair(float2* p, float u) {
  asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(u), "f"(1.0f) : "memory");
}

// MLP nodes -> walk -> compensated a_i.x and |a_i|^2 -> relaxed residual ->
// scatter-add into delta. The walk only records the row (voxel, chord) in
// thread-local memory; the gather of x for a_i.x and the scatter replay the
// record, outside the walk's divergent crossing loop, so no lane waits on a
// global load inside the walk. A row longer than kRowCap runs (none for valid
// records on the supported grids) is walked again for the gather and for the
// scatter instead.
//
// kPlain: plain instead of compensated summation (PCT_FLAG_NO_KAHAN).
// kCoherent: x may change while the kernel runs (the batched persistent
// kernel applies block updates between work items), so x is read with plain
// weak loads instead of the read-only path (which assumes data that never
// changes during the launch).
// cnt (kCount): also add every run to the block's run counts s_j (the first
// sweep after a load forms the DROP weights this way), in the gather's replay
// of the row rather than inside the walk.
//
// pair (kPair, instead of delta and cnt): the update and the run count of
// voxel j side by side, (delta_j, s_j) = pair[j], both added by one vector
// reduction per run; the count is a float, exact while below 2^24 (the block
// update checks that). A history without runs of positive length adds zero
// updates but still counts its runs.
template <bool kCoherent, bool kPlain, bool kCount, class Walk, bool kPair = false>
__device__ __forceinline__ void drop_history_core(const RecV& v, Walk&& walk, const float* __restrict__ x,
                                                  float* __restrict__ delta, float lambda,
                                                  unsigned int* __restrict__ cnt = nullptr,
                                                  float2* __restrict__ pair = nullptr) {
  auto xload = [&](int j) { return kCoherent ? ld_weak(x + j) : __ldg(x + j); };
  uint2 row[kRowCap];
  int nrow = 0;
  walk([&](int j, float l) {
    if (nrow < kRowCap) row[nrow] = make_uint2((unsigned)j, __float_as_uint(l));
    ++nrow;
  });
  float y = 0.f, c = 0.f, nn = 0.f;
  auto gather = [&](int j, float l) {
    const float xj = xload(j);
    if (kPlain) {
      y = __fmaf_rn(l, xj, y);
    } else {
      // Kahan-compensated sum of l * x_j: the true sum is y - c
      const float term = __fsub_rn(__fmul_rn(l, xj), c);
      const float t = __fadd_rn(y, term);
      c = __fsub_rn(__fsub_rn(t, y), term);
      y = t;
    }
    nn = __fmaf_rn(l, l, nn);
  };
  if (nrow <= kRowCap) {
    for (int q = 0; q < nrow; ++q) {
      const uint2 e = row[q];
      if (kCount) atomicAdd(cnt + e.x, 1u);
      gather((int)e.x, __uint_as_float(e.y));
    }
  } else {
    walk([&](int j, float l) {
      if (kCount) atomicAdd(cnt + j, 1u);
      gather(j, l);
    });
  }
  if (kPair) {
    const float res = __fadd_rn(__fsub_rn(v.wepl, y), c);
    const float ri = nn > 0.f ? lambda * res / nn : 0.f;
    if (nrow <= kRowCap) {
      for (int q = 0; q < nrow; ++q) {
        const uint2 e = row[q];
        red_add_pair(pair + e.x, __uint_as_float(e.y) * ri);
      }
    } else {
      walk([&](int j, float l) { red_add_pair(pair + j, l * ri); });
    }
    return;
  }
  if (!(nn > 0.f)) return;
  const float res = __fadd_rn(__fsub_rn(v.wepl, y), c);
  const float ri = lambda * res / nn;
  if (nrow <= kRowCap) {
    for (int q = 0; q < nrow; ++q) {
      const uint2 e = row[q];
      atomicAdd(delta + e.x, __uint_as_float(e.y) * ri);
    }
  } else {
    walk([&](int j, float l) { atomicAdd(delta + j, l * ri); });
  }
}

template <bool kCoherent = false, bool kPlain = false>
__device__ __forceinline__ void drop_history(const Geo& g, const float4* __restrict__ tab, const Rec& r, int64_t i,
                                             const float* __restrict__ x, float* __restrict__ delta, float lambda) {
  const RecV v = load_rec(r, i);
  drop_history_core<kCoherent, kPlain, false>(v, [&](auto&& visit) { walk_proton(g, tab, v, visit); }, x, delta,
                                              lambda);
}

// The same with an object hull (the MLP between the proton's hull nodes).
template <bool kPlain = false>
__device__ __forceinline__ void drop_history_hull(const Geo& g, const Hull& hull, const Rec& r, int64_t i,
                                                  const float* __restrict__ x, float* __restrict__ delta, float lambda) {
  const RecV v = load_rec(r, i);
  const int32_t range = __ldg(hull.range + i);
  drop_history_core<false, kPlain, false>(v, [&](auto&& visit) { walk_proton_hull(g, hull.fam, range, v, visit); },
                                          x, delta, lambda);
}

// drop_history that also adds every run to cnt (the block's run counts s_j).
template <bool kPlain = false>
__device__ __forceinline__ void drop_history_count(const Geo& g, const float4* __restrict__ tab, const Rec& r, int64_t i,
                                                   const float* __restrict__ x, float* __restrict__ delta, float lambda,
                                                   unsigned int* __restrict__ cnt) {
  const RecV v = load_rec(r, i);
  drop_history_core<false, kPlain, true>(v, [&](auto&& visit) { walk_proton(g, tab, v, visit); }, x, delta, lambda,
                                         cnt);
}

// drop_history that adds (a_ij r_i, 1) to pair[j] for every run (the block's
// update and run counts side by side).
template <bool kPlain = false>
__device__ __forceinline__ void drop_history_pair(const Geo& g, const float4* __restrict__ tab, const Rec& r, int64_t i,
                                                  const float* __restrict__ x, float lambda, float2* __restrict__ pair) {
  const RecV v = load_rec(r, i);
  auto walk = [&](auto&& visit) { walk_proton(g, tab, v, visit); };
  drop_history_core<false, kPlain, false, decltype(walk)&, true>(v, walk, x, nullptr, lambda, nullptr, pair);
}

template <bool kPlain = false>
__device__ __forceinline__ void drop_history_hull_count(const Geo& g, const Hull& hull, const Rec& r, int64_t i,
                                                        const float* __restrict__ x, float* __restrict__ delta,
                                                        float lambda, unsigned int* __restrict__ cnt) {
  const RecV v = load_rec(r, i);
  const int32_t range = __ldg(hull.range + i);
  drop_history_core<false, kPlain, true>(v, [&](auto&& visit) { walk_proton_hull(g, hull.fam, range, v, visit); }, x,
                                         delta, lambda, cnt);
}

// x_j += delta_j / s_j (optionally clamped), delta_j = 0. kCoherent: x and
// delta are read and written at L2 (other CTAs of the same launch use them).
template <bool kCoherent = false>
__device__ __forceinline__ void apply_voxel(float* __restrict__ x, float* __restrict__ delta,
                                            const float* __restrict__ inv_s, int64_t j, int clamp, float clamp_min) {
  if (kCoherent) {
    float xv = __fmaf_rn(__ldcg(delta + j), inv_s[j], __ldcg(x + j));
    if (clamp) xv = fmaxf(xv, clamp_min);
    __stcg(x + j, xv);
    __stcg(delta + j, 0.f);
  } else {
    float xv = __fmaf_rn(delta[j], inv_s[j], x[j]);
    if (clamp) xv = fmaxf(xv, clamp_min);
    x[j] = xv;
    delta[j] = 0.f;
  }
}

}  // namespace pct
