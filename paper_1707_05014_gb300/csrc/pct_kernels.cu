// Hot-path kernels: record validation, per-block run counts, the fused
// MLP + DROP projection kernel (and its first-sweep variant that also counts
// the block weights), the block apply, CARP, TVS, projection and residual,
// the CSR row export and the load-time ordering.
//
// DROP (arXiv 1707.05014 Sec. 2.1, Fig. 1), block b:
//   for i in b:  r_i = lambda (b_i - a_i.x) / |a_i|^2,  delta += r_i a_i
//   x_j += delta_j / s_j     (s_j = number of runs of block b in voxel j)
// The fused kernel walks each row a_i from the MLP once per sweep, keeps it
// in thread-local memory for the gather of a_i.x and the scatter, and never
// stores it across sweeps.
#include "pct_drop.cuh"

namespace pct {
namespace {

__device__ __forceinline__ void load_table(const float4* __restrict__ src, float4* dst, int n) {
  for (int k = threadIdx.x; k < n; k += blockDim.x) dst[k] = src[k];
  __syncthreads();
}

__device__ __forceinline__ bool bad_float(float v) { return !isfinite(v); }

__global__ void validate_kernel(Rec r, int64_t n, int64_t base, float pos_limit, unsigned long long* first_bad) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const RecV v = load_rec(r, i);
  bool bad = bad_float(v.t0) || bad_float(v.v0) || bad_float(v.st0) || bad_float(v.sv0) || bad_float(v.t2) ||
             bad_float(v.v2) || bad_float(v.st2) || bad_float(v.sv2) || bad_float(v.wepl) || bad_float(v.cp) ||
             bad_float(v.sp);
  bad = bad || fabsf(v.st0) >= 0.5f || fabsf(v.sv0) >= 0.5f || fabsf(v.st2) >= 0.5f || fabsf(v.sv2) >= 0.5f;
  bad = bad || fabsf(v.t0) > pos_limit || fabsf(v.v0) > pos_limit || fabsf(v.t2) > pos_limit ||
        fabsf(v.v2) > pos_limit;
  bad = bad || v.wepl < 0.f || fabsf(v.cp * v.cp + v.sp * v.sp - 1.f) > 1e-3f;
  if (bad) atomicMin(first_bad, (unsigned long long)(base + i));
}

__global__ void count_kernel(Geo g, Rec r, const float4* __restrict__ tab_g, Hull hull, int64_t first,
                             int64_t count, unsigned int* __restrict__ cnt) {
  extern __shared__ float4 tab[];
  load_table(tab_g, tab, g.K + 1);
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= count) return;
  const RecV v = load_rec(r, first + p);
  walk_any(g, tab, hull, first + p, v, [&](int j, float) { atomicAdd(cnt + j, 1u); });
}

__global__ void inv_counts_kernel(const unsigned int* __restrict__ cnt, float* __restrict__ inv_s, int64_t M) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= M) return;
  unsigned c = cnt[j];
  inv_s[j] = c ? 1.0f / (float)c : 0.0f;
}

__global__ void counts_to_float_kernel(const unsigned int* __restrict__ cnt, float* __restrict__ out, int64_t M) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= M) return;
  out[j] = (float)cnt[j];
}

// One thread per proton (see drop_history); kPlain: PCT_FLAG_NO_KAHAN.
template <bool kPlain>
__global__ void __launch_bounds__(128, 9) drop_fused_kernel(Geo g, Rec r, const float4* __restrict__ tab_g,
                                                          int64_t first, int64_t count, const float* __restrict__ x,
                                                          float* __restrict__ delta, float lambda) {
  extern __shared__ float4 tab[];
  load_table(tab_g, tab, g.K + 1);
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= count) return;
  drop_history<false, kPlain>(g, tab, r, first + p, x, delta, lambda);
}

// The same that also counts the block's runs per voxel into cnt (the first
// sweep after a load forms the DROP weights this way).
template <bool kPlain>
__global__ void __launch_bounds__(128, 9) drop_fused_count_kernel(Geo g, Rec r, const float4* __restrict__ tab_g,
                                                                int64_t first, int64_t count,
                                                                const float* __restrict__ x, float* __restrict__ delta,
                                                                float lambda, unsigned int* __restrict__ cnt) {
  extern __shared__ float4 tab[];
  load_table(tab_g, tab, g.K + 1);
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= count) return;
  drop_history_count<kPlain>(g, tab, r, first + p, x, delta, lambda, cnt);
}

// The counting sweep's kernel without a hull: the block's update and run
// counts go to pair, (a_ij r_i, 1) per run in one vector reduction.
template <bool kPlain>
__global__ void __launch_bounds__(128, 9) drop_fused_pair_kernel(Geo g, Rec r, const float4* __restrict__ tab_g,
                                                               int64_t first, int64_t count,
                                                               const float* __restrict__ x, float lambda,
                                                               float2* __restrict__ pair) {
  extern __shared__ float4 tab[];
  load_table(tab_g, tab, g.K + 1);
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= count) return;
  drop_history_pair<kPlain>(g, tab, r, first + p, x, lambda, pair);
}

// The counting sweep's block update: (delta_j, s_j) = pair[j]; 1/s_j into
// inv_s (0 where no run counted), x_j += delta_j / s_j (optionally clamped),
// pair[j] = 0. A float count is exact below 2^24; a count that reached 2^24
// may have lost runs, which sets *overflow.
__global__ void drop_apply_pair_kernel(float* __restrict__ x, float2* __restrict__ pair, float* __restrict__ inv_s,
                                       int64_t M, int clamp, float clamp_min, int* __restrict__ overflow) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= M) return;
  const float2 dc = pair[j];
  if (dc.y >= 16777216.f) atomicOr(overflow, 1);
  const float inv = dc.y > 0.f ? 1.0f / dc.y : 0.0f;
  inv_s[j] = inv;
  float xv = __fmaf_rn(dc.x, inv, x[j]);
  if (clamp) xv = fmaxf(xv, clamp_min);
  x[j] = xv;
  pair[j] = make_float2(0.f, 0.f);
}

// The same with an object hull (see walk_proton_hull). PCT_HULL_MIN_CTAS:
// resident 128-thread CTAs per SM its register allocation must allow.
#ifndef PCT_HULL_MIN_CTAS
#define PCT_HULL_MIN_CTAS 9
#endif
template <bool kPlain>
__global__ void __launch_bounds__(128, PCT_HULL_MIN_CTAS)
    drop_fused_hull_kernel(Geo g, Rec r, Hull hull, int64_t first, int64_t count, const float* __restrict__ x,
                           float* __restrict__ delta, float lambda) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= count) return;
  drop_history_hull<kPlain>(g, hull, r, first + p, x, delta, lambda);
}

template <bool kPlain>
__global__ void __launch_bounds__(128, PCT_HULL_MIN_CTAS)
    drop_fused_hull_count_kernel(Geo g, Rec r, Hull hull, int64_t first, int64_t count, const float* __restrict__ x,
                                 float* __restrict__ delta, float lambda, unsigned int* __restrict__ cnt) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= count) return;
  drop_history_hull_count<kPlain>(g, hull, r, first + p, x, delta, lambda, cnt);
}

// Compensated a_i.x (or plain with flags & 2), the arithmetic of the fused
// kernel's first pass. Returns y - c (Kahan: the true sum is y - c).
__device__ __forceinline__ float project_history(const Geo& g, const float4* __restrict__ tab, const Hull& hull,
                                                 int64_t i, const RecV& v, const float* __restrict__ x, int flags) {
  float y = 0.f, c = 0.f;
  if (flags & 2) {
    walk_any(g, tab, hull, i, v, [&](int j, float l) { y = __fmaf_rn(l, __ldg(x + j), y); });
    return y;
  }
  walk_any(g, tab, hull, i, v, [&](int j, float l) {
    const float term = __fsub_rn(__fmul_rn(l, __ldg(x + j)), c);
    const float t = __fadd_rn(y, term);
    c = __fsub_rn(__fsub_rn(t, y), term);
    y = t;
  });
  return __fsub_rn(y, c);
}

__global__ void __launch_bounds__(128) project_kernel(Geo g, Rec r, const float4* __restrict__ tab_g, Hull hull,
                                                      int64_t first, int64_t count, const int64_t* __restrict__ where,
                                                      const float* __restrict__ x, int flags, float* __restrict__ y) {
  extern __shared__ float4 tab[];
  load_table(tab_g, tab, g.K + 1);
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= count) return;
  const int64_t i = where ? where[first + p] : first + p;
  const RecV v = load_rec(r, i);
  y[p] = project_history(g, tab, hull, i, v, x, flags);
}

// sum over i = 0, stride, 2 stride, ... < n of (b_i - a_i.x)^2: per-CTA
// double reduction, one double atomic per CTA.
__global__ void __launch_bounds__(128) residual_kernel(Geo g, Rec r, const float4* __restrict__ tab_g, Hull hull,
                                                       int64_t n, int64_t stride, const float* __restrict__ x,
                                                       int flags, double* acc) {
  extern __shared__ float4 tab[];
  __shared__ double part[4];
  load_table(tab_g, tab, g.K + 1);
  int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * stride;
  double rr = 0.0;
  if (p < n) {
    const RecV v = load_rec(r, p);
    const double res = (double)v.wepl - (double)project_history(g, tab, hull, p, v, x, flags);
    rr = res * res;
  }
  for (int o = 16; o > 0; o >>= 1) rr += __shfl_down_sync(0xffffffffu, rr, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = rr;
  __syncthreads();
  if (threadIdx.x == 0) atomicAdd(acc, part[0] + part[1] + part[2] + part[3]);
}

__global__ void drop_apply_kernel(float* __restrict__ x, float* __restrict__ delta, const float* __restrict__ inv_s,
                                  int64_t M, int clamp, float clamp_min) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= M) return;
  apply_voxel(x, delta, inv_s, j, clamp, clamp_min);
}

// DROP block update from a block's update buffer and run counts summed over
// the ranks that share the block (Sec. 1 / 3.1: the data are distributed over
// processors): the same arithmetic as apply_voxel with 1/s_j formed here.
__global__ void apply_reduced_kernel(float* __restrict__ x, const float* __restrict__ delta,
                                     const float* __restrict__ counts, int64_t M, int clamp, float clamp_min) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= M) return;
  const float s = counts[j];
  float xv = __fmaf_rn(delta[j], s > 0.f ? 1.0f / s : 0.0f, x[j]);
  if (clamp) xv = fmaxf(xv, clamp_min);
  x[j] = xv;
}

// CARP (Sec. 2.2): after string s has swept its blocks on the working copy
// x_s, add it to the per-voxel sum where the string touched the voxel (any of
// its blocks has s_j > 0).
__global__ void carp_collect_kernel(const float* __restrict__ xs, const float* __restrict__ inv_s, int nb, int64_t M,
                                    float* __restrict__ sum, float* __restrict__ touch) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= M) return;
  bool hit = false;
  for (int b = 0; b < nb && !hit; ++b) hit = inv_s[(int64_t)b * M + j] > 0.f;
  if (hit) {
    sum[j] += xs[j];
    touch[j] += 1.f;
  }
}

// Component average: x_j = sum_j / touch_j where any string touched j, else
// the iteration's starting value; sum = touch = 0.
__global__ void carp_finish_kernel(float* __restrict__ x, const float* __restrict__ x0, float* __restrict__ sum,
                                   float* __restrict__ touch, int64_t M, int clamp, float clamp_min) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= M) return;
  const float t = touch[j];
  float xv = t > 0.f ? sum[j] / t : x0[j];
  if (clamp) xv = fmaxf(xv, clamp_min);
  x[j] = xv;
  sum[j] = 0.f;
  touch[j] = 0.f;
}

// ---- total-variation superiorization (TVS, Sec. 4.2) ----------------------
// TV_eps(x) = sum_v sqrt(dx^2 + dy^2 + dz^2 + eps^2), forward differences, 0
// across the far boundary. All decisions stay on the device (graph-safe).

__device__ __forceinline__ float tv_term(const float* __restrict__ x, int i, int j, int k, int nx, int ny, int nz,
                                         float eps) {
  const int64_t v = i + (int64_t)nx * (j + (int64_t)ny * k);
  const float xv = x[v];
  const float dx = i + 1 < nx ? x[v + 1] - xv : 0.f;
  const float dy = j + 1 < ny ? x[v + nx] - xv : 0.f;
  const float dz = k + 1 < nz ? x[v + (int64_t)nx * ny] - xv : 0.f;
  return sqrtf(dx * dx + dy * dy + dz * dz + eps * eps);
}

__device__ __forceinline__ void block_add2(double a, double b, double* out) {
  __shared__ double sa[8], sb[8];
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    sa[w] = a;
    sb[w] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ta = 0.0, tb = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
      ta += sa[q];
      tb += sb[q];
    }
    atomicAdd(out, ta);  // out[0] accumulates a, out[1] b
    atomicAdd(out + 1, tb);
  }
}

// g = grad TV_eps(x); acc[0] += |g|^2, acc[1] += TV(x)
__global__ void __launch_bounds__(256) tv_grad_kernel(const float* __restrict__ x, int nx, int ny, int nz, float eps,
                                                      float* __restrict__ g, double* acc) {
  const int64_t M = (int64_t)nx * ny * nz;
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double gg = 0.0, tv = 0.0;
  if (v < M) {
    const int i = (int)(v % nx), j = (int)((v / nx) % ny), k = (int)(v / ((int64_t)nx * ny));
    const float xv = x[v];
    const float t = tv_term(x, i, j, k, nx, ny, nz, eps);
    float gr = 0.f;
    if (i + 1 < nx) gr -= (x[v + 1] - xv) / t;
    if (j + 1 < ny) gr -= (x[v + nx] - xv) / t;
    if (k + 1 < nz) gr -= (x[v + (int64_t)nx * ny] - xv) / t;
    if (i > 0) gr += (xv - x[v - 1]) / tv_term(x, i - 1, j, k, nx, ny, nz, eps);
    if (j > 0) gr += (xv - x[v - nx]) / tv_term(x, i, j - 1, k, nx, ny, nz, eps);
    if (k > 0) gr += (xv - x[v - (int64_t)nx * ny]) / tv_term(x, i, j, k - 1, nx, ny, nz, eps);
    g[v] = gr;
    gg = (double)gr * gr;
    tv = t;
  }
  block_add2(gg, tv, acc);
}

// trial x' = x - beta_l g / rms(g), beta_l = beta0 alpha^l (skipped once accepted)
__global__ void tv_trial_kernel(const float* __restrict__ x, const float* __restrict__ g, float* __restrict__ xp,
                                int64_t M, const double* __restrict__ acc, const TvState* __restrict__ st,
                                float beta0, float alpha) {
  if (st->accepted) return;
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= M) return;
  const double rms = sqrt(acc[0] / (double)M);
  if (!(rms > 0.0)) return;
  const float beta = (float)((double)beta0 * pow((double)alpha, (double)st->ell));
  xp[v] = x[v] - beta * (float)((double)g[v] / rms);
}

// acc[2] += TV(x') (skipped once accepted)
__global__ void __launch_bounds__(256) tv_value_kernel(const float* __restrict__ xp, int nx, int ny, int nz, float eps,
                                                       double* acc, const TvState* __restrict__ st) {
  if (st->accepted) return;
  const int64_t M = (int64_t)nx * ny * nz;
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double tv = 0.0;
  if (v < M) {
    const int i = (int)(v % nx), j = (int)((v / nx) % ny), k = (int)(v / ((int64_t)nx * ny));
    tv = tv_term(xp, i, j, k, nx, ny, nz, eps);
  }
  for (int o = 16; o > 0; o >>= 1) tv += __shfl_down_sync(0xffffffffu, tv, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(acc + 2, tv);
}

// one thread: count the trial, accept if TV(x') <= TV(x)
__global__ void tv_decide_kernel(double* acc, TvState* st) {
  if (!st->accepted && acc[0] > 0.0) {
    st->ell += 1;
    if (acc[2] <= acc[1]) st->accepted = 1;
  }
  acc[2] = 0.0;
}

// x = x' if a trial was accepted; reset the per-application state
__global__ void tv_commit_kernel(float* __restrict__ x, const float* __restrict__ xp, int64_t M, TvState* st,
                                 double* acc) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v < M && st->accepted) x[v] = xp[v];
}

__global__ void tv_reset_kernel(double* acc, TvState* st) {
  acc[0] = acc[1] = acc[2] = 0.0;
  st->accepted = 0;
}

__global__ void row_count_kernel(Geo g, Rec r, const float4* __restrict__ tab_g, Hull hull, int64_t first,
                                 int64_t count, const int64_t* __restrict__ where, int64_t* __restrict__ row_ptr) {
  extern __shared__ float4 tab[];
  load_table(tab_g, tab, g.K + 1);
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= count) return;
  const int64_t i = where ? where[first + p] : first + p;
  const RecV v = load_rec(r, i);
  int64_t n = 0;
  walk_any(g, tab, hull, i, v, [&](int, float) { ++n; });
  row_ptr[p + 1] = n;
}

// In-place inclusive scan of row_ptr[1..count]; row_ptr[0] = 0. One CTA of
// 1024 threads, each owning a contiguous chunk (sized for the row export).
__global__ void __launch_bounds__(1024) scan_rows_kernel(int64_t* __restrict__ rp, int64_t count) {
  __shared__ long long sums[1024];
  const int t = threadIdx.x;
  const int64_t per = (count + 1023) / 1024;
  const int64_t lo = min((int64_t)t * per, count), hi = min(lo + per, count);
  long long s = 0;
  for (int64_t i = lo; i < hi; ++i) s += rp[1 + i];
  sums[t] = s;
  __syncthreads();
  if (t == 0) {
    long long acc = 0;
    for (int q = 0; q < 1024; ++q) {
      long long w = sums[q];
      sums[q] = acc;
      acc += w;
    }
    rp[0] = 0;
  }
  __syncthreads();
  long long acc = sums[t];
  for (int64_t i = lo; i < hi; ++i) {
    acc += rp[1 + i];
    rp[1 + i] = acc;
  }
}

__global__ void row_fill_kernel(Geo g, Rec r, const float4* __restrict__ tab_g, Hull hull, int64_t first,
                                int64_t count, const int64_t* __restrict__ where, const int64_t* __restrict__ row_ptr,
                                int32_t* __restrict__ vox, float* __restrict__ len, int32_t* __restrict__ nodes) {
  extern __shared__ float4 tab[];
  load_table(tab_g, tab, g.K + 1);
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= count) return;
  const int64_t i = where ? where[first + p] : first + p;
  const RecV v = load_rec(r, i);
  int64_t o = row_ptr[p];
  walk_any(g, tab, hull, i, v, [&](int j, float l) {
    vox[o] = j;
    len[o] = l;
    ++o;
  });
  if (nodes) {
    int32_t* out = nodes + (int64_t)p * (g.K + 1) * 3;
    const int32_t range = hull.range ? hull.range[i] : 0;
    for (int k = 0; k <= g.K; ++k) {
      const int3 Q = hull.range ? node_q_hull(g, hull.fam, range, v, k) : node_q(g, tab, v, k);
      out[3 * k + 0] = Q.x;
      out[3 * k + 1] = Q.y;
      out[3 * k + 2] = Q.z;
    }
  }
}


// ---- load-time ordering of each block: (gantry-angle bin, lateral bin of the
// path's midpoint, bin of its lateral change), so that the 32 lanes of a warp
// trace nearly the same path and cross the same faces at the same node steps.
// Counting sort: key -> histogram -> exclusive scan -> scatter.
//
// The key samples each history's own MLP (Sec. 2) at the quarter points of the
// slab, nodes k1 = K/4 and k3 = K - K/4 (lateral positions ta, tc, from the
// FP32 table). Two paths of one angle whose (ta + tc)/2 differ by dm and whose
// tc - ta differ by dd are about |dm| + |dd| u/R apart at depth u, the scattering
// slopes included; the bins are 1024 over the validated lateral range for the
// midpoint (0.49 mm on the 200x200x48 grid) and 32 over +-8 mm for the change
// (0.5 mm). On the 1e9-history head workload (90 angles, 2.2e5 histories per
// angle and block) a central bin holds about a warp's worth of histories.
__global__ void sort_key_kernel(Rec r, int64_t n, int n_ang, int n_lat, float lat_lim, const float4* __restrict__ tab,
                                int k1, int k3, unsigned* __restrict__ key) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float two_pi = 6.283185307f;
  float a = atan2f(r.sphi[i], r.cphi[i]);
  if (a < 0.f) a += two_pi;
  int ab = min(n_ang - 1, max(0, (int)(a * (n_ang / two_pi) + 0.5f) % n_ang));
  const float t0 = r.t0[i], t2 = r.t2[i], st0 = r.st0[i], st2 = r.st2[i];
  const float4 c1 = __ldg(tab + k1), c3 = __ldg(tab + k3);
  const float ta = fmaf(c1.w, st2, fmaf(c1.z, t2, fmaf(c1.y, st0, c1.x * t0)));
  const float tc = fmaf(c3.w, st2, fmaf(c3.z, t2, fmaf(c3.y, st0, c3.x * t0)));
  const float tmid = 0.5f * (ta + tc);
  int tb = (int)floorf((tmid + lat_lim) * (kSortMid / (2.f * lat_lim)));
  tb = min(kSortMid - 1, max(0, tb));
  int db = (int)floorf((tc - ta + kSortDiffLim) * (kSortDiff / (2.f * kSortDiffLim)));
  db = min(kSortDiff - 1, max(0, db));
  key[i] = (unsigned)(ab * n_lat + tb * kSortDiff + db);
}

__global__ void histogram_kernel(const unsigned* __restrict__ key, int64_t n, unsigned* __restrict__ hist) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  atomicAdd(hist + key[i], 1u);
}

// Exclusive scan of hist[0..nb) in place, in three launches: every CTA sums
// one tile of kScanTile bins (coalesced), one CTA scans the tile sums, and
// every CTA scans its tile from its offset. kScanThreads threads, each
// holding kScanTile / kScanThreads consecutive bins.
constexpr int kScanThreads = 256;
constexpr int kScanPer = 16;
constexpr int kScanTile = kScanThreads * kScanPer;  // 4096 bins
constexpr int kScanMaxTiles = 1024;                 // nb <= 4M bins

__device__ __forceinline__ unsigned block_excl_scan(unsigned v, unsigned* sh, unsigned& total) {
  // Hillis-Steele over the warp, then over the warp sums
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const unsigned y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) sh[w] = x;
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    unsigned s = lane < nw ? sh[lane] : 0u;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, s, d);
      if (lane >= d) s += y;
    }
    if (lane < nw) sh[lane] = s;
  }
  __syncthreads();
  total = sh[(blockDim.x >> 5) - 1];
  const unsigned before = w > 0 ? sh[w - 1] : 0u;
  __syncthreads();
  return before + x - v;
}

__global__ void __launch_bounds__(kScanThreads) scan_tile_sums_kernel(const unsigned* __restrict__ hist, int nb,
                                                                      unsigned* __restrict__ tile_sum) {
  __shared__ unsigned sh[32];
  const int base = blockIdx.x * kScanTile;
  unsigned s = 0;
  for (int q = threadIdx.x; q < kScanTile; q += kScanThreads)
    if (base + q < nb) s += hist[base + q];
  unsigned total;
  block_excl_scan(s, sh, total);
  if (threadIdx.x == 0) tile_sum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanMaxTiles) scan_tile_offsets_kernel(unsigned* __restrict__ tile_sum, int nt) {
  __shared__ unsigned sh[32];
  const unsigned v = threadIdx.x < nt ? tile_sum[threadIdx.x] : 0u;
  unsigned total;
  const unsigned ex = block_excl_scan(v, sh, total);
  if (threadIdx.x < nt) tile_sum[threadIdx.x] = ex;
}

__global__ void __launch_bounds__(kScanThreads) scan_tiles_kernel(unsigned* __restrict__ hist, int nb,
                                                                  const unsigned* __restrict__ tile_off) {
  __shared__ unsigned tile[kScanTile];
  __shared__ unsigned sh[32];
  const int base = blockIdx.x * kScanTile;
  for (int q = threadIdx.x; q < kScanTile; q += kScanThreads) tile[q] = base + q < nb ? hist[base + q] : 0u;
  __syncthreads();
  unsigned v[kScanPer];
  unsigned s = 0;
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    v[k] = tile[threadIdx.x * kScanPer + k];
    s += v[k];
  }
  unsigned total;
  unsigned acc = tile_off[blockIdx.x] + block_excl_scan(s, sh, total);
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    tile[threadIdx.x * kScanPer + k] = acc;
    acc += v[k];
  }
  __syncthreads();
  for (int q = threadIdx.x; q < kScanTile; q += kScanThreads)
    if (base + q < nb) hist[base + q] = tile[q];
}

// Counting-sort placement of record i: its stored position p (the next slot
// of its bin), order[p] = i, and where[base + i] = base + p (written here, in
// load order, so that the map is stored with coalesced writes).
__global__ void scatter_kernel(const unsigned* __restrict__ key, int64_t n, int64_t base, unsigned* __restrict__ offs,
                               unsigned* __restrict__ order, int64_t* __restrict__ where) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const unsigned p = atomicAdd(offs + key[i], 1u);
  order[p] = (unsigned)i;
  where[base + i] = base + p;
}

__device__ __forceinline__ const float* field_of(const Rec& r, int f) {
  switch (f) {
    case 0: return r.t0;
    case 1: return r.v0;
    case 2: return r.st0;
    case 3: return r.sv0;
    case 4: return r.t2;
    case 5: return r.v2;
    case 6: return r.st2;
    case 7: return r.sv2;
    case 8: return r.wepl;
    case 9: return r.cphi;
    default: return r.sphi;
  }
}

// dst.f[base + p] = src.f[order[p]] (order null: src.f[p]) for record field
// f = blockIdx.y. The CTAs of one field are dispatched before those of the
// next, so the random reads of a block's reordering stay within one field
// (4 B per record: 80 MB for 20M records), which the L2 holds, instead of
// spreading over all eleven.
__global__ void gather_kernel(Rec src, Rec dst, const unsigned* __restrict__ order, int64_t n, int64_t base) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int f = blockIdx.y;
  const int64_t i = order ? (int64_t)order[p] : p;
  const_cast<float*>(field_of(dst, f))[base + p] = field_of(src, f)[i];
}

inline unsigned grid_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

}  // namespace

cudaError_t launch_sort_block(const Rec& src, int64_t n, int64_t base, float lat_lim, const float4* tab, int K,
                              Rec dst_rec, int64_t* where, unsigned* key, unsigned* hist, unsigned* order,
                              cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int n_ang = kSortAngles, n_lat = kSortLateral;
  cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(unsigned) * n_ang * n_lat, s);
  if (e != cudaSuccess) return e;
  sort_key_kernel<<<grid_for(n, 256), 256, 0, s>>>(src, n, n_ang, n_lat, lat_lim, tab, K / 4, K - K / 4, key);
  histogram_kernel<<<grid_for(n, 256), 256, 0, s>>>(key, n, hist);
  {
    const int nb = n_ang * n_lat, nt = (nb + kScanTile - 1) / kScanTile;
    static_assert((kSortAngles * kSortLateral + kScanTile - 1) / kScanTile <= kScanMaxTiles, "bins exceed the scan");
    unsigned* tile_sum = hist + nb;  // nt entries past the bins (the array holds kSortHistEntries)
    static_assert(kSortHistEntries >= (int64_t)kSortAngles * kSortLateral + kScanMaxTiles, "bin array too small");
    scan_tile_sums_kernel<<<nt, kScanThreads, 0, s>>>(hist, nb, tile_sum);
    scan_tile_offsets_kernel<<<1, kScanMaxTiles, 0, s>>>(tile_sum, nt);
    scan_tiles_kernel<<<nt, kScanThreads, 0, s>>>(hist, nb, tile_sum);
  }
  scatter_kernel<<<grid_for(n, 256), 256, 0, s>>>(key, n, base, hist, order, where);
  gather_kernel<<<dim3(grid_for(n, 256), 11), 256, 0, s>>>(src, dst_rec, order, n, base);
  return cudaGetLastError();
}

cudaError_t launch_copy_block(const Rec& src, int64_t n, int64_t base, Rec dst_rec, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  gather_kernel<<<dim3(grid_for(n, 256), 11), 256, 0, s>>>(src, dst_rec, nullptr, n, base);
  return cudaGetLastError();
}

cudaError_t launch_validate(const Rec& r, int64_t n, int64_t base, float pos_limit, unsigned long long* first_bad,
                            cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  validate_kernel<<<grid_for(n, 256), 256, 0, s>>>(r, n, base, pos_limit, first_bad);
  return cudaGetLastError();
}

cudaError_t launch_count(const Geo& g, const Rec& r, const float4* tab, const Hull& hull, int64_t first,
                         int64_t count, unsigned int* cnt, int threads, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  count_kernel<<<grid_for(count, threads), threads, (g.K + 1) * sizeof(float4), s>>>(g, r, tab, hull, first, count,
                                                                                      cnt);
  return cudaGetLastError();
}

cudaError_t launch_inv_counts(const unsigned int* cnt, float* inv_s, int64_t M, cudaStream_t s) {
  inv_counts_kernel<<<grid_for(M, 256), 256, 0, s>>>(cnt, inv_s, M);
  return cudaGetLastError();
}

cudaError_t launch_counts_to_float(const unsigned int* cnt, float* out, int64_t M, cudaStream_t s) {
  counts_to_float_kernel<<<grid_for(M, 256), 256, 0, s>>>(cnt, out, M);
  return cudaGetLastError();
}

cudaError_t launch_drop_fused(const Geo& g, const Rec& r, const float4* tab, const Hull& hull, int64_t first,
                              int64_t count, const float* x, float* delta, float lambda, int flags, int lanes,
                              cudaStream_t s, unsigned int* cnt) {
  if (count <= 0) return cudaSuccess;
  if (lanes > 1 && !hull.range) return launch_drop_group(lanes, g, r, tab, first, count, x, delta, lambda, flags, s, cnt);
  const int threads = 128;
  const unsigned blocks = grid_for(count, threads);
  const bool plain = (flags & 2) != 0;
  if (hull.range) {
    if (cnt) {
      if (plain)
        drop_fused_hull_count_kernel<true><<<blocks, threads, 0, s>>>(g, r, hull, first, count, x, delta, lambda, cnt);
      else
        drop_fused_hull_count_kernel<false><<<blocks, threads, 0, s>>>(g, r, hull, first, count, x, delta, lambda, cnt);
    } else {
      if (plain)
        drop_fused_hull_kernel<true><<<blocks, threads, 0, s>>>(g, r, hull, first, count, x, delta, lambda);
      else
        drop_fused_hull_kernel<false><<<blocks, threads, 0, s>>>(g, r, hull, first, count, x, delta, lambda);
    }
    return cudaGetLastError();
  }
  const size_t smem = (g.K + 1) * sizeof(float4);
  if (cnt) {
    if (plain)
      drop_fused_count_kernel<true><<<blocks, threads, smem, s>>>(g, r, tab, first, count, x, delta, lambda, cnt);
    else
      drop_fused_count_kernel<false><<<blocks, threads, smem, s>>>(g, r, tab, first, count, x, delta, lambda, cnt);
  } else {
    if (plain)
      drop_fused_kernel<true><<<blocks, threads, smem, s>>>(g, r, tab, first, count, x, delta, lambda);
    else
      drop_fused_kernel<false><<<blocks, threads, smem, s>>>(g, r, tab, first, count, x, delta, lambda);
  }
  return cudaGetLastError();
}

cudaError_t launch_drop_fused_pair(const Geo& g, const Rec& r, const float4* tab, int64_t first, int64_t count,
                                   const float* x, float2* pair, float lambda, int flags, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  const int threads = 128;
  const unsigned blocks = grid_for(count, threads);
  const size_t smem = (g.K + 1) * sizeof(float4);
  if (flags & 2)
    drop_fused_pair_kernel<true><<<blocks, threads, smem, s>>>(g, r, tab, first, count, x, lambda, pair);
  else
    drop_fused_pair_kernel<false><<<blocks, threads, smem, s>>>(g, r, tab, first, count, x, lambda, pair);
  return cudaGetLastError();
}

cudaError_t launch_drop_apply_pair(float* x, float2* pair, float* inv_s, int64_t M, int clamp, float clamp_min,
                                   int* overflow, cudaStream_t s) {
  drop_apply_pair_kernel<<<grid_for(M, 256), 256, 0, s>>>(x, pair, inv_s, M, clamp, clamp_min, overflow);
  return cudaGetLastError();
}

cudaError_t launch_project(const Geo& g, const Rec& r, const float4* tab, const Hull& hull, int64_t first,
                           int64_t count, const int64_t* where, const float* x, int flags, float* y, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  project_kernel<<<grid_for(count, 128), 128, (g.K + 1) * sizeof(float4), s>>>(g, r, tab, hull, first, count, where,
                                                                                x, flags, y);
  return cudaGetLastError();
}

cudaError_t launch_residual(const Geo& g, const Rec& r, const float4* tab, const Hull& hull, int64_t n, int64_t stride,
                            const float* x, int flags, double* acc, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int64_t m = (n + stride - 1) / stride;
  residual_kernel<<<grid_for(m, 128), 128, (g.K + 1) * sizeof(float4), s>>>(g, r, tab, hull, n, stride, x, flags,
                                                                             acc);
  return cudaGetLastError();
}

cudaError_t launch_drop_apply(float* x, float* delta, const float* inv_s, int64_t M, int clamp, float clamp_min,
                              cudaStream_t s) {
  drop_apply_kernel<<<grid_for(M, 256), 256, 0, s>>>(x, delta, inv_s, M, clamp, clamp_min);
  return cudaGetLastError();
}

cudaError_t launch_apply_reduced(float* x, const float* delta, const float* counts, int64_t M, int clamp,
                                 float clamp_min, cudaStream_t s) {
  apply_reduced_kernel<<<grid_for(M, 256), 256, 0, s>>>(x, delta, counts, M, clamp, clamp_min);
  return cudaGetLastError();
}

cudaError_t launch_carp_collect(const float* xs, const float* inv_s, int nb, int64_t M, float* sum, float* touch,
                                cudaStream_t s) {
  carp_collect_kernel<<<grid_for(M, 256), 256, 0, s>>>(xs, inv_s, nb, M, sum, touch);
  return cudaGetLastError();
}

cudaError_t launch_carp_finish(float* x, const float* x0, float* sum, float* touch, int64_t M, int clamp,
                               float clamp_min, cudaStream_t s) {
  carp_finish_kernel<<<grid_for(M, 256), 256, 0, s>>>(x, x0, sum, touch, M, clamp, clamp_min);
  return cudaGetLastError();
}

cudaError_t launch_tvs(float* x, int nx, int ny, int nz, const TvsParams& p, float* g, float* xp, double* acc,
                       TvState* st, cudaStream_t s) {
  const int64_t M = (int64_t)nx * ny * nz;
  const unsigned b = grid_for(M, 256);
  tv_grad_kernel<<<b, 256, 0, s>>>(x, nx, ny, nz, p.eps, g, acc);
  for (int t = 0; t < p.tries; ++t) {
    tv_trial_kernel<<<b, 256, 0, s>>>(x, g, xp, M, acc, st, p.beta0, p.alpha);
    tv_value_kernel<<<b, 256, 0, s>>>(xp, nx, ny, nz, p.eps, acc, st);
    tv_decide_kernel<<<1, 1, 0, s>>>(acc, st);
  }
  tv_commit_kernel<<<b, 256, 0, s>>>(x, xp, M, st, acc);
  tv_reset_kernel<<<1, 1, 0, s>>>(acc, st);
  return cudaGetLastError();
}

cudaError_t launch_row_counts(const Geo& g, const Rec& r, const float4* tab, const Hull& hull, int64_t first,
                              int64_t count, const int64_t* where, int64_t* row_ptr, int lanes, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  if (lanes > 1 && !hull.range)
    return launch_rows_group(lanes, g, r, tab, first, count, where, row_ptr, nullptr, nullptr, nullptr, false, s);
  row_count_kernel<<<grid_for(count, 128), 128, (g.K + 1) * sizeof(float4), s>>>(g, r, tab, hull, first, count,
                                                                                  where, row_ptr);
  return cudaGetLastError();
}

cudaError_t launch_scan_rows(int64_t* row_ptr, int64_t count, cudaStream_t s) {
  scan_rows_kernel<<<1, 1024, 0, s>>>(row_ptr, count);
  return cudaGetLastError();
}

cudaError_t launch_row_fill(const Geo& g, const Rec& r, const float4* tab, const Hull& hull, int64_t first,
                            int64_t count, const int64_t* where, const int64_t* row_ptr, int32_t* vox, float* len,
                            int32_t* nodes, int lanes, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  if (lanes > 1 && !hull.range)
    return launch_rows_group(lanes, g, r, tab, first, count, where, const_cast<int64_t*>(row_ptr), vox, len, nodes,
                             true, s);
  row_fill_kernel<<<grid_for(count, 128), 128, (g.K + 1) * sizeof(float4), s>>>(g, r, tab, hull, first, count,
                                                                                 where, row_ptr, vox, len, nodes);
  return cudaGetLastError();
}

}  // namespace pct
