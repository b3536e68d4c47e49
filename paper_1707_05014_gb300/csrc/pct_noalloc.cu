// pct_drop_block_noalloc: one DROP block update that allocates no memory.
//
// Some callers cannot allocate device memory once they are running: services
// that reserve the whole GPU for a fixed memory plan at start-up, or plugins
// whose host application owns every device allocation. They pass their own
// input and output buffers; the only other device memory this entry point
// touches is the fixed scratch array below, which lives in the library image
// (every GPU that loads the library holds it until the process exits).
#include <math.h>
#include <stdio.h>

#include "../../include/pct.h"
#include "pct_walk.cuh"

namespace {

using pct::Geo;
using pct::Rec;
using pct::RecV;

constexpr int64_t kMaxVoxels = (int64_t)1 << 21;  // 2,097,152 voxels
constexpr int kMaxNodes = pct::kMaxNodes;          // K + 1 <= 2048

// Scratch layout (byte offsets, each 256-byte aligned):
//   delta  : kMaxVoxels floats   (run counts as unsigned during the count pass)
//   inv_s  : kMaxVoxels floats   (1 / s_j)
//   tab64  : kMaxNodes * 4 doubles
//   tab32  : kMaxNodes float4
//   flag   : one unsigned long long (first invalid record)
constexpr size_t kOffDelta = 0;
constexpr size_t kOffInv = kOffDelta + kMaxVoxels * sizeof(float);
constexpr size_t kOffTab64 = kOffInv + kMaxVoxels * sizeof(float);
constexpr size_t kOffTab32 = kOffTab64 + kMaxNodes * 4 * sizeof(double);
constexpr size_t kOffFlag = kOffTab32 + kMaxNodes * sizeof(float4);
constexpr size_t kScratchBytes = kOffFlag + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Errors are reported through pct_last_error(), like every other entry point.
pct_status noalloc_fail(pct_status code, const char* msg, cudaError_t e = cudaSuccess) {
  char buf[256];
  if (e != cudaSuccess)
    snprintf(buf, sizeof buf, "%s: %s", msg, cudaGetErrorString(e));
  else
    snprintf(buf, sizeof buf, "%s", msg);
  pct::set_error_text(buf);
  return code;
}

// The two-pass fused kernel without a row cache: the scatter walks the path a
// second time, so the kernel needs no per-thread scratch either.
__global__ void __launch_bounds__(128) drop_fused_rewalk_kernel(Geo g, Rec r, const float4* __restrict__ tab_g,
                                                                 int64_t count, const float* __restrict__ x,
                                                                 float* __restrict__ delta, float lambda, int flags) {
  extern __shared__ float4 tab[];
  for (int k = threadIdx.x; k <= g.K; k += blockDim.x) tab[k] = tab_g[k];
  __syncthreads();
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= count) return;
  const RecV v = pct::load_rec(r, p);
  float y = 0.f, c = 0.f, nn = 0.f;
  if (flags & PCT_FLAG_NO_KAHAN) {
    pct::walk_proton(g, tab, v, [&](int j, float l) {
      y = __fmaf_rn(l, __ldg(x + j), y);
      nn = __fmaf_rn(l, l, nn);
    });
  } else {
    pct::walk_proton(g, tab, v, [&](int j, float l) {
      const float term = __fsub_rn(__fmul_rn(l, __ldg(x + j)), c);
      const float t = __fadd_rn(y, term);
      c = __fsub_rn(__fsub_rn(t, y), term);
      y = t;
      nn = __fmaf_rn(l, l, nn);
    });
  }
  if (!(nn > 0.f)) return;
  const float ri = lambda * __fadd_rn(__fsub_rn(v.wepl, y), c) / nn;
  pct::walk_proton(g, tab, v, [&](int j, float l) { atomicAdd(delta + j, l * ri); });
}

}  // namespace

extern "C" pct_status pct_drop_block_noalloc(const pct_grid* grid, const pct_config* cfg, const pct_histories* h,
                                             float* x, void* stream) {
  if (!grid || !cfg || !h || !x) return noalloc_fail(PCT_ERR_INVALID_ARG, "NULL argument");
  const pct_grid& gr = *grid;
  if (gr.nx < 1 || gr.ny < 1 || gr.nz < 1 || gr.nx > pct::kMaxDim || gr.ny > pct::kMaxDim || gr.nz > pct::kMaxDim)
    return noalloc_fail(PCT_ERR_INVALID_ARG, "grid dims must be in [1, 512]");
  if (!(gr.hx > 0 && gr.hy > 0 && gr.hz > 0) || !isfinite(gr.hx) || !isfinite(gr.hy) || !isfinite(gr.hz))
    return noalloc_fail(PCT_ERR_INVALID_ARG, "voxel sizes must be finite and > 0");
  const int64_t M = (int64_t)gr.nx * gr.ny * gr.nz;
  if (M > kMaxVoxels) return noalloc_fail(PCT_ERR_CAPACITY, "grid exceeds the fixed scratch (2,097,152 voxels)");
  if (!(cfg->lambda > 0.f && cfg->lambda < 2.f)) return noalloc_fail(PCT_ERR_INVALID_ARG, "lambda must be in (0, 2)");
  if (h->n < 1 || h->n >= ((int64_t)1 << 31)) return noalloc_fail(PCT_ERR_INVALID_ARG, "n must be in [1, 2^31)");
  const float* src[11] = {h->t0, h->v0, h->st0, h->sv0, h->t2, h->v2, h->st2, h->sv2, h->wepl, h->cphi, h->sphi};
  for (int f = 0; f < 11; ++f)
    if (!src[f]) return noalloc_fail(PCT_ERR_INVALID_ARG, "history array is NULL");

  // geometry (the same derivation as pct_create)
  const double X = gr.nx * gr.hx, Y = gr.ny * gr.hy, Z = gr.nz * gr.hz;
  const double hmin = fmin(gr.hx, fmin(gr.hy, gr.hz));
  const double step = cfg->node_step_mm > 0 ? cfg->node_step_mm : 0.5 * hmin;
  const double R = 0.5 * fmin(X, Y);
  const int K = (int)ceil(2.0 * R / step - 1e-9);
  if (K < 2 || K + 1 > kMaxNodes) return noalloc_fail(PCT_ERR_INVALID_ARG, "node count outside [3, 2048]");
  const double du = 2.0 * R / K;
  const int E = (int)ceil((0.5 * sqrt(X * X + Y * Y) - R) / du) + 2;
  const float pos_limit = (float)(0.5 * sqrt(X * X + Y * Y + Z * Z) + R);
  const double qmax = (R + (E + 1) * du + pos_limit + 0.5 * (2.0 * R + E * du)) / hmin +
                      0.5 * fmax((double)gr.nx, fmax((double)gr.ny, (double)gr.nz));
  if (qmax >= pct::kQClamp) return noalloc_fail(PCT_ERR_INVALID_ARG, "grid too large for the fixed-point node range");
  // dmax stays unbounded: every history takes the general walk (reading the
  // table back to bound its steps would need a host buffer)
  const Geo g = pct::make_geo(gr.nx, gr.ny, gr.nz, gr.hx, gr.hy, gr.hz, R, du, K, E);
  const Rec r{src[0], src[1], src[2], src[3], src[4], src[5], src[6], src[7], src[8], src[9], src[10]};

  // Device address of the scratch array in the current device's context. The
  // host-side symbol is only a stand-in, so host code must ask for the address.
  // It is looked up on every call (it allocates nothing), never cached: a
  // cached address would go stale when the context is reset or another
  // context is current on the same device.
  unsigned char* base = nullptr;
  cudaError_t e = cudaGetSymbolAddress((void**)&base, g_noalloc_scratch);
  if (e != cudaSuccess) return noalloc_fail(PCT_ERR_CUDA, "cudaGetSymbolAddress", e);
  float* delta = (float*)(base + kOffDelta);
  float* inv_s = (float*)(base + kOffInv);
  double* tab64 = (double*)(base + kOffTab64);
  float4* tab32 = (float4*)(base + kOffTab32);
  unsigned long long* bad = (unsigned long long*)(base + kOffFlag);
  cudaStream_t s = (cudaStream_t)stream;

  // MLP table, validation (synchronises once to report invalid records)
  if ((e = pct::launch_mlp_table(R, du, K, tab64, tab32, s)) != cudaSuccess ||
      (e = cudaMemsetAsync(bad, 0xff, sizeof(unsigned long long), s)) != cudaSuccess ||
      (e = pct::launch_validate(r, h->n, 0, pos_limit, bad, s)) != cudaSuccess)
    return noalloc_fail(PCT_ERR_CUDA, "table/validation launch", e);
  unsigned long long fb = 0;
  if ((e = cudaMemcpyAsync(&fb, bad, sizeof fb, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return noalloc_fail(PCT_ERR_CUDA, "validation read-back", e);
  if (fb != ~0ull) return noalloc_fail(PCT_ERR_INVALID_DATA, "a history record failed validation");

  // run counts s_j of this block (counted in the delta area), then 1/s_j
  unsigned* cnt = (unsigned*)delta;
  if ((e = cudaMemsetAsync(cnt, 0, (size_t)M * sizeof(unsigned), s)) != cudaSuccess ||
      (e = pct::launch_count(g, r, tab32, pct::Hull{}, 0, h->n, cnt, 128, s)) != cudaSuccess ||
      (e = pct::launch_inv_counts(cnt, inv_s, M, s)) != cudaSuccess ||
      (e = cudaMemsetAsync(delta, 0, (size_t)M * sizeof(float), s)) != cudaSuccess)
    return noalloc_fail(PCT_ERR_CUDA, "count pass", e);

  // fused MLP + projection, then x += delta / s_j (the apply clears delta)
  const unsigned blocks = (unsigned)((h->n + 127) / 128);
  drop_fused_rewalk_kernel<<<blocks, 128, (K + 1) * sizeof(float4), s>>>(g, r, tab32, h->n, x, delta, cfg->lambda,
                                                                          cfg->flags);
  if ((e = cudaGetLastError()) != cudaSuccess) return noalloc_fail(PCT_ERR_CUDA, "fused kernel launch", e);
  if ((e = pct::launch_drop_apply(x, delta, inv_s, M, (cfg->flags & PCT_FLAG_CLAMP) != 0, cfg->clamp_min, s)) !=
      cudaSuccess)
    return noalloc_fail(PCT_ERR_CUDA, "apply launch", e);
  return PCT_OK;
}
