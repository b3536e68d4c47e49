// Learned warm start (no counterpart in the paper; a system feature): a small
// 3-D U-Net f predicts a better initial image x0 = x1 + f(x1) from the image
// x1 after the first DROP sweep, so that fewer sweeps reach the target
// accuracy. Trained by these kernels on pairs (x1, plain-solver result).
//
// Topology (4 levels, channels 16/32/64/128, 3x3x3 convolutions, zero pad):
//   L0: a0 = relu(conv(x1)), a1 = relu(conv(a0))                      16 ch
//   L1: b0 = relu(conv_s2(a1)), b1 = relu(conv(b0))                   32 ch
//   L2: c0 = relu(conv_s2(b1)), c1 = relu(conv(c0))                   64 ch
//   L3: d0 = relu(conv_s2(c1)), d1 = relu(conv(d0))                  128 ch
//   up: u2 = relu(upconv(d1) + c1), e2 = relu(conv(u2))                64 ch
//       u1 = relu(upconv(e2) + b1), e1 = relu(conv(u1))                32 ch
//       u0 = relu(upconv(e1) + a1), e0 = relu(conv(u0))                16 ch
//   out: f = conv(e0) (1 channel), x0 = x1 + f
// conv_s2 = stride 2; upconv = nearest x2 upsampling then a 3x3x3 conv.
// Activations are channels-last BF16 (channel counts padded to >= 16),
// weights BF16 for the products with FP32 master copies, every product
// accumulated in FP32 on the tensor cores (mma.sync m16n8k16 BF16).
// Every convolution, its data gradient and its weight gradient is one
// implicit GEMM with a gather of the A operand:
//   forward          A(m = out voxel, k = tap*Cin + ci) = in[src(m, tap)][ci]
//   data gradient    the same with spatially flipped, channel-transposed
//                    weights (stride 1) or a parity gather (stride 2)
//   weight gradient  dW(k, n) = sum over voxels m of A(m, k) dY(m, n)
#include <cuda_bf16.h>
#include <math.h>
#include <stdio.h>

#include <random>
#include <string>
#include <vector>

#include "../../include/pct.h"
#include "pct_internal.h"
#include "pct_trace.h"

namespace {

typedef __nv_bfloat16 bf16;

constexpr int BM = 128, BK = 32, NT = 128;

struct Dims {
  int D, H, W;
  __host__ __device__ int64_t n() const { return (int64_t)D * H * W; }
};

enum Gather { kS1 = 0, kS2 = 1, kUp = 2, kBwdS2 = 3 };

// Source voxel of output voxel (od, oh, ow) for tap t in the input grid, or -1.
template <int G>
__device__ __forceinline__ int64_t gather_src(Dims in, Dims out, int od, int oh, int ow, int t) {
  const int tz = t / 9, ty = (t / 3) % 3, tx = t % 3;
  int pz, py, px;
  if (G == kS1) {
    pz = od + tz - 1;
    py = oh + ty - 1;
    px = ow + tx - 1;
  } else if (G == kS2) {
    pz = 2 * od + tz - 1;
    py = 2 * oh + ty - 1;
    px = 2 * ow + tx - 1;
  } else if (G == kUp) {  // conv on the x2 nearest-upsampled input
    pz = od + tz - 1;
    py = oh + ty - 1;
    px = ow + tx - 1;
    if (pz < 0 || py < 0 || px < 0 || pz >= 2 * in.D || py >= 2 * in.H || px >= 2 * in.W) return -1;
    return ((int64_t)(pz >> 1) * in.H + (py >> 1)) * in.W + (px >> 1);
  } else {  // data gradient of a stride-2 conv: q = v + 1 - t must be even
    const int qz = od + 1 - tz, qy = oh + 1 - ty, qx = ow + 1 - tx;
    if ((qz | qy | qx) & 1) return -1;
    pz = qz >> 1;
    py = qy >> 1;
    px = qx >> 1;
  }
  if (pz < 0 || py < 0 || px < 0 || pz >= in.D || py >= in.H || px >= in.W) return -1;
  return ((int64_t)pz * in.H + py) * in.W + px;
}

// A operand of a convolution GEMM: rows = output voxels, k = tap * C + c.
template <int G>
struct ConvA {
  const bf16* in;
  Dims din, dout;
  int C;  // channels of `in` (multiple of 16)
  __device__ void load(bf16 (*As)[BK + 8], int64_t m0, int k0, int kend, int64_t M) const {
    for (int idx = threadIdx.x; idx < BM * (BK / 8); idx += NT) {
      const int r = idx / (BK / 8), cv = (idx % (BK / 8)) * 8;
      const int64_t m = m0 + r;
      const int k = k0 + cv;
      uint4 v = make_uint4(0, 0, 0, 0);
      if (m < M && k < kend) {
        const int ow = (int)(m % dout.W), oh = (int)((m / dout.W) % dout.H), od = (int)(m / ((int64_t)dout.W * dout.H));
        const int64_t s = gather_src<G>(din, dout, od, oh, ow, k / C);
        if (s >= 0) v = *reinterpret_cast<const uint4*>(in + s * C + (k % C));
      }
      *reinterpret_cast<uint4*>(&As[r][cv]) = v;
    }
  }
};

// B operand from a row-major [K][N] BF16 matrix (weights).
struct MatB {
  const bf16* w;
  int N;
  __device__ void load(bf16 (*Bs)[BK + 8], int bn, int n0, int k0, int kend) const {
    for (int idx = threadIdx.x; idx < BK * (bn / 8); idx += NT) {
      const int c = idx / (bn / 8), nv = (idx % (bn / 8)) * 8;
      const int k = k0 + c;
      uint4 v = make_uint4(0, 0, 0, 0);
      if (k < kend && n0 + nv < N) v = *reinterpret_cast<const uint4*>(w + (int64_t)k * N + n0 + nv);
      const bf16* e = reinterpret_cast<const bf16*>(&v);
#pragma unroll
      for (int q = 0; q < 8; ++q) Bs[nv + q][c] = e[q];
    }
  }
};

// Weight-gradient GEMM operands: rows = (tap, ci), reduction over voxels.
template <int G>
struct WgradA {
  const bf16* in;
  Dims din, dout;
  int C;
  __device__ void load(bf16 (*As)[BK + 8], int64_t m0, int k0, int kend, int64_t M) const {
    // As[r][c] = A_conv(voxel k0 + c, row m0 + r); vectors of 8 channels
    for (int idx = threadIdx.x; idx < (BM / 8) * BK; idx += NT) {
      const int c = idx % BK, rv = (idx / BK) * 8;
      const int64_t row = m0 + rv;
      const int64_t vox = (int64_t)k0 + c;
      uint4 v = make_uint4(0, 0, 0, 0);
      if (row < M && vox < kend) {
        const int ow = (int)(vox % dout.W), oh = (int)((vox / dout.W) % dout.H),
                  od = (int)(vox / ((int64_t)dout.W * dout.H));
        const int64_t s = gather_src<G>(din, dout, od, oh, ow, (int)(row / C));
        if (s >= 0) v = *reinterpret_cast<const uint4*>(in + s * C + (row % C));
      }
      const bf16* e = reinterpret_cast<const bf16*>(&v);
#pragma unroll
      for (int q = 0; q < 8; ++q) As[rv + q][c] = e[q];
    }
  }
};

struct WgradB {
  const bf16* dy;  // [voxels][N]
  int N;
  __device__ void load(bf16 (*Bs)[BK + 8], int bn, int n0, int k0, int kend) const {
    for (int idx = threadIdx.x; idx < BK * (bn / 8); idx += NT) {
      const int c = idx / (bn / 8), nv = (idx % (bn / 8)) * 8;
      const int64_t vox = (int64_t)k0 + c;
      uint4 v = make_uint4(0, 0, 0, 0);
      if (vox < kend && n0 + nv < N) v = *reinterpret_cast<const uint4*>(dy + vox * N + n0 + nv);
      const bf16* e = reinterpret_cast<const bf16*>(&v);
#pragma unroll
      for (int q = 0; q < 8; ++q) Bs[nv + q][c] = e[q];
    }
  }
};

// Epilogues: called once per output element (m, n) with the FP32 sum.
struct EpiAct {  // y = relu?(acc + bias + skip) -> bf16
  bf16* y;
  const float* bias;
  const bf16* skip;
  int N;
  int relu;
  __device__ void operator()(int64_t m, int n, float v) const {
    v += bias[n];
    if (skip) v += __bfloat162float(skip[m * N + n]);
    if (relu) v = fmaxf(v, 0.f);
    y[m * N + n] = __float2bfloat16_rn(v);
  }
};

struct EpiOut {  // x0 = x1 + f (channel 0 only)
  float* x0;
  const float* x1;
  const float* bias;
  __device__ void operator()(int64_t m, int n, float v) const {
    if (n == 0) x0[m] = x1[m] + v + bias[0];
  }
};

struct EpiGrad {  // d(pre-activation) = (acc + add) * [y > 0] -> bf16, or raw FP32
  bf16* dx;
  float* dx32;
  const bf16* add;
  const bf16* mask;
  int N;
  __device__ void operator()(int64_t m, int n, float v) const {
    if (dx32) {
      dx32[m * N + n] = v;
      return;
    }
    if (add) v += __bfloat162float(add[m * N + n]);
    if (mask && !(__bfloat162float(mask[m * N + n]) > 0.f)) v = 0.f;
    dx[m * N + n] = __float2bfloat16_rn(v);
  }
};

struct EpiWgrad {
  float* dw;
  int N;
  __device__ void operator()(int64_t m, int n, float v) const { atomicAdd(dw + m * N + n, v); }
};

__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// D[M x N] = sum_k A[m][k] B[k][n] over k in this CTA's split of [0, K).
// 128 threads: warp w owns rows [32w, 32w + 32) of the 128-row tile; BN
// columns (16, 32 or 64) per CTA.
template <int BN, class LA, class LB, class EP>
__global__ void __launch_bounds__(NT) igemm_kernel(LA la, LB lb, EP ep, int64_t M, int N, int64_t K,
                                                   int64_t k_split) {
  __shared__ __align__(16) bf16 As[BM][BK + 8];
  __shared__ __align__(16) bf16 Bs[BN][BK + 8];
  const int64_t m0 = (int64_t)blockIdx.x * BM;
  const int n0 = blockIdx.y * BN;
  const int64_t kbeg = (int64_t)blockIdx.z * k_split, kend = min(K, kbeg + k_split);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, tq = lane & 3;
  constexpr int NTILE = BN / 8;
  float acc[2][NTILE][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < NTILE; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
  for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
    la.load(As, m0, (int)(k0 - 0), (int)kend, M);
    lb.load(Bs, BN, n0, (int)k0, (int)kend);
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; kk += 16) {
      uint32_t a[2][4];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        const int r = warp * 32 + mt * 16 + g;
        a[mt][0] = *reinterpret_cast<const uint32_t*>(&As[r][kk + tq * 2]);
        a[mt][1] = *reinterpret_cast<const uint32_t*>(&As[r + 8][kk + tq * 2]);
        a[mt][2] = *reinterpret_cast<const uint32_t*>(&As[r][kk + tq * 2 + 8]);
        a[mt][3] = *reinterpret_cast<const uint32_t*>(&As[r + 8][kk + tq * 2 + 8]);
      }
#pragma unroll
      for (int nt = 0; nt < NTILE; ++nt) {
        const int c = nt * 8 + g;
        const uint32_t b0 = *reinterpret_cast<const uint32_t*>(&Bs[c][kk + tq * 2]);
        const uint32_t b1 = *reinterpret_cast<const uint32_t*>(&Bs[c][kk + tq * 2 + 8]);
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) mma_bf16(acc[mt][nt], a[mt], b0, b1);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < NTILE; ++nt) {
      const int64_t r0 = m0 + warp * 32 + mt * 16 + g, r1 = r0 + 8;
      const int c = n0 + nt * 8 + tq * 2;
      if (r0 < M && c < N) ep(r0, c, acc[mt][nt][0]);
      if (r0 < M && c + 1 < N) ep(r0, c + 1, acc[mt][nt][1]);
      if (r1 < M && c < N) ep(r1, c, acc[mt][nt][2]);
      if (r1 < M && c + 1 < N) ep(r1, c + 1, acc[mt][nt][3]);
    }
}

// ---- small element-wise kernels ------------------------------------------

__global__ void pad_input_kernel(const float* __restrict__ x, bf16* __restrict__ out, int64_t n, int C) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * C) return;
  out[i] = __float2bfloat16_rn((i % C) == 0 ? x[i / C] : 0.f);
}

// L1 loss gradient of x0 = x1 + f: d f = sign(x0 - target) / n (channel 0)
__global__ void loss_grad_kernel(const float* __restrict__ x0, const float* __restrict__ target, int64_t n, int C,
                                 bf16* __restrict__ df, double* loss) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double l = 0.0;
  if (i < n) {
    const float d = x0[i] - target[i];
    l = fabs((double)d);
    const float s = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
    for (int c = 0; c < C; ++c) df[i * C + c] = __float2bfloat16_rn(c == 0 ? s / (float)n : 0.f);
  }
  for (int o = 16; o > 0; o >>= 1) l += __shfl_down_sync(0xffffffffu, l, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, l / (double)n);
}

// dx_low[q][c] = sum of the 8 children of q in the x2 grid, times [y_low > 0];
// plus an optional second gradient (skip) added before the mask.
__global__ void pool_grad_kernel(const float* __restrict__ hi, Dims dlo, int C, const bf16* __restrict__ mask,
                                 bf16* __restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= dlo.n() * C) return;
  const int c = (int)(i % C);
  const int64_t q = i / C;
  const int w = (int)(q % dlo.W), h = (int)((q / dlo.W) % dlo.H), d = (int)(q / ((int64_t)dlo.W * dlo.H));
  const int H2 = 2 * dlo.H, W2 = 2 * dlo.W;
  float s = 0.f;
  for (int dz = 0; dz < 2; ++dz)
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx) s += hi[(((int64_t)(2 * d + dz) * H2 + (2 * h + dy)) * W2 + (2 * w + dx)) * C + c];
  if (!(__bfloat162float(mask[i]) > 0.f)) s = 0.f;
  out[i] = __float2bfloat16_rn(s);
}

// db[n] += sum_m g[m][n]
__global__ void bias_grad_kernel(const bf16* __restrict__ g, int64_t M, int N, float* __restrict__ db) {
  const int n = threadIdx.x % N;
  const int rows_per = blockDim.x / N;
  float s = 0.f;
  for (int64_t m = (int64_t)blockIdx.x * rows_per + threadIdx.x / N; m < M; m += (int64_t)gridDim.x * rows_per)
    s += __bfloat162float(g[m * N + n]);
  atomicAdd(db + n, s);
}

// BF16 weight copies for the products: forward [t][ci][co]; data gradient of a
// stride-1 conv [t'][co][ci] = W[26 - t'][ci][co]; of a stride-2 conv
// [t][co][ci] = W[t][ci][co].
__global__ void weight_copies_kernel(const float* __restrict__ w, int Cin, int Cout, bf16* __restrict__ wf,
                                     bf16* __restrict__ wflip, bf16* __restrict__ wtr) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 27LL * Cin * Cout) return;
  const int co = (int)(i % Cout), ci = (int)((i / Cout) % Cin), t = (int)(i / ((int64_t)Cout * Cin));
  const bf16 v = __float2bfloat16_rn(w[i]);
  wf[i] = v;
  wflip[((int64_t)(26 - t) * Cout + co) * Cin + ci] = v;
  wtr[((int64_t)t * Cout + co) * Cin + ci] = v;
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// ---- host-side network ------------------------------------------------------

struct Layer {
  int Cin, Cout;   // padded channel counts
  int kind;        // gather of the forward product: kS1, kS2 or kUp
  int in_level, out_level;
  int64_t w_off, b_off;  // offsets into the parameter vector
};

struct Act {
  bf16* p = nullptr;
  int level = 0, C = 0;
};

}  // namespace

struct pct_net {
  int device = 0;
  Dims lv[4];
  std::vector<Layer> layers;
  int64_t n_params = 0;
  float *params = nullptr, *grads = nullptr, *adam_m = nullptr, *adam_v = nullptr;
  bf16 *wf = nullptr, *wflip = nullptr, *wtr = nullptr;  // per-layer copies at w_off
  std::vector<Act> act;   // forward activations per layer output (and the padded input at index 15)
  std::vector<bf16*> grad_act;
  bf16* din = nullptr;    // padded input x1
  bf16* df = nullptr;     // gradient of f (16 ch)
  float* hi = nullptr;    // FP32 temp for up-conv data gradients
  int64_t hi_elems = 0;
  double* loss = nullptr;
  int64_t step = 0;
  cudaStream_t own_stream = nullptr;
};

namespace {

#define NET_CK(call)                                                                   \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) return nfail(PCT_ERR_CUDA, #call, cudaGetErrorString(e_));  \
  } while (0)

pct_status nfail(pct_status code, const char* what, const char* detail = "") {
  std::string m = std::string(what) + (detail[0] ? ": " : "") + detail;
  pct::set_error_text(m.c_str());
  return code;
}

template <int G, class EP>
cudaError_t launch_conv(int BNsel, const bf16* in, Dims din, int Cin, Dims dout, const bf16* w, int Cout, EP ep,
                        cudaStream_t s) {
  const int64_t M = dout.n();
  const int64_t K = 27LL * Cin;
  ConvA<G> la{in, din, dout, Cin};
  MatB lb{w, Cout};
  dim3 grid(blocks_for(M, BM), 1, 1);
  if (BNsel == 16) {
    grid.y = blocks_for(Cout, 16);
    igemm_kernel<16><<<grid, NT, 0, s>>>(la, lb, ep, M, Cout, K, K);
  } else if (BNsel == 32) {
    grid.y = blocks_for(Cout, 32);
    igemm_kernel<32><<<grid, NT, 0, s>>>(la, lb, ep, M, Cout, K, K);
  } else {
    grid.y = blocks_for(Cout, 64);
    igemm_kernel<64><<<grid, NT, 0, s>>>(la, lb, ep, M, Cout, K, K);
  }
  return cudaGetLastError();
}

int bn_for(int N) { return N <= 16 ? 16 : (N <= 32 ? 32 : 64); }

template <int G>
cudaError_t launch_wgrad(const bf16* in, Dims din, int Cin, Dims dout, const bf16* dy, int Cout, float* dw,
                         cudaStream_t s) {
  const int64_t Mr = 27LL * Cin, V = dout.n();
  WgradA<G> la{in, din, dout, Cin};
  WgradB lb{dy, Cout};
  EpiWgrad ep{dw, Cout};
  const int64_t split = 8192;
  dim3 grid(blocks_for(Mr, BM), 1, (unsigned)((V + split - 1) / split));
  const int bn = bn_for(Cout);
  grid.y = blocks_for(Cout, bn);
  if (bn == 16)
    igemm_kernel<16><<<grid, NT, 0, s>>>(la, lb, ep, Mr, Cout, V, split);
  else if (bn == 32)
    igemm_kernel<32><<<grid, NT, 0, s>>>(la, lb, ep, Mr, Cout, V, split);
  else
    igemm_kernel<64><<<grid, NT, 0, s>>>(la, lb, ep, Mr, Cout, V, split);
  return cudaGetLastError();
}

// forward of all layers; x0 = x1 + f(x1)
pct_status net_forward(pct_net* nt, const float* x1, float* x0, cudaStream_t s) {
  const Dims* L = nt->lv;
  const int64_t n0 = L[0].n();
  pad_input_kernel<<<blocks_for(n0 * 16, 256), 256, 0, s>>>(x1, nt->din, n0, 16);
  NET_CK(cudaGetLastError());
  // skip inputs of the up-convolutions: layer 8 <- c1 (layer 5), 10 <- b1 (3), 12 <- a1 (1)
  for (size_t li = 0; li < nt->layers.size(); ++li) {
    const Layer& ly = nt->layers[li];
    const bf16* in = li == 0 ? nt->din : nt->act[li - 1].p;
    const Dims din = L[ly.in_level], dout = L[ly.out_level];
    const bf16* w = nt->wf + ly.w_off;
    const float* b = nt->params + ly.b_off;
    cudaError_t e;
    if (li + 1 == nt->layers.size()) {
      EpiOut ep{x0, x1, b};
      e = launch_conv<kS1>(16, in, din, ly.Cin, dout, w, ly.Cout, ep, s);
    } else {
      const bf16* skip = li == 8 ? nt->act[5].p : (li == 10 ? nt->act[3].p : (li == 12 ? nt->act[1].p : nullptr));
      EpiAct ep{nt->act[li].p, b, skip, ly.Cout, 1};
      const int bn = bn_for(ly.Cout);
      if (ly.kind == kS1)
        e = launch_conv<kS1>(bn, in, din, ly.Cin, dout, w, ly.Cout, ep, s);
      else if (ly.kind == kS2)
        e = launch_conv<kS2>(bn, in, din, ly.Cin, dout, w, ly.Cout, ep, s);
      else
        e = launch_conv<kUp>(bn, in, din, ly.Cin, dout, w, ly.Cout, ep, s);
    }
    if (e != cudaSuccess) return nfail(PCT_ERR_CUDA, "conv forward", cudaGetErrorString(e));
  }
  return PCT_OK;
}

// gradients of the L1 loss w.r.t. every parameter (into nt->grads)
pct_status net_backward(pct_net* nt, const float* x1, const float* x0, const float* target, cudaStream_t s) {
  const Dims* L = nt->lv;
  const int64_t n0 = L[0].n();
  NET_CK(cudaMemsetAsync(nt->grads, 0, nt->n_params * sizeof(float), s));
  NET_CK(cudaMemsetAsync(nt->loss, 0, sizeof(double), s));
  loss_grad_kernel<<<blocks_for(n0, 256), 256, 0, s>>>(x0, target, n0, 16, nt->df, nt->loss);
  NET_CK(cudaGetLastError());
  const int nl = (int)nt->layers.size();
  // gradient flowing into layer li's output (pre-activation), bf16
  std::vector<const bf16*> gout(nl, nullptr);
  gout[nl - 1] = nt->df;
  // skip gradients: the pre-activation gradient of up-conv layer li also
  // flows to its skip source
  auto skip_src = [](int li) { return li == 8 ? 5 : (li == 10 ? 3 : (li == 12 ? 1 : -1)); };
  for (int li = nl - 1; li >= 0; --li) {
    const Layer& ly = nt->layers[li];
    const bf16* in = li == 0 ? nt->din : nt->act[li - 1].p;
    const Dims din = L[ly.in_level], dout = L[ly.out_level];
    const bf16* dy = gout[li];
    float* dw = nt->grads + ly.w_off;
    float* db = nt->grads + ly.b_off;
    cudaError_t e;
    // weight gradient
    if (ly.kind == kS1)
      e = launch_wgrad<kS1>(in, din, ly.Cin, dout, dy, ly.Cout, dw, s);
    else if (ly.kind == kS2)
      e = launch_wgrad<kS2>(in, din, ly.Cin, dout, dy, ly.Cout, dw, s);
    else
      e = launch_wgrad<kUp>(in, din, ly.Cin, dout, dy, ly.Cout, dw, s);
    if (e != cudaSuccess) return nfail(PCT_ERR_CUDA, "weight gradient", cudaGetErrorString(e));
    {
      const int N = ly.Cout, threads = 256 - 256 % N;
      bias_grad_kernel<<<304, threads, 0, s>>>(dy, dout.n(), N, db);
      NET_CK(cudaGetLastError());
    }
    if (li == 0) break;
    // data gradient into the previous layer's output, masked by its ReLU; the
    // skip sources also receive the gradient of the up-conv that reads them
    const int prev = li - 1;
    bf16* dx = nt->grad_act[prev];
    const bf16* mask = nt->act[prev].p;
    const bf16* add = nullptr;
    for (int u = 0; u < nl; ++u)
      if (skip_src(u) == prev) add = gout[u];
    if (ly.kind == kS1) {
      EpiGrad ep{dx, nullptr, add, mask, ly.Cin};
      e = launch_conv<kS1>(bn_for(ly.Cin), dy, dout, ly.Cout, din, nt->wflip + ly.w_off, ly.Cin, ep, s);
    } else if (ly.kind == kS2) {
      EpiGrad ep{dx, nullptr, add, mask, ly.Cin};
      e = launch_conv<kBwdS2>(bn_for(ly.Cin), dy, dout, ly.Cout, din, nt->wtr + ly.w_off, ly.Cin, ep, s);
    } else {
      // stride-1 data gradient on the x2 grid (FP32), then sum the 8 children
      const Dims dhi{2 * din.D, 2 * din.H, 2 * din.W};
      EpiGrad ep{nullptr, nt->hi, nullptr, nullptr, ly.Cin};
      e = launch_conv<kS1>(bn_for(ly.Cin), dy, dout, ly.Cout, dhi, nt->wflip + ly.w_off, ly.Cin, ep, s);
      if (e == cudaSuccess) {
        pool_grad_kernel<<<blocks_for(din.n() * ly.Cin, 256), 256, 0, s>>>(nt->hi, din, ly.Cin, mask, dx);
        e = cudaGetLastError();
      }
      if (e == cudaSuccess && add) return nfail(PCT_ERR_STATE, "up-conv input with a skip consumer");
    }
    if (e != cudaSuccess) return nfail(PCT_ERR_CUDA, "data gradient", cudaGetErrorString(e));
    gout[prev] = dx;
  }
  return PCT_OK;
}

pct_status refresh_weights(pct_net* nt, cudaStream_t s) {
  for (const Layer& ly : nt->layers) {
    const int64_t n = 27LL * ly.Cin * ly.Cout;
    weight_copies_kernel<<<blocks_for(n, 256), 256, 0, s>>>(nt->params + ly.w_off, ly.Cin, ly.Cout,
                                                           nt->wf + ly.w_off, nt->wflip + ly.w_off,
                                                           nt->wtr + ly.w_off);
    NET_CK(cudaGetLastError());
  }
  return PCT_OK;
}

}  // namespace

extern "C" {

pct_status pct_net_create(pct_net** out, int32_t nz, int32_t ny, int32_t nx, uint64_t seed, int device) {
  if (!out) return nfail(PCT_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (nz < 8 || ny < 8 || nx < 8 || nz % 8 || ny % 8 || nx % 8)
    return nfail(PCT_ERR_INVALID_ARG, "grid dims must be multiples of 8 (three x2 levels)");
  pct_net* nt = new pct_net();
  nt->device = device;
  for (int l = 0; l < 4; ++l) nt->lv[l] = Dims{nz >> l, ny >> l, nx >> l};
  // (Cin, Cout, gather, in level, out level)
  const int spec[15][5] = {{16, 16, kS1, 0, 0},  {16, 16, kS1, 0, 0},   {16, 32, kS2, 0, 1},  {32, 32, kS1, 1, 1},
                           {32, 64, kS2, 1, 2},  {64, 64, kS1, 2, 2},   {64, 128, kS2, 2, 3}, {128, 128, kS1, 3, 3},
                           {128, 64, kUp, 3, 2}, {64, 64, kS1, 2, 2},   {64, 32, kUp, 2, 1},  {32, 32, kS1, 1, 1},
                           {32, 16, kUp, 1, 0},  {16, 16, kS1, 0, 0},   {16, 16, kS1, 0, 0}};
  int64_t off = 0;
  for (auto& sp : spec) {
    Layer ly{sp[0], sp[1], sp[2], sp[3], sp[4], 0, 0};
    ly.w_off = off;
    off += 27LL * ly.Cin * ly.Cout;
    ly.b_off = off;
    off += ly.Cout;
    nt->layers.push_back(ly);
  }
  nt->n_params = off;
  // He-normal weights on the real channels (input channel 0 of layer 0,
  // output channel 0 of the last layer); zero biases and padding
  std::vector<float> p(off, 0.f);
  std::mt19937_64 rng(seed);
  std::normal_distribution<double> nd(0.0, 1.0);
  for (size_t li = 0; li < nt->layers.size(); ++li) {
    const Layer& ly = nt->layers[li];
    const int cin_real = li == 0 ? 1 : ly.Cin, cout_real = li + 1 == nt->layers.size() ? 1 : ly.Cout;
    const double sd = sqrt(2.0 / (27.0 * cin_real)) * (li + 1 == nt->layers.size() ? 0.1 : 1.0);
    for (int t = 0; t < 27; ++t)
      for (int ci = 0; ci < cin_real; ++ci)
        for (int co = 0; co < cout_real; ++co) p[ly.w_off + ((int64_t)t * ly.Cin + ci) * ly.Cout + co] = (float)(sd * nd(rng));
  }
  pct::DeviceGuard device_guard_;
  pct_status st = PCT_OK;
  do {
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&nt->own_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      st = nfail(PCT_ERR_CUDA, "net set-up", cudaGetErrorString(e));
      break;
    }
    bool ok = cudaMalloc((void**)&nt->params, off * sizeof(float)) == cudaSuccess &&
              cudaMalloc((void**)&nt->grads, off * sizeof(float)) == cudaSuccess &&
              cudaMalloc((void**)&nt->adam_m, off * sizeof(float)) == cudaSuccess &&
              cudaMalloc((void**)&nt->adam_v, off * sizeof(float)) == cudaSuccess &&
              cudaMalloc((void**)&nt->wf, off * sizeof(bf16)) == cudaSuccess &&
              cudaMalloc((void**)&nt->wflip, off * sizeof(bf16)) == cudaSuccess &&
              cudaMalloc((void**)&nt->wtr, off * sizeof(bf16)) == cudaSuccess &&
              cudaMalloc((void**)&nt->din, nt->lv[0].n() * 16 * sizeof(bf16)) == cudaSuccess &&
              cudaMalloc((void**)&nt->df, nt->lv[0].n() * 16 * sizeof(bf16)) == cudaSuccess &&
              cudaMalloc((void**)&nt->loss, sizeof(double)) == cudaSuccess;
    nt->act.resize(nt->layers.size());
    nt->grad_act.assign(nt->layers.size(), nullptr);
    for (size_t li = 0; ok && li < nt->layers.size(); ++li) {
      const Layer& ly = nt->layers[li];
      const int64_t n = nt->lv[ly.out_level].n() * ly.Cout;
      ok = cudaMalloc((void**)&nt->act[li].p, n * sizeof(bf16)) == cudaSuccess &&
           cudaMalloc((void**)&nt->grad_act[li], n * sizeof(bf16)) == cudaSuccess;
      nt->act[li].level = ly.out_level;
      nt->act[li].C = ly.Cout;
      if (ly.kind == kUp) nt->hi_elems = std::max(nt->hi_elems, nt->lv[ly.out_level].n() * ly.Cin);
    }
    ok = ok && cudaMalloc((void**)&nt->hi, nt->hi_elems * sizeof(float)) == cudaSuccess;
    if (!ok) {
      (void)cudaGetLastError();
      st = nfail(PCT_ERR_NO_MEMORY, "net allocation failed");
      break;
    }
    cudaStream_t s = nt->own_stream;
    if ((e = cudaMemcpyAsync(nt->params, p.data(), off * sizeof(float), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(nt->adam_m, 0, off * sizeof(float), s)) != cudaSuccess ||
        (e = cudaMemsetAsync(nt->adam_v, 0, off * sizeof(float), s)) != cudaSuccess) {
      st = nfail(PCT_ERR_CUDA, "net init", cudaGetErrorString(e));
      break;
    }
    if ((st = refresh_weights(nt, s)) != PCT_OK) break;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) st = nfail(PCT_ERR_CUDA, "net init", cudaGetErrorString(e));
  } while (0);
  if (st != PCT_OK) {
    pct_net_destroy(nt);
    return st;
  }
  *out = nt;
  return PCT_OK;
}

pct_status pct_net_destroy(pct_net* nt) {
  if (!nt) return PCT_OK;
  pct::DeviceGuard device_guard_;
  cudaSetDevice(nt->device);
  if (nt->own_stream) cudaStreamSynchronize(nt->own_stream);
  for (auto& a : nt->act) cudaFree(a.p);
  for (auto p : nt->grad_act) cudaFree(p);
  cudaFree(nt->params);
  cudaFree(nt->grads);
  cudaFree(nt->adam_m);
  cudaFree(nt->adam_v);
  cudaFree(nt->wf);
  cudaFree(nt->wflip);
  cudaFree(nt->wtr);
  cudaFree(nt->din);
  cudaFree(nt->df);
  cudaFree(nt->hi);
  cudaFree(nt->loss);
  if (nt->own_stream) cudaStreamDestroy(nt->own_stream);
  delete nt;
  return PCT_OK;
}

int64_t pct_net_param_count(const pct_net* nt) { return nt ? nt->n_params : 0; }

pct_status pct_net_get_params(pct_net* nt, float* out) {
  if (!nt || !out) return nfail(PCT_ERR_INVALID_ARG, "net or out is NULL");
  pct::DeviceGuard device_guard_;
  NET_CK(cudaSetDevice(nt->device));
  NET_CK(cudaMemcpy(out, nt->params, nt->n_params * sizeof(float), cudaMemcpyDeviceToHost));
  return PCT_OK;
}

pct_status pct_net_set_params(pct_net* nt, const float* in) {
  if (!nt || !in) return nfail(PCT_ERR_INVALID_ARG, "net or in is NULL");
  pct::DeviceGuard device_guard_;
  NET_CK(cudaSetDevice(nt->device));
  NET_CK(cudaMemcpy(nt->params, in, nt->n_params * sizeof(float), cudaMemcpyHostToDevice));
  pct_status st = refresh_weights(nt, nt->own_stream);
  if (st != PCT_OK) return st;
  NET_CK(cudaStreamSynchronize(nt->own_stream));
  return PCT_OK;
}

pct_status pct_net_forward(pct_net* nt, const float* x1, float* x0, void* stream) {
  pct::TraceRange trace_("pct_net_forward");
  if (!nt || !x1 || !x0) return nfail(PCT_ERR_INVALID_ARG, "NULL argument");
  pct::DeviceGuard device_guard_;
  NET_CK(cudaSetDevice(nt->device));
  return net_forward(nt, x1, x0, stream ? (cudaStream_t)stream : nt->own_stream);
}

pct_status pct_net_gradients(pct_net* nt, const float* x1, const float* target, float* x0_scratch, float* grads_host,
                             double* loss) {
  if (!nt || !x1 || !target || !x0_scratch) return nfail(PCT_ERR_INVALID_ARG, "NULL argument");
  pct::DeviceGuard device_guard_;
  NET_CK(cudaSetDevice(nt->device));
  cudaStream_t s = nt->own_stream;
  pct_status st = net_forward(nt, x1, x0_scratch, s);
  if (st == PCT_OK) st = net_backward(nt, x1, x0_scratch, target, s);
  if (st != PCT_OK) return st;
  if (grads_host) NET_CK(cudaMemcpyAsync(grads_host, nt->grads, nt->n_params * sizeof(float), cudaMemcpyDeviceToHost, s));
  if (loss) NET_CK(cudaMemcpyAsync(loss, nt->loss, sizeof(double), cudaMemcpyDeviceToHost, s));
  NET_CK(cudaStreamSynchronize(s));
  return PCT_OK;
}

pct_status pct_net_layer_shape(const pct_net* nt, int32_t layer, int32_t* cin, int32_t* cout, int32_t* in_level,
                               int32_t* out_level) {
  if (!nt || !cin || !cout || !in_level || !out_level) return nfail(PCT_ERR_INVALID_ARG, "NULL argument");
  if (layer < 0 || layer >= (int)nt->layers.size()) return nfail(PCT_ERR_INVALID_ARG, "layer out of range");
  const Layer& ly = nt->layers[layer];
  *cin = ly.Cin;
  *cout = ly.Cout;
  *in_level = ly.in_level;
  *out_level = ly.out_level;
  return PCT_OK;
}

pct_status pct_net_layer(pct_net* nt, int32_t layer, int32_t op, const void* in, const void* skip, const void* dy,
                         const void* mask, const void* add, void* out, void* stream) {
  if (!nt || !out) return nfail(PCT_ERR_INVALID_ARG, "net or out is NULL");
  const int nl = (int)nt->layers.size();
  if (layer < 0 || layer >= nl) return nfail(PCT_ERR_INVALID_ARG, "layer out of range");
  const Layer& ly = nt->layers[layer];
  const Dims din = nt->lv[ly.in_level], dout = nt->lv[ly.out_level];
  const bool has_skip = layer == 8 || layer == 10 || layer == 12;
  pct::DeviceGuard device_guard_;
  NET_CK(cudaSetDevice(nt->device));
  cudaStream_t s = stream ? (cudaStream_t)stream : nt->own_stream;
  cudaError_t e = cudaSuccess;
  if (op == PCT_NET_FORWARD) {
    if (layer == nl - 1) return nfail(PCT_ERR_INVALID_ARG, "the output layer's forward is pct_net_forward");
    if (!in || has_skip != (skip != nullptr)) return nfail(PCT_ERR_INVALID_ARG, "in, or skip (layers 8, 10, 12 only)");
    EpiAct ep{(bf16*)out, nt->params + ly.b_off, (const bf16*)skip, ly.Cout, 1};
    const bf16* w = nt->wf + ly.w_off;
    const int bn = bn_for(ly.Cout);
    if (ly.kind == kS1)
      e = launch_conv<kS1>(bn, (const bf16*)in, din, ly.Cin, dout, w, ly.Cout, ep, s);
    else if (ly.kind == kS2)
      e = launch_conv<kS2>(bn, (const bf16*)in, din, ly.Cin, dout, w, ly.Cout, ep, s);
    else
      e = launch_conv<kUp>(bn, (const bf16*)in, din, ly.Cin, dout, w, ly.Cout, ep, s);
  } else if (op == PCT_NET_DATA_GRAD) {
    if (layer == 0) return nfail(PCT_ERR_INVALID_ARG, "layer 0 has no data gradient");
    if (!dy || !mask) return nfail(PCT_ERR_INVALID_ARG, "dy or mask is NULL");
    if (ly.kind == kS1) {
      EpiGrad ep{(bf16*)out, nullptr, (const bf16*)add, (const bf16*)mask, ly.Cin};
      e = launch_conv<kS1>(bn_for(ly.Cin), (const bf16*)dy, dout, ly.Cout, din, nt->wflip + ly.w_off, ly.Cin, ep, s);
    } else if (ly.kind == kS2) {
      EpiGrad ep{(bf16*)out, nullptr, (const bf16*)add, (const bf16*)mask, ly.Cin};
      e = launch_conv<kBwdS2>(bn_for(ly.Cin), (const bf16*)dy, dout, ly.Cout, din, nt->wtr + ly.w_off, ly.Cin, ep, s);
    } else {
      if (add) return nfail(PCT_ERR_INVALID_ARG, "an up-convolution's input has no skip gradient");
      const Dims dhi{2 * din.D, 2 * din.H, 2 * din.W};
      EpiGrad ep{nullptr, nt->hi, nullptr, nullptr, ly.Cin};
      e = launch_conv<kS1>(bn_for(ly.Cin), (const bf16*)dy, dout, ly.Cout, dhi, nt->wflip + ly.w_off, ly.Cin, ep, s);
      if (e == cudaSuccess) {
        pool_grad_kernel<<<blocks_for(din.n() * ly.Cin, 256), 256, 0, s>>>(nt->hi, din, ly.Cin, (const bf16*)mask,
                                                                             (bf16*)out);
        e = cudaGetLastError();
      }
    }
  } else if (op == PCT_NET_WEIGHT_GRAD) {
    if (!in || !dy) return nfail(PCT_ERR_INVALID_ARG, "in or dy is NULL");
    float* dw = (float*)out;
    float* db = dw + 27LL * ly.Cin * ly.Cout;
    NET_CK(cudaMemsetAsync(dw, 0, (27LL * ly.Cin * ly.Cout + ly.Cout) * sizeof(float), s));
    if (ly.kind == kS1)
      e = launch_wgrad<kS1>((const bf16*)in, din, ly.Cin, dout, (const bf16*)dy, ly.Cout, dw, s);
    else if (ly.kind == kS2)
      e = launch_wgrad<kS2>((const bf16*)in, din, ly.Cin, dout, (const bf16*)dy, ly.Cout, dw, s);
    else
      e = launch_wgrad<kUp>((const bf16*)in, din, ly.Cin, dout, (const bf16*)dy, ly.Cout, dw, s);
    if (e == cudaSuccess) {
      const int N = ly.Cout, threads = 256 - 256 % N;
      bias_grad_kernel<<<304, threads, 0, s>>>((const bf16*)dy, dout.n(), N, db);
      e = cudaGetLastError();
    }
  } else {
    return nfail(PCT_ERR_INVALID_ARG, "op must be PCT_NET_FORWARD, PCT_NET_DATA_GRAD or PCT_NET_WEIGHT_GRAD");
  }
  if (e != cudaSuccess) return nfail(PCT_ERR_CUDA, "layer launch", cudaGetErrorString(e));
  return PCT_OK;
}

pct_status pct_net_train_step(pct_net* nt, const float* x1, const float* target, float* x0_scratch, float lr,
                              double* loss, void* stream) {
  pct::TraceRange trace_("pct_net_train_step");
  if (!nt || !x1 || !target || !x0_scratch) return nfail(PCT_ERR_INVALID_ARG, "NULL argument");
  if (!(lr > 0.f)) return nfail(PCT_ERR_INVALID_ARG, "lr must be > 0");
  pct::DeviceGuard device_guard_;
  NET_CK(cudaSetDevice(nt->device));
  cudaStream_t s = stream ? (cudaStream_t)stream : nt->own_stream;
  pct_status st = net_forward(nt, x1, x0_scratch, s);
  if (st == PCT_OK) st = net_backward(nt, x1, x0_scratch, target, s);
  if (st != PCT_OK) return st;
  nt->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)nt->step), c2 = 1.f - powf(b2, (float)nt->step);
  adam_kernel<<<blocks_for(nt->n_params, 256), 256, 0, s>>>(nt->params, nt->grads, nt->adam_m, nt->adam_v,
                                                           nt->n_params, lr, b1, b2, 1e-8f, c1, c2);
  NET_CK(cudaGetLastError());
  if ((st = refresh_weights(nt, s)) != PCT_OK) return st;
  if (loss) {
    NET_CK(cudaMemcpyAsync(loss, nt->loss, sizeof(double), cudaMemcpyDeviceToHost, s));
    NET_CK(cudaStreamSynchronize(s));
  }
  return PCT_OK;
}

}  // extern "C"
