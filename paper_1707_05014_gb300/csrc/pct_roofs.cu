// Roof microbenchmarks for the fused kernel's resources (pct_measure_roofs):
// float atomics into an L2-resident array at random and at warp-consecutive
// addresses, random 4-byte gathers from the same array, and dependent chains
// of integer (ALU pipe) and FP32 FMA instructions. Each figure is the best of
// a few timed launches (CUDA events) after one warm-up launch.
#include <stdint.h>

#include "../../include/pct.h"
#include "pct_internal.h"

namespace {

// Index sequence: a 32-bit LCG per thread (one IMAD per step), masked.
__device__ __forceinline__ uint32_t lcg(uint32_t s) { return s * 1664525u + 1013904223u; }

__global__ void __launch_bounds__(256) red_random_kernel(float* __restrict__ a, uint32_t mask, int iters) {
  uint32_t s = (blockIdx.x * blockDim.x + threadIdx.x) * 2654435761u;
  for (int i = 0; i < iters; ++i) {
    s = lcg(s);
    atomicAdd(a + ((s >> 7) & mask), 1.0f);
  }
}

// Lanes of a warp add to 32 consecutive floats (one 128-byte line), the
// line chosen at random per warp and step.
__global__ void __launch_bounds__(256) red_coherent_kernel(float* __restrict__ a, uint32_t mask, int iters) {
  uint32_t s = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 2654435761u;
  const uint32_t lane = threadIdx.x & 31;
  for (int i = 0; i < iters; ++i) {
    s = lcg(s);
    atomicAdd(a + ((((s >> 7) << 5) | lane) & mask), 1.0f);
  }
}

__global__ void __launch_bounds__(256) gather_kernel(const float* __restrict__ a, uint32_t mask, int iters,
                                                     float* __restrict__ out) {
  uint32_t s = (blockIdx.x * blockDim.x + threadIdx.x) * 2654435761u;
  float acc = 0.f;
  for (int i = 0; i < iters; ++i) {
    s = lcg(s);
    acc += __ldg(a + ((s >> 7) & mask));
  }
  if (acc == -1.f) out[0] = acc;  // keeps the loads; never true for the non-negative array
}

// Eight independent chains of 3-input logic / add / shift steps: every
// instruction issues to the integer ALU pipe.
__global__ void __launch_bounds__(256) alu_kernel(int iters, uint32_t* __restrict__ out) {
  uint32_t x[8];
  for (int j = 0; j < 8; ++j) x[j] = threadIdx.x * (j + 1) + blockIdx.x;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      x[j] = (x[j] ^ (x[j] >> 3)) + 0x9e3779b9u;  // shift, xor+add
      x[j] = x[j] ^ (x[j] << 5);                   // shift, xor
    }
  }
  uint32_t r = 0;
  for (int j = 0; j < 8; ++j) r ^= x[j];
  if (r == 0x12345678u) out[0] = r;
}

// Eight independent FP32 FMA chains.
__global__ void __launch_bounds__(256) fma_kernel(int iters, float* __restrict__ out) {
  float x[8];
  for (int j = 0; j < 8; ++j) x[j] = 1e-3f * (threadIdx.x + j);
  const float a = 0.999f, b = 1e-4f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = __fmaf_rn(x[j], a, b);
  }
  float r = 0.f;
  for (int j = 0; j < 8; ++j) r += x[j];
  if (r == -1.f) out[0] = r;
}

template <class Launch>
float best_ms(cudaStream_t s, int reps, Launch&& launch, cudaError_t* err) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  launch();  // warm-up
  for (int r = 0; r < reps; ++r) {
    cudaEventRecord(e0, s);
    launch();
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (*err == cudaSuccess) *err = cudaGetLastError();
  return best;
}

}  // namespace

extern "C" pct_status pct_measure_roofs(int device, int64_t array_bytes, pct_roofs* out) {
  if (!out) {
    pct::set_error_text("out is NULL");
    return PCT_ERR_INVALID_ARG;
  }
  if (array_bytes <= 0) array_bytes = 8 << 20;
  int64_t n = 1;
  while (n * 2 * (int64_t)sizeof(float) <= array_bytes) n *= 2;  // power of two
  if (n < 1024 || n > (1ll << 31)) {
    pct::set_error_text("array_bytes must give between 4 KB and 8 GB");
    return PCT_ERR_INVALID_ARG;
  }
  pct::DeviceGuard device_guard_;
  cudaError_t e = cudaSetDevice(device);
  cudaDeviceProp prop{};
  if (e == cudaSuccess) e = cudaGetDeviceProperties(&prop, device);
  if (e != cudaSuccess) {
    pct::set_error_text(cudaGetErrorString(e));
    return PCT_ERR_CUDA;
  }
  float* a = nullptr;
  float* sink = nullptr;
  if (cudaMalloc((void**)&a, (size_t)n * sizeof(float)) != cudaSuccess ||
      cudaMalloc((void**)&sink, 64) != cudaSuccess) {
    (void)cudaGetLastError();
    cudaFree(a);
    pct::set_error_text("roof microbenchmark buffers");
    return PCT_ERR_NO_MEMORY;
  }
  cudaStream_t s = nullptr;
  e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMemsetAsync(a, 0, (size_t)n * sizeof(float), s);
  const int sms = prop.multiProcessorCount;
  const int blocks = sms * 8, threads = 256;
  const double lanes = (double)blocks * threads;
  const uint32_t mask = (uint32_t)(n - 1);
  const int it_mem = 256, it_alu = 4096, reps = 5;
  if (e == cudaSuccess) {
    const float t_red = best_ms(s, reps, [&] { red_random_kernel<<<blocks, threads, 0, s>>>(a, mask, it_mem); }, &e);
    const float t_coh = best_ms(s, reps, [&] { red_coherent_kernel<<<blocks, threads, 0, s>>>(a, mask, it_mem); }, &e);
    const float t_gat = best_ms(s, reps, [&] { gather_kernel<<<blocks, threads, 0, s>>>(a, mask, it_mem, sink); }, &e);
    const float t_alu = best_ms(s, reps, [&] { alu_kernel<<<blocks, threads, 0, s>>>(it_alu, (uint32_t*)sink); }, &e);
    const float t_fma = best_ms(s, reps, [&] { fma_kernel<<<blocks, threads, 0, s>>>(it_alu, sink); }, &e);
    out->l2_red_per_s = lanes * it_mem / (t_red * 1e-3);
    out->l2_red_coherent_per_s = lanes * it_mem / (t_coh * 1e-3);
    out->l2_gather_per_s = lanes * it_mem / (t_gat * 1e-3);
    out->alu_ops_per_s = lanes * it_alu * 8 * 4 / (t_alu * 1e-3);  // shift, xor+add, shift, xor per chain step
    out->fma_ops_per_s = lanes * it_alu * 8 / (t_fma * 1e-3);
  }
  out->array_bytes = n * (int64_t)sizeof(float);
  out->l2_bytes = prop.l2CacheSize;
  out->sms = sms;
  if (s) cudaStreamDestroy(s);
  cudaFree(a);
  cudaFree(sink);
  if (e != cudaSuccess) {
    pct::set_error_text(cudaGetErrorString(e));
    return PCT_ERR_CUDA;
  }
  return PCT_OK;
}
