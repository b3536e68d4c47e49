// Object-hull set-up kernels (pct_set_hull, pct_carve_hull, pct_hull_ranges):
// each history's hull entry/exit nodes, space carving of the hull from
// low-WEPL histories with 6-neighbour growth, and the gather of ranges in
// load order. The hull path itself is walk_proton_hull (pct_walk.cuh). The
// MLP formalism that Sec. 2 cites estimates the path inside the object and
// takes it straight outside; the hull says where the object is.
#include "pct_walk.cuh"

namespace pct {
namespace {

int grid_for(int64_t n, int threads) { return (int)((n + threads - 1) / threads); }

__device__ __forceinline__ void load_table(const float4* __restrict__ src, float4* dst, int n) {
  for (int k = threadIdx.x; k < n; k += blockDim.x) dst[k] = src[k];
  __syncthreads();
}

// range[i] = iin | iout << 16: iin = the first node k in [0, K] whose entry-ray
// point lies in a hull voxel, iout = the last node whose exit-ray point does;
// (0, K) when either is missing or iout <= iin (the proton misses the hull).
__global__ void hull_range_kernel(Geo g, Rec r, int64_t n, const uint8_t* __restrict__ mask,
                                  int32_t* __restrict__ range) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const RecV v = load_rec(r, i);
  auto in_hull = [&](float t, float vv, int k) {
    const int3 Q = quantise3(node_grid(g, v, __fmaf_rn((float)k, g.du, g.u0), t, vv));
    const int ix = floor_q(Q.x), iy = floor_q(Q.y), iz = floor_q(Q.z);
    if ((unsigned)ix >= (unsigned)g.nx || (unsigned)iy >= (unsigned)g.ny || (unsigned)iz >= (unsigned)g.nz) return false;
    return mask[ix + (int64_t)g.nx * (iy + (int64_t)g.ny * iz)] != 0;
  };
  int iin = -1, iout = -1;
  for (int k = 0; k <= g.K && iin < 0; ++k) {
    const float dk = __fmul_rn((float)k, g.du);
    if (in_hull(__fmaf_rn(v.st0, dk, v.t0), __fmaf_rn(v.sv0, dk, v.v0), k)) iin = k;
  }
  for (int k = g.K; k >= 0 && iout < 0; --k) {
    const float dk = __fmul_rn((float)(k - g.K), g.du);
    if (in_hull(__fmaf_rn(v.st2, dk, v.t2), __fmaf_rn(v.sv2, dk, v.v2), k)) iout = k;
  }
  if (iin < 0 || iout < 0 || iout <= iin) {
    iin = 0;
    iout = g.K;
  }
  range[i] = iin | (iout << 16);
}

// out[j] = 0 on the row of every history with wepl <= wepl_max (voxels its
// hull-free path crosses are air); out starts at 1.
__global__ void carve_kernel(Geo g, Rec r, const float4* __restrict__ tab_g, int64_t n, float wepl_max,
                             uint8_t* __restrict__ out) {
  extern __shared__ float4 tab[];
  load_table(tab_g, tab, g.K + 1);
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (!(__ldg(r.wepl + i) <= wepl_max)) return;
  const RecV v = load_rec(r, i);
  walk_proton(g, tab, v, [&](int j, float) { out[j] = 0; });
}

// One 6-neighbour growth step of the hull: out = in, plus every voxel with a
// face neighbour in `in`.
__global__ void dilate_kernel(const uint8_t* __restrict__ in, uint8_t* __restrict__ out, int nx, int ny, int nz) {
  const int64_t M = (int64_t)nx * ny * nz;
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= M) return;
  const int x = (int)(j % nx), y = (int)((j / nx) % ny), z = (int)(j / ((int64_t)nx * ny));
  const int64_t sxy = (int64_t)nx * ny;
  const bool hit = in[j] || (x > 0 && in[j - 1]) || (x + 1 < nx && in[j + 1]) || (y > 0 && in[j - nx]) ||
                   (y + 1 < ny && in[j + nx]) || (z > 0 && in[j - sxy]) || (z + 1 < nz && in[j + sxy]);
  out[j] = hit ? 1 : 0;
}

}  // namespace

cudaError_t launch_hull_ranges(const Geo& g, const Rec& r, int64_t n, const uint8_t* mask, int32_t* range,
                               cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  hull_range_kernel<<<grid_for(n, 128), 128, 0, s>>>(g, r, n, mask, range);
  return cudaGetLastError();
}

__global__ void gather_ranges_kernel(const int32_t* __restrict__ range, const int64_t* __restrict__ where,
                                     int64_t first, int64_t count, int32_t* __restrict__ out) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= count) return;
  const int32_t v = range[where ? where[first + p] : first + p];
  out[2 * p] = v & 0xffff;
  out[2 * p + 1] = v >> 16;
}

cudaError_t launch_gather_ranges(const int32_t* range, const int64_t* where, int64_t first, int64_t count,
                                 int32_t* out, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  gather_ranges_kernel<<<grid_for(count, 256), 256, 0, s>>>(range, where, first, count, out);
  return cudaGetLastError();
}

cudaError_t launch_carve_hull(const Geo& g, const Rec& r, const float4* tab, int64_t n, float wepl_max, int dilate,
                              uint8_t* out, uint8_t* tmp, cudaStream_t s) {
  const int64_t M = (int64_t)g.nx * g.ny * g.nz;
  cudaError_t e = cudaMemsetAsync(out, 1, (size_t)M, s);
  if (e != cudaSuccess) return e;
  if (n > 0) carve_kernel<<<grid_for(n, 128), 128, (g.K + 1) * sizeof(float4), s>>>(g, r, tab, n, wepl_max, out);
  for (int it = 0; it < dilate; ++it) {
    e = cudaMemcpyAsync(tmp, out, (size_t)M, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    dilate_kernel<<<grid_for(M, 256), 256, 0, s>>>(tmp, out, g.nx, g.ny, g.nz);
  }
  return cudaGetLastError();
}

}  // namespace pct
