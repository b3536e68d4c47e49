// MLP coefficient table in FP64 on the GPU (arXiv 1707.05014 Sec. 2: the
// most-likely path from the measured entry/exit states, in the form of
// Schulte et al. 2008 that the paper cites).
//
// For a node at depth w1 between the planes (0 and W, in cm) the estimator is
//   y1 = (S1^-1 + R1^T S2^-1 R1)^-1 (S1^-1 R0 y0 + R1^T S2^-1 y2),
// y = (lateral position, slope). This kernel evaluates it in the equivalent
// conditioning form, which inverts only the well-conditioned total covariance
// C = R1 S1 R1^T + S2 (the direct form inverts S1, whose condition number
// grows like 1/w1^2 near the entry plane):
//   G  = S1 R1^T C^-1            (weight of y2)
//   A0 = (I - G R1) R0           (weight of y0)
// The scattering moments are closed-form polynomial integrals: after the
// substitution s = w1 - w (or W - w) each is a sum of s^(m+i+1)/(m+i+1)
// terms with non-negative powers, so no cancellation occurs.
#include "pct_internal.h"

namespace pct {
namespace {

// 1/(beta^2 p^2) of a 200 MeV proton in water, 5th-order polynomial in depth
// (cm), MeV^-2 cm^-i (Schulte et al. 2008).
__constant__ double kPoly[6] = {7.457e-6, 4.548e-7, -5.777e-8, 1.301e-8, -9.228e-10, 2.687e-11};
constexpr double kE0 = 13.6;   // MeV, Highland constant
constexpr double kX0 = 36.08;  // cm, radiation length of water

__device__ double binom(int n, int k) {
  double r = 1.0;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}

// m-th moment of f over a sub-slab ending at `end` with thickness `len`:
//   integral_0^len s^m f(end - s) ds.
__device__ double moment(double end, double len, int m) {
  double total = 0.0;
  for (int i = 0; i < 6; ++i) {
    // coefficient of s^i in f(end - s)
    double bi = 0.0, ep = 1.0;
    for (int j = i; j < 6; ++j) {
      bi += kPoly[j] * binom(j, i) * ep;
      ep *= end;
    }
    if (i & 1) bi = -bi;
    total += bi * pow(len, m + i + 1) / (m + i + 1);
  }
  return total;
}

__device__ double highland(double L) {
  double f = 1.0 + 0.038 * log(L / kX0);
  return kE0 * kE0 * f * f / kX0;
}

// Coefficients (c1, c2, c3, c4) of node m of a water layer W cm thick with
// nodes every du mm, entered at m = 0 and left at m = n.
__device__ void layer_entry(double W, double du, int n, int m, double c[4]) {
  if (m == 0 || m == n) {
    c[0] = (m == 0);
    c[1] = 0.0;
    c[2] = (m == n);
    c[3] = 0.0;
    return;
  }
  const double w1 = m * du / 10.0;
  const double w2 = W - w1;
  const double k1 = highland(w1), k2 = highland(w2);
  // S1 = k1 [[a, b], [b, c]], S2 = k2 [[d, e], [e, f]]
  const double a = k1 * moment(w1, w1, 2), b = k1 * moment(w1, w1, 1), cc = k1 * moment(w1, w1, 0);
  const double d = k2 * moment(W, w2, 2), e = k2 * moment(W, w2, 1), f = k2 * moment(W, w2, 0);
  // S1 R1^T with R1 = [[1, w2], [0, 1]]: [[a + b w2, b], [b + c w2, c]]
  const double p00 = a + b * w2, p01 = b, p10 = b + cc * w2, p11 = cc;
  // C = R1 S1 R1^T + S2
  const double C00 = p00 + w2 * p10 + d, C01 = p01 + w2 * p11 + e;
  const double C10 = p10 + e, C11 = p11 + f;
  const double det = C00 * C11 - C01 * C10;
  const double i00 = C11 / det, i01 = -C01 / det, i10 = -C10 / det, i11 = C00 / det;
  // first row of G = (S1 R1^T) C^-1
  const double g00 = p00 * i00 + p01 * i10, g01 = p00 * i01 + p01 * i11;
  // first row of (I - G R1) R0 with R0 = [[1, w1], [0, 1]]:
  //   (I - G R1) first row = [1 - g00, -(g00 w2 + g01)]
  const double r0 = 1.0 - g00, r1 = -(g00 * w2 + g01);
  c[0] = r0;
  c[1] = 10.0 * (r0 * w1 + r1);  // cm -> mm
  c[2] = g00;
  c[3] = 10.0 * g01;
}

// Thickness (cm) of a layer of n node intervals; n = K is the slab between
// the measurement planes, taken as 2R exactly so that its table is the plane
// table bit for bit.
__device__ double layer_cm(double R, double du, int K, int n) { return n == K ? 2.0 * R / 10.0 : n * du / 10.0; }

__global__ void mlp_table_kernel(double R, double du, int K, double* __restrict__ tab64, float4* __restrict__ tab32) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > K) return;
  double c[4];
  layer_entry(2.0 * R / 10.0, du, K, k, c);
  tab64[4 * k + 0] = c[0];
  tab64[4 * k + 1] = c[1];
  tab64[4 * k + 2] = c[2];
  tab64[4 * k + 3] = c[3];
  tab32[k] = make_float4((float)c[0], (float)c[1], (float)c[2], (float)c[3]);
}

// Tables of every hull thickness n = 1..K (blockIdx.y = n - 1), stored at
// fam + family_offset(n), entries m = 0..n; optionally the FP64 values of
// one thickness (tab64 for n == n64).
__global__ void mlp_family_kernel(double R, double du, int K, float4* __restrict__ fam, int n64,
                                  double* __restrict__ tab64) {
  const int n = blockIdx.y + 1;
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m > n) return;
  double c[4];
  layer_entry(layer_cm(R, du, K, n), du, n, m, c);
  if (fam) fam[family_offset(n) + m] = make_float4((float)c[0], (float)c[1], (float)c[2], (float)c[3]);
  if (n == n64 && tab64)
    for (int i = 0; i < 4; ++i) tab64[4 * m + i] = c[i];
}

}  // namespace

cudaError_t launch_mlp_table(double R, double du, int K, double* tab64, float4* tab32, cudaStream_t s) {
  int threads = 128, blocks = (K + 1 + threads - 1) / threads;
  mlp_table_kernel<<<blocks, threads, 0, s>>>(R, du, K, tab64, tab32);
  return cudaGetLastError();
}

cudaError_t launch_mlp_family(double R, double du, int K, float4* fam, int n64, double* tab64, cudaStream_t s) {
  const int threads = 128;
  const dim3 grid((K + 1 + threads - 1) / threads, K);
  mlp_family_kernel<<<grid, threads, 0, s>>>(R, du, K, fam, n64, tab64);
  return cudaGetLastError();
}

}  // namespace pct
