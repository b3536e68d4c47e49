// Internal declarations shared by the library's translation units (not part
// of the C ABI). Device-side structs are passed to kernels by value.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pct {

constexpr int kQBits = 20;               // Q20 fixed-point grid coordinates
constexpr int32_t kQOne = 1 << kQBits;   // one voxel
// Single-precision grid coordinates are formed kQOff voxels above their value
// (q = fma(p, 1/h, n/2 + kQOff)) and the offset is removed after rounding to
// Q20: every coordinate within 8 voxels of the grid is then >= 8, where a
// float is already a whole multiple of 2^-20, so there the rounding is exact
// and the float itself is the Q20 node.
constexpr int kQOff = 16;
constexpr float kQClamp = 1000.0f;       // |q| clamp in voxels (never reached for valid records)
constexpr int kMaxNodes = 2048;          // K + 1 limit (shared-memory MLP table)
constexpr int kMaxDim = 512;             // per-axis voxel limit
constexpr int kSortAngles = 128;         // load-time ordering: gantry-angle bins (49 mrad; the 90 angles of the head workloads each have their own)
constexpr int kSortMid = 1024;           // load-time ordering: bins of the MLP's lateral midpoint between the quarter points
constexpr int kSortDiff = 32;            // load-time ordering: bins of the MLP's lateral change between the quarter points
constexpr float kSortDiffLim = 8.f;      // range +-kSortDiffLim (mm) of that change
constexpr int kSortLateral = kSortMid * kSortDiff;
// entries of the ordering's bin array: the bins, then one sum per scan tile
constexpr int64_t kSortHistEntries = (int64_t)kSortAngles * kSortLateral + 1024;
constexpr int kRowCap = 512;             // runs kept per history between the fused kernel's two passes
constexpr int kGroupRowCap = 384;        // runs kept in shared memory per history by the group kernel

// Grid and node geometry in the single-precision form the kernels use.
struct Geo {
  int nx, ny, nz;
  int K;          // interior nodes k = 0..K
  int E;          // straight extension nodes per side (k = -E..-1, K+1..K+E)
  float du;       // node spacing (mm), rounded from FP64
  float u0;       // first measurement plane (-R), rounded from FP64
  float hx, hy, hz;     // voxel size (mm)
  float ihx, ihy, ihz;  // 1/h rounded from FP64
  float hnx, hny, hnz;  // n/2 + kQOff
  float bx, by;         // half box extents in x and y (mm)
  // Largest change between consecutive nodes of each FP32 table column
  // (c1..c4): bounds the lateral step of an MLP segment. INFINITY: no bound
  // known, every history takes the general walk.
  float dmax[4];
};

// Geometry of a grid in the kernels' single-precision form; R, du, K, E from
// the FP64 derivation of the context. dmax = INFINITY until the table is known.
inline Geo make_geo(int nx, int ny, int nz, double hx, double hy, double hz, double R, double du, int K, int E) {
  Geo G{};
  G.nx = nx;
  G.ny = ny;
  G.nz = nz;
  G.K = K;
  G.E = E;
  G.du = (float)du;
  G.u0 = (float)(-R);
  G.hx = (float)hx;
  G.hy = (float)hy;
  G.hz = (float)hz;
  G.ihx = (float)(1.0 / hx);
  G.ihy = (float)(1.0 / hy);
  G.ihz = (float)(1.0 / hz);
  G.hnx = 0.5f * (float)nx + (float)kQOff;
  G.hny = 0.5f * (float)ny + (float)kQOff;
  G.hnz = 0.5f * (float)nz + (float)kQOff;
  G.bx = (float)(0.5 * nx * hx);
  G.by = (float)(0.5 * ny * hy);
  for (int i = 0; i < 4; ++i) G.dmax[i] = __builtin_inff();
  return G;
}

// dmax from the FP32 table (K + 1 nodes, host copy).
inline void set_table_bound(Geo& G, const float4* tab, int K) {
  float d[4] = {0.f, 0.f, 0.f, 0.f};
  for (int k = 1; k <= K; ++k) {
    const float a[4] = {tab[k].x - tab[k - 1].x, tab[k].y - tab[k - 1].y, tab[k].z - tab[k - 1].z,
                        tab[k].w - tab[k - 1].w};
    for (int i = 0; i < 4; ++i) d[i] = a[i] < 0.f ? (-a[i] > d[i] ? -a[i] : d[i]) : (a[i] > d[i] ? a[i] : d[i]);
  }
  for (int i = 0; i < 4; ++i) G.dmax[i] = d[i];
}

// Structure-of-arrays history records (device pointers).
struct Rec {
  const float *t0, *v0, *st0, *sv0, *t2, *v2, *st2, *sv2, *wepl, *cphi, *sphi;
};

// Object hull of the MLP (device pointers; range == nullptr: no hull, every
// proton's MLP spans the measurement planes). range[i] = iin | iout << 16 for
// stored history i: its MLP runs between nodes iin and iout with the table of
// a layer of n = iout - iin node intervals, fam + family_offset(n).
struct Hull {
  const int32_t* range;
  const float4* fam;
};

// Start of the table of thickness n (entries m = 0..n) in the table family:
// the tables of thickness 1 .. n-1 hold 2 + 3 + ... + n entries.
__host__ __device__ constexpr int64_t family_offset(int n) { return (int64_t)(n - 1) * (n + 2) / 2; }

// Total-variation superiorization parameters and device state.
struct TvsParams {
  float beta0, alpha, eps;
  int tries;
};
struct TvState {
  long long ell;  // trials so far
  int accepted;   // a trial of the current application was taken
  int pad;
};

// Launchers (pct_kernels.cu / pct_table.cu). All enqueue on `s` and return
// the launch error (cudaSuccess when queued).
cudaError_t launch_mlp_table(double R, double du, int K, double* tab64, float4* tab32, cudaStream_t s);
// Table family of every hull thickness n = 1..K into fam (family_offset(K+1)
// float4, may be null); with tab64 non-null also the FP64 table of n = n64
// ((n64+1) x 4 doubles).
cudaError_t launch_mlp_family(double R, double du, int K, float4* fam, int n64, double* tab64, cudaStream_t s);
// range[i] for stored histories [0, n) against the hull mask (M bytes).
cudaError_t launch_hull_ranges(const Geo& g, const Rec& r, int64_t n, const uint8_t* mask, int32_t* range,
                               cudaStream_t s);
// out[2p], out[2p+1] = (iin, iout) of load-order history first + p (stored
// position where[first + p], or first + p without a map).
cudaError_t launch_gather_ranges(const int32_t* range, const int64_t* where, int64_t first, int64_t count,
                                 int32_t* out, cudaStream_t s);
// Space carving: out[j] = 0 for every voxel on the (hull-free) row of a stored
// history with wepl <= wepl_max, else 1; then `dilate` 6-neighbour growth
// steps (tmp: M bytes of scratch).
cudaError_t launch_carve_hull(const Geo& g, const Rec& r, const float4* tab, int64_t n, float wepl_max, int dilate,
                              uint8_t* out, uint8_t* tmp, cudaStream_t s);
cudaError_t launch_validate(const Rec& r, int64_t n, int64_t base, float pos_limit, unsigned long long* first_bad,
                            cudaStream_t s);
// Order n records of one block by (angle bin, lateral bins of the MLP at the
// quarter points; tab: the FP32 MLP table of K + 1 nodes) into
// dst_rec[base .. base+n); where[base + i] receives the stored position of
// input record i (where must not be null). key/order: n entries; hist:
// kSortHistEntries (the bins and the scan's tile sums).
cudaError_t launch_sort_block(const Rec& src, int64_t n, int64_t base, float lat_lim, const float4* tab, int K,
                              Rec dst_rec, int64_t* where, unsigned* key, unsigned* hist, unsigned* order,
                              cudaStream_t s);
// Copy n records into dst_rec[base ..) in input order.
cudaError_t launch_copy_block(const Rec& src, int64_t n, int64_t base, Rec dst_rec, cudaStream_t s);
cudaError_t launch_count(const Geo& g, const Rec& r, const float4* tab, const Hull& hull, int64_t first, int64_t count,
                         unsigned int* cnt, int threads, cudaStream_t s);
// The first sweep's block pass without a hull, one lane per history: the
// update and the run counts of the block added to pair (M float2, zero on
// entry) by one vector reduction per run; then the block update from pair
// (1/s_j into inv_s, x += delta/s, pair zeroed; *overflow set where a float
// count reached 2^24).
cudaError_t launch_drop_fused_pair(const Geo& g, const Rec& r, const float4* tab, int64_t first, int64_t count,
                                   const float* x, float2* pair, float lambda, int flags, cudaStream_t s);
cudaError_t launch_drop_apply_pair(float* x, float2* pair, float* inv_s, int64_t M, int clamp, float clamp_min,
                                   int* overflow, cudaStream_t s);
cudaError_t launch_inv_counts(const unsigned int* cnt, float* inv_s, int64_t M, cudaStream_t s);
cudaError_t launch_counts_to_float(const unsigned int* cnt, float* out, int64_t M, cudaStream_t s);
// cnt non-null: also count the block's runs per voxel into cnt (zeroed by the
// caller). lanes: lanes per history, 1 (one thread per history) or, without
// a hull, 2, 4, 8, 16 or 32 (the group walk).
cudaError_t launch_drop_fused(const Geo& g, const Rec& r, const float4* tab, const Hull& hull, int64_t first, int64_t count,
                              const float* x, float* delta, float lambda, int flags, int lanes, cudaStream_t s,
                              unsigned int* cnt = nullptr);
// The group walk (T lanes per history, T in {2, 4, 8, 16, 32}; no hull): the fused
// kernel and the row export. prepare_drop_group sets the fused kernels'
// shared-memory limit for K + 1 table nodes; call it outside stream capture
// before the first launch for that K.
bool group_lanes_supported(int T);
cudaError_t prepare_drop_group(int T, int K);
cudaError_t launch_drop_group(int T, const Geo& g, const Rec& r, const float4* tab, int64_t first, int64_t count,
                              const float* x, float* delta, float lambda, int flags, cudaStream_t s,
                              unsigned int* cnt = nullptr);
cudaError_t launch_rows_group(int T, const Geo& g, const Rec& r, const float4* tab, int64_t first, int64_t count,
                              const int64_t* where, int64_t* row_ptr, int32_t* vox, float* len, int32_t* nodes,
                              bool fill, cudaStream_t s);
cudaError_t launch_drop_apply(float* x, float* delta, const float* inv_s, int64_t M, int clamp, float clamp_min,
                              cudaStream_t s);
// x_j += delta_j / s_j where s_j = counts_j > 0 (else unchanged), optional
// clamp; delta and counts are left as they are (a reduced block update).
cudaError_t launch_apply_reduced(float* x, const float* delta, const float* counts, int64_t M, int clamp,
                                 float clamp_min, cudaStream_t s);
// CARP: add a string's swept copy xs to sum / touch where any of its nb
// blocks (inv_s: nb x M) touches the voxel; then x = sum / touch where
// touched, else x0, and sum = touch = 0.
cudaError_t launch_carp_collect(const float* xs, const float* inv_s, int nb, int64_t M, float* sum, float* touch,
                                cudaStream_t s);
cudaError_t launch_carp_finish(float* x, const float* x0, float* sum, float* touch, int64_t M, int clamp,
                               float clamp_min, cudaStream_t s);
// One TVS perturbation of x (gradient, up to p.tries trials, commit); g, xp:
// M floats of scratch; acc: 3 doubles and st: the state, both zero on entry
// and left zero (st->ell keeps counting).
cudaError_t launch_tvs(float* x, int nx, int ny, int nz, const TvsParams& p, float* g, float* xp, double* acc,
                       TvState* st, cudaStream_t s);
// y[p] = a_i.x for histories first+p (load order through `where`, if given).
cudaError_t launch_project(const Geo& g, const Rec& r, const float4* tab, const Hull& hull, int64_t first, int64_t count,
                           const int64_t* where, const float* x, int flags, float* y, cudaStream_t s);
// *acc += sum over stored histories i = 0, stride, ... < n of (b_i - a_i.x)^2.
cudaError_t launch_residual(const Geo& g, const Rec& r, const float4* tab, const Hull& hull, int64_t n, int64_t stride, const float* x,
                            int flags, double* acc, cudaStream_t s);
cudaError_t launch_row_counts(const Geo& g, const Rec& r, const float4* tab, const Hull& hull, int64_t first, int64_t count,
                              const int64_t* where, int64_t* row_ptr, int lanes, cudaStream_t s);
cudaError_t launch_scan_rows(int64_t* row_ptr, int64_t count, cudaStream_t s);
cudaError_t launch_row_fill(const Geo& g, const Rec& r, const float4* tab, const Hull& hull, int64_t first, int64_t count,
                            const int64_t* where, const int64_t* row_ptr, int32_t* vox, float* len, int32_t* nodes,
                            int lanes, cudaStream_t s);

// Saves the calling thread's current device and restores it when the entry
// point returns: the library switches to a context's device for its work and
// must not leave the caller (or a later call that uses the current device) on
// another one.
struct DeviceGuard {
  int prev = -1;
  DeviceGuard() {
    if (cudaGetDevice(&prev) != cudaSuccess) {
      (void)cudaGetLastError();
      prev = -1;
    }
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
  DeviceGuard(const DeviceGuard&) = delete;
  DeviceGuard& operator=(const DeviceGuard&) = delete;
};

// Set the text that pct_last_error() returns on the calling thread.
void set_error_text(const char* msg);

}  // namespace pct
