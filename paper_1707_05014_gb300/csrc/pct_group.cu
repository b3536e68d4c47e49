// Group walk: T lanes (T = 2, 4, 8, 16 or 32) share one history, each lane taking
// one segment of the polyline per step (arXiv 1707.05014 Sec. 2: the row a_i
// of a proton is the length of its most-likely path in every voxel it
// touches; Sec. 2.1, Fig. 1: DROP projects each row once per sweep).
//
// The runs are exactly those of the one-lane walk (walk_proton), in the same
// order; only the summation order of chord pieces and of a_i.x differs.
//
// Per step of T segments (nodes s = klo + 1 + c T + lane):
//   1. every lane evaluates its node Q (the same FP32 formulas as
//      for_each_node) and takes the previous node P from its neighbour;
//   2. lane-local: the faces its segment crosses (each axis at most one face
//      when history_fast holds), their exact order and ties (the two-product
//      comparison of seg_fast), the voxel after each crossing and the pieces
//      of chord between crossings;
//   3. group: the run that ends at a lane's first crossing began at the last
//      crossing of an earlier lane (or an earlier step): a segmented prefix
//      sum of the chord pieces across the lanes (segments start at lanes with
//      crossings) gives its length, ballots give its positive-extent flag
//      and every run's position in path order;
//   4. lane-local: the lane's runs (at most three) go to the visitor.
// Runs are emitted where the one-lane walk emits them: when their exact
// extent is positive and their voxel is inside the grid. Histories that fail
// history_fast (a segment may cross two faces of one axis) are walked by lane
// 0 with walk_proton while the other lanes wait.
//
// The fused DROP kernel built on it records each history's row (voxel,
// chord) in shared memory (a row buffer per group), then forms a_i.x
// (compensated per lane over every T-th run, then a compensated butterfly
// across the group) and |a_i|^2 from the buffer, and scatters r_i a_i from it
// with every lane of the group; a row longer than the buffer is walked again
// for the gather and for the scatter.
#include "pct_drop.cuh"

namespace pct {
namespace {


template <int T>
struct Group {
  unsigned mask;  // the group's lanes within the warp
  int ln;         // lane within the group
  int base;       // warp lane of the group's lane 0
  __device__ __forceinline__ Group() {
    const int lane = threadIdx.x & 31;
    base = lane & ~(T - 1);
    ln = lane - base;
    mask = T == 32 ? 0xffffffffu : (((1u << (T & 31)) - 1u) << base);
  }
  // the group's ballot, bit l = lane l of the group
  __device__ __forceinline__ unsigned ballot(bool p) const {
    const unsigned b = __ballot_sync(mask, p);
    return T == 32 ? b : (b >> base) & ((1u << (T & 31)) - 1u);
  }
  __device__ __forceinline__ float up(float v, int d) const { return __shfl_up_sync(mask, v, d, T); }
  __device__ __forceinline__ float bcast(float v, int l) const { return __shfl_sync(mask, v, l, T); }
  __device__ __forceinline__ int bcast(int v, int l) const { return __shfl_sync(mask, v, l, T); }
  __device__ __forceinline__ float xr(float v, int d) const { return __shfl_xor_sync(mask, v, d, T); }
};

__device__ __forceinline__ int hibit(unsigned m) { return 31 - __clz(m); }  // m != 0


// Lane-local analysis of one segment P -> Q (history_fast: each axis crosses
// at most one face). The events are the distinct crossing times in order
// (tied axes step together).
struct SegEv {
  int m;                 // distinct events, 0..3
  float t0, t1, t2;      // their float fractions of the segment
  float n0;              // exact distance to the first event's face (0: the event is at P)
  bool tpos;             // the last event lies strictly before Q
  int ix, iy, iz;        // voxel holding P
  int s0x, s0y, s0z;     // steps taken at event 0
  int s1x, s1y, s1z;     // steps taken at event 1
};

__device__ __forceinline__ SegEv seg_events(const float3 P, const float3 Q) {
  SegEv e;
  const float bPx = __fadd_rd(P.x, kFloorBias), bPy = __fadd_rd(P.y, kFloorBias), bPz = __fadd_rd(P.z, kFloorBias);
  const float bQx = __fadd_rd(Q.x, kFloorBias), bQy = __fadd_rd(Q.y, kFloorBias), bQz = __fadd_rd(Q.z, kFloorBias);
  e.ix = vox_of(bPx);
  e.iy = vox_of(bPy);
  e.iz = vox_of(bPz);
  const bool cx = bQx != bPx, cy = bQy != bPy, cz = bQz != bPz;  // crossings
  const bool ux = bQx > bPx, uy = bQy > bPy, uz = bQz > bPz;      // moving up
  // exact distance to the crossed face (up: the face floor(Q), down: floor(P))
  // and exact axis length of the segment (near the grid both are exact)
  const float ndx = fabsf(__fsub_rn(__fsub_rn(ux ? bQx : bPx, kFloorBias), P.x));
  const float ndy = fabsf(__fsub_rn(__fsub_rn(uy ? bQy : bPy, kFloorBias), P.y));
  const float ndz = fabsf(__fsub_rn(__fsub_rn(uz ? bQz : bPz, kFloorBias), P.z));
  const float ddx = fabsf(__fsub_rn(Q.x, P.x)), ddy = fabsf(__fsub_rn(Q.y, P.y)), ddz = fabsf(__fsub_rn(Q.z, P.z));
  // exact pairwise order (< 0: the first axis crosses first, 0: tie)
  const int oxy = cmp_prod(ndx, ddy, ndy, ddx);
  const int oxz = cmp_prod(ndx, ddz, ndz, ddx);
  const int oyz = cmp_prod(ndy, ddz, ndz, ddy);
  const bool xy = cx && cy, xz = cx && cz, yz = cy && cz;
  // axes strictly before each axis, and the distinct event each axis belongs to
  const int nbx = (xy && oxy > 0) + (xz && oxz > 0);
  const int nby = (xy && oxy < 0) + (yz && oyz > 0);
  const int nbz = (xz && oxz < 0) + (yz && oyz < 0);
  const int kx = nbx - (nbx == 2 && oyz == 0), ky = nby - (nby == 2 && oxz == 0), kz = nbz - (nbz == 2 && oxy == 0);
  e.m = max(cx ? kx + 1 : 0, max(cy ? ky + 1 : 0, cz ? kz + 1 : 0));
  const float tx = __fdividef(ndx, ddx), ty = __fdividef(ndy, ddy), tz = __fdividef(ndz, ddz);
  // event k: the first of x, y, z (in that priority) with index k
  const bool ex0 = cx && kx == 0, ey0 = cy && ky == 0, ez0 = cz && kz == 0;
  const bool ex1 = cx && kx == 1, ey1 = cy && ky == 1, ez1 = cz && kz == 1;
  const bool ex2 = cx && kx == 2, ey2 = cy && ky == 2;
  e.t0 = ex0 ? tx : (ey0 ? ty : tz);
  e.t1 = ex1 ? tx : (ey1 ? ty : tz);
  e.t2 = ex2 ? tx : (ey2 ? ty : tz);
  e.n0 = ex0 ? ndx : (ey0 ? ndy : ndz);
  // last event: strictly before Q
  const int kl = e.m - 1;
  const bool exl = cx && kx == kl, eyl = cy && ky == kl;
  const float nl = exl ? ndx : (eyl ? ndy : ndz), dl = exl ? ddx : (eyl ? ddy : ddz);
  e.tpos = nl < dl;
  const int sx = ux ? 1 : -1, sy = uy ? 1 : -1, sz = uz ? 1 : -1;
  e.s0x = ex0 ? sx : 0;
  e.s0y = ey0 ? sy : 0;
  e.s0z = ez0 ? sz : 0;
  e.s1x = ex1 ? sx : 0;
  e.s1y = ey1 ? sy : 0;
  e.s1z = ez1 ? sz : 0;
  return e;
}

// The same by the float fractions, for segments whose crossing fractions are
// at least kTieWindow apart and from 1 (near = false): then the float order
// is the exact order and there are no ties. near = true: the caller takes
// seg_events.
__device__ __forceinline__ SegEv seg_events_float(const float3 P, const float3 Q, bool& near) {
  SegEv e;
  const float bPx = __fadd_rd(P.x, kFloorBias), bPy = __fadd_rd(P.y, kFloorBias), bPz = __fadd_rd(P.z, kFloorBias);
  const float bQx = __fadd_rd(Q.x, kFloorBias), bQy = __fadd_rd(Q.y, kFloorBias), bQz = __fadd_rd(Q.z, kFloorBias);
  e.ix = vox_of(bPx);
  e.iy = vox_of(bPy);
  e.iz = vox_of(bPz);
  const bool cx = bQx != bPx, cy = bQy != bPy, cz = bQz != bPz;
  const bool ux = bQx > bPx, uy = bQy > bPy, uz = bQz > bPz;
  const float ndx = fabsf(__fsub_rn(__fsub_rn(ux ? bQx : bPx, kFloorBias), P.x));
  const float ndy = fabsf(__fsub_rn(__fsub_rn(uy ? bQy : bPy, kFloorBias), P.y));
  const float ndz = fabsf(__fsub_rn(__fsub_rn(uz ? bQz : bPz, kFloorBias), P.z));
  const float tx = cx ? __fdividef(ndx, fabsf(__fsub_rn(Q.x, P.x))) : INFINITY;
  const float ty = cy ? __fdividef(ndy, fabsf(__fsub_rn(Q.y, P.y))) : INFINITY;
  const float tz = cz ? __fdividef(ndz, fabsf(__fsub_rn(Q.z, P.z))) : INFINITY;
  const float tmax = fmaxf(cx ? tx : 0.f, fmaxf(cy ? ty : 0.f, cz ? tz : 0.f));
  near = fabsf(tx - ty) < kTieWindow || fabsf(tx - tz) < kTieWindow || fabsf(ty - tz) < kTieWindow ||
         tmax > 1.f - kTieWindow;
  e.m = (int)cx + (int)cy + (int)cz;
  e.t0 = fminf(tx, fminf(ty, tz));
  e.t1 = fmaxf(fminf(tx, ty), fminf(fmaxf(tx, ty), tz));  // the median: the second event when m >= 2
  e.t2 = tmax;
  e.n0 = e.t0;  // > 0 exactly when the distance to the first face is
  e.tpos = true;
  const int sx = ux ? 1 : -1, sy = uy ? 1 : -1, sz = uz ? 1 : -1;
  const bool ex0 = tx == e.t0, ey0 = !ex0 && ty == e.t0, ez0 = !ex0 && !ey0;
  const bool ex1 = tx == e.t1, ey1 = !ex1 && ty == e.t1, ez1 = !ex1 && !ey1;
  e.s0x = ex0 ? sx : 0;
  e.s0y = ey0 ? sy : 0;
  e.s0z = ez0 && cz ? sz : 0;
  e.s1x = ex1 ? sx : 0;
  e.s1y = ey1 ? sy : 0;
  e.s1z = ez1 && cz ? sz : 0;
  return e;
}

__device__ __forceinline__ bool in_grid(const Geo& g, int ix, int iy, int iz) {
  return (unsigned)ix < (unsigned)g.nx && (unsigned)iy < (unsigned)g.ny && (unsigned)iz < (unsigned)g.nz;
}

// Fast group walk of one history over nodes klo .. khi; visit(j, len, pos)
// for every run, pos = its index in path order. Returns the run count
// (the same on every lane of the group).
template <int T, class Visit>
__device__ __forceinline__ int group_walk_fast(const Group<T>& G, const Geo& g, const float4* __restrict__ tab,
                                               const RecV& r, int klo, int khi, Visit& visit) {
  float3 cq;  // the last node of the previous step
  {
    const float2 tv = node_tv(g, tab, r, klo);
    cq = node_grid(g, r, __fmaf_rn((float)klo, g.du, g.u0), tv.x, tv.y);
  }
  float carry = 0.f;  // length of the open run so far
  bool cpos = false;  // the open run has positive exact extent
  int nrow = 0;
  const int nseg = khi - klo;
  const unsigned lt = (1u << G.ln) - 1u;  // lanes before this one
  for (int c0 = 0; c0 < nseg; c0 += T) {
    const int nact = min(T, nseg - c0);
    const bool act = G.ln < nact;
    const int s = klo + 1 + c0 + G.ln;
    float3 Q = cq;
    if (act) {
      const float2 tv = node_tv(g, tab, r, s);
      Q = node_grid(g, r, __fmaf_rn((float)s, g.du, g.u0), tv.x, tv.y);
    }
    float3 P;
    P.x = G.up(Q.x, 1);
    P.y = G.up(Q.y, 1);
    P.z = G.up(Q.z, 1);
    if (G.ln == 0) P = cq;
    // segment length (mm)
    const float fx = __fmul_rn(__fsub_rn(Q.x, P.x), g.hx), fy = __fmul_rn(__fsub_rn(Q.y, P.y), g.hy),
                fz = __fmul_rn(__fsub_rn(Q.z, P.z), g.hz);
    const float L2 = __fmaf_rn(fx, fx, __fmaf_rn(fy, fy, __fmul_rn(fz, fz)));
    const float L = act ? L2 * rsqrtf(L2) : 0.f;
    bool near;
    SegEv e = seg_events_float(P, Q, near);
    if (G.ballot(act && near)) e = seg_events(P, Q);  // a near tie somewhere in the step: exact order
    if (!act) e.m = 0;
    const float tl = e.m == 1 ? e.t0 : (e.m == 2 ? e.t1 : e.t2);
    const float w = e.m > 0 ? (1.f - tl) * L : L;  // the piece after the last event (or the whole segment)
    // group: crossings, and a segmented scan of the pieces (segments start at
    // lanes with crossings)
    const unsigned E = G.ballot(e.m > 0);
    const unsigned TP = G.ballot(e.m > 0 && e.tpos);
    const unsigned upto = E & (lt | (1u << G.ln));
    const int st = upto ? hibit(upto) : 0;
    float sc = w;
#pragma unroll
    for (int d = 1; d < T; d <<= 1) {
      const float v = G.up(sc, d);
      if (G.ln - d >= st) sc += v;
    }
    const float before = G.up(sc, 1);  // pieces since the last crossing, up to this lane's P
    const float tot = G.bcast(sc, T - 1);
    // the run ending at this lane's first crossing
    const unsigned prevE = E & lt;
    const int p = prevE ? hibit(prevE) : -1;
    const float len0 = (G.ln > 0 ? before : 0.f) + (p < 0 ? carry : 0.f) + e.t0 * L;
    const bool pos0 = e.n0 > 0.f || (p >= 0 ? (G.ln - p > 1 || ((TP >> p) & 1u)) : (cpos || G.ln > 0));
    // voxels of the runs ending at events 0, 1, 2
    const int ax = e.ix + e.s0x, ay = e.iy + e.s0y, az = e.iz + e.s0z;
    const int bx = ax + e.s1x, by = ay + e.s1y, bz = az + e.s1z;
    const bool em0 = e.m >= 1 && pos0 && in_grid(g, e.ix, e.iy, e.iz);
    const bool em1 = e.m >= 2 && in_grid(g, ax, ay, az);
    const bool em2 = e.m >= 3 && in_grid(g, bx, by, bz);
    const int cnt = (int)em0 + (int)em1 + (int)em2;
    const unsigned B0 = G.ballot(cnt & 1), B1 = G.ballot(cnt & 2);
    int pos = nrow + __popc(B0 & lt) + 2 * __popc(B1 & lt);
    if (em0) visit(e.ix + g.nx * (e.iy + g.ny * e.iz), len0, pos++);
    if (em1) visit(ax + g.nx * (ay + g.ny * az), (e.t1 - e.t0) * L, pos++);
    if (em2) visit(bx + g.nx * (by + g.ny * bz), (e.t2 - e.t1) * L, pos);
    nrow += __popc(B0) + 2 * __popc(B1);
    // the open run after this step
    if (E) {
      const int last = hibit(E);
      carry = tot;
      cpos = ((TP >> last) & 1u) || last < nact - 1;
    } else {
      carry += tot;
      cpos = true;
    }
    const int ll = nact - 1;
    cq.x = G.bcast(Q.x, ll);
    cq.y = G.bcast(Q.y, ll);
    cq.z = G.bcast(Q.z, ll);
  }
  // the last run ends at node khi
  const int ix = vox_of(__fadd_rd(cq.x, kFloorBias)), iy = vox_of(__fadd_rd(cq.y, kFloorBias)),
            iz = vox_of(__fadd_rd(cq.z, kFloorBias));
  if (cpos && in_grid(g, ix, iy, iz)) {
    if (G.ln == 0) visit(ix + g.nx * (iy + g.ny * iz), carry, nrow);
    ++nrow;
  }
  return nrow;
}

// Either walk for the group: the fast group walk, or lane 0 alone with the
// one-lane walk (runs in path order with their positions).
template <int T, class Visit>
__device__ __forceinline__ int group_walk(const Group<T>& G, const Geo& g, const float4* __restrict__ tab,
                                          const RecV& r, Visit& visit) {
  int klo, khi;
  node_range(g, r, klo, khi);
  if (history_fast(g, r)) return group_walk_fast<T>(G, g, tab, r, klo, khi, visit);
  int n = 0;
  if (G.ln == 0) walk_proton(g, tab, r, [&](int j, float l) { visit(j, l, n++); });
  return G.bcast(n, 0);
}

// Sum over the group of a compensated pair (y, c): the true lane sum is y - c.
// Butterfly of TwoSum steps; every lane gets the total.
template <int T>
__device__ __forceinline__ float group_sum_comp(const Group<T>& G, float y, float c) {
  float s = y, err = -c;
#pragma unroll
  for (int d = T / 2; d >= 1; d >>= 1) {
    const float o = G.xr(s, d), oe = G.xr(err, d);
    const float t = __fadd_rn(s, o);
    const float bp = __fsub_rn(t, s);
    const float ts = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(o, bp));  // s + o = t + ts exactly
    s = t;
    err = __fadd_rn(__fadd_rn(err, oe), ts);
  }
  return __fadd_rn(s, err);
}

template <int T>
__device__ __forceinline__ float group_sum(const Group<T>& G, float v) {
#pragma unroll
  for (int d = T / 2; d >= 1; d >>= 1) v = __fadd_rn(v, G.xr(v, d));
  return v;
}

__device__ __forceinline__ void load_tab(const float4* __restrict__ src, float4* dst, int n) {
  for (int k = threadIdx.x; k < n; k += blockDim.x) dst[k] = src[k];
  __syncthreads();
}

// Threads per CTA of the group kernels: 256, or 32 groups for T < 8 (each
// group holds a kGroupRowCap-run row in shared memory, 3 KB, so 128 groups of
// two lanes would not fit). kGroupMinCtas: the register budget (64 per thread).
template <int T>
constexpr int kGroupThreads = T >= 8 ? 256 : 32 * T;
template <int T>
constexpr int kGroupMinCtas = 1024 / kGroupThreads<T>;
inline int group_threads(int T) { return T >= 8 ? 256 : 32 * T; }

// Fused MLP + DROP projection, T lanes per history; persistent over the
// block's histories (group q takes histories q, q + groups, ...). kCount:
// also count every run into cnt (the block's s_j).
template <int T, bool kPlain, bool kCount>
__global__ void __launch_bounds__(kGroupThreads<T>, kGroupMinCtas<T>) drop_group_kernel(Geo g, Rec r, const float4* __restrict__ tab_g,
                                                                  int64_t first, int64_t count,
                                                                  const float* __restrict__ x,
                                                                  float* __restrict__ delta, float lambda,
                                                                  unsigned int* __restrict__ cnt, int rowcap) {
  extern __shared__ float4 smem[];
  float4* tab = smem;
  load_tab(tab_g, tab, g.K + 1);
  const Group<T> G;
  const int gib = threadIdx.x / T;
  uint2* rows = reinterpret_cast<uint2*>(smem + (g.K + 1)) + (size_t)gib * rowcap;
  const int64_t groups = (int64_t)gridDim.x * (kGroupThreads<T> / T);
  for (int64_t p = (int64_t)blockIdx.x * (kGroupThreads<T> / T) + gib; p < count; p += groups) {
    const RecV v = load_rec(r, first + p);
    // walk: the row goes to the group's buffer (no global loads in the walk,
    // so no lane waits on memory between steps)
    auto record = [&](int j, float l, int pos) {
      if (pos < rowcap) rows[pos] = make_uint2((unsigned)j, __float_as_uint(l));
    };
    const int nrow = group_walk<T>(G, g, tab, v, record);
    __syncwarp(G.mask);
    float y = 0.f, c = 0.f, nn = 0.f;
    auto gather = [&](int j, float l) {
      const float xj = __ldg(x + j);
      if (kPlain) {
        y = __fmaf_rn(l, xj, y);
      } else {
        const float term = __fsub_rn(__fmul_rn(l, xj), c);
        const float t = __fadd_rn(y, term);
        c = __fsub_rn(__fsub_rn(t, y), term);
        y = t;
      }
      nn = __fmaf_rn(l, l, nn);
    };
    if (nrow <= rowcap) {
      // a_i.x and |a_i|^2: every lane takes every T-th run of the row
      for (int q = G.ln; q < nrow; q += T) {
        const uint2 e = rows[q];
        if (kCount) atomicAdd(cnt + e.x, 1u);
        gather((int)e.x, __uint_as_float(e.y));
      }
    } else {
      auto gather_walk = [&](int j, float l, int) {
        if (kCount) atomicAdd(cnt + j, 1u);
        gather(j, l);
      };
      group_walk<T>(G, g, tab, v, gather_walk);
    }
    const float yy = kPlain ? group_sum<T>(G, y) : group_sum_comp<T>(G, y, c);
    const float nsum = group_sum<T>(G, nn);
    if (nsum > 0.f) {
      const float ri = lambda * __fsub_rn(v.wepl, yy) / nsum;
      if (nrow <= rowcap) {
        for (int q = G.ln; q < nrow; q += T) {
          const uint2 e = rows[q];
          atomicAdd(delta + e.x, __uint_as_float(e.y) * ri);
        }
      } else {
        auto scatter = [&](int j, float l, int) { atomicAdd(delta + j, l * ri); };
        group_walk<T>(G, g, tab, v, scatter);
      }
    }
    __syncwarp(G.mask);  // the row buffer is reused by the next history
  }
}

// Row export through the group walk: counts, then (voxel, chord) in path
// order and, optionally, the Q20 nodes k = 0..K.
template <int T>
__global__ void __launch_bounds__(kGroupThreads<T>) row_count_group_kernel(Geo g, Rec r, const float4* __restrict__ tab_g,
                                                                       int64_t first, int64_t count,
                                                                       const int64_t* __restrict__ where,
                                                                       int64_t* __restrict__ row_ptr) {
  extern __shared__ float4 smem[];
  load_tab(tab_g, smem, g.K + 1);
  const Group<T> G;
  const int64_t groups = (int64_t)gridDim.x * (kGroupThreads<T> / T);
  for (int64_t p = (int64_t)blockIdx.x * (kGroupThreads<T> / T) + threadIdx.x / T; p < count; p += groups) {
    const int64_t i = where ? where[first + p] : first + p;
    const RecV v = load_rec(r, i);
    auto none = [](int, float, int) {};
    const int n = group_walk<T>(G, g, smem, v, none);
    if (G.ln == 0) row_ptr[p + 1] = n;
  }
}

template <int T>
__global__ void __launch_bounds__(kGroupThreads<T>) row_fill_group_kernel(Geo g, Rec r, const float4* __restrict__ tab_g,
                                                                      int64_t first, int64_t count,
                                                                      const int64_t* __restrict__ where,
                                                                      const int64_t* __restrict__ row_ptr,
                                                                      int32_t* __restrict__ vox,
                                                                      float* __restrict__ len,
                                                                      int32_t* __restrict__ nodes) {
  extern __shared__ float4 smem[];
  load_tab(tab_g, smem, g.K + 1);
  const Group<T> G;
  const int64_t groups = (int64_t)gridDim.x * (kGroupThreads<T> / T);
  for (int64_t p = (int64_t)blockIdx.x * (kGroupThreads<T> / T) + threadIdx.x / T; p < count; p += groups) {
    const int64_t i = where ? where[first + p] : first + p;
    const RecV v = load_rec(r, i);
    const int64_t o = row_ptr[p];
    auto put = [&](int j, float l, int pos) {
      vox[o + pos] = j;
      len[o + pos] = l;
    };
    group_walk<T>(G, g, smem, v, put);
    if (nodes) {
      int32_t* out = nodes + p * (g.K + 1) * 3;
      for (int k = G.ln; k <= g.K; k += T) {
        const int3 Q = node_q(g, smem, v, k);
        out[3 * k + 0] = Q.x;
        out[3 * k + 1] = Q.y;
        out[3 * k + 2] = Q.z;
      }
    }
  }
}

// Per-device state below is kept for devices 0 .. kMaxDevices - 1 (the
// current device when a context works on it).
constexpr int kMaxDevices = 64;

inline int current_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) dev = 0;
  return dev;
}

inline unsigned group_grid(int64_t count, int T, int per_sm) {
  static int sms[kMaxDevices];
  const int dev = current_device();
  if (!sms[dev]) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    sms[dev] = n > 0 ? n : 1;
  }
  const int per_cta = group_threads(T) / T;
  const int64_t need = (count + per_cta - 1) / per_cta;
  const int64_t cap = (int64_t)sms[dev] * per_sm;
  return (unsigned)(need < 1 ? 1 : (need < cap ? need : cap));
}

// Dynamic shared memory and resident blocks per SM of one drop_group_kernel
// instantiation on one device (the attribute is a device's). The attribute
// is raised (and the occupancy taken) once per size, outside stream capture:
// launch_drop_group is first reached from prepare_drop_group when a context
// is created.
struct GroupLaunchInfo {
  size_t smem_set = 0;   // largest dynamic shared memory allowed so far
  size_t smem_occ = 0;   // size the occupancy below was taken for
  int per_sm = 0;
};

template <int T, bool kPlain, bool kCount>
GroupLaunchInfo& launch_info() {
  static GroupLaunchInfo info[kMaxDevices];
  return info[current_device()];
}

inline size_t drop_group_smem(int T, int K) {
  return (size_t)(K + 1) * sizeof(float4) + (size_t)(group_threads(T) / T) * kGroupRowCap * sizeof(uint2);
}

template <int T, bool kPlain, bool kCount>
cudaError_t prepare_drop_group_t(int K) {
  GroupLaunchInfo& info = launch_info<T, kPlain, kCount>();
  const size_t smem = drop_group_smem(T, K);
  auto kern = drop_group_kernel<T, kPlain, kCount>;
  if (info.smem_set < smem) {
    const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    info.smem_set = smem;
  }
  if (info.smem_occ != smem) {
    int per_sm = 0;
    const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kGroupThreads<T>, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    info.per_sm = per_sm;
    info.smem_occ = smem;
  }
  return cudaSuccess;
}

template <int T, bool kPlain, bool kCount>
cudaError_t launch_drop_group_t(const Geo& g, const Rec& r, const float4* tab, int64_t first, int64_t count,
                                const float* x, float* delta, float lambda, unsigned* cnt, cudaStream_t s) {
  cudaError_t e = prepare_drop_group_t<T, kPlain, kCount>(g.K);
  if (e != cudaSuccess) return e;
  const GroupLaunchInfo& info = launch_info<T, kPlain, kCount>();
  drop_group_kernel<T, kPlain, kCount><<<group_grid(count, T, info.per_sm), kGroupThreads<T>, info.smem_occ, s>>>(
      g, r, tab, first, count, x, delta, lambda, cnt, kGroupRowCap);
  return cudaGetLastError();
}

template <int T>
cudaError_t prepare_drop_group_all(int K) {
  cudaError_t e = prepare_drop_group_t<T, false, false>(K);
  if (e == cudaSuccess) e = prepare_drop_group_t<T, true, false>(K);
  if (e == cudaSuccess) e = prepare_drop_group_t<T, false, true>(K);
  if (e == cudaSuccess) e = prepare_drop_group_t<T, true, true>(K);
  return e;
}

template <int T>
cudaError_t launch_drop_group_any(const Geo& g, const Rec& r, const float4* tab, int64_t first, int64_t count,
                                  const float* x, float* delta, float lambda, bool plain, unsigned* cnt,
                                  cudaStream_t s) {
  if (cnt)
    return plain ? launch_drop_group_t<T, true, true>(g, r, tab, first, count, x, delta, lambda, cnt, s)
                 : launch_drop_group_t<T, false, true>(g, r, tab, first, count, x, delta, lambda, cnt, s);
  return plain ? launch_drop_group_t<T, true, false>(g, r, tab, first, count, x, delta, lambda, cnt, s)
               : launch_drop_group_t<T, false, false>(g, r, tab, first, count, x, delta, lambda, cnt, s);
}

template <int T>
cudaError_t launch_rows_group_t(const Geo& g, const Rec& r, const float4* tab, int64_t first, int64_t count,
                                const int64_t* where, int64_t* row_ptr, int32_t* vox, float* len, int32_t* nodes,
                                bool fill, cudaStream_t s) {
  const size_t smem = (size_t)(g.K + 1) * sizeof(float4);  // <= 32 KB (K + 1 <= 2048)
  if (fill)
    row_fill_group_kernel<T><<<group_grid(count, T, 4), kGroupThreads<T>, smem, s>>>(g, r, tab, first, count, where,
                                                                                 row_ptr, vox, len, nodes);
  else
    row_count_group_kernel<T><<<group_grid(count, T, 4), kGroupThreads<T>, smem, s>>>(g, r, tab, first, count, where,
                                                                                  row_ptr);
  return cudaGetLastError();
}

}  // namespace

bool group_lanes_supported(int T) { return T == 2 || T == 4 || T == 8 || T == 16 || T == 32; }

cudaError_t prepare_drop_group(int T, int K) {
  switch (T) {
    case 2: return prepare_drop_group_all<2>(K);
    case 4: return prepare_drop_group_all<4>(K);
    case 8: return prepare_drop_group_all<8>(K);
    case 16: return prepare_drop_group_all<16>(K);
    case 32: return prepare_drop_group_all<32>(K);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_drop_group(int T, const Geo& g, const Rec& r, const float4* tab, int64_t first, int64_t count,
                              const float* x, float* delta, float lambda, int flags, cudaStream_t s,
                              unsigned int* cnt) {
  if (count <= 0) return cudaSuccess;
  const bool plain = (flags & 2) != 0;
  switch (T) {
    case 2: return launch_drop_group_any<2>(g, r, tab, first, count, x, delta, lambda, plain, cnt, s);
    case 4: return launch_drop_group_any<4>(g, r, tab, first, count, x, delta, lambda, plain, cnt, s);
    case 8: return launch_drop_group_any<8>(g, r, tab, first, count, x, delta, lambda, plain, cnt, s);
    case 16: return launch_drop_group_any<16>(g, r, tab, first, count, x, delta, lambda, plain, cnt, s);
    case 32: return launch_drop_group_any<32>(g, r, tab, first, count, x, delta, lambda, plain, cnt, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_rows_group(int T, const Geo& g, const Rec& r, const float4* tab, int64_t first, int64_t count,
                              const int64_t* where, int64_t* row_ptr, int32_t* vox, float* len, int32_t* nodes,
                              bool fill, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  switch (T) {
    case 2: return launch_rows_group_t<2>(g, r, tab, first, count, where, row_ptr, vox, len, nodes, fill, s);
    case 4: return launch_rows_group_t<4>(g, r, tab, first, count, where, row_ptr, vox, len, nodes, fill, s);
    case 8: return launch_rows_group_t<8>(g, r, tab, first, count, where, row_ptr, vox, len, nodes, fill, s);
    case 16: return launch_rows_group_t<16>(g, r, tab, first, count, where, row_ptr, vox, len, nodes, fill, s);
    case 32: return launch_rows_group_t<32>(g, r, tab, first, count, where, row_ptr, vox, len, nodes, fill, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace pct
