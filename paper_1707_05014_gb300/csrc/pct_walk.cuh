// Device-side MLP node evaluation and exact integer voxel walk.
//
// arXiv 1707.05014 Sec. 2: a row of A holds, for one proton, the length of
// its most-likely path in every voxel it touches. The path here is the
// polyline through the MLP nodes u_k = u0 + k du (k = 0..K between the
// measurement planes, from the FP64 coefficient table rounded to FP32) and
// the straight extensions along the measured slopes (k < 0 and k > K).
//
// Bit-exact contract (the oracle's FP32 mode follows the same definition):
//   t_k = fma(c4, st2, fma(c3, t2, fma(c2, st0, c1*t0)))   (same for v)
//   x = fma(u, cos, -(t*sin)), y = fma(u, sin, t*cos), z = v
//   q = fma(p, 1/h, n/2 + 16), clamped to +-1000,
//   Q = rint(q * 2^20) - 16 * 2^20 (half even)
// Every product is a separately rounded __fmul_rn and every fused step an
// explicit __fmaf_rn, so the compiler cannot contract or reorder them.
// Between consecutive nodes the face crossings are ordered exactly (by
// cross-multiplication of the Q20 distances); voxels are half-open [i, i+1),
// tied crossings step together, and a run (maximal stretch in one voxel) is
// reported only when its exact extent is positive. The indices are exact;
// chord lengths are single precision (segment length from the node
// differences, crossing parameters by fast division), within 1e-5 relative
// of the FP64 oracle.
//
// The 16-voxel offset of q makes every coordinate within 8 voxels of the grid
// at least 8, where a float is a whole multiple of 2^-20: there q IS the Q20
// node (q * 2^20 is an integer) and differences of such floats, and the
// fused products of two of them, are exact. The fast walk (walk_fast) uses
// this to take every decision that shapes an emitted run on the floats
// themselves, with the same outcome as the integer walk (walk_segment) on
// the quantised nodes; far from the grid, where the two may round a
// coordinate differently, nothing is emitted and both return to the same
// voxel before the grid is reached.
#pragma once

#include "pct_internal.h"

namespace pct {

struct RecV {
  float t0, v0, st0, sv0, t2, v2, st2, sv2, wepl, cp, sp;
};

// Records are streamed once per sweep: load them with the evict-first hint so
// that they do not push the image and the update buffer out of L2.
__device__ __forceinline__ RecV load_rec(const Rec& r, int64_t i) {
  RecV v;
  v.t0 = __ldcs(r.t0 + i);
  v.v0 = __ldcs(r.v0 + i);
  v.st0 = __ldcs(r.st0 + i);
  v.sv0 = __ldcs(r.sv0 + i);
  v.t2 = __ldcs(r.t2 + i);
  v.v2 = __ldcs(r.v2 + i);
  v.st2 = __ldcs(r.st2 + i);
  v.sv2 = __ldcs(r.sv2 + i);
  v.wepl = __ldcs(r.wepl + i);
  v.cp = __ldcs(r.cphi + i);
  v.sp = __ldcs(r.sphi + i);
  return v;
}

// Q = rint(q * 2^20) - kQOff * 2^20 (grid units). The contract also clamps q
// to +-1000 voxels first; pct_create rejects grids for which a validated
// record could reach that range, so the clamp is the identity here and is
// not evaluated.
__device__ __forceinline__ int32_t quantise(float q) {
  return __float2int_rn(__fmul_rn(q, (float)kQOne)) - kQOff * kQOne;
}

// Lateral (t) and vertical (v) position of node k in mm.
__device__ __forceinline__ float2 node_tv(const Geo& g, const float4* __restrict__ tab, const RecV& r, int k) {
  float t, v;
  if (k < 0) {
    const float dk = __fmul_rn((float)k, g.du);
    t = __fmaf_rn(r.st0, dk, r.t0);
    v = __fmaf_rn(r.sv0, dk, r.v0);
  } else if (k > g.K) {
    const float dk = __fmul_rn((float)(k - g.K), g.du);
    t = __fmaf_rn(r.st2, dk, r.t2);
    v = __fmaf_rn(r.sv2, dk, r.v2);
  } else {
    const float4 c = tab[k];
    t = __fmaf_rn(c.w, r.st2, __fmaf_rn(c.z, r.t2, __fmaf_rn(c.y, r.st0, __fmul_rn(c.x, r.t0))));
    v = __fmaf_rn(c.w, r.sv2, __fmaf_rn(c.z, r.v2, __fmaf_rn(c.y, r.sv0, __fmul_rn(c.x, r.v0))));
  }
  return make_float2(t, v);
}

// Grid coordinates (voxels, float) of the node at depth u with lateral and
// vertical position (t, v).
__device__ __forceinline__ float3 node_grid(const Geo& g, const RecV& r, float u, float t, float v) {
  const float ts = __fmul_rn(t, r.sp), tc = __fmul_rn(t, r.cp);
  const float x = __fmaf_rn(u, r.cp, -ts);
  const float y = __fmaf_rn(u, r.sp, tc);
  return make_float3(__fmaf_rn(x, g.ihx, g.hnx), __fmaf_rn(y, g.ihy, g.hny), __fmaf_rn(v, g.ihz, g.hnz));
}

__device__ __forceinline__ int3 quantise3(float3 q) { return make_int3(quantise(q.x), quantise(q.y), quantise(q.z)); }

// Q20 grid coordinates of node k.
__device__ __forceinline__ int3 node_q(const Geo& g, const float4* __restrict__ tab, const RecV& r, int k) {
  const float2 tv = node_tv(g, tab, r, k);
  return quantise3(node_grid(g, r, __fmaf_rn((float)k, g.du, g.u0), tv.x, tv.y));
}

__device__ __forceinline__ int floor_q(int32_t q) { return q >> kQBits; }  // arithmetic shift = floor

// Depth parameter at which the line p(u) = u d + (a + s u) e_t (xy only)
// enters (first = true: the largest entering u) or leaves (the smallest
// leaving u) the box |x| <= bx, |y| <= by. Non-finite results are replaced by
// the unconstrained value (-inf for entering, +inf for leaving).
__device__ __forceinline__ float box_param(const Geo& g, const RecV& r, float a, float s, bool entering) {
  // x(u) = u (c - s sn) - a sn,  y(u) = u (sn + s c) + a c
  const float ax = r.cp - s * r.sp, bx = -a * r.sp;
  const float ay = r.sp + s * r.cp, by = a * r.cp;
  float res = entering ? -INFINITY : INFINITY;
  const float A[2] = {ax, ay}, Bc[2] = {bx, by}, H[2] = {g.bx, g.by};
  for (int i = 0; i < 2; ++i) {
    if (fabsf(A[i]) < 1e-12f) continue;
    const float u1 = (-H[i] - Bc[i]) / A[i], u2 = (H[i] - Bc[i]) / A[i];
    const float lo = fminf(u1, u2), hi = fmaxf(u1, u2);
    if (entering) {
      if (isfinite(lo)) res = fmaxf(res, lo);
    } else {
      if (isfinite(hi)) res = fminf(res, hi);
    }
  }
  return res;
}

// Node range of one proton. Nodes before -E and after K+E lie outside the
// box's circumscribed cylinder. A straight line meets the convex box in one
// interval, so any range that starts before the entry ray reaches the box
// and ends after the exit ray leaves it gives the same runs; the range here
// is the box-clipped one widened by two nodes (one voxel) on each side.
__device__ __forceinline__ void node_range(const Geo& g, const RecV& r, int& klo, int& khi) {
  klo = -g.E;
  khi = g.K + g.E;
  // entry ray: t = t0 + st0 (u - u0) = (t0 - st0 u0) + st0 u
  const float ue = box_param(g, r, r.t0 - r.st0 * g.u0, r.st0, true);
  if (isfinite(ue)) klo = max(klo, min(0, (int)floorf((ue - g.u0) / g.du) - 2));
  // exit ray: t = t2 + st2 (u - u2) with u2 = -u0
  const float ux = box_param(g, r, r.t2 + r.st2 * g.u0, r.st2, false);
  if (isfinite(ux)) khi = min(khi, max(g.K, g.K + (int)ceilf((ux + g.u0) / g.du) + 2));
}

// Segment state carried along the polyline (see walk_proton for the rules).
struct WalkState {
  int3 P;        // current node, Q20
  float3 qP;     // current node, float grid coordinates
  int cx, cy, cz;  // voxel holding P
  float run;     // length of the current run so far (mm)
  bool pos;      // the current run has positive exact extent
};

template <class Visit>
__device__ __forceinline__ void emit_run(const Geo& g, WalkState& s, Visit& visit) {
  if (s.pos && (unsigned)s.cx < (unsigned)g.nx && (unsigned)s.cy < (unsigned)g.ny && (unsigned)s.cz < (unsigned)g.nz)
    visit(s.cx + g.nx * (s.cy + g.ny * s.cz), s.run);
  s.run = 0.f;
  s.pos = false;
}

// Advance the walk from s.P to the next node (Q, q), emitting finished runs.
template <class Visit>
__device__ __forceinline__ void walk_segment(const Geo& g, WalkState& s, const float3 q, Visit& visit) {
  const int3 Q = quantise3(q);
  const int Dx = Q.x - s.P.x, Dy = Q.y - s.P.y, Dz = Q.z - s.P.z;
  // Segment length. The float grid coordinates differ from the Q20 nodes by
  // at most 2^-21 voxel (the rounding to Q20), far inside the chord
  // tolerance; differences of nearby floats are exact.
  const float fx = (q.x - s.qP.x) * g.hx, fy = (q.y - s.qP.y) * g.hy, fz = (q.z - s.qP.z) * g.hz;
  const float L2 = __fmaf_rn(fx, fx, __fmaf_rn(fy, fy, fz * fz));
  const bool moved = (Dx | Dy | Dz) != 0;
  const float L = moved ? L2 * rsqrtf(L2) : 0.f;
  const int nx = floor_q(Q.x), ny = floor_q(Q.y), nz = floor_q(Q.z);
  const int sx = nx - s.cx, sy = ny - s.cy, sz = nz - s.cz;
  if ((sx | sy | sz) == 0) {
    // no face crossed: the whole segment extends the current run
    s.run += L;
    s.pos |= moved;
  } else if (abs(sx) <= 1 && abs(sy) <= 1 && abs(sz) <= 1) {
    // Each crossing axis crosses exactly one face, at the exact fraction
    // n/d of the segment. Events are ordered by the float fractions (fast
    // division, 2 ulp); where two of them lie within 1e-6 of each other the
    // exact 32x32->64-bit cross-multiplication decides order and ties. Two
    // distinct fractions differ by at least 1/(d1 d2) but may round alike,
    // hence the window; a float fraction is 0 exactly when n = 0.
    const uint32_t ddx = (uint32_t)abs(Dx), ddy = (uint32_t)abs(Dy), ddz = (uint32_t)abs(Dz);
    const uint32_t ndx = sx > 0 ? (uint32_t)(nx * kQOne - s.P.x) : (uint32_t)(s.P.x - s.cx * kQOne);
    const uint32_t ndy = sy > 0 ? (uint32_t)(ny * kQOne - s.P.y) : (uint32_t)(s.P.y - s.cy * kQOne);
    const uint32_t ndz = sz > 0 ? (uint32_t)(nz * kQOne - s.P.z) : (uint32_t)(s.P.z - s.cz * kQOne);
    float tx = sx ? __fdividef((float)ndx, (float)ddx) : INFINITY;
    float ty = sy ? __fdividef((float)ndy, (float)ddy) : INFINITY;
    float tz = sz ? __fdividef((float)ndz, (float)ddz) : INFINITY;
    float tprev = 0.f;
    bool first = true;
    uint32_t ln = 0, ld = 1;  // exact fraction of the latest event
    for (;;) {
      const float m = fminf(tx, fminf(ty, tz));
      if (m == INFINITY) break;
      const float lim = __fmaf_rn(m, 1e-6f, m) + 1e-7f;
      bool ex = tx <= lim, ey = ty <= lim, ez = tz <= lim;
      uint32_t bn, bd;
      if ((int)ex + (int)ey + (int)ez > 1) {
        // near tie: keep the exact minima only
        bn = 0xffffffffu;
        bd = 1;
        if (ex) {
          bn = ndx;
          bd = ddx;
        }
        if (ey && (uint64_t)ndy * bd < (uint64_t)bn * ddy) {
          bn = ndy;
          bd = ddy;
        }
        if (ez && (uint64_t)ndz * bd < (uint64_t)bn * ddz) {
          bn = ndz;
          bd = ddz;
        }
        ex = ex && (uint64_t)ndx * bd == (uint64_t)bn * ddx;
        ey = ey && (uint64_t)ndy * bd == (uint64_t)bn * ddy;
        ez = ez && (uint64_t)ndz * bd == (uint64_t)bn * ddz;
      } else {
        bn = ex ? ndx : (ey ? ndy : ndz);
        bd = ex ? ddx : (ey ? ddy : ddz);
      }
      s.run += (m - tprev) * L;
      s.pos |= !first || bn > 0;  // later events are exactly after the previous one
      emit_run(g, s, visit);
      if (ex) {
        s.cx += sx;
        tx = INFINITY;
      }
      if (ey) {
        s.cy += sy;
        ty = INFINITY;
      }
      if (ez) {
        s.cz += sz;
        tz = INFINITY;
      }
      tprev = m;
      first = false;
      ln = bn;
      ld = bd;
    }
    s.run += (1.f - tprev) * L;
    s.pos |= ln < ld;
  } else {
    // general case: an axis may cross several faces
    const uint32_t adx = (uint32_t)abs(Dx), ady = (uint32_t)abs(Dy), adz = (uint32_t)abs(Dz);
    uint32_t dx = Dx > 0 ? (uint32_t)((s.cx + 1) * kQOne - s.P.x) : (uint32_t)(s.P.x - s.cx * kQOne);
    uint32_t dy = Dy > 0 ? (uint32_t)((s.cy + 1) * kQOne - s.P.y) : (uint32_t)(s.P.y - s.cy * kQOne);
    uint32_t dz = Dz > 0 ? (uint32_t)((s.cz + 1) * kQOne - s.P.z) : (uint32_t)(s.P.z - s.cz * kQOne);
    uint32_t pn = 0, pd = 1;
    float tprev = 0.f;
    for (;;) {
      // tau <= 1 moving up (a point on a face belongs to the higher voxel),
      // tau < 1 moving down
      const bool ax = Dx > 0 ? dx <= adx : (Dx < 0 && dx < adx);
      const bool ay = Dy > 0 ? dy <= ady : (Dy < 0 && dy < ady);
      const bool az = Dz > 0 ? dz <= adz : (Dz < 0 && dz < adz);
      if (!(ax | ay | az)) break;
      uint32_t bn = 0, bd = 1;
      bool have = false;
      if (ax) {
        bn = dx;
        bd = adx;
        have = true;
      }
      if (ay && (!have || (uint64_t)dy * bd < (uint64_t)bn * ady)) {
        bn = dy;
        bd = ady;
        have = true;
      }
      if (az && (!have || (uint64_t)dz * bd < (uint64_t)bn * adz)) {
        bn = dz;
        bd = adz;
      }
      const float tc = __fdividef((float)bn, (float)bd);
      s.run += (tc - tprev) * L;
      s.pos |= (uint64_t)bn * pd > (uint64_t)pn * bd;
      emit_run(g, s, visit);
      if (ax && (uint64_t)dx * bd == (uint64_t)bn * adx) {
        s.cx += Dx > 0 ? 1 : -1;
        dx += kQOne;
      }
      if (ay && (uint64_t)dy * bd == (uint64_t)bn * ady) {
        s.cy += Dy > 0 ? 1 : -1;
        dy += kQOne;
      }
      if (az && (uint64_t)dz * bd == (uint64_t)bn * adz) {
        s.cz += Dz > 0 ? 1 : -1;
        dz += kQOne;
      }
      pn = bn;
      pd = bd;
      tprev = tc;
    }
    s.run += (1.f - tprev) * L;
    s.pos |= pn < pd;
  }
  s.P = Q;
  s.qP = q;
}

// Calls f(q, t, v) with the float grid coordinates and the lateral and
// vertical positions (mm) of nodes klo+1 .. khi in order.
// The node loop runs in three phases (entry extension, MLP nodes, exit
// extension) so that no per-node branch selects the node formula.
template <class F>
__device__ __forceinline__ void for_each_node(const Geo& g, const float4* __restrict__ tab, const RecV& r, int klo,
                                              int khi, F&& f) {
  int k = klo + 1;
  // entry extension: straight along the entry slope
  for (; k < 0 && k <= khi; ++k) {
    const float kf = (float)k;
    const float dk = __fmul_rn(kf, g.du);
    const float t = __fmaf_rn(r.st0, dk, r.t0), v = __fmaf_rn(r.sv0, dk, r.v0);
    f(node_grid(g, r, __fmaf_rn(kf, g.du, g.u0), t, v), t, v);
  }
  // MLP nodes between the measurement planes (kf counts k exactly in float)
  const int kmid = min(khi, g.K);
  float kf = (float)k;
  for (; k <= kmid; ++k, kf += 1.f) {
    const float4 c = tab[k];
    const float t = __fmaf_rn(c.w, r.st2, __fmaf_rn(c.z, r.t2, __fmaf_rn(c.y, r.st0, __fmul_rn(c.x, r.t0))));
    const float v = __fmaf_rn(c.w, r.sv2, __fmaf_rn(c.z, r.v2, __fmaf_rn(c.y, r.sv0, __fmul_rn(c.x, r.v0))));
    f(node_grid(g, r, __fmaf_rn(kf, g.du, g.u0), t, v), t, v);
  }
  // exit extension: straight along the exit slope
  for (; k <= khi; ++k) {
    const float dk = __fmul_rn((float)(k - g.K), g.du);
    const float t = __fmaf_rn(r.st2, dk, r.t2), v = __fmaf_rn(r.sv2, dk, r.v2);
    f(node_grid(g, r, __fmaf_rn((float)k, g.du, g.u0), t, v), t, v);
  }
}

// ---- fast walk --------------------------------------------------------------
//
// For a history whose every segment moves less than one voxel on each axis
// (history_fast), each axis crosses at most one face per segment and every
// decision is taken on the float nodes: with the 16-voxel offset a coordinate
// near the grid is an exact multiple of 2^-20, so the distance of a node to a
// face and the length of a segment along an axis are exact floats (Sterbenz),
// and two crossing fractions n1/d1, n2/d2 are ordered exactly by comparing
// n1*d2 with n2*d1 as an FMA two-product (cmp_prod). That is the integer
// walk's cross-multiplication on the same numbers, so the runs are the same.
// Crossing fractions that lie further apart than twice the division's error
// order the same way as the exact ones, so the exact comparison runs only
// for near ties. A voxel change is detected by comparing the floor of each
// coordinate (a round-down addition) with the current voxel's: no rounding to
// Q20 and no conversion in the node loop.

// Sign of a*b - c*d, exactly: p = a*b rounded, a*b = p + fma(a, b, -p) exactly
// (no underflow for the magnitudes here), and rounding is monotonic, so
// distinct rounded products order the exact ones and equal ones leave the
// remainders to decide.
__device__ __forceinline__ int cmp_prod(float a, float b, float c, float d) {
  const float p = __fmul_rn(a, b), q = __fmul_rn(c, d);
  if (p != q) return p < q ? -1 : 1;
  const float ep = __fmaf_rn(a, b, -p), eq = __fmaf_rn(c, d, -q);
  return ep < eq ? -1 : (ep > eq ? 1 : 0);
}

// Every segment of the history moves less than one voxel on every axis: the
// lateral step of a segment is at most |slope| du on the rays and
// sum_i dmax_i |coefficient input i| between the planes (the FP32 table's
// largest node-to-node change per column); 1e-3 voxel of margin covers the
// rounding of the float nodes.
__device__ __forceinline__ bool history_fast(const Geo& g, const RecV& r) {
  if (!(g.dmax[0] < INFINITY)) return false;
  const float bt = fmaxf(fmaxf(fabsf(r.st0), fabsf(r.st2)) * g.du,
                         g.dmax[0] * fabsf(r.t0) + g.dmax[1] * fabsf(r.st0) + g.dmax[2] * fabsf(r.t2) +
                             g.dmax[3] * fabsf(r.st2));
  const float bv = fmaxf(fmaxf(fabsf(r.sv0), fabsf(r.sv2)) * g.du,
                         g.dmax[0] * fabsf(r.v0) + g.dmax[1] * fabsf(r.sv0) + g.dmax[2] * fabsf(r.v2) +
                             g.dmax[3] * fabsf(r.sv2));
  const float ac = fabsf(r.cp), as = fabsf(r.sp);
  const float bx = (g.du * ac + bt * as) * g.ihx;
  const float by = (g.du * as + bt * ac) * g.ihy;
  const float bz = bv * g.ihz;
  return fmaxf(bx, fmaxf(by, bz)) < 0.999f;
}

// fadd_rd(q, kFloorBias) = floor(q) + kFloorBias exactly for |q| < 2^22: the
// sum lies in [2^23, 2^24), where floats are the integers, and rounding down
// is the floor. Its bit pattern minus kFloorBiasBits is floor(q).
constexpr float kFloorBias = 12582912.0f;  // 1.5 * 2^23
constexpr int kFloorBiasBits = 0x4B400000;

// Voxel index along one axis of a biased floor: floor(q) - kQOff.
__device__ __forceinline__ int vox_of(float bq) { return __float_as_int(bq) - kFloorBiasBits - kQOff; }

struct FastState {
  float3 qP;          // previous node, offset grid coordinates
  float bx, by, bz;   // floor of the previous node (the current voxel) + kFloorBias
  int cx, cy, cz;     // current voxel, grid indices
  float run;          // length of the current run so far (mm)
  bool pos;           // the current run has positive exact extent
};

template <class Visit>
__device__ __forceinline__ void emit_fast(const Geo& g, FastState& s, Visit& visit) {
  if (s.pos && (unsigned)s.cx < (unsigned)g.nx && (unsigned)s.cy < (unsigned)g.ny && (unsigned)s.cz < (unsigned)g.nz)
    visit(s.cx + g.nx * (s.cy + g.ny * s.cz), s.run);
  s.run = 0.f;
  s.pos = false;
}

// Crossings of one fast-walk segment ordered exactly (two-product
// comparisons; tied axes step together). rx/ry/rz: the axes that cross, xa..:
// crossing upwards; nd*: exact distance to the crossed face, dd*: exact axis
// length of the segment.
template <class Visit>
__device__ __forceinline__ void seg_fast_exact(const Geo& g, FastState& s, float L, bool rx, bool ry, bool rz, bool xa,
                                               bool ya, bool za, float ndx, float ndy, float ndz, float ddx, float ddy,
                                               float ddz, Visit& visit) {
  // exact pairwise order of the crossings (< 0: the first axis crosses first)
  const int oxy = rx && ry ? cmp_prod(ndx, ddy, ndy, ddx) : 0;
  const int oxz = rx && rz ? cmp_prod(ndx, ddz, ndz, ddx) : 0;
  const int oyz = ry && rz ? cmp_prod(ndy, ddz, ndz, ddy) : 0;
  float tl = 0.f, nl = 0.f, dl = 1.f;
  bool first = true;
  while (rx | ry | rz) {
    // the axes no remaining crossing precedes (tied axes step together)
    const bool mx = rx && !(ry && oxy > 0) && !(rz && oxz > 0);
    const bool my = ry && !(rx && oxy < 0) && !(rz && oyz > 0);
    const bool mz = rz && !(rx && oxz < 0) && !(ry && oyz < 0);
    const float n = mx ? ndx : (my ? ndy : ndz), d = mx ? ddx : (my ? ddy : ddz);
    const float t = __fdividef(n, d);
    s.run += (t - tl) * L;
    s.pos |= !first || n > 0.f;  // later events lie exactly after the previous one
    emit_fast(g, s, visit);
    if (mx) {
      s.cx += xa ? 1 : -1;
      rx = false;
    }
    if (my) {
      s.cy += ya ? 1 : -1;
      ry = false;
    }
    if (mz) {
      s.cz += za ? 1 : -1;
      rz = false;
    }
    tl = t;
    nl = n;
    dl = d;
    first = false;
  }
  s.run += (1.f - tl) * L;
  s.pos |= nl < dl;  // the last crossing lies before the node
}

// Crossing fractions closer than this to each other (or to the segment's
// end) are ordered by the exact comparison: __fdividef is within 2 ulp
// (< 1.2e-7 on [0, 1]), so fractions further apart order as the exact ones.
constexpr float kTieWindow = 4e-7f;

// Advance the fast walk from the previous node to the next one, q (offset
// grid coordinates).
template <class Visit>
__device__ __forceinline__ void seg_fast(const Geo& g, FastState& s, const float3 q, Visit& visit) {
  // Segment length from the grid coordinates, the polyline the crossings are
  // taken on (near the grid the differences are exact). The nodes of a
  // validated record are at least du / sqrt(2) apart in x or y (du >= 2R/2047),
  // far above the float spacing, so L2 > 0.
  const float ddx = fabsf(__fsub_rn(q.x, s.qP.x)), ddy = fabsf(__fsub_rn(q.y, s.qP.y)),
              ddz = fabsf(__fsub_rn(q.z, s.qP.z));
  const float fx = __fmul_rn(ddx, g.hx), fy = __fmul_rn(ddy, g.hy), fz = __fmul_rn(ddz, g.hz);
  const float L2 = __fmaf_rn(fx, fx, __fmaf_rn(fy, fy, __fmul_rn(fz, fz)));
  const float L = L2 * rsqrtf(L2);
  // the voxel of q against the current one (half-open voxels: a face reached
  // moving up is crossed, one reached moving down is not)
  const float bqx = __fadd_rd(q.x, kFloorBias), bqy = __fadd_rd(q.y, kFloorBias), bqz = __fadd_rd(q.z, kFloorBias);
  const bool rx = bqx != s.bx, ry = bqy != s.by, rz = bqz != s.bz;  // crossings to take
  if (!(rx | ry | rz)) {
    s.run += L;  // the segment moves, so the run's extent is positive
    s.pos = true;
    s.qP = q;
    return;
  }
  const bool xa = bqx > s.bx, ya = bqy > s.by, za = bqz > s.bz;  // crossing upwards
  // exact distance to the crossed face and exact axis length of the segment
  const float lx = __fsub_rn(s.bx, kFloorBias), ly = __fsub_rn(s.by, kFloorBias), lz = __fsub_rn(s.bz, kFloorBias);
  const float ndx = xa ? __fsub_rn(__fadd_rn(lx, 1.f), s.qP.x) : __fsub_rn(s.qP.x, lx);
  const float ndy = ya ? __fsub_rn(__fadd_rn(ly, 1.f), s.qP.y) : __fsub_rn(s.qP.y, ly);
  const float ndz = za ? __fsub_rn(__fadd_rn(lz, 1.f), s.qP.z) : __fsub_rn(s.qP.z, lz);
  float tx = rx ? __fdividef(ndx, ddx) : INFINITY;
  float ty = ry ? __fdividef(ndy, ddy) : INFINITY;
  float tz = rz ? __fdividef(ndz, ddz) : INFINITY;
  // near ties, and crossings at the node itself, take the exact order
  const float tmax = fmaxf(rx ? tx : 0.f, fmaxf(ry ? ty : 0.f, rz ? tz : 0.f));
  const bool near = fabsf(tx - ty) < kTieWindow || fabsf(tx - tz) < kTieWindow || fabsf(ty - tz) < kTieWindow ||
                    tmax > 1.f - kTieWindow;
  if (near) {
    seg_fast_exact(g, s, L, rx, ry, rz, xa, ya, za, ndx, ndy, ndz, ddx, ddy, ddz, visit);
  } else {
    // distinct fractions: the float order is the exact order, one axis per event
    float tl = 0.f;
    bool first = true;
    for (;;) {
      const float m = fminf(tx, fminf(ty, tz));
      if (m == INFINITY) break;
      s.run += (m - tl) * L;
      s.pos |= !first || m > 0.f;  // m > 0 exactly when the distance to the face is
      emit_fast(g, s, visit);
      const bool mx = tx == m, my = !mx && ty == m, mz = !mx && !my;
      if (mx) {
        s.cx += xa ? 1 : -1;
        tx = INFINITY;
      }
      if (my) {
        s.cy += ya ? 1 : -1;
        ty = INFINITY;
      }
      if (mz) {
        s.cz += za ? 1 : -1;
        tz = INFINITY;
      }
      tl = m;
      first = false;
    }
    s.run += (1.f - tl) * L;
    s.pos = true;  // the last crossing lies more than the tie window before the node
  }
  // each axis crossed at most one face: the voxel is now the floor of q
  s.bx = bqx;
  s.by = bqy;
  s.bz = bqz;
  s.qP = q;
}

template <class Visit>
__device__ __forceinline__ void walk_fast(const Geo& g, const float4* __restrict__ tab, const RecV& r, int klo,
                                          int khi, Visit& visit) {
  FastState s;
  {
    const float2 tv = node_tv(g, tab, r, klo);
    s.qP = node_grid(g, r, __fmaf_rn((float)klo, g.du, g.u0), tv.x, tv.y);
  }
  s.bx = __fadd_rd(s.qP.x, kFloorBias);
  s.by = __fadd_rd(s.qP.y, kFloorBias);
  s.bz = __fadd_rd(s.qP.z, kFloorBias);
  s.cx = vox_of(s.bx);
  s.cy = vox_of(s.by);
  s.cz = vox_of(s.bz);
  s.run = 0.f;
  s.pos = false;
  for_each_node(g, tab, r, klo, khi, [&](const float3 q, float, float) { seg_fast(g, s, q, visit); });
  emit_fast(g, s, visit);
}

// Walk one proton's polyline, calling visit(j, len) for every run in path
// order (j = voxel index, len = chord in mm).
//
// Per segment P -> Q the voxel index along an axis changes exactly when a face
// is crossed (floor(Q/2^20) != floor(P/2^20), with the half-open convention:
// a face reached exactly counts when moving up, not when moving down). A
// history whose segments all move less than a voxel per axis -- every valid
// record at the default node spacing of half a voxel -- takes the fast walk
// above. Any other takes the integer walk (walk_segment), whose general loop
// re-arms an axis after each face; both give the same runs.
template <class Visit>
__device__ __forceinline__ void walk_proton(const Geo& g, const float4* __restrict__ tab, const RecV& r,
                                            Visit&& visit) {
  int klo, khi;
  node_range(g, r, klo, khi);
  if (history_fast(g, r)) {
    walk_fast(g, tab, r, klo, khi, visit);
    return;
  }
  WalkState s;
  {
    const float2 tv = node_tv(g, tab, r, klo);
    s.qP = node_grid(g, r, __fmaf_rn((float)klo, g.du, g.u0), tv.x, tv.y);
    s.P = quantise3(s.qP);
  }
  s.cx = floor_q(s.P.x);
  s.cy = floor_q(s.P.y);
  s.cz = floor_q(s.P.z);
  s.run = 0.f;
  s.pos = false;
  for_each_node(g, tab, r, klo, khi, [&](const float3 q, float, float) { walk_segment(g, s, q, visit); });
  emit_run(g, s, visit);
}

// Walk with an object hull (same runs contract as walk_proton): the path is
// the entry ray up to node iin, the MLP of the layer between nodes iin and
// iout (table T = fam + family_offset(iout - iin), node k uses T[k - iin],
// from the ray positions at the hull, t_in = fma(st0, iin du, t0) and
// t_out = fma(st2, (iout - K) du, t2), and the measured slopes), then the exit
// ray from node iout:
//   t_k = fma(c4, st2, fma(c3, t_out, fma(c2, st0, c1 * t_in)))   (same for v)
// range = iin | iout << 16 (0 <= iin < iout <= K).
//
// The lanes of a warp enter and leave their hulls at different nodes, so the
// three pieces run in one loop: every node uses the four-term form, with
// (1, k du, 0, 0) on (t0, st0, -, -) for the entry ray and (0, 0, 1,
// (k - K) du) on (-, -, t2, st2) for the exit ray. A product with 0 adds a
// signed zero, which leaves every non-zero value unchanged and the grid
// coordinates q (offset by n/2 > 0) identical, so the nodes are those of the
// separate ray formulas bit for bit.
template <class Visit>
__device__ __forceinline__ void walk_proton_hull(const Geo& g, const float4* __restrict__ fam, int32_t range,
                                                 const RecV& r, Visit&& visit) {
  const int iin = range & 0xffff, iout = range >> 16;
  const float4* __restrict__ T = fam + family_offset(iout - iin) - iin;  // T[k] for iin < k < iout
  const float din = __fmul_rn((float)iin, g.du), dout = __fmul_rn((float)(iout - g.K), g.du);
  const float tin = __fmaf_rn(r.st0, din, r.t0), vin = __fmaf_rn(r.sv0, din, r.v0);
  const float tout = __fmaf_rn(r.st2, dout, r.t2), vout = __fmaf_rn(r.sv2, dout, r.v2);
  int klo, khi;
  node_range(g, r, klo, khi);
  WalkState s;
  {
    // klo <= 0 <= iin: the first node is on the entry ray
    const float dk = __fmul_rn((float)klo, g.du);
    s.qP = node_grid(g, r, __fmaf_rn((float)klo, g.du, g.u0), __fmaf_rn(r.st0, dk, r.t0), __fmaf_rn(r.sv0, dk, r.v0));
    s.P = quantise3(s.qP);
  }
  s.cx = floor_q(s.P.x);
  s.cy = floor_q(s.P.y);
  s.cz = floor_q(s.P.z);
  s.run = 0.f;
  s.pos = false;
  for (int k = klo + 1; k <= khi; ++k) {
    const bool exit = k >= iout, mlp = k > iin && !exit;
    float4 c;
    if (mlp) {
      c = __ldg(T + k);
    } else {
      const float dk = __fmul_rn((float)(exit ? k - g.K : k), g.du);
      c = exit ? make_float4(0.f, 0.f, 1.f, dk) : make_float4(1.f, dk, 0.f, 0.f);
    }
    const float at = mlp ? tin : r.t0, av = mlp ? vin : r.v0;
    const float bt = exit ? r.t2 : tout, bv = exit ? r.v2 : vout;
    const float t = __fmaf_rn(c.w, r.st2, __fmaf_rn(c.z, bt, __fmaf_rn(c.y, r.st0, __fmul_rn(c.x, at))));
    const float v = __fmaf_rn(c.w, r.sv2, __fmaf_rn(c.z, bv, __fmaf_rn(c.y, r.sv0, __fmul_rn(c.x, av))));
    walk_segment(g, s, node_grid(g, r, __fmaf_rn((float)k, g.du, g.u0), t, v), visit);
  }
  emit_run(g, s, visit);
}

// Q20 grid coordinates of node k (0 <= k <= K) on the hull path.
__device__ __forceinline__ int3 node_q_hull(const Geo& g, const float4* __restrict__ fam, int32_t range,
                                            const RecV& r, int k) {
  const int iin = range & 0xffff, iout = range >> 16;
  float t, v;
  if (k <= iin) {
    const float dk = __fmul_rn((float)k, g.du);
    t = __fmaf_rn(r.st0, dk, r.t0);
    v = __fmaf_rn(r.sv0, dk, r.v0);
  } else if (k >= iout) {
    const float dk = __fmul_rn((float)(k - g.K), g.du);
    t = __fmaf_rn(r.st2, dk, r.t2);
    v = __fmaf_rn(r.sv2, dk, r.v2);
  } else {
    const float din = __fmul_rn((float)iin, g.du), dout = __fmul_rn((float)(iout - g.K), g.du);
    const float tin = __fmaf_rn(r.st0, din, r.t0), vin = __fmaf_rn(r.sv0, din, r.v0);
    const float tout = __fmaf_rn(r.st2, dout, r.t2), vout = __fmaf_rn(r.sv2, dout, r.v2);
    const float4 c = __ldg(fam + family_offset(iout - iin) + (k - iin));
    t = __fmaf_rn(c.w, r.st2, __fmaf_rn(c.z, tout, __fmaf_rn(c.y, r.st0, __fmul_rn(c.x, tin))));
    v = __fmaf_rn(c.w, r.sv2, __fmaf_rn(c.z, vout, __fmaf_rn(c.y, r.sv0, __fmul_rn(c.x, vin))));
  }
  return quantise3(node_grid(g, r, __fmaf_rn((float)k, g.du, g.u0), t, v));
}

// Either walk: with a hull when hull.range is set (i = stored index).
template <class Visit>
__device__ __forceinline__ void walk_any(const Geo& g, const float4* __restrict__ tab, const Hull& hull, int64_t i,
                                         const RecV& r, Visit&& visit) {
  if (hull.range) walk_proton_hull(g, hull.fam, __ldg(hull.range + i), r, visit);
  else walk_proton(g, tab, r, visit);
}

}  // namespace pct
