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
//   q = fma(p, 1/h, n/2), clamped to +-1000, Q = rint(q * 2^20) (half even)
// Every product is a separately rounded __fmul_rn and every fused step an
// explicit __fmaf_rn, so the compiler cannot contract or reorder them.
// Between consecutive nodes an integer DDA orders the face crossings by
// exact 32x32->64-bit cross-multiplication; voxels are half-open [i, i+1),
// tied crossings step together, and a run (maximal stretch in one voxel) is
// reported only when its exact extent is positive.
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

__device__ __forceinline__ int32_t quantise(float q) {
  q = fminf(fmaxf(q, -kQClamp), kQClamp);
  return __float2int_rn(__fmul_rn(q, (float)kQOne));
}

// Q20 grid coordinates of node k. `tab` holds (c1, c2, c3, c4) per interior node.
__device__ __forceinline__ int3 node_q(const Geo& g, const float4* __restrict__ tab, const RecV& r, int k) {
  const float u = __fmaf_rn((float)k, g.du, g.u0);
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
  const float ts = __fmul_rn(t, r.sp), tc = __fmul_rn(t, r.cp);
  const float x = __fmaf_rn(u, r.cp, -ts);
  const float y = __fmaf_rn(u, r.sp, tc);
  int3 Q;
  Q.x = quantise(__fmaf_rn(x, g.ihx, g.hnx));
  Q.y = quantise(__fmaf_rn(y, g.ihy, g.hny));
  Q.z = quantise(__fmaf_rn(v, g.ihz, g.hnz));
  return Q;
}

__device__ __forceinline__ int floor_q(int32_t q) { return q >> kQBits; }  // arithmetic shift = floor

// Node range of one proton. Nodes before -E and after K+E lie outside the
// box's circumscribed cylinder; a tighter per-proton range that starts and
// ends outside the box gives the same runs (a straight line meets the convex
// box in one interval), so any conservative range is equivalent.
__device__ __forceinline__ void node_range(const Geo& g, const RecV& r, int& klo, int& khi) {
  klo = -g.E;
  khi = g.K + g.E;
}

// Walk one proton's polyline, calling visit(j, len) for every run in path
// order (j = voxel index, len = chord in mm).
template <class Visit>
__device__ __forceinline__ void walk_proton(const Geo& g, const float4* __restrict__ tab, const RecV& r,
                                            Visit&& visit) {
  int klo, khi;
  node_range(g, r, klo, khi);
  int3 P = node_q(g, tab, r, klo);
  int cx = floor_q(P.x), cy = floor_q(P.y), cz = floor_q(P.z);
  float run = 0.f;
  bool pos = false;
  for (int k = klo + 1; k <= khi; ++k) {
    const int3 Q = node_q(g, tab, r, k);
    const int Dx = Q.x - P.x, Dy = Q.y - P.y, Dz = Q.z - P.z;
    if ((Dx | Dy | Dz) != 0) {
      const uint32_t adx = (uint32_t)abs(Dx), ady = (uint32_t)abs(Dy), adz = (uint32_t)abs(Dz);
      // distance from P to the next face in the direction of travel
      uint32_t dx = Dx > 0 ? (uint32_t)((cx + 1) * kQOne - P.x) : (uint32_t)(P.x - cx * kQOne);
      uint32_t dy = Dy > 0 ? (uint32_t)((cy + 1) * kQOne - P.y) : (uint32_t)(P.y - cy * kQOne);
      uint32_t dz = Dz > 0 ? (uint32_t)((cz + 1) * kQOne - P.z) : (uint32_t)(P.z - cz * kQOne);
      const float fx = (float)Dx * g.lx, fy = (float)Dy * g.ly, fz = (float)Dz * g.lz;
      const float L = sqrtf(fx * fx + fy * fy + fz * fz);
      uint32_t pn = 0, pd = 1;  // previous crossing tau = pn / pd
      float tprev = 0.f;
      for (;;) {
        // a face is crossed within the segment if tau <= 1 moving up (a point
        // on a face belongs to the higher voxel) or tau < 1 moving down
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
        const float tc = __fdiv_rn((float)bn, (float)bd);
        run += (tc - tprev) * L;
        pos |= (uint64_t)bn * pd > (uint64_t)pn * bd;
        if (pos && (unsigned)cx < (unsigned)g.nx && (unsigned)cy < (unsigned)g.ny && (unsigned)cz < (unsigned)g.nz)
          visit(cx + g.nx * (cy + g.ny * cz), run);
        run = 0.f;
        pos = false;
        if (ax && (uint64_t)dx * bd == (uint64_t)bn * adx) {
          cx += Dx > 0 ? 1 : -1;
          dx += kQOne;
        }
        if (ay && (uint64_t)dy * bd == (uint64_t)bn * ady) {
          cy += Dy > 0 ? 1 : -1;
          dy += kQOne;
        }
        if (az && (uint64_t)dz * bd == (uint64_t)bn * adz) {
          cz += Dz > 0 ? 1 : -1;
          dz += kQOne;
        }
        pn = bn;
        pd = bd;
        tprev = tc;
      }
      run += (1.f - tprev) * L;
      pos |= pn < pd;
      P = Q;
    }
  }
  if (pos && (unsigned)cx < (unsigned)g.nx && (unsigned)cy < (unsigned)g.ny && (unsigned)cz < (unsigned)g.nz)
    visit(cx + g.nx * (cy + g.ny * cz), run);
}

}  // namespace pct
