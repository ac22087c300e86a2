// fmb_f32x2.cuh -- packed two-lane FP32 arithmetic (PTX add/mul/fma .f32x2, sm_100+)
// for the per-pair math of two rays at once: one issued instruction performs two
// IEEE round-to-nearest FP32 operations, so the results are bitwise those of the
// scalar fmaf/__fmul_rn/__fadd_rn path while the FP32 issue slots halve.
#pragma once

#include "fmb_internal.cuh"

namespace fmb {

struct f2 {
  unsigned long long v;
};

__device__ __forceinline__ f2 pk(float lo, float hi) {
  f2 r;
  asm("mov.b64 %0, {%1,%2};" : "=l"(r.v) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ f2 dup(float x) { return pk(x, x); }
__device__ __forceinline__ float lo(f2 a) {
  float l, h;
  asm("mov.b64 {%0,%1}, %2;" : "=f"(l), "=f"(h) : "l"(a.v));
  (void)h;
  return l;
}
__device__ __forceinline__ float hi(f2 a) {
  float l, h;
  asm("mov.b64 {%0,%1}, %2;" : "=f"(l), "=f"(h) : "l"(a.v));
  (void)l;
  return h;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
  f2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d.v) : "l"(a.v), "l"(b.v), "l"(c.v));
  return d;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
  f2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
  return d;
}
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
  f2 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
  return d;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
  f2 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
  return d;
}
__device__ __forceinline__ f2 as_f2(unsigned long long x) {
  f2 r;
  r.v = x;
  return r;
}
__device__ __forceinline__ f2 ex2_2(f2 a) { return pk(ex2_approx(lo(a)), ex2_approx(hi(a))); }
__device__ __forceinline__ f2 rcp_2(f2 a) { return pk(rcp_approx(lo(a)), rcp_approx(hi(a))); }
__device__ __forceinline__ f2 rsqrt_2(f2 a) { return pk(rsqrt_approx(lo(a)), rsqrt_approx(hi(a))); }

// A Gaussian record with every coefficient broadcast to both lanes, and the
// negated whitened mean and negated mean-relative-to-camera (so that the packed
// code needs no negations).
struct GaussRec2 {
  f2 L[6], nb[3], nmh[3], nbl[3], l2;
};
__device__ __forceinline__ GaussRec2 broadcast_rec(const GaussRec& g) {
  GaussRec2 r;
#pragma unroll
  for (int i = 0; i < 6; ++i) r.L[i] = dup(g.L[i]);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    r.nb[i] = dup(-g.b[i]);
    r.nmh[i] = dup(-g.mh[i]);
    r.nbl[i] = dup(g.nbl[i]);
  }
  r.l2 = dup(g.l2);
  return r;
}

// Two different Gaussians, one per lane (the backward's thread-owned pair).
__device__ __forceinline__ GaussRec2 pair_rec(const GaussRec& a, const GaussRec& b) {
  GaussRec2 r;
#pragma unroll
  for (int i = 0; i < 6; ++i) r.L[i] = pk(a.L[i], b.L[i]);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    r.nb[i] = pk(-a.b[i], -b.b[i]);
    r.nmh[i] = pk(-a.mh[i], -b.mh[i]);
    r.nbl[i] = pk(a.nbl[i], b.nbl[i]);
  }
  r.l2 = pk(a.l2, b.l2);
  return r;
}

// pair_geom for two lanes (two rays against one Gaussian, or one ray against two
// Gaussians); same operation sequence as
// the scalar pair_geom, so each lane's result is bitwise the scalar one.
// REFINE = false skips the second projection of u onto the complement of a: it
// only removes the component a dt that the rounding dt of t leaves in u, to which
// q = u.u is stationary (it changes q by dt^2 a.a, below fp32 resolution), so
// passes that use u only through q (no normal plane) do not need it; the normal
// g = L u does.
struct PairGeom2 {
  f2 a0, a1, a2, ninv, t, u0, u1, u2, q;  // ninv = -1 / a.a
};
template <bool REFINE = true>
__device__ __forceinline__ PairGeom2 pair_geom2(const GaussRec2& g, f2 v0, f2 v1, f2 v2, f2 vl0, f2 vl1, f2 vl2) {
  PairGeom2 G;
  G.a0 = fma2(g.L[3], v2, fma2(g.L[1], v1, mul2(g.L[0], v0)));
  G.a1 = fma2(g.L[4], v2, mul2(g.L[2], v1));
  G.a2 = mul2(g.L[5], v2);
  const f2 aa = fma2(G.a2, G.a2, fma2(G.a1, G.a1, mul2(G.a0, G.a0)));
  const f2 nab = fma2(G.a2, g.nb[2], fma2(G.a1, g.nb[1], mul2(G.a0, g.nb[0])));  // -a.b
  const f2 inv = rcp_2(aa);
  const f2 ninv = pk(-lo(inv), -hi(inv));
  G.ninv = ninv;
  G.t = mul2(nab, ninv);
  const f2 r0 = fma2(vl0, G.t, fma2(v0, G.t, g.nmh[0]));
  const f2 r1 = fma2(vl1, G.t, fma2(v1, G.t, g.nmh[1]));
  const f2 r2 = fma2(vl2, G.t, fma2(v2, G.t, g.nmh[2]));
  const f2 u0 = fma2(g.L[0], r0, fma2(g.L[1], r1, fma2(g.L[3], r2, g.nbl[0])));
  const f2 u1 = fma2(g.L[2], r1, fma2(g.L[4], r2, g.nbl[1]));
  const f2 u2 = fma2(g.L[5], r2, g.nbl[2]);
  if (REFINE) {
    const f2 nk = mul2(fma2(u2, G.a2, fma2(u1, G.a1, mul2(u0, G.a0))), ninv);
    G.u0 = fma2(nk, G.a0, u0);
    G.u1 = fma2(nk, G.a1, u1);
    G.u2 = fma2(nk, G.a2, u2);
  } else {
    G.u0 = u0;
    G.u1 = u1;
    G.u2 = u2;
  }
  G.q = fma2(G.u2, G.u2, fma2(G.u1, G.u1, mul2(G.u0, G.u0)));
  return G;
}

// pair_geom2 for a given hit depth t (the stored-intermediate backward, which
// reads the forward's t instead of recomputing it): the same operations after t,
// so with the forward's t the results are those pair_geom2 would give; q is not
// formed (the density comes stored too).
template <bool REFINE = true>
__device__ __forceinline__ PairGeom2 pair_geom2_given_t(const GaussRec2& g, f2 t, f2 v0, f2 v1, f2 v2, f2 vl0,
                                                        f2 vl1, f2 vl2) {
  PairGeom2 G;
  G.a0 = fma2(g.L[3], v2, fma2(g.L[1], v1, mul2(g.L[0], v0)));
  G.a1 = fma2(g.L[4], v2, mul2(g.L[2], v1));
  G.a2 = mul2(g.L[5], v2);
  const f2 aa = fma2(G.a2, G.a2, fma2(G.a1, G.a1, mul2(G.a0, G.a0)));
  const f2 inv = rcp_2(aa);
  const f2 ninv = pk(-lo(inv), -hi(inv));
  G.ninv = ninv;
  G.t = t;
  const f2 r0 = fma2(vl0, t, fma2(v0, t, g.nmh[0]));
  const f2 r1 = fma2(vl1, t, fma2(v1, t, g.nmh[1]));
  const f2 r2 = fma2(vl2, t, fma2(v2, t, g.nmh[2]));
  const f2 u0 = fma2(g.L[0], r0, fma2(g.L[1], r1, fma2(g.L[3], r2, g.nbl[0])));
  const f2 u1 = fma2(g.L[2], r1, fma2(g.L[4], r2, g.nbl[1]));
  const f2 u2 = fma2(g.L[5], r2, g.nbl[2]);
  if (REFINE) {
    const f2 nk = mul2(fma2(u2, G.a2, fma2(u1, G.a1, mul2(u0, G.a0))), ninv);
    G.u0 = fma2(nk, G.a0, u0);
    G.u1 = fma2(nk, G.a1, u1);
    G.u2 = fma2(nk, G.a2, u2);
  } else {
    G.u0 = u0;
    G.u1 = u1;
    G.u2 = u2;
  }
  G.q = dup(0.f);
  return G;
}

}  // namespace fmb
