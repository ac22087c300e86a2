// fmb_backward.cu -- adjoint of the forward render (the derivative of Eq. 2, 3, 4,
// 7, 8, 17 and of the Sec. 5 flow) with respect to the means, the precision
// factors L, the weights lambda and the camera poses.
//
// Layout of the work: a CTA takes one view, one tile of rays and one block of
// Gaussians.  Phase 1 turns each ray's upstream gradients into a record in shared
// memory (the per-pixel part of the adjoint: flow, normal renormalisation, alpha),
// every value stored twice so that one 16-byte load yields two broadcast pairs.
// When every view runs as two Gaussian blocks, grid mode launches the two CTAs of
// a ray tile as one 2-CTA cluster: each builds half of the tile's records and
// writes them into both CTAs' shared memory (distributed shared memory), so the
// per-ray work is done once per ray instead of once per block.
// Phase 2 is Gaussian-parallel: each thread owns two Gaussians, one per lane of
// packed FP32x2 arithmetic, recomputes their pair terms for every ray of its
// subgroup from the saved log-normaliser (no per-pair state was stored by the
// forward) and accumulates both Gaussians' gradient sums in registers.  Phase 3 combines the subgroups, converts the sums
// into gradients of mu, L, lambda and of the pose, and writes them once per CTA
// (fp32 atomics, or per-CTA partials that a second kernel adds in a fixed order).
//
// Adjoint in the whitened form (a = L^T v, b = L^T (mu - o), t = a.b/a.a,
// u = t a - b, q = u.u, g = L u, n = g/|g|, what = softmax of e):
//   ebar  = what (Dbar (t - D) + Nbar . n)            (softmax of Eq. 3)
//   dbar  = beta1 ebar + Abar e^{-sum delta} delta     (Eq. 7, Eq. 8)
//   tbar  = Dbar what - (beta2/eta) ebar + (L^T gbar) . a
//   gbar  = what/|g| (Nbar - (n . Nbar) n)             (Eq. 17 normalisation)
//   ubar  = L^T gbar - dbar u
//   y     = ubar - (tbar/a.a) a,  bbar = -y,  abar = t y - (tbar/a.a) u
// and per Gaussian: Lbar = lower(sum gbar u^T + sum v abar^T + (mu - o) bbar^T),
// mubar = L sum bbar, lambdabar = sum dbar / lambda.  The term -dbar u . a of tbar
// is dropped: u . a = 0 exactly at the max-likelihood depth.
#include <algorithm>

#include "fmb_f32x2.cuh"
#include "fmb_internal.cuh"

namespace fmb {

constexpr int kBwdMaxThreads = 160;
#ifndef FMB_BWD_UNROLL
#define FMB_BWD_UNROLL 2  // pair-loop unrolling (independent rays the scheduler can interleave)
#endif
#ifndef FMB_BWD_MIN_BLOCKS
#define FMB_BWD_MIN_BLOCKS 3
#endif
constexpr int kBwdMinBlocks = FMB_BWD_MIN_BLOCKS;  // resident CTAs per SM the register budget targets
constexpr int kBwdUnroll = FMB_BWD_UNROLL;
constexpr int kAccFloats = 38;  // 19 packed accumulators per thread in the reduction
// Colour mode adds three (sum of what x Cbar per channel).
template <bool COLOR>
__host__ __device__ constexpr int acc_floats() {
  return COLOR ? 44 : kAccFloats;
}

// Per-thread gradient sums of the thread's two Gaussians (one per lane).
struct BwdAcc2 {
  f2 nSd;                 // -sum dbar
  f2 Y0, Y1, Y2;          // sum y   (= -sum bbar)
  f2 G00, G10, G11, G20, G21, G22;  // sum gbar u^T (lower)
  f2 M[9];                // sum v abar^T (row-major)
  f2 Cb0, Cb1, Cb2;       // colour mode: sum what Cbar
};

// Shared-memory record of one ray, 7 x 16 bytes, every value duplicated:
//   [v0 v0 v1 v1 | v2 v2 -lse2 -lse2 | Dbar Dbar -KA -KA | -C -C Nb0 Nb0 |
//    Nb1 Nb1 Nb2 Nb2 | vl0 vl0 vl1 vl1 | vl2 vl2 0 0]
// Colour mode: 8 x 16 bytes, the last two [vl2 vl2 Cb0 Cb0 | Cb1 Cb1 Cb2 Cb2].
constexpr int kRayRec2 = 7;
template <bool COLOR>
__host__ __device__ constexpr int ray_rec2() {
  return COLOR ? 8 : kRayRec2;
}

// STORED: the pair's t, log2 weight and density come from the forward (`st`,
// `se`, `sd`) instead of being recomputed.  POSE = false (no pose gradient
// requested): only the lower triangle of sum v abar^T is needed, for Lbar, so it
// is accumulated together with sum gbar u^T into the six G sums and M stays zero.
template <bool NORMALS, bool STORED, bool COLOR = false, bool POSE = true>
__device__ __forceinline__ void bwd_pair2(BwdAcc2& A, const GaussRec2& gr, const ulonglong2* __restrict__ rr, f2 K2,
                                          f2 K3, f2 B1, f2 nB1, f2 nB2E, f2 tiny, f2 st, f2 se, f2 sd,
                                          f2 c0 = f2{}, f2 c1 = f2{}, f2 c2 = f2{}) {
  const ulonglong2 q0 = rr[0], q1 = rr[1], q2 = rr[2], q3 = rr[3], q4 = rr[4], q5 = rr[5], q6 = rr[6];
  // colour mode: Cbar . c_i joins the weight's gradient (Eq. 3 with colours)
  f2 cc = dup(0.f), Cb0 = dup(0.f), Cb1 = dup(0.f), Cb2 = dup(0.f);
  if (COLOR) {
    const ulonglong2 q7 = rr[7];
    Cb0 = as_f2(q6.y);
    Cb1 = as_f2(q7.x);
    Cb2 = as_f2(q7.y);
    cc = fma2(Cb2, c2, fma2(Cb1, c1, mul2(Cb0, c0)));
  }
  const f2 v0 = as_f2(q0.x), v1 = as_f2(q0.y), v2 = as_f2(q1.x), nlse = as_f2(q1.y);
  const f2 Dbar = as_f2(q2.x), nKA = as_f2(q2.y), nC = as_f2(q3.x);
  PairGeom2 G;
  f2 what, delta;
  if (STORED) {
    G = pair_geom2_given_t<NORMALS>(gr, st, v0, v1, v2, as_f2(q5.x), as_f2(q5.y), as_f2(q6.x));
    what = ex2_2(add2(se, nlse));
    delta = sd;
  } else {
    G = pair_geom2<NORMALS>(gr, v0, v1, v2, as_f2(q5.x), as_f2(q5.y), as_f2(q6.x));
    const f2 x = fma2(G.q, K3, gr.l2);  // log2(delta)
    what = ex2_2(fma2(x, B1, fma2(G.t, K2, nlse)));
    delta = ex2_2(x);
  }
  const f2 t = G.t;
  f2 ebar, ub0, ub1, ub2, tbar, gb0, gb1, gb2;
  if (NORMALS) {
    const f2 Nb0 = as_f2(q3.y), Nb1 = as_f2(q4.x), Nb2 = as_f2(q4.y);
    const f2 g0 = mul2(gr.L[0], G.u0);
    const f2 g1 = fma2(gr.L[2], G.u1, mul2(gr.L[1], G.u0));
    const f2 g2 = fma2(gr.L[5], G.u2, fma2(gr.L[4], G.u1, mul2(gr.L[3], G.u0)));
    const f2 gg = add2(fma2(g2, g2, fma2(g1, g1, mul2(g0, g0))), tiny);
    const f2 rs = rsqrt_2(gg);
    const f2 n0 = mul2(g0, rs), n1 = mul2(g1, rs), n2 = mul2(g2, rs);
    const f2 nN = fma2(n2, Nb2, fma2(n1, Nb1, mul2(n0, Nb0)));
    ebar = mul2(what, COLOR ? add2(add2(fma2(Dbar, t, nC), nN), cc) : add2(fma2(Dbar, t, nC), nN));
    const f2 sc = mul2(what, rs);
    const f2 sN = mul2(sc, nN);
    const f2 nsN = pk(-lo(sN), -hi(sN));
    gb0 = fma2(nsN, n0, mul2(sc, Nb0));
    gb1 = fma2(nsN, n1, mul2(sc, Nb1));
    gb2 = fma2(nsN, n2, mul2(sc, Nb2));
    ub0 = fma2(gr.L[3], gb2, fma2(gr.L[1], gb1, mul2(gr.L[0], gb0)));
    ub1 = fma2(gr.L[4], gb2, mul2(gr.L[2], gb1));
    ub2 = mul2(gr.L[5], gb2);
    tbar = fma2(ub2, G.a2, fma2(ub1, G.a1, fma2(ub0, G.a0, fma2(Dbar, what, mul2(nB2E, ebar)))));
  } else {
    ebar = mul2(what, COLOR ? add2(fma2(Dbar, t, nC), cc) : fma2(Dbar, t, nC));
    ub0 = ub1 = ub2 = gb0 = gb1 = gb2 = dup(0.f);
    tbar = fma2(Dbar, what, mul2(nB2E, ebar));
  }
  const f2 ndbar = fma2(nB1, ebar, mul2(nKA, delta));  // -dbar
  ub0 = fma2(ndbar, G.u0, ub0);
  ub1 = fma2(ndbar, G.u1, ub1);
  ub2 = fma2(ndbar, G.u2, ub2);
  const f2 ns2 = mul2(tbar, G.ninv);  // -tbar / a.a
  const f2 y0 = fma2(ns2, G.a0, ub0);
  const f2 y1 = fma2(ns2, G.a1, ub1);
  const f2 y2 = fma2(ns2, G.a2, ub2);
  const f2 ab0 = fma2(t, y0, mul2(ns2, G.u0));
  const f2 ab1 = fma2(t, y1, mul2(ns2, G.u1));
  const f2 ab2 = fma2(t, y2, mul2(ns2, G.u2));
  A.nSd = add2(A.nSd, ndbar);
  A.Y0 = add2(A.Y0, y0);
  A.Y1 = add2(A.Y1, y1);
  A.Y2 = add2(A.Y2, y2);
  if (POSE) {
    if (NORMALS) {
      A.G00 = fma2(gb0, G.u0, A.G00);
      A.G10 = fma2(gb1, G.u0, A.G10);
      A.G11 = fma2(gb1, G.u1, A.G11);
      A.G20 = fma2(gb2, G.u0, A.G20);
      A.G21 = fma2(gb2, G.u1, A.G21);
      A.G22 = fma2(gb2, G.u2, A.G22);
    }
    A.M[0] = fma2(v0, ab0, A.M[0]);
    A.M[1] = fma2(v0, ab1, A.M[1]);
    A.M[2] = fma2(v0, ab2, A.M[2]);
    A.M[3] = fma2(v1, ab0, A.M[3]);
    A.M[4] = fma2(v1, ab1, A.M[4]);
    A.M[5] = fma2(v1, ab2, A.M[5]);
    A.M[6] = fma2(v2, ab0, A.M[6]);
    A.M[7] = fma2(v2, ab1, A.M[7]);
    A.M[8] = fma2(v2, ab2, A.M[8]);
  } else {
    A.G00 = fma2(v0, ab0, NORMALS ? fma2(gb0, G.u0, A.G00) : A.G00);
    A.G10 = fma2(v1, ab0, NORMALS ? fma2(gb1, G.u0, A.G10) : A.G10);
    A.G11 = fma2(v1, ab1, NORMALS ? fma2(gb1, G.u1, A.G11) : A.G11);
    A.G20 = fma2(v2, ab0, NORMALS ? fma2(gb2, G.u0, A.G20) : A.G20);
    A.G21 = fma2(v2, ab1, NORMALS ? fma2(gb2, G.u1, A.G21) : A.G21);
    A.G22 = fma2(v2, ab2, NORMALS ? fma2(gb2, G.u2, A.G22) : A.G22);
  }
  if (COLOR) {
    A.Cb0 = fma2(what, Cb0, A.Cb0);
    A.Cb1 = fma2(what, Cb1, A.Cb1);
    A.Cb2 = fma2(what, Cb2, A.Cb2);
  }
}

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// CL = 2: launched as clusters of two CTAs, the two Gaussian blocks of one ray tile
// (grid mode, every view of the batch in two blocks); CL = 1: no cluster.
template <bool NORMALS, int NFLOW, bool STORED, bool COLOR = false, bool POSE = true, int CL = 1, class B = Batch>
__global__ void __launch_bounds__(kBwdMaxThreads, kBwdMinBlocks)
    backward_kernel(const __grid_constant__ B batch, Scene s, Consts k, const float4* __restrict__ records,
                    BwdIn in, BwdOut out, int ray_tile, int* counter) {
  pdl_enter();
  extern __shared__ float4 bsm[];
  constexpr int NPV = 12 * (1 + NFLOW);  // pose values reduced per CTA
  __shared__ float pose_ray[kBwdMaxThreads / 32][NPV];  // per-warp sums of the per-ray pose terms
  __shared__ float pose_gau[kBwdMaxThreads / 32][12];   // per-warp sums of the per-Gaussian pose terms
  __shared__ int s_item;

  for (int round = 0;; ++round) {
  const int item = next_item(counter, round, &s_item);
  if (item < 0 || item >= batch.n_items) break;
  int local;
  const int vi = find_item(batch, item, local);
  const DevView& V = batch.v[vi];
  const int tile = local / V.n_gblocks;
  const int gb = local - tile * V.n_gblocks;
  const int P = V.P;
  const int rt = V.rt > 0 ? V.rt : ray_tile;  // the view's tiles are balanced: rt <= ray_tile
  const int pix0 = tile * rt;
  const int nr = min(rt, P - pix0);
  const int tid = threadIdx.x;
  const int T = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5;
  const long long off = V.pix_off;
  const bool want_pose = out.gposes != nullptr;
  // In a cluster (CL = 2) each CTA builds the records of its half of the tile's
  // rays and writes them to both CTAs (its own shared memory and, through
  // distributed shared memory, its peer's), so a ray's record is built once, not
  // once per Gaussian block.
  const int crank = CL == 2 ? static_cast<int>(cluster_ctarank()) : 0;
  const int r_lo = CL == 2 ? (nr * crank) / 2 : 0;
  const int r_hi = CL == 2 ? (nr * (crank + 1)) / 2 : nr;
  // per-ray pose terms: once per ray (by the CTA that builds its record)
  const bool ray_pose = want_pose && (CL == 2 || gb == 0);

  // ---------------- phase 1: per-ray records (and the per-ray pose terms)
  {
    float R[9], tp[3];
    load_pose(s.poses, V.pose, R, tp);
    const float o0 = -fmaf(R[6], tp[2], fmaf(R[3], tp[1], R[0] * tp[0]));
    const float o1 = -fmaf(R[7], tp[2], fmaf(R[4], tp[1], R[1] * tp[0]));
    const float o2 = -fmaf(R[8], tp[2], fmaf(R[5], tp[1], R[2] * tp[0]));
    float pose_acc[NPV];
#pragma unroll
    for (int i = 0; i < NPV; ++i) pose_acc[i] = 0.f;
    float Rj[NFLOW > 0 ? NFLOW : 1][9], tj[NFLOW > 0 ? NFLOW : 1][3];
    bool has_t[NFLOW > 0 ? NFLOW : 1];
#pragma unroll
    for (int j = 0; j < NFLOW; ++j) {
      const int tg = j == 0 ? V.tgt0 : V.tgt1;
      has_t[j] = tg >= 0 && in.g_flow != nullptr;
      if (has_t[j]) load_pose(s.poses, tg, Rj[j], tj[j]);
    }
    for (int r = r_lo + tid; r < r_hi; r += T) {
      const int p = pix0 + r;
      float vc[3], v[3], vl[3], pxy[2];
      pixel_ray_dd(V, R, ray_pixel(V, p), vc, v, vl, pxy);
      const float D = in.depth[off + p];
      const float* sv = in.saved + 3 * off;
      const float lse2 = sv[p];
      const float Sd = sv[P + p];
      const float gD = in.g_depth ? in.g_depth[off + p] : 0.f;
      const float gA = in.g_alpha ? in.g_alpha[off + p] : 0.f;
      float pb0 = 0.f, pb1 = 0.f, pb2 = 0.f;
      if (NFLOW > 0) {
        const float p0 = fmaf(v[0], D, o0), p1 = fmaf(v[1], D, o1), p2 = fmaf(v[2], D, o2);
        const float* gf = in.g_flow + 2 * NFLOW * off;
#pragma unroll
        for (int j = 0; j < NFLOW; ++j) {
          if (!has_t[j]) continue;
          const float X0 = fmaf(Rj[j][2], p2, fmaf(Rj[j][1], p1, fmaf(Rj[j][0], p0, tj[j][0])));
          const float X1 = fmaf(Rj[j][5], p2, fmaf(Rj[j][4], p1, fmaf(Rj[j][3], p0, tj[j][1])));
          const float X2 = fmaf(Rj[j][8], p2, fmaf(Rj[j][7], p1, fmaf(Rj[j][6], p0, tj[j][2])));
          const float iz = 1.0f / X2;
          const float gu = gf[(2 * j) * P + p], gv = gf[(2 * j + 1) * P + p];
          const float Xb0 = gu * V.fx * iz;
          const float Xb1 = gv * V.fy * iz;
          const float Xb2 = -(Xb0 * X0 + Xb1 * X1) * iz;
          pb0 += fmaf(Rj[j][6], Xb2, fmaf(Rj[j][3], Xb1, Rj[j][0] * Xb0));
          pb1 += fmaf(Rj[j][7], Xb2, fmaf(Rj[j][4], Xb1, Rj[j][1] * Xb0));
          pb2 += fmaf(Rj[j][8], Xb2, fmaf(Rj[j][5], Xb1, Rj[j][2] * Xb0));
          if (ray_pose) {
            float* pa = pose_acc + 12 * (1 + j);
            const float Xb[3] = {Xb0, Xb1, Xb2};
            const float pp[3] = {p0, p1, p2};
#pragma unroll
            for (int a = 0; a < 3; ++a) {
#pragma unroll
              for (int c = 0; c < 3; ++c) pa[3 * a + c] = fmaf(Xb[a], pp[c], pa[3 * a + c]);
              pa[9 + a] += Xb[a];
            }
          }
        }
      }
      const float Dbar = fmaf(v[2], pb2, fmaf(v[1], pb1, fmaf(v[0], pb0, gD)));
      if (ray_pose && NFLOW > 0) {
        // p = o + v D with o = -R^T t, v = R^T vc:  Rbar += (D vc - t) pbar^T, tbar -= R pbar
        const float w[3] = {fmaf(D, vc[0], -tp[0]), fmaf(D, vc[1], -tp[1]), fmaf(D, vc[2], -tp[2])};
        const float pb[3] = {pb0, pb1, pb2};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
#pragma unroll
          for (int c = 0; c < 3; ++c) pose_acc[3 * a + c] = fmaf(w[a], pb[c], pose_acc[3 * a + c]);
          pose_acc[9 + a] -= fmaf(R[3 * a + 2], pb2, fmaf(R[3 * a + 1], pb1, R[3 * a] * pb0));
        }
      }
      float Nb0 = 0.f, Nb1 = 0.f, Nb2 = 0.f;
      if (NORMALS && in.g_normal != nullptr) {
        const float* nr3 = in.normal + 3 * off;
        const float* gn3 = in.g_normal + 3 * off;
        const float nc[3] = {nr3[p], nr3[P + p], nr3[2 * P + p]};
        const float gn[3] = {gn3[p], gn3[P + p], gn3[2 * P + p]};
        const float Nn = sv[2 * P + p];
        // world-frame blended normal and its upstream gradient (R^T applied)
        float nf[3], nfb[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          nf[c] = fmaf(R[6 + c], nc[2], fmaf(R[3 + c], nc[1], R[c] * nc[0]));
          nfb[c] = fmaf(R[6 + c], gn[2], fmaf(R[3 + c], gn[1], R[c] * gn[0]));
        }
        if (ray_pose) {
#pragma unroll
          for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int c = 0; c < 3; ++c) pose_acc[3 * a + c] = fmaf(gn[a], nf[c], pose_acc[3 * a + c]);
        }
        if (Nn > 0.f) {
          const float iN = 1.0f / Nn;
          const float sdot = fmaf(nf[2], nfb[2], fmaf(nf[1], nfb[1], nf[0] * nfb[0]));
          Nb0 = fmaf(-sdot, nf[0], nfb[0]) * iN;
          Nb1 = fmaf(-sdot, nf[1], nfb[1]) * iN;
          Nb2 = fmaf(-sdot, nf[2], nfb[2]) * iN;
        }
      }
      // Nbar is orthogonal to N, so the softmax centring term is Dbar * D alone (plus
      // Cbar . C, the blended colour's, in colour mode).
      float C = Dbar * D;
      float Cb[3] = {0.f, 0.f, 0.f};
      if (COLOR && in.g_color != nullptr) {
        const float* gc3 = in.g_color + 3 * off;
        const float* cp3 = in.color + 3 * off;
#pragma unroll
        for (int k3 = 0; k3 < 3; ++k3) {
          Cb[k3] = gc3[k3 * P + p];
          C = fmaf(Cb[k3], cp3[k3 * P + p], C);
        }
      }
      const float KA = gA * expf(-Sd);
      float4* rr = bsm + ray_rec2<COLOR>() * r;
      const float4 rec[8] = {make_float4(v[0], v[0], v[1], v[1]),     make_float4(v[2], v[2], -lse2, -lse2),
                             make_float4(Dbar, Dbar, -KA, -KA),       make_float4(-C, -C, Nb0, Nb0),
                             make_float4(Nb1, Nb1, Nb2, Nb2),         make_float4(vl[0], vl[0], vl[1], vl[1]),
                             make_float4(vl[2], vl[2], Cb[0], Cb[0]), make_float4(Cb[1], Cb[1], Cb[2], Cb[2])};
#pragma unroll
      for (int i = 0; i < ray_rec2<COLOR>(); ++i) {
        rr[i] = rec[i];
        if (CL == 2) st_cluster_f4(rr + i, crank ^ 1, rec[i]);
      }
    }
    // Reduce the per-ray pose terms now, so that they hold no registers in the loop.
    if (want_pose) {
#pragma unroll
      for (int i = 0; i < NPV; ++i) {
        const float x = warp_sum(pose_acc[i]);
        if (lane == 0) pose_ray[warp][i] = x;
      }
    }
  }
  // the records (the cluster's, through distributed shared memory) are complete
  if (CL == 2)
    cluster_sync();
  else
    __syncthreads();

  // ---------------- phase 2: Gaussian-parallel pair loop (two Gaussians per thread)
  const int GB = V.GB, S = V.S;
  const int GB2 = (GB + 1) / 2;  // threads per ray subgroup
  const int gl2 = tid % GB2;
  const int sg = tid / GB2;
  const int g0 = gb * GB + 2 * gl2;        // lane 0 Gaussian
  const bool has1 = 2 * gl2 + 1 < GB && g0 + 1 < V.K;  // lane 1 holds a real Gaussian
  const bool active = (sg < S) && (g0 < V.K);
  BwdAcc2 A;
  A.nSd = A.Y0 = A.Y1 = A.Y2 = dup(0.f);
  A.G00 = A.G10 = A.G11 = A.G20 = A.G21 = A.G22 = dup(0.f);
#pragma unroll
  for (int i = 0; i < 9; ++i) A.M[i] = dup(0.f);
  A.Cb0 = A.Cb1 = A.Cb2 = dup(0.f);
  GaussRec ga{}, gbr{};
  if (active) {
    const float4* rec = records + kRecFloat4 * (V.rec_off + g0);
    ga = unpack_rec(rec[0], rec[1], rec[2], rec[3]);
    if (has1) {
      const float4* rec1 = rec + kRecFloat4;
      gbr = unpack_rec(rec1[0], rec1[1], rec1[2], rec1[3]);
    } else {
      gbr = ga;  // a copy keeps the unused lane finite; its sums are never written
    }
    const GaussRec2 gr = pair_rec(ga, gbr);
    const f2 K2v = dup(k.K2), K3v = dup(k.K3), B1v = dup(k.beta1), nB1v = dup(-k.beta1), nB2E = dup(-k.b2e);
    const f2 tiny = dup(1e-30f);
    const ulonglong2* rays = reinterpret_cast<const ulonglong2*>(bsm);
    if (STORED) {
      // the two Gaussians' stored values are adjacent in the row of pixel p (g0 is even)
      const unsigned long long* pt =
          reinterpret_cast<const unsigned long long*>(in.pairs + V.pair_off + static_cast<long long>(pix0) * V.Kp + g0);
      const long long st2 = in.pair_stride / 2, row2 = V.Kp / 2;
#pragma unroll kBwdUnroll
      for (int r = sg; r < nr; r += S) {
        const unsigned long long* q = pt + static_cast<long long>(r) * row2;
        bwd_pair2<NORMALS, true>(A, gr, rays + kRayRec2 * r, K2v, K3v, B1v, nB1v, nB2E, tiny, as_f2(__ldg(q)),
                                 as_f2(__ldg(q + st2)), as_f2(__ldg(q + 2 * st2)));
      }
    } else if (COLOR) {
      // the two Gaussians' colours, one per lane
      const float4 ca = __ldg(s.crec + V.rec_off + g0), cb = has1 ? __ldg(s.crec + V.rec_off + g0 + 1) : ca;
      const f2 c0 = pk(ca.x, cb.x), c1 = pk(ca.y, cb.y), c2 = pk(ca.z, cb.z);
      const f2 z = dup(0.f);
#pragma unroll kBwdUnroll
      for (int r = sg; r < nr; r += S)
        bwd_pair2<NORMALS, false, true>(A, gr, rays + ray_rec2<true>() * r, K2v, K3v, B1v, nB1v, nB2E, tiny, z, z, z,
                                        c0, c1, c2);
    } else {
      const f2 z = dup(0.f);
#pragma unroll kBwdUnroll
      for (int r = sg; r < nr; r += S)
        bwd_pair2<NORMALS, false, false, POSE>(A, gr, rays + kRayRec2 * r, K2v, K3v, B1v, nB1v, nB2E, tiny, z, z, z);
    }
  }
  __syncthreads();  // ray records are dead; the shared memory is reused below

  // ---------------- phase 3: combine ray subgroups, finalise per Gaussian
  constexpr int NV = COLOR ? 22 : 19;  // sums per Gaussian
  constexpr int ACC = acc_floats<COLOR>();
  constexpr int NC = COLOR ? 13 : 10;  // gradient values per Gaussian in a partial slot
  float* red = reinterpret_cast<float*>(bsm);
  if (sg < S) {
    float* d = red + ACC * tid;
    const f2 v[22] = {A.nSd, A.Y0, A.Y1, A.Y2, A.G00, A.G10, A.G11, A.G20, A.G21, A.G22, A.M[0],
                      A.M[1], A.M[2], A.M[3], A.M[4], A.M[5], A.M[6], A.M[7], A.M[8], A.Cb0, A.Cb1, A.Cb2};
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      d[i] = lo(v[i]);
      d[NV + i] = hi(v[i]);
    }
  }
  __syncthreads();
  float* slot = nullptr;
  if (out.partials) {
    slot = out.partials + V.part_off + static_cast<long long>(tile * V.n_gblocks + gb) * V.slot_floats;
  }
  float pose_g[12];
#pragma unroll
  for (int i = 0; i < 12; ++i) pose_g[i] = 0.f;
  if (sg == 0 && gl2 < GB2) {
    float R[9], tp[3];
    const bool want_R = want_pose;
    if (want_R) load_pose(s.poses, V.pose, R, tp);
#pragma unroll
    for (int lane2 = 0; lane2 < 2; ++lane2) {
      const int gi = 2 * gl2 + lane2;  // Gaussian index within the block
      if (gi >= GB) break;
      const int g = gb * GB + gi;
      float acc[NV];
#pragma unroll
      for (int i = 0; i < NV; ++i) acc[i] = 0.f;
      for (int s2 = 0; s2 < S; ++s2) {
        const float* d = red + ACC * (s2 * GB2 + gl2) + NV * lane2;
#pragma unroll
        for (int i = 0; i < NV; ++i) acc[i] += d[i];
      }
      float gm[3] = {0, 0, 0}, gL[6] = {0, 0, 0, 0, 0, 0}, glam = 0.f;
      if (g < V.K && active) {
        const GaussRec& gr1 = lane2 == 0 ? ga : gbr;
        const long long gg = V.gauss_off + g;
        const float L00 = gr1.L[0], L10 = gr1.L[1], L11 = gr1.L[2], L20 = gr1.L[3], L21 = gr1.L[4], L22 = gr1.L[5];
        const float Bb0 = -acc[1], Bb1 = -acc[2], Bb2 = -acc[3];
        // mubar = L bbar_sum
        gm[0] = L00 * Bb0;
        gm[1] = fmaf(L11, Bb1, L10 * Bb0);
        gm[2] = fmaf(L22, Bb2, fmaf(L21, Bb1, L20 * Bb0));
        const float m0 = gr1.mh[0], m1 = gr1.mh[1], m2 = gr1.mh[2];
        const float* M = acc + 10;
        gL[0] = acc[4] + M[0] + m0 * Bb0;  // (0,0)
        gL[1] = acc[5] + M[3] + m1 * Bb0;  // (1,0)
        gL[2] = acc[6] + M[4] + m1 * Bb1;  // (1,1)
        gL[3] = acc[7] + M[6] + m2 * Bb0;  // (2,0)
        gL[4] = acc[8] + M[7] + m2 * Bb1;  // (2,1)
        gL[5] = acc[9] + M[8] + m2 * Bb2;  // (2,2)
        glam = -acc[0] / s.weights[gg];
        if (want_R) {
          // Rbar += R (M L^T) + t mubar^T ; tbar += R mubar
          float ML[9];
          const float Lf[9] = {L00, 0.f, 0.f, L10, L11, 0.f, L20, L21, L22};
#pragma unroll
          for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int c = 0; c < 3; ++c)
              ML[3 * a + c] =
                  fmaf(M[3 * a + 2], Lf[3 * c + 2], fmaf(M[3 * a + 1], Lf[3 * c + 1], M[3 * a] * Lf[3 * c]));
#pragma unroll
          for (int a = 0; a < 3; ++a) {
#pragma unroll
            for (int c = 0; c < 3; ++c)
              pose_g[3 * a + c] += fmaf(R[3 * a + 2], ML[6 + c], fmaf(R[3 * a + 1], ML[3 + c], R[3 * a] * ML[c])) +
                                   tp[a] * gm[c];
            pose_g[9 + a] += fmaf(R[3 * a + 2], gm[2], fmaf(R[3 * a + 1], gm[1], R[3 * a] * gm[0]));
          }
        }
        if (slot == nullptr) {
          atomicAdd(out.gmeans + 3 * gg + 0, gm[0]);
          atomicAdd(out.gmeans + 3 * gg + 1, gm[1]);
          atomicAdd(out.gmeans + 3 * gg + 2, gm[2]);
#pragma unroll
          for (int i = 0; i < 6; ++i) atomicAdd(out.gchol + 6 * gg + i, gL[i]);
          atomicAdd(out.gweights + gg, glam);
          if (COLOR) {
#pragma unroll
            for (int k3 = 0; k3 < 3; ++k3) atomicAdd(out.gcolors + 3 * gg + k3, acc[19 + k3]);
          }
        }
      }
      if (slot != nullptr) {
        float* d = slot + NC * gi;
        d[0] = gm[0]; d[1] = gm[1]; d[2] = gm[2];
#pragma unroll
        for (int i = 0; i < 6; ++i) d[3 + i] = gL[i];
        d[9] = glam;
        if (COLOR) {
#pragma unroll
          for (int k3 = 0; k3 < 3; ++k3) d[10 + k3] = (g < V.K && active) ? acc[19 + k3] : 0.f;
        }
      }
    }
  }

  // ---------------- phase 4: pose gradient of this CTA
  if (want_pose) {
#pragma unroll
    for (int i = 0; i < 12; ++i) {
      const float x = warp_sum(pose_g[i]);
      if (lane == 0) pose_gau[warp][i] = x;
    }
    __syncthreads();
    if (tid < NPV) {
      float x = 0.f;
      const int nw = (T + 31) / 32;
      for (int w = 0; w < nw; ++w) x += pose_ray[w][tid] + (tid < 12 ? pose_gau[w][tid] : 0.f);
      if (slot != nullptr) {
        slot[NC * GB + tid] = x;
      } else {
        const int j = tid / 12 - 1;
        const int pidx = j < 0 ? V.pose : (j == 0 ? V.tgt0 : V.tgt1);
        if (pidx >= 0) atomicAdd(out.gposes + 12 * static_cast<long long>(pidx) + tid % 12, x);
      }
    }
  }
  }  // item loop
}

static int bwd_smem_bytes(int ray_tile, int threads, bool color = false) {
  return std::max(ray_tile * (color ? ray_rec2<true>() : kRayRec2) * static_cast<int>(sizeof(float4)),
                  threads * (color ? acc_floats<true>() : kAccFloats) * static_cast<int>(sizeof(float)));
}

template <bool NORMALS, int NFLOW, bool STORED = false, bool COLOR = false, bool POSE = true, int CL = 1,
          class B = Batch>
static cudaError_t prepare_bwd_t(int smem) {
  // Dynamic plus static shared memory above the 48 KB default needs the opt-in.
  if (smem + static_cast<int>(sizeof(float) * (kBwdMaxThreads / 32) * 48) > 48 * 1024)
    return cudaFuncSetAttribute(backward_kernel<NORMALS, NFLOW, STORED, COLOR, POSE, CL, B>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  return cudaSuccess;
}

template <bool NORMALS, int NFLOW>
static int bwd_ctas_per_sm_t(int ray_tile, int threads) {
  const int smem = bwd_smem_bytes(ray_tile, threads);
  if (prepare_bwd_t<NORMALS, NFLOW>(smem) != cudaSuccess) return 1;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, backward_kernel<NORMALS, NFLOW, false>, threads, smem) !=
      cudaSuccess)
    return 1;
  return n > 0 ? n : 1;
}

// Cluster size of a grid-mode backward launch: 2 when every view of the batch runs
// as two Gaussian blocks (then each tile's two items are consecutive and 2-aligned,
// one cluster), else 1 (no cluster).
template <class B>
static int bwd_cluster_size(const B& b) {
  int C = 0;
  for (int i = 0; i < b.n_views; ++i) {
    const DevView& v = b.v[i];
    if (v.n_tiles <= 0) continue;
    if (C == 0) C = v.n_gblocks;
    if (v.n_gblocks != C) return 1;
  }
  if (C != 2 || b.n_items % C != 0) return 1;
  for (int j = 0; j < b.n_views; ++j)
    if (b.order_begin[j] % C != 0) return 1;
  return C;
}

template <bool NORMALS, int NFLOW, bool STORED, bool COLOR = false, bool POSE = true, class B>
static cudaError_t launch_bwd_s(const B& b, const Scene& s, const Consts& c, const float4* records,
                                int ray_tile, int threads, const BwdIn& in, const BwdOut& out, int* counter,
                                cudaStream_t st) {
  const int smem = bwd_smem_bytes(ray_tile, threads, COLOR);
  cudaError_t e = prepare_bwd_t<NORMALS, NFLOW, STORED, COLOR, POSE, 1, B>(smem);
  if (e != cudaSuccess) return e;
  int grid = b.n_items;
  if (counter) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    grid = std::min(b.n_items, std::max(1, sms) * bwd_ctas_per_sm_t<NORMALS, NFLOW>(ray_tile, threads));
  }
  if constexpr (!STORED && !COLOR) {
    if (counter == nullptr && bwd_cluster_size(b) == 2) {
      e = prepare_bwd_t<NORMALS, NFLOW, STORED, COLOR, POSE, 2, B>(smem);
      if (e != cudaSuccess) return e;
      return launch_kernel(backward_kernel<NORMALS, NFLOW, STORED, COLOR, POSE, 2, B>, dim3(grid), dim3(threads), smem,
                           st, 2, b, s, c, records, in, out, ray_tile, counter);
    }
  }
  return launch_kernel(backward_kernel<NORMALS, NFLOW, STORED, COLOR, POSE, 1, B>, dim3(grid), dim3(threads), smem, st,
                       1, b, s, c, records, in, out, ray_tile, counter);
}

template <bool NORMALS, int NFLOW, class B>
static cudaError_t launch_bwd_t(const B& b, const Scene& s, const Consts& c, const float4* records,
                                int ray_tile, int threads, const BwdIn& in, const BwdOut& out, int* counter,
                                cudaStream_t st) {
  if (in.pairs != nullptr)
    return launch_bwd_s<NORMALS, NFLOW, true>(b, s, c, records, ray_tile, threads, in, out, counter, st);
  if (out.gcolors != nullptr)
    return launch_bwd_s<NORMALS, NFLOW, false, true>(b, s, c, records, ray_tile, threads, in, out, counter, st);
  if (out.gposes == nullptr)
    return launch_bwd_s<NORMALS, NFLOW, false, false, false>(b, s, c, records, ray_tile, threads, in, out, counter,
                                                              st);
  return launch_bwd_s<NORMALS, NFLOW, false>(b, s, c, records, ray_tile, threads, in, out, counter, st);
}

template <class B>
static cudaError_t launch_backward_t(const B& b, const Scene& s, const Consts& c, const float4* records,
                                     bool normals, int n_flow, int ray_tile, int threads, const BwdIn& in,
                                     const BwdOut& out, int* counter, cudaStream_t st) {
  if (normals) {
    if (n_flow == 0) return launch_bwd_t<true, 0>(b, s, c, records, ray_tile, threads, in, out, counter, st);
    if (n_flow == 1) return launch_bwd_t<true, 1>(b, s, c, records, ray_tile, threads, in, out, counter, st);
    return launch_bwd_t<true, 2>(b, s, c, records, ray_tile, threads, in, out, counter, st);
  }
  if (n_flow == 0) return launch_bwd_t<false, 0>(b, s, c, records, ray_tile, threads, in, out, counter, st);
  if (n_flow == 1) return launch_bwd_t<false, 1>(b, s, c, records, ray_tile, threads, in, out, counter, st);
  return launch_bwd_t<false, 2>(b, s, c, records, ray_tile, threads, in, out, counter, st);
}
cudaError_t launch_backward(const Batch& b, const Scene& s, const Consts& c, const float4* records, bool normals,
                            int n_flow, int ray_tile, int threads, const BwdIn& in, const BwdOut& out,
                            int* counter, cudaStream_t st) {
  return launch_backward_t(b, s, c, records, normals, n_flow, ray_tile, threads, in, out, counter, st);
}
cudaError_t launch_backward(const BigBatch& b, const Scene& s, const Consts& c, const float4* records, bool normals,
                            int n_flow, int ray_tile, int threads, const BwdIn& in, const BwdOut& out,
                            int* counter, cudaStream_t st) {
  return launch_backward_t(b, s, c, records, normals, n_flow, ray_tile, threads, in, out, counter, st);
}

int backward_ctas_per_sm(bool normals, int n_flow, int ray_tile, int threads) {
  (void)normals;
  (void)n_flow;
  return bwd_ctas_per_sm_t<true, 1>(ray_tile, threads);
}

// ------------------------------------------------- zeroing of the outputs
// One launch clears the status word and every gradient output before the
// backward kernels accumulate into them.
__global__ void zero_kernel(ZeroJob job) {
  pdl_enter();
  const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
  long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  for (int b = 0; b < ZeroJob::kMax; ++b) {
    if (job.ptr[b] == nullptr) continue;
    for (long long j = i; j < job.n[b]; j += stride) job.ptr[b][j] = 0.f;
  }
}

cudaError_t launch_zero(const ZeroJob& job, cudaStream_t st) {
  return launch_kernel(zero_kernel, dim3(2 * 152), dim3(256), 0, st, 1, job);
}

// ------------------------------------------- deterministic second stage
// One warp per output value: lane l adds slots l, l+32, l+64, ... in order, then a
// fixed butterfly combines the lanes, so the result does not depend on timing.
__device__ __forceinline__ float warp_sum_fixed(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Gaussian gradients: warp w handles (Gaussian g, component comp), w = g * nc + comp
// (nc = 10, or 13 with colours: means 3, chol 6, weight 1, colour 3).
template <class B>
__global__ void reduce_gauss_kernel(const __grid_constant__ B batch, const float* __restrict__ partials,
                                    float* gmeans, float* gchol, float* gweights, float* gcolors, long long n_gauss,
                                    int nc) {
  pdl_enter();
  const long long w = (blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= n_gauss * nc) return;  // whole warps exit together
  const long long g = w / nc;
  const int comp = static_cast<int>(w - g * nc);
  float acc = 0.f;
  bool hit = false;
  for (int v = 0; v < batch.n_views; ++v) {
    const DevView& V = batch.v[v];
    if (g < V.gauss_off || g >= V.gauss_off + V.K) continue;
    hit = true;
    const int gi = static_cast<int>(g - V.gauss_off);
    const int gbk = gi / V.GB, gl = gi - gbk * V.GB;
    for (int t = lane; t < V.n_tiles; t += 32)
      acc += partials[V.part_off + static_cast<long long>(t * V.n_gblocks + gbk) * V.slot_floats + nc * gl + comp];
  }
  acc = warp_sum_fixed(acc);
  if (!hit || lane != 0) return;
  if (comp < 3)
    gmeans[3 * g + comp] += acc;
  else if (comp < 9)
    gchol[6 * g + comp - 3] += acc;
  else if (comp == 9)
    gweights[g] += acc;
  else
    gcolors[3 * g + comp - 10] += acc;
}

// Pose gradients: warp w handles (pose p, component comp), w = p * 12 + comp.
template <class B>
__global__ void reduce_pose_kernel(const __grid_constant__ B batch, const float* __restrict__ partials,
                                   float* gposes, int n_poses, int n_flow, int nc) {
  pdl_enter();
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= n_poses * 12) return;
  const int p = w / 12, comp = w % 12;
  float acc = 0.f;
  for (int v = 0; v < batch.n_views; ++v) {
    const DevView& V = batch.v[v];
    for (int j = -1; j < n_flow; ++j) {
      const int pidx = j < 0 ? V.pose : (j == 0 ? V.tgt0 : V.tgt1);
      if (pidx != p) continue;
      const int part = 12 * (j + 1) + comp;
      const int nslots = V.n_tiles * V.n_gblocks;
      for (int sl = lane; sl < nslots; sl += 32)
        acc += partials[V.part_off + static_cast<long long>(sl) * V.slot_floats + nc * V.GB + part];
    }
  }
  acc = warp_sum_fixed(acc);
  if (lane == 0) gposes[12 * static_cast<long long>(p) + comp] += acc;
}

template <class B>
static cudaError_t launch_backward_reduce_t(const B& b, int n_flow, long long n_gauss, int n_poses,
                                            const BwdOut& out, cudaStream_t st) {
  const int nc = out.gcolors != nullptr ? 13 : 10;
  const long long warps = n_gauss * nc;
  const dim3 grid(static_cast<unsigned>((warps * 32 + 255) / 256));
  const float* partials = out.partials;
  cudaError_t e = launch_kernel(reduce_gauss_kernel<B>, grid, dim3(256), 0, st, 1, b, partials, out.gmeans,
                                out.gchol, out.gweights, out.gcolors, n_gauss, nc);
  if (e != cudaSuccess || out.gposes == nullptr) return e;
  return launch_kernel(reduce_pose_kernel<B>, dim3((n_poses * 12 * 32 + 255) / 256), dim3(256), 0, st, 1, b,
                       partials, out.gposes, n_poses, n_flow, nc);
}
cudaError_t launch_backward_reduce(const Batch& b, int n_flow, long long n_gauss, int n_poses, const BwdOut& out,
                                   cudaStream_t st) {
  return launch_backward_reduce_t(b, n_flow, n_gauss, n_poses, out, st);
}
cudaError_t launch_backward_reduce(const BigBatch& b, int n_flow, long long n_gauss, int n_poses, const BwdOut& out,
                                   cudaStream_t st) {
  return launch_backward_reduce_t(b, n_flow, n_gauss, n_poses, out, st);
}

}  // namespace fmb
