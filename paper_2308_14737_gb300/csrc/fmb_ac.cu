// fmb_ac.cu -- the zero-parameter alpha-compositing variant of the renderer
// (Sec. 3.3, Eq. 9-10) and its adjoint.
//
// The weights of Eq. 3 become w_i = T_i (1 - e^-delta_i) with the transmittance
// T_i = exp(-sum_j delta_j [t_j < t_i]) of the hits strictly in front of hit i.
// That needs the hits of a ray in depth order, so one warp takes one ray: lane l
// evaluates Gaussians e = m * 32 + l (m < M, K <= 32 M), and a bitonic network over
// the warp sorts 32 M 64-bit keys (an order-preserving integer image of t in the
// high word, the Gaussian index in the low word).  Prefix sums of delta in that
// order give T; hits at exactly equal depth share the sum in front of their run
// (the indicator is strict).  The weights go back to index order through shared
// memory and the blend of Eq. 3 is a warp reduction.  Alpha is Eq. 8, as in the
// two-parameter model; the saved planes are (W = sum w, sum delta, |N|).
//
// The adjoint keeps the Gaussian-parallel layout of the two-parameter backward.  A
// warp-per-ray phase re-renders each ray of a 32-ray tile and turns the upstream
// gradients into, per (ray, Gaussian), dbar (the gradient of d_i = log delta_i)
// and c_i = w_i / W, kept in shared memory:
//   wbar_i     = (Dbar (t_i - D) + Nbar . (n_i - N)) / W
//   deltabar_k = wbar_k T_k e^-delta_k - sum_{i: t_i > t_k} wbar_i w_i + Abar e^-sum delta
//   dbar_k     = deltabar_k delta_k
// (the suffix sum runs over the sorted order, again run-aware for equal depths).
// A packed pair loop (two Gaussians per thread) then recomputes the geometry of
// every pair and accumulates the same per-Gaussian sums as the two-parameter
// backward, with t's direct gradient Dbar c_i and the normal's scale c_i.  With the
// forward's depth orders kept (keep_order), four threads per ray walk the stored
// order instead of a warp re-sorting each ray (the TPR instantiation).
#include <algorithm>

#include "fmb_ac.cuh"
#include "fmb_f32x2.cuh"
#include "fmb_internal.cuh"

namespace fmb {

int ac_rays_per_item() { return kAcRays; }
// Forward run length (rays per warp; a work item is kAcWarps runs): the longest power
// of two up to kAcMaxRun that still gives every SM about 32 warps of work, so that
// large batches keep long runs of incrementally ordered neighbouring rays while small
// ones (a single 64x64 view) spread over the whole GPU instead of a few SMs.
int ac_fwd_run(long long total_rays, int sms) {
  const long long target_warps = 32ll * std::max(sms, 1);
  int run = kAcMaxRun;
  while (run > 1 && total_rays < target_warps * run) run >>= 1;
  return run;
}
int ac_fwd_rays_per_item(int run) { return kAcWarps * run; }

// ------------------------------------------------------------------ forward
// Register budget: 5 resident CTAs (20 warps) per SM for M <= 4 -- 96 registers, no
// spills, 6.5 % faster on the orbit than the unconstrained 127 -- and 4 for M = 8.
template <bool NORMALS, int NFLOW, int M>
__global__ void __launch_bounds__(kAcThreads, M >= 8 ? 4 : 5) forward_ac_kernel(const __grid_constant__ Batch batch, Scene s,
                                                                Consts k, const float4* __restrict__ records,
                                                                FwdOut out, int run, int* status, int* counter) {
  pdl_enter();
  extern __shared__ float4 ac_smem[];  // records [32 M][kAcRecStride float4] | per warp: sd, sw, sT [32 M floats each]
  __shared__ int s_item;
  __shared__ float ep[kAcWarps][kAcMaxRun][9];  // per ray of a warp's run: W, WT, Sd, WN, WC
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float4* srec = ac_smem;
  float* scratch = reinterpret_cast<float*>(ac_smem + 32 * M * kAcRecStride) + warp * 3 * 32 * M;
  float* sd = scratch;
  float* sw = scratch + 32 * M;
  float* sT = scratch + 64 * M;
  (void)status;  // no bounded waits here: the records are staged by plain loads
  for (int round = 0;; ++round) {
    const int item = next_item(counter, round, &s_item);
    if (item < 0 || item >= batch.n_items) break;
    int tile;
    const int vi = find_item(batch, item, tile);
    const DevView& V = batch.v[vi];
    const int P = V.P;
    if (round > 0) __syncthreads();  // the previous item's records are dead
    ac_stage_records(srec, records + kRecFloat4 * V.rec_off, V.K);
    float R[9], tp[3];
    load_pose(s.poses, V.pose, R, tp);
    const float o0 = -fmaf(R[6], tp[2], fmaf(R[3], tp[1], R[0] * tp[0]));
    const float o1 = -fmaf(R[7], tp[2], fmaf(R[4], tp[1], R[1] * tp[0]));
    const float o2 = -fmaf(R[8], tp[2], fmaf(R[5], tp[1], R[2] * tp[0]));
    float Rj[NFLOW > 0 ? NFLOW : 1][9], tj[NFLOW > 0 ? NFLOW : 1][3];
    bool has_t[NFLOW > 0 ? NFLOW : 1];
#pragma unroll
    for (int j = 0; j < NFLOW; ++j) {
      const int tg = j == 0 ? V.tgt0 : V.tgt1;
      has_t[j] = tg >= 0;
      if (has_t[j]) load_pose(s.poses, tg, Rj[j], tj[j]);
    }
    const long long off = V.pix_off;
    // each warp takes a run of neighbouring rays, so each starts from the previous
    // ray's depth order
    unsigned long long key[M];
    for (int m = 0; m < M; ++m) key[m] = kNoKey;
    for (int j = 0; j < run; ++j) {
      const int p = (tile * kAcWarps + warp) * run + j;
      if (p >= P) break;
      float vc[3], v[3], vl[3], pxy[2];
      pixel_ray_dd(V, R, ray_pixel(V, p), vc, v, vl, pxy);
      float t[M], dl[M], n[M][3];
      const float4* crec = s.crec != nullptr && out.color != nullptr ? s.crec + V.rec_off : nullptr;
      // a ray batch's consecutive entries are not neighbouring pixels: sort each afresh
      const AcSums a = ac_render_ray<NORMALS, M>(srec, V.K, v, vl, k, lane, t, dl, n, sd, sw, sT, key,
                                                 j > 0 && V.rays == nullptr, crec);
      if (out.order != nullptr) ac_store_order<M>(out.order + (off + p) * (32 * M), key, lane);
      if (lane == 0) {  // the ray's sums, for the epilogue below
        float* e = ep[warp][j];
        e[0] = a.W;
        e[1] = a.WT;
        e[2] = a.Sd;
        e[3] = a.WN0;
        e[4] = a.WN1;
        e[5] = a.WN2;
        e[6] = a.WC0;
        e[7] = a.WC1;
        e[8] = a.WC2;
      }
      __syncwarp();  // the scratch of this ray is read before the next ray overwrites it
    }
    // Per-ray epilogue, one lane per ray of the run (it was lane 0's alone per ray):
    // the planes of Eq. 3, 8, 17 and the Sec. 5 flow from the ray's sums.
    const int p_run = (tile * kAcWarps + warp) * run;
    if (lane < run && p_run + lane < P) {
      const int p = p_run + lane;
      float vc[3], v[3], vl[3], pxy[2];
      pixel_ray_dd(V, R, ray_pixel(V, p), vc, v, vl, pxy);
      const float* e = ep[warp][lane];
      const float4* crec = s.crec != nullptr && out.color != nullptr ? s.crec + V.rec_off : nullptr;
      const float iW = e[0] > 0.f ? 1.0f / e[0] : 0.f;
      const float D = e[1] * iW;
      if (crec != nullptr) {
        float* col = out.color + 3 * off;
        col[p] = e[6] * iW;
        col[P + p] = e[7] * iW;
        col[2 * P + p] = e[8] * iW;
      }
      out.depth[off + p] = D;
      out.alpha[off + p] = -expm1f(-e[2]);
      float* sv = out.saved + 3 * off;
      sv[p] = e[0];
      sv[P + p] = e[2];
      if (NORMALS) {
        const float N0 = e[3] * iW, N1 = e[4] * iW, N2 = e[5] * iW;
        const float Nn = sqrtf(fmaf(N0, N0, fmaf(N1, N1, N2 * N2)));
        const float iN = Nn > 0.f ? 1.0f / Nn : 0.f;
        const float n0 = N0 * iN, n1 = N1 * iN, n2 = N2 * iN;
        float* nrm = out.normal + 3 * off;
        nrm[p] = fmaf(R[2], n2, fmaf(R[1], n1, R[0] * n0));
        nrm[P + p] = fmaf(R[5], n2, fmaf(R[4], n1, R[3] * n0));
        nrm[2 * P + p] = fmaf(R[8], n2, fmaf(R[7], n1, R[6] * n0));
        sv[2 * P + p] = Nn;
      } else {
        sv[2 * P + p] = 0.f;
      }
      if (NFLOW > 0) {
        const float p0 = fmaf(v[0], D, o0), p1 = fmaf(v[1], D, o1), p2 = fmaf(v[2], D, o2);
        float* fl = out.flow + 2 * NFLOW * off;
#pragma unroll
        for (int j = 0; j < NFLOW; ++j) {
          float fu = 0.f, fv = 0.f;
          if (has_t[j]) {
            const float X0 = fmaf(Rj[j][2], p2, fmaf(Rj[j][1], p1, fmaf(Rj[j][0], p0, tj[j][0])));
            const float X1 = fmaf(Rj[j][5], p2, fmaf(Rj[j][4], p1, fmaf(Rj[j][3], p0, tj[j][1])));
            const float X2 = fmaf(Rj[j][8], p2, fmaf(Rj[j][7], p1, fmaf(Rj[j][6], p0, tj[j][2])));
            const float iz = 1.0f / X2;
            fu = fmaf(V.fx * X0, iz, V.cx) - pxy[0];
            fv = fmaf(V.fy * X1, iz, V.cy) - pxy[1];
          }
          fl[(2 * j) * P + p] = fu;
          fl[(2 * j + 1) * P + p] = fv;
        }
      }
    }
    __syncwarp();  // ep is read before the next item's rays overwrite it
  }
}

// ----------------------------------------------------------------- backward
struct AcAcc2 {
  f2 nSd, Y0, Y1, Y2, G00, G10, G11, G20, G21, G22, M[9];
  f2 Cb0, Cb1, Cb2;  // colour mode: sum (w / W) Cbar
};

// One packed step: two Gaussians (lanes) against one ray.  rr: the ray's record
// (5 x 16 bytes, duplicated values), pd: (dbar, c) of both Gaussians.
template <bool NORMALS, bool COLOR = false>
__device__ __forceinline__ void bwd_pair_ac2(AcAcc2& A, const GaussRec2& gr, const ulonglong2* __restrict__ rr,
                                             float4 pd, f2 tiny) {
  const ulonglong2 q0 = rr[0], q1 = rr[1], q2 = rr[2], q3 = rr[3], q4 = rr[4];
  const f2 v0 = as_f2(q0.x), v1 = as_f2(q0.y), v2 = as_f2(q1.x), Dbar = as_f2(q1.y);
  const f2 ndbar = pk(-pd.x, -pd.z), c = pk(pd.y, pd.w);
  const PairGeom2 G = pair_geom2(gr, v0, v1, v2, as_f2(q3.y), as_f2(q4.x), as_f2(q4.y));
  const f2 t = G.t;
  f2 ub0, ub1, ub2, tbar, gb0, gb1, gb2;
  if (NORMALS) {
    const f2 Nb0 = as_f2(q2.x), Nb1 = as_f2(q2.y), Nb2 = as_f2(q3.x);
    const f2 g0 = mul2(gr.L[0], G.u0);
    const f2 g1 = fma2(gr.L[2], G.u1, mul2(gr.L[1], G.u0));
    const f2 g2 = fma2(gr.L[5], G.u2, fma2(gr.L[4], G.u1, mul2(gr.L[3], G.u0)));
    const f2 gg = add2(fma2(g2, g2, fma2(g1, g1, mul2(g0, g0))), tiny);
    const f2 rs = rsqrt_2(gg);
    const f2 n0 = mul2(g0, rs), n1 = mul2(g1, rs), n2 = mul2(g2, rs);
    const f2 nN = fma2(n2, Nb2, fma2(n1, Nb1, mul2(n0, Nb0)));
    const f2 sc = mul2(c, rs);
    const f2 sN = mul2(sc, nN);
    const f2 nsN = pk(-lo(sN), -hi(sN));
    gb0 = fma2(nsN, n0, mul2(sc, Nb0));
    gb1 = fma2(nsN, n1, mul2(sc, Nb1));
    gb2 = fma2(nsN, n2, mul2(sc, Nb2));
    ub0 = fma2(gr.L[3], gb2, fma2(gr.L[1], gb1, mul2(gr.L[0], gb0)));
    ub1 = fma2(gr.L[4], gb2, mul2(gr.L[2], gb1));
    ub2 = mul2(gr.L[5], gb2);
    tbar = fma2(ub2, G.a2, fma2(ub1, G.a1, fma2(ub0, G.a0, mul2(Dbar, c))));
  } else {
    ub0 = ub1 = ub2 = gb0 = gb1 = gb2 = dup(0.f);
    tbar = mul2(Dbar, c);
  }
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
  if (COLOR) {  // record slots 5-6: [Cb0 Cb0 Cb1 Cb1 | Cb2 Cb2 0 0]
    const ulonglong2 q5 = rr[5], q6 = rr[6];
    A.Cb0 = fma2(c, as_f2(q5.x), A.Cb0);
    A.Cb1 = fma2(c, as_f2(q5.y), A.Cb1);
    A.Cb2 = fma2(c, as_f2(q6.x), A.Cb2);
  }
}

// Per-ray part of the adjoint, shared by the warp-per-ray and the four-threads-per-
// ray phases: the colour's upstream gradient Cbar (colour mode), the depth's total
// upstream gradient Dbar (its own plus the flow's, Sec. 5), Nbar of the blended
// normal N = sum w n / W (the Eq. 17 renormalisation, world frame) and Abar e^-Sd
// (Eq. 8).  With pose_lane the ray's pose-gradient terms are added to pose_acc.
struct AcRayAdj {
  float Dbar, KA, Nb[3], Cb[3];
};
template <bool NORMALS, int NFLOW, int NPV>
__device__ __forceinline__ AcRayAdj ac_ray_adjoint(const DevView& V, const BwdIn& in, long long off, int p,
                                                   const float (&v)[3], const float (&vc)[3], const float (&R)[9],
                                                   const float (&tp)[3], float o0, float o1, float o2,
                                                   const float (&Rj)[NFLOW > 0 ? NFLOW : 1][9],
                                                   const float (&tj)[NFLOW > 0 ? NFLOW : 1][3],
                                                   const bool (&has_t)[NFLOW > 0 ? NFLOW : 1], float D,
                                                   const float (&N)[3], float Sd, bool color, bool pose_lane,
                                                   float (&pose_acc)[NPV]) {
  const int P = V.P;
  AcRayAdj r;
  float* Cb = r.Cb;
  Cb[0] = Cb[1] = Cb[2] = 0.f;
  if (color && in.g_color != nullptr) {
    const float* gc3 = in.g_color + 3 * off;
#pragma unroll
    for (int k3 = 0; k3 < 3; ++k3) Cb[k3] = gc3[k3 * P + p];
  }
  const float gD = in.g_depth ? in.g_depth[off + p] : 0.f;
  const float gA = in.g_alpha ? in.g_alpha[off + p] : 0.f;
  // flow (Sec. 5): p3 = o + v D, X = R_j p3 + t_j, flow = pi(X) - pixel
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
      if (pose_lane) {
        float* pa = pose_acc + 12 * (1 + j);
        const float Xb[3] = {Xb0, Xb1, Xb2};
        const float pp[3] = {p0, p1, p2};
#pragma unroll
        for (int a3 = 0; a3 < 3; ++a3) {
#pragma unroll
          for (int c = 0; c < 3; ++c) pa[3 * a3 + c] = fmaf(Xb[a3], pp[c], pa[3 * a3 + c]);
          pa[9 + a3] += Xb[a3];
        }
      }
    }
  }
  const float Dbar = fmaf(v[2], pb2, fmaf(v[1], pb1, fmaf(v[0], pb0, gD)));
  r.Dbar = Dbar;
  if (NFLOW > 0 && pose_lane) {
    const float w3[3] = {fmaf(D, vc[0], -tp[0]), fmaf(D, vc[1], -tp[1]), fmaf(D, vc[2], -tp[2])};
    const float pb[3] = {pb0, pb1, pb2};
#pragma unroll
    for (int a3 = 0; a3 < 3; ++a3) {
#pragma unroll
      for (int c = 0; c < 3; ++c) pose_acc[3 * a3 + c] = fmaf(w3[a3], pb[c], pose_acc[3 * a3 + c]);
      pose_acc[9 + a3] -= fmaf(R[3 * a3 + 2], pb2, fmaf(R[3 * a3 + 1], pb1, R[3 * a3] * pb0));
    }
  }
  // normal: ncam = R n_f, n_f = N / |N|, N = sum w n / W
  float* Nb = r.Nb;
  Nb[0] = Nb[1] = Nb[2] = 0.f;
  if (NORMALS && in.g_normal != nullptr) {
    const float Nn = sqrtf(fmaf(N[0], N[0], fmaf(N[1], N[1], N[2] * N[2])));
    const float iN = Nn > 0.f ? 1.0f / Nn : 0.f;
    const float nf[3] = {N[0] * iN, N[1] * iN, N[2] * iN};
    const float* gn3 = in.g_normal + 3 * off;
    const float gn[3] = {gn3[p], gn3[P + p], gn3[2 * P + p]};
    float nfb[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) nfb[c] = fmaf(R[6 + c], gn[2], fmaf(R[3 + c], gn[1], R[c] * gn[0]));
    if (pose_lane) {
#pragma unroll
      for (int a3 = 0; a3 < 3; ++a3)
#pragma unroll
        for (int c = 0; c < 3; ++c) pose_acc[3 * a3 + c] = fmaf(gn[a3], nf[c], pose_acc[3 * a3 + c]);
    }
    if (Nn > 0.f) {
      const float sdot = fmaf(nf[2], nfb[2], fmaf(nf[1], nfb[1], nf[0] * nfb[0]));
#pragma unroll
      for (int c = 0; c < 3; ++c) Nb[c] = fmaf(-sdot, nf[c], nfb[c]) * iN;
    }
  }
  r.KA = gA * __expf(-Sd);
  return r;
}

// Shared memory of the backward, in floats after the records:
//   ray records [kAcRays][kAcRayRec float4] | pair values [kAcRays][32 M][2] |
//   per warp scratch sd, sw, sT, sq [32 M floats each]
// The pair values region is reused for the per-thread sums of the reduction.
constexpr int kAcAccFloats = 44;  // 22 sums per thread, two Gaussians (with the colour sums)
template <int M>
__host__ __device__ constexpr int ac_pairv_floats() {
  return kAcRays * 32 * M * 2 > kAcThreads * kAcAccFloats ? kAcRays * 32 * M * 2 : kAcThreads * kAcAccFloats;
}
template <int M>
__host__ __device__ constexpr int ac_bwd_smem_floats() {
  return 32 * M * 4 * kAcRecStride + kAcRays * kAcRayRec * 4 + ac_pairv_floats<M>() + kAcWarps * 4 * 32 * M;
}

// TPR: the per-ray phase runs four threads per ray over the forward's stored depth
// order (keep_order; see the four-thread phase below), the warp-per-ray phase only
// for the rays whose stored order fails its check.  Register budget: 3 CTAs per SM
// (4 with TPR, whose phase spills 24-60 bytes at 128 registers and runs 1.2 %
// faster on the orbit; the re-sorting phase spills 148-164 bytes there and is 9 %
// slower), 2 for M = 8.
template <bool NORMALS, int NFLOW, int M, bool TPR>
__global__ void __launch_bounds__(kAcThreads, M >= 8 ? 2 : (TPR ? 4 : 3)) backward_ac_kernel(const __grid_constant__ Batch batch, Scene s,
                                                                 Consts k, const float4* __restrict__ records,
                                                                 BwdIn in, BwdOut out, int* status, int* counter) {
  pdl_enter();
  extern __shared__ float4 ac_smem[];
  constexpr int NPV = 12 * (1 + NFLOW);
  __shared__ float pose_ray[kAcWarps][NPV];
  __shared__ float pose_gau[kAcWarps][12];
  __shared__ int s_item;
  __shared__ unsigned s_bad;  // TPR: rays of the item left to the warp-per-ray phase
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float4* srec = ac_smem;
  float4* rays = ac_smem + 32 * M * kAcRecStride;
  float* pairv = reinterpret_cast<float*>(rays + kAcRays * kAcRayRec);
  float* scratch = pairv + ac_pairv_floats<M>() + warp * 4 * 32 * M;
  float* sd = scratch;
  float* sw = scratch + 32 * M;
  float* sT = scratch + 64 * M;
  float* sq = scratch + 96 * M;
  (void)status;  // no bounded waits here: the records are staged by plain loads
  const bool want_pose = out.gposes != nullptr;
  const bool color = s.crec != nullptr && out.gcolors != nullptr;  // colour mode (uniform)
  const int NC = color ? 13 : 10;  // gradient values per Gaussian in a partial slot
  for (int round = 0;; ++round) {
    const int item = next_item(counter, round, &s_item);
    if (item < 0 || item >= batch.n_items) break;
    int tile;
    const int vi = find_item(batch, item, tile);
    const DevView& V = batch.v[vi];
    const int P = V.P;
    const int K = V.K;
    const int pix0 = tile * kAcRays;
    const int nr = min(kAcRays, P - pix0);
    const long long off = V.pix_off;
    if (round > 0) __syncthreads();
    if (TPR && tid == 0) s_bad = 0u;  // published by the staging's barrier
    ac_stage_records(srec, records + kRecFloat4 * V.rec_off, K);

    // ------------- phase A: one warp per ray -> per-ray record and per-pair (dbar, c)
    float R[9], tp[3];
    load_pose(s.poses, V.pose, R, tp);
    const float o0 = -fmaf(R[6], tp[2], fmaf(R[3], tp[1], R[0] * tp[0]));
    const float o1 = -fmaf(R[7], tp[2], fmaf(R[4], tp[1], R[1] * tp[0]));
    const float o2 = -fmaf(R[8], tp[2], fmaf(R[5], tp[1], R[2] * tp[0]));
    float Rj[NFLOW > 0 ? NFLOW : 1][9], tj[NFLOW > 0 ? NFLOW : 1][3];
    bool has_t[NFLOW > 0 ? NFLOW : 1];
#pragma unroll
    for (int j = 0; j < NFLOW; ++j) {
      const int tg = j == 0 ? V.tgt0 : V.tgt1;
      has_t[j] = tg >= 0 && in.g_flow != nullptr;
      if (has_t[j]) load_pose(s.poses, tg, Rj[j], tj[j]);
    }
    float pose_acc[NPV];
#pragma unroll
    for (int i = 0; i < NPV; ++i) pose_acc[i] = 0.f;
    if (TPR) {
      // ------------- phase A': four threads per ray over the forward's depth order.
      // Thread `sub` of ray rr walks the ray's sorted positions [c0, c1).  A first pass
      // forms the chunk's sums of w, w (t - Dref), w n and w c with the transmittance of
      // the hits in front of it within the chunk; the four chunks combine by shuffles
      // (T = exp(-S_in) exp(-S_chunk), the sums of the earlier chunks give each chunk's
      // prefix); a second pass writes (dbar delta, w / W) per pair, the sums over the
      // hits behind a hit being the ray's totals minus the inclusive prefix, which the
      // linearity of wbar in (t, n, c) turns into U of Eq. 10's adjoint.  A ray whose
      // stored order is not strictly increasing in the recomputed depths (equal depths,
      // bytes from another call) or whose object has fewer than 8 Gaussians is left to
      // the warp-per-ray phase below.
      static_assert(kAcThreads / 4 == kAcRays, "four threads per ray of the item");
      static_assert(8 * 32 * M <= 4 * 32 * M * static_cast<int>(sizeof(float)), "a warp's 8 orders fit its scratch");
      const int rr = tid >> 2, sub = tid & 3;
      const bool live = rr < nr;
      const int p = pix0 + (live ? rr : 0);
      float vc[3], v[3], vl[3], pxy[2];
      pixel_ray_dd(V, R, ray_pixel(V, p), vc, v, vl, pxy);
      // the warp's eight stored orders, staged by 16-byte loads into its scratch (which
      // only the warp-per-ray phase uses, after this one)
      unsigned char* orows = reinterpret_cast<unsigned char*>(scratch);
      {
        constexpr int kRowU4 = 32 * M / 16;  // 16-byte words per row
        for (int i = lane; i < 8 * kRowU4; i += 32) {
          const int rj = warp * 8 + i / kRowU4;
          if (rj < nr)
            reinterpret_cast<uint4*>(orows)[i] =
                __ldg(reinterpret_cast<const uint4*>(in.order + (off + pix0 + rj) * (32 * M)) + i % kRowU4);
        }
        __syncwarp();
      }
      const unsigned char* orow = orows + (rr & 7) * (32 * M);
      const int c0 = (K * sub) >> 2, c1 = (K * (sub + 1)) >> 2;
      float Dref = in.depth[off + p];  // centres the depth sums (any finite value is exact)
      if (!(fabsf(Dref) < 1e30f)) Dref = 0.f;
      const float4* crec = color ? s.crec + V.rec_off : nullptr;
      constexpr int NS = 8;  // sums: w, w (t - Dref), w n (3), w c (3)
      bool ok = K >= 8;
      float Sc = 0.f, tl = -INFINITY, t0 = INFINITY;
      float sum[NS];
#pragma unroll
      for (int q = 0; q < NS; ++q) sum[q] = 0.f;
#pragma unroll 2
      for (int i = c0; i < c1; ++i) {
        const int e = orow[i];
        ok = ok && e < K;
        const AcPair q = ac_pair_eval<NORMALS>(srec + kAcRecStride * (e < K ? e : 0), v, vl, k);
        ok = ok && q.t > tl;  // strictly increasing: a sorted permutation without ties
        if (i == c0) t0 = q.t;
        tl = q.t;
        const float w = ex2_approx(-Sc * kLog2e) * one_minus_exp_neg(q.dl);
        Sc += q.dl;
        sum[0] += w;
        sum[1] = fmaf(w, q.t - Dref, sum[1]);
        if (NORMALS) {
#pragma unroll
          for (int c = 0; c < 3; ++c) sum[2 + c] = fmaf(w, q.n[c], sum[2 + c]);
        }
        if (color) {
          const float4 cc = __ldg(crec + (e < K ? e : 0));
          sum[5] = fmaf(w, cc.x, sum[5]);
          sum[6] = fmaf(w, cc.y, sum[6]);
          sum[7] = fmaf(w, cc.z, sum[7]);
        }
      }
      // the ray's four chunks, in depth order: lanes 4 rr .. 4 rr + 3 of the warp
      const float Sin = ac_excl4(Sc, sub);
      const float Sd = __shfl_sync(kFull, Sin + Sc, 3, 4);
      const float T0 = ex2_approx(-Sin * kLog2e);
      const float tprev = __shfl_up_sync(kFull, tl, 1, 4);
      ok = ok && (sub == 0 || t0 > tprev);
      const bool ok4 = __shfl_sync(kFull, ac_all4(ok) ? 1 : 0, 0, 4) != 0;
      float pre[NS], tot[NS];
#pragma unroll
      for (int q = 0; q < NS; ++q) {
        const float x = T0 * sum[q];
        pre[q] = ac_excl4(x, sub);
        tot[q] = __shfl_sync(kFull, pre[q] + x, 3, 4);
      }
      const float W = tot[0];
      const float iW = W > 0.f ? 1.0f / W : 0.f;
      const float Dc = tot[1] * iW;  // D - Dref
      const float N[3] = {tot[2] * iW, tot[3] * iW, tot[4] * iW};
      const float Cc[3] = {tot[5] * iW, tot[6] * iW, tot[7] * iW};
      const bool use = live && ok4;
      const AcRayAdj ra = ac_ray_adjoint<NORMALS, NFLOW, NPV>(V, in, off, p, v, vc, R, tp, o0, o1, o2, Rj, tj, has_t,
                                                              Dref + Dc, N, Sd, color, want_pose && use && sub == 0,
                                                              pose_acc);
      if (use) {
        float2* pv = reinterpret_cast<float2*>(pairv) + rr * 32 * M;
        float S2 = 0.f;
        float run[NS];
#pragma unroll
        for (int q = 0; q < NS; ++q) run[q] = 0.f;
#pragma unroll 2
        for (int i = c0; i < c1; ++i) {
          const int e = orow[i];
          const AcPair q = ac_pair_eval<NORMALS>(srec + kAcRecStride * e, v, vl, k);
          const float Tl = ex2_approx(-S2 * kLog2e);
          const float wl = Tl * one_minus_exp_neg(q.dl);
          S2 += q.dl;
          run[0] += wl;
          run[1] = fmaf(wl, q.t - Dref, run[1]);
          // sums over the hits strictly behind this one (its depth is unique on the ray)
          const float SW = W - (pre[0] + T0 * run[0]);
          float x = ra.Dbar * ((q.t - Dref) - Dc);
          float u = ra.Dbar * ((tot[1] - (pre[1] + T0 * run[1])) - Dc * SW);
          if (NORMALS) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              run[2 + c] = fmaf(wl, q.n[c], run[2 + c]);
              x = fmaf(ra.Nb[c], q.n[c] - N[c], x);
              u = fmaf(ra.Nb[c], (tot[2 + c] - (pre[2 + c] + T0 * run[2 + c])) - N[c] * SW, u);
            }
          }
          if (color) {
            const float4 cc = __ldg(crec + e);
            const float cv[3] = {cc.x, cc.y, cc.z};
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              run[5 + c] = fmaf(wl, cv[c], run[5 + c]);
              x = fmaf(ra.Cb[c], cv[c] - Cc[c], x);
              u = fmaf(ra.Cb[c], (tot[5 + c] - (pre[5 + c] + T0 * run[5 + c])) - Cc[c] * SW, u);
            }
          }
          const float wbar = x * iW;
          const float deltabar = fmaf(wbar * (T0 * Tl), ex2_approx(-q.dl * kLog2e), ra.KA - u * iW);
          pv[e] = make_float2(deltabar * q.dl, T0 * wl * iW);
        }
        if (sub == 0) {
          if (K & 1) pv[K] = make_float2(0.f, 0.f);  // the odd block's second lane in the pair loop
          float4* rec = rays + rr * kAcRayRec;
          rec[0] = make_float4(v[0], v[0], v[1], v[1]);
          rec[1] = make_float4(v[2], v[2], ra.Dbar, ra.Dbar);
          rec[2] = make_float4(ra.Nb[0], ra.Nb[0], ra.Nb[1], ra.Nb[1]);
          rec[3] = make_float4(ra.Nb[2], ra.Nb[2], vl[0], vl[0]);
          rec[4] = make_float4(vl[1], vl[1], vl[2], vl[2]);
          rec[5] = make_float4(ra.Cb[0], ra.Cb[0], ra.Cb[1], ra.Cb[1]);
          rec[6] = make_float4(ra.Cb[2], ra.Cb[2], 0.f, 0.f);
        }
      } else if (live && sub == 0) {
        atomicOr(&s_bad, 1u << rr);
      }
      if (want_pose) {
#pragma unroll
        for (int i = 0; i < NPV; ++i) {
          const float x = warp_allsum(pose_acc[i]);
          if (lane == 0) pose_ray[warp][i] = x;
          pose_acc[i] = 0.f;
        }
      }
      __syncthreads();  // s_bad is complete
    }
    constexpr int kPerWarp = kAcRays / kAcWarps;
    unsigned long long key[M];
    for (int m = 0; m < M; ++m) key[m] = kNoKey;
    for (int j = 0; j < kPerWarp; ++j) {
      const int rr = warp * kPerWarp + j;  // a run of neighbouring rays per warp
      if (rr >= nr) break;
      if (TPR && !((s_bad >> rr) & 1u)) continue;  // done by the four-thread phase
      const int p = pix0 + rr;
      float vc[3], v[3], vl[3], pxy[2];
      pixel_ray_dd(V, R, ray_pixel(V, p), vc, v, vl, pxy);
      float t[M], dl[M], n[M][3];
      const float4* crec = color ? s.crec + V.rec_off : nullptr;
      // the forward's order (keep_order): the refinement then only confirms it
      if (in.order != nullptr) ac_load_order<M>(in.order + (off + p) * (32 * M), K, lane, key);
      const AcSums a = ac_render_ray<NORMALS, M>(srec, K, v, vl, k, lane, t, dl, n, sd, sw, sT, key,
                                                 in.order != nullptr || (j > 0 && V.rays == nullptr), crec);
      const float iW = a.W > 0.f ? 1.0f / a.W : 0.f;
      const float D = a.WT * iW;
      // colour mode: Cbar and the blended colour C = sum w c / W
      const float Cc[3] = {a.WC0 * iW, a.WC1 * iW, a.WC2 * iW};
      const float N[3] = {a.WN0 * iW, a.WN1 * iW, a.WN2 * iW};
      const AcRayAdj ra = ac_ray_adjoint<NORMALS, NFLOW, NPV>(V, in, off, p, v, vc, R, tp, o0, o1, o2, Rj, tj, has_t,
                                                              D, N, a.Sd, color, want_pose && lane == 0, pose_acc);
      const float Dbar = ra.Dbar, KA = ra.KA;
      const float Nb[3] = {ra.Nb[0], ra.Nb[1], ra.Nb[2]}, Cb[3] = {ra.Cb[0], ra.Cb[1], ra.Cb[2]};
      // wbar_e (index order) and q_e = wbar_e w_e
      float wbar[M];
#pragma unroll
      for (int m = 0; m < M; ++m) {
        const int e = (m << 5) | lane;
        wbar[m] = 0.f;
        if (e < K) {
          float x = Dbar * (t[m] - D);
          if (NORMALS)
            x = fmaf(Nb[0], n[m][0] - N[0], fmaf(Nb[1], n[m][1] - N[1], fmaf(Nb[2], n[m][2] - N[2], x)));
          if (color) {
            const float4 c = __ldg(crec + e);
            x = fmaf(Cb[0], c.x - Cc[0], fmaf(Cb[1], c.y - Cc[1], fmaf(Cb[2], c.z - Cc[2], x)));
          }
          wbar[m] = x * iW;
          sq[e] = wbar[m] * sw[e];
        }
      }
      __syncwarp();
      // Suffix sums of q over the hits strictly behind each hit, in sorted order (the
      // keys ac_render_ray left sorted): U = total - (inclusive prefix at the end of
      // the hit's run of equal depth).
      {
        // sorted order, lane holding positions lane M + m: inclusive prefix Q of q
        float ts[M], Q[M];
        int idx[M];
        float lane_sum = 0.f;
#pragma unroll
        for (int m = 0; m < M; ++m) {
          const bool valid = key[m] != kNoKey;
          idx[m] = valid ? static_cast<int>(key[m] & 0xffffffffu) : -1;
          ts[m] = valid ? from_order_bits(static_cast<unsigned>(key[m] >> 32)) : INFINITY;
          lane_sum += valid ? sq[idx[m]] : 0.f;
          Q[m] = lane_sum;
        }
        const float incl_lane = warp_incl_sum(lane_sum, lane);
        const float Qtot = __shfl_sync(kFull, incl_lane, 31);
        const float before = incl_lane - lane_sum;
        float next_t = __shfl_down_sync(kFull, ts[0], 1);
        if (lane == 31) next_t = INFINITY;
        // Q at the end of each hit's run of equal depth: the first run end at or after
        // the position, within the lane (a backward pass) or in the lanes after it
        // (a segmented copy-from-the-right scan of each lane's first run end).
        float vloc[M];
        bool has[M];
        bool h = false;
        float vv = 0.f;
#pragma unroll
        for (int m = M - 1; m >= 0; --m) {
          if (ts[m] != (m == M - 1 ? next_t : ts[m + 1])) {
            h = true;
            vv = before + Q[m];
          }
          has[m] = h;
          vloc[m] = vv;
        }
        float F = vloc[0];
        bool Ff = has[0];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const float ov = __shfl_down_sync(kFull, F, o);
          const bool of = __shfl_down_sync(kFull, Ff ? 1 : 0, o) != 0;
          if (!Ff && lane + o < 32) {
            F = ov;
            Ff = of;
          }
        }
        const float cin = __shfl_down_sync(kFull, F, 1);
#pragma unroll
        for (int m = 0; m < M; ++m)
          if (idx[m] >= 0) sd[idx[m]] = Qtot - (has[m] ? vloc[m] : cin);  // sd now holds U
      }
      __syncwarp();
      // dbar and c per (ray, Gaussian) into the pair buffer; the ray record
      float2* pv = reinterpret_cast<float2*>(pairv) + rr * 32 * M;
#pragma unroll
      for (int m = 0; m < M; ++m) {
        const int e = (m << 5) | lane;
        float2 val = make_float2(0.f, 0.f);
        if (e < K) {
          const float U = sd[e];
          const float deltabar = fmaf(wbar[m] * sT[e], ex2_approx(-dl[m] * kLog2e), KA - U);
          val = make_float2(deltabar * dl[m], sw[e] * iW);
        }
        pv[e] = val;
      }
      if (lane == 0) {
        float4* rec = rays + rr * kAcRayRec;
        rec[0] = make_float4(v[0], v[0], v[1], v[1]);
        rec[1] = make_float4(v[2], v[2], Dbar, Dbar);
        rec[2] = make_float4(Nb[0], Nb[0], Nb[1], Nb[1]);
        rec[3] = make_float4(Nb[2], Nb[2], vl[0], vl[0]);
        rec[4] = make_float4(vl[1], vl[1], vl[2], vl[2]);
        rec[5] = make_float4(Cb[0], Cb[0], Cb[1], Cb[1]);
        rec[6] = make_float4(Cb[2], Cb[2], 0.f, 0.f);
      }
      __syncwarp();
    }
    if (want_pose) {
#pragma unroll
      for (int i = 0; i < NPV; ++i)
        if (lane == 0) pose_ray[warp][i] = TPR ? pose_ray[warp][i] + pose_acc[i] : pose_acc[i];
    }
    __syncthreads();

    // ------------- phase B: Gaussian-parallel packed pair loop over the tile's rays
    const int GB2 = (K + 1) / 2;
    const int S = max(1, kAcThreads / GB2);
    const int gl2 = tid % GB2;
    const int sg = tid / GB2;
    const int g0 = 2 * gl2;
    const bool active = sg < S;
    AcAcc2 A;
    A.nSd = A.Y0 = A.Y1 = A.Y2 = dup(0.f);
    A.Cb0 = A.Cb1 = A.Cb2 = dup(0.f);
    A.G00 = A.G10 = A.G11 = A.G20 = A.G21 = A.G22 = dup(0.f);
#pragma unroll
    for (int i = 0; i < 9; ++i) A.M[i] = dup(0.f);
    if (active) {
      const GaussRec ga = unpack_rec(srec[kAcRecStride * g0], srec[kAcRecStride * g0 + 1],
                                     srec[kAcRecStride * g0 + 2], srec[kAcRecStride * g0 + 3]);
      const int g1 = g0 + 1 < K ? g0 + 1 : g0;
      const GaussRec gbr = unpack_rec(srec[kAcRecStride * g1], srec[kAcRecStride * g1 + 1],
                                      srec[kAcRecStride * g1 + 2], srec[kAcRecStride * g1 + 3]);
      const GaussRec2 gr = pair_rec(ga, gbr);
      const f2 tiny = dup(1e-30f);
      const ulonglong2* rrec = reinterpret_cast<const ulonglong2*>(rays);
      const float4* pv4 = reinterpret_cast<const float4*>(pairv);
      if (color) {
#pragma unroll 2
        for (int r = sg; r < nr; r += S)
          bwd_pair_ac2<NORMALS, true>(A, gr, rrec + kAcRayRec * r, pv4[(r * 32 * M + g0) / 2], tiny);
      } else {
#pragma unroll 2
        for (int r = sg; r < nr; r += S)
          bwd_pair_ac2<NORMALS>(A, gr, rrec + kAcRayRec * r, pv4[(r * 32 * M + g0) / 2], tiny);
      }
    }
    __syncthreads();  // the pair buffer is dead; reuse it for the reduction

    // ------------- phase C: combine subgroups, finalise per Gaussian
    float* red = pairv;
    if (active) {
      float* d = red + kAcAccFloats * tid;
      const f2 vv[22] = {A.nSd, A.Y0, A.Y1, A.Y2, A.G00, A.G10, A.G11, A.G20, A.G21, A.G22, A.M[0],
                         A.M[1], A.M[2], A.M[3], A.M[4], A.M[5], A.M[6], A.M[7], A.M[8], A.Cb0, A.Cb1, A.Cb2};
#pragma unroll
      for (int i = 0; i < 22; ++i) {
        d[i] = lo(vv[i]);
        d[22 + i] = hi(vv[i]);
      }
    }
    __syncthreads();
    float* slot = nullptr;
    if (out.partials) slot = out.partials + V.part_off + static_cast<long long>(tile) * V.slot_floats;
    float pose_g[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) pose_g[i] = 0.f;
    // Atomic mode: the item's gradient values go to shared memory (the per-warp
    // scratch, dead after the pair loop) in the outputs' layout, and the CTA then adds
    // them with consecutive threads on consecutive floats: a Gaussian-per-thread
    // pattern (stride 3 or 6 floats) touched about 4.5 times as many 32-byte sectors,
    // and thousands of items add into the same few kilobytes of one object's
    // gradients (one L2 slice was 80 % busy with them on the orbit).
    float* cg = pairv + ac_pairv_floats<M>();  // 13 K floats: [3K means | 6K chol | K weights | 3K colours]
    static_assert(13 * 32 * M <= kAcWarps * 4 * 32 * M, "the staged gradients fit the scratch");
    for (int gi = tid; gi < K; gi += kAcThreads) {
      float acc[22];
#pragma unroll
      for (int i = 0; i < 22; ++i) acc[i] = 0.f;
      for (int s2 = 0; s2 < S; ++s2) {
        const float* d = red + kAcAccFloats * (s2 * GB2 + (gi >> 1)) + 22 * (gi & 1);
#pragma unroll
        for (int i = 0; i < 22; ++i) acc[i] += d[i];
      }
      const GaussRec g = unpack_rec(srec[kAcRecStride * gi], srec[kAcRecStride * gi + 1],
                                    srec[kAcRecStride * gi + 2], srec[kAcRecStride * gi + 3]);
      const long long gg = V.gauss_off + gi;
      const float L00 = g.L[0], L10 = g.L[1], L11 = g.L[2], L20 = g.L[3], L21 = g.L[4], L22 = g.L[5];
      const float Bb0 = -acc[1], Bb1 = -acc[2], Bb2 = -acc[3];
      float gm[3], gL[6];
      gm[0] = L00 * Bb0;
      gm[1] = fmaf(L11, Bb1, L10 * Bb0);
      gm[2] = fmaf(L22, Bb2, fmaf(L21, Bb1, L20 * Bb0));
      const float m0 = g.mh[0], m1 = g.mh[1], m2 = g.mh[2];
      const float* Mx = acc + 10;
      gL[0] = acc[4] + Mx[0] + m0 * Bb0;
      gL[1] = acc[5] + Mx[3] + m1 * Bb0;
      gL[2] = acc[6] + Mx[4] + m1 * Bb1;
      gL[3] = acc[7] + Mx[6] + m2 * Bb0;
      gL[4] = acc[8] + Mx[7] + m2 * Bb1;
      gL[5] = acc[9] + Mx[8] + m2 * Bb2;
      const float glam = -acc[0] / s.weights[gg];
      if (want_pose) {
        float ML[9];
        const float Lf[9] = {L00, 0.f, 0.f, L10, L11, 0.f, L20, L21, L22};
#pragma unroll
        for (int a3 = 0; a3 < 3; ++a3)
#pragma unroll
          for (int c = 0; c < 3; ++c)
            ML[3 * a3 + c] =
                fmaf(Mx[3 * a3 + 2], Lf[3 * c + 2], fmaf(Mx[3 * a3 + 1], Lf[3 * c + 1], Mx[3 * a3] * Lf[3 * c]));
#pragma unroll
        for (int a3 = 0; a3 < 3; ++a3) {
#pragma unroll
          for (int c = 0; c < 3; ++c)
            pose_g[3 * a3 + c] +=
                fmaf(R[3 * a3 + 2], ML[6 + c], fmaf(R[3 * a3 + 1], ML[3 + c], R[3 * a3] * ML[c])) + tp[a3] * gm[c];
          pose_g[9 + a3] += fmaf(R[3 * a3 + 2], gm[2], fmaf(R[3 * a3 + 1], gm[1], R[3 * a3] * gm[0]));
        }
      }
      if (slot == nullptr) {  // staged in the outputs' layout for the coalesced atomics below
        cg[3 * gi + 0] = gm[0];
        cg[3 * gi + 1] = gm[1];
        cg[3 * gi + 2] = gm[2];
#pragma unroll
        for (int i = 0; i < 6; ++i) cg[3 * K + 6 * gi + i] = gL[i];
        cg[9 * K + gi] = glam;
        if (color)
          for (int k3 = 0; k3 < 3; ++k3) cg[10 * K + 3 * gi + k3] = acc[19 + k3];
      } else {
        float* d = slot + NC * gi;
        d[0] = gm[0];
        d[1] = gm[1];
        d[2] = gm[2];
#pragma unroll
        for (int i = 0; i < 6; ++i) d[3 + i] = gL[i];
        d[9] = glam;
        if (color)
          for (int k3 = 0; k3 < 3; ++k3) d[10 + k3] = acc[19 + k3];
      }
    }

    if (slot == nullptr) {
      __syncthreads();
      const long long g0 = V.gauss_off;
      for (int i = tid; i < 3 * K; i += kAcThreads) atomicAdd(out.gmeans + 3 * g0 + i, cg[i]);
      for (int i = tid; i < 6 * K; i += kAcThreads) atomicAdd(out.gchol + 6 * g0 + i, cg[3 * K + i]);
      for (int i = tid; i < K; i += kAcThreads) atomicAdd(out.gweights + g0 + i, cg[9 * K + i]);
      if (color)
        for (int i = tid; i < 3 * K; i += kAcThreads) atomicAdd(out.gcolors + 3 * g0 + i, cg[10 * K + i]);
    }

    // ------------- phase D: pose gradient of this CTA
    if (want_pose) {
#pragma unroll
      for (int i = 0; i < 12; ++i) {
        const float x = warp_allsum(pose_g[i]);
        if (lane == 0) pose_gau[warp][i] = x;
      }
      __syncthreads();
      if (tid < NPV) {
        float x = 0.f;
        for (int w = 0; w < kAcWarps; ++w) x += pose_ray[w][tid] + (tid < 12 ? pose_gau[w][tid] : 0.f);
        if (slot != nullptr) {
          slot[NC * V.GB + tid] = x;
        } else {
          const int j = tid / 12 - 1;
          const int pidx = j < 0 ? V.pose : (j == 0 ? V.tgt0 : V.tgt1);
          if (pidx >= 0) atomicAdd(out.gposes + 12 * static_cast<long long>(pidx) + tid % 12, x);
        }
      }
    }
  }
}

// ------------------------------------------------------------------ launchers
template <int M>
static int ac_fwd_smem() {
  return 32 * M * kAcRecStride * 16 + kAcWarps * 3 * 32 * M * static_cast<int>(sizeof(float));
}

template <bool NORMALS, int NFLOW, int M>
static cudaError_t launch_fwd_ac_t(const Batch& b, const Scene& s, const Consts& c, const float4* records,
                                   const FwdOut& o, int run, int* status, int* counter, cudaStream_t st) {
  auto kern = forward_ac_kernel<NORMALS, NFLOW, M>;
  const int smem = ac_fwd_smem<M>();
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
  }
  int grid = b.n_items;
  if (counter) {
    int dev = 0, sms = 0, per = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kAcThreads, smem);
    grid = std::min(b.n_items, std::max(1, sms) * std::max(1, per));
  }
  return launch_kernel(kern, dim3(grid), dim3(kAcThreads), smem, st, 1, b, s, c, records, o, run, status, counter);
}

template <bool NORMALS, int NFLOW, int M>
static cudaError_t launch_bwd_ac_t(const Batch& b, const Scene& s, const Consts& c, const float4* records,
                                   const BwdIn& in, const BwdOut& out, int* status, int* counter, cudaStream_t st) {
  auto kern = in.order != nullptr ? backward_ac_kernel<NORMALS, NFLOW, M, true> : backward_ac_kernel<NORMALS, NFLOW, M, false>;
  const int smem = ac_bwd_smem_floats<M>() * static_cast<int>(sizeof(float));
  if (smem > 40 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
  }
  int grid = b.n_items;
  if (counter) {
    int dev = 0, sms = 0, per = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kAcThreads, smem);
    grid = std::min(b.n_items, std::max(1, sms) * std::max(1, per));
  }
  return launch_kernel(kern, dim3(grid), dim3(kAcThreads), smem, st, 1, b, s, c, records, in, out, status, counter);
}

template <int M>
static cudaError_t fwd_ac_m(const Batch& b, const Scene& s, const Consts& c, const float4* records, bool normals,
                            int n_flow, const FwdOut& o, int run, int* status, int* counter, cudaStream_t st) {
  if (normals) {
    if (n_flow == 0) return launch_fwd_ac_t<true, 0, M>(b, s, c, records, o, run, status, counter, st);
    if (n_flow == 1) return launch_fwd_ac_t<true, 1, M>(b, s, c, records, o, run, status, counter, st);
    return launch_fwd_ac_t<true, 2, M>(b, s, c, records, o, run, status, counter, st);
  }
  if (n_flow == 0) return launch_fwd_ac_t<false, 0, M>(b, s, c, records, o, run, status, counter, st);
  if (n_flow == 1) return launch_fwd_ac_t<false, 1, M>(b, s, c, records, o, run, status, counter, st);
  return launch_fwd_ac_t<false, 2, M>(b, s, c, records, o, run, status, counter, st);
}

template <int M>
static cudaError_t bwd_ac_m(const Batch& b, const Scene& s, const Consts& c, const float4* records, bool normals,
                            int n_flow, const BwdIn& in, const BwdOut& out, int* status, int* counter,
                            cudaStream_t st) {
  if (normals) {
    if (n_flow == 0) return launch_bwd_ac_t<true, 0, M>(b, s, c, records, in, out, status, counter, st);
    if (n_flow == 1) return launch_bwd_ac_t<true, 1, M>(b, s, c, records, in, out, status, counter, st);
    return launch_bwd_ac_t<true, 2, M>(b, s, c, records, in, out, status, counter, st);
  }
  if (n_flow == 0) return launch_bwd_ac_t<false, 0, M>(b, s, c, records, in, out, status, counter, st);
  if (n_flow == 1) return launch_bwd_ac_t<false, 1, M>(b, s, c, records, in, out, status, counter, st);
  return launch_bwd_ac_t<false, 2, M>(b, s, c, records, in, out, status, counter, st);
}

int ac_lanes_per_ray_elements(int maxK) { return maxK <= 64 ? 2 : (maxK <= 128 ? 4 : 8); }

cudaError_t launch_forward_ac(const Batch& b, const Scene& s, const Consts& c, const float4* records, bool normals,
                              int n_flow, int maxK, const FwdOut& o, int run, int* status, int* counter,
                              cudaStream_t st) {
  if (run < 1 || run > kAcMaxRun) return cudaErrorInvalidValue;
  switch (ac_lanes_per_ray_elements(maxK)) {
    case 2: return fwd_ac_m<2>(b, s, c, records, normals, n_flow, o, run, status, counter, st);
    case 4: return fwd_ac_m<4>(b, s, c, records, normals, n_flow, o, run, status, counter, st);
    default: return fwd_ac_m<8>(b, s, c, records, normals, n_flow, o, run, status, counter, st);
  }
}

cudaError_t launch_backward_ac(const Batch& b, const Scene& s, const Consts& c, const float4* records, bool normals,
                               int n_flow, int maxK, const BwdIn& in, const BwdOut& out, int* status, int* counter,
                               cudaStream_t st) {
  switch (ac_lanes_per_ray_elements(maxK)) {
    case 2: return bwd_ac_m<2>(b, s, c, records, normals, n_flow, in, out, status, counter, st);
    case 4: return bwd_ac_m<4>(b, s, c, records, normals, n_flow, in, out, status, counter, st);
    default: return bwd_ac_m<8>(b, s, c, records, normals, n_flow, in, out, status, counter, st);
  }
}

}  // namespace fmb
