// fmb_points.cu -- oriented point export (Sec. 6): the rendered point of every
// pixel with two normal estimates and a quality value, as input for a Poisson
// surface reconstruction.
//
//   point       p = o + v D, D the rendered depth (Eq. 3)
//   normal_tf   Eq. 17's per-Gaussian normal evaluated at the rendered depth D
//               instead of at the hit depth t_i -- n_i = Sigma_i^-1 (o + v D - mu_i)
//               / |.| -- blended by Eq. 3 with the variant's weights, renormalised
//               and turned to face the camera (at t_i every n_i is perpendicular to
//               the ray, so Eq. 17 itself gives no orientation)
//   normal_scr  Eq. 16: (p - p_x) x (p - p_y) / |.| from the rendered points of the
//               right and lower neighbour pixels (left / upper on the last column /
//               row), turned to face the camera
//   quality     max_i w_i / sum_j w_j, the direct-intersection quality Sec. 6
//               thresholds (typically at 0.9)
// All vectors in the world frame.  The pass reads the forward's depth and saved
// planes; the two-parameter weights come from the saved log2 normaliser
// (w_i / sum w = 2^(e2_i - lse2)), the alpha-compositing weights from a re-render
// of the ray (they need the depth order).
#include "fmb_ac.cuh"
#include "fmb_f32x2.cuh"
#include "fmb_internal.cuh"

namespace fmb {

constexpr int kPtsThreads = 128;

struct PtsOut {
  float* points;
  float* normal_tf;
  float* normal_scr;
  float* quality;
};

// Unit vector of (x, y, z), or 0; then negated if it points away from the camera
// (a positive component along the viewing ray v).
__device__ __forceinline__ void unit_facing(float& x, float& y, float& z, const float v[3]) {
  const float nn = sqrtf(fmaf(x, x, fmaf(y, y, z * z)));
  const float s = nn > 0.f ? 1.0f / nn : 0.f;
  x *= s;
  y *= s;
  z *= s;
  if (fmaf(x, v[0], fmaf(y, v[1], z * v[2])) > 0.f) {
    x = -x;
    y = -y;
    z = -z;
  }
}

// Per-Gaussian normal of Eq. 17 evaluated at depth D: g = L L^T (v D - m) with the
// ray and m = mu - o as float pairs (the same compensated residual as the hit
// geometry), returned unit length (0 for g = 0).
__device__ __forceinline__ void normal_at_depth(const GaussRec& g, const float v[3], const float vl[3], float D,
                                                float n[3]) {
  const float r0 = fmaf(vl[0], D, fmaf(v[0], D, -g.mh[0]));
  const float r1 = fmaf(vl[1], D, fmaf(v[1], D, -g.mh[1]));
  const float r2 = fmaf(vl[2], D, fmaf(v[2], D, -g.mh[2]));
  const float u0 = fmaf(g.L[0], r0, fmaf(g.L[1], r1, fmaf(g.L[3], r2, g.nbl[0])));
  const float u1 = fmaf(g.L[2], r1, fmaf(g.L[4], r2, g.nbl[1]));
  const float u2 = fmaf(g.L[5], r2, g.nbl[2]);
  const float g0 = g.L[0] * u0;
  const float g1 = fmaf(g.L[2], u1, g.L[1] * u0);
  const float g2 = fmaf(g.L[5], u2, fmaf(g.L[4], u1, g.L[3] * u0));
  const float gg = fmaf(g2, g2, fmaf(g1, g1, g0 * g0));
  const float rs = gg > 0.f ? rsqrt_approx(gg) : 0.f;
  n[0] = g0 * rs;
  n[1] = g1 * rs;
  n[2] = g2 * rs;
}

// Eq. 16 at pixel p of a view, from the depth plane (rendered points of p and of
// its horizontal and vertical neighbours).
__device__ __forceinline__ void screen_normal(const DevView& V, const float* R, const float o[3],
                                              const float* __restrict__ depth, int p, float ns[3]) {
  ns[0] = ns[1] = ns[2] = 0.f;
  if (V.W < 2 || V.H < 2) return;
  const int y = p / V.W, x = p - y * V.W;
  const int q[3] = {p, y * V.W + (x + 1 < V.W ? x + 1 : x - 1), (y + 1 < V.H ? y + 1 : y - 1) * V.W + x};
  float P[3][3], v0[3];
  for (int j = 0; j < 3; ++j) {
    float vc[3], v[3], pxy[2];
    pixel_ray(V, R, q[j], vc, v, pxy);
    const float D = depth[q[j]];
#pragma unroll
    for (int k = 0; k < 3; ++k) P[j][k] = fmaf(v[k], D, o[k]);
    if (j == 0) {
      v0[0] = v[0];
      v0[1] = v[1];
      v0[2] = v[2];
    }
  }
  float d0[3], d1[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    d0[k] = P[0][k] - P[1][k];
    d1[k] = P[0][k] - P[2][k];
  }
  ns[0] = fmaf(d0[1], d1[2], -d0[2] * d1[1]);
  ns[1] = fmaf(d0[2], d1[0], -d0[0] * d1[2]);
  ns[2] = fmaf(d0[0], d1[1], -d0[1] * d1[0]);
  unit_facing(ns[0], ns[1], ns[2], v0);
}

__device__ __forceinline__ void store_vec(float* plane, long long off, int P, int p, const float a[3]) {
  if (plane == nullptr) return;
  float* b = plane + 3 * off;
  b[p] = a[0];
  b[P + p] = a[1];
  b[2 * P + p] = a[2];
}

// Two-parameter weights: two pixels per thread (p and p + 128 of a 256-pixel work
// item), one per lane of packed FP32x2 arithmetic, so every packed instruction
// serves both pixels' pair with the same Gaussian (each lane's weight is bitwise
// the scalar evaluation's; the normal sum folds the weight into the normalisation,
// w rs g).  Pixels past the end compute a clamped pixel and store nothing.
__global__ void __launch_bounds__(kPtsThreads) points_kernel(const __grid_constant__ Batch batch, Scene s, Consts k,
                                                             const float4* __restrict__ records,
                                                             const float* __restrict__ depth,
                                                             const float* __restrict__ saved, PtsOut out) {
  pdl_enter();
  int tile;
  const int vi = find_item(batch, blockIdx.x, tile);
  const DevView& V = batch.v[vi];
  const int P = V.P;
  const int pa = tile * (2 * kPtsThreads) + threadIdx.x;
  if (pa >= P) return;  // the second pixel (pa + 128) is then past the end too
  const int pb = pa + kPtsThreads;
  const bool has_b = pb < P;
  const int pbc = has_b ? pb : pa;
  const long long off = V.pix_off;
  float R[9], tp[3];
  load_pose(s.poses, V.pose, R, tp);
  const float o[3] = {-fmaf(R[6], tp[2], fmaf(R[3], tp[1], R[0] * tp[0])),
                      -fmaf(R[7], tp[2], fmaf(R[4], tp[1], R[1] * tp[0])),
                      -fmaf(R[8], tp[2], fmaf(R[5], tp[1], R[2] * tp[0]))};
  float vca[3], va[3], vla[3], pxya[2], vcb[3], vb[3], vlb[3], pxyb[2];
  pixel_ray_dd(V, R, ray_pixel(V, pa), vca, va, vla, pxya);
  pixel_ray_dd(V, R, ray_pixel(V, pbc), vcb, vb, vlb, pxyb);
  const float Da = depth[off + pa], Db = depth[off + pbc];
  const f2 v0 = pk(va[0], vb[0]), v1 = pk(va[1], vb[1]), v2 = pk(va[2], vb[2]);
  const f2 vl0 = pk(vla[0], vlb[0]), vl1 = pk(vla[1], vlb[1]), vl2 = pk(vla[2], vlb[2]);
  const f2 D = pk(Da, Db);
  const f2 nlse = pk(-saved[3 * off + pa], -saved[3 * off + pbc]);
  const f2 K2v = dup(k.K2), K3v = dup(k.K3), B1v = dup(k.beta1);
  const bool want_n = out.normal_tf != nullptr;
  const float4* rec = records + kRecFloat4 * V.rec_off;
  float qa = 0.f, qb = 0.f;
  f2 N0 = dup(0.f), N1 = dup(0.f), N2 = dup(0.f);
  for (int i = 0; i < V.K; ++i) {
    const GaussRec g1 = unpack_rec(__ldg(rec + 4 * i), __ldg(rec + 4 * i + 1), __ldg(rec + 4 * i + 2),
                                   __ldg(rec + 4 * i + 3));
    const GaussRec2 g = broadcast_rec(g1);
    const PairGeom2 G = pair_geom2(g, v0, v1, v2, vl0, vl1, vl2);
    const f2 x = fma2(G.q, K3v, g.l2);
    const f2 w = ex2_2(fma2(x, B1v, fma2(G.t, K2v, nlse)));  // w_i / sum w
    qa = fmaxf(qa, lo(w));
    qb = fmaxf(qb, hi(w));
    if (want_n) {
      // Eq. 17's normal at the rendered depth (the compensated residual at t = D)
      const f2 r0 = fma2(vl0, D, fma2(v0, D, g.nmh[0]));
      const f2 r1 = fma2(vl1, D, fma2(v1, D, g.nmh[1]));
      const f2 r2 = fma2(vl2, D, fma2(v2, D, g.nmh[2]));
      const f2 u0 = fma2(g.L[0], r0, fma2(g.L[1], r1, fma2(g.L[3], r2, g.nbl[0])));
      const f2 u1 = fma2(g.L[2], r1, fma2(g.L[4], r2, g.nbl[1]));
      const f2 u2 = fma2(g.L[5], r2, g.nbl[2]);
      const f2 gg0 = mul2(g.L[0], u0);
      const f2 gg1 = fma2(g.L[2], u1, mul2(g.L[1], u0));
      const f2 gg2 = fma2(g.L[5], u2, fma2(g.L[4], u1, mul2(g.L[3], u0)));
      const f2 gg = fma2(gg2, gg2, fma2(gg1, gg1, mul2(gg0, gg0)));
      const f2 rs = pk(lo(gg) > 0.f ? rsqrt_approx(lo(gg)) : 0.f, hi(gg) > 0.f ? rsqrt_approx(hi(gg)) : 0.f);
      const f2 wr = mul2(w, rs);
      N0 = fma2(wr, gg0, N0);
      N1 = fma2(wr, gg1, N1);
      N2 = fma2(wr, gg2, N2);
    }
  }
  const float* vv[2] = {va, vb};
  const float Dv[2] = {Da, Db}, qv[2] = {qa, qb};
  const int pp[2] = {pa, pb};
  const float Nl[2][3] = {{lo(N0), lo(N1), lo(N2)}, {hi(N0), hi(N1), hi(N2)}};
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    if (h == 1 && !has_b) break;
    const float* v = vv[h];
    float N[3] = {Nl[h][0], Nl[h][1], Nl[h][2]};
    unit_facing(N[0], N[1], N[2], v);
    const float pt[3] = {fmaf(v[0], Dv[h], o[0]), fmaf(v[1], Dv[h], o[1]), fmaf(v[2], Dv[h], o[2])};
    store_vec(out.points, off, P, pp[h], pt);
    store_vec(out.normal_tf, off, P, pp[h], N);
    if (out.quality) out.quality[off + pp[h]] = qv[h];
    if (out.normal_scr) {
      float ns[3];
      screen_normal(V, R, o, depth + off, pp[h], ns);
      store_vec(out.normal_scr, off, P, pp[h], ns);
    }
  }
}

// Alpha-compositing weights: one warp per pixel (the weights need the depth order);
// a work item is 4 runs of `run` neighbouring pixels, one run per warp, each pixel
// starting from the previous one's depth order (the forward's run length).
template <int M>
__global__ void __launch_bounds__(kAcThreads) points_ac_kernel(const __grid_constant__ Batch batch, Scene s,
                                                               Consts k, const float4* __restrict__ records,
                                                               const float* __restrict__ depth, PtsOut out,
                                                               int run) {
  pdl_enter();
  __shared__ float scratch[kAcWarps][3 * 32 * M];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int tile;
  const int vi = find_item(batch, blockIdx.x, tile);
  const DevView& V = batch.v[vi];
  const int P = V.P;
  const long long off = V.pix_off;
  float R[9], tp[3];
  load_pose(s.poses, V.pose, R, tp);
  const float o[3] = {-fmaf(R[6], tp[2], fmaf(R[3], tp[1], R[0] * tp[0])),
                      -fmaf(R[7], tp[2], fmaf(R[4], tp[1], R[1] * tp[0])),
                      -fmaf(R[8], tp[2], fmaf(R[5], tp[1], R[2] * tp[0]))};
  const float4* rec = records + kRecFloat4 * V.rec_off;
  float* sd = scratch[warp];
  float* sw = sd + 32 * M;
  float* sT = sd + 64 * M;
  unsigned long long key[M];
  for (int m = 0; m < M; ++m) key[m] = kNoKey;
  for (int j = 0; j < run; ++j) {
    const int p = (tile * kAcWarps + warp) * run + j;  // a run of neighbouring rays: reuse the depth order
    if (p >= P) break;
    float vc[3], v[3], vl[3], pxy[2];
    pixel_ray_dd(V, R, ray_pixel(V, p), vc, v, vl, pxy);
    float t[M], dl[M], n[M][3];
    const AcSums a = ac_render_ray<false, M, kRecFloat4>(rec, V.K, v, vl, k, lane, t, dl, n, sd, sw, sT, key,
                                                         j > 0 && V.rays == nullptr);
    const float D = depth[off + p];
    const float iW = a.W > 0.f ? 1.0f / a.W : 0.f;
    float qmax = 0.f, N[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int m = 0; m < M; ++m) {
      const int e = (m << 5) | lane;
      if (e < V.K) {
        const float w = sw[e] * iW;
        qmax = fmaxf(qmax, w);
        const GaussRec g = unpack_rec(__ldg(rec + 4 * e), __ldg(rec + 4 * e + 1), __ldg(rec + 4 * e + 2),
                                      __ldg(rec + 4 * e + 3));
        float ne[3];
        normal_at_depth(g, v, vl, D, ne);
        N[0] = fmaf(w, ne[0], N[0]);
        N[1] = fmaf(w, ne[1], N[1]);
        N[2] = fmaf(w, ne[2], N[2]);
      }
    }
#pragma unroll
    for (int o2 = 16; o2 > 0; o2 >>= 1) {
      qmax = fmaxf(qmax, __shfl_xor_sync(kFull, qmax, o2));
      N[0] += __shfl_xor_sync(kFull, N[0], o2);
      N[1] += __shfl_xor_sync(kFull, N[1], o2);
      N[2] += __shfl_xor_sync(kFull, N[2], o2);
    }
    if (lane == 0) {
      unit_facing(N[0], N[1], N[2], v);
      const float pt[3] = {fmaf(v[0], D, o[0]), fmaf(v[1], D, o[1]), fmaf(v[2], D, o[2])};
      store_vec(out.points, off, P, p, pt);
      store_vec(out.normal_tf, off, P, p, N);
      if (out.quality) out.quality[off + p] = qmax;
      if (out.normal_scr) {
        float ns[3];
        screen_normal(V, R, o, depth + off, p, ns);
        store_vec(out.normal_scr, off, P, p, ns);
      }
    }
    __syncwarp();
  }
}

int points_rays_per_item() { return 2 * kPtsThreads; }

cudaError_t launch_points(const Batch& b, const Scene& s, const Consts& c, const float4* records, int variant,
                          int maxK, int ac_run, const float* depth, const float* saved, float* points, float* normal_tf,
                          float* normal_scr, float* quality, cudaStream_t st) {
  const PtsOut o{points, normal_tf, normal_scr, quality};
  if (variant == 1) {
    const int M = maxK <= 64 ? 2 : (maxK <= 128 ? 4 : 8);
    if (ac_run < 1 || ac_run > kAcMaxRun) return cudaErrorInvalidValue;
    const dim3 grid(b.n_items), block(kAcThreads);
    if (M == 2) return launch_kernel(points_ac_kernel<2>, grid, block, 0, st, 1, b, s, c, records, depth, o, ac_run);
    if (M == 4) return launch_kernel(points_ac_kernel<4>, grid, block, 0, st, 1, b, s, c, records, depth, o, ac_run);
    return launch_kernel(points_ac_kernel<8>, grid, block, 0, st, 1, b, s, c, records, depth, o, ac_run);
  }
  return launch_kernel(points_kernel, dim3(b.n_items), dim3(kPtsThreads), 0, st, 1, b, s, c, records, depth, saved, o);
}

}  // namespace fmb
