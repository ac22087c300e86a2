// fmb_attrib.cu -- loss attribution for the splitting criterion of Sec. 8
// (Eq. 19): for every Gaussian i, the sum over a batch of rays j of the ray's loss
// L_j times the Gaussian's normalised weight w_ij / sum_k w_kj on that ray.
//
// One warp takes one ray at a time and lane l the Gaussians e = m * 32 + l of the
// work item's block (up to 32 M = 256), so each lane keeps its Gaussians' sums in
// registers over all the warp's rays; the four warps of a CTA then add their sums
// in shared memory and write one atomic per Gaussian.  Two-parameter weights come
// from the forward's saved log2 normaliser (w_ij / sum w = 2^(e2_ij - lse2_j));
// alpha-compositing weights from a re-render of the ray (they need the depth
// order).  Rays with zero loss are skipped.
#include "fmb_ac.cuh"
#include "fmb_internal.cuh"

namespace fmb {

constexpr int kAttRaysPerWarp = 32;
constexpr int kAttRays = kAttRaysPerWarp * kAcWarps;  // rays per work item

int attribution_rays_per_item() { return kAttRays; }

template <int M, bool AC>
__global__ void __launch_bounds__(kAcThreads) attribution_kernel(const __grid_constant__ Batch batch, Scene s,
                                                                 Consts k, const float4* __restrict__ records,
                                                                 const float* __restrict__ saved,
                                                                 const float* __restrict__ loss, float* out) {
  __shared__ float scratch[kAcWarps][3 * 32 * M];
  __shared__ float sums[kAcWarps][32 * M];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int local;
  const int vi = find_item(batch, blockIdx.x, local);
  const DevView& V = batch.v[vi];
  const int tile = local / V.n_gblocks;
  const int gb = local - tile * V.n_gblocks;
  const int P = V.P;
  const long long off = V.pix_off;
  const int g_begin = gb * 32 * M;
  const int Kb = min(32 * M, V.K - g_begin);  // Gaussians of this block
  float R[9], tp[3];
  load_pose(s.poses, V.pose, R, tp);
  const float4* rec = records + kRecFloat4 * (V.rec_off + g_begin);
  float acc[M];
#pragma unroll
  for (int m = 0; m < M; ++m) acc[m] = 0.f;
  const int p0 = tile * kAttRays + warp * kAttRaysPerWarp;
  unsigned long long key[M];  // alpha compositing: the last rendered ray's depth order
  for (int m = 0; m < M; ++m) key[m] = kNoKey;
  bool have_order = false;
  for (int rr = 0; rr < kAttRaysPerWarp; ++rr) {
    const int p = p0 + rr;
    if (p >= P) break;
    const float Lj = loss[off + p];
    if (Lj == 0.f) continue;  // warp-uniform
    float vc[3], v[3], vl[3], pxy[2];
    pixel_ray_dd(V, R, ray_pixel(V, p), vc, v, vl, pxy);
    if (AC) {
      float t[M], dl[M], n[M][3];
      float* sd = scratch[warp];
      const AcSums a = ac_render_ray<false, M>(rec, Kb, v, vl, k, lane, t, dl, n, sd, sd + 32 * M, sd + 64 * M,
                                               key, have_order);
      have_order = true;
      const float c = a.W > 0.f ? Lj / a.W : 0.f;
#pragma unroll
      for (int m = 0; m < M; ++m) {
        const int e = (m << 5) | lane;
        if (e < Kb) acc[m] = fmaf(c, sd[32 * M + e], acc[m]);
      }
      __syncwarp();
    } else {
      const float lse2 = saved[3 * off + p];
#pragma unroll
      for (int m = 0; m < M; ++m) {
        const int e = (m << 5) | lane;
        if (e < Kb) {
          const GaussRec g = unpack_rec(__ldg(rec + 4 * e), __ldg(rec + 4 * e + 1), __ldg(rec + 4 * e + 2),
                                        __ldg(rec + 4 * e + 3));
          const PairGeom G = pair_geom(g.L, g.b, g.mh, g.nbl, v[0], v[1], v[2], vl[0], vl[1], vl[2]);
          const float x = fmaf(G.q, k.K3, g.l2);
          acc[m] = fmaf(Lj, ex2_approx(fmaf(x, k.beta1, fmaf(G.t, k.K2, -lse2))), acc[m]);
        }
      }
    }
  }
#pragma unroll
  for (int m = 0; m < M; ++m) sums[warp][(m << 5) | lane] = acc[m];
  __syncthreads();
  for (int e = tid; e < Kb; e += kAcThreads) {
    float x = 0.f;
#pragma unroll
    for (int w = 0; w < kAcWarps; ++w) x += sums[w][e];
    if (x != 0.f) atomicAdd(out + V.gauss_off + g_begin + e, x);
  }
}

cudaError_t launch_attribution(const Batch& b, const Scene& s, const Consts& c, const float4* records, int variant,
                               int maxK, const float* saved, const float* loss, float* out, cudaStream_t st) {
  const int M = maxK <= 64 ? 2 : (maxK <= 128 ? 4 : 8);
  if (variant == 1) {
    if (M == 2) attribution_kernel<2, true><<<b.n_items, kAcThreads, 0, st>>>(b, s, c, records, saved, loss, out);
    else if (M == 4) attribution_kernel<4, true><<<b.n_items, kAcThreads, 0, st>>>(b, s, c, records, saved, loss, out);
    else attribution_kernel<8, true><<<b.n_items, kAcThreads, 0, st>>>(b, s, c, records, saved, loss, out);
  } else {
    if (M == 2) attribution_kernel<2, false><<<b.n_items, kAcThreads, 0, st>>>(b, s, c, records, saved, loss, out);
    else if (M == 4) attribution_kernel<4, false><<<b.n_items, kAcThreads, 0, st>>>(b, s, c, records, saved, loss, out);
    else attribution_kernel<8, false><<<b.n_items, kAcThreads, 0, st>>>(b, s, c, records, saved, loss, out);
  }
  return cudaGetLastError();
}

}  // namespace fmb
