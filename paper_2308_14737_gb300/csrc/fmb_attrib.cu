// fmb_attrib.cu -- loss attribution for the splitting criterion of Sec. 8
// (Eq. 19): for every Gaussian i, the sum over a batch of rays j of the ray's loss
// L_j times the Gaussian's normalised weight w_ij / sum_k w_kj on that ray.
//
// Two-parameter model (attribution2_kernel): the weights come from the forward's
// saved log2 normaliser, w_ij / sum w = 2^(e2_ij - lse2_j), so the work has the
// backward's shape: a CTA takes one view, one tile of rays and one block of
// Gaussians; phase 1 packs the tile's rays with non-zero loss (in ray order) into
// shared-memory records, every value stored twice so that one 16-byte load gives
// two broadcast pairs; phase 2 gives each thread two Gaussians, one per lane of
// packed FP32x2 arithmetic, and accumulates L_j w_ij over its subgroup's rays in a
// register; phase 3 adds the subgroups and writes one atomic per Gaussian.
//
// Alpha compositing (attribution_kernel<M, true>): the weights need the depth
// order, so one warp re-renders one ray at a time with lane l holding the Gaussians
// e = m * 32 + l of the item's block (up to 32 M = 256); each lane keeps its
// Gaussians' sums in registers over the warp's rays, and the four warps add their
// sums in shared memory before one atomic per Gaussian.  Rays with zero loss are
// skipped in both kernels.
#include "fmb_ac.cuh"
#include "fmb_f32x2.cuh"
#include "fmb_internal.cuh"

namespace fmb {

constexpr int kAttRaysPerWarp = 32;
constexpr int kAttRays = kAttRaysPerWarp * kAcWarps;  // rays per work item

int attribution_rays_per_item() { return kAttRays; }

template <int M>
__global__ void __launch_bounds__(kAcThreads) attribution_kernel(const __grid_constant__ Batch batch, Scene s,
                                                                 Consts k, const float4* __restrict__ records,
                                                                 const float* __restrict__ loss, float* out) {
  pdl_enter();
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
  unsigned long long key[M];  // the last rendered ray's depth order
  for (int m = 0; m < M; ++m) key[m] = kNoKey;
  bool have_order = false;
  for (int rr = 0; rr < kAttRaysPerWarp; ++rr) {
    const int p = p0 + rr;
    if (p >= P) break;
    const float Lj = loss[off + p];
    if (Lj == 0.f) continue;  // warp-uniform
    float vc[3], v[3], vl[3], pxy[2];
    pixel_ray_dd(V, R, ray_pixel(V, p), vc, v, vl, pxy);
    float t[M], dl[M], n[M][3];
    float* sd = scratch[warp];
    const AcSums a = ac_render_ray<false, M, kRecFloat4>(rec, Kb, v, vl, k, lane, t, dl, n, sd, sd + 32 * M,
                                                         sd + 64 * M, key, have_order && V.rays == nullptr);
    have_order = true;
    const float c = a.W > 0.f ? Lj / a.W : 0.f;
#pragma unroll
    for (int m = 0; m < M; ++m) {
      const int e = (m << 5) | lane;
      if (e < Kb) acc[m] = fmaf(c, sd[32 * M + e], acc[m]);
    }
    __syncwarp();
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

// ------------------------------------------------------------ two-parameter model
constexpr int kAtt2Rec = 4;  // float4s per ray record
// [v0 v0 v1 v1 | v2 v2 -lse2 -lse2 | vl0 vl0 vl1 vl1 | vl2 vl2 L L]

int attribution2_ray_tile(int threads) { return 3 * threads; }

__global__ void __launch_bounds__(kAtt2MaxThreads) attribution2_kernel(const __grid_constant__ Batch batch, Scene s,
                                                                       Consts k, const float4* __restrict__ records,
                                                                       const float* __restrict__ saved,
                                                                       const float* __restrict__ loss, float* out,
                                                                       int ray_tile) {
  pdl_enter();
  extern __shared__ float4 asm_[];
  __shared__ int wtot[kAtt2MaxThreads / 32];
  int local;
  const int vi = find_item(batch, blockIdx.x, local);
  const DevView& V = batch.v[vi];
  const int tile = local / V.n_gblocks;
  const int gb = local - tile * V.n_gblocks;
  const int P = V.P;
  const long long off = V.pix_off;
  const int pix0 = tile * ray_tile;
  const int nr = min(ray_tile, P - pix0);
  const int tid = threadIdx.x, T = blockDim.x, lane = tid & 31, warp = tid >> 5;

  // phase 1: records of the tile's rays with non-zero loss, packed in ray order
  float R[9], tp[3];
  load_pose(s.poses, V.pose, R, tp);
  int n = 0;  // packed rays so far (block-uniform)
  for (int c0 = 0; c0 < nr; c0 += T) {
    const int r = c0 + tid;
    const int p = pix0 + r;
    const float Lj = r < nr ? loss[off + p] : 0.f;
    const bool keep = Lj != 0.f;
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    if (lane == 0) wtot[warp] = __popc(bal);
    __syncthreads();
    int base = n, tot = 0;
    for (int w = 0; w < T / 32; ++w) {
      base += w < warp ? wtot[w] : 0;
      tot += wtot[w];
    }
    if (keep) {
      const int slot = base + __popc(bal & ((1u << lane) - 1u));
      float vc[3], v[3], vl[3], pxy[2];
      pixel_ray_dd(V, R, ray_pixel(V, p), vc, v, vl, pxy);
      const float nl = -saved[3 * off + p];
      float4* q = asm_ + kAtt2Rec * slot;
      q[0] = make_float4(v[0], v[0], v[1], v[1]);
      q[1] = make_float4(v[2], v[2], nl, nl);
      q[2] = make_float4(vl[0], vl[0], vl[1], vl[1]);
      q[3] = make_float4(vl[2], vl[2], Lj, Lj);
    }
    n += tot;
    __syncthreads();  // wtot is rewritten by the next chunk; the records are complete
  }

  // phase 2: two Gaussians per thread, one per packed lane
  const int GB = V.GB, S = V.S;
  const int GB2 = (GB + 1) / 2;
  const int gl2 = tid % GB2, sg = tid / GB2;
  const int g0 = gb * GB + 2 * gl2;
  const bool has1 = 2 * gl2 + 1 < GB && g0 + 1 < V.K;
  const bool active = sg < S && 2 * gl2 < GB && g0 < V.K;
  f2 acc = dup(0.f);
  if (active) {
    const float4* rec = records + kRecFloat4 * (V.rec_off + g0);
    const GaussRec ga = unpack_rec(rec[0], rec[1], rec[2], rec[3]);
    const GaussRec gbr = has1 ? unpack_rec(rec[4], rec[5], rec[6], rec[7]) : ga;
    const GaussRec2 gr = pair_rec(ga, gbr);
    const f2 K2v = dup(k.K2), K3v = dup(k.K3), B1v = dup(k.beta1);
    const ulonglong2* rr = reinterpret_cast<const ulonglong2*>(asm_);
#pragma unroll 2
    for (int r = sg; r < n; r += S) {
      const ulonglong2 q0 = rr[kAtt2Rec * r], q1 = rr[kAtt2Rec * r + 1], q2 = rr[kAtt2Rec * r + 2],
                       q3 = rr[kAtt2Rec * r + 3];
      const PairGeom2 G = pair_geom2(gr, as_f2(q0.x), as_f2(q0.y), as_f2(q1.x), as_f2(q2.x), as_f2(q2.y),
                                     as_f2(q3.x));
      const f2 x = fma2(G.q, K3v, gr.l2);  // log2(delta)
      const f2 w = ex2_2(fma2(x, B1v, fma2(G.t, K2v, as_f2(q1.y))));
      acc = fma2(as_f2(q3.y), w, acc);
    }
  }
  __syncthreads();  // the records are dead; the shared memory holds the sums below

  // phase 3: add the subgroups, one atomic per Gaussian
  float* red = reinterpret_cast<float*>(asm_);
  if (active) {
    red[2 * tid] = lo(acc);
    red[2 * tid + 1] = hi(acc);
  }
  __syncthreads();
  for (int e = tid; e < GB; e += T) {
    const int gi = gb * GB + e;
    if (gi >= V.K) break;
    float x = 0.f;
    for (int g = 0; g < S; ++g) x += red[2 * (g * GB2 + (e >> 1)) + (e & 1)];
    if (x != 0.f) atomicAdd(out + V.gauss_off + gi, x);
  }
}

int attribution2_smem_bytes(int ray_tile, int threads) {
  const int rec = ray_tile * kAtt2Rec * static_cast<int>(sizeof(float4));
  const int red = 2 * threads * static_cast<int>(sizeof(float));
  return rec > red ? rec : red;
}

cudaError_t launch_attribution2(const Batch& b, const Scene& s, const Consts& c, const float4* records, int threads,
                                int ray_tile, const float* saved, const float* loss, float* out, cudaStream_t st) {
  if (threads < 32 || threads > kAtt2MaxThreads || threads % 32 != 0) return cudaErrorInvalidValue;
  const int smem = attribution2_smem_bytes(ray_tile, threads);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(attribution2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
  }
  return launch_kernel(attribution2_kernel, dim3(b.n_items), dim3(threads), smem, st, 1, b, s, c, records, saved, loss,
                       out, ray_tile);
}

cudaError_t launch_attribution_ac(const Batch& b, const Scene& s, const Consts& c, const float4* records, int maxK,
                                  const float* loss, float* out, cudaStream_t st) {
  const int M = maxK <= 64 ? 2 : (maxK <= 128 ? 4 : 8);
  const dim3 grid(b.n_items), block(kAcThreads);
  if (M == 2) return launch_kernel(attribution_kernel<2>, grid, block, 0, st, 1, b, s, c, records, loss, out);
  if (M == 4) return launch_kernel(attribution_kernel<4>, grid, block, 0, st, 1, b, s, c, records, loss, out);
  return launch_kernel(attribution_kernel<8>, grid, block, 0, st, 1, b, s, c, records, loss, out);
  return cudaGetLastError();
}

}  // namespace fmb
