// fmb_internal.cuh -- device-side structures and PTX helpers shared by the CUDA
// translation units of libfmb (forward, backward, C ABI).  Nothing here is part
// of the public ABI (include/fmb.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/fmb.h"

namespace fmb {

// Views per kernel launch.  The view table travels as a kernel parameter (a
// __grid_constant__ struct), so launches need no host->device copy and can be
// captured in CUDA graphs.  Two table sizes: up to 64 views (about 7 KB) for most
// calls, and up to 256 views (30 KB, within the 32 KB of kernel parameters of sm_90
// and later) for the two-parameter render and adjoint kernels of a call with more
// than 64 views, which then run as one launch per pass.  A graph launch costs the
// same with either block (measured on the GB300: 1.12-1.16 us per launch from 256
// bytes to 30 KB); an eager launch does not, since the host marshals the block each
// time (per-view calls of a single 64x64 view were 6 % slower with the 30 KB table),
// hence the small table wherever it suffices.
#ifndef FMB_MAX_BATCH_VIEWS
#define FMB_MAX_BATCH_VIEWS 64
#endif
constexpr int kMaxBatchViews = FMB_MAX_BATCH_VIEWS;
constexpr int kMaxBigBatchViews = 256;

// Per (view, Gaussian) record written by the prologue, 64 bytes (4 x float4):
//   [L00 L10 L11 L20 | L21 L22 b0 b1 | b2 mh0 mh1 mh2 | nbl0 nbl1 nbl2 l2]
// m = mu - o (the mean relative to the view's camera centre o) is kept as an
// unevaluated float pair mh + ml (exact to about 2^-48 relative); b = L^T mh is the
// whitened mean used for the max-likelihood depth, nbl = -L^T ml the low part of
// the whitened mean, l2 = log2(lambda).
constexpr int kRecFloat4 = 4;
constexpr int kRecBytes = 16 * kRecFloat4;

// Backward per-ray record in shared memory, 64 bytes (4 x float4):
//   [v0 v1 v2 lse2 | Dbar KA C Nb0 | Nb1 Nb2 vl0 vl1 | vl2 0 0 0]
// (v + vl is the ray direction as an unevaluated float pair.)
constexpr int kRayRecFloat4 = 4;

// Device status word values (first int of the workspace).
constexpr int kDevOk = 0;
constexpr int kDevTimeout = 1;

// Lazy max-shift threshold of the forward's running log-sum-exp, in log2 units:
// the shift m is raised only when a new exponent exceeds it by more than this, so
// partial sums stay below K * 2^64 (far from fp32 overflow) and the shift changes
// rarely.
constexpr float kLazyShift = 64.0f;

// Time limit of every device-side wait, in nanoseconds.
constexpr unsigned long long kWaitLimitNs = 1000000000ull;

struct DevView {
  int W, H;
  float fx, fy, cx, cy;
  int pose, tgt0, tgt1;
  int K;           // Gaussians of the view's object
  int n_tiles;     // ray tiles of this view
  int n_gblocks;   // backward: Gaussian blocks
  int GB, S;       // backward: Gaussians per block, ray subgroups per CTA
  int slot_floats;      // floats per (tile, gblock) slot in deterministic mode
  int Kp;               // stored-intermediate mode: row length (K rounded up to a multiple of 4)
  int P;                // plane entries of the view: n_rays, or W * H
  int rt;               // backward: rays per tile of this view (0: the launch's ray tile)
  int gauss_off;        // first Gaussian of the object in means/chol/weights (< 2^31, checked on the host)
  int rec_off;          // first record (in records) of this view in the workspace (< 2^28, checked)
  long long pix_off;    // first pixel of this view in the planes
  long long part_off;   // backward deterministic mode: float offset of the view's first slot
  long long pair_off;   // stored-intermediate mode: first float of the view's [P][Kp] block
  const int* rays;      // ray batch: pixel index of each plane entry, or null (whole image)
};
static_assert(sizeof(DevView) == 112, "DevView layout");

// Pixel rendered by plane entry i of a view.
__device__ __forceinline__ int ray_pixel(const DevView& V, int i) { return V.rays ? __ldg(V.rays + i) : i; }

// A launch's views.  Work items (forward: one ray tile; backward: one ray tile x
// Gaussian block) are numbered view by view in `order_view` order -- the views
// sorted by decreasing cost per item -- so both the hardware's block dispatch and
// the persistent work queue take the most expensive items first.
template <int CAP>
struct BatchT {
  static constexpr int kCapacity = CAP;
  int n_views;
  int n_items;
  int order_view[CAP];       // views by decreasing cost per item
  int order_begin[CAP + 1];  // first item of order_view[j]
  DevView v[CAP];
};
using Batch = BatchT<kMaxBatchViews>;
using BigBatch = BatchT<kMaxBigBatchViews>;
// Leaves room below the 32 764-byte kernel-parameter limit for the other arguments.
static_assert(sizeof(BigBatch) <= 31 * 1024, "a batch table must fit the kernel parameter space");

// Constants folded from the parameters (log2 domain).
// With x = log2(delta) = K3 q + log2(lambda), the log2 weight of Eq. 7 is
// e2 = beta1 x + K2 t.
struct Consts {
  float K2;   // -(beta2 / eta) * log2(e) : coefficient of t in the log2 weight
  float K3;   // -0.5 * log2(e)           : coefficient of q in log2(delta)
  float beta1;
  float b2e;  // beta2 / eta
};

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Programmatic dependent launch (sm_90 and later).  Every kernel of the library is
// launched with programmatic stream serialisation (launch_kernel below) and starts
// with pdl_enter(): it first waits until the grids before it in the stream have
// completed and their memory is visible (griddepcontrol.wait), so its memory
// accesses are ordered exactly as without the attribute, and then allows the next
// kernel of the stream to be launched (griddepcontrol.launch_dependents).  That
// launch takes effect once every CTA of this grid has started, so the next
// kernel's CTAs are scheduled into the SMs this grid's last wave leaves idle and
// wait there, instead of being launched only after this grid has drained.  In a
// kernel launched without the attribute both instructions do nothing.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
// Thread-block clusters (CUDA runtime intrinsics): this CTA's rank in its
// cluster; a 16-byte store to the same shared-memory offset of CTA `rank` of the
// cluster (distributed shared memory); and a barrier of all threads of the cluster
// (arrive with release, wait with acquire), after which such stores are visible
// to every CTA of the cluster.
__device__ __forceinline__ uint32_t cluster_ctarank() { return __clusterRelativeBlockRank(); }
__device__ __forceinline__ void st_cluster_f4(float4* local, int rank, float4 v) {
  *static_cast<float4*>(__cluster_map_shared_rank(local, static_cast<unsigned>(rank))) = v;
}
__device__ __forceinline__ void cluster_sync() {
  __cluster_barrier_arrive();
  __cluster_barrier_wait();
}
__device__ __forceinline__ unsigned long long global_timer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// Makes mbarrier initialisation visible to the async (bulk-copy) proxy.
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// Bulk (non-tensor) copy global -> this CTA's shared memory, completion counted on
// `bar`.  dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for phase `parity` of `bar` to complete, for at most kWaitLimitNs.  On
// timeout records kDevTimeout in *status and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int* status) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_timer_ns();
  for (;;) {
    for (int i = 0; i < 256; ++i)
      if (mbar_try_wait(bar, parity)) return true;
    if (global_timer_ns() - t0 > kWaitLimitNs) {
      atomicExch(status, kDevTimeout);
      return false;
    }
  }
}

// ------------------------------------------------ error-free transformations
// (Knuth's TwoSum and the FMA-based TwoProduct; exact as long as the compiler
// neither reassociates nor contracts them, which nvcc does not do to additions.)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = fmaf(a, b, -p);
}
// x = -(R^T t)_k as an unevaluated pair hi + lo (the camera centre o_k).
__device__ __forceinline__ void camera_centre_dd(const float R[9], const float t[3], int k, float& hi, float& lo) {
  float p0, e0, p1, e1, p2, e2, s1, f1, s2, f2;
  two_prod(R[k], t[0], p0, e0);
  two_prod(R[3 + k], t[1], p1, e1);
  two_prod(R[6 + k], t[2], p2, e2);
  two_sum(p0, p1, s1, f1);
  two_sum(s1, p2, s2, f2);
  const float l = __fadd_rn(__fadd_rn(__fadd_rn(e0, e1), __fadd_rn(e2, f1)), f2);
  float h2, l2;
  two_sum(s2, l, h2, l2);  // renormalise
  hi = -h2;
  lo = -l2;
}

// Geometry of one ray/Gaussian pair (Eq. 2 with the max-likelihood depth):
//   a = L^T v, t = a.b / a.a, r = v t - m (world frame, with the ray v = v + vl and
//   m = mh + ml as exact float pairs), u = L^T r projected once more orthogonal to a.
// The residual is formed from the exact pairs, and the final projection
// removes the component t's fp32 rounding leaves along a, so u is accurate
// relative to |u| even when |u| << |b| (rays passing close to a distant
// Gaussian's centre), where u = t a - b in plain fp32 would lose ~|b|/|u| ulps.
struct PairGeom {
  float a0, a1, a2, inv, t, u0, u1, u2, q;
};
template <bool REFINE = true>  // REFINE: the second projection (see pair_geom2)
__device__ __forceinline__ PairGeom pair_geom(const float L[6], const float b[3], const float mh[3],
                                              const float nbl[3], float v0, float v1, float v2, float vl0,
                                              float vl1, float vl2) {
  PairGeom G;
  const float L00 = L[0], L10 = L[1], L11 = L[2], L20 = L[3], L21 = L[4], L22 = L[5];
  G.a0 = fmaf(L20, v2, fmaf(L10, v1, L00 * v0));
  G.a1 = fmaf(L21, v2, L11 * v1);
  G.a2 = L22 * v2;
  const float aa = fmaf(G.a2, G.a2, fmaf(G.a1, G.a1, G.a0 * G.a0));
  const float ab = fmaf(G.a2, b[2], fmaf(G.a1, b[1], G.a0 * b[0]));
  G.inv = rcp_approx(aa);
  G.t = ab * G.inv;
  const float r0 = fmaf(vl0, G.t, fmaf(v0, G.t, -mh[0]));
  const float r1 = fmaf(vl1, G.t, fmaf(v1, G.t, -mh[1]));
  const float r2 = fmaf(vl2, G.t, fmaf(v2, G.t, -mh[2]));
  float u0 = fmaf(L00, r0, fmaf(L10, r1, fmaf(L20, r2, nbl[0])));
  float u1 = fmaf(L11, r1, fmaf(L21, r2, nbl[1]));
  float u2 = fmaf(L22, r2, nbl[2]);
  if (REFINE) {
    const float k = fmaf(u2, G.a2, fmaf(u1, G.a1, u0 * G.a0)) * G.inv;
    G.u0 = fmaf(-k, G.a0, u0);
    G.u1 = fmaf(-k, G.a1, u1);
    G.u2 = fmaf(-k, G.a2, u2);
  } else {
    G.u0 = u0;
    G.u1 = u1;
    G.u2 = u2;
  }
  G.q = fmaf(G.u2, G.u2, fmaf(G.u1, G.u1, G.u0 * G.u0));
  return G;
}

struct GaussRec {
  float L[6], b[3], mh[3], nbl[3], l2;
};
__device__ __forceinline__ GaussRec unpack_rec(const float4& r0, const float4& r1, const float4& r2,
                                               const float4& r3) {
  GaussRec g;
  g.L[0] = r0.x; g.L[1] = r0.y; g.L[2] = r0.z; g.L[3] = r0.w; g.L[4] = r1.x; g.L[5] = r1.y;
  g.b[0] = r1.z; g.b[1] = r1.w; g.b[2] = r2.x;
  g.mh[0] = r2.y; g.mh[1] = r2.z; g.mh[2] = r2.w;
  g.nbl[0] = r3.x; g.nbl[1] = r3.y; g.nbl[2] = r3.z;
  g.l2 = r3.w;
  return g;
}

// View and view-local index of work item `item`.
template <class B>
__device__ __forceinline__ int find_item(const B& batch, int item, int& local) {
  int lo = 0, hi = batch.n_views - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (batch.order_begin[mid] <= item)
      lo = mid;
    else
      hi = mid - 1;
  }
  local = item - batch.order_begin[lo];
  return batch.order_view[lo];
}

// Work-item source of a CTA: its block index (grid mode), or successive pops of a
// shared counter (persistent mode, `counter` != null).  Returns -1 when done.
// Every thread of the CTA must call it; it synchronises the CTA.
__device__ __forceinline__ int next_item(int* counter, int round, int* s_item) {
  if (counter == nullptr) return round == 0 ? static_cast<int>(blockIdx.x) : -1;
  __syncthreads();  // the previous item is finished with s_item and shared memory
  if (threadIdx.x == 0) *s_item = atomicAdd(counter, 1);
  __syncthreads();
  return *s_item;
}

// Pixel-centre ray of pixel p as an unevaluated float pair: camera-frame unit
// direction vc (high part), world direction v + vl = R^T (c / |c|) with
// c = ((x + 1/2 - cx)/fx, (y + 1/2 - cy)/fy, 1), accurate to a few units of 2^-48.
// Uses error-free transformations and one Newton step for 1/|c| in pair
// arithmetic.
__device__ __forceinline__ void pixel_ray_dd(const DevView& V, const float* R, int p, float vc[3], float v[3],
                                             float vl[3], float pxy[2]) {
  const int y = p / V.W;
  const int x = p - y * V.W;
  pxy[0] = static_cast<float>(x) + 0.5f;
  pxy[1] = static_cast<float>(y) + 0.5f;
  float ch[2], cl[2];
  const float f[2] = {V.fx, V.fy};
  const float cc[2] = {V.cx, V.cy};
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    float dh, dl;
    two_sum(pxy[k], -cc[k], dh, dl);
    ch[k] = __fdiv_rn(dh, f[k]);
    const float rem = fmaf(-ch[k], f[k], dh);  // exact remainder of the division
    cl[k] = __fdiv_rn(__fadd_rn(rem, dl), f[k]);
  }
  // s = |c|^2 = c0^2 + c1^2 + 1 as sh + sl
  float p0, e0, p1, e1, s1, f1, sh, f2;
  two_prod(ch[0], ch[0], p0, e0);
  two_prod(ch[1], ch[1], p1, e1);
  two_sum(p0, p1, s1, f1);
  two_sum(s1, 1.0f, sh, f2);
  const float sl = __fadd_rn(__fadd_rn(__fadd_rn(e0, e1), __fadd_rn(f1, f2)),
                             2.0f * fmaf(ch[0], cl[0], __fmul_rn(ch[1], cl[1])));
  // rn = 1/sqrt(s): one Newton step from rsqrtf, residual 1 - s rn0^2 in pair arithmetic
  const float rn0 = rsqrtf(sh);
  float hh, hl, wh, wl;
  two_prod(rn0, rn0, hh, hl);
  two_prod(sh, hh, wh, wl);
  const float resid = __fsub_rn(__fsub_rn(1.0f, wh), __fadd_rn(wl, fmaf(sh, hl, __fmul_rn(sl, hh))));
  float rnh, rnl;
  two_sum(rn0, __fmul_rn(0.5f * rn0, resid), rnh, rnl);
  // vc = c * rn
  float vch[3], vcl[3];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    two_prod(ch[k], rnh, vch[k], vcl[k]);
    vcl[k] = __fadd_rn(vcl[k], fmaf(ch[k], rnl, __fmul_rn(cl[k], rnh)));
  }
  vch[2] = rnh;
  vcl[2] = rnl;
  // v = R^T vc
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    float q0, g0, q1, g1, q2, g2, t1, h1, t2, h2;
    two_prod(R[j], vch[0], q0, g0);
    two_prod(R[3 + j], vch[1], q1, g1);
    two_prod(R[6 + j], vch[2], q2, g2);
    two_sum(q0, q1, t1, h1);
    two_sum(t1, q2, t2, h2);
    float lo = __fadd_rn(__fadd_rn(__fadd_rn(g0, g1), __fadd_rn(g2, h1)), h2);
    lo = fmaf(R[j], vcl[0], fmaf(R[3 + j], vcl[1], fmaf(R[6 + j], vcl[2], lo)));
    two_sum(t2, lo, v[j], vl[j]);
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) vc[k] = vch[k];
}

// Pixel-centre ray of pixel p: camera-frame unit direction vc and world direction
// v = R^T vc (plain fp32).
__device__ __forceinline__ void pixel_ray(const DevView& V, const float* R, int p, float vc[3], float v[3],
                                          float pxy[2]) {
  const int y = p / V.W;
  const int x = p - y * V.W;
  pxy[0] = static_cast<float>(x) + 0.5f;
  pxy[1] = static_cast<float>(y) + 0.5f;
  const float c0 = (pxy[0] - V.cx) / V.fx;
  const float c1 = (pxy[1] - V.cy) / V.fy;
  const float rn = rsqrtf(fmaf(c0, c0, fmaf(c1, c1, 1.0f)));
  vc[0] = c0 * rn;
  vc[1] = c1 * rn;
  vc[2] = rn;
  v[0] = fmaf(R[6], vc[2], fmaf(R[3], vc[1], R[0] * vc[0]));
  v[1] = fmaf(R[7], vc[2], fmaf(R[4], vc[1], R[1] * vc[0]));
  v[2] = fmaf(R[8], vc[2], fmaf(R[5], vc[1], R[2] * vc[0]));
}

__device__ __forceinline__ void load_pose(const float* poses, int idx, float R[9], float t[3]) {
  const float* p = poses + 12 * static_cast<long long>(idx);
#pragma unroll
  for (int k = 0; k < 9; ++k) R[k] = __ldg(p + k);
#pragma unroll
  for (int k = 0; k < 3; ++k) t[k] = __ldg(p + 9 + k);
}

// ----------------------------------------------------------- launchers (host)
// Launches kern<<<grid, block, smem, st>>>(args...) with programmatic stream
// serialisation (see pdl_enter), as a thread-block cluster of cluster_x CTAs if
// cluster_x > 1.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_kernel(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                 unsigned cluster_x, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[2];
  unsigned n = 0;
  at[n].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[n].val.programmaticStreamSerializationAllowed = 1;
  ++n;
  if (cluster_x > 1) {
    at[n].id = cudaLaunchAttributeClusterDimension;
    at[n].val.clusterDim.x = cluster_x;
    at[n].val.clusterDim.y = 1;
    at[n].val.clusterDim.z = 1;
    ++n;
  }
  cfg.attrs = at;
  cfg.numAttrs = n;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

struct Scene {
  const float* means;
  const float* chol;
  const float* weights;
  const float* poses;
  const float* colors = nullptr;  // per-Gaussian RGB [G][3], or null
  float4* crec = nullptr;         // colour records (r, g, b, 0) per (view, Gaussian) in the workspace
};

// Float arrays to clear (null entries skipped).
struct ZeroJob {
  static constexpr int kMax = 7;
  float* ptr[kMax];
  long long n[kMax];
};

// status_to_clear / counter_to_clear: if not null, the prologue also zeroes them;
// so it does with every array of `zero` (if not null).
cudaError_t launch_prologue(const Batch& b, const Scene& s, const Consts& c, float4* records, int maxK,
                            int* status_to_clear, int* counter_to_clear, cudaStream_t st,
                            const ZeroJob* zero = nullptr);
cudaError_t launch_prologue(const BigBatch& b, const Scene& s, const Consts& c, float4* records, int maxK,
                            int* status_to_clear, int* counter_to_clear, cudaStream_t st,
                            const ZeroJob* zero = nullptr);
// counter: persistent mode's work counter (zeroed before the launch), or null for
// one CTA per work item.
struct FwdOut;
cudaError_t launch_forward(const Batch& b, const Scene& s, const Consts& c, const float4* records, bool normals,
                           int n_flow, int rpt, int maxK, const FwdOut& o, int* status, int* counter,
                           cudaStream_t st);
cudaError_t launch_forward(const BigBatch& b, const Scene& s, const Consts& c, const float4* records, bool normals,
                           int n_flow, int rpt, int maxK, const FwdOut& o, int* status, int* counter,
                           cudaStream_t st);
// Gaussian-split forward: the merge of the splits' partial sums (o.part) into the
// planes; work items of forward_merge_rays_per_item() rays, the split count in DevView::S.
int forward_merge_rays_per_item();
cudaError_t launch_forward_merge(const Batch& b, const Scene& s, bool normals, int n_flow, const FwdOut& o,
                                 cudaStream_t st);
cudaError_t launch_forward_merge(const BigBatch& b, const Scene& s, bool normals, int n_flow, const FwdOut& o,
                                 cudaStream_t st);

struct FwdOut {
  float* depth;
  float* alpha;
  float* normal;
  float* flow;
  float* saved;
  float* pairs;             // stored-intermediate mode: [t | e2 | delta] arrays, else null
  long long pair_stride;    // floats per array
  float* color = nullptr;   // colour plane [3][P_v] per view (colour mode)
  float* part = nullptr;    // Gaussian-split forward: per-ray partial sums, 8 floats per (ray, split)
  unsigned char* order = nullptr;  // alpha compositing, keep_order: [plane entry][32 M] sorted Gaussian indices
};

cudaError_t launch_zero(const ZeroJob& job, cudaStream_t st);

struct BwdOut {
  float* gmeans;
  float* gchol;
  float* gweights;
  float* gposes;  // may be null
  float* partials;  // deterministic mode: workspace region, else null
  float* gcolors = nullptr;  // colour mode: [G][3]
};
struct BwdIn {
  const float* depth;
  const float* normal;
  const float* saved;
  const float* g_depth;
  const float* g_alpha;
  const float* g_normal;
  const float* g_flow;
  const float* pairs;      // stored-intermediate mode: [t | e2 | delta] arrays, else null
  long long pair_stride;   // floats per array
  const float* color = nullptr;    // colour mode: the forward's colour plane
  const float* g_color = nullptr;  // colour mode: its upstream gradient (may be null)
  const unsigned char* order = nullptr;  // alpha compositing, keep_order: the forward's per-ray depth order
};
cudaError_t launch_backward(const Batch& b, const Scene& s, const Consts& c, const float4* records, bool normals,
                            int n_flow, int ray_tile, int threads, const BwdIn& in, const BwdOut& out,
                            int* counter, cudaStream_t st);
cudaError_t launch_backward(const BigBatch& b, const Scene& s, const Consts& c, const float4* records, bool normals,
                            int n_flow, int ray_tile, int threads, const BwdIn& in, const BwdOut& out,
                            int* counter, cudaStream_t st);
// Resident CTAs per SM of the render kernels for this configuration (persistent
// grid sizing).
int forward_ctas_per_sm(bool normals, int n_flow, int rpt, int maxK);
int backward_ctas_per_sm(bool normals, int n_flow, int ray_tile, int threads);
// Alpha-compositing variant (Sec. 3.3): work items are 32-ray tiles, K <= 256 per
// view (maxK: the batch's largest K).
int ac_rays_per_item();
int ac_lanes_per_ray_elements(int maxK);  // M: each lane holds M of the 32 M sort keys of a ray
int ac_fwd_run(long long total_rays, int sms);  // forward rays per warp for a batch of total_rays
int ac_fwd_rays_per_item(int run);
cudaError_t launch_forward_ac(const Batch& b, const Scene& s, const Consts& c, const float4* records, bool normals,
                              int n_flow, int maxK, const FwdOut& o, int run, int* status, int* counter,
                              cudaStream_t st);
cudaError_t launch_backward_ac(const Batch& b, const Scene& s, const Consts& c, const float4* records, bool normals,
                               int n_flow, int maxK, const BwdIn& in, const BwdOut& out, int* status, int* counter,
                               cudaStream_t st);
// Oriented point export (Sec. 6): two-parameter work items of points_rays_per_item()
// pixels; alpha-compositing items of ac_fwd_rays_per_item(ac_run) pixels.
int points_rays_per_item();
cudaError_t launch_points(const Batch& b, const Scene& s, const Consts& c, const float4* records, int variant,
                          int maxK, int ac_run, const float* depth, const float* saved, float* points, float* normal_tf,
                          float* normal_scr, float* quality, cudaStream_t st);
// Loss attribution (Sec. 8, Eq. 19).  Two-parameter model: work items of ray_tile
// rays x a block of GB Gaussians (the backward's blocking, two Gaussians per thread);
// threads <= kAtt2MaxThreads.
constexpr int kAtt2MaxThreads = 256;
int attribution2_ray_tile(int threads);
cudaError_t launch_attribution2(const Batch& b, const Scene& s, const Consts& c, const float4* records, int threads,
                                int ray_tile, const float* saved, const float* loss, float* out, cudaStream_t st);
// Alpha compositing: work items of attribution_rays_per_item() rays x one block of up
// to 256 Gaussians (32 x M, M from the batch's largest K).
int attribution_rays_per_item();
cudaError_t launch_attribution_ac(const Batch& b, const Scene& s, const Consts& c, const float4* records, int maxK,
                                  const float* loss, float* out, cudaStream_t st);
cudaError_t launch_backward_reduce(const Batch& b, int n_flow, long long n_gauss, int n_poses,
                                   const BwdOut& out, cudaStream_t st);
cudaError_t launch_backward_reduce(const BigBatch& b, int n_flow, long long n_gauss, int n_poses,
                                   const BwdOut& out, cudaStream_t st);

}  // namespace fmb
