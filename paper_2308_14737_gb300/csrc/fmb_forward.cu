// fmb_forward.cu -- prologue (per view x Gaussian records) and forward render
// kernel of the two-parameter Fuzzy Metaballs renderer.
//
// Formulation (paper Eq. 2, 3, 4, 7, 8, 17; Sec. 5 flow), whitened per Gaussian:
// with Sigma^-1 = L L^T, a = L^T v and b = L^T (mu - o), the max-likelihood depth is
// t = a.b / a.a, the residual in the whitened frame is u = t a - b = L^T (o + v t - mu),
// q = u.u, d = -q/2 + ln(lambda), delta = e^d, and the weight exponent of Eq. 7 is
// e = beta1 d - (beta2/eta) t.  The local normal Sigma^-1 (o + v t - mu) of Eq. 17 is
// g = L u.  Everything is evaluated in the log2 domain so that the exponentials
// are single ex2 instructions.
#include <algorithm>

#include "fmb_f32x2.cuh"
#include "fmb_internal.cuh"

namespace fmb {

constexpr int kFwdThreads = 128;
constexpr int kChunk = 256;  // records per shared-memory stage (16 KB)

// ------------------------------------------------------------------ prologue
// One thread per (view, Gaussian): the record of unpack_rec.  The camera centre
// o = -R^T t and m = mu - o are formed as exact float pairs (error-free
// transformations), so that the per-pair residual can be evaluated to full fp32
// accuracy relative to its own size.  The same launch clears the arrays of `zero`
// (the backward's gradient outputs and status word, which its kernels then
// accumulate into), grid-stride over all its threads.
template <class B>
__global__ void __launch_bounds__(128) prologue_kernel(const __grid_constant__ B batch, Scene s, Consts k,
                                                        float4* __restrict__ records, int* status_to_clear,
                                                        int* counter_to_clear, ZeroJob zero) {
  pdl_enter();
  const DevView& V = batch.v[blockIdx.y];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0 && blockIdx.y == 0) {
    if (status_to_clear != nullptr) *status_to_clear = kDevOk;
    if (counter_to_clear != nullptr) *counter_to_clear = 0;
  }
  {
    const long long stride = static_cast<long long>(gridDim.x) * gridDim.y * blockDim.x;
    const long long j0 = (static_cast<long long>(blockIdx.y) * gridDim.x + blockIdx.x) * blockDim.x + threadIdx.x;
    for (int b = 0; b < ZeroJob::kMax; ++b) {
      if (zero.ptr[b] == nullptr) continue;
      for (long long j = j0; j < zero.n[b]; j += stride) zero.ptr[b][j] = 0.f;
    }
  }
  if (i >= V.K) return;
  float R[9], t[3];
  load_pose(s.poses, V.pose, R, t);
  const long long g = V.gauss_off + i;
  const float* L = s.chol + 6 * g;
  const float L00 = L[0], L10 = L[1], L11 = L[2], L20 = L[3], L21 = L[4], L22 = L[5];
  float mh[3], ml[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float oh, ol, sh, se;
    camera_centre_dd(R, t, c, oh, ol);
    two_sum(s.means[3 * g + c], -oh, sh, se);
    two_sum(sh, __fsub_rn(se, ol), mh[c], ml[c]);
  }
  const float b0 = fmaf(L20, mh[2], fmaf(L10, mh[1], L00 * mh[0]));
  const float b1 = fmaf(L21, mh[2], L11 * mh[1]);
  const float b2 = L22 * mh[2];
  const float nb0 = -fmaf(L20, ml[2], fmaf(L10, ml[1], L00 * ml[0]));
  const float nb1 = -fmaf(L21, ml[2], L11 * ml[1]);
  const float nb2 = -(L22 * ml[2]);
  const float l2 = log2f(s.weights[g]);
  float4* r = records + kRecFloat4 * (V.rec_off + i);
  r[0] = make_float4(L00, L10, L11, L20);
  r[1] = make_float4(L21, L22, b0, b1);
  r[2] = make_float4(b2, mh[0], mh[1], mh[2]);
  r[3] = make_float4(nb0, nb1, nb2, l2);
  if (s.crec != nullptr) {
    const float* c = s.colors + 3 * g;
    s.crec[V.rec_off + i] = make_float4(c[0], c[1], c[2], 0.f);
  }
  (void)k;
}

template <class B>
static cudaError_t launch_prologue_t(const B& b, const Scene& s, const Consts& c, float4* records, int maxK,
                                     int* status_to_clear, int* counter_to_clear, cudaStream_t st,
                                     const ZeroJob* zero) {
  dim3 grid((maxK + 127) / 128, b.n_views);
  return launch_kernel(prologue_kernel<B>, grid, dim3(128), 0, st, 1, b, s, c, records, status_to_clear,
                       counter_to_clear, zero != nullptr ? *zero : ZeroJob{});
}
cudaError_t launch_prologue(const Batch& b, const Scene& s, const Consts& c, float4* records, int maxK,
                            int* status_to_clear, int* counter_to_clear, cudaStream_t st, const ZeroJob* zero) {
  return launch_prologue_t(b, s, c, records, maxK, status_to_clear, counter_to_clear, st, zero);
}
cudaError_t launch_prologue(const BigBatch& b, const Scene& s, const Consts& c, float4* records, int maxK,
                            int* status_to_clear, int* counter_to_clear, cudaStream_t st, const ZeroJob* zero) {
  return launch_prologue_t(b, s, c, records, maxK, status_to_clear, counter_to_clear, st, zero);
}

// ------------------------------------------------------------------- forward
struct RayAcc {
  float v0, v1, v2;     // world ray direction (high part)
  float vl0, vl1, vl2;  // low part
  float m;           // running shift of the log2 weights
  float Sw, Swt, Sd;  // sum w, sum w t, sum delta
  float N0, N1, N2;   // sum w n
};

template <bool NORMALS>
__device__ __forceinline__ void fwd_pair(RayAcc& A, const GaussRec& g, const Consts& k) {
  const PairGeom G = pair_geom<NORMALS>(g.L, g.b, g.mh, g.nbl, A.v0, A.v1, A.v2, A.vl0, A.vl1, A.vl2);
  const float x = fmaf(G.q, k.K3, g.l2);  // log2(delta)
  A.Sd += ex2_approx(x);
  const float e2 = fmaf(x, k.beta1, G.t * k.K2);
  if (e2 > A.m + kLazyShift) {
    const float s = ex2_approx(A.m - e2);
    A.Sw *= s;
    A.Swt *= s;
    if (NORMALS) {
      A.N0 *= s;
      A.N1 *= s;
      A.N2 *= s;
    }
    A.m = e2;
  }
  const float w = ex2_approx(e2 - A.m);
  A.Sw += w;
  A.Swt = fmaf(w, G.t, A.Swt);
  if (NORMALS) {
    const float L00 = g.L[0], L10 = g.L[1], L11 = g.L[2], L20 = g.L[3], L21 = g.L[4], L22 = g.L[5];
    const float g0 = L00 * G.u0;
    const float g1 = fmaf(L11, G.u1, L10 * G.u0);
    const float g2 = fmaf(L22, G.u2, fmaf(L21, G.u1, L20 * G.u0));
    const float gg = fmaxf(fmaf(g2, g2, fmaf(g1, g1, g0 * g0)), 1e-30f);
    const float ws = w * rsqrt_approx(gg);
    A.N0 = fmaf(ws, g0, A.N0);
    A.N1 = fmaf(ws, g1, A.N1);
    A.N2 = fmaf(ws, g2, A.N2);
  }
}

// Two rays of one thread, packed lane-wise (lane 0 = even ray, lane 1 = odd ray).
struct RayAcc2 {
  f2 v0, v1, v2, vl0, vl1, vl2;
  f2 m, Sw, Swt, Sd, N0, N1, N2;
  f2 C0, C1, C2;  // colour mode: sum w c
};

// Per-pair values the stored-intermediate mode keeps for the backward: the hit
// depth t, the log2 weight e2 of Eq. 7 and the density delta of Eq. 4.
struct PairOut2 {
  f2 t, e2, delta;
};

template <bool NORMALS, bool COLOR = false>
__device__ __forceinline__ PairOut2 fwd_pair2(RayAcc2& A, const GaussRec2& g, f2 K2, f2 K3, f2 beta1, f2 tiny,
                                              float4 col = float4{}) {
  const PairGeom2 G = pair_geom2<NORMALS>(g, A.v0, A.v1, A.v2, A.vl0, A.vl1, A.vl2);
  const f2 x = fma2(G.q, K3, g.l2);  // log2(delta)
  const f2 delta = ex2_2(x);
  A.Sd = add2(A.Sd, delta);
  const f2 e2 = fma2(x, beta1, mul2(G.t, K2));
  f2 d = sub2(e2, A.m);
  if (fmaxf(lo(d), hi(d)) > kLazyShift) {  // rare: raise the shift of the lane(s) it no longer bounds
    float dl = lo(d), dh = hi(d), sl = 1.f, sh = 1.f, ml = lo(A.m), mh = hi(A.m);
    if (dl > kLazyShift) {
      sl = ex2_approx(-dl);
      ml = lo(e2);
      dl = 0.f;
    }
    if (dh > kLazyShift) {
      sh = ex2_approx(-dh);
      mh = hi(e2);
      dh = 0.f;
    }
    const f2 sc = pk(sl, sh);
    A.Sw = mul2(A.Sw, sc);
    A.Swt = mul2(A.Swt, sc);
    if (NORMALS) {
      A.N0 = mul2(A.N0, sc);
      A.N1 = mul2(A.N1, sc);
      A.N2 = mul2(A.N2, sc);
    }
    if (COLOR) {
      A.C0 = mul2(A.C0, sc);
      A.C1 = mul2(A.C1, sc);
      A.C2 = mul2(A.C2, sc);
    }
    A.m = pk(ml, mh);
    d = pk(dl, dh);
  }
  const f2 w = ex2_2(d);
  A.Sw = add2(A.Sw, w);
  A.Swt = fma2(w, G.t, A.Swt);
  if (COLOR) {
    A.C0 = fma2(w, dup(col.x), A.C0);
    A.C1 = fma2(w, dup(col.y), A.C1);
    A.C2 = fma2(w, dup(col.z), A.C2);
  }
  if (NORMALS) {
    const f2 g0 = mul2(g.L[0], G.u0);
    const f2 g1 = fma2(g.L[2], G.u1, mul2(g.L[1], G.u0));
    const f2 g2 = fma2(g.L[5], G.u2, fma2(g.L[4], G.u1, mul2(g.L[3], G.u0)));
    const f2 gg = add2(fma2(g2, g2, fma2(g1, g1, mul2(g0, g0))), tiny);
    const f2 ws = mul2(w, rsqrt_2(gg));
    A.N0 = fma2(ws, g0, A.N0);
    A.N1 = fma2(ws, g1, A.N1);
    A.N2 = fma2(ws, g2, A.N2);
  }
  return PairOut2{G.t, e2, delta};
}


// The accumulator of ray r of a thread (unpacked from its f32x2 lane when packed).
template <bool PACKED, int NA, int NP>
__device__ __forceinline__ RayAcc ray_acc_of(const RayAcc (&A)[NA], const RayAcc2 (&A2)[NP], int r) {
  if (!PACKED) return A[r];
  RayAcc a;
  const RayAcc2& b = A2[r / 2];
  const bool h = (r & 1) != 0;
  a.v0 = h ? hi(b.v0) : lo(b.v0);
  a.v1 = h ? hi(b.v1) : lo(b.v1);
  a.v2 = h ? hi(b.v2) : lo(b.v2);
  a.vl0 = a.vl1 = a.vl2 = 0.f;
  a.m = h ? hi(b.m) : lo(b.m);
  a.Sw = h ? hi(b.Sw) : lo(b.Sw);
  a.Swt = h ? hi(b.Swt) : lo(b.Swt);
  a.Sd = h ? hi(b.Sd) : lo(b.Sd);
  a.N0 = h ? hi(b.N0) : lo(b.N0);
  a.N1 = h ? hi(b.N1) : lo(b.N1);
  a.N2 = h ? hi(b.N2) : lo(b.N2);
  return a;
}

// Per-pixel epilogue (Eq. 3, Eq. 8, Sec. 5, Sec. 6) from a ray's sums: depth, alpha,
// the saved normalisers, the camera-frame unit normal and the flow to each target.
template <bool NORMALS, int NFLOW>
__device__ __forceinline__ void write_ray_outputs(const DevView& V, const float R[9], const float o[3],
                                                  const float (*Rj)[9], const float (*tj)[3], const bool* has_t,
                                                  const RayAcc& a, const float pxy[2], long long p,
                                                  const FwdOut& out) {
  const int P = V.P;
  const long long off = V.pix_off;
  const float iSw = 1.0f / a.Sw;
  const float D = a.Swt * iSw;
  out.depth[off + p] = D;
  out.alpha[off + p] = -expm1f(-a.Sd);
  float* sv = out.saved + 3 * off;
  sv[p] = a.m + log2f(a.Sw);
  sv[P + p] = a.Sd;
  if (NORMALS) {
    const float N0 = a.N0 * iSw, N1 = a.N1 * iSw, N2 = a.N2 * iSw;
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
    const float p0 = fmaf(a.v0, D, o[0]), p1 = fmaf(a.v1, D, o[1]), p2 = fmaf(a.v2, D, o[2]);
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

// Shared-memory stage: kChunk records (4 float4 each), then in colour mode their
// kChunk colour records (1 float4 each).
template <bool COLOR>
__host__ __device__ constexpr int fwd_stage_float4() {
  return kChunk * (kRecFloat4 + (COLOR ? 1 : 0));
}

// Minimum resident CTAs: 7 for the plain two-rays-per-thread kernels with normals and
// flow, whose default register allocation spills (one flow slot: 28 bytes at 72
// registers) or stops at 5 CTAs per SM (two flow slots: 96 registers); bounded they
// take 72 registers with 8 bytes of spill, and 70 with none (orbit forward 0.256 ->
// 0.252 ms).  0 leaves the others to the compiler: a bound made them slower.
template <bool NORMALS, int NFLOW, int RPT, bool STORE>
constexpr int fwd_min_blocks() {
  return (RPT == 2 && NORMALS && NFLOW > 0 && !STORE) ? 7 : 0;
}

template <bool NORMALS, int NFLOW, int RPT, bool STORE, bool COLOR = false, class B = Batch>
__global__ void __launch_bounds__(kFwdThreads, COLOR ? 0 : fwd_min_blocks<NORMALS, NFLOW, RPT, STORE>())
    forward_kernel(const __grid_constant__ B batch, Scene s,
                                                              Consts k, const float4* __restrict__ records,
                                                              FwdOut out, int* status, int* counter) {
  pdl_enter();
  extern __shared__ float4 fwd_smem[];  // 1 or 2 stages x kChunk records
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ int s_item;
  const int tid = threadIdx.x;
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  // Completed phases of each stage's barrier so far (their parity selects the next wait).
  unsigned uses0 = 0, uses1 = 0;

  for (int round = 0;; ++round) {
  const int item = next_item(counter, round, &s_item);
  if (item < 0 || item >= batch.n_items) break;
  int local;
  const int vi = find_item(batch, item, local);
  const DevView& V = batch.v[vi];
  const int P = V.P;
  // Gaussian split ks of n_gblocks (1 unless the batch is split): Gaussians
  // [ks GB, min(K, (ks + 1) GB)) of the view's object
  const int tile = local / V.n_gblocks;
  const int ks = local - tile * V.n_gblocks;
  const int kbeg = ks * V.GB;
  const int K = min(V.GB, V.K - kbeg);

  float R[9], tp[3];
  load_pose(s.poses, V.pose, R, tp);
  const float o0 = -fmaf(R[6], tp[2], fmaf(R[3], tp[1], R[0] * tp[0]));
  const float o1 = -fmaf(R[7], tp[2], fmaf(R[4], tp[1], R[1] * tp[0]));
  const float o2 = -fmaf(R[8], tp[2], fmaf(R[5], tp[1], R[2] * tp[0]));

  // Stage the first record chunks while the rays are set up.
  const float4* src = records + kRecFloat4 * (V.rec_off + kbeg);
  const int nchunks = (K + kChunk - 1) / kChunk;
  constexpr int SST = fwd_stage_float4<COLOR>();
  const float4* csrc = COLOR ? s.crec + V.rec_off + kbeg : nullptr;
  if (tid == 0) {
    for (int c = 0; c < 2 && c < nchunks; ++c) {
      const int n = min(kChunk, K - c * kChunk);
      mbar_arrive_expect_tx(&bars[c], n * 16u * (kRecFloat4 + (COLOR ? 1 : 0)));
      bulk_g2s(fwd_smem + c * SST, src + c * kChunk * kRecFloat4, n * 16u * kRecFloat4, &bars[c]);
      if (COLOR) bulk_g2s(fwd_smem + c * SST + kChunk * kRecFloat4, csrc + c * kChunk, n * 16u, &bars[c]);
    }
  }

  // RPT even: rays are processed as packed pairs (PACKED); RPT == 1: scalar.
  constexpr bool PACKED = (RPT % 2) == 0;
  constexpr int NA = PACKED ? 1 : RPT;
  constexpr int NP = PACKED ? RPT / 2 : 1;
  RayAcc A[NA];
  RayAcc2 A2[NP];
  int pix[RPT];
  float pxy[RPT][2];
  float vc[RPT][3];
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    int p = tile * (kFwdThreads * RPT) + r * kFwdThreads + tid;
    pix[r] = p;
    p = min(p, P - 1);  // rays past the end compute a valid pixel and store nothing
    float v[3], vl[3];
    pixel_ray_dd(V, R, ray_pixel(V, p), vc[r], v, vl, pxy[r]);
    if (!PACKED) {
      RayAcc& a = A[PACKED ? 0 : r];
      a.v0 = v[0];
      a.v1 = v[1];
      a.v2 = v[2];
      a.vl0 = vl[0];
      a.vl1 = vl[1];
      a.vl2 = vl[2];
      a.m = -INFINITY;
      a.Sw = a.Swt = a.Sd = 0.f;
      a.N0 = a.N1 = a.N2 = 0.f;
    } else {
      RayAcc2& a = A2[r / 2];
      if ((r & 1) == 0) {
        a.v0 = pk(v[0], 0.f); a.v1 = pk(v[1], 0.f); a.v2 = pk(v[2], 0.f);
        a.vl0 = pk(vl[0], 0.f); a.vl1 = pk(vl[1], 0.f); a.vl2 = pk(vl[2], 0.f);
      } else {
        a.v0 = pk(lo(a.v0), v[0]); a.v1 = pk(lo(a.v1), v[1]); a.v2 = pk(lo(a.v2), v[2]);
        a.vl0 = pk(lo(a.vl0), vl[0]); a.vl1 = pk(lo(a.vl1), vl[1]); a.vl2 = pk(lo(a.vl2), vl[2]);
      }
      a.m = dup(-INFINITY);
      a.Sw = a.Swt = a.Sd = dup(0.f);
      a.N0 = a.N1 = a.N2 = dup(0.f);
      a.C0 = a.C1 = a.C2 = dup(0.f);
    }
  }
  const f2 K2v = dup(k.K2), K3v = dup(k.K3), B1v = dup(k.beta1), tiny = dup(1e-30f);

  bool failed = false;
  for (int c = 0; c < nchunks; ++c) {
    const int stage = c & 1;
    const unsigned parity = ((stage == 0 ? uses0 : uses1) + (c >> 1)) & 1u;
    const bool ok = mbar_wait_bounded(&bars[stage], parity, status);
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    const int n = min(kChunk, K - c * kChunk);
    const float4* rec = fwd_smem + stage * SST;
    const float4* crs = rec + kChunk * kRecFloat4;  // colour mode: this stage's colour records
    if (STORE) {
      // Stored-intermediate mode (two rays per thread): the values of four
      // consecutive Gaussians are buffered and written as one 16-byte store per
      // ray and array into row p of the view's [pixel][Kp] block (Kp a multiple
      // of 4; the padding past K is written as zeros).
      const int p0 = pix[0], p1 = pix[1];
      for (int i0 = 0; i0 < n; i0 += 4) {
        float bt[2][4], be[2][4], bd[2][4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = i0 + u;
          if (i < n) {
            const GaussRec g = unpack_rec(rec[kRecFloat4 * i + 0], rec[kRecFloat4 * i + 1],
                                          rec[kRecFloat4 * i + 2], rec[kRecFloat4 * i + 3]);
            const PairOut2 po = fwd_pair2<NORMALS>(A2[0], broadcast_rec(g), K2v, K3v, B1v, tiny);
            bt[0][u] = lo(po.t), bt[1][u] = hi(po.t);
            be[0][u] = lo(po.e2), be[1][u] = hi(po.e2);
            bd[0][u] = lo(po.delta), bd[1][u] = hi(po.delta);
          } else {
            bt[0][u] = bt[1][u] = be[0][u] = be[1][u] = bd[0][u] = bd[1][u] = 0.f;
          }
        }
        const long long kk = static_cast<long long>(c) * kChunk + i0;
        float* base = out.pairs + V.pair_off + kk;
        const long long S2 = out.pair_stride;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int pp = h == 0 ? p0 : p1;
          if (pp >= P) continue;
          float* row = base + static_cast<long long>(pp) * V.Kp;
          *reinterpret_cast<float4*>(row) = make_float4(bt[h][0], bt[h][1], bt[h][2], bt[h][3]);
          *reinterpret_cast<float4*>(row + S2) = make_float4(be[h][0], be[h][1], be[h][2], be[h][3]);
          *reinterpret_cast<float4*>(row + 2 * S2) = make_float4(bd[h][0], bd[h][1], bd[h][2], bd[h][3]);
        }
      }
    } else {
#pragma unroll 2
      for (int i = 0; i < n; ++i) {
        const GaussRec g = unpack_rec(rec[kRecFloat4 * i + 0], rec[kRecFloat4 * i + 1], rec[kRecFloat4 * i + 2],
                                      rec[kRecFloat4 * i + 3]);
        if (PACKED) {
          const GaussRec2 g2 = broadcast_rec(g);
          const float4 col = COLOR ? crs[i] : float4{};
#pragma unroll
          for (int q = 0; q < NP; ++q) fwd_pair2<NORMALS, COLOR>(A2[q], g2, K2v, K3v, B1v, tiny, col);
        } else {
#pragma unroll
          for (int r = 0; r < NA; ++r) fwd_pair<NORMALS>(A[r], g, k);
        }
      }
    }
    __syncthreads();  // every thread is done with this stage before it is refilled
    if (tid == 0 && c + 2 < nchunks) {
      const int n2 = min(kChunk, K - (c + 2) * kChunk);
      mbar_arrive_expect_tx(&bars[stage], n2 * 16u * (kRecFloat4 + (COLOR ? 1 : 0)));
      if (COLOR)
        bulk_g2s(fwd_smem + stage * SST + kChunk * kRecFloat4, csrc + (c + 2) * kChunk, n2 * 16u, &bars[stage]);
      bulk_g2s(fwd_smem + stage * SST, src + (c + 2) * kChunk * kRecFloat4, n2 * 16u * kRecFloat4,
               &bars[stage]);
    }
  }
  if (failed) return;
  uses0 += (nchunks + 1) / 2;
  uses1 += nchunks / 2;

  if (V.n_gblocks > 1) {
    // Gaussian split: this split's partial sums for fwd_merge_kernel
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      if (pix[r] >= P) continue;
      const RayAcc a = ray_acc_of<PACKED, NA, NP>(A, A2, r);
      float4* q = reinterpret_cast<float4*>(out.part + V.part_off +
                                            8 * (static_cast<long long>(pix[r]) * V.n_gblocks + ks));
      q[0] = make_float4(a.m, a.Sw, a.Swt, a.Sd);
      q[1] = make_float4(a.N0, a.N1, a.N2, 0.f);
    }
    continue;
  }

  // Flow targets (uniform over the CTA).
  float Rj[NFLOW > 0 ? NFLOW : 1][9], tj[NFLOW > 0 ? NFLOW : 1][3];
  bool has_t[NFLOW > 0 ? NFLOW : 1];
#pragma unroll
  for (int j = 0; j < NFLOW; ++j) {
    const int tg = j == 0 ? V.tgt0 : V.tgt1;
    has_t[j] = tg >= 0;
    if (has_t[j]) load_pose(s.poses, tg, Rj[j], tj[j]);
  }

  const long long off = V.pix_off;
  const float o[3] = {o0, o1, o2};
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    if (pix[r] >= P) continue;
    const long long p = pix[r];
    const RayAcc a = ray_acc_of<PACKED, NA, NP>(A, A2, r);
    if (COLOR) {
      const float iSw = 1.0f / a.Sw;
      const RayAcc2& b = A2[r / 2];
      const bool h = (r & 1) != 0;
      float* col = out.color + 3 * off;
      col[p] = (h ? hi(b.C0) : lo(b.C0)) * iSw;
      col[P + p] = (h ? hi(b.C1) : lo(b.C1)) * iSw;
      col[2 * P + p] = (h ? hi(b.C2) : lo(b.C2)) * iSw;
    }
    write_ray_outputs<NORMALS, NFLOW>(V, R, o, Rj, tj, has_t, a, pxy[r], p, out);
  }
  (void)vc;
  }  // item loop
}

static int fwd_smem_bytes(int maxK, bool color = false) {
  const int stages = maxK > kChunk ? 2 : 1;  // a second stage only when K spans several chunks
  return stages * (color ? fwd_stage_float4<true>() : fwd_stage_float4<false>()) * static_cast<int>(sizeof(float4));
}

template <bool NORMALS, int NFLOW, int RPT>
static int fwd_ctas_per_sm_t(int maxK) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, forward_kernel<NORMALS, NFLOW, RPT, false>, kFwdThreads,
                                                    fwd_smem_bytes(maxK)) != cudaSuccess)
    return 1;
  return n > 0 ? n : 1;
}

template <bool NORMALS, int NFLOW, int RPT, bool STORE = false, bool COLOR = false, class B>
static cudaError_t launch_fwd_t(const B& b, const Scene& s, const Consts& c, const float4* records,
                                const FwdOut& o, int maxK, int* status, int* counter, cudaStream_t st) {
  auto kern = forward_kernel<NORMALS, NFLOW, RPT, STORE, COLOR, B>;
  const int smem = fwd_smem_bytes(maxK, COLOR);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
  }
  int grid = b.n_items;
  if (counter) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    grid = std::min(b.n_items, std::max(1, sms) * fwd_ctas_per_sm_t<NORMALS, NFLOW, RPT>(maxK));
  }
  return launch_kernel(kern, dim3(grid), dim3(kFwdThreads), smem, st, 1, b, s, c, records, o, status, counter);
}

template <bool NORMALS, int NFLOW, class B>
static cudaError_t launch_fwd_r(int rpt, const B& b, const Scene& s, const Consts& c, const float4* records,
                                const FwdOut& o, int maxK, int* status, int* counter, cudaStream_t st) {
  if (o.pairs != nullptr)  // stored-intermediate mode: two rays per thread only
    return launch_fwd_t<NORMALS, NFLOW, 2, true>(b, s, c, records, o, maxK, status, counter, st);
  if (o.color != nullptr)  // colour mode: two rays per thread only
    return launch_fwd_t<NORMALS, NFLOW, 2, false, true>(b, s, c, records, o, maxK, status, counter, st);
  switch (rpt) {
    case 1: return launch_fwd_t<NORMALS, NFLOW, 1>(b, s, c, records, o, maxK, status, counter, st);
    case 2: return launch_fwd_t<NORMALS, NFLOW, 2>(b, s, c, records, o, maxK, status, counter, st);
    default: return launch_fwd_t<NORMALS, NFLOW, 4>(b, s, c, records, o, maxK, status, counter, st);
  }
}

template <class B>
static cudaError_t launch_forward_t(const B& b, const Scene& s, const Consts& c, const float4* records,
                                    bool normals, int n_flow, int rpt, int maxK, const FwdOut& o, int* status,
                                    int* counter, cudaStream_t st) {
  if (normals) {
    if (n_flow == 0) return launch_fwd_r<true, 0>(rpt, b, s, c, records, o, maxK, status, counter, st);
    if (n_flow == 1) return launch_fwd_r<true, 1>(rpt, b, s, c, records, o, maxK, status, counter, st);
    return launch_fwd_r<true, 2>(rpt, b, s, c, records, o, maxK, status, counter, st);
  }
  if (n_flow == 0) return launch_fwd_r<false, 0>(rpt, b, s, c, records, o, maxK, status, counter, st);
  if (n_flow == 1) return launch_fwd_r<false, 1>(rpt, b, s, c, records, o, maxK, status, counter, st);
  return launch_fwd_r<false, 2>(rpt, b, s, c, records, o, maxK, status, counter, st);
}
cudaError_t launch_forward(const Batch& b, const Scene& s, const Consts& c, const float4* records, bool normals,
                           int n_flow, int rpt, int maxK, const FwdOut& o, int* status, int* counter,
                           cudaStream_t st) {
  return launch_forward_t(b, s, c, records, normals, n_flow, rpt, maxK, o, status, counter, st);
}
cudaError_t launch_forward(const BigBatch& b, const Scene& s, const Consts& c, const float4* records, bool normals,
                           int n_flow, int rpt, int maxK, const FwdOut& o, int* status, int* counter,
                           cudaStream_t st) {
  return launch_forward_t(b, s, c, records, normals, n_flow, rpt, maxK, o, status, counter, st);
}

int forward_rays_per_cta(int rpt) { return kFwdThreads * rpt; }

// ------------------------------------------------ merge of a Gaussian-split forward
// One thread per ray.  Each split left its max-shifted sums (m_s, Sw_s, Swt_s, Sd_s,
// N_s); brought to the largest shift m they add exactly like the terms of one pass:
// Sw = sum_s 2^(m_s - m) Sw_s (likewise Swt and N), Sd = sum_s Sd_s.  The epilogue
// then writes the planes as the unsplit forward does.
constexpr int kMergeThreads = 128;
int forward_merge_rays_per_item() { return kMergeThreads; }

template <bool NORMALS, int NFLOW, class B>
__global__ void __launch_bounds__(kMergeThreads) fwd_merge_kernel(const __grid_constant__ B batch, Scene s,
                                                                  FwdOut out) {
  pdl_enter();
  int local;
  const int vi = find_item(batch, blockIdx.x, local);
  const DevView& V = batch.v[vi];
  const int P = V.P;
  const long long p = static_cast<long long>(local) * kMergeThreads + threadIdx.x;
  if (p >= P) return;
  float R[9], tp[3];
  load_pose(s.poses, V.pose, R, tp);
  const float o[3] = {-fmaf(R[6], tp[2], fmaf(R[3], tp[1], R[0] * tp[0])),
                      -fmaf(R[7], tp[2], fmaf(R[4], tp[1], R[1] * tp[0])),
                      -fmaf(R[8], tp[2], fmaf(R[5], tp[1], R[2] * tp[0]))};
  float Rj[NFLOW > 0 ? NFLOW : 1][9], tj[NFLOW > 0 ? NFLOW : 1][3];
  bool has_t[NFLOW > 0 ? NFLOW : 1];
#pragma unroll
  for (int j = 0; j < NFLOW; ++j) {
    const int tg = j == 0 ? V.tgt0 : V.tgt1;
    has_t[j] = tg >= 0;
    if (has_t[j]) load_pose(s.poses, tg, Rj[j], tj[j]);
  }
  float vc[3], v[3], vl[3], pxy[2];
  pixel_ray_dd(V, R, ray_pixel(V, static_cast<int>(p)), vc, v, vl, pxy);
  const int S = V.S;  // splits of this view
  const float4* q = reinterpret_cast<const float4*>(out.part + V.part_off + 8 * p * S);
  float m = -INFINITY;
  for (int k = 0; k < S; ++k) m = fmaxf(m, q[2 * k].x);
  RayAcc a;
  a.v0 = v[0];
  a.v1 = v[1];
  a.v2 = v[2];
  a.vl0 = vl[0];
  a.vl1 = vl[1];
  a.vl2 = vl[2];
  a.m = m;
  a.Sw = a.Swt = a.Sd = a.N0 = a.N1 = a.N2 = 0.f;
  for (int k = 0; k < S; ++k) {
    const float4 q0 = q[2 * k], q1 = q[2 * k + 1];
    const float sc = ex2_approx(q0.x - m);
    a.Sw = fmaf(sc, q0.y, a.Sw);
    a.Swt = fmaf(sc, q0.z, a.Swt);
    a.Sd += q0.w;
    if (NORMALS) {
      a.N0 = fmaf(sc, q1.x, a.N0);
      a.N1 = fmaf(sc, q1.y, a.N1);
      a.N2 = fmaf(sc, q1.z, a.N2);
    }
  }
  write_ray_outputs<NORMALS, NFLOW>(V, R, o, Rj, tj, has_t, a, pxy, p, out);
}

template <class B>
static cudaError_t launch_forward_merge_t(const B& b, const Scene& s, bool normals, int n_flow, const FwdOut& o,
                                          cudaStream_t st) {
  if (b.n_items <= 0) return cudaSuccess;
  const dim3 grid(b.n_items), block(kMergeThreads);
  if (normals) {
    if (n_flow == 0) return launch_kernel(fwd_merge_kernel<true, 0, B>, grid, block, 0, st, 1, b, s, o);
    if (n_flow == 1) return launch_kernel(fwd_merge_kernel<true, 1, B>, grid, block, 0, st, 1, b, s, o);
    return launch_kernel(fwd_merge_kernel<true, 2, B>, grid, block, 0, st, 1, b, s, o);
  }
  if (n_flow == 0) return launch_kernel(fwd_merge_kernel<false, 0, B>, grid, block, 0, st, 1, b, s, o);
  if (n_flow == 1) return launch_kernel(fwd_merge_kernel<false, 1, B>, grid, block, 0, st, 1, b, s, o);
  return launch_kernel(fwd_merge_kernel<false, 2, B>, grid, block, 0, st, 1, b, s, o);
}
cudaError_t launch_forward_merge(const Batch& b, const Scene& s, bool normals, int n_flow, const FwdOut& o,
                                 cudaStream_t st) {
  return launch_forward_merge_t(b, s, normals, n_flow, o, st);
}
cudaError_t launch_forward_merge(const BigBatch& b, const Scene& s, bool normals, int n_flow, const FwdOut& o,
                                 cudaStream_t st) {
  return launch_forward_merge_t(b, s, normals, n_flow, o, st);
}

int forward_ctas_per_sm(bool normals, int n_flow, int rpt, int maxK) {
  (void)normals;
  (void)n_flow;
  switch (rpt) {
    case 1: return fwd_ctas_per_sm_t<true, 1, 1>(maxK);
    case 2: return fwd_ctas_per_sm_t<true, 1, 2>(maxK);
    default: return fwd_ctas_per_sm_t<true, 1, 4>(maxK);
  }
}

}  // namespace fmb
