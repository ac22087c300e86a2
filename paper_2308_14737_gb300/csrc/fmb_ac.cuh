// fmb_ac.cuh -- device helpers of the alpha-compositing variant (Sec. 3.3,
// Eq. 9-10), shared by its render, adjoint and point-export kernels: one warp per
// ray, a bitonic network over the warp's 32 M keys (t's order-preserving integer
// image in the high word, the Gaussian index in the low word), run-aware prefix
// sums of delta for the transmittance.
#pragma once

#include "fmb_internal.cuh"

namespace fmb {


constexpr int kAcWarps = 4;
constexpr int kAcThreads = 32 * kAcWarps;
constexpr int kAcRays = 32;          // rays per backward / export work item (8 per warp)
constexpr int kAcMaxRun = 32;        // longest forward run of neighbouring rays per warp
constexpr int kAcRayRec = 7;         // backward per-ray record, float4s (values duplicated)
// Gaussian records staged in shared memory every 5 float4s (80 bytes) instead of 4:
// lane l reads record 32 m + l, and with a 64-byte stride the 16-byte loads of
// eight neighbouring lanes fall into two of the eight 16-byte bank groups (a
// four-way conflict per quarter warp); with 80 bytes they fall into all eight.
constexpr int kAcRecStride = 5;
constexpr unsigned kFull = 0xffffffffu;
constexpr float kLog2e = 1.4426950408889634f;
constexpr unsigned long long kNoKey = ~0ull;

// Order-preserving map of a float to an unsigned integer (and back).
__device__ __forceinline__ unsigned order_bits(float t) {
  const unsigned u = __float_as_uint(t);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float from_order_bits(unsigned u) {
  return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// 1 - e^-x for x >= 0 without cancellation: the Maclaurin series for small x
// (relative truncation error below x^7 / 8! < 2e-9 for x < 1/4), else 1 - 2^(-x log2 e).
__device__ __forceinline__ float one_minus_exp_neg(float x) {
  const float series =
      x * (1.f - x * 0.5f * (1.f - x * (1.f / 3.f) * (1.f - x * 0.25f * (1.f - x * 0.2f * (1.f - x * (1.f / 6.f) *
                                                                                          (1.f - x * (1.f / 7.f)))))));
  return x < 0.25f ? series : 1.f - ex2_approx(-x * kLog2e);
}

// Ascending bitonic sort of the warp's 32 M keys in a blocked layout: sorting
// position i = lane * M + m, so lane l ends up holding the consecutive sorted
// positions l M .. l M + M - 1.  Partners closer than M are registers of the same
// lane; the log2(32) x (log2(32) + 1) / 2 + ... steps whose partner is another lane
// exchange one key per register by shuffle.  (Which key starts where does not
// matter: the network sorts any input arrangement.)
template <int M>
__device__ __forceinline__ void warp_bitonic_sort(unsigned long long (&key)[M], int lane) {
  constexpr int N = 32 * M;
#pragma unroll
  for (int k = 2; k <= N; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      if (j < M) {  // partner in register m ^ j of the same lane
#pragma unroll
        for (int m = 0; m < M; ++m) {
          if ((m & j) == 0) {
            const int m2 = m | j;
            const bool up = (((lane * M) + m) & k) == 0;
            const unsigned long long a = key[m], b = key[m2];
            const bool swap = up ? (a > b) : (a < b);
            key[m] = swap ? b : a;
            key[m2] = swap ? a : b;
          }
        }
      } else {  // partner in lane ^ (j / M), same register
        const int jl = j / M;
        const bool lower = (lane & jl) == 0;
#pragma unroll
        for (int m = 0; m < M; ++m) {
          const unsigned long long other = __shfl_xor_sync(kFull, key[m], jl);
          const bool up = (((lane * M) + m) & k) == 0;
          const bool other_smaller = other < key[m];
          key[m] = ((lower == up) == other_smaller) ? other : key[m];
        }
      }
    }
  }
}

// Ascending odd-even transposition passes over the same blocked layout until no
// pair is out of order: cheap when the keys arrive nearly sorted -- the previous,
// neighbouring ray's depth order.  At most max_passes passes (32 M sort any input);
// returns whether the keys are sorted.  Rays that are not neighbours (the entries of
// a random ray batch) are sorted by the bitonic network instead: from an unrelated
// order the refinement needs up to 32 M passes.
template <int M>
__device__ __forceinline__ bool warp_refine_sort(unsigned long long (&key)[M], int lane, int max_passes) {
  for (int pass = 0; pass < max_passes; ++pass) {
    bool swapped = false;
#pragma unroll
    for (int m = 0; m + 1 < M; m += 2) {  // even pairs (lane M + m, lane M + m + 1), m even
      const unsigned long long a = key[m], b = key[m + 1];
      if (a > b) {
        key[m] = b;
        key[m + 1] = a;
        swapped = true;
      }
    }
#pragma unroll
    for (int m = 1; m + 1 < M; m += 2) {  // odd pairs inside the lane
      const unsigned long long a = key[m], b = key[m + 1];
      if (a > b) {
        key[m] = b;
        key[m + 1] = a;
        swapped = true;
      }
    }
    // odd pair across lanes: (lane M + M - 1, (lane + 1) M)
    const unsigned long long next_first = __shfl_down_sync(kFull, key[0], 1);
    const unsigned long long prev_last = __shfl_up_sync(kFull, key[M - 1], 1);
    if (lane < 31 && key[M - 1] > next_first) {
      key[M - 1] = next_first;
      swapped = true;
    }
    if (lane > 0 && prev_last > key[0]) {
      key[0] = prev_last;
      swapped = true;
    }
    if (!__any_sync(kFull, swapped)) return true;
  }
  return false;
}



__device__ __forceinline__ float warp_incl_sum(float x, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  return x;
}
__device__ __forceinline__ float warp_incl_max(float x, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x = fmaxf(x, y);
  }
  return x;
}
// Over each aligned group of four lanes (sub = lane & 3): the sum of x over the
// group's lanes before this one (0 for sub 0), added in lane order; and whether
// every lane of the group has b.
__device__ __forceinline__ float ac_excl4(float x, int sub) {
  const float x0 = __shfl_sync(kFull, x, 0, 4), x1 = __shfl_sync(kFull, x, 1, 4), x2 = __shfl_sync(kFull, x, 2, 4);
  const float s01 = x0 + x1;
  return sub == 0 ? 0.f : (sub == 1 ? x0 : (sub == 2 ? s01 : s01 + x2));
}
__device__ __forceinline__ bool ac_all4(bool b) {
  int v = b ? 1 : 0;
  v &= __shfl_xor_sync(kFull, v, 1, 4);
  v &= __shfl_xor_sync(kFull, v, 2, 4);
  return v != 0;
}
__device__ __forceinline__ float warp_allsum(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
  return x;
}

// One (ray, Gaussian) pair of the alpha-compositing render: the hit depth t (Eq. 2),
// the density delta (Eq. 4) and, with NORMALS, the unit normal of Eq. 17 (zero
// otherwise).  r: the Gaussian's record.  The forward's per-ray sort and the
// adjoint's per-ray phases (the warp re-render and the four-thread walk) all take a
// pair's depth from this function, so a depth order the forward kept is the order
// of the depths the adjoint recomputes.
struct AcPair {
  float t, dl, n[3];
};
template <bool NORMALS>
__device__ __forceinline__ AcPair ac_pair_eval(const float4* __restrict__ r, const float v[3], const float vl[3],
                                               const Consts& k) {
  const GaussRec g = unpack_rec(r[0], r[1], r[2], r[3]);
  const PairGeom G = pair_geom(g.L, g.b, g.mh, g.nbl, v[0], v[1], v[2], vl[0], vl[1], vl[2]);
  AcPair q;
  q.t = G.t;
  q.dl = ex2_approx(fmaf(G.q, k.K3, g.l2));  // delta (Eq. 4)
  q.n[0] = q.n[1] = q.n[2] = 0.f;
  if (NORMALS) {
    const float g0 = g.L[0] * G.u0;
    const float g1 = fmaf(g.L[2], G.u1, g.L[1] * G.u0);
    const float g2 = fmaf(g.L[5], G.u2, fmaf(g.L[4], G.u1, g.L[3] * G.u0));
    const float rs = rsqrt_approx(fmaxf(fmaf(g2, g2, fmaf(g1, g1, g0 * g0)), 1e-30f));
    q.n[0] = g0 * rs;
    q.n[1] = g1 * rs;
    q.n[2] = g2 * rs;
  }
  return q;
}

// One ray of the alpha-compositing render, by one warp.  Per lane, for its
// Gaussians e = m * 32 + lane: hit depth t[m], density dl[m], Eq. 17 normal n[m]
// (NORMALS).  sd / sw / sT: the warp's shared scratch, indexed by Gaussian (32 M
// floats each).  Leaves w_e in sw and T_e in sT, and returns the warp-uniform sums.
struct AcSums {
  float W, WT, WN0, WN1, WN2, Sd;
  float WC0 = 0.f, WC1 = 0.f, WC2 = 0.f;  // colour mode: sum w c
};

// rec: the records, RS float4s apart (kAcRecStride in shared memory, kRecFloat4 in
// global memory).
template <bool NORMALS, int M, int RS = kAcRecStride>
__device__ __forceinline__ AcSums ac_render_ray(const float4* __restrict__ rec, int K, const float v[3],
                                                const float vl[3], const Consts& k, int lane, float (&t)[M],
                                                float (&dl)[M], float (&n)[M][3], float* sd, float* sw, float* sT,
                                                unsigned long long (&key)[M], bool reuse_order,
                                                const float4* __restrict__ crec = nullptr) {
  // key: in, with reuse_order, the previous ray's sorted keys (their Gaussian
  // indices give the starting order); out, this ray's sorted keys.
  int prev[M];
#pragma unroll
  for (int m = 0; m < M; ++m) prev[m] = key[m] != kNoKey ? static_cast<int>(key[m] & 0xffffffffu) : -1;
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const int e = (m << 5) | lane;
    t[m] = 0.f;
    dl[m] = 0.f;
    n[m][0] = n[m][1] = n[m][2] = 0.f;
    key[m] = kNoKey;
    if (e < K) {
      const AcPair q = ac_pair_eval<NORMALS>(rec + RS * e, v, vl, k);
      t[m] = q.t;
      dl[m] = q.dl;
      n[m][0] = q.n[0];
      n[m][1] = q.n[1];
      n[m][2] = q.n[2];
      sd[e] = dl[m];
      sT[e] = q.t;  // for the reordering below (overwritten by T afterwards)
      key[m] = (static_cast<unsigned long long>(order_bits(q.t)) << 32) | static_cast<unsigned>(e);
    }
  }
  __syncwarp();
  if (reuse_order) {
    // start from the previous ray's order (sorting position lane M + m) and refine
#pragma unroll
    for (int m = 0; m < M; ++m)
      key[m] = prev[m] >= 0 ? (static_cast<unsigned long long>(order_bits(sT[prev[m]])) << 32) |
                                  static_cast<unsigned>(prev[m])
                            : kNoKey;
    __syncwarp();
    warp_refine_sort<M>(key, lane, 32 * M);  // 32 M passes sort any input
  } else {
    warp_bitonic_sort<M>(key, lane);
  }
  // Sorted order (lane holds positions lane M + m): exclusive prefix sums of
  // delta, run-aware (Eq. 10's strict <).
  float ts[M], ds[M];
  int idx[M];
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const bool valid = key[m] != kNoKey;
    idx[m] = valid ? static_cast<int>(key[m] & 0xffffffffu) : -1;
    ts[m] = valid ? from_order_bits(static_cast<unsigned>(key[m] >> 32)) : INFINITY;
    ds[m] = valid ? sd[idx[m]] : 0.f;
  }
  float lane_sum = 0.f;
  float lex[M];  // exclusive sums within the lane
#pragma unroll
  for (int m = 0; m < M; ++m) {
    lex[m] = lane_sum;
    lane_sum += ds[m];
  }
  const float incl_lane = warp_incl_sum(lane_sum, lane);
  const float before = incl_lane - lane_sum;  // sum over the lanes in front
  const float total = __shfl_sync(kFull, incl_lane, 31);
  float prev_t = __shfl_up_sync(kFull, ts[M - 1], 1);
  // The sums P never decrease, so the sum in front of a hit's run is the largest
  // P at a run start up to it.
  float lmax = 0.f;
  float Sl[M];
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const float P = before + lex[m];
    const bool start = (lane == 0 && m == 0) || ts[m] != (m == 0 ? prev_t : ts[m - 1]);
    if (start) lmax = fmaxf(lmax, P);
    Sl[m] = lmax;
  }
  const float pmax_incl = warp_incl_max(lmax, lane);
  float pmax = __shfl_up_sync(kFull, pmax_incl, 1);
  if (lane == 0) pmax = 0.f;
#pragma unroll
  for (int m = 0; m < M; ++m) {
    if (idx[m] >= 0) {
      const float T = ex2_approx(-fmaxf(Sl[m], pmax) * kLog2e);
      sT[idx[m]] = T;
      sw[idx[m]] = T * one_minus_exp_neg(ds[m]);
    }
  }
  __syncwarp();
  const float carry = total;
  AcSums r{0.f, 0.f, 0.f, 0.f, 0.f, carry};
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const int e = (m << 5) | lane;
    if (e < K) {
      const float w = sw[e];
      r.W += w;
      r.WT = fmaf(w, t[m], r.WT);
      if (NORMALS) {
        r.WN0 = fmaf(w, n[m][0], r.WN0);
        r.WN1 = fmaf(w, n[m][1], r.WN1);
        r.WN2 = fmaf(w, n[m][2], r.WN2);
      }
      if (crec != nullptr) {
        const float4 c = __ldg(crec + e);
        r.WC0 = fmaf(w, c.x, r.WC0);
        r.WC1 = fmaf(w, c.y, r.WC1);
        r.WC2 = fmaf(w, c.z, r.WC2);
      }
    }
  }
  r.W = warp_allsum(r.W);
  r.WT = warp_allsum(r.WT);
  if (NORMALS) {
    r.WN0 = warp_allsum(r.WN0);
    r.WN1 = warp_allsum(r.WN1);
    r.WN2 = warp_allsum(r.WN2);
  }
  if (crec != nullptr) {
    r.WC0 = warp_allsum(r.WC0);
    r.WC1 = warp_allsum(r.WC1);
    r.WC2 = warp_allsum(r.WC2);
  }
  return r;
}

// keep_order: a ray's depth order as the indices of its sorted Gaussians, 32 M
// bytes per plane entry (sorting position lane M + m at byte lane M + m; K <= 256
// so an index fits a byte; positions >= K are unused).  Each lane moves its M bytes
// with one M-byte access.
template <int M>
__device__ __forceinline__ void ac_store_order(unsigned char* row, const unsigned long long (&key)[M], int lane) {
  unsigned long long w = 0;
#pragma unroll
  for (int m = 0; m < M; ++m)
    if (key[m] != kNoKey) w |= static_cast<unsigned long long>(key[m] & 0xffu) << (8 * m);
  unsigned char* dst = row + lane * M;
  if (M == 2) *reinterpret_cast<unsigned short*>(dst) = static_cast<unsigned short>(w);
  if (M == 4) *reinterpret_cast<unsigned*>(dst) = static_cast<unsigned>(w);
  if (M == 8) *reinterpret_cast<unsigned long long*>(dst) = w;
}
// The stored order as start keys for ac_render_ray's refinement (Gaussian index in
// the low word; the high word is filled in there from the recomputed depths).
// Indices are masked to the warp's 32 M scratch entries: a no-op for an order a
// forward of the same batch stored (indices below K <= 32 M), and it keeps the
// shared-memory reads inside the warp's slice for any other bytes.
template <int M>
__device__ __forceinline__ void ac_load_order(const unsigned char* __restrict__ row, int K, int lane,
                                              unsigned long long (&key)[M]) {
  const unsigned char* src = row + lane * M;
  unsigned long long w = 0;
  if (M == 2) w = __ldg(reinterpret_cast<const unsigned short*>(src));
  if (M == 4) w = __ldg(reinterpret_cast<const unsigned*>(src));
  if (M == 8) w = __ldg(reinterpret_cast<const unsigned long long*>(src));
#pragma unroll
  for (int m = 0; m < M; ++m) key[m] = lane * M + m < K ? (w >> (8 * m)) & (32u * M - 1u) & 0xffu : kNoKey;
}

// Stages a view's K records into shared memory, kAcRecStride float4s apart, by
// the whole CTA (coalesced 16-byte loads), and makes them visible to all threads.
__device__ __forceinline__ void ac_stage_records(float4* dst, const float4* __restrict__ src, int K) {
  for (int i = threadIdx.x; i < kRecFloat4 * K; i += blockDim.x)
    dst[kAcRecStride * (i / kRecFloat4) + i % kRecFloat4] = __ldg(src + i);
  __syncthreads();
}

}  // namespace fmb
