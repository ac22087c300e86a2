// fmb_probe.cu -- ALU throughput probes: long runs of independent scalar FP32
// FMAs, packed FP32x2 FMAs, and MUFU ex2 / rcp / rsqrt approximations, so that the
// FP32-pipe and SFU peaks of the GPU that runs the renderer can be measured
// instead of assumed.  Each thread keeps 8 independent chains; every result is
// stored so that nothing is eliminated.
#include "fmb_internal.cuh"

namespace fmb {

__device__ __forceinline__ unsigned long long pk2(float a, float b) {
  unsigned long long r;
  asm("mov.b64 %0, {%1,%2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ float sum2(unsigned long long a) {
  float lo, hi;
  asm("mov.b64 {%0,%1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a));
  return lo + hi;
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b, unsigned long long c) {
  unsigned long long d;
  asm volatile("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

template <int KIND>
__global__ void __launch_bounds__(256) probe_kernel(float* __restrict__ out, int iters, float seed) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  float x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = seed + 1e-3f * (threadIdx.x + j);
  if (KIND == 0) {  // scalar FMA: 8 chains
    const float b = 0.999999f, c = 1e-7f;
    for (int i = 0; i < iters; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) x[j] = fmaf(x[j], b, c);
  } else if (KIND == 1) {  // packed FMA: 8 chains of 2 lanes
    unsigned long long y[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) y[j] = pk2(x[j], x[j] + 0.5f);
    const unsigned long long b = pk2(0.999999f, 0.999998f), c = pk2(1e-7f, 2e-7f);
    for (int i = 0; i < iters; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) y[j] = fma2(y[j], b, c);
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = sum2(y[j]);
  } else if (KIND == 2) {  // ex2.approx
    for (int i = 0; i < iters; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) x[j] = ex2_approx(x[j]) - 1.0f;
  } else if (KIND == 3) {  // rcp.approx (plus a constant, so that no two reciprocals cancel)
    for (int i = 0; i < iters; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) x[j] = rcp_approx(x[j]) + 0.25f;
  } else {  // rsqrt.approx
    for (int i = 0; i < iters; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) x[j] = rsqrt_approx(x[j]);
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += x[j];
  out[tid] = s;
}

}  // namespace fmb

// Probe kernel launch: kind 0 = FFMA, 1 = packed FFMA2, 2 = ex2, 3 = rcp, 4 = rsqrt.
// out: device buffer of blocks * 256 floats.  Each thread issues 8 * iters
// operations (FFMA2: 16 * iters FP32 FMAs).
extern "C" fmb_status fmb_probe_alu(int kind, int blocks, int iters, float* out, fmb_stream_t stream) {
  if (!out || blocks < 1 || iters < 1 || kind < 0 || kind > 4) return FMB_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  switch (kind) {
    case 0: fmb::probe_kernel<0><<<blocks, 256, 0, s>>>(out, iters, 1.0f); break;
    case 1: fmb::probe_kernel<1><<<blocks, 256, 0, s>>>(out, iters, 1.0f); break;
    case 2: fmb::probe_kernel<2><<<blocks, 256, 0, s>>>(out, iters, 0.5f); break;
    case 3: fmb::probe_kernel<3><<<blocks, 256, 0, s>>>(out, iters, 1.5f); break;
    default: fmb::probe_kernel<4><<<blocks, 256, 0, s>>>(out, iters, 1.5f); break;
  }
  return cudaGetLastError() == cudaSuccess ? FMB_OK : FMB_ERR_CUDA;
}
