// fmb_adam.cu -- one fused Adam step (Kingma & Ba) over a flat parameter buffer,
// the optimiser of the reconstruction loop (paper Sec. 4 uses Adam).  Entries from
// `positive_begin` on are positive parameters (the Gaussian weights lambda) and are
// updated in log space: the gradient is taken with respect to log(p) and the
// update is multiplicative, so they stay positive.  The step counter lives on the
// device so that a captured CUDA graph can be replayed step after step.
#include "fmb_internal.cuh"

namespace fmb {

__global__ void adam_kernel(float* __restrict__ param, const float* __restrict__ grad, float* __restrict__ m,
                            float* __restrict__ v, long long n, long long positive_begin, float lr, float b1,
                            float b2, float eps, const int* __restrict__ step) {
  pdl_enter();
  const int t = *step + 1;
  const float c1 = 1.0f - powf(b1, static_cast<float>(t));
  const float c2 = 1.0f - powf(b2, static_cast<float>(t));
  const float lr_t = lr * sqrtf(c2) / c1;
  const float eps_t = eps * sqrtf(c2);
  const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n; i += stride) {
    const bool positive = i >= positive_begin;
    const float p = param[i];
    const float g = positive ? grad[i] * p : grad[i];  // d/d log(p) for positive entries
    const float mi = fmaf(b1, m[i], (1.0f - b1) * g);
    const float vi = fmaf(b2, v[i], (1.0f - b2) * g * g);
    m[i] = mi;
    v[i] = vi;
    const float upd = lr_t * mi / (sqrtf(vi) + eps_t);
    param[i] = positive ? p * expf(-upd) : p - upd;
  }
}

__global__ void increment_kernel(int* step) {
  pdl_enter();
  *step += 1;
}

}  // namespace fmb

extern "C" fmb_status fmb_adam_step(const fmb_adam_params* p, float* param, const float* grad, float* m, float* v,
                                    long long n, long long positive_begin, int* step_counter, fmb_stream_t stream) {
  if (!p || !param || !grad || !m || !v || !step_counter || n < 1 || positive_begin < 0 || positive_begin > n)
    return FMB_ERR_INVALID_ARG;
  if (!(p->lr > 0.f) || !(p->beta1 >= 0.f && p->beta1 < 1.f) || !(p->beta2 >= 0.f && p->beta2 < 1.f) ||
      !(p->eps > 0.f))
    return FMB_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const long long blocks = (n + 255) / 256;
  cudaError_t e = fmb::launch_kernel(fmb::adam_kernel, dim3(static_cast<unsigned>(blocks < 4 * 152 ? blocks : 4 * 152)),
                                     dim3(256), 0, s, 1, param, grad, m, v, n, positive_begin, p->lr, p->beta1,
                                     p->beta2, p->eps, static_cast<const int*>(step_counter));
  if (e == cudaSuccess) e = fmb::launch_kernel(fmb::increment_kernel, dim3(1), dim3(1), 0, s, 1, step_counter);
  return e == cudaSuccess ? FMB_OK : FMB_ERR_CUDA;
}
