// Optimiser step of the training loop (Sec. 3.2 "Optimizing 3D GS
// representations"; the paper names neither the optimiser nor the
// activations, so this is the 3DGS practice): Adam on unconstrained raw
// parameters
//   raw = (p, log s, q, log rho),   params = (p, exp(log s), q, exp(log rho)),
// the quaternion staying raw (the projection normalises it).  The gradient
// comes in with respect to params and is carried to raw by the chain rule
// (d/dlog s = s d/ds, d/dlog rho = rho d/drho).
#include <math.h>

#include "gem_internal.cuh"

namespace gem {

// Parameter group of entry m of a Gaussian: 0 centre, 1 scale, 2 rotation,
// 3 density.
__device__ __forceinline__ int group_of(int m) { return m < 3 ? 0 : (m < 6 ? 1 : (m < 10 ? 2 : 3)); }

__device__ __forceinline__ bool is_log(int m) { return (m >= 3 && m < 6) || m == 10; }

__global__ void __launch_bounds__(256) adam_step_kernel(AdamArgs a, int64_t n,
                                                        float *__restrict__ raw,
                                                        float *__restrict__ mo,
                                                        float *__restrict__ ve,
                                                        const float *__restrict__ grad,
                                                        float *__restrict__ params,
                                                        const float *__restrict__ iso) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int m = (int)(i % kNpar);
  const int64_t j = i / kNpar;
  float r = raw[i];
  if (iso && m >= 3 && m < 6) {
    // isotropic ablation: the scale is the given distance, not learnt
    r = logf(iso[j]);
    raw[i] = r;
    params[i] = iso[j];
    return;
  }
  const float p = is_log(m) ? expf(r) : r;
  float g = grad[i];
  if (is_log(m)) g *= p;
  if (!isfinite(g)) g = 0.f;
  const float mm = a.beta1 * mo[i] + (1.f - a.beta1) * g;
  const float vv = a.beta2 * ve[i] + (1.f - a.beta2) * g * g;
  mo[i] = mm;
  ve[i] = vv;
  const float mhat = mm * a.c1, vhat = vv * a.c2;
  r -= a.lr[group_of(m)] * mhat / (sqrtf(vhat) + a.eps);
  raw[i] = r;
  params[i] = is_log(m) ? expf(r) : r;
}

__global__ void __launch_bounds__(256) activate_kernel(int64_t n, const float *__restrict__ raw,
                                                       float *__restrict__ params) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int m = (int)(i % kNpar);
  params[i] = is_log(m) ? expf(raw[i]) : raw[i];
}

cudaError_t launch_adam(const AdamArgs &a, int64_t M, float *raw, float *m, float *v,
                        const float *grad, float *params, const float *iso, cudaStream_t st) {
  const int64_t n = M * kNpar;
  adam_step_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a, n, raw, m, v, grad, params,
                                                                iso);
  return cudaGetLastError();
}

cudaError_t launch_activate(int64_t M, const float *raw, float *params, cudaStream_t st) {
  const int64_t n = M * kNpar;
  activate_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, raw, params);
  return cudaGetLastError();
}

}  // namespace gem
