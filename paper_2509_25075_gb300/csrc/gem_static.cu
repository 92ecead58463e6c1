// gem_ctf_loss_static: the CTF + loss + adjoint step without any device
// allocation.
//
// Some callers cannot allocate device memory at the point where they need
// this step: code that runs inside a framework's memory pool with a fixed
// budget, a custom allocator that forbids cudaMalloc after start-up, or a
// runtime that must not synchronise the device (cudaMalloc and cudaFree can).
// For them this entry point keeps its scratch in file-scope device arrays of
// a fixed size, which exist on every GPU that loads the library until the
// process exits.  The caller still passes its own inputs and outputs.
//
// Limits: B * d * d <= 1,048,576 spectrum elements (8 MiB), at most 65,536
// loss partials (B * (d / 16 + 1)), d as for gem_create.
#include <math.h>

#include <mutex>

#include "gem.h"
#include "gem_internal.cuh"

namespace gem {
namespace {

constexpr int64_t kStaticSpectrum = 1 << 20;  // float2 elements
constexpr int64_t kStaticLoss = 1 << 16;      // doubles
constexpr int kStaticMaxD = 768;

// The arrays' names are host-side stand-ins in host code: their device
// addresses come from cudaGetSymbolAddress, once per device.
__device__ __align__(256) float2 g_spectrum[kStaticSpectrum];
__device__ __align__(256) double g_lossp[kStaticLoss];
__device__ __align__(256) float2 g_twiddle[kStaticMaxD];

struct StaticScratch {
  float2 *spectrum = nullptr;
  double *lossp = nullptr;
  float2 *twiddle = nullptr;
  bool ready = false;
};

constexpr int kMaxDevices = 64;
StaticScratch g_scratch[kMaxDevices];
std::mutex g_scratch_mu;

// Device addresses of the static arrays on the current device (looked up on
// the first call for that device and kept for the life of the process: a
// cudaDeviceReset, or anything else that tears down and re-creates the
// device's primary context, may load the module at other addresses, so the
// entry point must not be used across one).
cudaError_t static_scratch(int dev, StaticScratch &out) {
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  StaticScratch &s = g_scratch[dev];
  if (!s.ready) {
    cudaError_t e;
    if ((e = cudaGetSymbolAddress((void **)&s.spectrum, g_spectrum)) != cudaSuccess) return e;
    if ((e = cudaGetSymbolAddress((void **)&s.lossp, g_lossp)) != cudaSuccess) return e;
    if ((e = cudaGetSymbolAddress((void **)&s.twiddle, g_twiddle)) != cudaSuccess) return e;
    s.ready = true;
  }
  out = s;
  return cudaSuccess;
}

// tw[m] = e^{-2 pi i m / n}
__global__ void static_twiddle_kernel(float2 *__restrict__ tw, int n) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n) return;
  double s, c;
  sincospi(-2.0 * (double)m / (double)n, &s, &c);
  tw[m] = make_float2((float)c, (float)s);
}

bool static_d_ok(int d) {
  if (d < 16 || d > kStaticMaxD || d % 16 != 0) return false;
  int m = d;
  while (m % 2 == 0) m /= 2;
  while (m % 3 == 0) m /= 3;
  return m == 1;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace
}  // namespace gem

using namespace gem;

extern "C" int gem_ctf_loss_static(int32_t d, float apix, int32_t B, const float *proj,
                                   const float *ctf, const float *ctf_params,
                                   const float *images, float *pred, float *dproj,
                                   double *loss_img, double *loss, void *cuda_stream) {
  if (!static_d_ok(d) || !(apix > 0.f) || !isfinite(apix) || B < 1) return GEM_EINVAL;
  if (!proj || !images || (ctf == nullptr) == (ctf_params == nullptr)) return GEM_EINVAL;
  if (!aligned16(proj) || !aligned16(images) || !aligned16(pred) || !aligned16(dproj))
    return GEM_EINVAL;
  const int64_t nblk = (int64_t)ctf_partials(d);
  if ((int64_t)B * d * d > kStaticSpectrum || (int64_t)B * (nblk + 1) > kStaticLoss)
    return GEM_ECAPACITY;
  // an error left pending by the caller's own earlier work is reported and
  // left in place (peeked, not cleared); after this point any error is ours
  if (cudaPeekAtLastError() != cudaSuccess) return GEM_ECUDA;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GEM_ECUDA;
  StaticScratch s;
  if (static_scratch(dev, s) != cudaSuccess) return GEM_ECUDA;
  FftPlan plan;
  if (!fft_plan(d, plan)) return GEM_EINVAL;
  if (ctf_configure(d) != cudaSuccess) return GEM_ECUDA;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  static_twiddle_kernel<<<(d + 255) / 256, 256, 0, st>>>(s.twiddle, d);
  if (cudaGetLastError() != cudaSuccess) return GEM_ECUDA;
  if (launch_ctf_loss(d, B, apix, plan, s.twiddle, proj, ctf, ctf_params, images, s.spectrum,
                      s.lossp, pred, dproj, loss_img, loss, st) != cudaSuccess)
    return GEM_ECUDA;
  return GEM_OK;
}
