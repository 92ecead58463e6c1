// Steps a3 (raster forward) and a5 (raster backward) of the GEM hot path,
// plus the plain dense forms used as the baseline.
//
// a3: Eq. render restricted by Eq. accu.  One CTA per (image, 16x16 tile);
//     128 threads, each owning two horizontally adjacent pixels; warp w owns
//     rows 4w..4w+3 of the tile.  The tile's list (depth order) is staged in
//     shared memory 128 records at a time; every thread adds the kept terms
//     of each record in list order.  A warp skips a record whose extent does
//     not reach its four rows.
// a5: the "efficient gradient" of Sec. 1 (iii) / Sec. 3.2: only pairs kept by
//     Eq. accu.  One CTA per (image, tile), one thread per listed Gaussian:
//     the thread walks the tile's pixels inside its Gaussian's row range and
//     accumulates six moments of g * value, which a6 turns into parameter
//     gradients; one set of atomics per (tile, Gaussian).
#include "gem_internal.cuh"

namespace gem {

constexpr int kFwdThreads = 128;
constexpr int kBwdThreads = 128;

// kCount = true: the same walk, counting kept pairs into *kept instead of
// writing the projection (inspection only, never on the timed path).
template <bool kCount>
__global__ void __launch_bounds__(kFwdThreads) raster_fwd_kernel(
    const Rec *__restrict__ rec, const uint32_t *__restrict__ list,
    const int64_t *__restrict__ tile_start, int64_t cap, int64_t M, int d, float l2tau,
    float *__restrict__ proj, unsigned long long *__restrict__ kept) {
  __shared__ float4 sa[kFwdThreads], sb[kFwdThreads];
  const int nt = d / kTile, T = nt * nt;
  const int t = blockIdx.x, b = blockIdx.y;
  const int tx = t % nt, ty = t / nt;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = 4 * warp + (lane >> 3);
  const int col = 2 * (lane & 7);
  const float X0 = (float)(tx * kTile + col), X1 = X0 + 1.f;
  const float Y = (float)(ty * kTile + row);
  const float ywlo = (float)(ty * kTile + 4 * warp), ywhi = ywlo + 3.f;
  int64_t s = tile_start[(int64_t)b * T + t];
  int64_t e = tile_start[(int64_t)b * T + t + 1];
  e = min(e, cap);
  s = min(s, e);
  const Rec *rb = rec + (int64_t)b * M;
  double acc0 = 0.0, acc1 = 0.0;
  unsigned nkept = 0;
  for (int64_t base = s; base < e; base += kFwdThreads) {
    int n = (int)min((int64_t)kFwdThreads, e - base);
    __syncthreads();
    if (threadIdx.x < n) {
      uint32_t j = list[base + threadIdx.x];
      Rec r = rb[j];
      sa[threadIdx.x] = r.a;
      sb[threadIdx.x] = r.b;
    }
    __syncthreads();
    float p0 = 0.f, p1 = 0.f;
#pragma unroll 4
    for (int k = 0; k < n; ++k) {
      const float4 A = sa[k];
      const float4 Bv = sb[k];
      // warp-uniform: does the record's row extent reach this warp's rows?
      if (A.y + Bv.w < ywlo || A.y - Bv.w > ywhi) continue;
      const float dy = Y - A.y;
      const float bdy = A.w * dy;
      const float cdy = fmaf(Bv.x * dy, dy, Bv.y);
      const float dx0 = X0 - A.x, dx1 = X1 - A.x;
      const float e0 = fmaf(fmaf(A.z, dx0, bdy), dx0, cdy);
      const float e1 = fmaf(fmaf(A.z, dx1, bdy), dx1, cdy);
      if (kCount) {
        nkept += (e0 > l2tau) + (e1 > l2tau);
      } else {
        const float v0 = ex2_approx(e0), v1 = ex2_approx(e1);
        p0 += e0 > l2tau ? v0 : 0.f;
        p1 += e1 > l2tau ? v1 : 0.f;
      }
    }
    acc0 += (double)p0;
    acc1 += (double)p1;
  }
  if (kCount) {
    for (int o = 16; o > 0; o >>= 1) nkept += __shfl_xor_sync(0xffffffffu, nkept, o);
    if (lane == 0) atomicAdd(kept, (unsigned long long)nkept);
    return;
  }
  float2 out = make_float2((float)acc0, (float)acc1);
  *reinterpret_cast<float2 *>(proj + ((int64_t)b * d + (int64_t)(ty * kTile + row)) * d +
                              tx * kTile + col) = out;
}

cudaError_t launch_raster_fwd(const Rec *rec, const uint32_t *list, const int64_t *tile_start,
                              int64_t cap, int64_t M, int B, int d, float l2tau, float *proj,
                              cudaStream_t st) {
  int nt = d / kTile;
  dim3 grid(nt * nt, B);
  raster_fwd_kernel<false><<<grid, kFwdThreads, 0, st>>>(rec, list, tile_start, cap, M, d,
                                                         l2tau, proj, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_count_kept(const Rec *rec, const uint32_t *list, const int64_t *tile_start,
                              int64_t cap, int64_t M, int B, int d, float l2tau,
                              unsigned long long *kept, cudaStream_t st) {
  int nt = d / kTile;
  dim3 grid(nt * nt, B);
  raster_fwd_kernel<true><<<grid, kFwdThreads, 0, st>>>(rec, list, tile_start, cap, M, d,
                                                        l2tau, nullptr, kept);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(kBwdThreads) raster_bwd_kernel(
    const Rec *__restrict__ rec, const uint32_t *__restrict__ list,
    const int64_t *__restrict__ tile_start, int64_t cap, int64_t M, int d, float l2tau,
    const float *__restrict__ dproj, float *__restrict__ mom) {
  __shared__ float4 sg[kTile][kTile / 4];
  const int nt = d / kTile, T = nt * nt;
  const int t = blockIdx.x, b = blockIdx.y;
  const int tx = t % nt, ty = t / nt;
  const int x0 = tx * kTile, y0 = ty * kTile;
  // g tile: 16 rows x 4 float4
  if (threadIdx.x < kTile * kTile / 4) {
    int r = threadIdx.x >> 2, q = threadIdx.x & 3;
    sg[r][q] = *reinterpret_cast<const float4 *>(dproj + ((int64_t)b * d + y0 + r) * d + x0 +
                                                 4 * q);
  }
  __syncthreads();
  int64_t s = tile_start[(int64_t)b * T + t];
  int64_t e = tile_start[(int64_t)b * T + t + 1];
  e = min(e, cap);
  s = min(s, e);
  const Rec *rb = rec + (int64_t)b * M;
  float *mb = mom + (int64_t)b * M * 6;
  for (int64_t base = s; base < e; base += kBwdThreads) {
    int64_t i = base + threadIdx.x;
    if (i >= e) break;
    uint32_t j = list[i];
    Rec r = rb[j];
    const float px = r.a.x, py = r.a.y, ca = r.a.z, cb = r.a.w, cc = r.b.x, l2A = r.b.y;
    int vlo, vhi;
    if (!pixel_range(py, r.b.w, d, vlo, vhi)) continue;
    vlo = max(vlo, y0);
    vhi = min(vhi, y0 + kTile - 1);
    float m0 = 0.f, m1 = 0.f, m2 = 0.f, m3 = 0.f, m4 = 0.f, m5 = 0.f;
    for (int v = vlo; v <= vhi; ++v) {
      const float dy = (float)v - py;
      const float bdy = cb * dy;
      const float cdy = fmaf(cc * dy, dy, l2A);
      float r0 = 0.f, r1 = 0.f, r3 = 0.f;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float4 g4 = sg[v - y0][q];
        const float gq[4] = {g4.x, g4.y, g4.z, g4.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const float dx = (float)(x0 + 4 * q + k) - px;
          const float ee = fmaf(fmaf(ca, dx, bdy), dx, cdy);
          const float val = ex2_approx(ee);
          const float gv = ee > l2tau ? gq[k] * val : 0.f;
          r0 += gv;
          const float tt = gv * dx;
          r1 += tt;
          r3 = fmaf(tt, dx, r3);
        }
      }
      m0 += r0;
      m1 += r1;
      m2 = fmaf(dy, r0, m2);
      m3 += r3;
      m4 = fmaf(dy, r1, m4);
      m5 = fmaf(dy * dy, r0, m5);
    }
    float *mm = mb + (int64_t)j * 6;
    atomicAdd(mm + 0, m0);
    atomicAdd(mm + 1, m1);
    atomicAdd(mm + 2, m2);
    atomicAdd(mm + 3, m3);
    atomicAdd(mm + 4, m4);
    atomicAdd(mm + 5, m5);
  }
}

cudaError_t launch_raster_bwd(const Rec *rec, const uint32_t *list, const int64_t *tile_start,
                              int64_t cap, int64_t M, int B, int d, float l2tau,
                              const float *dproj, float *mom, cudaStream_t st) {
  int nt = d / kTile;
  dim3 grid(nt * nt, B);
  raster_bwd_kernel<<<grid, kBwdThreads, 0, st>>>(rec, list, tile_start, cap, M, d, l2tau,
                                                  dproj, mom);
  return cudaGetLastError();
}

// ------------------------------------------------------ plain dense -----

// One thread per pixel, every Gaussian of the image, no culling.
__global__ void __launch_bounds__(256) dense_fwd_kernel(const Rec *__restrict__ rec, int64_t M,
                                                        int d, float l2tau,
                                                        float *__restrict__ proj) {
  int b = blockIdx.y;
  int64_t pix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool act = pix < (int64_t)d * d;
  int u = (int)(pix % d), v = (int)(pix / d);
  const Rec *rb = rec + (int64_t)b * M;
  double acc = 0.0;
  float part = 0.f;
  for (int64_t j = 0; j < M; ++j) {
    Rec r = rb[j];
    float dx = (float)u - r.a.x, dy = (float)v - r.a.y;
    float ee = fmaf(fmaf(r.a.z, dx, r.a.w * dy), dx, fmaf(r.b.x * dy, dy, r.b.y));
    float val = ex2_approx(ee);
    part += ee > l2tau ? val : 0.f;
    if ((j & 127) == 127) {
      acc += part;
      part = 0.f;
    }
  }
  acc += part;
  if (act) proj[(int64_t)b * d * d + pix] = (float)acc;
}

// One thread per (image, Gaussian), every pixel of the image.
__global__ void __launch_bounds__(128) dense_bwd_kernel(const Rec *__restrict__ rec, int64_t M,
                                                        int d, float l2tau,
                                                        const float *__restrict__ dproj,
                                                        float *__restrict__ mom) {
  int b = blockIdx.y;
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= M) return;
  Rec r = rec[(int64_t)b * M + j];
  const float *g = dproj + (int64_t)b * d * d;
  float m[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int v = 0; v < d; ++v) {
    float dy = (float)v - r.a.y;
    float bdy = r.a.w * dy, cdy = fmaf(r.b.x * dy, dy, r.b.y);
    float r0 = 0.f, r1 = 0.f, r3 = 0.f;
    for (int u = 0; u < d; ++u) {
      float dx = (float)u - r.a.x;
      float ee = fmaf(fmaf(r.a.z, dx, bdy), dx, cdy);
      float val = ex2_approx(ee);
      float gv = ee > l2tau ? __ldg(g + (int64_t)v * d + u) * val : 0.f;
      r0 += gv;
      float tt = gv * dx;
      r1 += tt;
      r3 = fmaf(tt, dx, r3);
    }
    m[0] += r0;
    m[1] += r1;
    m[2] = fmaf(dy, r0, m[2]);
    m[3] += r3;
    m[4] = fmaf(dy, r1, m[4]);
    m[5] = fmaf(dy * dy, r0, m[5]);
  }
  float *mm = mom + ((int64_t)b * M + j) * 6;
#pragma unroll
  for (int k = 0; k < 6; ++k) mm[k] = m[k];
}

cudaError_t launch_dense_fwd(const Rec *rec, int64_t M, int B, int d, float l2tau, float *proj,
                             cudaStream_t st) {
  dim3 grid((unsigned)(((int64_t)d * d + 255) / 256), B);
  dense_fwd_kernel<<<grid, 256, 0, st>>>(rec, M, d, l2tau, proj);
  return cudaGetLastError();
}

cudaError_t launch_dense_bwd(const Rec *rec, int64_t M, int B, int d, float l2tau,
                             const float *dproj, float *mom, cudaStream_t st) {
  dim3 grid((unsigned)((M + 127) / 128), B);
  dense_bwd_kernel<<<grid, 128, 0, st>>>(rec, M, d, l2tau, dproj, mom);
  return cudaGetLastError();
}

}  // namespace gem
