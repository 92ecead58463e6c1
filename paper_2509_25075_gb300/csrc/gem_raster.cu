// Steps a3 (raster forward) and a5 (raster backward) of the GEM hot path,
// plus the plain dense forms used as the baseline.
//
// Both rasterisers run one CTA of 128 threads per (image, 16x16 tile) and
// stage the tile's list (depth order) in shared memory 128 records at a
// time.  The thread that stages a record also computes its quadrant mask:
// bit q is set when the record's region above tau meets the 8x8 quadrant q
// of the tile (exact ellipse-rectangle test), so work is spent only where a
// pair can be kept.
//
// a3: Eq. render restricted by Eq. accu.  Warp q owns quadrant q (8 rows x
//     8 columns, two horizontally adjacent pixels per lane) and walks, in
//     list order, only the staged records whose bit q is set (a ballot per
//     32 records).  Each pixel adds its kept terms from the lowest depth to
//     the highest.
// a5: the "efficient gradient" of Sec. 1 (iii) / Sec. 3.2: only pairs kept by
//     Eq. accu.  One thread per listed Gaussian; the staged batch is sorted
//     by quadrant mask so that a warp's threads walk the same quadrants.  The
//     thread accumulates six moments of g * value over its pixels, which a6
//     turns into parameter gradients; one set of atomics per (tile, Gaussian).
#include "gem_internal.cuh"

namespace gem {

constexpr int kFwdThreads = 128;
constexpr int kBwdThreads = 128;

// kCount = true: the same walk, counting kept pairs into kept[0] and
// evaluated pairs into kept[1] instead of writing the projection
// (inspection only, never on the timed path).
template <bool kCount>
__global__ void __launch_bounds__(kFwdThreads) raster_fwd_kernel(
    const Rec *__restrict__ rec, const uint32_t *__restrict__ list,
    const int64_t *__restrict__ tile_start, int64_t cap, int64_t M, int d, float l2tau,
    float *__restrict__ proj, unsigned long long *__restrict__ kept) {
  __shared__ float4 sa[kFwdThreads], sb[kFwdThreads];
  __shared__ unsigned smask[kFwdThreads];
  const int nt = d / kTile, T = nt * nt;
  const int t = blockIdx.x, b = blockIdx.y;
  const int tx = t % nt, ty = t / nt;
  const int x0 = tx * kTile, y0 = ty * kTile;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned qbit = 1u << warp;
  // quadrant (warp & 1, warp >> 1); lane -> row lane/4, columns 2 (lane%4) + {0,1}
  const int px_ = x0 + 8 * (warp & 1) + 2 * (lane & 3);
  const int py_ = y0 + 8 * (warp >> 1) + (lane >> 2);
  const float X0 = (float)px_, X1 = X0 + 1.f, Y = (float)py_;
  int64_t s = tile_start[(int64_t)b * T + t];
  int64_t e = tile_start[(int64_t)b * T + t + 1];
  e = min(e, cap);
  s = min(s, e);
  const Rec *rb = rec + (int64_t)b * M;
  double acc0 = 0.0, acc1 = 0.0;
  unsigned nkept = 0, neval = 0;
  for (int64_t base = s; base < e; base += kFwdThreads) {
    const int n = (int)min((int64_t)kFwdThreads, e - base);
    __syncthreads();
    if (threadIdx.x < n) {
      const Rec r = rb[list[base + threadIdx.x]];
      sa[threadIdx.x] = r.a;
      sb[threadIdx.x] = r.b;
      smask[threadIdx.x] = quadrant_mask(r, x0, y0, r.b.y - l2tau + kMargin);
    } else {
      smask[threadIdx.x] = 0;
    }
    __syncthreads();
    float p0 = 0.f, p1 = 0.f;
    for (int c = 0; c < n; c += 32) {
      unsigned bal = __ballot_sync(0xffffffffu, smask[c + lane] & qbit);
      while (bal) {
        const int k = c + __ffs(bal) - 1;
        bal &= bal - 1;
        const float4 A = sa[k];
        const float4 Bv = sb[k];
        const float dy = Y - A.y;
        const float bdy = A.w * dy;
        const float cdy = fmaf(Bv.x * dy, dy, Bv.y);
        const float dx0 = X0 - A.x, dx1 = X1 - A.x;
        const float e0 = fmaf(fmaf(A.z, dx0, bdy), dx0, cdy);
        const float e1 = fmaf(fmaf(A.z, dx1, bdy), dx1, cdy);
        if (kCount) {
          nkept += (e0 > l2tau) + (e1 > l2tau);
          neval += 2;
        } else {
          const float v0 = ex2_approx(e0), v1 = ex2_approx(e1);
          p0 += e0 > l2tau ? v0 : 0.f;
          p1 += e1 > l2tau ? v1 : 0.f;
        }
      }
    }
    acc0 += (double)p0;
    acc1 += (double)p1;
  }
  if (kCount) {
    for (int o = 16; o > 0; o >>= 1) {
      nkept += __shfl_xor_sync(0xffffffffu, nkept, o);
      neval += __shfl_xor_sync(0xffffffffu, neval, o);
    }
    if (lane == 0) {
      atomicAdd(kept, (unsigned long long)nkept);
      atomicAdd(kept + 1, (unsigned long long)neval);
    }
    return;
  }
  float2 out = make_float2((float)acc0, (float)acc1);
  *reinterpret_cast<float2 *>(proj + ((int64_t)b * d + py_) * d + px_) = out;
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
  __shared__ float4 sa[kBwdThreads], sb[kBwdThreads];
  __shared__ uint32_t sj[kBwdThreads];
  __shared__ unsigned char smask[kBwdThreads];
  __shared__ int hist[16];
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
  int64_t s = tile_start[(int64_t)b * T + t];
  int64_t e = tile_start[(int64_t)b * T + t + 1];
  e = min(e, cap);
  s = min(s, e);
  const Rec *rb = rec + (int64_t)b * M;
  float *mb = mom + (int64_t)b * M * 6;
  for (int64_t base = s; base < e; base += kBwdThreads) {
    const int n = (int)min((int64_t)kBwdThreads, e - base);
    __syncthreads();
    if (threadIdx.x < 16) hist[threadIdx.x] = 0;
    __syncthreads();
    // stage: own record and its quadrant mask, then counting sort by mask
    Rec r;
    uint32_t j = 0;
    unsigned m = 0;
    if (threadIdx.x < n) {
      j = list[base + threadIdx.x];
      r = rb[j];
      m = quadrant_mask(r, x0, y0, r.b.y - l2tau + kMargin);
      atomicAdd(&hist[m], 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int run = 0;
      for (int k = 0; k < 16; ++k) {
        int v = hist[k];
        hist[k] = run;
        run += v;
      }
    }
    __syncthreads();
    if (threadIdx.x < n) {
      int pos = atomicAdd(&hist[m], 1);
      sa[pos] = r.a;
      sb[pos] = r.b;
      sj[pos] = j;
      smask[pos] = (unsigned char)m;
    }
    __syncthreads();
    if (threadIdx.x >= n) continue;
    const float4 A = sa[threadIdx.x];
    const float4 Bv = sb[threadIdx.x];
    const unsigned mk = smask[threadIdx.x];
    const float px = A.x, py = A.y, ca = A.z, cb = A.w, cc = Bv.x, l2A = Bv.y;
    int vlo, vhi;
    if (mk == 0 || !pixel_range(py, Bv.w, d, vlo, vhi)) continue;
    float m0 = 0.f, m1 = 0.f, m2 = 0.f, m3 = 0.f, m4 = 0.f, m5 = 0.f;
#pragma unroll 1
    for (int q = 0; q < 4; ++q) {
      if (!(mk & (1u << q))) continue;
      const int qx = 8 * (q & 1), qy = 8 * (q >> 1);
      const int r0_ = max(vlo - y0, qy), r1_ = min(vhi - y0, qy + 7);
      for (int rr = r0_; rr <= r1_; ++rr) {
        const float dy = (float)(y0 + rr) - py;
        const float bdy = cb * dy;
        const float cdy = fmaf(cc * dy, dy, l2A);
        float a0 = 0.f, a1 = 0.f, a3 = 0.f;
#pragma unroll
        for (int hq = 0; hq < 2; ++hq) {
          const float4 g4 = sg[rr][(qx >> 2) + hq];
          const float gq[4] = {g4.x, g4.y, g4.z, g4.w};
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const float dx = (float)(x0 + qx + 4 * hq + k) - px;
            const float ee = fmaf(fmaf(ca, dx, bdy), dx, cdy);
            const float val = ex2_approx(ee);
            const float gv = ee > l2tau ? gq[k] * val : 0.f;
            a0 += gv;
            const float tt = gv * dx;
            a1 += tt;
            a3 = fmaf(tt, dx, a3);
          }
        }
        m0 += a0;
        m1 += a1;
        m2 = fmaf(dy, a0, m2);
        m3 += a3;
        m4 = fmaf(dy, a1, m4);
        m5 = fmaf(dy * dy, a0, m5);
      }
    }
    float *mm = mb + (int64_t)sj[threadIdx.x] * 6;
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
