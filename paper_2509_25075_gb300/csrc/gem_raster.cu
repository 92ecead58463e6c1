// Steps a3 (raster forward) and a5 (raster backward) of the GEM hot path,
// plus the plain dense forms used as the baseline.
//
// Both rasterisers run one CTA of 128 threads per (image, 16x16 tile) and
// walk the tile's list, which is in ascending depth and carries, per entry,
// the mask of the 4x4 pixel blocks the Gaussian's region above tau meets
// (computed once by the binning).  A Gaussian therefore costs 16 pixel
// evaluations per block it touches, instead of 256 per tile.
//
// a3: Eq. render restricted by Eq. accu.  The 16 blocks are owned by 8
//     threads each (two horizontally adjacent pixels per thread).  Records
//     are staged 128 at a time; ballots give every block the list of staged
//     records that touch it, in list order, and the block's threads walk
//     that list.  So each pixel adds its kept terms from the lowest depth to
//     the highest, deterministically (float partials per 128 records, summed
//     in double).
// a5: the "efficient gradient" of Sec. 1 (iii) / Sec. 3.2: only pairs kept by
//     Eq. accu.  Each warp takes every fourth 64-record window of the list,
//     sorts it by block count and runs it as two rounds of 32 records with
//     neighbouring counts, one lane per record: the lane walks the record's
//     blocks and accumulates six moments of g * value in registers.  No
//     barrier couples the warps.  a6 turns the moments into parameter
//     gradients.  One set of vector atomics per (tile, Gaussian) goes to
//     global memory.
#include "gem_internal.cuh"

namespace gem {

constexpr int kThreads = 128;

// (sum, compensation) + x, Kahan; the compensated value is sum - compensation.
__device__ __forceinline__ float2 kahan_add(float2 s, float x) {
  const float y = x - s.y;
  const float t = s.x + y;
  return make_float2(t, (t - s.x) - y);
}
constexpr int kWin = 128;  // records staged per window

// kCount = true: the same walk, counting kept pairs into kept[0] and
// evaluated pairs into kept[1] instead of writing the projection
// (inspection only, never on the timed path).
template <bool kCount>
__global__ void __launch_bounds__(kThreads) raster_fwd_kernel(
    const Rec *__restrict__ rec, const uint32_t *__restrict__ list,
    const uint16_t *__restrict__ lmask, const int64_t *__restrict__ tile_start, int64_t cap,
    int64_t M, int d, float l2tau, float *__restrict__ proj,
    unsigned long long *__restrict__ kept) {
  __shared__ float4 sa[kWin], sb[kWin];
  __shared__ unsigned char blist[16][kWin + 4];      // per block: staged slots touching it
                                                      // (rows padded: lists in different banks)
  __shared__ unsigned short wcnt[kThreads / 32][16];  // per warp, per block: how many
  __shared__ unsigned wbal[kThreads / 32][16];        // per warp, per block: which lanes
  __shared__ float2 pix[kTile * kTile];               // per-pixel compensated sums over windows
  __shared__ unsigned char sorder[16], slen[16];      // blocks by list length
  const int nt = d / kTile, T = nt * nt;
  const int t = blockIdx.x, b = blockIdx.y;
  const int tx = t % nt, ty = t / nt;
  const int x0 = tx * kTile, y0 = ty * kTile;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // thread group g (8 threads) takes, in each window, the block with the
  // g-th longest list; within it, pair pp: row pp/2, columns 2 (pp%2) + {0,1}
  const int grp = threadIdx.x >> 3, pp = threadIdx.x & 7;
  int64_t s = tile_start[(int64_t)b * T + t];
  int64_t e = tile_start[(int64_t)b * T + t + 1];
  e = min(e, cap);
  s = min(s, e);
  const Rec *rb = rec + (int64_t)b * M;
  const unsigned lt = (1u << lane) - 1u;
  for (int i = threadIdx.x; i < kTile * kTile; i += kThreads) pix[i] = make_float2(0.f, 0.f);
  unsigned nkept = 0, neval = 0;
  for (int64_t base = s; base < e; base += kWin) {
    const int n = (int)min((int64_t)kWin, e - base);
    __syncthreads();  // previous window fully consumed
    unsigned m = 0;
    if (threadIdx.x < n) {
      const Rec r = rb[list[base + threadIdx.x]];
      m = lmask[base + threadIdx.x];
      sa[threadIdx.x] = r.a;
      sb[threadIdx.x] = r.b;
    }
    unsigned mybal = 0;  // lane k < 16: which of this warp's records touch block k
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      unsigned bk = __ballot_sync(0xffffffffu, (m >> k) & 1u);
      if (lane == k) mybal = bk;
    }
    if (lane < 16) {
      wcnt[warp][lane] = (unsigned short)__popc(mybal);
      wbal[warp][lane] = mybal;
    }
    __syncthreads();
    // place my record in the lists of its blocks: after the records of lower
    // warps and lower lanes touching the same block
    for (unsigned mm = m; mm; mm &= mm - 1) {
      const int k = __ffs(mm) - 1;
      int pos = __popc(wbal[warp][k] & lt);
      for (int w = 0; w < warp; ++w) pos += wcnt[w][k];
      blist[k][pos] = (unsigned char)threadIdx.x;
    }
    // warp 0 orders the blocks by list length (longest first, ties by
    // index): group g takes block sorder[g]
    if (warp == 0) {
      int len = 0;
      if (lane < 16)
#pragma unroll
        for (int w = 0; w < kThreads / 32; ++w) len += wcnt[w][lane];
      int rank = 0;
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int lq = __shfl_sync(0xffffffffu, len, q);
        rank += (lq > len) || (lq == len && q < lane);
      }
      if (lane < 16) {
        sorder[rank] = (unsigned char)lane;
        slen[rank] = (unsigned char)len;
      }
    }
    __syncthreads();
    const int blk = sorder[grp], nb = slen[grp];
    const int px_ = x0 + 4 * (blk & 3) + 2 * (pp & 1);
    const int py_ = y0 + 4 * (blk >> 2) + (pp >> 1);
    const float X0 = (float)px_, X1 = X0 + 1.f, Y = (float)py_;
    float p0 = 0.f, p1 = 0.f;
    for (int i = 0; i < nb; ++i) {
      const int slot = blist[blk][i];
      const float4 A = sa[slot];
      const float4 Bv = sb[slot];
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
    // the window's sum joins the pixel's running sum (one owner per pixel
    // per window, windows in list order; Kahan-compensated)
    const int pl = (py_ - y0) * kTile + (px_ - x0);
    pix[pl] = kahan_add(pix[pl], p0);
    pix[pl + 1] = kahan_add(pix[pl + 1], p1);
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
  __syncthreads();
  for (int i = threadIdx.x; i < kTile * kTile / 2; i += kThreads) {
    const int r = (2 * i) / kTile, c = (2 * i) % kTile;
    *reinterpret_cast<float2 *>(proj + ((int64_t)b * d + y0 + r) * d + x0 + c) =
        make_float2(pix[2 * i].x - pix[2 * i].y, pix[2 * i + 1].x - pix[2 * i + 1].y);
  }
}

cudaError_t launch_raster_fwd(const Rec *rec, const uint32_t *list, const uint16_t *lmask,
                              const int64_t *tile_start, int64_t cap, int64_t M, int B, int d,
                              float l2tau, float *proj, cudaStream_t st) {
  int nt = d / kTile;
  dim3 grid(nt * nt, B);
  raster_fwd_kernel<false><<<grid, kThreads, 0, st>>>(rec, list, lmask, tile_start, cap, M, d,
                                                      l2tau, proj, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_count_kept(const Rec *rec, const uint32_t *list, const uint16_t *lmask,
                              const int64_t *tile_start, int64_t cap, int64_t M, int B, int d,
                              float l2tau, unsigned long long *kept, cudaStream_t st) {
  int nt = d / kTile;
  dim3 grid(nt * nt, B);
  raster_fwd_kernel<true><<<grid, kThreads, 0, st>>>(rec, list, lmask, tile_start, cap, M, d,
                                                     l2tau, nullptr, kept);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(kThreads) raster_bwd_kernel(
    const Rec *__restrict__ rec, const uint32_t *__restrict__ list,
    const uint16_t *__restrict__ lmask, const int64_t *__restrict__ tile_start, int64_t cap,
    int64_t M, int d, float l2tau, const float *__restrict__ dproj, float *__restrict__ mom) {
  constexpr int kWarps = kThreads / 32;
  constexpr int kPer = 2;            // records per lane per window
  constexpr int kWW = 32 * kPer;     // records per warp window
  __shared__ float4 sg[16][4];  // g by 4x4 block: [block][row] = 4 pixels
  __shared__ float4 sa[kWarps][kWW], sb[kWarps][kWW];
  __shared__ uint32_t sj[kWarps][kWW];
  __shared__ unsigned short smask[kWarps][kWW];
  __shared__ int hist[kWarps][17];
  const int nt = d / kTile, T = nt * nt;
  const int t = blockIdx.x, b = blockIdx.y;
  const int tx = t % nt, ty = t / nt;
  const int x0 = tx * kTile, y0 = ty * kTile;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // g tile, stored block by block
  if (threadIdx.x < kTile * kTile / 4) {
    const int r = threadIdx.x >> 2, q = threadIdx.x & 3;  // pixel row, 4-column group
    sg[4 * (r >> 2) + q][r & 3] =
        *reinterpret_cast<const float4 *>(dproj + ((int64_t)b * d + y0 + r) * d + x0 + 4 * q);
  }
  __syncthreads();
  int64_t s = tile_start[(int64_t)b * T + t];
  int64_t e = tile_start[(int64_t)b * T + t + 1];
  e = min(e, cap);
  s = min(s, e);
  const Rec *rb = rec + (int64_t)b * M;
  float *mb = mom + (int64_t)b * M * 6;
  int *h = hist[warp];
  // warp w takes windows w, w + 4, ... of 64 records; no barrier couples the
  // warps after the g tile is in place
  for (int64_t base = s + kWW * warp; base < e; base += kWW * kWarps) {
    Rec r[kPer];
    uint32_t j[kPer];
    unsigned m[kPer];
    __syncwarp();  // previous window's reads are done
    if (lane < 17) h[lane] = 0;
    __syncwarp();
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int64_t i = base + q * 32 + lane;
      j[q] = 0;
      m[q] = 0;
      if (i < e) {
        j[q] = list[i];
        r[q] = rb[j[q]];
        m[q] = lmask[i];
      }
      atomicAdd(&h[__popc(m[q])], 1);
    }
    __syncwarp();
    // exclusive scan of the count histogram, most blocks first
    if (lane == 0) {
      int run = 0;
      for (int v = 16; v >= 0; --v) {
        const int c = h[v];
        h[v] = run;
        run += c;
      }
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int pos = atomicAdd(&h[__popc(m[q])], 1);
      sa[warp][pos] = r[q].a;
      sb[warp][pos] = r[q].b;
      sj[warp][pos] = j[q];
      smask[warp][pos] = (unsigned short)m[q];
    }
    __syncwarp();
    // rounds of 32 records with neighbouring block counts
#pragma unroll 1
    for (int q = 0; q < kPer; ++q) {
      const int slot = q * 32 + lane;
      const unsigned mk = smask[warp][slot];
      if (!mk) continue;
      const float4 A = sa[warp][slot];
      const float4 Bv = sb[warp][slot];
      const float ca = A.z, cb = A.w, cc = Bv.x, l2A = Bv.y;
      float m0 = 0.f, m1 = 0.f, m2 = 0.f, m3 = 0.f, m4 = 0.f, m5 = 0.f;
      for (unsigned mm = mk; mm; mm &= mm - 1) {
        const int k = __ffs(mm) - 1;
        const float fx = (float)(x0 + 4 * (k & 3)) - A.x;
        const float fy = (float)(y0 + 4 * (k >> 2)) - A.y;
#pragma unroll
        for (int rr = 0; rr < 4; ++rr) {
          const float dy = fy + (float)rr;
          const float bdy = cb * dy;
          const float cdy = fmaf(cc * dy, dy, l2A);
          const float4 g4 = sg[k][rr];
          const float gq[4] = {g4.x, g4.y, g4.z, g4.w};
          float a0 = 0.f, a1 = 0.f, a3 = 0.f;
#pragma unroll
          for (int c4 = 0; c4 < 4; ++c4) {
            const float dx = fx + (float)c4;
            const float ee = fmaf(fmaf(ca, dx, bdy), dx, cdy);
            const float val = ex2_approx(ee);
            const float gv = ee > l2tau ? gq[c4] * val : 0.f;
            a0 += gv;
            const float tt = gv * dx;
            a1 += tt;
            a3 = fmaf(tt, dx, a3);
          }
          m0 += a0;
          m1 += a1;
          m2 = fmaf(dy, a0, m2);
          m3 += a3;
          m4 = fmaf(dy, a1, m4);
          m5 = fmaf(dy * dy, a0, m5);
        }
      }
      float2 *mo = reinterpret_cast<float2 *>(mb + (int64_t)sj[warp][slot] * 6);
      atomicAdd(mo + 0, make_float2(m0, m1));
      atomicAdd(mo + 1, make_float2(m2, m3));
      atomicAdd(mo + 2, make_float2(m4, m5));
    }
  }
}

cudaError_t launch_raster_bwd(const Rec *rec, const uint32_t *list, const uint16_t *lmask,
                              const int64_t *tile_start, int64_t cap, int64_t M, int B, int d,
                              float l2tau, const float *dproj, float *mom, cudaStream_t st) {
  int nt = d / kTile;
  dim3 grid(nt * nt, B);
  raster_bwd_kernel<<<grid, kThreads, 0, st>>>(rec, list, lmask, tile_start, cap, M, d, l2tau,
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
