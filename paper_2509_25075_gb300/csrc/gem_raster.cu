// Steps a3 (raster forward) and a5 (raster backward) of the GEM hot path,
// plus the plain dense forms used as the baseline.
//
// Both rasterisers run one CTA of 128 threads per (image, 16x16 tile) and
// walk the tile's list, which is in ascending depth and carries, per entry,
// the mask of the 4x4 pixel blocks the Gaussian's region above tau meets
// (computed once by the binning).  A Gaussian therefore costs 16 pixel
// evaluations per block it touches, instead of 256 per tile.
//
// a3: Eq. render restricted by Eq. accu.  Records are staged 256 at a time;
//     ballots give every 4x4 block the list of staged records that touch it,
//     in list order.  A group of 8 threads takes one block (blocks by
//     decreasing list length, so a warp's groups run loops of similar
//     length); each thread takes two pixel rows of the block and every
//     fourth record of the block's list, and evaluates its 8 pixels for the
//     record from registers (the record is read from shared memory once per
//     8 evaluations).  At the end of the window a fixed butterfly over the 4
//     lanes sharing the rows sums the partials, each lane keeping two
//     pixels, and the window's sums join the pixels' running sums with Kahan
//     compensation.  Each pixel's sum is therefore
//     formed window by window in depth order, deterministically.
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
constexpr int kSub = 2;                // forward: records staged per thread per window
constexpr int kWin = kThreads * kSub;  // records staged per window

// kCount = true: the same walk, counting kept pairs into kept[0] and
// evaluated pairs into kept[1] instead of writing the projection
// (inspection only, never on the timed path).
template <bool kCount>
__global__ void __launch_bounds__(kThreads, 12) raster_fwd_kernel(
    const Rec *__restrict__ rec, const uint32_t *__restrict__ list,
    const uint16_t *__restrict__ lmask, const int64_t *__restrict__ tile_start, int64_t cap,
    int64_t M, int d, float l2tau, float *__restrict__ proj,
    unsigned long long *__restrict__ kept) {
  constexpr int kWarps = kThreads / 32;
  __shared__ float4 sa[kWin], sb[kWin];
  using Slot = unsigned char;
  __shared__ Slot blist[16][kWin + 4];            // per block: staged slots touching it
                                                   // (rows padded: lists in different banks)
  __shared__ unsigned short wcnt[kSub][kWarps][16];  // per sub-window, warp, block: how many
  __shared__ unsigned wbal[kSub][kWarps][16];        // per sub-window, warp, block: which lanes
  __shared__ float2 pix[kTile * kTile];              // per-pixel compensated sums over windows
  __shared__ unsigned char sorder[16];               // blocks by list length
  __shared__ unsigned short slen[16];
  const int nt = d / kTile, T = nt * nt;
  const int t = blockIdx.x, b = blockIdx.y;
  const int tx = t % nt, ty = t / nt;
  const int x0 = tx * kTile, y0 = ty * kTile;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // thread group g (8 threads) takes, in each window, the block with the
  // g-th longest list
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
    // record slot u * kThreads + threadIdx.x of sub-window u
    unsigned m[kSub];
#pragma unroll
    for (int u = 0; u < kSub; ++u) {
      const int slot = u * kThreads + threadIdx.x;
      m[u] = 0;
      if (slot < n) {
        const Rec r = rb[list[base + slot]];
        m[u] = lmask[base + slot];
        sa[slot] = r.a;
        sb[slot] = r.b;
      }
      unsigned mybal = 0;  // lane k < 16: which of this warp's records touch block k
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const unsigned bk = __ballot_sync(0xffffffffu, (m[u] >> k) & 1u);
        if (lane == k) mybal = bk;
      }
      if (lane < 16) {
        wcnt[u][warp][lane] = (unsigned short)__popc(mybal);
        wbal[u][warp][lane] = mybal;
      }
    }
    __syncthreads();
    // place my records in the lists of their blocks: after the records of
    // earlier sub-windows, lower warps and lower lanes touching the same block
#pragma unroll
    for (int u = 0; u < kSub; ++u) {
      for (unsigned mm = m[u]; mm; mm &= mm - 1) {
        const int k = __ffs(mm) - 1;
        int pos = __popc(wbal[u][warp][k] & lt);
        for (int v = 0; v < u; ++v)
#pragma unroll
          for (int w = 0; w < kWarps; ++w) pos += wcnt[v][w][k];
        for (int w = 0; w < warp; ++w) pos += wcnt[u][w][k];
        blist[k][pos] = (Slot)(u * kThreads + threadIdx.x);
      }
    }
    // warp 0 orders the blocks by list length (longest first, ties by
    // index): group g takes block sorder[g]
    if (warp == 0) {
      int len = 0;
      if (lane < 16)
#pragma unroll
        for (int u = 0; u < kSub; ++u)
#pragma unroll
          for (int w = 0; w < kWarps; ++w) len += wcnt[u][w][lane];
      int rank = 0;
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int lq = __shfl_sync(0xffffffffu, len, q);
        rank += (lq > len) || (lq == len && q < lane);
      }
      if (lane < 16) {
        sorder[rank] = (unsigned char)lane;
        slen[rank] = (unsigned short)len;
      }
    }
    __syncthreads();
    // group g takes block sorder[g]; thread pp of the group takes rows
    // 2h, 2h + 1 of the block (h = pp / 4) for every fourth record of the
    // block's list (records i = pp % 4 mod 4): eight pixels per record
    const int blk = sorder[grp], nb = slen[grp];
    const int h = pp >> 2, ph = pp & 3;
    const float X0 = (float)(x0 + 4 * (blk & 3)), Y0 = (float)(y0 + 4 * (blk >> 2) + 2 * h);
    float acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = 0.f;
    for (int i = ph; i < nb; i += 4) {
      const int slot = blist[blk][i];
      const float4 A = sa[slot];
      const float4 Bv = sb[slot];
      float dx[4], cadx[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        dx[c] = X0 + (float)c - A.x;
        cadx[c] = A.z * dx[c];
      }
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        // e = (ca dx + cb dy) dx + (cc dy^2 + l2A)
        const float dy = Y0 + (float)r - A.y;
        const float bdy = A.w * dy;
        const float cdy = fmaf(Bv.x * dy, dy, Bv.y);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const float ev = fmaf(cadx[c] + bdy, dx[c], cdy);
          if (kCount) {
            nkept += ev > l2tau;
          } else {
            const float v = ex2_approx(ev);
            if (ev > l2tau) acc[4 * r + c] += v;
          }
        }
      }
      if (kCount) neval += 8;
    }
    // reduce-scatter over the 4 lanes sharing the rows (lane bit 1 picks the
    // row, bit 0 the column pair): lane pp ends with row 2h + bit 1, columns
    // 2 bit 0 + {0, 1}
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const bool hi = (pp & 2) != 0;
      const float send = hi ? acc[q] : acc[4 + q];
      const float keep = hi ? acc[4 + q] : acc[q];
      acc[q] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const bool hi = (pp & 1) != 0;
      const float send = hi ? acc[q] : acc[2 + q];
      const float keep = hi ? acc[2 + q] : acc[q];
      acc[q] = keep + __shfl_xor_sync(0xffffffffu, send, 1);
    }
    // the window's sums join the pixels' running sums (one owner per pixel
    // per window, windows in list order; Kahan-compensated)
    const int pl = (4 * (blk >> 2) + 2 * h + ((pp >> 1) & 1)) * kTile + 4 * (blk & 3) + 2 * (pp & 1);
    if (!kCount) {
      pix[pl] = kahan_add(pix[pl], acc[0]);
      pix[pl + 1] = kahan_add(pix[pl + 1], acc[1]);
    }
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
