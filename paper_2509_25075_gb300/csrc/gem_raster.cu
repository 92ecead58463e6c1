// Steps a3 (raster forward) and a5 (raster backward) of the GEM hot path,
// plus the plain dense forms used as the baseline.
//
// Both rasterisers run CTAs of 128 threads over (image, 16x16 tile) work
// items — one per tile on a per-tile grid, or taken from a counter over a
// longest-first tile order on a persistent grid of a chosen number of CTAs
// per SM — and walk the tile's list, which is in ascending depth and
// carries, per entry, the mask of the 4x4 pixel blocks the Gaussian's
// region above tau meets (computed once by the binning).  A Gaussian
// therefore costs 16 pixel evaluations per block it touches, instead of 256
// per tile.  Pixels are evaluated in whitened coordinates (Rec): the
// exponent is l2A - (u11 dx + u12 dy)^2 - (u22 dy)^2.
//
// a3: Eq. render restricted by Eq. accu.  Records are staged 256 at a time
//     (a window; only the 24 bytes the evaluation reads).  One warp bit
//     transpose of the lanes' packed block masks gives each block's record
//     set; the window's (block, record) items are laid out block after
//     block, each block's records in list order, and each block gets a
//     share of the 128 threads in proportion to its items, so a thread
//     never leaves its block.  A thread evaluates the 16 pixels of its block
//     for each of its items (packed float pairs) and writes one partial
//     image of the block; at the end of the window each pixel sums its
//     block's partials in thread order and joins its running sum with Kahan
//     compensation.  (The equal-runs form, raster_fwd_kernel, cuts the
//     items into 128 equal runs across blocks instead.)  The result is
//     deterministic and follows the list's depth order run by run.
// a5: the "efficient gradient" of Sec. 1 (iii) / Sec. 3.2: only pairs kept by
//     Eq. accu.  Each warp takes windows of 64, 128 or 256 records of the
//     list (the next one not yet taken), sorts the window by block count
//     and runs it in rounds of records with neighbouring counts, one or two
//     lanes per record: the lanes walk the record's blocks and accumulate
//     six moments of w = g * value in the record's whitened coordinates
//     (per row: the sums of w, w z1, w z1^2 in packed float pairs, weighted
//     by z2).  The second moments are taken about the whitened S^, c^2 I:
//     for a wide Gaussian under a smooth upstream gradient the conic and
//     amplitude terms of dL/dS^ nearly cancel, and this form lets that
//     cancellation happen inside an accurate sum instead of in the float32
//     chain rule.  Each block's sums join the lane's totals, and the (tile,
//     Gaussian) partial goes to float64 moments in global memory (L2
//     atomics), so the sum over a Gaussian's tiles loses nothing to
//     rounding.  No barrier couples the warps within a tile.  a6 turns the
//     moments into parameter gradients.
#include <type_traits>

#include "gem_internal.cuh"

namespace gem {

constexpr int kThreads = 128;

// (sum, compensation) + x, Kahan; the compensated value is sum - compensation.
__device__ __forceinline__ float2 kahan_add(float2 s, float x) {
  const float y = x - s.y;
  const float t = s.x + y;
  return make_float2(t, (t - s.x) - y);
}
// The 32 x 32 bit matrix whose row r is lane r's x, transposed: lane k gets
// the bits k of all lanes (bit r from lane r), as 32 ballots would give it.
// Five butterfly stages; at distance j the lanes of a pair swap the j-bit
// halves of their 2j-bit groups that lie off the diagonal.
__device__ __forceinline__ unsigned warp_transpose32(unsigned x, int lane) {
  const unsigned hi[5] = {0xffff0000u, 0xff00ff00u, 0xf0f0f0f0u, 0xccccccccu, 0xaaaaaaaau};
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    const int j = 16 >> s;
    const unsigned y = __shfl_xor_sync(0xffffffffu, x, j);
    x = (lane & j) ? ((x & hi[s]) | ((y >> j) & ~hi[s])) : ((x & ~hi[s]) | ((y << j) & hi[s]));
  }
  return x;
}

constexpr int kSub = 2;                // forward: records staged per thread per window
constexpr int kWin = kThreads * kSub;  // records staged per window
static_assert(kThreads == 128, "the forward splits items with shifts by 7");
constexpr int kFwdMinBlocks = 9;      // forward: CTAs per SM (10, with fewer registers, ran slower)

// kCount = true: the same walk, counting kept pairs into kept[0] and
// evaluated pairs into kept[1] instead of writing the projection
// (inspection only, never on the timed path).
template <bool kCount>
__global__ void __launch_bounds__(kThreads, kFwdMinBlocks) raster_fwd_kernel(
    const Rec *__restrict__ rec, const uint2 *__restrict__ list,
    const int64_t *__restrict__ tile_start, int64_t cap,
    int64_t M, int d, float l2tau, float *__restrict__ proj,
    unsigned long long *__restrict__ kept) {
  constexpr int kWarps = kThreads / 32;
  constexpr int kPieces = 16 + kThreads - 1;
  __shared__ float4 sa[kWin];                         // px, py, u11, u12
  __shared__ float2 sb[kWin];                         // u22, log2 A
  __shared__ unsigned char flat[16 * kWin];           // staged slot of each (block, record) item,
                                                      // blocks in order, records in list order
  __shared__ unsigned short wcnt[kSub][kWarps][16];  // per sub-window, warp, block: how many
  __shared__ unsigned wbal[kSub][kWarps][16];        // per sub-window, warp, block: which lanes
  __shared__ int woff[kWarps][kSub][16];             // where a warp's records go in flat
  __shared__ int pstart[kWarps][17];                 // block k's items: [pstart[k], pstart[k+1])
  __shared__ float4 part[kPieces][4];                // piece (block k, thread u) at k + u
  const int nt = d / kTile, T = nt * nt;
  const int t = blockIdx.x, b = blockIdx.y;
  const int tx = t % nt, ty = t / nt;
  const int x0 = tx * kTile, y0 = ty * kTile;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const float nl2tau = -l2tau;  // kept: -e < -log2(tau)
  int64_t s = tile_start[(int64_t)b * T + t];
  int64_t e = tile_start[(int64_t)b * T + t + 1];
  e = min(e, cap);
  s = min(s, e);
  // lists that overflowed their capacity are incomplete: every list counts
  // as empty (the status word reports it)
  if (tile_start[(int64_t)gridDim.y * T] > cap) e = s;
  const Rec *rb = rec + (int64_t)b * M;
  const unsigned lt = (1u << lane) - 1u;
  // pixels owned across windows: two columns of one row of block ob
  const int ob = tid >> 3, ow = tid & 7;
  float2 own0 = make_float2(0.f, 0.f), own1 = make_float2(0.f, 0.f);  // Kahan (sum, comp)
  unsigned nkept = 0, neval = 0;
  for (int64_t base = s; base < e; base += kWin) {
    const int n = (int)min((int64_t)kWin, e - base);
    __syncthreads();  // previous window fully consumed
    // record slot u * kThreads + tid of sub-window u
    unsigned m[kSub];
#pragma unroll
    for (int u = 0; u < kSub; ++u) {
      const int slot = u * kThreads + tid;
      m[u] = 0;
      // an entry whose Gaussian index is out of range (a list position left
      // unwritten when the lists overflowed their capacity) counts as empty
      const uint2 ent = slot < n ? list[base + slot] : make_uint2(0u, 0u);
      const uint32_t jj = ent.x;
      if (slot < n && jj < (uint64_t)M) {
        const Rec *rp = rb + jj;
        const float4 ra = rp->a;
        const float2 rbv = *reinterpret_cast<const float2 *>(&rp->b);
        m[u] = ent.y & 0xffffu;
        sa[slot] = ra;
        sb[slot] = rbv;
      }
    }
    // which of this warp's records touch block k, both sub-windows at once:
    // lane k < 16 gets block k of sub-window 0, lane 16 + k block k of
    // sub-window 1 (the lanes' packed masks, transposed as a bit matrix)
    static_assert(kSub == 2, "two 16-bit masks per lane");
    {
      const unsigned bal = warp_transpose32(m[0] | (m[1] << 16), lane);
      wcnt[lane >> 4][warp][lane & 15] = (unsigned short)__popc(bal);
      wbal[lane >> 4][warp][lane & 15] = bal;
    }
    __syncthreads();
    // every warp: block lengths, their prefix (the items of all blocks laid
    // out block after block) and where its own records go: after the
    // records of earlier sub-windows and lower warps touching the block
    {
      int len = 0, wo[kSub];
#pragma unroll
      for (int u = 0; u < kSub; ++u) {
        wo[u] = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
          if (w == warp) wo[u] = len;
          if (lane < 16) len += wcnt[u][w][lane];
        }
      }
      int incl = len;
#pragma unroll
      for (int o = 1; o < 16; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
      }
      if (lane < 16) {
        pstart[warp][lane] = incl - len;
#pragma unroll
        for (int u = 0; u < kSub; ++u) woff[warp][u][lane] = incl - len + wo[u];
      }
      if (lane == 15) pstart[warp][16] = incl;
      __syncwarp();
    }
#pragma unroll
    for (int u = 0; u < kSub; ++u) {
      for (unsigned mm = m[u]; mm; mm &= mm - 1) {
        const int k = __ffs(mm) - 1;
        flat[woff[warp][u][k] + __popc(wbal[u][warp][k] & lt)] = (unsigned char)(u * kThreads + tid);
      }
    }
    __syncthreads();
    // thread tid takes items [lo, hi) of the concatenation: a run of
    // records of one block or a few consecutive blocks, 16 pixels each;
    // each block it leaves (a piece) goes to part[k + tid]
    const int *ps = pstart[0];
    const int N = ps[16];
    const int lo = (tid * N) >> 7, hi = ((tid + 1) * N) >> 7;
    if (lo < hi) {
      int k = 0;
      while (ps[k + 1] <= lo) ++k;
      float2 acc[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) acc[q] = make_float2(0.f, 0.f);
      float X0 = (float)(x0 + 4 * (k & 3)), Y0 = (float)(y0 + 4 * (k >> 2));
      int kend = ps[k + 1];  // end of block k's items
      for (int i = lo; i < hi; ++i) {
        if (i >= kend) {  // the run enters the next non-empty block
          if (!kCount) {
#pragma unroll
            for (int r = 0; r < 4; ++r)
              part[k + tid][r] = make_float4(acc[2 * r].x, acc[2 * r].y, acc[2 * r + 1].x,
                                             acc[2 * r + 1].y);
          }
#pragma unroll
          for (int q = 0; q < 8; ++q) acc[q] = make_float2(0.f, 0.f);
          do ++k;
          while (ps[k + 1] <= i);
          kend = ps[k + 1];
          X0 = (float)(x0 + 4 * (k & 3));
          Y0 = (float)(y0 + 4 * (k >> 2));
        }
        const int slot = flat[i];
        const float4 A = sa[slot];
        const float2 Bv = sb[slot];
        const float2 npx = f2(-A.x);
        const float2 dx01 = add2(make_float2(X0, X0 + 1.f), npx);
        const float2 dx23 = add2(make_float2(X0 + 2.f, X0 + 3.f), npx);
        const float2 u11 = f2(A.z);
        const float2 ux01 = mul2(u11, dx01), ux23 = mul2(u11, dx23);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          // -e = z1^2 + (z2^2 - l2A), z1 = u11 dx + u12 dy, z2 = u22 dy
          const float dy = Y0 + (float)r - A.y;
          const float2 uy = f2(A.w * dy);
          const float z2 = Bv.x * dy;
          const float2 nc = f2(fmaf(z2, z2, -Bv.y));
          const float2 z01 = add2(ux01, uy), z23 = add2(ux23, uy);
          const float2 f01 = fma2(z01, z01, nc), f23 = fma2(z23, z23, nc);
          if (kCount) {
            nkept += (f01.x < nl2tau) + (f01.y < nl2tau) + (f23.x < nl2tau) + (f23.y < nl2tau);
          } else {
            // value on kept pairs (value > tau), zero elsewhere
            acc[2 * r] = fma2(make_float2(ex2_approx(-f01.x), ex2_approx(-f01.y)),
                              make_float2(set_lt(f01.x, nl2tau), set_lt(f01.y, nl2tau)), acc[2 * r]);
            acc[2 * r + 1] =
                fma2(make_float2(ex2_approx(-f23.x), ex2_approx(-f23.y)),
                     make_float2(set_lt(f23.x, nl2tau), set_lt(f23.y, nl2tau)), acc[2 * r + 1]);
          }
        }
        if (kCount) neval += 16;
      }
      if (!kCount) {
#pragma unroll
        for (int r = 0; r < 4; ++r)
          part[k + tid][r] =
              make_float4(acc[2 * r].x, acc[2 * r].y, acc[2 * r + 1].x, acc[2 * r + 1].y);
      }
    }
    if (kCount) continue;
    __syncthreads();
    // each owned pixel sums the pieces of its block in thread order (runs
    // in list order), then joins its running sum (Kahan)
    {
      const int pk = ps[ob], pe = ps[ob + 1];
      if (pe > pk) {
        // threads holding items pk and pe - 1
        const int ulo = (kThreads * (pk + 1) + N - 1) / N - 1;
        const int uhi = (kThreads * pe + N - 1) / N - 1;
        float2 w = make_float2(0.f, 0.f);
        for (int u = ulo; u <= uhi; ++u) {
          if (((u * N) >> 7) == (((u + 1) * N) >> 7)) continue;  // empty run
          const float2 v = reinterpret_cast<const float2 *>(&part[ob + u][ow >> 1])[ow & 1];
          w.x += v.x;
          w.y += v.y;
        }
        own0 = kahan_add(own0, w.x);
        own1 = kahan_add(own1, w.y);
      }
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
  const int px = x0 + 4 * (ob & 3) + 2 * (ow & 1), py = y0 + 4 * (ob >> 2) + (ow >> 1);
  *reinterpret_cast<float2 *>(proj + ((int64_t)b * d + py) * d + px) =
      make_float2(own0.x - own0.y, own1.x - own1.y);
}

// a3, block-aligned form.  The window's (block, record) items are laid out
// block after block as above, but the 128 threads are shared among the
// blocks in proportion to their item counts (every non-empty block gets at
// least one thread: thread range [T_k, T_k+1) with T_k = (non-empty blocks
// before k) + floor((128 - non-empty) * start_k / N)), and a block's threads
// take its items interleaved.  A thread never leaves its block, so each thread ends
// the window with one partial image of its block (16 pixels), and each pixel
// sums the partials of its block's thread range in thread order (runs in
// list order), then joins its running sum with Kahan compensation.  The
// longest run is within 128 / (128 - 16) of the mean.  kSub sub-windows of
// 128 records make a window; flat slots are bytes up to 256 records.
template <int kSubW>
struct FlatSlot {
  using T = typename std::conditional<(kSubW * 128 <= 256), unsigned char, unsigned short>::type;
};

template <int kSubW, int kMinB, bool kCount>
__global__ void __launch_bounds__(kThreads, kMinB) raster_fwd_aligned_kernel(
    const Rec *__restrict__ rec, const uint2 *__restrict__ list,
    const int64_t *__restrict__ tile_start, int64_t cap,
    int64_t M, int d, float l2tau, const uint32_t *__restrict__ order, int ntiles,
    unsigned *__restrict__ next_tile, float *__restrict__ proj,
    unsigned long long *__restrict__ kept) {
  constexpr int kWarps = kThreads / 32;
  constexpr int kWinW = kThreads * kSubW;
  using Slot = typename FlatSlot<kSubW>::T;
  __shared__ float4 sa[kWinW];                        // px, py, u11, u12
  __shared__ float2 sb[kWinW];                        // u22, log2 A
  __shared__ Slot flat[16 * kWinW];                   // staged slot of each (block, record) item
  __shared__ unsigned short wcnt[kSubW][kWarps][16];  // per sub-window, warp, block: how many
  __shared__ unsigned wbal[kSubW][kWarps][16];        // per sub-window, warp, block: which lanes
  __shared__ int woff[kWarps][kSubW][16];             // where a warp's records go in flat
  __shared__ int pstart[kWarps][17];                  // block k's items: [pstart[k], pstart[k+1])
  __shared__ int tfirst[kWarps][17];                  // block k's threads: [tfirst[k], tfirst[k+1])
  __shared__ float4 part[kThreads][4];                // each thread's partial image of its block
  __shared__ int tile_sh;
  const int nt = d / kTile, T = nt * nt;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const float nl2tau = -l2tau;  // kept: -e < -log2(tau)
  const unsigned lt = (1u << lane) - 1u;
  // pixels owned across windows: two columns of one row of block ob
  const int ob = tid >> 3, ow = tid & 7;
  unsigned nkept = 0, neval = 0;
  // tiles come from the grid (order == nullptr) or, in the persistent form,
  // from a shared counter over a longest-first order
  for (int it = 0;; ++it) {
    int bt;
    if (order == nullptr) {
      if (it > 0) break;
      bt = blockIdx.y * T + blockIdx.x;
    } else {
      __syncthreads();  // every thread has read the previous tile_sh
      if (tid == 0) tile_sh = (int)atomicAdd(next_tile, 1u);
      __syncthreads();
      const int q = tile_sh;
      if (q >= ntiles) break;
      bt = (int)order[q];
    }
    const int b = bt / T, t = bt - b * T;
    const int tx = t % nt, ty = t / nt;
    const int x0 = tx * kTile, y0 = ty * kTile;
    int64_t s = tile_start[bt];
    int64_t e = tile_start[bt + 1];
    e = min(e, cap);
    s = min(s, e);
    // lists that overflowed their capacity are incomplete: every list
    // counts as empty (the status word reports it)
    if (tile_start[order == nullptr ? (int64_t)gridDim.y * T : (int64_t)ntiles] > cap) e = s;
    const Rec *rb = rec + (int64_t)b * M;
    float2 own0 = make_float2(0.f, 0.f), own1 = make_float2(0.f, 0.f);  // Kahan (sum, comp)
    for (int64_t base = s; base < e; base += kWinW) {
      const int n = (int)min((int64_t)kWinW, e - base);
      __syncthreads();  // previous window fully consumed
      unsigned m[kSubW];
#pragma unroll
      for (int u = 0; u < kSubW; ++u) {
        const int slot = u * kThreads + tid;
        m[u] = 0;
        // an entry whose Gaussian index is out of range (a list position
        // left unwritten when the lists overflowed their capacity) counts as
        // empty
        const uint2 ent = slot < n ? list[base + slot] : make_uint2(0u, 0u);
        const uint32_t jj = ent.x;
        if (slot < n && jj < (uint64_t)M) {
          const Rec *rp = rb + jj;
          const float4 ra = rp->a;
          const float2 rbv = *reinterpret_cast<const float2 *>(&rp->b);
          m[u] = ent.y & 0xffffu;
          sa[slot] = ra;
          sb[slot] = rbv;
        }
      }
      // which of this warp's records touch block k, both sub-windows at once:
      // lane k < 16 gets block k of sub-window 0, lane 16 + k block k of
      // sub-window 1 (the lanes' packed masks, transposed as a bit matrix)
      static_assert(kSubW == 2, "two 16-bit masks per lane");
      {
        const unsigned bal = warp_transpose32(m[0] | (m[1] << 16), lane);
        wcnt[lane >> 4][warp][lane & 15] = (unsigned short)__popc(bal);
        wbal[lane >> 4][warp][lane & 15] = bal;
      }
      __syncthreads();
      // every warp: block lengths, their prefix, where its own records go,
      // and the thread ranges of the blocks
      {
        int len = 0, wo[kSubW];
#pragma unroll
        for (int u = 0; u < kSubW; ++u) {
          wo[u] = 0;
#pragma unroll
          for (int w = 0; w < kWarps; ++w) {
            if (w == warp) wo[u] = len;
            if (lane < 16) len += wcnt[u][w][lane];
          }
        }
        int incl = len, ne = (lane < 16 && len > 0) ? 1 : 0;
#pragma unroll
        for (int o = 1; o < 16; o <<= 1) {
          const int v = __shfl_up_sync(0xffffffffu, incl, o);
          const int c = __shfl_up_sync(0xffffffffu, ne, o);
          if (lane >= o) {
            incl += v;
            ne += c;
          }
        }
        const int N = __shfl_sync(0xffffffffu, incl, 15);
        const int nne = __shfl_sync(0xffffffffu, ne, 15);
        if (lane < 16) {
          const int st = incl - len;
          pstart[warp][lane] = st;
#pragma unroll
          for (int u = 0; u < kSubW; ++u) woff[warp][u][lane] = st + wo[u];
          // non-empty blocks before this one, plus its share of the rest
          const int neb = ne - ((len > 0) ? 1 : 0);
          // floor(a / N) for a = (128 - nne) st < 2^19, N <= 16 kWinW: a / N is a
          // multiple of 1 / N, so (a + 1/2) / N sits at least 1 / (2 N) from
          // an integer, far more than the few-ulp error of the fast division
          const float a = (float)((kThreads - nne) * st) + 0.5f;
          tfirst[warp][lane] = neb + (N > 0 ? (int)__fdividef(a, (float)N) : 0);
        }
        if (lane == 15) {
          pstart[warp][16] = incl;
          tfirst[warp][16] = kThreads;
        }
        __syncwarp();
      }
#pragma unroll
      for (int u = 0; u < kSubW; ++u) {
        for (unsigned mm = m[u]; mm; mm &= mm - 1) {
          const int k = __ffs(mm) - 1;
          flat[woff[warp][u][k] + __popc(wbal[u][warp][k] & lt)] = (Slot)(u * kThreads + tid);
        }
      }
      __syncthreads();
      // this thread's block and its share of the block's items
      const int *ps = pstart[warp];
      const int *tf = tfirst[warp];
      int k = 0;
#pragma unroll
      for (int q = 8; q >= 1; q >>= 1)
        if (k + q <= 15 && tf[k + q] <= tid) k += q;
      // tf is non-decreasing and tf[16] = 128 > tid: k is the last block
      // whose range starts at or before tid; an empty block's range is empty
      const int t0 = tf[k], tk = tf[k + 1] - t0;
      float2 acc[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) acc[q] = make_float2(0.f, 0.f);
      if (tk > 0 && tid < tf[k + 1]) {
        const int j = tid - t0;
        // the block's threads take its items interleaved (thread j: items
        // j, j + tk, ...), each in list order; at every step they read
        // neighbouring items, whose slots ascend, which spreads the record
        // gathers over the banks better than contiguous runs did
        const int L = ps[k + 1] - ps[k];
        const float X0 = (float)(x0 + 4 * (k & 3)), Y0 = (float)(y0 + 4 * (k >> 2));
        const float2 xs01 = make_float2(X0, X0 + 1.f), xs23 = make_float2(X0 + 2.f, X0 + 3.f);
        for (int i = ps[k] + j; i < ps[k] + L; i += tk) {
          const int slot = flat[i];
          const float4 A = sa[slot];
          const float2 Bv = sb[slot];
          const float2 npx = f2(-A.x);
          const float2 dx01 = add2(xs01, npx);
          const float2 dx23 = add2(xs23, npx);
          const float2 u11 = f2(A.z);
          const float2 ux01 = mul2(u11, dx01), ux23 = mul2(u11, dx23);
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            // -e = z1^2 + (z2^2 - l2A), z1 = u11 dx + u12 dy, z2 = u22 dy
            const float dy = Y0 + (float)r - A.y;
            const float2 uy = f2(A.w * dy);
            const float z2 = Bv.x * dy;
            const float2 nc = f2(fmaf(z2, z2, -Bv.y));
            const float2 z01 = add2(ux01, uy), z23 = add2(ux23, uy);
            const float2 f01 = fma2(z01, z01, nc), f23 = fma2(z23, z23, nc);
            if (kCount) {
              nkept += (f01.x < nl2tau) + (f01.y < nl2tau) + (f23.x < nl2tau) + (f23.y < nl2tau);
            } else {
              // value on kept pairs (value > tau), zero elsewhere
              acc[2 * r] = fma2(make_float2(ex2_approx(-f01.x), ex2_approx(-f01.y)),
                                make_float2(set_lt(f01.x, nl2tau), set_lt(f01.y, nl2tau)), acc[2 * r]);
              acc[2 * r + 1] =
                  fma2(make_float2(ex2_approx(-f23.x), ex2_approx(-f23.y)),
                       make_float2(set_lt(f23.x, nl2tau), set_lt(f23.y, nl2tau)), acc[2 * r + 1]);
            }
          }
          if (kCount) neval += 16;
        }
      }
      if (!kCount) {
#pragma unroll
        for (int r = 0; r < 4; ++r)
          part[tid][r] = make_float4(acc[2 * r].x, acc[2 * r].y, acc[2 * r + 1].x, acc[2 * r + 1].y);
        __syncthreads();
        // each owned pixel sums its block's partials in thread order (runs
        // in list order), then joins its running sum (Kahan)
        const int u0 = tf[ob], u1 = tf[ob + 1];
        float2 w = make_float2(0.f, 0.f);
        for (int u = u0; u < u1; ++u) {
          const float2 v = reinterpret_cast<const float2 *>(&part[u][ow >> 1])[ow & 1];
          w.x += v.x;
          w.y += v.y;
        }
        if (u1 > u0) {
          own0 = kahan_add(own0, w.x);
          own1 = kahan_add(own1, w.y);
        }
      }
    }
    if (!kCount) {
      const int px = x0 + 4 * (ob & 3) + 2 * (ow & 1), py = y0 + 4 * (ob >> 2) + (ow >> 1);
      *reinterpret_cast<float2 *>(proj + ((int64_t)b * d + py) * d + px) =
          make_float2(own0.x - own0.y, own1.x - own1.y);
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
  }
}

// Longest-first order of the B*T tiles for the persistent forms: a counting
// sort of the tiles by the bit length of their list length (32 classes,
// longest class first), so that the longest tiles start in the first wave
// and the launch does not end waiting for one.  One CTA walks the tiles in
// index order, 1024 at a time, so within a class the order follows the
// index (image after image) up to the order of the warps of one round.  CTA
// 0 also resets the work counter.  Which tile runs when changes nothing in
// its result.  Lanes of a warp with the same class share one shared-memory
// atomic (tiles mostly fall in a few classes).  (Ordering image by image,
// longest tile first within each image, kept more records in L2 but ran
// slower: the long tiles of the last images started late.)
__device__ __forceinline__ int tile_class(const int64_t *__restrict__ tile_start, int64_t i) {
  const int64_t len = tile_start[i + 1] - tile_start[i];
  return 31 - min(31, 64 - __clzll((unsigned long long)max(len, (int64_t)0)));
}

__global__ void __launch_bounds__(1024) tile_order_kernel(const int64_t *__restrict__ tile_start,
                                                         int ntiles, uint32_t *__restrict__ order,
                                                         unsigned *__restrict__ next_tile) {
  __shared__ unsigned hist[32], cur[32];
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  if (threadIdx.x < 32) hist[threadIdx.x] = 0;
  __syncthreads();
  // every warp runs the same number of rounds, so all its lanes take part in
  // each match
  const int rounds = (ntiles + blockDim.x - 1) / blockDim.x;
  for (int r = 0; r < rounds; ++r) {
    const int i = r * blockDim.x + threadIdx.x;
    const int c = i < ntiles ? tile_class(tile_start, i) : 32 + lane;
    const unsigned peers = __match_any_sync(0xffffffffu, c);
    if (c < 32 && (peers & lt) == 0) atomicAdd(&hist[c], (unsigned)__popc(peers));
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned run = 0;
    for (int c = 0; c < 32; ++c) {
      cur[c] = run;
      run += hist[c];
    }
    *next_tile = 0u;
  }
  __syncthreads();
  for (int r = 0; r < rounds; ++r) {
    const int i = r * blockDim.x + threadIdx.x;
    const int c = i < ntiles ? tile_class(tile_start, i) : 32 + lane;
    const unsigned peers = __match_any_sync(0xffffffffu, c);
    const int leader = __ffs(peers) - 1;
    unsigned base = 0;
    if (c < 32 && lane == leader) base = atomicAdd(&cur[c], (unsigned)__popc(peers));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (c < 32) order[base + __popc(peers & lt)] = (uint32_t)i;
    __syncthreads();  // rounds in index order
  }
}

// The forward's kernel configurations (the autotuner's search space).
static const FwdCfg kFwdCfgs[] = {
    {0, 2, 9, 0, 0, "runs, 256-record windows, 9 CTAs/SM"},
    {1, 2, 9, 0, 0, "aligned, 256-record windows, 9 CTAs/SM"},
    {1, 2, 8, 0, 0, "aligned, 256-record windows, 8 CTAs/SM"},
    {1, 2, 9, 1, 9, "aligned, 256-record windows, 9 CTAs/SM, persistent longest-first"},
    {1, 2, 8, 1, 8, "aligned, 256-record windows, 8 CTAs/SM, persistent longest-first"},
    {1, 2, 8, 1, 7, "aligned, 256-record windows, 7 CTAs/SM, persistent longest-first"},
    {1, 2, 8, 1, 6, "aligned, 256-record windows, 6 CTAs/SM, persistent longest-first"},
    {1, 2, 8, 1, 5, "aligned, 256-record windows, 5 CTAs/SM, persistent longest-first"},
};
int fwd_config_count() { return (int)(sizeof(kFwdCfgs) / sizeof(kFwdCfgs[0])); }
const FwdCfg &fwd_config(int i) { return kFwdCfgs[i]; }

template <int kSubW, int kMinB, bool kCount>
static cudaError_t launch_aligned(const FwdCfg &c, const Rec *rec, const uint2 *list,
                                  const int64_t *tile_start, int64_t cap,
                                  int64_t M, int B, int d, float l2tau, float *proj,
                                  unsigned long long *kept, uint32_t *order, unsigned *next_tile,
                                  cudaStream_t st) {
  const int nt = d / kTile, ntiles = nt * nt * B;
  if (c.persistent) {
    tile_order_kernel<<<1, 1024, 0, st>>>(tile_start, ntiles, order, next_tile);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = max(1, min(ntiles, sms * min(c.ctas, kMinB)));
    raster_fwd_aligned_kernel<kSubW, kMinB, kCount><<<grid, kThreads, 0, st>>>(
        rec, list, tile_start, cap, M, d, l2tau, order, ntiles, next_tile, proj, kept);
  } else {
    dim3 grid(nt * nt, B);
    raster_fwd_aligned_kernel<kSubW, kMinB, kCount><<<grid, kThreads, 0, st>>>(
        rec, list, tile_start, cap, M, d, l2tau, nullptr, 0, nullptr, proj, kept);
  }
  return cudaGetLastError();
}

template <bool kCount>
static cudaError_t launch_fwd_any(int cfg, const Rec *rec, const uint2 *list,
                                  const int64_t *tile_start, int64_t cap,
                                  int64_t M, int B, int d, float l2tau, float *proj,
                                  unsigned long long *kept, uint32_t *order, unsigned *next_tile,
                                  cudaStream_t st) {
  if (cfg < 0 || cfg >= fwd_config_count()) return cudaErrorInvalidValue;
  const FwdCfg &c = kFwdCfgs[cfg];
  if (c.persistent && (order == nullptr || next_tile == nullptr)) return cudaErrorInvalidValue;
  if (c.form == 0) {
    const int nt = d / kTile;
    dim3 grid(nt * nt, B);
    raster_fwd_kernel<kCount><<<grid, kThreads, 0, st>>>(rec, list, tile_start, cap, M, d,
                                                         l2tau, proj, kept);
    return cudaGetLastError();
  }
  if (c.minb == 9)
    return launch_aligned<2, 9, kCount>(c, rec, list, tile_start, cap, M, B, d, l2tau, proj,
                                        kept, order, next_tile, st);
  return launch_aligned<2, 8, kCount>(c, rec, list, tile_start, cap, M, B, d, l2tau, proj,
                                      kept, order, next_tile, st);
}

cudaError_t launch_raster_fwd(int cfg, const Rec *rec, const uint2 *list,
                              const int64_t *tile_start, int64_t cap, int64_t M, int B, int d,
                              float l2tau, float *proj, uint32_t *order, unsigned *next_tile,
                              cudaStream_t st) {
  return launch_fwd_any<false>(cfg, rec, list, tile_start, cap, M, B, d, l2tau, proj,
                               nullptr, order, next_tile, st);
}

cudaError_t launch_count_kept(int cfg, const Rec *rec, const uint2 *list,
                              const int64_t *tile_start, int64_t cap,
                              int64_t M, int B, int d, float l2tau, unsigned long long *kept,
                              uint32_t *order, unsigned *next_tile, cudaStream_t st) {
  return launch_fwd_any<true>(cfg, rec, list, tile_start, cap, M, B, d, l2tau, nullptr,
                              kept, order, next_tile, st);
}

// The g tile is stored [pixel row in block][block ^ g_swizzle(row)]: rows 2
// and 3 have their blocks permuted by k ^ 4, so the two lanes of a record
// in the two-lane form (rows 0 and 2, then 1 and 3 of the same block) read
// different banks (a float4's bank group is its index mod 8).
__device__ __forceinline__ int g_swizzle(int row) { return (row & 2) << 1; }

// The six moments of w = g * value over pixel rows row0 .. row0 + kRows - 1
// of block k of the tile at (x0, y0) for one record (centre A.x, A.y, first
// row of U in A.z, A.w; u22, l2A), in the record's whitened coordinates
// z1 = u11 dx + u12 dy, z2 = u22 dy, added to the running totals
// (n0, n1), (n2, n3), (n4, n5):
//   n0 = sum w, n1 = sum w z1, n2 = sum w z2,
//   n3 = sum w (z1^2 - c^2), n4 = sum w z1 z2, n5 = sum w (z2^2 - c^2)
// (per row: the sums of w, w z1, w z1^2 in packed float pairs, weighted by
// z2, which is constant along a row; the second moments taken about c^2 I,
// the whitened S^, per block).  sg is the g tile, [pixel row in block][block].
template <int kRows>
__device__ __forceinline__ void block_moments(const float4 (*__restrict__ sg)[16], int k, int x0,
                                              int y0, int row0, const float4 &A, float u22,
                                              float l2A, float nl2tau, float2 &s01, float2 &s23,
                                              float2 &s45) {
  const float2 u11 = f2(A.z);
  const float u12 = A.w;
  // dx and dy rounded exactly as the forward rounds them (pixel index
  // minus centre), so both decide Eq. accu on the same exponent
  const float X0 = (float)(x0 + 4 * (k & 3)), Y0 = (float)(y0 + 4 * (k >> 2) + row0);
  const float2 npx = f2(-A.x);
  const float2 ux01 = mul2(u11, add2(make_float2(X0, X0 + 1.f), npx));
  const float2 ux23 = mul2(u11, add2(make_float2(X0 + 2.f, X0 + 3.f), npx));
  // this block's rows: sums of w, w z1, w z2, w z1^2, w z1 z2, w z2^2
  float m0 = 0.f, m1 = 0.f, m2 = 0.f, m3 = 0.f, m4 = 0.f, m5 = 0.f;
#pragma unroll
  for (int rr = 0; rr < kRows; ++rr) {
    const float dy = Y0 + (float)rr - A.y;
    const float2 uy = f2(u12 * dy);
    const float z2 = u22 * dy;
    const float2 nc = f2(fmaf(z2, z2, -l2A));
    // -e = z1^2 + (z2^2 - l2A), as in the forward's terms
    const float2 z01 = add2(ux01, uy), z23 = add2(ux23, uy);
    const float2 f01 = fma2(z01, z01, nc), f23 = fma2(z23, z23, nc);
    const float4 g4 = sg[row0 + rr][k ^ g_swizzle(row0 + rr)];
    // w = g * value on kept pairs (value > tau), zero elsewhere: g is masked
    // to +0 on the integer pipe, which leaves the FMA pipe (this loop's
    // busiest) the multiply
    const float2 gm01 = make_float2(keep_or_zero(g4.x, f01.x, nl2tau), keep_or_zero(g4.y, f01.y, nl2tau));
    const float2 gm23 = make_float2(keep_or_zero(g4.z, f23.x, nl2tau), keep_or_zero(g4.w, f23.y, nl2tau));
    const float2 w01 = mul2(gm01, make_float2(ex2_approx(-f01.x), ex2_approx(-f01.y)));
    const float2 w23 = mul2(gm23, make_float2(ex2_approx(-f23.x), ex2_approx(-f23.y)));
    // the row's sums of w, w z1 and w z1^2, then weighted by z2
    const float2 wz01 = mul2(w01, z01), wz23 = mul2(w23, z23);
    const float2 s0 = add2(w01, w23);
    const float2 s1 = add2(wz01, wz23);
    const float2 s2 = fma2(wz23, z23, mul2(wz01, z01));
    const float r0 = s0.x + s0.y, r1 = s1.x + s1.y, r2 = s2.x + s2.y;
    m0 += r0;
    m1 += r1;
    m3 += r2;
    m2 = fmaf(r0, z2, m2);
    m4 = fmaf(r1, z2, m4);
    m5 = fmaf(r0 * z2, z2, m5);
  }
  // second moments about c^2 I, then into the totals
  m3 = fmaf(-kC2, m0, m3);
  m5 = fmaf(-kC2, m0, m5);
  s01 = add2(s01, make_float2(m0, m1));
  s23 = add2(s23, make_float2(m2, m3));
  s45 = add2(s45, make_float2(m4, m5));
}

// kLpr lanes share one record (lane q of the group takes pixel rows
// q * 4 / kLpr .. of every block of the record), so a round runs 32 / kLpr
// records of neighbouring block counts; a warp window holds 32 * kPer
// records.
template <int kLpr, int kPer>
__global__ void __launch_bounds__(kThreads, 8) raster_bwd_kernel(
    const Rec *__restrict__ rec, const uint2 *__restrict__ list,
    const int64_t *__restrict__ tile_start, int64_t cap,
    int64_t M, int d, float l2tau, const float *__restrict__ dproj, double *__restrict__ mom,
    const uint32_t *__restrict__ order, int ntiles, unsigned *__restrict__ next_tile) {
  constexpr int kWarps = kThreads / 32;
  constexpr int kWW = 32 * kPer;     // records per warp window
  constexpr int kRpr = 32 / kLpr;    // records per round
  constexpr int kRows = 4 / kLpr;    // pixel rows of a block per lane
  // g by pixel row within a block and block: [row][block ^ g_swizzle(row)]
  // = 4 pixels (see g_swizzle)
  __shared__ float4 sg[4][16];
  __shared__ float4 sa[kWarps][kWW];  // px, py, u11, u12
  __shared__ float2 sb[kWarps][kWW];  // u22, log2 A
  __shared__ uint32_t sj[kWarps][kWW];
  __shared__ unsigned short smask[kWarps][kWW];
  __shared__ int hist[kWarps][32];
  __shared__ int next_win;
  __shared__ int tile_sh;
  const int nt = d / kTile, T = nt * nt;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float nl2tau = -l2tau;  // kept: -e < -log2(tau)
  const int64_t total = tile_start[order == nullptr ? (int64_t)gridDim.y * T : (int64_t)ntiles];
  // tiles come from the grid (order == nullptr) or, in the persistent form,
  // from a shared counter over a longest-first order
  for (int it = 0;; ++it) {
  int bt;
  if (order == nullptr) {
    if (it > 0) break;
    bt = blockIdx.y * T + blockIdx.x;
  } else {
    __syncthreads();  // every warp is done with the previous tile
    if (threadIdx.x == 0) tile_sh = (int)atomicAdd(next_tile, 1u);
    __syncthreads();
    const int qq = tile_sh;
    if (qq >= ntiles) break;
    bt = (int)order[qq];
  }
  const int b = bt / T, t = bt - b * T;
  const int tx = t % nt, ty = t / nt;
  const int x0 = tx * kTile, y0 = ty * kTile;
  // g tile, stored block by block
  if (threadIdx.x < kTile * kTile / 4) {
    const int r = threadIdx.x >> 2, q = threadIdx.x & 3;  // pixel row, 4-column group
    sg[r & 3][(4 * (r >> 2) + q) ^ g_swizzle(r & 3)] =
        *reinterpret_cast<const float4 *>(dproj + ((int64_t)b * d + y0 + r) * d + x0 + 4 * q);
  }
  if (threadIdx.x == 0) next_win = kWarps;
  __syncthreads();
  int64_t s = tile_start[bt];
  int64_t e = tile_start[bt + 1];
  e = min(e, cap);
  s = min(s, e);
  if (total > cap) e = s;  // overflowed: every list empty
  const Rec *rb = rec + (int64_t)b * M;
  double *mb = mom + (int64_t)b * M * 6;
  int *h = hist[warp];
  const int gq = lane % kLpr;                                   // lane within the record's group
  const unsigned gmask = ((1u << kLpr) - 1u) << (lane - gq);    // the group's lanes
  const int row0 = gq * kRows;
  // warp w takes window w first, then the next window not yet taken; no
  // barrier couples the warps after the g tile is in place
  int64_t base = s + kWW * warp;
  while (base < e) {
    uint32_t j[kPer];
    unsigned m[kPer];
    __syncwarp();  // previous window's reads are done
    h[lane] = 0;
    __syncwarp();
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int64_t i = base + q * 32 + lane;
      j[q] = 0;
      m[q] = 0;
      if (i < e) {
        // the entry's two words read apart, the mask only for a valid index
        // (fewer registers in flight than one 8-byte load per entry)
        const uint32_t *ew = reinterpret_cast<const uint32_t *>(list + i);
        j[q] = ew[0];
        // an out-of-range index (an entry left unwritten when the lists
        // overflowed their capacity) counts as empty
        m[q] = j[q] < (uint64_t)M ? ew[1] & 0xffffu : 0u;
      }
      atomicAdd(&h[__popc(m[q])], 1);
    }
    __syncwarp();
    // exclusive scan of the count histogram, most blocks first: lane v gets
    // the number of records with more than v blocks
    {
      const int c = h[lane];
      int run = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_down_sync(0xffffffffu, run, o);
        if (lane + o < 32) run += u;
      }
      __syncwarp();
      h[lane] = run - c;
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int pos = atomicAdd(&h[__popc(m[q])], 1);
      if (m[q]) {
        const Rec *rp = rb + j[q];
        sa[warp][pos] = rp->a;
        sb[warp][pos] = *reinterpret_cast<const float2 *>(&rp->b);
      }
      sj[warp][pos] = j[q];
      smask[warp][pos] = (unsigned short)m[q];
    }
    __syncwarp();
    // rounds of 32 / kLpr records with neighbouring block counts
#pragma unroll 1
    for (int q = 0; q < kWW / kRpr; ++q) {
      const int slot = q * kRpr + lane / kLpr;
      const unsigned mk = smask[warp][slot];
      if (!mk) continue;  // the whole group skips: the counts are sorted
      const float4 A = sa[warp][slot];
      const float2 Bv = sb[warp][slot];
      float2 s01 = make_float2(0.f, 0.f), s23 = s01, s45 = s01;  // lane totals: (n0, n1), (n2, n3), (n4, n5)
      for (unsigned mm = mk; mm; mm &= mm - 1)
        block_moments<kRows>(sg, __ffs(mm) - 1, x0, y0, row0, A, Bv.x, Bv.y, nl2tau, s01, s23, s45);
      float m0 = s01.x, m1 = s01.y, m2 = s23.x, m3 = s23.y, m4 = s45.x, m5 = s45.y;
#pragma unroll
      for (int o = 1; o < kLpr; o <<= 1) {
        m0 += __shfl_xor_sync(gmask, m0, o);
        m1 += __shfl_xor_sync(gmask, m1, o);
        m2 += __shfl_xor_sync(gmask, m2, o);
        m3 += __shfl_xor_sync(gmask, m3, o);
        m4 += __shfl_xor_sync(gmask, m4, o);
        m5 += __shfl_xor_sync(gmask, m5, o);
      }
      if (gq == 0) {
        double *mo = mb + (int64_t)sj[warp][slot] * 6;
        atomicAdd(mo + 0, (double)m0);
        atomicAdd(mo + 1, (double)m1);
        atomicAdd(mo + 2, (double)m2);
        atomicAdd(mo + 3, (double)m3);
        atomicAdd(mo + 4, (double)m4);
        atomicAdd(mo + 5, (double)m5);
      }
    }
    int wn = 0;
    if (lane == 0) wn = atomicAdd(&next_win, 1);
    base = s + (int64_t)kWW * __shfl_sync(0xffffffffu, wn, 0);
  }
  }  // tiles
}

// The backward's kernel configurations (the autotuner's search space):
// lanes per record, records per lane per warp window, persistent grid and
// its CTAs per SM.
static const BwdCfg kBwdCfgs[] = {
    {2, 4, 0, 0, "2 lanes per record, 128-record warp windows"},
    {1, 4, 0, 0, "1 lane per record, 128-record warp windows"},
    {2, 4, 1, 8, "2 lanes per record, 128-record warp windows, persistent longest-first"},
    {1, 4, 1, 8, "1 lane per record, 128-record warp windows, persistent longest-first"},
    {1, 2, 1, 8, "1 lane per record, 64-record warp windows, persistent longest-first"},
    {1, 8, 1, 7, "1 lane per record, 256-record warp windows, persistent longest-first"},
    {2, 8, 1, 7, "2 lanes per record, 256-record warp windows, persistent longest-first"},
    {1, 4, 1, 6, "1 lane per record, 128-record warp windows, persistent longest-first, 6 CTAs/SM"},
    {1, 8, 1, 6, "1 lane per record, 256-record warp windows, persistent longest-first, 6 CTAs/SM"},
    {1, 8, 1, 5, "1 lane per record, 256-record warp windows, persistent longest-first, 5 CTAs/SM"},
};
int bwd_config_count() { return (int)(sizeof(kBwdCfgs) / sizeof(kBwdCfgs[0])); }
const BwdCfg &bwd_config(int i) { return kBwdCfgs[i]; }

template <int kLpr, int kPer>
static void launch_bwd_lanes(dim3 grid, const Rec *rec, const uint2 *list,
                             const int64_t *tile_start, int64_t cap,
                             int64_t M, int d, float l2tau, const float *dproj, double *mom,
                             const uint32_t *order, int ntiles, unsigned *next_tile,
                             cudaStream_t st) {
  raster_bwd_kernel<kLpr, kPer><<<grid, kThreads, 0, st>>>(rec, list, tile_start, cap, M,
                                                           d, l2tau, dproj, mom, order, ntiles,
                                                           next_tile);
}

cudaError_t launch_raster_bwd(int cfg, const Rec *rec, const uint2 *list,
                              const int64_t *tile_start, int64_t cap, int64_t M, int B, int d,
                              float l2tau, const float *dproj, double *mom, uint32_t *order,
                              unsigned *next_tile, bool order_ready, cudaStream_t st) {
  if (cfg < 0 || cfg >= bwd_config_count()) return cudaErrorInvalidValue;
  const BwdCfg &c = kBwdCfgs[cfg];
  if (c.persistent && (order == nullptr || next_tile == nullptr)) return cudaErrorInvalidValue;
  const int nt = d / kTile, ntiles = nt * nt * B;
  dim3 grid(nt * nt, B);
  const uint32_t *ord = nullptr;
  unsigned *ctr = nullptr;
  if (c.persistent) {
    if (order_ready) {
      const cudaError_t e = cudaMemsetAsync(next_tile, 0, sizeof(unsigned), st);
      if (e != cudaSuccess) return e;
    } else {
      tile_order_kernel<<<1, 1024, 0, st>>>(tile_start, ntiles, order, next_tile);
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    grid = dim3((unsigned)max(1, min(ntiles, sms * c.ctas)), 1);
    ord = order;
    ctr = next_tile;
  }
  if (c.lanes == 2 && c.per == 8)
    launch_bwd_lanes<2, 8>(grid, rec, list, tile_start, cap, M, d, l2tau, dproj, mom, ord,
                           ntiles, ctr, st);
  else if (c.lanes == 2)
    launch_bwd_lanes<2, 4>(grid, rec, list, tile_start, cap, M, d, l2tau, dproj, mom, ord,
                           ntiles, ctr, st);

  else if (c.per == 2)
    launch_bwd_lanes<1, 2>(grid, rec, list, tile_start, cap, M, d, l2tau, dproj, mom, ord,
                           ntiles, ctr, st);
  else if (c.per == 8)
    launch_bwd_lanes<1, 8>(grid, rec, list, tile_start, cap, M, d, l2tau, dproj, mom, ord,
                           ntiles, ctr, st);
  else
    launch_bwd_lanes<1, 4>(grid, rec, list, tile_start, cap, M, d, l2tau, dproj, mom, ord,
                           ntiles, ctr, st);
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
  const float nl2tau = -l2tau;
  double acc = 0.0;
  float part = 0.f;
  for (int64_t j = 0; j < M; ++j) {
    Rec r = rb[j];
    float dx = (float)u - r.a.x, dy = (float)v - r.a.y;
    // -e = z1^2 + (z2^2 - l2A), rounded as the tiled forms round it
    float z1 = __fadd_rn(__fmul_rn(r.a.z, dx), __fmul_rn(r.a.w, dy));
    float z2 = __fmul_rn(r.b.x, dy);
    float ff = __fmaf_rn(z1, z1, __fmaf_rn(z2, z2, -r.b.y));
    float val = ex2_approx(-ff);
    part += ff < nl2tau ? val : 0.f;
    if ((j & 127) == 127) {
      acc += part;
      part = 0.f;
    }
  }
  acc += part;
  if (act) proj[(int64_t)b * d * d + pix] = (float)acc;
}

// One thread per (image, Gaussian), every pixel of the image; the same six
// moments as the tiled backward (whitened coordinates, second moments about
// c^2 I, taken per row).
__global__ void __launch_bounds__(128) dense_bwd_kernel(const Rec *__restrict__ rec, int64_t M,
                                                        int d, float l2tau,
                                                        const float *__restrict__ dproj,
                                                        double *__restrict__ mom) {
  int b = blockIdx.y;
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= M) return;
  Rec r = rec[(int64_t)b * M + j];
  const float *g = dproj + (int64_t)b * d * d;
  const float nl2tau = -l2tau;
  float m[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int v = 0; v < d; ++v) {
    float dy = (float)v - r.a.y;
    float uy = __fmul_rn(r.a.w, dy), z2 = __fmul_rn(r.b.x, dy);
    float nc = __fmaf_rn(z2, z2, -r.b.y);
    float r0 = 0.f, r1 = 0.f, r3 = 0.f;
    for (int u = 0; u < d; ++u) {
      float dx = (float)u - r.a.x;
      float z1 = __fadd_rn(__fmul_rn(r.a.z, dx), uy);
      float ff = __fmaf_rn(z1, z1, nc);
      float val = ex2_approx(-ff);
      float gv = ff < nl2tau ? __ldg(g + (int64_t)v * d + u) * val : 0.f;
      r0 += gv;
      float tt = gv * z1;
      r1 += tt;
      r3 = fmaf(tt, z1, r3);
    }
    m[0] += r0;
    m[1] += r1;
    m[2] = fmaf(z2, r0, m[2]);
    m[3] += fmaf(-kC2, r0, r3);
    m[4] = fmaf(z2, r1, m[4]);
    m[5] = fmaf(fmaf(z2, z2, -kC2), r0, m[5]);
  }
  if (!(r.b.z >= 0.f)) {  // no region above tau: no tile, no moments
#pragma unroll
    for (int k = 0; k < 6; ++k) m[k] = 0.f;
  }
  double *mm = mom + ((int64_t)b * M + j) * 6;
#pragma unroll
  for (int k = 0; k < 6; ++k) mm[k] = (double)m[k];
}

cudaError_t launch_dense_fwd(const Rec *rec, int64_t M, int B, int d, float l2tau, float *proj,
                             cudaStream_t st) {
  dim3 grid((unsigned)(((int64_t)d * d + 255) / 256), B);
  dense_fwd_kernel<<<grid, 256, 0, st>>>(rec, M, d, l2tau, proj);
  return cudaGetLastError();
}

cudaError_t launch_dense_bwd(const Rec *rec, int64_t M, int B, int d, float l2tau,
                             const float *dproj, double *mom, cudaStream_t st) {
  dim3 grid((unsigned)((M + 127) / 128), B);
  dense_bwd_kernel<<<grid, 128, 0, st>>>(rec, M, d, l2tau, dproj, mom);
  return cudaGetLastError();
}

}  // namespace gem
