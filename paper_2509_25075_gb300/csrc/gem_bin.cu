// Step a2 of the GEM hot path: bin the kept (image, Gaussian) pairs into
// 16 x 16 pixel tiles, each tile's Gaussians in ascending depth z'.
//
// Sec. 3.2 (after Eq. accu) sorts the selected Gaussians along z and
// accumulates from the lowest z to the highest.  Here:
//   1. per image, a stable sort of the Gaussians by a 16-bit depth key
//      (written by the preprocess; two 8-bit counting passes, ties keep
//      index order), giving each image's depth order;
//   2. a stable counting sort of the (Gaussian, tile) incidences by tile,
//      fed in depth order, so every tile list comes out in depth order.
// Both are chunked counting sorts: count per chunk, scan per image and bin
// across chunks, then scatter with a rank inside the chunk that preserves
// input order.  The result is deterministic: no position depends on thread
// timing.  Each list entry also gets the mask of the 4x4 pixel blocks of
// its tile that the Gaussian's region above tau meets.  The tile count pass
// does all the geometry (candidate tiles, block-row ranges, block masks) and
// records each hit; the scatter pass only ranks and writes them.
#include "gem_internal.cuh"

namespace gem {

constexpr int kChunkD = 4096;   // elements per chunk, depth passes
constexpr int kDThreads = 512;  // 16 warps x 256 elements
constexpr int kChunkT = 256;    // Gaussians per chunk, tile binning

size_t bin_chunks_depth(int64_t M) { return (size_t)((M + kChunkD - 1) / kChunkD); }
size_t bin_chunks_tiles(int64_t M) { return (size_t)((M + kChunkT - 1) / kChunkT); }

// ------------------------------------------------ depth passes ---------

// Digit of element i: pass 0 reads the low byte of the 16-bit key; pass 1
// reads the high byte carried in the top 8 bits of the packed word
// (high byte << 24 | Gaussian index) that pass 0 wrote.
template <int kPass>
__device__ __forceinline__ unsigned digit_of(const uint16_t *__restrict__ key,
                                             const uint32_t *__restrict__ packed, int64_t i) {
  if (kPass == 0) return key[i] & 255u;
  return packed[i] >> 24;
}

// Histogram of the pass's digit per chunk: cnt[b][c][256].
template <int kPass>
__global__ void __launch_bounds__(kDThreads) digit_count_kernel(
    const uint16_t *__restrict__ key, const uint32_t *__restrict__ packed, int64_t M, int nch,
    uint32_t *__restrict__ cnt) {
  __shared__ uint32_t h[256];
  int c = blockIdx.x, b = blockIdx.y;
  if (threadIdx.x < 256) h[threadIdx.x] = 0;
  __syncthreads();
  int64_t base = (int64_t)b * M + (int64_t)c * kChunkD;
  int64_t lim = min((int64_t)kChunkD, M - (int64_t)c * kChunkD);
  // all of a thread's digits are loaded before the first increment
  constexpr int kEach = kChunkD / kDThreads;
  unsigned dg[kEach];
#pragma unroll
  for (int r = 0; r < kEach; ++r) {
    const int i = threadIdx.x + r * kDThreads;
    dg[r] = i < lim ? digit_of<kPass>(key, packed, base + i) : 256u;
  }
#pragma unroll
  for (int r = 0; r < kEach; ++r)
    if (dg[r] < 256u) atomicAdd(&h[dg[r]], 1u);
  __syncthreads();
  if (threadIdx.x < 256) cnt[((int64_t)b * nch + c) * 256 + threadIdx.x] = h[threadIdx.x];
}

// Turn cnt[b][c][bin] into the output offset (within image b) of the first
// element of chunk c with that digit: per bin, exclusive scan over chunks,
// plus the number of elements of image b with a smaller digit.  Thread
// (g, bin) takes the g-th quarter of the chunks of its bin, 8 loads in
// flight: a pass of range sums, the ranges' and bins' prefixes, a pass that
// writes the offsets.
constexpr int kScanGroups = 4;
__global__ void __launch_bounds__(256 * kScanGroups) digit_scan_kernel(uint32_t *__restrict__ cnt,
                                                                        int nch) {
  __shared__ uint32_t part[kScanGroups][256];
  __shared__ uint32_t wsum[8];
  const int b = blockIdx.x, bin = threadIdx.x & 255, g = threadIdx.x >> 8;
  const int per = (nch + kScanGroups - 1) / kScanGroups;
  const int c0 = min(nch, g * per), c1 = min(nch, c0 + per);
  uint32_t *col = cnt + (int64_t)b * nch * 256 + bin;
  uint32_t sum = 0;
  int c = c0;
  for (; c + 8 <= c1; c += 8) {
    uint32_t v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = col[(int64_t)(c + k) * 256];
#pragma unroll
    for (int k = 0; k < 8; ++k) sum += v[k];
  }
  for (; c < c1; ++c) sum += col[(int64_t)c * 256];
  part[g][bin] = sum;
  __syncthreads();
  uint32_t before = 0, tot = 0;
#pragma unroll
  for (int q = 0; q < kScanGroups; ++q) {
    const uint32_t v = part[q][bin];
    if (q < g) before += v;
    tot += v;
  }
  // exclusive prefix of the bin totals (group 0's 8 warps hold bins 0..255)
  uint32_t incl = tot;
  const int lane = threadIdx.x & 31, warp = bin >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (g == 0 && lane == 31) wsum[warp] = incl;
  __syncthreads();
  uint32_t run = incl - tot + before;
  for (int w = 0; w < warp; ++w) run += wsum[w];
  c = c0;
  for (; c + 8 <= c1; c += 8) {
    uint32_t v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = col[(int64_t)(c + k) * 256];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      col[(int64_t)(c + k) * 256] = run;
      run += v[k];
    }
  }
  for (; c < c1; ++c) {
    const uint32_t v = col[(int64_t)c * 256];
    col[(int64_t)c * 256] = run;
    run += v;
  }
}

// Lanes of the warp holding the same kBits-bit value: one ballot per bit
// (faster here than a match instruction).
template <int kBits>
__device__ __forceinline__ unsigned same_value_lanes(int v) {
  unsigned p = 0xffffffffu;
#pragma unroll
  for (int bit = 0; bit < kBits; ++bit) {
    const bool set = (v >> bit) & 1;
    const unsigned bal = __ballot_sync(0xffffffffu, set);
    p &= set ? bal : ~bal;
  }
  return p;
}

// Stable scatter.  Warp w of the block owns elements [256 w, 256 w + 256) of
// the chunk and visits them in order, 32 at a time; lanes holding the same
// digit are ranked by lane with a peer mask.  Per-warp digit counts give
// each warp's base inside the chunk.  Pass 0 writes (high byte << 24 | j),
// pass 1 writes j: the image's depth order.
template <int kPass>
__global__ void __launch_bounds__(kDThreads) digit_scatter_kernel(
    const uint16_t *__restrict__ key, const uint32_t *__restrict__ packed, int64_t M, int nch,
    const uint32_t *__restrict__ off, uint32_t *__restrict__ out) {
  constexpr int kWarps = kDThreads / 32;
  constexpr int kPer = kChunkD / kWarps;  // 256
  __shared__ uint32_t wc[kWarps][256];
  int c = blockIdx.x, b = blockIdx.y;
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < kWarps * 256; i += kDThreads) (&wc[0][0])[i] = 0;
  __syncthreads();
  const int64_t cbase = (int64_t)c * kChunkD + warp * kPer;
  const int64_t ibase = (int64_t)b * M;
  const unsigned lt = (1u << lane) - 1u;
  // the warp's 256 elements, loaded once: digit and output word per round
  constexpr int kRounds = kPer / 32;
  int dig[kRounds];
  uint32_t word[kRounds];
#pragma unroll
  for (int r = 0; r < kRounds; ++r) {
    const int64_t e = cbase + r * 32 + lane;
    dig[r] = 256 + lane;  // tail lanes: a value no digit has
    word[r] = 0;
    if (e < M) {
      if (kPass == 0) {
        const uint16_t k = key[ibase + e];
        dig[r] = k & 255;
        word[r] = ((uint32_t)(k >> 8) << 24) | (uint32_t)e;
      } else {
        const uint32_t wd = packed[ibase + e];
        dig[r] = (int)(wd >> 24);
        word[r] = wd & 0xffffffu;
      }
    }
  }
  // per-warp digit counts (order does not matter here: plain increments)
#pragma unroll
  for (int r = 0; r < kRounds; ++r)
    if (dig[r] < 256) atomicAdd(&wc[warp][dig[r]], 1u);
  __syncthreads();
  // exclusive prefix over warps, plus the chunk's offset
  if (threadIdx.x < 256) {
    int bin = threadIdx.x;
    uint32_t run = off[((int64_t)b * nch + c) * 256 + bin];
    for (int w = 0; w < kWarps; ++w) {
      uint32_t v = wc[w][bin];
      wc[w][bin] = run;
      run += v;
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kRounds; ++r) {
    const bool act = cbase + r * 32 + lane < M;
    // a full round has no tail lanes, so the 8 digit bits decide alone;
    // the last round of a chunk also tells tail lanes (digit 256 + lane) apart
    const bool full = cbase + r * 32 + 31 < M;
    unsigned peers = full ? same_value_lanes<8>(dig[r]) : same_value_lanes<9>(dig[r]);
    int leader = __ffs(peers) - 1;
    uint32_t pos = 0;
    if (act) pos = wc[warp][dig[r]] + __popc(peers & lt);
    __syncwarp();
    if (act && lane == leader) wc[warp][dig[r]] += __popc(peers);
    __syncwarp();
    if (act && pos < (uint32_t)M) out[ibase + pos] = word[r];
  }
}

// ------------------------------------------------------ tile binning ----

// Geometry of the region e > log2(tau) - margin of one record, in pixel
// units: Q(dx, dy) = al dx^2 + be dx dy + ga dy^2 <= kap with Q = |U d|^2
// and kap = l2A - log2(tau) + margin, reduced to what the
// block-row ranges need (computed once per record).  Row dy of the region
// spans dx in [c(dy) - h(dy), c(dy) + h(dy)] with
//   c(dy) = -be dy / (2 al),  h(dy) = sqrt(4 al kap - D dy^2) / (2 al),
//   D = 4 al ga - be^2;
// the region's y-extent is +-sqrt(4 al kap / D), its x-extent
// +-sqrt(4 ga kap / D), reached at dy = dyL = be xext / (2 ga) (left) and
// -dyL (right).
struct RowGeo {
  float px, py;  // centre
  float k4a, D;  // 4 al kap (infinite when tau = 0), 4 al ga - be^2
  float i2a, sl; // 1 / (2 al), -be / (2 al)
  float dyL;
  float xext, yext;
};

// The approximate square roots and divisions (a few ulp) are absorbed by the
// margin already in kap, so the ranges stay supersets of the exact ones.
__device__ __forceinline__ float sqrt_approx(float x) {
  x = fmaxf(x, 0.f);
  return x * rsqrtf(fmaxf(x, 1e-30f));
}

__device__ __forceinline__ RowGeo make_row_geo(const Rec &r, float l2tau) {
  // Q = |U d|^2: al = u11^2, be = 2 u11 u12, ga = u12^2 + u22^2, and
  // D = 4 al ga - be^2 = (2 u11 u22)^2 without the cancellation
  const float u11 = r.a.z, u12 = r.a.w, u22 = r.b.x;
  const float al = u11 * u11, be = 2.f * u11 * u12, ga = fmaf(u12, u12, u22 * u22);
  const float kap = r.b.y - l2tau + kMargin;
  RowGeo G;
  G.px = r.a.x;
  G.py = r.a.y;
  G.i2a = __fdividef(0.5f, al);
  G.sl = -__fdividef(u12, u11);
  const float t = 2.f * u11 * u22;
  G.D = t * t;
  G.k4a = 4.f * al * kap;
  const float iD = __fdividef(1.f, G.D);
  G.xext = sqrt_approx(4.f * ga * kap * iD);
  G.yext = sqrt_approx(G.k4a * iD);
  G.dyL = be * G.xext * __fdividef(0.5f, ga);
  return G;
}

// Block columns (4-pixel columns of the whole image, 0 .. nb-1) that the
// region meets in block row by (pixel rows 4 by .. 4 by + 3), packed as
// lo | hi << 8, or kNoRow.  Inside the strip the region's x-range is
// [c - h, c + h] at the strip's two ends, widened to the region's own
// x-extreme where the strip contains the row that reaches it.  Every
// rounding step is explicit (no contraction the compiler could choose per
// call site), so each inlined copy returns the same bits for the same input.
constexpr unsigned kNoRow = 0x00ffu;  // lo = 255 > hi = 0
// sqrt_approx with its product rounded on its own (never fused into a
// neighbouring add)
__device__ __forceinline__ float sqrt_rn_approx(float x) {
  x = fmaxf(x, 0.f);
  return __fmul_rn(x, rsqrtf(fmaxf(x, 1e-30f)));
}
__device__ __forceinline__ unsigned block_row_range(const RowGeo &G, int by, int nb) {
  if (!(G.k4a < INFINITY)) return (unsigned)(nb - 1) << 8;  // tau = 0: every pixel counts
  float a = __fsub_rn((float)(4 * by), G.py), b = __fadd_rn(a, 3.f);
  a = fmaxf(a, -G.yext);
  b = fminf(b, G.yext);
  if (!(a <= b)) return kNoRow;
  const float ha = __fmul_rn(sqrt_rn_approx(__fmaf_rn(__fmul_rn(-G.D, a), a, G.k4a)), G.i2a);
  const float hb = __fmul_rn(sqrt_rn_approx(__fmaf_rn(__fmul_rn(-G.D, b), b, G.k4a)), G.i2a);
  const float ca = __fmul_rn(G.sl, a), cb = __fmul_rn(G.sl, b);
  float xmin = fminf(__fsub_rn(ca, ha), __fsub_rn(cb, hb));
  float xmax = fmaxf(__fadd_rn(ca, ha), __fadd_rn(cb, hb));
  if (G.dyL >= a && G.dyL <= b) xmin = -G.xext;
  if (-G.dyL >= a && -G.dyL <= b) xmax = G.xext;
  // columns bx whose pixel centres [4 bx, 4 bx + 3] meet [px + xmin, px + xmax]
  const float lo = fmaxf(ceilf(__fmul_rn(__fsub_rn(__fadd_rn(G.px, xmin), 3.f), 0.25f)), 0.f);
  const float hi = fminf(floorf(__fmul_rn(__fadd_rn(G.px, xmax), 0.25f)), (float)(nb - 1));
  if (!(lo <= hi)) return kNoRow;
  return (unsigned)lo | ((unsigned)hi << 8);
}

// Shared staging of one chunk of 256 Gaussians (depth order): each
// Gaussian's row geometry, candidate tile rectangle (the tiles its extent
// box meets) and block-row range, with exclusive prefixes of the candidate
// and block-row counts, so that the chunk's (Gaussian, block row) and
// (Gaussian, candidate tile) items can be spread evenly over the threads
// whatever the Gaussians' sizes.  Each block row's column range is computed
// once and shared by every candidate tile of the Gaussian in that row.
constexpr int kOwnerCap = 2048;  // candidates per chunk with a byte owner map and cached masks
constexpr int kRowCap = 2048;    // block rows per chunk whose ranges are staged

struct ChunkStage {
  RowGeo geo[kChunkT];
  unsigned rect[kChunkT];  // tx0 | ty0 << 8 | width << 16 | first block row << 24
  float inv_w[kChunkT];    // 1 / width, to split a candidate index into rows
  int off[kChunkT + 1];    // exclusive prefix of candidate counts; off[kChunkT] = total
  int roff[kChunkT + 1];   // exclusive prefix of block-row counts; roff[kChunkT] = rows
  int wsum[kChunkT / 32], wrow[kChunkT / 32];
  unsigned char owner[kOwnerCap];   // owner slot of each candidate (when they fit)
  unsigned short cmask[kOwnerCap];  // block mask of each candidate (when they fit)
  unsigned char rowner[kRowCap];    // owner slot of each block row (when they fit)
  unsigned short rowx[kRowCap];     // block-row column ranges (when they fit)
};

// A Gaussian whose extent box meets at most 2 x 2 tiles (most of them, for
// Gaussians of a few pixels) is binned by its own thread: its block-row
// ranges go straight into up to four tile masks held in registers, and it
// takes no part in the chunk's (Gaussian, block row) and (Gaussian,
// candidate) items.  w = 0: not such a Gaussian.
struct SmallBox {
  int tx0, ty0, w, by0, by1;  // first tile, tile columns (1 or 2), block rows by0..by1
};

__device__ __forceinline__ void stage_chunk(ChunkStage &S, const Rec *__restrict__ rec,
                                            const uint32_t *__restrict__ perm, int64_t M,
                                            int b, int c, int d, float l2tau, SmallBox &sbx) {
  const int i = threadIdx.x, lane = i & 31, warp = i >> 5;
  const int64_t r = (int64_t)c * kChunkT + i;
  int ncand = 0, nrow = 0;
  unsigned packed = 0;
  sbx.w = 0;
  if (r < M) {
    const uint32_t j = perm ? perm[(int64_t)b * M + r] : (uint32_t)r;
    const Rec rc = rec[(int64_t)b * M + j];
    S.geo[i] = make_row_geo(rc, l2tau);
    int ulo, uhi, vlo, vhi;
    if (pixel_range(rc.a.x, rc.b.z, d, ulo, uhi) && pixel_range(rc.a.y, rc.b.w, d, vlo, vhi)) {
      const int tx0 = ulo / kTile, ty0 = vlo / kTile;
      const int w = uhi / kTile - tx0 + 1, h = vhi / kTile - ty0 + 1;
      if (w <= 2 && h <= 2) {
        sbx.tx0 = tx0;
        sbx.ty0 = ty0;
        sbx.w = w;
        sbx.by0 = vlo >> 2;
        sbx.by1 = vhi >> 2;
      } else {
        ncand = w * h;
        nrow = (vhi >> 2) - (vlo >> 2) + 1;
        packed = (unsigned)tx0 | ((unsigned)ty0 << 8) | ((unsigned)w << 16) |
                 ((unsigned)(vlo >> 2) << 24);
        S.inv_w[i] = 1.f / (float)w;
      }
    }
  }
  S.rect[i] = packed;
  // both counts in one scan: a warp's candidates fit 17 bits (32 x 48 x 48),
  // its block rows 13 (32 x 192)
  int inc = ncand | (nrow << 17);
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int v = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += v;
  }
  const int incc = inc & 0x1ffff, incr = inc >> 17;
  if (lane == 31) {
    S.wsum[warp] = incc;
    S.wrow[warp] = incr;
  }
  __syncthreads();
  int base = 0, total = 0, rbase = 0, rows = 0;
#pragma unroll
  for (int w = 0; w < kChunkT / 32; ++w) {
    if (w < warp) {
      base += S.wsum[w];
      rbase += S.wrow[w];
    }
    total += S.wsum[w];
    rows += S.wrow[w];
  }
  const int my = base + incc - ncand, myr = rbase + incr - nrow;
  S.off[i] = my;
  S.roff[i] = myr;
  if (i == 0) {
    S.off[kChunkT] = total;
    S.roff[kChunkT] = rows;
  }
  if (total <= kOwnerCap)
    for (int q = 0; q < ncand; ++q) S.owner[my + q] = (unsigned char)i;
  if (rows <= kRowCap)
    for (int q = 0; q < nrow; ++q) S.rowner[myr + q] = (unsigned char)i;
  __syncthreads();
}

// Tile of candidate q (row-major in its rectangle) of a staged Gaussian.
// q < 48 * 48 and w <= 48, so (q + 1/2) / w in float32 is at least 1 / (2 w)
// away from an integer and its floor is the exact row.
__device__ __forceinline__ void candidate_tile(const ChunkStage &S, int o, int q, int &tx,
                                               int &ty) {
  const unsigned pr = S.rect[o];
  const int w = (int)((pr >> 16) & 0xffu);
  const int row = (int)(((float)q + 0.5f) * S.inv_w[o]);
  tx = (int)(pr & 0xffu) + (q - row * w);
  ty = (int)((pr >> 8) & 0xffu) + row;
}

// Owner (Gaussian slot) of candidate k: from the byte map when the chunk's
// candidates fit it, else the last slot whose offset is <= k.
__device__ __forceinline__ int candidate_owner(const ChunkStage &S, int k, int total) {
  if (total <= kOwnerCap) return S.owner[k];
  int lo = 0, hi = kChunkT - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (S.off[mid] <= k) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// 4x4-block mask of candidate tile (tx, ty) of slot o: bit 4 lb + bx set when
// the Gaussian's range in block row 4 ty + lb covers block column 4 tx + bx.
// The rows come from the staging, or, when the chunk's rows did not fit it,
// from block_row_range directly; either way the count and the write pass of
// a candidate get the same bits.
__device__ __forceinline__ unsigned candidate_mask(const ChunkStage &S, bool staged, int o,
                                                   int tx, int ty, int nb) {
  const int by0 = (int)(S.rect[o] >> 24), r0 = S.roff[o], nr = S.roff[o + 1] - r0;
  const int bx0 = 4 * tx;
  unsigned m = 0;
#pragma unroll
  for (int lb = 0; lb < 4; ++lb) {
    const int rr = 4 * ty + lb - by0;
    if (rr < 0 || rr >= nr) continue;
    const unsigned v = staged ? (unsigned)S.rowx[r0 + rr] : block_row_range(S.geo[o], by0 + rr, nb);
    const int l = max((int)(v & 255u), bx0), h = min((int)(v >> 8), bx0 + 3);
    if (l <= h) m |= ((1u << (h - l + 1)) - 1u) << (4 * lb + l - bx0);
  }
  return m;
}

// Per chunk of 256 Gaussians (depth order) of image b: how many hit each
// tile, tcnt[b][c][t] (one contiguous row per chunk); and every hit, (slot o in the chunk, tile, 4x4-block
// mask), in a run of hits[] claimed from a shared cursor, so that the scatter
// pass repeats none of the geometry.  A candidate tile is a hit when its
// block mask is not empty.  The run's contents and layout (threads in
// order, each thread's candidates in order) do not depend on timing; only
// where it starts does.
__device__ __forceinline__ uint64_t pack_hit(int o, int t, unsigned mask) {
  return (uint64_t)o | ((uint64_t)t << 8) | ((uint64_t)mask << 24);
}

__global__ void __launch_bounds__(kChunkT, 6) tile_count_kernel(
    const Rec *__restrict__ rec, const uint32_t *__restrict__ perm, int64_t M, int d,
    float l2tau, int nch, uint32_t *__restrict__ tcnt, BinScratch bs) {
  extern __shared__ uint32_t tc[];
  __shared__ ChunkStage S;
  __shared__ int wh[kChunkT / 32];
  __shared__ int64_t run_base;
  const int c = blockIdx.x, b = blockIdx.y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nt = d / kTile, T = nt * nt, nb = d / 4;
  for (int i = threadIdx.x; i < T; i += blockDim.x) tc[i] = 0;
  SmallBox sbx;
  stage_chunk(S, rec, perm, M, b, c, d, l2tau, sbx);
  const int total = S.off[kChunkT], rows = S.roff[kChunkT];
  const bool staged = rows <= kRowCap;
  if (staged && rows > 0) {  // (rows is the chunk's: the barrier is uniform)
    // (Gaussian, block row) items spread over the threads
    for (int q = threadIdx.x; q < rows; q += kChunkT) {
      const int o = S.rowner[q];
      S.rowx[q] = (unsigned short)block_row_range(S.geo[o], (int)(S.rect[o] >> 24) + q - S.roff[o], nb);
    }
    __syncthreads();
  }
  int nhc = 0;
  for (int k = threadIdx.x; k < total; k += kChunkT) {
    const int o = candidate_owner(S, k, total);
    int tx, ty;
    candidate_tile(S, o, k - S.off[o], tx, ty);
    const unsigned m = candidate_mask(S, staged, o, tx, ty, nb);
    if (total <= kOwnerCap) S.cmask[k] = (unsigned short)m;
    if (m) {
      atomicAdd(&tc[ty * nt + tx], 1u);
      ++nhc;
    }
  }
  // this thread's own Gaussian when it meets at most 2 x 2 tiles (after its
  // share of the candidates, so that one barrier waits for both): the masks
  // of tiles (ty0 + a, tx0 + q) in sm[2 a + q], each row's range clipped to
  // each tile column as candidate_mask clips it
  unsigned sm0 = 0, sm1 = 0, sm2 = 0, sm3 = 0;
  int nhs = 0;
  if (sbx.w > 0) {
    const RowGeo myg = S.geo[threadIdx.x];
    for (int by = sbx.by0; by <= sbx.by1; ++by) {
      const unsigned v = block_row_range(myg, by, nb);
      const int lo = (int)(v & 255u), hi = (int)(v >> 8), sh = 4 * (by & 3);
      const int bx0 = 4 * sbx.tx0;
      unsigned c0 = 0, c1 = 0;
      int l = max(lo, bx0), h = min(hi, bx0 + 3);
      if (l <= h) c0 = ((1u << (h - l + 1)) - 1u) << (sh + l - bx0);
      l = max(lo, bx0 + 4);
      h = min(hi, bx0 + 7);
      if (sbx.w > 1 && l <= h) c1 = ((1u << (h - l + 1)) - 1u) << (sh + l - bx0 - 4);
      if ((by >> 2) == sbx.ty0) {
        sm0 |= c0;
        sm1 |= c1;
      } else {
        sm2 |= c0;
        sm3 |= c1;
      }
    }
    const int t0 = sbx.ty0 * nt + sbx.tx0;
    if (sm0) atomicAdd(&tc[t0], 1u), ++nhs;
    if (sm1) atomicAdd(&tc[t0 + 1], 1u), ++nhs;
    if (sm2) atomicAdd(&tc[t0 + nt], 1u), ++nhs;
    if (sm3) atomicAdd(&tc[t0 + nt + 1], 1u), ++nhs;
  }
  const int nh = nhs + nhc;
  // this thread's hits go after those of lower threads
  int inc = nh;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += v;
  }
  if (lane == 31) wh[warp] = inc;
  __syncthreads();
  int before = inc - nh, H = 0;
#pragma unroll
  for (int w = 0; w < kChunkT / 32; ++w) {
    if (w < warp) before += wh[w];
    H += wh[w];
  }
  if (threadIdx.x == 0) {
    const int64_t base = (int64_t)atomicAdd(bs.hit_ctr, (unsigned long long)H);
    run_base = base;
    bs.chunk_base[(int64_t)b * nch + c] = base;
    bs.chunk_n[(int64_t)b * nch + c] = (uint32_t)H;
  }
  __syncthreads();
  // the same candidates again, in the same order, with the same masks (this
  // thread's own cached ones, or computed again from the same inputs)
  int64_t dst = run_base + before;
  if (nhs > 0) {
    const int o = threadIdx.x, t0 = sbx.ty0 * nt + sbx.tx0;
    auto put = [&](unsigned m, int t) {
      if (!m) return;
      if (dst < bs.cap) bs.hits[dst] = pack_hit(o, t, m);
      ++dst;
    };
    put(sm0, t0);
    put(sm1, t0 + 1);
    put(sm2, t0 + nt);
    put(sm3, t0 + nt + 1);
  }
  for (int k = threadIdx.x; k < total && nhc > 0; k += kChunkT) {
    const unsigned mc = total <= kOwnerCap ? S.cmask[k] : 1u;
    if (!mc) continue;
    const int o = candidate_owner(S, k, total);
    int tx, ty;
    candidate_tile(S, o, k - S.off[o], tx, ty);
    const unsigned m = total <= kOwnerCap ? mc : candidate_mask(S, staged, o, tx, ty, nb);
    if (!m) continue;
    if (dst < bs.cap) bs.hits[dst] = pack_hit(o, ty * nt + tx, m);
    ++dst;
    --nhc;
  }
  __syncthreads();
  uint32_t *out = tcnt + ((int64_t)b * nch + c) * T;
  for (int i = threadIdx.x; i < T; i += blockDim.x) out[i] = tc[i];
}

// Exclusive scan over the chunks of every (image, tile) column of
// tcnt[b][c][t], in place; the column totals go to tile_n[b * T + t].  A
// CTA takes 32 tiles of one image (one per lane, so every access reads 32
// consecutive counts of a chunk row) and its 8 warps take 8 consecutive
// ranges of chunks: a pass of range sums, their exclusive prefix across the
// warps, then a pass that writes the prefix.
constexpr int kScanWarps = 8;
__global__ void __launch_bounds__(32 * kScanWarps) tile_scan_cols_kernel(
    uint32_t *__restrict__ tcnt, int nch, int T, int64_t *__restrict__ tile_n) {
  __shared__ uint32_t part[kScanWarps][32];
  const int b = blockIdx.y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int t = blockIdx.x * 32 + lane;
  const bool act = t < T;
  uint32_t *col = tcnt + (int64_t)b * nch * T + t;
  const int per = (nch + kScanWarps - 1) / kScanWarps;
  const int c0 = min(nch, warp * per), c1 = min(nch, c0 + per);
  // eight loads in flight per lane in both passes (the chunk walk is
  // otherwise one dependent load per step)
  constexpr int kU = 8;
  uint32_t sum = 0;
  if (act) {
    int c = c0;
    for (; c + kU <= c1; c += kU) {
      uint32_t v[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) v[u] = col[(int64_t)(c + u) * T];
#pragma unroll
      for (int u = 0; u < kU; ++u) sum += v[u];
    }
    for (; c < c1; ++c) sum += col[(int64_t)c * T];
  }
  part[warp][lane] = sum;
  __syncthreads();
  uint32_t run = 0;
  for (int w = 0; w < warp; ++w) run += part[w][lane];
  if (act) {
    int c = c0;
    for (; c + kU <= c1; c += kU) {
      uint32_t v[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) v[u] = col[(int64_t)(c + u) * T];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        col[(int64_t)(c + u) * T] = run;
        run += v[u];
      }
    }
    for (; c < c1; ++c) {
      const uint32_t v = col[(int64_t)c * T];
      col[(int64_t)c * T] = run;
      run += v;
    }
    if (warp == kScanWarps - 1) tile_n[(int64_t)b * T + t] = run;
  }
}

// In-place exclusive scan of n counts (one block of 1024), total in x[n].
// Flags the capacity bit when the total exceeds cap.  Each round scans 4096
// counts as four consecutive runs of 1024 (one per sub-round q), with one
// set of barriers; every thread keeps the running carry itself.
__global__ void __launch_bounds__(1024) scan_tiles_kernel(int64_t *__restrict__ x, int64_t n,
                                                          int64_t cap, int *__restrict__ status) {
  constexpr int kQ = 4;
  __shared__ int64_t wtot[kQ][32];  // per run: exclusive prefix of the warps' sums
  __shared__ int64_t qtot[kQ];      // per run: its total
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t carry = 0;
  for (int64_t base = 0; base < n; base += kQ * 1024) {
    int64_t v[kQ], inc[kQ];
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
      const int64_t i = base + q * 1024 + threadIdx.x;
      v[q] = i < n ? x[i] : 0;
    }
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
      inc[q] = v[q];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int64_t u = __shfl_up_sync(0xffffffffu, inc[q], o);
        if (lane >= o) inc[q] += u;
      }
      if (lane == 31) wtot[q][warp] = inc[q];
    }
    __syncthreads();
    if (warp < kQ) {
      const int64_t w = wtot[warp][lane];
      int64_t wi = w;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int64_t u = __shfl_up_sync(0xffffffffu, wi, o);
        if (lane >= o) wi += u;
      }
      wtot[warp][lane] = wi - w;
      if (lane == 31) qtot[warp] = wi;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
      const int64_t i = base + q * 1024 + threadIdx.x;
      if (i < n) x[i] = carry + wtot[q][warp] + inc[q] - v[q];
      carry += qtot[q];
    }
    __syncthreads();  // wtot and qtot are read before the next round rewrites them
  }
  if (threadIdx.x == 0) {
    x[n] = carry;
    if (carry > cap) atomicOr(status, kStatusCapacity);
  }
}

// Scatter: the chunk's hits (from the count pass) set bit o in the bitmap of
// their tile; a hit's place in its tile's list is the tile's start, plus the
// chunk's offset for that tile, plus the number of lower bits set (so the
// list keeps the chunk's depth order).  Beside the Gaussian's index the
// entry stores its 4x4-block mask, both in one 8-byte word (one scattered
// store per hit).  Only the tiles the chunk hits are
// touched: each hit clears its own tile's bitmap words first (a chunk hits
// a few hundred of the image's tiles at most, and large images have
// thousands), and looks up its own tile's list base.
__global__ void __launch_bounds__(kChunkT) tile_scatter_kernel(
    const uint32_t *__restrict__ perm, int64_t M, int d, int nch,
    const uint32_t *__restrict__ tcnt, const int64_t *__restrict__ tile_start, BinScratch bs) {
  // bitmaps word-major, [8][T]: a warp's hits are mostly one Gaussian's
  // neighbouring tiles, which then fall in neighbouring banks
  extern __shared__ __align__(16) uint32_t bm[];
  __shared__ uint32_t sj[kChunkT];   // Gaussian index of each slot
  const int c = blockIdx.x, b = blockIdx.y;
  const int nt = d / kTile, T = nt * nt;
  const int64_t r0 = (int64_t)c * kChunkT;
  if (r0 + threadIdx.x < M)
    sj[threadIdx.x] = perm ? perm[(int64_t)b * M + r0 + threadIdx.x] : (uint32_t)(r0 + threadIdx.x);
  // up to 1024 tiles (d <= 512) every bitmap word is cleared at once, while
  // the hits are still on their way; above that each hit clears its own
  // tile's words once it has arrived
  const bool zero_all = T <= 1024;
  if (zero_all)
    for (int q = 4 * threadIdx.x; q < 8 * T; q += 4 * kChunkT)
      *reinterpret_cast<uint4 *>(bm + q) = make_uint4(0u, 0u, 0u, 0u);
  const int64_t hb = bs.chunk_base[(int64_t)b * nch + c];
  const int64_t hn = min((int64_t)bs.chunk_n[(int64_t)b * nch + c], max(bs.cap - hb, (int64_t)0));
  const int H = (int)hn;
  const uint64_t *hr = bs.hits + hb;
  // the first kHold hits of each thread (i = thread + k * kChunkT) stay in
  // registers across the three phases (the index k is a compile-time
  // constant of an unrolled loop, so the array never leaves registers); a
  // chunk with more hits reads the rest again from global memory
  constexpr int kHold = 4;
  uint64_t hold[kHold];
#pragma unroll
  for (int k = 0; k < kHold; ++k) {
    const int i = threadIdx.x + k * kChunkT;
    hold[k] = i < H ? hr[i] : 0ull;
  }
  auto zero_tile = [&](uint64_t h) {
    const int t = (int)((h >> 8) & 0xffffu);
#pragma unroll
    for (int q = 0; q < 8; ++q) bm[q * T + t] = 0u;
  };
  auto set_bit = [&](uint64_t h) {
    const int o = (int)(h & 255u), t = (int)((h >> 8) & 0xffffu);
    atomicOr(&bm[(o >> 5) * T + t], 1u << (o & 31));
  };
  // list base of a hit's tile: the tile's start plus the chunk's offset in it
  const uint32_t *coff = tcnt + ((int64_t)b * nch + c) * T;
  auto list_base = [&](uint64_t h) {
    const int t = (int)((h >> 8) & 0xffffu);
    return tile_start[(int64_t)b * T + t] + (int64_t)coff[t];
  };
  auto place = [&](uint64_t h, int64_t lb) {
    const int o = (int)(h & 255u), t = (int)((h >> 8) & 0xffffu);
    const uint32_t *bw = bm + t;
    const int word = o >> 5;
    uint32_t rank = __popc(bw[word * T] & ((1u << (o & 31)) - 1u));
    for (int kk = 0; kk < word; ++kk) rank += __popc(bw[kk * T]);
    const int64_t pos = lb + rank;
    if (pos < bs.cap) bs.list[pos] = make_uint2(sj[o], (uint32_t)(h >> 24) & 0xffffu);
  };
  // the held hits' list bases are loaded now, so that their latency passes
  // while the bitmaps are cleared and filled
  int64_t hbase[kHold];
#pragma unroll
  for (int k = 0; k < kHold; ++k)
    hbase[k] = threadIdx.x + k * kChunkT < H ? list_base(hold[k]) : 0;
  if (!zero_all) {
#pragma unroll
    for (int k = 0; k < kHold; ++k)
      if (threadIdx.x + k * kChunkT < H) zero_tile(hold[k]);
    for (int i = threadIdx.x + kHold * kChunkT; i < H; i += blockDim.x) zero_tile(hr[i]);
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kHold; ++k)
    if (threadIdx.x + k * kChunkT < H) set_bit(hold[k]);
  for (int i = threadIdx.x + kHold * kChunkT; i < H; i += blockDim.x) set_bit(hr[i]);
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kHold; ++k)
    if (threadIdx.x + k * kChunkT < H) place(hold[k], hbase[k]);
  for (int i = threadIdx.x + kHold * kChunkT; i < H; i += blockDim.x) {
    const uint64_t h = hr[i];
    place(h, list_base(h));
  }
}

// Bitmaps (8 words per tile, word-major).
static int tile_smem_bytes(int d) {
  int nt = d / kTile;
  return nt * nt * 8 * (int)sizeof(uint32_t);
}

// The dynamic shared memory of both tile kernels (bitmaps, counters) is
// declared for every image side, so that it never depends on what the
// static part leaves of the default 48 KB.
cudaError_t bin_configure(int d) {
  const int smem = tile_smem_bytes(d);
  cudaError_t e = cudaFuncSetAttribute(tile_scatter_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(tile_count_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (d / kTile) * (d / kTile) * (int)sizeof(uint32_t));
}

cudaError_t launch_sort16(const uint16_t *key, int64_t M, int B, uint32_t *dcnt,
                          uint32_t *packed, uint32_t *perm, cudaStream_t st) {
  int nch = (int)bin_chunks_depth(M);
  dim3 g(nch, B);
  // low byte, then high byte (LSD); ties keep index order
  digit_count_kernel<0><<<g, kDThreads, 0, st>>>(key, nullptr, M, nch, dcnt);
  digit_scan_kernel<<<B, 256 * kScanGroups, 0, st>>>(dcnt, nch);
  digit_scatter_kernel<0><<<g, kDThreads, 0, st>>>(key, nullptr, M, nch, dcnt, packed);
  digit_count_kernel<1><<<g, kDThreads, 0, st>>>(nullptr, packed, M, nch, dcnt);
  digit_scan_kernel<<<B, 256 * kScanGroups, 0, st>>>(dcnt, nch);
  digit_scatter_kernel<1><<<g, kDThreads, 0, st>>>(nullptr, packed, M, nch, dcnt, perm);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(256) map_slots_kernel(const uint2 *__restrict__ list,
                                                        const uint32_t *__restrict__ slot_gauss,
                                                        int64_t n, uint32_t *__restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = slot_gauss ? slot_gauss[list[i].x] : list[i].x;
}

cudaError_t launch_map_slots(const uint2 *list, const uint32_t *slot_gauss, int64_t n,
                             uint32_t *out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  map_slots_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(list, slot_gauss, n, out);
  return cudaGetLastError();
}

cudaError_t launch_bin(const Rec *rec, const uint16_t *key, int64_t M, int B, int d,
                       float l2tau, int zsort, BinScratch &s, const uint32_t **perm_out,
                       cudaStream_t st) {
  cudaError_t e;
  const uint32_t *perm = nullptr;
  if (zsort) {
    if ((e = launch_sort16(key, M, B, s.dcnt, s.packed, s.perm, st)) != cudaSuccess) return e;
    perm = s.perm;
  }
  int nt = d / kTile, T = nt * nt;
  int nch = (int)bin_chunks_tiles(M);
  dim3 g(nch, B);
  int cnt_smem = T * (int)sizeof(uint32_t);
  if ((e = cudaMemsetAsync(s.hit_ctr, 0, sizeof(unsigned long long), st)) != cudaSuccess) return e;
  tile_count_kernel<<<g, 256, cnt_smem, st>>>(rec, perm, M, d, l2tau, nch, s.tcnt, s);
  int64_t ncols = (int64_t)B * T;
  tile_scan_cols_kernel<<<dim3((unsigned)((T + 31) / 32), (unsigned)B), 32 * kScanWarps, 0, st>>>(
      s.tcnt, nch, T, s.tile_start);
  scan_tiles_kernel<<<1, 1024, 0, st>>>(s.tile_start, ncols, s.cap, s.status);
  tile_scatter_kernel<<<g, 256, tile_smem_bytes(d), st>>>(perm, M, d, nch, s.tcnt, s.tile_start, s);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  *perm_out = perm;
  return cudaSuccess;
}

}  // namespace gem
