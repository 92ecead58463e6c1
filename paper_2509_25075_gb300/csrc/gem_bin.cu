// Step a2 of the GEM hot path: bin the kept (image, Gaussian) pairs into
// 16 x 16 pixel tiles, each tile's Gaussians in ascending depth z'.
//
// Sec. 3.2 (after Eq. accu) sorts the selected Gaussians along z and
// accumulates from the lowest z to the highest.  Here:
//   1. per image, a stable sort of the Gaussians by a 16-bit depth key
//      (two 8-bit counting passes; ties keep index order), giving a rank;
//   2. a stable counting sort of the (Gaussian, tile) incidences by tile,
//      fed in rank order, so every tile list comes out in depth order.
// Both are chunked counting sorts: count per chunk, scan per image and bin
// across chunks, then scatter with a rank inside the chunk that preserves
// input order.  The result is deterministic: no position depends on thread
// timing.
#include "gem_internal.cuh"

namespace gem {

constexpr int kChunkD = 1024;  // elements per chunk, depth passes
constexpr int kChunkT = 256;   // Gaussians per chunk, tile binning

size_t bin_chunks_depth(int64_t M) { return (size_t)((M + kChunkD - 1) / kChunkD); }
size_t bin_chunks_tiles(int64_t M) { return (size_t)((M + kChunkT - 1) / kChunkT); }

// ------------------------------------------------------ depth key -------

__global__ void __launch_bounds__(256) depth_key_kernel(const float *__restrict__ depth,
                                                        int64_t n, float inv_range,
                                                        uint16_t *__restrict__ key) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  // map [-range, range] onto 0..65535; out-of-range depths clamp
  float z = depth[i] * inv_range;
  float k = floorf((z + 1.f) * 32768.f);
  k = fminf(fmaxf(k, 0.f), 65535.f);
  key[i] = (uint16_t)k;
}

// ------------------------------------------------ counting pass --------

// Histogram of one 8-bit digit per chunk: cnt[b][c][256].
__global__ void __launch_bounds__(256) digit_count_kernel(const uint16_t *__restrict__ key,
                                                          int64_t M, int shift, int nch,
                                                          uint32_t *__restrict__ cnt) {
  __shared__ uint32_t h[256];
  int c = blockIdx.x, b = blockIdx.y;
  h[threadIdx.x] = 0;
  __syncthreads();
  int64_t base = (int64_t)b * M + (int64_t)c * kChunkD;
  int64_t lim = min((int64_t)kChunkD, M - (int64_t)c * kChunkD);
  for (int i = threadIdx.x; i < lim; i += 256) atomicAdd(&h[(key[base + i] >> shift) & 255], 1u);
  __syncthreads();
  cnt[((int64_t)b * nch + c) * 256 + threadIdx.x] = h[threadIdx.x];
}

// Turn cnt[b][c][bin] into the output offset (within image b) of the first
// element of chunk c with that digit: per bin, exclusive scan over chunks,
// plus the number of elements of image b with a smaller digit.
__global__ void __launch_bounds__(256) digit_scan_kernel(uint32_t *__restrict__ cnt, int nch) {
  int b = blockIdx.x, bin = threadIdx.x;
  uint32_t *col = cnt + (int64_t)b * nch * 256 + bin;
  uint32_t run = 0;
  for (int c = 0; c < nch; ++c) {
    uint32_t v = col[(int64_t)c * 256];
    col[(int64_t)c * 256] = run;
    run += v;
  }
  // exclusive scan of the bin totals across the block
  __shared__ uint32_t tot[256];
  tot[bin] = run;
  __syncthreads();
  for (int off = 1; off < 256; off <<= 1) {
    uint32_t v = bin >= off ? tot[bin - off] : 0;
    __syncthreads();
    tot[bin] += v;
    __syncthreads();
  }
  uint32_t base = tot[bin] - run;
  for (int c = 0; c < nch; ++c) col[(int64_t)c * 256] += base;
}

// Stable scatter.  Warp w of the block owns elements [128 w, 128 w + 128) of
// the chunk and visits them in order, 32 at a time; lanes holding the same
// digit are ranked by lane with a match mask.  Per-warp digit counts give
// each warp's base inside the chunk.
__global__ void __launch_bounds__(256) digit_scatter_kernel(
    const uint16_t *__restrict__ kin, const uint32_t *__restrict__ vin, int64_t M, int shift,
    int nch, const uint32_t *__restrict__ off, uint16_t *__restrict__ kout,
    uint32_t *__restrict__ vout) {
  __shared__ uint32_t wc[8][256];
  int c = blockIdx.x, b = blockIdx.y;
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < 8 * 256; i += 256) (&wc[0][0])[i] = 0;
  __syncthreads();
  int64_t cbase = (int64_t)c * kChunkD;
  int64_t ibase = (int64_t)b * M;
  const unsigned lt = (1u << lane) - 1u;
  // pass 1: per-warp digit counts
  for (int r = 0; r < 4; ++r) {
    int64_t e = cbase + warp * 128 + r * 32 + lane;
    int dig = e < M ? ((kin[ibase + e] >> shift) & 255) : 256 + lane;  // tail lanes never match
    unsigned peers = __match_any_sync(0xffffffffu, dig);
    int leader = __ffs(peers) - 1;
    if (dig < 256 && lane == leader) wc[warp][dig] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // exclusive prefix over warps, plus the chunk's global offset
  {
    int bin = threadIdx.x;
    uint32_t run = off[((int64_t)b * nch + c) * 256 + bin];
    for (int w = 0; w < 8; ++w) {
      uint32_t v = wc[w][bin];
      wc[w][bin] = run;
      run += v;
    }
  }
  __syncthreads();
  // pass 2: positions
  for (int r = 0; r < 4; ++r) {
    int64_t e = cbase + warp * 128 + r * 32 + lane;
    bool act = e < M;
    uint16_t k = act ? kin[ibase + e] : 0;
    int dig = act ? ((k >> shift) & 255) : 256 + lane;
    unsigned peers = __match_any_sync(0xffffffffu, dig);
    int leader = __ffs(peers) - 1;
    uint32_t pos = 0;
    if (act) pos = wc[warp][dig] + __popc(peers & lt);
    __syncwarp();
    if (act && lane == leader) wc[warp][dig] += __popc(peers);
    __syncwarp();
    if (act && pos < (uint32_t)M) {
      kout[ibase + pos] = k;
      vout[ibase + pos] = vin ? vin[ibase + e] : (uint32_t)e;
    }
  }
}

// ------------------------------------------------------ tile binning ----

// The tiles a record may touch: the pixel rectangle of its extent, cut to
// the image, then each tile tested exactly against the ellipse.
struct TileRect {
  int tx0, tx1, ty0, ty1;
};

__device__ __forceinline__ bool rec_tiles(const Rec &r, int d, TileRect &tr) {
  int ulo, uhi, vlo, vhi;
  if (!pixel_range(r.a.x, r.b.z, d, ulo, uhi)) return false;
  if (!pixel_range(r.a.y, r.b.w, d, vlo, vhi)) return false;
  tr.tx0 = ulo / kTile;
  tr.tx1 = uhi / kTile;
  tr.ty0 = vlo / kTile;
  tr.ty1 = vhi / kTile;
  return true;
}

__global__ void __launch_bounds__(256) tile_count_kernel(const Rec *__restrict__ rec,
                                                         const uint32_t *__restrict__ perm,
                                                         int64_t M, int d, float l2tau, int nch,
                                                         uint32_t *__restrict__ tcnt) {
  extern __shared__ uint32_t tc[];
  int c = blockIdx.x, b = blockIdx.y;
  int nt = d / kTile, T = nt * nt;
  for (int i = threadIdx.x; i < T; i += blockDim.x) tc[i] = 0;
  __syncthreads();
  int64_t r = (int64_t)c * kChunkT + threadIdx.x;
  if (r < M) {
    uint32_t j = perm ? perm[(int64_t)b * M + r] : (uint32_t)r;
    Rec rc = rec[(int64_t)b * M + j];
    TileRect tr;
    if (rec_tiles(rc, d, tr)) {
      float kappa = rc.b.y - l2tau + kMargin;
      for (int ty = tr.ty0; ty <= tr.ty1; ++ty)
        for (int tx = tr.tx0; tx <= tr.tx1; ++tx)
          if (tile_hit(rc, tx * kTile, ty * kTile, kappa)) atomicAdd(&tc[ty * nt + tx], 1u);
    }
  }
  __syncthreads();
  uint32_t *dst = tcnt + ((int64_t)b * nch + c) * T;
  for (int i = threadIdx.x; i < T; i += blockDim.x) dst[i] = tc[i];
}

// Per (image, tile): exclusive scan of the chunk counts; the tile total goes
// to tile_n[b * T + t].
__global__ void __launch_bounds__(256) tile_scan_cols_kernel(uint32_t *__restrict__ tcnt,
                                                             int nch, int T,
                                                             int64_t *__restrict__ tile_n) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  int b = blockIdx.y;
  if (t >= T) return;
  uint32_t *col = tcnt + (int64_t)b * nch * T + t;
  uint32_t run = 0;
  for (int c = 0; c < nch; ++c) {
    uint32_t v = col[(int64_t)c * T];
    col[(int64_t)c * T] = run;
    run += v;
  }
  tile_n[(int64_t)b * T + t] = run;
}

// In-place exclusive scan of n counts (one block), total in x[n].  Flags the
// capacity bit when the total exceeds cap.
__global__ void __launch_bounds__(1024) scan_tiles_kernel(int64_t *__restrict__ x, int64_t n,
                                                          int64_t cap, int *__restrict__ status) {
  __shared__ int64_t part[1024];
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < n; base += 1024) {
    int64_t i = base + threadIdx.x;
    int64_t v = i < n ? x[i] : 0;
    part[threadIdx.x] = v;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
      int64_t u = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
      __syncthreads();
      part[threadIdx.x] += u;
      __syncthreads();
    }
    if (i < n) x[i] = carry + part[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry += part[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    x[n] = carry;
    if (carry > cap) atomicOr(status, kStatusCapacity);
  }
}

// Scatter: Gaussian i of the chunk (rank order) sets bit i in the bitmap of
// every tile it hits; its position in a tile's list is the tile's start,
// plus the chunk's offset for that tile, plus the number of lower bits set.
__global__ void __launch_bounds__(256) tile_scatter_kernel(
    const Rec *__restrict__ rec, const uint32_t *__restrict__ perm, int64_t M, int d,
    float l2tau, int nch, const uint32_t *__restrict__ tcnt,
    const int64_t *__restrict__ tile_start, int64_t cap, uint32_t *__restrict__ list) {
  extern __shared__ uint32_t bm[];  // [T][8]
  int c = blockIdx.x, b = blockIdx.y;
  int nt = d / kTile, T = nt * nt;
  for (int i = threadIdx.x; i < T * 8; i += blockDim.x) bm[i] = 0;
  __syncthreads();
  int64_t r = (int64_t)c * kChunkT + threadIdx.x;
  int word = threadIdx.x >> 5;
  uint32_t bit = 1u << (threadIdx.x & 31);
  Rec rc;
  TileRect tr;
  uint32_t j = 0;
  bool have = false;
  float kappa = 0.f;
  if (r < M) {
    j = perm ? perm[(int64_t)b * M + r] : (uint32_t)r;
    rc = rec[(int64_t)b * M + j];
    have = rec_tiles(rc, d, tr);
    kappa = rc.b.y - l2tau + kMargin;
  }
  if (have)
    for (int ty = tr.ty0; ty <= tr.ty1; ++ty)
      for (int tx = tr.tx0; tx <= tr.tx1; ++tx)
        if (tile_hit(rc, tx * kTile, ty * kTile, kappa)) atomicOr(&bm[(ty * nt + tx) * 8 + word], bit);
  __syncthreads();
  if (!have) return;
  const uint32_t *coff = tcnt + ((int64_t)b * nch + c) * T;
  for (int ty = tr.ty0; ty <= tr.ty1; ++ty)
    for (int tx = tr.tx0; tx <= tr.tx1; ++tx) {
      int t = ty * nt + tx;
      const uint32_t *w = bm + t * 8;
      if (!(w[word] & bit)) continue;
      uint32_t rank = __popc(w[word] & (bit - 1u));
      for (int k = 0; k < word; ++k) rank += __popc(w[k]);
      int64_t pos = tile_start[(int64_t)b * T + t] + coff[t] + rank;
      if (pos < cap) list[pos] = j;
    }
}

static int tile_smem_bytes(int d) {
  int nt = d / kTile;
  return nt * nt * 8 * (int)sizeof(uint32_t);
}

cudaError_t bin_configure(int d) {
  int smem = tile_smem_bytes(d);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(tile_scatter_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_bin(const Rec *rec, const float *depth, int64_t M, int B, int d,
                       float l2tau, float zrange, int zsort, BinScratch &s,
                       const uint32_t **perm_out, cudaStream_t st) {
  cudaError_t e;
  const uint32_t *perm = nullptr;
  if (zsort) {
    int64_t n = M * B;
    depth_key_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(depth, n, 1.f / zrange, s.keyA);
    int nch = (int)bin_chunks_depth(M);
    dim3 g(nch, B);
    // low byte, then high byte (LSD); the first pass seeds index order
    digit_count_kernel<<<g, 256, 0, st>>>(s.keyA, M, 0, nch, s.dcnt);
    digit_scan_kernel<<<B, 256, 0, st>>>(s.dcnt, nch);
    digit_scatter_kernel<<<g, 256, 0, st>>>(s.keyA, nullptr, M, 0, nch, s.dcnt, s.keyB, s.valA);
    digit_count_kernel<<<g, 256, 0, st>>>(s.keyB, M, 8, nch, s.dcnt);
    digit_scan_kernel<<<B, 256, 0, st>>>(s.dcnt, nch);
    digit_scatter_kernel<<<g, 256, 0, st>>>(s.keyB, s.valA, M, 8, nch, s.dcnt, s.keyA, s.valB);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    perm = s.valB;
  }
  int nt = d / kTile, T = nt * nt;
  int nch = (int)bin_chunks_tiles(M);
  dim3 g(nch, B);
  int cnt_smem = T * (int)sizeof(uint32_t);
  tile_count_kernel<<<g, 256, cnt_smem, st>>>(rec, perm, M, d, l2tau, nch, s.tcnt);
  dim3 gs((T + 255) / 256, B);
  tile_scan_cols_kernel<<<gs, 256, 0, st>>>(s.tcnt, nch, T, s.tile_start);
  scan_tiles_kernel<<<1, 1024, 0, st>>>(s.tile_start, (int64_t)B * T, s.cap, s.status);
  tile_scatter_kernel<<<g, 256, tile_smem_bytes(d), st>>>(rec, perm, M, d, l2tau, nch, s.tcnt,
                                                         s.tile_start, s.cap, s.list);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  *perm_out = perm;
  return cudaSuccess;
}

}  // namespace gem
