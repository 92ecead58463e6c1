// k nearest neighbours of the Gaussian centres.
//
// The isotropic-scaling ablation (Sec. 4, Design Choices of 3DGS for cryo-EM)
// sets S_j = s_j I with s_j the distance of Gaussian j to its nearest
// neighbour; the same distances serve as a scale initialisation.
//
// Uniform grid: the centres' bounding box is cut into about M/2 cubic cells;
// a counting sort by cell lists each cell's members; each query walks
// Chebyshev rings of cells around its own until the k-th best distance is
// shorter than anything an unvisited ring can hold.  The result is exact:
// the k smallest (distance^2, index) pairs in lexicographic order, which
// does not depend on the order the candidates were met.
#include "gem_internal.cuh"

namespace gem {

constexpr int kKnnBlk = 256;
constexpr int kScanPer = 4096;  // elements per block of the cell-count scan

// Per-block min / max of the centres: part[blk][6] = (min x, y, z, max x, y, z).
__global__ void __launch_bounds__(kKnnBlk) knn_bbox_kernel(const float *__restrict__ params,
                                                           int64_t M, float *__restrict__ part) {
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < M;
       j += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      float v = params[j * kNpar + a];
      if (isfinite(v)) {
        lo[a] = fminf(lo[a], v);
        hi[a] = fmaxf(hi[a], v);
      }
    }
  }
  __shared__ float red[kKnnBlk / 32][6];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
      hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
    }
  if (lane == 0)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      red[warp][a] = lo[a];
      red[warp][3 + a] = hi[a];
    }
  __syncthreads();
  if (threadIdx.x < 6) {
    float v = red[0][threadIdx.x];
    for (int w = 1; w < kKnnBlk / 32; ++w)
      v = threadIdx.x < 3 ? fminf(v, red[w][threadIdx.x]) : fmaxf(v, red[w][threadIdx.x]);
    part[blockIdx.x * 6 + threadIdx.x] = v;
  }
}

// One thread: fold the partial boxes and pick the cell size.  Cells are
// cubes of side h with about M / 2 of them over the box; at most cap cells.
__global__ void knn_grid_kernel(const float *__restrict__ part, int nblk, int64_t M, int64_t cap,
                                KnnGrid *__restrict__ g) {
  if (threadIdx.x != 0) return;
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int b = 0; b < nblk; ++b)
    for (int a = 0; a < 3; ++a) {
      lo[a] = fminf(lo[a], part[b * 6 + a]);
      hi[a] = fmaxf(hi[a], part[b * 6 + 3 + a]);
    }
  float ext[3];
  for (int a = 0; a < 3; ++a) {
    if (!(lo[a] <= hi[a])) lo[a] = hi[a] = 0.f;  // no finite centre
    ext[a] = hi[a] - lo[a];
  }
  const float emax = fmaxf(ext[0], fmaxf(ext[1], ext[2]));
  const double target = fmax(1.0, 0.5 * (double)M);
  // side from the volume, kept above emax / 1024 so flat or linear sets of
  // centres do not make the grid explode
  double h = cbrt(fmax((double)ext[0] * ext[1] * ext[2], 0.0) / target);
  h = fmax(h, (double)emax / 1024.0);
  if (!(h > 0.0)) h = 1.0;
  int n[3] = {1, 1, 1};
  bool fits = false;
  for (int it = 0; it < 512 && !fits; ++it, h *= 1.25) {
    double cells = 1.0;
    for (int a = 0; a < 3; ++a) {
      double na = floor(ext[a] / h) + 1.0;
      n[a] = na < 1.0e6 ? (int)na : 1000000;
      cells *= n[a];
    }
    fits = cells <= (double)cap;
    if (fits) break;
  }
  if (!fits || !(h > 0.0) || !isfinite(h)) {  // absurd coordinates: one cell holds all
    n[0] = n[1] = n[2] = 1;
    h = 1.0e30;
  }
  for (int a = 0; a < 3; ++a) g->lo[a] = lo[a];
  g->h = (float)h;
  g->ih = (float)(1.0 / h);
  for (int a = 0; a < 3; ++a) g->n[a] = n[a];
  g->ncell = n[0] * n[1] * n[2];
}

__device__ __forceinline__ int knn_axis_cell(float v, float lo, float ih, int n) {
  int c = (int)floorf((v - lo) * ih);
  return min(max(c, 0), n - 1);
}

// Cell of every centre (non-finite centres go to cell 0 and are never
// reported as neighbours) and per-cell counts.
__global__ void __launch_bounds__(kKnnBlk) knn_cell_kernel(const float *__restrict__ params,
                                                           int64_t M,
                                                           const KnnGrid *__restrict__ g,
                                                           int *__restrict__ cell,
                                                           int *__restrict__ cnt) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= M) return;
  const KnnGrid G = *g;
  const float *p = params + j * kNpar;
  int c = 0;
  if (isfinite(p[0]) && isfinite(p[1]) && isfinite(p[2])) {
    int cx = knn_axis_cell(p[0], G.lo[0], G.ih, G.n[0]);
    int cy = knn_axis_cell(p[1], G.lo[1], G.ih, G.n[1]);
    int cz = knn_axis_cell(p[2], G.lo[2], G.ih, G.n[2]);
    c = (cz * G.n[1] + cy) * G.n[0] + cx;
  }
  cell[j] = c;
  atomicAdd(cnt + c, 1);
}

// Exclusive scan of cnt[0 .. ncell) into start (start[ncell] = total), in
// three steps: block sums, scan of the block sums, block scans.
__global__ void __launch_bounds__(1024) knn_scan_sums_kernel(const int *__restrict__ cnt,
                                                             const KnnGrid *__restrict__ g,
                                                             int *__restrict__ bsum) {
  const int n = g->ncell;
  const int64_t base = (int64_t)blockIdx.x * kScanPer;
  int s = 0;
  for (int i = threadIdx.x; i < kScanPer; i += 1024)
    if (base + i < n) s += cnt[base + i];
  s = __reduce_add_sync(0xffffffffu, s);
  __shared__ int ws[32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    int v = __reduce_add_sync(0xffffffffu, ws[threadIdx.x]);
    if (threadIdx.x == 0) bsum[blockIdx.x] = v;
  }
}

__device__ __forceinline__ int block_exclusive_scan(int v, int *ws, int &total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int u = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += u;
  }
  if (lane == 31) ws[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    int w = ws[lane], wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int u = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += u;
    }
    ws[lane] = wi - w;
    if (lane == 31) ws[32] = wi;
  }
  __syncthreads();
  int r = ws[warp] + inc - v;
  total = ws[32];
  __syncthreads();
  return r;
}

// bsum[0 .. nb) becomes its exclusive scan; bsum[nb] = the total.
__global__ void __launch_bounds__(1024) knn_scan_top_kernel(int *__restrict__ bsum, int nb) {
  __shared__ int ws[33];
  int carry = 0;
  for (int base = 0; base < nb; base += 1024) {
    int i = base + threadIdx.x;
    int v = i < nb ? bsum[i] : 0;
    int tot;
    int ex = block_exclusive_scan(v, ws, tot);
    if (i < nb) bsum[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) bsum[nb] = carry;
}

__global__ void __launch_bounds__(1024) knn_scan_blocks_kernel(const int *__restrict__ cnt,
                                                               const KnnGrid *__restrict__ g,
                                                               const int *__restrict__ bsum,
                                                               int *__restrict__ start,
                                                               int *__restrict__ fill) {
  __shared__ int ws[33];
  const int n = g->ncell;
  const int64_t base = (int64_t)blockIdx.x * kScanPer;
  int carry = bsum[blockIdx.x];
  // 4 elements per thread, in order
  const int64_t i0 = base + 4 * threadIdx.x;
  int v[4], s = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    v[k] = (i0 + k < n) ? cnt[i0 + k] : 0;
    s += v[k];
  }
  int tot;
  int ex = block_exclusive_scan(s, ws, tot) + carry;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (i0 + k < n) {
      start[i0 + k] = ex;
      fill[i0 + k] = ex;
    }
    ex += v[k];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) start[n] = bsum[gridDim.x];
}

__global__ void __launch_bounds__(kKnnBlk) knn_scatter_kernel(const int *__restrict__ cell,
                                                              int64_t M, int *__restrict__ fill,
                                                              int *__restrict__ order) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= M) return;
  int pos = atomicAdd(fill + cell[j], 1);
  order[pos] = (int)j;
}

// Squared distance without contraction into FMA, so that it is the same
// number whatever the compiler does.
__device__ __forceinline__ float dist2_rn(float ax, float ay, float az, float bx, float by,
                                          float bz) {
  float dx = __fsub_rn(ax, bx), dy = __fsub_rn(ay, by), dz = __fsub_rn(az, bz);
  return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

template <int K>
__global__ void __launch_bounds__(kKnnBlk) knn_query_kernel(
    const float *__restrict__ params, int64_t M, const KnnGrid *__restrict__ g,
    const int *__restrict__ start, const int *__restrict__ order, float *__restrict__ dist,
    int32_t *__restrict__ idx) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= M) return;
  const int i = order[t];  // neighbouring threads query neighbouring centres
  const KnnGrid G = *g;
  const float px = params[(int64_t)i * kNpar], py = params[(int64_t)i * kNpar + 1],
              pz = params[(int64_t)i * kNpar + 2];
  float bd[K];
  int bi[K];
#pragma unroll
  for (int m = 0; m < K; ++m) {
    bd[m] = INFINITY;
    bi[m] = -1;
  }
  const bool fin = isfinite(px) && isfinite(py) && isfinite(pz);
  if (fin) {
    const int cx = knn_axis_cell(px, G.lo[0], G.ih, G.n[0]);
    const int cy = knn_axis_cell(py, G.lo[1], G.ih, G.n[1]);
    const int cz = knn_axis_cell(pz, G.lo[2], G.ih, G.n[2]);
    const int rmax = max(G.n[0], max(G.n[1], G.n[2]));
    for (int r = 0; r <= rmax; ++r) {
      for (int dz = -r; dz <= r; ++dz) {
        const int z = cz + dz;
        if (z < 0 || z >= G.n[2]) continue;
        for (int dy = -r; dy <= r; ++dy) {
          const int y = cy + dy;
          if (y < 0 || y >= G.n[1]) continue;
          // inner rows of the ring hold only its two end cells (r > 0 there)
          const bool face = (dz == -r || dz == r || dy == -r || dy == r);
          const int step = face ? 1 : 2 * r;
          for (int dx = -r; dx <= r; dx += step) {
            const int x = cx + dx;
            if (x < 0 || x >= G.n[0]) continue;
            const int c = (z * G.n[1] + y) * G.n[0] + x;
            for (int q = start[c], qe = start[c + 1]; q < qe; ++q) {
              const int j = order[q];
              if (j == i) continue;
              const float *pj = params + (int64_t)j * kNpar;
              const float qx = pj[0], qy = pj[1], qz = pj[2];
              if (!(isfinite(qx) && isfinite(qy) && isfinite(qz))) continue;
              const float d2 = dist2_rn(px, py, pz, qx, qy, qz);
              if (d2 < bd[K - 1] || (d2 == bd[K - 1] && j < bi[K - 1])) {
                // insert, keeping (d2, j) ascending: from the end, each slot
                // takes its left neighbour while the newcomer sorts before
                // it, else the newcomer if it sorts before the slot
#pragma unroll
                for (int m = K - 1; m > 0; --m) {
                  const bool before_left = d2 < bd[m - 1] || (d2 == bd[m - 1] && j < bi[m - 1]);
                  const bool before_here = d2 < bd[m] || (d2 == bd[m] && j < bi[m]);
                  if (before_left) {
                    bd[m] = bd[m - 1];
                    bi[m] = bi[m - 1];
                  } else if (before_here) {
                    bd[m] = d2;
                    bi[m] = j;
                  }
                }
                if (d2 < bd[0] || (d2 == bd[0] && j < bi[0])) {
                  bd[0] = d2;
                  bi[0] = j;
                }
              }
            }
          }
        }
      }
      // everything in rings beyond r lies farther than r * h from the point
      const float reach = (float)r * G.h * (1.f - 1e-4f);
      if (bi[K - 1] >= 0 && bd[K - 1] <= reach * reach) break;
    }
  }
#pragma unroll
  for (int m = 0; m < K; ++m) {
    dist[(int64_t)i * K + m] = bi[m] >= 0 ? sqrtf(bd[m]) : INFINITY;
    if (idx) idx[(int64_t)i * K + m] = bi[m];
  }
}

// One instance per k, so that the k best live in registers.
template <int K>
void launch_query(int k, unsigned gm, cudaStream_t st, const float *params, int64_t M,
                  const KnnGrid *g, const int *start, const int *order, float *dist,
                  int32_t *idx) {
  if (k == K)
    knn_query_kernel<K><<<gm, kKnnBlk, 0, st>>>(params, M, g, start, order, dist, idx);
  else if constexpr (K < 16)
    launch_query<K + 1>(k, gm, st, params, M, g, start, order, dist, idx);
}

int knn_scan_blocks(int64_t cap) { return (int)((cap + kScanPer - 1) / kScanPer); }

cudaError_t launch_knn(const float *params, int64_t M, int k, const KnnScratch &s, float *dist,
                       int32_t *idx, cudaStream_t st) {
  cudaError_t e;
  const int64_t nbl = (M + kKnnBlk - 1) / kKnnBlk;
  const int nbb = (int)(nbl < 608 ? nbl : 608);  // KnnScratch::part holds 608 boxes
  knn_bbox_kernel<<<nbb, kKnnBlk, 0, st>>>(params, M, s.part);
  knn_grid_kernel<<<1, 32, 0, st>>>(s.part, nbb, M, s.cap, s.grid);
  if ((e = cudaMemsetAsync(s.cnt, 0, (size_t)s.cap * sizeof(int), st)) != cudaSuccess) return e;
  const unsigned gm = (unsigned)((M + kKnnBlk - 1) / kKnnBlk);
  knn_cell_kernel<<<gm, kKnnBlk, 0, st>>>(params, M, s.grid, s.cell, s.cnt);
  const int nb = knn_scan_blocks(s.cap);
  knn_scan_sums_kernel<<<nb, 1024, 0, st>>>(s.cnt, s.grid, s.bsum);
  knn_scan_top_kernel<<<1, 1024, 0, st>>>(s.bsum, nb);
  knn_scan_blocks_kernel<<<nb, 1024, 0, st>>>(s.cnt, s.grid, s.bsum, s.start, s.fill);
  knn_scatter_kernel<<<gm, kKnnBlk, 0, st>>>(s.cell, M, s.fill, s.order);
  launch_query<1>(k, gm, st, params, M, s.grid, s.start, s.order, dist, idx);
  return cudaGetLastError();
}

}  // namespace gem
