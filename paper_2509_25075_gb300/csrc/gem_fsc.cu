// Fourier shell correlation of two maps (Eq. fsc; Sec. 4, Gold-Standard
// Fourier Shell Correlation) and its threshold crossing.
//
//   FSC(r_i) = sum_{k in shell i} F1(k) F2(k)^* /
//              sqrt(sum |F1(k)|^2 . sum |F2(k)|^2),
//
// shell i holding the frequencies with round(|k|) = i (k in signed DFT
// indices, shells 0 .. d/2).  Both real maps ride in one complex volume
// z = X1 + i X2; after the 3D DFT, F1(k) = (Z(k) + Z(-k)^*) / 2 and
// F2(k) = (Z(k) - Z(-k)^*) / (2i).  The 3D DFT is three passes of line FFTs
// in shared memory, each along the contiguous axis, each writing its output
// with the axes rotated so the next axis becomes contiguous:
//   [z][y][x] -> [kx][z][y] -> [ky][kx][z] -> [kz][ky][kx].
#include <math.h>

#include "gem_fft.cuh"
#include "gem_internal.cuh"

namespace gem {

constexpr int kFL = 16;  // lines per CTA
constexpr int kFThreads = 256;
constexpr int kShellBlocks = 608;  // 4 per SM on 152 SMs

// shared-memory lines padded by one element (conflict-free column access)
static size_t fsc_smem(int d) { return (size_t)(2 * kFL * (d + 1) + d) * sizeof(float2); }

// x pass: rows y0 .. y0+15 of slab z of z = X1 + i X2, FFT along x, written
// as A[kx][z][y].
__global__ void __launch_bounds__(kFThreads) fsc_pass_real_kernel(
    const float *__restrict__ X1, const float *__restrict__ X2, FftPlan pl,
    const float2 *__restrict__ tw, float2 *__restrict__ A) {
  extern __shared__ float2 sm[];
  const int d = pl.n;
  const int ls = d + 1;
  float2 *a = sm, *bb = sm + kFL * ls, *tws = sm + 2 * kFL * ls;
  const int y0 = blockIdx.x * kFL, z = blockIdx.y;
  for (int i = threadIdx.x; i < d; i += blockDim.x) tws[i] = tw[i];
  const int64_t base = ((int64_t)z * d + y0) * d;
  for (int i = threadIdx.x; i < kFL * d; i += blockDim.x) {
    const int l = fdiv_small(i, 1.f / (float)d), x = i - l * d;
    a[l * ls + x] = make_float2(X1[base + i], X2[base + i]);
  }
  __syncthreads();
  const float2 *res = fft_lines(a, bb, kFL, pl, tws, ls);
  for (int i = threadIdx.x; i < kFL * d; i += blockDim.x) {
    const int l = i % kFL, k = i / kFL;
    A[((int64_t)k * d + z) * d + y0 + l] = res[l * ls + k];
  }
}

// Complex pass: B[k][i0][i1] = FFT along i2 of A[i0][i1][:], lines
// i1 = i1_0 .. i1_0 + 15 of slab i0.
__global__ void __launch_bounds__(kFThreads) fsc_pass_cplx_kernel(const float2 *__restrict__ A,
                                                                  FftPlan pl,
                                                                  const float2 *__restrict__ tw,
                                                                  float2 *__restrict__ Bo) {
  extern __shared__ float2 sm[];
  const int d = pl.n;
  const int ls = d + 1;
  float2 *a = sm, *bb = sm + kFL * ls, *tws = sm + 2 * kFL * ls;
  const int i10 = blockIdx.x * kFL, i0 = blockIdx.y;
  for (int i = threadIdx.x; i < d; i += blockDim.x) tws[i] = tw[i];
  const int64_t base = ((int64_t)i0 * d + i10) * d;
  for (int i = threadIdx.x; i < kFL * d; i += blockDim.x) {
    const int l = fdiv_small(i, 1.f / (float)d), x = i - l * d;
    a[l * ls + x] = A[base + i];
  }
  __syncthreads();
  const float2 *res = fft_lines(a, bb, kFL, pl, tws, ls);
  for (int i = threadIdx.x; i < kFL * d; i += blockDim.x) {
    const int l = i % kFL, k = i / kFL;
    Bo[((int64_t)k * d + i0) * d + i10 + l] = res[l * ls + k];
  }
}

// Shell of a frequency with squared norm k2: the integer s with
// (s - 1/2)^2 <= k2 < (s + 1/2)^2, i.e. 4 s^2 - 4 s + 1 <= 4 k2 < 4 s^2 + 4 s + 1.
__device__ __forceinline__ int shell_of(int k2) {
  int s = (int)floorf(sqrtf((float)k2) + 0.5f);
  while (s > 0 && 4 * k2 < 4 * s * s - 4 * s + 1) --s;
  while (4 * k2 >= 4 * s * s + 4 * s + 1) ++s;
  return s;
}

// Inclusive sum of v over the run of equal keys ending at each lane (runs
// are maximal sequences of consecutive lanes with the same key; bit l of
// run_mask is set when lane l continues the run of lane l - 1).
__device__ __forceinline__ float seg_scan(float v, int lane, unsigned run_mask) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float u = __shfl_up_sync(0xffffffffu, v, o);
    // lane - o lies in the same run iff every lane in (lane - o, lane] does
    const unsigned need = ((1u << o) - 1u) << (lane - o + 1);
    if (lane >= o && (run_mask & need) == need) v += u;
  }
  return v;
}

// Per-block sums over the shells 0 .. nsh-1 of Re(F1 F2^*), |F1|^2, |F2|^2,
// written to part[blk][3][nsh].  A warp takes 32 consecutive frequencies;
// neighbouring frequencies mostly share a shell, so each run of equal shells
// (at most 32 terms) is summed in float32 by a segmented warp scan and added
// to the block's float64 accumulators once.  Voxel indices fit in 32 bits
// (d <= 768).
__global__ void __launch_bounds__(kFThreads) fsc_shell_kernel(const float2 *__restrict__ F,
                                                              int d, int nsh,
                                                              double *__restrict__ part) {
  extern __shared__ double acc[];  // [3][nsh]
  for (int i = threadIdx.x; i < 3 * nsh; i += blockDim.x) acc[i] = 0.0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const unsigned n = (unsigned)d * d * d, ud = (unsigned)d;
  const int h = d / 2;
  const unsigned stride = gridDim.x * blockDim.x;
  for (unsigned base = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < n; base += stride) {
    const unsigned i = base + lane;
    int s = nsh;  // out of range: contributes nothing
    float num = 0.f, p1 = 0.f, p2 = 0.f;
    if (i < n) {
      const unsigned row = i / ud;
      const int kx = (int)(i - row * ud), ky = (int)(row % ud), kz = (int)(row / ud);
      const int sx = kx < h ? kx : kx - d, sy = ky < h ? ky : ky - d, sz = kz < h ? kz : kz - d;
      s = shell_of(sx * sx + sy * sy + sz * sz);
      if (s < nsh) {
        const int mx = kx ? d - kx : 0, my = ky ? d - ky : 0, mz = kz ? d - kz : 0;
        const float2 Z = F[i];
        const float2 Zm = F[((unsigned)mz * ud + (unsigned)my) * ud + (unsigned)mx];
        const float f1r = 0.5f * (Z.x + Zm.x), f1i = 0.5f * (Z.y - Zm.y);
        const float f2r = 0.5f * (Z.y + Zm.y), f2i = -0.5f * (Z.x - Zm.x);
        num = fmaf(f1r, f2r, f1i * f2i);
        p1 = fmaf(f1r, f1r, f1i * f1i);
        p2 = fmaf(f2r, f2r, f2i * f2i);
      } else {
        s = nsh;
      }
    }
    const int prev = __shfl_up_sync(0xffffffffu, s, 1);
    const unsigned run_mask = __ballot_sync(0xffffffffu, lane > 0 && prev == s);
    num = seg_scan(num, lane, run_mask);
    p1 = seg_scan(p1, lane, run_mask);
    p2 = seg_scan(p2, lane, run_mask);
    const int next = __shfl_down_sync(0xffffffffu, s, 1);
    if ((lane == 31 || next != s) && s < nsh) {
      atomicAdd(&acc[s], (double)num);
      atomicAdd(&acc[nsh + s], (double)p1);
      atomicAdd(&acc[2 * nsh + s], (double)p2);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 3 * nsh; i += blockDim.x)
    part[(size_t)blockIdx.x * 3 * nsh + i] = acc[i];
}

// One block per shell: the block sums in a fixed order.
__global__ void __launch_bounds__(256) fsc_fold_kernel(const double *__restrict__ part, int nblk,
                                                       int nsh, double *__restrict__ tot) {
  const int s = blockIdx.x;
  double a = 0, b = 0, c = 0;
  for (int k = threadIdx.x; k < nblk; k += blockDim.x) {
    const double *p = part + (int64_t)k * 3 * nsh;
    a += p[s];
    b += p[nsh + s];
    c += p[2 * nsh + s];
  }
  __shared__ double red[3][256];
  red[0][threadIdx.x] = a;
  red[1][threadIdx.x] = b;
  red[2][threadIdx.x] = c;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int q = 0; q < 3; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 3) tot[threadIdx.x * nsh + s] = red[threadIdx.x][0];
}

// FSC per shell from the folded sums, and the threshold crossing: the first
// shell i >= 1 with FSC < thr, interpolated linearly between shells i-1 and
// i; resolution = d apix / k* (Angstrom).  No crossing: the Nyquist shell
// d/2 (resolution 2 apix).
__global__ void __launch_bounds__(512) fsc_final_kernel(const double *__restrict__ tot, int nsh,
                                                        int d, float apix, float thr,
                                                        double *__restrict__ fsc,
                                                        double *__restrict__ sums,
                                                        double *__restrict__ resolution) {
  extern __shared__ double f[];  // [nsh]
  for (int s = threadIdx.x; s < nsh; s += blockDim.x) {
    const double a = tot[s], b = tot[nsh + s], c = tot[2 * nsh + s];
    const double den = sqrt(b * c);
    f[s] = den > 0.0 ? a / den : 0.0;
    fsc[s] = f[s];
    if (sums) {
      sums[s] = a;
      sums[nsh + s] = b;
      sums[2 * nsh + s] = c;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && resolution) {
    double kstar = (double)(nsh - 1);
    for (int s = 1; s < nsh; ++s) {
      if (f[s] < thr) {
        const double a = f[s - 1], b = f[s];
        const double frac = a > b ? (a - thr) / (a - b) : 0.0;
        kstar = (s - 1) + fmin(fmax(frac, 0.0), 1.0);
        break;
      }
    }
    resolution[0] = kstar > 0.0 ? (double)d * apix / kstar : INFINITY;
  }
}

cudaError_t fsc_configure(int d) {
  const size_t smem = fsc_smem(d);
  cudaError_t e = cudaFuncSetAttribute(fsc_pass_real_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(fsc_pass_cplx_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem);
}

// block partials, then the folded sums
int fsc_partial_count(int d) { return (kShellBlocks + 1) * 3 * (d / 2 + 1); }

cudaError_t launch_fsc(int d, float apix, float thr, const FftPlan &plan, const float2 *tw,
                       const float *X1, const float *X2, float2 *P, float2 *Q, double *part,
                       double *fsc, double *sums, double *resolution, cudaStream_t st) {
  const size_t smem = fsc_smem(d);
  const dim3 g(d / kFL, d);
  fsc_pass_real_kernel<<<g, kFThreads, smem, st>>>(X1, X2, plan, tw, P);
  fsc_pass_cplx_kernel<<<g, kFThreads, smem, st>>>(P, plan, tw, Q);
  fsc_pass_cplx_kernel<<<g, kFThreads, smem, st>>>(Q, plan, tw, P);
  const int nsh = d / 2 + 1;
  fsc_shell_kernel<<<kShellBlocks, kFThreads, 3 * nsh * sizeof(double), st>>>(P, d, nsh, part);
  double *tot = part + (size_t)kShellBlocks * 3 * nsh;
  fsc_fold_kernel<<<nsh, 256, 0, st>>>(part, kShellBlocks, nsh, tot);
  fsc_final_kernel<<<1, 512, nsh * sizeof(double), st>>>(tot, nsh, d, apix, thr, fsc, sums,
                                                         resolution);
  return cudaGetLastError();
}

}  // namespace gem
