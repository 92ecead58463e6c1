// Radix-4/2/3 Stockham FFT of lines held in shared memory (n = 2^a 3^b),
// shared by the CTF step and the Fourier shell correlation.  The plan
// (FftPlan, from fft_plan) lists the radix of every stage; tw[m] =
// e^{-2 pi i m / n}.
#pragma once

#include "gem_internal.cuh"

namespace gem {

// x / D for 0 <= x <= 16 n and D <= n <= 768, given r = 1/D rounded to
// float: (x + 1/2) r, one fused rounding, is within 1e-4 of (x + 1/2) / D,
// which is at least 1/(2 D) >= 6.5e-4 away from an integer, so truncation
// gives the exact quotient (checked exhaustively for every supported n).
__device__ __forceinline__ int fdiv_small(int x, float r) {
  return (int)fmaf((float)x, r, 0.5f * r);
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// One radix-R Stockham stage on every line (nl lines of length n, line l
// starting at element l * ls).
// Butterfly jj of a line reads elements jj + r n/R, twiddles them by
// W^(r k n/(Ns R)), k = jj mod Ns, and writes (jj / Ns) Ns R + k + r Ns.
template <int R>
__device__ __forceinline__ void fft_stage(const float2 *__restrict__ src, float2 *__restrict__ dst,
                                          int nl, int n, int ls, int Ns,
                                          const float2 *__restrict__ tw) {
  const int nb = n / R;
  const int tws = n / (Ns * R);
  const int total = nl * nb;
  const float rnb = 1.f / (float)nb, rns = 1.f / (float)Ns;
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int line = fdiv_small(idx, rnb);
    const int jj = idx - line * nb;
    const float2 *in = src + line * ls;
    float2 *out = dst + line * ls;
    const int q = fdiv_small(jj, rns);
    const int k = jj - q * Ns;
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = in[jj + r * nb];
#pragma unroll
    for (int r = 1; r < R; ++r) v[r] = cmul(v[r], tw[r * k * tws]);
    if (R == 4) {
      float2 a0 = make_float2(v[0].x + v[2].x, v[0].y + v[2].y);
      float2 a1 = make_float2(v[0].x - v[2].x, v[0].y - v[2].y);
      float2 a2 = make_float2(v[1].x + v[3 % R].x, v[1].y + v[3 % R].y);
      float2 a3 = make_float2(v[1].y - v[3 % R].y, v[3 % R].x - v[1].x);  // (v1 - v3) (-i)
      v[0] = make_float2(a0.x + a2.x, a0.y + a2.y);
      v[2 % R] = make_float2(a0.x - a2.x, a0.y - a2.y);
      v[1] = make_float2(a1.x + a3.x, a1.y + a3.y);
      v[3 % R] = make_float2(a1.x - a3.x, a1.y - a3.y);
    } else if (R == 2) {
      float2 a0 = v[0];
      v[0] = make_float2(a0.x + v[1].x, a0.y + v[1].y);
      v[1] = make_float2(a0.x - v[1].x, a0.y - v[1].y);
    } else {  // R == 3
      const float h = 0.8660254037844386f;  // sqrt(3)/2
      float2 t1 = make_float2(v[1].x + v[2 % R].x, v[1].y + v[2 % R].y);
      float2 t2 = make_float2(v[0].x - 0.5f * t1.x, v[0].y - 0.5f * t1.y);
      float2 t3 = make_float2(h * (v[1].y - v[2 % R].y), -h * (v[1].x - v[2 % R].x));
      v[0] = make_float2(v[0].x + t1.x, v[0].y + t1.y);
      v[1] = make_float2(t2.x + t3.x, t2.y + t3.y);
      v[2 % R] = make_float2(t2.x - t3.x, t2.y - t3.y);
    }
    const int obase = q * Ns * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) out[obase + r * Ns] = v[r];
  }
}

// Forward (e^{-2 pi i}) FFT of nl lines of length n, line l at element
// l * ls of each buffer, src -> dst -> src ...; returns the buffer holding
// the result.  tw[m] = e^{-2 pi i m / n}.  A line stride of n + 1 keeps
// column-wise accesses (element k of 16 lines) free of bank conflicts.
__device__ inline float2 *fft_lines(float2 *src, float2 *dst, int nl, const FftPlan &pl,
                                    const float2 *__restrict__ tw, int ls) {
  const int n = pl.n;
  int Ns = 1;
  for (int s = 0; s < pl.nst; ++s) {
    const unsigned c = (pl.code >> (2 * s)) & 3u;
    const int R = c == 2 ? 4 : (c == 1 ? 3 : 2);
    if (R == 4)
      fft_stage<4>(src, dst, nl, n, ls, Ns, tw);
    else if (R == 2)
      fft_stage<2>(src, dst, nl, n, ls, Ns, tw);
    else
      fft_stage<3>(src, dst, nl, n, ls, Ns, tw);
    __syncthreads();
    float2 *tmp = src;
    src = dst;
    dst = tmp;
    Ns *= R;
  }
  return src;
}

}  // namespace gem
