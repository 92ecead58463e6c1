// Step a4 of the GEM hot path: Eq. loss and its adjoint.
//
//   I_pred = F^-1(H . F(I^)),  r = I_pred - I,  L = (1/B) sum_b mean(r^2),
//   dL/dI^ = F^-1(H . F(2 r / (B d^2)))   (H real and even: self-adjoint).
//
// Both real images of a view are packed into one complex image
// z = I^ + i I, so F(z) = X + i Y with X = F(I^), Y = F(I) recovered from the
// Hermitian symmetry of real spectra.  In Fourier space
//   P = H X,  R = H X - Y  (= F(r)),  G = H R,
// the loss is (by Parseval) sum |R|^2 / d^4 per image, and one inverse
// transform of W = P + i G returns I_pred (real part) and, times
// 2 / (B d^2), dL/dI^ (imaginary part).  G is transformed unscaled so that
// both halves of W have comparable magnitude and share the FFT's rounding
// fairly.  So each image costs one forward and one inverse complex 2D FFT.
//
// Three passes through a [B][d][d] complex buffer, stored transposed
// (Z[b][kx][y]) so that every FFT runs on contiguous lines:
//   pass 1: FFT along x of kLines rows of z, written transposed;
//   pass 2: FFT along y of the lines kx and d - kx (kLines / 2 pairs per CTA; the
//           first CTA holds the self-paired lines 0 and d/2 in the slots
//           of line 0's pair), CTF, loss, W, inverse FFT along y, written
//           back in place;
//   pass 3: inverse FFT along x of kLines rows, split into I_pred and dL/dI^.
// FFTs are radix-4/2/3 Stockham transforms in shared memory (d = 2^a 3^b).
#include <math.h>

#include "gem_fft.cuh"
#include "gem_internal.cuh"

namespace gem {

bool fft_plan(int n, FftPlan &p) {
  p.n = n;
  p.nst = 0;
  p.code = 0;
  int m = n;
  auto push = [&](unsigned c) {
    p.code |= c << (2 * p.nst);
    ++p.nst;
  };
  while (m % 3 == 0 && p.nst < 16) {
    push(1);
    m /= 3;
  }
  while (m % 4 == 0 && p.nst < 16) {
    push(2);
    m /= 4;
  }
  if (m % 2 == 0 && p.nst < 16) {
    push(0);
    m /= 2;
  }
  return m == 1;
}

// Lines per CTA in every pass (kLines, a template parameter): 16 where two
// line buffers of 16 lines leave room for four CTAs per SM, else 8 (large
// images: more, smaller CTAs, so the last wave is short).
constexpr int kCtfThreads = 256;

// line stride in shared memory: one element of padding per line
__host__ __device__ constexpr int ctf_ls(int d) { return d + 1; }
static size_t ctf_smem(int lines, int d) {
  return (size_t)(2 * lines * ctf_ls(d) + d) * sizeof(float2);
}
static int ctf_lines(int d) { return ctf_smem(16, d) <= 56 * 1024 ? 16 : 8; }

__device__ __forceinline__ void load_twiddles(float2 *tw_s, const float2 *__restrict__ tw,
                                              int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) tw_s[i] = tw[i];
}

// pass 1: rows y0 .. y0 + kLines - 1 of z = proj + i images -> FFT along x -> Z[b][kx][y]
template <int kLines>
__global__ void __launch_bounds__(kCtfThreads) ctf_pass1_kernel(
    const float *__restrict__ proj, const float *__restrict__ images, FftPlan pl,
    const float2 *__restrict__ tw, float2 *__restrict__ Z) {
  extern __shared__ float2 sm[];
  const int d = pl.n;
  const int ls = ctf_ls(d);
  float2 *a = sm, *bb = sm + kLines * ls, *tws = sm + 2 * kLines * ls;
  const int y0 = blockIdx.x * kLines, b = blockIdx.y;
  load_twiddles(tws, tw, d);
  const float *pr = proj + ((int64_t)b * d + y0) * d;
  const float *im = images + ((int64_t)b * d + y0) * d;
  const float rd = 1.f / (float)d;
  for (int i = threadIdx.x; i < kLines * d; i += blockDim.x) {
    const int l = fdiv_small(i, rd), x = i - l * d;
    a[l * ls + x] = make_float2(pr[i], im[i]);
  }
  __syncthreads();
  float2 *res = fft_lines(a, bb, kLines, pl, tws, ls);
  float2 *zb = Z + (int64_t)b * d * d;
  for (int i = threadIdx.x; i < kLines * d; i += blockDim.x) {
    int l = i % kLines, kx = i / kLines;
    zb[(int64_t)kx * d + y0 + l] = res[l * ls + kx];
  }
}

// A float-float number hi + lo (|lo| <= ulp(hi) / 2).
struct FF {
  float hi, lo;
};

__device__ __forceinline__ FF ff_split(double x) {
  FF r;
  r.hi = (float)x;
  r.lo = (float)(x - (double)r.hi);
  return r;
}

// c * N for an integer-valued float N (|N| < 2^24), reduced modulo 1: the
// product of the high parts is error-free (fmaf), its integer part dropped.
__device__ __forceinline__ FF ff_mul_mod1(FF c, float N) {
  float p = c.hi * N;
  float e = fmaf(c.hi, N, -p);
  FF r;
  r.hi = p - rintf(p);
  r.lo = fmaf(c.lo, N, e);
  return r;
}

__device__ __forceinline__ FF ff_add(FF a, FF b) {
  float s = a.hi + b.hi;
  float bb = s - a.hi;
  float err = (a.hi - (s - bb)) + (b.hi - bb);
  FF r;
  r.hi = s;
  r.lo = err + a.lo + b.lo;
  return r;
}

// Per-image CTF constants for the parameter form, in turns (chi / 2 pi):
//   chi / (2 pi) = lambda/2 dF(angle) k^2 - Cs lambda^3 k^4 / 4 + phase / (2 pi),
// with k = n / (d apix) for the signed bin indices n = (kx, ky).
// dF(angle) k^2 expands into integer multiples (kx^2 + ky^2, kx^2 - ky^2,
// 2 kx ky) of per-image constants, so no angle is formed, and every term is
// a constant times an integer, evaluated in float-float and reduced modulo
// one turn (tens of turns at Nyquist would otherwise cost float32 its
// accuracy).
struct CtfConst {
  FF c1;   // turns per (kx^2 + ky^2), mean defocus
  FF c2;   // turns per (kx^2 - ky^2), astigmatism
  FF c3;   // turns per 2 kx ky, astigmatism
  FF c4;   // turns per (kx^2 + ky^2)^2, spherical aberration
  FF ph;   // phase shift, turns
  float sw, w;  // sqrt(1 - w^2), w
  float bq;     // B-factor damping per (kx^2 + ky^2)
};

__device__ CtfConst ctf_const(const float *__restrict__ prm, int d, float apix) {
  double dU = prm[0], dV = prm[1], volt = (double)prm[3] * 1e3;
  double cs = (double)prm[4] * 1e7, w = prm[5], phase = prm[6], bf = prm[7];
  double lam = 12.2643247 / sqrt(volt * (1.0 + 0.978466e-6 * volt));
  double cf = 1.0 / ((double)d * apix * (double)d * apix);
  double mean = 0.5 * (dU + dV), half = 0.5 * (dU - dV);
  // the astigmatism terms reach a fraction of a turn at Nyquist, so the
  // angle's cosine and sine need float accuracy only (kept off the slow
  // double-precision path, which this single thread runs while its CTA waits)
  float s2a, c2a;
  sincosf(2.f * prm[2], &s2a, &c2a);
  CtfConst c;
  c.c1 = ff_split(0.5 * lam * mean * cf);
  c.c2 = ff_split(0.5 * lam * half * (double)c2a * cf);
  c.c3 = ff_split(0.5 * lam * half * (double)s2a * cf);
  c.c4 = ff_split(-0.25 * cs * lam * lam * lam * cf * cf);
  c.ph = ff_split(phase / (2.0 * 3.14159265358979323846));
  c.sw = (float)sqrt(1.0 - w * w);
  c.w = (float)w;
  c.bq = (float)(bf * cf / 4.0);
  return c;
}

// CTF at signed bin indices (sx, sy).
__device__ __forceinline__ float ctf_at(const CtfConst &c, int sx, int sy) {
  float x2 = (float)(sx * sx), y2 = (float)(sy * sy);
  float n2 = x2 + y2;  // exact (< 2^24)
  FF t = ff_mul_mod1(c.c1, n2);
  t = ff_add(t, ff_mul_mod1(c.c2, x2 - y2));
  t = ff_add(t, ff_mul_mod1(c.c3, (float)(2 * sx * sy)));
  // (n2)^2 as an exact float-float q + qe, then c4 q mod 1 + c4 qe
  float q = n2 * n2;
  float qe = fmaf(n2, n2, -q);
  FF t4 = ff_mul_mod1(c.c4, q);
  t4.lo = fmaf(c.c4.hi, qe, t4.lo);
  t = ff_add(t, t4);
  t = ff_add(t, c.ph);
  float turns = (t.hi - rintf(t.hi)) + t.lo;
  float s, co;
  sincospif(2.f * turns, &s, &co);
  return -(c.sw * s + c.w * co) * __expf(-c.bq * n2);
}

__device__ __forceinline__ int signed_bin(int k, int d) { return k < d / 2 ? k : k - d; }

// Line kx held in slot i of pass-2 CTA blk (see ctf_pass2_kernel).
template <int kHalf>
__device__ __forceinline__ int pass2_line(int blk, int i, int d) {
  const int kx1 = kHalf * blk + (i & (kHalf - 1));
  return i < kHalf ? kx1 : (kx1 == 0 ? d / 2 : d - kx1);
}

// pass 2: slots i < kHalf hold the lines kx1 = kHalf c + i (kx1 < d/2),
// slots kHalf + i their partners d - kx1; line 0 is its own partner, so its
// slot kHalf holds the other self-paired line, d/2.  d is a multiple of
// kLines, so the d / kLines CTAs of an image hold every line once.
template <int kLines>
__global__ void __launch_bounds__(kCtfThreads) ctf_pass2_kernel(
    FftPlan pl, const float2 *__restrict__ tw, const float *__restrict__ ctf,
    const float *__restrict__ ctf_params, float apix, float2 *__restrict__ Z,
    double *__restrict__ lossp, int nblk) {
  constexpr int kHalf = kLines / 2;  // line pairs per CTA
  extern __shared__ float2 sm[];
  __shared__ CtfConst cc;
  __shared__ double red[kCtfThreads / 32];
  const int d = pl.n, hd = d / 2;
  const int ls = ctf_ls(d);
  float2 *a = sm, *bb = sm + kLines * ls, *tws = sm + 2 * kLines * ls;
  const int blk = blockIdx.x, b = blockIdx.y;
  load_twiddles(tws, tw, d);
  if (ctf_params && threadIdx.x == 0) cc = ctf_const(ctf_params + 8 * b, d, apix);
  float2 *zb = Z + (int64_t)b * d * d;
  const float rd = 1.f / (float)d;
  // load the kLines lines
  for (int idx = threadIdx.x; idx < kLines * d; idx += blockDim.x) {
    const int i = fdiv_small(idx, rd), y = idx - i * d;
    a[i * ls + y] = zb[(int64_t)pass2_line<kHalf>(blk, i, d) * d + y];
  }
  __syncthreads();
  float2 *L = fft_lines(a, bb, kLines, pl, tws, ls);
  // combine: thread per (pair i, ky); the first CTA has one more "pair",
  // the self-paired line d/2 in slot kHalf
  float lsum = 0.f;
  const int npair = blk == 0 ? kHalf + 1 : kHalf;
  for (int idx = threadIdx.x; idx < npair * d; idx += blockDim.x) {
    int i = fdiv_small(idx, rd), ky = idx - i * d;
    int kx = i < kHalf ? kHalf * blk + i : hd;
    bool self = (kx == 0 || kx == hd);
    if (self && ky > hd) continue;
    int mky = ky == 0 ? 0 : d - ky;
    float2 *l1 = L + i * ls;
    float2 *l2 = self ? l1 : L + (kHalf + i) * ls;
    float2 z1 = l1[ky], z2 = l2[mky];
    // X = (z1 + conj z2) / 2,  Y = (z1 - conj z2) / (2 i)
    float2 X = make_float2(0.5f * (z1.x + z2.x), 0.5f * (z1.y - z2.y));
    float2 Yv = make_float2(0.5f * (z1.y + z2.y), -0.5f * (z1.x - z2.x));
    float h;
    if (ctf_params) {
      int sx = signed_bin(kx, d), sy = signed_bin(ky, d);
      h = ctf_at(cc, sx, sy);
      if (kx == hd || ky == hd) {
        int px = signed_bin(kx == 0 ? 0 : d - kx, d), py = signed_bin(mky, d);
        h = 0.5f * (h + ctf_at(cc, px, py));
      }
    } else {
      const float *hb = ctf + (int64_t)b * d * (hd + 1);
      h = hb[(int64_t)ky * (hd + 1) + kx];
      if (self) h = 0.5f * (h + hb[(int64_t)mky * (hd + 1) + kx]);
    }
    float2 P = make_float2(h * X.x, h * X.y);
    float2 Rr = make_float2(P.x - Yv.x, P.y - Yv.y);
    float2 G = make_float2(h * Rr.x, h * Rr.y);
    float r2 = Rr.x * Rr.x + Rr.y * Rr.y;
    bool lone = self && (ky == 0 || ky == hd);
    lsum += lone ? r2 : 2.f * r2;
    // W(k) = P + i G;  W(-k) = conj P + i conj G.  Stored conjugated: the
    // inverse transform runs as conj(FFT(conj .)).
    float2 W = make_float2(P.x - G.y, P.y + G.x);
    float2 Wm = make_float2(P.x + G.y, -P.y + G.x);
    l1[ky] = make_float2(W.x, -W.y);
    l2[mky] = make_float2(Wm.x, -Wm.y);
  }
  // block reduction of the loss partial in float64
  double lw = (double)lsum;
  for (int o = 16; o > 0; o >>= 1) lw += __shfl_xor_sync(0xffffffffu, lw, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = lw;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kCtfThreads / 32; ++w) s += red[w];
    lossp[(int64_t)b * nblk + blk] = s;
  }
  // inverse along y (conjugated forward transform)
  float2 *other = (L == a) ? bb : a;
  float2 *R2 = fft_lines(L, other, kLines, pl, tws, ls);
  for (int idx = threadIdx.x; idx < kLines * d; idx += blockDim.x) {
    const int i = fdiv_small(idx, rd), y = idx - i * d;
    const float2 v = R2[i * ls + y];
    zb[(int64_t)pass2_line<kHalf>(blk, i, d) * d + y] = make_float2(v.x, -v.y);
  }
}

// pass 3: rows y0 .. y0 + kLines - 1 of W (read transposed) -> inverse FFT along x ->
// I_pred = Re / d^2, dL/dI^ = Im (2 / (B d^2)) / d^2.
template <int kLines>
__global__ void __launch_bounds__(kCtfThreads) ctf_pass3_kernel(
    FftPlan pl, const float2 *__restrict__ tw, const float2 *__restrict__ Z, float inv_n2,
    float gscale, float *__restrict__ pred, float *__restrict__ dproj) {
  extern __shared__ float2 sm[];
  const int d = pl.n;
  const int ls = ctf_ls(d);
  float2 *a = sm, *bb = sm + kLines * ls, *tws = sm + 2 * kLines * ls;
  const int y0 = blockIdx.x * kLines, b = blockIdx.y;
  load_twiddles(tws, tw, d);
  const float2 *zb = Z + (int64_t)b * d * d;
  for (int i = threadIdx.x; i < kLines * d; i += blockDim.x) {
    int l = i % kLines, kx = i / kLines;
    float2 v = zb[(int64_t)kx * d + y0 + l];
    a[l * ls + kx] = make_float2(v.x, -v.y);
  }
  __syncthreads();
  float2 *res = fft_lines(a, bb, kLines, pl, tws, ls);
  int64_t off = ((int64_t)b * d + y0) * d;
  const float rd = 1.f / (float)d;
  for (int i = threadIdx.x; i < kLines * d; i += blockDim.x) {
    const int l = fdiv_small(i, rd), x = i - l * d;
    float2 v = res[l * ls + x];
    if (pred) pred[off + i] = v.x * inv_n2;
    if (dproj) dproj[off + i] = -v.y * gscale;
  }
}

// loss_img[b] = sum of image b's partials / d^4 (one warp per image, fixed
// order: deterministic); loss = mean over images (one block, fixed order).
__global__ void __launch_bounds__(256) loss_img_kernel(const double *__restrict__ lossp, int B,
                                                       int nblk, double inv_d4,
                                                       double *__restrict__ loss_img) {
  int b = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (b >= B) return;
  double s = 0.0;
  for (int c = lane; c < nblk; c += 32) s += lossp[(int64_t)b * nblk + c];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) loss_img[b] = s * inv_d4;
}

__global__ void __launch_bounds__(256) loss_mean_kernel(const double *__restrict__ loss_img,
                                                        int B, double *__restrict__ loss) {
  __shared__ double red[8];
  double s = 0.0;
  for (int b = threadIdx.x; b < B; b += blockDim.x) s += loss_img[b];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    *loss = t / B;
  }
}

size_t ctf_partials(int d) { return (size_t)(d / ctf_lines(d)); }

template <int kLines>
static cudaError_t ctf_configure_lines(int d) {
  int smem = (int)ctf_smem(kLines, d);
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(ctf_pass1_kernel<kLines>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(ctf_pass2_kernel<kLines>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess)
    return e;
  return cudaFuncSetAttribute(ctf_pass3_kernel<kLines>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

cudaError_t ctf_configure(int d) {
  return ctf_lines(d) == 16 ? ctf_configure_lines<16>(d) : ctf_configure_lines<8>(d);
}

template <int kLines>
static void launch_ctf_passes(int d, int B, float apix, const FftPlan &plan, const float2 *tw,
                              const float *proj, const float *ctf, const float *ctf_params,
                              const float *images, float2 *Z, double *lossp, float *pred,
                              float *dproj, cudaStream_t st) {
  const size_t smem = ctf_smem(kLines, d);
  const int nblk = d / kLines;
  const float cscale = (float)(2.0 / ((double)B * d * d));
  ctf_pass1_kernel<kLines><<<dim3(d / kLines, B), kCtfThreads, smem, st>>>(proj, images, plan, tw,
                                                                           Z);
  ctf_pass2_kernel<kLines><<<dim3(nblk, B), kCtfThreads, smem, st>>>(plan, tw, ctf, ctf_params,
                                                                     apix, Z, lossp, nblk);
  ctf_pass3_kernel<kLines><<<dim3(d / kLines, B), kCtfThreads, smem, st>>>(
      plan, tw, Z, (float)(1.0 / ((double)d * d)), (float)(cscale / ((double)d * d)), pred,
      dproj);
}

cudaError_t launch_ctf_loss(int d, int B, float apix, const FftPlan &plan, const float2 *tw,
                            const float *proj, const float *ctf, const float *ctf_params,
                            const float *images, float2 *Z, double *lossp, float *pred,
                            float *dproj, double *loss_img, double *loss, cudaStream_t st) {
  const int nblk = (int)ctf_partials(d);
  if (ctf_lines(d) == 16)
    launch_ctf_passes<16>(d, B, apix, plan, tw, proj, ctf, ctf_params, images, Z, lossp, pred,
                          dproj, st);
  else
    launch_ctf_passes<8>(d, B, apix, plan, tw, proj, ctf, ctf_params, images, Z, lossp, pred,
                         dproj, st);
  if (loss_img || loss) {
    // per-image losses land in loss_img, or after the partials when the
    // caller does not want them (lossp holds max_B * nblk + max_B doubles)
    double *li = loss_img ? loss_img : lossp + (int64_t)B * nblk;
    double inv_d4 = 1.0 / ((double)d * d * (double)d * d);
    loss_img_kernel<<<(B + 7) / 8, 256, 0, st>>>(lossp, B, nblk, inv_d4, li);
    if (loss) loss_mean_kernel<<<1, 256, 0, st>>>(li, B, loss);
  }
  return cudaGetLastError();
}

}  // namespace gem
