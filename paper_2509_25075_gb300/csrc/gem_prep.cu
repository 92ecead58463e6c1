// Steps a1 (preprocess) and a6 (preprocess backward) of the GEM hot path.
//
// a1: per Gaussian, the factors of Sigma = R_q S S^T R_q^T (Eq. G, Sec. 3.2);
//     per (view, Gaussian), the 2D Gaussian of Eq. render: centre, the
//     triangular factor U of its exponent's quadratic form (U^T U =
//     log2(e)/2 S^^-1), amplitude and the extent of the region where it can
//     exceed tau (Eq. accu).
// a6: chain rule from the per-(view, Gaussian) moments accumulated by the
//     raster backward to dL/d(p, s, q, rho), summed over the views.
#include "gem_internal.cuh"

namespace gem {

// ---------------------------------------------------------------- a1 -----

// The parameters a Gaussian actually uses: with kNoRotation the quaternion is
// (1, 0, 0, 0); with kIsotropic all three scales equal the first.
struct Shape {
  float s0, s1, s2, qw, qx, qy, qz;
};

__device__ __forceinline__ Shape effective_shape(const float *th, int shape) {
  Shape e;
  e.s0 = th[3];
  e.s1 = (shape & kIsotropic) ? th[3] : th[4];
  e.s2 = (shape & kIsotropic) ? th[3] : th[5];
  const bool fixed = (shape & kNoRotation) != 0;
  e.qw = fixed ? 1.f : th[6];
  e.qx = fixed ? 0.f : th[7];
  e.qy = fixed ? 0.f : th[8];
  e.qz = fixed ? 0.f : th[9];
  return e;
}

// Slot order of the Gaussians: every per-Gaussian and per-(view, Gaussian)
// array of the path (GaussPrep, records, depth keys, tile lists, moments) is
// indexed by slot, and slot i holds Gaussian slot_gauss[i].  The slots
// follow a 3D Morton order of the means (a stable sort by a 15-bit key:
// 5 bits per axis over the box of side d apix centred on the origin, ties in
// index order), so Gaussians close in space, which meet the same tiles in
// every view, sit close in memory: the rasterisers' record gathers and the
// backward's moment updates then share cache lines and stay in L2.  The
// order changes no result beyond the summation order of Gaussians with equal
// 16-bit depth keys.
__device__ __forceinline__ unsigned morton_cell(float p, float inv_side) {
  // separately rounded steps (no contraction), so the cell is reproducible
  const float c = floorf(__fadd_rn(__fmul_rn(p, inv_side), 0.5f) * 32.f);
  return (unsigned)fminf(fmaxf(c, 0.f), 31.f);  // NaN clamps to 0
}

__global__ void __launch_bounds__(256) morton_key_kernel(const float *__restrict__ params,
                                                         int64_t M, float inv_side,
                                                         uint16_t *__restrict__ key) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= M) return;
  const float *th = params + j * kNpar;
  const unsigned cx = morton_cell(th[0], inv_side), cy = morton_cell(th[1], inv_side),
                 cz = morton_cell(th[2], inv_side);
  unsigned k = 0;
#pragma unroll
  for (int b = 0; b < 5; ++b)
    k |= (((cx >> b) & 1u) << (3 * b)) | (((cy >> b) & 1u) << (3 * b + 1)) |
         (((cz >> b) & 1u) << (3 * b + 2));
  key[j] = (uint16_t)k;
}

cudaError_t launch_morton_key(const float *params, int64_t M, float side, uint16_t *key,
                              cudaStream_t st) {
  morton_key_kernel<<<(unsigned)((M + 255) / 256), 256, 0, st>>>(params, M, 1.f / side, key);
  return cudaGetLastError();
}

// Per slot i (Gaussian j = slot_gauss[i]): GaussPrep, the slot-ordered copy
// of the parameters (read again by the preprocess backward) and the inverse
// map gauss_slot[j] = i.  A warp gathers its 32 parameter rows through
// shared memory, 32 consecutive words of the rows per load, and writes the
// slot-ordered copy the same way.
__global__ void __launch_bounds__(256) gauss_prep_kernel(const float *__restrict__ params,
                                                         const uint32_t *__restrict__ slot_gauss,
                                                         int64_t M, int norm_mode, int shape,
                                                         GaussPrep *__restrict__ gp,
                                                         float *__restrict__ psort,
                                                         uint32_t *__restrict__ gauss_slot) {
  __shared__ float rows[8][32 * kNpar];
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t i0 = i - lane;  // the warp's first slot
  const uint32_t j = i < M ? (slot_gauss ? slot_gauss[i] : (uint32_t)i) : 0u;
  float *buf = rows[threadIdx.x >> 5];
  for (int k = lane; k < 32 * kNpar; k += 32) {  // element k: row k / 11, entry k % 11
    const int r = k / kNpar;
    const uint32_t jr = __shfl_sync(0xffffffffu, j, r);
    buf[k] = i0 + r < M ? params[(int64_t)jr * kNpar + (k - r * kNpar)] : 0.f;
  }
  __syncwarp();
  if (psort)
    for (int k = lane; k < 32 * kNpar; k += 32)
      if (i0 + k / kNpar < M) psort[i0 * kNpar + k] = buf[k];
  if (i >= M) return;
  if (psort) gauss_slot[j] = (uint32_t)i;
  const float *th = buf + lane * kNpar;
  float p0 = th[0], p1 = th[1], p2 = th[2];
  const Shape e = effective_shape(th, shape);
  float s0 = e.s0, s1 = e.s1, s2 = e.s2;
  float qw = e.qw, qx = e.qx, qy = e.qy, qz = e.qz;
  float rho = th[10];
  float qn = sqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
  bool ok = qn > 0.f && isfinite(qn) && rho > 0.f && isfinite(rho) && isfinite(s0) &&
            isfinite(s1) && isfinite(s2) && isfinite(p0) && isfinite(p1) && isfinite(p2);
  GaussPrep g;
  g.p[0] = p0;
  g.p[1] = p1;
  g.p[2] = p2;
  float iq = ok ? 1.f / qn : 0.f;
  float R[9];
  quat_rot(qw * iq, qx * iq, qy * iq, qz * iq, R);
  // Sigma = R diag(s^2) R^T, kept as its factors (see GaussPrep)
#pragma unroll
  for (int k = 0; k < 9; ++k) g.rq[k] = R[k];
  g.a[0] = s0 * s0;
  g.a[1] = s1 * s1;
  g.a[2] = s2 * s2;
  // amplitude constant: A = 2^l2k / sqrt(det S^ [Angstrom^4])
  //   mode 0 (Eq. render):           2^l2k = rho / (2 pi)
  //   mode 1 (line integral of G):   2^l2k = rho sqrt(2 pi) |s0 s1 s2|
  const float two_pi = 6.283185307179586f;
  if (norm_mode == 0)
    g.l2k = log2f(rho / two_pi);
  else
    g.l2k = log2f(rho * sqrtf(two_pi) * fabsf(s0 * s1 * s2));
  if (!(ok && isfinite(g.l2k))) g.l2k = -INFINITY;
  gp[i] = g;
}

cudaError_t launch_gauss_prep(const float *params, const uint32_t *slot_gauss, int64_t M,
                              int norm_mode, int shape, GaussPrep *gp, float *psort,
                              uint32_t *gauss_slot, cudaStream_t st) {
  int blocks = (int)((M + 255) / 256);
  gauss_prep_kernel<<<blocks, 256, 0, st>>>(params, slot_gauss, M, norm_mode, shape, gp, psort,
                                            gauss_slot);
  return cudaGetLastError();
}

// 16-bit depth key: [-range, range] onto 0..65535 (out-of-range depths clamp).
__device__ __forceinline__ uint16_t depth_key(float z, float inv_range) {
  float k = floorf((z * inv_range + 1.f) * 32768.f);
  return (uint16_t)fminf(fmaxf(k, 0.f), 65535.f);
}

// One thread per Gaussian and group of kViewGroup views: the Gaussian's
// 64 B are read once per group, the group's views come from shared memory.
constexpr int kViewGroup = 8;
__global__ void __launch_bounds__(256) view_prep_kernel(const GaussPrep *__restrict__ gp,
                                                        int64_t M, int B, const float *__restrict__ R,
                                                        const float *__restrict__ t,
                                                        float apix, int d, float l2tau,
                                                        float inv_range, Rec *__restrict__ rec,
                                                        uint16_t *__restrict__ key) {
  __shared__ float sv[kViewGroup][12];  // R (9), t (2)
  const int b0 = blockIdx.y * kViewGroup, nv = min(kViewGroup, B - b0);
  if (threadIdx.x < kViewGroup * 11) {
    const int v = threadIdx.x / 11, k = threadIdx.x - v * 11;
    if (v < nv) sv[v][k] = k < 9 ? R[9 * (b0 + v) + k] : t[2 * (b0 + v) + (k - 9)];
  }
  __syncthreads();
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= M) return;
  const GaussPrep g = gp[j];
  for (int vv = 0; vv < nv; ++vv) {
    const int b = b0 + vv;
    View2D v = view_project(g, sv[vv], sv[vv] + 9, apix, d);
    Rec r;
    float kap = v.l2A - l2tau;  // exponent headroom above the threshold
    if (v.valid) {
      r.a = make_float4(v.px, v.py, v.u11, v.u12);
      r.b = make_float4(v.u22, v.l2A, -1.f, -1.f);
      if (kap > 0.f) {
        // |U d|^2 <= kappa + margin  =>
        //   |dx| <= sqrt((kappa + margin) * Sxx * 2 / log2 e), same for y
        float km = (kap + kMargin) * (2.f / kLog2e);
        r.b.z = sqrtf(km * v.sxx);
        r.b.w = sqrtf(km * v.syy);
      }
      // no headroom: no extent, so no tile; every per-pair test fails anyway
    } else {
      r.a = make_float4(v.px, v.py, 0.f, 0.f);
      r.b = make_float4(0.f, -INFINITY, -1.f, -1.f);
    }
    rec[(int64_t)b * M + j] = r;
    key[(int64_t)b * M + j] = depth_key(v.depth, inv_range);
  }
}

cudaError_t launch_view_prep(const GaussPrep *gp, int64_t M, int B, const float *R,
                             const float *t, float apix, int d, float l2tau, float zrange,
                             Rec *rec, uint16_t *key, cudaStream_t st) {
  dim3 grid((unsigned)((M + 255) / 256), (unsigned)((B + kViewGroup - 1) / kViewGroup));
  view_prep_kernel<<<grid, 256, 0, st>>>(gp, M, B, R, t, apix, d, l2tau, 1.f / zrange, rec, key);
  return cudaGetLastError();
}

// Record of (view b, slot s) to out[b][Gaussian of slot s][8].
__global__ void inspect_records_kernel(const Rec *__restrict__ rec,
                                       const GaussPrep *__restrict__ gp,
                                       const uint32_t *__restrict__ slot_gauss, int64_t M,
                                       int64_t n, const float *__restrict__ R,
                                       const float *__restrict__ t, float apix, int d,
                                       float *__restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  Rec r = rec[i];
  int b = (int)(i / M);
  const int64_t sl = i - (int64_t)b * M;
  float Rl[9], tl[2];
  for (int k = 0; k < 9; ++k) Rl[k] = R[9 * b + k];
  tl[0] = t[2 * b];
  tl[1] = t[2 * b + 1];
  const float depth = view_project(gp[sl], Rl, tl, apix, d).depth;
  float *o = out + ((int64_t)b * M + (slot_gauss ? (int64_t)slot_gauss[sl] : sl)) * 8;
  bool valid = r.b.y > -INFINITY;
  // conic C = U^T U / c^2
  const float u11 = r.a.z, u12 = r.a.w, u22 = r.b.x;
  o[0] = r.a.x;
  o[1] = r.a.y;
  o[2] = u11 * u11 * (1.f / kC2);
  o[3] = u11 * u12 * (1.f / kC2);
  o[4] = fmaf(u12, u12, u22 * u22) * (1.f / kC2);
  o[5] = r.b.y;
  o[6] = depth;
  o[7] = valid ? 1.f : 0.f;
}

cudaError_t launch_inspect_records(const Rec *rec, const GaussPrep *gp,
                                   const uint32_t *slot_gauss, int64_t M, int B, const float *R,
                                   const float *t, float apix, int d, float *out,
                                   cudaStream_t st) {
  int64_t n = M * B;
  inspect_records_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(rec, gp, slot_gauss, M, n,
                                                                      R, t, apix, d, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- a6 -----

// Compensated (Kahan) accumulation in float32.
struct Kahan {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    float y = x - c;
    float t = s + y;
    c = (t - s) - y;
    s = t;
  }
};

// Moments of one (view, Gaussian), accumulated by the raster backward over
// the kept pixels in float64, in the record's whitened coordinates
// z = U d (d = (u - px, v - py) in pixels, U^T U = c^2 C, C = S^^-1 the
// conic, c^2 = log2(e) / 2; w = g * value, g = dL/dproj):
//   m0 = sum w,  m1 = sum w z1,  m2 = sum w z2,
//   N = [[m3, m4], [m4, m5]] = sum w (z z^T - c^2 I).
// Since value = A exp(-1/2 d^T C d) and C = 2 ln2 U^T U:
//   dL/dpx, dL/dpy = sum w C d = 2 ln2 U^T (m1, m2)
//   dL/dS^ = 1/2 C (sum w d d^T) C - 1/2 m0 C = 2 ln2^2 U^T N U
//            (the conic's term and the amplitude's, A ~ |S^|^-1/2, already
//             combined in N: d d^T - S^ = U^-1 (z z^T - c^2 I) U^-T)
//   dL/dSigma = R2^T dL/dS^ R2 / apix^2    (S^ = R2 Sigma R2^T / apix^2)
//   dL/dp = R2^T (dL/dpx, dL/dpy) / apix
//   dL/drho = m0 / rho;  mode 1 adds m0 / s_k to dL/ds_k.
// For an elongated Gaussian every term here is of the size of its result;
// the same quantities in pixel coordinates (C (sum w d d^T) C) cancel.
// The view-independent part (Sigma -> s, q) is applied once per thread to
// the summed dL/dSigma.
// One thread per (slot, view group): params, gp, the moments and the
// partial gradient part[group][slot][11] are all by slot.
__global__ void __launch_bounds__(128) prep_bwd_kernel(
    const float *__restrict__ params, const GaussPrep *__restrict__ gp, int64_t M, int B,
    const float *__restrict__ R, const float *__restrict__ t, float apix, int d, int norm_mode,
    int shape, double *__restrict__ mom, int per_group, float *__restrict__ part) {
  const int64_t sl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int bg = blockIdx.y;
  if (sl >= M) return;
  GaussPrep g = gp[sl];
  float *out = part + ((int64_t)bg * M + sl) * kNpar;
  if (!gp_valid(g)) {
#pragma unroll
    for (int m = 0; m < kNpar; ++m) out[m] = 0.f;
    return;
  }
  Kahan GS[6], DP[3], M0;
  float inv = 1.f / apix;
  int b0 = bg * per_group, b1 = min(B, b0 + per_group);
  // the next view's moments are loaded while this view's are used
  longlong2 na = make_longlong2(0, 0), nb = na, nc = na;
  if (b0 < b1) {
    const longlong2 *m0p = reinterpret_cast<const longlong2 *>(mom + ((int64_t)b0 * M + sl) * 6);
    na = m0p[0];
    nb = m0p[1];
    nc = m0p[2];
  }
  for (int b = b0; b < b1; ++b) {
    longlong2 *mm = reinterpret_cast<longlong2 *>(mom + ((int64_t)b * M + sl) * 6);
    const longlong2 ma = na, mb = nb, mc = nc;
    if (b + 1 < b1) {
      const longlong2 *mn = mm + 3 * M;  // view b + 1
      na = mn[0];
      nb = mn[1];
      nc = mn[2];
    }
    // all six zero (bit patterns: no FP64 compare): the Gaussian has no
    // kept pixel in this view
    if ((ma.x | ma.y | mb.x | mb.y | mc.x | mc.y) == 0) continue;
    // leave the moments cleared for the next backward pass
    mm[0] = mm[1] = mm[2] = make_longlong2(0, 0);
    const float m0 = (float)__longlong_as_double(ma.x), m1 = (float)__longlong_as_double(ma.y);
    const float m2 = (float)__longlong_as_double(mb.x), m3 = (float)__longlong_as_double(mb.y);
    const float m4 = (float)__longlong_as_double(mc.x), m5 = (float)__longlong_as_double(mc.y);
    float Rl[9], tl[2];
#pragma unroll
    for (int i = 0; i < 9; ++i) Rl[i] = __ldg(R + 9 * b + i);
    tl[0] = __ldg(t + 2 * b);
    tl[1] = __ldg(t + 2 * b + 1);
    View2D v = view_project(g, Rl, tl, apix, d);
    if (!v.valid) continue;
    // d/dp^ (pixel units) = 2 ln2 U^T (m1, m2)
    constexpr float k2ln2 = 1.3862943611198906f, k2ln2sq = 0.96090602783640285f;  // 2 ln2, 2 ln2^2
    const float u11 = v.u11, u12 = v.u12, u22 = v.u22;
    float gpx = k2ln2 * (u11 * m1);
    float gpy = k2ln2 * fmaf(u12, m1, u22 * m2);
    // dL/dS^ = 2 ln2^2 U^T N U: P = N U (its second column), H = U^T P
    float p01 = fmaf(m3, u12, m4 * u22), p11 = fmaf(m4, u12, m5 * u22);
    float hxx = k2ln2sq * (u11 * u11 * m3);
    float hxy = k2ln2sq * (u11 * p01);
    float hyy = k2ln2sq * fmaf(u12, p01, u22 * p11);
    // dL/dSigma = R2^T H R2 / apix^2
    float i2 = inv * inv;
    float r0[3] = {Rl[0], Rl[1], Rl[2]}, r1[3] = {Rl[3], Rl[4], Rl[5]};
    int idx = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int c = a; c < 3; ++c) {
        float val = r0[a] * (hxx * r0[c] + hxy * r1[c]) + r1[a] * (hxy * r0[c] + hyy * r1[c]);
        GS[idx++].add(val * i2);
      }
    // dL/dp = R2^T (gpx, gpy) / apix
#pragma unroll
    for (int a = 0; a < 3; ++a) DP[a].add((r0[a] * gpx + r1[a] * gpy) * inv);
    M0.add(m0);
  }
  // view-independent part: Sigma = Rq D Rq^T, D = diag(s^2)
  const float *th = params + sl * kNpar;
  const Shape e = effective_shape(th, shape);
  float s[3] = {e.s0, e.s1, e.s2};
  float qw = e.qw, qx = e.qx, qy = e.qy, qz = e.qz, rho = th[10];
  float qn = sqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
  float iq = 1.f / qn;
  float w = qw * iq, x = qx * iq, y = qy * iq, z = qz * iq;
  float Rq[9];
  quat_rot(w, x, y, z, Rq);
  // symmetric G (3x3) from the 6 accumulated entries (xx xy xz yy yz zz);
  // off-diagonal entries of the matrix gradient appear twice in tr(G dSigma)
  float G[9];
  G[0] = GS[0].s;
  G[4] = GS[3].s;
  G[8] = GS[5].s;
  G[1] = G[3] = GS[1].s;
  G[2] = G[6] = GS[2].s;
  G[5] = G[7] = GS[4].s;
  // K = G Rq ; dL/ds_k = 2 s_k (Rq^T G Rq)_kk ; dL/dRq = 2 G Rq D
  float K[9];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      K[3 * a + c] = G[3 * a] * Rq[c] + G[3 * a + 1] * Rq[3 + c] + G[3 * a + 2] * Rq[6 + c];
  float ds[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float dk = Rq[k] * K[k] + Rq[3 + k] * K[3 + k] + Rq[6 + k] * K[6 + k];
    ds[k] = 2.f * s[k] * dk;
    if (norm_mode != 0) ds[k] += M0.s / s[k];
  }
  float dR[9];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) dR[3 * a + c] = 2.f * K[3 * a + c] * s[c] * s[c];
  // derivatives of the entry formula of quat_rot with respect to (w, x, y, z)
  float dw = 2.f * (-z * dR[1] + y * dR[2] + z * dR[3] - x * dR[5] - y * dR[6] + x * dR[7]);
  float dx = 2.f * (y * dR[1] + z * dR[2] + y * dR[3] - 2.f * x * dR[4] - w * dR[5] +
                    z * dR[6] + w * dR[7] - 2.f * x * dR[8]);
  float dy = 2.f * (-2.f * y * dR[0] + x * dR[1] + w * dR[2] + x * dR[3] + z * dR[5] -
                    w * dR[6] + z * dR[7] - 2.f * y * dR[8]);
  float dz = 2.f * (-2.f * z * dR[0] - w * dR[1] + x * dR[2] + w * dR[3] - 2.f * z * dR[4] +
                    y * dR[5] + x * dR[6] + y * dR[7]);
  // through the normalisation q / |q|
  float dot = w * dw + x * dx + y * dy + z * dz;
  out[0] = DP[0].s;
  out[1] = DP[1].s;
  out[2] = DP[2].s;
  // a shared isotropic scale collects the three entries' gradients; a fixed
  // rotation has none
  const bool iso = (shape & kIsotropic) != 0, fixed = (shape & kNoRotation) != 0;
  out[3] = iso ? ds[0] + ds[1] + ds[2] : ds[0];
  out[4] = iso ? 0.f : ds[1];
  out[5] = iso ? 0.f : ds[2];
  out[6] = fixed ? 0.f : (dw - w * dot) * iq;
  out[7] = fixed ? 0.f : (dx - x * dot) * iq;
  out[8] = fixed ? 0.f : (dy - y * dot) * iq;
  out[9] = fixed ? 0.f : (dz - z * dot) * iq;
  out[10] = M0.s / rho;
}

// grad[j][m] = sum over the view groups of part[group][slot of j][m].
__global__ void __launch_bounds__(256) grad_sum_kernel(const float *__restrict__ part,
                                                       const uint32_t *__restrict__ gauss_slot,
                                                       int nbg, int64_t M,
                                                       float *__restrict__ grad) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n = M * kNpar;
  if (i >= n) return;
  const int64_t j = i / kNpar, m = i - j * kNpar;
  const int64_t src = (gauss_slot ? (int64_t)gauss_slot[j] : j) * kNpar + m;
  // the groups' partials are loaded kU at a time, all in flight together,
  // and summed in group order
  constexpr int kU = 4;
  Kahan acc;
  for (int g0 = 0; g0 < nbg; g0 += kU) {
    float v[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) v[u] = g0 + u < nbg ? part[(int64_t)(g0 + u) * n + src] : 0.f;
#pragma unroll
    for (int u = 0; u < kU; ++u)
      if (g0 + u < nbg) acc.add(v[u]);
  }
  grad[i] = acc.s;
}

cudaError_t launch_prep_bwd(const float *params, const uint32_t *gauss_slot, const GaussPrep *gp,
                            int64_t M, int B, const float *R, const float *t, float apix, int d,
                            int norm_mode, int shape, double *mom, float *part, int nbg,
                            float *grad, cudaStream_t st) {
  // views per thread: enough (Gaussian, view-group) threads to fill the GPU
  // (about 2^20), and no more, so that the per-Gaussian reads, the
  // view-independent chain rule and the partial sums are shared by as many
  // views as possible
  const int64_t want = ((int64_t)1 << 20) / (M > 0 ? M : 1) + 1;
  const int use = (int)(want < nbg ? want : nbg);
  int per = (B + use - 1) / use;
  int groups = (B + per - 1) / per;
  dim3 grid((unsigned)((M + 127) / 128), (unsigned)groups);
  prep_bwd_kernel<<<grid, 128, 0, st>>>(params, gp, M, B, R, t, apix, d, norm_mode, shape, mom,
                                        per, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int64_t n = M * kNpar;
  grad_sum_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(part, gauss_slot, groups, M, grad);
  return cudaGetLastError();
}

}  // namespace gem
