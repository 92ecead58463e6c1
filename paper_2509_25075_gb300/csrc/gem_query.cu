// Density query (Eq. query): V(x) = sum_j G_j(x) on the d^3 voxel grid,
// with the contribution threshold of Eq. accu applied per voxel.
//
// Each z-slice of the volume is rendered as an image by the same binning and
// forward rasteriser as the projections.  Restricted to the plane z = z_k, a
// 3D Gaussian is exactly a 2D Gaussian: with P = Sigma^-1 split into its xy
// block P_aa and the rest,
//   (x - p)^T P (x - p) = (a - m)^T P_aa (a - m) + (z - p_z)^2 / Sigma_zz,
//   m = p_a + (Sigma_az / Sigma_zz) (z - p_z)            (Schur complement),
// so the slice record has conic P_aa, centre m(z_k) and log2 amplitude
// log2 A3 - (log2 e / 2) (z_k - p_z)^2 / Sigma_zz.  Slices are independent
// "images" and run in batches of the context's max_B.
#include "gem_internal.cuh"

namespace gem {

__global__ void __launch_bounds__(256) query_prep_kernel(const float *__restrict__ params,
                                                         int64_t M, int norm_mode, int shape,
                                                         QueryPrep *__restrict__ qp) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= M) return;
  const float *th = params + j * kNpar;
  const bool iso = (shape & kIsotropic) != 0, fixed = (shape & kNoRotation) != 0;
  const float s0 = th[3], s1 = iso ? th[3] : th[4], s2 = iso ? th[3] : th[5];
  const float qw = fixed ? 1.f : th[6], qx = fixed ? 0.f : th[7], qy = fixed ? 0.f : th[8],
              qz = fixed ? 0.f : th[9];
  const float rho = th[10];
  const float qn = sqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
  QueryPrep o;
  o.p[0] = th[0];
  o.p[1] = th[1];
  o.p[2] = th[2];
  const float iq = qn > 0.f ? 1.f / qn : 0.f;
  float R[9];
  quat_rot(qw * iq, qx * iq, qy * iq, qz * iq, R);
  const float a0 = s0 * s0, a1 = s1 * s1, a2 = s2 * s2;
  const float b0 = 1.f / a0, b1 = 1.f / a1, b2 = 1.f / a2;
  // P = R diag(1/s^2) R^T (xy block), Sigma = R diag(s^2) R^T (z column)
  o.pxx = R[0] * R[0] * b0 + R[1] * R[1] * b1 + R[2] * R[2] * b2;
  o.pxy = R[0] * R[3] * b0 + R[1] * R[4] * b1 + R[2] * R[5] * b2;
  o.pyy = R[3] * R[3] * b0 + R[4] * R[4] * b1 + R[5] * R[5] * b2;
  // det of that block by Cauchy-Binet (the squared 2x2 minors of the first
  // two rows of R, weighted): positive terms, no cancellation for an
  // elongated Gaussian
  const float m12 = fmaf(R[1], R[5], -R[2] * R[4]);
  const float m20 = fmaf(R[2], R[3], -R[0] * R[5]);
  const float m01 = fmaf(R[0], R[4], -R[1] * R[3]);
  o.pdet = b1 * b2 * m12 * m12 + b0 * b2 * m20 * m20 + b0 * b1 * m01 * m01;
  const float sxz = R[0] * R[6] * a0 + R[1] * R[7] * a1 + R[2] * R[8] * a2;
  const float syz = R[3] * R[6] * a0 + R[4] * R[7] * a1 + R[5] * R[8] * a2;
  const float szz = R[6] * R[6] * a0 + R[7] * R[7] * a1 + R[8] * R[8] * a2;
  o.hz = 1.f / szz;
  o.mx = sxz * o.hz;
  o.my = syz * o.hz;
  // 3D amplitude: rho (peak density, Eq. G) in mode 1; rho / ((2 pi)^3/2
  // |s0 s1 s2|) in mode 0, the density whose line integral is Eq. render
  const float two_pi = 6.283185307179586f;
  o.l2A = norm_mode == 0 ? log2f(rho / (two_pi * sqrtf(two_pi) * fabsf(s0 * s1 * s2)))
                         : log2f(rho);
  const bool ok = qn > 0.f && isfinite(qn) && rho > 0.f && isfinite(rho) && isfinite(o.l2A) &&
                  isfinite(o.pxx) && isfinite(o.pxy) && isfinite(o.pyy) && isfinite(o.hz) &&
                  isfinite(o.mx) && isfinite(o.my) && isfinite(o.p[0]) && isfinite(o.p[1]) &&
                  o.pdet > 0.f && isfinite(o.pdet) &&
                  isfinite(o.p[2]) && a0 > 0.f && a1 > 0.f && a2 > 0.f;
  o.valid = ok ? 1.f : 0.f;
  qp[j] = o;
}

// Record of (slice k0 + blockIdx.y, Gaussian j), in the layout of Rec.
__global__ void __launch_bounds__(256) slice_prep_kernel(const QueryPrep *__restrict__ qp,
                                                         int64_t M, int k0, float apix, int d,
                                                         float l2tau, Rec *__restrict__ rec) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int b = blockIdx.y;
  if (j >= M) return;
  const QueryPrep g = qp[j];
  const float z = ((float)(k0 + b) - 0.5f * d) * apix;
  const float dz = z - g.p[2];
  const float inv = 1.f / apix;
  const float px = fmaf(fmaf(g.mx, dz, g.p[0]), inv, 0.5f * d);
  const float py = fmaf(fmaf(g.my, dz, g.p[1]), inv, 0.5f * d);
  const float a2 = apix * apix;
  const float cxx = g.pxx * a2, cxy = g.pxy * a2, cyy = g.pyy * a2;  // 1/pixel^2
  const float l2A = g.l2A - 0.5f * kLog2e * dz * dz * g.hz;
  const float det = g.pdet * a2 * a2;
  // U^T U = c^2 [[cxx, cxy], [cxy, cyy]] (the record layout of Rec)
  const float u11 = kC * sqrtf(cxx);
  const float u12 = u11 * (cxy / cxx);
  const float u22 = kC2 * sqrtf(det) / u11;
  Rec r;
  if (g.valid != 0.f && det > 0.f && isfinite(l2A) && u11 > 0.f && u22 > 0.f && isfinite(u11) &&
      isfinite(u12) && isfinite(u22)) {
    r.a = make_float4(px, py, u11, u12);
    r.b = make_float4(u22, l2A, -1.f, -1.f);
    const float kap = l2A - l2tau;
    if (kap > 0.f) {
      const float km = (kap + kMargin) * (2.f / kLog2e);
      r.b.z = sqrtf(km * cyy / det);  // covariance xx = cyy / det
      r.b.w = sqrtf(km * cxx / det);
    }
  } else {
    r.a = make_float4(px, py, 0.f, 0.f);
    r.b = make_float4(0.f, -INFINITY, -1.f, -1.f);
  }
  rec[(int64_t)b * M + j] = r;
}

cudaError_t launch_query_prep(const float *params, int64_t M, int norm_mode, int shape,
                              QueryPrep *qp, cudaStream_t st) {
  query_prep_kernel<<<(unsigned)((M + 255) / 256), 256, 0, st>>>(params, M, norm_mode, shape, qp);
  return cudaGetLastError();
}

cudaError_t launch_slice_prep(const QueryPrep *qp, int64_t M, int k0, int nslice, float apix,
                              int d, float l2tau, Rec *rec, cudaStream_t st) {
  dim3 grid((unsigned)((M + 255) / 256), (unsigned)nslice);
  slice_prep_kernel<<<grid, 256, 0, st>>>(qp, M, k0, apix, d, l2tau, rec);
  return cudaGetLastError();
}

}  // namespace gem
