// FP64 check mode: the whole step (a1-a6) in double precision, by the plain
// dense forms -- every pixel against every Gaussian, exponentials in double,
// explicit separable DFTs -- with the same decomposition as the float path
// (per-view 2D Gaussians, six moments per (view, Gaussian), the same chain
// rule).  It is for checking the method's arithmetic to ~1e-12, not for
// speed.
//
//   a1  per Gaussian Sigma = R S S^T R^T; per (view, Gaussian) the 2D
//       Gaussian of Eq. render in pixel units (natural-log amplitude).
//   a3  Eq. render with Eq. accu (value > tau), pixels summed over the
//       Gaussians in index order.
//   a4  Eq. loss through 2D DFTs: I_pred = F^-1(Hs F(I^)), the adjoint
//       F^-1(Hs F(2 r / (B d^2))), Hs the symmetrised transfer function.
//   a5  moments sum g val {1, dx, dy, dx^2, dx dy, dy^2} over kept pixels.
//   a6  the chain rule of the float path, in double.
#include <math.h>

#include "gem_internal.cuh"

namespace gem {

namespace {

__device__ void quat_rot_d(double w, double x, double y, double z, double R[9]) {
  R[0] = 1.0 - 2.0 * (y * y + z * z);
  R[1] = 2.0 * (x * y - w * z);
  R[2] = 2.0 * (x * z + w * y);
  R[3] = 2.0 * (x * y + w * z);
  R[4] = 1.0 - 2.0 * (x * x + z * z);
  R[5] = 2.0 * (y * z - w * x);
  R[6] = 2.0 * (x * z - w * y);
  R[7] = 2.0 * (y * z + w * x);
  R[8] = 1.0 - 2.0 * (x * x + y * y);
}

struct ShapeD {
  double s[3], q[4];
};

__device__ ShapeD shape_d(const double *th, int shape) {
  ShapeD e;
  const bool iso = (shape & kIsotropic) != 0, fixed = (shape & kNoRotation) != 0;
  e.s[0] = th[3];
  e.s[1] = iso ? th[3] : th[4];
  e.s[2] = iso ? th[3] : th[5];
  e.q[0] = fixed ? 1.0 : th[6];
  e.q[1] = fixed ? 0.0 : th[7];
  e.q[2] = fixed ? 0.0 : th[8];
  e.q[3] = fixed ? 0.0 : th[9];
  return e;
}

// a1, per Gaussian: centre, Sigma (xx xy xz yy yz zz), natural log of the
// amplitude constant (mode 0: rho / 2 pi; mode 1: rho sqrt(2 pi) |s0 s1 s2|),
// valid flag.
__global__ void f64_gauss_kernel(const double *__restrict__ params, int64_t M, int norm_mode,
                                 int shape, G64 *__restrict__ out) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= M) return;
  const double *th = params + j * kNpar;
  const ShapeD e = shape_d(th, shape);
  const double rho = th[10];
  const double qn = sqrt(e.q[0] * e.q[0] + e.q[1] * e.q[1] + e.q[2] * e.q[2] + e.q[3] * e.q[3]);
  G64 g;
  for (int a = 0; a < 3; ++a) g.p[a] = th[a];
  const double iq = qn > 0.0 ? 1.0 / qn : 0.0;
  double R[9];
  quat_rot_d(e.q[0] * iq, e.q[1] * iq, e.q[2] * iq, e.q[3] * iq, R);
  const double a0 = e.s[0] * e.s[0], a1 = e.s[1] * e.s[1], a2 = e.s[2] * e.s[2];
  g.sig[0] = R[0] * R[0] * a0 + R[1] * R[1] * a1 + R[2] * R[2] * a2;
  g.sig[1] = R[0] * R[3] * a0 + R[1] * R[4] * a1 + R[2] * R[5] * a2;
  g.sig[2] = R[0] * R[6] * a0 + R[1] * R[7] * a1 + R[2] * R[8] * a2;
  g.sig[3] = R[3] * R[3] * a0 + R[4] * R[4] * a1 + R[5] * R[5] * a2;
  g.sig[4] = R[3] * R[6] * a0 + R[4] * R[7] * a1 + R[5] * R[8] * a2;
  g.sig[5] = R[6] * R[6] * a0 + R[7] * R[7] * a1 + R[8] * R[8] * a2;
  const double two_pi = 6.283185307179586476925;
  g.lnk = norm_mode == 0 ? log(rho / two_pi) : log(rho * sqrt(two_pi) * fabs(e.s[0] * e.s[1] * e.s[2]));
  g.valid = qn > 0.0 && isfinite(qn) && rho > 0.0 && isfinite(rho) && isfinite(g.lnk);
  out[j] = g;
}

// The 2D Gaussian of one (view, Gaussian) in pixel units.
struct View64 {
  double px, py, sxx, sxy, syy, cxx, cxy, cyy, lnA;
  bool valid;
};

__device__ View64 view_d(const G64 &g, const double *Rv, const double *tv, double apix, int d) {
  View64 o;
  const double mx = Rv[0] * g.p[0] + Rv[1] * g.p[1] + Rv[2] * g.p[2] + tv[0];
  const double my = Rv[3] * g.p[0] + Rv[4] * g.p[1] + Rv[5] * g.p[2] + tv[1];
  o.px = mx / apix + 0.5 * d;
  o.py = my / apix + 0.5 * d;
  const double *s = g.sig;
  const double v0x = Rv[0] * s[0] + Rv[1] * s[1] + Rv[2] * s[2];
  const double v0y = Rv[0] * s[1] + Rv[1] * s[3] + Rv[2] * s[4];
  const double v0z = Rv[0] * s[2] + Rv[1] * s[4] + Rv[2] * s[5];
  const double v1x = Rv[3] * s[0] + Rv[4] * s[1] + Rv[5] * s[2];
  const double v1y = Rv[3] * s[1] + Rv[4] * s[3] + Rv[5] * s[4];
  const double v1z = Rv[3] * s[2] + Rv[4] * s[4] + Rv[5] * s[5];
  const double axx = v0x * Rv[0] + v0y * Rv[1] + v0z * Rv[2];
  const double axy = v0x * Rv[3] + v0y * Rv[4] + v0z * Rv[5];
  const double ayy = v1x * Rv[3] + v1y * Rv[4] + v1z * Rv[5];
  const double det = axx * ayy - axy * axy;  // Angstrom^4
  const double i2 = 1.0 / (apix * apix);
  o.sxx = axx * i2;
  o.sxy = axy * i2;
  o.syy = ayy * i2;
  const double detp = o.sxx * o.syy - o.sxy * o.sxy;
  o.cxx = o.syy / detp;
  o.cyy = o.sxx / detp;
  o.cxy = -o.sxy / detp;
  o.lnA = g.lnk - 0.5 * log(det);
  o.valid = g.valid && det > 0.0 && detp > 0.0 && isfinite(det) && isfinite(o.px) &&
            isfinite(o.py) && isfinite(o.lnA);
  return o;
}

__global__ void f64_view_kernel(const G64 *__restrict__ g, int64_t M, int B,
                                const double *__restrict__ R, const double *__restrict__ t,
                                double apix, int d, V64 *__restrict__ rec) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)B * M) return;
  const int b = (int)(i / M);
  const View64 v = view_d(g[i % M], R + 9 * b, t + 2 * b, apix, d);
  V64 r;
  r.px = v.px;
  r.py = v.py;
  r.cxx = v.cxx;
  r.cxy = v.cxy;
  r.cyy = v.cyy;
  r.lnA = v.valid ? v.lnA : -INFINITY;
  rec[i] = r;
}

__device__ __forceinline__ double value_d(const V64 &r, double u, double v, double &dx,
                                          double &dy) {
  dx = u - r.px;
  dy = v - r.py;
  const double q = r.cxx * dx * dx + 2.0 * r.cxy * dx * dy + r.cyy * dy * dy;
  return exp(r.lnA - 0.5 * q);
}

// a3: one thread per pixel, every Gaussian, index order.
__global__ void f64_project_kernel(const V64 *__restrict__ rec, int64_t M, int B, int d,
                                   double tau, double *__restrict__ proj) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n2 = (int64_t)d * d;
  if (i >= (int64_t)B * n2) return;
  const int b = (int)(i / n2);
  const int pix = (int)(i % n2);
  const double u = (double)(pix % d), v = (double)(pix / d);
  const V64 *rb = rec + (int64_t)b * M;
  double acc = 0.0;
  for (int64_t j = 0; j < M; ++j) {
    const V64 r = rb[j];
    if (r.lnA == -INFINITY) continue;
    double dx, dy;
    const double val = value_d(r, u, v, dx, dy);
    if (val > tau) acc += val;
  }
  proj[i] = acc;
}

// a5: one thread per (view, Gaussian), every pixel.
__global__ void f64_moments_kernel(const V64 *__restrict__ rec, int64_t M, int B, int d,
                                   double tau, const double *__restrict__ g,
                                   double *__restrict__ mom) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)B * M) return;
  const int b = (int)(i / M);
  const V64 r = rec[i];
  double m[6] = {0, 0, 0, 0, 0, 0};
  if (r.lnA != -INFINITY) {
    const double *gb = g + (int64_t)b * d * d;
    for (int v = 0; v < d; ++v)
      for (int u = 0; u < d; ++u) {
        double dx, dy;
        const double val = value_d(r, (double)u, (double)v, dx, dy);
        if (!(val > tau)) continue;
        const double gv = gb[(int64_t)v * d + u] * val;
        m[0] += gv;
        m[1] += gv * dx;
        m[2] += gv * dy;
        m[3] += gv * dx * dx;
        m[4] += gv * dx * dy;
        m[5] += gv * dy * dy;
      }
  }
  for (int k = 0; k < 6; ++k) mom[i * 6 + k] = m[k];
}

// a6: the float path's chain rule in double, summed over every view.
__global__ void f64_chain_kernel(const double *__restrict__ params, const G64 *__restrict__ gp,
                                 int64_t M, int B, const double *__restrict__ R,
                                 const double *__restrict__ t, double apix, int d, int norm_mode,
                                 int shape, const double *__restrict__ mom,
                                 double *__restrict__ grad) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= M) return;
  const G64 g = gp[j];
  double *out = grad + j * kNpar;
  for (int k = 0; k < kNpar; ++k) out[k] = 0.0;
  if (!g.valid) return;
  double GS[6] = {0, 0, 0, 0, 0, 0}, DP[3] = {0, 0, 0}, M0 = 0.0;
  const double inv = 1.0 / apix;
  for (int b = 0; b < B; ++b) {
    const double *mm = mom + ((int64_t)b * M + j) * 6;
    const View64 v = view_d(g, R + 9 * b, t + 2 * b, apix, d);
    if (!v.valid) continue;
    const double m0 = mm[0], m1 = mm[1], m2 = mm[2], m3 = mm[3], m4 = mm[4], m5 = mm[5];
    const double gpx = v.cxx * m1 + v.cxy * m2, gpy = v.cxy * m1 + v.cyy * m2;
    const double gxx = -0.5 * m3, gxy = -0.5 * m4, gyy = -0.5 * m5;
    const double u_xx = v.cxx * gxx + v.cxy * gxy, u_xy = v.cxx * gxy + v.cxy * gyy;
    const double u_yx = v.cxy * gxx + v.cyy * gxy, u_yy = v.cxy * gxy + v.cyy * gyy;
    const double t_xx = u_xx * v.cxx + u_xy * v.cxy;
    const double t_xy = u_xx * v.cxy + u_xy * v.cyy;
    const double t_yy = u_yx * v.cxy + u_yy * v.cyy;
    const double hxx = -t_xx - 0.5 * m0 * v.cxx;
    const double hxy = -t_xy - 0.5 * m0 * v.cxy;
    const double hyy = -t_yy - 0.5 * m0 * v.cyy;
    const double *Rl = R + 9 * b;
    const double r0[3] = {Rl[0], Rl[1], Rl[2]}, r1[3] = {Rl[3], Rl[4], Rl[5]};
    int idx = 0;
    for (int a = 0; a < 3; ++a)
      for (int c = a; c < 3; ++c)
        GS[idx++] += (r0[a] * (hxx * r0[c] + hxy * r1[c]) + r1[a] * (hxy * r0[c] + hyy * r1[c])) *
                     inv * inv;
    for (int a = 0; a < 3; ++a) DP[a] += (r0[a] * gpx + r1[a] * gpy) * inv;
    M0 += m0;
  }
  const double *th = params + j * kNpar;
  const ShapeD e = shape_d(th, shape);
  const double rho = th[10];
  const double qn = sqrt(e.q[0] * e.q[0] + e.q[1] * e.q[1] + e.q[2] * e.q[2] + e.q[3] * e.q[3]);
  const double iq = 1.0 / qn;
  const double w = e.q[0] * iq, x = e.q[1] * iq, y = e.q[2] * iq, z = e.q[3] * iq;
  double Rq[9];
  quat_rot_d(w, x, y, z, Rq);
  double G[9];
  G[0] = GS[0];
  G[4] = GS[3];
  G[8] = GS[5];
  G[1] = G[3] = GS[1];
  G[2] = G[6] = GS[2];
  G[5] = G[7] = GS[4];
  double K[9];
  for (int a = 0; a < 3; ++a)
    for (int c = 0; c < 3; ++c)
      K[3 * a + c] = G[3 * a] * Rq[c] + G[3 * a + 1] * Rq[3 + c] + G[3 * a + 2] * Rq[6 + c];
  double ds[3];
  for (int k = 0; k < 3; ++k) {
    const double dk = Rq[k] * K[k] + Rq[3 + k] * K[3 + k] + Rq[6 + k] * K[6 + k];
    ds[k] = 2.0 * e.s[k] * dk;
    if (norm_mode != 0) ds[k] += M0 / e.s[k];
  }
  double dR[9];
  for (int a = 0; a < 3; ++a)
    for (int c = 0; c < 3; ++c) dR[3 * a + c] = 2.0 * K[3 * a + c] * e.s[c] * e.s[c];
  const double dw = 2.0 * (-z * dR[1] + y * dR[2] + z * dR[3] - x * dR[5] - y * dR[6] + x * dR[7]);
  const double dxq = 2.0 * (y * dR[1] + z * dR[2] + y * dR[3] - 2.0 * x * dR[4] - w * dR[5] +
                            z * dR[6] + w * dR[7] - 2.0 * x * dR[8]);
  const double dyq = 2.0 * (-2.0 * y * dR[0] + x * dR[1] + w * dR[2] + x * dR[3] + z * dR[5] -
                            w * dR[6] + z * dR[7] - 2.0 * y * dR[8]);
  const double dzq = 2.0 * (-2.0 * z * dR[0] - w * dR[1] + x * dR[2] + w * dR[3] - 2.0 * z * dR[4] +
                            y * dR[5] + x * dR[6] + y * dR[7]);
  const double dot = w * dw + x * dxq + y * dyq + z * dzq;
  const bool iso = (shape & kIsotropic) != 0, fixed = (shape & kNoRotation) != 0;
  out[0] = DP[0];
  out[1] = DP[1];
  out[2] = DP[2];
  out[3] = iso ? ds[0] + ds[1] + ds[2] : ds[0];
  out[4] = iso ? 0.0 : ds[1];
  out[5] = iso ? 0.0 : ds[2];
  out[6] = fixed ? 0.0 : (dw - w * dot) * iq;
  out[7] = fixed ? 0.0 : (dxq - x * dot) * iq;
  out[8] = fixed ? 0.0 : (dyq - y * dot) * iq;
  out[9] = fixed ? 0.0 : (dzq - z * dot) * iq;
  out[10] = M0 / rho;
}

// ---- a4 in double --------------------------------------------------------

__global__ void f64_twiddle_kernel(double2 *__restrict__ tw, int d) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= d) return;
  double s, c;
  sincospi(-2.0 * (double)m / (double)d, &s, &c);
  tw[m] = make_double2(c, s);
}

__device__ __forceinline__ int signed_bin_d(int k, int d) { return k < d / 2 ? k : k - d; }

// The CTF of the parameter form at signed bin indices (sx, sy): the textbook
// formula, evaluated directly in double.
__device__ double ctf_value_d(const double *prm, int sx, int sy, int d, double apix) {
  const double dU = prm[0], dV = prm[1], ang = prm[2], volt = prm[3] * 1e3;
  const double cs = prm[4] * 1e7, w = prm[5], phase = prm[6], bf = prm[7];
  const double lam = 12.2643247 / sqrt(volt * (1.0 + 0.978466e-6 * volt));
  const double fx = sx / (d * apix), fy = sy / (d * apix);
  const double k2 = fx * fx + fy * fy;
  const double th = atan2(fy, fx);
  const double df = 0.5 * (dU + dV) + 0.5 * (dU - dV) * cos(2.0 * (th - ang));
  const double pi = 3.14159265358979323846;
  const double chi = pi * lam * df * k2 - 0.5 * pi * cs * lam * lam * lam * k2 * k2 + phase;
  return -(sqrt(1.0 - w * w) * sin(chi) + w * cos(chi)) * exp(-bf * k2 / 4.0);
}

// Hs[b][ky][kx] = (H(k) + H(-k mod d)) / 2 from parameters or the rfft grid.
__global__ void f64_ctf_grid_kernel(int d, int B, double apix, const double *__restrict__ prm,
                                    const double *__restrict__ half, double *__restrict__ Hs) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n2 = (int64_t)d * d;
  if (i >= (int64_t)B * n2) return;
  const int b = (int)(i / n2), ky = (int)((i % n2) / d), kx = (int)(i % d);
  const int mx = (d - kx) % d, my = (d - ky) % d;
  double h1, h2;
  if (prm) {
    const double *p = prm + 8 * b;
    h1 = ctf_value_d(p, signed_bin_d(kx, d), signed_bin_d(ky, d), d, apix);
    h2 = ctf_value_d(p, signed_bin_d(mx, d), signed_bin_d(my, d), d, apix);
  } else {
    const int hw = d / 2 + 1;
    const double *hb = half + (int64_t)b * d * hw;
    // the full grid from the half grid: H(kx, ky) = H(-kx, -ky)
    auto at = [&](int x, int y) {
      return x <= d / 2 ? hb[(int64_t)y * hw + x] : hb[(int64_t)((d - y) % d) * hw + (d - x)];
    };
    h1 = at(kx, ky);
    h2 = at(mx, my);
  }
  Hs[i] = 0.5 * (h1 + h2);
}

// One axis of a 2D DFT, [B][d][d] complex: axis 0 transforms along x
// (rows), axis 1 along y (columns).  sign -1 forward, +1 inverse (no 1/d).
__global__ void f64_dft_axis_kernel(const double2 *__restrict__ in, double2 *__restrict__ out,
                                    int d, int B, int axis, int sign,
                                    const double2 *__restrict__ tw) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n2 = (int64_t)d * d;
  if (i >= (int64_t)B * n2) return;
  const int b = (int)(i / n2), y = (int)((i % n2) / d), x = (int)(i % d);
  const double2 *ib = in + (int64_t)b * n2;
  double re = 0.0, im = 0.0;
  const int k = axis == 0 ? x : y;
  for (int m = 0; m < d; ++m) {
    const double2 v = axis == 0 ? ib[(int64_t)y * d + m] : ib[(int64_t)m * d + x];
    const double2 w = tw[(int)(((int64_t)k * m) % d)];
    const double wi = sign < 0 ? w.y : -w.y;
    re += v.x * w.x - v.y * wi;
    im += v.x * wi + v.y * w.x;
  }
  out[i] = make_double2(re, im);
}

__global__ void f64_real_to_complex(const double *__restrict__ x, double2 *__restrict__ z,
                                    int64_t n, double scale) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) z[i] = make_double2(scale * x[i], 0.0);
}

__global__ void f64_scale_by_h(double2 *__restrict__ z, const double *__restrict__ Hs, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) z[i] = make_double2(z[i].x * Hs[i], z[i].y * Hs[i]);
}

// pred = Re(z) / d^2; r = pred - images, kept as a double for the loss.
__global__ void f64_residual_kernel(const double2 *__restrict__ z, const double *__restrict__ img,
                                    int64_t n, double inv_n2, double *__restrict__ pred,
                                    double *__restrict__ r) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double p = z[i].x * inv_n2;
  if (pred) pred[i] = p;
  r[i] = p - img[i];
}

// loss_img[b] = mean of r^2 over the image (one block per image, fixed order).
__global__ void f64_loss_kernel(const double *__restrict__ r, int d, double *__restrict__ li) {
  __shared__ double red[256];
  const int b = blockIdx.x;
  const int64_t n2 = (int64_t)d * d;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n2; i += blockDim.x) {
    const double v = r[(int64_t)b * n2 + i];
    s += v * v;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) li[b] = red[0] / (double)n2;
}

__global__ void f64_loss_mean_kernel(const double *__restrict__ li, int B,
                                     double *__restrict__ loss, double *__restrict__ loss_img) {
  if (threadIdx.x != 0) return;
  double s = 0.0;
  for (int b = 0; b < B; ++b) {
    s += li[b];
    if (loss_img) loss_img[b] = li[b];
  }
  if (loss) loss[0] = s / B;
}

__global__ void f64_real_part(const double2 *__restrict__ z, int64_t n, double scale,
                              double *__restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = z[i].x * scale;
}

// blocks of 256 threads covering n items (every launch below uses 256)
inline unsigned nblk(int64_t n) { return (unsigned)((n + 255) / 256); }

}  // namespace

// Array conversions of the check mode (float inputs widened, float outputs
// narrowed; plain IEEE conversions, speed is not the point here).
__global__ void f64_widen_kernel(const float *__restrict__ x, double *__restrict__ y, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = (double)x[i];
}
__global__ void f64_narrow_kernel(const double *__restrict__ x, float *__restrict__ y, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = (float)x[i];
}

cudaError_t launch_f64_widen(const float *x, double *y, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  f64_widen_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x, y, n);
  return cudaGetLastError();
}

cudaError_t launch_f64_narrow(const double *x, float *y, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  f64_narrow_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x, y, n);
  return cudaGetLastError();
}

cudaError_t launch_f64_project(const double *params, int64_t M, int B, const double *R,
                               const double *t, double apix, int d, int norm_mode, int shape,
                               double tau, G64 *gp, V64 *rec, double *proj, cudaStream_t st) {
  f64_gauss_kernel<<<nblk(M), 256, 0, st>>>(params, M, norm_mode, shape, gp);
  f64_view_kernel<<<nblk((int64_t)B * M), 256, 0, st>>>(gp, M, B, R, t, apix, d, rec);
  f64_project_kernel<<<nblk((int64_t)B * d * d), 256, 0, st>>>(rec, M, B, d, tau, proj);
  return cudaGetLastError();
}

cudaError_t launch_f64_backward(const double *params, const G64 *gp, const V64 *rec, int64_t M,
                                int B, const double *R, const double *t, double apix, int d,
                                int norm_mode, int shape, double tau, const double *dproj,
                                double *mom, double *grad, cudaStream_t st) {
  f64_moments_kernel<<<nblk((int64_t)B * M), 256, 0, st>>>(rec, M, B, d, tau, dproj, mom);
  f64_chain_kernel<<<nblk(M), 256, 0, st>>>(params, gp, M, B, R, t, apix, d, norm_mode, shape,
                                            mom, grad);
  return cudaGetLastError();
}

// Eq. loss and its adjoint in double.  Scratch: tw [d], Hs [B][d][d],
// Za, Zb [B][d][d] complex, r [B][d][d], li [B].
cudaError_t launch_f64_ctf_loss(int d, int B, double apix, const double *proj, const double *ctf,
                                const double *prm, const double *images, double *pred,
                                double *dproj, double *loss_img, double *loss, double2 *tw,
                                double *Hs, double2 *Za, double2 *Zb, double *r, double *li,
                                cudaStream_t st) {
  const int64_t n = (int64_t)B * d * d;
  const double inv_n2 = 1.0 / ((double)d * d);
  f64_twiddle_kernel<<<nblk(d), 256, 0, st>>>(tw, d);
  f64_ctf_grid_kernel<<<nblk(n), 256, 0, st>>>(d, B, apix, prm, ctf, Hs);
  // I_pred = F^-1(Hs F(I^)) / d^2
  f64_real_to_complex<<<nblk(n), 256, 0, st>>>(proj, Za, n, 1.0);
  f64_dft_axis_kernel<<<nblk(n), 256, 0, st>>>(Za, Zb, d, B, 0, -1, tw);
  f64_dft_axis_kernel<<<nblk(n), 256, 0, st>>>(Zb, Za, d, B, 1, -1, tw);
  f64_scale_by_h<<<nblk(n), 256, 0, st>>>(Za, Hs, n);
  f64_dft_axis_kernel<<<nblk(n), 256, 0, st>>>(Za, Zb, d, B, 0, +1, tw);
  f64_dft_axis_kernel<<<nblk(n), 256, 0, st>>>(Zb, Za, d, B, 1, +1, tw);
  f64_residual_kernel<<<nblk(n), 256, 0, st>>>(Za, images, n, inv_n2, pred, r);
  f64_loss_kernel<<<B, 256, 0, st>>>(r, d, li);
  f64_loss_mean_kernel<<<1, 32, 0, st>>>(li, B, loss, loss_img);
  if (dproj) {
    // dL/dI^ = F^-1(Hs F(2 r / (B d^2))) / d^2
    f64_real_to_complex<<<nblk(n), 256, 0, st>>>(r, Za, n, 2.0 / ((double)B * d * d));
    f64_dft_axis_kernel<<<nblk(n), 256, 0, st>>>(Za, Zb, d, B, 0, -1, tw);
    f64_dft_axis_kernel<<<nblk(n), 256, 0, st>>>(Zb, Za, d, B, 1, -1, tw);
    f64_scale_by_h<<<nblk(n), 256, 0, st>>>(Za, Hs, n);
    f64_dft_axis_kernel<<<nblk(n), 256, 0, st>>>(Za, Zb, d, B, 0, +1, tw);
    f64_dft_axis_kernel<<<nblk(n), 256, 0, st>>>(Zb, Za, d, B, 1, +1, tw);
    f64_real_part<<<nblk(n), 256, 0, st>>>(Za, n, inv_n2, dproj);
  }
  return cudaGetLastError();
}

}  // namespace gem
