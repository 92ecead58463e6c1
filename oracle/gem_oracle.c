/*
 * gem_oracle.c -- plain FP64 CPU statement of the GEM hot path.
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark load this library.  The CUDA library never calls it,
 * and the two share no code, header, table or helper.
 *
 * Method: GEM, "3D Gaussian Splatting for Efficient and Accurate Cryo-EM
 * Reconstruction" (arXiv 2509.25075).
 *   Eq. G (Sec. 3.2)       G_j(x) = rho_j exp(-1/2 (x-p_j)^T Sigma_j^-1 (x-p_j)),
 *                          Sigma_j = R_j S_j S_j^T R_j^T.
 *   Eq. render (Sec. 3.2)  I^(r) = sum_j rho_j / (2 pi |S^_j|^1/2)
 *                                   exp(-1/2 (x^-p^_j)^T S^_j^-1 (x^-p^_j)),
 *                          p^, S^ = first two rows / columns of the viewed
 *                          mean and covariance (Appendix, "Derivation of 3DGS
 *                          Projection": parallel rays, J = I).
 *   Eq. accu (Sec. 3.2)    only terms whose 2D value exceeds tau are summed.
 *   Eq. loss (Sec. 3.2)    I_pred = F^-1(F(C) . F(I^)),  L = ||I_pred - I||^2,
 *                          taken as a mean squared error.
 *
 * Everything is brute force: every pixel against every Gaussian (no culling,
 * no tiles, no order), explicit O(d^3) separable DFTs, and gradients summed
 * pixel by pixel from d(value)/d(theta).  The accumulation order of Eq. accu
 * (the z-sort of Sec. 3.2) only changes rounding of an additive sum, so the
 * oracle sums in Gaussian index order.
 *
 * Readings of points the paper leaves open (each is also listed in the design
 * notes of the repository):
 *   - 11 parameters per Gaussian, in this order: p (3, Angstrom), s (3, the
 *     diagonal of S, Angstrom, sign irrelevant), q (4, quaternion w,x,y,z,
 *     normalised here), rho (1).
 *   - norm_mode 0 uses the amplitude of Eq. render, rho / (2 pi |S^|^1/2)
 *     ("rho is a mass").  norm_mode 1 uses the exact line integral of Eq. G,
 *     rho (2 pi)^1/2 (|Sigma| / |S^|)^1/2 ("rho is a peak density"); the
 *     appendix keeps the (2 pi)^3/2 |Sigma|^1/2 factor on one line and drops
 *     it on the next, so both readings are offered.
 *   - The projection integral runs over the whole line (the appendix does;
 *     Eq. ctf writes a half line).
 *   - Pixel (row v, column u) of a d x d image sits at
 *     x^ = ((u - d/2) apix, (v - d/2) apix) Angstrom.
 *   - View b: camera coordinates x' = R_b x + (t_b, 0); the beam runs along z'.
 *   - A Gaussian whose projected covariance is not positive definite, whose
 *     quaternion is zero, or whose rho is not positive contributes nothing
 *     (with tau >= 0 no negative value can pass Eq. accu).
 *   - CTF: a real transfer function H on the 2D frequency grid.  On the
 *     half-spectrum (rfft) grid [d][d/2+1] the full grid is filled by
 *     H(-k) = H(k), and the operator uses Hs(k) = (H(k) + H(-k)) / 2, which
 *     keeps I_pred real; for a symmetric H this is irfft2(H . rfft2(I^)).
 *     Forward DFT unnormalised, inverse with 1/d^2, circular, no padding.
 *   - Loss: L = (1/B) sum_b (1/d^2) sum_pixels (I_pred - I)^2.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NPAR 11
static const double PI = 3.14159265358979323846;

int gem_oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* One Gaussian seen from one view: the 2D Gaussian of Eq. render and its    */
/* derivatives with respect to the 11 parameters.                            */
/* ------------------------------------------------------------------------ */
typedef struct {
  int valid;
  double mean[2];          /* p^ (Angstrom)                                 */
  double cov[2][2];        /* S^ (Angstrom^2)                               */
  double icov[2][2];       /* S^^-1                                         */
  double amp;              /* value of the 2D term at its centre            */
  double depth;            /* z' of the centre                              */
  double dmean[2][NPAR];   /* d p^ / d theta                                */
  double dcov[2][2][NPAR]; /* d S^ / d theta                                */
  double dlnamp[NPAR];     /* d ln(amp) / d theta                           */
} proj_t;

/* Rotation of a unit quaternion (w, v):  R = (w^2 - v.v) I + 2 v v^T + 2 w [v]x */
static void rot_of_unit_quat(double w, const double v[3], double R[3][3]) {
  double c = w * w - (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) R[a][b] = (a == b ? c : 0.0) + 2.0 * v[a] * v[b];
  R[0][1] -= 2.0 * w * v[2];
  R[0][2] += 2.0 * w * v[1];
  R[1][0] += 2.0 * w * v[2];
  R[1][2] -= 2.0 * w * v[0];
  R[2][0] -= 2.0 * w * v[1];
  R[2][1] += 2.0 * w * v[0];
}

/* Derivative of the formula above with respect to component n of (w, v):
 *   dR/dw   = 2 w I + 2 [v]x
 *   dR/dv_i = -2 v_i I + 2 (e_i v^T + v e_i^T) + 2 w [e_i]x                  */
static void drot_of_unit_quat(double w, const double v[3], int n, double D[3][3]) {
  double cross[3][3];
  memset(D, 0, sizeof(double) * 9);
  if (n == 0) {
    double vx[3][3] = {{0, -v[2], v[1]}, {v[2], 0, -v[0]}, {-v[1], v[0], 0}};
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) D[a][b] = (a == b ? 2.0 * w : 0.0) + 2.0 * vx[a][b];
    return;
  }
  int i = n - 1;
  double e[3] = {0, 0, 0};
  e[i] = 1.0;
  double ex[3][3] = {{0, -e[2], e[1]}, {e[2], 0, -e[0]}, {-e[1], e[0], 0}};
  memcpy(cross, ex, sizeof(cross));
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      D[a][b] = (a == b ? -2.0 * v[i] : 0.0) + 2.0 * (e[a] * v[b] + v[a] * e[b]) +
                2.0 * w * cross[a][b];
}

/* theta: 11 parameters; Rv: 3x3 row-major view rotation; tv: 2 translation (A). */
static void project_one(const double *theta, const double *Rv, const double *tv,
                        int norm_mode, int want_jac, proj_t *o) {
  memset(o, 0, sizeof(*o));
  const double *p = theta, *s = theta + 3, *q = theta + 6;
  double rho = theta[10];
  double qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  if (!(qn > 0.0) || !isfinite(qn) || !(rho > 0.0)) return;
  double w = q[0] / qn, v[3] = {q[1] / qn, q[2] / qn, q[3] / qn};
  double Rq[3][3];
  rot_of_unit_quat(w, v, Rq);
  /* V = (first two rows of R_b) . R_q */
  double V[2][3];
  for (int a = 0; a < 2; ++a)
    for (int k = 0; k < 3; ++k) {
      double acc = 0;
      for (int m = 0; m < 3; ++m) acc += Rv[a * 3 + m] * Rq[m][k];
      V[a][k] = acc;
    }
  double s2[3] = {s[0] * s[0], s[1] * s[1], s[2] * s[2]};
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      double acc = 0;
      for (int k = 0; k < 3; ++k) acc += V[a][k] * s2[k] * V[b][k];
      o->cov[a][b] = acc;
    }
  double det = o->cov[0][0] * o->cov[1][1] - o->cov[0][1] * o->cov[1][0];
  if (!(det > 0.0) || !isfinite(det)) return;
  o->icov[0][0] = o->cov[1][1] / det;
  o->icov[1][1] = o->cov[0][0] / det;
  o->icov[0][1] = -o->cov[0][1] / det;
  o->icov[1][0] = -o->cov[1][0] / det;
  for (int a = 0; a < 2; ++a) {
    double acc = tv[a];
    for (int m = 0; m < 3; ++m) acc += Rv[a * 3 + m] * p[m];
    o->mean[a] = acc;
  }
  o->depth = Rv[6] * p[0] + Rv[7] * p[1] + Rv[8] * p[2];
  if (norm_mode == 0) {
    o->amp = rho / (2.0 * PI * sqrt(det));
  } else {
    double detS = s2[0] * s2[1] * s2[2];
    o->amp = rho * sqrt(2.0 * PI) * sqrt(detS / det);
    if (!(o->amp > 0.0)) return;
  }
  o->valid = 1;
  if (!want_jac) return;

  /* d mean / d p */
  for (int a = 0; a < 2; ++a)
    for (int m = 0; m < 3; ++m) o->dmean[a][m] = Rv[a * 3 + m];
  /* d cov / d s_k = 2 s_k V[:,k] V[:,k]^T */
  for (int k = 0; k < 3; ++k)
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) o->dcov[a][b][3 + k] = 2.0 * s[k] * V[a][k] * V[b][k];
  /* d cov / d q_m through the normalisation qbar = q / |q| */
  double qb[4] = {w, v[0], v[1], v[2]};
  double dR[4][3][3];
  for (int n = 0; n < 4; ++n) drot_of_unit_quat(w, v, n, dR[n]);
  for (int m = 0; m < 4; ++m) {
    double dRq[3][3] = {{0}};
    for (int n = 0; n < 4; ++n) {
      double dqbar = ((n == m ? 1.0 : 0.0) - qb[n] * qb[m]) / qn;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) dRq[a][b] += dR[n][a][b] * dqbar;
    }
    double dV[2][3];
    for (int a = 0; a < 2; ++a)
      for (int k = 0; k < 3; ++k) {
        double acc = 0;
        for (int mm = 0; mm < 3; ++mm) acc += Rv[a * 3 + mm] * dRq[mm][k];
        dV[a][k] = acc;
      }
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) {
        double acc = 0;
        for (int k = 0; k < 3; ++k) acc += dV[a][k] * s2[k] * V[b][k] + V[a][k] * s2[k] * dV[b][k];
        o->dcov[a][b][6 + m] = acc;
      }
  }
  /* d ln amp: -1/2 tr(S^^-1 dS^) for every parameter, plus the explicit parts */
  for (int m = 0; m < NPAR; ++m) {
    double tr = 0;
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) tr += o->icov[a][b] * o->dcov[b][a][m];
    o->dlnamp[m] = -0.5 * tr;
  }
  o->dlnamp[10] += 1.0 / rho;
  if (norm_mode != 0)
    for (int k = 0; k < 3; ++k) o->dlnamp[3 + k] += 1.0 / s[k];
}

/* Value of the projected Gaussian at x^ (Angstrom). */
static double value_at(const proj_t *g, double x, double y) {
  double dx = x - g->mean[0], dy = y - g->mean[1];
  double qf = dx * (g->icov[0][0] * dx + g->icov[0][1] * dy) +
              dy * (g->icov[1][0] * dx + g->icov[1][1] * dy);
  return g->amp * exp(-0.5 * qf);
}

static double pix_coord(int idx, int d, double apix) { return ((double)idx - 0.5 * d) * apix; }

/* ------------------------------------------------------------------------ */
/* Eq. render + Eq. accu                                                     */
/* ------------------------------------------------------------------------ */

/* Projected-Gaussian summary per (view, Gaussian): mean x, mean y, cov xx,
 * cov xy, cov yy, amp, depth, valid.  out: [B][M][8]. */
void gem_oracle_preprocess(int norm_mode, int64_t M, const double *params, int B,
                           const double *Rv, const double *tv, double *out) {
#pragma omp parallel for collapse(2) schedule(static)
  for (int b = 0; b < B; ++b)
    for (int64_t j = 0; j < M; ++j) {
      proj_t g;
      project_one(params + j * NPAR, Rv + 9 * b, tv + 2 * b, norm_mode, 0, &g);
      double *o = out + ((int64_t)b * M + j) * 8;
      o[0] = g.mean[0];
      o[1] = g.mean[1];
      o[2] = g.cov[0][0];
      o[3] = g.cov[0][1];
      o[4] = g.cov[1][1];
      o[5] = g.amp;
      o[6] = g.depth;
      o[7] = g.valid;
    }
}

/* img: [B][d][d] (row v, column u). */
void gem_oracle_project(int d, double apix, double tau, int norm_mode, int64_t M,
                        const double *params, int B, const double *Rv, const double *tv,
                        double *img) {
  proj_t *g = (proj_t *)malloc(sizeof(proj_t) * (size_t)(M > 0 ? M : 1));
  for (int b = 0; b < B; ++b) {
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < M; ++j)
      project_one(params + j * NPAR, Rv + 9 * b, tv + 2 * b, norm_mode, 0, &g[j]);
#pragma omp parallel for schedule(dynamic, 1)
    for (int v = 0; v < d; ++v)
      for (int u = 0; u < d; ++u) {
        double x = pix_coord(u, d, apix), y = pix_coord(v, d, apix), acc = 0;
        for (int64_t j = 0; j < M; ++j) {
          if (!g[j].valid) continue;
          double val = value_at(&g[j], x, y);
          if (val > tau) acc += val;
        }
        img[((int64_t)b * d + v) * d + u] = acc;
      }
  }
  free(g);
}

/* Same sum at selected pixels only.  pix[i] = (b * d + v) * d + u. */
void gem_oracle_project_pixels(int d, double apix, double tau, int norm_mode, int64_t M,
                               const double *params, int B, const double *Rv,
                               const double *tv, int64_t npix, const int64_t *pix,
                               double *out) {
  (void)B;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t i = 0; i < npix; ++i) {
    int64_t b = pix[i] / ((int64_t)d * d);
    int64_t rem = pix[i] % ((int64_t)d * d);
    int v = (int)(rem / d), u = (int)(rem % d);
    double x = pix_coord(u, d, apix), y = pix_coord(v, d, apix), acc = 0;
    for (int64_t j = 0; j < M; ++j) {
      proj_t g;
      project_one(params + j * NPAR, Rv + 9 * b, tv + 2 * b, norm_mode, 0, &g);
      if (!g.valid) continue;
      double val = value_at(&g, x, y);
      if (val > tau) acc += val;
    }
    out[i] = acc;
  }
}

/* For every (view, Gaussian, tile): 1 if some pixel centre of the tile has a
 * value above tau.  Tiles are tile x tile pixels, numbered row-major over the
 * (d/tile) x (d/tile) grid.  out: [B][M][T] bytes. */
void gem_oracle_tile_hits(int d, double apix, double tau, int norm_mode, int tile, int64_t M,
                          const double *params, int B, const double *Rv, const double *tv,
                          uint8_t *out) {
  int nt = d / tile, T = nt * nt;
#pragma omp parallel for collapse(2) schedule(dynamic, 16)
  for (int b = 0; b < B; ++b)
    for (int64_t j = 0; j < M; ++j) {
      proj_t g;
      project_one(params + j * NPAR, Rv + 9 * b, tv + 2 * b, norm_mode, 0, &g);
      uint8_t *o = out + ((int64_t)b * M + j) * T;
      for (int t = 0; t < T; ++t) {
        o[t] = 0;
        if (!g.valid) continue;
        int ty = t / nt, tx = t % nt;
        for (int v = ty * tile; v < (ty + 1) * tile && !o[t]; ++v)
          for (int u = tx * tile; u < (tx + 1) * tile; ++u)
            if (value_at(&g, pix_coord(u, d, apix), pix_coord(v, d, apix)) > tau) {
              o[t] = 1;
              break;
            }
      }
    }
}

/* ------------------------------------------------------------------------ */
/* CTF (Eq. loss)                                                            */
/* ------------------------------------------------------------------------ */

/* Signed frequency index of DFT bin k (bin d/2 is -d/2). */
static int signed_bin(int k, int d) { return k < d / 2 ? k : k - d; }

/* Textbook CTF at spatial frequency (fx, fy) in 1/Angstrom.
 * prm: defocus U (A), defocus V (A), astigmatism angle (rad), voltage (kV),
 *      Cs (mm), amplitude contrast w, phase shift (rad), B-factor (A^2).
 *   lambda = 12.2643247 / sqrt(V (1 + 0.978466e-6 V))  (relativistic electron
 *            wavelength in Angstrom, V in volts)
 *   dF(a)  = (dU + dV)/2 + (dU - dV)/2 cos(2 (a - a_ast)),  a = atan2(fy, fx)
 *   chi    = pi lambda dF k^2 - pi/2 Cs lambda^3 k^4 + phase
 *   H      = -(sqrt(1 - w^2) sin chi + w cos chi) exp(-B k^2 / 4)          */
double gem_oracle_ctf_value(const double *prm, double fx, double fy) {
  double volt = prm[3] * 1e3;
  double lam = 12.2643247 / sqrt(volt * (1.0 + 0.978466e-6 * volt));
  double k2 = fx * fx + fy * fy;
  double ang = atan2(fy, fx);
  double df = 0.5 * (prm[0] + prm[1]) + 0.5 * (prm[0] - prm[1]) * cos(2.0 * (ang - prm[2]));
  double cs = prm[4] * 1e7;
  double chi = PI * lam * df * k2 - 0.5 * PI * cs * lam * lam * lam * k2 * k2 + prm[6];
  double w = prm[5];
  return -(sqrt(1.0 - w * w) * sin(chi) + w * cos(chi)) * exp(-prm[7] * k2 / 4.0);
}

/* Full-grid symmetrised transfer function from CTF parameters.
 * Bin k carries the formula at its signed frequency; the operator uses the
 * mean of bin k and its DFT partner bin (-k mod d).  The two differ only on
 * the Nyquist row/column, where the partner bin has the same (negative)
 * Nyquist frequency rather than the opposite one.
 * prm: [B][8]; full: [B][d][d] indexed [ky][kx]. */
void gem_oracle_ctf_grid_from_params(int d, double apix, int B, const double *prm,
                                     double *full) {
  for (int b = 0; b < B; ++b)
    for (int ky = 0; ky < d; ++ky)
      for (int kx = 0; kx < d; ++kx) {
        int mkx = (d - kx) % d, mky = (d - ky) % d;
        double h = gem_oracle_ctf_value(prm + 8 * b, signed_bin(kx, d) / (d * apix),
                                        signed_bin(ky, d) / (d * apix));
        double hm = gem_oracle_ctf_value(prm + 8 * b, signed_bin(mkx, d) / (d * apix),
                                         signed_bin(mky, d) / (d * apix));
        full[((int64_t)b * d + ky) * d + kx] = 0.5 * (h + hm);
      }
}

/* Full-grid symmetrised transfer function from a half-spectrum array.
 * half: [B][d][d/2+1] indexed [ky][kx]; full: [B][d][d]. */
void gem_oracle_ctf_grid_from_half(int d, int B, const double *half, double *full) {
  int hw = d / 2 + 1;
  for (int b = 0; b < B; ++b) {
    const double *h = half + (int64_t)b * d * hw;
    for (int ky = 0; ky < d; ++ky)
      for (int kx = 0; kx < d; ++kx) {
        int mky = (d - ky) % d, mkx = (d - kx) % d;
        double a = kx <= d / 2 ? h[ky * hw + kx] : h[mky * hw + mkx];
        double c = mkx <= d / 2 ? h[mky * hw + mkx] : h[ky * hw + kx];
        full[((int64_t)b * d + ky) * d + kx] = 0.5 * (a + c);
      }
  }
}

/* 2D DFT of a complex d x d array, separable, O(d^3).  sign -1: forward. */
static void dft2(int d, int sign, const double *re_in, const double *im_in, double *re_out,
                 double *im_out) {
  double *cr = (double *)malloc(sizeof(double) * d), *ci = (double *)malloc(sizeof(double) * d);
  double *tr = (double *)malloc(sizeof(double) * d * d), *ti = (double *)malloc(sizeof(double) * d * d);
  for (int m = 0; m < d; ++m) {
    cr[m] = cos(2.0 * PI * m / d);
    ci[m] = sign * sin(2.0 * PI * m / d);
  }
  /* along x (within each row) */
  for (int y = 0; y < d; ++y)
    for (int k = 0; k < d; ++k) {
      double ar = 0, ai = 0;
      for (int x = 0; x < d; ++x) {
        int m = (int)(((int64_t)k * x) % d);
        double xr = re_in[y * d + x], xi = im_in ? im_in[y * d + x] : 0.0;
        ar += xr * cr[m] - xi * ci[m];
        ai += xr * ci[m] + xi * cr[m];
      }
      tr[y * d + k] = ar;
      ti[y * d + k] = ai;
    }
  /* along y (within each column) */
  for (int k = 0; k < d; ++k)
    for (int x = 0; x < d; ++x) {
      double ar = 0, ai = 0;
      for (int y = 0; y < d; ++y) {
        int m = (int)(((int64_t)k * y) % d);
        ar += tr[y * d + x] * cr[m] - ti[y * d + x] * ci[m];
        ai += tr[y * d + x] * ci[m] + ti[y * d + x] * cr[m];
      }
      re_out[k * d + x] = ar;
      im_out[k * d + x] = ai;
    }
  free(cr);
  free(ci);
  free(tr);
  free(ti);
}

/* out_b = Re F^-1( Hs_b . F(in_b) ), unnormalised forward, 1/d^2 inverse.
 * hfull: [B][d][d] (already symmetrised); in, out: [B][d][d]. */
void gem_oracle_ctf_apply(int d, int B, const double *hfull, const double *in, double *out) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int b = 0; b < B; ++b) {
    int64_t n = (int64_t)d * d;
    double *fr = (double *)malloc(sizeof(double) * n), *fi = (double *)malloc(sizeof(double) * n);
    double *gr = (double *)malloc(sizeof(double) * n), *gi = (double *)malloc(sizeof(double) * n);
    dft2(d, -1, in + b * n, NULL, fr, fi);
    for (int64_t i = 0; i < n; ++i) {
      fr[i] *= hfull[b * n + i];
      fi[i] *= hfull[b * n + i];
    }
    dft2(d, +1, fr, fi, gr, gi);
    for (int64_t i = 0; i < n; ++i) out[b * n + i] = gr[i] / (double)n;
    free(fr);
    free(fi);
    free(gr);
    free(gi);
  }
}

/* Eq. loss with its adjoint.
 *   pred = C * proj,  r = pred - images,
 *   loss_img[b] = (1/d^2) sum r^2,  return (1/B) sum_b loss_img[b],
 *   g = dL/dproj = C^T (2 r / (B d^2)) = C * (2 r / (B d^2))  (Hs real, even).
 * Any of pred, loss_img, g may be NULL. */
double gem_oracle_loss(int d, int B, const double *hfull, const double *proj,
                       const double *images, double *pred, double *loss_img, double *g) {
  int64_t n = (int64_t)d * d;
  double *p = (double *)malloc(sizeof(double) * n * B);
  double *r = (double *)malloc(sizeof(double) * n * B);
  gem_oracle_ctf_apply(d, B, hfull, proj, p);
  double total = 0;
  for (int b = 0; b < B; ++b) {
    double acc = 0;
    for (int64_t i = 0; i < n; ++i) {
      double e = p[b * n + i] - images[b * n + i];
      acc += e * e;
      r[b * n + i] = 2.0 * e / ((double)B * (double)n);
    }
    if (loss_img) loss_img[b] = acc / (double)n;
    total += acc / (double)n;
  }
  if (pred) memcpy(pred, p, sizeof(double) * n * B);
  if (g) gem_oracle_ctf_apply(d, B, hfull, r, g);
  free(p);
  free(r);
  return total / B;
}

/* ------------------------------------------------------------------------ */
/* Gradient of L with respect to the 11 parameters, given g = dL/dproj.      */
/* dL/dtheta = sum_b sum_pixels g_b(pixel) [value > tau] d value / d theta,   */
/* d value/d theta = value (d ln amp + (S^-1 dx) . d p^                       */
/*                          + 1/2 (S^-1 dx)^T dS^ (S^-1 dx)).                 */
/* sel: indices of the Gaussians wanted (NULL: all M, then nsel = M).        */
/* grad: [nsel][11].                                                         */
/* ------------------------------------------------------------------------ */
/* absolute != 0: the same loop summing |g * dvalue/dtheta| instead (the scale
 * against which the rounding error of a float sum of these terms is bounded;
 * test infrastructure, not part of the method).  border > 0: sum
 * |g * dvalue/dtheta| over the pairs whose value lies within border * tau of
 * tau, on either side (the pairs a float32 evaluation of Eq. accu may keep
 * or drop differently from this double one; test infrastructure). */
static void grad_loop(int d, double apix, double tau, int norm_mode, const double *params, int B,
                      const double *Rv, const double *tv, const double *g, int64_t nsel,
                      const int64_t *sel, int absolute, double border, double *grad);

void gem_oracle_grad(int d, double apix, double tau, int norm_mode, int64_t M,
                     const double *params, int B, const double *Rv, const double *tv,
                     const double *g, int64_t nsel, const int64_t *sel, double *grad) {
  (void)M;
  grad_loop(d, apix, tau, norm_mode, params, B, Rv, tv, g, nsel, sel, 0, 0.0, grad);
}

void gem_oracle_grad_abs(int d, double apix, double tau, int norm_mode, int64_t M,
                         const double *params, int B, const double *Rv, const double *tv,
                         const double *g, int64_t nsel, const int64_t *sel, double *grad) {
  (void)M;
  grad_loop(d, apix, tau, norm_mode, params, B, Rv, tv, g, nsel, sel, 1, 0.0, grad);
}

void gem_oracle_grad_border(int d, double apix, double tau, int norm_mode, int64_t M,
                            const double *params, int B, const double *Rv, const double *tv,
                            const double *g, int64_t nsel, const int64_t *sel, double rel,
                            double *grad) {
  (void)M;
  grad_loop(d, apix, tau, norm_mode, params, B, Rv, tv, g, nsel, sel, 1, rel, grad);
}

static void grad_loop(int d, double apix, double tau, int norm_mode, const double *params, int B,
                      const double *Rv, const double *tv, const double *g, int64_t nsel,
                      const int64_t *sel, int absolute, double border, double *grad) {
  int64_t n = (int64_t)d * d;
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t i = 0; i < nsel; ++i) {
    int64_t j = sel ? sel[i] : i;
    double acc[NPAR] = {0};
    for (int b = 0; b < B; ++b) {
      proj_t pg;
      project_one(params + j * NPAR, Rv + 9 * b, tv + 2 * b, norm_mode, 1, &pg);
      if (!pg.valid) continue;
      for (int v = 0; v < d; ++v)
        for (int u = 0; u < d; ++u) {
          double x = pix_coord(u, d, apix), y = pix_coord(v, d, apix);
          double val = value_at(&pg, x, y);
          if (border > 0.0 ? !(fabs(val - tau) <= border * tau) : !(val > tau)) continue;
          double gv = g[b * n + (int64_t)v * d + u] * val;
          double dx = x - pg.mean[0], dy = y - pg.mean[1];
          double w0 = pg.icov[0][0] * dx + pg.icov[0][1] * dy;
          double w1 = pg.icov[1][0] * dx + pg.icov[1][1] * dy;
          for (int m = 0; m < NPAR; ++m) {
            double t = pg.dlnamp[m] + w0 * pg.dmean[0][m] + w1 * pg.dmean[1][m] +
                       0.5 * (w0 * (pg.dcov[0][0][m] * w0 + pg.dcov[0][1][m] * w1) +
                              w1 * (pg.dcov[1][0][m] * w0 + pg.dcov[1][1][m] * w1));
            acc[m] += absolute ? fabs(gv * t) : gv * t;
          }
        }
    }
    for (int m = 0; m < NPAR; ++m) grad[i * NPAR + m] = acc[m];
  }
}

/* ------------------------------------------------------------------------ */
/* Eq. query: density of the Gaussians on the voxel grid                     */
/* ------------------------------------------------------------------------ */

/* The 3D Gaussian of Eq. G: mean, precision Sigma^-1 (cofactors over the
 * determinant of Sigma = R S S^T R^T), amplitude.  norm_mode 1: amplitude rho
 * (a peak density, Eq. G as printed); norm_mode 0: rho / ((2 pi)^3/2
 * |Sigma|^1/2), the normalised density of mass rho whose line integral is the
 * Eq. render term.  Returns 0 when the Gaussian contributes nothing. */
static int gauss3(const double *theta, int norm_mode, double mean[3], double P[3][3],
                  double *amp) {
  const double *s = theta + 3, *q = theta + 6;
  double rho = theta[10];
  double qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  if (!(qn > 0.0) || !isfinite(qn) || !(rho > 0.0)) return 0;
  double w = q[0] / qn, v[3] = {q[1] / qn, q[2] / qn, q[3] / qn};
  double Rq[3][3], S[3][3];
  rot_of_unit_quat(w, v, Rq);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double acc = 0;
      for (int k = 0; k < 3; ++k) acc += Rq[a][k] * s[k] * s[k] * Rq[b][k];
      S[a][b] = acc;
    }
  double C[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      int a1 = (a + 1) % 3, a2 = (a + 2) % 3, b1 = (b + 1) % 3, b2 = (b + 2) % 3;
      C[a][b] = S[a1][b1] * S[a2][b2] - S[a1][b2] * S[a2][b1];
    }
  double det = S[0][0] * C[0][0] + S[0][1] * C[0][1] + S[0][2] * C[0][2];
  if (!(det > 0.0) || !isfinite(det)) return 0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) P[a][b] = C[b][a] / det;
  for (int a = 0; a < 3; ++a) mean[a] = theta[a];
  *amp = norm_mode == 0 ? rho / (pow(2.0 * PI, 1.5) * sqrt(det)) : rho;
  return 1;
}

static double voxel_value(const double mean[3], const double P[3][3], double amp, double x,
                          double y, double z) {
  double dv[3] = {x - mean[0], y - mean[1], z - mean[2]};
  double qf = 0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) qf += dv[a] * P[a][b] * dv[b];
  return amp * exp(-0.5 * qf);
}

/* Density at selected flat voxel indices vox = (z d + y) d + x: every
 * Gaussian, terms above tau only (Eq. accu applied to the 3D value). */
void gem_oracle_query_voxels(int d, double apix, double tau, int norm_mode, int64_t M,
                             const double *params, int64_t n, const int64_t *vox, double *out) {
  double(*mean)[3] = malloc(sizeof(double[3]) * (size_t)M);
  double(*P)[3][3] = malloc(sizeof(double[3][3]) * (size_t)M);
  double *amp = malloc(sizeof(double) * (size_t)M);
  int *ok = malloc(sizeof(int) * (size_t)M);
  for (int64_t j = 0; j < M; ++j) ok[j] = gauss3(params + j * NPAR, norm_mode, mean[j], P[j], &amp[j]);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    int64_t v = vox[i];
    int x = (int)(v % d), y = (int)((v / d) % d), z = (int)(v / ((int64_t)d * d));
    double X = pix_coord(x, d, apix), Y = pix_coord(y, d, apix), Z = pix_coord(z, d, apix);
    double acc = 0;
    for (int64_t j = 0; j < M; ++j) {
      if (!ok[j]) continue;
      double val = voxel_value(mean[j], P[j], amp[j], X, Y, Z);
      if (val > tau) acc += val;
    }
    out[i] = acc;
  }
  free(mean);
  free(P);
  free(amp);
  free(ok);
}

/* The whole d^3 grid, vol[z][y][x]. */
void gem_oracle_query(int d, double apix, double tau, int norm_mode, int64_t M,
                      const double *params, double *vol) {
  int64_t n = (int64_t)d * d * d;
  int64_t *vox = malloc(sizeof(int64_t) * (size_t)n);
  for (int64_t i = 0; i < n; ++i) vox[i] = i;
  gem_oracle_query_voxels(d, apix, tau, norm_mode, M, params, n, vox, vol);
  free(vox);
}
