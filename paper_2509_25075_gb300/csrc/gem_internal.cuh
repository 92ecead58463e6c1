// Internal declarations of the GEM sm_103a library: record layout, device
// helpers and the kernel launchers each .cu file provides to gem_api.cu.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gem {

constexpr int kTile = 16;     // tile side in pixels (Sec. 3.2 rasteriser, tiled)
constexpr int kNpar = 11;     // parameters per Gaussian (Sec. 1, Sec. 3.2)
constexpr float kLog2e = 1.4426950408889634f;
// Margin, in log2 units of the exponent, by which tile lists and row ranges
// are widened so that rounding in float32 never drops a pair whose value is
// above tau; the per-pair test itself is exact (value > tau).
constexpr float kMargin = 1e-3f;

// Device status bits (mirror GEM_STATUS_* in gem.h).
constexpr int kStatusCapacity = 1;

// Per-Gaussian quantities independent of the view (64 B): p (3), log2 of
// the amplitude constant (-inf for a Gaussian that contributes nothing),
// the rotation Rq of its unit quaternion (row-major) and its variances
// a = s^2.  Sigma = Rq diag(a) Rq^T is never formed entry by entry: for an
// elongated Gaussian its entries, rounded at the scale of the largest
// variance, lose the small ones.
struct __align__(16) GaussPrep {
  float p[3];
  float l2k;
  float rq[9];
  float a[3];
};
__device__ __forceinline__ bool gp_valid(const GaussPrep &g) { return g.l2k > -INFINITY; }

// c^2 = log2(e) / 2 and c: the base-2 exponent of a 2D Gaussian is
// l2A - c^2 d^T C d = l2A - |U d|^2 with U = c chol(C).
constexpr float kC2 = 0.72134752044448170f;
constexpr float kC = 0.84932180028801904f;

// Projected record of one (view, Gaussian), 32 B, read by the binning and
// the rasterisers as two float4:
//   a = (px, py, u11, u12)  centre (pixel coordinates), first row of U
//   b = (u22, l2A, rx, ry)  last entry of U, log2 amplitude, half extents
// U is the upper-triangular factor of the exponent's quadratic form,
// U^T U = (log2 e / 2) S^^-1.  The base-2 exponent of the 2D value at pixel
// (u, v) is
//   e = l2A - z1^2 - z2^2,  z1 = u11 dx + u12 dy,  z2 = u22 dy,
//   dx = u - px, dy = v - py,
// so value = 2^e; the pair is kept when e > log2(tau).  (z1, z2) are the
// whitened coordinates of the pixel: for a Gaussian a hundred times longer
// than wide they stay of order one where the entries of S^^-1 would cancel
// to three digits.  rx, ry bound the region where e > log2(tau) - margin.
// A record whose amplitude cannot exceed tau has rx = ry = -1 (no tile); an
// invalid record also has l2A = -inf and u11 = u12 = u22 = 0.
struct __align__(16) Rec {
  float4 a;
  float4 b;
};

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// 1.0f when a < b, else 0.0f (false for NaN operands).
__device__ __forceinline__ float set_lt(float a, float b) {
  float y;
  asm("set.lt.f32.f32 %0, %1, %2;" : "=f"(y) : "f"(a), "f"(b));
  return y;
}

// g when a < b, else +0 (also +0 for NaN operands): a compare that yields
// an all-ones or all-zeros word, and a bitwise and.
__device__ __forceinline__ float keep_or_zero(float g, float a, float b) {
  unsigned m;
  asm("set.lt.u32.f32 %0, %1, %2;" : "=r"(m) : "f"(a), "f"(b));
  return __uint_as_float(__float_as_uint(g) & m);
}

// Packed float32 pairs (sm_100 family): each component rounds exactly like
// the scalar operation, two components per issued instruction.
__device__ __forceinline__ float2 f2(float x) { return make_float2(x, x); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }

// Rotation matrix of a unit quaternion (w, x, y, z), entry formula.
__device__ __forceinline__ void quat_rot(float w, float x, float y, float z, float R[9]) {
  R[0] = 1.f - 2.f * (y * y + z * z);
  R[1] = 2.f * (x * y - w * z);
  R[2] = 2.f * (x * z + w * y);
  R[3] = 2.f * (x * y + w * z);
  R[4] = 1.f - 2.f * (x * x + z * z);
  R[5] = 2.f * (y * z - w * x);
  R[6] = 2.f * (x * z - w * y);
  R[7] = 2.f * (y * z + w * x);
  R[8] = 1.f - 2.f * (x * x + y * y);
}

// The 2D Gaussian of one Gaussian in one view, in pixel units (Eq. render).
// Both the forward preprocessing and the backward chain rule call this, so
// the two sides see bit-identical quantities.
struct View2D {
  float px, py;          // centre, pixel coordinates
  float sxx, sxy, syy;   // projected covariance S^, pixel^2
  float u11, u12, u22;   // U^T U = (log2 e / 2) S^^-1, U upper triangular
  float l2A;             // log2 amplitude
  float depth;           // z' (Angstrom)
  bool valid;
};

// S^ = W2 diag(a) W2^T with W2 the first two rows of W = R_b Rq: a sum of
// three rank-one terms, each entry accurate to its own size.  Its
// determinant comes from the Cauchy-Binet formula, det S^ = sum over column
// pairs (k, l) of a_k a_l m_kl^2, m_kl the 2x2 minors of W2: a sum of
// positive terms, accurate where det = sxx syy - sxy^2 would cancel (an
// elongated Gaussian seen side on).  U follows from S^ and det S^ alone:
//   u11 = c sqrt(syy / det),  u12 = -u11 sxy / syy,  u22 = c^2 / (u11 sqrt(det)).
__device__ __forceinline__ View2D view_project(const GaussPrep &g, const float *__restrict__ Rv,
                                               const float *__restrict__ tv, float apix, int d) {
  View2D o;
  // mean: p' = R p + (t, 0)
  float mx = Rv[0] * g.p[0] + Rv[1] * g.p[1] + Rv[2] * g.p[2] + tv[0];
  float my = Rv[3] * g.p[0] + Rv[4] * g.p[1] + Rv[5] * g.p[2] + tv[1];
  o.depth = Rv[6] * g.p[0] + Rv[7] * g.p[1] + Rv[8] * g.p[2];
  float inv = 1.f / apix;
  o.px = fmaf(mx, inv, 0.5f * d);
  o.py = fmaf(my, inv, 0.5f * d);
  const float *q = g.rq;
  float w0[3], w1[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    w0[k] = Rv[0] * q[k] + Rv[1] * q[3 + k] + Rv[2] * q[6 + k];
    w1[k] = Rv[3] * q[k] + Rv[4] * q[3 + k] + Rv[5] * q[6 + k];
  }
  const float a0 = g.a[0], a1 = g.a[1], a2 = g.a[2];
  // Angstrom^2
  float axx = a0 * w0[0] * w0[0] + a1 * w0[1] * w0[1] + a2 * w0[2] * w0[2];
  float axy = a0 * w0[0] * w1[0] + a1 * w0[1] * w1[1] + a2 * w0[2] * w1[2];
  float ayy = a0 * w1[0] * w1[0] + a1 * w1[1] * w1[1] + a2 * w1[2] * w1[2];
  const float m12 = fmaf(w0[1], w1[2], -w0[2] * w1[1]);
  const float m20 = fmaf(w0[2], w1[0], -w0[0] * w1[2]);
  const float m01 = fmaf(w0[0], w1[1], -w0[1] * w1[0]);
  float det = a1 * a2 * m12 * m12 + a0 * a2 * m20 * m20 + a0 * a1 * m01 * m01;  // Angstrom^4
  float inv2 = inv * inv;
  o.sxx = axx * inv2;
  o.sxy = axy * inv2;
  o.syy = ayy * inv2;
  float detp = det * inv2 * inv2;
  o.u11 = kC * sqrtf(o.syy / detp);
  o.u12 = -o.u11 * (o.sxy / o.syy);
  o.u22 = kC2 / (o.u11 * sqrtf(detp));
  o.l2A = g.l2k - 0.5f * log2f(det);
  o.valid = gp_valid(g) && det > 0.f && detp > 0.f && o.syy > 0.f && isfinite(det) &&
            isfinite(o.px) && isfinite(o.py) && isfinite(o.l2A) && o.u11 > 0.f &&
            o.u22 > 0.f && isfinite(o.u11) && isfinite(o.u12) && isfinite(o.u22);
  return o;
}

// Pixel range [lo, hi] covered by a centre c and half extent r inside
// [0, d-1]; false if empty.
__device__ __forceinline__ bool pixel_range(float c, float r, int d, int &lo, int &hi) {
  if (!(r >= 0.f)) return false;
  float l = fmaxf(ceilf(c - r), 0.f);
  float h = fminf(floorf(c + r), (float)(d - 1));
  if (!(l <= h)) return false;
  lo = (int)l;
  hi = (int)h;
  return true;
}

// ---- launchers (each returns cudaError_t of the launch) ------------------

// gem_prep.cu
// Shape constraints of the ablation study (Sec. 4, Design Choices): R_j = I,
// and S_j = s_j I with s_j the first scale entry.
constexpr int kNoRotation = 1;
constexpr int kIsotropic = 2;

// 15-bit 3D Morton key of every Gaussian's mean (cells of side / 32 over the
// box of that side centred on the origin).
cudaError_t launch_morton_key(const float *params, int64_t M, float side, uint16_t *key,
                              cudaStream_t st);
// slot_gauss: slot -> Gaussian (NULL: slot i is Gaussian i); gp is by slot.
// psort [M][11] (the parameters by slot) and gauss_slot [M] (Gaussian ->
// slot) are written unless psort is NULL.
cudaError_t launch_gauss_prep(const float *params, const uint32_t *slot_gauss, int64_t M,
                              int norm_mode, int shape, GaussPrep *gp, float *psort,
                              uint32_t *gauss_slot, cudaStream_t st);
cudaError_t launch_view_prep(const GaussPrep *gp, int64_t M, int B, const float *R,
                             const float *t, float apix, int d, float l2tau, float zrange,
                             Rec *rec, uint16_t *key, cudaStream_t st);
// Reads the float64 moments [B][M][6] and leaves them zero (the next
// backward pass accumulates into them).
// params (the slot-ordered copy), gp and the moments are by slot; grad
// comes out by Gaussian through gauss_slot (NULL: slot i is Gaussian i).
cudaError_t launch_prep_bwd(const float *params, const uint32_t *gauss_slot, const GaussPrep *gp,
                            int64_t M, int B, const float *R, const float *t, float apix, int d,
                            int norm_mode, int shape, double *mom, float *part, int nbg,
                            float *grad, cudaStream_t st);
cudaError_t launch_inspect_records(const Rec *rec, const GaussPrep *gp,
                                   const uint32_t *slot_gauss, int64_t M, int B, const float *R,
                                   const float *t, float apix, int d, float *out,
                                   cudaStream_t st);

// gem_query.cu
// Per-Gaussian quantities of the density query (48 B): centre, xy block of
// Sigma^-1 (1/Angstrom^2), Sigma_xz / Sigma_zz, Sigma_yz / Sigma_zz,
// 1 / Sigma_zz, log2 of the 3D amplitude, valid flag.
struct __align__(16) QueryPrep {
  float p[3];
  float pxx, pxy, pyy;
  float mx, my, hz;
  float l2A;
  float valid;
  float pdet;  // det of the xy block of Sigma^-1 (1/Angstrom^4), by Cauchy-Binet
};
cudaError_t launch_query_prep(const float *params, int64_t M, int norm_mode, int shape,
                              QueryPrep *qp, cudaStream_t st);
cudaError_t launch_slice_prep(const QueryPrep *qp, int64_t M, int k0, int nslice, float apix,
                              int d, float l2tau, Rec *rec, cudaStream_t st);

// gem_f64.cu (FP64 check mode)
struct G64 {
  double p[3], sig[6], lnk;
  bool valid;
};
struct V64 {
  double px, py, cxx, cxy, cyy, lnA;  // lnA = -inf: contributes nothing
};
cudaError_t launch_f64_project(const double *params, int64_t M, int B, const double *R,
                               const double *t, double apix, int d, int norm_mode, int shape,
                               double tau, G64 *gp, V64 *rec, double *proj, cudaStream_t st);
cudaError_t launch_f64_backward(const double *params, const G64 *gp, const V64 *rec, int64_t M,
                                int B, const double *R, const double *t, double apix, int d,
                                int norm_mode, int shape, double tau, const double *dproj,
                                double *mom, double *grad, cudaStream_t st);
cudaError_t launch_f64_widen(const float *x, double *y, int64_t n, cudaStream_t st);
cudaError_t launch_f64_narrow(const double *x, float *y, int64_t n, cudaStream_t st);
cudaError_t launch_f64_ctf_loss(int d, int B, double apix, const double *proj, const double *ctf,
                                const double *prm, const double *images, double *pred,
                                double *dproj, double *loss_img, double *loss, double2 *tw,
                                double *Hs, double2 *Za, double2 *Zb, double *r, double *li,
                                cudaStream_t st);

// gem_adam.cu
struct AdamArgs {
  float lr[4];  // centre, log scale, quaternion, log density
  float beta1, beta2, eps;
  float c1, c2;  // bias corrections 1 / (1 - beta^t)
};
cudaError_t launch_adam(const AdamArgs &a, int64_t M, float *raw, float *m, float *v,
                        const float *grad, float *params, const float *iso, cudaStream_t st);
cudaError_t launch_activate(int64_t M, const float *raw, float *params, cudaStream_t st);

// gem_knn.cu
struct KnnGrid {
  float lo[3];  // corner of the centres' bounding box
  float h, ih;  // cell side and its inverse
  int n[3];     // cells per axis
  int ncell;
};
struct KnnScratch {
  float *part;     // [nbb][6] partial boxes (nbb <= 608)
  KnnGrid *grid;
  int *cell;       // [M] cell of each centre
  int *cnt;        // [cap] members per cell
  int *start;      // [cap + 1] first member of each cell in order[]
  int *fill;       // [cap] scatter cursors
  int *order;      // [M] centres grouped by cell
  int *bsum;       // [knn_scan_blocks(cap) + 1]
  int64_t cap;     // most cells the grid may use
};
int knn_scan_blocks(int64_t cap);
cudaError_t launch_knn(const float *params, int64_t M, int k, const KnnScratch &s, float *dist,
                       int32_t *idx, cudaStream_t st);

// gem_bin.cu
struct BinScratch {
  uint16_t *key;           // [B][M] 16-bit depth keys (written by the preprocess)
  uint32_t *packed;        // [B][M] (high key byte << 24 | index) after the first pass
  uint32_t *perm;          // [B][M] Gaussian indices in depth order
  uint32_t *dcnt;          // [B][nchD][256]
  uint32_t *tcnt;          // [B][nchT][T] per chunk: hits per tile, then offsets
  int64_t *tile_start;     // [B*T + 1]
  uint2 *list;             // [cap] entries: x = Gaussian index, y = 4x4-block mask (16 bits)
  uint64_t *hits;          // [cap] (slot in chunk, tile, 4x4-block mask) of every hit,
                           // grouped by chunk (written by the count pass)
  int64_t *chunk_base;     // [B][nchT] where a chunk's hits start in hits[]
  uint32_t *chunk_n;       // [B][nchT] how many hits the chunk has
  unsigned long long *hit_ctr;  // [1] hits[] allocation cursor
  int64_t cap;
  int *status;
};
// Stable sort of 16-bit keys [B][M] per row (two 8-bit counting passes,
// ties in index order): perm[b][r] = index of rank r.  dcnt and packed are
// scratch of the binning's sizes.
cudaError_t launch_sort16(const uint16_t *key, int64_t M, int B, uint32_t *dcnt,
                          uint32_t *packed, uint32_t *perm, cudaStream_t st);
// Gaussian of each list entry: out[i] = slot_gauss[list[i].x] (the entries
// hold slots), or list[i].x when slot_gauss is NULL.
cudaError_t launch_map_slots(const uint2 *list, const uint32_t *slot_gauss, int64_t n,
                             uint32_t *out, cudaStream_t st);
// Returns the permutation used for binning in *perm_out (NULL: index order).
cudaError_t launch_bin(const Rec *rec, const uint16_t *key, int64_t M, int B, int d,
                       float l2tau, int zsort, BinScratch &s, const uint32_t **perm_out,
                       cudaStream_t st);
size_t bin_chunks_depth(int64_t M);
size_t bin_chunks_tiles(int64_t M);
cudaError_t bin_configure(int d);

// gem_raster.cu
// A configuration of the forward rasteriser: form 0 = equal runs across
// blocks, 1 = block-aligned runs; sub = 128-record sub-windows per window;
// minb = CTAs per SM the launch bound asks for; persistent = a grid of
// minb CTAs per SM pulling tiles longest-first from a counter.
struct FwdCfg {
  int form, sub, minb, persistent;
  int ctas;  // persistent grid: CTAs per SM (at most minb, the kernel's bound)
  const char *name;
};
int fwd_config_count();
const FwdCfg &fwd_config(int i);
// order [B*T] and next_tile [1] are scratch of the persistent forms.
cudaError_t launch_raster_fwd(int cfg, const Rec *rec, const uint2 *list,
                              const int64_t *tile_start, int64_t cap, int64_t M, int B, int d,
                              float l2tau, float *proj, uint32_t *order, unsigned *next_tile,
                              cudaStream_t st);
// A configuration of the backward rasteriser: lanes sharing one record,
// records per lane per warp window, persistent grid (tiles longest-first
// from a counter; order [B*T] and next_tile [1] are its scratch).
struct BwdCfg {
  int lanes, per, persistent;
  int ctas;  // persistent grid: CTAs per SM (fewer tiles in flight keep more of
             // their records and moments in L2)
  const char *name;
};
int bwd_config_count();
const BwdCfg &bwd_config(int i);
// order_ready: `order` already holds the longest-first order of these bins
// (a persistent forward computed it); the persistent forms then only reset
// their counter.
cudaError_t launch_raster_bwd(int cfg, const Rec *rec, const uint2 *list,
                              const int64_t *tile_start, int64_t cap, int64_t M, int B, int d,
                              float l2tau, const float *dproj, double *mom, uint32_t *order,
                              unsigned *next_tile, bool order_ready, cudaStream_t st);
cudaError_t launch_count_kept(int cfg, const Rec *rec, const uint2 *list,
                              const int64_t *tile_start, int64_t cap,
                              int64_t M, int B, int d, float l2tau, unsigned long long *kept,
                              uint32_t *order, unsigned *next_tile, cudaStream_t st);
cudaError_t launch_dense_fwd(const Rec *rec, int64_t M, int B, int d, float l2tau, float *proj,
                             cudaStream_t st);
cudaError_t launch_dense_bwd(const Rec *rec, int64_t M, int B, int d, float l2tau,
                             const float *dproj, double *mom, cudaStream_t st);

// gem_ctf.cu
// Radix sequence of an n-point FFT, 2 bits per stage (0: radix 2,
// 1: radix 3, 2: radix 4), first stage in the low bits.
struct FftPlan {
  int n;
  int nst;
  unsigned code;
};
bool fft_plan(int n, FftPlan &p);
cudaError_t ctf_configure(int d);
size_t ctf_partials(int d);
// gem_fsc.cu
cudaError_t fsc_configure(int d);
int fsc_partial_count(int d);  // doubles of block partial sums
cudaError_t launch_fsc(int d, float apix, float thr, const FftPlan &plan, const float2 *tw,
                       const float *X1, const float *X2, float2 *P, float2 *Q, double *part,
                       double *fsc, double *sums, double *resolution, cudaStream_t st);

cudaError_t launch_ctf_loss(int d, int B, float apix, const FftPlan &plan, const float2 *tw,
                            const float *proj, const float *ctf, const float *ctf_params,
                            const float *images, float2 *Z, double *lossp, float *pred,
                            float *dproj, double *loss_img, double *loss, cudaStream_t st);

}  // namespace gem
