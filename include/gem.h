/*
 * gem.h -- C ABI of the GB300 (sm_103a) library for the GEM hot path.
 *
 * GEM (arXiv 2509.25075) writes a protein density as M anisotropic 3D
 * Gaussians (11 values each, Sec. 3.2, Eq. G), projects them in closed form
 * to particle images (Eq. render), keeps only terms above a threshold tau
 * (Eq. accu), accumulates each pixel's terms from the lowest depth to the
 * highest (Sec. 3.2, after Eq. accu), applies the CTF in Fourier space and
 * scores the result with an L2 loss (Eq. loss), and back-propagates only
 * through the (pixel, Gaussian) pairs that were kept (Sec. 1 (iii), Sec. 3.2
 * "Efficient Gradient Computation").  Poses and CTFs are known inputs
 * (Eq. recon).
 *
 * Conventions shared by every call
 *   - Every array pointer is a DEVICE pointer owned by the caller, unless a
 *     comment says otherwise.  The library never frees caller memory.  It
 *     allocates its own scratch once, in gem_create, and frees it in
 *     gem_destroy.
 *   - Every call is asynchronous on the context's CUDA stream and does no
 *     host synchronisation, except gem_status and gem_inspect_* (which
 *     synchronise that stream).
 *   - Return value: GEM_OK (0) or a negative GEM_E* code.  The message of
 *     the last failure is available from gem_last_error.  A failed call
 *     launches nothing.  No C++ exception crosses this interface.
 *   - Device-side conditions (a list that overflowed its capacity) are
 *     recorded in a status word that gem_status reads; they do not fault.
 *   - Floating point is float32 (IEEE, row-major, contiguous) unless stated;
 *     losses are float64.  Image arrays ([B][d][d]) must be 16-byte aligned.
 *   - Image b, row v, column u is element [b][v][u] of a [B][d][d] array;
 *     its centre sits at ((u - d/2) apix, (v - d/2) apix) Angstrom.
 *   - Gaussian j is row j of a [M][11] array: p (3, Angstrom), s (3, the
 *     diagonal of S in Eq. G, Angstrom), q (4, rotation quaternion w x y z,
 *     normalised by the library), rho (1).  A Gaussian with a zero
 *     quaternion, a non-positive rho, a singular projected covariance or a
 *     non-finite value contributes nothing and receives a zero gradient.
 *   - View b: R [B][3][3] row-major rotation, t [B][2] Angstrom; camera
 *     coordinates are x' = R x + (t, 0) and the beam runs along z'.
 *   - A context is not thread-safe; use one per stream.
 */
#ifndef GEM_H
#define GEM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GEM_OK 0
#define GEM_EINVAL (-1)    /* bad argument (null pointer, size out of range, bad config) */
#define GEM_ENOMEM (-2)    /* device allocation failed in gem_create                      */
#define GEM_ECUDA (-3)     /* a CUDA runtime call or kernel launch failed                 */
#define GEM_ESTATE (-4)    /* call order violated (backward before forward, ...)          */
#define GEM_ECAPACITY (-5) /* returned by gem_status: the pair list overflowed max_pairs  */
#define GEM_ETIMEOUT (-6)  /* reserved: a device-side wait ran out.  No kernel of this    */
                           /* library waits on another (work is claimed from counters    */
                           /* that never block), so no call returns it today.            */

/* Device status bits reported by gem_status. */
#define GEM_STATUS_CAPACITY 1

typedef struct gem_ctx gem_ctx;

typedef struct gem_config {
  int32_t d;         /* image side in pixels: a multiple of 16, 16..768, of the form 2^a 3^b  */
  float apix;        /* pixel size in Angstrom, > 0                                          */
  float tau;         /* threshold of Eq. accu on the 2D value, >= 0 (0: every pair counts)   */
  int32_t norm_mode; /* 0: amplitude of Eq. render, rho / (2 pi |S^|^1/2) (rho is a mass);    */
                     /* 1: exact line integral of Eq. G, rho (2 pi)^1/2 (|Sigma|/|S^|)^1/2    */
  int32_t max_B;     /* largest batch any call will pass, >= 1                                */
  int64_t max_M;     /* largest Gaussian count any call will pass, 1..2^24                    */
  int64_t max_pairs; /* capacity of the (image, tile, Gaussian) lists; 0 picks 16*max_B*max_M */
  int32_t zsort;     /* 1: accumulate each pixel from the lowest depth z' to the highest      */
                     /*    (Sec. 3.2); 0: in slot order (see gem_project).  Changes        */
                     /*    rounding only.                                                  */
  int32_t no_rotation; /* 1: every Gaussian uses R_j = I and q is ignored (its gradient is 0); */
                       /*    the "No Rotation" ablation of Sec. 4 (Design Choices, Table 4)  */
  int32_t isotropic;   /* 1: S_j = s_j I with s_j = the first scale entry; the other two are   */
                       /*    ignored and get zero gradient ("Isotropic Scaling", same table;   */
                       /*    the paper sets s_j to the nearest-neighbour distance, which       */
                       /*    gem_nn_distance computes)                                         */
  int32_t tile;        /* side of the square pixel tiles the Gaussians are binned into: 16    */
                       /*    (0 selects it; the rasterisers are built for 16 x 16 tiles of     */
                       /*    4 x 4-pixel blocks, so any other value is GEM_EINVAL)             */
  int32_t fp64_check;  /* 1: gem_forward and gem_backward compute in float64 (the FP64 check  */
                       /*    mode below, on the same float arrays: inputs widened, pred and   */
                       /*    grad rounded back to float, the loss a float64); 0: float32 path */
} gem_config;

/* Fill *cfg with defaults: tau = 0, norm_mode 0, zsort 1, max_pairs 0, no ablation,
 * tile 16, fp64_check 0. */
int gem_config_default(gem_config *cfg, int32_t d, float apix, int32_t max_B, int64_t max_M);

/* Create a context.  cuda_stream is a cudaStream_t (NULL: the legacy default
 * stream).  Allocates all scratch on the current device: about
 * 32 B x max_B x max_M (projected records) + 48 B x max_B x max_M (moments)
 * + 16 B x max_pairs (list entries with their block masks, and the
 * binning's hit records) + 20 B x max_B x d^2 (images, spectra) and
 * a few small tables.  Errors: GEM_EINVAL, GEM_ENOMEM, GEM_ECUDA. */
int gem_create(gem_ctx **out, const gem_config *cfg, void *cuda_stream);

/* Message of the last gem_create that failed on this thread ("" after a success). */
const char *gem_create_error(void);

/* Free every allocation of the context (synchronises its stream).  NULL is allowed. */
int gem_destroy(gem_ctx *ctx);

/* Message of the last failure on this context ("" if none); valid until the next call. */
const char *gem_last_error(const gem_ctx *ctx);

/* Change the stream later calls use. */
int gem_set_stream(gem_ctx *ctx, void *cuda_stream);

/* Synchronise the context's stream and return GEM_OK, GEM_ECAPACITY (a
 * projection since the last read needed more than max_pairs list entries:
 * its lists are incomplete, so the rasterisers treat every list of that
 * call as empty, and its projection, and a backward of it, come out zero)
 * or GEM_ECUDA.  Clears the status word. */
int gem_status(gem_ctx *ctx);

/* ---- steps of the hot path -------------------------------------------- */

/* Steps a1-a3: Eq. render with Eq. accu.
 *   params [M][11], R [B][3][3], t [B][2]  ->  proj [B][d][d].
 * Preprocesses every (view, Gaussian), bins the kept pairs into 16 x 16
 * pixel tiles (each tile's Gaussians in ascending depth when zsort = 1) and
 * rasterises.  Internally the Gaussians are held in slot order, a stable
 * sort by the 3D Morton key of their means (5 bits per axis over the box of
 * side d apix centred on the origin), so that Gaussians close in space are
 * close in memory; Gaussians with equal 16-bit depth keys accumulate in
 * slot order.  Every output is in the caller's Gaussian order.  The context
 * keeps the bins and the pointers params, R, t for gem_project_backward:
 * they must stay valid and unchanged until then.
 * Errors: GEM_EINVAL (M < 1 or > max_M, B < 1 or > max_B, null pointer). */
int gem_project(gem_ctx *ctx, const float *params, int64_t M, int32_t B, const float *R,
                const float *t, float *proj);

/* Step a4: Eq. loss and its adjoint, for B images.
 *   proj [B][d][d], images [B][d][d], and exactly one of
 *     ctf        [B][d][d/2+1]  real transfer function on the rfft grid
 *                               [ky][kx]; where H(k) and H(-k mod d) differ
 *                               (columns kx = 0 and d/2) their mean is used,
 *     ctf_params [B][8]         defocus U (A), defocus V (A), astigmatism
 *                               angle (rad), voltage (kV), Cs (mm), amplitude
 *                               contrast, phase shift (rad), B-factor (A^2):
 *                               H = -(sqrt(1-w^2) sin chi + w cos chi)
 *                                   exp(-B k^2 / 4),
 *                               chi = pi lambda dF(angle) k^2
 *                                     - pi/2 Cs lambda^3 k^4 + phase.
 *   pred    = F^-1(H . F(proj))              [B][d][d]   (may be NULL)
 *   dproj   = dL/dproj = F^-1(H . F(2 r / (B d^2))), r = pred - images
 *                                            [B][d][d]   (may be NULL)
 *   loss_img[b] = (1/d^2) sum_pixels r^2     [B] float64 (may be NULL)
 *   loss    = (1/B) sum_b loss_img[b]        [1] float64 (may be NULL)
 * Circular convolution, no padding; forward DFT unnormalised, inverse 1/d^2.
 * Errors: GEM_EINVAL (both or neither CTF form, B out of range, null input). */
int gem_ctf_loss(gem_ctx *ctx, int32_t B, const float *proj, const float *ctf,
                 const float *ctf_params, const float *images, float *pred, float *dproj,
                 double *loss_img, double *loss);

/* Steps a5-a6: gradient of the loss with respect to all 11 M parameters,
 * given dproj = dL/dproj [B][d][d] for the projection of the last
 * gem_project (same params, R, t, M, B).  Only the pairs kept by Eq. accu
 * contribute.  grad [M][11] is overwritten.
 * Errors: GEM_ESTATE (no projection yet), GEM_EINVAL. */
int gem_project_backward(gem_ctx *ctx, const float *dproj, float *grad);

/* The Gaussians of the density representation (Eq. recon: the unknown the
 * images are fitted to), [M][11] device float32, caller-owned.  The context
 * keeps the pointer and M (no copy): gem_forward with params = NULL uses
 * them, so they must stay valid and unchanged until that forward's
 * gem_backward has been enqueued.  Errors: GEM_EINVAL (NULL, M outside
 * 1..max_M). */
int gem_set_gaussians(gem_ctx *ctx, const float *params, int64_t M);

/* a1-a4 in one call: gem_project into the context's own image buffer, then
 * gem_ctf_loss with the adjoint kept inside the context for gem_backward.
 * params = NULL: the Gaussians of the last gem_set_gaussians (M is then
 * ignored; GEM_ESTATE if none were set).  pred may be NULL; loss is a device
 * float64 [1].  With fp64_check the whole step runs in float64 (see the
 * config field). */
int gem_forward(gem_ctx *ctx, const float *params, int64_t M, int32_t B, const float *R,
                const float *t, const float *ctf, const float *ctf_params, const float *images,
                float *pred, double *loss);

/* a5-a6 for the last gem_forward: grad [M][11] = dL/dparams.
 * Errors: GEM_ESTATE (no gem_forward since the last projection). */
int gem_backward(gem_ctx *ctx, float *grad);

/* ---- plain dense forms (no tiles, no binning, no ordering) -------------- */

/* Same result as gem_project, computed by one thread per pixel over all M
 * Gaussians.  Keeps the same state for gem_project_backward_dense (no tile
 * lists: gem_project_backward after it returns GEM_ESTATE). */
int gem_project_dense(gem_ctx *ctx, const float *params, int64_t M, int32_t B, const float *R,
                      const float *t, float *proj);

/* Same result as gem_project_backward, computed by one thread per
 * (view, Gaussian) over all d^2 pixels. */
int gem_project_backward_dense(gem_ctx *ctx, const float *dproj, float *grad);

/* ---- inspection (synchronise the stream) ------------------------------- */

/* Number of (image, tile, Gaussian) entries the last binning listed: that of
 * the last gem_project, or of the last slice batch of gem_query.  The
 * inspection and pair-statistics calls below read the same lists.
 * GEM_ESTATE when there are none. */
int gem_pair_count(gem_ctx *ctx, int64_t *n_pairs);

/* Copy the bins of the last gem_project into caller device memory:
 *   tile_start [B*T + 1] int64: entries of tile t of image b are
 *              list[tile_start[b*T + t] .. tile_start[b*T + t + 1]),
 *              T = (d/16)^2, tiles numbered row-major;
 *   list       [list_cap] uint32 Gaussian indices, in accumulation order.
 * Errors: GEM_ESTATE, GEM_EINVAL (list_cap smaller than the pair count). */
int gem_inspect_bins(gem_ctx *ctx, int64_t *tile_start, uint32_t *list, int64_t list_cap);

/* Copy the projected records of the last gem_project, [B][M][8] float32:
 * centre x, centre y (pixel coordinates: pixel u sits at x = u),
 * conic xx, conic xy, conic yy (inverse projected covariance, pixel units),
 * log2 of the 2D amplitude, depth z' (Angstrom), valid flag (1 or 0). */
int gem_inspect_records(gem_ctx *ctx, float *out);

/* Pair statistics of the last binning (see gem_pair_count), counted by a
 * separate pass over the bins (not part of the hot path; synchronises the
 * stream):
 *   kept      (pixel, Gaussian) pairs with value > tau (Eq. accu),
 *   evaluated pairs the tiled forward rasteriser evaluates to find them
 *             (may be NULL). */
int gem_pair_stats(gem_ctx *ctx, int64_t *kept, int64_t *evaluated);

/* ---- beyond the training step ---------------------------------------------- */

/* Density query (Eq. query, Fig. query): the density of the Gaussians on the
 * context's d x d x d voxel grid,
 *   V(x) = sum_j [G_j(x) > tau] G_j(x),
 *   G_j(x) = A_j exp(-1/2 (x - p_j)^T Sigma_j^-1 (x - p_j))   (Eq. G),
 * with A_j = rho_j in norm_mode 1 (rho a peak density, Eq. G as printed) and
 * A_j = rho_j / ((2 pi)^3/2 |Sigma_j|^1/2) in norm_mode 0 (rho a mass: the
 * density whose line integral is Eq. render).  The ablation flags apply.
 *   params  device [M][11], M <= max_M (caller-owned);
 *   tau     threshold on the 3D value (>= 0; 0 keeps every pair);
 *   vol     device float [d][d][d], written in full: vol[z][y][x] is the
 *           voxel centred at ((x - d/2) apix, (y - d/2) apix, (z - d/2) apix) A;
 *           16-byte aligned.
 * Gaussians with a zero scale, a zero quaternion (unless no_rotation) or
 * rho <= 0 contribute nothing.  Slices run in batches of max_B through the
 * projection scratch, so the call ends the state kept for gem_backward
 * (a later gem_backward returns GEM_ESTATE).  Pair lists that overflow
 * max_pairs are reported by gem_status (GEM_ECAPACITY).  Asynchronous.
 * Errors: GEM_EINVAL, GEM_ECUDA. */
int gem_query(gem_ctx *ctx, const float *params, int64_t M, float tau, float *vol);

/* Fourier shell correlation of two maps (Eq. fsc; Sec. 4, Gold-Standard
 * Fourier Shell Correlation) on the context's d x d x d grid:
 *   FSC(i) = Re sum_{k in shell i} F1(k) F2(k)^* / sqrt(sum |F1|^2 . sum |F2|^2),
 * F1, F2 the 3D DFTs of the maps, shell i = the frequencies whose signed
 * DFT indices k have round(|k|) = i, i = 0 .. d/2 (the corners beyond the
 * Nyquist sphere are not used).  Shell i is the resolution d apix / i A.
 *   map1, map2  device float [d][d][d] (e.g. two gem_query outputs);
 *   threshold   the FSC level whose crossing sets the resolution (0.143 in
 *               the paper), in (-1, 1);
 *   fsc         device double [d/2 + 1];
 *   sums        device double [3][d/2 + 1] or NULL: per shell the numerator
 *               and the two power sums;
 *   resolution  device double [1] or NULL: d apix / k*, k* the first
 *               crossing below the threshold (first shell i >= 1 with
 *               FSC < threshold, interpolated linearly from shell i - 1);
 *               2 apix (Nyquist) when the curve never crosses.
 * A shell without power has FSC 0.  The first call allocates 16 d^3 bytes
 * of scratch that the context keeps.  Asynchronous.  The sums are reduced
 * in double with shared-memory atomics: not bitwise repeatable, ~1e-15.
 * Errors: GEM_EINVAL, GEM_ENOMEM, GEM_ECUDA. */
int gem_fsc(gem_ctx *ctx, const float *map1, const float *map2, float threshold, double *fsc,
            double *sums, double *resolution);

/* k nearest neighbours of the Gaussian centres (Sec. 4, Design Choices of
 * 3DGS for cryo-EM: the isotropic-scaling ablation takes s_j = the distance
 * of Gaussian j to its nearest neighbour; also a scale initialisation).
 *   params  device [M][11] (only the centre p, Angstrom, is read), M <= max_M;
 *   k       1..16;
 *   dist    device float [M][k]: the k smallest Euclidean distances from
 *           p_j to the other centres, ascending (INFINITY where fewer than
 *           k others exist, or where p_j is not finite);
 *   idx     device int32 [M][k] or NULL: the neighbours' indices, -1 with
 *           INFINITY.  Among equal distances the smaller index comes first.
 * Exact (every centre that can be among the k nearest is examined); the
 * squared distances are float32 sums of squared float32 differences,
 * rounded in this order.  Centres that are not finite are never neighbours.
 * Asynchronous on the context's stream; uses the context's grid scratch (it
 * does not disturb the state kept for gem_backward).  Errors: GEM_EINVAL
 * (M or k out of range, NULL pointers), GEM_ECUDA. */
int gem_nn_distance(gem_ctx *ctx, const float *params, int64_t M, int32_t k, float *dist,
                    int32_t *idx);

/* ---- FP64 check mode --------------------------------------------------------- */

/* Steps a1-a6 in double precision by the plain dense forms: every pixel
 * against every Gaussian with exp() in double, explicit separable DFTs for
 * the CTF, the same moments and chain rule as the float path.  For checking
 * the method's arithmetic (agreement with an FP64 reference to ~1e-12), not
 * for speed: the cost is B d^2 M exponentials per projection and again per
 * backward, and O(d^3) per image for the CTF.  The context's d, apix, tau,
 * norm_mode and ablation flags apply; all arrays are double, on the device,
 * caller-owned, with the layouts of the float calls; as for gem_project,
 * params, R and t of gem_project_f64 are read again by
 * gem_project_backward_f64 and must stay valid and unchanged until then.
 * The first call
 * allocates about (80 max_B max_M + 48 max_B d^2) bytes of scratch that the
 * context keeps.  Asynchronous.  Errors: GEM_EINVAL, GEM_ENOMEM, GEM_ECUDA,
 * GEM_ESTATE (backward without a projection). */
int gem_project_f64(gem_ctx *ctx, const double *params, int64_t M, int32_t B, const double *R,
                    const double *t, double *proj);
int gem_ctf_loss_f64(gem_ctx *ctx, int32_t B, const double *proj, const double *ctf,
                     const double *ctf_params, const double *images, double *pred,
                     double *dproj, double *loss_img, double *loss);
int gem_project_backward_f64(gem_ctx *ctx, const double *dproj, double *grad);

/* ---- training loop: optimiser step ------------------------------------------ */

/* The paper optimises the Gaussians against the images (Sec. 3.2,
 * "Optimizing 3D GS representations") without naming the optimiser or the
 * parameter activations; these follow 3DGS practice.  Parameters are kept
 * unconstrained ("raw"): raw = (p, log s, q, log rho); the model parameters
 * the projection takes are params = (p, exp(log s), q, exp(log rho)) (the
 * quaternion is normalised by the projection). */
typedef struct gem_adam_config {
  float lr[4];   /* learning rates: centre (A), log scale, quaternion, log density */
  float beta1;   /* first-moment decay, in [0, 1)  (0.9)                           */
  float beta2;   /* second-moment decay, in [0, 1) (0.999)                         */
  float eps;     /* added to sqrt(v^), > 0          (1e-15 in 3DGS; 1e-8 typical)   */
  int32_t step;  /* 1 on the first step: bias corrections 1 / (1 - beta^step)        */
} gem_adam_config;

/* One Adam step on raw [M][11] from grad = dL/dparams [M][11] (the output of
 * gem_backward), chain rule through the activations included:
 *   g_raw = grad (centre, quaternion),  grad * s (log s),  grad * rho (log rho)
 *   m = b1 m + (1 - b1) g,  v = b2 v + (1 - b2) g^2,
 *   raw -= lr_group * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps),
 * then params = activation(raw).  Non-finite gradient entries count as 0.
 *   raw, m, v, params  device float [M][11] (m, v start at 0), updated;
 *   iso_scale          device float [M] or NULL: when given, the three scale
 *                      entries of Gaussian j are set to iso_scale[j] (raw to
 *                      its log) and not learnt: the isotropic-scaling ablation
 *                      with s_j = the nearest-neighbour distance
 *                      (gem_nn_distance), recomputed by the caller each step.
 * Asynchronous.  Errors: GEM_EINVAL (M, pointers, hyper-parameters), GEM_ECUDA. */
int gem_adam_step(gem_ctx *ctx, int64_t M, const gem_adam_config *cfg, float *raw, float *m,
                  float *v, const float *grad, float *params, const float *iso_scale);

/* params [M][11] = activation(raw [M][11]) (device arrays).  Asynchronous. */
int gem_activate(gem_ctx *ctx, int64_t M, const float *raw, float *params);

/* ---- allocation-free variant ---------------------------------------------- */

/* Step a4 (gem_ctf_loss) for callers that cannot allocate device memory at
 * the point of the call: code running under a fixed memory budget, behind an
 * allocator that forbids cudaMalloc after start-up, or where a device
 * allocation's implicit synchronisation is not allowed.  No context and no
 * allocation: the scratch (spectrum and loss partials) lives in file-scope
 * device arrays of fixed size that every GPU loading the library holds until
 * the process exits.  The paper has no counterpart; this is plumbing.
 *   d, apix      image side and pixel size, the same rules as gem_config;
 *   B, proj, ctf, ctf_params, images, pred, dproj, loss_img, loss
 *                exactly as for gem_ctf_loss (caller-owned device memory);
 *   cuda_stream  cudaStream_t to run on (NULL: the legacy default stream).
 * Limits: B * d * d <= 1,048,576 and B * (P + 1) <= 65,536, P the loss
 * partials per image (d / 16 or d / 8, so the first limit implies the
 * second); beyond them the call returns GEM_ECAPACITY and launches nothing.  Other bad
 * arguments return GEM_EINVAL; CUDA failures GEM_ECUDA.
 * The first call on each device looks up the arrays' device addresses
 * (cudaGetSymbolAddress) and keeps them for the life of the process; make
 * that first call before any stream capture, and do not use the entry point
 * across a cudaDeviceReset (or any re-creation of the device's primary
 * context), after which the arrays may sit at other addresses.
 * A CUDA error already pending when the call starts (from the caller's own
 * earlier work) is reported as GEM_ECUDA and left pending, not cleared.
 * Every call on a device shares the same arrays, which keep the last call's
 * contents (every call rewrites what it reads); calls that overlap on the
 * GPU (different streams, no ordering between them) race on them. */
int gem_ctf_loss_static(int32_t d, float apix, int32_t B, const float *proj, const float *ctf,
                        const float *ctf_params, const float *images, float *pred,
                        float *dproj, double *loss_img, double *loss, void *cuda_stream);

/* ---- rasteriser configurations and the autotuner ----------------------- */

/* Both rasterisers come in several kernel configurations that compute the
 * same result (bitwise, for a given configuration; within float rounding
 * across configurations): the forward (step a3) as equal runs of items
 * across blocks or runs aligned to blocks, at 8 or 9 CTAs per SM, on a
 * per-tile grid or a persistent grid (5 to 9 CTAs per SM) that takes tiles
 * longest-first from a counter; the backward (a5) with 1 or 2 lanes per record, on either grid,
 * and with warp windows of 64, 128 or 256 records and 5 to 8 CTAs per SM
 * on the persistent grid.
 * Which is
 * fastest depends on the image side, the batch and the Gaussians' sizes.
 * Counts of each kind (kind 0: forward, 1: backward); a configuration's
 * description ("" if out of range). */
int gem_raster_config_count(int32_t *n_fwd, int32_t *n_bwd);
const char *gem_raster_config_name(int32_t kind, int32_t i);

/* Use configurations fwd, bwd (indices; -1 for either: the autotuner's
 * choice for the call's shape, else the library default).  Errors:
 * GEM_EINVAL (index out of range). */
int gem_set_raster_config(gem_ctx *ctx, int32_t fwd, int32_t bwd);

/* The configurations a call with B images and M Gaussians would use. */
int gem_get_raster_config(const gem_ctx *ctx, int32_t B, int64_t M, int32_t *fwd, int32_t *bwd);

/* Autotuner: project params, R, t (as gem_project) once, then time every
 * forward configuration and every backward configuration reps times each
 * (after one warm-up launch) on these bins with CUDA events, and record the
 * fastest of each for this shape (device, d, B, bit length of M) in a
 * process-wide table that every context consults when its configuration is
 * -1 (the default).  Writes the choices to *fwd, *bwd (either may be NULL).
 * Synchronises the stream (not capturable); the first call allocates
 * max_M x 11 floats of scratch that the context keeps; ends the state kept
 * for gem_backward.  Errors: as gem_project, GEM_ENOMEM, GEM_ECUDA. */
int gem_autotune(gem_ctx *ctx, const float *params, int64_t M, int32_t B, const float *R,
                 const float *t, int32_t reps, int32_t *fwd, int32_t *bwd);

/* ---- per-stage timing ---------------------------------------------------- */

/* Stages of the hot path, as timed by gem_timing_read. */
#define GEM_STAGE_PREP 0       /* a1: per-Gaussian and per-(view, Gaussian) preprocess   */
#define GEM_STAGE_BIN 1        /* a2: depth sort and tile binning                         */
#define GEM_STAGE_RASTER_FWD 2 /* a3: raster forward (or the dense forward)               */
#define GEM_STAGE_CTF 3        /* a4: CTF, loss and adjoint                               */
#define GEM_STAGE_RASTER_BWD 4 /* a5: moment clear + raster backward (or dense backward)  */
#define GEM_STAGE_PREP_BWD 5   /* a6: chain rule to the 11 parameters, sum over views     */
#define GEM_NSTAGES 6

/* enable != 0: from now on record CUDA events on the context's stream around
 * each stage and count the library's kernel launches per stage.  Resets the
 * counters.  Timing does not change any result. */
int gem_timing(gem_ctx *ctx, int enable);

/* Synchronise the stream; write each stage's device time (ms, the last time
 * it ran since the previous read; 0 if it did not run) to ms[GEM_NSTAGES]
 * and the number of kernels the library launched per stage since the
 * previous read to launches[GEM_NSTAGES] (either may be NULL).  Resets. */
int gem_timing_read(gem_ctx *ctx, float *ms, int64_t *launches);

#ifdef __cplusplus
}
#endif

#endif /* GEM_H */
