// C ABI of the GEM hot-path library (declared in include/gem.h).
//
// The context owns every scratch buffer (allocated once at creation, sized
// by max_B, max_M, d and max_pairs) and records what the last projection
// left behind for the backward pass.  Calls validate their arguments, then
// enqueue kernels on the context's stream without synchronising.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "gem.h"
#include "gem_internal.cuh"

using namespace gem;

struct gem_ctx {
  gem_config cfg;
  cudaStream_t stream = nullptr;
  char err[512] = {0};
  int T = 0;
  float l2tau = 0.f;
  FftPlan plan{};
  // scratch
  GaussPrep *gp = nullptr;       // [max_M] by slot
  Rec *rec = nullptr;            // [max_B][max_M] by view, slot
  uint32_t *slot_gauss = nullptr;  // [max_M] Gaussian of each slot (3D Morton order)
  uint32_t *gauss_slot = nullptr;  // [max_M] slot of each Gaussian
  float *psort = nullptr;          // [max_M][11] parameters by slot
  uint16_t *mkey = nullptr;        // [max_M] Morton keys

  BinScratch bin{};
  double *mom = nullptr;   // [max_B][max_M][6] moments of the raster backward
  bool mom_clean = false;  // every moment is zero (prep_bwd leaves them so)
  float *part = nullptr;
  int nbg = 1;
  float *proj = nullptr;   // internal projection of gem_forward
  float *dproj = nullptr;  // internal adjoint of gem_forward
  float2 *Z = nullptr;
  float2 *tw = nullptr;
  double *lossp = nullptr;
  int *status = nullptr;
  unsigned long long *kept = nullptr;
  KnnScratch knn{};
  QueryPrep *qp = nullptr;
  // FSC scratch, allocated by the first gem_fsc: two d^3 complex volumes
  float2 *fscP = nullptr, *fscQ = nullptr;
  double *fsc_part = nullptr;
  // FP64 check mode scratch, allocated by the first *_f64 call
  struct {
    G64 *gp = nullptr;
    V64 *rec = nullptr;
    double *mom = nullptr;
    double2 *tw = nullptr, *Za = nullptr, *Zb = nullptr;
    double *Hs = nullptr, *r = nullptr, *li = nullptr;
    bool have = false;  // a projection to differentiate
    const double *params = nullptr, *R = nullptr, *t = nullptr;
    int64_t M = 0;
    int B = 0;
    // fp64_check contexts: float inputs of gem_forward widened, and the
    // step's float64 intermediates (allocated by gem_create)
    double *params_in = nullptr, *R_in = nullptr, *t_in = nullptr, *images_in = nullptr;
    double *ctf_in = nullptr, *proj = nullptr, *pred = nullptr, *dproj = nullptr, *grad = nullptr;
    bool have_dproj = false;
  } f64;
  // Gaussians given by gem_set_gaussians (used by gem_forward with params = NULL)
  const float *set_params = nullptr;
  int64_t set_M = 0;
  // rasteriser kernel configurations (indices into the tables of
  // gem_raster.cu); -1: the autotuner's cached choice for the call's shape,
  // else the default
  int fwd_cfg = -1, bwd_cfg = -1;
  uint32_t *order = nullptr;     // [max_B * T] tile order of the persistent forward
  unsigned *next_tile = nullptr;  // [2] work counters of the persistent forward, backward
  float *tune_grad = nullptr;     // [max_M][11] gradient the autotuner's backward writes
  std::vector<void *> allocs;
  // per-stage timing (events recorded around each stage when enabled)
  bool timing = false;
  cudaEvent_t ev[GEM_NSTAGES][2] = {};
  bool recorded[GEM_NSTAGES] = {};
  int64_t launches[GEM_NSTAGES] = {};
  // state of the last projection
  bool have_proj = false;
  // tile lists of the last gem_project (bins_of_proj) or of the last slice
  // batch of gem_query, binned for M = bins_M Gaussians, B = bins_B images
  // with threshold bins_l2tau
  bool have_bins = false;
  // binnings so far, and the one whose longest-first tile order `order`
  // holds (a persistent forward computed it): the backward reuses it
  uint64_t bins_gen = 0, order_gen = ~0ull;
  bool bins_of_proj = false;
  int64_t bins_M = 0;
  int bins_B = 0;
  float bins_l2tau = 0.f;
  bool have_dproj = false;
  const float *params = nullptr;
  const float *R = nullptr;
  const float *t = nullptr;
  int64_t M = 0;
  int B = 0;
};

// The configurations used when neither the context nor the autotuner's cache
// names one (the fastest measured on the benchmark workloads).
constexpr int kDefaultFwdCfg = 3;  // block-aligned, 256-record windows, persistent longest-first
constexpr int kDefaultBwdCfg = 3;  // one lane per record, persistent longest-first

// The autotuner's choices, shared by every context of the process: keyed by
// device, image side, batch and the bit length of M (shapes that bin alike).
namespace {
struct TuneKey {
  int dev, d, B, mbits;
  bool operator<(const TuneKey &o) const {
    return std::tie(dev, d, B, mbits) < std::tie(o.dev, o.d, o.B, o.mbits);
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, std::pair<int, int>> g_tune;

TuneKey tune_key(int d, int B, int64_t M) {
  int dev = 0;
  cudaGetDevice(&dev);
  int bits = 0;
  while (bits < 63 && ((int64_t)1 << bits) <= M) ++bits;
  return TuneKey{dev, d, B, bits};
}
}  // namespace

static int active_fwd(const gem_ctx *c, int B, int64_t M);
static int active_bwd(const gem_ctx *c, int B, int64_t M);

static int fail(gem_ctx *c, int code, const char *fmt, ...) {
  if (c) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(c->err, sizeof(c->err), fmt, ap);
    va_end(ap);
  }
  return code;
}

static int cuda_fail(gem_ctx *c, cudaError_t e, const char *what) {
  return fail(c, GEM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

static bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

static int shape_flags(const gem_config &g) {
  return (g.no_rotation ? kNoRotation : 0) | (g.isotropic ? kIsotropic : 0);
}

// Brackets one stage with events when timing is on and counts its kernels.
struct StageScope {
  gem_ctx *c;
  int st;
  StageScope(gem_ctx *c_, int st_, int kernels) : c(c_), st(st_) {
    c->launches[st] += kernels;
    if (c->timing) cudaEventRecord(c->ev[st][0], c->stream);
  }
  ~StageScope() {
    if (c->timing) {
      cudaEventRecord(c->ev[st][1], c->stream);
      c->recorded[st] = true;
    }
  }
};

template <class T>
static bool alloc(gem_ctx *c, T **p, size_t count) {
  void *q = nullptr;
  if (count == 0) count = 1;
  if (cudaMalloc(&q, count * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  c->allocs.push_back(q);
  *p = (T *)q;
  return true;
}

static bool d_ok(int d) {
  if (d < 16 || d > 768 || d % 16 != 0) return false;
  int m = d;
  while (m % 2 == 0) m /= 2;
  while (m % 3 == 0) m /= 3;
  return m == 1;
}

static thread_local char g_create_err[512];

extern "C" {

const char *gem_create_error(void) { return g_create_err; }

int gem_config_default(gem_config *cfg, int32_t d, float apix, int32_t max_B, int64_t max_M) {
  if (!cfg) return GEM_EINVAL;
  memset(cfg, 0, sizeof(*cfg));
  cfg->d = d;
  cfg->apix = apix;
  cfg->tau = 0.f;
  cfg->norm_mode = 0;
  cfg->max_B = max_B;
  cfg->max_M = max_M;
  cfg->max_pairs = 0;
  cfg->zsort = 1;
  cfg->no_rotation = 0;
  cfg->isotropic = 0;
  cfg->tile = kTile;
  cfg->fp64_check = 0;
  return GEM_OK;
}

static int f64_scratch(gem_ctx *c);

int gem_create(gem_ctx **out, const gem_config *cfg, void *cuda_stream) {
  if (!out || !cfg) return GEM_EINVAL;
  *out = nullptr;
  gem_ctx *c = new (std::nothrow) gem_ctx();
  if (!c) return GEM_ENOMEM;
  c->cfg = *cfg;
  c->stream = (cudaStream_t)cuda_stream;
  const gem_config &g = c->cfg;
  int code = GEM_OK;
  if (!d_ok(g.d))
    code = fail(c, GEM_EINVAL, "d=%d: need a multiple of 16 in 16..768 of the form 2^a 3^b", g.d);
  else if (!(g.apix > 0.f) || !isfinite(g.apix))
    code = fail(c, GEM_EINVAL, "apix must be > 0");
  else if (!(g.tau >= 0.f) || !isfinite(g.tau))
    code = fail(c, GEM_EINVAL, "tau must be finite and >= 0");
  else if (g.norm_mode != 0 && g.norm_mode != 1)
    code = fail(c, GEM_EINVAL, "norm_mode must be 0 or 1");
  else if (g.max_B < 1 || g.max_B > 65535)
    code = fail(c, GEM_EINVAL, "max_B must be in 1..65535");
  else if (g.max_M < 1 || g.max_M > (int64_t)1 << 24)
    code = fail(c, GEM_EINVAL, "max_M must be in 1..2^24");
  else if (g.max_pairs < 0)
    code = fail(c, GEM_EINVAL, "max_pairs must be >= 0");
  else if (g.zsort != 0 && g.zsort != 1)
    code = fail(c, GEM_EINVAL, "zsort must be 0 or 1");
  else if (g.no_rotation != 0 && g.no_rotation != 1)
    code = fail(c, GEM_EINVAL, "no_rotation must be 0 or 1");
  else if (g.isotropic != 0 && g.isotropic != 1)
    code = fail(c, GEM_EINVAL, "isotropic must be 0 or 1");
  else if (g.tile != 0 && g.tile != kTile)
    code = fail(c, GEM_EINVAL, "tile=%d: the rasterisers use %d x %d tiles (0 selects them)", g.tile,
                kTile, kTile);
  else if (g.fp64_check != 0 && g.fp64_check != 1)
    code = fail(c, GEM_EINVAL, "fp64_check must be 0 or 1");
  if (code != GEM_OK) {
    snprintf(g_create_err, sizeof(g_create_err), "%s", c->err);
    delete c;
    return code;
  }
  if (c->cfg.max_pairs == 0) c->cfg.max_pairs = 16 * (int64_t)g.max_B * g.max_M;
  c->cfg.tile = kTile;
  const int d = g.d;
  c->T = (d / kTile) * (d / kTile);
  c->l2tau = g.tau > 0.f ? log2f(g.tau) : -INFINITY;
  fft_plan(d, c->plan);
  const size_t BM = (size_t)g.max_B * (size_t)g.max_M;
  const size_t nchD = bin_chunks_depth(g.max_M), nchT = bin_chunks_tiles(g.max_M);
  c->nbg = g.max_B < 16 ? g.max_B : 16;
  bool ok = alloc(c, &c->gp, g.max_M) && alloc(c, &c->slot_gauss, g.max_M) &&
            alloc(c, &c->gauss_slot, g.max_M) && alloc(c, &c->psort, (size_t)g.max_M * kNpar) &&
            alloc(c, &c->mkey, g.max_M) && alloc(c, &c->rec, BM) && alloc(c, &c->bin.key, BM) &&
            alloc(c, &c->bin.packed, BM) && alloc(c, &c->bin.perm, BM) &&
            alloc(c, &c->bin.dcnt, (size_t)g.max_B * nchD * 256) &&
            alloc(c, &c->bin.tcnt, (size_t)g.max_B * nchT * c->T) &&
            alloc(c, &c->bin.tile_start, (size_t)g.max_B * c->T + 1) &&
            alloc(c, &c->bin.list, (size_t)c->cfg.max_pairs) &&
            alloc(c, &c->bin.hits, (size_t)c->cfg.max_pairs) &&
            alloc(c, &c->bin.chunk_base, (size_t)g.max_B * nchT) &&
            alloc(c, &c->bin.chunk_n, (size_t)g.max_B * nchT) && alloc(c, &c->bin.hit_ctr, 1) &&
            alloc(c, &c->mom, BM * 6) &&
            alloc(c, &c->part, (size_t)c->nbg * g.max_M * kNpar) &&
            alloc(c, &c->proj, (size_t)g.max_B * d * d) &&
            alloc(c, &c->dproj, (size_t)g.max_B * d * d) &&
            alloc(c, &c->Z, (size_t)g.max_B * d * d) && alloc(c, &c->tw, (size_t)d) &&
            alloc(c, &c->lossp, (size_t)g.max_B * (ctf_partials(d) + 1)) && alloc(c, &c->status, 1) &&
            alloc(c, &c->kept, 2) &&
            alloc(c, &c->order, (size_t)g.max_B * c->T) && alloc(c, &c->next_tile, 2);
  // nearest-neighbour grid: at most 2 max_M + 64 cells
  c->knn.cap = 2 * g.max_M + 64;
  ok = ok && alloc(c, &c->knn.part, 608 * 6) && alloc(c, &c->knn.grid, 1) &&
       alloc(c, &c->knn.cell, g.max_M) && alloc(c, &c->knn.cnt, c->knn.cap) &&
       alloc(c, &c->knn.start, c->knn.cap + 1) && alloc(c, &c->knn.fill, c->knn.cap) &&
       alloc(c, &c->knn.order, g.max_M) &&
       alloc(c, &c->knn.bsum, (size_t)knn_scan_blocks(c->knn.cap) + 1) &&
       alloc(c, &c->qp, g.max_M);
  if (ok && g.fp64_check) {
    const size_t n = (size_t)g.max_B * d * d;
    ok = f64_scratch(c) == GEM_OK && alloc(c, &c->f64.params_in, (size_t)g.max_M * kNpar) &&
         alloc(c, &c->f64.R_in, (size_t)g.max_B * 9) && alloc(c, &c->f64.t_in, (size_t)g.max_B * 2) &&
         alloc(c, &c->f64.images_in, n) &&
         alloc(c, &c->f64.ctf_in, (size_t)g.max_B * d * (d / 2 + 1)) &&
         alloc(c, &c->f64.proj, n) && alloc(c, &c->f64.pred, n) && alloc(c, &c->f64.dproj, n) &&
         alloc(c, &c->f64.grad, (size_t)g.max_M * kNpar);
  }
  if (!ok) {
    snprintf(g_create_err, sizeof(g_create_err), "device allocation failed");
    gem_destroy(c);
    return GEM_ENOMEM;
  }
  c->bin.cap = c->cfg.max_pairs;
  c->bin.status = c->status;
  std::vector<float2> tw(d);
  for (int m = 0; m < d; ++m) {
    double a = -2.0 * 3.14159265358979323846 * m / d;
    tw[m] = make_float2((float)cos(a), (float)sin(a));
  }
  cudaError_t e;
  if ((e = cudaMemcpy(c->tw, tw.data(), d * sizeof(float2), cudaMemcpyHostToDevice)) !=
          cudaSuccess ||
      (e = cudaMemset(c->status, 0, sizeof(int))) != cudaSuccess ||
      (e = bin_configure(d)) != cudaSuccess || (e = ctf_configure(d)) != cudaSuccess) {
    snprintf(g_create_err, sizeof(g_create_err), "set-up: %s", cudaGetErrorString(e));
    gem_destroy(c);
    return GEM_ECUDA;
  }
  g_create_err[0] = 0;
  *out = c;
  return GEM_OK;
}

int gem_destroy(gem_ctx *c) {
  if (!c) return GEM_OK;
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  for (void *p : c->allocs) cudaFree(p);
  for (int i = 0; i < GEM_NSTAGES; ++i)
    for (int k = 0; k < 2; ++k)
      if (c->ev[i][k]) cudaEventDestroy(c->ev[i][k]);
  delete c;
  return GEM_OK;
}

const char *gem_last_error(const gem_ctx *c) { return c ? c->err : ""; }

int gem_set_stream(gem_ctx *c, void *s) {
  if (!c) return GEM_EINVAL;
  c->stream = (cudaStream_t)s;
  return GEM_OK;
}

int gem_status(gem_ctx *c) {
  if (!c) return GEM_EINVAL;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "stream synchronise");
  int st = 0;
  if ((e = cudaMemcpy(&st, c->status, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(c, e, "status read");
  if ((e = cudaMemset(c->status, 0, sizeof(int))) != cudaSuccess)
    return cuda_fail(c, e, "status clear");
  if (st & GEM_STATUS_CAPACITY)
    return fail(c, GEM_ECAPACITY, "pair list exceeded max_pairs=%lld",
                (long long)c->cfg.max_pairs);
  return GEM_OK;
}

static int check_project_args(gem_ctx *c, const float *params, int64_t M, int32_t B,
                              const float *R, const float *t, const float *proj) {
  if (!c) return GEM_EINVAL;
  if (!params || !R || !t || !proj) return fail(c, GEM_EINVAL, "null pointer argument");
  if (!aligned16(proj)) return fail(c, GEM_EINVAL, "proj must be 16-byte aligned");
  if (M < 1 || M > c->cfg.max_M)
    return fail(c, GEM_EINVAL, "M=%lld outside 1..max_M=%lld", (long long)M,
                (long long)c->cfg.max_M);
  if (B < 1 || B > c->cfg.max_B)
    return fail(c, GEM_EINVAL, "B=%d outside 1..max_B=%d", B, c->cfg.max_B);
  return GEM_OK;
}

static int prep(gem_ctx *c, const float *params, int64_t M, int32_t B, const float *R,
                const float *t) {
  StageScope sc(c, GEM_STAGE_PREP, 9);
  cudaError_t e;
  const gem_config &g = c->cfg;
  // slot order: a stable sort of the Gaussians by the 3D Morton key of their
  // means (the binning's depth-pass scratch is free until the binning)
  if ((e = launch_morton_key(params, M, (float)g.d * g.apix, c->mkey, c->stream)) != cudaSuccess ||
      (e = launch_sort16(c->mkey, M, 1, c->bin.dcnt, c->bin.packed, c->slot_gauss, c->stream)) !=
          cudaSuccess)
    return cuda_fail(c, e, "slot order");
  if ((e = launch_gauss_prep(params, c->slot_gauss, M, g.norm_mode, shape_flags(g), c->gp,
                             c->psort, c->gauss_slot, c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "gauss_prep");
  // depth keys span [-d apix, d apix]: the half-diagonal of the box is shorter
  const float zrange = (float)g.d * g.apix;
  if ((e = launch_view_prep(c->gp, M, B, R, t, g.apix, g.d, c->l2tau, zrange, c->rec,
                            c->bin.key, c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "view_prep");
  c->params = params;
  c->R = R;
  c->t = t;
  c->M = M;
  c->B = B;
  return GEM_OK;
}

int gem_project(gem_ctx *c, const float *params, int64_t M, int32_t B, const float *R,
                const float *t, float *proj) {
  int rc = check_project_args(c, params, M, B, R, t, proj);
  if (rc) return rc;
  c->have_proj = false;
  c->have_dproj = false;
  if ((rc = prep(c, params, M, B, R, t))) return rc;
  cudaError_t e;
  const gem_config &g = c->cfg;
  const uint32_t *perm = nullptr;
  {
    StageScope sc(c, GEM_STAGE_BIN, g.zsort ? 10 : 4);
    c->have_bins = false;
    ++c->bins_gen;
    if ((e = launch_bin(c->rec, c->bin.key, M, B, g.d, c->l2tau, g.zsort, c->bin, &perm,
                        c->stream)) != cudaSuccess)
      return cuda_fail(c, e, "bin");
    c->have_bins = true;
    c->bins_of_proj = true;
    c->bins_M = M;
    c->bins_B = B;
    c->bins_l2tau = c->l2tau;
  }
  {
    const int fc = active_fwd(c, B, M);
    StageScope sc(c, GEM_STAGE_RASTER_FWD, fwd_config(fc).persistent ? 2 : 1);
    if ((e = launch_raster_fwd(fc, c->rec, c->bin.list,
                               c->bin.tile_start, c->bin.cap, M, B, g.d, c->l2tau, proj, c->order,
                               c->next_tile, c->stream)) != cudaSuccess)
      return cuda_fail(c, e, "raster_fwd");
    if (fwd_config(fc).persistent) c->order_gen = c->bins_gen;
  }
  c->have_proj = true;
  return GEM_OK;
}

int gem_project_dense(gem_ctx *c, const float *params, int64_t M, int32_t B, const float *R,
                      const float *t, float *proj) {
  int rc = check_project_args(c, params, M, B, R, t, proj);
  if (rc) return rc;
  c->have_proj = false;
  c->have_dproj = false;
  if ((rc = prep(c, params, M, B, R, t))) return rc;
  c->have_bins = false;  // the records changed; any tile lists are stale
  cudaError_t e;
  StageScope sc(c, GEM_STAGE_RASTER_FWD, 1);
  if ((e = launch_dense_fwd(c->rec, M, B, c->cfg.d, c->l2tau, proj, c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "dense_fwd");
  c->have_proj = true;
  return GEM_OK;
}

int gem_ctf_loss(gem_ctx *c, int32_t B, const float *proj, const float *ctf,
                 const float *ctf_params, const float *images, float *pred, float *dproj,
                 double *loss_img, double *loss) {
  if (!c) return GEM_EINVAL;
  if (!proj || !images) return fail(c, GEM_EINVAL, "null proj or images");
  if (!aligned16(proj) || !aligned16(images) || !aligned16(pred) || !aligned16(dproj))
    return fail(c, GEM_EINVAL, "image arrays must be 16-byte aligned");
  if ((ctf == nullptr) == (ctf_params == nullptr))
    return fail(c, GEM_EINVAL, "pass exactly one of ctf and ctf_params");
  if (B < 1 || B > c->cfg.max_B)
    return fail(c, GEM_EINVAL, "B=%d outside 1..max_B=%d", B, c->cfg.max_B);
  StageScope sc(c, GEM_STAGE_CTF, 3 + (loss_img || loss ? 1 : 0) + (loss ? 1 : 0));
  cudaError_t e = launch_ctf_loss(c->cfg.d, B, c->cfg.apix, c->plan, c->tw, proj, ctf,
                                  ctf_params, images, c->Z, c->lossp, pred, dproj, loss_img,
                                  loss, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "ctf_loss");
  return GEM_OK;
}

static int backward_common(gem_ctx *c, const float *dproj, float *grad, bool dense) {
  if (!c) return GEM_EINVAL;
  if (!dproj || !grad) return fail(c, GEM_EINVAL, "null dproj or grad");
  if (!aligned16(dproj)) return fail(c, GEM_EINVAL, "dproj must be 16-byte aligned");
  if (!c->have_proj) return fail(c, GEM_ESTATE, "no projection to differentiate");
  if (!dense && !(c->have_bins && c->bins_of_proj))
    return fail(c, GEM_ESTATE, "the last projection was dense: no tile lists to differentiate");
  const gem_config &g = c->cfg;
  cudaError_t e;
  // the whole buffer, should an earlier pass have stopped before clearing it
  size_t mbytes = (size_t)g.max_B * g.max_M * 6 * sizeof(double);
  {
    // the persistent forms add a tile-order launch unless the forward's
    // order of these bins is reused (then a counter reset, no kernel)
    StageScope sc(c, GEM_STAGE_RASTER_BWD,
                  1 + (!dense && bwd_config(active_bwd(c, c->B, c->M)).persistent &&
                               c->order_gen != c->bins_gen
                           ? 1
                           : 0));
    if (!dense && !c->mom_clean && (e = cudaMemsetAsync(c->mom, 0, mbytes, c->stream)) != cudaSuccess)
      return cuda_fail(c, e, "moment clear");
    c->mom_clean = false;
    if (dense)
      e = launch_dense_bwd(c->rec, c->M, c->B, g.d, c->l2tau, dproj, c->mom, c->stream);
    else
      e = launch_raster_bwd(active_bwd(c, c->B, c->M), c->rec, c->bin.list,
                            c->bin.tile_start, c->bin.cap, c->M, c->B, g.d, c->l2tau, dproj, c->mom,
                            c->order, c->next_tile + 1, c->order_gen == c->bins_gen, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "raster_bwd");
  }
  StageScope sc(c, GEM_STAGE_PREP_BWD, 2);
  if ((e = launch_prep_bwd(c->psort, c->gauss_slot, c->gp, c->M, c->B, c->R, c->t, g.apix, g.d, g.norm_mode, shape_flags(g),
                           c->mom, c->part, c->nbg, grad, c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "prep_bwd");
  c->mom_clean = true;
  return GEM_OK;
}

int gem_project_backward(gem_ctx *c, const float *dproj, float *grad) {
  return backward_common(c, dproj, grad, false);
}

int gem_project_backward_dense(gem_ctx *c, const float *dproj, float *grad) {
  return backward_common(c, dproj, grad, true);
}

int gem_set_gaussians(gem_ctx *c, const float *params, int64_t M) {
  if (!c) return GEM_EINVAL;
  if (!params) return fail(c, GEM_EINVAL, "null params");
  if (M < 1 || M > c->cfg.max_M)
    return fail(c, GEM_EINVAL, "M=%lld outside 1..max_M=%lld", (long long)M,
                (long long)c->cfg.max_M);
  c->set_params = params;
  c->set_M = M;
  return GEM_OK;
}

// gem_forward of an fp64_check context: the float inputs widened into the
// context's float64 buffers, then the FP64 check-mode steps.
static int forward_f64(gem_ctx *c, const float *params, int64_t M, int32_t B, const float *R,
                       const float *t, const float *ctf, const float *ctf_params,
                       const float *images, float *pred, double *loss) {
  int rc = check_project_args(c, params, M, B, R, t, c->proj);
  if (rc) return rc;
  const gem_config &g = c->cfg;
  const int64_t n = (int64_t)B * g.d * g.d;
  c->f64.have_dproj = false;
  cudaError_t e;
  if ((e = launch_f64_widen(params, c->f64.params_in, M * kNpar, c->stream)) != cudaSuccess ||
      (e = launch_f64_widen(R, c->f64.R_in, (int64_t)B * 9, c->stream)) != cudaSuccess ||
      (e = launch_f64_widen(t, c->f64.t_in, (int64_t)B * 2, c->stream)) != cudaSuccess ||
      (e = launch_f64_widen(images, c->f64.images_in, n, c->stream)) != cudaSuccess ||
      (e = launch_f64_widen(ctf ? ctf : ctf_params, c->f64.ctf_in,
                            ctf ? (int64_t)B * g.d * (g.d / 2 + 1) : (int64_t)B * 8, c->stream)) !=
          cudaSuccess)
    return cuda_fail(c, e, "fp64_check widen");
  if ((rc = gem_project_f64(c, c->f64.params_in, M, B, c->f64.R_in, c->f64.t_in, c->f64.proj)))
    return rc;
  if ((rc = gem_ctf_loss_f64(c, B, c->f64.proj, ctf ? c->f64.ctf_in : nullptr,
                             ctf ? nullptr : c->f64.ctf_in, c->f64.images_in,
                             pred ? c->f64.pred : nullptr, c->f64.dproj, nullptr, loss)))
    return rc;
  if (pred && (e = launch_f64_narrow(c->f64.pred, pred, n, c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "fp64_check narrow");
  c->f64.have_dproj = true;
  c->M = M;
  return GEM_OK;
}

int gem_forward(gem_ctx *c, const float *params, int64_t M, int32_t B, const float *R,
                const float *t, const float *ctf, const float *ctf_params, const float *images,
                float *pred, double *loss) {
  if (!c) return GEM_EINVAL;
  if (!images) return fail(c, GEM_EINVAL, "null images");
  if ((ctf == nullptr) == (ctf_params == nullptr))
    return fail(c, GEM_EINVAL, "pass exactly one of ctf and ctf_params");
  if (!params) {
    if (!c->set_params) return fail(c, GEM_ESTATE, "params NULL and no gem_set_gaussians");
    params = c->set_params;
    M = c->set_M;
  }
  c->have_dproj = false;
  if (c->cfg.fp64_check)
    return forward_f64(c, params, M, B, R, t, ctf, ctf_params, images, pred, loss);
  int rc = gem_project(c, params, M, B, R, t, c->proj);
  if (rc) return rc;
  rc = gem_ctf_loss(c, B, c->proj, ctf, ctf_params, images, pred, c->dproj, nullptr, loss);
  if (rc) return rc;
  c->have_dproj = true;
  return GEM_OK;
}

int gem_backward(gem_ctx *c, float *grad) {
  if (!c) return GEM_EINVAL;
  if (c->cfg.fp64_check) {
    if (!c->f64.have_dproj) return fail(c, GEM_ESTATE, "gem_backward needs a gem_forward first");
    if (!grad) return fail(c, GEM_EINVAL, "null grad");
    int rc = gem_project_backward_f64(c, c->f64.dproj, c->f64.grad);
    if (rc) return rc;
    cudaError_t e = launch_f64_narrow(c->f64.grad, grad, c->f64.M * kNpar, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "fp64_check narrow");
    return GEM_OK;
  }
  if (!c->have_dproj) return fail(c, GEM_ESTATE, "gem_backward needs a gem_forward first");
  return gem_project_backward(c, c->dproj, grad);
}

int gem_pair_count(gem_ctx *c, int64_t *n) {
  if (!c || !n) return GEM_EINVAL;
  if (!c->have_bins) return fail(c, GEM_ESTATE, "no tile lists yet");
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "synchronise");
  e = cudaMemcpy(n, c->bin.tile_start + (int64_t)c->bins_B * c->T, sizeof(int64_t),
                 cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "pair count read");
  return GEM_OK;
}

int gem_inspect_bins(gem_ctx *c, int64_t *tile_start, uint32_t *list, int64_t list_cap) {
  if (!c || !tile_start || !list) return GEM_EINVAL;
  int64_t n = 0;
  int rc = gem_pair_count(c, &n);
  if (rc) return rc;
  if (n > c->bin.cap) return fail(c, GEM_ECAPACITY, "lists overflowed max_pairs");
  if (list_cap < n) return fail(c, GEM_EINVAL, "list_cap %lld < pair count %lld",
                                (long long)list_cap, (long long)n);
  cudaError_t e;
  size_t ts = ((size_t)c->bins_B * c->T + 1) * sizeof(int64_t);
  // the lists of a projection hold slots: map them to Gaussian indices
  if ((e = cudaMemcpy(tile_start, c->bin.tile_start, ts, cudaMemcpyDeviceToDevice)) !=
          cudaSuccess ||
      (e = launch_map_slots(c->bin.list, c->bins_of_proj ? c->slot_gauss : nullptr, n, list,
                            c->stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "inspect copy");
  return GEM_OK;
}

int gem_inspect_records(gem_ctx *c, float *out) {
  if (!c || !out) return GEM_EINVAL;
  if (!c->have_proj) return fail(c, GEM_ESTATE, "no projection yet");
  cudaError_t e = launch_inspect_records(c->rec, c->gp, c->slot_gauss, c->M, c->B, c->R, c->t, c->cfg.apix,
                                         c->cfg.d, out, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "inspect records");
  if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "synchronise");
  return GEM_OK;
}

int gem_pair_stats(gem_ctx *c, int64_t *kept, int64_t *evaluated) {
  if (!c || !kept) return GEM_EINVAL;
  if (!c->have_bins) return fail(c, GEM_ESTATE, "no tile lists yet");
  const gem_config &g = c->cfg;
  cudaError_t e;
  if ((e = cudaMemsetAsync(c->kept, 0, 2 * sizeof(unsigned long long), c->stream)) !=
          cudaSuccess ||
      (e = launch_count_kept(active_fwd(c, c->bins_B, c->bins_M), c->rec, c->bin.list,
                             c->bin.tile_start, c->bin.cap, c->bins_M, c->bins_B, g.d,
                             c->bins_l2tau, c->kept, c->order, c->next_tile, c->stream)) !=
          cudaSuccess ||
      (e = cudaStreamSynchronize(c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "pair count");
  unsigned long long h[2] = {0, 0};
  if ((e = cudaMemcpy(h, c->kept, sizeof(h), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(c, e, "pair count read");
  *kept = (int64_t)h[0];
  if (evaluated) *evaluated = (int64_t)h[1];
  return GEM_OK;
}

int gem_timing(gem_ctx *c, int enable) {
  if (!c) return GEM_EINVAL;
  if (enable && !c->ev[0][0]) {
    for (int i = 0; i < GEM_NSTAGES; ++i)
      for (int k = 0; k < 2; ++k) {
        cudaError_t e = cudaEventCreate(&c->ev[i][k]);
        if (e != cudaSuccess) return cuda_fail(c, e, "event create");
      }
  }
  c->timing = enable != 0;
  for (int i = 0; i < GEM_NSTAGES; ++i) {
    c->recorded[i] = false;
    c->launches[i] = 0;
  }
  return GEM_OK;
}

int gem_timing_read(gem_ctx *c, float *ms, int64_t *launches) {
  if (!c) return GEM_EINVAL;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "synchronise");
  for (int i = 0; i < GEM_NSTAGES; ++i) {
    float t = 0.f;
    if (c->recorded[i] && (e = cudaEventElapsedTime(&t, c->ev[i][0], c->ev[i][1])) != cudaSuccess)
      return cuda_fail(c, e, "event elapsed");
    if (ms) ms[i] = t;
    if (launches) launches[i] = c->launches[i];
    c->recorded[i] = false;
    c->launches[i] = 0;
  }
  return GEM_OK;
}

int gem_query(gem_ctx *c, const float *params, int64_t M, float tau, float *vol) {
  if (!c) return GEM_EINVAL;
  if (!params || !vol) return fail(c, GEM_EINVAL, "null params or vol");
  if (!aligned16(vol)) return fail(c, GEM_EINVAL, "vol must be 16-byte aligned");
  if (M < 1 || M > c->cfg.max_M)
    return fail(c, GEM_EINVAL, "M=%lld outside 1..max_M=%lld", (long long)M,
                (long long)c->cfg.max_M);
  if (!(tau >= 0.f) || !isfinite(tau)) return fail(c, GEM_EINVAL, "tau must be finite and >= 0");
  const gem_config &g = c->cfg;
  // the slices reuse the projection scratch: the backward state is gone
  c->have_proj = false;
  c->have_dproj = false;
  c->have_bins = false;
  const float l2tau = tau > 0.f ? log2f(tau) : -INFINITY;
  cudaError_t e;
  if ((e = launch_query_prep(params, M, g.norm_mode, shape_flags(g), c->qp, c->stream)) !=
      cudaSuccess)
    return cuda_fail(c, e, "query prep");
  const size_t slice = (size_t)g.d * g.d;
  for (int k0 = 0; k0 < g.d; k0 += g.max_B) {
    const int ns = g.d - k0 < g.max_B ? g.d - k0 : g.max_B;
    const uint32_t *perm = nullptr;
    ++c->bins_gen;  // the slices' bins replace the projection's
    if ((e = launch_slice_prep(c->qp, M, k0, ns, g.apix, g.d, l2tau, c->rec, c->stream)) !=
            cudaSuccess ||
        (e = launch_bin(c->rec, c->bin.key, M, ns, g.d, l2tau, 0, c->bin, &perm, c->stream)) !=
            cudaSuccess ||
        (e = launch_raster_fwd(active_fwd(c, ns, M), c->rec, c->bin.list,
                               c->bin.tile_start, c->bin.cap, M, ns, g.d, l2tau,
                               vol + (size_t)k0 * slice, c->order, c->next_tile, c->stream)) !=
            cudaSuccess)
      return cuda_fail(c, e, "query");
    c->have_bins = true;
    c->bins_of_proj = false;
    c->bins_M = M;
    c->bins_B = ns;
    c->bins_l2tau = l2tau;
  }
  return GEM_OK;
}

int gem_fsc(gem_ctx *c, const float *map1, const float *map2, float threshold, double *fsc,
            double *sums, double *resolution) {
  if (!c) return GEM_EINVAL;
  if (!map1 || !map2 || !fsc) return fail(c, GEM_EINVAL, "null map or fsc");
  if (!(threshold > -1.f && threshold < 1.f))
    return fail(c, GEM_EINVAL, "threshold must lie in (-1, 1)");
  const int d = c->cfg.d;
  if (!c->fscP) {
    const size_t n = (size_t)d * d * d;
    if (!alloc(c, &c->fscP, n) || !alloc(c, &c->fscQ, n) ||
        !alloc(c, &c->fsc_part, (size_t)fsc_partial_count(d)))
      return fail(c, GEM_ENOMEM, "FSC scratch (%zu bytes) allocation failed", 16 * n);
    cudaError_t e = fsc_configure(d);
    if (e != cudaSuccess) return cuda_fail(c, e, "fsc configure");
  }
  cudaError_t e = launch_fsc(d, c->cfg.apix, threshold, c->plan, c->tw, map1, map2, c->fscP,
                             c->fscQ, c->fsc_part, fsc, sums, resolution, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "fsc");
  return GEM_OK;
}

static int f64_scratch(gem_ctx *c) {
  if (c->f64.gp) return GEM_OK;
  const gem_config &g = c->cfg;
  const size_t BM = (size_t)g.max_B * g.max_M, n = (size_t)g.max_B * g.d * g.d;
  if (!alloc(c, &c->f64.gp, g.max_M) || !alloc(c, &c->f64.rec, BM) ||
      !alloc(c, &c->f64.mom, BM * 6) || !alloc(c, &c->f64.tw, (size_t)g.d) ||
      !alloc(c, &c->f64.Za, n) || !alloc(c, &c->f64.Zb, n) || !alloc(c, &c->f64.Hs, n) ||
      !alloc(c, &c->f64.r, n) || !alloc(c, &c->f64.li, (size_t)g.max_B)) {
    c->f64.gp = nullptr;
    return fail(c, GEM_ENOMEM, "FP64 check-mode scratch allocation failed");
  }
  return GEM_OK;
}

int gem_project_f64(gem_ctx *c, const double *params, int64_t M, int32_t B, const double *R,
                    const double *t, double *proj) {
  if (!c) return GEM_EINVAL;
  if (!params || !R || !t || !proj) return fail(c, GEM_EINVAL, "null pointer argument");
  if (M < 1 || M > c->cfg.max_M)
    return fail(c, GEM_EINVAL, "M=%lld outside 1..max_M=%lld", (long long)M,
                (long long)c->cfg.max_M);
  if (B < 1 || B > c->cfg.max_B)
    return fail(c, GEM_EINVAL, "B=%d outside 1..max_B=%d", B, c->cfg.max_B);
  int rc = f64_scratch(c);
  if (rc) return rc;
  const gem_config &g = c->cfg;
  c->f64.have = false;
  cudaError_t e = launch_f64_project(params, M, B, R, t, (double)g.apix, g.d, g.norm_mode,
                                     shape_flags(g), (double)g.tau, c->f64.gp, c->f64.rec, proj,
                                     c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "project f64");
  c->f64.have = true;
  c->f64.params = params;
  c->f64.R = R;
  c->f64.t = t;
  c->f64.M = M;
  c->f64.B = B;
  return GEM_OK;
}

int gem_ctf_loss_f64(gem_ctx *c, int32_t B, const double *proj, const double *ctf,
                     const double *ctf_params, const double *images, double *pred,
                     double *dproj, double *loss_img, double *loss) {
  if (!c) return GEM_EINVAL;
  if (!proj || !images) return fail(c, GEM_EINVAL, "null proj or images");
  if ((ctf == nullptr) == (ctf_params == nullptr))
    return fail(c, GEM_EINVAL, "pass exactly one of ctf and ctf_params");
  if (B < 1 || B > c->cfg.max_B)
    return fail(c, GEM_EINVAL, "B=%d outside 1..max_B=%d", B, c->cfg.max_B);
  int rc = f64_scratch(c);
  if (rc) return rc;
  cudaError_t e = launch_f64_ctf_loss(c->cfg.d, B, (double)c->cfg.apix, proj, ctf, ctf_params,
                                      images, pred, dproj, loss_img, loss, c->f64.tw, c->f64.Hs,
                                      c->f64.Za, c->f64.Zb, c->f64.r, c->f64.li, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "ctf_loss f64");
  return GEM_OK;
}

int gem_project_backward_f64(gem_ctx *c, const double *dproj, double *grad) {
  if (!c) return GEM_EINVAL;
  if (!dproj || !grad) return fail(c, GEM_EINVAL, "null dproj or grad");
  if (!c->f64.have) return fail(c, GEM_ESTATE, "no FP64 projection to differentiate");
  const gem_config &g = c->cfg;
  cudaError_t e = launch_f64_backward(c->f64.params, c->f64.gp, c->f64.rec, c->f64.M, c->f64.B,
                                      c->f64.R, c->f64.t, (double)g.apix, g.d, g.norm_mode,
                                      shape_flags(g), (double)g.tau, dproj, c->f64.mom, grad,
                                      c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "backward f64");
  return GEM_OK;
}

int gem_adam_step(gem_ctx *c, int64_t M, const gem_adam_config *cfg, float *raw, float *m,
                  float *v, const float *grad, float *params, const float *iso_scale) {
  if (!c) return GEM_EINVAL;
  if (!cfg || !raw || !m || !v || !grad || !params)
    return fail(c, GEM_EINVAL, "null argument");
  if (M < 1 || M > c->cfg.max_M)
    return fail(c, GEM_EINVAL, "M=%lld outside 1..max_M=%lld", (long long)M,
                (long long)c->cfg.max_M);
  if (!(cfg->beta1 >= 0.f && cfg->beta1 < 1.f) || !(cfg->beta2 >= 0.f && cfg->beta2 < 1.f) ||
      !(cfg->eps > 0.f) || cfg->step < 1)
    return fail(c, GEM_EINVAL, "need 0 <= beta < 1, eps > 0, step >= 1");
  AdamArgs a;
  for (int k = 0; k < 4; ++k) {
    if (!(cfg->lr[k] >= 0.f) || !isfinite(cfg->lr[k]))
      return fail(c, GEM_EINVAL, "learning rates must be finite and >= 0");
    a.lr[k] = cfg->lr[k];
  }
  a.beta1 = cfg->beta1;
  a.beta2 = cfg->beta2;
  a.eps = cfg->eps;
  a.c1 = (float)(1.0 / (1.0 - pow((double)cfg->beta1, (double)cfg->step)));
  a.c2 = (float)(1.0 / (1.0 - pow((double)cfg->beta2, (double)cfg->step)));
  cudaError_t e = launch_adam(a, M, raw, m, v, grad, params, iso_scale, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "adam");
  return GEM_OK;
}

int gem_activate(gem_ctx *c, int64_t M, const float *raw, float *params) {
  if (!c) return GEM_EINVAL;
  if (!raw || !params) return fail(c, GEM_EINVAL, "null argument");
  if (M < 1 || M > c->cfg.max_M)
    return fail(c, GEM_EINVAL, "M=%lld outside 1..max_M=%lld", (long long)M,
                (long long)c->cfg.max_M);
  cudaError_t e = launch_activate(M, raw, params, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "activate");
  return GEM_OK;
}

int gem_nn_distance(gem_ctx *c, const float *params, int64_t M, int32_t k, float *dist,
                    int32_t *idx) {
  if (!c) return GEM_EINVAL;
  if (!params || !dist) return fail(c, GEM_EINVAL, "null params or dist");
  if (M < 1 || M > c->cfg.max_M)
    return fail(c, GEM_EINVAL, "M=%lld outside 1..max_M=%lld", (long long)M,
                (long long)c->cfg.max_M);
  if (k < 1 || k > 16) return fail(c, GEM_EINVAL, "k=%d outside 1..16", k);
  cudaError_t e = launch_knn(params, M, k, c->knn, dist, idx, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "nearest neighbours");
  return GEM_OK;
}

int gem_raster_config_count(int32_t *n_fwd, int32_t *n_bwd) {
  if (n_fwd) *n_fwd = fwd_config_count();
  if (n_bwd) *n_bwd = bwd_config_count();
  return GEM_OK;
}

const char *gem_raster_config_name(int32_t kind, int32_t i) {
  if (kind == 0 && i >= 0 && i < fwd_config_count()) return fwd_config(i).name;
  if (kind == 1 && i >= 0 && i < bwd_config_count()) return bwd_config(i).name;
  return "";
}

int gem_set_raster_config(gem_ctx *c, int32_t fwd, int32_t bwd) {
  if (!c) return GEM_EINVAL;
  if (fwd < -1 || fwd >= fwd_config_count() || bwd < -1 || bwd >= bwd_config_count())
    return fail(c, GEM_EINVAL, "raster config (%d, %d) outside -1..(%d, %d)", fwd, bwd,
                fwd_config_count() - 1, bwd_config_count() - 1);
  c->fwd_cfg = fwd;
  c->bwd_cfg = bwd;
  return GEM_OK;
}

int gem_get_raster_config(const gem_ctx *c, int32_t B, int64_t M, int32_t *fwd, int32_t *bwd) {
  if (!c || !fwd || !bwd) return GEM_EINVAL;
  *fwd = active_fwd(c, B, M);
  *bwd = active_bwd(c, B, M);
  return GEM_OK;
}

int gem_autotune(gem_ctx *c, const float *params, int64_t M, int32_t B, const float *R,
                 const float *t, int32_t reps, int32_t *fwd_out, int32_t *bwd_out) {
  if (!c) return GEM_EINVAL;
  if (reps < 1 || reps > 1000) return fail(c, GEM_EINVAL, "reps=%d outside 1..1000", reps);
  int rc = check_project_args(c, params, M, B, R, t, c->proj);
  if (rc) return rc;
  const gem_config &g = c->cfg;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return cuda_fail(c, e, "autotune events");
  }
  if (!c->tune_grad && !alloc(c, &c->tune_grad, (size_t)g.max_M * kNpar)) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return fail(c, GEM_ENOMEM, "autotune scratch allocation failed");
  }
  const int keep_f = c->fwd_cfg, keep_b = c->bwd_cfg;
  const bool keep_timing = c->timing;
  c->timing = false;
  // bins of this shape, then each forward configuration on them
  c->fwd_cfg = kDefaultFwdCfg;
  c->bwd_cfg = kDefaultBwdCfg;
  rc = gem_project(c, params, M, B, R, t, c->proj);
  float best_f = INFINITY, best_b = INFINITY;
  int bf = kDefaultFwdCfg, bb = kDefaultBwdCfg;
  for (int i = 0; rc == GEM_OK && i < fwd_config_count(); ++i) {
    float ms = 0.f;
    for (int r = -1; r < reps; ++r) {  // r = -1: warm-up
      cudaEventRecord(e0, c->stream);
      e = launch_raster_fwd(i, c->rec, c->bin.list, c->bin.tile_start, c->bin.cap, M,
                            B, g.d, c->l2tau, c->proj, c->order, c->next_tile, c->stream);
      if (e == cudaSuccess && fwd_config(i).persistent) c->order_gen = c->bins_gen;
      cudaEventRecord(e1, c->stream);
      if (e != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess) {
        rc = cuda_fail(c, e, "autotune forward");
        break;
      }
      float x = 0.f;
      cudaEventElapsedTime(&x, e0, e1);
      if (r >= 0) ms += x;
    }
    if (rc == GEM_OK && ms < best_f) best_f = ms, bf = i;
  }
  // each backward configuration, upstream gradient = the projection (the
  // cost does not depend on its values), moments cleared by the chain rule
  for (int i = 0; rc == GEM_OK && i < bwd_config_count(); ++i) {
    c->bwd_cfg = i;
    float ms = 0.f;
    for (int r = -1; r < reps && rc == GEM_OK; ++r) {
      cudaEventRecord(e0, c->stream);
      rc = backward_common(c, c->proj, c->tune_grad, false);
      cudaEventRecord(e1, c->stream);
      if (rc == GEM_OK && (e = cudaEventSynchronize(e1)) != cudaSuccess) rc = cuda_fail(c, e, "autotune backward");
      float x = 0.f;
      if (rc == GEM_OK) cudaEventElapsedTime(&x, e0, e1);
      if (r >= 0) ms += x;
    }
    if (rc == GEM_OK && ms < best_b) best_b = ms, bb = i;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->timing = keep_timing;
  c->fwd_cfg = keep_f;
  c->bwd_cfg = keep_b;
  c->have_proj = false;  // the autotuner's projection is not the caller's
  c->have_dproj = false;
  if (rc) return rc;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune[tune_key(g.d, B, M)] = std::make_pair(bf, bb);
  }
  if (fwd_out) *fwd_out = bf;
  if (bwd_out) *bwd_out = bb;
  return GEM_OK;
}

}  // extern "C"

static int active_fwd(const gem_ctx *c, int B, int64_t M) {
  if (c->fwd_cfg >= 0) return c->fwd_cfg;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  auto it = g_tune.find(tune_key(c->cfg.d, B, M));
  return it == g_tune.end() ? kDefaultFwdCfg : it->second.first;
}

static int active_bwd(const gem_ctx *c, int B, int64_t M) {
  if (c->bwd_cfg >= 0) return c->bwd_cfg;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  auto it = g_tune.find(tune_key(c->cfg.d, B, M));
  return it == g_tune.end() ? kDefaultBwdCfg : it->second.second;
}
