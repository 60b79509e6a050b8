// lfsr_apply_normal_noalloc: the x-step normal-matrix product q = M p and
// <p, M p> without a handle and without any device allocation.
//
// The two kernels it runs (the generic NLTV kernel in NL_APPLY mode and the
// operator kernel, specialised or generic, in OP_NORMAL mode) need global
// scratch for their float64 block partials, last-block counters, finished
// totals.  Here that scratch is a file-scope __device__ array of
// fixed size, present on every GPU that loads the library until the process
// exits.  Host code only holds a host-side stand-in for the array's name, so
// the array's device address is looked up with cudaGetSymbolAddress once per
// device (with that device current) and passed to the kernels.
#include <cmath>
#include <cstddef>
#include <mutex>

#include "lfsr.h"
#include "lfsr_internal.cuh"

using namespace lfsr;

// The no-allocation scratch: block partials, counters and totals of the two
// grid reductions.  Zero-initialised at module load; cleared again (the
// scalars) at the start of every call.
static __device__ __align__(256) unsigned char g_noalloc_scratch[LFSR_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxCtas = LFSR_NOALLOC_MAX_TILES;
constexpr int kMaxDevices = 64;

constexpr int kMaxOpCtas = 1024;

struct NoallocScratch {
  DevScalars sc;
  unsigned int counter;            // the specialised operator kernel's arrival counter
  float2 theta[LFSR_MAX_VIEWS];    // angular offsets of the views
  double nl_partials[kMaxCtas];    // NLTV part, one per 32 x 32 tile
  double op_partials[kMaxOpCtas];  // operator part, one per CTA
};

static_assert(sizeof(NoallocScratch) <= LFSR_NOALLOC_SCRATCH_BYTES, "scratch size");

struct DeviceSetup {
  bool ready = false;
  uint64_t geom_ready = 0;   // bit 16 z + kb: operator kernels of (scale, kb) prepared
  NoallocScratch* scratch = nullptr;
  int sm_count = 0;
  int optin = 0;
};

std::mutex g_mu;
DeviceSetup g_dev[kMaxDevices];

// Per-device set-up (first call on a device): device address of the scratch
// array, SM count, shared-memory limits of the kernels.
int setup_device(int dev, const Geom& g, DeviceSetup* out, const char** err) {
  std::lock_guard<std::mutex> lock(g_mu);
  DeviceSetup& d = g_dev[dev];
  if (!d.ready) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || ptr == nullptr) {
      *err = "cudaGetSymbolAddress of the no-allocation scratch failed";
      return LFSR_ECUDA;
    }
    if (cudaDeviceGetAttribute(&d.sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&d.optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
            cudaSuccess ||
        nl_prepare(d.optin) != cudaSuccess) {
      *err = "device query / kernel attributes failed";
      return LFSR_ECUDA;
    }
    d.scratch = static_cast<NoallocScratch*>(ptr);
    d.ready = true;
  }
  const uint64_t bit = 1ull << (16 * (g.zeta - 1) + g.kb);
  if (!(d.geom_ready & bit)) {
    if (op_prepare(g, d.optin) != cudaSuccess) {
      *err = "kernel attributes failed";
      return LFSR_ECUDA;
    }
    d.geom_ready |= bit;
  }
  *out = d;
  return LFSR_OK;
}

// the message is readable with lfsr_last_error(NULL)
int nfail(int code, const char* msg) {
  set_thread_error(msg);
  return code;
}

}  // namespace

extern "C" int lfsr_apply_normal_noalloc(const lfsr_params* pr, const float* d_disparity,
                                         const float* d_xw, const float* d_p, float* d_q,
                                         double* pMp, void* cuda_stream) {
  if (!pr || pr->struct_size != sizeof(lfsr_params))
    return nfail(LFSR_EINVAL, "params missing or struct_size mismatch");
  if (!d_disparity || !d_xw || !d_p || !d_q)
    return nfail(LFSR_EINVAL, "device pointers d_disparity, d_xw, d_p, d_q are required");
  if (!pr->blur || !pr->disparity) return nfail(LFSR_EINVAL, "params blur and disparity are required");
  if (pr->U < 1 || pr->V < 1 || !(pr->U & 1) || !(pr->V & 1) || pr->U * pr->V > LFSR_MAX_VIEWS)
    return nfail(LFSR_EINVAL, "U and V must be odd, >= 1, with U*V <= 289");
  if (pr->H < 1 || pr->W < 1 || pr->scale < 1 || pr->scale > 4 || pr->kb < 1 || !(pr->kb & 1) ||
      pr->kb > LFSR_MAX_KB || pr->nltv_window < 3 || pr->nltv_window > 15 ||
      !(pr->nltv_window & 1) || pr->nltv_patch < 1 || pr->nltv_patch > 7 ||
      !(pr->nltv_patch & 1) || !(pr->nltv_h > 0.0) || !(pr->mu > 0.0) ||
      !(pr->lambda1 >= 0.0) || !(pr->lambda2 >= 0.0))
    return nfail(LFSR_EINVAL, "invalid size or parameter");
  if (pr->weights != LFSR_WEIGHTS_PATCH)
    return nfail(pr->weights == LFSR_WEIGHTS_PAPER ? LFSR_EUNSUPPORTED : LFSR_EINVAL,
                 "the no-allocation entry point takes the patch weights only");
  if (pr->disparity_views || pr->adjoint != LFSR_ADJOINT_EXACT)
    return nfail(pr->adjoint == LFSR_ADJOINT_BACKWARD_WARP || pr->disparity_views
                     ? LFSR_EUNSUPPORTED : LFSR_EINVAL,
                 "the no-allocation entry point takes one disparity map and the exact adjoint");
  const long long Hh = (long long)pr->scale * pr->H, Wh = (long long)pr->scale * pr->W;
  // the NLTV kernel runs one CTA per 32 x 32 HR tile; its partials must fit
  const long long nl_tiles = ((Hh + 31) / 32) * ((Wh + 31) / 32);
  if (nl_tiles > kMaxCtas)
    return nfail(LFSR_EINVAL,
                 "HR image too large for the no-allocation scratch (at most 4096 tiles of 32x32)");

  Geom g{};
  g.U = pr->U;
  g.V = pr->V;
  if (pr->views && (pr->n_views < 1 || pr->n_views > pr->U * pr->V))
    return nfail(LFSR_EINVAL, "n_views must be in [1, U*V]");
  for (int j = 0; pr->views && j < pr->n_views; ++j)
    if (pr->views[j] < 0 || pr->views[j] >= pr->U * pr->V || (j && pr->views[j] <= pr->views[j - 1]))
      return nfail(LFSR_EINVAL, "views must be strictly ascending grid indices in [0, U*V)");
  g.sk = pr->views ? pr->n_views : pr->U * pr->V;
  g.H = pr->H;
  g.W = pr->W;
  g.Hh = (int)Hh;
  g.Wh = (int)Wh;
  g.zeta = pr->scale;
  g.kb = pr->kb;
  g.r = (pr->kb - 1) / 2;
  {
    const int kb = pr->kb;
    int am = 0, bm = 0;
    double best = -1.0;
    for (int i = 0; i < kb * kb; ++i) {
      g.k2[i] = pr->blur[i];
      if (std::fabs((double)pr->blur[i]) > best) {
        best = std::fabs((double)pr->blur[i]);
        am = i / kb;
        bm = i % kb;
      }
    }
    g.separable = 0;
    if (best > 0.0) {
      const double pivot = pr->blur[am * kb + bm];
      double err = 0.0;
      for (int a = 0; a < kb; ++a)
        for (int b = 0; b < kb; ++b)
          err = std::fmax(err, std::fabs((double)pr->blur[a * kb + bm] *
                                             (double)pr->blur[am * kb + b] / pivot -
                                         (double)pr->blur[a * kb + b]));
      if (err <= 1e-7 * best) {
        g.separable = 1;
        for (int a = 0; a < kb; ++a) g.kv[a] = pr->blur[a * kb + bm];
        for (int b = 0; b < kb; ++b) g.kh[b] = (float)((double)pr->blur[am * kb + b] / pivot);
      }
    }
  }
  double max_disp = 0.0;
  for (long long i = 0; i < Hh * Wh; ++i)
    max_disp = std::fmax(max_disp, std::fabs((double)pr->disparity[i]));
  g.S = (int)std::ceil(max_disp * 0.5 * (double)((pr->U > pr->V ? pr->U : pr->V) - 1));
  for (int j = 0; j < g.sk; ++j) {
    const int k = pr->views ? pr->views[j] : j;
    g.tu[j] = (float)((k % pr->U) - 0.5 * (pr->U - 1));
    g.tv[j] = (float)((k / pr->U) - 0.5 * (pr->V - 1));
  }
  g.win_r = (pr->nltv_window - 1) / 2;
  g.patch_r = (pr->nltv_patch - 1) / 2;
  g.sh = (pr->nltv_window * pr->nltv_window - 1) / 2;
  for (int a = -g.win_r, n = 0; a <= g.win_r && n < g.sh; ++a)
    for (int b = -g.win_r; b <= g.win_r && n < g.sh; ++b, ++n) {
      g.di[n] = (int8_t)a;
      g.dj[n] = (int8_t)b;
    }
  g.inv_h2 = (float)(1.0 / (pr->nltv_h * pr->nltv_h));
  g.inv_np = (float)(1.0 / (double)(pr->nltv_patch * pr->nltv_patch));
  g.lambda1 = (float)pr->lambda1;
  g.lambda2 = (float)pr->lambda2;
  g.mu = (float)pr->mu;
  g.cA = (float)(pr->lambda2 + 0.5 * pr->mu * pr->lambda1 * pr->lambda1);
  g.thr = (float)(1.0 / pr->mu);
  g.tau = pr->cg_tol;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return nfail(LFSR_ECUDA, "no usable current device");
  DeviceSetup ds;
  const char* err = "no error";
  const int rc = setup_device(dev, g, &ds, &err);
  if (rc != LFSR_OK) return nfail(rc, err);

  OpPlan op{};
  NlPlan nl{};
  const int smem_limit = ds.optin - 1024;
  if (op_plan(g, &op, ds.sm_count, smem_limit) != cudaSuccess)
    return nfail(LFSR_EUNSUPPORTED, "disparity * angular offset too large for the tile");
  if (nl_plan(g, &nl, smem_limit) != cudaSuccess)
    return nfail(LFSR_EUNSUPPORTED, "NLTV window / patch too large");
  const int op_units = op.fast ? op.n_tiles * ((g.sk + FAST_VIEWS - 1) / FAST_VIEWS)
                              : op.n_tiles * g.sk;
  const int grid = op_grid(op, op_units, ds.sm_count);
  if (grid > kMaxOpCtas || nl.n_tiles > kMaxCtas)
    return nfail(LFSR_EINVAL, "launch larger than the no-allocation scratch");

  cudaStream_t s = (cudaStream_t)cuda_stream;
  NoallocScratch* scr = ds.scratch;
  {
    float2 th[LFSR_MAX_VIEWS];
    for (int j = 0; j < g.sk; ++j) th[j] = make_float2(g.tu[j], g.tv[j]);
    if (cudaMemcpyAsync(scr->theta, th, g.sk * sizeof(float2), cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
      return nfail(LFSR_ECUDA, "writing the view offsets failed");
  }
  // counters and totals start at zero on every call
  if (cudaMemsetAsync(&scr->sc, 0, sizeof(DevScalars), s) != cudaSuccess ||
      cudaMemsetAsync(&scr->counter, 0, sizeof(unsigned int), s) != cudaSuccess)
    return nfail(LFSR_ECUDA, "clearing the scratch scalars failed");
  NlArgs na{};
  na.x = d_xw;
  na.p_old = d_p;
  na.out = d_q;
  na.partials = scr->nl_partials;
  na.sc = &scr->sc;
  if (nl_launch(NL_APPLY, g, nl, na, s) != cudaSuccess)
    return nfail(LFSR_ECUDA, "NLTV kernel launch failed");
  cudaError_t le;
  if (op.fast) {
    JobArgs j{};
    j.H = g.H;
    j.W = g.W;
    j.Hh = g.Hh;
    j.Wh = g.Wh;
    j.U = g.U;
    j.V = g.V;
    j.unit0 = 0;
    j.units = op_units;
    j.tiles_x = op.tiles_x;
    j.view0 = 0;
    j.nviews = g.sk;
    j.scale = g.cA;
    j.disp = d_disparity;
    j.theta = scr->theta;
    j.src = d_p;
    j.out = d_q;
    j.sc = &scr->sc;
    TableArgs t{};   // the light field itself goes by value
    t.jobs = nullptr;
    t.unit_job = nullptr;
    t.n_jobs = 1;
    t.total_units = op_units;
    t.partials = scr->op_partials;
    t.counter = &scr->counter;
    le = fast_launch(OP_NORMAL, g, op, t, grid, s, &j);
  } else {
    OpArgs on{};
    on.src = d_p;
    on.disp = d_disparity;
    on.out = d_q;
    on.scale = g.cA;
    on.view0 = 0;
    on.nviews = g.sk;
    on.units = op_units;
    on.partials = scr->op_partials;
    on.sc = &scr->sc;
    le = op_launch(OP_NORMAL, g, op, on, grid, s);
  }
  if (le != cudaSuccess) return nfail(LFSR_ECUDA, "operator kernel launch failed");
  double pap = 0.0;
  if (cudaMemcpyAsync(&pap, &scr->sc.pAp, sizeof(double), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return nfail(LFSR_ECUDA, "reading <p, M p> failed");
  if (pMp) *pMp = pap;
  return LFSR_OK;
}
