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
#include <cstring>
#include <mutex>

#include "lfsr.h"
#include "handle.cuh"
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
  unsigned int disp_absmax_bits;   // max |d_disparity| (float bits), then
  unsigned int disp_nonfinite;     // 1 if d_disparity holds a NaN or an infinity
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

// Largest |d| over n values (as the bits of a non-negative float, whose
// unsigned order is the float order) into bits[0]; bits[1] := 1 if some
// value is not finite.
__global__ void k_disp_absmax(const float* __restrict__ d, long long n, unsigned int* bits) {
  float m = 0.f;
  unsigned int bad = 0u;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float a = fabsf(d[i]);
    if (a <= 3.402823466e38f)
      m = fmaxf(m, a);
    else
      bad = 1u;   // NaN or infinity
  }
  for (int o = 16; o > 0; o >>= 1) {
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    bad |= __shfl_xor_sync(0xffffffffu, bad, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(bits, __float_as_uint(m));
    if (bad) atomicOr(bits + 1, 1u);
  }
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
  // the same validation and geometry as lfsr_create
  Geom g{};
  {
    const int rc = geom_from_params(pr, &g);
    if (rc != LFSR_OK) return rc;   // the message is already on the thread
  }
  if (!d_disparity || !d_xw || !d_p || !d_q)
    return nfail(LFSR_EINVAL, "device pointers d_disparity, d_xw, d_p, d_q are required");
  if (pr->weights != LFSR_WEIGHTS_PATCH)
    return nfail(LFSR_EUNSUPPORTED, "the no-allocation entry point takes the patch weights only");
  if (pr->disparity_views || pr->adjoint != LFSR_ADJOINT_EXACT)
    return nfail(LFSR_EUNSUPPORTED,
                 "the no-allocation entry point takes one disparity map and the exact adjoint");
  if (pr->precision != LFSR_FP32)
    return nfail(LFSR_EUNSUPPORTED,
                 "the no-allocation entry point computes in float32 only (precision LFSR_FP32)");
  // the NLTV kernel runs one CTA per 32 x 32 HR tile; its partials must fit
  const long long nl_tiles = ((g.Hh + 31LL) / 32) * ((g.Wh + 31LL) / 32);
  if (nl_tiles > kMaxCtas)
    return nfail(LFSR_EINVAL,
                 "HR image too large for the no-allocation scratch (at most 4096 tiles of 32x32)");

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return nfail(LFSR_ECUDA, "no usable current device");
  DeviceSetup ds;
  const char* err = "no error";
  const int rc = setup_device(dev, g, &ds, &err);
  if (rc != LFSR_OK) return nfail(rc, err);

  cudaStream_t s = (cudaStream_t)cuda_stream;
  NoallocScratch* scr = ds.scratch;
  // The kernels warp by d_disparity while the halo S above comes from the
  // host map: take S over the device map too (and refuse non-finite values),
  // so that every tap stays inside the staged tile whatever the caller
  // passed.
  {
    unsigned int words[2] = {0u, 0u};
    if (cudaMemsetAsync(&scr->disp_absmax_bits, 0, 2 * sizeof(unsigned int), s) != cudaSuccess)
      return nfail(LFSR_ECUDA, "clearing the disparity check failed");
    k_disp_absmax<<<ds.sm_count * 2, 256, 0, s>>>(d_disparity, (long long)g.Hh * g.Wh,
                                                  &scr->disp_absmax_bits);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(words, &scr->disp_absmax_bits, sizeof(words), cudaMemcpyDeviceToHost,
                        s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return nfail(LFSR_ECUDA, "checking d_disparity failed");
    if (words[1]) return nfail(LFSR_EINVAL, "d_disparity has non-finite values");
    float dmax;
    std::memcpy(&dmax, &words[0], sizeof(float));
    const int sd = shift_bound((double)dmax, pr->U, pr->V);
    if (sd > g.S) g.S = sd;
  }

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
