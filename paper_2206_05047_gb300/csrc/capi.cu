// C ABI of liblfsr: handle, validation, device state, the ADMM iteration
// schedule (Algorithm 1 with the CG x-step of Algorithm 2) and its CUDA-graph
// replay.  See include/lfsr.h for the contract of every entry point.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <mutex>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "handle.cuh"

using namespace lfsr;

namespace {

thread_local std::string t_err = "no error";

constexpr int NUM_CLASSES = KD_NUM;  // profiling classes, see lfsr_stats_t

}  // namespace


namespace {

int fail(lfsr_handle* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  t_err = msg;
  return code;
}

int cuda_fail(lfsr_handle* h, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  return fail(h, e == cudaErrorMemoryAllocation ? LFSR_ENOMEM : LFSR_ECUDA, m);
}

#define CK(h, expr, what)                          \
  do {                                             \
    cudaError_t e_ = (expr);                       \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, what); \
  } while (0)

bool finite_all(const float* a, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(a[i])) return false;
  return true;
}

void free_all(lfsr_handle* h) {
  if (h->graph_pair) cudaGraphExecDestroy(h->graph_pair);
  for (auto& gs : h->graph_single)
    if (gs) cudaGraphExecDestroy(gs);
  for (auto& ev : h->prof) {
    cudaEventDestroy(ev.a);
    cudaEventDestroy(ev.b);
  }
  void* bufs[] = {h->disp, h->y, h->x[0], h->x[1], h->wA[0], h->wA[1], h->wS[0],
                  h->wS[1], h->R, h->P[0], h->P[1], h->Q, h->io, h->wt, h->V, h->occ,
                  h->disp_views, h->hlr, h->wt_map, h->cta_unit0};
  for (void* b : bufs)
    if (b) cudaFree(b);
  if (h->partials) cudaFree(h->partials);
  if (h->sc) cudaFree(h->sc);
  if (h->jobs_dev) cudaFree(h->jobs_dev);
  if (h->theta) cudaFree(h->theta);
  if (h->jobs_scratch) cudaFree(h->jobs_scratch);
  if (h->counters) cudaFree(h->counters);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
}

template <class T>
cudaError_t dalloc(lfsr_handle* h, T** p, size_t n) {
  if (fault_alloc()) return cudaErrorMemoryAllocation;
  cudaError_t e = cudaMalloc((void**)p, n * sizeof(T) > 0 ? n * sizeof(T) : 16);
  if (e == cudaSuccess) h->state_bytes += (int64_t)(n * sizeof(T));
  return e;
}

cudaError_t dalloc_st(lfsr_handle* h, void** p, size_t n, size_t esize) {
  const size_t bytes = n * esize;
  if (fault_alloc()) return cudaErrorMemoryAllocation;
  cudaError_t e = cudaMalloc(p, bytes > 0 ? bytes : 16);
  if (e == cudaSuccess) h->state_bytes += (int64_t)bytes;
  return e;
}

// Copies n floats from a caller buffer of kind `mem` into device memory dst.
cudaError_t to_dev(lfsr_handle* h, float* dst, const float* src, size_t n, int mem) {
  return cudaMemcpyAsync(dst, src, n * sizeof(float),
                         mem == LFSR_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                         h->stream);
}

cudaError_t from_dev(lfsr_handle* h, float* dst, const float* src, size_t n, int mem) {
  return cudaMemcpyAsync(dst, src, n * sizeof(float),
                         mem == LFSR_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                         h->stream);
}

// The float staging buffer for host transfers and layout conversions is
// allocated on first use, so light fields that only move device memory
// (batches, servers) never hold it.
cudaError_t ensure_io(lfsr_handle* h) {
  if (h->io) return cudaSuccess;
  return dalloc(h, &h->io, h->io_floats);
}

int check_mem(lfsr_handle* h, int mem) {
  if (mem != LFSR_MEM_HOST && mem != LFSR_MEM_DEVICE)
    return fail(h, LFSR_EINVAL, "mem_kind must be LFSR_MEM_HOST or LFSR_MEM_DEVICE");
  return LFSR_OK;
}

// Launch helpers ------------------------------------------------------------

double* part_slot(lfsr_handle* h, int slot) { return h->partials + (size_t)slot * h->max_grid; }

// W_k's disparity maps in a generic-operator launch: the per-view maps
// omega_k when given (Sec. 4.1), else the shared map.
void set_warp_maps(const lfsr_handle* h, OpArgs* a) {
  a->disp = h->disp_views ? h->disp_views : h->disp;
  a->disp_stride = h->disp_views ? h->p : 0;
}

// The backward-warp x-step's operator part (a = the OP_NORMAL arguments):
// h_k = A_k p into the LR buffer, then q += cA sum_k W_k^* B^T D^T h_k with
// <p, .> and the CG step length.
cudaError_t bw_normal(lfsr_handle* h, const OpArgs& a, cudaStream_t s) {
  OpArgs f = a;
  f.out = h->hlr;
  f.partials = nullptr;
  cudaError_t e = op_launch(OP_FWD, h->g, h->op, f, h->grid_op, s);
  if (e != cudaSuccess) return e;
  OpArgs b = a;
  b.src = h->hlr;
  b.disp = h->disp;
  b.disp_stride = 0;
  b.pdot = a.src;
  return bw_launch(h->g, h->bw, b, s);
}

// Runs `launch` (one kernel) with profiling events around it when enabled.
template <class F>
cudaError_t timed(lfsr_handle* h, cudaStream_t s, int cls, F&& launch) {
  if (!h->profiling) return launch();
  NvtxRange range(kind_name(cls));
  ProfEvent ev{cls, nullptr, nullptr};
  cudaError_t e = cudaEventCreate(&ev.a);
  if (e == cudaSuccess) e = cudaEventCreate(&ev.b);
  if (e != cudaSuccess) return e;
  cudaEventRecord(ev.a, s);
  e = launch();
  cudaEventRecord(ev.b, s);
  h->prof.push_back(ev);
  return e;
}

// Table of one entry for launch `kind` at (b, pb) of this handle.
TableArgs handle_table(lfsr_handle* h, int kind, int b, int pb) {
  TableArgs t{};
  t.jobs = h->jobs_dev + (2 * b + pb) * KD_NUM + kind;
  t.unit_job = nullptr;
  t.n_jobs = 1;
  t.total_units = kind_units(h, kind);
  t.check_done = (kind == KD_NLA || kind == KD_NORMAL) ? 1 : 0;
  t.partials = part_slot(h, kind_slot(kind));
  t.counter = h->counters + kind;
  if (kind == KD_NORMAL || kind == KD_DATA) t.cta_unit0 = h->cta_unit0;
  return t;
}

// One ADMM iteration (Algorithm 1) on parity b: reads x[b], w*[b], writes
// x[1-b], w*[1-b].  The specialised kernels run from this handle's job
// tables; geometries they do not cover take the generic kernels.
cudaError_t enqueue_iteration(lfsr_handle* h, int b, cudaStream_t s) {
  const int nb = 1 - b;
  const Geom& g = h->g;
  DevScalars* sc = h->sc;
  // v: accumulated in V (zero at entry) on the stored-weight NLTV path, else
  // stored by the generic NLTV block into R
  float* const vbuf = h->nlf ? h->V : h->R;
  cudaError_t e;
  // regulariser rows: weights from x^(n-1), z/w-step, v := mu/2 S^T f
  e = timed(h, s, KD_NLW, [&] {
    if (h->nlf) return nlw2_launch(1, g, handle_table(h, KD_NLW, b, 0), s);
    NlArgs nbk{};
    nbk.x = h->x[b];
    nbk.out = h->R;
    nbk.wS_old = h->wS[b];
    nbk.wS_new = h->wS[nb];
    nbk.occ = h->occ;
    nbk.partials = part_slot(h, RED_DW_S);
    nbk.sc = sc;
    return nl_launch(NL_BLOCK, g, h->nl, nbk, s);
  });
  if (e != cudaSuccess) return e;
  // data rows: a = A x - b, z/w-step, v += A^T (l2 a + mu/2 l1 f)
  e = timed(h, s, KD_DATA, [&] {
    if (h->op.fast)
      return fast_launch(OP_DATA, g, h->op, handle_table(h, KD_DATA, b, 0), h->grid_op, s,
                         &h->jobs_host[(2 * b) * KD_NUM + KD_DATA]);
    OpArgs od{};
    od.src = h->x[b];
    set_warp_maps(h, &od);
    od.out = g.adjoint_bw ? h->hlr : vbuf;
    od.y = h->y;
    od.wA_old = h->wA[b];
    od.wA_new = h->wA[nb];
    od.scale = 1.f;
    od.view0 = 0;
    od.nviews = g.sk;
    od.units = h->op.n_tiles * g.sk;
    od.partials = part_slot(h, RED_DW_A);
    od.sc = sc;
    return op_launch(g.adjoint_bw ? OP_DATA_LR : OP_DATA, g, h->op, od, h->grid_op, s);
  });
  if (e != cudaSuccess) return e;
  if (g.adjoint_bw) {
    // v += sum_k W_k^* B^T D^T h_k (the paper's backward warp)
    e = timed(h, s, KD_DATA, [&] {
      OpArgs ob{};
      ob.src = h->hlr;
      ob.disp = h->disp;
      ob.out = vbuf;
      ob.scale = 1.f;
      ob.view0 = 0;
      ob.nviews = g.sk;
      ob.sc = sc;
      return bw_launch(g, h->bw, ob, s);
    });
    if (e != cudaSuccess) return e;
  }
  // x-step (Algorithm 2): r = -v, x' = x, pi = <r, r> (part of the data
  // launch when fused)
  if (!h->fused_init) {
    e = timed(h, s, KD_INIT, [&] {
      const TableArgs t = handle_table(h, KD_INIT, b, 0);
      return h->nlf ? cg_init_acc_launch(g, t, s) : cg_init_launch(g, t, s);
    });
    if (e != cudaSuccess) return e;
  }
  for (int k = 0; k < h->prm.cg_iters; ++k) {
    const int pb = k & 1;
    e = timed(h, s, KD_NLA, [&] {
      if (h->nlf)
        return h->nla_tma ? nla2t_launch(g, handle_table(h, KD_NLA, b, pb), s)
                          : nla2_launch(g, handle_table(h, KD_NLA, b, pb), s);
      NlArgs na{};
      na.x = h->x[b];
      na.occ = h->occ;
      na.r = h->R;
      na.p_old = h->P[1 - pb];
      na.p_new = h->P[pb];
      na.out = h->Q;
      na.partials = part_slot(h, RED_NLTV);
      na.sc = sc;
      na.use_beta = 1;
      na.check_done = 1;
      return nl_launch(NL_APPLY, g, h->nl, na, s);
    });
    if (e != cudaSuccess) return e;
    e = timed(h, s, KD_NORMAL, [&] {
      if (h->op.fast)
        return fast_launch(OP_NORMAL, g, h->op, handle_table(h, KD_NORMAL, b, pb), h->grid_op, s,
                           &h->jobs_host[(2 * b + pb) * KD_NUM + KD_NORMAL]);
      OpArgs on{};
      on.src = h->P[pb];
      set_warp_maps(h, &on);
      on.out = h->Q;
      on.scale = g.cA;
      on.view0 = 0;
      on.nviews = g.sk;
      on.units = h->op.n_tiles * g.sk;
      on.partials = part_slot(h, RED_OP);
      on.sc = sc;
      on.check_done = 1;
      if (g.adjoint_bw) return bw_normal(h, on, s);
      return op_launch(OP_NORMAL, g, h->op, on, h->grid_op, s);
    });
    if (e != cudaSuccess) return e;
    if (h->fused) continue;   // the normal-matrix launch finished the CG step
    e = timed(h, s, KD_UPDATE,
              [&] { return cg_update_launch(g, handle_table(h, KD_UPDATE, b, pb), s); });
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int launches_per_iteration(const lfsr_handle* h) {
  // the backward warp adds its gather launch to the data block and each CG step
  const int bw = h->g.adjoint_bw ? 1 : 0;
  const int upd = h->fused ? 0 : 1;   // the fused normal-matrix launch holds the CG update
  const int init = h->fused_init ? 0 : 1;   // the fused data launch holds the initialisation
  return 2 + init + bw + (2 + upd + bw) * h->prm.cg_iters;
}

cudaError_t build_graph(lfsr_handle* h, int first_parity, int n, cudaGraphExec_t* out) {
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaError_t el = cudaSuccess;
  for (int i = 0; i < n && el == cudaSuccess; ++i)
    el = enqueue_iteration(h, (first_parity + i) & 1, h->cap_stream);
  e = cudaStreamEndCapture(h->cap_stream, &graph);
  if (el != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return el;
  }
  if (e != cudaSuccess) return e;
  e = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  return e;
}

int separable_factor(const std::vector<float>& K, int kb, float* kv, float* kh) {
  int am = 0, bm = 0;
  double best = -1.0;
  for (int a = 0; a < kb; ++a)
    for (int b = 0; b < kb; ++b)
      if (std::fabs((double)K[a * kb + b]) > best) {
        best = std::fabs((double)K[a * kb + b]);
        am = a;
        bm = b;
      }
  if (best <= 0.0) return 0;
  const double pivot = K[am * kb + bm];
  double err = 0.0;
  for (int a = 0; a < kb; ++a)
    for (int b = 0; b < kb; ++b) {
      const double rec = (double)K[a * kb + bm] * (double)K[am * kb + b] / pivot;
      err = std::fmax(err, std::fabs(rec - (double)K[a * kb + b]));
    }
  if (err > 1e-7 * best) return 0;
  for (int a = 0; a < kb; ++a) kv[a] = K[a * kb + bm];
  for (int b = 0; b < kb; ++b) kh[b] = (float)((double)K[am * kb + b] / pivot);
  return 1;
}

int validate(const lfsr_params* pr) {
  if (!pr) return fail(nullptr, LFSR_EINVAL, "params is NULL");
  if (pr->struct_size != sizeof(lfsr_params))
    return fail(nullptr, LFSR_EINVAL, "params->struct_size != sizeof(lfsr_params)");
  if (pr->U < 1 || pr->V < 1 || !(pr->U & 1) || !(pr->V & 1) || pr->U * pr->V > LFSR_MAX_VIEWS)
    return fail(nullptr, LFSR_EINVAL, "U and V must be odd, >= 1, with U*V <= 289");
  if (pr->H < 1 || pr->W < 1 || pr->H > 65536 || pr->W > 65536)
    return fail(nullptr, LFSR_EINVAL, "H and W must be in [1, 65536]");
  if (pr->scale < 1 || pr->scale > 4)
    return fail(nullptr, LFSR_EUNSUPPORTED, "scale must be 1, 2, 3 or 4");
  if ((long long)pr->scale * pr->H * pr->scale * pr->W > (1LL << 31))
    return fail(nullptr, LFSR_EINVAL, "HR image too large");
  if (pr->kb < 1 || !(pr->kb & 1) || pr->kb > LFSR_MAX_KB)
    return fail(nullptr, LFSR_EINVAL, "kb must be odd and <= 15");
  if (!pr->blur || !pr->disparity) return fail(nullptr, LFSR_EINVAL, "blur and disparity are required");
  if (!(pr->lambda1 >= 0.0) || !(pr->lambda2 >= 0.0) || !std::isfinite(pr->lambda1) ||
      !std::isfinite(pr->lambda2) || (pr->lambda1 == 0.0 && pr->lambda2 == 0.0))
    return fail(nullptr, LFSR_EINVAL, "lambda1, lambda2 must be finite, >= 0 and not both 0");
  if (!(pr->mu > 0.0) || !std::isfinite(pr->mu)) return fail(nullptr, LFSR_EINVAL, "mu must be > 0");
  if (pr->nltv_window < 3 || pr->nltv_window > 15 || !(pr->nltv_window & 1))
    return fail(nullptr, LFSR_EINVAL, "nltv_window must be odd in [3, 15]");
  if (pr->nltv_patch < 1 || pr->nltv_patch > 7 || !(pr->nltv_patch & 1))
    return fail(nullptr, LFSR_EINVAL, "nltv_patch must be odd in [1, 7]");
  if (!(pr->nltv_h > 0.0) || !std::isfinite(pr->nltv_h)) return fail(nullptr, LFSR_EINVAL, "nltv_h must be > 0");
  if (pr->cg_iters < 0 || pr->cg_iters > 10000) return fail(nullptr, LFSR_EINVAL, "cg_iters must be in [0, 10000]");
  if (pr->views) {
    if (pr->n_views < 1 || pr->n_views > pr->U * pr->V)
      return fail(nullptr, LFSR_EINVAL, "n_views must be in [1, U*V]");
    for (int j = 0; j < pr->n_views; ++j)
      if (pr->views[j] < 0 || pr->views[j] >= pr->U * pr->V || (j && pr->views[j] <= pr->views[j - 1]))
        return fail(nullptr, LFSR_EINVAL, "views must be strictly ascending grid indices in [0, U*V)");
  }
  if (!(pr->cg_tol >= 0.0) || !std::isfinite(pr->cg_tol)) return fail(nullptr, LFSR_EINVAL, "cg_tol must be >= 0");
  const int base = pr->precision & ~LFSR_KEEP_VIEWS_FP32;
  if (base != LFSR_FP32 && base != LFSR_FP16_STORAGE && base != LFSR_BF16_STORAGE)
    return fail(nullptr, LFSR_EINVAL,
                "precision must be LFSR_FP32, LFSR_FP16_STORAGE or LFSR_BF16_STORAGE, "
                "optionally | LFSR_KEEP_VIEWS_FP32");
  if (pr->adjoint != LFSR_ADJOINT_EXACT && pr->adjoint != LFSR_ADJOINT_BACKWARD_WARP)
    return fail(nullptr, LFSR_EINVAL, "adjoint must be LFSR_ADJOINT_EXACT or LFSR_ADJOINT_BACKWARD_WARP");
  if (pr->weights != LFSR_WEIGHTS_PATCH && pr->weights != LFSR_WEIGHTS_PAPER)
    return fail(nullptr, LFSR_EINVAL, "weights must be LFSR_WEIGHTS_PATCH or LFSR_WEIGHTS_PAPER");
  if (pr->weights == LFSR_WEIGHTS_PAPER) {
    const float sg[4] = {pr->sigma_s, pr->sigma_e, pr->sigma_o1, pr->sigma_o2};
    for (float v : sg)
      if (!(v >= 0.f) || !std::isfinite(v))
        return fail(nullptr, LFSR_EINVAL, "sigma_s, sigma_e, sigma_o1, sigma_o2 must be finite and >= 0");
  }
  if (base == LFSR_FP16_STORAGE && 1.0 / pr->mu > LFSR_FP16_MAX_INV_MU)
    return fail(nullptr, LFSR_EUNSUPPORTED,
                "LFSR_FP16_STORAGE needs 1/mu <= 8192 (duals are bounded by 1/mu)");
  return LFSR_OK;
}

}  // namespace

namespace {

// One-entry table in the handle's scratch slot `slot` for a standalone
// operator call (the host entry is copied at once; calls on the handle are
// stream-ordered).
cudaError_t scratch_table(lfsr_handle* h, int slot, const JobArgs& j, int red_slot, TableArgs* t) {
  cudaError_t e = cudaMemcpyAsync(h->jobs_scratch + slot, &j, sizeof(JobArgs),
                                  cudaMemcpyHostToDevice, h->stream);
  *t = TableArgs{};
  t->jobs = h->jobs_scratch + slot;
  t->unit_job = nullptr;
  t->n_jobs = 1;
  t->total_units = j.units;
  t->check_done = 0;
  t->partials = part_slot(h, red_slot);
  t->counter = h->counters + KD_NUM + slot;
  return e;
}

// Common fields of a standalone operator-call entry.
JobArgs standalone_job(const lfsr_handle* h) {
  JobArgs j{};
  j.H = h->g.H;
  j.W = h->g.W;
  j.Hh = h->g.Hh;
  j.Wh = h->g.Wh;
  j.U = h->g.U;
  j.V = h->g.V;
  j.disp = h->disp;
  j.theta = h->theta;
  j.occ = h->occ;
  j.sc = h->sc + 1;
  return j;
}

}  // namespace

// Cost-balanced split of operator units over the CTAs of a launch.  A unit
// is one (tile, view pair); a CTA takes a contiguous range (consecutive
// pairs of a tile share its staged source and its scatter accumulator).
// Units differ in cost with their tile's disparity content (the spread of
// the sub-pixel shifts decides how many scatter taps merge and how often
// shared-memory accesses collide), and a CTA pays for staging and flushing
// each tile it starts.  The even split leaves the slowest CTA well above
// the mean, and the launch (and, fused, every CG step's grid barrier) waits
// for the slowest one.
//
// The costs come from one timing launch on the even split: unit costs from
// the differences of the start clocks, the cost of a tile switch from the
// median excess of a range's tile-starting unit over the next unit.  The
// ranges are the contiguous split with the smallest maximum predicted cost
// (bisection on that maximum, greedy packing).
namespace {

struct SplitCost {
  std::vector<double> base;       // per unit, without tile staging
  const std::vector<char>* tile_start = nullptr;
  double sw = 0.0;                // staging and flushing one tile
};

// CTAs that greedy packing with at most `cap` per CTA needs (starts filled
// in when non-NULL).
int pack_units(const SplitCost& c, double cap, std::vector<int>* starts) {
  const int units = (int)c.base.size();
  int ctas = 0;
  double cur = 0.0;
  bool open = false;
  for (int u = 0; u < units; ++u) {
    const double add = c.base[u] + ((*c.tile_start)[u] ? c.sw : 0.0);
    if (!open || cur + add > cap) {
      if (starts) starts->push_back(u);
      ++ctas;
      open = true;
      cur = c.base[u] + c.sw;   // a range's first unit stages its tile
    } else {
      cur += add;
    }
  }
  return ctas;
}

}  // namespace

bool lfsr::split_by_unit_costs(const std::vector<double>& base, double sw,
                               const std::vector<char>& tile_start, int grid,
                               std::vector<int>* r0, double* max_cost, double* mean_cost) {
  const int units = (int)base.size();
  if (units < 1 || grid < 1 || (int)tile_start.size() != units) return false;
  SplitCost sc;
  sc.tile_start = &tile_start;
  sc.sw = sw;
  sc.base = base;
  double total = 0.0, lo = 0.0;
  for (int u = 0; u < units; ++u) {
    total += sc.base[u] + (tile_start[u] ? sc.sw : 0.0);
    lo = std::max(lo, sc.base[u] + sc.sw);
  }
  double hi = total + grid * sc.sw;
  for (int it = 0; it < 60 && hi - lo > 1e-6 * hi; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (pack_units(sc, mid, nullptr) <= grid) hi = mid;
    else lo = mid;
  }
  std::vector<int> starts;
  if (pack_units(sc, hi, &starts) > grid) return false;
  double bal_max = 0.0, bal_sum = 0.0;
  for (size_t r = 0; r < starts.size(); ++r) {
    const int ue = r + 1 < starts.size() ? starts[r + 1] : units;
    double v = sc.sw;
    for (int u = starts[r]; u < ue; ++u)
      v += sc.base[u] + (u > starts[r] && tile_start[u] ? sc.sw : 0.0);
    bal_max = std::max(bal_max, v);
    bal_sum += v;
  }
  *max_cost = bal_max;
  *mean_cost = bal_sum / grid;
  r0->assign((size_t)grid + 1, units);
  for (size_t r = 0; r < starts.size(); ++r) (*r0)[r] = starts[r];
  (*r0)[0] = 0;
  return true;
}

bool lfsr::split_by_cost(const std::vector<long long>& clk, int units, int grid,
                         const std::vector<char>& tile_start, std::vector<int>* r0,
                         double ratio[2], std::vector<double>* base_out, double* sw_out) {
  ratio[0] = ratio[1] = 0.0;
  if (units < 1 || grid < 1 || (int)tile_start.size() != units ||
      clk.size() != (size_t)units + grid)
    return false;
  std::vector<double> cost(units);
  std::vector<char> staged(units, 0);
  std::vector<double> even(grid, 0.0), excess;
  for (int b = 0; b < grid; ++b) {
    const int ub = (int)((long long)b * units / grid), ue = (int)((long long)(b + 1) * units / grid);
    for (int u = ub; u < ue; ++u) {
      const long long next = u + 1 < ue ? clk[u + 1] : clk[(size_t)units + b];
      cost[u] = next > clk[u] ? (double)(next - clk[u]) : 1.0;
      staged[u] = (u == ub || tile_start[u]) ? 1 : 0;
      even[b] += cost[u];
    }
    for (int u = ub; u + 1 < ue; ++u)
      if (staged[u] && !staged[u + 1]) excess.push_back(cost[u] - cost[u + 1]);
  }
  double sw = 0.0;
  if (!excess.empty()) {
    std::nth_element(excess.begin(), excess.begin() + excess.size() / 2, excess.end());
    sw = std::max(0.0, excess[excess.size() / 2]);
  }
  std::vector<double> base(units);
  for (int u = 0; u < units; ++u) base[u] = std::max(1.0, cost[u] - (staged[u] ? sw : 0.0));
  if (base_out) *base_out = base;
  if (sw_out) *sw_out = sw;
  double even_max = 0.0, even_sum = 0.0;
  for (double v : even) {
    even_max = std::max(even_max, v);
    even_sum += v;
  }
  ratio[0] = even_max / (even_sum / grid);
  double bal_max = 0.0, bal_mean = 0.0;
  if (!split_by_unit_costs(base, sw, tile_start, grid, r0, &bal_max, &bal_mean)) return false;
  ratio[1] = bal_max / bal_mean;
  if (!(bal_max < 0.99 * even_max)) {   // not worth a change: the even split stays
    ratio[1] = ratio[0];
    return false;
  }
  return true;
}

namespace {

// The single-light-field operator launches of h: a timing launch of the
// normal-matrix kernel after a warm-up one (P[0] is zero, Q is scratch, the
// clocks go to R, all unused until the first load), then the balanced
// ranges when they beat the even split.
cudaError_t balance_operator_units(lfsr_handle* h) {
  const int units = h->op_units, grid = h->grid_op;
  const size_t bytes = (size_t)(units + grid) * sizeof(long long);
  // nothing to balance with fewer than two units per CTA (R: 8-byte aligned)
  if (!h->fused || units < 2 * grid || bytes > h->p * sizeof(float)) return cudaSuccess;
  long long* clk = reinterpret_cast<long long*>(h->R);
  JobArgs j = make_job(h, KD_NORMAL, 0, 0, 0);
  j.fuse = 0;             // the operator part alone
  TableArgs t = handle_table(h, KD_NORMAL, 0, 0);
  t.cta_unit0 = nullptr;  // the even split
  t.check_done = 0;
  t.unit_clock = clk;     // timing launches leave the scalars alone
  cudaError_t e = fast_launch(OP_NORMAL, h->g, h->op, t, grid, h->stream, &j);   // warm-up
  if (e == cudaSuccess) e = fast_launch(OP_NORMAL, h->g, h->op, t, grid, h->stream, &j);
  std::vector<long long> c((size_t)units + grid);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c.data(), clk, bytes, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return e;
  const int upt = std::max(1, units / std::max(1, h->op.n_tiles));
  std::vector<char> tile_start(units);
  for (int u = 0; u < units; ++u) tile_start[u] = u % upt == 0;
  std::vector<int> r0;
  if (!split_by_cost(c, units, grid, tile_start, &r0, h->op_split, &h->unit_cost,
                     &h->unit_cost_tile))
    return cudaSuccess;
  e = dalloc(h, &h->cta_unit0, (size_t)grid + 1);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->cta_unit0, r0.data(), r0.size() * sizeof(int), cudaMemcpyHostToDevice,
                        h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);   // r0 is a local buffer
  return e;
}

}  // namespace

int lfsr::geom_from_params(const lfsr_params* pr, Geom* out) {
  int rc = validate(pr);
  if (rc != LFSR_OK) return rc;
  const int Hh = pr->scale * pr->H, Wh = pr->scale * pr->W;
  const size_t p = (size_t)Hh * Wh;
  std::vector<float> K(pr->blur, pr->blur + (size_t)pr->kb * pr->kb);
  if (!finite_all(K.data(), K.size()) || !finite_all(pr->disparity, p))
    return fail(nullptr, LFSR_EINVAL, "blur or disparity has non-finite values");
  if (pr->weights == LFSR_WEIGHTS_PAPER && pr->proj_err && !finite_all(pr->proj_err, p))
    return fail(nullptr, LFSR_EINVAL, "proj_err has non-finite values");
  const size_t n_views = pr->views ? (size_t)pr->n_views : (size_t)pr->U * pr->V;
  if (pr->disparity_views && !finite_all(pr->disparity_views, n_views * p))
    return fail(nullptr, LFSR_EINVAL, "disparity_views has non-finite values");
  Geom& g = *out;
  g = Geom{};
  g.U = pr->U;
  g.V = pr->V;
  g.sk = pr->views ? pr->n_views : pr->U * pr->V;
  g.H = pr->H;
  g.W = pr->W;
  g.Hh = Hh;
  g.Wh = Wh;
  g.zeta = pr->scale;
  g.kb = pr->kb;
  g.r = (pr->kb - 1) / 2;
  for (int i = 0; i < pr->kb * pr->kb; ++i) g.k2[i] = K[i];
  g.separable = separable_factor(K, pr->kb, g.kv, g.kh);
  double max_disp = 0.0;
  for (size_t i = 0; i < p; ++i) max_disp = std::fmax(max_disp, std::fabs((double)pr->disparity[i]));
  g.S = shift_bound(max_disp, pr->U, pr->V);
  g.warp_views = pr->disparity_views ? 1 : 0;
  g.adjoint_bw = pr->adjoint == LFSR_ADJOINT_BACKWARD_WARP ? 1 : 0;
  if (pr->disparity_views) {
    // W_k reads omega_k: the shift bound covers every per-view map too
    double mv = 0.0;
    for (size_t i = 0; i < n_views * p; ++i) mv = std::fmax(mv, std::fabs((double)pr->disparity_views[i]));
    const int sv = shift_bound(mv, pr->U, pr->V);
    if (sv > g.S) g.S = sv;
  }
  // angular offsets of the views of the data (the grid, or the listed subset)
  for (int j = 0; j < g.sk; ++j) {
    const int k = pr->views ? pr->views[j] : j;
    g.tu[j] = (float)((k % pr->U) - 0.5 * (pr->U - 1));
    g.tv[j] = (float)((k / pr->U) - 0.5 * (pr->V - 1));
  }
  g.win_r = (pr->nltv_window - 1) / 2;
  g.patch_r = (pr->nltv_patch - 1) / 2;
  g.sh = (pr->nltv_window * pr->nltv_window - 1) / 2;
  {
    int n = 0;
    for (int a = -g.win_r; a <= g.win_r && n < g.sh; ++a)
      for (int b = -g.win_r; b <= g.win_r && n < g.sh; ++b) {
        g.di[n] = (int8_t)a;
        g.dj[n] = (int8_t)b;
        ++n;
      }
  }
  g.inv_h2 = (float)(1.0 / (pr->nltv_h * pr->nltv_h));
  g.inv_np = (float)(1.0 / (double)(pr->nltv_patch * pr->nltv_patch));
  g.wscheme = pr->weights == LFSR_WEIGHTS_PAPER ? WS_PAPER : WS_PATCH;
  if (g.wscheme == WS_PAPER) {
    // no patches; the x halo of one pixel feeds the edge factor's central
    // differences
    g.patch_r = 1;
    g.inv_np = 1.f / 9.f;
    g.inv_sig_s = pr->sigma_s > 0.f ? (float)(1.0 / pr->sigma_s) : 0.f;
    g.inv_sig_e = pr->sigma_e > 0.f ? (float)(1.0 / pr->sigma_e) : 0.f;
  }
  g.lambda1 = (float)pr->lambda1;
  g.lambda2 = (float)pr->lambda2;
  g.mu = (float)pr->mu;
  g.cA = (float)(pr->lambda2 + 0.5 * pr->mu * pr->lambda1 * pr->lambda1);
  g.thr = (float)(1.0 / pr->mu);
  g.tau = pr->cg_tol;
  {
    const int base = pr->precision & ~LFSR_KEEP_VIEWS_FP32;
    g.st = base == LFSR_FP16_STORAGE ? ST_F16 : base == LFSR_BF16_STORAGE ? ST_BF16 : ST_F32;
    g.st_y = (pr->precision & LFSR_KEEP_VIEWS_FP32) ? ST_F32 : g.st;
  }
  g.wait_ns = LFSR_DEFAULT_WAIT_NS;
  g.wait_unreachable = 0;
  return LFSR_OK;
}

int lfsr::shift_bound(double max_abs_disparity, int U, int V) {
  const double max_theta = 0.5 * (double)((U > V ? U : V) - 1);
  return (int)std::ceil(max_abs_disparity * max_theta);
}

void lfsr::set_thread_error(const char* msg) { t_err = msg; }

bool lfsr::fault_alloc() {
  static std::mutex mu;
  static std::string spec;
  static long long count = 0;
  const char* env = std::getenv("LFSR_FAULT");
  const std::string cur = env ? env : "";
  std::lock_guard<std::mutex> lock(mu);
  if (cur != spec) {   // a new setting starts a new count
    spec = cur;
    count = 0;
  }
  if (cur.compare(0, 5, "alloc") != 0) return false;
  if (cur.size() == 5) return true;
  if (cur[5] != ':') return false;
  const long long k = std::atoll(cur.c_str() + 6);
  ++count;
  return k >= 1 && count == k;
}

int lfsr::handle_fail(lfsr_handle* h, int code, const std::string& msg) { return fail(h, code, msg); }
int lfsr::handle_cuda_fail(lfsr_handle* h, cudaError_t e, const char* what) {
  return cuda_fail(h, e, what);
}

int64_t lfsr::estimate_state_bytes(const lfsr_params* pr) {
  const int64_t Hh = (int64_t)pr->scale * pr->H, Wh = (int64_t)pr->scale * pr->W;
  const int64_t p = Hh * Wh, q = (int64_t)pr->H * pr->W;
  const int64_t sk = pr->views ? (int64_t)pr->n_views : (int64_t)pr->U * pr->V;
  const int64_t sh = ((int64_t)pr->nltv_window * pr->nltv_window - 1) / 2;
  const int64_t nA = sk * q, nS = 2 * sh * p;
  const int base = pr->precision & ~LFSR_KEEP_VIEWS_FP32;
  const int64_t es = base == LFSR_FP32 ? 4 : 2;
  const int64_t ey = (base == LFSR_FP32 || (pr->precision & LFSR_KEEP_VIEWS_FP32)) ? 4 : 2;
  const bool paper = pr->weights == LFSR_WEIGHTS_PAPER;
  const bool nlf = pr->nltv_window >= 3 && pr->nltv_window <= 7 && (paper || pr->nltv_patch <= 5);
  int64_t b = 4 * p              // disparity
              + ey * nA          // views
              + 2 * 4 * p        // x ping-pong
              + 2 * es * nA      // data duals
              + 2 * es * nS      // regulariser duals
              + 4 * 4 * p;       // P ping-pong, R, Q
  if (nlf) b += es * sh * p + 4 * p + 128; // stored weights, accumulated v, their tensor map
  if (paper) b += 4 * p;                    // occlusion factor
  if (pr->disparity_views) b += 4 * sk * p;  // per-view disparity maps
  if (pr->adjoint == LFSR_ADJOINT_BACKWARD_WARP) b += 4 * nA;   // LR buffer
  const int64_t nl_tiles = ((Hh + 31) / 32) * ((Wh + 31) / 32);
  b += (int64_t)RED_NUM * 8 * (nl_tiles > 4096 ? nl_tiles : 4096);   // reduction slots (bound)
  b += 2 * (int64_t)sizeof(DevScalars) + (4 * KD_NUM + 4) * (int64_t)sizeof(JobArgs) +
       (KD_NUM + 4) * 4 + 8 * sk;
  b += 4 * (4096 + 1);                      // balanced operator ranges (bound)
  return b;
}

int lfsr::kind_slot(int kind) {
  switch (kind) {
    case KD_NLW: return RED_DW_S;
    case KD_DATA: return RED_DW_A;
    case KD_NLA: return RED_NLTV;
    case KD_NORMAL: return RED_OP;
    default: return RED_PI;   // KD_INIT, KD_UPDATE
  }
}

int lfsr::kind_units(const lfsr_handle* h, int kind) {
  switch (kind) {
    case KD_NLW:
    case KD_NLA: return h->nl_units;
    case KD_DATA:
    case KD_NORMAL: return h->op_units;
    case KD_UPDATE: return h->upd_units;
    default: return h->vec_units;
  }
}

JobArgs lfsr::make_job(const lfsr_handle* h, int kind, int b, int pb, int unit0) {
  const Geom& g = h->g;
  const int nb = 1 - b;
  JobArgs j{};
  j.H = g.H;
  j.W = g.W;
  j.Hh = g.Hh;
  j.Wh = g.Wh;
  j.U = g.U;
  j.V = g.V;
  j.unit0 = unit0;
  j.units = kind_units(h, kind);
  j.disp = h->disp;
  j.theta = h->theta;
  j.occ = h->occ;
  j.sc = h->sc;
  switch (kind) {
    case KD_NLW:   // weights from x^(n-1), regulariser z/w-step, v += mu/2 S^T f
      j.tiles_x = h->nl_tiles_x;
      j.src = h->x[b];
      j.out = h->V;
      j.wS_old = h->wS[b];
      j.wS_new = h->wS[nb];
      j.wt = h->wt;
      break;
    case KD_DATA:  // data rows, v += A^T (...)
      j.tiles_x = h->op.tiles_x;
      j.view0 = 0;
      j.nviews = g.sk;
      j.scale = 1.f;
      j.src = h->x[b];
      j.out = h->nlf ? h->V : h->R;
      j.y = h->y;
      j.wA_old = h->wA[b];
      j.wA_new = h->wA[nb];
      if (h->fused_init) {  // ... then r = -v, v := 0, x' = x, pi (fused initialisation)
        j.fuse = 1;
        j.fchunk = h->fchunk;
        j.fpart = h->partials + (size_t)RED_PI * h->max_grid;
        j.vacc = h->V;
        j.rr = h->R;
        j.x_next = h->x[nb];
      }
      break;
    case KD_INIT:  // r = -v (v := 0 when accumulated), x' = x
      j.chunk = h->vec_chunk;
      j.out = h->R;
      j.vacc = h->V;
      j.src = h->x[b];
      j.x_next = h->x[nb];
      break;
    case KD_NLA:   // p = r + beta p_old, q = mu S^T W^2 S p
      j.tiles_x = h->nl_tiles_x;
      j.use_beta = 1;
      j.r = h->R;
      j.p_old = h->P[1 - pb];
      j.p_new = h->P[pb];
      j.out = h->Q;
      j.wt = h->wt;
      j.wt_map = h->nla_tma ? h->wt_map : nullptr;
      break;
    case KD_NORMAL:  // q += cA sum_k A_k^T A_k p
      j.tiles_x = h->op.tiles_x;
      j.view0 = 0;
      j.nviews = g.sk;
      j.scale = g.cA;
      j.src = h->P[pb];
      j.out = h->Q;
      if (h->fused) {  // ... then x += alpha p, r -= alpha q, pi', beta (fused CG step)
        j.fuse = 1;
        j.fchunk = h->fchunk;
        j.fpart = h->partials + (size_t)RED_PI * h->max_grid;
        j.p_old = h->P[pb];
        j.q = h->Q;
        j.rr = h->R;
        j.x_next = h->x[nb];
      }
      break;
    default:       // KD_UPDATE: x += alpha p, r -= alpha q
      j.chunk = h->upd_chunk;
      j.p_old = h->P[pb];
      j.q = h->Q;
      j.rr = h->R;
      j.x_next = h->x[nb];
      break;
  }
  return j;
}

extern "C" {

int lfsr_create(const lfsr_params* pr, void* cuda_stream, lfsr_handle** out) {
  return create_handle(pr, cuda_stream, out, true);
}

}  // extern "C"

int lfsr::create_handle(const lfsr_params* pr, void* cuda_stream, lfsr_handle** out,
                        bool balance) {
  if (!out) return fail(nullptr, LFSR_EINVAL, "out is NULL");
  *out = nullptr;
  Geom geom{};
  int rc = geom_from_params(pr, &geom);
  if (rc != LFSR_OK) return rc;
  const int Hh = geom.Hh, Wh = geom.Wh;
  const size_t p = (size_t)Hh * Wh, q = (size_t)pr->H * pr->W;

  lfsr_handle* h = new (std::nothrow) lfsr_handle();
  if (!h) return fail(nullptr, LFSR_ENOMEM, "host allocation failed");
  h->prm = *pr;
  h->prm.blur = nullptr;
  h->prm.disparity = nullptr;
  h->prm.views = nullptr;
  h->prm.proj_err = nullptr;
  h->prm.disparity_views = nullptr;
  if (pr->views) h->views.assign(pr->views, pr->views + pr->n_views);
  h->stream = (cudaStream_t)cuda_stream;
  h->g = geom;
  const Geom& g = h->g;
  h->esize = storage_bytes(g.st);
  h->esize_y = storage_bytes(g.st_y);
  h->p = p;
  h->q = q;
  h->nA = (size_t)g.sk * q;
  h->nS = (size_t)(2 * g.sh) * p;
  h->nSpair = h->nS;

  int optin = 0;
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
  if (e != cudaSuccess) {
    rc = cuda_fail(nullptr, e, "device query");
    delete h;
    return rc;
  }
  e = op_prepare(g, optin);
  if (e == cudaSuccess) e = nl_prepare(optin);
  if (e == cudaSuccess && nla2t_supported(g)) e = nla2t_prepare(optin);
  if (e == cudaSuccess && g.adjoint_bw) e = bw_prepare(optin);
  if (e != cudaSuccess) {
    rc = cuda_fail(nullptr, e, "kernel attributes");
    delete h;
    return rc;
  }
  // static shared memory of the kernels (reduction scratch) stays below 1 KB
  const int smem_limit = optin - 1024;
  if (op_plan(g, &h->op, h->sm_count, smem_limit) != cudaSuccess) {
    delete h;
    return fail(nullptr, LFSR_EUNSUPPORTED,
                "disparity * angular offset too large for the shared-memory tile");
  }
  if (nl_plan(g, &h->nl, smem_limit) != cudaSuccess) {
    delete h;
    return fail(nullptr, LFSR_EUNSUPPORTED, "NLTV window / patch too large");
  }
  if (g.adjoint_bw && bw_plan(g, &h->bw, smem_limit) != cudaSuccess) {
    delete h;
    return fail(nullptr, LFSR_EUNSUPPORTED,
                "disparity * angular offset too large for the backward-warp tile");
  }
  h->op_units = h->op.n_tiles * ((g.sk + FAST_VIEWS - 1) / FAST_VIEWS);
  h->grid_op = op_grid(h->op, h->op.fast ? h->op_units : h->op.n_tiles * g.sk, h->sm_count);
  h->grid_vec = h->sm_count * 2;
  h->nl_tiles_x = (Wh + NLF_TILE - 1) / NLF_TILE;
  h->nl_units = h->nl_tiles_x * ((Hh + NLF_TILE - 1) / NLF_TILE);
  {
    // vector kernels: two CTAs per SM (a whole number of waves), chunks of
    // a multiple of 32 pixels, at least 256
    size_t chunk = (p + (size_t)h->grid_vec - 1) / (size_t)h->grid_vec;
    chunk = (chunk + 31) / 32 * 32;
    if (chunk < 256) chunk = 256;
    h->vec_chunk = (int)chunk;
    h->vec_units = (int)((p + chunk - 1) / chunk);
    // the CG update streams four vectors with little work per pixel: one
    // CTA per SM (measured faster than two; the initialisation, with its 48
    // divergence loads per pixel, keeps two)
    size_t uc = (p + (size_t)h->sm_count - 1) / (size_t)h->sm_count;
    uc = (uc + 31) / 32 * 32;
    if (uc < 256) uc = 256;
    h->upd_chunk = (int)uc;
    h->upd_units = (int)((p + uc - 1) / uc);
    // the fused tails of the operator launches: grid_op CTAs cover the image
    size_t fc = (p + (size_t)h->grid_op - 1) / (size_t)h->grid_op;
    fc = (fc + 31) / 32 * 32;
    h->fchunk = (int)fc;
  }
  h->max_grid = h->grid_op;
  if (h->nl.n_tiles > h->max_grid) h->max_grid = h->nl.n_tiles;
  if (h->nl_units > h->max_grid) h->max_grid = h->nl_units;
  if (h->grid_vec > h->max_grid) h->max_grid = h->grid_vec;
  if (h->vec_units > h->max_grid) h->max_grid = h->vec_units;
  if (g.adjoint_bw && h->bw.n_tiles > h->max_grid) h->max_grid = h->bw.n_tiles;
  h->io_floats = h->nA > h->nS ? h->nA : h->nS;
  if (h->io_floats < p) h->io_floats = p;

  e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = dalloc(h, &h->disp, p);
  if (e == cudaSuccess) e = dalloc_st(h, &h->y, h->nA, h->esize_y);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
    e = dalloc(h, &h->x[i], p);
    if (e == cudaSuccess) e = dalloc_st(h, &h->wA[i], h->nA, h->esize);
    if (e == cudaSuccess) e = dalloc_st(h, &h->wS[i], h->nSpair, h->esize);
    if (e == cudaSuccess) e = dalloc(h, &h->P[i], p);
  }
  if (e == cudaSuccess) e = dalloc(h, &h->R, p);
  if (e == cudaSuccess) e = dalloc(h, &h->Q, p);
  h->nlf = nlf_supported(g);
  // the specialised operator kernel finishes each CG step itself (grid
  // barriers in a cooperative launch); the generic path keeps the separate
  // CG update launch
  h->fused = h->op.fast != 0;
  // ... and the data block the x-step initialisation, when v accumulates in
  // V (stored-weight NLTV path)
  h->fused_init = h->fused && h->nlf;
  if (e == cudaSuccess && h->nlf) e = dalloc_st(h, &h->wt, (size_t)g.sh * p, h->esize);
  // the NLTV apply stages the weight planes with TMA when their rows are
  // 16-byte multiples: its tensor map lives in device memory for the jobs
  if (e == cudaSuccess && h->nlf && nla2t_supported(g)) {
    unsigned char map[NLA_TMA_MAP_BYTES];
    if (nla2t_make_map(g, h->wt, map) == cudaSuccess) {
      e = dalloc(h, &h->wt_map, (size_t)NLA_TMA_MAP_BYTES);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->wt_map, map, NLA_TMA_MAP_BYTES, cudaMemcpyHostToDevice, h->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);   // map is a stack buffer
      h->nla_tma = e == cudaSuccess;
    }
  }
  if (e == cudaSuccess && h->nlf) e = dalloc(h, &h->V, p);
  if (e == cudaSuccess && h->nlf) e = cudaMemsetAsync(h->V, 0, p * sizeof(float), h->stream);
  if (e == cudaSuccess && g.wscheme == WS_PAPER) e = dalloc(h, &h->occ, p);
  if (e == cudaSuccess && g.warp_views) e = dalloc(h, &h->disp_views, (size_t)g.sk * p);
  if (e == cudaSuccess && g.adjoint_bw) e = dalloc(h, &h->hlr, h->nA);
  if (e == cudaSuccess) e = dalloc(h, &h->partials, (size_t)RED_NUM * h->max_grid);
  if (e == cudaSuccess) e = dalloc(h, &h->sc, 2);
  if (e == cudaSuccess) e = dalloc(h, &h->theta, (size_t)g.sk);
  if (e == cudaSuccess) {
    std::vector<float2> th(g.sk);
    for (int j = 0; j < g.sk; ++j) th[j] = make_float2(g.tu[j], g.tv[j]);
    e = cudaMemcpy(h->theta, th.data(), th.size() * sizeof(float2), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = dalloc(h, &h->jobs_dev, (size_t)4 * KD_NUM);
  if (e == cudaSuccess) e = dalloc(h, &h->jobs_scratch, 4);
  if (e == cudaSuccess) e = dalloc(h, &h->counters, (size_t)KD_NUM + 4);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->counters, 0, (KD_NUM + 4) * sizeof(unsigned int), h->stream);
  h->jobs_host.resize(4 * KD_NUM);
  for (int b = 0; b < 2; ++b)
    for (int pb = 0; pb < 2; ++pb)
      for (int kd = 0; kd < KD_NUM; ++kd)
        h->jobs_host[(2 * b + pb) * KD_NUM + kd] = make_job(h, kd, b, pb, 0);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->jobs_dev, h->jobs_host.data(), h->jobs_host.size() * sizeof(JobArgs),
                        cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->disp, pr->disparity, p * sizeof(float), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess && g.warp_views)
    e = cudaMemcpyAsync(h->disp_views, pr->disparity_views, (size_t)g.sk * p * sizeof(float),
                        cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess && g.wscheme == WS_PAPER) {
    // occlusion factor of the disparity map and the projection error (R
    // holds the projection error until the first load)
    const float* pe = nullptr;
    if (pr->proj_err && pr->sigma_o2 > 0.f) {
      e = cudaMemcpyAsync(h->R, pr->proj_err, p * sizeof(float), cudaMemcpyHostToDevice, h->stream);
      pe = h->R;
    }
    const double s1 = pr->sigma_o1, s2 = pr->sigma_o2;
    if (e == cudaSuccess)
      e = occlusion_launch(Hh, Wh, h->disp, pe, s1 > 0.0 ? (float)(0.5 / (s1 * s1)) : 0.f,
                           s2 > 0.0 ? (float)(0.5 / (s2 * s2)) : 0.f, h->occ, h->stream);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(h->sc, 0, 2 * sizeof(DevScalars), h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->P[0], 0, p * sizeof(float), h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->P[1], 0, p * sizeof(float), h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e == cudaSuccess && balance) e = balance_operator_units(h);
  if (e != cudaSuccess) {
    rc = cuda_fail(nullptr, e, "lfsr_create");
    free_all(h);
    delete h;
    return rc;
  }
  *out = h;
  return LFSR_OK;
}

extern "C" {

void lfsr_destroy(lfsr_handle* h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  free_all(h);
  delete h;
}

const char* lfsr_last_error(const lfsr_handle* h) { return h ? h->err.c_str() : t_err.c_str(); }

int lfsr_load(lfsr_handle* h, const float* lr_views, const float* x0, int mem) {
  NvtxRange range("lfsr_load (io: views and x0 in)");
  return load_state(h, lr_views, x0, mem, 0);
}

}  // extern "C"

int lfsr::load_state(lfsr_handle* h, const float* lr_views, const float* x0, int mem, int parity) {
  if (!h) return fail(nullptr, LFSR_EINVAL, "handle is NULL");
  if (!lr_views || !x0) return fail(h, LFSR_EINVAL, "lr_views and x0 are required");
  if (check_mem(h, mem)) return LFSR_EINVAL;
  const int b = parity & 1;
  CK(h, scalars_reset(h->sc, h->stream), "reset scalars");
  if (h->g.st_y == ST_F32) {
    CK(h, to_dev(h, (float*)h->y, lr_views, h->nA, mem), "upload views");
  } else {
    const float* src = lr_views;
    if (mem == LFSR_MEM_HOST) {
      CK(h, ensure_io(h), "staging buffer");
      CK(h, to_dev(h, h->io, lr_views, h->nA, mem), "upload views");
      src = h->io;
    }
    CK(h, to_storage(h->g.st_y, src, h->y, h->nA, h->sc, h->grid_vec, h->stream), "store views");
  }
  CK(h, to_dev(h, h->x[b], x0, h->p, mem), "upload x0");
  CK(h, cudaMemsetAsync(h->wA[b], 0, h->nA * h->esize, h->stream), "clear data duals");
  CK(h, cudaMemsetAsync(h->wS[b], 0, h->nSpair * h->esize, h->stream), "clear NLTV duals");
  if (h->V) CK(h, cudaMemsetAsync(h->V, 0, h->p * sizeof(float), h->stream), "clear v");
  h->parity = b;
  h->iters = 0;
  h->launches = 0;
  return LFSR_OK;
}

extern "C" {

int lfsr_iterate(lfsr_handle* h, int iterations) {
  NvtxRange range("lfsr_iterate (wz-step and x-step)");
  if (!h) return fail(nullptr, LFSR_EINVAL, "handle is NULL");
  if (iterations < 0) return fail(h, LFSR_EINVAL, "iterations must be >= 0");
  if (h->profiling) {
    for (int i = 0; i < iterations; ++i) {
      CK(h, enqueue_iteration(h, h->parity, h->stream), "iteration");
      h->parity ^= 1;
    }
  } else {
    int left = iterations;
    while (left > 0) {
      if (h->parity == 0 && left >= 2) {
        if (!h->graph_pair) CK(h, build_graph(h, 0, 2, &h->graph_pair), "capture");
        CK(h, cudaGraphLaunch(h->graph_pair, h->stream), "graph launch");
        left -= 2;
      } else {
        cudaGraphExec_t& gs = h->graph_single[h->parity];
        if (!gs) CK(h, build_graph(h, h->parity, 1, &gs), "capture");
        CK(h, cudaGraphLaunch(gs, h->stream), "graph launch");
        h->parity ^= 1;
        left -= 1;
      }
    }
  }
  h->iters += iterations;
  h->launches += (int64_t)iterations * launches_per_iteration(h);
  return LFSR_OK;
}

static int read_status(lfsr_handle* h, DevScalars* hs) {
  CK(h, cudaMemcpyAsync(hs, h->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, h->stream), "read scalars");
  CK(h, cudaStreamSynchronize(h->stream), "synchronize");
  if (hs->status == LFSR_EINVAL)
    return fail(h, LFSR_EINVAL, "a view or data-dual value given to the solver is not finite or outside the storage type's range");
  if (hs->status == LFSR_ETIMEOUT)
    return fail(h, LFSR_ETIMEOUT,
                "a grid barrier of the fused CG step gave up waiting (device wait limit reached)");
  if (hs->status != 0)
    return fail(h, hs->status, "non-finite or negative curvature in the CG x-step");
  return LFSR_OK;
}

int lfsr_get_x(lfsr_handle* h, float* x_out, int mem) {
  NvtxRange range("lfsr_get_x (io: x out)");
  if (!h) return fail(nullptr, LFSR_EINVAL, "handle is NULL");
  if (!x_out) return fail(h, LFSR_EINVAL, "x_out is NULL");
  if (check_mem(h, mem)) return LFSR_EINVAL;
  CK(h, from_dev(h, x_out, h->x[h->parity], h->p, mem), "download x");
  DevScalars hs;
  return read_status(h, &hs);
}

int lfsr_solve(lfsr_handle* h, const float* lr_views, int iterations, const float* x0,
               float* x_out, int mem) {
  NvtxRange range("lfsr_solve");
  int rc = lfsr_load(h, lr_views, x0, mem);
  if (rc) return rc;
  rc = lfsr_iterate(h, iterations);
  if (rc) return rc;
  return lfsr_get_x(h, x_out, mem);
}

int lfsr_stats(const lfsr_handle* hc, lfsr_stats_t* out) {
  lfsr_handle* h = const_cast<lfsr_handle*>(hc);
  if (!h) return fail(nullptr, LFSR_EINVAL, "handle is NULL");
  if (!out || out->struct_size != sizeof(lfsr_stats_t))
    return fail(h, LFSR_EINVAL, "out->struct_size != sizeof(lfsr_stats_t)");
  DevScalars hs;
  CK(h, cudaMemcpyAsync(&hs, h->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, h->stream), "read scalars");
  CK(h, cudaStreamSynchronize(h->stream), "synchronize");
  for (auto& ev : h->prof) {
    float ms = 0.f;
    CK(h, cudaEventElapsedTime(&ms, ev.a, ev.b), "event time");
    h->prof_ms[ev.cls] += ms;
    h->prof_n[ev.cls] += 1;
    cudaEventDestroy(ev.a);
    cudaEventDestroy(ev.b);
  }
  h->prof.clear();
  std::memset((char*)out + sizeof(uint32_t), 0, sizeof(lfsr_stats_t) - sizeof(uint32_t));
  out->iterations = h->iters;
  out->cg_steps = hs.cg_steps;
  out->status = hs.status;
  out->dual_change_sq = hs.dw2;
  out->cg_pi = hs.pi;
  out->state_bytes = h->state_bytes;
  out->launches = h->launches;
  out->op_split_even = h->op_split[0];
  out->op_split_balanced = h->op_split[1];
  for (int c = 0; c < NUM_CLASSES; ++c) {
    out->kernel_ms[c] = h->prof_ms[c];
    out->kernel_launches[c] = h->prof_n[c];
  }
  return LFSR_OK;
}

int64_t lfsr_estimate_state_bytes(const lfsr_params* params) {
  if (validate(params) != LFSR_OK) return -1;
  return estimate_state_bytes(params);
}

int lfsr_set_device_wait(lfsr_handle* h, int64_t limit_ns, int test_unreachable) {
  if (!h) return fail(nullptr, LFSR_EINVAL, "handle is NULL");
  if (limit_ns < 0) return fail(h, LFSR_EINVAL, "limit_ns must be >= 0");
  CK(h, cudaStreamSynchronize(h->stream), "synchronize");
  h->g.wait_ns = (unsigned long long)limit_ns;
  h->g.wait_unreachable = test_unreachable ? 1 : 0;
  // the captured iterations hold the old limit: capture again on next use
  if (h->graph_pair) cudaGraphExecDestroy(h->graph_pair);
  h->graph_pair = nullptr;
  for (auto& gs : h->graph_single) {
    if (gs) cudaGraphExecDestroy(gs);
    gs = nullptr;
  }
  return LFSR_OK;
}

int lfsr_set_profiling(lfsr_handle* h, int on) {
  if (!h) return fail(nullptr, LFSR_EINVAL, "handle is NULL");
  h->profiling = on != 0;
  for (int c = 0; c < 8; ++c) {
    h->prof_ms[c] = 0.0;
    h->prof_n[c] = 0;
  }
  return LFSR_OK;
}

int lfsr_set_state(lfsr_handle* h, const float* x, const float* wA, const float* wS, int mem) {
  if (!h) return fail(nullptr, LFSR_EINVAL, "handle is NULL");
  if (check_mem(h, mem)) return LFSR_EINVAL;
  CK(h, ensure_io(h), "staging buffer");
  const int b = h->parity;
  if (x) CK(h, to_dev(h, h->x[b], x, h->p, mem), "set x");
  if (wA && h->g.st == ST_F32) CK(h, to_dev(h, (float*)h->wA[b], wA, h->nA, mem), "set data duals");
  if (wA && h->g.st != ST_F32) {
    const float* src = wA;
    if (mem == LFSR_MEM_HOST) {
      CK(h, to_dev(h, h->io, wA, h->nA, mem), "set data duals");
      src = h->io;
    }
    CK(h, to_storage(h->g.st, src, h->wA[b], h->nA, h->sc, h->grid_vec, h->stream), "store duals");
  }
  if (wS) {
    CK(h, to_dev(h, h->io, wS, h->nS, mem), "set NLTV duals");
    CK(h, pair_from_canonical(h->g, h->io, h->wS[b], h->stream), "dual layout");
  }
  return LFSR_OK;
}

int lfsr_get_state(lfsr_handle* h, float* x, float* wA, float* wS, int mem) {
  if (!h) return fail(nullptr, LFSR_EINVAL, "handle is NULL");
  if (check_mem(h, mem)) return LFSR_EINVAL;
  CK(h, ensure_io(h), "staging buffer");
  const int b = h->parity;
  if (x) CK(h, from_dev(h, x, h->x[b], h->p, mem), "get x");
  if (wA && h->g.st == ST_F32) CK(h, from_dev(h, wA, (const float*)h->wA[b], h->nA, mem), "get data duals");
  if (wA && h->g.st != ST_F32) {
    CK(h, from_storage(h->g.st, h->wA[b], h->io, h->nA, h->grid_vec, h->stream), "load duals");
    CK(h, from_dev(h, wA, h->io, h->nA, mem), "get data duals");
  }
  if (wS) {
    CK(h, pair_to_canonical(h->g, h->wS[b], h->io, h->stream), "dual layout");
    CK(h, from_dev(h, wS, h->io, h->nS, mem), "get NLTV duals");
  }
  DevScalars hs;
  return read_status(h, &hs);
}

int lfsr_apply_A(lfsr_handle* h, int view, const float* x, float* out, int mem) {
  if (!h) return fail(nullptr, LFSR_EINVAL, "handle is NULL");
  if (!x || !out) return fail(h, LFSR_EINVAL, "x and out are required");
  if (check_mem(h, mem)) return LFSR_EINVAL;
  CK(h, ensure_io(h), "staging buffer");
  if (view < -1 || view >= h->g.sk) return fail(h, LFSR_EINVAL, "view out of range");
  const int nv = view < 0 ? h->g.sk : 1;
  const float* xs = x;
  float* os = out;
  if (mem == LFSR_MEM_HOST) {
    CK(h, to_dev(h, h->Q, x, h->p, mem), "upload x");
    xs = h->Q;
    os = h->io;
  }
  if (h->op.fast) {
    JobArgs j = standalone_job(h);
    j.tiles_x = h->op.tiles_x;
    j.view0 = view < 0 ? 0 : view;
    j.nviews = nv;
    j.units = h->op.n_tiles * ((nv + FAST_VIEWS - 1) / FAST_VIEWS);
    j.src = xs;
    j.out = os - (size_t)j.view0 * h->q;   // the kernel indexes out by view
    TableArgs t;
    CK(h, scratch_table(h, 0, j, RED_OP, &t), "operator table");
    CK(h, fast_launch(OP_FWD, h->g, h->op, t, op_grid(h->op, j.units, h->sm_count), h->stream, &j),
       "apply A");
  } else {
    OpArgs a{};
    a.src = xs;
    set_warp_maps(h, &a);
    a.out = os - (size_t)(view < 0 ? 0 : view) * h->q;  // kernel indexes out by view
    a.view0 = view < 0 ? 0 : view;
    a.nviews = nv;
    a.units = h->op.n_tiles * nv;
    a.sc = h->sc + 1;
    CK(h, op_launch(OP_FWD, h->g, h->op, a, op_grid(h->op, a.units, h->sm_count), h->stream),
       "apply A");
  }
  if (mem == LFSR_MEM_HOST) CK(h, from_dev(h, out, h->io, (size_t)nv * h->q, mem), "download");
  CK(h, cudaStreamSynchronize(h->stream), "synchronize");
  return LFSR_OK;
}

int lfsr_apply_AT(lfsr_handle* h, int view, const float* gin, float* out, int mem) {
  if (!h) return fail(nullptr, LFSR_EINVAL, "handle is NULL");
  if (!gin || !out) return fail(h, LFSR_EINVAL, "g and out are required");
  if (check_mem(h, mem)) return LFSR_EINVAL;
  CK(h, ensure_io(h), "staging buffer");
  if (view < -1 || view >= h->g.sk) return fail(h, LFSR_EINVAL, "view out of range");
  const int nv = view < 0 ? h->g.sk : 1;
  const float* gs = gin;
  float* os = out;
  if (mem == LFSR_MEM_HOST) {
    CK(h, to_dev(h, h->io, gin, (size_t)nv * h->q, mem), "upload g");
    gs = h->io;
    os = h->Q;
  }
  CK(h, cudaMemsetAsync(os, 0, h->p * sizeof(float), h->stream), "clear out");
  if (h->op.fast) {
    JobArgs j = standalone_job(h);
    j.tiles_x = h->op.tiles_x;
    j.view0 = view < 0 ? 0 : view;
    j.nviews = nv;
    j.units = h->op.n_tiles * ((nv + FAST_VIEWS - 1) / FAST_VIEWS);
    j.scale = 1.f;
    j.src = gs - (size_t)j.view0 * h->q;
    j.out = os;
    TableArgs t;
    CK(h, scratch_table(h, 0, j, RED_OP, &t), "operator table");
    CK(h, fast_launch(OP_ADJ, h->g, h->op, t, op_grid(h->op, j.units, h->sm_count), h->stream, &j),
       "apply A^T");
  } else {
    OpArgs a{};
    a.src = gs - (size_t)(view < 0 ? 0 : view) * h->q;
    set_warp_maps(h, &a);
    a.out = os;
    a.scale = 1.f;
    a.view0 = view < 0 ? 0 : view;
    a.nviews = nv;
    a.units = h->op.n_tiles * nv;
    a.sc = h->sc + 1;
    if (h->g.adjoint_bw) {
      // the solver's A_k^*: the backward warp by the reference map
      a.disp = h->disp;
      a.disp_stride = 0;
      CK(h, bw_launch(h->g, h->bw, a, h->stream), "apply A^*");
    } else {
      CK(h, op_launch(OP_ADJ, h->g, h->op, a, op_grid(h->op, a.units, h->sm_count), h->stream),
         "apply A^T");
    }
  }
  if (mem == LFSR_MEM_HOST) CK(h, from_dev(h, out, h->Q, h->p, mem), "download");
  CK(h, cudaStreamSynchronize(h->stream), "synchronize");
  return LFSR_OK;
}

int lfsr_weights(lfsr_handle* h, const float* x, float* w, int mem) {
  if (!h) return fail(nullptr, LFSR_EINVAL, "handle is NULL");
  if (!x || !w) return fail(h, LFSR_EINVAL, "x and w are required");
  if (check_mem(h, mem)) return LFSR_EINVAL;
  CK(h, ensure_io(h), "staging buffer");
  const float* xs = x;
  float* ws = w;
  if (mem == LFSR_MEM_HOST) {
    CK(h, to_dev(h, h->Q, x, h->p, mem), "upload x");
    xs = h->Q;
    ws = h->io;
  }
  CK(h, cudaMemsetAsync(ws, 0, h->nS * sizeof(float), h->stream), "clear w");
  if (h->nlf && h->g.wscheme == WS_PATCH) {
    JobArgs j = standalone_job(h);
    j.tiles_x = h->nl_tiles_x;
    j.units = h->nl_units;
    j.src = xs;
    j.wt = h->wt;
    TableArgs t;
    CK(h, scratch_table(h, 0, j, RED_NLTV, &t), "NLTV table");
    CK(h, nlw2_launch(0, h->g, t, h->stream), "weights");
    CK(h, weights_to_canonical(h->g, h->wt, ws, h->stream), "weights layout");
  } else {
    // the paper's directed weights (the stored edge weights hold their
    // root mean square per edge), or windows beyond the stored-weight path
    NlArgs a{};
    a.x = xs;
    a.occ = h->occ;
    a.out = ws;
    a.sc = h->sc + 1;
    CK(h, nl_launch(NL_WEIGHTS, h->g, h->nl, a, h->stream), "weights");
  }
  if (mem == LFSR_MEM_HOST) CK(h, from_dev(h, w, h->io, h->nS, mem), "download");
  CK(h, cudaStreamSynchronize(h->stream), "synchronize");
  return LFSR_OK;
}

int lfsr_apply_normal(lfsr_handle* h, const float* xw, const float* p, float* qo, double* pMp,
                      int mem) {
  if (!h) return fail(nullptr, LFSR_EINVAL, "handle is NULL");
  if (!xw || !p || !qo) return fail(h, LFSR_EINVAL, "xw, p and q are required");
  if (check_mem(h, mem)) return LFSR_EINVAL;
  CK(h, ensure_io(h), "staging buffer");
  const float* xs = xw;
  const float* ps = p;
  float* qs = qo;
  if (mem == LFSR_MEM_HOST) {
    CK(h, to_dev(h, h->io, xw, h->p, mem), "upload xw");
    CK(h, to_dev(h, h->io + h->p, p, h->p, mem), "upload p");
    xs = h->io;
    ps = h->io + h->p;
    qs = h->io + 2 * h->p;
  }
  DevScalars* sc = h->sc + 1;
  if (h->nlf) {
    JobArgs jw = standalone_job(h);   // weights of xw
    jw.tiles_x = h->nl_tiles_x;
    jw.units = h->nl_units;
    jw.src = xs;
    jw.wt = h->wt;
    JobArgs ja = jw;                  // q := mu S^T W^2 S p
    ja.src = nullptr;
    ja.use_beta = 0;
    ja.p_old = ps;
    ja.out = qs;
    TableArgs tw, ta;
    CK(h, scratch_table(h, 0, jw, RED_NLTV, &tw), "NLTV table");
    CK(h, scratch_table(h, 1, ja, RED_NLTV, &ta), "NLTV table");
    CK(h, nlw2_launch(0, h->g, tw, h->stream), "normal (weights)");
    CK(h, nla2_launch(h->g, ta, h->stream), "normal (NLTV part)");
  } else {
    NlArgs na{};
    na.x = xs;
    na.occ = h->occ;
    na.p_old = ps;
    na.out = qs;
    na.partials = part_slot(h, RED_NLTV);
    na.sc = sc;
    CK(h, nl_launch(NL_APPLY, h->g, h->nl, na, h->stream), "normal (NLTV part)");
  }
  if (h->op.fast) {
    JobArgs j = standalone_job(h);
    j.tiles_x = h->op.tiles_x;
    j.view0 = 0;
    j.nviews = h->g.sk;
    j.units = h->op_units;
    j.scale = h->g.cA;
    j.src = ps;
    j.out = qs;
    TableArgs t;
    CK(h, scratch_table(h, 2, j, RED_OP, &t), "operator table");
    CK(h, fast_launch(OP_NORMAL, h->g, h->op, t, h->grid_op, h->stream, &j),
       "normal (operator part)");
  } else {
    OpArgs on{};
    on.src = ps;
    set_warp_maps(h, &on);
    on.out = qs;
    on.scale = h->g.cA;
    on.view0 = 0;
    on.nviews = h->g.sk;
    on.units = h->op.n_tiles * h->g.sk;
    on.partials = part_slot(h, RED_OP);
    on.sc = sc;
    if (h->g.adjoint_bw) {
      CK(h, bw_normal(h, on, h->stream), "normal (operator part)");
    } else {
      CK(h, op_launch(OP_NORMAL, h->g, h->op, on, h->grid_op, h->stream), "normal (operator part)");
    }
  }
  if (mem == LFSR_MEM_HOST) CK(h, from_dev(h, qo, qs, h->p, mem), "download q");
  DevScalars hs;
  CK(h, cudaMemcpyAsync(&hs, sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, h->stream), "read");
  CK(h, cudaStreamSynchronize(h->stream), "synchronize");
  if (pMp) *pMp = hs.pAp;
  return LFSR_OK;
}

}  // extern "C"
