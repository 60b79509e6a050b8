// Private to liblfsr: the solver state of one light field (lfsr_handle) and
// the helpers that the batch entry points share with the single-light-field
// ones.
#pragma once

#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "lfsr.h"
#include "lfsr_internal.cuh"

namespace lfsr {

// NVTX range for the host-side phases (the paper splits a solve's time into
// io, wz-step and x-step, Sec. 6): visible in a profiler's timeline, a no-op
// without one attached.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
// Names of the launch classes (KD_*) in the profiling mode's NVTX ranges.
inline const char* kind_name(int kind) {
  static const char* names[] = {"nltv_block (z/w-step, regulariser rows)",
                                "data_block (z/w-step, data rows; x-step init when fused)",
                                "cg_init (x-step)", "nltv_apply (x-step, S^T W^2 S p)",
                                "normal_apply (x-step, A^T A p; CG update when fused)",
                                "cg_update (x-step)"};
  return kind >= 0 && kind < 6 ? names[kind] : "lfsr";
}

struct ProfEvent {
  int cls;
  cudaEvent_t a, b;
  int grp;   // operator group of a batch launch (0 otherwise)
};

// Launch kinds of one ADMM iteration, in schedule order (also the profiling
// classes of lfsr_stats_t): NLTV block, data block, x-step init, then per CG
// step NLTV apply, normal-matrix operator, CG update.
enum { KD_NLW = 0, KD_DATA = 1, KD_INIT = 2, KD_NLA = 3, KD_NORMAL = 4, KD_UPDATE = 5, KD_NUM = 6 };

}  // namespace lfsr

struct lfsr_handle {
  lfsr_params prm{};
  lfsr::Geom g{};
  lfsr::OpPlan op{};
  lfsr::NlPlan nl{};
  cudaStream_t stream = nullptr;      // caller's stream
  cudaStream_t cap_stream = nullptr;  // private stream used for graph capture
  int device = 0, sm_count = 0;
  size_t p = 0, q = 0, nA = 0, nS = 0, nSpair = 0;
  int grid_op = 0, grid_vec = 0, max_grid = 0;
  // device buffers
  float* disp = nullptr;
  float* occ = nullptr;                // paper weights: occlusion factor o (HR)
  float* disp_views = nullptr;         // per-view disparity maps omega_k (s_k x p)
  float* hlr = nullptr;                // backward warp: LR buffer of h_k (s_k x q)
  lfsr::BwPlan bw{};                   // backward warp: plan of its gather kernel
  float2* theta = nullptr;             // angular offsets of the data's views
  std::vector<int32_t> views;          // the listed subset (empty: the grid)
  float* x[2] = {nullptr, nullptr};
  float* R = nullptr;   // v, then the CG residual r
  float* P[2] = {nullptr, nullptr};
  float* Q = nullptr;
  float* V = nullptr;   // accumulated v of the z/w-step (stored-weight NLTV path; zero
                        // between iterations: the x-step initialisation clears it)
  // streams in the storage kind g.st (float, half or bfloat16), esize bytes
  // each; the views in kind g.st_y (esize_y bytes)
  size_t esize = 4, esize_y = 4;
  void* y = nullptr;
  void* wA[2] = {nullptr, nullptr};
  void* wS[2] = {nullptr, nullptr};
  void* wt = nullptr;   // stored NLTV edge weights [s_d/2][p] (when supported)
  bool nlf = false;
  unsigned char* wt_map = nullptr;   // tensor map of the weight planes (TMA NLTV apply)
  bool nla_tma = false;              // the NLTV apply stages the weights with TMA
  bool fused = false;   // the normal-matrix launch finishes each CG step (no update launch)
  bool fused_init = false;   // the data launch does the x-step initialisation (no init launch)
  float* io = nullptr;  // staging for host <-> device and layout conversion
  size_t io_floats = 0;
  double* partials = nullptr;
  lfsr::DevScalars* sc = nullptr;  // [0] solver, [1] standalone operator calls
  int64_t state_bytes = 0;
  // schedule state
  int parity = 0;
  int iters = 0;
  int64_t launches = 0;
  cudaGraphExec_t graph_pair = nullptr;     // iterations at parity 0 then 1
  cudaGraphExec_t graph_single[2] = {nullptr, nullptr};
  // table-driven launches (specialised operator, stored-weight NLTV, CG
  // vector kernels): one JobArgs per (iteration parity b, CG direction
  // parity pb, kind), entry (2 b + pb) KD_NUM + kind
  std::vector<lfsr::JobArgs> jobs_host;     // host copies (by-value operator launches)
  lfsr::JobArgs* jobs_dev = nullptr;
  lfsr::JobArgs* jobs_scratch = nullptr;    // standalone operator calls: 4 entries
  unsigned int* counters = nullptr;         // arrival counters: KD_NUM + 4
  int nl_tiles_x = 0, nl_units = 0;         // 32 x 32 NLTV tiles
  int op_units = 0;                         // (64 x 64 tile, view pair) units
  int vec_chunk = 0, vec_units = 0;         // HR pixels per vector-kernel CTA, CTAs
  int upd_chunk = 0, upd_units = 0;         // the same for the CG update (one CTA per SM)
  int fchunk = 0;                           // HR pixels per CTA of the fused operator tails
  int* cta_unit0 = nullptr;                 // cost-balanced operator ranges (grid_op + 1), or NULL
  double op_split[2] = {0.0, 0.0};          // max / mean CTA cost: even split, balanced ranges
  // measured cost of each operator unit (SM clocks, without tile staging) and
  // of staging a tile, from the timing launch at creation (empty when not
  // measured); a batch that cannot time its own launches splits with them
  std::vector<double> unit_cost;
  double unit_cost_tile = 0.0;
  bool profiling = false;
  std::vector<lfsr::ProfEvent> prof;
  double prof_ms[8] = {0};
  int64_t prof_n[8] = {0};
  std::string err = "no error";
};

namespace lfsr {

// JobArgs of launch `kind` of an iteration at parity b (reads state b,
// writes state 1 - b) and CG direction parity pb, for a table whose first
// unit of this light field is unit0.
JobArgs make_job(const lfsr_handle* h, int kind, int b, int pb, int unit0);
// lfsr_create; balance: measure the operator units' costs and split them
// over the CTAs by cost (single-light-field launches; light fields that run
// only inside batch tables skip it).
int create_handle(const lfsr_params* params, void* cuda_stream, lfsr_handle** out, bool balance);
// Contiguous split of `units` operator units over `grid` CTAs with the
// smallest maximum measured cost.  clk: the clocks of one timing launch on
// the even split (units start clocks, then grid range-end clocks);
// tile_start[u]: unit u is the first of its tile.  ratio: the slowest CTA's
// cost over the mean, for the even split and for the chosen split.  True,
// with r0 = the grid + 1 range starts, when the split beats the even one by
// more than 1 %.
bool split_by_cost(const std::vector<long long>& clk, int units, int grid,
                   const std::vector<char>& tile_start, std::vector<int>* r0, double ratio[2],
                   std::vector<double>* base_out = nullptr, double* sw_out = nullptr);
// The same split from per-unit costs (base[u], without tile staging) and
// the cost sw of staging a tile: r0 = the grid + 1 range starts, the
// slowest range's cost and the mean range cost.  False when the units do
// not fit `grid` ranges.
bool split_by_unit_costs(const std::vector<double>& base, double sw,
                         const std::vector<char>& tile_start, int grid, std::vector<int>* r0,
                         double* max_cost, double* mean_cost);
// Work units of a launch kind for this light field.
int kind_units(const lfsr_handle* h, int kind);
// Reduction slot (RED_*) of a launch kind.
int kind_slot(int kind);
// lfsr_load into state `parity` (x[parity] := x0, duals[parity] := 0).
int load_state(lfsr_handle* h, const float* lr_views, const float* x0, int mem, int parity);
// Upper bound of the device bytes lfsr_create allocates for params (the
// staging buffer excluded: it is allocated on first host transfer).
int64_t estimate_state_bytes(const lfsr_params* params);
// Batches: an empty batch over light fields owned by someone else; its
// launch structure rebuilt over `jobs` (see batch.cu); its state parity.
lfsr_batch* batch_new_shared(cudaStream_t stream);
cudaError_t batch_assign(lfsr_batch* b, const std::vector<lfsr_handle*>& jobs);
int batch_parity(const lfsr_batch* b);
// Solver parameters all light fields of one batch or server must share.
bool same_solver(const lfsr_params& a, const lfsr_params& c);
// Validates params (sizes, parameters, finiteness of the blur and of every
// disparity map) and fills the geometry and solver constants every kernel
// takes; the message of a failure goes to the thread (lfsr_last_error(NULL)).
int geom_from_params(const lfsr_params* params, Geom* g);
// Integer bound S on |theta_k * omega| over a U x V grid (the halo of the
// warp) for a disparity map whose largest magnitude is max_abs_disparity.
int shift_bound(double max_abs_disparity, int U, int V);
// Host-side allocation-fault injection (LFSR_FAULT=alloc or alloc:K, see
// lfsr.h): true when the library's next device allocation is to fail.
bool fault_alloc();
// Records an error on h (and the thread) and returns code.
int handle_fail(lfsr_handle* h, int code, const std::string& msg);
int handle_cuda_fail(lfsr_handle* h, cudaError_t e, const char* what);

}  // namespace lfsr
