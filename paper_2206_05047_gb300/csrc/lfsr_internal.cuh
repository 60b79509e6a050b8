// Internal declarations shared by the CUDA translation units of liblfsr.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define LFSR_MAX_KB 15
#define LFSR_MAX_VIEWS 289
#define LFSR_MAX_HALF_DIRS 112   // (15*15 - 1) / 2

namespace lfsr {

// Storage kinds of the large streams (values of lfsr_params.precision).
enum { ST_F32 = 0, ST_F16 = 1, ST_BF16 = 2 };
inline size_t storage_bytes(int st) { return st == ST_F32 ? 4 : 2; }
// Weight schemes of the regulariser (values of lfsr_params.weights).
enum { WS_PATCH = 0, WS_PAPER = 1 };

// Geometry and solver constants, passed by value to every kernel (lives in
// the kernel-parameter constant bank; all reads are warp-uniform).
struct Geom {
  int U, V, sk;          // angular grid, s_k
  int H, W;              // LR size
  int Hh, Wh;            // HR size
  int zeta;              // scale
  int kb, r;             // blur size and radius
  int separable;         // blur = kv (rows) x kh (cols)
  int S;                 // integer bound on |theta_k * omega| over views/pixels
  int win_r, patch_r;    // NLTV window / patch radius
  int sh;                // half direction count s_d / 2
  float inv_h2;          // 1 / h^2
  float inv_np;          // 1 / patch^2
  float lambda1, lambda2, mu;
  float cA;              // lambda2 + mu lambda1^2 / 2
  float thr;             // 1 / mu (prox threshold, Eq. sr_l1l2l1_prox)
  double tau;            // CG threshold
  int st;                // storage kind of the duals and stored weights (ST_*)
  int st_y;              // storage kind of the LR views
  int wscheme;           // WS_PATCH or WS_PAPER
  float inv_sig_s;       // paper weights: 1 / sigma_s (0: spatial factor 1)
  float inv_sig_e;       // paper weights: 1 / sigma_e (0: edge factor 1)
  int warp_views;        // W_k uses per-view disparity maps (generic operator kernel)
  int adjoint_bw;        // x-step uses the backward warp W_k^* (generic operator kernel)
  unsigned long long wait_ns;  // limit of a device-side wait (grid barrier), ns of %globaltimer
  int wait_unreachable;  // test mode: every wait's target lies beyond the arrivals (runs out)
  float kv[LFSR_MAX_KB], kh[LFSR_MAX_KB];
  float k2[LFSR_MAX_KB * LFSR_MAX_KB];
  float tu[LFSR_MAX_VIEWS], tv[LFSR_MAX_VIEWS];
  int8_t di[LFSR_MAX_HALF_DIRS], dj[LFSR_MAX_HALF_DIRS];  // half direction set
};

// Device-resident scalars of the CG x-step (Algorithm 2) and diagnostics.
struct DevScalars {
  double pi;        // |r|^2
  double pAp;       // <p, M p>
  double alpha;     // pi / pAp
  double beta;      // pi_new / pi_old
  double dwA, dwS;  // |dw|^2 of the data / regulariser duals
  double dw2;       // total of the last iteration
  int cg_done;      // x-step finished (pi <= tau, or a numeric failure)
  int cg_first;     // next direction is p = r (first CG step)
  int cg_steps;
  int status;       // sticky LFSR_* status
  unsigned int counter[8];   // last-block counters of the grid reductions
  double red[8];    // finalized totals of the grid reductions (RED_* slots)
  unsigned long long bar;    // arrivals at the grid barriers of the fused launches
};

// Reduction slots (partials arrays and last-block counters).
enum { RED_NLTV = 0, RED_OP = 1, RED_PI = 2, RED_DW_A = 3, RED_DW_S = 4, RED_NUM = 5 };

// Operator-kernel modes.
// OP_DATA_LR: the data block's per-LR-pixel step, its result h_k stored to
// an LR buffer (the backward-warp x-step applies its adjoint separately).
enum { OP_NORMAL = 0, OP_DATA = 1, OP_FWD = 2, OP_ADJ = 3, OP_DATA_LR = 4 };
// NLTV-kernel modes.
enum { NL_BLOCK = 0, NL_APPLY = 1, NL_WEIGHTS = 2 };

// Launch plan of the operator kernels (tile shape and smem layout).
struct OpPlan {
  int TH, TW;            // tile of HR source pixels
  int tiles_x, tiles_y, n_tiles;
  int NLr, NLc;          // max LR rows / cols touching a tile
  int NEr, NEc;          // max warp-sample rows / cols
  int NPr, NPc;          // staged source rows / cols
  int NAr, NAc;          // accumulator rows / cols
  int off_P, off_W, off_H, off_G, off_A;   // float offsets in dynamic smem
  size_t smem_bytes;
  int ctas_per_sm;
  int threads;
  int fast;              // specialised compile-time kernel (op_fast.cu)
};

struct OpArgs {
  const float* src;      // HR source (x or p) for FWD/NORMAL/DATA; LR g for ADJ
  const float* disp;     // HR disparity (view 0's map when disp_stride != 0)
  size_t disp_stride;    // floats between the per-view maps of W_k (0: one shared map)
  const float* pdot;     // backward-warp adjoint: <pdot, result> reduced and alpha formed
  float* out;            // HR accumulator target (atomics) or LR output (FWD)
  const void* y;         // DATA: LR views (storage kind g.st_y)
  const void* wA_old;    // DATA: data duals (read, g.st)
  void* wA_new;          // DATA: data duals (written, g.st)
  float scale;           // multiplies the accumulator on flush
  int view0, nviews;     // views of this launch
  int units;             // n_tiles * nviews
  double* partials;      // per-CTA partials of this kernel's reduction
  DevScalars* sc;
  int check_done;        // return at once when sc->cg_done (CG steps)
};

struct NlArgs {
  const float* x;        // weights source x^(n-1)
  const float* r;        // APPLY: CG residual
  const float* p_old;    // APPLY: previous direction
  float* p_new;          // APPLY: new direction (written)
  float* out;            // BLOCK: v (stored); APPLY: q (stored); WEIGHTS: w
  const void* wS_old;    // BLOCK: pair-layout duals (read, g.st)
  void* wS_new;          // BLOCK: pair-layout duals (written, g.st)
  const float* occ;      // paper weights: occlusion factor o (HR)
  double* partials;
  DevScalars* sc;
  int use_beta;          // APPLY: p_new = r + beta p_old (else p_new = src p)
  int check_done;
};

// One light field's share of a launch of a table-driven kernel (the
// specialised operator kernel, the stored-weight NLTV kernels and the CG
// vector kernels).  Each launch reads a device table of these, one entry per
// light field, so one launch covers many light fields of different sizes;
// a single solve is a table of one.  Pointers are this light field's
// buffers in the roles of this launch.
struct JobArgs {
  int H, W, Hh, Wh, U, V;     // geometry
  int unit0, units;           // work units of this light field: [unit0, unit0 + units)
  int tiles_x;                // tile columns (operator: 64 x 64, NLTV: 32 x 32 HR pixels)
  int chunk;                  // vector kernels: HR pixels per unit
  int view0, nviews;          // operator: views of this launch
  float scale;                // operator: factor of the flushed accumulator
  int use_beta;               // NLTV apply: p_new = r + beta p_old (else p_old is the direction)
  const float* disp;          // HR disparity
  const float2* theta;        // angular offset (tu, tv) of each view of the data
  const float* src;           // operator: x or p (HR), g (LR, adjoint); NLTV: weights source x;
                              // vector init: x
  float* out;                 // operator: HR accumulator or LR output; NLTV block: v;
                              // NLTV apply: q; vector init: v, replaced by r = -v
  const void* y;              // operator DATA: views (kind g.st_y)
  const void* wA_old;         // operator DATA: data duals (kind g.st)
  void* wA_new;
  const void* wS_old;         // NLTV block: regulariser duals, pair layout (kind g.st)
  void* wS_new;
  void* wt;                   // NLTV: stored edge weights (kind g.st)
  float* vacc;                // accumulated v of the z/w-step (stored-weight NLTV block and
                              // data block add into it; the x-step initialisation reads and
                              // clears it)
  const float* occ;           // NLTV (paper weights): occlusion factor o (HR)
  const float* r;             // NLTV apply: CG residual
  const float* p_old;         // NLTV apply: previous direction; vector update: p
  float* p_new;               // NLTV apply: new direction
  const float* q;             // vector update: M p
  float* rr;                  // vector update: residual r, updated in place
  float* x_next;              // vector: iterate of the x-step
  DevScalars* sc;             // this light field's device scalars
  // Fused launches (one light field, fields by value): the normal-matrix
  // operator finishes the CG step behind a grid barrier (x' += alpha p,
  // r -= alpha q, pi' = <r, r>, beta), its CTAs each taking fchunk HR
  // pixels; fpart holds their partial sums of <r, r>.
  int fuse;
  int fchunk;
  double* fpart;
  // NLTV apply with TMA-staged weights: the device address of the weight
  // planes' tensor map (a CUtensorMap, 64-byte aligned), or NULL.
  const void* wt_map;
};

// Launch-wide arguments of a table-driven kernel.
struct TableArgs {
  const JobArgs* jobs;        // device table
  const int* unit_job;        // unit -> table index (NULL: every unit is entry 0)
  int n_jobs;
  int total_units;
  int check_done;             // CG steps: skip light fields whose x-step has finished
  double* partials;           // reduction slots
  unsigned int* counter;      // arrival counter of the grid reduction (re-armed by the kernel)
  // Operator launches: the first unit of each CTA's contiguous range
  // (grid + 1 entries, split by measured cost), or NULL for the even split.
  // A timing launch passes unit_clock: the kernel records there the SM
  // clock at the start of each unit and, after its units, at the end of
  // each CTA's range, and leaves the device scalars alone (no final
  // reduction).
  const int* cta_unit0;
  long long* unit_clock;
};

struct NlPlan {
  int TH, TW, tiles_x, tiles_y, n_tiles;
  int NXr, NXc;          // staged x region
  int NQr, NQc;          // squared-difference / box region
  size_t smem_bytes;
  int threads;
};

// Raises a kernel's dynamic shared-memory limit to the device's opt-in
// maximum minus the kernel's static shared memory.
template <class K>
inline cudaError_t set_max_dynamic_smem(K kernel, int smem_optin) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              smem_optin - (int)fa.sharedSizeBytes);
}

// Host launchers (stream-ordered, no synchronisation).
cudaError_t op_prepare(const Geom& g, int smem_optin);
cudaError_t nl_prepare(int smem_optin);
cudaError_t op_plan(const Geom& g, OpPlan* plan, int sm_count, int smem_limit);
cudaError_t op_launch(int mode, const Geom& g, const OpPlan& plan, const OpArgs& a,
                      int grid, cudaStream_t s);
int op_grid(const OpPlan& plan, int units, int sm_count);

cudaError_t nl_plan(const Geom& g, NlPlan* plan, int smem_limit);

// NLTV with stored edge weights (window radius 1-3, patch radius 0-2).
bool nlf_supported(const Geom& g);
// Table-driven: one CTA per 32 x 32 tile (t.total_units tiles); wt holds
// s_d/2 x p values of the storage kind g.st; the block mode adds the
// regulariser divergence into the jobs' v (out), which must start at zero.
constexpr int NLF_TILE = 32;
cudaError_t weights_to_canonical(const Geom& g, const void* wt, float* can, cudaStream_t s);
cudaError_t nlw2_launch(int block, const Geom& g, const TableArgs& t, cudaStream_t s);
// chunk: directions per batch of weight loads, 6 (default) or 3.
constexpr int NLA_CHUNK = 6;
cudaError_t nla2_launch(const Geom& g, const TableArgs& t, cudaStream_t s, int chunk = NLA_CHUNK);
// The same with the weights staged by TMA (nltv_tma.cu): needs every job's
// wt_map, a row of the weight planes a multiple of 16 bytes and the driver's
// tensor-map encoder.  The map covers the s_d/2 planes of wt (kind g.st);
// map_out is host memory of sizeof(CUtensorMap) = 128 bytes.
constexpr int NLA_TMA_MAP_BYTES = 128;
bool nla2t_supported(const Geom& g);
cudaError_t nla2t_prepare(int smem_optin);
cudaError_t nla2t_make_map(const Geom& g, const void* wt, void* map_out);
cudaError_t nla2t_launch(const Geom& g, const TableArgs& t, cudaStream_t s);
// x-step initialisation from the accumulated v (jobs' vacc): r = -v, v := 0.
cudaError_t cg_init_acc_launch(const Geom& g, const TableArgs& t, cudaStream_t s);
// The paper's weights (g.wscheme == WS_PAPER): the stored-weight
// z/w-step (called by nlw2_launch), and the occlusion factor
// o = exp(-b^2 inv2_o1) exp(-pe^2 inv2_o2) of the disparity map disp and the
// projection error pe (NULL: 0), Hh x Wh floats each.
cudaError_t nlw2p_launch(int block, const Geom& g, const TableArgs& t, cudaStream_t s);
cudaError_t occlusion_launch(int Hh, int Wh, const float* disp, const float* pe, float inv2_o1,
                             float inv2_o2, float* occ, cudaStream_t s);

// The paper's backward warp (Sec. 4.1) in the x-step: out += scale sum_k
// W_k^* B^T D^T g_k with g the LR buffer a.src (s_k x q), gathered at
// u - theta_k omega_0(u) (a.disp); one CTA per 32 x 32 tile over all views,
// no atomics.  With a.pdot, also <pdot, sum_k ...> into RED_OP and the CG
// step length (as OP_NORMAL).
struct BwPlan {
  int tiles_x, tiles_y, n_tiles;
  int NEr, NEc;          // adjoint-blurred region: tile + 2 (S + 1)
  int NLr, NLc;          // LR pixels whose blur touches it
  int off_G, off_H, off_T;
  size_t smem_bytes;
};
constexpr int BW_TILE = 32;
cudaError_t bw_plan(const Geom& g, BwPlan* plan, int smem_limit);
cudaError_t bw_prepare(int smem_optin);
cudaError_t bw_launch(const Geom& g, const BwPlan& plan, const OpArgs& a, cudaStream_t s);

// Specialised operator kernel for separable kernels of common (zeta, kb).
bool fast_supported(const Geom& g);
cudaError_t fast_prepare(const Geom& g, int smem_optin);
cudaError_t fast_plan(const Geom& g, OpPlan* plan, int smem_limit);
// Table-driven: t.total_units (64 x 64 tile, view pair) units over `grid`
// CTAs; the partial slots are t.n_jobs x grid.
constexpr int FAST_TILE = 64;
constexpr int FAST_VIEWS = 2;
// single != NULL: one light field, its fields by value (t.jobs unused);
// else the table t (data block and normal-matrix modes).
cudaError_t fast_launch(int mode, const Geom& g, const OpPlan& plan, const TableArgs& t, int grid,
                        cudaStream_t s, const JobArgs* single);
cudaError_t fast_launch_table(int mode, const Geom& g, const OpPlan& plan, const TableArgs& t,
                              int grid, cudaStream_t s);
cudaError_t fast_prepare_table(int zeta, int kb, int smem_optin);
// Plan of the table variant for tile side 64 or 32 (the batch autotuner's
// candidates); plan.TH selects the variant at launch.
cudaError_t fast_plan_table(const Geom& g, OpPlan* plan, int smem_limit, int tile);
cudaError_t nl_launch(int mode, const Geom& g, const NlPlan& plan, const NlArgs& a,
                      cudaStream_t s);

// The persistent batch iteration (batch_persist.cu): one cooperative launch
// per ADMM iteration runs every phase of Algorithm 1 for every light field
// of a batch -- the regulariser block, the data block of each operator
// group, the x-step initialisation and K x (NLTV apply, normal matrix of
// each group, CG update) -- over the same work units as the per-phase
// launches, with a bounded grid barrier between dependent phases.  The
// launch arguments of one iteration parity live in device memory.
constexpr int PERSIST_MAX_GROUPS = 2;
struct PersistArgs {
  TableArgs nlw, init;               // regulariser block, x-step initialisation
  TableArgs nla[2], upd[2];          // per CG-step parity
  TableArgs data[PERSIST_MAX_GROUPS];
  TableArgs norm[2][PERSIST_MAX_GROUPS];
  OpPlan P[PERSIST_MAX_GROUPS];      // operator plan of each group (64 x 64 tiles)
  int cg_iters;
  int sx_off;                        // float offset of the regulariser block's divergence tile
};
// The (scale, kb) of each group, the NLTV window and patch radii and the
// storage kind decide whether a compiled persistent kernel exists; order[]
// receives the batch's group index for each slot of PersistArgs.
bool persist_supported(const Geom& g, const Geom* gg, const int* tile, int n_groups, int* order);
cudaError_t persist_prepare(const Geom& g, const Geom* gg, const int* order, int n_groups,
                            int smem_optin);
// Dynamic shared memory of the launch and CTAs per SM at that size (0: the
// kernel cannot run with one CTA per SM).
size_t persist_smem(const Geom& g, const OpPlan* P, int n_groups, int* sx_off);
int persist_occupancy(const Geom& g, const Geom* gg, const int* order, int n_groups,
                      size_t smem);
// args: device pointer of the iteration's PersistArgs; bar: the batch's
// grid-barrier arrival counter; grid: SMs x 1 (every CTA co-resident).
cudaError_t persist_launch(const Geom& g, const Geom* gg, const int* order, int n_groups,
                           const PersistArgs* args, unsigned long long* bar, size_t smem,
                           int grid, cudaStream_t s);

// Table-driven vector kernels: one CTA per chunk of HR pixels.
constexpr int VEC_THREADS = 512;
cudaError_t cg_init_launch(const Geom& g, const TableArgs& t, cudaStream_t s);
cudaError_t cg_update_launch(const Geom& g, const TableArgs& t, cudaStream_t s);
// Regulariser duals: canonical float [d][u] <-> edge-pair layout of kind g.st.
cudaError_t pair_from_canonical(const Geom& g, const float* can, void* pair, cudaStream_t s);
cudaError_t pair_to_canonical(const Geom& g, const void* pair, float* can, cudaStream_t s);
// n floats -> storage kind st (round to nearest even).  A value that is
// not finite or outside the kind's finite range sets sc->status to
// LFSR_EINVAL (sticky) and is stored saturated (0 for NaN).
cudaError_t to_storage(int st, const float* src, void* dst, size_t n, DevScalars* sc, int grid,
                       cudaStream_t s);
cudaError_t from_storage(int st, const void* src, float* dst, size_t n, int grid, cudaStream_t s);
cudaError_t scalars_reset(DevScalars* sc, cudaStream_t s);

// Sets the thread-local message that lfsr_last_error(NULL) returns.
void set_thread_error(const char* msg);

}  // namespace lfsr
