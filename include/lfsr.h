/*
 * lfsr.h -- C ABI of the GB300 light-field super-resolution solver.
 *
 * The solver reconstructs the high-resolution (HR) reference view x of a 4D
 * light field from U*V low-resolution (LR) sub-aperture views y_k by
 * minimising (Eq. sr_fin)
 *
 *   J(x) = l1 sum_k |A_k x - y_k|_1 + l2 sum_k |A_k x - y_k|_2^2
 *          + sum_d |W_d (S_d - I) x|_1,        A_k = D B W_k (Eq. sr_model_vec)
 *
 * with the rotated ADMM of Algorithm 1 and the conjugate-gradient x-step of
 * Algorithm 2 (Sec. 4-5).  Every step runs in hand-written sm_103a CUDA
 * kernels on one GPU; there is no CPU fallback.
 *
 * Conventions
 *  - Images passed through this interface are row-major float32 (the
 *    solver may keep its state in 16 bits, see LFSR_FP16_STORAGE).  LR size H x W; HR size (scale*H) x
 *    (scale*W) = Hh x Wh; p = Hh*Wh, q = H*W.
 *  - View k = v*U + u has angular offset theta_k = (u-(U-1)/2, v-(V-1)/2);
 *    U and V are odd so the centre view is the reference (Sec. 3.1).
 *  - W_k samples x bilinearly at (i + tv*omega(i,j), j + tu*omega(i,j)),
 *    zero outside the image (Sec. 4.1 forward warp); its adjoint is the exact
 *    scatter of the same taps.  B correlates with the kb x kb kernel, zero
 *    padded; D keeps the top-left pixel of every scale x scale block
 *    (Sec. 4.1).
 *  - NLTV weights w_d(u) = exp(-pd/h^2), pd the mean of squared differences
 *    between the patch at u and the patch at u+d (clamp-to-edge reads), 0 if
 *    u+d leaves the image; directions d = window offsets minus the centre,
 *    in raster order (s_d = window^2 - 1).  Weights are rebuilt from the
 *    current x at the start of every ADMM iteration (Sec. 6.1).
 *  - Regulariser duals in the canonical layout are s_d x Hh x Wh, the dual
 *    of direction d at pixel u at [d][u] (Eq. sr_admm_compact row order);
 *    data duals are s_k x H x W.
 *  - s_k is the number of views used: U*V, or n_views when params->views
 *    lists a subset; the views' data (LR views, data duals, apply_A's view
 *    argument) are indexed 0 .. s_k-1 in the order of that list.
 *
 * Memory kinds: LFSR_MEM_HOST pointers are ordinary host memory (pinned or
 * pageable; the call copies through the handle's stream); LFSR_MEM_DEVICE
 * pointers are device memory of the current device (e.g. a torch tensor's
 * data_ptr) and all work is ordered on the handle's stream.  The caller owns
 * every buffer it passes; the handle owns all solver state.
 *
 * Errors: every int-returning call returns LFSR_OK (0) or a negative
 * LFSR_E* code and stores a message readable with lfsr_last_error().  No
 * call aborts or throws.  A handle is not thread-safe; different handles
 * are independent.
 */
#ifndef LFSR_H
#define LFSR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LFSR_OK            0
#define LFSR_EINVAL       (-1)  /* bad size, parameter or pointer            */
#define LFSR_ENOMEM       (-2)  /* device allocation failed                  */
#define LFSR_ECUDA        (-3)  /* CUDA runtime error (message has details)  */
#define LFSR_ENUMERIC     (-4)  /* non-finite or negative CG curvature       */
#define LFSR_ETIMEOUT     (-5)  /* a bounded device wait gave up             */
#define LFSR_EUNSUPPORTED (-6)  /* valid but not implemented on this path    */

#define LFSR_MEM_HOST   0
#define LFSR_MEM_DEVICE 1

/* Default limit of a device-side wait (a grid barrier of the fused CG
 * step), in nanoseconds: after it the wait gives up and the call reports
 * LFSR_ETIMEOUT (see lfsr_set_device_wait). */
#define LFSR_DEFAULT_WAIT_NS 1000000000LL

/* Precision of the solver state (lfsr_params.precision).
 *
 * LFSR_FP32: all state and arithmetic in float32.
 *
 * LFSR_FP16_STORAGE / LFSR_BF16_STORAGE: the large streams -- the LR views
 * y, the data duals, the regulariser duals and the stored NLTV edge
 * weights -- are kept in IEEE half or bfloat16 (round to nearest even on
 * every store); every kernel widens them to float and computes in float32.
 * The HR iterate x, the CG vectors (r, p, q, v), the disparity map and the
 * per-edge divergence terms of the z/w-step (an intermediate) stay
 * float32, and the inner products of the x-step and the residual norms
 * accumulate in float64, as in LFSR_FP32.  The errors against the float64
 * algorithm are stated per workload by the tests.
 *
 * LFSR_KEEP_VIEWS_FP32 may be or-ed into a 16-bit precision to keep the
 * views y in float32 (rounding the views perturbs the data itself, the
 * largest single error term of half storage; the views are read once per
 * ADMM iteration, so keeping them costs little bandwidth).
 *
 * Range: a view value (or a data dual given to lfsr_set_state) that is not
 * finite or exceeds the type's largest finite value (65504 for half) is
 * stored saturated and makes the next blocking call return LFSR_EINVAL.
 * The duals are bounded by 1/mu, so LFSR_FP16_STORAGE requires
 * 1/mu <= LFSR_FP16_MAX_INV_MU (else lfsr_create returns
 * LFSR_EUNSUPPORTED).  Values below half's smallest subnormal (about
 * 6e-8), e.g. vanishing NLTV weights, store as 0. */
#define LFSR_FP32 0
#define LFSR_FP16_STORAGE 1
#define LFSR_BF16_STORAGE 2
#define LFSR_KEEP_VIEWS_FP32 256
#define LFSR_FP16_MAX_INV_MU 8192.0

/* Weight scheme of the regulariser (lfsr_params.weights).
 *
 * LFSR_WEIGHTS_PATCH (0): w_d(u) = exp(-pd/h^2), the patch distance of the
 * conventions above; symmetric in the pixel pair.
 *
 * LFSR_WEIGHTS_PAPER (1): the paper's weights (Sec. 3.4, Eq. weight_occ),
 *   w_d(u) = exp(-|d|^2/sigma_s) * e(u) * o(u),   0 if u+d leaves the image,
 *   e(u) = exp(-|grad x(u)|^2/sigma_e), grad x by central differences
 *          (x(i+1,j) - x(i-1,j))/2, (x(i,j+1) - x(i,j-1))/2, clamped indices,
 *          from the current x (rebuilt every ADMM iteration, like the patch
 *          weights),
 *   o(u) = exp(-b(u)^2/(2 sigma_o1^2)) * exp(-p(u)^2/(2 sigma_o2^2)),
 *          b(u) = min(0, (omega(i+1,j) - omega(i,j)) + (omega(i,j+1) - omega(i,j)))
 *          (forward differences, 0 across the last row / column), p the
 *          projection error (lfsr_params.proj_err, 0 when NULL); o is fixed
 *          by the disparity map and computed once by lfsr_create.
 * A sigma of 0 makes its factor 1.  These weights are directed:
 * w_{-d}(u+d) = exp(-|d|^2/sigma_s) e(u+d) o(u+d) differs from w_d(u), and
 * the z/w-step uses each.  nltv_patch and nltv_h are ignored. */
#define LFSR_WEIGHTS_PATCH 0
#define LFSR_WEIGHTS_PAPER 1

/* Warps (Sec. 4.1).
 *
 * Per-view disparity maps (lfsr_params.disparity_views): W_k samples x at
 * z + theta_k omega_k(z) with omega_k the disparity map of view k on its own
 * HR grid (the paper associates a map with each perspective); without them
 * every W_k uses the reference map `disparity`.
 *
 * lfsr_params.adjoint selects what the x-step uses for A_k^T:
 * LFSR_ADJOINT_EXACT (0): the exact adjoint of A_k (W_k^T scatters the
 *   bilinear taps), so the x-step's matrix is symmetric and CG applies.
 * LFSR_ADJOINT_BACKWARD_WARP (1): the paper's backward warp W_k^*, which
 *   samples bilinearly at u - theta_k omega_0(u) with the reference map
 *   omega_0 = `disparity`.  It equals W_k^T where the disparity is locally
 *   constant and differs near disparity edges (and with per-view maps); the
 *   x-step then runs Algorithm 2 on that matrix, as the paper does.
 *   lfsr_apply_AT applies W_k^* B^T D^T, lfsr_apply_normal the same matrix.
 * Both options run on the generic operator kernel (not in batches, servers
 * or lfsr_apply_normal_noalloc: LFSR_EUNSUPPORTED). */
#define LFSR_ADJOINT_EXACT 0
#define LFSR_ADJOINT_BACKWARD_WARP 1

/* Problem and solver parameters (copied by lfsr_create).  struct_size must
 * be sizeof(lfsr_params). */
typedef struct lfsr_params {
  uint32_t struct_size;
  int32_t U, V;            /* angular grid, odd, U*V <= 289                 */
  int32_t H, W;            /* LR view size, >= 1                            */
  int32_t scale;           /* zeta in {1,2,3,4} (Sec. 3.1)                  */
  int32_t kb;              /* blur size, odd, <= 15                         */
  const float *blur;       /* host, kb*kb taps K[a][b], a = row offset + r  */
  const float *disparity;  /* host, Hh*Wh disparity map omega (HR px per
                              unit angular step) on the reference grid      */
  double lambda1, lambda2; /* >= 0, not both 0 (Eq. sr_fin)                 */
  double mu;               /* ADMM penalty vartheta > 0 (Algorithm 1)       */
  int32_t nltv_window;     /* odd, 3..15                                    */
  int32_t nltv_patch;      /* odd, 1..7                                     */
  double nltv_h;           /* > 0                                           */
  int32_t cg_iters;        /* K of Algorithm 2, >= 0                        */
  double cg_tol;           /* tau: CG stops once pi = |r|^2 <= tau          */
  int32_t precision;       /* LFSR_FP32, LFSR_FP16_STORAGE or
                              LFSR_BF16_STORAGE [| LFSR_KEEP_VIEWS_FP32]      */
  const int32_t *views;    /* host, optional: the grid indices k = v*U + u of
                              the views used, strictly ascending (Sec. 6.1's
                              x4 experiment uses a star of 17 of 5 x 5);
                              NULL: all U*V.  Copied.                        */
  int32_t n_views;         /* entries of views (ignored when views is NULL)  */
  int32_t weights;         /* LFSR_WEIGHTS_PATCH or LFSR_WEIGHTS_PAPER        */
  float sigma_s, sigma_e;  /* paper weights: spatial, edge scale; >= 0      */
  float sigma_o1, sigma_o2;/* paper weights: occlusion boundary, projection
                              error scale; >= 0 (0: factor 1)               */
  const float *proj_err;   /* host, optional: Hh*Wh projection error p of the
                              occlusion factor; NULL: p = 0.  Read by
                              lfsr_create only.                             */
  const float *disparity_views; /* host, optional: s_k*Hh*Wh per-view maps
                              omega_k (view k's HR grid, the data's view
                              order); NULL: W_k uses disparity.  Copied.    */
  int32_t adjoint;         /* LFSR_ADJOINT_EXACT or LFSR_ADJOINT_BACKWARD_WARP */
} lfsr_params;

typedef struct lfsr_handle lfsr_handle;

typedef struct lfsr_stats_t {
  uint32_t struct_size;    /* set to sizeof(lfsr_stats_t) before the call   */
  int32_t iterations;      /* ADMM iterations run since the last load       */
  int32_t cg_steps;        /* CG steps the last x-step took                 */
  int32_t status;          /* sticky device status (LFSR_OK or LFSR_E*)     */
  double dual_change_sq;   /* |w_n - w_{n-1}|^2 of the last iteration       */
  double cg_pi;            /* |r|^2 at the end of the last x-step           */
  int64_t state_bytes;     /* device bytes owned by the handle              */
  int64_t launches;        /* kernels launched since the last load          */
  /* profiling mode only (lfsr_set_profiling): summed kernel time in ms and
   * launch counts, by kernel class: 0 nltv-block, 1 data-block, 2 cg-init,
   * 3 nltv-apply, 4 normal-apply, 5 cg-update                              */
  double kernel_ms[8];
  int64_t kernel_launches[8];
  /* load balance of the specialised operator launches, measured once by
   * lfsr_create (one launch that times every (tile, view pair) unit): the
   * slowest CTA's cost over the mean for the even split of the units and
   * for the cost-balanced contiguous ranges the launches use (equal when
   * the balanced ranges would not be faster and the even split stays);
   * 0 when not measured (generic operator kernel, or fewer than two units
   * per CTA)                                                               */
  double op_split_even;
  double op_split_balanced;
} lfsr_stats_t;

/* Creates a solver for one light-field geometry.  Copies blur and
 * disparity to the device, allocates all ADMM state (x, data and
 * regulariser duals, CG vectors) and validates every parameter.
 * cuda_stream: a cudaStream_t (NULL = the legacy default stream) on which
 * every later call of this handle is ordered.  Returns LFSR_EINVAL for bad
 * parameters, LFSR_ENOMEM / LFSR_ECUDA on device failures; *out is set to
 * NULL on failure. */
int lfsr_create(const lfsr_params *params, void *cuda_stream, lfsr_handle **out);

/* Full solve (Algorithm 1): x := x0, all duals := 0, then `iterations`
 * ADMM iterations, each rebuilding the NLTV weights from the current x
 * and running the K-step CG x-step of Algorithm 2.  lr_views holds s_k*q
 * floats ([k][i][j]), x0 and x_out p floats.  Blocks until x_out is
 * written.  Returns LFSR_ENUMERIC if the CG curvature became non-finite
 * or negative (a curvature of exactly 0 ends the x-step: its direction has
 * vanished), LFSR_EINVAL if a view value does not fit the storage
 * type (16-bit precisions). */
int lfsr_solve(lfsr_handle *h, const float *lr_views, int iterations,
               const float *x0, float *x_out, int mem_kind);

/* Frees the handle and all device memory it owns.  NULL is a no-op. */
void lfsr_destroy(lfsr_handle *h);

/* Message of the last failing call on h (or of the last failing create /
 * NULL-handle call of this thread when h is NULL).  Never NULL. */
const char *lfsr_last_error(const lfsr_handle *h);

/* Synchronises the handle's stream and reports the last iteration's
 * diagnostics. */
int lfsr_stats(const lfsr_handle *h, lfsr_stats_t *out);

/* ---- resident-state stepping (the solve split into its parts) -------- */

/* Uploads the LR views, sets x := x0 and all duals := 0 (Algorithm 1,
 * lines 1-2).  Asynchronous on the handle's stream. */
int lfsr_load(lfsr_handle *h, const float *lr_views, const float *x0, int mem_kind);

/* Enqueues `iterations` ADMM iterations on the resident state (no host
 * synchronisation; one CUDA graph launch per two iterations). */
int lfsr_iterate(lfsr_handle *h, int iterations);

/* Copies the current x (p floats) out; blocks until done. */
int lfsr_get_x(lfsr_handle *h, float *x_out, int mem_kind);

/* Sets / reads the full ADMM state in the canonical layout: x (p floats),
 * data duals wA (s_k*q), regulariser duals wS (s_d*p).  Any pointer may be
 * NULL to skip that part.  lfsr_get_state blocks until done.  With a
 * 16-bit precision the duals are rounded to the storage type on set and
 * widened exactly on get. */
int lfsr_set_state(lfsr_handle *h, const float *x, const float *wA,
                   const float *wS, int mem_kind);
int lfsr_get_state(lfsr_handle *h, float *x, float *wA, float *wS, int mem_kind);

/* ---- single operators (Sec. 4.1 kernels; for checking and reuse) ------ */

/* out = A_k x (q floats), or for view == -1 all views (s_k*q floats). */
int lfsr_apply_A(lfsr_handle *h, int view, const float *x, float *out, int mem_kind);

/* out = A_k^T g (p floats); for view == -1, out = sum_k A_k^T g_k with g
 * holding s_k*q floats. */
int lfsr_apply_AT(lfsr_handle *h, int view, const float *g, float *out, int mem_kind);

/* NLTV weights of x in the canonical layout (s_d*p floats): w_d(u) at
 * [d][u].  With 16-bit storage and the patch weights these are the stored
 * (rounded) edge weights; the paper's directed weights are returned in
 * float32. */
int lfsr_weights(lfsr_handle *h, const float *x, float *w, int mem_kind);

/* q = M p with M = (l2 + mu l1^2/2) sum_k A_k^T A_k + mu/2 sum_d S_d^T S_d
 * (the normal matrix G^T G of the x-step, Sec. 5), the NLTV weights built
 * from xw; *pMp (host) receives <p, M p> accumulated in float64. */
int lfsr_apply_normal(lfsr_handle *h, const float *xw, const float *p, float *q,
                      double *pMp, int mem_kind);

/* Profiling mode: when on, lfsr_iterate launches kernels one by one (no
 * graph) with CUDA events around each and lfsr_stats reports per-class
 * kernel time.  Off by default. */
int lfsr_set_profiling(lfsr_handle *h, int on);

/* Host-side fault injection (for testing the failure paths; no device
 * fault is involved).  The environment variable LFSR_FAULT, read at every
 * device allocation the library makes (lfsr_create, lfsr_batch_create,
 * server admission, staging buffers):
 *   LFSR_FAULT=alloc     every allocation fails,
 *   LFSR_FAULT=alloc:K   the K-th allocation fails (K >= 1, counted from
 *                        the moment the variable took this value),
 * as if cudaMalloc had returned cudaErrorMemoryAllocation: the call frees
 * what it holds and returns LFSR_ENOMEM.  A dry-run server counts each
 * admission as one allocation.  Unset (or any other value): no fault. */

/* Device-side waits.  With the specialised operator kernel (separable
 * blur, common scale and blur size) each CG step of the x-step (Algorithm
 * 2) is one cooperative launch: the normal-matrix product, then a grid
 * barrier, the step length alpha = pi / <p, M p>, the updates x += alpha p
 * and r -= alpha q with their <r, r>, a second grid barrier and beta.  No
 * barrier waits without a bound: after limit_ns nanoseconds (default
 * LFSR_DEFAULT_WAIT_NS) a waiting CTA gives up, the CG step is abandoned
 * and the next blocking call returns LFSR_ETIMEOUT; the device context stays
 * usable and the next lfsr_load / lfsr_solve starts clean.  test_unreachable
 * != 0 makes every barrier wait for one arrival more than the launch has,
 * so that every wait runs out (a test of the timeout path; the solve then
 * fails with LFSR_ETIMEOUT).  The setting applies from the next iteration
 * (the captured graphs are rebuilt); the call synchronises the handle's
 * stream. */
int lfsr_set_device_wait(lfsr_handle *h, int64_t limit_ns, int test_unreachable);

/* ---- batches of light fields ------------------------------------------
 *
 * A batch steps many light fields -- of different angular grids, LR sizes,
 * scales and blurs -- through the ADMM iteration together (Algorithm 1 with
 * the CG x-step of Algorithm 2, exactly as lfsr_iterate does for each of
 * them).  Each phase of an iteration is one launch over a work list that
 * spans every light field of the batch (NLTV tiles, (tile, view pair)
 * operator units, chunks of HR pixels); the operator phases take one launch
 * per group of light fields that share the scale and the blur kernel.  Two
 * iterations are captured as one CUDA graph and replayed.  The CG scalars
 * stay per light field; every light field's result equals its result alone
 * up to the order of float atomic additions.
 *
 * Requirements: the light fields share lambda1, lambda2, mu, the NLTV
 * window, patch and h, cg_iters, cg_tol and precision (else LFSR_EINVAL),
 * and each takes the specialised kernels -- a separable blur with (scale,
 * kb) in {(1,3) (1,5) (1,7) (2,3) (2,5) (2,7) (2,9) (3,5) (3,7) (3,9) (4,7)
 * (4,9)} and an NLTV window of 3, 5 or 7 with a patch of 1, 3 or 5 (else
 * LFSR_EUNSUPPORTED).  Each light field's state is allocated as by
 * lfsr_create.  All calls are ordered on cuda_stream.  Not thread-safe. */
#define LFSR_BATCH_MAX 4096

typedef struct lfsr_batch lfsr_batch;

/* Creates a batch of n light fields, params[j] describing light field j
 * (copied).  *out is NULL on failure. */
int lfsr_batch_create(const lfsr_params *params, int n, void *cuda_stream, lfsr_batch **out);

/* Frees the batch and all its device memory.  NULL is a no-op. */
void lfsr_batch_destroy(lfsr_batch *b);

/* Message of the last failing call on b (NULL: of this thread's last
 * failing batch call).  Never NULL. */
const char *lfsr_batch_last_error(const lfsr_batch *b);

/* Number of light fields (0 for NULL). */
int lfsr_batch_size(const lfsr_batch *b);

/* As lfsr_load for light field `job`: views and x0 in, duals := 0.  Also
 * re-arms the batch's reduction counters (needed after LFSR_ETIMEOUT). */
int lfsr_batch_load(lfsr_batch *b, int job, const float *lr_views, const float *x0,
                    int mem_kind);

/* Enqueues `iterations` ADMM iterations of every light field (no host
 * synchronisation). */
int lfsr_batch_iterate(lfsr_batch *b, int iterations);

/* As lfsr_get_x / lfsr_stats for light field `job` (blocking). */
int lfsr_batch_get_x(lfsr_batch *b, int job, float *x_out, int mem_kind);
int lfsr_batch_stats(const lfsr_batch *b, int job, lfsr_stats_t *out);

/* Kernel launches per ADMM iteration of the whole batch. */
int lfsr_batch_launches_per_iteration(const lfsr_batch *b);

/* Autotuner: times, on the loaded light fields, the candidate tile shapes
 * of the operator kernel (64 x 64 and 32 x 32 HR pixels per work unit) for
 * each group of light fields sharing scale and blur, the stencil blocking
 * of the NLTV divergence kernel (6 or 3 window directions per batch of
 * weight loads) and, where the persistent form is available, the launch
 * form (per-phase launches or one persistent launch per iteration), and
 * keeps the fastest of each.  It runs about 3 x (candidate tiles) x
 * (groups) + 10 ADMM iterations on the loaded state, which therefore has to
 * be loaded again (lfsr_batch_load) before a solve whose result matters.
 * Synchronous. */
int lfsr_batch_autotune(lfsr_batch *b);

/* The current choices: op_tile[g] for g < min(groups, max_groups) and
 * *nla_chunk (either pointer may be NULL).  Returns the number of operator
 * groups (0 for NULL). */
int lfsr_batch_tuning(const lfsr_batch *b, int *op_tile, int max_groups, int *nla_chunk);

/* Sets the choices directly (e.g. ones saved from an earlier autotune):
 * op_tile holds one tile side (64 or 32) per operator group, in the order
 * lfsr_batch_tuning reports them; nla_chunk is 6 or 3. */
int lfsr_batch_set_tuning(lfsr_batch *b, const int *op_tile, int n_groups, int nla_chunk);

/* Launch forms of a batch iteration (Algorithm 1 with K CG steps of
 * Algorithm 2 for every light field).
 *   LFSR_BATCH_PHASES: one launch per phase (per operator group for the
 *     operator phases), 2 + G + K (2 + G) launches for G groups.
 *   LFSR_BATCH_PERSISTENT: one cooperative launch per iteration runs every
 *     phase over the same work units on one CTA per SM, a grid barrier
 *     between dependent phases.  Every barrier wait is bounded (the limit of
 *     lfsr_batch_set_device_wait, default LFSR_DEFAULT_WAIT_NS): a CTA whose
 *     wait runs out records LFSR_ETIMEOUT in every light field's status
 *     (reported by lfsr_batch_get_x) and abandons the iteration's work; the
 *     light fields must then be loaded again.  Compiled for the NLTV window
 *     5 (patch 3) with (scale, kb) = (2, 5), and the window 7 (patch 3) with
 *     (2, 7), (3, 9) or both groups, patch-distance weights, float or half
 *     storage, 64 x 64 operator tiles.
 * Results of the two forms agree up to the order of float atomic additions.
 * Both forms run two iterations per CUDA graph; profiling mode always times
 * the per-phase launches. */
#define LFSR_BATCH_PHASES 0
#define LFSR_BATCH_PERSISTENT 1

/* 1 when a compiled persistent iteration fits the batch as it is now
 * (operator groups, tile sides, NLTV window, weights, storage), else 0. */
int lfsr_batch_persistent_available(const lfsr_batch *b);

/* The current launch form (-1 for NULL). */
int lfsr_batch_form(const lfsr_batch *b);

/* Selects the launch form (LFSR_EUNSUPPORTED for the persistent form when
 * lfsr_batch_persistent_available is 0).  A change of tuning that makes the
 * persistent form unavailable falls back to LFSR_BATCH_PHASES.  Synchronises
 * the batch's stream. */
int lfsr_batch_set_form(lfsr_batch *b, int form);

/* As lfsr_set_device_wait, for the grid barriers of the persistent form:
 * limit_ns of %globaltimer per wait; test_unreachable != 0 makes every wait
 * run out (the test path of LFSR_ETIMEOUT). */
int lfsr_batch_set_device_wait(lfsr_batch *b, int64_t limit_ns, int test_unreachable);

/* Profiling mode (as lfsr_set_profiling): lfsr_batch_iterate launches one by
 * one with CUDA events around each launch; lfsr_batch_kernel_times
 * synchronises and returns the summed milliseconds and launch counts by
 * class (the classes of lfsr_stats_t; 8 entries each) since profiling was
 * switched on. */
int lfsr_batch_set_profiling(lfsr_batch *b, int on);
int lfsr_batch_kernel_times(lfsr_batch *b, double *ms, int64_t *launches);

/* Upper bound of the device bytes lfsr_create allocates for params (the
 * state of one light field; the float staging buffer for host transfers,
 * allocated on first use, excluded).  -1 for invalid params.  No device
 * call. */
int64_t lfsr_estimate_state_bytes(const lfsr_params *params);

/* ---- continuous-batching server ---------------------------------------
 *
 * Requests (one light field each, any geometry the batches accept) arrive at
 * any time and are admitted in arrival order as soon as an active slot is
 * free and the sum of the active light fields' state bytes
 * (lfsr_estimate_state_bytes) stays within the budget; a request that does
 * not fit waits, and none behind it overtakes it.  An admitted request's
 * state is created and loaded at once and stays on the device; all active
 * light fields step through the ADMM iteration together (one launch per
 * phase for all of them, as a batch), so requests that arrive while others
 * run share the GPU with them.  A request leaves exactly at its
 * `iterations`-th iteration: its result is copied to host memory and its
 * device state freed.  Every result equals the request's own lfsr_solve up
 * to the order of float atomic additions.  Requests must share the solver
 * constants (as in a batch).  A request can be cancelled at any time
 * (lfsr_server_cancel); one that fails (its admission could not allocate,
 * LFSR_ENOMEM; a kernel it needs is missing, LFSR_EUNSUPPORTED) frees its
 * slot and budget and the requests around it continue unchanged.  The entry
 * points of one server may be called from several host threads: each call
 * holds the server's lock (a step holds it while the GPU runs its
 * iterations). */
#define LFSR_SERVER_DRY_RUN 1   /* flags: schedule without a device (checks) */

#define LFSR_REQ_QUEUED    0
#define LFSR_REQ_ACTIVE    1
#define LFSR_REQ_DONE      2
#define LFSR_REQ_FETCHED   3
#define LFSR_REQ_FAILED    4
#define LFSR_REQ_CANCELLED 5

typedef struct lfsr_server lfsr_server;

typedef struct lfsr_server_config {
  uint32_t struct_size;        /* sizeof(lfsr_server_config)                 */
  int64_t hbm_budget_bytes;    /* device bytes for the active light fields    */
  int32_t max_active;          /* active slots, 1 .. LFSR_BATCH_MAX          */
  int32_t iterations;          /* ADMM iterations per request (N)            */
  int32_t iterations_per_step; /* iterations between scheduling points (>= 1) */
  int32_t flags;               /* LFSR_SERVER_DRY_RUN or 0                   */
} lfsr_server_config;

typedef struct lfsr_server_stats_t {
  uint32_t struct_size;        /* set to sizeof(lfsr_server_stats_t)         */
  int32_t queued, active, done, failed;
  int64_t bytes_in_use, bytes_peak;
  int64_t iterations;          /* batch iterations run                       */
  int64_t batch_rebuilds;      /* launch-structure rebuilds (active set changed) */
  int64_t admitted, retired;
  int64_t launches;            /* kernel launches of the batch iterations    */
  int64_t cancelled;           /* requests cancelled (queued, active or done) */
} lfsr_server_stats_t;

/* Creates a server; work is ordered on cuda_stream.  No device call. */
int lfsr_server_create(const lfsr_server_config *cfg, void *cuda_stream, lfsr_server **out);
void lfsr_server_destroy(lfsr_server *s);
const char *lfsr_server_last_error(const lfsr_server *s);

/* Queues a request: params as for lfsr_create (host blur and disparity,
 * optional view list and projection error), views (s_k*q floats) and x0
 * (p floats) in host memory; all are copied.  *id receives the request's
 * id (0, 1, 2, ... in submission order).  Per-view disparity maps and the
 * backward-warp adjoint are not served (LFSR_EUNSUPPORTED). */
int lfsr_server_submit(lfsr_server *s, const lfsr_params *params, const float *lr_views,
                       const float *x0, int64_t *id);

/* One scheduling round: admit what fits, then run the active light fields
 * up to iterations_per_step iterations (fewer when one of them is due
 * sooner), then retire the ones that reached their N.  Blocks until the
 * iterations are done.  Returns the number of active requests afterwards
 * (>= 0) or a negative LFSR_E* code.  Admission creates the light field's
 * state as lfsr_create does, including the two timing launches that measure
 * its operator units' costs; the active set's launches split their units
 * over the CTAs by those costs. */
int lfsr_server_step(lfsr_server *s);

/* *state (LFSR_REQ_*) and *iterations of request id.  Returns LFSR_OK, the
 * request's error code if it failed, or LFSR_EINVAL for an unknown id. */
int lfsr_server_status(const lfsr_server *s, int64_t id, int *state, int *iterations);

/* Copies a done request's x (p floats) to x_out and drops the server's
 * copy. */
int lfsr_server_fetch(lfsr_server *s, int64_t id, float *x_out, int mem_kind);

int lfsr_server_stats(const lfsr_server *s, lfsr_server_stats_t *out);

/* Cancels request id: a queued one leaves the queue (the requests behind it
 * may be admitted at the next step), an active one leaves the active set
 * at once (its device state, slot and budget are freed; the others are
 * rebuilt into the next step's launches and continue from their state), a
 * done one drops its result.  The request's state becomes
 * LFSR_REQ_CANCELLED.  Returns LFSR_EINVAL for an unknown id or a request
 * already fetched, failed or cancelled. */
int lfsr_server_cancel(lfsr_server *s, int64_t id);

/* ---- no-allocation variant ------------------------------------------
 *
 * Some callers cannot allocate device memory: code that runs inside a host
 * framework whose allocator owns the whole device heap (a cudaMalloc behind
 * its back fragments or exhausts its pool), callers in processes held to a
 * hard device-memory cap, and latency-critical callers that cannot afford
 * the device-wide synchronisation cudaMalloc and cudaFree may imply.  For
 * them this entry point computes what lfsr_apply_normal computes -- q = M p
 * and <p, M p> -- without a handle and without allocating anything.  It has
 * no counterpart in the paper; it is a packaging of the same kernels.
 *
 * The kernels' scratch (float64 block partials, reduction counters and
 * totals) lives in one fixed array of LFSR_NOALLOC_SCRATCH_BYTES in device
 * memory, defined at file scope in the library: every GPU that loads the
 * library holds it until the process exits.
 *   - The first call on each device (with that device current) looks up
 *     the array's device address and raises the kernels' shared-memory
 *     limits; make that first call before any stream capture.
 *   - Every call uses the same array and clears its counters first.  Calls
 *     that overlap on the GPU (other streams, other host threads) race on
 *     it: serialise them.
 *   - Sizes beyond the array are rejected with LFSR_EINVAL: the HR image may
 *     hold at most LFSR_NOALLOC_MAX_TILES tiles of 32 x 32 pixels (e.g.
 *     2048 x 2048).
 *
 * params: validated as by lfsr_create (host blur; host disparity, which
 * must hold the same map as d_disparity); precision must be LFSR_FP32.
 * d_disparity, d_xw (weights source), d_p and d_q are device pointers of
 * the current device (Hh*Wh floats each); *pMp (host) receives <p, M p> in
 * float64.  The kernels warp by d_disparity: before they run, a check kernel
 * reads it, refuses NaN or infinite values (LFSR_EINVAL) and sizes the warp
 * halo over the larger of the two maps' magnitudes, so a device map that
 * differs from the host one cannot move a tap outside the staged tile.  Work
 * is ordered on cuda_stream; the call synchronises that stream twice (after
 * the check and at the end) and returns when <p, M p> is on the host.  The
 * message of a failure is readable with lfsr_last_error(NULL).  Only the
 * patch weights, the shared disparity map and the exact adjoint are
 * supported here (LFSR_WEIGHTS_PAPER, disparity_views,
 * LFSR_ADJOINT_BACKWARD_WARP and 16-bit precision return
 * LFSR_EUNSUPPORTED). */
#define LFSR_NOALLOC_MAX_TILES 4096
#define LFSR_NOALLOC_SCRATCH_BYTES (64 * 1024 + 256)

int lfsr_apply_normal_noalloc(const lfsr_params *params, const float *d_disparity,
                              const float *d_xw, const float *d_p, float *d_q,
                              double *pMp, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* LFSR_H */
