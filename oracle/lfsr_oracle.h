/*
 * FP64 CPU oracle for the light-field super-resolution ADMM of
 * "A GPU-Accelerated Light-field Super-resolution Framework Based on Mixed
 * Noise Model and Weighted Regularization" (arXiv 2206.05047).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, plain reference that
 * the CUDA path is checked against.  Only the test-suite, the smoke check and
 * the benchmark's CPU-baseline leg may load it; the product path never does.
 * It shares no code, header or table with the CUDA library.
 *
 * Images are row-major double arrays.  HR images are (zeta*H) x (zeta*W),
 * LR images H x W, view k = v*U + u.
 */
#ifndef LFSR_ORACLE_H
#define LFSR_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_problem {
  int U, V;               /* angular grid                                   */
  int H, W;               /* LR size                                        */
  int zeta;               /* scale factor                                   */
  int kb;                 /* blur kernel size (odd)                         */
  const double *blur;     /* kb*kb taps, K[a+r][b+r]                        */
  const double *disp;     /* HR disparity map on the reference grid         */
  double lambda1, lambda2;/* data-term weights (Eq. sr_fin)                 */
  double mu;              /* ADMM penalty (vartheta in Algorithm 1)         */
  int window, patch;      /* NLTV search window and patch (odd)             */
  double h;               /* NLTV filtering parameter                       */
  int cg_iters;           /* K of Algorithm 2                               */
  double cg_tol;          /* tau of Algorithm 2 (stop when pi <= tau)       */
  int freeze_weights;     /* test option: weights from x0, then fixed       */
  int n_views;            /* views used (0: all U*V)                        */
  const int *views;       /* their grid indices k = v*U + u, ascending      */
  /* weight scheme: 0 patch distance (exp(-pd/h^2)); 1 the paper's
   * spatial * edge * occlusion weights of Sec. 3.4 (each factor whose sigma
   * is 0 is 1)                                                             */
  int weight_scheme;
  double sigma_s, sigma_e;   /* spatial exp(-|d|^2/s_s), edge exp(-|grad x|^2/s_e) */
  double sigma_o1, sigma_o2; /* occlusion: boundary b, projection error p   */
  const double *proj_err;    /* HR projection error p(u); NULL: p = 0        */
  /* warps (Sec. 4.1): disp_views (optional, s_k x HR, data order) gives
   * W_k its own map omega_k on view k's grid (NULL: every W_k uses disp);
   * adjoint 0: W_k^T is the exact adjoint (scatter); 1: the paper's
   * backward warp by the reference map, (W_k^* g)(u) = g(u - theta_k
   * omega_0(u)) sampled bilinearly, which is not W_k's adjoint where the
   * disparity varies */
  const double *disp_views;
  int adjoint;
} orc_problem;

int    orc_num_threads(void);
void   orc_set_threads(int n);

/* geometry */
int    orc_num_dirs(const orc_problem *P);
void   orc_dirs(const orc_problem *P, int *di, int *dj);
/* Views: the data of view j (0 <= j < orc_num_views) is y_j; its grid index
 * is views[j] (or j for the full grid). */
int    orc_num_views(const orc_problem *P);
void   orc_view_theta(const orc_problem *P, int j, double *tu, double *tv);

/* degradation operators (Eq. sr_model_op, Sec. 4.1) and their adjoints */
void   orc_warp  (const orc_problem *P, int k, const double *x, double *out);
void   orc_warp_T(const orc_problem *P, int k, const double *g, double *out);
/* the paper's backward warp W_k^* (used for A_k^* when adjoint == 1) */
void   orc_warp_bw(const orc_problem *P, int k, const double *g, double *out);
void   orc_blur  (const orc_problem *P, const double *x, double *out);
void   orc_blur_T(const orc_problem *P, const double *g, double *out);
void   orc_down  (const orc_problem *P, const double *x, double *out);
void   orc_up    (const orc_problem *P, const double *g, double *out);
void   orc_A     (const orc_problem *P, int k, const double *x, double *out);
void   orc_A_T   (const orc_problem *P, int k, const double *g, double *out);
/* A_k's counterpart in the x-step: A_k^T, or W_k^* B^T D^T (adjoint == 1) */

/* weighted non-local TV (Eq. sr_reg, Sec. 4.1 wdg / wdd) */
void   orc_weights(const orc_problem *P, const double *x, double *w);
/* factors of the paper's weights (Sec. 3.4, Eq. weight_occ): the edge
 * factor e(u) of x and the occlusion factor o(u) of the disparity map and
 * projection error, HR images */
void   orc_edge_factor(const orc_problem *P, const double *x, double *e);
void   orc_occlusion_factor(const orc_problem *P, double *o);
void   orc_S  (const orc_problem *P, const double *w, const double *x, double *out);
void   orc_S_T(const orc_problem *P, const double *w, const double *g, double *out);

/* ADMM pieces */
void   orc_prox(long n, const double *u, double t, double *z);
void   orc_normal_apply(const orc_problem *P, const double *w, const double *p, double *q);
double orc_cost(const orc_problem *P, const double *y, const double *w, const double *x);
int    orc_cg(const orc_problem *P, const double *w, const double *v, double *x,
              int K, double tau, double *pi_out);
int    orc_admm(const orc_problem *P, const double *y, const double *x0, int N,
                double *x, double *wA, double *wS, double *diag);

#ifdef __cplusplus
}
#endif
#endif
