/*
 * FP64 CPU oracle for the light-field super-resolution ADMM of arXiv
 * 2206.05047.  TEST INFRASTRUCTURE ONLY: the plain, slow reference the CUDA
 * path is checked against.  Every operator is its textbook definition
 * written out over full images, in double precision, with fixed-order
 * reductions.  OpenMP only splits independent output pixels or views;
 * per-view results are summed in view order, so the result does not depend
 * on the thread count.
 *
 * Readings of the paper taken here (where it is silent or garbled):
 *  - B and W_k read zero outside the image; S_d pairs that leave the image
 *    are dropped (Sec. 4.1 gives no boundary rule).
 *  - W_k gathers bilinearly at z + theta_k * omega(z) from one HR disparity
 *    map on the reference grid; its adjoint is the exact scatter of the same
 *    taps (Sec. 4.1 states a forward / backward warp pair).
 *  - theta_k = (u - (U-1)/2, v - (V-1)/2); u shifts columns, v shifts rows.
 *  - NLTV weights: w_d(u) = exp(-pd/h^2), pd the mean over the patch of
 *    squared differences with clamp-to-edge reads; 0 if u+d leaves the
 *    image.  Directions: the full window minus the centre, raster order.
 *  - The paper's own weights (Sec. 3.4, weight_scheme 1) with exp(-...)
 *    where the paper prints exp(+...) for the spatial and edge factors;
 *    central differences for grad x, forward differences for the
 *    disparity gradient of the occlusion boundary b.
 *  - Compact form without the 1/sqrt(lambda2) scaling:
 *    F = [lambda1 A; S], b' = [lambda1 y; 0]; the normal matrix is
 *    (lambda2 + mu lambda1^2 / 2) sum_k A_k^T A_k + mu/2 sum_d S_d^T S_d.
 *  - Algorithm 2 as standard CG on M delta = -v, warm-started at x, run
 *    while pi > tau for at most K steps (the printed signs and loop test
 *    are inverted).
 *  - Per-view disparity maps (Sec. 4.1): omega_k lives on view k's HR grid
 *    and W_k gathers at z + theta_k omega_k(z).  The paper's backward warp
 *    samples at u - theta_k omega_0(u) (its printed formula repeats the
 *    same symbols on both sides).
 */
#include "lfsr_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define HR_H(P) ((P)->zeta * (P)->H)
#define HR_W(P) ((P)->zeta * (P)->W)

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_threads(int n) {
#ifdef _OPENMP
  omp_set_max_active_levels(1);
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* Views are split across threads and each operator call inside runs
 * serially: keep nested parallel regions off. */
__attribute__((constructor)) static void orc_init(void) {
#ifdef _OPENMP
  omp_set_max_active_levels(1);
#endif
}

static double *dalloc(long n) {
  double *p = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  return p;
}

/* ------------------------------------------------------------------ */
/* geometry                                                             */
/* ------------------------------------------------------------------ */

/* Direction set U of the weighted directional gradient (Sec. 4.1):
 * all offsets of the search window except the centre, raster order. */
int orc_num_dirs(const orc_problem *P) { return P->window * P->window - 1; }

void orc_dirs(const orc_problem *P, int *di, int *dj) {
  int r = (P->window - 1) / 2, n = 0;
  for (int a = -r; a <= r; ++a)
    for (int b = -r; b <= r; ++b) {
      if (a == 0 && b == 0) continue;
      di[n] = a;
      dj[n] = b;
      ++n;
    }
}

/* Angular offset of view k = v*U + u relative to the centre view. */
int orc_num_views(const orc_problem *P) {
  return (P->views && P->n_views > 0) ? P->n_views : P->U * P->V;
}

/* Angular offset of data view j: grid index k = views[j] (Sec. 6.1 uses a
 * subset of the grid, e.g. a star of 17 of 5 x 5 views). */
void orc_view_theta(const orc_problem *P, int j, double *tu, double *tv) {
  const int k = (P->views && P->n_views > 0) ? P->views[j] : j;
  int u = k % P->U, v = k / P->U;
  *tu = u - 0.5 * (P->U - 1);
  *tv = v - 0.5 * (P->V - 1);
}

/* ------------------------------------------------------------------ */
/* W_k: disparity warp (Sec. 4.1, forward warping function)             */
/* (W_k x)(i,j) = bilinear sample of x at (i + tv*w(i,j), j + tu*w(i,j)) */
/* ------------------------------------------------------------------ */
/* The disparity map W_k samples with: omega_k (disp_views) or the shared
 * reference map. */
static const double *warp_map(const orc_problem *P, int k) {
  return P->disp_views ? P->disp_views + (long)k * HR_H(P) * HR_W(P) : P->disp;
}

void orc_warp(const orc_problem *P, int k, const double *x, double *out) {
  const int Hh = HR_H(P), Wh = HR_W(P);
  const double *omk = warp_map(P, k);
  double tu, tv;
  orc_view_theta(P, k, &tu, &tv);
#pragma omp parallel for schedule(static)
  for (int i = 0; i < Hh; ++i)
    for (int j = 0; j < Wh; ++j) {
      double om = omk[(long)i * Wh + j];
      double sy = i + tv * om, sx = j + tu * om;
      double fy0 = floor(sy), fx0 = floor(sx);
      int i0 = (int)fy0, j0 = (int)fx0;
      double fy = sy - fy0, fx = sx - fx0;
      double acc = 0.0;
      for (int a = 0; a <= 1; ++a)
        for (int b = 0; b <= 1; ++b) {
          int ii = i0 + a, jj = j0 + b;
          if (ii < 0 || ii >= Hh || jj < 0 || jj >= Wh) continue;
          double wgt = (a ? fy : 1.0 - fy) * (b ? fx : 1.0 - fx);
          acc += wgt * x[(long)ii * Wh + jj];
        }
      out[(long)i * Wh + j] = acc;
    }
}

/* W_k^T: exact adjoint, scatter of the same bilinear taps (serial: the
 * scatter targets overlap). */
void orc_warp_T(const orc_problem *P, int k, const double *g, double *out) {
  const int Hh = HR_H(P), Wh = HR_W(P);
  const double *omk = warp_map(P, k);
  double tu, tv;
  orc_view_theta(P, k, &tu, &tv);
  memset(out, 0, sizeof(double) * (size_t)Hh * Wh);
  for (int i = 0; i < Hh; ++i)
    for (int j = 0; j < Wh; ++j) {
      double om = omk[(long)i * Wh + j];
      double sy = i + tv * om, sx = j + tu * om;
      double fy0 = floor(sy), fx0 = floor(sx);
      int i0 = (int)fy0, j0 = (int)fx0;
      double fy = sy - fy0, fx = sx - fx0;
      double val = g[(long)i * Wh + j];
      for (int a = 0; a <= 1; ++a)
        for (int b = 0; b <= 1; ++b) {
          int ii = i0 + a, jj = j0 + b;
          if (ii < 0 || ii >= Hh || jj < 0 || jj >= Wh) continue;
          double wgt = (a ? fy : 1.0 - fy) * (b ? fx : 1.0 - fx);
          out[(long)ii * Wh + jj] += wgt * val;
        }
    }
}

/* The paper's backward warp (Sec. 4.1): the reference pixel u is seen in
 * view k at u - theta_k omega_0(u); (W_k^* g)(u) samples g there with the
 * bilinear taps of orc_warp, zero outside the image. */
void orc_warp_bw(const orc_problem *P, int k, const double *g, double *out) {
  const int Hh = HR_H(P), Wh = HR_W(P);
  double tu, tv;
  orc_view_theta(P, k, &tu, &tv);
#pragma omp parallel for schedule(static)
  for (int i = 0; i < Hh; ++i)
    for (int j = 0; j < Wh; ++j) {
      double om = P->disp[(long)i * Wh + j];
      double sy = i - tv * om, sx = j - tu * om;
      double fy0 = floor(sy), fx0 = floor(sx);
      int i0 = (int)fy0, j0 = (int)fx0;
      double fy = sy - fy0, fx = sx - fx0;
      double acc = 0.0;
      for (int a = 0; a <= 1; ++a)
        for (int b = 0; b <= 1; ++b) {
          int ii = i0 + a, jj = j0 + b;
          if (ii < 0 || ii >= Hh || jj < 0 || jj >= Wh) continue;
          double wgt = (a ? fy : 1.0 - fy) * (b ? fx : 1.0 - fx);
          acc += wgt * g[(long)ii * Wh + jj];
        }
      out[(long)i * Wh + j] = acc;
    }
}

/* ------------------------------------------------------------------ */
/* B: kb x kb correlation with zero padding (Sec. 4.1 blur) and B^T.    */
/* ------------------------------------------------------------------ */
void orc_blur(const orc_problem *P, const double *x, double *out) {
  const int Hh = HR_H(P), Wh = HR_W(P), kb = P->kb, r = (P->kb - 1) / 2;
#pragma omp parallel for schedule(static)
  for (int i = 0; i < Hh; ++i)
    for (int j = 0; j < Wh; ++j) {
      double acc = 0.0;
      for (int a = -r; a <= r; ++a)
        for (int b = -r; b <= r; ++b) {
          int ii = i + a, jj = j + b;
          if (ii < 0 || ii >= Hh || jj < 0 || jj >= Wh) continue;
          acc += P->blur[(a + r) * kb + (b + r)] * x[(long)ii * Wh + jj];
        }
      out[(long)i * Wh + j] = acc;
    }
}

void orc_blur_T(const orc_problem *P, const double *g, double *out) {
  const int Hh = HR_H(P), Wh = HR_W(P), kb = P->kb, r = (P->kb - 1) / 2;
#pragma omp parallel for schedule(static)
  for (int i = 0; i < Hh; ++i)
    for (int j = 0; j < Wh; ++j) {
      double acc = 0.0;
      for (int a = -r; a <= r; ++a)
        for (int b = -r; b <= r; ++b) {
          int ii = i - a, jj = j - b;
          if (ii < 0 || ii >= Hh || jj < 0 || jj >= Wh) continue;
          acc += P->blur[(a + r) * kb + (b + r)] * g[(long)ii * Wh + jj];
        }
      out[(long)i * Wh + j] = acc;
    }
}

/* ------------------------------------------------------------------ */
/* D: keep the top-left pixel of each zeta x zeta block; D^T: put back  */
/* (Sec. 4.1 down-sampling).                                            */
/* ------------------------------------------------------------------ */
void orc_down(const orc_problem *P, const double *x, double *out) {
  const int Wh = HR_W(P), z = P->zeta;
  for (int i = 0; i < P->H; ++i)
    for (int j = 0; j < P->W; ++j)
      out[(long)i * P->W + j] = x[(long)(z * i) * Wh + z * j];
}

void orc_up(const orc_problem *P, const double *g, double *out) {
  const int Hh = HR_H(P), Wh = HR_W(P), z = P->zeta;
  memset(out, 0, sizeof(double) * (size_t)Hh * Wh);
  for (int i = 0; i < P->H; ++i)
    for (int j = 0; j < P->W; ++j)
      out[(long)(z * i) * Wh + z * j] = g[(long)i * P->W + j];
}

/* A_k = D B W_k (Eq. sr_model_vec) and A_k^T = W_k^T B^T D^T. */
void orc_A(const orc_problem *P, int k, const double *x, double *out) {
  long p = (long)HR_H(P) * HR_W(P);
  double *t1 = dalloc(p), *t2 = dalloc(p);
  orc_warp(P, k, x, t1);
  orc_blur(P, t1, t2);
  orc_down(P, t2, out);
  free(t1);
  free(t2);
}

void orc_A_T(const orc_problem *P, int k, const double *g, double *out) {
  long p = (long)HR_H(P) * HR_W(P);
  double *t1 = dalloc(p), *t2 = dalloc(p);
  orc_up(P, g, t1);
  orc_blur_T(P, t1, t2);
  orc_warp_T(P, k, t2, out);
  free(t1);
  free(t2);
}

/* ------------------------------------------------------------------ */
/* NLTV weights (Eq. sr_reg; patch-distance weights of non-local TV),   */
/* w[d*p + u].                                                          */
/* ------------------------------------------------------------------ */
static inline int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

static void patch_weights(const orc_problem *P, const double *x, double *w) {
  const int Hh = HR_H(P), Wh = HR_W(P), sd = orc_num_dirs(P);
  const int rp = (P->patch - 1) / 2;
  const long p = (long)Hh * Wh;
  const double inv_h2 = 1.0 / (P->h * P->h);
  const double inv_np = 1.0 / (double)(P->patch * P->patch);
  int *di = (int *)malloc(sizeof(int) * sd), *dj = (int *)malloc(sizeof(int) * sd);
  orc_dirs(P, di, dj);
  for (int d = 0; d < sd; ++d) {
#pragma omp parallel for schedule(static)
    for (int i = 0; i < Hh; ++i)
      for (int j = 0; j < Wh; ++j) {
        int ni = i + di[d], nj = j + dj[d];
        double val = 0.0;
        if (ni >= 0 && ni < Hh && nj >= 0 && nj < Wh) {
          double pd = 0.0;
          for (int a = -rp; a <= rp; ++a)
            for (int b = -rp; b <= rp; ++b) {
              double xa = x[(long)clampi(i + a, 0, Hh - 1) * Wh + clampi(j + b, 0, Wh - 1)];
              double xb = x[(long)clampi(ni + a, 0, Hh - 1) * Wh + clampi(nj + b, 0, Wh - 1)];
              pd += (xa - xb) * (xa - xb);
            }
          pd *= inv_np;
          val = exp(-pd * inv_h2);
        }
        w[d * p + (long)i * Wh + j] = val;
      }
  }
  free(di);
  free(dj);
}

/* Edge factor of the paper's weights (Sec. 3.4): e(u) = exp(-|grad x(u)|^2
 * / sigma_e), grad x by central differences (x(i+1,j) - x(i-1,j)) / 2 and
 * (x(i,j+1) - x(i,j-1)) / 2 with clamp-to-edge indices; 1 if sigma_e = 0. */
void orc_edge_factor(const orc_problem *P, const double *x, double *e) {
  const int Hh = HR_H(P), Wh = HR_W(P);
#pragma omp parallel for schedule(static)
  for (int i = 0; i < Hh; ++i)
    for (int j = 0; j < Wh; ++j) {
      double val = 1.0;
      if (P->sigma_e > 0.0) {
        const double gi = 0.5 * (x[(long)clampi(i + 1, 0, Hh - 1) * Wh + j] -
                                 x[(long)clampi(i - 1, 0, Hh - 1) * Wh + j]);
        const double gj = 0.5 * (x[(long)i * Wh + clampi(j + 1, 0, Wh - 1)] -
                                 x[(long)i * Wh + clampi(j - 1, 0, Wh - 1)]);
        val = exp(-(gi * gi + gj * gj) / P->sigma_e);
      }
      e[(long)i * Wh + j] = val;
    }
}

/* Occlusion factor (Sec. 3.4, Eq. weight_occ):
 *   o(u) = exp(-b(u)^2 / (2 sigma_o1^2)) exp(-p(u)^2 / (2 sigma_o2^2)),
 * b(u) the sum of the two components of the disparity gradient when that
 * sum is negative, else 0; the gradient by one-sided (forward) differences
 * omega(i+1,j) - omega(i,j) and omega(i,j+1) - omega(i,j), 0 across the last
 * row / column.  p(u) is the given projection error (0 without one).  A
 * factor whose sigma is 0 is 1. */
void orc_occlusion_factor(const orc_problem *P, double *o) {
  const int Hh = HR_H(P), Wh = HR_W(P);
  const double *om = P->disp;
#pragma omp parallel for schedule(static)
  for (int i = 0; i < Hh; ++i)
    for (int j = 0; j < Wh; ++j) {
      const long u = (long)i * Wh + j;
      double val = 1.0;
      if (P->sigma_o1 > 0.0) {
        const double gi = (i + 1 < Hh) ? om[u + Wh] - om[u] : 0.0;
        const double gj = (j + 1 < Wh) ? om[u + 1] - om[u] : 0.0;
        const double b = (gi + gj < 0.0) ? gi + gj : 0.0;
        val *= exp(-b * b / (2.0 * P->sigma_o1 * P->sigma_o1));
      }
      if (P->sigma_o2 > 0.0 && P->proj_err) {
        const double pe = P->proj_err[u];
        val *= exp(-pe * pe / (2.0 * P->sigma_o2 * P->sigma_o2));
      }
      o[u] = val;
    }
}

/* The paper's weights (Sec. 3.4): w_d(u) = w_s(d) e(u) o(u) with the
 * spatial factor w_s(d) = exp(-|d|^2 / sigma_s) (1 if sigma_s = 0); 0 if
 * u+d leaves the image.  Unlike the patch weights they are not symmetric in
 * the pixel pair: w_{-d}(u+d) = w_s(d) e(u+d) o(u+d). */
static void paper_weights(const orc_problem *P, const double *x, double *w) {
  const int Hh = HR_H(P), Wh = HR_W(P), sd = orc_num_dirs(P);
  const long p = (long)Hh * Wh;
  double *e = dalloc(p), *o = dalloc(p);
  int *di = (int *)malloc(sizeof(int) * sd), *dj = (int *)malloc(sizeof(int) * sd);
  orc_dirs(P, di, dj);
  orc_edge_factor(P, x, e);
  orc_occlusion_factor(P, o);
  for (int d = 0; d < sd; ++d) {
    const double ws = P->sigma_s > 0.0 ? exp(-(double)(di[d] * di[d] + dj[d] * dj[d]) / P->sigma_s)
                                       : 1.0;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < Hh; ++i)
      for (int j = 0; j < Wh; ++j) {
        const int ni = i + di[d], nj = j + dj[d];
        const long u = (long)i * Wh + j;
        w[d * p + u] = (ni >= 0 && ni < Hh && nj >= 0 && nj < Wh) ? ws * e[u] * o[u] : 0.0;
      }
  }
  free(e);
  free(o);
  free(di);
  free(dj);
}

void orc_weights(const orc_problem *P, const double *x, double *w) {
  if (P->weight_scheme == 1)
    paper_weights(P, x, w);
  else
    patch_weights(P, x, w);
}

/* S: weighted directional gradient G_d(u) = w_d(u) (x(u) - x(u+d))
 * (Sec. 4.1, wdg); pairs leaving the image give 0. */
void orc_S(const orc_problem *P, const double *w, const double *x, double *out) {
  const int Hh = HR_H(P), Wh = HR_W(P), sd = orc_num_dirs(P);
  const long p = (long)Hh * Wh;
  int *di = (int *)malloc(sizeof(int) * sd), *dj = (int *)malloc(sizeof(int) * sd);
  orc_dirs(P, di, dj);
  for (int d = 0; d < sd; ++d) {
#pragma omp parallel for schedule(static)
    for (int i = 0; i < Hh; ++i)
      for (int j = 0; j < Wh; ++j) {
        int ni = i + di[d], nj = j + dj[d];
        double val = 0.0;
        if (ni >= 0 && ni < Hh && nj >= 0 && nj < Wh)
          val = w[d * p + (long)i * Wh + j] * (x[(long)i * Wh + j] - x[(long)ni * Wh + nj]);
        out[d * p + (long)i * Wh + j] = val;
      }
  }
  free(di);
  free(dj);
}

/* S^T: weighted directional divergence (Sec. 4.1, wdd), the exact adjoint
 * of S:  (S_d^T g)(u) = w_d(u) g_d(u) [u+d in image]
 *                      - w_d(u-d) g_d(u-d) [u-d in image].  */
void orc_S_T(const orc_problem *P, const double *w, const double *g, double *out) {
  const int Hh = HR_H(P), Wh = HR_W(P), sd = orc_num_dirs(P);
  const long p = (long)Hh * Wh;
  int *di = (int *)malloc(sizeof(int) * sd), *dj = (int *)malloc(sizeof(int) * sd);
  orc_dirs(P, di, dj);
#pragma omp parallel for schedule(static)
  for (int i = 0; i < Hh; ++i)
    for (int j = 0; j < Wh; ++j) {
      double acc = 0.0;
      for (int d = 0; d < sd; ++d) {
        int ni = i + di[d], nj = j + dj[d];
        if (ni >= 0 && ni < Hh && nj >= 0 && nj < Wh)
          acc += w[d * p + (long)i * Wh + j] * g[d * p + (long)i * Wh + j];
        int mi = i - di[d], mj = j - dj[d];
        if (mi >= 0 && mi < Hh && mj >= 0 && mj < Wh)
          acc -= w[d * p + (long)mi * Wh + mj] * g[d * p + (long)mi * Wh + mj];
      }
      out[(long)i * Wh + j] = acc;
    }
  free(di);
  free(dj);
}

/* ------------------------------------------------------------------ */
/* ADMM                                                                 */
/* ------------------------------------------------------------------ */

/* Soft threshold, the closed-form prox of t*|.|_1 (Eq. sr_l1l2l1_prox). */
void orc_prox(long n, const double *u, double t, double *z) {
  for (long i = 0; i < n; ++i) {
    double a = fabs(u[i]) - t;
    double s = (u[i] > 0.0) ? 1.0 : ((u[i] < 0.0) ? -1.0 : 0.0);
    z[i] = (a > 0.0 ? a : 0.0) * s;
  }
}

/* out = sum_k A_k^T g_k.  Views run in parallel (each operator call is
 * serial inside, nested parallelism is off), per-view buffers are summed in
 * view order. */
/* A_k^* g: the exact adjoint A_k^T g, or with the paper's backward warp
 * (adjoint == 1) W_k^* B^T D^T g. */
static void A_star(const orc_problem *P, int k, const double *g, double *out) {
  if (P->adjoint != 1) {
    orc_A_T(P, k, g, out);
    return;
  }
  long p = (long)HR_H(P) * HR_W(P);
  double *t1 = dalloc(p), *t2 = dalloc(p);
  orc_up(P, g, t1);
  orc_blur_T(P, t1, t2);
  orc_warp_bw(P, k, t2, out);
  free(t1);
  free(t2);
}

/* out = sum_k A_k^* g_k (the x-step's transposed data operator). */
static void sum_AT(const orc_problem *P, const double *g, double *out) {
  const int sk = orc_num_views(P);
  const long p = (long)HR_H(P) * HR_W(P), q = (long)P->H * P->W;
  double *buf = dalloc(p * sk);
#pragma omp parallel for schedule(dynamic, 1)
  for (int k = 0; k < sk; ++k) A_star(P, k, g + k * q, buf + k * p);
#pragma omp parallel for schedule(static)
  for (long i = 0; i < p; ++i) {
    double acc = 0.0;
    for (int k = 0; k < sk; ++k) acc += buf[k * p + i];
    out[i] = acc;
  }
  free(buf);
}

/* out[k] = A_k x for every view. */
static void all_A(const orc_problem *P, const double *x, double *out) {
  const int sk = orc_num_views(P);
  const long q = (long)P->H * P->W;
#pragma omp parallel for schedule(dynamic, 1)
  for (int k = 0; k < sk; ++k) orc_A(P, k, x, out + k * q);
}

/* M p with M = (lambda2 + mu lambda1^2/2) sum_k A_k^T A_k + mu/2 S^T S,
 * the normal matrix G^T G of the x-step least squares (Sec. 4.2); with the
 * paper's backward warp A_k^T becomes A_k^* and M is not symmetric where
 * the disparity varies (CG then runs as printed, on that M). */
void orc_normal_apply(const orc_problem *P, const double *w, const double *p, double *q) {
  const int sk = orc_num_views(P), sd = orc_num_dirs(P);
  const long np = (long)HR_H(P) * HR_W(P), nq = (long)P->H * P->W;
  const double cA = P->lambda2 + 0.5 * P->mu * P->lambda1 * P->lambda1;
  double *Ap = dalloc(nq * sk), *AtAp = dalloc(np), *Sp = dalloc(np * sd), *StSp = dalloc(np);
  all_A(P, p, Ap);
  sum_AT(P, Ap, AtAp);
  orc_S(P, w, p, Sp);
  orc_S_T(P, w, Sp, StSp);
  for (long i = 0; i < np; ++i) q[i] = cA * AtAp[i] + 0.5 * P->mu * StSp[i];
  free(Ap);
  free(AtAp);
  free(Sp);
  free(StSp);
}

/* J(x) of Eq. sr_fin with the given weights. */
double orc_cost(const orc_problem *P, const double *y, const double *w, const double *x) {
  const int sk = orc_num_views(P), sd = orc_num_dirs(P);
  const long np = (long)HR_H(P) * HR_W(P), nq = (long)P->H * P->W;
  double *Ax = dalloc(nq * sk), *Sx = dalloc(np * sd);
  all_A(P, x, Ax);
  orc_S(P, w, x, Sx);
  double l1 = 0.0, l2 = 0.0, tv = 0.0;
  for (long i = 0; i < nq * sk; ++i) {
    double r = Ax[i] - y[i];
    l1 += fabs(r);
    l2 += r * r;
  }
  for (long i = 0; i < np * sd; ++i) tv += fabs(Sx[i]);
  free(Ax);
  free(Sx);
  return P->lambda1 * l1 + P->lambda2 * l2 + tv;
}

static double dot(long n, const double *a, const double *b) {
  double s = 0.0;
  for (long i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

/* x-step (Algorithm 2): CG on M delta = -v warm-started at x (x is
 * updated in place).  Returns the number of steps taken. */
int orc_cg(const orc_problem *P, const double *w, const double *v, double *x,
           int K, double tau, double *pi_out) {
  const long np = (long)HR_H(P) * HR_W(P);
  double *r = dalloc(np), *pp = dalloc(np), *q = dalloc(np);
  for (long i = 0; i < np; ++i) {
    r[i] = -v[i];
    pp[i] = r[i];
  }
  double pi = dot(np, r, r);
  int steps = 0;
  for (int k = 0; k < K; ++k) {
    if (!(pi > tau)) break;
    orc_normal_apply(P, w, pp, q);
    double pq = dot(np, pp, q);
    double alpha = pi / pq;
    for (long i = 0; i < np; ++i) {
      x[i] += alpha * pp[i];
      r[i] -= alpha * q[i];
    }
    double pi_new = dot(np, r, r);
    double beta = pi_new / pi;
    for (long i = 0; i < np; ++i) pp[i] = r[i] + beta * pp[i];
    pi = pi_new;
    ++steps;
  }
  if (pi_out) *pi_out = pi;
  free(r);
  free(pp);
  free(q);
  return steps;
}

/* Algorithm 1 (rotated ADMM: z-step, w-step, then x-step), scaled dual.
 * State in/out: x (HR), wA (s_k*q, data rows), wS (s_d*p, regulariser
 * rows).  Starting from x = x0 and wA = wS = 0 gives the solver of
 * Algorithm 1.  diag (N x 5, may be NULL): ||w_n - w_{n-1}||^2,
 * ||z_n - z_{n-1}||^2 (NaN at n = 1), J(x_n) with iteration n's weights,
 * final CG pi, CG steps. */
int orc_admm(const orc_problem *P, const double *y, const double *x0, int N,
             double *x, double *wA, double *wS, double *diag) {
  const int sk = orc_num_views(P), sd = orc_num_dirs(P);
  const long np = (long)HR_H(P) * HR_W(P), nq = (long)P->H * P->W;
  const long nA = nq * sk, nS = np * sd;
  const double t = 1.0 / P->mu;
  double *w = dalloc(nS), *a = dalloc(nA), *uA = dalloc(nA), *uS = dalloc(nS);
  double *zA = dalloc(nA), *zS = dalloc(nS), *zA_prev = dalloc(nA), *zS_prev = dalloc(nS);
  double *fA = dalloc(nA), *fS = dalloc(nS), *gA = dalloc(nA), *v = dalloc(np);
  double *t1 = dalloc(np), *Sx = dalloc(nS);
  if (x != x0) memcpy(x, x0, sizeof(double) * (size_t)np);
  for (int n = 1; n <= N; ++n) {
    /* weights from x^(n-1), recomputed every iteration */
    if (!P->freeze_weights || n == 1) orc_weights(P, x, w);
    /* a := A x - b ; u := F x - b' + w   (Algorithm 1, lines 4-5) */
    all_A(P, x, a);
    for (long i = 0; i < nA; ++i) {
      a[i] -= y[i];
      uA[i] = P->lambda1 * a[i] + wA[i];
    }
    orc_S(P, w, x, Sx);
    for (long i = 0; i < nS; ++i) uS[i] = Sx[i] + wS[i];
    /* z := prox(u); w_new := u - z; f := 2 w_new - w_old  (lines 6-8) */
    orc_prox(nA, uA, t, zA);
    orc_prox(nS, uS, t, zS);
    double dw2 = 0.0, dz2 = 0.0;
    for (long i = 0; i < nA; ++i) {
      double wn = uA[i] - zA[i];
      fA[i] = 2.0 * wn - wA[i];
      dw2 += (wn - wA[i]) * (wn - wA[i]);
      if (n > 1) dz2 += (zA[i] - zA_prev[i]) * (zA[i] - zA_prev[i]);
      wA[i] = wn;
    }
    for (long i = 0; i < nS; ++i) {
      double wn = uS[i] - zS[i];
      fS[i] = 2.0 * wn - wS[i];
      dw2 += (wn - wS[i]) * (wn - wS[i]);
      if (n > 1) dz2 += (zS[i] - zS_prev[i]) * (zS[i] - zS_prev[i]);
      wS[i] = wn;
    }
    /* v := A^T a + mu/2 F^T f  (line 9), with A = sqrt(lambda2)[A_k],
     * F = [lambda1 A_k ; S] */
    for (long i = 0; i < nA; ++i) gA[i] = P->lambda2 * a[i] + 0.5 * P->mu * P->lambda1 * fA[i];
    sum_AT(P, gA, v);
    orc_S_T(P, w, fS, t1);
    for (long i = 0; i < np; ++i) v[i] += 0.5 * P->mu * t1[i];
    /* x := xstep(v, x)  (line 10, Algorithm 2) */
    double pi = 0.0;
    int steps = orc_cg(P, w, v, x, P->cg_iters, P->cg_tol, &pi);
    if (diag) {
      diag[(n - 1) * 5 + 0] = dw2;
      diag[(n - 1) * 5 + 1] = (n > 1) ? dz2 : NAN;
      diag[(n - 1) * 5 + 2] = orc_cost(P, y, w, x);
      diag[(n - 1) * 5 + 3] = pi;
      diag[(n - 1) * 5 + 4] = steps;
    }
    memcpy(zA_prev, zA, sizeof(double) * (size_t)nA);
    memcpy(zS_prev, zS, sizeof(double) * (size_t)nS);
  }
  free(w); free(a); free(uA); free(uS); free(zA); free(zS); free(zA_prev); free(zS_prev);
  free(fA); free(fS); free(gA); free(v); free(t1); free(Sx);
  return 0;
}
