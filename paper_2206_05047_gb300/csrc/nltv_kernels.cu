// Weighted non-local TV: NLTV weights, weighted directional gradient (wdg)
// and divergence (wdd) of Sec. 4.1 / Eq. sr_reg, in three modes:
//   NL_BLOCK    regulariser rows of Algorithm 1: u = S x + w, w' = clamp(u),
//               f = 2 w' - w, v := mu/2 S^T f (stores v; the data block adds
//               its part afterwards)
//   NL_APPLY    x-step matvec part: q := mu/2 S^T S p and <p, .> (stores q;
//               the operator kernel adds cA sum_k A_k^T A_k p afterwards);
//               optionally first forms the CG direction p = r + beta p_old
//   NL_WEIGHTS  the weights themselves, canonical [d][u] layout
//
// Two weight schemes (g.wscheme): the patch distance below, and the paper's
// directed weights w_d(u) = w_s(d) g(u) of Sec. 3.4 (g = edge factor of x
// times the stored occlusion factor, staged over the tile + window halo).
// The edge (u, u+d) then carries w_a = w_s(d) g(u) and w_b = w_s(d) g(u+d):
// c = w_a g_a - w_b g_b and, for S^T S, the pair weight (w_a^2 + w_b^2) / 2
// in place of w^2.
//
// Patch weights are symmetric in the pixel pair: w_d(u) = w_{-d}(u+d) (the
// patch distance is symmetric and clamped reads use the same pixel pairs).  The
// kernel therefore visits each undirected edge (u, u+d) once, for d in the
// half window H = {d : d before 0 in raster order}, and keeps both duals
// of the edge -- direction d at u and direction -d at u+d -- side by side
// ("pair layout": [idx][0][u], [idx][1][u]).  In this form
//   sum_d S_d^T g_d (u) = sum_{d in H} c(u) - c(u-d),  c(v) = w (g_a - g_b),
//   sum_d S_d^T S_d p (u) = 2 sum_{d in H} e(u) - e(u-d), e(v) = w^2 (p(v)-p(v+d)),
// a gather over the tile and its (tile - d) halo with no atomics.
//
// Per tile and direction: squared patch differences and their box sums run
// in shared memory over the tile + halo (separable 2 r_p + 1 sums), then
// the edge quantity c or e on tile U (tile - d), then the gather.
#include "lfsr_device.cuh"

namespace lfsr {

constexpr int NL_THREADS = 256;
constexpr int NL_WARPS = NL_THREADS / 32;
constexpr int NL_TH = 32;
constexpr int NL_TW = 32;
constexpr int NL_PIX = NL_TH * NL_TW / NL_THREADS;   // owned pixels per thread

template <int MODE>
__global__ void __launch_bounds__(NL_THREADS)
k_nltv(const Geom g, const NlPlan P, const NlArgs a) {
  extern __shared__ __align__(16) float smem[];
  if (a.check_done && a.sc->cg_done) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wr = g.win_r, pr = g.patch_r;
  const int Hh = g.Hh, Wh = g.Wh;
  const size_t p = (size_t)Hh * Wh;
  const int ty = blockIdx.x / P.tiles_x, tx = blockIdx.x - ty * P.tiles_x;
  const int i0 = ty * NL_TH, j0 = tx * NL_TW;
  const int TRr = min(NL_TH, Hh - i0), TRc = min(NL_TW, Wh - j0);
  const int hx = wr + pr;                       // x halo
  const int NXc = P.NXc;
  float* sX = smem;                             // NXr x NXc, clamp-to-edge x
  float* sP = sX + P.NXr * NXc;                 // (TH+2wr) x (TW+2wr), APPLY only
  const int NPc = NL_TW + 2 * wr;
  float* sQ = sP + (NL_TH + 2 * wr) * NPc;      // box sums, NQr x NQc
  float* sC = sQ + P.NQr * P.NQc;               // edge quantity, NQr x NQc
  float* sG = sC + P.NQr * P.NQc;               // paper weights: g over tile + wr
  const bool paper = g.wscheme == WS_PAPER;     // (then pr = 1: x halo wr + 1)

  // stage x (clamped) and, for APPLY, the CG direction (zero outside)
  for (int rr = warp; rr < P.NXr; rr += NL_WARPS) {
    const int hi = clampi(i0 - hx + rr, 0, Hh - 1);
    for (int cc = lane; cc < NXc; cc += 32) {
      const int hj = clampi(j0 - hx + cc, 0, Wh - 1);
      sX[rr * NXc + cc] = __ldg(a.x + (size_t)hi * Wh + hj);
    }
  }
  if (MODE == NL_APPLY) {
    const int first = a.sc->cg_first;
    const float beta = (float)a.sc->beta;
    for (int rr = warp; rr < NL_TH + 2 * wr; rr += NL_WARPS) {
      const int hi = i0 - wr + rr;
      const bool row_in = hi >= 0 && hi < Hh;
      for (int cc = lane; cc < NPc; cc += 32) {
        const int hj = j0 - wr + cc;
        float v = 0.f;
        if (row_in && hj >= 0 && hj < Wh) {
          const size_t gi = (size_t)hi * Wh + hj;
          if (a.use_beta) {
            v = __ldg(a.r + gi);
            if (!first) v = fmaf(beta, __ldg(a.p_old + gi), v);
            if (rr >= wr && rr < wr + TRr && cc >= wr && cc < wr + TRc) a.p_new[gi] = v;
          } else {
            v = __ldg(a.p_old + gi);
          }
        }
        sP[rr * NPc + cc] = v;
      }
    }
  }
  __syncthreads();
  if (paper) {
    // g(v) = exp(-|grad x(v)|^2 / sigma_e) o(v), central differences of the
    // clamped x; 0 outside the image (read only by dropped edges)
    for (int rr = warp; rr < NL_TH + 2 * wr; rr += NL_WARPS) {
      const int vi = i0 - wr + rr;
      for (int cc = lane; cc < NPc; cc += 32) {
        const int vj = j0 - wr + cc;
        float gv = 0.f;
        if (vi >= 0 && vi < Hh && vj >= 0 && vj < Wh) {
          gv = __ldg(a.occ + (size_t)vi * Wh + vj);
          if (g.inv_sig_e > 0.f) {
            const float* xc = sX + (rr + pr) * NXc + (cc + pr);
            const float gi = 0.5f * (xc[NXc] - xc[-NXc]);
            const float gj = 0.5f * (xc[1] - xc[-1]);
            gv *= expf(-fmaf(gi, gi, gj * gj) * g.inv_sig_e);
          }
        }
        sG[rr * NPc + cc] = gv;
      }
    }
    __syncthreads();
  }

  float acc[NL_PIX];
#pragma unroll
  for (int m = 0; m < NL_PIX; ++m) acc[m] = 0.f;
  double part = 0.0;
  const int sd = 2 * g.sh;

  for (int idx = 0; idx < g.sh; ++idx) {
    const int di = g.di[idx], dj = g.dj[idx];   // di <= 0
    // E_d = tile U (tile - d), origin (er0, ec0) relative to (i0, j0)
    const int er0 = 0, ec0 = min(0, -dj);
    const int ne_r = TRr - di, ne_c = TRc + (dj < 0 ? -dj : dj);
    const float ws = paper ? expf(-(float)(di * di + dj * dj) * g.inv_sig_s) : 1.f;
    // 1. horizontal box sums of squared patch differences, rows of E_d +- pr
    const int nq_r = paper ? 0 : ne_r + 2 * pr;
    for (int qa = warp; qa < nq_r; qa += NL_WARPS) {
      const int xr = er0 - pr + qa + hx;        // row in sX of v
      const float* rowA = sX + xr * NXc;
      const float* rowB = sX + (xr + di) * NXc;
      for (int qc = lane; qc < ne_c; qc += 32) {
        const int xc = ec0 + qc + hx - pr;
        float s = 0.f;
        for (int b = 0; b <= 2 * pr; ++b) {
          const float dlt = rowA[xc + b] - rowB[xc + b + dj];
          s = fmaf(dlt, dlt, s);
        }
        sQ[qa * P.NQc + qc] = s;
      }
    }
    __syncthreads();
    // 2. vertical box sums -> weight -> edge quantity on E_d
    for (int ea = warp; ea < ne_r; ea += NL_WARPS) {
      const int vi = i0 + er0 + ea;
      for (int ec = lane; ec < ne_c; ec += 32) {
        const int vj = j0 + ec0 + ec;
        const bool v_in = vi >= 0 && vi < Hh && vj >= 0 && vj < Wh;
        const bool valid = v_in && (vi + di >= 0) && (vi + di < Hh) && (vj + dj >= 0) && (vj + dj < Wh);
        float w = 0.f, w_a = 0.f, w_b = 0.f;   // patch: w_a = w_b = w
        if (paper) {
          if (valid) {
            const float* gv = sG + (er0 + ea + wr) * NPc + (ec0 + ec + wr);
            w_a = ws * gv[0];
            w_b = ws * gv[di * NPc + dj];
          }
        } else {
          float pd = 0.f;
          for (int b = 0; b <= 2 * pr; ++b) pd += sQ[(ea + b) * P.NQc + ec];
          w = valid ? expf(-pd * g.inv_np * g.inv_h2) : 0.f;
          w_a = w_b = w;
        }
        const bool own = ea < TRr && (ec + ec0) >= 0 && (ec + ec0) < TRc;
        float cval = 0.f;
        if (MODE == NL_BLOCK) {
          if (v_in) {
            const size_t gi = (size_t)vi * Wh + vj;
            const float wa = ld_kind(a.wS_old, (size_t)(2 * idx) * p + gi, g.st);
            const float wb = ld_kind(a.wS_old, (size_t)(2 * idx + 1) * p + gi, g.st);
            const int xr = er0 + ea + hx, xc = ec0 + ec + hx;
            const float diff = valid ? (sX[xr * NXc + xc] - sX[(xr + di) * NXc + xc + dj]) : 0.f;
            const float ua = fmaf(w_a, diff, wa);        // (S_d x)(v) + w
            const float ub = fmaf(-w_b, diff, wb);       // (S_-d x)(v+d) + w
            const float an = fminf(fmaxf(ua, -g.thr), g.thr);
            const float bn = fminf(fmaxf(ub, -g.thr), g.thr);
            const float fa = 2.f * an - wa, fb = 2.f * bn - wb;
            cval = paper ? fmaf(w_a, fa, -w_b * fb) : w * (fa - fb);
            if (own) {
              st_kind(a.wS_new, (size_t)(2 * idx) * p + gi, g.st, an);
              st_kind(a.wS_new, (size_t)(2 * idx + 1) * p + gi, g.st, bn);
              const double da = (double)an - wa, db = (double)bn - wb;
              part += da * da + db * db;
            }
          }
        } else if (MODE == NL_APPLY) {
          const int pr_ = er0 + ea + wr, pc_ = ec0 + ec + wr;
          const float dp = sP[pr_ * NPc + pc_] - sP[(pr_ + di) * NPc + pc_ + dj];
          const float w2 = paper ? 0.5f * fmaf(w_a, w_a, w_b * w_b) : w * w;
          cval = w2 * dp;
          if (own) part += (double)w2 * (double)dp * (double)dp;
        } else {  // NL_WEIGHTS
          if (own) {
            const size_t gi = (size_t)vi * Wh + vj;
            a.out[(size_t)idx * p + gi] = w_a;
            if (valid) a.out[(size_t)(sd - 1 - idx) * p + (size_t)(vi + di) * Wh + (vj + dj)] = w_b;
          }
        }
        sC[ea * P.NQc + ec] = cval;
      }
    }
    __syncthreads();
    // 3. gather: acc(u) += c(u) - c(u - d)
    if (MODE != NL_WEIGHTS) {
#pragma unroll
      for (int m = 0; m < NL_PIX; ++m) {
        const int iu = warp + m * NL_WARPS, ju = lane;
        if (iu < TRr && ju < TRc) {
          const int ca = iu - er0, cc = ju - ec0;
          acc[m] += sC[ca * P.NQc + cc] - sC[(ca - di) * P.NQc + (cc - dj)];
        }
      }
    }
    __syncthreads();
  }

  if (MODE != NL_WEIGHTS) {
    const float scale = (MODE == NL_BLOCK) ? 0.5f * g.mu : g.mu;
#pragma unroll
    for (int m = 0; m < NL_PIX; ++m) {
      const int iu = warp + m * NL_WARPS, ju = lane;
      if (iu < TRr && ju < TRc) a.out[(size_t)(i0 + iu) * Wh + (j0 + ju)] = scale * acc[m];
    }
    const int slot = (MODE == NL_BLOCK) ? RED_DW_S : RED_NLTV;
    double total = 0.0;
    if (grid_sum_last<NL_THREADS>(part, a.partials, &a.sc->counter[slot], &total) &&
        threadIdx.x == 0) {
      a.sc->red[slot] = total;
      if (MODE == NL_BLOCK) a.sc->dwS = total;
    }
  }
}

cudaError_t nl_plan(const Geom& g, NlPlan* P, int smem_limit) {
  const int wr = g.win_r, pr = g.patch_r;
  P->TH = NL_TH;
  P->TW = NL_TW;
  P->tiles_x = (g.Wh + NL_TW - 1) / NL_TW;
  P->tiles_y = (g.Hh + NL_TH - 1) / NL_TH;
  P->n_tiles = P->tiles_x * P->tiles_y;
  P->NXr = NL_TH + 2 * (wr + pr);
  P->NXc = NL_TW + 2 * (wr + pr);
  P->NQr = NL_TH + wr + 2 * pr;
  P->NQc = NL_TW + wr;
  size_t floats = (size_t)P->NXr * P->NXc + (size_t)(NL_TH + 2 * wr) * (NL_TW + 2 * wr) +
                  2 * (size_t)P->NQr * P->NQc;
  if (g.wscheme == WS_PAPER) {
    if (pr < 1) return cudaErrorInvalidValue;   // the edge factor reads x at +-1
    floats += (size_t)(NL_TH + 2 * wr) * (NL_TW + 2 * wr);
  }
  P->smem_bytes = floats * sizeof(float);
  P->threads = NL_THREADS;
  return P->smem_bytes <= (size_t)smem_limit ? cudaSuccess : cudaErrorInvalidValue;
}

template <int MODE>
static cudaError_t nl_launch_t(const Geom& g, const NlPlan& P, const NlArgs& a, cudaStream_t s) {
  k_nltv<MODE><<<P.n_tiles, NL_THREADS, P.smem_bytes, s>>>(g, P, a);
  return cudaGetLastError();
}

// Raises the dynamic shared-memory limit of the NLTV kernels (current
// device; called outside any stream capture).
cudaError_t nl_prepare(int optin) {
  cudaError_t e = set_max_dynamic_smem(k_nltv<NL_BLOCK>, optin);
  if (e == cudaSuccess) e = set_max_dynamic_smem(k_nltv<NL_APPLY>, optin);
  if (e == cudaSuccess) e = set_max_dynamic_smem(k_nltv<NL_WEIGHTS>, optin);
  return e;
}

cudaError_t nl_launch(int mode, const Geom& g, const NlPlan& P, const NlArgs& a, cudaStream_t s) {
  switch (mode) {
    case NL_BLOCK: return nl_launch_t<NL_BLOCK>(g, P, a, s);
    case NL_APPLY: return nl_launch_t<NL_APPLY>(g, P, a, s);
    case NL_WEIGHTS: return nl_launch_t<NL_WEIGHTS>(g, P, a, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace lfsr
