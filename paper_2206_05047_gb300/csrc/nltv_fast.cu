// Weighted non-local TV with stored edge weights, for window radius
// WR in {1,2,3} and patch radius PR in {0,1,2} (compile time).  The weights
// of one ADMM iteration (Eq. sr_reg; patch-distance weights from x^(n-1),
// one per undirected edge (u, u+d), d in the half window: s_d/2 x p floats)
// are written once and read by the K CG steps while they sit in L2.
#include "lfsr_device.cuh"

namespace lfsr {

constexpr int NF_THREADS = 256;
constexpr int NF_T = 32;
constexpr int NF_PIX = NF_T * NF_T / NF_THREADS;

enum { NLW_BLOCK = 0, NLW_ONLY = 1 };

// Pixel-owner kernels, no shared-memory exchange between directions.
// Each thread owns a strip of NF_PIX = 4 consecutive rows of one column of
// a 32 x 32 tile (rows 4 warp + m, column lane).  The half window's
// directions are compile-time constants (raster order, the same table the
// host builds), so the direction loops unroll and every global load of a
// thread is independent of the others.
template <int WR>
struct HalfDirs {
  static constexpr int W = 2 * WR + 1;
  static constexpr int SH = (W * W - 1) / 2;
  static __device__ __forceinline__ constexpr int di(int idx) { return idx / W - WR; }
  static __device__ __forceinline__ constexpr int dj(int idx) { return idx % W - WR; }
};

// k_nlw2<BLOCK>: per owned pixel u and direction d: the edge weight
//   w(u, u+d) from the staged (clamped) x, stored in wt[idx][u]; the two
//   duals of the edge updated; c(u, d) = w (f_a - f_b) stored in cb[idx][u];
//   v(u) := 0 (the data block accumulates into v next, the divergence of c
//   is added by k_cg_init_nltv).  Patch sums of the strip share rows: the
//   4 + 2 PR row sums of squared differences give all 4 patch distances.
// k_nlw2<ONLY>: the weights alone.
template <int MODE, int WR, int PR>
__global__ void __launch_bounds__(NF_THREADS)
k_nlw2(const Geom g, const NlPlan P, const NlArgs a, float* __restrict__ wt,
       float* __restrict__ cb) {
  using D = HalfDirs<WR>;
  constexpr int T = NF_T, HX = WR + PR, NX = T + 2 * HX, NXp = NX | 1;
  constexpr int PW = 2 * PR + 1, NS = NF_PIX + 2 * PR;
  __shared__ float sX[NX * NXp];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int Hh = g.Hh, Wh = g.Wh;
  const size_t p = (size_t)Hh * Wh;
  const int ty = blockIdx.x / P.tiles_x, tx = blockIdx.x - ty * P.tiles_x;
  const int i0 = ty * T, j0 = tx * T;
  for (int t = tid; t < NX * NX; t += NF_THREADS) {
    const int rr = t / NX, cc = t - rr * NX;
    const int hi = clampi(i0 - HX + rr, 0, Hh - 1), hj = clampi(j0 - HX + cc, 0, Wh - 1);
    sX[rr * NXp + cc] = __ldg(a.x + (size_t)hi * Wh + hj);
  }
  __syncthreads();
  const int ju = lane, uj = j0 + ju;
  const int iu0 = NF_PIX * warp;            // strip rows iu0 .. iu0 + 3
  const bool col_in = uj < Wh;
  if (MODE == NLW_BLOCK && col_in) {
#pragma unroll
    for (int m = 0; m < NF_PIX; ++m) {
      const int ui = i0 + iu0 + m;
      if (ui < Hh) a.out[(size_t)ui * Wh + uj] = 0.f;
    }
  }
  float psum = 0.f;
  // patch origin (u - PR) of the strip's first pixel, in sX coordinates
  const float* xs = sX + (iu0 + WR) * NXp + (ju + WR);
  // directions in chunks of DB: the chunk's dual loads are issued first
  constexpr int DB = 3;
#pragma unroll
  for (int i0d = 0; i0d < D::SH; i0d += DB) {
    float wa_[DB][NF_PIX], wb_[DB][NF_PIX];
    if (MODE == NLW_BLOCK) {
#pragma unroll
      for (int e = 0; e < DB; ++e) {
        const int idx = i0d + e;
        if (idx >= D::SH) break;
#pragma unroll
        for (int m = 0; m < NF_PIX; ++m) {
          const int ui = i0 + iu0 + m;
          const size_t gi = (size_t)ui * Wh + uj;
          const bool in = ui < Hh && col_in;
          wa_[e][m] = in ? __ldg(a.wS_old + (size_t)(2 * idx) * p + gi) : 0.f;
          wb_[e][m] = in ? __ldg(a.wS_old + (size_t)(2 * idx + 1) * p + gi) : 0.f;
        }
      }
    }
#pragma unroll
    for (int e = 0; e < DB; ++e) {
      const int idx = i0d + e;
      if (idx >= D::SH) break;
      const int di = D::di(idx), dj = D::dj(idx);
      float hs[NS];
#pragma unroll
      for (int r = 0; r < NS; ++r) {
        float sacc = 0.f;
#pragma unroll
        for (int c2 = 0; c2 < PW; ++c2) {
          const float dl = xs[r * NXp + c2] - xs[(r + di) * NXp + c2 + dj];
          sacc = fmaf(dl, dl, sacc);
        }
        hs[r] = sacc;
      }
#pragma unroll
      for (int m = 0; m < NF_PIX; ++m) {
        const int ui = i0 + iu0 + m;
        if (ui >= Hh || !col_in) continue;
        const size_t gi = (size_t)ui * Wh + uj;
        float pd = 0.f;
#pragma unroll
        for (int r2 = 0; r2 < PW; ++r2) pd += hs[m + r2];
        const bool valid = (ui + di >= 0) && (uj + dj >= 0) && (uj + dj < Wh);
        const float w = valid ? expf(-pd * g.inv_np * g.inv_h2) : 0.f;
        wt[(size_t)idx * p + gi] = w;
        if (MODE == NLW_BLOCK) {
          const float wa = wa_[e][m], wb = wb_[e][m];
          const float* xc = xs + (m + PR) * NXp + PR;      // x(u) in sX
          const float diff = valid ? (xc[0] - xc[di * NXp + dj]) : 0.f;
          const float an = fminf(fmaxf(fmaf(w, diff, wa), -g.thr), g.thr);
          const float bn = fminf(fmaxf(fmaf(-w, diff, wb), -g.thr), g.thr);
          a.wS_new[(size_t)(2 * idx) * p + gi] = an;
          a.wS_new[(size_t)(2 * idx + 1) * p + gi] = bn;
          cb[(size_t)idx * p + gi] = w * ((2.f * an - wa) - (2.f * bn - wb));
          const float da = an - wa, db = bn - wb;
          psum = fmaf(da, da, fmaf(db, db, psum));
        }
      }
    }
  }
  if (MODE == NLW_BLOCK) {
    double total = 0.0;
    if (grid_sum_last<NF_THREADS>((double)psum, a.partials, &a.sc->counter[RED_DW_S], &total) &&
        threadIdx.x == 0) {
      a.sc->red[RED_DW_S] = total;
      a.sc->dwS = total;
    }
  }
}

// k_nla2: q(u) = mu sum_d w(u,u+d)^2 (p(u) - p(u+d)) + w(u-d,u)^2 (p(u) - p(u-d)),
// with <p, q>'s NLTV part sum_d w(u,u+d)^2 (p(u) - p(u+d))^2 (each edge once).
template <int WR>
__global__ void __launch_bounds__(NF_THREADS)
k_nla2(const Geom g, const NlPlan P, const NlArgs a, const float* __restrict__ wt) {
  using D = HalfDirs<WR>;
  constexpr int T = NF_T, NP = T + 2 * WR, NPp = NP | 1;
  __shared__ float sP[NP * NPp];
  if (a.check_done && a.sc->cg_done) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int Hh = g.Hh, Wh = g.Wh;
  const size_t p = (size_t)Hh * Wh;
  const int ty = blockIdx.x / P.tiles_x, tx = blockIdx.x - ty * P.tiles_x;
  const int i0 = ty * T, j0 = tx * T;
  const int TRr = min(T, Hh - i0), TRc = min(T, Wh - j0);
  const int first = a.sc->cg_first;
  const float beta = (float)a.sc->beta;
  for (int t = tid; t < NP * NP; t += NF_THREADS) {
    const int rr = t / NP, cc = t - rr * NP;
    const int hi = i0 - WR + rr, hj = j0 - WR + cc;
    float v = 0.f;
    if (hi >= 0 && hi < Hh && hj >= 0 && hj < Wh) {
      const size_t gi = (size_t)hi * Wh + hj;
      if (a.use_beta) {
        v = __ldg(a.r + gi);
        if (!first) v = fmaf(beta, __ldg(a.p_old + gi), v);
        if (rr >= WR && rr < WR + TRr && cc >= WR && cc < WR + TRc) a.p_new[gi] = v;
      } else {
        v = __ldg(a.p_old + gi);
      }
    }
    sP[rr * NPp + cc] = v;
  }
  __syncthreads();
  const int ju = lane, uj = j0 + ju;
  const int iu0 = NF_PIX * warp;
  const bool col_in = uj < Wh;
  float acc[NF_PIX];
#pragma unroll
  for (int m = 0; m < NF_PIX; ++m) acc[m] = 0.f;
  float psum = 0.f;
  // directions in chunks of DB: all weight loads of a chunk are issued
  // before any is used (memory-level parallelism)
  constexpr int DB = 6;
#pragma unroll
  for (int i0d = 0; i0d < D::SH; i0d += DB) {
    float wf[DB][NF_PIX], wb[DB][NF_PIX];
#pragma unroll
    for (int e = 0; e < DB; ++e) {
      const int idx = i0d + e;
      if (idx >= D::SH) break;
      const int di = D::di(idx), dj = D::dj(idx);
      const float* wd = wt + (size_t)idx * p;
#pragma unroll
      for (int m = 0; m < NF_PIX; ++m) {
        const int ui = i0 + iu0 + m;
        const int bi = ui - di, bj = uj - dj;
        const bool in = ui < Hh && col_in;
        wf[e][m] = in ? __ldg(wd + (size_t)ui * Wh + uj) : 0.f;
        wb[e][m] = (in && bi < Hh && bj >= 0 && bj < Wh) ? __ldg(wd + (size_t)bi * Wh + bj) : 0.f;
      }
    }
#pragma unroll
    for (int e = 0; e < DB; ++e) {
      const int idx = i0d + e;
      if (idx >= D::SH) break;
      const int di = D::di(idx), dj = D::dj(idx);
#pragma unroll
      for (int m = 0; m < NF_PIX; ++m) {
        const float* pu = sP + (iu0 + m + WR) * NPp + (ju + WR);
        const float p0 = pu[0];
        const float df = p0 - pu[di * NPp + dj];
        const float db = p0 - pu[-di * NPp - dj];
        const float wf2 = wf[e][m] * wf[e][m];
        acc[m] = fmaf(wf2, df, fmaf(wb[e][m] * wb[e][m], db, acc[m]));
        psum = fmaf(wf2 * df, df, psum);
      }
    }
  }
#pragma unroll
  for (int m = 0; m < NF_PIX; ++m) {
    const int ui = i0 + iu0 + m;
    if (ui < Hh && col_in) a.out[(size_t)ui * Wh + uj] = g.mu * acc[m];
  }
  double total = 0.0;
  if (grid_sum_last<NF_THREADS>((double)psum, a.partials, &a.sc->counter[RED_NLTV], &total) &&
      threadIdx.x == 0)
    a.sc->red[RED_NLTV] = total;
}

// x-step initialisation (Algorithm 2) with the regulariser divergence of
// the z/w-step folded in: v = v_data + mu/2 sum_d (c(u,d) - c(u-d,d));
// r = -v; x' = x; pi = <r, r>.
template <int WR>
__global__ void __launch_bounds__(512)
k_cg_init_nltv(const Geom g, float* __restrict__ rv, const float* __restrict__ cb,
               const float* __restrict__ x, float* __restrict__ x_next, double* partials,
               DevScalars* sc) {
  using D = HalfDirs<WR>;
  const int Hh = g.Hh, Wh = g.Wh;
  const size_t n = (size_t)Hh * Wh;
  const float half_mu = 0.5f * g.mu;
  double part = 0.0;
  for (size_t i = (size_t)blockIdx.x * 512 + threadIdx.x; i < n; i += (size_t)gridDim.x * 512) {
    const int ui = (int)(i / Wh), uj = (int)(i - (size_t)ui * Wh);
    float div = 0.f;
    constexpr int DB = 8;
#pragma unroll
    for (int i0d = 0; i0d < D::SH; i0d += DB) {
      float cf[DB], cbk[DB];
#pragma unroll
      for (int e = 0; e < DB; ++e) {
        const int idx = i0d + e;
        if (idx >= D::SH) break;
        const float* cd = cb + (size_t)idx * n;
        const int bi = ui - D::di(idx), bj = uj - D::dj(idx);
        cf[e] = __ldg(cd + i);
        cbk[e] = (bi < Hh && bj >= 0 && bj < Wh) ? __ldg(cd + (size_t)bi * Wh + bj) : 0.f;
      }
#pragma unroll
      for (int e = 0; e < DB; ++e)
        if (i0d + e < D::SH) div += cf[e] - cbk[e];
    }
    const float r = -fmaf(half_mu, div, rv[i]);
    rv[i] = r;
    x_next[i] = x[i];
    part += (double)r * (double)r;
  }
  double total = 0.0;
  if (grid_sum_last<512>(part, partials, &sc->counter[RED_PI], &total) && threadIdx.x == 0) {
    sc->pi = total;
    sc->cg_first = 1;
    sc->cg_steps = 0;
    sc->beta = 0.0;
    sc->dw2 = sc->dwA + sc->dwS;
    if (!isfinite(total)) sc->status = -4;
    sc->cg_done = (total > g.tau && isfinite(total)) ? 0 : 1;
  }
}

// canonical weights [d][u] from the stored edge weights wt[idx][u]
__global__ void k_weights_to_canonical(const Geom g, const float* __restrict__ wt,
                                       float* __restrict__ can) {
  const size_t p = (size_t)g.Hh * g.Wh;
  const int sd = 2 * g.sh;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < (size_t)sd * p;
       t += (size_t)gridDim.x * blockDim.x) {
    const int d = (int)(t / p);
    const size_t u = t - (size_t)d * p;
    float v = 0.f;
    if (d < g.sh) {
      v = wt[(size_t)d * p + u];
    } else {
      const int idx = sd - 1 - d;
      const int ui = (int)(u / g.Wh), uj = (int)(u - (size_t)ui * g.Wh);
      const int vi = ui - g.di[idx], vj = uj - g.dj[idx];
      if (vi >= 0 && vi < g.Hh && vj >= 0 && vj < g.Wh) v = wt[(size_t)idx * p + (size_t)vi * g.Wh + vj];
    }
    can[t] = v;
  }
}

// ---------------------------------------------------------------------------
bool nlf_supported(const Geom& g) {
  return g.win_r >= 1 && g.win_r <= 3 && g.patch_r >= 0 && g.patch_r <= 2;
}

template <int MODE>
static cudaError_t nlw2_dispatch(const Geom& g, const NlPlan& P, const NlArgs& a, float* wt,
                                 float* cb, cudaStream_t s) {
#define NLW2_CASE(wr, pr)                                                          \
  if (g.win_r == wr && g.patch_r == pr) {                                          \
    k_nlw2<MODE, wr, pr><<<P.n_tiles, NF_THREADS, 0, s>>>(g, P, a, wt, cb);        \
    return cudaGetLastError();                                                     \
  }
  NLW2_CASE(1, 0) NLW2_CASE(1, 1) NLW2_CASE(1, 2)
  NLW2_CASE(2, 0) NLW2_CASE(2, 1) NLW2_CASE(2, 2)
  NLW2_CASE(3, 0) NLW2_CASE(3, 1) NLW2_CASE(3, 2)
#undef NLW2_CASE
  return cudaErrorInvalidValue;
}

cudaError_t nlw2_launch(int block, const Geom& g, const NlPlan& P, const NlArgs& a, float* wt,
                        float* cb, cudaStream_t s) {
  return block ? nlw2_dispatch<NLW_BLOCK>(g, P, a, wt, cb, s)
               : nlw2_dispatch<NLW_ONLY>(g, P, a, wt, cb, s);
}

cudaError_t nla2_launch(const Geom& g, const NlPlan& P, const NlArgs& a, const float* wt,
                        cudaStream_t s) {
  switch (g.win_r) {
    case 1: k_nla2<1><<<P.n_tiles, NF_THREADS, 0, s>>>(g, P, a, wt); break;
    case 2: k_nla2<2><<<P.n_tiles, NF_THREADS, 0, s>>>(g, P, a, wt); break;
    case 3: k_nla2<3><<<P.n_tiles, NF_THREADS, 0, s>>>(g, P, a, wt); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t cg_init_nltv_launch(const Geom& g, float* rv, const float* cb, const float* x,
                                float* x_next, double* partials, DevScalars* sc, int grid,
                                cudaStream_t s) {
  switch (g.win_r) {
    case 1: k_cg_init_nltv<1><<<grid, 512, 0, s>>>(g, rv, cb, x, x_next, partials, sc); break;
    case 2: k_cg_init_nltv<2><<<grid, 512, 0, s>>>(g, rv, cb, x, x_next, partials, sc); break;
    case 3: k_cg_init_nltv<3><<<grid, 512, 0, s>>>(g, rv, cb, x, x_next, partials, sc); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t weights_to_canonical(const Geom& g, const float* wt, float* can, cudaStream_t s) {
  k_weights_to_canonical<<<1024, 256, 0, s>>>(g, wt, can);
  return cudaGetLastError();
}

}  // namespace lfsr
