// Weighted non-local TV with stored edge weights, for window radius
// WR in {1,2,3} and patch radius PR in {0,1,2} (compile time):
//
//   k_nlw<NLW_BLOCK>  once per ADMM iteration: the NLTV weights of every
//                     undirected edge (u, u+d), d in the half window, from
//                     x^(n-1) (Eq. sr_reg; patch-distance weights), stored
//                     as wt[idx][u]; plus the regulariser rows of
//                     Algorithm 1 (dual update and v := mu/2 S^T f) exactly
//                     as k_nltv<NL_BLOCK> does.
//   k_nlw<NLW_ONLY>   the weights alone.
//   k_nla             every CG step: q := mu/2 sum_d S_d^T S_d p and its
//                     <p, .> part from the stored weights -- no patch sums and
//                     no exp -- optionally first forming p = r + beta p_old.
//
// The weights of one iteration (s_d/2 x p floats) are written once and read
// K times while they sit in L2.  Each region below has a fixed compile-time
// shape: the tile (32 x 32) grown by WR rows and WR columns, which holds
// tile U (tile - d) for every d of the half window once its column origin is
// shifted by min(0, -dj).
#include "lfsr_device.cuh"

namespace lfsr {

constexpr int NF_THREADS = 256;
constexpr int NF_T = 32;
constexpr int NF_PIX = NF_T * NF_T / NF_THREADS;

enum { NLW_BLOCK = 0, NLW_ONLY = 1 };

template <int MODE, int WR, int PR>
__global__ void __launch_bounds__(NF_THREADS)
k_nlw(const Geom g, const NlPlan P, const NlArgs a, float* __restrict__ wt) {
  constexpr int T = NF_T, HX = WR + PR, NX = T + 2 * HX, NXp = NX | 1;
  constexpr int NR = T + WR, NRp = NR | 1, NQR = NR + 2 * PR;
  __shared__ float sX[NX * NXp];
  __shared__ float sQ[NQR * NRp];
  __shared__ float sC[NR * NRp];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int Hh = g.Hh, Wh = g.Wh;
  const size_t p = (size_t)Hh * Wh;
  const int ty = blockIdx.x / P.tiles_x, tx = blockIdx.x - ty * P.tiles_x;
  const int i0 = ty * T, j0 = tx * T;
  const int TRr = min(T, Hh - i0), TRc = min(T, Wh - j0);

  for (int t = tid; t < NX * NX; t += NF_THREADS) {
    const int rr = t / NX, cc = t - rr * NX;
    const int hi = clampi(i0 - HX + rr, 0, Hh - 1), hj = clampi(j0 - HX + cc, 0, Wh - 1);
    sX[rr * NXp + cc] = __ldg(a.x + (size_t)hi * Wh + hj);
  }
  __syncthreads();

  float acc[NF_PIX];
#pragma unroll
  for (int m = 0; m < NF_PIX; ++m) acc[m] = 0.f;
  double part = 0.0;

  for (int idx = 0; idx < g.sh; ++idx) {
    const int di = g.di[idx], dj = g.dj[idx];   // di <= 0
    const int ec0 = min(0, -dj);
    // 1. horizontal sums of squared patch differences (rows of region +- PR)
    for (int t = tid; t < NQR * NR; t += NF_THREADS) {
      const int qa = t / NR, qc = t - qa * NR;
      const float* ra = sX + (qa + WR) * NXp + (ec0 + qc + WR);
      const float* rb = ra + di * NXp + dj;
      float s = 0.f;
#pragma unroll
      for (int b = 0; b <= 2 * PR; ++b) {
        const float dl = ra[b] - rb[b];
        s = fmaf(dl, dl, s);
      }
      sQ[qa * NRp + qc] = s;
    }
    __syncthreads();
    // 2. vertical sums -> weight (stored for owned edges) -> edge quantity
    float psum = 0.f;
    for (int t = tid; t < NR * NR; t += NF_THREADS) {
      const int ea = t / NR, ec = t - ea * NR;
      const int vi = i0 + ea, vj = j0 + ec0 + ec;
      float pd = 0.f;
#pragma unroll
      for (int b = 0; b <= 2 * PR; ++b) pd += sQ[(ea + b) * NRp + ec];
      const bool v_in = vi < Hh && vj >= 0 && vj < Wh;
      const bool valid = v_in && (vi + di >= 0) && (vj + dj >= 0) && (vj + dj < Wh);
      const float w = valid ? expf(-pd * g.inv_np * g.inv_h2) : 0.f;
      const bool own = ea < TRr && (ec + ec0) >= 0 && (ec + ec0) < TRc;
      const size_t gi = (size_t)vi * Wh + vj;
      if (own) wt[(size_t)idx * p + gi] = w;
      if (MODE == NLW_BLOCK) {
        float cval = 0.f;
        if (v_in) {
          const float wa = __ldg(a.wS_old + (size_t)(2 * idx) * p + gi);
          const float wb = __ldg(a.wS_old + (size_t)(2 * idx + 1) * p + gi);
          const float* xv = sX + (ea + HX) * NXp + (ec0 + ec + HX);
          const float diff = valid ? (xv[0] - xv[di * NXp + dj]) : 0.f;
          const float ua = fmaf(w, diff, wa);
          const float ub = fmaf(-w, diff, wb);
          const float an = fminf(fmaxf(ua, -g.thr), g.thr);
          const float bn = fminf(fmaxf(ub, -g.thr), g.thr);
          cval = w * ((2.f * an - wa) - (2.f * bn - wb));
          if (own) {
            a.wS_new[(size_t)(2 * idx) * p + gi] = an;
            a.wS_new[(size_t)(2 * idx + 1) * p + gi] = bn;
            const float da = an - wa, db = bn - wb;
            psum = fmaf(da, da, fmaf(db, db, psum));
          }
        }
        sC[ea * NRp + ec] = cval;
      }
    }
    part += (double)psum;
    __syncthreads();
    if (MODE == NLW_BLOCK) {
#pragma unroll
      for (int m = 0; m < NF_PIX; ++m) {
        const int iu = warp + m * (NF_THREADS / 32), ju = lane;
        const int cc = ju - ec0;
        acc[m] += sC[iu * NRp + cc] - sC[(iu - di) * NRp + (cc - dj)];
      }
      __syncthreads();
    }
  }

  if (MODE == NLW_BLOCK) {
    const float scale = 0.5f * g.mu;
#pragma unroll
    for (int m = 0; m < NF_PIX; ++m) {
      const int iu = warp + m * (NF_THREADS / 32), ju = lane;
      if (iu < TRr && ju < TRc) a.out[(size_t)(i0 + iu) * Wh + (j0 + ju)] = scale * acc[m];
    }
    double total = 0.0;
    if (grid_sum_last<NF_THREADS>(part, a.partials, &a.sc->counter[RED_DW_S], &total) &&
        threadIdx.x == 0) {
      a.sc->red[RED_DW_S] = total;
      a.sc->dwS = total;
    }
  }
}

template <int WR>
__global__ void __launch_bounds__(NF_THREADS)
k_nla(const Geom g, const NlPlan P, const NlArgs a, const float* __restrict__ wt) {
  constexpr int T = NF_T, NP = T + 2 * WR, NPp = NP | 1, NR = T + WR, NRp = NR | 1;
  __shared__ float sP[NP * NPp];
  __shared__ float sC[NR * NRp];
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

  float acc[NF_PIX];
#pragma unroll
  for (int m = 0; m < NF_PIX; ++m) acc[m] = 0.f;
  double part = 0.0;
  for (int idx = 0; idx < g.sh; ++idx) {
    const int di = g.di[idx], dj = g.dj[idx];
    const int ec0 = min(0, -dj);
    float psum = 0.f;
    for (int t = tid; t < NR * NR; t += NF_THREADS) {
      const int ea = t / NR, ec = t - ea * NR;
      const int vi = i0 + ea, vj = j0 + ec0 + ec;
      float w = 0.f;
      if (vi < Hh && vj >= 0 && vj < Wh) w = __ldg(wt + (size_t)idx * p + (size_t)vi * Wh + vj);
      const float* pv = sP + (ea + WR) * NPp + (ec0 + ec + WR);
      const float dp = pv[0] - pv[di * NPp + dj];
      const float w2 = w * w;
      sC[ea * NRp + ec] = w2 * dp;
      if (ea < TRr && (ec + ec0) >= 0 && (ec + ec0) < TRc) psum = fmaf(w2 * dp, dp, psum);
    }
    part += (double)psum;
    __syncthreads();
#pragma unroll
    for (int m = 0; m < NF_PIX; ++m) {
      const int iu = warp + m * (NF_THREADS / 32), ju = lane;
      const int cc = ju - ec0;
      acc[m] += sC[iu * NRp + cc] - sC[(iu - di) * NRp + (cc - dj)];
    }
    __syncthreads();
  }
#pragma unroll
  for (int m = 0; m < NF_PIX; ++m) {
    const int iu = warp + m * (NF_THREADS / 32), ju = lane;
    if (iu < TRr && ju < TRc) a.out[(size_t)(i0 + iu) * Wh + (j0 + ju)] = g.mu * acc[m];
  }
  double total = 0.0;
  if (grid_sum_last<NF_THREADS>(part, a.partials, &a.sc->counter[RED_NLTV], &total) &&
      threadIdx.x == 0)
    a.sc->red[RED_NLTV] = total;
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
static cudaError_t nlw_dispatch(const Geom& g, const NlPlan& P, const NlArgs& a, float* wt,
                                cudaStream_t s) {
#define NLW_CASE(wr, pr)                                                           \
  if (g.win_r == wr && g.patch_r == pr) {                                          \
    k_nlw<MODE, wr, pr><<<P.n_tiles, NF_THREADS, 0, s>>>(g, P, a, wt);             \
    return cudaGetLastError();                                                     \
  }
  NLW_CASE(1, 0) NLW_CASE(1, 1) NLW_CASE(1, 2)
  NLW_CASE(2, 0) NLW_CASE(2, 1) NLW_CASE(2, 2)
  NLW_CASE(3, 0) NLW_CASE(3, 1) NLW_CASE(3, 2)
#undef NLW_CASE
  return cudaErrorInvalidValue;
}

cudaError_t nlw_launch(int block, const Geom& g, const NlPlan& P, const NlArgs& a, float* wt,
                       cudaStream_t s) {
  return block ? nlw_dispatch<NLW_BLOCK>(g, P, a, wt, s) : nlw_dispatch<NLW_ONLY>(g, P, a, wt, s);
}

cudaError_t nla_launch(const Geom& g, const NlPlan& P, const NlArgs& a, const float* wt,
                       cudaStream_t s) {
  switch (g.win_r) {
    case 1: k_nla<1><<<P.n_tiles, NF_THREADS, 0, s>>>(g, P, a, wt); break;
    case 2: k_nla<2><<<P.n_tiles, NF_THREADS, 0, s>>>(g, P, a, wt); break;
    case 3: k_nla<3><<<P.n_tiles, NF_THREADS, 0, s>>>(g, P, a, wt); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t weights_to_canonical(const Geom& g, const float* wt, float* can, cudaStream_t s) {
  k_weights_to_canonical<<<1024, 256, 0, s>>>(g, wt, can);
  return cudaGetLastError();
}

}  // namespace lfsr
