// Weighted non-local TV with stored edge weights, part 2: the weighted
// divergence S^T W^2 S p of every CG step and the canonical-layout export
// of the weights.  The weights (s_d/2 x p values of the storage type ST,
// written by nltv_block.cu) are read while they sit in L2; all arithmetic
// is float.
#include "nltv_fast.cuh"

namespace lfsr {

// k_nla2: q(u) = mu sum_d w(u,u+d)^2 (p(u) - p(u+d)) + w(u-d,u)^2 (p(u) - p(u-d)),
// with <p, q>'s NLTV part sum_d w(u,u+d)^2 (p(u) - p(u+d))^2 (each edge once).
// DB: directions per chunk of weight loads (the stencil blocking the batch
// autotuner chooses: 6 or 3).
template <int WR, class ST, int DB>
__global__ void __launch_bounds__(NA_THREADS, 2)
k_nla2(const Geom g, const TableArgs tb) {
  using D = HalfDirs<WR>;
  constexpr int T = NF_T, NP = T + 2 * WR, NPp = NP | 1;
  __shared__ float sP[NP * NPp];
  __shared__ double s_red[NA_THREADS / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // this CTA's tile: unit blockIdx.x of the table
  const JobArgs* jp = tb.jobs + table_job(tb, blockIdx.x);
  DevScalars* sc = jp->sc;
  const bool skip = tb.check_done && ((volatile int*)&sc->cg_done)[0];
  float psum = 0.f;
  if (!skip) {
  const int Hh = jp->Hh, Wh = jp->Wh;
  const size_t p = (size_t)Hh * Wh;
  const ST* __restrict__ wt = (const ST*)jp->wt;
  const int tile = blockIdx.x - jp->unit0;
  const int ty = tile / jp->tiles_x, tx = tile - ty * jp->tiles_x;
  const int i0 = ty * T, j0 = tx * T;
  const int TRr = min(T, Hh - i0), TRc = min(T, Wh - j0);
  const int first = sc->cg_first;
  const float beta = (float)sc->beta;
  for (int t = tid; t < NP * NP; t += NA_THREADS) {
    const int rr = t / NP, cc = t - rr * NP;
    const int hi = i0 - WR + rr, hj = j0 - WR + cc;
    float v = 0.f;
    if (hi >= 0 && hi < Hh && hj >= 0 && hj < Wh) {
      const size_t gi = (size_t)hi * Wh + hj;
      if (jp->use_beta) {
        v = __ldg(jp->r + gi);
        if (!first) v = fmaf(beta, __ldg(jp->p_old + gi), v);
        if (rr >= WR && rr < WR + TRr && cc >= WR && cc < WR + TRc) jp->p_new[gi] = v;
      } else {
        v = __ldg(jp->p_old + gi);
      }
    }
    sP[rr * NPp + cc] = v;
  }
  __syncthreads();
  const int ju = lane, uj = j0 + ju;
  const int iu0 = NA_PIX * warp;
  const bool col_in = uj < Wh;
  // 32-bit offset of the strip's first pixel (p < 2^31); in an interior
  // tile every owned pixel and its backward neighbours u - d (di <= 0) lie
  // inside the image, so the loads need no bounds checks
  const int off0 = (i0 + iu0) * Wh + uj;
  const bool interior = i0 + T + WR <= Hh && j0 >= WR && j0 + T + WR <= Wh;
  float acc[NA_PIX];
#pragma unroll
  for (int m = 0; m < NA_PIX; ++m) acc[m] = 0.f;
  // directions in chunks of DB: all weight loads of a chunk are issued
  // before any is used (memory-level parallelism)
#pragma unroll
  for (int i0d = 0; i0d < D::SH; i0d += DB) {
    using B = SBits<ST>;
    typename B::R wf[DB][NA_PIX], wb[DB][NA_PIX];
#pragma unroll
    for (int e = 0; e < DB; ++e) {
      const int idx = i0d + e;
      if (idx >= D::SH) break;
      const int di = D::di(idx), dj = D::dj(idx);
      const ST* wd = wt + (size_t)idx * p + off0;   // this direction's plane at the strip
      const int bo = di * Wh + dj;                  // u - d is bo floats before u
      if (interior) {
#pragma unroll
        for (int m = 0; m < NA_PIX; ++m) {
          wf[e][m] = B::ld(wd + m * Wh);
          wb[e][m] = B::ld(wd + (m * Wh - bo));
        }
      } else {
#pragma unroll
        for (int m = 0; m < NA_PIX; ++m) {
          const int ui = i0 + iu0 + m;
          const int bi = ui - di, bj = uj - dj;
          const bool in = ui < Hh && col_in;
          wf[e][m] = in ? B::ld(wd + m * Wh) : typename B::R(0);
          wb[e][m] = (in && bi < Hh && bj >= 0 && bj < Wh) ? B::ld(wd + (m * Wh - bo))
                                                            : typename B::R(0);
        }
      }
    }
#pragma unroll
    for (int e = 0; e < DB; ++e) {
      const int idx = i0d + e;
      if (idx >= D::SH) break;
      const int di = D::di(idx), dj = D::dj(idx);
#pragma unroll
      for (int m = 0; m < NA_PIX; ++m) {
        const float* pu = sP + (iu0 + m + WR) * NPp + (ju + WR);
        const float p0 = pu[0];
        const float df = p0 - pu[di * NPp + dj];
        const float db = p0 - pu[-di * NPp - dj];
        const float wfv = B::f(wf[e][m]), wbv = B::f(wb[e][m]);
        const float wf2 = wfv * wfv;
        acc[m] = fmaf(wf2, df, fmaf(wbv * wbv, db, acc[m]));
        psum = fmaf(wf2 * df, df, psum);
      }
    }
  }
#pragma unroll
  for (int m = 0; m < NA_PIX; ++m) {
    const int ui = i0 + iu0 + m;
    if (ui < Hh && col_in) jp->out[(size_t)ui * Wh + uj] = g.mu * acc[m];
  }
  }  // !skip
  // NLTV part of <p, M p> per light field: one slot per tile
  const double bs = block_sum<NA_THREADS>((double)psum, s_red);
  if (tid == 0) tb.partials[blockIdx.x] = bs;
  if (table_arrive_last(tb.counter)) {
    for (int j = warp; j < tb.n_jobs; j += NA_THREADS / 32) {
      const JobArgs* jj = tb.jobs + j;
      const double total = warp_sum_slots(tb.partials + jj->unit0, jj->units);
      if (lane == 0) jj->sc->red[RED_NLTV] = total;
    }
  }
}

// canonical weights [d][u] from the stored edge weights wt[idx][u]
template <class ST>
__global__ void k_weights_to_canonical(const Geom g, const ST* __restrict__ wt,
                                       float* __restrict__ can) {
  const size_t p = (size_t)g.Hh * g.Wh;
  const int sd = 2 * g.sh;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < (size_t)sd * p;
       t += (size_t)gridDim.x * blockDim.x) {
    const int d = (int)(t / p);
    const size_t u = t - (size_t)d * p;
    float v = 0.f;
    if (d < g.sh) {
      v = ld_s(wt + (size_t)d * p + u);
    } else {
      const int idx = sd - 1 - d;
      const int ui = (int)(u / g.Wh), uj = (int)(u - (size_t)ui * g.Wh);
      const int vi = ui - g.di[idx], vj = uj - g.dj[idx];
      if (vi >= 0 && vi < g.Hh && vj >= 0 && vj < g.Wh)
        v = ld_s(wt + (size_t)idx * p + (size_t)vi * g.Wh + vj);
    }
    can[t] = v;
  }
}

// ---------------------------------------------------------------------------
bool nlf_supported(const Geom& g) {
  return g.win_r >= 1 && g.win_r <= 3 && g.patch_r >= 0 && g.patch_r <= 2;
}

template <class ST, int DB>
static cudaError_t nla2_st(const Geom& g, const TableArgs& t, cudaStream_t s) {
  switch (g.win_r) {
    case 1: k_nla2<1, ST, DB><<<t.total_units, NA_THREADS, 0, s>>>(g, t); break;
    case 2: k_nla2<2, ST, DB><<<t.total_units, NA_THREADS, 0, s>>>(g, t); break;
    case 3: k_nla2<3, ST, DB><<<t.total_units, NA_THREADS, 0, s>>>(g, t); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <class ST>
static cudaError_t nla2_db(const Geom& g, const TableArgs& t, cudaStream_t s, int chunk) {
  if (chunk == 6) return nla2_st<ST, 6>(g, t, s);
  if (chunk == 3) return nla2_st<ST, 3>(g, t, s);
  return cudaErrorInvalidValue;
}

cudaError_t nla2_launch(const Geom& g, const TableArgs& t, cudaStream_t s, int chunk) {
  if (t.total_units < 1) return cudaErrorInvalidValue;
  switch (g.st) {
    case ST_F32: return nla2_db<float>(g, t, s, chunk);
    case ST_F16: return nla2_db<__half>(g, t, s, chunk);
    case ST_BF16: return nla2_db<__nv_bfloat16>(g, t, s, chunk);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t weights_to_canonical(const Geom& g, const void* wt, float* can, cudaStream_t s) {
  switch (g.st) {
    case ST_F32: k_weights_to_canonical<<<1024, 256, 0, s>>>(g, (const float*)wt, can); break;
    case ST_F16: k_weights_to_canonical<<<1024, 256, 0, s>>>(g, (const __half*)wt, can); break;
    case ST_BF16:
      k_weights_to_canonical<<<1024, 256, 0, s>>>(g, (const __nv_bfloat16*)wt, can);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace lfsr
