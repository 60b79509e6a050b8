// Weighted non-local TV with stored edge weights, part 1: the weight
// construction and the z/w-step of the regulariser rows (Eq. sr_reg;
// patch-distance weights from x^(n-1), one per undirected edge (u, u+d), d
// in the half window: s_d/2 x p values, written once per ADMM iteration and
// read by the K CG steps in nltv_fast.cu while they sit in L2).  Duals and
// weights are kept in the storage type ST (float, half or bfloat16); the
// regulariser's divergence (mu/2) S^T f goes straight into the accumulated v
// (DivAcc) and all arithmetic is float.
#include "nltv_fast.cuh"

namespace lfsr {

// k_nlw2<BLOCK>: per owned pixel u and direction d: the edge weight
//   w(u, u+d) from the staged (clamped) x, stored in wt[idx][u]; the two
//   duals of the edge updated; c(u, d) = (mu/2) w (f_a - f_b) added to v(u)
//   and subtracted from v(u+d) (v, zero before the launch, is the light
//   field's accumulated v: the data block adds its part next and the x-step
//   initialisation reads and clears it).  Patch sums of the strip share
//   rows: the NF_PIX + 2 PR row sums of squared differences give all NF_PIX
//   patch distances.
// k_nlw2<ONLY>: the weights alone.
template <int MODE, int WR, int PR, class ST>
__global__ void __launch_bounds__(NF_THREADS)
k_nlw2(const Geom g, const TableArgs tb) {
  using D = HalfDirs<WR>;
  constexpr int T = NF_T, HX = WR + PR, NX = T + 2 * HX, NXp = NX | 1;
  constexpr int PW = 2 * PR + 1, NS = NF_PIX + 2 * PR;
  using DA = DivAcc<WR>;
  __shared__ float sX[NX * NXp];
  __shared__ float sV[MODE == NLW_BLOCK ? DA::SIZE : 1];
  __shared__ double s_red[NF_THREADS / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // this CTA's tile: unit blockIdx.x of the table
  const JobArgs* jp = tb.jobs + table_job(tb, blockIdx.x);
  const int Hh = jp->Hh, Wh = jp->Wh;
  const float* __restrict__ x = jp->src;
  float* __restrict__ vout = jp->out;
  const ST* __restrict__ wS_old = (const ST*)jp->wS_old;
  ST* __restrict__ wS_new = (ST*)jp->wS_new;
  ST* __restrict__ wt = (ST*)jp->wt;
  const size_t p = (size_t)Hh * Wh;
  const int tile = blockIdx.x - jp->unit0;
  const int ty = tile / jp->tiles_x, tx = tile - ty * jp->tiles_x;
  const int i0 = ty * T, j0 = tx * T;
  for (int t = tid; t < NX * NX; t += NF_THREADS) {
    const int rr = t / NX, cc = t - rr * NX;
    const int hi = clampi(i0 - HX + rr, 0, Hh - 1), hj = clampi(j0 - HX + cc, 0, Wh - 1);
    sX[rr * NXp + cc] = __ldg(x + (size_t)hi * Wh + hj);
  }
  if (MODE == NLW_BLOCK) DA::clear(sV, tid, NF_THREADS);
  __syncthreads();
  const int ju = lane, uj = j0 + ju;
  const int iu0 = NF_PIX * warp;            // strip rows iu0 .. iu0 + NF_PIX - 1
  const bool col_in = uj < Wh;
  const float half_mu = 0.5f * g.mu;
  float vown[NF_PIX];                       // this strip's own share of v
#pragma unroll
  for (int m = 0; m < NF_PIX; ++m) vown[m] = 0.f;
  float psum = 0.f;
  // patch origin (u - PR) of the strip's first pixel, in sX coordinates
  const float* xs = sX + (iu0 + WR) * NXp + (ju + WR);
  // directions in chunks of DB: the chunk's dual loads are issued first
  constexpr int DB = 4;   // directions per chunk: the fastest of 3, 4, 6, 8 measured
  // the chunk loop stays rolled: fully unrolled, the 24 edges of a 7 x 7
  // window overflow the instruction cache (warps stalled on fetch)
#pragma unroll 1
  for (int i0d = 0; i0d < D::SH; i0d += DB) {
    using B = SBits<ST>;
    typename B::R wa_[DB][NF_PIX], wb_[DB][NF_PIX];
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
          wa_[e][m] = in ? B::ld(wS_old + (size_t)(2 * idx) * p + gi) : typename B::R(0);
          wb_[e][m] = in ? B::ld(wS_old + (size_t)(2 * idx + 1) * p + gi) : typename B::R(0);
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
        st_s(wt + (size_t)idx * p + gi, w);
        if (MODE == NLW_BLOCK) {
          const float wa = B::f(wa_[e][m]), wb = B::f(wb_[e][m]);
          const float* xc = xs + (m + PR) * NXp + PR;      // x(u) in sX
          const float diff = valid ? (xc[0] - xc[di * NXp + dj]) : 0.f;
          const float an = fminf(fmaxf(fmaf(w, diff, wa), -g.thr), g.thr);
          const float bn = fminf(fmaxf(fmaf(-w, diff, wb), -g.thr), g.thr);
          st_s(wS_new + (size_t)(2 * idx) * p + gi, an);
          st_s(wS_new + (size_t)(2 * idx + 1) * p + gi, bn);
          // the edge's divergence term: + at u, - at u + d (zero for an
          // edge that leaves the image: w = 0)
          const float c = half_mu * w * ((2.f * an - wa) - (2.f * bn - wb));
          vown[m] += c;
          if (valid) atomicAdd(sV + DA::at(iu0 + m + di, ju + dj), -c);
          const float da = an - wa, db = bn - wb;
          psum = fmaf(da, da, fmaf(db, db, psum));
        }
      }
    }
  }
  if (MODE == NLW_BLOCK) {
#pragma unroll
    for (int m = 0; m < NF_PIX; ++m)
      if (vown[m] != 0.f) atomicAdd(sV + DA::at(iu0 + m, ju), vown[m]);
    __syncthreads();
    DA::flush(sV, vout, i0, j0, Hh, Wh, tid, NF_THREADS);
    // |w_S' - w_S|^2 per light field: one slot per tile, summed by the last CTA
    const double bs = block_sum<NF_THREADS>((double)psum, s_red);
    if (tid == 0) tb.partials[blockIdx.x] = bs;
    if (table_arrive_last(tb.counter)) {
      for (int j = warp; j < tb.n_jobs; j += NF_THREADS / 32) {
        const JobArgs* jj = tb.jobs + j;
        const double total = warp_sum_slots(tb.partials + jj->unit0, jj->units);
        if (lane == 0) {
          jj->sc->red[RED_DW_S] = total;
          jj->sc->dwS = total;
        }
      }
    }
  }
}

template <int MODE, class ST>
static cudaError_t nlw2_dispatch(const Geom& g, const TableArgs& t, cudaStream_t s) {
#define NLW2_CASE(wr, pr)                                                          \
  if (g.win_r == wr && g.patch_r == pr) {                                          \
    k_nlw2<MODE, wr, pr, ST><<<t.total_units, NF_THREADS, 0, s>>>(g, t);           \
    return cudaGetLastError();                                                     \
  }
  NLW2_CASE(1, 0) NLW2_CASE(1, 1) NLW2_CASE(1, 2)
  NLW2_CASE(2, 0) NLW2_CASE(2, 1) NLW2_CASE(2, 2)
  NLW2_CASE(3, 0) NLW2_CASE(3, 1) NLW2_CASE(3, 2)
#undef NLW2_CASE
  return cudaErrorInvalidValue;
}

template <class ST>
static cudaError_t nlw2_st(int block, const Geom& g, const TableArgs& t, cudaStream_t s) {
  return block ? nlw2_dispatch<NLW_BLOCK, ST>(g, t, s) : nlw2_dispatch<NLW_ONLY, ST>(g, t, s);
}

cudaError_t nlw2_launch(int block, const Geom& g, const TableArgs& t, cudaStream_t s) {
  if (g.wscheme == WS_PAPER) return nlw2p_launch(block, g, t, s);
  if (t.total_units < 1) return cudaErrorInvalidValue;
  switch (g.st) {
    case ST_F32: return nlw2_st<float>(block, g, t, s);
    case ST_F16: return nlw2_st<__half>(block, g, t, s);
    case ST_BF16: return nlw2_st<__nv_bfloat16>(block, g, t, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace lfsr
