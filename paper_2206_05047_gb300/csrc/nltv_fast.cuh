// Shared constants of the stored-weight NLTV kernels (window radius WR in
// {1,2,3}, patch radius PR in {0,1,2}, compile time): tile and thread
// layout and the half window's direction table.
#pragma once

#include "lfsr_device.cuh"

namespace lfsr {

constexpr int NF_THREADS = 512;
constexpr int NF_T = 32;
constexpr int NF_PIX = NF_T * NF_T / NF_THREADS;
// The weighted-divergence kernel (k_nla2) is bound by the latency of its
// weight loads: it runs the same tiles with twice the threads (strips of 2
// rows), 27 warps per SM instead of 13.
constexpr int NA_THREADS = 512;
constexpr int NA_PIX = NF_T * NF_T / NA_THREADS;

enum { NLW_BLOCK = 0, NLW_ONLY = 1 };

// Pixel-owner kernels, no shared-memory exchange between directions.
// Each thread owns a strip of NF_PIX consecutive rows of one column of a
// 32 x 32 tile (rows NF_PIX warp + m, column lane).  The half window's
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

// Divergence accumulator of one NLTV tile (the regulariser's share of v in
// the z/w-step, Sec. 4.1 wdd): every edge term c(u, d) of the tile's pixels
// u adds c to v(u) and -c to v(u + d).  With d in the half window (d_i <= 0)
// the targets lie in the tile, WR rows above it and WR columns either side.
// A CTA gathers them in shared memory (float shared atomics) and adds the
// whole region to the light field's v with global float atomics, so tiles
// whose halos overlap add up; v must be zero before the NLTV block runs.
template <int WR>
struct DivAcc {
  static constexpr int NR = NF_T + WR;          // rows: WR above the tile
  static constexpr int NC = NF_T + 2 * WR;      // columns: WR either side
  static constexpr int NCp = NC | 1;
  static constexpr int SIZE = NR * NCp;
  // smem index of tile-local pixel (r, c), -WR <= r < NF_T, -WR <= c < NF_T + WR
  static __device__ __forceinline__ int at(int r, int c) { return (r + WR) * NCp + (c + WR); }
  static __device__ __forceinline__ void clear(float* acc, int tid, int nthreads) {
    for (int t = tid; t < SIZE; t += nthreads) acc[t] = 0.f;
  }
  // adds the region to v (Hh x Wh); entries outside the image are zero
  static __device__ __forceinline__ void flush(const float* acc, float* v, int i0, int j0, int Hh,
                                               int Wh, int tid, int nthreads) {
    for (int t = tid; t < NR * NC; t += nthreads) {
      const int rr = t / NC, cc = t - rr * NC;
      const int hi = i0 - WR + rr, hj = j0 - WR + cc;
      const float val = acc[rr * NCp + cc];
      if (val != 0.f && hi >= 0 && hi < Hh && hj >= 0 && hj < Wh)
        atomicAdd(v + (size_t)hi * Wh + hj, val);
    }
  }
};

// Shared memory of one CTA of k_nlw2: the staged x and the divergence
// accumulator (floats).
template <int MODE, int WR, int PR>
struct Nlw2Smem {
  static constexpr int NX = NF_T + 2 * (WR + PR), NXp = NX | 1;
  static constexpr int X = NX * NXp;
  static constexpr int V = MODE == NLW_BLOCK ? DivAcc<WR>::SIZE : 1;
};

// k_nlw2<BLOCK>: per owned pixel u and direction d: the edge weight
//   w(u, u+d) from the staged (clamped) x, stored in wt[idx][u]; the two
//   duals of the edge updated; c(u, d) = (mu/2) w (f_a - f_b) added to v(u)
//   and subtracted from v(u+d) (v, zero before the launch, is the light
//   field's accumulated v: the data block adds its part next and the x-step
//   initialisation reads and clears it).  Patch sums of the strip share
//   rows: the NF_PIX + 2 PR row sums of squared differences give all NF_PIX
//   patch distances.
// k_nlw2<ONLY>: the weights alone.
// nlw2_unit runs one tile (work unit `unit` of the table); every thread of
// the CTA calls it, and its slot of the reduction is partials[unit].
template <int MODE, int WR, int PR, class ST>
__device__ __forceinline__ void nlw2_unit(const Geom& g, const TableArgs& tb, int unit, float* sX,
                                          float* sV, double* s_red) {
  using D = HalfDirs<WR>;
  constexpr int T = NF_T, HX = WR + PR, NX = T + 2 * HX, NXp = NX | 1;
  constexpr int PW = 2 * PR + 1, NS = NF_PIX + 2 * PR;
  using DA = DivAcc<WR>;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const JobArgs* jp = tb.jobs + table_job(tb, unit);
  const int Hh = jp->Hh, Wh = jp->Wh;
  const float* __restrict__ x = jp->src;
  float* __restrict__ vout = jp->out;
  const ST* __restrict__ wS_old = (const ST*)jp->wS_old;
  ST* __restrict__ wS_new = (ST*)jp->wS_new;
  ST* __restrict__ wt = (ST*)jp->wt;
  const size_t p = (size_t)Hh * Wh;
  const int tile = unit - jp->unit0;
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
    if (tid == 0) tb.partials[unit] = bs;
  }
}

// After a CTA's last tile: the CTA that arrives last finishes each light
// field's |w_S' - w_S|^2 from its tile slots.
__device__ __forceinline__ void nlw2_finish(const TableArgs& tb) {
  if (!table_arrive_last(tb.counter)) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j = warp; j < tb.n_jobs; j += NF_THREADS / 32) {
    const JobArgs* jj = tb.jobs + j;
    const double total = warp_sum_slots(tb.partials + jj->unit0, jj->units);
    if (lane == 0) {
      jj->sc->red[RED_DW_S] = total;
      jj->sc->dwS = total;
    }
  }
}

// Shared memory of one CTA of k_nla2: the direction p on the tile and its
// window halo (floats).
template <int WR>
struct Nla2Smem {
  static constexpr int NP = NF_T + 2 * WR, NPp = NP | 1;
  static constexpr int P = NP * NPp;
};

// k_nla2: q(u) = mu sum_d w(u,u+d)^2 (p(u) - p(u+d)) + w(u-d,u)^2 (p(u) - p(u-d)),
// with <p, q>'s NLTV part sum_d w(u,u+d)^2 (p(u) - p(u+d))^2 (each edge once).
// DB: directions per chunk of weight loads (the stencil blocking the batch
// autotuner chooses: 6 or 3).  nla2_unit runs one tile (work unit `unit` of
// the table); every thread of the CTA calls it, and its slot of the
// reduction is partials[unit].
template <int WR, class ST, int DB>
__device__ __forceinline__ void nla2_unit(const Geom& g, const TableArgs& tb, int unit, float* sP,
                                          double* s_red) {
  using D = HalfDirs<WR>;
  constexpr int T = NF_T, NP = T + 2 * WR, NPp = NP | 1;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const JobArgs* jp = tb.jobs + table_job(tb, unit);
  DevScalars* sc = jp->sc;
  const bool skip = tb.check_done && ((volatile int*)&sc->cg_done)[0];
  float psum = 0.f;
  if (!skip) {
  const int Hh = jp->Hh, Wh = jp->Wh;
  const size_t p = (size_t)Hh * Wh;
  const ST* __restrict__ wt = (const ST*)jp->wt;
  const int tile = unit - jp->unit0;
  const int ty = tile / jp->tiles_x, tx = tile - ty * jp->tiles_x;
  const int i0 = ty * T, j0 = tx * T;
  const int TRr = min(T, Hh - i0), TRc = min(T, Wh - j0);
  // p = r + beta p_old (or p_old) over the tile and a WR halo: every
  // thread's loads are issued before any is used
  const int first = sc->cg_first;
  const float beta = (float)sc->beta;
  const bool use_beta = jp->use_beta != 0;
  const float* __restrict__ r_in = jp->r;
  const float* __restrict__ p_in = jp->p_old;
  float* __restrict__ p_out = jp->p_new;
  constexpr int NST = (NP * NP + NA_THREADS - 1) / NA_THREADS;
  float ra[NST], pa[NST];
#pragma unroll
  for (int it = 0; it < NST; ++it) {
    const int t = tid + it * NA_THREADS;
    const int rr = t / NP, cc = t - rr * NP;
    const int hi = i0 - WR + rr, hj = j0 - WR + cc;
    const bool in = t < NP * NP && hi >= 0 && hi < Hh && hj >= 0 && hj < Wh;
    const size_t gi = in ? (size_t)hi * Wh + hj : 0;
    ra[it] = (in && use_beta) ? __ldg(r_in + gi) : 0.f;
    pa[it] = (in && !(use_beta && first)) ? __ldg(p_in + gi) : 0.f;
  }
#pragma unroll
  for (int it = 0; it < NST; ++it) {
    const int t = tid + it * NA_THREADS;
    if (t >= NP * NP) break;
    const int rr = t / NP, cc = t - rr * NP;
    // outside the image both loads gave 0, so v = 0 there
    const float v = use_beta ? (first ? ra[it] : fmaf(beta, pa[it], ra[it])) : pa[it];
    if (use_beta && rr >= WR && rr < WR + TRr && cc >= WR && cc < WR + TRc)
      p_out[(size_t)(i0 - WR + rr) * Wh + (j0 - WR + cc)] = v;
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
  if (tid == 0) tb.partials[unit] = bs;
}

// After a CTA's last tile: the CTA that arrives last finishes each light
// field's NLTV part of <p, M p> from its tile slots.
__device__ __forceinline__ void nla2_finish(const TableArgs& tb) {
  if (!table_arrive_last(tb.counter)) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j = warp; j < tb.n_jobs; j += NA_THREADS / 32) {
    const JobArgs* jj = tb.jobs + j;
    const double total = warp_sum_slots(tb.partials + jj->unit0, jj->units);
    if (lane == 0) jj->sc->red[RED_NLTV] = total;
  }
}


}  // namespace lfsr
