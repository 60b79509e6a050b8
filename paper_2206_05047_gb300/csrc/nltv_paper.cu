// The paper's regulariser weights (Sec. 3.4, Eq. weight_occ) on the
// stored-weight NLTV path:
//   w_d(u) = w_s(d) g(u),  w_s(d) = exp(-|d|^2 / sigma_s),
//   g(u) = e(u) o(u),      e(u) = exp(-|grad x(u)|^2 / sigma_e),
// with the occlusion factor o fixed by the disparity map (k_occlusion, once
// per light field).  The weights are directed: the edge (u, u+d) carries
// w_a = w_s(d) g(u) for direction d at u and w_b = w_s(d) g(u+d) for
// direction -d at u+d.  The z/w-step updates each dual with its own weight;
// the x-step sees the edge through w_a^2 + w_b^2, so the stored edge weight
// is the root mean square sqrt((w_a^2 + w_b^2) / 2) and the CG kernel
// (k_nla2, which squares it) is shared with the patch weights.
#include "nltv_fast.cuh"

namespace lfsr {

// o(u) = exp(-b(u)^2 inv2_o1) exp(-pe(u)^2 inv2_o2), b(u) = min(0, forward
// differences of omega down + right), 0 across the last row / column; a
// factor with inv2 = 0 is 1, pe = NULL reads as 0.
__global__ void k_occlusion(const int Hh, const int Wh, const float* __restrict__ disp,
                            const float* __restrict__ pe, const float inv2_o1,
                            const float inv2_o2, float* __restrict__ occ) {
  const size_t n = (size_t)Hh * Wh;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / Wh), j = (int)(t - (size_t)i * Wh);
    float o = 1.f;
    if (inv2_o1 > 0.f) {
      const float w0 = disp[t];
      const float gi = (i + 1 < Hh) ? disp[t + Wh] - w0 : 0.f;
      const float gj = (j + 1 < Wh) ? disp[t + 1] - w0 : 0.f;
      const float b = fminf(gi + gj, 0.f);
      o = expf(-b * b * inv2_o1);
    }
    if (pe && inv2_o2 > 0.f) {
      const float e = pe[t];
      o *= expf(-e * e * inv2_o2);
    }
    occ[t] = o;
  }
}

// k_nlw2p<BLOCK>: per owned pixel u and half-window direction d: the edge's
//   directed weights from g staged over the tile + window halo, the stored
//   edge weight, both duals of the edge updated, c(u, d) = (mu/2) (w_a f_a -
//   w_b f_b) (f = 2 w' - w, the over-relaxed duals) added to v(u) and
//   subtracted from v(u+d) (DivAcc; v is zero before the launch).
// k_nlw2p<ONLY>: the stored edge weights alone.
// Thread layout as k_nlw2: a strip of NF_PIX rows of one column per thread.
template <int MODE, int WR, class ST>
__global__ void __launch_bounds__(NF_THREADS, 2)   // two CTAs per SM: <= 64 registers
k_nlw2p(const Geom g, const TableArgs tb) {
  using D = HalfDirs<WR>;
  // x over the tile + (WR + 1): central differences at the halo's g
  constexpr int T = NF_T, HX = WR + 1, NX = T + 2 * HX, NXp = NX | 1;
  constexpr int NG = T + 2 * WR, NGp = NG | 1;
  using DA = DivAcc<WR>;
  __shared__ float sX[NX * NXp];
  __shared__ float sG[NG * NGp];
  __shared__ float sV[MODE == NLW_BLOCK ? DA::SIZE : 1];
  __shared__ double s_red[NF_THREADS / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const JobArgs* jp = tb.jobs + table_job(tb, blockIdx.x);
  const int Hh = jp->Hh, Wh = jp->Wh;
  const float* __restrict__ x = jp->src;
  const float* __restrict__ occ = jp->occ;
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
  // g(v) over the tile + WR; 0 outside the image (only edges that leave
  // the image read it there, and those are dropped)
  for (int t = tid; t < NG * NG; t += NF_THREADS) {
    const int rr = t / NG, cc = t - rr * NG;
    const int vi = i0 - WR + rr, vj = j0 - WR + cc;
    float gv = 0.f;
    if (vi >= 0 && vi < Hh && vj >= 0 && vj < Wh) {
      gv = __ldg(occ + (size_t)vi * Wh + vj);
      if (g.inv_sig_e > 0.f) {
        const float* xc = sX + (rr + 1) * NXp + (cc + 1);    // x(v), clamped neighbours
        const float gi = 0.5f * (xc[NXp] - xc[-NXp]);
        const float gj = 0.5f * (xc[1] - xc[-1]);
        gv *= expf(-fmaf(gi, gi, gj * gj) * g.inv_sig_e);
      }
    }
    sG[rr * NGp + cc] = gv;
  }
  __syncthreads();
  const int ju = lane, uj = j0 + ju;
  const int iu0 = NF_PIX * warp;
  const bool col_in = uj < Wh;
  const float half_mu = 0.5f * g.mu;
  float vown[NF_PIX];                       // this strip's own share of v
#pragma unroll
  for (int m = 0; m < NF_PIX; ++m) vown[m] = 0.f;
  float psum = 0.f;
  const float* gs = sG + (iu0 + WR) * NGp + (ju + WR);   // g(u) of the strip's first pixel
  const float* xs = sX + (iu0 + HX) * NXp + (ju + HX);   // x(u) of the strip's first pixel
  constexpr int DB = 8;   // directions per chunk: the fastest of 3, 4, 6, 8 measured
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
      const float ws = expf(-(float)(di * di + dj * dj) * g.inv_sig_s);
#pragma unroll
      for (int m = 0; m < NF_PIX; ++m) {
        const int ui = i0 + iu0 + m;
        if (ui >= Hh || !col_in) continue;
        const size_t gi = (size_t)ui * Wh + uj;
        // di <= 0 in the half window: u + d never passes the last row
        const bool valid = (ui + di >= 0) && (uj + dj >= 0) && (uj + dj < Wh);
        const float* gu = gs + m * NGp;
        const float w_a = valid ? ws * gu[0] : 0.f;
        const float w_b = valid ? ws * gu[di * NGp + dj] : 0.f;
        st_s(wt + (size_t)idx * p + gi, sqrtf(0.5f * fmaf(w_a, w_a, w_b * w_b)));
        if (MODE == NLW_BLOCK) {
          const float wa = B::f(wa_[e][m]), wb = B::f(wb_[e][m]);
          const float* xc = xs + m * NXp;
          const float diff = valid ? (xc[0] - xc[di * NXp + dj]) : 0.f;
          const float an = fminf(fmaxf(fmaf(w_a, diff, wa), -g.thr), g.thr);
          const float bn = fminf(fmaxf(fmaf(-w_b, diff, wb), -g.thr), g.thr);
          st_s(wS_new + (size_t)(2 * idx) * p + gi, an);
          st_s(wS_new + (size_t)(2 * idx + 1) * p + gi, bn);
          // the edge's divergence term: + at u, - at u + d (zero for an
          // edge that leaves the image: w_a = w_b = 0)
          const float c = half_mu * fmaf(w_a, 2.f * an - wa, -w_b * (2.f * bn - wb));
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
static cudaError_t nlw2p_dispatch(const Geom& g, const TableArgs& t, cudaStream_t s) {
  switch (g.win_r) {
    case 1: k_nlw2p<MODE, 1, ST><<<t.total_units, NF_THREADS, 0, s>>>(g, t); break;
    case 2: k_nlw2p<MODE, 2, ST><<<t.total_units, NF_THREADS, 0, s>>>(g, t); break;
    case 3: k_nlw2p<MODE, 3, ST><<<t.total_units, NF_THREADS, 0, s>>>(g, t); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <class ST>
static cudaError_t nlw2p_st(int block, const Geom& g, const TableArgs& t, cudaStream_t s) {
  return block ? nlw2p_dispatch<NLW_BLOCK, ST>(g, t, s) : nlw2p_dispatch<NLW_ONLY, ST>(g, t, s);
}

cudaError_t nlw2p_launch(int block, const Geom& g, const TableArgs& t, cudaStream_t s) {
  if (t.total_units < 1) return cudaErrorInvalidValue;
  switch (g.st) {
    case ST_F32: return nlw2p_st<float>(block, g, t, s);
    case ST_F16: return nlw2p_st<__half>(block, g, t, s);
    case ST_BF16: return nlw2p_st<__nv_bfloat16>(block, g, t, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t occlusion_launch(int Hh, int Wh, const float* disp, const float* pe, float inv2_o1,
                             float inv2_o2, float* occ, cudaStream_t s) {
  const size_t n = (size_t)Hh * Wh;
  if (n == 0) return cudaErrorInvalidValue;
  const size_t blocks = (n + 255) / 256;
  k_occlusion<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(Hh, Wh, disp, pe, inv2_o1,
                                                                       inv2_o2, occ);
  return cudaGetLastError();
}

}  // namespace lfsr
