// The paper's backward warp in the x-step (Sec. 4.1): W_k^* takes an image
// on view k's grid back to the reference grid by sampling it bilinearly at
// u - theta_k omega_0(u) (omega_0 the reference view's disparity map), zero
// outside the image.  It replaces the exact adjoint W_k^T (a scatter) where
// the solver forms A_k^* g = W_k^* B^T D^T g: the data block's divergence
// and the x-step's normal matrix.  Being a gather, it needs no atomics: each
// CTA owns one 32 x 32 tile of the output and runs every view.
//
// Per tile R and view k: the LR values g_k of the pixels whose blur touches
// E = R +- (S + 1) (S bounds |theta_k omega_0|, so every tap of a sample
// for u in R lies in E), the adjoint blur onto E (columns then rows for a
// separable kernel), then per owned pixel the bilinear sample.
#include "lfsr_device.cuh"

namespace lfsr {

constexpr int BW_THREADS = 256;
constexpr int BW_PIX = BW_TILE * BW_TILE / BW_THREADS;   // owned pixels per thread (rows)

template <int Z>
__global__ void __launch_bounds__(BW_THREADS)
k_adjoint_bw(const Geom g, const BwPlan P, const OpArgs a) {
  extern __shared__ __align__(16) float smem[];
  if (a.check_done && a.sc->cg_done) return;
  float* sG = smem + P.off_G;   // NLr x NLc LR values
  float* sH = smem + P.off_H;   // NEr x NLc column pass (separable)
  float* sT = smem + P.off_T;   // NEr x NEc adjoint-blurred image on E
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int r = g.r, kb = g.kb, S1 = g.S + 1;
  const int ty = blockIdx.x / P.tiles_x, tx = blockIdx.x - ty * P.tiles_x;
  const int i0 = ty * BW_TILE, j0 = tx * BW_TILE;
  const int TRr = min(BW_TILE, g.Hh - i0), TRc = min(BW_TILE, g.Wh - j0);
  // E clipped to the image (taps outside the image read zero)
  const int e_r0 = max(0, i0 - S1), e_r1 = min(g.Hh - 1, i0 + TRr - 1 + S1);
  const int e_c0 = max(0, j0 - S1), e_c1 = min(g.Wh - 1, j0 + TRc - 1 + S1);
  const int ner = e_r1 - e_r0 + 1, nec = e_c1 - e_c0 + 1;
  const int lr_lo = max(0, ceil_div(e_r0 - r, Z)), lr_hi = min(g.H - 1, floor_div(e_r1 + r, Z));
  const int lc_lo = max(0, ceil_div(e_c0 - r, Z)), lc_hi = min(g.W - 1, floor_div(e_c1 + r, Z));
  const int lr_n = lr_hi - lr_lo + 1, lc_n = lc_hi - lc_lo + 1;
  const size_t q_lr = (size_t)g.H * g.W;

  // owned pixels: rows BW_PIX * warp + m of column lane
  float acc[BW_PIX], om[BW_PIX];
#pragma unroll
  for (int m = 0; m < BW_PIX; ++m) {
    const int ui = i0 + BW_PIX * warp + m, uj = j0 + lane;
    acc[m] = 0.f;
    om[m] = (ui < g.Hh && uj < g.Wh) ? __ldg(a.disp + (size_t)ui * g.Wh + uj) : 0.f;
  }

  for (int vi = 0; vi < a.nviews; ++vi) {
    const int k = a.view0 + vi;
    __syncthreads();   // the previous view's sT is consumed
    for (int t = tid; t < lr_n * lc_n; t += BW_THREADS) {
      const int lr = t / lc_n, lc = t - lr * lc_n;
      sG[lr * P.NLc + lc] =
          __ldg(a.src + (size_t)k * q_lr + (size_t)(lr_lo + lr) * g.W + (lc_lo + lc));
    }
    __syncthreads();
    if (g.separable) {
      // columns: sH[i][m] = sum_l kv[hi - Z l + r] g(l, m)
      for (int t = tid; t < ner * lc_n; t += BW_THREADS) {
        const int i = t / lc_n, lc = t - i * lc_n;
        const int hi = e_r0 + i;
        const int l_a = max(lr_lo, ceil_div(hi - r, Z)), l_b = min(lr_hi, floor_div(hi + r, Z));
        float s = 0.f;
        for (int l = l_a; l <= l_b; ++l) s = fmaf(g.kv[hi - Z * l + r], sG[(l - lr_lo) * P.NLc + lc], s);
        sH[i * P.NLc + lc] = s;
      }
      __syncthreads();
      // rows: t(i, j) = sum_m kh[hj - Z m + r] sH[i][m]
      for (int t = tid; t < ner * nec; t += BW_THREADS) {
        const int i = t / nec, j = t - i * nec;
        const int hj = e_c0 + j;
        const int m_a = max(lc_lo, ceil_div(hj - r, Z)), m_b = min(lc_hi, floor_div(hj + r, Z));
        float s = 0.f;
        for (int mm = m_a; mm <= m_b; ++mm)
          s = fmaf(g.kh[hj - Z * mm + r], sH[i * P.NLc + (mm - lc_lo)], s);
        sT[i * P.NEc + j] = s;
      }
    } else {
      for (int t = tid; t < ner * nec; t += BW_THREADS) {
        const int i = t / nec, j = t - i * nec;
        const int hi = e_r0 + i, hj = e_c0 + j;
        const int l_a = max(lr_lo, ceil_div(hi - r, Z)), l_b = min(lr_hi, floor_div(hi + r, Z));
        const int m_a = max(lc_lo, ceil_div(hj - r, Z)), m_b = min(lc_hi, floor_div(hj + r, Z));
        float s = 0.f;
        for (int l = l_a; l <= l_b; ++l)
          for (int mm = m_a; mm <= m_b; ++mm)
            s = fmaf(g.k2[(hi - Z * l + r) * kb + (hj - Z * mm + r)],
                     sG[(l - lr_lo) * P.NLc + (mm - lc_lo)], s);
        sT[i * P.NEc + j] = s;
      }
    }
    __syncthreads();
    // gather: bilinear sample of t at u - theta_k omega_0(u), zero outside
    const float tu = g.tu[k], tv = g.tv[k];
#pragma unroll
    for (int m = 0; m < BW_PIX; ++m) {
      const int ui = i0 + BW_PIX * warp + m, uj = j0 + lane;
      if (ui >= g.Hh || uj >= g.Wh) continue;
      const float sy = (float)ui - tv * om[m], sx = (float)uj - tu * om[m];
      const float fy0 = floorf(sy), fx0 = floorf(sx);
      const float fy = sy - fy0, fx = sx - fx0;
      const int ti = (int)fy0, tj = (int)fx0;
      float v[2][2];
#pragma unroll
      for (int aa = 0; aa < 2; ++aa)
#pragma unroll
        for (int bb = 0; bb < 2; ++bb) {
          const int ii = ti + aa, jj = tj + bb;
          float val = 0.f;
          if (ii >= 0 && ii < g.Hh && jj >= 0 && jj < g.Wh) {
            // inside the image and within S + 1 of the tile: inside E; the
            // clamp only guards shared-memory addressing
            const int si = clampi(ii - e_r0, 0, ner - 1), sj = clampi(jj - e_c0, 0, nec - 1);
            val = sT[si * P.NEc + sj];
          }
          v[aa][bb] = val;
        }
      const float top = fmaf(fx, v[0][1] - v[0][0], v[0][0]);
      const float bot = fmaf(fx, v[1][1] - v[1][0], v[1][0]);
      acc[m] += fmaf(fy, bot - top, top);
    }
  }

  double part = 0.0;
#pragma unroll
  for (int m = 0; m < BW_PIX; ++m) {
    const int ui = i0 + BW_PIX * warp + m, uj = j0 + lane;
    if (ui >= g.Hh || uj >= g.Wh) continue;
    const size_t gi = (size_t)ui * g.Wh + uj;
    a.out[gi] += a.scale * acc[m];
    if (a.pdot) part += (double)__ldg(a.pdot + gi) * (double)acc[m];
  }
  if (a.pdot) {
    double total = 0.0;
    if (grid_sum_last<BW_THREADS>(part, a.partials, &a.sc->counter[RED_OP], &total) &&
        threadIdx.x == 0) {
      a.sc->red[RED_OP] = total;
      // alpha = pi / <p, M p>  (Algorithm 2), M with the backward warp
      cg_set_alpha(a.sc, (double)g.cA * total + (double)g.mu * a.sc->red[RED_NLTV]);
    }
  }
}

cudaError_t bw_plan(const Geom& g, BwPlan* P, int smem_limit) {
  const int Z = g.zeta, r = g.r, S1 = g.S + 1;
  P->tiles_x = (g.Wh + BW_TILE - 1) / BW_TILE;
  P->tiles_y = (g.Hh + BW_TILE - 1) / BW_TILE;
  P->n_tiles = P->tiles_x * P->tiles_y;
  P->NEr = BW_TILE + 2 * S1;
  P->NEc = BW_TILE + 2 * S1;
  // LR pixels l with |hi - Z l| <= r for hi in an interval of NE rows
  P->NLr = (P->NEr - 1 + 2 * r) / Z + 2;
  P->NLc = (P->NEc - 1 + 2 * r) / Z + 2;
  auto al = [](int n) { return (n + 3) & ~3; };
  int off = 0;
  P->off_G = off; off += al(P->NLr * P->NLc);
  P->off_H = off; off += al(P->NEr * P->NLc);
  P->off_T = off; off += al(P->NEr * P->NEc);
  P->smem_bytes = (size_t)off * sizeof(float);
  return P->smem_bytes <= (size_t)smem_limit ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t bw_prepare(int optin) {
  cudaError_t e = set_max_dynamic_smem(k_adjoint_bw<1>, optin);
  if (e == cudaSuccess) e = set_max_dynamic_smem(k_adjoint_bw<2>, optin);
  if (e == cudaSuccess) e = set_max_dynamic_smem(k_adjoint_bw<3>, optin);
  if (e == cudaSuccess) e = set_max_dynamic_smem(k_adjoint_bw<4>, optin);
  return e;
}

cudaError_t bw_launch(const Geom& g, const BwPlan& P, const OpArgs& a, cudaStream_t s) {
  switch (g.zeta) {
    case 1: k_adjoint_bw<1><<<P.n_tiles, BW_THREADS, P.smem_bytes, s>>>(g, P, a); break;
    case 2: k_adjoint_bw<2><<<P.n_tiles, BW_THREADS, P.smem_bytes, s>>>(g, P, a); break;
    case 3: k_adjoint_bw<3><<<P.n_tiles, BW_THREADS, P.smem_bytes, s>>>(g, P, a); break;
    case 4: k_adjoint_bw<4><<<P.n_tiles, BW_THREADS, P.smem_bytes, s>>>(g, P, a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace lfsr
