// Fused degradation operator A_k = D B W_k and its exact adjoint
// (Eq. sr_model_vec; Sec. 4.1 fwarp / blur / down / up / bwarp kernels),
// in four modes:
//   OP_NORMAL  q += cA * sum_k A_k^T A_k p, and <p, cA sum_k A_k^T A_k p>
//              as cA sum_k |A_k p|^2 (x-step matvec, Sec. 5)
//   OP_DATA    data block of Algorithm 1: r_k = A_k x - y_k, prox / dual
//              update of the data rows, v += A_k^T (l2 r_k + mu/2 l1 f_k)
//   OP_FWD     out_k = A_k x
//   OP_ADJ     out += A_k^T g_k
//   OP_DATA_LR the data block's steps 1-3, h_k stored to the LR buffer out
//              (the backward-warp x-step adds its adjoint in op_bw.cu)
//
// W_k reads view k's own disparity map when a.disp_stride != 0 (per-view
// maps, Sec. 4.1), else the shared map.
//
// One CTA runs a contiguous range of (tile, view) work units of a
// persistent grid.  For a tile R of HR pixels it stages the source image
// (R plus a halo of 2r + S + 1 pixels) in shared memory once, then per view:
//   1. warped samples W_k x on the pixels the blur of the touching LR
//      pixels reads (R +- 2r),
//   2. separable blur evaluated only at decimated columns, then rows
//      (D B never forms the full blurred image),
//   3. the mode's per-LR-pixel step,
//   4. adjoint blur of the zero-filled LR image onto R (columns then rows),
//   5. bilinear scatter (W_k^T) into a shared-memory accumulator covering
//      R + S + 1, flushed to global memory with atomics when the tile changes.
// LR pixels are owned by the tile that holds their HR position; halo LR
// pixels are recomputed bit-identically by neighbouring tiles.
#include "lfsr_device.cuh"

namespace lfsr {

constexpr int OP_THREADS = 512;
constexpr int OP_WARPS = OP_THREADS / 32;

__device__ __forceinline__ float bilerp_smem(const float* sP, int pitch, int rows, int cols,
                                             int li, int lj, float sy, float sx) {
  const float fy0 = floorf(sy), fx0 = floorf(sx);
  const float fy = sy - fy0, fx = sx - fx0;
  // the shift bound S keeps the taps inside the staged region; the clamp
  // only guards shared-memory addressing
  const int ii = clampi(li + (int)fy0, 0, rows - 2);
  const int jj = clampi(lj + (int)fx0, 0, cols - 2);
  const float* q = sP + ii * pitch + jj;
  const float top = fmaf(fx, q[1] - q[0], q[0]);
  const float bot = fmaf(fx, q[pitch + 1] - q[pitch], q[pitch]);
  return fmaf(fy, bot - top, top);
}

__device__ __forceinline__ void scatter_smem(float* sA, int pitch, int rows, int cols, int li,
                                             int lj, float sy, float sx, float t) {
  const float fy0 = floorf(sy), fx0 = floorf(sx);
  const float fy = sy - fy0, fx = sx - fx0;
  const int ii = clampi(li + (int)fy0, 0, rows - 2);
  const int jj = clampi(lj + (int)fx0, 0, cols - 2);
  float* q = sA + ii * pitch + jj;
  const float ty = fy * t, by = t - ty;   // (fy) t, (1 - fy) t
  atomicAdd(q, by - fx * by);
  atomicAdd(q + 1, fx * by);
  atomicAdd(q + pitch, ty - fx * ty);
  atomicAdd(q + pitch + 1, fx * ty);
}

template <int MODE, int Z>
__global__ void __launch_bounds__(OP_THREADS, 1)
k_operator(const Geom g, const OpPlan P, const OpArgs a) {
  extern __shared__ __align__(16) float smem[];
  if (a.check_done && a.sc->cg_done) return;
  float* sP = smem + P.off_P;
  float* sW = smem + P.off_W;
  float* sH = smem + P.off_H;
  float* sG = smem + P.off_G;
  float* sA = smem + P.off_A;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int r = g.r, kb = g.kb, S = g.S;
  const int u_begin = (int)((long long)blockIdx.x * a.units / gridDim.x);
  const int u_end = (int)((long long)(blockIdx.x + 1) * a.units / gridDim.x);
  const size_t q_lr = (size_t)g.H * g.W;
  double part = 0.0;

  int cur_tile = -1;
  int i0 = 0, j0 = 0, TRr = 0, TRc = 0;
  int lr_lo = 0, lr_n = 0, lc_lo = 0, lc_n = 0;
  int e_r0 = 0, e_c0 = 0, NEr = 0, NEc = 0;
  int p_r0 = 0, p_c0 = 0;
  int a_r0 = 0, a_c0 = 0, NAr = 0, NAc = 0;

  constexpr bool ACC = MODE != OP_FWD && MODE != OP_DATA_LR;   // HR accumulator in use
  if (ACC)
    for (int idx = tid; idx < P.NAr * P.NAc; idx += OP_THREADS) sA[idx] = 0.f;

  for (int u = u_begin; u < u_end; ++u) {
    const int tile = u / a.nviews;
    const int k = a.view0 + (u - tile * a.nviews);
    if (tile != cur_tile) {
      if (cur_tile >= 0 && ACC) {
        // flush the accumulator of the previous tile
        __syncthreads();
        for (int ar = warp; ar < NAr; ar += OP_WARPS) {
          const int hi = a_r0 + ar;
          const bool row_in = (hi >= 0 && hi < g.Hh);
          for (int ac = lane; ac < NAc; ac += 32) {
            const int hj = a_c0 + ac;
            const float v = sA[ar * P.NAc + ac];
            if (row_in && hj >= 0 && hj < g.Wh && v != 0.f)
              atomicAdd(a.out + (size_t)hi * g.Wh + hj, a.scale * v);
            sA[ar * P.NAc + ac] = 0.f;
          }
        }
      }
      cur_tile = tile;
      const int ty = tile / P.tiles_x, tx = tile - ty * P.tiles_x;
      i0 = ty * P.TH;
      j0 = tx * P.TW;
      TRr = min(P.TH, g.Hh - i0);
      TRc = min(P.TW, g.Wh - j0);
      lr_lo = max(0, ceil_div(i0 - r, Z));
      lr_n = min(g.H - 1, floor_div(i0 + TRr - 1 + r, Z)) - lr_lo + 1;
      lc_lo = max(0, ceil_div(j0 - r, Z));
      lc_n = min(g.W - 1, floor_div(j0 + TRc - 1 + r, Z)) - lc_lo + 1;
      e_r0 = Z * lr_lo - r;
      e_c0 = Z * lc_lo - r;
      NEr = Z * (lr_n - 1) + 2 * r + 1;
      NEc = Z * (lc_n - 1) + 2 * r + 1;
      p_r0 = e_r0 - S;
      p_c0 = e_c0 - S;
      a_r0 = i0 - S;
      a_c0 = j0 - S;
      NAr = TRr + 2 * S + 1;
      NAc = TRc + 2 * S + 1;
      if (MODE != OP_ADJ) {
        __syncthreads();
        const int npr = NEr + 2 * S + 1, npc = NEc + 2 * S + 1;
        for (int pr = warp; pr < npr; pr += OP_WARPS) {
          const int hi = p_r0 + pr;
          const bool row_in = (hi >= 0 && hi < g.Hh);
          for (int pc = lane; pc < npc; pc += 32) {
            const int hj = p_c0 + pc;
            sP[pr * P.NPc + pc] =
                (row_in && hj >= 0 && hj < g.Wh) ? __ldg(a.src + (size_t)hi * g.Wh + hj) : 0.f;
          }
        }
      }
      __syncthreads();
    }

    const float tu = g.tu[k], tv = g.tv[k];
    const float* __restrict__ disp_k = a.disp + (size_t)k * a.disp_stride;
    if (MODE != OP_ADJ) {
      // 1. warped samples on the blur support of the touching LR pixels
      for (int er = warp; er < NEr; er += OP_WARPS) {
        const int hi = e_r0 + er;
        const bool row_in = (hi >= 0 && hi < g.Hh);
        for (int ec = lane; ec < NEc; ec += 32) {
          const int hj = e_c0 + ec;
          float val = 0.f;
          if (row_in && hj >= 0 && hj < g.Wh) {
            const float om = __ldg(disp_k + (size_t)hi * g.Wh + hj);
            val = bilerp_smem(sP, P.NPc, P.NPr, P.NPc, er + S, ec + S, tv * om, tu * om);
          }
          sW[er * P.NEc + ec] = val;
        }
      }
      __syncthreads();
      // 2. blur at the decimated positions (D B)
      if (g.separable) {
        for (int er = warp; er < NEr; er += OP_WARPS)
          for (int lc = lane; lc < lc_n; lc += 32) {
            const float* w = sW + er * P.NEc + Z * lc;
            float acc = 0.f;
            for (int b = 0; b < kb; ++b) acc = fmaf(g.kh[b], w[b], acc);
            sH[er * P.NLc + lc] = acc;
          }
        __syncthreads();
      }
      for (int lr = warp; lr < lr_n; lr += OP_WARPS)
        for (int lc = lane; lc < lc_n; lc += 32) {
          float acc = 0.f;
          if (g.separable) {
            const float* hc = sH + (Z * lr) * P.NLc + lc;
            for (int b = 0; b < kb; ++b) acc = fmaf(g.kv[b], hc[b * P.NLc], acc);
          } else {
            const float* w = sW + (Z * lr) * P.NEc + Z * lc;
            for (int aa = 0; aa < kb; ++aa)
              for (int b = 0; b < kb; ++b) acc = fmaf(g.k2[aa * kb + b], w[aa * P.NEc + b], acc);
          }
          // 3. per-LR-pixel step
          const int gr = lr_lo + lr, gc = lc_lo + lc;
          const bool owned = (Z * gr >= i0) && (Z * gr < i0 + TRr) && (Z * gc >= j0) &&
                             (Z * gc < j0 + TRc);
          float h = acc;
          if (MODE == OP_NORMAL) {
            if (owned) part += (double)acc * (double)acc;
          } else if (MODE == OP_DATA || MODE == OP_DATA_LR) {
            const size_t gi = (size_t)k * q_lr + (size_t)gr * g.W + gc;
            const float yv = ld_kind(a.y, gi, g.st_y), wa = ld_kind(a.wA_old, gi, g.st);
            const float res = acc - yv;                      // a = A x - b
            const float uu = fmaf(g.lambda1, res, wa);       // u = F x - b' + w
            const float wn = fminf(fmaxf(uu, -g.thr), g.thr);  // w = u - prox(u)
            const float f = 2.f * wn - wa;                   // f = 2 w_n - w_{n-1}
            h = fmaf(g.lambda2, res, 0.5f * g.mu * g.lambda1 * f);
            if (owned) {
              st_kind(a.wA_new, gi, g.st, wn);
              const double dd = (double)wn - (double)wa;
              part += dd * dd;
              if (MODE == OP_DATA_LR) a.out[gi] = h;
            }
          } else if (MODE == OP_FWD) {
            if (owned) a.out[(size_t)k * q_lr + (size_t)gr * g.W + gc] = acc;
          }
          sG[lr * P.NLc + lc] = h;
        }
    } else {
      for (int lr = warp; lr < lr_n; lr += OP_WARPS)
        for (int lc = lane; lc < lc_n; lc += 32)
          sG[lr * P.NLc + lc] =
              __ldg(a.src + (size_t)k * q_lr + (size_t)(lr_lo + lr) * g.W + (lc_lo + lc));
    }
    __syncthreads();
    if (!ACC) continue;

    // 4. adjoint blur of the zero-filled LR values onto the tile
    if (g.separable) {
      for (int i = warp; i < TRr; i += OP_WARPS) {
        const int hi = i0 + i;
        const int l_a = max(lr_lo, ceil_div(hi - r, Z));
        const int l_b = min(lr_lo + lr_n - 1, floor_div(hi + r, Z));
        for (int lc = lane; lc < lc_n; lc += 32) {
          float acc = 0.f;
          for (int l = l_a; l <= l_b; ++l)
            acc = fmaf(g.kv[hi - Z * l + r], sG[(l - lr_lo) * P.NLc + lc], acc);
          sH[i * P.NLc + lc] = acc;
        }
      }
      __syncthreads();
    }
    // 5. rows of the adjoint blur, then the bilinear scatter (W_k^T)
    for (int i = warp; i < TRr; i += OP_WARPS) {
      const int hi = i0 + i;
      for (int j = lane; j < TRc; j += 32) {
        const int hj = j0 + j;
        const int m_a = max(lc_lo, ceil_div(hj - r, Z));
        const int m_b = min(lc_lo + lc_n - 1, floor_div(hj + r, Z));
        float t = 0.f;
        if (g.separable) {
          for (int m = m_a; m <= m_b; ++m)
            t = fmaf(g.kh[hj - Z * m + r], sH[i * P.NLc + (m - lc_lo)], t);
        } else {
          const int l_a = max(lr_lo, ceil_div(hi - r, Z));
          const int l_b = min(lr_lo + lr_n - 1, floor_div(hi + r, Z));
          for (int l = l_a; l <= l_b; ++l)
            for (int m = m_a; m <= m_b; ++m)
              t = fmaf(g.k2[(hi - Z * l + r) * kb + (hj - Z * m + r)],
                       sG[(l - lr_lo) * P.NLc + (m - lc_lo)], t);
        }
        const float om = __ldg(disp_k + (size_t)hi * g.Wh + hj);
        scatter_smem(sA, P.NAc, P.NAr, P.NAc, i + S, j + S, tv * om, tu * om, t);
      }
    }
    __syncthreads();
  }

  if (ACC && cur_tile >= 0) {
    __syncthreads();
    for (int ar = warp; ar < NAr; ar += OP_WARPS) {
      const int hi = a_r0 + ar;
      const bool row_in = (hi >= 0 && hi < g.Hh);
      for (int ac = lane; ac < NAc; ac += 32) {
        const int hj = a_c0 + ac;
        const float v = sA[ar * P.NAc + ac];
        if (row_in && hj >= 0 && hj < g.Wh && v != 0.f)
          atomicAdd(a.out + (size_t)hi * g.Wh + hj, a.scale * v);
      }
    }
  }

  if (MODE == OP_NORMAL || MODE == OP_DATA || MODE == OP_DATA_LR) {
    const int slot = (MODE == OP_NORMAL) ? RED_OP : RED_DW_A;
    double total = 0.0;
    if (grid_sum_last<OP_THREADS>(part, a.partials, &a.sc->counter[slot], &total) &&
        threadIdx.x == 0) {
      a.sc->red[slot] = total;
      if (MODE == OP_NORMAL) {
        // alpha = pi / <p, M p>  (Algorithm 2)
        cg_set_alpha(a.sc, (double)g.cA * total + (double)g.mu * a.sc->red[RED_NLTV]);
      } else {
        a.sc->dwA = total;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static size_t op_layout(const Geom& g, int TH, int TW, OpPlan* P) {
  const int Z = g.zeta, r = g.r, S = g.S;
  P->TH = TH;
  P->TW = TW;
  P->NLr = (TH + 2 * r + Z - 1) / Z;
  P->NLc = (TW + 2 * r + Z - 1) / Z;
  P->NEr = Z * (P->NLr - 1) + 2 * r + 1;
  P->NEc = Z * (P->NLc - 1) + 2 * r + 1;
  P->NPr = P->NEr + 2 * S + 1;
  P->NPc = P->NEc + 2 * S + 1;
  P->NAr = TH + 2 * S + 1;
  P->NAc = TW + 2 * S + 1;
  auto al = [](int n) { return (n + 3) & ~3; };
  int off = 0;
  P->off_P = off; off += al(P->NPr * P->NPc);
  P->off_W = off; off += al(P->NEr * P->NEc);
  P->off_H = off; off += al((P->NEr > TH ? P->NEr : TH) * P->NLc);
  P->off_G = off; off += al(P->NLr * P->NLc);
  P->off_A = off; off += al(P->NAr * P->NAc);
  P->smem_bytes = (size_t)off * sizeof(float);
  P->tiles_x = (g.Wh + TW - 1) / TW;
  P->tiles_y = (g.Hh + TH - 1) / TH;
  P->n_tiles = P->tiles_x * P->tiles_y;
  P->threads = OP_THREADS;
  return P->smem_bytes;
}

template <int MODE, int Z>
static cudaError_t op_launch_t(const Geom& g, const OpPlan& P, const OpArgs& a, int grid,
                               cudaStream_t s) {
  k_operator<MODE, Z><<<grid, OP_THREADS, P.smem_bytes, s>>>(g, P, a);
  return cudaGetLastError();
}

template <int Z>
static cudaError_t op_prepare_z(int optin) {
  cudaError_t e = set_max_dynamic_smem(k_operator<OP_NORMAL, Z>, optin);
  if (e == cudaSuccess) e = set_max_dynamic_smem(k_operator<OP_DATA, Z>, optin);
  if (e == cudaSuccess) e = set_max_dynamic_smem(k_operator<OP_FWD, Z>, optin);
  if (e == cudaSuccess) e = set_max_dynamic_smem(k_operator<OP_ADJ, Z>, optin);
  if (e == cudaSuccess) e = set_max_dynamic_smem(k_operator<OP_DATA_LR, Z>, optin);
  return e;
}

// Raises the dynamic shared-memory limit of every operator kernel this
// geometry can use (the current device; called outside any stream capture).
cudaError_t op_prepare(const Geom& g, int optin) {
  cudaError_t e = cudaErrorInvalidValue;
  switch (g.zeta) {
    case 1: e = op_prepare_z<1>(optin); break;
    case 2: e = op_prepare_z<2>(optin); break;
    case 3: e = op_prepare_z<3>(optin); break;
    case 4: e = op_prepare_z<4>(optin); break;
  }
  if (e == cudaSuccess && fast_supported(g)) e = fast_prepare(g, optin);
  return e;
}

template <int MODE>
static cudaError_t op_launch_m(const Geom& g, const OpPlan& P, const OpArgs& a, int grid,
                               cudaStream_t s) {
  switch (g.zeta) {
    case 1: return op_launch_t<MODE, 1>(g, P, a, grid, s);
    case 2: return op_launch_t<MODE, 2>(g, P, a, grid, s);
    case 3: return op_launch_t<MODE, 3>(g, P, a, grid, s);
    case 4: return op_launch_t<MODE, 4>(g, P, a, grid, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t op_launch(int mode, const Geom& g, const OpPlan& P, const OpArgs& a, int grid,
                      cudaStream_t s) {
  if (grid <= 0) return cudaSuccess;
  if (P.fast) return cudaErrorInvalidValue;  // the specialised kernel is table-driven: fast_launch
  switch (mode) {
    case OP_NORMAL: return op_launch_m<OP_NORMAL>(g, P, a, grid, s);
    case OP_DATA: return op_launch_m<OP_DATA>(g, P, a, grid, s);
    case OP_FWD: return op_launch_m<OP_FWD>(g, P, a, grid, s);
    case OP_ADJ: return op_launch_m<OP_ADJ>(g, P, a, grid, s);
    case OP_DATA_LR: return op_launch_m<OP_DATA_LR>(g, P, a, grid, s);
  }
  return cudaErrorInvalidValue;
}

template <int Z>
static int op_occupancy(size_t smem) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_operator<OP_NORMAL, Z>, OP_THREADS, smem) !=
      cudaSuccess)
    return 1;
  return n > 0 ? n : 1;
}

// Picks the largest tile whose shared-memory layout fits, and the resident
// CTAs per SM (op_prepare must have raised the smem limit first).
cudaError_t op_plan(const Geom& g, OpPlan* P, int sm_count, int smem_limit) {
  (void)sm_count;
  const size_t limit = (size_t)smem_limit;
  P->fast = 0;
  if (fast_supported(g) && fast_plan(g, P, smem_limit) == cudaSuccess) return cudaSuccess;
  P->fast = 0;
  static const int shapes[][2] = {{64, 64}, {32, 64}, {32, 32}, {16, 32}, {16, 16}, {8, 16}, {8, 8}};
  for (auto& sh : shapes) {
    if (op_layout(g, sh[0], sh[1], P) <= limit) {
      switch (g.zeta) {
        case 1: P->ctas_per_sm = op_occupancy<1>(P->smem_bytes); break;
        case 2: P->ctas_per_sm = op_occupancy<2>(P->smem_bytes); break;
        case 3: P->ctas_per_sm = op_occupancy<3>(P->smem_bytes); break;
        default: P->ctas_per_sm = op_occupancy<4>(P->smem_bytes); break;
      }
      return cudaSuccess;
    }
  }
  return cudaErrorInvalidValue;
}

int op_grid(const OpPlan& P, int units, int sm_count) {
  int g = sm_count * P.ctas_per_sm;
  return units < g ? units : g;
}

}  // namespace lfsr
