// Specialised fused operator kernel for separable blur kernels of size
// KB in {3,5,7,9} and scale Z in {1,2,3,4}: the same per-(tile, view)
// pipeline as k_operator (warped samples -> decimated separable blur ->
// per-LR-pixel step -> adjoint blur -> bilinear scatter), with every size of
// the 64 x 64 tile known at compile time:
//   * blur taps are compile-time-indexed kernel parameters (no dynamic
//     constant-bank indexing), all tap loops unrolled;
//   * each thread computes several outputs from a register sliding window
//     (a row or column segment), so one shared-memory load feeds several FMAs;
//   * the adjoint of "zero-fill then blur" runs in polyphase form: output
//     row Z m + ph takes LR rows m + delta with compile-time deltas and
//     coefficients kv[ph + R - Z delta] -- no division, no zero taps;
//   * the disparity tile is staged once per tile and reused by all views;
//   * lanes run along the dimension whose shared-memory pitch is odd, so
//     loads, stores and the scatter atomics are free of bank conflicts;
//   * floor / fraction of the sub-pixel shift use an FP32 add with round-down
//     against 2^23 (exact for 0 <= t < 2^23) instead of conversions;
//   * the <p, M p> partial sums in FP32 within a (tile, view) unit and in
//     FP64 across units.
// Algorithmic definitions: Eq. sr_model_vec (A_k = D B W_k) and Sec. 4.1.
#include "lfsr_device.cuh"

namespace lfsr {

constexpr int FT_THREADS = 512;

template <int Z, int KB>
struct FastShape {
  static constexpr int T = 64;                               // tile side (HR px)
  static constexpr int R = (KB - 1) / 2;                     // blur radius
  static constexpr int NL = (T + 2 * R + Z - 1) / Z;         // LR rows/cols touching a tile
  static constexpr int NE = Z * (NL - 1) + 2 * R + 1;        // warp samples per row/col
  static constexpr int MG = (R + Z - 1) / Z + 1;             // zero margin of the LR grid
  static constexpr int NG = NL + 2 * MG;                     // LR grid with margins
  static constexpr int NGp = NG | 1;                         // its (odd) pitch
  // stage 2 (horizontal forward): MB2 LR columns per task
  static constexpr int MB2 = (NL % 5 == 0) ? 5 : 4;
  static constexpr int NB2 = (NL + MB2 - 1) / MB2;
  static constexpr int W2 = Z * (MB2 - 1) + KB;              // window length
  static constexpr int NEp = ((Z * (NB2 * MB2 - 1) + KB) > NE ? (Z * (NB2 * MB2 - 1) + KB) : NE) | 1;
  // stage 3 (vertical forward): MB3 LR rows per task
  static constexpr int MB3 = MB2;
  static constexpr int NB3 = NB2;
  static constexpr int W3 = W2;
  static constexpr int NEr = (Z * (NB3 * MB3 - 1) + KB) > NE ? (Z * (NB3 * MB3 - 1) + KB) : NE;
  static constexpr int NHp = NL | 1;                         // pitch of the forward H buffer
  // stage 5 (adjoint rows): m = floor(hi / Z) over the tile, MB5 per task
  static constexpr int NM = (T - 1) / Z + 2;                 // max m values per tile
  static constexpr int MB5 = 4;
  static constexpr int NB5 = (NM + MB5 - 1) / MB5;
  static constexpr int DMIN = -(R / Z) - 1;                  // safe delta bounds (all phases)
  static constexpr int DMAX = (Z - 1 + R) / Z;
  static constexpr int W5 = MB5 + DMAX - DMIN;
  static constexpr int NVp = NG | 1;                         // pitch of the adjoint V buffer
  // stage 6 (adjoint columns + scatter): n = floor(hj / Z), MB6 per task
  static constexpr int NN = NM;
  static constexpr int MB6 = (Z == 1) ? 8 : 4;
  static constexpr int NB6 = (NN + MB6 - 1) / MB6;
  static constexpr int W6 = MB6 + DMAX - DMIN;
  static constexpr int HV = (NEr * NHp > T * NVp) ? NEr * NHp : T * NVp;  // shared H/V buffer
};

__device__ __forceinline__ void split_shift(float t, int& ip, float& fr) {
  // t in [0, 2^23): ip = floor(t), fr = t - floor(t), exactly, on the FP32 pipe
  const float f = __fadd_rd(t, 8388608.0f);
  ip = __float_as_int(f) - 0x4B000000;
  fr = t - (f - 8388608.0f);
}

template <int MODE, int Z, int KB>
__global__ void __launch_bounds__(FT_THREADS, 1)
k_operator_fast(const Geom g, const OpPlan P, const OpArgs a) {
  using SH = FastShape<Z, KB>;
  constexpr int T = SH::T, R = SH::R, NL = SH::NL, NE = SH::NE, MG = SH::MG, NGp = SH::NGp;
  constexpr int NEp = SH::NEp, NHp = SH::NHp, NVp = SH::NVp;
  extern __shared__ __align__(16) float smem[];
  if (a.check_done && a.sc->cg_done) return;
  float* sP = smem + P.off_P;   // source, (NE + 2S + 1) rows, pitch P.NPc
  float* sO = smem + P.off_W;   // disparity on the sample region, NE x NEp
  float* sW = sO + NE * NEp;    // warped samples, NE x NEp
  float* sHV = smem + P.off_H;  // forward H (NEr x NHp) / adjoint V (T x NVp)
  float* sG = smem + P.off_G;   // LR grid with zero margins, NG x NGp
  float* sA = smem + P.off_A;   // scatter accumulator, NAr x NAc (pitch odd)
  const int tid = threadIdx.x;
  const int S = g.S;
  const float Sf = (float)S;
  const int NPc = P.NPc, NAc = P.NAc;
  const int u_begin = (int)((long long)blockIdx.x * a.units / gridDim.x);
  const int u_end = (int)((long long)(blockIdx.x + 1) * a.units / gridDim.x);
  const size_t q_lr = (size_t)g.H * g.W;
  double part = 0.0;

  int cur_tile = -1;
  int i0 = 0, j0 = 0, lr_lo = 0, lr_n = 0, lc_lo = 0, lc_n = 0, e_r0 = 0, e_c0 = 0;
  int NAr_t = 0, NAc_t = 0;

  for (int t = tid; t < SH::NG * NGp; t += FT_THREADS) sG[t] = 0.f;
  if (MODE != OP_FWD)
    for (int t = tid; t < P.NAr * NAc; t += FT_THREADS) sA[t] = 0.f;

  auto flush = [&]() {
    for (int t = tid; t < NAr_t * NAc_t; t += FT_THREADS) {
      const int ar = t / NAc_t, ac = t - ar * NAc_t;
      const int hi = i0 - S + ar, hj = j0 - S + ac;
      const float v = sA[ar * NAc + ac];
      if (hi >= 0 && hi < g.Hh && hj >= 0 && hj < g.Wh && v != 0.f)
        atomicAdd(a.out + (size_t)hi * g.Wh + hj, a.scale * v);
      sA[ar * NAc + ac] = 0.f;
    }
  };

  for (int u = u_begin; u < u_end; ++u) {
    const int tile = u / a.nviews;
    const int k = a.view0 + (u - tile * a.nviews);
    if (tile != cur_tile) {
      __syncthreads();
      if (cur_tile >= 0 && MODE != OP_FWD) {
        flush();
        __syncthreads();
      }
      cur_tile = tile;
      const int ty = tile / P.tiles_x, tx = tile - ty * P.tiles_x;
      i0 = ty * T;
      j0 = tx * T;
      const int TRr = min(T, g.Hh - i0), TRc = min(T, g.Wh - j0);
      lr_lo = max(0, ceil_div(i0 - R, Z));
      lr_n = min(g.H - 1, floor_div(i0 + TRr - 1 + R, Z)) - lr_lo + 1;
      lc_lo = max(0, ceil_div(j0 - R, Z));
      lc_n = min(g.W - 1, floor_div(j0 + TRc - 1 + R, Z)) - lc_lo + 1;
      e_r0 = Z * lr_lo - R;
      e_c0 = Z * lc_lo - R;
      NAr_t = TRr + 2 * S + 1;
      NAc_t = TRc + 2 * S + 1;
      // stage the source (zero outside the image) and the disparity
      if (MODE != OP_ADJ) {
        const int np = NE + 2 * S + 1;
        for (int t = tid; t < np * np; t += FT_THREADS) {
          const int pr = t / np, pc = t - pr * np;
          const int hi = e_r0 - S + pr, hj = e_c0 - S + pc;
          sP[pr * NPc + pc] = (hi >= 0 && hi < g.Hh && hj >= 0 && hj < g.Wh)
                                  ? __ldg(a.src + (size_t)hi * g.Wh + hj) : 0.f;
        }
      }
      for (int t = tid; t < NE * NE; t += FT_THREADS) {
        const int er = t / NE, ec = t - er * NE;
        const int hi = e_r0 + er, hj = e_c0 + ec;
        sO[er * NEp + ec] = (hi >= 0 && hi < g.Hh && hj >= 0 && hj < g.Wh)
                                ? __ldg(a.disp + (size_t)hi * g.Wh + hj) : 0.f;
      }
      __syncthreads();
    }
    const float tu = g.tu[k], tv = g.tv[k];

    if (MODE != OP_ADJ) {
      // 1. warped samples: outside the image the disparity is 0 and the
      //    staged source is 0, so the sample is 0 without a branch
      for (int t = tid; t < NE * NE; t += FT_THREADS) {
        const int er = t / NE, ec = t - er * NE;
        const float om = sO[er * NEp + ec];
        int iy, ix;
        float fy, fx;
        split_shift(fmaf(tv, om, Sf), iy, fy);
        split_shift(fmaf(tu, om, Sf), ix, fx);
        const float* q = sP + (er + iy) * NPc + (ec + ix);
        const float top = fmaf(fx, q[1] - q[0], q[0]);
        const float bot = fmaf(fx, q[NPc + 1] - q[NPc], q[NPc]);
        sW[er * NEp + ec] = fmaf(fy, bot - top, top);
      }
      __syncthreads();
      // 2. horizontal blur at decimated columns; lanes along rows
      for (int t = tid; t < NE * SH::NB2; t += FT_THREADS) {
        const int er = t % NE, cb = t / NE;
        const float* w = sW + er * NEp + Z * SH::MB2 * cb;
        float win[SH::W2];
#pragma unroll
        for (int c = 0; c < SH::W2; ++c) win[c] = w[c];
#pragma unroll
        for (int o = 0; o < SH::MB2; ++o) {
          float acc = 0.f;
#pragma unroll
          for (int b = 0; b < KB; ++b) acc = fmaf(g.kh[b], win[Z * o + b], acc);
          const int lc = cb * SH::MB2 + o;
          if (lc < NL) sHV[er * NHp + lc] = acc;
        }
      }
      __syncthreads();
      // 3. vertical blur at decimated rows, then the per-LR-pixel step;
      //    lanes along LR columns
      float psum = 0.f;
      for (int t = tid; t < NL * SH::NB3; t += FT_THREADS) {
        const int lc = t % NL, rb = t / NL;
        const float* hcol = sHV + (Z * SH::MB3 * rb) * NHp + lc;
        float win[SH::W3];
#pragma unroll
        for (int c = 0; c < SH::W3; ++c) win[c] = hcol[c * NHp];
#pragma unroll
        for (int o = 0; o < SH::MB3; ++o) {
          const int lr = rb * SH::MB3 + o;
          if (lr >= NL) continue;
          float acc = 0.f;
#pragma unroll
          for (int b = 0; b < KB; ++b) acc = fmaf(g.kv[b], win[Z * o + b], acc);
          float h = 0.f;
          if (lr < lr_n && lc < lc_n) {
            const int gr = lr_lo + lr, gc = lc_lo + lc;
            const bool owned = (Z * gr >= i0) && (Z * gr < i0 + T) && (Z * gc >= j0) &&
                               (Z * gc < j0 + T);
            h = acc;
            if (MODE == OP_NORMAL) {
              if (owned) psum = fmaf(acc, acc, psum);
            } else if (MODE == OP_DATA) {
              const size_t gi = (size_t)k * q_lr + (size_t)gr * g.W + gc;
              const float yv = __ldg(a.y + gi), wa = __ldg(a.wA_old + gi);
              const float res = acc - yv;
              const float uu = fmaf(g.lambda1, res, wa);
              const float wn = fminf(fmaxf(uu, -g.thr), g.thr);
              const float f = 2.f * wn - wa;
              h = fmaf(g.lambda2, res, 0.5f * g.mu * g.lambda1 * f);
              if (owned) {
                a.wA_new[gi] = wn;
                const float dd = wn - wa;
                psum = fmaf(dd, dd, psum);
              }
            } else if (MODE == OP_FWD) {
              if (owned) a.out[(size_t)k * q_lr + (size_t)gr * g.W + gc] = acc;
            }
          }
          sG[(lr + MG) * NGp + (lc + MG)] = h;
        }
      }
      part += (double)psum;
    } else {
      for (int t = tid; t < NL * NL; t += FT_THREADS) {
        const int lr = t / NL, lc = t - lr * NL;
        float v = 0.f;
        if (lr < lr_n && lc < lc_n)
          v = __ldg(a.src + (size_t)k * q_lr + (size_t)(lr_lo + lr) * g.W + (lc_lo + lc));
        sG[(lr + MG) * NGp + (lc + MG)] = v;
      }
    }
    __syncthreads();
    if (MODE == OP_FWD) continue;

    // 4. adjoint blur, rows (polyphase): V(hi, c) for hi in the tile and
    //    every column c of the LR grid (margins included, they are zero)
    const int m_lo = floor_div(i0, Z);
    for (int t = tid; t < SH::NG * SH::NB5; t += FT_THREADS) {
      const int c = t % SH::NG, mb = t / SH::NG;
      const int m0 = m_lo + mb * SH::MB5;
      // window rows l = m0 + DMIN .. m0 + MB5 - 1 + DMAX (grid row l - lr_lo + MG)
      const int r0 = m0 + SH::DMIN - lr_lo + MG;
      float win[SH::W5];
#pragma unroll
      for (int w = 0; w < SH::W5; ++w) {
        const int rr = r0 + w;
        win[w] = (rr >= 0 && rr < SH::NG) ? sG[rr * NGp + c] : 0.f;
      }
#pragma unroll
      for (int o = 0; o < SH::MB5; ++o) {
#pragma unroll
        for (int ph = 0; ph < Z; ++ph) {
          const int hi = Z * (m0 + o) + ph;
          float acc = 0.f;
#pragma unroll
          for (int d = SH::DMIN; d <= SH::DMAX; ++d) {
            const int ai = ph + R - Z * d;
            if (ai >= 0 && ai <= 2 * R) acc = fmaf(g.kv[ai], win[o + d - SH::DMIN], acc);
          }
          const int ri = hi - i0;
          if (ri >= 0 && ri < T) sHV[ri * NVp + c] = acc;
        }
      }
    }
    __syncthreads();
    // 5. adjoint blur, columns (polyphase), then the bilinear scatter W_k^T;
    //    lanes along rows
    const int n_lo = floor_div(j0, Z);
    const int TRr = min(T, g.Hh - i0);
    for (int t = tid; t < T * SH::NB6; t += FT_THREADS) {
      const int i = t % T, nb = t / T;
      if (i >= TRr) continue;
      const int n0 = n_lo + nb * SH::MB6;
      const int c0 = n0 + SH::DMIN - lc_lo + MG;
      float win[SH::W6];
#pragma unroll
      for (int w = 0; w < SH::W6; ++w) {
        const int cc = c0 + w;
        win[w] = (cc >= 0 && cc < SH::NG) ? sHV[i * NVp + cc] : 0.f;
      }
      const int hi = i0 + i;
#pragma unroll
      for (int o = 0; o < SH::MB6; ++o) {
#pragma unroll
        for (int ph = 0; ph < Z; ++ph) {
          const int hj = Z * (n0 + o) + ph;
          if (hj < j0 || hj >= j0 + T || hj >= g.Wh) continue;
          float tv_ = 0.f;
#pragma unroll
          for (int d = SH::DMIN; d <= SH::DMAX; ++d) {
            const int ai = ph + R - Z * d;
            if (ai >= 0 && ai <= 2 * R) tv_ = fmaf(g.kh[ai], win[o + d - SH::DMIN], tv_);
          }
          const float om = sO[(hi - e_r0) * NEp + (hj - e_c0)];
          int iy, ix;
          float fy, fx;
          split_shift(fmaf(tv, om, Sf), iy, fy);
          split_shift(fmaf(tu, om, Sf), ix, fx);
          float* q = sA + (i + iy) * NAc + (hj - j0 + ix);
          const float ty = fy * tv_, by = tv_ - ty;
          atomicAdd(q, by - fx * by);
          atomicAdd(q + 1, fx * by);
          atomicAdd(q + NAc, ty - fx * ty);
          atomicAdd(q + NAc + 1, fx * ty);
        }
      }
    }
    __syncthreads();
  }

  if (MODE != OP_FWD && cur_tile >= 0) {
    __syncthreads();
    flush();
  }
  if (MODE == OP_NORMAL || MODE == OP_DATA) {
    const int slot = (MODE == OP_NORMAL) ? RED_OP : RED_DW_A;
    double total = 0.0;
    if (grid_sum_last<FT_THREADS>(part, a.partials, &a.sc->counter[slot], &total) &&
        threadIdx.x == 0) {
      a.sc->red[slot] = total;
      if (MODE == OP_NORMAL) {
        const double pAp = (double)g.cA * total + (double)g.mu * a.sc->red[RED_NLTV];
        a.sc->pAp = pAp;
        if (!(pAp > 0.0) || !isfinite(pAp)) {
          a.sc->status = -4;  // LFSR_ENUMERIC
          a.sc->cg_done = 1;
          a.sc->alpha = 0.0;
        } else {
          a.sc->alpha = a.sc->pi / pAp;
        }
      } else {
        a.sc->dwA = total;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
template <int Z, int KB>
static size_t fast_layout(const Geom& g, OpPlan* P) {
  using SH = FastShape<Z, KB>;
  const int S = g.S;
  auto al = [](size_t n) { return (n + 3) & ~(size_t)3; };
  P->TH = P->TW = SH::T;
  P->NLr = P->NLc = SH::NL;
  P->NEr = P->NEc = SH::NE;
  P->NPr = SH::NE + 2 * S + 1;
  P->NPc = (SH::NE + 2 * S + 2) | 1;         // +1: the last tap column; odd pitch
  P->NAr = SH::T + 2 * S + 2;
  P->NAc = (SH::T + 2 * S + 2) | 1;
  size_t off = 0;
  P->off_P = (int)off; off += al((size_t)(P->NPr + 1) * P->NPc);
  P->off_W = (int)off; off += al((size_t)2 * SH::NE * SH::NEp);
  P->off_H = (int)off; off += al((size_t)SH::HV);
  P->off_G = (int)off; off += al((size_t)SH::NG * SH::NGp);
  P->off_A = (int)off; off += al((size_t)P->NAr * P->NAc);
  P->smem_bytes = off * sizeof(float);
  P->tiles_x = (g.Wh + SH::T - 1) / SH::T;
  P->tiles_y = (g.Hh + SH::T - 1) / SH::T;
  P->n_tiles = P->tiles_x * P->tiles_y;
  P->threads = FT_THREADS;
  return P->smem_bytes;
}

template <int Z, int KB>
static cudaError_t fast_prepare_zk(int optin) {
  cudaError_t e = set_max_dynamic_smem(k_operator_fast<OP_NORMAL, Z, KB>, optin);
  if (e == cudaSuccess) e = set_max_dynamic_smem(k_operator_fast<OP_DATA, Z, KB>, optin);
  if (e == cudaSuccess) e = set_max_dynamic_smem(k_operator_fast<OP_FWD, Z, KB>, optin);
  if (e == cudaSuccess) e = set_max_dynamic_smem(k_operator_fast<OP_ADJ, Z, KB>, optin);
  return e;
}

template <int Z, int KB>
static int fast_occupancy(size_t smem) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_operator_fast<OP_NORMAL, Z, KB>,
                                                    FT_THREADS, smem) != cudaSuccess)
    return 1;
  return n > 0 ? n : 1;
}

template <int Z, int KB>
static cudaError_t fast_launch_zk(int mode, const Geom& g, const OpPlan& P, const OpArgs& a,
                                  int grid, cudaStream_t s) {
  switch (mode) {
    case OP_NORMAL: k_operator_fast<OP_NORMAL, Z, KB><<<grid, FT_THREADS, P.smem_bytes, s>>>(g, P, a); break;
    case OP_DATA: k_operator_fast<OP_DATA, Z, KB><<<grid, FT_THREADS, P.smem_bytes, s>>>(g, P, a); break;
    case OP_FWD: k_operator_fast<OP_FWD, Z, KB><<<grid, FT_THREADS, P.smem_bytes, s>>>(g, P, a); break;
    case OP_ADJ: k_operator_fast<OP_ADJ, Z, KB><<<grid, FT_THREADS, P.smem_bytes, s>>>(g, P, a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// (Z, KB) pairs with a specialised kernel.
#define LFSR_FAST_CASES(X) \
  X(1, 3) X(1, 5) X(1, 7) X(2, 3) X(2, 5) X(2, 7) X(2, 9) X(3, 5) X(3, 7) X(3, 9) X(4, 7) X(4, 9)

bool fast_supported(const Geom& g) {
  if (!g.separable) return false;
#define X(z, k) if (g.zeta == z && g.kb == k) return true;
  LFSR_FAST_CASES(X)
#undef X
  return false;
}

cudaError_t fast_prepare(const Geom& g, int optin) {
#define X(z, k) if (g.zeta == z && g.kb == k) return fast_prepare_zk<z, k>(optin);
  LFSR_FAST_CASES(X)
#undef X
  return cudaErrorInvalidValue;
}

cudaError_t fast_plan(const Geom& g, OpPlan* P, int smem_limit) {
#define X(z, k)                                                     \
  if (g.zeta == z && g.kb == k) {                                   \
    if (fast_layout<z, k>(g, P) > (size_t)smem_limit)               \
      return cudaErrorInvalidValue;                                 \
    P->ctas_per_sm = fast_occupancy<z, k>(P->smem_bytes);           \
    P->fast = 1;                                                    \
    return cudaSuccess;                                             \
  }
  LFSR_FAST_CASES(X)
#undef X
  return cudaErrorInvalidValue;
}

cudaError_t fast_launch(int mode, const Geom& g, const OpPlan& P, const OpArgs& a, int grid,
                        cudaStream_t s) {
#define X(z, k) if (g.zeta == z && g.kb == k) return fast_launch_zk<z, k>(mode, g, P, a, grid, s);
  LFSR_FAST_CASES(X)
#undef X
  return cudaErrorInvalidValue;
}

}  // namespace lfsr
