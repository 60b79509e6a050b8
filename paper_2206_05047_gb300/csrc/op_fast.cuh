// Specialised fused operator kernel for separable blur kernels of size
// KB in {3,5,7,9} and scale Z in {1,2,3,4}.  One launch runs the (tile,
// view pair) units of one light field (SINGLE) or of every light field of a
// table (a contiguous range of units per CTA, which may span light fields of
// different sizes and angular grids that share zeta, the blur and the
// solver constants).  The same per-(tile, view) pipeline as k_operator
// (warped samples -> decimated separable blur -> per-LR-pixel step ->
// adjoint blur -> bilinear scatter), with every size of the 64 x 64 tile
// known at compile time:
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
#pragma once

#include "lfsr_device.cuh"

namespace lfsr {

constexpr int FT_THREADS = 512;
constexpr int FT_VB = 2;   // views processed together per pass through the stages

// Outputs per task m in [lo, 8] that needs the fewest 512-thread passes for
// `rows` x ceil(n / m) tasks (ties: the smaller m, i.e. fewer registers and
// a shorter chain per thread).
constexpr int pick_block(int rows, int n, int lo = 4) {
  int best = lo, best_passes = 1 << 30;
  for (int m = lo; m <= 8; ++m) {
    const int passes = (rows * ((n + m - 1) / m) + FT_THREADS - 1) / FT_THREADS;
    if (passes < best_passes) {
      best_passes = passes;
      best = m;
    }
  }
  return best;
}

template <int Z, int KB, int TILE = FAST_TILE>
struct FastShape {
  static constexpr int T = TILE;                             // tile side (HR px)
  static constexpr int VB = FT_VB;
  static constexpr int R = (KB - 1) / 2;                     // blur radius
  static constexpr int NL = (T + 2 * R + Z - 1) / Z;         // LR rows/cols touching a tile
  static constexpr int NE = Z * (NL - 1) + 2 * R + 1;        // warp samples per row/col
  static constexpr int MG = (R + Z - 1) / Z + 1;             // zero margin of the LR grid
  static constexpr int NG = NL + 2 * MG;                     // LR grid with margins
  static constexpr int NGp = NG | 1;                         // its (odd) pitch
  // stage 2 (horizontal forward): MB2 LR columns of both views per task
  static constexpr int MB2 = pick_block(NE, NL);
  static constexpr int NB2 = (NL + MB2 - 1) / MB2;
  static constexpr int W2 = Z * (MB2 - 1) + KB;              // window length
  // pitch of the sample buffer: NE itself when odd (the sample index is then
  // the task index); stage 2's last windows read up to NE2 - NE columns past
  // a row, which feed only outputs beyond the LR grid (never stored); the
  // last view's last row reads into the next buffer
  static constexpr int NE2 = (Z * (NB2 * MB2 - 1) + KB) > NE ? (Z * (NB2 * MB2 - 1) + KB) : NE;
  static constexpr int NEp = NE | 1;
  // stage 3 (vertical forward): MB3 LR rows per task
  static constexpr int MB3 = pick_block(VB * NL, NL);
  static constexpr int NB3 = (NL + MB3 - 1) / MB3;
  static constexpr int W3 = Z * (MB3 - 1) + KB;
  static constexpr int NEr = (Z * (NB3 * MB3 - 1) + KB) > NE ? (Z * (NB3 * MB3 - 1) + KB) : NE;
  static constexpr int IT3 = (VB * NL * NB3 + FT_THREADS - 1) / FT_THREADS;
  static constexpr int NHp = NL | 1;                         // pitch of the forward H buffer
  // stage 4 (adjoint rows): m = floor(hi / Z) over the tile, MB5 per task;
  // tiles start at multiples of T, so when Z divides T every tile holds
  // exactly T / Z values of m
  static constexpr bool ALIGNED = (T % Z) == 0;
  static constexpr int NM = ALIGNED ? T / Z : (T - 1) / Z + 2;  // m values per tile
  // (from 3: a single pass then keeps more warps busy with shorter chains)
  static constexpr int MB5 = pick_block(NG, NM, 3);   // both views per task
  static constexpr int NB5 = (NM + MB5 - 1) / MB5;
  static constexpr int DMIN = -(R / Z) - 1;                  // safe delta bounds (all phases)
  static constexpr int DMAX = (Z - 1 + R) / Z;
  static constexpr int W5 = MB5 + DMAX - DMIN;
  static constexpr int NVp = NG | 1;                         // pitch of the adjoint V buffer
  // stage 5 (adjoint columns + scatter): n = floor(hj / Z), MB6 per task
  static constexpr int NN = NM;
  static constexpr int MB6 = pick_block(T, NN);
  static constexpr int NB6 = (NN + MB6 - 1) / MB6;
  static constexpr int W6 = MB6 + DMAX - DMIN;
  static constexpr int HS = NEr * NHp;                       // forward H buffer per view
  static constexpr int VS = T * NVp;                         // adjoint V buffer per view
  static constexpr int GS = NG * NGp;                        // LR grid per view
  static constexpr int WS = NE * NEp;                        // sample buffer per view
  static constexpr int NS1 = NE * NE;                        // warp samples per view
  static constexpr int IT1 = (NS1 + FT_THREADS - 1) / FT_THREADS;
};

// 4-byte asynchronous global -> shared copy; valid == false writes 0 (no
// bytes are read from src, which only has to be a valid address).
__device__ __forceinline__ void cp_async_f32(float* sdst, const float* gsrc, bool valid) {
  const unsigned saddr = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(saddr), "l"(gsrc),
               "r"(valid ? 4 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// Two FP32 lanes per instruction (the packed FFMA2 / FADD2 / FMUL2 of this
// architecture): the two views of a pass go through the same arithmetic in
// the two lanes.  Every lane rounds as the scalar operation it replaces;
// x - y is fma(y, -1, x), one rounding of the exact difference.
__device__ __forceinline__ float2 pk(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}
__device__ __forceinline__ float2 add2_rd(float2 a, float2 b) {
  unsigned long long ra, rb, rd;
  asm("mov.b64 %0, {%1, %2};" : "=l"(ra) : "f"(a.x), "f"(a.y));
  asm("mov.b64 %0, {%1, %2};" : "=l"(rb) : "f"(b.x), "f"(b.y));
  asm("add.rm.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
  float2 d;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(d.x), "=f"(d.y) : "l"(rd));
  return d;
}
// Floor and fraction of a sub-pixel shift t in [0, 2^23), in both lanes,
// exactly, on the FP32 pipe: f = t + 2^23 rounded down holds floor(t) in its
// low mantissa bits, and t - (f - 2^23) is the fraction.  The integer parts
// are left biased: b = floor(t) + SHIFT_BIAS as an unsigned word.  Index arithmetic folds the bias into a
// base term once (unsigned arithmetic wraps modulo 2^32, and every true
// index is small and non-negative), instead of removing it per sample.
constexpr unsigned SHIFT_BIAS = 0x4B000000u;
__device__ __forceinline__ void split_bits2(float2 t, unsigned& b0, unsigned& b1, float2& fr) {
  const float2 f = add2_rd(t, make_float2(8388608.0f, 8388608.0f));
  b0 = __float_as_uint(f.x);
  b1 = __float_as_uint(f.y);
  fr = sub2(t, __fadd2_rn(f, make_float2(-8388608.0f, -8388608.0f)));
}

// SINGLE: one light field whose fields come by value (kernel parameters,
// read from the constant bank); else a table of light fields, the fields of
// the current one in registers.
// The body runs in the kernel below and, as one phase among others, in the
// persistent batch iteration (batch_persist.cuh): every CTA of the launch
// calls it, with the dynamic shared memory laid out by P.  run == false
// takes no unit (the CTA still zeroes its partial slots and arrives at the
// final reduction, which keeps the arrival counters aligned).
template <int MODE, int Z, int KB, bool SINGLE, int TILE = FAST_TILE>
__device__ __forceinline__ void op_fast_body(const Geom& g, const OpPlan& P, const TableArgs& t,
                                             const JobArgs& one, bool run = true) {
  using SH = FastShape<Z, KB, TILE>;
  constexpr int T = SH::T, R = SH::R, NL = SH::NL, NE = SH::NE, MG = SH::MG, NGp = SH::NGp;
  constexpr int NEp = SH::NEp, NHp = SH::NHp, NVp = SH::NVp, VB = SH::VB;
  extern __shared__ __align__(16) float smem[];
  __shared__ double s_red[FT_THREADS / 32];
  float* sP = smem + P.off_P;   // source, (NE + 2S + 1) rows, pitch P.NPc
  float* sO = smem + P.off_W;   // disparity on the sample region, NE x NEp
  float* sW = sO + SH::WS;      // warped samples, VB x NE x NEp
  float* sH = smem + P.off_H;   // forward H, VB x NEr x NHp
  float* sV = sH + VB * SH::HS; // adjoint V, VB x T x NVp (separate from H, so one unit's
                                // scatter may overlap the next unit's forward stages)
  float* sG = smem + P.off_G;   // LR grid with zero margins, VB x NG x NGp
  float* sA = smem + P.off_A;   // scatter accumulator, NAr x NAc (pitch odd)
  const int tid = threadIdx.x;
  const int S = g.S;
  const float Sf = (float)S;
  const int NPc = P.NPc, NAc = P.NAc;
  const int units = run ? t.total_units : 0;
  // this CTA's contiguous range of units: cost-balanced ranges when given,
  // else the even split
  const bool ranged = run && t.cta_unit0 != nullptr;
  const int u_begin = ranged ? __ldg(t.cta_unit0 + blockIdx.x)
                             : (int)((long long)blockIdx.x * units / gridDim.x);
  const int u_end = ranged ? __ldg(t.cta_unit0 + blockIdx.x + 1)
                           : (int)((long long)(blockIdx.x + 1) * units / gridDim.x);
  long long* const clk = t.unit_clock;
  constexpr bool REDUCE = MODE == OP_NORMAL || MODE == OP_DATA;
  // this CTA's partial slot of every light field of the table starts at 0
  if (REDUCE)
    for (int j = tid; j < t.n_jobs; j += FT_THREADS)
      t.partials[(size_t)j * gridDim.x + blockIdx.x] = 0.0;
  double part = 0.0;

  // the light field of the current unit (a CTA's contiguous range of units
  // may span several; all fields are block-uniform)
  // the current light field's fields: kernel parameters (SINGLE) or a
  // shared-memory copy of its table entry, read where used (block-uniform
  // values that never occupy registers across the stages)
  __shared__ JobArgs s_job;
  // SINGLE: the fields and their derived values, computed once from the
  // kernel parameters
  const int p_H = one.H, p_W = one.W, p_Hh = one.Hh, p_Wh = one.Wh;
  const int p_tiles_x = one.tiles_x, p_view0 = one.view0, p_nviews = one.nviews;
  const int p_unit0 = one.unit0;
  const float p_scale = one.scale;
  const float* const p_src = one.src;
  const float* const p_disp = one.disp;
  float* const p_out = one.out;
  const void* const p_y = one.y;
  const void* const p_wA_old = one.wA_old;
  void* const p_wA_new = one.wA_new;
  const int p_nvb = (one.nviews + VB - 1) / VB;
  const size_t p_qlr = (size_t)one.H * one.W;
  const float2* const p_theta = one.theta;
#define JF(f) (SINGLE ? p_##f : s_job.f)
#define JNVB (SINGLE ? p_nvb : (s_job.nviews + VB - 1) / VB)
#define JQLR (SINGLE ? p_qlr : (size_t)s_job.H * s_job.W)

  int jb = -1, j_end = 0;
  bool skip = false;
  // angular offset theta_k of data view k (Sec. 3.1), from the light
  // field's table (the views may be a subset of the grid)
  auto tu_of = [&](int k) { return __ldg(&JF(theta)[k].x); };
  auto tv_of = [&](int k) { return __ldg(&JF(theta)[k].y); };

  static_assert(VB == 2, "the sample and scatter stages handle view pairs");
  int cur_tile = -1;
  int i0 = 0, j0 = 0, lr_lo = 0, lr_n = 0, lc_lo = 0, lc_n = 0, e_r0 = 0, e_c0 = 0;
  int or0 = 0, or1 = 0, oc0 = 0, oc1 = 0;   // LR rows / columns owned by the tile (grid-local)
  int NAr_t = 0, NAc_t = 0;
  // this thread's warp-sample positions (fixed for all views of a tile):
  // staged-source index of the (0, 0) tap before the shift (less the bias
  // of the shift's split, SHIFT_BIAS (NPc + 1)), and disparity
  unsigned s1_base[SH::IT1];
  float s1_om[SH::IT1];

  for (int t = tid; t < VB * SH::GS; t += FT_THREADS) sG[t] = 0.f;
  if (MODE != OP_FWD)
    for (int t = tid; t < P.NAr * NAc; t += FT_THREADS) sA[t] = 0.f;

  auto flush = [&]() {
    const int warp = tid >> 5, lane = tid & 31;
    for (int ar = warp; ar < NAr_t; ar += FT_THREADS / 32) {
      const int hi = i0 - S + ar;
      const bool row_in = hi >= 0 && hi < JF(Hh);
      for (int ac = lane; ac < NAc_t; ac += 32) {
        const int hj = j0 - S + ac;
        const float v = sA[ar * NAc + ac];
        if (row_in && hj >= 0 && hj < JF(Wh) && v != 0.f)
          atomicAdd(JF(out) + (size_t)hi * JF(Wh) + hj, JF(scale) * v);
        sA[ar * NAc + ac] = 0.f;
      }
    }
  };
  // end of this CTA's share of a light field: flush the last tile, store
  // the partial sum in the light field's slot
  auto end_job = [&]() {
    __syncthreads();
    if (cur_tile >= 0 && MODE != OP_FWD) flush();
    cur_tile = -1;
    if (REDUCE) {
      const double bs = block_sum<FT_THREADS>(part, s_red);
      if (tid == 0) t.partials[(size_t)jb * gridDim.x + blockIdx.x] = bs;
      part = 0.0;
    }
    __syncthreads();
  };

  if (SINGLE) {
    jb = 0;
    j_end = units;
    skip = t.check_done && ((volatile int*)&one.sc->cg_done)[0];
  }

  for (int u = u_begin; u < u_end; ++u) {
    if (clk && tid == 0) clk[u] = clock64();
    if (!SINGLE && u >= j_end) {
      if (jb >= 0) end_job();
      jb = table_job(t, u);
      if (tid == 0) s_job = t.jobs[jb];
      __syncthreads();
      j_end = s_job.unit0 + s_job.units;
      skip = t.check_done && ((volatile int*)&s_job.sc->cg_done)[0];
    }
    if (skip) continue;
    const int ul = u - JF(unit0);
    const int tile = ul / JNVB;
    const int kbase = JF(view0) + VB * (ul - tile * JNVB);
    const int nv = min(VB, JF(view0) + JF(nviews) - kbase);   // views of this unit
    if (tile != cur_tile) {
      __syncthreads();
      if (cur_tile >= 0 && MODE != OP_FWD) {
        flush();
        __syncthreads();
      }
      cur_tile = tile;
      const int ty = tile / JF(tiles_x), tx = tile - ty * JF(tiles_x);
      i0 = ty * T;
      j0 = tx * T;
      const int TRr = min(T, JF(Hh) - i0), TRc = min(T, JF(Wh) - j0);
      lr_lo = max(0, ceil_div(i0 - R, Z));
      lr_n = min(JF(H) - 1, floor_div(i0 + TRr - 1 + R, Z)) - lr_lo + 1;
      lc_lo = max(0, ceil_div(j0 - R, Z));
      lc_n = min(JF(W) - 1, floor_div(j0 + TRc - 1 + R, Z)) - lc_lo + 1;
      e_r0 = Z * lr_lo - R;
      e_c0 = Z * lc_lo - R;
      // LR pixel (gr, gc) belongs to the tile when its HR position (Z gr, Z gc)
      // lies in it: gr in [ceil(i0 / Z), ceil((i0 + T) / Z))
      or0 = ceil_div(i0, Z) - lr_lo;
      or1 = ceil_div(i0 + T, Z) - lr_lo;
      oc0 = ceil_div(j0, Z) - lc_lo;
      oc1 = ceil_div(j0 + T, Z) - lc_lo;
      NAr_t = TRr + 2 * S + 1;
      NAc_t = TRc + 2 * S + 1;
      // stage the source (zero outside the image) and the disparity with
      // asynchronous copies: every copy of the tile is in flight at once
      {
        const int warp = tid >> 5, lane = tid & 31;
        constexpr int NWARP = FT_THREADS / 32;
        if (MODE != OP_ADJ) {
          const int np = NE + 2 * S + 1;
          for (int pr = warp; pr < np; pr += NWARP) {
            const int hi = e_r0 - S + pr;
            const bool row_in = hi >= 0 && hi < JF(Hh);
            const float* src_row = JF(src) + (size_t)(row_in ? hi : 0) * JF(Wh);
            for (int pc = lane; pc < np; pc += 32) {
              const int hj = e_c0 - S + pc;
              const bool ok = row_in && hj >= 0 && hj < JF(Wh);
              cp_async_f32(sP + pr * NPc + pc, ok ? src_row + hj : JF(src), ok);
            }
          }
        }
        for (int er = warp; er < NE; er += NWARP) {
          const int hi = e_r0 + er;
          const bool row_in = hi >= 0 && hi < JF(Hh);
          const float* d_row = JF(disp) + (size_t)(row_in ? hi : 0) * JF(Wh);
          for (int ec = lane; ec < NE; ec += 32) {
            const int hj = e_c0 + ec;
            const bool ok = row_in && hj >= 0 && hj < JF(Wh);
            cp_async_f32(sO + er * NEp + ec, ok ? d_row + hj : JF(disp), ok);
          }
        }
        cp_async_wait_all();
      }
      __syncthreads();
      if (MODE != OP_ADJ) {
#pragma unroll
        for (int it = 0; it < SH::IT1; ++it) {
          const int t = tid + it * FT_THREADS;
          const int er = t / NE, ec = t - er * NE;
          const bool ok = t < SH::NS1;
          s1_base[it] = ok ? (unsigned)(er * NPc + ec) - SHIFT_BIAS * (unsigned)(NPc + 1) : 0u;
          s1_om[it] = ok ? sO[er * NEp + ec] : 0.f;
        }
      }
    }

    // data block: fetch the views' LR values and duals now, so the loads are
    // in flight during the warp and blur stages
    // (raw words of the storage kinds; widened at use)
    unsigned int pre_y[SH::IT3][SH::MB3], pre_w[SH::IT3][SH::MB3];
    if (MODE == OP_DATA) {
#pragma unroll
      for (int it = 0; it < SH::IT3; ++it) {
        const int t = tid + it * FT_THREADS;
        const int v = t / (NL * SH::NB3), r3 = t - v * (NL * SH::NB3);
        const int lc = r3 % NL, rb = r3 / NL;
#pragma unroll
        for (int o = 0; o < SH::MB3; ++o) {
          const int lr = rb * SH::MB3 + o;
          pre_y[it][o] = 0u;
          pre_w[it][o] = 0u;
          if (v < nv && lr < lr_n && lc < lc_n) {
            const size_t gi = (size_t)(kbase + v) * JQLR + (size_t)(lr_lo + lr) * JF(W) + (lc_lo + lc);
            pre_y[it][o] = ld_raw_kind(JF(y), gi, g.st_y);
            pre_w[it][o] = ld_raw_kind(JF(wA_old), gi, g.st);
          }
        }
      }
    }

    if (MODE != OP_ADJ) {
      // 1. warped samples: outside the image the disparity is 0 and the
      //    staged source is 0, so the sample is 0 without a branch.  The
      //    two views of the pass share the disparity read and, when they
      //    lie in the same row of the angular grid, the vertical split.
      //    Both views in the two lanes of packed FP32 operations (for a
      //    single-view pass the second lane repeats the first view and is
      //    not stored).
      const bool two = nv > 1;
      {
        const int k1 = kbase + (two ? 1 : 0);
        const float2 tu2 = pk(tu_of(kbase), tu_of(k1)), tv2 = pk(tv_of(kbase), tv_of(k1));
        const float2 S2 = pk(Sf, Sf);
#pragma unroll
        for (int it = 0; it < SH::IT1; ++it) {
          const int t = tid + it * FT_THREADS;
          if (it < SH::IT1 - 1 || t < SH::NS1) {
            const int si = (NEp == NE) ? t : (t / NE) * NEp + (t % NE);
            const float2 om2 = pk(s1_om[it], s1_om[it]);
            unsigned by0, by1, bx0, bx1;
            float2 fy, fx;
            split_bits2(fma2(tv2, om2, S2), by0, by1, fy);
            split_bits2(fma2(tu2, om2, S2), bx0, bx1, fx);
            const float* qa = sP + (int)(s1_base[it] + by0 * (unsigned)NPc + bx0);
            const float* qc = sP + (int)(s1_base[it] + by1 * (unsigned)NPc + bx1);
            const float2 a = pk(qa[0], qc[0]), b = pk(qa[1], qc[1]);
            const float2 c = pk(qa[NPc], qc[NPc]), d = pk(qa[NPc + 1], qc[NPc + 1]);
            const float2 top = fma2(fx, sub2(b, a), a);
            const float2 bot = fma2(fx, sub2(d, c), c);
            const float2 o = fma2(fy, sub2(bot, top), top);
            sW[si] = o.x;
            if (two) sW[SH::WS + si] = o.y;
          }
        }
      }
      __syncthreads();
      // 2. horizontal blur at decimated columns, both views per task; lanes
      //    along rows
      for (int t = tid; t < NE * SH::NB2; t += FT_THREADS) {
        const int er = t % NE, cb = t / NE;
        const float* w = sW + er * NEp + Z * SH::MB2 * cb;
        float2 win[SH::W2];
#pragma unroll
        for (int c = 0; c < SH::W2; ++c) win[c] = pk(w[c], w[SH::WS + c]);
#pragma unroll
        for (int o = 0; o < SH::MB2; ++o) {
          float2 acc = pk(0.f, 0.f);
#pragma unroll
          for (int b = 0; b < KB; ++b) acc = fma2(pk(g.kh[b], g.kh[b]), win[Z * o + b], acc);
          const int lc = cb * SH::MB2 + o;
          if (lc < NL) {
            sH[er * NHp + lc] = acc.x;
            if (two) sH[SH::HS + er * NHp + lc] = acc.y;
          }
        }
      }
      __syncthreads();
      // 3. vertical blur at decimated rows, then the per-LR-pixel step;
      //    lanes along LR columns
      float psum = 0.f;
#pragma unroll
      for (int it = 0; it < SH::IT3; ++it) {
        const int t = tid + it * FT_THREADS;
        const int v = t / (NL * SH::NB3), r3 = t - v * (NL * SH::NB3);
        if (v >= nv) break;
        const int lc = r3 % NL, rb = r3 / NL;
        const int k = kbase + v;
        const bool col_in = lc < lc_n, col_own = lc >= oc0 && lc < oc1;
        const float* hcol = sH + v * SH::HS + (Z * SH::MB3 * rb) * NHp + lc;
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
          if (lr < lr_n && col_in) {
            const int gr = lr_lo + lr, gc = lc_lo + lc;
            const bool owned = col_own && lr >= or0 && lr < or1;
            h = acc;
            if (MODE == OP_NORMAL) {
              if (owned) psum = fmaf(acc, acc, psum);
            } else if (MODE == OP_DATA) {
              const size_t gi = (size_t)k * JQLR + (size_t)gr * JF(W) + gc;
              const float yv = raw_to_float(pre_y[it][o], g.st_y);
              const float wa = raw_to_float(pre_w[it][o], g.st);
              const float res = acc - yv;
              const float uu = fmaf(g.lambda1, res, wa);
              const float wn = fminf(fmaxf(uu, -g.thr), g.thr);
              const float f = 2.f * wn - wa;
              h = fmaf(g.lambda2, res, 0.5f * g.mu * g.lambda1 * f);
              if (owned) {
                st_kind(JF(wA_new), gi, g.st, wn);
                const float dd = wn - wa;
                psum = fmaf(dd, dd, psum);
              }
            } else if (MODE == OP_FWD) {
              if (owned) JF(out)[(size_t)k * JQLR + (size_t)gr * JF(W) + gc] = acc;
            }
          }
          sG[v * SH::GS + (lr + MG) * NGp + (lc + MG)] = h;
        }
      }
      part += (double)psum;
    } else {
      for (int t = tid; t < VB * NL * NL; t += FT_THREADS) {
        const int v = t / (NL * NL), r0 = t - v * (NL * NL);
        if (v >= nv) continue;
        const int lr = r0 / NL, lc = r0 - lr * NL;
        float val = 0.f;
        if (lr < lr_n && lc < lc_n)
          val = __ldg(JF(src) + (size_t)(kbase + v) * JQLR + (size_t)(lr_lo + lr) * JF(W) + (lc_lo + lc));
        sG[v * SH::GS + (lr + MG) * NGp + (lc + MG)] = val;
      }
    }
    __syncthreads();
    if (MODE == OP_FWD) continue;

    // 4. adjoint blur, rows (polyphase): V(hi, c) for hi in the tile and
    //    every column c of the LR grid (margins included, they are zero)
    const int m_lo = floor_div(i0, Z);
    const bool two = nv > 1;
    for (int t = tid; t < SH::NG * SH::NB5; t += FT_THREADS) {
      const int c = t % SH::NG, mb = t / SH::NG;
      const int m0 = m_lo + mb * SH::MB5;
      // window rows l = m0 + DMIN .. m0 + MB5 - 1 + DMAX (grid row l - lr_lo + MG),
      // both views (the second view's grid is stale for a single-view pass)
      const int r0 = m0 + SH::DMIN - lr_lo + MG;
      float2 win[SH::W5];
#pragma unroll
      for (int w = 0; w < SH::W5; ++w) {
        const int rr = r0 + w;
        win[w] = (rr >= 0 && rr < SH::NG) ? pk(sG[rr * NGp + c], sG[SH::GS + rr * NGp + c])
                                          : pk(0.f, 0.f);
      }
#pragma unroll
      for (int o = 0; o < SH::MB5; ++o) {
#pragma unroll
        for (int ph = 0; ph < Z; ++ph) {
          const int hi = Z * (m0 + o) + ph;
          float2 acc = pk(0.f, 0.f);
#pragma unroll
          for (int d = SH::DMIN; d <= SH::DMAX; ++d) {
            const int ai = ph + R - Z * d;
            if (ai >= 0 && ai <= 2 * R)
              acc = fma2(pk(g.kv[ai], g.kv[ai]), win[o + d - SH::DMIN], acc);
          }
          const int ri = hi - i0;
          if (ri >= 0 && ri < T) {
            sV[ri * NVp + c] = acc.x;
            if (two) sV[SH::VS + ri * NVp + c] = acc.y;
          }
        }
      }
    }
    __syncthreads();
    // 5. adjoint blur, columns (polyphase), then the bilinear scatter W_k^T;
    //    lanes along rows; one task covers the same pixels in both views
    const int n_lo = floor_div(j0, Z);
    const int TRr = min(T, JF(Hh) - i0);
    const bool full_cols = j0 + T <= JF(Wh);
    const int k1 = kbase + (two ? 1 : 0);
    const float2 tu2 = pk(tu_of(kbase), tu_of(k1)), tv2 = pk(tv_of(kbase), tv_of(k1));
    const float2 S2 = pk(Sf, Sf);
    for (int t = tid; t < T * SH::NB6; t += FT_THREADS) {
      const int i = t % T, nb = t / T;
      if (i >= TRr) continue;
      const int n0 = n_lo + nb * SH::MB6;
      const int c0 = n0 + SH::DMIN - lc_lo + MG;     // in [0, NG - W6] for every tile
      float2 win[SH::W6];
      {
        const float* v0 = sV + i * NVp + c0;
        const float* v1 = v0 + SH::VS;
#pragma unroll
        for (int w = 0; w < SH::W6; ++w) win[w] = pk(v0[w], two ? v1[w] : 0.f);
      }
      const int hi = i0 + i;
      const float* orow = sO + (hi - e_r0) * NEp - e_c0;
      // accumulator index of the (0, 0) tap of pixel (hi, Z n0) before its
      // shift, less the bias of the shift's split
      const unsigned a_row = (unsigned)(i * NAc + Z * n0 - j0) - SHIFT_BIAS * (unsigned)(NAc + 1);
      // taps of consecutive pixels of this row segment: when a pixel's
      // integer shift equals its left neighbour's, its left taps coincide
      // with the neighbour's right taps and are added before one atomic
      bool pend0 = false, pend1 = false;
      unsigned pa0 = 0u, pa1 = 0u;
      float pt0 = 0.f, pb0 = 0.f, pt1 = 0.f, pb1 = 0.f;
      // tl, bl, tr, br: the bilinear weights times the value, for the taps
      // a, a + NAc, a + 1, a + NAc + 1 (a: accumulator index of the top-left)
      auto scatter = [&](float tl, float bl, float tr, float br, unsigned a, bool& pend,
                         unsigned& pa, float& pt, float& pb) {
        const bool merged = pend && pa == a;
        if (pend && !merged) {
          atomicAdd(sA + pa, pt);
          atomicAdd(sA + pa + NAc, pb);
        }
        tl += merged ? pt : 0.f;
        bl += merged ? pb : 0.f;
        atomicAdd(sA + a, tl);
        atomicAdd(sA + a + NAc, bl);
        pend = true;
        pa = a + 1;
        pt = tr;
        pb = br;
      };
      auto pixel = [&](int o, int ph) {
        const int hj = Z * (n0 + o) + ph;
        float2 tv = pk(0.f, 0.f);          // the adjoint-blurred value of both views
#pragma unroll
        for (int d = SH::DMIN; d <= SH::DMAX; ++d) {
          const int ai = ph + R - Z * d;
          if (ai >= 0 && ai <= 2 * R) tv = fma2(pk(g.kh[ai], g.kh[ai]), win[o + d - SH::DMIN], tv);
        }
        const float om = orow[hj];
        const float2 om2 = pk(om, om);
        const unsigned ap = a_row + (unsigned)(Z * o + ph);
        unsigned by0, by1, bx0, bx1;
        float2 fy, fx;
        split_bits2(fma2(tv2, om2, S2), by0, by1, fy);
        split_bits2(fma2(tu2, om2, S2), bx0, bx1, fx);
        // weights times the value: the bottom / top rows' shares, then the
        // right taps' shares and the left ones as the remainders
        const float2 ty = mul2(fy, tv);
        const float2 by = sub2(tv, ty);
        const float2 tr = mul2(fx, by), br = mul2(fx, ty);
        const float2 tl = sub2(by, tr), bl = sub2(ty, br);
        scatter(tl.x, bl.x, tr.x, br.x, ap + by0 * (unsigned)NAc + bx0, pend0, pa0, pt0, pb0);
        if (two) scatter(tl.y, bl.y, tr.y, br.y, ap + by1 * (unsigned)NAc + bx1, pend1, pa1, pt1, pb1);
      };
      if (SH::ALIGNED && full_cols) {
#pragma unroll
        for (int o = 0; o < SH::MB6; ++o)
#pragma unroll
          for (int ph = 0; ph < Z; ++ph) pixel(o, ph);
      } else {
#pragma unroll
        for (int o = 0; o < SH::MB6; ++o)
#pragma unroll
          for (int ph = 0; ph < Z; ++ph) {
            const int hj = Z * (n0 + o) + ph;
            if (hj >= j0 && hj < j0 + T && hj < JF(Wh)) pixel(o, ph);
          }
      }
      if (pend0) {
        atomicAdd(sA + pa0, pt0);
        atomicAdd(sA + pa0 + NAc, pb0);
      }
      if (pend1) {
        atomicAdd(sA + pa1, pt1);
        atomicAdd(sA + pa1 + NAc, pb1);
      }
    }
    // no barrier here: the next unit's stages 1-2 write sW and sH, which this
    // stage does not read, and sG / sV are rewritten only after two barriers;
    // a tile change starts with a barrier before the flush
  }

  if (jb >= 0) end_job();   // (SINGLE: always; ends with a barrier after the last flush)
  if (clk) {                // a timing launch
    if (tid == 0) clk[units + blockIdx.x] = clock64();
    return;
  }
  if (SINGLE && MODE == OP_DATA && one.fuse) {
    // The x-step initialisation (Algorithm 2) in the same launch: once
    // every CTA has flushed its v atomics, each CTA takes its chunk of the
    // accumulated v (the regulariser's part came from the NLTV block):
    // r = -v, v := 0 for the next iteration, x' = x, and its partial of
    // pi = <r, r>; after a second barrier CTA 0 finishes pi and the fresh
    // CG state.
    DevScalars* sc = one.sc;
    const bool ok1 = grid_barrier(&sc->bar, g);
    if (ok1 && blockIdx.x == 0 && tid < 32) {
      const double total = warp_sum_slots(t.partials, gridDim.x);
      if (tid == 0) {
        sc->red[RED_DW_A] = total;
        sc->dwA = total;
      }
    }
    double rr = 0.0;
    const int n = p_Hh * p_Wh;
    const int c0 = blockIdx.x * one.fchunk;
    const int c1 = min(n, c0 + one.fchunk);   // may be <= c0: the last CTAs can have no pixels
    if (ok1 && c0 < c1) {
      float* __restrict__ va = one.vacc;
      float* __restrict__ rv = one.rr;
      const float* __restrict__ xs = one.src;
      float* __restrict__ xn = one.x_next;
      const int v0 = c0 >> 2, v1 = c1 >> 2;
      const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int v = v0 + tid; v < v1; v += FT_THREADS) {
        const float4 a4 = __ldcg(reinterpret_cast<const float4*>(va) + v);
        reinterpret_cast<float4*>(va)[v] = z4;
        const float4 r4 = make_float4(-a4.x, -a4.y, -a4.z, -a4.w);
        reinterpret_cast<float4*>(rv)[v] = r4;
        reinterpret_cast<float4*>(xn)[v] = __ldg(reinterpret_cast<const float4*>(xs) + v);
        rr += (double)r4.x * (double)r4.x;
        rr += (double)r4.y * (double)r4.y;
        rr += (double)r4.z * (double)r4.z;
        rr += (double)r4.w * (double)r4.w;
      }
      for (int i = 4 * v1 + tid; i < c1; i += FT_THREADS) {
        const float r = -__ldcg(va + i);
        va[i] = 0.f;
        rv[i] = r;
        xn[i] = xs[i];
        rr += (double)r * (double)r;
      }
    }
    {
      const double bs = block_sum<FT_THREADS>(rr, s_red);
      if (tid == 0) one.fpart[blockIdx.x] = bs;
    }
    const bool ok2 = grid_barrier(&sc->bar, g);
    if (!ok1 || !ok2) {
      if (tid == 0) set_status(sc, -5);   // LFSR_ETIMEOUT
      return;
    }
    if (blockIdx.x == 0 && tid < 32) {
      const double total = warp_sum_slots(one.fpart, gridDim.x);
      if (tid == 0) {
        sc->pi = total;
        sc->cg_first = 1;
        sc->cg_steps = 0;
        sc->beta = 0.0;
        sc->dw2 = sc->dwA + sc->dwS;
        if (!isfinite(total)) set_status(sc, -4);  // LFSR_ENUMERIC
        sc->cg_done = (total > g.tau && isfinite(total)) ? 0 : 1;
      }
    }
    return;
  }
  if (SINGLE && MODE == OP_NORMAL && one.fuse) {
    // The rest of the CG step (Algorithm 2) in the same launch: once every
    // CTA has flushed its q atomics and stored its <p, A^T A p> partial, each
    // CTA forms the step length from the partials (the same sum in the same
    // order in every CTA), updates its chunk of x' and r, and its partial of
    // pi' = <r, r>; after a second barrier CTA 0 finishes pi', beta and the
    // step count.  A finished x-step (skip) returns in every CTA alike.
    if (skip) return;
    DevScalars* sc = one.sc;
    __shared__ double s_alpha;
    __shared__ int s_go;
    const bool ok1 = grid_barrier(&sc->bar, g);
    if (tid < 32) {
      const double total = warp_sum_slots(t.partials, gridDim.x);
      if (tid == 0) {
        const double pAp =
            (double)g.cA * total + (double)g.mu * ((volatile double*)sc->red)[RED_NLTV];
        const bool good = pAp > 0.0 && isfinite(pAp);
        s_alpha = good ? ((volatile double*)&sc->pi)[0] / pAp : 0.0;
        s_go = ok1 && good;
        if (blockIdx.x == 0 && ok1) {
          sc->red[RED_OP] = total;
          sc->pAp = pAp;
          sc->alpha = s_alpha;
          if (!good) {
            // a curvature of exactly 0 ends the x-step; a negative or
            // non-finite one is a numeric failure (as cg_set_alpha)
            sc->cg_done = 1;
            if (!(pAp == 0.0)) set_status(sc, -4);  // LFSR_ENUMERIC
          }
        }
      }
    }
    __syncthreads();
    double rr = 0.0;
    const int n = p_Hh * p_Wh;
    const int c0 = blockIdx.x * one.fchunk;
    const int c1 = min(n, c0 + one.fchunk);   // may be <= c0: the last CTAs can have no pixels
    if (s_go && c0 < c1) {
      const float alpha = (float)s_alpha;
      const float* __restrict__ pv = one.p_old;
      const float* __restrict__ qv = one.q;
      float* __restrict__ rv = one.rr;
      float* __restrict__ xv = one.x_next;
      // chunks are whole multiples of 32 floats on 256-byte aligned buffers
      const int v0 = c0 >> 2, v1 = c1 >> 2;
      for (int v = v0 + tid; v < v1; v += FT_THREADS) {
        const float4 pp = __ldg(reinterpret_cast<const float4*>(pv) + v);
        const float4 qq = __ldcg(reinterpret_cast<const float4*>(qv) + v);
        float4 r4 = reinterpret_cast<const float4*>(rv)[v];
        float4 x4 = reinterpret_cast<const float4*>(xv)[v];
        x4.x = fmaf(alpha, pp.x, x4.x);
        x4.y = fmaf(alpha, pp.y, x4.y);
        x4.z = fmaf(alpha, pp.z, x4.z);
        x4.w = fmaf(alpha, pp.w, x4.w);
        r4.x = fmaf(-alpha, qq.x, r4.x);
        r4.y = fmaf(-alpha, qq.y, r4.y);
        r4.z = fmaf(-alpha, qq.z, r4.z);
        r4.w = fmaf(-alpha, qq.w, r4.w);
        reinterpret_cast<float4*>(xv)[v] = x4;
        reinterpret_cast<float4*>(rv)[v] = r4;
        rr += (double)r4.x * (double)r4.x;
        rr += (double)r4.y * (double)r4.y;
        rr += (double)r4.z * (double)r4.z;
        rr += (double)r4.w * (double)r4.w;
      }
      for (int i = 4 * v1 + tid; i < c1; i += FT_THREADS) {
        xv[i] = fmaf(alpha, pv[i], xv[i]);
        const float rn = fmaf(-alpha, __ldcg(qv + i), rv[i]);
        rv[i] = rn;
        rr += (double)rn * (double)rn;
      }
    }
    {
      const double bs = block_sum<FT_THREADS>(rr, s_red);
      if (tid == 0) one.fpart[blockIdx.x] = bs;
    }
    const bool ok2 = grid_barrier(&sc->bar, g);
    if (!ok1 || !ok2) {
      if (tid == 0) set_status(sc, -5);   // LFSR_ETIMEOUT
      return;
    }
    if (blockIdx.x == 0 && s_go && tid < 32) {
      const double total = warp_sum_slots(one.fpart, gridDim.x);
      if (tid == 0) {
        const double pi_old = sc->pi;
        sc->beta = total / pi_old;
        sc->pi = total;
        sc->cg_first = 0;
        sc->cg_steps += 1;
        if (!isfinite(total)) set_status(sc, -4);  // LFSR_ENUMERIC
        if (!(total > g.tau) || !isfinite(total)) sc->cg_done = 1;
      }
    }
    return;
  }
  if (REDUCE && table_arrive_last(t.counter)) {
    // every light field's total over the CTAs' slots, one warp per light field
    const int warp = tid >> 5, lane = tid & 31;
    for (int j = warp; j < t.n_jobs; j += FT_THREADS / 32) {
      DevScalars* sc = SINGLE ? one.sc : t.jobs[j].sc;
      if (t.check_done && ((volatile int*)&sc->cg_done)[0]) continue;
      const double total = warp_sum_slots(t.partials + (size_t)j * gridDim.x, gridDim.x);
      if (lane != 0) continue;
      if (MODE == OP_NORMAL) {
        sc->red[RED_OP] = total;
        cg_set_alpha(sc, (double)g.cA * total + (double)g.mu * sc->red[RED_NLTV]);
      } else {
        sc->red[RED_DW_A] = total;
        sc->dwA = total;
      }
    }
  }
#undef JF
#undef JNVB
#undef JQLR
}

template <int MODE, int Z, int KB, bool SINGLE, int TILE = FAST_TILE>
__global__ void __launch_bounds__(FT_THREADS, 1)
k_operator_fast(const Geom g, const OpPlan P, const TableArgs t, const JobArgs one) {
  op_fast_body<MODE, Z, KB, SINGLE, TILE>(g, P, t, one);
}

// Shared-memory layout and tiling of the specialised kernel for tile side
// TILE (host side; S from g).
// bank_pitch: the staged source's row pitch is congruent to NE modulo 32,
// so that the warp-sample reads of consecutive sample indices t (rows of NE
// samples wrap inside a warp) fall on bank t mod 32 where the shifts agree;
// else the smallest odd pitch (less shared memory).
template <int Z, int KB, int TILE = FAST_TILE>
inline size_t fast_layout(const Geom& g, OpPlan* P, bool bank_pitch = true) {
  using SH = FastShape<Z, KB, TILE>;
  const int S = g.S;
  auto al = [](size_t n) { return (n + 3) & ~(size_t)3; };
  P->TH = P->TW = SH::T;
  P->NLr = P->NLc = SH::NL;
  P->NEr = P->NEc = SH::NE;
  P->NPr = SH::NE + 2 * S + 1;
  const int np = SH::NE + 2 * S + 2;         // +1: the last tap column
  P->NPc = bank_pitch ? SH::NE + 32 * ((np - SH::NE + 31) / 32) : (np | 1);
  P->NAr = SH::T + 2 * S + 2;
  P->NAc = (SH::T + 2 * S + 2) | 1;
  size_t off = 0;
  P->off_P = (int)off; off += al((size_t)(P->NPr + 1) * P->NPc);
  P->off_W = (int)off; off += al((size_t)(1 + SH::VB) * SH::WS);
  P->off_H = (int)off; off += al((size_t)SH::VB * (SH::HS + SH::VS));
  P->off_G = (int)off; off += al((size_t)SH::VB * SH::GS);
  P->off_A = (int)off; off += al((size_t)P->NAr * P->NAc);
  P->smem_bytes = off * sizeof(float);
  P->tiles_x = (g.Wh + SH::T - 1) / SH::T;
  P->tiles_y = (g.Hh + SH::T - 1) / SH::T;
  P->n_tiles = P->tiles_x * P->tiles_y;
  P->threads = FT_THREADS;
  return P->smem_bytes;
}

// (Z, KB) pairs with a specialised kernel.
#define LFSR_FAST_CASES(X) \
  X(1, 3) X(1, 5) X(1, 7) X(2, 3) X(2, 5) X(2, 7) X(2, 9) X(3, 5) X(3, 7) X(3, 9) X(4, 7) X(4, 9)

}  // namespace lfsr
