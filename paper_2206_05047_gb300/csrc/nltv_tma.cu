// Weighted non-local TV with stored edge weights, the weighted divergence
// S^T W^2 S p of a CG step (Sec. 4.1 wdg/wdd, the regulariser part of the
// normal matrix, Sec. 5) with the edge weights staged by the tensor memory
// accelerator.  For a 32 x 32 tile and a direction d of the half window the
// pixel u uses the weight of edge (u, u + d), stored at u, and of edge
// (u - d, u), stored at u - d: both lie in one box of the direction's weight
// plane, the tile plus WR rows below and WR columns either side.  A CTA
// loads the boxes of CH directions at a time with one cp.async.bulk.tensor
// copy (out-of-image elements read as zero, which is the weight of an edge
// that leaves the image) into one of two shared-memory buffers, computes
// from shared memory while the next chunk is in flight, and so reads each
// weight once, in bulk, instead of twice with a load of its own.  The
// arithmetic is that of k_nla2 (nltv_fast.cu), in the same order.
#include <cuda.h>

#include <cstring>

#include "nltv_fast.cuh"

namespace lfsr {

namespace {

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// 3-D tiled copy of one box of the tensor map at (x, y, z) into dst,
// completing on bar.
__device__ __forceinline__ void tma_load_3d(void* dst, const void* map, int x, int y, int z,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}
// Waits, bounded by g.wait_ns of %globaltimer, for phase `parity` of bar.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity,
                                                  const Geom& g) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (global_ns() - t0 >= g.wait_ns) return false;
    __nanosleep(32);
  }
  return true;
}

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__half v) { return __half2float(v); }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }

}  // namespace

// Box of one direction: rows i0 .. i0 + 31 + WR, columns j0 - XO .. j0 + 31 + XO
// (XO = 16 bytes of elements, so that the box starts on a 16-byte boundary).
template <int WR, class ST, int CH>
struct TmaBox {
  static constexpr int XO = 16 / (int)sizeof(ST);
  static constexpr int BR = NF_T + WR;
  static constexpr int BC = NF_T + 2 * XO;
  static constexpr int ELEMS = BR * BC;
  static constexpr unsigned CHUNK_BYTES = (unsigned)(CH * ELEMS * sizeof(ST));   // one copy
  // a buffer's stride: a TMA destination in shared memory starts on a
  // 128-byte boundary
  static constexpr unsigned BUF_BYTES = (CHUNK_BYTES + 127u) & ~127u;
  static constexpr size_t SMEM = 2 * (size_t)BUF_BYTES + 128;   // + room to align the base
};

template <int WR, class ST, int CH>
__global__ void __launch_bounds__(NA_THREADS, 2)
k_nla2t(const Geom g, const TableArgs tb) {
  using D = HalfDirs<WR>;
  using BX = TmaBox<WR, ST, CH>;
  static_assert(BX::XO >= WR, "the box covers the backward neighbours' columns");
  constexpr int T = NF_T, NP = T + 2 * WR, NPp = NP | 1;
  constexpr int NCH = (D::SH + CH - 1) / CH;     // chunks of directions
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // two buffers of CH boxes of BR x BC, each on a 128-byte boundary
  unsigned char* sbase = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  __shared__ float sP[NP * NPp];
  __shared__ double s_red[NA_THREADS / 32];
  __shared__ __align__(8) unsigned long long s_bar[2];
  __shared__ int s_fail;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const JobArgs* jp = tb.jobs + table_job(tb, blockIdx.x);
  DevScalars* sc = jp->sc;
  const bool skip = tb.check_done && ((volatile int*)&sc->cg_done)[0];
  float psum = 0.f;
  if (!skip) {
    const int Hh = jp->Hh, Wh = jp->Wh;
    const int tile = blockIdx.x - jp->unit0;
    const int ty = tile / jp->tiles_x, tx = tile - ty * jp->tiles_x;
    const int i0 = ty * T, j0 = tx * T;
    const int TRr = min(T, Hh - i0), TRc = min(T, Wh - j0);
    const void* map = jp->wt_map;
    if (tid == 0) {
      mbar_init(&s_bar[0], 1);
      mbar_init(&s_bar[1], 1);
      // alignment the copies need (checked, never assumed): destination on a
      // 128-byte boundary, tensor map on a 64-byte boundary, x on 16 bytes
      s_fail = ((smem_u32(sbase) & 127u) != 0 || (reinterpret_cast<size_t>(map) & 63u) != 0 ||
                (((j0 - BX::XO) * (int)sizeof(ST)) & 15) != 0)
                   ? 1
                   : 0;
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const bool aligned = s_fail == 0;
    // chunk c into buffer c & 1 (thread 0); the last chunk's box may reach
    // past the last direction plane (read as zero, not used)
    auto issue = [&](int c) {
      unsigned long long* bar = &s_bar[c & 1];
      mbar_expect_tx(bar, BX::CHUNK_BYTES);
      tma_load_3d(sbase + (size_t)(c & 1) * BX::BUF_BYTES, map, j0 - BX::XO, i0, c * CH, bar);
    };
    if (tid == 0 && aligned) issue(0);
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
    const int ju = lane;
    const int iu0 = NA_PIX * warp;
    float acc[NA_PIX];
#pragma unroll
    for (int m = 0; m < NA_PIX; ++m) acc[m] = 0.f;
    int c_fail = aligned ? -1 : NCH;               // the chunk whose copy did not arrive
    for (int c = 0; c < NCH && aligned; ++c) {
      if (tid == 0 && c + 1 < NCH) {
        // buffer (c + 1) & 1 was read in step c - 1 (all threads passed the
        // barrier below since); order those generic-proxy reads before the
        // async-proxy write
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue(c + 1);
      }
      if (!mbar_wait_bounded(&s_bar[c & 1], (unsigned)((c >> 1) & 1), g)) s_fail = 1;
      __syncthreads();
      if (s_fail) {
        c_fail = c;
        break;
      }
      const ST* buf = reinterpret_cast<const ST*>(sbase + (size_t)(c & 1) * BX::BUF_BYTES);
#pragma unroll
      for (int e = 0; e < CH; ++e) {
        const int idx = c * CH + e;
        if (idx >= D::SH) break;
        const int di = D::di(idx), dj = D::dj(idx);
        const ST* wb = buf + (size_t)e * BX::ELEMS;
#pragma unroll
        for (int m = 0; m < NA_PIX; ++m) {
          const int r = iu0 + m;
          const float wfv = to_f(wb[r * BX::BC + ju + BX::XO]);
          const float wbv = to_f(wb[(r - di) * BX::BC + ju - dj + BX::XO]);
          const float* pu = sP + (r + WR) * NPp + (ju + WR);
          const float p0 = pu[0];
          const float df = p0 - pu[di * NPp + dj];
          const float db = p0 - pu[-di * NPp - dj];
          const float wf2 = wfv * wfv;
          acc[m] = fmaf(wf2, df, fmaf(wbv * wbv, db, acc[m]));
          psum = fmaf(wf2 * df, df, psum);
        }
      }
      __syncthreads();   // buffer c & 1 is free for chunk c + 2
    }
    if (c_fail >= 0) {
      // a copy did not arrive in time (or none was issued: an alignment the
      // copies need did not hold): record it and let the copies still in
      // flight (chunks c_fail and c_fail + 1) land, bounded again, before
      // the CTA's shared memory is released
      if (tid == 0) {
        set_status(sc, aligned ? -5 : -3);   // LFSR_ETIMEOUT, or LFSR_ECUDA for a misalignment
        for (int c = c_fail; c < NCH && c <= c_fail + 1; ++c)
          (void)mbar_wait_bounded(&s_bar[c & 1], (unsigned)((c >> 1) & 1), g);
      }
      psum = 0.f;
    } else {
#pragma unroll
      for (int m = 0; m < NA_PIX; ++m) {
        const int ui = i0 + iu0 + m, uj = j0 + ju;
        if (ui < Hh && uj < Wh) jp->out[(size_t)ui * Wh + uj] = g.mu * acc[m];
      }
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

namespace {

constexpr int NLA_TMA_CHUNK = 6;

template <int WR, class ST>
size_t tma_smem_bytes() {
  return TmaBox<WR, ST, NLA_TMA_CHUNK>::SMEM;
}

template <class ST>
cudaError_t nla2t_st(const Geom& g, const TableArgs& t, cudaStream_t s) {
  switch (g.win_r) {
#define NLA2T_CASE(wr)                                                                   \
  case wr: {                                                                             \
    const size_t smem = tma_smem_bytes<wr, ST>();                                        \
    k_nla2t<wr, ST, NLA_TMA_CHUNK><<<t.total_units, NA_THREADS, smem, s>>>(g, t);        \
    return cudaGetLastError();                                                           \
  }
    NLA2T_CASE(1)
    NLA2T_CASE(2)
    NLA2T_CASE(3)
#undef NLA2T_CASE
    default: return cudaErrorInvalidValue;
  }
}

template <class ST>
cudaError_t nla2t_prepare_st(int optin) {
  cudaError_t e = set_max_dynamic_smem(k_nla2t<1, ST, NLA_TMA_CHUNK>, optin);
  if (e == cudaSuccess) e = set_max_dynamic_smem(k_nla2t<2, ST, NLA_TMA_CHUNK>, optin);
  if (e == cudaSuccess) e = set_max_dynamic_smem(k_nla2t<3, ST, NLA_TMA_CHUNK>, optin);
  return e;
}

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                 const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                 const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn() {
  static EncodeTiled fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
  }
  return fn;
}

}  // namespace

bool nla2t_supported(const Geom& g) {
  const size_t es = storage_bytes(g.st);
  return nlf_supported(g) && ((size_t)g.Wh * es) % 16 == 0 && encode_fn() != nullptr;
}

cudaError_t nla2t_prepare(int optin) {
  cudaError_t e = nla2t_prepare_st<float>(optin);
  if (e == cudaSuccess) e = nla2t_prepare_st<__half>(optin);
  if (e == cudaSuccess) e = nla2t_prepare_st<__nv_bfloat16>(optin);
  return e;
}

cudaError_t nla2t_make_map(const Geom& g, const void* wt, void* map_out) {
  EncodeTiled fn = encode_fn();
  if (!fn || !nla2t_supported(g)) return cudaErrorNotSupported;
  const size_t es = storage_bytes(g.st);
  const CUtensorMapDataType dt = g.st == ST_F32   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                 : g.st == ST_F16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                  : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  const int xo = (int)(16 / es);
  const cuuint64_t dims[3] = {(cuuint64_t)g.Wh, (cuuint64_t)g.Hh, (cuuint64_t)g.sh};
  const cuuint64_t strides[2] = {(cuuint64_t)g.Wh * es, (cuuint64_t)g.Wh * g.Hh * es};
  const cuuint32_t box[3] = {(cuuint32_t)(NF_T + 2 * xo), (cuuint32_t)(NF_T + g.win_r),
                             (cuuint32_t)NLA_TMA_CHUNK};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUtensorMap m;
  const CUresult r =
      fn(&m, dt, 3, const_cast<void*>(wt), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
         CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  std::memcpy(map_out, &m, sizeof(m));
  return cudaSuccess;
}

cudaError_t nla2t_launch(const Geom& g, const TableArgs& t, cudaStream_t s) {
  if (t.total_units < 1) return cudaErrorInvalidValue;
  switch (g.st) {
    case ST_F32: return nla2t_st<float>(g, t, s);
    case ST_F16: return nla2t_st<__half>(g, t, s);
    case ST_BF16: return nla2t_st<__nv_bfloat16>(g, t, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace lfsr
