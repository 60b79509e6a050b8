// Device helpers shared by the kernel translation units of liblfsr.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "lfsr_internal.cuh"

namespace lfsr {

// Element access of the streams kept in the storage type (LR views, data
// and regulariser duals, stored NLTV weights): loads widen to float, stores
// round to nearest even.  Arithmetic stays float.  The 16-bit loads are
// plain (compiler-visible) unsigned-short loads, so they can be predicated
// and batched like float loads; widening to float is exact for both types.
__device__ __forceinline__ float ld_s(const float* p) { return __ldg(p); }
__device__ __forceinline__ float ld_s(const __half* p) {
  return __half2float(__ushort_as_half(__ldg(reinterpret_cast<const unsigned short*>(p))));
}
__device__ __forceinline__ float ld_s(const __nv_bfloat16* p) {
  return __bfloat162float(__ushort_as_bfloat16(__ldg(reinterpret_cast<const unsigned short*>(p))));
}
__device__ __forceinline__ void st_s(float* p, float v) { *p = v; }
__device__ __forceinline__ void st_s(__half* p, float v) {
  *reinterpret_cast<unsigned short*>(p) = __half_as_ushort(__float2half_rn(v));
}
__device__ __forceinline__ void st_s(__nv_bfloat16* p, float v) {
  *reinterpret_cast<unsigned short*>(p) = __bfloat16_as_ushort(__float2bfloat16_rn(v));
}

// Split load / widen for latency hiding: a kernel issues all raw loads of a
// batch (predicated, 0 when masked) and widens each value only where it is
// used, so no conversion waits on a load that the batch could overlap.
template <class ST> struct SBits;
template <> struct SBits<float> {
  using R = float;
  static __device__ __forceinline__ R ld(const float* p) { return __ldg(p); }
  static __device__ __forceinline__ float f(R r) { return r; }
};
template <> struct SBits<__half> {
  using R = unsigned short;
  static __device__ __forceinline__ R ld(const __half* p) {
    return __ldg(reinterpret_cast<const unsigned short*>(p));
  }
  static __device__ __forceinline__ float f(R r) { return __half2float(__ushort_as_half(r)); }
};
template <> struct SBits<__nv_bfloat16> {
  using R = unsigned short;
  static __device__ __forceinline__ R ld(const __nv_bfloat16* p) {
    return __ldg(reinterpret_cast<const unsigned short*>(p));
  }
  static __device__ __forceinline__ float f(R r) { return __bfloat162float(__ushort_as_bfloat16(r)); }
};

// Run-time storage kind: raw 32-bit word (float bits or a zero-extended
// 16-bit value) and its widening, for the per-LR-pixel accesses of the
// operator kernels (warp-uniform kind).
__device__ __forceinline__ unsigned int ld_raw_kind(const void* base, size_t i, int st) {
  if (st == ST_F32) return __ldg(reinterpret_cast<const unsigned int*>(base) + i);
  return __ldg(reinterpret_cast<const unsigned short*>(base) + i);
}
__device__ __forceinline__ float raw_to_float(unsigned int r, int st) {
  if (st == ST_F16) return __half2float(__ushort_as_half((unsigned short)r));
  if (st == ST_BF16) return __bfloat162float(__ushort_as_bfloat16((unsigned short)r));
  return __uint_as_float(r);
}

// The same with the storage kind (ST_*) known only at run time; for the
// few per-LR-pixel accesses of the operator kernels (warp-uniform branch).
__device__ __forceinline__ float ld_kind(const void* base, size_t i, int st) {
  if (st == ST_F16) return ld_s((const __half*)base + i);
  if (st == ST_BF16) return ld_s((const __nv_bfloat16*)base + i);
  return ld_s((const float*)base + i);
}
__device__ __forceinline__ void st_kind(void* base, size_t i, int st, float v) {
  if (st == ST_F16) st_s((__half*)base + i, v);
  else if (st == ST_BF16) st_s((__nv_bfloat16*)base + i, v);
  else st_s((float*)base + i, v);
}

// Sticky device status: the first error recorded stays.
__device__ __forceinline__ void set_status(DevScalars* sc, int code) {
  atomicCAS(&sc->status, 0, code);
}

// CG step length (Algorithm 2): alpha = pi / <p, M p>.  A curvature of
// exactly 0 means the direction has vanished below float resolution (the
// x-step has converged, e.g. a problem of one unknown after its first step)
// or lies where M is singular: the x-step stops there.  A negative or
// non-finite curvature is a numeric failure (LFSR_ENUMERIC).
__device__ __forceinline__ void cg_set_alpha(DevScalars* sc, double pAp) {
  sc->pAp = pAp;
  if (pAp > 0.0 && isfinite(pAp)) {
    sc->alpha = sc->pi / pAp;
    return;
  }
  sc->alpha = 0.0;
  sc->cg_done = 1;
  if (!(pAp == 0.0)) set_status(sc, -4);  // LFSR_ENUMERIC
}

// Floor / ceil division for a possibly negative numerator and positive d.
__host__ __device__ __forceinline__ int floor_div(int n, int d) {
  return (n >= 0) ? (n / d) : -((-n + d - 1) / d);
}
__host__ __device__ __forceinline__ int ceil_div(int n, int d) {
  return (n >= 0) ? ((n + d - 1) / d) : -((-n) / d);
}
__host__ __device__ __forceinline__ int clampi(int v, int lo, int hi) {
  return v < lo ? lo : (v > hi ? hi : v);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the block in a fixed order (result valid in thread 0).  Every
// thread of the block must call it.
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* red /* >= NT/32 */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (warp == 0) {
    t = (lane < NT / 32) ? red[lane] : 0.0;
    t = warp_sum(t);
  }
  return t;
}

// Grid reduction without a second launch: each CTA stores its partial in
// partials[blockIdx.x]; the CTA that arrives last sums all partials in
// index order (deterministic for a given grid) and returns true with the
// total in *total (valid in thread 0).  The counter is re-armed for the
// next launch.
template <int NT>
__device__ __forceinline__ bool grid_sum_last(double part, double* partials, unsigned int* counter,
                                              double* total) {
  __shared__ double red[NT / 32];
  __shared__ int am_last;
  double s = block_sum<NT>(part, red);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = s;
    __threadfence();
    const unsigned int t = atomicAdd(counter, 1u);
    am_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!am_last) return false;
  __threadfence();
  double acc = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += NT) acc += ((volatile double*)partials)[i];
  acc = block_sum<NT>(acc, red);
  if (threadIdx.x == 0) {
    *total = acc;
    *counter = 0u;
  }
  return true;
}

// Reductions of the table-driven kernels.  Every CTA writes its partial
// slot(s) and then arrives here; the CTA that arrives last gets true and may
// then read every slot (fenced).  The counter is re-armed for the next launch.
__device__ __forceinline__ bool table_arrive_last(unsigned int* counter) {
  __shared__ int am_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int t = atomicAdd(counter, 1u);
    am_last = (t == gridDim.x - 1);
    if (am_last) *counter = 0u;   // every CTA has arrived
  }
  __syncthreads();
  if (!am_last) return false;
  __threadfence();
  return true;
}

// Sum of n slots by one warp in a fixed order; the total in every lane.
__device__ __forceinline__ double warp_sum_slots(const double* slots, int n) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int i = lane; i < n; i += 32) s += ((const volatile double*)slots)[i];
  s = warp_sum(s);
  return __shfl_sync(0xffffffffu, s, 0);
}

// x-step initialisation totals (Algorithm 2), per light field of the table:
// pi = <r, r> from the unit slots and a fresh CG state.  Run by the last CTA.
template <int NT>
__device__ __forceinline__ void cg_init_finalize(const Geom& g, const TableArgs& tb) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int j = warp; j < tb.n_jobs; j += NT / 32) {
    const JobArgs* jj = tb.jobs + j;
    const double total = warp_sum_slots(tb.partials + jj->unit0, jj->units);
    if (lane == 0) {
      DevScalars* sc = jj->sc;
      sc->pi = total;
      sc->cg_first = 1;
      sc->cg_steps = 0;
      sc->beta = 0.0;
      sc->dw2 = sc->dwA + sc->dwS;
      if (!isfinite(total)) set_status(sc, -4);  // LFSR_ENUMERIC
      sc->cg_done = (total > g.tau && isfinite(total)) ? 0 : 1;
    }
  }
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier of a launch whose CTAs are all resident (a cooperative
// launch of at most the co-resident CTA count).  *arrivals counts every
// CTA's arrival at every barrier, monotonically across the launches that
// share it (all with the same grid size; reset to 0 when a solve loads):
// the CTA that arrives as number a waits until the count reaches the end of
// its generation, G (a / G + 1).  The wait is bounded: after g.wait_ns of
// %globaltimer it gives up and returns false (the caller records
// LFSR_ETIMEOUT).  The arrival is counted either way, so the barriers after
// a failed one keep their alignment.  Every thread of the CTA must call it;
// the result is block-uniform.  Memory: the writes of every CTA before the
// barrier are visible to every CTA after it (fences on both sides).
__device__ __forceinline__ bool grid_barrier(unsigned long long* arrivals, const Geom& g) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned long long G = gridDim.x;
    const unsigned long long a = atomicAdd(arrivals, 1ull);
    const unsigned long long target = (a / G + 1ull) * G + (g.wait_unreachable ? 1ull : 0ull);
    const unsigned long long t0 = global_ns();
    int ok = 1;
    while (ld_acquire_u64(arrivals) < target) {
      if (global_ns() - t0 >= g.wait_ns) {
        ok = 0;
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Table entry of work unit u.
__device__ __forceinline__ int table_job(const TableArgs& t, int u) {
  return t.unit_job ? __ldg(t.unit_job + u) : 0;
}

}  // namespace lfsr
