// Vector steps of the conjugate-gradient x-step (Algorithm 2): the
// initialisation r = -v, pi = <r, r> and the update x += alpha p,
// r -= alpha q, pi' = <r, r>, beta = pi'/pi.  Inner products accumulate in
// float64 and finish with a last-block reduction, so the scalars never leave
// the device.  Also the conversions between the canonical regulariser-dual
// layout [d][u] and the kernels' edge-pair layout, and between float and the
// storage type of the large streams.
#include <cfloat>

#include "cg_vec.cuh"

namespace lfsr {

// Table-driven: one CTA per chunk of HR pixels of one light field (unit
// blockIdx.x of the table); the inner products go to one slot per unit.

// x-step initialisation without stored NLTV terms: r = -v, x' = x, pi = <r, r>.
__global__ void __launch_bounds__(VEC_THREADS)
k_cg_init(const Geom g, const TableArgs tb) {
  __shared__ double s_red[VEC_THREADS / 32];
  const JobArgs* jp = tb.jobs + table_job(tb, blockIdx.x);
  const size_t n = (size_t)jp->Hh * jp->Wh;
  float* __restrict__ rv = jp->out;
  const float* __restrict__ x = jp->src;
  float* __restrict__ x_next = jp->x_next;
  const size_t c0 = (size_t)(blockIdx.x - jp->unit0) * jp->chunk;
  const size_t c1 = min(n, c0 + (size_t)jp->chunk);
  double part = 0.0;
  for (size_t i = c0 + threadIdx.x; i < c1; i += VEC_THREADS) {
    const float r = -rv[i];
    rv[i] = r;
    x_next[i] = x[i];
    part += (double)r * (double)r;
  }
  const double bs = block_sum<VEC_THREADS>(part, s_red);
  if (threadIdx.x == 0) tb.partials[blockIdx.x] = bs;
  if (table_arrive_last(tb.counter)) cg_init_finalize<VEC_THREADS>(g, tb);
}

// x-step initialisation from the accumulated v (the stored-weight NLTV
// block and the data block add into it): r = -v, v := 0 for the next
// iteration, x' = x, pi = <r, r>.
__global__ void __launch_bounds__(VEC_THREADS)
k_cg_init_acc(const Geom g, const TableArgs tb) {
  __shared__ double s_red[VEC_THREADS / 32];
  cg_init_acc_unit(tb, blockIdx.x, s_red);
  cg_init_finish(g, tb);
}

// CG update: x += alpha p, r -= alpha q, pi' = <r, r>, beta = pi' / pi.
__global__ void __launch_bounds__(VEC_THREADS)
k_cg_update(const Geom g, const TableArgs tb) {
  __shared__ double s_red[VEC_THREADS / 32];
  cg_update_unit(tb, blockIdx.x, s_red);
  cg_update_finish(g, tb);
}

cudaError_t cg_init_launch(const Geom& g, const TableArgs& t, cudaStream_t s) {
  if (t.total_units < 1) return cudaErrorInvalidValue;
  k_cg_init<<<t.total_units, VEC_THREADS, 0, s>>>(g, t);
  return cudaGetLastError();
}

cudaError_t cg_init_acc_launch(const Geom& g, const TableArgs& t, cudaStream_t s) {
  if (t.total_units < 1) return cudaErrorInvalidValue;
  k_cg_init_acc<<<t.total_units, VEC_THREADS, 0, s>>>(g, t);
  return cudaGetLastError();
}

cudaError_t cg_update_launch(const Geom& g, const TableArgs& t, cudaStream_t s) {
  if (t.total_units < 1) return cudaErrorInvalidValue;
  k_cg_update<<<t.total_units, VEC_THREADS, 0, s>>>(g, t);
  return cudaGetLastError();
}

// canonical [d][u] (d over the full window minus the centre, raster order)
// <-> pair layout [idx][0][u] = dual of d_idx at u,
//                 [idx][1][u] = dual of -d_idx at u + d_idx   (idx < s_d/2)
template <class ST>
__global__ void k_pair_from_canonical(const Geom g, const float* __restrict__ can,
                                      ST* __restrict__ pair) {
  const size_t p = (size_t)g.Hh * g.Wh;
  const int sd = 2 * g.sh;
  const size_t total = (size_t)g.sh * p;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int idx = (int)(t / p);
    const size_t u = t - (size_t)idx * p;
    const int ui = (int)(u / g.Wh), uj = (int)(u - (size_t)ui * g.Wh);
    const int vi = ui + g.di[idx], vj = uj + g.dj[idx];
    st_s(pair + (size_t)(2 * idx) * p + u, can[(size_t)idx * p + u]);
    float b = 0.f;
    if (vi >= 0 && vi < g.Hh && vj >= 0 && vj < g.Wh)
      b = can[(size_t)(sd - 1 - idx) * p + (size_t)vi * g.Wh + vj];
    st_s(pair + (size_t)(2 * idx + 1) * p + u, b);
  }
}

template <class ST>
__global__ void k_pair_to_canonical(const Geom g, const ST* __restrict__ pair,
                                    float* __restrict__ can) {
  const size_t p = (size_t)g.Hh * g.Wh;
  const int sd = 2 * g.sh;
  const size_t total = (size_t)sd * p;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int d = (int)(t / p);
    const size_t u = t - (size_t)d * p;
    float val = 0.f;
    if (d < g.sh) {
      val = ld_s(pair + (size_t)(2 * d) * p + u);
    } else {
      // direction -d_idx at u is the second dual of edge (u - d_idx, u)
      const int idx = sd - 1 - d;
      const int ui = (int)(u / g.Wh), uj = (int)(u - (size_t)ui * g.Wh);
      const int vi = ui - g.di[idx], vj = uj - g.dj[idx];
      if (vi >= 0 && vi < g.Hh && vj >= 0 && vj < g.Wh)
        val = ld_s(pair + (size_t)(2 * idx + 1) * p + (size_t)vi * g.Wh + vj);
    }
    can[t] = val;
  }
}

cudaError_t pair_from_canonical(const Geom& g, const float* can, void* pair, cudaStream_t s) {
  switch (g.st) {
    case ST_F32: k_pair_from_canonical<<<1024, 256, 0, s>>>(g, can, (float*)pair); break;
    case ST_F16: k_pair_from_canonical<<<1024, 256, 0, s>>>(g, can, (__half*)pair); break;
    case ST_BF16: k_pair_from_canonical<<<1024, 256, 0, s>>>(g, can, (__nv_bfloat16*)pair); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t pair_to_canonical(const Geom& g, const void* pair, float* can, cudaStream_t s) {
  switch (g.st) {
    case ST_F32: k_pair_to_canonical<<<1024, 256, 0, s>>>(g, (const float*)pair, can); break;
    case ST_F16: k_pair_to_canonical<<<1024, 256, 0, s>>>(g, (const __half*)pair, can); break;
    case ST_BF16:
      k_pair_to_canonical<<<1024, 256, 0, s>>>(g, (const __nv_bfloat16*)pair, can);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// Float -> storage kind with a range check: the largest finite value of
// the kind (65504 for half; float's own range for bfloat16).  A value
// outside it, or not finite, raises the sticky status and is stored
// saturated (NaN as 0), so no infinity or NaN enters the solver state.
template <class ST>
__global__ void __launch_bounds__(VEC_THREADS)
k_to_storage(const float* __restrict__ src, ST* __restrict__ dst, size_t n, float vmax,
             DevScalars* sc) {
  bool bad = false;
  for (size_t i = (size_t)blockIdx.x * VEC_THREADS + threadIdx.x; i < n;
       i += (size_t)gridDim.x * VEC_THREADS) {
    float v = src[i];
    if (!(fabsf(v) <= vmax)) {
      bad = true;
      v = (v != v) ? 0.f : copysignf(vmax, v);
    }
    st_s(dst + i, v);
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) set_status(sc, -1);  // LFSR_EINVAL
}

template <class ST>
__global__ void __launch_bounds__(VEC_THREADS)
k_from_storage(const ST* __restrict__ src, float* __restrict__ dst, size_t n) {
  for (size_t i = (size_t)blockIdx.x * VEC_THREADS + threadIdx.x; i < n;
       i += (size_t)gridDim.x * VEC_THREADS)
    dst[i] = ld_s(src + i);
}

cudaError_t to_storage(int st, const float* src, void* dst, size_t n, DevScalars* sc, int grid,
                       cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  switch (st) {
    case ST_F32:
      k_to_storage<<<grid, VEC_THREADS, 0, s>>>(src, (float*)dst, n, FLT_MAX, sc);
      break;
    case ST_F16:
      k_to_storage<<<grid, VEC_THREADS, 0, s>>>(src, (__half*)dst, n, 65504.f, sc);
      break;
    case ST_BF16:
      // the largest finite bfloat16 (0x7f7f); larger floats would round to infinity
      k_to_storage<<<grid, VEC_THREADS, 0, s>>>(src, (__nv_bfloat16*)dst, n,
                                                3.3895313892515355e38f, sc);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t from_storage(int st, const void* src, float* dst, size_t n, int grid, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  switch (st) {
    case ST_F32: k_from_storage<<<grid, VEC_THREADS, 0, s>>>((const float*)src, dst, n); break;
    case ST_F16: k_from_storage<<<grid, VEC_THREADS, 0, s>>>((const __half*)src, dst, n); break;
    case ST_BF16:
      k_from_storage<<<grid, VEC_THREADS, 0, s>>>((const __nv_bfloat16*)src, dst, n);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t scalars_reset(DevScalars* sc, cudaStream_t s) {
  return cudaMemsetAsync(sc, 0, sizeof(DevScalars), s);
}

}  // namespace lfsr
