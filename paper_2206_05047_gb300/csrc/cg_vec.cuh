// Vector steps of the CG x-step (Algorithm 2) over table work units (chunks
// of HR pixels of one light field): the initialisation from the accumulated
// v and the update.  Each *_unit runs one chunk (every thread of a
// VEC_THREADS CTA calls it) and stores its partial of pi in
// partials[unit]; each *_finish is called once per CTA after its last
// chunk, and the CTA that arrives last finishes every light field's
// scalars from its slots in a fixed order.  The kernels in vec_kernels.cu
// run one chunk per CTA; the persistent batch iteration loops over them.
#pragma once

#include "lfsr_device.cuh"

namespace lfsr {

// r = -v, v := 0 for the next iteration, x' = x, partial of pi = <r, r>.
__device__ __forceinline__ void cg_init_acc_unit(const TableArgs& tb, int unit, double* s_red) {
  const JobArgs* jp = tb.jobs + table_job(tb, unit);
  const int n = jp->Hh * jp->Wh;              // p < 2^31: 32-bit offsets
  float* __restrict__ va = jp->vacc;
  float* __restrict__ rv = jp->out;
  const float* __restrict__ x = jp->src;
  float* __restrict__ x_next = jp->x_next;
  const int c0 = (unit - jp->unit0) * jp->chunk;
  const int c1 = min(n, c0 + jp->chunk);
  double part = 0.0;
  // chunks are whole multiples of 32 floats and every buffer starts on a
  // 256-byte boundary: [c0, c1 & ~3) in float4 steps, then the tail
  const int v0 = c0 >> 2, v1 = c1 >> 2;
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int v = v0 + (int)threadIdx.x; v < v1; v += VEC_THREADS) {
    const float4 a4 = reinterpret_cast<const float4*>(va)[v];
    reinterpret_cast<float4*>(va)[v] = z4;
    const float4 r4 = make_float4(-a4.x, -a4.y, -a4.z, -a4.w);
    reinterpret_cast<float4*>(rv)[v] = r4;
    reinterpret_cast<float4*>(x_next)[v] = __ldg(reinterpret_cast<const float4*>(x) + v);
    part += (double)r4.x * (double)r4.x;
    part += (double)r4.y * (double)r4.y;
    part += (double)r4.z * (double)r4.z;
    part += (double)r4.w * (double)r4.w;
  }
  for (int i = 4 * v1 + (int)threadIdx.x; i < c1; i += VEC_THREADS) {
    const float r = -va[i];
    va[i] = 0.f;
    rv[i] = r;
    x_next[i] = x[i];
    part += (double)r * (double)r;
  }
  const double bs = block_sum<VEC_THREADS>(part, s_red);
  if (threadIdx.x == 0) tb.partials[unit] = bs;
}

__device__ __forceinline__ void cg_init_finish(const Geom& g, const TableArgs& tb) {
  if (table_arrive_last(tb.counter)) cg_init_finalize<VEC_THREADS>(g, tb);
}

// x' += alpha p, r -= alpha q, partial of pi' = <r, r> (light fields whose
// x-step has finished are skipped).
__device__ __forceinline__ void cg_update_unit(const TableArgs& tb, int unit, double* s_red) {
  const JobArgs* jp = tb.jobs + table_job(tb, unit);
  DevScalars* sc = jp->sc;
  double part = 0.0;
  if (!((volatile int*)&sc->cg_done)[0]) {
    const int n = jp->Hh * jp->Wh;            // p < 2^31: 32-bit offsets
    const float* __restrict__ p = jp->p_old;
    const float* __restrict__ q = jp->q;
    float* __restrict__ r = jp->rr;
    float* __restrict__ x_next = jp->x_next;
    const float alpha = (float)sc->alpha;
    const int c0 = (unit - jp->unit0) * jp->chunk;
    const int c1 = min(n, c0 + jp->chunk);
    // chunks are whole multiples of 32 floats and every buffer starts on a
    // 256-byte boundary: [c0, c1 & ~3) in float4 steps, then the tail
    const int v0 = c0 >> 2, v1 = c1 >> 2;
    for (int v = v0 + (int)threadIdx.x; v < v1; v += VEC_THREADS) {
      const float4 pv = __ldg(reinterpret_cast<const float4*>(p) + v);
      const float4 qv = __ldg(reinterpret_cast<const float4*>(q) + v);
      float4 rv = reinterpret_cast<const float4*>(r)[v];
      float4 xv = reinterpret_cast<const float4*>(x_next)[v];
      xv.x = fmaf(alpha, pv.x, xv.x);
      xv.y = fmaf(alpha, pv.y, xv.y);
      xv.z = fmaf(alpha, pv.z, xv.z);
      xv.w = fmaf(alpha, pv.w, xv.w);
      rv.x = fmaf(-alpha, qv.x, rv.x);
      rv.y = fmaf(-alpha, qv.y, rv.y);
      rv.z = fmaf(-alpha, qv.z, rv.z);
      rv.w = fmaf(-alpha, qv.w, rv.w);
      reinterpret_cast<float4*>(x_next)[v] = xv;
      reinterpret_cast<float4*>(r)[v] = rv;
      part += (double)rv.x * (double)rv.x;
      part += (double)rv.y * (double)rv.y;
      part += (double)rv.z * (double)rv.z;
      part += (double)rv.w * (double)rv.w;
    }
    for (int i = 4 * v1 + (int)threadIdx.x; i < c1; i += VEC_THREADS) {
      x_next[i] = fmaf(alpha, p[i], x_next[i]);
      const float rn = fmaf(-alpha, q[i], r[i]);
      r[i] = rn;
      part += (double)rn * (double)rn;
    }
  }
  const double bs = block_sum<VEC_THREADS>(part, s_red);
  if (threadIdx.x == 0) tb.partials[unit] = bs;
}

// pi' and beta = pi' / pi per light field; the step count and the tau test.
__device__ __forceinline__ void cg_update_finish(const Geom& g, const TableArgs& tb) {
  if (!table_arrive_last(tb.counter)) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int j = warp; j < tb.n_jobs; j += VEC_THREADS / 32) {
    const JobArgs* jj = tb.jobs + j;
    DevScalars* s = jj->sc;
    if (((volatile int*)&s->cg_done)[0]) continue;
    const double total = warp_sum_slots(tb.partials + jj->unit0, jj->units);
    if (lane == 0) {
      const double pi_old = s->pi;
      s->beta = total / pi_old;
      s->pi = total;
      s->cg_first = 0;
      s->cg_steps += 1;
      if (!isfinite(total)) set_status(s, -4);  // LFSR_ENUMERIC
      if (!(total > g.tau) || !isfinite(total)) s->cg_done = 1;
    }
  }
}

}  // namespace lfsr
