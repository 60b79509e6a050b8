// The persistent batch iteration: one cooperative launch per ADMM iteration
// (Algorithm 1, with the K CG steps of Algorithm 2) for every light field
// of a batch.  Each phase runs the same work units as its per-phase launch
// -- 32 x 32 NLTV tiles, (64 x 64 tile, view pair) operator units of each
// group, chunks of HR pixels -- through the same device bodies, looped over
// the resident CTAs; a grid barrier separates phases that depend on each
// other, and the per-light-field reductions finish as in the per-phase
// kernels (the CTA that arrives last sums the slots in a fixed order).
//
// Every barrier wait is bounded (g.wait_ns of %globaltimer).  A CTA whose
// wait runs out records LFSR_ETIMEOUT in every light field's status and
// skips the rest of the iteration's work, but still arrives at each later
// barrier and reduction of the launch, so the arrival counters stay aligned
// for the next launch; the light fields must then be loaded again.
#pragma once

#include "cg_vec.cuh"
#include "nltv_fast.cuh"
#include "op_fast.cuh"

namespace lfsr {

// Counts this CTA's arrival at a grid barrier without waiting.
__device__ __forceinline__ void grid_arrive(unsigned long long* arrivals) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(arrivals, 1ull);
  }
  __syncthreads();
}

// One operator phase of group slot (Z, KB): the table variant of the
// specialised kernel's body over the group's units (run == false: none).
template <int MODE, int Z, int KB>
__device__ __forceinline__ void persist_op(const Geom& gg, const OpPlan& P, const TableArgs& t,
                                           bool run) {
  const JobArgs none{};
  op_fast_body<MODE, Z, KB, false, FAST_TILE>(gg, P, t, none, run);
}

// g: the batch's solver constants (NLTV and vector phases, barrier limit);
// g0, g1: the constants of operator group slots 0 and 1 (Z1 == 0: one group,
// g1 unused).  a: this iteration parity's arguments (device memory).
template <class ST, int WR, int PR, int Z0, int KB0, int Z1, int KB1>
__global__ void __launch_bounds__(FT_THREADS, 1)
k_batch_iter(const Geom g, const Geom g0, const Geom g1, const PersistArgs* __restrict__ a,
             unsigned long long* bar) {
  static_assert(NF_THREADS == FT_THREADS && NA_THREADS == FT_THREADS &&
                    VEC_THREADS == FT_THREADS,
                "every phase body runs on the same 512-thread CTA");
  extern __shared__ __align__(16) float smem[];
  __shared__ double s_red[FT_THREADS / 32];
  bool ok = true;   // block-uniform: no barrier of this launch has run out in this CTA
  auto sync = [&]() {
    if (ok) {
      ok = grid_barrier(bar, g);
      if (!ok && threadIdx.x == 0)
        for (int j = 0; j < a->nlw.n_jobs; ++j) set_status(a->nlw.jobs[j].sc, -5);  // LFSR_ETIMEOUT
    } else {
      grid_arrive(bar);
    }
  };

  // z/w-step of the regulariser rows: edge weights from x^(n-1), the duals,
  // the divergence into each light field's accumulated v
  if (ok)
    for (int u = blockIdx.x; u < a->nlw.total_units; u += gridDim.x)
      nlw2_unit<NLW_BLOCK, WR, PR, ST>(g, a->nlw, u, smem, smem + a->sx_off, s_red);
  nlw2_finish(a->nlw);
  // no barrier: the data rows read none of what the regulariser block
  // writes (both only add into v, with atomics, and use their own reduction
  // slots and counters); the initialisation below waits for both
  // data rows of each operator group: A_k x - y_k, prox, duals, v += A_k^T (...)
  persist_op<OP_DATA, Z0, KB0>(g0, a->P[0], a->data[0], ok);
  if constexpr (Z1 != 0) {
    sync();   // the groups share the reduction slots of the launch kind
    persist_op<OP_DATA, Z1, KB1>(g1, a->P[1], a->data[1], ok);
  }
  sync();
  // x-step initialisation: r = -v, v := 0, x' = x, pi
  if (ok)
    for (int u = blockIdx.x; u < a->init.total_units; u += gridDim.x)
      cg_init_acc_unit(a->init, u, s_red);
  cg_init_finish(g, a->init);
  sync();
  for (int k = 0; k < a->cg_iters; ++k) {
    const int pb = k & 1;
    // p = r + beta p, q = mu S^T W^2 S p and its part of <p, M p>
    const TableArgs& nla = a->nla[pb];
    if (ok)
      for (int u = blockIdx.x; u < nla.total_units; u += gridDim.x)
        nla2_unit<WR, ST, NLA_CHUNK>(g, nla, u, smem, s_red);
    nla2_finish(nla);
    sync();
    // q += cA sum_k A_k^T A_k p per group; alpha
    persist_op<OP_NORMAL, Z0, KB0>(g0, a->P[0], a->norm[pb][0], ok);
    if constexpr (Z1 != 0) {
      sync();
      persist_op<OP_NORMAL, Z1, KB1>(g1, a->P[1], a->norm[pb][1], ok);
    }
    sync();
    // x' += alpha p, r -= alpha q, pi', beta
    const TableArgs& upd = a->upd[pb];
    if (ok)
      for (int u = blockIdx.x; u < upd.total_units; u += gridDim.x)
        cg_update_unit(upd, u, s_red);
    cg_update_finish(g, upd);
    if (k + 1 < a->cg_iters) sync();
  }
}

}  // namespace lfsr
