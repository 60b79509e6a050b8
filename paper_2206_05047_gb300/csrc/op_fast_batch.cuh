// Table (batch) variants of the specialised operator kernel (op_fast.cuh):
// the data block and the normal-matrix product over the (tile, view pair)
// units of every light field of a job table, per tile side.  Each tile side
// is instantiated in its own translation unit (op_fast_batch.cu: 64,
// op_fast_batch32.cu: 32) so the two compile in parallel.
#pragma once

#include "op_fast.cuh"

namespace lfsr {

template <int Z, int KB, int TILE>
inline cudaError_t table_prepare_zkt(int optin) {
  cudaError_t e = set_max_dynamic_smem(k_operator_fast<OP_NORMAL, Z, KB, false, TILE>, optin);
  if (e == cudaSuccess) e = set_max_dynamic_smem(k_operator_fast<OP_DATA, Z, KB, false, TILE>, optin);
  return e;
}

template <int Z, int KB, int TILE>
inline cudaError_t table_launch_zkt(int mode, const Geom& g, const OpPlan& P, const TableArgs& t,
                                    int grid, cudaStream_t s) {
  const JobArgs none{};
  switch (mode) {
    case OP_NORMAL:
      k_operator_fast<OP_NORMAL, Z, KB, false, TILE>
          <<<grid, FT_THREADS, P.smem_bytes, s>>>(g, P, t, none);
      break;
    case OP_DATA:
      k_operator_fast<OP_DATA, Z, KB, false, TILE>
          <<<grid, FT_THREADS, P.smem_bytes, s>>>(g, P, t, none);
      break;
    default: return cudaErrorInvalidValue;   // the standalone operators run one light field
  }
  return cudaGetLastError();
}

template <int Z, int KB, int TILE>
inline cudaError_t table_plan_zkt(const Geom& g, OpPlan* P, int smem_limit) {
  if (fast_layout<Z, KB, TILE>(g, P, true) > (size_t)smem_limit &&
      fast_layout<Z, KB, TILE>(g, P, false) > (size_t)smem_limit)
    return cudaErrorInvalidValue;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &n, k_operator_fast<OP_NORMAL, Z, KB, false, TILE>, FT_THREADS, P->smem_bytes) !=
      cudaSuccess)
    n = 1;
  P->ctas_per_sm = n > 0 ? n : 1;
  P->fast = 1;
  return cudaSuccess;
}

// per-tile-side entry points (defined in the tile's translation unit)
#define LFSR_TABLE_TILE_DECL(T)                                                               \
  cudaError_t table_prepare_t##T(int zeta, int kb, int optin);                                \
  cudaError_t table_plan_t##T(const Geom& g, OpPlan* P, int smem_limit);                      \
  cudaError_t table_launch_t##T(int mode, const Geom& g, const OpPlan& P, const TableArgs& t, \
                                int grid, cudaStream_t s);
LFSR_TABLE_TILE_DECL(64)
LFSR_TABLE_TILE_DECL(32)
#undef LFSR_TABLE_TILE_DECL

// The definitions of one tile side's entry points (used once per tile).
#define LFSR_TABLE_TILE_DEFS(T)                                                               \
  cudaError_t table_prepare_t##T(int zeta, int kb, int optin) {                               \
    LFSR_FAST_CASES(LFSR_X_PREP)                                                              \
    return cudaErrorInvalidValue;                                                             \
  }                                                                                           \
  cudaError_t table_plan_t##T(const Geom& g, OpPlan* P, int smem_limit) {                     \
    LFSR_FAST_CASES(LFSR_X_PLAN)                                                              \
    return cudaErrorInvalidValue;                                                             \
  }                                                                                           \
  cudaError_t table_launch_t##T(int mode, const Geom& g, const OpPlan& P, const TableArgs& t, \
                                int grid, cudaStream_t s) {                                   \
    LFSR_FAST_CASES(LFSR_X_LAUNCH)                                                            \
    return cudaErrorInvalidValue;                                                             \
  }

}  // namespace lfsr
