// Table variants of the specialised operator kernel for tile side 64
// (see op_fast_batch.cuh).
#include "op_fast_batch.cuh"

namespace lfsr {

#define LFSR_X_PREP(z, k) \
  if (zeta == z && kb == k) return table_prepare_zkt<z, k, 64>(optin);
#define LFSR_X_PLAN(z, k) \
  if (g.zeta == z && g.kb == k) return table_plan_zkt<z, k, 64>(g, P, smem_limit);
#define LFSR_X_LAUNCH(z, k) \
  if (g.zeta == z && g.kb == k) return table_launch_zkt<z, k, 64>(mode, g, P, t, grid, s);
LFSR_TABLE_TILE_DEFS(64)
#undef LFSR_X_PREP
#undef LFSR_X_PLAN
#undef LFSR_X_LAUNCH

// Dispatch on the tile side of the plan (the autotuner's choice).
cudaError_t fast_prepare_table(int zeta, int kb, int optin) {
  cudaError_t e = table_prepare_t64(zeta, kb, optin);
  return e == cudaSuccess ? table_prepare_t32(zeta, kb, optin) : e;
}

cudaError_t fast_plan_table(const Geom& g, OpPlan* P, int smem_limit, int tile) {
  if (tile == 64) return table_plan_t64(g, P, smem_limit);
  if (tile == 32) return table_plan_t32(g, P, smem_limit);
  return cudaErrorInvalidValue;
}

cudaError_t fast_launch_table(int mode, const Geom& g, const OpPlan& P, const TableArgs& t, int grid,
                              cudaStream_t s) {
  if (P.TH == 64) return table_launch_t64(mode, g, P, t, grid, s);
  if (P.TH == 32) return table_launch_t32(mode, g, P, t, grid, s);
  return cudaErrorInvalidValue;
}

}  // namespace lfsr
