// Table variants of the specialised operator kernel for tile side 32
// (see op_fast_batch.cuh).
#include "op_fast_batch.cuh"

namespace lfsr {

#define LFSR_X_PREP(z, k) \
  if (zeta == z && kb == k) return table_prepare_zkt<z, k, 32>(optin);
#define LFSR_X_PLAN(z, k) \
  if (g.zeta == z && g.kb == k) return table_plan_zkt<z, k, 32>(g, P, smem_limit);
#define LFSR_X_LAUNCH(z, k) \
  if (g.zeta == z && g.kb == k) return table_launch_zkt<z, k, 32>(mode, g, P, t, grid, s);
LFSR_TABLE_TILE_DEFS(32)
#undef LFSR_X_PREP
#undef LFSR_X_PLAN
#undef LFSR_X_LAUNCH

}  // namespace lfsr
