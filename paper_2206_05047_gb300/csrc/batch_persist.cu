// Host side of the persistent batch iteration (batch_persist.cuh): which
// compiled instances exist, their shared memory, occupancy and the
// cooperative launch.  The float-storage instances are compiled here, the
// half-storage ones in batch_persist_h.cu (the two compile in parallel).
#include "batch_persist.cuh"

namespace lfsr {

using PersistKernel = void (*)(const Geom, const Geom, const Geom, const PersistArgs*,
                               unsigned long long*);

// The compiled instances: NLTV window / patch radius and the (scale, kb) of
// the group slots -- the light-field workloads' combinations.
#define LFSR_PERSIST_CASES(X, ST) \
  X(ST, 2, 1, 2, 5, 0, 0)         \
  X(ST, 3, 1, 2, 7, 0, 0)         \
  X(ST, 3, 1, 3, 9, 0, 0)         \
  X(ST, 3, 1, 2, 7, 3, 9)

#define LFSR_PERSIST_PICK(ST, wr, pr, z0, k0, z1, k1)                          \
  if (WR == wr && PR == pr && Z0 == z0 && K0 == k0 && Z1 == z1 && K1 == k1) \
    return k_batch_iter<ST, wr, pr, z0, k0, z1, k1>;

PersistKernel persist_kernel_f32(int WR, int PR, int Z0, int K0, int Z1, int K1) {
  LFSR_PERSIST_CASES(LFSR_PERSIST_PICK, float)
  return nullptr;
}
PersistKernel persist_kernel_f16(int WR, int PR, int Z0, int K0, int Z1, int K1);

namespace {

// Slot order of the groups for the compiled instances: one group, or the
// (2, 7) group then the (3, 9) group.
bool slot_order(const Geom* gg, int n, int* order) {
  if (n == 1) {
    order[0] = 0;
    return true;
  }
  if (n != 2) return false;
  const bool first27 = gg[0].zeta == 2 && gg[0].kb == 7;
  order[0] = first27 ? 0 : 1;
  order[1] = first27 ? 1 : 0;
  return true;
}

PersistKernel pick(const Geom& g, const Geom* gg, const int* order, int n) {
  if (n < 1 || n > PERSIST_MAX_GROUPS) return nullptr;
  const Geom& a = gg[order[0]];
  const int z1 = n == 2 ? gg[order[1]].zeta : 0, k1 = n == 2 ? gg[order[1]].kb : 0;
  if (g.st == ST_F32) return persist_kernel_f32(g.win_r, g.patch_r, a.zeta, a.kb, z1, k1);
  if (g.st == ST_F16) return persist_kernel_f16(g.win_r, g.patch_r, a.zeta, a.kb, z1, k1);
  return nullptr;
}

}  // namespace

bool persist_supported(const Geom& g, const Geom* gg, const int* tile, int n, int* order) {
  if (g.wscheme != WS_PATCH || n < 1 || n > PERSIST_MAX_GROUPS) return false;
  for (int i = 0; i < n; ++i)
    if (tile[i] != FAST_TILE || !gg[i].separable) return false;
  if (!slot_order(gg, n, order)) return false;
  return pick(g, gg, order, n) != nullptr;
}

cudaError_t persist_prepare(const Geom& g, const Geom* gg, const int* order, int n,
                            int smem_optin) {
  PersistKernel k = pick(g, gg, order, n);
  if (!k) return cudaErrorInvalidValue;
  return set_max_dynamic_smem(k, smem_optin);
}

size_t persist_smem(const Geom& g, const OpPlan* P, int n, int* sx_off) {
  size_t bytes = 0;
  for (int i = 0; i < n; ++i)
    if (P[i].smem_bytes > bytes) bytes = P[i].smem_bytes;
  // NLTV phases: the staged x, then the divergence tile on a 16-byte boundary
  const int nx = NF_T + 2 * (g.win_r + g.patch_r), nxp = nx | 1;
  const int x_floats = (nx * nxp + 3) & ~3;
  const int nr = NF_T + g.win_r, ncp = (NF_T + 2 * g.win_r) | 1;
  const size_t nlw = (size_t)(x_floats + nr * ncp) * sizeof(float);
  const int np = NF_T + 2 * g.win_r;
  const size_t nla = (size_t)np * (np | 1) * sizeof(float);
  if (nlw > bytes) bytes = nlw;
  if (nla > bytes) bytes = nla;
  *sx_off = x_floats;
  return bytes;
}

int persist_occupancy(const Geom& g, const Geom* gg, const int* order, int n, size_t smem) {
  PersistKernel k = pick(g, gg, order, n);
  int blocks = 0;
  if (!k || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k, FT_THREADS, smem) !=
                cudaSuccess)
    return 0;
  return blocks;
}

cudaError_t persist_launch(const Geom& g, const Geom* gg, const int* order, int n,
                           const PersistArgs* args, unsigned long long* bar, size_t smem,
                           int grid, cudaStream_t s) {
  PersistKernel k = pick(g, gg, order, n);
  if (!k || grid < 1) return cudaErrorInvalidValue;
  // the phases wait at grid barriers: a cooperative launch guarantees that
  // every CTA is resident (grid = SMs x the one CTA per SM the kernel holds)
  cudaLaunchConfig_t cfg{};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(FT_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const Geom& g0 = gg[order[0]];
  const Geom& g1 = n == 2 ? gg[order[1]] : g0;
  return cudaLaunchKernelEx(&cfg, k, g, g0, g1, args, bar);
}

}  // namespace lfsr
