// Host side of the specialised operator kernel (op_fast.cuh): shared-memory
// layout, occupancy, kernel attributes and the single-light-field launches.
// The table (batch) instantiations live in op_fast_batch.cu.
#include "op_fast.cuh"

namespace lfsr {

template <int Z, int KB>
static cudaError_t fast_prepare_zk(int optin) {
  cudaError_t e = set_max_dynamic_smem(k_operator_fast<OP_NORMAL, Z, KB, true>, optin);
  if (e == cudaSuccess) e = set_max_dynamic_smem(k_operator_fast<OP_DATA, Z, KB, true>, optin);
  if (e == cudaSuccess) e = set_max_dynamic_smem(k_operator_fast<OP_FWD, Z, KB, true>, optin);
  if (e == cudaSuccess) e = set_max_dynamic_smem(k_operator_fast<OP_ADJ, Z, KB, true>, optin);
  if (e == cudaSuccess) e = fast_prepare_table(Z, KB, optin);
  return e;
}

template <int Z, int KB>
static int fast_occupancy(size_t smem) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_operator_fast<OP_NORMAL, Z, KB, true>,
                                                    FT_THREADS, smem) != cudaSuccess)
    return 1;
  return n > 0 ? n : 1;
}

template <int Z, int KB>
static cudaError_t fast_launch_zk(int mode, const Geom& g, const OpPlan& P, const TableArgs& t,
                                  const JobArgs& one, int grid, cudaStream_t s) {
  switch (mode) {
    case OP_NORMAL:
      if (one.fuse) {
        // the fused CG step waits at grid barriers: a cooperative launch
        // guarantees that every CTA is resident (the grid never exceeds the
        // co-resident count, see op_grid)
        cudaLaunchConfig_t cfg{};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeCooperative;
        at[0].val.cooperative = 1;
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(FT_THREADS);
        cfg.dynamicSmemBytes = P.smem_bytes;
        cfg.stream = s;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, k_operator_fast<OP_NORMAL, Z, KB, true>, g, P, t, one);
      }
      k_operator_fast<OP_NORMAL, Z, KB, true><<<grid, FT_THREADS, P.smem_bytes, s>>>(g, P, t, one);
      break;
    case OP_DATA:
      if (one.fuse) {
        cudaLaunchConfig_t cfg{};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeCooperative;
        at[0].val.cooperative = 1;
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(FT_THREADS);
        cfg.dynamicSmemBytes = P.smem_bytes;
        cfg.stream = s;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, k_operator_fast<OP_DATA, Z, KB, true>, g, P, t, one);
      }
      k_operator_fast<OP_DATA, Z, KB, true><<<grid, FT_THREADS, P.smem_bytes, s>>>(g, P, t, one);
      break;
    case OP_FWD:
      k_operator_fast<OP_FWD, Z, KB, true><<<grid, FT_THREADS, P.smem_bytes, s>>>(g, P, t, one);
      break;
    case OP_ADJ:
      k_operator_fast<OP_ADJ, Z, KB, true><<<grid, FT_THREADS, P.smem_bytes, s>>>(g, P, t, one);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

bool fast_supported(const Geom& g) {
  if (!g.separable || g.warp_views || g.adjoint_bw) return false;
#define X(z, k) if (g.zeta == z && g.kb == k) return true;
  LFSR_FAST_CASES(X)
#undef X
  return false;
}

cudaError_t fast_prepare(const Geom& g, int optin) {
#define X(z, k) if (g.zeta == z && g.kb == k) return fast_prepare_zk<z, k>(optin);
  LFSR_FAST_CASES(X)
#undef X
  return cudaErrorInvalidValue;
}

cudaError_t fast_plan(const Geom& g, OpPlan* P, int smem_limit) {
#define X(z, k)                                                     \
  if (g.zeta == z && g.kb == k) {                                   \
    if (fast_layout<z, k>(g, P, true) > (size_t)smem_limit &&       \
        fast_layout<z, k>(g, P, false) > (size_t)smem_limit)        \
      return cudaErrorInvalidValue;                                 \
    P->ctas_per_sm = fast_occupancy<z, k>(P->smem_bytes);           \
    P->fast = 1;                                                    \
    return cudaSuccess;                                             \
  }
  LFSR_FAST_CASES(X)
#undef X
  return cudaErrorInvalidValue;
}

cudaError_t fast_launch(int mode, const Geom& g, const OpPlan& P, const TableArgs& t, int grid,
                        cudaStream_t s, const JobArgs* single) {
  if (grid < 1 || t.total_units < 0) return cudaErrorInvalidValue;
  if (!single) return fast_launch_table(mode, g, P, t, grid, s);
#define X(z, k) \
  if (g.zeta == z && g.kb == k) return fast_launch_zk<z, k>(mode, g, P, t, *single, grid, s);
  LFSR_FAST_CASES(X)
#undef X
  return cudaErrorInvalidValue;
}

}  // namespace lfsr
