// Table (batch) instantiations of the specialised operator kernel
// (op_fast.cuh): the data block and the normal-matrix product over the
// (tile, view pair) units of every light field of a job table.
#include "op_fast.cuh"

namespace lfsr {

template <int Z, int KB>
static cudaError_t table_prepare_zk(int optin) {
  cudaError_t e = set_max_dynamic_smem(k_operator_fast<OP_NORMAL, Z, KB, false>, optin);
  if (e == cudaSuccess) e = set_max_dynamic_smem(k_operator_fast<OP_DATA, Z, KB, false>, optin);
  return e;
}

template <int Z, int KB>
static cudaError_t table_launch_zk(int mode, const Geom& g, const OpPlan& P, const TableArgs& t,
                                   int grid, cudaStream_t s) {
  const JobArgs none{};
  switch (mode) {
    case OP_NORMAL:
      k_operator_fast<OP_NORMAL, Z, KB, false><<<grid, FT_THREADS, P.smem_bytes, s>>>(g, P, t, none);
      break;
    case OP_DATA:
      k_operator_fast<OP_DATA, Z, KB, false><<<grid, FT_THREADS, P.smem_bytes, s>>>(g, P, t, none);
      break;
    default: return cudaErrorInvalidValue;   // the standalone operators run one light field
  }
  return cudaGetLastError();
}

cudaError_t fast_prepare_table(int zeta, int kb, int optin) {
#define X(z, k) if (zeta == z && kb == k) return table_prepare_zk<z, k>(optin);
  LFSR_FAST_CASES(X)
#undef X
  return cudaErrorInvalidValue;
}

cudaError_t fast_launch_table(int mode, const Geom& g, const OpPlan& P, const TableArgs& t, int grid,
                              cudaStream_t s) {
#define X(z, k) if (g.zeta == z && g.kb == k) return table_launch_zk<z, k>(mode, g, P, t, grid, s);
  LFSR_FAST_CASES(X)
#undef X
  return cudaErrorInvalidValue;
}

}  // namespace lfsr
