// Weighted non-local TV with stored edge weights, part 1: the weight
// construction and the z/w-step of the regulariser rows (Eq. sr_reg;
// patch-distance weights from x^(n-1), one per undirected edge (u, u+d), d
// in the half window: s_d/2 x p values, written once per ADMM iteration and
// read by the K CG steps in nltv_fast.cu while they sit in L2).  Duals and
// weights are kept in the storage type ST (float, half or bfloat16); the
// regulariser's divergence (mu/2) S^T f goes straight into the accumulated v
// (DivAcc) and all arithmetic is float.
#include "nltv_fast.cuh"

namespace lfsr {

template <int MODE, int WR, int PR, class ST>
__global__ void __launch_bounds__(NF_THREADS)
k_nlw2(const Geom g, const TableArgs tb) {
  using SM = Nlw2Smem<MODE, WR, PR>;
  __shared__ float sX[SM::X];
  __shared__ float sV[SM::V];
  __shared__ double s_red[NF_THREADS / 32];
  // this CTA's tile: unit blockIdx.x of the table
  nlw2_unit<MODE, WR, PR, ST>(g, tb, blockIdx.x, sX, sV, s_red);
  if (MODE == NLW_BLOCK) nlw2_finish(tb);
}

template <int MODE, class ST>
static cudaError_t nlw2_dispatch(const Geom& g, const TableArgs& t, cudaStream_t s) {
#define NLW2_CASE(wr, pr)                                                          \
  if (g.win_r == wr && g.patch_r == pr) {                                          \
    k_nlw2<MODE, wr, pr, ST><<<t.total_units, NF_THREADS, 0, s>>>(g, t);           \
    return cudaGetLastError();                                                     \
  }
  NLW2_CASE(1, 0) NLW2_CASE(1, 1) NLW2_CASE(1, 2)
  NLW2_CASE(2, 0) NLW2_CASE(2, 1) NLW2_CASE(2, 2)
  NLW2_CASE(3, 0) NLW2_CASE(3, 1) NLW2_CASE(3, 2)
#undef NLW2_CASE
  return cudaErrorInvalidValue;
}

template <class ST>
static cudaError_t nlw2_st(int block, const Geom& g, const TableArgs& t, cudaStream_t s) {
  return block ? nlw2_dispatch<NLW_BLOCK, ST>(g, t, s) : nlw2_dispatch<NLW_ONLY, ST>(g, t, s);
}

cudaError_t nlw2_launch(int block, const Geom& g, const TableArgs& t, cudaStream_t s) {
  if (g.wscheme == WS_PAPER) return nlw2p_launch(block, g, t, s);
  if (t.total_units < 1) return cudaErrorInvalidValue;
  switch (g.st) {
    case ST_F32: return nlw2_st<float>(block, g, t, s);
    case ST_F16: return nlw2_st<__half>(block, g, t, s);
    case ST_BF16: return nlw2_st<__nv_bfloat16>(block, g, t, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace lfsr
