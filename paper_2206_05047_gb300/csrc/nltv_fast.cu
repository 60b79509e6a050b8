// Weighted non-local TV with stored edge weights, part 2: the weighted
// divergence S^T W^2 S p of every CG step and the canonical-layout export
// of the weights.  The weights (s_d/2 x p values of the storage type ST,
// written by nltv_block.cu) are read while they sit in L2; all arithmetic
// is float.
#include "nltv_fast.cuh"

namespace lfsr {

template <int WR, class ST, int DB>
__global__ void __launch_bounds__(NA_THREADS, 2)
k_nla2(const Geom g, const TableArgs tb) {
  __shared__ float sP[Nla2Smem<WR>::P];
  __shared__ double s_red[NA_THREADS / 32];
  // this CTA's tile: unit blockIdx.x of the table
  nla2_unit<WR, ST, DB>(g, tb, blockIdx.x, sP, s_red);
  nla2_finish(tb);
}

// canonical weights [d][u] from the stored edge weights wt[idx][u]
template <class ST>
__global__ void k_weights_to_canonical(const Geom g, const ST* __restrict__ wt,
                                       float* __restrict__ can) {
  const size_t p = (size_t)g.Hh * g.Wh;
  const int sd = 2 * g.sh;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < (size_t)sd * p;
       t += (size_t)gridDim.x * blockDim.x) {
    const int d = (int)(t / p);
    const size_t u = t - (size_t)d * p;
    float v = 0.f;
    if (d < g.sh) {
      v = ld_s(wt + (size_t)d * p + u);
    } else {
      const int idx = sd - 1 - d;
      const int ui = (int)(u / g.Wh), uj = (int)(u - (size_t)ui * g.Wh);
      const int vi = ui - g.di[idx], vj = uj - g.dj[idx];
      if (vi >= 0 && vi < g.Hh && vj >= 0 && vj < g.Wh)
        v = ld_s(wt + (size_t)idx * p + (size_t)vi * g.Wh + vj);
    }
    can[t] = v;
  }
}

// ---------------------------------------------------------------------------
bool nlf_supported(const Geom& g) {
  return g.win_r >= 1 && g.win_r <= 3 && g.patch_r >= 0 && g.patch_r <= 2;
}

template <class ST, int DB>
static cudaError_t nla2_st(const Geom& g, const TableArgs& t, cudaStream_t s) {
  switch (g.win_r) {
    case 1: k_nla2<1, ST, DB><<<t.total_units, NA_THREADS, 0, s>>>(g, t); break;
    case 2: k_nla2<2, ST, DB><<<t.total_units, NA_THREADS, 0, s>>>(g, t); break;
    case 3: k_nla2<3, ST, DB><<<t.total_units, NA_THREADS, 0, s>>>(g, t); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <class ST>
static cudaError_t nla2_db(const Geom& g, const TableArgs& t, cudaStream_t s, int chunk) {
  if (chunk == 6) return nla2_st<ST, 6>(g, t, s);
  if (chunk == 3) return nla2_st<ST, 3>(g, t, s);
  return cudaErrorInvalidValue;
}

cudaError_t nla2_launch(const Geom& g, const TableArgs& t, cudaStream_t s, int chunk) {
  if (t.total_units < 1) return cudaErrorInvalidValue;
  switch (g.st) {
    case ST_F32: return nla2_db<float>(g, t, s, chunk);
    case ST_F16: return nla2_db<__half>(g, t, s, chunk);
    case ST_BF16: return nla2_db<__nv_bfloat16>(g, t, s, chunk);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t weights_to_canonical(const Geom& g, const void* wt, float* can, cudaStream_t s) {
  switch (g.st) {
    case ST_F32: k_weights_to_canonical<<<1024, 256, 0, s>>>(g, (const float*)wt, can); break;
    case ST_F16: k_weights_to_canonical<<<1024, 256, 0, s>>>(g, (const __half*)wt, can); break;
    case ST_BF16:
      k_weights_to_canonical<<<1024, 256, 0, s>>>(g, (const __nv_bfloat16*)wt, can);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace lfsr
