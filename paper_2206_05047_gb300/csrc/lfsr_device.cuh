// Device helpers shared by the kernel translation units of liblfsr.
#pragma once

#include "lfsr_internal.cuh"

namespace lfsr {

// Floor / ceil division for a possibly negative numerator and positive d.
__host__ __device__ __forceinline__ int floor_div(int n, int d) {
  return (n >= 0) ? (n / d) : -((-n + d - 1) / d);
}
__host__ __device__ __forceinline__ int ceil_div(int n, int d) {
  return (n >= 0) ? ((n + d - 1) / d) : -((-n) / d);
}
__host__ __device__ __forceinline__ int clampi(int v, int lo, int hi) {
  return v < lo ? lo : (v > hi ? hi : v);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the block in a fixed order (result valid in thread 0).  Every
// thread of the block must call it.
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* red /* >= NT/32 */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (warp == 0) {
    t = (lane < NT / 32) ? red[lane] : 0.0;
    t = warp_sum(t);
  }
  return t;
}

// Grid reduction without a second launch: each CTA stores its partial in
// partials[blockIdx.x]; the CTA that arrives last sums all partials in
// index order (deterministic for a given grid) and returns true with the
// total in *total (valid in thread 0).  The counter is re-armed for the
// next launch.
template <int NT>
__device__ __forceinline__ bool grid_sum_last(double part, double* partials, unsigned int* counter,
                                              double* total) {
  __shared__ double red[NT / 32];
  __shared__ int am_last;
  double s = block_sum<NT>(part, red);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = s;
    __threadfence();
    const unsigned int t = atomicAdd(counter, 1u);
    am_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!am_last) return false;
  __threadfence();
  double acc = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += NT) acc += ((volatile double*)partials)[i];
  acc = block_sum<NT>(acc, red);
  if (threadIdx.x == 0) {
    *total = acc;
    *counter = 0u;
  }
  return true;
}

}  // namespace lfsr
