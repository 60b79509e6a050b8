// Shared constants of the stored-weight NLTV kernels (window radius WR in
// {1,2,3}, patch radius PR in {0,1,2}, compile time): tile and thread
// layout and the half window's direction table.
#pragma once

#include "lfsr_device.cuh"

namespace lfsr {

constexpr int NF_THREADS = 256;
constexpr int NF_T = 32;
constexpr int NF_PIX = NF_T * NF_T / NF_THREADS;
// The weighted-divergence kernel (k_nla2) is bound by the latency of its
// weight loads: it runs the same tiles with twice the threads (strips of 2
// rows), 27 warps per SM instead of 13.
constexpr int NA_THREADS = 512;
constexpr int NA_PIX = NF_T * NF_T / NA_THREADS;

enum { NLW_BLOCK = 0, NLW_ONLY = 1 };

// Pixel-owner kernels, no shared-memory exchange between directions.
// Each thread owns a strip of NF_PIX = 4 consecutive rows of one column of
// a 32 x 32 tile (rows 4 warp + m, column lane).  The half window's
// directions are compile-time constants (raster order, the same table the
// host builds), so the direction loops unroll and every global load of a
// thread is independent of the others.
template <int WR>
struct HalfDirs {
  static constexpr int W = 2 * WR + 1;
  static constexpr int SH = (W * W - 1) / 2;
  static __device__ __forceinline__ constexpr int di(int idx) { return idx / W - WR; }
  static __device__ __forceinline__ constexpr int dj(int idx) { return idx % W - WR; }
};

}  // namespace lfsr
