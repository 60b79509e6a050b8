// Shared constants of the stored-weight NLTV kernels (window radius WR in
// {1,2,3}, patch radius PR in {0,1,2}, compile time): tile and thread
// layout and the half window's direction table.
#pragma once

#include "lfsr_device.cuh"

namespace lfsr {

constexpr int NF_THREADS = 512;
constexpr int NF_T = 32;
constexpr int NF_PIX = NF_T * NF_T / NF_THREADS;
// The weighted-divergence kernel (k_nla2) is bound by the latency of its
// weight loads: it runs the same tiles with twice the threads (strips of 2
// rows), 27 warps per SM instead of 13.
constexpr int NA_THREADS = 512;
constexpr int NA_PIX = NF_T * NF_T / NA_THREADS;

enum { NLW_BLOCK = 0, NLW_ONLY = 1 };

// Pixel-owner kernels, no shared-memory exchange between directions.
// Each thread owns a strip of NF_PIX consecutive rows of one column of a
// 32 x 32 tile (rows NF_PIX warp + m, column lane).  The half window's
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

// Divergence accumulator of one NLTV tile (the regulariser's share of v in
// the z/w-step, Sec. 4.1 wdd): every edge term c(u, d) of the tile's pixels
// u adds c to v(u) and -c to v(u + d).  With d in the half window (d_i <= 0)
// the targets lie in the tile, WR rows above it and WR columns either side.
// A CTA gathers them in shared memory (float shared atomics) and adds the
// whole region to the light field's v with global float atomics, so tiles
// whose halos overlap add up; v must be zero before the NLTV block runs.
template <int WR>
struct DivAcc {
  static constexpr int NR = NF_T + WR;          // rows: WR above the tile
  static constexpr int NC = NF_T + 2 * WR;      // columns: WR either side
  static constexpr int NCp = NC | 1;
  static constexpr int SIZE = NR * NCp;
  // smem index of tile-local pixel (r, c), -WR <= r < NF_T, -WR <= c < NF_T + WR
  static __device__ __forceinline__ int at(int r, int c) { return (r + WR) * NCp + (c + WR); }
  static __device__ __forceinline__ void clear(float* acc, int tid, int nthreads) {
    for (int t = tid; t < SIZE; t += nthreads) acc[t] = 0.f;
  }
  // adds the region to v (Hh x Wh); entries outside the image are zero
  static __device__ __forceinline__ void flush(const float* acc, float* v, int i0, int j0, int Hh,
                                               int Wh, int tid, int nthreads) {
    for (int t = tid; t < NR * NC; t += nthreads) {
      const int rr = t / NC, cc = t - rr * NC;
      const int hi = i0 - WR + rr, hj = j0 - WR + cc;
      const float val = acc[rr * NCp + cc];
      if (val != 0.f && hi >= 0 && hi < Hh && hj >= 0 && hj < Wh)
        atomicAdd(v + (size_t)hi * Wh + hj, val);
    }
  }
};

}  // namespace lfsr
