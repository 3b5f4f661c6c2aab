// Plane-window scheduling of the window gridding (grid_win.cu).
//
// The plan bins every slot (visibility x tile its footprint touches) by tile
// and pair ps >> 1 of its first w-plane ps, sorted by its tile-local row start
// b0: window j of a tile holds the slots whose W <= 7 planes lie in
// [2j, 2j + 8). A CTA takes one tile (or one part of a heavy tile: its share
// of every window) and walks the windows in order, in chunks of GW_C slots;
// chunk c of a window run of L slots (nc = ceil(L / GW_C) chunks) takes every
// nc-th slot from c, a sample of all row starts in b0 order, so every warp
// (which owns four tile rows) finds work in every chunk.
#pragma once

#include "pc_internal.cuh"

namespace pc {
namespace gwin {

constexpr int T = 32;                    // tile side (the plan's)
constexpr int Q = 8;                     // planes per window
constexpr int C = 128;                   // slots per chunk
constexpr int THREADS = 256;             // 8 warps x 4 tile rows
constexpr int RS = T + 1;                // ring row stride (float2): rows one bank pair apart
constexpr int PS = RS * T + 4;           // ring plane stride (float2): planes four bank pairs apart
constexpr int MAXW = 128;                // plane windows per plan (w-planes up to 2 x 128 + W - 2)

__device__ __forceinline__ uint64_t pack2(float x, float y) {
  return (uint64_t)__float_as_uint(x) | ((uint64_t)__float_as_uint(y) << 32);
}
__device__ __forceinline__ float2 unpack2(uint64_t v) {
  return make_float2(__uint_as_float((uint32_t)v), __uint_as_float((uint32_t)(v >> 32)));
}

// Chunk descriptor {window j, first slot, slot stride nc, slots} (j < 0: none).
__host__ __device__ __forceinline__ int4 chunk_at(const int2* wr, int j, int c) {
  const int L = wr[j].y, nc = (L + C - 1) / C;
  return make_int4(j, wr[j].x + c, nc, (L - c + nc - 1) / nc);
}
__host__ __device__ __forceinline__ int4 chunk_after(const int2* wr, int Pw, int4 d) {
  if (d.x < 0) return d;
  const int c = d.y - wr[d.x].x;
  if (c + 1 < d.z) return chunk_at(wr, d.x, c + 1);
  for (int jj = d.x + 1; jj < Pw; ++jj)
    if (wr[jj].y > 0) return chunk_at(wr, jj, 0);
  return make_int4(-1, 0, 1, 0);
}

// Part `part` of `parts` of the slot range [bs, be): {first, count}; the
// parts are contiguous and cover the range once.
__host__ __device__ __forceinline__ int2 part_range(int bs, int be, int part, int parts) {
  const long long len = be - bs;
  const int s0 = bs + (int)(len * part / parts), s1 = bs + (int)(len * (part + 1) / parts);
  return make_int2(s0, s1 - s0);
}

// The degridding's tap block of a footprint starting at tile-local column
// (or row) a0 in [-(W - 1), T - 1]: its corner clamped into the tile. The
// footprint's cells inside the tile are the block's taps i with
// 0 <= i + corner - a0 < W (the footprint's own tap index); the others get
// weight zero.
__host__ __device__ __forceinline__ int tap_corner(int a0, int W) {
  return a0 < 0 ? 0 : (a0 > T - W ? T - W : a0);
}

// This part's slot range {first, count} of every window of the tile (all
// threads), then (after a barrier) the first three chunk descriptors (thread 0).
// Ends with a barrier.
__device__ __forceinline__ void schedule(const int* __restrict__ win_off, int tile, int part, int parts, int Pw,
                                         int2* wr, int4* desc) {
  for (int t = threadIdx.x; t < Pw; t += blockDim.x) {
    const int bs = __ldg(win_off + (size_t)tile * Pw + t), be = __ldg(win_off + (size_t)tile * Pw + t + 1);
    wr[t] = part_range(bs, be, part, parts);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int4 d = make_int4(-1, 0, 1, 0);
    for (int jj = 0; jj < Pw; ++jj)
      if (wr[jj].y > 0) {
        d = chunk_at(wr, jj, 0);
        break;
      }
    desc[0] = d;
    desc[1] = d = chunk_after(wr, Pw, d);
    desc[2] = chunk_after(wr, Pw, d);
  }
  __syncthreads();
}

// The run [lo, hi) of chunk slots whose rows [b0, b0 + W) meet warp w's rows
// [4w, 4w + 4): meta[k] >> 8 = b0 + 8, ascending over the chunk's slots, and
// above every bound past its count.
template <int W>
__device__ __forceinline__ int2 warp_run(const int* meta, int warp, int lane) {
  const int4 m4 = reinterpret_cast<const int4*>(meta)[lane];
  const int blo = 4 * warp - W + 1 + 8, bhi = 4 * warp + 4 + 8;
  const int v0 = m4.x >> 8, v1 = m4.y >> 8, v2 = m4.z >> 8, v3 = m4.w >> 8;
  const unsigned nlo = (v0 < blo) + (v1 < blo) + (v2 < blo) + (v3 < blo);
  const unsigned nhi = (v0 < bhi) + (v1 < bhi) + (v2 < bhi) + (v3 < bhi);
  return make_int2((int)__reduce_add_sync(0xffffffffu, nlo), (int)__reduce_add_sync(0xffffffffu, nhi));
}

}  // namespace gwin
}  // namespace pc
