// Shared-memory Stockham FFT used by the certificate's FFT passes (fft.cu) and
// by the degridding passes of the forward operator (degrid.cu).
#pragma once

#include "pc_internal.cuh"

namespace pc {

// Stockham autosort inverse FFT of `rows` rows of length G (row stride S)
// held in buffer a, using b as scratch. All threads of the block take part.
// Returns the buffer holding the result.
__device__ __forceinline__ float2* fft_rows_smem(float2* a, float2* b, int rows, int G, int logG, int S,
                                 const float2* tw) {
  const int nthr = blockDim.x;
  int ns = 1;
  if (logG & 1) {
    const int half = G >> 1;
    for (int f = threadIdx.x; f < rows * half; f += nthr) {
      const int r = f / half, j = f - r * half;
      const float2 v0 = a[r * S + j], v1 = a[r * S + j + half];
      b[r * S + 2 * j] = make_float2(v0.x + v1.x, v0.y + v1.y);
      b[r * S + 2 * j + 1] = make_float2(v0.x - v1.x, v0.y - v1.y);
    }
    __syncthreads();
    float2* t = a;
    a = b;
    b = t;
    ns = 2;
  }
  const int quarter = G >> 2;
  for (; ns < G; ns <<= 2) {
    const int step = G / (4 * ns);
    for (int f = threadIdx.x; f < rows * quarter; f += nthr) {
      const int r = f / quarter, j = f - r * quarter;
      const int k = j & (ns - 1);
      const float2* ar = a + r * S;
      float2 v0 = ar[j], v1 = ar[j + quarter], v2 = ar[j + 2 * quarter], v3 = ar[j + 3 * quarter];
      if (ns > 1) {
        v1 = cmul(v1, tw[k * step]);
        v2 = cmul(v2, tw[2 * k * step]);
        v3 = cmul(v3, tw[3 * k * step]);
      }
      const float2 s0 = make_float2(v0.x + v2.x, v0.y + v2.y);
      const float2 d0 = make_float2(v0.x - v2.x, v0.y - v2.y);
      const float2 s1 = make_float2(v1.x + v3.x, v1.y + v3.y);
      const float2 d1 = make_float2(v1.x - v3.x, v1.y - v3.y);
      float2* br = b + r * S + (j - k) * 4 + k;
      br[0] = make_float2(s0.x + s1.x, s0.y + s1.y);
      br[ns] = make_float2(d0.x - d1.y, d0.y + d1.x);        // d0 + i d1
      br[2 * ns] = make_float2(s0.x - s1.x, s0.y - s1.y);
      br[3 * ns] = make_float2(d0.x + d1.y, d0.y - d1.x);    // d0 - i d1
    }
    __syncthreads();
    float2* t = a;
    a = b;
    b = t;
  }
  return a;
}

}  // namespace pc
