// One-warp inverse FFT of length G = 32 L (L = 16 or 32) held in registers.
//
// Lane l holds x[l + 32 m] in v[m], m < L, so a row is loaded with one
// coalesced 256-byte access per register. With n = l + 32 m and
// k = k1 + L k2 (k1 < L, k2 < 32):
//
//   X[k] = sum_l e^{+2 pi i l k2 / 32} e^{+2 pi i l k1 / G} sum_m x[l + 32 m] e^{+2 pi i m k1 / L}
//
// Step 1 is an L-point DFT along m in each lane's registers, step 2 the
// twiddle e^{+2 pi i l k1 / G}, step 3 a 32-point DFT along l. Step 3 needs
// the values of every lane for one k1: a transpose through a per-warp shared
// buffer (L = 32: lane t takes k1 = t; L = 16: the lane pair 2 k1, 2 k1 + 1
// splits it into its even and odd l, and one radix-2 step across the pair
// finishes it). The register DFTs are radix-2 decimation in frequency with
// compile-time indices, so the arrays stay in registers and the outputs come
// bit-reversed at no cost. No __syncthreads: a warp only waits on itself.
#pragma once

#include "pc_internal.cuh"

namespace pc {
namespace wfft {

__host__ __device__ constexpr int brev(int k, int bits) {
  int r = 0;
  for (int b = 0; b < bits; ++b) r |= ((k >> b) & 1) << (bits - 1 - b);
  return r;
}

// e^{+2 pi i m / 32}, m in [0, 16), as float
__device__ __forceinline__ float2 w32(int m) {
  constexpr float c1 = 0.98078528040323044f, c2 = 0.92387953251128674f, c3 = 0.83146961230254524f,
                  c4 = 0.70710678118654752f, c5 = 0.55557023301960218f, c6 = 0.38268343236508977f,
                  c7 = 0.19509032201612826f;
  switch (m) {
    case 0: return make_float2(1.f, 0.f);
    case 1: return make_float2(c1, c7);
    case 2: return make_float2(c2, c6);
    case 3: return make_float2(c3, c5);
    case 4: return make_float2(c4, c4);
    case 5: return make_float2(c5, c3);
    case 6: return make_float2(c6, c2);
    case 7: return make_float2(c7, c1);
    case 8: return make_float2(0.f, 1.f);
    case 9: return make_float2(-c7, c1);
    case 10: return make_float2(-c6, c2);
    case 11: return make_float2(-c5, c3);
    case 12: return make_float2(-c4, c4);
    case 13: return make_float2(-c3, c5);
    case 14: return make_float2(-c2, c6);
    default: return make_float2(-c1, c7);
  }
}

// v * e^{+2 pi i m / 32} for a compile-time m (after unrolling) in [0, 16)
__device__ __forceinline__ float2 rot32(float2 v, int m) {
  if (m == 0) return v;
  if (m == 8) return make_float2(-v.y, v.x);
  if (m == 4) {
    const float h = 0.70710678118654752f;
    return make_float2(h * (v.x - v.y), h * (v.x + v.y));
  }
  if (m == 12) {
    const float h = 0.70710678118654752f;
    return make_float2(-h * (v.x + v.y), h * (v.x - v.y));
  }
  return cmul(v, w32(m));
}

// In-place n-point inverse DFT (n = 16 or 32) of v[0..n): afterwards
// v[brev(k)] = sum_j v_in[j] e^{+2 pi i j k / n}.
template <int n>
__device__ __forceinline__ void dft_dif(float2* v) {
#pragma unroll
  for (int span = n / 2; span >= 1; span >>= 1) {
#pragma unroll
    for (int s = 0; s < n; s += 2 * span) {
#pragma unroll
      for (int k = 0; k < span; ++k) {
        const float2 a = v[s + k], b = v[s + k + span];
        v[s + k] = make_float2(a.x + b.x, a.y + b.y);
        // e^{+2 pi i k / (2 span)} = e^{+2 pi i (16 k / span) / 32}
        v[s + k + span] = rot32(make_float2(a.x - b.x, a.y - b.y), k * (16 / span));
      }
    }
  }
}

__host__ __device__ constexpr int log2c(int n) { return n <= 1 ? 0 : 1 + log2c(n / 2); }

// Per-warp shared buffer (float2 elements): the transpose needs L rows of
// 32 (+ padding); the padded row length keeps both the transposed writes and
// reads free of bank conflicts. The extra 2 elements make consecutive warps'
// buffers start 4 banks apart (conflict-free gathers across warps).
template <int L> struct Shape {
  static constexpr int row = (L == 32) ? 33 : 34;
  static constexpr int buf = L * row + 2;
  static constexpr int kept = L / 2;       // outputs per lane inside the N <= G / 2 image
};

// The inverse G-point FFT of the row held in v (see the top of the file).
// Afterwards output frequency f of lane `lane` is at
//   L = 32: f = lane + 32 k2                          in v[brev(k2, 5)], k2 < 32
//   L = 16: f = (lane >> 1) + 16 k' + 256 (lane & 1)  in v[brev(k', 4)], k' < 16
// `buf` is this warp's buffer (Shape<L>::buf elements); it is free again on
// return. T2 is the plan's global table T2[k1 * 32 + l] = e^{+2 pi i l k1 / G}
// (8 KB at G = 1024, read through the L1 cache: every warp reads all of it).
template <int L>
__device__ __forceinline__ void fft(float2 (&v)[L], float2* buf, const float2* __restrict__ T2, int lane) {
  constexpr int LB = log2c(L);
  constexpr int RW = Shape<L>::row;
  dft_dif<L>(v);                                       // v[brev(k1)] = step-1 output k1
#pragma unroll
  for (int k1 = 0; k1 < L; ++k1) {
    float2 y = v[brev(k1, LB)];
    if (k1 > 0) y = cmul(y, __ldg(T2 + k1 * 32 + lane));
    buf[k1 * RW + lane] = y;
  }
  __syncwarp();
  if (L == 32) {
#pragma unroll
    for (int l = 0; l < L; ++l) v[l] = buf[lane * RW + l];
    __syncwarp();
    dft_dif<L>(v);
  } else {
    const int k1 = lane >> 1, e = lane & 1;
#pragma unroll
    for (int l = 0; l < L; ++l) v[l] = buf[k1 * RW + 2 * l + e];
    __syncwarp();
    dft_dif<L>(v);                                     // 16-point DFT of the even / odd l
    // X[k1 + 16 (k' + 16 h)] = Z0[k'] + (-1)^h e^{+2 pi i k' / 32} Z1[k']:
    // the odd lane twiddles its Z1, the pair swaps, each keeps its own h = e
#pragma unroll
    for (int kp = 0; kp < L; ++kp) {
      const int r = brev(kp, LB);
      const float2 own = e ? rot32(v[r], kp) : v[r];
      const float2 other = make_float2(__shfl_xor_sync(0xffffffffu, own.x, 1),
                                       __shfl_xor_sync(0xffffffffu, own.y, 1));
      v[r] = e ? make_float2(other.x - own.x, other.y - own.y)
               : make_float2(own.x + other.x, own.y + other.y);
    }
  }
}

// The kept outputs: image index i = (f + N/2) mod G is inside [0, N) only for
// f < N - N/2 <= G/4 or f >= G - N/2 >= 3G/4, which are always among these
// Shape<L>::kept registers of each lane (c counts them).
//   L = 32: c < 8 -> k2 = c; c >= 8 -> k2 = c + 16
//   L = 16: k' = c + 8 (lane & 1)
template <int L>
__device__ __forceinline__ float2 kept_value(const float2 (&v)[L], int c, int lane) {
  if (L == 32) {
    const int k2 = c < 8 ? c : c + 16;
    return v[brev(k2, 5)];
  }
  const float2 lo = v[brev(c, 4)], hi = v[brev(c + 8, 4)];
  return (lane & 1) ? hi : lo;
}

template <int L>
__host__ __device__ __forceinline__ int kept_freq(int c, int lane) {
  if (L == 32) return lane + 32 * (c < 8 ? c : c + 16);
  return (lane >> 1) + 16 * (c + 8 * (lane & 1)) + 256 * (lane & 1);
}

}  // namespace wfft
}  // namespace pc
