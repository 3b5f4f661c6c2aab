// One-CTA inverse FFT of length G = 512 R (R = 4, 8 or 16 warps; G = 2048,
// 4096, 8192) for the grids whose rows do not fit one warp's registers.
//
// With n = n' + 512 r (n' < 512, r < R) and k = k1 + R f (k1 < R, f < 512):
//
//   X[k1 + R f] = sum_n' e^{+2 pi i n' f / 512} [ e^{+2 pi i n' k1 / G} sum_r x[n' + 512 r] e^{+2 pi i r k1 / R} ]
//
// Step A, every thread: for each of its n' = t + 32 R j (j < 16 / R), an
// R-point DFT over r in registers, the twiddle e^{+2 pi i n' k1 / G}, and a
// store to row k1 of the CTA's exchange buffer Z. Step B, warp w: the
// 512-point one-warp FFT (fft_warp.cuh) of row w of Z, which that warp then
// also uses as its transpose buffer. One block barrier per transform.
//
// Thread t holds u[j R + r] = x[t + 32 R j + 512 r] on entry. On return lane
// `lane` of warp k1 holds X[k1 + R f] in u[brev(k', 4)] with
// f = (lane >> 1) + 16 k' + 256 (lane & 1) (the one-warp FFT's order), and
// the kept outputs of an image of side N <= G / 2 are its registers c < 8 of
// wfft::kept_value<16> (frequencies below G / 4 or from 3 G / 4 on).
#pragma once

#include "fft_warp.cuh"

namespace pc {
namespace cfft {

constexpr int L = 16;                              // one-warp FFT of 32 L = 512 points
constexpr int ZS = wfft::Shape<L>::buf;            // Z row stride (>= 512; the warp's FFT buffer)

template <int R>
struct Cfg {
  static_assert(R == 4 || R == 8 || R == 16, "G = 512 R with R = 4, 8 or 16");
  static constexpr int G = 512 * R;
  static constexpr int THREADS = 32 * R;
  static constexpr int J = L / R;                  // n' values per thread
  static constexpr int Z_ELEMS = R * ZS;           // float2 elements of shared memory
};

// Position n of register e of thread t (u[e], e = j R + r).
template <int R>
__host__ __device__ __forceinline__ int pos(int t, int e) {
  return t + 32 * R * (e / R) + 512 * (e % R);
}

// Whether register e can hold a value of a length-N sequence centred on the
// row (position n <-> index (n + N/2) mod G, inside [0, N) for N <= G / 2 only
// if n < G / 4 or n >= 3 G / 4): a compile-time property of e's r = e mod R.
template <int R>
__host__ __device__ constexpr bool centred_reg(int e) {
  return (e % R) < R / 4 || (e % R) >= 3 * R / 4;
}

// Full output frequency k of register u[brev(kp, 4)] of lane `lane` in warp k1.
template <int R>
__host__ __device__ __forceinline__ int freq(int k1, int lane, int kp) {
  return k1 + R * ((lane >> 1) + 16 * kp + 256 * (lane & 1));
}

// Kept output c < 8 (wfft::kept_value<16>) of lane `lane` in warp k1.
template <int R>
__host__ __device__ __forceinline__ int kept_freq(int k1, int lane, int c) {
  return k1 + R * wfft::kept_freq<L>(c, lane);
}

// Shared-memory slot of output frequency k (< G) when a CTA stages a
// transformed row in Z. The 16 lanes of a half-warp hold frequencies
// k = k1 + R f with f = (lane >> 1) + 16 k' + X (lane & 1) (X = 256; 128 for
// the kept outputs folded into [0, G / 2)), i.e. multiples of R apart, which
// would put them on a few of the 16 eight-byte bank pairs. XOR-ing the bits
// of k1 with bits of f (the low ones, and bit PB for the lane pair) spreads
// them over all 16; the map is a bijection that keeps every aligned group of
// R slots in place, so runs of consecutive k stay conflict-free too.
template <int R, int PB>
__host__ __device__ __forceinline__ int stage_mask(int k) {
  constexpr int LR = wfft::log2c(R);
  const int f = k >> LR;
  return ((f >> (4 - LR)) & ((1 << (LR - 1)) - 1)) | (((f >> PB) & 1) << (LR - 1));
}
template <int R, int PB>
__host__ __device__ __forceinline__ int stage_pos(int k) {
  return k ^ stage_mask<R, PB>(k);
}
// A lane's outputs differ only in f's bits 4..7 (16 k'; bit 8 or 7 is the
// lane pair's), which the mask does not read: one mask serves all of them.

// tw[k1 * 512 + n'] = e^{+2 pi i n' k1 / G} (R x 512 = G entries: a warp's
// reads for one k1 are contiguous); T2[k1 * 32 + l] = e^{+2 pi i l k1 / 512}
// (k1 < 16). Z: Cfg<R>::Z_ELEMS float2 of shared memory, free on entry; the
// caller places a __syncthreads() between this call's return and any other
// use of Z.
template <int R>
__device__ __forceinline__ void fft(float2 (&u)[L], float2* Z, const float2* __restrict__ tw,
                                   const float2* __restrict__ T2) {
  constexpr int G = Cfg<R>::G, J = Cfg<R>::J, LR = wfft::log2c(R);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
#pragma unroll
  for (int j = 0; j < J; ++j) wfft::dft_dif<R>(u + j * R);   // u[jR + brev(k1)] = sum_r ...
#pragma unroll
  for (int j = 0; j < J; ++j) {
    const int np = t + 32 * R * j;
#pragma unroll
    for (int k1 = 0; k1 < R; ++k1) {
      float2 y = u[j * R + wfft::brev(k1, LR)];
      if (k1 > 0) y = cmul(y, __ldg(tw + k1 * 512 + np));
      Z[k1 * ZS + np] = y;
    }
  }
  __syncthreads();
  const float2* row = Z + warp * ZS;
#pragma unroll
  for (int m = 0; m < L; ++m) u[m] = row[lane + 32 * m];
  __syncwarp();
  wfft::fft<L>(u, Z + warp * ZS, T2, lane);
}

}  // namespace cfft
}  // namespace pc
