// Lanczos step size of the restricted LASSO (the reweighting of Sect. 5.1):
// L = 1.01 x the top eigenvalue of the restricted Hessian, from the top Ritz
// value of a Lanczos tridiagonalisation that stops when that value changes by
// less than LZ_TOL between checks (every 4 steps) or after LZ_MAX steps.
// Shared by the Gram-form APGD kernels (apgd.cu) and the operator-form
// reweighting (reweight_op.cu).
#pragma once

#include "pc_internal.cuh"

namespace pc {

constexpr int LZ_MAX = 64;
constexpr float LZ_TOL = 1e-5f;   // relative change of the top Ritz value that stops Lanczos

// Largest eigenvalue of the symmetric tridiagonal matrix (diagonal al[0..m),
// off-diagonal be[0..m-1)) by multisection with Sturm counts: warp 0 narrows
// the Gershgorin interval 33-fold per round, on the matrix scaled by its
// Gershgorin bound (relative accuracy ~1e-6, enough for a step size that
// carries a 1 % margin). Same inputs in every CTA give the same result.
__device__ inline float tridiag_top(const float* al, const float* be, int m, float* s_out) {
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    float glo = 3e38f, ghi = -3e38f;
    for (int i = 0; i < m; ++i) {
      const float r = (i > 0 ? fabsf(be[i - 1]) : 0.f) + (i + 1 < m ? fabsf(be[i]) : 0.f);
      glo = fminf(glo, al[i] - r);
      ghi = fmaxf(ghi, al[i] + r);
    }
    float scale = fmaxf(fabsf(glo), fabsf(ghi));
    if (!(scale > 0.f)) scale = 1.f;
    const float inv = 1.f / scale;
    float lo = glo * inv, hi = ghi * inv;
    for (int round = 0; round < 6; ++round) {   // 33^-6 ~ 8e-10 of the Gershgorin width
      const float x = lo + (hi - lo) * (float)(lane + 1) * (1.0f / 33.0f);
      int below = 0;                          // eigenvalues below x = negative LDL^T pivots
      float d = al[0] * inv - x;
      if (d == 0.0f) d = -1e-30f;
      below += d < 0.0f;
      for (int i = 1; i < m; ++i) {
        const float bi = be[i - 1] * inv;
        d = (al[i] * inv - x) - __fdividef(bi * bi, d);
        if (d == 0.0f || !isfinite(d)) d = -1e-30f;
        below += d < 0.0f;
      }
      const unsigned has_top = __ballot_sync(0xffffffffu, below < m);   // an eigenvalue >= x
      const int L = has_top ? 31 - __clz(has_top) : -1;
      const float xl = __shfl_sync(0xffffffffu, x, L >= 0 ? L : 0);
      const float xr = __shfl_sync(0xffffffffu, x, L + 1 < 32 ? (L + 1 >= 0 ? L + 1 : 0) : 31);
      const float nlo = L >= 0 ? xl : lo;
      const float nhi = L < 31 ? xr : hi;
      lo = nlo;
      hi = nhi;
    }
    if (lane == 0) *s_out = hi * scale;
  }
  __syncthreads();
  return *s_out;
}

}  // namespace pc
