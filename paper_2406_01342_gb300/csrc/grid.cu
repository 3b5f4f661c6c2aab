// Gridding (type-1 spreading) of a visibility vector onto the w-stacked,
// oversampled uv grid: the first step of evaluating the adjoint of Sect. 2.2
// as a non-uniform FFT (Sect. 4.2). For plane q:
//
//   grid_q[b][a] += h_k tau_k phi(a - g_u,k) phi(b - g_v,k) phi(q - x_w,k)
//
// with phi the exponential-of-semicircle kernel of width W (in cells / planes)
// and tau_k = e^{j 2 pi (w_k - w0) s_c} the pre-twiddle that centres the
// w-screen frequencies. One CTA per gridding sub-problem (a tile of T x T
// cells, a group of Qg planes and at most 2048 binned visibilities): the
// visibilities are streamed with coalesced 16-byte loads, the tile is
// accumulated in shared memory, then added to the grid in HBM.
#include "pc_internal.cuh"

namespace pc {

__device__ __forceinline__ void red_add_f32x2(float2* addr, float2 v) {
  asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(addr), "f"(v.x), "f"(v.y)
               : "memory");
}

template <int W>
__global__ void __launch_bounds__(256)
k_grid(const int4* __restrict__ subs, const int2* __restrict__ slot_vis,
       const float4* __restrict__ slot_geom, const float2* __restrict__ h, int G, int T, int nT,
       int P, int Qg, float beta, int wstack, float2* __restrict__ grid) {
  extern __shared__ float2 acc[];  // [Qg][T][T]
  const int4 sub = subs[blockIdx.x];
  const int tu = sub.x % nT, tv = sub.x / nT;
  const int q0 = sub.y * Qg;
  const int Q = min(Qg, P - q0);
  const int TT = T * T;
  for (int c = threadIdx.x; c < Q * TT; c += blockDim.x) acc[c] = make_float2(0.f, 0.f);
  __syncthreads();

  const float two_over_w = 2.0f / W;
  for (int j = sub.z + threadIdx.x; j < sub.w; j += blockDim.x) {
    const int2 sv = slot_vis[j];
    const float4 gm = slot_geom[j];
    float2 hv = h[sv.x];
    const int a0 = (sv.y & 0xff) - 64;
    const int b0 = ((sv.y >> 8) & 0xff) - 64;
    const int ps = sv.y >> 16;
    float fu[W], fv[W];
#pragma unroll
    for (int c = 0; c < W; ++c) {
      fu[c] = es_kernel((c - gm.x) * two_over_w, beta);
      fv[c] = es_kernel((c - gm.y) * two_over_w, beta);
    }
    int cw_lo = 0, cw_hi = 1;
    float fw[W];
    if (wstack) {
      float sn, cs;
      sincospif(2.0f * gm.w, &sn, &cs);
      hv = cmul(hv, make_float2(cs, sn));
#pragma unroll
      for (int c = 0; c < W; ++c) fw[c] = es_kernel((c - gm.z) * two_over_w, beta);
      cw_lo = max(0, q0 - ps);
      cw_hi = min(W, q0 + Q - ps);
    } else {
#pragma unroll
      for (int c = 0; c < W; ++c) fw[c] = 1.0f;
    }
    for (int cw = cw_lo; cw < cw_hi; ++cw) {
      const float2 hw = make_float2(hv.x * fw[cw], hv.y * fw[cw]);
      float2* plane = acc + (ps + cw - q0) * TT;
#pragma unroll
      for (int bb = 0; bb < W; ++bb) {
        const int bl = b0 + bb;
        if (bl < 0 || bl >= T) continue;
        const float2 hb = make_float2(hw.x * fv[bb], hw.y * fv[bb]);
        float2* row = plane + bl * T;
#pragma unroll
        for (int aa = 0; aa < W; ++aa) {
          const int al = a0 + aa;
          if (al < 0 || al >= T) continue;
          atomicAdd(&row[al].x, hb.x * fu[aa]);
          atomicAdd(&row[al].y, hb.y * fu[aa]);
        }
      }
    }
  }
  __syncthreads();
  const size_t GG = (size_t)G * G;
  for (int c = threadIdx.x; c < Q * TT; c += blockDim.x) {
    const float2 v = acc[c];
    if (v.x == 0.0f && v.y == 0.0f) continue;
    const int q = c / TT, rem = c % TT;
    const int bl = rem / T, al = rem % T;
    float2* dst = grid + (size_t)(q0 + q) * GG + (size_t)(tv * T + bl) * G + (tu * T + al);
    red_add_f32x2(dst, v);
  }
}

int launch_grid(pc_plan_s* p, const float2* h, cudaStream_t st) {
  ProfScope prof_scope_(PROF_GRID, st);
  const size_t bytes = (size_t)p->P * p->G * p->G * sizeof(float2);
  PC_CUDA(cudaMemsetAsync(p->grid, 0, bytes, st));
  prof_scope_.kernels = 1;
  if (p->n_sub == 0) return PC_OK;
  prof_scope_.kernels = 2;
  const size_t smem = (size_t)p->Qg * p->T * p->T * sizeof(float2);
  const float beta = (float)p->beta;
  const int ws = p->wstack ? 1 : 0;
#define PC_GRID_CASE(WW)                                                                     \
  case WW: {                                                                                 \
    static bool attr_set = false;                                                            \
    if (!attr_set) {                                                                         \
      PC_CUDA(cudaFuncSetAttribute(k_grid<WW>, cudaFuncAttributeMaxDynamicSharedMemorySize,  \
                                   200 * 1024));                                             \
      attr_set = true;                                                                       \
    }                                                                                        \
    k_grid<WW><<<p->n_sub, 256, smem, st>>>(p->subs, p->slot_vis, p->slot_geom, h, p->G,     \
                                             p->T, p->nT, p->P, p->Qg, beta, ws, p->grid);   \
    break;                                                                                   \
  }
  switch (p->W) {
    PC_GRID_CASE(4)
    PC_GRID_CASE(5)
    PC_GRID_CASE(6)
    PC_GRID_CASE(7)
    PC_GRID_CASE(8)
    default:
      return fail(PC_ERR_INVALID_ARG, "gridding: unsupported kernel width %d", p->W);
  }
#undef PC_GRID_CASE
  PC_LAUNCH_CHECK();
  return PC_OK;
}

}  // namespace pc
