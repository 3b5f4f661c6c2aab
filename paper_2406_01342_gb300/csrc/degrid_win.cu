// Degridding interpolation (the last step of the type-2 non-uniform FFT of
// Sect. 5.2, the adjoint of the gridding's spread) over plane windows:
//
//   y_k += e^{-j 2 pi tau_k} sum_{q, b, a} phi(q - x_w,k) phi(b - g_v,k)
//                                          phi(a - g_u,k) grid_q[b][a]
//
// on the window gridding's schedule (grid_win.cuh): one CTA per tile (or part
// of a heavy tile) walks the tile's plane windows in order, keeping the
// window's 8 planes in a ring in shared memory (each window brings in only the
// planes the previous one did not hold). One thread per slot: every slot of
// window j has all its W planes inside [2j, 2j + 8), so the threads of a warp
// run the same plane loop (fixed plane groups leave each thread with about
// half of the group's planes and the warp with all of them). Per slot the
// W x W x W taps are read from the ring; the sum, times the conjugate
// pre-twiddle, is added to y_k with a vector reduction (a footprint may
// span several tiles).
#include "grid_win.cuh"

namespace pc {
namespace {

constexpr int DW_T = gwin::T, DW_Q = gwin::Q, DW_THREADS = gwin::THREADS;
constexpr int DW_RS = gwin::RS, DW_PS = gwin::PS, DW_MAXW = gwin::MAXW;

struct __align__(16) DwShared {
  float2 ring[DW_Q * DW_PS];    // the tile's planes 2j .. 2j + 7 at slots (plane & 7)
  int2 wr[DW_MAXW];             // this CTA's slot range {first, count} in every window
  int4 desc[4];                 // (filled by the shared schedule; unused here)
};

__device__ __forceinline__ void red_add_v2(float2* addr, float2 v) {
  asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(addr), "f"(v.x), "f"(v.y) : "memory");
}

// Planes [qa, qb) of the tile into the ring (zeros past the last plane).
__device__ __forceinline__ void planes_in(DwShared& S, int qa, int qb, const float2* tile_base, size_t GG, int G,
                                          int P) {
  const int e = threadIdx.x, row = e >> 3, c4 = (e & 7) * 4;
  for (int pl = qa; pl < qb; ++pl) {
    float4 u = make_float4(0.f, 0.f, 0.f, 0.f), v = u;
    if (pl < P) {
      const float4* src = reinterpret_cast<const float4*>(tile_base + (size_t)pl * GG + (size_t)row * G + c4);
      u = __ldg(src);
      v = __ldg(src + 1);
    }
    float2* dst = S.ring + (pl & (DW_Q - 1)) * DW_PS + row * DW_RS + c4;
    dst[0] = make_float2(u.x, u.y);
    dst[1] = make_float2(u.z, u.w);
    dst[2] = make_float2(v.x, v.y);
    dst[3] = make_float2(v.z, v.w);
  }
}

template <int W>
__global__ void __launch_bounds__(DW_THREADS, 3)
k_degrid_win(const int4* __restrict__ subs, const int* __restrict__ win_off, const int2* __restrict__ slot_vis,
             const float4* __restrict__ slot_geom, const float2* __restrict__ grid, int G, int nT, int P, int Pw,
             float beta, float2* __restrict__ y) {
  static_assert(W >= 2 && W <= 7, "a window of 8 planes holds the footprints of two plane starts");
  extern __shared__ __align__(16) unsigned char dw_raw[];
  DwShared& S = *reinterpret_cast<DwShared*>(dw_raw);
  const int4 sub = subs[blockIdx.x];
  const int tile = sub.x, tu = tile % nT, tv = tile / nT;
  const float two_over_w = 2.0f / W;
  const size_t GG = (size_t)G * G;
  const float2* const tile_base = grid + (size_t)(tv * DW_T) * G + tu * DW_T;
  gwin::schedule(win_off, tile, sub.y, sub.z, Pw, S.wr, S.desc);

  int held = -1;                                  // window whose planes the ring holds
  for (int j = 0; j < Pw; ++j) {
    const int2 wr = S.wr[j];                      // CTA-uniform
    if (wr.y <= 0) continue;
    const int q0 = 2 * j;
    // the planes of window j the ring does not hold yet
    planes_in(S, held < 0 ? q0 : max(2 * held + DW_Q, q0), q0 + DW_Q, tile_base, GG, G, P);
    held = j;
    __syncthreads();
    for (int s = wr.x + (int)threadIdx.x; s < wr.x + wr.y; s += DW_THREADS) {
      const int2 sv = slot_vis[s];
      const float4 gm = slot_geom[s];
      const int a0 = (sv.y & 0xff) - 64, b0 = ((sv.y >> 8) & 0xff) - 64;
      const int d = (sv.y >> 16) - q0;           // 0 or 1: the slot's first plane in the window
      // The footprint's cells inside the tile lie in the W x W block at
      // (a0c, b0c), the corner clamped into the tile; taps of that block
      // outside the footprint get weight zero, so every slot runs the same
      // unclipped tap loop.
      const int a0c = gwin::tap_corner(a0, W), b0c = gwin::tap_corner(b0, W);
      float fu[W], fv[W];
#pragma unroll
      for (int i = 0; i < W; ++i) {
        const int cu = i + a0c - a0, cv = i + b0c - b0;
        fu[i] = (cu >= 0 && cu < W) ? es_kernel((cu - gm.x) * two_over_w, beta) : 0.f;
        fv[i] = (cv >= 0 && cv < W) ? es_kernel((cv - gm.y) * two_over_w, beta) : 0.f;
      }
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll 1
      for (int c = 0; c < W; ++c) {
        const float2* t0 = S.ring + ((q0 + d + c) & (DW_Q - 1)) * DW_PS + b0c * DW_RS + a0c;
        float2 pq = make_float2(0.f, 0.f);
#pragma unroll
        for (int jb = 0; jb < W; ++jb) {
          float2 rr = make_float2(0.f, 0.f);
#pragma unroll
          for (int ia = 0; ia < W; ++ia) rr = __ffma2_rn(make_float2(fu[ia], fu[ia]), t0[jb * DW_RS + ia], rr);
          pq = __ffma2_rn(make_float2(fv[jb], fv[jb]), rr, pq);
        }
        const float fw = (q0 + d + c < P) ? es_kernel((c - gm.z) * two_over_w, beta) : 0.f;
        acc = __ffma2_rn(make_float2(fw, fw), pq, acc);
      }
      if (acc.x == 0.f && acc.y == 0.f) continue;
      float sn, cs;
      sincospif(2.0f * gm.w, &sn, &cs);
      red_add_v2(y + sv.x, cmul(acc, make_float2(cs, -sn)));     // e^{-j 2 pi tau}
    }
    __syncthreads();                              // the ring's readers are done before it changes
  }
}

}  // namespace

int launch_degrid_win(pc_plan_s* p, float2* y, cudaStream_t st) {
  if (p->n_dwsub == 0) return PC_OK;
  if (!p->wstack || p->W > 7 || p->T != DW_T || p->Pw > DW_MAXW)
    return fail(PC_ERR_INVALID_ARG, "window degridding: needs w-stacking, W <= 7, 32-cell tiles, <= %d windows",
                DW_MAXW);
  const int smem = (int)sizeof(DwShared);
  const float beta = (float)p->beta;
#define PC_DW_LAUNCH(WW)                                                                                    \
  case WW: {                                                                                                \
    static bool attr = false;                                                                               \
    if (!attr) {                                                                                            \
      PC_CUDA(cudaFuncSetAttribute(k_degrid_win<WW>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));  \
      attr = true;                                                                                          \
    }                                                                                                       \
    k_degrid_win<WW><<<p->n_dwsub, DW_THREADS, smem, st>>>(p->dwsubs, p->win_off, p->slot_vis, p->slot_geom,  \
                                                         p->grid, p->G, p->nT, p->P, p->Pw, beta, y);        \
    break;                                                                                                  \
  }
  switch (p->W) {
    PC_DW_LAUNCH(4)
    PC_DW_LAUNCH(5)
    PC_DW_LAUNCH(6)
    PC_DW_LAUNCH(7)
    default:
      return fail(PC_ERR_INVALID_ARG, "window degridding: unsupported kernel width %d", p->W);
  }
#undef PC_DW_LAUNCH
  PC_LAUNCH_CHECK();
  return PC_OK;
}

}  // namespace pc
