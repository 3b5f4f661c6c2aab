// Gridding (type-1 spreading) of a visibility vector onto the w-stacked,
// oversampled uv grid: the first step of evaluating the adjoint of Sect. 2.2
// as a non-uniform FFT (Sect. 5.2). For plane q:
//
//   grid_q[b][a] += h_k tau_k phi(a - g_u,k) phi(b - g_v,k) phi(q - x_w,k)
//
// with phi the exponential-of-semicircle kernel of width W (in cells / planes)
// and tau_k = e^{j 2 pi (w_k - w0) s_c} the pre-twiddle that centres the
// w-screen frequencies.
//
// One CTA per gridding sub-problem: a 32 x 32 tile, a group of at most 8
// planes and at most 1024 binned visibilities (every visibility whose
// footprint touches the tile was binned into it at plan time). The tile is
// accumulated in registers, not in shared memory: warp w owns rows
// [4w, 4w + 4) of the tile for every plane of the group, lane a owns column a.
// Visibilities are processed in chunks of 256: first each thread evaluates
// the kernel weights of one visibility (W in u, W in v, one per plane of the
// group) into shared memory, then every warp sweeps the chunk, skips the
// visibilities whose footprint misses its 4 rows, and accumulates
// h * phi_u[a] * phi_v[b] * phi_w[q] with plain FMAs. No atomics touch shared
// memory; the finished tile is added to the grid with vector reductions
// (sub-problems of one tile may run on several CTAs).
#include "pc_internal.cuh"

namespace pc {

__device__ __forceinline__ void red_add_f32x2(float2* addr, float2 v) {
  asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(addr), "f"(v.x), "f"(v.y)
               : "memory");
}

constexpr int GRID_T = 32;        // tile side (one lane per column)
constexpr int GRID_CHUNK = 256;   // visibilities staged per chunk
constexpr int GRID_ROWS = 4;      // tile rows per warp (8 warps x 4 = 32)

template <int W, int QMAX>
__global__ void __launch_bounds__(256)
k_grid(const int4* __restrict__ subs, const int2* __restrict__ slot_vis,
       const float4* __restrict__ slot_geom, const float2* __restrict__ h, int G, int nT, int P,
       int Qg, float beta, int wstack, float2* __restrict__ grid) {
  __shared__ float s_fu[GRID_CHUNK][8];
  __shared__ float s_fv[GRID_CHUNK][8];
  __shared__ float s_fw[GRID_CHUNK][QMAX];
  __shared__ float2 s_h[GRID_CHUNK];
  __shared__ int s_ab[GRID_CHUNK];        // (a0 + 64) | (b0 + 64) << 8

  const int4 sub = subs[blockIdx.x];
  const int tu = sub.x % nT, tv = sub.x / nT;
  const int q0 = sub.y * Qg;
  const int Q = min(Qg, P - q0);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int r0 = warp * GRID_ROWS;
  const float two_over_w = 2.0f / W;

  float2 acc[GRID_ROWS][QMAX];
#pragma unroll
  for (int r = 0; r < GRID_ROWS; ++r)
#pragma unroll
    for (int q = 0; q < QMAX; ++q) acc[r][q] = make_float2(0.f, 0.f);

  for (int c0 = sub.z; c0 < sub.w; c0 += GRID_CHUNK) {
    const int cnt = min(GRID_CHUNK, sub.w - c0);
    // ---- phase 1: kernel weights of one visibility per thread
    if (tid < cnt) {
      const int j = c0 + tid;
      const int2 sv = slot_vis[j];
      const float4 gm = slot_geom[j];
      float2 hv = h[sv.x];
      if (wstack) {
        float sn, cs;
        sincospif(2.0f * gm.w, &sn, &cs);
        hv = cmul(hv, make_float2(cs, sn));
      }
#pragma unroll
      for (int c = 0; c < W; ++c) {
        s_fu[tid][c] = es_kernel((c - gm.x) * two_over_w, beta);
        s_fv[tid][c] = es_kernel((c - gm.y) * two_over_w, beta);
      }
      const int ps = sv.y >> 16;
#pragma unroll
      for (int q = 0; q < QMAX; ++q) {
        const int cw = q0 + q - ps;
        float f = 0.f;
        if (q < Q)
          f = wstack ? ((cw >= 0 && cw < W) ? es_kernel((cw - gm.z) * two_over_w, beta) : 0.f) : 1.f;
        s_fw[tid][q] = f;
      }
      s_h[tid] = hv;
      s_ab[tid] = sv.y & 0xffff;
    }
    __syncthreads();
    // ---- phase 2: every warp accumulates its 4-row band
    for (int t = 0; t < cnt; ++t) {
      const int ab = s_ab[t];
      const int b0 = ((ab >> 8) & 0xff) - 64;
      if (b0 > r0 + GRID_ROWS - 1 || b0 + W - 1 < r0) continue;     // warp-uniform
      const int da = lane - ((ab & 0xff) - 64);
      const float wu = (da >= 0 && da < W) ? s_fu[t][da] : 0.f;
      const float2 hh = s_h[t];
      const float2 hu = make_float2(hh.x * wu, hh.y * wu);
      float fw[QMAX];
#pragma unroll
      for (int q = 0; q < QMAX; ++q) fw[q] = s_fw[t][q];
#pragma unroll
      for (int r = 0; r < GRID_ROWS; ++r) {
        const int db = r0 + r - b0;
        const float wv = (db >= 0 && db < W) ? s_fv[t][db] : 0.f;
        const float2 hr = make_float2(hu.x * wv, hu.y * wv);
#pragma unroll
        for (int q = 0; q < QMAX; ++q) {
          acc[r][q].x = fmaf(hr.x, fw[q], acc[r][q].x);
          acc[r][q].y = fmaf(hr.y, fw[q], acc[r][q].y);
        }
      }
    }
    __syncthreads();
  }
  // ---- add the band to the grid (plane-major, b rows, a contiguous)
  const size_t GG = (size_t)G * G;
#pragma unroll
  for (int q = 0; q < QMAX; ++q) {
    if (q >= Q) break;
#pragma unroll
    for (int r = 0; r < GRID_ROWS; ++r) {
      const float2 v = acc[r][q];
      if (v.x == 0.f && v.y == 0.f) continue;
      float2* dst = grid + (size_t)(q0 + q) * GG + (size_t)(tv * GRID_T + r0 + r) * G +
                    (tu * GRID_T + lane);
      red_add_f32x2(dst, v);
    }
  }
}

// Zero the grid rows that visibilities can reach (every plane); the other
// rows are never written and stay zero. cols: the 32-column groups to clear
// (all when the first FFT pass reads whole rows; else only the groups that
// hold visibilities, the only ones the one-warp pass reads).
__global__ void k_zero_rows(float2* __restrict__ grid, const int* __restrict__ rows, int n_rows,
                            int G, int P, const uint32_t* __restrict__ colw) {
  const int rr = blockIdx.x, q = blockIdx.y;
  if (rr >= n_rows) return;
  float4* dst = reinterpret_cast<float4*>(grid + ((size_t)q * G + rows[rr]) * G);
  for (int c = threadIdx.x; c < G / 2; c += blockDim.x) {
    const int g = c >> 4;                          // 32-column group of the pair of cells
    if (!colw || ((__ldg(colw + (g >> 5)) >> (g & 31)) & 1u)) dst[c] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

int launch_grid(pc_plan_s* p, const float2* h, cudaStream_t st) {
  ProfScope prof_scope_(PROF_GRID, st);
  if (p->n_sub == 0) return PC_OK;        // nothing is ever written: the grid stays zero
  {
    dim3 zg(p->n_active_rows, p->P);
    // the one-warp and one-CTA first passes read only the column groups that
    // can hold data; the Stockham pass reads whole rows
    const uint32_t* cols = (fft_rows_warp(p) || fft_rows_big(p)) ? p->col_bits : nullptr;
    k_zero_rows<<<zg, 256, 0, st>>>(p->grid, p->active_rows, p->n_active_rows, p->G, p->P, cols);
    PC_LAUNCH_CHECK();
  }
  prof_scope_.kernels = 1;
  if (p->T != GRID_T || p->Qg > 8)
    return fail(PC_ERR_INVALID_ARG, "gridding: needs 32-cell tiles and <= 8 planes per group");
  prof_scope_.kernels = 2;
  // tensor cores for w-stacked plans (the coplanar case has one plane and
  // would leave 7/8 of the tensor-core tile empty); iscal[7] = timeout flag
  if (grid_win_mode(p)) return launch_grid_win(p, h, st);
  if (p->wstack && p->grid_mode != 1) return launch_grid_tc(p, h, p->iscal + 7, st);
  const float beta = (float)p->beta;
  const int ws = p->wstack ? 1 : 0;
#define PC_GRID_CASE(WW)                                                                      \
  case WW:                                                                                    \
    if (p->Qg == 1)                                                                           \
      k_grid<WW, 1><<<p->n_sub, 256, 0, st>>>(p->subs, p->slot_vis, p->slot_geom, h, p->G,    \
                                               p->nT, p->P, p->Qg, beta, ws, p->grid);        \
    else                                                                                      \
      k_grid<WW, 8><<<p->n_sub, 256, 0, st>>>(p->subs, p->slot_vis, p->slot_geom, h, p->G,    \
                                               p->nT, p->P, p->Qg, beta, ws, p->grid);        \
    break;
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
