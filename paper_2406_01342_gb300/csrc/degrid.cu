// The forward equation of Sect. 2.2 on a dense image, evaluated as a type-2
// non-uniform FFT (degridding; the type-2 half of the NUFFT the paper uses
// for its operators, Sect. 5.2):
//
//   Phi(I)[k] = sum_p I_p / n_p e^{-j 2 pi (u_k l_p + v_k m_p + w_k (n_p - 1))}.
//
// It is built as the exact adjoint of the certificate path (gridding, two
// inverse FFT passes, epilogue): writing that path as mu = Re(L h) with L
// complex-linear, Re<Phi x, h> = <x, Phi* h> for every h gives Phi x = L^H x,
// i.e. in reverse order
//
//   1. k_degrid_cols   z_q[i][j] = c_ij e^{+j 2 pi q t_ij} x_ij on the N x N
//                      centre of a length-G row (c_ij, t_ij: the epilogue's
//                      per-pixel coefficient and w-screen turns), a forward
//                      FFT along j, kept at the grid rows b a visibility can
//                      reach: X_q[b][i];
//   2. k_degrid_rows   a forward FFT along i of each such row, placed on the
//                      N-entry centre of a length-G vector: grid_q[b][a];
//   3. k_degrid        per gridding sub-problem (tile, plane group, binned
//                      slots) the tile in shared memory; per slot the W x W x Q
//                      kernel-weighted sum of the tile, times e^{-j 2 pi tau}
//                      (the conjugate of the gridding pre-twiddle), added to
//                      y_k (a visibility's footprint may span several tiles).
//
// A forward FFT is evaluated as conj(IFFT(conj(.))) with the inverse FFTs of
// the certificate path, so both directions share one FFT code path: one warp
// per row in registers where G is 512 or 1024 (fft_warp.cuh), else the
// shared-memory Stockham stages (fft.cuh).
#include "fft.cuh"
#include "fft_warp.cuh"

namespace pc {
namespace {

constexpr int DG_R1 = 4;   // image rows per CTA of the first pass

__device__ __forceinline__ float2 conj2(float2 v) { return make_float2(v.x, -v.y); }

__global__ void __launch_bounds__(256)
k_degrid_cols(const float* __restrict__ x, const float4* __restrict__ pix, int N, int G, int logG, int P,
              int wstack, const float2* __restrict__ tw, const int* __restrict__ active_rows, int n_active,
              float2* __restrict__ Xt) {
  extern __shared__ float2 sm[];
  float2* A = sm;
  float2* B = sm + DG_R1 * G;
  float2* T = sm + 2 * DG_R1 * G;
  for (int k = threadIdx.x; k < G; k += blockDim.x) T[k] = tw[k];
  const int i0 = blockIdx.x * DG_R1;
  const int rows = min(DG_R1, N - i0);
  const int mask = G - 1, hN = N >> 1;
  for (int q = 0; q < P; ++q) {
    for (int e = threadIdx.x; e < DG_R1 * G; e += blockDim.x) A[e] = make_float2(0.f, 0.f);
    __syncthreads();
    const float qf = (float)q;
    for (int e = threadIdx.x; e < rows * N; e += blockDim.x) {
      const int r = e / N, j = e - r * N;
      const size_t p = (size_t)(i0 + r) * N + j;
      const float4 pt = pix[p];
      float2 c = make_float2(pt.x, pt.y);
      if (wstack) {
        // q t in turns, t = t_hi + t_lo, reduced exactly before sincospi (as the epilogue)
        const float pp = qf * pt.z;
        const float ee = fmaf(qf, pt.z, -pp) + qf * pt.w;
        const float th = (pp - rintf(pp)) + ee;
        float sn, cs;
        sincospif(2.0f * th, &sn, &cs);
        c = cmul(c, make_float2(cs, sn));
      }
      const float xv = x[p];
      // conj of the forward-FFT input conj(c) e^{-j 2 pi q t} x: the inverse FFT below
      A[r * G + ((j - hN + G) & mask)] = make_float2(c.x * xv, c.y * xv);
    }
    __syncthreads();
    const float2* res = fft_rows_smem(A, B, rows, G, logG, G, T);
    for (int e = threadIdx.x; e < n_active * rows; e += blockDim.x) {
      const int ar = e / rows, r = e - ar * rows;
      const int b = active_rows[ar];
      Xt[((size_t)q * n_active + ar) * N + i0 + r] = conj2(res[r * G + b]);
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256)
k_degrid_rows(const float2* __restrict__ Xt, int N, int G, int logG, int R, const float2* __restrict__ tw,
              const int* __restrict__ active_rows, int n_active, float2* __restrict__ grid) {
  extern __shared__ float2 sm[];
  const int S = G + 1;
  float2* A = sm;
  float2* B = sm + R * S;
  float2* T = B + R * S;
  for (int k = threadIdx.x; k < G; k += blockDim.x) T[k] = tw[k];
  const int q = blockIdx.y;
  const int ar0 = blockIdx.x * R;
  const int rows = min(R, n_active - ar0);
  const int mask = G - 1, hN = N >> 1;
  for (int e = threadIdx.x; e < R * S; e += blockDim.x) A[e] = make_float2(0.f, 0.f);
  __syncthreads();
  for (int e = threadIdx.x; e < rows * N; e += blockDim.x) {
    const int r = e / N, i = e - r * N;
    A[r * S + ((i - hN + G) & mask)] = conj2(Xt[((size_t)q * n_active + ar0 + r) * N + i]);
  }
  __syncthreads();
  const float2* res = fft_rows_smem(A, B, rows, G, logG, S, T);
  for (int e = threadIdx.x; e < rows * G; e += blockDim.x) {
    const int r = e / G, a = e - r * G;
    grid[((size_t)q * G + active_rows[ar0 + r]) * G + a] = conj2(res[r * S + a]);
  }
}

// Pass 1 on one-warp FFTs: a CTA takes 8 image rows of one plane, one per
// warp; each row's transform is staged in its warp's buffer and the CTA
// writes the reachable rows b as 64-byte runs Xt_q[b][i0 .. i0 + 8).
template <int L>
__global__ void __launch_bounds__(256, 2)
k_degrid_cols_w(const float* __restrict__ x, const float4* __restrict__ pix, int N, int wstack,
                const float2* __restrict__ T2, const int* __restrict__ active_rows, int n_active,
                float2* __restrict__ Xt) {
  constexpr int G = 32 * L, WB = wfft::Shape<L>::buf;
  extern __shared__ float2 bufs[];                  // 8 warps x WB
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = blockIdx.y, i0 = blockIdx.x * 8, i = i0 + warp;
  const int hN = N >> 1;
  const float qf = (float)q;
  float2 v[L];
#pragma unroll
  for (int m = 0; m < L; ++m) {
    const int j = (lane + 32 * m + hN) & (G - 1);     // pixel at row position lane + 32 m
    v[m] = make_float2(0.f, 0.f);
    if (i < N && j < N) {
      const size_t p = (size_t)i * N + j;
      const float4 pt = pix[p];
      float2 c = make_float2(pt.x, pt.y);
      if (wstack) {
        // q t in turns, t = t_hi + t_lo, reduced exactly to [-1/2, 1/2] (as the
        // one-warp epilogue; the fast sine and cosine are accurate to ~4e-7 there)
        const float pp = qf * pt.z;
        const float ee = fmaf(qf, pt.z, -pp) + qf * pt.w;
        const float th = (pp - rintf(pp)) + ee;
        float sn, cs;
        __sincosf(6.283185307179586f * th, &sn, &cs);
        c = cmul(c, make_float2(cs, sn));
      }
      const float xv = x[p];
      // conj of the forward-FFT input conj(c) e^{-j 2 pi q t} x: inverse FFT below
      v[m] = make_float2(c.x * xv, c.y * xv);
    }
  }
  float2* buf = bufs + warp * WB;
  wfft::fft<L>(v, buf, T2, lane);
  // every output frequency: L = 32 lane + 32 k2; L = 16 (lane >> 1) + 16 k' + 256 (lane & 1)
#pragma unroll
  for (int k = 0; k < L; ++k) {
    const int f = (L == 32) ? lane + 32 * k : (lane >> 1) + 16 * k + 256 * (lane & 1);
    buf[f] = v[wfft::brev(k, wfft::log2c(L))];
  }
  __syncthreads();
  const int rows = min(8, N - i0);
  for (int e = threadIdx.x; e < n_active * 8; e += 256) {
    const int ar = e >> 3, r = e & 7;
    if (r < rows) Xt[((size_t)q * n_active + ar) * N + i0 + r] = conj2(bufs[r * WB + active_rows[ar]]);
  }
}

// Pass 2 on one-warp FFTs: one warp per (plane, reachable row); the N inputs
// sit on the centre of the length-G row, and the transformed row is stored
// with coalesced 256-byte (L = 32) or 128-byte (L = 16) runs in the 32-column
// groups that hold visibilities (col_mask: the interpolation reads no other).
template <int L>
__global__ void __launch_bounds__(256, 2)
k_degrid_rows_w(const float2* __restrict__ Xt, int N, const float2* __restrict__ T2,
                const int* __restrict__ active_rows, int n_active, uint32_t col_mask,
                float2* __restrict__ grid) {
  constexpr int G = 32 * L, WB = wfft::Shape<L>::buf;
  extern __shared__ float2 bufs[];                  // 8 warps x WB
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = blockIdx.y, ar = blockIdx.x * 8 + warp;
  const int hN = N >> 1;
  float2 v[L];
  const float2* src = Xt + ((size_t)q * n_active + ar) * N;
#pragma unroll
  for (int m = 0; m < L; ++m) {
    const int i = (lane + 32 * m + hN) & (G - 1);
    v[m] = (ar < n_active && i < N) ? conj2(src[i]) : make_float2(0.f, 0.f);
  }
  if (ar >= n_active) return;                       // no block barrier in this kernel
  wfft::fft<L>(v, bufs + warp * WB, T2, lane);
  float2* dst = grid + ((size_t)q * G + active_rows[ar]) * G;
#pragma unroll
  for (int k = 0; k < L; ++k) {
    const int f = (L == 32) ? lane + 32 * k : (lane >> 1) + 16 * k + 256 * (lane & 1);
    if ((col_mask >> (f >> 5)) & 1u) dst[f] = conj2(v[wfft::brev(k, wfft::log2c(L))]);
  }
}

constexpr int DG_T = 32;   // tile side (the plan's)
constexpr int DG_TP = 33;  // padded tile row in shared memory: rows start on different banks

template <int W>
__global__ void __launch_bounds__(256)
k_degrid(const int4* __restrict__ subs, const int2* __restrict__ slot_vis, const float4* __restrict__ slot_geom,
         const float2* __restrict__ grid, int G, int nT, int P, int Qg, float beta, int wstack,
         float2* __restrict__ y) {
  extern __shared__ float2 tile[];   // [Q][32][33] (row padded)
  const int4 sub = subs[blockIdx.x];
  const int tu = sub.x % nT, tv = sub.x / nT;
  const int q0 = sub.y * Qg;
  const int Q = min(Qg, P - q0);
  for (int e = threadIdx.x; e < Q * DG_T * DG_T; e += blockDim.x) {
    const int q = e / (DG_T * DG_T), rem = e - q * DG_T * DG_T;
    const int bb = rem / DG_T, aa = rem - bb * DG_T;
    tile[(q * DG_T + bb) * DG_TP + aa] = grid[((size_t)(q0 + q) * G + tv * DG_T + bb) * G + tu * DG_T + aa];
  }
  __syncthreads();
  const float two_over_w = 2.0f / W;
  for (int j = sub.z + threadIdx.x; j < sub.w; j += blockDim.x) {
    const int2 sv = slot_vis[j];
    const float4 gm = slot_geom[j];
    const int a0 = (sv.y & 0xff) - 64, b0 = ((sv.y >> 8) & 0xff) - 64, ps = sv.y >> 16;
    float fu[W], fv[W];
#pragma unroll
    for (int c = 0; c < W; ++c) {
      fu[c] = es_kernel((c - gm.x) * two_over_w, beta);
      fv[c] = es_kernel((c - gm.y) * two_over_w, beta);
    }
    float re = 0.f, im = 0.f;
    for (int q = 0; q < Q; ++q) {
      const int cw = q0 + q - ps;
      float fw = 1.f;
      if (wstack) {
        if (cw < 0 || cw >= W) continue;
        fw = es_kernel((cw - gm.z) * two_over_w, beta);
      }
      const float2* tq = tile + q * DG_T * DG_TP;
      float pr = 0.f, pi = 0.f;
#pragma unroll
      for (int jb = 0; jb < W; ++jb) {
        const int b = b0 + jb;
        if (b < 0 || b >= DG_T) continue;
        float rr = 0.f, ri = 0.f;
#pragma unroll
        for (int ia = 0; ia < W; ++ia) {
          const int a = a0 + ia;
          if (a < 0 || a >= DG_T) continue;
          const float2 g = tq[b * DG_TP + a];
          rr = fmaf(fu[ia], g.x, rr);
          ri = fmaf(fu[ia], g.y, ri);
        }
        pr = fmaf(fv[jb], rr, pr);
        pi = fmaf(fv[jb], ri, pi);
      }
      re = fmaf(fw, pr, re);
      im = fmaf(fw, pi, im);
    }
    if (re == 0.f && im == 0.f) continue;
    float2 v = make_float2(re, im);
    if (wstack) {
      float sn, cs;
      sincospif(2.0f * gm.w, &sn, &cs);
      v = cmul(v, make_float2(cs, -sn));      // e^{-j 2 pi tau}
    }
    atomicAdd(&y[sv.x].x, v.x);
    atomicAdd(&y[sv.x].y, v.y);
  }
}

}  // namespace

// The two FFT passes of the degridding (image -> grid planes): class
// "degrid_fft"; the interpolation is timed as "degrid".
static int degrid_ffts(pc_plan_s* p, const float* img, cudaStream_t st) {
  ProfScope prof_scope_(PROF_DEGRID_FFT, st);
  const int N = p->N, G = p->G, n_act = p->n_active_rows;
  const int ws = p->wstack ? 1 : 0;
  if (fft_big_size(G) && p->fft_warp != 0) {
    // one-CTA transforms (fft_big.cu) for G = 2048 .. 8192
    PC_TRY(launch_degrid_ffts_big(p, img, st));
  } else {
  PC_TRY(p->degrid_buf.ensure(sizeof(float2) * (size_t)p->P * n_act * N));
  float2* Xt = p->degrid_buf.as<float2>();
  if (fft_cols_warp(p)) {
    // one-warp FFTs for both passes (the plan's choice for its second FFT pass)
    const int L = G / 32;
    const size_t smem = 8 * (size_t)(L == 32 ? wfft::Shape<32>::buf : wfft::Shape<16>::buf) * sizeof(float2);
    dim3 g1(ceil_div(N, 8), p->P), g2(ceil_div(n_act, 8), p->P);
    if (L == 32) {
      static bool attr = false;
      if (!attr) {
        PC_CUDA(cudaFuncSetAttribute(k_degrid_cols_w<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        PC_CUDA(cudaFuncSetAttribute(k_degrid_rows_w<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr = true;
      }
      k_degrid_cols_w<32><<<g1, 256, smem, st>>>(img, p->pix_tab, N, ws, p->tw2, p->active_rows, n_act, Xt);
      PC_LAUNCH_CHECK();
      k_degrid_rows_w<32><<<g2, 256, smem, st>>>(Xt, N, p->tw2, p->active_rows, n_act, p->col_mask,
                                                    p->grid);
      PC_LAUNCH_CHECK();
    } else {
      static bool attr = false;
      if (!attr) {
        PC_CUDA(cudaFuncSetAttribute(k_degrid_cols_w<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        PC_CUDA(cudaFuncSetAttribute(k_degrid_rows_w<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr = true;
      }
      k_degrid_cols_w<16><<<g1, 256, smem, st>>>(img, p->pix_tab, N, ws, p->tw2, p->active_rows, n_act, Xt);
      PC_LAUNCH_CHECK();
      k_degrid_rows_w<16><<<g2, 256, smem, st>>>(Xt, N, p->tw2, p->active_rows, n_act, p->col_mask,
                                                    p->grid);
      PC_LAUNCH_CHECK();
    }
  } else {
  {
    const size_t smem = ((size_t)2 * DG_R1 * G + G) * sizeof(float2);
    if (smem > 200 * 1024) return fail(PC_ERR_INVALID_ARG, "forward: grid side %d too large for degridding", G);
    static bool attr = false;
    if (!attr) {
      PC_CUDA(cudaFuncSetAttribute(k_degrid_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
      attr = true;
    }
    k_degrid_cols<<<ceil_div(N, DG_R1), 256, smem, st>>>(img, p->pix_tab, N, G, p->logG, p->P, ws, p->twiddle,
                                                          p->active_rows, n_act, Xt);
    PC_LAUNCH_CHECK();
  }
  {
    int R = 1;
    while (R < 4 && ((size_t)2 * (2 * R) * (G + 1) + G) * sizeof(float2) <= 200 * 1024) R *= 2;
    const size_t smem = ((size_t)2 * R * (G + 1) + G) * sizeof(float2);
    static bool attr = false;
    if (!attr) {
      PC_CUDA(cudaFuncSetAttribute(k_degrid_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
      attr = true;
    }
    dim3 grid(ceil_div(n_act, R), p->P);
    k_degrid_rows<<<grid, 256, smem, st>>>(Xt, N, G, p->logG, R, p->twiddle, p->active_rows, n_act, p->grid);
    PC_LAUNCH_CHECK();
  }
  }
  }
  prof_scope_.kernels = 2;
  return PC_OK;
}

int forward_grid_impl(pc_plan_s* p, const float* img, float2* y, cudaStream_t st) {
  if (p->M <= 0) return PC_OK;
  if (p->n_sub == 0 || p->n_active_rows == 0) {
    ProfScope prof_scope_(PROF_DEGRID, st);
    PC_CUDA(cudaMemsetAsync(y, 0, sizeof(float2) * (size_t)p->M, st));
    prof_scope_.kernels = 1;
    return PC_OK;
  }
  PC_TRY(degrid_ffts(p, img, st));
  ProfScope prof_scope_(PROF_DEGRID, st);
  PC_CUDA(cudaMemsetAsync(y, 0, sizeof(float2) * (size_t)p->M, st));
  const int G = p->G, ws = p->wstack ? 1 : 0;
  if (grid_win_mode(p)) {
    PC_TRY(launch_degrid_win(p, y, st));
  } else {
    if (p->T != DG_T || p->Qg > 8) return fail(PC_ERR_INVALID_ARG, "forward: needs 32-cell tiles, <= 8 planes");
    const size_t smem = sizeof(float2) * (size_t)p->Qg * DG_T * DG_TP;
    const float beta = (float)p->beta;
#define PC_DEGRID_CASE(WW)                                                                              \
  case WW: {                                                                                            \
    static bool attr = false;                                                                           \
    if (!attr) {                                                                                        \
      PC_CUDA(cudaFuncSetAttribute(k_degrid<WW>, cudaFuncAttributeMaxDynamicSharedMemorySize,            \
                                   (int)(sizeof(float2) * 8 * DG_T * DG_TP)));                         \
      attr = true;                                                                                      \
    }                                                                                                   \
    k_degrid<WW><<<p->n_sub, 256, smem, st>>>(p->subs, p->slot_vis, p->slot_geom, p->grid, G, p->nT, p->P, \
                                              p->Qg, beta, ws, y);                                      \
    break;                                                                                              \
  }
    switch (p->W) {
      PC_DEGRID_CASE(4)
      PC_DEGRID_CASE(5)
      PC_DEGRID_CASE(6)
      PC_DEGRID_CASE(7)
      PC_DEGRID_CASE(8)
      default:
        return fail(PC_ERR_INVALID_ARG, "forward: unsupported kernel width %d", p->W);
    }
#undef PC_DEGRID_CASE
    PC_LAUNCH_CHECK();
  }
  prof_scope_.kernels = 2;
  return PC_OK;
}

}  // namespace pc

using namespace pc;

extern "C" int pc_forward_grid(pc_plan_t p, const float* img, pc_c32* y, void* stream) {
  clear_error();
  if (!p) return fail(PC_ERR_INVALID_ARG, "pc_forward_grid: NULL plan");
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != p->device) return fail(PC_ERR_INVALID_ARG, "pc_forward_grid: plan was built on another device");
  if (!is_device_ptr(img)) return fail(PC_ERR_INVALID_ARG, "pc_forward_grid: img_dev is not a device pointer");
  if (p->M > 0 && !is_device_ptr(y)) return fail(PC_ERR_INVALID_ARG, "pc_forward_grid: y_dev is not a device pointer");
  return forward_grid_impl(p, img, reinterpret_cast<float2*>(y), static_cast<cudaStream_t>(stream));
}
