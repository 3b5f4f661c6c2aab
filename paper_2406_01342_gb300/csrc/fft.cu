// Pruned 2-D inverse FFT of every w-plane and the image-domain epilogue.
//
// After gridding, plane q holds grid_q[b][a] (a contiguous). The adjoint
// needs, for image pixel (i, j) with i' = i - N/2, j' = j - N/2,
//
//   F_q[i'][j'] = sum_{a,b} grid_q[b][a] e^{+j 2 pi (a i' + b j') / G}
//   mu[i][j]    = Re{ c_ij sum_q e^{+j 2 pi q t_ij} F_q[i'][j'] } * scale
//
// with c_ij = e^{j 2 pi w0 s_ij} / (n_ij psi(i'/G) psi(j'/G) psi(t_ij)),
// t_ij = dw (s_ij - s_c), s = n - 1 (the w-screen of Sect. 2.1 and the
// 1/n of the adjoint equation of Sect. 2.2); scale = 1/lambda for the
// certificate of Sect. 4.2.
//
// Pass 1 (k_fft_rows): for each plane and row b, a length-G inverse FFT
// along a, keeping the N outputs i' in [-N/2, N/2), stored transposed as
// X_q[i][b] so that pass 2 reads contiguous rows.
// Pass 2 (k_fft_cols): one CTA per image row i; for every plane a length-G
// inverse FFT along b, keep N outputs, apply the plane phase and accumulate
// in registers; then the per-pixel correction, write mu and its max |mu|.
// Where G is 512 or 1024 both passes give each row to one warp, which holds
// it in registers (fft_warp.cuh): no block-wide barrier inside a transform.
// Otherwise, and where the autotuner measured it faster, they run radix-4
// (plus one radix-2) Stockham stages in shared memory with a twiddle table
// e^{+2 pi i k / G}.
#include "pc_internal.cuh"
#include "fft.cuh"
#include "fft_warp.cuh"

namespace pc {

__global__ void __launch_bounds__(256)
k_fft_rows(const float2* __restrict__ grid, float2* __restrict__ X, int G, int logG, int N, int R,
           const float2* __restrict__ tw, const int* __restrict__ active_rows) {
  extern __shared__ float2 sm[];
  const int S = G + 1;
  float2* A = sm;
  float2* B = sm + R * S;
  float2* T = B + R * S;                          // twiddles, staged once per CTA
  for (int k = threadIdx.x; k < G; k += blockDim.x) T[k] = tw[k];
  const int q = blockIdx.y;
  const int b0 = active_rows[blockIdx.x * R];     // R consecutive active rows (R divides 32)
  const float2* src = grid + ((size_t)q * G + b0) * G;
  for (int f = threadIdx.x; f < R * G; f += blockDim.x) {
    const int r = f / G, a = f - r * G;
    A[r * S + a] = src[(size_t)r * G + a];
  }
  __syncthreads();
  const float2* res = fft_rows_smem(A, B, R, G, logG, S, T);
  float2* dst = X + (size_t)q * N * G + b0;
  const int mask = G - 1, hN = N >> 1;
  for (int f = threadIdx.x; f < N * R; f += blockDim.x) {
    const int i = f / R, r = f - i * R;
    dst[(size_t)i * G + r] = res[r * S + ((i - hN + G) & mask)];
  }
}

// Pass 1 on one-warp FFTs: a CTA takes 8 consecutive active rows of one
// plane, one per warp, and writes the N kept outputs of each, staged in the
// warps' buffers, as 64-byte runs X_q[i][b0 .. b0 + 8). Only the 32-column
// groups that can hold data (col_mask) are read; the rest of a row is zero.
template <int L>
__global__ void __launch_bounds__(256, 2)
k_fft_rows_w(const float2* __restrict__ grid, float2* __restrict__ X, int N,
             const float2* __restrict__ T2, const int* __restrict__ active_rows, uint32_t col_mask) {
  constexpr int G = 32 * L, WB = wfft::Shape<L>::buf;
  extern __shared__ float2 bufs[];                 // 8 warps x WB
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = blockIdx.y;
  const int b0 = active_rows[blockIdx.x * 8];     // 8 consecutive active rows (8 divides 32)
  const float2* src = grid + ((size_t)q * G + b0 + warp) * G + lane;
  float2 v[L];
#pragma unroll
  for (int m = 0; m < L; ++m) v[m] = ((col_mask >> m) & 1u) ? src[32 * m] : make_float2(0.f, 0.f);
  float2* buf = bufs + warp * WB;
  wfft::fft<L>(v, buf, T2, lane);
  const int hN = N >> 1;
#pragma unroll
  for (int c = 0; c < wfft::Shape<L>::kept; ++c) {
    const int i = (wfft::kept_freq<L>(c, lane) + hN) & (G - 1);
    if (i < N) buf[i] = wfft::kept_value<L>(v, c, lane);
  }
  __syncthreads();
  float2* dst = X + (size_t)q * N * G + b0;
  for (int e = threadIdx.x; e < N * 8; e += 256) {
    const int i = e >> 3, r = e & 7;
    dst[(size_t)i * G + r] = bufs[r * WB + i];
  }
}

// Pass 2 on one-warp FFTs: a CTA takes 8 / WPR image rows, WPR warps per
// row; warp w of a row transforms planes w, w + WPR, ... (reading only the
// 32-entry groups of reachable grid rows, row_mask) and sums the
// plane-phased kept outputs (ONE: exactly one plane per warp, written
// straight to its buffer; else running sums in shared memory). The rows' w-screen turns are staged in shared
// memory while the first loads are in flight. The warps' partial sums meet in
// shared memory, are added in warp order and get the per-pixel correction.
template <int L>
__device__ __forceinline__ float2 plane_phased(float2 val, float2 t, float qf, bool wstack) {
  if (!wstack) return val;
  // q t in turns, with t = t_hi + t_lo, reduced exactly to [-1/2, 1/2]
  // (the fast sine and cosine are accurate to ~4e-7 absolute there)
  const float p = qf * t.x;
  const float e = fmaf(qf, t.x, -p) + qf * t.y;
  const float th = (p - rintf(p)) + e;
  float sn, cs;
  __sincosf(6.283185307179586f * th, &sn, &cs);
  return make_float2(val.x * cs - val.y * sn, val.x * sn + val.y * cs);
}

template <int L, bool ONE>
__global__ void __launch_bounds__(256, 2)
k_fft_cols_w(const float2* __restrict__ X, const float4* __restrict__ pix, float* __restrict__ mu, int N,
             int P, int WPR, int wstack, const float2* __restrict__ T2, uint32_t row_mask, float scale,
             unsigned* __restrict__ maxbits) {
  constexpr int G = 32 * L, WB = wfft::Shape<L>::buf, KEPT = wfft::Shape<L>::kept;
  extern __shared__ float2 sm[];
  float2* bufs = sm;                              // 8 warps x WB
  float2* tz = sm + 8 * WB;                       // (t_hi, t_lo) of the CTA's rows, RPC x N
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int RPC = 8 / WPR;
  const int i = blockIdx.x * RPC + warp / WPR;
  const int hN = N >> 1;
  float2* buf = bufs + warp * WB;
  int q = warp % WPR;
  float2 v[L];
  const bool live = i < N && q < P;
  if (live) {
    const float2* src = X + ((size_t)q * N + i) * G + lane;
#pragma unroll
    for (int m = 0; m < L; ++m) v[m] = ((row_mask >> m) & 1u) ? src[32 * m] : make_float2(0.f, 0.f);
  }
  if (wstack) {
    const int i0 = blockIdx.x * RPC;
    for (int e = threadIdx.x; e < RPC * N; e += 256) {
      if (i0 + e / N < N) {
        const float4 pt = pix[(size_t)i0 * N + e];
        tz[e] = make_float2(pt.z, pt.w);
      }
    }
  }
  __syncthreads();                                // turns staged
  const float2* tzr = tz + (size_t)(warp / WPR) * N;
  if (ONE) {
    if (live) {
      wfft::fft<L>(v, buf, T2, lane);
      const float qf = (float)q;
#pragma unroll
      for (int c = 0; c < KEPT; ++c) {
        const int j = (wfft::kept_freq<L>(c, lane) + hN) & (G - 1);
        if (j < N) buf[j] = plane_phased<L>(wfft::kept_value<L>(v, c, lane), wstack ? tzr[j] : make_float2(0.f, 0.f),
                                            qf, wstack);
      }
    } else {
      for (int j = lane; j < N; j += 32) buf[j] = make_float2(0.f, 0.f);
    }
  } else {
    // several planes per warp: the running sums live in the warp's own N
    // entries after the turns (each lane owns its pixels: no races)
    float2* acc = tz + (size_t)RPC * N + (size_t)warp * N;
    for (int j = lane; j < N; j += 32) acc[j] = make_float2(0.f, 0.f);
    __syncwarp();
    if (live) {
      for (;;) {
        wfft::fft<L>(v, buf, T2, lane);
        const float qf = (float)q;
#pragma unroll
        for (int c = 0; c < KEPT; ++c) {
          const int j = (wfft::kept_freq<L>(c, lane) + hN) & (G - 1);
          if (j < N) {
            const float2 pv = plane_phased<L>(wfft::kept_value<L>(v, c, lane),
                                              wstack ? tzr[j] : make_float2(0.f, 0.f), qf, wstack);
            acc[j].x += pv.x;
            acc[j].y += pv.y;
          }
        }
        q += WPR;
        if (q >= P) break;
        const float2* src = X + ((size_t)q * N + i) * G + lane;
#pragma unroll
        for (int m = 0; m < L; ++m) v[m] = ((row_mask >> m) & 1u) ? src[32 * m] : make_float2(0.f, 0.f);
      }
    }
  }
  __syncthreads();
  // partial sums of warp w at part + w * pstride
  const float2* part = ONE ? bufs : tz + (size_t)RPC * N;
  const int pstride = ONE ? WB : N;
  float amax = 0.0f;
  unsigned skey = 0;   // order-preserving key of the signed maximum (0 below every number)
  for (int e = threadIdx.x; e < RPC * N; e += 256) {
    const int r = e / N, j = e - r * N;
    const int ii = blockIdx.x * RPC + r;
    if (ii >= N) continue;
    const float2* pb = part + (size_t)r * WPR * pstride + j;
    float2 s = pb[0];
    for (int w = 1; w < WPR; ++w) {
      s.x += pb[w * pstride].x;
      s.y += pb[w * pstride].y;
    }
    const float4 pt = pix[(size_t)ii * N + j];
    const float m = (pt.x * s.x - pt.y * s.y) * scale;
    mu[(size_t)ii * N + j] = m;
    amax = fmaxf(amax, fabsf(m));
    if (m != m) amax = __int_as_float(0x7fc00000);
    skey = max(skey, float_order_key(m));
  }
  unsigned bits = __float_as_uint(amax);
  for (int off = 16; off; off >>= 1) {
    bits = max(bits, __shfl_xor_sync(0xffffffffu, bits, off));
    skey = max(skey, __shfl_xor_sync(0xffffffffu, skey, off));
  }
  if (lane == 0 && maxbits) {
    atomicMax(maxbits, bits);
    atomicMax(maxbits + 1, skey);
  }
}

template <int JPT>
__global__ void __launch_bounds__(256)
k_fft_cols(const float2* __restrict__ X, const float4* __restrict__ pix, float* __restrict__ mu,
           int G, int logG, int N, int P, int PG, int wstack, const float2* __restrict__ tw, float scale,
           unsigned* __restrict__ maxbits) {
  extern __shared__ float2 sm[];
  float2* A = sm;                                 // PG planes' rows at a time
  float2* B = sm + (size_t)PG * G;
  float2* T = sm + 2 * (size_t)PG * G;            // twiddles, staged once per CTA
  for (int k = threadIdx.x; k < G; k += blockDim.x) T[k] = tw[k];
  const int i = blockIdx.x;
  const int mask = G - 1, hN = N >> 1;
  float2 acc[JPT];
  float4 pt[JPT];
#pragma unroll
  for (int jj = 0; jj < JPT; ++jj) {
    acc[jj] = make_float2(0.f, 0.f);
    const int j = threadIdx.x + jj * blockDim.x;
    pt[jj] = j < N ? pix[(size_t)i * N + j] : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  for (int q0 = 0; q0 < P; q0 += PG) {
    // rows of PG planes loaded and transformed together: fewer barriers per
    // plane and PG independent loads in flight
    const int Qn = min(PG, P - q0);
    for (int e = threadIdx.x; e < Qn * G; e += blockDim.x) {
      const int r = e / G, a = e - r * G;
      A[e] = X[((size_t)(q0 + r) * N + i) * G + a];
    }
    __syncthreads();
    const float2* res = fft_rows_smem(A, B, Qn, G, logG, G, T);
    for (int r = 0; r < Qn; ++r) {
    const float qf = (float)(q0 + r);
#pragma unroll
    for (int jj = 0; jj < JPT; ++jj) {
      const int j = threadIdx.x + jj * blockDim.x;
      if (j < N) {
        const float2 v = res[(size_t)r * G + ((j - hN + G) & mask)];
        if (wstack) {
          // q t in turns, with t = t_hi + t_lo, reduced exactly before sincospi
          const float p = qf * pt[jj].z;
          const float e = fmaf(qf, pt[jj].z, -p) + qf * pt[jj].w;
          const float th = (p - rintf(p)) + e;
          float sn, cs;
          sincospif(2.0f * th, &sn, &cs);
          acc[jj].x += v.x * cs - v.y * sn;
          acc[jj].y += v.x * sn + v.y * cs;
        } else {
          acc[jj].x += v.x;
          acc[jj].y += v.y;
        }
      }
    }
    }
    __syncthreads();
  }
  float amax = 0.0f;
  unsigned skey = 0;   // order-preserving key of the signed maximum (0 below every number)
#pragma unroll
  for (int jj = 0; jj < JPT; ++jj) {
    const int j = threadIdx.x + jj * blockDim.x;
    if (j < N) {
      const float m = (pt[jj].x * acc[jj].x - pt[jj].y * acc[jj].y) * scale;
      mu[(size_t)i * N + j] = m;
      amax = fmaxf(amax, fabsf(m));
      if (m != m) amax = __int_as_float(0x7fc00000);
      skey = max(skey, float_order_key(m));
    }
  }
  unsigned bits = __float_as_uint(amax);
  for (int off = 16; off; off >>= 1) {
    bits = max(bits, __shfl_xor_sync(0xffffffffu, bits, off));
    skey = max(skey, __shfl_xor_sync(0xffffffffu, skey, off));
  }
  if ((threadIdx.x & 31) == 0 && maxbits) {
    atomicMax(maxbits, bits);
    atomicMax(maxbits + 1, skey);
  }
}

namespace {

bool warp_fft_size(int G) { return G == 512 || G == 1024; }

// the 8 warps' buffers, plus (second pass) the w-screen turns of the CTA's rows
size_t warp_fft_smem(int G, int turns = 0) {
  const int WB = G == 1024 ? wfft::Shape<32>::buf : wfft::Shape<16>::buf;
  return (8 * (size_t)WB + (size_t)turns) * sizeof(float2);
}

// opt in once to the shared memory any plan's launch may ask for
template <typename K>
int allow_smem(K* kernel, bool& done) {
  if (!done) {
    PC_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    done = true;
  }
  return PC_OK;
}

}  // namespace

bool fft_rows_warp(const pc_plan_s* p) {
  return warp_fft_size(p->G) && (p->fft_warp < 0 || (p->fft_warp & 1));
}

bool fft_cols_warp(const pc_plan_s* p) {
  return warp_fft_size(p->G) && (p->fft_warp < 0 || (p->fft_warp & 2));
}

int launch_fft_rows(pc_plan_s* p, cudaStream_t st) {
  ProfScope prof_scope_(PROF_FFT_ROWS, st);
  if (p->n_active_rows == 0) return PC_OK;     // all-zero grid: the output stays zero
  if (fft_rows_big(p)) {
    prof_scope_.kernels = 1;
    return launch_fft_rows_big(p, st);
  }
  if (fft_rows_warp(p)) {
    const size_t smem = warp_fft_smem(p->G);
    dim3 grid(p->n_active_rows / 8, p->P);
    prof_scope_.kernels = 1;
    if (p->G == 1024) {
      static bool done = false;
      PC_TRY(allow_smem(k_fft_rows_w<32>, done));
      k_fft_rows_w<32><<<grid, 256, smem, st>>>(p->grid, p->fft1, p->N, p->tw2, p->active_rows, p->col_mask);
    } else {
      static bool done = false;
      PC_TRY(allow_smem(k_fft_rows_w<16>, done));
      k_fft_rows_w<16><<<grid, 256, smem, st>>>(p->grid, p->fft1, p->N, p->tw2, p->active_rows, p->col_mask);
    }
    PC_LAUNCH_CHECK();
    return PC_OK;
  }
  // rows per CTA (default): R * (G + 1) * 8 bytes * 2 buffers ~ 33 KB;
  // R divides the 32-row tile so a CTA's rows are consecutive active rows
  int R = p->fft_R > 0 ? p->fft_R : 2048 / p->G;
  if (R < 1) R = 1;
  if (R > 32) R = 32;
  const size_t smem = ((size_t)2 * R * (p->G + 1) + p->G) * sizeof(float2);
  if (smem > 200 * 1024) return fail(PC_ERR_INVALID_ARG, "fft: %d rows per CTA do not fit shared memory", R);
  static bool attr_set = false;
  if (!attr_set) {
    PC_CUDA(cudaFuncSetAttribute(k_fft_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr_set = true;
  }
  dim3 grid(p->n_active_rows / R, p->P);
  prof_scope_.kernels = 1;
  k_fft_rows<<<grid, 256, smem, st>>>(p->grid, p->fft1, p->G, p->logG, p->N, R, p->twiddle,
                                      p->active_rows);
  PC_LAUNCH_CHECK();
  return PC_OK;
}

// Planes per pass of the second FFT pass: the plan's choice (autotuner), else
// 2 (five CTAs per SM at G = 1024), never more than shared memory holds.
int cols_planes_per_pass(const pc_plan_s* p) {
  int pg = p->fft_cols_pg > 0 ? p->fft_cols_pg : 2;
  pg = std::min(pg, p->P);
  while (pg > 1 && ((size_t)2 * pg * p->G + p->G) * sizeof(float2) > 200 * 1024) --pg;
  return std::max(pg, 1);
}

int launch_fft_cols_epilogue(pc_plan_s* p, float* mu, float scale, unsigned* maxbits,
                             cudaStream_t st) {
  ProfScope prof_scope_(PROF_FFT_COLS, st);
  if (fft_cols_big(p)) {
    if (p->n_active_rows == 0) {                // nothing reaches the grid: mu = 0
      PC_CUDA(cudaMemsetAsync(mu, 0, sizeof(float) * (size_t)p->N * p->N, st));
      return PC_OK;
    }
    prof_scope_.kernels = 1;
    return launch_fft_cols_big(p, mu, scale, maxbits, st);
  }
  if (fft_cols_warp(p)) {
    int wpr = 8;                                   // warps per image row: a power of 2 <= P
    while (wpr > p->P) wpr >>= 1;
    const int rpc = 8 / wpr;
    const int ws = p->wstack ? 1 : 0;
    const bool one = wpr == p->P;                  // every warp exactly one plane
    // turns of the CTA's rows; with several planes per warp also 8 running sums of N
    const size_t smem = warp_fft_smem(p->G, one ? (ws ? rpc * p->N : 0) : rpc * p->N + 8 * p->N);
    prof_scope_.kernels = 1;
    const unsigned nb = (unsigned)ceil_div(p->N, rpc);
#define PC_COLS_W(LL, ONE)                                                                        \
  {                                                                                               \
    static bool done = false;                                                                     \
    PC_TRY(allow_smem(k_fft_cols_w<LL, ONE>, done));                                              \
    k_fft_cols_w<LL, ONE><<<nb, 256, smem, st>>>(p->fft1, p->pix_tab, mu, p->N, p->P, wpr, ws,   \
                                                 p->tw2, p->row_mask, scale, maxbits);            \
  }
    if (p->G == 1024) {
      if (one) PC_COLS_W(32, true) else PC_COLS_W(32, false)
    } else {
      if (one) PC_COLS_W(16, true) else PC_COLS_W(16, false)
    }
#undef PC_COLS_W
    PC_LAUNCH_CHECK();
    return PC_OK;
  }
  const int PG = cols_planes_per_pass(p);
  const size_t smem = ((size_t)2 * PG * p->G + p->G) * sizeof(float2);
  const int jpt = (p->N + 255) / 256;
  prof_scope_.kernels = 1;
  const int ws = p->wstack ? 1 : 0;
#define PC_COLS_CASE(J)                                                                         \
  case J: {                                                                                     \
    static bool attr_set = false;                                                               \
    if (!attr_set) {                                                                            \
      PC_CUDA(cudaFuncSetAttribute(k_fft_cols<J>, cudaFuncAttributeMaxDynamicSharedMemorySize,  \
                                   200 * 1024));                                                \
      attr_set = true;                                                                          \
    }                                                                                           \
    k_fft_cols<J><<<p->N, 256, smem, st>>>(p->fft1, p->pix_tab, mu, p->G, p->logG, p->N, p->P,  \
                                           PG, ws, p->twiddle, scale, maxbits);                 \
    break;                                                                                      \
  }
  switch (jpt) {
    PC_COLS_CASE(1)
    PC_COLS_CASE(2)
    case 3:
    PC_COLS_CASE(4)
    case 5: case 6: case 7:
    PC_COLS_CASE(8)
    case 9: case 10: case 11: case 12: case 13: case 14: case 15:
    PC_COLS_CASE(16)
    default:
      return fail(PC_ERR_INVALID_ARG, "fft: image side %d too large", p->N);
  }
#undef PC_COLS_CASE
  PC_LAUNCH_CHECK();
  return PC_OK;
}

}  // namespace pc
