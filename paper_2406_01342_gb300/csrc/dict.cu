// Synthesis-form LASSO over a multi-scale Gaussian dictionary (Sect. 4.3; the
// diffuse experiment of Sect. 6):
//
//   argmin_theta 1/2 ||V - Phi Psi theta||^2 + lambda ||theta||_1,
//   Psi theta = sum_i gamma_i g~_i * theta_i,
//   g~_i[n, m] = g1_i[n] g1_i[m],  g1_i[n] = e^{-n^2/sigma_i^2} / sum_n' e^{-n'^2/sigma_i^2},  |n| <= floor(2 sigma_i)
//
// (the normalised 2-D Gaussian of the paper is exactly the product of two
// normalised 1-D factors, which is what makes Psi* separable here).
//
// Kernels:
//   k_dict_corr     eta = Psi* mu on every coefficient: one CTA per 32 x 32
//                   output tile stages mu with a halo of the largest radius in
//                   shared memory, runs the row then the column pass of every
//                   scale and writes the max |eta| / signed max as order keys;
//   k_dict_columns  columns of Phi Psi for the atoms entering the active set:
//                   the direct sum of the measurement operator over the atom's
//                   footprint pixels (same fixed-point phases as the pixel
//                   path), summed row by row of the footprint for accuracy;
//   k_dict_gram     Gram rows Re(C_new^H [C_active | V]) from the cached
//                   columns, FP32 tiles flushed to float64 per K-slice;
//   k_dict_apply    r = V - C_S theta (or y = C_S theta) with ||r||^2 in float64.
//
// The solve keeps the columns of the active set resident (|S| x M complex64),
// so an atom's footprint sum is evaluated once, when it enters the active set;
// the certificate reuses the pixel path's gridding / FFT / epilogue and adds
// the correlation; selection, old positions, APGD and the Gram finalisation
// are the pixel path's kernels over coefficient indices.
#include "solver.cuh"

#include <cmath>

namespace pc {
namespace {

constexpr int DK = PC_DICT_MAX_RADIUS;      // largest kernel radius
constexpr int DTAPS = 2 * DK + 1;

struct DictParams {
  int n_scales;
  int K[PC_DICT_MAX_SCALES];                 // radius floor(2 sigma_i)
  float gamma[PC_DICT_MAX_SCALES];
  float g1[PC_DICT_MAX_SCALES][DTAPS];       // g1[i][n + K_i]
};

int make_params(const pc_dictionary* d, const char* fn, DictParams* out) {
  if (!d) return fail(PC_ERR_INVALID_ARG, "%s: NULL dictionary", fn);
  if (d->version != PC_ABI_VERSION)
    return fail(PC_ERR_INVALID_ARG, "%s: dictionary version %d, library %d", fn, d->version, PC_ABI_VERSION);
  if (d->n_scales < 1 || d->n_scales > PC_DICT_MAX_SCALES)
    return fail(PC_ERR_INVALID_ARG, "%s: n_scales %d not in [1, %d]", fn, d->n_scales, PC_DICT_MAX_SCALES);
  DictParams P{};
  P.n_scales = d->n_scales;
  for (int i = 0; i < d->n_scales; ++i) {
    const double s = d->sigma[i], g = d->gamma[i];
    if (!std::isfinite(s) || s < 0.0 || std::floor(2.0 * s) > DK)
      return fail(PC_ERR_INVALID_ARG, "%s: sigma[%d] = %g outside [0, %g]", fn, i, s, DK / 2.0);
    if (!std::isfinite(g) || !(g > 0.0)) return fail(PC_ERR_INVALID_ARG, "%s: gamma[%d] must be positive", fn, i);
    const int K = s == 0.0 ? 0 : (int)std::floor(2.0 * s);
    P.K[i] = K;
    P.gamma[i] = (float)g;
    double e[DTAPS], sum = 0.0;
    for (int n = -K; n <= K; ++n) {
      e[n + K] = s == 0.0 ? 1.0 : std::exp(-(double)(n * n) / (s * s));
      sum += e[n + K];
    }
    for (int n = 0; n <= 2 * K; ++n) P.g1[i][n] = (float)(e[n] / sum);
  }
  *out = P;
  return PC_OK;
}

inline int round4(int n) { return (n + 3) & ~3; }

// ---------------------------------------------------------------- Psi*

constexpr int CT = 32;             // output tile side
constexpr int CH = CT + 2 * DK;    // staged tile side (with the halo)

__global__ void __launch_bounds__(256)
k_dict_corr(const float* __restrict__ img, int N, const __grid_constant__ DictParams D,
            float* __restrict__ eta, unsigned* __restrict__ maxbits) {
  __shared__ float H[CH][CH + 1];
  __shared__ float T[CH][CT + 1];
  __shared__ float taps[PC_DICT_MAX_SCALES][DTAPS];
  const int x0 = blockIdx.y * CT, y0 = blockIdx.x * CT;
  for (int e = threadIdx.x; e < PC_DICT_MAX_SCALES * DTAPS; e += blockDim.x)
    taps[e / DTAPS][e % DTAPS] = D.g1[e / DTAPS][e % DTAPS];
  for (int e = threadIdx.x; e < CH * CH; e += blockDim.x) {
    const int r = e / CH, c = e - r * CH;
    const int x = x0 - DK + r, y = y0 - DK + c;
    H[r][c] = (x >= 0 && x < N && y >= 0 && y < N) ? img[(size_t)x * N + y] : 0.f;
  }
  __syncthreads();
  const size_t NN = (size_t)N * N;
  float amax = 0.f, smax = -INFINITY;
  for (int i = 0; i < D.n_scales; ++i) {
    const int K = D.K[i];
    const float* g = taps[i];
    // along y: T[r][c] = sum_m g[m] H[r][c + m] for the rows the x pass reads
    const int r0 = DK - K, nr = CT + 2 * K;
    for (int e = threadIdx.x; e < nr * CT; e += blockDim.x) {
      const int r = r0 + e / CT, c = e % CT;
      float s = 0.f;
      for (int m = -K; m <= K; ++m) s = fmaf(g[m + K], H[r][DK + c + m], s);
      T[r][c] = s;
    }
    __syncthreads();
    // along x, times gamma_i
    for (int e = threadIdx.x; e < CT * CT; e += blockDim.x) {
      const int r = e / CT, c = e % CT;
      const int x = x0 + r, y = y0 + c;
      float s = 0.f;
      for (int n = -K; n <= K; ++n) s = fmaf(g[n + K], T[DK + r + n][c], s);
      const float v = D.gamma[i] * s;
      if (x < N && y < N) {
        eta[i * NN + (size_t)x * N + y] = v;
        amax = fmaxf(amax, fabsf(v));
        smax = fmaxf(smax, v);
      }
    }
    __syncthreads();
  }
  for (int off = 16; off; off >>= 1) {
    amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, off));
    smax = fmaxf(smax, __shfl_xor_sync(0xffffffffu, smax, off));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&maxbits[0], __float_as_uint(amax));
    if (smax > -INFINITY) atomicMax(&maxbits[1], float_order_key(smax));
  }
}

// ---------------------------------------------------------------- columns of Phi Psi

__global__ void __launch_bounds__(256)
k_dict_columns(const int4* __restrict__ vis, int64_t M, const int32_t* __restrict__ idx,
               const int32_t* __restrict__ rows, int n_rows, int N, const float4* __restrict__ atom_tab,
               const __grid_constant__ DictParams D, float2* __restrict__ C, int64_t ldc) {
  __shared__ float4 fp[DTAPS * DTAPS];
  const int r = blockIdx.y;
  if (r >= n_rows) return;
  const int slot = rows ? rows[r] : r;
  const int a = idx[slot];
  const int NN = N * N;
  const int i = a / NN, p = a - i * NN;
  const int x0 = p / N, y0 = p - x0 * N;
  const int K = D.K[i], side = 2 * K + 1;
  const float gam = D.gamma[i];
  for (int f = threadIdx.x; f < side * side; f += blockDim.x) {
    const int n = f / side - K, m = f - (f / side) * side - K;
    const int x = x0 + n, y = y0 + m;
    const bool in = x >= 0 && x < N && y >= 0 && y < N;
    const float w = in ? gam * D.g1[i][n + K] * D.g1[i][m + K] : 0.f;
    float4 at = atom_tab[in ? x * N + y : p];                // weight w / n_pixel
    at.w *= w;
    fp[f] = at;
  }
  __syncthreads();
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= M) return;
  const int4 vk = vis[k];
  float re = 0.f, im = 0.f;
  for (int n = 0; n < side; ++n) {          // one footprint row at a time
    float rr = 0.f, ri = 0.f;
    for (int m = 0; m < side; ++m) {
      const float4 at = fp[n * side + m];
      float sn, cs;
      // phase reduced exactly to [-1/2, 1/2] turns: fast sine and cosine
      // accurate to ~4e-7 absolute there (as the other phase kernels)
      __sincosf(6.283185307179586f * phase_turns(vk, at), &sn, &cs);
      rr = fmaf(at.w, cs, rr);
      ri = fmaf(-at.w, sn, ri);
    }
    re += rr;
    im += ri;
  }
  C[(size_t)slot * ldc + k] = make_float2(re, im);
}

// ---------------------------------------------------------------- Gram rows

constexpr int DG_T = 64;      // tile (rows x columns)
constexpr int DG_KC = 32;     // visibilities per staged chunk
constexpr int DG_LD = DG_T + 4;

// acc[r][c] += Re(conj(C[rows[r]]) . B[c]) over one K-slice of ks visibilities,
// B[c] = C[c] (c < n_cols) or V (c == n_cols, when V is given).
__global__ void __launch_bounds__(256)
k_dict_gram(const float2* __restrict__ C, int64_t ldc, int64_t M, int64_t ks, const int32_t* __restrict__ rows,
            int n_rows, int n_cols, const float2* __restrict__ V, double* __restrict__ acc, int ldacc) {
  __shared__ __align__(16) float Ar[DG_KC][DG_LD];
  __shared__ __align__(16) float Ai[DG_KC][DG_LD];
  __shared__ __align__(16) float Br[DG_KC][DG_LD];
  __shared__ __align__(16) float Bi[DG_KC][DG_LD];
  const int a_base = blockIdx.y * DG_T, b_base = blockIdx.x * DG_T;
  const int64_t k_lo = (int64_t)blockIdx.z * ks;
  const int64_t k_hi = min(M, k_lo + ks);
  const int n_be = n_cols + (V ? 1 : 0);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float accO[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) accO[i][j] = 0.f;
  for (int64_t k0 = k_lo; k0 < k_hi; k0 += DG_KC) {
    for (int e = threadIdx.x; e < DG_KC * DG_T; e += blockDim.x) {
      const int c = e / DG_KC, kk = e - c * DG_KC;
      const int64_t k = k0 + kk;
      float2 av = make_float2(0.f, 0.f), bv = make_float2(0.f, 0.f);
      if (k < k_hi) {
        const int ra = a_base + c;
        if (ra < n_rows) av = C[(size_t)rows[ra] * ldc + k];
        const int cb = b_base + c;
        if (cb < n_cols) bv = C[(size_t)cb * ldc + k];
        else if (cb == n_cols && V) bv = V[k];
      }
      Ar[kk][c] = av.x;
      Ai[kk][c] = av.y;
      Br[kk][c] = bv.x;
      Bi[kk][c] = bv.y;
    }
    __syncthreads();
    float accI[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) accI[i][j] = 0.f;
#pragma unroll 8
    for (int kk = 0; kk < DG_KC; ++kk) {
      const float4 ar = *reinterpret_cast<const float4*>(&Ar[kk][ty * 4]);
      const float4 ai = *reinterpret_cast<const float4*>(&Ai[kk][ty * 4]);
      const float4 br = *reinterpret_cast<const float4*>(&Br[kk][tx * 4]);
      const float4 bi = *reinterpret_cast<const float4*>(&Bi[kk][tx * 4]);
      const float a_r[4] = {ar.x, ar.y, ar.z, ar.w}, a_i[4] = {ai.x, ai.y, ai.z, ai.w};
      const float b_r[4] = {br.x, br.y, br.z, br.w}, b_i[4] = {bi.x, bi.y, bi.z, bi.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) accI[i][j] = fmaf(a_r[i], b_r[j], fmaf(a_i[i], b_i[j], accI[i][j]));
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) accO[i][j] += accI[i][j];
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int row = a_base + ty * 4 + i;
    if (row >= n_rows) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int col = b_base + tx * 4 + j;
      if (col < n_be) atomicAdd(&acc[(size_t)row * ldacc + col], (double)accO[i][j]);
    }
  }
}

__global__ void k_b_from_acc(const double* __restrict__ acc, int ldacc, const int32_t* __restrict__ rows,
                             int n_rows, int n_cols, float* __restrict__ b) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n_rows) b[rows[r]] = (float)acc[(size_t)r * ldacc + n_cols];
}

// ---------------------------------------------------------------- residual / forward

constexpr int AP_CHUNK = 1024;

// out[k] = base[k] + sign * sum_s theta_s C[s][k] (base may be null or alias
// out); sumsq += ||out||^2 in float64 when given.
__global__ void __launch_bounds__(256)
k_dict_apply(const float2* __restrict__ C, int64_t ldc, const float* __restrict__ th, int nS, int64_t M,
             const float2* base, float sign, float2* out, double* __restrict__ sumsq) {
  __shared__ float s_th[AP_CHUNK];
  __shared__ double red[8];
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = k < M;
  float re = 0.f, im = 0.f;
  for (int s0 = 0; s0 < nS; s0 += AP_CHUNK) {
    const int cnt = min(AP_CHUNK, nS - s0);
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) s_th[t] = th[s0 + t];
    __syncthreads();
    if (active) {
      for (int t0 = 0; t0 < cnt; t0 += 64) {
        float pr = 0.f, pi = 0.f;
        const int t1 = min(cnt, t0 + 64);
        for (int t = t0; t < t1; ++t) {
          const float2 c = C[(size_t)(s0 + t) * ldc + k];
          pr = fmaf(s_th[t], c.x, pr);
          pi = fmaf(s_th[t], c.y, pi);
        }
        re += pr;
        im += pi;
      }
    }
    __syncthreads();
  }
  double local = 0.0;
  if (active) {
    float2 o = make_float2(sign * re, sign * im);
    if (base) {
      const float2 bv = base[k];
      o = make_float2(bv.x + o.x, bv.y + o.y);
    }
    out[k] = o;
    local = (double)o.x * o.x + (double)o.y * o.y;
  }
  if (sumsq) {
    for (int off = 16; off; off >>= 1) local += __shfl_xor_sync(0xffffffffu, local, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = local;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
      atomicAdd(sumsq, t);
    }
  }
}

// ---------------------------------------------------------------- gathers and small kernels

template <class T>
__global__ void k_dgather(const T* __restrict__ src, const int32_t* __restrict__ map, int n,
                          T* __restrict__ dst, T fill) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int m = map[i];
  dst[i] = m >= 0 ? src[m] : fill;
}

// Gd[i][j] = Gs[map i][map j] where both map entries are >= 0 (old atoms).
__global__ void k_dgather_G(const float* __restrict__ Gs, int lds, const int32_t* __restrict__ map, int n,
                            float* __restrict__ Gd, int ldd) {
  const int i = blockIdx.y;
  const int mi = map[i];
  if (mi < 0) return;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    const int mj = map[j];
    if (mj >= 0) Gd[(size_t)i * ldd + j] = Gs[(size_t)mi * lds + mj];
  }
}

// Cd[i][:] = Cs[map i][:] where map[i] >= 0.
__global__ void k_dgather_cols(const float2* __restrict__ Cs, const int32_t* __restrict__ map,
                               float2* __restrict__ Cd, int64_t ldc, int64_t M) {
  const int i = blockIdx.y;
  const int mi = map[i];
  if (mi < 0) return;
  const float2* s = Cs + (size_t)mi * ldc;
  float2* d = Cd + (size_t)i * ldc;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < M; k += (int64_t)gridDim.x * blockDim.x)
    d[k] = s[k];
}

__global__ void k_dl1(const float* __restrict__ x, int n, double* __restrict__ out) {
  __shared__ double ws[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += fabs((double)x[i]);
  for (int off = 16; off; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
    *out = t;
  }
}

__global__ void k_check_idx(const int32_t* __restrict__ idx, int S, int64_t n_atoms, int* __restrict__ bad) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  const int a = idx[s];
  if (a < 0 || a >= n_atoms || (s > 0 && idx[s - 1] >= a)) atomicOr(bad, 1);
}

// ---------------------------------------------------------------- launchers

int launch_corr(const float* img, int N, const DictParams& D, float* eta, unsigned* maxbits, cudaStream_t st) {
  ProfScope prof_scope_(PROF_DICT_CORR, st);
  prof_scope_.kernels = 1;
  dim3 grid(ceil_div(N, CT), ceil_div(N, CT));
  k_dict_corr<<<grid, 256, 0, st>>>(img, N, D, eta, maxbits);
  PC_LAUNCH_CHECK();
  return PC_OK;
}

int launch_columns(pc_plan_s* p, const int32_t* idx, const int32_t* rows, int n_rows, const DictParams& D,
                   float2* C, int64_t ldc, cudaStream_t st) {
  ProfScope prof_scope_(PROF_DICT_COLUMNS, st);
  if (n_rows <= 0 || p->M <= 0) return PC_OK;
  prof_scope_.kernels = 1;
  dim3 grid(ceil_div(p->M, 256), n_rows);
  k_dict_columns<<<grid, 256, 0, st>>>(p->vis_fx, p->M, idx, rows, n_rows, p->N, p->atom_tab, D, C, ldc);
  PC_LAUNCH_CHECK();
  return PC_OK;
}

int launch_apply(const float2* C, int64_t ldc, const float* th, int nS, int64_t M, const float2* base,
                 float sign, float2* out, double* sumsq, cudaStream_t st) {
  ProfScope prof_scope_(PROF_RESIDUAL, st);
  if (M <= 0) return PC_OK;
  prof_scope_.kernels = 1;
  k_dict_apply<<<ceil_div(M, 256), 256, 0, st>>>(C, ldc, th, nS, M, base, sign, out, sumsq);
  PC_LAUNCH_CHECK();
  return PC_OK;
}

void swap_buf(DevBuf& a, DevBuf& b) {
  std::swap(a.p, b.p);
  std::swap(a.bytes, b.bytes);
}

DictWork& work(pc_plan_s* p) {
  if (!p->dict) p->dict = new DictWork();
  return *p->dict;
}

// eta / marks / selection counts for n_atoms coefficients, the mu image.
int ensure_atom_buffers(pc_plan_s* p, int64_t n_atoms, cudaStream_t st) {
  DictWork& W = work(p);
  PC_TRY(W.img.ensure(sizeof(float) * (size_t)p->N * p->N));
  if (W.n_atoms >= n_atoms) return PC_OK;
  const int nblk = ceil_div(n_atoms, kSelItems);
  PC_TRY(W.eta.ensure(sizeof(float) * (size_t)n_atoms));
  PC_TRY(W.mark.ensure((size_t)n_atoms));
  PC_TRY(W.sel.ensure(sizeof(int32_t) * ((size_t)nblk + 2)));
  PC_CUDA(cudaMemsetAsync(W.mark.p, 0, (size_t)n_atoms, st));
  PC_CUDA(cudaMemsetAsync(W.sel.p, 0, sizeof(int32_t) * ((size_t)nblk + 2), st));
  W.n_atoms = n_atoms;
  return PC_OK;
}

// Both working sets at capacity cap; the first n_keep entries of set `keep_set`
// survive (copied when the buffers are reallocated).
int ensure_sets(pc_plan_s* p, int cap, int keep_set, int n_keep, cudaStream_t st) {
  DictWork& W = work(p);
  if (cap <= W.cap) return PC_OK;
  const int64_t M = std::max<int64_t>(p->M, 1);
  const int ld_old = round4(std::max(W.cap, 1)), ld = round4(cap);
  for (int s = 0; s < 2; ++s) {
    DevBuf idx, th, b, G, C;
    PC_TRY(idx.ensure(sizeof(int32_t) * cap));
    PC_TRY(th.ensure(sizeof(float) * cap));
    PC_TRY(b.ensure(sizeof(float) * cap));
    PC_TRY(G.ensure(sizeof(float) * (size_t)ld * ld));
    PC_TRY(C.ensure(sizeof(float2) * (size_t)cap * M));
    if (s == keep_set && n_keep > 0) {
      PC_CUDA(cudaMemcpyAsync(idx.p, W.idx[s].p, sizeof(int32_t) * n_keep, cudaMemcpyDeviceToDevice, st));
      PC_CUDA(cudaMemcpyAsync(th.p, W.th[s].p, sizeof(float) * n_keep, cudaMemcpyDeviceToDevice, st));
      PC_CUDA(cudaMemcpyAsync(b.p, W.b[s].p, sizeof(float) * n_keep, cudaMemcpyDeviceToDevice, st));
      PC_CUDA(cudaMemcpy2DAsync(G.p, sizeof(float) * ld, W.G[s].p, sizeof(float) * ld_old,
                                sizeof(float) * n_keep, n_keep, cudaMemcpyDeviceToDevice, st));
      PC_CUDA(cudaMemcpyAsync(C.p, W.C[s].p, sizeof(float2) * (size_t)n_keep * M, cudaMemcpyDeviceToDevice,
                              st));
      PC_CUDA(cudaStreamSynchronize(st));   // the old buffers are freed below
    }
    swap_buf(W.idx[s], idx);
    swap_buf(W.th[s], th);
    swap_buf(W.b[s], b);
    swap_buf(W.G[s], G);
    swap_buf(W.C[s], C);
    idx.release();
    th.release();
    b.release();
    G.release();
    C.release();
  }
  PC_TRY(W.oldpos.ensure(sizeof(int32_t) * cap));
  PC_TRY(W.newrows.ensure(sizeof(int32_t) * cap));
  PC_TRY(W.keep.ensure(sizeof(int32_t) * cap));
  W.cap = cap;
  return PC_OK;
}

// mu-image = scale Phi* h, eta = Psi* mu-image, max keys in uscal[0..1]
// (uscal[2..3] take the image's own keys). Asynchronous.
int dict_certificate(pc_plan_s* p, const DictParams& D, const float2* h, float scale, float* eta,
                     cudaStream_t st) {
  DictWork& W = work(p);
  PC_CUDA(cudaMemsetAsync(p->uscal, 0, 4 * sizeof(unsigned), st));
  PC_TRY(adjoint_grid_impl(p, h, W.img.as<float>(), scale, p->uscal + 2, st));
  return launch_corr(W.img.as<float>(), p->N, D, eta, p->uscal, st);
}

int dict_gram_rows(pc_plan_s* p, const float2* V, const float2* C, int64_t ldc, const int32_t* rows,
                   int n_new, int n_act, const int32_t* oldpos, float* G, int ldg, float* b, cudaStream_t st) {
  if (n_new <= 0) return PC_OK;
  DictWork& W = work(p);
  const int ldacc = n_act + 1;
  PC_TRY(W.acc.ensure(sizeof(double) * (size_t)n_new * ldacc));
  double* acc = W.acc.as<double>();
  {
    ProfScope prof_scope_(PROF_GRAM, st);
    prof_scope_.kernels = 2;
    PC_CUDA(cudaMemsetAsync(acc, 0, sizeof(double) * (size_t)n_new * ldacc, st));
    if (p->M > 0) {
      // K-slices so that the grid holds about four CTAs per SM (thin row blocks
      // would otherwise leave most of the GPU idle), each at least 256 visibilities
      const int gx = ceil_div(ldacc, DG_T), gy = ceil_div(n_new, DG_T);
      const int64_t want = std::max<int64_t>(1, ceil_div(4 * 152, (int64_t)gx * gy));
      const int64_t slices = std::min<int64_t>(want, ceil_div(p->M, 256));
      const int64_t ks = (int64_t)ceil_div(ceil_div(p->M, slices), DG_KC) * DG_KC;
      dim3 grid(gx, gy, ceil_div(p->M, ks));
      k_dict_gram<<<grid, 256, 0, st>>>(C, ldc, p->M, ks, rows, n_new, n_act, V, acc, ldacc);
      PC_LAUNCH_CHECK();
    }
  }
  PC_TRY(launch_gram_finalize(acc, ldacc, rows, n_new, n_act, oldpos, G, ldg, st));
  ProfScope prof_scope_(PROF_MISC, st);
  prof_scope_.kernels = 1;
  k_b_from_acc<<<ceil_div(n_new, 256), 256, 0, st>>>(acc, ldacc, rows, n_new, n_act, b);
  PC_LAUNCH_CHECK();
  return PC_OK;
}

int dict_solve(pc_plan_s* p, const DictParams& D, const float2* V, double lambda, double delta,
               const SolveCfg& c, int32_t* idx_out, float* th_out, int cap_out, float* eta_out,
               pc_solve_stats* stats, pc_iter_record* hist, int hist_cap, cudaStream_t st) {
  const int N = p->N;
  const int64_t NN = (int64_t)N * N, n_atoms = D.n_scales * NN, M = p->M;
  const int64_t ldc = std::max<int64_t>(M, 1);
  PC_TRY(ensure_atom_buffers(p, n_atoms, st));
  DictWork& W = work(p);
  {
    // first capacity: 1024 atoms, fewer when M is large (columns of 2 GB at most)
    int cap0 = 1024;
    while (cap0 > 64 && (int64_t)cap0 * ldc * 8 > (2ll << 30)) cap0 >>= 1;
    PC_TRY(ensure_sets(p, std::max(W.cap, cap0), 0, 0, st));
  }
  int cur = 0, nS = 0;
  auto I = [&](int s) { return W.idx[s].as<int32_t>(); };
  auto TH = [&](int s) { return W.th[s].as<float>(); };
  auto B = [&](int s) { return W.b[s].as<float>(); };
  auto GM = [&](int s) { return W.G[s].as<float>(); };
  auto CC = [&](int s) { return W.C[s].as<float2>(); };
  uint8_t* mark = W.mark.as<uint8_t>();

  // r = V, ||V||^2
  PC_CUDA(cudaMemsetAsync(p->iscal, 0, 7 * sizeof(int32_t), st));
  PC_CUDA(cudaMemsetAsync(p->dscal, 0, 2 * sizeof(double), st));
  PC_TRY(launch_apply(CC(cur), ldc, TH(cur), 0, M, V, -1.f, p->resid, p->dscal, st));
  double hd[2] = {0.0, 0.0};
  PC_CUDA(cudaMemcpyAsync(hd, p->dscal, sizeof(double), cudaMemcpyDeviceToHost, st));
  PC_CUDA(cudaStreamSynchronize(st));
  const double sumsqV = hd[0];
  double F_prev = 0.5 * sumsqV, F = F_prev, mu_inf = 0.0;
  double Delta = (c.rule == 1 && c.lmax > 0) ? (1.0 - delta) * c.lmax : -1.0;
  int status = PC_ERR_NOT_CONVERGED, k = 0, n_hist = 0;
  int rc = PC_OK;
  for (k = 0; k < c.max_fw; ++k) {
    // ---- certificate of the iterate and the exploration threshold
    rc = dict_certificate(p, D, p->resid, (float)(1.0 / lambda), W.eta.as<float>(), st);
    if (rc != PC_OK) break;
    unsigned ub[2];
    PC_CUDA(cudaMemcpyAsync(ub, p->uscal, sizeof(ub), cudaMemcpyDeviceToHost, st));
    if ((rc = grid_flag_sync(p, st, "pc_solve_synthesis")) != PC_OK) break;
    mu_inf = (double)bits_to_float(ub[0]);
    const double top = c.positive ? (double)key_to_float(ub[1]) : mu_inf;
    if (!std::isfinite(mu_inf)) {
      rc = fail(PC_ERR_NUMERIC, "pc_solve_synthesis: non-finite certificate at iteration %d", k);
      break;
    }
    float thr = (float)(1.0 - delta);
    if (c.rule == 1) {
      if (Delta < 0.0) Delta = (1.0 - delta) * lambda * std::max(top, 0.0);
      thr = (float)(top - 2.0 * Delta / ((k + 2) * lambda));
      if (c.positive) thr = std::max(thr, 1.4e-45f);
    }
    // ---- exploration and union with the support (marked), ascending
    const int nxt = 1 - cur;
    int n_act = 0;
    for (;;) {
      rc = launch_select(W.eta.as<float>(), n_atoms, thr, mark, I(nxt), p->iscal, W.sel.as<int32_t>(), W.cap,
                         st, c.positive != 0);
      if (rc != PC_OK) break;
      PC_CUDA(cudaMemcpyAsync(&n_act, p->iscal, sizeof(int), cudaMemcpyDeviceToHost, st));
      PC_CUDA(cudaStreamSynchronize(st));
      if (n_act <= W.cap) break;
      if (n_act > 60000) {
        rc = fail(PC_ERR_CAPACITY, "pc_solve_synthesis: active set of %d atoms too large", n_act);
        break;
      }
      int nc = W.cap;
      while (nc < n_act) nc *= 2;
      if ((rc = ensure_sets(p, nc, cur, nS, st)) != PC_OK) break;
    }
    if (rc != PC_OK) break;
    const int n_new = n_act - nS;
    const int ld = round4(W.cap);
    // ---- old positions, carried-over columns / Gram / b / warm start, new columns and Gram rows
    int32_t* oldpos = W.oldpos.as<int32_t>();
    int32_t* newrows = W.newrows.as<int32_t>();
    if (n_act > 0) {
      if ((rc = launch_old_positions(I(nxt), n_act, I(cur), nS, oldpos, st)) != PC_OK) break;
      if ((rc = launch_compact_new(oldpos, n_act, newrows, p->iscal + 1, st)) != PC_OK) break;
      {
        ProfScope prof_scope_(PROF_MISC, st);
        prof_scope_.kernels = 4;
        k_dgather<float><<<ceil_div(n_act, 256), 256, 0, st>>>(TH(cur), oldpos, n_act, TH(nxt), 0.f);
        k_dgather<float><<<ceil_div(n_act, 256), 256, 0, st>>>(B(cur), oldpos, n_act, B(nxt), 0.f);
        if (nS > 0) {
          dim3 gg(std::max(1, std::min(ceil_div(n_act, 256), 32)), n_act);
          k_dgather_G<<<gg, 256, 0, st>>>(GM(cur), ld, oldpos, n_act, GM(nxt), ld);
          dim3 gc(std::max(1, std::min(ceil_div(M, 1024), 64)), n_act);
          k_dgather_cols<<<gc, 1024, 0, st>>>(CC(cur), oldpos, CC(nxt), ldc, M);
        }
        PC_LAUNCH_CHECK();
      }
      if ((rc = launch_columns(p, I(nxt), newrows, n_new, D, CC(nxt), ldc, st)) != PC_OK) break;
      if ((rc = dict_gram_rows(p, V, CC(nxt), ldc, newrows, n_new, n_act, oldpos, GM(nxt), ld, B(nxt), st)) !=
          PC_OK)
        break;
      // ---- reweighting (APGD), warm-started
      const double eps = std::max(c.eps_min, c.eps0 * std::ldexp(1.0, -k));
      if ((rc = run_apgd(GM(nxt), ld, B(nxt), n_act, lambda, eps, c.apgd_max, TH(nxt), p->iscal + 2,
                         p->dscal + 2, p->dscal + 3, st, p->iscal + 5, p->iscal + 4, c.positive != 0)) != PC_OK)
        break;
    }
    // ---- pruning: support marks off, nonzero positions, gathers into the current set
    if ((rc = launch_mark(mark, I(cur), nS, 0, st)) != PC_OK) break;
    int nS_new = 0;
    if (n_act > 0) {
      int32_t* keep = W.keep.as<int32_t>();
      if ((rc = launch_compact_nonzero(TH(nxt), n_act, keep, p->iscal + 3, st)) != PC_OK) break;
      int32_t hi[4];
      PC_CUDA(cudaMemcpyAsync(hi, p->iscal + 2, sizeof(hi), cudaMemcpyDeviceToHost, st));
      double hL = 0.0;
      PC_CUDA(cudaMemcpyAsync(&hL, p->dscal + 2, sizeof(double), cudaMemcpyDeviceToHost, st));
      PC_CUDA(cudaStreamSynchronize(st));
      if (hi[2]) {
        rc = fail(PC_ERR_TIMEOUT, "pc_solve_synthesis: a bounded device wait expired");
        break;
      }
      nS_new = hi[1];
      {
        ProfScope prof_scope_(PROF_MISC, st);
        prof_scope_.kernels = 4;
        if (nS_new > 0) {
          k_dgather<int32_t><<<ceil_div(nS_new, 256), 256, 0, st>>>(I(nxt), keep, nS_new, I(cur), 0);
          k_dgather<float><<<ceil_div(nS_new, 256), 256, 0, st>>>(TH(nxt), keep, nS_new, TH(cur), 0.f);
          k_dgather<float><<<ceil_div(nS_new, 256), 256, 0, st>>>(B(nxt), keep, nS_new, B(cur), 0.f);
          dim3 gg(std::max(1, std::min(ceil_div(nS_new, 256), 32)), nS_new);
          k_dgather_G<<<gg, 256, 0, st>>>(GM(nxt), ld, keep, nS_new, GM(cur), ld);
          dim3 gc(std::max(1, std::min(ceil_div(M, 1024), 64)), nS_new);
          k_dgather_cols<<<gc, 1024, 0, st>>>(CC(nxt), keep, CC(cur), ldc, M);
          PC_LAUNCH_CHECK();
        }
      }
      if ((rc = launch_mark(mark, I(cur), nS_new, 1, st)) != PC_OK) break;
      if (hist && n_hist < hist_cap) {
        pc_iter_record& h = hist[n_hist];
        h = pc_iter_record{};
        h.k = k;
        h.n_new = n_new;
        h.n_active = n_act;
        h.n_support = nS_new;
        h.apgd_iterations = hi[0];
        h.lanczos_steps = hi[3];
        h.mu_inf = c.positive ? top : mu_inf;
        h.lipschitz = hL;
      }
    } else if (hist && n_hist < hist_cap) {
      hist[n_hist] = pc_iter_record{};
      hist[n_hist].k = k;
      hist[n_hist].mu_inf = c.positive ? top : mu_inf;
    }
    nS = nS_new;
    // ---- residual, objective, stop test
    PC_CUDA(cudaMemsetAsync(p->dscal, 0, 2 * sizeof(double), st));
    if ((rc = launch_apply(CC(cur), ldc, TH(cur), nS, M, V, -1.f, p->resid, p->dscal, st)) != PC_OK) break;
    if (nS > 0) {
      k_dl1<<<1, 1024, 0, st>>>(TH(cur), nS, p->dscal + 1);
      PC_LAUNCH_CHECK();
    }
    PC_CUDA(cudaMemcpyAsync(hd, p->dscal, sizeof(hd), cudaMemcpyDeviceToHost, st));
    PC_CUDA(cudaStreamSynchronize(st));
    F = 0.5 * hd[0] + lambda * hd[1];
    if (!std::isfinite(F)) {
      rc = fail(PC_ERR_NUMERIC, "pc_solve_synthesis: non-finite objective at iteration %d", k);
      break;
    }
    const double rel = F_prev > 0 ? (F_prev - F) / F_prev : 0.0;
    if (hist && n_hist < hist_cap) {
      hist[n_hist].objective = F;
      hist[n_hist].rel_improvement = rel;
    }
    ++n_hist;
    F_prev = F;
    if (rel < c.tol) {
      status = PC_OK;
      ++k;
      break;
    }
  }
  // leave the marks all-zero for the next call on this plan
  const int rc_mark = launch_mark(mark, I(cur), nS, 0, st);
  if (rc != PC_OK) return rc;
  PC_TRY(rc_mark);
  if (k > c.max_fw) k = c.max_fw;
  // final certificate
  if (eta_out) {
    PC_TRY(dict_certificate(p, D, p->resid, (float)(1.0 / lambda), eta_out, st));
    unsigned ub[2];
    PC_CUDA(cudaMemcpyAsync(ub, p->uscal, sizeof(ub), cudaMemcpyDeviceToHost, st));
    PC_TRY(grid_flag_sync(p, st, "pc_solve_synthesis"));
    mu_inf = (double)bits_to_float(ub[0]);
  }
  if (stats) {
    stats->status = status;
    stats->iterations = k;
    stats->n_support = nS;
    stats->n_history = std::min(n_hist, hist_cap);
    stats->objective = F;
    stats->lambda = lambda;
    stats->mu_inf = mu_inf;
    stats->sumsq_V = sumsqV;
  }
  if (nS > cap_out) return fail(PC_ERR_CAPACITY, "pc_solve_synthesis: support of %d atoms exceeds capacity %d", nS, cap_out);
  if (nS > 0) {
    PC_CUDA(cudaMemcpyAsync(idx_out, I(cur), sizeof(int32_t) * nS, cudaMemcpyDeviceToDevice, st));
    PC_CUDA(cudaMemcpyAsync(th_out, TH(cur), sizeof(float) * nS, cudaMemcpyDeviceToDevice, st));
  }
  PC_CUDA(cudaStreamSynchronize(st));
  if (status == PC_ERR_NOT_CONVERGED)
    return fail(PC_ERR_NOT_CONVERGED, "pc_solve_synthesis: no convergence after %d Frank-Wolfe iterations", k);
  return status;
}

}  // namespace
}  // namespace pc

using namespace pc;

extern "C" int pc_dict_adjoint(pc_plan_t p, const pc_dictionary* dict, const pc_c32* h, double scale,
                               float* eta_out, void* stream) {
  clear_error();
  PC_TRY(check_plan(p, "pc_dict_adjoint"));
  DictParams D;
  PC_TRY(make_params(dict, "pc_dict_adjoint", &D));
  PC_TRY(check_dev(h, p->M > 0, "pc_dict_adjoint", "h_dev"));
  PC_TRY(check_dev(eta_out, true, "pc_dict_adjoint", "eta_out_dev"));
  if (!std::isfinite(scale)) return fail(PC_ERR_INVALID_ARG, "pc_dict_adjoint: non-finite scale");
  cudaStream_t st = SS(stream);
  PC_TRY(ensure_atom_buffers(p, (int64_t)D.n_scales * p->N * p->N, st));
  return dict_certificate(p, D, reinterpret_cast<const float2*>(h), (float)scale, eta_out, st);
}

extern "C" int pc_dict_forward_sparse(pc_plan_t p, const pc_dictionary* dict, const int32_t* idx,
                                      const float* theta, int32_t S, pc_c32* y_out, void* stream) {
  clear_error();
  PC_TRY(check_plan(p, "pc_dict_forward_sparse"));
  DictParams D;
  PC_TRY(make_params(dict, "pc_dict_forward_sparse", &D));
  if (S < 0) return fail(PC_ERR_INVALID_ARG, "pc_dict_forward_sparse: negative S");
  PC_TRY(check_dev(idx, S > 0, "pc_dict_forward_sparse", "idx_dev"));
  PC_TRY(check_dev(theta, S > 0, "pc_dict_forward_sparse", "theta_dev"));
  PC_TRY(check_dev(y_out, p->M > 0, "pc_dict_forward_sparse", "y_out_dev"));
  cudaStream_t st = SS(stream);
  const int64_t M = p->M, n_atoms = (int64_t)D.n_scales * p->N * p->N;
  float2* y = reinterpret_cast<float2*>(y_out);
  if (M == 0) return PC_OK;
  if (S == 0) {
    PC_CUDA(cudaMemsetAsync(y, 0, sizeof(float2) * M, st));
    return PC_OK;
  }
  int* bad = p->iscal + 6;
  PC_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), st));
  k_check_idx<<<ceil_div(S, 256), 256, 0, st>>>(idx, S, n_atoms, bad);
  PC_LAUNCH_CHECK();
  int hbad = 0;
  PC_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
  PC_CUDA(cudaStreamSynchronize(st));
  if (hbad)
    return fail(PC_ERR_INVALID_ARG, "pc_dict_forward_sparse: indices must be strictly ascending in [0, %lld)",
                (long long)n_atoms);
  // columns in chunks of at most 256 MB, accumulated into y
  DictWork& W = work(p);
  const int chunk = (int)std::max<int64_t>(1, std::min<int64_t>(S, (256ll << 20) / (8 * M)));
  PC_TRY(W.tmpC.ensure(sizeof(float2) * (size_t)chunk * M));
  for (int s0 = 0; s0 < S; s0 += chunk) {
    const int cnt = std::min(chunk, S - s0);
    PC_TRY(launch_columns(p, idx + s0, nullptr, cnt, D, W.tmpC.as<float2>(), M, st));
    PC_TRY(launch_apply(W.tmpC.as<float2>(), M, theta + s0, cnt, M, s0 == 0 ? nullptr : y, 1.f, y, nullptr, st));
  }
  return PC_OK;
}

extern "C" int pc_dict_lambda_max(pc_plan_t p, const pc_dictionary* dict, const pc_c32* V, int32_t positive,
                                  double* out, void* stream) {
  clear_error();
  PC_TRY(check_plan(p, "pc_dict_lambda_max"));
  DictParams D;
  PC_TRY(make_params(dict, "pc_dict_lambda_max", &D));
  PC_TRY(check_dev(V, p->M > 0, "pc_dict_lambda_max", "V_dev"));
  if (!out) return fail(PC_ERR_INVALID_ARG, "pc_dict_lambda_max: NULL output");
  cudaStream_t st = SS(stream);
  PC_TRY(ensure_atom_buffers(p, (int64_t)D.n_scales * p->N * p->N, st));
  PC_TRY(dict_certificate(p, D, reinterpret_cast<const float2*>(V), 1.0f, work(p).eta.as<float>(), st));
  unsigned ub[2] = {0, 0};
  PC_CUDA(cudaMemcpyAsync(ub, p->uscal, sizeof(ub), cudaMemcpyDeviceToHost, st));
  PC_TRY(grid_flag_sync(p, st, "pc_dict_lambda_max"));
  const float a = bits_to_float(ub[0]);
  if (!std::isfinite(a)) return fail(PC_ERR_NUMERIC, "pc_dict_lambda_max: non-finite certificate");
  *out = positive ? std::max(0.0, (double)key_to_float(ub[1])) : (double)a;
  return PC_OK;
}

extern "C" int pc_solve_synthesis(pc_plan_t p, const pc_dictionary* dict, const pc_c32* V, double lambda,
                                  double delta, const pc_solve_opts* opts, int32_t* idx_out, float* theta_out,
                                  int32_t cap, float* eta_out, pc_solve_stats* stats, pc_iter_record* hist,
                                  int32_t hist_cap, void* stream) {
  clear_error();
  PC_TRY(check_plan(p, "pc_solve_synthesis"));
  DictParams D;
  PC_TRY(make_params(dict, "pc_solve_synthesis", &D));
  if (!(lambda > 0.0) || !std::isfinite(lambda))
    return fail(PC_ERR_INVALID_ARG, "pc_solve_synthesis: lambda must be positive and finite");
  if (!(delta > 0.0 && delta <= 1.0)) return fail(PC_ERR_INVALID_ARG, "pc_solve_synthesis: delta must be in (0, 1]");
  if (cap < 0 || hist_cap < 0) return fail(PC_ERR_INVALID_ARG, "pc_solve_synthesis: negative capacity");
  PC_TRY(check_dev(V, p->M > 0, "pc_solve_synthesis", "V_dev"));
  PC_TRY(check_dev(idx_out, cap > 0, "pc_solve_synthesis", "idx_out_dev"));
  PC_TRY(check_dev(theta_out, cap > 0, "pc_solve_synthesis", "theta_out_dev"));
  if (eta_out) PC_TRY(check_dev(eta_out, true, "pc_solve_synthesis", "eta_out_dev"));
  SolveCfg c;
  PC_TRY(parse_solve_opts(opts, "pc_solve_synthesis", &c));
  return dict_solve(p, D, reinterpret_cast<const float2*>(V), lambda, delta, c, idx_out, theta_out, cap,
                    eta_out, stats, hist, hist_cap, SS(stream));
}
