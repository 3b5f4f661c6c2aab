// Sparse-support operators (the forward equation of Sect. 2.2 restricted to
// the active set of Algorithm 2, a type-3 sum in the paper's HVOX, Sect. 5.2)
// and the support contraction that turns step 2 of Algorithm 2 into a small
// dense problem:
//
//   Phi_S[k, s] = e^{-j 2 pi theta_ks} / n_s,  theta_ks = u_k l_s + v_k m_s + w_k (n_s - 1)
//   residual    r = V - Phi_S x
//   Gram        G = Re(Phi_S^H Phi_S),  b = Re(Phi_S^H V)
//
// Phases are generated on the fly: the lattice part i' U_k + j' V_k in exact
// 32-bit fixed-point turns, the w-term as a double-float product, one FP32
// sincospi per (visibility, atom) pair.
#include "pc_internal.cuh"

namespace pc {
namespace {

__global__ void k_make_atoms(const int32_t* __restrict__ idx, const float* __restrict__ x, int S,
                             int N, double dl, float4* __restrict__ atoms, int* __restrict__ bad,
                             const int32_t* __restrict__ S_dev) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (S_dev) S = min(S, *S_dev);   // count held on the device (S: its upper bound)
  if (s >= S) return;
  const int p = idx[s];
  if (bad && (p < 0 || p >= N * N || (s > 0 && idx[s - 1] >= p))) atomicOr(bad, 1);
  atoms[s] = make_atom(p, x ? x[s] : 1.f, x != nullptr, N, dl);
}

constexpr int RES_CHUNK = 1024;

// out = V - Phi_S x  (or Phi_S x when V is null); sumsq += ||out||^2 in float64.
__global__ void __launch_bounds__(256)
k_residual(const int4* __restrict__ vis, const float2* __restrict__ V, int64_t M,
           const float4* __restrict__ atoms, int S, float2* __restrict__ out,
           double* __restrict__ sumsq, const int32_t* __restrict__ S_dev) {
  __shared__ float4 sa[RES_CHUNK];
  __shared__ double red[8];
  if (S_dev) S = min(S, *S_dev);
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool active = k < M;
  const int4 vk = active ? vis[k] : make_int4(0, 0, 0, 0);
  float ar = 0.f, ai = 0.f;
  for (int s0 = 0; s0 < S; s0 += RES_CHUNK) {
    const int cnt = min(RES_CHUNK, S - s0);
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) sa[t] = atoms[s0 + t];
    __syncthreads();
    if (active) {
      for (int t = 0; t < cnt; ++t) {
        const float4 at = sa[t];
        // the phase is reduced exactly to [-1/2, 1/2] turns, where the fast
        // sine and cosine are accurate to ~4e-7 absolute (as in the Gram kernels)
        float sn, cs;
        __sincosf(6.283185307179586f * phase_turns(vk, at), &sn, &cs);
        ar = fmaf(at.w, cs, ar);
        ai = fmaf(-at.w, sn, ai);
      }
    }
    __syncthreads();
  }
  double local = 0.0;
  if (active) {
    float2 r;
    if (V) {
      const float2 v = V[k];
      r = make_float2(v.x - ar, v.y - ai);
    } else {
      r = make_float2(ar, ai);
    }
    out[k] = r;
    local = (double)r.x * r.x + (double)r.y * r.y;
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

constexpr int GT = 128;      // Gram tile (atoms x atoms)
constexpr int GKC = 32;      // visibilities per shared-memory chunk
constexpr int GKS = 8192;    // visibilities per K-slice (one float64 flush per slice)

// acc[a][c] += sum_k Re(conj(Phi[k, a]) B[k, c]) over one K-slice, where
// B[:, c] = Phi[:, atomB_c] for c < nB and B[:, nB] = V when with_v.
__global__ void __launch_bounds__(256)
k_gram(const int4* __restrict__ vis, const float2* __restrict__ V, int64_t M,
       const float4* __restrict__ atomsA, int nA, const float4* __restrict__ atomsB, int nB,
       int with_v, double* __restrict__ acc, int ldacc) {
  extern __shared__ float gsm[];
  float* Are = gsm;
  float* Aim = Are + GKC * GT;
  float* Bre = Aim + GKC * GT;
  float* Bim = Bre + GKC * GT;
  __shared__ float4 sA[GT], sB[GT];
  const int a_base = blockIdx.y * GT, b_base = blockIdx.x * GT;
  const int64_t k_lo = (int64_t)blockIdx.z * GKS;
  const int64_t k_hi = min((int64_t)M, k_lo + GKS);
  const int nBe = nB + (with_v ? 1 : 0);
  for (int t = threadIdx.x; t < GT; t += blockDim.x) {
    sA[t] = (a_base + t < nA) ? atomsA[a_base + t] : make_float4(0.f, 0.f, 0.f, 0.f);
    sB[t] = (b_base + t < nB) ? atomsB[b_base + t] : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float accO[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) accO[i][j] = 0.f;
  __syncthreads();

  for (int64_t k0 = k_lo; k0 < k_hi; k0 += GKC) {
    for (int e = threadIdx.x; e < GKC * GT; e += blockDim.x) {
      const int kk = e / GT, c = e - kk * GT;
      const int64_t k = k0 + kk;
      float are = 0.f, aim = 0.f, bre = 0.f, bim = 0.f;
      if (k < k_hi) {
        const int4 vk = vis[k];
        if (a_base + c < nA) {
          const float4 at = sA[c];
          float sn, cs;
          sincospif(2.0f * phase_turns(vk, at), &sn, &cs);
          are = cs * at.w;
          aim = sn * at.w;
        }
        const int col = b_base + c;
        if (col < nB) {
          const float4 bt = sB[c];
          float sn, cs;
          sincospif(2.0f * phase_turns(vk, bt), &sn, &cs);
          bre = cs * bt.w;
          bim = sn * bt.w;
        } else if (col == nB && with_v) {
          const float2 v = V[k];
          bre = v.x;
          bim = -v.y;
        }
      }
      Are[kk * GT + c] = are;
      Aim[kk * GT + c] = aim;
      Bre[kk * GT + c] = bre;
      Bim[kk * GT + c] = bim;
    }
    __syncthreads();
    float accI[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) accI[i][j] = 0.f;
#pragma unroll 4
    for (int kk = 0; kk < GKC; ++kk) {
      float ar[8], ai[8], br[8], bi[8];
      const float4* pa = reinterpret_cast<const float4*>(Are + kk * GT + ty * 8);
      const float4* pai = reinterpret_cast<const float4*>(Aim + kk * GT + ty * 8);
      const float4* pb = reinterpret_cast<const float4*>(Bre + kk * GT + tx * 8);
      const float4* pbi = reinterpret_cast<const float4*>(Bim + kk * GT + tx * 8);
      float4 t0 = pa[0], t1 = pa[1];
      ar[0] = t0.x; ar[1] = t0.y; ar[2] = t0.z; ar[3] = t0.w;
      ar[4] = t1.x; ar[5] = t1.y; ar[6] = t1.z; ar[7] = t1.w;
      t0 = pai[0]; t1 = pai[1];
      ai[0] = t0.x; ai[1] = t0.y; ai[2] = t0.z; ai[3] = t0.w;
      ai[4] = t1.x; ai[5] = t1.y; ai[6] = t1.z; ai[7] = t1.w;
      t0 = pb[0]; t1 = pb[1];
      br[0] = t0.x; br[1] = t0.y; br[2] = t0.z; br[3] = t0.w;
      br[4] = t1.x; br[5] = t1.y; br[6] = t1.z; br[7] = t1.w;
      t0 = pbi[0]; t1 = pbi[1];
      bi[0] = t0.x; bi[1] = t0.y; bi[2] = t0.z; bi[3] = t0.w;
      bi[4] = t1.x; bi[5] = t1.y; bi[6] = t1.z; bi[7] = t1.w;
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) accI[i][j] = fmaf(ar[i], br[j], fmaf(ai[i], bi[j], accI[i][j]));
    }
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) accO[i][j] += accI[i][j];
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int row = a_base + ty * 8 + i;
    if (row >= nA) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int col = b_base + tx * 8 + j;
      if (col < nBe) atomicAdd(&acc[(size_t)row * ldacc + col], (double)accO[i][j]);
    }
  }
}

constexpr int THIN_RMAX = 16;     // rows (atoms + the V row) of the thin contraction
constexpr int THIN_COLS = 128;    // columns (atoms) per CTA
constexpr int THIN_CHUNK = 256;   // visibilities staged per chunk
constexpr int THIN_SLICE_MAX = 4096;  // visibilities per CTA at most (the launcher picks the slice)

// Thin contraction for a few rows: for row r < nA (an atom of atomsA) and
// column c (an atom of atomsB)
//   acc[r][c] += sum_k Re(conj(Phi[k, A_r]) Phi[k, B_c])
// and, when V is given, the extra row
//   b64[c]    += sum_k Re(conj(Phi[k, B_c]) V_k)
// over one slice of visibilities. Thread (c, half) generates the phase of its
// column atom for every other visibility of a chunk; the row phases of the
// chunk are generated once into shared memory. No tile padding: the cost is
// one phase per (visibility, column) plus 2 FMAs per row.
template <int R>
__global__ void __launch_bounds__(256)
k_gram_thin(const int4* __restrict__ vis, const float2* __restrict__ V, int64_t M,
            const float4* __restrict__ atomsA, int nA, const float4* __restrict__ atomsB, int nB,
            double* __restrict__ acc, int ldacc, double* __restrict__ b64, int slice) {
  __shared__ float sRe[R][THIN_CHUNK];
  __shared__ float sIm[R][THIN_CHUNK];
  __shared__ int4 sVis[THIN_CHUNK];
  __shared__ float4 sA[R];
  __shared__ float sRed[R][THIN_COLS];
  const int rows = nA + (V ? 1 : 0);
  const int tid = threadIdx.x, col = tid % THIN_COLS, half = tid / THIN_COLS;
  const int c_glob = blockIdx.x * THIN_COLS + col;
  const float4 bt = c_glob < nB ? atomsB[c_glob] : make_float4(0.f, 0.f, 0.f, 0.f);
  if (tid < R) sA[tid] = tid < nA ? atomsA[tid] : make_float4(0.f, 0.f, 0.f, 0.f);
  const int64_t k_lo = (int64_t)blockIdx.y * slice;
  const int64_t k_hi = min(M, k_lo + slice);
  float outer[R];
#pragma unroll
  for (int r = 0; r < R; ++r) outer[r] = 0.f;
  for (int64_t k0 = k_lo; k0 < k_hi; k0 += THIN_CHUNK) {
    const int cnt = (int)min((int64_t)THIN_CHUNK, k_hi - k0);
    __syncthreads();
    sVis[tid] = tid < cnt ? vis[k0 + tid] : make_int4(0, 0, 0, 0);
    __syncthreads();
    for (int e = tid; e < rows * THIN_CHUNK; e += blockDim.x) {
      const int r = e / THIN_CHUNK, t = e - r * THIN_CHUNK;
      float re = 0.f, im = 0.f;
      if (t < cnt) {
        if (r < nA) {
          float sn, cs;
          __sincosf(6.283185307179586f * phase_turns(sVis[t], sA[r]), &sn, &cs);
          re = cs * sA[r].w;
          im = sn * sA[r].w;
        } else {
          const float2 v = V[k0 + t];
          re = v.x;
          im = -v.y;
        }
      }
      sRe[r][t] = re;
      sIm[r][t] = im;
    }
    __syncthreads();
    float inner[R];
#pragma unroll
    for (int r = 0; r < R; ++r) inner[r] = 0.f;
    // columns past nB (the last CTA's unused threads) skip the phase work
    for (int t = half; t < (c_glob < nB ? cnt : 0); t += 2) {
      float sn, cs;
      __sincosf(6.283185307179586f * phase_turns(sVis[t], bt), &sn, &cs);
      const float br = cs * bt.w, bi = sn * bt.w;
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (r < rows) inner[r] = fmaf(sRe[r][t], br, fmaf(sIm[r][t], bi, inner[r]));
    }
#pragma unroll
    for (int r = 0; r < R; ++r) outer[r] += inner[r];
  }
  __syncthreads();
  if (half == 1)
#pragma unroll
    for (int r = 0; r < R; ++r) sRed[r][col] = outer[r];
  __syncthreads();
  if (half == 0 && c_glob < nB) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (r >= rows) break;
      const double v = (double)outer[r] + (double)sRed[r][col];
      if (r < nA) atomicAdd(&acc[(size_t)r * ldacc + c_glob], v);
      else atomicAdd(&b64[c_glob], v);
    }
  }
}

// Tensor-core path: rows r < n_new and columns c < n_act of acc are in the
// permuted atom order perm (new atoms first); column n_act is b. Writes
// G[perm[r]][perm[c]] and its mirror (a new-new pair only from r <= c, so G
// stays exactly symmetric) and b[perm[r]].
__global__ void k_gram_finalize_perm(const double* __restrict__ acc, int ldacc, int n_new, int n_act,
                                     const int32_t* __restrict__ perm, float* __restrict__ G, int ldg,
                                     float* __restrict__ b) {
  const int r = blockIdx.y;
  if (r >= n_new) return;
  const int pr = perm ? perm[r] : r;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n_act; c += gridDim.x * blockDim.x) {
    if (c < n_new && c < r) continue;
    const int pc = perm ? perm[c] : c;
    const float v = (float)acc[(size_t)r * ldacc + c];
    G[(size_t)pr * ldg + pc] = v;
    G[(size_t)pc * ldg + pr] = v;
  }
  if (b && blockIdx.x == 0 && threadIdx.x == 0) b[pr] = (float)acc[(size_t)r * ldacc + n_act];
}

__global__ void k_d2f(const double* __restrict__ in, int n, float* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (float)in[i];
}

// Write Gram rows of the "new" atoms into G (and their mirror columns).
// Row r of acc belongs to the atom at position rows[r]; a column c that is
// also new (oldpos[c] < 0) is written only from the row whose position is
// <= c, so that G stays exactly symmetric.
__global__ void k_gram_finalize(const double* __restrict__ acc, int ldacc,
                                const int32_t* __restrict__ rows, int nrows, int ncols,
                                const int32_t* __restrict__ oldpos,
                                float* __restrict__ G, int ldg) {
  const int r = blockIdx.y;
  if (r >= nrows) return;
  const int pr = rows ? rows[r] : r;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncols; c += gridDim.x * blockDim.x) {
    const bool c_new = oldpos ? (oldpos[c] < 0) : true;
    if (c_new && c < pr) continue;
    const float v = (float)acc[(size_t)r * ldacc + c];
    G[(size_t)pr * ldg + c] = v;
    G[(size_t)c * ldg + pr] = v;
  }
}

}  // namespace

int launch_make_atoms(const int32_t* idx, const float* x, int S, int N, double dl, float4* atoms,
                      cudaStream_t st, const int32_t* S_dev) {
  ProfScope prof_scope_(PROF_MISC, st);
  if (S <= 0) return PC_OK;
  prof_scope_.kernels = 1;
  k_make_atoms<<<ceil_div(S, 256), 256, 0, st>>>(idx, x, S, N, dl, atoms, nullptr, S_dev);
  PC_LAUNCH_CHECK();
  return PC_OK;
}

// Validating variant for the public entry points: returns PC_ERR_INVALID_ARG
// when idx is not strictly ascending inside [0, N^2). Synchronises the stream.
int make_atoms_checked(const int32_t* idx, const float* x, int S, int N, double dl,
                       float4* atoms, int* dflag, cudaStream_t st) {
  if (S <= 0) return PC_OK;
  PC_CUDA(cudaMemsetAsync(dflag, 0, sizeof(int), st));
  k_make_atoms<<<ceil_div(S, 256), 256, 0, st>>>(idx, x, S, N, dl, atoms, dflag, nullptr);
  PC_LAUNCH_CHECK();
  int h = 0;
  PC_CUDA(cudaMemcpyAsync(&h, dflag, sizeof(int), cudaMemcpyDeviceToHost, st));
  PC_CUDA(cudaStreamSynchronize(st));
  if (h) return fail(PC_ERR_INVALID_ARG, "support indices must be strictly ascending in [0, N*N)");
  return PC_OK;
}

int launch_residual(const int4* vis_fx, const float2* V, int64_t M, const float4* atoms, int S,
                    float2* out, double* sumsq, cudaStream_t st, const int32_t* S_dev) {
  ProfScope prof_scope_(PROF_RESIDUAL, st);
  if (M <= 0) return PC_OK;
  prof_scope_.kernels = 1;
  k_residual<<<ceil_div(M, 256), 256, 0, st>>>(vis_fx, V, M, atoms, S, out, sumsq, S_dev);
  PC_LAUNCH_CHECK();
  return PC_OK;
}

int launch_gram(const int4* vis_fx, const float2* V, int64_t M, const float4* atomsA, int nA,
                const float4* atomsB, int nB, bool with_v, double* acc, int ldacc,
                cudaStream_t st, bool clear) {
  ProfScope prof_scope_(PROF_GRAM, st);
  const int nBe = nB + (with_v ? 1 : 0);
  if (clear) {
    PC_CUDA(cudaMemsetAsync(acc, 0, sizeof(double) * (size_t)nA * ldacc, st));
    prof_scope_.kernels = 1;
  }
  if (M <= 0 || nA <= 0 || nBe <= 0) return PC_OK;
  static bool attr_set = false;
  const size_t smem = (size_t)4 * GKC * GT * sizeof(float);
  if (!attr_set) {
    PC_CUDA(cudaFuncSetAttribute(k_gram, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr_set = true;
  }
  dim3 grid(ceil_div(nBe, GT), ceil_div(nA, GT), ceil_div(M, GKS));
  prof_scope_.kernels += 1;
  k_gram<<<grid, 256, smem, st>>>(vis_fx, V, M, atomsA, nA, atomsB, nB, with_v ? 1 : 0, acc,
                                  ldacc);
  PC_LAUNCH_CHECK();
  return PC_OK;
}

int launch_gram_thin(const int4* vis_fx, const float2* V, int64_t M, const float4* atomsA, int nA,
                     const float4* atomsB, int nB, double* acc, int ldacc, double* b64,
                     cudaStream_t st) {
  ProfScope prof_scope_(PROF_GRAM_THIN, st);
  if (M <= 0 || nB <= 0 || (nA <= 0 && !V)) return PC_OK;
  if (nA + (V ? 1 : 0) > THIN_RMAX) return fail(PC_ERR_INVALID_ARG, "thin Gram: too many rows");
  prof_scope_.kernels = 1;
  // visibilities per CTA: a multiple of the chunk, sized for about six CTAs
  // per SM (the phase chains are latency-bound; each CTA adds its partial
  // sums to the float64 accumulators once)
  static int n_sm = 0;
  if (n_sm == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n_sm <= 0) n_sm = 152;
  }
  const int gx = ceil_div(nB, THIN_COLS);
  int64_t slice = ((int64_t)M * gx + (int64_t)n_sm * 6 - 1) / ((int64_t)n_sm * 6);
  slice = std::min<int64_t>(THIN_SLICE_MAX, std::max<int64_t>(THIN_CHUNK, ceil_div(slice, THIN_CHUNK) * (int64_t)THIN_CHUNK));
  dim3 grid(gx, ceil_div(M, slice));
  const int sl = (int)slice;
  // rows padded to a power of two: the per-row loops are unrolled at that size
  const int rows = nA + (V ? 1 : 0);
  if (rows <= 1)
    k_gram_thin<1><<<grid, 256, 0, st>>>(vis_fx, V, M, atomsA, nA, atomsB, nB, acc, ldacc, b64, sl);
  else if (rows <= 2)
    k_gram_thin<2><<<grid, 256, 0, st>>>(vis_fx, V, M, atomsA, nA, atomsB, nB, acc, ldacc, b64, sl);
  else if (rows <= 4)
    k_gram_thin<4><<<grid, 256, 0, st>>>(vis_fx, V, M, atomsA, nA, atomsB, nB, acc, ldacc, b64, sl);
  else if (rows <= 8)
    k_gram_thin<8><<<grid, 256, 0, st>>>(vis_fx, V, M, atomsA, nA, atomsB, nB, acc, ldacc, b64, sl);
  else
    k_gram_thin<16><<<grid, 256, 0, st>>>(vis_fx, V, M, atomsA, nA, atomsB, nB, acc, ldacc, b64, sl);
  PC_LAUNCH_CHECK();
  return PC_OK;
}

int launch_gram_finalize_perm(const double* acc, int ldacc, int n_new, int n_act, const int32_t* perm,
                              float* G, int ldg, float* b, cudaStream_t st) {
  ProfScope prof_scope_(PROF_GRAM_FINALIZE, st);
  if (n_new <= 0) return PC_OK;
  prof_scope_.kernels = 1;
  dim3 grid(std::max(1, std::min(ceil_div(n_act, 256), 64)), n_new);
  k_gram_finalize_perm<<<grid, 256, 0, st>>>(acc, ldacc, n_new, n_act, perm, G, ldg, b);
  PC_LAUNCH_CHECK();
  return PC_OK;
}

int launch_d2f(const double* in, int n, float* out, cudaStream_t st) {
  ProfScope prof_scope_(PROF_MISC, st);
  if (n <= 0) return PC_OK;
  prof_scope_.kernels = 1;
  k_d2f<<<ceil_div(n, 256), 256, 0, st>>>(in, n, out);
  PC_LAUNCH_CHECK();
  return PC_OK;
}

int launch_gram_finalize(const double* acc, int ldacc, const int32_t* rows, int nrows, int ncols,
                         const int32_t* oldpos, float* G, int ldg, cudaStream_t st) {
  ProfScope prof_scope_(PROF_GRAM_FINALIZE, st);
  if (nrows <= 0) return PC_OK;
  dim3 grid(std::max(1, std::min(ceil_div(ncols, 256), 64)), nrows);
  prof_scope_.kernels = 1;
  k_gram_finalize<<<grid, 256, 0, st>>>(acc, ldacc, rows, nrows, ncols, oldpos, G, ldg);
  PC_LAUNCH_CHECK();
  return PC_OK;
}

}  // namespace pc
