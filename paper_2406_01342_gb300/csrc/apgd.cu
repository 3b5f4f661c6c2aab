// Restricted LASSO solve of step 2 of Algorithm 2 by accelerated proximal
// gradient (FISTA, the APGD the paper names in Sect. 3.4 / 4.1) on the Gram
// form of the support problem:
//
//   f(x) = 1/2 x^T G x - b^T x + lambda ||x||_1,   G = Re(Phi_S^H Phi_S), b = Re(Phi_S^H V)
//
// Readings (the paper gives no constants): step 1/L with L = 1.01 x the
// largest eigenvalue of G; the monotone FISTA variant; stop when
// ||z - y|| <= eps ||z||. The eigenvalue comes from Lanczos on G started from
// the all-ones vector: the largest Ritz value of the tridiagonal matrix (by
// Sturm-count multisection), until it changes by < 1e-6 relative between
// checks every 4 steps, at most 64 steps (or n, or an invariant subspace).
//
// GB300 mapping: one thread-block cluster (16 CTAs when the device allows it,
// else 8). CTA r owns a contiguous block of rows of G (cached in its shared
// memory when it fits) and of every vector. Each iteration does one GEMV:
// the CTAs publish their slice of the proximal point z in shared memory, a
// cluster barrier, every CTA gathers the whole z through distributed shared
// memory, multiplies its rows, publishes five float64 partial sums, a second
// barrier, and every CTA reduces the partials in the same order (so all take
// identical decisions). G z is the only matrix product per iteration: G y and
// G x are kept as linear combinations of previous products.
#include <cooperative_groups.h>

#include <cmath>

#include "pc_internal.cuh"

namespace cg = cooperative_groups;

namespace pc {
namespace {

struct ApgdArgs {
  const float* G;
  int ldg;
  const float* b;
  int n;
  float lam;
  float eps;
  int max_iter;
  float* x;
  int* out_iters;
  double* out_L;
  double* out_F;
  int rows_per;
  int n_pad;
  int cache;      // 1: rows of G cached in shared memory
  int vec_ok;     // 1: float4 loads of G rows are aligned
};

constexpr int APGD_THREADS = 512;
constexpr int NPART = 5;

struct Smem {
  float* zfull;   // n_pad
  float* pub;     // rows_per (published slice)
  float* y;
  float* Gy;
  float* x;
  float* Gx;
  float* z;
  float* Gz;
  float* bb;
  double* part;   // NPART
  float* Gc;      // rows_per * n_pad (optional)
};

__device__ Smem carve(float* base, const ApgdArgs& a) {
  Smem s;
  float* p = base;
  s.zfull = p; p += a.n_pad;
  s.pub = p; p += a.rows_per;
  s.y = p; p += a.rows_per;
  s.Gy = p; p += a.rows_per;
  s.x = p; p += a.rows_per;
  s.Gx = p; p += a.rows_per;
  s.z = p; p += a.rows_per;
  s.Gz = p; p += a.rows_per;
  s.bb = p; p += a.rows_per;
  p = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(p) + 15) & ~uintptr_t(15));
  s.part = reinterpret_cast<double*>(p); p += 2 * 16;   // two partial-sum buffers of 8
  s.Gc = p;
  return s;
}

// Gather the published slices of every CTA into zfull.
__device__ void gather(cg::cluster_group& cl, const Smem& s, const ApgdArgs& a) {
  const int CS = (int)cl.num_blocks();
  for (int idx = threadIdx.x; idx < a.n; idx += blockDim.x) {
    const int rr = idx / a.rows_per;
    const int off = idx - rr * a.rows_per;
    const float* remote = cl.map_shared_rank(s.pub, rr);
    s.zfull[idx] = remote[off];
  }
  for (int idx = a.n + threadIdx.x; idx < a.n_pad; idx += blockDim.x) s.zfull[idx] = 0.f;
  (void)CS;
}

// out[r] = G[r0 + r, :] . zfull for the nr own rows; one warp per row.
__device__ void gemv_rows(const Smem& s, const ApgdArgs& a, int r0, int nr, float* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int r = warp; r < nr; r += nw) {
    const float* row = a.cache ? s.Gc + (size_t)r * a.n_pad : a.G + (size_t)(r0 + r) * a.ldg;
    float acc = 0.f;
    if (a.cache || a.vec_ok) {
      // full float4 groups inside [0, n), then a scalar tail: columns >= n of a
      // caller's G are never read
      const float4* r4 = reinterpret_cast<const float4*>(row);
      const float4* z4 = reinterpret_cast<const float4*>(s.zfull);
      const int n4 = a.n >> 2;
      for (int c = lane; c < n4; c += 32) {
        const float4 g = r4[c];
        const float4 z = z4[c];
        acc = fmaf(g.x, z.x, acc);
        acc = fmaf(g.y, z.y, acc);
        acc = fmaf(g.z, z.z, acc);
        acc = fmaf(g.w, z.w, acc);
      }
      for (int c = 4 * n4 + lane; c < a.n; c += 32) acc = fmaf(row[c], s.zfull[c], acc);
    } else {
      for (int c = lane; c < a.n; c += 32) acc = fmaf(row[c], s.zfull[c], acc);
    }
    for (int off = 16; off; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) out[r] = acc;
  }
}

// Block-wide float64 sums of NPART per-thread values, written to part[] by thread 0.
__device__ void block_sums(double v[NPART], double* part, double* scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int q = 0; q < NPART; ++q)
    for (int off = 16; off; off >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], off);
  if (lane == 0)
    for (int q = 0; q < NPART; ++q) scratch[warp * NPART + q] = v[q];
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 0; q < NPART; ++q) {
      double t = 0.0;
      for (int w = 0; w < nw; ++w) t += scratch[w * NPART + q];
      part[q] = t;
    }
  }
  __syncthreads();
}

constexpr int LZ_MAX = 64;

// Largest eigenvalue of the symmetric tridiagonal matrix (diagonal al[0..m),
// off-diagonal be[0..m-1)) by multisection with Sturm counts: warp 0 narrows
// the Gershgorin interval 33-fold per round, in FP32 on the matrix scaled by
// its Gershgorin bound (relative accuracy ~1e-6, enough for a step size that
// carries a 1 % margin). Same inputs in every CTA give the same result.
__device__ double tridiag_top(const double* al, const double* be, int m, double* s_out) {
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    double glo = 1e300, ghi = -1e300;
    for (int i = 0; i < m; ++i) {
      const double r = (i > 0 ? fabs(be[i - 1]) : 0.0) + (i + 1 < m ? fabs(be[i]) : 0.0);
      glo = fmin(glo, al[i] - r);
      ghi = fmax(ghi, al[i] + r);
    }
    const double scale = fmax(fabs(glo), fabs(ghi)) > 0.0 ? fmax(fabs(glo), fabs(ghi)) : 1.0;
    float lo = (float)(glo / scale), hi = (float)(ghi / scale);
    for (int round = 0; round < 8; ++round) {
      const float x = lo + (hi - lo) * (float)(lane + 1) / 33.0f;
      int below = 0;                          // eigenvalues below x = negative LDL^T pivots
      float d = (float)(al[0] / scale) - x;
      if (d == 0.0f) d = -1e-30f;
      below += d < 0.0f;
      for (int i = 1; i < m; ++i) {
        const float bi = (float)(be[i - 1] / scale);
        d = ((float)(al[i] / scale) - x) - bi * bi / d;
        if (d == 0.0f) d = -1e-30f;
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
    if (lane == 0) *s_out = (double)hi * scale;
  }
  __syncthreads();
  return *s_out;
}

// Sum the published partials of all CTAs: warp 0 reads each CTA's partials
// once over distributed shared memory and reduces them with a fixed butterfly
// (the same order in every CTA, so every CTA takes the same decisions).
__device__ void cluster_sums(cg::cluster_group& cl, double* part, double* s_tot,
                             double out[NPART]) {
  const int CS = (int)cl.num_blocks();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    const double* rp = lane < CS ? cl.map_shared_rank(part, lane) : nullptr;
    for (int q = 0; q < NPART; ++q) {
      double v = rp ? rp[q] : 0.0;
      for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
      if (lane == 0) s_tot[q] = v;
    }
  }
  __syncthreads();
  for (int q = 0; q < NPART; ++q) out[q] = s_tot[q];
}

__global__ void __launch_bounds__(APGD_THREADS, 1) k_apgd(ApgdArgs a) {
  extern __shared__ __align__(16) float apgd_sm[];
  __shared__ double scratch[(APGD_THREADS / 32) * NPART];
  __shared__ double s_tot[NPART];
  __shared__ double s_al[LZ_MAX], s_be[LZ_MAX], s_theta;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const Smem s = carve(apgd_sm, a);
  const int r0 = rank * a.rows_per;
  const int nr = max(0, min(a.n, r0 + a.rows_per) - r0);

  if (a.cache) {
    for (int e = threadIdx.x; e < nr * a.n_pad; e += blockDim.x) {
      const int r = e / a.n_pad, c = e - r * a.n_pad;
      s.Gc[e] = c < a.n ? a.G[(size_t)(r0 + r) * a.ldg + c] : 0.f;
    }
  }
  for (int r = threadIdx.x; r < a.rows_per; r += blockDim.x) {
    const bool own = r < nr;
    s.bb[r] = own ? a.b[r0 + r] : 0.f;
    s.x[r] = own ? a.x[r0 + r] : 0.f;
    const float v0 = own ? rsqrtf((float)a.n) : 0.f;   // Lanczos start: all ones / sqrt(n)
    s.y[r] = v0;        // v_j
    s.z[r] = 0.f;       // v_{j-1}
    s.pub[r] = v0;
  }
  __syncthreads();

  // ---- Lipschitz constant: Lanczos, two cluster reductions per step
  // (alpha = v^T G v first, then ||w||); the second uses the other partial buffer.
  double* part2 = s.part + 8;
  double theta = 0.0, theta_prev = 0.0, beta_prev = 0.0;
  int m = 0;
  for (int j = 0; j < LZ_MAX; ++j) {
    cl.sync();
    gather(cl, s, a);
    __syncthreads();
    gemv_rows(s, a, r0, nr, s.Gz);                  // w = G v_j
    __syncthreads();
    double v[NPART] = {0, 0, 0, 0, 0};
    for (int r = threadIdx.x; r < nr; r += blockDim.x) v[0] += (double)s.y[r] * s.Gz[r];
    block_sums(v, s.part, scratch);
    cl.sync();
    double tot[NPART];
    cluster_sums(cl, s.part, s_tot, tot);
    const double alpha = tot[0];
    const float fa = (float)alpha, fb = (float)beta_prev;
    double v2[NPART] = {0, 0, 0, 0, 0};
    for (int r = threadIdx.x; r < nr; r += blockDim.x) {
      const float w = s.Gz[r] - fa * s.y[r] - fb * s.z[r];
      s.Gz[r] = w;
      v2[0] += (double)w * w;
    }
    block_sums(v2, part2, scratch);
    cl.sync();
    cluster_sums(cl, part2, s_tot, tot);
    const double beta = sqrt(tot[0]);
    if (threadIdx.x == 0) {
      s_al[j] = alpha;
      s_be[j] = beta;
    }
    m = j + 1;
    __syncthreads();
    const bool last = (m == a.n) || (m == LZ_MAX) || !(beta > 1e-7 * fabs(alpha));
    if (last || (m % 4) == 0) {
      theta = tridiag_top(s_al, s_be, m, &s_theta);
      if (last || fabs(theta - theta_prev) <= 1e-6 * fabs(theta)) break;
      theta_prev = theta;
    }
    const float inv = (float)(1.0 / beta);
    for (int r = threadIdx.x; r < nr; r += blockDim.x) {
      const float vn = s.Gz[r] * inv;
      s.z[r] = s.y[r];
      s.y[r] = vn;
      s.pub[r] = vn;
    }
    beta_prev = beta;
  }
  const double L = 1.01 * (theta > 0.0 ? theta : 1.0);
  const float invL = (float)(1.0 / L);
  const float thr = (float)(a.lam / L);

  // ---- initial G x
  for (int r = threadIdx.x; r < nr; r += blockDim.x) s.pub[r] = s.x[r];
  cl.sync();
  gather(cl, s, a);
  __syncthreads();
  gemv_rows(s, a, r0, nr, s.Gx);
  __syncthreads();
  double Fx;
  {
    double v[NPART] = {0, 0, 0, 0, 0};
    for (int r = threadIdx.x; r < nr; r += blockDim.x) {
      v[0] += (double)s.x[r] * s.Gx[r];
      v[1] += (double)s.bb[r] * s.x[r];
      v[2] += fabs((double)s.x[r]);
    }
    block_sums(v, s.part, scratch);
    cl.sync();
    double tot[NPART];
    cluster_sums(cl, s.part, s_tot, tot);
    Fx = 0.5 * tot[0] - tot[1] + (double)a.lam * tot[2];
  }
  for (int r = threadIdx.x; r < nr; r += blockDim.x) {
    s.y[r] = s.x[r];
    s.Gy[r] = s.Gx[r];
  }
  __syncthreads();

  // ---- monotone FISTA
  double t = 1.0;
  int it = 0;
  for (it = 1; it <= a.max_iter; ++it) {
    for (int r = threadIdx.x; r < nr; r += blockDim.x) {
      const float u = s.y[r] - (s.Gy[r] - s.bb[r]) * invL;
      const float zr = copysignf(fmaxf(fabsf(u) - thr, 0.f), u);
      s.z[r] = zr;
      s.pub[r] = zr;
    }
    cl.sync();
    gather(cl, s, a);
    __syncthreads();
    gemv_rows(s, a, r0, nr, s.Gz);
    __syncthreads();
    double v[NPART] = {0, 0, 0, 0, 0};
    for (int r = threadIdx.x; r < nr; r += blockDim.x) {
      const double zr = s.z[r];
      v[0] += zr * s.Gz[r];
      v[1] += (double)s.bb[r] * zr;
      v[2] += fabs(zr);
      const double d = zr - (double)s.y[r];
      v[3] += d * d;
      v[4] += zr * zr;
    }
    block_sums(v, s.part, scratch);
    cl.sync();
    double tot[NPART];
    cluster_sums(cl, s.part, s_tot, tot);
    const double Fz = 0.5 * tot[0] - tot[1] + (double)a.lam * tot[2];
    const double step = sqrt(tot[3]);
    const double nz = sqrt(tot[4]);
    const double t1 = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
    const bool accept = Fz <= Fx;
    const float c1 = (float)(t / t1), c2 = (float)((t - 1.0) / t1);
    for (int r = threadIdx.x; r < nr; r += blockDim.x) {
      const float xo = s.x[r], Gxo = s.Gx[r];
      const float xn = accept ? s.z[r] : xo;
      const float Gxn = accept ? s.Gz[r] : Gxo;
      s.y[r] = xn + c1 * (s.z[r] - xn) + c2 * (xn - xo);
      s.Gy[r] = Gxn + c1 * (s.Gz[r] - Gxn) + c2 * (Gxn - Gxo);
      s.x[r] = xn;
      s.Gx[r] = Gxn;
    }
    if (accept) Fx = Fz;
    t = t1;
    __syncthreads();
    if (step <= (double)a.eps * nz) break;
  }
  if (it > a.max_iter) it = a.max_iter;
  for (int r = threadIdx.x; r < nr; r += blockDim.x) a.x[r0 + r] = s.x[r];
  if (rank == 0 && threadIdx.x == 0) {
    if (a.out_iters) *a.out_iters = it;
    if (a.out_L) *a.out_L = L;
    if (a.out_F) *a.out_F = Fx;
  }
  cl.sync();   // no CTA leaves while others may still read its shared memory
}

}  // namespace

int run_apgd(const float* G, int ldg, const float* b, int S, double lambda, double eps,
             int max_iter, float* x, int* iters, double* L, double* Fx, cudaStream_t st) {
  if (S <= 0) return PC_OK;
  static int cs_max = 0;
  if (cs_max == 0) {
    cudaError_t e = cudaFuncSetAttribute(k_apgd, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cs_max = (e == cudaSuccess) ? 16 : 8;
    if (e != cudaSuccess) cudaGetLastError();
  }
  // cluster size: about 64 rows per CTA, a power of two, at most cs_max
  int CS = 1;
  while (CS < cs_max && CS * 64 < S) CS *= 2;
  const int n_pad = (S + 3) & ~3;
  int rows_per = ceil_div(S, CS);
  size_t base_bytes = sizeof(float) * ((size_t)n_pad + 8 * (size_t)rows_per) + 16 + 16 * sizeof(double);
  // (two partial-sum buffers of 8 doubles each follow the vectors)
  const size_t limit = 200 * 1024;
  if (base_bytes > limit)
    return fail(PC_ERR_CAPACITY, "apgd: support of %d atoms exceeds the cluster solver", S);
  const size_t cache_bytes = sizeof(float) * (size_t)rows_per * n_pad;
  const int cache = (base_bytes + cache_bytes <= limit) ? 1 : 0;
  const size_t smem = base_bytes + (cache ? cache_bytes : 0);
  PC_CUDA(cudaFuncSetAttribute(k_apgd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));

  ApgdArgs a;
  a.G = G;
  a.ldg = ldg;
  a.b = b;
  a.n = S;
  a.lam = (float)lambda;
  a.eps = (float)eps;
  a.max_iter = max_iter;
  a.x = x;
  a.out_iters = iters;
  a.out_L = L;
  a.out_F = Fx;
  a.rows_per = rows_per;
  a.n_pad = n_pad;
  a.cache = cache;
  a.vec_ok = ((ldg & 3) == 0 && (reinterpret_cast<uintptr_t>(G) & 15) == 0) ? 1 : 0;

  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CS, 1, 1);
  cfg.blockDim = dim3(APGD_THREADS, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e;
  {
    ProfScope prof_scope_(PROF_APGD, st);
    prof_scope_.kernels = 1;
    e = cudaLaunchKernelEx(&cfg, k_apgd, a);
  }
  if (e != cudaSuccess && CS == 16) {
    // fall back to a portable cluster size
    cudaGetLastError();
    cs_max = 8;
    return run_apgd(G, ldg, b, S, lambda, eps, max_iter, x, iters, L, Fx, st);
  }
  PC_CUDA(e);
  return PC_OK;
}

}  // namespace pc
