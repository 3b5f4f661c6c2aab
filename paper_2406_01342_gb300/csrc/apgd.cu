// Restricted LASSO solve of step 2 of Algorithm 2 by accelerated proximal
// gradient (FISTA, the APGD the paper names in Sect. 4.4 / 4.1) on the Gram
// form of the support problem:
//
//   f(x) = 1/2 x^T G x - b^T x + lambda ||x||_1,   G = Re(Phi_S^H Phi_S), b = Re(Phi_S^H V)
//
// Readings (the paper gives no constants): step 1/L with L = 1.01 x the
// largest eigenvalue of G; the monotone FISTA variant; stop when
// ||z - y|| <= eps ||z||. The eigenvalue comes from Lanczos on G started from
// the all-ones vector: the largest Ritz value of the tridiagonal matrix (by
// Sturm-count multisection), until it changes by < 1e-5 relative between
// checks every 4 steps, at most 64 steps (or n, or an invariant subspace).
// Ritz values approach the top eigenvalue from below and converge faster than
// linearly, so the 1 % margin of L covers the remaining error many times.
//
// GB300 mapping: one thread-block cluster, as few CTAs as let each CTA keep
// its rows of G in shared memory (1 CTA up to n ~ 220, 16 for n ~ 900). CTA r
// owns a contiguous block of rows of G and of every vector. Each iteration does
// one GEMV: the CTAs publish their slice of the proximal point z in shared
// memory, a cluster barrier, every CTA gathers the whole z through distributed
// shared memory, multiplies its rows, publishes its partial sums, a second
// barrier, and every CTA reduces the partials in the same order (so all take
// identical decisions). G z is the only matrix product per iteration: G y and
// G x are kept as linear combinations of previous products.
//
// Arithmetic: FP32 vectors and no float64 instruction in any loop (float64 has
// a low rate and long dependent latency on this GPU; it made an iteration take
// ~10 us). The monotone test F(z) <= F(x) needs the sign of a difference of two
// ~1e7 numbers: the full-vector kernel sums the difference directly as
// sum_i (z_i - x_i)((Gz_i + Gx_i)/2 - b_i) + lambda(|z_i| - |x_i|), whose terms
// all vanish as z -> x, in FP32; the row-slice kernel (large supports) carries
// the objective itself as double-float pairs (hi + lo, exact products and
// error-free sums, ~44 bits).
#include <cooperative_groups.h>

#include <cmath>

#include "lanczos.cuh"
#include "pc_internal.cuh"

namespace cg = cooperative_groups;

namespace pc {
namespace {

// ---- double-float arithmetic (Dekker / Knuth error-free transformations)
struct Df {
  float hi, lo;
};

__device__ __forceinline__ Df df_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return {s, e};
}
__device__ __forceinline__ Df df_add(Df a, Df b) {
  Df s = df_two_sum(a.hi, b.hi);
  const float e = s.lo + a.lo + b.lo;
  const float hi = s.hi + e;
  return {hi, e - (hi - s.hi)};
}
__device__ __forceinline__ Df df_prod(float a, float b) {   // exact a * b
  const float p = a * b;
  return {p, fmaf(a, b, -p)};
}
__device__ __forceinline__ Df df_scale(Df a, float b) {
  const float p = a.hi * b;
  float e = fmaf(a.hi, b, -p);
  e = fmaf(a.lo, b, e);
  const float hi = p + e;
  return {hi, e - (hi - p)};
}
__device__ __forceinline__ Df df_neg(Df a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ bool df_le(Df a, Df b) {          // a <= b
  const Df d = df_add(a, df_neg(b));
  return d.hi < 0.f || (d.hi == 0.f && d.lo <= 0.f);
}
__device__ __forceinline__ Df df_shfl_xor(Df a, int off) {
  return {__shfl_xor_sync(0xffffffffu, a.hi, off), __shfl_xor_sync(0xffffffffu, a.lo, off)};
}

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
  int* out_lanczos;
  int* err;       // set to 1 if a bounded wait expired (may be null)
  int positive;   // 1: x >= 0 (proximal map max(z - lambda/L, 0))
  int rows_per;
  int n_pad;
  int cache;      // 1: rows of G cached in shared memory
  int vec_ok;     // 1: float4 loads of G rows are aligned
};

// Rows [r0, r0 + nr) of G (leading dimension ldg, n columns) into dst (row
// stride ld floats, ld a multiple of 4, dst 16-byte aligned), columns [n, ld)
// zero, by asynchronous copies: a warp per row, no register round trip per
// element, so every load of the block is in flight at once. The calling
// thread's copies are complete on return; the caller's barrier publishes them.
__device__ void load_rows_async(float* dst, int ld, const float* __restrict__ G, int ldg, int r0, int nr,
                                int n, bool vec) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int r = warp; r < nr; r += nw) {
    const float* src = G + (size_t)(r0 + r) * ldg;
    float* d = dst + (size_t)r * ld;
    if (vec) {
      for (int c = 4 * lane; c < ld; c += 128) {
        const int bytes = max(0, min(16, (n - c) * 4));
        const uint32_t da = (uint32_t)__cvta_generic_to_shared(d + c);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(da), "l"(bytes > 0 ? src + c : src),
                     "r"(bytes)
                     : "memory");
      }
    } else {
      for (int c = lane; c < ld; c += 32) {
        if (c < n) {
          const uint32_t da = (uint32_t)__cvta_generic_to_shared(d + c);
          asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(da), "l"(src + c) : "memory");
        } else {
          d[c] = 0.f;
        }
      }
    }
  }
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// Several independent restricted problems in one launch: cluster c of the
// grid solves job c (all jobs of a launch share the cluster size).
constexpr int APGD_BATCH_MAX = 16;
struct ApgdBatch {
  ApgdArgs job[APGD_BATCH_MAX];
  int n_jobs;
};

constexpr int APGD_THREADS = 256;
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
  Df* part;       // 2 buffers of 8 partial sums (the second for back-to-back reductions)
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
  s.part = reinterpret_cast<Df*>(p); p += 2 * 16;
  s.Gc = p;
  return s;
}

// Gather the published slices of every CTA into zfull.
__device__ void gather(cg::cluster_group& cl, const Smem& s, const ApgdArgs& a) {
  for (int idx = threadIdx.x; idx < a.n; idx += blockDim.x) {
    const int rr = idx / a.rows_per;
    const int off = idx - rr * a.rows_per;
    const float* remote = cl.map_shared_rank(s.pub, rr);
    s.zfull[idx] = remote[off];
  }
  for (int idx = a.n + threadIdx.x; idx < a.n_pad; idx += blockDim.x) s.zfull[idx] = 0.f;
}

// out[r] = G[r0 + r, :] . zfull for the nr own rows. A warp takes 4 rows at
// a time (independent accumulators and shuffle chains, so their latencies
// overlap); full float4 groups inside [0, n), then a scalar tail: columns >= n
// of a caller's G are never read.
__device__ void gemv_rows(const Smem& s, const ApgdArgs& a, int r0, int nr, float* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const bool vec = a.cache || a.vec_ok;
  const int n4 = a.n >> 2;
  const float4* z4 = reinterpret_cast<const float4*>(s.zfull);
  for (int rb = 4 * warp; rb < nr; rb += 4 * nw) {
    const float* rows[4];
    float acc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int r = min(rb + q, nr - 1);
      rows[q] = a.cache ? s.Gc + (size_t)r * a.n_pad : a.G + (size_t)(r0 + r) * a.ldg;
      acc[q] = 0.f;
    }
    if (vec) {
      for (int c = lane; c < n4; c += 32) {
        const float4 z = z4[c];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float4 g = reinterpret_cast<const float4*>(rows[q])[c];
          acc[q] = fmaf(g.x, z.x, acc[q]);
          acc[q] = fmaf(g.y, z.y, acc[q]);
          acc[q] = fmaf(g.z, z.z, acc[q]);
          acc[q] = fmaf(g.w, z.w, acc[q]);
        }
      }
      for (int c = 4 * n4 + lane; c < a.n; c += 32)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] = fmaf(rows[q][c], s.zfull[c], acc[q]);
    } else {
      for (int c = lane; c < a.n; c += 32)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] = fmaf(rows[q][c], s.zfull[c], acc[q]);
    }
    for (int off = 16; off; off >>= 1)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], off);
    if (lane < 4 && rb + lane < nr) {
      float v = acc[0];
#pragma unroll
      for (int q = 1; q < 4; ++q)
        if (lane == q) v = acc[q];
      out[rb + lane] = v;
    }
  }
}

// Block-wide double-float sums of NPART per-thread values, written to part[] by thread 0.
__device__ void block_sums(Df v[NPART], Df* part, Df* scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int off = 16; off; off >>= 1)
#pragma unroll
    for (int q = 0; q < NPART; ++q) v[q] = df_add(v[q], df_shfl_xor(v[q], off));
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < NPART; ++q) scratch[warp * NPART + q] = v[q];
  __syncthreads();
  if (warp == 0) {   // the nw (<= 8) warp sums: a 3-level butterfly in warp 0
#pragma unroll
    for (int q = 0; q < NPART; ++q) v[q] = lane < nw ? scratch[lane * NPART + q] : Df{0.f, 0.f};
    for (int off = 4; off; off >>= 1)
#pragma unroll
      for (int q = 0; q < NPART; ++q) v[q] = df_add(v[q], df_shfl_xor(v[q], off));
    if (lane < NPART) {
      Df t = v[0];
#pragma unroll
      for (int q = 1; q < NPART; ++q)
        if (lane == q) t = v[q];
      part[lane] = t;
    }
  }
  __syncthreads();
}

// Sum the published partials of all CTAs: warp 0 reads each CTA's partials
// once over distributed shared memory and reduces them with a fixed butterfly
// (the same order in every CTA, so every CTA takes the same decisions).
__device__ void cluster_sums(cg::cluster_group& cl, Df* part, Df* s_tot, Df out[NPART]) {
  const int CS = (int)cl.num_blocks();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    const Df* rp = lane < CS ? cl.map_shared_rank(part, lane) : nullptr;
    Df v[NPART];
#pragma unroll
    for (int q = 0; q < NPART; ++q) v[q] = rp ? rp[q] : Df{0.f, 0.f};
    for (int off = 16; off; off >>= 1)
#pragma unroll
      for (int q = 0; q < NPART; ++q) v[q] = df_add(v[q], df_shfl_xor(v[q], off));
    if (lane == 0)
#pragma unroll
      for (int q = 0; q < NPART; ++q) s_tot[q] = v[q];
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NPART; ++q) out[q] = s_tot[q];
}

__global__ void __launch_bounds__(APGD_THREADS, 1) k_apgd(const __grid_constant__ ApgdBatch batch) {
  extern __shared__ __align__(16) float apgd_sm[];
  __shared__ Df scratch[(APGD_THREADS / 32) * NPART];
  __shared__ Df s_tot[NPART];
  __shared__ float s_al[LZ_MAX], s_be[LZ_MAX], s_theta;
  cg::cluster_group cl = cg::this_cluster();
  const ApgdArgs& a = batch.job[blockIdx.x / cl.num_blocks()];
  const int rank = (int)cl.block_rank();
  const Smem s = carve(apgd_sm, a);
  const int r0 = rank * a.rows_per;
  const int nr = max(0, min(a.n, r0 + a.rows_per) - r0);
  Df* part2 = s.part + 8;

  if (a.cache) load_rows_async(s.Gc, a.n_pad, a.G, a.ldg, r0, nr, a.n, a.vec_ok != 0);
  const float v0 = rsqrtf((float)a.n);        // Lanczos start: all ones / sqrt(n)
  for (int r = threadIdx.x; r < a.rows_per; r += blockDim.x) {
    const bool own = r < nr;
    s.bb[r] = own ? a.b[r0 + r] : 0.f;
    s.x[r] = own ? a.x[r0 + r] : 0.f;
    s.y[r] = own ? v0 : 0.f;    // v_j
    s.z[r] = 0.f;               // v_{j-1}
    s.pub[r] = own ? v0 : 0.f;
  }
  __syncthreads();

  // ---- Lipschitz constant: Lanczos (alpha = v^T G v, then beta = ||w||)
  float theta = 0.f, theta_prev = 0.f, beta_prev = 0.f;
  int m = 0;
  for (int j = 0; j < LZ_MAX; ++j) {
    cl.sync();
    gather(cl, s, a);
    __syncthreads();
    gemv_rows(s, a, r0, nr, s.Gz);                  // w = G v_j
    __syncthreads();
    Df v[NPART] = {};
    for (int r = threadIdx.x; r < nr; r += blockDim.x) v[0] = df_add(v[0], df_prod(s.y[r], s.Gz[r]));
    block_sums(v, s.part, scratch);
    cl.sync();
    Df tot[NPART];
    cluster_sums(cl, s.part, s_tot, tot);
    const float alpha = tot[0].hi + tot[0].lo;
    Df v2[NPART] = {};
    for (int r = threadIdx.x; r < nr; r += blockDim.x) {
      const float w = s.Gz[r] - alpha * s.y[r] - beta_prev * s.z[r];
      s.Gz[r] = w;
      v2[0] = df_add(v2[0], df_prod(w, w));
    }
    block_sums(v2, part2, scratch);
    cl.sync();
    cluster_sums(cl, part2, s_tot, tot);
    const float beta = sqrtf(fmaxf(tot[0].hi + tot[0].lo, 0.f));
    if (threadIdx.x == 0) {
      s_al[j] = alpha;
      s_be[j] = beta;
    }
    m = j + 1;
    __syncthreads();
    const bool last = (m == a.n) || (m == LZ_MAX) || !(beta > 1e-7f * fabsf(alpha));
    if (last || (m % 4) == 0) {
      theta = tridiag_top(s_al, s_be, m, &s_theta);
      if (last || fabsf(theta - theta_prev) <= LZ_TOL * fabsf(theta)) break;
      theta_prev = theta;
    }
    const float inv = 1.f / beta;
    for (int r = threadIdx.x; r < nr; r += blockDim.x) {
      const float vn = s.Gz[r] * inv;
      s.z[r] = s.y[r];
      s.y[r] = vn;
      s.pub[r] = vn;
    }
    beta_prev = beta;
  }
  const float L = 1.01f * (theta > 0.f ? theta : 1.f);
  const float invL = 1.f / L;
  const float thr = a.lam * invL;

  // ---- initial G x
  for (int r = threadIdx.x; r < nr; r += blockDim.x) s.pub[r] = s.x[r];
  cl.sync();
  gather(cl, s, a);
  __syncthreads();
  gemv_rows(s, a, r0, nr, s.Gx);
  __syncthreads();
  Df Fx;
  {
    Df v[NPART] = {};
    for (int r = threadIdx.x; r < nr; r += blockDim.x) {
      v[0] = df_add(v[0], df_prod(s.x[r], s.Gx[r]));
      v[1] = df_add(v[1], df_prod(s.bb[r], s.x[r]));
      v[2] = df_add(v[2], Df{fabsf(s.x[r]), 0.f});
    }
    block_sums(v, s.part, scratch);
    cl.sync();
    Df tot[NPART];
    cluster_sums(cl, s.part, s_tot, tot);
    Fx = df_add(df_add(df_scale(tot[0], 0.5f), df_neg(tot[1])), df_scale(tot[2], a.lam));
  }
  for (int r = threadIdx.x; r < nr; r += blockDim.x) {
    s.y[r] = s.x[r];
    s.Gy[r] = s.Gx[r];
  }
  __syncthreads();

  // ---- monotone FISTA
  float t = 1.f;
  int it = 0;
  for (it = 1; it <= a.max_iter; ++it) {
    for (int r = threadIdx.x; r < nr; r += blockDim.x) {
      const float u = s.y[r] - (s.Gy[r] - s.bb[r]) * invL;
      const float zr = (a.positive ? fmaxf(u - thr, 0.f) : copysignf(fmaxf(fabsf(u) - thr, 0.f), u));
      s.z[r] = zr;
      s.pub[r] = zr;
    }
    cl.sync();
    gather(cl, s, a);
    __syncthreads();
    gemv_rows(s, a, r0, nr, s.Gz);
    __syncthreads();
    Df v[NPART] = {};
    for (int r = threadIdx.x; r < nr; r += blockDim.x) {
      const float zr = s.z[r];
      v[0] = df_add(v[0], df_prod(zr, s.Gz[r]));
      v[1] = df_add(v[1], df_prod(s.bb[r], zr));
      v[2] = df_add(v[2], Df{fabsf(zr), 0.f});
      const float d = zr - s.y[r];
      v[3] = df_add(v[3], df_prod(d, d));
      v[4] = df_add(v[4], df_prod(zr, zr));
    }
    block_sums(v, s.part, scratch);
    cl.sync();
    Df tot[NPART];
    cluster_sums(cl, s.part, s_tot, tot);
    const Df Fz = df_add(df_add(df_scale(tot[0], 0.5f), df_neg(tot[1])), df_scale(tot[2], a.lam));
    const float step = sqrtf(tot[3].hi + tot[3].lo);
    const float nz = sqrtf(tot[4].hi + tot[4].lo);
    const float t1 = 0.5f * (1.f + sqrtf(1.f + 4.f * t * t));
    const bool accept = df_le(Fz, Fx);
    const float c1 = t / t1, c2 = (t - 1.f) / t1;
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
    if (step <= a.eps * nz) break;
  }
  if (it > a.max_iter) it = a.max_iter;
  for (int r = threadIdx.x; r < nr; r += blockDim.x) a.x[r0 + r] = s.x[r];
  if (rank == 0 && threadIdx.x == 0) {
    if (a.out_iters) *a.out_iters = it;
    if (a.out_L) *a.out_L = (double)L;
    if (a.out_F) *a.out_F = (double)Fx.hi + (double)Fx.lo;
    if (a.out_lanczos) *a.out_lanczos = m;
  }
  cl.sync();   // no CTA leaves while others may still read its shared memory
}

// Block-wide FP32 sums of K per-thread values (a fixed butterfly: the same
// inputs give the same sums in every CTA); every thread receives them.
template <int K>
__device__ void block_sum_f(float (&v)[K], float* scratch, float* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int off = 16; off; off >>= 1)
#pragma unroll
    for (int q = 0; q < K; ++q) v[q] += __shfl_xor_sync(0xffffffffu, v[q], off);
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < K; ++q) scratch[warp * K + q] = v[q];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < K; ++q) v[q] = lane < nw ? scratch[lane * K + q] : 0.f;
    for (int off = 4; off; off >>= 1)
#pragma unroll
      for (int q = 0; q < K; ++q) v[q] += __shfl_xor_sync(0xffffffffu, v[q], off);
    if (lane == 0)
#pragma unroll
      for (int q = 0; q < K; ++q) out[q] = v[q];
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < K; ++q) v[q] = out[q];
}

// ---------------------------------------------------------------------------
// Full-vector variant (used whenever its vectors fit): every CTA keeps all n
// entries of x, y, z, Gx, Gy and b, and owns rows [r0, r0 + nr) of G (nr a
// multiple of 4 except in the last CTA). A matrix-vector product multiplies
// the own rows by the (local) full vector into a local slice and PUSHES the
// slice to every CTA of the cluster with one bulk copy each (shared memory to
// distributed shared memory), whose bytes complete on the receiver's
// mbarrier; each CTA then waits (bounded) on its own mbarrier until all
// entries have landed. No cluster barrier and no remote loads sit on the
// iteration path, only the one-way latency of the copies.
// The reductions and updates are then done redundantly over all n entries --
// identical data and order in every CTA, hence identical decisions.
//
// Two receive buffers (and two local slices) alternate. A CTA pushes product
// i + 2 into buffer i mod 2 only after it has received every CTA's product
// i + 1, which each CTA sends only after it has consumed product i and
// re-armed that buffer's mbarrier, so a buffer is never overwritten while it
// is read, bytes never arrive before the phase that counts them is armed, and
// a local slice is rewritten only after every copy that read it has landed.

constexpr long long APGD_WAIT_CYCLES = 4000000000ll;   // ~2 s at 2 GHz

struct SmemF {
  float* pub0;    // rows_per each: this CTA's slices of the last two products
  float* pub1;
  float* rx0;     // n_pad each: the two receive buffers of the products
  float* rx1;
  float* x;       // n_pad each, full vectors
  float* Gx;
  float* y;
  float* Gy;
  float* z;
  float* bb;
  float* Gc;      // rows_per x n_pad (optional)
};

__device__ SmemF carve_full(float* base, const ApgdArgs& a) {
  SmemF s;
  float* p = base;
  s.pub0 = p; p += a.rows_per;
  s.pub1 = p; p += a.rows_per;
  s.rx0 = p; p += a.n_pad;
  s.rx1 = p; p += a.n_pad;
  s.x = p; p += a.n_pad;
  s.Gx = p; p += a.n_pad;
  s.y = p; p += a.n_pad;
  s.Gy = p; p += a.n_pad;
  s.z = p; p += a.n_pad;
  s.bb = p; p += a.n_pad;
  s.Gc = p;
  return s;
}

__device__ __forceinline__ uint32_t cluster_addr(uint32_t saddr, int rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
  return r;
}
__device__ __forceinline__ void mbar_arm(uint32_t mbar, uint32_t tx) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(tx) : "memory");
}
__device__ __forceinline__ bool mbar_try_cluster(uint32_t mbar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(done)
      : "r"(mbar), "r"(parity)
      : "memory");
  return done != 0;
}
__device__ bool mbar_wait_cluster(uint32_t mbar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try_cluster(mbar, parity))
    if (clock64() - t0 > APGD_WAIT_CYCLES) return false;
  return true;
}

struct Exchange {
  uint32_t rx0, rx1;     // shared::cta addresses of the receive buffers
  uint32_t bar0, bar1;   // ... and of their mbarriers
  uint32_t phase;        // parity bit per buffer
  int buf;
  int CS;
  __device__ uint32_t rx(int b) const { return b ? rx1 : rx0; }
  __device__ uint32_t bar(int b) const { return b ? bar1 : bar0; }
};

// G vec for all n rows, in every CTA; returns the receive buffer holding it.
// *ok becomes false (in every thread of the CTA) if the bounded wait expired.
__device__ float* cluster_gemv(const ApgdArgs& a, const SmemF& s, const float* vec, int r0, int nr,
                               Exchange& ex, bool& ok) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int b = ex.buf;
  // a one-CTA cluster writes the product straight into its receive buffer: no
  // bulk copy to itself, no mbarrier round trip
  const bool solo = ex.CS == 1;
  float* pub = solo ? (b ? s.rx1 : s.rx0) : (b ? s.pub1 : s.pub0);
  const bool vecld = a.cache || a.vec_ok;
  const int n4 = a.n >> 2;
  const float4* v4 = reinterpret_cast<const float4*>(vec);
  for (int rb = 4 * warp; rb < nr; rb += 4 * nw) {
    const float* rows[4];
    float acc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int r = min(rb + q, nr - 1);
      rows[q] = a.cache ? s.Gc + (size_t)r * a.n_pad : a.G + (size_t)(r0 + r) * a.ldg;
      acc[q] = 0.f;
    }
    if (vecld) {
      for (int c = lane; c < n4; c += 32) {
        const float4 z = v4[c];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float4 g = reinterpret_cast<const float4*>(rows[q])[c];
          acc[q] = fmaf(g.x, z.x, acc[q]);
          acc[q] = fmaf(g.y, z.y, acc[q]);
          acc[q] = fmaf(g.z, z.z, acc[q]);
          acc[q] = fmaf(g.w, z.w, acc[q]);
        }
      }
      for (int c = 4 * n4 + lane; c < a.n; c += 32)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] = fmaf(rows[q][c], vec[c], acc[q]);
    } else {
      for (int c = lane; c < a.n; c += 32)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] = fmaf(rows[q][c], vec[c], acc[q]);
    }
    for (int off = 16; off; off >>= 1)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], off);
    if (lane < 4 && rb + lane < nr) {
      float v = acc[0];
#pragma unroll
      for (int q = 1; q < 4; ++q)
        if (lane == q) v = acc[q];
      pub[rb + lane] = v;
    }
  }
  // the slice (padded to 4 floats) goes to every CTA in one bulk copy each
  const int nr4 = (nr + 3) & ~3;
  for (int r = nr + threadIdx.x; r < nr4; r += blockDim.x) pub[r] = 0.f;
  if (solo) {
    __syncthreads();
    ex.buf ^= 1;
    return pub;
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  if ((int)threadIdx.x < ex.CS && nr4 > 0) {
    const int d = threadIdx.x;
    const uint32_t src = (uint32_t)__cvta_generic_to_shared(pub);
    const uint32_t dst = cluster_addr(ex.rx(b) + (uint32_t)r0 * 4u, d);
    asm volatile(
        "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "r"(src), "r"((uint32_t)nr4 * 4u), "r"(cluster_addr(ex.bar(b), d))
        : "memory");
  }
  const bool mine = mbar_wait_cluster(ex.bar(b), (ex.phase >> b) & 1u);
  ok = !__syncthreads_or(!mine);
  if (ok) {
    ex.phase ^= 1u << b;
    ex.buf ^= 1;
    // re-arm for this buffer's next use (two products from now)
    if (threadIdx.x == 0) mbar_arm(ex.bar(b), (uint32_t)a.n_pad * 4u);
  }
  return b ? s.rx1 : s.rx0;
}

__global__ void __launch_bounds__(APGD_THREADS, 1) k_apgd_full(const __grid_constant__ ApgdBatch batch) {
  extern __shared__ __align__(16) float apgdf_sm[];
  __shared__ Df scratch[(APGD_THREADS / 32) * NPART];
  __shared__ Df s_part[NPART];
  __shared__ float s_fscr[(APGD_THREADS / 32) * 3], s_fout[3];
  __shared__ float s_al[LZ_MAX], s_be[LZ_MAX], s_theta;
  __shared__ __align__(8) uint64_t s_rxbar[2];
  cg::cluster_group cl = cg::this_cluster();
  const ApgdArgs& a = batch.job[blockIdx.x / cl.num_blocks()];
  const int rank = (int)cl.block_rank();
  const SmemF s = carve_full(apgdf_sm, a);
  const int r0 = rank * a.rows_per;
  const int nr = max(0, min(a.n, r0 + a.rows_per) - r0);
  const int n = a.n, tid = threadIdx.x, nt = blockDim.x;
  bool ok = true;

  Exchange ex;
  ex.rx0 = (uint32_t)__cvta_generic_to_shared(s.rx0);
  ex.rx1 = (uint32_t)__cvta_generic_to_shared(s.rx1);
  ex.bar0 = (uint32_t)__cvta_generic_to_shared(&s_rxbar[0]);
  ex.bar1 = (uint32_t)__cvta_generic_to_shared(&s_rxbar[1]);
  ex.phase = 0;
  ex.buf = 0;
  ex.CS = (int)cl.num_blocks();
  if (tid == 0) {
    for (int b = 0; b < 2; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(ex.bar(b)));
      mbar_arm(ex.bar(b), (uint32_t)a.n_pad * 4u);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }

  if (a.cache) load_rows_async(s.Gc, a.n_pad, a.G, a.ldg, r0, nr, n, a.vec_ok != 0);
  const float v0 = rsqrtf((float)n);        // Lanczos start: all ones / sqrt(n)
  for (int i = tid; i < a.n_pad; i += nt) {
    const bool in = i < n;
    s.bb[i] = in ? a.b[i] : 0.f;
    s.x[i] = in ? a.x[i] : 0.f;
    s.y[i] = in ? v0 : 0.f;   // v_j
    s.z[i] = 0.f;             // v_{j-1}
  }
  cl.sync();   // every CTA's mbarriers are initialised and armed before any push

  // ---- Lipschitz constant: Lanczos (alpha = v^T G v, then beta = ||w||)
  float theta = 0.f, theta_prev = 0.f, beta_prev = 0.f;
  int m = 0;
  for (int j = 0; j < LZ_MAX && ok; ++j) {
    float* Gv = cluster_gemv(a, s, s.y, r0, nr, ex, ok);       // G v_j
    if (!ok) break;
    float va[1] = {0.f};
    for (int i = tid; i < n; i += nt) va[0] = fmaf(s.y[i], Gv[i], va[0]);
    block_sum_f<1>(va, s_fscr, s_fout);
    const float alpha = va[0];
    float vb[1] = {0.f};
    for (int i = tid; i < n; i += nt) {
      const float w = Gv[i] - alpha * s.y[i] - beta_prev * s.z[i];
      Gv[i] = w;
      vb[0] = fmaf(w, w, vb[0]);
    }
    block_sum_f<1>(vb, s_fscr, s_fout);
    const float beta = sqrtf(fmaxf(vb[0], 0.f));
    if (tid == 0) {
      s_al[j] = alpha;
      s_be[j] = beta;
    }
    m = j + 1;
    __syncthreads();
    const bool last = (m == n) || (m == LZ_MAX) || !(beta > 1e-7f * fabsf(alpha));
    if (last || (m % 4) == 0) {
      theta = tridiag_top(s_al, s_be, m, &s_theta);
      if (last || fabsf(theta - theta_prev) <= LZ_TOL * fabsf(theta)) break;
      theta_prev = theta;
    }
    const float inv = 1.f / beta;
    for (int i = tid; i < n; i += nt) {
      const float vn = Gv[i] * inv;
      s.z[i] = s.y[i];
      s.y[i] = vn;
    }
    beta_prev = beta;
    __syncthreads();
  }
  const float L = 1.01f * (theta > 0.f ? theta : 1.f);
  const float invL = 1.f / L;
  const float thr = a.lam * invL;

  // ---- initial G x
  if (ok) {
    const float* Gxr = cluster_gemv(a, s, s.x, r0, nr, ex, ok);
    if (ok) {
      for (int i = tid; i < n; i += nt) {
        const float gx = Gxr[i];
        s.Gx[i] = gx;
        s.y[i] = s.x[i];
        s.Gy[i] = gx;
      }
      __syncthreads();
    }
  }

  // ---- monotone FISTA
  float t = 1.f;
  int it = 0;
  for (it = 1; it <= a.max_iter && ok; ++it) {
    for (int i = tid; i < n; i += nt) {
      const float u = s.y[i] - (s.Gy[i] - s.bb[i]) * invL;
      s.z[i] = (a.positive ? fmaxf(u - thr, 0.f) : copysignf(fmaxf(fabsf(u) - thr, 0.f), u));
    }
    __syncthreads();
    const float* Gz = cluster_gemv(a, s, s.z, r0, nr, ex, ok);
    if (!ok) break;
    // F(z) - F(x) = sum_i (z_i - x_i) ((Gz_i + Gx_i) / 2 - b_i) + lambda (|z_i| - |x_i|)
    // (G symmetric): every term vanishes as z -> x, so an FP32 sum resolves the
    // sign of the difference where F itself (~1e7) would need ~50 bits
    float v[3] = {0.f, 0.f, 0.f};
    for (int i = tid; i < n; i += nt) {
      const float zr = s.z[i], xr = s.x[i];
      const float dF = fmaf(zr - xr, 0.5f * (Gz[i] + s.Gx[i]) - s.bb[i], a.lam * (fabsf(zr) - fabsf(xr)));
      v[0] += dF;
      const float d = zr - s.y[i];
      v[1] = fmaf(d, d, v[1]);
      v[2] = fmaf(zr, zr, v[2]);
    }
    block_sum_f<3>(v, s_fscr, s_fout);
    const float step = sqrtf(v[1]);
    const float nz = sqrtf(v[2]);
    const float t1 = 0.5f * (1.f + sqrtf(1.f + 4.f * t * t));
    const bool accept = v[0] <= 0.f;
    const float c1 = t / t1, c2 = (t - 1.f) / t1;
    for (int i = tid; i < n; i += nt) {
      const float xo = s.x[i], Gxo = s.Gx[i];
      const float xn = accept ? s.z[i] : xo;
      const float Gxn = accept ? Gz[i] : Gxo;
      s.y[i] = xn + c1 * (s.z[i] - xn) + c2 * (xn - xo);
      s.Gy[i] = Gxn + c1 * (Gz[i] - Gxn) + c2 * (Gxn - Gxo);
      s.x[i] = xn;
      s.Gx[i] = Gxn;
    }
    t = t1;
    __syncthreads();
    if (step <= a.eps * nz) break;
  }
  if (it > a.max_iter) it = a.max_iter;
  // objective of the returned x, in double-float (reported only)
  Df Fx = {0.f, 0.f};
  if (ok) {
    Df v[NPART] = {};
    for (int i = tid; i < n; i += nt) {
      v[0] = df_add(v[0], df_prod(s.x[i], s.Gx[i]));
      v[1] = df_add(v[1], df_prod(s.bb[i], s.x[i]));
      v[2] = df_add(v[2], Df{fabsf(s.x[i]), 0.f});
    }
    block_sums(v, s_part, scratch);
    Fx = df_add(df_add(df_scale(s_part[0], 0.5f), df_neg(s_part[1])), df_scale(s_part[2], a.lam));
  }
  if (ok) {
    for (int r = tid; r < nr; r += nt) a.x[r0 + r] = s.x[r0 + r];
    if (rank == 0 && tid == 0) {
      if (a.out_iters) *a.out_iters = it;
      if (a.out_L) *a.out_L = (double)L;
      if (a.out_F) *a.out_F = (double)Fx.hi + (double)Fx.lo;
      if (a.out_lanczos) *a.out_lanczos = m;
    }
  } else {
    // a wait expired: report it, and give pushes still addressed to this CTA
    // (bounded) time to land before it leaves
    if (tid == 0) {
      if (a.err) atomicExch(a.err, 1);
      mbar_wait_cluster(ex.bar(ex.buf), (ex.phase >> ex.buf) & 1u);
    }
    __syncthreads();
  }
  cl.sync();   // no CTA leaves while others may still address its shared memory
}

// ---------------------------------------------------------------------------
// One-warp variant for small supports (n <= 64, the later Frank-Wolfe
// iterations): the same Lanczos step size, monotone FISTA, stop rule and
// reported objective as k_apgd_full, with G in shared memory, lane l owning
// rows l and l + 32 of every vector, warp-shuffle reductions and no block or
// cluster barrier in the loop: an iteration is a few hundred instructions.
constexpr int WARP_NMAX = 64;

__device__ __forceinline__ float warp_sum(float v) {
  for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}
__device__ __forceinline__ Df warp_df_sum(Df v) {
  for (int off = 16; off; off >>= 1) v = df_add(v, df_shfl_xor(v, off));
  return v;
}

__global__ void __launch_bounds__(32) k_apgd_warp(const __grid_constant__ ApgdBatch batch) {
  __shared__ __align__(16) float vs[WARP_NMAX];
  __shared__ float s_al[LZ_MAX], s_be[LZ_MAX], s_theta;
  const ApgdArgs& a = batch.job[blockIdx.x];
  const int n = a.n, lane = threadIdx.x;
  const int i0 = lane, i1 = lane + 32;
  const bool v0ok = i0 < n, v1ok = i1 < n;
  // the lane's two rows of G live in registers (zero beyond n): every load in
  // flight at once, and a product reads only the broadcast input vector
  float g0[WARP_NMAX], g1[WARP_NMAX];
#pragma unroll
  for (int j = 0; j < WARP_NMAX; ++j) {
    g0[j] = (v0ok && j < n) ? a.G[(size_t)i0 * a.ldg + j] : 0.f;
    g1[j] = (v1ok && j < n) ? a.G[(size_t)i1 * a.ldg + j] : 0.f;
  }
  float bb0 = v0ok ? a.b[i0] : 0.f, bb1 = v1ok ? a.b[i1] : 0.f;
  float x0 = v0ok ? a.x[i0] : 0.f, x1 = v1ok ? a.x[i1] : 0.f;
  // G v for the lane's two rows (v broadcast through shared memory, 16-byte
  // reads; four partial sums per row for independent FMA chains)
  auto gemv = [&](float v0, float v1, float& g0o, float& g1o) {
    vs[i0] = v0;
    vs[i1] = v1;
    __syncwarp();
    float p0[4] = {0.f, 0.f, 0.f, 0.f}, p1[4] = {0.f, 0.f, 0.f, 0.f};
    const float4* v4 = reinterpret_cast<const float4*>(vs);
#pragma unroll
    for (int j4 = 0; j4 < WARP_NMAX / 4; ++j4) {
      const float4 z = v4[j4];
      p0[0] = fmaf(g0[4 * j4], z.x, p0[0]);
      p0[1] = fmaf(g0[4 * j4 + 1], z.y, p0[1]);
      p0[2] = fmaf(g0[4 * j4 + 2], z.z, p0[2]);
      p0[3] = fmaf(g0[4 * j4 + 3], z.w, p0[3]);
      p1[0] = fmaf(g1[4 * j4], z.x, p1[0]);
      p1[1] = fmaf(g1[4 * j4 + 1], z.y, p1[1]);
      p1[2] = fmaf(g1[4 * j4 + 2], z.z, p1[2]);
      p1[3] = fmaf(g1[4 * j4 + 3], z.w, p1[3]);
    }
    __syncwarp();
    g0o = v0ok ? (p0[0] + p0[1]) + (p0[2] + p0[3]) : 0.f;
    g1o = v1ok ? (p1[0] + p1[1]) + (p1[2] + p1[3]) : 0.f;
  };

  // ---- Lipschitz constant: Lanczos from the all-ones vector
  const float vinit = rsqrtf((float)n);
  float y0 = v0ok ? vinit : 0.f, y1 = v1ok ? vinit : 0.f;   // v_j
  float z0 = 0.f, z1 = 0.f;                                 // v_{j-1}
  float theta = 0.f, theta_prev = 0.f, beta_prev = 0.f;
  int m = 0;
  for (int j = 0; j < LZ_MAX; ++j) {
    float g0, g1;
    gemv(y0, y1, g0, g1);
    const float alpha = warp_sum(fmaf(y0, g0, y1 * g1));
    const float w0 = g0 - alpha * y0 - beta_prev * z0;
    const float w1 = g1 - alpha * y1 - beta_prev * z1;
    const float beta = sqrtf(fmaxf(warp_sum(fmaf(w0, w0, w1 * w1)), 0.f));
    if (lane == 0) {
      s_al[j] = alpha;
      s_be[j] = beta;
    }
    m = j + 1;
    __syncwarp();
    const bool last = (m == n) || (m == LZ_MAX) || !(beta > 1e-7f * fabsf(alpha));
    if (last || (m % 4) == 0) {
      theta = tridiag_top(s_al, s_be, m, &s_theta);
      if (last || fabsf(theta - theta_prev) <= LZ_TOL * fabsf(theta)) break;
      theta_prev = theta;
    }
    const float inv = 1.f / beta;
    z0 = y0;
    z1 = y1;
    y0 = w0 * inv;
    y1 = w1 * inv;
    beta_prev = beta;
  }
  const float L = 1.01f * (theta > 0.f ? theta : 1.f);
  const float invL = 1.f / L;
  const float thr = a.lam * invL;

  // ---- monotone FISTA
  float Gx0, Gx1;
  gemv(x0, x1, Gx0, Gx1);
  y0 = x0;
  y1 = x1;
  float Gy0 = Gx0, Gy1 = Gx1;
  float t = 1.f;
  int it = 0;
  for (it = 1; it <= a.max_iter; ++it) {
    const float u0 = y0 - (Gy0 - bb0) * invL, u1 = y1 - (Gy1 - bb1) * invL;
    float zz0 = a.positive ? fmaxf(u0 - thr, 0.f) : copysignf(fmaxf(fabsf(u0) - thr, 0.f), u0);
    float zz1 = a.positive ? fmaxf(u1 - thr, 0.f) : copysignf(fmaxf(fabsf(u1) - thr, 0.f), u1);
    if (!v0ok) zz0 = 0.f;
    if (!v1ok) zz1 = 0.f;
    float Gz0, Gz1;
    gemv(zz0, zz1, Gz0, Gz1);
    // F(z) - F(x) from the difference itself (see k_apgd_full)
    const float dF = warp_sum(fmaf(zz0 - x0, 0.5f * (Gz0 + Gx0) - bb0, a.lam * (fabsf(zz0) - fabsf(x0))) +
                              fmaf(zz1 - x1, 0.5f * (Gz1 + Gx1) - bb1, a.lam * (fabsf(zz1) - fabsf(x1))));
    const float d0 = zz0 - y0, d1 = zz1 - y1;
    const float step = sqrtf(warp_sum(fmaf(d0, d0, d1 * d1)));
    const float nz = sqrtf(warp_sum(fmaf(zz0, zz0, zz1 * zz1)));
    const float t1 = 0.5f * (1.f + sqrtf(1.f + 4.f * t * t));
    const bool accept = dF <= 0.f;
    const float c1 = t / t1, c2 = (t - 1.f) / t1;
    const float xn0 = accept ? zz0 : x0, xn1 = accept ? zz1 : x1;
    const float Gxn0 = accept ? Gz0 : Gx0, Gxn1 = accept ? Gz1 : Gx1;
    y0 = xn0 + c1 * (zz0 - xn0) + c2 * (xn0 - x0);
    y1 = xn1 + c1 * (zz1 - xn1) + c2 * (xn1 - x1);
    Gy0 = Gxn0 + c1 * (Gz0 - Gxn0) + c2 * (Gxn0 - Gx0);
    Gy1 = Gxn1 + c1 * (Gz1 - Gxn1) + c2 * (Gxn1 - Gx1);
    x0 = xn0;
    x1 = xn1;
    Gx0 = Gxn0;
    Gx1 = Gxn1;
    t = t1;
    if (step <= a.eps * nz) break;
  }
  if (it > a.max_iter) it = a.max_iter;
  // objective of the returned x, in double-float (reported only)
  const Df xg = warp_df_sum(df_add(df_prod(x0, Gx0), df_prod(x1, Gx1)));
  const Df bx = warp_df_sum(df_add(df_prod(bb0, x0), df_prod(bb1, x1)));
  const Df l1 = warp_df_sum(df_add(Df{fabsf(x0), 0.f}, Df{fabsf(x1), 0.f}));
  const Df Fx = df_add(df_add(df_scale(xg, 0.5f), df_neg(bx)), df_scale(l1, a.lam));
  if (v0ok) a.x[i0] = x0;
  if (v1ok) a.x[i1] = x1;
  if (lane == 0) {
    if (a.out_iters) *a.out_iters = it;
    if (a.out_L) *a.out_L = (double)L;
    if (a.out_F) *a.out_F = (double)Fx.hi + (double)Fx.lo;
    if (a.out_lanczos) *a.out_lanczos = m;
  }
}

// ---------------------------------------------------------------------------
// One-CTA variant for mid-size supports (WARP_NMAX < n <= CTA_NMAX): the same
// Lanczos step size, monotone FISTA, stop rule and reported objective, with G
// cached in shared memory and thread i owning row i of every vector, so the
// matrix-vector product (thread i: its row of G against the broadcast input)
// and all elementwise steps need no exchange. A FISTA iteration crosses two
// block barriers (input vector complete; partial sums complete) instead of a
// cluster exchange and five barriers.
constexpr int CTA_NMAX = 224;
constexpr int CTA_LDG = 228;   // G row stride in floats: 16-byte aligned, 57 x 16 B (odd) so
                               // eight rows read by a 128-bit phase hit distinct banks

__device__ __forceinline__ float row_dot(const float* __restrict__ Grow, const float* __restrict__ v, int n4) {
  float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
  const float4* g4 = reinterpret_cast<const float4*>(Grow);
  const float4* v4 = reinterpret_cast<const float4*>(v);
#pragma unroll 4
  for (int c = 0; c < n4; ++c) {
    const float4 g = g4[c], z = v4[c];
    a0 = fmaf(g.x, z.x, a0);
    a1 = fmaf(g.y, z.y, a1);
    a2 = fmaf(g.z, z.z, a2);
    a3 = fmaf(g.w, z.w, a3);
  }
  return (a0 + a1) + (a2 + a3);
}

// Sum of K per-thread values over the block, the same in every thread (each
// adds the warps' partials in warp order). buf alternates between two
// halves, so back-to-back reductions need no extra barrier.
template <int K>
__device__ __forceinline__ void cta_sum(float (&v)[K], float* red, int& parity) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int off = 16; off; off >>= 1)
#pragma unroll
    for (int q = 0; q < K; ++q) v[q] += __shfl_xor_sync(0xffffffffu, v[q], off);
  float* buf = red + parity * (APGD_THREADS / 32) * 4;
  parity ^= 1;
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < K; ++q) buf[warp * 4 + q] = v[q];
  __syncthreads();
#pragma unroll
  for (int q = 0; q < K; ++q) {
    float t = 0.f;
    for (int w = 0; w < nw; ++w) t += buf[w * 4 + q];
    v[q] = t;
  }
}

__global__ void __launch_bounds__(APGD_THREADS, 1) k_apgd_cta(const __grid_constant__ ApgdBatch batch) {
  extern __shared__ __align__(16) float apgdc_sm[];
  __shared__ __align__(16) float vs[CTA_LDG];      // the broadcast input of a product
  __shared__ float s_red[2 * (APGD_THREADS / 32) * 4];
  __shared__ Df s_dred[(APGD_THREADS / 32) * 3];
  __shared__ float s_al[LZ_MAX], s_be[LZ_MAX], s_theta;
  const ApgdArgs& a = batch.job[blockIdx.x];
  float* Gc = apgdc_sm;                             // n rows of CTA_LDG floats
  const int n = a.n, tid = threadIdx.x;
  const int n4 = (n + 3) >> 2;
  load_rows_async(Gc, CTA_LDG, a.G, a.ldg, 0, n, n, a.vec_ok != 0);
  const bool own = tid < n;
  const float* Grow = Gc + (size_t)(own ? tid : 0) * CTA_LDG;
  const float bb = own ? a.b[tid] : 0.f;
  float x = own ? a.x[tid] : 0.f;
  int parity = 0;

  // ---- Lipschitz constant: Lanczos from the all-ones vector
  float v = own ? rsqrtf((float)n) : 0.f, vprev = 0.f;
  if (tid < CTA_LDG) vs[tid] = v;
  __syncthreads();
  float theta = 0.f, theta_prev = 0.f, beta_prev = 0.f;
  int m = 0;
  for (int j = 0; j < LZ_MAX; ++j) {
    const float g = own ? row_dot(Grow, vs, n4) : 0.f;
    float ra[1] = {v * g};
    cta_sum<1>(ra, s_red, parity);
    const float alpha = ra[0];
    const float w = own ? g - alpha * v - beta_prev * vprev : 0.f;
    float rb[1] = {w * w};
    cta_sum<1>(rb, s_red, parity);
    const float beta = sqrtf(fmaxf(rb[0], 0.f));
    if (tid == 0) {
      s_al[j] = alpha;
      s_be[j] = beta;
    }
    m = j + 1;
    const bool last = (m == n) || (m == LZ_MAX) || !(beta > 1e-7f * fabsf(alpha));
    if (last || (m % 4) == 0) {
      __syncthreads();                              // s_al, s_be written
      theta = tridiag_top(s_al, s_be, m, &s_theta);
      if (last || fabsf(theta - theta_prev) <= LZ_TOL * fabsf(theta)) break;
      theta_prev = theta;
    }
    vprev = v;
    v = w / beta;
    if (own) vs[tid] = v;                           // every read of vs ended before the sums
    beta_prev = beta;
    __syncthreads();
  }
  const float L = 1.01f * (theta > 0.f ? theta : 1.f);
  const float invL = 1.f / L;
  const float thr = a.lam * invL;

  // ---- initial G x
  __syncthreads();                                  // every read of vs ended
  if (own) vs[tid] = x;
  __syncthreads();
  float Gx = own ? row_dot(Grow, vs, n4) : 0.f;
  float y = x, Gy = Gx;
  __syncthreads();                                  // every read of vs ended

  // ---- monotone FISTA
  float t = 1.f;
  int it = 0;
  for (it = 1; it <= a.max_iter; ++it) {
    const float u = y - (Gy - bb) * invL;
    float z = a.positive ? fmaxf(u - thr, 0.f) : copysignf(fmaxf(fabsf(u) - thr, 0.f), u);
    if (!own) z = 0.f;
    if (own) vs[tid] = z;                           // the last product's reads ended before its sums
    __syncthreads();
    const float Gz = own ? row_dot(Grow, vs, n4) : 0.f;
    // F(z) - F(x) from the difference itself (see k_apgd_full)
    const float d = z - y;
    float r3[3] = {own ? fmaf(z - x, 0.5f * (Gz + Gx) - bb, a.lam * (fabsf(z) - fabsf(x))) : 0.f, d * d, z * z};
    cta_sum<3>(r3, s_red, parity);
    const float step = sqrtf(r3[1]);
    const float nz = sqrtf(r3[2]);
    const float t1 = 0.5f * (1.f + sqrtf(1.f + 4.f * t * t));
    const bool accept = r3[0] <= 0.f;
    const float c1 = t / t1, c2 = (t - 1.f) / t1;
    const float xn = accept ? z : x, Gxn = accept ? Gz : Gx;
    y = xn + c1 * (z - xn) + c2 * (xn - x);
    Gy = Gxn + c1 * (Gz - Gxn) + c2 * (Gxn - Gx);
    x = xn;
    Gx = Gxn;
    t = t1;
    if (step <= a.eps * nz) break;
  }
  if (it > a.max_iter) it = a.max_iter;
  // objective of the returned x, in double-float (reported only)
  {
    const int lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    Df p[3] = {df_prod(x, Gx), df_prod(bb, x), Df{fabsf(x), 0.f}};
    for (int off = 16; off; off >>= 1)
#pragma unroll
      for (int q = 0; q < 3; ++q) p[q] = df_add(p[q], df_shfl_xor(p[q], off));
    if (lane == 0)
#pragma unroll
      for (int q = 0; q < 3; ++q) s_dred[warp * 3 + q] = p[q];
    __syncthreads();
    if (tid == 0) {
      Df tot[3] = {};
      for (int w = 0; w < nw; ++w)
#pragma unroll
        for (int q = 0; q < 3; ++q) tot[q] = df_add(tot[q], s_dred[w * 3 + q]);
      const Df Fx = df_add(df_add(df_scale(tot[0], 0.5f), df_neg(tot[1])), df_scale(tot[2], a.lam));
      if (a.out_iters) *a.out_iters = it;
      if (a.out_L) *a.out_L = (double)L;
      if (a.out_F) *a.out_F = (double)Fx.hi + (double)Fx.lo;
      if (a.out_lanczos) *a.out_lanczos = m;
    }
  }
  if (own) a.x[tid] = x;
}

}  // namespace

namespace {

// Launch shape of one restricted problem: which kernel, cluster size, rows per
// CTA, whether the CTAs cache their rows of G, dynamic shared memory.
struct ApgdShape {
  bool warp = false;   // one-warp kernel (n <= WARP_NMAX)
  bool cta = false;    // one-CTA kernel (WARP_NMAX < n <= CTA_NMAX)
  bool full;
  int CS;
  int rows_per;
  int cache;
  int n_pad;
  size_t smem;
};

// dynamic shared memory ceilings: 227 KB per CTA minus the kernels' static arrays
constexpr size_t kLimitRows = 200 * 1024;
constexpr size_t kLimitFull = 226 * 1024;

int apgd_setup(int* cs_max_out) {
  static int cs_max = 0;
  static bool attrs_set = false;
  if (cs_max == 0) {
    cudaError_t e1 = cudaFuncSetAttribute(k_apgd, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaError_t e2 = cudaFuncSetAttribute(k_apgd_full, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cs_max = (e1 == cudaSuccess && e2 == cudaSuccess) ? 16 : 8;
    cudaGetLastError();
  }
  if (!attrs_set) {
    PC_CUDA(cudaFuncSetAttribute(k_apgd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLimitRows));
    PC_CUDA(cudaFuncSetAttribute(k_apgd_full, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kLimitFull));
    PC_CUDA(cudaFuncSetAttribute(k_apgd_cta, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(sizeof(float) * CTA_NMAX * CTA_LDG)));
    attrs_set = true;
  }
  *cs_max_out = cs_max;
  return PC_OK;
}

int apgd_shape(int S, int cs_max, ApgdShape* out) {
  const int n_pad = (S + 3) & ~3;
  // full-vector kernel: 2 local slices, 2 receive buffers and 6 full vectors
  // (+ cached rows of G); its slices hold a multiple of 4 rows (bulk copies)
  auto rows_full = [&](int cs) { return (ceil_div(S, cs) + 3) & ~3; };
  auto bytes_full = [&](int cs, bool cached) {
    const size_t rp = (size_t)rows_full(cs);
    return sizeof(float) * (2 * rp + 8 * (size_t)n_pad) + (cached ? sizeof(float) * rp * n_pad : 0);
  };
  // row-slice kernel (larger supports): one full vector + 8 row slices
  auto bytes_rows = [&](int cs, bool cached) {
    const size_t rp = (size_t)ceil_div(S, cs);
    return sizeof(float) * ((size_t)n_pad + 8 * rp) + 16 + 16 * sizeof(Df) +
           (cached ? sizeof(float) * rp * n_pad : 0);
  };
  // cluster size: the smallest power of two whose CTAs each cache at most
  // ~64 KB of G in shared memory (a matrix-vector product then streams it in
  // ~500 cycles), else the smallest that caches G at all, else cs_max
  ApgdShape sh;
  if (S <= WARP_NMAX) {
    sh.warp = true;
    sh.full = true;
    sh.CS = 1;
    sh.cache = 1;
    sh.smem = 0;
    sh.rows_per = S;
    sh.n_pad = n_pad;
    *out = sh;
    return PC_OK;
  }
  if (S <= CTA_NMAX) {
    sh.cta = true;
    sh.full = true;
    sh.CS = 1;
    sh.cache = 1;
    sh.smem = sizeof(float) * (size_t)S * CTA_LDG;
    sh.rows_per = S;
    sh.n_pad = n_pad;
    *out = sh;
    return PC_OK;
  }
  sh.full = true;
  sh.CS = 1;
  const size_t share_target = 64 * 1024;
  while (sh.CS < cs_max && (bytes_full(sh.CS, true) > kLimitFull ||
                            sizeof(float) * (size_t)rows_full(sh.CS) * n_pad > share_target))
    sh.CS *= 2;
  sh.cache = bytes_full(sh.CS, true) <= kLimitFull ? 1 : 0;
  sh.smem = bytes_full(sh.CS, sh.cache != 0);
  if (sh.smem > kLimitFull) {
    sh.full = false;
    sh.CS = 1;
    while (sh.CS < cs_max && bytes_rows(sh.CS, true) > kLimitRows) sh.CS *= 2;
    if (bytes_rows(sh.CS, false) > kLimitRows)
      return fail(PC_ERR_CAPACITY, "apgd: support of %d atoms exceeds the cluster solver", S);
    sh.cache = bytes_rows(sh.CS, true) <= kLimitRows ? 1 : 0;
    sh.smem = bytes_rows(sh.CS, sh.cache != 0);
  }
  sh.rows_per = sh.full ? rows_full(sh.CS) : ceil_div(S, sh.CS);
  sh.n_pad = n_pad;
  *out = sh;
  return PC_OK;
}

ApgdArgs make_args(const ApgdJob& j, const ApgdShape& sh) {
  ApgdArgs a;
  a.G = j.G;
  a.ldg = j.ldg;
  a.b = j.b;
  a.n = j.n;
  a.lam = (float)j.lambda;
  a.eps = (float)j.eps;
  a.max_iter = j.max_iter;
  a.x = j.x;
  a.out_iters = j.iters;
  a.out_L = j.L;
  a.out_F = j.F;
  a.out_lanczos = j.lanczos;
  a.err = j.err;
  a.positive = j.positive ? 1 : 0;
  a.rows_per = sh.rows_per;
  a.n_pad = sh.n_pad;
  a.cache = sh.cache;
  a.vec_ok = ((j.ldg & 3) == 0 && (reinterpret_cast<uintptr_t>(j.G) & 15) == 0) ? 1 : 0;
  return a;
}

}  // namespace

int run_apgd_jobs(const ApgdJob* jobs, int n_jobs, cudaStream_t st) {
  int cs_max = 0;
  PC_TRY(apgd_setup(&cs_max));
  std::vector<ApgdShape> shapes(n_jobs);
  for (int i = 0; i < n_jobs; ++i)
    if (jobs[i].n > 0) PC_TRY(apgd_shape(jobs[i].n, cs_max, &shapes[i]));
  std::vector<char> done(n_jobs, 0);
  for (int i = 0; i < n_jobs; ++i)
    if (jobs[i].n <= 0) done[i] = 1;
  // one launch per (kernel, cluster size) group, at most APGD_BATCH_MAX jobs each
  for (int i = 0; i < n_jobs; ++i) {
    if (done[i]) continue;
    ApgdBatch batch{};
    size_t smem = 0;
    const bool full = shapes[i].full;
    const bool warp = shapes[i].warp, cta = shapes[i].cta;
    const int CS = shapes[i].CS;
    for (int j = i; j < n_jobs && batch.n_jobs < APGD_BATCH_MAX; ++j) {
      if (done[j] || shapes[j].full != full || shapes[j].CS != CS || shapes[j].warp != warp ||
          shapes[j].cta != cta)
        continue;
      batch.job[batch.n_jobs++] = make_args(jobs[j], shapes[j]);
      smem = std::max(smem, shapes[j].smem);
      done[j] = 1;
    }
    if (warp) {
      ProfScope prof_scope_(PROF_APGD, st);
      prof_scope_.kernels = 1;
      k_apgd_warp<<<batch.n_jobs, 32, 0, st>>>(batch);
      PC_LAUNCH_CHECK();
      continue;
    }
    if (cta) {
      ProfScope prof_scope_(PROF_APGD, st);
      prof_scope_.kernels = 1;
      k_apgd_cta<<<batch.n_jobs, APGD_THREADS, smem, st>>>(batch);
      PC_LAUNCH_CHECK();
      continue;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CS * batch.n_jobs, 1, 1);
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
      e = full ? cudaLaunchKernelEx(&cfg, k_apgd_full, batch) : cudaLaunchKernelEx(&cfg, k_apgd, batch);
    }
    PC_CUDA(e);
  }
  return PC_OK;
}

int run_apgd(const float* G, int ldg, const float* b, int S, double lambda, double eps,
             int max_iter, float* x, int* iters, double* L, double* Fx, cudaStream_t st,
             int* lanczos, int* err, bool positive) {
  if (S <= 0) return PC_OK;
  ApgdJob j{G, ldg, b, S, lambda, eps, max_iter, x, iters, L, Fx, lanczos, err, positive};
  return run_apgd_jobs(&j, 1, st);
}

}  // namespace pc
