// The reweighting step of Algorithm 2 (Sect. 5.1) in operator form: the
// restricted LASSO
//
//   min_x 1/2 ||V - Phi_S x||^2 + lambda ||x||_1     (x on the active set S)
//
// by the same monotone FISTA as the Gram-form kernels (apgd.cu: Lanczos step
// size, warm start, accept test, stop rule), but with the gradient
//
//   g(v) = Re Phi_S^H (Phi_S v - V)
//
// evaluated through the measurement operator on every iteration, as the
// paper's reweighting does: Phi_S v by degridding the image that holds v on
// S (the type-2 NUFFT, degrid.cu) and Phi_S^H by the certificate's gridding,
// FFT and epilogue (the type-1 NUFFT) read at S. One operator pair per FISTA
// iteration and per Lanczos step, no |S| x |S| matrix: for active sets of
// many thousands of atoms over millions of visibilities this is far cheaper
// than the contraction that forms G_S (12 M |S|^2 / 2 flops). The solver
// chooses between the two forms per Frank-Wolfe iteration by their cost.
//
// Since g is affine, the accept test and the momentum step need only
// g(z), g(x) and g(y) = c1 g(z) + (1 - c1 + c2) g(x_new) - c2 g(x_old):
//   F(z) - F(x) = sum_i (z_i - x_i) (g(z)_i + g(x)_i) / 2 + lambda (|z_i| - |x_i|).
// The FISTA and Lanczos bookkeeping runs in one-CTA kernels whose decisions
// the host reads after each step (one small copy per operator pair).
#include "lanczos.cuh"
#include "solver.cuh"

namespace pc {
namespace {

constexpr int OP_THREADS = 1024;
// Lanczos tolerance of the operator form: each step is an operator pair, so
// the estimate stops early (the top Ritz value moved by at most 5 % over 4
// steps, from step 5): it rises towards the Hessian's top eigenvalue, and
// where 1.01 x that value falls short of the curvature a FISTA step meets,
// the backtracking of k_op_update raises L (one extra pair per rejection).
constexpr float LZ_TOL_OP = 5e-2f;
constexpr int LZ_MIN_OP = 5;       // first step at which the test compares with four steps back

struct OpState {
  float L;          // step size 1.01 x top Ritz value (valid once lz_done)
  float t;          // FISTA momentum
  float theta_prev; // unused (kept for layout)
  int lz_m;         // Lanczos steps taken
  int lz_done;
  int it;           // FISTA iterations taken
  int done;
  int backtracks;   // FISTA steps rejected because L was below the curvature along them
  float al[LZ_MAX], be[LZ_MAX];
  float th[LZ_MAX];  // top Ritz value after each step
};

// sum over the block of K values per thread (every thread gets the sums)
template <int K>
__device__ void block_sums(float (&v)[K], float* red /* 32 * K */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < K; ++q)
    for (int off = 16; off; off >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], off);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < K; ++q) red[warp * K + q] = v[q];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < K; ++q) {
      float s = lane < nw ? red[lane * K + q] : 0.f;
      for (int off = 16; off; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
      if (lane == 0) red[32 * K + q] = s;
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < K; ++q) v[q] = red[32 * K + q];
}

__global__ void k_op_scatter(const int32_t* __restrict__ idx, const float* __restrict__ v, int n,
                             float* __restrict__ img) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) img[idx[i]] = v[i];
}

__global__ void k_op_sub(float2* __restrict__ y, const float2* __restrict__ V, int64_t M) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < M; k += (int64_t)gridDim.x * blockDim.x) {
    const float2 a = y[k], b = V[k];
    y[k] = make_float2(a.x - b.x, a.y - b.y);
  }
}

// g[i] = cimg[idx[i]]; the scatter image is cleared again at S
__global__ void k_op_gather(const float* __restrict__ cimg, const int32_t* __restrict__ idx, int n,
                            float* __restrict__ g, float* __restrict__ img) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const int p = idx[i];
    g[i] = cimg[p];
    img[p] = 0.f;
  }
}

__global__ void k_lz_init(float* __restrict__ v, float* __restrict__ vprev, int n, OpState* __restrict__ s) {
  const float v0 = rsqrtf((float)n);   // all ones / sqrt(n)
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    v[i] = v0;
    vprev[i] = 0.f;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    s->L = 1.f;
    s->t = 1.f;
    s->theta_prev = 0.f;
    s->lz_m = 0;
    s->lz_done = 0;
    s->it = 0;
    s->backtracks = 0;
    s->done = 0;
  }
}

// Lanczos start vector b_S / ||b_S||, b_S = Re Phi_S^H V read from the
// dirty image at S: b = G_S x_true + noise is one power step from the sky, so
// it leans towards the top eigenvectors and Lanczos settles in fewer steps
// (each an operator pair here) than from all ones; all ones if b_S = 0.
__global__ void __launch_bounds__(OP_THREADS) k_lz_init_dirty(const float* __restrict__ dirty,
                                                              const int32_t* __restrict__ idx, int n,
                                                              float* __restrict__ v, float* __restrict__ vprev,
                                                              OpState* __restrict__ s) {
  __shared__ float red[32 + 1];
  float a[1] = {0.f};
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float b = dirty[idx[i]];
    v[i] = b;
    vprev[i] = 0.f;
    a[0] = fmaf(b, b, a[0]);
  }
  block_sums<1>(a, red);
  const bool use = a[0] > 0.f && isfinite(a[0]);
  const float scale = use ? rsqrtf(a[0]) : 0.f, v0 = rsqrtf((float)n);
  for (int i = threadIdx.x; i < n; i += blockDim.x) v[i] = use ? v[i] * scale : v0;
  if (threadIdx.x == 0) {
    s->L = 1.f;
    s->t = 1.f;
    s->theta_prev = 0.f;
    s->lz_m = 0;
    s->lz_done = 0;
    s->it = 0;
    s->backtracks = 0;
    s->done = 0;
  }
}

// One Lanczos step on w = G v_j: alpha = v.w, w -= alpha v_j + beta_{j-1} v_{j-1},
// beta = ||w||, v_{j+1} = w / beta. The stop test has the Gram kernels' form
// (the top Ritz value changed by at most LZ_TOL_OP over the last 4 steps),
// from step LZ_MIN_OP on, evaluated after every step rather than every
// fourth: each step costs an operator pair here, the Ritz value a few
// microseconds.
__global__ void __launch_bounds__(OP_THREADS) k_lz_step(float* __restrict__ w, float* __restrict__ v,
                                                        float* __restrict__ vprev, int n, OpState* __restrict__ s) {
  __shared__ float red[32 * 2 + 2];
  __shared__ float s_theta;
  if (s->lz_done) return;
  const int j = s->lz_m;
  const float beta_prev = j > 0 ? s->be[j - 1] : 0.f;
  float a[1] = {0.f};
  for (int i = threadIdx.x; i < n; i += blockDim.x) a[0] = fmaf(v[i], w[i], a[0]);
  block_sums<1>(a, red);
  const float alpha = a[0];
  float b[1] = {0.f};
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float wi = w[i] - alpha * v[i] - beta_prev * vprev[i];
    w[i] = wi;
    b[0] = fmaf(wi, wi, b[0]);
  }
  block_sums<1>(b, red);
  const float beta = sqrtf(fmaxf(b[0], 0.f));
  if (threadIdx.x == 0) {
    s->al[j] = alpha;
    s->be[j] = beta;
  }
  __syncthreads();
  const int m = j + 1;
  const bool last = (m == n) || (m == LZ_MAX) || !(beta > 1e-7f * fabsf(alpha));
  const float theta = tridiag_top(s->al, s->be, m, &s_theta);
  const bool stop = last || (m >= LZ_MIN_OP && fabsf(theta - s->th[m - 5]) <= LZ_TOL_OP * fabsf(theta));
  __syncthreads();
  if (threadIdx.x == 0) {
    s->th[j] = theta;
    if (stop) s->L = 1.01f * (theta > 0.f ? theta : 1.f);
  }
  if (!stop) {
    const float inv = 1.f / beta;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      vprev[i] = v[i];
      v[i] = w[i] * inv;
    }
  }
  if (threadIdx.x == 0) {
    s->lz_m = m;
    s->lz_done = stop ? 1 : 0;
  }
}

__global__ void k_op_start(const float* __restrict__ x, const float* __restrict__ gx, float* __restrict__ y,
                           float* __restrict__ gy, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    y[i] = x[i];
    gy[i] = gx[i];
  }
}

// z = prox(y - g(y) / L, lambda / L)
__global__ void k_op_prox(const float* __restrict__ y, const float* __restrict__ gy, float* __restrict__ z, int n,
                          float lam, int positive, const OpState* __restrict__ s) {
  if (s->done) return;
  const float invL = 1.f / s->L;
  const float thr = lam * invL;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float u = y[i] - gy[i] * invL;
    z[i] = positive ? fmaxf(u - thr, 0.f) : copysignf(fmaxf(fabsf(u) - thr, 0.f), u);
  }
}

// Monotone accept test, momentum step and stop rule (as k_apgd_full).
__global__ void __launch_bounds__(OP_THREADS) k_op_update(float* __restrict__ x, float* __restrict__ gx,
                                                          float* __restrict__ y, float* __restrict__ gy,
                                                          const float* __restrict__ z, const float* __restrict__ gz,
                                                          int n, float lam, float eps, int max_iter,
                                                          OpState* __restrict__ s) {
  __shared__ float red[32 * 4 + 4];
  if (s->done) return;
  float v[4] = {0.f, 0.f, 0.f, 0.f};
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float zr = z[i], xr = x[i];
    v[0] += fmaf(zr - xr, 0.5f * (gz[i] + gx[i]), lam * (fabsf(zr) - fabsf(xr)));
    const float d = zr - y[i];
    v[1] = fmaf(d, d, v[1]);
    v[2] = fmaf(zr, zr, v[2]);
    v[3] = fmaf(d, gz[i] - gy[i], v[3]);            // d^T H d (g is affine: g(z) - g(y) = H d)
  }
  block_sums<4>(v, red);
  // Backtracking on L (Beck and Teboulle's FISTA with backtracking, in its
  // exact form for a quadratic): the step from y is valid when the curvature
  // d^T H d / |d|^2 along it stays at or below L. Above, L is raised past that
  // curvature (a lower bound of the Hessian's top eigenvalue) and the step is
  // taken again from the same y; x, y, their gradients and the momentum are
  // left as they are. The Lanczos estimate only has to be close.
  const float L = s->L;
  const bool too_long = v[1] > 0.f && v[3] > L * v[1];
  if (!too_long) {
    const float t = s->t;
    const float t1 = 0.5f * (1.f + sqrtf(1.f + 4.f * t * t));
    const bool accept = v[0] <= 0.f;
    const float c1 = t / t1, c2 = (t - 1.f) / t1;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const float xo = x[i], gxo = gx[i];
      const float xn = accept ? z[i] : xo;
      const float gxn = accept ? gz[i] : gxo;
      y[i] = xn + c1 * (z[i] - xn) + c2 * (xn - xo);
      gy[i] = gxn + c1 * (gz[i] - gxn) + c2 * (gxn - gxo);
      x[i] = xn;
      gx[i] = gxn;
    }
    __syncthreads();
    if (threadIdx.x == 0) s->t = t1;
  }
  if (threadIdx.x == 0) {
    s->it += 1;
    if (too_long) {
      s->L = 1.05f * (v[3] / v[1]);
      s->backtracks += 1;
      if (s->it >= max_iter) s->done = 1;
    } else if (sqrtf(v[1]) <= eps * sqrtf(v[2]) || s->it >= max_iter) {
      s->done = 1;
    }
  }
}

__global__ void k_op_finish(const OpState* __restrict__ s, int* __restrict__ iters, double* __restrict__ L,
                            int* __restrict__ lz) {
  if (iters) *iters = s->it;
  if (L) *L = (double)s->L;
  if (lz) *lz = s->lz_m;
}

struct OpWork {
  float* img;     // N^2, zero except while a vector is scattered into it
  float* cimg;    // N^2, adjoint output
  float2* yv;     // M
  float *v, *vprev, *w, *y, *gy, *z, *gz, *gx;   // n each
  OpState* s;
  int* rows;          // N: image rows holding atoms (ascending), then their count
  int* row_count;
  uint32_t* row_bits; // ceil(N / 32) words
};

// The image rows that hold atoms of S: bit mask and ascending list (one CTA).
__global__ void __launch_bounds__(OP_THREADS) k_op_rows(const int32_t* __restrict__ idx, int n, int N,
                                                        uint32_t* __restrict__ bits, int* __restrict__ rows,
                                                        int* __restrict__ count) {
  __shared__ int warp_tot[32];
  const int words = (N + 31) >> 5;
  for (int k = threadIdx.x; k < words; k += blockDim.x) bits[k] = 0u;
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int r = idx[i] / N;
    atomicOr(bits + (r >> 5), 1u << (r & 31));
  }
  __syncthreads();
  // ascending compaction, one bit per row: each thread owns a run of rows
  const int per = (N + blockDim.x - 1) / blockDim.x;
  const int r0 = threadIdx.x * per, r1 = min(N, r0 + per);
  int mine = 0;
  for (int r = r0; r < r1; ++r) mine += (bits[r >> 5] >> (r & 31)) & 1u;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int incl = mine;
  for (int off = 1; off < 32; off <<= 1) {
    const int o = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += o;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  int base = 0;
  for (int w = 0; w < warp; ++w) base += warp_tot[w];
  int pos = base + incl - mine;
  for (int r = r0; r < r1; ++r)
    if ((bits[r >> 5] >> (r & 31)) & 1u) rows[pos++] = r;
  if (threadIdx.x == blockDim.x - 1) *count = pos;
}

int op_workspace(pc_plan_s* p, int n, OpWork* w, cudaStream_t st) {
  const size_t NN = (size_t)p->N * p->N;
  const size_t nn = (size_t)((n + 63) / 64) * 64;
  const size_t rows_words = (size_t)(p->N + 31) / 32;
  const size_t bytes = sizeof(float) * 2 * NN + sizeof(float2) * (size_t)std::max<int64_t>(p->M, 1) +
                       sizeof(float) * 8 * nn + sizeof(OpState) + sizeof(int) * ((size_t)p->N + 4) +
                       sizeof(uint32_t) * rows_words + 512;
  const bool fresh = p->opw.bytes < bytes;
  PC_TRY(p->opw.ensure(bytes));
  char* b = static_cast<char*>(p->opw.p);
  w->img = reinterpret_cast<float*>(b);
  w->cimg = w->img + NN;
  w->yv = reinterpret_cast<float2*>(w->cimg + NN);
  float* f = reinterpret_cast<float*>(w->yv + std::max<int64_t>(p->M, 1));
  float** vecs[8] = {&w->v, &w->vprev, &w->w, &w->y, &w->gy, &w->z, &w->gz, &w->gx};
  for (int k = 0; k < 8; ++k) *vecs[k] = f + k * nn;
  w->s = reinterpret_cast<OpState*>(f + 8 * nn);
  w->rows = reinterpret_cast<int*>(reinterpret_cast<char*>(w->s) + ((sizeof(OpState) + 15) / 16) * 16);
  w->row_count = w->rows + p->N;
  w->row_bits = reinterpret_cast<uint32_t*>(w->row_count + 4);
  if (fresh) PC_CUDA(cudaMemsetAsync(w->img, 0, sizeof(float) * NN, st));   // kept zero between uses
  return PC_OK;
}

// out = g(v) = Re Phi_S^H (Phi_S v - V) at S (Re Phi_S^H Phi_S v without V)
// (the degridding and gridding record their own kernel classes; the
// vector work around them is the "apgd_op" class)
int op_apply(pc_plan_s* p, const OpWork& w, const float2* V, const int32_t* idx, int n, const float* v,
             float* out, cudaStream_t st) {
  {
    ProfScope ps(PROF_APGD_OP, st);
    ps.kernels = 1;
    k_op_scatter<<<ceil_div(n, 256), 256, 0, st>>>(idx, v, n, w.img);
    PC_LAUNCH_CHECK();
  }
  PC_TRY(forward_grid_impl(p, w.img, w.yv, st));
  if (V) {
    ProfScope ps(PROF_APGD_OP, st);
    ps.kernels = 1;
    k_op_sub<<<(int)std::min<int64_t>(4096, ceil_div(p->M, 256)), 256, 0, st>>>(w.yv, V, p->M);
    PC_LAUNCH_CHECK();
  }
  PC_TRY(adjoint_grid_impl(p, w.yv, w.cimg, 1.0f, nullptr, st));
  ProfScope ps(PROF_APGD_OP, st);
  ps.kernels = 1;
  k_op_gather<<<ceil_div(n, 256), 256, 0, st>>>(w.cimg, idx, n, out, w.img);
  PC_LAUNCH_CHECK();
  return PC_OK;
}

int read_flag(const int* dev_flag, cudaStream_t st, int* host) {
  PC_CUDA(cudaMemcpyAsync(host, dev_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  PC_CUDA(cudaStreamSynchronize(st));
  return PC_OK;
}

}  // namespace

int op_pair_seconds(pc_plan_s* p, cudaStream_t st, double* out) {
  if (p->op_pair_s > 0.0) {
    *out = p->op_pair_s;
    return PC_OK;
  }
  OpWork w;
  PC_TRY(op_workspace(p, 1, &w, st));
  // a unit image on one pixel through both operators, timed by events
  int32_t* idx1 = reinterpret_cast<int32_t*>(w.v);
  const int32_t centre = (p->N / 2) * p->N + p->N / 2;
  PC_CUDA(cudaMemcpyAsync(idx1, &centre, sizeof(int32_t), cudaMemcpyHostToDevice, st));
  PC_CUDA(cudaMemsetAsync(w.w, 0, sizeof(float), st));        // the input vector: one zero weight
  cudaEvent_t a = nullptr, b = nullptr;
  PC_CUDA(cudaEventCreate(&a));
  PC_CUDA(cudaEventCreate(&b));
  int rc = op_apply(p, w, nullptr, idx1, 1, w.w, w.gz, st);   // warm (also loads the kernels)
  if (rc == PC_OK) {
    cudaEventRecord(a, st);
    rc = op_apply(p, w, nullptr, idx1, 1, w.w, w.gz, st);
    cudaEventRecord(b, st);
  }
  float ms = 0.f;
  if (rc == PC_OK && cudaEventSynchronize(b) == cudaSuccess) cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  PC_TRY(rc);
  p->op_pair_s = std::max(1e-6, (double)ms * 1e-3);
  *out = p->op_pair_s;
  return PC_OK;
}

int run_operator_apgd(pc_plan_s* p, const float2* V, const float* dirty, const int32_t* idx, int n,
                      double lambda, double eps, int max_iter, bool positive, float* x, int* iters_dev,
                      double* L_dev, int* lz_dev, cudaStream_t st) {
  if (n <= 0) return PC_OK;
  OpWork w;
  PC_TRY(op_workspace(p, n, &w, st));
  const int gb = std::min(ceil_div(n, 256), 1024);
  int flag = 0;
  // the image rows that hold the atoms: the one-CTA FFT passes of the
  // operator pairs transform only those on the image side
  struct Restrict {
    pc_plan_s* p;
    ~Restrict() {
      p->n_img_rows = 0;
      p->img_rows = nullptr;
      p->img_row_bits = nullptr;
    }
  } restrict_guard{p};
  if (fft_big_size(p->G)) {
    {
      ProfScope ps(PROF_APGD_OP, st);
      ps.kernels = 1;
      k_op_rows<<<1, OP_THREADS, 0, st>>>(idx, n, p->N, w.row_bits, w.rows, w.row_count);
      PC_LAUNCH_CHECK();
    }
    int n_rows = 0;
    PC_TRY(read_flag(w.row_count, st, &n_rows));
    if (n_rows > 0 && n_rows < p->N) {
      p->img_rows = w.rows;
      p->img_row_bits = w.row_bits;
      p->n_img_rows = n_rows;
    }
  }
  auto book = [&](auto launch) {                 // a bookkeeping launch, timed as "apgd_op"
    ProfScope ps(PROF_APGD_OP, st);
    ps.kernels = 1;
    launch();
    return cudaPeekAtLastError() == cudaSuccess ? PC_OK
                                                : fail(PC_ERR_CUDA, "reweighting: %s",
                                                       cudaGetErrorString(cudaGetLastError()));
  };
  if (dirty)
    PC_TRY(book([&] { k_lz_init_dirty<<<1, OP_THREADS, 0, st>>>(dirty, idx, n, w.v, w.vprev, w.s); }));
  else
    PC_TRY(book([&] { k_lz_init<<<gb, 256, 0, st>>>(w.v, w.vprev, n, w.s); }));
  for (int j = 0; j < LZ_MAX; ++j) {
    PC_TRY(op_apply(p, w, nullptr, idx, n, w.v, w.w, st));
    PC_TRY(book([&] { k_lz_step<<<1, OP_THREADS, 0, st>>>(w.w, w.v, w.vprev, n, w.s); }));
    PC_TRY(read_flag(&w.s->lz_done, st, &flag));
    if (flag) break;
  }
  const float lam = (float)lambda;
  PC_TRY(op_apply(p, w, V, idx, n, x, w.gx, st));                // g(x) at the warm start
  PC_TRY(book([&] { k_op_start<<<gb, 256, 0, st>>>(x, w.gx, w.y, w.gy, n); }));
  for (int it = 0; it < max_iter; ++it) {
    PC_TRY(book([&] { k_op_prox<<<gb, 256, 0, st>>>(w.y, w.gy, w.z, n, lam, positive ? 1 : 0, w.s); }));
    PC_TRY(op_apply(p, w, V, idx, n, w.z, w.gz, st));
    PC_TRY(book([&] {
      k_op_update<<<1, OP_THREADS, 0, st>>>(x, w.gx, w.y, w.gy, w.z, w.gz, n, lam, (float)eps, max_iter, w.s);
    }));
    PC_TRY(read_flag(&w.s->done, st, &flag));
    if (flag) break;
  }
  return book([&] { k_op_finish<<<1, 1, 0, st>>>(w.s, iters_dev, L_dev, lz_dev); });
}

}  // namespace pc
