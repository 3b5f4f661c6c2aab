// C ABI entry points: operators, hot-path steps and the Polyatomic
// Frank-Wolfe driver (Algorithm 2). The driver runs on the host and keeps all
// state on the device; it reads back a handful of scalars per Frank-Wolfe
// iteration (objective, ||mu||_inf, |S u I|, |supp|) to size the next launches
// and to take the stopping decision.
#include <algorithm>
#include <cmath>
#include <map>

#include "pc_internal.cuh"
#include "solver.cuh"

namespace pc {
namespace {

// Gdst[i][j] = Gsrc[map[i]][map[j]] where both map entries are >= 0.
__global__ void k_gather_sym(const float* __restrict__ Gsrc, int lds, const int32_t* __restrict__ map,
                             int n, float* __restrict__ Gdst, int ldd, const int32_t* __restrict__ n_dev) {
  if (n_dev) n = min(n, *n_dev);   // count held on the device (n: its upper bound)
  const int i = blockIdx.y;
  if (i >= n) return;
  const int mi = map[i];
  if (mi < 0) return;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    const int mj = map[j];
    if (mj >= 0) Gdst[(size_t)i * ldd + j] = Gsrc[(size_t)mi * lds + mj];
  }
}

// dst[i] = map[i] >= 0 ? src[map[i]] : fill
template <class T>
__global__ void k_gather_vec(const T* __restrict__ src, const int32_t* __restrict__ map, int n,
                             T* __restrict__ dst, T fill, const int32_t* __restrict__ n_dev) {
  if (n_dev) n = min(n, *n_dev);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int m = map[i];
  dst[i] = m >= 0 ? src[m] : fill;
}

// sum |x| in float64 (one block)
__global__ void k_l1(const float* __restrict__ x, int n, double* __restrict__ out,
                     const int32_t* __restrict__ n_dev) {
  __shared__ double ws[32];
  if (n_dev) n = min(n, *n_dev);
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

int gather_sym(const float* Gsrc, int lds, const int32_t* map, int n, float* Gdst, int ldd,
               cudaStream_t st, const int32_t* n_dev = nullptr) {
  ProfScope prof_scope_(PROF_MISC, st);
  if (n <= 0) return PC_OK;
  dim3 grid(std::max(1, std::min(ceil_div(n, 256), 32)), n);
  prof_scope_.kernels = 1;
  k_gather_sym<<<grid, 256, 0, st>>>(Gsrc, lds, map, n, Gdst, ldd, n_dev);
  PC_LAUNCH_CHECK();
  return PC_OK;
}

template <class T>
int gather_vec(const T* src, const int32_t* map, int n, T* dst, T fill, cudaStream_t st,
               const int32_t* n_dev = nullptr) {
  ProfScope prof_scope_(PROF_MISC, st);
  if (n <= 0) return PC_OK;
  prof_scope_.kernels = 1;
  k_gather_vec<T><<<ceil_div(n, 256), 256, 0, st>>>(src, map, n, dst, fill, n_dev);
  PC_LAUNCH_CHECK();
  return PC_OK;
}


// Pruning (step 3 of Algorithm 2) in one launch: row i of the new support is
// entry keep[i] of the active set; copies its Gram row (columns keep[.]) and,
// in block (0, i), its index, weight, b, atom, support mark and |x| into the
// objective's l1 sum. The count n is read on the device (bound: its maximum).
__global__ void k_prune(const int32_t* __restrict__ keep, const int32_t* __restrict__ n_dev, int bound,
                        const int32_t* __restrict__ idxB, const float* __restrict__ xB,
                        const float* __restrict__ bB, const float* __restrict__ GB, int ld,
                        int32_t* __restrict__ idxA, float* __restrict__ xA, float* __restrict__ bA,
                        float* __restrict__ GA, float4* __restrict__ atomsA, uint8_t* __restrict__ mark,
                        double* __restrict__ l1, const float4* __restrict__ atom_tab) {
  const int n = min(bound, *n_dev);
  for (int i = blockIdx.y; i < n; i += gridDim.y) {
    const int ki = keep[i];
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
      GA[(size_t)i * ld + j] = GB[(size_t)ki * ld + keep[j]];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      const int p = idxB[ki];
      const float x = xB[ki];
      idxA[i] = p;
      xA[i] = x;
      bA[i] = bB[ki];
      float4 at = atom_tab[p];
      at.w *= x;
      atomsA[i] = at;
      mark[p] = 1;
      atomicAdd(l1, fabs((double)x));
    }
  }
}

// Resume: the given support becomes the pruned support of the previous
// iteration (what k_prune leaves): indices, weights, weighted atoms, support
// marks, ||x||_1 and the support count.
__global__ void k_resume_support(const int32_t* __restrict__ idx, const float* __restrict__ x, int S,
                                 int32_t* __restrict__ idxA, float* __restrict__ xA,
                                 float4* __restrict__ atomsA, uint8_t* __restrict__ mark,
                                 double* __restrict__ l1, int32_t* __restrict__ n_sup,
                                 const float4* __restrict__ atom_tab) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < S; i += gridDim.x * blockDim.x) {
    const int p = idx[i];
    const float w = x[i];
    idxA[i] = p;
    xA[i] = w;
    float4 at = atom_tab[p];
    at.w *= w;
    atomsA[i] = at;
    mark[p] = 1;
    atomicAdd(l1, fabs((double)w));
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *n_sup = S;
}

// After the exploration, in one block: for each active atom its position in
// the old (pruned) support or -1 (binary search), the warm start and b of the
// old atoms, its atom (unit weight), the ascending list of the new positions
// and their count; finally the support marks are cleared.
__global__ void __launch_bounds__(1024)
k_post_select(const int32_t* __restrict__ idxB, int n_act, const int32_t* __restrict__ idxA, int nS,
              const float* __restrict__ xA, const float* __restrict__ bA, int32_t* __restrict__ oldpos,
              int32_t* __restrict__ newrows, int32_t* __restrict__ n_new_dev, float* __restrict__ xB,
              float* __restrict__ bB, float4* __restrict__ atomsB, uint8_t* __restrict__ mark,
              const float4* __restrict__ atom_tab) {
  __shared__ int wcount[32];
  __shared__ int run_s;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) run_s = 0;
  __syncthreads();
  for (int base = 0; base < n_act; base += blockDim.x) {
    const int i = base + threadIdx.x;
    bool is_new = false;
    if (i < n_act) {
      const int v = idxB[i];
      int lo = 0, hi = nS;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (idxA[mid] < v) lo = mid + 1; else hi = mid;
      }
      const int op = (lo < nS && idxA[lo] == v) ? lo : -1;
      oldpos[i] = op;
      xB[i] = op >= 0 ? xA[op] : 0.f;
      bB[i] = op >= 0 ? bA[op] : 0.f;
      atomsB[i] = atom_tab[v];
      is_new = op < 0;
    }
    const unsigned bal = __ballot_sync(0xffffffffu, is_new);
    if (lane == 0) wcount[warp] = __popc(bal);
    __syncthreads();
    int before = 0, total = 0;
    for (int w = 0; w < nw; ++w) {
      if (w < warp) before += wcount[w];
      total += wcount[w];
    }
    if (is_new) newrows[run_s + before + __popc(bal & ((1u << lane) - 1u))] = i;
    __syncthreads();
    if (threadIdx.x == 0) run_s += total;
    __syncthreads();
  }
  if (threadIdx.x == 0) *n_new_dev = run_s;
  for (int j = threadIdx.x; j < nS; j += blockDim.x) mark[idxA[j]] = 0;
}

// Exploration threshold of rule R1 (Algorithm 2) from the certificate maxima
// on the device: thr = top - 2 Delta / ((k + 2) lambda) with top = max |mu|
// (max mu under positivity); at k = 0 without a given lambda_max, Delta =
// (1 - delta) lambda max(top, 0) is stored in *Delta for later iterations.
__global__ void k_r1_threshold(const unsigned* __restrict__ maxbits, int positive, double lambda,
                               double delta, int k, double* __restrict__ Delta, float* __restrict__ thr) {
  const unsigned key = maxbits[1];
  float top;
  if (positive) {
    const unsigned u = key == 0 ? 0xff800000u : ((key & 0x80000000u) ? (key & 0x7fffffffu) : ~key);
    top = __uint_as_float(u);
  } else {
    top = __uint_as_float(maxbits[0]);
  }
  if (*Delta < 0.0) *Delta = (1.0 - delta) * lambda * fmax((double)top, 0.0);
  float t = (float)((double)top - 2.0 * (*Delta) / ((k + 2) * lambda));
  if (positive) t = fmaxf(t, 1.4e-45f);   // mu >= smallest positive float: mu > 0
  *thr = t;
}

__global__ void k_iota(int32_t* __restrict__ a, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = i;
}

// Gram rows of the n_new new atoms against all n_act active atoms, written
// into G (leading dimension ldg, both triangles) and b = Re(Phi^H V).
// atomsB: the active atoms in position order; newrows: ascending positions of
// the new atoms; oldpos: per position the old index or -1 (null: all new).
// Up to 15 new atoms take the thin kernel, mode 1 the FP32 tile kernel (both
// then write b for every atom); otherwise the tensor cores (mode 0 when the
// block has >= 4096 entries, mode 2, or the self-test mode 3) take the atoms
// in the order new-first and write the G rows and b of the new atoms (b of
// the old atoms is the caller's). err_dev receives the tensor-core timeout flag.
int gram_update(pc_plan_s* p, const float2* V, const float4* atomsB, int n_act,
                const int32_t* newrows, int n_new, const int32_t* oldpos, float* G, int ldg,
                float* b, int mode, int* err_dev, cudaStream_t st) {
  if (n_new <= 0) return PC_OK;
  const bool thin = n_new + 1 <= 16 && mode < 2;
  const bool tc = !thin && (mode >= 2 || (mode == 0 && (int64_t)n_new * n_act >= 64 * 64));
  if (!tc) {
    const int ldacc = n_act;
    PC_TRY(p->acc.ensure(sizeof(double) * ((size_t)n_new * ldacc + n_act)));
    double* acc = p->acc.as<double>();
    double* b64 = acc + (size_t)n_new * ldacc;
    PC_TRY(p->atomsA.ensure(sizeof(float4) * n_new));
    PC_TRY(gather_vec<float4>(atomsB, newrows, n_new, p->atomsA.as<float4>(),
                              make_float4(0.f, 0.f, 0.f, 0.f), st));
    PC_CUDA(cudaMemsetAsync(acc, 0, sizeof(double) * ((size_t)n_new * ldacc + n_act), st));
    if (thin) {
      PC_TRY(launch_gram_thin(p->vis_fx, V, p->M, p->atomsA.as<float4>(), n_new, atomsB, n_act, acc,
                              ldacc, b64, st));
    } else {
      PC_TRY(launch_gram(p->vis_fx, nullptr, p->M, p->atomsA.as<float4>(), n_new, atomsB, n_act,
                         false, acc, ldacc, st, false));
      if (V) PC_TRY(launch_gram_thin(p->vis_fx, V, p->M, nullptr, 0, atomsB, n_act, nullptr, 0, b64, st));
    }
    PC_TRY(launch_gram_finalize(acc, ldacc, newrows, n_new, n_act, oldpos, G, ldg, st));
    if (V && b) PC_TRY(launch_d2f(b64, n_act, b, st));
    return PC_OK;
  }
  // tensor cores: atoms in the order new-first
  PC_TRY(p->perm.ensure(sizeof(int32_t) * n_act));
  PC_TRY(p->atomsP.ensure(sizeof(float4) * n_act));
  int32_t* perm = p->perm.as<int32_t>();
  PC_CUDA(cudaMemcpyAsync(perm, newrows, sizeof(int32_t) * n_new, cudaMemcpyDeviceToDevice, st));
  if (oldpos && n_act > n_new)
    PC_TRY(launch_compact_old(oldpos, n_act, perm + n_new, p->iscal + 6, st));
  PC_TRY(gather_vec<float4>(atomsB, perm, n_act, p->atomsP.as<float4>(),
                            make_float4(0.f, 0.f, 0.f, 0.f), st));
  const int ldacc = n_act + 1;
  PC_TRY(p->acc.ensure(sizeof(double) * (size_t)n_new * ldacc));
  double* acc = p->acc.as<double>();
  PC_CUDA(cudaMemsetAsync(acc, 0, sizeof(double) * (size_t)n_new * ldacc, st));
  PC_TRY(launch_gram_tc(p->vis_fx, V, p->M, p->atomsP.as<float4>(), n_act, n_new, acc, ldacc, err_dev,
                        st, mode == 3, p->pbuf, reinterpret_cast<float*>(p->dscal + 6), p->uscal + 7));
  PC_TRY(launch_gram_finalize_perm(acc, ldacc, n_new, n_act, perm, G, ldg, V ? b : nullptr, st));
  return PC_OK;
}

}  // namespace

int adjoint_grid_impl(pc_plan_s* p, const float2* h, float* img, float scale, unsigned* maxbits,
                      cudaStream_t st) {
  PC_TRY(launch_grid(p, h, st));
  PC_TRY(launch_fft_rows(p, st));
  PC_TRY(launch_fft_cols_epilogue(p, img, scale, maxbits, st));
  return PC_OK;
}

int check_plan(pc_plan_s* p, const char* fn) {
  if (!p) return fail(PC_ERR_INVALID_ARG, "%s: NULL plan", fn);
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != p->device)
    return fail(PC_ERR_INVALID_ARG, "%s: plan was built on device %d, current is %d", fn,
                p->device, dev);
  return PC_OK;
}

int check_dev(const void* ptr, bool needed, const char* fn, const char* name) {
  if (!needed) return PC_OK;
  if (!is_device_ptr(ptr)) return fail(PC_ERR_INVALID_ARG, "%s: %s is not a device pointer", fn, name);
  return PC_OK;
}

int sync_read(void* host, const void* dev, size_t bytes, cudaStream_t st) {
  PC_CUDA(cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, st));
  PC_CUDA(cudaStreamSynchronize(st));
  return PC_OK;
}

// Synchronise the stream (after any reads the caller queued) and report an
// expired bounded wait of the tensor-core gridding (flag iscal[7], cleared here).
int grid_flag_sync(pc_plan_s* p, cudaStream_t st, const char* fn) {
  int32_t flag = 0;
  PC_CUDA(cudaMemcpyAsync(&flag, p->iscal + 7, sizeof(flag), cudaMemcpyDeviceToHost, st));
  PC_CUDA(cudaStreamSynchronize(st));
  if (flag) {
    PC_CUDA(cudaMemsetAsync(p->iscal + 7, 0, sizeof(int32_t), st));
    return fail(PC_ERR_TIMEOUT, "%s: a bounded tensor-core gridding wait expired", fn);
  }
  return PC_OK;
}

float bits_to_float(unsigned b) {
  float f;
  std::memcpy(&f, &b, sizeof(f));
  return f;
}

// Inverse of float_order_key (a zero key, "nothing seen", maps to -infinity).
float key_to_float(unsigned key) {
  if (key == 0) return -INFINITY;
  return bits_to_float((key & 0x80000000u) ? (key & 0x7fffffffu) : ~key);
}

namespace {

// Small per-device scratch for pc_apgd (no plan): 4 ints + 4 doubles.
int apgd_scratch(void** out) {
  static std::map<int, void*> bufs;
  int dev = 0;
  cudaGetDevice(&dev);
  auto it = bufs.find(dev);
  if (it != bufs.end()) {
    *out = it->second;
    return PC_OK;
  }
  void* p = nullptr;
  PC_CUDA(cudaMalloc(&p, 64));
  bufs[dev] = p;
  *out = p;
  return PC_OK;
}

}  // namespace
}  // namespace pc

using namespace pc;

extern "C" int pc_forward_sparse(pc_plan_t p, const int32_t* idx, const float* x, int32_t S,
                                 pc_c32* y, void* stream) {
  clear_error();
  PC_TRY(check_plan(p, "pc_forward_sparse"));
  if (S < 0) return fail(PC_ERR_INVALID_ARG, "pc_forward_sparse: S < 0");
  PC_TRY(check_dev(idx, S > 0, "pc_forward_sparse", "idx_dev"));
  PC_TRY(check_dev(x, S > 0, "pc_forward_sparse", "x_dev"));
  PC_TRY(check_dev(y, p->M > 0, "pc_forward_sparse", "y_dev"));
  cudaStream_t st = SS(stream);
  PC_TRY(p->atomsA.ensure(sizeof(float4) * std::max(S, 1)));
  PC_TRY(make_atoms_checked(idx, x, S, p->N, p->dl, p->atomsA.as<float4>(), p->iscal, st));
  PC_TRY(launch_residual(p->vis_fx, nullptr, p->M, p->atomsA.as<float4>(), S,
                         reinterpret_cast<float2*>(y), nullptr, st));
  return PC_OK;
}

extern "C" int pc_adjoint_sparse(pc_plan_t p, const pc_c32* y, const int32_t* idx, int32_t S,
                                 float* out, void* stream) {
  clear_error();
  PC_TRY(check_plan(p, "pc_adjoint_sparse"));
  if (S < 0) return fail(PC_ERR_INVALID_ARG, "pc_adjoint_sparse: S < 0");
  if (S == 0) return PC_OK;
  PC_TRY(check_dev(idx, true, "pc_adjoint_sparse", "idx_dev"));
  PC_TRY(check_dev(out, true, "pc_adjoint_sparse", "out_dev"));
  PC_TRY(check_dev(y, p->M > 0, "pc_adjoint_sparse", "y_dev"));
  cudaStream_t st = SS(stream);
  PC_TRY(p->atomsA.ensure(sizeof(float4) * S));
  PC_TRY(p->acc.ensure(sizeof(double) * (size_t)S));
  PC_TRY(make_atoms_checked(idx, nullptr, S, p->N, p->dl, p->atomsA.as<float4>(), p->iscal, st));
  PC_CUDA(cudaMemsetAsync(p->acc.p, 0, sizeof(double) * (size_t)S, st));
  PC_TRY(launch_gram_thin(p->vis_fx, reinterpret_cast<const float2*>(y), p->M, nullptr, 0,
                          p->atomsA.as<float4>(), S, nullptr, 0, p->acc.as<double>(), st));
  PC_TRY(launch_d2f(p->acc.as<double>(), S, out, st));
  return PC_OK;
}

extern "C" int pc_adjoint_grid(pc_plan_t p, const pc_c32* y, float* img, void* stream) {
  clear_error();
  PC_TRY(check_plan(p, "pc_adjoint_grid"));
  PC_TRY(check_dev(y, p->M > 0, "pc_adjoint_grid", "y_dev"));
  PC_TRY(check_dev(img, true, "pc_adjoint_grid", "img_dev"));
  return adjoint_grid_impl(p, reinterpret_cast<const float2*>(y), img, 1.0f, nullptr, SS(stream));
}

extern "C" int pc_lambda_max(pc_plan_t p, const pc_c32* V, double* out, void* stream) {
  clear_error();
  PC_TRY(check_plan(p, "pc_lambda_max"));
  PC_TRY(check_dev(V, p->M > 0, "pc_lambda_max", "V_dev"));
  if (!out) return fail(PC_ERR_INVALID_ARG, "pc_lambda_max: NULL output");
  cudaStream_t st = SS(stream);
  PC_CUDA(cudaMemsetAsync(p->uscal, 0, 2 * sizeof(unsigned), st));
  PC_TRY(adjoint_grid_impl(p, reinterpret_cast<const float2*>(V), p->mu, 1.0f, p->uscal, st));
  unsigned b = 0;
  PC_CUDA(cudaMemcpyAsync(&b, p->uscal, sizeof(b), cudaMemcpyDeviceToHost, st));
  PC_TRY(grid_flag_sync(p, st, "pc_lambda_max"));
  const float f = bits_to_float(b);
  if (!std::isfinite(f)) return fail(PC_ERR_NUMERIC, "pc_lambda_max: non-finite dirty image");
  *out = (double)f;
  return PC_OK;
}

extern "C" int pc_lambda_max_positive(pc_plan_t p, const pc_c32* V, double* out, void* stream) {
  clear_error();
  PC_TRY(check_plan(p, "pc_lambda_max_positive"));
  PC_TRY(check_dev(V, p->M > 0, "pc_lambda_max_positive", "V_dev"));
  if (!out) return fail(PC_ERR_INVALID_ARG, "pc_lambda_max_positive: NULL output");
  cudaStream_t st = SS(stream);
  PC_CUDA(cudaMemsetAsync(p->uscal, 0, 2 * sizeof(unsigned), st));
  PC_TRY(adjoint_grid_impl(p, reinterpret_cast<const float2*>(V), p->mu, 1.0f, p->uscal, st));
  unsigned b[2] = {0, 0};
  PC_CUDA(cudaMemcpyAsync(b, p->uscal, sizeof(b), cudaMemcpyDeviceToHost, st));
  PC_TRY(grid_flag_sync(p, st, "pc_lambda_max_positive"));
  const float f = key_to_float(b[1]);
  if (!std::isfinite(f) || !std::isfinite(bits_to_float(b[0])))
    return fail(PC_ERR_NUMERIC, "pc_lambda_max_positive: non-finite dirty image");
  *out = std::max(0.0, (double)f);
  return PC_OK;
}

extern "C" int pc_certificate(pc_plan_t p, const pc_c32* V, const int32_t* idx, const float* x,
                              int32_t S, double lambda, float* mu, double* mu_inf_host,
                              double* sumsq_host, void* stream) {
  clear_error();
  PC_TRY(check_plan(p, "pc_certificate"));
  if (S < 0) return fail(PC_ERR_INVALID_ARG, "pc_certificate: S < 0");
  if (!(lambda > 0.0) || !std::isfinite(lambda))
    return fail(PC_ERR_INVALID_ARG, "pc_certificate: lambda must be positive and finite");
  PC_TRY(check_dev(V, p->M > 0, "pc_certificate", "V_dev"));
  PC_TRY(check_dev(idx, S > 0, "pc_certificate", "idx_dev"));
  PC_TRY(check_dev(x, S > 0, "pc_certificate", "x_dev"));
  PC_TRY(check_dev(mu, true, "pc_certificate", "mu_dev"));
  cudaStream_t st = SS(stream);
  PC_TRY(p->atomsA.ensure(sizeof(float4) * std::max(S, 1)));
  PC_TRY(make_atoms_checked(idx, x, S, p->N, p->dl, p->atomsA.as<float4>(), p->iscal, st));
  PC_CUDA(cudaMemsetAsync(p->dscal, 0, sizeof(double), st));
  PC_CUDA(cudaMemsetAsync(p->uscal, 0, 2 * sizeof(unsigned), st));
  PC_TRY(launch_residual(p->vis_fx, reinterpret_cast<const float2*>(V), p->M,
                         p->atomsA.as<float4>(), S, p->resid, p->dscal, st));
  PC_TRY(adjoint_grid_impl(p, p->resid, mu, (float)(1.0 / lambda), p->uscal, st));
  if (mu_inf_host || sumsq_host) {
    unsigned b = 0;
    double ss = 0.0;
    PC_CUDA(cudaMemcpyAsync(&b, p->uscal, sizeof(b), cudaMemcpyDeviceToHost, st));
    PC_CUDA(cudaMemcpyAsync(&ss, p->dscal, sizeof(ss), cudaMemcpyDeviceToHost, st));
    PC_TRY(grid_flag_sync(p, st, "pc_certificate"));
    if (mu_inf_host) *mu_inf_host = (double)bits_to_float(b);
    if (sumsq_host) *sumsq_host = ss;
  }
  return PC_OK;
}

extern "C" int pc_select(pc_plan_t p, const float* mu, float thr, const int32_t* prev, int32_t n_prev,
                         int32_t* out, int32_t cap, int32_t* n_out_host, void* stream) {
  clear_error();
  PC_TRY(check_plan(p, "pc_select"));
  if (n_prev < 0 || cap < 0 || !n_out_host) return fail(PC_ERR_INVALID_ARG, "pc_select: bad sizes");
  PC_TRY(check_dev(mu, true, "pc_select", "mu_dev"));
  PC_TRY(check_dev(prev, n_prev > 0, "pc_select", "prev_idx_dev"));
  PC_TRY(check_dev(out, cap > 0, "pc_select", "out_idx_dev"));
  cudaStream_t st = SS(stream);
  const int64_t npix = (int64_t)p->N * p->N;
  if (n_prev > 0) {
    PC_TRY(p->atomsA.ensure(sizeof(float4) * n_prev));
    PC_TRY(make_atoms_checked(prev, nullptr, n_prev, p->N, p->dl, p->atomsA.as<float4>(), p->iscal, st));
  }
  PC_TRY(launch_mark(p->mark, prev, n_prev, 1, st));
  PC_TRY(launch_select(mu, npix, thr, p->mark, out, p->iscal, p->sel_blocks, cap, st));
  PC_TRY(launch_mark(p->mark, prev, n_prev, 0, st));
  int32_t n = 0;
  PC_TRY(sync_read(&n, p->iscal, sizeof(n), st));
  *n_out_host = n;
  if (n > cap) return fail(PC_ERR_CAPACITY, "pc_select: %d atoms exceed capacity %d", n, cap);
  return PC_OK;
}

extern "C" int pc_gram(pc_plan_t p, const pc_c32* V, const int32_t* idx, int32_t S, float* G,
                       int32_t ldg, float* b, int32_t mode, void* stream) {
  clear_error();
  PC_TRY(check_plan(p, "pc_gram"));
  if (S < 0 || ldg < S) return fail(PC_ERR_INVALID_ARG, "pc_gram: need S >= 0 and ldg >= S");
  if (mode < 0 || mode > 3) return fail(PC_ERR_INVALID_ARG, "pc_gram: mode must be 0, 1, 2 or 3");
  if (S == 0) return PC_OK;
  PC_TRY(check_dev(idx, true, "pc_gram", "idx_dev"));
  PC_TRY(check_dev(G, true, "pc_gram", "G_dev"));
  const bool with_v = V != nullptr;
  PC_TRY(check_dev(V, with_v && p->M > 0, "pc_gram", "V_dev"));
  PC_TRY(check_dev(b, with_v, "pc_gram", "b_dev"));
  cudaStream_t st = SS(stream);
  PC_TRY(p->atomsB.ensure(sizeof(float4) * S));
  PC_TRY(p->newrows.ensure(sizeof(int32_t) * S));
  PC_TRY(make_atoms_checked(idx, nullptr, S, p->N, p->dl, p->atomsB.as<float4>(), p->iscal, st));
  k_iota<<<ceil_div(S, 256), 256, 0, st>>>(p->newrows.as<int32_t>(), S);   // every atom is new
  PC_LAUNCH_CHECK();
  PC_CUDA(cudaMemsetAsync(p->iscal + 4, 0, sizeof(int32_t), st));
  PC_TRY(gram_update(p, reinterpret_cast<const float2*>(V), p->atomsB.as<float4>(), S,
                     p->newrows.as<int32_t>(), S, nullptr, G, ldg, b, mode, p->iscal + 4, st));
  int32_t err = 0;
  PC_TRY(sync_read(&err, p->iscal + 4, sizeof(err), st));
  if (err) return fail(PC_ERR_TIMEOUT, "pc_gram: a bounded tensor-core wait expired");
  return PC_OK;
}

extern "C" int pc_apgd(const float* G, int32_t ldg, const float* b, int32_t S, double lambda,
                       double eps, int32_t max_iter, int32_t positive, float* x, int32_t* iters_host,
                       double* lipschitz_host, void* stream) {
  clear_error();
  if (S < 0 || ldg < S || max_iter < 1 || !(lambda >= 0.0) || !(eps >= 0.0) ||
      (positive != 0 && positive != 1))
    return fail(PC_ERR_INVALID_ARG, "pc_apgd: bad arguments");
  if (S == 0) return PC_OK;
  PC_TRY(check_dev(G, true, "pc_apgd", "G_dev"));
  PC_TRY(check_dev(b, true, "pc_apgd", "b_dev"));
  PC_TRY(check_dev(x, true, "pc_apgd", "x_dev"));
  cudaStream_t st = SS(stream);
  void* scr = nullptr;
  PC_TRY(apgd_scratch(&scr));
  int* d_it = static_cast<int*>(scr);
  double* d_d = reinterpret_cast<double*>(static_cast<char*>(scr) + 16);
  PC_CUDA(cudaMemsetAsync(d_it + 1, 0, sizeof(int), st));
  PC_TRY(run_apgd(G, ldg, b, S, lambda, eps, max_iter, x, d_it, d_d, d_d + 1, st, nullptr, d_it + 1,
                  positive != 0));
  int hi[2] = {0, 0};
  double L = 0.0;
  PC_CUDA(cudaMemcpyAsync(hi, d_it, sizeof(hi), cudaMemcpyDeviceToHost, st));
  PC_CUDA(cudaMemcpyAsync(&L, d_d, sizeof(L), cudaMemcpyDeviceToHost, st));
  PC_CUDA(cudaStreamSynchronize(st));
  if (hi[1]) return fail(PC_ERR_TIMEOUT, "pc_apgd: a bounded device wait expired");
  if (iters_host) *iters_host = hi[0];
  if (lipschitz_host) *lipschitz_host = L;
  return PC_OK;
}

// ------------------------------------------------------------------ the solver

namespace pc {
namespace {

inline int round4(int n) { return (n + 3) & ~3; }

}  // namespace

// ------------------------------------------------------------------ the solve as a job

int parse_solve_opts(const pc_solve_opts* opts, const char* fn, SolveCfg* out, bool resume_ok) {
  SolveCfg c;
  if (opts) {
    if (opts->version != PC_ABI_VERSION)
      return fail(PC_ERR_INVALID_ARG, "%s: opts->version %d != %d", fn, opts->version, PC_ABI_VERSION);
    if (opts->select_rule) c.rule = opts->select_rule;
    if (opts->max_fw) c.max_fw = opts->max_fw;
    if (opts->apgd_max_iter) c.apgd_max = opts->apgd_max_iter;
    if (opts->tol > 0) c.tol = opts->tol;
    if (opts->eps0 > 0) c.eps0 = opts->eps0;
    if (opts->eps_min > 0) c.eps_min = opts->eps_min;
    if (opts->lambda_max > 0) c.lmax = opts->lambda_max;
    c.gram_mode = opts->gram_mode;
    c.positive = opts->positivity;
    c.reweight = opts->reweight;
    c.init_idx = opts->init_idx;
    c.init_x = opts->init_x;
    c.init_S = opts->init_S;
    c.init_k = opts->init_k;
  }
  if (c.init_S != 0 && !resume_ok)
    return fail(PC_ERR_INVALID_ARG, "%s: a resume state (init_S > 0) is accepted by pc_solve only", fn);
  if (c.init_S < 0 || c.init_S > 60000)
    return fail(PC_ERR_INVALID_ARG, "%s: init_S must be in [0, 60000]", fn);
  if (c.init_S > 0) {
    PC_TRY(check_dev(c.init_idx, true, fn, "init_idx"));
    PC_TRY(check_dev(c.init_x, true, fn, "init_x"));
  }
  if (c.init_k < 0 || c.init_k >= c.max_fw)
    return fail(PC_ERR_INVALID_ARG, "%s: init_k must be in [0, max_fw)", fn);
  if (c.reweight < 0 || c.reweight > 2) return fail(PC_ERR_INVALID_ARG, "%s: reweight must be 0, 1 or 2", fn);
  if (c.positive != 0 && c.positive != 1) return fail(PC_ERR_INVALID_ARG, "%s: positivity must be 0 or 1", fn);
  if (c.rule != 1 && c.rule != 2) return fail(PC_ERR_INVALID_ARG, "%s: select_rule must be 1 or 2", fn);
  if (c.gram_mode < 0 || c.gram_mode > 2) return fail(PC_ERR_INVALID_ARG, "%s: gram_mode must be 0, 1 or 2", fn);
  if (c.max_fw < 1 || c.apgd_max < 1) return fail(PC_ERR_INVALID_ARG, "%s: iteration caps must be positive", fn);
  *out = c;
  return PC_OK;
}

SolveJob::~SolveJob() { end_fw_range(); }   // rb, ev, own and the graph stay with the plan

int SolveJob::grow(int need) {
  if (need <= wcap && p->idxB.p) return PC_OK;
  while (wcap < need) wcap *= 2;
  const size_t g = (size_t)round4(wcap) * round4(wcap) * sizeof(float);
  PC_TRY(p->idxA.ensure(sizeof(int32_t) * wcap));
  PC_TRY(p->idxB.ensure(sizeof(int32_t) * wcap));
  PC_TRY(p->xA.ensure(sizeof(float) * wcap));
  PC_TRY(p->xB.ensure(sizeof(float) * wcap));
  PC_TRY(p->bA.ensure(sizeof(float) * wcap));
  PC_TRY(p->bB.ensure(sizeof(float) * wcap));
  PC_TRY(p->oldpos.ensure(sizeof(int32_t) * wcap));
  PC_TRY(p->newrows.ensure(sizeof(int32_t) * wcap));
  PC_TRY(p->keep.ensure(sizeof(int32_t) * wcap));
  PC_TRY(p->atomsA.ensure(sizeof(float4) * wcap));
  PC_TRY(p->atomsB.ensure(sizeof(float4) * wcap));
  PC_TRY(p->GA.ensure(g));
  PC_TRY(p->GB.ensure(g));
  return PC_OK;
}

int SolveJob::start(pc_plan_s* plan, const float2* V_dev, double lambda_, double delta_,
                    const SolveCfg& cfg, float* mu_out, pc_iter_record* hist_, int hist_cap_,
                    cudaStream_t stream) {
  p = plan;
  caller = st = stream;
  V = V_dev;
  lambda = lambda_;
  delta = delta_;
  c = cfg;
  hist = hist_;
  hist_cap = hist_cap_;
  mu_dst = mu_out ? mu_out : p->mu;
  if (!p->scache) p->scache = new SolveCache();
  SolveCache& sc = *p->scache;
  if (!sc.rb && !(sc.rb = pinned_get(sizeof(Readback))))
    return fail(PC_ERR_OOM, "pc_solve: pinned host allocation failed");
  if (!sc.ev) PC_CUDA(cudaEventCreateWithFlags(&sc.ev, cudaEventDisableTiming));
  rb = static_cast<Readback*>(sc.rb);
  ev = sc.ev;
  if (stream == nullptr || stream == cudaStreamLegacy) {
    if (!sc.own && !(sc.own = stream_get())) return fail(PC_ERR_CUDA, "pc_solve: stream creation failed");
    own = sc.own;
    PC_CUDA(cudaEventRecord(ev, stream));
    PC_CUDA(cudaStreamWaitEvent(own, ev, 0));
    st = own;
  }
  PC_TRY(grow(1024));
  // support marks cleared: a solve that ended (converged, capped or failed)
  // after a pruning leaves its support marked, and the first exploration of
  // the next solve on this plan would add those pixels to its active set
  PC_CUDA(cudaMemsetAsync(p->mark, 0, (size_t)p->N * p->N, st));
  // ||V||^2 and r = V; counters, the pruned-support count and the tensor-core
  // flag cleared (the gridding flag iscal[7] may still report an earlier call)
  PC_CUDA(cudaMemsetAsync(p->iscal, 0, 7 * sizeof(int32_t), st));
  PC_CUDA(cudaMemsetAsync(p->dscal, 0, 2 * sizeof(double), st));
  PC_TRY(launch_residual(p->vis_fx, V, p->M, nullptr, 0, p->resid, p->dscal, st));
  rb->hd[1] = (c.rule == 1 && c.lmax > 0) ? (1.0 - delta) * c.lmax : -1.0;   // Delta of rule R1
  PC_CUDA(cudaMemcpyAsync(p->dscal + 4, &rb->hd[1], sizeof(double), cudaMemcpyHostToDevice, st));
  PC_CUDA(cudaMemcpyAsync(&rb->hd[0], p->dscal, sizeof(double), cudaMemcpyDeviceToHost, st));
  PC_CUDA(cudaStreamSynchronize(st));
  sumsqV = rb->hd[0];
  F_prev = F = 0.5 * sumsqV;
  if (c.init_S > 0) PC_TRY(load_resume_state());
  return queue_iteration();
}

// Resume: checks the state on the host (strictly ascending pixels inside the
// image, finite weights, non-negative under positivity), sizes the working
// set for it and starts at iteration init_k. The first chain then prunes
// nothing: it installs the support (k_resume_support), and its readback
// gives F of the given image for the first stop test. G of the support is
// not known, so the first Gram-form reweighting contracts all its rows.
int SolveJob::load_resume_state() {
  const int S = c.init_S;
  std::vector<int32_t> hidx(S);
  std::vector<float> hx(S);
  PC_CUDA(cudaMemcpyAsync(hidx.data(), c.init_idx, sizeof(int32_t) * S, cudaMemcpyDeviceToHost, st));
  PC_CUDA(cudaMemcpyAsync(hx.data(), c.init_x, sizeof(float) * S, cudaMemcpyDeviceToHost, st));
  PC_CUDA(cudaStreamSynchronize(st));
  const int64_t npix = (int64_t)p->N * p->N;
  for (int i = 0; i < S; ++i) {
    if (hidx[i] < 0 || hidx[i] >= npix || (i > 0 && hidx[i] <= hidx[i - 1]))
      return fail(PC_ERR_INVALID_ARG, "pc_solve: init_idx must be strictly ascending pixels below N*N (entry %d)", i);
    if (!std::isfinite(hx[i]) || (c.positive && hx[i] < 0.f))
      return fail(PC_ERR_INVALID_ARG, "pc_solve: init_x[%d] must be finite%s", i,
                  c.positive ? " and non-negative" : "");
  }
  PC_TRY(grow(S));
  k = c.init_k;
  ldB_prev = ld();
  gram_valid = false;
  warm = true;
  return PC_OK;
}

bool SolveJob::ready() const { return cudaEventQuery(ev) == cudaSuccess; }

int SolveJob::explore() {
  const int64_t npix = (int64_t)p->N * p->N;
  int32_t* n_sup_dev = p->iscal + 3;      // support count after the last pruning
  const float* thr_d = nullptr;
  if (c.rule == 1) {
    ProfScope prof_scope_(PROF_MISC, st);
    prof_scope_.kernels = 1;
    k_r1_threshold<<<1, 1, 0, st>>>(p->uscal, c.positive, lambda, delta, k, p->dscal + 4,
                                    reinterpret_cast<float*>(p->dscal + 5));
    PC_LAUNCH_CHECK();
    thr_d = reinterpret_cast<float*>(p->dscal + 5);
  }
  // union with the support: its pixels were marked by the pruning kernel
  // (cleared again after the exploration by k_post_select)
  PC_TRY(launch_select(mu_dst, npix, (float)(1.0 - delta), p->mark, p->idxB.as<int32_t>(), p->iscal,
                       p->sel_blocks, wcap, st, c.positive != 0, thr_d));
  return PC_OK;
}

// The chain of one iteration up to its readback, with every count kept on the
// device (bound: an upper bound of the previous active-set size): the pruning
// of the previous reweighting, the residual and objective of the iterate, its
// certificate and the exploration set.
int SolveJob::enqueue_chain(int bound, int warm_S) {
  int32_t* n_sup_dev = p->iscal + 3;
  PC_CUDA(cudaMemsetAsync(p->dscal, 0, 2 * sizeof(double), st));
  if (warm_S > 0) {
    // resume: the given support in place of the pruning
    ProfScope prof_scope_(PROF_MISC, st);
    prof_scope_.kernels = 1;
    k_resume_support<<<std::min(ceil_div(warm_S, 256), 64), 256, 0, st>>>(
        c.init_idx, c.init_x, warm_S, p->idxA.as<int32_t>(), p->xA.as<float>(), p->atomsA.as<float4>(), p->mark,
        p->dscal + 1, n_sup_dev, p->atom_tab);
    PC_LAUNCH_CHECK();
    bound = warm_S;
  } else if (bound > 0) {
    // pruning: gathers, atoms, support marks and ||x||_1 in one launch
    ProfScope prof_scope_(PROF_MISC, st);
    prof_scope_.kernels = 1;
    dim3 grid(std::max(1, std::min(ceil_div(bound, 256), 32)), std::min(bound, 1024));
    k_prune<<<grid, 256, 0, st>>>(p->keep.as<int32_t>(), n_sup_dev, bound, p->idxB.as<int32_t>(),
                                  p->xB.as<float>(), p->bB.as<float>(), p->GB.as<float>(), ld(),
                                  p->idxA.as<int32_t>(), p->xA.as<float>(), p->bA.as<float>(),
                                  p->GA.as<float>(), p->atomsA.as<float4>(), p->mark, p->dscal + 1,
                                  p->atom_tab);
    PC_LAUNCH_CHECK();
  }
  PC_TRY(launch_residual(p->vis_fx, V, p->M, p->atomsA.as<float4>(), bound, p->resid, p->dscal, st,
                         n_sup_dev));
  PC_CUDA(cudaMemsetAsync(p->uscal, 0, 2 * sizeof(unsigned), st));
  PC_TRY(adjoint_grid_impl(p, p->resid, mu_dst, (float)(1.0 / lambda), p->uscal, st));
  PC_TRY(explore());
  PC_CUDA(cudaMemcpyAsync(rb->hi, p->iscal, sizeof(rb->hi), cudaMemcpyDeviceToHost, st));
  PC_CUDA(cudaMemcpyAsync(rb->hd, p->dscal, sizeof(rb->hd), cudaMemcpyDeviceToHost, st));
  PC_CUDA(cudaMemcpyAsync(rb->mb, p->uscal, sizeof(rb->mb), cudaMemcpyDeviceToHost, st));
  return PC_OK;
}

std::vector<uint64_t> SolveJob::graph_key() const {
  auto u = [](const void* q) { return (uint64_t)(uintptr_t)q; };
  const float inv_l = (float)(1.0 / lambda), thr = (float)(1.0 - delta);
  uint32_t bl, bt;
  std::memcpy(&bl, &inv_l, 4);
  std::memcpy(&bt, &thr, 4);
  return {u(V), u(mu_dst), u(rb), bl, bt, (uint64_t)c.positive, (uint64_t)wcap, u(p->keep.p),
          u(p->idxA.p), u(p->idxB.p), u(p->xA.p), u(p->xB.p), u(p->bA.p), u(p->bB.p), u(p->GA.p),
          u(p->GB.p), u(p->atomsA.p)};
}

// One iteration. With rule R2 (its threshold does not depend on k) and no
// kernel-class timing, the chain is captured as a CUDA graph (bounds = the
// working-set capacity, every count read on the device) and replayed each
// iteration: one launch instead of a dozen. The plan keeps the instantiated
// graph with the arguments it was captured for; it is captured again (and
// the executable updated in place where the topology allows) only when one
// of them changes, e.g. when the working set grows or another V is solved.
int SolveJob::queue_iteration() {
  end_fw_range();
  {
    char name[48];
    std::snprintf(name, sizeof(name), "Frank-Wolfe iteration %d", k);
    fw_range = nvtxRangeStartA(name);
    fw_range_open = true;
  }
  if (k > 0) ldA = ldB_prev;
  if (warm) {
    // the resumed first chain (not captured: the graph holds the pruning)
    PC_TRY(enqueue_chain(0, c.init_S));
  } else if (c.rule == 2 && !prof_active()) {
    SolveCache& sc = *p->scache;
    std::vector<uint64_t> key = graph_key();
    if (!sc.gexec || sc.key != key) {
      cudaGraph_t g = nullptr;
      PC_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
      const int rc = enqueue_chain(wcap);
      const cudaError_t e = cudaStreamEndCapture(st, &g);
      PC_TRY(rc);
      PC_CUDA(e);
      if (sc.gexec) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(sc.gexec, g, &info) != cudaSuccess) {
          cudaGetLastError();
          cudaGraphExecDestroy(sc.gexec);
          sc.gexec = nullptr;
        }
      }
      cudaError_t ei = cudaSuccess;
      if (!sc.gexec) ei = cudaGraphInstantiate(&sc.gexec, g, 0);
      cudaGraphDestroy(g);
      if (ei != cudaSuccess) sc.gexec = nullptr;
      PC_CUDA(ei);
      sc.key = std::move(key);
    }
    PC_CUDA(cudaGraphLaunch(sc.gexec, st));
  } else {
    PC_TRY(enqueue_chain(k > 0 ? n_prev_act : 0));
  }
  PC_CUDA(cudaEventRecord(ev, st));
  return PC_OK;
}

int SolveJob::process() {
  need_apgd = false;
  const Readback r = *rb;
  if (r.hi[7]) {
    PC_CUDA(cudaMemsetAsync(p->iscal + 7, 0, sizeof(int32_t), st));
    return fail(PC_ERR_TIMEOUT, "pc_solve: a bounded tensor-core gridding wait expired");
  }
  if (r.hi[4]) return fail(PC_ERR_TIMEOUT, "pc_solve: a bounded device wait expired");
  mu_inf = (double)bits_to_float(r.mb[0]);
  if (!std::isfinite(mu_inf)) return fail(PC_ERR_NUMERIC, "pc_solve: non-finite certificate at iteration %d", k);
  const double mu_top = c.positive ? (double)key_to_float(r.mb[1]) : mu_inf;
  if (warm) {
    // the resumed image: its support and objective start the run
    warm = false;
    nS = r.hi[3];
    F = 0.5 * r.hd[0] + lambda * r.hd[1];
    F_prev = F;
    if (!std::isfinite(F)) return fail(PC_ERR_NUMERIC, "pc_solve: non-finite objective of the resume state");
  } else if (k > 0) {
    nS = r.hi[3];
    F = 0.5 * r.hd[0] + lambda * r.hd[1];
    const double rel = F_prev > 0 ? (F_prev - F) / F_prev : 0.0;
    if (have_cur) {
      cur.n_support = nS;
      cur.apgd_iterations = r.hi[2];
      last_apgd_iters = r.hi[2];
      cur.lanczos_steps = r.hi[5];
      cur.lipschitz = r.hd[2];
      cur.objective = F;
      cur.rel_improvement = rel;
      if (n_hist < hist_cap && hist) hist[n_hist] = cur;
      ++n_hist;
      have_cur = false;
    }
    F_prev = F;
    if (!std::isfinite(F)) return fail(PC_ERR_NUMERIC, "pc_solve: non-finite objective at iteration %d", k);
    if (rel < c.tol) {
      status = PC_OK;
      done = true;
      return PC_OK;
    }
    if (k >= c.max_fw) {
      status = PC_ERR_NOT_CONVERGED;
      done = true;
      return PC_OK;
    }
  }
  n_act = r.hi[0];
  while (n_act > wcap) {
    if (n_act > 60000) return fail(PC_ERR_CAPACITY, "pc_solve: active set of %d atoms too large", n_act);
    // grow, keeping the current support and weights
    int32_t* old_idx = nullptr;
    const size_t gbytes = (size_t)nS * ldA * sizeof(float);
    PC_TRY(dmalloc(reinterpret_cast<void**>(&old_idx), sizeof(int32_t) * std::max(nS, 1) * 3 + gbytes + 16, st));
    float* old_x = reinterpret_cast<float*>(old_idx + std::max(nS, 1));
    float* old_b = old_x + std::max(nS, 1);
    float* old_G = old_b + std::max(nS, 1);
    PC_CUDA(cudaMemcpyAsync(old_idx, p->idxA.p, sizeof(int32_t) * nS, cudaMemcpyDeviceToDevice, st));
    PC_CUDA(cudaMemcpyAsync(old_x, p->xA.p, sizeof(float) * nS, cudaMemcpyDeviceToDevice, st));
    PC_CUDA(cudaMemcpyAsync(old_b, p->bA.p, sizeof(float) * nS, cudaMemcpyDeviceToDevice, st));
    PC_CUDA(cudaMemcpyAsync(old_G, p->GA.p, gbytes, cudaMemcpyDeviceToDevice, st));
    PC_CUDA(cudaStreamSynchronize(st));
    int rc = grow(n_act);
    if (rc == PC_OK) {
      cudaMemcpyAsync(p->idxA.p, old_idx, sizeof(int32_t) * nS, cudaMemcpyDeviceToDevice, st);
      cudaMemcpyAsync(p->xA.p, old_x, sizeof(float) * nS, cudaMemcpyDeviceToDevice, st);
      cudaMemcpyAsync(p->bA.p, old_b, sizeof(float) * nS, cudaMemcpyDeviceToDevice, st);
      cudaMemcpyAsync(p->GA.p, old_G, gbytes, cudaMemcpyDeviceToDevice, st);
      cudaStreamSynchronize(st);
    }
    dfree(old_idx, st);
    PC_TRY(rc);
    PC_LAUNCH_CHECK();
    PC_TRY(explore());
    PC_TRY(sync_read(&n_act, p->iscal, sizeof(int), st));
  }
  const int n_new = n_act - nS;
  cur = pc_iter_record{};
  cur.k = k;
  cur.n_new = n_new;
  cur.n_active = n_act;
  cur.mu_inf = mu_top;
  have_cur = true;

  ldB = ld();
  if (n_act > 0) {
    int32_t* oldpos = p->oldpos.as<int32_t>();
    PC_TRY(choose_form(n_new, n_act, &op_form));
    {
      // old positions, new-atom list, warm start, b of the old atoms, atoms; marks cleared
      ProfScope prof_scope_(PROF_MISC, st);
      prof_scope_.kernels = 1;
      k_post_select<<<1, 1024, 0, st>>>(p->idxB.as<int32_t>(), n_act, p->idxA.as<int32_t>(), nS,
                                        p->xA.as<float>(), p->bA.as<float>(), oldpos,
                                        p->newrows.as<int32_t>(), p->iscal + 1, p->xB.as<float>(),
                                        p->bB.as<float>(), p->atomsB.as<float4>(), p->mark, p->atom_tab);
      PC_LAUNCH_CHECK();
    }
    eps = std::max(c.eps_min, c.eps0 * std::pow(2.0, -k));
    need_apgd = true;
    if (op_form) {
      // operator form: no Gram; the next Gram-form iteration rebuilds all of G_S
      gram_valid = false;
      return PC_OK;
    }
    if (gram_valid) {
      // old-old block of G
      PC_TRY(gather_sym(p->GA.as<float>(), ldA, oldpos, n_act, p->GB.as<float>(), ldB, st));
      // Gram rows of the new atoms against every active atom, and b
      if (n_new > 0) {
        PC_TRY(gram_update(p, V, p->atomsB.as<float4>(), n_act, p->newrows.as<int32_t>(), n_new, oldpos,
                           p->GB.as<float>(), ldB, p->bB.as<float>(), c.gram_mode, p->iscal + 4, st));
      }
    } else {
      // after an operator-form iteration: every row of G_S and all of b
      k_iota<<<ceil_div(n_act, 256), 256, 0, st>>>(p->newrows.as<int32_t>(), n_act);
      PC_LAUNCH_CHECK();
      PC_TRY(gram_update(p, V, p->atomsB.as<float4>(), n_act, p->newrows.as<int32_t>(), n_act, nullptr,
                         p->GB.as<float>(), ldB, p->bB.as<float>(), c.gram_mode, p->iscal + 4, st));
      gram_valid = true;
    }
    return PC_OK;
  }
  PC_CUDA(cudaMemsetAsync(p->iscal + 3, 0, sizeof(int32_t), st));
  n_prev_act = 0;
  ldB_prev = ldB;
  ++k;
  return queue_iteration();
}

// The form of this iteration's reweighting: the Gram form costs the
// contraction of the Gram rows it needs (all of them after an operator-form
// iteration) plus a negligible APGD on G; the operator form costs one
// degridding + gridding pair per Lanczos step (about 16) and per FISTA
// iteration (estimated by the previous reweighting's count, at least 20).
// Contraction rates are the ones measured on this GPU for the kernel the
// Gram form would use (tensor cores ~0.5 PFLOP/s on split FP16 including the
// phase generation; FP32 CUDA cores ~24 TFLOP/s on full tiles).
int SolveJob::choose_form(int n_new, int n_act, bool* op) {
  *op = false;
  if (c.reweight == 1 || p->M <= 0) return PC_OK;
  if (c.reweight == 2) {
    *op = true;
    return PC_OK;
  }
  const double M = (double)p->M;
  const int rows = gram_valid ? n_new : n_act;            // Gram rows to contract
  if (rows <= 0) return PC_OK;
  const bool thin = rows + 1 <= 16 && c.gram_mode < 2;
  const bool tc = !thin && (c.gram_mode >= 2 || (c.gram_mode == 0 && (int64_t)rows * n_act >= 64 * 64));
  const double entries = (double)rows * (n_act + 1) - (double)rows * (rows - 1) / 2.0;
  double t_gram;
  if (tc) t_gram = 12.0 * M * entries / 5.0e14;
  else if (thin) t_gram = 2.0 * M * (double)(rows + 1) * n_act / 2.0e12;   // latency-bound phase chains
  else t_gram = 4.0 * M * (double)rows * (n_act + 1) / 2.4e13;
  if (t_gram < 0.02) return PC_OK;                         // not worth timing the operators
  double pair = 0.0;
  PC_TRY(op_pair_seconds(p, st, &pair));
  const double iters = std::max(20, last_apgd_iters) + 16;
  *op = iters * pair < t_gram;
  return PC_OK;
}

int SolveJob::run_apgd_op() {
  if (!dirty_ready) {
    // Re Phi* V on every pixel, once per solve: its values on the active set start Lanczos
    PC_TRY(p->dirty.ensure(sizeof(float) * (size_t)p->N * p->N));
    PC_TRY(adjoint_grid_impl(p, V, p->dirty.as<float>(), 1.0f, nullptr, st));
    dirty_ready = true;
  }
  return run_operator_apgd(p, V, p->dirty.as<float>(), p->idxB.as<int32_t>(), n_act, lambda, eps, c.apgd_max,
                           c.positive != 0, p->xB.as<float>(), p->iscal + 2, p->dscal + 2, p->iscal + 5, st);
}

ApgdJob SolveJob::apgd_job() const {
  return ApgdJob{p->GB.as<float>(), ldB, p->bB.as<float>(), n_act, lambda, eps, c.apgd_max,
                 p->xB.as<float>(), p->iscal + 2, p->dscal + 2, p->dscal + 3, p->iscal + 5,
                 p->iscal + 4, c.positive != 0};
}

int SolveJob::after_apgd() {
  need_apgd = false;
  // the nonzero positions; the gathers run at the start of the next iteration
  PC_TRY(launch_compact_nonzero(p->xB.as<float>(), n_act, p->keep.as<int32_t>(), p->iscal + 3, st));
  n_prev_act = n_act;
  ldB_prev = ldB;
  ++k;
  return queue_iteration();
}

int SolveJob::finish(int32_t* idx_out, float* x_out, int32_t cap, pc_solve_stats* stats) {
  end_fw_range();
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
  if (nS > cap) return fail(PC_ERR_CAPACITY, "pc_solve: support of %d atoms exceeds capacity %d", nS, cap);
  if (nS > 0) {
    PC_CUDA(cudaMemcpyAsync(idx_out, p->idxA.p, sizeof(int32_t) * nS, cudaMemcpyDeviceToDevice, st));
    PC_CUDA(cudaMemcpyAsync(x_out, p->xA.p, sizeof(float) * nS, cudaMemcpyDeviceToDevice, st));
  }
  if (own) {
    PC_CUDA(cudaEventRecord(ev, st));
    PC_CUDA(cudaStreamWaitEvent(caller, ev, 0));
  }
  if (status == PC_ERR_NOT_CONVERGED)
    fail(PC_ERR_NOT_CONVERGED, "pc_solve: no convergence after %d Frank-Wolfe iterations", k);
  return status;
}

}  // namespace pc

using namespace pc;

extern "C" int pc_solve(pc_plan_t p, const pc_c32* V_, double lambda, double delta,
                        const pc_solve_opts* opts, int32_t* idx_out, float* x_out, int32_t cap,
                        float* mu_out, pc_solve_stats* stats, pc_iter_record* hist,
                        int32_t hist_cap, void* stream) {
  clear_error();
  PC_TRY(check_plan(p, "pc_solve"));
  if (!(lambda > 0.0) || !std::isfinite(lambda))
    return fail(PC_ERR_INVALID_ARG, "pc_solve: lambda must be positive and finite");
  if (!(delta > 0.0 && delta <= 1.0)) return fail(PC_ERR_INVALID_ARG, "pc_solve: delta must be in (0, 1]");
  if (cap < 0 || hist_cap < 0) return fail(PC_ERR_INVALID_ARG, "pc_solve: negative capacity");
  PC_TRY(check_dev(V_, p->M > 0, "pc_solve", "V_dev"));
  PC_TRY(check_dev(idx_out, cap > 0, "pc_solve", "idx_out_dev"));
  PC_TRY(check_dev(x_out, cap > 0, "pc_solve", "x_out_dev"));
  if (mu_out) PC_TRY(check_dev(mu_out, true, "pc_solve", "mu_out_dev"));
  SolveCfg c;
  PC_TRY(parse_solve_opts(opts, "pc_solve", &c, true));
  cudaStream_t st = SS(stream);
  // NVTX: the whole call, with one range per Frank-Wolfe iteration inside
  struct SolveRange {
    SolveRange() { nvtxRangePushA("pc_solve"); }
    ~SolveRange() { nvtxRangePop(); }
  } solve_range;
  SolveJob j;
  PC_TRY(j.start(p, reinterpret_cast<const float2*>(V_), lambda, delta, c, mu_out, hist, hist_cap, st));
  while (!j.done) {
    PC_CUDA(cudaEventSynchronize(j.ev));
    PC_TRY(j.process());
    if (j.need_apgd) {
      if (j.op_form) {
        PC_TRY(j.run_apgd_op());
      } else {
        const ApgdJob aj = j.apgd_job();
        PC_TRY(run_apgd_jobs(&aj, 1, j.st));
      }
      PC_TRY(j.after_apgd());
    }
  }
  return j.finish(idx_out, x_out, cap, stats);
}

extern "C" int pc_solve_host(const double* uvw_host, const pc_c32* V_host, int64_t M, int32_t N,
                             double fov_rad, double alpha, double delta, const pc_solve_opts* opts,
                             int32_t* idx_out_host, float* x_out_host, int32_t cap,
                             pc_solve_stats* stats_host, void* stream) {
  clear_error();
  if (M < 0 || (M > 0 && (!uvw_host || !V_host)) || cap < 0 || (cap > 0 && (!idx_out_host || !x_out_host)))
    return fail(PC_ERR_INVALID_ARG, "pc_solve_host: bad arguments");
  if (!(alpha > 0.0 && alpha <= 1.0)) return fail(PC_ERR_INVALID_ARG, "pc_solve_host: alpha must be in (0, 1]");
  if (opts && opts->init_S != 0)
    return fail(PC_ERR_INVALID_ARG, "pc_solve_host: a resume state (init_S > 0) is accepted by pc_solve only");
  cudaStream_t st = SS(stream);
  void* buf = nullptr;
  const size_t b_uvw = sizeof(double) * 3 * (size_t)std::max<int64_t>(M, 1);
  const size_t b_V = sizeof(pc_c32) * (size_t)std::max<int64_t>(M, 1);
  const size_t b_idx = sizeof(int32_t) * (size_t)std::max(cap, 1);
  const size_t b_x = sizeof(float) * (size_t)std::max(cap, 1);
  PC_TRY(dmalloc(&buf, b_uvw + b_V + b_idx + b_x + 64, st));
  char* base = static_cast<char*>(buf);
  double* d_uvw = reinterpret_cast<double*>(base);
  pc_c32* d_V = reinterpret_cast<pc_c32*>(base + b_uvw);
  int32_t* d_idx = reinterpret_cast<int32_t*>(base + b_uvw + b_V);
  float* d_x = reinterpret_cast<float*>(base + b_uvw + b_V + b_idx);
  int rc = PC_OK;
  pc_plan_t plan = nullptr;
  pc_solve_stats local{};
  do {
    if (M > 0) {
      if (cudaMemcpyAsync(d_uvw, uvw_host, sizeof(double) * 3 * M, cudaMemcpyHostToDevice, st) != cudaSuccess ||
          cudaMemcpyAsync(d_V, V_host, sizeof(pc_c32) * M, cudaMemcpyHostToDevice, st) != cudaSuccess) {
        rc = fail(PC_ERR_CUDA, "pc_solve_host: host-to-device copy failed");
        break;
      }
    }
    rc = pc_plan_create(d_uvw, M, N, fov_rad, nullptr, stream, &plan);
    if (rc != PC_OK) break;
    double lmax = 0.0;
    // under positivity lambda_max is max(0, max Phi* V) (the optimality condition at x = 0)
    rc = (opts && opts->positivity) ? pc_lambda_max_positive(plan, d_V, &lmax, stream)
                                    : pc_lambda_max(plan, d_V, &lmax, stream);
    if (rc != PC_OK) break;
    if (!(lmax > 0.0)) {   // V == 0: the solution is x = 0
      local.status = PC_OK;
      local.n_support = 0;
      break;
    }
    rc = pc_solve(plan, d_V, alpha * lmax, delta, opts, d_idx, d_x, cap, nullptr, &local, nullptr, 0, stream);
    if (rc != PC_OK && rc != PC_ERR_NOT_CONVERGED) break;
    const int n = std::min(local.n_support, cap);
    if (n > 0) {
      cudaMemcpyAsync(idx_out_host, d_idx, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st);
      cudaMemcpyAsync(x_out_host, d_x, sizeof(float) * n, cudaMemcpyDeviceToHost, st);
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) rc = fail(PC_ERR_CUDA, "pc_solve_host: device-to-host copy failed");
  } while (0);
  if (plan) pc_plan_destroy(plan);
  dfree(buf, st);
  if (stats_host) *stats_host = local;
  return rc;
}
