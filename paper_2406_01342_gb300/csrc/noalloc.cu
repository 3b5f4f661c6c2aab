// Allocation-free adjoint on a pixel subset: pc_adjoint_sparse_noalloc.
//
// Some callers cannot allocate device memory at all: code running inside an
// arena that has handed out every byte up front, real-time pipelines whose
// memory budget is fixed once at start-up, or hosts that forbid new
// allocations while other work is queued. pc_adjoint_sparse needs a plan,
// and building a plan allocates. This entry point takes the raw uvw array
// instead of a plan and keeps its only scratch -- one float64 accumulator per
// requested pixel -- in a file-scope __device__ array of fixed size, so that
// no call ever allocates.
//
// Scratch rules: the array holds kNoAllocMaxPixels doubles (64 KB) on every
// device that loads the library, until the process exits. Each call clears
// the part it uses before accumulating into it. All calls share the one
// array, so calls whose kernels overlap on the GPU (different streams, or
// different host threads) race on it and give wrong results: serialise them.
// The first call on a device looks up the array's device address with
// cudaGetSymbolAddress (with that device current); under lazy module loading
// (the CUDA default) that first call also loads this file's kernels and the
// array itself, which takes device memory at that moment. So make the first
// call at start-up, before an arena or a memory budget takes the device's
// memory, and before any stream capture begins; later calls allocate nothing.
// At most 65535 x 8192 visibilities (the launch's y dimension) per call.
#include <mutex>

#include "pc_internal.cuh"

namespace pc {
namespace {

constexpr int kNoAllocMaxPixels = 8192;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_acc[kNoAllocMaxPixels];

constexpr int NA_PIX = 128;        // pixels per CTA
constexpr int NA_CHUNK = 256;      // visibilities staged per shared-memory chunk
constexpr int NA_SLICE = 8192;     // visibilities per CTA (one float64 flush per slice)
// The slices are the launch's y dimension (at most 65535 blocks).
constexpr int64_t kNoAllocMaxVis = 65535ll * NA_SLICE;

// acc[s] += sum_k Re(y_k e^{+j 2 pi theta_ks}) / n_s over one slice of visibilities,
// phases formed exactly as in the plan-based path (32-bit fixed-point lattice
// turns from float64 u dl, v dl; double-float w-term).
__global__ void __launch_bounds__(256)
k_adjoint_sparse_noalloc(const double* __restrict__ uvw, int64_t M, int N, double dl,
                         const float2* __restrict__ y, const int32_t* __restrict__ idx, int S,
                         double* __restrict__ acc) {
  __shared__ float4 s_atom[NA_PIX];
  __shared__ int4 s_vis[NA_CHUNK];
  __shared__ float2 s_y[NA_CHUNK];
  __shared__ float s_part[256];
  const int p0 = blockIdx.x * NA_PIX;
  for (int t = threadIdx.x; t < NA_PIX; t += blockDim.x) {
    const int s = p0 + t;
    float4 at = make_float4(0.f, 0.f, 0.f, 0.f);
    if (s < S) {
      const int p = min(max(idx[s], 0), N * N - 1);
      const int ip = p / N - N / 2, jp = p % N - N / 2;
      const double l = ip * dl, m = jp * dl, r2 = l * l + m * m;
      const double n = sqrt(1.0 - r2), sv = -r2 / (1.0 + n);
      const float s_hi = (float)sv;
      const int packed = (int)(((unsigned)ip << 16) | ((unsigned)jp & 0xffffu));
      at = make_float4(__int_as_float(packed), s_hi, (float)(sv - (double)s_hi), (float)(1.0 / n));
    }
    s_atom[t] = at;
  }
  const int col = threadIdx.x % NA_PIX;
  const int half = threadIdx.x / NA_PIX;
  const int64_t k_lo = (int64_t)blockIdx.y * NA_SLICE;
  const int64_t k_hi = min(M, k_lo + NA_SLICE);
  float outer = 0.f;
  for (int64_t k0 = k_lo; k0 < k_hi; k0 += NA_CHUNK) {
    __syncthreads();
    for (int t = threadIdx.x; t < NA_CHUNK; t += blockDim.x) {
      const int64_t k = k0 + t;
      int4 v = make_int4(0, 0, 0, 0);
      float2 h = make_float2(0.f, 0.f);
      if (k < k_hi) {
        const double U = uvw[3 * k] * dl, Vv = uvw[3 * k + 1] * dl, w = uvw[3 * k + 2];
        const double fu = U - rint(U), fv = Vv - rint(Vv);
        const float w_hi = (float)w;
        v = make_int4((int)(unsigned)(long long)llrint(fu * 4294967296.0),
                      (int)(unsigned)(long long)llrint(fv * 4294967296.0), __float_as_int(w_hi),
                      __float_as_int((float)(w - (double)w_hi)));
        h = y[k];
      }
      s_vis[t] = v;
      s_y[t] = h;
    }
    __syncthreads();
    const float4 at = s_atom[col];
    float inner = 0.f;
    for (int t = half; t < NA_CHUNK; t += 2) {
      float sn, cs;
      sincospif(2.0f * phase_turns(s_vis[t], at), &sn, &cs);
      const float2 h = s_y[t];
      inner = fmaf(h.x, cs, fmaf(-h.y, sn, inner));
    }
    outer += inner * at.w;
  }
  s_part[threadIdx.x] = outer;
  __syncthreads();
  if (half == 0 && p0 + col < S)
    atomicAdd(&acc[p0 + col], (double)s_part[threadIdx.x] + (double)s_part[threadIdx.x + NA_PIX]);
}

// out[s] = acc[s]; NaN for a pixel index outside [0, N*N).
__global__ void k_noalloc_finish(const double* __restrict__ acc, const int32_t* __restrict__ idx,
                                 int S, int NN, float* __restrict__ out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  const int p = idx[s];
  out[s] = (p >= 0 && p < NN) ? (float)acc[s] : __int_as_float(0x7fc00000);
}

std::mutex g_setup_mu;
double* g_acc_addr[kMaxDevices] = {nullptr};

int noalloc_scratch(int dev, double** out) {
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_acc_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_acc);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(PC_ERR_CUDA, "pc_adjoint_sparse_noalloc: cudaGetSymbolAddress failed: %s",
                  cudaGetErrorString(e));
    }
    g_acc_addr[dev] = static_cast<double*>(p);
  }
  *out = g_acc_addr[dev];
  return PC_OK;
}

}  // namespace
}  // namespace pc

using namespace pc;

extern "C" int pc_adjoint_sparse_noalloc(const double* uvw_dev, int64_t M, int32_t N,
                                         double fov_rad, const pc_c32* y_dev,
                                         const int32_t* idx_dev, int32_t S, float* out_dev,
                                         void* stream) {
  clear_error();
  if (S < 0 || S > kNoAllocMaxPixels)
    return fail(PC_ERR_INVALID_ARG,
                "pc_adjoint_sparse_noalloc: S = %d pixels, the allocation-free path takes at most %d",
                S, kNoAllocMaxPixels);
  if (M < 0 || N < 2 || N > 4096 || (N & 1) || !(fov_rad > 0.0) || !(fov_rad < 1.4))
    return fail(PC_ERR_INVALID_ARG, "pc_adjoint_sparse_noalloc: bad geometry (M, N, fov)");
  if (M > kNoAllocMaxVis)
    return fail(PC_ERR_INVALID_ARG,
                "pc_adjoint_sparse_noalloc: M = %lld visibilities, the allocation-free path takes at most %lld",
                (long long)M, (long long)kNoAllocMaxVis);
  if (S == 0) return PC_OK;
  if (!is_device_ptr(idx_dev) || !is_device_ptr(out_dev) ||
      (M > 0 && (!is_device_ptr(uvw_dev) || !is_device_ptr(y_dev))))
    return fail(PC_ERR_INVALID_ARG, "pc_adjoint_sparse_noalloc: arguments must be device pointers");
  int dev = 0;
  PC_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices)
    return fail(PC_ERR_INVALID_ARG, "pc_adjoint_sparse_noalloc: device %d out of range", dev);
  double* acc = nullptr;
  PC_TRY(noalloc_scratch(dev, &acc));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  PC_CUDA(cudaMemsetAsync(acc, 0, sizeof(double) * (size_t)S, st));
  if (M > 0) {
    dim3 grid(ceil_div(S, NA_PIX), ceil_div(M, NA_SLICE));
    k_adjoint_sparse_noalloc<<<grid, 256, 0, st>>>(uvw_dev, M, N, fov_rad / N,
                                                   reinterpret_cast<const float2*>(y_dev), idx_dev,
                                                   S, acc);
    PC_LAUNCH_CHECK();
  }
  k_noalloc_finish<<<ceil_div(S, 256), 256, 0, st>>>(acc, idx_dev, S, N * N, out_dev);
  PC_LAUNCH_CHECK();
  return PC_OK;
}
