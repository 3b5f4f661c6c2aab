// Atom selection and support bookkeeping of Algorithm 2:
//   exploration (step 1a)  I = {p : |mu_p| >= thr}  (mu_p >= thr with the
//                          positivity constraint: candidates only at positive values)
//   union (step 1b)        S u I in ascending raster order (stream compaction
//                          over all N^2 pixels of  |mu_p| >= thr  or  p in S)
//   pruning (step 3)       positions of the nonzero weights
#include "pc_internal.cuh"

namespace pc {
namespace {

constexpr int SEL_THREADS = 256;
constexpr int SEL_ITEMS = kSelItems;   // 1024 per block: 256 blocks for 512 x 512, several per SM
constexpr int SEL_ROUNDS = SEL_ITEMS / SEL_THREADS;

__device__ __forceinline__ bool sel_flag(const float* mu, const uint8_t* mark, int64_t p, float thr,
                                         int positive) {
  const float v = mu[p];
  return (positive ? v : fabsf(v)) >= thr || mark[p] != 0;
}

// Exclusive scan of n ints in place by one block; a[n] receives the total.
__device__ void block_exclusive_scan(int32_t* a, int n) {
  __shared__ int warp_tot[32];
  const int chunk = (n + blockDim.x - 1) / blockDim.x;
  const int lo = threadIdx.x * chunk, hi = min(lo + chunk, n);
  int s = 0;
  for (int i = lo; i < hi; ++i) s += ((volatile int32_t*)a)[i];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int incl = s;
  for (int off = 1; off < 32; off <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += t;
  }
  if (lane == 31) warp_tot[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    int t = lane < nw ? warp_tot[lane] : 0;
    int ti = t;
    for (int off = 1; off < 32; off <<= 1) {
      int u = __shfl_up_sync(0xffffffffu, ti, off);
      if (lane >= off) ti += u;
    }
    if (lane < nw) warp_tot[lane] = ti - t;
    if (lane == nw - 1) a[n] = ti;
  }
  __syncthreads();
  int run = warp_tot[wid] + incl - s;
  for (int i = lo; i < hi; ++i) {
    const int v = ((volatile int32_t*)a)[i];
    a[i] = run;
    run += v;
  }
}

// Per-block counts; the last block to finish scans them (block_counts[nblk]
// = total, also written to *count_dev) and resets the arrival counter
// block_counts[nblk + 1], so the write pass needs no separate scan launch.
__global__ void k_sel_count(const float* __restrict__ mu, const uint8_t* __restrict__ mark,
                            int64_t npix, float thr, int positive, int32_t* __restrict__ block_counts,
                            const float* __restrict__ thr_dev, int nblk, int32_t* __restrict__ count_dev) {
  __shared__ int wsum[SEL_THREADS / 32];
  __shared__ bool s_last;
  if (thr_dev) thr = *thr_dev;
  int c = 0;
  const int64_t base = (int64_t)blockIdx.x * SEL_ITEMS;
  for (int r = 0; r < SEL_ROUNDS; ++r) {
    const int64_t p = base + r * SEL_THREADS + threadIdx.x;
    if (p < npix && sel_flag(mu, mark, p, thr, positive)) ++c;
  }
  for (int off = 16; off; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < SEL_THREADS / 32; ++w) t += wsum[w];
    block_counts[blockIdx.x] = t;
    __threadfence();
    s_last = atomicAdd(&block_counts[nblk + 1], 1) == nblk - 1;
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    block_exclusive_scan(block_counts, nblk);
    if (threadIdx.x == 0) {
      *count_dev = block_counts[nblk];
      block_counts[nblk + 1] = 0;
    }
  }
}

__global__ void k_sel_write(const float* __restrict__ mu, const uint8_t* __restrict__ mark,
                            int64_t npix, float thr, int positive, const int32_t* __restrict__ block_off,
                            int32_t* __restrict__ out, int cap, const float* __restrict__ thr_dev) {
  __shared__ int wcount[SEL_THREADS / 32];
  __shared__ int run_s;
  if (thr_dev) thr = *thr_dev;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) run_s = block_off[blockIdx.x];
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * SEL_ITEMS;
  for (int r = 0; r < SEL_ROUNDS; ++r) {
    const int64_t p = base + r * SEL_THREADS + threadIdx.x;
    const bool f = p < npix && sel_flag(mu, mark, p, thr, positive);
    const unsigned bal = __ballot_sync(0xffffffffu, f);
    if (lane == 0) wcount[warp] = __popc(bal);
    __syncthreads();
    int before = 0, total = 0;
    for (int w = 0; w < SEL_THREADS / 32; ++w) {
      const int cw = wcount[w];
      if (w < warp) before += cw;
      total += cw;
    }
    if (f) {
      const int pos = run_s + before + __popc(bal & ((1u << lane) - 1u));
      if (pos < cap) out[pos] = (int32_t)p;
    }
    __syncthreads();
    if (threadIdx.x == 0) run_s += total;
    __syncthreads();
  }
}

__global__ void k_mark(uint8_t* __restrict__ mark, const int32_t* __restrict__ idx, int n,
                       uint8_t value, const int32_t* __restrict__ n_dev) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (n_dev) n = min(n, *n_dev);
  if (s < n) mark[idx[s]] = value;
}

// oldpos[i] = position of newidx[i] in the ascending list oldidx, or -1.
__global__ void k_old_positions(const int32_t* __restrict__ newidx, int n_new,
                                const int32_t* __restrict__ oldidx, int n_old,
                                int32_t* __restrict__ oldpos) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_new) return;
  const int v = newidx[i];
  int lo = 0, hi = n_old;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (oldidx[mid] < v) lo = mid + 1; else hi = mid;
  }
  oldpos[i] = (lo < n_old && oldidx[lo] == v) ? lo : -1;
}

// Ascending positions i that satisfy the predicate (mode 0: x[i] != 0;
// 1: oldpos[i] < 0, a new atom; 2: oldpos[i] >= 0, an old atom);
// count_dev[0] = their number. One block.
__global__ void k_compact_single(const float* __restrict__ x, const int32_t* __restrict__ oldpos,
                                 int n, int32_t* __restrict__ out, int32_t* __restrict__ count_dev,
                                 int mode) {
  __shared__ int wcount[32];
  __shared__ int run_s;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) run_s = 0;
  __syncthreads();
  for (int base = 0; base < n; base += blockDim.x) {
    const int i = base + threadIdx.x;
    bool f = false;
    if (i < n) f = mode == 0 ? (x[i] != 0.0f) : (mode == 1 ? oldpos[i] < 0 : oldpos[i] >= 0);
    const unsigned bal = __ballot_sync(0xffffffffu, f);
    if (lane == 0) wcount[warp] = __popc(bal);
    __syncthreads();
    int before = 0, total = 0;
    for (int w = 0; w < nw; ++w) {
      if (w < warp) before += wcount[w];
      total += wcount[w];
    }
    if (f) out[run_s + before + __popc(bal & ((1u << lane) - 1u))] = i;
    __syncthreads();
    if (threadIdx.x == 0) run_s += total;
    __syncthreads();
  }
  if (threadIdx.x == 0) count_dev[0] = run_s;
}

}  // namespace

int launch_select(const float* mu, int64_t npix, float thr, const uint8_t* mark, int32_t* out,
                  int32_t* count_dev, int32_t* block_counts, int cap, cudaStream_t st, bool positive,
                  const float* thr_dev) {
  ProfScope prof_scope_(PROF_SELECT, st);
  const int nblk = ceil_div(npix, SEL_ITEMS);
  prof_scope_.kernels = 2;
  k_sel_count<<<nblk, SEL_THREADS, 0, st>>>(mu, mark, npix, thr, positive ? 1 : 0, block_counts, thr_dev,
                                             nblk, count_dev);
  PC_LAUNCH_CHECK();
  k_sel_write<<<nblk, SEL_THREADS, 0, st>>>(mu, mark, npix, thr, positive ? 1 : 0, block_counts, out, cap,
                                             thr_dev);
  PC_LAUNCH_CHECK();
  return PC_OK;
}

int launch_mark(uint8_t* mark, const int32_t* idx, int n, uint8_t value, cudaStream_t st,
                const int32_t* n_dev) {
  ProfScope prof_scope_(PROF_MISC, st);
  if (n <= 0) return PC_OK;
  prof_scope_.kernels = 1;
  k_mark<<<ceil_div(n, 256), 256, 0, st>>>(mark, idx, n, value, n_dev);
  PC_LAUNCH_CHECK();
  return PC_OK;
}

int launch_old_positions(const int32_t* newidx, int n_new, const int32_t* oldidx, int n_old,
                         int32_t* oldpos, cudaStream_t st) {
  ProfScope prof_scope_(PROF_MISC, st);
  if (n_new <= 0) return PC_OK;
  prof_scope_.kernels = 1;
  k_old_positions<<<ceil_div(n_new, 256), 256, 0, st>>>(newidx, n_new, oldidx, n_old, oldpos);
  PC_LAUNCH_CHECK();
  return PC_OK;
}

int launch_compact_nonzero(const float* x, int n, int32_t* keep, int32_t* count_dev,
                           cudaStream_t st) {
  ProfScope prof_scope_(PROF_MISC, st);
  prof_scope_.kernels = 1;
  k_compact_single<<<1, 1024, 0, st>>>(x, nullptr, n, keep, count_dev, 0);
  PC_LAUNCH_CHECK();
  return PC_OK;
}

int launch_compact_new(const int32_t* oldpos, int n, int32_t* rows, int32_t* count_dev,
                       cudaStream_t st) {
  ProfScope prof_scope_(PROF_MISC, st);
  prof_scope_.kernels = 1;
  k_compact_single<<<1, 1024, 0, st>>>(nullptr, oldpos, n, rows, count_dev, 1);
  PC_LAUNCH_CHECK();
  return PC_OK;
}

int launch_compact_old(const int32_t* oldpos, int n, int32_t* rows, int32_t* count_dev,
                       cudaStream_t st) {
  ProfScope prof_scope_(PROF_MISC, st);
  prof_scope_.kernels = 1;
  k_compact_single<<<1, 1024, 0, st>>>(nullptr, oldpos, n, rows, count_dev, 2);
  PC_LAUNCH_CHECK();
  return PC_OK;
}

}  // namespace pc
