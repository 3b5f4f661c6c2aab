// Support contraction on the 5th-generation tensor cores (tcgen05):
//
//   G[a][c] = Re(Phi_A^H Phi_C)[a][c] = sum_k Re(Phi[k,a]) Re(Phi[k,c]) + Im(Phi[k,a]) Im(Phi[k,c])
//   b[a]    = Re(Phi_A^H V)[a]
//
// for the "new" atoms a (the MMA M dimension) against every active atom c and
// the visibility vector V (N), contracting over the visibilities (K: for each
// visibility its real and imaginary part, interleaved).
//
// Two kernels per K-chunk:
//  1. k_phase_gen evaluates every phase once -- exact fixed-point lattice turns
//     plus a double-float w-term, then sin/cos -- splits each value into
//     FP16 hi + lo and writes both into HBM in the exact K-major core-matrix
//     layout the tensor core reads (8 rows x 16 bytes per core matrix). Rows
//     are ordered as the caller gives the atoms (new atoms first), then one
//     row for V scaled by an exact power of two (so it fits FP16).
//  2. k_gram_bulk is a warp-specialised GEMM: one producer thread streams the
//     A tile (128 new atoms) and the B tile (up to 256 rows) of each 16-
//     visibility stage into one of four shared-memory buffers with
//     cp.async.bulk (completion counted in bytes on an mbarrier); four MMA
//     warps wait for a full buffer, one thread issues three tcgen05 MMAs per
//     K-step (hi*hi + hi*lo + lo*hi, FP32 accumulate in tensor memory) and
//     commits to the buffer's "empty" mbarrier, which the producer waits on
//     before refilling it. CTAs with the same K-slice run together, so a slice
//     of the phase buffer is read from HBM once and then from L2.
//
// Accumulation: the tensor core adds each MMA result into its FP32 accumulator
// with truncation (measured: 2.6e-5 relative drift after ~750 adds). Each
// sub-slice of 256 visibilities (96 MMA adds per entry; 3.1e-6 relative error of
// the whole Gram measured at M = 200k) therefore accumulates in a "fast" TMEM buffer
// that the MMA warps then add, rounded to nearest, into a "slow" TMEM buffer
// (tcgen05.ld / tcgen05.st); each 8192-visibility K-slice is added to a
// float64 accumulator in HBM.
//
// Every mbarrier wait is bounded (about 2 s of SM clock) and also watches a
// shared abort flag; on expiry the kernel sets *err, waits (bounded) for the
// copies and MMAs it issued, frees its tensor memory and returns, so the host
// reports PC_ERR_TIMEOUT instead of hanging the GPU.
#include <cuda_fp16.h>

#include "pc_internal.cuh"
#include "tcgen05.cuh"

namespace pc {
namespace {

constexpr int GB_M = 128;               // MMA M (rows of the A tile)
constexpr int GB_KV = 16;               // visibilities per stage
constexpr int GB_ROW_BYTES = 4 * GB_KV; // 16 complex fp16 per row per stage = 64 bytes
constexpr int GB_KG = GB_KV / 4;        // 16-byte K-groups per row per stage
constexpr uint32_t GB_LBO = 128;        // K-adjacent core matrices
constexpr uint32_t GB_SBO = GB_KG * 128; // 8-row groups (512 bytes)
constexpr int GB_NBUF = 4;              // stage buffers
constexpr int GB_SLICE = 8192;          // visibilities per CTA (one float64 flush)
constexpr int GB_SUB = 16;              // stages per fast-accumulator sub-slice (256 visibilities)
constexpr int GB_THREADS = 160;         // warps 0-3: MMA group; warp 4: producer
constexpr long long GB_WAIT_CYCLES = 4000000000ll;

using tc::mma_commit;
using tc::mma_f16;
using tc::smem_u32;
using tc::tmem_ld32;
using tc::tmem_st32;

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) { return tc::smem_desc(saddr, GB_LBO, GB_SBO); }
__device__ __forceinline__ uint32_t instr_desc(int M, int N) { return tc::instr_desc_f16(M, N); }
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, volatile int* abort_flag) {
  return tc::mbar_wait(mbar, parity, abort_flag, GB_WAIT_CYCLES);
}

// slow += fast (slow = fast when first) for this warp's 32 accumulator lanes
// (lane quadrant = warp, warps 0..3) and all NT columns.
__device__ void fold_fast_into_slow(uint32_t t_fast, uint32_t t_slow, int NT, bool first) {
  const int q = threadIdx.x >> 5;
  const uint32_t lane_off = (uint32_t)(32 * q) << 16;
  __syncwarp();
  for (int c0 = 0; c0 < NT; c0 += 32) {
    uint32_t f[32], s[32];
    tmem_ld32(t_fast + lane_off + (uint32_t)c0, f);
    if (!first) {
      tmem_ld32(t_slow + lane_off + (uint32_t)c0, s);
#pragma unroll
      for (int j = 0; j < 32; ++j) f[j] = __float_as_uint(__uint_as_float(f[j]) + __uint_as_float(s[j]));
    }
    tmem_st32(t_slow + lane_off + (uint32_t)c0, f);
  }
}

__device__ __forceinline__ void named_sync_mma_group() {
  asm volatile("barrier.sync 1, 128;" ::: "memory");
}

// ------------------------------------------------------------------ phase generation

// max |Re V|, |Im V| over the visibilities (as float bits, non-negative floats order as uints).
__global__ void k_vmax(const float2* __restrict__ V, int64_t M, unsigned* __restrict__ bits) {
  float m = 0.f;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < M;
       k += (int64_t)gridDim.x * blockDim.x) {
    const float2 v = V[k];
    m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
  }
  for (int off = 16; off; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0) atomicMax(bits, __float_as_uint(m));
}

// scale[0] = 2^-e, scale[1] = 2^e with 2^e > max component of V (exact powers of two).
__global__ void k_vscale(const unsigned* __restrict__ bits, float* __restrict__ scale) {
  const float m = __uint_as_float(*bits);
  int e = 0;
  if (m > 0.f && isfinite(m)) e = ilogbf(m) + 1;
  scale[0] = ldexpf(1.f, -e);
  scale[1] = ldexpf(1.f, e);
}

// One thread per (row, stage): the 16 visibilities of the stage for one atom
// (or the V row), as four 16-byte items of FP16 re/im pairs in hi and in lo.
// Item order equals memory order: [stage][row group][K-group][row in group],
// so a warp (32 consecutive rows) writes 4 x 128 contiguous bytes per K-group.
// The atom stays in registers across the stages a thread visits; every thread
// of a block visits the same stages, whose visibilities 16 threads copy into
// shared memory one stage ahead (asynchronous copies), so the phase work
// never waits on a global load.
// Threads 0..15 copy the visibilities of a stage into dst (asynchronously);
// every thread commits its (possibly empty) group of copies.
__device__ __forceinline__ void phase_prefetch(const int4* __restrict__ vis, int4* dst, int64_t k0, int64_t k_end,
                                               int stage, int n_stages) {
  if (threadIdx.x < GB_KV && stage < n_stages) {
    const int64_t k = k0 + (int64_t)stage * GB_KV + threadIdx.x;
    if (k < k_end) {
      const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst + threadIdx.x);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(vis + k) : "memory");
    }
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

__global__ void __launch_bounds__(256, 6)
k_phase_gen(const int4* __restrict__ vis, const float2* __restrict__ V, int64_t k0, int64_t k_end,
            const float4* __restrict__ atoms, int n_atoms, int v_row, int rows_pad, int n_stages,
            const float* __restrict__ vscale, uint4* __restrict__ hi, uint4* __restrict__ lo) {
  __shared__ __align__(16) int4 s_vis[2][GB_KV];
  const int row = blockIdx.x * blockDim.x + threadIdx.x;   // < rows_pad (a multiple of 256)
  const float sc = V ? vscale[0] : 0.f;
  const bool is_atom = row < n_atoms, is_v = row == v_row;
  const float4 at = is_atom ? atoms[row] : make_float4(0.f, 0.f, 0.f, 0.f);
  const size_t row_item = (size_t)(row >> 3) * (GB_KG * 8) + (row & 7);
  const size_t stage_items = (size_t)rows_pad * GB_KG;
  int b = 0;
  phase_prefetch(vis, s_vis[0], k0, k_end, blockIdx.y, n_stages);
  for (int stage = blockIdx.y; stage < n_stages; stage += gridDim.y, b ^= 1) {
    phase_prefetch(vis, s_vis[b ^ 1], k0, k_end, stage + gridDim.y, n_stages);
    asm volatile("cp.async.wait_group 1;" ::: "memory");   // this stage's copies landed
    __syncthreads();
    const int64_t kbase = k0 + (int64_t)stage * GB_KV;
    const size_t base = (size_t)stage * stage_items + row_item;
#pragma unroll
    for (int kg = 0; kg < GB_KG; ++kg) {
      uint32_t h[4], l[4];
#pragma unroll
      for (int v = 0; v < 4; v += 2) {
        float re[2], im[2];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          const int j = kg * 4 + v + s;
          const int64_t k = kbase + j;
          re[s] = 0.f;
          im[s] = 0.f;
          if (k < k_end) {
            if (is_atom) {
              float sn, cs;
              __sincosf(6.283185307179586f * phase_turns(s_vis[b][j], at), &sn, &cs);
              re[s] = cs * at.w;
              im[s] = sn * at.w;
            } else if (is_v) {
              const float2 vv = V[k];
              re[s] = vv.x * sc;
              im[s] = -vv.y * sc;
            }
          }
        }
        // pairs (re, im) of two visibilities: split each into hi + lo
        tc::split_f16x2(re[0], im[0], h[v], l[v]);
        tc::split_f16x2(re[1], im[1], h[v + 1], l[v + 1]);
      }
      const size_t item = base + (size_t)kg * 8;
      hi[item] = make_uint4(h[0], h[1], h[2], h[3]);
      lo[item] = make_uint4(l[0], l[1], l[2], l[3]);
    }
    __syncthreads();   // every read of s_vis[b] ended before the next prefetch overwrites it
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// ------------------------------------------------------------------ bulk-copy GEMM

struct GbArgs {
  const unsigned char* hi;   // phase buffer (this chunk)
  const unsigned char* lo;
  int rows_pad;
  int n_stages;              // stages in this chunk
  int nA;                    // rows of A (new atoms, the first rows)
  int nB;                    // columns: atoms + the V row
  int v_col;                 // column index of V, or -1
  const float* vscale;       // [1] = 2^e, multiplies the V column
  int NT;
  double* acc;
  int ldacc;
  int* err;
  int withhold;              // self-test: issue no MMA / commit, so the first buffer wait expires
  int slice_stages;          // stages per K-slice (blockIdx.z)
};

__global__ void __launch_bounds__(GB_THREADS, 1) k_gram_bulk(GbArgs g) {
  extern __shared__ __align__(1024) unsigned char gb_sm[];
  __shared__ __align__(8) uint64_t full_bar[GB_NBUF];
  __shared__ __align__(8) uint64_t empty_bar[GB_NBUF];
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int s_abort;
  __shared__ int s_issued, s_consumed, s_last;   // stages copied / consumed, last committed
  __shared__ int s_go[2], s_go_end;              // MMA-group decisions published by its thread 0

  const int NT = g.NT;
  // Rows and the first nA columns are the same (new) atoms: a tile whose
  // columns all lie below its first row holds only entries that symmetry
  // gives (the caller reads G[r][c] of two new atoms for c >= r only).
  if ((int)(blockIdx.x + 1) * NT <= (int)blockIdx.y * GB_M) return;
  const int a_bytes = GB_M * GB_ROW_BYTES;            // 8 KB
  const int b_bytes = NT * GB_ROW_BYTES;              // NT * 64
  const int buf_bytes = 2 * a_bytes + 2 * b_bytes;
  const uint32_t tx_bytes = (uint32_t)buf_bytes;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int a0 = blockIdx.y * GB_M, b0 = blockIdx.x * NT;
  const int s_lo = blockIdx.z * g.slice_stages;
  const int s_hi = min(g.n_stages, s_lo + g.slice_stages);
  const int nst = max(0, s_hi - s_lo);
  const uint32_t ncols = (uint32_t)(2 * NT);          // fast + slow accumulators
  const size_t stage_stride = (size_t)g.rows_pad * GB_ROW_BYTES;

  if (tid == 0) {
    for (int b = 0; b < GB_NBUF; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full_bar[b])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty_bar[b])));
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_abort = 0;
    s_issued = 0;
    s_consumed = 0;
    s_last = -1;
  }
  __syncwarp();
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const uint32_t t_fast = tmem, t_slow = tmem + (uint32_t)NT;

  if (warp == 4) {
    // ---------------- producer: one thread streams the stage tiles
    if ((tid & 31) == 0) {
      for (int i = 0; i < nst; ++i) {
        const int b = i % GB_NBUF;
        if (i >= GB_NBUF && !mbar_wait(smem_u32(&empty_bar[b]), (uint32_t)(((i / GB_NBUF) - 1) & 1), &s_abort)) {
          s_abort = 1;
          break;
        }
        if (s_abort) break;
        const size_t soff = (size_t)(s_lo + i) * stage_stride;
        unsigned char* dst = gb_sm + (size_t)b * buf_bytes;
        const uint32_t fb = smem_u32(&full_bar[b]);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(tx_bytes)
                     : "memory");
        const unsigned char* srcs[4] = {g.hi + soff + (size_t)a0 * GB_ROW_BYTES,
                                        g.lo + soff + (size_t)a0 * GB_ROW_BYTES,
                                        g.hi + soff + (size_t)b0 * GB_ROW_BYTES,
                                        g.lo + soff + (size_t)b0 * GB_ROW_BYTES};
        const uint32_t dsts[4] = {smem_u32(dst), smem_u32(dst + a_bytes), smem_u32(dst + 2 * a_bytes),
                                  smem_u32(dst + 2 * a_bytes + b_bytes)};
        const uint32_t sizes[4] = {(uint32_t)a_bytes, (uint32_t)a_bytes, (uint32_t)b_bytes,
                                   (uint32_t)b_bytes};
#pragma unroll
        for (int c = 0; c < 4; ++c)
          asm volatile(
              "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                  dsts[c]),
              "l"(srcs[c]), "r"(sizes[c]), "r"(fb)
              : "memory");
        s_issued = i + 1;
      }
    }
    __syncwarp();
  } else {
    // ---------------- MMA group (warps 0..3). Thread 0 does every wait and
    // publishes the outcome; the group reads it after a named barrier, so all
    // 128 threads take the same branch and always meet at the same barriers.
    const uint32_t idesc = instr_desc(GB_M, NT);
    bool slow_empty = true;
    bool ok = true;
    int last = -1;     // last stage whose MMAs were committed
    for (int i = 0; i < nst; ++i) {
      const int b = i % GB_NBUF;
      const bool fold = i > 0 && (i % GB_SUB) == 0 && !g.withhold;
      if (tid == 0) {
        bool good = mbar_wait(smem_u32(&full_bar[b]), (uint32_t)((i / GB_NBUF) & 1), &s_abort);
        // folding needs the MMAs of stage i-1 finished
        if (good && fold)
          good = mbar_wait(smem_u32(&empty_bar[(i - 1) % GB_NBUF]), (uint32_t)(((i - 1) / GB_NBUF) & 1),
                           &s_abort);
        if (!good) s_abort = 1;
        if (good) s_consumed = i + 1;
        s_go[i & 1] = good ? 1 : 0;   // double-buffered: read before the next barrier
      }
      named_sync_mma_group();
      if (!s_go[i & 1]) {
        ok = false;
        break;
      }
      if (fold) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        fold_fast_into_slow(t_fast, t_slow, NT, slow_empty);
        slow_empty = false;
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        named_sync_mma_group();
      }
      if (tid == 0 && !g.withhold) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t a_hi = smem_u32(gb_sm + (size_t)b * buf_bytes), a_lo = a_hi + a_bytes;
        const uint32_t b_hi = a_hi + 2 * a_bytes, b_lo = b_hi + b_bytes;
#pragma unroll
        for (int ks = 0; ks < GB_KG / 2; ++ks) {     // K = 16 fp16 elements per MMA
          const uint32_t koff = ks * 2 * GB_LBO;
          const uint32_t acc_on = ((i % GB_SUB) | ks) != 0;
          mma_f16(t_fast, smem_desc(a_hi + koff), smem_desc(b_hi + koff), idesc, acc_on);
          mma_f16(t_fast, smem_desc(a_hi + koff), smem_desc(b_lo + koff), idesc, 1u);
          mma_f16(t_fast, smem_desc(a_lo + koff), smem_desc(b_hi + koff), idesc, 1u);
        }
        mma_commit(smem_u32(&empty_bar[b]));
        s_last = i;
      }
      if (!g.withhold) last = i;
    }
    // wait for the last commit, fold the last sub-slice, add to the float64 accumulator
    if (ok && last >= 0) {
      if (tid == 0) {
        const bool good =
            mbar_wait(smem_u32(&empty_bar[last % GB_NBUF]), (uint32_t)((last / GB_NBUF) & 1), &s_abort);
        if (!good) s_abort = 1;
        s_go_end = good ? 1 : 0;
      }
      named_sync_mma_group();
      ok = s_go_end != 0;
    }
    if (ok && last >= 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      fold_fast_into_slow(t_fast, t_slow, NT, slow_empty);
      const int q = warp, lane = tid & 31;
      const int row = a0 + 32 * q + lane;
      const float vmul = g.vscale ? g.vscale[1] : 1.f;
      for (int c0 = 0; c0 < NT; c0 += 32) {
        uint32_t r[32];
        __syncwarp();
        tmem_ld32(t_slow + ((uint32_t)(32 * q) << 16) + (uint32_t)c0, r);
        if (row < g.nA) {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int col = b0 + c0 + j;
            if (col < g.nB) {
              float v = __uint_as_float(r[j]);
              if (col == g.v_col) v *= vmul;
              atomicAdd(&g.acc[(size_t)row * g.ldacc + col], (double)v);
            }
          }
        }
      }
    }
  }
  // On abort every copy and MMA already issued must finish before the CTA
  // exits: bounded waits on the "full" phases of the stages copied but not
  // consumed, and on the last MMA commit.
  __syncthreads();
  if (s_abort && tid == 0) {
    volatile int no_abort = 0;
    for (int i = s_consumed; i < s_issued; ++i)
      mbar_wait(smem_u32(&full_bar[i % GB_NBUF]), (uint32_t)((i / GB_NBUF) & 1), &no_abort);
    if (s_last >= 0)
      mbar_wait(smem_u32(&empty_bar[s_last % GB_NBUF]), (uint32_t)((s_last / GB_NBUF) & 1), &no_abort);
    atomicExch(g.err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  __syncwarp();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
}

}  // namespace

// acc[r][c] += Re(Phi_A^H [Phi_atoms | V])[r][c] for the nA first rows of the
// atom list (A) against all n_atoms atoms plus, when V is given, the V column
// (index n_atoms), except entries c < r with c < nA (tiles wholly below the
// diagonal are skipped; they mirror computed ones). acc must be cleared by the caller. err_dev (int) is set to
// 1 if a bounded wait expired. pbuf is the phase buffer (grown here).
int launch_gram_tc(const int4* vis_fx, const float2* V, int64_t M, const float4* atoms, int n_atoms,
                   int nA, double* acc, int ldacc, int* err_dev, cudaStream_t st, bool withhold,
                   DevBuf& pbuf, float* vscale_dev, unsigned* vbits_dev) {
  if (M <= 0 || nA <= 0 || n_atoms <= 0) return PC_OK;
  const int rows = n_atoms + (V ? 1 : 0);
  const int rows_pad = ceil_div(rows, 256) * 256;
  const int NT = rows > 128 ? 256 : (rows > 64 ? 128 : 64);
  // chunk of visibilities: the phase buffer (hi + lo) stays within ~2 GB
  const int64_t per_vis = (int64_t)rows_pad * 8;
  int64_t KC = (2ll << 30) / per_vis;
  KC = std::max<int64_t>(GB_SLICE, (KC / GB_SLICE) * GB_SLICE);
  const int64_t Mpad = ((M + GB_KV - 1) / GB_KV) * GB_KV;
  KC = std::min(KC, Mpad);
  const size_t half = (size_t)rows_pad * KC * 4;
  PC_TRY(pbuf.ensure(2 * half));
  uint4* hi = pbuf.as<uint4>();
  uint4* lo = reinterpret_cast<uint4*>(reinterpret_cast<unsigned char*>(pbuf.p) + half);
  const size_t smem = (size_t)GB_NBUF * (2 * GB_M * GB_ROW_BYTES + 2 * NT * GB_ROW_BYTES);
  static bool attr_set = false;
  if (!attr_set) {
    PC_CUDA(cudaFuncSetAttribute(k_gram_bulk, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr_set = true;
  }
  // timed as two classes: the phase generation (HBM-bound; the V scale with
  // the first chunk) and the contraction
  for (int64_t k0 = 0; k0 < M; k0 += KC) {
    const int64_t kc = std::min(KC, M - k0);
    const int n_stages = (int)((kc + GB_KV - 1) / GB_KV);
    {
      ProfScope ps(PROF_PHASE_GEN, st);
      ps.kernels = 1;
      if (V && k0 == 0) {
        PC_CUDA(cudaMemsetAsync(vbits_dev, 0, sizeof(unsigned), st));
        k_vmax<<<(int)std::min<int64_t>(1024, ceil_div(M, 256)), 256, 0, st>>>(V, M, vbits_dev);
        k_vscale<<<1, 1, 0, st>>>(vbits_dev, vscale_dev);
        PC_LAUNCH_CHECK();
        ps.kernels += 2;
      }
      // ~16 resident 256-thread blocks per SM; each thread walks stages with stride gridDim.y
      const int bx = rows_pad / 256;
      const int by = (int)std::min<int64_t>(n_stages, std::max<int64_t>(1, (int64_t)152 * 16 / bx));
      k_phase_gen<<<dim3(bx, by), 256, 0, st>>>(vis_fx, V, k0, k0 + kc, atoms, n_atoms, V ? n_atoms : -1,
                                                rows_pad, n_stages, vscale_dev, hi, lo);
      PC_LAUNCH_CHECK();
    }
    // K-slices: the count that makes the CTAs left after the diagonal skip fill
    // whole waves (a partial last wave idles most of the GPU for a slice's
    // time), fewest slices among the best (fewer float64 flushes)
    const int gx = ceil_div(rows, NT), gy = ceil_div(nA, GB_M);
    int tiles = 0;
    for (int y = 0; y < gy; ++y)
      for (int x = 0; x < gx; ++x) tiles += ((x + 1) * NT <= y * GB_M) ? 0 : 1;
    static int n_sm = 0;
    if (n_sm == 0) {
      int dev = 0;
      cudaGetDevice(&dev);
      if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n_sm <= 0) n_sm = 152;
    }
    const int z_max = std::max(1, n_stages / 16);          // slices of at least 256 visibilities
    int best_z = 1;
    int64_t best_cost = INT64_MAX;
    for (int z = 1; z <= z_max; ++z) {
      const int64_t waves = ceil_div((int64_t)tiles * z, n_sm);
      const int64_t cost = waves * ceil_div(n_stages, z);
      if (cost < best_cost) {
        best_cost = cost;
        best_z = z;
      }
    }
    const int slice_stages = ceil_div(n_stages, best_z);
    GbArgs a{reinterpret_cast<const unsigned char*>(hi), reinterpret_cast<const unsigned char*>(lo),
             rows_pad, n_stages, nA, rows, V ? n_atoms : -1, V ? vscale_dev : nullptr, NT, acc, ldacc,
             err_dev, withhold ? 1 : 0, slice_stages};
    dim3 grid(gx, gy, ceil_div(n_stages, slice_stages));
    ProfScope pg(PROF_GRAM_TC, st);
    pg.kernels = 1;
    k_gram_bulk<<<grid, GB_THREADS, smem, st>>>(a);
    PC_LAUNCH_CHECK();
  }
  return PC_OK;
}

}  // namespace pc
