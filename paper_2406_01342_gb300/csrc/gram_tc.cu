// Support contraction on the 5th-generation tensor cores (tcgen05):
//
//   G[a][b] = Re(Phi_A^H Phi_B)[a][b] = sum_k Re(Phi[k,a]) Re(Phi[k,b]) + Im(Phi[k,a]) Im(Phi[k,b])
//
// for a tile of 128 "new" atoms (rows, the MMA M dimension) against up to 256
// active atoms (columns, N), contracting over the visibilities (K: for each
// visibility its real and imaginary part, interleaved). The phase matrix is
// never stored: every CTA generates, stage by stage, the K-major operand
// tiles of 32 visibilities straight into shared memory (exact fixed-point
// lattice turns + double-float w-term, then sin/cos), as split FP16 pairs
// x = hi + lo, and one elected thread issues three MMAs per K-step
// (hi*hi + hi*lo + lo*hi, FP32 accumulate in tensor memory). Two stage
// buffers alternate: the tensor core works on stage s while the CTA
// generates stage s+1; an mbarrier signalled by tcgen05.commit tells the
// generators when a buffer is free again.
//
// Accumulation: the tensor core adds each MMA result into its FP32 accumulator
// with truncation, so a long accumulation drifts low (measured: 2.6e-5 relative
// after ~750 adds). The CTA therefore accumulates a sub-slice of 128
// visibilities (48 MMA adds) in a "fast" TMEM accumulator, then adds it,
// rounded to nearest on the CUDA cores, into a "slow" TMEM accumulator
// (tcgen05.ld / tcgen05.st); after its K-slice of 8192 visibilities it adds the
// slow accumulator to a float64 accumulator in HBM.
//
// Every mbarrier wait is bounded (about 2 s of SM clock); on expiry the
// kernel sets *err, drains with bounded waits, frees its tensor memory and
// returns, so the host reports PC_ERR_TIMEOUT instead of hanging the GPU.
#include <cuda_fp16.h>

#include "pc_internal.cuh"

namespace pc {
namespace {

constexpr int TC_M = 128;              // MMA M (rows = atoms of the A tile)
constexpr int TC_KV = 32;              // visibilities per stage
constexpr int TC_ROW_BYTES = 4 * TC_KV; // 64 fp16 K-elements per row per stage = 128 bytes
constexpr int TC_SLICE = 8192;         // visibilities per CTA (float64 flush per slice)
constexpr int TC_SUB = 4;              // stages per fast-accumulator sub-slice (128 visibilities)
constexpr int TC_THREADS = 768;
constexpr long long TC_WAIT_CYCLES = 4000000000ll;

// K-major, no-swizzle canonical layout: core matrices of 8 rows x 16 bytes;
// the 8 K-groups of a row-group are adjacent (LBO = 128 B), row-groups are
// 1024 B apart (SBO).
constexpr uint32_t TC_LBO = 128;
constexpr uint32_t TC_SBO = 1024;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint32_t core_off(int row, int kg) {
  return (uint32_t)((row >> 3) * TC_SBO + kg * TC_LBO + (row & 7) * 16);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((TC_LBO >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((TC_SBO >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;              // descriptor version of tcgen05; no swizzle
  return d;
}

// kind::f16 instruction descriptor: FP32 accumulator, FP16 A and B, both K-major.
__device__ __forceinline__ uint32_t instr_desc(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc,
                                        uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
      "l"(da), "l"(db), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t mbar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(done)
      : "r"(mbar), "r"(parity)
      : "memory");
  return done != 0;
}

// Bounded wait for the completion of the phase with the given parity.
__device__ bool mbar_wait_bounded(uint32_t mbar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try(mbar, parity)) {
    if (clock64() - t0 > TC_WAIT_CYCLES) return false;
  }
  return true;
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
      "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, "
      "%17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
      "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]),
      "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]),
      "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]),
      "r"(r[29]), "r"(r[30]), "r"(r[31])
      : "memory");
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// slow += fast (or slow = fast when first) for the 128-lane x NT accumulator;
// warps 0..7: lane quadrant (warp & 3), column half (warp >> 2).
__device__ void fold_fast_into_slow(uint32_t t_fast, uint32_t t_slow, int NT, bool first) {
  const int warp = threadIdx.x >> 5;
  if (warp >= 8) return;
  const int q = warp & 3, half = warp >> 2, cols = NT / 2;
  const uint32_t lane_off = (uint32_t)(32 * q) << 16;
  for (int c0 = half * cols; c0 < (half + 1) * cols; c0 += 32) {
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

struct TcArgs {
  const int4* vis;
  int64_t M;
  const float4* atomsA;
  int nA;
  const float4* atomsB;
  int nB;
  int NT;          // columns per CTA (64, 128 or 256)
  double* acc;
  int ldacc;
  int* err;
  int withhold;    // self-test: issue no MMA / commit, so the first buffer wait expires
};

__global__ void __launch_bounds__(TC_THREADS, 1) k_gram_tc(TcArgs g) {
  extern __shared__ __align__(1024) unsigned char tc_sm[];
  const int NT = g.NT;
  const int a_bytes = TC_M * TC_ROW_BYTES;
  const int b_bytes = NT * TC_ROW_BYTES;
  const int stage_bytes = 2 * a_bytes + 2 * b_bytes;
  unsigned char* stage_base = tc_sm;
  float4* sAtom = reinterpret_cast<float4*>(tc_sm + 2 * stage_bytes);   // 128 + NT atoms
  int4* sVis = reinterpret_cast<int4*>(sAtom + TC_M + NT);              // [2][TC_KV]
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sVis + 2 * TC_KV);       // [2]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + 2);
  int* s_flag = reinterpret_cast<int*>(tmem_slot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int a_base = blockIdx.y * TC_M, b_base = blockIdx.x * NT;
  const int64_t k_lo = (int64_t)blockIdx.z * TC_SLICE;
  const int64_t k_hi = min(g.M, k_lo + TC_SLICE);
  const int nrows = TC_M + NT;
  const uint32_t ncols = (uint32_t)(2 * NT);   // fast + slow accumulators, power of two

  for (int r = tid; r < nrows; r += blockDim.x) {
    float4 at = make_float4(0.f, 0.f, 0.f, 0.f);
    if (r < TC_M) {
      if (a_base + r < g.nA) at = g.atomsA[a_base + r];
    } else if (b_base + r - TC_M < g.nB) {
      at = g.atomsB[b_base + r - TC_M];
    }
    sAtom[r] = at;
  }
  if (tid < TC_KV) {
    const int64_t k = k_lo + tid;
    sVis[tid] = k < k_hi ? g.vis[k] : make_int4(0, 0, 0, 0);
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *s_flag = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const uint32_t t_fast = tmem, t_slow = tmem + (uint32_t)NT;
  const uint32_t idesc = instr_desc(TC_M, NT);
  bool slow_empty = true;

  const int nstages = (int)((k_hi - k_lo + TC_KV - 1) / TC_KV);
  int committed[2] = {0, 0};
  bool timed_out = false;

  for (int s = 0; s < nstages; ++s) {
    const int b = s & 1;
    bool bad = false;
    if (s >= 2) bad = !mbar_wait_bounded(smem_u32(&mbar[b]), (uint32_t)(((s - 2) >> 1) & 1));
    if (__syncthreads_or(bad)) {
      timed_out = true;
      break;
    }
    // prefetch the next stage's visibilities into the other staging slot
    if (tid < TC_KV) {
      const int64_t k = k_lo + (int64_t)(s + 1) * TC_KV + tid;
      sVis[((s + 1) & 1) * TC_KV + tid] = k < k_hi ? g.vis[k] : make_int4(0, 0, 0, 0);
    }
    unsigned char* sb = stage_base + b * stage_bytes;
    // items (row, K-group of 4 visibilities): a warp covers 32 consecutive rows
    // of one K-group, so its 16-byte stores fill whole 128-byte wavefronts.
    // Warp 0 issues the MMAs and generates nothing, so a blocking MMA issue
    // never delays the next stage's operands.
    for (int f = tid - 32; f < nrows * (TC_KV / 4); f += blockDim.x - 32) {
      if (f < 0) break;
      const int kg = f / nrows, rr = f - kg * nrows;
      const bool isA = rr < TC_M;
      const int row = isA ? rr : rr - TC_M;
      const float4 my_atom = sAtom[rr];
      unsigned char* hi_base = isA ? sb : sb + 2 * a_bytes;
      unsigned char* lo_base = isA ? sb + a_bytes : sb + 2 * a_bytes + b_bytes;
      const int4* vs = sVis + b * TC_KV;
      {
        __half2 h[4], l[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const int kv = kg * 4 + v;
          const bool live = k_lo + (int64_t)s * TC_KV + kv < k_hi;
          float sn = 0.f, cs = 0.f;
          if (live) __sincosf(6.283185307179586f * phase_turns(vs[kv], my_atom), &sn, &cs);
          const float re = cs * my_atom.w, im = sn * my_atom.w;
          h[v] = __floats2half2_rn(re, im);
          const float2 hf = __half22float2(h[v]);
          l[v] = __floats2half2_rn(re - hf.x, im - hf.y);
        }
        uint4 hv, lv;
        hv.x = *reinterpret_cast<uint32_t*>(&h[0]);
        hv.y = *reinterpret_cast<uint32_t*>(&h[1]);
        hv.z = *reinterpret_cast<uint32_t*>(&h[2]);
        hv.w = *reinterpret_cast<uint32_t*>(&h[3]);
        lv.x = *reinterpret_cast<uint32_t*>(&l[0]);
        lv.y = *reinterpret_cast<uint32_t*>(&l[1]);
        lv.z = *reinterpret_cast<uint32_t*>(&l[2]);
        lv.w = *reinterpret_cast<uint32_t*>(&l[3]);
        const uint32_t off = core_off(row, kg);
        *reinterpret_cast<uint4*>(hi_base + off) = hv;
        *reinterpret_cast<uint4*>(lo_base + off) = lv;
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    const bool new_sub = s > 0 && (s % TC_SUB) == 0;
    if (new_sub) {
      // fold the finished sub-slice: wait for the MMAs of stage s-1, slow += fast
      bool bad2 = !mbar_wait_bounded(smem_u32(&mbar[(s - 1) & 1]), (uint32_t)(((s - 1) >> 1) & 1));
      if (__syncthreads_or(bad2)) {
        timed_out = true;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      fold_fast_into_slow(t_fast, t_slow, NT, slow_empty);
      slow_empty = false;
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
    }
    if (tid == 0 && !g.withhold) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a_hi = smem_u32(sb), a_lo = a_hi + a_bytes;
      const uint32_t b_hi = a_hi + 2 * a_bytes, b_lo = b_hi + b_bytes;
#pragma unroll
      for (int ks = 0; ks < TC_KV / 8; ++ks) {       // K = 16 fp16 elements per MMA
        const uint32_t koff = ks * 2 * TC_LBO;
        mma_f16(t_fast, smem_desc(a_hi + koff), smem_desc(b_hi + koff), idesc,
                ((s % TC_SUB) | ks) != 0);
        mma_f16(t_fast, smem_desc(a_hi + koff), smem_desc(b_lo + koff), idesc, 1u);
        mma_f16(t_fast, smem_desc(a_lo + koff), smem_desc(b_hi + koff), idesc, 1u);
      }
      mma_commit(smem_u32(&mbar[b]));
    }
    if (!g.withhold) committed[b] += 1;
  }

  // drain: wait for the last commit on each buffer (bounded)
  bool drained = true;
  for (int b = 0; b < 2; ++b)
    if (committed[b] > 0 && !mbar_wait_bounded(smem_u32(&mbar[b]), (uint32_t)((committed[b] - 1) & 1)))
      drained = false;
  const bool ok = !timed_out && drained;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok && nstages > 0) {
    fold_fast_into_slow(t_fast, t_slow, NT, slow_empty);    // the last sub-slice
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }

  if (ok && nstages > 0 && warp < 8) {
    const int q = warp & 3, half = warp >> 2;
    const int row = a_base + 32 * q + lane;
    const int cols_per = NT / 2;
    for (int c0 = half * cols_per; c0 < (half + 1) * cols_per; c0 += 32) {
      uint32_t r[32];
      tmem_ld32(t_slow + ((uint32_t)(32 * q) << 16) + (uint32_t)c0, r);
      if (row < g.nA) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int col = b_base + c0 + j;
          if (col < g.nB) atomicAdd(&g.acc[(size_t)row * g.ldacc + col], (double)__uint_as_float(r[j]));
        }
      }
    }
  }
  if (!ok && tid == 0) atomicExch(g.err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
}

}  // namespace

// acc[a][c] += G rows of atomsA against atomsB on the tensor cores (acc must be
// cleared by the caller); err_dev (int) is set to 1 if a bounded wait expired.
int launch_gram_tc(const int4* vis_fx, int64_t M, const float4* atomsA, int nA,
                   const float4* atomsB, int nB, double* acc, int ldacc, int* err_dev,
                   cudaStream_t st, bool withhold) {
  ProfScope prof_scope_(PROF_GRAM_TC, st);
  if (M <= 0 || nA <= 0 || nB <= 0) return PC_OK;
  const int NT = nB > 128 ? 256 : (nB > 64 ? 128 : 64);
  const size_t stage_bytes = (size_t)2 * TC_M * TC_ROW_BYTES + (size_t)2 * NT * TC_ROW_BYTES;
  const size_t smem = 2 * stage_bytes + (size_t)(TC_M + NT) * sizeof(float4) +
                      2 * TC_KV * sizeof(int4) + 2 * sizeof(uint64_t) + 16;
  static bool attr_set = false;
  if (!attr_set) {
    PC_CUDA(cudaFuncSetAttribute(k_gram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
    attr_set = true;
  }
  TcArgs a{vis_fx, M, atomsA, nA, atomsB, nB, NT, acc, ldacc, err_dev, withhold ? 1 : 0};
  dim3 grid(ceil_div(nB, NT), ceil_div(nA, TC_M), ceil_div(M, TC_SLICE));
  prof_scope_.kernels = 1;
  k_gram_tc<<<grid, TC_THREADS, smem, st>>>(a);
  PC_LAUNCH_CHECK();
  return PC_OK;
}

}  // namespace pc
