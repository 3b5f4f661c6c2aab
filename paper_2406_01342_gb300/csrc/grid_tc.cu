// Gridding (type-1 spreading, the first step of the adjoint of Sect. 2.2
// evaluated as a non-uniform FFT, Sect. 5.2) on the tensor cores.
//
// For one gridding sub-problem -- a 32 x 32 tile, a group of Q <= 8 w-planes
// and its K <= 1024 binned visibilities -- the spread is a contraction over
// the visibilities:
//
//   grid_q[b][a] += sum_k  phi_w(q - x_k) phi_u(a - u_k)  *  h_k phi_v(b - v_k)
//                          `------- A[(q, a), k] -------'    `-- B[(b, re|im), k] --'
//
// so the tile (all planes) is C = A B^T with M = 8 x 32 = 256 rows (two MMA
// tiles of 128), N = 32 rows x {Re, Im} = 64 columns, K = visibilities, the
// form in which a tile is a GEMM. Per stage of 64 visibilities the CTA
//   1. evaluates the kernel weights of each visibility (W in u, W in v, one per
//      plane; one role per warp pair, so no warp diverges) and its
//      pre-twiddled, power-of-two scaled value h, then tabulates the products
//      phi_w(q) phi_u(i) and h phi_v(i) once per visibility, each already
//      split into an FP16 {hi, lo} pair,
//   2. assembles A and B from the tables (byte permutes, no arithmetic)
//      straight into the K-major core-matrix layout (8 rows x 16 bytes) the
//      tensor core reads,
//   3. one thread issues 2 x 4 x 3 tcgen05 MMAs (hi*hi + hi*lo + lo*hi,
//      FP32 accumulators in tensor memory) and commits them to an mbarrier,
//   4. all eight warps wait (bounded), read the stage's partial tile from
//      tensor memory and add it, rounded to nearest, to FP32 registers (the
//      tensor core's own accumulation truncates; one stage adds only 12
//      products per accumulator).
// The finished tile is added to the grid with vector reductions (sub-problems
// of one tile and plane group may run on several CTAs). Two CTAs fit on an
// SM, so one CTA's weight generation overlaps the other's MMAs.
//
// The only wait is bounded (about 2 s of SM clock); on expiry the CTA sets
// *err, waits (bounded) for its MMAs, frees its tensor memory and returns.
#include <cuda_fp16.h>

#include "pc_internal.cuh"
#include "tcgen05.cuh"

namespace pc {
namespace {

constexpr int GT_T = 32;                       // tile side
constexpr int GT_Q = 8;                        // planes per group (max)
constexpr int GT_KS = 64;                      // visibilities per stage
constexpr int GT_M = GT_Q * GT_T;              // A rows (plane, column)
constexpr int GT_N = 2 * GT_T;                 // B rows (row, Re | Im)
constexpr uint32_t GT_LBO = 128;               // K-adjacent core matrices
constexpr uint32_t GT_SBO = (GT_KS / 8) * 128; // 8-row groups: 1024 bytes
constexpr int GT_A_BYTES = GT_M * GT_KS * 2;   // 32 KB per half (hi or lo)
constexpr int GT_B_BYTES = GT_N * GT_KS * 2;   // 8 KB per half
constexpr int GT_SMEM = 2 * GT_A_BYTES + 2 * GT_B_BYTES;   // 80 KB
constexpr int GT_THREADS = 256;
constexpr uint32_t GT_TMEM_COLS = 128;         // two 128 x 64 accumulators
constexpr long long GT_WAIT_CYCLES = 4000000000ll;
constexpr int GT_FOLD = 4;                     // stages accumulated in TMEM per fold

__device__ __forceinline__ void red_add_v2(float2* addr, float x, float y) {
  asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(addr), "f"(x), "f"(y) : "memory");
}

template <int W>
__global__ void __launch_bounds__(GT_THREADS, 2)
k_grid_tc(const int4* __restrict__ subs, const int2* __restrict__ slot_vis,
          const float4* __restrict__ slot_geom, const float2* __restrict__ h, int G, int nT, int P,
          int Qg, float beta, float2* __restrict__ grid, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char gt_sm[];
  __shared__ float s_fu[GT_KS][8];
  __shared__ float s_fv[GT_KS][8];
  __shared__ float s_fw[GT_KS][GT_Q];
  __shared__ float2 s_h[GT_KS];
  __shared__ int s_a0[GT_KS], s_b0[GT_KS];
  __shared__ __align__(8) uint64_t s_mbar;
  __shared__ uint32_t s_tmem;
  __shared__ float s_red[GT_THREADS / 32];
  __shared__ int s_go;

  unsigned char* A_hi = gt_sm;
  unsigned char* A_lo = gt_sm + GT_A_BYTES;
  unsigned char* B_hi = gt_sm + 2 * GT_A_BYTES;
  unsigned char* B_lo = B_hi + GT_B_BYTES;

  const int4 sub = subs[blockIdx.x];
  const int tu = sub.x % nT, tv = sub.x / nT;
  const int q0 = sub.y * Qg;
  const int Q = min(Qg, P - q0);
  const int n_tiles = Q > 4 ? 2 : 1;             // MMA tiles holding planes
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const float two_over_w = 2.0f / W;

  if (tid == 0) {
    tc::mbar_init(tc::smem_u32(&s_mbar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  if (warp == 0) tc::tmem_alloc(&s_tmem, GT_TMEM_COLS);

  // Power-of-two scale for h so that every B entry lies in (-1, 1) (FP16 range).
  float hmax = 0.f;
  for (int j = sub.z + tid; j < sub.w; j += GT_THREADS) {
    const float2 v = h[slot_vis[j].x];
    hmax = fmaxf(hmax, sqrtf(v.x * v.x + v.y * v.y));
  }
  for (int off = 16; off; off >>= 1) hmax = fmaxf(hmax, __shfl_xor_sync(0xffffffffu, hmax, off));
  if (lane == 0) s_red[warp] = hmax;
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = s_tmem;
  float m = 0.f;
#pragma unroll
  for (int w = 0; w < GT_THREADS / 32; ++w) m = fmaxf(m, s_red[w]);
  const int e = (m > 0.f && isfinite(m)) ? ilogbf(m) + 1 : 0;
  const float hscale = ldexpf(1.f, -e), hunscale = ldexpf(1.f, e);

  // register accumulators: warp w reads TMEM lanes 32 (w % 4) .. of MMA tile w / 4
  const int my_tile = warp >> 2;
  float acc[GT_N];
#pragma unroll
  for (int c = 0; c < GT_N; ++c) acc[c] = 0.f;

  const uint32_t idesc = tc::instr_desc_f16(128, GT_N);
  bool ok = true;
  bool pending = false;        // thread 0: MMAs committed and not yet waited for
  int committed = 0;           // thread 0: stage of the last commit
  int stage = 0;
  if (tid == 0) s_go = 1;
  for (int c0 = sub.z; c0 < sub.w; c0 += GT_KS, ++stage) {
    const int cnt = min(GT_KS, sub.w - c0);
    // ---- 1a. per-visibility weights, one role per warp pair (no divergence):
    //      warps 0-1 phi_u, 2-3 phi_v, 4-5 phi_w per plane, 6-7 h
    {
      const int k = ((warp & 1) << 5) | lane, role = warp >> 1;
      const bool valid = k < cnt;
      int2 sv = make_int2(0, 0);
      float4 gm = make_float4(0.f, 0.f, 0.f, 0.f);
      if (valid) {
        sv = slot_vis[c0 + k];
        gm = slot_geom[c0 + k];
      }
      if (role == 0) {
#pragma unroll
        for (int c = 0; c < 8; ++c)
          s_fu[k][c] = (valid && c < W) ? es_kernel((c - gm.x) * two_over_w, beta) : 0.f;
        s_a0[k] = valid ? (sv.y & 0xff) - 64 : -64;
      } else if (role == 1) {
#pragma unroll
        for (int c = 0; c < 8; ++c)
          s_fv[k][c] = (valid && c < W) ? es_kernel((c - gm.y) * two_over_w, beta) : 0.f;
        s_b0[k] = valid ? ((sv.y >> 8) & 0xff) - 64 : -64;
      } else if (role == 2) {
        const int ps = sv.y >> 16;
#pragma unroll
        for (int q = 0; q < GT_Q; ++q) {
          const int cw = q0 + q - ps;
          s_fw[k][q] = (valid && q < Q && cw >= 0 && cw < W) ? es_kernel((cw - gm.z) * two_over_w, beta)
                                                              : 0.f;
        }
      } else {
        float2 hv = make_float2(0.f, 0.f);
        if (valid) {
          hv = h[sv.x];
          float sn, cs;
          sincospif(2.0f * gm.w, &sn, &cs);
          hv = cmul(hv, make_float2(cs, sn));
          hv.x *= hscale;
          hv.y *= hscale;
        }
        s_h[k] = hv;
      }
    }
    __syncthreads();
    // the previous stage's MMAs still read A and B: wait for them (bounded)
    // before overwriting; their latency hid behind step 1
    if (tid == 0 && pending) {
      s_go = tc::mbar_wait(tc::smem_u32(&s_mbar), (uint32_t)(committed & 1), nullptr, GT_WAIT_CYCLES) ? 1 : 0;
      pending = !s_go;
    }
    __syncthreads();
    if (!s_go) {
      ok = false;
      break;
    }
    // ---- 2a. clear the operand rows in use (16-byte stores)
    {
      const int a_words = n_tiles * 128 * GT_KS * 2 / 16;   // per half
      uint4* ah = reinterpret_cast<uint4*>(A_hi);
      uint4* al = reinterpret_cast<uint4*>(A_lo);
      uint4* bh = reinterpret_cast<uint4*>(B_hi);
      const uint4 z = make_uint4(0u, 0u, 0u, 0u);
      for (int e = tid; e < a_words; e += GT_THREADS) {
        ah[e] = z;
        al[e] = z;
      }
      for (int e = tid; e < 2 * GT_B_BYTES / 16; e += GT_THREADS) bh[e] = z;   // B_hi and B_lo
    }
    __syncthreads();
    // ---- 2b. scatter the nonzero entries, each an FP16 {hi, lo} split of its
    //      FP32 value, into the K-major core-matrix layout: A[(q, a0 + i), k] =
    //      phi_w(q) phi_u(i) and B[(b0 + i, Re|Im), k] = (Re|Im h) phi_v(i); only
    //      the W x Q and 2 W entries a visibility touches are written
    {
      const int k = tid & (GT_KS - 1), part = tid >> 6;   // 4 threads per visibility
      const int a0 = s_a0[k], b0 = s_b0[k];
      const uint32_t koff = (uint32_t)(k >> 3) * 128 + (uint32_t)(k & 7) * 2;
#pragma unroll
      for (int qq = 0; qq < 2; ++qq) {
        const int q = part + 4 * qq;
        if (q >= Q) continue;
        const float fw = s_fw[k][q];
        if (fw == 0.f) continue;
#pragma unroll
        for (int i = 0; i < W; ++i) {
          const int a = a0 + i;
          if (a < 0 || a >= GT_T) continue;
          const float v = fw * s_fu[k][i];
          const __half hh = __float2half_rn(v);
          const __half hl = __float2half_rn(v - __half2float(hh));
          const int R = q * GT_T + a;
          const uint32_t off = (uint32_t)(R >> 3) * GT_SBO + (uint32_t)(R & 7) * 16 + koff;
          *reinterpret_cast<__half*>(A_hi + off) = hh;
          *reinterpret_cast<__half*>(A_lo + off) = hl;
        }
      }
      const float2 hv = s_h[k];
      for (int j = part; j < 2 * W; j += 4) {
        const int i = j >> 1, c = j & 1;
        const int b = b0 + i;
        if (b < 0 || b >= GT_T) continue;
        const float v = (c ? hv.y : hv.x) * s_fv[k][i];
        const __half hh = __float2half_rn(v);
        const __half hl = __float2half_rn(v - __half2float(hh));
        const int n = 2 * b + c;
        const uint32_t off = (uint32_t)(n >> 3) * GT_SBO + (uint32_t)(n & 7) * 16 + koff;
        *reinterpret_cast<__half*>(B_hi + off) = hh;
        *reinterpret_cast<__half*>(B_lo + off) = hl;
      }
    }
    tc::fence_proxy_async_smem();
    __syncthreads();
    // ---- 3. MMAs (one thread) and commit; the accumulators restart after each fold
    const bool fold_now = (stage % GT_FOLD) == GT_FOLD - 1 || c0 + GT_KS >= sub.w;
    if (tid == 0) {
      tc::fence_after_sync();
      const uint32_t ah = tc::smem_u32(A_hi), al = tc::smem_u32(A_lo);
      const uint32_t bh = tc::smem_u32(B_hi), bl = tc::smem_u32(B_lo);
      for (int t = 0; t < n_tiles; ++t) {
        const uint32_t d = tmem + (uint32_t)(t * GT_N);
        const uint32_t toff = (uint32_t)t * 16 * GT_SBO;     // 128 rows = 16 row groups
#pragma unroll
        for (int ks = 0; ks < GT_KS / 16; ++ks) {
          const uint32_t koff = (uint32_t)ks * 2 * GT_LBO;
          tc::mma_f16(d, tc::smem_desc(ah + toff + koff, GT_LBO, GT_SBO),
                      tc::smem_desc(bh + koff, GT_LBO, GT_SBO), idesc,
                      (ks > 0 || stage % GT_FOLD != 0) ? 1u : 0u);
          tc::mma_f16(d, tc::smem_desc(ah + toff + koff, GT_LBO, GT_SBO),
                      tc::smem_desc(bl + koff, GT_LBO, GT_SBO), idesc, 1u);
          tc::mma_f16(d, tc::smem_desc(al + toff + koff, GT_LBO, GT_SBO),
                      tc::smem_desc(bh + koff, GT_LBO, GT_SBO), idesc, 1u);
        }
      }
      tc::mma_commit(tc::smem_u32(&s_mbar));
      pending = true;
      committed = stage;
      if (fold_now) {
        s_go = tc::mbar_wait(tc::smem_u32(&s_mbar), (uint32_t)(stage & 1), nullptr, GT_WAIT_CYCLES) ? 1 : 0;
        pending = !s_go;
      }
    }
    if (!fold_now) continue;
    __syncthreads();
    if (!s_go) {
      ok = false;
      break;
    }
    // ---- 4. fold the partial tile of the last GT_FOLD stages into the registers
    tc::fence_after_sync();
    if (my_tile < n_tiles) {
      __syncwarp();
      const uint32_t base = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(my_tile * GT_N);
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        uint32_t r[32];
        tc::tmem_ld32(base + (uint32_t)(32 * half), r);
#pragma unroll
        for (int j = 0; j < 32; ++j) acc[32 * half + j] += __uint_as_float(r[j]);
      }
    }
    tc::fence_before_sync();
    __syncthreads();
  }

  if (!ok) {
    // MMAs may still be running: wait for them (bounded) before freeing tensor
    // memory; report the expiry
    if (tid == 0) {
      if (pending)
        tc::mbar_wait(tc::smem_u32(&s_mbar), (uint32_t)(committed & 1), nullptr, GT_WAIT_CYCLES);
      atomicExch(err, 1);
    }
  } else {
    // ---- add the tile to the grid: row (q, a) of this thread, columns (b, Re|Im)
    const int q = my_tile * 4 + (warp & 3), a = lane;
    if (my_tile < n_tiles && q < Q) {
      const size_t GG = (size_t)G * G;
      float2* dst = grid + (size_t)(q0 + q) * GG + (size_t)(tv * GT_T) * G + (tu * GT_T + a);
#pragma unroll
      for (int b = 0; b < GT_T; ++b) {
        const float x = acc[2 * b] * hunscale, y = acc[2 * b + 1] * hunscale;
        if (x != 0.f || y != 0.f) red_add_v2(dst + (size_t)b * G, x, y);
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    __syncwarp();
    tc::tmem_dealloc(tmem, GT_TMEM_COLS);
  }
}

}  // namespace

// Tensor-core gridding of h onto the plan's grid (rows already cleared).
int launch_grid_tc(pc_plan_s* p, const float2* h, int* err_dev, cudaStream_t st) {
  static bool attr_set[9] = {};
  const float beta = (float)p->beta;
#define PC_GRID_TC_CASE(WW)                                                                          \
  case WW:                                                                                           \
    if (!attr_set[WW]) {                                                                             \
      PC_CUDA(cudaFuncSetAttribute(k_grid_tc<WW>, cudaFuncAttributeMaxDynamicSharedMemorySize,     \
                                   GT_SMEM));                                                        \
      PC_CUDA(cudaFuncSetAttribute(k_grid_tc<WW>, cudaFuncAttributePreferredSharedMemoryCarveout,  \
                                   100));                                                            \
      attr_set[WW] = true;                                                                           \
    }                                                                                                \
    k_grid_tc<WW><<<p->n_sub, GT_THREADS, GT_SMEM, st>>>(p->subs, p->slot_vis, p->slot_geom, h,     \
                                                         p->G, p->nT, p->P, p->Qg, beta, p->grid,   \
                                                         err_dev);                                   \
    break;
  switch (p->W) {
    PC_GRID_TC_CASE(4)
    PC_GRID_TC_CASE(5)
    PC_GRID_TC_CASE(6)
    PC_GRID_TC_CASE(7)
    PC_GRID_TC_CASE(8)
    default:
      return fail(PC_ERR_INVALID_ARG, "gridding: unsupported kernel width %d", p->W);
  }
#undef PC_GRID_TC_CASE
  PC_LAUNCH_CHECK();
  return PC_OK;
}

}  // namespace pc
