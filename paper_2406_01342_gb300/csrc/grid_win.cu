// Gridding (type-1 spreading, the first step of the adjoint of Sect. 2.2
// evaluated as a non-uniform FFT, Sect. 5.2) on CUDA cores over plane
// windows:
//
//   grid_q[b][a] += h_k tau_k phi(a - g_u,k) phi(b - g_v,k) phi(q - x_w,k)
//
// The plan bins every visibility into the tiles its footprint touches and,
// within a tile, by the pair ps >> 1 of its first plane ps, sorted by its row
// start b0. A visibility of pair j touches only planes of the window
// [2j, 2j + 8) (W <= 7 planes from ps = 2j or 2j + 1), so it is spread once,
// with 7 of the window's 8 planes in use; fixed plane groups would cut about
// three footprints in four across two groups.
//
// One CTA per tile (a heavy tile is split into parts, each taking its share
// of every window). Lane (q, r) of warp w owns plane q of the window and tile
// row b = 4w + r for all 32 columns: 32 complex accumulators in registers.
// Per chunk of 128 slots (every nc-th slot of the window's run, so that each
// chunk samples all row starts and every warp finds work in it between two
// block barriers) the CTA evaluates each slot's kernel weights into
// shared memory (h phi_u at the W columns, phi_v padded with zeros, phi_w at
// the window's planes); each warp then takes the contiguous run of slots whose
// rows meet its four rows (read off the b0 order) and, per slot, adds
// (phi_v phi_w) (h phi_u) to the accumulators of the slot's W columns: a jump
// table over the column start selects the registers, one packed FP32x2 FMA
// per complex cell.
//
// After each window the accumulators are added into an 8-plane ring holding
// the tile in shared memory (each cell owned by one lane, no atomics); planes
// 2j and 2j + 1 are then final: they leave for the grid (plain stores when the
// CTA owns the tile, vector reductions when the tile is split) and their ring
// slots are cleared for planes 2j + 8 and 2j + 9. No waits, no atomics on
// shared memory; every cell of a tile's planes is written once per part.
#include "pc_internal.cuh"
#include "grid_win_spread.inc"

namespace pc {
namespace {

constexpr int GW_T = 32;                    // tile side (the plan's)
constexpr int GW_Q = 8;                     // planes per window
constexpr int GW_C = 128;                   // slots per chunk
constexpr int GW_THREADS = 256;
constexpr int GW_RS = GW_T + 1;             // ring row stride (float2): rows one bank pair apart
constexpr int GW_PS = GW_RS * GW_T + 4;     // ring plane stride (float2): planes four bank pairs apart
constexpr int GW_FV = 16;                   // padded phi_v entries per slot
constexpr int GW_FIRST = 48;                // b0 + 8 lies in [1, 39]

// Per-slot rows are padded by one 16-byte unit so that the vector stores of
// 32 consecutive slots fall on distinct bank groups.
struct __align__(16) GwShared {
  float2 ring[GW_Q * GW_PS];    // the tile's planes 2j .. 2j + 7 at slots (plane & 7)
  float4 hu[GW_C][5];           // h phi_u(i), i < 8, two complex values per float4 (+ pad)
  float4 fv[GW_C][5];           // phi_v(i) at float entry i + 4, zeros elsewhere (+ pad)
  float4 fw[GW_C][3];           // phi_w at the window's 8 planes, 0 off the footprint (+ pad)
  int meta[GW_C];               // (a0 + 8) | (b0 + 8) << 8, tile-local footprint starts
  int first[GW_FIRST];          // first chunk slot with b0 + 8 >= x (the chunk's count if none)
};

__device__ __forceinline__ void red_add_v4(float2* addr, float2 u, float2 v) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(u.x), "f"(u.y), "f"(v.x),
               "f"(v.y)
               : "memory");
}

__device__ __forceinline__ uint64_t pack2(float x, float y) {
  return (uint64_t)__float_as_uint(x) | ((uint64_t)__float_as_uint(y) << 32);
}
__device__ __forceinline__ float2 unpack2(uint64_t v) {
  return make_float2(__uint_as_float((uint32_t)v), __uint_as_float((uint32_t)(v >> 32)));
}

// acc[a0 + i] += t * hu[i] for the tile columns a0 + i, i < W: one packed
// FP32x2 FMA per complex cell, the column start dispatched by a jump table
// (case a0 + W - 1; the generated PTX is in grid_win_spread.inc).
template <int W>
__device__ __forceinline__ void spread(uint64_t (&acc)[GW_T], const uint64_t (&hu)[8], uint64_t t2, int cs);

#define PC_GW_SPREAD_DEF(WW)                                                                                  \
  template <>                                                                                              \
  __device__ __forceinline__ void spread<WW>(uint64_t (&acc)[GW_T], const uint64_t (&hu)[8], uint64_t t2,     \
                                             int cs) {                                                      \
    asm volatile(PC_GW_SPREAD_ASM_##WW                                                                      \
                 : "+l"(acc[0]), "+l"(acc[1]), "+l"(acc[2]), "+l"(acc[3]), "+l"(acc[4]), "+l"(acc[5]),        \
                   "+l"(acc[6]), "+l"(acc[7]), "+l"(acc[8]), "+l"(acc[9]), "+l"(acc[10]), "+l"(acc[11]),      \
                   "+l"(acc[12]), "+l"(acc[13]), "+l"(acc[14]), "+l"(acc[15]), "+l"(acc[16]), "+l"(acc[17]),  \
                   "+l"(acc[18]), "+l"(acc[19]), "+l"(acc[20]), "+l"(acc[21]), "+l"(acc[22]), "+l"(acc[23]),  \
                   "+l"(acc[24]), "+l"(acc[25]), "+l"(acc[26]), "+l"(acc[27]), "+l"(acc[28]), "+l"(acc[29]),  \
                   "+l"(acc[30]), "+l"(acc[31])                                                             \
                 : "l"(hu[0]), "l"(hu[1]), "l"(hu[2]), "l"(hu[3]), "l"(hu[4]), "l"(hu[5]), "l"(hu[6]),       \
                   "l"(t2), "r"(cs));                                                                       \
  }
PC_GW_SPREAD_DEF(4)
PC_GW_SPREAD_DEF(5)
PC_GW_SPREAD_DEF(6)
PC_GW_SPREAD_DEF(7)
#undef PC_GW_SPREAD_DEF

// Planes [qa, qb) of the ring to the grid (store, or add when the tile is
// split), ring slots cleared. One (row, 4-column group) per thread and plane.
__device__ __forceinline__ void planes_out(GwShared& S, int qa, int qb, float2* tile_base, size_t GG, int G,
                                           bool owner) {
  const int e = threadIdx.x, row = e >> 3, c4 = (e & 7) * 4;
  for (int pl = qa; pl < qb; ++pl) {
    float2* src = S.ring + (pl & (GW_Q - 1)) * GW_PS + row * GW_RS + c4;
    const float2 v0 = src[0], v1 = src[1], v2 = src[2], v3 = src[3];
    src[0] = src[1] = src[2] = src[3] = make_float2(0.f, 0.f);
    float2* dst = tile_base + (size_t)pl * GG + (size_t)row * G + c4;
    if (owner) {
      reinterpret_cast<float4*>(dst)[0] = make_float4(v0.x, v0.y, v1.x, v1.y);
      reinterpret_cast<float4*>(dst)[1] = make_float4(v2.x, v2.y, v3.x, v3.y);
    } else {
      if (v0.x != 0.f || v0.y != 0.f || v1.x != 0.f || v1.y != 0.f) red_add_v4(dst, v0, v1);
      if (v2.x != 0.f || v2.y != 0.f || v3.x != 0.f || v3.y != 0.f) red_add_v4(dst + 2, v2, v3);
    }
  }
}

template <int W>
__global__ void __launch_bounds__(GW_THREADS, 2)
k_grid_win(const int4* __restrict__ subs, const int* __restrict__ win_off, const int2* __restrict__ slot_vis,
           const float4* __restrict__ slot_geom, const float2* __restrict__ h, int G, int nT, int P, int Pw,
           float beta, float2* __restrict__ grid) {
  static_assert(W >= 2 && W <= 7, "a window of 8 planes holds the footprints of two plane starts");
  extern __shared__ __align__(16) unsigned char gw_raw[];
  GwShared& S = *reinterpret_cast<GwShared*>(gw_raw);

  const int4 sub = subs[blockIdx.x];
  const int tile = sub.x, part = sub.y, parts = sub.z;
  const int tu = tile % nT, tv = tile / nT;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int q = lane >> 2, r = lane & 3, b = 4 * warp + r;
  const float two_over_w = 2.0f / W;
  const size_t GG = (size_t)G * G;
  float2* const tile_base = grid + (size_t)(tv * GW_T) * G + tu * GW_T;
  const bool owner = parts == 1;

  for (int e = tid; e < GW_Q * GW_PS; e += GW_THREADS) S.ring[e] = make_float2(0.f, 0.f);
  uint64_t acc[GW_T];          // column accumulators, packed (Re, Im)
#pragma unroll
  for (int c = 0; c < GW_T; ++c) acc[c] = 0ull;

  for (int j = 0; j < Pw; ++j) {
    const int q0 = 2 * j;
    const int bs = __ldg(win_off + (size_t)tile * Pw + j), be = __ldg(win_off + (size_t)tile * Pw + j + 1);
    const long long len = be - bs;
    const int s0 = bs + (int)(len * part / parts), s1 = bs + (int)(len * (part + 1) / parts);
    // chunk c takes every nc-th slot from s0 + c: a sample of the whole b0
    // range (so every warp finds rows in every chunk), still in b0 order
    const int L = s1 - s0, nc = (L + GW_C - 1) / GW_C;
    for (int c = 0; c < nc; ++c) {
      const int cnt = (L - c + nc - 1) / nc;
      __syncthreads();   // the previous chunk's readers (and the ring clear) are done
      // ---- weights of one slot per thread pair: role 0 h phi_u, role 1 phi_v and phi_w
      {
        const int k = tid & (GW_C - 1), role = tid >> 7;
        if (k < cnt) {
          const int jj = s0 + c + nc * k;
          const int2 sv = slot_vis[jj];
          const float4 gm = slot_geom[jj];
          const int a0 = (sv.y & 0xff) - 64, b0 = ((sv.y >> 8) & 0xff) - 64;
          if (role == 0) {
            float2 hv = h[sv.x];
            float sn, cs;
            sincospif(2.0f * gm.w, &sn, &cs);
            hv = cmul(hv, make_float2(cs, sn));
            float f[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) f[i] = i < W ? es_kernel((i - gm.x) * two_over_w, beta) : 0.f;
#pragma unroll
            for (int m = 0; m < 4; ++m)
              S.hu[k][m] = make_float4(hv.x * f[2 * m], hv.y * f[2 * m], hv.x * f[2 * m + 1], hv.y * f[2 * m + 1]);
            S.meta[k] = (a0 + 8) | ((b0 + 8) << 8);
            // first-slot table of the chunk's b0 order (ascending within a bin)
            const int v = b0 + 8;
            const int pv = k > 0 ? ((slot_vis[jj - nc].y >> 8) & 0xff) - 64 + 8 : -1;
            for (int x = pv + 1; x <= v; ++x) S.first[x] = k;
            if (k == cnt - 1)
              for (int x = v + 1; x < GW_FIRST; ++x) S.first[x] = cnt;
          } else {
            float f[GW_FV];
#pragma unroll
            for (int i = 0; i < GW_FV; ++i)
              f[i] = (i >= 4 && i < 4 + W) ? es_kernel(((i - 4) - gm.y) * two_over_w, beta) : 0.f;
#pragma unroll
            for (int m = 0; m < 4; ++m) S.fv[k][m] = make_float4(f[4 * m], f[4 * m + 1], f[4 * m + 2], f[4 * m + 3]);
            const int d = (sv.y >> 16) - q0;             // 0 or 1
            float g[GW_Q];
#pragma unroll
            for (int qq = 0; qq < GW_Q; ++qq) {
              const int cw = qq - d;
              g[qq] = (cw >= 0 && cw < W && q0 + qq < P) ? es_kernel((cw - gm.z) * two_over_w, beta) : 0.f;
            }
            S.fw[k][0] = make_float4(g[0], g[1], g[2], g[3]);
            S.fw[k][1] = make_float4(g[4], g[5], g[6], g[7]);
          }
        }
      }
      __syncthreads();
      // ---- the slots whose rows meet this warp's rows [4w, 4w + 4)
      const int lo = S.first[4 * warp - W + 9], hi = S.first[4 * warp + 12];
#pragma unroll 1
      for (int jj = lo; jj < hi; ++jj) {
        const int m = S.meta[jj];
        const int a0 = (m & 0xff) - 8, b0 = (m >> 8) - 8;
        const float t = reinterpret_cast<const float*>(S.fv[jj])[b - b0 + 4] *
                        reinterpret_cast<const float*>(S.fw[jj])[q];
        const ulonglong2 h01 = reinterpret_cast<const ulonglong2*>(S.hu[jj])[0];
        const ulonglong2 h23 = reinterpret_cast<const ulonglong2*>(S.hu[jj])[1];
        const ulonglong2 h45 = reinterpret_cast<const ulonglong2*>(S.hu[jj])[2];
        const ulonglong2 h67 = reinterpret_cast<const ulonglong2*>(S.hu[jj])[3];
        const uint64_t hu[8] = {h01.x, h01.y, h23.x, h23.y, h45.x, h45.y, h67.x, h67.y};
        spread<W>(acc, hu, pack2(t, t), a0 + W - 1);
      }
    }
    if (s1 > s0) {
      // ---- the window's accumulators into the ring (cell (q0 + q, b, *) is this lane's)
      if (q0 + q < P) {
        float2* row = S.ring + ((q0 + q) & (GW_Q - 1)) * GW_PS + b * GW_RS;
#pragma unroll
        for (int c = 0; c < GW_T; ++c) row[c] = __fadd2_rn(row[c], unpack2(acc[c]));
      }
#pragma unroll
      for (int c = 0; c < GW_T; ++c) acc[c] = 0ull;
    }
    __syncthreads();
    // ---- planes 2j and 2j + 1 are final (later windows start at 2j + 2)
    planes_out(S, q0, min(q0 + 2, P), tile_base, GG, G, owner);
  }
  __syncthreads();
  planes_out(S, 2 * Pw, P, tile_base, GG, G, owner);
}

}  // namespace

// Mode 3, or the default (mode 0) on grids of side 2048 and more, where it
// measured faster than the tensor-core gridding (2048^2 / 2M: 0.81 against
// 1.31 ms; 4096^2 / 10M: 2.8 against 4.9 ms; at 512^2 / 200k the tensor cores
// win, 0.10 against 0.15 ms).
bool grid_win_mode(const pc_plan_s* p) {
  return p->wstack && p->W <= 7 && (p->grid_mode == 3 || (p->grid_mode == 0 && p->G >= 2048));
}

int launch_grid_win(pc_plan_s* p, const float2* h, cudaStream_t st) {
  if (p->n_wsub == 0) return PC_OK;
  if (!p->wstack || p->W > 7 || p->T != GW_T)
    return fail(PC_ERR_INVALID_ARG, "window gridding: needs w-stacking, W <= 7 and 32-cell tiles");
  const int smem = (int)sizeof(GwShared);
  const float beta = (float)p->beta;
#define PC_GW_LAUNCH(WW)                                                                                  \
  case WW: {                                                                                              \
    static bool attr = false;                                                                             \
    if (!attr) {                                                                                          \
      PC_CUDA(cudaFuncSetAttribute(k_grid_win<WW>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));  \
      attr = true;                                                                                        \
    }                                                                                                     \
    k_grid_win<WW><<<p->n_wsub, GW_THREADS, smem, st>>>(p->wsubs, p->win_off, p->slot_vis, p->slot_geom, h, \
                                                       p->G, p->nT, p->P, p->Pw, beta, p->grid);          \
    break;                                                                                                \
  }
  switch (p->W) {
    PC_GW_LAUNCH(4)
    PC_GW_LAUNCH(5)
    PC_GW_LAUNCH(6)
    PC_GW_LAUNCH(7)
    default:
      return fail(PC_ERR_INVALID_ARG, "window gridding: unsupported kernel width %d", p->W);
  }
#undef PC_GW_LAUNCH
  PC_LAUNCH_CHECK();
  return PC_OK;
}

}  // namespace pc
