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
// block barriers; the chunks of all windows form one software pipeline whose
// slot records and visibility values are loaded one and two chunks ahead,
// so no global-memory latency falls between two barriers) the CTA evaluates
// each slot's kernel weights into
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
#include "grid_win.cuh"
#include "grid_win_spread.inc"

namespace pc {
namespace {

using gwin::pack2;
using gwin::unpack2;
constexpr int GW_T = gwin::T, GW_Q = gwin::Q, GW_C = gwin::C, GW_THREADS = gwin::THREADS;
constexpr int GW_RS = gwin::RS, GW_PS = gwin::PS, GW_MAXW = gwin::MAXW;

// Per-slot rows are padded by one 16-byte unit so that the vector stores of
// 32 consecutive slots fall on distinct bank groups.
struct __align__(16) GwShared {
  float2 ring[GW_Q * GW_PS];    // the tile's planes 2j .. 2j + 7 at slots (plane & 7)
  float4 hu[GW_C][5];           // h phi_u(i), i < 8, two complex values per float4 (+ pad)
  float4 fv[GW_C][5];           // phi_v(i) at float entry i + 4, zeros elsewhere (+ pad)
  float4 fw[GW_C][3];           // phi_w at the window's 8 planes, 0 off the footprint (+ pad)
  int meta[GW_C];               // (a0 + 8) | (b0 + 8) << 8, tile-local footprint starts
  int2 wr[GW_MAXW];             // this CTA's slot range {first, count} in every window
  int4 desc[4];                 // chunk descriptors n .. n + 3 (ring)
};

__device__ __forceinline__ void red_add_v4(float2* addr, float2 u, float2 v) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(u.x), "f"(u.y), "f"(v.x),
               "f"(v.y)
               : "memory");
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
  const int k = tid & (GW_C - 1), role = tid >> 7;     // prep: slot k, role 0 h phi_u, role 1 phi_v, phi_w
  const float two_over_w = 2.0f / W;
  const size_t GG = (size_t)G * G;
  float2* const tile_base = grid + (size_t)(tv * GW_T) * G + tu * GW_T;
  const bool owner = parts == 1;

  // this part's slot range of every window, the first chunks, the ring cleared
  for (int e = tid; e < GW_Q * GW_PS; e += GW_THREADS) S.ring[e] = make_float2(0.f, 0.f);
  gwin::schedule(win_off, tile, part, parts, Pw, S.wr, S.desc);
  {
    // planes before the first window with slots stay zero
    const int j0 = S.desc[0].x;
    planes_out(S, 0, j0 < 0 ? P : 2 * j0, tile_base, GG, G, owner);
  }

  uint64_t acc[GW_T];          // column accumulators, packed (Re, Im)
#pragma unroll
  for (int c = 0; c < GW_T; ++c) acc[c] = 0ull;

  // registers of the software pipeline: slot records of chunk n (c) and n + 1
  // (n), the visibility value of chunk n + 1, the slot record of chunk n + 2
  int2 sv_c = make_int2(0, 0), sv_n = make_int2(0, 0);
  float4 gm_c = make_float4(0.f, 0.f, 0.f, 0.f);
  float2 h_c = make_float2(0.f, 0.f);
  {
    const int4 d0 = S.desc[0], d1 = S.desc[1];
    if (d0.x >= 0 && k < d0.w) {
      const int jj = d0.y + d0.z * k;
      sv_c = slot_vis[jj];
      gm_c = slot_geom[jj];
      if (role == 0) h_c = h[sv_c.x];
    }
    if (d1.x >= 0 && k < d1.w) sv_n = slot_vis[d1.y + d1.z * k];
  }

  for (int n = 0;; ++n) {
    const int4 D = S.desc[n & 3], Dn = S.desc[(n + 1) & 3], Dnn = S.desc[(n + 2) & 3];
    if (D.x < 0) break;
    // ---- prefetch: the rest of chunk n + 1 and the slot records of chunk n + 2
    float4 gm_n = make_float4(0.f, 0.f, 0.f, 0.f);
    float2 h_n = make_float2(0.f, 0.f);
    int2 sv_nn = make_int2(0, 0);
    if (Dn.x >= 0 && k < Dn.w) {
      gm_n = slot_geom[Dn.y + Dn.z * k];
      if (role == 0) h_n = h[sv_n.x];
    }
    if (Dnn.x >= 0 && k < Dnn.w) sv_nn = slot_vis[Dnn.y + Dnn.z * k];
    // ---- weights of chunk n (slot k): role 0 h phi_u and the footprint starts,
    //      role 1 phi_v; phi_w at the window's planes split between the roles
    const int q0 = 2 * D.x;
    if (k < D.w) {
      const int a0 = (sv_c.y & 0xff) - 64, b0 = ((sv_c.y >> 8) & 0xff) - 64;
      if (role == 0) {
        float sn, cs;
        sincospif(2.0f * gm_c.w, &sn, &cs);
        const float2 hv = cmul(h_c, make_float2(cs, sn));
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const float f0 = 2 * m < W ? es_kernel((2 * m - gm_c.x) * two_over_w, beta) : 0.f;
          const float f1 = 2 * m + 1 < W ? es_kernel((2 * m + 1 - gm_c.x) * two_over_w, beta) : 0.f;
          S.hu[k][m] = make_float4(hv.x * f0, hv.y * f0, hv.x * f1, hv.y * f1);
        }
        S.meta[k] = (a0 + 8) | ((b0 + 8) << 8);
      }
      {
        // phi_w at planes 4 role .. 4 role + 3 of the window (the roles share it)
        const int d = (sv_c.y >> 16) - q0;             // 0 or 1
        float g[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int qq = 4 * role + e, cw = qq - d;
          g[e] = (cw >= 0 && cw < W && q0 + qq < P) ? es_kernel((cw - gm_c.z) * two_over_w, beta) : 0.f;
        }
        S.fw[k][role] = make_float4(g[0], g[1], g[2], g[3]);
      }
      if (role == 1) {
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          float f[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int i = 4 * m + e - 4;
            f[e] = (i >= 0 && i < W) ? es_kernel((i - gm_c.y) * two_over_w, beta) : 0.f;
          }
          S.fv[k][m] = make_float4(f[0], f[1], f[2], f[3]);
        }
      }
    } else if (role == 0 && k < GW_C) {
      S.meta[k] = 0x7fff0000;                          // beyond every warp's rows
    }
    if (tid == 0) S.desc[(n + 3) & 3] = gwin::chunk_after(S.wr, Pw, Dnn);
    __syncthreads();
    // ---- this warp's run of slots: rows meeting [4w, 4w + 4), from the b0 order
    {
      const int2 run = gwin::warp_run<W>(S.meta, warp, lane);
      const int lo = run.x, hi = run.y;
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
    if (Dn.x != D.x) {
      // ---- window D.x ends: its accumulators into the ring (cell (q0 + q, b, *)
      //      is this lane's), then the planes no later window reaches leave
      if (q0 + q < P) {
        float2* row = S.ring + ((q0 + q) & (GW_Q - 1)) * GW_PS + b * GW_RS;
#pragma unroll
        for (int c = 0; c < GW_T; ++c) row[c] = __fadd2_rn(row[c], unpack2(acc[c]));
      }
#pragma unroll
      for (int c = 0; c < GW_T; ++c) acc[c] = 0ull;
      __syncthreads();
      planes_out(S, q0, Dn.x < 0 ? P : 2 * Dn.x, tile_base, GG, G, owner);
    }
    __syncthreads();   // chunk n's readers are done before chunk n + 1's weights overwrite
    sv_c = sv_n;
    gm_c = gm_n;
    h_c = h_n;
    sv_n = sv_nn;
  }
}

}  // namespace

// Mode 3, or the default (mode 0) on grids of side 2048 and more, where it
// measured faster than the tensor-core gridding (2048^2 / 2M: 0.81 against
// 1.31 ms; 4096^2 / 10M: 2.8 against 4.9 ms; at 512^2 / 200k the tensor cores
// win, 0.10 against 0.15 ms).
bool grid_win_mode(const pc_plan_s* p) {
  return p->wstack && p->W <= 7 && p->Pw <= GW_MAXW && (p->grid_mode == 3 || (p->grid_mode == 0 && p->G >= 2048));
}

int launch_grid_win(pc_plan_s* p, const float2* h, cudaStream_t st) {
  if (p->n_wsub == 0) return PC_OK;
  if (!p->wstack || p->W > 7 || p->T != GW_T || p->Pw > GW_MAXW)
    return fail(PC_ERR_INVALID_ARG, "window gridding: needs w-stacking, W <= 7, 32-cell tiles, <= %d windows",
                GW_MAXW);
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
