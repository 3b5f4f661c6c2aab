// FFT passes of the certificate (adjoint) and of the degridding forward
// operator for grids of side G = 2048, 4096 and 8192, one CTA per row
// (fft_cta.cuh), with the pass-1 output kept only at the grid rows b that a
// visibility can reach.
//
// Compact pass-1 storage. The c-th reachable row (c < n_rows, ascending b)
// of plane q holds N image-domain values i, stored in blocks of four rows:
//
//   Xc[((q * nb + c / 4) * N + i) * 4 + c % 4],   nb = ceil(n_rows / 4).
//
// A CTA that owns one row c writes every fourth 8-byte word (the three
// sibling rows, owned by the CTAs launched next to it, fill the rest of
// each 32-byte sector in L2); a CTA that owns one image row i reads its
// n_rows values as whole 32-byte sectors. At 4096^2 with 23 w-planes this is
// ~1.4k of 8192 rows: the pass-2 input shrinks six-fold against full rows.
//
// Certificate (the adjoint of Sect. 2.2 via the NUFFT of Sect. 5.2):
//   k_fft_rows_big   per (reachable row b, plane q): inverse FFT along a of
//                    grid_q[b][.] (only the 32-column groups that can hold
//                    data are read), the N kept outputs -> Xc;
//   k_fft_cols_big   per image row i: for every plane an inverse FFT along b
//                    of the compact row, the plane phase e^{+2 pi i q t_ij},
//                    summed in registers; then the per-pixel correction, mu
//                    and its maxima (as k_fft_cols).
// Degridding (the exact adjoint of the above, in reverse order, with the
// forward FFTs as conj(IFFT(conj(.))), as degrid.cu):
//   k_degrid_cols_big  per image row i: for every plane c_ij e^{+2 pi i q t_ij}
//                      x_ij centred on a length-G row, inverse FFT along j,
//                      conjugated outputs at the reachable rows b -> Xc;
//   k_degrid_rows_big  per (reachable row, plane): the N values of Xc centred
//                      on a length-G row, inverse FFT along i, conjugated ->
//                      grid_q[b][.] in the column groups that hold data.
#include <cudaTypedefs.h>

#include "fft_cta.cuh"
#include "tcgen05.cuh"

namespace pc {
namespace {

constexpr long long FB_WAIT_CYCLES = 4000000000ll;   // bounded TMA waits (~2 s of SM clock)

// Shared-memory layout of k_fft_cols_big: the FFT exchange buffer Z, then two
// stage buffers for the compact rows of consecutive planes (TMA boxes of
// `by` rows of four complex values), each 128-byte aligned.
template <int R>
__host__ __device__ constexpr size_t cols_z_bytes() {
  return ((sizeof(float2) * cfft::Cfg<R>::Z_ELEMS + 127) / 128) * 128;
}
__host__ __device__ inline size_t cols_stage_bytes(int n_box, int by) { return (size_t)n_box * by * 32; }

__device__ __forceinline__ bool group_on(const uint32_t* __restrict__ colw, int n) {
  const int g = n >> 5;
  return (__ldg(colw + (g >> 5)) >> (g & 31)) & 1u;
}

__device__ __forceinline__ float2 conj2(float2 v) { return make_float2(v.x, -v.y); }

// e^{+2 pi i q t} for t = t_hi + t_lo, q t reduced exactly to [-1/2, 1/2]
// before the fast sine and cosine (accurate to ~4e-7 absolute there).
__device__ __forceinline__ float2 plane_phase(float qf, float2 t) {
  const float p = qf * t.x;
  const float e = fmaf(qf, t.x, -p) + qf * t.y;
  const float th = (p - rintf(p)) + e;
  float sn, cs;
  __sincosf(6.283185307179586f * th, &sn, &cs);
  return make_float2(cs, sn);
}

template <int R>
__global__ void __launch_bounds__(32 * R, 2)
k_fft_rows_big(const float2* __restrict__ grid, float2* __restrict__ Xc, int N, int nb,
               const int* __restrict__ active_rows, const uint32_t* __restrict__ colw,
               const float2* __restrict__ tw, const float2* __restrict__ T2) {
  constexpr int G = cfft::Cfg<R>::G;
  extern __shared__ float2 Z[];
  const int c = blockIdx.x, q = blockIdx.y;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const float2* src = grid + ((size_t)q * G + active_rows[c]) * G;
  float2 u[cfft::L];
#pragma unroll
  for (int e = 0; e < cfft::L; ++e) {
    const int n = cfft::pos<R>(t, e);
    u[e] = group_on(colw, n) ? src[n] : make_float2(0.f, 0.f);
  }
  cfft::fft<R>(u, Z, tw, T2);
  __syncthreads();                                  // every warp is done with its row of Z
  // the kept outputs, staged by frequency: folded into [0, G / 2) and
  // swizzled (cfft::stage_pos) so the stores are free of bank conflicts
  const int hN = N >> 1;
  const int k0 = cfft::kept_freq<R>(warp, lane, 0);
  const int msk = cfft::stage_mask<R, 7>(k0 < G / 2 ? k0 : k0 - G / 2);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int kf = cfft::kept_freq<R>(warp, lane, k);
    const int i = (kf + hN) & (G - 1);
    if (i < N) Z[(kf < G / 2 ? kf : kf - G / 2) ^ msk] = wfft::kept_value<cfft::L>(u, k, lane);
  }
  __syncthreads();
  float2* dst = Xc + (size_t)(q * nb + (c >> 2)) * N * 4 + (c & 3);
  for (int i = t; i < N; i += 32 * R) {
    const int kf = (i - hN) & (G - 1);
    dst[(size_t)i * 4] = Z[cfft::stage_pos<R, 7>(kf < G / 2 ? kf : kf - G / 2)];
  }
}

// The compact rows of plane q for image row i are Xc[q][cb][i][0..4), cb <
// nb: a 2-D TMA box of {4 complex values, by blocks} from the tensor map over
// Xc viewed as [P nb blocks][N x 4 complex] gathers them into shared memory
// in compact-row order (the transpose of the pass-1 layout). Thread 0 issues
// the boxes of plane q + 1 while every thread transforms plane q (two stage
// buffers, each completing on its own mbarrier), so the loads hide behind the
// FFTs. Every wait is bounded: on expiry the CTA sets *err, waits (bounded)
// for the copies it issued and leaves.
template <int R>
__global__ void __launch_bounds__(32 * R, R == 16 ? 1 : 2)
k_fft_cols_big(const __grid_constant__ CUtensorMap xmap, int n_box, int by, const float4* __restrict__ pix,
               float* __restrict__ mu, int N, int P, int nb, int wstack, const int* __restrict__ row_pos,
               const float2* __restrict__ tw, const float2* __restrict__ T2, float scale,
               unsigned* __restrict__ maxbits, int* __restrict__ err, const int* __restrict__ img_rows) {
  constexpr int G = cfft::Cfg<R>::G;
  extern __shared__ __align__(128) unsigned char fb_sm[];
  __shared__ __align__(8) uint64_t s_bar[2];
  float2* Z = reinterpret_cast<float2*>(fb_sm);
  float2* stage[2] = {reinterpret_cast<float2*>(fb_sm + cols_z_bytes<R>()),
                      reinterpret_cast<float2*>(fb_sm + cols_z_bytes<R>() + cols_stage_bytes(n_box, by))};
  const int i = img_rows ? img_rows[blockIdx.x] : (int)blockIdx.x;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int hN = N >> 1;
  const uint32_t tx_bytes = (uint32_t)cols_stage_bytes(n_box, by);
  if (t == 0) {
    tc::mbar_init(tc::smem_u32(&s_bar[0]), 1);
    tc::mbar_init(tc::smem_u32(&s_bar[1]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // thread 0: the boxes of plane q into stage buffer q & 1
  auto issue = [&](int q) {
    const int b = q & 1;
    const uint32_t bar = tc::smem_u32(&s_bar[b]);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // earlier reads of the buffer first
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(tx_bytes) : "memory");
    for (int j = 0; j < n_box; ++j) {
      const uint32_t dst = tc::smem_u32(stage[b] + (size_t)j * by * 4);
      const int x = 8 * i, y = q * nb + j * by;
      asm volatile(
          "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
          ::"r"(dst), "l"(reinterpret_cast<uint64_t>(&xmap)), "r"(x), "r"(y), "r"(bar)
          : "memory");
    }
  };
  if (t == 0) issue(0);
  // compact row of each input register (-1: a row no visibility reaches)
  int cpos[cfft::L];
#pragma unroll
  for (int e = 0; e < cfft::L; ++e) cpos[e] = __ldg(row_pos + cfft::pos<R>(t, e));
  // w-screen turns of the kept outputs' pixels
  float2 tz[8];
  float2 acc[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int j = (cfft::kept_freq<R>(warp, lane, k) + hN) & (G - 1);
    tz[k] = make_float2(0.f, 0.f);
    if (wstack && j < N) {
      const float4 pt = pix[(size_t)i * N + j];
      tz[k] = make_float2(pt.z, pt.w);
    }
    acc[k] = make_float2(0.f, 0.f);
  }
  int issued = 1, consumed = 0;
  bool ok = true;
  for (int q = 0; q < P; ++q) {
    if (t == 0 && q + 1 < P) {
      issue(q + 1);
      issued = q + 2;
    }
    const int b = q & 1;
    const bool got = tc::mbar_wait(tc::smem_u32(&s_bar[b]), (uint32_t)((q >> 1) & 1), nullptr, FB_WAIT_CYCLES);
    if (__syncthreads_or(!got)) {
      ok = false;
      break;
    }
    consumed = q + 1;
    const float2* src = stage[b];
    float2 u[cfft::L];
#pragma unroll
    for (int e = 0; e < cfft::L; ++e) {
      const int cc = cpos[e];
      u[e] = cc >= 0 ? src[cc] : make_float2(0.f, 0.f);
    }
    cfft::fft<R>(u, Z, tw, T2);
    const float qf = (float)q;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      float2 v = wfft::kept_value<cfft::L>(u, k, lane);
      if (wstack) v = cmul(v, plane_phase(qf, tz[k]));
      acc[k].x += v.x;
      acc[k].y += v.y;
    }
    __syncthreads();                                // Z and the stage buffer are free again
  }
  if (!ok) {
    // a wait expired: report it, let the copies this CTA issued land (bounded), leave
    if (t == 0) {
      atomicExch(err, 1);
      for (int q = consumed; q < issued; ++q)
        tc::mbar_wait(tc::smem_u32(&s_bar[q & 1]), (uint32_t)((q >> 1) & 1), nullptr, FB_WAIT_CYCLES);
    }
    __syncthreads();
    return;
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int j = (cfft::kept_freq<R>(warp, lane, k) + hN) & (G - 1);
    if (j < N) Z[j] = acc[k];
  }
  __syncthreads();
  float amax = 0.0f;
  unsigned skey = 0;   // order-preserving key of the signed maximum (0 below every number)
  for (int j = t; j < N; j += 32 * R) {
    const float4 pt = pix[(size_t)i * N + j];
    const float2 s = Z[j];
    const float m = (pt.x * s.x - pt.y * s.y) * scale;
    mu[(size_t)i * N + j] = m;
    amax = fmaxf(amax, fabsf(m));
    if (m != m) amax = __int_as_float(0x7fc00000);
    skey = max(skey, float_order_key(m));
  }
  unsigned bits = __float_as_uint(amax);
  for (int off = 16; off; off >>= 1) {
    bits = max(bits, __shfl_xor_sync(0xffffffffu, bits, off));
    skey = max(skey, __shfl_xor_sync(0xffffffffu, skey, off));
  }
  if (lane == 0 && maxbits) {
    atomicMax(maxbits, bits);
    atomicMax(maxbits + 1, skey);
  }
}

template <int R>
__global__ void __launch_bounds__(32 * R, R == 16 ? 1 : 2)
k_degrid_cols_big(const float* __restrict__ x, const float4* __restrict__ pix, int N, int P, int nb, int n_rows,
                  int wstack, const int* __restrict__ row_pos, const int* __restrict__ active_rows,
                  const float2* __restrict__ tw, const float2* __restrict__ T2, float2* __restrict__ Xc,
                  const int* __restrict__ img_rows) {
  constexpr int G = cfft::Cfg<R>::G;
  extern __shared__ float2 Z[];
  const int i = img_rows ? img_rows[blockIdx.x] : (int)blockIdx.x;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int hN = N >> 1;
  // input register e sits at row position n, pixel j = (n + N/2) mod G (< N
  // only for n < N/2 or n >= G - N/2): its c_ij x_ij and w-screen turns
  float2 base[cfft::L], tz[cfft::L];
#pragma unroll
  for (int e = 0; e < cfft::L; ++e) {
    const int j = (cfft::pos<R>(t, e) + hN) & (G - 1);
    base[e] = make_float2(0.f, 0.f);
    tz[e] = make_float2(0.f, 0.f);
    if (cfft::centred_reg<R>(e) && j < N) {
      const size_t p = (size_t)i * N + j;
      const float4 pt = pix[p];
      const float xv = x[p];
      base[e] = make_float2(pt.x * xv, pt.y * xv);
      tz[e] = make_float2(pt.z, pt.w);
    }
  }
  // which output registers are reachable rows (bit kp), and the lane's
  // staging mask (cfft::stage_mask: conflict-free stores by frequency)
  unsigned reach = 0;
#pragma unroll
  for (int kp = 0; kp < cfft::L; ++kp) reach |= (__ldg(row_pos + cfft::freq<R>(warp, lane, kp)) >= 0 ? 1u : 0u) << kp;
  const int msk = cfft::stage_mask<R, 8>(cfft::freq<R>(warp, lane, 0));
  for (int q = 0; q < P; ++q) {
    const float qf = (float)q;
    float2 u[cfft::L];
#pragma unroll
    for (int e = 0; e < cfft::L; ++e)
      u[e] = !cfft::centred_reg<R>(e) ? make_float2(0.f, 0.f)
             : wstack                 ? cmul(base[e], plane_phase(qf, tz[e]))
                                      : base[e];
    cfft::fft<R>(u, Z, tw, T2);
    __syncthreads();                                // Z free: stage the reachable rows' values
#pragma unroll
    for (int kp = 0; kp < cfft::L; ++kp)
      if ((reach >> kp) & 1u) Z[cfft::freq<R>(warp, lane, kp) ^ msk] = conj2(u[wfft::brev(kp, 4)]);
    __syncthreads();
    float2* dst = Xc + (size_t)q * nb * N * 4 + (size_t)i * 4;
    for (int c = t; c < n_rows; c += 32 * R)
      dst[(size_t)(c >> 2) * N * 4 + (c & 3)] = Z[cfft::stage_pos<R, 8>(__ldg(active_rows + c))];
    __syncthreads();
  }
}

template <int R>
__global__ void __launch_bounds__(32 * R, 2)
k_degrid_rows_big(const float2* __restrict__ Xc, int N, int nb, const int* __restrict__ active_rows,
                  const uint32_t* __restrict__ colw, const float2* __restrict__ tw, const float2* __restrict__ T2,
                  float2* __restrict__ grid, const uint32_t* __restrict__ img_row_bits) {
  constexpr int G = cfft::Cfg<R>::G;
  extern __shared__ float2 Z[];
  const int c = blockIdx.x, q = blockIdx.y;
  const int t = threadIdx.x;
  const int hN = N >> 1;
  const float2* src = Xc + (size_t)(q * nb + (c >> 2)) * N * 4 + (c & 3);
  float2 u[cfft::L];
#pragma unroll
  for (int e = 0; e < cfft::L; ++e) {
    const int i = (cfft::pos<R>(t, e) + hN) & (G - 1);
    // image rows outside the restriction hold zeros (their pass-1 values were not written)
    const bool on = cfft::centred_reg<R>(e) && i < N &&
                    (!img_row_bits || ((__ldg(img_row_bits + (i >> 5)) >> (i & 31)) & 1u));
    u[e] = on ? conj2(src[(size_t)i * 4]) : make_float2(0.f, 0.f);
  }
  cfft::fft<R>(u, Z, tw, T2);
  __syncthreads();
  const int warp = t >> 5, lane = t & 31;
  // staged by frequency, swizzled inside each group of R (cfft::stage_pos:
  // conflict-free stores); a pair 2h, 2h + 1 stays in one 16-byte slot,
  // swapped when the swizzle flips bit 0
  const int msk = cfft::stage_mask<R, 8>(cfft::freq<R>(warp, lane, 0));
#pragma unroll
  for (int kp = 0; kp < cfft::L; ++kp) Z[cfft::freq<R>(warp, lane, kp) ^ msk] = conj2(u[wfft::brev(kp, 4)]);
  __syncthreads();
  float4* dst = reinterpret_cast<float4*>(grid + ((size_t)q * G + active_rows[c]) * G);
  const float4* s4 = reinterpret_cast<const float4*>(Z);
  for (int h = t; h < G / 2; h += 32 * R)
    if (group_on(colw, 2 * h)) {
      const int sp = cfft::stage_pos<R, 8>(2 * h);
      const float4 v = s4[sp >> 1];
      dst[h] = (sp & 1) ? make_float4(v.z, v.w, v.x, v.y) : v;
    }
}

template <typename K>
int allow(K* kernel, size_t smem) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess
             ? PC_OK
             : fail(PC_ERR_CUDA, "fft: shared-memory opt-in failed");
}

}  // namespace

bool fft_big_size(int G) { return G == 2048 || G == 4096 || G == 8192; }

bool fft_rows_big(const pc_plan_s* p) { return fft_big_size(p->G) && (p->fft_warp < 0 || (p->fft_warp & 1)); }

bool fft_cols_big(const pc_plan_s* p) { return fft_big_size(p->G) && (p->fft_warp < 0 || (p->fft_warp & 2)); }

int compact_blocks(const pc_plan_s* p) { return ceil_div(std::max(p->n_active_rows, 1), 4); }

#define PC_BIG_DISPATCH(G, CALL)   \
  switch (G) {                     \
    case 2048: { CALL(4) } break;  \
    case 4096: { CALL(8) } break;  \
    default: { CALL(16) } break;   \
  }

int launch_fft_rows_big(pc_plan_s* p, cudaStream_t st) {
  const int nb = compact_blocks(p);
  PC_TRY(p->xc.ensure(sizeof(float2) * (size_t)p->P * nb * p->N * 4));
  float2* Xc = p->xc.as<float2>();
#define PC_ROWS(RR)                                                                                        \
  const size_t smem = sizeof(float2) * cfft::Cfg<RR>::Z_ELEMS;                                             \
  static bool done = false;                                                                                \
  if (!done) {                                                                                             \
    PC_TRY(allow(k_fft_rows_big<RR>, smem));                                                               \
    done = true;                                                                                           \
  }                                                                                                        \
  k_fft_rows_big<RR><<<dim3(p->n_active_rows, p->P), 32 * RR, smem, st>>>(p->grid, Xc, p->N, nb,           \
                                                                           p->active_rows, p->col_bits,    \
                                                                           p->tw_big, p->tw_in);
  PC_BIG_DISPATCH(p->G, PC_ROWS)
#undef PC_ROWS
  PC_LAUNCH_CHECK();
  return PC_OK;
}

// The tensor map over the compact pass-1 rows (made once, at plan time): a
// 2-D float32 tensor of P nb rows of 8 N floats (the N x 4 complex values of
// one block of four reachable rows), boxes of 8 floats x by rows.
int make_xc_tensor_map(pc_plan_s* p) {
  const int nb = compact_blocks(p);
  // box height a multiple of 4 rows (every box lands 128-byte aligned in
  // shared memory); a last box that runs past the plane reads rows of the next
  // plane, or zeros past the tensor, which the kernel ignores
  p->xmap_by = std::min(256, ((nb + 3) / 4) * 4);
  p->xmap_boxes = ceil_div(nb, p->xmap_by);
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
      cudaGetLastError();
      return fail(PC_ERR_CUDA, "plan: cuTensorMapEncodeTiled is not available");
    }
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const cuuint64_t dims[2] = {(cuuint64_t)8 * p->N, (cuuint64_t)p->P * nb};
  const cuuint64_t strides[1] = {(cuuint64_t)8 * p->N * sizeof(float)};
  const cuuint32_t box[2] = {8, (cuuint32_t)p->xmap_by};
  const cuuint32_t elem[2] = {1, 1};
  const CUresult r = encode(&p->xmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, p->xc.p, dims, strides, box, elem,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(PC_ERR_CUDA, "plan: tensor map of the compact FFT rows failed (%d)", (int)r);
  return PC_OK;
}

int launch_fft_cols_big(pc_plan_s* p, float* mu, float scale, unsigned* maxbits, cudaStream_t st) {
  const int nb = compact_blocks(p);
  const int ws = p->wstack ? 1 : 0;
  const size_t stage = cols_stage_bytes(p->xmap_boxes, p->xmap_by);
  const bool restricted = p->n_img_rows > 0;
  const int rows_img = restricted ? p->n_img_rows : p->N;
  const int* list = restricted ? p->img_rows : nullptr;
#define PC_COLS(RR)                                                                                        \
  const size_t smem = cols_z_bytes<RR>() + 2 * stage;                                                      \
  if (smem > 200 * 1024) return fail(PC_ERR_INVALID_ARG, "fft: %d reachable grid rows exceed shared memory", \
                                     p->n_active_rows);                                                    \
  static bool done = false;                                                                                \
  if (!done) {                                                                                             \
    PC_TRY(allow(k_fft_cols_big<RR>, 200 * 1024));                                                         \
    done = true;                                                                                           \
  }                                                                                                        \
  k_fft_cols_big<RR><<<rows_img, 32 * RR, smem, st>>>(p->xmap, p->xmap_boxes, p->xmap_by, p->pix_tab, mu,     \
                                                     p->N, p->P, nb, ws, p->row_pos, p->tw_big, p->tw_in,   \
                                                     scale, maxbits, p->iscal + 7, list);
  PC_BIG_DISPATCH(p->G, PC_COLS)
#undef PC_COLS
  PC_LAUNCH_CHECK();
  return PC_OK;
}

// The degridding's two FFT passes: img (N x N) -> grid_q[b][.] at the reachable rows.
int launch_degrid_ffts_big(pc_plan_s* p, const float* img, cudaStream_t st) {
  const int nb = compact_blocks(p);
  PC_TRY(p->xc.ensure(sizeof(float2) * (size_t)p->P * nb * p->N * 4));
  float2* Xc = p->xc.as<float2>();
  const int ws = p->wstack ? 1 : 0;
  const bool restricted = p->n_img_rows > 0;
  const int rows_img = restricted ? p->n_img_rows : p->N;
  const int* list = restricted ? p->img_rows : nullptr;
  const uint32_t* bits = restricted ? p->img_row_bits : nullptr;
#define PC_DG(RR)                                                                                          \
  const size_t smem = sizeof(float2) * cfft::Cfg<RR>::Z_ELEMS;                                             \
  static bool done = false;                                                                                \
  if (!done) {                                                                                             \
    PC_TRY(allow(k_degrid_cols_big<RR>, smem));                                                            \
    PC_TRY(allow(k_degrid_rows_big<RR>, smem));                                                            \
    done = true;                                                                                           \
  }                                                                                                        \
  k_degrid_cols_big<RR><<<rows_img, 32 * RR, smem, st>>>(img, p->pix_tab, p->N, p->P, nb,                 \
                                                        p->n_active_rows, ws, p->row_pos, p->active_rows,   \
                                                        p->tw_big, p->tw_in, Xc, list);                    \
  PC_LAUNCH_CHECK();                                                                                       \
  k_degrid_rows_big<RR><<<dim3(p->n_active_rows, p->P), 32 * RR, smem, st>>>(                              \
      Xc, p->N, nb, p->active_rows, p->col_bits, p->tw_big, p->tw_in, p->grid, bits);
  PC_BIG_DISPATCH(p->G, PC_DG)
#undef PC_DG
  PC_LAUNCH_CHECK();
  return PC_OK;
}

#undef PC_BIG_DISPATCH

}  // namespace pc
