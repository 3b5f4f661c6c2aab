// Plan construction: visibility binning by (gridding tile, w-plane), stable
// radix sort, sub-problem list, per-pixel kernel-correction table, workspace.
//
// The adjoint Phi* of Sect. 2.2 is evaluated as a type-1 non-uniform FFT
// (Sect. 5.2): each visibility is spread with an exponential-of-semicircle
// kernel of width W onto a 2x (or more) oversampled uv grid of side G, and
// onto P w-planes (w-stacking, the w-term of Sect. 2.1); every plane is
// inverse-FFT'd and the image is corrected for the kernel's Fourier transform,
// the w-screen and the 1/n factor.
//
// Geometry (all in FP64 here, once per plan):
//   g_u = frac(u dl) G  in [0, G)   grid coordinate in cells (the uv grid is G-periodic)
//   x_w = (w - w0) / dw             plane coordinate
//   planes p = ceil(x_w - W/2) ... + W - 1, with dw = 1 / (2 (s_max - s_min)),
//   s = n - 1 over the image, so that |dw (s - s_c)| <= 1/4 (oversampling 2 in w).
// Each visibility is replicated into every tile its W x W footprint touches
// (at most 2 x 2 tiles since W <= T), so a gridding CTA only ever reads the
// visibilities that touch its own tile.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "pc_internal.cuh"

namespace pc {

// ------------------------------------------------------------------ host math

// Gauss-Legendre nodes and weights on [0, 1] (Newton on the Legendre recurrence).
static void gauss_legendre01(int n, std::vector<double>& x, std::vector<double>& w) {
  x.resize(n);
  w.resize(n);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
    }
    x[i] = 0.5 * (1.0 + z);
    w[i] = 0.5 * 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// Fourier transform of the ES kernel in cell units at frequency t (cycles per cell):
//   psi(t) = int_{-W/2}^{W/2} phi(2y/W) e^{-j 2 pi y t} dy = W int_0^1 phi(z) cos(pi W z t) dz.
static double psi_hat_host(double t, int W, double beta, const std::vector<double>& gx,
                           const std::vector<double>& gw) {
  double s = 0.0;
  for (size_t q = 0; q < gx.size(); ++q) {
    double z = gx[q];
    double phi = std::exp(beta * (std::sqrt(std::max(0.0, 1.0 - z * z)) - 1.0));
    s += gw[q] * phi * std::cos(M_PI * W * z * t);
  }
  return W * s;
}

// ------------------------------------------------------------------ device kernels

// Order-preserving map of a double to uint64 (for atomic min / max).
__device__ __forceinline__ unsigned long long ordered_bits(double d) {
  unsigned long long b = (unsigned long long)__double_as_longlong(d);
  return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}

__global__ void k_uvw_scan(const double* __restrict__ uvw, int64_t M,
                           unsigned long long* wmin, unsigned long long* wmax, int* bad) {
  unsigned long long lo = ~0ull, hi = 0ull;
  int nonfinite = 0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < M;
       k += (int64_t)gridDim.x * blockDim.x) {
    double u = uvw[3 * k], v = uvw[3 * k + 1], w = uvw[3 * k + 2];
    if (!isfinite(u) || !isfinite(v) || !isfinite(w)) nonfinite = 1;
    unsigned long long o = ordered_bits(w);
    lo = o < lo ? o : lo;
    hi = o > hi ? o : hi;
  }
  for (int off = 16; off; off >>= 1) {
    unsigned long long a = __shfl_xor_sync(0xffffffffu, lo, off);
    unsigned long long b = __shfl_xor_sync(0xffffffffu, hi, off);
    lo = a < lo ? a : lo;
    hi = b > hi ? b : hi;
    nonfinite |= __shfl_xor_sync(0xffffffffu, nonfinite, off);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(wmin, lo);
    atomicMax(wmax, hi);
    if (nonfinite) atomicOr(bad, 1);
  }
}

// Bins: (tile, pair of plane starts ps >> 1); within a bin the slots are
// ordered by their tile-local row start b0 (then ps & 1). A sort key is
// bin << 7 | (b0 + 8) << 1 | (ps & 1), b0 in [-(W - 1), T - 1].
struct BinGeom {
  double dl, w0, dw, s_c;
  int G, T, nT, W, P;
  int Pw;           // plane-start pairs (plane windows): ((P - W) >> 1) + 1, or 1 without w-stacking
  unsigned nbins;   // tiles x Pw
};
constexpr int kBinSubBits = 7;

__device__ __forceinline__ int floor_div(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

// Grid coordinate in cells of a baseline component: frac(u dl) G in [0, G).
__device__ __forceinline__ double grid_coord(double u, double dl, int G, double* frac_out) {
  double U = u * dl;
  double f = U - rint(U);
  *frac_out = f;
  double g = f * G;
  if (g < 0.0) g += G;
  if (g >= G) g -= G;
  return g;
}

// Per visibility: fixed-point phase coefficients and up to 4 bin keys (one per
// tile touched by the footprint); unused key slots get the key nbins.
__global__ void k_vis_prep(const double* __restrict__ uvw, int64_t M, BinGeom g,
                           int4* __restrict__ vis_fx, unsigned* __restrict__ keys,
                           unsigned* __restrict__ ids) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= M) return;
  double u = uvw[3 * k], v = uvw[3 * k + 1], w = uvw[3 * k + 2];
  double fu, fv;
  double gu = grid_coord(u, g.dl, g.G, &fu);
  double gv = grid_coord(v, g.dl, g.G, &fv);
  // 32-bit fixed-point turns of u dl and v dl (two's complement wrap = mod 1)
  int Ufx = (int)(unsigned)(long long)llrint(fu * 4294967296.0);
  int Vfx = (int)(unsigned)(long long)llrint(fv * 4294967296.0);
  float w_hi = (float)w;
  float w_lo = (float)(w - (double)w_hi);
  vis_fx[k] = make_int4(Ufx, Vfx, __float_as_int(w_hi), __float_as_int(w_lo));

  int a0 = (int)ceil(gu - 0.5 * g.W);
  int b0 = (int)ceil(gv - 0.5 * g.W);
  int ta0 = floor_div(a0, g.T), ta1 = floor_div(a0 + g.W - 1, g.T);
  int tb0 = floor_div(b0, g.T), tb1 = floor_div(b0 + g.W - 1, g.T);
  int ps = 0;
  if (g.P > 1) ps = (int)ceil((w - g.w0) / g.dw - 0.5 * g.W);
  for (int c = 0; c < 4; ++c) {
    int ta = ta0 + (c & 1), tb = tb0 + (c >> 1);
    unsigned key = g.nbins << kBinSubBits;
    if (ta <= ta1 && tb <= tb1) {
      int tu = ((ta % g.nT) + g.nT) % g.nT;
      int tv = ((tb % g.nT) + g.nT) % g.nT;
      const unsigned bin = (unsigned)((tv * g.nT + tu) * g.Pw + (ps >> 1));
      const unsigned b0l = (unsigned)(b0 - tb * g.T + 8);       // in [1, T + 7]
      key = (bin << kBinSubBits) | (b0l << 1) | (unsigned)(ps & 1);
    }
    keys[4 * k + c] = key;
    ids[4 * k + c] = (unsigned)(4 * k + c);
  }
}

// ---- stable LSD radix sort, 8-bit digits, 4096 keys per block

constexpr int RS_THREADS = 256;
constexpr int RS_ROUNDS = 16;
constexpr int RS_ITEMS = RS_THREADS * RS_ROUNDS;

__global__ void k_rs_hist(const unsigned* __restrict__ keys, int64_t n, int shift,
                          unsigned* __restrict__ hist, int nblk) {
  __shared__ unsigned h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * RS_ITEMS;
  for (int r = 0; r < RS_ROUNDS; ++r) {
    int64_t i = base + r * RS_THREADS + threadIdx.x;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * nblk + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of L unsigned values by one block of 1024 threads.
__global__ void k_scan_single(unsigned* __restrict__ a, int64_t L) {
  __shared__ unsigned warp_tot[32];
  int64_t chunk = (L + blockDim.x - 1) / blockDim.x;
  int64_t lo = threadIdx.x * chunk, hi = lo + chunk < L ? lo + chunk : L;
  unsigned s = 0;
  for (int64_t i = lo; i < hi; ++i) s += a[i];
  // block exclusive scan of s
  unsigned lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned incl = s;
  for (int off = 1; off < 32; off <<= 1) {
    unsigned t = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += t;
  }
  if (lane == 31) warp_tot[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    unsigned t = warp_tot[lane];
    unsigned ti = t;
    for (int off = 1; off < 32; off <<= 1) {
      unsigned u = __shfl_up_sync(0xffffffffu, ti, off);
      if (lane >= off) ti += u;
    }
    warp_tot[lane] = ti - t;
  }
  __syncthreads();
  unsigned run = warp_tot[wid] + incl - s;
  for (int64_t i = lo; i < hi; ++i) {
    unsigned v = a[i];
    a[i] = run;
    run += v;
  }
}

__global__ void k_rs_scatter(const unsigned* __restrict__ kin, const unsigned* __restrict__ vin,
                             unsigned* __restrict__ kout, unsigned* __restrict__ vout, int64_t n,
                             int shift, const unsigned* __restrict__ hist, int nblk) {
  __shared__ unsigned s_base[256];
  __shared__ unsigned s_w[RS_THREADS / 32][256];
  int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  s_base[tid] = hist[(int64_t)tid * nblk + blockIdx.x];
  int64_t base = (int64_t)blockIdx.x * RS_ITEMS;
  unsigned lt_mask = (1u << lane) - 1u;
  for (int r = 0; r < RS_ROUNDS; ++r) {
    for (int w = 0; w < RS_THREADS / 32; ++w) s_w[w][tid] = 0;
    __syncthreads();
    int64_t i = base + r * RS_THREADS + tid;
    bool valid = i < n;
    unsigned key = valid ? kin[i] : 0u;
    unsigned val = valid ? vin[i] : 0u;
    unsigned d = valid ? ((key >> shift) & 255u) : 256u;
    unsigned peers = __match_any_sync(0xffffffffu, d);
    unsigned rank = __popc(peers & lt_mask);
    if (valid && lane == __ffs(peers) - 1) s_w[warp][d] = __popc(peers);
    __syncthreads();
    unsigned run = 0;
    for (int w = 0; w < RS_THREADS / 32; ++w) {
      unsigned c = s_w[w][tid];
      s_w[w][tid] = run;
      run += c;
    }
    __syncthreads();
    if (valid) {
      unsigned pos = s_base[d] + s_w[warp][d] + rank;
      kout[pos] = key;
      vout[pos] = val;
    }
    __syncthreads();
    s_base[tid] += run;
  }
}

// off[b] = first sorted position with key >= b, for b in [0, nbins]; keys <= nbins.
__global__ void k_bin_offsets(const unsigned* __restrict__ keys, int64_t n, unsigned nbins,
                              int* __restrict__ off) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j > n) return;
  long long kcur = j < n ? (long long)(keys[j] >> kBinSubBits) : (long long)nbins;
  long long kprev = j == 0 ? -1 : (long long)(keys[j - 1] >> kBinSubBits);
  for (long long b = kprev + 1; b <= kcur && b <= (long long)nbins; ++b) off[b] = (int)j;
}

// Slot records in sorted order.
__global__ void k_slot_gather(const double* __restrict__ uvw, const unsigned* __restrict__ ids,
                              int64_t n_slots, BinGeom g, int2* __restrict__ slot_vis,
                              float4* __restrict__ slot_geom) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= n_slots) return;
  unsigned id = ids[j];
  int64_t k = id >> 2;
  int c = id & 3;
  double u = uvw[3 * k], v = uvw[3 * k + 1], w = uvw[3 * k + 2];
  double fu, fv;
  double gu = grid_coord(u, g.dl, g.G, &fu);
  double gv = grid_coord(v, g.dl, g.G, &fv);
  int a0 = (int)ceil(gu - 0.5 * g.W);
  int b0 = (int)ceil(gv - 0.5 * g.W);
  int ta = floor_div(a0, g.T) + (c & 1);
  int tb = floor_div(b0, g.T) + (c >> 1);
  int a0l = a0 - ta * g.T;   // footprint start relative to the tile, in [-W+1, T-1]
  int b0l = b0 - tb * g.T;
  float xw = 0.0f, tau = 0.0f;
  int ps = 0;
  if (g.P > 1) {
    double x = (w - g.w0) / g.dw;
    ps = (int)ceil(x - 0.5 * g.W);
    xw = (float)(x - ps);
    double tt = (w - g.w0) * g.s_c;     // pre-twiddle e^{j 2 pi (w - w0) s_c}, in turns
    tau = (float)(tt - rint(tt));
  }
  slot_vis[j] = make_int2((int)k, (int)((unsigned)(a0l + 64) | ((unsigned)(b0l + 64) << 8) | ((unsigned)ps << 16)));
  slot_geom[j] = make_float4((float)(gu - a0), (float)(gv - b0), xw, tau);
}

struct PixGeom {
  double dl, w0, dw, s_c, beta;
  int N, W;
  bool wstack;
};

// Per-pixel epilogue coefficients: {Re, Im} of e^{j 2 pi w0 s} / (n psi(i') psi(j') psi_w(t))
// and t = dw (s - s_c) as a double-float (hi, lo).
__global__ void k_pix_tab(PixGeom g, const double* __restrict__ psi_uv,
                          const double* __restrict__ glx, const double* __restrict__ glw,
                          int nq, float4* __restrict__ out) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t NN = (int64_t)g.N * g.N;
  if (p >= NN) return;
  int i = (int)(p / g.N), j = (int)(p % g.N);
  double l = (i - g.N / 2) * g.dl, m = (j - g.N / 2) * g.dl;
  double r2 = l * l + m * m;
  double n = sqrt(1.0 - r2);
  double s = -r2 / (1.0 + n);        // n - 1 without cancellation
  double t = 0.0, psiw = 1.0;
  if (g.wstack) {
    // psi_w(t) = W sum_q w_q phi(z_q) cos(pi W z_q t): glx holds W z_q and glw
    // w_q phi(z_q) (node-only factors, from the host); |W z_q t| <= W/4, where an
    // FP32 cosine is accurate to ~1e-7
    t = g.dw * (s - g.s_c);
    double acc = 0.0;
    for (int q = 0; q < nq; ++q) acc += glw[q] * (double)cospif((float)(glx[q] * t));
    psiw = g.W * acc;
  }
  double ct = g.w0 * s;
  ct -= rint(ct);                    // exact reduction to [-1/2, 1/2] turns in FP64
  float snf, csf;                    // then an FP32 sine / cosine (~1e-7): FP64 ones are slow here
  sincospif(2.0f * (float)ct, &snf, &csf);
  const double sn = snf, cs = csf;
  double d = 1.0 / (n * psi_uv[i] * psi_uv[j] * psiw);
  float t_hi = (float)t;
  float t_lo = (float)(t - (double)t_hi);
  out[p] = make_float4((float)(cs * d), (float)(sn * d), t_hi, t_lo);
}

// Per-pixel unit-weight atoms, evaluated once per plan: their s = n - 1 and
// 1 / n take FP64 square roots and divisions, a slow pipe on this GPU, which
// the solver's per-iteration bookkeeping then only gathers.
__global__ void k_atom_tab(int N, double dl, float4* __restrict__ out) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= (int64_t)N * N) return;
  out[p] = make_atom((int)p, 1.f, false, N, dl);
}

// The stream plan construction runs on: plan buffers come from the library's
// pool ordered on it (construction ends with a synchronisation of this stream,
// after which every stream may use them).
static thread_local cudaStream_t g_build_stream = nullptr;

static int dev_alloc(pc_plan_s* p, void** ptr, size_t bytes) {
  PC_TRY(dmalloc(ptr, bytes == 0 ? 16 : bytes, g_build_stream));
  p->owned.push_back(*ptr);
  return PC_OK;
}

template <class T>
static int dev_alloc_t(pc_plan_s* p, T** ptr, size_t count) {
  return dev_alloc(p, reinterpret_cast<void**>(ptr), count * sizeof(T));
}

// Temporary device buffers of plan construction, freed on every exit path.
struct TmpBufs {
  std::vector<void*> v;
  cudaStream_t st = nullptr;
  ~TmpBufs() {
    for (void* q : v) dfree(q, st);   // ordered after their last use on st
  }
  int alloc(void** ptr, size_t bytes) {
    PC_TRY(dmalloc(ptr, bytes == 0 ? 16 : bytes, st));
    v.push_back(*ptr);
    return PC_OK;
  }
};

// Splits every (tile, plane group) slot range into equal pieces of at most
// `piece` slots (multiples of 64, the tensor-core stage) and uploads the list.
// Window CTAs: a tile whose slots exceed `cap` is split into equal parts
// (each part takes its share of every plane window of the tile); heaviest
// CTAs first, so the last wave holds the light ones.
static int split_win_parts(pc_plan_s* p, int cap, int4* dst, int* n_out, cudaStream_t st) {
  cap = std::max(cap, 64);
  std::vector<int4> subs;
  for (const int2& t : p->win_tiles) {
    const int parts = ceil_div(t.y, cap);
    for (int k = 0; k < parts; ++k) subs.push_back(make_int4(t.x, k, parts, ceil_div(t.y, parts)));
  }
  std::stable_sort(subs.begin(), subs.end(), [](const int4& a, const int4& b) { return a.w > b.w; });
  if ((int64_t)subs.size() > p->wsub_cap) return fail(PC_ERR_CAPACITY, "plan: %zu window CTAs", subs.size());
  *n_out = (int)subs.size();
  if (!subs.empty())
    PC_CUDA(cudaMemcpyAsync(dst, subs.data(), sizeof(int4) * subs.size(), cudaMemcpyHostToDevice, st));
  PC_CUDA(cudaStreamSynchronize(st));   // the host vector goes out of scope
  return PC_OK;
}

// The window gridding's CTAs (each part adds its tile to the grid).
int split_wsubs(pc_plan_s* p, int cap, cudaStream_t st) {
  PC_TRY(split_win_parts(p, cap, p->wsubs, &p->n_wsub, st));
  p->win_cap = std::max(cap, 64);
  return PC_OK;
}

// The window degridding's CTAs (each part reads its tile's planes; no part
// writes the grid, so the split only costs plane loads).
int split_dwsubs(pc_plan_s* p, int cap, cudaStream_t st) {
  PC_TRY(split_win_parts(p, cap, p->dwsubs, &p->n_dwsub, st));
  p->dwin_cap = std::max(cap, 64);
  return PC_OK;
}

static int split_subs(pc_plan_s* p, int piece, cudaStream_t st) {
  std::vector<int4> subs;
  for (const int4& r : p->sub_ranges) {
    const int len = r.w - r.z;
    const int n_pieces = ceil_div(len, piece);
    const int sz = ceil_div(ceil_div(len, n_pieces), 64) * 64;
    for (int s = r.z; s < r.w; s += sz) subs.push_back(make_int4(r.x, r.y, s, std::min(r.w, s + sz)));
  }
  if ((int)subs.size() > p->sub_cap) return fail(PC_ERR_CAPACITY, "plan: %zu sub-problems", subs.size());
  p->n_sub = (int)subs.size();
  p->grid_piece = piece;
  if (!subs.empty())
    PC_CUDA(cudaMemcpyAsync(p->subs, subs.data(), sizeof(int4) * subs.size(), cudaMemcpyHostToDevice, st));
  PC_CUDA(cudaStreamSynchronize(st));   // the host vector goes out of scope
  return PC_OK;
}

__global__ void k_fill_ones(float2* __restrict__ h, int64_t M) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < M; k += (int64_t)gridDim.x * blockDim.x)
    h[k] = make_float2(1.0f, 0.5f);
}

// Median of `reps` timed calls of f (after one untimed call), in microseconds.
template <class F>
static int time_us(cudaStream_t st, int reps, F f, double* out) {
  cudaEvent_t a, b;
  PC_CUDA(cudaEventCreate(&a));
  PC_CUDA(cudaEventCreate(&b));
  std::vector<double> t;
  int rc = f();
  for (int i = 0; i < reps && rc == PC_OK; ++i) {
    cudaEventRecord(a, st);
    rc = f();
    cudaEventRecord(b, st);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    t.push_back(1e3 * ms);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  PC_TRY(rc);
  std::sort(t.begin(), t.end());
  *out = t[t.size() / 2];
  return PC_OK;
}

// Plan-time autotuner: times, on this plan's binned visibilities, the
// gridding kernels (tensor cores vs CUDA cores, w-stacked plans) x the
// sub-problem sizes, then the first FFT pass's rows per CTA, and keeps the
// fastest of each.
static int autotune(pc_plan_s* p, cudaStream_t st) {
  if (p->M <= 0 || p->n_sub == 0) return PC_OK;
  k_fill_ones<<<(int)std::min<int64_t>(4096, (p->M + 255) / 256), 256, 0, st>>>(p->resid, p->M);
  PC_LAUNCH_CHECK();
  const int user_mode = p->grid_mode;
  std::vector<int> modes = {user_mode};
  if (user_mode == 0 && p->wstack) modes = p->W <= 7 ? std::vector<int>{3, 2, 1} : std::vector<int>{2, 1};
  double best = 1e300;
  int best_mode = user_mode, best_piece = grid_win_mode(p) ? p->win_cap : p->grid_piece;
  for (int mode : modes) {
    p->grid_mode = mode;
    const bool win = grid_win_mode(p);
    // window gridding: slots per CTA before a tile is split; else the sub-problem size
    const std::vector<int> pieces = win ? std::vector<int>{1024, 4096, 16384, 65536}
                                        : std::vector<int>{256, 512, 1024, 2048, 4096};
    for (int piece : pieces) {
      p->grid_mode = mode;
      PC_TRY(win ? split_wsubs(p, piece, st) : split_subs(p, piece, st));
      double us = 0.0;
      PC_TRY(time_us(st, 3, [&] { return launch_grid(p, p->resid, st); }, &us));
      if (us < best) {
        best = us;
        best_mode = mode;
        best_piece = piece;
      }
    }
  }
  p->grid_mode = best_mode;
  PC_TRY(grid_win_mode(p) ? split_wsubs(p, best_piece, st) : split_subs(p, best_piece, st));
  p->tune_grid_us = best;
  PC_TRY(launch_grid(p, p->resid, st));         // a gridded plane set for the FFT timing
  // first pass: the one-warp register FFT (where G allows it) against the
  // shared-memory Stockham kernel at each rows-per-CTA
  double best_fft = 1e300;
  int best_R = 0, best_rw = 0;
  p->fft_warp = 1;
  if (fft_rows_warp(p) || fft_rows_big(p)) {
    PC_TRY(time_us(st, 3, [&] { return launch_fft_rows(p, st); }, &best_fft));
    best_rw = 1;
  }
  p->fft_warp = 0;
  for (int R : {1, 2, 4, 8, 16, 32}) {
    if (((size_t)2 * R * (p->G + 1) + p->G) * sizeof(float2) > 200 * 1024) break;
    p->fft_R = R;
    double us = 0.0;
    PC_TRY(time_us(st, 3, [&] { return launch_fft_rows(p, st); }, &us));
    if (us < best_fft) {
      best_fft = us;
      best_R = R;
      best_rw = 0;
    }
  }
  p->fft_R = best_R;
  p->tune_fft_us = best_fft;
  p->fft_warp = best_rw;
  // second pass: one-warp register FFTs against the Stockham kernel at each
  // number of planes transformed together (shared memory vs CTAs per SM)
  PC_TRY(launch_fft_rows(p, st));
  double best_cols = 1e300;
  int best_pg = 1, best_cw = 0;
  p->fft_warp = best_rw | 2;
  if (fft_cols_warp(p) || fft_cols_big(p)) {
    PC_TRY(time_us(st, 3, [&] { return launch_fft_cols_epilogue(p, p->mu, 1.0f, nullptr, st); },
                   &best_cols));
    best_cw = 2;
  }
  p->fft_warp = best_rw;
  for (int pg : {1, 2, 4, 8}) {
    p->fft_cols_pg = pg;
    if (cols_planes_per_pass(p) != pg) break;   // beyond the planes or shared memory
    double us = 0.0;
    PC_TRY(time_us(st, 3, [&] { return launch_fft_cols_epilogue(p, p->mu, 1.0f, nullptr, st); }, &us));
    if (us < best_cols) {
      best_cols = us;
      best_pg = pg;
      best_cw = 0;
    }
  }
  p->fft_cols_pg = best_pg;
  p->tune_fft_cols_us = best_cols;
  p->fft_warp = best_rw | best_cw;
  // window degridding: slots per CTA before a tile is split (into the
  // residual buffer, cleared below; the grid holds the planes timed above)
  if (grid_win_mode(p)) {
    double best_dw = 1e300;
    int best_cap = p->dwin_cap;
    for (int cap : {2048, 4096, 8192, 16384}) {
      PC_TRY(split_dwsubs(p, cap, st));
      double us = 0.0;
      PC_TRY(time_us(st, 3, [&] { return launch_degrid_win(p, p->resid, st); }, &us));
      if (us < best_dw) {
        best_dw = us;
        best_cap = cap;
      }
    }
    PC_TRY(split_dwsubs(p, best_cap, st));
    p->tune_degrid_us = best_dw;
  }
  p->tuned = true;
  PC_CUDA(cudaMemsetAsync(p->resid, 0, sizeof(float2) * p->M, st));
  PC_CUDA(cudaStreamSynchronize(st));
  return PC_OK;
}

static int build_plan(pc_plan_s* p, const double* uvw, cudaStream_t st, int max_planes) {
  const int64_t M = p->M;
  const int N = p->N;
  g_build_stream = st;
  TmpBufs tmp;
  tmp.st = st;

  // ---- w range and finiteness
  if (M > 0) {
    unsigned long long* dmm;
    int* dbad;
    PC_TRY(tmp.alloc((void**)&dmm, 2 * sizeof(unsigned long long) + sizeof(int) * 2));
    dbad = reinterpret_cast<int*>(dmm + 2);
    unsigned long long init[2] = {~0ull, 0ull};
    int zero[2] = {0, 0};
    PC_CUDA(cudaMemcpyAsync(dmm, init, sizeof(init), cudaMemcpyHostToDevice, st));
    PC_CUDA(cudaMemcpyAsync(dbad, zero, sizeof(zero), cudaMemcpyHostToDevice, st));
    int blocks = (int)std::min<int64_t>(4096, (M + 255) / 256);
    k_uvw_scan<<<blocks, 256, 0, st>>>(uvw, M, dmm, dmm + 1, dbad);
    PC_LAUNCH_CHECK();
    unsigned long long hmm[2];
    int hbad[2];
    PC_CUDA(cudaMemcpyAsync(hmm, dmm, sizeof(hmm), cudaMemcpyDeviceToHost, st));
    PC_CUDA(cudaMemcpyAsync(hbad, dbad, sizeof(hbad), cudaMemcpyDeviceToHost, st));
    PC_CUDA(cudaStreamSynchronize(st));
    if (hbad[0]) return fail(PC_ERR_INVALID_ARG, "plan: uvw contains NaN or Inf");
    auto unmap = [](unsigned long long o) {
      unsigned long long b = (o & 0x8000000000000000ull) ? (o & 0x7fffffffffffffffull) : ~o;
      double d;
      std::memcpy(&d, &b, sizeof(d));
      return d;
    };
    p->w_min = unmap(hmm[0]);
    p->w_max = unmap(hmm[1]);
  }

  // ---- geometry
  p->G = 32;
  while (p->G < 2 * N) p->G *= 2;
  p->logG = 0;
  while ((1 << p->logG) < p->G) ++p->logG;
  p->nT = p->G / p->T;
  p->dl = p->fov / N;
  p->beta = 2.30 * p->W;
  const double half = 0.5 * N * p->dl;
  const double r2c = 2.0 * half * half;
  const double s_min = -r2c / (1.0 + std::sqrt(1.0 - r2c));
  const double s_max = 0.0;
  if (M > 0 && p->w_max > p->w_min) {
    p->wstack = true;
    p->dw = 1.0 / (2.0 * (s_max - s_min));
    long long planes = (long long)std::ceil((p->w_max - p->w_min) / p->dw) + p->W;
    if (planes > max_planes)
      return fail(PC_ERR_INVALID_ARG, "plan: %lld w-planes needed, max_planes is %d", planes,
                  max_planes);
    p->P = (int)planes;
    p->w0 = p->w_min - 0.5 * p->W * p->dw;
    p->s_c = 0.5 * (s_min + s_max);
  } else {
    p->wstack = false;
    p->P = 1;
    p->dw = 1.0;
    p->w0 = M > 0 ? p->w_min : 0.0;
    p->s_c = 0.0;
  }
  {
    int ngroups = ceil_div(p->P, 8);      // gridding keeps <= 8 planes of a tile in registers
    p->Qg = ceil_div(p->P, ngroups);
  }

  // ---- tables: ES transform, twiddles, per-pixel corrections
  std::vector<double> gx, gw;
  gauss_legendre01(kGlNodes, gx, gw);
  std::vector<double> psi(N);
  for (int i = 0; i < N; ++i) psi[i] = psi_hat_host((double)(i - N / 2) / p->G, p->W, p->beta, gx, gw);
  double *d_psi, *d_gx, *d_gw;
  PC_TRY(tmp.alloc((void**)&d_psi, sizeof(double) * (N + 2 * kGlNodes)));
  d_gx = d_psi + N;
  d_gw = d_gx + kGlNodes;
  PC_CUDA(cudaMemcpyAsync(d_psi, psi.data(), sizeof(double) * N, cudaMemcpyHostToDevice, st));
  // node factors of the w-kernel correction: W z_q and w_q phi(z_q)
  std::vector<double> wz(kGlNodes), wphi(kGlNodes);
  for (int q = 0; q < kGlNodes; ++q) {
    wz[q] = p->W * gx[q];
    wphi[q] = gw[q] * std::exp(p->beta * (std::sqrt(std::max(0.0, 1.0 - gx[q] * gx[q])) - 1.0));
  }
  PC_CUDA(cudaMemcpyAsync(d_gx, wz.data(), sizeof(double) * kGlNodes, cudaMemcpyHostToDevice, st));
  PC_CUDA(cudaMemcpyAsync(d_gw, wphi.data(), sizeof(double) * kGlNodes, cudaMemcpyHostToDevice, st));
  const int64_t NN = (int64_t)N * N;
  PC_TRY(dev_alloc_t(p, &p->pix_tab, NN));
  {
    PixGeom pg{p->dl, p->w0, p->dw, p->s_c, p->beta, N, p->W, p->wstack};
    k_pix_tab<<<ceil_div(NN, 256), 256, 0, st>>>(pg, d_psi, d_gx, d_gw, kGlNodes, p->pix_tab);
    PC_LAUNCH_CHECK();
  }
  PC_TRY(dev_alloc_t(p, &p->atom_tab, NN));
  k_atom_tab<<<ceil_div(NN, 256), 256, 0, st>>>(N, p->dl, p->atom_tab);
  PC_LAUNCH_CHECK();
  std::vector<float2> tw(p->G);
  for (int k = 0; k < p->G; ++k) {
    double a = 2.0 * M_PI * k / p->G;
    tw[k] = make_float2((float)std::cos(a), (float)std::sin(a));
  }
  PC_TRY(dev_alloc_t(p, &p->twiddle, p->G));
  PC_CUDA(cudaMemcpyAsync(p->twiddle, tw.data(), sizeof(float2) * p->G, cudaMemcpyHostToDevice, st));
  if (p->G == 512 || p->G == 1024) {
    const int L = p->G / 32;
    std::vector<float2> t2((size_t)32 * L);
    for (int k1 = 0; k1 < L; ++k1)
      for (int l = 0; l < 32; ++l) t2[(size_t)k1 * 32 + l] = tw[(size_t)(k1 * l) % p->G];
    PC_TRY(dev_alloc_t(p, &p->tw2, t2.size()));
    PC_CUDA(cudaMemcpyAsync(p->tw2, t2.data(), sizeof(float2) * t2.size(), cudaMemcpyHostToDevice, st));
  }

  if (fft_big_size(p->G)) {
    // the 512-point one-warp FFT inside the one-CTA transform: e^{+2 pi i l k1 / 512}
    std::vector<float2> t2(16 * 32);
    const int step = p->G / 512;
    for (int k1 = 0; k1 < 16; ++k1)
      for (int l = 0; l < 32; ++l) t2[(size_t)k1 * 32 + l] = tw[(size_t)(k1 * l * step) % p->G];
    PC_TRY(dev_alloc_t(p, &p->tw_in, t2.size()));
    PC_CUDA(cudaMemcpyAsync(p->tw_in, t2.data(), sizeof(float2) * t2.size(), cudaMemcpyHostToDevice, st));
    // its first step's twiddles by (k1, n'): e^{+2 pi i n' k1 / G}, n' < 512
    std::vector<float2> ta((size_t)p->G);
    for (int k1 = 0; k1 < p->G / 512; ++k1)
      for (int n = 0; n < 512; ++n) ta[(size_t)k1 * 512 + n] = tw[((size_t)n * k1) % p->G];
    PC_TRY(dev_alloc_t(p, &p->tw_big, ta.size()));
    PC_CUDA(cudaMemcpyAsync(p->tw_big, ta.data(), sizeof(float2) * ta.size(), cudaMemcpyHostToDevice, st));
  }

  // ---- workspaces
  PC_TRY(dev_alloc_t(p, &p->grid, (size_t)p->P * p->G * p->G));
  PC_CUDA(cudaMemsetAsync(p->grid, 0, sizeof(float2) * (size_t)p->P * p->G * p->G, st));
  // the Stockham passes' transposed pass-1 output (every G up to 1024; for
  // larger grids only when those passes can be chosen: forced, or timed by
  // the autotuner; the one-CTA passes use the compact buffer xc instead)
  if (!fft_big_size(p->G) || p->fft_warp == 0 || p->want_tune) {
    PC_TRY(dev_alloc_t(p, &p->fft1, (size_t)p->P * N * p->G));
    // columns b of the transposed pass-1 output whose grid rows never hold a
    // visibility stay zero for every certificate: clear them once here
    PC_CUDA(cudaMemsetAsync(p->fft1, 0, sizeof(float2) * (size_t)p->P * N * p->G, st));
  }
  PC_TRY(dev_alloc_t(p, &p->resid, (size_t)std::max<int64_t>(M, 1)));
  PC_TRY(dev_alloc_t(p, &p->mu, (size_t)NN));
  PC_TRY(dev_alloc_t(p, &p->mark, (size_t)NN));
  PC_CUDA(cudaMemsetAsync(p->mark, 0, NN, st));
  PC_TRY(dev_alloc_t(p, &p->dscal, 8));
  PC_TRY(dev_alloc_t(p, &p->uscal, 8));
  PC_TRY(dev_alloc_t(p, &p->iscal, 8));
  PC_CUDA(cudaMemsetAsync(p->iscal, 0, 8 * sizeof(int32_t), st));
  p->sel_blocks_n = ceil_div(NN, kSelItems);
  PC_TRY(dev_alloc_t(p, &p->sel_blocks, (size_t)p->sel_blocks_n + 2));
  PC_CUDA(cudaMemsetAsync(p->sel_blocks, 0, sizeof(int32_t) * ((size_t)p->sel_blocks_n + 2), st));
  PC_TRY(dev_alloc_t(p, &p->vis_fx, (size_t)std::max<int64_t>(M, 1)));

  if (M == 0) {
    p->n_slots = 0;
    p->n_sub = 0;
    PC_TRY(dev_alloc_t(p, &p->slot_vis, 1));
    PC_TRY(dev_alloc_t(p, &p->slot_geom, 1));
    PC_TRY(dev_alloc_t(p, &p->subs, 1));
    PC_CUDA(cudaStreamSynchronize(st));
    return PC_OK;
  }

  // ---- binning keys
  p->Pw = p->wstack ? ((p->P - p->W) >> 1) + 1 : 1;
  const unsigned nbins = (unsigned)((int64_t)p->nT * p->nT * p->Pw);
  if ((int64_t)p->nT * p->nT * p->Pw >= (1ll << (32 - kBinSubBits)))
    return fail(PC_ERR_INVALID_ARG, "plan: too many (tile, plane pair) bins");
  const int64_t nkeys = 4 * M;
  unsigned *k0, *k1, *v0, *v1, *hist;
  int* off;
  PC_TRY(tmp.alloc((void**)&k0, sizeof(unsigned) * nkeys));
  PC_TRY(tmp.alloc((void**)&k1, sizeof(unsigned) * nkeys));
  PC_TRY(tmp.alloc((void**)&v0, sizeof(unsigned) * nkeys));
  PC_TRY(tmp.alloc((void**)&v1, sizeof(unsigned) * nkeys));
  const int nblk = ceil_div(nkeys, RS_ITEMS);
  PC_TRY(tmp.alloc((void**)&hist, sizeof(unsigned) * 256 * (size_t)nblk));
  PC_TRY(tmp.alloc((void**)&off, sizeof(int) * ((size_t)nbins + 1)));
  BinGeom bg{p->dl, p->w0, p->dw, p->s_c, p->G, p->T, p->nT, p->W, p->P, p->Pw, nbins};
  k_vis_prep<<<ceil_div(M, 256), 256, 0, st>>>(uvw, M, bg, p->vis_fx, k0, v0);
  PC_LAUNCH_CHECK();

  // ---- stable radix sort of the keys (values = slot ids)
  int nbits = 1;
  while ((1ull << nbits) <= ((unsigned long long)nbins << kBinSubBits)) ++nbits;
  unsigned *kin = k0, *vin = v0, *kout = k1, *vout = v1;
  for (int shift = 0; shift < nbits; shift += 8) {
    k_rs_hist<<<nblk, RS_THREADS, 0, st>>>(kin, nkeys, shift, hist, nblk);
    PC_LAUNCH_CHECK();
    k_scan_single<<<1, 1024, 0, st>>>(hist, 256 * (int64_t)nblk);
    PC_LAUNCH_CHECK();
    k_rs_scatter<<<nblk, RS_THREADS, 0, st>>>(kin, vin, kout, vout, nkeys, shift, hist, nblk);
    PC_LAUNCH_CHECK();
    std::swap(kin, kout);
    std::swap(vin, vout);
  }
  k_bin_offsets<<<ceil_div(nkeys + 1, 256), 256, 0, st>>>(kin, nkeys, nbins, off);
  PC_LAUNCH_CHECK();
  std::vector<int> hoff((size_t)nbins + 1);
  PC_CUDA(cudaMemcpyAsync(hoff.data(), off, sizeof(int) * hoff.size(), cudaMemcpyDeviceToHost, st));
  PC_CUDA(cudaStreamSynchronize(st));
  p->n_slots = hoff[nbins];

  PC_TRY(dev_alloc_t(p, &p->slot_vis, (size_t)std::max<int64_t>(p->n_slots, 1)));
  PC_TRY(dev_alloc_t(p, &p->slot_geom, (size_t)std::max<int64_t>(p->n_slots, 1)));
  if (p->n_slots > 0) {
    k_slot_gather<<<ceil_div(p->n_slots, 256), 256, 0, st>>>(uvw, vin, p->n_slots, bg,
                                                             p->slot_vis, p->slot_geom);
    PC_LAUNCH_CHECK();
  }

  // ---- gridding sub-problems: the slot range of each (tile, plane group),
  // split into equal pieces of at most kMaxSlotsPerSub slots (multiples of 64,
  // the tensor-core stage) sized so that the pieces fill the GPU in about two
  // even waves of two CTAs per SM -- a few long sub-problems left over for a
  // second wave would otherwise double the gridding time.
  const int kMaxSlotsPerSub = 512;   // the autotuner's usual pick (smaller pieces: more CTAs in flight)
  std::vector<int4> ranges;
  int64_t total_slots = 0;
  const int ngroups = ceil_div(p->P, p->Qg);
  for (int t = 0; t < p->nT * p->nT; ++t) {
    for (int gq = 0; gq < ngroups; ++gq) {
      int q0 = gq * p->Qg;
      // plane starts whose footprint meets the group, widened to whole pairs
      // (the extra slots' footprints miss the group: zero weights there)
      int ps_lo = 0, ps_hi = 0;
      if (p->wstack) {
        ps_lo = std::max(0, q0 - p->W + 1);
        ps_hi = std::min(p->P - p->W, q0 + p->Qg - 1);
      }
      if (ps_hi < ps_lo) continue;
      int s0 = hoff[(size_t)t * p->Pw + (ps_lo >> 1)];
      int s1 = hoff[(size_t)t * p->Pw + (ps_hi >> 1) + 1];
      if (s1 > s0) {
        ranges.push_back(make_int4(t, gq, s0, s1));
        total_slots += s1 - s0;
      }
    }
  }
  int n_sm = 152;
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, p->device);
  const int64_t want = 4ll * n_sm;
  int piece = (int)std::min<int64_t>(kMaxSlotsPerSub, std::max<int64_t>(128, (total_slots + want - 1) / want));
  piece = ceil_div(piece, 64) * 64;
  p->sub_ranges = ranges;
  // tile rows / columns that hold visibilities (the one-warp FFTs skip the rest, which stay zero)
  p->row_mask = p->col_mask = 0;
  if (p->nT <= 32)
    for (const int4& s : ranges) {
      p->row_mask |= 1u << (s.x / p->nT);
      p->col_mask |= 1u << (s.x % p->nT);
    }
  // room for the finest split the autotuner may try (pieces of 64 slots)
  p->sub_cap = (int)(total_slots / 64 + (int64_t)ranges.size() + 1);
  PC_TRY(dev_alloc_t(p, &p->subs, (size_t)p->sub_cap));
  PC_TRY(split_subs(p, piece, st));
  // window gridding: the bin offsets on the device, the tiles that hold slots,
  // and the CTA list. Measured (2048^2 / 2M and 4096^2 / 10M): splitting a
  // tile costs more than it balances once the tiles alone give eight CTAs per
  // SM, so then only tiles beyond 65536 slots are split; with fewer tiles,
  // parts of at most 4096 slots
  PC_TRY(dev_alloc_t(p, &p->win_off, (size_t)nbins + 1));
  PC_CUDA(cudaMemcpyAsync(p->win_off, off, sizeof(int) * ((size_t)nbins + 1), cudaMemcpyDeviceToDevice, st));
  p->win_tiles.clear();
  for (int t = 0; t < p->nT * p->nT; ++t) {
    const int n = hoff[(size_t)(t + 1) * p->Pw] - hoff[(size_t)t * p->Pw];
    if (n > 0) p->win_tiles.push_back(make_int2(t, n));
  }
  p->wsub_cap = p->n_slots / 64 + (int64_t)p->win_tiles.size() + 1;
  PC_TRY(dev_alloc_t(p, &p->wsubs, (size_t)p->wsub_cap));
  PC_TRY(split_wsubs(p, (int64_t)p->win_tiles.size() >= 8ll * n_sm ? 65536 : 4096, st));
  PC_TRY(dev_alloc_t(p, &p->dwsubs, (size_t)p->wsub_cap));
  // window degridding: parts of at most 8192 slots (measured best or within
  // 2 % of the best cap on 2048^2 / 2M and 4096^2 / 10M; the tuner times it)
  PC_TRY(split_dwsubs(p, 8192, st));
  // grid rows that any visibility can reach: the rows of tile rows with a sub-problem
  {
    std::vector<char> row_on(p->nT, 0);
    for (const int4& s : ranges) row_on[s.x / p->nT] = 1;
    std::vector<int> rows;
    for (int tv = 0; tv < p->nT; ++tv)
      if (row_on[tv])
        for (int b = 0; b < p->T; ++b) rows.push_back(tv * p->T + b);
    p->n_active_rows = (int)rows.size();
    PC_TRY(dev_alloc_t(p, &p->active_rows, std::max<size_t>(rows.size(), 1)));
    if (!rows.empty())
      PC_CUDA(cudaMemcpyAsync(p->active_rows, rows.data(), sizeof(int) * rows.size(),
                              cudaMemcpyHostToDevice, st));
    // compact position of every grid row, and the column groups that can hold data
    std::vector<int> pos(p->G, -1);
    for (size_t c = 0; c < rows.size(); ++c) pos[rows[c]] = (int)c;
    PC_TRY(dev_alloc_t(p, &p->row_pos, (size_t)p->G));
    PC_CUDA(cudaMemcpyAsync(p->row_pos, pos.data(), sizeof(int) * p->G, cudaMemcpyHostToDevice, st));
    std::vector<uint32_t> colw((size_t)std::max(1, p->G / 1024), 0u);
    for (const int4& s : ranges) {
      const int g = s.x % p->nT;                  // a tile column is one 32-column group
      colw[(size_t)g >> 5] |= 1u << (g & 31);
    }
    p->n_active_col_groups = 0;
    for (uint32_t word : colw) p->n_active_col_groups += __builtin_popcount(word);
    PC_TRY(dev_alloc_t(p, &p->col_bits, colw.size()));
    PC_CUDA(cudaMemcpyAsync(p->col_bits, colw.data(), sizeof(uint32_t) * colw.size(), cudaMemcpyHostToDevice,
                            st));
    if (fft_big_size(p->G)) {
      // the one-CTA passes' compact rows, allocated here (never inside a captured solve)
      const size_t nb = (size_t)ceil_div(std::max(p->n_active_rows, 1), 4);
      PC_TRY(p->xc.ensure(sizeof(float2) * (size_t)p->P * nb * N * 4));
      PC_TRY(make_xc_tensor_map(p));
    }
  }
  PC_CUDA(cudaStreamSynchronize(st));
  return PC_OK;
}

// Device bytes a plan and its solve may hold (an upper estimate used to admit
// jobs by memory): the gridding planes, the pass-1 FFT buffer, the pixel
// tables, the binned visibilities, the working set of the solver and the
// tensor-core phase buffer (chunked at 2 GB).
int64_t plan_bytes_estimate(int64_t M, int N, double fov, double w_min, double w_max, int W) {
  int64_t G = 32;
  while (G < 2 * N) G *= 2;
  const double dl = fov / N;
  const double half = 0.5 * N * dl;
  const double r2c = 2.0 * half * half;
  const double s_min = -r2c / (1.0 + std::sqrt(std::max(1.0 - r2c, 1e-12)));
  int64_t P = 1;
  if (M > 0 && w_max > w_min) {
    const double dw = 1.0 / (2.0 * (0.0 - s_min));
    P = (int64_t)std::ceil((w_max - w_min) / dw) + W;
  }
  const int64_t groups = (P + 7) / 8;
  const int64_t NN = (int64_t)N * N;
  int64_t b = 0;
  b += P * G * G * 8;                       // grid planes
  b += P * N * G * 8;                       // pass-1 FFT output
  b += NN * (16 + 16 + 4 + 1 + 4);          // pixel and atom tables, mu, marks, selection
  b += M * (16 + 8);                        // fixed-point visibilities, residual
  b += M * groups * 2 * 24;                 // binned slots (replication into tiles and plane groups)
  b += 2 * 4096ll * 4096ll * 4;             // Gram working set (grown on demand; 4096 atoms)
  b += std::min<int64_t>(2ll << 30, 1024 * M * 8);   // phase buffer of the tensor-core Gram
  b += 64ll << 20;                          // scratch
  return b;
}

}  // namespace pc

using namespace pc;

extern "C" int pc_plan_create(const double* uvw_dev, int64_t M, int32_t N, double fov_rad,
                              const pc_plan_opts* opts, void* stream, pc_plan_t* plan_out) {
  clear_error();
  if (!plan_out) return fail(PC_ERR_INVALID_ARG, "pc_plan_create: plan_out is NULL");
  *plan_out = nullptr;
  if (opts && opts->version != PC_ABI_VERSION)
    return fail(PC_ERR_INVALID_ARG, "pc_plan_create: opts->version %d != %d", opts->version,
                PC_ABI_VERSION);
  if (M < 0 || M > (1ll << 29))
    return fail(PC_ERR_INVALID_ARG, "pc_plan_create: M = %lld out of range [0, 2^29]", (long long)M);
  if (N < 16 || N > 4096 || (N & 1))
    return fail(PC_ERR_INVALID_ARG, "pc_plan_create: N = %d must be even and in [16, 4096]", N);
  if (!(fov_rad > 0.0) || !(fov_rad < 1.4))
    return fail(PC_ERR_INVALID_ARG, "pc_plan_create: fov_rad = %g must be in (0, 1.4)", fov_rad);
  if (M > 0 && !is_device_ptr(uvw_dev))
    return fail(PC_ERR_INVALID_ARG, "pc_plan_create: uvw_dev is not a device pointer");
  int W = (opts && opts->kernel_width) ? opts->kernel_width : 7;
  int T = (opts && opts->tile) ? opts->tile : 32;
  int maxP = (opts && opts->max_planes) ? opts->max_planes : 256;
  if (W < 4 || W > kMaxW) return fail(PC_ERR_INVALID_ARG, "pc_plan_create: kernel_width %d not in [4, 8]", W);
  if (T != 32) return fail(PC_ERR_INVALID_ARG, "pc_plan_create: tile %d must be 32", T);
  if (maxP < 1 || maxP > 4096) return fail(PC_ERR_INVALID_ARG, "pc_plan_create: max_planes %d", maxP);
  const int grid_mode = opts ? opts->grid_mode : 0;
  if (grid_mode < 0 || grid_mode > 3)
    return fail(PC_ERR_INVALID_ARG, "pc_plan_create: grid_mode %d not in [0, 3]", grid_mode);
  const int tune = opts ? opts->autotune : 0;
  if (tune != 0 && tune != 1) return fail(PC_ERR_INVALID_ARG, "pc_plan_create: autotune must be 0 or 1");
  const int fft_kernel = opts ? opts->fft_kernel : 0;
  if (fft_kernel != 0 && fft_kernel != 1)
    return fail(PC_ERR_INVALID_ARG, "pc_plan_create: fft_kernel must be 0 or 1");

  pc_plan_s* p = new pc_plan_s();
  cudaGetDevice(&p->device);
  p->M = M;
  p->N = N;
  p->fov = fov_rad;
  p->W = W;
  p->T = T;
  p->grid_mode = grid_mode;
  p->fft_warp = fft_kernel == 1 ? 0 : -1;
  p->want_tune = tune == 1;
  int rc = build_plan(p, uvw_dev, (cudaStream_t)stream, maxP);
  if (rc == PC_OK && tune) rc = autotune(p, (cudaStream_t)stream);
  if (rc != PC_OK) {
    pc_plan_destroy(p);
    return rc;
  }
  *plan_out = p;
  return PC_OK;
}

extern "C" int pc_plan_tuning_info(pc_plan_t p, pc_plan_tuning* out) {
  clear_error();
  if (!p || !out) return fail(PC_ERR_INVALID_ARG, "pc_plan_tuning_info: NULL argument");
  out->tuned = p->tuned ? 1 : 0;
  out->grid_mode = grid_win_mode(p) ? 3 : (p->wstack && p->grid_mode != 1) ? 2 : 1;
  out->grid_piece = grid_win_mode(p) ? p->win_cap : p->grid_piece;
  int R = p->fft_R > 0 ? p->fft_R : 2048 / p->G;
  const bool rw = fft_rows_warp(p) || fft_rows_big(p), cw = fft_cols_warp(p) || fft_cols_big(p);
  out->fft_rows_per_cta = fft_rows_big(p) ? 1 : rw ? 8 : std::min(std::max(R, 1), 32);
  out->grid_us = p->tune_grid_us;
  out->fft_rows_us = p->tune_fft_us;
  out->fft_cols_planes = cw ? 1 : cols_planes_per_pass(p);
  out->fft_cols_us = p->tune_fft_cols_us;
  out->fft_warp = (rw ? 1 : 0) | (cw ? 2 : 0);
  out->degrid_piece = grid_win_mode(p) ? p->dwin_cap : 0;
  out->reserved = 0;
  out->degrid_us = p->tune_degrid_us;
  return PC_OK;
}

extern "C" void pc_plan_destroy(pc_plan_t p) {
  if (!p) return;
  // the buffers may still be in use on any stream: wait for the device once
  // (as cudaFree would), then return them to the pool
  cudaDeviceSynchronize();
  for (void* q : p->owned) dfree(q, 0);
  p->atomsA.release();
  p->atomsB.release();
  p->idxA.release();
  p->idxB.release();
  p->xA.release();
  p->xB.release();
  p->oldpos.release();
  p->newrows.release();
  p->keep.release();
  p->GA.release();
  p->GB.release();
  p->bA.release();
  p->bB.release();
  p->acc.release();
  p->perm.release();
  p->atomsP.release();
  p->pbuf.release();
  p->degrid_buf.release();
  p->xc.release();
  p->opw.release();
  p->dirty.release();
  if (p->dict) {
    p->dict->release();
    delete p->dict;
  }
  if (p->scache) {
    p->scache->release();
    delete p->scache;
  }
  delete p;
}

extern "C" int pc_plan_reach(pc_plan_t p, int32_t* rows, int32_t* col_groups) {
  clear_error();
  if (!p) return fail(PC_ERR_INVALID_ARG, "pc_plan_reach: NULL plan");
  if (rows) *rows = p->n_active_rows;
  if (col_groups) *col_groups = p->n_active_col_groups;
  return PC_OK;
}

extern "C" int pc_plan(const double* uvw_dev, int64_t M, int32_t N, double fov_rad,
                       const pc_plan_opts* opts, void* stream, pc_plan_t* plan_out) {
  return pc_plan_create(uvw_dev, M, N, fov_rad, opts, stream, plan_out);
}

extern "C" int pc_plan_info(pc_plan_t p, int32_t* grid_side, int32_t* tile, int32_t* n_planes,
                            int64_t* n_slots, int32_t* kernel_width, double* dw) {
  if (!p) return fail(PC_ERR_INVALID_ARG, "pc_plan_info: NULL plan");
  if (grid_side) *grid_side = p->G;
  if (tile) *tile = p->T;
  if (n_planes) *n_planes = p->P;
  if (n_slots) *n_slots = p->n_slots;
  if (kernel_width) *kernel_width = p->W;
  if (dw) *dw = p->dw;
  return PC_OK;
}
