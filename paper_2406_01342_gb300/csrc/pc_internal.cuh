// Internal declarations of the PolyCLEAN GB300 library (not part of the C ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "polyclean.h"

namespace pc {

// ------------------------------------------------------------------ errors

int fail(int code, const char* fmt, ...);          // records a message, returns code
void clear_error();

#define PC_CUDA(call)                                                                  \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return ::pc::fail(e_ == cudaErrorMemoryAllocation ? PC_ERR_OOM : PC_ERR_CUDA,    \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__,     \
                        __LINE__);                                                     \
  } while (0)

#define PC_LAUNCH_CHECK() PC_CUDA(cudaGetLastError())

#define PC_TRY(expr)              \
  do {                            \
    int s_ = (expr);              \
    if (s_ != PC_OK) return s_;   \
  } while (0)

// Device pointer check: true for device or managed memory of any device.
bool is_device_ptr(const void* p);

// Memory of the library. Device memory comes from a stream-ordered pool per
// device that keeps freed blocks for reuse (cudaFree, and the unmapping it
// implies, costs 0.05-1 ms per call; a plan holds about twenty buffers);
// pc_trim_memory returns the cached memory. Pinned host blocks and
// non-blocking streams are recycled through free lists.
int dmalloc(void** ptr, size_t bytes, cudaStream_t st);   // ordered on st
void dfree(void* ptr, cudaStream_t st);                    // ordered on st
void dfree_idle(void* ptr);                                // after a device synchronisation
void* pinned_get(size_t bytes);                            // nullptr on failure
void pinned_put(void* q);
cudaStream_t stream_get();                                 // non-blocking; nullptr on failure
void stream_put(cudaStream_t s);
int trim_memory();

// Grow-only device buffer.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  int ensure(size_t nbytes);
  void release();
  template <class T> T* as() const { return static_cast<T*>(p); }
};

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// Kernel timing (see pc_profile_begin): prof_start() returns a token or -1
// when recording is off; prof_stop() records the end event of that token.
enum ProfClass { PROF_PLAN = 0, PROF_GRID, PROF_FFT_ROWS, PROF_FFT_COLS, PROF_RESIDUAL,
                 PROF_GRAM, PROF_GRAM_FINALIZE, PROF_APGD, PROF_SELECT, PROF_MISC,
                 PROF_GRAM_TC, PROF_GRAM_THIN, PROF_DICT_CORR, PROF_DICT_COLUMNS, PROF_PHASE_GEN,
                 PROF_APGD_OP, PROF_DEGRID, PROF_DEGRID_FFT, PROF_NCLASSES };
int prof_start(int cls, cudaStream_t st);
bool prof_active();   // kernel-class timing is recording
void prof_stop(int token, cudaStream_t st, int kernels);

// Records the launches of one launcher function; `kernels` counts the CUDA
// kernels and memsets it issued (set before the scope ends).
struct ProfScope {
  int token;
  cudaStream_t st;
  int kernels = 0;
  ProfScope(int cls, cudaStream_t s) : token(prof_start(cls, s)), st(s) {}
  ~ProfScope() { prof_stop(token, st, kernels); }
};

// Workspace of the synthesis-dictionary calls (dict.cu), created on first use
// and owned by the plan: the certificate on every coefficient, membership
// marks, selection block counts, the mu image, and two working sets (support /
// active set) of indices, weights, b, Gram (ld = capacity rounded to 4) and
// columns of Phi Psi (capacity x M complex64).
struct DictWork {
  DevBuf eta, mark, sel, img, tmpC, oldpos, newrows, keep, acc;
  DevBuf idx[2], th[2], b[2], G[2], C[2];
  int64_t n_atoms = 0;
  int cap = 0;
  void release() {
    for (DevBuf* d : {&eta, &mark, &sel, &img, &tmpC, &oldpos, &newrows, &keep, &acc}) d->release();
    for (int s = 0; s < 2; ++s)
      for (DevBuf* d : {&idx[s], &th[s], &b[s], &G[s], &C[s]}) d->release();
  }
};

// Per-plan resources of the solver loop, created by the first solve on the
// plan and kept until it is destroyed: the pinned readback buffer, the
// completion event, a private stream for callers on the legacy default
// stream, and the instantiated graph of the iteration chain together with the
// arguments it was captured for (a later solve with the same arguments
// launches it without capturing again).
struct SolveCache {
  void* rb = nullptr;
  cudaEvent_t ev = nullptr;
  cudaStream_t own = nullptr;
  cudaGraphExec_t gexec = nullptr;
  std::vector<uint64_t> key;
  void release() {
    if (gexec) cudaGraphExecDestroy(gexec);
    stream_put(own);
    if (ev) cudaEventDestroy(ev);
    pinned_put(rb);
    gexec = nullptr;
    own = nullptr;
    ev = nullptr;
    rb = nullptr;
  }
};

// ------------------------------------------------------------------ constants

constexpr int kMaxW = 8;              // largest supported ES kernel width
constexpr int kGlNodes = 48;          // Gauss-Legendre nodes on [0, 1] for the ES transform

// Exponential-of-semicircle kernel phi(z) = exp(beta (sqrt(1 - z^2) - 1)) on |z| <= 1
// (Barnett, Magland & af Klinteberg 2019). z is clamped into the support.
__device__ __forceinline__ float es_kernel(float z, float beta) {
  float q = fmaxf(1.0f - z * z, 0.0f);
  return expf(beta * (sqrtf(q) - 1.0f));
}

// Phase of visibility k at atom s, in turns, reduced to [-1/2, 1/2]:
//   theta = i' U_k + j' V_k + w_k (n_s - 1)
// i' U + j' V is formed exactly in 32-bit fixed-point turns (wrapping
// arithmetic is exact reduction mod 1), the w-term as a double-float product.
// vis = {U_fx, V_fx, w_hi, w_lo}; atom = {packed (i',j'), s_hi, s_lo, scale}.
__device__ __forceinline__ float phase_turns(int4 vis, float4 atom) {
  int packed = __float_as_int(atom.x);
  int ip = packed >> 16;                       // arithmetic shift: signed i'
  int jp = (int)(short)(packed & 0xffff);      // signed j'
  unsigned th = (unsigned)ip * (unsigned)vis.x + (unsigned)jp * (unsigned)vis.y;
  float t_lm = (float)(int)th * 2.3283064365386963e-10f;   // 2^-32
  float w_hi = __int_as_float(vis.z), w_lo = __int_as_float(vis.w);
  float p = w_hi * atom.y;
  float e = fmaf(w_hi, atom.y, -p);
  e = fmaf(w_hi, atom.z, e);
  e = fmaf(w_lo, atom.y, e);
  float t = t_lm + (p - rintf(p)) + e;
  return t - rintf(t);
}

// Atom of pixel p (raster index, clamped to the image) with weight x (1 when
// no weight): packed signed offsets i' = i - N/2, j' = j - N/2 (16 bits each),
// s = n - 1 as a double-float pair, and x / n -- what the phase kernels read.
__device__ __forceinline__ float4 make_atom(int p, float x, bool weighted, int N, double dl) {
  p = min(max(p, 0), N * N - 1);
  const int i = p / N, j = p - (p / N) * N;
  const int ip = i - N / 2, jp = j - N / 2;
  const double l = ip * dl, m = jp * dl;
  const double r2 = l * l + m * m;
  const double n = sqrt(1.0 - r2);
  const double sv = -r2 / (1.0 + n);
  const float s_hi = (float)sv;
  const float s_lo = (float)(sv - (double)s_hi);
  const double w = weighted ? (double)x : 1.0;
  const int packed = (int)(((unsigned)ip << 16) | ((unsigned)jp & 0xffffu));
  return make_float4(__int_as_float(packed), s_hi, s_lo, (float)(w / n));
}

// Order-preserving map of a float onto unsigned (atomicMax of signed values):
// non-negative floats get the sign bit set, negative ones are inverted.
__host__ __device__ __forceinline__ unsigned float_order_key(float f) {
#ifdef __CUDA_ARCH__
  const unsigned u = __float_as_uint(f);
#else
  unsigned u;
  std::memcpy(&u, &f, sizeof(u));
#endif
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// ------------------------------------------------------------------ kernels (host launchers)

// sparse.cu
// S_dev (optional): the count is read on the device, S is its upper bound
int launch_make_atoms(const int32_t* idx, const float* x, int S, int N, double dl, float4* atoms,
                      cudaStream_t st, const int32_t* S_dev = nullptr);
int launch_residual(const int4* vis_fx, const float2* V, int64_t M, const float4* atoms, int S,
                    float2* out, double* sumsq, cudaStream_t st, const int32_t* S_dev = nullptr);
int launch_gram(const int4* vis_fx, const float2* V, int64_t M, const float4* atomsA, int nA,
                const float4* atomsB, int nB, bool with_v, double* acc, int ldacc,
                cudaStream_t st, bool clear = true);
// gram_tc.cu: tensor-core rows of the Gram (acc cleared by the caller)
struct DevBuf;
int launch_gram_tc(const int4* vis_fx, const float2* V, int64_t M, const float4* atoms, int n_atoms,
                   int nA, double* acc, int ldacc, int* err_dev, cudaStream_t st, bool withhold,
                   DevBuf& pbuf, float* vscale_dev, unsigned* vbits_dev);
int launch_gram_finalize(const double* acc, int ldacc, const int32_t* rows, int nrows, int ncols,
                         const int32_t* oldpos, float* G, int ldg, cudaStream_t st);
// thin contraction: rows = nA atoms (+ the V row when V != null), see sparse.cu
int launch_gram_thin(const int4* vis_fx, const float2* V, int64_t M, const float4* atomsA, int nA,
                     const float4* atomsB, int nB, double* acc, int ldacc, double* b64,
                     cudaStream_t st);
int launch_d2f(const double* in, int n, float* out, cudaStream_t st);
int launch_gram_finalize_perm(const double* acc, int ldacc, int n_new, int n_act, const int32_t* perm,
                              float* G, int ldg, float* b, cudaStream_t st);
int make_atoms_checked(const int32_t* idx, const float* x, int S, int N, double dl,
                       float4* atoms, int* dflag, cudaStream_t st);

// select.cu
// thr_dev (optional): the threshold is read on the device
// candidates examined per selection block; block_counts needs ceil(npix / kSelItems) + 2 entries
constexpr int kSelItems = 1024;
int launch_select(const float* mu, int64_t npix, float thr, const uint8_t* mark, int32_t* out,
                  int32_t* count_dev, int32_t* block_counts, int cap, cudaStream_t st,
                  bool positive = false, const float* thr_dev = nullptr);
// n_dev (optional): the count is read on the device, n is its upper bound
int launch_mark(uint8_t* mark, const int32_t* idx, int n, uint8_t value, cudaStream_t st,
                const int32_t* n_dev = nullptr);
int launch_old_positions(const int32_t* newidx, int n_new, const int32_t* oldidx, int n_old,
                         int32_t* oldpos, cudaStream_t st);
int launch_compact_nonzero(const float* x, int n, int32_t* keep, int32_t* count_dev,
                           cudaStream_t st);
int launch_compact_new(const int32_t* oldpos, int n, int32_t* rows, int32_t* count_dev,
                       cudaStream_t st);
int launch_compact_old(const int32_t* oldpos, int n, int32_t* rows, int32_t* count_dev,
                       cudaStream_t st);

// apgd.cu
// One restricted LASSO for the batched APGD (run_apgd_jobs): several jobs in one launch.
struct ApgdJob {
  const float* G;
  int ldg;
  const float* b;
  int n;
  double lambda, eps;
  int max_iter;
  float* x;
  int* iters;
  double* L;
  double* F;
  int* lanczos;
  int* err;
  bool positive;
};
int run_apgd_jobs(const ApgdJob* jobs, int n_jobs, cudaStream_t st);
int run_apgd(const float* G, int ldg, const float* b, int S, double lambda, double eps,
             int max_iter, float* x, int* iters, double* L, double* Fx, cudaStream_t st,
             int* lanczos = nullptr, int* err = nullptr, bool positive = false);

// grid.cu / fft.cu
int launch_grid(pc_plan_s* p, const float2* r, cudaStream_t st);
// plan.cu: upper estimate of a plan's device bytes (with its solve), for admission by memory
int64_t plan_bytes_estimate(int64_t M, int N, double fov, double w_min, double w_max, int W = 7);
// grid_tc.cu: tensor-core gridding (w-stacking plans); err_dev set to 1 if a bounded wait expired
int launch_grid_tc(pc_plan_s* p, const float2* h, int* err_dev, cudaStream_t st);
// grid_win.cu: CUDA-core gridding over plane windows, one CTA per tile (or
// part of a heavy tile); w-stacking plans
int launch_grid_win(pc_plan_s* p, const float2* h, cudaStream_t st);
bool grid_win_mode(const pc_plan_s* p);   // the plan grids (and degrids) over plane windows
// degrid_win.cu: degridding interpolation over plane windows, one thread per
// slot (y added to)
int launch_degrid_win(pc_plan_s* p, float2* y, cudaStream_t st);
// plan.cu: window gridding CTAs for at most `cap` slots each
int split_wsubs(pc_plan_s* p, int cap, cudaStream_t st);
int split_dwsubs(pc_plan_s* p, int cap, cudaStream_t st);
int launch_fft_rows(pc_plan_s* p, cudaStream_t st);
int launch_fft_cols_epilogue(pc_plan_s* p, float* mu, float scale, unsigned* maxbits,
                             cudaStream_t st);
int cols_planes_per_pass(const pc_plan_s* p);
bool fft_rows_warp(const pc_plan_s* p);   // the first pass runs the one-warp register FFT
bool fft_cols_warp(const pc_plan_s* p);   // the second pass does
// fft_big.cu: one-CTA FFT passes for G = 2048, 4096, 8192 (compact pass-1 rows)
bool fft_big_size(int G);
bool fft_rows_big(const pc_plan_s* p);
bool fft_cols_big(const pc_plan_s* p);
int launch_fft_rows_big(pc_plan_s* p, cudaStream_t st);
int launch_fft_cols_big(pc_plan_s* p, float* mu, float scale, unsigned* maxbits, cudaStream_t st);
int launch_degrid_ffts_big(pc_plan_s* p, const float* img, cudaStream_t st);
int make_xc_tensor_map(pc_plan_s* p);   // after xc is allocated
// degrid.cu: y = Phi(img) for a dense N x N image (type-2 NUFFT), y cleared first
int forward_grid_impl(pc_plan_s* p, const float* img, float2* y, cudaStream_t st);

}  // namespace pc

// ------------------------------------------------------------------ plan object

struct pc_plan_s {
  int device = 0;
  int64_t M = 0;
  int N = 0;          // image side
  int G = 0;          // oversampled grid side (power of two >= 2N)
  int logG = 0;
  int T = 32;         // gridding tile side
  int nT = 0;         // tiles per side = G / T
  int W = 7;          // ES kernel width
  int P = 1;          // number of w-planes (1: no w-stacking)
  int Qg = 1;         // planes per gridding CTA
  double fov = 0, dl = 0, beta = 0;
  double w0 = 0, dw = 1, s_c = 0, w_min = 0, w_max = 0;
  bool wstack = false;
  int grid_mode = 0;  // 0 auto, 1 CUDA cores, 2 tensor cores, 3 CUDA cores over plane
                      // windows (2 and 3: w-stacking only; else mode 1 runs)
  int grid_piece = 0; // gridding sub-problem size in slots (0: chosen for even waves)
  int fft_R = 0;      // rows per CTA of the first FFT pass (0: 2048 / G)
  int fft_cols_pg = 0; // planes per pass of the second FFT pass (0: default)
  int fft_warp = -1;  // bit 0 / bit 1: first / second FFT pass as one-warp register FFTs
                      // (-1: both wherever G is 512 or 1024, the sizes those kernels take)
  bool tuned = false; // grid_mode / grid_piece / fft_R picked by the plan-time autotuner
  bool want_tune = false; // the autotuner will run (it may pick the Stockham passes)
  double tune_grid_us = 0.0, tune_fft_us = 0.0, tune_fft_cols_us = 0.0, tune_degrid_us = 0.0;
  int Pw = 1;         // plane windows: pairs of plane starts ((P - W) >> 1) + 1 (1 without w-stacking)
  std::vector<int4> sub_ranges;   // (tile, plane group, first slot, end) before splitting
  std::vector<int2> win_tiles;    // (tile, binned slots) of every tile that holds slots
  int win_cap = 0;                // window gridding: slots per CTA before a tile is split
  int n_wsub = 0;
  int dwin_cap = 0;               // window degridding: slots per CTA before a tile is split
  int n_dwsub = 0;
  int64_t wsub_cap = 0;           // capacity of wsubs (parts of at most 64 slots)
  int sub_cap = 0;                // capacity of subs (the finest split)
  int64_t n_slots = 0;
  int n_sub = 0;

  // per visibility
  int4* vis_fx = nullptr;        // {U_fx, V_fx, w_hi, w_lo}
  // binned slots (sorted by tile, plane start)
  int2* slot_vis = nullptr;      // {visibility, (a0 + 64) | (b0 + 64) << 8 | plane_start << 16}
  float4* slot_geom = nullptr;   // {gu - a0, gv - b0, xw - plane_start, tau (turns)}
  int4* subs = nullptr;          // gridding sub-problems {tile, plane group, start, end}
  int* win_off = nullptr;        // first slot of each (tile, plane pair) bin (nT^2 Pw + 1)
  int4* wsubs = nullptr;         // window gridding CTAs {tile, part, parts, slots}, heaviest first
  int4* dwsubs = nullptr;        // window degridding CTAs (the same form, their own split)
  int* active_rows = nullptr;    // grid rows b that visibilities can reach (ascending)
  int n_active_rows = 0;
  // image-domain tables
  float4* pix_tab = nullptr;     // per pixel {Re c d, Im c d, t_hi, t_lo}
  float4* atom_tab = nullptr;    // per pixel its unit-weight atom (make_atom); a weighted
                                 // atom is the entry with .w times the weight
  float2* twiddle = nullptr;     // e^{+2 pi i k / G}
  float2* tw2 = nullptr;         // one-warp FFT twiddles e^{+2 pi i l k1 / G}, [k1 < G/32][l < 32]
  uint32_t row_mask = 0;         // G <= 1024: bit t set if grid rows 32 t .. 32 t + 31 can hold data
  uint32_t col_mask = 0;         // G <= 1024: the same for grid columns
  uint32_t* col_bits = nullptr;  // G / 1024 words: bit g set if grid columns 32 g .. 32 g + 31 can hold data
  int* row_pos = nullptr;        // G entries: compact index of a reachable grid row, else -1
  int n_active_col_groups = 0;   // bits set in col_bits
  float2* tw_in = nullptr;       // G >= 2048: the 512-point one-warp FFT's twiddles [k1 < 16][l < 32]
  float2* tw_big = nullptr;      // G >= 2048: the one-CTA FFT's first-step twiddles [k1 < G / 512][n' < 512]
  // workspaces
  float2* grid = nullptr;        // P x G x G  (b-major rows, a contiguous)
  float2* fft1 = nullptr;        // P x N x G  (after the pass along a)
  float2* resid = nullptr;       // M
  float* mu = nullptr;           // N x N
  uint8_t* mark = nullptr;       // N x N membership marks (kept all-zero between calls)
  double* dscal = nullptr;       // 8 float64 scalars
  unsigned* uscal = nullptr;     // 8 uint scalars
  int32_t* iscal = nullptr;      // 8 int scalars
  int32_t* sel_blocks = nullptr; // per-block counts of the select
  int sel_blocks_n = 0;

  // solver workspace (grown on demand)
  pc::DevBuf atomsA, atomsB, idxA, idxB, xA, xB, oldpos, newrows, keep, GA, GB, bA, bB, acc;
  pc::DevBuf perm, atomsP, pbuf;   // tensor-core Gram: atom order (new first), atoms, phase buffer
  pc::DictWork* dict = nullptr;    // synthesis-dictionary workspace (created on first use)
  pc::SolveCache* scache = nullptr; // solver-loop resources (created by the first solve)
  pc::DevBuf degrid_buf;            // forward on a dense image: P x active rows x N (first pass)
  pc::DevBuf xc;                    // G >= 2048: compact pass-1 rows, P x ceil(rows / 4) x N x 4
  alignas(64) CUtensorMap xmap;     // TMA map over xc (2-D: P ceil(rows / 4) x 8 N floats)
  int xmap_by = 0, xmap_boxes = 0;  // its box height and boxes per plane
  pc::DevBuf opw;                   // operator-form reweighting: images, visibilities, vectors
  pc::DevBuf dirty;                 // operator-form reweighting: Re Phi* V of the solve (N x N)
  double op_pair_s = 0.0;           // measured time of one degridding + gridding pair (0: not yet)
  // While the operator-form reweighting runs, the image rows holding its atoms
  // (list and bit mask, n_img_rows > 0): the one-CTA passes of G >= 2048 then
  // transform only those rows on the image side (the others are not needed).
  const int* img_rows = nullptr;
  const uint32_t* img_row_bits = nullptr;
  int n_img_rows = 0;

  std::vector<void*> owned;      // every cudaMalloc of the plan (freed on destroy)
};
