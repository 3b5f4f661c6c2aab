/*
 * polyclean.h -- C ABI of the GB300 (sm_103a) PolyCLEAN hot path.
 *
 * The library implements, as hand-written CUDA kernels, the operators and the
 * solver loop of PolyCLEAN (Polyatomic Frank-Wolfe for the LASSO imaging
 * problem, Sect. 4.1 and Algorithm 2 of the paper):
 *
 *   Phi  : R^{N x N} -> C^M   Phi(I)[k]  = sum_p I_p / n_p exp(-j2pi(u_k l_p + v_k m_p + w_k (n_p - 1)))
 *                             (the discrete forward equation, Sect. 2.2)
 *   Phi* : C^M -> R^{N x N}   Phi*(h)[p] = Re sum_k h_k / n_p exp(+j2pi(u_k l_p + v_k m_p + w_k (n_p - 1)))
 *                             (the adjoint equation, Sect. 2.2)
 *   mu   = Phi*(V - Phi x) / lambda          (dual certificate, Sect. 4.2)
 *   lambda_max = ||Phi* V||_inf              (Sect. 5.3)
 *   argmin_x 1/2 ||V - Phi x||^2 + lambda ||x||_1 by Polyatomic Frank-Wolfe (Algorithm 2)
 *
 * Conventions shared by every call:
 *   - uvw: float64, M x 3 row-major, in wavelengths.
 *   - Image: N x N float32 row-major; raster index p = i*N + j; i indexes the
 *     direction cosine l and j indexes m, l_i = (i - N/2) fov/N,
 *     m_j = (j - N/2) fov/N (N even), n = sqrt(1 - l^2 - m^2).
 *   - Visibilities: interleaved complex float32 (pc_c32), original order of uvw.
 *   - Sparse images: strictly ascending unique raster indices (int32) plus
 *     float32 weights.
 *   - Every array argument is a DEVICE pointer owned by the caller, unless the
 *     name ends in _host. A host pointer where a device pointer is expected is
 *     rejected with PC_ERR_INVALID_ARG; there is no CPU fallback.
 *   - Every call is ordered on the given CUDA stream (cudaStream_t passed as
 *     void*, NULL = legacy default stream). Calls that return values in host
 *     memory (*_host outputs, pc_solve_stats) synchronise that stream.
 *   - A plan owns its device workspace. Calls on one plan must not overlap
 *     (they share the workspace); use one plan per concurrent stream.
 *   - Return value: PC_OK (0) or a negative pc_status. pc_last_error()
 *     returns a thread-local message describing the last failure.
 */
#ifndef POLYCLEAN_H
#define POLYCLEAN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PC_ABI_VERSION 5

typedef enum {
  PC_OK = 0,
  PC_ERR_INVALID_ARG = -1,   /* bad size, NULL, host pointer, non-finite input      */
  PC_ERR_OOM = -2,           /* device allocation failed; the plan stays valid       */
  PC_ERR_CUDA = -3,          /* a CUDA runtime call failed (message has the text)     */
  PC_ERR_NOT_CONVERGED = -4, /* iteration cap reached; the returned result is valid  */
  PC_ERR_TIMEOUT = -5,       /* a bounded device wait expired                         */
  PC_ERR_NUMERIC = -6,       /* NaN/Inf met in a result                               */
  PC_ERR_CAPACITY = -7       /* support larger than the caller's output capacity     */
} pc_status;

typedef struct { float re, im; } pc_c32;

typedef struct pc_plan_s* pc_plan_t;

/* Plan options. Zero-initialise and set version = PC_ABI_VERSION; a zero field
 * takes its default. */
typedef struct {
  int32_t version;
  int32_t kernel_width;   /* ES kernel width W in grid cells (default 7; 4..8)         */
  int32_t tile;           /* gridding tile side in cells (32, the only supported value) */
  int32_t max_planes;     /* cap on the number of w-planes (default 256)                */
  int32_t grid_mode;      /* gridding: 0 (default) when w-stacking, mode 3 on grids of side
                             >= 2048 (kernel_width <= 7), else tensor cores; CUDA cores
                             without w-stacking. 1: FP32 CUDA cores; 2: tensor cores
                             whenever w-stacking; 3: FP32 CUDA cores over plane windows,
                             one CTA per tile, when w-stacking with kernel_width <= 7
                             (else as 2). The degridding follows: over plane windows in
                             mode 3 (one thread per binned slot), else over the fixed
                             plane groups                                                */
  int32_t autotune;       /* 1: time the candidate gridding kernels, gridding sub-problem
                             sizes and FFT kernels on this plan's visibilities and keep
                             the fastest (adds a few ms to plan creation); 0 (default): off */
  int32_t fft_kernel;     /* FFT passes: 0 (default) one warp per row, in registers, where G
                             is 512 or 1024, else shared-memory Stockham stages; 1: Stockham
                             everywhere. The autotuner, when on, chooses per pass instead. */
} pc_plan_opts;

/* What the plan-time autotuner chose (tuned = 0 when it did not run). */
typedef struct {
  int32_t tuned;
  int32_t grid_mode;        /* 1: CUDA cores, 2: tensor cores, 3: plane windows      */
  int32_t grid_piece;       /* gridding sub-problem size in binned slots (mode 3:
                               slots per CTA before a tile is split into parts)      */
  int32_t fft_rows_per_cta; /* rows per CTA of the first FFT pass                    */
  double  grid_us;          /* measured time of one gridding with that choice        */
  double  fft_rows_us;      /* measured time of one first FFT pass with that choice  */
  int32_t fft_cols_planes;  /* w-planes transformed together by the second FFT pass   */
  int32_t fft_warp;         /* bit 0 / bit 1: the first / second FFT pass gives each row
                               to one warp, which transforms it in registers (G = 512 or
                               1024; 8 rows per CTA in the first pass, one plane per warp
                               in the second)                                           */
  double  fft_cols_us;      /* measured time of one second FFT pass with that choice */
  int32_t degrid_piece;     /* mode 3: slots per degridding CTA before a tile is split
                               into parts (0 in the other modes)                      */
  int32_t reserved;
  double  degrid_us;        /* measured time of one degridding interpolation with that
                               choice (0 when not timed)                              */
} pc_plan_tuning;

/* Solver options (Algorithm 2 and its sub-solver). Zero fields take defaults. */
typedef struct {
  int32_t version;
  int32_t select_rule;    /* 2 (default): |mu| >= 1 - delta;  1: |eta| >= ||eta||_inf - 2 Delta/(k+2) */
  int32_t max_fw;         /* Frank-Wolfe iteration cap (default 100)                                 */
  int32_t apgd_max_iter;  /* sub-solver iteration cap (default 10000)                                */
  int32_t gram_mode;      /* 0 (default): tensor cores for large blocks; 1: FP32 only; 2: tensor cores */
  int32_t positivity;     /* 1: x >= 0 (remark of Sect. 5.1): candidates only where mu >= thr,
                             reweighting with the non-negative proximal map; 0 (default): off */
  double  tol;            /* stop when (F_k - F_{k+1}) / F_k < tol (default 1e-4, Sect. 6.1)          */
  double  eps0;           /* sub-solver accuracy eps_k = max(eps_min, eps0 2^-k) (default 1e-2)       */
  double  eps_min;        /* (default 1e-5)                                                           */
  double  lambda_max;     /* for rule 1: lambda_max if known (<= 0: computed; under positivity the
                             positive lambda_max of pc_lambda_max_positive)                          */
  int32_t reweight;       /* form of the reweighting (step 2 of Algorithm 2): 0 (default) per
                             Frank-Wolfe iteration the cheaper of the Gram form (G_S, b_S contracted,
                             then APGD on them) and the operator form (APGD whose gradient
                             Re Phi_S^H (Phi_S x - V) is evaluated by degridding and gridding every
                             iteration, Sect. 5.1); 1: always the Gram form; 2: always the operator
                             form (same iterations, step size and stop rule)                          */
  int32_t reserved;
  /* Resume / warm start (checkpoint of Algorithm 2: its state at the start of
   * iteration k is (k, S_k, I_k)). init_S > 0: the solve starts from the image
   * with weights init_x on the pixels init_idx (device pointers, init_S entries,
   * strictly ascending raster indices < N*N, finite weights, >= 0 under
   * positivity; read before pc_solve returns, the caller keeps ownership) at
   * iteration init_k (0 <= init_k < max_fw: the eps_k schedule and rule R1's
   * threshold continue from there; the first stop test compares against the
   * objective of the given image). A run resumed from the support and weights
   * an uninterrupted run had after its iteration k - 1, with init_k = k,
   * repeats that run's remaining iterations. init_S = 0 (default): cold start.
   * PC_ERR_INVALID_ARG for an invalid state; pc_solve only (the host, server
   * and synthesis entry points require init_S = 0). */
  const int32_t* init_idx;
  const float*   init_x;
  int32_t init_S;
  int32_t init_k;
} pc_solve_opts;

/* Per-iteration record of pc_solve (host memory). */
typedef struct {
  int32_t k;              /* Frank-Wolfe iteration                                   */
  int32_t n_new;          /* atoms added by the exploration step                     */
  int32_t n_active;       /* |S_k u I_{k+1}| before the reweighting                  */
  int32_t n_support;      /* |S_{k+1}| after pruning                                 */
  int32_t apgd_iterations;
  int32_t lanczos_steps;  /* Lanczos steps of the step-size estimate                */
  double  mu_inf;         /* ||mu_k||_inf (eta_k / lambda) at the start of iteration k;
                             max mu_k under positivity                              */
  double  objective;      /* F(I_{k+1})                                              */
  double  rel_improvement;
  double  lipschitz;
} pc_iter_record;

typedef struct {
  int32_t status;         /* PC_OK or PC_ERR_NOT_CONVERGED                          */
  int32_t iterations;     /* Frank-Wolfe iterations run                             */
  int32_t n_support;      /* entries written to idx_out / x_out                     */
  int32_t n_history;      /* records written to history (<= history_capacity)       */
  double  objective;      /* final F                                                */
  double  lambda;         /* lambda used                                            */
  double  mu_inf;         /* ||mu||_inf of the final certificate                    */
  double  sumsq_V;        /* ||V||^2                                                */
} pc_solve_stats;

/* ------------------------------------------------------------------ plan */

/* Build a plan for M visibilities (uvw_dev, M x 3 float64) and an N x N image
 * with full field-of-view side fov_rad (direction cosine units). Sorts and bins
 * the visibilities by (gridding tile, w-plane), precomputes the kernel
 * corrections and allocates the gridding / FFT workspace (the plan owns it).
 * Sect. 2.2 (pixel grid, operators) and Sect. 5.2 (the operator is evaluated
 * with a non-uniform FFT: here exponential-of-semicircle gridding on a 2x
 * oversampled grid with w-stacking). N must be even, 16 <= N <= 4096.
 * M may be 0 (all operators then return zeros). */
int pc_plan_create(const double* uvw_dev, int64_t M, int32_t N, double fov_rad,
                   const pc_plan_opts* opts, void* stream, pc_plan_t* plan_out);
/* The same call under the short name of the problem statement (plan of the
 * measurement operator for uvw, M, N_pix, fov): identical arguments and
 * behaviour. */
int pc_plan(const double* uvw_dev, int64_t M, int32_t N, double fov_rad, const pc_plan_opts* opts,
            void* stream, pc_plan_t* plan_out);
void pc_plan_destroy(pc_plan_t plan);

/* Plan geometry: oversampled grid side, tile side, number of w-planes, number
 * of binned (replicated) visibility slots, kernel width. Any pointer may be NULL. */
int pc_plan_info(pc_plan_t plan, int32_t* grid_side, int32_t* tile, int32_t* n_planes,
                 int64_t* n_slots, int32_t* kernel_width, double* dw);
int pc_plan_tuning_info(pc_plan_t plan, pc_plan_tuning* out_host);
/* The part of each w-plane's grid that visibilities can reach (the gridding,
 * the FFT's first pass and the degridding touch nothing else): the number of
 * reachable grid rows and of reachable 32-column groups. Either pointer may
 * be NULL. */
int pc_plan_reach(pc_plan_t plan, int32_t* rows, int32_t* col_groups);

/* ------------------------------------------------------------------ operators */

/* y = Phi restricted to the support: y[k] = sum_s x[s]/n_s exp(-j2pi theta_ks),
 * direct sum over the support (the forward equation of Sect. 2.2 for a sparse
 * image; the paper evaluates it as a type-3 NUFFT, Sect. 5.2).
 * idx_dev: S ascending raster indices; x_dev: S weights; y_dev: M outputs. */
int pc_forward_sparse(pc_plan_t plan, const int32_t* idx_dev, const float* x_dev, int32_t S,
                      pc_c32* y_dev, void* stream);

/* out[s] = Phi*(y)[idx[s]]: the adjoint restricted to S pixels, direct sum. */
int pc_adjoint_sparse(pc_plan_t plan, const pc_c32* y_dev, const int32_t* idx_dev, int32_t S,
                      float* out_dev, void* stream);

/* img = Phi*(y) on all N x N pixels (the adjoint equation of Sect. 2.2), by
 * gridding on the oversampled grid, w-stacking, 2-D inverse FFT and kernel
 * correction. With y = V this is the dirty image. img_dev: N*N floats. */
int pc_adjoint_grid(pc_plan_t plan, const pc_c32* y_dev, float* img_dev, void* stream);

/* y = Phi(img) for a dense N x N image (the forward equation of Sect. 2.2), by
 * degridding (Sect. 5.2: the type-2 half of the non-uniform FFT): the exact
 * adjoint of pc_adjoint_grid's steps in reverse -- per-pixel correction and
 * w-screen, two forward FFT passes per w-plane, interpolation of the binned
 * visibilities with the same kernel. Cost independent of how many pixels are
 * nonzero (use it instead of pc_forward_sparse for dense or extended images).
 * img_dev: N*N floats; y_dev: M complex (overwritten, original order of uvw).
 * Uses the plan's grid workspace: not concurrent with other calls on the plan. */
int pc_forward_grid(pc_plan_t plan, const float* img_dev, pc_c32* y_dev, void* stream);

/* lambda_max = ||Phi* V||_inf (Sect. 5.3), returned in host memory. */
int pc_lambda_max(pc_plan_t plan, const pc_c32* V_dev, double* lambda_max_host, void* stream);

/* max(0, max_p Phi*(V)_p): the smallest lambda for which x = 0 is optimal under
 * the positivity constraint (remark of Sect. 5.1; lambda = alpha times it),
 * returned in host memory. */
int pc_lambda_max_positive(pc_plan_t plan, const pc_c32* V_dev, double* lambda_max_host,
                           void* stream);

/* mu = Phi*(V - Phi x) / lambda (Sect. 4.2), x given on a support of S pixels.
 * mu_dev: N*N floats. mu_inf_host (may be NULL): ||mu||_inf. sumsq_host (may
 * be NULL): ||V - Phi x||^2 accumulated in float64. */
int pc_certificate(pc_plan_t plan, const pc_c32* V_dev, const int32_t* idx_dev,
                   const float* x_dev, int32_t S, double lambda, float* mu_dev,
                   double* mu_inf_host, double* sumsq_host, void* stream);

/* ------------------------------------------------------------------ hot-path steps */

/* Exploration + union (Algorithm 2, steps 1a/1b). From a certificate mu (N*N)
 * select I = {p : |mu_p| >= thr} and write the ascending union of I with the
 * support prev_idx (n_prev entries, ascending) to out_idx (capacity cap).
 * *n_out_host receives |S u I|. PC_ERR_CAPACITY if it exceeds cap (nothing
 * else is written then). */
int pc_select(pc_plan_t plan, const float* mu_dev, float thr, const int32_t* prev_idx_dev,
              int32_t n_prev, int32_t* out_idx_dev, int32_t cap, int32_t* n_out_host,
              void* stream);

/* Support contraction (step 2 of Algorithm 2, in Gram form): for the S atoms
 * idx, G = Re(Phi_S^H Phi_S) (S x S, row-major, leading dimension ldg) and
 * b = Re(Phi_S^H V) (S; skipped when V_dev is NULL). mode 1: FP32 CUDA-core
 * products, phases generated per tile in shared memory; mode 2: tcgen05
 * tensor cores on split-FP16 (hi + lo) operands with FP32 accumulation
 * (hi*hi + hi*lo + lo*hi), the phases of each chunk of visibilities (at most
 * ~2 GB of FP16 pairs) written once to a plan-owned buffer in HBM and streamed
 * into the MMA pipeline from L2; mode 0: tensor cores when S*S >= 4096.
 * Both accumulate K-slices in float64. PC_ERR_TIMEOUT if a bounded
 * tensor-core wait expired. mode 3 is a self-test of that path: the tensor-core
 * kernel withholds its MMAs, its first buffer wait expires after about 2 s and
 * the call returns PC_ERR_TIMEOUT with the CUDA context intact. */
int pc_gram(pc_plan_t plan, const pc_c32* V_dev, const int32_t* idx_dev, int32_t S,
            float* G_dev, int32_t ldg, float* b_dev, int32_t mode, void* stream);

/* Restricted LASSO by monotone FISTA on the Gram form (Sect. 4.4 / 4.1):
 * min_x 1/2 x^T G x - b^T x + lambda ||x||_1, warm start x_dev (in/out),
 * step 1/L with L = 1.01 x the top eigenvalue of G (Lanczos, ~1e-6 relative),
 * stop when ||z - y|| <= eps ||z|| or after max_iter iterations. Synchronises
 * the stream. iters_host / lipschitz_host (may be NULL) receive the iteration
 * count and L. positive = 1 adds the constraint x >= 0 (proximal map
 * max(z - lambda/L, 0); the positivity remark of Sect. 5.1). PC_ERR_TIMEOUT if
 * a bounded wait between the CTAs of the solver's thread-block cluster expired
 * (x_dev is then unchanged). */
int pc_apgd(const float* G_dev, int32_t ldg, const float* b_dev, int32_t S, double lambda,
            double eps, int32_t max_iter, int32_t positive, float* x_dev, int32_t* iters_host,
            double* lipschitz_host, void* stream);

/* ------------------------------------------------------------------ solver */

/* PolyCLEAN solve (Algorithm 2): argmin_x 1/2||V - Phi x||^2 + lambda||x||_1.
 * Writes the support (ascending raster indices) and weights to idx_out_dev /
 * x_out_dev (capacity cap), the final certificate to mu_out_dev (N*N, may be
 * NULL), statistics to *stats_host and up to history_capacity iteration
 * records to history_host (may be NULL). delta is the exploration parameter
 * (rule 2: atoms with |mu| >= 1 - delta; rule 1: quality of Algorithm 2).
 * Returns PC_OK, PC_ERR_NOT_CONVERGED (result valid) or an error. */
int pc_solve(pc_plan_t plan, const pc_c32* V_dev, double lambda, double delta,
             const pc_solve_opts* opts, int32_t* idx_out_dev, float* x_out_dev, int32_t cap,
             float* mu_out_dev, pc_solve_stats* stats_host, pc_iter_record* history_host,
             int32_t history_capacity, void* stream);

/* End-to-end call on HOST buffers: copies uvw (M x 3 float64) and V (M
 * complex) to the device, builds a plan, solves with lambda = alpha *
 * lambda_max (the positive lambda_max of pc_lambda_max_positive when
 * opts->positivity is set), copies the support and weights back (capacity
 * cap), frees everything. The host buffers may be pageable or pinned. */
int pc_solve_host(const double* uvw_host, const pc_c32* V_host, int64_t M, int32_t N,
                  double fov_rad, double alpha, double delta, const pc_solve_opts* opts,
                  int32_t* idx_out_host, float* x_out_host, int32_t cap,
                  pc_solve_stats* stats_host, void* stream);

/* ------------------------------------------------------------------ synthesis dictionary */

/* Multi-scale synthesis dictionary Psi (Sect. 4.3; the diffuse experiment of
 * Sect. 6 uses sigma = {0, 2, 5, 8}, gamma_i = 1.2^i). The image is
 * I = Psi theta = sum_i gamma_i g~_i * theta_i with g~_i[n, m] proportional to
 * exp(-(n^2 + m^2) / sigma_i^2) on the square |n|, |m| <= floor(2 sigma_i),
 * unit l1 norm; sigma = 0 is the single-pixel (point-source) atom. Each
 * kernel is centred on its coefficient's pixel and what falls outside the
 * N x N image is dropped (no renormalisation at the border); Psi* is the
 * matching correlation over the image. Coefficients are indexed
 * a = i * N*N + p (scale-major, p the raster pixel), n_scales * N*N of them.
 * Constraints: 1 <= n_scales <= PC_DICT_MAX_SCALES, 0 <= sigma_i with
 * floor(2 sigma_i) <= PC_DICT_MAX_RADIUS, gamma_i > 0 and finite. */
#define PC_DICT_MAX_SCALES 8
#define PC_DICT_MAX_RADIUS 16
typedef struct {
  int32_t version;        /* PC_ABI_VERSION                                      */
  int32_t n_scales;
  double  sigma[PC_DICT_MAX_SCALES];
  double  gamma[PC_DICT_MAX_SCALES];
} pc_dictionary;

/* eta_out[a] = scale * (Psi* Phi* h)[a] for every coefficient
 * (n_scales * N*N float32, scale-major). Sect. 4.3 with the adjoint of Sect. 2.2.
 * Asynchronous on the stream. */
int pc_dict_adjoint(pc_plan_t plan, const pc_dictionary* dict, const pc_c32* h_dev, double scale,
                    float* eta_out_dev, void* stream);

/* y_out = Phi Psi theta for S coefficients (idx_dev: strictly ascending in
 * [0, n_scales N*N); theta_dev float32): each column of Phi Psi is evaluated
 * as the direct sum of the measurement operator over the atom's footprint
 * pixels, weighted gamma_i g~_i. Returns PC_ERR_INVALID_ARG for a bad index
 * list (synchronises the stream to check it). */
int pc_dict_forward_sparse(pc_plan_t plan, const pc_dictionary* dict, const int32_t* idx_dev,
                           const float* theta_dev, int32_t S, pc_c32* y_out_dev, void* stream);

/* lambda_max of the synthesis problem: ||Psi* Phi* V||_inf, or with positive
 * != 0 max(0, max Psi* Phi* V) (the smallest lambda with theta = 0 optimal;
 * the paper takes lambda_max with Psi). Synchronises the stream. */
int pc_dict_lambda_max(pc_plan_t plan, const pc_dictionary* dict, const pc_c32* V_dev,
                       int32_t positive, double* lambda_max_host, void* stream);

/* Synthesis-form solve (Sect. 4.3 with Algorithm 2):
 * argmin_theta 1/2 ||V - Phi Psi theta||^2 + lambda ||theta||_1 (theta >= 0 with
 * opts->positivity). Same options, statistics and history as pc_solve, over
 * the coefficient atoms (rule 2 selects |eta| >= 1 - delta with
 * eta = Psi* Phi* r / lambda). The diffuse experiment stops at tol = 1e-5.
 * Writes the support (ascending coefficient indices) and coefficients to
 * idx_out_dev / theta_out_dev (capacity cap) and, when eta_out_dev is not
 * NULL, the final certificate (n_scales N*N float32). The columns of Phi Psi
 * on the active set are kept on the device (M x |S| complex64), so the
 * working set is limited by device memory (PC_ERR_CAPACITY beyond 60000 atoms). */
int pc_solve_synthesis(pc_plan_t plan, const pc_dictionary* dict, const pc_c32* V_dev,
                       double lambda, double delta, const pc_solve_opts* opts,
                       int32_t* idx_out_dev, float* theta_out_dev, int32_t cap, float* eta_out_dev,
                       pc_solve_stats* stats_host, pc_iter_record* history_host,
                       int32_t history_capacity, void* stream);

/* ------------------------------------------------------------------ allocation-free variant */

/* The paper has no counterpart of this call; it exists for callers that
 * cannot allocate device memory: code that runs inside an arena which handed
 * out all its memory at start-up, real-time pipelines with a fixed memory
 * budget, or hosts that forbid allocation while work is queued. Building a
 * plan allocates, so this variant of pc_adjoint_sparse takes the raw uvw
 * array (M x 3 float64, device) and the geometry (N, fov_rad) instead:
 * out[s] = Phi*(y)[idx[s]] for S pixels (direct sum, same phases as the plan
 * path). The caller passes every input and output; the only scratch is a
 * file-scope __device__ array of PC_NOALLOC_MAX_PIXELS float64 accumulators
 * (64 KB per device that loads the library, held until the process exits).
 * The call never allocates or frees device memory once the library's module
 * is resident on the device. S > PC_NOALLOC_MAX_PIXELS or M >
 * PC_NOALLOC_MAX_VIS is rejected with PC_ERR_INVALID_ARG. An index outside
 * [0, N*N) gives NaN in its output slot (no ordering is required). All
 * calls share the scratch array and each clears the part it uses: calls
 * whose kernels overlap on the GPU race on it and must be serialised. The
 * first call on a device looks up the array's address (cudaGetSymbolAddress,
 * that device current); under lazy module loading, the CUDA default, that
 * first call also loads the kernels and the 64 KB array, which takes device
 * memory then. Make the first call at start-up, before an arena or budget
 * takes the device's memory and before any stream capture. */
#define PC_NOALLOC_MAX_PIXELS 8192
#define PC_NOALLOC_MAX_VIS (65535LL * 8192LL)
int pc_adjoint_sparse_noalloc(const double* uvw_dev, int64_t M, int32_t N, double fov_rad,
                              const pc_c32* y_dev, const int32_t* idx_dev, int32_t S,
                              float* out_dev, void* stream);

/* ------------------------------------------------------------------ serving loop
 *
 * Continuous batching of imaging requests (each one the solve of
 * pc_solve_host: plan, lambda = alpha lambda_max, Algorithm 2). The paper
 * names parallel processing as future work (Sect. 7); this loop serves many
 * requests of different grid and visibility sizes on one GPU. A scheduler
 * thread admits queued requests while fewer than max_jobs are active and their
 * estimated device bytes fit the memory budget, keeps each job's plan,
 * binned visibilities and support on the device, advances every active job on
 * its own stream (their kernels overlap on the GPU) and launches the
 * reweightings (APGD) of all jobs that reach that step together, several
 * jobs per launch. Requests that arrive while others run are admitted as slots
 * and memory free up. */

typedef struct pc_server_s* pc_server_t;

typedef struct {
  int32_t version;          /* PC_ABI_VERSION                                              */
  int32_t max_jobs;         /* concurrently active jobs (default 8)                        */
  int64_t memory_budget;    /* device bytes for active jobs (<= 0: half the free memory)    */
  int32_t batch_apgd;       /* 1 (default): one launch for all ready reweightings; 2: one per job */
  int32_t reserved;
} pc_server_opts;

/* Per-request timing on the server's steady clock (seconds since its creation). */
typedef struct {
  double submitted;         /* pc_server_submit returned                                   */
  double admitted;          /* inputs on the device, plan building starts                  */
  double finished;          /* result ready (latency = finished - submitted)               */
} pc_job_times;

int pc_server_create(const pc_server_opts* opts, pc_server_t* server_out);
/* Queues one request; the host inputs are copied (the caller may free them on
 * return). uvw: M x 3 float64 wavelengths, V: M complex64; alpha in (0, 1],
 * delta in (0, 1]; opts as pc_solve (NULL = defaults). *job_id_out > 0. */
int pc_server_submit(pc_server_t server, const double* uvw_host, const pc_c32* V_host, int64_t M,
                     int32_t N, double fov_rad, double alpha, double delta,
                     const pc_solve_opts* opts, int64_t* job_id_out);
/* Blocks until the job is done; copies its support and weights (host, up to
 * cap) and statistics, releases the job and returns its status (as pc_solve;
 * PC_ERR_INVALID_ARG for an unknown or already collected job). times may be NULL. */
int pc_server_wait(pc_server_t server, int64_t job_id, int32_t* idx_out_host, float* x_out_host,
                   int32_t cap, pc_solve_stats* stats_host, pc_job_times* times_host);
/* Finishes every queued and active job, then frees the server. */
void pc_server_destroy(pc_server_t server);

/* ------------------------------------------------------------------ profiling */

/* Per-kernel-class timing with CUDA events recorded on the launching stream.
 * pc_profile_begin() clears the records and starts recording every kernel
 * launch of the library; pc_profile_end() synchronises on the recorded
 * events, stops recording and writes one entry per kernel class (at most
 * cap entries; *n_out receives the number of classes seen). Recording costs
 * two event records per launch; it is off unless begun. Not thread-safe.
 * The forward operator by degridding records two classes: "degrid_fft" (its
 * two FFT passes, image to grid planes) and "degrid" (the interpolation). */
typedef struct {
  char name[32];          /* kernel class, e.g. "grid", "fft_rows", "apgd"        */
  int64_t launches;       /* timed launcher calls of this class                    */
  int64_t kernels;        /* CUDA kernels (and memsets) those calls launched       */
  double total_ms;        /* sum of event-measured launch durations              */
} pc_kernel_time;

int pc_profile_begin(void);
/* As pc_profile_begin, recording only the comma-separated classes named in
 * `classes` (e.g. "gram_tc"; NULL or "" = all); PC_ERR_INVALID_ARG for an
 * unknown name. Recording one class costs two event records per launch of
 * that class only. */
int pc_profile_begin_classes(const char* classes);
int pc_profile_end(pc_kernel_time* out_host, int32_t cap, int32_t* n_out_host);

/* ------------------------------------------------------------------ misc */

const char* pc_last_error(void);
int pc_abi_version(void);

/* Device memory the library allocates (plans, solver working sets, the
 * server's per-request buffers) comes from a stream-ordered pool per device
 * that keeps freed memory for reuse, so repeated plans and solves do not pay
 * for cudaMalloc / cudaFree; pinned host blocks and streams are recycled the
 * same way. pc_trim_memory waits for the device, then returns every cached
 * block that no plan or server holds to the system. PC_ERR_CUDA reports an
 * earlier asynchronous error. */
int pc_trim_memory(void);

#ifdef __cplusplus
}
#endif

#endif /* POLYCLEAN_H */
