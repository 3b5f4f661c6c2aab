// The Frank-Wolfe solve of one plan as a resumable job (Algorithm 2 with the
// reweighting of Sect. 5.1): each iteration is queued on the job's stream up
// to one readback of the host-side decisions (objective, certificate maxima,
// active-set size, flags) into pinned memory, marked by an event; after the
// host processes it the job either finishes or queues the Gram update and
// then needs its reweighting (APGD), which the caller launches -- alone
// (pc_solve) or batched with other jobs in one launch (the serving loop) --
// before queueing the next iteration.
#pragma once

#include "pc_internal.cuh"

#include <nvtx3/nvToolsExt.h>

namespace pc {

inline cudaStream_t SS(void* s) { return static_cast<cudaStream_t>(s); }

// Shared by the solve entry points (solve.cu, dict.cu):
// mu-image = scale * Phi*(h) on every pixel (gridding, FFT, epilogue), with the
// max |.| and the signed max as order keys in maxbits[0..1]
int adjoint_grid_impl(pc_plan_s* p, const float2* h, float* img, float scale, unsigned* maxbits,
                      cudaStream_t st);
int check_plan(pc_plan_s* p, const char* fn);
int check_dev(const void* ptr, bool needed, const char* fn, const char* name);
// synchronises st and reports an expired bounded wait of the tensor-core gridding
int grid_flag_sync(pc_plan_s* p, cudaStream_t st, const char* fn);
float bits_to_float(unsigned b);
float key_to_float(unsigned key);   // inverse of float_order_key (0 -> -infinity)

struct SolveCfg {
  int rule = 2, max_fw = 100, apgd_max = 10000, gram_mode = 0, positive = 0, reweight = 0;
  double tol = 1e-4, eps0 = 1e-2, eps_min = 1e-5, lmax = 0.0;
  // resume from (init_k, init_idx, init_x) when init_S > 0 (device arrays)
  const int32_t* init_idx = nullptr;
  const float* init_x = nullptr;
  int init_S = 0, init_k = 0;
};

// Validates and reads pc_solve_opts (NULL = defaults); resume_ok: the entry
// point accepts a resume state (else init_S must be 0).
int parse_solve_opts(const pc_solve_opts* opts, const char* fn, SolveCfg* out, bool resume_ok = false);

// reweight_op.cu: the reweighting in operator form (monotone FISTA on
// g(v) = Re Phi_S^H (Phi_S v - V), one degridding + gridding pair per step)
// on the n atoms idx (raster order), warm start and result in x; iterations,
// step size and Lanczos steps written to the device scalars given.
// dirty (N x N, may be null): Re Phi* V, whose values at idx start Lanczos.
int run_operator_apgd(pc_plan_s* p, const float2* V, const float* dirty, const int32_t* idx, int n,
                      double lambda, double eps, int max_iter, bool positive, float* x, int* iters_dev,
                      double* L_dev, int* lz_dev, cudaStream_t st);
// Measured seconds of one degridding + gridding pair on this plan (cached).
int op_pair_seconds(pc_plan_s* p, cudaStream_t st, double* out);

struct SolveJob {
  // ---- inputs
  pc_plan_s* p = nullptr;
  cudaStream_t st = nullptr;
  const float2* V = nullptr;
  double lambda = 0.0, delta = 0.0;
  SolveCfg c;
  float* mu_dst = nullptr;             // certificate of the iterate (the final one at the end)
  pc_iter_record* hist = nullptr;
  int hist_cap = 0;

  // ---- state
  int wcap = 1024;                      // working-set capacity (grown on demand)
  int k = 0, nS = 0, ldA = 4, n_prev_act = 0, ldB_prev = 4, n_hist = 0;
  int status = PC_ERR_NOT_CONVERGED;
  bool done = false;
  double F_prev = 0.0, F = 0.0, sumsqV = 0.0, mu_inf = 0.0;
  pc_iter_record cur{};
  bool have_cur = false;

  // the reweighting this iteration needs (valid when need_apgd); op_form:
  // it runs in operator form (run_apgd_op), else on the Gram form (apgd_job)
  bool need_apgd = false;
  bool op_form = false;
  bool gram_valid = true;               // GA holds G of the support (false after an operator-form step)
  bool dirty_ready = false;             // the plan's dirty image holds Re Phi* V of this solve
  bool warm = false;                    // the queued chain starts from the resume state (no pruning)
  // NVTX range of the current Frank-Wolfe iteration (from queueing its chain
  // to queueing the next one, or to the end of the solve); free when no tool
  // is attached
  nvtxRangeId_t fw_range = 0;
  bool fw_range_open = false;
  void end_fw_range() {
    if (fw_range_open) nvtxRangeEnd(fw_range);
    fw_range_open = false;
  }
  int last_apgd_iters = 0;
  int n_act = 0, ldB = 4;
  double eps = 0.0;

  // host readback of an iteration (pinned) and its completion event
  struct Readback {
    int32_t hi[8];
    double hd[3];
    unsigned mb[2];
  };
  // readback buffer, event and private stream belong to the plan's SolveCache
  Readback* rb = nullptr;
  cudaEvent_t ev = nullptr;
  // The legacy default stream cannot be captured: a job given it runs on the
  // plan's private stream, ordered after the caller's earlier work and before
  // its later work by events.
  cudaStream_t caller = nullptr;
  cudaStream_t own = nullptr;

  ~SolveJob();   // ends an open iteration range
  // Allocates the working set, computes ||V||^2 (synchronises) and queues iteration 0.
  int start(pc_plan_s* plan, const float2* V_dev, double lambda, double delta, const SolveCfg& cfg,
            float* mu_out, pc_iter_record* hist, int hist_cap, cudaStream_t stream);
  // True when the queued iteration's readback has landed (non-blocking).
  bool ready() const;
  // Processes the readback: history, stop test (sets done), and, when the
  // solve goes on, queues the Gram update and sets need_apgd (or queues the
  // next iteration directly when the active set is empty).
  int process();
  // The job's reweighting as a batched-APGD entry (Gram form).
  ApgdJob apgd_job() const;
  // The job's reweighting in operator form (op_form), on the job's stream.
  int run_apgd_op();
  // After the reweighting: pruning count, then the next iteration's queue.
  int after_apgd();
  // Copies the support and weights (device), fills the statistics and orders
  // the caller's stream after the job.
  int finish(int32_t* idx_out, float* x_out, int32_t cap, pc_solve_stats* stats);

 private:
  int ld() const { return (wcap + 3) & ~3; }   // leading dimension of the Gram buffers
  std::vector<uint64_t> graph_key() const;     // every argument the captured chain depends on
  int grow(int need);
  int explore();
  int enqueue_chain(int bound, int warm_S = 0);
  int load_resume_state();
  int queue_iteration();
  int choose_form(int n_new, int n_act, bool* op);
};

}  // namespace pc
