// Serving loop: continuous batching of imaging requests on one GPU.
//
// Each request is the solve of pc_solve_host (plan, lambda = alpha
// lambda_max, Algorithm 2 of Sect. 5.1); the paper leaves parallel and
// distributed processing as future work (Sect. 7). One scheduler thread owns
// every CUDA call of the server:
//   * admission: queued requests are admitted, oldest first, while fewer than
//     max_jobs are active and their estimated device bytes fit the budget; an
//     admitted job gets its own stream, its visibilities on the device, its
//     plan and lambda_max;
//   * progress: every active job's iteration is queued on its stream up to a
//     readback marked by an event (SolveJob); the scheduler polls the events
//     and processes whichever job is ready, so the jobs' kernels overlap;
//   * batching: the reweightings (APGD) of all jobs that reach that step in
//     the same pass are launched together, several jobs per launch (one
//     thread-block cluster per job), on a batch stream that waits for each
//     job's stream and that each job's stream then waits for;
//   * completion: support, weights and statistics are copied to the host and
//     the job's device memory is released, which admits the next request.
// Requests that arrive while others run are admitted as soon as a slot and
// memory are free.
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>

#include "pc_internal.cuh"
#include "solver.cuh"

namespace pc {
namespace {

double now_s(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

struct Request {
  int64_t id = 0;
  int64_t M = 0;
  int N = 0;
  double fov = 0, alpha = 0, delta = 0;
  SolveCfg cfg;
  double* uvw = nullptr;     // pinned host copies
  pc_c32* V = nullptr;
  int64_t est_bytes = 0;
  double t_submit = 0;
};

struct Result {
  bool done = false;
  int status = PC_OK;
  std::string error;
  std::vector<int32_t> idx;
  std::vector<float> x;
  pc_solve_stats stats{};
  pc_job_times times{};
};

struct Active {
  std::unique_ptr<Request> req;
  cudaStream_t st = nullptr;
  double* d_uvw = nullptr;
  float2* d_V = nullptr;
  int32_t* d_idx = nullptr;
  float* d_x = nullptr;
  int cap = 0;
  pc_plan_s* plan = nullptr;
  std::unique_ptr<SolveJob> job;
  double t_admit = 0;
  bool finished = false;
  int status = PC_OK;
  std::string error;
};

}  // namespace
}  // namespace pc

struct pc_server_s {
  pc_server_opts opts{};
  int device = 0;
  int64_t budget = 0;
  std::chrono::steady_clock::time_point t0;
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  int64_t next_id = 1;
  std::deque<std::unique_ptr<pc::Request>> queue;
  std::map<int64_t, pc::Result> results;
  // scheduler thread only
  std::vector<std::unique_ptr<pc::Active>> active;
  int64_t bytes_active = 0;
  cudaStream_t batch_stream = nullptr;
  std::vector<cudaEvent_t> events;
};

namespace pc {
namespace {

cudaEvent_t pool_event(pc_server_s* s, size_t i) {
  while (s->events.size() <= i) {
    cudaEvent_t e = nullptr;
    cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    s->events.push_back(e);
  }
  return s->events[i];
}

void release(Active* a) {
  a->job.reset();                                   // pinned readback, event
  if (a->plan) pc_plan_destroy(a->plan);
  a->plan = nullptr;
  if (a->d_uvw) dfree(a->d_uvw, a->st);
  a->d_uvw = nullptr;
  if (a->st) {
    cudaStreamSynchronize(a->st);
    stream_put(a->st);
  }
  a->st = nullptr;
  if (a->req) {
    pinned_put(a->req->uvw);
    pinned_put(a->req->V);
    a->req->uvw = nullptr;
    a->req->V = nullptr;
  }
}

// Inputs to the device, plan, lambda = alpha lambda_max, first iteration queued.
int admit(pc_server_s* s, Active* a) {
  Request& r = *a->req;
  if (!(a->st = stream_get())) return fail(PC_ERR_CUDA, "pc_server: stream creation failed");
  a->cap = (int)std::min<int64_t>((int64_t)r.N * r.N, 1 << 20);
  const size_t b_uvw = sizeof(double) * 3 * (size_t)std::max<int64_t>(r.M, 1);
  const size_t b_V = sizeof(float2) * (size_t)std::max<int64_t>(r.M, 1);
  const size_t b_out = (sizeof(int32_t) + sizeof(float)) * (size_t)a->cap;
  char* base = nullptr;
  PC_TRY(dmalloc(reinterpret_cast<void**>(&base), b_uvw + b_V + b_out + 64, a->st));
  a->d_uvw = reinterpret_cast<double*>(base);
  a->d_V = reinterpret_cast<float2*>(base + b_uvw);
  a->d_idx = reinterpret_cast<int32_t*>(base + b_uvw + b_V);
  a->d_x = reinterpret_cast<float*>(base + b_uvw + b_V + sizeof(int32_t) * (size_t)a->cap);
  if (r.M > 0) {
    PC_CUDA(cudaMemcpyAsync(a->d_uvw, r.uvw, sizeof(double) * 3 * r.M, cudaMemcpyHostToDevice, a->st));
    PC_CUDA(cudaMemcpyAsync(a->d_V, r.V, sizeof(float2) * r.M, cudaMemcpyHostToDevice, a->st));
  }
  PC_TRY(pc_plan_create(a->d_uvw, r.M, r.N, r.fov, nullptr, a->st, &a->plan));
  double lmax = 0.0;
  const pc_c32* Vc = reinterpret_cast<const pc_c32*>(a->d_V);
  if (r.cfg.positive)
    PC_TRY(pc_lambda_max_positive(a->plan, Vc, &lmax, a->st));
  else
    PC_TRY(pc_lambda_max(a->plan, Vc, &lmax, a->st));
  a->job.reset(new SolveJob());
  if (!(lmax > 0.0)) {          // V == 0 (or no positive part): the solution is x = 0
    a->finished = true;
    a->status = PC_OK;
    return PC_OK;
  }
  PC_TRY(a->job->start(a->plan, a->d_V, r.alpha * lmax, r.delta, r.cfg, nullptr, nullptr, 0, a->st));
  return PC_OK;
}

// Result to the host, device memory released.
void complete(pc_server_s* s, Active* a) {
  Result res;
  res.done = true;
  res.status = a->status;
  res.error = a->error;
  if (a->status == PC_OK || a->status == PC_ERR_NOT_CONVERGED) {
    if (a->job && a->job->rb) {
      const int rc = a->job->finish(a->d_idx, a->d_x, a->cap, &res.stats);
      if (rc != PC_OK && rc != PC_ERR_NOT_CONVERGED) {
        res.status = rc;
        res.error = pc_last_error();
      }
      const int n = res.stats.n_support;
      if (rc == PC_OK || rc == PC_ERR_NOT_CONVERGED) {
        res.idx.resize(n);
        res.x.resize(n);
        if (n > 0) {
          cudaMemcpyAsync(res.idx.data(), a->d_idx, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, a->st);
          cudaMemcpyAsync(res.x.data(), a->d_x, sizeof(float) * n, cudaMemcpyDeviceToHost, a->st);
        }
        if (cudaStreamSynchronize(a->st) != cudaSuccess) {
          cudaGetLastError();
          res.status = PC_ERR_CUDA;
          res.error = "serving: result copy failed";
        }
      }
    } else {                               // x = 0: F(0) = ||V||^2 / 2
      double ss = 0.0;
      for (int64_t k = 0; k < a->req->M; ++k)
        ss += (double)a->req->V[k].re * a->req->V[k].re + (double)a->req->V[k].im * a->req->V[k].im;
      res.stats.status = PC_OK;
      res.stats.objective = 0.5 * ss;
      res.stats.sumsq_V = ss;
    }
  }
  res.times.submitted = a->req->t_submit;
  res.times.admitted = a->t_admit;
  res.times.finished = now_s(s->t0);
  const int64_t id = a->req->id;
  release(a);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->results[id] = std::move(res);
  }
  s->cv_done.notify_all();
}

void fail_job(Active* a, int status) {
  a->finished = true;
  a->status = status;
  a->error = pc_last_error();
}

void scheduler(pc_server_s* s) {
  cudaSetDevice(s->device);
  cudaStreamCreateWithFlags(&s->batch_stream, cudaStreamNonBlocking);
  for (;;) {
    bool progressed = false;
    // ---- admission, oldest first, by slots and memory
    for (;;) {
      std::unique_ptr<Request> r;
      {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->queue.empty() || (int)s->active.size() >= s->opts.max_jobs) break;
        const int64_t need = s->queue.front()->est_bytes;
        // a job larger than the whole budget runs alone
        if (s->bytes_active > 0 && s->bytes_active + need > s->budget) break;
        r = std::move(s->queue.front());
        s->queue.pop_front();
      }
      std::unique_ptr<Active> a(new Active());
      a->req = std::move(r);
      a->t_admit = now_s(s->t0);
      s->bytes_active += a->req->est_bytes;
      const int rc = admit(s, a.get());
      if (rc != PC_OK) fail_job(a.get(), rc);
      s->active.push_back(std::move(a));
      progressed = true;
    }
    // ---- progress of the jobs whose readback has landed
    std::vector<Active*> want_apgd;
    for (auto& ap : s->active) {
      Active* a = ap.get();
      if (a->finished || !a->job || a->job->need_apgd || !a->job->ready()) continue;
      const int rc = a->job->process();
      progressed = true;
      if (rc != PC_OK) {
        fail_job(a, rc);
        continue;
      }
      if (a->job->done) {
        a->finished = true;
        a->status = a->job->status;
      } else if (a->job->need_apgd) {
        want_apgd.push_back(a);
      }
    }
    // ---- reweightings in operator form (large active sets): one operator
    // pair per step on the job's own stream, not batchable with the others
    for (size_t i = 0; i < want_apgd.size();) {
      Active* a = want_apgd[i];
      if (!a->job->op_form) {
        ++i;
        continue;
      }
      int rc = a->job->run_apgd_op();
      if (rc == PC_OK) rc = a->job->after_apgd();
      if (rc != PC_OK) fail_job(a, rc);
      want_apgd.erase(want_apgd.begin() + (long)i);
      progressed = true;
    }
    // ---- the reweightings, batched
    if (!want_apgd.empty()) {
      if (s->opts.batch_apgd == 2) {
        for (Active* a : want_apgd) {
          const ApgdJob j = a->job->apgd_job();
          int rc = run_apgd_jobs(&j, 1, a->st);
          if (rc == PC_OK) rc = a->job->after_apgd();
          if (rc != PC_OK) fail_job(a, rc);
        }
      } else {
        std::vector<ApgdJob> jobs;
        for (size_t i = 0; i < want_apgd.size(); ++i) {
          cudaEvent_t e = pool_event(s, i);
          cudaEventRecord(e, want_apgd[i]->st);
          cudaStreamWaitEvent(s->batch_stream, e, 0);
          jobs.push_back(want_apgd[i]->job->apgd_job());
        }
        const int rc = run_apgd_jobs(jobs.data(), (int)jobs.size(), s->batch_stream);
        cudaEvent_t done_ev = pool_event(s, want_apgd.size());
        cudaEventRecord(done_ev, s->batch_stream);
        for (Active* a : want_apgd) {
          if (rc != PC_OK) {
            fail_job(a, rc);
            continue;
          }
          cudaStreamWaitEvent(a->st, done_ev, 0);
          const int rc2 = a->job->after_apgd();
          if (rc2 != PC_OK) fail_job(a, rc2);
        }
      }
      progressed = true;
    }
    // ---- completions
    for (size_t i = 0; i < s->active.size();) {
      Active* a = s->active[i].get();
      if (a->finished) {
        s->bytes_active -= a->req->est_bytes;
        complete(s, a);
        s->active.erase(s->active.begin() + i);
        progressed = true;
      } else {
        ++i;
      }
    }
    {
      std::unique_lock<std::mutex> lk(s->mu);
      if (s->stop && s->queue.empty() && s->active.empty()) break;
      if (!progressed && s->active.empty() && s->queue.empty())
        s->cv_work.wait_for(lk, std::chrono::milliseconds(50));
    }
    // jobs in flight: poll their events again at once (a readback lands every
    // few hundred microseconds; sleeping would add that much latency)
    if (!progressed) std::this_thread::yield();
  }
  for (cudaEvent_t e : s->events) cudaEventDestroy(e);
  s->events.clear();
  cudaStreamDestroy(s->batch_stream);
}

}  // namespace
}  // namespace pc

using namespace pc;

extern "C" int pc_server_create(const pc_server_opts* opts, pc_server_t* out) {
  clear_error();
  if (!out) return fail(PC_ERR_INVALID_ARG, "pc_server_create: NULL output");
  *out = nullptr;
  pc_server_opts o{PC_ABI_VERSION, 8, 0, 1, 0};
  if (opts) {
    if (opts->version != PC_ABI_VERSION)
      return fail(PC_ERR_INVALID_ARG, "pc_server_create: opts->version %d != %d", opts->version,
                  PC_ABI_VERSION);
    if (opts->max_jobs) o.max_jobs = opts->max_jobs;
    o.memory_budget = opts->memory_budget;
    if (opts->batch_apgd) o.batch_apgd = opts->batch_apgd;
  }
  if (o.max_jobs < 1 || o.max_jobs > 1024 || (o.batch_apgd != 1 && o.batch_apgd != 2))
    return fail(PC_ERR_INVALID_ARG, "pc_server_create: max_jobs in [1, 1024], batch_apgd 1 or 2");
  pc_server_s* s = new pc_server_s();
  s->opts = o;
  cudaGetDevice(&s->device);
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return fail(PC_ERR_CUDA, "pc_server_create: no usable device");
  }
  s->budget = o.memory_budget > 0 ? o.memory_budget : (int64_t)(free_b / 2);
  s->t0 = std::chrono::steady_clock::now();
  s->worker = std::thread(scheduler, s);
  *out = s;
  return PC_OK;
}

extern "C" int pc_server_submit(pc_server_t s, const double* uvw, const pc_c32* V, int64_t M, int32_t N,
                                double fov, double alpha, double delta, const pc_solve_opts* opts,
                                int64_t* id_out) {
  clear_error();
  if (!s || !id_out) return fail(PC_ERR_INVALID_ARG, "pc_server_submit: NULL server or output");
  if (M < 0 || M > (1ll << 29) || (M > 0 && (!uvw || !V)))
    return fail(PC_ERR_INVALID_ARG, "pc_server_submit: bad visibilities");
  if (N < 16 || N > 4096 || (N & 1) || !(fov > 0.0 && fov < 1.4))
    return fail(PC_ERR_INVALID_ARG, "pc_server_submit: N must be even in [16, 4096], fov in (0, 1.4)");
  if (!(alpha > 0.0 && alpha <= 1.0) || !(delta > 0.0 && delta <= 1.0))
    return fail(PC_ERR_INVALID_ARG, "pc_server_submit: alpha and delta must be in (0, 1]");
  std::unique_ptr<Request> r(new Request());
  PC_TRY(parse_solve_opts(opts, "pc_server_submit", &r->cfg));
  r->M = M;
  r->N = N;
  r->fov = fov;
  r->alpha = alpha;
  r->delta = delta;
  r->uvw = static_cast<double*>(pinned_get(sizeof(double) * 3 * std::max<int64_t>(M, 1)));
  r->V = static_cast<pc_c32*>(pinned_get(sizeof(pc_c32) * std::max<int64_t>(M, 1)));
  if (!r->uvw || !r->V) {
    pinned_put(r->uvw);
    pinned_put(r->V);
    return fail(PC_ERR_OOM, "pc_server_submit: pinned host allocation failed");
  }
  double wmin = 0.0, wmax = 0.0;
  if (M > 0) {
    std::memcpy(r->uvw, uvw, sizeof(double) * 3 * M);
    std::memcpy(r->V, V, sizeof(pc_c32) * M);
    wmin = wmax = uvw[2];
    for (int64_t k = 1; k < M; ++k) {
      wmin = std::min(wmin, uvw[3 * k + 2]);
      wmax = std::max(wmax, uvw[3 * k + 2]);
    }
  }
  r->est_bytes = plan_bytes_estimate(M, N, fov, wmin, wmax);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) {
      pinned_put(r->uvw);
      pinned_put(r->V);
      return fail(PC_ERR_INVALID_ARG, "pc_server_submit: server is shutting down");
    }
    r->id = s->next_id++;
    r->t_submit = now_s(s->t0);
    *id_out = r->id;
    s->results[r->id] = Result();
    s->queue.push_back(std::move(r));
  }
  s->cv_work.notify_one();
  return PC_OK;
}

extern "C" int pc_server_wait(pc_server_t s, int64_t id, int32_t* idx_out, float* x_out, int32_t cap,
                              pc_solve_stats* stats, pc_job_times* times) {
  clear_error();
  if (!s || cap < 0 || (cap > 0 && (!idx_out || !x_out)))
    return fail(PC_ERR_INVALID_ARG, "pc_server_wait: bad arguments");
  Result res;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->results.find(id);
    if (it == s->results.end()) return fail(PC_ERR_INVALID_ARG, "pc_server_wait: unknown job %lld", (long long)id);
    s->cv_done.wait(lk, [&] { return s->results[id].done; });
    res = std::move(s->results[id]);
    s->results.erase(id);
  }
  if (stats) *stats = res.stats;
  if (times) *times = res.times;
  if (res.status != PC_OK && res.status != PC_ERR_NOT_CONVERGED)
    return fail(res.status, "%s", res.error.empty() ? "serving: job failed" : res.error.c_str());
  const int n = (int)res.idx.size();
  if (n > cap) return fail(PC_ERR_CAPACITY, "pc_server_wait: support of %d atoms exceeds capacity %d", n, cap);
  if (n > 0) {
    std::memcpy(idx_out, res.idx.data(), sizeof(int32_t) * n);
    std::memcpy(x_out, res.x.data(), sizeof(float) * n);
  }
  if (res.status == PC_ERR_NOT_CONVERGED)
    return fail(PC_ERR_NOT_CONVERGED, "%s", res.error.empty() ? "serving: no convergence" : res.error.c_str());
  return PC_OK;
}

extern "C" void pc_server_destroy(pc_server_t s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  delete s;
}
