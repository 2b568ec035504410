// Solve server: many independent hyperelastic Newton solves of different meshes, degrees, materials
// and loads, continuously batched on one GPU.
//
// Requests are queued in arrival order. A pool of worker threads, each with its own non-blocking CUDA
// stream, admits the request at the head of the queue as soon as a worker is free and the request's
// device footprint (hy_footprint, the exact mirror of a context's allocations) fits in the remaining
// budget; the head is never bypassed, so a large request cannot starve. An admitted request builds its
// own context (hierarchy, caches, V-cycle graph) on the worker's stream, keeps it resident for its whole
// Newton solve and releases it when done, at which point the next request is admitted. Requests that
// arrive while others run therefore join them on the device: their kernels overlap through the
// concurrent streams. Latency is measured from submission to completion.
//
// A solve that fails only because its coarsest level's tangent is not positive definite (a coarse mesh
// that does not resolve the inclusion, under a large load) is run again from its start state with that
// level dropped, as long as two levels remain and the budget has room for the larger coarse level.
//
// Batched solves (hy_server_set_batching): the linear solves of the running Newton iterations are fused
// across requests. Each worker still linearises its own request (state, diagonals, eigenvalue estimates,
// V-cycle graph) on its own stream, but hands its outer preconditioned CG to a batcher thread and waits.
// The batcher collects the solves that are waiting -- until every running Newton solve has one waiting, or
// for at most the batching window after the oldest arrived -- groups them by (dimension, degree, cache
// variants, finest-level precision, CG tolerance and cap) and advances each group as one work-list batch:
// per PCG iteration one CUDA-graph replay, in which ONE kernel launch applies the finest-level tangents of
// all members and the members' V-cycles run as concurrent branches (hy_batch_pcg). Groups of different
// degree cannot share a launch (the kernel's shared-memory layout, threads per block and registers are
// those of its degree) and run side by side on their own batches instead.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "../../include/hyperelastic.h"
#include "serve_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Req {
  uint64_t id = 0;
  int dim = 0, degree = 0, m = 0, nlev = 0;
  uint32_t fm[6] = {};
  std::vector<uint8_t> mats;  // concatenated per-level material ids, coarsest level first
  std::vector<double> mu, lam;
  hy_newton_params np{};
  hy_solver_params sp{};
  int law = HY_LAW_LOG2;
  int64_t bytes = 0;
  int state = 0;  // 0 queued, 1 running, 2 done, 3 failed
  hy_status status = HY_OK;
  std::string err;
  hy_newton_report rep{};
  std::vector<double> u;
  std::vector<double> u_start;  // empty: start from zero
  int dropped = 0;              // coarsest levels dropped after an indefinite coarse tangent
  Clock::time_point t_submit, t_start, t_end;
};

// One outer linear solve handed to the batcher by a worker's Newton iteration.
struct SolveJob {
  hy_ctx* ctx = nullptr;
  const double* rhs = nullptr;
  double* x = nullptr;
  double rtol = 0.0;
  int max_iter = 0;
  int iterations = 0;
  hy_status status = HY_OK;
  bool done = false;
  Clock::time_point t_queued;
};

}  // namespace

struct hy_server {
  int device = 0;
  int64_t budget = 0;
  int max_active = 1;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Req*> queue;
  std::unordered_map<uint64_t, std::unique_ptr<Req>> reqs;
  int64_t in_use = 0, peak = 0;
  int active = 0;
  int64_t submitted = 0, completed = 0, failed = 0, retried = 0;
  bool stop = false;
  uint64_t next_id = 1;
  std::vector<std::thread> workers;
  // batched solves
  bool batching = false;
  double window_ms = 2.0;
  int in_newton = 0;                 // workers inside a Newton solve (potential batch members)
  std::deque<SolveJob*> jobs;        // waiting for the batcher
  std::condition_variable cv_jobs, cv_jobs_done;
  bool stop_batcher = false;
  std::thread batcher;
  std::vector<hy_batch*> batches;    // one per group that can run at once, created on first use
  int64_t batched_solves = 0, batch_runs = 0;
};

namespace {

long long level_cells(const Req& r, int l) {
  long long ml = (long long)r.m >> (r.nlev - 1 - l), c = 1;
  for (int i = 0; i < r.dim; ++i) c *= ml;
  return c;
}

// One attempt of a request on the worker's stream with its `drop` coarsest levels left out: context,
// hierarchy, materials, Newton solve, result to host. *coarse_indefinite tells whether it failed on a
// coarsest-level tangent that is not positive definite.
// The solve hook of a batching server: queue the solve for the batcher and wait for its result.
hy_status batched_solve(void* user, hy_ctx* ctx, const double* rhs, double* x, double rtol, int max_iter,
                        int* iterations) {
  hy_server* sv = static_cast<hy_server*>(user);
  SolveJob job;
  job.ctx = ctx;
  job.rhs = rhs;
  job.x = x;
  job.rtol = rtol;
  job.max_iter = max_iter;
  std::unique_lock<std::mutex> lock(sv->mu);
  job.t_queued = Clock::now();
  sv->jobs.push_back(&job);
  sv->cv_jobs.notify_all();
  sv->cv_jobs_done.wait(lock, [&] { return job.done; });
  *iterations = job.iterations;
  return job.status;
}

hy_status run_attempt(hy_server* sv, Req& r, int drop, int device, cudaStream_t st, bool* coarse_indefinite) {
  *coarse_indefinite = false;
  hy_ctx* ctx = nullptr;
  double* u = nullptr;
  const int nlev = r.nlev - drop;
  hy_solver_params sp = r.sp;
  hy_status s = hy_create(&ctx, device, st);
  if (s == HY_OK) s = hy_mesh_setup(ctx, r.dim, r.degree, r.m, nlev, r.fm);
  int64_t n_coarse = 0;
  if (s == HY_OK) s = hy_num_dofs(ctx, 0, &n_coarse);
  if (s == HY_OK && drop > 0 && n_coarse > 6000) sp.coarse_solver = 0;  // beyond the dense inverse: Chebyshev
  if (s == HY_OK) s = hy_set_solver_params(ctx, &sp);
  if (s == HY_OK) s = hy_set_material_law(ctx, r.law);
  size_t off = 0;
  for (int l = 0; l < drop; ++l) off += (size_t)level_cells(r, l);
  for (int l = drop; l < r.nlev && s == HY_OK; ++l) {
    s = hy_set_material(ctx, l - drop, r.mats.data() + off, r.mu.data(), r.lam.data(), (int)r.mu.size());
    off += (size_t)level_cells(r, l);
  }
  int64_t n = 0;
  if (s == HY_OK) s = hy_num_dofs(ctx, -1, &n);
  if (s == HY_OK) {
    if (cudaMallocAsync((void**)&u, sizeof(double) * n, st) != cudaSuccess)
      s = HY_ERR_OOM;
    else if ((r.u_start.empty() ? cudaMemsetAsync(u, 0, sizeof(double) * n, st)
                                : cudaMemcpyAsync(u, r.u_start.data(), sizeof(double) * n, cudaMemcpyHostToDevice,
                                                  st)) != cudaSuccess)
      s = HY_ERR_CUDA;
  }
  const bool counted = s == HY_OK && sv->batching;
  if (counted) {
    hy_ctx_set_solve_hook(ctx, batched_solve, sv);
    std::lock_guard<std::mutex> lock(sv->mu);
    sv->in_newton++;
  }
  if (s == HY_OK) s = hy_newton_solve(ctx, &r.np, u, &r.rep);
  if (counted) {
    {
      std::lock_guard<std::mutex> lock(sv->mu);
      sv->in_newton--;
    }
    sv->cv_jobs.notify_all();  // the batcher may now have every running solve waiting
  }
  if (s == HY_OK) {
    r.u.resize((size_t)n);
    if (cudaMemcpyAsync(r.u.data(), u, sizeof(double) * n, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      s = HY_ERR_CUDA;
  }
  if (s != HY_OK) {
    r.err = ctx ? hy_last_error(ctx) : "context creation failed";
    *coarse_indefinite = s == HY_ERR_NOCONV && r.err.rfind("coarsest-level tangent is not positive definite", 0) == 0;
  }
  if (u) cudaFreeAsync(u, st);
  hy_destroy(ctx);
  cudaStreamSynchronize(st);
  return s;
}

// Device bytes of the request with `drop` coarsest levels left out (the coarse solver as run_attempt
// picks it), or -1.
int64_t attempt_bytes(const Req& r, int drop) {
  const int nlev = r.nlev - drop;
  hy_solver_params sp = r.sp;
  const long long mc = (long long)r.m >> (nlev - 1);
  const double nc = r.dim * std::pow(r.degree * (double)mc + 1.0, r.dim);
  if (drop > 0 && nc > 6000.0) sp.coarse_solver = 0;
  int64_t bytes = 0;
  if (hy_footprint_general(r.dim, r.degree, r.m, nlev, r.np.variant, r.np.level_dtype, &sp, r.fm,
                           r.law != HY_LAW_LOG2, &bytes) != HY_OK)
    return -1;
  return bytes + (int64_t)sizeof(double) * r.dim * (int64_t)std::llround(std::pow(r.degree * r.m + 1.0, r.dim));
}

void run_request(hy_server* sv, Req& r, cudaStream_t st) {
  for (int drop = 0;; ++drop) {
    bool coarse_indefinite = false;
    r.status = run_attempt(sv, r, drop, sv->device, st, &coarse_indefinite);
    r.dropped = drop;
    if (!coarse_indefinite || r.nlev - drop <= 2) return;
    // retry with the coarsest level dropped if the budget has room for it
    const int64_t need = attempt_bytes(r, drop + 1);
    if (need < 0) return;
    {
      std::lock_guard<std::mutex> lock(sv->mu);
      const int64_t extra = std::max<int64_t>(0, need - r.bytes);
      if (sv->in_use + extra > sv->budget) return;
      sv->in_use += extra;
      sv->peak = std::max(sv->peak, sv->in_use);
      r.bytes += extra;
      sv->retried++;
    }
    r.rep = hy_newton_report{};
  }
}

// Advance one group of waiting solves (same batch key, tolerance and cap) as one work-list batch.
void run_group(hy_server* sv, hy_batch* b, std::vector<SolveJob*>& g) {
  const int cnt = (int)g.size();
  std::vector<hy_ctx*> ctxs(cnt);
  std::vector<const double*> rhs(cnt);
  std::vector<double*> xs(cnt);
  std::vector<int> its(cnt, 0);
  std::vector<hy_status> sts(cnt, HY_OK);
  for (int i = 0; i < cnt; ++i) {
    ctxs[i] = g[i]->ctx;
    rhs[i] = g[i]->rhs;
    xs[i] = g[i]->x;
  }
  hy_status st = hy_batch_bind(b, ctxs.data(), cnt);
  if (st == HY_OK) st = hy_batch_pcg(b, rhs.data(), xs.data(), g[0]->rtol, g[0]->max_iter, its.data(), sts.data());
  for (int i = 0; i < cnt; ++i) {
    g[i]->iterations = its[i];
    g[i]->status = st != HY_OK ? st : sts[i];
  }
  (void)sv;
}

void batcher_loop(hy_server* sv) {
  cudaSetDevice(sv->device);
  std::unique_lock<std::mutex> lock(sv->mu);
  for (;;) {
    sv->cv_jobs.wait(lock, [&] { return sv->stop_batcher || !sv->jobs.empty(); });
    if (sv->jobs.empty()) break;  // stop_batcher, nothing left
    // gather: until every running Newton solve has a solve waiting, or the window after the oldest closes
    const auto deadline = sv->jobs.front()->t_queued + std::chrono::duration_cast<Clock::duration>(
                                                            std::chrono::duration<double, std::milli>(sv->window_ms));
    sv->cv_jobs.wait_until(lock, deadline, [&] { return (int)sv->jobs.size() >= sv->in_newton; });
    std::vector<SolveJob*> take(sv->jobs.begin(), sv->jobs.end());
    sv->jobs.clear();
    lock.unlock();
    // groups of one batch key, tolerance, cap and size class: a batch returns when its slowest member has
    // converged, so members within a factor of 4 in dofs are fused and the others run side by side
    std::vector<std::vector<SolveJob*>> groups;
    std::vector<std::tuple<long long, double, int, int>> keys;
    for (SolveJob* j : take) {
      int64_t nd = 1;
      hy_num_dofs(j->ctx, -1, &nd);
      int size_class = 0;
      while (nd > 1) {
        nd >>= 2;
        ++size_class;
      }
      const auto key = std::make_tuple(hy_ctx_batch_key(j->ctx), j->rtol, j->max_iter, size_class);
      size_t gi = 0;
      while (gi < keys.size() && keys[gi] != key) ++gi;
      if (gi == keys.size()) {
        keys.push_back(key);
        groups.emplace_back();
      }
      groups[gi].push_back(j);
    }
    while (sv->batches.size() < groups.size()) {
      hy_batch* b = nullptr;
      if (hy_batch_create_empty(&b, sv->device, sv->max_active) != HY_OK) break;
      sv->batches.push_back(b);
    }
    if (sv->batches.size() < groups.size()) {
      for (SolveJob* j : take) j->status = HY_ERR_OOM;
    } else if (groups.size() == 1) {
      run_group(sv, sv->batches[0], groups[0]);
    } else {  // groups of different degree (or dimension, variant, precision) side by side
      std::vector<std::thread> th;
      for (size_t gi = 0; gi < groups.size(); ++gi)
        th.emplace_back([sv, gi, &groups]() {
          cudaSetDevice(sv->device);
          run_group(sv, sv->batches[gi], groups[gi]);
        });
      for (auto& t : th) t.join();
    }
    lock.lock();
    sv->batched_solves += (int64_t)take.size();
    sv->batch_runs += (int64_t)groups.size();
    for (SolveJob* j : take) j->done = true;
    sv->cv_jobs_done.notify_all();
  }
}

void worker_loop(hy_server* sv) {
  cudaSetDevice(sv->device);
  cudaStream_t st = nullptr;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  for (;;) {
    Req* r = nullptr;
    {
      std::unique_lock<std::mutex> lock(sv->mu);
      sv->cv_work.wait(lock, [&] {
        return sv->stop || (!sv->queue.empty() && sv->in_use + sv->queue.front()->bytes <= sv->budget);
      });
      if (sv->stop) break;
      r = sv->queue.front();
      sv->queue.pop_front();
      sv->in_use += r->bytes;
      sv->peak = std::max(sv->peak, sv->in_use);
      sv->active++;
      r->state = 1;
      r->t_start = Clock::now();
    }
    sv->cv_work.notify_all();  // the next head may fit as well
    run_request(sv, *r, st);
    {
      std::lock_guard<std::mutex> lock(sv->mu);
      sv->in_use -= r->bytes;
      sv->active--;
      r->t_end = Clock::now();
      r->state = r->status == HY_OK ? 2 : 3;
      if (r->status == HY_OK) sv->completed++;
      else sv->failed++;
    }
    sv->cv_done.notify_all();
    sv->cv_work.notify_all();
  }
  cudaStreamDestroy(st);
}

}  // namespace

extern "C" {

hy_status hy_server_create(hy_server** out, int device, int64_t hbm_budget_bytes, int max_active) {
  if (!out || hbm_budget_bytes <= 0 || max_active < 1 || max_active > 64) return HY_ERR_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return HY_ERR_ARG;
  hy_server* sv = new (std::nothrow) hy_server();
  if (!sv) return HY_ERR_OOM;
  sv->device = device;
  sv->budget = hbm_budget_bytes;
  sv->max_active = max_active;
  for (int i = 0; i < max_active; ++i) sv->workers.emplace_back(worker_loop, sv);
  *out = sv;
  return HY_OK;
}

void hy_server_destroy(hy_server* sv) {
  if (!sv) return;
  {
    // running requests finish (workers look at `stop` only between requests); queued ones are dropped
    std::lock_guard<std::mutex> lock(sv->mu);
    for (Req* r : sv->queue) r->state = 3;
    sv->queue.clear();
    sv->stop = true;
  }
  sv->cv_work.notify_all();
  sv->cv_done.notify_all();
  for (auto& t : sv->workers) t.join();
  if (sv->batcher.joinable()) {  // after the workers: their last solves may still need it
    {
      std::lock_guard<std::mutex> lock(sv->mu);
      sv->stop_batcher = true;
    }
    sv->cv_jobs.notify_all();
    sv->batcher.join();
  }
  cudaSetDevice(sv->device);
  for (hy_batch* b : sv->batches) hy_batch_destroy(b);
  delete sv;
}

hy_status hy_server_set_batching(hy_server* sv, int enable, double window_ms) {
  if (!sv || !(window_ms >= 0.0) || window_ms > 1000.0) return HY_ERR_ARG;
  std::lock_guard<std::mutex> lock(sv->mu);
  if (sv->submitted > 0 || sv->batching) return HY_ERR_STATE;
  sv->window_ms = window_ms;
  if (enable) {
    sv->batching = true;
    sv->batcher = std::thread(batcher_loop, sv);
  }
  return HY_OK;
}

hy_status hy_server_submit(hy_server* sv, const hy_request* q, uint64_t* ticket) {
  if (!sv || !q || !ticket) return HY_ERR_ARG;
  if ((q->dim != 2 && q->dim != 3) || q->degree < 1 || q->degree > 4 || q->cells_per_dir < 1 || q->n_levels < 1 ||
      !q->cell_mat_levels || !q->mu || !q->lambda || q->n_mat < 1 || q->n_mat > 16)
    return HY_ERR_ARG;
  auto r = std::make_unique<Req>();
  r->dim = q->dim;
  r->degree = q->degree;
  r->m = q->cells_per_dir;
  r->nlev = q->n_levels;
  std::memcpy(r->fm, q->face_masks, sizeof(r->fm));
  size_t total = 0;
  for (int l = 0; l < r->nlev; ++l) {
    if (((long long)r->m >> (r->nlev - 1 - l)) < 1) return HY_ERR_ARG;
    total += (size_t)level_cells(*r, l);
  }
  r->mats.assign(q->cell_mat_levels, q->cell_mat_levels + total);
  r->mu.assign(q->mu, q->mu + q->n_mat);
  r->lam.assign(q->lambda, q->lambda + q->n_mat);
  r->np = q->newton;
  r->sp = q->solver;
  if (q->law != HY_LAW_LOG2 && q->law != HY_LAW_J2) return HY_ERR_ARG;
  r->law = q->law;
  int64_t bytes = 0;
  hy_status s = hy_footprint_general(r->dim, r->degree, r->m, r->nlev, q->newton.variant, q->newton.level_dtype,
                                     &q->solver, r->fm, q->law != HY_LAW_LOG2, &bytes);
  if (s != HY_OK) return s;
  const int64_t n_u = r->dim * (int64_t)std::llround(std::pow(r->degree * r->m + 1.0, r->dim));
  r->bytes = bytes + (int64_t)sizeof(double) * n_u;  // + u
  if (q->u_start) r->u_start.assign(q->u_start, q->u_start + n_u);
  if (r->bytes > sv->budget) return HY_ERR_OOM;  // could never be admitted
  {
    std::lock_guard<std::mutex> lock(sv->mu);
    if (sv->stop) return HY_ERR_STATE;
    r->id = sv->next_id++;
    r->t_submit = Clock::now();
    *ticket = r->id;
    sv->queue.push_back(r.get());
    sv->reqs[r->id] = std::move(r);
    sv->submitted++;
  }
  sv->cv_work.notify_all();
  return HY_OK;
}

hy_status hy_server_poll(hy_server* sv, uint64_t ticket, int* state, hy_newton_report* rep, double* u_host,
                         int64_t n_u, double* latency_ms) {
  if (!sv || !state) return HY_ERR_ARG;
  std::lock_guard<std::mutex> lock(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) return HY_ERR_ARG;
  Req& r = *it->second;
  *state = r.state;
  if (r.state >= 2) {
    if (rep) *rep = r.rep;
    if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r.t_end - r.t_submit).count();
    if (u_host && r.state == 2) {
      if (n_u != (int64_t)r.u.size()) return HY_ERR_ARG;
      std::memcpy(u_host, r.u.data(), sizeof(double) * r.u.size());
    }
    if (r.state == 3) return r.status == HY_OK ? HY_ERR_STATE : r.status;
  }
  return HY_OK;
}

hy_status hy_server_wait(hy_server* sv, uint64_t ticket, double timeout_s) {
  if (!sv) return HY_ERR_ARG;
  std::unique_lock<std::mutex> lock(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) return HY_ERR_ARG;
  Req* r = it->second.get();
  const bool ok = sv->cv_done.wait_for(lock, std::chrono::duration<double>(timeout_s), [&] { return r->state >= 2; });
  return ok ? HY_OK : HY_ERR_TIMEOUT;
}

hy_status hy_server_release(hy_server* sv, uint64_t ticket) {
  if (!sv) return HY_ERR_ARG;
  std::lock_guard<std::mutex> lock(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end() || it->second->state < 2) return HY_ERR_ARG;
  sv->reqs.erase(it);
  return HY_OK;
}

hy_status hy_server_stats_get(hy_server* sv, hy_server_stats* st) {
  if (!sv || !st) return HY_ERR_ARG;
  std::lock_guard<std::mutex> lock(sv->mu);
  st->submitted = sv->submitted;
  st->completed = sv->completed;
  st->failed = sv->failed;
  st->active = sv->active;
  st->queued = (int64_t)sv->queue.size();
  st->bytes_in_use = sv->in_use;
  st->bytes_peak = sv->peak;
  st->budget = sv->budget;
  st->retried = sv->retried;
  st->batched_solves = sv->batched_solves;
  st->batch_runs = sv->batch_runs;
  return HY_OK;
}

}  // extern "C"
