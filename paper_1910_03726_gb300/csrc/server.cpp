// Continuous-batching MGRIT server (mgrit_server_create / mgrit_submit /
// mgrit_poll / mgrit_server_destroy).
//
// A host worker thread owns one CUDA stream.  Each turn it
//   1. admits queued requests, first come first served, while their device
//      state fits in the HBM budget and fewer than max_active are running
//      (fitted coarse operators are cached per problem/options);
//   2. advances every admitted solve by one MGRIT cycle: one batched
//      FCF-relaxation launch per nx over all intervals of all solves, one
//      batched norm launch, one read-back of all norms, then the coarse solves
//      (one batched cluster march per cluster size for two-level periodic
//      solves; the handle's own coarse kernels for multilevel, rediscretised
//      and inflow/outflow ones);
//   3. retires converged (or failed) solves: copies their output to host
//      memory, frees their device state, and wakes pollers.
// Requests that arrive while others run join at the next turn, so their work
// overlaps on the device with the solves already in flight.  Per-solve
// arithmetic is the single-solve path's (same kernels, same block shapes),
// so a result is the same alone and in the mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "../../include/mgrit.h"
#include "device.h"
#include "handle.h"
#include "setup.h"

using namespace mg;

namespace {

struct Request {
  uint64_t ticket = 0;
  mgrit_problem prob{};
  mgrit_opts opts{};
  std::vector<double> u0;
  int state = 0;  // 0 queued, 1 active, 2 done
  mgrit_status status = MGRIT_OK;
  std::string error;
  mgrit_result res{};
  std::vector<double> out;
  mgrit_handle* h = nullptr;
  int cur = 0, it = 0;
  double r0 = 0.0, t_submit = 0.0;
  size_t bytes = 0;
};

struct PlanKey {
  int nx, nt, family, p, q, m, levels, rule, halfwidth;
  double cfl, eta, rho;
  bool operator<(const PlanKey& o) const {
    return std::memcmp(this, &o, sizeof(PlanKey)) < 0;
  }
};

// Device copy of an array that grows as needed.
template <typename T>
struct DevArray {
  T* p = nullptr;
  size_t cap = 0;
  bool reserve(size_t n) {
    if (n <= cap) return true;
    if (p) cudaFree(p);
    p = nullptr;
    cap = std::max<size_t>(n, 2 * cap);
    if (cudaMalloc(&p, cap * sizeof(T)) != cudaSuccess) {
      cudaGetLastError();
      cap = 0;
      return false;
    }
    return true;
  }
  void free() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
  }
};

}  // namespace

struct mgrit_server {
  mgrit_server_opts o{};
  cudaStream_t stream = nullptr;
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request*> queue;
  std::vector<Request*> active;
  std::unordered_map<uint64_t, Request*> reqs;
  bool stop = false;
  uint64_t next_ticket = 1;
  size_t resident = 0;
  // Coarse operators per problem shape, fitted by a pool of host threads as
  // requests arrive (so the worker never fits one while the GPU waits).
  struct PlanEntry {
    int state = 0;  // 0 pending, 1 ready, 2 failed
    std::vector<CoarseOp> ops;
    mgrit_status st = MGRIT_OK;
    std::string msg;
  };
  std::map<PlanKey, PlanEntry> plans;  // guarded by mu; entries are never erased
  std::deque<std::tuple<PlanKey, mgrit_problem, mgrit_opts>> plan_jobs;
  std::vector<std::thread> planners;
  std::condition_variable plan_cv;
  DevArray<BatchSolve> dS;
  DevArray<BatchItem> dItems;
  DevArray<DevTaps> dTaps;
  DevArray<int> dIds;
  DevArray<double> dNorm;
  double* hNorm = nullptr;
  size_t hNormCap = 0;
  std::string fatal;
  mgrit_server_counters stats{};
  double active_sum = 0.0;
};

static PlanKey key_of(const mgrit_problem& p, const mgrit_opts& o) {
  PlanKey k;
  std::memset(&k, 0, sizeof(k));
  k.nx = p.nx; k.nt = p.nt; k.family = p.family; k.p = p.rk_order; k.q = p.upwind_order;
  k.m = o.m; k.levels = o.levels; k.rule = o.psi_rule; k.halfwidth = o.psi_halfwidth;
  k.cfl = p.cfl; k.eta = o.psi_eta; k.rho = o.psi_rho;
  return k;
}

static void finish(mgrit_server* S, Request* r, mgrit_status st, const std::string& msg) {
  r->status = st;
  r->error = msg;
  if (r->h) {
    mgrit_destroy(r->h);
    r->h = nullptr;
    S->resident -= std::min(S->resident, r->bytes);
  }
  if (st == MGRIT_OK) S->stats.completed++;
  else S->stats.failed++;
  r->res.solve_s = now_s() - r->t_submit;
  r->res.dof_per_s = r->res.solve_s > 0 ? (double)r->prob.nx * r->prob.nt / r->res.solve_s : 0.0;
  r->state = 2;
}

// Admit queued requests that fit (called with the lock held; releases it
// around the host setup).  Returns the newly admitted requests.
static std::vector<Request*> admit(mgrit_server* S, std::unique_lock<std::mutex>& lk) {
  std::vector<Request*> fresh;
  const size_t max_active = S->o.max_active > 0 ? (size_t)S->o.max_active : 4096;
  while (!S->queue.empty() && S->active.size() + fresh.size() < max_active) {
    Request* r = S->queue.front();
    const auto itp = S->plans.find(key_of(r->prob, r->opts));
    if (itp == S->plans.end() || itp->second.state == 0) break;  // its operators are still being fitted
    if (itp->second.state == 2) {
      S->queue.pop_front();
      finish(S, r, itp->second.st, itp->second.msg);
      S->cv.notify_all();
      continue;
    }
    if ((double)(S->resident + r->bytes) > S->o.hbm_budget_bytes && !(S->active.empty() && fresh.empty())) break;
    S->queue.pop_front();
    S->resident += r->bytes;
    const std::vector<CoarseOp>* cached = &itp->second.ops;
    lk.unlock();
    mgrit_status st = handle_create(&r->prob, &r->opts, S->stream, cached, &r->h, false, true);
    if (st == MGRIT_OK) S->stats.tune_s += r->h->tune_s;
    std::string msg = st == MGRIT_OK ? "" : mgrit_last_error();
    if (st == MGRIT_OK) {
      mgrit_handle* h = r->h;
      st = load_iterate(h, r->u0.data(), nullptr);
      reset_stats(h);
      std::memset(&r->res, 0, sizeof(r->res));
      r->res.n_levels = h->L;
      r->res.setup_s = h->setup_s;
      r->res.op_complexity = h->op_complexity;
      if (st == MGRIT_OK) st = initial_residual_async(h, h->u0buf);  // read after the admission batch's one sync
      if (st != MGRIT_OK) msg = mgrit_last_error();
    }
    lk.lock();
    if (st != MGRIT_OK) {
      S->resident -= std::min(S->resident, r->bytes);
      r->bytes = 0;
      finish(S, r, st, msg);
      S->cv.notify_all();
      continue;
    }
    S->resident = S->resident - std::min(S->resident, r->bytes) + r->h->bytes;
    S->stats.peak_resident_bytes = std::max(S->stats.peak_resident_bytes, (double)S->resident);
    r->bytes = r->h->bytes;
    r->state = 1;
    fresh.push_back(r);
  }
  if (!fresh.empty()) {  // one sync for the batch: set-up errors and the initial residuals
    lk.unlock();
    const cudaError_t e = cudaStreamSynchronize(S->stream);
    lk.lock();
    if (e != cudaSuccess) {
      cudaGetLastError();
      S->fatal = std::string("admission: ") + cudaGetErrorString(e);
    }
    for (Request* r : fresh) {
      r->r0 = std::sqrt(r->h->norm_host[0]);
      r->res.r0_norm = r->r0;
    }
  }
  return fresh;
}

// One MGRIT cycle for every active solve.  Called without the lock.
static mgrit_status cycle(mgrit_server* S, const std::vector<Request*>& act, std::vector<char>* done) {
  const int n = (int)act.size();
  std::vector<BatchSolve> hs(n);
  std::vector<DevTaps> taps(2 * n);
  for (int k = 0; k < n; ++k) {
    mgrit_handle* h = act[k]->h;
    BatchSolve& b = hs[k];
    std::memset(&b, 0, sizeof(b));
    b.fcf.u_old = h->c[act[k]->cur];
    b.fcf.cstride = h->nx;
    b.fcf.c_new = h->c[1 - act[k]->cur];
    b.fcf.g = nullptr;
    b.fcf.r = h->r[1];
    b.fcf.r_f = h->rf[1];
    b.fcf.partial = h->partial;
    b.fcf.nx = h->nx;
    b.fcf.m = h->fine_collapse ? 1 : h->m;  // collapsed: one application of Phi^m per pass
    b.fcf.N = h->Nl[1];
    b.fcf.zero_old = 0;
    b.fcf.relax_f = h->opts.relax == MGRIT_RELAX_F;
    b.fcf.value_residual = fine_prec(h) == 0 && !b.fcf.relax_f;
    b.fcf.fx = h->fine_collapse ? h->fx_phim : h->fx_phi;  // boundary rows (inflow/outflow problems)
    b.fcf.df_store = h->dfc;
    b.prec = fine_prec(h);
    b.taps = 2 * k;
    b.psi = 2 * k + 1;
    b.cluster = h->march_cluster;
    b.sd = h->dsplan;
    taps[2 * k] = h->fine_collapse ? h->dphim : h->dphi;
    taps[2 * k + 1] = h->dpsi.back();
  }
  if (!S->dS.reserve(n) || !S->dTaps.reserve(2 * n) || !S->dIds.reserve(n) || !S->dNorm.reserve(n))
    return fail(MGRIT_ERR_OOM, "server batch descriptors");
  cudaMemcpyAsync(S->dS.p, hs.data(), n * sizeof(BatchSolve), cudaMemcpyHostToDevice, S->stream);
  cudaMemcpyAsync(S->dTaps.p, taps.data(), 2 * n * sizeof(DevTaps), cudaMemcpyHostToDevice, S->stream);
  // ---- batched FCF, one launch per (nx, launch shape): each solve keeps the
  // shape it was tuned to, so its arithmetic is the single-solve path's.
  // SDIRK fine levels: one launch per (nx, recurrence orders, precision).
  std::map<std::tuple<int, int, int, int>, std::vector<int>> groups, sgroups;
  for (int k = 0; k < n; ++k) {
    mgrit_handle* h = act[k]->h;
    if (h->sdirk)
      sgroups[{h->nx, h->splan.kf, h->splan.kb, hs[k].prec == 0 ? 0 : 1}].push_back(k);
    else
      groups[{h->nx, h->fine_tile, h->fine_threads, taps[2 * k].span}].push_back(k);
  }
  std::vector<BatchItem> items;
  std::vector<std::pair<size_t, size_t>> ranges, sranges;
  for (auto* G : {&groups, &sgroups})
    for (auto& g : *G) {
      const size_t b0 = items.size();
      for (int k : g.second)
        for (int j = 1; j <= hs[k].fcf.N; ++j) items.push_back({k, j});
      (G == &groups ? ranges : sranges).push_back({b0, items.size()});
    }
  if (!S->dItems.reserve(items.size())) return fail(MGRIT_ERR_OOM, "server batch items");
  cudaMemcpyAsync(S->dItems.p, items.data(), items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice, S->stream);
  size_t gi = 0;
  for (auto& g : groups) {
    const int nx = std::get<0>(g.first), tile = std::get<1>(g.first), th = std::get<2>(g.first);
    const int span = std::get<3>(g.first);
    const auto rg = ranges[gi++];
    cudaError_t e = launch_fcf_batched(S->dS.p, S->dItems.p + rg.first, (int)(rg.second - rg.first), S->dTaps.p, nx,
                                       th, tile, span, S->stream);
    if (e != cudaSuccess) return launch_ok(e, "fcf_batched");
    for (int k : g.second) act[k]->h->kcount[MGRIT_K_FCF]++;
  }
  gi = 0;
  for (auto& g : sgroups) {
    const auto rg = sranges[gi++];
    size_t smem = 0;
    for (int k : g.second) smem = std::max(smem, sdirk_smem(act[k]->h->splan));
    cudaError_t e = launch_fcf_sdirk_batched(S->dS.p, S->dItems.p + rg.first, (int)(rg.second - rg.first),
                                             act[g.second[0]]->h->splan, smem, std::get<3>(g.first), S->stream);
    if (e != cudaSuccess) return launch_ok(e, "fcf_sdirk_batched");
    for (int k : g.second) act[k]->h->kcount[MGRIT_K_FCF]++;
  }
  // ---- value-form residuals of the FP64 solves (no-op for the others)
  {
    cudaError_t e = launch_residual_value_batched(S->dS.p, S->dItems.p, (int)items.size(), S->stream);
    if (e != cudaSuccess) return launch_ok(e, "residual_value_batched");
  }
  // ---- norms of all solves, one read-back
  std::vector<int> ids(n);
  for (int k = 0; k < n; ++k) ids[k] = k;
  cudaMemcpyAsync(S->dIds.p, ids.data(), n * sizeof(int), cudaMemcpyHostToDevice, S->stream);
  cudaError_t e = launch_norm_batched(S->dS.p, S->dIds.p, n, S->dNorm.p, S->stream);
  if (e != cudaSuccess) return launch_ok(e, "norm_batched");
  if ((size_t)n > S->hNormCap) {
    if (S->hNorm) cudaFreeHost(S->hNorm);
    S->hNormCap = std::max<size_t>(n, 2 * S->hNormCap);
    if (cudaMallocHost(&S->hNorm, S->hNormCap * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      S->hNorm = nullptr;
      S->hNormCap = 0;
      return fail(MGRIT_ERR_OOM, "pinned norms");
    }
  }
  cudaMemcpyAsync(S->hNorm, S->dNorm.p, n * sizeof(double), cudaMemcpyDeviceToHost, S->stream);
  e = cudaStreamSynchronize(S->stream);
  if (e != cudaSuccess) return launch_ok(e, "server cycle");
  // ---- convergence decisions (Section 2.2 stopping test, per solve)
  std::vector<int> two_level;
  std::map<int, std::vector<int>> by_cluster;
  for (int k = 0; k < n; ++k) {
    Request* r = act[k];
    r->h->kcount[MGRIT_K_NORM]++;
    const double rel =
        !std::isfinite(r->r0) ? r->r0 : (r->r0 > 0.0 ? std::sqrt(S->hNorm[k]) / r->r0 : 0.0);
    if (r->res.n_history < MGRIT_MAX_HISTORY) r->res.history[r->res.n_history++] = rel;
    r->res.rel_residual = rel;
    r->res.iterations = r->it;
    if (!std::isfinite(rel) || (rel > 1e6 && !(r->opts.flags & MGRIT_FLAG_NO_DIVERGENCE_STOP))) {
      r->status = MGRIT_ERR_DIVERGED;
      r->error = "residual not finite or grew above 1e6 x initial";
      (*done)[k] = 1;
    } else if (rel <= r->opts.tol) {
      r->res.converged = 1;
      (*done)[k] = 1;
    } else if (r->it >= r->opts.max_iter) {
      r->status = MGRIT_ERR_NOT_CONVERGED;
      r->error = "max_iter reached";
      (*done)[k] = 1;
    } else if (r->h->L == 2 && !r->h->redisc && !r->h->inflow && !r->h->fft_coarse) {
      by_cluster[r->h->march_cluster].push_back(k);
    }
  }
  // ---- coarse solves: batched cluster marches (two-level), V-cycles (multilevel)
  for (auto& g : by_cluster) {
    int max_w = 0, max_halo = 0;
    for (int k : g.second) {
      const mgrit_handle* h = act[k]->h;
      max_w = std::max(max_w, h->nx / g.first);
      max_halo = std::max(max_halo, h->dpsi.back().hi - h->dpsi.back().lo);
    }
    cudaMemcpyAsync(S->dIds.p, g.second.data(), g.second.size() * sizeof(int), cudaMemcpyHostToDevice, S->stream);
    e = launch_march_batched(S->dS.p, S->dIds.p, (int)g.second.size(), S->dTaps.p, g.first, max_w, max_halo,
                             S->stream);
    if (e != cudaSuccess) return launch_ok(e, "march_batched");
    for (int k : g.second) act[k]->h->kcount[MGRIT_K_MARCH]++;
    // the ids buffer is reused by the next group: keep launches ordered
    e = cudaStreamSynchronize(S->stream);
    if (e != cudaSuccess) return launch_ok(e, "march_batched");
  }
  for (int k = 0; k < n; ++k) {
    Request* r = act[k];
    if ((*done)[k]) continue;
    if (r->h->L > 2 || r->h->redisc || r->h->inflow || r->h->fft_coarse) {  // the handle's own coarse solve
      mgrit_status st = coarse_cycle(r->h, r->h->c[1 - r->cur]);
      if (st != MGRIT_OK) {
        r->status = st;
        r->error = mgrit_last_error();
        (*done)[k] = 1;
        continue;
      }
    }
    r->cur = 1 - r->cur;
    r->it++;
  }
  return MGRIT_OK;
}

static void retire(mgrit_server* S, Request* r) {
  mgrit_handle* h = r->h;
  if (r->status == MGRIT_OK || r->status == MGRIT_ERR_NOT_CONVERGED) {
    const size_t rows = r->opts.output == MGRIT_OUT_FINAL ? 1
                        : r->opts.output == MGRIT_OUT_CPOINTS ? (size_t)h->Nl[1] + 1
                                                              : (size_t)h->nt + 1;
    r->out.assign(rows * h->nx, 0.0);
    mgrit_status st = write_output(h, h->c[1 - r->cur], r->out.data());
    if (st == MGRIT_OK && cudaStreamSynchronize(S->stream) != cudaSuccess) st = MGRIT_ERR_CUDA;
    if (st != MGRIT_OK) {
      r->status = st;
      r->error = mgrit_last_error();
    }
  }
  collect_stats(h, &r->res);
  mgrit_destroy(h);  // device state released here, accounted under the lock by the caller
  r->h = nullptr;
  r->res.solve_s = now_s() - r->t_submit;
  r->res.dof_per_s = r->res.solve_s > 0 ? (double)r->prob.nx * r->prob.nt / r->res.solve_s : 0.0;
}

// Under the lock: a retired request becomes visible to pollers.
static void publish(mgrit_server* S, Request* r) {
  S->resident -= std::min(S->resident, r->bytes);
  if (r->status == MGRIT_OK) S->stats.completed++;
  else S->stats.failed++;
  r->state = 2;
}

// The queue's head can be admitted or failed (its operators are fitted).
static bool head_ready(mgrit_server* S) {
  if (S->queue.empty()) return false;
  const auto it = S->plans.find(key_of(S->queue.front()->prob, S->queue.front()->opts));
  return it != S->plans.end() && it->second.state != 0;
}

static void planner_main(mgrit_server* S) {
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    S->plan_cv.wait(lk, [&] { return S->stop || !S->plan_jobs.empty(); });
    if (S->stop) return;
    auto job = S->plan_jobs.front();
    S->plan_jobs.pop_front();
    lk.unlock();
    const double t0 = now_s();
    std::vector<CoarseOp> ops;
    const mgrit_status st = plan(&std::get<1>(job), &std::get<2>(job), &ops);
    const std::string msg = st == MGRIT_OK ? "" : mgrit_last_error();
    const double dt = now_s() - t0;
    lk.lock();
    auto& e = S->plans[std::get<0>(job)];
    e.ops = std::move(ops);
    e.st = st;
    e.msg = msg;
    e.state = st == MGRIT_OK ? 1 : 2;
    S->stats.plan_s += dt;
    S->cv.notify_all();
  }
}

static void worker_main(mgrit_server* S) {
  std::unique_lock<std::mutex> lk(S->mu);
  if (!S->stream) {
    if (cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      S->fatal = "cudaStreamCreate failed";
    }
  }
  while (!S->stop) {
    if (!S->fatal.empty()) {
      for (Request* r : S->queue) finish(S, r, MGRIT_ERR_CUDA, S->fatal);
      S->queue.clear();
      S->cv.notify_all();
      S->cv.wait(lk, [&] { return S->stop || !S->queue.empty(); });
      continue;
    }
    const double ta = now_s();
    std::vector<Request*> fresh = admit(S, lk);
    S->stats.admit_s += now_s() - ta;
    for (Request* r : fresh) S->active.push_back(r);
    if (S->active.empty()) {
      S->cv.notify_all();
      S->cv.wait(lk, [&] { return S->stop || head_ready(S); });
      continue;
    }
    std::vector<Request*> act = S->active;
    lk.unlock();
    std::vector<char> done(act.size(), 0);
    const double tc = now_s();
    mgrit_status st = cycle(S, act, &done);
    const double tr = now_s();
    std::string msg = st == MGRIT_OK ? "" : mgrit_last_error();
    if (st != MGRIT_OK)
      for (size_t k = 0; k < act.size(); ++k) {
        done[k] = 1;
        act[k]->status = st;
        act[k]->error = msg;
      }
    for (size_t k = 0; k < act.size(); ++k)
      if (done[k]) retire(S, act[k]);
    const double te = now_s();
    lk.lock();
    for (size_t k = 0; k < act.size(); ++k)
      if (done[k]) publish(S, act[k]);
    S->stats.cycles++;
    S->stats.cycle_s += tr - tc;
    S->stats.retire_s += te - tr;
    S->active_sum += (double)act.size();
    S->stats.mean_active = S->active_sum / (double)S->stats.cycles;
    std::vector<Request*> keep;
    for (size_t k = 0; k < act.size(); ++k)
      if (!done[k]) keep.push_back(act[k]);
    S->active.swap(keep);
    S->cv.notify_all();
  }
  // drain: everything still queued or active fails with TIMEOUT-free cancellation
  for (Request* r : S->active) finish(S, r, MGRIT_ERR_CUDA, "server destroyed");
  for (Request* r : S->queue) finish(S, r, MGRIT_ERR_CUDA, "server destroyed");
  S->active.clear();
  S->queue.clear();
  S->cv.notify_all();
}

extern "C" mgrit_status mgrit_server_create(const mgrit_server_opts* sopts, void* stream, mgrit_server** out) {
  if (!out) return fail(MGRIT_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!sopts || !(sopts->hbm_budget_bytes > 0.0) || sopts->max_active < 0)
    return fail(MGRIT_ERR_INVALID, "server options need hbm_budget_bytes > 0 and max_active >= 0");
  mgrit_server* S = new mgrit_server();
  S->o = *sopts;
  S->stream = (cudaStream_t)stream;
  S->worker = std::thread(worker_main, S);
  const unsigned hc = std::thread::hardware_concurrency();
  const unsigned np = std::max(1u, std::min(8u, hc > 2 ? hc - 2 : 1u));
  for (unsigned k = 0; k < np; ++k) S->planners.emplace_back(planner_main, S);
  *out = S;
  return MGRIT_OK;
}

extern "C" mgrit_status mgrit_submit(mgrit_server* S, const mgrit_problem* prob, const mgrit_opts* opts,
                                     const double* u0, uint64_t* ticket) {
  if (!S || !ticket || !u0) return fail(MGRIT_ERR_INVALID, "server, u0 and ticket must be non-NULL");
  mgrit_status st = validate_problem(prob);
  if (st == MGRIT_OK) st = validate_opts(prob, opts);
  if (st != MGRIT_OK) return st;
  if (opts->psi_rule == MGRIT_PSI_USER) return fail(MGRIT_ERR_UNSUPPORTED, "the server fits Psi itself");
  if (opts->init_guess != MGRIT_INIT_ZERO)
    return fail(MGRIT_ERR_UNSUPPORTED, "the server starts every request from the zero iterate");
  Request* r = new Request();
  r->prob = *prob;
  r->opts = *opts;
  r->opts.psi_user_nnz = nullptr;
  r->opts.psi_user_offsets = nullptr;
  r->opts.psi_user_coeffs = nullptr;
  r->bytes = handle_bytes(prob, opts);
  if ((double)r->bytes > S->o.hbm_budget_bytes) {
    delete r;
    return fail(MGRIT_ERR_OVER_BUDGET, "request needs more device memory than the server budget");
  }
  r->u0.resize(prob->nx);
  if (is_device_ptr(u0)) {
    if (cudaMemcpy(r->u0.data(), u0, prob->nx * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) {
      cudaGetLastError();
      delete r;
      return fail(MGRIT_ERR_CUDA, "copying u0 from the device");
    }
  } else {
    std::memcpy(r->u0.data(), u0, prob->nx * sizeof(double));
  }
  r->t_submit = now_s();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    r->ticket = S->next_ticket++;
    S->stats.submitted++;
    const PlanKey key = key_of(r->prob, r->opts);
    if (S->plans.find(key) == S->plans.end()) {
      S->plans[key];  // pending
      S->plan_jobs.emplace_back(key, r->prob, r->opts);
      S->plan_cv.notify_one();
    }
    S->reqs[r->ticket] = r;
    S->queue.push_back(r);
    *ticket = r->ticket;
  }
  S->cv.notify_all();
  return MGRIT_OK;
}

extern "C" mgrit_status mgrit_poll(mgrit_server* S, uint64_t ticket, double* out, mgrit_result* res) {
  if (!S) return fail(MGRIT_ERR_INVALID, "server is NULL");
  Request* r = nullptr;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return fail(MGRIT_ERR_UNKNOWN_TICKET, "ticket unknown or already released");
    r = it->second;
    if (r->state != 2) return MGRIT_PENDING;
    S->reqs.erase(it);
  }
  if (out && !r->out.empty()) {
    if (is_device_ptr(out)) {
      if (cudaMemcpy(out, r->out.data(), r->out.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
        cudaGetLastError();
    } else {
      std::memcpy(out, r->out.data(), r->out.size() * sizeof(double));
    }
  }
  if (res) {
    *res = r->res;
    grid_spacings(&r->prob, &res->dx, &res->dt);
  }
  const mgrit_status st = r->status;
  if (st != MGRIT_OK) fail(st, r->error);
  delete r;
  return st;
}

extern "C" mgrit_status mgrit_server_stats(mgrit_server* S, mgrit_server_counters* out) {
  if (!S || !out) return fail(MGRIT_ERR_INVALID, "server and out must be non-NULL");
  std::lock_guard<std::mutex> lk(S->mu);
  *out = S->stats;
  return MGRIT_OK;
}

extern "C" void mgrit_server_destroy(mgrit_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv.notify_all();
  S->plan_cv.notify_all();
  if (S->worker.joinable()) S->worker.join();
  for (auto& t : S->planners)
    if (t.joinable()) t.join();
  for (auto& kv : S->reqs) delete kv.second;
  S->reqs.clear();
  S->dS.free();
  S->dItems.free();
  S->dTaps.free();
  S->dIds.free();
  S->dNorm.free();
  if (S->hNorm) cudaFreeHost(S->hNorm);
  delete S;
}
