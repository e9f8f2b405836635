// Continuous-batching MGRIT server (mgrit_server_create / mgrit_submit /
// mgrit_poll / mgrit_server_destroy).
//
// A host worker thread owns one CUDA stream for the cycles and one for
// set-up copies.  Each turn it
//   1. queues one MGRIT cycle of every admitted solve: one batched
//      FCF-relaxation launch per (nx, launch shape) over all intervals of all
//      those solves, one batched norm launch and one read-back of all norms;
//   2. while the GPU runs them, admits queued requests, first come first
//      served, while their device state fits in the HBM budget and fewer than
//      max_active are running (coarse operators fitted by planner threads as
//      requests arrive; set-up copies and initial residuals on the upload
//      stream); they join at the next turn;
//   3. after the one synchronisation of the turn takes the stopping decisions
//      and queues the coarse solves (one batched cluster march per cluster
//      size for two-level periodic solves; the handle's own coarse kernels for
//      multilevel, rediscretised and inflow/outflow ones);
//   4. retires converged (or failed) solves: copies their output to host
//      memory, frees their device state, and wakes pollers.
// Requests that arrive while others run join at the next turn, so their work
// overlaps on the device with the solves already in flight.  Per-solve
// arithmetic is the single-solve path's (same kernels, same block shapes),
// so a result is the same alone and in the mix.  (The batched FCF applies
// Phi^m as a stencil: a MIXED solve alone matches it with the Fourier-space
// FP64 pass off, MGRIT_FCF_FOURIER=0; with it on, to that pass's rounding.)
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <condition_variable>
#include <cstdint>
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
  int slot = -1;  // its two stencils' place in the server's device tap table
  int cur = 0, it = 0;
  double r0 = 0.0, t_submit = 0.0;
  size_t bytes = 0;
};

// Requests admitted before the first cycle of a busy period starts; the rest
// join while cycles run.  Admission during a cycle stops when the cycle's
// relaxation is done, once at least kMinBatch solves are active: a cycle costs
// about the time of its longest coarse march whatever the number of solves,
// so small cycles waste it.
constexpr size_t kStartBatch = 64;
constexpr size_t kMinBatch = 512;

struct PlanKey {
  int nx, nt, family, p, q, m, levels, rule, halfwidth;
  double cfl, eta, rho;
  bool operator<(const PlanKey& o) const {
    return std::memcmp(this, &o, sizeof(PlanKey)) < 0;
  }
};

// Pinned host staging for a descriptor array (an asynchronous copy from
// pageable memory would first wait for the stream to drain).
template <typename T>
struct PinnedArray {
  T* p = nullptr;
  size_t cap = 0;
  bool reserve(size_t n) {
    if (n <= cap) return true;
    if (p) cudaFreeHost(p);
    p = nullptr;
    cap = std::max<size_t>(n, 2 * cap);
    if (cudaMallocHost(&p, cap * sizeof(T)) != cudaSuccess) {
      cudaGetLastError();
      cap = 0;
      return false;
    }
    return true;
  }
  void free() {
    if (p) cudaFreeHost(p);
    p = nullptr;
    cap = 0;
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
  // phase boundaries of a cycle: 0 FCF start, 1 FCF end, 2 norms end, 4 coarse
  // start, 3 coarse end (read at the next cycle's synchronisation)
  cudaEvent_t ev[5] = {};
  int device = 0;          // the creating thread's device; the worker runs on it
  cudaEvent_t ev_front_done = nullptr;  // recorded after a cycle's relaxation and norms (no timing)
  // Device tap table: slot k holds the fine stencil (2k) and the coarse one
  // (2k+1) of an active solve, uploaded once at admission
  DevTaps* taps = nullptr;
  int slots = 0;
  std::vector<int> free_slots;
  // pinned staging: the outputs of the solves retired together, the cycle's
  // descriptors
  PinnedArray<double> stage;
  PinnedArray<BatchSolve> hS;
  PinnedArray<BatchItem> hItems;
  PinnedArray<int> hIds;
  double t_created = 0.0;
  bool cycled = false;     // ev[3] holds the previous cycle's end
  cudaStream_t upload = nullptr;    // admissions: set-up copies and initial residuals, beside the cycles
  cudaStream_t download = nullptr;  // retirements: output copies, beside the cycles
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
  if (r->slot >= 0) S->free_slots.push_back(r->slot);
  r->slot = -1;
  if (st == MGRIT_OK) S->stats.completed++;
  else S->stats.failed++;
  r->res.solve_s = now_s() - r->t_submit;
  r->res.dof_per_s = r->res.solve_s > 0 ? (double)r->prob.nx * r->prob.nt / r->res.solve_s : 0.0;
  r->state = 2;
}

// Admit queued requests that fit (called with the lock held; releases it
// around the host setup).  Returns the newly admitted requests.
// limit: most requests to admit in this call.  until: an event the cycle
// stream records when its relaxation is done; admission stops once it has
// completed (after at least one request), so the GPU does not wait for the
// host to finish admitting before the cycle's coarse solves are queued.
static std::vector<Request*> admit(mgrit_server* S, std::unique_lock<std::mutex>& lk, size_t limit = SIZE_MAX,
                                   cudaEvent_t until = nullptr) {
  std::vector<Request*> fresh;
  const size_t max_active = S->o.max_active > 0 ? (size_t)S->o.max_active : 4096;
  while (!S->queue.empty() && S->active.size() + fresh.size() < max_active && fresh.size() < limit) {
    if (until && !fresh.empty() && S->active.size() + fresh.size() >= kMinBatch && cudaEventQuery(until) == cudaSuccess)
      break;
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
    // set up on the upload stream, so that its copies (some from pageable
    // memory) and initial residual run beside the cycle the GPU is running
    mgrit_status st = handle_create(&r->prob, &r->opts, S->upload, cached, &r->h, false, true);
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
    if (S->free_slots.empty()) {
      lk.unlock();
      mgrit_destroy(r->h);
      r->h = nullptr;
      lk.lock();
      S->resident -= std::min(S->resident, r->bytes);
      r->bytes = 0;
      finish(S, r, MGRIT_ERR_OOM, "server tap table full");
      S->cv.notify_all();
      continue;
    }
    r->slot = S->free_slots.back();
    S->free_slots.pop_back();
    {
      mgrit_handle* h = r->h;
      const DevTaps* fine = h->fine_collapse ? &h->dphim : &h->dphi;
      cudaMemcpyAsync(S->taps + 2 * r->slot, fine, sizeof(DevTaps), cudaMemcpyHostToDevice, S->upload);
      cudaMemcpyAsync(S->taps + 2 * r->slot + 1, &h->dpsi.back(), sizeof(DevTaps), cudaMemcpyHostToDevice,
                      S->upload);
    }
    S->resident = S->resident - std::min(S->resident, r->bytes) + r->h->bytes;
    S->stats.peak_resident_bytes = std::max(S->stats.peak_resident_bytes, (double)S->resident);
    r->bytes = r->h->bytes;
    r->state = 1;
    fresh.push_back(r);
  }
  if (!fresh.empty()) {  // one sync of the upload stream for the batch: set-up errors and initial residuals
    lk.unlock();
    const cudaError_t e = cudaStreamSynchronize(S->upload);
    lk.lock();
    if (e != cudaSuccess) {
      cudaGetLastError();
      S->fatal = std::string("admission: ") + cudaGetErrorString(e);
    }
    for (Request* r : fresh) {
      r->r0 = std::sqrt(r->h->norm_host[0]);
      r->res.r0_norm = r->r0;
      r->h->stream = S->stream;  // every later launch of the solve is a cycle's
    }
  }
  return fresh;
}

// One MGRIT cycle for every active solve, in two halves around the one
// synchronisation of the cycle: cycle_front queues the batched FCF, residual
// and norm launches and the norms' read-back (the worker admits new requests
// while they run); cycle_back takes the stopping decisions and queues the
// coarse solves.  Called without the lock.
static mgrit_status cycle_front(mgrit_server* S, const std::vector<Request*>& act) {
  const int n = (int)act.size();
  std::vector<BatchSolve> hs(n);
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
    b.taps = 2 * act[k]->slot;
    b.psi = 2 * act[k]->slot + 1;
    b.cluster = h->march_cluster;
    b.sd = h->dsplan;
  }
  if (!S->dS.reserve(n) || !S->dIds.reserve(n) || !S->dNorm.reserve(n) || !S->hS.reserve(n) || !S->hIds.reserve(n))
    return fail(MGRIT_ERR_OOM, "server batch descriptors");
  std::memcpy(S->hS.p, hs.data(), n * sizeof(BatchSolve));
  cudaMemcpyAsync(S->dS.p, S->hS.p, n * sizeof(BatchSolve), cudaMemcpyHostToDevice, S->stream);
  // ---- batched FCF, one launch per (nx, launch shape): each solve keeps the
  // shape it was tuned to, so its arithmetic is the single-solve path's.
  // SDIRK fine levels: one launch per (nx, recurrence orders, precision).
  std::map<std::tuple<int, int, int, int>, std::vector<int>> groups, sgroups;
  for (int k = 0; k < n; ++k) {
    mgrit_handle* h = act[k]->h;
    if (h->sdirk)
      sgroups[{h->nx, h->splan.kf, h->splan.kb, hs[k].prec == 0 ? 0 : 1}].push_back(k);
    else
      groups[{h->nx, h->fine_tile, h->fine_threads, (h->fine_collapse ? h->dphim : h->dphi).span}].push_back(k);
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
  if (!S->dItems.reserve(items.size()) || !S->hItems.reserve(items.size()))
    return fail(MGRIT_ERR_OOM, "server batch items");
  std::memcpy(S->hItems.p, items.data(), items.size() * sizeof(BatchItem));
  const bool timed = S->ev[0] != nullptr;
  if (timed) cudaEventRecord(S->ev[0], S->stream);
  if (S->stats.cycles == 0 && S->stats.first_cycle_s == 0.0) S->stats.first_cycle_s = now_s() - S->t_created;
  cudaMemcpyAsync(S->dItems.p, S->hItems.p, items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice, S->stream);
  size_t gi = 0;
  for (auto& g : groups) {
    const int nx = std::get<0>(g.first), tile = std::get<1>(g.first), th = std::get<2>(g.first);
    const int span = std::get<3>(g.first);
    const auto rg = ranges[gi++];
    cudaError_t e = launch_fcf_batched(S->dS.p, S->dItems.p + rg.first, (int)(rg.second - rg.first), S->taps, nx,
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
  if (timed) cudaEventRecord(S->ev[1], S->stream);
  // ---- value-form residuals of the FP64 solves (no-op for the others)
  {
    cudaError_t e = launch_residual_value_batched(S->dS.p, S->dItems.p, (int)items.size(), S->stream);
    if (e != cudaSuccess) return launch_ok(e, "residual_value_batched");
  }
  // ---- norms of all solves, one read-back
  for (int k = 0; k < n; ++k) S->hIds.p[k] = k;
  cudaMemcpyAsync(S->dIds.p, S->hIds.p, n * sizeof(int), cudaMemcpyHostToDevice, S->stream);
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
  if (timed) cudaEventRecord(S->ev[2], S->stream);
  cudaMemcpyAsync(S->hNorm, S->dNorm.p, n * sizeof(double), cudaMemcpyDeviceToHost, S->stream);
  if (S->ev_front_done) cudaEventRecord(S->ev_front_done, S->stream);
  return MGRIT_OK;
}

static mgrit_status cycle_back(mgrit_server* S, const std::vector<Request*>& act, std::vector<char>* done) {
  const int n = (int)act.size();
  const bool timed = S->ev[0] != nullptr;
  cudaError_t e = cudaStreamSynchronize(S->stream);
  if (e != cudaSuccess) return launch_ok(e, "server cycle");
  if (timed) {
    float a = 0.0f, b = 0.0f, g = 0.0f;
    if (cudaEventElapsedTime(&a, S->ev[0], S->ev[1]) == cudaSuccess) S->stats.gpu_fcf_ms += a;
    if (cudaEventElapsedTime(&b, S->ev[1], S->ev[2]) == cudaSuccess) S->stats.gpu_norm_ms += b;
    if (S->cycled && cudaEventElapsedTime(&g, S->ev[3], S->ev[0]) == cudaSuccess) S->stats.gpu_gap_ms += g;
    float c = 0.0f;
    if (S->cycled && cudaEventElapsedTime(&c, S->ev[4], S->ev[3]) == cudaSuccess) S->stats.gpu_coarse_ms += c;
    cudaGetLastError();
  }
  if (timed) cudaEventRecord(S->ev[4], S->stream);
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
  // ---- few two-level solves: a Fourier-space coarse solve each (workspace set
  // up on first use, within the budget) when their summed cost is below the
  // batched march's, which is that of its longest march.  Estimates from the
  // measured kernels: a march step 0.6 us + 1 ns per point (a Psi step on the
  // cluster and its barrier); a Fourier-space solve 80 us + 0.04 ns per coarse
  // point (two transforms of log2 nx dependent stages and two scan passes).
  {
    double march_us = 0.0, fft_us = 0.0;
    for (auto& g : by_cluster)
      for (int k : g.second) {
        const mgrit_handle* h = act[k]->h;
        march_us = std::max(march_us, h->Nl[1] * (0.6 + 1e-3 * h->nx));
        fft_us += 80.0 + 4e-5 * (double)h->Nl[1] * h->nx;
      }
    if (fft_us < march_us) {
      std::lock_guard<std::mutex> lk(S->mu);
      for (auto& g : by_cluster) {
        std::vector<int> keep;
        for (int k : g.second) {
          Request* r = act[k];
          if ((double)(S->resident + coarse_fft_bytes(r->h)) <= S->o.hbm_budget_bytes && enable_coarse_fft(r->h)) {
            S->resident += r->h->bytes - std::min(r->h->bytes, r->bytes);
            r->bytes = r->h->bytes;
            S->stats.peak_resident_bytes = std::max(S->stats.peak_resident_bytes, (double)S->resident);
            S->stats.fft_coarse_solves++;
          } else {
            keep.push_back(k);
          }
        }
        g.second.swap(keep);
      }
      for (auto it = by_cluster.begin(); it != by_cluster.end();)
        it = it->second.empty() ? by_cluster.erase(it) : std::next(it);
    }
  }
  // ---- coarse solves: batched cluster marches (two-level), V-cycles (multilevel);
  // each group's solve ids at their own offset, so no group waits for another
  {
    size_t tot = 0;
    for (auto& g : by_cluster) tot += g.second.size();
    if (!S->dIds.reserve(std::max<size_t>(tot, (size_t)n))) return fail(MGRIT_ERR_OOM, "server batch ids");
  }
  size_t id_off = 0;
  for (auto& g : by_cluster) {
    int max_w = 0, max_halo = 0;
    for (int k : g.second) {
      const mgrit_handle* h = act[k]->h;
      max_w = std::max(max_w, (h->nx + g.first - 1) / g.first);
      max_halo = std::max(max_halo, h->dpsi.back().hi - h->dpsi.back().lo);
    }
    int* ids = S->dIds.p + id_off;
    id_off += g.second.size();
    cudaMemcpyAsync(ids, g.second.data(), g.second.size() * sizeof(int), cudaMemcpyHostToDevice, S->stream);
    e = launch_march_batched(S->dS.p, ids, (int)g.second.size(), S->taps, g.first, max_w, max_halo, S->stream);
    if (e != cudaSuccess) return launch_ok(e, "march_batched");
    for (int k : g.second) act[k]->h->kcount[MGRIT_K_MARCH]++;
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
  if (timed) {
    cudaEventRecord(S->ev[3], S->stream);  // read at the next cycle's synchronisation (or at exit)
    S->cycled = true;
  }
  return MGRIT_OK;
}

// Retire solves together, without the lock: their outputs come back through
// one pinned staging area on the download stream with one synchronisation, while
// the cycle stream runs the next cycle; then their device state is released
// (stream-ordered frees behind that cycle).  Nothing of the next cycle touches
// a retired solve's buffers.
static void retire_batch(mgrit_server* S, const std::vector<Request*>& done) {
  auto rows_of = [](const Request* r) {
    const mgrit_handle* h = r->h;
    return r->opts.output == MGRIT_OUT_FINAL ? (size_t)1
           : r->opts.output == MGRIT_OUT_CPOINTS ? (size_t)h->Nl[1] + 1 : (size_t)h->nt + 1;
  };
  auto wants = [](const Request* r) { return r->status == MGRIT_OK || r->status == MGRIT_ERR_NOT_CONVERGED; };
  std::vector<size_t> off(done.size(), 0);
  size_t total = 0;
  for (size_t k = 0; k < done.size(); ++k)
    if (wants(done[k])) {
      off[k] = total;
      total += rows_of(done[k]) * done[k]->h->nx;
    }
  const bool staged = S->stage.reserve(std::max<size_t>(total, 1));
  for (size_t k = 0; k < done.size(); ++k) {
    Request* r = done[k];
    if (!wants(r)) continue;
    mgrit_handle* h = r->h;
    h->stream = S->download;
    mgrit_status st = staged ? write_output(h, h->c[1 - r->cur], S->stage.p + off[k])
                             : fail(MGRIT_ERR_OOM, "pinned output staging");
    h->stream = S->stream;
    if (st != MGRIT_OK) {
      r->status = st;
      r->error = mgrit_last_error();
    }
  }
  const cudaError_t e = cudaStreamSynchronize(S->download);
  for (size_t k = 0; k < done.size(); ++k) {
    Request* r = done[k];
    mgrit_handle* h = r->h;
    if (wants(r)) {
      if (e != cudaSuccess) {
        r->status = MGRIT_ERR_CUDA;
        r->error = cudaGetErrorString(e);
      } else {
        const double* src = S->stage.p + off[k];
        r->out.assign(src, src + rows_of(r) * h->nx);
      }
    }
    collect_stats(h, &r->res);
    mgrit_destroy(h);  // device state released here, accounted under the lock by publish
    r->h = nullptr;
    r->res.solve_s = now_s() - r->t_submit;
    r->res.dof_per_s = r->res.solve_s > 0 ? (double)r->prob.nx * r->prob.nt / r->res.solve_s : 0.0;
  }
  if (e != cudaSuccess) cudaGetLastError();
}

// Under the lock: a retired request becomes visible to pollers.
static void publish(mgrit_server* S, Request* r) {
  S->resident -= std::min(S->resident, r->bytes);
  if (r->slot >= 0) S->free_slots.push_back(r->slot);
  r->slot = -1;
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
  if (cudaSetDevice(S->device) != cudaSuccess) {
    cudaGetLastError();
    S->fatal = "cudaSetDevice failed in the server worker";
  }
  if (!S->stream) {
    if (cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      S->fatal = "cudaStreamCreate failed";
    }
  }
  // the side streams run at the device's highest priority: their small
  // kernels (initial residuals, float-float output conversions) are scheduled
  // ahead of the pending CTAs of a running cycle instead of behind all of them
  int lo_prio = 0, hi_prio = 0;
  if (cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio) != cudaSuccess) {
    cudaGetLastError();
    hi_prio = 0;
  }
  if (cudaStreamCreateWithPriority(&S->upload, cudaStreamNonBlocking, hi_prio) != cudaSuccess ||
      cudaStreamCreateWithPriority(&S->download, cudaStreamNonBlocking, hi_prio) != cudaSuccess) {
    cudaGetLastError();
    S->fatal = "cudaStreamCreate failed (side streams)";
  }
  bool evs = true;
  for (auto& ev : S->ev)
    if (cudaEventCreate(&ev) != cudaSuccess) {
      cudaGetLastError();
      ev = nullptr;
      evs = false;
    }
  if (!evs)  // phase timing off
    for (auto& ev : S->ev) {
      if (ev) cudaEventDestroy(ev);
      ev = nullptr;
    }
  const int slots = S->o.max_active > 0 ? S->o.max_active : 4096;
  if (cudaMalloc(&S->taps, 2 * (size_t)slots * sizeof(DevTaps)) != cudaSuccess) {
    cudaGetLastError();
    S->taps = nullptr;
    S->fatal = "server tap table: cudaMalloc failed";
  } else {
    S->slots = slots;
    for (int k = slots - 1; k >= 0; --k) S->free_slots.push_back(k);
  }
  if (cudaEventCreateWithFlags(&S->ev_front_done, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    S->ev_front_done = nullptr;
  }
  bool queued = false;  // the active set's next cycle_front is already on the stream
  mgrit_status queued_status = MGRIT_OK;
  while (!S->stop) {
    if (!S->fatal.empty()) {
      for (Request* r : S->queue) finish(S, r, MGRIT_ERR_CUDA, S->fatal);
      S->queue.clear();
      S->cv.notify_all();
      S->cv.wait(lk, [&] { return S->stop || !S->queue.empty(); });
      continue;
    }
    if (S->active.empty()) {  // nothing running: admit a few, then cycle (more join during the cycles)
      queued = false;
      const double ta = now_s();
      std::vector<Request*> fresh = admit(S, lk, kStartBatch);
      S->stats.admit_s += now_s() - ta;
      for (Request* r : fresh) S->active.push_back(r);
      if (S->active.empty()) {
        S->cv.notify_all();
        S->cv.wait(lk, [&] { return S->stop || head_ready(S); });
      }
      continue;
    }
    std::vector<Request*> act = S->active;
    lk.unlock();
    const double tc = now_s();
    mgrit_status st = queued ? queued_status : cycle_front(S, act);
    queued = false;
    // admit while the GPU runs the cycle's relaxation (set-up on the upload stream)
    lk.lock();
    const double ta = now_s();
    std::vector<Request*> fresh = admit(S, lk, SIZE_MAX, S->ev_front_done);
    const double admit_dt = now_s() - ta;
    S->stats.admit_s += admit_dt;
    lk.unlock();
    std::vector<char> done(act.size(), 0);
    if (st == MGRIT_OK) st = cycle_back(S, act, &done);
    std::string msg = st == MGRIT_OK ? "" : mgrit_last_error();
    if (st != MGRIT_OK)
      for (size_t k = 0; k < act.size(); ++k) {
        done[k] = 1;
        act[k]->status = st;
        act[k]->error = msg;
      }
    std::vector<Request*> next, finished;
    for (size_t k = 0; k < act.size(); ++k) (done[k] ? finished : next).push_back(act[k]);
    for (Request* r : fresh) next.push_back(r);
    // queue the next cycle's relaxation behind this cycle's coarse solves before
    // retiring, so the GPU is not idle while the host copies outputs out
    if (!next.empty() && st == MGRIT_OK) {
      queued_status = cycle_front(S, next);
      queued = true;
    }
    const double tr = now_s();
    retire_batch(S, finished);
    const double te = now_s();
    lk.lock();
    for (Request* r : finished) publish(S, r);
    S->stats.cycles++;
    S->stats.cycle_s += tr - tc - admit_dt;
    S->stats.retire_s += te - tr;
    S->active_sum += (double)act.size();
    S->stats.mean_active = S->active_sum / (double)S->stats.cycles;
    S->active.swap(next);
    S->cv.notify_all();
  }
  if (S->ev[0] && S->cycled) {  // the last cycle's coarse solves
    float c = 0.0f;
    if (cudaEventSynchronize(S->ev[3]) == cudaSuccess && cudaEventElapsedTime(&c, S->ev[4], S->ev[3]) == cudaSuccess)
      S->stats.gpu_coarse_ms += c;
    cudaGetLastError();
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
  if (cudaGetDevice(&S->device) != cudaSuccess) {
    cudaGetLastError();
    S->device = 0;
  }
  S->o = *sopts;
  S->t_created = now_s();
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
  for (auto& ev : S->ev)
    if (ev) cudaEventDestroy(ev);
  if (S->stream) cudaStreamSynchronize(S->stream);
  if (S->ev_front_done) cudaEventDestroy(S->ev_front_done);
  if (S->taps) cudaFree(S->taps);
  S->stage.free();
  S->hS.free();
  S->hItems.free();
  S->hIds.free();
  if (S->upload) cudaStreamDestroy(S->upload);
  if (S->download) cudaStreamDestroy(S->download);
  S->dS.free();
  S->dItems.free();
  S->dTaps.free();
  S->dIds.free();
  S->dNorm.free();
  if (S->hNorm) cudaFreeHost(S->hNorm);
  delete S;
}
