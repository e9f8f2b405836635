// Internal interface shared by the C ABI's translation units (driver.cpp,
// server.cpp): the handle of one solve and the helpers that build, run and
// release it.  Not part of the ABI.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/mgrit.h"
#include "device.h"
#include "setup.h"

struct DevBuf {
  double* p = nullptr;
  size_t n = 0;
  mgrit_free_fn freefn = nullptr;
  void* ctx = nullptr;
};

struct mgrit_handle {
  mgrit_problem prob;
  mgrit_opts opts;
  cudaStream_t stream = nullptr;
  int nx = 0, nt = 0, m = 0, L = 0;
  std::vector<int> Nl;            // Nl[l] intervals of level l (l = 1..L-1)
  mg::Taps phi;                       // fine propagator (ERK, collapsed)
  std::vector<mg::CoarseOp> ops;      // ops[l-2] = Psi_l, l = 2..L
  mg::DevTaps dphi;
  mg::DevTaps dphim;                  // Phi^m as one stencil (ERK, if <= 256 taps)
  bool have_phim = false;
  bool sdirk = false;             // fine level is SDIRK (stage solves)
  mg::SdirkPlan splan;            // host copy (its table pointers are device addresses)
  mg::SdirkPlan* dsplan = nullptr;  // device copy (batched launches)
  bool redisc = false;              // Psi = the SDIRK step at m dt (cplan)
  mg::SdirkPlan cplan;
  std::vector<mg::DevTaps> dpsi;      // dpsi[l-2]
  // Inflow/outflow boundaries (Section 4.5): the rows of Phi and Phi^m that
  // differ from the circulant (device tables); every Psi_l is truncated at
  // both ends by the kernels' loads
  bool inflow = false;
  // coarsest-level solve in Fourier space (periodic, nx a power of two)
  bool fft_coarse = false;
  mg::CoarseFft cfft = {};
  mg::Fixup fx_phi = {};
  mg::Fixup fx_phim = {};             // of Phi^m (the collapsed path)
  std::vector<DevBuf> bufs;       // everything allocated, for release
  // A server's handle allocates from the stream-ordered pool of its stream
  // (cudaMallocAsync) whatever allocator mgrit_set_allocator installed: the
  // server's worker thread admits thousands of solves, and callbacks into a
  // host language per buffer stalled it (seconds per 4096-solve batch).
  bool pool_alloc = false;
  double* c[2] = {nullptr, nullptr};
  std::vector<double*> r, u, cnew;  // indexed by level (size L+1)
  // Mixed modes keep level 1's residual and every coarse-level array in FP32
  // (rf, uf, cnewf; the FP64 pointers of those arrays stay null).
  bool f32c = false;
  std::vector<float*> rf, uf, cnewf;
  // MIXED_DF on an ERK fine level: c[0], c[1] hold float-float pairs
  // (hi, lo) instead of FP64 values, converted only at load and output
  bool dfc = false;
  double* u0buf = nullptr;        // u0 in FP64 (the initial residual reads it)
  int last = -1;                  // c[last]: C-points of the last solve (-1: none yet)
  double r0_last = 0.0;           // that solve's initial residual norm
  double* partial = nullptr;
  double* scratch = nullptr;      // 2*nx + 1 doubles
  double* norm_host = nullptr;    // pinned
  int fcf_threads = 512, march_cluster = 1, march_threads = 256;
  int fine_tile = -1, fine_threads = 0;   // level-1 FCF launch shape (autotuned)
  int fine_collapse = 0;                  // 1: each pass applies Phi^m once
  // MIXED, periodic, nx = 2^p: the level-1 FCF may take its FP64 pass in
  // Fourier space (twiddles and the symbol of Phi^m / (2 nx) in ftab on the
  // device); fine_fourier = its CTA size when the autotuner picked it, else 0
  double* ftab = nullptr;
  int fine_fourier = 0;
  // a whole solve as one CUDA graph (WHILE over cycles, IF around each
  // coarse correction), built at the first solve
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  cudaStream_t cap_stream = nullptr;
  bool graph_failed = false;
  int graph_coarse_launches = 0;          // kernels of one coarse correction
  mg::CheckState* dstate = nullptr;       // device
  mg::CheckState* hstate = nullptr;       // pinned host
  // mgrit_solve_async: one pinned CheckState slot, one event and the enqueue
  // time per outstanding solve, finished in order by mgrit_solve_wait
  mg::CheckState* ring = nullptr;         // pinned, MGRIT_MAX_INFLIGHT slots
  cudaEvent_t ring_ev[MGRIT_MAX_INFLIGHT] = {};
  double ring_t0[MGRIT_MAX_INFLIGHT] = {};
  int ring_r0_launches[MGRIT_MAX_INFLIGHT] = {};
  int ring_head = 0, ring_count = 0;
  bool iterate_random = false;            // load_iterate drew the random iterate
  // per-solve launch accounting (and CUDA-event timing with MGRIT_FLAG_TIME_KERNELS)
  int kcount[MGRIT_K_KINDS] = {0};
  std::vector<cudaEvent_t> evpool;
  std::vector<int> evkind;      // kind of each recorded (start, stop) pair
  size_t evused = 0;
  double setup_s = 0.0, op_complexity = 0.0;
  double tune_s = 0.0;            // of setup_s: timing launch shapes
  size_t bytes = 0;
};


mgrit_status fail(mgrit_status s, const std::string& msg);
double now_s();
mgrit_status dalloc(mgrit_handle* h, size_t count, double** out);
void release(mgrit_handle* h);
mg::DevTaps to_dev(const mg::Taps& t);
bool is_device_ptr(const void* p);
cudaMemcpyKind kind_to_dev(const void* src);
cudaMemcpyKind kind_from_dev(const void* dst);
mgrit_status validate_problem(const mgrit_problem* p);
mgrit_status validate_opts(const mgrit_problem* p, const mgrit_opts* o);
// Physical spacings of Eq. 1's grid: dx = (xmax - xmin)/nx, dt = c dx/alpha.
void grid_spacings(const mgrit_problem* p, double* dx, double* dt);
mgrit_status plan(const mgrit_problem* p, const mgrit_opts* o, std::vector<mg::CoarseOp>* ops);
int pick_cluster(int nx, const mg::Taps& t);
mgrit_status launch_ok(cudaError_t e, const char* what);
void reset_stats(mgrit_handle* h);
cudaEvent_t next_event(mgrit_handle* h);
void collect_stats(mgrit_handle* h, mgrit_result* R);
mgrit_status run_march(mgrit_handle* h, const mg::MarchArgs& a, const mg::DevTaps& t);
// The coarsest-level solve (a march without initial value): in Fourier space
// when the handle has the workspace, else the cluster march.
mgrit_status run_coarse_solve(mgrit_handle* h, const mg::MarchArgs& a, const mg::DevTaps& t);
mgrit_status initial_residual(mgrit_handle* h, const double* u0dev, double* r0);
mgrit_status initial_residual_async(mgrit_handle* h, const double* u0dev);
// ||r^(0)||^2 of the loaded iterate into the device double dst: the random
// iterate's space-time residual, or ||Phi u0||^2 for the zero iterate.
// Returns the number of kernels launched through *launches.
mgrit_status enqueue_r0sq(mgrit_handle* h, double* dst, int* launches);
// Initial iterate into the handle's C-point arrays (u0 with a zero iterate,
// or all C-points c_init); u0 in FP64 into u0buf.
mgrit_status load_iterate(mgrit_handle* h, const double* u0, const double* c_init);
mgrit_status coarse_cycle(mgrit_handle* h, double* c_new);
// Two-level periodic solve (nx = 2^p, at least 16 coarse steps): allocate and
// fill the Fourier-space coarse solve's workspace on the handle's stream and
// use it from then on; false (nothing changed) where it does not apply.
bool enable_coarse_fft(mgrit_handle* h);
size_t coarse_fft_bytes(const mgrit_handle* h);  // device bytes enable_coarse_fft adds
// Build a handle; ops != nullptr supplies an already fitted hierarchy.
// batched: a server's handle.  Its two-level coarse solves run in the
// server's batched march (with about a thousand solves active, one batched
// launch beats per-solve transforms), so no Fourier-space workspace.
mgrit_status handle_create(const mgrit_problem* prob, const mgrit_opts* opts, cudaStream_t stream,
                           const std::vector<mg::CoarseOp>* ops, mgrit_handle** out,
                           bool sync = true, bool batched = false);
// Device bytes a handle for this request will allocate (admission control).
size_t handle_bytes(const mgrit_problem* prob, const mgrit_opts* opts);
// SDIRK stage-solve plan for the problem (factored stage matrix), checked on
// the host against the stage matrix itself.
mgrit_status make_sdirk_plan(const mgrit_problem* prob, mg::SdirkPlan* out, std::vector<double>* tables);
// Fine-level FCF arithmetic of a handle: 0 FP64, 1 FP64 + FP32, 3 float-float + FP32.
int fine_prec(const mgrit_handle* h);
// Pick the level-1 FCF launch shape (register tile, CTA size) by timing the
// candidates on the handle's buffers; cached per shape key for the process.
void autotune_fine(mgrit_handle* h);
// Launch the fine-level FCF (ERK stencil or SDIRK) of a handle.
cudaError_t launch_fine_fcf(mgrit_handle* h, const mg::FcfArgs& f, int prec);
// Copy the converged C-points cres out per opts.output (FULL interpolates).
mgrit_status write_output(mgrit_handle* h, const double* cres, double* out);

// Launch one kernel of `kind` through fn(); counts it and, when asked,
// brackets it with CUDA events on the handle's stream.
template <typename F>
inline mgrit_status klaunch(mgrit_handle* h, int kind, const char* what, F&& fn) {
  const bool timed = (h->opts.flags & MGRIT_FLAG_TIME_KERNELS) != 0;
  cudaEvent_t e0 = timed ? next_event(h) : nullptr;
  if (e0) cudaEventRecord(e0, h->stream);
  mgrit_status st = fn();
  if (st != MGRIT_OK) return st;
  if (e0) {
    cudaEvent_t e1 = next_event(h);
    if (e1) {
      cudaEventRecord(e1, h->stream);
      h->evkind.push_back(kind);
    } else {
      h->evused--;
    }
  }
  h->kcount[kind]++;
  (void)what;
  return MGRIT_OK;
}

