// Kernel argument blocks shared by the host driver and the CUDA kernels.
// Internal interface (not part of the ABI).
#pragma once
#include <cuda_runtime.h>

namespace mg {

constexpr int kMaxDevTaps = 256;
constexpr int kMaxSpan = 256;

// A circulant stencil passed by value in the kernel parameter space (or
// copied into shared memory by the batched kernels):
// (T v)_r = sum_t c[t] v_{r + off[t]}.  lo <= 0 <= hi bound the offsets.
// The dense form d64/d32 holds the coefficients of offsets lo..hi (zeros for
// absent offsets) when span = hi - lo + 1 <= kMaxSpan (else span = 0).
// shift (sigma) is the moving-frame shift used by the sequential march.
struct DevTaps {
  int n, lo, hi, span;
  int shift;
  float one;       // 1.0f, read at run time (see the float-float accumulation)
  int pad1, pad2;
  int off[kMaxDevTaps];
  double c64[kMaxDevTaps];
  float c32[kMaxDevTaps];
  double d64[kMaxSpan];
  float d32[kMaxSpan];
  // float-float split of the coefficients (c = hi + lo, |lo| <= ulp(hi)/2)
  float chi[kMaxDevTaps], clo[kMaxDevTaps];
  float dhi[kMaxSpan], dlo[kMaxSpan];
};

// Fill a DevTaps from n (offset, coefficient) pairs; false if n > kMaxDevTaps.
bool make_dev_taps(const int* off, const double* coef, int n, DevTaps* out);

// FCF-relaxation of one level with the fused C-point residual.
// Interval j = 1..N starts at C-point j-1.  For every j the kernel computes
//   v_j   = m steps of u <- T u + g from u_old[C(j-1)]   (F- then C-relaxation)
//   rho_j = v_j - u_old[C(j)];  c_new[j] = v_j
//   r_{j+1} = T^m rho_j  (j < N)  = residual at C-point j+1 after the second
//   F-relaxation, and partial[j] = ||r_{j+1}||^2.
struct FcfArgs {
  const double* u_old;     // C-point j at u_old + j*cstride (unused if zero_old)
  long long cstride;
  double* c_new;           // c_new + j*nx
  const double* g;         // right-hand side, point n at g + n*nx (nullptr: none)
  double* r;               // r + j*nx, j = 2..N written
  double* partial;         // partial[j], j = 1..N-1 (nullptr: skip)
  int nx, m, N, zero_old;  // zero_old: u_old is identically zero
};

// Sequential march u_n = T u_{n-1} + g_n, n = 1..P-1, on one thread-block
// cluster whose CTAs split x; halos move through distributed shared memory.
struct MarchArgs {
  const double* init;      // u_0 (nullptr: zero)
  const double* g;         // point n at g + n*nx (nullptr: none)
  double* u_out;           // store u_n at u_out + (n/store_every)*nx when n % store_every == 0
  int store_every;
  double* c_add;           // c_add + n*nx += u_n for n >= 1 (nullptr: none)
  int nx, P;
};

// Correction and F-relaxation (ideal interpolation) of one level:
// u[(j-1)m] = c_new[j-1] + e[j-1], then m-1 steps with g; interval N also
// writes u[Nm] = c_new[N] + e[N].  e == nullptr reads as zero (final
// interpolation of the fine level's F-points from its C-points).
struct CorrectArgs {
  const double* c_new;     // c_new + j*nx
  const double* e;         // e + j*nx (next level's solution)
  const double* g;         // point n at g + n*nx (nullptr: none)
  double* u;               // all points of the level, point n at u + n*nx
  int nx, m, N;
};

// tile: register tile (0, 4 or 8), kFixedTile for the fixed-span path of the
// collapsed ERK stencils; -1 = the default for this stencil and nx.
constexpr int kFixedTile = 99;
cudaError_t launch_fcf(const FcfArgs& a, const DevTaps& t, int precision, int threads,
                       cudaStream_t s, int tile = -1);

// Shared-memory slab length for nx points in the padded layout (one pad
// element per 8 so that per-thread chunks of 8 are bank-conflict free).
__host__ __device__ inline int padded_len(int nx) { return nx + (nx >> 3) + 1; }

// ------------------------------------------------------- device-side cycle test
// State of the stopping test when a whole solve runs as one CUDA graph: the
// check kernel reads ||r||^2 (and ||r^(0)||^2), records the relative
// residual, and drives the graph's WHILE/IF conditions.
struct CheckState {
  double r0sq;            // ||r^(0)||^2 (written by the initial-residual kernel)
  double tol;
  int max_iter;
  int it;                 // coarse corrections applied so far
  int done;               // 1 once the test has stopped the loop
  int status;             // mgrit_status of the stop
  int result_cur;         // buffer index read by the final FCF (result in c[1-cur])
  int nhist;
  double rel;
  double hist[128];
};
cudaError_t launch_check(const double* norm2, CheckState* st, unsigned long long while_handle,
                         unsigned long long if_handle, int cur, cudaStream_t s);

// ------------------------------------------------------------- SDIRK steps
// One SDIRK step (stage form, Appendix A tableaux):
//   K_i = M^{-1} dtL (u + sum_{j<i} a_ij K_j),  M = I - gamma dtL,
//   u_new = u + sum_i b_i K_i  (stiffly accurate: b = last row of A).
// M = E^{-ql} p_d prod_r (E - z_r), E the forward shift: each linear factor is
// a periodic first-order recurrence solved by a chunked parallel scan in its
// stable direction (forward if |z_r| < 1, backward otherwise) closed by an
// exact rank-one periodic wrap.
constexpr int kMaxStages = 5;
constexpr int kMaxFactors = 5;
struct SdirkPlan {
  int s;                        // stages
  int nL;                       // taps of dt L
  int ql;                       // input shift of the solve
  int nf;                       // linear factors of M
  int offL[6];
  double cL[6];
  float cL32[6];
  double a[kMaxStages][kMaxStages];
  float a32[kMaxStages][kMaxStages];
  double gamma;
  float gamma32;
  int dir[kMaxFactors];         // +1: forward recurrence x_i = m x_{i-1} + b_i; -1: backward
  double mre[kMaxFactors], mim[kMaxFactors];   // recurrence multiplier m (|m| < 1)
  double bscale_re[kMaxFactors], bscale_im[kMaxFactors];  // input scale of the factor
  double inv_pd;                // 1 / leading coefficient
};
int sdirk_slots(const SdirkPlan& p);                      // shared slabs a step needs
size_t sdirk_smem(const SdirkPlan& p, int nx, int prec);  // bytes of an FCF CTA
int sdirk_threads(int nx);                                // CTA size (0: nx unsupported)
cudaError_t launch_fcf_sdirk(const FcfArgs& a, const SdirkPlan& p, int precision, cudaStream_t s);
cudaError_t launch_propagate_sdirk(const double* in, double* out, int count, int nx, int k, const SdirkPlan& p,
                                   double* partial, cudaStream_t s);
cudaError_t launch_interp_sdirk(const double* c, double* u, int nx, int m, int N, const SdirkPlan& p,
                                cudaStream_t s);
cudaError_t launch_seq_sdirk(const double* u0, double* out, int nx, int P, int store_every, const SdirkPlan& p,
                             cudaStream_t s);

// ------------------------------------------------------------ batched solves
// One entry per active solve of a batched launch (server).
struct BatchSolve {
  FcfArgs fcf;         // level-1 FCF arguments (host updates u_old/c_new per cycle)
  int prec;            // 0 FP64, 1 mixed
  int taps;            // index of the fine stencil in the taps array
  int psi;             // index of the coarse stencil (two-level march)
  int cluster;         // CTAs per march cluster
};
struct BatchItem {
  int solve, j;        // solve index, interval j (1..N)
};
cudaError_t launch_fcf_batched(const BatchSolve* S, const BatchItem* items, int nitems, const DevTaps* taps,
                               int max_nx, int threads, int tile, int span, cudaStream_t s);
int default_threads(int nx, int tile);        // CTA size the launches pick for nx
int default_tile(const DevTaps& t, int nx);   // register tile the launches pick
cudaError_t launch_norm_batched(const BatchSolve* S, const int* ids, int count, double* out, cudaStream_t s);
cudaError_t launch_march_batched(const BatchSolve* S, const int* ids, int count, const DevTaps* taps, int cluster,
                                 int max_w, int max_halo, cudaStream_t s);
cudaError_t launch_march(const MarchArgs& a, const DevTaps& t, int cluster, int threads,
                         cudaStream_t s);
cudaError_t launch_correct(const CorrectArgs& a, const DevTaps& t, int threads, cudaStream_t s, int fp32 = 0);
cudaError_t launch_norm(const double* partial, int n, double* out, cudaStream_t s);
cudaError_t launch_add(double* c, const double* e, long long count, cudaStream_t s);
cudaError_t launch_propagate(const double* in, double* out, int count, int nx, int k,
                             const DevTaps& t, double* partial, int threads, cudaStream_t s);
int march_max_cluster();
void set_tile(int r);   // register tile of the stencil kernels: 8, 4 or 0
int get_tile();

}  // namespace mg
