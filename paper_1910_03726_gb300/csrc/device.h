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

// Rows of a level's operator that differ from its circulant on the
// non-periodic domain (Section 4.5): rows 0..nl-1 read columns 0..cl-1, rows
// nx-nr..nx-1 read columns nx-cr..nx-1; coefficients row-major, left block
// first, in FP64 (w64) and FP32 (w32), device memory.  The stencil kernels
// compute every row as the circulant and then overwrite these rows
// ("fix-up"); nl = nr = 0 (periodic) skips it.
struct Fixup {
  int nl, cl, nr, cr;
  const double* w64;
  const float* w32;
};

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
  int relax_f;             // F-relaxation only: c_new = u_old, r_j = Phi^m c_{j-1} - c_j (j = 1..N)
  // Value-form residual (FP64, level 1): the second pass propagates c_new_j
  // itself and stores Phi^m c_new_j in r row j+1; residual_value then forms
  // r_{j+1} = Phi^m c_new_j - c_new_{j+1} (the oracle's form, whose
  // cancellation keeps exact C-points bitwise exact) and the norms.
  int value_residual;
  // FP32 storage (mixed modes): r_f replaces r (any precision); on an FP32
  // coarse level (precision 2) u_old_f, c_new_f, g_f and r_f replace all four.
  const float* u_old_f;
  float* c_new_f;
  const float* g_f;
  float* r_f;
  Fixup fx;                // boundary rows of T (non-periodic problems)
  int trunc;               // T truncated at both ends: taps outside 0..nx-1 read zero
  // Precision 3: u_old and c_new hold float-float pairs (hi, lo) instead of
  // FP64 values (same 8 bytes), so level 1 runs on the FP32 pipes only.
  int df_store;
  int fused;               // set by launch_fcf only: the fused narrow-stencil body runs
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
  const float* g_f;        // FP32 right-hand side (replaces g when set)
  float* u_out_f;          // FP32 output (replaces u_out when set)
  // T truncated at both ends (Toeplitz, inflow/outflow Psi): a tap whose
  // column (in the frame that does not move) leaves 0..nx-1 drops out.
  int trunc;
  int c_add_df;            // c_add holds float-float pairs
};

// Coarse solve of a periodic level in Fourier space (fft.cu): the march
// e_n = Psi e_{n-1} + g_n becomes, per mode k, E_n = mu_k E_{n-1} + G_n.
// spec: rows x (nx/2 + 1) complex FP64 (re, im interleaved) of workspace,
// rows >= P - 1; tw: nx/2 twiddles exp(-2 pi i k / nx); mu: the symbols
// mu_k = sum_i psi_i exp(+2 pi i i k / nx), k < nx.  All device memory.
struct CoarseFft {
  double* spec;
  int rows;
  const double* tw;
  const double* mu;
  double* carry;           // kMaxScanBlocks x (nx/2 + 1) complex: last value of each block of rows
};
constexpr int kMaxScanBlocks = 64;  // blocks of the chunked scan over the coarse steps
bool fft_coarse_supported(int nx);   // nx = 2^p, 64 <= nx <= 8192
// Fill tw (nx/2 complex) and mu (nx complex) of CoarseFft from the stencil.
cudaError_t launch_fft_tables(const DevTaps& psi, int nx, double* tw, double* mu, cudaStream_t s);
// Same result as launch_march with a.init == nullptr and periodic T (three
// launches: forward transforms, recurrences, inverse transforms + epilogue).
cudaError_t launch_coarse_fft(const MarchArgs& a, const CoarseFft& f, cudaStream_t s);
// Kernels launch_coarse_fft issues for P time levels (three or four).
int coarse_fft_launches(int nx, int P);

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
  // FP32 storage (an FP32 coarse level): used by the FP32 kernel instead
  const float* c_new_f;
  const float* e_f;
  const float* g_f;
  float* u_f;
  Fixup fx;                // boundary rows of T (non-periodic problems)
  int trunc;               // T truncated at both ends
};

// tile: register tile (0, 4 or 8), kFixedTile for the fixed-span path of the
// collapsed ERK stencils; -1 = the default for this stencil and nx.
constexpr int kFixedTile = 99;
// kChunkTile: any dense span, taken in chunks of 8 taps whose window of
// R + 7 inputs is loaded into registers once per chunk (R = 8).
constexpr int kChunkTile = 98;
cudaError_t launch_fcf(const FcfArgs& a, const DevTaps& t, int precision, int threads,
                       cudaStream_t s, int tile = -1);

// Level-1 FCF (MIXED, periodic) with the FP64 pass Phi^m c_{j-1} taken in
// Fourier space: forward FFT of the slab, product with the collapsed
// stencil's symbol, inverse FFT; the residual's pass is the MIXED body's with
// the collapsed stencil t (a.m = 1).  tab (fourier_table_doubles(nx) doubles,
// 16-byte aligned) is filled by launch_fourier_tables(t, ...): twiddles and
// the symbol.  threads: 128 or 256.
bool fourier_fcf_supported(int nx);  // nx = 2^p, 256 <= nx <= 8192
bool fourier_fcf_args_ok(const FcfArgs& a);
size_t fourier_table_doubles(int nx);
cudaError_t launch_fourier_tables(const DevTaps& t, int nx, double* tab, cudaStream_t s);
cudaError_t launch_fcf_fourier(const FcfArgs& a, const DevTaps& t, const double* tab, int threads, cudaStream_t s);

// Shared-memory slab length for nx points in the padded layout (one pad
// element per 8 so that per-thread chunks of 8 are bank-conflict free).
__host__ __device__ inline int padded_len(int nx) { return nx + (nx >> 3) + 1; }
// The FCF and propagation kernels hold two padded FP64 slabs in dynamic
// shared memory, beside their static shared memory: at most 227 KiB per CTA
// in all.  kSlabStaticReserve covers the largest static part of those kernels
// (the batched FCF's copy of its stencil, 11.3 KiB; the others' reduction
// scratch, 256 B): nx <= kMaxSlabNx.
constexpr int kMaxSmemBytes = 227 * 1024;
constexpr int kSlabStaticReserve = 12 * 1024;
__host__ __device__ constexpr bool slab_pair_fits(int nx) {
  return 2LL * (nx + (nx >> 3) + 1) * (long long)sizeof(double) <= kMaxSmemBytes - kSlabStaticReserve;
}
constexpr int kMaxSlabNx = 12231;
static_assert(slab_pair_fits(kMaxSlabNx) && !slab_pair_fits(kMaxSlabNx + 1), "kMaxSlabNx");

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
  double diverge;         // stop as diverged above this ratio (<= 0: only when not finite)
};
cudaError_t launch_check(const double* norm2, CheckState* st, unsigned long long while_handle,
                         unsigned long long if_handle, int cur, cudaStream_t s);

// ------------------------------------------------------------- SDIRK steps
// One SDIRK step (stage form, Appendix A tableaux, all stiffly accurate):
//   (I - gamma dtL) K_i = dtL A_i,  A_i = u + sum_{j<i} a_ij K_j,
//   u_new = A_s + gamma K_s.
// With M = I - gamma dtL the stage is K_i = (M^{-1} A_i - A_i) / gamma, so a
// stage is one periodic banded solve and no separate application of dtL.
// M = p_d E^{lo} prod_r (E - z_r) (E the forward shift) splits into
//   forward part  prod_{|z|<1} (I - z S),   S = E^{-1}: x_i = sum_q af_q x_{i-q} + y_i
//   backward part prod_{|z|>1} (I - E/z):             x_i = sum_q ab_q x_{i+q} + y_i
// (real coefficients: conjugate roots stay on one side), a shift E^{ql} and a
// scale.  Each periodic recurrence runs as a chunked parallel scan over the
// slab (C points per thread, warp-shuffle and cross-warp scans of the K-vector
// states with the powers of the companion matrix, exact periodic closure
// (I - T^nx)^{-1}); every table is computed on the host in FP64.
constexpr int kMaxStages = 5;
constexpr int kMaxRec = 5;       // order of one directional recurrence
constexpr int kSdirkCMax = 16;   // points per thread
struct SdirkPlan {
  int s;                 // stages
  int kf, kb;            // orders of the forward / backward recurrences
  int ql;                // input shift of the solve: x_i = y_{i+ql}
  int C, threads;        // points per thread and CTA size, nx = threads * C
  int nx;
  int tab_len;           // elements of one precision's recurrence tables
  int steps_f, steps_b;  // warp-scan doubling steps that matter per direction
  int trunc_f, trunc_b;  // 1: A^32 below rounding (previous-warp carry only)
  double a[kMaxStages][kMaxStages];
  float a32[kMaxStages][kMaxStages];
  double gamma, inv_gamma, scale;   // scale = 1 / (p_d prod_{|z|>1} (-z))
  float gamma32, inv_gamma32, scale32;
  double af[kMaxRec], ab[kMaxRec];  // recurrence coefficients (host copy)
  const double* tab64;   // device: tables, FP64
  const float* tab32;    // device: tables, FP32
};
// Elements of the tables of one direction of order K with C points per
// thread: a[K], (A^k)_{k=0..32}, ((A^32)^k)_{k=0..16} (A = T^C, T the
// companion matrix, K x K row-major), G[C][K] (row 0 of T^{c+1}) and
// Q = (I - T^nx)^{-1}.
__host__ __device__ constexpr int sdirk_rec_len(int K, int C) { return K == 0 ? 0 : K + 51 * K * K + C * K; }
int sdirk_slots(const SdirkPlan& p);                      // shared slabs a step needs
size_t sdirk_smem(const SdirkPlan& p);                    // bytes of shared memory of a CTA
int sdirk_threads(int nx);                                // CTA size (0: nx unsupported)
bool sdirk_orders_supported(int kf, int kb);
cudaError_t launch_fcf_sdirk(const FcfArgs& a, const SdirkPlan& p, int precision, cudaStream_t s);
cudaError_t launch_propagate_sdirk(const double* in, double* out, int count, int nx, int k, const SdirkPlan& p,
                                   double* partial, cudaStream_t s);
cudaError_t launch_interp_sdirk(const double* c, double* u, int nx, int m, int N, const SdirkPlan& p,
                                cudaStream_t s);
cudaError_t launch_seq_sdirk(const double* u0, double* out, int nx, int P, int store_every, const SdirkPlan& p,
                             cudaStream_t s);
// Two-level coarse solve with the rediscretised SDIRK step (one CTA):
// e_0 = 0, e_n = Phi_c e_{n-1} + g_n, c_add[n] += e_n for n = 1..P-1; g is
// FP64 (g) or FP32 (g_f, used when set).
cudaError_t launch_coarse_march_sdirk(const double* g, const float* g_f, double* c_add, int nx, int P,
                                      const SdirkPlan& p, cudaStream_t s);

// ------------------------------------------------------------ batched solves
// One entry per active solve of a batched launch (server).
struct BatchSolve {
  FcfArgs fcf;         // level-1 FCF arguments (host updates u_old/c_new per cycle)
  int prec;            // 0 FP64, 1 mixed
  int taps;            // index of the fine stencil in the taps array
  int psi;             // index of the coarse stencil (two-level march)
  int cluster;         // CTAs per march cluster
  const SdirkPlan* sd; // device copy of the SDIRK plan (SDIRK fine levels)
};
struct BatchItem {
  int solve, j;        // solve index, interval j (1..N)
};
cudaError_t launch_fcf_batched(const BatchSolve* S, const BatchItem* items, int nitems, const DevTaps* taps,
                               int max_nx, int threads, int tile, int span, cudaStream_t s);
// SDIRK fine levels of several solves with the same nx, recurrence orders and
// precision; smem_bytes = the largest sdirk_smem of the group.
cudaError_t launch_fcf_sdirk_batched(const BatchSolve* S, const BatchItem* items, int nitems, const SdirkPlan& any,
                                     size_t smem_bytes, int precision, cudaStream_t s);
int default_threads(int nx, int tile);        // CTA size the launches pick for nx
int default_tile(const DevTaps& t, int nx);   // register tile the launches pick
cudaError_t launch_norm_batched(const BatchSolve* S, const int* ids, int count, double* out, cudaStream_t s);
cudaError_t launch_march_batched(const BatchSolve* S, const int* ids, int count, const DevTaps* taps, int cluster,
                                 int max_w, int max_halo, cudaStream_t s);
cudaError_t launch_march(const MarchArgs& a, const DevTaps& t, int cluster, int threads,
                         cudaStream_t s);
cudaError_t launch_correct(const CorrectArgs& a, const DevTaps& t, int threads, cudaStream_t s, int fp32 = 0);
cudaError_t launch_norm(const double* partial, int n, double* out, cudaStream_t s);
// Bitwise comparison of the integer-pipe binary32 -> binary64 conversion with
// the conversion instruction over 2n hashed patterns; mismatches added to *bad.
cudaError_t launch_conversion_check(unsigned long long n, unsigned long long seed, unsigned long long* bad,
                                    cudaStream_t s);
// r[j+1] -= c_new[j+1] and partial[j] = ||r[j+1]||^2 for j = 1..N-1.
cudaError_t launch_residual_value(const double* c_new, double* r, double* partial, int nx, int N, cudaStream_t s);
cudaError_t launch_residual_value_batched(const BatchSolve* S, const BatchItem* items, int nitems, cudaStream_t s);
cudaError_t launch_add(double* c, const double* e, long long count, cudaStream_t s);
cudaError_t launch_add_f(double* c, const float* e, long long count, cudaStream_t s, int df_store = 0);
// FP64 <-> float-float pairs, count values (to_df: in FP64, out pairs).
cudaError_t launch_convert_df(const double* in, double* out, long long count, int to_df, cudaStream_t s);
cudaError_t launch_propagate(const double* in, double* out, int count, int nx, int k,
                             const DevTaps& t, double* partial, int threads, cudaStream_t s,
                             const Fixup* fx = nullptr, int trunc = 0);
// Sequential stepping of a non-periodic level on one CTA (the slab stays in
// shared memory): u_n = T u_{n-1}, n = 1..P-1, u_n stored at
// out + (n/store_every)*nx when n % store_every == 0 (u_0 is not written).
cudaError_t launch_seq_slab(const double* u0, double* out, int nx, int P, int store_every, const DevTaps& t,
                            const Fixup& fx, int threads, cudaStream_t s);
// ------------------------------------------------- random initial iterate
// The paper's tests start from a uniformly random space-time iterate
// (Section 2.2).  Point i of time level n draws Philox4x32-10 (Salmon,
// Moraes, Dror, Shaw, SC'11: counter (i, n, 0, 0), key (seed lo, seed hi))
// and joins its first two words into a double in [0, 1) with 53 random bits.
// rows slabs: slab k is time level n = first_n + k * stride_n (u0 where n = 0).
cudaError_t launch_random_rows(double* out, const double* u0, int nx, long long first_n, long long stride_n,
                               int rows, unsigned long long seed, cudaStream_t s);
// partial[k] = || phi_u[k] - u_{first_n + k + 1} ||^2 for the random levels u_n
// (the space-time residual of the random iterate, one slab per CTA).
cudaError_t launch_random_residual(const double* phi_u, double* partial, int nx, long long first_n, int rows,
                                   unsigned long long seed, cudaStream_t s);
// *acc = sum partial[0..n) (first) or *acc += that sum, in a fixed order.
cudaError_t launch_accumulate(const double* partial, int n, double* acc, int first, cudaStream_t s);
// CheckState of a solve set on the device (stream-ordered, so several solves
// may be queued back to back): zero counters, the stopping parameters, r0sq.
cudaError_t launch_state_init(CheckState* st, double tol, int max_iter, double diverge, double r0sq, cudaStream_t s);
// out = rows [row0, row0 + rows) of c[1 - st->result_cur] (the C-points of a
// finished graph solve), converted from float-float pairs when df is set.
cudaError_t launch_result_rows(const CheckState* st, const double* c0, const double* c1, double* out, int nx,
                               long long row0, long long rows, int df, cudaStream_t s);
int march_max_cluster();
void set_tile(int r);   // register tile of the stencil kernels: 8, 4 or 0
// Form of the fused float-float FCF: 1 register-resident (default, upwind
// stencils), 0 slab in shared memory, 2 and 3 runs of intervals per CTA.
void set_stream_fused(int mode);
int get_tile();

}  // namespace mg
