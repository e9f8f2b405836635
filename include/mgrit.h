/*
 * mgrit.h -- C ABI of the GB300 MGRIT/Parareal library for periodic linear
 * advection with least-squares optimised coarse-grid operators.
 *
 * Method: De Sterck, Falgout, Friedhoff, Krzysik, MacLachlan, "Optimizing
 * multigrid reduction-in-time (MGRIT) and Parareal coarse-grid operators for
 * linear advection", Numer. Linear Algebra Appl. (2021).
 *
 *   PDE        u_t + alpha u_x = 0 on periodic [-1, 1)            (Eq. 1)
 *   space      nx points x_i = -1 + i dx, dx = 2/nx; U_p upwind    (Section 2.1)
 *   time       nt steps of ERKp or SDIRKp, u^{n+1} = Phi u^n      (Eq. 3, App. A)
 *   CFL        c = alpha dt / dx                                  (Eq. 3')
 *   solver     FCF-relaxation, C-point residual, injection, coarse
 *              system e_j = Psi e_{j-1} + r_j                      (Section 2.2, Eq. 5)
 *   Psi        sparse circulant fitted by weighted least squares   (Eq. 6, Section 4)
 *
 * Conventions for every entry point
 *   - Plain C types only.  Arrays are row-major doubles with x contiguous:
 *     time level n of a solution occupies [n*nx, (n+1)*nx).
 *   - Pointers marked "host or device" may point to either; the library
 *     detects which with cudaPointerGetAttributes and copies accordingly.
 *   - Caller buffers stay owned by the caller and are only read/written for
 *     the duration of the call.  Library objects (handles, servers) are owned
 *     by the library and released with the matching destroy call.
 *   - No entry point aborts or throws.  Each returns an mgrit_status; on an
 *     error, mgrit_last_error() returns a message for the calling thread.
 *   - Every call that touches the GPU runs on the CUDA stream given at
 *     creation (NULL = the legacy default stream) and returns after that
 *     stream has finished the call's work, except mgrit_solve_async and
 *     mgrit_fcf_residual_static, which only enqueue it.
 */
#ifndef MGRIT_GB300_H
#define MGRIT_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MGRIT_ABI_VERSION 6
#define MGRIT_MAX_LEVELS 8
#define MGRIT_MAX_HISTORY 128
#define MGRIT_MAX_TAPS 256

typedef enum mgrit_status {
  MGRIT_OK = 0,
  MGRIT_PENDING = 1,              /* mgrit_poll: request not finished yet          */
  MGRIT_ERR_INVALID = -1,         /* bad argument or unsupported combination       */
  MGRIT_ERR_UNSTABLE = -2,        /* ERK CFL number above the limit (Table 1)      */
  MGRIT_ERR_PSI_ILLCOND = -3,     /* fit rejected: |Im psi| > 1e-8 (Section 4.1)   */
  MGRIT_ERR_NOT_CONVERGED = -4,   /* max_iter reached above tol                    */
  MGRIT_ERR_DIVERGED = -5,        /* residual not finite or grew by > 1e6 (flags)  */
  MGRIT_ERR_OVER_BUDGET = -6,     /* server: request larger than the HBM budget    */
  MGRIT_ERR_OOM = -7,             /* device allocation failed                      */
  MGRIT_ERR_TIMEOUT = -8,         /* a bounded device wait ran out                 */
  MGRIT_ERR_CUDA = -9,            /* CUDA runtime error                            */
  MGRIT_ERR_UNSUPPORTED = -10,    /* valid request the library does not implement  */
  MGRIT_ERR_UNKNOWN_TICKET = -11  /* mgrit_poll: ticket never issued or released   */
} mgrit_status;

enum { MGRIT_ERK = 0, MGRIT_SDIRK = 1 };

/* Spatial boundary conditions.
 *  PERIODIC  Eq. 1 on the periodic interval (every operator a circulant).
 *  INFLOW    Section 4.5: inflow at x = -1 with zero inflow data (the
 *            homogeneous problem), no condition at the outflow x = 1; the
 *            unknowns are x_i = -1 + (i+1) dx, i = 0..nx-1 (the outflow point
 *            included).  Every Runge-Kutta stage sees zero ghost values left
 *            of the domain and, right of it, the values of the degree-q
 *            polynomial (q = upwind_order) through the last q+1 unknowns.
 *            Psi is the periodic problem's fit truncated at both ends
 *            (Toeplitz).  ERK only; not with MGRIT_PSI_IDEAL; the two ends'
 *            closures must stay apart: nx >= 2 s q + q + 2 for s stages
 *            (MGRIT_ERR_UNSUPPORTED otherwise).  Iteration counts: Table 5. */
enum { MGRIT_BC_PERIODIC = 0, MGRIT_BC_INFLOW = 1 };

/* Arithmetic of the relaxation (Section 2.2 reading, see the library notes):
 *  FP64   every step in FP64.
 *  MIXED  the C-point update and its residual rho_j = Phi^m c_{j-1} - c_j in
 *         FP64; the second F-relaxation, which only acts on the correction
 *         rho, in FP32.  Below level 1 the V-cycle relaxes the error
 *         equation in FP32 on levels 2..L-1; the coarsest-level solve (the
 *         sequential march) and the convergence test stay FP64.
 *  MIXED_DF  as MIXED, with the FP64 pass of an ERK fine level evaluated in
 *         float-float (pairs of FP32, about 44 significant bits) on the FP32
 *         pipes; SDIRK fine levels keep their FP64 pass. */
enum { MGRIT_PREC_FP64 = 0, MGRIT_PREC_MIXED = 1, MGRIT_PREC_MIXED_DF = 2 };

/* Coarse-operator sparsity rule (Sections 4.2-4.4, 4.6). */
enum {
  MGRIT_PSI_AUTO = 0,       /* ERK: widest-mass contiguous window grown until the
                               fit is acceptable and Eq. 4's bound <= psi_rho;
                               SDIRK: threshold with the paper's eta_tol(p, m)  */
  MGRIT_PSI_HALFWIDTH = 1,  /* 2h+1 offsets centred on argmax |phi~^m_i|      */
  MGRIT_PSI_THRESHOLD = 2,  /* |phi~^m_i| >= psi_eta * max |phi~^m|            */
  MGRIT_PSI_USER = 3,       /* caller supplies offsets and coefficients        */
  MGRIT_PSI_IDEAL = 4,      /* Psi = Phi^m exactly (ERK, two levels)           */
  MGRIT_PSI_REDISC = 5      /* Psi = the fine scheme rediscretised with time
                               step m dt (Section 2.3, Table 2): SDIRK, two
                               levels; an implicit coarse step, no stencil  */
};

enum { MGRIT_OUT_FINAL = 0, MGRIT_OUT_CPOINTS = 1, MGRIT_OUT_FULL = 2 };

/* Initial space-time iterate at t > 0 (Section 2.2; u^0 is always the initial
 * condition):
 *  ZERO    every point 0 (the relative tolerance then refers to ||Phi u^0||).
 *  RANDOM  every point, C and F, drawn uniform on [0, 1) as the paper's tests
 *          do: point i of time level n takes the first two 32-bit words of
 *          Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) with counter
 *          (i, n, 0, 0) and key (seed mod 2^32, seed / 2^32), joined as
 *          ((w0 >> 5) 2^26 + (w1 >> 6)) 2^-53.  The relative tolerance
 *          refers to the full space-time residual of this iterate, F-points
 *          included, computed on the device. */
enum { MGRIT_INIT_ZERO = 0, MGRIT_INIT_RANDOM = 1 };

/* Cycle below level 1 (Section 4.4, Section 5): V-cycle, or F-cycle (the
 * coarse error equation of each level is solved by an F-cycle from zero
 * followed by a V-cycle from its result; one exact solve on the level above
 * the coarsest). */
enum { MGRIT_CYCLE_V = 0, MGRIT_CYCLE_F = 1 };

/* Relaxation on level 1 (Section 2.2): FCF (the paper's choice) or F only
 * (with two levels: Parareal).  Coarse levels always use FCF. */
enum { MGRIT_RELAX_FCF = 0, MGRIT_RELAX_F = 1 };

/* MGRIT_FLAG_TIME_KERNELS: bracket every kernel launch of a solve with CUDA
 * events on the handle's stream and report per-kind device time in
 * mgrit_result.kernel_ms (adds two event records per launch). */
/* MGRIT_FLAG_NO_AUTOTUNE: skip the setup-time timing of the level-1 FCF
 * launch shapes and use the built-in defaults. */
/* MGRIT_FLAG_HOST_LOOP: drive the cycles from the host (one read-back per
 * cycle) instead of the default single CUDA-graph launch per solve, whose
 * WHILE/IF conditional nodes are set by an on-device stopping test.
 * MGRIT_FLAG_TIME_KERNELS implies the host loop. */
/* MGRIT_FLAG_NO_DIVERGENCE_STOP: stop as diverged only on a non-finite
 * residual, not when it grows above 1e6 x the initial one (the paper's
 * divergent configurations, Table 2, converge by finite termination after
 * large transient growth). */
enum { MGRIT_FLAG_TIME_KERNELS = 1, MGRIT_FLAG_NO_AUTOTUNE = 2, MGRIT_FLAG_HOST_LOOP = 4,
       MGRIT_FLAG_NO_DIVERGENCE_STOP = 8 };

/* Kernel kinds reported in mgrit_result.kernel_ms / kernel_count. */
enum {
  MGRIT_K_FCF = 0,         /* level-1 FCF-relaxation + fused residual            */
  MGRIT_K_FCF_COARSE = 1,  /* FCF-relaxation on levels 2..L-1                    */
  MGRIT_K_MARCH = 2,       /* sequential coarsest-level march (cluster)          */
  MGRIT_K_CORRECT = 3,     /* coarse-level correction + F-relaxation             */
  MGRIT_K_NORM = 4,        /* residual norm reduction                            */
  MGRIT_K_ADD = 5,         /* level-1 correction c += e                          */
  MGRIT_K_PROPAGATE = 6,   /* initial residual / propagate                       */
  MGRIT_K_OTHER = 7,
  MGRIT_K_KINDS = 8
};

typedef struct mgrit_problem {
  int32_t nx;            /* spatial points, >= 8                                   */
  int32_t nt;            /* time steps; divisible by m^(levels-1)                  */
  int32_t family;        /* MGRIT_ERK or MGRIT_SDIRK                               */
  int32_t rk_order;      /* ERK 1..5, SDIRK 1..4 (Appendix A)                      */
  int32_t upwind_order;  /* U1..U5 (Section 2.1)                                   */
  int32_t boundary;      /* MGRIT_BC_* (0 = periodic)                              */
  double cfl;            /* c = alpha dt / dx (> 0)                                */
  /* Eq. 1's wave speed and domain.  The discrete operators depend on c only
   * (dt L = c times the U_p stencil), so these fix the physical spacings
   * dx = (xmax - xmin) / nx and dt = c dx / alpha that mgrit_result reports.
   * alpha > 0 (a wave moving right, the upwind direction of U_p); 0 selects
   * 1.  xmin < xmax; xmin = xmax = 0 selects [-1, 1]. */
  double alpha;
  double xmin, xmax;
} mgrit_problem;

typedef struct mgrit_opts {
  int32_t m;             /* coarsening factor >= 2                                 */
  int32_t levels;        /* 2 = two-level (Parareal-like), up to MGRIT_MAX_LEVELS  */
  int32_t max_iter;      /* cap on coarse corrections                              */
  int32_t precision;     /* MGRIT_PREC_*                                           */
  int32_t psi_rule;      /* MGRIT_PSI_*                                            */
  int32_t psi_halfwidth; /* for MGRIT_PSI_HALFWIDTH                                */
  int32_t output;        /* MGRIT_OUT_*                                            */
  int32_t min_coarse;    /* smallest admissible number of coarsest-level steps     */
  int32_t flags;         /* MGRIT_FLAG_* bits                                      */
  int32_t cycle;         /* MGRIT_CYCLE_*                                          */
  int32_t relax;         /* MGRIT_RELAX_*                                          */
  int32_t init_guess;    /* MGRIT_INIT_* (mgrit_solve and mgrit_solve_async)       */
  double tol;            /* stop when ||r|| <= tol ||r^(0)|| (Section 2.2)         */
  double psi_eta;        /* threshold eta_tol; <= 0 = paper's table (Section 4.6)  */
  double psi_rho;        /* bound target of MGRIT_PSI_AUTO (default 0.15)          */
  uint64_t seed;         /* key of the MGRIT_INIT_RANDOM draws                     */
  /* MGRIT_PSI_USER: coarse level l = 2..levels has psi_user_nnz[l-2] taps; the
   * offsets (diagonal index i: (Psi v)_r = sum_i psi_i v_{r+i}) and
   * coefficients of all levels are concatenated in level order. */
  const int32_t* psi_user_nnz;
  const int32_t* psi_user_offsets;
  const double* psi_user_coeffs;
} mgrit_opts;

typedef struct mgrit_result {
  int32_t iterations;    /* coarse-grid corrections applied before the test passed */
  int32_t n_levels;
  int32_t converged;     /* 1 if rel_residual <= tol                               */
  int32_t n_history;     /* entries of history[] used                              */
  double rel_residual;   /* ||r|| / ||r^(0)|| after the final FCF-relaxation       */
  double r0_norm;        /* ||r^(0)||, zero initial iterate: ||Phi u0||            */
  double setup_s;        /* host setup of this handle (Psi fit, allocation)         */
  double solve_s;        /* wall time of the solve call                             */
  double dof_per_s;      /* nx * nt / solve_s                                       */
  double op_complexity;  /* Eq. 5 (ERK; 0 for SDIRK, whose Phi is dense)            */
  double history[MGRIT_MAX_HISTORY]; /* relative residual after each FCF            */
  int32_t launches;      /* kernels this call launched                              */
  int32_t fine_tile;     /* level-1 FCF launch shape picked by the autotuner:       */
  int32_t fine_threads;  /*   register tile (99 = fixed-span path) and CTA size     */
  int32_t graph;         /* 1 if the solve ran as one CUDA-graph launch             */
  int32_t fine_collapsed; /* 1 if each FCF pass applies Phi^m as one stencil        */
  int32_t fine_fourier;  /* 1 if the FP64 pass ran in Fourier space (MIXED)         */
  int32_t kernel_count[MGRIT_K_KINDS];  /* launches per kind                         */
  double kernel_ms[MGRIT_K_KINDS];      /* device time per kind (FLAG_TIME_KERNELS)  */
  double dx, dt;         /* physical spacings of the problem (alpha, xmin, xmax)    */
} mgrit_result;

typedef struct mgrit_handle mgrit_handle;
typedef struct mgrit_server mgrit_server;

/* Fill *o with the defaults: m 8, levels 2, max_iter 100, FP64, PSI_AUTO,
 * halfwidth 3, OUT_CPOINTS, min_coarse 2, flags 0, V-cycle, FCF-relaxation,
 * INIT_ZERO, seed 0, tol 1e-10, eta <= 0, rho 0.15. */
void mgrit_opts_default(mgrit_opts* o);

/* Optional device allocator used for all later allocations (NULL, NULL
 * restores cudaMallocAsync/cudaFreeAsync on the handle's stream).  The
 * callbacks receive the byte count / pointer, the CUDA stream and ctx. */
typedef void* (*mgrit_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*mgrit_free_fn)(void* ptr, void* stream, void* ctx);
void mgrit_set_allocator(mgrit_alloc_fn alloc, mgrit_free_fn release, void* ctx);

/* Environment variables read at mgrit_setup, or where the launches are issued
 * (when a solve's graph is built, or per launch on the host-driven path);
 * diagnostics and profiling, the defaults are the tuned behaviour:
 *   MGRIT_FCF_SHAPE=tile,threads[,collapse[,fourier]]  pin the level-1 FCF
 *                     launch shape instead of timing the candidates (tile 99
 *                     fixed span, 98 chunked, 8/4 sliding window, 0 one tap
 *                     at a time; fourier 128 or 256: the Fourier-space form
 *                     below with that CTA size, 0: not).
 *   MGRIT_FCF_FOURIER=0|1  the MIXED level-1 FCF of a periodic problem with
 *                     nx = 2^p (256..8192) takes its FP64 pass, Phi^m applied
 *                     to each old C-point, in Fourier space: a real FFT of the
 *                     slab, the product with Phi^m's symbol (Lemma 1), the
 *                     inverse FFT.  0 never, 1 always (256 threads); by
 *                     default it is one of the autotuner's candidates.
 *   MGRIT_COARSE=march|fft  solve the coarsest level by the cluster march, or
 *                     in Fourier space (periodic, nx = 2^p, 64..8192) even when
 *                     it has fewer than 16 steps.  By default a periodic
 *                     coarsest level with nx = 2^p and at least 16 steps is
 *                     solved in Fourier space (per-mode recurrences with Psi's
 *                     symbol between FFTs).  A server marches its two-level
 *                     solves in one batched launch, and switches a solve to the
 *                     Fourier-space solve in cycles where few need a coarse
 *                     solve (MGRIT_COARSE=march: never).
 *   MGRIT_FFT_SPLIT=0|1  the Fourier-space solve's transforms with each slab
 *                     split over a cluster of four CTAs; by default where the
 *                     level has fewer slabs than SMs and nx >= 2048.
 *   MGRIT_SDIRK_SPLIT=0|1  the SDIRK level-1 FCF with each interval split over
 *                     a cluster of two CTAs; by default where one CTA per
 *                     interval would have 512 threads (nx = 8192).
 *   MGRIT_FCF_STREAM=0..4  form of the level-1 FCF on upwind collapsed stencils
 *                     of at most 5 taps (MIXED and MIXED_DF): 1 (default)
 *                     register-resident runs of intervals, 0 one interval per
 *                     CTA; 2..4 MIXED_DF test forms.  All give the same C-points.
 *   MGRIT_TILE=8|4|0  register tile of the stencil kernels whose shape the
 *                     autotuner does not pick (coarse levels, correction,
 *                     propagation, sequential stepping). */

/* ---------------------------------------------------------------- host only */

/* Taps of the fine propagator Phi as one circulant stencil (Corollary 1):
 * (Phi v)_r = sum_k coeffs[k] v_{r + offsets[k]}.  ERK only (SDIRK's Phi is
 * dense).  cap = capacity of the arrays.  No GPU is touched.  For
 * MGRIT_BC_INFLOW these are Phi's interior rows. */
mgrit_status mgrit_phi_taps(const mgrit_problem* prob, int32_t cap, int32_t* ntaps,
                            int32_t* offsets, double* coeffs);

/* Rows of Phi^m (m >= 1 fine steps) of an MGRIT_BC_INFLOW problem that
 * differ from its interior stencil (Section 4.5), as the library builds them:
 * dims receives {nl, cl, nr, cr}: rows 0..nl-1 over columns 0..cl-1 and rows
 * nx-nr..nx-1 over columns nx-cr..nx-1; w (capacity cap doubles) receives the
 * coefficients row-major, the left block first (nl*cl + nr*cr values).  Every
 * other row is the circulant one (for m = 1, sum_k coeffs[k] v_{r+offsets[k]}
 * of mgrit_phi_taps).  ERK only.  No GPU is touched. */
mgrit_status mgrit_phi_boundary(const mgrit_problem* prob, int32_t m, int32_t cap, int32_t* dims, double* w);

/* Coarse operators Psi_2..Psi_L that mgrit_setup would build (Eq. 6 on the
 * rule's pattern, recursively per level, Section 4.4).  nnz[levels-1];
 * offsets/coeffs concatenated (capacity cap); diag[3*(levels-1)] receives per
 * level {max |Im psi| of the complex fit, max_k Eq. 4 bound, max_k |mu_k|}.
 * No GPU is touched. */
mgrit_status mgrit_psi_plan(const mgrit_problem* prob, const mgrit_opts* opts, int32_t cap,
                            int32_t* nnz, int32_t* offsets, double* coeffs, double* diag);

/* ------------------------------------------------------------ single solves */

/* Validate, fit Psi on the host (FP64), allocate device state, and upload the
 * stencils.  stream: a cudaStream_t (NULL = default stream). */
mgrit_status mgrit_setup(const mgrit_problem* prob, const mgrit_opts* opts, void* stream,
                         mgrit_handle** out);

/* MGRIT for the block lower-bidiagonal system of Eq. 3 (Section 2.2:
 * FCF-relaxation, C-point residual, injection, the coarse system of Eq. 5
 * solved sequentially or by recursion, ideal interpolation; stopping when the
 * space-time residual falls below tol times the initial one).
 * Solve from u0 (nx values, host or device) with the initial iterate at
 * t > 0 that opts.init_guess names (Section 2.2).  out (host or device)
 * receives, per opts.output: FINAL the nx values at t = T; CPOINTS
 * (nt/m + 1) * nx C-point values; FULL (nt + 1) * nx values (F-points
 * recomputed by a final F-relaxation, ideal interpolation).  out may be
 * NULL.  res may be NULL. */
mgrit_status mgrit_solve(mgrit_handle* h, const double* u0, double* out, mgrit_result* res);

/* The same solve, only enqueued on the handle's stream (Section 2.2's
 * iteration as one CUDA-graph launch with the stopping test on the device):
 * the call returns without waiting, so a caller can queue several solves
 * back to back and the GPU runs them without host round trips in between.
 * out: device memory or NULL (FINAL or CPOINTS output; FULL is
 * MGRIT_ERR_UNSUPPORTED, as are MGRIT_FLAG_HOST_LOOP and
 * MGRIT_FLAG_TIME_KERNELS).  u0 (host or device) and out must stay valid,
 * and u0 unchanged, until mgrit_solve_wait has returned for this solve.  At
 * most MGRIT_MAX_INFLIGHT solves may be outstanding on one handle
 * (MGRIT_ERR_INVALID beyond).  They run in call order on the stream and share
 * the handle's device state, so each one's output is final only when its
 * mgrit_solve_wait returns. */
#define MGRIT_MAX_INFLIGHT 64
mgrit_status mgrit_solve_async(mgrit_handle* h, const double* u0, double* out);

/* Wait for the oldest outstanding mgrit_solve_async of the handle and return
 * its status (MGRIT_OK, MGRIT_ERR_NOT_CONVERGED or MGRIT_ERR_DIVERGED, as
 * mgrit_solve); res (may be NULL) receives its result, with solve_s the time
 * from the enqueue call to the end of the wait.  MGRIT_ERR_INVALID when none
 * is outstanding. */
mgrit_status mgrit_solve_wait(mgrit_handle* h, mgrit_result* res);

/* As mgrit_solve, from a given initial iterate (a warm start, or the
 * paper's random initial iterate of Section 2.2): c_init holds its C-points,
 * (nt/m + 1) * nx values (host or device), row 0 = the initial condition.
 * F-relaxation recomputes the F-points, so only the C-points enter the
 * iteration.  r0_norm > 0 is the norm the relative tolerance refers to (the
 * space-time residual norm of the initial iterate, F-points included, which
 * the caller knows); r0_norm <= 0 uses ||Phi u0||, the zero iterate's. */
mgrit_status mgrit_solve_from(mgrit_handle* h, const double* c_init, double r0_norm, double* out,
                              mgrit_result* res);

/* Level-1 FCF-relaxation sweeps without coarse-grid correction (Section
 * 2.2) on the C-points of the handle's last mgrit_solve / mgrit_solve_from
 * (a relaxation-only smoother).  Each sweep is one launch of the fine FCF
 * kernel (plus the residual kernel in FP64), queued back to back with no
 * host synchronisation between sweeps.  rel_residual (may be NULL) receives
 * the residual after the last sweep relative to that solve's initial
 * residual norm.  The relaxed C-points become the handle's current iterate:
 * a later mgrit_relax continues from them; mgrit_solve starts afresh.
 * MGRIT_ERR_INVALID before the first solve or for sweeps < 0. */
mgrit_status mgrit_relax(mgrit_handle* h, int32_t sweeps, double* rel_residual);

/* Plain sequential time stepping u^{n+1} = Phi u^n on the GPU (FP64), the
 * baseline of Section 5; out as for mgrit_solve.  seconds may be NULL. */
mgrit_status mgrit_sequential(mgrit_handle* h, const double* u0, double* out, double* seconds);

/* Apply Phi_level^k to `count` vectors: in and out are count * nx doubles
 * (device).  level 1 = fine Phi, level l >= 2 = Psi_l.  Used to check single
 * fine steps against the definition. */
mgrit_status mgrit_propagate(mgrit_handle* h, int32_t level, int32_t k, int32_t count,
                             const double* in, double* out);

/* Copy back the coarse operator of level l (2..levels) as built on the
 * handle: nnz, offsets, coeffs (capacity cap). */
mgrit_status mgrit_psi_info(mgrit_handle* h, int32_t level, int32_t cap, int32_t* nnz,
                            int32_t* offsets, double* coeffs);

/* Bytes of device memory this handle holds. */
size_t mgrit_device_bytes(const mgrit_handle* h);

void mgrit_destroy(mgrit_handle* h);

/* --------------------------------------------------------------- serving */

typedef struct mgrit_server_opts {
  double hbm_budget_bytes;   /* admission budget for resident solve state       */
  int32_t max_active;        /* most solves advanced together (0 = 4096)         */
  int32_t reserved;
} mgrit_server_opts;

/* Continuous-batching server.  The paper has no counterpart: this is a
 * serving layer around the solve of Section 2.2, whose per-solve arithmetic
 * is mgrit_solve's (its batched level-1 FCF applies Phi^m as a stencil, as
 * mgrit_solve does with MGRIT_FCF_FOURIER=0).  A host thread admits submitted solves while their state
 * fits in the budget, advances every admitted solve by one MGRIT cycle per
 * batched launch, retires converged solves and frees their slots.  It runs
 * on the device that is current when the server is created. */
mgrit_status mgrit_server_create(const mgrit_server_opts* sopts, void* stream, mgrit_server** out);

/* Queue a solve (u0 host or device, copied before return) of the problem and
 * options as mgrit_setup takes them (Section 2.2's iteration from the zero
 * iterate; MGRIT_INIT_RANDOM and MGRIT_PSI_USER are MGRIT_ERR_UNSUPPORTED
 * here).  *ticket identifies it.  MGRIT_ERR_OVER_BUDGET if it could never fit
 * the budget. */
mgrit_status mgrit_submit(mgrit_server* s, const mgrit_problem* prob, const mgrit_opts* opts,
                          const double* u0, uint64_t* ticket);

/* MGRIT_PENDING until the solve has finished; then copies the output (layout
 * as mgrit_solve, host or device; may be NULL) and the result, releases the
 * request, and returns its final status.  A released ticket gives
 * MGRIT_ERR_UNKNOWN_TICKET. */
mgrit_status mgrit_poll(mgrit_server* s, uint64_t ticket, double* out, mgrit_result* res);

/* Counters of a server since its creation (observability). */
typedef struct mgrit_server_counters {
  uint64_t submitted, completed, failed;  /* requests                          */
  uint64_t cycles;              /* batched MGRIT cycles run                   */
  double admit_s;               /* worker time admitting (set-up, uploads)     */
  double plan_s;                /*   of which fitting coarse operators         */
  double tune_s;                /*   of which timing launch shapes             */
  double cycle_s;               /* worker time in cycles                      */
  double retire_s;              /* worker time retiring (output copies)        */
  double mean_active;           /* average solves per cycle                    */
  double peak_resident_bytes;   /* largest device state held at once           */
  double gpu_fcf_ms;            /* device time of the cycles' FCF launches     */
  double gpu_norm_ms;           /*   residuals and norms                      */
  double gpu_coarse_ms;         /*   coarse solves                             */
  double gpu_gap_ms;            /* server stream idle between consecutive cycles */
  double first_cycle_s;         /* server creation to its first cycle's launch */
  uint64_t fft_coarse_solves;   /* solves switched to the Fourier-space coarse
                                   solve (chosen per cycle when few two-level
                                   solves need a coarse solve; ABI 6) */
} mgrit_server_counters;
mgrit_status mgrit_server_stats(mgrit_server* s, mgrit_server_counters* out);

void mgrit_server_destroy(mgrit_server* s);

/* ------------------------------------------------- no-allocation variant */

/* The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory where they relax (a memory manager owns
 * every device byte, a real-time loop may not stall on an allocation, or a
 * plug-in is handed pre-sized buffers).
 *
 * One FCF-relaxation with the fused C-point residual, as mgrit_solve performs
 * it on the fine level: for j = 1..n_intervals
 *   c_new[j]   = T^m c_old[j-1]                  (F- then C-relaxation)
 *   r[j+1]     = T^m (c_new[j] - c_old[j])       (residual after the second
 *                                                 F-relaxation, j < n_intervals)
 *   *norm2     = sum_j ||r[j+1]||^2
 * with (T v)_i = sum_k coeffs[k] v_{(i + offsets[k]) mod nx} (for example the
 * taps of mgrit_phi_taps).  c_old, c_new, r: (n_intervals + 1) * nx doubles;
 * c_new slab 0 and r slabs 0 and 1 are not written.  norm2: one double.  All
 * four are device pointers; offsets/coeffs are host arrays of ntaps entries.
 * precision: MGRIT_PREC_FP64 or MGRIT_PREC_MIXED (second pass in FP32).
 *
 * Allocates nothing: the per-interval partial norms live in a static device
 * array of MGRIT_STATIC_MAX_INTERVALS doubles (512 KiB) that every GPU which
 * loads the library keeps until exit; n_intervals above that is rejected with
 * MGRIT_ERR_INVALID.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture.  Every call shares the one array, so calls
 * whose work overlaps on the GPU (other streams, other threads) race.  The
 * call only enqueues work on `stream` and returns; synchronise the stream
 * before reading the outputs. */
#define MGRIT_STATIC_MAX_INTERVALS 65536
mgrit_status mgrit_fcf_residual_static(const double* c_old, double* c_new, double* r, double* norm2,
                                       int32_t nx, int32_t m, int32_t n_intervals, int32_t ntaps,
                                       const int32_t* offsets, const double* coeffs, int32_t precision,
                                       void* stream);

/* Self-check of the format conversion the kernels do with integer
 * instructions (binary32 -> binary64, exact, from the IEEE 754 bit fields)
 * against the GPU's conversion instruction, over 2n hashed binary32 bit
 * patterns (seeded; zeros, subnormals, normals, infinities and NaNs among
 * them).  *mismatches = patterns whose results differ bitwise: 0 expected.
 * Runs on the current device and waits for the result. */
mgrit_status mgrit_check_conversions(uint64_t n, uint64_t seed, uint64_t* mismatches);

/* Message of the last failing call on this thread ("" if none). */
const char* mgrit_last_error(void);

int32_t mgrit_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MGRIT_GB300_H */
