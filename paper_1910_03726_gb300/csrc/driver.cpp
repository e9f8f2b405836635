// C ABI of the GB300 MGRIT library: validation, device state, the cycle
// loop (FCF-relaxation, residual test, coarse solve or V-cycle, correction),
// sequential stepping, and the host-only planning entry points.
// Section 2.2 defines the cycle; Eq. 5 the coarse system; Section 4 the Psi fit.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <map>
#include <mutex>
#include <tuple>
#include <complex>
#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mgrit.h"
#include "device.h"
#include "handle.h"
#include "setup.h"

using namespace mg;

// --------------------------------------------------------------- error text

static thread_local std::string g_err;

mgrit_status fail(mgrit_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

namespace mg {
void set_error(const std::string& msg) { g_err = msg; }
}  // namespace mg

#define CUDA_TRY(expr)                                                              \
  do {                                                                              \
    cudaError_t e_ = (expr);                                                        \
    if (e_ != cudaSuccess)                                                          \
      return fail(e_ == cudaErrorMemoryAllocation ? MGRIT_ERR_OOM : MGRIT_ERR_CUDA, \
                  std::string(#expr) + ": " + cudaGetErrorString(e_));              \
  } while (0)

// ---------------------------------------------------------------- allocator

static mgrit_alloc_fn g_alloc = nullptr;
static mgrit_free_fn g_free = nullptr;
static void* g_alloc_ctx = nullptr;

extern "C" void mgrit_set_allocator(mgrit_alloc_fn a, mgrit_free_fn f, void* ctx) {
  g_alloc = a;
  g_free = f;
  g_alloc_ctx = ctx;
}

// Pinned host slots of 8 doubles (a handle's norm read-back), carved from
// chunks of 4096 so that admitting thousands of server solves costs no
// pinned allocation (and no release) per solve.
static std::mutex g_pin_mu;
static std::vector<double*> g_pin_free;

double* pinned_slot() {
  std::lock_guard<std::mutex> lk(g_pin_mu);
  if (g_pin_free.empty()) {
    constexpr int kChunk = 4096;
    double* p = nullptr;
    if (cudaMallocHost(&p, kChunk * 8 * sizeof(double)) != cudaSuccess) {  // kept until exit
      cudaGetLastError();
      return nullptr;
    }
    for (int k = kChunk - 1; k >= 0; --k) g_pin_free.push_back(p + 8 * k);
  }
  double* s = g_pin_free.back();
  g_pin_free.pop_back();
  return s;
}

void pinned_slot_release(double* p) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(g_pin_mu);
  g_pin_free.push_back(p);
}

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// ------------------------------------------------------------------- handle

mgrit_status dalloc(mgrit_handle* h, size_t count, double** out) {
  const size_t bytes = std::max<size_t>(count, 1) * sizeof(double);
  void* p = nullptr;
  DevBuf b;
  if (g_alloc && !h->pool_alloc) {
    p = g_alloc(bytes, (void*)h->stream, g_alloc_ctx);
    if (!p) return fail(MGRIT_ERR_OOM, "allocator callback returned NULL");
    b.freefn = g_free;
    b.ctx = g_alloc_ctx;
  } else {
    cudaError_t e = cudaMallocAsync(&p, bytes, h->stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(e == cudaErrorMemoryAllocation ? MGRIT_ERR_OOM : MGRIT_ERR_CUDA,
                  std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
    }
  }
  b.p = (double*)p;
  b.n = count;
  h->bufs.push_back(b);
  h->bytes += bytes;
  *out = (double*)p;
  return MGRIT_OK;
}

void release(mgrit_handle* h) {
  for (auto& b : h->bufs) {
    if (!b.p) continue;
    if (b.freefn) b.freefn(b.p, (void*)h->stream, b.ctx);
    else cudaFreeAsync(b.p, h->stream);
  }
  h->bufs.clear();
  pinned_slot_release(h->norm_host);
  h->norm_host = nullptr;
  for (auto ev : h->evpool) cudaEventDestroy(ev);
  h->evpool.clear();
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->graph) cudaGraphDestroy(h->graph);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->hstate) cudaFreeHost(h->hstate);
  if (h->ring) cudaFreeHost(h->ring);
  for (auto& ev : h->ring_ev)
    if (ev) cudaEventDestroy(ev);
  h->ring = nullptr;
  h->gexec = nullptr;
  h->graph = nullptr;
  h->cap_stream = nullptr;
  h->hstate = nullptr;
  // a server's handle: its frees are stream-ordered behind the cycles still
  // running, and its worker does not wait for them
  if (!h->pool_alloc) cudaStreamSynchronize(h->stream);
}

DevTaps to_dev(const Taps& t) {
  DevTaps d;
  make_dev_taps(t.off.data(), t.coef.data(), t.size(), &d);
  return d;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

cudaMemcpyKind kind_to_dev(const void* src) {
  return is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
}
cudaMemcpyKind kind_from_dev(const void* dst) {
  return is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
}

// ------------------------------------------------------------- validation

extern "C" void mgrit_opts_default(mgrit_opts* o) {
  std::memset(o, 0, sizeof(*o));
  o->m = 8;
  o->levels = 2;
  o->max_iter = 100;
  o->precision = MGRIT_PREC_FP64;
  o->psi_rule = MGRIT_PSI_AUTO;
  o->psi_halfwidth = 3;
  o->output = MGRIT_OUT_CPOINTS;
  o->min_coarse = 2;
  o->flags = 0;
  o->cycle = MGRIT_CYCLE_V;
  o->relax = MGRIT_RELAX_FCF;
  o->tol = 1e-10;
  o->psi_eta = 0.0;
  o->psi_rho = 0.15;
}

extern "C" int32_t mgrit_abi_version(void) { return MGRIT_ABI_VERSION; }

extern "C" mgrit_status mgrit_check_conversions(uint64_t n, uint64_t seed, uint64_t* mismatches) {
  if (!mismatches) return fail(MGRIT_ERR_INVALID, "mismatches is NULL");
  unsigned long long* d = nullptr;
  cudaError_t e = cudaMalloc(&d, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(d, 0, sizeof(unsigned long long));
  if (e == cudaSuccess) e = launch_conversion_check(n, seed, d, nullptr);
  unsigned long long h = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(h), cudaMemcpyDeviceToHost);
  if (d) cudaFree(d);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(MGRIT_ERR_CUDA, std::string("conversion check: ") + cudaGetErrorString(e));
  }
  *mismatches = h;
  return MGRIT_OK;
}

extern "C" const char* mgrit_last_error(void) { return g_err.c_str(); }

mgrit_status validate_problem(const mgrit_problem* p) {
  if (!p) return fail(MGRIT_ERR_INVALID, "problem is NULL");
  if (p->nx < 8) return fail(MGRIT_ERR_INVALID, "nx must be >= 8");
  if (p->nt < 1) return fail(MGRIT_ERR_INVALID, "nt must be >= 1");
  if (p->family != MGRIT_ERK && p->family != MGRIT_SDIRK) return fail(MGRIT_ERR_INVALID, "family must be ERK or SDIRK");
  if (p->family == MGRIT_ERK && (p->rk_order < 1 || p->rk_order > 5))
    return fail(MGRIT_ERR_INVALID, "ERK order must be 1..5");
  if (p->family == MGRIT_SDIRK && (p->rk_order < 1 || p->rk_order > 4))
    return fail(MGRIT_ERR_INVALID, "SDIRK order must be 1..4");
  if (p->upwind_order < 1 || p->upwind_order > 5) return fail(MGRIT_ERR_INVALID, "upwind order must be 1..5");
  if (!(p->cfl > 0.0) || !std::isfinite(p->cfl)) return fail(MGRIT_ERR_INVALID, "cfl must be > 0");
  if (p->boundary != MGRIT_BC_PERIODIC && p->boundary != MGRIT_BC_INFLOW)
    return fail(MGRIT_ERR_INVALID, "unknown boundary");
  if (p->boundary == MGRIT_BC_INFLOW && p->family != MGRIT_ERK)
    return fail(MGRIT_ERR_UNSUPPORTED, "inflow/outflow boundaries are implemented for ERK only");
  if (!std::isfinite(p->alpha) || !std::isfinite(p->xmin) || !std::isfinite(p->xmax))
    return fail(MGRIT_ERR_INVALID, "alpha, xmin and xmax must be finite");
  if (p->alpha < 0.0)
    return fail(MGRIT_ERR_UNSUPPORTED, "alpha must be > 0: U_p is upwind for a wave moving to the right");
  if (!(p->xmin == 0.0 && p->xmax == 0.0) && !(p->xmin < p->xmax))
    return fail(MGRIT_ERR_INVALID, "xmin must be < xmax (both 0 select [-1, 1])");
  if (p->family == MGRIT_ERK && p->rk_order == p->upwind_order) {
    // Table 1 limits as printed (last digit rounded up)
    static const double cmax[6] = {0, 1.0, 0.5, 1.62590, 1.04450, 1.96584};
    if (p->cfl > cmax[p->rk_order])
      return fail(MGRIT_ERR_UNSTABLE, "ERK CFL number above the stability limit of Table 1");
  } else if (p->family == MGRIT_ERK) {
    if (p->cfl > erk_cfl_limit(p->rk_order, p->upwind_order))
      return fail(MGRIT_ERR_UNSTABLE, "ERK CFL number above the stability limit");
  }
  return MGRIT_OK;
}

mgrit_status validate_opts(const mgrit_problem* p, const mgrit_opts* o) {
  if (!o) return fail(MGRIT_ERR_INVALID, "opts is NULL");
  if (o->m < 2) return fail(MGRIT_ERR_INVALID, "m must be >= 2");
  if (o->levels < 2 || o->levels > MGRIT_MAX_LEVELS) return fail(MGRIT_ERR_INVALID, "levels must be 2..8");
  long long div = 1;
  for (int l = 1; l < o->levels; ++l) {
    div *= o->m;
    if (p->nt % div != 0) return fail(MGRIT_ERR_INVALID, "nt must be divisible by m^(levels-1)");
  }
  if (p->nt / div < std::max(1, o->min_coarse))
    return fail(MGRIT_ERR_INVALID, "coarsest level has fewer than min_coarse steps");
  if (!(o->tol > 0.0)) return fail(MGRIT_ERR_INVALID, "tol must be > 0");
  if (o->max_iter < 0) return fail(MGRIT_ERR_INVALID, "max_iter must be >= 0");
  if (o->precision < 0 || o->precision > 2) return fail(MGRIT_ERR_INVALID, "unknown precision");
  if (o->output < 0 || o->output > 2) return fail(MGRIT_ERR_INVALID, "unknown output");
  if (o->psi_rule == MGRIT_PSI_IDEAL && (p->family != MGRIT_ERK || o->levels != 2))
    return fail(MGRIT_ERR_INVALID, "PSI_IDEAL needs ERK and two levels");
  if (o->psi_rule == MGRIT_PSI_IDEAL && p->boundary == MGRIT_BC_INFLOW)
    return fail(MGRIT_ERR_UNSUPPORTED, "PSI_IDEAL is the periodic Phi^m; not for inflow/outflow boundaries");
  if (o->psi_rule == MGRIT_PSI_REDISC && (p->family != MGRIT_SDIRK || o->levels != 2))
    return fail(MGRIT_ERR_INVALID, "PSI_REDISC needs SDIRK and two levels");
  if (o->psi_rule < MGRIT_PSI_AUTO || o->psi_rule > MGRIT_PSI_REDISC) return fail(MGRIT_ERR_INVALID, "unknown psi_rule");
  if (o->psi_rule == MGRIT_PSI_HALFWIDTH && o->psi_halfwidth < 0)
    return fail(MGRIT_ERR_INVALID, "psi_halfwidth must be >= 0");
  if (o->cycle != MGRIT_CYCLE_V && o->cycle != MGRIT_CYCLE_F) return fail(MGRIT_ERR_INVALID, "unknown cycle");
  if (o->relax != MGRIT_RELAX_FCF && o->relax != MGRIT_RELAX_F) return fail(MGRIT_ERR_INVALID, "unknown relax");
  if (o->init_guess != MGRIT_INIT_ZERO && o->init_guess != MGRIT_INIT_RANDOM)
    return fail(MGRIT_ERR_INVALID, "unknown init_guess");
  return MGRIT_OK;
}

// Physical spacings of Eq. 1's grid: dx = (xmax - xmin)/nx, dt = c dx/alpha.
void grid_spacings(const mgrit_problem* p, double* dx, double* dt) {
  const double a = p->alpha > 0.0 ? p->alpha : 1.0;
  const bool dflt = p->xmin == 0.0 && p->xmax == 0.0;
  *dx = (dflt ? 2.0 : p->xmax - p->xmin) / p->nx;
  *dt = p->cfl * *dx / a;
}

static PlanRequest make_request(const mgrit_problem* p, const mgrit_opts* o) {
  PlanRequest rq;
  rq.nx = p->nx; rq.nt = p->nt; rq.family = p->family; rq.rk_order = p->rk_order;
  rq.upwind_order = p->upwind_order; rq.cfl = p->cfl;
  rq.m = o->m; rq.levels = o->levels; rq.rule = o->psi_rule; rq.halfwidth = o->psi_halfwidth;
  rq.eta = o->psi_eta; rq.rho = o->psi_rho > 0.0 ? o->psi_rho : 0.15;
  rq.user_nnz = o->psi_user_nnz; rq.user_off = o->psi_user_offsets; rq.user_coef = o->psi_user_coeffs;
  return rq;
}

mgrit_status plan(const mgrit_problem* p, const mgrit_opts* o, std::vector<CoarseOp>* ops) {
  std::string err;
  if (o->psi_rule == MGRIT_PSI_REDISC) {  // an SDIRK step, not a stencil: placeholder op
    ops->assign(1, CoarseOp());
    ops->back().taps.off = {0};
    ops->back().taps.coef = {1.0};
    return MGRIT_OK;
  }
  if (!build_hierarchy(make_request(p, o), ops, &err)) return fail(MGRIT_ERR_INVALID, err);
  for (size_t l = 0; l < ops->size(); ++l) {
    if ((*ops)[l].imag > 1e-8)
      return fail(MGRIT_ERR_PSI_ILLCOND, "least-squares Psi has an imaginary part above 1e-8 (level " +
                                             std::to_string(l + 2) + ")");
  }
  return MGRIT_OK;
}

// ----------------------------------------------------------- host-only ABI

extern "C" mgrit_status mgrit_phi_taps(const mgrit_problem* prob, int32_t cap, int32_t* ntaps, int32_t* offsets,
                                       double* coeffs) {
  mgrit_status st = validate_problem(prob);
  if (st != MGRIT_OK) return st;
  if (prob->family != MGRIT_ERK) return fail(MGRIT_ERR_INVALID, "Phi is a single stencil only for ERK");
  Taps t = erk_phi_taps(prob->rk_order, prob->upwind_order, prob->cfl);
  if (ntaps) *ntaps = t.size();
  if (t.size() > cap) return fail(MGRIT_ERR_INVALID, "capacity too small");
  for (int k = 0; k < t.size(); ++k) {
    if (offsets) offsets[k] = t.off[k];
    if (coeffs) coeffs[k] = t.coef[k];
  }
  return MGRIT_OK;
}

extern "C" mgrit_status mgrit_phi_boundary(const mgrit_problem* prob, int32_t m, int32_t cap, int32_t* dims,
                                           double* w) {
  mgrit_status st = validate_problem(prob);
  if (st != MGRIT_OK) return st;
  if (prob->boundary != MGRIT_BC_INFLOW) return fail(MGRIT_ERR_INVALID, "the problem is periodic");
  if (m < 1) return fail(MGRIT_ERR_INVALID, "m must be >= 1");
  const BoundaryRows B = inflow_phi_rows(prob->rk_order, prob->upwind_order, prob->cfl, prob->nx, m);
  if (B.nl + B.nr == 0) return fail(MGRIT_ERR_UNSUPPORTED, "nx too small for the boundary closures");
  if (dims) {
    dims[0] = B.nl; dims[1] = B.cl; dims[2] = B.nr; dims[3] = B.cr;
  }
  if ((int)B.w.size() > cap) return fail(MGRIT_ERR_INVALID, "capacity too small");
  if (w) std::copy(B.w.begin(), B.w.end(), w);
  return MGRIT_OK;
}

extern "C" mgrit_status mgrit_psi_plan(const mgrit_problem* prob, const mgrit_opts* opts, int32_t cap, int32_t* nnz,
                                       int32_t* offsets, double* coeffs, double* diag) {
  if (opts && opts->psi_rule == MGRIT_PSI_REDISC)
    return fail(MGRIT_ERR_UNSUPPORTED, "the rediscretised Psi is an implicit step, not a stencil");
  mgrit_status st = validate_problem(prob);
  if (st == MGRIT_OK) st = validate_opts(prob, opts);
  if (st != MGRIT_OK) return st;
  std::vector<CoarseOp> ops;
  std::string err;
  if (!build_hierarchy(make_request(prob, opts), &ops, &err)) return fail(MGRIT_ERR_INVALID, err);
  int pos = 0;
  for (size_t l = 0; l < ops.size(); ++l) {
    const Taps& t = ops[l].taps;
    if (nnz) nnz[l] = t.size();
    if (diag) {
      diag[3 * l] = ops[l].imag;
      diag[3 * l + 1] = ops[l].bound;
      diag[3 * l + 2] = ops[l].mumax;
    }
    if (pos + t.size() > cap) return fail(MGRIT_ERR_INVALID, "capacity too small");
    for (int k = 0; k < t.size(); ++k) {
      if (offsets) offsets[pos + k] = t.off[k];
      if (coeffs) coeffs[pos + k] = t.coef[k];
    }
    pos += t.size();
  }
  for (size_t l = 0; l < ops.size(); ++l)
    if (ops[l].imag > 1e-8) return fail(MGRIT_ERR_PSI_ILLCOND, "imaginary part above 1e-8");
  return MGRIT_OK;
}

// ------------------------------------------------------------------- setup

// Cluster size of the march: the largest power of two <= 16 with at least 64
// points per CTA and a CTA at least as wide as the stencil (the march runs in
// the stencil's moving frame, so only the width matters).  CTAs own
// ceil(nx / cs) points each and the last one the rest, so cs need not divide
// nx (the march kernel holds at most 16 x 256 points per CTA in registers).
int pick_cluster(int nx, const Taps& t) {
  int lo = t.off.empty() ? 0 : t.off[0], hi = lo;
  for (int o : t.off) {
    lo = std::min(lo, o);
    hi = std::max(hi, o);
  }
  const int width = hi - lo;
  for (int cs = march_max_cluster(); cs > 1; cs >>= 1)
    if (nx / cs >= std::max(64, width) && nx - (cs - 1) * ((nx + cs - 1) / cs) >= 1) return cs;
  return 1;
}

namespace {
using Mat = std::vector<double>;  // K x K row-major

Mat mat_mul(const Mat& A, const Mat& B, int K) {
  Mat C(K * K, 0.0);
  for (int i = 0; i < K; ++i)
    for (int k = 0; k < K; ++k)
      for (int j = 0; j < K; ++j) C[i * K + j] += A[i * K + k] * B[k * K + j];
  return C;
}
Mat mat_eye(int K) {
  Mat I(K * K, 0.0);
  for (int i = 0; i < K; ++i) I[i * K + i] = 1.0;
  return I;
}
Mat mat_pow(Mat A, long long n, int K) {
  Mat R = mat_eye(K);
  while (n > 0) {
    if (n & 1) R = mat_mul(R, A, K);
    A = mat_mul(A, A, K);
    n >>= 1;
  }
  return R;
}
// Inverse by Gauss-Jordan elimination with partial pivoting (K <= 5).
bool mat_inv(Mat A, int K, Mat* out) {
  Mat I = mat_eye(K);
  for (int c = 0; c < K; ++c) {
    int piv = c;
    for (int r = c + 1; r < K; ++r)
      if (std::fabs(A[r * K + c]) > std::fabs(A[piv * K + c])) piv = r;
    if (std::fabs(A[piv * K + c]) < 1e-300) return false;
    for (int j = 0; j < K; ++j) {
      std::swap(A[c * K + j], A[piv * K + j]);
      std::swap(I[c * K + j], I[piv * K + j]);
    }
    const double d = 1.0 / A[c * K + c];
    for (int j = 0; j < K; ++j) {
      A[c * K + j] *= d;
      I[c * K + j] *= d;
    }
    for (int r = 0; r < K; ++r)
      if (r != c) {
        const double f = A[r * K + c];
        for (int j = 0; j < K; ++j) {
          A[r * K + j] -= f * A[c * K + j];
          I[r * K + j] -= f * I[c * K + j];
        }
      }
  }
  *out = I;
  return true;
}
// Companion matrix of x_i = sum_q a_q x_{i-q} + y_i on the state
// (x_i, x_{i-1}, ..., x_{i-K+1}).
Mat companion(const double* a, int K) {
  Mat T(K * K, 0.0);
  for (int q = 0; q < K; ++q) T[q] = a[q];
  for (int q = 1; q < K; ++q) T[q * K + q - 1] = 1.0;
  return T;
}
// Tables of one direction (layout of sdirk_rec_len): a, A^k (k <= 32),
// (A^32)^k (k <= 16), G[c] = row 0 of T^{c+1}, Q = (I - T^nx)^{-1}.
bool rec_tables(const double* a, int K, int C, int nx, std::vector<double>* out) {
  if (K == 0) return true;
  const Mat T = companion(a, K);
  const Mat A = mat_pow(T, C, K);
  const Mat A32 = mat_pow(A, 32, K);
  for (int q = 0; q < K; ++q) out->push_back(a[q]);
  Mat P = mat_eye(K);
  for (int k = 0; k <= 32; ++k) {
    out->insert(out->end(), P.begin(), P.end());
    P = mat_mul(P, A, K);
  }
  P = mat_eye(K);
  for (int k = 0; k <= 16; ++k) {
    out->insert(out->end(), P.begin(), P.end());
    P = mat_mul(P, A32, K);
  }
  P = T;
  for (int c = 0; c < C; ++c) {
    for (int q = 0; q < K; ++q) out->push_back(P[q]);
    P = mat_mul(P, T, K);
  }
  Mat M = mat_pow(T, nx, K), Q;
  for (int i = 0; i < K * K; ++i) M[i] = (i % (K + 1) == 0 ? 1.0 : 0.0) - M[i];
  if (!mat_inv(M, K, &Q)) return false;
  out->insert(out->end(), Q.begin(), Q.end());
  return true;
}
// One periodic recurrence over y (forward, or backward over reversed order),
// sequentially: a zero-state pass, the closure s_{-1} = (I - T^n)^{-1} s_{n-1},
// and the pass from s_{-1}.
void host_rec(const double* a, int K, bool backward, std::vector<double>& y) {
  if (K == 0) return;
  const int n = (int)y.size();
  auto at = [&](int k) -> double& { return y[backward ? n - 1 - k : k]; };
  std::vector<double> w(n);
  std::vector<double> st(K, 0.0);
  for (int k = 0; k < n; ++k) {
    double v = at(k);
    for (int q = 0; q < K; ++q) v += a[q] * st[q];
    for (int q = K - 1; q > 0; --q) st[q] = st[q - 1];
    st[0] = v;
  }
  Mat M = mat_pow(companion(a, K), n, K), Q;
  for (int i = 0; i < K * K; ++i) M[i] = (i % (K + 1) == 0 ? 1.0 : 0.0) - M[i];
  if (!mat_inv(M, K, &Q)) return;
  std::vector<double> s0(K, 0.0);
  for (int r = 0; r < K; ++r)
    for (int q = 0; q < K; ++q) s0[r] += Q[r * K + q] * st[q];
  st = s0;
  for (int k = 0; k < n; ++k) {
    double v = at(k);
    for (int q = 0; q < K; ++q) v += a[q] * st[q];
    for (int q = K - 1; q > 0; --q) st[q] = st[q - 1];
    st[0] = v;
    w[k] = v;
  }
  for (int k = 0; k < n; ++k) at(k) = w[k];
}
}  // namespace

// Host reference of the stage solve M^{-1} y (checks the plan).
static void host_sdirk_solve(const SdirkPlan& P, std::vector<double>& y) {
  const int n = (int)y.size();
  std::vector<double> x(n);
  for (int i = 0; i < n; ++i) x[i] = y[((i + P.ql) % n + n) % n];
  host_rec(P.af, P.kf, false, x);
  host_rec(P.ab, P.kb, true, x);
  for (int i = 0; i < n; ++i) y[i] = x[i] * P.scale;
}

// Expand prod_r (1 - w_r t) = 1 - sum_q a_q t^q; returns a_1..a_K.
static std::vector<double> rec_coeffs(const std::vector<std::complex<double>>& w) {
  std::vector<std::complex<double>> c(1, 1.0);
  for (auto z : w) {
    std::vector<std::complex<double>> n(c.size() + 1, 0.0);
    for (size_t k = 0; k < c.size(); ++k) {
      n[k] += c[k];
      n[k + 1] -= z * c[k];
    }
    c = n;
  }
  std::vector<double> a;
  for (size_t q = 1; q < c.size(); ++q) a.push_back(-c[q].real());
  return a;
}

mgrit_status make_sdirk_plan(const mgrit_problem* prob, SdirkPlan* out, std::vector<double>* tables) {
  SdirkPlan P;
  std::memset(&P, 0, sizeof(P));
  Tableau tb = sdirk_tableau(prob->rk_order);
  Taps L = dtL_taps(prob->upwind_order, prob->cfl);
  if (tb.s < 1 || tb.s > kMaxStages || L.size() > 6) return fail(MGRIT_ERR_INVALID, "unsupported SDIRK scheme");
  for (int j = 0; j < tb.s; ++j)
    if (std::fabs(tb.b[j] - tb.a(tb.s - 1, j)) > 1e-15)
      return fail(MGRIT_ERR_UNSUPPORTED, "SDIRK tableau is not stiffly accurate");
  P.s = tb.s;
  for (int i = 0; i < tb.s; ++i)
    for (int j = 0; j < tb.s; ++j) {
      P.a[i][j] = tb.a(i, j);
      P.a32[i][j] = (float)tb.a(i, j);
    }
  P.gamma = tb.a(0, 0);
  P.inv_gamma = 1.0 / P.gamma;
  P.gamma32 = (float)P.gamma;
  P.inv_gamma32 = (float)P.inv_gamma;
  // M = I - gamma dtL = E^{lo} sum_k m_k E^{k-lo}: polynomial of degree hi-lo
  const int lo = L.lo(), hi = L.hi(), d = hi - lo;
  std::vector<double> poly(d + 1, 0.0);
  for (int k = 0; k < L.size(); ++k) poly[L.off[k] - lo] += -P.gamma * L.coef[k];
  poly[-lo] += 1.0;
  std::vector<std::complex<double>> roots = poly_roots(poly);
  std::vector<std::complex<double>> fwd, bwd;
  std::complex<double> scale = 1.0 / poly[d];
  for (auto z : roots) {
    if (std::fabs(std::abs(z) - 1.0) < 1e-8) return fail(MGRIT_ERR_INVALID, "stage matrix has a root on |z| = 1");
    if (std::abs(z) < 1.0) {
      fwd.push_back(z);
    } else {
      bwd.push_back(1.0 / z);
      scale /= -z;
    }
  }
  P.kf = (int)fwd.size();
  P.kb = (int)bwd.size();
  if (!sdirk_orders_supported(P.kf, P.kb))
    return fail(MGRIT_ERR_UNSUPPORTED, "stage matrix splits into unsupported recurrence orders");
  const std::vector<double> af = rec_coeffs(fwd), ab = rec_coeffs(bwd);
  for (int q = 0; q < P.kf; ++q) P.af[q] = af[q];
  for (int q = 0; q < P.kb; ++q) P.ab[q] = ab[q];
  P.ql = -lo - P.kf;
  P.scale = scale.real();
  P.scale32 = (float)P.scale;
  P.nx = prob->nx;
  P.threads = sdirk_threads(prob->nx);
  if (!P.threads) return fail(MGRIT_ERR_UNSUPPORTED, "SDIRK needs nx = threads * C, threads a multiple of 32 <= 512");
  P.C = prob->nx / P.threads;
  tables->clear();
  if (!rec_tables(P.af, P.kf, P.C, P.nx, tables) || !rec_tables(P.ab, P.kb, P.C, P.nx, tables))
    return fail(MGRIT_ERR_INVALID, "periodic closure of the stage recurrences is singular");
  P.tab_len = (int)tables->size();
  // truncation of the scans: drop terms whose factor A^d lies below FP64
  // rounding (max-row-sum norm < 1e-18)
  for (int dir = 0; dir < 2; ++dir) {
    const int K = dir == 0 ? P.kf : P.kb;
    int steps = 5, trunc = 0;
    if (K > 0) {
      const Mat A = mat_pow(companion(dir == 0 ? P.af : P.ab, K), P.C, K);
      auto norm = [&](const Mat& M) {
        double n = 0.0;
        for (int i = 0; i < K; ++i) {
          double r = 0.0;
          for (int j = 0; j < K; ++j) r += std::fabs(M[i * K + j]);
          n = std::max(n, r);
        }
        return n;
      };
      for (int D = 0; D <= 5; ++D)
        if (norm(mat_pow(A, 1LL << D, K)) < 1e-18) {
          steps = D;
          break;
        }
      trunc = norm(mat_pow(A, 32, K)) < 1e-18 ? 1 : 0;
    }
    (dir == 0 ? P.steps_f : P.steps_b) = steps;
    (dir == 0 ? P.trunc_f : P.trunc_b) = trunc;
  }
  if (P.tab_len != sdirk_rec_len(P.kf, P.C) + sdirk_rec_len(P.kb, P.C))
    return fail(MGRIT_ERR_INVALID, "SDIRK table layout mismatch");
  // check: M (M^{-1} y) = y on a test vector of the solve's size
  const int n = prob->nx;
  std::vector<double> y(n), x(n);
  for (int i = 0; i < n; ++i) y[i] = std::sin(0.37 * i) + 0.25 * std::cos(1.9 * i * i);
  x = y;
  host_sdirk_solve(P, x);
  double err = 0.0, ref = 0.0;
  for (int i = 0; i < n; ++i) {
    double mx = x[i];
    for (int k = 0; k < L.size(); ++k) mx -= P.gamma * L.coef[k] * x[((i + L.off[k]) % n + n) % n];
    err = std::max(err, std::fabs(mx - y[i]));
    ref = std::max(ref, std::fabs(y[i]));
  }
  if (!(err <= 1e-12 * ref)) return fail(MGRIT_ERR_INVALID, "stage-matrix factorisation check failed");
  *out = P;
  return MGRIT_OK;
}

int fine_prec(const mgrit_handle* h) {
  if (h->opts.precision == MGRIT_PREC_FP64) return 0;
  if (h->opts.precision == MGRIT_PREC_MIXED_DF && !h->sdirk) return 3;
  return 1;  // SDIRK keeps its FP64 pass in MIXED_DF
}

namespace {
struct TuneKey {
  int prec, nx, span, ntaps, m, inflow, fourier;  // fourier: the Fourier form was a candidate
  bool operator<(const TuneKey& o) const {
    return std::tie(prec, nx, span, ntaps, m, inflow, fourier) <
           std::tie(o.prec, o.nx, o.span, o.ntaps, o.m, o.inflow, o.fourier);
  }
};
struct TunePick {
  int collapse, tile, threads, fourier;
};
std::map<TuneKey, TunePick> g_tune;
std::mutex g_tune_mu;

bool fixed_span(int span) { return span == 2 || span == 5 || span == 10 || span == 17 || span == 31; }
}  // namespace

// Level-1 FCF launch shape: step by step with Phi (m steps per pass) or one
// application of the collapsed Phi^m per pass; register tile (fixed-span,
// sliding window 8 or 4, one tap at a time) and CTA size.  Timed on the
// handle's own interval count at set-up and cached per problem shape.
// MGRIT_FCF_FOURIER=0 / 1 keeps the Fourier-space FP64 pass off / takes it
// (256 threads) wherever the handle has its tables; unset, it is a candidate.
static int fourier_env() {
  const char* e = std::getenv("MGRIT_FCF_FOURIER");
  if (!e) return -1;
  return std::atoi(e) != 0 ? 1 : 0;
}

void autotune_fine(mgrit_handle* h) {
  const int prec = fine_prec(h);
  h->fine_collapse = 0;
  h->fine_tile = default_tile(h->dphi, h->nx);
  h->fine_threads = default_threads(h->nx, h->fine_tile);
  h->fine_fourier = 0;
  const int fenv = h->ftab ? fourier_env() : 0;
  if (fenv == 1) h->fine_fourier = 256;
  if (h->sdirk || (h->opts.flags & MGRIT_FLAG_NO_AUTOTUNE)) return;
  const int nx = h->nx;
  auto valid = [&](int collapse, int tile) {
    if (collapse && !h->have_phim) return false;
    const DevTaps& t = collapse ? h->dphim : h->dphi;
    const bool dense = t.span > 0 && nx >= 64;
    if (tile == kFixedTile) return dense && fixed_span(t.span);  // Phi, or Phi^m whose span is compiled
    if (tile == kChunkTile) return dense && t.span >= 8;
    if (tile == 8 || tile == 4) return dense;
    return tile == 0;
  };
  // MGRIT_FCF_SHAPE="tile,threads[,collapse[,fourier threads]]" pins the
  // shape (reproducible profiling)
  if (const char* shape = std::getenv("MGRIT_FCF_SHAPE")) {
    int tile = 0, th = 0, col = 0, fo = 0;
    const int n = std::sscanf(shape, "%d,%d,%d,%d", &tile, &th, &col, &fo);
    if (n >= 2 && (th == 128 || th == 256 || th == 512) && (col == 0 || col == 1) && valid(col, tile)) {
      h->fine_collapse = col;
      h->fine_tile = tile;
      h->fine_threads = th;
      if (n >= 4 && h->ftab && fenv != 0) h->fine_fourier = (fo == 128 || fo == 256) ? fo : 0;
      return;
    }
  }
  const TuneKey key{prec, nx, h->dphi.span, h->dphi.n, h->m, h->inflow ? 1 : 0, h->ftab ? 1 : 0};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      h->fine_collapse = it->second.collapse;
      h->fine_tile = it->second.tile;
      h->fine_threads = it->second.threads;
      if (fenv == -1 && h->ftab) h->fine_fourier = it->second.fourier;
      return;
    }
  }
  // time the candidates on an otherwise idle device (other streams' work would
  // distort the comparison).  A server's handle is the exception: it tunes on
  // the server's high-priority set-up stream while a cycle runs, since
  // waiting for the device would hold every admission behind that cycle.
  if (!h->pool_alloc && cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  FcfArgs f = {};
  f.u_old = h->c[0];
  f.cstride = nx;
  f.c_new = h->c[1];
  f.r = h->r[1];
  f.r_f = h->rf[1];
  f.partial = h->partial;
  f.nx = nx;
  f.fx = h->fx_phi;
  f.df_store = h->dfc;
  // a sample of the handle's intervals, large enough (12 per SM) that the last
  // wave's share is small for every CTA size
  f.N = std::min(h->Nl[1], 12 * 152);
  // nonzero trial data (every byte 0x3F: each double is 4.8e-4), so that no
  // interval takes the zero-slab shortcut while it is timed
  cudaMemsetAsync(h->c[0], 0x3F, ((size_t)f.N + 1) * nx * sizeof(double), h->stream);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  // candidates: the shapes that can win (wide collapsed stencils chunked or
  // sliding; step by step fixed-span or chunked; one tap at a time only for
  // stencils without a dense form)
  struct Cand { int collapse, tile, threads; };
  std::vector<Cand> cands;
  for (Cand c : {Cand{1, kChunkTile, 256}, Cand{1, kChunkTile, 512}, Cand{1, 8, 256}, Cand{1, kFixedTile, 256},
                 Cand{1, kFixedTile, 512}, Cand{0, kFixedTile, 256}, Cand{0, kFixedTile, 512}, Cand{0, kChunkTile, 256},
                 Cand{0, 8, 256}, Cand{0, 0, 128}, Cand{0, 0, 256}})
    if (valid(c.collapse, c.tile)) cands.push_back(c);
  bool dense_found = false;
  for (const Cand& c : cands) dense_found |= c.tile != 0;
  float best = 1e30f;
  TunePick pick{0, h->fine_tile, h->fine_threads, 0};
  bool warmed = false;
  for (const Cand& c : cands) {
    if (c.tile == 0 && dense_found) continue;
    const DevTaps& t = c.collapse ? h->dphim : h->dphi;
    f.m = c.collapse ? 1 : h->m;
    f.fx = c.collapse ? h->fx_phim : h->fx_phi;
    const int per = c.tile == kFixedTile ? 4 : (c.tile == kChunkTile ? 8 : (c.tile > 0 ? c.tile : 1));
    if (c.threads > std::max(32, (nx / per + 31) / 32 * 32)) continue;
    if (!warmed) {
      if (launch_fcf(f, t, prec, c.threads, h->stream, c.tile) != cudaSuccess) {
        cudaGetLastError();
        continue;
      }
      warmed = true;
    }
    float tm = 1e30f;
    for (int rep = 0; rep < 2; ++rep) {
      cudaEventRecord(e0, h->stream);
      if (launch_fcf(f, t, prec, c.threads, h->stream, c.tile) != cudaSuccess) {
        cudaGetLastError();
        break;
      }
      cudaEventRecord(e1, h->stream);
      float ms = 0.0f;
      if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess)
        tm = std::min(tm, ms);
      else
        cudaGetLastError();
    }
    if (tm < best) {
      best = tm;
      pick = {c.collapse, c.tile, c.threads, 0};
    }
  }
  // the Fourier-space FP64 pass (collapsed residual pass), where it applies
  if (fenv == -1 && h->ftab) {
    f.m = 1;
    f.fx = h->fx_phim;
    for (int th : {256, 128}) {
      if (!fourier_fcf_args_ok(f)) break;
      float tm = 1e30f;
      for (int rep = 0; rep < 3; ++rep) {  // the first launch sets the shared-memory limit
        cudaEventRecord(e0, h->stream);
        if (launch_fcf_fourier(f, h->dphim, h->ftab, th, h->stream) != cudaSuccess) {
          cudaGetLastError();
          break;
        }
        cudaEventRecord(e1, h->stream);
        float ms = 0.0f;
        if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) {
          if (rep > 0) tm = std::min(tm, ms);
        } else {
          cudaGetLastError();
        }
      }
      if (tm < best) {
        best = tm;
        pick.fourier = th;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->fine_collapse = pick.collapse;
  h->fine_tile = pick.tile;
  h->fine_threads = pick.threads;
  if (fenv == -1) h->fine_fourier = pick.fourier;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = pick;
}

cudaError_t launch_fine_fcf(mgrit_handle* h, const FcfArgs& f, int prec) {
  if (h->sdirk) return launch_fcf_sdirk(f, h->splan, prec == 0 ? 0 : 1, h->stream);
  if (h->fine_fourier && prec == 1) {  // FP64 pass in Fourier space, collapsed residual pass
    FcfArgs g = f;
    g.m = 1;
    g.fx = h->fx_phim;
    if (fourier_fcf_args_ok(g)) return launch_fcf_fourier(g, h->dphim, h->ftab, h->fine_fourier, h->stream);
  }
  FcfArgs g = f;
  g.fx = h->fx_phi;  // boundary rows (inflow/outflow)
  if (h->fine_collapse) {  // each pass is one application of Phi^m
    g.m = 1;
    g.fx = h->fx_phim;
    return launch_fcf(g, h->dphim, prec, h->fine_threads, h->stream, h->fine_tile);
  }
  return launch_fcf(g, h->dphi, prec, h->fine_threads, h->stream, h->fine_tile);
}

// Boundary rows of Phi and Phi^m (stage-wise closures), FP64 then FP32, in
// one device table (inflow/outflow problems; Psi_l is truncated by the
// kernels' loads and needs no table).
static mgrit_status upload_boundaries(mgrit_handle* h) {
  const int nx = h->nx;
  std::vector<BoundaryRows> rows;
  rows.push_back(inflow_phi_rows(h->prob.rk_order, h->prob.upwind_order, h->prob.cfl, nx));
  if (rows[0].nl + rows[0].nr == 0) return fail(MGRIT_ERR_UNSUPPORTED, "nx too small for the boundary closures");
  // Phi^m's rows for the collapsed path (dropped if its blocks would meet)
  rows.push_back(h->have_phim ? inflow_phi_rows(h->prob.rk_order, h->prob.upwind_order, h->prob.cfl, nx, h->m)
                              : BoundaryRows{});
  if (rows[1].nl + rows[1].nr == 0) h->have_phim = false;
  std::vector<double> w64;
  for (const BoundaryRows& b : rows) w64.insert(w64.end(), b.w.begin(), b.w.end());
  const size_t n = std::max<size_t>(w64.size(), 1);
  double* tab = nullptr;
  mgrit_status st = dalloc(h, n + (n + 1) / 2, &tab);
  if (st != MGRIT_OK) return st;
  float* tab32 = reinterpret_cast<float*>(tab + n);
  const std::vector<float> w32(w64.begin(), w64.end());
  if (!w64.empty()) {
    CUDA_TRY(cudaMemcpyAsync(tab, w64.data(), w64.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    // pageable sources: the copies have staged them when they return
    CUDA_TRY(cudaMemcpyAsync(tab32, w32.data(), w32.size() * sizeof(float), cudaMemcpyHostToDevice, h->stream));
  }
  size_t pos = 0;
  for (size_t k = 0; k < rows.size(); ++k) {
    const BoundaryRows& b = rows[k];
    const Fixup f = {b.nl, b.cl, b.nr, b.cr, tab + pos, tab32 + pos};
    if (k == 0) h->fx_phi = f;
    else h->fx_phim = f;
    pos += b.w.size();
  }
  return MGRIT_OK;
}

// Workspace and tables of the Fourier-space coarsest-level solve (periodic
// stencil Psi, nx = 2^p): twiddles exp(-2 pi i k / nx) and the symbols
// mu_k = sum_i psi_i exp(+2 pi i i k / nx) of the coarsest Psi, in FP64 on
// the device.  Used when the coarsest level has at least kFftMinRows steps:
// the two transforms cost a fixed latency (one CTA per slab, log2(nx)
// dependent stages) that a short march beats.  MGRIT_COARSE=march or =fft
// forces either.
constexpr int kFftMinRows = 16;
// Whether a handle for this request solves its coarsest level in Fourier space.
static bool wants_coarse_fft(const mgrit_problem* p, const mgrit_opts* o, long long rows) {
  const char* cm = std::getenv("MGRIT_COARSE");
  const bool force = cm && std::strcmp(cm, "fft") == 0;
  if ((cm && std::strcmp(cm, "march") == 0) || p->boundary == MGRIT_BC_INFLOW || o->psi_rule == MGRIT_PSI_REDISC ||
      !fft_coarse_supported(p->nx))
    return false;
  return rows >= kFftMinRows || force;
}
static mgrit_status alloc_coarse_fft(mgrit_handle* h);
static mgrit_status setup_coarse_fft(mgrit_handle* h) {
  if (!wants_coarse_fft(&h->prob, &h->opts, h->Nl[h->L - 1])) return MGRIT_OK;
  return alloc_coarse_fft(h);
}
// A server's two-level solve switched to the Fourier-space coarse solve on
// first use (the server picks it per cycle when few solves need a coarse solve;
// a batched march then costs its longest march).  Returns false, with nothing
// changed, where the solve does not qualify.
bool enable_coarse_fft(mgrit_handle* h) {
  if (h->fft_coarse) return true;
  const char* cm = std::getenv("MGRIT_COARSE");
  if ((cm && std::strcmp(cm, "march") == 0) || h->L != 2 || h->redisc || h->inflow ||
      !fft_coarse_supported(h->nx) || h->Nl[1] < kFftMinRows)
    return false;
  if (alloc_coarse_fft(h) != MGRIT_OK) {
    cudaGetLastError();
    return false;
  }
  return true;
}
size_t coarse_fft_bytes(const mgrit_handle* h) {
  const size_t nh = (size_t)h->nx / 2 + 1;
  return (2 * (size_t)h->Nl[h->L - 1] * nh + 3 * (size_t)h->nx + 2 * (size_t)kMaxScanBlocks * nh) * sizeof(double);
}
static mgrit_status alloc_coarse_fft(mgrit_handle* h) {
  const int nx = h->nx, rows = h->Nl[h->L - 1];
  double *spec = nullptr, *tab = nullptr, *carry = nullptr;
  mgrit_status st;
  const size_t nh = (size_t)nx / 2 + 1;  // independent modes of a real slab
  if ((st = dalloc(h, 2 * (size_t)rows * nh, &spec)) != MGRIT_OK || (st = dalloc(h, 3 * (size_t)nx, &tab)) != MGRIT_OK ||
      (st = dalloc(h, 2 * (size_t)kMaxScanBlocks * nh, &carry)) != MGRIT_OK)
    return st;
  // tables on the device: no host work and no pageable copy behind the stream
  CUDA_TRY(launch_fft_tables(h->dpsi.back(), nx, tab, tab + nx, h->stream));
  h->cfft = {spec, rows, tab, tab + nx, carry};
  h->fft_coarse = true;
  return MGRIT_OK;
}

size_t handle_bytes(const mgrit_problem* prob, const mgrit_opts* opts) {
  const size_t nx = prob->nx, m = opts->m, L = opts->levels;
  std::vector<size_t> N(L + 1, 0);
  N[1] = prob->nt / m;
  for (size_t l = 2; l < L; ++l) N[l] = N[l - 1] / m;
  // doubles: two C-point arrays, partials, scratch; the residual and coarse
  // arrays take half as many in the mixed modes (FP32)
  const bool f32 = opts->precision != MGRIT_PREC_FP64;
  auto arr = [&](size_t count) { return f32 ? (count + 1) / 2 : count; };
  size_t d = 2 * (N[1] + 1) * nx + arr((N[1] + 1) * nx) + (N[1] + 1) + 3 * nx + 8;
  for (size_t l = 2; l <= L; ++l) {
    const size_t P = N[l - 1] + 1;
    if (l < L || L > 2) d += arr(P * nx);
    if (l < L) d += 2 * arr((N[l] + 1) * nx);
  }
  if (prob->family == MGRIT_SDIRK) d += 4096;  // recurrence tables and the device plan
  if (prob->boundary == MGRIT_BC_INFLOW) d += 1 << 16;  // boundary-row tables
  return d * sizeof(double);
}

mgrit_status handle_create(const mgrit_problem* prob, const mgrit_opts* opts, cudaStream_t stream,
                           const std::vector<CoarseOp>* ops, mgrit_handle** out, bool sync, bool batched) {
  *out = nullptr;
  const double t0 = now_s();
  mgrit_status st = validate_problem(prob);
  if (st == MGRIT_OK) st = validate_opts(prob, opts);
  if (st != MGRIT_OK) return st;
  if (!slab_pair_fits(prob->nx))
    return fail(MGRIT_ERR_UNSUPPORTED, "nx too large for two shared-memory slabs (max " +
                                           std::to_string(kMaxSlabNx) + ")");
  mgrit_handle* h = new mgrit_handle();
  h->prob = *prob;
  h->opts = *opts;
  h->opts.psi_user_nnz = nullptr;
  h->opts.psi_user_offsets = nullptr;
  h->opts.psi_user_coeffs = nullptr;
  h->stream = stream;
  h->pool_alloc = batched;
  h->nx = prob->nx;
  h->nt = prob->nt;
  h->m = opts->m;
  h->L = opts->levels;
  if (ops) h->ops = *ops;
  else st = plan(prob, opts, &h->ops);
  if (st != MGRIT_OK) {
    delete h;
    return st;
  }
  std::vector<double> sd_tables, cd_tables;
  if (prob->family == MGRIT_SDIRK) {
    h->sdirk = true;
    if ((st = make_sdirk_plan(prob, &h->splan, &sd_tables)) != MGRIT_OK) {
      delete h;
      return st;
    }
    if (sdirk_smem(h->splan) > 227 * 1024) {
      delete h;
      return fail(MGRIT_ERR_UNSUPPORTED, "nx too large for the SDIRK stage slabs in shared memory");
    }
    if (opts->psi_rule == MGRIT_PSI_REDISC) {  // coarse step: the same scheme at m dt
      mgrit_problem pc = *prob;
      pc.cfl = prob->cfl * opts->m;
      h->redisc = true;
      if ((st = make_sdirk_plan(&pc, &h->cplan, &cd_tables)) != MGRIT_OK) {
        delete h;
        return st;
      }
    }
    // Phi is dense for SDIRK; only its order-1 stencil placeholder is kept
    h->phi.off = {0};
    h->phi.coef = {1.0};
  } else {
    h->phi = erk_phi_taps(prob->rk_order, prob->upwind_order, prob->cfl);
  }
  if (h->phi.size() > kMaxDevTaps) {
    delete h;
    return fail(MGRIT_ERR_UNSUPPORTED, "fine stencil too wide");
  }
  for (auto& op : h->ops)
    if (op.taps.size() > kMaxDevTaps) {
      delete h;
      return fail(MGRIT_ERR_UNSUPPORTED, "coarse stencil wider than 256 taps");
    }
  h->dphi = to_dev(h->phi);
  h->inflow = prob->boundary == MGRIT_BC_INFLOW;
  if (!h->sdirk) {  // Phi^m as one stencil (the m-step propagator of an interval)
    Taps pm = taps_power(h->phi, h->m);
    const int reach = std::max(-pm.lo(), pm.hi());
    if (pm.size() <= kMaxDevTaps && pm.size() + 8 < h->nx && reach + 8 < h->nx) {  // indices wrap at most once
      h->dphim = to_dev(pm);
      h->have_phim = true;
    }
  }
  for (auto& op : h->ops) h->dpsi.push_back(to_dev(op.taps));
  // operator complexity, Eq. 5 (ERK)
  {
    double s = h->phi.size();
    double f = 1.0;
    for (auto& op : h->ops) {
      f /= h->m;
      s += f * op.taps.size();
    }
    h->op_complexity = h->sdirk ? 0.0 : s / h->phi.size();
  }
  const int nx = h->nx, L = h->L, m = h->m;
  h->Nl.assign(L + 1, 0);
  h->Nl[1] = h->nt / m;
  for (int l = 2; l < L; ++l) h->Nl[l] = h->Nl[l - 1] / m;
  h->r.assign(L + 1, nullptr);
  h->u.assign(L + 1, nullptr);
  h->cnew.assign(L + 1, nullptr);
  h->rf.assign(L + 1, nullptr);
  h->uf.assign(L + 1, nullptr);
  h->cnewf.assign(L + 1, nullptr);
  h->f32c = opts->precision != MGRIT_PREC_FP64;
  const size_t N1 = h->Nl[1];
  auto A = [&](size_t count, double** p) { return dalloc(h, count, p); };
  // an array of `count` values, FP32 in the mixed modes, zero-filled
  auto AZ = [&](size_t count, double** pd, float** pf) -> mgrit_status {
    mgrit_status s2;
    if (h->f32c) {
      double* d = nullptr;
      if ((s2 = dalloc(h, (count + 1) / 2, &d)) != MGRIT_OK) return s2;
      *pf = reinterpret_cast<float*>(d);
      cudaMemsetAsync(d, 0, count * sizeof(float), h->stream);
    } else {
      if ((s2 = dalloc(h, count, pd)) != MGRIT_OK) return s2;
      cudaMemsetAsync(*pd, 0, count * sizeof(double), h->stream);
    }
    return MGRIT_OK;
  };
  // the level-1 residual: FP32 in the mixed modes (the FCF residual comes out
  // of the FP32 pass), except two-level F-relaxation, whose residual is the
  // FP64 pass's and feeds the FP64 march directly
  const bool r1_f32 = h->f32c && !(opts->relax == MGRIT_RELAX_F && L == 2);
  auto AZ1 = [&](size_t count) -> mgrit_status {
    if (r1_f32) return AZ(count, &h->r[1], &h->rf[1]);
    mgrit_status s2 = dalloc(h, count, &h->r[1]);
    if (s2 == MGRIT_OK) cudaMemsetAsync(h->r[1], 0, count * sizeof(double), h->stream);
    return s2;
  };
  h->dfc = fine_prec(h) == 3;  // MIXED_DF, ERK: level-1 C-points as float-float pairs
  if ((st = A((N1 + 1) * nx, &h->c[0])) != MGRIT_OK || (st = A((N1 + 1) * nx, &h->c[1])) != MGRIT_OK ||
      (st = A(nx, &h->u0buf)) != MGRIT_OK ||
      (st = AZ1((N1 + 1) * nx)) != MGRIT_OK || (st = A(N1 + 1, &h->partial)) != MGRIT_OK ||
      (st = A(2 * (size_t)nx + 8, &h->scratch)) != MGRIT_OK) {
    release(h);
    delete h;
    return st;
  }
  cudaMemsetAsync(h->partial, 0, (N1 + 1) * sizeof(double), h->stream);
  for (int l = 2; l <= L; ++l) {
    const size_t P = (size_t)h->Nl[l - 1] + 1;  // points of level l
    if (l < L || L > 2)
      if ((st = AZ(P * nx, &h->u[l], &h->uf[l])) != MGRIT_OK) break;
    if (l < L) {
      const size_t Nc = (size_t)h->Nl[l] + 1;
      if ((st = AZ(Nc * nx, &h->cnew[l], &h->cnewf[l])) != MGRIT_OK ||
          (st = AZ(Nc * nx, &h->r[l], &h->rf[l])) != MGRIT_OK)
        break;
    }
  }
  if (st != MGRIT_OK) {
    release(h);
    delete h;
    return st;
  }
  if (h->inflow && (st = upload_boundaries(h)) != MGRIT_OK) {
    release(h);
    delete h;
    return st;
  }
  if (!batched && (st = setup_coarse_fft(h)) != MGRIT_OK) {
    release(h);
    delete h;
    return st;
  }
  if (!(h->norm_host = pinned_slot())) {
    release(h);
    delete h;
    return fail(MGRIT_ERR_OOM, "pinned host buffer");
  }
  if (h->sdirk) {  // recurrence tables (FP64 then FP32) and a device copy of the plan
    const size_t tl = (size_t)h->splan.tab_len;
    double* tab = nullptr;
    double* dplan = nullptr;
    if ((st = A(tl + (tl + 1) / 2, &tab)) != MGRIT_OK || (st = A((sizeof(SdirkPlan) + 7) / 8, &dplan)) != MGRIT_OK) {
      release(h);
      delete h;
      return st;
    }
    const std::vector<float> t32(sd_tables.begin(), sd_tables.end());
    h->splan.tab64 = tab;
    h->splan.tab32 = reinterpret_cast<float*>(tab + tl);
    h->dsplan = reinterpret_cast<SdirkPlan*>(dplan);
    cudaMemcpyAsync(tab, sd_tables.data(), tl * sizeof(double), cudaMemcpyHostToDevice, h->stream);
    cudaMemcpyAsync(tab + tl, t32.data(), tl * sizeof(float), cudaMemcpyHostToDevice, h->stream);
    cudaMemcpyAsync(dplan, &h->splan, sizeof(SdirkPlan), cudaMemcpyHostToDevice, h->stream);
    if (h->redisc) {
      const size_t tc = (size_t)h->cplan.tab_len;
      double* ctab = nullptr;
      if ((st = A(tc + (tc + 1) / 2, &ctab)) != MGRIT_OK) {
        release(h);
        delete h;
        return st;
      }
      const std::vector<float> c32(cd_tables.begin(), cd_tables.end());
      h->cplan.tab64 = ctab;
      h->cplan.tab32 = reinterpret_cast<float*>(ctab + tc);
      cudaMemcpyAsync(ctab, cd_tables.data(), tc * sizeof(double), cudaMemcpyHostToDevice, h->stream);
      cudaMemcpyAsync(ctab + tc, c32.data(), tc * sizeof(float), cudaMemcpyHostToDevice, h->stream);
    }
  }
  h->fcf_threads = 0;  // chosen per launch from nx and the register tile
  if (const char* tile = std::getenv("MGRIT_TILE")) set_tile(std::atoi(tile));
  if (const char* sf = std::getenv("MGRIT_FCF_STREAM")) set_stream_fused(std::atoi(sf));
  const Taps& coarsest = h->ops.back().taps;
  h->march_cluster = pick_cluster(nx, coarsest);
  h->march_threads = std::min(256, (nx + h->march_cluster - 1) / h->march_cluster);
  // tables of the Fourier-space FP64 pass (MIXED periodic level 1; not for a
  // server's handles, whose level-1 FCF is the batched launch)
  if (fine_prec(h) == 1 && !h->sdirk && !h->inflow && !h->pool_alloc && h->have_phim && fourier_fcf_supported(nx) &&
      fourier_env() != 0) {
    double* tab = nullptr;
    if (dalloc(h, fourier_table_doubles(nx), &tab) == MGRIT_OK &&
        launch_fourier_tables(h->dphim, nx, tab, h->stream) == cudaSuccess) {
      h->ftab = tab;
    } else {
      cudaGetLastError();
    }
  }
  const double tt = now_s();
  autotune_fine(h);
  h->tune_s = now_s() - tt;
  cudaError_t e = sync ? cudaStreamSynchronize(h->stream) : cudaGetLastError();
  if (e != cudaSuccess) {
    release(h);
    delete h;
    return fail(MGRIT_ERR_CUDA, cudaGetErrorString(e));
  }
  h->setup_s = now_s() - t0;
  *out = h;
  return MGRIT_OK;
}

extern "C" mgrit_status mgrit_setup(const mgrit_problem* prob, const mgrit_opts* opts, void* stream,
                                    mgrit_handle** out) {
  if (!out) return fail(MGRIT_ERR_INVALID, "out is NULL");
  return handle_create(prob, opts, (cudaStream_t)stream, nullptr, out);
}

extern "C" void mgrit_destroy(mgrit_handle* h) {
  if (!h) return;
  release(h);
  delete h;
}

extern "C" size_t mgrit_device_bytes(const mgrit_handle* h) { return h ? h->bytes : 0; }

extern "C" mgrit_status mgrit_psi_info(mgrit_handle* h, int32_t level, int32_t cap, int32_t* nnz, int32_t* offsets,
                                       double* coeffs) {
  if (!h) return fail(MGRIT_ERR_INVALID, "handle is NULL");
  if (level < 2 || level > h->L) return fail(MGRIT_ERR_INVALID, "level must be 2..levels");
  if (h->redisc) return fail(MGRIT_ERR_UNSUPPORTED, "the rediscretised Psi is an implicit step, not a stencil");
  const Taps& t = h->ops[level - 2].taps;
  if (nnz) *nnz = t.size();
  if (t.size() > cap) return fail(MGRIT_ERR_INVALID, "capacity too small");
  for (int k = 0; k < t.size(); ++k) {
    if (offsets) offsets[k] = t.off[k];
    if (coeffs) coeffs[k] = t.coef[k];
  }
  return MGRIT_OK;
}

// ------------------------------------------------------------------- solve

mgrit_status launch_ok(cudaError_t e, const char* what) {
  if (e != cudaSuccess) return fail(MGRIT_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return MGRIT_OK;
}

void reset_stats(mgrit_handle* h) {
  for (int k = 0; k < MGRIT_K_KINDS; ++k) h->kcount[k] = 0;
  h->evkind.clear();
  h->evused = 0;
}

cudaEvent_t next_event(mgrit_handle* h) {
  if (h->evused == h->evpool.size()) {
    cudaEvent_t ev;
    if (cudaEventCreate(&ev) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    h->evpool.push_back(ev);
  }
  return h->evpool[h->evused++];
}

void collect_stats(mgrit_handle* h, mgrit_result* R) {
  int total = 0;
  for (int k = 0; k < MGRIT_K_KINDS; ++k) {
    R->kernel_count[k] = h->kcount[k];
    R->kernel_ms[k] = 0.0;
    total += h->kcount[k];
  }
  R->launches = total;
  R->fine_tile = h->fine_tile;
  R->fine_threads = h->fine_threads;
  R->fine_collapsed = h->fine_collapse;
  R->fine_fourier = h->fine_fourier ? 1 : 0;
  for (size_t p = 0; p < h->evkind.size(); ++p) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, h->evpool[2 * p], h->evpool[2 * p + 1]) == cudaSuccess)
      R->kernel_ms[h->evkind[p]] += ms;
    else
      cudaGetLastError();
  }
}

// Launch a march, shrinking the cluster if the device refuses the size.
mgrit_status run_march(mgrit_handle* h, const MarchArgs& a, const DevTaps& t) {
  return klaunch(h, MGRIT_K_MARCH, "march", [&]() -> mgrit_status {
    for (;;) {
      int threads = std::min(256, (a.nx + h->march_cluster - 1) / h->march_cluster);
      cudaError_t e = launch_march(a, t, h->march_cluster, threads, h->stream);
      if (e == cudaSuccess) return MGRIT_OK;
      cudaGetLastError();
      if (h->march_cluster == 1) return launch_ok(e, "march_kernel");
      h->march_cluster >>= 1;
    }
  });
}

mgrit_status run_coarse_solve(mgrit_handle* h, const MarchArgs& a, const DevTaps& t) {
  if (!h->fft_coarse) return run_march(h, a, t);
  mgrit_status st = klaunch(h, MGRIT_K_MARCH, "coarse fft", [&] {
    return launch_ok(launch_coarse_fft(a, h->cfft, h->stream), "coarse solve (Fourier space)");
  });
  if (st == MGRIT_OK) h->kcount[MGRIT_K_MARCH] += coarse_fft_launches(a.nx, a.P) - 1;  // klaunch counted one
  return st;
}

// ||Phi u0||: residual of the zero initial iterate (only time level 1 is nonzero).
mgrit_status initial_residual(mgrit_handle* h, const double* u0dev, double* r0) {
  mgrit_status st = initial_residual_async(h, u0dev);
  if (st != MGRIT_OK) return st;
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  *r0 = std::sqrt(h->norm_host[0]);
  return MGRIT_OK;
}

// Enqueue ||r^(0)||^2 into h->norm_host[0] (read after a stream sync):
// ||Phi u0||^2 for the zero iterate, the full space-time residual for the
// random one.
mgrit_status initial_residual_async(mgrit_handle* h, const double* u0dev) {
  mgrit_status st;
  double* out = h->scratch;
  double* part = h->scratch + h->nx;
  if (h->iterate_random) {
    int launches = 0;
    if ((st = enqueue_r0sq(h, part, &launches)) != MGRIT_OK) return st;
    h->kcount[MGRIT_K_PROPAGATE] += launches;
    CUDA_TRY(cudaMemcpyAsync(h->norm_host, part, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    return MGRIT_OK;
  }
  if ((st = klaunch(h, MGRIT_K_PROPAGATE, "propagate", [&] {
         if (h->sdirk) return launch_ok(launch_propagate_sdirk(u0dev, out, 1, h->nx, 1, h->splan, part, h->stream),
                                        "propagate");
         return launch_ok(
             launch_propagate(u0dev, out, 1, h->nx, 1, h->dphi, part, h->fcf_threads, h->stream, &h->fx_phi),
             "propagate");
       })) != MGRIT_OK)
    return st;
  CUDA_TRY(cudaMemcpyAsync(h->norm_host, part, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  return MGRIT_OK;
}

mgrit_status enqueue_r0sq(mgrit_handle* h, double* dst, int* launches) {
  const int nx = h->nx;
  *launches = 0;
  if (!h->iterate_random) {
    *launches = 1;
    if (h->sdirk)
      return launch_ok(launch_propagate_sdirk(h->u0buf, h->scratch, 1, nx, 1, h->splan, dst, h->stream), "propagate");
    return launch_ok(launch_propagate(h->u0buf, h->scratch, 1, nx, 1, h->dphi, dst, h->fcf_threads, h->stream,
                                      &h->fx_phi),
                     "propagate");
  }
  // r_n = Phi u_{n-1} - u_n for n = 1..nt over chunks of N1 levels: draw
  // u_{n-1} into rows 1..N1 of c[1] (free until the first FCF writes them),
  // step them in place, and sum the squared differences to the draws of u_n
  const int rows = h->Nl[1];
  double* buf = h->c[1] + nx;
  const unsigned long long seed = h->opts.seed;
  int q = 0;
  for (long long n0 = 0; n0 < h->nt; n0 += rows, ++q) {
    const int cnt = (int)std::min<long long>(rows, h->nt - n0);
    cudaError_t e = launch_random_rows(buf, h->u0buf, nx, n0, 1, cnt, seed, h->stream);
    if (e == cudaSuccess)
      e = h->sdirk ? launch_propagate_sdirk(buf, buf, cnt, nx, 1, h->splan, nullptr, h->stream)
                   : launch_propagate(buf, buf, cnt, nx, 1, h->dphi, nullptr, h->fcf_threads, h->stream, &h->fx_phi);
    if (e == cudaSuccess) e = launch_random_residual(buf, h->partial, nx, n0, cnt, seed, h->stream);
    if (e == cudaSuccess) e = launch_accumulate(h->partial, cnt, dst, q == 0, h->stream);
    if (e != cudaSuccess) return launch_ok(e, "random initial residual");
    *launches += 4;
  }
  // the residual norms of the cycles sum partial[0], which no relaxation
  // writes: leave the partials as zero as the handle was created with them
  CUDA_TRY(cudaMemsetAsync(h->partial, 0, (size_t)(rows + 1) * sizeof(double), h->stream));
  return MGRIT_OK;
}

// Cycles below level 1.  Level l (2..L-1) keeps all its points in u[l], its
// relaxed C-points in cnew[l] and its C-point residual (level l+1's right-hand
// side) in r[l]; level l's right-hand side is r[l-1]; the coarsest level L
// marches into u[L].  Coarse levels relax the error equation: FP32 in the
// mixed modes.
namespace {
int coarse_prec(const mgrit_handle* h) { return h->opts.precision == MGRIT_PREC_FP64 ? 0 : 2; }

// FCF-relaxation of level l from zero (the first visit) or from u[l].
mgrit_status relax_level(mgrit_handle* h, int l, bool from_zero) {
  const int nx = h->nx, m = h->m, prec = coarse_prec(h);
  FcfArgs f = {};
  f.u_old = h->u[l];
  f.cstride = (long long)m * nx;
  f.c_new = h->cnew[l];
  f.g = h->r[l - 1];
  f.r = h->r[l];
  f.u_old_f = h->uf[l];
  f.c_new_f = h->cnewf[l];
  f.g_f = h->rf[l - 1];
  f.r_f = h->rf[l];
  f.partial = nullptr;
  f.nx = nx;
  f.m = m;
  f.N = h->Nl[l];
  f.zero_old = from_zero ? 1 : 0;
  f.trunc = h->inflow;
  return klaunch(h, MGRIT_K_FCF_COARSE, "fcf", [&] {
    return launch_ok(launch_fcf(f, h->dpsi[l - 2], prec, h->fcf_threads, h->stream), "fcf(coarse)");
  });
}

// Exact solve of the coarsest level: u[L] from r[L-1].
mgrit_status solve_coarsest(mgrit_handle* h) {
  const int L = h->L;
  MarchArgs a = {};
  a.g = h->r[L - 1];
  a.g_f = h->rf[L - 1];
  a.u_out = h->u[L];
  a.u_out_f = h->uf[L];
  a.store_every = 1;
  a.nx = h->nx;
  a.trunc = h->inflow;
  a.P = h->Nl[L - 1] + 1;
  return run_coarse_solve(h, a, h->dpsi[L - 2]);
}

// u[l] = relaxed C-points + u[l+1], then F-relaxation (ideal interpolation).
mgrit_status correct_level(mgrit_handle* h, int l) {
  const int prec = coarse_prec(h);
  CorrectArgs c = {};
  c.c_new = h->cnew[l];
  c.e = h->u[l + 1];
  c.g = h->r[l - 1];
  c.u = h->u[l];
  c.c_new_f = h->cnewf[l];
  c.e_f = h->uf[l + 1];
  c.g_f = h->rf[l - 1];
  c.u_f = h->uf[l];
  c.nx = h->nx;
  c.m = h->m;
  c.N = h->Nl[l];
  c.trunc = h->inflow;
  return klaunch(h, MGRIT_K_CORRECT, "correct", [&] {
    return launch_ok(launch_correct(c, h->dpsi[l - 2], h->fcf_threads, h->stream, prec == 2), "correct");
  });
}

mgrit_status vcycle_level(mgrit_handle* h, int l, bool from_zero) {
  if (l == h->L) return solve_coarsest(h);
  mgrit_status st;
  if ((st = relax_level(h, l, from_zero)) != MGRIT_OK) return st;
  if ((st = vcycle_level(h, l + 1, true)) != MGRIT_OK) return st;
  return correct_level(h, l);
}

// F-cycle: the coarse error equation is solved by an F-cycle from zero and
// then a V-cycle from that result (once, exactly, above the coarsest level).
mgrit_status fcycle_level(mgrit_handle* h, int l) {
  if (l == h->L) return solve_coarsest(h);
  mgrit_status st;
  if ((st = relax_level(h, l, true)) != MGRIT_OK) return st;
  if ((st = fcycle_level(h, l + 1)) != MGRIT_OK) return st;
  if (l + 1 < h->L && (st = vcycle_level(h, l + 1, false)) != MGRIT_OK) return st;
  return correct_level(h, l);
}
}  // namespace

// One coarse-grid correction of level 1: c_new += e (e from the coarse
// levels; fused into the march when L = 2).
mgrit_status coarse_cycle(mgrit_handle* h, double* c_new) {
  const int L = h->L, nx = h->nx;
  mgrit_status st;
  if (L == 2 && h->redisc) {  // e_j = Phi(m dt) e_{j-1} + r_j, c_j += e_j, one CTA
    return klaunch(h, MGRIT_K_MARCH, "march", [&] {
      return launch_ok(launch_coarse_march_sdirk(h->r[1], h->rf[1], c_new, nx, h->Nl[1] + 1, h->cplan, h->stream),
                       "coarse march (SDIRK)");
    });
  }
  if (L == 2) {
    MarchArgs a = {};
    a.init = nullptr;
    a.g = h->r[1];
    a.g_f = h->rf[1];
    a.c_add = c_new;
    a.c_add_df = h->dfc;
    a.nx = nx;
    a.trunc = h->inflow;
    a.P = h->Nl[1] + 1;
    a.store_every = 1;
    return run_coarse_solve(h, a, h->dpsi[0]);
  }
  st = h->opts.cycle == MGRIT_CYCLE_F ? fcycle_level(h, 2) : vcycle_level(h, 2, true);
  if (st != MGRIT_OK) return st;
  return klaunch(h, MGRIT_K_ADD, "add", [&] {
    if (h->f32c)
      return launch_ok(launch_add_f(c_new + nx, h->uf[2] + nx, (long long)h->Nl[1] * nx, h->stream, h->dfc), "add");
    return launch_ok(launch_add(c_new + nx, h->u[2] + nx, (long long)h->Nl[1] * nx, h->stream), "add");
  });
}

mgrit_status write_output(mgrit_handle* h, const double* cres, double* out) {
  const int nx = h->nx, m = h->m;
  const size_t N1 = h->Nl[1];
  const size_t slab = (size_t)nx * sizeof(double);
  mgrit_status st;
  if (h->dfc) {  // float-float C-points: to FP64 in the other (now free) C-point array
    double* tmp = cres == h->c[0] ? h->c[1] : h->c[0];
    if ((st = klaunch(h, MGRIT_K_OTHER, "convert", [&] {
           return launch_ok(launch_convert_df(cres, tmp, (long long)(N1 + 1) * nx, 0, h->stream), "convert");
         })) != MGRIT_OK)
      return st;
    cres = tmp;
  }
  if (h->opts.output == MGRIT_OUT_FINAL) {
    CUDA_TRY(cudaMemcpyAsync(out, cres + N1 * nx, slab, kind_from_dev(out), h->stream));
  } else if (h->opts.output == MGRIT_OUT_CPOINTS) {
    CUDA_TRY(cudaMemcpyAsync(out, cres, (N1 + 1) * slab, kind_from_dev(out), h->stream));
  } else {
    // F-points by one F-relaxation from the C-points (ideal interpolation)
    double* full = nullptr;
    const bool dev = is_device_ptr(out);
    if (dev) full = out;
    else if ((st = dalloc(h, (size_t)(h->nt + 1) * nx, &full)) != MGRIT_OK) return st;
    CorrectArgs c = {};
    c.c_new = cres;
    c.e = nullptr;
    c.g = nullptr;
    c.u = full;
    c.nx = nx;
    c.m = m;
    c.N = (int)N1;
    c.fx = h->fx_phi;
    if ((st = klaunch(h, MGRIT_K_OTHER, "interp", [&] {
           if (h->sdirk)
             return launch_ok(launch_interp_sdirk(cres, full, nx, m, (int)N1, h->splan, h->stream), "interp");
           return launch_ok(launch_correct(c, h->dphi, h->fcf_threads, h->stream), "interp");
         })) != MGRIT_OK)
      return st;
    if (!dev) {
      CUDA_TRY(cudaMemcpyAsync(out, full, (size_t)(h->nt + 1) * slab, cudaMemcpyDeviceToHost, h->stream));
      CUDA_TRY(cudaStreamSynchronize(h->stream));
      DevBuf b = h->bufs.back();
      h->bufs.pop_back();
      h->bytes -= std::max<size_t>(b.n, 1) * sizeof(double);
      if (b.freefn) b.freefn(b.p, (void*)h->stream, b.ctx);
      else cudaFreeAsync(b.p, h->stream);
    }
  }
  return MGRIT_OK;
}

// ----------------------------------------------------------- graph solve

// Capture the launches fn() issues on the handle into `body` (a conditional
// node's body graph); *leaf receives the last captured node.
template <typename F>
static mgrit_status capture_into(mgrit_handle* h, cudaGraph_t body, F&& fn, cudaGraphNode_t* leaf) {
  cudaStream_t saved = h->stream;
  cudaError_t e = cudaStreamBeginCaptureToGraph(h->cap_stream, body, nullptr, nullptr, 0,
                                                cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) return launch_ok(e, "begin capture");
  h->stream = h->cap_stream;
  mgrit_status st = fn();
  h->stream = saved;
  cudaStreamCaptureStatus cs;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  e = cudaStreamGetCaptureInfo(h->cap_stream, &cs, nullptr, nullptr, &deps, nullptr, &ndeps);
  if (e == cudaSuccess && leaf) *leaf = ndeps ? deps[0] : nullptr;
  cudaGraph_t out = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &out);
  if (st != MGRIT_OK) return st;
  if (e != cudaSuccess) return launch_ok(e, "capture info");
  return launch_ok(e2, "end capture");
}

static mgrit_status add_conditional(cudaGraph_t g, cudaGraphNode_t dep, cudaGraphConditionalHandle hd,
                                    cudaGraphConditionalNodeType type, cudaGraph_t* body) {
  cudaGraphNodeParams p = {};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = hd;
  p.conditional.type = type;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  cudaError_t e = cudaGraphAddNode(&node, g, dep ? &dep : nullptr, nullptr, dep ? 1 : 0, &p);
  if (e != cudaSuccess) return launch_ok(e, "conditional node");
  *body = p.conditional.phGraph_out[0];
  return MGRIT_OK;
}

// One level-1 FCF + norm + stopping test reading c[cur], writing c[1-cur].
static mgrit_status graph_cycle(mgrit_handle* h, int cur, cudaGraphConditionalHandle hw,
                                cudaGraphConditionalHandle hif) {
  const int nx = h->nx;
  FcfArgs f = {};
  f.u_old = h->c[cur];
  f.cstride = nx;
  f.c_new = h->c[1 - cur];
  f.r = h->r[1];
  f.r_f = h->rf[1];
  f.partial = h->partial;
  f.nx = nx;
  f.m = h->m;
  f.N = h->Nl[1];
  f.relax_f = h->opts.relax == MGRIT_RELAX_F;
  f.value_residual = fine_prec(h) == 0 && !f.relax_f;
  f.df_store = h->dfc;
  mgrit_status st;
  if ((st = launch_ok(launch_fine_fcf(h, f, fine_prec(h)), "fcf")) != MGRIT_OK) return st;
  if (f.value_residual &&
      (st = launch_ok(launch_residual_value(f.c_new, f.r, f.partial, nx, f.N, h->stream), "residual")) != MGRIT_OK)
    return st;
  if ((st = launch_ok(launch_norm(h->partial, h->Nl[1] + f.relax_f, h->scratch + 2 * nx, h->stream), "norm")) !=
      MGRIT_OK)
    return st;
  return launch_ok(launch_check(h->scratch + 2 * nx, h->dstate, hw, hif, cur, h->stream), "check");
}

// WHILE(not stopped) { cycle(0); IF(go on) { coarse -> c[1]; cycle(1); IF(go on) { coarse -> c[0] } } }
static mgrit_status build_solve_graph(mgrit_handle* h) {
  mgrit_status st;
  if (!h->cap_stream && cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
    return launch_ok(cudaGetLastError(), "capture stream");
  if (!h->dstate) {
    double* p = nullptr;
    if ((st = dalloc(h, sizeof(CheckState) / sizeof(double) + 1, &p)) != MGRIT_OK) return st;
    h->dstate = reinterpret_cast<CheckState*>(p);
  }
  if (!h->hstate && cudaMallocHost(&h->hstate, sizeof(CheckState)) != cudaSuccess)
    return launch_ok(cudaGetLastError(), "pinned state");
  cudaGraph_t g = nullptr;
  if (cudaGraphCreate(&g, 0) != cudaSuccess) return launch_ok(cudaGetLastError(), "graph");
  h->graph = g;
  // each conditional handle belongs to the graph that holds its node
  cudaGraphConditionalHandle hw, hif0, hif1;
  cudaError_t e = cudaGraphConditionalHandleCreate(&hw, g, 1, cudaGraphCondAssignDefault);
  if (e != cudaSuccess) return launch_ok(e, "conditional handle");
  cudaGraph_t body_w, body_if0, body_if1;
  cudaGraphNode_t leaf = nullptr;
  if ((st = add_conditional(g, nullptr, hw, cudaGraphCondTypeWhile, &body_w)) != MGRIT_OK) return st;
  if ((e = cudaGraphConditionalHandleCreate(&hif0, body_w, 0, cudaGraphCondAssignDefault)) != cudaSuccess)
    return launch_ok(e, "conditional handle");
  if ((st = capture_into(h, body_w, [&] { return graph_cycle(h, 0, hw, hif0); }, &leaf)) != MGRIT_OK) return st;
  if ((st = add_conditional(body_w, leaf, hif0, cudaGraphCondTypeIf, &body_if0)) != MGRIT_OK) return st;
  if ((e = cudaGraphConditionalHandleCreate(&hif1, body_if0, 0, cudaGraphCondAssignDefault)) != cudaSuccess)
    return launch_ok(e, "conditional handle");
  const int before = h->kcount[MGRIT_K_MARCH] + h->kcount[MGRIT_K_FCF_COARSE] + h->kcount[MGRIT_K_CORRECT] +
                     h->kcount[MGRIT_K_ADD];
  if ((st = capture_into(h, body_if0, [&] {
         mgrit_status s2 = coarse_cycle(h, h->c[1]);
         return s2 != MGRIT_OK ? s2 : graph_cycle(h, 1, hw, hif1);
       }, &leaf)) != MGRIT_OK)
    return st;
  h->graph_coarse_launches = h->kcount[MGRIT_K_MARCH] + h->kcount[MGRIT_K_FCF_COARSE] +
                             h->kcount[MGRIT_K_CORRECT] + h->kcount[MGRIT_K_ADD] - before;
  if ((st = add_conditional(body_if0, leaf, hif1, cudaGraphCondTypeIf, &body_if1)) != MGRIT_OK) return st;
  if ((st = capture_into(h, body_if1, [&] { return coarse_cycle(h, h->c[0]); }, nullptr)) != MGRIT_OK) return st;
  e = cudaGraphInstantiate(&h->gexec, g, 0);
  if (e != cudaSuccess) return launch_ok(e, "graph instantiate");
  return MGRIT_OK;
}

// Whole solve: prologue on the stream, one graph launch, one read-back.
// Initial iterate on the device: C-points from c_init (rows 0..N1) or zero
// (row 0 = u0).
// The initial iterate into c[0] (C-point 0 also into c[1]) and u0 in FP64
// into u0buf; float-float pairs when the handle stores its C-points so.
mgrit_status load_iterate(mgrit_handle* h, const double* u0, const double* c_init) {
  const int nx = h->nx;
  const size_t N1 = h->Nl[1];
  const size_t slab = (size_t)nx * sizeof(double);
  double* dst = h->dfc ? h->c[1] : h->c[0];  // float-float: stage the FP64 values in c[1]
  h->iterate_random = false;
  if (!c_init && h->opts.init_guess == MGRIT_INIT_RANDOM) {
    // Section 2.2: u0 at t = 0, uniform draws at every later C-point
    // (row j = time level j m); F-points are drawn where the initial residual
    // needs them
    CUDA_TRY(cudaMemcpyAsync(h->u0buf, u0, slab, kind_to_dev(u0), h->stream));
    CUDA_TRY(launch_random_rows(dst, h->u0buf, nx, 0, h->m, (int)N1 + 1, h->opts.seed, h->stream));
    if (h->dfc) CUDA_TRY(launch_convert_df(dst, h->c[0], (long long)(N1 + 1) * nx, 1, h->stream));
    h->iterate_random = true;
  } else if (c_init) {
    CUDA_TRY(cudaMemcpyAsync(dst, c_init, (N1 + 1) * slab, kind_to_dev(c_init), h->stream));
    CUDA_TRY(cudaMemcpyAsync(h->u0buf, dst, slab, cudaMemcpyDeviceToDevice, h->stream));
    if (h->dfc) CUDA_TRY(launch_convert_df(dst, h->c[0], (long long)(N1 + 1) * nx, 1, h->stream));
  } else {
    CUDA_TRY(cudaMemcpyAsync(h->u0buf, u0, slab, kind_to_dev(u0), h->stream));
    if (h->dfc) CUDA_TRY(launch_convert_df(h->u0buf, h->c[0], nx, 1, h->stream));
    else CUDA_TRY(cudaMemcpyAsync(h->c[0], h->u0buf, slab, cudaMemcpyDeviceToDevice, h->stream));
    CUDA_TRY(cudaMemsetAsync(h->c[0] + nx, 0, N1 * slab, h->stream));  // zero bits: 0.0 in both forms
  }
  CUDA_TRY(cudaMemcpyAsync(h->c[1], h->c[0], slab, cudaMemcpyDeviceToDevice, h->stream));
  return MGRIT_OK;
}

static mgrit_status solve_graph(mgrit_handle* h, const double* u0, const double* c_init, double r0_norm,
                                double* out, mgrit_result* R) {
  const int nx = h->nx;
  mgrit_status st;
  if ((st = load_iterate(h, u0, c_init)) != MGRIT_OK) return st;
  std::memset(h->hstate, 0, sizeof(CheckState));
  h->hstate->tol = h->opts.tol;
  h->hstate->max_iter = h->opts.max_iter;
  h->hstate->diverge = (h->opts.flags & MGRIT_FLAG_NO_DIVERGENCE_STOP) ? 0.0 : 1e6;
  h->hstate->r0sq = r0_norm > 0.0 ? r0_norm * r0_norm : 0.0;
  CUDA_TRY(cudaMemcpyAsync(h->dstate, h->hstate, sizeof(CheckState), cudaMemcpyHostToDevice, h->stream));
  // otherwise ||r^(0)||^2 straight into the state (zero initial iterate:
  // r^(0) = Phi u0; random iterate: its full space-time residual)
  int r0_launches = 0;
  if (!(r0_norm > 0.0) && (st = enqueue_r0sq(h, &h->dstate->r0sq, &r0_launches)) != MGRIT_OK) return st;
  CUDA_TRY(cudaGraphLaunch(h->gexec, h->stream));
  CUDA_TRY(cudaMemcpyAsync(h->hstate, h->dstate, sizeof(CheckState), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  const CheckState& S = *h->hstate;
  R->r0_norm = std::sqrt(S.r0sq);
  R->iterations = S.it;
  R->rel_residual = S.rel;
  R->n_history = std::min(S.nhist, MGRIT_MAX_HISTORY);
  for (int k = 0; k < R->n_history; ++k) R->history[k] = S.hist[k];
  R->converged = S.status == 0 && S.done ? 1 : 0;
  // launches: initial residual, (it+1) x (fcf, norm, check), it x coarse correction
  reset_stats(h);
  h->kcount[MGRIT_K_PROPAGATE] = r0_launches;
  h->kcount[MGRIT_K_FCF] = S.it + 1;
  h->kcount[MGRIT_K_NORM] = (fine_prec(h) == 0 && h->opts.relax == MGRIT_RELAX_FCF ? 2 : 1) * (S.it + 1);
  h->kcount[MGRIT_K_OTHER] = S.it + 1;
  h->last = 1 - S.result_cur;
  h->r0_last = R->r0_norm;
  if (out && (st = write_output(h, h->c[1 - S.result_cur], out)) != MGRIT_OK) return st;
  if (!S.done) return fail(MGRIT_ERR_CUDA, "graph ended without a stopping decision");
  if (S.status == -5) return fail(MGRIT_ERR_DIVERGED, "residual not finite or grew above 1e6 x initial");
  if (S.status == -4) return fail(MGRIT_ERR_NOT_CONVERGED, "max_iter reached");
  return MGRIT_OK;
}

// Build the solve graph at the first graph solve; false (and no half-built
// graph kept) when the device refuses it: the host-driven loop runs instead.
static bool ensure_graph(mgrit_handle* h) {
  if (h->graph_failed) return false;
  if (h->gexec) return true;
  const std::string keep = g_err;
  if (build_solve_graph(h) == MGRIT_OK) return true;
  h->graph_failed = true;
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->graph) cudaGraphDestroy(h->graph);
  h->gexec = nullptr;
  h->graph = nullptr;
  cudaGetLastError();
  g_err = keep;
  return false;
}

static mgrit_status solve_impl(mgrit_handle* h, const double* u0, const double* c_init, double r0_norm,
                               double* out, mgrit_result* res) {
  const double t0 = now_s();
  const int nx = h->nx, m = h->m;
  const size_t N1 = h->Nl[1];
  const size_t slab = (size_t)nx * sizeof(double);
  mgrit_result R;
  std::memset(&R, 0, sizeof(R));
  R.n_levels = h->L;
  R.setup_s = h->setup_s;
  R.op_complexity = h->op_complexity;
  reset_stats(h);
  grid_spacings(&h->prob, &R.dx, &R.dt);
  const bool host_loop = (h->opts.flags & (MGRIT_FLAG_TIME_KERNELS | MGRIT_FLAG_HOST_LOOP)) != 0;
  if (!host_loop && ensure_graph(h)) {
    mgrit_status gs = solve_graph(h, u0, c_init, r0_norm, out, &R);
    if (gs == MGRIT_OK || gs == MGRIT_ERR_NOT_CONVERGED || gs == MGRIT_ERR_DIVERGED) {
      CUDA_TRY(cudaStreamSynchronize(h->stream));
      R.solve_s = now_s() - t0;
      R.dof_per_s = R.solve_s > 0 ? (double)nx * h->nt / R.solve_s : 0.0;
      collect_stats(h, &R);
      R.launches += R.iterations * h->graph_coarse_launches;
      R.graph = 1;
      if (res) *res = R;
    }
    return gs;
  }
  int cur = 0;
  mgrit_status st = load_iterate(h, u0, c_init);
  if (st != MGRIT_OK) return st;
  double r0 = r0_norm;
  if (!(r0_norm > 0.0) && (st = initial_residual(h, h->u0buf, &r0)) != MGRIT_OK) return st;
  R.r0_norm = r0;
  const int prec = fine_prec(h);
  mgrit_status final_status = MGRIT_OK;
  int it = 0;
  for (;;) {
    FcfArgs f = {};
    f.u_old = h->c[cur];
    f.cstride = nx;
    f.c_new = h->c[1 - cur];
    f.g = nullptr;
    f.r = h->r[1];
    f.r_f = h->rf[1];
    f.partial = h->partial;
    f.nx = nx;
    f.m = m;
    f.N = (int)N1;
    f.zero_old = 0;
    f.relax_f = h->opts.relax == MGRIT_RELAX_F;
    f.value_residual = prec == 0 && !f.relax_f;
    f.df_store = h->dfc;
    if ((st = klaunch(h, MGRIT_K_FCF, "fcf", [&] {
           return launch_ok(launch_fine_fcf(h, f, prec), "fcf");
         })) != MGRIT_OK)
      return st;
    if (f.value_residual && (st = klaunch(h, MGRIT_K_NORM, "residual", [&] {
                               return launch_ok(launch_residual_value(f.c_new, f.r, f.partial, nx, f.N, h->stream),
                                                "residual");
                             })) != MGRIT_OK)
      return st;
    if ((st = klaunch(h, MGRIT_K_NORM, "norm", [&] {
           return launch_ok(launch_norm(h->partial, (int)N1 + f.relax_f, h->scratch + 2 * nx, h->stream), "norm");
         })) != MGRIT_OK)
      return st;
    CUDA_TRY(cudaMemcpyAsync(h->norm_host, h->scratch + 2 * nx, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    const double rel = !std::isfinite(r0) ? r0 : (r0 > 0.0 ? std::sqrt(h->norm_host[0]) / r0 : 0.0);
    if (R.n_history < MGRIT_MAX_HISTORY) R.history[R.n_history++] = rel;
    R.rel_residual = rel;
    if (!std::isfinite(rel) || (rel > 1e6 && !(h->opts.flags & MGRIT_FLAG_NO_DIVERGENCE_STOP))) {
      final_status = fail(MGRIT_ERR_DIVERGED, "residual not finite or grew above 1e6 x initial");
      break;
    }
    if (rel <= h->opts.tol) {
      R.converged = 1;
      break;
    }
    if (it >= h->opts.max_iter) {
      final_status = fail(MGRIT_ERR_NOT_CONVERGED, "max_iter reached");
      break;
    }
    if ((st = coarse_cycle(h, h->c[1 - cur])) != MGRIT_OK) return st;
    cur = 1 - cur;
    ++it;
  }
  R.iterations = it;
  // result: C-points after the final FCF-relaxation live in c[1-cur]
  h->last = 1 - cur;
  h->r0_last = r0;
  if (out && (st = write_output(h, h->c[1 - cur], out)) != MGRIT_OK) return st;
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  R.solve_s = now_s() - t0;
  collect_stats(h, &R);
  R.dof_per_s = R.solve_s > 0 ? (double)nx * h->nt / R.solve_s : 0.0;
  if (res) *res = R;
  return final_status;
}

extern "C" mgrit_status mgrit_solve(mgrit_handle* h, const double* u0, double* out, mgrit_result* res) {
  if (!h) return fail(MGRIT_ERR_INVALID, "handle is NULL");
  if (!u0) return fail(MGRIT_ERR_INVALID, "u0 is NULL");
  return solve_impl(h, u0, nullptr, 0.0, out, res);
}

extern "C" mgrit_status mgrit_solve_from(mgrit_handle* h, const double* c_init, double r0_norm, double* out,
                                         mgrit_result* res) {
  if (!h) return fail(MGRIT_ERR_INVALID, "handle is NULL");
  if (!c_init) return fail(MGRIT_ERR_INVALID, "c_init is NULL");
  if (!std::isfinite(r0_norm)) return fail(MGRIT_ERR_INVALID, "r0_norm must be finite");
  return solve_impl(h, c_init, c_init, r0_norm, out, res);
}

// ----------------------------------------------------------- queued solves

extern "C" mgrit_status mgrit_solve_async(mgrit_handle* h, const double* u0, double* out) {
  if (!h) return fail(MGRIT_ERR_INVALID, "handle is NULL");
  if (!u0) return fail(MGRIT_ERR_INVALID, "u0 is NULL");
  if (out && !is_device_ptr(out)) return fail(MGRIT_ERR_INVALID, "out must be device memory (or NULL)");
  if (h->opts.output == MGRIT_OUT_FULL)
    return fail(MGRIT_ERR_UNSUPPORTED, "mgrit_solve_async writes FINAL or CPOINTS output; use mgrit_solve for FULL");
  if (h->opts.flags & (MGRIT_FLAG_TIME_KERNELS | MGRIT_FLAG_HOST_LOOP))
    return fail(MGRIT_ERR_UNSUPPORTED, "mgrit_solve_async runs the graph solve (no host loop or kernel timing)");
  if (h->ring_count >= MGRIT_MAX_INFLIGHT)
    return fail(MGRIT_ERR_INVALID, "MGRIT_MAX_INFLIGHT solves outstanding: call mgrit_solve_wait first");
  if (!ensure_graph(h)) return fail(MGRIT_ERR_UNSUPPORTED, "the device refused the solve graph");
  if (!h->ring) {
    if (cudaMallocHost(&h->ring, MGRIT_MAX_INFLIGHT * sizeof(CheckState)) != cudaSuccess) {
      h->ring = nullptr;
      return launch_ok(cudaGetLastError(), "pinned result slots");
    }
    for (auto& ev : h->ring_ev) CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  }
  const double t0 = now_s();
  const int nx = h->nx;
  const long long N1 = h->Nl[1];
  mgrit_status st;
  if ((st = load_iterate(h, u0, nullptr)) != MGRIT_OK) return st;
  const double diverge = (h->opts.flags & MGRIT_FLAG_NO_DIVERGENCE_STOP) ? 0.0 : 1e6;
  CUDA_TRY(launch_state_init(h->dstate, h->opts.tol, h->opts.max_iter, diverge, 0.0, h->stream));
  int r0_launches = 0;
  if ((st = enqueue_r0sq(h, &h->dstate->r0sq, &r0_launches)) != MGRIT_OK) return st;
  CUDA_TRY(cudaGraphLaunch(h->gexec, h->stream));
  const int slot = (h->ring_head + h->ring_count) % MGRIT_MAX_INFLIGHT;
  CUDA_TRY(cudaMemcpyAsync(&h->ring[slot], h->dstate, sizeof(CheckState), cudaMemcpyDeviceToHost, h->stream));
  if (out) {
    const bool fin = h->opts.output == MGRIT_OUT_FINAL;
    CUDA_TRY(launch_result_rows(h->dstate, h->c[0], h->c[1], out, nx, fin ? N1 : 0, fin ? 1 : N1 + 1, h->dfc,
                                h->stream));
  }
  CUDA_TRY(cudaEventRecord(h->ring_ev[slot], h->stream));
  h->ring_t0[slot] = t0;
  h->ring_r0_launches[slot] = r0_launches + 1 + (out ? 1 : 0);  // + state init, result rows
  h->ring_count++;
  return MGRIT_OK;
}

extern "C" mgrit_status mgrit_solve_wait(mgrit_handle* h, mgrit_result* res) {
  if (!h) return fail(MGRIT_ERR_INVALID, "handle is NULL");
  if (h->ring_count == 0) return fail(MGRIT_ERR_INVALID, "no mgrit_solve_async outstanding on this handle");
  const int slot = h->ring_head;
  CUDA_TRY(cudaEventSynchronize(h->ring_ev[slot]));
  h->ring_head = (h->ring_head + 1) % MGRIT_MAX_INFLIGHT;
  h->ring_count--;
  const CheckState S = h->ring[slot];
  mgrit_result R;
  std::memset(&R, 0, sizeof(R));
  R.n_levels = h->L;
  R.setup_s = h->setup_s;
  R.op_complexity = h->op_complexity;
  grid_spacings(&h->prob, &R.dx, &R.dt);
  R.r0_norm = std::sqrt(S.r0sq);
  R.iterations = S.it;
  R.rel_residual = S.rel;
  R.n_history = std::min(S.nhist, MGRIT_MAX_HISTORY);
  for (int k = 0; k < R.n_history; ++k) R.history[k] = S.hist[k];
  R.converged = S.status == 0 && S.done ? 1 : 0;
  R.solve_s = now_s() - h->ring_t0[slot];
  R.dof_per_s = R.solve_s > 0 ? (double)h->nx * h->nt / R.solve_s : 0.0;
  reset_stats(h);
  h->kcount[MGRIT_K_FCF] = S.it + 1;
  h->kcount[MGRIT_K_NORM] = (fine_prec(h) == 0 && h->opts.relax == MGRIT_RELAX_FCF ? 2 : 1) * (S.it + 1);
  h->kcount[MGRIT_K_OTHER] = S.it + 1;                       // stopping tests
  h->kcount[MGRIT_K_PROPAGATE] = h->ring_r0_launches[slot];  // initial residual, state, output
  collect_stats(h, &R);
  R.launches += R.iterations * h->graph_coarse_launches;
  R.graph = 1;
  h->last = 1 - S.result_cur;
  h->r0_last = R.r0_norm;
  if (res) *res = R;
  if (!S.done) return fail(MGRIT_ERR_CUDA, "graph ended without a stopping decision");
  if (S.status == -5) return fail(MGRIT_ERR_DIVERGED, "residual not finite or grew above 1e6 x initial");
  if (S.status == -4) return fail(MGRIT_ERR_NOT_CONVERGED, "max_iter reached");
  return MGRIT_OK;
}

extern "C" mgrit_status mgrit_relax(mgrit_handle* h, int32_t sweeps, double* rel_residual) {
  if (!h) return fail(MGRIT_ERR_INVALID, "handle is NULL");
  if (h->last < 0) return fail(MGRIT_ERR_INVALID, "no iterate yet: call mgrit_solve first");
  if (sweeps < 0) return fail(MGRIT_ERR_INVALID, "sweeps must be >= 0");
  const int nx = h->nx;
  const int prec = fine_prec(h);
  reset_stats(h);
  mgrit_status st;
  FcfArgs f = {};
  f.cstride = nx;
  f.r = h->r[1];
  f.r_f = h->rf[1];
  f.partial = h->partial;
  f.nx = nx;
  f.m = h->m;
  f.N = h->Nl[1];
  f.relax_f = h->opts.relax == MGRIT_RELAX_F;
  f.value_residual = prec == 0 && !f.relax_f;
  f.df_store = h->dfc;
  // C-point 0 (the initial condition) of the other buffer: no sweep writes it,
  // and an output of float-float C-points is converted through that buffer
  if (sweeps > 0)
    CUDA_TRY(cudaMemcpyAsync(h->c[1 - h->last], h->c[h->last], (size_t)nx * sizeof(double), cudaMemcpyDeviceToDevice,
                             h->stream));
  for (int k = 0; k < sweeps; ++k) {  // back to back on the stream: no host synchronisation between sweeps
    f.u_old = h->c[h->last];
    f.c_new = h->c[1 - h->last];
    if ((st = klaunch(h, MGRIT_K_FCF, "fcf", [&] { return launch_ok(launch_fine_fcf(h, f, prec), "fcf"); })) !=
        MGRIT_OK)
      return st;
    if (f.value_residual && (st = klaunch(h, MGRIT_K_NORM, "residual", [&] {
                               return launch_ok(launch_residual_value(f.c_new, f.r, f.partial, nx, f.N, h->stream),
                                                "residual");
                             })) != MGRIT_OK)
      return st;
    h->last = 1 - h->last;
  }
  if ((st = klaunch(h, MGRIT_K_NORM, "norm", [&] {
         return launch_ok(launch_norm(h->partial, f.N + f.relax_f, h->scratch + 2 * nx, h->stream), "norm");
       })) != MGRIT_OK)
    return st;
  CUDA_TRY(cudaMemcpyAsync(h->norm_host, h->scratch + 2 * nx, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  if (rel_residual) *rel_residual = h->r0_last > 0.0 ? std::sqrt(h->norm_host[0]) / h->r0_last : 0.0;
  return MGRIT_OK;
}

extern "C" mgrit_status mgrit_sequential(mgrit_handle* h, const double* u0, double* out, double* seconds) {
  if (!h) return fail(MGRIT_ERR_INVALID, "handle is NULL");
  if (!u0) return fail(MGRIT_ERR_INVALID, "u0 is NULL");
  const double t0 = now_s();
  const int nx = h->nx;
  const size_t slab = (size_t)nx * sizeof(double);
  const int every = h->opts.output == MGRIT_OUT_FULL ? 1 : (h->opts.output == MGRIT_OUT_CPOINTS ? h->m : h->nt);
  const size_t nstore = (size_t)h->nt / every + 1;
  double* dst = nullptr;
  mgrit_status st;
  const bool final_only = h->opts.output == MGRIT_OUT_FINAL;
  const bool dev = out && is_device_ptr(out) && !final_only;
  bool temp = false;
  if (dev) dst = out;
  else {
    if ((st = dalloc(h, nstore * nx, &dst)) != MGRIT_OK) return st;
    temp = true;
  }
  double* init = h->scratch;
  CUDA_TRY(cudaMemcpyAsync(init, u0, slab, kind_to_dev(u0), h->stream));
  CUDA_TRY(cudaMemcpyAsync(dst, init, slab, cudaMemcpyDeviceToDevice, h->stream));
  MarchArgs a = {};
  a.init = init;
  a.u_out = dst;
  a.store_every = every;
  a.nx = nx;
  a.P = h->nt + 1;
  reset_stats(h);
  if (h->sdirk) {
    st = klaunch(h, MGRIT_K_MARCH, "seq", [&] {
      return launch_ok(launch_seq_sdirk(init, dst, nx, h->nt + 1, every, h->splan, h->stream), "seq_sdirk");
    });
  } else if (h->inflow) {  // Phi's boundary rows: one CTA keeps the slab and fixes them up every step
    st = klaunch(h, MGRIT_K_MARCH, "seq", [&] {
      return launch_ok(launch_seq_slab(init, dst, nx, h->nt + 1, every, h->dphi, h->fx_phi, 0, h->stream),
                       "seq_slab");
    });
  } else {
    int saved = h->march_cluster;
    h->march_cluster = pick_cluster(nx, h->phi);
    st = run_march(h, a, h->dphi);
    h->march_cluster = saved;
  }
  if (st != MGRIT_OK) return st;
  if (out && !dev) {
    if (final_only)
      CUDA_TRY(cudaMemcpyAsync(out, dst + (nstore - 1) * nx, slab, kind_from_dev(out), h->stream));
    else
      CUDA_TRY(cudaMemcpyAsync(out, dst, nstore * slab, cudaMemcpyDeviceToHost, h->stream));
  }
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  if (temp) {
    DevBuf b = h->bufs.back();
    h->bufs.pop_back();
    h->bytes -= std::max<size_t>(b.n, 1) * sizeof(double);
    if (b.freefn) b.freefn(b.p, (void*)h->stream, b.ctx);
    else cudaFreeAsync(b.p, h->stream);
    CUDA_TRY(cudaStreamSynchronize(h->stream));
  }
  if (seconds) *seconds = now_s() - t0;
  return MGRIT_OK;
}

extern "C" mgrit_status mgrit_propagate(mgrit_handle* h, int32_t level, int32_t k, int32_t count, const double* in,
                                        double* out) {
  if (!h) return fail(MGRIT_ERR_INVALID, "handle is NULL");
  if (level < 1 || level > h->L) return fail(MGRIT_ERR_INVALID, "level must be 1..levels");
  if (k < 0 || count < 0 || !in || !out) return fail(MGRIT_ERR_INVALID, "bad arguments");
  const DevTaps& t = level == 1 ? h->dphi : h->dpsi[level - 2];
  reset_stats(h);
  mgrit_status st = klaunch(h, MGRIT_K_PROPAGATE, "propagate", [&] {
    if (level == 1 && h->sdirk)
      return launch_ok(launch_propagate_sdirk(in, out, count, h->nx, k, h->splan, nullptr, h->stream), "propagate");
    if (level == 2 && h->redisc)
      return launch_ok(launch_propagate_sdirk(in, out, count, h->nx, k, h->cplan, nullptr, h->stream), "propagate");
    if (level == 1)
      return launch_ok(launch_propagate(in, out, count, h->nx, k, t, nullptr, h->fcf_threads, h->stream, &h->fx_phi),
                       "propagate");
    return launch_ok(
        launch_propagate(in, out, count, h->nx, k, t, nullptr, h->fcf_threads, h->stream, nullptr, h->inflow),
        "propagate");
  });
  if (st != MGRIT_OK) return st;
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  return MGRIT_OK;
}
