// SDIRK fine steps (sm_103a): stage form of Appendix A's L-stable tableaux with
// the implicit stage matrix M = I - gamma dt L solved exactly.
//
// Solve M K = y (M circulant, banded by U_p).  On the host M is written as
//   M = E^{-ql} p_d prod_r (E - z_r),   E the forward shift,
// and each root is turned into a factor in its stable direction:
//   |z| < 1:  (E - z) = E (I - z E^{-1})     x_i = z x_{i-1} + y_i  (forward)
//   |z| > 1:  (E - z) = -z (I - z^{-1} E)     x_i = z^{-1} x_{i+1} + y_i  (backward)
// A complex-conjugate pair acting on real data needs one complex recurrence:
//   (I - zS)^{-1}(I - conj(z) S)^{-1} y = Im(z F) / Im(z),  F = (I - zS)^{-1} y.
// The leftover shift E^{ql - n_forward} and scale 1/(p_d prod_b(-z)) are
// applied at load/store.
//
// Each first-order periodic recurrence runs as a chunked parallel scan: every
// thread owns C consecutive points in registers, scans them with zero carry,
// the chunk-end values are combined by a warp-shuffle scan and a cross-warp
// scan (multiplier A = m^C per chunk), the periodic wrap is closed exactly
// (x_{-1} = total / (1 - m^n), a rank-one correction), and each thread adds
// m^{c+1} times its carry-in.  Powers of A come from per-CTA tables.
#include <cuda_runtime.h>

#include "device.h"

namespace mg {

namespace {

template <typename T>
struct cx {
  T re, im;
};

template <typename T>
__device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b) {
  return {fma(a.re, b.re, -a.im * b.im), fma(a.re, b.im, a.im * b.re)};
}
template <typename T>
__device__ __forceinline__ cx<T> cfma(cx<T> a, cx<T> b, cx<T> c) {
  return {fma(a.re, b.re, fma(-a.im, b.im, c.re)), fma(a.re, b.im, fma(a.im, b.re, c.im))};
}
template <typename T>
__device__ __forceinline__ cx<T> cadd(cx<T> a, cx<T> b) {
  return {a.re + b.re, a.im + b.im};
}

// Uniform interface for real and complex scan values.
template <typename T>
struct RealOps {
  using V = T;
  static __device__ __forceinline__ V zero() { return (T)0; }
  static __device__ __forceinline__ V fmav(V a, V b, V c) { return fma(a, b, c); }
  static __device__ __forceinline__ V mul(V a, V b) { return a * b; }
  static __device__ __forceinline__ V from(cx<double> a) { return (T)a.re; }
  static __device__ __forceinline__ V shfl_up(V v, int d) { return __shfl_up_sync(0xffffffffu, v, d); }
  static __device__ __forceinline__ V shfl_down(V v, int d) { return __shfl_down_sync(0xffffffffu, v, d); }
  static __device__ __forceinline__ V div_one_minus(V a, V b) { return a / ((T)1 - b); }
};
template <typename T>
struct CplxOps {
  using V = cx<T>;
  static __device__ __forceinline__ V zero() { return {(T)0, (T)0}; }
  static __device__ __forceinline__ V fmav(V a, V b, V c) { return cfma(a, b, c); }
  static __device__ __forceinline__ V mul(V a, V b) { return cmul(a, b); }
  static __device__ __forceinline__ V from(cx<double> a) { return {(T)a.re, (T)a.im}; }
  static __device__ __forceinline__ V shfl_up(V v, int d) {
    return {__shfl_up_sync(0xffffffffu, v.re, d), __shfl_up_sync(0xffffffffu, v.im, d)};
  }
  static __device__ __forceinline__ V shfl_down(V v, int d) {
    return {__shfl_down_sync(0xffffffffu, v.re, d), __shfl_down_sync(0xffffffffu, v.im, d)};
  }
  static __device__ __forceinline__ V div_one_minus(V a, V b) {
    const T dr = (T)1 - b.re, di = -b.im, den = dr * dr + di * di;
    return {(a.re * dr + a.im * di) / den, (a.im * dr - a.re * di) / den};
  }
};

constexpr int kCMax = 16;        // points per thread
constexpr int kLanePow = 33;     // A^0..A^32
constexpr int kWarpPow = 17;     // (A^32)^0..(A^32)^16
struct FactorTables {
  cx<double> lanep[kMaxFactors][kLanePow];
  cx<double> warpp[kMaxFactors][kWarpPow];
};

__host__ __device__ constexpr size_t tables_bytes() { return (sizeof(FactorTables) + 255) / 256 * 256; }

__device__ __forceinline__ int wrapn(int k, int nx) {
  k = (k < 0) ? k + nx : k;
  return (k >= nx) ? k - nx : k;
}
__device__ __forceinline__ int pix(int e) { return e + (e >> 3); }

__device__ cx<double> cpow(cx<double> a, int k) {
  cx<double> r = {1.0, 0.0};
  while (k > 0) {
    if (k & 1) r = cmul(r, a);
    a = cmul(a, a);
    k >>= 1;
  }
  return r;
}

// Per-CTA tables of A^k and (A^32)^k, A = m^C, for every factor.
__device__ void build_tables(const SdirkPlan& p, int C, FactorTables* tb) {
  for (int f = 0; f < p.nf; ++f) {
    const cx<double> m = {p.mre[f], p.mim[f]};
    const cx<double> A = cpow(m, C);
    const cx<double> A32 = cpow(A, 32);
    for (int k = threadIdx.x; k < kLanePow; k += blockDim.x) tb->lanep[f][k] = cpow(A, k);
    for (int k = threadIdx.x; k < kWarpPow; k += blockDim.x) tb->warpp[f][k] = cpow(A32, k);
  }
}

// Periodic first-order recurrence over the whole slab, data in registers:
// forward x_i = m x_{i-1} + y_i, backward x_i = m x_{i+1} + y_i.
template <class Ops, int C>
__device__ __forceinline__ void rec_scan(typename Ops::V (&x)[C], const typename Ops::V m,
                                         const cx<double>* lanep, const cx<double>* warpp, const bool backward,
                                         typename Ops::V* smw) {
  using V = typename Ops::V;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  V X;
  if (!backward) {
    V prev = Ops::zero();
#pragma unroll
    for (int c = 0; c < C; ++c) { x[c] = Ops::fmav(m, prev, x[c]); prev = x[c]; }
    X = prev;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const V Y = Ops::shfl_up(X, d);
      if (lane >= d) X = Ops::fmav(Ops::from(lanep[d]), Y, X);
    }
    if (lane == 31) smw[warp] = X;
    __syncthreads();
    if (warp == 0) {
      V W = lane < nw ? smw[lane] : Ops::zero();
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const V Y = Ops::shfl_up(W, d);
        if (lane >= d && d < kWarpPow) W = Ops::fmav(Ops::from(warpp[d]), Y, W);
      }
      if (lane < nw) smw[lane] = W;
    }
    __syncthreads();
    const V P = warp > 0 ? smw[warp - 1] : Ops::zero();
    const V X0 = Ops::fmav(Ops::from(lanep[lane + 1]), P, X);
    const V xm1 = Ops::div_one_minus(smw[nw - 1], Ops::from(warpp[nw]));
    V prevX0 = Ops::shfl_up(X0, 1);
    if (lane == 0) prevX0 = P;
    const V At = Ops::mul(Ops::from(lanep[lane]), Ops::from(warpp[warp]));
    const V cin = Ops::fmav(At, xm1, prevX0);
    V mp = m;
#pragma unroll
    for (int c = 0; c < C; ++c) { x[c] = Ops::fmav(mp, cin, x[c]); mp = Ops::mul(mp, m); }
  } else {
    V next = Ops::zero();
#pragma unroll
    for (int c = C - 1; c >= 0; --c) { x[c] = Ops::fmav(m, next, x[c]); next = x[c]; }
    X = next;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const V Y = Ops::shfl_down(X, d);
      if (lane + d < 32) X = Ops::fmav(Ops::from(lanep[d]), Y, X);
    }
    if (lane == 0) smw[warp] = X;
    __syncthreads();
    if (warp == 0) {
      V W = lane < nw ? smw[nw - 1 - lane] : Ops::zero();
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const V Y = Ops::shfl_up(W, d);
        if (lane >= d && d < kWarpPow) W = Ops::fmav(Ops::from(warpp[d]), Y, W);
      }
      __syncwarp();
      if (lane < nw) smw[nw - 1 - lane] = W;
    }
    __syncthreads();
    const V Sx = warp < nw - 1 ? smw[warp + 1] : Ops::zero();
    const V X0 = Ops::fmav(Ops::from(lanep[32 - lane]), Sx, X);
    const V x0 = Ops::div_one_minus(smw[0], Ops::from(warpp[nw]));
    V nextX0 = Ops::shfl_down(X0, 1);
    if (lane == 31) nextX0 = Sx;
    const V Ar = Ops::mul(Ops::from(lanep[31 - lane]), Ops::from(warpp[nw - 1 - warp]));
    const V cin = Ops::fmav(Ar, x0, nextX0);
    V mp = m;
#pragma unroll
    for (int c = C - 1; c >= 0; --c) { x[c] = Ops::fmav(mp, cin, x[c]); mp = Ops::mul(mp, m); }
  }
  __syncthreads();  // smw is reused by the next scan
}

// K <- M^{-1} K in place (shared slab, padded layout); C points per thread.
template <typename T, int C>
__device__ void stage_solve(const SdirkPlan& p, T* K, int nx, const FactorTables* tb, void* smw_raw) {
  const int base = threadIdx.x * C;
  T x[C];
#pragma unroll
  for (int c = 0; c < C; ++c) x[c] = K[pix(wrapn(base + c + p.ql, nx))];
  __syncthreads();
  for (int f = 0; f < p.nf; ++f) {
    const bool back = p.dir[f] < 0;
    if (p.mim[f] == 0.0) {
      rec_scan<RealOps<T>, C>(x, (T)p.mre[f], tb->lanep[f], tb->warpp[f], back, reinterpret_cast<T*>(smw_raw));
    } else {
      cx<T> z[C];
#pragma unroll
      for (int c = 0; c < C; ++c) z[c] = {x[c], (T)0};
      const cx<T> m = {(T)p.mre[f], (T)p.mim[f]};
      rec_scan<CplxOps<T>, C>(z, m, tb->lanep[f], tb->warpp[f], back, reinterpret_cast<cx<T>*>(smw_raw));
      const T inv_im = (T)(1.0 / p.mim[f]);
#pragma unroll
      for (int c = 0; c < C; ++c) x[c] = fma(m.re, z[c].im, m.im * z[c].re) * inv_im;  // Im(m z) / Im(m)
    }
  }
  const T sc = (T)p.inv_pd;
#pragma unroll
  for (int c = 0; c < C; ++c) K[pix(base + c)] = x[c] * sc;
  __syncthreads();
}

template <typename T>
__device__ __forceinline__ T aij(const SdirkPlan& p, int i, int j);
template <>
__device__ __forceinline__ double aij<double>(const SdirkPlan& p, int i, int j) { return p.a[i][j]; }
template <>
__device__ __forceinline__ float aij<float>(const SdirkPlan& p, int i, int j) { return p.a32[i][j]; }
template <typename T>
__device__ __forceinline__ T cl(const SdirkPlan& p, int k);
template <>
__device__ __forceinline__ double cl<double>(const SdirkPlan& p, int k) { return p.cL[k]; }
template <>
__device__ __forceinline__ float cl<float>(const SdirkPlan& p, int k) { return p.cL32[k]; }

// dst = dt L src
template <typename T>
__device__ __forceinline__ void apply_L(const SdirkPlan& p, const T* src, T* dst, int nx) {
  for (int i = threadIdx.x; i < nx; i += blockDim.x) {
    T acc = (T)0;
    for (int k = 0; k < p.nL; ++k) acc = fma(cl<T>(p, k), src[pix(wrapn(i + p.offL[k], nx))], acc);
    dst[pix(i)] = acc;
  }
}

// u <- Phi u, u in slot[0]; slots 1.. are work space (sdirk_slots(p) in total).
template <typename T, int C>
__device__ void sdirk_step(const SdirkPlan& p, T* slab, int plen, int nx, const FactorTables* tb, void* smw) {
  const int s = p.s;
  T* X = slab;
  T* K = slab + plen;
  // stage 1: K_1 = M^{-1} dtL u
  apply_L<T>(p, X, K, nx);
  __syncthreads();
  stage_solve<T, C>(p, K, nx, tb, smw);
  if (s == 1) {
    for (int i = threadIdx.x; i < nx; i += blockDim.x) X[pix(i)] += K[pix(i)];  // b_1 = 1
    __syncthreads();
    return;
  }
  // accumulators A_l = u + a_l1 K_1: A_3..A_s in extra slots, A_2 in place of u
  for (int i = threadIdx.x; i < nx; i += blockDim.x) {
    const T u = X[pix(i)], k1 = K[pix(i)];
    for (int l = 3; l <= s; ++l) slab[(l - 1) * plen + pix(i)] = fma(aij<T>(p, l - 1, 0), k1, u);
    X[pix(i)] = fma(aij<T>(p, 1, 0), k1, u);
  }
  __syncthreads();
  for (int st = 2; st <= s; ++st) {
    T* Ai = (st == 2) ? X : slab + (st - 1) * plen;
    apply_L<T>(p, Ai, K, nx);
    __syncthreads();
    stage_solve<T, C>(p, K, nx, tb, smw);
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
      const T k = K[pix(i)];
      for (int l = st + 1; l <= s; ++l) {
        T* Al = slab + (l - 1) * plen;
        Al[pix(i)] = fma(aij<T>(p, l - 1, st - 1), k, Al[pix(i)]);
      }
      if (st == s) X[pix(i)] = fma(aij<T>(p, s - 1, s - 1), k, Ai[pix(i)]);  // u_new = A_s + gamma K_s
    }
    __syncthreads();
  }
}

}  // namespace

int sdirk_slots(const SdirkPlan& p) { return p.s <= 2 ? 2 : p.s; }

// CTA size for nx: nx = threads * C with C in {1, 2, 4, 8, 16}, threads a
// multiple of 32 and at most 512 (0 if no such split exists).
int sdirk_threads(int nx) {
  for (int C = 1; C <= kCMax; C <<= 1)
    if (nx % C == 0 && nx / C <= 512 && (nx / C) % 32 == 0) return nx / C;
  return 0;
}

size_t sdirk_smem(const SdirkPlan& p, int nx, int prec) {
  (void)prec;
  return tables_bytes() + (size_t)sdirk_slots(p) * padded_len(nx) * sizeof(double);
}

// ------------------------------------------------------------------ kernels

__device__ __forceinline__ double block_sum_sd(double ss) {
  __shared__ double ws[32];
  for (int o = 16; o; o >>= 1) ss += __shfl_down_sync(0xffffffffu, ss, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) ws[wid] = ss;
  __syncthreads();
  if (wid == 0) {
    ss = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0.0;
    for (int o = 16; o; o >>= 1) ss += __shfl_down_sync(0xffffffffu, ss, o);
  }
  return ss;
}

template <int PREC, int C>
__global__ void __launch_bounds__(512) fcf_sdirk_kernel(const FcfArgs a, const SdirkPlan p) {
  extern __shared__ __align__(256) unsigned char smraw[];
  __shared__ __align__(16) double smw[64];
  FactorTables* tb = reinterpret_cast<FactorTables*>(smraw);
  double* slab = reinterpret_cast<double*>(smraw + tables_bytes());
  const int nx = a.nx, m = a.m, plen = padded_len(nx), j = blockIdx.x + 1;
  build_tables(p, C, tb);
  const double* start = a.u_old + (long long)(j - 1) * a.cstride;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) slab[pix(i)] = a.zero_old ? 0.0 : start[i];
  __syncthreads();
  for (int s = 0; s < m; ++s) sdirk_step<double, C>(p, slab, plen, nx, tb, smw);
  const double* oldj = a.u_old + (long long)j * a.cstride;
  double* cn = a.c_new + (long long)j * nx;
  const bool more = j < a.N;
  double ss = 0.0;
  if (PREC == 0) {
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
      const double v = slab[pix(i)];
      cn[i] = v;
      slab[pix(i)] = v - (a.zero_old ? 0.0 : oldj[i]);
    }
    __syncthreads();
    if (!more) return;
    for (int s = 0; s < m; ++s) sdirk_step<double, C>(p, slab, plen, nx, tb, smw);
    double* rr = a.r + (long long)(j + 1) * nx;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
      const double v = slab[pix(i)];
      rr[i] = v;
      ss = fma(v, v, ss);
    }
  } else {
    // each thread owns points i = tid + k*blockDim (k < C): read all FP64
    // values before the FP32 slab (same storage) is written
    float* fs = reinterpret_cast<float*>(slab);
    double vals[C];
#pragma unroll
    for (int k = 0; k < C; ++k) vals[k] = slab[pix(threadIdx.x + k * blockDim.x)];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < C; ++k) {
      const int i = threadIdx.x + k * blockDim.x;
      cn[i] = vals[k];
      fs[pix(i)] = (float)(vals[k] - (a.zero_old ? 0.0 : oldj[i]));
    }
    __syncthreads();
    if (!more) return;
    for (int s = 0; s < m; ++s) sdirk_step<float, C>(p, fs, plen, nx, tb, smw);
    double* rr = a.r + (long long)(j + 1) * nx;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
      const double v = (double)fs[pix(i)];
      rr[i] = v;
      ss = fma(v, v, ss);
    }
  }
  if (a.partial) {
    ss = block_sum_sd(ss);
    if (threadIdx.x == 0) a.partial[j] = ss;
  }
}

template <int C>
__global__ void __launch_bounds__(512) propagate_sdirk_kernel(const double* in, double* out, int nx, int k,
                                                              const SdirkPlan p, double* partial) {
  extern __shared__ __align__(256) unsigned char smraw[];
  __shared__ __align__(16) double smw[64];
  FactorTables* tb = reinterpret_cast<FactorTables*>(smraw);
  double* slab = reinterpret_cast<double*>(smraw + tables_bytes());
  const int plen = padded_len(nx);
  const long long v = blockIdx.x;
  build_tables(p, C, tb);
  for (int i = threadIdx.x; i < nx; i += blockDim.x) slab[pix(i)] = in[v * nx + i];
  __syncthreads();
  for (int s = 0; s < k; ++s) sdirk_step<double, C>(p, slab, plen, nx, tb, smw);
  double ss = 0.0;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) {
    const double x = slab[pix(i)];
    out[v * nx + i] = x;
    ss = fma(x, x, ss);
  }
  if (partial) {
    ss = block_sum_sd(ss);
    if (threadIdx.x == 0) partial[v] = ss;
  }
}

// F-points of the fine level from its C-points (ideal interpolation output).
template <int C>
__global__ void __launch_bounds__(512) interp_sdirk_kernel(const double* c, double* u, int nx, int m, int N,
                                                           const SdirkPlan p) {
  extern __shared__ __align__(256) unsigned char smraw[];
  __shared__ __align__(16) double smw[64];
  FactorTables* tb = reinterpret_cast<FactorTables*>(smraw);
  double* slab = reinterpret_cast<double*>(smraw + tables_bytes());
  const int plen = padded_len(nx), j = blockIdx.x + 1;
  build_tables(p, C, tb);
  const long long p0 = (long long)(j - 1) * m;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) {
    const double v = c[(long long)(j - 1) * nx + i];
    slab[pix(i)] = v;
    u[p0 * nx + i] = v;
  }
  __syncthreads();
  for (int s = 1; s < m; ++s) {
    sdirk_step<double, C>(p, slab, plen, nx, tb, smw);
    for (int i = threadIdx.x; i < nx; i += blockDim.x) u[(p0 + s) * nx + i] = slab[pix(i)];
  }
  if (j == N)
    for (int i = threadIdx.x; i < nx; i += blockDim.x) u[(long long)N * m * nx + i] = c[(long long)N * nx + i];
}

// Plain sequential stepping on one CTA (store every store_every-th level).
template <int C>
__global__ void __launch_bounds__(512) seq_sdirk_kernel(const double* u0, double* out, int nx, int P,
                                                        int store_every, const SdirkPlan p) {
  extern __shared__ __align__(256) unsigned char smraw[];
  __shared__ __align__(16) double smw[64];
  FactorTables* tb = reinterpret_cast<FactorTables*>(smraw);
  double* slab = reinterpret_cast<double*>(smraw + tables_bytes());
  const int plen = padded_len(nx);
  build_tables(p, C, tb);
  for (int i = threadIdx.x; i < nx; i += blockDim.x) slab[pix(i)] = u0[i];
  __syncthreads();
  for (int n = 1; n < P; ++n) {
    sdirk_step<double, C>(p, slab, plen, nx, tb, smw);
    if (n % store_every == 0)
      for (int i = threadIdx.x; i < nx; i += blockDim.x) out[(long long)(n / store_every) * nx + i] = slab[pix(i)];
  }
}

template <typename K>
static cudaError_t smem_attr(K kernel, size_t bytes) {
  if (bytes > 48 * 1024) return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  return cudaSuccess;
}

// Call f.template operator()<C>() with the compile-time chunk length of nx.
template <typename F>
static cudaError_t with_chunk(int nx, F&& f) {
  const int th = sdirk_threads(nx);
  if (!th) return cudaErrorInvalidValue;
  switch (nx / th) {
    case 1: return f.template operator()<1>(th);
    case 2: return f.template operator()<2>(th);
    case 4: return f.template operator()<4>(th);
    case 8: return f.template operator()<8>(th);
    case 16: return f.template operator()<16>(th);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_fcf_sdirk(const FcfArgs& a, const SdirkPlan& p, int precision, cudaStream_t s) {
  if (a.N < 1) return cudaSuccess;
  const size_t smem = sdirk_smem(p, a.nx, precision);
  return with_chunk(a.nx, [&]<int C>(int th) -> cudaError_t {
    cudaError_t e;
    if (precision == 0) {
      if ((e = smem_attr(fcf_sdirk_kernel<0, C>, smem)) != cudaSuccess) return e;
      fcf_sdirk_kernel<0, C><<<a.N, th, smem, s>>>(a, p);
    } else {
      if ((e = smem_attr(fcf_sdirk_kernel<1, C>, smem)) != cudaSuccess) return e;
      fcf_sdirk_kernel<1, C><<<a.N, th, smem, s>>>(a, p);
    }
    return cudaGetLastError();
  });
}

cudaError_t launch_propagate_sdirk(const double* in, double* out, int count, int nx, int k, const SdirkPlan& p,
                                   double* partial, cudaStream_t s) {
  if (count < 1) return cudaSuccess;
  const size_t smem = sdirk_smem(p, nx, 0);
  return with_chunk(nx, [&]<int C>(int th) -> cudaError_t {
    cudaError_t e = smem_attr(propagate_sdirk_kernel<C>, smem);
    if (e != cudaSuccess) return e;
    propagate_sdirk_kernel<C><<<count, th, smem, s>>>(in, out, nx, k, p, partial);
    return cudaGetLastError();
  });
}

cudaError_t launch_interp_sdirk(const double* c, double* u, int nx, int m, int N, const SdirkPlan& p,
                                cudaStream_t s) {
  if (N < 1) return cudaSuccess;
  const size_t smem = sdirk_smem(p, nx, 0);
  return with_chunk(nx, [&]<int C>(int th) -> cudaError_t {
    cudaError_t e = smem_attr(interp_sdirk_kernel<C>, smem);
    if (e != cudaSuccess) return e;
    interp_sdirk_kernel<C><<<N, th, smem, s>>>(c, u, nx, m, N, p);
    return cudaGetLastError();
  });
}

cudaError_t launch_seq_sdirk(const double* u0, double* out, int nx, int P, int store_every, const SdirkPlan& p,
                             cudaStream_t s) {
  if (P < 2) return cudaSuccess;
  const size_t smem = sdirk_smem(p, nx, 0);
  return with_chunk(nx, [&]<int C>(int th) -> cudaError_t {
    cudaError_t e = smem_attr(seq_sdirk_kernel<C>, smem);
    if (e != cudaSuccess) return e;
    seq_sdirk_kernel<C><<<1, th, smem, s>>>(u0, out, nx, P, store_every, p);
    return cudaGetLastError();
  });
}

}  // namespace mg
