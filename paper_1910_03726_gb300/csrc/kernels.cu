// CUDA kernels (sm_103a) of the MGRIT hot path for periodic advection:
//   fcf_kernel / fcf_batched_kernel   FCF-relaxation + fused C-point residual
//                                     (Section 2.2), one CTA per coarse interval
//   march_kernel / march_batched_kernel  sequential march u_n = T u_{n-1} + g_n on
//                                     a thread-block cluster (coarse solve, Eq. 5;
//                                     sequential stepping, Eq. 3)
//   correct_kernel                    correction + F-relaxation (ideal interpolation)
//   norm_kernel / norm_batched_kernel deterministic residual 2-norm (stopping test)
//   propagate_kernel                  T^k applied to a batch of vectors
//   seq_slab_kernel                   sequential stepping of a non-periodic level
// Every stencil is a circulant (Corollary 1): periodic indices wrap modulo nx.
// On the inflow/outflow domain (Section 4.5) the rows of Phi that reach past
// either end are recomputed after each step from their own coefficients
// (Fixup); Psi is truncated at both ends (Toeplitz): its taps read zero
// outside the domain (TR).
#include <cooperative_groups.h>

#include <cstring>
#include <type_traits>

#include "device.h"

namespace cg = cooperative_groups;

namespace mg {

bool make_dev_taps(const int* off, const double* coef, int n, DevTaps* d) {
  if (n < 1 || n > kMaxDevTaps) return false;
  std::memset(d, 0, sizeof(*d));
  d->n = n;
  int lo = off[0], hi = off[0];
  for (int k = 0; k < n; ++k) {
    d->off[k] = off[k];
    d->c64[k] = coef[k];
    d->c32[k] = (float)coef[k];
    lo = off[k] < lo ? off[k] : lo;
    hi = off[k] > hi ? off[k] : hi;
  }
  d->lo = lo;
  d->hi = hi;
  d->one = 1.0f;
  d->span = hi - lo + 1 <= kMaxSpan ? hi - lo + 1 : 0;
  if (d->span)
    for (int k = 0; k < n; ++k) d->d64[off[k] - lo] += coef[k];
  for (int k = 0; k < d->span; ++k) d->d32[k] = (float)d->d64[k];
  for (int k = 0; k < n; ++k) {
    d->chi[k] = (float)coef[k];
    d->clo[k] = (float)(coef[k] - (double)d->chi[k]);
  }
  for (int k = 0; k < d->span; ++k) {
    d->dhi[k] = (float)d->d64[k];
    d->dlo[k] = (float)(d->d64[k] - (double)d->dhi[k]);
  }
  // frame shift for the march: centre of the offsets (floor)
  d->shift = (lo + hi) >= 0 ? (lo + hi) / 2 : -((-(lo + hi) + 1) / 2);
  return true;
}

__device__ __forceinline__ int wrapi(int k, int nx) {
  k = (k < 0) ? k + nx : k;
  return (k >= nx) ? k - nx : k;
}

// Padded shared-memory index: one pad element after every 8, so that threads
// owning consecutive chunks of 8 elements hit distinct banks.
__device__ __forceinline__ int pidx(int e) { return e + (e >> 3); }

// Float-float value: hi + lo with |lo| <= ulp(hi)/2 (about 48 significant
// bits), evaluated on the FP32 pipes.
struct __align__(8) df64 {
  float hi, lo;
};

// acc + c * x, c and x float-float: exact hi*hi product (TwoProd by FMA), the
// cross terms into the low word, TwoSum on the high words.  Half of the
// additions run as fma(a, one, b) (one = 1.0f from the kernel parameters, so
// it is not folded): the same rounding as a + b, issued to the FMA pipe to
// balance it against the add pipe.
__device__ __forceinline__ df64 df_fma1(df64 c, df64 x, df64 acc, float one) {
  const float p = c.hi * x.hi;
  float e = fmaf(c.hi, x.hi, -p);
  e = fmaf(c.hi, x.lo, e);
  e = fmaf(c.lo, x.hi, e);
  const float s = fmaf(p, one, acc.hi);
  const float bb = fmaf(acc.hi, -one, s);
  const float err = (acc.hi - (s - bb)) + (p - bb);
  return {s, fmaf(fmaf(err, one, e), one, acc.lo)};
}
__device__ __forceinline__ df64 df_fma(df64 c, df64 x, df64 acc) { return df_fma1(c, x, acc, 1.0f); }
// c * x as an unnormalised pair: the exact product of the high words and
// the cross terms (the first tap of a sum, which needs no TwoSum).
__device__ __forceinline__ df64 df_mul(df64 c, df64 x) {
  const float p = c.hi * x.hi;
  float e = fmaf(c.hi, x.hi, -p);
  e = fmaf(c.hi, x.lo, e);
  return {p, fmaf(c.lo, x.hi, e)};
}
__device__ __forceinline__ df64 df_norm(df64 a) {
  const float s = a.hi + a.lo;
  return {s, a.lo - (s - a.hi)};
}
__device__ __forceinline__ df64 df_from(double v) {
  const float h = (float)v;
  return {h, (float)(v - (double)h)};
}
__device__ __forceinline__ double df_to(df64 a) { return (double)a.hi + (double)a.lo; }
// a - b in FP32 (the C-point residual rho, which only the FP32 second pass
// reads): (a.hi - b.hi) + (a.lo - b.lo).  Where the high words are within a
// factor of two of each other -- rho small against the C-points, as it is
// once the iteration has started converging -- their difference is exact
// (Sterbenz) and rho carries FP32 rounding once; elsewhere rho is large and
// two FP32 roundings of it are what the FP32 pass needs.  Three instructions
// instead of a TwoSum's eight.
__device__ __forceinline__ float df_sub_f(df64 a, df64 b) { return (a.hi - b.hi) + (a.lo - b.lo); }
// a + e (e FP32), normalised: TwoSum of the high words, low words added.
__device__ __forceinline__ df64 df_add_f(df64 a, float e) {
  const float s = a.hi + e;
  const float bb = s - a.hi;
  const float err = (a.hi - (s - bb)) + (e - bb);
  return df_norm({s, err + a.lo});
}

// binary32 -> binary64 (exact) from the IEEE 754 bit fields with integer
// instructions: sign as is, exponent rebiased by 1023 - 127, the 23-bit
// fraction moved to the top of the 52-bit one.  GB300 issues the conversion
// instruction on its FP64 pipe, which an FP64 add right after already needs.
// Zeros map directly; subnormal, infinite and NaN inputs (exponent field 0
// with a nonzero fraction, or 255) take the conversion instruction.
__device__ __forceinline__ double f32_to_f64(float x) {
  const unsigned u = __float_as_uint(x);
  const unsigned ex = (u >> 23) & 0xffu;
  if ((u & 0x7fffffffu) == 0u) return __longlong_as_double((long long)((unsigned long long)u << 32));
  if (ex == 0u || ex == 0xffu) return (double)x;
  const unsigned long long b = ((unsigned long long)(u & 0x80000000u) << 32) |
                               ((unsigned long long)(ex + (1023u - 127u)) << 52) |
                               ((unsigned long long)(u & 0x7fffffu) << 29);
  return __longlong_as_double((long long)b);
}

// Generic arithmetic over double, float and df64 slabs.
template <typename T>
__device__ __forceinline__ T vzero() { return (T)0; }
template <>
__device__ __forceinline__ df64 vzero<df64>() { return {0.0f, 0.0f}; }
template <typename T>
__device__ __forceinline__ T vfrom(double v) { return (T)v; }
template <>
__device__ __forceinline__ df64 vfrom<df64>(double v) { return df_from(v); }
template <typename T>
__device__ __forceinline__ T vfma(T c, T x, T acc) { return fma(c, x, acc); }
template <>
__device__ __forceinline__ df64 vfma<df64>(df64 c, df64 x, df64 acc) { return df_fma(c, x, acc); }
template <typename T>
__device__ __forceinline__ T vfma1(T c, T x, T acc, float one) { return fma(c, x, acc); }
template <>
__device__ __forceinline__ df64 vfma1<df64>(df64 c, df64 x, df64 acc, float one) { return df_fma1(c, x, acc, one); }
template <typename T>
__device__ __forceinline__ T vfinish(T a) { return a; }
template <>
__device__ __forceinline__ df64 vfinish<df64>(df64 a) { return df_norm(a); }
template <typename T>
__device__ __forceinline__ bool vnonzero(T c) { return c != (T)0; }
template <>
__device__ __forceinline__ bool vnonzero<df64>(df64 c) { return c.hi != 0.0f || c.lo != 0.0f; }

// Right-hand-side load: FP64 or FP32 storage into the slab's type.
template <typename T>
__device__ __forceinline__ T gload(const double* p) { return vfrom<T>(__ldg(p)); }
template <typename T>
__device__ __forceinline__ T gload(const float* p) { return (T)__ldg(p); }
template <>
__device__ __forceinline__ df64 gload<df64>(const float* p) { return {__ldg(p), 0.0f}; }
// A typed "no right-hand side".
constexpr const double* kNoG = nullptr;
// "No right-hand side" for FP32 and float-float steps: typed float, so that
// the steps hold no double-to-float conversion (its FP64-pipe instruction
// would be issued even when the g test is false).
constexpr const float* kNoGf = nullptr;

template <typename T>
__device__ __forceinline__ T sparse_coef(const DevTaps& t, int k);
template <>
__device__ __forceinline__ double sparse_coef<double>(const DevTaps& t, int k) { return t.c64[k]; }
template <>
__device__ __forceinline__ float sparse_coef<float>(const DevTaps& t, int k) { return t.c32[k]; }
template <typename T>
__device__ __forceinline__ T dense_coef(const DevTaps& t, int k);
template <>
__device__ __forceinline__ double dense_coef<double>(const DevTaps& t, int k) { return t.d64[k]; }
template <>
__device__ __forceinline__ float dense_coef<float>(const DevTaps& t, int k) { return t.d32[k]; }
template <>
__device__ __forceinline__ df64 sparse_coef<df64>(const DevTaps& t, int k) { return {t.chi[k], t.clo[k]}; }
template <>
__device__ __forceinline__ df64 dense_coef<df64>(const DevTaps& t, int k) { return {t.dhi[k], t.dlo[k]}; }

// Element k of a slab for a stencil row: periodic (k wraps at most once), or
// for a stencil truncated at both ends (TR: Psi on the inflow/outflow domain,
// Section 4.5) zero outside 0..nx-1.
template <bool TR, typename T>
__device__ __forceinline__ T sld(const T* __restrict__ s, int k, int nx) {
  if constexpr (TR) return (unsigned)k < (unsigned)nx ? s[pidx(k)] : vzero<T>();
  else return s[pidx(wrapi(k, nx))];
}

// dst = T src (+ g): one tap at a time, any offsets (padded layout).
template <typename T, typename G, bool TR = false>
__device__ __forceinline__ void step_sparse(const DevTaps& t, const T* __restrict__ src, T* __restrict__ dst,
                                           const G* __restrict__ g, int nx) {
  for (int i = threadIdx.x; i < nx; i += blockDim.x) {
    T acc = g ? gload<T>(g + i) : vzero<T>();
    for (int k = 0; k < t.n; ++k) acc = vfma<T>(sparse_coef<T>(t, k), sld<TR>(src, i + t.off[k], nx), acc);
    dst[pidx(i)] = vfinish<T>(acc);
  }
}

// dst = T src (+ g), register-tiled: each thread produces R consecutive
// outputs from a sliding window of R inputs that advances one offset per tap,
// so each tap costs one shared load and R FMAs.  Needs the dense form and
// nx >= 64 (so that every index below wraps at most once).
// FP32 and FP64 take the taps in groups of R first: the window holds 2R
// inputs, indexed at compile time, so a group costs R loads, R * R FMAs and R
// moves (one tap at a time costs R - 1 moves per tap).  The FMAs of every
// output run in the same order either way.
template <typename T, int R, typename G, bool TR = false>
__device__ __forceinline__ void step_tiled(const DevTaps& t, const T* __restrict__ src, T* __restrict__ dst,
                                           const G* __restrict__ g, int nx) {
  const int lo = t.lo, span = t.span;
  constexpr bool kGroups = !std::is_same_v<T, df64>;
  for (int i0 = threadIdx.x * R; i0 < nx; i0 += blockDim.x * R) {
    T acc[R], w[kGroups ? 2 * R : R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      acc[r] = (g && i0 + r < nx) ? gload<T>(g + i0 + r) : vzero<T>();
      w[r] = sld<TR>(src, i0 + lo + r, nx);
    }
    int k = 0;
    if constexpr (kGroups) {
      for (; k + R <= span; k += R) {
#pragma unroll
        for (int q = 0; q < R; ++q) w[R + q] = sld<TR>(src, i0 + lo + k + R + q, nx);
#pragma unroll
        for (int kk = 0; kk < R; ++kk) {
          const T c = dense_coef<T>(t, k + kk);
          if (vnonzero<T>(c)) {
#pragma unroll
            for (int r = 0; r < R; ++r) acc[r] = vfma<T>(c, w[r + kk], acc[r]);
          }
        }
#pragma unroll
        for (int q = 0; q < R; ++q) w[q] = w[R + q];
      }
    }
    for (; k < span; ++k) {
      const T c = dense_coef<T>(t, k);
      if (vnonzero<T>(c)) {
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = vfma<T>(c, w[r], acc[r]);
      }
#pragma unroll
      for (int r = 0; r < R - 1; ++r) w[r] = w[r + 1];
      w[R - 1] = sld<TR>(src, i0 + lo + k + R, nx);
    }
#pragma unroll
    for (int r = 0; r < R; ++r)
      if (i0 + r < nx) dst[pidx(i0 + r)] = vfinish<T>(acc[r]);
  }
}

// dst = T src (+ g) for a stencil whose dense span is the compile-time SPAN:
// each thread loads its R + SPAN - 1 inputs once and keeps them in registers;
// coefficients are read from the kernel parameters (constant bank).
template <typename T, int R, int SPAN, typename G>
__device__ __forceinline__ void step_fixed(const DevTaps& t, const T* __restrict__ src, T* __restrict__ dst,
                                           const G* __restrict__ g, int nx) {
  const int lo = t.lo;
  for (int i0 = threadIdx.x * R; i0 < nx; i0 += blockDim.x * R) {
    T w[R + SPAN - 1];
#pragma unroll
    for (int q = 0; q < R + SPAN - 1; ++q) w[q] = src[pidx(wrapi(i0 + lo + q, nx))];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      T acc = (g && i0 + r < nx) ? gload<T>(g + i0 + r) : vzero<T>();
#pragma unroll
      for (int k = 0; k < SPAN; ++k) acc = vfma1<T>(dense_coef<T>(t, k), w[r + k], acc, t.one);
      if (i0 + r < nx) dst[pidx(i0 + r)] = vfinish<T>(acc);
    }
  }
}

// dst = T src (+ g) for any dense span: the span is taken in chunks of CH
// taps; per chunk each thread loads its R + CH - 1 inputs into registers once
// and does CH * R FMAs with compile-time indices; the last span % CH taps
// read their inputs directly.  Suits the wide collapsed stencils of Phi^m.
constexpr int kChunked = -8;
template <typename T, int R, int CH, typename G>
__device__ __forceinline__ void step_chunked(const DevTaps& t, const T* __restrict__ src, T* __restrict__ dst,
                                             const G* __restrict__ g, int nx) {
  const int lo = t.lo, span = t.span;
  for (int i0 = threadIdx.x * R; i0 < nx; i0 += blockDim.x * R) {
    T acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = (g && i0 + r < nx) ? gload<T>(g + i0 + r) : vzero<T>();
    int k = 0;
    for (; k + CH <= span; k += CH) {
      T w[R + CH - 1];
#pragma unroll
      for (int q = 0; q < R + CH - 1; ++q) w[q] = src[pidx(wrapi(i0 + lo + k + q, nx))];
#pragma unroll
      for (int kk = 0; kk < CH; ++kk) {
        const T c = dense_coef<T>(t, k + kk);
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = vfma1<T>(c, w[r + kk], acc[r], t.one);
      }
    }
    for (; k < span; ++k) {
      const T c = dense_coef<T>(t, k);
#pragma unroll
      for (int r = 0; r < R; ++r) acc[r] = vfma1<T>(c, src[pidx(wrapi(i0 + lo + k + r, nx))], acc[r], t.one);
    }
#pragma unroll
    for (int r = 0; r < R; ++r)
      if (i0 + r < nx) dst[pidx(i0 + r)] = vfinish<T>(acc[r]);
  }
}

// R encodes the path: 0 one tap at a time; 4, 8 sliding window; SPAN > 0
// selects the fixed-span path with register tile R; SPAN == kChunked the
// chunked path.  TR (truncated stencil) exists for the first two.
template <typename T, int R, int SPAN = 0, bool TR = false, typename G = double>
__device__ __forceinline__ void slab_step(const DevTaps& t, const T* src, T* dst, const G* g, int nx) {
  static_assert(!TR || SPAN == 0, "truncated stencils use the sliding-window or one-tap path");
  if constexpr (TR && R > 0) step_tiled<T, R, G, true>(t, src, dst, g, nx);
  else if constexpr (TR) step_sparse<T, G, true>(t, src, dst, g, nx);
  else if constexpr (SPAN == kChunked) step_chunked<T, R, 8, G>(t, src, dst, g, nx);
  else if constexpr (SPAN > 0) step_fixed<T, R, SPAN, G>(t, src, dst, g, nx);
  else if constexpr (R > 0) step_tiled<T, R, G>(t, src, dst, g, nx);
  else step_sparse<T, G>(t, src, dst, g, nx);
}

// ------------------------------------------------------- boundary rows
// Non-periodic levels (Section 4.5): after the circulant step, the rows that
// reach past either end are recomputed from their own coefficients (Fixup).
// One warp per row: its lanes split the row's columns, a shuffle tree sums.
template <typename T>
__device__ __forceinline__ T fx_coef(const Fixup& f, long long k);
template <>
__device__ __forceinline__ double fx_coef<double>(const Fixup& f, long long k) { return __ldg(f.w64 + k); }
template <>
__device__ __forceinline__ float fx_coef<float>(const Fixup& f, long long k) { return __ldg(f.w32 + k); }
template <>
__device__ __forceinline__ df64 fx_coef<df64>(const Fixup& f, long long k) { return df_from(__ldg(f.w64 + k)); }

template <typename T>
__device__ __forceinline__ T warp_add(T v, float one) {
  for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
template <>
__device__ __forceinline__ df64 warp_add<df64>(df64 v, float one) {
  for (int o = 16; o; o >>= 1) {
    const df64 u = {__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o)};
    v = df_fma1({one, 0.0f}, u, v, one);
  }
  return v;
}

template <typename T, typename G>
__device__ __forceinline__ void fixup_rows(const Fixup& f, const T* __restrict__ src, T* __restrict__ dst,
                                           const G* __restrict__ g, int nx, float one) {
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int q = threadIdx.x >> 5; q < f.nl + f.nr; q += nw) {
    const bool left = q < f.nl;
    const int row = left ? q : nx - f.nr + (q - f.nl);
    const int c0 = left ? 0 : nx - f.cr;
    const int nc = left ? f.cl : f.cr;
    const long long w0 = left ? (long long)q * f.cl : (long long)f.nl * f.cl + (long long)(q - f.nl) * f.cr;
    T acc = (g && lane == 0) ? gload<T>(g + row) : vzero<T>();
    for (int c = lane; c < nc; c += 32) acc = vfma1<T>(fx_coef<T>(f, w0 + c), src[pidx(c0 + c)], acc, one);
    acc = warp_add<T>(acc, one);
    if (lane == 0) dst[pidx(row)] = vfinish<T>(acc);
  }
}

// slab_step, then (non-periodic levels) the boundary rows; the caller's
// barrier after the step covers the fix-up as well.
template <typename T, int R, int SPAN = 0, bool TR = false, typename G = double>
__device__ __forceinline__ void slab_step_fx(const DevTaps& t, const Fixup& fx, const T* src, T* dst, const G* g,
                                             int nx) {
  slab_step<T, R, SPAN, TR, G>(t, src, dst, g, nx);
  if (fx.nl + fx.nr) {
    __syncthreads();
    fixup_rows<T, G>(fx, src, dst, g, nx, t.one);
  }
}

// Element loop i = tid, tid + blockDim.x, ... < nx in groups of K per
// thread: the K global loads of a group (ld, L2-cached) are issued before any
// value is used, so K requests per thread are in flight; a plain loop that
// stores each value to shared memory waits for every load in turn.
template <int K, typename V, typename L, typename F>
__device__ __forceinline__ void batched_loads(int nx, L&& ld, F&& use) {
  const int bs = blockDim.x;
  for (int i0 = threadIdx.x; i0 < nx; i0 += K * bs) {
    V v[K];
#pragma unroll
    for (int u = 0; u < K; ++u) {
      const int i = i0 + u * bs;
      if (i < nx) v[u] = ld(i);
    }
#pragma unroll
    for (int u = 0; u < K; ++u) {
      const int i = i0 + u * bs;
      if (i < nx) use(i, v[u]);
    }
  }
}
constexpr int kLoadBatch = 8;

// Fast path of the slab loops when nx is a multiple of 2 * blockDim.x: each
// thread takes pairs of neighbouring points e = 2 (tid + k blockDim.x), one
// 16-byte (df64, FP64) or 8-byte (FP32) global access per pair, no bounds
// tests, and up to 8 pairs' loads in flight before the first use.  Returns
// false (nothing done) when nx does not fit; the caller then runs the
// element loop.  Pairs never straddle a padding gap (groups of 8 start at
// even points), so a pair sits at pidx(e), pidx(e) + 1 in shared memory.
template <typename V2, typename L, typename F>
__device__ __forceinline__ bool pair_loop(int nx, bool aligned, L&& ld2, F&& use2) {
  const int bs = blockDim.x;
  if (!aligned || nx % (2 * bs) != 0) return false;
  const int per = nx / (2 * bs);
  for (int k0 = 0; k0 < per; k0 += 8) {
    V2 v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (k0 + u < per) v[u] = ld2(2 * (threadIdx.x + (k0 + u) * bs));
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (k0 + u < per) use2(2 * (threadIdx.x + (k0 + u) * bs), v[u]);
  }
  return true;
}
// Pair accesses need every row start they touch aligned to the pair's size
// (caller-supplied arrays may not be).
__device__ __forceinline__ bool pairs_aligned(const void* p, const void* q, long long stride_elems, int bytes) {
  const unsigned long long m = 2ull * bytes - 1;
  return ((reinterpret_cast<unsigned long long>(p) | reinterpret_cast<unsigned long long>(q)) & m) == 0 &&
         (stride_elems & 1) == 0;
}
struct df2 {  // two neighbouring float-float values
  df64 a, b;
};
__device__ __forceinline__ df2 ldcg_df2(const df64* p) {
  const float4 v = __ldcg(reinterpret_cast<const float4*>(p));
  return {{v.x, v.y}, {v.z, v.w}};
}
__device__ __forceinline__ void st_df2(df64* p, df64 a, df64 b) {
  *reinterpret_cast<float4*>(p) = make_float4(a.hi, a.lo, b.hi, b.lo);
}

// Ask L2 for `bytes` from p (one request per 128-byte line, spread over the
// block): the slab a later phase of the CTA reads then arrives while the
// current phase's loads and steps run.
__device__ __forceinline__ void prefetch_l2(const void* p, long long bytes) {
  const char* c = static_cast<const char*>(p);
  for (long long o = (long long)threadIdx.x * 128; o < bytes; o += (long long)blockDim.x * 128)
    asm volatile("prefetch.global.L2 [%0];" ::"l"(c + o));
}
__device__ __forceinline__ df64 ldcg_df(const df64* p) {
  const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
  return {v.x, v.y};
}

// Nonzero bits of v without its sign (0 iff v == +-0): integer instructions,
// where a double comparison would take an issue slot of the FP64 pipe.
__device__ __forceinline__ int dnz(double v) {
  const long long b = __double_as_longlong(v);
  return (int)(((unsigned)(b >> 32) & 0x7fffffffu) | (unsigned)b);
}

// Sum over the block in a fixed order (deterministic); result valid in thread 0.
__device__ double block_sum(double v) {
  __shared__ double ws[32];
  for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) ws[wid] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  v = (threadIdx.x < nw) ? ws[threadIdx.x] : 0.0;
  if (wid == 0)
    for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// ----------------------------------------------------------------------------
// FCF-relaxation with the fused residual for interval j.  The interval's slab
// lives in shared memory for all 2m fine steps, so each C-point crosses HBM
// once per cycle.  PREC 0: both passes FP64.  PREC 1: the second pass (acting
// on the correction rho) in FP32.
// ----------------------------------------------------------------------------
// PREC 2: both passes in FP32 with FP32 storage (coarse levels of the mixed
// modes, where every quantity is a correction of the error equation): reads
// u_old_f and g_f, writes c_new_f and r_f.
template <int R, int SPAN = 0, bool TR = false>
__device__ __forceinline__ void fcf_body_fp32(const FcfArgs& a, const int j, const DevTaps& t, unsigned char* smraw) {
  const int nx = a.nx, m = a.m, plen = padded_len(nx);
  float* b0 = reinterpret_cast<float*>(smraw);
  float* b1 = b0 + plen;
  const float* start = a.u_old_f + (long long)(j - 1) * a.cstride;
  if (!a.zero_old) prefetch_l2(a.u_old_f + (long long)j * a.cstride, (long long)nx * sizeof(float));
  int nz = 0;
  const bool al = pairs_aligned(a.u_old_f, a.c_new_f, a.cstride, 4);
  if (!pair_loop<float2>(
          nx, al, [&](int e) { return a.zero_old ? make_float2(0.0f, 0.0f) : __ldcg(reinterpret_cast<const float2*>(start + e)); },
          [&](int e, float2 v) {
            const int q = pidx(e);
            b0[q] = v.x;
            b0[q + 1] = v.y;
            nz |= (v.x != 0.0f) | (v.y != 0.0f);
          }))
    batched_loads<kLoadBatch, float>(
        nx, [&](int i) { return a.zero_old ? 0.0f : __ldcg(start + i); },
        [&](int i, float v) {
          b0[pidx(i)] = v;
          nz |= v != 0.0f;
        });
  const bool run1 = __syncthreads_or(nz) || a.g_f;  // zero slab, no rhs: Phi^m 0 = 0
  for (int s = 1; s <= m && run1; ++s) {
    const float* g = a.g_f ? a.g_f + ((long long)(j - 1) * m + s) * nx : nullptr;
    slab_step_fx<float, R, SPAN, TR>(t, a.fx, b0, b1, g, nx);
    __syncthreads();
    float* tmp = b0; b0 = b1; b1 = tmp;
  }
  const float* oldj = a.u_old_f + (long long)j * a.cstride;
  float* cn = a.c_new_f + (long long)j * nx;
  nz = 0;
  if (!pair_loop<float2>(
          nx, al, [&](int e) { return a.zero_old ? make_float2(0.0f, 0.0f) : __ldcg(reinterpret_cast<const float2*>(oldj + e)); },
          [&](int e, float2 old) {
            const int q = pidx(e);
            const float v0 = b0[q], v1 = b0[q + 1];
            *reinterpret_cast<float2*>(cn + e) = make_float2(v0, v1);
            const float r0 = v0 - old.x, r1 = v1 - old.y;
            b1[q] = r0;
            b1[q + 1] = r1;
            nz |= (r0 != 0.0f) | (r1 != 0.0f);
          }))
    batched_loads<kLoadBatch, float>(
        nx, [&](int i) { return a.zero_old ? 0.0f : __ldcg(oldj + i); },
        [&](int i, float old) {
          const float v = b0[pidx(i)];
          cn[i] = v;
          const float rho = v - old;
          b1[pidx(i)] = rho;
          nz |= rho != 0.0f;
        });
  const bool run2 = __syncthreads_or(nz);
  if (j >= a.N) return;
  float* x0 = b1;
  float* x1 = b0;
  for (int s = 1; s <= m && run2; ++s) {
    slab_step_fx<float, R, SPAN, TR>(t, a.fx, x0, x1, kNoGf, nx);
    __syncthreads();
    float* tmp = x0; x0 = x1; x1 = tmp;
  }
  float* rr = a.r_f + (long long)(j + 1) * nx;
  float ss = 0.0f;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) {
    const float v = x0[pidx(i)];
    rr[i] = v;
    ss = fmaf(v, v, ss);
  }
  if (a.partial) {
    const double tot = block_sum((double)ss);
    if (threadIdx.x == 0) a.partial[j] = tot;
  }
}

// Residual epilogue of an FP32 second pass: r_{j+1} (FP32 storage if r_f,
// else FP64) and the interval's squared norm (per-thread FP32 sums).
__device__ __forceinline__ void store_residual_f32(const FcfArgs& a, int j, const float* x) {
  const int nx = a.nx;
  float ss = 0.0f;
  if (a.r_f && nx % (2 * blockDim.x) == 0 && pairs_aligned(a.r_f, a.r_f, nx, 4)) {  // pairs, 8-byte stores
    float* rr = a.r_f + (long long)(j + 1) * nx;
    for (int e = 2 * threadIdx.x; e < nx; e += 2 * blockDim.x) {
      const int q = pidx(e);
      const float v0 = x[q], v1 = x[q + 1];
      *reinterpret_cast<float2*>(rr + e) = make_float2(v0, v1);
      ss = fmaf(v0, v0, ss);
      ss = fmaf(v1, v1, ss);
    }
  } else if (a.r_f) {
    float* rr = a.r_f + (long long)(j + 1) * nx;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
      const float v = x[pidx(i)];
      rr[i] = v;
      ss = fmaf(v, v, ss);
    }
  } else {
    double* rr = a.r + (long long)(j + 1) * nx;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
      const float v = x[pidx(i)];
      rr[i] = (double)v;
      ss = fmaf(v, v, ss);
    }
  }
  if (a.partial) {
    const double tot = block_sum((double)ss);
    if (threadIdx.x == 0) a.partial[j] = tot;
  }
}

// F-relaxation epilogue: the C-point keeps its value, r_j = v - c_j in FP64
// (stored FP32 if r_f), squared norm from the FP64 values.
template <typename V>
__device__ __forceinline__ void store_f_relaxation(const FcfArgs& a, int j, const V* b0) {
  const int nx = a.nx;
  const double* oldj = a.u_old + (long long)j * a.cstride;
  double* cn = a.c_new + (long long)j * nx;
  double ss = 0.0;
  if constexpr (std::is_same<V, df64>::value) {
    if (a.df_store) {  // C-points as float-float pairs: the FP32 pipes only, the norm from FP32 values
      const df64* od = reinterpret_cast<const df64*>(a.u_old) + (long long)j * a.cstride;
      df64* cd = reinterpret_cast<df64*>(a.c_new) + (long long)j * nx;
      float sf = 0.0f;
      for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        const df64 old = a.zero_old ? vzero<df64>() : od[i];
        const float rho = df_sub_f(b0[pidx(i)], old);
        cd[i] = old;
        if (a.r_f) a.r_f[(long long)j * nx + i] = rho;
        else a.r[(long long)j * nx + i] = (double)rho;
        sf = fmaf(rho, rho, sf);
      }
      if (a.partial) {
        ss = block_sum((double)sf);
        if (threadIdx.x == 0) a.partial[j] = ss;
      }
      return;
    }
  }
  for (int i = threadIdx.x; i < nx; i += blockDim.x) {
    const double old = a.zero_old ? 0.0 : oldj[i];
    double v;
    if constexpr (std::is_same<V, df64>::value) v = df_to(b0[pidx(i)]);
    else v = b0[pidx(i)];
    const double rho = v - old;
    cn[i] = old;
    if (a.r_f) a.r_f[(long long)j * nx + i] = (float)rho;
    else a.r[(long long)j * nx + i] = rho;
    ss = fma(rho, rho, ss);
  }
  if (a.partial) {
    ss = block_sum(ss);
    if (threadIdx.x == 0) a.partial[j] = ss;
  }
}

// The R outputs of chunk i0 (a multiple of 8) of a fixed-span step into
// registers (no right-hand side).  A window inside 0..nx-1 skips the wrap
// test, and its padded offsets are those of the stencil shifted by i0.
template <typename T, int R, int SPAN>
__device__ __forceinline__ void fixed_chunk(const DevTaps& t, const T* __restrict__ src, int i0, int nx,
                                            T (&out)[R]) {
  const int b = i0 + t.lo;
  T w[R + SPAN - 1];
  if (b >= 0 && b + R + SPAN - 1 <= nx) {
    const int p0 = i0 + (i0 >> 3);
#pragma unroll
    for (int q = 0; q < R + SPAN - 1; ++q) {
      const int d = t.lo + q;
      w[q] = src[p0 + d + (d >> 3)];
    }
  } else {
#pragma unroll
    for (int q = 0; q < R + SPAN - 1; ++q) w[q] = src[pidx(wrapi(b + q, nx))];
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    T acc;
    if constexpr (std::is_same<T, df64>::value) acc = df_mul(dense_coef<T>(t, 0), w[r]);
    else acc = dense_coef<T>(t, 0) * w[r];
#pragma unroll
    for (int k = 1; k < SPAN; ++k) acc = vfma1<T>(dense_coef<T>(t, k), w[r + k], acc, t.one);
    out[r] = vfinish<T>(acc);
  }
}

// PREC 3 with float-float C-points, one application of the collapsed Phi^m
// per pass, fixed span <= 5, FCF, no boundary rows, nx a multiple of 8
// blockDim.x, aligned rows (the launcher checks all of it and sets a.fused;
// the CTA then has one float-float slab and one FP32 slab of shared memory):
// each step's outputs go from registers straight to their uses (pass 1:
// c_new and rho against the old C-point, loaded before the arithmetic;
// pass 2: r and its squared norm) instead of through a second slab.  The
// values are the unfused body's; only the order of the norm's FP32 partial
// sums differs.

template <int SPAN>
__device__ __forceinline__ void fcf_body_df_fused(const FcfArgs& a, const int j, const DevTaps& t,
                                                  unsigned char* smraw) {
  constexpr int R = 8;
  const int nx = a.nx, plen = padded_len(nx);
  df64* b0 = reinterpret_cast<df64*>(smraw);
  float* f0 = reinterpret_cast<float*>(b0 + plen);
  const df64* startd = reinterpret_cast<const df64*>(a.u_old) + (long long)(j - 1) * a.cstride;
  const df64* oldd = reinterpret_cast<const df64*>(a.u_old) + (long long)j * a.cstride;
  df64* cnd = reinterpret_cast<df64*>(a.c_new) + (long long)j * nx;
  int nz = 0;
  pair_loop<df2>(
      nx, true, [&](int e) { return a.zero_old ? df2{} : ldcg_df2(startd + e); },
      [&](int e, df2 v) {
        const int q = pidx(e);
        b0[q] = v.a;
        b0[q + 1] = v.b;
        nz |= vnonzero<df64>(v.a) | vnonzero<df64>(v.b);
      });
  const bool run1 = __syncthreads_or(nz);  // zero slab: Phi^m 0 = 0
  int nzr = 0;
  for (int i0 = threadIdx.x * R; i0 < nx; i0 += blockDim.x * R) {
    df64 old[R];
#pragma unroll
    for (int r = 0; r < R; r += 2) {
      const df2 o = a.zero_old ? df2{} : ldcg_df2(oldd + i0 + r);
      old[r] = o.a;
      old[r + 1] = o.b;
    }
    df64 v[R];
    if (run1) {
      fixed_chunk<df64, R, SPAN>(t, b0, i0, nx, v);
    } else {
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = vzero<df64>();
    }
    const int p0 = pidx(i0);
#pragma unroll
    for (int r = 0; r < R; r += 2) st_df2(cnd + i0 + r, v[r], v[r + 1]);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const float rho = df_sub_f(v[r], old[r]);
      f0[p0 + r] = rho;
      nzr |= rho != 0.0f;
    }
  }
  const bool run2 = __syncthreads_or(nzr);
  if (j >= a.N) return;
  float* rr = a.r_f + (long long)(j + 1) * nx;
  float ss = 0.0f;
  for (int i0 = threadIdx.x * R; i0 < nx; i0 += blockDim.x * R) {
    float v[R];
    if (run2) {
      fixed_chunk<float, R, SPAN>(t, f0, i0, nx, v);
    } else {
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = 0.0f;
    }
    *reinterpret_cast<float4*>(rr + i0) = make_float4(v[0], v[1], v[2], v[3]);
    *reinterpret_cast<float4*>(rr + i0 + 4) = make_float4(v[4], v[5], v[6], v[7]);
#pragma unroll
    for (int r = 0; r < R; ++r) ss = fmaf(v[r], v[r], ss);
  }
  if (a.partial) {
    const double tot = block_sum((double)ss);
    if (threadIdx.x == 0) a.partial[j] = tot;
  }
}

// Streaming form of the fused body above for the memory-bound instances: CTA
// b owns the consecutive intervals j0..j1-1 (a balanced split of 1..N) and
// keeps two float-float slabs A (c_{j-1}, the F+C pass's input) and B (c_j,
// the old C-point rho is taken against) plus the FP32 rho slab in shared
// memory.  Once pass 1 has read A, the next interval's B = c_{j+1} is copied
// into A with cp.async while pass 2 runs, and the two swap roles: every slab
// crosses HBM once per run instead of twice per interval.  The zero-slab
// shortcut (Phi^m 0 = 0) reads B's high words as pass 1 loads them, so it
// costs no extra pass.  Arithmetic per point is the fused body's, in the same
// order: the results are bitwise those of fcf_body_df_fused.
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gmem_src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// One slab (nx float-float values) into padded shared memory, asynchronously.
__device__ __forceinline__ void slab_async(df64* dst, const df64* src, int nx) {
  for (int i = threadIdx.x; i < nx; i += blockDim.x) cp_async8(dst + pidx(i), src + i);
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}

template <int SPAN, bool ASYNC>
__global__ void __launch_bounds__(512, 2) fcf_df_stream_kernel(const FcfArgs a, const DevTaps t) {
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int R = 8;
  const int nx = a.nx, plen = padded_len(nx);
  df64* const S0 = reinterpret_cast<df64*>(smraw);  // slabs S0 and S0 + plen take turns as A and B
  float* f0 = reinterpret_cast<float*>(S0 + 2 * plen);
  const int N = a.N, G = gridDim.x, b = blockIdx.x;
  const int j0 = 1 + (int)((long long)b * N / G), j1 = 1 + (int)((long long)(b + 1) * N / G);
  if (j0 >= j1) return;
  const df64* cold = reinterpret_cast<const df64*>(a.u_old);
  df64* cnew = reinterpret_cast<df64*>(a.c_new);
  // run start: A = c_{j0-1} through registers (its zero test); with ASYNC
  // also B = c_{j0}, copied in asynchronously
  int nz = 0;
  if (!a.zero_old) {
    if constexpr (ASYNC) slab_async(S0 + plen, cold + (long long)j0 * a.cstride, nx);
    const df64* src = cold + (long long)(j0 - 1) * a.cstride;
    pair_loop<df2>(nx, true, [&](int e) { return ldcg_df2(src + e); },
                   [&](int e, df2 v) {
                     const int q = pidx(e);
                     S0[q] = v.a;
                     S0[q + 1] = v.b;
                     nz |= __float_as_uint(v.a.hi) | __float_as_uint(v.b.hi);
                   });
  }
  bool runA = __syncthreads_or(nz & 0x7fffffff);  // a float-float zero has a zero high word
  int cur = 0;
  for (int j = j0; j < j1; ++j) {
    const df64* A = S0 + cur * plen;
    df64* B = S0 + (plen - cur * plen);
    if constexpr (ASYNC) {
      cp_async_wait_all();
      __syncthreads();  // B complete and visible
    }
    int nzr = 0, nzb = 0;
    df64* cnd = cnew + (long long)j * nx;
    const df64* oldd = cold + (long long)j * a.cstride;
    for (int i0 = threadIdx.x * R; i0 < nx; i0 += blockDim.x * R) {
      const int p0 = pidx(i0);
      df64 old[R];
      if constexpr (ASYNC) {
#pragma unroll
        for (int r = 0; r < R; ++r) old[r] = a.zero_old ? vzero<df64>() : B[p0 + r];
      } else {  // c_j through registers: rho's operand now, the next interval's A after the barrier
#pragma unroll
        for (int r = 0; r < R; r += 2) {
          const df2 o = a.zero_old ? df2{} : ldcg_df2(oldd + i0 + r);
          old[r] = o.a;
          old[r + 1] = o.b;
        }
      }
      df64 v[R];
      if (runA) {
        fixed_chunk<df64, R, SPAN>(t, A, i0, nx, v);
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = vzero<df64>();
      }
#pragma unroll
      for (int r = 0; r < R; r += 2) st_df2(cnd + i0 + r, v[r], v[r + 1]);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        nzb |= __float_as_uint(old[r].hi);
        if constexpr (!ASYNC) B[p0 + r] = old[r];
        const float rho = df_sub_f(v[r], old[r]);
        f0[p0 + r] = rho;
        nzr |= __float_as_uint(rho);
      }
    }
    const bool runB = __syncthreads_or(nzb & 0x7fffffff);  // A is free from here on; B holds c_j
    const bool run2 = __syncthreads_or(nzr & 0x7fffffff);
    if constexpr (ASYNC)
      if (j + 1 < j1 && !a.zero_old) slab_async(const_cast<df64*>(A), cold + (long long)(j + 1) * a.cstride, nx);
    if (j < N) {
      float* rr = a.r_f + (long long)(j + 1) * nx;
      float ss = 0.0f;
      for (int i0 = threadIdx.x * R; i0 < nx; i0 += blockDim.x * R) {
        float v[R];
        if (run2) {
          fixed_chunk<float, R, SPAN>(t, f0, i0, nx, v);
        } else {
#pragma unroll
          for (int r = 0; r < R; ++r) v[r] = 0.0f;
        }
        *reinterpret_cast<float4*>(rr + i0) = make_float4(v[0], v[1], v[2], v[3]);
        *reinterpret_cast<float4*>(rr + i0 + 4) = make_float4(v[4], v[5], v[6], v[7]);
#pragma unroll
        for (int r = 0; r < R; ++r) ss = fmaf(v[r], v[r], ss);
      }
      if (a.partial) {
        const double tot = block_sum((double)ss);  // its barriers also retire this pass's reads of rho
        if (threadIdx.x == 0) a.partial[j] = tot;
      }
    }
    __syncthreads();  // rho (f0) is read; the next interval overwrites f0 and reads A/B swapped
    runA = runB;
    cur = 1 - cur;
  }
  if constexpr (ASYNC) cp_async_wait_all();
}

// Register-resident form of the fused body for upwind stencils (offsets
// -(SPAN-1)..0, ERK1+U1's collapsed Phi^m): one CTA per interval, nx/8
// threads, each holding its 8 points in registers.  The SPAN-1 points left of
// a thread's chunk come from the lane below by warp shuffle (lane 0 loads its
// own from the slab, with the periodic wrap); the rho values the residual
// pass needs across a warp boundary go through shared memory once.  No slab
// is staged in shared memory, so neither pass waits on shared-memory loads,
// and the zero-slab shortcut is a warp vote.  Per output the arithmetic is
// fcf_body_df_fused's, in the same order: bitwise its results.
template <int SPAN>
__global__ void __launch_bounds__(1024) fcf_df_reg_kernel(const FcfArgs a, const DevTaps t) {
  constexpr int R = 8, H = SPAN - 1;
  __shared__ float xh[32][H > 0 ? H : 1];  // each warp's last H rho values
  const int nx = a.nx, j = blockIdx.x + 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int i0 = threadIdx.x * R;
  const df64* xs = reinterpret_cast<const df64*>(a.u_old) + (long long)(j - 1) * a.cstride;
  const df64* os = reinterpret_cast<const df64*>(a.u_old) + (long long)j * a.cstride;
  df64 w[R + H], old[R];
#pragma unroll
  for (int r = 0; r < R; r += 2) {
    const df2 v = a.zero_old ? df2{} : ldcg_df2(xs + i0 + r);
    w[H + r] = v.a;
    w[H + r + 1] = v.b;
    const df2 o = a.zero_old ? df2{} : ldcg_df2(os + i0 + r);
    old[r] = o.a;
    old[r + 1] = o.b;
  }
  unsigned nzw = 0;
#pragma unroll
  for (int q = 0; q < H; ++q) {
    float hi = __shfl_up_sync(0xffffffffu, w[R + q].hi, 1);
    float lo = __shfl_up_sync(0xffffffffu, w[R + q].lo, 1);
    if (lane == 0) {  // the chunk left of lane 0's: another warp's (or, periodic, the slab's end)
      float2 g = make_float2(0.0f, 0.0f);
      if (!a.zero_old) g = __ldcg(reinterpret_cast<const float2*>(xs) + wrapi(i0 - H + q, nx));
      hi = g.x;
      lo = g.y;
    }
    w[q] = {hi, lo};
  }
#pragma unroll
  for (int q = 0; q < R + H; ++q) nzw |= __float_as_uint(w[q].hi);
  df64 v[R];
  if (__any_sync(0xffffffffu, (nzw & 0x7fffffffu) != 0)) {  // Phi^m 0 = 0
#pragma unroll
    for (int r = 0; r < R; ++r) {
      df64 acc = df_mul(dense_coef<df64>(t, 0), w[r]);
#pragma unroll
      for (int k = 1; k < SPAN; ++k) acc = vfma1<df64>(dense_coef<df64>(t, k), w[r + k], acc, t.one);
      v[r] = vfinish<df64>(acc);
    }
  } else {
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = vzero<df64>();
  }
  df64* cnd = reinterpret_cast<df64*>(a.c_new) + (long long)j * nx;
#pragma unroll
  for (int r = 0; r < R; r += 2) st_df2(cnd + i0 + r, v[r], v[r + 1]);
  float rw[R + H];
  unsigned nzr = 0;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    rw[H + r] = df_sub_f(v[r], old[r]);
    nzr |= __float_as_uint(rw[H + r]);
  }
  if (j >= a.N) return;  // the last interval has no residual (uniform over the CTA)
  if (lane == 31)
#pragma unroll
    for (int q = 0; q < H; ++q) xh[warp][q] = rw[R + q];
  __syncthreads();
  const int wl = warp == 0 ? nw - 1 : warp - 1;  // periodic: warp 0's left neighbour is the last warp
#pragma unroll
  for (int q = 0; q < H; ++q) {
    const float u = __shfl_up_sync(0xffffffffu, rw[R + q], 1);
    rw[q] = lane == 0 ? xh[wl][q] : u;
    nzr |= __float_as_uint(rw[q]);
  }
  float* rr = a.r_f + (long long)(j + 1) * nx;
  float o[R];
  if (__any_sync(0xffffffffu, (nzr & 0x7fffffffu) != 0)) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      float acc = dense_coef<float>(t, 0) * rw[r];
#pragma unroll
      for (int k = 1; k < SPAN; ++k) acc = vfma1<float>(dense_coef<float>(t, k), rw[r + k], acc, t.one);
      o[r] = vfinish<float>(acc);
    }
  } else {
#pragma unroll
    for (int r = 0; r < R; ++r) o[r] = 0.0f;
  }
  *reinterpret_cast<float4*>(rr + i0) = make_float4(o[0], o[1], o[2], o[3]);
  *reinterpret_cast<float4*>(rr + i0 + 4) = make_float4(o[4], o[5], o[6], o[7]);
  float ss = 0.0f;
#pragma unroll
  for (int r = 0; r < R; ++r) ss = fmaf(o[r], o[r], ss);
  if (a.partial) {
    const double tot = block_sum((double)ss);
    if (threadIdx.x == 0) a.partial[j] = tot;
  }
}

// Persistent form of the register-resident body: CTA b owns the intervals
// j0..j1-1 (a balanced split of 1..N).  Interval j+1's input c_j is interval
// j's old C-point, already in registers, so a run reads each slab from HBM
// once: each thread copies its own chunk of the next one, c_{j+1}, into
// shared memory with 16-byte cp.async while interval j computes (three
// buffers, slab k in buffer k mod 3).  The SPAN-1 points left of a thread's
// chunk are the tail of its left neighbour's chunk (periodic across the
// slab): c_{j-1}'s tail is read from the neighbour's buffer units, published
// by the previous interval's barrier and not overwritten before the next one;
// rho's tail goes through a parity-double-buffered per-thread slot at the
// one barrier of an interval.  Thread t's unit u (16 bytes, two points) sits
// at 4t + (u ^ ((t >> 1) & 3)), so a quarter-warp's 16-byte loads hit 8
// distinct bank groups.  The norm is one fixed-order block reduction per
// run, stored at partial[j0] (zeros at the run's other intervals): the sum
// the norm kernel forms is the same quantity, in another order.  Arithmetic
// per output: fcf_body_df_fused's (V = df64, MIXED_DF) or the FP64 pass of
// fcf_body with the FP32 second pass (V = double, MIXED); either C-point type
// takes 8 bytes per point, so the layout and the copies are the same.
__device__ __forceinline__ int swz_unit(int t, int u) { return 4 * t + (u ^ ((t >> 1) & 3)); }

template <typename V>
struct RunOps;
template <>
struct RunOps<df64> {
  static __device__ __forceinline__ void unit(const df64* p, df64& x, df64& y) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    x = {q.x, q.y};
    y = {q.z, q.w};
  }
  static __device__ __forceinline__ void st2(df64* p, df64 x, df64 y) { st_df2(p, x, y); }
  static constexpr unsigned kNzMask = 0x7fffffffu;  // nz(v) & kNzMask != 0 iff v != 0
  static __device__ __forceinline__ unsigned nz(df64 v) { return __float_as_uint(v.hi); }
  static __device__ __forceinline__ df64 mul(df64 c, df64 w) { return df_mul(c, w); }
  static __device__ __forceinline__ float sub_f(df64 x, df64 y) { return df_sub_f(x, y); }
};
template <>
struct RunOps<double> {
  static __device__ __forceinline__ void unit(const double* p, double& x, double& y) {
    const double2 q = *reinterpret_cast<const double2*>(p);
    x = q.x;
    y = q.y;
  }
  static __device__ __forceinline__ void st2(double* p, double x, double y) {
    *reinterpret_cast<double2*>(p) = make_double2(x, y);
  }
  static constexpr unsigned kNzMask = ~0u;
  static __device__ __forceinline__ unsigned nz(double v) { return (unsigned)dnz(v); }
  static __device__ __forceinline__ double mul(double c, double w) { return c * w; }
  static __device__ __forceinline__ float sub_f(double x, double y) { return (float)(x - y); }
};

template <int SPAN, typename V>
__global__ void __launch_bounds__(1024) fcf_regrun_kernel(const FcfArgs a, const DevTaps t) {
  using Op = RunOps<V>;
  constexpr int R = 8, H = SPAN - 1;
  static_assert(H >= 1 && H <= 4, "the left halo is at most the neighbour's last two units");
  extern __shared__ __align__(16) unsigned char smraw[];
  const int nx = a.nx, N = a.N, G = gridDim.x, b = blockIdx.x;
  const int j0 = 1 + (int)((long long)b * N / G), j1 = 1 + (int)((long long)(b + 1) * N / G);
  if (j0 >= j1) return;
  const int tid = threadIdx.x, T = blockDim.x;
  const int tl = tid == 0 ? T - 1 : tid - 1;  // the left neighbour (periodic)
  const int i0 = tid * R;
  V* const B0 = reinterpret_cast<V*>(smraw);                            // three slabs
  float4* const RX = reinterpret_cast<float4*>(B0 + 3 * (long long)nx);  // rho tails, two by parity
  const V* cold = reinterpret_cast<const V*>(a.u_old);
  auto prefetch = [&](int jj) {  // this thread's chunk of c_jj into buffer jj mod 3
    V* dst = B0 + (long long)(jj % 3) * nx;
    const V* src = cold + (long long)jj * a.cstride + i0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const unsigned d = (unsigned)__cvta_generic_to_shared(dst + 2 * swz_unit(tid, u));
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src + 2 * u) : "memory");
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  auto load_units = [&](const V* buf, int th, int u0, int nu, V* out) {  // units u0.. of thread th
    for (int u = 0; u < nu; ++u) Op::unit(buf + 2 * swz_unit(th, u0 + u), out[2 * u], out[2 * u + 1]);
  };
  V cur[R];  // c_{j-1} of this thread's chunk
  if (!a.zero_old) {
    prefetch(j0 - 1);
    prefetch(j0);
    asm volatile("cp.async.wait_all;\n" ::: "memory");
  }
  __syncthreads();  // c_{j0-1} of every chunk visible (the first interval's halo)
  if (a.zero_old) {
#pragma unroll
    for (int r = 0; r < R; ++r) cur[r] = vzero<V>();
  } else {
    load_units(B0 + (long long)((j0 - 1) % 3) * nx, tid, 0, 4, cur);
  }
  float ss = 0.0f;
  for (int j = j0; j < j1; ++j) {
    const int par = j & 1;
    V old[R];
    V w[R + H];
    if (a.zero_old) {
#pragma unroll
      for (int r = 0; r < R; ++r) old[r] = vzero<V>();
#pragma unroll
      for (int q = 0; q < H; ++q) w[q] = vzero<V>();
    } else {
      asm volatile("cp.async.wait_all;\n" ::: "memory");  // this thread's chunk of c_j
      if (j + 1 < j1) prefetch(j + 1);  // into the buffer of c_{j-2}, read by its last reader before the last barrier
      load_units(B0 + (long long)(j % 3) * nx, tid, 0, 4, old);
      V tail[4];
      load_units(B0 + (long long)((j + 2) % 3) * nx, tl, 2, 2, tail);  // c_{j-1}, points 4..7 of the neighbour
#pragma unroll
      for (int q = 0; q < H; ++q) w[q] = tail[4 - H + q];
    }
#pragma unroll
    for (int r = 0; r < R; ++r) w[H + r] = cur[r];
    unsigned nzw = 0;
#pragma unroll
    for (int q = 0; q < R + H; ++q) nzw |= Op::nz(w[q]);
    V v[R];
    if (__any_sync(0xffffffffu, (nzw & Op::kNzMask) != 0)) {  // Phi^m 0 = 0
#pragma unroll
      for (int r = 0; r < R; ++r) {
        V acc = Op::mul(dense_coef<V>(t, 0), w[r]);
#pragma unroll
        for (int k = 1; k < SPAN; ++k) acc = vfma1<V>(dense_coef<V>(t, k), w[r + k], acc, t.one);
        v[r] = vfinish<V>(acc);
      }
    } else {
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = vzero<V>();
    }
    V* cnd = reinterpret_cast<V*>(a.c_new) + (long long)j * nx;
#pragma unroll
    for (int r = 0; r < R; r += 2) Op::st2(cnd + i0 + r, v[r], v[r + 1]);
    float rw[R + H];
    unsigned nzr = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      rw[H + r] = Op::sub_f(v[r], old[r]);
      nzr |= __float_as_uint(rw[H + r]);
      cur[r] = old[r];
    }
    if (j < N) {  // uniform over the CTA (only the problem's last interval has no residual)
      RX[par * T + tid] = make_float4(rw[R + H - 4], rw[R + H - 3], rw[R + H - 2], rw[R + H - 1]);  // last 4 rho
      __syncthreads();
      const float4 q = RX[par * T + tl];
      const float qa[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
      for (int k = 0; k < H; ++k) {
        rw[k] = qa[4 - H + k];
        nzr |= __float_as_uint(rw[k]);
      }
      float* rr = a.r_f + (long long)(j + 1) * nx;
      float o[R];
      if (__any_sync(0xffffffffu, (nzr & 0x7fffffffu) != 0)) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
          float acc = dense_coef<float>(t, 0) * rw[r];
#pragma unroll
          for (int k = 1; k < SPAN; ++k) acc = vfma1<float>(dense_coef<float>(t, k), rw[r + k], acc, t.one);
          o[r] = vfinish<float>(acc);
        }
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) o[r] = 0.0f;
      }
      *reinterpret_cast<float4*>(rr + i0) = make_float4(o[0], o[1], o[2], o[3]);
      *reinterpret_cast<float4*>(rr + i0 + 4) = make_float4(o[4], o[5], o[6], o[7]);
#pragma unroll
      for (int r = 0; r < R; ++r) ss = fmaf(o[r], o[r], ss);
      if (a.partial && tid == 0 && j > j0) a.partial[j] = 0.0;
    }
  }
  if (a.partial && j0 < N) {
    const double tot = block_sum((double)ss);
    if (tid == 0) a.partial[j0] = tot;
  }
  if (!a.zero_old) asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// PREC 3: pass 1 (C-point update and residual rho) in float-float, pass 2 in
// FP32.  A df64 slab occupies as many bytes as an FP64 slab.
template <int R, int SPAN = 0, bool TR = false, bool FUSE = true>
__device__ __forceinline__ void fcf_body_df(const FcfArgs& a, const int j, const DevTaps& t, unsigned char* smraw) {
  // narrow collapsed stencils only: wider windows would raise every path's
  // register count (and so cut the CTAs per SM)
  if constexpr (FUSE && SPAN > 0 && SPAN <= 5 && !TR) {
    if (a.fused) {  // the launcher's decision (it sized shared memory for it)
      fcf_body_df_fused<SPAN>(a, j, t, smraw);
      return;
    }
  }
  const int nx = a.nx, m = a.m, plen = padded_len(nx);
  df64* b0 = reinterpret_cast<df64*>(smraw);
  df64* b1 = b0 + plen;
  const double* start = a.u_old + (long long)(j - 1) * a.cstride;
  const df64* startd = reinterpret_cast<const df64*>(a.u_old) + (long long)(j - 1) * a.cstride;
  if (!a.zero_old) prefetch_l2(a.u_old + (long long)j * a.cstride, (long long)nx * 8);
  int nz = 0;
  const bool al = pairs_aligned(a.u_old, a.c_new, a.cstride, 8);
  if (a.df_store) {  // float-float C-points: no conversion on the FP64 pipe
    if (!pair_loop<df2>(
            nx, al, [&](int e) { return a.zero_old ? df2{} : ldcg_df2(startd + e); },
            [&](int e, df2 v) {
              const int q = pidx(e);
              b0[q] = v.a;
              b0[q + 1] = v.b;
              nz |= vnonzero<df64>(v.a) | vnonzero<df64>(v.b);
            }))
      batched_loads<kLoadBatch, df64>(
          nx, [&](int i) { return a.zero_old ? vzero<df64>() : ldcg_df(startd + i); },
          [&](int i, df64 v) {
            b0[pidx(i)] = v;
            nz |= vnonzero<df64>(v);
          });
  } else {
    batched_loads<kLoadBatch, double>(
        nx, [&](int i) { return a.zero_old ? 0.0 : __ldcg(start + i); },
        [&](int i, double v) {
          b0[pidx(i)] = df_from(v);
          nz |= dnz(v);
        });
  }
  // precision 3 runs only on level 1, which has no right-hand side
  const bool run1 = __syncthreads_or(nz);  // zero slab: Phi^m 0 = 0
  for (int s = 1; s <= m && run1; ++s) {
    slab_step_fx<df64, R, SPAN, TR>(t, a.fx, b0, b1, kNoGf, nx);
    __syncthreads();
    df64* tmp = b0; b0 = b1; b1 = tmp;
  }
  const double* oldj = a.u_old + (long long)j * a.cstride;
  double* cn = a.c_new + (long long)j * nx;
  if (a.relax_f) {
    store_f_relaxation(a, j, b0);
    return;
  }
  float* f0 = reinterpret_cast<float*>(b1);
  float* f1 = f0 + plen;
  nz = 0;
  if (a.df_store) {
    const df64* oldd = reinterpret_cast<const df64*>(a.u_old) + (long long)j * a.cstride;
    df64* cnd = reinterpret_cast<df64*>(a.c_new) + (long long)j * nx;
    if (!pair_loop<df2>(
            nx, al, [&](int e) { return a.zero_old ? df2{} : ldcg_df2(oldd + e); },
            [&](int e, df2 old) {
              const int q = pidx(e);
              const df64 v0 = b0[q], v1 = b0[q + 1];
              st_df2(cnd + e, v0, v1);
              const float r0 = df_sub_f(v0, old.a), r1 = df_sub_f(v1, old.b);
              f0[q] = r0;
              f0[q + 1] = r1;
              nz |= (r0 != 0.0f) | (r1 != 0.0f);
            }))
      batched_loads<kLoadBatch, df64>(
          nx, [&](int i) { return a.zero_old ? vzero<df64>() : ldcg_df(oldd + i); },
          [&](int i, df64 old) {
            const df64 v = b0[pidx(i)];
            cnd[i] = v;
            const float rho = df_sub_f(v, old);
            f0[pidx(i)] = rho;
            nz |= rho != 0.0f;
          });
  } else {
    batched_loads<kLoadBatch, double>(
        nx, [&](int i) { return a.zero_old ? 0.0 : __ldcg(oldj + i); },
        [&](int i, double old) {
          const double v = df_to(b0[pidx(i)]);
          cn[i] = v;
          const float rho = (float)(v - old);
          f0[pidx(i)] = rho;
          nz |= rho != 0.0f;
        });
  }
  const bool run2 = __syncthreads_or(nz);
  if (j >= a.N) return;
  for (int s = 1; s <= m && run2; ++s) {
    slab_step_fx<float, R, SPAN, TR>(t, a.fx, f0, f1, kNoGf, nx);
    __syncthreads();
    float* tmp = f0; f0 = f1; f1 = tmp;
  }
  store_residual_f32(a, j, f0);
}

template <int PREC, int R, int SPAN = 0, bool TR = false, bool FUSE = true>
__device__ __forceinline__ void fcf_body(const FcfArgs& a, const int j, const DevTaps& t, unsigned char* smraw) {
  if constexpr (PREC == 2) {
    fcf_body_fp32<R, SPAN, TR>(a, j, t, smraw);
    return;
  }
  if constexpr (PREC == 3) {
    fcf_body_df<R, SPAN, TR, FUSE>(a, j, t, smraw);
    return;
  }
  const int nx = a.nx, m = a.m, plen = padded_len(nx);
  double* b0 = reinterpret_cast<double*>(smraw);
  double* b1 = b0 + plen;
  const double* start = a.u_old + (long long)(j - 1) * a.cstride;
  if (!a.zero_old && !a.value_residual)
    prefetch_l2(a.u_old + (long long)j * a.cstride, (long long)nx * sizeof(double));
  int nz = 0;
  const bool al = pairs_aligned(a.u_old, a.c_new, a.cstride, 8);
  if (!pair_loop<double2>(
          nx, al, [&](int e) { return a.zero_old ? make_double2(0.0, 0.0) : __ldcg(reinterpret_cast<const double2*>(start + e)); },
          [&](int e, double2 v) {
            const int q = pidx(e);
            b0[q] = v.x;
            b0[q + 1] = v.y;
            nz |= dnz(v.x) | dnz(v.y);
          }))
    batched_loads<kLoadBatch, double>(
        nx, [&](int i) { return a.zero_old ? 0.0 : __ldcg(start + i); },
        [&](int i, double v) {
          b0[pidx(i)] = v;
          nz |= dnz(v);
        });
  // Phi^m of an identically zero slab is zero (no right-hand side): the
  // steps are skipped, which leaves the result exactly as computed
  const bool run1 = __syncthreads_or(nz) || a.g;
  for (int s = 1; s <= m && run1; ++s) {
    const double* g = a.g ? a.g + ((long long)(j - 1) * m + s) * nx : nullptr;
    slab_step_fx<double, R, SPAN, TR>(t, a.fx, b0, b1, g, nx);
    __syncthreads();
    double* tmp = b0; b0 = b1; b1 = tmp;
  }
  const double* oldj = a.u_old + (long long)j * a.cstride;
  double* cn = a.c_new + (long long)j * nx;
  const bool more = j < a.N;
  double ss = 0.0;
  if (a.relax_f) {
    store_f_relaxation(a, j, b0);
    return;
  }
  if (PREC == 0) {
    nz = 0;
    batched_loads<kLoadBatch, double>(
        nx, [&](int i) { return (a.value_residual || a.zero_old) ? 0.0 : __ldcg(oldj + i); },
        [&](int i, double old) {
          const double v = b0[pidx(i)];
          cn[i] = v;
          const double rho = a.value_residual ? v : v - old;
          b1[pidx(i)] = rho;
          nz |= dnz(rho);
        });
    const bool run2 = __syncthreads_or(nz);
    if (!more) return;
    double* x0 = b1;
    double* x1 = b0;
    for (int s = 1; s <= m && run2; ++s) {
      slab_step_fx<double, R, SPAN, TR>(t, a.fx, x0, x1, kNoG, nx);
      __syncthreads();
      double* tmp = x0; x0 = x1; x1 = tmp;
    }
    double* rr = a.r + (long long)(j + 1) * nx;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
      const double v = x0[pidx(i)];
      rr[i] = v;
      ss = fma(v, v, ss);
    }
    if (a.value_residual) return;  // Phi^m c_new_j stored; residual_value finishes
  } else {
    float* f0 = reinterpret_cast<float*>(b1);
    float* f1 = f0 + plen;
    nz = 0;
    if (!pair_loop<double2>(
            nx, al, [&](int e) { return a.zero_old ? make_double2(0.0, 0.0) : __ldcg(reinterpret_cast<const double2*>(oldj + e)); },
            [&](int e, double2 old) {
              const int q = pidx(e);
              const double v0 = b0[q], v1 = b0[q + 1];
              *reinterpret_cast<double2*>(cn + e) = make_double2(v0, v1);
              const float r0 = (float)(v0 - old.x), r1 = (float)(v1 - old.y);
              f0[q] = r0;
              f0[q + 1] = r1;
              nz |= (r0 != 0.0f) | (r1 != 0.0f);
            }))
      batched_loads<kLoadBatch, double>(
          nx, [&](int i) { return a.zero_old ? 0.0 : __ldcg(oldj + i); },
          [&](int i, double old) {
            const double v = b0[pidx(i)];
            cn[i] = v;
            const float rho = (float)(v - old);
            f0[pidx(i)] = rho;
            nz |= rho != 0.0f;
          });
    const bool run2 = __syncthreads_or(nz);
    if (!more) return;
    for (int s = 1; s <= m && run2; ++s) {
      slab_step_fx<float, R, SPAN, TR>(t, a.fx, f0, f1, kNoGf, nx);
      __syncthreads();
      float* tmp = f0; f0 = f1; f1 = tmp;
    }
    store_residual_f32(a, j, f0);
    return;
  }
  if (a.partial) {
    ss = block_sum(ss);
    if (threadIdx.x == 0) a.partial[j] = ss;
  }
}

template <int PREC, int R, int SPAN = 0, bool TR = false>
__global__ void __launch_bounds__(R == 8 ? 512 : 1024) fcf_kernel(const FcfArgs a, const DevTaps t) {
  extern __shared__ __align__(16) unsigned char smraw[];
  fcf_body<PREC, R, SPAN, TR>(a, blockIdx.x + 1, t, smraw);
}

// Batched: one CTA per (solve, interval) item across all admitted solves; the
// solve's stencil is copied into shared memory first.
template <int R, int SPAN = 0>
__global__ void __launch_bounds__(R == 8 ? 512 : 1024) fcf_batched_kernel(const BatchSolve* __restrict__ S,
                                                            const BatchItem* __restrict__ items,
                                                            const DevTaps* __restrict__ taps) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ __align__(16) DevTaps st;
  const BatchItem it = items[blockIdx.x];
  const BatchSolve* s = S + it.solve;
  const int* src = reinterpret_cast<const int*>(taps + s->taps);
  int* dst = reinterpret_cast<int*>(&st);
  for (int k = threadIdx.x; k < (int)(sizeof(DevTaps) / sizeof(int)); k += blockDim.x) dst[k] = src[k];
  __syncthreads();
  const FcfArgs a = s->fcf;
  if (s->prec == 0) fcf_body<0, R, SPAN>(a, it.j, st, smraw);
  else if (s->prec == 3) fcf_body<3, R, SPAN, false, false>(a, it.j, st, smraw);  // one register budget for all
  else fcf_body<1, R, SPAN>(a, it.j, st, smraw);
}

// ----------------------------------------------------------------------------
// Level-1 FCF-relaxation of a periodic problem with its FP64 pass in Fourier
// space (MIXED).  The collapsed Phi^m is circulant, so the discrete Fourier
// transform diagonalises it (Lemma 1): with X_k = sum_x x[x] w^{xk},
// w = exp(-2 pi i / nx), the new C-point c'_j = Phi^m c_{j-1} has the
// spectrum S_k X_k, S_k = sum_q c_q exp(+2 pi i o_q k / nx) the symbol of the
// collapsed stencil (offsets o_q, coefficients c_q).  Per interval the slab
// is transformed as one complex FFT of half length h = nx/2 (z_q = x_{2q} +
// i x_{2q+1}; radix-4 decimation in frequency, natural order in, bit-reversed
// out), its modes are split into X_0..X_h, multiplied by S and recombined
// (one thread per mode pair k, h-k, in the bit-reversed positions), and a
// radix-4 decimation-in-time inverse (bit-reversed in, natural out) returns
// c'_j.  That takes about 45 FP64 instructions per point where the collapsed
// stencil takes one FMA per tap (73 for ERK3+U3 at m = 8).  The residual's
// pass (rho = c'_j - c_j in FP32, r_{j+1} = Phi^m rho) is the MIXED body's.
// The factors 1/2 of the split and recombination and the inverse's 1/h are
// one exact power of two folded into S (the table holds S_k / (2 nx)).  An
// identically zero slab skips the transforms and stays exactly zero.
// ----------------------------------------------------------------------------
struct zc64 {
  double re, im;
};
__device__ __forceinline__ zc64 zmul(zc64 a, zc64 b) {
  return {fma(a.re, b.re, -a.im * b.im), fma(a.re, b.im, a.im * b.re)};
}
__device__ __forceinline__ zc64 ldz(const zc64* p) {
  const double2 v = __ldg(reinterpret_cast<const double2*>(p));
  return {v.x, v.y};
}

// Sign flip on the integer pipe (an FP64 negation would take an FP64 issue).
__device__ __forceinline__ double dneg(double x) {
  return __hiloint2double(__double2hiint(x) ^ (int)0x80000000, __double2loint(x));
}
// a * conj(w)
__device__ __forceinline__ zc64 zmulc(zc64 a, zc64 w) {
  return {fma(a.re, w.re, a.im * w.im), fma(a.im, w.re, -a.re * w.im)};
}
// w^k, w = exp(-2 pi i / nx), 0 <= k < 3h/2 (nx = 2h), from the quarter
// table tw[0..h/4]: w^(h/2 - k) = -i conj(w^k) folds (h/4, h/2) onto
// [0, h/4), w^(h/2) = -i and w^h = -1 the rest; sign flips and swaps only.
__device__ __forceinline__ zc64 twq(const zc64* __restrict__ tw, int k, int h) {
  const int hh = h >> 1;
  const int sector = k >= h ? 2 : (k >= hh ? 1 : 0);
  const int kk = k - sector * hh;
  zc64 r;
  if (kk <= (h >> 2)) {
    r = ldz(tw + kk);
  } else {
    const zc64 c = ldz(tw + (hh - kk));
    r = {dneg(c.im), dneg(c.re)};
  }
  if (sector == 1) r = {r.im, dneg(r.re)};
  else if (sector == 2) r = {dneg(r.re), dneg(r.im)};
  return r;
}

// The radix-2 pass of span 1 (twiddle 1): the last forward pass, the first
// inverse one, when log2 h is odd.
__device__ __forceinline__ void radix2_unit_pass(zc64* x, int h) {
  for (int b = threadIdx.x; b < (h >> 1); b += blockDim.x) {
    const zc64 u = x[2 * b], v = x[2 * b + 1];
    x[2 * b] = {u.re + v.re, u.im + v.im};
    x[2 * b + 1] = {u.re - v.re, u.im - v.im};
  }
  __syncthreads();
}

// One radix-4 pass of span q over x[0..h): butterfly (g, pos) takes
// x[4qg + pos + {0, q, 2q, 3q}], pos < q, g < h/4q.  A thread keeps one
// position while it can (q <= CTA size: every group of its position), so
// its three twiddles are looked up once per position, not per butterfly.
// Forward (DIF, the work of the radix-2 passes of spans 2q and q; twiddles
// W^pos, W^2pos, W^3pos of W = exp(-2 pi i / 4q) on the outputs), or inverse
// (DIT, conjugate twiddles on the inputs, the two passes in reverse order).
template <bool INV>
__device__ __forceinline__ void radix4_pass(zc64* x, const zc64* __restrict__ tw, int h, int q) {
  const int bs = blockDim.x, tid = threadIdx.x;
  const int s = h / (2 * q), groups = h / (4 * q);  // W^pos = w^(pos s)
  const bool wide = q >= bs;
  const int gstep = wide ? 1 : bs / q;
  for (int pos = wide ? tid : (tid & (q - 1)); pos < q; pos += wide ? bs : q) {
    zc64 w1 = {1.0, 0.0}, w2 = {1.0, 0.0}, w3 = {1.0, 0.0};
    if (pos) {
      w1 = twq(tw, pos * s, h);
      w2 = twq(tw, 2 * pos * s, h);
      w3 = twq(tw, 3 * pos * s, h);
    }
    for (int g = wide ? 0 : tid / q; g < groups; g += gstep) {
      const int i0 = 4 * q * g + pos;
      if constexpr (!INV) {
        const zc64 x0 = x[i0], x1 = x[i0 + q], x2 = x[i0 + 2 * q], x3 = x[i0 + 3 * q];
        const zc64 a0 = {x0.re + x2.re, x0.im + x2.im}, a1 = {x0.re - x2.re, x0.im - x2.im};
        const zc64 a2 = {x1.re + x3.re, x1.im + x3.im};
        const zc64 a3 = {x1.im - x3.im, x3.re - x1.re};  // -i (x1 - x3)
        zc64 y1 = {a0.re - a2.re, a0.im - a2.im};
        zc64 y2 = {a1.re + a3.re, a1.im + a3.im};
        zc64 y3 = {a1.re - a3.re, a1.im - a3.im};
        x[i0] = {a0.re + a2.re, a0.im + a2.im};
        if (pos) {
          y1 = zmul(y1, w2);
          y2 = zmul(y2, w1);
          y3 = zmul(y3, w3);
        }
        x[i0 + q] = y1;
        x[i0 + 2 * q] = y2;
        x[i0 + 3 * q] = y3;
      } else {
        zc64 v0 = x[i0], v1 = x[i0 + q], v2 = x[i0 + 2 * q], v3 = x[i0 + 3 * q];
        if (pos) {
          v1 = zmulc(v1, w2);
          v2 = zmulc(v2, w1);
          v3 = zmulc(v3, w3);
        }
        const zc64 p0 = {v0.re + v1.re, v0.im + v1.im}, m0 = {v0.re - v1.re, v0.im - v1.im};
        const zc64 p1 = {v2.re + v3.re, v2.im + v3.im};
        const zc64 m1 = {v3.im - v2.im, v2.re - v3.re};  // i (v2 - v3)
        x[i0] = {p0.re + p1.re, p0.im + p1.im};
        x[i0 + 2 * q] = {p0.re - p1.re, p0.im - p1.im};
        x[i0 + q] = {m0.re + m1.re, m0.im + m1.im};
        x[i0 + 3 * q] = {m0.re - m1.re, m0.im - m1.im};
      }
    }
  }
  __syncthreads();
}

// Forward transform of x[0..h) in place, natural order in, bit-reversed out:
// radix-4 passes of spans h/4, h/16, ..., then a radix-2 pass of span 1 if
// log2 h is odd.
__device__ __forceinline__ void dif_forward(zc64* x, const zc64* __restrict__ tw, int h, int logh) {
  for (int q = h >> 2; q >= 1; q >>= 2) radix4_pass<false>(x, tw, h, q);
  if (logh & 1) radix2_unit_pass(x, h);
}

// Inverse transform (conjugate twiddles, no 1/h), bit-reversed order in,
// natural out: the forward passes' inverses in reverse order.
__device__ __forceinline__ void dit_inverse(zc64* x, const zc64* __restrict__ tw, int h, int logh) {
  int q = 1;
  if (logh & 1) {
    radix2_unit_pass(x, h);
    q = 2;
  }
  for (; q <= (h >> 2); q <<= 2) radix4_pass<true>(x, tw, h, q);
}

__device__ __forceinline__ int bitrev_n(int i, int logn) { return (int)(__brev((unsigned)i) >> (32 - logn)); }

// Multiply the spectrum of the slab by S, in place on the half-length
// transform Z (bit-reversed order).  Mode pair (k, h-k), k = 0..h/2, with
// A = Z_k + conj Z_{h-k}, B = -i (Z_k - conj Z_{h-k}) (twice the transforms
// of the even and odd points), T = w^k B:
//   X_k = A + T,  X_{h-k} = conj(A - T)      (twice the slab's modes; k = 0
//                                             gives X_0 and X_h)
//   Y = S X;  A' = Y_k + conj Y_{h-k},  B' = (Y_k - conj Y_{h-k}) conj(w^k)
//   Z'_k = A' + i B',  Z'_{h-k} = conj(A') + i conj(B')
// Pair t < h/2 is the mode k = bitrev(2t) < h/2 held at the even position 2t
// (its partner's positions then run contiguously too, so neither access
// meets more than two-way bank conflicts); pair h/2 is the mode h/2 itself.
// spec[3t..3t+2] = w^k, S_k, S_{h-k} of pair t.
__device__ __forceinline__ void spectral_multiply(zc64* z, const zc64* __restrict__ spec, int h, int logh) {
  for (int t = threadIdx.x; t <= (h >> 1); t += blockDim.x) {
    const int pk = t < (h >> 1) ? 2 * t : 1;
    const int k = bitrev_n(pk, logh);
    const int hk = (h - k) & (h - 1);
    const int ph = bitrev_n(hk, logh);
    const zc64 a = z[pk], b = z[ph];
    const zc64 w = ldz(spec + 3 * t), Sk = ldz(spec + 3 * t + 1), Sh = ldz(spec + 3 * t + 2);
    const zc64 A = {a.re + b.re, a.im - b.im};
    const zc64 B = {a.im + b.im, b.re - a.re};
    const zc64 T = zmul(w, B);
    const zc64 Yk = zmul(Sk, zc64{A.re + T.re, A.im + T.im});
    const zc64 Yh = zmul(Sh, zc64{A.re - T.re, T.im - A.im});
    const zc64 Ap = {Yk.re + Yh.re, Yk.im - Yh.im};
    const zc64 Bp = zmulc(zc64{Yk.re - Yh.re, Yk.im + Yh.im}, w);
    z[pk] = {Ap.re - Bp.im, Ap.im + Bp.re};
    if (k != 0 && hk != k) z[ph] = {Ap.re + Bp.im, Bp.re - Ap.im};
  }
}

// One CTA per interval j = blockIdx.x + 1.  Shared memory: the slab as h
// complex values (nx doubles), then the FP32 residual slab (padded); the
// second FP32 slab of the residual pass reuses the complex buffer.  The host
// checks the conditions (periodic, no right-hand side, FCF, MIXED with FP32
// residual storage, nx = 2^p, 16-byte aligned rows).
template <int R, int SPAN>
__global__ void __launch_bounds__(256) fcf_fourier_kernel(const FcfArgs a, const DevTaps t,
                                                          const zc64* __restrict__ tw,
                                                          const zc64* __restrict__ spec, int logh) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int nx = a.nx, h = nx >> 1, j = blockIdx.x + 1;
  zc64* z = reinterpret_cast<zc64*>(smraw);
  float* f0 = reinterpret_cast<float*>(smraw + (size_t)nx * sizeof(double));
  float* f1 = reinterpret_cast<float*>(smraw);
  const double2* start = reinterpret_cast<const double2*>(a.u_old + (long long)(j - 1) * a.cstride);
  const double* oldj = a.u_old + (long long)j * a.cstride;
  prefetch_l2(oldj, (long long)nx * sizeof(double));
  int nz = 0;
  for (int q = threadIdx.x; q < h; q += blockDim.x) {
    const double2 v = __ldcg(start + q);
    z[q] = {v.x, v.y};
    nz |= dnz(v.x) | dnz(v.y);
  }
  // a zero slab maps to zero: the transforms are skipped
  if (__syncthreads_or(nz)) {
    dif_forward(z, tw, h, logh);
    spectral_multiply(z, spec, h, logh);
    __syncthreads();
    dit_inverse(z, tw, h, logh);
  }
  const double* v = reinterpret_cast<const double*>(z);
  double* cn = a.c_new + (long long)j * nx;
  nz = 0;
  for (int e = 2 * threadIdx.x; e < nx; e += 2 * blockDim.x) {
    const double2 old = __ldcg(reinterpret_cast<const double2*>(oldj + e));
    const double v0 = v[e], v1 = v[e + 1];
    *reinterpret_cast<double2*>(cn + e) = make_double2(v0, v1);
    const float r0 = (float)(v0 - old.x), r1 = (float)(v1 - old.y);
    const int q = pidx(e);
    f0[q] = r0;
    f0[q + 1] = r1;
    nz |= (r0 != 0.0f) | (r1 != 0.0f);
  }
  const bool run2 = __syncthreads_or(nz);
  if (j >= a.N) return;
  float* x0 = f0;
  float* x1 = f1;
  if (run2) {
    slab_step_fx<float, R, SPAN, false>(t, a.fx, x0, x1, kNoGf, nx);
    __syncthreads();
    x0 = f1;
  }
  store_residual_f32(a, j, x0);
}

// Fourier FCF tables (FP64): tw[k] = w^k, k = 0..nx/8 (the quarter table of
// w = exp(-2 pi i / nx)), and spec[3t..3t+2] = w^k, scale S_k, scale S_{h-k}
// for pair t = 0..nx/4 of spectral_multiply (k = bitrev(2t), or nx/4 for the
// last), S_k = sum_q c_q exp(+2 pi i o_q k / nx).
__device__ __forceinline__ zc64 stencil_symbol(const DevTaps& t, int k, int nx, double scale) {
  double re = 0.0, im = 0.0, s, c;
  for (int q = 0; q < t.n; ++q) {
    long long ik = ((long long)t.off[q] * k) % nx;
    if (ik < 0) ik += nx;
    sincospi(2.0 * (double)ik / nx, &s, &c);
    re = fma(t.c64[q], c, re);
    im = fma(t.c64[q], s, im);
  }
  return {re * scale, im * scale};
}
__global__ void __launch_bounds__(256) fourier_tables_kernel(const DevTaps t, int nx, int logh, double scale,
                                                             zc64* __restrict__ tw, zc64* __restrict__ spec) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int h = nx / 2;
  double s, c;
  if (i <= h / 4) {
    sincospi(-2.0 * i / nx, &s, &c);
    tw[i] = {c, s};
  }
  if (i <= h / 2) {
    const int k = i < h / 2 ? bitrev_n(2 * i, logh) : h / 2;
    sincospi(-2.0 * k / nx, &s, &c);
    spec[3 * i] = {c, s};
    spec[3 * i + 1] = stencil_symbol(t, k, nx, scale);
    spec[3 * i + 2] = stencil_symbol(t, h - k, nx, scale);
  }
}

// ----------------------------------------------------------------------------
// Sequential march on one thread-block cluster, in a frame that moves with the
// stencil: the shared buffers hold B_n[x] = u_n[(x + S_n) mod nx] with
// S_n = -n*sigma, sigma the centre of the stencil's offsets, so that
// B_n[x] = sum_k c_k B_{n-1}[x + off_k - sigma] + g_n[x + S_n] needs halos of
// the stencil's width only, not of its (characteristic) shift.  CTA `rank`
// owns frame positions [rank*w, min((rank+1)*w, nx)), w = ceil(nx/cs); its buffer holds
// [left halo | own | right halo].  Per step: compute, cluster barrier, pull
// halos from the owners' shared memory (DSMEM), block barrier.  Two buffers
// alternate so a neighbour's reads of step n never meet its writes of n+1.
// The next step's g and c_add values are loaded one step ahead.
// ----------------------------------------------------------------------------
__device__ __forceinline__ int modnx(long long v, int nx) {
  long long r = v % nx;
  return (int)(r < 0 ? r + nx : r);
}

template <int PPT, bool TR = false>
__device__ __forceinline__ void march_body(const MarchArgs& a, const DevTaps& t, unsigned char* smraw,
                                           cg::cluster_group& cl) {
  const int cs = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  // CTAs own w = ceil(nx / cs) positions each, the last one the remainder
  const int nx = a.nx, w = (nx + cs - 1) / cs, base = rank * w, own = min(w, nx - base);
  const int sigma = t.shift;
  const int L = sigma - t.lo, R = t.hi - sigma, W = L + w + R;
  double* B0 = reinterpret_cast<double*>(smraw);
  double* B1 = B0 + W;
  const int tid = threadIdx.x, bs = blockDim.x;
  for (int k = tid; k < L + own + R; k += bs) {
    const int gi = modnx((long long)base - L + k, nx);
    B0[k] = a.init ? a.init[gi] : 0.0;
  }
  __syncthreads();
  // next step's right-hand side and C-points, loaded one step ahead (an FP32
  // right-hand side stays FP32 until it is used, so the load is not waited on)
  double gq[PPT], cq[PPT];
  float gqf[PPT];
  df64 cqd[PPT];
#pragma unroll
  for (int p = 0; p < PPT; ++p) { gq[p] = 0.0; cq[p] = 0.0; gqf[p] = 0.0f; cqd[p] = {0.0f, 0.0f}; }
  auto prefetch = [&](int n, int Sn) {
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
      const int i = tid + p * bs;
      if (i < own) {
        const long long o = (long long)n * nx + wrapi(base + i + Sn, nx);
        if (a.g_f) gqf[p] = __ldcg(a.g_f + o);
        else if (a.g) gq[p] = __ldcg(a.g + o);
        if (a.c_add && a.c_add_df) {
          const float2 v = __ldcg(reinterpret_cast<const float2*>(a.c_add) + o);
          cqd[p] = {v.x, v.y};
        } else if (a.c_add) {
          cq[p] = __ldcg(a.c_add + o);
        }
      }
    }
  };
  int S = modnx(-(long long)sigma, nx);  // S_1
  if (a.P > 1) prefetch(1, S);
  for (int n = 1; n < a.P; ++n) {
    double* cur = (n & 1) ? B0 : B1;
    double* nxt = (n & 1) ? B1 : B0;
    double gc[PPT], cc[PPT];
    df64 ccd[PPT];
#pragma unroll
    for (int p = 0; p < PPT; ++p) { gc[p] = a.g_f ? f32_to_f64(gqf[p]) : gq[p]; cc[p] = cq[p]; ccd[p] = cqd[p]; }
    const int Snext = modnx((long long)S - sigma, nx);
    if (n + 1 < a.P) prefetch(n + 1, Snext);
    const bool store = (a.u_out || a.u_out_f) && (n % a.store_every) == 0;
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
      const int i = tid + p * bs;
      if (i < own) {
        double acc = gc[p];
        const double* c = cur + L + i - sigma;
        const int gi = wrapi(base + i + S, nx);
        if constexpr (TR) {  // truncated stencil: the taps whose column gi + off leaves 0..nx-1 drop out
          for (int k = 0; k < t.n; ++k)
            if ((unsigned)(gi + t.off[k]) < (unsigned)nx) acc = fma(t.c64[k], c[t.off[k]], acc);
        } else {
          for (int k = 0; k < t.n; ++k) acc = fma(t.c64[k], c[t.off[k]], acc);
        }
        nxt[L + i] = acc;
        if (a.c_add && a.c_add_df) {  // float-float C-points: c + e in FP64, split back
          reinterpret_cast<df64*>(a.c_add)[(long long)n * nx + gi] = df_from(df_to(ccd[p]) + acc);
        } else if (a.c_add) {
          a.c_add[(long long)n * nx + gi] = cc[p] + acc;
        }
        if (store) {
          const long long o = (long long)(n / a.store_every) * nx + gi;
          if (a.u_out_f) a.u_out_f[o] = (float)acc;
          else a.u_out[o] = acc;
        }
      }
    }
    cl.sync();
    for (int k = tid; k < L + R; k += bs) {
      int dst, fi;
      if (k < L) { dst = k; fi = base - L + k; }
      else { dst = own + k; fi = base + own + (k - L); }
      fi = modnx(fi, nx);
      const int owner = fi / w, loc = fi - owner * w;
      const double* rem = cl.map_shared_rank(nxt, owner);
      nxt[dst] = rem[L + loc];
    }
    __syncthreads();
    S = Snext;
  }
  cl.sync();  // no CTA leaves while a neighbour may still read its shared memory
}

template <int PPT, bool TR>
__global__ void __launch_bounds__(256) march_kernel(const MarchArgs a, const DevTaps t) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cg::cluster_group cl = cg::this_cluster();
  march_body<PPT, TR>(a, t, smraw, cl);
}

// Batched two-level coarse solve: cluster c marches solve ids[c] with its
// coarse stencil and adds e_j into its new C-points.
template <int PPT>
__global__ void __launch_bounds__(256) march_batched_kernel(const BatchSolve* __restrict__ S,
                                                             const int* __restrict__ ids,
                                                             const DevTaps* __restrict__ taps) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ __align__(16) DevTaps st;
  cg::cluster_group cl = cg::this_cluster();
  const int c = blockIdx.x / (int)cl.num_blocks();
  const BatchSolve* s = S + ids[c];
  const int* src = reinterpret_cast<const int*>(taps + s->psi);
  int* dst = reinterpret_cast<int*>(&st);
  for (int k = threadIdx.x; k < (int)(sizeof(DevTaps) / sizeof(int)); k += blockDim.x) dst[k] = src[k];
  __syncthreads();
  MarchArgs a = {};
  a.init = nullptr;
  a.g = s->fcf.r;
  a.g_f = s->fcf.r_f;
  a.u_out = nullptr;
  a.store_every = 1;
  a.c_add = s->fcf.c_new;
  a.c_add_df = s->fcf.df_store;
  a.nx = s->fcf.nx;
  a.P = s->fcf.N + 1;
  march_body<PPT>(a, st, smraw, cl);
}

// ----------------------------------------------------------------------------
// Correction + F-relaxation of a level (ideal interpolation).
// ----------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ const T* pick(const double* d, const float* f) {
  if constexpr (std::is_same<T, float>::value) return f;
  else return d;
}
template <typename T>
__device__ __forceinline__ T* pick(double* d, float* f) {
  if constexpr (std::is_same<T, float>::value) return f;
  else return d;
}

// Storage of the level in T: FP64 fields for T = double, FP32 fields for
// T = float (FP32 coarse levels).
template <typename T, int R, bool TR = false>
__global__ void __launch_bounds__(R == 8 ? 512 : 1024) correct_kernel(const CorrectArgs a, const DevTaps t) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int nx = a.nx, m = a.m, j = blockIdx.x + 1, plen = padded_len(nx);
  const T* cnew = pick<T>(a.c_new, a.c_new_f);
  const T* e = pick<T>(a.e, a.e_f);
  const T* gg = pick<T>(a.g, a.g_f);
  T* u = pick<T>(a.u, a.u_f);
  T* b0 = reinterpret_cast<T*>(smraw);
  T* b1 = b0 + plen;
  const long long p0 = (long long)(j - 1) * m;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) {
    const T v = cnew[(long long)(j - 1) * nx + i] + (e ? e[(long long)(j - 1) * nx + i] : (T)0);
    b0[pidx(i)] = v;
    u[p0 * nx + i] = v;
  }
  __syncthreads();
  for (int s = 1; s < m; ++s) {
    const T* g = gg ? gg + (p0 + s) * nx : nullptr;
    slab_step_fx<T, R, 0, TR>(t, a.fx, b0, b1, g, nx);
    __syncthreads();
    for (int i = threadIdx.x; i < nx; i += blockDim.x) u[(p0 + s) * nx + i] = b1[pidx(i)];
    T* tmp = b0; b0 = b1; b1 = tmp;
  }
  if (j == a.N)
    for (int i = threadIdx.x; i < nx; i += blockDim.x)
      u[(long long)a.N * m * nx + i] = cnew[(long long)a.N * nx + i] + (e ? e[(long long)a.N * nx + i] : (T)0);
}

// Self-check of f32_to_f64 against the conversion instruction over n hashed
// binary32 bit patterns (the SplitMix64 finaliser of Steele, Lea and Flood,
// OOPSLA 2014, applied to seed and index; every class of value: zeros,
// subnormals, normals, infinities, NaNs).  Counts the patterns whose results
// differ bitwise.
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}
__global__ void __launch_bounds__(256) conversion_check_kernel(unsigned long long n, unsigned long long seed,
                                                               unsigned long long* bad) {
  unsigned long long local = 0;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n; i += stride) {
    const unsigned long long h = mix64(seed ^ mix64(i + 1));
    for (int q = 0; q < 2; ++q) {
      unsigned u = (unsigned)(h >> (32 * q));
      if (((h >> 8) & 7ull) == 0) u &= 0x807fffffu;  // exponent field 0: zeros and subnormals
      const float f = __uint_as_float(u);
      if (__double_as_longlong(f32_to_f64(f)) != __double_as_longlong((double)f)) ++local;
    }
  }
  if (local) atomicAdd(bad, local);
}

cudaError_t launch_conversion_check(unsigned long long n, unsigned long long seed, unsigned long long* bad,
                                    cudaStream_t s) {
  conversion_check_kernel<<<152 * 8, 256, 0, s>>>(n, seed, bad);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(1024) norm_kernel(const double* __restrict__ partial, int n, double* out) {
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += partial[i];
  v = block_sum(v);
  if (threadIdx.x == 0) out[0] = v;
}

__global__ void __launch_bounds__(1024) norm_batched_kernel(const BatchSolve* __restrict__ S,
                                                            const int* __restrict__ ids, double* out) {
  const BatchSolve* s = S + ids[blockIdx.x];
  const double* partial = s->fcf.partial;
  double v = 0.0;
  const int n = s->fcf.N + (s->fcf.relax_f ? 1 : 0);  // F-relaxation: residuals 1..N
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += partial[i];
  v = block_sum(v);
  if (threadIdx.x == 0) out[blockIdx.x] = v;
}

// Value-form residual: r_{j+1} = Phi^m c_new_j - c_new_{j+1} (r row j+1 holds
// Phi^m c_new_j) and its squared norm into partial[j]; one CTA per row.
__device__ __forceinline__ void residual_value_row(const double* c_new, double* r, double* partial, int nx, int j) {
  const double* cn = c_new + (long long)(j + 1) * nx;
  double* rr = r + (long long)(j + 1) * nx;
  double ss = 0.0;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) {
    const double v = rr[i] - cn[i];
    rr[i] = v;
    ss = fma(v, v, ss);
  }
  if (partial) {
    ss = block_sum(ss);
    if (threadIdx.x == 0) partial[j] = ss;
  }
}
__global__ void __launch_bounds__(512) residual_value_kernel(const double* __restrict__ c_new, double* r,
                                                             double* partial, int nx) {
  residual_value_row(c_new, r, partial, nx, blockIdx.x + 1);
}
__global__ void __launch_bounds__(512) residual_value_batched_kernel(const BatchSolve* __restrict__ S,
                                                                     const BatchItem* __restrict__ items) {
  const BatchItem it = items[blockIdx.x];
  const FcfArgs& a = S[it.solve].fcf;
  if (!a.value_residual || it.j >= a.N) return;
  residual_value_row(a.c_new, a.r, a.partial, a.nx, it.j);
}

__global__ void add_kernel(double* __restrict__ c, const double* __restrict__ e, long long count) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    c[i] += e[i];
}

// c += e (level-1 correction from the FP32 level-2 array), two points per
// thread and step (16-byte and 8-byte accesses) where both arrays allow it.
__global__ void add_f_kernel(double* __restrict__ c, const float* __restrict__ e, long long count) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const bool pairs = ((reinterpret_cast<unsigned long long>(c) | reinterpret_cast<unsigned long long>(e)) & 15ull) == 0;
  long long done = 0;
  if (pairs) {
    const long long n2 = count / 2;
    for (long long i = t0; i < n2; i += stride) {
      const float2 v = reinterpret_cast<const float2*>(e)[i];
      double2 w = reinterpret_cast<double2*>(c)[i];
      w.x += f32_to_f64(v.x);
      w.y += f32_to_f64(v.y);
      reinterpret_cast<double2*>(c)[i] = w;
    }
    done = 2 * n2;
  }
  for (long long i = done + t0; i < count; i += stride) c[i] += f32_to_f64(e[i]);
}

// Float-float C-points: c += e on the FP32 pipes; conversions to and from FP64.
__global__ void add_df_f_kernel(df64* __restrict__ c, const float* __restrict__ e, long long count) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    c[i] = df_add_f(c[i], e[i]);
}
__global__ void f64_to_df_kernel(const double* __restrict__ in, df64* __restrict__ out, long long count) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = df_from(in[i]);
}
__global__ void df_to_f64_kernel(const df64* __restrict__ in, double* __restrict__ out, long long count) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = df_to(in[i]);
}

template <int R, bool TR = false>
__global__ void __launch_bounds__(R == 8 ? 512 : 1024) propagate_kernel(const double* in, double* out, int nx, int k,
                                                         const DevTaps t, double* partial, const Fixup fx) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int plen = padded_len(nx);
  double* b0 = reinterpret_cast<double*>(smraw);
  double* b1 = b0 + plen;
  const long long v = blockIdx.x;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) b0[pidx(i)] = in[v * nx + i];
  __syncthreads();
  for (int s = 0; s < k; ++s) {
    slab_step_fx<double, R, 0, TR>(t, fx, b0, b1, kNoG, nx);
    __syncthreads();
    double* tmp = b0; b0 = b1; b1 = tmp;
  }
  double ss = 0.0;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) {
    const double x = b0[pidx(i)];
    out[v * nx + i] = x;
    ss = fma(x, x, ss);
  }
  if (partial) {
    ss = block_sum(ss);
    if (threadIdx.x == 0) partial[v] = ss;
  }
}

// ----------------------------------------------------------------------------
// Stopping test inside a graph (one thread): relative residual, history, and
// the WHILE (keep cycling) / IF (apply this cycle's coarse correction)
// conditions.  Same decisions, in the same order, as the host loop.
// ----------------------------------------------------------------------------
__global__ void check_kernel(const double* __restrict__ norm2, CheckState* st, cudaGraphConditionalHandle hw,
                             cudaGraphConditionalHandle hif, int cur) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double r0 = sqrt(st->r0sq);
  const double rel = !isfinite(r0) ? r0 : (r0 > 0.0 ? sqrt(norm2[0]) / r0 : 0.0);
  if (st->nhist < 128) st->hist[st->nhist++] = rel;
  st->rel = rel;
  int stop = 0;
  if (!isfinite(rel) || (st->diverge > 0.0 && rel > st->diverge)) { st->status = -5; stop = 1; }
  else if (rel <= st->tol) { st->status = 0; stop = 1; }
  else if (st->it >= st->max_iter) { st->status = -4; stop = 1; }
  if (stop) {
    st->done = 1;
    st->result_cur = cur;
    cudaGraphSetConditional(hif, 0);
    cudaGraphSetConditional(hw, 0);
  } else {
    st->it += 1;
    cudaGraphSetConditional(hif, 1);
  }
}

// ------------------------------------------------------------------ launches

cudaError_t launch_check(const double* norm2, CheckState* st, unsigned long long while_handle,
                         unsigned long long if_handle, int cur, cudaStream_t s) {
  check_kernel<<<1, 32, 0, s>>>(norm2, st, (cudaGraphConditionalHandle)while_handle,
                                (cudaGraphConditionalHandle)if_handle, cur);
  return cudaGetLastError();
}

static int g_tile = 8;  // register tile of the stencil (0 = one tap at a time)
// fused float-float FCF (MGRIT_FCF_STREAM): 1 register-resident runs of
// intervals per CTA with cp.async prefetch (default, upwind stencils); 4
// register-resident, one interval per CTA; 0 one interval per CTA with the slab
// in shared memory; 2, 3 runs with the slabs in shared memory (through
// registers or cp.async)
static int g_stream_fused = 1;
void set_stream_fused(int mode) { g_stream_fused = mode >= 0 && mode <= 4 ? mode : 1; }

void set_tile(int r) { g_tile = (r == 4 || r == 8) ? r : 0; }
int get_tile() { return g_tile; }

static int tile_for(const DevTaps& t, int nx) { return (t.span > 0 && nx >= 64) ? g_tile : 0; }

static int threads_for(int nx, int R, int hint);
int default_threads(int nx, int R) { return threads_for(nx, R, 0); }
int default_tile(const DevTaps& t, int nx) { return (t.span > 0 && nx >= 64) ? g_tile : 0; }

static int threads_for(int nx, int R, int hint) {
  const int cap = 512;
  if (hint > 0) return hint < cap ? hint : cap;
  if (R == kFixedTile || R == kChunkTile) R = 8;
  const int per = R > 0 ? R : 4;
  int th = (nx + per - 1) / per;
  th = ((th + 31) / 32) * 32;
  return th < 32 ? 32 : (th > cap ? cap : th);
}

template <typename K>
static cudaError_t set_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024) return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  return cudaSuccess;
}

template <int PREC, int R, int SPAN = 0, bool TR = false>
static cudaError_t launch_fcf_t(const FcfArgs& a, const DevTaps& t, int threads, cudaStream_t s) {
  const size_t smem = 2 * (size_t)padded_len(a.nx) * (PREC == 2 ? sizeof(float) : sizeof(double));
  cudaError_t e = set_smem(fcf_kernel<PREC, R, SPAN, TR>, smem);
  if (e != cudaSuccess) return e;
  FcfArgs f = a;
  f.fused = 0;  // two full slabs: the general body
  fcf_kernel<PREC, R, SPAN, TR><<<a.N, threads_for(a.nx, R, threads), smem, s>>>(f, t);
  return cudaGetLastError();
}

// Fixed-span instantiations: the collapsed ERK1..ERK5 stencils (spans
// s(w-1)+1 = 2, 5, 10, 17, 31).
static bool fixed_span_ok(int span) {
  return span == 2 || span == 5 || span == 10 || span == 17 || span == 31;
}

// The fused narrow-stencil body of precision 3 (see fcf_body_df_fused): the
// host checks every condition the body assumes, then launches with one
// float-float and one FP32 slab of shared memory.
static bool host_fused_ok(const FcfArgs& a, const DevTaps& t, int threads) {
  auto al = [](const void* p) { return (reinterpret_cast<unsigned long long>(p) & 15ull) == 0; };
  return t.span > 0 && t.span <= 5 && a.df_store && a.m == 1 && a.fx.nl + a.fx.nr == 0 && !a.relax_f && !a.trunc &&
         a.r_f && !a.g && threads > 0 && a.nx % (8 * threads) == 0 && al(a.u_old) && al(a.c_new) && al(a.r_f) &&
         (a.cstride & 1) == 0;
}

static int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) !=
                                                 cudaSuccess || n < 1) {
      cudaGetLastError();
      n = 152;
    }
  }
  return n;
}

// Shared memory of the streaming fused body: two float-float slabs and one
// FP32 slab, padded.
static size_t stream_smem(int nx) { return (size_t)padded_len(nx) * (2 * sizeof(double) + sizeof(float)); }

// The streaming fused body: two CTAs per SM where their slabs fit (one for
// nx above about 5000), each a balanced run of intervals, 512 threads (or
// fewer, so that nx is a multiple of 8 per thread).
template <int SPAN>
static cudaError_t launch_fcf_stream(const FcfArgs& a, const DevTaps& t, cudaStream_t s) {
  int th = 512;
  while (th > 32 && a.nx % (8 * th) != 0) th >>= 1;
  if (a.nx % (8 * th) != 0) return cudaErrorInvalidValue;
  const size_t smem = stream_smem(a.nx);
  auto kern = g_stream_fused == 3 ? fcf_df_stream_kernel<SPAN, true> : fcf_df_stream_kernel<SPAN, false>;
  cudaError_t e = set_smem(kern, smem);
  if (e != cudaSuccess) return e;
  const int per_sm = 2 * smem <= (size_t)kMaxSmemBytes ? 2 : 1;
  const int grid = a.N < per_sm * sm_count() ? a.N : per_sm * sm_count();
  kern<<<grid, th, smem, s>>>(a, t);
  return cudaGetLastError();
}

// The register-resident run (fcf_regrun_kernel): an upwind stencil of SPAN
// taps ending at the output point, nx / 8 threads of eight points each, three
// slabs and the rho-tail slots in shared memory; persistent grid of as many
// CTAs as fit on the SMs (at 64 registers per thread), at most one per
// interval.
template <int SPAN>
static bool regrun_shape_ok(const FcfArgs& a, const DevTaps& t) {
  return t.lo == -(SPAN - 1) && t.hi == 0 && a.nx % 256 == 0 && a.nx / 8 <= 1024;
}
static size_t regrun_smem(int nx) { return 3 * (size_t)nx * sizeof(double) + 2 * (size_t)(nx / 8) * sizeof(float4); }
template <int SPAN, typename V>
static cudaError_t launch_regrun(const FcfArgs& a, const DevTaps& t, cudaStream_t s) {
  const size_t rsmem = regrun_smem(a.nx);
  cudaError_t e = set_smem(fcf_regrun_kernel<SPAN, V>, rsmem);
  if (e != cudaSuccess) return e;
  const int th = a.nx / 8;
  int per_sm = (int)((228 * 1024) / (rsmem + 1024));                // shared memory per SM
  per_sm = per_sm < 2048 / th ? per_sm : 2048 / th;                  // threads per SM
  per_sm = per_sm < 65536 / (64 * th) ? per_sm : 65536 / (64 * th);  // 64 registers per thread
  per_sm = per_sm < 1 ? 1 : per_sm;
  const int grid = a.N < per_sm * sm_count() ? a.N : per_sm * sm_count();
  fcf_regrun_kernel<SPAN, V><<<grid, th, rsmem, s>>>(a, t);
  return cudaGetLastError();
}

template <int SPAN>
static cudaError_t launch_fcf_fused(const FcfArgs& a, const DevTaps& t, int threads, cudaStream_t s) {
  const bool upwind = regrun_shape_ok<SPAN>(a, t);
  if (g_stream_fused == 1 && upwind && regrun_smem(a.nx) <= (size_t)kMaxSmemBytes) {
    return launch_regrun<SPAN, df64>(a, t, s);
  }
  if (g_stream_fused == 4 && upwind) {
    fcf_df_reg_kernel<SPAN><<<a.N, a.nx / 8, 0, s>>>(a, t);
    return cudaGetLastError();
  }
  if (g_stream_fused >= 2 && stream_smem(a.nx) <= (size_t)kMaxSmemBytes) return launch_fcf_stream<SPAN>(a, t, s);
  FcfArgs f = a;
  f.fused = 1;
  const size_t smem = (size_t)padded_len(a.nx) * (sizeof(double) + sizeof(float));
  cudaError_t e = set_smem(fcf_kernel<3, 8, SPAN>, smem);
  if (e != cudaSuccess) return e;
  fcf_kernel<3, 8, SPAN><<<a.N, threads, smem, s>>>(f, t);
  return cudaGetLastError();
}

// MIXED (FP64 pass 1, FP32 pass 2 and residual) on the register-resident
// run: the conditions of host_fused_ok with FP64 C-points, and the run's
// shape.
template <int SPAN>
static bool host_regrun_mixed_ok(const FcfArgs& a, const DevTaps& t) {
  auto al = [](const void* p) { return (reinterpret_cast<unsigned long long>(p) & 15ull) == 0; };
  return g_stream_fused == 1 && t.span == SPAN && !a.df_store && a.m == 1 && a.fx.nl + a.fx.nr == 0 &&
         !a.relax_f && !a.trunc && !a.value_residual && a.r_f && !a.g && regrun_shape_ok<SPAN>(a, t) &&
         regrun_smem(a.nx) <= (size_t)kMaxSmemBytes && al(a.u_old) && al(a.c_new) && al(a.r_f) &&
         (a.cstride & 1) == 0;
}

template <int PREC>
static cudaError_t launch_fcf_fixed(const FcfArgs& a, const DevTaps& t, int threads, cudaStream_t s) {
  if constexpr (PREC == 3) {
    const int th = threads_for(a.nx, kFixedTile, threads);
    if (host_fused_ok(a, t, th)) {
      if (t.span == 2) return launch_fcf_fused<2>(a, t, th, s);
      if (t.span == 5) return launch_fcf_fused<5>(a, t, th, s);
    }
  }
  if constexpr (PREC == 1) {
    if (host_regrun_mixed_ok<2>(a, t)) return launch_regrun<2, double>(a, t, s);
    if (host_regrun_mixed_ok<5>(a, t)) return launch_regrun<5, double>(a, t, s);
  }
  switch (t.span) {
    case 2: return launch_fcf_t<PREC, 8, 2>(a, t, threads, s);
    case 5: return launch_fcf_t<PREC, 8, 5>(a, t, threads, s);
    case 10: return launch_fcf_t<PREC, 8, 10>(a, t, threads, s);
    case 17: return launch_fcf_t<PREC, 4, 17>(a, t, threads, s);
    case 31: return launch_fcf_t<PREC, 4, 31>(a, t, threads, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_fcf(const FcfArgs& a, const DevTaps& t, int precision, int threads, cudaStream_t s, int tile) {
  if (a.N < 1) return cudaSuccess;
  if (a.trunc) {  // truncated coarse stencils: FP64 or FP32 levels, sliding window or one tap at a time
    if (tile == kChunkTile || tile == kFixedTile || (precision != 0 && precision != 2)) return cudaErrorInvalidValue;
    const int R = (tile >= 0 && (tile == 0 || (t.span > 0 && a.nx >= 64))) ? tile : tile_for(t, a.nx);
    if (precision == 0) {
      if (R == 8) return launch_fcf_t<0, 8, 0, true>(a, t, threads, s);
      if (R == 4) return launch_fcf_t<0, 4, 0, true>(a, t, threads, s);
      return launch_fcf_t<0, 0, 0, true>(a, t, threads, s);
    }
    if (R == 8) return launch_fcf_t<2, 8, 0, true>(a, t, threads, s);
    if (R == 4) return launch_fcf_t<2, 4, 0, true>(a, t, threads, s);
    return launch_fcf_t<2, 0, 0, true>(a, t, threads, s);
  }
  if (tile == kChunkTile) {
    if (!(t.span > 0) || a.nx < 64) return cudaErrorInvalidValue;
    switch (precision) {
      case 0: return launch_fcf_t<0, 8, kChunked>(a, t, threads, s);
      case 1: return launch_fcf_t<1, 8, kChunked>(a, t, threads, s);
      case 2: return launch_fcf_t<2, 8, kChunked>(a, t, threads, s);
      default: return launch_fcf_t<3, 8, kChunked>(a, t, threads, s);
    }
  }
  if (tile == kFixedTile) {
    if (!fixed_span_ok(t.span) || a.nx < 64) return cudaErrorInvalidValue;
    switch (precision) {
      case 0: return launch_fcf_fixed<0>(a, t, threads, s);
      case 1: return launch_fcf_fixed<1>(a, t, threads, s);
      case 2: return launch_fcf_fixed<2>(a, t, threads, s);
      default: return launch_fcf_fixed<3>(a, t, threads, s);
    }
  }
  const int R = (tile >= 0 && (tile == 0 || (t.span > 0 && a.nx >= 64))) ? tile : tile_for(t, a.nx);
  if (precision == 0) {
    if (R == 8) return launch_fcf_t<0, 8>(a, t, threads, s);
    if (R == 4) return launch_fcf_t<0, 4>(a, t, threads, s);
    return launch_fcf_t<0, 0>(a, t, threads, s);
  }
  if (precision == 2) {
    if (R == 8) return launch_fcf_t<2, 8>(a, t, threads, s);
    if (R == 4) return launch_fcf_t<2, 4>(a, t, threads, s);
    return launch_fcf_t<2, 0>(a, t, threads, s);
  }
  if (precision == 3) {
    if (R == 8) return launch_fcf_t<3, 8>(a, t, threads, s);
    if (R == 4) return launch_fcf_t<3, 4>(a, t, threads, s);
    return launch_fcf_t<3, 0>(a, t, threads, s);
  }
  if (R == 8) return launch_fcf_t<1, 8>(a, t, threads, s);
  if (R == 4) return launch_fcf_t<1, 4>(a, t, threads, s);
  return launch_fcf_t<1, 0>(a, t, threads, s);
}

// ------------------------------------------------- FCF with the FP64 pass in Fourier space
bool fourier_fcf_supported(int nx) {
  return nx >= 256 && nx <= 8192 && (nx & (nx - 1)) == 0 &&
         (size_t)nx * sizeof(double) + (size_t)padded_len(nx) * sizeof(float) <= (size_t)(kMaxSmemBytes - 1024);
}

static int log2_half(int nx) {
  int logh = 0;
  while ((2 << logh) < nx) ++logh;
  return logh;
}
size_t fourier_table_doubles(int nx) { return 2 * (size_t)(nx / 8 + 1) + 6 * (size_t)(nx / 4 + 1); }

cudaError_t launch_fourier_tables(const DevTaps& t, int nx, double* tab, cudaStream_t s) {
  if (!fourier_fcf_supported(nx)) return cudaErrorInvalidValue;
  const int n = nx / 4 + 1;
  fourier_tables_kernel<<<(n + 255) / 256, 256, 0, s>>>(t, nx, log2_half(nx), 1.0 / (2.0 * nx),
                                                        reinterpret_cast<zc64*>(tab),
                                                        reinterpret_cast<zc64*>(tab + 2 * (nx / 8 + 1)));
  return cudaGetLastError();
}

bool fourier_fcf_args_ok(const FcfArgs& a) {
  auto al = [](const void* p) { return (reinterpret_cast<unsigned long long>(p) & 15ull) == 0; };
  return fourier_fcf_supported(a.nx) && a.m == 1 && !a.g && !a.relax_f && !a.value_residual && !a.zero_old &&
         !a.df_store && !a.trunc && a.fx.nl + a.fx.nr == 0 && a.r_f && a.u_old && a.c_new && al(a.u_old) &&
         al(a.c_new) && (a.cstride & 1) == 0;
}

template <int R, int SPAN>
static cudaError_t launch_fourier_t(const FcfArgs& a, const DevTaps& t, const double* tab, int threads,
                                    cudaStream_t s) {
  const size_t smem = (size_t)a.nx * sizeof(double) + (size_t)padded_len(a.nx) * sizeof(float);
  cudaError_t e = set_smem(fcf_fourier_kernel<R, SPAN>, smem);
  if (e != cudaSuccess) return e;
  fcf_fourier_kernel<R, SPAN><<<a.N, threads, smem, s>>>(
      a, t, reinterpret_cast<const zc64*>(tab), reinterpret_cast<const zc64*>(tab + 2 * (a.nx / 8 + 1)),
      log2_half(a.nx));
  return cudaGetLastError();
}

cudaError_t launch_fcf_fourier(const FcfArgs& a, const DevTaps& t, const double* tab, int threads, cudaStream_t s) {
  if (a.N < 1) return cudaSuccess;
  if (!fourier_fcf_args_ok(a) || !tab || (threads != 128 && threads != 256)) return cudaErrorInvalidValue;
  FcfArgs f = a;
  f.fused = 0;
  if (t.span >= 8 && a.nx >= 64) return launch_fourier_t<8, kChunked>(f, t, tab, threads, s);
  if (t.span > 0 && a.nx >= 64) return launch_fourier_t<8, 0>(f, t, tab, threads, s);
  return launch_fourier_t<0, 0>(f, t, tab, threads, s);
}

template <int R, int SPAN = 0>
static cudaError_t launch_fcf_batched_t(const BatchSolve* S, const BatchItem* items, int nitems, const DevTaps* taps,
                                        int max_nx, int threads, cudaStream_t s) {
  const size_t smem = 2 * (size_t)padded_len(max_nx) * sizeof(double);
  cudaError_t e = set_smem(fcf_batched_kernel<R, SPAN>, smem);
  if (e != cudaSuccess) return e;
  fcf_batched_kernel<R, SPAN><<<nitems, threads, smem, s>>>(S, items, taps);
  return cudaGetLastError();
}

cudaError_t launch_fcf_batched(const BatchSolve* S, const BatchItem* items, int nitems, const DevTaps* taps,
                               int max_nx, int threads, int tile, int span, cudaStream_t s) {
  if (nitems < 1) return cudaSuccess;
  if (tile == kChunkTile) return launch_fcf_batched_t<8, kChunked>(S, items, nitems, taps, max_nx, threads, s);
  if (tile == kFixedTile) {
    switch (span) {
      case 2: return launch_fcf_batched_t<8, 2>(S, items, nitems, taps, max_nx, threads, s);
      case 5: return launch_fcf_batched_t<8, 5>(S, items, nitems, taps, max_nx, threads, s);
      case 10: return launch_fcf_batched_t<8, 10>(S, items, nitems, taps, max_nx, threads, s);
      case 17: return launch_fcf_batched_t<4, 17>(S, items, nitems, taps, max_nx, threads, s);
      case 31: return launch_fcf_batched_t<4, 31>(S, items, nitems, taps, max_nx, threads, s);
      default: return cudaErrorInvalidValue;
    }
  }
  if (tile == 8) return launch_fcf_batched_t<8>(S, items, nitems, taps, max_nx, threads, s);
  if (tile == 4) return launch_fcf_batched_t<4>(S, items, nitems, taps, max_nx, threads, s);
  return launch_fcf_batched_t<0>(S, items, nitems, taps, max_nx, threads, s);
}

template <typename K>
static cudaError_t launch_cluster(K kernel, int grid, int cluster, int threads, size_t smem, cudaStream_t s,
                                  void** args) {
  cudaError_t e = set_smem(kernel, smem);
  if (e != cudaSuccess) return e;
  if (cluster > 8) {
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cluster;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, (const void*)kernel, args);
}

template <int PPT>
static cudaError_t launch_march_t(const MarchArgs& a, const DevTaps& t, int cluster, int threads, cudaStream_t s) {
  const int w = (a.nx + cluster - 1) / cluster;
  const size_t smem = 2 * (size_t)(w + t.hi - t.lo) * sizeof(double);
  MarchArgs aa = a;
  DevTaps tt = t;
  void* args[] = {&aa, &tt};
  if (a.trunc) return launch_cluster(march_kernel<PPT, true>, cluster, cluster, threads, smem, s, args);
  return launch_cluster(march_kernel<PPT, false>, cluster, cluster, threads, smem, s, args);
}

cudaError_t launch_march(const MarchArgs& a, const DevTaps& t, int cluster, int threads, cudaStream_t s) {
  const int w = (a.nx + cluster - 1) / cluster;
  const int ppt = (w + threads - 1) / threads;
  if (a.P < 2) return cudaSuccess;
  switch (ppt) {
    case 1: return launch_march_t<1>(a, t, cluster, threads, s);
    case 2: return launch_march_t<2>(a, t, cluster, threads, s);
    case 3: case 4: return launch_march_t<4>(a, t, cluster, threads, s);
    case 5: case 6: case 7: case 8: return launch_march_t<8>(a, t, cluster, threads, s);
    default:
      if (ppt <= 16) return launch_march_t<16>(a, t, cluster, threads, s);
      return cudaErrorInvalidConfiguration;
  }
}

template <int PPT>
static cudaError_t launch_march_batched_t(const BatchSolve* S, const int* ids, int count, const DevTaps* taps,
                                          int cluster, int max_w, int max_halo, cudaStream_t s) {
  const size_t smem = 2 * (size_t)(max_w + max_halo) * sizeof(double);
  const BatchSolve* SS = S;
  const int* ii = ids;
  const DevTaps* tt = taps;
  void* args[] = {&SS, &ii, &tt};
  const int threads = max_w < 256 ? ((max_w + 31) / 32) * 32 : 256;
  return launch_cluster(march_batched_kernel<PPT>, count * cluster, cluster, threads, smem, s, args);
}

cudaError_t launch_march_batched(const BatchSolve* S, const int* ids, int count, const DevTaps* taps, int cluster,
                                 int max_w, int max_halo, cudaStream_t s) {
  if (count < 1) return cudaSuccess;
  const int threads = max_w < 256 ? ((max_w + 31) / 32) * 32 : 256;
  const int ppt = (max_w + threads - 1) / threads;
  switch (ppt) {
    case 1: return launch_march_batched_t<1>(S, ids, count, taps, cluster, max_w, max_halo, s);
    case 2: return launch_march_batched_t<2>(S, ids, count, taps, cluster, max_w, max_halo, s);
    case 3: case 4: return launch_march_batched_t<4>(S, ids, count, taps, cluster, max_w, max_halo, s);
    case 5: case 6: case 7: case 8: return launch_march_batched_t<8>(S, ids, count, taps, cluster, max_w, max_halo, s);
    default:
      if (ppt <= 16) return launch_march_batched_t<16>(S, ids, count, taps, cluster, max_w, max_halo, s);
      return cudaErrorInvalidConfiguration;
  }
}

int march_max_cluster() { return 16; }

template <typename T, int R, bool TR>
static cudaError_t launch_correct_t(const CorrectArgs& a, const DevTaps& t, int threads, cudaStream_t s) {
  const size_t smem = 2 * (size_t)padded_len(a.nx) * sizeof(T);
  cudaError_t e = set_smem(correct_kernel<T, R, TR>, smem);
  if (e != cudaSuccess) return e;
  correct_kernel<T, R, TR><<<a.N, threads_for(a.nx, R, threads), smem, s>>>(a, t);
  return cudaGetLastError();
}

template <bool TR>
static cudaError_t launch_correct_tr(const CorrectArgs& a, const DevTaps& t, int threads, cudaStream_t s, int fp32) {
  const int R = tile_for(t, a.nx);
  if (fp32) {
    if (R == 8) return launch_correct_t<float, 8, TR>(a, t, threads, s);
    if (R == 4) return launch_correct_t<float, 4, TR>(a, t, threads, s);
    return launch_correct_t<float, 0, TR>(a, t, threads, s);
  }
  if (R == 8) return launch_correct_t<double, 8, TR>(a, t, threads, s);
  if (R == 4) return launch_correct_t<double, 4, TR>(a, t, threads, s);
  return launch_correct_t<double, 0, TR>(a, t, threads, s);
}

cudaError_t launch_correct(const CorrectArgs& a, const DevTaps& t, int threads, cudaStream_t s, int fp32) {
  if (a.N < 1) return cudaSuccess;
  if (a.trunc) return launch_correct_tr<true>(a, t, threads, s, fp32);
  return launch_correct_tr<false>(a, t, threads, s, fp32);
}

cudaError_t launch_residual_value(const double* c_new, double* r, double* partial, int nx, int N, cudaStream_t s) {
  if (N < 2) return cudaSuccess;
  residual_value_kernel<<<N - 1, nx >= 512 ? 512 : ((nx + 31) / 32) * 32, 0, s>>>(c_new, r, partial, nx);
  return cudaGetLastError();
}

cudaError_t launch_residual_value_batched(const BatchSolve* S, const BatchItem* items, int nitems, cudaStream_t s) {
  if (nitems < 1) return cudaSuccess;
  residual_value_batched_kernel<<<nitems, 256, 0, s>>>(S, items);
  return cudaGetLastError();
}

cudaError_t launch_norm(const double* partial, int n, double* out, cudaStream_t s) {
  norm_kernel<<<1, 1024, 0, s>>>(partial, n, out);
  return cudaGetLastError();
}

cudaError_t launch_norm_batched(const BatchSolve* S, const int* ids, int count, double* out, cudaStream_t s) {
  if (count < 1) return cudaSuccess;
  norm_batched_kernel<<<count, 256, 0, s>>>(S, ids, out);
  return cudaGetLastError();
}

cudaError_t launch_add(double* c, const double* e, long long count, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  long long blocks = (count + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  add_kernel<<<(int)blocks, 256, 0, s>>>(c, e, count);
  return cudaGetLastError();
}

cudaError_t launch_add_f(double* c, const float* e, long long count, cudaStream_t s, int df_store) {
  if (count <= 0) return cudaSuccess;
  long long blocks = (count + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (df_store) add_df_f_kernel<<<(int)blocks, 256, 0, s>>>(reinterpret_cast<df64*>(c), e, count);
  else add_f_kernel<<<(int)blocks, 256, 0, s>>>(c, e, count);
  return cudaGetLastError();
}

cudaError_t launch_convert_df(const double* in, double* out, long long count, int to_df, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  long long blocks = (count + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (to_df) f64_to_df_kernel<<<(int)blocks, 256, 0, s>>>(in, reinterpret_cast<df64*>(out), count);
  else df_to_f64_kernel<<<(int)blocks, 256, 0, s>>>(reinterpret_cast<const df64*>(in), out, count);
  return cudaGetLastError();
}

// ------------------------------------------------- random initial iterate

// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32 x 32 -> 64-bit
// products with the key bumped by the Weyl constants between rounds.
__device__ __forceinline__ double philox_unit(unsigned long long seed, unsigned int i, unsigned int n) {
  unsigned int c0 = i, c1 = n, c2 = 0u, c3 = 0u;
  unsigned int k0 = (unsigned int)seed, k1 = (unsigned int)(seed >> 32);
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned int lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
    const unsigned int lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
    const unsigned int n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  const unsigned long long bits = ((unsigned long long)(c0 >> 5) << 26) | (unsigned long long)(c1 >> 6);
  return (double)bits * 0x1.0p-53;
}

__global__ void random_rows_kernel(double* __restrict__ out, const double* __restrict__ u0, int nx,
                                   long long first_n, long long stride_n, unsigned long long seed) {
  const long long k = blockIdx.y;
  const long long n = first_n + k * stride_n;
  double* row = out + k * nx;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nx; i += gridDim.x * blockDim.x)
    row[i] = n == 0 ? u0[i] : philox_unit(seed, (unsigned int)i, (unsigned int)n);
}

__global__ void __launch_bounds__(256) random_residual_kernel(const double* __restrict__ phi_u,
                                                              double* __restrict__ partial, int nx,
                                                              long long first_n, unsigned long long seed) {
  const long long k = blockIdx.x;
  const unsigned int n = (unsigned int)(first_n + k + 1);
  const double* row = phi_u + k * nx;
  double ss = 0.0;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) {
    const double d = row[i] - philox_unit(seed, (unsigned int)i, n);
    ss = fma(d, d, ss);
  }
  ss = block_sum(ss);
  if (threadIdx.x == 0) partial[k] = ss;
}

__global__ void __launch_bounds__(1024) accumulate_kernel(const double* __restrict__ partial, int n, double* acc,
                                                          int first) {
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += partial[i];
  v = block_sum(v);
  if (threadIdx.x == 0) acc[0] = first ? v : acc[0] + v;
}

__global__ void state_init_kernel(CheckState* st, double tol, int max_iter, double diverge, double r0sq) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  st->r0sq = r0sq;
  st->tol = tol;
  st->max_iter = max_iter;
  st->it = 0;
  st->done = 0;
  st->status = 0;
  st->result_cur = 0;
  st->nhist = 0;
  st->rel = 0.0;
  st->diverge = diverge;
}

__global__ void result_rows_kernel(const CheckState* __restrict__ st, const double* c0, const double* c1,
                                   double* __restrict__ out, long long first, long long count, int df) {
  const double* src = (st->result_cur == 0 ? c1 : c0) + first;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = df ? df_to(reinterpret_cast<const df64*>(src)[i]) : src[i];
}

cudaError_t launch_random_rows(double* out, const double* u0, int nx, long long first_n, long long stride_n,
                               int rows, unsigned long long seed, cudaStream_t s) {
  const int bx = (nx + 255) / 256 < 8 ? (nx + 255) / 256 : 8;
  for (int k0 = 0; k0 < rows; k0 += 65535) {  // gridDim.y <= 65535
    const int r = rows - k0 < 65535 ? rows - k0 : 65535;
    random_rows_kernel<<<dim3(bx, r), 256, 0, s>>>(out + (long long)k0 * nx, u0, nx, first_n + k0 * stride_n,
                                                   stride_n, seed);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_random_residual(const double* phi_u, double* partial, int nx, long long first_n, int rows,
                                   unsigned long long seed, cudaStream_t s) {
  if (rows < 1) return cudaSuccess;
  random_residual_kernel<<<rows, 256, 0, s>>>(phi_u, partial, nx, first_n, seed);
  return cudaGetLastError();
}

cudaError_t launch_accumulate(const double* partial, int n, double* acc, int first, cudaStream_t s) {
  accumulate_kernel<<<1, 1024, 0, s>>>(partial, n, acc, first);
  return cudaGetLastError();
}

cudaError_t launch_state_init(CheckState* st, double tol, int max_iter, double diverge, double r0sq, cudaStream_t s) {
  state_init_kernel<<<1, 32, 0, s>>>(st, tol, max_iter, diverge, r0sq);
  return cudaGetLastError();
}

cudaError_t launch_result_rows(const CheckState* st, const double* c0, const double* c1, double* out, int nx,
                               long long row0, long long rows, int df, cudaStream_t s) {
  const long long count = rows * nx;
  if (count <= 0) return cudaSuccess;
  long long blocks = (count + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  result_rows_kernel<<<(int)blocks, 256, 0, s>>>(st, c0, c1, out, row0 * nx, count, df);
  return cudaGetLastError();
}

template <int R, bool TR>
static cudaError_t launch_propagate_t(const double* in, double* out, int count, int nx, int k, const DevTaps& t,
                                      double* partial, int threads, cudaStream_t s, const Fixup& fx) {
  const size_t smem = 2 * (size_t)padded_len(nx) * sizeof(double);
  cudaError_t e = set_smem(propagate_kernel<R, TR>, smem);
  if (e != cudaSuccess) return e;
  propagate_kernel<R, TR><<<count, threads_for(nx, R, threads), smem, s>>>(in, out, nx, k, t, partial, fx);
  return cudaGetLastError();
}

cudaError_t launch_propagate(const double* in, double* out, int count, int nx, int k, const DevTaps& t,
                             double* partial, int threads, cudaStream_t s, const Fixup* fx, int trunc) {
  if (count < 1) return cudaSuccess;
  const Fixup f = fx ? *fx : Fixup{};
  const int R = tile_for(t, nx);
  if (trunc) {
    if (R == 8) return launch_propagate_t<8, true>(in, out, count, nx, k, t, partial, threads, s, f);
    if (R == 4) return launch_propagate_t<4, true>(in, out, count, nx, k, t, partial, threads, s, f);
    return launch_propagate_t<0, true>(in, out, count, nx, k, t, partial, threads, s, f);
  }
  if (R == 8) return launch_propagate_t<8, false>(in, out, count, nx, k, t, partial, threads, s, f);
  if (R == 4) return launch_propagate_t<4, false>(in, out, count, nx, k, t, partial, threads, s, f);
  return launch_propagate_t<0, false>(in, out, count, nx, k, t, partial, threads, s, f);
}

template <int R>
__global__ void __launch_bounds__(R == 8 ? 512 : 1024) seq_slab_kernel(const double* __restrict__ u0, double* out,
                                                                       int nx, int P, int every, const DevTaps t,
                                                                       const Fixup fx) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int plen = padded_len(nx);
  double* b0 = reinterpret_cast<double*>(smraw);
  double* b1 = b0 + plen;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) b0[pidx(i)] = u0[i];
  __syncthreads();
  for (int n = 1; n < P; ++n) {
    slab_step_fx<double, R>(t, fx, b0, b1, kNoG, nx);
    __syncthreads();
    if (n % every == 0)
      for (int i = threadIdx.x; i < nx; i += blockDim.x) out[(long long)(n / every) * nx + i] = b1[pidx(i)];
    double* tmp = b0; b0 = b1; b1 = tmp;
  }
}

template <int R>
static cudaError_t launch_seq_slab_t(const double* u0, double* out, int nx, int P, int every, const DevTaps& t,
                                     const Fixup& fx, int threads, cudaStream_t s) {
  const size_t smem = 2 * (size_t)padded_len(nx) * sizeof(double);
  cudaError_t e = set_smem(seq_slab_kernel<R>, smem);
  if (e != cudaSuccess) return e;
  seq_slab_kernel<R><<<1, threads_for(nx, R, threads), smem, s>>>(u0, out, nx, P, every, t, fx);
  return cudaGetLastError();
}

cudaError_t launch_seq_slab(const double* u0, double* out, int nx, int P, int store_every, const DevTaps& t,
                            const Fixup& fx, int threads, cudaStream_t s) {
  if (P < 2) return cudaSuccess;
  if (store_every < 1) return cudaErrorInvalidValue;
  const int R = tile_for(t, nx);
  if (R == 8) return launch_seq_slab_t<8>(u0, out, nx, P, store_every, t, fx, threads, s);
  if (R == 4) return launch_seq_slab_t<4>(u0, out, nx, P, store_every, t, fx, threads, s);
  return launch_seq_slab_t<0>(u0, out, nx, P, store_every, t, fx, threads, s);
}

}  // namespace mg
