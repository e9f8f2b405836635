// SDIRK fine steps (sm_103a), device side: the stage form of Appendix A's
// stiffly accurate L-stable tableaux with the implicit stage matrix
// M = I - gamma dt L solved exactly by periodic recurrences (Section 2.1).
//
// Stage i of a step:  K_i = (M^{-1} A_i - A_i) / gamma,  A_i = u + sum_{j<i} a_ij K_j,
// and u_new = A_s + gamma K_s.  M^{-1} = scale * E^{ql} * B^{-1} * F^{-1} with
//   F: x_i = sum_{q=1..KF} af_q x_{i-q} + y_i   (roots of M inside the unit circle)
//   B: x_i = sum_{q=1..KB} ab_q x_{i+q} + y_i   (roots outside), both periodic.
//
// A periodic recurrence of order K over the slab runs as a chunked scan:
//   1. each thread owns C consecutive points and runs the recurrence over
//      them from a zero state (the state is the vector of the last K values);
//   2. the chunk-end states are combined by an inclusive Kogge-Stone scan
//      over the warp (state_t += A^d state_{t-d}, A = T^C, T the companion
//      matrix) and over the warps (with A^32);
//   3. the periodic closure is exact: the state before point 0 equals the
//      state after point nx-1, s_{-1} = (I - T^nx)^{-1} P_last;
//   4. each thread's carry-in state is P_{t-1} + A^t s_{-1}, and point c of
//      its chunk gets (row 0 of T^{c+1}) . carry.
// The backward recurrence is the same scan over mirrored thread and point
// order.  Every table (powers of A, G, the closure matrix Q) comes from the
// host in FP64 (and its FP32 rounding for the FP32 pass).
//
// Template parameters: PREC (0 FP64, 1 FP64 + FP32 second F-relaxation),
// C (points per thread), KF/KB (recurrence orders: 1/0, 2/0, 2/1, 3/1, 3/2
// for U1..U5, whose stage matrices keep -lo roots inside the unit circle).
// Each instantiation file compiles one (KF, KB) pair.
#pragma once
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "device.h"

namespace mg {
namespace sd {

// CL = 1: one CTA per slab.  CL = 2: the slab split over a cluster of two
// CTAs (CTA r owns points r*nx/2 ..), which exchange the scans' warp totals
// through distributed shared memory; a barrier that orders those exchanges
// spans the cluster.
template <int CL>
__device__ __forceinline__ void csync() {
  if constexpr (CL == 1) __syncthreads();
  else cooperative_groups::this_cluster().sync();
}
// The two halves of a cluster barrier (release / acquire), so that work that
// needs no other CTA's data runs while the partner arrives.
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory"); }

__device__ __forceinline__ int wrapn(int k, int nx) {
  k = (k < 0) ? k + nx : k;
  return (k >= nx) ? k - nx : k;
}
__device__ __forceinline__ int pix(int e) { return e + (e >> 3); }

template <typename T>
struct Prec;
template <>
struct Prec<double> {
  static __device__ __forceinline__ double a(const SdirkPlan& p, int i, int j) { return p.a[i][j]; }
  static __device__ __forceinline__ double gamma(const SdirkPlan& p) { return p.gamma; }
  static __device__ __forceinline__ double inv_gamma(const SdirkPlan& p) { return p.inv_gamma; }
  static __device__ __forceinline__ double scale(const SdirkPlan& p) { return p.scale; }
};
template <>
struct Prec<float> {
  static __device__ __forceinline__ float a(const SdirkPlan& p, int i, int j) { return p.a32[i][j]; }
  static __device__ __forceinline__ float gamma(const SdirkPlan& p) { return p.gamma32; }
  static __device__ __forceinline__ float inv_gamma(const SdirkPlan& p) { return p.inv_gamma32; }
  static __device__ __forceinline__ float scale(const SdirkPlan& p) { return p.scale32; }
};

template <typename T>
__device__ __forceinline__ T shfl_prev(T v, int d, bool bwd) {
  return bwd ? __shfl_down_sync(0xffffffffu, v, d) : __shfl_up_sync(0xffffffffu, v, d);
}

// y += M x for a K x K row-major matrix M.
template <typename T, int K>
__device__ __forceinline__ void matvec_acc(const T* M, const T (&x)[K], T (&y)[K]) {
#pragma unroll
  for (int r = 0; r < K; ++r) {
    T acc = y[r];
#pragma unroll
    for (int q = 0; q < K; ++q) acc = fma(M[r * K + q], x[q], acc);
    y[r] = acc;
  }
}

// Periodic recurrence of order K over the slab held in registers (x[c] is
// point threadIdx.x * C + c).  tb: this direction's tables; smw: 16*K scratch
// owned by this direction.  steps: warp-scan doubling steps that matter
// (terms carrying A^(2^steps) or more lie below FP64 rounding); trunc: A^32
// lies below rounding too, so a chunk only feels the previous warp's total
// (periodically: warp 0 feels the last warp's) and the closure is the
// identity.  Both are decided on the host from the norms of the powers.
// With CL = 2 the warps of both CTAs form one scan over the slab (global
// warp rank * warps + w): lane 31 of each warp stores its chunk-end state in
// its own and in the partner's smw (smw_peer), and after the cluster barrier
// every CTA reads all warp totals locally.
template <typename T, int C, int K, bool BWD, int CL = 1>
__device__ __forceinline__ void rec_scan(T (&x)[C], const T* __restrict__ tb, T* smw, T* smw_peer, int rank,
                                         int steps, bool trunc) {
  if constexpr (K > 0) {
    const T* lanep = tb + K;
    const T* warpp = lanep + 33 * K * K;
    const T* G = warpp + 17 * K * K;
    const T* Q = G + C * K;
    const int nwl = blockDim.x >> 5;
    const int nw = nwl * CL;
    const int gw = rank * nwl + (int)(threadIdx.x >> 5);
    const int lane = BWD ? 31 - (int)(threadIdx.x & 31) : (int)(threadIdx.x & 31);
    const int warp = BWD ? nw - 1 - gw : gw;
#define MG_XM(cc) x[BWD ? C - 1 - (cc) : (cc)]
    T aq[K];
#pragma unroll
    for (int q = 0; q < K; ++q) aq[q] = tb[q];
    // 1. chunk from a zero state; the term of the value just computed comes
    // last, so one FMA per point lies on the recurrence's dependency chain
#pragma unroll
    for (int cc = 0; cc < C; ++cc) {
      T acc = MG_XM(cc);
#pragma unroll
      for (int q = K; q >= 1; --q)
        if (cc - q >= 0) acc = fma(aq[q - 1], MG_XM(cc - q), acc);
      MG_XM(cc) = acc;
    }
    T S[K];
#pragma unroll
    for (int q = 0; q < K; ++q) S[q] = (C - 1 - q >= 0) ? MG_XM(C - 1 - q) : (T)0;
    // 2. scan of chunk-end states over the warp ...
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      if (i >= steps) break;
      const int d = 1 << i;
      T Y[K];
#pragma unroll
      for (int q = 0; q < K; ++q) Y[q] = shfl_prev(S[q], d, BWD);
      if (lane >= d) matvec_acc<T, K>(lanep + d * K * K, Y, S);
    }
    if (lane == 31)
#pragma unroll
      for (int q = 0; q < K; ++q) {
        smw[warp * K + q] = S[q];
        if constexpr (CL > 1) smw_peer[warp * K + q] = S[q];
      }
    if constexpr (CL > 1) cluster_arrive();
    else __syncthreads();
    T P[K], V[K];
#pragma unroll
    for (int q = 0; q < K; ++q) {
      const T v = shfl_prev(S[q], 1, BWD);
      P[q] = lane > 0 ? v : (T)0;
    }
    if constexpr (CL > 1) cluster_wait();
    if (trunc) {
      // 3'. carry from the previous warp's total (the last warp's for warp 0)
      const int wp = warp == 0 ? nw - 1 : warp - 1;
#pragma unroll
      for (int q = 0; q < K; ++q) V[q] = smw[wp * K + q];
    } else {
      // ... and over the warps (one warp, mirrored warp index = lane)
      if (threadIdx.x < 32) {
        const int l = threadIdx.x;
        T W[K];
#pragma unroll
        for (int q = 0; q < K; ++q) W[q] = l < nw ? smw[l * K + q] : (T)0;
#pragma unroll
        for (int d = 1; d < 16; d <<= 1) {
          T Y[K];
#pragma unroll
          for (int q = 0; q < K; ++q) Y[q] = __shfl_up_sync(0xffffffffu, W[q], d);
          if (l >= d) matvec_acc<T, K>(warpp + d * K * K, Y, W);
        }
        __syncwarp();
        if (l < nw)
#pragma unroll
          for (int q = 0; q < K; ++q) smw[l * K + q] = W[q];
      }
      __syncthreads();
      // 3. periodic closure and 4. carry-in state of this chunk
      T last[K], sm1[K];
#pragma unroll
      for (int q = 0; q < K; ++q) {
        last[q] = smw[(nw - 1) * K + q];
        sm1[q] = (T)0;
        V[q] = warp > 0 ? smw[(warp - 1) * K + q] : (T)0;
      }
      matvec_acc<T, K>(Q, last, sm1);
      matvec_acc<T, K>(warpp + warp * K * K, sm1, V);
    }
    matvec_acc<T, K>(lanep + lane * K * K, V, P);
#pragma unroll
    for (int cc = 0; cc < C; ++cc) {
      T acc = MG_XM(cc);
#pragma unroll
      for (int q = 0; q < K; ++q) acc = fma(G[cc * K + q], P[q], acc);
      MG_XM(cc) = acc;
    }
#undef MG_XM
    // smw is written again only after the caller's next barrier (CL = 2: a
    // cluster barrier, which the partner must pass before its next store)
  }
}

// u <- Phi u.  u in slot 0; slots 1..s-2 hold A_3..A_s (A_2 replaces u in slot 0).
template <typename T, int C, int KF, int KB, int CL = 1>
__device__ __forceinline__ void sdirk_step(const SdirkPlan& p, T* slab, int plen, int nx, const T* tab, T* smw,
                                           T* smw_peer = nullptr, int rank = 0) {
  const int s = p.s, base = threadIdx.x * C;
  const T sc = Prec<T>::scale(p), ig = Prec<T>::inv_gamma(p), g = Prec<T>::gamma(p);
  const T* tf = tab;
  const T* tb = tab + sdirk_rec_len(KF, C);
  for (int st = 1; st <= s; ++st) {
    T* in = st <= 2 ? slab : slab + (st - 2) * plen;
    T x[C];
#pragma unroll
    for (int c = 0; c < C; ++c) x[c] = in[pix(wrapn(base + c + p.ql, nx))];
    rec_scan<T, C, KF, false, CL>(x, tf, smw, smw_peer, rank, p.steps_f, p.trunc_f);
    rec_scan<T, C, KB, true, CL>(x, tb, smw + 16 * kMaxRec, CL > 1 ? smw_peer + 16 * kMaxRec : nullptr, rank,
                                 p.steps_b, p.trunc_b);
    if constexpr (KF == 0 && KB == 0) __syncthreads();
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const int e = pix(base + c);
      const T A = in[e];
      const T kv = fma(x[c], sc, -A) * ig;  // K_st = (M^{-1} A_st - A_st) / gamma
      if (st == 1) {
        for (int l = 3; l <= s; ++l) slab[(l - 2) * plen + e] = fma(Prec<T>::a(p, l - 1, 0), kv, A);
        in[e] = fma(s >= 2 ? Prec<T>::a(p, 1, 0) : g, kv, A);
      } else {
        for (int l = st + 1; l <= s; ++l) {
          T* Al = slab + (l - 2) * plen;
          Al[e] = fma(Prec<T>::a(p, l - 1, st - 1), kv, Al[e]);
        }
        if (st == s) slab[e] = fma(g, kv, A);  // u_new = A_s + gamma K_s
      }
    }
    // CL = 2: a store into the partner's smw of one direction waits for the
    // partner's reads of that direction in the stage before.  With both
    // directions the other direction's cluster barrier lies between them; a
    // forward recurrence alone needs this barrier to span the cluster.
    if constexpr (CL > 1 && KB == 0) csync<CL>();
    else __syncthreads();
  }
}

__device__ __forceinline__ double block_sum(double ss) {
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

__host__ __device__ constexpr size_t round256(size_t b) { return (b + 255) / 256 * 256; }

// Shared memory: FP64 tables, FP32 tables, then the slabs.
struct Smem {
  double* t64;
  float* t32;
  double* slab;
};
__device__ __forceinline__ Smem carve(unsigned char* raw, const SdirkPlan& p) {
  Smem m;
  m.t64 = reinterpret_cast<double*>(raw);
  m.t32 = reinterpret_cast<float*>(raw + round256((size_t)p.tab_len * 8));
  m.slab = reinterpret_cast<double*>(raw + round256((size_t)p.tab_len * 8) + round256((size_t)p.tab_len * 4));
  return m;
}
__device__ __forceinline__ void load_tables(const SdirkPlan& p, const Smem& m) {
  for (int i = threadIdx.x; i < p.tab_len; i += blockDim.x) {
    m.t64[i] = p.tab64[i];
    m.t32[i] = p.tab32[i];
  }
}

// What a CTA of a 2-CTA cluster shares with its partner beyond the scans: the
// partner's smw, its own rank, and slots (own and partner's) for the
// cluster-wide zero-slab votes and the two halves' squared norms.
struct ClusterLink {
  double* smw_peer = nullptr;
  int rank = 0;
  int* vote = nullptr;
  int* vote_peer = nullptr;
  double* ss = nullptr;
  double* ss_peer = nullptr;
};

// __syncthreads_or over the slab: with CL = 2 both CTAs take the same branch.
// Each call site has its own pair of slots.
template <int CL>
__device__ __forceinline__ bool slab_or(int v, const ClusterLink& L, int site) {
  const int mine = __syncthreads_or(v);
  if constexpr (CL == 1) {
    return mine != 0;
  } else {
    if (threadIdx.x == 0) {
      L.vote[2 * site + L.rank] = mine;
      L.vote_peer[2 * site + L.rank] = mine;
    }
    csync<CL>();
    return (L.vote[2 * site] | L.vote[2 * site + 1]) != 0;
  }
}

// partial[j] = the slab's squared norm (a block sum per CTA; with CL = 2 rank
// 0 adds its half and the partner's, in that order).
template <int CL>
__device__ __forceinline__ void store_partial(double* partial, int j, double ss, const ClusterLink& L) {
  ss = block_sum(ss);
  if constexpr (CL == 1) {
    if (threadIdx.x == 0) partial[j] = ss;
  } else {
    if (threadIdx.x == 0) {
      L.ss[L.rank] = ss;
      L.ss_peer[L.rank] = ss;
    }
    csync<CL>();
    if (L.rank == 0 && threadIdx.x == 0) partial[j] = L.ss[0] + L.ss[1];
  }
}

// One interval's FCF-relaxation and fused residual (see fcf_kernel): m steps
// from c_{j-1}, rho_j = v - c_j, then r_{j+1} = Phi^m rho_j.  CL = 2: this CTA
// holds points x0 .. x0 + nx/2 - 1 of the slab (x0 = rank * nx/2).
template <int PREC, int C, int KF, int KB, int CL = 1>
__device__ __forceinline__ void fcf_body(const FcfArgs& a, const SdirkPlan& p, int j, const Smem& sm,
                                         double* smw, const ClusterLink& L = ClusterLink()) {
  const int nxg = a.nx, nx = nxg / CL, x0 = L.rank * nx, m = a.m, plen = padded_len(nx);
  double* slab = sm.slab;
  const double* start = a.u_old + (long long)(j - 1) * a.cstride + x0;
  int nz = 0;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) {
    const double v = a.zero_old ? 0.0 : start[i];
    slab[pix(i)] = v;
    nz |= v != 0.0;
  }
  // Phi^m of an identically zero slab is zero: the steps are skipped
  const bool run1 = slab_or<CL>(nz, L, 0);
  for (int s = 0; s < m && run1; ++s)
    sdirk_step<double, C, KF, KB, CL>(p, slab, plen, nx, sm.t64, smw, L.smw_peer, L.rank);
  const double* oldj = a.u_old + (long long)j * a.cstride + x0;
  double* cn = a.c_new + (long long)j * nxg + x0;
  const bool more = j < a.N;
  double ss = 0.0;
  if (a.relax_f) {  // F-relaxation only: the C-point keeps its value, r_j = v - c_j
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
      const double old = a.zero_old ? 0.0 : oldj[i];
      const double rho = slab[pix(i)] - old;
      cn[i] = old;
      if (a.r_f) a.r_f[(long long)j * nxg + x0 + i] = (float)rho;
      else a.r[(long long)j * nxg + x0 + i] = rho;
      ss = fma(rho, rho, ss);
    }
    if (a.partial) store_partial<CL>(a.partial, j, ss, L);
    return;
  }
  if (PREC == 0) {
    nz = 0;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
      const double v = slab[pix(i)];
      cn[i] = v;
      const double rho = a.value_residual ? v : v - (a.zero_old ? 0.0 : oldj[i]);
      slab[pix(i)] = rho;
      nz |= rho != 0.0;
    }
    const bool run2 = slab_or<CL>(nz, L, 1);
    if (!more) return;
    for (int s = 0; s < m && run2; ++s)
      sdirk_step<double, C, KF, KB, CL>(p, slab, plen, nx, sm.t64, smw, L.smw_peer, L.rank);
    double* rr = a.r + (long long)(j + 1) * nxg + x0;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
      const double v = slab[pix(i)];
      rr[i] = v;
      ss = fma(v, v, ss);
    }
    if (a.value_residual) return;  // Phi^m c_new_j stored; residual_value finishes
  } else {
    // each thread owns points i = tid + k*blockDim (k < C): read all FP64
    // values before the FP32 slab (same storage) is written
    float* fs = reinterpret_cast<float*>(slab);
    double vals[C];
#pragma unroll
    for (int k = 0; k < C; ++k) vals[k] = slab[pix(threadIdx.x + k * blockDim.x)];
    __syncthreads();
    nz = 0;
#pragma unroll
    for (int k = 0; k < C; ++k) {
      const int i = threadIdx.x + k * blockDim.x;
      cn[i] = vals[k];
      const float rho = (float)(vals[k] - (a.zero_old ? 0.0 : oldj[i]));
      fs[pix(i)] = rho;
      nz |= rho != 0.0f;
    }
    const bool run2 = slab_or<CL>(nz, L, 1);
    if (!more) return;
    for (int s = 0; s < m && run2; ++s)
      sdirk_step<float, C, KF, KB, CL>(p, fs, plen, nx, sm.t32, reinterpret_cast<float*>(smw),
                                       reinterpret_cast<float*>(L.smw_peer), L.rank);
    float ssf = 0.0f;  // FP32 residual (FP32 storage if r_f), per-thread FP32 sums
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
      const float v = fs[pix(i)];
      if (a.r_f) a.r_f[(long long)(j + 1) * nxg + x0 + i] = v;
      else a.r[(long long)(j + 1) * nxg + x0 + i] = (double)v;
      ssf = fmaf(v, v, ssf);
    }
    ss = (double)ssf;
  }
  if (a.partial) store_partial<CL>(a.partial, j, ss, L);
}

template <int PREC, int C, int KF, int KB>
__global__ void __launch_bounds__(512) fcf_sdirk_kernel(const FcfArgs a, const SdirkPlan p) {
  extern __shared__ __align__(256) unsigned char smraw[];
  __shared__ __align__(16) double smw[2 * 16 * kMaxRec];
  const Smem sm = carve(smraw, p);
  load_tables(p, sm);
  fcf_body<PREC, C, KF, KB>(a, p, blockIdx.x + 1, sm, smw);
}

// One interval per cluster of two CTAs (blocks 2(j-1), 2(j-1)+1), each with
// half the slab, half the threads and half the shared memory of
// fcf_sdirk_kernel, so that two CTAs of different intervals share an SM.
// Needs ql = 0 (a stage's input is the thread's own points; every U1..U5
// stage matrix has -lo roots inside the unit circle, so ql = -lo - KF = 0).
template <int PREC, int C, int KF, int KB>
__global__ void __launch_bounds__(256, 2) fcf_sdirk_cluster_kernel(const FcfArgs a, const SdirkPlan p, int j0) {
  extern __shared__ __align__(256) unsigned char smraw[];
  __shared__ __align__(16) double smw[2 * 16 * kMaxRec];
  __shared__ int vote[4];
  __shared__ double ssum[2];
  cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
  ClusterLink L;
  L.rank = (int)cl.block_rank();
  L.smw_peer = cl.map_shared_rank(smw, L.rank ^ 1);
  L.vote = vote;
  L.vote_peer = cl.map_shared_rank(vote, L.rank ^ 1);
  L.ss = ssum;
  L.ss_peer = cl.map_shared_rank(ssum, L.rank ^ 1);
  const Smem sm = carve(smraw, p);
  load_tables(p, sm);
  cl.sync();  // both CTAs run before either stores into the other's shared memory
  fcf_body<PREC, C, KF, KB, 2>(a, p, j0 + (int)(blockIdx.x >> 1), sm, smw, L);
  cl.sync();  // no CTA leaves while its partner may still store into it
}

// Batched over solves: one CTA per (solve, interval) item.
template <int PREC, int C, int KF, int KB>
__global__ void __launch_bounds__(512) fcf_sdirk_batched_kernel(const BatchSolve* __restrict__ S,
                                                                const BatchItem* __restrict__ items) {
  extern __shared__ __align__(256) unsigned char smraw[];
  __shared__ __align__(16) double smw[2 * 16 * kMaxRec];
  __shared__ SdirkPlan p;
  const BatchItem it = items[blockIdx.x];
  const BatchSolve& b = S[it.solve];
  {
    const int* src = reinterpret_cast<const int*>(b.sd);
    int* dst = reinterpret_cast<int*>(&p);
    for (int i = threadIdx.x; i < (int)(sizeof(SdirkPlan) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();
  const Smem sm = carve(smraw, p);
  load_tables(p, sm);
  const FcfArgs a = b.fcf;
  fcf_body<PREC, C, KF, KB>(a, p, it.j, sm, smw);
}

// Runs `steps` SDIRK steps on each of gridDim.x slabs: CTA v starts from
// in + v*in_stride and stores to out + v*out_stride row r = n/store_every - 1
// (+1 and the starting slab as row 0 when store_first) after step n; with
// partial, the squared norm of its final slab goes to partial[v].  Serves
// propagation, sequential stepping and the F-point interpolation.
template <int C, int KF, int KB>
__global__ void __launch_bounds__(512) steps_sdirk_kernel(const double* in, long long in_stride, double* out,
                                                          long long out_stride, int nx, int steps, int store_every,
                                                          int store_first, const SdirkPlan p, double* partial) {
  extern __shared__ __align__(256) unsigned char smraw[];
  __shared__ __align__(16) double smw[2 * 16 * kMaxRec];
  const Smem sm = carve(smraw, p);
  load_tables(p, sm);
  double* slab = sm.slab;
  const int plen = padded_len(nx);
  const long long v = blockIdx.x;
  const double* src = in + v * in_stride;
  double* dst = out + v * out_stride;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) {
    const double x = src[i];
    slab[pix(i)] = x;
    if (store_first) dst[i] = x;
  }
  __syncthreads();
  for (int n = 1; n <= steps; ++n) {
    sdirk_step<double, C, KF, KB>(p, slab, plen, nx, sm.t64, smw);
    if (n % store_every == 0) {
      double* row = dst + (long long)(n / store_every - 1 + store_first) * nx;
      for (int i = threadIdx.x; i < nx; i += blockDim.x) row[i] = slab[pix(i)];
    }
  }
  if (partial) {
    double ss = 0.0;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
      const double x = slab[pix(i)];
      ss = fma(x, x, ss);
    }
    ss = block_sum(ss);
    if (threadIdx.x == 0) partial[v] = ss;
  }
}

// Two-level coarse solve with an SDIRK step: e_0 = 0, e_n = Phi e_{n-1} + g_n,
// c_add[n] += e_n (one CTA, sequential in n).
template <int C, int KF, int KB>
__global__ void __launch_bounds__(512) coarse_march_sdirk_kernel(const double* g, const float* g_f, double* c_add,
                                                                 int nx, int P, const SdirkPlan p) {
  extern __shared__ __align__(256) unsigned char smraw[];
  __shared__ __align__(16) double smw[2 * 16 * kMaxRec];
  const Smem sm = carve(smraw, p);
  load_tables(p, sm);
  double* slab = sm.slab;
  const int plen = padded_len(nx);
  for (int i = threadIdx.x; i < nx; i += blockDim.x) slab[pix(i)] = 0.0;
  __syncthreads();
  for (int n = 1; n < P; ++n) {
    if (n > 1) sdirk_step<double, C, KF, KB>(p, slab, plen, nx, sm.t64, smw);  // Phi 0 = 0
    const long long o = (long long)n * nx;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
      const double e = slab[pix(i)] + (g_f ? (double)g_f[o + i] : g[o + i]);
      slab[pix(i)] = e;
      c_add[o + i] += e;
    }
    __syncthreads();
  }
}

template <typename Kern>
static cudaError_t smem_attr(Kern kernel, size_t bytes) {
  if (bytes > 48 * 1024) return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  return cudaSuccess;
}

// Call f.template operator()<C>() with the plan's compile-time chunk length
// (C in {1, 4, 16}, see sdirk_threads).
template <typename F>
static cudaError_t with_chunk(int C, F&& f) {
  switch (C) {
    case 1: return f.template operator()<1>();
    case 4: return f.template operator()<4>();
    case 16: return f.template operator()<16>();
    default: return cudaErrorInvalidValue;
  }
}

// Shared memory of one CTA of the split form: the full tables, half the slabs.
inline size_t split_smem(const SdirkPlan& p) {
  return round256((size_t)p.tab_len * 8) + round256((size_t)p.tab_len * 4) +
         (size_t)sdirk_slots(p) * padded_len(p.nx / 2) * sizeof(double);
}
template <typename Kern>
static cudaError_t launch_split_part(Kern kernel, const FcfArgs& a, const SdirkPlan& p, int j0, int count,
                                     size_t smem, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2 * count);
  cfg.blockDim = dim3(p.threads / 2);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, a, p, j0);
}
// Two CTAs of the split form fit on an SM, so its CTAs run in waves of
// 2 x SMs, each CTA sharing its SM.  Where the last wave would be at most one
// CTA per SM, it is launched apart with enough shared memory requested that
// each of its CTAs has an SM to itself (and runs about twice as fast): the
// whole waves take intervals 1..N-t, the tail N-t+1..N.
template <typename Kern>
static cudaError_t launch_split(Kern kernel, const FcfArgs& a, const SdirkPlan& p, cudaStream_t s) {
  const size_t smem = split_smem(p);
  const size_t alone = 116 * 1024;  // more than half of an SM's 228 KB: one CTA per SM
  cudaError_t e = smem_attr(kernel, smem > alone ? smem : alone);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                cudaSuccess || sms < 2) {
    cudaGetLastError();
    sms = 152;
  }
  const int wave = sms;                        // intervals per wave at two CTAs per SM
  const int tail = a.N > wave ? a.N % wave : 0;  // intervals of the last wave
  if (2 * smem + 16 * 1024 <= 228 * 1024 && tail > 0 && 2 * tail <= sms) {  // two per SM in the whole waves
    if ((e = launch_split_part(kernel, a, p, 1, a.N - tail, smem, s)) != cudaSuccess) return e;
    return launch_split_part(kernel, a, p, a.N - tail + 1, tail, alone, s);
  }
  return launch_split_part(kernel, a, p, 1, a.N, smem, s);
}

}  // namespace sd

// Launchers for one (KF, KB) pair; instantiated by sdirk_k<KF><KB>.cu.
template <int KF, int KB>
cudaError_t sdirk_fcf(const FcfArgs& a, const SdirkPlan& p, int precision, cudaStream_t s) {
  const size_t smem = sdirk_smem(p);
  return sd::with_chunk(p.C, [&]<int C>() -> cudaError_t {
    cudaError_t e;
    if (precision == 0) {
      if ((e = sd::smem_attr(sd::fcf_sdirk_kernel<0, C, KF, KB>, smem)) != cudaSuccess) return e;
      sd::fcf_sdirk_kernel<0, C, KF, KB><<<a.N, p.threads, smem, s>>>(a, p);
    } else {
      if ((e = sd::smem_attr(sd::fcf_sdirk_kernel<1, C, KF, KB>, smem)) != cudaSuccess) return e;
      sd::fcf_sdirk_kernel<1, C, KF, KB><<<a.N, p.threads, smem, s>>>(a, p);
    }
    return cudaGetLastError();
  });
}

template <int KF, int KB>
cudaError_t sdirk_fcf_batched(const BatchSolve* S, const BatchItem* items, int nitems, const SdirkPlan& any,
                              size_t smem, int precision, cudaStream_t s) {
  return sd::with_chunk(any.C, [&]<int C>() -> cudaError_t {
    cudaError_t e;
    if (precision == 0) {
      if ((e = sd::smem_attr(sd::fcf_sdirk_batched_kernel<0, C, KF, KB>, smem)) != cudaSuccess) return e;
      sd::fcf_sdirk_batched_kernel<0, C, KF, KB><<<nitems, any.threads, smem, s>>>(S, items);
    } else {
      if ((e = sd::smem_attr(sd::fcf_sdirk_batched_kernel<1, C, KF, KB>, smem)) != cudaSuccess) return e;
      sd::fcf_sdirk_batched_kernel<1, C, KF, KB><<<nitems, any.threads, smem, s>>>(S, items);
    }
    return cudaGetLastError();
  });
}

template <int KF, int KB>
cudaError_t sdirk_steps(const double* in, long long in_stride, double* out, long long out_stride, int count, int nx,
                        int steps, int store_every, int store_first, const SdirkPlan& p, double* partial,
                        cudaStream_t s) {
  const size_t smem = sdirk_smem(p);
  return sd::with_chunk(p.C, [&]<int C>() -> cudaError_t {
    cudaError_t e = sd::smem_attr(sd::steps_sdirk_kernel<C, KF, KB>, smem);
    if (e != cudaSuccess) return e;
    sd::steps_sdirk_kernel<C, KF, KB><<<count, p.threads, smem, s>>>(in, in_stride, out, out_stride, nx, steps,
                                                                     store_every, store_first, p, partial);
    return cudaGetLastError();
  });
}

template <int KF, int KB>
cudaError_t sdirk_coarse_march(const double* g, const float* g_f, double* c_add, int nx, int P, const SdirkPlan& p,
                               cudaStream_t s) {
  const size_t smem = sdirk_smem(p);
  return sd::with_chunk(p.C, [&]<int C>() -> cudaError_t {
    cudaError_t e = sd::smem_attr(sd::coarse_march_sdirk_kernel<C, KF, KB>, smem);
    if (e != cudaSuccess) return e;
    sd::coarse_march_sdirk_kernel<C, KF, KB><<<1, p.threads, smem, s>>>(g, g_f, c_add, nx, P, p);
    return cudaGetLastError();
  });
}

// The split form (C = 16 only); instantiated by sdirk_s<KF><KB>.cu.
template <int KF, int KB>
cudaError_t sdirk_fcf_split(const FcfArgs& a, const SdirkPlan& p, int precision, cudaStream_t s) {
  constexpr int C = kSdirkCMax;
  if (p.C != C) return cudaErrorInvalidValue;
  return precision == 0 ? sd::launch_split(sd::fcf_sdirk_cluster_kernel<0, C, KF, KB>, a, p, s)
                        : sd::launch_split(sd::fcf_sdirk_cluster_kernel<1, C, KF, KB>, a, p, s);
}
#define MG_SDIRK_SPLIT_INSTANTIATE(KF, KB) \
  template cudaError_t sdirk_fcf_split<KF, KB>(const FcfArgs&, const SdirkPlan&, int, cudaStream_t);

#define MG_SDIRK_INSTANTIATE(KF, KB)                                                                             \
  template cudaError_t sdirk_fcf<KF, KB>(const FcfArgs&, const SdirkPlan&, int, cudaStream_t);                   \
  template cudaError_t sdirk_fcf_batched<KF, KB>(const BatchSolve*, const BatchItem*, int, const SdirkPlan&,      \
                                                 size_t, int, cudaStream_t);                                     \
  template cudaError_t sdirk_steps<KF, KB>(const double*, long long, double*, long long, int, int, int, int, int, \
                                           const SdirkPlan&, double*, cudaStream_t);                              \
  template cudaError_t sdirk_coarse_march<KF, KB>(const double*, const float*, double*, int, int, const SdirkPlan&, \
                                                  cudaStream_t);

}  // namespace mg
