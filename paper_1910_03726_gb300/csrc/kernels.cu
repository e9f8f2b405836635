// CUDA kernels (sm_103a) of the MGRIT hot path for periodic advection:
//   fcf_kernel      FCF-relaxation + fused C-point residual (Section 2.2)
//   march_kernel    sequential march u_n = T u_{n-1} + g_n on a thread-block
//                   cluster (coarse solve, Eq. 5; sequential stepping, Eq. 3)
//   correct_kernel  coarse-level correction + F-relaxation (ideal interpolation)
//   norm_kernel     deterministic residual 2-norm (Section 2.2 stopping test)
//   propagate_kernel  T^k applied to a batch of vectors
// Every stencil is a circulant (Corollary 1): periodic indices wrap modulo nx.
#include <cooperative_groups.h>

#include "device.h"

namespace cg = cooperative_groups;

namespace mg {

__device__ __forceinline__ int wrapi(int k, int nx) {
  k = (k < 0) ? k + nx : k;
  return (k >= nx) ? k - nx : k;
}

template <typename T>
__device__ __forceinline__ T tap_coef(const DevTaps& t, int k);
template <>
__device__ __forceinline__ double tap_coef<double>(const DevTaps& t, int k) { return t.c64[k]; }
template <>
__device__ __forceinline__ float tap_coef<float>(const DevTaps& t, int k) { return t.c32[k]; }

// dst[i] = g[i] + sum_t c_t src[(i + off_t) mod nx] over the whole slab.
template <typename T>
__device__ __forceinline__ void slab_step(const DevTaps& t, const T* __restrict__ src, T* __restrict__ dst,
                                          const double* __restrict__ g, int nx) {
  for (int i = threadIdx.x; i < nx; i += blockDim.x) {
    T acc = g ? (T)__ldg(g + i) : (T)0;
    for (int k = 0; k < t.n; ++k) acc = fma(tap_coef<T>(t, k), src[wrapi(i + t.off[k], nx)], acc);
    dst[i] = acc;
  }
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
// FCF-relaxation with the fused residual.  One CTA per coarse interval; the
// interval's slab lives in shared memory for all 2m fine steps, so each C-point
// crosses HBM once per cycle.  PREC 0: both passes FP64.  PREC 1: the second
// pass (acting on the correction rho) in FP32.
// ----------------------------------------------------------------------------
template <int PREC>
__global__ void __launch_bounds__(1024) fcf_kernel(const FcfArgs a, const DevTaps t) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int nx = a.nx, m = a.m;
  const int j = blockIdx.x + 1;
  double* b0 = reinterpret_cast<double*>(smraw);
  double* b1 = b0 + nx;
  const double* start = a.u_old + (long long)(j - 1) * a.cstride;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) b0[i] = a.zero_old ? 0.0 : start[i];
  __syncthreads();
  for (int s = 1; s <= m; ++s) {
    const double* g = a.g ? a.g + ((long long)(j - 1) * m + s) * nx : nullptr;
    slab_step<double>(t, b0, b1, g, nx);
    __syncthreads();
    double* tmp = b0; b0 = b1; b1 = tmp;
  }
  const double* oldj = a.u_old + (long long)j * a.cstride;
  double* cn = a.c_new + (long long)j * nx;
  const bool more = j < a.N;
  double ss = 0.0;
  if (PREC == 0) {
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
      const double v = b0[i];
      cn[i] = v;
      b1[i] = v - (a.zero_old ? 0.0 : oldj[i]);
    }
    __syncthreads();
    if (!more) return;
    double* x0 = b1;
    double* x1 = b0;
    for (int s = 1; s <= m; ++s) {
      slab_step<double>(t, x0, x1, nullptr, nx);
      __syncthreads();
      double* tmp = x0; x0 = x1; x1 = tmp;
    }
    double* rr = a.r + (long long)(j + 1) * nx;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
      const double v = x0[i];
      rr[i] = v;
      ss = fma(v, v, ss);
    }
  } else {
    float* f0 = reinterpret_cast<float*>(b1);
    float* f1 = f0 + nx;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
      const double v = b0[i];
      cn[i] = v;
      f0[i] = (float)(v - (a.zero_old ? 0.0 : oldj[i]));
    }
    __syncthreads();
    if (!more) return;
    for (int s = 1; s <= m; ++s) {
      slab_step<float>(t, f0, f1, nullptr, nx);
      __syncthreads();
      float* tmp = f0; f0 = f1; f1 = tmp;
    }
    double* rr = a.r + (long long)(j + 1) * nx;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
      const double v = (double)f0[i];
      rr[i] = v;
      ss = fma(v, v, ss);
    }
  }
  if (a.partial) {
    ss = block_sum(ss);
    if (threadIdx.x == 0) a.partial[j] = ss;
  }
}

// ----------------------------------------------------------------------------
// Sequential march on one thread-block cluster.  CTA `rank` owns x in
// [rank*w, (rank+1)*w); its shared buffer holds [left halo | own | right halo].
// Per step: compute own points, cluster barrier, pull halos from the owning
// CTAs' shared memory (DSMEM), block barrier.  Two buffers alternate so a
// neighbour's reads of step n never meet its writes of step n+1.
// The next step's g and c_add values are loaded one step ahead.
// ----------------------------------------------------------------------------
template <int PPT>
__global__ void __launch_bounds__(256) march_kernel(const MarchArgs a, const DevTaps t) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cg::cluster_group cl = cg::this_cluster();
  const int cs = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int nx = a.nx, w = nx / cs, base = rank * w;
  const int L = -t.lo, R = t.hi, W = L + w + R;
  double* B0 = reinterpret_cast<double*>(smraw);
  double* B1 = B0 + W;
  const int tid = threadIdx.x, bs = blockDim.x;
  for (int k = tid; k < W; k += bs) {
    const int gi = wrapi(base - L + k, nx);
    B0[k] = a.init ? a.init[gi] : 0.0;
  }
  __syncthreads();
  double gq[PPT], cq[PPT];
#pragma unroll
  for (int p = 0; p < PPT; ++p) { gq[p] = 0.0; cq[p] = 0.0; }
  auto prefetch = [&](int n) {
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
      const int i = tid + p * bs;
      if (i < w) {
        const long long o = (long long)n * nx + base + i;
        if (a.g) gq[p] = __ldcg(a.g + o);
        if (a.c_add) cq[p] = __ldcg(a.c_add + o);
      }
    }
  };
  if (a.P > 1) prefetch(1);
  for (int n = 1; n < a.P; ++n) {
    double* cur = (n & 1) ? B0 : B1;
    double* nxt = (n & 1) ? B1 : B0;
    double gc[PPT], cc[PPT];
#pragma unroll
    for (int p = 0; p < PPT; ++p) { gc[p] = gq[p]; cc[p] = cq[p]; }
    if (n + 1 < a.P) prefetch(n + 1);
    const bool store = a.u_out && (n % a.store_every) == 0;
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
      const int i = tid + p * bs;
      if (i < w) {
        double acc = gc[p];
        const double* c = cur + L + i;
        for (int k = 0; k < t.n; ++k) acc = fma(t.c64[k], c[t.off[k]], acc);
        nxt[L + i] = acc;
        const long long o = (long long)n * nx + base + i;
        if (a.c_add) a.c_add[o] = cc[p] + acc;
        if (store) a.u_out[(long long)(n / a.store_every) * nx + base + i] = acc;
      }
    }
    cl.sync();
    for (int k = tid; k < L + R; k += bs) {
      int dst, gi;
      if (k < L) { dst = k; gi = base - L + k; }
      else { dst = w + k; gi = base + w + (k - L); }
      gi = wrapi(gi, nx);
      const int owner = gi / w, loc = gi - owner * w;
      const double* rem = cl.map_shared_rank(nxt, owner);
      nxt[dst] = rem[L + loc];
    }
    __syncthreads();
  }
  cl.sync();  // no CTA leaves while a neighbour may still read its shared memory
}

// ----------------------------------------------------------------------------
// Correction + F-relaxation of a coarse level (ideal interpolation).
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) correct_kernel(const CorrectArgs a, const DevTaps t) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int nx = a.nx, m = a.m, j = blockIdx.x + 1;
  double* b0 = reinterpret_cast<double*>(smraw);
  double* b1 = b0 + nx;
  const long long p0 = (long long)(j - 1) * m;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) {
    const double v = a.c_new[(long long)(j - 1) * nx + i] + (a.e ? a.e[(long long)(j - 1) * nx + i] : 0.0);
    b0[i] = v;
    a.u[p0 * nx + i] = v;
  }
  __syncthreads();
  for (int s = 1; s < m; ++s) {
    const double* g = a.g ? a.g + (p0 + s) * nx : nullptr;
    slab_step<double>(t, b0, b1, g, nx);
    __syncthreads();
    for (int i = threadIdx.x; i < nx; i += blockDim.x) a.u[(p0 + s) * nx + i] = b1[i];
    double* tmp = b0; b0 = b1; b1 = tmp;
  }
  if (j == a.N)
    for (int i = threadIdx.x; i < nx; i += blockDim.x)
      a.u[(long long)a.N * m * nx + i] = a.c_new[(long long)a.N * nx + i] + (a.e ? a.e[(long long)a.N * nx + i] : 0.0);
}

__global__ void __launch_bounds__(1024) norm_kernel(const double* __restrict__ partial, int n, double* out) {
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += partial[i];
  v = block_sum(v);
  if (threadIdx.x == 0) out[0] = v;
}

__global__ void add_kernel(double* __restrict__ c, const double* __restrict__ e, long long count) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    c[i] += e[i];
}

__global__ void __launch_bounds__(1024) propagate_kernel(const double* in, double* out, int nx, int k,
                                                         const DevTaps t, double* partial) {
  extern __shared__ __align__(16) unsigned char smraw[];
  double* b0 = reinterpret_cast<double*>(smraw);
  double* b1 = b0 + nx;
  const long long v = blockIdx.x;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) b0[i] = in[v * nx + i];
  __syncthreads();
  for (int s = 0; s < k; ++s) {
    slab_step<double>(t, b0, b1, nullptr, nx);
    __syncthreads();
    double* tmp = b0; b0 = b1; b1 = tmp;
  }
  double ss = 0.0;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) {
    out[v * nx + i] = b0[i];
    ss = fma(b0[i], b0[i], ss);
  }
  if (partial) {
    ss = block_sum(ss);
    if (threadIdx.x == 0) partial[v] = ss;
  }
}

// ------------------------------------------------------------------ launches

template <typename K>
static cudaError_t set_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024) return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  return cudaSuccess;
}

cudaError_t launch_fcf(const FcfArgs& a, const DevTaps& t, int precision, int threads, cudaStream_t s) {
  if (a.N < 1) return cudaSuccess;
  const size_t smem = 2 * (size_t)a.nx * sizeof(double);
  cudaError_t e;
  if (precision == 0) {
    if ((e = set_smem(fcf_kernel<0>, smem)) != cudaSuccess) return e;
    fcf_kernel<0><<<a.N, threads, smem, s>>>(a, t);
  } else {
    if ((e = set_smem(fcf_kernel<1>, smem)) != cudaSuccess) return e;
    fcf_kernel<1><<<a.N, threads, smem, s>>>(a, t);
  }
  return cudaGetLastError();
}

template <int PPT>
static cudaError_t launch_march_t(const MarchArgs& a, const DevTaps& t, int cluster, int threads,
                                  cudaStream_t s) {
  const int w = a.nx / cluster;
  const size_t smem = 2 * (size_t)(w - t.lo + t.hi) * sizeof(double);
  cudaError_t e = set_smem(march_kernel<PPT>, smem);
  if (e != cudaSuccess) return e;
  if (cluster > 8) {
    e = cudaFuncSetAttribute(march_kernel<PPT>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cluster);
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
  return cudaLaunchKernelEx(&cfg, march_kernel<PPT>, a, t);
}

cudaError_t launch_march(const MarchArgs& a, const DevTaps& t, int cluster, int threads, cudaStream_t s) {
  const int w = a.nx / cluster;
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

int march_max_cluster() { return 16; }

cudaError_t launch_correct(const CorrectArgs& a, const DevTaps& t, int threads, cudaStream_t s) {
  if (a.N < 1) return cudaSuccess;
  const size_t smem = 2 * (size_t)a.nx * sizeof(double);
  cudaError_t e = set_smem(correct_kernel, smem);
  if (e != cudaSuccess) return e;
  correct_kernel<<<a.N, threads, smem, s>>>(a, t);
  return cudaGetLastError();
}

cudaError_t launch_norm(const double* partial, int n, double* out, cudaStream_t s) {
  norm_kernel<<<1, 1024, 0, s>>>(partial, n, out);
  return cudaGetLastError();
}

cudaError_t launch_add(double* c, const double* e, long long count, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  long long blocks = (count + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  add_kernel<<<(int)blocks, 256, 0, s>>>(c, e, count);
  return cudaGetLastError();
}

cudaError_t launch_propagate(const double* in, double* out, int count, int nx, int k, const DevTaps& t,
                             double* partial, int threads, cudaStream_t s) {
  if (count < 1) return cudaSuccess;
  const size_t smem = 2 * (size_t)nx * sizeof(double);
  cudaError_t e = set_smem(propagate_kernel, smem);
  if (e != cudaSuccess) return e;
  propagate_kernel<<<count, threads, smem, s>>>(in, out, nx, k, t, partial);
  return cudaGetLastError();
}

}  // namespace mg
