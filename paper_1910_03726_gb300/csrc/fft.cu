// Coarse-level solve of the periodic problem in Fourier space.
//
// The coarse system e_0 = 0, e_n = Psi e_{n-1} + g_n (Eq. 5's block
// bidiagonal system, Psi circulant) is diagonalised by the discrete Fourier
// transform: with E_n(k) = sum_x e_n(x) w^{xk}, w = exp(-2 pi i / nx),
//   E_n(k) = mu_k E_{n-1}(k) + G_n(k),   mu_k = sum_i psi_i w^{-ik},
// one scalar recurrence per mode (mu_k is the symbol of Psi, Lemma 1).  So
// instead of marching n sequentially over a cluster, the slabs g_1..g_{P-1}
// are transformed independently (one CTA per slab), the recurrences run in
// parallel over the modes (and, as a chunked scan, over blocks of n), and
// the slabs are transformed back, with the march's epilogue (store u_n, or
// c_n += e_n) fused into the inverse.
//
// FFT: the slabs are real, so each is transformed as one complex FFT of
// half length, z_j = x_{2j} + i x_{2j+1} (FP64, in place in shared memory:
// loaded in bit-reversed order, p-1 radix-2 decimation-in-time stages), and
// split into the nx/2 + 1 independent modes with
//   X_k = A_k + w^k B_k,  A_k = (Z_k + conj Z_{h-k}) / 2,
//   B_k = (Z_k - conj Z_{h-k}) / 2i,  h = nx/2
// (A, B: the transforms of the even and odd points); the other modes are
// their conjugates (Psi is real) and are never formed.  The inverse
// recombines Z_k = A_k + i B_k from X_k and X_{h-k}.  A slab that
// is identically zero transforms to exact zeros, and a zero spectrum back to
// exact zeros, so coarse corrections of C-points that are already exact stay
// exactly zero (as in the march).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cstdlib>

#include "device.h"

namespace mg {

namespace {

namespace cg = cooperative_groups;

struct cplx64 {
  double re, im;
};

__device__ __forceinline__ cplx64 cmul(cplx64 a, cplx64 b) {
  return {fma(a.re, b.re, -a.im * b.im), fma(a.re, b.im, a.im * b.re)};
}

// In-place radix-2 DIT passes over x[0..n) (bit-reversed input, natural
// output).  tw[k] = exp(-2 pi i k / (2n)), k < n: the stages use every second
// entry (exp(-2 pi i k / n)); inverse conjugates them.
template <bool INV>
__device__ __forceinline__ void fft_passes(cplx64* x, const cplx64* __restrict__ tw, int n) {
  for (int half = 1; half < n; half <<= 1) {
    const int stride = 2 * (n / (2 * half));  // twiddle step of this stage in the 2n-point table
    for (int b = threadIdx.x; b < n / 2; b += blockDim.x) {
      const int pos = b & (half - 1);
      const int i = ((b - pos) << 1) + pos;  // group * 2 * half + pos
      const int j = i + half;
      cplx64 w = tw[pos * stride];
      if (INV) w.im = -w.im;
      const cplx64 t = cmul(w, x[j]);
      const cplx64 u = x[i];
      x[i] = {u.re + t.re, u.im + t.im};
      x[j] = {u.re - t.re, u.im - t.im};
    }
    __syncthreads();
  }
}

__device__ __forceinline__ int bitrev(int i, int logn) { return (int)(__brev((unsigned)i) >> (32 - logn)); }

// Slab n = blockIdx.x + 1 of g (FP64 or FP32) -> spectrum row n-1 of spec
// (nh = nx/2 + 1 modes per row).  logh = log2(nx/2).
__global__ void __launch_bounds__(512) fft_forward_kernel(const double* __restrict__ g, const float* __restrict__ g_f,
                                                          cplx64* __restrict__ spec, const cplx64* __restrict__ tw,
                                                          int nx, int logh) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cplx64* z = reinterpret_cast<cplx64*>(smraw);
  const int h = nx / 2;
  const long long n = blockIdx.x + 1;
  for (int j = threadIdx.x; j < h; j += blockDim.x) {
    double a, b;
    if (g_f) {
      const float2 v = __ldcg(reinterpret_cast<const float2*>(g_f + n * nx) + j);
      a = v.x;
      b = v.y;
    } else {
      const double2 v = __ldcg(reinterpret_cast<const double2*>(g + n * nx) + j);
      a = v.x;
      b = v.y;
    }
    z[bitrev(j, logh)] = {a, b};
  }
  __syncthreads();
  fft_passes<false>(z, tw, h);
  cplx64* out = spec + (n - 1) * (h + 1);
  for (int k = threadIdx.x; k <= h; k += blockDim.x) {
    const cplx64 zk = z[k == h ? 0 : k];
    const cplx64 zc = z[k == 0 ? 0 : h - k];  // Z_{h-k}, Z_h = Z_0
    const cplx64 e = {0.5 * (zk.re + zc.re), 0.5 * (zk.im - zc.im)};
    const cplx64 o = {0.5 * (zk.im + zc.im), -0.5 * (zk.re - zc.re)};  // (Z_k - conj Z_{h-k}) / 2i
    const cplx64 w = k == h ? cplx64{-1.0, 0.0} : tw[k];
    const cplx64 wo = cmul(w, o);
    out[k] = {e.re + wo.re, e.im + wo.im};
  }
}

// E_n(k) = mu_k E_{n-1}(k) + G_n(k), n = 1..P-1, for the nm = nx/2 + 1 modes
// (rows of nm), in place, as a chunked scan over n so that all SMs work: the
// rows are split into blocks of L.
// Pass 1 (one thread per mode and block): the block's recurrence from zero;
// its last value goes to carry[b][k].  Pass 2: the block's incoming value
// C_b = sum over earlier blocks of mu^(L (b-1-b')) last_b' (a recurrence over
// b with mu^L), then E_n += mu^(n - n_b + 1) C_b along the block.  A block
// whose rows and incoming value are zero stays exactly zero.
__global__ void __launch_bounds__(256) fft_recur_local_kernel(cplx64* __restrict__ spec, const cplx64* __restrict__ mu,
                                                              cplx64* __restrict__ carry, int nm, int rows, int L) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int b = blockIdx.y;
  const int r0 = b * L, r1 = min(rows, r0 + L);
  if (k >= nm || r0 >= rows) return;
  const cplx64 m = mu[k];
  cplx64 e = {0.0, 0.0};
  cplx64 nxt = spec[(long long)r0 * nm + k];
  for (int r = r0; r < r1; ++r) {
    const cplx64 gk = nxt;
    if (r + 1 < r1) nxt = spec[(long long)(r + 1) * nm + k];
    const cplx64 me = cmul(m, e);
    e = {me.re + gk.re, me.im + gk.im};
    spec[(long long)r * nm + k] = e;
  }
  carry[(long long)b * nm + k] = e;
}

__global__ void __launch_bounds__(256) fft_recur_carry_kernel(cplx64* __restrict__ spec, const cplx64* __restrict__ mu,
                                                              const cplx64* __restrict__ carry, int nm, int rows,
                                                              int L) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int b = blockIdx.y + 1;  // block 0 has no incoming value
  const int r0 = b * L, r1 = min(rows, r0 + L);
  if (k >= nm || r0 >= rows) return;
  const cplx64 m = mu[k];
  cplx64 mL = {1.0, 0.0};  // mu^L by squaring
  {
    cplx64 base = m;
    for (int e = L; e; e >>= 1) {
      if (e & 1) mL = cmul(mL, base);
      base = cmul(base, base);
    }
  }
  cplx64 c = {0.0, 0.0};  // value entering block b (blocks before b are full)
  for (int bb = 0; bb < b; ++bb) {
    const cplx64 t = cmul(mL, c);
    const cplx64 last = carry[(long long)bb * nm + k];
    c = {t.re + last.re, t.im + last.im};
  }
  if (c.re == 0.0 && c.im == 0.0) return;
  cplx64 p = m;  // mu^(r - r0 + 1)
  for (int r = r0; r < r1; ++r) {
    cplx64* s = spec + (long long)r * nm + k;
    const cplx64 add = cmul(p, c);
    const cplx64 v = *s;
    *s = {v.re + add.re, v.im + add.im};
    p = cmul(p, m);
  }
}

// Spectrum row n-1 -> e_n, then the march's epilogue for point n.
__global__ void __launch_bounds__(512) fft_inverse_kernel(const cplx64* __restrict__ spec, const cplx64* __restrict__ tw,
                                                          int nx, int logh, MarchArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cplx64* z = reinterpret_cast<cplx64*>(smraw);
  const int h = nx / 2;
  const long long n = blockIdx.x + 1;
  const cplx64* in = spec + (n - 1) * (h + 1);
  for (int k = threadIdx.x; k < h; k += blockDim.x) {
    const cplx64 xk = in[k];
    const cplx64 xc = in[h - k];  // X_{h-k}
    const cplx64 e = {0.5 * (xk.re + xc.re), 0.5 * (xk.im - xc.im)};
    const cplx64 d = {0.5 * (xk.re - xc.re), 0.5 * (xk.im + xc.im)};  // (X_k - conj X_{h-k}) / 2
    const cplx64 w = {tw[k].re, -tw[k].im};
    const cplx64 o = cmul(w, d);
    z[bitrev(k, logh)] = {e.re - o.im, e.im + o.re};  // E_k + i O_k
  }
  __syncthreads();
  fft_passes<true>(z, tw, h);
  const double scale = 1.0 / h;
  const bool store = (a.u_out || a.u_out_f) && (n % a.store_every) == 0;
  for (int j = threadIdx.x; j < h; j += blockDim.x) {
    const double ev[2] = {z[j].re * scale, z[j].im * scale};
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int i = 2 * j + q;
      const double e = ev[q];
      if (a.c_add && a.c_add_df) {  // float-float C-points
        float2* c = reinterpret_cast<float2*>(a.c_add) + n * nx + i;
        const float2 v = *c;
        const double s = ((double)v.x + (double)v.y) + e;
        const float hi = (float)s;
        *c = make_float2(hi, (float)(s - (double)hi));
      } else if (a.c_add) {
        a.c_add[n * nx + i] += e;
      }
      if (store) {
        const long long o = (n / a.store_every) * nx + i;
        if (a.u_out_f) a.u_out_f[o] = (float)e;
        else a.u_out[o] = e;
      }
    }
  }
}

// The same transforms with a slab split over a cluster of kFftSplit CTAs, for
// coarse levels with fewer slabs than SMs (one CTA per slab would leave most
// SMs idle while it runs its log2 h dependent passes).  CTA r holds points
// r q .. (r+1) q - 1 of the half-length array (q = h / kFftSplit): the first
// log2 q passes pair points inside a CTA's block (twiddles as in fft_passes:
// a block starts at a multiple of 2 half); the last log2 kFftSplit pair points
// of different CTAs, read through distributed shared memory and written to
// the other of two buffers, one cluster barrier per pass.
constexpr int kFftSplit = 4;

template <bool INV>
__device__ __forceinline__ cplx64 tw_at(const cplx64* __restrict__ tw, int k) {
  cplx64 w = tw[k];
  if (INV) w.im = -w.im;
  return w;
}

// Passes of the split transform; returns the buffer that holds the result.
template <bool INV>
__device__ __forceinline__ cplx64* fft_passes_split(cplx64* b0, cplx64* b1, const cplx64* __restrict__ tw, int h,
                                                    int q, int rank, cg::cluster_group& cl) {
  for (int half = 1; half < q; half <<= 1) {  // inside the block
    const int stride = 2 * (h / (2 * half));
    for (int b = threadIdx.x; b < q / 2; b += blockDim.x) {
      const int pos = b & (half - 1);
      const int i = ((b - pos) << 1) + pos;
      const int j = i + half;
      const cplx64 t = cmul(tw_at<INV>(tw, pos * stride), b0[j]);
      const cplx64 u = b0[i];
      b0[i] = {u.re + t.re, u.im + t.im};
      b0[j] = {u.re - t.re, u.im - t.im};
    }
    __syncthreads();
  }
  cl.sync();  // every block's inner passes done before the blocks are read across the cluster
  cplx64* cur = b0;
  cplx64* nxt = b1;
  const int base = rank * q;
  for (int half = q; half < h; half <<= 1) {  // across blocks
    const int stride = 2 * (h / (2 * half));
    for (int p = threadIdx.x; p < q; p += blockDim.x) {
      const int g = base + p;
      const int gi = g & ~half, gj = gi | half;
      const cplx64* su = cl.map_shared_rank(cur, (unsigned)(gi / q));
      const cplx64* sv = cl.map_shared_rank(cur, (unsigned)(gj / q));
      const cplx64 u = su[gi % q];
      const cplx64 t = cmul(tw_at<INV>(tw, (gi & (half - 1)) * stride), sv[gj % q]);
      nxt[p] = g == gi ? cplx64{u.re + t.re, u.im + t.im} : cplx64{u.re - t.re, u.im - t.im};
    }
    cl.sync();  // the pass's reads done everywhere before the next pass writes the buffer they read
    cplx64* tmp = cur;
    cur = nxt;
    nxt = tmp;
  }
  return cur;
}

__global__ void __launch_bounds__(512) fft_forward_split_kernel(const double* __restrict__ g,
                                                                const float* __restrict__ g_f,
                                                                cplx64* __restrict__ spec,
                                                                const cplx64* __restrict__ tw, int nx, int logh) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cg::cluster_group cl = cg::this_cluster();
  const int h = nx / 2, q = h / kFftSplit, rank = (int)cl.block_rank(), base = rank * q;
  cplx64* b0 = reinterpret_cast<cplx64*>(smraw);
  cplx64* b1 = b0 + q;
  const long long n = blockIdx.x / kFftSplit + 1;
  for (int p = threadIdx.x; p < q; p += blockDim.x) {
    const int j = bitrev(base + p, logh);
    double a, b;
    if (g_f) {
      const float2 v = __ldcg(reinterpret_cast<const float2*>(g_f + n * nx) + j);
      a = v.x;
      b = v.y;
    } else {
      const double2 v = __ldcg(reinterpret_cast<const double2*>(g + n * nx) + j);
      a = v.x;
      b = v.y;
    }
    b0[p] = {a, b};
  }
  __syncthreads();
  const cplx64* z = fft_passes_split<false>(b0, b1, tw, h, q, rank, cl);
  cplx64* out = spec + (n - 1) * (h + 1);
  for (int p = threadIdx.x; p <= q; p += blockDim.x) {
    const int k = base + p;
    if (p == q && k != h) break;  // mode h: the last CTA
    const int ka = k == h ? 0 : k, kc = k == 0 ? 0 : h - k;
    const cplx64 zk = cl.map_shared_rank(z, (unsigned)(ka / q))[ka % q];
    const cplx64 zc = cl.map_shared_rank(z, (unsigned)(kc / q))[kc % q];  // Z_{h-k}, Z_h = Z_0
    const cplx64 e = {0.5 * (zk.re + zc.re), 0.5 * (zk.im - zc.im)};
    const cplx64 o = {0.5 * (zk.im + zc.im), -0.5 * (zk.re - zc.re)};
    const cplx64 w = k == h ? cplx64{-1.0, 0.0} : tw[k];
    const cplx64 wo = cmul(w, o);
    out[k] = {e.re + wo.re, e.im + wo.im};
  }
  cl.sync();  // no CTA leaves while another may still read its shared memory
}

__global__ void __launch_bounds__(512) fft_inverse_split_kernel(const cplx64* __restrict__ spec,
                                                                const cplx64* __restrict__ tw, int nx, int logh,
                                                                MarchArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cg::cluster_group cl = cg::this_cluster();
  const int h = nx / 2, q = h / kFftSplit, rank = (int)cl.block_rank(), base = rank * q;
  cplx64* b0 = reinterpret_cast<cplx64*>(smraw);
  cplx64* b1 = b0 + q;
  const long long n = blockIdx.x / kFftSplit + 1;
  const cplx64* in = spec + (n - 1) * (h + 1);
  for (int p = threadIdx.x; p < q; p += blockDim.x) {
    const int k = bitrev(base + p, logh);
    const cplx64 xk = in[k];
    const cplx64 xc = in[h - k];
    const cplx64 e = {0.5 * (xk.re + xc.re), 0.5 * (xk.im - xc.im)};
    const cplx64 d = {0.5 * (xk.re - xc.re), 0.5 * (xk.im + xc.im)};
    const cplx64 w = {tw[k].re, -tw[k].im};
    const cplx64 o = cmul(w, d);
    b0[p] = {e.re - o.im, e.im + o.re};
  }
  __syncthreads();
  const cplx64* z = fft_passes_split<true>(b0, b1, tw, h, q, rank, cl);
  const double scale = 1.0 / h;
  const bool store = (a.u_out || a.u_out_f) && (n % a.store_every) == 0;
  for (int p = threadIdx.x; p < q; p += blockDim.x) {
    const int j = base + p;
    const double ev[2] = {z[p].re * scale, z[p].im * scale};
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int i = 2 * j + r;
      const double e = ev[r];
      if (a.c_add && a.c_add_df) {
        float2* c = reinterpret_cast<float2*>(a.c_add) + n * nx + i;
        const float2 v = *c;
        const double s = ((double)v.x + (double)v.y) + e;
        const float hi = (float)s;
        *c = make_float2(hi, (float)(s - (double)hi));
      } else if (a.c_add) {
        a.c_add[n * nx + i] += e;
      }
      if (store) {
        const long long o = (n / a.store_every) * nx + i;
        if (a.u_out_f) a.u_out_f[o] = (float)e;
        else a.u_out[o] = e;
      }
    }
  }
  // the last cross pass ended with a cluster barrier: no other CTA reads this
  // one's shared memory any more
}

// tw[k] = exp(-2 pi i k / nx), k < nx/2, and mu_k = sum_t psi_t
// exp(2 pi i (off_t k mod nx) / nx), k < nx, in FP64 (sincospi keeps the
// reduced argument exact).
__global__ void __launch_bounds__(256) fft_tables_kernel(const DevTaps t, int nx, cplx64* __restrict__ tw,
                                                         cplx64* __restrict__ mu) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nx) return;
  double s, c;
  if (k < nx / 2) {
    sincospi(-2.0 * k / nx, &s, &c);
    tw[k] = {c, s};
  }
  double re = 0.0, im = 0.0;
  for (int q = 0; q < t.n; ++q) {
    long long ik = ((long long)t.off[q] * k) % nx;
    if (ik < 0) ik += nx;
    sincospi(2.0 * (double)ik / nx, &s, &c);
    re = fma(t.c64[q], c, re);
    im = fma(t.c64[q], s, im);
  }
  mu[k] = {re, im};
}

int fft_threads(int nx) { return nx >= 2048 ? 512 : (nx / 4 < 32 ? 32 : nx / 4); }

}  // namespace

bool fft_coarse_supported(int nx) { return nx >= 64 && nx <= 8192 && (nx & (nx - 1)) == 0; }

cudaError_t launch_fft_tables(const DevTaps& psi, int nx, double* tw, double* mu, cudaStream_t s) {
  if (!fft_coarse_supported(nx)) return cudaErrorInvalidValue;
  fft_tables_kernel<<<(nx + 255) / 256, 256, 0, s>>>(psi, nx, reinterpret_cast<cplx64*>(tw),
                                                     reinterpret_cast<cplx64*>(mu));
  return cudaGetLastError();
}

// Blocks of rows of the chunked scan: enough for about four CTAs per SM, but
// no more than about sqrt(rows) (pass 2 walks the earlier blocks' ends one by
// one), at most kMaxScanBlocks, and none empty.
static int scan_blocks(int rows, int mblocks) {
  int nb = (4 * 152 + mblocks - 1) / mblocks;
  int sq = 1;
  while (sq * sq < rows) ++sq;
  nb = nb > sq ? sq : nb;
  nb = nb < 1 ? 1 : (nb > kMaxScanBlocks ? kMaxScanBlocks : nb);
  nb = nb > rows ? rows : nb;
  const int L = (rows + nb - 1) / nb;
  return (rows + L - 1) / L;
}

// The split transforms where a coarse level has fewer slabs than SMs and a
// CTA's block keeps at least 256 points (nx >= 2048); MGRIT_FFT_SPLIT = 0 / 1
// turns them off / on wherever the size allows.
static int sm_count_fft() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
      cudaGetLastError();
      n = 152;
    }
  }
  return n;
}
static bool use_fft_split(int nx, int rows) {
  if (nx / 2 / kFftSplit < 256) return false;
  const char* e = std::getenv("MGRIT_FFT_SPLIT");
  if (e && *e) return std::atoi(e) != 0;
  return rows < sm_count_fft();
}
template <typename Kern, typename... Args>
static cudaError_t launch_split(Kern kernel, int nx, int rows, cudaStream_t s, Args... args) {
  const int q = nx / 2 / kFftSplit;
  const size_t smem = 2 * (size_t)q * sizeof(cplx64);
  cudaError_t e = cudaSuccess;
  if (smem > 48 * 1024 &&
      (e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
    return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(rows * kFftSplit);
  cfg.blockDim = dim3(q / 2);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = kFftSplit;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

int coarse_fft_launches(int nx, int P) {
  if (P < 2) return 0;
  return scan_blocks(P - 1, (nx / 2 + 1 + 255) / 256) > 1 ? 4 : 3;
}

cudaError_t launch_coarse_fft(const MarchArgs& a, const CoarseFft& f, cudaStream_t s) {
  if (a.P < 2) return cudaSuccess;
  if (!fft_coarse_supported(a.nx) || a.init || a.trunc || !f.spec || !f.carry || a.P - 1 > f.rows ||
      (!a.g && !a.g_f))
    return cudaErrorInvalidValue;
  int logh = 0;
  while ((2 << logh) < a.nx) ++logh;
  const int nh = a.nx / 2 + 1;  // independent modes of a real slab
  const size_t smem = (size_t)(a.nx / 2) * sizeof(cplx64);
  const int th = fft_threads(a.nx);
  cplx64* spec = reinterpret_cast<cplx64*>(f.spec);
  const cplx64* tw = reinterpret_cast<const cplx64*>(f.tw);
  const cplx64* mu = reinterpret_cast<const cplx64*>(f.mu);
  cudaError_t e = cudaSuccess;
  if (smem > 48 * 1024) {
    if ((e = cudaFuncSetAttribute(fft_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
            cudaSuccess ||
        (e = cudaFuncSetAttribute(fft_inverse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
            cudaSuccess)
      return e;
  }
  const bool split = use_fft_split(a.nx, a.P - 1);
  if (split) e = launch_split(fft_forward_split_kernel, a.nx, a.P - 1, s, a.g_f ? nullptr : a.g, a.g_f, spec, tw,
                              a.nx, logh);
  else fft_forward_kernel<<<a.P - 1, th, smem, s>>>(a.g_f ? nullptr : a.g, a.g_f, spec, tw, a.nx, logh);
  if (e != cudaSuccess || (e = cudaGetLastError()) != cudaSuccess) return e;
  const int rows = a.P - 1;
  const int mblocks = (nh + 255) / 256;
  const int nb = scan_blocks(rows, mblocks);
  const int L = (rows + nb - 1) / nb;
  cplx64* carry = reinterpret_cast<cplx64*>(f.carry);
  fft_recur_local_kernel<<<dim3(mblocks, nb), 256, 0, s>>>(spec, mu, carry, nh, rows, L);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (nb > 1) {
    fft_recur_carry_kernel<<<dim3(mblocks, nb - 1), 256, 0, s>>>(spec, mu, carry, nh, rows, L);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (split) {
    e = launch_split(fft_inverse_split_kernel, a.nx, a.P - 1, s, (const cplx64*)spec, tw, a.nx, logh, a);
    if (e != cudaSuccess) return e;
  } else {
    fft_inverse_kernel<<<a.P - 1, th, smem, s>>>(spec, tw, a.nx, logh, a);
  }
  return cudaGetLastError();
}

}  // namespace mg
