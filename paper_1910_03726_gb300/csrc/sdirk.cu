// SDIRK fine steps: host-side launch dispatch over the recurrence orders
// (KF, KB) of the stage matrix.  The kernels live in sdirk_impl.cuh and are
// compiled once per (KF, KB) pair in sdirk_k<KF><KB>.cu (the split level-1
// FCF in sdirk_s<KF><KB>.cu).
#include <cuda_runtime.h>

#include <cstdlib>

#include "device.h"

namespace mg {

template <int KF, int KB>
cudaError_t sdirk_fcf(const FcfArgs& a, const SdirkPlan& p, int precision, cudaStream_t s);
template <int KF, int KB>
cudaError_t sdirk_fcf_split(const FcfArgs& a, const SdirkPlan& p, int precision, cudaStream_t s);
template <int KF, int KB>
cudaError_t sdirk_fcf_batched(const BatchSolve* S, const BatchItem* items, int nitems, const SdirkPlan& any,
                              size_t smem, int precision, cudaStream_t s);
template <int KF, int KB>
cudaError_t sdirk_coarse_march(const double* g, const float* g_f, double* c_add, int nx, int P, const SdirkPlan& p,
                               cudaStream_t s);
template <int KF, int KB>
cudaError_t sdirk_steps(const double* in, long long in_stride, double* out, long long out_stride, int count, int nx,
                        int steps, int store_every, int store_first, const SdirkPlan& p, double* partial,
                        cudaStream_t s);

// Stage matrices of U1..U5 keep -lo roots inside the unit circle and hi
// outside (the symbol of I - gamma dtL has positive real part, so it does not
// wind around 0): (KF, KB) = (1,0), (2,0), (2,1), (3,1), (3,2).
bool sdirk_orders_supported(int kf, int kb) {
  return (kf == 1 && kb == 0) || (kf == 2 && kb == 0) || (kf == 2 && kb == 1) || (kf == 3 && kb == 1) ||
         (kf == 3 && kb == 2);
}

template <typename F>
static cudaError_t with_orders(const SdirkPlan& p, F&& f) {
  if (p.kf == 1 && p.kb == 0) return f.template operator()<1, 0>();
  if (p.kf == 2 && p.kb == 0) return f.template operator()<2, 0>();
  if (p.kf == 2 && p.kb == 1) return f.template operator()<2, 1>();
  if (p.kf == 3 && p.kb == 1) return f.template operator()<3, 1>();
  if (p.kf == 3 && p.kb == 2) return f.template operator()<3, 2>();
  return cudaErrorInvalidValue;
}

int sdirk_slots(const SdirkPlan& p) { return p.s <= 2 ? 1 : p.s - 1; }

// CTA size for nx: nx = threads * C with C in {16, 4, 1} (the largest that
// leaves at least two warps), threads a multiple of 32 and at most 512;
// 0 if no such split exists.
int sdirk_threads(int nx) {
  for (int min_threads : {64, 32})
    for (int C : {kSdirkCMax, 4, 1})
      if (nx % C == 0 && nx / C <= 512 && (nx / C) % 32 == 0 && nx / C >= min_threads) return nx / C;
  return 0;
}

size_t sdirk_smem(const SdirkPlan& p) {
  auto r256 = [](size_t b) { return (b + 255) / 256 * 256; };
  return r256((size_t)p.tab_len * 8) + r256((size_t)p.tab_len * 4) +
         (size_t)sdirk_slots(p) * padded_len(p.nx) * sizeof(double);
}

// The level-1 FCF with each interval's slab split over a cluster of two CTAs
// (fcf_sdirk_cluster_kernel): chosen when one CTA per interval would hold 512
// threads, which with the slab in registers during the scans leaves one CTA
// per SM; needs C = 16, ql = 0 and half the threads a whole number of warps.
// MGRIT_SDIRK_SPLIT = 0 / 1 turns it off / on wherever it applies.
static bool sdirk_split_ok(const SdirkPlan& p) {
  if (p.C != kSdirkCMax || p.ql != 0 || (p.threads / 2) % 32 != 0) return false;
  const char* e = std::getenv("MGRIT_SDIRK_SPLIT");
  if (e && *e) return std::atoi(e) != 0;
  return p.threads == 512;
}

cudaError_t launch_fcf_sdirk(const FcfArgs& a, const SdirkPlan& p, int precision, cudaStream_t s) {
  if (a.N < 1) return cudaSuccess;
  if (sdirk_split_ok(p))
    return with_orders(p, [&]<int KF, int KB>() { return sdirk_fcf_split<KF, KB>(a, p, precision, s); });
  return with_orders(p, [&]<int KF, int KB>() { return sdirk_fcf<KF, KB>(a, p, precision, s); });
}

cudaError_t launch_fcf_sdirk_batched(const BatchSolve* S, const BatchItem* items, int nitems, const SdirkPlan& any,
                                     size_t smem, int precision, cudaStream_t s) {
  if (nitems < 1) return cudaSuccess;
  return with_orders(any, [&]<int KF, int KB>() {
    return sdirk_fcf_batched<KF, KB>(S, items, nitems, any, smem, precision, s);
  });
}

cudaError_t launch_propagate_sdirk(const double* in, double* out, int count, int nx, int k, const SdirkPlan& p,
                                   double* partial, cudaStream_t s) {
  if (count < 1) return cudaSuccess;
  return with_orders(p, [&]<int KF, int KB>() {
    return sdirk_steps<KF, KB>(in, nx, out, nx, count, nx, k, k > 0 ? k : 1, k == 0 ? 1 : 0, p, partial, s);
  });
}

cudaError_t launch_interp_sdirk(const double* c, double* u, int nx, int m, int N, const SdirkPlan& p,
                                cudaStream_t s) {
  if (N < 1) return cudaSuccess;
  cudaError_t e = with_orders(p, [&]<int KF, int KB>() {
    return sdirk_steps<KF, KB>(c, nx, u, (long long)m * nx, N, nx, m - 1, 1, 1, p, nullptr, s);
  });
  if (e != cudaSuccess) return e;
  return cudaMemcpyAsync(u + (long long)N * m * nx, c + (long long)N * nx, (size_t)nx * sizeof(double),
                         cudaMemcpyDeviceToDevice, s);
}

cudaError_t launch_seq_sdirk(const double* u0, double* out, int nx, int P, int store_every, const SdirkPlan& p,
                             cudaStream_t s) {
  if (P < 2) return cudaSuccess;
  return with_orders(p, [&]<int KF, int KB>() {
    return sdirk_steps<KF, KB>(u0, 0, out, 0, 1, nx, P - 1, store_every, 1, p, nullptr, s);
  });
}

cudaError_t launch_coarse_march_sdirk(const double* g, const float* g_f, double* c_add, int nx, int P,
                                      const SdirkPlan& p, cudaStream_t s) {
  if (P < 2) return cudaSuccess;
  return with_orders(p, [&]<int KF, int KB>() { return sdirk_coarse_march<KF, KB>(g, g_f, c_add, nx, P, p, s); });
}

}  // namespace mg
