// Gaussian-fit noise mode of a whole array: the noise is the width of the
// least-squares Gaussian, centred at 0, through a 256-bin histogram of its
// finite values over about +-5 MAD noises (rule and fit in sc_gaussfit.cuh).
//
// It runs after the exact MAD measurement of the same array, whose noise sets
// the bins; without a root of the fit the MAD noise stands
// (SC_WARN_GAUSS_FALLBACK), and a zero MAD noise stays zero.
//
// k_gauss_hist is a streaming pass over the array (4 bytes a value, HBM
// bound); k_gauss_fit is one block of 128 threads, one per mirror pair of
// bins, in float64.
#include "sc_gaussfit.cuh"
#include "sc_internal.h"

namespace sc {
namespace {

constexpr int kGBins = kGaussBins;
constexpr int kGHThreads = 512;
constexpr int kGHWarps = kGHThreads / 32;
constexpr int kGFitThreads = gfit::kHalf;
static_assert(kGBins == gfit::kBins, "one bin layout");

__device__ __forceinline__ void ghist_add(unsigned int* h, float s, float k) {
  const int b = gfit::bin_of(s, k);
  if (b >= 0) atomicAdd(h + b, 1u);
}

// Per-warp histograms in shared memory (a warp's lanes still collide on the
// central bins, other warps do not), summed into the global 64-bit counts.
__global__ void __launch_bounds__(kGHThreads) k_gauss_hist(const float* __restrict__ src, long long n,
                                                           const DevState* st, unsigned long long* ghist) {
  __shared__ unsigned int sh[kGHWarps][kGBins];
  if (st->plan.flags & PLAN_EMPTY) return;
  const double sm = st->sigma_cur_d;
  if (!(sm > 0.0)) return;
  const float k = gfit::scale_of(sm);
  for (int i = threadIdx.x; i < kGHWarps * kGBins; i += kGHThreads) (&sh[0][0])[i] = 0u;
  __syncthreads();
  unsigned int* h = sh[threadIdx.x >> 5];
  // 16-byte loads from the first 16-byte boundary on; the few values before it
  // and after the last full quad go one by one
  const long long head = (long long)(((16u - (reinterpret_cast<uintptr_t>(src) & 15u)) & 15u) >> 2);
  const long long pre = head < n ? head : n;
  const long long nq = (n - pre) >> 2;
  const float4* q4 = reinterpret_cast<const float4*>(src + pre);
  const long long tid = (long long)blockIdx.x * kGHThreads + threadIdx.x;
  const long long stride = (long long)gridDim.x * kGHThreads;
  long long i = tid;
  for (; i + stride < nq; i += 2 * stride) {
    const float4 a = __ldg(q4 + i), b = __ldg(q4 + i + stride);
    ghist_add(h, a.x, k); ghist_add(h, a.y, k); ghist_add(h, a.z, k); ghist_add(h, a.w, k);
    ghist_add(h, b.x, k); ghist_add(h, b.y, k); ghist_add(h, b.z, k); ghist_add(h, b.w, k);
  }
  if (i < nq) {
    const float4 a = __ldg(q4 + i);
    ghist_add(h, a.x, k); ghist_add(h, a.y, k); ghist_add(h, a.z, k); ghist_add(h, a.w, k);
  }
  if (tid < pre) ghist_add(h, __ldg(src + tid), k);
  const long long tail0 = pre + 4 * nq;
  if (tail0 + tid < n && tid < 4) ghist_add(h, __ldg(src + tail0 + tid), k);
  __syncthreads();
  for (int b = threadIdx.x; b < kGBins; b += kGHThreads) {
    unsigned long long t = 0;
#pragma unroll
    for (int w = 0; w < kGHWarps; ++w) t += sh[w][b];
    if (t) atomicAdd(ghist + b, t);
  }
}

// One block of 128 threads, thread t the folded bin pair 128 + t, 127 - t.
__global__ void __launch_bounds__(kGFitThreads) k_gauss_fit(DevState* st, const unsigned long long* ghist, int pair,
                                                            int clip) {
  __shared__ double red[kGFitThreads / 32 + 1][6];
  const int flags = st->plan.flags;
  const double sm = st->sigma_cur_d;
  __syncthreads();  // every thread has read the plan before thread 0 rewrites it
  if (flags & PLAN_EMPTY) return;
  // the clip of this measurement needs a pass of its own once sigma is known
  if (clip && threadIdx.x == 0) st->plan.flags = flags | PLAN_CLIP | PLAN_CLIP_FULL;
  if (!(sm > 0.0)) return;  // sigma stays 0: the clip adds nothing
  const float k = gfit::scale_of(sm);
  const int t = threadIdx.x;
  const double hh[1] = {(double)ghist[gfit::kHalf + t] + (double)ghist[gfit::kHalf - 1 - t]};
  const double x2[1] = {gfit::xi2_of(t)};
  const bool use[1] = {true};
  const double tau = gfit::fit_tau(hh, x2, use, gfit::BlockSum6<kGFitThreads / 32>{red});
  if (t != 0) return;
  if (!(tau > 0.0)) {
    st->warn |= SC_WARN_GAUSS_FALLBACK;
    return;  // the MAD noise stands
  }
  const double sd = gfit::noise_of(tau, k);
  const float sg = __double2float_rn(sd);
  st->sigma_cur_d = sd;
  st->sigma_cur = sg;
  if (pair >= 0) st->sigma[pair] = sg;
}

}  // namespace

cudaError_t launch_gauss_hist(const float* src, long long n, const DevState* st, unsigned long long* ghist, int sms,
                              cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(ghist, 0, sizeof(unsigned long long) * kGBins, s);
  if (e != cudaSuccess) return e;
  const long long want = (n / 4 + 2 * kGHThreads - 1) / (2 * kGHThreads);
  const int grid = (int)(want < 1 ? 1 : (want > 4LL * sms ? 4LL * sms : want));
  k_gauss_hist<<<grid, kGHThreads, 0, s>>>(src, n, st, ghist);
  return cudaGetLastError();
}

cudaError_t launch_gauss_fit(DevState* st, const unsigned long long* ghist, int pair, int clip, cudaStream_t s) {
  k_gauss_fit<<<1, kGFitThreads, 0, s>>>(st, ghist, pair, clip);
  return cudaGetLastError();
}

}  // namespace sc
