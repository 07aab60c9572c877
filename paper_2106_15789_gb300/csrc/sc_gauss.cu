// Gaussian-fit noise mode: the noise of an array is the width of the
// least-squares Gaussian, centred at 0, through a 256-bin histogram of its
// finite values over about +-5 MAD noises.
//
// The paper only says that the RMS noise is measured robustly (Sect. 4.1); this
// mode is the library's own definition, run after the exact MAD measurement:
//   k = fl32(128 / (5 sigma_M))                  bins per data unit
//   bin(s) = floor(fl32(s * k)) + 128            kept when in [0, 256)
//   xi_i = (i + 0.5) / 128 - 1                   bin centres (half-range units)
//   minimise sum_i (h_i - A exp(-xi_i^2 / (2 tau^2)))^2 over A and tau
//   sigma = tau * 128 / k
// For a fixed tau the best A is sum(h g) / sum(g^2), and the profile is
// stationary where
//   D(tau) = sum(g^2) sum(h xi^2 g) - sum(h g) sum(xi^2 g^2) = 0.
// D > 0 for Gaussians much narrower than the counts and D < 0 for much wider
// ones, so bisection over tau in [0.05, 0.8], keeping D(lo) > 0 >= D(hi),
// finds the root to the last bit (the kernel takes Newton steps inside that
// bracket to the same root). Without a sign change at the bracket's ends
// the MAD noise stands (SC_WARN_GAUSS_FALLBACK); a zero MAD noise stays zero.
//
// k_gauss_hist is a streaming pass over the array (4 bytes a value, HBM
// bound); k_gauss_fit is one block of 128 threads, one per mirror pair of
// bins, in float64.
#include "sc_internal.h"

namespace sc {
namespace {

constexpr int kGBins = kGaussBins;
constexpr int kGHalf = kGBins / 2;
constexpr int kGHThreads = 512;
constexpr int kGHWarps = kGHThreads / 32;
constexpr double kGRange = 5.0;  // half-range in MAD noises
constexpr double kGTauLo = 0.05, kGTauHi = 0.8;

__device__ __forceinline__ void ghist_add(unsigned int* h, float s, float k) {
  // NaN and +-Inf fail both compares; so does every value outside the bins
  const float q = floorf(__fmul_rn(s, k));
  if (q >= -(float)kGHalf && q < (float)kGHalf) atomicAdd(h + (int)q + kGHalf, 1u);
}

// Per-warp histograms in shared memory (a warp's lanes still collide on the
// central bins, other warps do not), summed into the global 64-bit counts.
__global__ void __launch_bounds__(kGHThreads) k_gauss_hist(const float* __restrict__ src, long long n,
                                                           const DevState* st, unsigned long long* ghist) {
  __shared__ unsigned int sh[kGHWarps][kGBins];
  if (st->plan.flags & PLAN_EMPTY) return;
  const double sm = st->sigma_cur_d;
  if (!(sm > 0.0)) return;
  const float k = __double2float_rn((double)kGHalf / (kGRange * sm));
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

// Sum of v over the fit block's 128 threads in a fixed order (xor tree in
// each warp, then warps 0..3 in turn); every thread gets the same totals.
constexpr int kGFitThreads = kGHalf;
__device__ __forceinline__ void block_sum6(double v[6], double (*red)[6]) {
#pragma unroll
  for (int j = 0; j < 6; ++j)
    for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_xor_sync(0xffffffffu, v[j], o);
  const int warp = threadIdx.x >> 5;
  __syncthreads();  // the previous call's readers are done with red
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int j = 0; j < 6; ++j) red[warp][j] = v[j];
  __syncthreads();
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    double t = 0.0;
    for (int w = 0; w < kGFitThreads / 32; ++w) t += red[w][j];
    v[j] = t;
  }
}

// D(tau) and dD/dtau over the folded bins. Thread t holds the mirror pair of
// bins 128 + t and 127 - t, which share xi^2 = ((t + 0.5) / 128)^2, with
// H = their summed counts. Over half the bins,
//   A = sum g^2, B = sum H xi^2 g, C = sum H g, E = sum xi^2 g^2,
// and the full-histogram D is 2 (A B - C E): same sign, same root. With
// dg/dtau = g xi^2 / tau^3 (F = sum H xi^4 g, G = sum xi^4 g^2):
//   d(A B - C E)/dtau = (E B + A F - 2 C G) / tau^3.
__device__ __forceinline__ double gauss_d(double tau, double hh, double x2, double (*red)[6], double* slope) {
  const double c = 0.5 / (tau * tau);
  const double g = exp(-x2 * c);
  const double gg = g * g, hg = hh * g;
  double v[6] = {gg, hg * x2, hg, gg * x2, hg * x2 * x2, gg * x2 * x2};
  block_sum6(v, red);
  *slope = (__dmul_rn(v[3], v[1]) + __dmul_rn(v[0], v[4]) - 2.0 * __dmul_rn(v[2], v[5])) / (tau * tau * tau);
  return __dsub_rn(__dmul_rn(v[0], v[1]), __dmul_rn(v[2], v[3]));
}

// The root of D in [0.05, 0.8] by Newton steps kept inside the bracket
// (a step that would leave it bisects instead); D(lo) > 0 >= D(hi) holds
// throughout, so this converges to the root the bisection of the definition
// converges to, within the rounding of the sums.
__global__ void __launch_bounds__(kGFitThreads) k_gauss_fit(DevState* st, const unsigned long long* ghist, int pair,
                                                            int clip) {
  __shared__ double red[kGFitThreads / 32][6];
  const int flags = st->plan.flags;
  const double sm = st->sigma_cur_d;
  __syncthreads();  // every thread has read the plan before thread 0 rewrites it
  if (flags & PLAN_EMPTY) return;
  // the clip of this measurement needs a pass of its own once sigma is known
  if (clip && threadIdx.x == 0) st->plan.flags = flags | PLAN_CLIP | PLAN_CLIP_FULL;
  if (!(sm > 0.0)) return;  // sigma stays 0: the clip adds nothing
  const float k = __double2float_rn((double)kGHalf / (kGRange * sm));
  const int t = threadIdx.x;
  const double xi = ((double)(kGHalf + t) + 0.5) / (double)kGHalf - 1.0;
  const double x2 = xi * xi;
  const double hh = (double)ghist[kGHalf + t] + (double)ghist[kGHalf - 1 - t];
  double lo = kGTauLo, hi = kGTauHi, slope = 0.0;
  const bool bracket = gauss_d(lo, hh, x2, red, &slope) > 0.0 && gauss_d(hi, hh, x2, red, &slope) < 0.0;
  double tau = 0.5 * (lo + hi);
  if (bracket) {
    // every thread holds the same totals, so the loop is block-uniform
    for (int it = 0; it < 200; ++it) {
      const double d = gauss_d(tau, hh, x2, red, &slope);
      if (d == 0.0) break;
      if (d > 0.0) {
        lo = tau;
      } else {
        hi = tau;
      }
      double next = tau - d / slope;
      if (fabs(next - tau) <= 0x1p-50 * tau) {  // converged: keep the step, inside the bracket
        tau = fmin(fmax(next, lo), hi);
        break;
      }
      if (!(next > lo && next < hi)) next = 0.5 * (lo + hi);
      if (hi - lo <= 0x1p-50 * tau) {
        tau = 0.5 * (lo + hi);
        break;
      }
      tau = next;
    }
  }
  if (t != 0) return;
  if (!bracket) {
    st->warn |= SC_WARN_GAUSS_FALLBACK;
    return;  // the MAD noise stands
  }
  const double sd = tau * (double)kGHalf / (double)k;
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
