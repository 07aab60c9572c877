// Gaussian-fit noise, the parts every kernel that measures it shares: the bin
// rule and the least-squares fit. The definition (the library's own; the
// paper only asks for a robust noise, Sect. 4.1):
//   k = fl32(128 / (5 sigma_M))              bins per data unit, sigma_M the MAD noise
//   bin(s) = floor(fl32(s * k)) + 128        kept when in [0, 256)
//   xi_i = (i + 0.5) / 128 - 1               bin centres in half-range units
//   minimise sum_i (h_i - A exp(-xi_i^2 / (2 tau^2)))^2 over A and tau
//   noise = tau * 128 / k
// For a fixed tau the best A is sum(h g) / sum(g^2); the profile is stationary
// where D(tau) = sum(g^2) sum(h xi^2 g) - sum(h g) sum(xi^2 g^2) = 0, which is
// positive for Gaussians much narrower than the counts and negative for much
// wider ones. tau is the root in [0.05, 0.8] (bisected to the last bit by the
// definition; reached here by Newton steps that stay inside the bracket).
// Without a sign change at the bracket's ends the MAD noise stands.
//
// Bins 128 + t and 127 - t share xi^2 = ((t + 0.5) / 128)^2, so the fit works
// on 128 folded bins with H_t = h_{128+t} + h_{127-t}: over half the bins,
//   A = sum g^2, B = sum H xi^2 g, C = sum H g, E = sum xi^2 g^2,
// the full-histogram D is 2 (A B - C E) (same sign, same root), and with
// dg/dtau = g xi^2 / tau^3, F = sum H xi^4 g, G = sum xi^4 g^2:
//   d(A B - C E)/dtau = (E B + A F - 2 C G) / tau^3.
#pragma once

#include <cuda_runtime.h>

namespace sc {
namespace gfit {

constexpr int kBins = 256;
constexpr int kHalf = kBins / 2;
constexpr double kRange = 5.0;  // half-range in MAD noises
constexpr double kTauLo = 0.05, kTauHi = 0.8;

__device__ __forceinline__ float scale_of(double sigma_mad) {
  return __double2float_rn((double)kHalf / (kRange * sigma_mad));
}

// Bin of s, or -1 (outside the bins; NaN and Inf fail both compares).
__device__ __forceinline__ int bin_of(float s, float k) {
  const float q = floorf(__fmul_rn(s, k));
  return (q >= -(float)kHalf && q < (float)kHalf) ? (int)q + kHalf : -1;
}

// xi^2 of folded bin t (bins kHalf + t and kHalf - 1 - t).
__device__ __forceinline__ double xi2_of(int t) {
  const double xi = ((double)(kHalf + t) + 0.5) / (double)kHalf - 1.0;
  return xi * xi;
}

// Sums of v[6] over WARPS warps of a block in a fixed order (xor tree in each
// warp, then warps 0.. in turn, added by lanes 0..5 of warp 0: float64 adds
// are slow on this part, so only six threads make the totals); every thread
// gets the same totals. red holds (WARPS + 1) x 6 doubles of shared memory;
// every thread of the block calls it.
template <int WARPS>
struct BlockSum6 {
  double (*red)[6];
  __device__ __forceinline__ void operator()(double (&v)[6]) const {
#pragma unroll
    for (int j = 0; j < 6; ++j)
      for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_xor_sync(0xffffffffu, v[j], o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();  // the previous call's readers are done with red
    if (lane == 0)
#pragma unroll
      for (int j = 0; j < 6; ++j) red[warp][j] = v[j];
    __syncthreads();
    if (warp == 0 && lane < 6) {
      double t = 0.0;
      for (int w = 0; w < WARPS; ++w) t += red[w][lane];
      red[WARPS][lane] = t;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 6; ++j) v[j] = red[WARPS][j];
  }
};

// The same over the 32 lanes of one warp.
struct WarpSum6 {
  __device__ __forceinline__ void operator()(double (&v)[6]) const {
#pragma unroll
    for (int j = 0; j < 6; ++j)
      for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_xor_sync(0xffffffffu, v[j], o);
  }
};

// D(tau) (in the folded form A B - C E) and its slope. A thread holds PER
// folded bins: counts hh[j] and xi^2 x2[j]; use[j] false adds nothing.
template <int PER, class Reduce>
__device__ __forceinline__ double eval_d(double tau, const double (&hh)[PER], const double (&x2)[PER],
                                         const bool (&use)[PER], const Reduce& reduce, double* slope) {
  const double c = 0.5 / (tau * tau);
  double v[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    if (!use[j]) continue;
    const double g = exp(-x2[j] * c);
    const double gg = g * g, hg = hh[j] * g;
    v[0] += gg;
    v[1] += hg * x2[j];
    v[2] += hg;
    v[3] += gg * x2[j];
    v[4] += hg * x2[j] * x2[j];
    v[5] += gg * x2[j] * x2[j];
  }
  reduce(v);
  *slope = (__dmul_rn(v[3], v[1]) + __dmul_rn(v[0], v[4]) - 2.0 * __dmul_rn(v[2], v[5])) / (tau * tau * tau);
  return __dsub_rn(__dmul_rn(v[0], v[1]), __dmul_rn(v[2], v[3]));
}

// tau of the fit, or -1 when the bracket's ends do not straddle a root. Every
// thread of the reduction group calls it and gets the same answer (the
// reduction hands every thread identical totals, so every branch is uniform).
template <int PER, class Reduce>
__device__ double fit_tau(const double (&hh)[PER], const double (&x2)[PER], const bool (&use)[PER],
                          const Reduce& reduce) {
  double lo = kTauLo, hi = kTauHi, slope = 0.0;
  const bool bracket = eval_d(lo, hh, x2, use, reduce, &slope) > 0.0 && eval_d(hi, hh, x2, use, reduce, &slope) < 0.0;
  if (!bracket) return -1.0;
  double tau = 1.0 / kRange;  // the MAD noise's own width: close to the root for noise-like data
  for (int it = 0; it < 200; ++it) {
    const double d = eval_d(tau, hh, x2, use, reduce, &slope);
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
  return tau;
}

// The noise from tau and the scale k.
__device__ __forceinline__ double noise_of(double tau, float k) { return tau * (double)kHalf / (double)k; }

}  // namespace gfit
}  // namespace sc
