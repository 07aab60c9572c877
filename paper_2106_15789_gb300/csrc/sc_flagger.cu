// Auto-flagger (SoFiA 2 Sect. 4.1): channels and spatial pixels whose noise
// deviates from the median noise across all channels / pixels by more than k
// times the MAD-based RMS are blanked.
//
//   k_chan_noise   one block per channel: the noise of its plane (exact
//                  median and MAD by radix selection over the plane streamed
//                  from memory, or compensated sums for STD)
//   k_pix_noise    one block per 32 pixels of a row: their spectra staged in
//                  shared memory, each pixel's noise by one warp with the
//                  spectrum in registers (exact selections by bisection on
//                  the keys)
//   k_noise_stats  one block: median M and MAD-based RMS R of a noise array
//   k_flag         flags: |noise - M| > k R
//   k_blank        out = NaN on flagged channels and pixels, else in
//
// The noises are kept in float32; M, R and the flag test are in double.
#include <cstdint>

#include "sc_device.cuh"
#include "sc_gaussfit.cuh"
#include "sc_internal.h"

namespace sc {
namespace flag {

constexpr int kThreads = 1024;
constexpr int kWarps = kThreads / 32;
constexpr int kBins = 2048;
constexpr unsigned kNone = 0xffffffffu;
constexpr double kMadToSigma = 1.4826;

struct Scratch {
  unsigned hist[kBins];
  unsigned part[kWarps + 1];
  unsigned digit, rank, next, count;
  double dpart[kWarps + 1];
};

__device__ __forceinline__ void hist_add_warp(unsigned* hist, unsigned bin) {
  const unsigned peers = __match_any_sync(0xffffffffu, bin);
  if ((threadIdx.x & 31) == __ffs(peers) - 1 && bin < (unsigned)kBins) atomicAdd(&hist[bin], __popc(peers));
}

__device__ __forceinline__ unsigned block_scan_incl(unsigned v, unsigned* part) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned t = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += t;
  }
  if (lane == 31) part[warp] = x;
  __syncthreads();
  if (warp == 0) {
    const unsigned w = part[lane];
    unsigned wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    part[lane] = wi - w;
  }
  __syncthreads();
  return part[warp] + x;
}

__device__ __forceinline__ double block_sum_d(double v, double* part) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) part[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double t = lane < kWarps ? part[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) part[32] = t;
  }
  __syncthreads();
  const double r = part[32];
  __syncthreads();
  return r;
}

__device__ __forceinline__ void neumaier_add(float* s, float* c, float x) {
  const float t = __fadd_rn(*s, x);
  const float e = fabsf(*s) >= fabsf(x) ? __fadd_rn(__fsub_rn(*s, t), x) : __fadd_rn(__fsub_rn(x, t), *s);
  *c = __fadd_rn(*c, e);
  *s = t;
}

__device__ __forceinline__ float two_diff(float x, float b, float* err) {
  const float s = __fsub_rn(x, b);
  const float bb = __fsub_rn(s, x);
  *err = __fadd_rn(__fsub_rn(x, __fsub_rn(s, bb)), __fsub_rn(-b, bb));
  return s;
}

// The float of |x - m|, m = (a + b) / 2 (a == b for an odd count): correctly
// rounded for an odd count, faithfully (TwoSum) for an even one.
__device__ __forceinline__ unsigned mad_key(float x, float a, float b, bool even) {
  float d;
  if (!even) {
    d = __fsub_rn(x, a);
  } else {
    float e1, e2;
    const float t = two_diff(x, 0.5f * a, &e1);
    const float u = two_diff(t, 0.5f * b, &e2);
    d = __fadd_rn(u, __fadd_rn(e1, e2));
  }
  return __float_as_uint(fabsf(d)) | 0x80000000u;
}

// Order statistic `rank` (and, with want_next, rank + 1) of key_of(x) over
// the finite values x of src[0 .. n), streamed from memory: radix digits of
// 11, 11 and 10 bits counted in a shared histogram. All threads call it.
template <class KeyOf>
__device__ unsigned stream_select(const float* __restrict__ src, long long n, unsigned rank, KeyOf key_of,
                                  Scratch* S, bool want_next, unsigned* next) {
  const int tid = threadIdx.x, lane = tid & 31;
  unsigned prefix = 0u, pmask = 0u;
  for (int round = 0; round < 3; ++round) {
    const int shift = round == 0 ? 21 : (round == 1 ? 10 : 0);
    const unsigned dmask = round == 2 ? 0x3ffu : 0x7ffu;
    for (int i = tid; i < kBins; i += kThreads) S->hist[i] = 0u;
    __syncthreads();
    for (long long base = tid - lane; base < n; base += kThreads) {
      const long long i = base + lane;
      const float x = i < n ? __ldg(src + i) : __int_as_float(0x7fc00000);
      const unsigned k = isfinite(x) ? key_of(x) : kNone;
      hist_add_warp(S->hist, (k != kNone && (k & pmask) == prefix) ? (k >> shift) & dmask : (unsigned)kBins);
    }
    __syncthreads();
    const unsigned a = S->hist[2 * tid], b = S->hist[2 * tid + 1];
    const unsigned incl = block_scan_incl(a + b, S->part);
    const unsigned excl = incl - a - b;
    if (rank >= excl && rank < excl + a) {
      S->digit = 2u * tid;
      S->rank = rank - excl;
    } else if (rank >= excl + a && rank < incl) {
      S->digit = 2u * tid + 1u;
      S->rank = rank - excl - a;
    }
    __syncthreads();
    const unsigned d = S->digit;
    rank = S->rank;
    prefix |= d << shift;
    pmask |= dmask << shift;
    if (round == 2 && want_next) {
      if (tid == 0) S->next = (rank + 1u < S->hist[d]) ? prefix : kNone;
      __syncthreads();
      if (S->next == kNone) {
        for (int i = (int)d + 1 + tid; i < 1024; i += kThreads)
          if (S->hist[i] != 0u) atomicMin(&S->next, (prefix & ~dmask) | (unsigned)i);
        __syncthreads();
        if (S->next == kNone) {
          for (long long i = tid; i < n; i += kThreads) {
            const float x = __ldg(src + i);
            if (isfinite(x)) {
              const unsigned k = key_of(x);
              if (k > prefix) atomicMin(&S->next, k);
            }
          }
          __syncthreads();
        }
      }
      *next = S->next;
    }
    __syncthreads();
  }
  return prefix;
}

// Noise of the finite values of src[0 .. n) (NaN if none) in the S+C sense
// (mode SC_NOISE_MAD, _STD or _GAUSS); for MAD mode also the median m (the
// stats kernel needs it). All threads call it and get the same values.
__device__ void block_noise(const float* __restrict__ src, long long n, int mode, Scratch* S, double* sigma,
                            double* median) {
  const bool std_mode = mode == SC_NOISE_STD;
  const int tid = threadIdx.x, lane = tid & 31;
  // finite count
  unsigned c = 0u;
  for (long long i = tid; i < n; i += kThreads) c += isfinite(__ldg(src + i)) ? 1u : 0u;
  c = __reduce_add_sync(0xffffffffu, c);
  if (tid == 0) S->count = 0u;
  __syncthreads();
  if (lane == 0) atomicAdd(&S->count, c);
  __syncthreads();
  const unsigned nf = S->count;
  __syncthreads();
  if (nf == 0u) {
    *sigma = __longlong_as_double(0x7ff8000000000000LL);
    *median = *sigma;
    return;
  }
  if (std_mode) {
    float s = 0.0f, sc = 0.0f;
    for (long long i = tid; i < n; i += kThreads) {
      const float x = __ldg(src + i);
      if (isfinite(x)) neumaier_add(&s, &sc, x);
    }
    const double mean = block_sum_d((double)s + (double)sc, S->dpart) / (double)nf;
    const float mh = __double2float_rn(mean), ml = __double2float_rn(mean - (double)mh);
    float q = 0.0f, qc = 0.0f;
    for (long long i = tid; i < n; i += kThreads) {
      const float x = __ldg(src + i);
      if (isfinite(x)) {
        const float d = __fsub_rn(__fsub_rn(x, mh), ml);
        neumaier_add(&q, &qc, __fmul_rn(d, d));
      }
    }
    const double qq = block_sum_d((double)q + (double)qc, S->dpart);
    *sigma = nf > 1u ? sqrt(qq / (double)(nf - 1u)) : 0.0;
    *median = mean;
    return;
  }
  const unsigned r1 = (nf - 1u) / 2u;
  const bool even = (nf & 1u) == 0u;
  unsigned k2 = 0u;
  const unsigned k1 = stream_select(src, n, r1, [](float x) { return fkey(x); }, S, even, &k2);
  const float ma = fkey_inv(k1), mb = even ? fkey_inv(k2) : ma;
  unsigned a2 = 0u;
  const unsigned a1 =
      stream_select(src, n, r1, [=](float x) { return mad_key(x, ma, mb, even); }, S, even, &a2);
  const double mad = even ? 0.5 * ((double)fkey_inv(a1) + (double)fkey_inv(a2)) : (double)fkey_inv(a1);
  *sigma = kMadToSigma * mad;
  *median = even ? 0.5 * ((double)ma + (double)mb) : (double)ma;
  if (mode == SC_NOISE_GAUSS && *sigma > 0.0) {
    // the 256-bin histogram of the finite values, then the fit (the MAD noise
    // stands without a root)
    const float k = gfit::scale_of(*sigma);
    __syncthreads();  // the selection is done with S->hist
    for (int i = tid; i < gfit::kBins; i += kThreads) S->hist[i] = 0u;
    __syncthreads();
    for (long long i = tid; i < n; i += kThreads) {
      const int b = gfit::bin_of(__ldg(src + i), k);
      if (b >= 0) atomicAdd(&S->hist[b], 1u);
    }
    __syncthreads();
    // one warp fits (four folded bins a lane, no block barriers); the others wait
    if (tid < 32) {
      double hh[4], x2[4];
      bool use[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int t = lane + 32 * j;
        hh[j] = (double)S->hist[gfit::kHalf + t] + (double)S->hist[gfit::kHalf - 1 - t];
        x2[j] = gfit::xi2_of(t);
        use[j] = true;
      }
      const double tau = gfit::fit_tau(hh, x2, use, gfit::WarpSum6{});
      if (lane == 0) S->dpart[0] = tau;
    }
    __syncthreads();
    const double tau = S->dpart[0];
    if (tau > 0.0) *sigma = gfit::noise_of(tau, k);
    __syncthreads();
  }
}

// ---- per-pixel noise: a warp per pixel, the spectrum in registers ----------
constexpr int kPixWarps = 8;
constexpr int kPixThreads = 32 * kPixWarps;

// Order statistic `rank` of the VPL keys per lane held by a warp, by
// bisection on the 32-bit key (keys kNone never count).
template <int VPL>
__device__ __forceinline__ unsigned warp_select(const unsigned (&k)[VPL], unsigned rank) {
  unsigned ans = 0u;
  for (int bit = 31; bit >= 0; --bit) {
    const unsigned t = ans | (1u << bit);
    unsigned c = 0u;
#pragma unroll
    for (int i = 0; i < VPL; ++i) c += k[i] < t ? 1u : 0u;
    c = __reduce_add_sync(0xffffffffu, c);
    if (c <= rank) ans = t;
  }
  return ans;
}

}  // namespace flag

__global__ void __launch_bounds__(flag::kThreads, 1)
    k_chan_noise(const float* __restrict__ cube, long long plane, int nz, int mode, float* __restrict__ noise) {
  __shared__ flag::Scratch S;
  for (int z = blockIdx.x; z < nz; z += gridDim.x) {
    double sigma, m;
    flag::block_noise(cube + (long long)z * plane, plane, mode, &S, &sigma, &m);
    if (threadIdx.x == 0) noise[z] = __double2float_rn(sigma);
    __syncthreads();
  }
}

// stats[0] = median M, stats[1] = R = 1.4826 * MAD of the finite noises
// (NaN if none).
__global__ void __launch_bounds__(flag::kThreads, 1) k_noise_stats(const float* __restrict__ noise, long long n,
                                                                   double* stats) {
  __shared__ flag::Scratch S;
  double sigma, m;
  flag::block_noise(noise, n, SC_NOISE_MAD, &S, &sigma, &m);
  if (threadIdx.x == 0) {
    stats[0] = m;
    stats[1] = sigma;
  }
}

template <int VPL>
__global__ void __launch_bounds__(flag::kPixThreads) k_pix_noise(const float* __restrict__ cube, int nx, int ny,
                                                                 int nz, int mode, float* __restrict__ noise) {
  using namespace flag;
  extern __shared__ float tile[];  // [nz][33]: 32 pixels of a row (one padding column)
  // Gaussian-fit mode: then 256 counts per warp
  unsigned* const whist = reinterpret_cast<unsigned*>(tile + 33 * nz) + (threadIdx.x >> 5) * gfit::kBins;
  const bool std_mode = mode == SC_NOISE_STD;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long plane = (long long)nx * ny;
  const int xtiles = (nx + 31) / 32;
  const long long ntiles = (long long)xtiles * ny;
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int y = (int)(t / xtiles), x0 = (int)(t - (long long)y * xtiles) * 32;
    __syncthreads();  // the tile of the previous iteration is consumed
    for (int z = warp; z < nz; z += kPixWarps) {
      const int x = x0 + lane;
      tile[z * 33 + lane] = x < nx ? __ldg(cube + (long long)z * plane + (long long)y * nx + x)
                                   : __int_as_float(0x7fc00000);
    }
    __syncthreads();
    for (int p = warp; p < 32 && x0 + p < nx; p += kPixWarps) {
      float v[VPL];
      unsigned k[VPL];
      unsigned nfl = 0u;
#pragma unroll
      for (int i = 0; i < VPL; ++i) {
        const int z = lane + 32 * i;
        v[i] = z < nz ? tile[z * 33 + p] : __int_as_float(0x7fc00000);
        const bool ok = isfinite(v[i]);
        k[i] = ok ? fkey(v[i]) : kNone;
        nfl += ok ? 1u : 0u;
      }
      const unsigned nf = __reduce_add_sync(0xffffffffu, nfl);
      float out;
      if (nf == 0u) {
        out = __int_as_float(0x7fc00000);
      } else if (std_mode) {
        float s = 0.0f, sc = 0.0f;
#pragma unroll
        for (int i = 0; i < VPL; ++i)
          if (k[i] != kNone) neumaier_add(&s, &sc, v[i]);
        double ds = (double)s + (double)sc;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ds += __shfl_xor_sync(0xffffffffu, ds, o);
        const double mean = ds / (double)nf;
        const float mh = __double2float_rn(mean), ml = __double2float_rn(mean - (double)mh);
        float q = 0.0f, qc = 0.0f;
#pragma unroll
        for (int i = 0; i < VPL; ++i)
          if (k[i] != kNone) {
            const float d = __fsub_rn(__fsub_rn(v[i], mh), ml);
            neumaier_add(&q, &qc, __fmul_rn(d, d));
          }
        double dq = (double)q + (double)qc;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dq += __shfl_xor_sync(0xffffffffu, dq, o);
        out = __double2float_rn(nf > 1u ? sqrt(dq / (double)(nf - 1u)) : 0.0);
      } else {
        const unsigned r1 = (nf - 1u) / 2u;
        const bool even = (nf & 1u) == 0u;
        const unsigned k1 = warp_select<VPL>(k, r1);
        const unsigned k2 = even ? warp_select<VPL>(k, r1 + 1u) : k1;
        const float ma = fkey_inv(k1), mb = fkey_inv(k2);
#pragma unroll
        for (int i = 0; i < VPL; ++i)
          if (k[i] != kNone) k[i] = mad_key(v[i], ma, mb, even);
        const unsigned a1 = warp_select<VPL>(k, r1);
        const unsigned a2 = even ? warp_select<VPL>(k, r1 + 1u) : a1;
        const double mad = 0.5 * ((double)fkey_inv(a1) + (double)fkey_inv(a2));
        double sigma = kMadToSigma * mad;
        if (mode == SC_NOISE_GAUSS && sigma > 0.0) {
          // the spectrum's 256-bin histogram in this warp's counts, then a
          // warp-wide fit over the 128 folded bins (4 a lane)
          for (int i = lane; i < gfit::kBins; i += 32) whist[i] = 0u;
          __syncwarp();
          const float ks = gfit::scale_of(sigma);
#pragma unroll
          for (int i = 0; i < VPL; ++i) {
            const int b = gfit::bin_of(v[i], ks);  // NaN (and padding) give -1
            if (b >= 0) atomicAdd(whist + b, 1u);
          }
          __syncwarp();
          double hh[4], x2[4];
          bool use[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int t = lane + 32 * j;
            hh[j] = (double)whist[gfit::kHalf + t] + (double)whist[gfit::kHalf - 1 - t];
            x2[j] = gfit::xi2_of(t);
            use[j] = true;
          }
          const double tau = gfit::fit_tau(hh, x2, use, gfit::WarpSum6{});
          if (tau > 0.0) sigma = gfit::noise_of(tau, ks);
          __syncwarp();  // the counts are reset by the next pixel
        }
        out = __double2float_rn(sigma);
      }
      if (lane == 0) noise[(long long)y * nx + x0 + p] = out;
    }
  }
}

__global__ void k_flag(const float* __restrict__ noise, long long n, const double* __restrict__ stats, double k,
                       uint8_t* __restrict__ flags) {
  const double m = stats[0], r = stats[1];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float v = noise[i];
    flags[i] = (isfinite(v) && isfinite(m) && fabs((double)v - m) > k * r) ? 1 : 0;
  }
}

__global__ void k_blank(const float* in, float* out, int nx, int ny, int nz, const uint8_t* __restrict__ fchan,
                        const uint8_t* __restrict__ fpix) {
  const long long plane = (long long)nx * ny, n = plane * nz;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
    const long long z = v / plane, p = v - z * plane;
    const bool f = (fchan && fchan[z]) || (fpix && fpix[p]);
    out[v] = f ? __int_as_float(0x7fc00000) : in[v];
  }
}

// ---------------------------------------------------------------------------
namespace {
template <int VPL>
cudaError_t launch_pix(const float* cube, int nx, int ny, int nz, int mode, float* noise, int sms,
                       cudaStream_t s) {
  const size_t smem = sizeof(float) * 33 * (size_t)nz +
                      (mode == SC_NOISE_GAUSS ? sizeof(unsigned) * gfit::kBins * flag::kPixWarps : 0);
  cudaFuncSetAttribute(k_pix_noise<VPL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const long long tiles = (long long)((nx + 31) / 32) * ny;
  const int grid = (int)(tiles < 4LL * sms ? tiles : 4LL * sms);
  k_pix_noise<VPL><<<grid, flag::kPixThreads, smem, s>>>(cube, nx, ny, nz, mode, noise);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_autoflag(const float* cube, const long long dims[3], double k, int channels, int pixels,
                            int mode, float* out, float* chan_noise, float* pix_noise, uint8_t* chan_flags,
                            uint8_t* pix_flags, double* stats, int sms, cudaStream_t s) {
  const int nx = (int)dims[0], ny = (int)dims[1], nz = (int)dims[2];
  const long long plane = (long long)nx * ny, n = plane * nz;
  cudaError_t e = cudaSuccess;
  if (channels) {
    k_chan_noise<<<nz < 2 * sms ? nz : 2 * sms, flag::kThreads, 0, s>>>(cube, plane, nz, mode, chan_noise);
    k_noise_stats<<<1, flag::kThreads, 0, s>>>(chan_noise, nz, stats);
    k_flag<<<(nz + 255) / 256, 256, 0, s>>>(chan_noise, nz, stats, k, chan_flags);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (pixels) {
    if (nz <= 256) e = launch_pix<8>(cube, nx, ny, nz, mode, pix_noise, sms, s);
    else if (nz <= 512) e = launch_pix<16>(cube, nx, ny, nz, mode, pix_noise, sms, s);
    else if (nz <= 1024) e = launch_pix<32>(cube, nx, ny, nz, mode, pix_noise, sms, s);
    else e = launch_pix<48>(cube, nx, ny, nz, mode, pix_noise, sms, s);
    if (e != cudaSuccess) return e;
    k_noise_stats<<<1, flag::kThreads, 0, s>>>(pix_noise, plane, stats + 2);
    const long long g = (plane + 255) / 256;
    k_flag<<<(unsigned)(g < 16LL * sms ? g : 16LL * sms), 256, 0, s>>>(pix_noise, plane, stats + 2, k, pix_flags);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  const long long gb = (n + 255) / 256;
  k_blank<<<(unsigned)(gb < 16LL * sms ? gb : 16LL * sms), 256, 0, s>>>(cube, out, nx, ny, nz,
                                                                      channels ? chan_flags : nullptr,
                                                                      pixels ? pix_flags : nullptr);
  return cudaGetLastError();
}

}  // namespace sc
