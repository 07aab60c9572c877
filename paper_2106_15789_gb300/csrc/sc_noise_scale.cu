// Local noise normalisation (SoFiA 2 Sect. 4.1, windows of 31 pixels and
// channels in the speed test of Sect. 5): the cube is divided by the noise
// level measured in a window around each voxel's cell.
//
//   k_noise_window  one block per cell (persistent over cells): the finite
//                   voxels of the cell's window, clipped to the cube, go into
//                   shared memory as order-preserving keys; the noise of the
//                   chosen mode comes from them: MAD by two exact radix
//                   selections in shared memory (the median, then the median
//                   of |x - m| with the same key rounding as the S+C noise),
//                   STD by two double-precision passes. Writes the cell's
//                   noise (double) and the float32 reciprocal used below.
//   k_noise_apply   out = in * (1 / sigma) per voxel (NaN where the input is
//                   not finite or the cell has no positive noise).
//
// Cells are gx x gy x gz voxels (the last one along an axis may be shorter);
// a cell's window is centred on voxel start + (extent - 1) / 2 of each axis.
#include <cstdint>

#include "sc_device.cuh"
#include "sc_internal.h"

namespace sc {
namespace nscale {

constexpr int kThreads = 1024;
constexpr int kWarps = kThreads / 32;
constexpr int kBins = 2048;              // radix digits: 11, 11 and 10 bits
constexpr unsigned kNone = 0xffffffffu;  // key of a non-finite voxel: above every finite key
constexpr double kMadToSigma = 1.4826;

struct Geo {
  long long nx, ny, nz;
  int wx, wy, wz;     // window (odd)
  int gx, gy, gz;     // cell size
  int ncx, ncy, ncz;  // cells per axis
};

// Window of the cell with index c along an axis of length n: [lo, hi).
__device__ __forceinline__ void window_range(int c, int g, int w, long long n, long long* lo, long long* hi) {
  const long long start = (long long)c * g;
  const long long extent = min((long long)g, n - start);
  const long long centre = start + (extent - 1) / 2;
  const int r = (w - 1) / 2;
  *lo = max(centre - r, 0LL);
  *hi = min(centre + r + 1, n);
}

// Inclusive block scan of one value per thread; returns the block total in
// *total. Uses part[kWarps] of shared scratch (two barriers).
__device__ __forceinline__ unsigned block_scan_incl(unsigned v, unsigned* part, unsigned* total) {
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
    unsigned w = part[lane], wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    part[lane] = wi - w;  // exclusive prefix of the warps
    if (lane == 31) part[32] = wi;
  }
  __syncthreads();
  *total = part[32];
  return part[warp] + x;
}

struct SelScratch {
  unsigned hist[kBins];
  unsigned part[kWarps + 1];
  unsigned digit, rank, next;
};

// Key of order statistic `rank` (0-based) of keys[0 .. n) in shared memory,
// by three rounds of radix digits (11, 11, 10 bits) counted in a shared
// histogram over the keys that share the digits found so far. With want_next,
// *next receives the key of order statistic rank + 1 (the caller guarantees
// it exists). All threads of the block call it and get the same results.
__device__ unsigned block_select(const unsigned* keys, int n, unsigned rank, SelScratch* S, bool want_next,
                                 unsigned* next) {
  const int tid = threadIdx.x;
  unsigned prefix = 0u, pmask = 0u;
  for (int round = 0; round < 3; ++round) {
    const int shift = round == 0 ? 21 : (round == 1 ? 10 : 0);
    const unsigned dmask = round == 2 ? 0x3ffu : 0x7ffu;
    for (int i = tid; i < kBins; i += kThreads) S->hist[i] = 0u;
    __syncthreads();
    for (int e = tid; e < n; e += kThreads) {
      const unsigned k = keys[e];
      if ((k & pmask) == prefix) atomicAdd(&S->hist[(k >> shift) & dmask], 1u);
    }
    __syncthreads();
    // two bins per thread: find the one whose cumulative range holds rank
    const unsigned a = S->hist[2 * tid], b = S->hist[2 * tid + 1];
    unsigned total;
    const unsigned incl = block_scan_incl(a + b, S->part, &total);
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
      // the successor: the same key if it occurs again, else the next
      // non-empty bin of this round, else the smallest larger key
      if (tid == 0) S->next = (rank + 1u < S->hist[d]) ? prefix : kNone;
      __syncthreads();
      if (S->next == kNone) {
        for (int i = (int)d + 1 + tid; i < 1024; i += kThreads)
          if (S->hist[i] != 0u) atomicMin(&S->next, (prefix & ~dmask) | (unsigned)i);
        __syncthreads();
        if (S->next == kNone) {
          for (int e = tid; e < n; e += kThreads) {
            const unsigned k = keys[e];
            if (k > prefix) atomicMin(&S->next, k);
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

__device__ __forceinline__ double key_value(unsigned k) { return (double)fkey_inv(k); }

__device__ __forceinline__ double block_sum_d(double v, double* part) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) part[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (warp == 0) {
    t = lane < kWarps ? part[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) part[32] = t;
  }
  __syncthreads();
  t = part[32];
  __syncthreads();
  return t;
}

}  // namespace nscale

__global__ void __launch_bounds__(nscale::kThreads, 1)
    k_noise_window(const float* __restrict__ cube, nscale::Geo g, int std_mode, double* __restrict__ sig_out,
                   float* __restrict__ rinv_out) {
  using namespace nscale;
  extern __shared__ __align__(16) unsigned char ns_smem[];
  unsigned* const keys = reinterpret_cast<unsigned*>(ns_smem);
  __shared__ SelScratch S;
  __shared__ double dpart[kWarps + 1];
  __shared__ unsigned s_count;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const long long n_cells = (long long)g.ncx * g.ncy * g.ncz;
  const long long plane = g.nx * g.ny;
  for (long long cell = blockIdx.x; cell < n_cells; cell += gridDim.x) {
    const int cx = (int)(cell % g.ncx);
    const int cy = (int)((cell / g.ncx) % g.ncy);
    const int cz = (int)(cell / ((long long)g.ncx * g.ncy));
    long long x0, x1, y0, y1, z0, z1;
    window_range(cx, g.gx, g.wx, g.nx, &x0, &x1);
    window_range(cy, g.gy, g.wy, g.ny, &y0, &y1);
    window_range(cz, g.gz, g.wz, g.nz, &z0, &z1);
    const int lx = (int)(x1 - x0), ly = (int)(y1 - y0), lz = (int)(z1 - z0);
    const int n = lx * ly * lz;
    if (tid == 0) s_count = 0u;
    __syncthreads();
    // the window's keys, one warp per row
    unsigned finite = 0u;
    for (int row = warp; row < ly * lz; row += kWarps) {
      const int dz = row / ly, dy = row - dz * ly;
      const float* src = cube + (z0 + dz) * plane + (y0 + dy) * g.nx + x0;
      for (int dx = lane; dx < lx; dx += 32) {
        const float v = __ldg(src + dx);
        const bool ok = isfinite(v);
        keys[row * lx + dx] = ok ? fkey(v) : kNone;
        finite += ok ? 1u : 0u;
      }
    }
    finite = __reduce_add_sync(0xffffffffu, finite);
    if (lane == 0) atomicAdd(&s_count, finite);
    __syncthreads();
    const unsigned nf = s_count;
    double sigma;
    if (nf == 0u) {
      sigma = __longlong_as_double(0x7ff8000000000000LL);  // NaN: no finite voxel
    } else if (std_mode) {
      double s = 0.0;
      for (int e = tid; e < n; e += kThreads)
        if (keys[e] != kNone) s += key_value(keys[e]);
      const double mean = block_sum_d(s, dpart) / (double)nf;
      double q = 0.0;
      for (int e = tid; e < n; e += kThreads)
        if (keys[e] != kNone) {
          const double d = key_value(keys[e]) - mean;
          q += d * d;
        }
      q = block_sum_d(q, dpart);
      sigma = nf > 1u ? sqrt(q / (double)(nf - 1u)) : 0.0;
    } else {
      // median: order statistics (nf - 1) / 2 and nf / 2
      const unsigned r1 = (nf - 1u) / 2u;
      const bool even = (nf & 1u) == 0u;
      unsigned k2 = 0u;
      const unsigned k1 = block_select(keys, n, r1, &S, even, &k2);
      const double m = even ? 0.5 * (key_value(k1) + key_value(k2)) : key_value(k1);
      // MAD keys: the float of |x - m| (as the S+C noise measures it)
      for (int e = tid; e < n; e += kThreads) {
        const unsigned k = keys[e];
        keys[e] = k == kNone ? kNone : fkey(__double2float_rn(fabs(key_value(k) - m)));
      }
      __syncthreads();
      unsigned a2 = 0u;
      const unsigned a1 = block_select(keys, n, r1, &S, even, &a2);
      const double mad = even ? 0.5 * (key_value(a1) + key_value(a2)) : key_value(a1);
      sigma = kMadToSigma * mad;
    }
    if (tid == 0) {
      sig_out[cell] = sigma;
      rinv_out[cell] = sigma > 0.0 ? __double2float_rn(1.0 / sigma) : __int_as_float(0x7fc00000);
    }
    __syncthreads();  // the keys are overwritten by the next cell
  }
}

__global__ void k_noise_apply(const float* in, float* out, nscale::Geo g, const float* __restrict__ rinv) {
  const long long rows = g.ny * g.nz;
  for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
    const long long z = row / g.ny, y = row - z * g.ny;
    const float* rr = rinv + ((z / g.gz) * g.ncy + y / g.gy) * (long long)g.ncx;
    const float* src = in + row * g.nx;
    float* dst = out + row * g.nx;
    for (int x = threadIdx.x; x < g.nx; x += blockDim.x) {
      const float v = src[x];
      const float r = __ldg(rr + x / g.gx);
      dst[x] = isfinite(v) ? __fmul_rn(v, r) : __int_as_float(0x7fc00000);
    }
  }
}

size_t noise_window_smem(long long window_voxels) { return sizeof(unsigned) * (size_t)window_voxels; }

namespace {
nscale::Geo make_geo(const long long dims[3], const int window[3], const int grid[3]) {
  nscale::Geo g;
  g.nx = dims[0];
  g.ny = dims[1];
  g.nz = dims[2];
  g.wx = window[0];
  g.wy = window[1];
  g.wz = window[2];
  g.gx = grid[0];
  g.gy = grid[1];
  g.gz = grid[2];
  g.ncx = (int)((g.nx + g.gx - 1) / g.gx);
  g.ncy = (int)((g.ny + g.gy - 1) / g.gy);
  g.ncz = (int)((g.nz + g.gz - 1) / g.gz);
  return g;
}
}  // namespace

cudaError_t launch_noise_window(const float* cube, const long long dims[3], const int window[3], const int grid[3],
                                int std_mode, double* sig_dev, float* rinv_dev, int sms, cudaStream_t s) {
  const nscale::Geo g = make_geo(dims, window, grid);
  const long long cells = (long long)g.ncx * g.ncy * g.ncz;
  const long long wvox = (long long)min((long long)g.wx, g.nx) * min((long long)g.wy, g.ny) * min((long long)g.wz, g.nz);
  const int blocks = (int)(cells < sms ? cells : sms);
  k_noise_window<<<blocks, nscale::kThreads, noise_window_smem(wvox), s>>>(cube, g, std_mode, sig_dev, rinv_dev);
  return cudaGetLastError();
}

cudaError_t launch_noise_apply(const float* cube, const long long dims[3], const int window[3], const int grid[3],
                               float* out, const float* rinv_dev, int sms, cudaStream_t s) {
  const nscale::Geo g = make_geo(dims, window, grid);
  const long long rows = g.ny * g.nz;
  const int blocks = (int)(rows < 8LL * sms ? rows : 8LL * sms);
  k_noise_apply<<<blocks, 256, 0, s>>>(cube, out, g, rinv_dev);
  return cudaGetLastError();
}

void init_noise_scale_attrs() {
  cudaFuncSetAttribute(k_noise_window, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)noise_window_smem(kNoiseScaleMaxWindow));
}

}  // namespace sc
