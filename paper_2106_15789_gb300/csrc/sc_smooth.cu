// Smoothing of one S+C kernel pair (SoFiA 2, Sect. 4.2 and 5; Hydra-field
// figure caption in Sect. 7: a spatial Gaussian of given FWHM and a spectral
// boxcar), with the replacement of already-detected voxels (Sect. 6.2).
//
// Arithmetic. The spatial Gaussian is a cascade of three centred boxcars
// (Kovesi 2010 widths), i.e. a 1-D kernel with integer taps a_i summing to
// Wxy = w0 w1 w2; the spectral boxcar has unit taps summing to wz. Inputs are
// quantised once to X_q = rint(X * 2^f) (int64, f chosen per pair from max|X|
// so that no sum can reach 2^62), every sum is exact in int64, and the result
// sum(a_i a_j X_q) is scaled by 2^-f / (Wxy^2 wz) and rounded once to float.
// The smoothed value is therefore the exact convolution of the zero-padded
// cube up to one quantisation (2^-f, far below float resolution) and the final
// rounding, independent of tiling or summation order.
//
// Structure. A block owns a tile of tx x ty output columns and a chunk of lz
// planes. It walks the planes in z: loads the plane's tile with a halo of h
// (zero outside the cube), applies NaN -> 0 and the replacement, quantises,
// runs the x pass and the y pass in shared memory, and pushes the smoothed
// plane into a ring of wz planes that keeps the running spectral sum.
#include <algorithm>

#include <cuda_fp16.h>

#include "sc_device.cuh"
#include "sc_internal.h"

namespace sc {

constexpr int kSmoothThreads = 256;
constexpr int kMaxOuts = 4;  // outputs per thread (tile area <= 1024)

struct SmoothLayout {
  int px, rows;  // quantised-input tile: rows x px (px = tx + 2h, rows = ty + 2h)
  size_t off_x, off_b, off_ring, off_taps, off_hist, total;
};

__host__ __device__ inline SmoothLayout smooth_layout(int tx, int ty, int h, int wz, bool hist) {
  SmoothLayout L;
  L.px = tx + 2 * h;
  L.rows = ty + 2 * h;
  size_t o = 0;
  L.off_x = o;
  o += sizeof(long long) * (size_t)L.rows * L.px;
  L.off_b = o;
  o += (h > 0) ? sizeof(long long) * (size_t)L.rows * tx : 0;
  L.off_ring = o;
  o += sizeof(long long) * (size_t)wz * tx * ty;
  L.off_taps = o;
  o += sizeof(int) * (2 * h + 1);
  o = (o + 15) & ~(size_t)15;
  L.off_hist = o;
  o += hist ? sizeof(unsigned int) * kNumBins : 0;
  L.total = o;
  return L;
}

size_t smooth_smem_bytes(const SmoothArgs& a) {
  return smooth_layout(a.tx, a.ty, a.pd.h, a.pd.wz, a.hist != nullptr).total;
}

// Exact sum of taps[k] * v[k * stride], k < n: 32-bit halves accumulated
// separately (one wide multiply-add each), recombined modulo 2^64.
__device__ __forceinline__ long long fir(const long long* __restrict__ v, int stride, const int* __restrict__ taps,
                                         int n) {
  unsigned long long acc_lo = 0ull;
  long long acc_hi = 0ll;
  for (int k = 0; k < n; ++k) {
    const long long x = v[k * stride];
    const int t = taps[k];
    acc_lo += (unsigned long long)(unsigned int)(x & 0xffffffffll) * (unsigned long long)(unsigned int)t;
    acc_hi += (long long)(int)(x >> 32) * (long long)t;
  }
  return (long long)(acc_lo + ((unsigned long long)acc_hi << 32));
}

__global__ void __launch_bounds__(kSmoothThreads) k_smooth_generic(SmoothArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int h = a.pd.h, wz = a.pd.wz, r = (wz - 1) / 2;
  const int tx = a.tx, ty = a.ty;
  const SmoothLayout L = smooth_layout(tx, ty, h, wz, a.hist != nullptr);
  long long* Xt = reinterpret_cast<long long*>(smem + L.off_x);
  long long* Bt = reinterpret_cast<long long*>(smem + L.off_b);
  long long* ring = reinterpret_cast<long long*>(smem + L.off_ring);
  int* taps = reinterpret_cast<int*>(smem + L.off_taps);
  unsigned int* hist = reinterpret_cast<unsigned int*>(smem + L.off_hist);
  const int tid = threadIdx.x;
  const int ntap = 2 * h + 1;
  for (int i = tid; i < ntap; i += blockDim.x) taps[i] = a.pd.taps[i];
  if (a.hist)
    for (int i = tid; i < kNumBins; i += blockDim.x) hist[i] = 0u;
  const BinCfg cfg = a.win ? a.st->win : kFullRange;
  const float fscale = a.st->fx_scale[a.pair];
  const float inv = a.st->fx_inv[a.pair];
  const long long qrepl = a.st->fx_qrepl[a.pair];
  const bool do_repl = qrepl > 0 && a.mbits != nullptr;
  const long long nx = a.nx, ny = a.ny, nz = a.nz;
  const int area = tx * ty;
  const long long n_items = (long long)a.tiles_x * a.tiles_y * a.zchunks;
  __syncthreads();

  for (long long item = blockIdx.x; item < n_items; item += gridDim.x) {
    const int tile = (int)(item % ((long long)a.tiles_x * a.tiles_y));
    const int zc = (int)(item / ((long long)a.tiles_x * a.tiles_y));
    const int x0 = (tile % a.tiles_x) * tx, y0 = (tile / a.tiles_x) * ty;
    const int z0 = zc * a.lz;
    const int z1 = min((long long)z0 + a.lz, nz);
    long long zsum[kMaxOuts];
#pragma unroll
    for (int i = 0; i < kMaxOuts; ++i) zsum[i] = 0ll;
    for (int i = tid; i < wz * area; i += blockDim.x) ring[i] = 0ll;
    __syncthreads();
    const int n_steps = (z1 - z0) + 2 * r;
    for (int j = 0; j < n_steps; ++j) {
      const int zp = z0 - r + j;
      const bool valid = (zp >= 0 && zp < nz);
      long long P[kMaxOuts];
      if (valid) {
        const long long pbase = (long long)zp * ny * nx;
        const float cs = a.h16.fmt ? __ldg(a.h16.scale + zp) : 1.0f;
        for (int e = tid; e < L.rows * L.px; e += blockDim.x) {
          const int row = e / L.px, col = e - row * L.px;
          const long long gx = (long long)x0 - h + col, gy = (long long)y0 - h + row;
          long long q = 0ll;
          if (gx >= 0 && gx < nx && gy >= 0 && gy < ny) {
            const long long v = pbase + gy * nx + gx;
            const float c = a.h16.fmt ? half16_value(__ldg(a.h16.bits + v), a.h16.fmt, cs) : __ldg(a.C + v);
            if (isfinite(c)) {
              if (do_repl && mask_bit(a.mbits, v)) {
                q = (c >= 0.0f) ? qrepl : -qrepl;
              } else {
                q = quantize(c, fscale);
              }
            }
          }
          Xt[e] = q;
        }
        __syncthreads();
        if (h > 0) {
          for (int e = tid; e < L.rows * tx; e += blockDim.x) {
            const int row = e / tx, c = e - row * tx;
            Bt[e] = fir(Xt + row * L.px + c, 1, taps, ntap);
          }
          __syncthreads();
        }
#pragma unroll
        for (int i = 0; i < kMaxOuts; ++i) {
          const int o = tid + i * kSmoothThreads;
          P[i] = 0ll;
          if (o < area) {
            const int oy = o / tx, ox = o - oy * tx;
            P[i] = (h > 0) ? fir(Bt + oy * tx + ox, tx, taps, ntap) : Xt[oy * L.px + ox];
          }
        }
      } else {
#pragma unroll
        for (int i = 0; i < kMaxOuts; ++i) P[i] = 0ll;
      }
      const int slot = j % wz;
      const int zo = zp - r;
#pragma unroll
      for (int i = 0; i < kMaxOuts; ++i) {
        const int o = tid + i * kSmoothThreads;
        if (o >= area) continue;
        long long* rp = ring + (size_t)slot * area + o;
        zsum[i] += P[i] - *rp;
        *rp = P[i];
        if (j >= 2 * r && zo >= z0 && zo < z1) {
          const int oy = o / tx, ox = o - oy * tx;
          const long long gx = x0 + ox, gy = y0 + oy;
          if (gx < nx && gy < ny) {
            const long long v = ((long long)zo * ny + gy) * nx + gx;
            const float c = a.h16.fmt ? half16_value(__ldg(a.h16.bits + v), a.h16.fmt, __ldg(a.h16.scale + zo))
                                      : __ldg(a.C + v);
            float s;
            if (isfinite(c)) {
              s = dequantize(zsum[i], inv);
              if (a.hist) atomicAdd(&hist[bin_of(s, cfg)], 1u);
            } else {
              s = __int_as_float(0x7fc00000);
            }
            a.S[v] = s;
          }
        }
      }
      __syncthreads();
    }
  }
  if (a.hist) {
    __syncthreads();
    for (int i = tid; i < kNumBins; i += blockDim.x)
      if (hist[i]) atomicAdd(a.hist + i, (unsigned long long)hist[i]);
  }
}

// (0, 0) pair with a possibly non-empty mask: S = X, blanked at non-finite voxels.
__global__ void __launch_bounds__(512) k_identity(SmoothArgs a, long long n) {
  extern __shared__ unsigned int hsh[];
  if (a.hist)
    for (int i = threadIdx.x; i < kNumBins; i += blockDim.x) hsh[i] = 0u;
  __syncthreads();
  const BinCfg cfg = a.win ? a.st->win : kFullRange;
  const float repl = a.use_fixed_repl ? a.repl_value : a.st->repl;
  const bool do_repl = repl > 0.0f && a.mbits != nullptr;
  // a 16-bit cube: the plane of v (for its scale), advanced with v
  const long long plane = (long long)a.nx * a.ny, stride = (long long)gridDim.x * blockDim.x;
  const long long dz = stride / plane, doff = stride - dz * plane;
  long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long z = v / plane, off = v - z * plane;
  for (; v < n; v += stride) {
    const float c = a.h16.fmt ? half16_value(__ldg(a.h16.bits + v), a.h16.fmt, __ldg(a.h16.scale + z)) : __ldg(a.C + v);
    z += dz;
    off += doff;
    if (off >= plane) {
      off -= plane;
      ++z;
    }
    float s;
    if (isfinite(c)) {
      s = (do_repl && mask_bit(a.mbits, v)) ? ((c >= 0.0f) ? repl : -repl) : c;
      if (a.hist) atomicAdd(&hsh[bin_of(s, cfg)], 1u);
    } else {
      s = __int_as_float(0x7fc00000);
    }
    a.S[v] = s;
  }
  if (a.hist) {
    __syncthreads();
    for (int i = threadIdx.x; i < kNumBins; i += blockDim.x)
      if (hsh[i]) atomicAdd(a.hist + i, (unsigned long long)hsh[i]);
  }
}

cudaError_t launch_identity(const SmoothArgs& a, int sms, cudaStream_t s) {
  const size_t smem = a.hist ? kNumBins * sizeof(unsigned int) : 0;
  const long long n = (long long)a.nx * a.ny * a.nz;
  long long want = (n + 511) / 512;
  int grid = (int)(want < 1 ? 1 : (want > 4LL * sms ? 4LL * sms : want));
  k_identity<<<grid, 512, smem, s>>>(a, n);
  return cudaGetLastError();
}

void choose_tiles(SmoothArgs* a) {
  const int h = a->pd.h, wz = a->pd.wz;
  static const int cand[][2] = {{32, 32}, {32, 16}, {16, 16}, {32, 8}, {16, 8}, {8, 8}, {8, 4}, {4, 4}};
  const size_t limit = 227 * 1024;
  a->tx = 4;
  a->ty = 4;
  for (auto& c : cand) {
    if (smooth_layout(c[0], c[1], h, wz, a->hist != nullptr).total <= limit) {
      a->tx = c[0];
      a->ty = c[1];
      break;
    }
  }
  // no point in tiles much wider than the cube
  while (a->tx > 8 && a->tx / 2 >= a->nx) a->tx /= 2;
  while (a->ty > 8 && a->ty / 2 >= a->ny) a->ty /= 2;
  a->tiles_x = (a->nx + a->tx - 1) / a->tx;
  a->tiles_y = (a->ny + a->ty - 1) / a->ty;
}

cudaError_t launch_smooth_tile(const SmoothArgs& a, int sms, cudaStream_t s, bool* done);
cudaError_t launch_smooth_ws(const SmoothArgs& a, int sms, cudaStream_t s, bool* done);
cudaError_t launch_smooth_fir(const SmoothArgs& a, int sms, cudaStream_t s, bool* done);
cudaError_t launch_smooth_z(const SmoothArgs& a, int sms, cudaStream_t s, bool* done);
void init_tile_attrs();
void init_ws_attrs();
void init_fir_attrs();
void init_ws16_attrs();
void init_z_attrs();

__global__ void k_fill_noise(float* __restrict__ x, long long n, unsigned int seed) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    // splitmix64 of (seed, i)
    unsigned long long z = ((unsigned long long)seed << 40) ^ (unsigned long long)i;
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    z ^= z >> 31;
    x[i] = (float)(z >> 40) * 0x1p-23f - 1.0f;
  }
}

// C = float(x) * scale[z] for a cube stored as BF16 (bf16 != 0) or FP16 bit
// patterns with one float32 scale per channel (plane of `plane` voxels); the
// product is rounded once to float32.
__global__ void k_decode_half(const uint16_t* __restrict__ x, const float* __restrict__ scale, long long plane,
                              long long n, int bf16, float* __restrict__ out) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const unsigned short h = __ldg(x + i);
    const float v = bf16 ? __uint_as_float((unsigned)h << 16) : __half2float(__ushort_as_half(h));
    out[i] = __fmul_rn(v, __ldg(scale + i / plane));
  }
}

cudaError_t launch_decode_half(const uint16_t* x, const float* scale, long long plane, long long n, int bf16,
                               float* out, int sms, cudaStream_t s) {
  k_decode_half<<<8 * sms, 256, 0, s>>>(x, scale, plane, n, bf16, out);
  return cudaGetLastError();
}

cudaError_t launch_fill_noise(float* x, long long n, unsigned int seed, int sms, cudaStream_t s) {
  k_fill_noise<<<8 * sms, 256, 0, s>>>(x, n, seed);
  return cudaGetLastError();
}

cudaError_t launch_smooth(const SmoothArgs& a0, int sms, cudaStream_t s, int* launches, int* kernel) {
  bool done = false;
  cudaError_t et = cudaSuccess;
  auto ran = [&](int code) {
    if (launches) ++*launches;
    if (kernel) *kernel = code;
    return cudaSuccess;
  };
  // a kernel fixed by the autotuner, if it serves this pair (else the default order)
  if (a0.tune_kind == TUNE_TILE) {
    et = launch_smooth_tile(a0, sms, s, &done);
  } else if (a0.tune_kind == TUNE_GENERIC) {
    SmoothArgs g = a0;
    g.generic = 1;
    g.tune_kind = TUNE_AUTO;
    return launch_smooth(g, sms, s, launches, kernel);
  }
  if (et != cudaSuccess) return et;
  if (done) return ran(SC_KERNEL_TILE);
  et = launch_smooth_z(a0, sms, s, &done);
  if (et != cudaSuccess) return et;
  if (done) return ran(SC_KERNEL_Z);
  et = launch_smooth_ws(a0, sms, s, &done);
  if (et != cudaSuccess) return et;
  if (done) return ran(ws_tile_rows(a0) == 16 ? SC_KERNEL_WS16 : SC_KERNEL_WS32);
  et = launch_smooth_fir(a0, sms, s, &done);
  if (et != cudaSuccess) return et;
  if (done) return ran(SC_KERNEL_FIR);
  et = launch_smooth_tile(a0, sms, s, &done);
  if (et != cudaSuccess) return et;
  if (done) return ran(SC_KERNEL_TILE);
  SmoothArgs a = a0;
  if (a.tx == 0) choose_tiles(&a);
  const size_t smem = smooth_smem_bytes(a);
  int occ = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_smooth_generic, kSmoothThreads, smem);
  if (occ < 1) occ = 1;
  const long long tiles = (long long)a.tiles_x * a.tiles_y;
  if (a.lz <= 0) {
    const long long target = 4LL * sms * occ;
    long long zch = (target + tiles - 1) / tiles;
    const long long max_ch = std::max(1LL, (long long)a.nz / 16);
    zch = std::max(1LL, std::min(zch, max_ch));
    a.lz = (int)((a.nz + zch - 1) / zch);
  }
  a.zchunks = (a.nz + a.lz - 1) / a.lz;
  const long long items = tiles * a.zchunks;
  const int grid = (int)std::min<long long>(items, (long long)sms * occ);
  k_smooth_generic<<<grid, kSmoothThreads, smem, s>>>(a);
  et = cudaGetLastError();
  if (et != cudaSuccess) return et;
  return ran(SC_KERNEL_GENERIC);
}

void init_noise_attrs();
void init_noise_scale_attrs();

// Raise the dynamic shared-memory limits once per device (called by sc_create).
void init_kernel_attrs() {
  cudaFuncSetAttribute(k_smooth_generic, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  init_tile_attrs();
  init_ws_attrs();
  init_fir_attrs();
  init_ws16_attrs();
  init_z_attrs();
  init_share_attrs();
  init_noise_attrs();
  init_noise_scale_attrs();
}

// ---------------------------------------------------------------------------
// Host: kernel-pair description.
int cascade_widths(double fwhm, int w[3]) {
  // Kovesi (2010): n = 3 boxes; sigma = FWHM / sqrt(8 ln 2);
  // w_ideal = sqrt(12 sigma^2 / n + 1); w_l = largest odd <= w_ideal;
  // m = round((12 sigma^2 - n w_l^2 - 4 n w_l - 3 n) / (-4 w_l - 4)) boxes of
  // w_l, the other n - m of w_l + 2.
  if (!(fwhm > 0.0)) {
    w[0] = w[1] = w[2] = 1;
    return 0;
  }
  const int n = 3;
  const double sigma = fwhm / sqrt(8.0 * log(2.0));
  const double var12 = 12.0 * sigma * sigma;
  const double w_ideal = sqrt(var12 / n + 1.0);
  if (!(w_ideal < 4096.0)) return -1;
  int wl = (int)floor(w_ideal);
  if (wl % 2 == 0) wl -= 1;
  const double m_real = (var12 - n * (double)wl * wl - 4.0 * n * wl - 3.0 * n) / (-4.0 * wl - 4.0);
  int m = (int)floor(m_real + 0.5);
  m = std::min(std::max(m, 0), n);
  for (int i = 0; i < 3; ++i) w[i] = (i < m) ? wl : wl + 2;
  return 0;
}

int gauss_taps(double fwhm, int* taps, int max_taps) {
  // sigma = FWHM / sqrt(8 ln 2); taps at offsets |i| <= floor(4 sigma), each
  // exp(-i^2 / (2 sigma^2)) in units of 1/1024 of the central sample, rounded
  // to the nearest integer (ties to even).
  if (!(fwhm > 0.0)) {
    if (max_taps < 1) return -1;
    taps[0] = kGaussTapUnit;
    return 1;
  }
  const double sigma = fwhm / sqrt(8.0 * log(2.0));
  const double hr = floor(4.0 * sigma);
  if (!(hr < 4096.0) || 2 * (int)hr + 1 > max_taps) return -1;
  const int h = (int)hr;
  for (int i = -h; i <= h; ++i)
    taps[i + h] = (int)llrint(kGaussTapUnit * exp(-(double)i * i / (2.0 * sigma * sigma)));
  return 2 * h + 1;
}

int make_pair(const sc_kernel& k, PairDesc* pd, bool sampled) {
  if (!(k.fwhm_spatial_px >= 0.0f) || !isfinite(k.fwhm_spatial_px)) return SC_ERR_ARG;
  if (k.boxcar_chan < 0 || (k.boxcar_chan > 1 && k.boxcar_chan % 2 == 0)) return SC_ERR_ARG;
  if (k.boxcar_chan > kMaxBoxcar) return SC_ERR_UNSUPPORTED;
  pd->wz = k.boxcar_chan > 1 ? k.boxcar_chan : 1;
  pd->sampled = 0;
  long long t[2 * kMaxHalf + 1] = {0};
  int len = 1;
  if (sampled) {
    // the sampled Gaussian: its taps, less the zero taps at both ends (which
    // add nothing), so that the support is as short as the kernel allows
    if (cascade_widths(k.fwhm_spatial_px, pd->w) != 0) return SC_ERR_ARG;  // the same FWHM range
    int g[2 * 4096 + 1];
    const int n = gauss_taps(k.fwhm_spatial_px, g, 2 * 4096 + 1);
    if (n < 1) return SC_ERR_ARG;
    int lo = 0;
    while (2 * lo + 1 < n && g[lo] == 0) ++lo;
    len = n - 2 * lo;
    if ((len - 1) / 2 > kMaxHalf) return SC_ERR_UNSUPPORTED;
    for (int i = 0; i < len; ++i) t[i] = g[lo + i];
    if (len > 1) {
      pd->sampled = 1;
      pd->w[0] = pd->w[1] = pd->w[2] = 0;  // no cascade kernel serves this pair
    } else {
      pd->w[0] = pd->w[1] = pd->w[2] = 1;  // a single tap: no spatial smoothing
      t[0] = 1;
    }
  } else {
    if (cascade_widths(k.fwhm_spatial_px, pd->w) != 0) return SC_ERR_ARG;
    // composed integer kernel: convolution of three all-ones boxes
    t[0] = 1;
    for (int b = 0; b < 3; ++b) {
      const int w = pd->w[b];
      if ((len - 1) / 2 + (w - 1) / 2 > kMaxHalf) return SC_ERR_UNSUPPORTED;
      long long nt[2 * kMaxHalf + 1] = {0};
      for (int i = 0; i < len; ++i)
        for (int d = 0; d < w; ++d) nt[i + d] += t[i];
      len += w - 1;
      for (int i = 0; i < len; ++i) t[i] = nt[i];
    }
  }
  pd->h = (len - 1) / 2;
  long long tsum = 0;
  for (int i = 0; i < 2 * kMaxHalf + 1; ++i) {
    pd->taps[i] = (i < len) ? (int)t[i] : 0;
    tsum += (i < len) ? t[i] : 0;
  }
  pd->W = tsum * tsum * pd->wz;
  pd->Wf = tsum * tsum * (pd->wz > kShareMaxWz ? pd->wz : kShareMaxWz);
  return SC_OK;
}

}  // namespace sc
