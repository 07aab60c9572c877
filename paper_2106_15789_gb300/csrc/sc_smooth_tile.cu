// Specialised smoothing kernel: compile-time boxcar widths, streamed register
// box cascades, TMA tile loads, the spectral ring in Tensor Memory.
//
// Same arithmetic as the generic kernel (exact int64 fixed point, one final
// rounding; see sc_smooth.cu), so both produce identical floats.
//
// A block (256 threads, one per SM) owns a 64 x 32 column tile and a chunk of
// planes. Per plane:
//   load    the plane's raw float tile with its halo ((32 + 2R) x (64 + 2RA)
//           values, RA = R rounded up to 4 so the TMA x coordinate is 16-byte
//           aligned) arrives by TMA into one of two shared buffers, one plane
//           ahead, on an mbarrier (zero fill outside the cube is the padding);
//           rows that are not a multiple of 16 bytes use cp.async instead.
//           The mask words of the next plane are prefetched into registers.
//   convert every halo'd value once: NaN -> 0, masked -> +-repl, else
//           rint(x * 2^f), into an int64 tile.
//   x pass  (32 + 2R) rows x 4 segments of 16 outputs; the three boxcars run
//           as one interleaved stream of running sums (three independent
//           dependency chains per step).
//   y pass  64 columns x 4 segments of 8 outputs, the same way down a column.
//   z       each thread's 8 values enter a ring of wz planes kept in TMEM
//           (16 columns of the thread's lane per plane) and a running int64
//           sum gives the spectral boxcar.
//   out     plane r = (wz - 1)/2 behind is final: NaN where the input voxel is
//           NaN (a per-thread bit history), else the scaled float; store and
//           histogram.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdint>
#include <cstring>

#include "sc_device.cuh"
#include "sc_internal.h"
#include "sc_tile_common.cuh"

namespace sc {

namespace tile {

constexpr int kThreads = 512;
constexpr int TX = 64, TY = 32;
constexpr int SEGX = 8, SEGY = 4;
constexpr int kMaxWz = 15;                 // TMEM ring: 16 slots of 4 int64 per thread
constexpr int kStages = 3;                  // raw-tile buffers (loads run two planes ahead)
using namespace tc;

template <int W1, int W2, int W3>
struct Geo {
  static constexpr int R = (W1 - 1) / 2 + (W2 - 1) / 2 + (W3 - 1) / 2;
  static constexpr int RA = (R + 3) & ~3;  // halo of the raw tile in x, 16-byte aligned
  static constexpr int BX = TX + 2 * RA;   // raw tile width
  static constexpr int BY = TY + 2 * R;    // raw tile height = quantised tile height
  static constexpr int PX = TX + 2 * R;    // quantised tile width
  static constexpr int XP = PX | 1;        // odd pitch (8-byte words)
  static constexpr int BP = TX + 1;        // odd pitch of the x-pass output
  static constexpr int ROWS_PER_WARP = (BY + 7) / 8;
  static constexpr int COL_SLOTS = (PX + 31) / 32;
};

struct Smem {
  size_t raw[3], mw, x, b, hist, mbar, total;
};

template <int W1, int W2, int W3>
__host__ __device__ constexpr Smem smem_layout(bool hist) {
  using G = Geo<W1, W2, W3>;
  Smem s{};
  size_t o = 0;
  for (int b = 0; b < kStages; ++b) {
    s.raw[b] = o;
    o = al128(o + sizeof(float) * (size_t)G::BY * G::BX);
  }
  s.mw = o;
  o = al128(o + sizeof(unsigned) * (size_t)G::BY * 5);
  s.x = o;
  o = al128(o + sizeof(long long) * (size_t)G::BY * G::XP);
  s.b = o;
  o = al128(o + sizeof(long long) * (size_t)G::BY * G::BP);
  s.hist = o;
  o = al128(o + (hist ? sizeof(unsigned) * kNumBins : 0));
  s.mbar = o;
  o = al128(o + kStages * sizeof(unsigned long long));
  s.total = o + 128;  // room to align the dynamic base to 128 bytes at run time
  return s;
}

// TMEM ring: 16 warps; warp w uses lanes 32*(w%4) and columns 128*(w/4) ..
// +127, so each thread owns 128 32-bit words of one lane: 16 ring slots of
// 4 int64.
constexpr int kSlotCols = 2 * SEGY;  // TMEM columns per ring slot

}  // namespace tile

template <int W1, int W2, int W3, bool TMA, bool REPL>
__global__ void __launch_bounds__(tile::kThreads, 1)
    k_smooth_tile(const __grid_constant__ CUtensorMap tmap, SmoothArgs a) {
  using namespace tile;
  using G = Geo<W1, W2, W3>;
  constexpr int R = G::R, RA = G::RA;
  constexpr int NCONV = (G::BY * G::PX + kThreads - 1) / kThreads;  // conversions per thread
  extern __shared__ __align__(128) unsigned char smem_dyn[];
  // 128-byte aligned base (TMA destinations, mbarriers)
  unsigned char* smem = smem_dyn + ((128u - (smem_u32(smem_dyn) & 127u)) & 127u);
  const Smem L = smem_layout<W1, W2, W3>(a.hist != nullptr);
  float* const raw0 = reinterpret_cast<float*>(smem + L.raw[0]);
  constexpr size_t kRawStride = al128(sizeof(float) * (size_t)G::BY * G::BX) / sizeof(float);
  unsigned* mw = reinterpret_cast<unsigned*>(smem + L.mw);  // [BY][4] mask words, then [BY] bit offsets
  long long* Xt = reinterpret_cast<long long*>(smem + L.x);
  long long* Bt = reinterpret_cast<long long*>(smem + L.b);
  unsigned* hist = reinterpret_cast<unsigned*>(smem + L.hist);
  const unsigned mbar0 = smem_u32(smem + L.mbar);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int wz = a.pd.wz, r = (wz - 1) / 2;
  if (a.hist)
    for (int i = tid; i < kNumBins; i += kThreads) hist[i] = 0u;
  const BinCfg cfg = a.win ? a.st->win : kFullRange;
  const float fscale = a.st->fx_scale[a.pair];
  const float inv = a.st->fx_inv[a.pair];
  const long long qrepl = a.st->fx_qrepl[a.pair];
  const bool do_repl = REPL && qrepl > 0;
  const long long nx = a.nx, ny = a.ny, nz = a.nz;
  const long long plane = nx * ny;
  const long long n_tiles = (long long)a.tiles_x * a.tiles_y;
  const long long n_items = n_tiles * a.zchunks;
  const int yc = tid & (TX - 1), ys = tid / TX;  // y pass / output ownership

  __shared__ unsigned tmem_holder;
  if (warp == 0) tmem_alloc(&tmem_holder);
  if (TMA && tid == 0) {
    for (int b = 0; b < kStages; ++b) mbar_init(mbar0 + 8 * b, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  tmem_fence_before();
  __syncthreads();
  tmem_fence_after();
  const unsigned tbase = tmem_holder;
  const unsigned tmine = tbase + ((unsigned)(32 * (warp & 3)) << 16) + (unsigned)(128 * (warp >> 2));
  bool timed_out = false;

  auto item_geo = [&](long long it, int* x0, int* y0, int* z0, int* ns) {
    const long long t = it % n_tiles;
    const int zc = (int)(it / n_tiles);
    *x0 = (int)(t % a.tiles_x) * TX;
    *y0 = (int)(t / a.tiles_x) * TY;
    *z0 = zc * a.lz;
    *ns = (int)(min((long long)*z0 + a.lz, nz) - *z0) + 2 * r;
  };
  // raw tile of plane zp of tile (x0, y0) into stage b
  auto issue = [&](int b, int x0, int y0, int zp) {
    float* dst = raw0 + b * kRawStride;
    if (TMA) {
      if (tid == 0) {
        mbar_expect_tx(mbar0 + 8 * b, (unsigned)(sizeof(float) * G::BX * G::BY));
        tma_load_3d(smem_u32(dst), &tmap, x0 - RA, y0 - R, zp, mbar0 + 8 * b);
      }
    } else {
      const bool zok = zp >= 0 && zp < nz;
      for (int e = tid; e < G::BX * G::BY; e += kThreads) {
        const int row = e / G::BX, col = e - row * G::BX;
        const long long gx = (long long)x0 - RA + col, gy = (long long)y0 - R + row;
        const bool ok = zok && gx >= 0 && gx < nx && gy >= 0 && gy < ny;
        cp_async4(smem_u32(dst + e), ok ? a.C + (long long)zp * plane + gy * nx + gx : a.C, ok);
      }
      cp_async_commit();
    }
  };
  // lookahead cursor of the raw-tile loads (kStages - 1 planes ahead)
  long long la_item = blockIdx.x;
  int la_j = 0, la_x0 = 0, la_y0 = 0, la_z0 = 0, la_n = 0;
  if (la_item < n_items) item_geo(la_item, &la_x0, &la_y0, &la_z0, &la_n);
  long long issued = 0;
  auto issue_next = [&]() {
    if (la_item >= n_items) return;
    issue((int)(issued % kStages), la_x0, la_y0, la_z0 - r + la_j);
    ++issued;
    if (++la_j == la_n) {
      la_item += gridDim.x;
      la_j = 0;
      if (la_item < n_items) item_geo(la_item, &la_x0, &la_y0, &la_z0, &la_n);
    }
  };
  // Mask bits of plane zp re-aligned to the quantised tile: word k of row
  // `row` holds the bits of columns 32k .. 32k+31 (column c <-> gx = x0 - R + c),
  // with bits of columns outside the cube cleared. One word per thread
  // (tid < 4 * BY); the two source words straddling it are funnel-shifted.
  auto fetch_mask = [&](int x0, int y0, int zp) -> unsigned {
    unsigned w = 0u;
    if (do_repl && tid < 4 * G::BY) {
      const int row = tid >> 2, k = tid & 3;
      const long long gy = (long long)y0 - R + row;
      if (zp >= 0 && zp < nz && gy >= 0 && gy < ny) {
        const long long vb = (long long)zp * plane + gy * nx + ((long long)x0 - R) + 32 * k;  // flat index of bit 0
        const long long wi = vb >> 5;                                                           // floor division
        const unsigned off = (unsigned)(vb & 31);
        const long long nwords = (plane * nz + 31) >> 5;
        const unsigned w0 = (wi >= 0 && wi < nwords) ? __ldg(a.mbits + wi) : 0u;
        const unsigned w1 = (wi + 1 >= 0 && wi + 1 < nwords) ? __ldg(a.mbits + wi + 1) : 0u;
        w = __funnelshift_r(w0, w1, off);
        // keep columns with gx = x0 - R + 32k + bit in [0, nx)
        const int g0 = x0 - R + 32 * k;  // gx of bit 0
        const int lo = g0 < 0 ? -g0 : 0;
        const int hi = (long long)nx - g0 > 32 ? 32 : (int)((long long)nx - g0);
        unsigned keep = 0u;
        if (hi > lo) keep = (hi - lo >= 32) ? 0xffffffffu : (((1u << (hi - lo)) - 1u) << lo);
        w &= keep;
      }
    }
    return w;
  };

  for (int k = 0; k < kStages - 1; ++k) issue_next();
  long long g = 0;  // plane steps consumed so far: stage g % kStages, parity (g / kStages) & 1
  for (long long item = blockIdx.x; item < n_items; item += gridDim.x) {
    int x0, y0, z0, n_steps;
    item_geo(item, &x0, &y0, &z0, &n_steps);
    long long zsum[SEGY];
#pragma unroll
    for (int i = 0; i < SEGY; ++i) zsum[i] = 0;
    if (wz > 1) {
      unsigned zero[kSlotCols];
#pragma unroll
      for (int i = 0; i < kSlotCols; ++i) zero[i] = 0u;
      for (int s = 0; s < wz; ++s) tmem_st8(tmine + (unsigned)(kSlotCols * s), zero);
      tmem_wait_st();
    }
    unsigned long long nan_hist = 0ull;
    unsigned mword = fetch_mask(x0, y0, z0 - r);

    for (int j = 0; j < n_steps; ++j, ++g) {
      const int zp = z0 - r + j;
      const int b = (int)(g % kStages);
      if (do_repl && tid < 4 * G::BY) mw[tid] = mword;
      if (TMA) {
        if (!mbar_wait(mbar0 + 8 * b, (unsigned)((g / kStages) & 1))) timed_out = true;
      } else {
        // groups complete in order: allow the newer one to stay in flight
        if (issued > g + 1) cp_async_wait_one_pending();
        else cp_async_wait_all();
      }
      __syncthreads();
      issue_next();
      if (j + 1 < n_steps) mword = fetch_mask(x0, y0, zp + 1);
      // ring slot of this plane: load early, use after the passes
      unsigned old[kSlotCols];
      const unsigned ta = tmine + (unsigned)(kSlotCols * (j % (wz > 1 ? wz : 1)));
      if (wz > 1) tmem_ld8(ta, old);
      const float* rb = raw0 + b * kRawStride;
      // convert the halo'd tile once (flattened, branch-free per element)
#pragma unroll
      for (int k = 0; k < NCONV; ++k) {
        const int e = tid + k * kThreads;
        if (k + 1 < NCONV || e < G::BY * G::PX) {
          const int row = e / G::PX, col = e - row * G::PX;
          const float v = rb[row * G::BX + col + (RA - R)];
          const bool fin = (__float_as_uint(v) & 0x7f800000u) != 0x7f800000u;
          long long q = quantize(v, fscale);
          if (do_repl) {
            const unsigned word = mw[row * 4 + (col >> 5)];
            const long long qr = v >= 0.0f ? qrepl : -qrepl;
            q = ((word >> (col & 31)) & 1u) ? qr : q;
          }
          Xt[row * G::XP + col] = fin ? q : 0ll;
        }
      }
      __syncthreads();
      // x pass
      for (int it = tid; it < G::BY * (TX / SEGX); it += kThreads) {
        const int row = it % G::BY, seg = it / G::BY;
        const long long* src = Xt + row * G::XP + seg * SEGX;
        long long* dst = Bt + row * G::BP + seg * SEGX;
        cascade_stream<W1, W2, W3, SEGX>([&](int i) { return src[i]; }, [&](int k, long long v) { dst[k] = v; });
      }
      __syncthreads();
      // y pass
      long long P[SEGY];
      {
        const long long* src = Bt + (ys * SEGY) * G::BP + yc;
        cascade_stream<W1, W2, W3, SEGY>([&](int i) { return src[i * G::BP]; }, [&](int k, long long v) { P[k] = v; });
      }
      unsigned nanbits = 0u;
#pragma unroll
      for (int i = 0; i < SEGY; ++i) {
        const float c = rb[(ys * SEGY + i + R) * G::BX + yc + RA];
        nanbits |= ((__float_as_uint(c) & 0x7f800000u) == 0x7f800000u ? 1u : 0u) << i;
      }
      nan_hist = (nan_hist << SEGY) | nanbits;
      // spectral boxcar
      if (wz > 1) {
        unsigned nw[kSlotCols];
        tmem_wait_ld();
#pragma unroll
        for (int i = 0; i < SEGY; ++i) {
          const long long o = (long long)(((unsigned long long)old[2 * i + 1] << 32) | old[2 * i]);
          zsum[i] += P[i] - o;
          nw[2 * i] = (unsigned)((unsigned long long)P[i] & 0xffffffffull);
          nw[2 * i + 1] = (unsigned)((unsigned long long)P[i] >> 32);
        }
        tmem_st8(ta, nw);
      } else {
#pragma unroll
        for (int i = 0; i < SEGY; ++i) zsum[i] = P[i];
      }
      if (j >= 2 * r) {
        const int zo = zp - r;
        const unsigned nb = (unsigned)(nan_hist >> (SEGY * r)) & ((1u << SEGY) - 1u);
        const long long gx = (long long)x0 + yc;
        float* out = a.S + (long long)zo * plane + ((long long)y0 + ys * SEGY) * nx + gx;
#pragma unroll
        for (int i = 0; i < SEGY; ++i) {
          const bool inb = gx < nx && (long long)y0 + ys * SEGY + i < ny;
          const bool isnan_out = (nb >> i) & 1u;
          const float sv = dequantize(zsum[i], inv);
          const float s = isnan_out ? __int_as_float(0x7fc00000) : sv;
          if (inb) {
            out[i * nx] = s;
            if (a.hist && !isnan_out) atomicAdd(&hist[bin_of(s, cfg)], 1u);
          }
        }
      }
      if (wz > 1) tmem_wait_st();
      __syncthreads();
    }
  }
  if (!TMA) cp_async_wait_all();
  tmem_fence_before();
  __syncthreads();
  tmem_fence_after();
  if (warp == 0) tmem_dealloc(tbase);
  if (timed_out && (tid & 31) == 0) atomicOr(&a.st->status, (unsigned)SC_ST_TIMEOUT);
  if (a.hist)
    for (int i = tid; i < kNumBins; i += kThreads)
      if (hist[i]) atomicAdd(a.hist + i, (unsigned long long)hist[i]);
}

// ---------------------------------------------------------------------------
namespace {

template <int W1, int W2, int W3>
cudaError_t launch_tile(const SmoothArgs& a0, int sms, cudaStream_t s, bool* done) {
  using namespace tile;
  using G = Geo<W1, W2, W3>;
  SmoothArgs a = a0;
  const Smem L = smem_layout<W1, W2, W3>(a.hist != nullptr);
  if (L.total + 1024 > 227 * 1024) return cudaSuccess;  // not served: caller falls back
  a.tx = TX;
  a.ty = TY;
  a.tiles_x = (a.nx + TX - 1) / TX;
  a.tiles_y = (a.ny + TY - 1) / TY;
  const long long tiles = (long long)a.tiles_x * a.tiles_y;
  const long long zch = z_chunks(a, tiles, sms, (a.nz + 31) / 32);
  a.lz = (int)((a.nz + zch - 1) / zch);
  a.zchunks = (a.nz + a.lz - 1) / a.lz;
  const long long items = tiles * a.zchunks;
  const int grid = (int)(items < sms ? items : sms);
  // TMA needs 16-byte aligned rows and base address
  CUtensorMap map;
  const bool tma = tc::encode_cube_map(&map, a.C, a.nx, a.ny, a.nz, G::BX, G::BY);
  const bool repl = a.mbits != nullptr && a.repl_possible;
  // one block per SM (it holds all of the SM's TMEM)
  const size_t smem_req = tc::one_block_per_sm_smem(L.total);
  if (tma) {
    if (repl) k_smooth_tile<W1, W2, W3, true, true><<<grid, kThreads, smem_req, s>>>(map, a);
    else k_smooth_tile<W1, W2, W3, true, false><<<grid, kThreads, smem_req, s>>>(map, a);
  } else {
    if (repl) k_smooth_tile<W1, W2, W3, false, true><<<grid, kThreads, smem_req, s>>>(map, a);
    else k_smooth_tile<W1, W2, W3, false, false><<<grid, kThreads, smem_req, s>>>(map, a);
  }
  *done = true;
  return cudaGetLastError();
}

template <int W1, int W2, int W3>
void set_attr() {
  tc::set_dyn_smem_limit(k_smooth_tile<W1, W2, W3, false, false>);
  tc::set_dyn_smem_limit(k_smooth_tile<W1, W2, W3, true, false>);
  tc::set_dyn_smem_limit(k_smooth_tile<W1, W2, W3, false, true>);
  tc::set_dyn_smem_limit(k_smooth_tile<W1, W2, W3, true, true>);
}

}  // namespace

void init_tile_attrs() {
  set_attr<1, 1, 1>();
  set_attr<1, 3, 3>();
  set_attr<3, 5, 5>();
  set_attr<5, 5, 5>();
  set_attr<7, 9, 9>();
}

// Specialised kernel for the common cascades (FWHM 0, 3, 5, 6, 10 px) with
// spectral widths up to 15; *done = false when the pair is not served.
cudaError_t launch_smooth_tile(const SmoothArgs& a, int sms, cudaStream_t s, bool* done) {
  *done = false;
  if (a.generic || a.h16.fmt || a.pd.wz > tile::kMaxWz) return cudaSuccess;  // float32 cubes only
  const int* w = a.pd.w;
  if (w[0] == 1 && w[1] == 1 && w[2] == 1) return launch_tile<1, 1, 1>(a, sms, s, done);
  if (w[0] == 1 && w[1] == 3 && w[2] == 3) return launch_tile<1, 3, 3>(a, sms, s, done);
  if (w[0] == 3 && w[1] == 5 && w[2] == 5) return launch_tile<3, 5, 5>(a, sms, s, done);
  if (w[0] == 5 && w[1] == 5 && w[2] == 5) return launch_tile<5, 5, 5>(a, sms, s, done);
  if (w[0] == 7 && w[1] == 9 && w[2] == 9) return launch_tile<7, 9, 9>(a, sms, s, done);
  return cudaSuccess;
}

}  // namespace sc
