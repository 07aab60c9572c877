// Warp-specialised smoothing kernel for the spatial cascades of FWHM 3, 5, 6
// and 10 px (SoFiA 2 Sect. 4.2 / 5) with spectral boxcars up to 15 channels
// (31 with 64 x 16 tiles), and the replacement of Sect. 6.2. Instances with
// W1 = 0 run the sampled Gaussian's integer FIR of half-width W2 instead of a
// cascade (sc_smooth_fir.cu); instances with EB = 2 read a 16-bit cube with
// per-channel scales (sc_smooth_ws16.cu).
//
// Same exact int64 fixed-point arithmetic as every other smoothing kernel of
// this library (quantise once, exact box sums, one final rounding), hence the
// same floats. A block (one per SM) owns a 64 x 32 column tile and a chunk of
// planes, and its warps split into two groups that hand planes over through
// double buffers guarded by mbarriers, so neither group waits for the other
// at a block-wide barrier:
//
//   producers (8 warps)  wait for the plane's raw halo'd tile (loaded two
//                        planes ahead into four buffers: by TMA, issued by
//                        one producer, or, for cubes whose rows are not
//                        16-byte multiples, by the consumers with 4-byte
//                        cp.async copies), quantise it into an int64 tile
//                        (NaN -> 0, masked -> +-replacement; mask words are
//                        loaded two planes ahead), then run the x cascade of
//                        every row into buffer g % 2. With two quantised tiles
//                        (R <= 8) one producer barrier per plane suffices.
//   consumers (8 warps)  take buffer g % 2, run the y cascade down a column
//                        (8 outputs per thread), read which of those voxels
//                        are NaN from the raw tile, release both, and push
//                        the 8 values into their spectral ring in TMEM (wz
//                        slots of 16 columns of the thread's lane); the plane
//                        (wz - 1)/2 behind is final: store and histogram.
//
// Hand-off barriers: bt_full[b] (one arrival per producer warp once its x
// pass items are written) and bt_empty[b] (one arrival per consumer warp; it
// also frees the raw tile of that plane, which the TMA refills two planes
// later). Every wait is bounded in wall time; a wait that runs out sets
// SC_ST_TIMEOUT and the kernel finishes without further waiting.
#pragma once

#include <cstdint>

#include "sc_device.cuh"
#include "sc_internal.h"
#include "sc_tile_common.cuh"

namespace sc {

namespace ws {

using namespace tc;

constexpr int kPW = 8;               // producer warps
constexpr int kPT = 32 * kPW;        // producer threads
constexpr int TX = 64;               // tile width
constexpr int SEGY = 8;              // consecutive rows per consumer thread
constexpr int kStages = 4;           // raw-tile buffers: being read by consumers, converted, two in flight
constexpr int kLookahead = 2;        // planes loaded ahead of the one being converted
constexpr int kSlotCols = 2 * SEGY;  // TMEM columns per ring slot (8 int64)
constexpr unsigned kBarProducers = 1;

// Tile height TY: one consumer thread per 8-row column segment, so TY/4
// consumer warps; a consumer warp's TMEM lane quarter is shared by TY/16
// warps, which bounds the ring to kMaxWz planes (15 for TY = 32, 31 for 16).
template <int TY>
struct Tile {
  static constexpr int kCW = TY / 4;
  static constexpr int kCT = 32 * kCW;
  static constexpr int kThreads = kPT + kCT;
  static constexpr int kColsPerWarp = kTmemCols / (kCW / 4);
  static constexpr int kMaxWz = ((kColsPerWarp / kSlotCols) - 1) | 1;
  static_assert(kCT == TX * (TY / SEGY), "one consumer thread per column segment");
  static_assert(kCW % 4 == 0, "consumer warps cover the four TMEM lane quarters evenly");
};

// W1 == 0: the FIR of half-width W2 (sampled Gaussian) instead of a cascade.
// EB: bytes per raw cube value (4: float32; 2: a 16-bit cube decoded in the
// producers with its per-channel scale).
template <int W1, int W2, int W3, int TY, int EB = 4>
struct Geo {
  static constexpr int R = W1 == 0 ? W2 : (W1 - 1) / 2 + (W2 - 1) / 2 + (W3 - 1) / 2;
  static constexpr int RA = (R + 16 / EB - 1) & ~(16 / EB - 1);  // x halo (16-byte aligned TMA x coordinate)
  static constexpr int BX = TX + 2 * RA;   // raw tile width
  static constexpr int BY = TY + 2 * R;    // raw and quantised tile height
  static constexpr int PX = TX + 2 * R;    // quantised tile width
  static constexpr int XP = PX | 1;        // odd pitch (8-byte words)
  static constexpr int BP = TX + 1;        // odd pitch of the x-pass output
  static constexpr int SEGX = BY * (TX / 8) <= kPT ? 8 : 16;  // x outputs per producer item
  static constexpr int XITEMS = BY * (TX / SEGX);
  static constexpr int NCONV = (BY * PX + kPT - 1) / kPT;
  static constexpr int XBUF = (R <= 8 || (TY <= 16 && R <= 12)) ? 2 : 1;  // quantised tiles (two if they fit)
  static_assert(XITEMS <= kPT, "one x-pass item per producer thread");
  static_assert(4 * BY <= kPT, "one mask word per producer thread");
  static_assert(PX <= 128, "four mask words per row");
};

struct Smem {
  size_t raw[kStages], mw, x, b, hist, mbar, total;
};

template <int W1, int W2, int W3, int TY, int EB = 4>
__host__ __device__ constexpr Smem smem_layout(bool hist) {
  using G = Geo<W1, W2, W3, TY, EB>;
  Smem s{};
  size_t o = 0;
  for (int b = 0; b < kStages; ++b) {
    s.raw[b] = o;
    o = al128(o + (size_t)EB * G::BY * G::BX);
  }
  s.mw = o;  // [2][BY][4] tile-aligned mask words
  o = al128(o + sizeof(unsigned) * 2 * (size_t)G::BY * 4);
  s.x = o;  // [XBUF][BY][XP] quantised tiles
  o = al128(o + sizeof(long long) * G::XBUF * (size_t)G::BY * G::XP);
  s.b = o;  // [2][BY][BP] x-pass output
  o = al128(o + sizeof(long long) * 2 * (size_t)G::BY * G::BP);
  s.hist = o;
  o = al128(o + (hist ? sizeof(unsigned) * kNumBins : 0));
  s.mbar = o;  // raw_full[kStages], bt_full[2], bt_empty[2]
  o = al128(o + (kStages + 4) * sizeof(unsigned long long));
  s.total = o + 128;  // room to align the dynamic base to 128 bytes
  return s;
}

// Quantise the halo'd raw tile into X, in chunks of kConvChunk elements whose
// loads are all issued before their stores (the pointers do not alias).
template <int W1, int W2, int W3, int TY, bool REPL, int EB>
__device__ __forceinline__ void convert_tile(const void* __restrict__ rbv, const unsigned* __restrict__ mwb,
                                             long long* __restrict__ X, int pt, float fscale, long long qrepl,
                                             bool do_repl, int fmt16, float cscale) {
  constexpr int kConvChunk = 4;
  using G = Geo<W1, W2, W3, TY, EB>;
  constexpr int R = G::R, RA = G::RA;
#pragma unroll
  for (int k0 = 0; k0 < G::NCONV; k0 += kConvChunk) {
    float v[kConvChunk];
    unsigned word[kConvChunk];
#pragma unroll
    for (int i = 0; i < kConvChunk; ++i) {
      const int k = k0 + i, e = pt + k * kPT;
      const bool ok = k < G::NCONV && (k + 1 < G::NCONV || e < G::BY * G::PX);
      const int row = e / G::PX, col = e - row * G::PX;
      const int ri = row * G::BX + col + (RA - R);
      if constexpr (EB == 4) {
        v[i] = ok ? static_cast<const float*>(rbv)[ri] : 0.0f;
      } else {
        v[i] = ok ? half16_value(static_cast<const unsigned short*>(rbv)[ri], fmt16, cscale) : 0.0f;
      }
      word[i] = (REPL && do_repl && ok) ? mwb[row * 4 + (col >> 5)] : 0u;
    }
#pragma unroll
    for (int i = 0; i < kConvChunk; ++i) {
      const int k = k0 + i, e = pt + k * kPT;
      if (k < G::NCONV && (k + 1 < G::NCONV || e < G::BY * G::PX)) {
        const int row = e / G::PX, col = e - row * G::PX;
        const bool masked = REPL && do_repl && ((word[i] >> (col & 31)) & 1u);
        X[row * G::XP + col] = quantize_repl(v[i], fscale, masked, qrepl);
      }
    }
  }
}

// x pass of one row segment (SEGX outputs). The pointers do not alias, so
// the stream's loads need not wait for its stores.
template <int W1, int W2, int W3, int TY>
__device__ __forceinline__ void xpass_item(const int* __restrict__ taps, const long long* __restrict__ src,
                                           long long* __restrict__ dst) {
  using G = Geo<W1, W2, W3, TY>;
  spatial_stream<W1, W2, W3, G::SEGX>(taps, [&](int i) { return src[i]; },
                                      [&](int k, long long v) { dst[k] = v; });
}

}  // namespace ws

template <int W1, int W2, int W3, bool REPL, bool TMA, int TY, int EB = 4>
__global__ void __launch_bounds__(ws::Tile<TY>::kThreads, 1)
    k_smooth_ws(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ SmoothArgs a) {
  using namespace ws;
  using G = Geo<W1, W2, W3, TY, EB>;
  static_assert(EB == 4 || TMA, "16-bit cubes are loaded by TMA only");
  using T = Tile<TY>;
  constexpr int kCW = T::kCW, kCT = T::kCT, kThreads = T::kThreads;
  constexpr int R = G::R, RA = G::RA;
  if (a.gate && *a.gate == 0u) return;  // a fallback launch that is not needed (block-uniform)
  extern __shared__ __align__(128) unsigned char smem_dyn[];
  unsigned char* smem = smem_dyn + ((128u - (smem_u32(smem_dyn) & 127u)) & 127u);
  const Smem L = smem_layout<W1, W2, W3, TY, EB>(a.hist != nullptr);
  float* const raw0 = reinterpret_cast<float*>(smem + L.raw[0]);  // (EB == 2: 16-bit values)
  constexpr size_t kRawStride = al128((size_t)EB * G::BY * G::BX) / sizeof(float);
  unsigned* const mw = reinterpret_cast<unsigned*>(smem + L.mw);
  long long* const Xt = reinterpret_cast<long long*>(smem + L.x);
  long long* const Bt = reinterpret_cast<long long*>(smem + L.b);
  unsigned* const hist = reinterpret_cast<unsigned*>(smem + L.hist);
  const unsigned mbar = smem_u32(smem + L.mbar);
  const unsigned raw_full = mbar, bt_full = mbar + 8 * kStages, bt_empty = mbar + 8 * (kStages + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wz = a.pd.wz, r = (wz - 1) / 2;
  const long long nx = a.nx, ny = a.ny, nz = a.nz, plane = nx * ny;
  const long long n_tiles = (long long)a.tiles_x * a.tiles_y;
  const long long n_items = n_tiles * a.zchunks;
  if (a.hist)
    for (int i = tid; i < kNumBins; i += kThreads) hist[i] = 0u;

  __shared__ unsigned tmem_holder;
  if (warp == 0) tmem_alloc(&tmem_holder);
  if (tid == 0) {
    // TMA: one arrival with the byte count; cp.async: one arrival per consumer
    for (int s = 0; s < kStages; ++s) mbar_init(raw_full + 8 * s, TMA ? 1u : (unsigned)kCT);
    for (int b = 0; b < 2; ++b) {
      mbar_init(bt_full + 8 * b, kPW);
      mbar_init(bt_empty + 8 * b, kCW);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  tmem_fence_before();
  __syncthreads();
  tmem_fence_after();
  const unsigned tbase = tmem_holder;
  bool timed_out = false;
  const unsigned long long wait_ns = a.test_skip_handoff ? 1000000ull : kWaitNs;

  auto item_geo = [&](long long it, int* x0, int* y0, int* z0, int* ns) {
    const long long t = it % n_tiles;
    const int zc = (int)(it / n_tiles);
    *x0 = (int)(t % a.tiles_x) * TX;
    *y0 = (int)(t / a.tiles_x) * TY;
    *z0 = zc * a.lz;
    *ns = (int)(min((long long)*z0 + a.lz, nz) - *z0) + 2 * r;
  };

  // Lookahead cursor over the block's planes (its items in order, n_steps
  // planes each): the next raw tile to load and its buffer.
  long long la_item = blockIdx.x;
  int la_j = 0, la_x0 = 0, la_y0 = 0, la_z0 = 0, la_n = 0;
  if (la_item < n_items) item_geo(la_item, &la_x0, &la_y0, &la_z0, &la_n);
  long long issued = 0;
  auto advance = [&]() {
    ++issued;
    if (++la_j == la_n) {
      la_item += gridDim.x;
      la_j = 0;
      if (la_item < n_items) item_geo(la_item, &la_x0, &la_y0, &la_z0, &la_n);
    }
  };
  // TMA load of the next raw tile (one thread)
  auto issue_tma = [&]() {
    if (la_item >= n_items) return;
    const int s = (int)(issued % kStages);
    mbar_expect_tx(raw_full + 8 * s, (unsigned)(EB * G::BX * G::BY));
    tma_load_3d(smem_u32(raw0 + s * kRawStride), &tmap, la_x0 - RA, la_y0 - R, la_z0 - r + la_j, raw_full + 8 * s);
    advance();
  };
  // cp.async load of the next raw tile by the consumers (thread ct copies
  // elements ct, ct + kCT, ...; zero fill outside the cube), completing on the
  // buffer's barrier once each thread's copies have landed
  auto issue_async = [&](int ct) {
    if constexpr (EB == 4) {
      if (la_item >= n_items) return;
      const int s = (int)(issued % kStages);
      float* dst = raw0 + s * kRawStride;
      const long long zp = (long long)la_z0 - r + la_j;
      const bool zok = zp >= 0 && zp < nz;
      for (int e = ct; e < G::BY * G::BX; e += kCT) {
        const int row = e / G::BX, col = e - row * G::BX;
        const long long gx = (long long)la_x0 - RA + col, gy = (long long)la_y0 - R + row;
        const bool ok = zok && gx >= 0 && gx < nx && gy >= 0 && gy < ny;
        cp_async4(smem_u32(dst + e), ok ? a.C + zp * plane + gy * nx + gx : a.C, ok);
      }
      asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(raw_full + 8 * s) : "memory");
      advance();
    }
  };

  if (warp < kPW) {
    // ======================= producers =======================
    const int pt = tid;
    const float fscale = a.st->fx_scale[a.pair];
    const long long qrepl = a.st->fx_qrepl[a.pair];
    const bool do_repl = REPL && qrepl > 0;
    // Mask word k of row `row` of plane zp, aligned to the quantised tile:
    // bit c <-> column 32k + c (gx = x0 - R + 32k + c); bits outside the cube
    // clear. Issued as two loads (MaskLd) and finished once they have arrived.
    struct MaskLd {
      unsigned w0, w1, off;
    };
    const int mrow = pt >> 2, mk = pt & 3;
    auto mask_load = [&](int x0, int y0, int zp) -> MaskLd {
      MaskLd m{0u, 0u, 0u};
      if (do_repl && pt < 4 * G::BY) {
        const long long gy = (long long)y0 - R + mrow;
        if (zp >= 0 && zp < nz && gy >= 0 && gy < ny) {
          const long long vb = (long long)zp * plane + gy * nx + ((long long)x0 - R) + 32 * mk;
          const long long wi = vb >> 5;  // floor division
          const long long nwords = (plane * nz + 31) >> 5;
          m.off = (unsigned)(vb & 31);
          m.w0 = (wi >= 0 && wi < nwords) ? __ldg(a.mbits + wi) : 0u;
          m.w1 = (wi + 1 >= 0 && wi + 1 < nwords) ? __ldg(a.mbits + wi + 1) : 0u;
        }
      }
      return m;
    };
    auto mask_finish = [&](int x0, const MaskLd& m) -> unsigned {
      const unsigned w = __funnelshift_r(m.w0, m.w1, m.off);
      const int g0 = x0 - R + 32 * mk;
      const int lo = g0 < 0 ? -g0 : 0;
      const int hi = (long long)nx - g0 > 32 ? 32 : (int)((long long)nx - g0);
      unsigned keep = 0u;
      if (hi > lo) keep = (hi - lo >= 32) ? 0xffffffffu : (((1u << (hi - lo)) - 1u) << lo);
      return w & keep;
    };
    if (TMA && pt == 0)
      for (int k = 0; k < kLookahead; ++k) issue_tma();
    long long g = 0;
    for (long long item = blockIdx.x; item < n_items; item += gridDim.x) {
      int x0, y0, z0, n_steps;
      item_geo(item, &x0, &y0, &z0, &n_steps);
      MaskLd m_next{0u, 0u, 0u};  // words of plane j + 1, in flight
      if (do_repl) {
        const MaskLd m0 = mask_load(x0, y0, z0 - r);
        m_next = mask_load(x0, y0, z0 - r + 1);
        if (pt < 4 * G::BY) mw[(g & 1) * 4 * G::BY + pt] = mask_finish(x0, m0);
      }
      // a 16-bit cube's values are decoded with their plane's scale, loaded a
      // plane ahead so that its latency hides behind the hand-off waits
      auto plane_scale = [&](int zq) { return (EB == 2 && zq >= 0 && zq < nz) ? __ldg(a.h16.scale + zq) : 1.0f; };
      float cs_next = plane_scale(z0 - r);
      named_bar_sync(kBarProducers, kPT);
      for (int j = 0; j < n_steps; ++j, ++g) {
        const int zp = z0 - r + j;
        const int s = (int)(g % kStages), b = (int)(g & 1);
        const float cs = cs_next;
        cs_next = plane_scale(zp + 1);
        const MaskLd m_after = (do_repl && j + 2 < n_steps) ? mask_load(x0, y0, zp + 2) : MaskLd{0u, 0u, 0u};
        mbar_wait_bounded(raw_full + 8 * s, (unsigned)((g / kStages) & 1), &timed_out, wait_ns);
        mbar_wait_bounded(bt_empty + 8 * b, (unsigned)(((g >> 1) & 1) ^ 1), &timed_out, wait_ns);
        const float* rb = raw0 + s * kRawStride;
        const unsigned* mwb = mw + b * 4 * G::BY;
        long long* const X = Xt + (G::XBUF == 2 ? (size_t)b * G::BY * G::XP : 0);
        // quantise the halo'd tile once
        convert_tile<W1, W2, W3, TY, REPL, EB>(rb, mwb, X, pt, fscale, qrepl, do_repl, a.h16.fmt, cs);
        if (do_repl && j + 1 < n_steps && pt < 4 * G::BY) mw[((g + 1) & 1) * 4 * G::BY + pt] = mask_finish(x0, m_next);
        m_next = m_after;
        // quantised tile and next mask words done; with two tiles, also every
        // producer's x pass of the plane before, so its tile may be refilled
        named_bar_sync(kBarProducers, kPT);
        if (TMA && pt == 0) issue_tma();  // into the buffer of plane g - 2, released by the consumers
        // x pass into buffer b
        if (pt < G::XITEMS) {
          const int row = pt % G::BY, seg = pt / G::BY;
          xpass_item<W1, W2, W3, TY>(a.pd.taps, X + row * G::XP + seg * G::SEGX,
                                 Bt + (size_t)b * G::BY * G::BP + row * G::BP + seg * G::SEGX);
        }
        __syncwarp();
        if (lane == 0 && !(a.test_skip_handoff && warp == 0 && g == 1)) mbar_arrive(bt_full + 8 * b);
        if (G::XBUF == 1) named_bar_sync(kBarProducers, kPT);  // the only quantised tile is free again
      }
    }
    // after a timed-out wait: let the loads still in flight land (bounded)
    // before the block's shared memory is given up
    if (TMA && pt == 0)
      for (long long q = g; q < issued; ++q) {
        bool late = false;
        mbar_wait_bounded(raw_full + 8 * (int)(q % kStages), (unsigned)((q / kStages) & 1), &late);
      }
  } else {
    // ======================= consumers =======================
    const int ct = tid - kPT;
    const int xc = ct & (TX - 1), grp = ct / TX;
    const BinCfg cfg = a.win ? a.st->win : kFullRange;
    const float inv = a.st->fx_inv[a.pair];
    const unsigned tmine =
        tbase + ((unsigned)(32 * (warp & 3)) << 16) + (unsigned)(T::kColsPerWarp * ((warp - kPW) >> 2));
    if (!TMA)
      for (int k = 0; k < kLookahead; ++k) issue_async(ct);
    long long g = 0;
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
        for (int s = 0; s < wz; ++s) tmem_st16(tmine + (unsigned)(kSlotCols * s), zero);
        tmem_wait_st();
      }
      unsigned long long nan_lo = 0ull, nan_hi = 0ull;  // NaN bytes of the last 16 planes, newest lowest
      const long long gx = (long long)x0 + xc;
      const long long gy0 = (long long)y0 + grp * SEGY;
      unsigned rows_in = 0u;  // rows of this thread inside the cube
#pragma unroll
      for (int i = 0; i < SEGY; ++i) rows_in |= (gx < nx && gy0 + i < ny ? 1u : 0u) << i;
      auto plane_scale = [&](int zq) { return (EB == 2 && zq >= 0 && zq < nz) ? __ldg(a.h16.scale + zq) : 1.0f; };
      float cs_next = plane_scale(z0 - r);  // 16-bit cube: the plane's scale, a plane ahead
      for (int j = 0; j < n_steps; ++j, ++g) {
        const int zp = z0 - r + j;
        const int b = (int)(g & 1);
        const float cs_plane = cs_next;
        cs_next = plane_scale(zp + 1);
        // ring slot of this plane: load early, use after the y pass
        unsigned old[kSlotCols];
        const unsigned ta = tmine + (unsigned)(kSlotCols * (j % (wz > 1 ? wz : 1)));
        if (wz > 1) tmem_ld16(ta, old);
        mbar_wait_bounded(bt_full + 8 * b, (unsigned)((g >> 1) & 1), &timed_out, wait_ns);
        long long P[SEGY];
        {
          const long long* src = Bt + (size_t)b * G::BY * G::BP + (grp * SEGY) * G::BP + xc;
          spatial_stream<W1, W2, W3, SEGY>(a.pd.taps, [&](int i) { return src[i * G::BP]; },
                                           [&](int k, long long v) { P[k] = v; });
        }
        unsigned nbyte = 0u;  // which of the 8 voxels are NaN / Inf
        {
          // the tile's load completed before the producers used it; observing
          // its barrier makes the TMA writes visible to this thread as well
          mbar_wait_bounded(raw_full + 8 * (int)(g % kStages), (unsigned)((g / kStages) & 1), &timed_out, wait_ns);
          const float* rbase = raw0 + (size_t)(g % kStages) * kRawStride;
          const int ro = (R + grp * SEGY) * G::BX + RA + xc;
          if constexpr (EB == 4) {
#pragma unroll
            for (int i = 0; i < SEGY; ++i)
              nbyte |= ((__float_as_uint(rbase[ro + i * G::BX]) & 0x7f800000u) == 0x7f800000u ? 1u : 0u) << i;
          } else {
            // the decoded value decides (a finite 16-bit value times its scale may overflow)
            const unsigned short* rb16 = reinterpret_cast<const unsigned short*>(rbase) + ro;
#pragma unroll
            for (int i = 0; i < SEGY; ++i) {
              const float v = half16_value(rb16[i * G::BX], a.h16.fmt, cs_plane);
              nbyte |= ((__float_as_uint(v) & 0x7f800000u) == 0x7f800000u ? 1u : 0u) << i;
            }
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(bt_empty + 8 * b);
        // The buffer of plane g - 2 is free: every consumer warp released that
        // plane before the producers could finish plane g, whose hand-off this
        // thread has passed. Refill it with plane g + 2.
        if (!TMA) issue_async(ct);
        nan_hi = (nan_hi << SEGY) | (nan_lo >> (64 - SEGY));
        nan_lo = (nan_lo << SEGY) | nbyte;
        if (a.pout && j >= r && j < n_steps - r) {
          // the plane's spatial sums and nonfinite flags for the later pairs
          // of this spatial kernel (planes of this chunk only); the thread's
          // 8 rows start at a multiple of 8, so their flags are one byte
          long long* po = a.pout + ((long long)zp * ny + gy0) * a.ppitch + gx;
#pragma unroll
          for (int i = 0; i < SEGY; ++i)
            if ((rows_in >> i) & 1u) po[i * a.ppitch] = P[i];
          if (rows_in & 1u) a.nfout[((long long)zp * ((ny + 7) / 8) + gy0 / 8) * a.nfpitch + gx] = (unsigned char)nbyte;
        }
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
          tmem_st16(ta, nw);
        } else {
#pragma unroll
          for (int i = 0; i < SEGY; ++i) zsum[i] = P[i];
        }
        if (j >= 2 * r) {
          const long long zo = zp - r;
          const unsigned nb =
              (unsigned)((r < 8 ? nan_lo >> (SEGY * r) : nan_hi >> (SEGY * (r - 8))) & ((1ull << SEGY) - 1ull));
          float* out = a.S + zo * plane + gy0 * nx + gx;
#pragma unroll
          for (int i = 0; i < SEGY; ++i) {
            const bool isnan_out = (nb >> i) & 1u;
            const float sv = dequantize(zsum[i], inv);
            const float s = isnan_out ? __int_as_float(0x7fc00000) : sv;
            if ((rows_in >> i) & 1u) {
              out[i * nx] = s;
              if (a.hist && !isnan_out) atomicAdd(&hist[bin_of(s, cfg)], 1u);
            }
          }
        }
        if (wz > 1) tmem_wait_st();
      }
    }
    if (!TMA) cp_async_wait_all();
  }
  tmem_fence_before();
  __syncthreads();
  tmem_fence_after();
  if (warp == 0) tmem_dealloc(tbase);
  if (timed_out) atomicOr(&a.st->status, (unsigned)SC_ST_TIMEOUT);
  if (a.hist)
    for (int i = tid; i < kNumBins; i += kThreads)
      if (hist[i]) atomicAdd(a.hist + i, (unsigned long long)hist[i]);
}

namespace ws {

// One launch of the warp-specialised kernel for the pair (EB = 2: the cube is
// the 16-bit one in a.h16, loaded by TMA; no launch, *done = false, where the
// tiles do not fit or a 16-bit cube is not TMA-addressable).
template <int W1, int W2, int W3, int TY, int EB = 4>
cudaError_t launch_ws(const SmoothArgs& a0, int sms, cudaStream_t s, bool* done) {
  using namespace ws;
  using G = Geo<W1, W2, W3, TY, EB>;
  constexpr int kThreads = Tile<TY>::kThreads;
  SmoothArgs a = a0;
  const Smem L = smem_layout<W1, W2, W3, TY, EB>(a.hist != nullptr);
  if (L.total + 1024 > 227 * 1024) return cudaSuccess;  // not served: the caller falls back
  CUtensorMap map;
  bool tma;
  if constexpr (EB == 4) {
    tma = encode_cube_map(&map, a.C, a.nx, a.ny, a.nz, G::BX, G::BY);  // else the cp.async variant
  } else {
    tma = encode_cube16_map(&map, a.h16.bits, a.nx, a.ny, a.nz, G::BX, G::BY);
    if (!tma) return cudaSuccess;
  }
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
  const bool repl = a.mbits != nullptr && a.repl_possible;
  const size_t smem_req = one_block_per_sm_smem(L.total);
  if (tma) {
    if (repl) k_smooth_ws<W1, W2, W3, true, true, TY, EB><<<grid, kThreads, smem_req, s>>>(map, a);
    else k_smooth_ws<W1, W2, W3, false, true, TY, EB><<<grid, kThreads, smem_req, s>>>(map, a);
  } else if constexpr (EB == 4) {
    if (repl) k_smooth_ws<W1, W2, W3, true, false, TY><<<grid, kThreads, smem_req, s>>>(map, a);
    else k_smooth_ws<W1, W2, W3, false, false, TY><<<grid, kThreads, smem_req, s>>>(map, a);
  }
  *done = true;
  return cudaGetLastError();
}

// Tile height for a spectral width: 32 rows while the ring of w planes fits
// two consumer warps per TMEM lane quarter, else (or when the autotuner chose
// it) 16 rows.
template <int W1, int W2, int W3, int EB = 4>
cudaError_t launch_ws_for_wz(const SmoothArgs& a, int sms, cudaStream_t s, bool* done) {
  const int rows = ws_tile_rows(a);
  if (rows == 32) return launch_ws<W1, W2, W3, 32, EB>(a, sms, s, done);
  if (rows == 16) return launch_ws<W1, W2, W3, 16, EB>(a, sms, s, done);
  return cudaSuccess;
}

template <int W1, int W2, int W3, int TY, int EB = 4>
void set_ws_attr_ty() {
  tc::set_dyn_smem_limit(k_smooth_ws<W1, W2, W3, false, true, TY, EB>);
  tc::set_dyn_smem_limit(k_smooth_ws<W1, W2, W3, true, true, TY, EB>);
  if constexpr (EB == 4) {
    tc::set_dyn_smem_limit(k_smooth_ws<W1, W2, W3, false, false, TY>);
    tc::set_dyn_smem_limit(k_smooth_ws<W1, W2, W3, true, false, TY>);
  }
}

template <int W1, int W2, int W3, int EB = 4>
void set_ws_attr() {
  set_ws_attr_ty<W1, W2, W3, 32, EB>();
  set_ws_attr_ty<W1, W2, W3, 16, EB>();
}

}  // namespace ws

}  // namespace sc
