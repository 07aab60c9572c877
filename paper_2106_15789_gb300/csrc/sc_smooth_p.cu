// Shared spatial passes of the smoothing (SoFiA 2 Sect. 4.2 and 5: one
// spatial Gaussian combined with several spectral boxcars; Sect. 6.2: the
// replacement of already-detected voxels at the start of every pair).
//
// For the pairs (K_xy, w_1), (K_xy, w_2), ... of one spatial kernel, the
// replaced input of pair j differs from that of the first pair only at the
// voxels masked since then (the mask only grows):
//
//   X_j = X_1 + D_j,   D_j(v) = sgn(C(v)) n sigma_0 - C(v)  on M_j \ M_1, else 0.
//
// The smoothing is linear and exact in the fixed-point arithmetic of this
// library (every pair of one spatial kernel quantises with the same scale), so
//
//   K_xy * X_j,q = P + K_xy * D_j,q  exactly,   P = K_xy * X_1,q.
//
// The first pair's warp-specialised kernel stores P (int64 per voxel) and
// the nonfinite flags of C (a bit per voxel). Every later pair then:
//
//   prep        lists the voxels of M_j \ M_1 once per bucket (a 64 x ty tile
//               of this kernel and a plane) whose halo'd region holds them,
//               with their cube values: a count pass, an exclusive scan and a
//               fill pass over the two masks;
//   k_smooth_p  streams the P tiles and their flag words by TMA and the
//               bucket's list by a bulk copy; every voxel gathers
//               d K(a) K(b), d = X_j,q - X_1,q, from the listed voxels within
//               reach; then the spectral boxcar runs over the corrected
//               planes (ring in Tensor Memory) and S and its histogram are
//               written.
//
// The result is bit for bit the full kernel's on X_j: the two differ only in
// the order of exact integer additions. Reading 8 bytes of P replaces the
// cube read, quantisation and both spatial cascades of the pair. When a
// pair's list does not fit its buffer, k_smooth_p does nothing and a gated
// launch of the full kernel computes the pair instead.
#include <algorithm>
#include <cstdint>
#include <cstring>

#include "sc_device.cuh"
#include "sc_internal.h"
#include "sc_tile_common.cuh"

namespace sc {
namespace share {

using namespace tc;

constexpr int TX = 64;            // tile width
constexpr int kEnt = 768;         // list entries staged per plane (the rest are read from global memory)
constexpr int kScanChunk = 4096;  // counts per scan block (1024 threads x 4)
// Zero taps either side of the 1-D taps in shared memory: a correction's tap
// index along x (32 columns of a warp against an entry within R) or y
// (4 or 8 rows) then never needs a range check.
constexpr int kTapPad = 32;

__device__ __forceinline__ int floor_div64(int a) { return a >= 0 ? a / TX : -((-a + TX - 1) / TX); }
__device__ __forceinline__ int floor_divt(int a, int t) { return a >= 0 ? a / t : -((-a + t - 1) / t); }

// Calls f(bucket, pos) for every bucket whose halo'd region holds the voxel
// at (x, y) of plane z: tiles t with t*T - R <= c < t*T + T + R along each
// axis; pos = (hy << 8) | hx is the voxel's place in that region. Returns the
// number of buckets.
template <class F>
__device__ __forceinline__ int for_buckets(long long z, int y, int x, const ShareArgs& sh, int R, F f) {
  const int tx_lo = max(0, floor_div64(x - R)), tx_hi = min(sh.tiles_x - 1, (x + R) / TX);
  const int ty_lo = max(0, floor_divt(y - R, sh.ty)), ty_hi = min(sh.tiles_y - 1, (y + R) / sh.ty);
  for (int ty = ty_lo; ty <= ty_hi; ++ty)
    for (int tx = tx_lo; tx <= tx_hi; ++tx) {
      const long long b = (z * sh.tiles_y + ty) * sh.tiles_x + tx;
      const unsigned pos = ((unsigned)(y - (ty * sh.ty - R)) << 8) | (unsigned)(x - (tx * TX - R));
      f(b, pos);
    }
  return (tx_hi - tx_lo + 1) * (ty_hi - ty_lo + 1);
}

// Delta words M_j & ~M_1, four at a time (both masks carry padding words).
// An entry holds the voxel's cube value (high 32 bits) and its place
// (hy << 8 | hx) in the bucket's halo'd tile (low 16 bits).
template <bool FILL>
__global__ void __launch_bounds__(256) k_share_list(const uint32_t* __restrict__ mbits, const float* __restrict__ C,
                                                    Half16 h16, long long n, long long nx, long long ny, ShareArgs sh,
                                                    int R) {
  const long long nq = ((n + 31) / 32 + 3) / 4;
  const long long plane = nx * ny;
  const uint4* m4 = reinterpret_cast<const uint4*>(mbits);
  const uint4* s4 = reinterpret_cast<const uint4*>(sh.msnap);
  const bool write = FILL && sh.ss->overflow == 0u;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < nq;
       q += (long long)gridDim.x * blockDim.x) {
    const uint4 a = __ldg(m4 + q), b = __ldg(s4 + q);
    const unsigned d[4] = {a.x & ~b.x, a.y & ~b.y, a.z & ~b.z, a.w & ~b.w};
    if ((d[0] | d[1] | d[2] | d[3]) == 0u) continue;
    // coordinates of the group's first voxel (divisions once per 128 voxels),
    // then followed voxel by voxel
    long long vcur = 128 * q;
    long long z = vcur / plane;
    const long long rem = vcur - z * plane;
    int y = (int)(rem / nx), x = (int)(rem - (long long)y * nx);
    // counts: consecutive voxels whose halo reaches one and the same bucket
    // (the common case) add to it with one atomic
    long long run_b = -1;
    unsigned run_n = 0u;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      unsigned w = d[k];
      while (w) {
        const int bit = __ffs(w) - 1;
        w &= w - 1u;
        const long long v = (4 * q + k) * 32 + bit;
        if (v >= n) break;
        x += (int)(v - vcur);
        vcur = v;
        while (x >= nx) {
          x -= (int)nx;
          if (++y == ny) {
            y = 0;
            ++z;
          }
        }
        if (FILL) {
          const float cv = h16.fmt ? half16_value(__ldg(h16.bits + v), h16.fmt, __ldg(h16.scale + z)) : __ldg(C + v);
          const unsigned long long cb = (unsigned long long)__float_as_uint(cv) << 32;
          for_buckets(z, y, x, sh, R, [&](long long bk, unsigned pos) {
            const unsigned slot = atomicSub(sh.cnt + bk, 1u) - 1u;
            const unsigned long long idx = (unsigned long long)__ldg(sh.offs + bk) + slot;
            if (write && idx < sh.cap) sh.ent[idx] = cb | pos;
          });
        } else {
          long long only = -1;
          const int nb = for_buckets(z, y, x, sh, R, [&](long long bk, unsigned) { only = bk; });
          if (nb == 1 && only == run_b) {
            ++run_n;
          } else {
            if (run_n) atomicAdd(sh.cnt + run_b, run_n);
            run_b = -1;
            run_n = 0u;
            if (nb == 1) {
              run_b = only;
              run_n = 1u;
            } else {
              for_buckets(z, y, x, sh, R, [&](long long bk, unsigned) { atomicAdd(sh.cnt + bk, 1u); });
            }
          }
        }
      }
    }
    if (!FILL && run_n) atomicAdd(sh.cnt + run_b, run_n);
  }
}

// Exclusive scan of m counts, in chunks of kScanChunk: the chunk's own scan
// and its total.
__global__ void __launch_bounds__(1024) k_share_scan1(const unsigned* __restrict__ cnt, unsigned* __restrict__ offs,
                                                      unsigned long long* __restrict__ bsum, long long m) {
  __shared__ unsigned wsum[32];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const long long base = (long long)blockIdx.x * kScanChunk + 4 * t;
  unsigned v[4], tot = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    v[k] = base + k < m ? cnt[base + k] : 0u;
    tot += v[k];
  }
  unsigned inc = tot;  // inclusive scan over the warp
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) wsum[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    unsigned x = wsum[lane], xi = x;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, xi, o);
      if (lane >= o) xi += y;
    }
    wsum[lane] = xi - x;  // exclusive over warps
    if (lane == 31) bsum[blockIdx.x] = xi;
  }
  __syncthreads();
  unsigned run = wsum[warp] + inc - tot;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (base + k < m) offs[base + k] = run;
    run += v[k];
  }
}

// Adds the totals of the chunks before each chunk; the last chunk's block
// records the grand total and whether it exceeds the list's capacity.
__global__ void __launch_bounds__(1024) k_share_scan2(unsigned* __restrict__ offs,
                                                      const unsigned long long* __restrict__ bsum, long long m,
                                                      ShareState* ss, unsigned long long cap) {
  __shared__ unsigned long long red[32];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  unsigned long long p = 0;
  for (long long i = t; i < blockIdx.x; i += 1024) p += bsum[i];
  for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
  if (lane == 0) red[warp] = p;
  __syncthreads();
  unsigned long long pre = 0;
  for (int w = 0; w < 32; ++w) pre += red[w];
  const long long base = (long long)blockIdx.x * kScanChunk;
  for (int k = t; k < kScanChunk; k += 1024)
    if (base + k < m) offs[base + k] += (unsigned)pre;
  if (blockIdx.x == gridDim.x - 1 && t == 0) {
    const unsigned long long total = pre + bsum[blockIdx.x];
    ss->total = total;
    ss->overflow = total > cap ? 1u : 0u;
  }
}

__device__ __forceinline__ void bulk_load(unsigned dst, const void* src, unsigned bytes, unsigned mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(mbar)
               : "memory");
}

template <int VPT>
struct TmRing;
template <>
struct TmRing<8> {
  static __device__ __forceinline__ void ld(unsigned t, unsigned (&v)[16]) { tmem_ld16(t, v); }
  static __device__ __forceinline__ void st(unsigned t, const unsigned (&v)[16]) { tmem_st16(t, v); }
};
template <>
struct TmRing<4> {
  static __device__ __forceinline__ void ld(unsigned t, unsigned (&v)[8]) { tmem_ld8(t, v); }
  static __device__ __forceinline__ void st(unsigned t, const unsigned (&v)[8]) { tmem_st8(t, v); }
};

struct Meta {
  int item;  // work item of the stage (-1: no more items)
  int j;     // plane index within the item
  unsigned cnt, off0, shift, pad;
};

// Composed integer taps of a three-box cascade (the spatial kernels this
// pass serves, identified by their half-width R), known at compile time.
struct TapArr {
  int v[2 * 11 + 1];
};
__host__ __device__ constexpr TapArr box_taps(int w1, int w2, int w3) {
  TapArr t{};
  const int ws[3] = {w1, w2, w3};
  int len = 1;
  t.v[0] = 1;
  for (int b = 0; b < 3; ++b) {
    TapArr n{};
    for (int i = 0; i < len; ++i)
      for (int d = 0; d < ws[b]; ++d) n.v[i + d] += t.v[i];
    len += ws[b] - 1;
    t = n;
  }
  return t;
}
template <int R>
__host__ __device__ constexpr TapArr taps_for() {
  return R == 2 ? box_taps(1, 3, 3) : (R == 5 ? box_taps(3, 5, 5) : (R == 6 ? box_taps(5, 5, 5) : box_taps(7, 9, 9)));
}

// Roles of a block: kCW compute warps (a thread owns VPT rows of one column
// of the 64 x TY tile, so a warp owns 32 columns x VPT rows; the warps of one
// TMEM lane quarter split its 512 columns, which bounds the spectral ring to
// kMaxWz planes: 7 for TY 64, 15 for TY 32, 31 for TY 16) and one issuing
// warp. TY 64 tiles give a thread 8 rows (the per-plane work of a thread is
// spread over twice the voxels, and twice the voxels are in flight) and keep
// 4 P tiles of 32 KB in flight; the others 8 tiles of 16 or 8 KB.
template <int TY, int R>
struct PGeo {
  static constexpr int VPT = TY >= 64 ? 8 : 4;
  static constexpr int kStages = TY >= 64 ? 4 : 8;  // P tiles in flight (a power of two)
  static constexpr int kBars = 2 * kStages;          // full[kStages] (TMA landed), empty[kStages] (consumed)
  static constexpr int kCW = TX * TY / (32 * VPT);   // compute warps
  static constexpr int kCT = 32 * kCW;
  static constexpr int kIssuer = kCW;          // warp index of the issuing warp
  static constexpr int kThreads = kCT + 32;
  static constexpr int NT = 2 * R + 1;         // taps per axis
  static constexpr int kSlotCols = 2 * VPT;    // TMEM columns per ring slot
  static constexpr int kColsPerWarp = kTmemCols / (kCW / 4);
  static constexpr int kMaxWz = (kColsPerWarp / kSlotCols - 1) | 1;
  static constexpr size_t kPBytes = sizeof(long long) * TY * TX;
  static constexpr size_t kNfBytes = TX * (TY / 8);  // a flag byte per column and 8 rows
  static_assert(kCT == TX * (TY / VPT), "one compute thread per column segment");
  static_assert(kCW % 4 == 0, "compute warps cover the TMEM lane quarters evenly");
  static_assert(VPT <= 8 && 8 % VPT == 0, "a thread's rows lie in one flag byte");
  static_assert(VPT - 1 <= kTapPad, "row tap indices stay inside the padded taps");
  static_assert(TY + 2 * R <= 256 && TX + 2 * R <= 256, "positions fit 8 bits per axis");
};

struct PSmem {
  size_t p, nf, e, kk, meta, hist, mbar, total;
};

template <int TY, int R>
__host__ __device__ constexpr PSmem p_layout() {
  using G = PGeo<TY, R>;
  constexpr int kStages = G::kStages;
  PSmem s{};
  size_t o = 0;
  s.p = o;  // [kStages][TY][64] P tiles
  o = al128(o + kStages * G::kPBytes);
  s.nf = o;  // [kStages][TY / 8][64] flag bytes
  o = al128(o + kStages * G::kNfBytes);
  s.e = o;  // [kStages][kEnt] list entries
  o = al128(o + sizeof(unsigned long long) * kStages * kEnt);
  s.kk = o;  // [kTapPad + NT + kTapPad] 1-D taps, zero outside
  o = al128(o + sizeof(int) * (G::NT + 2 * kTapPad));
  s.meta = o;
  o = al128(o + sizeof(Meta) * kStages);
  s.hist = o;
  o = al128(o + sizeof(unsigned) * kNumBins);
  s.mbar = o;
  o = al128(o + G::kBars * sizeof(unsigned long long));
  s.total = o + 128;
  return s;
}

}  // namespace share

// Work items (a 64 x TY tile and a chunk of lz planes, with r halo planes on
// each side) are handed out by an atomic counter, so blocks whose tiles hold
// many corrections do not hold the kernel up. Per plane: the issuing warp
// takes a free stage and loads the P tile and its flag words (TMA) and the bucket's list (bulk
// copy); each compute warp gathers the corrections of its 32 x VPT voxels
// from the list (32 entries tested at once by a ballot; a lane adds only to
// its own voxels, so no atomics), runs the spectral ring and writes S. Stages carry the item and plane index,
// and a last stage with item -1 ends the block.
template <int TY, int R>
__global__ void __launch_bounds__(share::PGeo<TY, R>::kThreads, 1)
    k_smooth_p(const __grid_constant__ CUtensorMap pmap, const __grid_constant__ CUtensorMap nfmap, SmoothArgs a,
               ShareArgs sh) {
  using namespace share;
  using G = PGeo<TY, R>;
  constexpr int NT = G::NT, kCW = G::kCW, kThreads = G::kThreads, VPT = G::VPT, kStages = G::kStages;
  if (sh.ss->overflow) return;  // the gated full kernel computes this pair (block-uniform)
  extern __shared__ __align__(128) unsigned char smem_dyn[];
  unsigned char* smem = smem_dyn + ((128u - (smem_u32(smem_dyn) & 127u)) & 127u);
  constexpr PSmem L = p_layout<TY, R>();
  long long* const Ps = reinterpret_cast<long long*>(smem + L.p);
  const unsigned char* const NFs = smem + L.nf;
  unsigned long long* const Es = reinterpret_cast<unsigned long long*>(smem + L.e);
  int* const taps1 = reinterpret_cast<int*>(smem + L.kk);
  Meta* const meta = reinterpret_cast<Meta*>(smem + L.meta);
  unsigned* const hist = reinterpret_cast<unsigned*>(smem + L.hist);
  const unsigned mbar = smem_u32(smem + L.mbar);
  const unsigned full = mbar, empty = mbar + 8 * kStages;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wz = a.pd.wz, r = (wz - 1) / 2;
  const long long nx = a.nx, ny = a.ny, nz = a.nz, plane = nx * ny;
  const long long n_tiles = (long long)sh.tiles_x * sh.tiles_y;
  const long long n_items = n_tiles * a.zchunks;

  if (a.hist)
    for (int i = tid; i < kNumBins; i += kThreads) hist[i] = 0u;
  for (int i = tid; i < NT + 2 * kTapPad; i += kThreads) taps1[i] = 0;
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NT; ++i)
    if (tid == i) taps1[kTapPad + i] = a.pd.taps[i];  // compile-time indices: read from the kernel parameters
  __shared__ unsigned tmem_holder;
  if (warp == 0) tmem_alloc(&tmem_holder);
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(full + 8 * s, 1u);
      mbar_init(empty + 8 * s, (unsigned)kCW);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  tmem_fence_before();
  __syncthreads();
  tmem_fence_after();
  const unsigned tbase = tmem_holder;
  bool timed_out = false;

  auto item_geo = [&](long long it, int* x0, int* y0, int* z0, int* ns) {
    const long long t = it % n_tiles;
    const int zc = (int)(it / n_tiles);
    *x0 = (int)(t % sh.tiles_x) * TX;
    *y0 = (int)(t / sh.tiles_x) * TY;
    *z0 = zc * a.lz;
    *ns = (int)(min((long long)*z0 + a.lz, nz) - *z0) + 2 * r;
  };

  if (warp == G::kIssuer) {
    // ===================== issuing warp =====================
    auto grab = [&]() -> long long {
      unsigned long long v = 0ull;
      if (lane == 0) v = atomicAdd(&sh.ss->next_item, 1ull);
      return (long long)__shfl_sync(0xffffffffu, v, 0);
    };
    // List bounds of up to 32 planes of one item per batch; lane l holds those
    // of plane j0 + l. The next batch is fetched while this one is issued.
    auto load_batch = [&](long long it, int j0, unsigned* o0, unsigned* o1) {
      *o0 = 0u;
      *o1 = 0u;
      if (!sh.offs || it >= n_items) return;
      int x0, y0, z0, ns;
      item_geo(it, &x0, &y0, &z0, &ns);
      const int jl = j0 + lane;
      const long long zl = (long long)z0 - r + jl;
      if (jl < ns && zl >= 0 && zl < nz) {
        const long long b = (zl * sh.tiles_y + y0 / TY) * sh.tiles_x + x0 / TX;
        *o0 = __ldg(sh.offs + b);
        *o1 = __ldg(sh.offs + b + 1);
      }
    };
    unsigned g = 0;  // stages published
    long long cur = grab();
    long long nxt = cur < n_items ? grab() : n_items;
    int j0 = 0;
    unsigned c0, c1;
    load_batch(cur, 0, &c0, &c1);
    while (cur < n_items) {
      int x0, y0, z0, ns;
      item_geo(cur, &x0, &y0, &z0, &ns);
      const bool last = j0 + 32 >= ns;
      unsigned n0, n1;
      load_batch(last ? nxt : cur, last ? 0 : j0 + 32, &n0, &n1);
      const int nj = min(32, ns - j0);
      for (int jj = 0; jj < nj; ++jj, ++g) {
        const unsigned b0 = __shfl_sync(0xffffffffu, c0, jj), b1 = __shfl_sync(0xffffffffu, c1, jj);
        if (lane == 0) {
          const int s = (int)(g & (kStages - 1));
          mbar_wait_bounded(empty + 8 * s, ((g / kStages) & 1u) ^ 1u, &timed_out);
          const unsigned cnt = b1 - b0, shift = b0 & 1u;
          unsigned ncp = cnt ? min(cnt + shift, (unsigned)kEnt) : 0u;
          ncp = (ncp + 1u) & ~1u;  // whole 16-byte units (the list has two spare entries)
          meta[s] = Meta{(int)cur, j0 + jj, cnt, b0, shift, 0u};
          mbar_expect_tx(full + 8 * s, (unsigned)(G::kPBytes + G::kNfBytes + 8u * ncp));
          tma_load_3d(smem_u32(Ps + (size_t)s * TY * TX), &pmap, x0, y0, z0 - r + j0 + jj, full + 8 * s);
          tma_load_3d(smem_u32(NFs + (size_t)s * G::kNfBytes), &nfmap, x0, y0 / 8, z0 - r + j0 + jj, full + 8 * s);
          if (ncp) bulk_load(smem_u32(Es + (size_t)s * kEnt), sh.ent + (b0 - shift), 8u * ncp, full + 8 * s);
        }
        __syncwarp();
      }
      c0 = n0;
      c1 = n1;
      if (last) {
        cur = nxt;
        nxt = cur < n_items ? grab() : n_items;
        j0 = 0;
      } else {
        j0 += 32;
      }
    }
    if (lane == 0) {
      // the last stage: no item
      const int s = (int)(g & (kStages - 1));
      mbar_wait_bounded(empty + 8 * s, ((g / kStages) & 1u) ^ 1u, &timed_out);
      meta[s] = Meta{-1, 0, 0u, 0u, 0u, 0u};
      mbar_arrive(full + 8 * s);
      ++g;
      // let every load still in flight land before the block gives up its shared memory
      for (unsigned q = g > (unsigned)kStages ? g - kStages : 0u; q < g; ++q) {
        bool late = false;
        mbar_wait_bounded(full + 8 * (int)(q & (kStages - 1)), (q / kStages) & 1u, &late);
      }
    }
    __syncwarp();
  } else {
    // ===================== compute warps =====================
    const int xc = tid & (TX - 1), grp = tid >> 6;
    const unsigned tmine =
        tbase + ((unsigned)(32 * (warp & 3)) << 16) + (unsigned)(G::kColsPerWarp * (warp >> 2));
    const BinCfg cfg = a.win ? a.st->win : kFullRange;
    const float inv = a.st->fx_inv[a.pair];
    const float fscale = a.st->fx_scale[a.pair];
    const long long qrepl = a.st->fx_qrepl[a.pair];
    const int wx0 = xc & ~31, wy0 = grp * VPT;  // the warp's 32 x VPT voxels
    const bool want_hist = a.hist != nullptr;
    // histogram bin (as bin_of): magnitude bits shifted, windowed, clamped, mirrored for negatives
    const int bin_shift = 23 - cfg.MB, bin_base = (cfg.e_base << cfg.MB) - 1, bin_top = (cfg.E << cfg.MB) + 1;
    long long zsum[VPT];
    unsigned long long nfh = 0ull;  // nonfinite flags of the recent planes, newest lowest
    unsigned rows_in = 0u;
    float* out = nullptr;
    int slot = 0;
    for (unsigned g = 0;; ++g) {
      const int s = (int)(g & (kStages - 1));
      mbar_wait_bounded(full + 8 * s, (g / kStages) & 1u, &timed_out);
      if (timed_out) break;
      const Meta md = meta[s];
      if (md.item < 0) break;
      if (md.j == 0) {
        int x0, y0, z0, ns;
        item_geo(md.item, &x0, &y0, &z0, &ns);
#pragma unroll
        for (int i = 0; i < VPT; ++i) zsum[i] = 0;
        if (wz > 1) {
          unsigned zero[2 * VPT];
#pragma unroll
          for (int i = 0; i < 2 * VPT; ++i) zero[i] = 0u;
          for (int k = 0; k < wz; ++k) TmRing<VPT>::st(tmine + (unsigned)(G::kSlotCols * k), zero);
          tmem_wait_st();
        }
        nfh = 0ull;
        slot = 0;
        const long long gx = (long long)x0 + xc;
        const long long gy0 = (long long)y0 + grp * VPT;
        rows_in = 0u;
#pragma unroll
        for (int i = 0; i < VPT; ++i) rows_in |= (gx < nx && gy0 + i < ny ? 1u : 0u) << i;
        out = a.S + (long long)z0 * plane + gy0 * nx + gx;  // output plane z0 + (j - 2r) once j >= 2r
      }
      // 4 rows a thread: the ring's oldest plane is loaded before the
      // corrections, so that its latency overlaps them
      unsigned old[8];
      const unsigned ta = tmine + (unsigned)(G::kSlotCols * slot);
      if constexpr (VPT == 4) {
        if (wz > 1) TmRing<4>::ld(ta, old);
      }
      long long p[VPT];
      const long long* pt = Ps + (size_t)s * TY * TX + (grp * VPT) * TX + xc;
#pragma unroll
      for (int i = 0; i < VPT; ++i) p[i] = pt[i * TX];
      if (md.cnt > 0u && qrepl > 0) {
        // corrections d K(a) K(b) of the listed voxels within reach: the lanes
        // load 32 entries at once, a ballot marks those that can reach the
        // warp's 32 x VPT voxels, and only those are broadcast and applied
        const unsigned long long* es = Es + (size_t)s * kEnt;
        for (unsigned i0 = 0; i0 < md.cnt; i0 += 32) {
          const unsigned i = i0 + (unsigned)lane;
          unsigned long long e = 0xffffull;  // beyond the list: a place no warp can reach
          if (i < md.cnt) e = (i + md.shift < (unsigned)kEnt) ? es[i + md.shift] : __ldg(sh.ent + md.off0 + i);
          const int ly = (int)(((unsigned)e >> 8) & 0xffu) - R, lx = (int)((unsigned)e & 0xffu) - R;
          const bool near = lx + R >= wx0 && lx - R < wx0 + 32 && ly + R >= wy0 && ly - R < wy0 + VPT;
          unsigned reach = __ballot_sync(0xffffffffu, near);
          // each lane quantises its own entry: d = X_j,q - X_1,q at that voxel,
          // sgn(C) (qrepl - rint(|C| 2^f)) with sgn(0) = +1
          long long dl = 0;
          if (near) {
            const float c = __uint_as_float((unsigned)(e >> 32));
            dl = qrepl - quantize(fabsf(c), fscale);
            if (c < 0.0f) dl = -dl;
          }
          while (reach) {
            // two entries per round, so that their latencies overlap (a
            // missing second one is the unreachable place)
            const int s0 = __ffs(reach) - 1;
            reach &= reach - 1u;
            const int s1 = reach ? __ffs(reach) - 1 : 0;
            const bool two = reach != 0u;
            reach &= reach - 1u;
            const unsigned ej0 = __shfl_sync(0xffffffffu, (unsigned)e, s0);
            const unsigned ej1 = __shfl_sync(0xffffffffu, (unsigned)e, two ? s1 : s0);
            const long long d0 = __shfl_sync(0xffffffffu, dl, s0);
            const long long d1 = two ? __shfl_sync(0xffffffffu, dl, s1) : 0ll;  // a missing second entry adds 0
            // entries within reach: tap indices b in [-31, 31 + 2R] along x and
            // a in [-3, 3 + 2R] along y, inside the zero-padded taps
            const int jy0 = (int)((ej0 >> 8) & 0xffu) - R, jx0 = (int)(ej0 & 0xffu) - R;
            const int jy1 = (int)((ej1 >> 8) & 0xffu) - R, jx1 = (int)(ej1 & 0xffu) - R;
            const int* tp = taps1 + kTapPad + R;
            const long long dk0 = d0 * tp[xc - jx0];
            const long long dk1 = d1 * tp[xc - jx1];
#pragma unroll
            for (int k = 0; k < VPT; ++k) {
              p[k] += dk0 * tp[wy0 + k - jy0];
              p[k] += dk1 * tp[wy0 + k - jy1];
            }
          }
        }
      }
      // rows grp VPT .. + VPT - 1: the flag byte of their 8 rows, or half of it
      const unsigned nb = ((unsigned)NFs[(size_t)s * G::kNfBytes + (grp * VPT / 8) * TX + xc] >> ((grp * VPT) & 7)) &
                          ((1u << VPT) - 1u);
      __syncwarp();
      if (lane == 0) mbar_arrive(empty + 8 * s);
      if (wz > 1) {
        // 8 rows a thread: the oldest plane is taken and replaced 4 rows at a
        // time (fewer registers live across the corrections)
#pragma unroll
        for (int h = 0; h < VPT / 4; ++h) {
          unsigned nw[8];
          if constexpr (VPT == 8) tmem_ld8(ta + 8u * h, old);
          tmem_wait_ld();
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const long long o = (long long)(((unsigned long long)old[2 * i + 1] << 32) | old[2 * i]);
            zsum[4 * h + i] += p[4 * h + i] - o;
            nw[2 * i] = (unsigned)((unsigned long long)p[4 * h + i] & 0xffffffffull);
            nw[2 * i + 1] = (unsigned)((unsigned long long)p[4 * h + i] >> 32);
          }
          tmem_st8(ta + 8u * h, nw);
        }
        if (++slot == wz) slot = 0;
      } else {
#pragma unroll
        for (int i = 0; i < VPT; ++i) zsum[i] = p[i];
      }
      nfh = (nfh << VPT) | nb;
      if (md.j >= 2 * r) {
        const unsigned nbo = (unsigned)(nfh >> (VPT * r)) & ((1u << VPT) - 1u);
#pragma unroll
        for (int i = 0; i < VPT; ++i) {
          const bool isn = (nbo >> i) & 1u;
          const float sv = dequantize(zsum[i], inv);
          const float sval = isn ? __int_as_float(0x7fc00000) : sv;
          if ((rows_in >> i) & 1u) {
            out[i * nx] = sval;
            if (want_hist && !isn) {
              const unsigned u = __float_as_uint(sval);
              const int bm = min(max((int)((u & 0x7fffffffu) >> bin_shift) - bin_base, 0), bin_top);
              atomicAdd(&hist[kBinsPerSign + (bm ^ ((int)u >> 31))], 1u);
            }
          }
        }
        out += plane;
      }
      if (wz > 1) tmem_wait_st();
    }
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

// ---------------------------------------------------------------------------
namespace {

// int64 tensor map of a [nz][ny][pitch] array with an nx-wide row, (bx, ty, 1) boxes
bool encode_p_map(CUtensorMap* map, const long long* base, long long nx, long long ny, long long nz, long long pitch,
                  int bx, int ty) {
  memset(map, 0, sizeof(*map));
  if (pitch % 2 != 0 || (reinterpret_cast<uintptr_t>(base) & 15u) != 0) return false;
  PFN_cuTensorMapEncodeTiled_v12000 enc = tc::tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
  const cuuint64_t strides[2] = {(cuuint64_t)pitch * 8, (cuuint64_t)pitch * ny * 8};
  const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)ty, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult cr = enc(map, CU_TENSOR_MAP_DATA_TYPE_INT64, 3, const_cast<long long*>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return cr == CUDA_SUCCESS;
}

// uint8 tensor map of the [nz][nyb][pitch] flag bytes, (bx, by, 1) boxes
bool encode_nf_map(CUtensorMap* map, const unsigned char* base, long long nx, long long nyb, long long nz,
                   long long pitch, int bx, int by) {
  memset(map, 0, sizeof(*map));
  if (pitch % 16 != 0 || (reinterpret_cast<uintptr_t>(base) & 15u) != 0) return false;
  PFN_cuTensorMapEncodeTiled_v12000 enc = tc::tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)nyb, (cuuint64_t)nz};
  const cuuint64_t strides[2] = {(cuuint64_t)pitch, (cuuint64_t)pitch * nyb};
  const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult cr = enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, const_cast<unsigned char*>(base), dims, strides, box,
                          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return cr == CUDA_SUCCESS;
}

// Half-width R of the shared-pass instance that serves a spatial kernel: the
// cascades' own half-widths; for a sampled Gaussian of half-width h the
// smallest instantiated R >= h (its taps centred and zero-padded to 2R + 1).
int share_R(const PairDesc& pd) {
  if (pd.sampled) {
    for (int r : {4, 8, 9, 12, 16})
      if (pd.h <= r) return pd.h >= 1 ? r : -1;
    return -1;
  }
  const int* w = pd.w;
  if (w[0] == 1 && w[1] == 3 && w[2] == 3) return 2;
  if (w[0] == 3 && w[1] == 5 && w[2] == 5) return 5;
  if (w[0] == 5 && w[1] == 5 && w[2] == 5) return 6;
  if (w[0] == 7 && w[1] == 9 && w[2] == 9) return 11;
  return -1;
}

template <int TY, int R>
cudaError_t launch_p(const SmoothArgs& a0, const ShareArgs& sh, int sms, cudaStream_t s) {
  using namespace share;
  constexpr PSmem L = p_layout<TY, R>();
  SmoothArgs a = a0;
  if (a0.pd.sampled) {
    // the sampled Gaussian's 2h + 1 taps centred in 2R + 1
    const int h = a0.pd.h;
    if (h > R) return cudaErrorInvalidValue;
    for (int i = 0; i < 2 * kMaxHalf + 1; ++i) a.pd.taps[i] = 0;
    for (int i = 0; i < 2 * h + 1; ++i) a.pd.taps[R - h + i] = a0.pd.taps[i];
  } else if (R <= 11) {
    constexpr TapArr K = taps_for<(R <= 11 ? R : 11)>();
    for (int i = 0; i < 2 * R + 1; ++i)
      if (a0.pd.taps[i] != K.v[i]) return cudaErrorInvalidValue;  // not the cascade this instance serves
  } else {
    return cudaErrorInvalidValue;
  }
  CUtensorMap map, nfmap;
  if (!encode_p_map(&map, sh.P, a.nx, a.ny, a.nz, sh.pitch, TX, TY) ||
      !encode_nf_map(&nfmap, sh.nf, a.nx, (a.ny + 7) / 8, a.nz, sh.nfpitch, TX, TY / 8))
    return cudaErrorInvalidValue;
  // z chunks (items are handed out dynamically): the planes a block streams
  // on average, halo planes included, plus one item's planes for the tail
  const long long tiles = (long long)sh.tiles_x * sh.tiles_y;
  const int r = (a.pd.wz - 1) / 2;
  long long best = -1;
  double best_cost = 0.0;
  const long long max_ch = std::max(1LL, (long long)a.nz / 16);
  for (long long zch = 1; zch <= std::min(max_ch, 64LL); ++zch) {
    const long long lz = (a.nz + zch - 1) / zch;
    const long long chunks = (a.nz + lz - 1) / lz;
    const double cost = (double)(a.nz + chunks * 2 * r) * tiles / sms + (double)(lz + 2 * r);
    if (best < 0 || cost < best_cost) {
      best = lz;
      best_cost = cost;
    }
  }
  a.lz = (int)best;
  a.zchunks = (a.nz + a.lz - 1) / a.lz;
  const long long items = tiles * a.zchunks;
  const int grid = (int)std::min<long long>(items, (long long)sms);
  k_smooth_p<TY, R><<<grid, PGeo<TY, R>::kThreads, tc::one_block_per_sm_smem(L.total), s>>>(map, nfmap, a, sh);
  return cudaGetLastError();
}

template <int TY>
cudaError_t launch_p_ty(const SmoothArgs& a, const ShareArgs& sh, int R, int sms, cudaStream_t s) {
  switch (R) {
    case 2: return launch_p<TY, 2>(a, sh, sms, s);
    case 4: return launch_p<TY, 4>(a, sh, sms, s);
    case 5: return launch_p<TY, 5>(a, sh, sms, s);
    case 6: return launch_p<TY, 6>(a, sh, sms, s);
    case 8: return launch_p<TY, 8>(a, sh, sms, s);
    case 9: return launch_p<TY, 9>(a, sh, sms, s);
    case 11: return launch_p<TY, 11>(a, sh, sms, s);
    case 12: return launch_p<TY, 12>(a, sh, sms, s);
    case 16: return launch_p<TY, 16>(a, sh, sms, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int TY, int R>
void set_p_attr() {
  tc::set_dyn_smem_limit(k_smooth_p<TY, R>);
}

}  // namespace

int share_tile_rows(int wz) {
  if (wz <= share::PGeo<64, 2>::kMaxWz) return 64;
  if (wz <= share::PGeo<32, 2>::kMaxWz) return 32;
  if (wz <= share::PGeo<16, 2>::kMaxWz) return 16;
  return 0;
}

bool share_supported(const PairDesc& pd) {
  const int R = share_R(pd);
  return pd.h > 0 && (pd.sampled ? R >= pd.h : R == pd.h) && pd.wz <= kShareMaxWz && share_tile_rows(pd.wz) > 0;
}

cudaError_t launch_share_prep(const SmoothArgs& a, const ShareArgs& sh, int sms, cudaStream_t s) {
  using namespace share;
  const long long n = (long long)a.nx * a.ny * a.nz;
  const int R = share_R(a.pd);  // the reach the shared pass decodes its entries with
  const long long m = sh.n_buckets + 1;
  const long long nblk = (m + kScanChunk - 1) / kScanChunk;
  k_share_list<false><<<8 * sms, 256, 0, s>>>(a.mbits, a.C, a.h16, n, a.nx, a.ny, sh, R);
  k_share_scan1<<<(unsigned)nblk, 1024, 0, s>>>(sh.cnt, sh.offs, sh.bsum, m);
  k_share_scan2<<<(unsigned)nblk, 1024, 0, s>>>(sh.offs, sh.bsum, m, sh.ss, sh.cap);
  k_share_list<true><<<8 * sms, 256, 0, s>>>(a.mbits, a.C, a.h16, n, a.nx, a.ny, sh, R);
  return cudaGetLastError();
}

cudaError_t launch_smooth_p(const SmoothArgs& a, const ShareArgs& sh, int sms, cudaStream_t s, bool* done) {
  *done = false;
  if (!share_supported(a.pd)) return cudaSuccess;
  const int ty = share_tile_rows(a.pd.wz);
  if (ty != sh.ty) return cudaSuccess;
  const int R = share_R(a.pd);
  const cudaError_t e = ty == 64   ? launch_p_ty<64>(a, sh, R, sms, s)
                        : ty == 32 ? launch_p_ty<32>(a, sh, R, sms, s)
                                   : launch_p_ty<16>(a, sh, R, sms, s);
  if (e == cudaSuccess) *done = true;
  return e;
}

void init_share_attrs() {
  set_p_attr<64, 2>();
  set_p_attr<64, 5>();
  set_p_attr<64, 6>();
  set_p_attr<64, 11>();
  set_p_attr<32, 2>();
  set_p_attr<32, 5>();
  set_p_attr<32, 6>();
  set_p_attr<32, 11>();
  set_p_attr<16, 2>();
  set_p_attr<16, 5>();
  set_p_attr<16, 6>();
  set_p_attr<16, 11>();
  // sampled Gaussians (half-widths up to 4, 8, 9, 12, 16)
  set_p_attr<64, 4>();
  set_p_attr<64, 8>();
  set_p_attr<64, 9>();
  set_p_attr<64, 12>();
  set_p_attr<64, 16>();
  set_p_attr<32, 4>();
  set_p_attr<32, 8>();
  set_p_attr<32, 9>();
  set_p_attr<32, 12>();
  set_p_attr<32, 16>();
  set_p_attr<16, 4>();
  set_p_attr<16, 8>();
  set_p_attr<16, 9>();
  set_p_attr<16, 12>();
  set_p_attr<16, 16>();
}

}  // namespace sc
