// Specialised smoothing kernel: compile-time boxcar widths, register-resident
// box cascades, a 64 x 32 output tile per block.
//
// Same arithmetic as the generic kernel (exact int64 fixed point, one final
// rounding; see sc_smooth.cu), so both produce identical floats. Per plane:
//   load   every thread fetches its share of the plane's halo'd tile
//          ((32 + 2R) rows x (64 + 2R) columns) for the NEXT plane into
//          registers while the current plane is processed, then quantises it
//          (NaN -> 0, replacement of masked voxels) into shared memory;
//   x pass (32 + 2R) rows x 4 segments of 16 outputs; each thread slides the
//          three boxcars over its 16 + 2R inputs in registers;
//   y pass 64 columns x 4 segments of 8 outputs, the same way down a column;
//   z      the thread's 8 smoothed values enter a ring of wz planes in shared
//          memory and a running int64 sum gives the spectral boxcar;
//   out    the plane r = (wz - 1) / 2 behind is finished: scale to float, NaN
//          where the input voxel is NaN (from a per-thread bit history), store,
//          histogram.
#include <cstdint>

#include "sc_device.cuh"
#include "sc_internal.h"

namespace sc {

namespace tile {

constexpr int kThreads = 256;
constexpr int TX = 64, TY = 32;
constexpr int SEGX = 16, SEGY = 8;
constexpr int kMaxWzSmem = 7;  // spectral widths served by the shared-memory ring

template <int W1, int W2, int W3>
struct Geo {
  static constexpr int R = (W1 - 1) / 2 + (W2 - 1) / 2 + (W3 - 1) / 2;
  static constexpr int PX = TX + 2 * R;               // quantised tile width
  static constexpr int PY = TY + 2 * R;               // quantised tile height
  static constexpr int XP = PX | 1;                   // odd pitch (int64 units): conflict-free column access
  static constexpr int BP = TX + 1;                   // odd pitch of the x-pass output
  static constexpr int LOAD_SLOTS = (PX + 31) / 32;   // loads per row per lane
  static constexpr int LOAD_ROWS = (PY + 7) / 8;      // rows per warp
  static constexpr int NLOAD = LOAD_SLOTS * LOAD_ROWS;
};

// Sliding sum of W consecutive values of in[0..N) -> out[0..N-W+1), unrolled.
template <int W, int N>
__device__ __forceinline__ void box(const long long (&in)[N], long long (&out)[N - W + 1]) {
  long long s = 0;
#pragma unroll
  for (int k = 0; k < W; ++k) s += in[k];
  out[0] = s;
#pragma unroll
  for (int i = 1; i < N - W + 1; ++i) {
    s += in[i + W - 1] - in[i - 1];
    out[i] = s;
  }
}

template <int W1, int W2, int W3, int N>
__device__ __forceinline__ void cascade(const long long (&in)[N], long long (&out)[N - (W1 - 1) - (W2 - 1) - (W3 - 1)]) {
  long long b1[N - W1 + 1];
  box<W1, N>(in, b1);
  long long b2[N - W1 + 1 - W2 + 1];
  box<W2, N - W1 + 1>(b1, b2);
  box<W3, N - W1 + 1 - W2 + 1>(b2, out);
}

// ---- Tensor Memory (TMEM) as ring storage --------------------------------
// A block allocates all 512 columns of its SM's TMEM (one block per SM). Warp w
// may touch lanes 32*(w%4) .. +31; warps 0-3 use columns 0..255, warps 4-7
// columns 256..511, so every thread owns 256 32-bit words of one lane: 16 ring
// slots of 8 int64 values.
constexpr int kTmemCols = 512;

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void tmem_alloc(unsigned* holder) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(holder)),
               "r"(kTmemCols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(unsigned base) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base), "r"(kTmemCols) : "memory");
}
__device__ __forceinline__ void tmem_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// 8 int64 values <-> 16 consecutive 32-bit columns of the thread's lane.
__device__ __forceinline__ void tmem_ld8(unsigned taddr, unsigned (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tmem_st8(unsigned taddr, const unsigned (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
      "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
      : "memory");
}
constexpr int kMaxWzTmem = 16;  // ring slots per thread in TMEM

struct Smem {
  size_t x, b, ring, hist, total;
};

template <int W1, int W2, int W3>
__host__ __device__ constexpr Smem smem_layout(int wz, bool hist, bool tmem_ring) {
  using G = Geo<W1, W2, W3>;
  Smem s{};
  size_t o = 0;
  s.x = o;
  o += sizeof(long long) * (size_t)G::PY * G::XP;
  s.b = o;
  o += sizeof(long long) * (size_t)G::PY * G::BP;
  s.ring = o;
  o += (tmem_ring || wz <= 1) ? 0 : sizeof(long long) * (size_t)wz * TX * TY;
  s.hist = o;
  o += hist ? sizeof(unsigned int) * kNumBins : 0;
  s.total = o;
  return s;
}

}  // namespace tile

template <int W1, int W2, int W3, bool TMEM>
__global__ void __launch_bounds__(tile::kThreads, 1) k_smooth_tile(SmoothArgs a) {
  using namespace tile;
  using G = Geo<W1, W2, W3>;
  constexpr int R = G::R;
  extern __shared__ __align__(16) unsigned char smem[];
  const int wz = a.pd.wz, r = (wz - 1) / 2;
  const Smem L = smem_layout<W1, W2, W3>(wz, a.hist != nullptr, TMEM);
  long long* Xt = reinterpret_cast<long long*>(smem + L.x);
  long long* Bt = reinterpret_cast<long long*>(smem + L.b);
  long long* ring = reinterpret_cast<long long*>(smem + L.ring);
  unsigned int* hist = reinterpret_cast<unsigned int*>(smem + L.hist);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (a.hist)
    for (int i = tid; i < kNumBins; i += kThreads) hist[i] = 0u;
  const BinCfg cfg = a.win ? a.st->win : kFullRange;
  const int f = a.st->fx_shift[a.pair];
  const float inv = a.st->fx_inv[a.pair];
  const long long qrepl = a.st->fx_qrepl[a.pair];
  const bool do_repl = qrepl > 0 && a.mbits != nullptr;
  const long long nx = a.nx, ny = a.ny, nz = a.nz;
  const long long plane = nx * ny;
  const long long n_items = (long long)a.tiles_x * a.tiles_y * a.zchunks;
  // y pass / output ownership: column yc, rows ys*8 .. ys*8+7
  const int yc = tid & (TX - 1), ys = tid / TX;
  __shared__ unsigned tmem_holder;
  unsigned tbase = 0u;
  if (TMEM) {
    if (warp == 0) tmem_alloc(&tmem_holder);
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    tbase = tmem_holder;
  }
  // this thread's lane and first column in TMEM
  const unsigned tmine = tbase + ((unsigned)(32 * (warp & 3)) << 16) + (unsigned)(256 * (warp >> 2));
  __syncthreads();

  for (long long item = blockIdx.x; item < n_items; item += gridDim.x) {
    const long long tile_id = item % ((long long)a.tiles_x * a.tiles_y);
    const int zc = (int)(item / ((long long)a.tiles_x * a.tiles_y));
    const int x0 = (int)(tile_id % a.tiles_x) * TX, y0 = (int)(tile_id / a.tiles_x) * TY;
    const int z0 = zc * a.lz;
    const int z1 = (int)min((long long)z0 + a.lz, nz);
    const int n_steps = (z1 - z0) + 2 * r;

    long long zsum[SEGY];
#pragma unroll
    for (int i = 0; i < SEGY; ++i) zsum[i] = 0;
    if (wz > 1) {
      if (TMEM) {
        unsigned zero[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) zero[i] = 0u;
        for (int s = 0; s < wz; ++s) tmem_st8(tmine + 16u * s, zero);
        tmem_wait_st();
      } else {
        for (int s = 0; s < wz; ++s)
#pragma unroll
          for (int i = 0; i < SEGY; ++i) ring[((size_t)s * TY + ys * SEGY + i) * TX + yc] = 0;
      }
    }
    unsigned long long nan_hist = 0ull;  // SEGY bits per plane, newest in the low byte

    // register prefetch of one plane's halo'd tile
    static_assert(G::NLOAD <= 32, "mask prefetch bits fit one word");
    float pre[G::NLOAD];
    unsigned int prem = 0u;
    auto fetch = [&](int zp) {
      const bool zok = (zp >= 0 && zp < nz);
      prem = 0u;
#pragma unroll
      for (int rr = 0; rr < G::LOAD_ROWS; ++rr) {
        const int row = warp + 8 * rr;
        const long long gy = (long long)y0 - R + row;
#pragma unroll
        for (int sl = 0; sl < G::LOAD_SLOTS; ++sl) {
          const int col = lane + 32 * sl;
          const long long gx = (long long)x0 - R + col;
          float v = 0.0f;
          unsigned int mb = 0u;
          if (zok && row < G::PY && col < G::PX && gy >= 0 && gy < ny && gx >= 0 && gx < nx) {
            const long long idx = (long long)zp * plane + gy * nx + gx;
            v = __ldg(a.C + idx);
            if (do_repl) mb = (__ldg(a.mbits + (idx >> 5)) >> (idx & 31)) & 1u;
          }
          pre[rr * G::LOAD_SLOTS + sl] = v;
          prem |= mb << (rr * G::LOAD_SLOTS + sl);
        }
      }
    };
    auto commit = [&]() {
#pragma unroll
      for (int rr = 0; rr < G::LOAD_ROWS; ++rr) {
        const int row = warp + 8 * rr;
#pragma unroll
        for (int sl = 0; sl < G::LOAD_SLOTS; ++sl) {
          const int col = lane + 32 * sl;
          if (row < G::PY && col < G::PX) {
            const float v = pre[rr * G::LOAD_SLOTS + sl];
            long long q = 0;
            if (isfinite(v)) {
              q = quantize(v, f);
              if ((prem >> (rr * G::LOAD_SLOTS + sl)) & 1u) q = (v >= 0.0f) ? qrepl : -qrepl;
            }
            Xt[row * G::XP + col] = q;
          }
        }
      }
    };

    fetch(z0 - r);
    for (int j = 0; j < n_steps; ++j) {
      const int zp = z0 - r + j;
      const bool valid = (zp >= 0 && zp < nz);
      // NaN flags of this thread's 8 output voxels in plane zp (center values)
      unsigned int nanbits = 0u;
      if (valid) {
        commit();
      }
      if (j + 1 < n_steps) fetch(zp + 1);
      long long P[SEGY];
      if (valid) {
        __syncthreads();
        // x pass: items (row, segment), row fastest so a warp spans rows
        for (int it = tid; it < G::PY * (TX / SEGX); it += kThreads) {
          const int row = it % G::PY, seg = it / G::PY;
          long long in[SEGX + 2 * R];
#pragma unroll
          for (int k = 0; k < SEGX + 2 * R; ++k) in[k] = Xt[row * G::XP + seg * SEGX + k];
          long long out[SEGX];
          cascade<W1, W2, W3, SEGX + 2 * R>(in, out);
#pragma unroll
          for (int k = 0; k < SEGX; ++k) Bt[row * G::BP + seg * SEGX + k] = out[k];
        }
        __syncthreads();
        {
          long long in[SEGY + 2 * R];
#pragma unroll
          for (int k = 0; k < SEGY + 2 * R; ++k) in[k] = Bt[(ys * SEGY + k) * G::BP + yc];
          cascade<W1, W2, W3, SEGY + 2 * R>(in, P);
        }
        // NaN status of the output voxels' own inputs (tile centre)
        {
          const long long gx = (long long)x0 + yc;
#pragma unroll
          for (int i = 0; i < SEGY; ++i) {
            const long long gy = (long long)y0 + ys * SEGY + i;
            if (gx < nx && gy < ny) {
              const float c = __ldg(a.C + (long long)zp * plane + gy * nx + gx);
              if (!isfinite(c)) nanbits |= 1u << i;
            }
          }
        }
      } else {
#pragma unroll
        for (int i = 0; i < SEGY; ++i) P[i] = 0;
      }
      nan_hist = (nan_hist << SEGY) | nanbits;
      // spectral boxcar: running sum over the last wz planes
      if (wz > 1) {
        const int slot = j % wz;
        if (TMEM) {
          unsigned old[16], nw[16];
          tmem_ld8(tmine + 16u * slot, old);
          tmem_wait_ld();
#pragma unroll
          for (int i = 0; i < SEGY; ++i) {
            const long long o = (long long)(((unsigned long long)old[2 * i + 1] << 32) | old[2 * i]);
            zsum[i] += P[i] - o;
            nw[2 * i] = (unsigned)((unsigned long long)P[i] & 0xffffffffull);
            nw[2 * i + 1] = (unsigned)((unsigned long long)P[i] >> 32);
          }
          tmem_st8(tmine + 16u * slot, nw);
          tmem_wait_st();
        } else {
#pragma unroll
          for (int i = 0; i < SEGY; ++i) {
            long long* rp = ring + ((size_t)slot * TY + ys * SEGY + i) * TX + yc;
            zsum[i] += P[i] - *rp;
            *rp = P[i];
          }
        }
      } else {
#pragma unroll
        for (int i = 0; i < SEGY; ++i) zsum[i] = P[i];
      }
      const int zo = zp - r;
      if (j >= 2 * r) {
        const unsigned int nb = (unsigned int)(nan_hist >> (SEGY * r)) & ((1u << SEGY) - 1u);
        const long long gx = (long long)x0 + yc;
#pragma unroll
        for (int i = 0; i < SEGY; ++i) {
          const long long gy = (long long)y0 + ys * SEGY + i;
          if (gx < nx && gy < ny) {
            float s;
            if ((nb >> i) & 1u) {
              s = __int_as_float(0x7fc00000);
            } else {
              s = dequantize(zsum[i], inv);
              if (a.hist) atomicAdd(&hist[bin_of(s, cfg)], 1u);
            }
            a.S[(long long)zo * plane + gy * nx + gx] = s;
          }
        }
      }
      __syncthreads();
    }
  }
  if (TMEM) {
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    if (warp == 0) tmem_dealloc(tbase);
  }
  if (a.hist) {
    __syncthreads();
    for (int i = tid; i < kNumBins; i += kThreads)
      if (hist[i]) atomicAdd(a.hist + i, (unsigned long long)hist[i]);
  }
}

// ---------------------------------------------------------------------------
namespace {

template <int W1, int W2, int W3, bool TMEM>
cudaError_t launch_tile(const SmoothArgs& a0, int sms, cudaStream_t s, bool* done) {
  using namespace tile;
  SmoothArgs a = a0;
  const Smem L = smem_layout<W1, W2, W3>(a.pd.wz, a.hist != nullptr, TMEM);
  if (L.total + 1024 > 227 * 1024) return cudaSuccess;  // not served: caller falls back
  a.tx = TX;
  a.ty = TY;
  a.tiles_x = (a.nx + TX - 1) / TX;
  a.tiles_y = (a.ny + TY - 1) / TY;
  const long long tiles = (long long)a.tiles_x * a.tiles_y;
  const long long target = 2LL * sms;
  long long zch = (target + tiles - 1) / tiles;
  const long long max_ch = (a.nz + 31) / 32;
  zch = zch < 1 ? 1 : (zch > max_ch ? max_ch : zch);
  a.lz = (int)((a.nz + zch - 1) / zch);
  a.zchunks = (a.nz + a.lz - 1) / a.lz;
  const long long items = tiles * a.zchunks;
  const int grid = (int)(items < sms ? items : sms);
  k_smooth_tile<W1, W2, W3, TMEM><<<grid, kThreads, L.total, s>>>(a);
  *done = true;
  return cudaGetLastError();
}

// Dynamic shared memory limit = the per-block maximum minus the kernel's
// static shared memory.
template <typename K>
void set_dyn_smem_limit(K kernel) {
  cudaFuncAttributes fa{};
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) return;
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}

template <int W1, int W2, int W3>
void set_attr() {
  set_dyn_smem_limit(k_smooth_tile<W1, W2, W3, false>);
  set_dyn_smem_limit(k_smooth_tile<W1, W2, W3, true>);
}

template <int W1, int W2, int W3>
cudaError_t launch_tile_any(const SmoothArgs& a, int sms, cudaStream_t s, bool* done) {
  if (a.pd.wz <= tile::kMaxWzSmem) return launch_tile<W1, W2, W3, false>(a, sms, s, done);
  return launch_tile<W1, W2, W3, true>(a, sms, s, done);
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
// spectral widths up to 7 (ring in shared memory) or 15 (ring in TMEM);
// *done = false when the pair is not served.
cudaError_t launch_smooth_tile(const SmoothArgs& a, int sms, cudaStream_t s, bool* done) {
  *done = false;
  if (a.generic || a.pd.wz > tile::kMaxWzTmem) return cudaSuccess;
  const int* w = a.pd.w;
  if (w[0] == 1 && w[1] == 1 && w[2] == 1) return launch_tile_any<1, 1, 1>(a, sms, s, done);
  if (w[0] == 1 && w[1] == 3 && w[2] == 3) return launch_tile_any<1, 3, 3>(a, sms, s, done);
  if (w[0] == 3 && w[1] == 5 && w[2] == 5) return launch_tile_any<3, 5, 5>(a, sms, s, done);
  if (w[0] == 5 && w[1] == 5 && w[2] == 5) return launch_tile_any<5, 5, 5>(a, sms, s, done);
  if (w[0] == 7 && w[1] == 9 && w[2] == 9) return launch_tile_any<7, 9, 9>(a, sms, s, done);
  return cudaSuccess;
}

}  // namespace sc
