// Local noise normalisation (SoFiA 2 Sect. 4.1, windows of 31 pixels and
// channels in the speed test of Sect. 5): the cube is divided by the noise
// level measured in a window around each voxel's cell.
//
//   k_noise_window  one block per cell (persistent over cells): the finite
//                   voxels of the cell's window, clipped to the cube, go into
//                   shared memory as order-preserving keys; the noise of the
//                   chosen mode comes from them: MAD by two exact radix
//                   selections in shared memory (the median, then the median
//                   of the float32 keys |x - m|, rounded correctly for an odd
//                   count and faithfully for an even one), STD by two passes
//                   of compensated float32 sums combined in double. Writes
//                   the cell's noise (double) and the float32 reciprocal used
//                   below.
//   k_noise_apply   out = in * (1 / sigma) per voxel (NaN where the input is
//                   not finite or the cell has no positive noise).
//
// Cells are gx x gy x gz voxels (the last one along an axis may be shorter);
// a cell's window is centred on voxel start + (extent - 1) / 2 of each axis.
#include <cstdint>

#include "sc_device.cuh"
#include "sc_gaussfit.cuh"
#include "sc_internal.h"

namespace sc {
namespace nscale {

constexpr int kThreads = 1024;
constexpr int kWarps = kThreads / 32;
constexpr int kBins = 2048;              // radix digits: 11, 11 and 10 bits
constexpr unsigned kNone = 0xffffffffu;  // key of a non-finite voxel: above every finite key
constexpr double kMadToSigma = 1.4826;
constexpr int kCandCap = 6144;  // keys of one round-0 bin copied aside for the later rounds

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
  unsigned digit, rank, next, count, below;
};

// Adds this lane's digit to a histogram; lanes of the warp with the same digit
// add once. bin == kBins: nothing to add. All 32 lanes must call it.
__device__ __forceinline__ void hist_add_warp(unsigned* hist, unsigned bin) {
  const unsigned peers = __match_any_sync(0xffffffffu, bin);
  if ((threadIdx.x & 31) == __ffs(peers) - 1 && bin < (unsigned)kBins) atomicAdd(&hist[bin], __popc(peers));
}

// Appends k to out[] (at most cap entries) where `take`; the counter ends as
// the number of takers, which may exceed cap. All 32 lanes must call it.
__device__ __forceinline__ void append_warp(bool take, unsigned k, unsigned* out, unsigned cap, unsigned* counter) {
  const unsigned ball = __ballot_sync(0xffffffffu, take);
  if (ball) {
    const int lane = threadIdx.x & 31;
    unsigned off = 0u;
    if (lane == 0) off = atomicAdd(counter, (unsigned)__popc(ball));
    off = __shfl_sync(0xffffffffu, off, 0);
    const unsigned pos = off + (unsigned)__popc(ball & ((1u << lane) - 1u));
    if (take && pos < cap) out[pos] = k;
  }
}

// The digit whose cumulative range in S->hist holds `rank`, and the rank
// within it (S->digit, S->rank; the histogram is left intact).
__device__ __forceinline__ void find_digit(SelScratch* S, unsigned rank) {
  const int tid = threadIdx.x;
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
}

// Exact radix selection (digits of 11, 11 and 10 bits, counted in a shared
// histogram with warp-aggregated additions) of order statistic `rank` among
// the m keys of src (all below kNone). With want_next, *next is the key of
// order statistic rank + 1 of src, or kNone when rank is its last. All
// threads of the block call it.
__device__ unsigned select_keys(const unsigned* src, int m, unsigned rank, SelScratch* S, bool want_next,
                                unsigned* next) {
  const int tid = threadIdx.x, lane = tid & 31;
  unsigned prefix = 0u, pmask = 0u;
  for (int round = 0; round < 3; ++round) {
    const int shift = round == 0 ? 21 : (round == 1 ? 10 : 0);
    const unsigned dmask = round == 2 ? 0x3ffu : 0x7ffu;
    for (int i = tid; i < kBins; i += kThreads) S->hist[i] = 0u;
    __syncthreads();
    for (int base = tid - lane; base < m; base += kThreads) {
      const int e = base + lane;
      const unsigned k = e < m ? src[e] : kNone;
      hist_add_warp(S->hist, (e < m && (k & pmask) == prefix) ? (k >> shift) & dmask : (unsigned)kBins);
    }
    __syncthreads();
    find_digit(S, rank);
    const unsigned d = S->digit;
    rank = S->rank;
    prefix |= d << shift;
    pmask |= dmask << shift;
    if (round == 2 && want_next) {
      // the successor: the same key if it occurs again, else the next
      // non-empty bin of this round, else the smallest larger key of src
      if (tid == 0) S->next = (rank + 1u < S->hist[d]) ? prefix : kNone;
      __syncthreads();
      if (S->next == kNone) {
        for (int i = (int)d + 1 + tid; i < 1024; i += kThreads)
          if (S->hist[i] != 0u) atomicMin(&S->next, (prefix & ~dmask) | (unsigned)i);
        __syncthreads();
        if (S->next == kNone) {
          for (int e = tid; e < m; e += kThreads) {
            const unsigned k = src[e];
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

constexpr int kSampleStride = 8;  // every 8th voxel of the window is sampled for the bracket

// Order statistics r and (with want_next) r + 1 of key_of(k) over the finite
// keys k of keys[0 .. n) (nf of them). A sample of the window brackets the
// rank: the keys inside the bracket are copied into cand in one counting
// pass and selected there; when the bracket misses (or overflows cand), or
// the window is small, the selection runs over all keys. When `rewrite`, the
// keys are replaced by key_of(k) if the full selection is needed (the caller
// needs them no more).
template <class KeyOf>
__device__ bool select_order(unsigned* keys, int n, unsigned nf, unsigned r, bool want_next, KeyOf key_of,
                             bool rewrite, unsigned* cand, SelScratch* S, unsigned* k1, unsigned* k2) {
  const int tid = threadIdx.x, lane = tid & 31;
  unsigned nx = kNone;
  if (nf <= (unsigned)kCandCap) {  // small window: select over a copy of all finite keys
    if (tid == 0) S->count = 0u;
    __syncthreads();
    for (int base = tid - lane; base < n; base += kThreads) {
      const int e = base + lane;
      const unsigned k = e < n ? keys[e] : kNone;
      append_warp(k != kNone, k != kNone ? key_of(k) : kNone, cand, kCandCap, &S->count);
    }
    __syncthreads();
    *k1 = select_keys(cand, (int)nf, r, S, want_next, &nx);
    *k2 = nx;
    __syncthreads();
    return false;  // the keys are as they were
  }
  // sample every kSampleStride-th voxel
  if (tid == 0) S->count = 0u;
  __syncthreads();
  for (int j0 = tid - lane; j0 * kSampleStride < n; j0 += kThreads) {
    const int e = (j0 + lane) * kSampleStride;
    const unsigned k = e < n ? keys[e] : kNone;
    append_warp(k != kNone, k != kNone ? key_of(k) : kNone, cand, kCandCap, &S->count);
  }
  __syncthreads();
  const unsigned s = min(S->count, (unsigned)kCandCap);
  bool done = false;
  if (s >= 64u) {
    // sample ranks around the expected one, 4 binomial standard deviations
    // wide, widened to whole top-11-bit bins of one histogram of the sample
    const unsigned p = (unsigned)(((unsigned long long)r * s) / nf);
    const unsigned delta = 2u * (unsigned)sqrtf((float)s) + 4u;
    const unsigned rlo = p > delta ? p - delta : 0u, rhi = min(p + delta, s - 1u);
    for (int i = tid; i < kBins; i += kThreads) S->hist[i] = 0u;
    __syncthreads();
    for (int base = tid - lane; base < (int)s; base += kThreads) {
      const int e = base + lane;
      hist_add_warp(S->hist, e < (int)s ? cand[e] >> 21 : (unsigned)kBins);
    }
    __syncthreads();
    find_digit(S, rlo);
    const unsigned lo = S->digit << 21;
    find_digit(S, rhi);
    const unsigned hi = (S->digit << 21) | 0x1fffffu;
    // one counting pass: keys below the bracket, keys inside it into cand
    if (tid == 0) {
      S->count = 0u;
      S->below = 0u;
    }
    __syncthreads();
    unsigned below = 0u;
    for (int base = tid - lane; base < n; base += kThreads) {
      const int e = base + lane;
      const unsigned k = e < n ? keys[e] : kNone;
      const unsigned a = k != kNone ? key_of(k) : kNone;
      below += (a < lo) ? 1u : 0u;
      append_warp(a != kNone && a >= lo && a <= hi, a, cand, kCandCap, &S->count);
    }
    below = __reduce_add_sync(0xffffffffu, below);
    if (lane == 0) atomicAdd(&S->below, below);
    __syncthreads();
    const unsigned c_lo = S->below, cnt = S->count;
    if (cnt <= (unsigned)kCandCap && r >= c_lo && r < c_lo + cnt) {
      *k1 = select_keys(cand, (int)cnt, r - c_lo, S, want_next, &nx);
      if (want_next && nx == kNone) {
        // order statistic r + 1 lies above the bracket: the smallest key above it
        if (tid == 0) S->next = kNone;
        __syncthreads();
        for (int e = tid; e < n; e += kThreads) {
          const unsigned k = keys[e];
          if (k != kNone) {
            const unsigned a = key_of(k);
            if (a > hi) atomicMin(&S->next, a);
          }
        }
        __syncthreads();
        nx = S->next;
      }
      *k2 = nx;
      done = true;
    }
    __syncthreads();
  }
  if (!done) {  // the whole window (rare for noise-like data)
    if (rewrite) {
      for (int e = tid; e < n; e += kThreads)
        if (keys[e] != kNone) keys[e] = key_of(keys[e]);
      __syncthreads();
    }
    // select_keys needs keys below kNone only: count the kNone slots out by
    // giving the selection all n slots (they sort last) and the same rank
    *k1 = select_keys(keys, n, r, S, want_next, &nx);
    *k2 = nx;
  }
  __syncthreads();
  return !done && rewrite;  // keys[] now holds key_of of the original keys
}

__device__ __forceinline__ double key_value(unsigned k) { return (double)fkey_inv(k); }

// *s + *c += x with Neumaier's compensation (the running error of the float
// sum is kept in *c).
__device__ __forceinline__ void neumaier_add(float* s, float* c, float x) {
  const float t = __fadd_rn(*s, x);
  const float e = fabsf(*s) >= fabsf(x) ? __fadd_rn(__fsub_rn(*s, t), x) : __fadd_rn(__fsub_rn(x, t), *s);
  *c = __fadd_rn(*c, e);
  *s = t;
}

// x - b exactly as s + err (Knuth's TwoSum, round-to-nearest float ops).
__device__ __forceinline__ float two_diff(float x, float b, float* err) {
  const float s = __fsub_rn(x, b);
  const float bb = __fsub_rn(s, x);
  *err = __fadd_rn(__fsub_rn(x, __fsub_rn(s, bb)), __fsub_rn(-b, bb));
  return s;
}

// The MAD key of x: the float of |x - m| with m = (a + b) / 2 (a == b for an
// odd count: one correctly rounded subtraction). For an even count, x - a/2
// and then - b/2 are taken exactly as sums of two floats and added back, which
// rounds the exact difference faithfully (within one unit in the last place)
// in single precision, without the slow FP64 pipe.
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
  return __float_as_uint(fabsf(d)) | 0x80000000u;  // fkey of a non-negative float
}

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
    k_noise_window(const float* __restrict__ cube, nscale::Geo g, int mode, double* __restrict__ sig_out,
                   float* __restrict__ rinv_out) {
  using namespace nscale;
  const bool std_mode = mode == SC_NOISE_STD;
  extern __shared__ __align__(16) unsigned char ns_smem[];
  unsigned* const cand = reinterpret_cast<unsigned*>(ns_smem);  // [kCandCap]
  unsigned* const keys = cand + kCandCap;                          // [window voxels]
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
    // Median bracket (MAD mode, windows larger than the copy-aside buffer): a
    // sample of every kSampleStride-th voxel, read straight from the cube,
    // and its top-11-bit histogram give key bounds [lo, hi] around the middle
    // rank, so that the load pass below can count the keys under lo and copy
    // those inside into cand.
    bool med_bracket = !std_mode && n > kCandCap;
    unsigned lo = 0u, hi = kNone - 1u;
    if (med_bracket) {
      if (tid == 0) S.count = 0u;
      __syncthreads();
      const int lxy = lx * ly;
      for (int j0 = tid - lane; j0 * kSampleStride < n; j0 += kThreads) {
        const int e = (j0 + lane) * kSampleStride;
        unsigned k = kNone;
        if (e < n) {
          const int dz = e / lxy, rem = e - dz * lxy, dy = rem / lx, dx = rem - dy * lx;
          const float v = __ldg(cube + (z0 + dz) * plane + (y0 + dy) * g.nx + x0 + dx);
          if (isfinite(v)) k = fkey(v);
        }
        append_warp(k != kNone, k, cand, kCandCap, &S.count);
      }
      __syncthreads();
      const unsigned ns = min(S.count, (unsigned)kCandCap);
      med_bracket = ns >= 64u;
      if (med_bracket) {
        const unsigned p = (ns - 1u) / 2u;
        const unsigned delta = 2u * (unsigned)sqrtf((float)ns) + 4u;
        for (int i = tid; i < kBins; i += kThreads) S.hist[i] = 0u;
        __syncthreads();
        for (int base = tid - lane; base < (int)ns; base += kThreads) {
          const int e = base + lane;
          hist_add_warp(S.hist, e < (int)ns ? cand[e] >> 21 : (unsigned)kBins);
        }
        __syncthreads();
        find_digit(&S, p > delta ? p - delta : 0u);
        lo = S.digit << 21;
        find_digit(&S, min(p + delta, ns - 1u));
        hi = (S.digit << 21) | 0x1fffffu;
      }
      if (tid == 0) {
        S.count = 0u;
        S.below = 0u;
      }
    }
    __syncthreads();
    // the window's keys: warps over rows, four planes' loads issued together;
    // with a bracket, also the keys under it counted and those in it copied
    unsigned finite = 0u, below = 0u;
    constexpr int kPlanesAtOnce = 4;
    for (int dz0 = 0; dz0 < lz; dz0 += kPlanesAtOnce) {
      for (int dy = warp; dy < ly; dy += kWarps) {
        for (int dx0 = 0; dx0 < lx; dx0 += 32) {
          const int dx = dx0 + lane;
          float v[kPlanesAtOnce];
#pragma unroll
          for (int u = 0; u < kPlanesAtOnce; ++u)
            v[u] = (dz0 + u < lz && dx < lx) ? __ldg(cube + (z0 + dz0 + u) * plane + (y0 + dy) * g.nx + x0 + dx)
                                             : __int_as_float(0x7fc00000);
#pragma unroll
          for (int u = 0; u < kPlanesAtOnce; ++u) {
            const bool ok = isfinite(v[u]);
            const unsigned k = ok ? fkey(v[u]) : kNone;
            if (dz0 + u < lz && dx < lx) keys[((dz0 + u) * ly + dy) * lx + dx] = k;
            finite += ok ? 1u : 0u;
            if (med_bracket) {
              below += (ok && k < lo) ? 1u : 0u;
              append_warp(ok && k >= lo && k <= hi, k, cand, kCandCap, &S.count);
            }
          }
        }
      }
    }
    finite = __reduce_add_sync(0xffffffffu, finite);
    below = __reduce_add_sync(0xffffffffu, below);
    if (lane == 0) {
      atomicAdd(&s_count, finite);
      if (med_bracket) atomicAdd(&S.below, below);
    }
    __syncthreads();
    const unsigned nf = s_count;
    double sigma;
    if (nf == 0u) {
      sigma = __longlong_as_double(0x7ff8000000000000LL);  // NaN: no finite voxel
    } else if (std_mode) {
      // float32 sums with Neumaier compensation per thread (the FP64 pipe is
      // slow on this part), combined in double across the block
      float s = 0.0f, sc = 0.0f;
      for (int e = tid; e < n; e += kThreads)
        if (keys[e] != kNone) neumaier_add(&s, &sc, fkey_inv(keys[e]));
      const double mean = block_sum_d((double)s + (double)sc, dpart) / (double)nf;
      const float mh = __double2float_rn(mean), ml = __double2float_rn(mean - (double)mh);
      float q = 0.0f, qc = 0.0f;
      for (int e = tid; e < n; e += kThreads)
        if (keys[e] != kNone) {
          const float d = __fsub_rn(__fsub_rn(fkey_inv(keys[e]), mh), ml);
          neumaier_add(&q, &qc, __fmul_rn(d, d));
        }
      const double qq = block_sum_d((double)q + (double)qc, dpart);
      sigma = nf > 1u ? sqrt(qq / (double)(nf - 1u)) : 0.0;
    } else {
      // median: order statistics (nf - 1) / 2 and nf / 2
      const unsigned r1 = (nf - 1u) / 2u;
      const bool even = (nf & 1u) == 0u;
      unsigned k1 = 0u, k2 = 0u;
      const unsigned c_lo = S.below, cnt = S.count;
      if (med_bracket && cnt <= (unsigned)kCandCap && r1 >= c_lo && r1 < c_lo + cnt) {
        unsigned nx = kNone;
        k1 = select_keys(cand, (int)cnt, r1 - c_lo, &S, even, &nx);
        if (even && nx == kNone) {  // the next order statistic lies above the bracket
          if (tid == 0) S.next = kNone;
          __syncthreads();
          for (int e = tid; e < n; e += kThreads) {
            const unsigned k = keys[e];
            if (k != kNone && k > hi) atomicMin(&S.next, k);
          }
          __syncthreads();
          nx = S.next;
        }
        k2 = nx;
        __syncthreads();
      } else {
        select_order(keys, n, nf, r1, even, [](unsigned k) { return k; }, false, cand, &S, &k1, &k2);
      }
      // MAD: the same order statistics of |x - m|, m = (k1 + k2) / 2, as
      // float32 keys computed on the fly
      const float ma = fkey_inv(k1), mb = even ? fkey_inv(k2) : ma;
      unsigned a1 = 0u, a2 = 0u;
      const bool rewrote =
          select_order(keys, n, nf, r1, even, [=](unsigned k) { return mad_key(fkey_inv(k), ma, mb, even); }, true,
                       cand, &S, &a1, &a2);
      const double mad = even ? 0.5 * (key_value(a1) + key_value(a2)) : key_value(a1);
      sigma = kMadToSigma * mad;
      if (mode == SC_NOISE_GAUSS && sigma > 0.0) {
        // the window's 256-bin histogram (from the keys in shared memory, or
        // read again from the cube where the selection rewrote them), then a
        // one-warp fit; the MAD noise stands without a root
        const float k = gfit::scale_of(sigma);
        __syncthreads();  // the selection is done with S.hist
        for (int i = tid; i < gfit::kBins; i += kThreads) S.hist[i] = 0u;
        __syncthreads();
        if (!rewrote) {
          for (int e = tid; e < n; e += kThreads) {
            const unsigned key = keys[e];
            const int b = key != kNone ? gfit::bin_of(fkey_inv(key), k) : -1;
            if (b >= 0) atomicAdd(&S.hist[b], 1u);
          }
        } else {
          for (int dz = 0; dz < lz; ++dz)
            for (int dy = warp; dy < ly; dy += kWarps)
              for (int dx = lane; dx < lx; dx += 32) {
                const int b = gfit::bin_of(__ldg(cube + (z0 + dz) * plane + (y0 + dy) * g.nx + x0 + dx), k);
                if (b >= 0) atomicAdd(&S.hist[b], 1u);
              }
        }
        __syncthreads();
        if (warp == 0) {
          double hh[4], x2[4];
          bool use[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int t = lane + 32 * j;
            hh[j] = (double)S.hist[gfit::kHalf + t] + (double)S.hist[gfit::kHalf - 1 - t];
            x2[j] = gfit::xi2_of(t);
            use[j] = true;
          }
          const double tau = gfit::fit_tau(hh, x2, use, gfit::WarpSum6{});
          if (lane == 0) dpart[0] = tau;
        }
        __syncthreads();
        const double tau = dpart[0];
        if (tau > 0.0) sigma = gfit::noise_of(tau, k);
      }
    }
    if (tid == 0) {
      sig_out[cell] = sigma;
      rinv_out[cell] = sigma > 0.0 ? __double2float_rn(1.0 / sigma) : __int_as_float(0x7fc00000);
    }
    __syncthreads();  // the keys are overwritten by the next cell
  }
}

// One warp per (y, z) row; four voxels per lane step when the rows allow
// 16-byte accesses.
__global__ void __launch_bounds__(256) k_noise_apply(const float* in, float* out, nscale::Geo g,
                                                     const float* __restrict__ rinv, int vec) {
  const int lane = threadIdx.x & 31;
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  const long long rows = g.ny * g.nz;
  const float qnan = __int_as_float(0x7fc00000);
  for (long long row = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); row < rows; row += warps) {
    const long long z = row / g.ny, y = row - z * g.ny;
    const float* rr = rinv + ((z / g.gz) * g.ncy + y / g.gy) * (long long)g.ncx;
    const float* src = in + row * g.nx;
    float* dst = out + row * g.nx;
    if (vec) {
      const int nq = (int)(g.nx >> 2);
      for (int q = lane; q < nq; q += 32) {
        const int x = 4 * q;
        int c = x / g.gx, r = x - c * g.gx;  // cell and position in it of voxel x
        const float4 v = reinterpret_cast<const float4*>(src)[q];
        float o[4];
        const float vin[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          o[k] = isfinite(vin[k]) ? __fmul_rn(vin[k], __ldg(rr + c)) : qnan;
          if (++r == g.gx) {
            ++c;
            r = 0;
          }
        }
        reinterpret_cast<float4*>(dst)[q] = make_float4(o[0], o[1], o[2], o[3]);
      }
    } else {
      for (int x = lane; x < g.nx; x += 32) {
        const float v = src[x];
        dst[x] = isfinite(v) ? __fmul_rn(v, __ldg(rr + x / g.gx)) : qnan;
      }
    }
  }
}

size_t noise_window_smem(long long window_voxels) {
  return sizeof(unsigned) * ((size_t)nscale::kCandCap + (size_t)window_voxels);
}

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
                                int noise_mode, double* sig_dev, float* rinv_dev, int sms, cudaStream_t s) {
  const nscale::Geo g = make_geo(dims, window, grid);
  const long long cells = (long long)g.ncx * g.ncy * g.ncz;
  const long long wvox = (long long)min((long long)g.wx, g.nx) * min((long long)g.wy, g.ny) * min((long long)g.wz, g.nz);
  const int blocks = (int)(cells < sms ? cells : sms);
  k_noise_window<<<blocks, nscale::kThreads, noise_window_smem(wvox), s>>>(cube, g, noise_mode, sig_dev, rinv_dev);
  return cudaGetLastError();
}

cudaError_t launch_noise_apply(const float* cube, const long long dims[3], const int window[3], const int grid[3],
                               float* out, const float* rinv_dev, int sms, cudaStream_t s) {
  const nscale::Geo g = make_geo(dims, window, grid);
  const long long rows = g.ny * g.nz;
  const long long want = (rows + 7) / 8;  // eight warps (rows) per block
  const int blocks = (int)(want < 16LL * sms ? want : 16LL * sms);
  const int vec = (g.nx % 4 == 0) && (reinterpret_cast<uintptr_t>(cube) & 15u) == 0 &&
                  (reinterpret_cast<uintptr_t>(out) & 15u) == 0;
  k_noise_apply<<<blocks, 256, 0, s>>>(cube, out, g, rinv_dev, vec);
  return cudaGetLastError();
}

void init_noise_scale_attrs() {
  cudaFuncSetAttribute(k_noise_window, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)noise_window_smem(kNoiseScaleMaxWindow));
}

}  // namespace sc
