// Robust noise measurement and clipping (SoFiA 2, Sect. 4.1 and 4.2).
//
// sigma = 1.4826 * median(|S - median(S)|) over the finite voxels, with both
// medians exact order statistics of the float32 values (mean of the two
// middle ones for an even count), then mask |= |S| > t * sigma.
//
// Data flow for one measurement over an array S of n values:
//   k_hist      (or the smoothing kernel's epilogue): histogram of S over
//               bins of the float bits (monotone in the value).
//   k_plan      one block: ranks of the middle order statistics -> the bins
//               holding the median; from the bin counts alone, thresholds
//               T1 < MAD < T2 and the value windows that can hold the MAD's
//               elements; bounds on t*sigma for the clip; capacity checks.
//   k_pass2     one read of S: collects median candidates (values in the
//               median bins), MAD candidates (values not surely inside or
//               outside the MAD band), counts values surely inside the band,
//               sets the mask bits that are certain whatever sigma is inside
//               its bounds, and lists the few voxels whose clip is not yet
//               decided.
//   k_sel_*     exact radix selection (11+11+10 bits) of the wanted order
//               statistics inside the candidate lists, then of |s - m|.
//   k_resolve   decides the listed voxels with the exact sigma.
// When a candidate set would exceed its buffer, the plan switches that part
// to full passes over S (k_sel_* on the whole array, k_clip_full); results are
// identical, only slower.
#include <atomic>
#include <cfloat>
#include <cstdio>

#include "sc_device.cuh"
#include "sc_internal.h"

namespace sc {

constexpr double kMadToSigma = 1.4826;

// sigma from the MAD, rounded once to float. Monotone in mad, so the plan's
// bounds on the MAD give bounds on sigma through the same function.
__device__ __forceinline__ float sigma_of_mad(double mad) { return __double2float_rn(kMadToSigma * mad); }

// ---------------------------------------------------------------------------
// Histogram (and max |x|) of the finite values of an array.
__global__ void __launch_bounds__(512) k_hist(const float* __restrict__ x, long long n, DevState* st,
                                              unsigned long long* __restrict__ hist, int win, int want_maxabs) {
  extern __shared__ unsigned int sh[];
  for (int i = threadIdx.x; i < kNumBins; i += blockDim.x) sh[i] = 0u;
  __syncthreads();
  const BinCfg cfg = win ? st->win : kFullRange;
  unsigned int mx = 0u;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const bool vec = ((reinterpret_cast<uintptr_t>(x) & 15u) == 0);
  if (vec) {
    const long long n4 = n >> 2;
    const float4* x4 = reinterpret_cast<const float4*>(x);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
      float4 v = __ldg(x4 + i);
      float a[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        if (isfinite(a[c])) {
          atomicAdd(&sh[bin_of(a[c], cfg)], 1u);
          mx = max(mx, __float_as_uint(fabsf(a[c])));
        }
      }
    }
    for (long long i = (n4 << 2) + (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
      float a = __ldg(x + i);
      if (isfinite(a)) {
        atomicAdd(&sh[bin_of(a, cfg)], 1u);
        mx = max(mx, __float_as_uint(fabsf(a)));
      }
    }
  } else {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
      float a = __ldg(x + i);
      if (isfinite(a)) {
        atomicAdd(&sh[bin_of(a, cfg)], 1u);
        mx = max(mx, __float_as_uint(fabsf(a)));
      }
    }
  }
  if (want_maxabs) {
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0 && mx) atomicMax(&st->maxabs_bits, mx);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kNumBins; i += blockDim.x)
    if (sh[i]) atomicAdd(hist + i, (unsigned long long)sh[i]);
}

cudaError_t launch_hist(const float* x, long long n, DevState* st, unsigned long long* hist, int win,
                        int want_maxabs, int sms, cudaStream_t s) {
  const size_t smem = kNumBins * sizeof(unsigned int);
  long long want = (n / 4 + 511) / 512;
  int grid = (int)(want < 1 ? 1 : (want > 4LL * sms ? 4LL * sms : want));
  k_hist<<<grid, 512, smem, s>>>(x, n, st, hist, win, want_maxabs);
  return cudaGetLastError();
}

// The same histogram (and max |value|) of a 16-bit cube, whose planes hold a
// multiple of 8 values: a thread takes 8 values (16 bytes) at a time and
// decodes them with their plane's scale (the plane followed along the
// grid-stride loop). With out != null the decoded float32 values are written
// there as well (the cube for the passes that read it as float32).
__global__ void __launch_bounds__(512) k_hist16(Half16 h, long long plane, long long n, DevState* st,
                                                unsigned long long* __restrict__ hist, int win, int want_maxabs,
                                                float* __restrict__ out) {
  extern __shared__ unsigned int sh[];
  for (int i = threadIdx.x; i < kNumBins; i += blockDim.x) sh[i] = 0u;
  __syncthreads();
  const BinCfg cfg = win ? st->win : kFullRange;
  unsigned int mx = 0u;
  const long long ng = n / 8, pg = plane / 8;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long dz = stride / pg, doff = stride - dz * pg;
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long z = g / pg, off = g - z * pg;
  const uint4* b4 = reinterpret_cast<const uint4*>(h.bits);
  for (; g < ng; g += stride) {
    const uint4 q = __ldg(b4 + g);
    const float cs = __ldg(h.scale + z);
    const unsigned w[4] = {q.x, q.y, q.z, q.w};
    float v[8];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      v[2 * k] = half16_value((unsigned short)(w[k] & 0xffffu), h.fmt, cs);
      v[2 * k + 1] = half16_value((unsigned short)(w[k] >> 16), h.fmt, cs);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      if (isfinite(v[i])) {
        atomicAdd(&sh[bin_of(v[i], cfg)], 1u);
        mx = max(mx, __float_as_uint(fabsf(v[i])));
      }
    }
    if (out) {
      float4* o4 = reinterpret_cast<float4*>(out) + 2 * g;
      o4[0] = make_float4(v[0], v[1], v[2], v[3]);
      o4[1] = make_float4(v[4], v[5], v[6], v[7]);
    }
    z += dz;
    off += doff;
    if (off >= pg) {
      off -= pg;
      ++z;
    }
  }
  if (want_maxabs) {
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0 && mx) atomicMax(&st->maxabs_bits, mx);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kNumBins; i += blockDim.x)
    if (sh[i]) atomicAdd(hist + i, (unsigned long long)sh[i]);
}

cudaError_t launch_hist16(const Half16& h, long long plane, long long n, DevState* st, unsigned long long* hist,
                          int win, int want_maxabs, float* out, int sms, cudaStream_t s) {
  if (plane % 8 != 0 || (reinterpret_cast<uintptr_t>(h.bits) & 15u) != 0 ||
      (out && (reinterpret_cast<uintptr_t>(out) & 15u) != 0))
    return cudaErrorInvalidValue;  // the caller takes the 16-bit path only for such cubes
  const size_t smem = kNumBins * sizeof(unsigned int);
  long long want = (n / 8 + 511) / 512;
  int grid = (int)(want < 1 ? 1 : (want > 4LL * sms ? 4LL * sms : want));
  k_hist16<<<grid, 512, smem, s>>>(h, plane, n, st, hist, win, want_maxabs, out);
  return cudaGetLastError();
}

// Max |x| over finite values only (for sc_smooth's fixed-point scale).
__global__ void k_maxabs(const float* __restrict__ x, long long n, DevState* st) {
  unsigned int mx = 0u;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    float a = __ldg(x + i);
    if (isfinite(a)) mx = max(mx, __float_as_uint(fabsf(a)));
  }
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0 && mx) atomicMax(&st->maxabs_bits, mx);
}

cudaError_t launch_maxabs(const float* x, long long n, DevState* st, int sms, cudaStream_t s) {
  long long want = (n + 255) / 256;
  int grid = (int)(want < 1 ? 1 : (want > 8LL * sms ? 8LL * sms : want));
  k_maxabs<<<grid, 256, 0, s>>>(x, n, st);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Plan: one block of 1024 threads.
struct PlanCtx {
  const unsigned long long* cum;  // exclusive prefix counts, kNumBins + 1 entries
  BinCfg cfg;
  double m_min, m_max;
};

__device__ __forceinline__ unsigned long long cum_range(const PlanCtx& P, int b1, int b2) {
  // count of values in bins b1..b2 inclusive (0 if empty range)
  if (b2 < b1) return 0ull;
  return P.cum[b2 + 1] - P.cum[b1];
}
__device__ __forceinline__ float f_down(double v) { return nextafterf(__double2float_rd(v), -INFINITY); }
__device__ __forceinline__ float f_up(double v) { return nextafterf(__double2float_ru(v), INFINITY); }

// Values that can possibly lie within T of some m in [m_min, m_max].
__device__ unsigned long long f_possible(const PlanCtx& P, float T) {
  float lo = f_down(P.m_min - (double)T), hi = f_up(P.m_max + (double)T);
  return cum_range(P, bin_of(lo, P.cfg), bin_of(hi, P.cfg));
}
// Values that surely lie within T of every m in [m_min, m_max] (whole bins
// strictly inside [m_max - T, m_min + T]).
__device__ unsigned long long f_sure(const PlanCtx& P, float T) {
  float lo = f_up(P.m_max - (double)T), hi = f_down(P.m_min + (double)T);
  if (!(lo <= hi)) return 0ull;
  return cum_range(P, bin_of(lo, P.cfg) + 1, bin_of(hi, P.cfg) - 1);
}

// Class of a 16-bit cell of the float encoding (sign, 8 exponent bits, top
// 7 mantissa bits). Every histogram bin is a union of whole cells (bins
// resolve at most 7 mantissa bits), so the median and MAD classes are exact
// functions of the cell. CLS_SURE marks cells wholly above thr_hi in |s| (all
// their values are detected whatever sigma is); CLS_AMB marks cells that
// overlap (thr_lo, thr_hi] and is refined per value by the candidate pass.
constexpr int kClsCells = (int)kClassTableBytes;
enum : unsigned int { CLS_MED = 1u, CLS_MAD = 2u, CLS_AMB = 4u, CLS_SURE = 8u };

__device__ __forceinline__ unsigned int cell_class(unsigned int cell, const NoisePlan& p, BinCfg cfg, bool med,
                                                   bool mad, bool amb) {
  const unsigned int u = cell << 16;
  if (((u >> 23) & 0xffu) == 0xffu) return 0u;  // Inf and NaN are never candidates
  const int b = bin_of_bits(u, cfg);
  unsigned int k = 0u;
  if (med && b >= p.b_med_lo && b <= p.b_med_hi) k |= CLS_MED;
  if (mad && b >= p.bA_lo && b <= p.bA_hi && !(b >= p.bB_lo && b <= p.bB_hi)) k |= CLS_MAD;
  if (amb) {
    const float lo = fabsf(__uint_as_float(u)), hi = fabsf(__uint_as_float(u | 0xffffu));
    if (hi > p.thr_lo && lo <= p.thr_hi) k |= CLS_AMB;
    if (lo > p.thr_hi) k |= CLS_SURE;
  }
  return k;
}

// All threads of the block write the 64 KiB class table (one byte per cell).
__device__ void fill_class_table(const NoisePlan& p, BinCfg cfg, unsigned char* cls) {
  const bool live = !(p.flags & (PLAN_EMPTY | PLAN_STD));
  const bool med = live && !(p.flags & PLAN_MED_FULL);
  const bool mad = live && !(p.flags & PLAN_MAD_FULL);
  const bool amb = live && (p.flags & PLAN_CLIP) && !(p.flags & PLAN_CLIP_FULL);
  for (int i = threadIdx.x; i < kClsCells / 16; i += blockDim.x) {
    unsigned int w[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      unsigned int x = 0u;
#pragma unroll
      for (int b = 0; b < 4; ++b) x |= cell_class((unsigned)(i * 16 + j * 4 + b), p, cfg, med, mad, amb) << (8 * b);
      w[j] = x;
    }
    reinterpret_cast<uint4*>(cls)[i] = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

__device__ __noinline__ NoisePlan plan_of(DevState* st, const unsigned long long* cum, int win, const float* src,
                                          long long n_total, Lists L, float threshold, int clip, int std_mode,
                                          unsigned int force_flags);

__global__ void __launch_bounds__(1024) k_plan(DevState* st, const unsigned long long* __restrict__ hist, int win,
                                               const float* src, long long n_total, Lists L, float threshold,
                                               int clip, int std_mode, unsigned int force_flags) {
  extern __shared__ unsigned long long cum[];  // kNumBins + 1
  __shared__ unsigned long long wsum[32];
  const int tid = threadIdx.x;
  constexpr int kPer = (kNumBins + 1023) / 1024;
  unsigned long long loc[kPer];
  unsigned long long s = 0;
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    int b = tid * kPer + j;
    loc[j] = b < kNumBins ? hist[b] : 0ull;
    s += loc[j];
  }
  // block exclusive scan of s
  unsigned long long incl = s;
  for (int o = 1; o < 32; o <<= 1) {
    unsigned long long t = __shfl_up_sync(0xffffffffu, incl, o);
    if ((tid & 31) >= o) incl += t;
  }
  if ((tid & 31) == 31) wsum[tid >> 5] = incl;
  __syncthreads();
  if (tid < 32) {
    unsigned long long w = wsum[tid], wi = w;
    for (int o = 1; o < 32; o <<= 1) {
      unsigned long long t = __shfl_up_sync(0xffffffffu, wi, o);
      if (tid >= o) wi += t;
    }
    wsum[tid] = wi - w;
  }
  __syncthreads();
  unsigned long long run = wsum[tid >> 5] + incl - s;
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    int b = tid * kPer + j;
    if (b < kNumBins) cum[b] = run;
    run += loc[j];
  }
  if (tid == 1023) cum[kNumBins] = run;
  // reset counters and selection state
  for (int i = tid; i < 3 * kSelBins; i += blockDim.x) {
    (&st->sel_med.hist[0][0])[i] = 0ull;
    (&st->sel_mad.hist[0][0])[i] = 0ull;
  }
  __syncthreads();
  __shared__ NoisePlan s_plan;
  if (tid == 0) s_plan = plan_of(st, cum, win, src, n_total, L, threshold, clip, std_mode, force_flags);
  __syncthreads();
  if (L.cls != nullptr) {
    BinCfg cfg = kFullRange;
    if (win) cfg = st->win;
    fill_class_table(s_plan, cfg, L.cls);
  }
}

// The plan proper (one thread). Returns the plan it stored in st->plan.
__device__ __noinline__ NoisePlan plan_of(DevState* st, const unsigned long long* cum, int win, const float* src,
                                          long long n_total, Lists L, float threshold, int clip, int std_mode,
                                          unsigned int force_flags) {
  NoisePlan p;
  p.flags = (int)force_flags;
  p.threshold = threshold;
  p.has_B = 0;
  p.B_lo = 1.0f;
  p.B_hi = 0.0f;
  p.A_lo = -INFINITY;
  p.A_hi = INFINITY;
  p.thr_lo = 0.0f;
  p.thr_hi = INFINITY;
  p.T1 = 0.0f;
  p.T2 = INFINITY;
  p.bound_med = p.bound_mad = p.bound_amb = 0ull;
  p.bA_lo = 0;
  p.bA_hi = kNumBins - 1;
  p.bB_lo = 1;
  p.bB_hi = 0;
  p.n_B = 0ull;
  const unsigned long long n = cum[kNumBins];
  p.n = n;
  st->n_cand_med = st->n_cand_mad = st->n_amb = st->n_below = 0ull;
  st->sum = st->sum2 = 0.0;
  st->count = 0ull;
  if (clip) p.flags |= PLAN_CLIP;
  if (std_mode) p.flags |= PLAN_STD | PLAN_CLIP_FULL;
  SelJob* J[2] = {&st->sel_med, &st->sel_mad};
  for (int w = 0; w < 2; ++w) {
    J[w]->c_le = 0ull;
    J[w]->min_gt = 0xffffffffu;
    J[w]->key_lo = 0u;
    J[w]->count_fixed = 0ull;
    J[w]->count_ptr = nullptr;
    J[w]->list = src;
    J[w]->rank_lo = J[w]->rank_hi = 0ull;
  }
  if (n == 0ull) {
    p.flags |= PLAN_EMPTY;
    st->status |= SC_ST_ALLNAN;
    st->plan = p;
    return p;
  }
  p.k_lo = (n - 1ull) / 2ull;
  p.k_hi = n / 2ull;
  // bins of the two middle order statistics
  int lo = 0, hi = kNumBins - 1;
  while (lo < hi) {  // first bin b with cum[b + 1] > k_lo
    int mid = (lo + hi) >> 1;
    if (cum[mid + 1] > p.k_lo) hi = mid; else lo = mid + 1;
  }
  p.b_med_lo = lo;
  hi = kNumBins - 1;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (cum[mid + 1] > p.k_hi) hi = mid; else lo = mid + 1;
  }
  p.b_med_hi = lo;
  p.below_med = cum[p.b_med_lo];
  p.bound_med = cum[p.b_med_hi + 1] - cum[p.b_med_lo];
  if (p.bound_med > L.cap.med) p.flags |= PLAN_MED_FULL;

  if (!std_mode) {
    const BinCfg cfg = win ? st->win : kFullRange;
    PlanCtx P{cum, cfg, bin_lo_value(p.b_med_lo, cfg), bin_hi_value(p.b_med_hi, cfg)};
    if (!(isfinite(P.m_min) && isfinite(P.m_max))) {
      p.flags |= PLAN_MAD_FULL | PLAN_CLIP_FULL;
    } else {
      // T1: largest T with possibly-within count <= k_lo (then MAD > T1)
      if (f_possible(P, 0.0f) <= p.k_lo) {
        unsigned int a = 0u, b = 0x7f800000u;
        while (b - a > 1u) {
          unsigned int mid = a + ((b - a) >> 1);
          if (f_possible(P, __uint_as_float(mid)) <= p.k_lo) a = mid; else b = mid;
        }
        p.T1 = __uint_as_float(a);
        p.has_B = 1;
        p.B_lo = f_up(P.m_max - (double)p.T1);
        p.B_hi = f_down(P.m_min + (double)p.T1);
        // B as whole bins strictly inside [B_lo, B_hi]: its count is exact
        // from the histogram, so the candidate pass need not count it.
        if (p.B_lo <= p.B_hi) {
          p.bB_lo = bin_of(p.B_lo, cfg) + 1;
          p.bB_hi = bin_of(p.B_hi, cfg) - 1;
        }
      }
      // T2: smallest T with surely-within count >= k_hi + 1 (then MAD < T2)
      const unsigned int fmax_bits = 0x7f7fffffu;
      if (f_sure(P, __uint_as_float(fmax_bits)) >= p.k_hi + 1ull) {
        unsigned int a = 0u, b = fmax_bits;
        while (b - a > 1u) {
          unsigned int mid = a + ((b - a) >> 1);
          if (f_sure(P, __uint_as_float(mid)) >= p.k_hi + 1ull) b = mid; else a = mid;
        }
        p.T2 = __uint_as_float(b);
        p.A_lo = f_down(P.m_min - (double)p.T2);
        p.A_hi = f_up(P.m_max + (double)p.T2);
      }
      // bound on the MAD candidates: values neither surely inside nor outside
      p.bA_lo = bin_of(p.A_lo, cfg);
      p.bA_hi = bin_of(p.A_hi, cfg);
      p.n_B = cum_range(P, p.bB_lo, p.bB_hi);  // B lies inside A: its values are within T1 < T2
      p.bound_mad = cum_range(P, p.bA_lo, p.bA_hi) - p.n_B;
      if (p.bound_mad > L.cap.mad) p.flags |= PLAN_MAD_FULL;
      if (clip) {
        if (!p.has_B || !(p.T1 > 0.0f) || !isfinite(p.T2)) {
          p.flags |= PLAN_CLIP_FULL;
        } else {
          const float s_lo = sigma_of_mad((double)p.T1), s_hi = sigma_of_mad((double)p.T2);
          p.thr_lo = __fmul_rn(threshold, s_lo);
          p.thr_hi = __fmul_rn(threshold, s_hi);
          p.bound_amb = cum_range(P, bin_of(-p.thr_hi, cfg), bin_of(-p.thr_lo, cfg)) +
                        cum_range(P, bin_of(p.thr_lo, cfg), bin_of(p.thr_hi, cfg));
          if (p.bound_amb > L.cap.amb) p.flags |= PLAN_CLIP_FULL;
        }
      }
    }
  }
  // selection jobs
  const bool med_full = (p.flags & PLAN_MED_FULL) != 0, mad_full = (p.flags & PLAN_MAD_FULL) != 0;
  st->sel_med.list = med_full ? src : L.med;
  st->sel_med.count_fixed = med_full ? (unsigned long long)n_total : L.cap.med;
  st->sel_med.count_ptr = med_full ? nullptr : &st->n_cand_med;
  st->sel_med.mode = SEL_VALUE;
  st->sel_med.rank_lo = med_full ? p.k_lo : p.k_lo - p.below_med;
  st->sel_med.rank_hi = st->sel_med.rank_lo + (p.k_hi - p.k_lo);
  st->sel_mad.list = mad_full ? src : L.mad;
  st->sel_mad.count_fixed = mad_full ? (unsigned long long)n_total : L.cap.mad;
  st->sel_mad.count_ptr = mad_full ? nullptr : &st->n_cand_mad;
  st->sel_mad.mode = SEL_ABSDEV;
  st->sel_mad.rank_lo = p.k_lo;  // minus n_below unless full
  st->sel_mad.rank_hi = p.k_hi;
  st->n_below = mad_full ? 0ull : p.n_B;
  st->plan = p;
  return p;
}

cudaError_t launch_plan(DevState* st, const unsigned long long* hist, int win, const float* src, long long n_total,
                        Lists L, float threshold, int clip, int std_mode, unsigned int force_flags,
                        cudaStream_t s) {
  const size_t smem = (kNumBins + 1) * sizeof(unsigned long long);
  k_plan<<<1, 1024, smem, s>>>(st, hist, win, src, n_total, L, threshold, clip, std_mode, force_flags);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Candidate pass. A warp takes chunks of 128 consecutive values; lane l reads
// values l, l + 32, l + 64 and l + 96 of a chunk, so one ballot per read is
// exactly one word of the bit mask. Each value costs a class-table lookup
// (shared memory), whose SURE bit feeds the mask ballot; the few values whose
// cell is a candidate cell take the slow path, which stages list entries in the warp's own
// shared-memory region and flushes them with one atomic per batch.
constexpr int kP2Threads = 512;
constexpr int kP2Warps = kP2Threads / 32;
constexpr int kP2Unroll = 2;                 // chunks a warp classifies per iteration (the next ones load meanwhile)
constexpr int kP2FlushAt = 64;               // flush a list holding more than this after a chunk
constexpr int kP2Stage = kP2FlushAt + 128;   // one chunk adds at most 128 entries per list
constexpr size_t kP2Smem =
    kClsCells + (size_t)kP2Warps * kP2Stage * (2 * sizeof(float) + sizeof(unsigned long long));

template <typename T>
__device__ __forceinline__ void stage_flush(T* stage, int& cnt, T* glob, unsigned long long* gcount,
                                            unsigned long long cap, unsigned int* status) {
  __syncwarp();
  const int lane = threadIdx.x & 31;
  unsigned long long base = 0;
  if (lane == 0 && cnt > 0) base = atomicAdd(gcount, (unsigned long long)cnt);
  base = __shfl_sync(0xffffffffu, base, 0);
  if (base + (unsigned long long)cnt > cap) {
    if (lane == 0) atomicOr(status, (unsigned int)SC_ST_OVERFLOW);
  } else {
    for (int i = lane; i < cnt; i += 32) glob[base + i] = stage[i];
  }
  __syncwarp();
  cnt = 0;
}

// Appends val from the lanes whose bit is set in b (the warp's ballot of pred).
template <typename T>
__device__ __forceinline__ void stage_push(unsigned int b, bool pred, unsigned int lanes_below, T val, T* stage,
                                           int& cnt) {
  if (pred) stage[cnt + __popc(b & lanes_below)] = val;
  cnt += __popc(b);
}

// Loads the kP2Unroll chunks of 128 values from chunk ch0 on; values past n
// read as NaN (class 0, never sure, never listed).
__device__ __forceinline__ void p2_load(const float* __restrict__ src, long long n, long long ch0, int lane,
                                        float (&a)[kP2Unroll][4]) {
  const float* base = src + ch0 * 128 + lane;
  if ((ch0 + kP2Unroll) * 128 <= n) {
#pragma unroll
    for (int u = 0; u < kP2Unroll; ++u)
#pragma unroll
      for (int c = 0; c < 4; ++c) a[u][c] = __ldg(base + 128 * u + 32 * c);
  } else {
#pragma unroll
    for (int u = 0; u < kP2Unroll; ++u)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const long long v = (ch0 + u) * 128 + 32 * c + lane;
        a[u][c] = v < n ? __ldg(src + v) : __int_as_float(0x7fc00000);
      }
  }
}

__global__ void __launch_bounds__(kP2Threads, 2) k_pass2(const float* __restrict__ src, long long n,
                                                         uint32_t* mbits, DevState* st, Lists L) {
  extern __shared__ __align__(16) unsigned char p2_smem[];
  const NoisePlan p = st->plan;
  if (p.flags & (PLAN_EMPTY | PLAN_STD)) return;
  const bool do_clip = (p.flags & PLAN_CLIP) && !(p.flags & PLAN_CLIP_FULL) && mbits != nullptr;
  if ((p.flags & PLAN_MED_FULL) && (p.flags & PLAN_MAD_FULL) && !do_clip) return;
  unsigned char* cls = p2_smem;
  for (int i = threadIdx.x; i < kClsCells / 16; i += kP2Threads)
    reinterpret_cast<uint4*>(cls)[i] = __ldg(reinterpret_cast<const uint4*>(L.cls) + i);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* smed = reinterpret_cast<float*>(p2_smem + kClsCells) + warp * kP2Stage;
  float* smad = reinterpret_cast<float*>(p2_smem + kClsCells) + (kP2Warps + warp) * kP2Stage;
  unsigned long long* samb =
      reinterpret_cast<unsigned long long*>(p2_smem + kClsCells + 2 * kP2Warps * kP2Stage * sizeof(float)) +
      warp * kP2Stage;
  __syncthreads();
  const float thr_lo = p.thr_lo, thr_hi = p.thr_hi;
  const unsigned int lanes_below = (1u << lane) - 1u;
  int nmed = 0, nmad = 0, namb = 0;
  const long long nchunks = (n + 127) >> 7;
  const long long wstride = (long long)gridDim.x * kP2Warps * kP2Unroll;
  float a[kP2Unroll][4], nxt[kP2Unroll][4];
  long long ch0 = ((long long)blockIdx.x * kP2Warps + warp) * kP2Unroll;
  if (ch0 < nchunks) p2_load(src, n, ch0, lane, a);
  for (; ch0 < nchunks; ch0 += wstride) {
    if (ch0 + wstride < nchunks) p2_load(src, n, ch0 + wstride, lane, nxt);
#pragma unroll
    for (int u = 0; u < kP2Unroll; ++u) {
      const long long ch = ch0 + u;
      unsigned int k[4], sure_w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
      for (int c = 0; c < 4; ++c) k[c] = cls[__float_as_uint(a[u][c]) >> 16];
      bool any_sure = false;  // warp-uniform
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        // most groups of 32 values hold no listed, sure or ambiguous value:
        // one vote settles them
        if (!__any_sync(0xffffffffu, k[c] != 0u)) continue;
        // the classes present in the group, one reduction for the warp
        const unsigned int present = __reduce_or_sync(0xffffffffu, k[c]);
        if (present & CLS_SURE) sure_w[c] = __ballot_sync(0xffffffffu, (k[c] & CLS_SURE) != 0u);
        const unsigned int kc = k[c] & ~CLS_SURE, listed = present & ~CLS_SURE;
        if (listed == CLS_MAD) {
          // the common case: MAD candidates only (values around +-MAD)
          const bool pa = kc != 0u;
          stage_push(__ballot_sync(0xffffffffu, pa), pa, lanes_below, a[u][c], smad, nmad);
        } else if (listed != 0u) {
          const float s = a[u][c];
          const float as = fabsf(s);
          const bool pm = (k[c] & CLS_MED) != 0u, pa = (k[c] & CLS_MAD) != 0u;
          const bool amb_cell = (k[c] & CLS_AMB) != 0u;  // finite: the cell is not Inf / NaN
          const bool sure = amb_cell && as > thr_hi;
          const bool pamb = amb_cell && as > thr_lo && !sure;
          sure_w[c] |= __ballot_sync(0xffffffffu, sure);
          const unsigned int bmed = __ballot_sync(0xffffffffu, pm);
          const unsigned int bmad = __ballot_sync(0xffffffffu, pa);
          const unsigned int bamb = __ballot_sync(0xffffffffu, pamb);
          stage_push(bmad, pa, lanes_below, s, smad, nmad);
          stage_push(bmed, pm, lanes_below, s, smed, nmed);
          stage_push(bamb, pamb, lanes_below, (unsigned long long)(ch * 128 + 32 * c + lane), samb, namb);
        }
        any_sure |= sure_w[c] != 0u;
      }
      if (any_sure) {
        // lane c owns mask word 4 * ch + c of this chunk (no SURE cells, so
        // no words, without a clip)
        unsigned int w = sure_w[0];
        w = lane == 1 ? sure_w[1] : w;
        w = lane == 2 ? sure_w[2] : w;
        w = lane == 3 ? sure_w[3] : w;
        if (do_clip && lane < 4 && w != 0u) atomicOr(mbits + ch * 4 + lane, w);
      }
      if (max(nmad, max(nmed, namb)) > kP2FlushAt) {
        if (nmad > kP2FlushAt) stage_flush(smad, nmad, L.mad, &st->n_cand_mad, L.cap.mad, &st->status);
        if (nmed > kP2FlushAt) stage_flush(smed, nmed, L.med, &st->n_cand_med, L.cap.med, &st->status);
        if (namb > kP2FlushAt) stage_flush(samb, namb, L.amb, &st->n_amb, L.cap.amb, &st->status);
      }
    }
#pragma unroll
    for (int u = 0; u < kP2Unroll; ++u)
#pragma unroll
      for (int c = 0; c < 4; ++c) a[u][c] = nxt[u][c];
  }
  stage_flush(smed, nmed, L.med, &st->n_cand_med, L.cap.med, &st->status);
  stage_flush(smad, nmad, L.mad, &st->n_cand_mad, L.cap.mad, &st->status);
  stage_flush(samb, namb, L.amb, &st->n_amb, L.cap.amb, &st->status);
}

cudaError_t launch_pass2(const float* src, long long n, uint32_t* mbits, DevState* st, Lists L, int sms,
                         cudaStream_t s) {
  const long long chunks = (n + 127) / 128;
  long long want = (chunks + kP2Warps * kP2Unroll - 1) / (kP2Warps * kP2Unroll);
  int grid = (int)(want < 1 ? 1 : (want > 2LL * sms ? 2LL * sms : want));
  k_pass2<<<grid, kP2Threads, kP2Smem, s>>>(src, n, mbits, st, L);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Radix selection. MAD keys are the correctly rounded float of the exact
// |s - m| (m is the exact median, a double): rounding is monotone, so the
// order statistics of the keys are the rounded order statistics of |s - m|.
__device__ __forceinline__ bool sel_key(const SelJob& J, double m, float s, unsigned int* key) {
  if (!isfinite(s)) return false;
  if (J.mode == SEL_VALUE) {
    *key = fkey(s);
  } else {
    *key = fkey(__double2float_rn(fabs((double)s - m)));
  }
  return true;
}

// A candidate list of |s - m| keys (not the whole array) holds, after the
// first round, the keys themselves in place of the values: that round forms
// each key once in float64 (slow on this GPU) and the later rounds read it.
// kNoKey marks a non-finite value (no finite key is that large; read as a
// float it is a NaN, so it is no value either).
constexpr unsigned int kNoKey = 0xffffffffu;
__device__ __forceinline__ bool sel_keys_stored(const SelJob& J) {
  return J.mode == SEL_ABSDEV && J.count_ptr != nullptr;
}
__device__ __forceinline__ bool sel_key_of(const SelJob& J, bool stored, double m, float v, unsigned int* key) {
  if (stored) {
    *key = __float_as_uint(v);
    return *key != kNoKey;
  }
  return sel_key(J, m, v, key);
}

// The lists are read kSelUnroll values a thread at a time, loads first, so
// that enough of them are in flight (a list of millions of candidates is
// otherwise bound by the latency of one load per thread).
constexpr int kSelUnroll = 16;
__device__ __forceinline__ void sel_load(const float* __restrict__ list, unsigned long long i0,
                                         unsigned long long stride, unsigned long long count,
                                         float (&v)[kSelUnroll]) {
#pragma unroll
  for (int u = 0; u < kSelUnroll; ++u) {
    const unsigned long long i = i0 + u * stride;
    v[u] = i < count ? __ldg(list + i) : __uint_as_float(kNoKey);  // past the end: no key either way
  }
}

// Elements in the list: the candidate count, clamped to the buffer capacity
// (count_fixed), or the whole array.
__device__ __forceinline__ unsigned long long sel_count(const SelJob& J) {
  return J.count_ptr ? min(*J.count_ptr, J.count_fixed) : J.count_fixed;
}

// Every block redoes the pick of round r-1 from its histogram (same result
// everywhere); block 0 records it.
__device__ void sel_pick(SelJob* J, int r, unsigned int* prefix, unsigned long long* rank, unsigned int* status) {
  __shared__ unsigned long long s_part[32];
  __shared__ unsigned int s_digit;
  __shared__ unsigned long long s_rank;
  const unsigned long long* h = J->hist[r - 1];
  const int tid = threadIdx.x, nt = blockDim.x;  // nt == 256 or 1024
  const int per = kSelBins / nt;
  unsigned long long loc = 0;
  for (int j = 0; j < per; ++j) loc += h[tid * per + j];
  // exclusive scan over threads
  unsigned long long incl = loc;
  for (int o = 1; o < 32; o <<= 1) {
    unsigned long long t = __shfl_up_sync(0xffffffffu, incl, o);
    if ((tid & 31) >= o) incl += t;
  }
  if ((tid & 31) == 31) s_part[tid >> 5] = incl;
  __syncthreads();
  if (tid < 32) {
    unsigned long long w = (tid < nt / 32) ? s_part[tid] : 0ull, wi = w;
    for (int o = 1; o < 32; o <<= 1) {
      unsigned long long t = __shfl_up_sync(0xffffffffu, wi, o);
      if (tid >= o) wi += t;
    }
    s_part[tid] = wi - w;
  }
  if (tid == 0) { s_digit = 0xffffffffu; s_rank = 0ull; }
  __syncthreads();
  const unsigned long long want = *rank;
  unsigned long long run = s_part[tid >> 5] + incl - loc;
  for (int j = 0; j < per; ++j) {
    const unsigned long long c = h[tid * per + j];
    if (want >= run && want < run + c) {
      s_digit = (unsigned)(tid * per + j);
      s_rank = want - run;
    }
    run += c;
  }
  __syncthreads();
  if (s_digit == 0xffffffffu) {
    if (tid == 0) atomicOr(status, (unsigned int)SC_ST_INTERNAL);
    *prefix = 0u;
    *rank = 0ull;
  } else {
    *prefix = ((*prefix) << sel_bits(r - 1)) | s_digit;
    *rank = s_rank;
  }
  __syncthreads();
}

__device__ __forceinline__ unsigned long long sel_rank0(const DevState* st, const SelJob* J, int which) {
  unsigned long long r = J->rank_lo;
  if (which == 1 && J->count_ptr != nullptr) r -= st->n_below;
  return r;
}

__global__ void __launch_bounds__(256) k_sel_round(DevState* st, int which, int r) {
  __shared__ unsigned int sh[kSelBins];
  SelJob* J = which ? &st->sel_mad : &st->sel_med;
  const NoisePlan& p = st->plan;
  if (p.flags & (PLAN_EMPTY | PLAN_STD)) return;
  unsigned int prefix = 0u;
  unsigned long long rank = sel_rank0(st, J, which);
  const unsigned long long count = sel_count(*J);
  if (r == 0 && rank >= count) {
    if (threadIdx.x == 0 && blockIdx.x == 0) atomicOr(&st->status, (unsigned int)SC_ST_INTERNAL);
    return;
  }
  if (r > 0) {
    prefix = J->prefix[r - 1 + 0];
    rank = J->rank_in[r - 1 + 0];
    if (r == 1) { prefix = 0u; rank = sel_rank0(st, J, which); }
    sel_pick(J, r, &prefix, &rank, &st->status);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      J->prefix[r] = prefix;
      J->rank_in[r] = rank;
    }
  }
  for (int i = threadIdx.x; i < kSelBins; i += blockDim.x) sh[i] = 0u;
  __syncthreads();
  const double m = st->m;
  const int shift_prev = (r == 0) ? 32 : sel_shift(r - 1);
  const int shift = sel_shift(r);
  const unsigned int dmask = (1u << sel_bits(r)) - 1u;
  const SelJob Jl = *J;
  const bool stored = r > 0 && sel_keys_stored(Jl);
  // the first round of a list of |s - m| values writes their keys over them
  float* const keys_out = (r == 0 && sel_keys_stored(Jl)) ? const_cast<float*>(Jl.list) : nullptr;
  // whole warps iterate together: a warp whose 32 values share one digit (a
  // list's candidates cluster in few digits, in the first round mostly in
  // one) adds to its bin once
  const unsigned lane = threadIdx.x & 31u;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long w0 = (unsigned long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); w0 < count;
       w0 += kSelUnroll * stride) {
    float v[kSelUnroll];
    sel_load(Jl.list, w0 + lane, stride, count, v);
#pragma unroll
    for (int u = 0; u < kSelUnroll; ++u) {
      const unsigned long long i = w0 + u * stride + lane;
      unsigned int key = 0u;
      bool ok = i < count && sel_key_of(Jl, stored, m, v[u], &key);
      if (keys_out && i < count) keys_out[i] = __uint_as_float(ok ? key : kNoKey);
      ok = ok && !(shift_prev < 32 && (key >> shift_prev) != prefix);
      const unsigned digit = ok ? (key >> shift) & dmask : 0xffffffffu;
      const unsigned d0 = __shfl_sync(0xffffffffu, digit, 0);
      if (__all_sync(0xffffffffu, digit == d0)) {
        if (lane == 0 && ok) atomicAdd(&sh[d0], 32u);
      } else if (ok) {
        atomicAdd(&sh[digit], 1u);
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kSelBins; i += blockDim.x)
    if (sh[i]) atomicAdd(&J->hist[r][i], (unsigned long long)sh[i]);
}

__global__ void __launch_bounds__(256) k_sel_succ(DevState* st, int which) {
  __shared__ unsigned long long s_c[8];
  __shared__ unsigned int s_m[8];
  SelJob* J = which ? &st->sel_mad : &st->sel_med;
  const NoisePlan& p = st->plan;
  if (p.flags & (PLAN_EMPTY | PLAN_STD)) return;
  const unsigned long long count = sel_count(*J);
  if (sel_rank0(st, J, which) >= count) return;
  unsigned int prefix = J->prefix[2];
  unsigned long long rank = J->rank_in[2];
  sel_pick(J, 3, &prefix, &rank, &st->status);
  const unsigned int key_lo = prefix;
  if (blockIdx.x == 0 && threadIdx.x == 0) J->key_lo = key_lo;
  const double m = st->m;
  const SelJob Jl = *J;
  const bool stored = sel_keys_stored(Jl);
  unsigned long long c = 0;
  unsigned int mn = 0xffffffffu;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i0 = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i0 < count;
       i0 += kSelUnroll * stride) {
    float v[kSelUnroll];
    sel_load(Jl.list, i0, stride, count, v);
#pragma unroll
    for (int u = 0; u < kSelUnroll; ++u) {
      unsigned int key;
      if (!sel_key_of(Jl, stored, m, v[u], &key)) continue;  // includes the places past the end
      if (key <= key_lo) ++c; else mn = min(mn, key);
    }
  }
  c = warp_sum_u64(c);
  for (int o = 16; o > 0; o >>= 1) mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
  const int warp = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { s_c[warp] = c; s_m[warp] = mn; }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long ct = 0;
    unsigned int mt = 0xffffffffu;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { ct += s_c[w]; mt = min(mt, s_m[w]); }
    if (ct) atomicAdd(&J->c_le, ct);
    if (mt != 0xffffffffu) atomicMin(&J->min_gt, mt);
  }
}

__global__ void k_sel_final(DevState* st, int which, int pair) {
  SelJob* J = which ? &st->sel_mad : &st->sel_med;
  const NoisePlan& p = st->plan;
  if (p.flags & (PLAN_EMPTY | PLAN_STD)) return;
  const unsigned long long count = sel_count(*J);
  const unsigned long long r_lo = sel_rank0(st, J, which);
  if (r_lo >= count) {
    atomicOr(&st->status, (unsigned int)SC_ST_INTERNAL);
    return;
  }
  const unsigned long long r_hi = r_lo + (p.k_hi - p.k_lo);
  const unsigned int k_lo = J->key_lo;
  unsigned int k_hi = k_lo;
  if (r_hi >= J->c_le) {
    k_hi = J->min_gt;
    if (k_hi == 0xffffffffu) {
      atomicOr(&st->status, (unsigned int)SC_ST_INTERNAL);
      k_hi = k_lo;
    }
  }
  const double v_lo = (double)fkey_inv(k_lo), v_hi = (double)fkey_inv(k_hi);
  const double v = (k_hi == k_lo) ? v_lo : 0.5 * (v_lo + v_hi);
  if (which == 0) {
    st->m = v;
  } else {
    st->mad = v;
    st->sigma_cur_d = kMadToSigma * v;
    const float sg = sigma_of_mad(v);
    st->sigma_cur = sg;
    if (pair >= 0) st->sigma[pair] = sg;
    if (!(sg > 0.0f)) st->warn |= SC_WARN_ZERO_SIGMA;
  }
}

cudaError_t launch_select(DevState* st, int which, int pair, int sms, cudaStream_t s) {
  const int grid = 2 * sms;
  for (int r = 0; r < 3; ++r) {
    k_sel_round<<<grid, 256, 0, s>>>(st, which, r);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  k_sel_succ<<<grid, 256, 0, s>>>(st, which);
  k_sel_final<<<1, 1, 0, s>>>(st, which, pair);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// STD mode: float64 sums (the float32 data's squares can overflow or
// underflow float32), two passes: mean, then sum of squared deviations.
__global__ void __launch_bounds__(256) k_std_pass(const float* __restrict__ x, long long n, DevState* st, int second) {
  __shared__ double s_a[8];
  __shared__ unsigned long long s_n[8];
  if (st->plan.flags & PLAN_EMPTY) return;
  const double mean = second ? st->sum / (double)st->count : 0.0;
  double acc = 0.0;
  unsigned long long cnt = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float s = __ldg(x + i);
    if (!isfinite(s)) continue;
    if (second) {
      const double d = (double)s - mean;
      acc = fma(d, d, acc);
    } else {
      acc += (double)s;
    }
    ++cnt;
  }
  double a = acc;
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  cnt = warp_sum_u64(cnt);
  const int warp = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { s_a[warp] = a; s_n[warp] = cnt; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double at = 0.0;
    unsigned long long ct = 0;
    for (int w = 0; w < 8; ++w) { at += s_a[w]; ct += s_n[w]; }
    if (second) {
      atomicAdd(&st->sum2, at);
    } else {
      atomicAdd(&st->sum, at);
      atomicAdd(&st->count, ct);
    }
  }
}

__global__ void k_std_final(DevState* st, int pair) {
  if (st->plan.flags & PLAN_EMPTY) return;
  const unsigned long long c = st->count;
  const double sd = c > 1ull ? sqrt(st->sum2 / (double)(c - 1ull)) : 0.0;
  const float sg = (float)sd;
  st->sigma_cur = sg;
  st->sigma_cur_d = sd;
  if (pair >= 0) st->sigma[pair] = sg;
  if (!(sg > 0.0f)) st->warn |= SC_WARN_ZERO_SIGMA;
}

cudaError_t launch_std(const float* src, long long n, DevState* st, int sms, cudaStream_t s) {
  long long want = (n + 255) / 256;
  int grid = (int)(want < 1 ? 1 : (want > 4LL * sms ? 4LL * sms : want));
  k_std_pass<<<grid, 256, 0, s>>>(src, n, st, 0);
  k_std_pass<<<grid, 256, 0, s>>>(src, n, st, 1);
  return cudaGetLastError();
}

cudaError_t launch_std_final(DevState* st, int pair, cudaStream_t s) {
  k_std_final<<<1, 1, 0, s>>>(st, pair);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Clip: the undecided voxels, or a full pass when the plan asked for one.
__global__ void k_resolve(const float* __restrict__ src, uint32_t* mbits, DevState* st, Lists L) {
  const NoisePlan& p = st->plan;
  if (!(p.flags & PLAN_CLIP) || (p.flags & (PLAN_CLIP_FULL | PLAN_EMPTY))) return;
  const float sg = st->sigma_cur;
  if (!(sg > 0.0f)) return;
  const float thr = __fmul_rn(p.threshold, sg);
  const unsigned long long na = min(st->n_amb, L.cap.amb);
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < na;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long v = L.amb[i];
    if (fabsf(__ldg(src + v)) > thr) atomicOr(mbits + (v >> 5), 1u << (v & 31ull));
  }
}

cudaError_t launch_resolve(const float* src, uint32_t* mbits, DevState* st, Lists L, int sms, cudaStream_t s) {
  k_resolve<<<sms, 256, 0, s>>>(src, mbits, st, L);
  return cudaGetLastError();
}

// resident k_clip_full blocks per SM (init_noise_attrs, which every context
// creation runs, possibly from several host threads at once)
static std::atomic<int> g_clip_blocks_per_sm{0};

// Lane l holds values l, l + 32, l + 64 and l + 96 of chunk ch (each load
// instruction reads 128 contiguous bytes), so ballot c is mask word 4 ch + c
// as it stands; 0 past n.
__device__ __forceinline__ void clip_load(const float* __restrict__ src, long long n, long long ch, int lane,
                                          float (&a)[4]) {
  const long long v0 = ch * 128 + lane;
  if (ch * 128 + 128 <= n) {
#pragma unroll
    for (int c = 0; c < 4; ++c) a[c] = __ldg(src + v0 + 32 * c);
  } else {
#pragma unroll
    for (int c = 0; c < 4; ++c) a[c] = (v0 + 32 * c < n) ? __ldg(src + v0 + 32 * c) : 0.0f;
  }
}

// Sets chunk ch's detected bits: lane c < 4 owns word 4 ch + c.
__device__ __forceinline__ void clip_store(uint32_t* mbits, long long ch, int lane, float thr, const float (&a)[4]) {
  unsigned int w = 0u;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const float m = fabsf(a[c]);  // NaN fails the first compare, Inf the second
    const unsigned int b = __ballot_sync(0xffffffffu, m > thr && m <= FLT_MAX);
    w = lane == c ? b : w;
  }
  if (lane < 4 && w) atomicOr(mbits + ch * 4 + lane, w);  // no return value: no wait for the word
}

__global__ void __launch_bounds__(256) k_clip_full(const float* __restrict__ src, long long n, uint32_t* mbits,
                                                   DevState* st) {
  const NoisePlan& p = st->plan;
  if (!(p.flags & PLAN_CLIP) || !(p.flags & PLAN_CLIP_FULL) || (p.flags & PLAN_EMPTY)) return;
  const float sg = st->sigma_cur;
  if (!(sg > 0.0f)) return;
  const float thr = __fmul_rn(p.threshold, sg);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long nchunks = (n + 127) / 128;
  const long long stride = (long long)gridDim.x * 8;
  // two chunks a warp per iteration, all eight loads issued before a ballot
  for (long long ch = (long long)blockIdx.x * 8 + warp; ch < nchunks; ch += 2 * stride) {
    const long long ch2 = ch + stride;
    float a[4], b[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    clip_load(src, n, ch, lane, a);
    if (ch2 < nchunks) clip_load(src, n, ch2, lane, b);
    clip_store(mbits, ch, lane, thr, a);
    if (ch2 < nchunks) clip_store(mbits, ch2, lane, thr, b);
  }
}

cudaError_t launch_clip_full(const float* src, long long n, uint32_t* mbits, DevState* st, int sms,
                             cudaStream_t s) {
  // one wave: as many blocks as are resident at once (a second, partial wave
  // would run on a fraction of the SMs)
  const int per_sm = g_clip_blocks_per_sm.load(std::memory_order_relaxed);
  const long long cap = (long long)(per_sm > 0 ? per_sm : 4) * sms;
  long long want = (n + 1023) / 1024;
  int grid = (int)(want < 1 ? 1 : (want > cap ? cap : want));
  k_clip_full<<<grid, 256, 0, s>>>(src, n, mbits, st);
  return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// After sigma_0: replacement value, bin window, fixed-point scales.
// Fixed-point shift of every pair: X_q = rint(X * 2^f) with
// max|X| * 2^f * Wf <= 2^62 (Wf >= W), so that no exact sum can overflow
// int64. The replacement value repl_d (float64) is quantised once per pair.
__device__ void fx_setup(DevState* st, double repl_d, const PairWeights& W, int n_pairs) {
  const float maxabs = __uint_as_float(st->maxabs_bits);
  const float mx = fmaxf(maxabs, __double2float_ru(repl_d));
  int ex = 0;
  frexpf(mx, &ex);  // mx < 2^ex
  if (mx == 0.0f) ex = 0;
  // f depends on the spatial kernel (through wf) but not on a spectral width up
  // to kShareMaxWz, so pairs with one spatial kernel quantise alike and can
  // share their stored spatial sums.
  for (int k = 0; k < n_pairs; ++k) {
    const long long w = W.w[k];
    const int bits = 64 - __clzll((unsigned long long)(W.wf[k] - 1));  // bit length of wf - 1
    int f = 62 - ex - bits;
    if (f > 120) f = 120;
    if (f < -120) f = -120;
    st->fx_shift[k] = f;
    st->fx_scale[k] = ldexpf(1.0f, f);
    st->fx_inv[k] = (float)(ldexp(1.0, -f) / (double)w);
    st->fx_qrepl[k] = __double2ll_rn(ldexp(repl_d, f));
  }
}

__global__ void k_fx_setup(DevState* st, float repl_value, PairWeights W, int n_pairs) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    st->repl_d = (double)repl_value;
    st->repl = repl_value;
    fx_setup(st, (double)repl_value, W, n_pairs);
  }
}

cudaError_t launch_fx_setup(DevState* st, float repl_value, const PairWeights& W, int n_pairs, cudaStream_t s) {
  k_fx_setup<<<1, 1, 0, s>>>(st, repl_value, W, n_pairs);
  return cudaGetLastError();
}

// Window of the fine histogram of the raw cube: the bin of the median of |x|
// gives the scale, and the window spans 2^-20 .. 2^12 of it (as for the
// smoothed cubes), so the plan of the sigma_0 measurement resolves 128 bins
// per octave instead of 16. The median |x| comes from kWinSample values at
// a fixed step through the cube (all of them in a smaller cube): a window 32
// octaves wide needs its scale only roughly, and the exact selection that
// follows does not depend on it (a poorly placed window costs candidates,
// never exactness).
constexpr int kWinThreads = 1024;
constexpr long long kWinSample = 65536;
constexpr int kWinPerThread = (int)(kWinSample / kWinThreads);
__global__ void __launch_bounds__(kWinThreads) k_window_from_sample(const float* __restrict__ x, Half16 h,
                                                                    long long plane, long long n, DevState* st) {
  extern __shared__ unsigned int wh[];  // full-range histogram of the sample
  __shared__ unsigned long long s_w[32];
  __shared__ int s_mb;
  const BinCfg full = kFullRange;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  for (int i = t; i < kNumBins; i += kWinThreads) wh[i] = 0u;
  __syncthreads();
  // m values step apart (every value of a cube of at most kWinSample)
  const long long m = n < kWinSample ? n : kWinSample, step = n / (m > 0 ? m : 1);
  constexpr int kBatch = 16;  // loads in flight per thread
  for (int j0 = 0; j0 < kWinPerThread; j0 += kBatch) {
    float v[kBatch];
#pragma unroll
    for (int j = 0; j < kBatch; ++j) {
      const long long k = (long long)(j0 + j) * kWinThreads + t;
      const long long i = k * step;
      v[j] = __int_as_float(0x7fc00000);
      if (k < m) v[j] = h.fmt ? half16_value(__ldg(h.bits + i), h.fmt, __ldg(h.scale + i / plane)) : __ldg(x + i);
    }
#pragma unroll
    for (int j = 0; j < kBatch; ++j)
      if (isfinite(v[j])) atomicAdd(&wh[bin_of(v[j], full)], 1u);
  }
  __syncthreads();
  // thread t holds magnitude bins [t * per, t * per + per), both signs
  constexpr int per = (kBinsPerSign + kWinThreads - 1) / kWinThreads;
  unsigned long long c[per], loc = 0;
#pragma unroll
  for (int j = 0; j < per; ++j) {
    const int mb = t * per + j;
    c[j] = mb < kBinsPerSign ? (unsigned long long)wh[kBinsPerSign + mb] + wh[kBinsPerSign - 1 - mb] : 0ull;
    loc += c[j];
  }
  unsigned long long inc = loc;  // inclusive scan over the warp, then over the warps
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) s_w[warp] = inc;
  if (t == 0) s_mb = -1;
  __syncthreads();
  if (warp == 0) {
    const unsigned long long xw = s_w[lane];
    unsigned long long xi = xw;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, xi, o);
      if (lane >= o) xi += y;
    }
    s_w[lane] = xi;  // inclusive over warps; s_w[31] is the total
  }
  __syncthreads();
  const unsigned long long total = s_w[31];
  // the first magnitude bin whose cumulative count exceeds half of the sample
  unsigned long long run = (warp ? s_w[warp - 1] : 0ull) + inc - loc;
#pragma unroll
  for (int j = 0; j < per; ++j) {
    if (2 * run <= total && 2 * (run + c[j]) > total) s_mb = t * per + j;
    run += c[j];
  }
  __syncthreads();
  if (t == 0) {
    const float scale = (total > 0 && s_mb >= 0) ? (float)mag_hi(s_mb, full) : 0.0f;
    st->win = window_cfg(isfinite(scale) ? scale : 3.0e38f);
  }
}

cudaError_t launch_window_from_sample(const float* x, const Half16* h16, long long plane, long long n, DevState* st,
                                      cudaStream_t s) {
  Half16 h{};
  if (h16) h = *h16;
  k_window_from_sample<<<1, kWinThreads, kNumBins * sizeof(unsigned int), s>>>(x, h, plane, n, st);
  return cudaGetLastError();
}

__global__ void k_sigma0_done(DevState* st, float replacement, PairWeights W, int n_pairs) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const float s0 = st->sigma_cur;
  st->sigma0 = s0;
  st->repl_d = (replacement > 0.0f) ? (double)replacement * st->sigma_cur_d : 0.0;
  st->repl = __double2float_rn(st->repl_d);
  st->win = window_cfg(s0);
  const float mx = fmaxf(__uint_as_float(st->maxabs_bits), st->repl);
  if (s0 > 0.0f && mx > s0 * 1048576.0f) st->warn |= SC_WARN_RANGE;
  fx_setup(st, st->repl_d, W, n_pairs);
}

cudaError_t launch_sigma0_done(DevState* st, float replacement, const PairWeights& W, int n_pairs, cudaStream_t s) {
  k_sigma0_done<<<1, 1, 0, s>>>(st, replacement, W, n_pairs);
  return cudaGetLastError();
}

// The latest run's sigmas for sc_copy_sigmas: out[k] = sigma_k (k < n),
// out[n] = sigma_0, all zero when the run's device-side status is an error
// (its sigmas are then meaningless).
__global__ void k_sigma_out(const DevState* st, int n, float* out) {
  const bool ok = st->status == 0u;
  for (int k = threadIdx.x; k <= n; k += blockDim.x) out[k] = ok ? (k < n ? st->sigma[k] : st->sigma0) : 0.0f;
}

cudaError_t launch_sigma_out(const DevState* st, int n, float* out, cudaStream_t s) {
  k_sigma_out<<<1, 64, 0, s>>>(st, n, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// uint8 mask <-> 1-bit working mask.
// Working mask from a caller's uint8 mask: a bit for every set voxel whose
// cube value is finite (non-finite voxels are never replaced, and no clip
// ever sets their bit, so the working mask holds finite voxels only).
__global__ void k_pack(const uint8_t* __restrict__ m8, const float* __restrict__ cube, long long n,
                       uint32_t* __restrict__ mbits) {
  const long long nw = (n + 31) / 32;
  for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += (long long)gridDim.x * blockDim.x) {
    unsigned int bits = 0u;
    const long long v0 = w * 32;
    for (int i = 0; i < 32; ++i)
      if (v0 + i < n && m8[v0 + i] && isfinite(__ldg(cube + v0 + i))) bits |= 1u << i;
    mbits[w] = bits;
  }
}
// The same for a 16-bit cube (finiteness of the decoded value).
__global__ void k_pack16(const uint8_t* __restrict__ m8, Half16 h, long long plane, long long n,
                         uint32_t* __restrict__ mbits) {
  const long long nw = (n + 31) / 32;
  for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += (long long)gridDim.x * blockDim.x) {
    unsigned int bits = 0u;
    const long long v0 = w * 32;
    const long long z0 = v0 / plane, next = (z0 + 1) * plane;
    for (int i = 0; i < 32; ++i) {
      const long long v = v0 + i;
      if (v < n && m8[v]) {
        const float cs = __ldg(h.scale + (v >= next ? z0 + 1 : z0));
        if (isfinite(half16_value(__ldg(h.bits + v), h.fmt, cs))) bits |= 1u << i;
      }
    }
    mbits[w] = bits;
  }
}

cudaError_t launch_pack16(const uint8_t* m8, const Half16& h, long long plane, long long n, uint32_t* mbits,
                          cudaStream_t s) {
  long long nw = (n + 31) / 32;
  long long want = (nw + 255) / 256;
  int grid = (int)(want < 1 ? 1 : (want > 4096 ? 4096 : want));
  k_pack16<<<grid, 256, 0, s>>>(m8, h, plane, n, mbits);
  return cudaGetLastError();
}

cudaError_t launch_pack(const uint8_t* m8, const float* cube, long long n, uint32_t* mbits, cudaStream_t s) {
  long long nw = (n + 31) / 32;
  long long want = (nw + 255) / 256;
  int grid = (int)(want < 1 ? 1 : (want > 4096 ? 4096 : want));
  k_pack<<<grid, 256, 0, s>>>(m8, cube, n, mbits);
  return cudaGetLastError();
}

// uint8 mask from the working mask; with keep, OR-ed into the caller's mask
// (whose set voxels at non-finite values the working mask does not hold).
__global__ void k_expand(const uint32_t* __restrict__ mbits, long long n, uint8_t* __restrict__ m8, int keep) {
  // each thread writes 16 bytes
  const bool vec = ((reinterpret_cast<uintptr_t>(m8) & 15u) == 0);
  const long long ng = (n + 15) / 16;
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += (long long)gridDim.x * blockDim.x) {
    const long long v0 = g * 16;
    const unsigned int w = __ldg(mbits + (v0 >> 5)) >> (v0 & 31);
    if (vec && v0 + 16 <= n) {
      uint4 o = keep ? *reinterpret_cast<const uint4*>(m8 + v0) : make_uint4(0u, 0u, 0u, 0u);
      unsigned int* po = &o.x;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        unsigned int b = 0u;
#pragma unroll
        for (int i = 0; i < 4; ++i) b |= ((w >> (4 * q + i)) & 1u) << (8 * i);
        // 0x01 in every byte of the caller's word that is non-zero
        const unsigned int t = po[q];
        const unsigned int nz = ((((t & 0x7f7f7f7fu) + 0x7f7f7f7fu) | t) >> 7) & 0x01010101u;
        po[q] = keep ? (b | nz) : b;
      }
      *reinterpret_cast<uint4*>(m8 + v0) = o;
    } else {
      for (int i = 0; i < 16 && v0 + i < n; ++i)
        m8[v0 + i] = (uint8_t)((((w >> i) & 1u) != 0u || (keep && m8[v0 + i] != 0)) ? 1u : 0u);
    }
  }
}
cudaError_t launch_expand(const uint32_t* mbits, long long n, uint8_t* m8, int keep, cudaStream_t s) {
  long long ng = (n + 15) / 16;
  long long want = (ng + 255) / 256;
  int grid = (int)(want < 1 ? 1 : (want > 8192 ? 8192 : want));
  k_expand<<<grid, 256, 0, s>>>(mbits, n, m8, keep);
  return cudaGetLastError();
}

void init_noise_attrs() {
  cudaFuncSetAttribute(k_plan, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)((kNumBins + 1) * sizeof(unsigned long long)));
  cudaFuncSetAttribute(k_pass2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kP2Smem);
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_clip_full, 256, 0) != cudaSuccess) {
    cudaGetLastError();
    b = 0;
  }
  if (b > 0) g_clip_blocks_per_sm.store(b, std::memory_order_relaxed);
}

}  // namespace sc
