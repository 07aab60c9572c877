// Device helpers: order-preserving float keys, histogram bins, exact
// fixed-point conversions.
#pragma once

#include <cstdint>

#include <cuda_fp16.h>

#include "sc_internal.h"

namespace sc {

// Order-preserving uint32 key of a float: key(a) < key(b) iff a < b for
// non-NaN a, b (with -0 just below +0).
__device__ __forceinline__ unsigned int fkey(float s) {
  unsigned int u = __float_as_uint(s);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float fkey_inv(unsigned int k) {
  unsigned int u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
  return __uint_as_float(u);
}

__host__ __device__ __forceinline__ BinCfg window_cfg(float sigma0) {
  // 32 octaves [2^-20, 2^12) x sigma0, clamped to the exponent range.
  unsigned int u;
#ifdef __CUDA_ARCH__
  u = __float_as_uint(sigma0);
#else
  __builtin_memcpy(&u, &sigma0, 4);
#endif
  int e = (int)((u >> 23) & 0xff) - kWindowBelow;
  if (e < 1) e = 1;
  if (e > 255 - kWindowE) e = 255 - kWindowE;
  return BinCfg{e, kWindowE, kWindowMB};
}

// Histogram bin of a non-NaN float (monotone in the value): the magnitude's
// top 9 + MB bits (exponent and MB mantissa bits), offset by the window base
// and clamped to the underflow / overflow bins.
__host__ __device__ __forceinline__ int bin_of_bits(unsigned int u, BinCfg c) {
  const int key = (int)((u & 0x7fffffffu) >> (23 - c.MB));
  int b = key - (c.e_base << c.MB) + 1;
  b = b < 0 ? 0 : b;
  b = b > (c.E << c.MB) + 1 ? (c.E << c.MB) + 1 : b;
  // negative values mirror: kBinsPerSign - 1 - b = kBinsPerSign + (b ^ -1)
  return kBinsPerSign + (b ^ -(int)(u >> 31));
}
__device__ __forceinline__ int bin_of(float s, BinCfg c) { return bin_of_bits(__float_as_uint(s), c); }

// Smallest and largest magnitude (inclusive, conservative) of magnitude bin mb.
__device__ __forceinline__ double mag_lo(int mb, BinCfg c) {
  if (mb == 0) return 0.0;
  if (mb == (c.E << c.MB) + 1) return (double)__uint_as_float((unsigned)(c.e_base + c.E) << 23);
  int e = c.e_base + ((mb - 1) >> c.MB);
  unsigned int mt = (unsigned)(mb - 1) & ((1u << c.MB) - 1u);
  unsigned int bits = ((unsigned)e << 23) | (mt << (23 - c.MB));
  if (e >= 255) return __longlong_as_double(0x7ff0000000000000LL);
  return (double)__uint_as_float(bits);
}
__device__ __forceinline__ double mag_hi(int mb, BinCfg c) {
  const double inf = __longlong_as_double(0x7ff0000000000000LL);
  if (mb == (c.E << c.MB) + 1) return inf;
  unsigned int bits;
  if (mb == 0) {
    bits = (unsigned)c.e_base << 23;
  } else {
    int e = c.e_base + ((mb - 1) >> c.MB);
    unsigned int mt = (unsigned)(mb - 1) & ((1u << c.MB) - 1u);
    bits = (((unsigned)e << 23) | (mt << (23 - c.MB))) + (1u << (23 - c.MB));
  }
  if ((bits >> 23) >= 255u) return inf;
  return (double)__uint_as_float(bits);
}
__device__ __forceinline__ double bin_lo_value(int i, BinCfg c) {
  return i >= kBinsPerSign ? mag_lo(i - kBinsPerSign, c) : -mag_hi(kBinsPerSign - 1 - i, c);
}
__device__ __forceinline__ double bin_hi_value(int i, BinCfg c) {
  return i >= kBinsPerSign ? mag_hi(i - kBinsPerSign, c) : -mag_lo(kBinsPerSign - 1 - i, c);
}

// rint(x * 2^f) (ties to even) as an exact int64, for |x| * 2^f < 2^62,
// given scale = 2^f. Uses the FMA and conversion pipes rather than the
// integer pipe (the 64-bit cvt instructions run on the FP64 pipe): with
// y = |x| * 2^f (exact), hi = floor(y * 2^-32) and lo = y - hi * 2^32 (an
// exact FMA, 0 <= lo < 2^32) each convert exactly, lo with the rounding.
// NaN or infinite x give an unspecified value (callers blank them).
__device__ __forceinline__ long long quantize(float x, float scale) {
  const float y = __fmul_rn(fabsf(x), scale);
  const float th = floorf(__fmul_rn(y, 2.3283064365386963e-10f));  // 2^-32
  const float lo_f = __fmaf_rn(-th, 4294967296.0f, y);
  const unsigned int hi = __float2uint_rz(th);
  const unsigned int lo = __float2uint_rn(lo_f);
  const long long r = (long long)(((unsigned long long)hi << 32) | lo);
  return x < 0.0f ? -r : r;
}

// quantize() with the replacement of a masked voxel folded in: the magnitude
// is the replacement's when `masked`, then one sign step for x < 0 (so -0 and
// positive values take +, as sgn(0) = +1 requires). x + (x - x) makes NaN and
// Inf quantise to 0; masked voxels are finite.
__device__ __forceinline__ long long quantize_repl(float x, float scale, bool masked, long long qrepl) {
  const float xf = x + (x - x);
  const float y = __fmul_rn(fabsf(xf), scale);
  const float th = floorf(__fmul_rn(y, 2.3283064365386963e-10f));  // 2^-32
  const float lo_f = __fmaf_rn(-th, 4294967296.0f, y);
  const unsigned int hi = __float2uint_rz(th);
  const unsigned int lo = __float2uint_rn(lo_f);
  const long long r = (long long)(((unsigned long long)hi << 32) | lo);
  const long long m = masked ? qrepl : r;
  return x < 0.0f ? -m : m;
}

// Correctly rounded (to nearest, ties to even) float of an unsigned 64-bit
// integer, from integer operations (the 64-bit cvt runs on the FP64 pipe).
// Branch-free.
__device__ __forceinline__ float u64_to_float_rn(unsigned long long a) {
  const int lz = __clzll((long long)a);                   // 64 for a == 0
  const unsigned long long n = a << (lz & 63);            // leading one at bit 63
  unsigned int mant = (unsigned int)(n >> 40);            // 24 significant bits
  const unsigned long long rest = n & 0xffffffffffull;
  const unsigned long long half = 0x8000000000ull;
  mant += (rest > half || (rest == half && (mant & 1u))) ? 1u : 0u;  // may carry to 2^24
  const unsigned int e = (unsigned int)(63 - lz + 127);
  const unsigned int bits = (e << 23) + (mant - 0x800000u);  // a carry moves into the exponent
  return __uint_as_float(a == 0ull ? 0u : bits);
}

// float of q * inv from two 32-bit conversions (signed high word, unsigned
// low word), one FMA and one multiply. The low word's rounding costs at most
// 2^7 units of q (|error| <= 2^7 * inv absolute, far below the float
// resolution of any value above 2^31 * inv); above that the result is within
// about 2 ulp of the exact product.
__device__ __forceinline__ float dequantize(long long q, float inv) {
  const float hi = __int2float_rn((int)(q >> 32));
  const float lo = __uint2float_rn((unsigned int)((unsigned long long)q & 0xffffffffull));
  return __fmul_rn(__fmaf_rn(hi, 4294967296.0f, lo), inv);
}

// Value of a 16-bit cube element: the BF16 or FP16 number times its channel's
// float32 scale, one float32 rounding (the same product the decoding pass
// forms, so both paths see identical values).
__device__ __forceinline__ float half16_value(unsigned short b, int fmt, float scale) {
  const float v = fmt == SC_STORE_BF16 ? __uint_as_float((unsigned)b << 16) : __half2float(__ushort_as_half(b));
  return __fmul_rn(v, scale);
}

__device__ __forceinline__ bool mask_bit(const uint32_t* mbits, long long v) {
  return mbits != nullptr && ((__ldg(mbits + (v >> 5)) >> (v & 31)) & 1u);
}

__device__ __forceinline__ float warp_sum_f(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace sc
