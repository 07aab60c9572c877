// Building blocks shared by the tiled smoothing kernels: streamed box
// cascades, Tensor Memory (TMEM) used as ring storage, mbarriers, TMA tile
// loads and the host-side tensor-map / shared-memory set-up.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdint>

namespace sc {
namespace tc {

__host__ __device__ constexpr size_t al128(size_t v) { return (v + 127) & ~(size_t)127; }

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// Streams NOUT + W1 + W2 + W3 - 3 inputs load(i) through three centred
// boxcars of widths W1, W2, W3 as running int64 sums (all indices are
// compile-time after unrolling); out(k, v) receives output k, the sum over the
// composed kernel's support.
template <int W1, int W2, int W3, int NOUT, class Load, class Out>
__device__ __forceinline__ void cascade_stream(Load load, Out out) {
  // Each running sum takes its entering and leaving values as one difference
  // computed off the recurrence, so a step adds one 64-bit add to each chain.
  constexpr int N0 = NOUT + (W1 - 1) + (W2 - 1) + (W3 - 1);
  long long h1[W1], h2[W2], h3[W3];
  long long s1 = 0, s2 = 0, s3 = 0;
#pragma unroll
  for (int i = 0; i < N0; ++i) {
    const long long x = load(i);
    if (W1 == 1) {
      s1 = x;
    } else {
      s1 += (i >= W1) ? x - h1[i % W1] : x;
      h1[i % W1] = x;
    }
    if (i >= W1 - 1) {
      const int i1 = i - (W1 - 1);
      if (W2 == 1) {
        s2 = s1;
      } else {
        s2 += (i1 >= W2) ? s1 - h2[i1 % W2] : s1;
        h2[i1 % W2] = s1;
      }
      if (i1 >= W2 - 1) {
        const int i2 = i1 - (W2 - 1);
        if (W3 == 1) {
          s3 = s2;
        } else {
          s3 += (i2 >= W3) ? s2 - h3[i2 % W3] : s2;
          h3[i2 % W3] = s2;
        }
        if (i2 >= W3 - 1) out(i2 - (W3 - 1), s3);
      }
    }
  }
}

// Streams NOUT + 2R inputs load(i) through a centred FIR of 2R + 1 symmetric
// integer taps (taps[d] == taps[2R - d], non-negative, below 2^20): out(k, v)
// receives the exact sum v = sum_d taps[d] * load(k + d), d = 0..2R, taken as
// taps[R] * x[k + R] + sum_{d < R} taps[d] * (x[k + d] + x[k + 2R - d]), so
// that the two inputs sharing a tap are added before one multiplication. Each
// int64 operand is split into its unsigned low and signed high 32-bit halves,
// whose wide products with the tap accumulate in two 64-bit sums (neither can
// overflow for fewer than 2^12 taps); the two recombine modulo 2^64, exact
// whenever the true sum fits in int64 (so does every pair sum, each at most
// twice an input). Outputs are made C at a time from a register window of
// C + 2R inputs. With compile-time indices the taps are read straight from
// the kernel's parameters.
template <int R, int NOUT, class Load, class Out>
__device__ __forceinline__ void fir_stream(const int* __restrict__ taps, Load load, Out out) {
  constexpr int C = NOUT < 4 ? NOUT : 4;
#pragma unroll
  for (int c0 = 0; c0 < NOUT; c0 += C) {
    long long w[C + 2 * R];
#pragma unroll
    for (int i = 0; i < C + 2 * R; ++i) w[i] = (c0 + i < NOUT + 2 * R) ? load(c0 + i) : 0ll;
#pragma unroll
    for (int k = 0; k < C; ++k) {
      if (c0 + k < NOUT) {
        const long long xc = w[k + R];
        unsigned long long lo_acc = (unsigned long long)(unsigned)((unsigned long long)xc & 0xffffffffull) *
                                    (unsigned)taps[R];
        long long hi_acc = (long long)(int)(xc >> 32) * (long long)taps[R];
#pragma unroll
        for (int d = 0; d < R; ++d) {
          const long long p = w[k + d] + w[k + 2 * R - d];
          lo_acc += (unsigned long long)(unsigned)((unsigned long long)p & 0xffffffffull) * (unsigned)taps[d];
          hi_acc += (long long)(int)(p >> 32) * (long long)taps[d];
        }
        out(c0 + k, (long long)(lo_acc + ((unsigned long long)hi_acc << 32)));
      }
    }
  }
}

// The spatial kernel along one axis: the 3-box cascade <W1, W2, W3>, or, for
// W1 == 0, the FIR of half-width W2 with the 2 W2 + 1 taps `taps` (unused by
// the cascade).
template <int W1, int W2, int W3, int NOUT, class Load, class Out>
__device__ __forceinline__ void spatial_stream(const int* __restrict__ taps, Load load, Out out) {
  if constexpr (W1 == 0) {
    fir_stream<W2, NOUT>(taps, load, out);
  } else {
    cascade_stream<W1, W2, W3, NOUT>(load, out);
  }
}

// ---- Tensor Memory as ring storage ----------------------------------------
// A block allocates all 512 columns of its SM's TMEM (one block per SM). Warp
// w may access lanes 32*(w%4) .. +31 only.
constexpr int kTmemCols = 512;

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
__device__ __forceinline__ void tmem_ld8(unsigned taddr, unsigned (&v)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
               : "r"(taddr)
               : "memory");
}
__device__ __forceinline__ void tmem_st8(unsigned taddr, const unsigned (&v)[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "r"(v[0]),
               "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
               : "memory");
}
__device__ __forceinline__ void tmem_ld16(unsigned taddr, unsigned (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tmem_st16(unsigned taddr, const unsigned (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
          taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
      "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
      : "memory");
}

// ---- mbarrier / named barriers / TMA / cp.async ---------------------------
constexpr long long kMaxSpins = 1LL << 24;        // bound of an iteration-counted wait
constexpr unsigned long long kWaitNs = 200000000;  // bound of a time-limited wait (0.2 s)

__device__ __forceinline__ void mbar_init(unsigned addr, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(addr), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned addr, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(addr), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned addr) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(addr) : "memory");
}
__device__ __forceinline__ bool mbar_try(unsigned addr, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(addr), "r"(parity)
      : "memory");
  return ok != 0u;
}
// Wait for the barrier phase with the given parity, at most kMaxSpins tries.
__device__ __forceinline__ bool mbar_wait(unsigned addr, unsigned parity) {
  for (long long it = 0; it < kMaxSpins; ++it)
    if (mbar_try(addr, parity)) return true;
  return false;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait for the barrier phase with the given parity for at most limit_ns of
// wall time (kWaitNs by default). A thread whose wait ran out sets
// *timed_out and from then on waits no more, so a broken hand-off ends the
// kernel quickly with an error.
__device__ __forceinline__ void mbar_wait_bounded(unsigned addr, unsigned parity, bool* timed_out,
                                                  unsigned long long limit_ns = kWaitNs) {
  if (*timed_out) return;
  if (mbar_try(addr, parity)) return;
  const unsigned long long t0 = global_ns();
  while (!mbar_try(addr, parity)) {
    if (global_ns() - t0 > limit_ns) {
      *timed_out = true;
      return;
    }
  }
}
// Barrier among `count` threads (a multiple of 32) on hardware barrier `id`.
__device__ __forceinline__ void named_bar_sync(unsigned id, unsigned count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void tma_load_3d(unsigned dst, const CUtensorMap* map, int x, int y, int z, unsigned mbar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          dst),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(mbar)
      : "memory");
}
__device__ __forceinline__ void cp_async4(unsigned dst, const float* src, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(valid ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_one_pending() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// ---- host side --------------------------------------------------------------
// cuTensorMapEncodeTiled from the driver (nullptr if unavailable).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();

// Float32 tensor map of a (nx, ny, nz) cube with a (bx, by, 1) box, zero fill
// outside. False when the cube is not TMA-addressable (row pitch or base not
// 16-byte aligned) or the driver refuses.
bool encode_cube_map(CUtensorMap* map, const float* base, long long nx, long long ny, long long nz, int bx, int by);
// The same for a 16-bit cube (rows must be 16-byte multiples: nx % 8 == 0).
bool encode_cube16_map(CUtensorMap* map, const unsigned short* base, long long nx, long long ny, long long nz, int bx,
                       int by);

// Let `kernel` use all opt-in shared memory left beside its static shared memory.
template <typename K>
void set_dyn_smem_limit(K kernel) {
  cudaFuncAttributes fa{};
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) return;
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}

// Dynamic shared memory to request so that at most one block fits per SM
// (such a block holds all of its SM's TMEM).
size_t one_block_per_sm_smem(size_t need);

}  // namespace tc
}  // namespace sc
