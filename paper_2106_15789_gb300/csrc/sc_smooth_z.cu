// Spectral-only smoothing (spatial FWHM 0, boxcar of wz channels), SoFiA 2
// Sect. 4.2 / 5, with the replacement of Sect. 6.2.
//
// With no spatial kernel, S(v) = (1/wz) * sum_{|d|<=r} X(v + d * plane) on the
// flattened plane, so no tiles, halos or block barriers are needed: each
// thread owns VPT consecutive voxels of the plane and walks through z, with
// the wz most recent quantised values of its voxels in Tensor Memory (the
// ring of the running sum) and the next plane's values prefetched into
// registers. Same exact fixed-point arithmetic as the other smoothing kernels,
// hence identical floats.
#include <cstdint>

#include "sc_device.cuh"
#include "sc_internal.h"
#include "sc_tile_common.cuh"

namespace sc {
namespace zonly {

constexpr int kThreads = 256;
constexpr int kTmemCols = 512;

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// 2*VPT consecutive 32-bit TMEM columns of the thread's lane <-> VPT int64.
template <int VPT>
struct Tm;
template <>
struct Tm<8> {
  static __device__ __forceinline__ void ld(unsigned t, unsigned (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(t)
        : "memory");
  }
  static __device__ __forceinline__ void st(unsigned t, const unsigned (&v)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(t),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
        "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
        : "memory");
  }
};
template <>
struct Tm<4> {
  static __device__ __forceinline__ void ld(unsigned t, unsigned (&v)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                 : "r"(t)
                 : "memory");
  }
  static __device__ __forceinline__ void st(unsigned t, const unsigned (&v)[8]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(t), "r"(v[0]),
                 "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
                 : "memory");
  }
};
template <>
struct Tm<1> {
  static __device__ __forceinline__ void ld(unsigned t, unsigned (&v)[2]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];" : "=r"(v[0]), "=r"(v[1]) : "r"(t) : "memory");
  }
  static __device__ __forceinline__ void st(unsigned t, const unsigned (&v)[2]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1,%2};" ::"r"(t), "r"(v[0]), "r"(v[1]) : "memory");
  }
};

constexpr int kDepth = 8;  // planes in flight per thread (cp.async ring in shared memory)

__device__ __forceinline__ void cp16(unsigned dst, const void* src, bool ok) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(ok ? 16 : 0) : "memory");
}
__device__ __forceinline__ void cp8(unsigned dst, const void* src, bool ok) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst), "l"(src), "r"(ok ? 8 : 0) : "memory");
}
__device__ __forceinline__ void cp4(unsigned dst, const void* src, bool ok) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(ok ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

}  // namespace zonly

// EB: bytes per cube value (4: float32; 2: a 16-bit cube, copied as such and
// decoded with its channel's scale when a thread takes its values).
template <int VPT, bool VEC, bool REPL, int THREADS, int EB = 4>
__global__ void __launch_bounds__(THREADS, 1) k_smooth_z(SmoothArgs a) {
  using namespace zonly;
  static_assert(EB == 4 || (VEC && VPT >= 4), "16-bit cubes take the vector copies");
  extern __shared__ __align__(16) unsigned char zsmem[];
  unsigned char* const zring = zsmem;  // [kDepth][THREADS * VPT] values of EB bytes
  unsigned long long* const zmask =
      reinterpret_cast<unsigned long long*>(zsmem + (size_t)EB * kDepth * THREADS * VPT);  // [kDepth][THREADS]
  unsigned int* const zhist =
      reinterpret_cast<unsigned int*>(zsmem + (size_t)EB * kDepth * THREADS * VPT + 8 * kDepth * THREADS);
  __shared__ unsigned tmem_holder;
  const int tid = threadIdx.x, warp = tid >> 5;
  if (a.hist)
    for (int i = tid; i < kNumBins; i += THREADS) zhist[i] = 0u;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_holder)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tbase = tmem_holder;
  // THREADS / 128 warp groups share the 512 columns of the four lane quarters
  constexpr int kGroupCols = kTmemCols / (THREADS / 128);
  const unsigned tmine = tbase + ((unsigned)(32 * (warp & 3)) << 16) + (unsigned)(kGroupCols * (warp >> 2));

  const BinCfg cfg = a.win ? a.st->win : kFullRange;
  const float fscale = a.st->fx_scale[a.pair];
  const float inv = a.st->fx_inv[a.pair];
  const long long qrepl = a.st->fx_qrepl[a.pair];
  const bool do_repl = REPL && qrepl > 0;
  const int wz = a.pd.wz, r = (wz - 1) / 2;
  const long long nz = a.nz, P = (long long)a.nx * a.ny, N = P * nz;
  const long long per_block = (long long)THREADS * VPT;
  const long long groups = (P + per_block - 1) / per_block;
  const long long n_items = groups * a.zchunks;
  constexpr int W = 2 * VPT;  // TMEM columns per ring slot

  for (long long item = blockIdx.x; item < n_items; item += gridDim.x) {
    const long long grp = item % groups;
    const int zc = (int)(item / groups);
    const long long p0 = grp * per_block + (long long)tid * VPT;
    const int nv = (int)(P - p0 < 0 ? 0 : (P - p0 > VPT ? VPT : P - p0));  // voxels this thread owns
    const int z0 = zc * a.lz;
    const int z1 = (int)min((long long)z0 + a.lz, nz);
    const int n_steps = (z1 - z0) + 2 * r;
    // the thread's voxels that enter the histogram (all of them but past the plane's end)
    const unsigned hist_rows = a.hist ? (nv >= VPT ? (1u << VPT) - 1u : (1u << nv) - 1u) : 0u;
    long long zsum[VPT];
#pragma unroll
    for (int i = 0; i < VPT; ++i) zsum[i] = 0;
    {
      unsigned zero[W];
#pragma unroll
      for (int i = 0; i < W; ++i) zero[i] = 0u;
      for (int s = 0; s < wz; ++s) Tm<VPT>::st(tmine + (unsigned)(W * s), zero);
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    unsigned long long nan_hist = 0ull;

    // Per-thread ring of kDepth planes in shared memory, filled by cp.async:
    // the thread's VPT values and the mask word(s) holding its bits. Each
    // thread reads back only what it copied itself, so no barrier is needed.
    unsigned char* my_vals = zring + (size_t)EB * tid * VPT;          // stage stride THREADS*VPT values
    unsigned long long* my_mask = zmask + tid;                        // stage stride THREADS
    auto issue = [&](int zp, int stage) {
      const bool zok = zp >= 0 && zp < nz;
      const long long base = (long long)zp * P + p0;
      unsigned char* dv = my_vals + (size_t)EB * stage * THREADS * VPT;
      if constexpr (EB == 2) {
        // 16-bit values: VPT of them in one 16-byte (VPT 8) or 8-byte (VPT 4)
        // copy; nv is a multiple of VPT here (the plane and p0 are)
        const bool ok = zok && nv > 0;
        const unsigned short* src = ok ? a.h16.bits + base : a.h16.bits;
        if (VPT == 8) cp16(smem_u32(dv), src, ok);
        else cp8(smem_u32(dv), src, ok);
      } else if (VEC) {
        // nv is a multiple of 4 here (the plane and p0 are), so whole quads
#pragma unroll
        for (int q = 0; q < VPT / 4; ++q) {
          const bool ok = zok && 4 * q < nv;
          cp16(smem_u32(dv + 16 * q), ok ? (const void*)(a.C + base + 4 * q) : (const void*)a.C, ok);
        }
      } else {
#pragma unroll
        for (int i = 0; i < VPT; ++i)
          cp4(smem_u32(dv + 4 * i), zok && i < nv ? (const void*)(a.C + base + i) : (const void*)a.C, zok && i < nv);
      }
      if (do_repl) {
        unsigned* dm = reinterpret_cast<unsigned*>(my_mask + (size_t)stage * THREADS);
        const long long w = base >> 5;
        const bool ok = zok && nv > 0;
        cp4(smem_u32(dm), ok ? (const void*)(a.mbits + w) : (const void*)a.mbits, ok);
        const bool ok2 = ok && ((base & 31) + VPT > 32) && (w + 1) * 32 < N;
        cp4(smem_u32(dm + 1), ok2 ? (const void*)(a.mbits + w + 1) : (const void*)a.mbits, ok2);
      }
      cp_commit();
    };
    for (int k = 0; k < kDepth - 1; ++k) issue(z0 - r + k, k);  // plane index beyond n_steps: harmless zero fill
    // a 16-bit cube: its planes' scales, loaded a plane ahead
    auto plane_scale = [&](int zq) { return (EB == 2 && zq >= 0 && zq < nz) ? __ldg(a.h16.scale + zq) : 1.0f; };
    float cs_next = plane_scale(z0 - r);
    for (int j = 0; j < n_steps; ++j) {
      const int zp = z0 - r + j;
      const float cs_plane = cs_next;
      cs_next = plane_scale(zp + 1);
      issue(zp + kDepth - 1, (j + kDepth - 1) % kDepth);
      cp_wait<kDepth - 1>();
      const int st = j % kDepth;
      float cur[VPT];
      const unsigned char* sv = my_vals + (size_t)EB * st * THREADS * VPT;
      if constexpr (EB == 2) {
        const unsigned short* sv16 = reinterpret_cast<const unsigned short*>(sv);
#pragma unroll
        for (int i = 0; i < VPT; ++i) cur[i] = half16_value(sv16[i], a.h16.fmt, cs_plane);
      } else {
        const float* svf = reinterpret_cast<const float*>(sv);
#pragma unroll
        for (int i = 0; i < VPT; ++i) cur[i] = svf[i];
      }
      unsigned mcur = 0u;
      if (do_repl && zp >= 0 && zp < nz && nv > 0) {
        const unsigned* mm = reinterpret_cast<const unsigned*>(my_mask + (size_t)st * THREADS);
        const unsigned long long two = (unsigned long long)mm[0] | ((unsigned long long)mm[1] << 32);
        const long long base = (long long)zp * P + p0;
        mcur = (unsigned)(two >> (base & 31)) & ((1u << VPT) - 1u);
        mcur &= (nv >= 32 ? 0xffffffffu : ((1u << nv) - 1u));
      }
      const unsigned ta = tmine + (unsigned)(W * (j % wz));
      unsigned old[W], nw[W];
      Tm<VPT>::ld(ta, old);
      unsigned nanbits = 0u;
      long long Pq[VPT];
#pragma unroll
      for (int i = 0; i < VPT; ++i) {
        const float c = cur[i];
        // c - c is NaN exactly for NaN and Inf, whose quantised value is then 0
        const float d = c - c;
        Pq[i] = quantize(c + d, fscale);
        nanbits |= (d != d ? 1u : 0u) << i;
      }
      if (do_repl && mcur != 0u) {  // masked voxels are finite (the working mask holds no others)
#pragma unroll
        for (int i = 0; i < VPT; ++i)
          if ((mcur >> i) & 1u) Pq[i] = cur[i] >= 0.0f ? qrepl : -qrepl;
      }
      nan_hist = (nan_hist << VPT) | nanbits;
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int i = 0; i < VPT; ++i) {
        const long long o = (long long)(((unsigned long long)old[2 * i + 1] << 32) | old[2 * i]);
        zsum[i] += Pq[i] - o;
        nw[2 * i] = (unsigned)((unsigned long long)Pq[i] & 0xffffffffull);
        nw[2 * i + 1] = (unsigned)((unsigned long long)Pq[i] >> 32);
      }
      Tm<VPT>::st(ta, nw);
      if (j >= 2 * r && nv > 0) {
        const int zo = zp - r;
        const unsigned nb = (unsigned)(nan_hist >> (VPT * r)) & ((1u << VPT) - 1u);
        const unsigned binned = hist_rows & ~nb;  // finite voxels of the thread's own, when histogrammed
        float s[VPT];
#pragma unroll
        for (int i = 0; i < VPT; ++i) {
          const bool isn = (nb >> i) & 1u;
          const float sv = dequantize(zsum[i], inv);
          s[i] = isn ? __int_as_float(0x7fc00000) : sv;
          if ((binned >> i) & 1u) atomicAdd(&zhist[bin_of(s[i], cfg)], 1u);
        }
        float* out = a.S + (long long)zo * P + p0;
        if (VEC) {
#pragma unroll
          for (int q = 0; q < VPT / 4; ++q)
            if (4 * q < nv)
              reinterpret_cast<float4*>(out)[q] = make_float4(s[4 * q], s[4 * q + 1], s[4 * q + 2], s[4 * q + 3]);
        } else {
#pragma unroll
          for (int i = 0; i < VPT; ++i)
            if (i < nv) out[i] = s[i];
        }
      }
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    cp_wait<0>();  // drain the copies issued past the item's last plane
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(kTmemCols) : "memory");
  if (a.hist)
    for (int i = tid; i < kNumBins; i += THREADS)
      if (zhist[i]) atomicAdd(a.hist + i, (unsigned long long)zhist[i]);
}

namespace {


template <int VPT, bool VEC, bool REPL, int THREADS, int EB = 4>
void set_z_attr() {
  cudaFuncAttributes fa{};
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (cudaFuncGetAttributes(&fa, k_smooth_z<VPT, VEC, REPL, THREADS, EB>) != cudaSuccess) return;
  cudaFuncSetAttribute(k_smooth_z<VPT, VEC, REPL, THREADS, EB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       optin - (int)fa.sharedSizeBytes);
}

template <int VPT, int THREADS = zonly::kThreads>
void set_z_attrs() {
  set_z_attr<VPT, false, false, THREADS>();
  set_z_attr<VPT, false, true, THREADS>();
  set_z_attr<VPT, true, false, THREADS>();
  set_z_attr<VPT, true, true, THREADS>();
  if constexpr (VPT >= 4) {
    set_z_attr<VPT, true, false, THREADS, 2>();
    set_z_attr<VPT, true, true, THREADS, 2>();
  }
}

template <int VPT, bool VEC, bool REPL, int THREADS, int EB = 4>
cudaError_t launch_z(const SmoothArgs& a0, int sms, cudaStream_t s) {
  SmoothArgs a = a0;
  const long long P = (long long)a.nx * a.ny;
  const long long per_block = (long long)THREADS * VPT;
  const long long groups = (P + per_block - 1) / per_block;
  const long long zch = z_chunks(a, groups, sms, (a.nz + 15) / 16);
  a.lz = (int)((a.nz + zch - 1) / zch);
  a.zchunks = (a.nz + a.lz - 1) / a.lz;
  const long long items = groups * a.zchunks;
  const int grid = (int)(items < sms ? items : sms);
  // one block per SM (it holds all of the SM's TMEM): request more than half
  // of the shared memory
  const size_t need = (size_t)EB * zonly::kDepth * THREADS * VPT + 8 * zonly::kDepth * THREADS +
                      (a.hist ? sizeof(unsigned) * kNumBins : 0);
  const size_t smem = tc::one_block_per_sm_smem(need);
  k_smooth_z<VPT, VEC, REPL, THREADS, EB><<<grid, THREADS, smem, s>>>(a);
  return cudaGetLastError();
}

template <int VPT, int THREADS = zonly::kThreads>
cudaError_t launch_z_vpt(const SmoothArgs& a, int sms, cudaStream_t s) {
  if constexpr (VPT >= 4) {
    if (a.h16.fmt) {  // the caller checked z16_ok
      const bool repl = a.mbits != nullptr && a.repl_possible;
      return repl ? launch_z<VPT, true, true, THREADS, 2>(a, sms, s) : launch_z<VPT, true, false, THREADS, 2>(a, sms, s);
    }
  }
  const bool vec = VPT >= 4 && ((long long)a.nx * a.ny) % 4 == 0 && (reinterpret_cast<uintptr_t>(a.C) & 15u) == 0 &&
                   (reinterpret_cast<uintptr_t>(a.S) & 15u) == 0;
  const bool repl = a.mbits != nullptr && a.repl_possible;
  if (vec) return repl ? launch_z<VPT, true, true, THREADS>(a, sms, s) : launch_z<VPT, true, false, THREADS>(a, sms, s);
  return repl ? launch_z<VPT, false, true, THREADS>(a, sms, s) : launch_z<VPT, false, false, THREADS>(a, sms, s);
}

}  // namespace

void init_z_attrs() {
  set_z_attrs<8, 512>();
  set_z_attrs<4, 512>();
  set_z_attrs<8>();
  set_z_attrs<4>();
  set_z_attrs<1>();
}

// Spectral-only pairs (no spatial smoothing, boxcar up to 127 channels).
// A 16-bit cube takes 16- and 8-byte copies of 8 and 4 values: its planes
// must be multiples of 8 values, its base and S 16-byte aligned, and the
// boxcar at most 31 (the forms with 4 or 8 values per thread).
bool z16_ok(const SmoothArgs& a) {
  return ((long long)a.nx * a.ny) % 8 == 0 && (reinterpret_cast<uintptr_t>(a.h16.bits) & 15u) == 0 &&
         (reinterpret_cast<uintptr_t>(a.S) & 15u) == 0 && a.pd.wz <= 31;
}

cudaError_t launch_smooth_z(const SmoothArgs& a, int sms, cudaStream_t s, bool* done) {
  *done = false;
  if (a.generic || a.pd.h != 0 || a.pd.wz <= 1) return cudaSuccess;
  if (a.h16.fmt && !z16_ok(a)) return cudaSuccess;
  *done = true;
  if (a.tune_kind == TUNE_Z4 && a.pd.wz <= 31) return launch_z_vpt<4>(a, sms, s);
  // 512 threads of 4 voxels: twice the warps per scheduler, a 16-slot ring
  if (a.tune_kind == TUNE_Z4W && a.pd.wz <= 15) return launch_z_vpt<4, 512>(a, sms, s);
  // 512 threads of 8 voxels: as many warps, 8 ring slots
  if (a.tune_kind == TUNE_Z8W && a.pd.wz <= 7) return launch_z_vpt<8, 512>(a, sms, s);
  if (a.pd.wz <= 15) return launch_z_vpt<8>(a, sms, s);
  if (a.pd.wz <= 31) return launch_z_vpt<4>(a, sms, s);
  return launch_z_vpt<1>(a, sms, s);
}

}  // namespace sc
