// sc_noise_static: the noise measurement of sc_noise without any allocation.
//
// Some callers cannot allocate device memory at the time they need a noise
// level: processes whose device memory is owned by another allocator or a
// fixed pool, real-time pipelines that forbid allocation (and its implicit
// device synchronisation) once they are running, or plug-ins that are handed
// only a stream and buffers. For them this entry point keeps all of its
// scratch (measurement state, value histogram, candidate lists) in one
// file-scope device array that exists on every GPU that loads this library,
// from load until process exit. Nothing is allocated or freed per call.
//
// Limits and sharing: at most kStaticMaxValues input values per call. All
// calls on a device share the one scratch array and leave their contents in
// it; every call clears what must start at zero, but calls that overlap on the
// GPU (other streams, other host threads) race on it and must be serialised
// by the caller.
#include <cstring>
#include <mutex>

#include "sc_internal.h"

namespace sc {
void init_kernel_attrs();
}

using namespace sc;

namespace {

constexpr long long kStaticMaxValues = 1LL << 22;               // 4 Mi values (16 MiB of float32 input)
constexpr unsigned long long kStaticCapMed = 1ull << 16;        // median candidates
constexpr unsigned long long kStaticCapMad = 1ull << 19;        // MAD candidates (full-range bins: <= ~6 %)
constexpr size_t kAlign = 256;
constexpr size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }
constexpr size_t kOffState = 0;
constexpr size_t kOffHist = align_up(kOffState + sizeof(DevState));
constexpr size_t kOffMed = align_up(kOffHist + sizeof(unsigned long long) * kNumBins);
constexpr size_t kOffMad = align_up(kOffMed + sizeof(float) * kStaticCapMed);
constexpr size_t kOffCls = align_up(kOffMad + sizeof(float) * kStaticCapMad);
constexpr size_t kOffGHist = align_up(kOffCls + kClassTableBytes);
constexpr size_t kStaticBytes = align_up(kOffGHist + sizeof(unsigned long long) * kGaussBins);

// The scratch itself. In host code this name is a host-side stand-in, not a
// device address: only the pointer from cudaGetSymbolAddress goes to kernels.
static __device__ __align__(256) unsigned char g_noise_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch on the current device (set up once per device).
int scratch_for_current_device(unsigned char** out, int* sms) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SC_ERR_CUDA;
  if (cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return SC_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noise_scratch) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return SC_ERR_CUDA;
    }
    init_kernel_attrs();
    g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_ptr[dev];
  return SC_OK;
}

#define CKS(x)                                 \
  do {                                         \
    if ((x) != cudaSuccess) return SC_ERR_CUDA; \
  } while (0)

}  // namespace

extern "C" int sc_noise_static(const float* data_dev, int64_t n, int noise_mode, double* sigma_host,
                               void* cuda_stream) {
  if (!data_dev || !sigma_host || n <= 0) return SC_ERR_ARG;
  if (n > kStaticMaxValues) return SC_ERR_BUDGET;
  if (noise_mode != SC_NOISE_MAD && noise_mode != SC_NOISE_STD && noise_mode != SC_NOISE_GAUSS) return SC_ERR_ARG;
  unsigned char* base = nullptr;
  int sms = 0;
  int rc = scratch_for_current_device(&base, &sms);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  DevState* st = reinterpret_cast<DevState*>(base + kOffState);
  unsigned long long* hist = reinterpret_cast<unsigned long long*>(base + kOffHist);
  Lists L{};
  L.med = reinterpret_cast<float*>(base + kOffMed);
  L.mad = reinterpret_cast<float*>(base + kOffMad);
  L.amb = nullptr;
  L.cls = base + kOffCls;
  L.cap = Caps{kStaticCapMed, kStaticCapMad, 0ull};
  const int std_mode = (noise_mode == SC_NOISE_STD);
  // the previous call's contents stay in the array: clear state and histogram
  CKS(cudaMemsetAsync(st, 0, sizeof(DevState), s));
  CKS(cudaMemsetAsync(hist, 0, sizeof(unsigned long long) * kNumBins, s));
  CKS(launch_hist(data_dev, n, st, hist, 0, 0, sms, s));
  CKS(launch_plan(st, hist, 0, data_dev, n, L, 1.0f, 0, std_mode, 0u, s));
  if (std_mode) {
    CKS(launch_std(data_dev, n, st, sms, s));
    CKS(launch_std_final(st, SC_MAX_KERNELS, s));
  } else {
    CKS(launch_pass2(data_dev, n, nullptr, st, L, sms, s));
    CKS(launch_select(st, 0, -1, sms, s));
    CKS(launch_select(st, 1, SC_MAX_KERNELS, sms, s));
  }
  if (noise_mode == SC_NOISE_GAUSS) {
    unsigned long long* ghist = reinterpret_cast<unsigned long long*>(base + kOffGHist);
    CKS(launch_gauss_hist(data_dev, n, st, ghist, sms, s));
    CKS(launch_gauss_fit(st, ghist, SC_MAX_KERNELS, 0, s));
  }
  unsigned int status = 0u;
  float sigma = 0.0f;
  CKS(cudaMemcpyAsync(&status, reinterpret_cast<unsigned char*>(st) + offsetof(DevState, status), sizeof(status),
                      cudaMemcpyDeviceToHost, s));
  CKS(cudaMemcpyAsync(&sigma, reinterpret_cast<unsigned char*>(st) + offsetof(DevState, sigma_cur), sizeof(sigma),
                      cudaMemcpyDeviceToHost, s));
  CKS(cudaStreamSynchronize(s));
  if (status & SC_ST_ALLNAN) return SC_ERR_ALLNAN;
  if (status & (SC_ST_INTERNAL | SC_ST_OVERFLOW)) return SC_ERR_INTERNAL;
  *sigma_host = (double)sigma;
  return SC_OK;
}
