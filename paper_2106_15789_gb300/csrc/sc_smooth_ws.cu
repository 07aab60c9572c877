// Warp-specialised smoothing kernel (sc_smooth_ws.cuh) for the 3-box cascades
// of FWHM 3, 5, 6 and 10 px, and the host helpers of the tiled kernels.
#include <cstdint>
#include <cstring>

#include "sc_smooth_ws.cuh"

namespace sc {

// ---- host helpers of the tiled kernels ------------------------------------
namespace tc {

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    cudaGetLastError();
  }
  return fn;
}

bool encode_cube_map(CUtensorMap* map, const float* base, long long nx, long long ny, long long nz, int bx, int by) {
  memset(map, 0, sizeof(*map));
  if (nx % 4 != 0 || (reinterpret_cast<uintptr_t>(base) & 15u) != 0) return false;
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
  const cuuint64_t strides[2] = {(cuuint64_t)nx * 4, (cuuint64_t)nx * ny * 4};
  const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult cr = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return cr == CUDA_SUCCESS;
}

bool encode_cube16_map(CUtensorMap* map, const unsigned short* base, long long nx, long long ny, long long nz, int bx,
                       int by) {
  memset(map, 0, sizeof(*map));
  if (nx % 8 != 0 || (reinterpret_cast<uintptr_t>(base) & 15u) != 0 || bx % 8 != 0) return false;
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
  const cuuint64_t strides[2] = {(cuuint64_t)nx * 2, (cuuint64_t)nx * ny * 2};
  const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult cr = enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT16, 3, const_cast<unsigned short*>(base), dims, strides,
                          box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return cr == CUDA_SUCCESS;
}

size_t one_block_per_sm_smem(size_t need) {
  int dev = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  const size_t half = (size_t)per_sm / 2 + 1024;
  return need > half ? need : half;
}

}  // namespace tc

void init_ws_attrs() {
  ws::set_ws_attr<1, 3, 3>();
  ws::set_ws_attr<3, 5, 5>();
  ws::set_ws_attr<5, 5, 5>();
  ws::set_ws_attr<7, 9, 9>();
}

// Tile height of the warp-specialised kernel for a pair: 32 rows for spectral
// widths up to 15 (unless the autotuner chose 16), 16 rows up to 31, else 0.
int ws_tile_rows(const SmoothArgs& a) {
  if (a.pd.wz <= ws::Tile<32>::kMaxWz && a.tune_kind != TUNE_WS16) return 32;
  if (a.pd.wz <= ws::Tile<16>::kMaxWz) return 16;
  return 0;
}

// The warp-specialised kernel for the cascades of FWHM 3, 5, 6 and 10 px with
// spectral widths up to 31 (64 x 32 tiles up to 15, 64 x 16 tiles beyond; TMA
// loads where the cube allows them, cp.async otherwise); *done = false for
// other pairs.
cudaError_t launch_smooth_ws16(const SmoothArgs& a, int sms, cudaStream_t s, bool* done);

cudaError_t launch_smooth_ws(const SmoothArgs& a, int sms, cudaStream_t s, bool* done) {
  *done = false;
  if (a.generic || a.pd.wz > ws::Tile<16>::kMaxWz) return cudaSuccess;
  if (a.h16.fmt) return launch_smooth_ws16(a, sms, s, done);  // a 16-bit cube read as such
  const int* w = a.pd.w;
  if (w[0] == 1 && w[1] == 3 && w[2] == 3) return ws::launch_ws_for_wz<1, 3, 3>(a, sms, s, done);
  if (w[0] == 3 && w[1] == 5 && w[2] == 5) return ws::launch_ws_for_wz<3, 5, 5>(a, sms, s, done);
  if (w[0] == 5 && w[1] == 5 && w[2] == 5) return ws::launch_ws_for_wz<5, 5, 5>(a, sms, s, done);
  if (w[0] == 7 && w[1] == 9 && w[2] == 9) return ws::launch_ws_for_wz<7, 9, 9>(a, sms, s, done);
  return cudaSuccess;
}

}  // namespace sc
