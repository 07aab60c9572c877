// The warp-specialised smoothing kernel (sc_smooth_ws.cuh) on a cube stored
// in 16 bits (BF16 or FP16 with one float32 scale per channel): TMA brings
// the 16-bit halo'd tiles into shared memory, the producers decode each value
// with its channel's scale as they quantise it, and the consumers read the
// NaN flags from the same tiles. Same exact fixed-point arithmetic, hence the
// same floats as smoothing the decoded float32 cube; half the cube bytes.
#include "sc_smooth_ws.cuh"

namespace sc {

void init_ws16_attrs() {
  ws::set_ws_attr<1, 3, 3, 2>();
  ws::set_ws_attr<3, 5, 5, 2>();
  ws::set_ws_attr<5, 5, 5, 2>();
  ws::set_ws_attr<7, 9, 9, 2>();
}

// The cascades of FWHM 3, 5, 6 and 10 px on a 16-bit cube whose rows are
// 16-byte multiples; *done = false otherwise.
cudaError_t launch_smooth_ws16(const SmoothArgs& a, int sms, cudaStream_t s, bool* done) {
  *done = false;
  if (!a.h16.fmt || a.generic || a.pd.sampled || a.pd.wz > ws::Tile<16>::kMaxWz) return cudaSuccess;
  const int* w = a.pd.w;
  if (w[0] == 1 && w[1] == 3 && w[2] == 3) return ws::launch_ws_for_wz<1, 3, 3, 2>(a, sms, s, done);
  if (w[0] == 3 && w[1] == 5 && w[2] == 5) return ws::launch_ws_for_wz<3, 5, 5, 2>(a, sms, s, done);
  if (w[0] == 5 && w[1] == 5 && w[2] == 5) return ws::launch_ws_for_wz<5, 5, 5, 2>(a, sms, s, done);
  if (w[0] == 7 && w[1] == 9 && w[2] == 9) return ws::launch_ws_for_wz<7, 9, 9, 2>(a, sms, s, done);
  return cudaSuccess;
}

}  // namespace sc
