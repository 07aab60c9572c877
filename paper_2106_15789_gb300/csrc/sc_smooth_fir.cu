// The warp-specialised smoothing kernel (sc_smooth_ws.cuh) with the sampled
// spatial Gaussian of a given FWHM (SoFiA 2 Sect. 5 and the Hydra-field figure
// caption of Sect. 7: a Gaussian of FWHM f px) in place of the 3-box cascade:
// the x and y passes are exact integer FIRs of the Gaussian's integer taps
// (2R + 1 of them, read from the kernel's parameters), everything else -
// quantisation, replacement, spectral ring in TMEM, NaN blanking, histogram -
// as for the cascades, so the result is the same exact fixed-point convolution
// the generic kernel computes.
//
// The half-width R is a template parameter (the tile halo): a pair of
// half-width h runs on the smallest instantiated R >= h with its taps centred
// and zero-padded to 2R + 1.
#include "sc_smooth_ws.cuh"

namespace sc {
namespace {

// Re-centre the pair's 2h + 1 taps on a support of 2R + 1 (zeros outside).
// The sampled Gaussian's taps are symmetric, as the FIR passes require.
SmoothArgs padded_taps(const SmoothArgs& a0, int R) {
  SmoothArgs a = a0;
  const int h = a0.pd.h;
  for (int i = 0; i < 2 * kMaxHalf + 1; ++i) a.pd.taps[i] = 0;
  for (int i = 0; i < 2 * h + 1; ++i) a.pd.taps[R - h + i] = a0.pd.taps[i];
  return a;
}

template <int R>
cudaError_t launch_fir(const SmoothArgs& a0, int sms, cudaStream_t s, bool* done) {
  const SmoothArgs a = padded_taps(a0, R);
  // 64 x 32 tiles for spectral widths up to 15 where the halo'd tiles fit in
  // shared memory, else 64 x 16 tiles (spectral widths up to 31)
  if (ws_tile_rows(a) == 32) {
    const cudaError_t e = ws::launch_ws<0, R, 0, 32>(a, sms, s, done);
    if (e != cudaSuccess || *done) return e;
  }
  if (a.pd.wz <= ws::Tile<16>::kMaxWz) return ws::launch_ws<0, R, 0, 16>(a, sms, s, done);
  return cudaSuccess;
}

}  // namespace

void init_fir_attrs() {
  ws::set_ws_attr<0, 4, 0>();
  ws::set_ws_attr<0, 8, 0>();
  ws::set_ws_attr<0, 9, 0>();
  ws::set_ws_attr<0, 12, 0>();
  ws::set_ws_attr<0, 16, 0>();
}

// Sampled-Gaussian pairs of half-width 1..16 (FWHM up to about 10 px) with
// spectral widths up to 31; *done = false for other pairs.
cudaError_t launch_smooth_fir(const SmoothArgs& a, int sms, cudaStream_t s, bool* done) {
  *done = false;
  if (a.generic || a.h16.fmt || !a.pd.sampled || a.pd.h < 1 || a.pd.wz > ws::Tile<16>::kMaxWz) return cudaSuccess;
  const int h = a.pd.h;
  for (int i = 0; i < h; ++i)
    if (a.pd.taps[i] != a.pd.taps[2 * h - i]) return cudaSuccess;  // not symmetric: not served
  if (h <= 4) return launch_fir<4>(a, sms, s, done);
  if (h <= 8) return launch_fir<8>(a, sms, s, done);
  if (h <= 9) return launch_fir<9>(a, sms, s, done);
  if (h <= 12) return launch_fir<12>(a, sms, s, done);
  if (h <= 16) return launch_fir<16>(a, sms, s, done);
  return cudaSuccess;
}

}  // namespace sc
