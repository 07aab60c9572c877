// Internal declarations shared by the host library and its CUDA kernels.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "sc.h"

namespace sc {

// ---------------------------------------------------------------------------
// Value histogram used by the exact median / MAD selection.
//
// Bins follow the float's own bits: per sign, an underflow bin, E exponents
// of 2^MB mantissa sub-bins each (E << MB == 4096), and an overflow bin.
// Negative values map below positive ones, so the bin index is monotone in
// the value. The full-range layout (e_base 0, E 256, MB 4) needs no prior
// knowledge of the data; the windowed one (E 32, MB 7) centres 32 octaves on
// the raw cube's noise level for 8x finer bins where the order statistics lie.
constexpr int kBinsPerSign = 4096 + 2;
constexpr int kNumBins = 2 * kBinsPerSign;

struct BinCfg {
  int e_base;  // first exponent field value with its own bins
  int E;       // number of exponents with their own bins
  int MB;      // mantissa bits per exponent (E << MB == 4096)
};

constexpr BinCfg kFullRange = {0, 256, 4};
constexpr int kWindowE = 32, kWindowMB = 7, kWindowBelow = 20;  // window [2^-20, 2^12) x sigma_0

// ---------------------------------------------------------------------------
// Radix selection of one order statistic among candidate values.
// digits of 11, 11 and 10 bits, from the top of the 32-bit key
__host__ __device__ constexpr int sel_bits(int r) { return r < 2 ? 11 : 10; }
__host__ __device__ constexpr int sel_shift(int r) { return r == 0 ? 21 : (r == 1 ? 10 : 0); }  // key >> shift after round r
constexpr int kSelBins = 2048;

enum SelMode : int { SEL_VALUE = 0, SEL_ABSDEV = 1 };

struct SelJob {
  const float* list;              // candidate values (or the whole array in full mode)
  unsigned long long count_fixed; // element count when count_ptr is null
  unsigned long long* count_ptr;  // element count filled in by the candidate pass
  int mode;                       // SEL_VALUE: key(s); SEL_ABSDEV: key(|s - m|)
  int pad;
  unsigned long long rank_lo;     // order statistics wanted, relative to the list
  unsigned long long rank_hi;
  unsigned int prefix[4];         // key prefix after each round (prefix[0] unused)
  unsigned long long rank_in[4];  // remaining rank of rank_lo inside the prefix
  unsigned long long hist[3][kSelBins];
  unsigned long long c_le;        // elements with key <= key_lo
  unsigned int min_gt;            // smallest key > key_lo
  unsigned int key_lo;
};

// ---------------------------------------------------------------------------
// Plan of one noise measurement, written by k_plan from the value histogram.
enum PlanFlags : int {
  PLAN_EMPTY = 1,      // no finite value
  PLAN_MED_FULL = 2,   // median candidates above capacity: select over the whole array
  PLAN_MAD_FULL = 4,   // MAD candidates above capacity (or no bracket): whole array
  PLAN_CLIP = 8,       // this measurement also clips into the mask
  PLAN_CLIP_FULL = 16, // clip needs its own pass after sigma is known
  PLAN_STD = 32,       // STD noise mode
};

struct NoisePlan {
  unsigned long long n;           // finite values
  unsigned long long k_lo, k_hi;  // median / MAD order statistics (0-based)
  unsigned long long below_med;   // values in bins below the median bins
  int b_med_lo, b_med_hi;         // bins holding the two middle values
  int flags;
  int has_B;
  float B_lo, B_hi;  // s in [B_lo, B_hi]  =>  |s - m| <= T1 < MAD for sure
  float A_lo, A_hi;  // s < A_lo or > A_hi =>  |s - m| >  T2 > MAD for sure
  float thr_lo, thr_hi;  // |S| > thr_hi: detected for sure; |S| <= thr_lo: not detected
  float threshold;       // t
  float T1, T2;
  unsigned long long bound_med, bound_mad, bound_amb;  // candidate counts bounds from the histogram
  int bA_lo, bA_hi;        // bins that may hold MAD candidates
  int bB_lo, bB_hi;        // bins surely inside the MAD band (empty if bB_lo > bB_hi)
  unsigned long long n_B;  // values in those bins
};

// Device-resident state of one sc_run (one context owns one).
struct DevState {
  unsigned int status;   // SC_ST_* error bits
  unsigned int warn;     // SC_WARN_* bits
  float sigma0;          // noise of the raw cube
  float repl;            // n * sigma0 (0: replacement off)
  unsigned int maxabs_bits;  // max |C| over finite voxels (float bits; monotone for >= 0)
  double m;              // median of the current measurement (exact: mean of two floats)
  double mad;            // MAD of the current measurement
  float sigma_cur;       // sigma of the current measurement
  double sigma_cur_d;    // the same before rounding to float
  double repl_d;         // n * sigma0 in float64 (replacement value)
  BinCfg win;            // windowed bin layout for smoothed cubes
  double sum, sum2;      // STD mode accumulators
  unsigned long long count;
  // counters filled by the candidate pass
  unsigned long long n_cand_med, n_cand_mad, n_amb, n_below;
  NoisePlan plan;
  SelJob sel_med, sel_mad;
  // fixed-point smoothing scale of every pair
  int fx_shift[SC_MAX_KERNELS];      // f: X_q = rint(X * 2^f)
  float fx_scale[SC_MAX_KERNELS];    // 2^f
  float fx_inv[SC_MAX_KERNELS];      // 2^-f / W (W = integer weight total of the pair)
  long long fx_qrepl[SC_MAX_KERNELS];  // rint(repl_d * 2^f): replaced voxels in fixed point
  float sigma[SC_MAX_KERNELS + 1];   // per pair; [SC_MAX_KERNELS] = scratch for sc_noise
};

enum StatusBits : unsigned int {
  SC_ST_ALLNAN = 1u,
  SC_ST_INTERNAL = 2u,
  SC_ST_OVERFLOW = 4u,
  SC_ST_TIMEOUT = 8u,   // a bounded device-side wait gave up
};

struct Caps {
  unsigned long long med, mad, amb;
};

constexpr size_t kClassTableBytes = 1 << 16;  // one byte per 16-bit cell of the float encoding

// Candidate lists owned by the context.
struct Lists {
  float* med;
  float* mad;
  unsigned long long* amb;
  unsigned char* cls;  // 65536-byte class table written by the plan (16-byte aligned)
  Caps cap;
};

// ---------------------------------------------------------------------------
// Smoothing of one kernel pair.
constexpr int kMaxHalf = 40;    // largest spatial half-width (sum of (w-1)/2)
constexpr int kMaxBoxcar = 127; // largest spectral boxcar

// Spectral widths up to this share one fixed-point scale per spatial kernel
// (so that the pairs of one spatial kernel can share its spatial passes).
constexpr int kShareMaxWz = 31;
constexpr int kGaussTapUnit = 1024;  // central tap of the sampled Gaussian: taps are in its 1/1024 units

struct PairDesc {
  int w[3];       // spatial cascade widths (1 = identity; 0 = not a cascade: sampled Gaussian)
  int h;          // spatial half-width
  int wz;         // spectral width (1 = identity)
  int sampled;    // 1: the spatial kernel is the sampled Gaussian (taps below), not a cascade
  long long W;    // integer weight total T^2 * wz, T = sum of the 1-D taps (w0 w1 w2 for a cascade)
  long long Wf;   // weight bound fixing the scale: T^2 * max(wz, kShareMaxWz)
  int taps[2 * kMaxHalf + 1];  // composed integer kernel, 2h+1 taps, sum T
};

struct PairWeights {
  long long w[SC_MAX_KERNELS];   // integer weight total of every pair (passed by value to kernels)
  long long wf[SC_MAX_KERNELS];  // the bound that fixes each pair's fixed-point scale
};

// A cube stored in 16 bits (SC_STORE_BF16 / SC_STORE_FP16) with one float32
// scale per channel, read as such by the kernels: value = fl32(v * scale[z]).
struct Half16 {
  const unsigned short* bits;  // [nz][ny][nx]
  const float* scale;          // [nz]
  int fmt;                     // 0: no 16-bit cube; SC_STORE_BF16 or SC_STORE_FP16
};

struct SmoothArgs {
  const float* C;         // float32 cube (null when h16.fmt != 0)
  Half16 h16;             // the cube in its 16-bit form (fmt 0: C is the cube)
  const uint32_t* mbits;  // working mask, 1 bit per voxel, flat order (may be null: empty)
  float* S;
  int nx, ny, nz;
  int pair;               // index into DevState fixed-point arrays
  int use_fixed_repl;     // 1: replacement value below instead of DevState::repl
  int repl_possible;      // 0: replacement is off for this pair (skip the mask entirely)
  float repl_value;
  DevState* st;
  unsigned long long* hist;  // null: no histogram
  int win;                   // 1: windowed bins (DevState::win), 0: full range
  PairDesc pd;
  int tx, ty, lz;            // tile and z-chunk sizes
  int tiles_x, tiles_y, zchunks;
  int generic;               // force the generic FIR path
  int tune_kind;             // TUNE_* kernel choice (TUNE_AUTO: the dispatcher decides)
  int tune_zfactor;          // work items per SM targeted by the z chunking (0: the balance model)
  // Shared spatial passes (warp-specialised kernel only): when pout is set,
  // the kernel also stores the spatial sum P of X_q at every voxel (row pitch
  // ppitch elements) and the nonfinite flags of C in nfout, a byte per column
  // and 8 rows (bit y % 8 of byte [(z ceil(ny/8) + y/8) nfpitch + x]).
  long long* pout;
  long long ppitch;
  unsigned char* nfout;
  long long nfpitch;
  const unsigned* gate;      // non-null: the kernel runs only if *gate != 0
  // Test hook of the warp-specialised kernel (0: off): producer warp 0 skips
  // its hand-off of the block's second plane, and every wait is limited to
  // 1 ms, so that a consumer's bounded wait runs out (SC_ST_TIMEOUT).
  int test_skip_handoff;
};

// ---------------------------------------------------------------------------
// Shared spatial passes (sc_smooth_p.cu). For the later pairs of a run of
// pairs with one spatial kernel, S comes from the stored P' of the run's
// first pair plus the corrections of voxels masked since then.
struct ShareState {
  unsigned long long total;      // correction entries of the current pair
  unsigned overflow;             // 1: more entries than the list holds (the full kernel runs)
  unsigned pad;
  unsigned long long next_item;  // work-item counter of the shared pass (zero before each pair)
};

struct ShareArgs {
  long long* P;              // spatial sums of the run's first pair, [nz][ny][pitch]
  long long pitch;
  const unsigned char* nf;   // nonfinite flags, [nz][ceil(ny/8)][nfpitch] bytes (bit y % 8)
  long long nfpitch;         // bytes per row of bytes (a multiple of 16 for TMA)
  const uint32_t* msnap;     // working mask when P' was made
  unsigned* cnt;             // [n_buckets + 1] per-bucket counts (all zero between pairs)
  unsigned* offs;            // [n_buckets + 1] exclusive scan of cnt (offs[n_buckets] = total); null: no corrections
  unsigned long long* bsum;  // block sums of the scan
  unsigned long long* ent;   // entries: low 16 bits (hy << 8 | hx) in the halo'd tile, high 32 the cube value's bits
  unsigned long long cap;    // entry capacity (the buffer holds cap + 2)
  ShareState* ss;
  int ty;                    // tile height of the buckets and of k_smooth_p (32 or 16)
  int tiles_x, tiles_y;
  long long n_buckets;       // tiles_x * tiles_y * nz
};

// Tile height (32 or 16) of the shared-pass kernel for a spectral width, 0 if none.
int share_tile_rows(int wz);
// True if a pair's spatial passes can be stored for / taken from another pair.
bool share_supported(const PairDesc& pd);
// Per-pair correction lists: counts, scan and fill (with R = the pair's spatial half-width).
cudaError_t launch_share_prep(const SmoothArgs& a, const ShareArgs& sh, int sms, cudaStream_t s);
// The spectral pass over P' with the corrections; *done = false if it does not serve the pair.
cudaError_t launch_smooth_p(const SmoothArgs& a, const ShareArgs& sh, int sms, cudaStream_t s, bool* done);
void init_share_attrs();

// Kernel choices the autotuner may fix for a (dims, kernel pair).
enum TuneKind : int {
  TUNE_AUTO = 0,     // the dispatcher decides
  TUNE_WS = 1,       // warp-specialised kernel, default tile height
  TUNE_TILE = 2,     // single-group tile kernel
  TUNE_GENERIC = 3,  // generic FIR kernel
  TUNE_Z8 = 4,       // spectral-only kernel, 8 voxels per thread
  TUNE_Z4 = 5,       // spectral-only kernel, 4 voxels per thread
  TUNE_WS16 = 6,     // warp-specialised kernel with 64 x 16 tiles
  TUNE_Z4W = 7,      // spectral-only kernel, 4 voxels per thread, 512 threads per block
  TUNE_Z8W = 8       // spectral-only kernel, 8 voxels per thread, 512 threads per block (boxcars up to 7)
};
static_assert(TUNE_WS == SC_VARIANT_WS && TUNE_TILE == SC_VARIANT_TILE && TUNE_GENERIC == SC_VARIANT_GENERIC &&
                  TUNE_Z8 == SC_VARIANT_Z8 && TUNE_Z4 == SC_VARIANT_Z4 && TUNE_WS16 == SC_VARIANT_WS16 &&
                  TUNE_Z4W == SC_VARIANT_Z4_512 && TUNE_Z8W == SC_VARIANT_Z8_512,
              "the public variant codes are the tuning kinds");
// Z chunks of the (tiles x chunks) work items that the blocks of a smoothing
// kernel take round-robin (at most max_ch chunks). An autotuner factor asks
// for about that many items per SM; without one, the chunking whose busiest
// block streams the fewest planes: ceil(items / blocks) items of lz planes
// plus the 2r halo planes of the spectral boxcar each.
inline long long z_chunks(const SmoothArgs& a, long long tiles, int sms, long long max_ch) {
  max_ch = max_ch < 1 ? 1 : max_ch;
  if (a.tune_zfactor > 0) {
    const long long zch = (a.tune_zfactor * sms + tiles - 1) / tiles;
    return zch < 1 ? 1 : (zch > max_ch ? max_ch : zch);
  }
  const long long nz = a.nz, r = a.pd.wz > 1 ? (a.pd.wz - 1) / 2 : 0;
  long long best = 1, best_cost = -1;
  for (long long zch = 1; zch <= max_ch && zch <= 64; ++zch) {
    const long long lz = (nz + zch - 1) / zch, chunks = (nz + lz - 1) / lz;
    const long long items = tiles * chunks, blocks = items < sms ? items : sms;
    const long long cost = (items + blocks - 1) / blocks * (lz + 2 * r);
    if (best_cost < 0 || cost < best_cost) {
      best = zch;
      best_cost = cost;
    }
  }
  return best;
}

// ---------------------------------------------------------------------------
// Launchers (all enqueue on `s`, return cudaError_t of the launch).
cudaError_t launch_hist(const float* x, long long n, DevState* st, unsigned long long* hist, int win,
                        int want_maxabs, int sms, cudaStream_t s);
// Histogram (and max) of a 16-bit cube, decoding it into out (if non-null).
cudaError_t launch_hist16(const Half16& h, long long plane, long long n, DevState* st, unsigned long long* hist,
                          int win, int want_maxabs, float* out, int sms, cudaStream_t s);
cudaError_t launch_plan(DevState* st, const unsigned long long* hist, int win, const float* src, long long n_total,
                        Lists L, float threshold, int clip, int std_mode, unsigned int force_flags, cudaStream_t s);
cudaError_t launch_pass2(const float* src, long long n, uint32_t* mbits, DevState* st, Lists L, int sms,
                         cudaStream_t s);
// which: 0 median (result in DevState::m), 1 MAD (DevState::mad, sigma_cur, sigma[pair] if pair >= 0)
cudaError_t launch_select(DevState* st, int which, int pair, int sms, cudaStream_t s);
cudaError_t launch_resolve(const float* src, uint32_t* mbits, DevState* st, Lists L, int sms, cudaStream_t s);
cudaError_t launch_clip_full(const float* src, long long n, uint32_t* mbits, DevState* st, int sms,
                             cudaStream_t s);
cudaError_t launch_std(const float* src, long long n, DevState* st, int sms, cudaStream_t s);
cudaError_t launch_std_final(DevState* st, int pair, cudaStream_t s);
// Gaussian-fit noise (after the MAD measurement of the same array): the
// 256-bin histogram over +-5 MAD noises into ghist[256], then the fit, which
// replaces sigma_cur (and sigma[pair] for pair >= 0) and, with clip, marks the
// plan for a full clip pass.
constexpr int kGaussBins = 256;
cudaError_t launch_gauss_hist(const float* src, long long n, const DevState* st, unsigned long long* ghist, int sms,
                              cudaStream_t s);
cudaError_t launch_gauss_fit(DevState* st, const unsigned long long* ghist, int pair, int clip, cudaStream_t s);
// DevState::win from the full-range histogram of a raw cube (median of |x|)
// Window of the raw cube's fine histogram from an even sample of its values
// (the 16-bit cube when h16 is non-null, else x).
cudaError_t launch_window_from_sample(const float* x, const Half16* h16, long long plane, long long n, DevState* st,
                                      cudaStream_t s);
cudaError_t launch_sigma0_done(DevState* st, float replacement, const PairWeights& W, int n_pairs,
                               cudaStream_t s);
// out[0..n-1] = sigma_k, out[n] = sigma_0, or zeros after a device-side error
cudaError_t launch_sigma_out(const DevState* st, int n, float* out, cudaStream_t s);
cudaError_t launch_fx_setup(DevState* st, float repl_value, const PairWeights& W, int n_pairs, cudaStream_t s);
cudaError_t launch_pack(const uint8_t* m8, const float* cube, long long n, uint32_t* mbits, cudaStream_t s);
cudaError_t launch_pack16(const uint8_t* m8, const Half16& h, long long plane, long long n, uint32_t* mbits,
                          cudaStream_t s);
cudaError_t launch_expand(const uint32_t* mbits, long long n, uint8_t* m8, int keep, cudaStream_t s);
cudaError_t launch_maxabs(const float* x, long long n, DevState* st, int sms, cudaStream_t s);
// out[i] = float(x[i]) * scale[i / plane], x BF16 (bf16 != 0) or FP16 bits
cudaError_t launch_decode_half(const uint16_t* x, const float* scale, long long plane, long long n, int bf16,
                               float* out, int sms, cudaStream_t s);
// x[i] = uniform pseudo-random value in [-1, 1) from (i, seed) (autotuning input)
cudaError_t launch_fill_noise(float* x, long long n, unsigned int seed, int sms, cudaStream_t s);
// Launch the smoothing kernel of a pair; adds the launches to *launches and
// stores the SC_KERNEL_* code of the kernel that ran in *kernel (either may
// be null).
cudaError_t launch_smooth(const SmoothArgs& a, int sms, cudaStream_t s, int* launches, int* kernel = nullptr);
cudaError_t launch_identity(const SmoothArgs& a, int sms, cudaStream_t s);
// Tile height (32 or 16) of the warp-specialised kernel for a pair, 0 if none.
int ws_tile_rows(const SmoothArgs& a);

// Local noise normalisation: the noise of every cell's window (sig_dev,
// rinv_dev = float 1 / sigma or NaN, one per cell), then out = cube * rinv.
constexpr long long kNoiseScaleMaxWindow = 47104;  // window voxels held in shared memory
cudaError_t launch_noise_window(const float* cube, const long long dims[3], const int window[3], const int grid[3],
                                int noise_mode, double* sig_dev, float* rinv_dev, int sms, cudaStream_t s);
cudaError_t launch_noise_apply(const float* cube, const long long dims[3], const int window[3], const int grid[3],
                               float* out, const float* rinv_dev, int sms, cudaStream_t s);
void init_noise_scale_attrs();

// Linker: components (lab = roots; chunk_off = exclusive scan of the roots
// per chunk; *d_total = their number), then ids in raster order of the first
// voxels with extents, and the size filters (lab renumbered, ext_out = kept
// rows, *d_total = kept). ext etc. may be null when there is no component.
// Auto-flagger: channel and pixel noises, their median / RMS (stats[0..1]
// channels, [2..3] pixels), flags and the blanked cube.
constexpr int kFlagMaxChannelsForPixels = 1536;  // spectra staged in shared memory
cudaError_t launch_autoflag(const float* cube, const long long dims[3], double k, int channels, int pixels,
                            int noise_mode, float* out, float* chan_noise, float* pix_noise, uint8_t* chan_flags,
                            uint8_t* pix_flags, double* stats, int sms, cudaStream_t s);

constexpr int kLinkMaxRadius = 32;  // merging radii in voxels
long long link_chunks(long long n);
cudaError_t launch_link_components(const uint8_t* mask, const long long dims[3], int r_xy, int r_z, int* lab,
                                   int* chunk_off, int* d_total, int sms, cudaStream_t s);
cudaError_t launch_link_filter(const long long dims[3], int* lab, int* chunk_off, int ncomp, int min_xy, int min_z,
                               int max_xy, int max_z, int* ext, int* keep, int* ext_out, int* new_id, int* d_total,
                               int sms, cudaStream_t s);

// Host helpers.
int cascade_widths(double fwhm, int w[3]);
// Integer taps of the sampled Gaussian of this FWHM (2h+1 of them, h =
// floor(4 sigma)); returns 2h+1, or -1 if more than max_taps would be needed.
int gauss_taps(double fwhm, int* taps, int max_taps);
int make_pair(const sc_kernel& k, PairDesc* pd, bool sampled = false);
void choose_tiles(SmoothArgs* a);
size_t smooth_smem_bytes(const SmoothArgs& a);

}  // namespace sc
