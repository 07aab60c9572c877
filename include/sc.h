/*
 * sc.h - C ABI of the GB300 smooth-and-clip (S+C) source finder.
 *
 * S+C is the default source finder of SoFiA 2 (Westmeier et al. 2021,
 * arXiv:2106.15789, Sect. 4.2): the data cube is smoothed on several spatial
 * (Gaussian, FWHM in pixels) and spectral (boxcar, channels) scales; on each
 * scale the noise sigma of the smoothed cube is measured and every voxel with
 * |S| > t*sigma, positive or negative, is added to one 8-bit source mask.
 * Voxels already in the mask are set to +-n*sigma_0 (sign kept) before each
 * smoothing (Sect. 6.2, "Integrated flux"). NaN voxels are blanked.
 *
 * Conventions of every entry point
 *   - Cubes are float32, C-contiguous, axis order [z][y][x] with x fastest
 *     (FITS order, Sect. 4.1). dims[3] = {nx, ny, nz}, all > 0.
 *   - "_dev" pointers are CUDA device pointers on the context's device, owned
 *     by the caller; "_host" pointers are host memory owned by the caller.
 *     The library never frees caller memory.
 *   - All GPU work is enqueued on the caller's stream (cudaStream_t passed as
 *     void*; NULL = legacy default stream). Calls that return sigma values to
 *     the host synchronise that stream once, at the end.
 *   - Every call returns SC_OK (0) or a negative SC_ERR_* code; nothing
 *     aborts, traps or prints. sc_strerror() names a code.
 *   - A context is not thread-safe: one host thread per context at a time.
 *     Calls on one context share its workspace, so calls on different streams
 *     of one context must not overlap.
 */
#ifndef SC_H
#define SC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define SC_OK 0
#define SC_ERR_ARG (-1)         /* invalid argument (dims, kernel, threshold, NULL pointer, size) */
#define SC_ERR_NOMEM (-2)       /* device or pinned-host allocation failed */
#define SC_ERR_CUDA (-3)        /* a CUDA runtime call or kernel launch failed */
#define SC_ERR_ALLNAN (-4)      /* the cube has no finite voxel: no noise level exists */
#define SC_ERR_TIMEOUT (-5)     /* a bounded device-side wait gave up */
#define SC_ERR_UNSUPPORTED (-6) /* option outside what the kernels serve (window, spectrum or boxcar too large) */
#define SC_ERR_BUDGET (-7)      /* request exceeds the context's sizes / memory budget */
#define SC_ERR_INTERNAL (-8)    /* a device-side consistency check failed */

/* ---- noise estimators (Sect. 4.1: robust RMS from the MAD) ------------ */
#define SC_NOISE_MAD 0   /* 1.4826 * median(|S - median(S)|), exact medians */
#define SC_NOISE_STD 1   /* sqrt(sum((S - mean)^2) / (n - 1)) */
#define SC_NOISE_GAUSS 2 /* width of the least-squares Gaussian through a histogram of S (below) */

/* SC_NOISE_GAUSS is the library's own definition (the paper names no such
 * estimator). With sigma_M the MAD noise and k = fl32(128 / (5 sigma_M)),
 * every finite value s goes to bin floor(fl32(s * k)) + 128 when that lies in
 * [0, 256). A Gaussian A exp(-xi^2 / (2 tau^2)) centred at 0 is fitted by
 * least squares to the counts at the bin centres xi_i = (i + 0.5) / 128 - 1
 * (A profiled out; tau the root of the stationarity condition in
 * [0.05, 0.8], bisected to the last bit); the noise is tau * 128 / k. Without
 * a root in that bracket the MAD noise stands (SC_WARN_GAUSS_FALLBACK); a zero
 * MAD noise stays zero. It costs one more pass over S per measurement, and
 * the clip then takes a pass of its own. */

/* ---- flags for sc_run ------------------------------------------------- */
#define SC_FLAG_ACCUMULATE 0x1u /* start from the caller's mask (nonzero = detected) instead of an empty one */
#define SC_FLAG_GENERIC 0x2u    /* use the generic (any-width) smoothing kernels even where a specialised one exists */
#define SC_FLAG_NO_FAST_SELECT 0x4u /* skip the one-pass candidate selection; select by full passes (slow, for tests) */
#define SC_FLAG_GRAPH 0x8u          /* sc_run_batch: capture the batch once into a CUDA graph and replay it */
#define SC_FLAG_NO_SHARE 0x10u      /* smooth every pair in full (no shared spatial passes; same results, slower) */
#define SC_FLAG_SAMPLED_GAUSS 0x20u /* spatial kernels are sampled Gaussians (sc_gauss_taps), not 3-box cascades */
#define SC_FLAG_HALF_DIRECT 0x40u   /* sc_run_half / 16-bit jobs: every kernel reads the 16-bit cube (no float32 copy) */

/* ---- warning bits (sc_stats.warnings, set per run) -------------------- */
#define SC_WARN_ZERO_SIGMA 0x1u     /* some pair had sigma == 0 and added nothing to the mask */
#define SC_WARN_FULL_SELECT 0x2u    /* a selection needed full passes (candidate set above capacity) */
#define SC_WARN_FULL_CLIP 0x4u      /* a clip needed a separate pass (ambiguous set above capacity) */
#define SC_WARN_RANGE 0x8u          /* max|X| / sigma_0 exceeds 2^20: smoothed values may lose exactness */
#define SC_WARN_GAUSS_FALLBACK 0x10u /* SC_NOISE_GAUSS: a histogram without a Gaussian-fit root; the MAD noise stood */

typedef struct sc_ctx sc_ctx;

/* One smoothing kernel pair. fwhm_spatial_px <= 0: no spatial smoothing.
 * boxcar_chan: odd width in channels; 0 or 1: no spectral smoothing. */
typedef struct {
  float fwhm_spatial_px;
  int32_t boxcar_chan;
} sc_kernel;

/* Largest number of kernel pairs in one run. */
#define SC_MAX_KERNELS 64

/* sc_smooth only: run a given kernel variant where it serves the pair (the
 * dispatcher's choice otherwise), flags |= SC_SMOOTH_VARIANT(v). Every variant
 * gives the same floats; this exists for tests and tuning experiments. */
#define SC_VARIANT_WS 1        /* warp-specialised, 64 x 32 tiles */
#define SC_VARIANT_TILE 2      /* one tile per block */
#define SC_VARIANT_GENERIC 3   /* generic kernel */
#define SC_VARIANT_Z8 4        /* spectral-only, 8 voxels per thread */
#define SC_VARIANT_Z4 5        /* spectral-only, 4 voxels per thread */
#define SC_VARIANT_WS16 6      /* warp-specialised, 64 x 16 tiles */
#define SC_VARIANT_Z4_512 7    /* spectral-only, 4 voxels per thread, 512-thread blocks */
#define SC_VARIANT_Z8_512 8    /* spectral-only, 8 voxels per thread, 512-thread blocks (boxcars up to 7) */
#define SC_SMOOTH_VARIANT(v) (((uint32_t)(v) & 0xffu) << 16)

/* Smoothing kernel a kernel pair ran on (sc_stats.smooth_kernel_pair). */
#define SC_KERNEL_NONE 0     /* no smoothing launch: the pair is the unsmoothed cube */
#define SC_KERNEL_IDENTITY 1 /* copy of the cube (a later (0, 1) pair) */
#define SC_KERNEL_Z 2        /* spectral boxcar only */
#define SC_KERNEL_WS32 3     /* warp-specialised spatial cascade + boxcar, 64 x 32 tiles */
#define SC_KERNEL_WS16 4     /* the same with 64 x 16 tiles */
#define SC_KERNEL_TILE 5     /* one tile per block, spatial cascade + boxcar */
#define SC_KERNEL_GENERIC 6  /* any kernel pair */
#define SC_KERNEL_SHARED 7   /* spectral pass over the spatial sums of an earlier pair with the same spatial kernel */
#define SC_KERNEL_FIR 8      /* warp-specialised kernel with the sampled Gaussian's x and y FIRs + boxcar */

/* Counters and timings of the context (cumulative unless reset). */
typedef struct {
  uint64_t launches;      /* CUDA kernels this library launched */
  uint64_t runs;          /* completed sc_run / sc_run_host calls */
  uint32_t warnings;      /* SC_WARN_* bits of the last run */
  uint32_t half_path;     /* last run's cube: 0 float32; 16-bit (sc_run_half, 16-bit jobs): 1 read as such by
                             every kernel (SC_FLAG_HALF_DIRECT), 2 decoded into a float32 copy by a pass of its
                             own, 3 decoded into that copy by the raw-cube histogram pass */
  double ms_smooth;       /* device time of smoothing kernels (only while profiling is on) */
  double ms_select;       /* device time of histogram/plan/candidate/select kernels */
  double ms_clip;         /* device time of mask kernels and of the 16-bit decode (sc_run_half) */
  uint64_t smooth_launches; /* smoothing-kernel launches timed in ms_smooth */
  uint64_t smooth_voxels;   /* output voxels those launches produced */
  double ms_smooth_pair[SC_MAX_KERNELS];          /* ms_smooth split by kernel-pair index of the run */
  uint64_t smooth_launches_pair[SC_MAX_KERNELS];  /* smooth_launches split the same way */
  int32_t smooth_kernel_pair[SC_MAX_KERNELS];     /* SC_KERNEL_* of each pair's latest smoothing (not reset) */
  double ms_noise_window;  /* sc_noise_scale: device time of the per-cell window noise (while profiling) */
  double ms_noise_apply;   /* sc_noise_scale: device time of the division pass (while profiling) */
  double ms_gauss_hist;    /* SC_NOISE_GAUSS: device time of the 256-bin histogram passes (while profiling) */
  double ms_gauss_fit;     /* SC_NOISE_GAUSS: device time of the least-squares fits (while profiling) */
  uint64_t gauss_hist_values; /* values those histogram passes read */
  double ms_share_prep;    /* shared spatial passes: device time of the correction lists and of the gated
                              full-kernel launch, which holds the pair's smoothing when its list was over the
                              cap (while profiling; not in ms_smooth) */
} sc_stats;

/* Create a context on CUDA device `device` with workspace for cubes of up to
 * max_voxels voxels: one float32 smoothed cube (the second cube copy of the
 * paper's memory model, Sect. 5), a 1-bit working mask and small selection
 * buffers. *out receives the context. Errors: SC_ERR_ARG (out NULL,
 * max_voxels 0), SC_ERR_CUDA (bad device), SC_ERR_NOMEM. */
int sc_create(sc_ctx **out, int device, size_t max_voxels);

/* Free the context and all its device memory. NULL is accepted. */
void sc_destroy(sc_ctx *ctx);

/* Static description of a status code (never NULL). */
const char *sc_strerror(int code);

/* Text of the last CUDA failure behind an SC_ERR_CUDA returned on the calling
 * host thread (CUDA's error string, code and the failing call), or "" if none.
 * The buffer is thread-local and overwritten by the next failure. */
const char *sc_last_cuda_error(void);

/* Host helper: the 3 boxcar widths whose cascade approximates a Gaussian of
 * this FWHM (Kovesi 2010 construction; FWHM <= 0 gives widths {1,1,1}, the
 * identity). widths must hold 3 ints. Errors: SC_ERR_ARG (NULL, FWHM not
 * finite or so large that a width exceeds 4095). */
int sc_cascade_widths(float fwhm_px, int32_t *widths);

/* Host helper: the integer taps of the sampled spatial Gaussian of this FWHM,
 * the spatial kernel of runs with SC_FLAG_SAMPLED_GAUSS. The paper names a
 * Gaussian of given FWHM (Sect. 5; Hydra-field figure caption, Sect. 7); this
 * is its sampled form: sigma = FWHM / sqrt(8 ln 2), offsets i = -h..h with
 * h = floor(4 sigma), tap i = exp(-i^2 / (2 sigma^2)) in units of 1/1024 of the
 * central sample rounded to the nearest integer; the kernel is the taps over
 * their sum, applied along x and then y with zero padding (the cube edges are
 * not renormalised). FWHM <= 0 gives the single tap 1024. Writes 2h+1 taps to
 * taps[] and returns 2h+1. The smoothing kernels drop zero taps at both ends
 * (which add nothing) and serve half-widths up to 40 after that, i.e. FWHM up
 * to about 23.5 px; beyond that a run returns SC_ERR_UNSUPPORTED.
 * Errors: SC_ERR_ARG (NULL, FWHM not finite, or more than max_taps taps). */
int sc_gauss_taps(float fwhm_px, int32_t *taps, int max_taps);

/* Full S+C (Sect. 4.2) on a device cube.
 *   cube_dev     float32 [nz][ny][nx], read only.
 *   kernels      n_kernels pairs, run in the order given (Sect. 5 uses
 *                spatial {0,5,10} x spectral {0,3,7,15}).
 *   threshold    t > 0: a voxel is detected when |S| > t*sigma_k.
 *   noise_mode   SC_NOISE_MAD, SC_NOISE_STD or SC_NOISE_GAUSS.
 *   replacement  n: masked voxels become sign(C)*n*sigma_0 before smoothing
 *                (Sect. 6.2); n <= 0 switches replacement off.
 *   mask_dev     uint8 [nz][ny][nx] output, 1 = detected, 0 = not. Zeroed
 *                first unless flags has SC_FLAG_ACCUMULATE.
 *   sigma_host   NULL or double[n_kernels]: sigma of every pair (0 when a
 *                pair's sigma is 0; that pair then adds nothing).
 *   sigma0_host  NULL or double[1]: noise of the raw cube.
 * Returns after the stream has finished when sigma_host or sigma0_host is
 * given (needed to copy them), with the run's device-side status
 * (SC_ERR_ALLNAN, SC_ERR_TIMEOUT, SC_ERR_INTERNAL). Otherwise it returns once
 * all work is enqueued: launch errors are still returned, but that device-side
 * status is not read (the next run clears it), so a caller that needs it
 * passes sigma0_host.
 * Spatial kernel: the 3-box cascade of sc_cascade_widths, or with
 * SC_FLAG_SAMPLED_GAUSS the sampled Gaussian of sc_gauss_taps (half-widths up
 * to 40 after its zero end taps are dropped; wider ones SC_ERR_UNSUPPORTED).
 * Shared spatial passes: when consecutive pairs have the same spatial kernel
 * (cascades of FWHM 3, 5, 6 or 10 px, sampled Gaussians of half-width up to
 * 16, boxcars up to 31 channels), the first of them also
 * stores its spatial sums (int64 per voxel) and each later one adds only the
 * corrections for voxels masked since then (Sect. 6.2 replacement is the only
 * difference between their inputs, and the smoothing is linear and exact).
 * The results are bit for bit those of smoothing every pair in full
 * (SC_FLAG_NO_SHARE). The context allocates for this, on first use, 8 bytes
 * per voxel of the cube (and a bit per voxel for the cube's NaN flags), a
 * correction list of max(2^20, max_voxels/16) entries of 8 bytes and a copy
 * of the working mask; a failed allocation only switches the sharing off.
 * Errors: SC_ERR_ARG (dims <= 0, more voxels than max_voxels -> SC_ERR_BUDGET,
 * even boxcar, negative or non-finite FWHM, t <= 0 or not finite, n_kernels
 * outside 1..SC_MAX_KERNELS, NULL pointers, unknown noise mode),
 * SC_ERR_ALLNAN (no finite voxel; mask left zero), SC_ERR_CUDA. */
int sc_run(sc_ctx *ctx, const float *cube_dev, const int64_t *dims, const sc_kernel *kernels, int n_kernels,
           float threshold, int noise_mode, float replacement, uint8_t *mask_dev, double *sigma_host,
           double *sigma0_host, uint32_t flags, void *cuda_stream);

/* Stream-ordered copy of the sigmas of the latest sc_run on this context:
 * sigma_k of its first n_kernels pairs into sigma_dst[n_kernels] and sigma_0
 * into sigma0_dst[1], as float32 (the precision the device keeps them in;
 * sc_run's sigma_host holds the same values widened to double). The copies
 * are enqueued on cuda_stream behind the work already there and nothing
 * synchronises, so a pipeline of sc_run calls made without sigma pointers
 * can collect every run's sigmas without stopping. Each destination may be
 * NULL, device memory or pinned host memory; it holds the values once the
 * stream has reached the copy. A run whose device-side status was an error
 * (no finite voxel, a timed-out wait, a failed consistency check) leaves
 * zeros in both: a small kernel stages the values, or zeros, in stream order
 * before the copies. Errors: SC_ERR_ARG (NULL ctx, n_kernels outside
 * 1..SC_MAX_KERNELS), SC_ERR_CUDA. */
int sc_copy_sigmas(sc_ctx *ctx, float *sigma_dst, float *sigma0_dst, int n_kernels, void *cuda_stream);

/* Copy of the smoothed cube S of the last kernel pair of the context's latest
 * sc_run / sc_run_host / sc_run_half (float32 [nz][ny][nx] of that cube, NaN
 * at non-finite input voxels) into dst (device or pinned host memory), the
 * first n values, stream-ordered after that run on cuda_stream. When the run's
 * only pair is (0, 0) its S is the cube itself and the buffer holds no value
 * of that run. Library addition (the paper's S+C keeps this second cube copy
 * internally, Sect. 5); used to check smoothed values. Errors: SC_ERR_ARG
 * (NULL, n < 0), SC_ERR_BUDGET (n > max_voxels), SC_ERR_CUDA. */
int sc_copy_smoothed(sc_ctx *ctx, float *dst, int64_t n, void *cuda_stream);

/* Test of the device-side failure path: with enable != 0, the next sc_run on
 * this context makes one producer warp of its first warp-specialised
 * smoothing launch skip its hand-off of one plane, and limits that kernel's
 * waits to 1 ms, so that a consumer's bounded wait runs out. The run then
 * returns SC_ERR_TIMEOUT (when it reads its status: sigma pointers given),
 * its mask and sigmas are meaningless, and the context stays usable. The
 * hook clears itself after that run. No GPU fault, trap or unbounded wait is
 * involved. Library addition for tests. Errors: SC_ERR_ARG (NULL ctx). */
int sc_test_skip_handoff(sc_ctx *ctx, int enable);

/* Cap on the correction list of the shared spatial passes (see sc_run), in
 * entries (an entry is a voxel masked since the spatial sums were stored,
 * once for each tile whose halo holds it). A pair whose corrections exceed
 * the cap is smoothed in full instead, with the same results: the decision
 * is taken on the device, so no synchronisation is needed. 0 restores the
 * default, a cost bound of max(65536, voxels/128) entries beyond which the
 * full smoothing is the faster one; any cap is limited by the list's
 * capacity. Library addition with no counterpart in the paper; it lets tests
 * reach both paths and lets callers tune the trade-off.
 * Errors: SC_ERR_ARG (NULL ctx). */
int sc_set_share_limit(sc_ctx *ctx, uint64_t max_entries);

/* S+C over many independent cubes (the sub-regions SoFiA-X splits a survey
 * into, Sect. 3): each cube gets its own sigma_0 and sigma_k, all with the
 * same kernel list and parameters as sc_run.
 *   n_cubes      >= 1.
 *   cubes        n_cubes device pointers, cube i float32 [nz][ny][nx] with
 *                dims[3*i .. 3*i+2] = {nx, ny, nz}, each <= max_voxels voxels.
 *   masks        n_cubes device uint8 masks of the same shapes (output; zeroed
 *                unless SC_FLAG_ACCUMULATE).
 *   sigma_host   NULL or double[n_cubes * n_kernels], row i = cube i.
 *   sigma0_host  NULL or double[n_cubes].
 * The cubes run with no host synchronisation between them on eight
 * concurrent lanes (the context's workspace and seven more of the same size,
 * created on first use, each with its own stream forked from and joined back
 * into cuda_stream), so one cube's selection overlaps another's smoothing.
 * With SC_FLAG_GRAPH the whole
 * batch is captured once into a CUDA graph (kept in the context and replayed
 * while the cube and mask pointers, shapes, kernels, parameters and tuning
 * are unchanged) and launched as one graph; do not make the first such call
 * inside a caller's own stream capture. Returns after the stream has finished
 * when sigma is wanted. Errors: as sc_run for any cube (nothing is enqueued
 * when an argument is invalid); the first failing cube's status when a cube
 * fails on the device (its sigma row is 0). */
int sc_run_batch(sc_ctx *ctx, int n_cubes, const float *const *cubes, const int64_t *dims, const sc_kernel *kernels,
                 int n_kernels, float threshold, int noise_mode, float replacement, uint8_t *const *masks,
                 double *sigma_host, double *sigma0_host, uint32_t flags, void *cuda_stream);

/* Choose, for a cube shape and each kernel pair, the smoothing kernel variant
 * and z-chunking that run fastest, by timing the candidates on a synthetic
 * noise cube of that shape (in the context's staging buffer) on this GPU.
 * The choices are kept in the context and used by sc_run / sc_run_batch /
 * sc_run_host for cubes of exactly that shape; results are identical for
 * every choice (exact arithmetic), only the time differs. Uses the working
 * mask and device state (no run may be in flight on another stream).
 * Synchronises. Errors: SC_ERR_ARG, SC_ERR_BUDGET, SC_ERR_NOMEM, SC_ERR_CUDA. */
int sc_autotune(sc_ctx *ctx, const int64_t *dims, const sc_kernel *kernels, int n_kernels, void *cuda_stream);

/* S+C on a cube stored in 16 bits with one float32 scale per channel (the
 * precision form: half the bytes of storage and host-to-device transfer).
 *   cube_dev        uint16 [nz][ny][nx]: BF16 bit patterns if is_bf16 != 0,
 *                   else IEEE FP16; read only.
 *   chan_scale_dev  float32 [nz] device array; the cube value of voxel
 *                   (x, y, z) is the float32 product decode(x) * scale[z]
 *                   (rounded once; NaN and Inf decode as such).
 * S+C then runs exactly as sc_run on those values (same arguments, outputs
 * and errors, bit-identical results). How the 16-bit cube is read
 * (sc_stats.half_path):
 *   3 (default, nx a multiple of 8 and cube_dev 16-byte aligned): the
 *     raw-cube histogram pass of sigma_0 reads the 16-bit values and also
 *     writes the decoded cube into the context's float32 staging cube
 *     (allocated on first use, max_voxels floats), which every later pass
 *     reads; no decoding pass of its own.
 *   1 (SC_FLAG_HALF_DIRECT, same shapes): no float32 copy at all: every
 *     kernel reads the 16-bit values (TMA tiles of 16-bit values in the
 *     warp-specialised kernel, 16- and 8-byte copies in the spectral one,
 *     the correction lists and mask pack likewise); the sampled-Gaussian and
 *     generic kernels have no 16-bit forms, so runs with SC_FLAG_SAMPLED_GAUSS
 *     or SC_FLAG_GENERIC take path 3. Saves the staging cube's memory; on
 *     GB300 the 16-bit decoding in the warp-specialised kernel's producers
 *     makes it slower than the default.
 *   2 (other shapes): a decoding pass writes the staging cube first. */
int sc_run_half(sc_ctx *ctx, const uint16_t *cube_dev, int is_bf16, const float *chan_scale_dev,
                const int64_t *dims, const sc_kernel *kernels, int n_kernels, float threshold, int noise_mode,
                float replacement, uint8_t *mask_dev, double *sigma_host, double *sigma0_host, uint32_t flags,
                void *cuda_stream);

/* ---- stream of sub-cubes: asynchronous submission with admission -------
 * Storage of a submitted cube: float32, or 16-bit with per-channel scales
 * (as sc_run_half). */
#define SC_STORE_F32 0
#define SC_STORE_BF16 1
#define SC_STORE_FP16 2

/* Admission budget of sc_submit in bytes (0 = no limit): the cube and mask
 * bytes of the jobs submitted and not yet returned by sc_poll never exceed it. */
int sc_set_budget(sc_ctx *ctx, uint64_t bytes);

/* Enqueue S+C of one cube and return at once with *job_id (> 0). The job runs
 * on one of the context's seven job lanes (workspaces of max_voxels voxels
 * with their own streams, shared with sc_run_batch: do not run a batch while
 * jobs are in flight), round robin, after the lane's earlier jobs; 16-bit
 * storage is read as sc_run_half reads it (decoded into the lane's staging
 * cube by its first histogram pass, or by a pass of its own). The caller keeps
 * cube_dev, chan_scale_dev (16-bit storage only) and mask_dev alive and
 * untouched until sc_poll returns the job. The job starts after the work
 * enqueued on cuda_stream before the call (whatever produced the cube); once
 * sc_poll has returned it, its mask may be read from any stream. Arguments as
 * sc_run otherwise.
 * Errors: SC_ERR_BUDGET when admitting the job would exceed the budget
 * (nothing is enqueued; poll and retry), the argument errors of sc_run,
 * SC_ERR_NOMEM, SC_ERR_CUDA. */
int sc_submit(sc_ctx *ctx, const void *cube_dev, int storage, const float *chan_scale_dev, const int64_t *dims,
              const sc_kernel *kernels, int n_kernels, float threshold, int noise_mode, float replacement,
              uint8_t *mask_dev, uint32_t flags, int64_t *job_id, void *cuda_stream);

/* Return one finished job, if any: 1 with *job_id, *status (SC_OK or the
 * job's error code), *latency_s (host time of the device's completion minus
 * the host time of sc_submit) and the job's sigmas (sigma_host must hold its
 * n_kernels values; either pointer may be NULL); 0 when no job has finished
 * (wait = 0) or none is in flight. wait != 0 blocks until the oldest job
 * finishes when none has. Negative on a CUDA error. */
int sc_poll(sc_ctx *ctx, int wait, int64_t *job_id, int *status, double *latency_s, double *sigma_host,
            double *sigma0_host);

/* sc_run on host buffers: copies cube_host to a device staging cube owned by
 * the context (allocated on first use, max_voxels floats), runs S+C and copies
 * the mask back to mask_host. Pinned (cudaHostAlloc'd / registered) host
 * buffers give full copy bandwidth; pageable memory works but is slower.
 * Same arguments and errors as sc_run; always synchronises the stream. */
int sc_run_host(sc_ctx *ctx, const float *cube_host, const int64_t *dims, const sc_kernel *kernels,
                int n_kernels, float threshold, int noise_mode, float replacement, uint8_t *mask_host,
                double *sigma_host, double *sigma0_host, uint32_t flags, void *cuda_stream);

/* S+C on n_cubes cubes of one shape in host memory, with the copies
 * overlapped: while cube i runs on cuda_stream, cube i + 1 is copied to the
 * device and cube i - 1's mask back, on a copy stream of the context (two
 * device input / mask sets of max_voxels, allocated on first use).
 *   cubes_host[i]        float32 [nz][ny][nx] (storage SC_STORE_F32) or the
 *                        BF16 / FP16 bits (SC_STORE_BF16 / SC_STORE_FP16);
 *   chan_scales_host[i]  float32 [nz] per-channel scales of 16-bit cubes
 *                        (ignored, may be NULL, for float32);
 *   masks_host[i]        uint8 [nz][ny][nx], the output mask (read first with
 *                        SC_FLAG_ACCUMULATE);
 *   sigma_host           NULL or double[n_cubes * n_kernels], row i = cube i;
 *   sigma0_host          NULL or double[n_cubes].
 * Every cube's result is sc_run's (float32) or sc_run_half's (16-bit) on the
 * same values. Pinned host memory gives full copy bandwidth. Returns after all
 * cubes have finished (the stream is synchronised), with the first failing
 * cube's status (its sigmas 0). Errors: as sc_run / sc_run_half, SC_ERR_NOMEM. */
int sc_run_host_many(sc_ctx *ctx, int n_cubes, const void *const *cubes_host, int storage,
                     const float *const *chan_scales_host, const int64_t *dims, const sc_kernel *kernels,
                     int n_kernels, float threshold, int noise_mode, float replacement, uint8_t *const *masks_host,
                     double *sigma_host, double *sigma0_host, uint32_t flags, void *cuda_stream);

/* One pair's smoothed cube S (Sect. 4.2 smoothing, Sect. 6.2 replacement):
 *   X = C with NaN -> 0 and, where mask_dev != 0 and C is finite,
 *       sign(C)*replacement_value (sign(0) = +1; replacement_value <= 0: off);
 *   S = spectral boxcar * spatial cascade (x, y) of the zero-padded X (the
 *       sampled Gaussian of sc_gauss_taps instead with SC_FLAG_SAMPLED_GAUSS);
 *   S = NaN where C is NaN.
 * mask_dev may be NULL (empty mask). out_dev: float32 [nz][ny][nx], may not
 * alias cube_dev. The smoothing is exact fixed-point integer arithmetic
 * rounded once to float32. flags: SC_FLAG_GENERIC, SC_FLAG_SAMPLED_GAUSS and
 * SC_SMOOTH_VARIANT(v). Errors as sc_run. Asynchronous. */
int sc_smooth(sc_ctx *ctx, const float *cube_dev, const int64_t *dims, sc_kernel kernel, const uint8_t *mask_dev,
              float replacement_value, float *out_dev, uint32_t flags, void *cuda_stream);

/* Noise level (Sect. 4.1 estimator) of the finite values of a device float32
 * array of n elements (NaN skipped). *sigma_host receives it (synchronises).
 * Errors: SC_ERR_ARG (NULL pointer, n <= 0, unknown mode), SC_ERR_BUDGET
 * (n > max_voxels), SC_ERR_ALLNAN, SC_ERR_CUDA. */
int sc_noise(sc_ctx *ctx, const float *data_dev, int64_t n, int noise_mode, double *sigma_host, uint32_t flags,
             void *cuda_stream);

/* Local noise normalisation (SoFiA 2 Sect. 4.1: when the noise varies across
 * the cube, measure it in a running window and divide the data by it; the
 * speed test of Sect. 5 uses windows of 31 pixels / channels). The cube is
 * cut into cells of grid[0] x grid[1] x grid[2] voxels (x, y, z; the last cell
 * along an axis may be shorter; grid {1, 1, 1} is the literal running window,
 * one cell per voxel). A cell's noise is sc_noise's statistic (noise_mode) of
 * the finite voxels in the window of window[0] x window[1] x window[2] voxels
 * (odd sizes) centred on the cell's centre voxel, start + (extent - 1) / 2 per
 * axis, clipped to the cube. Then, for every voxel,
 *   out[v] = cube[v] * fl32(1 / sigma(cell(v)))   (within 2^-23 relative of
 *            cube[v] / sigma), or NaN where cube[v] is not finite or the
 *            window's noise is 0 or undefined (no finite voxel).
 *   cube_dev, out_dev  float32 [nz][ny][nx] device buffers (caller-owned);
 *                out_dev may equal cube_dev (in place).
 *   dims         {nx, ny, nz}, each in 1 .. 2^31 - 1.
 *   sigma_host   NULL or double[ncz * ncy * ncx] (ncx = ceil(nx / grid[0]),
 *                ...; x fastest): the noise of every cell, NaN for a window
 *                without finite voxels. With it the call synchronises.
 *   flags        reserved, pass 0.
 * The window's voxels (clipped to the cube) must fit in shared memory:
 * min(wx, nx) * min(wy, ny) * min(wz, nz) <= 47104. The library keeps a
 * per-cell buffer of 12 bytes per cell in the context (grown on demand).
 * Errors: SC_ERR_ARG (NULL pointer, dims, even or non-positive window, grid
 * < 1, unknown mode), SC_ERR_UNSUPPORTED (window too large),
 * SC_ERR_NOMEM, SC_ERR_CUDA. Asynchronous unless sigma_host is given. */
int sc_noise_scale(sc_ctx *ctx, const float *cube_dev, const int64_t *dims, const int32_t *window,
                   const int32_t *grid, int noise_mode, float *out_dev, double *sigma_host, uint32_t flags,
                   void *cuda_stream);

/* Linker (SoFiA 2 Sect. 4.3; radius 2 and minimum sizes 8 pixels / 5
 * channels in Sect. 6): turns a detection mask into numbered detections by
 * friends-of-friends linking and removes those outside the size limits.
 * Two mask voxels are friends when dx^2 + dy^2 <= r_xy^2 and |dz| <= r_z;
 * a detection is a connected component of the mask under that relation.
 * A detection's size along an axis is its extent (max - min + 1); it is
 * removed when its x or y extent is below min_xy or its z extent below
 * min_z, or, for a limit above 0, when its x or y extent exceeds max_xy or
 * its z extent max_z. The kept detections are numbered 1 .. n in raster order
 * (z, then y, then x) of their first voxel.
 *   mask_dev     uint8 [nz][ny][nx] device buffer, nonzero = detected.
 *   dims         {nx, ny, nz}; nx * ny * nz < 2^31 - 1 (int32 voxel indices).
 *   r_xy, r_z    merging radii in voxels, 0 .. 32.
 *   labels_dev   int32 [nz][ny][nx] device buffer (caller-owned, output): the
 *                detection id of every voxel, 0 for none. Also the
 *                union-find workspace, so it may not alias mask_dev.
 *   *n_out       number of kept detections.
 *   extents_host NULL or int32[extents_cap][7]: for detections 1 .. n (the
 *                first extents_cap of them) x_min, x_max, y_min, y_max,
 *                z_min, z_max and the voxel count.
 *   flags        reserved, pass 0.
 * The library keeps per-chunk and per-detection buffers in the context (grown
 * on demand). Synchronises the stream (the number of detections sizes the
 * second half). Errors: SC_ERR_ARG (NULL pointer, dims, radii, negative
 * limits), SC_ERR_NOMEM, SC_ERR_CUDA. */
int sc_link(sc_ctx *ctx, const uint8_t *mask_dev, const int64_t *dims, int r_xy, int r_z, int min_xy, int min_z,
            int max_xy, int max_z, int32_t *labels_dev, int64_t *n_out, int32_t *extents_host, int64_t extents_cap,
            uint32_t flags, void *cuda_stream);

/* Auto-flagger (SoFiA 2 Sect. 4.1): blanks spectral channels and / or
 * spatial pixels whose noise deviates from the median noise across all
 * channels (pixels) by more than k times the RMS estimated from the MAD.
 * The noise of a channel is sc_noise's statistic (noise_mode) of its plane's
 * finite voxels, that of a pixel of its spectrum's finite voxels; both are
 * kept as float32. Across the channels (pixels) with a noise: M = median,
 * R = 1.4826 * median(|noise - M|); a channel (pixel) is flagged when
 * |noise - M| > k * R (in double). With both kinds requested, both are
 * measured on the input and blanked together.
 *   cube_dev, out_dev  float32 [nz][ny][nx]; out_dev may equal cube_dev.
 *   what         SC_AUTOFLAG_CHANNELS and / or SC_AUTOFLAG_PIXELS.
 *   chan_flags_host / chan_noise_host  NULL or [nz];
 *   pix_flags_host / pix_noise_host    NULL or [ny * nx] (x fastest);
 *   n_flagged    NULL or int64[2]: flagged channels, flagged pixels.
 *   flags        reserved, pass 0.
 * Pixels mode needs nz <= 1536 (a tile of spectra in shared memory). The
 * library keeps 5 bytes per channel and per pixel in the context. Synchronises
 * when any host output is given. Errors: SC_ERR_ARG (NULL pointer, dims,
 * k < 0, what, unknown mode), SC_ERR_UNSUPPORTED (pixels with nz > 1536),
 * SC_ERR_NOMEM, SC_ERR_CUDA. */
#define SC_AUTOFLAG_CHANNELS 0x1u
#define SC_AUTOFLAG_PIXELS 0x2u
int sc_autoflag(sc_ctx *ctx, const float *cube_dev, const int64_t *dims, double k, uint32_t what, int noise_mode,
                float *out_dev, uint8_t *chan_flags_host, uint8_t *pix_flags_host, float *chan_noise_host,
                float *pix_noise_host, int64_t *n_flagged, uint32_t flags, void *cuda_stream);

/* Noise level of a device float32 array, like sc_noise, for callers that
 * cannot allocate device memory when they need it: processes whose device
 * memory belongs to another allocator or a fixed pool, real-time pipelines
 * that forbid allocation (and the device synchronisation it implies) once
 * running, plug-ins that are handed only a stream and buffers. It needs no
 * context and allocates nothing: its scratch (2,593,024 bytes) is one static
 * device array that every GPU loading this library holds until the process
 * exits. The paper has no counterpart; this is a library-level addition.
 *   - n <= 4194304 (4 Mi values), else SC_ERR_BUDGET.
 *   - Runs on the calling thread's current device; data_dev must live there.
 *   - The first call on each device looks up the array's device address and
 *     sets kernel attributes; make that first call before any stream capture.
 *   - All calls on a device share the array (each clears what must start at
 *     zero); calls that overlap on the GPU race and must be serialised.
 *   - Synchronises cuda_stream to return *sigma_host. Other errors as sc_noise. */
int sc_noise_static(const float *data_dev, int64_t n, int noise_mode, double *sigma_host, void *cuda_stream);

/* Device-timed profiling of the library's kernels with CUDA events on the
 * launching stream (adds a few microseconds per launch). on = 0 / 1. */
int sc_set_profiling(sc_ctx *ctx, int on);

/* Copy the context's counters to *out; reset = 1 zeroes them afterwards.
 * Synchronises the last stream used so that timings are complete. */
int sc_get_stats(sc_ctx *ctx, sc_stats *out, int reset);

#ifdef __cplusplus
}
#endif
#endif /* SC_H */
