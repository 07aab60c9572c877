// C ABI of the smooth-and-clip library: context, workspace and the order of
// the device steps of one S+C run (SoFiA 2, Sect. 4.2).
//
// One run, all on the caller's stream, no host synchronisation until the end:
//   sigma_0      histogram + plan + candidate pass + exact selections over
//                the raw cube (also max|C| for the fixed-point scales); when
//                the first pair is (0, 0) on an empty mask it is the same
//                measurement, and its clip is done in the same passes.
//   every pair   smoothing kernel (writes S and its histogram), plan,
//                candidate pass over S (also sets the certain mask bits),
//                selections of median and MAD, clip of the undecided voxels.
//   end          1-bit working mask -> caller's uint8 mask; sigmas to host.
#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <deque>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "sc_internal.h"

using namespace sc;

namespace sc {
void init_kernel_attrs();
}  // namespace sc

struct sc_ctx {
  int device = 0;
  int sms = 0;
  size_t max_voxels = 0;
  float* S = nullptr;
  uint32_t* mbits = nullptr;
  unsigned long long* hist = nullptr;
  unsigned long long* ghist = nullptr;  // SC_NOISE_GAUSS: 256 bin counts
  Lists L{};
  DevState* st = nullptr;
  DevState* st_host = nullptr;   // pinned mirror for read-back
  float* stage_cube = nullptr;   // sc_run_host staging (lazy)
  float* sig_out = nullptr;      // sc_copy_sigmas staging: SC_MAX_KERNELS + 1 floats
  double* ns_sig = nullptr;      // sc_noise_scale: noise of every cell (lazy, grown)
  float* ns_rinv = nullptr;      // and its float reciprocal
  size_t ns_cap = 0;             // cells both hold
  int* lk_chunk = nullptr;       // sc_link: per-chunk root counts / offsets (lazy, grown)
  size_t lk_chunk_cap = 0;
  int* lk_tot = nullptr;         // sc_link: one device int (a total)
  int* lk_comp = nullptr;        // sc_link: [4 arrays of cap][7 or 1 ints] per detection
  size_t lk_comp_cap = 0;
  unsigned char* af_buf = nullptr;  // sc_autoflag: noises, flags and statistics (lazy, grown)
  size_t af_cap = 0;
  uint8_t* stage_mask = nullptr;
  // sc_run_host_many (lazy): two device input / mask sets, the per-channel
  // scales of 16-bit cubes, the copy stream and its events, per-cube results
  void* hm_in[2] = {nullptr, nullptr};       // max_voxels float32 (16-bit cubes use half)
  uint8_t* hm_mask[2] = {nullptr, nullptr};
  float* hm_scale[2] = {nullptr, nullptr};
  size_t hm_scale_cap = 0;
  cudaStream_t hm_copy = nullptr;
  cudaEvent_t hm_ev[6] = {};                 // loaded[2], computed[2], sent[2]
  unsigned char* hm_res = nullptr;           // pinned: one BatchRes per cube
  size_t hm_res_cap = 0;
  int profiling = 0;
  sc_stats stats{};
  struct Ev {
    cudaEvent_t a, b;
    int kind;
    unsigned long long voxels;
    int pair;  // kernel-pair index for smoothing events, else -1
  };
  std::vector<Ev> events;     // recorded, not yet accumulated
  std::vector<cudaEvent_t> pool;
  cudaStream_t last = nullptr;
  // kernel choices fixed by sc_autotune: (nx, ny, nz, w1, w2, w3, wz) -> (kind, items per SM)
  std::map<std::array<long long, 7>, std::array<int, 2>> tune;
  // sc_run_batch: per-cube results on the device and their pinned host mirror
  unsigned char* batch_res = nullptr;
  unsigned char* batch_res_host = nullptr;
  size_t batch_res_cap = 0;
  // sc_run_batch with SC_FLAG_GRAPH: the captured batch and its signature
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  unsigned long long graph_key = 0;
  unsigned long long graph_launches = 0;
  bool capturing = false;  // no profiling events inside a capture
  // sc_run_batch: extra workspaces ("lanes", full contexts of their own) that
  // run other cubes of the batch concurrently on their own streams
  std::vector<sc_ctx*> lanes;
  std::vector<cudaStream_t> lane_streams;
  std::vector<cudaEvent_t> lane_done;
  cudaEvent_t fork = nullptr;
  // sc_submit / sc_poll: jobs in flight, their admission budget and the clock
  // reference that maps device completion times to host time
  struct Job {
    long long id;
    int lane;
    int n_kernels;
    cudaEvent_t done;
    double t_submit;
    unsigned long long bytes;
    unsigned char* slot;  // pinned per-job results (status, warnings, sigmas)
  };
  std::deque<Job> jobs;
  long long next_job = 1;
  unsigned long long budget = 0;  // 0: no limit
  unsigned long long in_flight = 0;
  std::vector<cudaEvent_t> job_events;
  std::vector<unsigned char*> job_slots;
  cudaEvent_t clock_ev = nullptr;
  double clock_host = 0.0;
  // shared spatial passes (allocated on first use, grown for larger cubes)
  long long* sh_P = nullptr;          // spatial sums of the first pair of a spatial kernel
  size_t sh_P_cap = 0;                // elements
  unsigned char* sh_nf = nullptr;     // their cube's nonfinite flags, a byte per column and 8 rows
  size_t sh_nf_cap = 0;               // bytes
  uint32_t* sh_snap = nullptr;        // working mask when P' was made (max_voxels bits + padding)
  unsigned* sh_cnt = nullptr;         // per-bucket counts (kept zero between pairs)
  unsigned* sh_offs = nullptr;        // their exclusive scan
  unsigned long long* sh_bsum = nullptr;
  size_t sh_bk_cap = 0;               // buckets + 1 the three arrays hold
  unsigned long long* sh_ent = nullptr;  // correction entries
  unsigned long long sh_ent_cap = 0;
  unsigned long long sh_limit = 0;    // sc_set_share_limit (0: the buffer's capacity)
  int test_skip_handoff = 0;          // sc_test_skip_handoff: armed for the next run
  ShareState* sh_ss = nullptr;
};

namespace {
constexpr int kBatchLanes = 8;  // concurrent cubes of a batch (the context itself and 7 lanes)
}

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

cudaEvent_t take_event(sc_ctx* c) {
  if (!c->pool.empty()) {
    cudaEvent_t e = c->pool.back();
    c->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

enum { EV_SMOOTH = 0, EV_SELECT = 1, EV_CLIP = 2, EV_NOISE_WINDOW = 3, EV_NOISE_APPLY = 4, EV_GAUSS_HIST = 5,
       EV_GAUSS_FIT = 6, EV_SHARE_PREP = 7 };

struct Phase {
  sc_ctx* c;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  int kind;
  unsigned long long vox;
  int pair;
  Phase(sc_ctx* c_, cudaStream_t s_, int kind_, unsigned long long vox_ = 0, int pair_ = -1)
      : c(c_), s(s_), kind(kind_), vox(vox_), pair(pair_) {
    if (c->profiling && !c->capturing) {
      a = take_event(c);
      cudaEventRecord(a, s);
    }
  }
  ~Phase() {
    if (c->profiling && !c->capturing && a) {
      cudaEvent_t b = take_event(c);
      cudaEventRecord(b, s);
      c->events.push_back({a, b, kind, vox, pair});
    }
  }
};

void flush_events(sc_ctx* c) {
  for (auto& e : c->events) {
    cudaEventSynchronize(e.b);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e.a, e.b);
    if (e.kind == EV_SMOOTH) {
      c->stats.ms_smooth += ms;
      c->stats.smooth_launches += 1;
      c->stats.smooth_voxels += e.voxels;
      if (e.pair >= 0 && e.pair < SC_MAX_KERNELS) {
        c->stats.ms_smooth_pair[e.pair] += ms;
        c->stats.smooth_launches_pair[e.pair] += 1;
      }
    } else if (e.kind == EV_SELECT) {
      c->stats.ms_select += ms;
    } else if (e.kind == EV_NOISE_WINDOW) {
      c->stats.ms_noise_window += ms;
    } else if (e.kind == EV_NOISE_APPLY) {
      c->stats.ms_noise_apply += ms;
    } else if (e.kind == EV_GAUSS_HIST) {
      c->stats.ms_gauss_hist += ms;
      c->stats.gauss_hist_values += e.voxels;
    } else if (e.kind == EV_SHARE_PREP) {
      c->stats.ms_share_prep += ms;
    } else if (e.kind == EV_GAUSS_FIT) {
      c->stats.ms_gauss_fit += ms;
    } else {
      c->stats.ms_clip += ms;
    }
    c->pool.push_back(e.a);
    c->pool.push_back(e.b);
  }
  c->events.clear();
}

thread_local char g_last_cuda_error[256] = "";

int cuda_fail(cudaError_t e, const char* what, int line) {
  snprintf(g_last_cuda_error, sizeof(g_last_cuda_error), "%s (%d) at %s:%d", cudaGetErrorString(e), (int)e, what,
           line);
  return SC_ERR_CUDA;
}

#define CK(x)                                                   \
  do {                                                          \
    cudaError_t e_ = (x);                                       \
    if (e_ != cudaSuccess) return cuda_fail(e_, #x, __LINE__);  \
  } while (0)

int check_dims(const sc_ctx* c, const int64_t* dims, long long* n) {
  if (!dims) return SC_ERR_ARG;
  if (dims[0] <= 0 || dims[1] <= 0 || dims[2] <= 0) return SC_ERR_ARG;
  if (dims[0] > (1 << 30) || dims[1] > (1 << 30) || dims[2] > (1 << 30)) return SC_ERR_ARG;
  const long double nn = (long double)dims[0] * dims[1] * dims[2];
  if (nn > (long double)c->max_voxels) return SC_ERR_BUDGET;
  *n = (long long)dims[0] * dims[1] * dims[2];
  return SC_OK;
}

int status_to_code(const DevState& h) {
  if (h.status & SC_ST_TIMEOUT) return SC_ERR_TIMEOUT;
  if (h.status & SC_ST_ALLNAN) return SC_ERR_ALLNAN;
  if (h.status & (SC_ST_INTERNAL | SC_ST_OVERFLOW)) return SC_ERR_INTERNAL;
  return SC_OK;
}

// One noise measurement (and optional clip) over src, whose histogram is in
// c->hist. pair: index for sigma[] (-1: none).
int measure(sc_ctx* c, const float* src, long long n, int win, float t, int clip, int noise_mode, int pair,
            unsigned int force, cudaStream_t s) {
  const int std_mode = noise_mode == SC_NOISE_STD;
  const bool gauss = noise_mode == SC_NOISE_GAUSS;
  {
    Phase ph(c, s, EV_SELECT);
    // the Gaussian fit moves sigma after the MAD: its clip waits for the fit
    CK(launch_plan(c->st, c->hist, win, src, n, c->L, t, gauss ? 0 : clip, std_mode, force, s));
    c->stats.launches += 1;
    if (std_mode) {
      CK(launch_std(src, n, c->st, c->sms, s));
      CK(launch_std_final(c->st, pair, s));
      c->stats.launches += 3;
    } else {
      CK(launch_pass2(src, n, c->mbits, c->st, c->L, c->sms, s));
      CK(launch_select(c->st, 0, -1, c->sms, s));
      CK(launch_select(c->st, 1, pair, c->sms, s));
      c->stats.launches += 11;
    }
  }
  if (gauss) {
    {
      Phase ph(c, s, EV_GAUSS_HIST, (unsigned long long)n);
      CK(launch_gauss_hist(src, n, c->st, c->ghist, c->sms, s));
    }
    Phase ph(c, s, EV_GAUSS_FIT);
    CK(launch_gauss_fit(c->st, c->ghist, pair, clip, s));
    c->stats.launches += 2;
  }
  if (clip) {
    Phase ph(c, s, EV_CLIP);
    if (!std_mode && !gauss) {
      CK(launch_resolve(src, c->mbits, c->st, c->L, c->sms, s));
      c->stats.launches += 1;
    }
    CK(launch_clip_full(src, n, c->mbits, c->st, c->sms, s));
    c->stats.launches += 1;
  }
  return SC_OK;
}

int validate_common(sc_ctx* c, const float* cube, const int64_t* dims, const sc_kernel* kernels, int nk, float t,
                    int noise_mode, long long* n, std::vector<PairDesc>* pds, uint32_t flags) {
  if (!c || !cube || !kernels) return SC_ERR_ARG;
  int rc = check_dims(c, dims, n);
  if (rc) return rc;
  if (nk < 1 || nk > SC_MAX_KERNELS) return SC_ERR_ARG;
  if (!(t > 0.0f) || !std::isfinite(t)) return SC_ERR_ARG;
  if (noise_mode != SC_NOISE_MAD && noise_mode != SC_NOISE_STD && noise_mode != SC_NOISE_GAUSS) return SC_ERR_ARG;
  pds->resize(nk);
  for (int k = 0; k < nk; ++k) {
    rc = make_pair(kernels[k], &(*pds)[k], (flags & SC_FLAG_SAMPLED_GAUSS) != 0);
    if (rc) return rc;
  }
  return SC_OK;
}

std::array<long long, 7> tune_key(const int64_t* dims, const PairDesc& pd) {
  return {dims[0], dims[1], dims[2], pd.w[0], pd.w[1], pd.w[2], pd.wz};
}

// Kernel choice of sc_autotune for this cube shape and pair, if any.
void apply_tuning(sc_ctx* c, const int64_t* dims, SmoothArgs* a) {
  if (c->tune.empty() || a->pd.sampled) return;  // the tuner times cascade pairs only
  auto it = c->tune.find(tune_key(dims, a->pd));
  if (it == c->tune.end()) return;
  a->tune_kind = it->second[0];
  a->tune_zfactor = it->second[1];
}

// Sizes of the shared-pass buffers a cube needs: its spatial sums (an even
// pitch: 16-byte aligned rows for TMA) and its buckets (those of the smaller
// tile height, 16 rows, bound those of both heights).
// Bytes per row of the nonfinite-flag map (16-byte aligned rows for TMA).
long long nf_pitch(long long nx) { return (nx + 15) & ~15LL; }

struct ShareNeeds {
  size_t p, bk, nf;
};

ShareNeeds share_needs(const int64_t* dims) {
  const long long nx = dims[0], ny = dims[1], nz = dims[2];
  return ShareNeeds{(size_t)((nx + 1) & ~1LL) * ny * nz, (size_t)((nx + 63) / 64) * ((ny + 15) / 16) * nz + 1,
                    (size_t)nf_pitch(nx) * ((ny + 7) / 8) * nz};
}

// Buffers of the shared spatial passes for these sizes (allocated or grown
// here; never inside a stream capture).
int ensure_share_sized(sc_ctx* c, const ShareNeeds& nd) {
  const size_t need_p = nd.p, need_bk = nd.bk;
  const bool fits = c->sh_P_cap >= need_p && c->sh_bk_cap >= need_bk && c->sh_nf_cap >= nd.nf && c->sh_ent &&
                    c->sh_snap && c->sh_ss;
  if (fits) return SC_OK;
  if (c->capturing) return SC_ERR_BUDGET;
  if (!c->sh_snap) {
    const size_t nwords = (c->max_voxels + 31) / 32 + 8;
    const unsigned long long cap = std::max<unsigned long long>(1ull << 20, (unsigned long long)c->max_voxels / 16);
    if (cudaMalloc(&c->sh_snap, sizeof(uint32_t) * nwords) != cudaSuccess ||
        cudaMalloc(&c->sh_ent, sizeof(unsigned long long) * (cap + 2)) != cudaSuccess ||
        cudaMalloc(&c->sh_ss, sizeof(ShareState)) != cudaSuccess) {
      cudaGetLastError();
      return SC_ERR_NOMEM;
    }
    c->sh_ent_cap = cap;
    if (cudaMemset(c->sh_snap, 0, sizeof(uint32_t) * nwords) != cudaSuccess ||
        cudaMemset(c->sh_ent, 0, sizeof(unsigned long long) * (cap + 2)) != cudaSuccess ||
        cudaMemset(c->sh_ss, 0, sizeof(ShareState)) != cudaSuccess)
      return SC_ERR_CUDA;
  }
  if (c->sh_P_cap < need_p) {
    cudaStreamSynchronize(c->last);
    cudaFree(c->sh_P);
    c->sh_P = nullptr;
    c->sh_P_cap = 0;
    if (cudaMalloc(&c->sh_P, sizeof(long long) * need_p) != cudaSuccess) {
      cudaGetLastError();
      return SC_ERR_NOMEM;
    }
    c->sh_P_cap = need_p;
  }
  if (c->sh_nf_cap < nd.nf) {
    cudaStreamSynchronize(c->last);
    cudaFree(c->sh_nf);
    c->sh_nf = nullptr;
    c->sh_nf_cap = 0;
    if (cudaMalloc(&c->sh_nf, nd.nf) != cudaSuccess) {
      cudaGetLastError();
      return SC_ERR_NOMEM;
    }
    c->sh_nf_cap = nd.nf;
  }
  if (c->sh_bk_cap < need_bk) {
    cudaStreamSynchronize(c->last);
    cudaFree(c->sh_cnt);
    cudaFree(c->sh_offs);
    cudaFree(c->sh_bsum);
    c->sh_cnt = nullptr;
    c->sh_offs = nullptr;
    c->sh_bsum = nullptr;
    c->sh_bk_cap = 0;
    const size_t nb = need_bk + 4096;
    if (cudaMalloc(&c->sh_cnt, sizeof(unsigned) * nb) != cudaSuccess ||
        cudaMalloc(&c->sh_offs, sizeof(unsigned) * nb) != cudaSuccess ||
        cudaMalloc(&c->sh_bsum, sizeof(unsigned long long) * (nb / 4096 + 2)) != cudaSuccess) {
      cudaGetLastError();
      return SC_ERR_NOMEM;
    }
    if (cudaMemset(c->sh_cnt, 0, sizeof(unsigned) * nb) != cudaSuccess) return SC_ERR_CUDA;
    c->sh_bk_cap = need_bk;
  }
  return SC_OK;
}

int ensure_share(sc_ctx* c, const int64_t* dims) { return ensure_share_sized(c, share_needs(dims)); }

bool same_spatial(const PairDesc& a, const PairDesc& b) {
  if (a.sampled != b.sampled || a.h != b.h) return false;
  for (int i = 0; i < 2 * a.h + 1; ++i)
    if (a.taps[i] != b.taps[i]) return false;
  return a.w[0] == b.w[0] && a.w[1] == b.w[1] && a.w[2] == b.w[2];
}

SmoothArgs base_args(sc_ctx* c, const float* cube, const int64_t* dims, const Half16* h16 = nullptr) {
  SmoothArgs a;
  memset(&a, 0, sizeof(a));
  a.C = cube;
  if (h16) a.h16 = *h16;
  a.mbits = c->mbits;
  a.S = c->S;
  a.nx = (int)dims[0];
  a.ny = (int)dims[1];
  a.nz = (int)dims[2];
  a.st = c->st;
  return a;
}

// A 16-bit cube is read by the kernels (the raw-cube histograms, and with
// SC_FLAG_HALF_DIRECT every kernel) when its rows are 16-byte multiples (TMA
// tiles of 16-bit values, 16-byte loads of 8 values within a plane) and its
// base is 16-byte aligned; otherwise it is decoded by a pass of its own.
bool half_in_kernel(const void* cube_dev, const int64_t* dims) {
  return dims[0] % 8 == 0 && (reinterpret_cast<uintptr_t>(cube_dev) & 15u) == 0;
}

// The generic and sampled-Gaussian kernels have no 16-bit forms: such runs
// read the float32 copy.
uint32_t half_flags(uint32_t flags) {
  return (flags & (SC_FLAG_GENERIC | SC_FLAG_SAMPLED_GAUSS)) ? flags & ~(uint32_t)SC_FLAG_HALF_DIRECT : flags;
}

// Device staging cube and mask of max_voxels elements (allocated on first use).
int ensure_stage(sc_ctx* c) {
  if (c->stage_cube) return SC_OK;
  if (cudaMalloc(&c->stage_cube, sizeof(float) * c->max_voxels) != cudaSuccess ||
      cudaMalloc(&c->stage_mask, c->max_voxels) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(c->stage_cube);
    cudaFree(c->stage_mask);
    c->stage_cube = nullptr;
    c->stage_mask = nullptr;
    return SC_ERR_NOMEM;
  }
  return SC_OK;
}

// One S+C run on the device. The cube is the float32 one at `cube`, or, with
// h16 (cube null), a 16-bit one. The raw-cube histogram pass reads the
// 16-bit values; by default it also decodes the cube into the context's
// float32 working copy, which every later pass reads (the float32 kernels, no
// decoding pass of its own). With SC_FLAG_HALF_DIRECT no copy is made: the
// histogram pass decodes into S (the float32 cube the sigma_0 selection and
// the first pair read) and the smoothing kernels and correction lists decode
// their own 16-bit values.
int run_device(sc_ctx* c, const float* cube, const int64_t* dims, const sc_kernel* kernels, int nk, float t,
               int noise_mode, float replacement, uint8_t* mask_dev, uint32_t flags, cudaStream_t s,
               const Half16* h16 = nullptr) {
  long long n = 0;
  std::vector<PairDesc> pds;
  int rc = validate_common(c, h16 ? reinterpret_cast<const float*>(h16->bits) : cube, dims, kernels, nk, t,
                           noise_mode, &n, &pds, flags);
  if (rc) return rc;
  if (!mask_dev) return SC_ERR_ARG;
  if (!std::isfinite(replacement)) return SC_ERR_ARG;
  const int std_mode = (noise_mode == SC_NOISE_STD);
  const unsigned int force = (flags & SC_FLAG_NO_FAST_SELECT) ? (PLAN_MED_FULL | PLAN_MAD_FULL | PLAN_CLIP_FULL) : 0u;
  PairWeights W{};
  for (int k = 0; k < nk; ++k) {
    W.w[k] = pds[k].W;
    W.wf[k] = pds[k].Wf;
  }
  CK(cudaMemsetAsync(c->st, 0, sizeof(DevState), s));
  const long long nwords = (n + 31) / 32;
  const long long plane = dims[0] * dims[1];
  const bool direct = h16 && (flags & SC_FLAG_HALF_DIRECT);
  if (h16 && !direct) {
    rc = ensure_stage(c);  // the float32 working copy
    if (rc) return rc;
  }
  c->stats.half_path = h16 ? (direct ? 1u : 3u) : 0u;
  if (flags & SC_FLAG_ACCUMULATE) {
    if (h16) CK(launch_pack16(mask_dev, *h16, plane, n, c->mbits, s));  // (before the copy exists)
    else CK(launch_pack(mask_dev, cube, n, c->mbits, s));
    c->stats.launches += 1;
  } else {
    CK(cudaMemsetAsync(c->mbits, 0, sizeof(uint32_t) * nwords, s));
  }
  const bool first_identity = (pds[0].h == 0 && pds[0].wz == 1) && !(flags & SC_FLAG_ACCUMULATE);

  // sigma_0 of the raw cube (and the first pair when it is (0, 0))
  CK(cudaMemsetAsync(c->hist, 0, sizeof(unsigned long long) * kNumBins, s));
  // the float32 raw cube the sigma_0 selection reads: the cube, the working
  // copy of a 16-bit cube, or (direct) S
  const float* src0 = h16 ? (direct ? c->S : c->stage_cube) : cube;
  {
    Phase ph(c, s, EV_SELECT);
    // one histogram pass with max |C| (a 16-bit cube: decoded by it into the
    // working copy, or into S when direct): windowed around the median |C| of
    // an even sample (a fine plan), or over the full range for STD mode
    if (!std_mode) {
      CK(launch_window_from_sample(cube, h16, plane, n, c->st, s));
      c->stats.launches += 1;
    }
    const int win0 = std_mode ? 0 : 1;
    if (h16)
      CK(launch_hist16(*h16, plane, n, c->st, c->hist, win0, 1, direct ? c->S : c->stage_cube, c->sms, s));
    else CK(launch_hist(cube, n, c->st, c->hist, win0, 1, c->sms, s));
    c->stats.launches += 1;
  }
  rc = measure(c, src0, n, std_mode ? 0 : 1, t, first_identity ? 1 : 0, noise_mode, first_identity ? 0 : -1, force,
               s);
  if (rc) return rc;
  if (h16 && !direct) {  // the pairs read the float32 working copy
    cube = c->stage_cube;
    h16 = nullptr;
  }
  CK(launch_sigma0_done(c->st, replacement, W, nk, s));
  c->stats.launches += 1;

  if (first_identity) c->stats.smooth_kernel_pair[0] = SC_KERNEL_NONE;
  // Shared spatial passes: the first of consecutive pairs with one spatial
  // kernel stores its spatial sums, the later ones reuse them.
  const bool share_on = !(flags & (SC_FLAG_NO_SHARE | SC_FLAG_GENERIC));
  bool share_cnt_clear = false;
  int p_owner = -1;  // pair whose spatial sums sh_P holds
  for (int k = first_identity ? 1 : 0; k < nk; ++k) {
    CK(cudaMemsetAsync(c->hist, 0, sizeof(unsigned long long) * kNumBins, s));
    SmoothArgs a = base_args(c, cube, dims, h16);
    a.pd = pds[k];
    a.pair = k;
    apply_tuning(c, dims, &a);
    a.hist = c->hist;
    a.win = 1;
    a.generic = (flags & SC_FLAG_GENERIC) ? 1 : 0;
    a.repl_possible = replacement > 0.0f ? 1 : 0;
    int share_mode = 0;  // 0: plain, 1: store the spatial sums, 2: reuse them
    if (share_on && share_supported(a.pd)) {
      if (p_owner >= 0 && same_spatial(pds[p_owner], a.pd)) {
        share_mode = 2;
      } else if (k + 1 < nk && share_supported(pds[k + 1]) && same_spatial(a.pd, pds[k + 1]) &&
                 ensure_share(c, dims) == SC_OK) {
        share_mode = 1;
      }
    }
    if (share_mode != 2) p_owner = -1;
    if (share_mode == 2) {
      ShareArgs sh{};
      sh.P = c->sh_P;
      sh.pitch = (dims[0] + 1) & ~1LL;
      sh.nf = c->sh_nf;
      sh.nfpitch = nf_pitch(dims[0]);
      sh.msnap = c->sh_snap;
      sh.cnt = c->sh_cnt;
      sh.bsum = c->sh_bsum;
      sh.ent = c->sh_ent;
      // the caller's cap, else a cost bound (beyond about one correction per
      // 128 voxels the full kernel is the faster one), within the list's capacity
      sh.cap = c->sh_limit > 0 ? c->sh_limit
                               : std::max<unsigned long long>(1ull << 16, (unsigned long long)n / 128);
      sh.cap = std::min(sh.cap, c->sh_ent_cap);
      sh.ss = c->sh_ss;
      sh.ty = share_tile_rows(a.pd.wz);
      sh.tiles_x = (int)((dims[0] + 63) / 64);
      sh.tiles_y = (int)((dims[1] + sh.ty - 1) / sh.ty);
      sh.n_buckets = (long long)sh.tiles_x * sh.tiles_y * dims[2];
      {  // the correction lists, and the full kernel gated on their size
        Phase ph(c, s, EV_SHARE_PREP);
        CK(cudaMemsetAsync(c->sh_ss, 0, sizeof(ShareState), s));
        if (a.repl_possible) {
          // voxels masked since the spatial sums were made, listed per bucket
          if (!share_cnt_clear) {
            CK(cudaMemsetAsync(c->sh_cnt, 0, sizeof(unsigned) * c->sh_bk_cap, s));  // every tile height
            share_cnt_clear = true;
          }
          sh.offs = c->sh_offs;
          CK(launch_share_prep(a, sh, c->sms, s));
          c->stats.launches += 4;
        }
        // the full kernel, run only if the list overflowed
        SmoothArgs full = a;
        full.gate = &c->sh_ss->overflow;
        full.tune_kind = TUNE_AUTO;
        int l = 0, code = SC_KERNEL_NONE;
        CK(launch_smooth(full, c->sms, s, &l, &code));
        c->stats.launches += l;
      }
      Phase ph(c, s, EV_SMOOTH, (unsigned long long)n, k);
      bool done = false;
      CK(launch_smooth_p(a, sh, c->sms, s, &done));
      if (!done) return SC_ERR_INTERNAL;
      c->stats.launches += 1;
      c->stats.smooth_kernel_pair[k] = SC_KERNEL_SHARED;
    } else {
      Phase ph(c, s, EV_SMOOTH, (unsigned long long)n, k);
      if (c->test_skip_handoff) {
        a.test_skip_handoff = 1;  // taken by the first warp-specialised launch
        a.tune_kind = TUNE_AUTO;
      }
      if (share_mode == 1) {
        CK(cudaMemcpyAsync(c->sh_snap, c->mbits, sizeof(uint32_t) * nwords, cudaMemcpyDeviceToDevice, s));
        a.pout = c->sh_P;
        a.ppitch = (dims[0] + 1) & ~1LL;
        a.nfout = c->sh_nf;
        a.nfpitch = nf_pitch(dims[0]);
        a.tune_kind = TUNE_AUTO;
      }
      if (a.pd.h == 0 && a.pd.wz == 1) {
        CK(launch_identity(a, c->sms, s));
        c->stats.launches += 1;
        c->stats.smooth_kernel_pair[k] = SC_KERNEL_IDENTITY;
      } else {
        int l = 0, code = SC_KERNEL_NONE;
        CK(launch_smooth(a, c->sms, s, &l, &code));
        c->stats.launches += l;
        c->stats.smooth_kernel_pair[k] = code;
        // the warp-specialised kernel (cascade or FIR) takes the test hook and
        // is the one that stores the spatial sums
        const bool ws_kernel = code == SC_KERNEL_WS32 || code == SC_KERNEL_WS16 || code == SC_KERNEL_FIR;
        if (ws_kernel) c->test_skip_handoff = 0;
        if (share_mode == 1 && ws_kernel) p_owner = k;
      }
    }
    rc = measure(c, c->S, n, 1, t, 1, noise_mode, k, force, s);
    if (rc) return rc;
  }
  {
    Phase ph(c, s, EV_CLIP);
    CK(launch_expand(c->mbits, n, mask_dev, (flags & SC_FLAG_ACCUMULATE) ? 1 : 0, s));
    c->stats.launches += 1;
  }
  c->test_skip_handoff = 0;  // the hook serves one run
  return SC_OK;
}

int finish(sc_ctx* c, int nk, double* sigma_host, double* sigma0_host, cudaStream_t s, bool force_sync) {
  if (!sigma_host && !sigma0_host && !force_sync) return SC_OK;
  CK(cudaMemcpyAsync(c->st_host, c->st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const DevState& h = *c->st_host;
  c->stats.warnings = h.warn;
  const int rc = status_to_code(h);
  if (sigma0_host) *sigma0_host = (rc == SC_OK) ? (double)h.sigma0 : 0.0;
  if (sigma_host)
    for (int k = 0; k < nk; ++k) sigma_host[k] = (rc == SC_OK) ? (double)h.sigma[k] : 0.0;
  return rc;
}

}  // namespace

extern "C" {

const char* sc_last_cuda_error(void) { return g_last_cuda_error; }

const char* sc_strerror(int code) {
  switch (code) {
    case SC_OK: return "ok";
    case SC_ERR_ARG: return "invalid argument";
    case SC_ERR_NOMEM: return "out of memory";
    case SC_ERR_CUDA: return "CUDA error";
    case SC_ERR_ALLNAN: return "cube has no finite voxel";
    case SC_ERR_TIMEOUT: return "device-side wait timed out";
    case SC_ERR_UNSUPPORTED: return "unsupported option";
    case SC_ERR_BUDGET: return "request exceeds the context's budget";
    case SC_ERR_INTERNAL: return "internal consistency check failed";
    default: return "unknown status code";
  }
}

int sc_cascade_widths(float fwhm_px, int32_t* widths) {
  if (!widths || !std::isfinite(fwhm_px)) return SC_ERR_ARG;
  int w[3];
  if (cascade_widths(fwhm_px, w) != 0) return SC_ERR_ARG;
  for (int i = 0; i < 3; ++i) widths[i] = w[i];
  return SC_OK;
}

int sc_gauss_taps(float fwhm_px, int32_t* taps, int max_taps) {
  if (!taps || max_taps < 1 || !std::isfinite(fwhm_px)) return SC_ERR_ARG;
  std::vector<int> t((size_t)max_taps);
  const int n = gauss_taps(fwhm_px, t.data(), max_taps);
  if (n < 1) return SC_ERR_ARG;
  for (int i = 0; i < n; ++i) taps[i] = t[i];
  return n;
}

int sc_create(sc_ctx** out, int device, size_t max_voxels) {
  if (!out || max_voxels == 0) return SC_ERR_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return SC_ERR_CUDA;
  DeviceGuard g(device);
  sc_ctx* c = new (std::nothrow) sc_ctx();
  if (!c) return SC_ERR_NOMEM;
  c->device = device;
  c->max_voxels = max_voxels;
  cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device);
  init_kernel_attrs();
  const unsigned long long nv = max_voxels;
  c->L.cap.med = std::max<unsigned long long>(1ull << 20, nv / 64);
  c->L.cap.mad = std::max<unsigned long long>(1ull << 22, nv / 16);
  c->L.cap.amb = std::max<unsigned long long>(1ull << 20, nv / 64);
  const size_t nwords = (max_voxels + 31) / 32 + 8;
  bool ok = cudaMalloc(&c->S, sizeof(float) * max_voxels) == cudaSuccess &&
            cudaMalloc(&c->mbits, sizeof(uint32_t) * nwords) == cudaSuccess &&
            cudaMalloc(&c->hist, sizeof(unsigned long long) * kNumBins) == cudaSuccess &&
            cudaMalloc(&c->ghist, sizeof(unsigned long long) * kGaussBins) == cudaSuccess &&
            cudaMalloc(&c->L.med, sizeof(float) * c->L.cap.med) == cudaSuccess &&
            cudaMalloc(&c->L.mad, sizeof(float) * c->L.cap.mad) == cudaSuccess &&
            cudaMalloc(&c->L.amb, sizeof(unsigned long long) * c->L.cap.amb) == cudaSuccess &&
            cudaMalloc(&c->L.cls, kClassTableBytes) == cudaSuccess &&
            cudaMalloc(&c->st, sizeof(DevState)) == cudaSuccess &&
            cudaMalloc(&c->sig_out, sizeof(float) * (SC_MAX_KERNELS + 1)) == cudaSuccess &&
            cudaHostAlloc(&c->st_host, sizeof(DevState), cudaHostAllocDefault) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    sc_destroy(c);
    return SC_ERR_NOMEM;
  }
  cudaMemset(c->mbits, 0, sizeof(uint32_t) * nwords);
  cudaMemset(c->st, 0, sizeof(DevState));
  if (cudaDeviceSynchronize() != cudaSuccess) {
    sc_destroy(c);
    return SC_ERR_CUDA;
  }
  *out = c;
  return SC_OK;
}

void sc_destroy(sc_ctx* c) {
  if (!c) return;
  DeviceGuard g(c->device);
  cudaDeviceSynchronize();
  for (auto& e : c->events) {
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  for (auto e : c->pool) cudaEventDestroy(e);
  cudaFree(c->S);
  cudaFree(c->mbits);
  cudaFree(c->hist);
  cudaFree(c->ghist);
  cudaFree(c->L.med);
  cudaFree(c->L.mad);
  cudaFree(c->L.amb);
  cudaFree(c->L.cls);
  cudaFree(c->st);
  cudaFree(c->sig_out);
  cudaFree(c->stage_cube);
  cudaFree(c->stage_mask);
  cudaFree(c->ns_sig);
  cudaFree(c->ns_rinv);
  cudaFree(c->lk_chunk);
  cudaFree(c->lk_tot);
  cudaFree(c->lk_comp);
  cudaFree(c->af_buf);
  cudaFree(c->sh_P);
  cudaFree(c->sh_nf);
  cudaFree(c->sh_snap);
  cudaFree(c->sh_cnt);
  cudaFree(c->sh_offs);
  cudaFree(c->sh_bsum);
  cudaFree(c->sh_ent);
  cudaFree(c->sh_ss);
  if (c->st_host) cudaFreeHost(c->st_host);
  for (int i = 0; i < 2; ++i) {
    cudaFree(c->hm_in[i]);
    cudaFree(c->hm_mask[i]);
    cudaFree(c->hm_scale[i]);
  }
  if (c->hm_copy) cudaStreamDestroy(c->hm_copy);
  for (cudaEvent_t e : c->hm_ev)
    if (e) cudaEventDestroy(e);
  if (c->hm_res) cudaFreeHost(c->hm_res);
  cudaFree(c->batch_res);
  if (c->batch_res_host) cudaFreeHost(c->batch_res_host);
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  if (c->graph) cudaGraphDestroy(c->graph);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  for (sc_ctx* l : c->lanes)
    if (l != c) sc_destroy(l);  // lane 0 is the context itself
  for (cudaStream_t ls : c->lane_streams) cudaStreamDestroy(ls);
  for (cudaEvent_t e : c->lane_done) cudaEventDestroy(e);
  if (c->fork) cudaEventDestroy(c->fork);
  for (auto& j : c->jobs) {
    cudaEventDestroy(j.done);
    cudaFreeHost(j.slot);
  }
  for (cudaEvent_t e : c->job_events) cudaEventDestroy(e);
  for (unsigned char* p : c->job_slots) cudaFreeHost(p);
  if (c->clock_ev) cudaEventDestroy(c->clock_ev);
  cudaGetLastError();
  delete c;
}

int sc_run(sc_ctx* c, const float* cube_dev, const int64_t* dims, const sc_kernel* kernels, int n_kernels,
           float threshold, int noise_mode, float replacement, uint8_t* mask_dev, double* sigma_host,
           double* sigma0_host, uint32_t flags, void* cuda_stream) {
  if (!c) return SC_ERR_ARG;
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  c->last = s;
  int rc = run_device(c, cube_dev, dims, kernels, n_kernels, threshold, noise_mode, replacement, mask_dev, flags, s);
  if (rc) return rc;
  rc = finish(c, n_kernels, sigma_host, sigma0_host, s, false);
  if (rc == SC_OK) c->stats.runs += 1;
  return rc;
}

namespace {

// The batch lanes (created on first use, same workspace size as the context).
int ensure_lanes(sc_ctx* c) {
  if (!c->lanes.empty()) return SC_OK;
  if (cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming) != cudaSuccess) return SC_ERR_CUDA;
  for (int l = 0; l < kBatchLanes; ++l) {
    sc_ctx* lc = nullptr;
    if (l > 0) {
      const int rc = sc_create(&lc, c->device, c->max_voxels);
      if (rc) return rc;
    }
    cudaStream_t ls = nullptr;
    cudaEvent_t ev = nullptr;
    if (cudaStreamCreateWithFlags(&ls, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
      if (lc) sc_destroy(lc);
      cudaGetLastError();
      return SC_ERR_CUDA;
    }
    c->lanes.push_back(l == 0 ? c : lc);
    c->lane_streams.push_back(ls);
    c->lane_done.push_back(ev);
  }
  return SC_OK;
}

// Per-cube results of a batch, copied out of DevState after each cube.
struct BatchRes {
  unsigned int status, warn;
  float sigma0;
  float sigma[SC_MAX_KERNELS];
};
static_assert(offsetof(DevState, status) == 0 && offsetof(DevState, warn) == 4 && offsetof(DevState, sigma0) == 8,
              "status, warn and sigma_0 lead DevState");

unsigned long long fnv1a(unsigned long long h, const void* p, size_t n) {
  const unsigned char* b = static_cast<const unsigned char*>(p);
  for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
  return h;
}

int status_code(unsigned int status) {
  DevState h;
  memset(&h, 0, sizeof(h));
  h.status = status;
  return status_to_code(h);
}

}  // namespace

int sc_run_batch(sc_ctx* c, int n_cubes, const float* const* cubes, const int64_t* dims, const sc_kernel* kernels,
                 int n_kernels, float threshold, int noise_mode, float replacement, uint8_t* const* masks,
                 double* sigma_host, double* sigma0_host, uint32_t flags, void* cuda_stream) {
  if (!c || n_cubes < 1 || !cubes || !dims || !masks || !kernels) return SC_ERR_ARG;
  if (n_kernels < 1 || n_kernels > SC_MAX_KERNELS || !std::isfinite(replacement)) return SC_ERR_ARG;
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  c->last = s;
  // validate every cube before anything is enqueued
  for (int i = 0; i < n_cubes; ++i) {
    if (!cubes[i] || !masks[i]) return SC_ERR_ARG;
    long long n = 0;
    std::vector<PairDesc> pds;
    const int rc =
        validate_common(c, cubes[i], dims + 3 * i, kernels, n_kernels, threshold, noise_mode, &n, &pds, flags);
    if (rc) return rc;
  }
  const size_t need = sizeof(BatchRes) * (size_t)n_cubes;
  if (need > c->batch_res_cap) {
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->graph_exec = nullptr;
    c->graph = nullptr;
    cudaFree(c->batch_res);
    if (c->batch_res_host) cudaFreeHost(c->batch_res_host);
    c->batch_res = c->batch_res_host = nullptr;
    c->batch_res_cap = 0;
    if (cudaMalloc(&c->batch_res, need) != cudaSuccess ||
        cudaHostAlloc(&c->batch_res_host, need, cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      return SC_ERR_NOMEM;
    }
    c->batch_res_cap = need;
  }
  BatchRes* res = reinterpret_cast<BatchRes*>(c->batch_res);
  const uint32_t rflags = flags & ~(uint32_t)SC_FLAG_GRAPH;
  int rc_lanes = ensure_lanes(c);
  if (rc_lanes) return rc_lanes;
  const int n_lanes = (int)std::min<size_t>(c->lanes.size(), (size_t)n_cubes);
  if (!(flags & (SC_FLAG_NO_SHARE | SC_FLAG_GENERIC))) {
    // shared-pass buffers for the largest cube, made before any capture (a
    // lane that cannot get them smooths every pair in full)
    ShareNeeds m{0, 0, 0};
    for (int i = 0; i < n_cubes; ++i) {
      const ShareNeeds nd = share_needs(dims + 3 * i);
      m.p = std::max(m.p, nd.p);
      m.bk = std::max(m.bk, nd.bk);
      m.nf = std::max(m.nf, nd.nf);
    }
    for (int l = 0; l < n_lanes; ++l) ensure_share_sized(c->lanes[l], m);
  }
  // Cube i runs on lane i % n_lanes; the lanes' streams fork from q and join
  // back into it, so cubes on different lanes overlap.
  auto enqueue = [&](cudaStream_t q) -> int {
    CK(cudaEventRecord(c->fork, q));
    for (int l = 0; l < n_lanes; ++l) {
      sc_ctx* lc = c->lanes[l];
      if (lc != c) {
        lc->tune = c->tune;
        lc->profiling = c->profiling;
        lc->capturing = c->capturing;
      }
      CK(cudaStreamWaitEvent(c->lane_streams[l], c->fork, 0));
    }
    for (int i = 0; i < n_cubes; ++i) {
      const int l = i % n_lanes;
      sc_ctx* lc = c->lanes[l];
      cudaStream_t ls = c->lane_streams[l];
      const int rc = run_device(lc, cubes[i], dims + 3 * i, kernels, n_kernels, threshold, noise_mode, replacement,
                                masks[i], rflags, ls);
      if (rc) return rc;
      CK(cudaMemcpyAsync(&res[i], lc->st, 3 * sizeof(unsigned int), cudaMemcpyDeviceToDevice, ls));
      CK(cudaMemcpyAsync(res[i].sigma, lc->st->sigma, sizeof(float) * n_kernels, cudaMemcpyDeviceToDevice, ls));
    }
    for (int l = 0; l < n_lanes; ++l) {
      CK(cudaEventRecord(c->lane_done[l], c->lane_streams[l]));
      CK(cudaStreamWaitEvent(q, c->lane_done[l], 0));
      sc_ctx* lc = c->lanes[l];
      if (lc != c) {  // the lanes' launch counts, kernels and timing events belong to the context
        c->stats.launches += lc->stats.launches;
        lc->stats.launches = 0;
        memcpy(c->stats.smooth_kernel_pair, lc->stats.smooth_kernel_pair, sizeof(c->stats.smooth_kernel_pair));
        c->events.insert(c->events.end(), lc->events.begin(), lc->events.end());
        lc->events.clear();
      }
    }
    return SC_OK;
  };
  if (flags & SC_FLAG_GRAPH) {
    unsigned long long key = 1469598103934665603ull;
    key = fnv1a(key, &n_cubes, sizeof(n_cubes));
    key = fnv1a(key, cubes, sizeof(*cubes) * n_cubes);
    key = fnv1a(key, dims, sizeof(*dims) * 3 * n_cubes);
    key = fnv1a(key, masks, sizeof(*masks) * n_cubes);
    key = fnv1a(key, kernels, sizeof(*kernels) * n_kernels);
    key = fnv1a(key, &n_kernels, sizeof(n_kernels));
    key = fnv1a(key, &threshold, sizeof(threshold));
    key = fnv1a(key, &noise_mode, sizeof(noise_mode));
    key = fnv1a(key, &replacement, sizeof(replacement));
    key = fnv1a(key, &rflags, sizeof(rflags));
    key = fnv1a(key, &c->batch_res, sizeof(c->batch_res));
    for (const auto& kv : c->tune) {
      key = fnv1a(key, kv.first.data(), sizeof(long long) * kv.first.size());
      key = fnv1a(key, kv.second.data(), sizeof(int) * kv.second.size());
    }
    if (!c->graph_exec || key != c->graph_key) {
      if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
      if (c->graph) cudaGraphDestroy(c->graph);
      c->graph_exec = nullptr;
      c->graph = nullptr;
      if (!c->cap_stream) CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
      const unsigned long long l0 = c->stats.launches;
      CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
      c->capturing = true;
      const int rc = enqueue(c->cap_stream);
      cudaGraph_t gr = nullptr;
      const cudaError_t ec = cudaStreamEndCapture(c->cap_stream, &gr);
      c->capturing = false;
      if (rc != SC_OK || ec != cudaSuccess) {
        if (gr) cudaGraphDestroy(gr);
        cudaGetLastError();
        return rc != SC_OK ? rc : cuda_fail(ec, "cudaStreamEndCapture", __LINE__);
      }
      const cudaError_t ei = cudaGraphInstantiate(&c->graph_exec, gr, 0);
      if (ei != cudaSuccess) {
        cudaGraphDestroy(gr);
        c->graph_exec = nullptr;
        return cuda_fail(ei, "cudaGraphInstantiate", __LINE__);
      }
      c->graph = gr;
      c->graph_key = key;
      c->graph_launches = c->stats.launches - l0;
      c->stats.launches = l0;  // counted per replay
    }
    CK(cudaGraphLaunch(c->graph_exec, s));
    c->stats.launches += c->graph_launches;
  } else {
    const int rc = enqueue(s);
    if (rc) return rc;
  }
  if (!sigma_host && !sigma0_host) return SC_OK;
  CK(cudaMemcpyAsync(c->batch_res_host, res, need, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const BatchRes* h = reinterpret_cast<const BatchRes*>(c->batch_res_host);
  int first = SC_OK;
  c->stats.warnings = 0;
  for (int i = 0; i < n_cubes; ++i) {
    const int code = status_code(h[i].status);
    if (code != SC_OK && first == SC_OK) first = code;
    c->stats.warnings |= h[i].warn;
    if (sigma0_host) sigma0_host[i] = code == SC_OK ? (double)h[i].sigma0 : 0.0;
    if (sigma_host)
      for (int k = 0; k < n_kernels; ++k) sigma_host[(size_t)i * n_kernels + k] = code == SC_OK ? (double)h[i].sigma[k] : 0.0;
  }
  if (first == SC_OK) c->stats.runs += (unsigned long long)n_cubes;
  return first;
}

namespace {

double host_seconds() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace

int sc_set_budget(sc_ctx* c, uint64_t bytes) {
  if (!c) return SC_ERR_ARG;
  c->budget = bytes;
  return SC_OK;
}

int sc_submit(sc_ctx* c, const void* cube_dev, int storage, const float* chan_scale_dev, const int64_t* dims,
              const sc_kernel* kernels, int n_kernels, float threshold, int noise_mode, float replacement,
              uint8_t* mask_dev, uint32_t flags, int64_t* job_id, void* cuda_stream) {
  if (!c || !cube_dev || !mask_dev || !job_id) return SC_ERR_ARG;
  if (storage != SC_STORE_F32 && storage != SC_STORE_BF16 && storage != SC_STORE_FP16) return SC_ERR_ARG;
  if (storage != SC_STORE_F32 && !chan_scale_dev) return SC_ERR_ARG;
  DeviceGuard g(c->device);
  long long n = 0;
  std::vector<PairDesc> pds;
  int rc = validate_common(c, storage == SC_STORE_F32 ? (const float*)cube_dev : c->S, dims, kernels, n_kernels,
                           threshold, noise_mode, &n, &pds, flags);
  if (rc) return rc;
  if (!std::isfinite(replacement)) return SC_ERR_ARG;
  const unsigned long long bytes = (unsigned long long)n * ((storage == SC_STORE_F32 ? 4u : 2u) + 1u);
  if (c->budget && c->in_flight + bytes > c->budget) return SC_ERR_BUDGET;
  rc = ensure_lanes(c);
  if (rc) return rc;
  if (!c->clock_ev) {
    // device-to-host clock reference: an event completed at a known host time
    if (cudaEventCreate(&c->clock_ev) != cudaSuccess || cudaEventRecord(c->clock_ev, c->lane_streams[0]) != cudaSuccess ||
        cudaEventSynchronize(c->clock_ev) != cudaSuccess) {
      cudaGetLastError();
      return SC_ERR_CUDA;
    }
    c->clock_host = host_seconds();
  }
  // jobs use the lanes other than the context itself, round robin
  const int n_job_lanes = (int)c->lanes.size() - 1;
  const int l = 1 + (int)((c->next_job - 1) % n_job_lanes);
  sc_ctx* lc = c->lanes[l];
  cudaStream_t ls = c->lane_streams[l];
  lc->tune = c->tune;
  lc->profiling = 0;
  // the job starts after the work already enqueued on the caller's stream
  CK(cudaEventRecord(c->fork, (cudaStream_t)cuda_stream));
  CK(cudaStreamWaitEvent(ls, c->fork, 0));
  cudaEvent_t done = nullptr;
  if (!c->job_events.empty()) {
    done = c->job_events.back();
    c->job_events.pop_back();
  } else {
    CK(cudaEventCreate(&done));
  }
  unsigned char* slot = nullptr;
  if (!c->job_slots.empty()) {
    slot = c->job_slots.back();
    c->job_slots.pop_back();
  } else if (cudaHostAlloc(&slot, sizeof(BatchRes), cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    c->job_events.push_back(done);
    return SC_ERR_NOMEM;
  }
  const double t_submit = host_seconds();
  const float* src = (const float*)cube_dev;
  const bool h_in = storage != SC_STORE_F32 && half_in_kernel(cube_dev, dims);
  const Half16 h{(const unsigned short*)cube_dev, chan_scale_dev, storage};
  if (storage != SC_STORE_F32 && !h_in) {
    rc = ensure_stage(lc);
    if (rc == SC_OK && launch_decode_half((const uint16_t*)cube_dev, chan_scale_dev, (long long)dims[0] * dims[1], n,
                                         storage == SC_STORE_BF16 ? 1 : 0, lc->stage_cube, lc->sms, ls) != cudaSuccess)
      rc = cuda_fail(cudaGetLastError(), "launch_decode_half", __LINE__);
    src = lc->stage_cube;
  }
  if (rc == SC_OK)
    rc = run_device(lc, h_in ? nullptr : src, dims, kernels, n_kernels, threshold, noise_mode, replacement, mask_dev,
                    h_in ? half_flags(flags) : flags & ~(uint32_t)SC_FLAG_HALF_DIRECT, ls, h_in ? &h : nullptr);
  if (rc == SC_OK) {
    BatchRes* r = reinterpret_cast<BatchRes*>(slot);
    if (cudaMemcpyAsync(r, lc->st, 3 * sizeof(unsigned int), cudaMemcpyDeviceToHost, ls) != cudaSuccess ||
        cudaMemcpyAsync(r->sigma, lc->st->sigma, sizeof(float) * n_kernels, cudaMemcpyDeviceToHost, ls) !=
            cudaSuccess ||
        cudaEventRecord(done, ls) != cudaSuccess)
      rc = cuda_fail(cudaGetLastError(), "sc_submit", __LINE__);
  }
  c->stats.launches += lc->stats.launches + (storage != SC_STORE_F32 && !h_in ? 1 : 0);
  lc->stats.launches = 0;
  memcpy(c->stats.smooth_kernel_pair, lc->stats.smooth_kernel_pair, sizeof(c->stats.smooth_kernel_pair));
  if (rc) {
    c->job_events.push_back(done);
    c->job_slots.push_back(slot);
    return rc;
  }
  c->jobs.push_back({c->next_job, l, n_kernels, done, t_submit, bytes, slot});
  c->in_flight += bytes;
  *job_id = c->next_job++;
  return SC_OK;
}

int sc_poll(sc_ctx* c, int wait, int64_t* job_id, int* status, double* latency_s, double* sigma_host,
            double* sigma0_host) {
  if (!c || !job_id) return SC_ERR_ARG;
  if (c->jobs.empty()) return 0;
  DeviceGuard g(c->device);
  for (;;) {
    for (auto it = c->jobs.begin(); it != c->jobs.end(); ++it) {
      const cudaError_t q = cudaEventQuery(it->done);
      if (q == cudaErrorNotReady) continue;
      if (q != cudaSuccess) return cuda_fail(q, "cudaEventQuery", __LINE__);
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, c->clock_ev, it->done);
      const BatchRes* r = reinterpret_cast<const BatchRes*>(it->slot);
      const int code = status_code(r->status);
      *job_id = it->id;
      if (status) *status = code;
      if (latency_s) *latency_s = c->clock_host + 1e-3 * ms - it->t_submit;
      if (sigma0_host) *sigma0_host = code == SC_OK ? (double)r->sigma0 : 0.0;
      if (sigma_host)
        for (int k = 0; k < it->n_kernels; ++k) sigma_host[k] = code == SC_OK ? (double)r->sigma[k] : 0.0;
      c->stats.warnings = r->warn;
      if (code == SC_OK) c->stats.runs += 1;
      c->in_flight -= it->bytes;
      c->job_events.push_back(it->done);
      c->job_slots.push_back(it->slot);
      c->jobs.erase(it);
      return 1;
    }
    if (!wait) return 0;
    const cudaError_t e = cudaEventSynchronize(c->jobs.front().done);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize", __LINE__);
  }
}

int sc_autotune(sc_ctx* c, const int64_t* dims, const sc_kernel* kernels, int n_kernels, void* cuda_stream) {
  if (!c || !dims || !kernels || n_kernels < 1 || n_kernels > SC_MAX_KERNELS) return SC_ERR_ARG;
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  c->last = s;
  long long n = 0;
  int rc = check_dims(c, dims, &n);
  if (rc) return rc;
  std::vector<PairDesc> pds(n_kernels);
  for (int k = 0; k < n_kernels; ++k) {
    rc = make_pair(kernels[k], &pds[k]);
    if (rc) return rc;
  }
  rc = ensure_stage(c);
  if (rc) return rc;
  // a synthetic cube of the requested shape (uniform noise) and an empty mask
  CK(launch_fill_noise(c->stage_cube, n, 20210630u, c->sms, s));
  CK(cudaMemsetAsync(c->mbits, 0, sizeof(uint32_t) * ((n + 31) / 32), s));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  struct Cand {
    int kind, zf;
  };
  std::map<std::array<long long, 7>, std::array<int, 2>> done;
  int out = SC_OK;
  for (int k = 0; k < n_kernels && out == SC_OK; ++k) {
    const PairDesc& pd = pds[k];
    if (pd.h == 0 && pd.wz <= 1) continue;  // identity: nothing to choose
    const auto key = tune_key(dims, pd);
    if (done.count(key)) continue;
    std::vector<Cand> cands;
    for (int zf : {0, 2, 4}) {  // 0: the chunking of the balance model
      if (pd.h > 0) {
        cands.push_back({TUNE_WS, zf});
        cands.push_back({TUNE_WS16, zf});
        cands.push_back({TUNE_TILE, zf});
      } else {
        cands.push_back({TUNE_Z8, zf});
        cands.push_back({TUNE_Z4, zf});
        if (pd.wz <= 15) cands.push_back({TUNE_Z4W, zf});
        if (pd.wz <= 7) cands.push_back({TUNE_Z8W, zf});
      }
    }
    // fixed-point scales of this pair on the synthetic cube, replacement value 1
    PairWeights W{};
    W.w[0] = pd.W;
    W.wf[0] = pd.Wf;
    if (cudaMemsetAsync(c->st, 0, sizeof(DevState), s) != cudaSuccess ||
        launch_maxabs(c->stage_cube, n, c->st, c->sms, s) != cudaSuccess ||
        launch_fx_setup(c->st, 1.0f, W, 1, s) != cudaSuccess) {
      out = cuda_fail(cudaGetLastError(), "autotune setup", __LINE__);
      break;
    }
    float best = 1e30f;
    std::array<int, 2> choice{TUNE_AUTO, 0};
    for (const Cand& cd : cands) {
      SmoothArgs a = base_args(c, c->stage_cube, dims);
      a.pd = pd;
      a.pair = 0;
      a.hist = c->hist;
      a.win = 0;
      a.repl_possible = 1;
      a.tune_kind = cd.kind;
      a.tune_zfactor = cd.zf;
      cudaError_t e = launch_smooth(a, c->sms, s, nullptr);  // warm-up
      e = e == cudaSuccess ? cudaEventRecord(e0, s) : e;
      for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = launch_smooth(a, c->sms, s, nullptr);
      e = e == cudaSuccess ? cudaEventRecord(e1, s) : e;
      e = e == cudaSuccess ? cudaEventSynchronize(e1) : e;
      float ms = 0.0f;
      e = e == cudaSuccess ? cudaEventElapsedTime(&ms, e0, e1) : e;
      if (e != cudaSuccess) {
        out = cuda_fail(e, "autotune candidate", __LINE__);
        break;
      }
      if (ms < best) {
        best = ms;
        choice = {cd.kind, cd.zf};
      }
    }
    done[key] = choice;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (out == SC_OK)
    for (const auto& kv : done) c->tune[kv.first] = kv.second;
  return out;
}

int sc_run_half(sc_ctx* c, const uint16_t* cube_dev, int is_bf16, const float* chan_scale_dev, const int64_t* dims,
                const sc_kernel* kernels, int n_kernels, float threshold, int noise_mode, float replacement,
                uint8_t* mask_dev, double* sigma_host, double* sigma0_host, uint32_t flags, void* cuda_stream) {
  if (!c || !cube_dev || !chan_scale_dev || !mask_dev) return SC_ERR_ARG;
  DeviceGuard g(c->device);
  long long n = 0;
  int rc = check_dims(c, dims, &n);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  c->last = s;
  if (half_in_kernel(cube_dev, dims)) {
    const Half16 h{cube_dev, chan_scale_dev, is_bf16 ? SC_STORE_BF16 : SC_STORE_FP16};
    rc = run_device(c, nullptr, dims, kernels, n_kernels, threshold, noise_mode, replacement, mask_dev,
                    half_flags(flags), s, &h);
  } else {
    rc = ensure_stage(c);
    if (rc) return rc;
    {
      Phase ph(c, s, EV_CLIP);
      CK(launch_decode_half(cube_dev, chan_scale_dev, (long long)dims[0] * dims[1], n, is_bf16 ? 1 : 0,
                            c->stage_cube, c->sms, s));
      c->stats.launches += 1;
    }
    rc = run_device(c, c->stage_cube, dims, kernels, n_kernels, threshold, noise_mode, replacement, mask_dev,
                    flags & ~(uint32_t)SC_FLAG_HALF_DIRECT, s);
    c->stats.half_path = 2u;
  }
  if (rc) return rc;
  rc = finish(c, n_kernels, sigma_host, sigma0_host, s, false);
  if (rc == SC_OK) c->stats.runs += 1;
  return rc;
}

int sc_run_host(sc_ctx* c, const float* cube_host, const int64_t* dims, const sc_kernel* kernels, int n_kernels,
                float threshold, int noise_mode, float replacement, uint8_t* mask_host, double* sigma_host,
                double* sigma0_host, uint32_t flags, void* cuda_stream) {
  if (!c || !cube_host || !mask_host) return SC_ERR_ARG;
  DeviceGuard g(c->device);
  long long n = 0;
  int rc = check_dims(c, dims, &n);
  if (rc) return rc;
  rc = ensure_stage(c);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  c->last = s;
  CK(cudaMemcpyAsync(c->stage_cube, cube_host, sizeof(float) * n, cudaMemcpyHostToDevice, s));
  if (flags & SC_FLAG_ACCUMULATE) CK(cudaMemcpyAsync(c->stage_mask, mask_host, n, cudaMemcpyHostToDevice, s));
  rc = run_device(c, c->stage_cube, dims, kernels, n_kernels, threshold, noise_mode, replacement, c->stage_mask, flags,
                  s);
  if (rc) return rc;
  CK(cudaMemcpyAsync(mask_host, c->stage_mask, n, cudaMemcpyDeviceToHost, s));
  rc = finish(c, n_kernels, sigma_host, sigma0_host, s, true);
  if (rc == SC_OK) c->stats.runs += 1;
  return rc;
}

int sc_run_host_many(sc_ctx* c, int n_cubes, const void* const* cubes_host, int storage,
                     const float* const* chan_scales_host, const int64_t* dims, const sc_kernel* kernels,
                     int n_kernels, float threshold, int noise_mode, float replacement, uint8_t* const* masks_host,
                     double* sigma_host, double* sigma0_host, uint32_t flags, void* cuda_stream) {
  if (!c || n_cubes < 1 || !cubes_host || !masks_host || !dims) return SC_ERR_ARG;
  if (storage != SC_STORE_F32 && storage != SC_STORE_BF16 && storage != SC_STORE_FP16) return SC_ERR_ARG;
  if (storage != SC_STORE_F32 && !chan_scales_host) return SC_ERR_ARG;
  if (n_kernels < 1 || n_kernels > SC_MAX_KERNELS || !std::isfinite(replacement)) return SC_ERR_ARG;
  for (int i = 0; i < n_cubes; ++i)
    if (!cubes_host[i] || !masks_host[i] || (storage != SC_STORE_F32 && !chan_scales_host[i])) return SC_ERR_ARG;
  DeviceGuard g(c->device);
  long long n = 0;
  int rc = check_dims(c, dims, &n);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  c->last = s;
  const size_t in_bytes = (storage == SC_STORE_F32 ? 4u : 2u) * (size_t)n;
  const size_t nz = (size_t)dims[2];
  // buffers, copy stream and events (first use)
  for (int b = 0; b < 2; ++b) {
    if (!c->hm_in[b] && cudaMalloc(&c->hm_in[b], sizeof(float) * c->max_voxels) != cudaSuccess) {
      cudaGetLastError();
      return SC_ERR_NOMEM;
    }
    if (!c->hm_mask[b] && cudaMalloc(&c->hm_mask[b], c->max_voxels) != cudaSuccess) {
      cudaGetLastError();
      return SC_ERR_NOMEM;
    }
  }
  if (storage != SC_STORE_F32 && nz > c->hm_scale_cap) {
    for (int b = 0; b < 2; ++b) {
      cudaFree(c->hm_scale[b]);
      c->hm_scale[b] = nullptr;
    }
    c->hm_scale_cap = 0;
    for (int b = 0; b < 2; ++b)
      if (cudaMalloc(&c->hm_scale[b], sizeof(float) * nz) != cudaSuccess) {
        cudaGetLastError();
        return SC_ERR_NOMEM;
      }
    c->hm_scale_cap = nz;
  }
  if (!c->hm_copy) CK(cudaStreamCreateWithFlags(&c->hm_copy, cudaStreamNonBlocking));
  for (cudaEvent_t& e : c->hm_ev)
    if (!e) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  const size_t need = sizeof(BatchRes) * (size_t)n_cubes;
  if (need > c->hm_res_cap) {
    if (c->hm_res) cudaFreeHost(c->hm_res);
    c->hm_res = nullptr;
    c->hm_res_cap = 0;
    if (cudaHostAlloc(&c->hm_res, need, cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      return SC_ERR_NOMEM;
    }
    c->hm_res_cap = need;
  }
  cudaEvent_t* loaded = c->hm_ev;
  cudaEvent_t* computed = c->hm_ev + 2;
  cudaEvent_t* sent = c->hm_ev + 4;
  cudaStream_t cp = c->hm_copy;
  BatchRes* res = reinterpret_cast<BatchRes*>(c->hm_res);
  auto load = [&](int i, int b) -> int {
    CK(cudaMemcpyAsync(c->hm_in[b], cubes_host[i], in_bytes, cudaMemcpyHostToDevice, cp));
    if (storage != SC_STORE_F32)
      CK(cudaMemcpyAsync(c->hm_scale[b], chan_scales_host[i], sizeof(float) * nz, cudaMemcpyHostToDevice, cp));
    if (flags & SC_FLAG_ACCUMULATE) CK(cudaMemcpyAsync(c->hm_mask[b], masks_host[i], n, cudaMemcpyHostToDevice, cp));
    CK(cudaEventRecord(loaded[b], cp));
    return SC_OK;
  };
  // The copy stream starts after the work enqueued on s; cube i + 1 is copied
  // in, and cube i - 1's mask out, while cube i computes on s.
  CK(cudaEventRecord(computed[1], s));
  CK(cudaStreamWaitEvent(cp, computed[1], 0));
  rc = load(0, 0);
  if (rc) return rc;
  for (int i = 0; i < n_cubes; ++i) {
    const int b = i & 1, nb = b ^ 1;
    if (i + 1 < n_cubes) {
      if (i >= 1) CK(cudaStreamWaitEvent(cp, computed[nb], 0));  // cube i - 1 is done with that set
      if (i >= 1) CK(cudaStreamWaitEvent(cp, sent[nb], 0));
      rc = load(i + 1, nb);
      if (rc) return rc;
    }
    CK(cudaStreamWaitEvent(s, loaded[b], 0));
    if (i >= 2) CK(cudaStreamWaitEvent(s, sent[b], 0));  // its mask of cube i - 2 has left the device
    if (storage == SC_STORE_F32) {
      rc = run_device(c, static_cast<const float*>(c->hm_in[b]), dims, kernels, n_kernels, threshold, noise_mode,
                      replacement, c->hm_mask[b], flags & ~(uint32_t)SC_FLAG_HALF_DIRECT, s);
    } else if (half_in_kernel(c->hm_in[b], dims)) {
      const Half16 h{static_cast<const unsigned short*>(c->hm_in[b]), c->hm_scale[b], storage};
      rc = run_device(c, nullptr, dims, kernels, n_kernels, threshold, noise_mode, replacement, c->hm_mask[b],
                      half_flags(flags), s, &h);
    } else {
      rc = ensure_stage(c);
      if (rc) return rc;
      CK(launch_decode_half(static_cast<const uint16_t*>(c->hm_in[b]), c->hm_scale[b], dims[0] * dims[1], n,
                            storage == SC_STORE_BF16 ? 1 : 0, c->stage_cube, c->sms, s));
      c->stats.launches += 1;
      rc = run_device(c, c->stage_cube, dims, kernels, n_kernels, threshold, noise_mode, replacement, c->hm_mask[b],
                      flags & ~(uint32_t)SC_FLAG_HALF_DIRECT, s);
    }
    if (rc) return rc;
    CK(cudaMemcpyAsync(&res[i], c->st, 3 * sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(res[i].sigma, c->st->sigma, sizeof(float) * n_kernels, cudaMemcpyDeviceToHost, s));
    CK(cudaEventRecord(computed[b], s));
    CK(cudaStreamWaitEvent(cp, computed[b], 0));
    CK(cudaMemcpyAsync(masks_host[i], c->hm_mask[b], n, cudaMemcpyDeviceToHost, cp));
    CK(cudaEventRecord(sent[b], cp));
  }
  CK(cudaStreamWaitEvent(s, sent[(n_cubes - 1) & 1], 0));
  CK(cudaStreamSynchronize(s));
  int first = SC_OK;
  c->stats.warnings = 0;
  for (int i = 0; i < n_cubes; ++i) {
    const int code = status_code(res[i].status);
    if (code != SC_OK && first == SC_OK) first = code;
    c->stats.warnings |= res[i].warn;
    if (sigma0_host) sigma0_host[i] = code == SC_OK ? (double)res[i].sigma0 : 0.0;
    if (sigma_host)
      for (int k = 0; k < n_kernels; ++k)
        sigma_host[(size_t)i * n_kernels + k] = code == SC_OK ? (double)res[i].sigma[k] : 0.0;
  }
  if (first == SC_OK) c->stats.runs += (unsigned long long)n_cubes;
  return first;
}

int sc_smooth(sc_ctx* c, const float* cube_dev, const int64_t* dims, sc_kernel kernel, const uint8_t* mask_dev,
              float replacement_value, float* out_dev, uint32_t flags, void* cuda_stream) {
  if (!c || !cube_dev || !out_dev || (const void*)cube_dev == (const void*)out_dev) return SC_ERR_ARG;
  if (((flags >> 16) & 0xffu) > (unsigned)SC_VARIANT_Z8_512) return SC_ERR_ARG;
  if (!std::isfinite(replacement_value)) return SC_ERR_ARG;
  DeviceGuard g(c->device);
  long long n = 0;
  int rc = check_dims(c, dims, &n);
  if (rc) return rc;
  PairDesc pd;
  rc = make_pair(kernel, &pd, (flags & SC_FLAG_SAMPLED_GAUSS) != 0);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  c->last = s;
  CK(cudaMemsetAsync(c->st, 0, sizeof(DevState), s));
  if (mask_dev) {
    CK(launch_pack(mask_dev, cube_dev, n, c->mbits, s));
    c->stats.launches += 1;
  }
  const float repl = replacement_value > 0.0f ? replacement_value : 0.0f;  // quantised exactly per pair
  PairWeights W{};
  W.w[0] = pd.W;
  W.wf[0] = pd.Wf;
  CK(launch_maxabs(cube_dev, n, c->st, c->sms, s));
  CK(launch_fx_setup(c->st, repl, W, 1, s));
  c->stats.launches += 2;
  SmoothArgs a = base_args(c, cube_dev, dims);
  a.mbits = mask_dev ? c->mbits : nullptr;
  a.S = out_dev;
  a.pd = pd;
  a.pair = 0;
  a.use_fixed_repl = 1;
  a.repl_value = repl;
  a.hist = nullptr;
  a.generic = (flags & SC_FLAG_GENERIC) ? 1 : 0;
  a.repl_possible = repl > 0.0f ? 1 : 0;
  a.tune_kind = (int)((flags >> 16) & 0xffu);  // a variant chosen by the caller (SC_SMOOTH_VARIANT)
  {
    Phase ph(c, s, EV_SMOOTH, (unsigned long long)n, 0);
    if (pd.h == 0 && pd.wz == 1) {
      CK(launch_identity(a, c->sms, s));
      c->stats.launches += 1;
      c->stats.smooth_kernel_pair[0] = SC_KERNEL_IDENTITY;
    } else {
      int l = 0, code = SC_KERNEL_NONE;
      CK(launch_smooth(a, c->sms, s, &l, &code));
      c->stats.launches += l;
      c->stats.smooth_kernel_pair[0] = code;
    }
  }
  return SC_OK;
}

int sc_copy_smoothed(sc_ctx* c, float* dst, int64_t n, void* cuda_stream) {
  if (!c || !dst || n < 0) return SC_ERR_ARG;
  if ((unsigned long long)n > c->max_voxels) return SC_ERR_BUDGET;
  DeviceGuard g(c->device);
  CK(cudaMemcpyAsync(dst, c->S, sizeof(float) * (size_t)n, cudaMemcpyDefault, (cudaStream_t)cuda_stream));
  return SC_OK;
}

int sc_test_skip_handoff(sc_ctx* c, int enable) {
  if (!c) return SC_ERR_ARG;
  c->test_skip_handoff = enable ? 1 : 0;
  return SC_OK;
}

int sc_set_share_limit(sc_ctx* c, uint64_t max_entries) {
  if (!c) return SC_ERR_ARG;
  c->sh_limit = max_entries;
  return SC_OK;
}

int sc_copy_sigmas(sc_ctx* c, float* sigma_dst, float* sigma0_dst, int n_kernels, void* cuda_stream) {
  if (!c || n_kernels < 1 || n_kernels > SC_MAX_KERNELS) return SC_ERR_ARG;
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  if (!sigma_dst && !sigma0_dst) return SC_OK;
  // staged by a kernel that writes zeros when the run's status is an error
  CK(launch_sigma_out(c->st, n_kernels, c->sig_out, s));
  c->stats.launches += 1;
  if (sigma_dst) CK(cudaMemcpyAsync(sigma_dst, c->sig_out, sizeof(float) * n_kernels, cudaMemcpyDefault, s));
  if (sigma0_dst) CK(cudaMemcpyAsync(sigma0_dst, c->sig_out + n_kernels, sizeof(float), cudaMemcpyDefault, s));
  return SC_OK;
}

int sc_noise(sc_ctx* c, const float* data_dev, int64_t n, int noise_mode, double* sigma_host, uint32_t flags,
             void* cuda_stream) {
  if (!c || !data_dev || !sigma_host || n <= 0) return SC_ERR_ARG;
  if ((unsigned long long)n > c->max_voxels) return SC_ERR_BUDGET;
  if (noise_mode != SC_NOISE_MAD && noise_mode != SC_NOISE_STD && noise_mode != SC_NOISE_GAUSS) return SC_ERR_ARG;
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  c->last = s;
  const unsigned int force = (flags & SC_FLAG_NO_FAST_SELECT) ? (PLAN_MED_FULL | PLAN_MAD_FULL) : 0u;
  CK(cudaMemsetAsync(c->st, 0, sizeof(DevState), s));
  CK(cudaMemsetAsync(c->hist, 0, sizeof(unsigned long long) * kNumBins, s));
  CK(launch_hist(data_dev, n, c->st, c->hist, 0, 0, c->sms, s));
  c->stats.launches += 1;
  int rc = measure(c, data_dev, n, 0, 1.0f, 0, noise_mode, SC_MAX_KERNELS, force, s);
  if (rc) return rc;
  CK(cudaMemcpyAsync(c->st_host, c->st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  rc = status_to_code(*c->st_host);
  *sigma_host = rc == SC_OK ? (double)c->st_host->sigma_cur : 0.0;
  return rc;
}

int sc_noise_scale(sc_ctx* c, const float* cube_dev, const int64_t* dims, const int32_t* window, const int32_t* grid,
                   int noise_mode, float* out_dev, double* sigma_host, uint32_t flags, void* cuda_stream) {
  (void)flags;
  if (!c || !cube_dev || !dims || !window || !grid || !out_dev) return SC_ERR_ARG;
  if (noise_mode != SC_NOISE_MAD && noise_mode != SC_NOISE_STD && noise_mode != SC_NOISE_GAUSS) return SC_ERR_ARG;
  long long d[3];
  int w[3], g[3];
  long long cells = 1, wvox = 1;
  for (int i = 0; i < 3; ++i) {
    d[i] = dims[i];
    w[i] = window[i];
    g[i] = grid[i];
    if (d[i] <= 0 || d[i] > (1LL << 31) - 1 || w[i] <= 0 || w[i] % 2 == 0 || g[i] <= 0) return SC_ERR_ARG;
    cells *= (d[i] + g[i] - 1) / g[i];
    wvox *= std::min((long long)w[i], d[i]);
  }
  if (wvox > kNoiseScaleMaxWindow) return SC_ERR_UNSUPPORTED;
  DeviceGuard guard(c->device);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  c->last = s;
  if ((size_t)cells > c->ns_cap) {
    cudaFree(c->ns_sig);
    cudaFree(c->ns_rinv);
    c->ns_sig = nullptr;
    c->ns_rinv = nullptr;
    c->ns_cap = 0;
    if (cudaMalloc(&c->ns_sig, sizeof(double) * cells) != cudaSuccess ||
        cudaMalloc(&c->ns_rinv, sizeof(float) * cells) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(c->ns_sig);
      cudaFree(c->ns_rinv);
      c->ns_sig = nullptr;
      c->ns_rinv = nullptr;
      return SC_ERR_NOMEM;
    }
    c->ns_cap = (size_t)cells;
  }
  {
    Phase ph(c, s, EV_NOISE_WINDOW);
    CK(launch_noise_window(cube_dev, d, w, g, noise_mode, c->ns_sig, c->ns_rinv, c->sms, s));
  }
  {
    Phase ph(c, s, EV_NOISE_APPLY);
    CK(launch_noise_apply(cube_dev, d, w, g, out_dev, c->ns_rinv, c->sms, s));
  }
  c->stats.launches += 2;
  if (sigma_host) {
    CK(cudaMemcpyAsync(sigma_host, c->ns_sig, sizeof(double) * cells, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  }
  return SC_OK;
}

int sc_link(sc_ctx* c, const uint8_t* mask_dev, const int64_t* dims, int r_xy, int r_z, int min_xy, int min_z,
            int max_xy, int max_z, int32_t* labels_dev, int64_t* n_out, int32_t* extents_host, int64_t extents_cap,
            uint32_t flags, void* cuda_stream) {
  (void)flags;
  if (!c || !mask_dev || !dims || !labels_dev || !n_out) return SC_ERR_ARG;
  if (r_xy < 0 || r_z < 0 || r_xy > kLinkMaxRadius || r_z > kLinkMaxRadius || min_xy < 0 || min_z < 0 || max_xy < 0 ||
      max_z < 0 || extents_cap < 0 || (extents_cap > 0 && !extents_host))
    return SC_ERR_ARG;
  long long d[3];
  long long n = 1;
  for (int i = 0; i < 3; ++i) {
    d[i] = dims[i];
    if (d[i] <= 0 || d[i] > INT32_MAX) return SC_ERR_ARG;
    n *= d[i];
    if (n >= (long long)INT32_MAX) return SC_ERR_ARG;  // voxel indices are int32
  }
  DeviceGuard guard(c->device);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  c->last = s;
  const long long chunks = link_chunks(n);
  if (!c->lk_tot && cudaMalloc(&c->lk_tot, sizeof(int) * 2) != cudaSuccess) {
    cudaGetLastError();
    c->lk_tot = nullptr;
    return SC_ERR_NOMEM;
  }
  if ((size_t)chunks > c->lk_chunk_cap) {
    cudaFree(c->lk_chunk);
    c->lk_chunk_cap = 0;
    if (cudaMalloc(&c->lk_chunk, sizeof(int) * chunks) != cudaSuccess) {
      cudaGetLastError();
      c->lk_chunk = nullptr;
      return SC_ERR_NOMEM;
    }
    c->lk_chunk_cap = (size_t)chunks;
  }
  CK(launch_link_components(mask_dev, d, r_xy, r_z, labels_dev, c->lk_chunk, c->lk_tot, c->sms, s));
  c->stats.launches += 4;
  int ncomp = 0;
  CK(cudaMemcpyAsync(&ncomp, c->lk_tot, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  int kept = 0;
  int *ext = nullptr, *ext_out = nullptr, *keep = nullptr, *new_id = nullptr;
  if (ncomp > 0) {
    if ((size_t)ncomp > c->lk_comp_cap) {
      cudaFree(c->lk_comp);
      c->lk_comp_cap = 0;
      if (cudaMalloc(&c->lk_comp, sizeof(int) * 16 * (size_t)ncomp) != cudaSuccess) {
        cudaGetLastError();
        c->lk_comp = nullptr;
        return SC_ERR_NOMEM;
      }
      c->lk_comp_cap = (size_t)ncomp;
    }
    ext = c->lk_comp;
    ext_out = ext + 7 * (size_t)ncomp;
    keep = ext_out + 7 * (size_t)ncomp;
    new_id = keep + (size_t)ncomp;
  }
  // numbering, final labels and extents, then the size filters
  CK(launch_link_filter(d, labels_dev, c->lk_chunk, ncomp, min_xy, min_z, max_xy, max_z, ext, keep, ext_out, new_id,
                        c->lk_tot, c->sms, s));
  c->stats.launches += ncomp > 0 ? 7 : 2;
  if (ncomp > 0) {
    CK(cudaMemcpyAsync(&kept, c->lk_tot, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const long long rows = std::min<long long>(kept, extents_cap);
    if (rows > 0) {
      CK(cudaMemcpyAsync(extents_host, ext_out, sizeof(int) * 7 * (size_t)rows, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
    }
  }
  *n_out = kept;
  return SC_OK;
}

int sc_autoflag(sc_ctx* c, const float* cube_dev, const int64_t* dims, double k, uint32_t what, int noise_mode,
                float* out_dev, uint8_t* chan_flags_host, uint8_t* pix_flags_host, float* chan_noise_host,
                float* pix_noise_host, int64_t* n_flagged, uint32_t flags, void* cuda_stream) {
  (void)flags;
  if (!c || !cube_dev || !dims || !out_dev || !(k >= 0.0) || what == 0u ||
      (what & ~(SC_AUTOFLAG_CHANNELS | SC_AUTOFLAG_PIXELS)))
    return SC_ERR_ARG;
  if (noise_mode != SC_NOISE_MAD && noise_mode != SC_NOISE_STD && noise_mode != SC_NOISE_GAUSS) return SC_ERR_ARG;
  long long d[3];
  for (int i = 0; i < 3; ++i) {
    d[i] = dims[i];
    if (d[i] <= 0 || d[i] > INT32_MAX) return SC_ERR_ARG;
  }
  const bool ch = (what & SC_AUTOFLAG_CHANNELS) != 0u, px = (what & SC_AUTOFLAG_PIXELS) != 0u;
  if (px && d[2] > kFlagMaxChannelsForPixels) return SC_ERR_UNSUPPORTED;
  const long long plane = d[0] * d[1];
  // layout: stats[4] doubles | chan noise [nz] | pix noise [plane] | chan flags [nz] | pix flags [plane]
  const size_t need = 64 + sizeof(float) * (size_t)(d[2] + plane) + (size_t)(d[2] + plane) + 16;
  DeviceGuard guard(c->device);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  c->last = s;
  if (need > c->af_cap) {
    cudaFree(c->af_buf);
    c->af_cap = 0;
    if (cudaMalloc(&c->af_buf, need) != cudaSuccess) {
      cudaGetLastError();
      c->af_buf = nullptr;
      return SC_ERR_NOMEM;
    }
    c->af_cap = need;
  }
  double* stats = reinterpret_cast<double*>(c->af_buf);
  float* cn = reinterpret_cast<float*>(c->af_buf + 64);
  float* pn = cn + d[2];
  uint8_t* cf = reinterpret_cast<uint8_t*>(pn + plane);
  uint8_t* pf = cf + d[2];
  CK(launch_autoflag(cube_dev, d, k, ch ? 1 : 0, px ? 1 : 0, noise_mode, out_dev, cn, pn, cf,
                     pf, stats, c->sms, s));
  c->stats.launches += (ch ? 3 : 0) + (px ? 3 : 0) + 1;
  const bool want_counts = n_flagged != nullptr;
  std::vector<uint8_t> cf_h, pf_h;
  if (ch && (chan_flags_host || want_counts)) {
    cf_h.resize((size_t)d[2]);
    CK(cudaMemcpyAsync(cf_h.data(), cf, (size_t)d[2], cudaMemcpyDeviceToHost, s));
  }
  if (px && (pix_flags_host || want_counts)) {
    pf_h.resize((size_t)plane);
    CK(cudaMemcpyAsync(pf_h.data(), pf, (size_t)plane, cudaMemcpyDeviceToHost, s));
  }
  if (ch && chan_noise_host) CK(cudaMemcpyAsync(chan_noise_host, cn, sizeof(float) * d[2], cudaMemcpyDeviceToHost, s));
  if (px && pix_noise_host) CK(cudaMemcpyAsync(pix_noise_host, pn, sizeof(float) * plane, cudaMemcpyDeviceToHost, s));
  if (!cf_h.empty() || !pf_h.empty() || chan_noise_host || pix_noise_host) CK(cudaStreamSynchronize(s));
  if (chan_flags_host) {
    if (ch) memcpy(chan_flags_host, cf_h.data(), (size_t)d[2]);
    else memset(chan_flags_host, 0, (size_t)d[2]);
  }
  if (pix_flags_host) {
    if (px) memcpy(pix_flags_host, pf_h.data(), (size_t)plane);
    else memset(pix_flags_host, 0, (size_t)plane);
  }
  if (want_counts) {
    long long nc = 0, np = 0;
    for (uint8_t f : cf_h) nc += f;
    for (uint8_t f : pf_h) np += f;
    n_flagged[0] = nc;
    n_flagged[1] = np;
  }
  return SC_OK;
}

int sc_set_profiling(sc_ctx* c, int on) {
  if (!c) return SC_ERR_ARG;
  c->profiling = on ? 1 : 0;
  return SC_OK;
}

int sc_get_stats(sc_ctx* c, sc_stats* out, int reset) {
  if (!c || !out) return SC_ERR_ARG;
  DeviceGuard g(c->device);
  flush_events(c);
  *out = c->stats;
  if (reset) {
    const uint32_t w = c->stats.warnings;
    int32_t kern[SC_MAX_KERNELS];
    memcpy(kern, c->stats.smooth_kernel_pair, sizeof(kern));
    memset(&c->stats, 0, sizeof(c->stats));
    c->stats.warnings = w;
    memcpy(c->stats.smooth_kernel_pair, kern, sizeof(kern));
  }
  return SC_OK;
}

}  // extern "C"
