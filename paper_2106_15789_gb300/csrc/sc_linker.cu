// Linker (SoFiA 2 Sect. 4.3; merging radius and size limits of Sect. 6): the
// detected voxels of a mask become numbered detections by friends-of-friends
// linking, then size filters remove the too small and too large ones.
//
// Friends: dx^2 + dy^2 <= r_xy^2 and |dz| <= r_z. Detections are the
// connected components, numbered 1, 2, ... in raster order of their first
// voxel; sizes are the extents along x, y and z.
//
//   k_cc_init      lab[v] = start of v's row run in the mask, kBackground
//                  elsewhere
//   k_cc_union     every run links to the runs within reach after it in
//                  raster order (a warp per run, lanes along the rows):
//                  lock-free union-find on lab, the larger root hung under the
//                  smaller, so that a component's root is its first voxel
//   k_cc_compress  lab[v] = root of v (read-only walks); roots per chunk of
//                  kChunk voxels
//   k_scan_block   exclusive scan of the chunk counts (one block); the host
//                  reads the number of components and sizes the rest
//   k_cc_number    lab[root] = -(id), ids consecutive in raster order
//   k_cc_final     lab[v] = id of v's root (0 outside the mask), and the
//                  bounding box and voxel count per detection (atomics)
//   k_cc_keep      size filters -> keep flags; k_scan_block -> new ids
//   k_cc_relabel   lab[v] = new id (0 for removed detections)
#include <climits>
#include <cstdint>

#include "sc_internal.h"

namespace sc {
namespace link {

constexpr int kChunk = 4096;        // voxels per numbering chunk (1024 threads x 4)
constexpr int kChunkThreads = 1024;
constexpr int kBackground = INT_MIN;

struct Geo {
  int nx, ny, nz;
  long long n;
  int rxy, rz;
};

__device__ __forceinline__ int find_root(int* lab, int x) {
  int p = lab[x];
  while (p != x) {
    const int gp = lab[p];
    if (gp != p) lab[x] = gp;  // path halving (a benign race: any ancestor will do)
    x = p;
    p = gp;
  }
  return x;
}

// Links the trees of a and b, the larger root under the smaller.
__device__ __forceinline__ void unite(int* lab, int a, int b) {
  while (true) {
    a = find_root(lab, a);
    b = find_root(lab, b);
    if (a == b) return;
    if (a > b) {
      const int t = a;
      a = b;
      b = t;
    }
    const int old = atomicCAS(&lab[b], b, a);
    if (old == b) return;  // b was still a root and now hangs under a
    b = old;               // b got a parent meanwhile: retry from there
  }
}

}  // namespace link

using link::Geo;

// lab[v] = start of v's run (the maximal row segment of mask voxels holding
// v; consecutive voxels of a row are friends when r_xy >= 1) in the mask,
// kBackground elsewhere. Run starts are the smallest index of their run, so
// they are consistent with roots hung under smaller indices.
__global__ void k_cc_init(const uint8_t* __restrict__ mask, int* __restrict__ lab, Geo g) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < g.n; v += (long long)gridDim.x * blockDim.x) {
    if (!mask[v]) {
      lab[v] = link::kBackground;
      continue;
    }
    long long s = v;
    if (g.rxy >= 1) {
      const long long row0 = (v / g.nx) * g.nx;
      while (s > row0 && mask[s - 1]) --s;
    }
    lab[v] = (int)s;
  }
}

// Friends-of-friends between runs: every run links once to the next run of
// its row within reach and to the first voxel of every run that meets its
// reach in each friend row after it in raster order (dz > 0, or dz == 0 and
// dy > 0); the other half of the relation is the mirror of these. A warp
// takes 32 consecutive voxels, finds the runs that start among them, and
// works through each run with all 32 lanes (row positions side by side).
__global__ void k_cc_union(const uint8_t* __restrict__ mask, int* lab, Geo g) {
  const long long plane = (long long)g.nx * g.ny;
  const int lane = threadIdx.x & 31;
  const long long nseg = (g.n + 31) / 32;
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  const int r2 = g.rxy * g.rxy;
  for (long long seg = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); seg < nseg; seg += warps) {
    const long long b = seg * 32;
    const long long v = b + lane;
    // x of every lane (a segment may cross a row boundary)
    int x = (int)(b % g.nx) + lane;
    while (x >= g.nx) x -= g.nx;
    const bool in = v < g.n && mask[v];
    const bool starts = in && (g.rxy == 0 || x == 0 || !mask[v - 1]);
    unsigned todo = __ballot_sync(0xffffffffu, starts);
    while (todo) {
      const int ls = __ffs(todo) - 1;
      todo &= todo - 1;
      const long long vs = b + ls;  // the run's first voxel
      const int z = (int)(vs / plane), rem = (int)(vs - (long long)z * plane), y = rem / g.nx, xs = rem - y * g.nx;
      const long long rowv = vs - xs;
      // end of the run
      int e = xs;
      if (g.rxy >= 1) {
        for (int off = 0;; off += 32) {
          const int xx = xs + off + lane;
          const bool m = xx < g.nx && mask[rowv + xx];
          const unsigned gap = __ballot_sync(0xffffffffu, !m);
          if (gap) {
            e = xs + off + __ffs(gap) - 2;
            break;
          }
        }
      }
      // the same row: the next run within reach (further runs in reach chain to it)
      if (g.rxy >= 2) {
        const int xx = e + 2 + lane;
        const bool m = lane <= g.rxy - 2 && xx < g.nx && mask[rowv + xx];
        const unsigned bal = __ballot_sync(0xffffffffu, m);
        if (bal && lane == __ffs(bal) - 1) link::unite(lab, (int)vs, (int)(rowv + xx));
      }
      for (int dz = 0; dz <= g.rz; ++dz) {
        const int zz = z + dz;
        if (zz >= g.nz) break;
        for (int dy = (dz == 0 ? 1 : -g.rxy); dy <= g.rxy; ++dy) {
          const int yy = y + dy;
          if (yy < 0 || yy >= g.ny) continue;
          int ddx = (int)sqrtf((float)(r2 - dy * dy));  // largest |dx| with dx^2 + dy^2 <= r_xy^2
          while ((ddx + 1) * (ddx + 1) + dy * dy <= r2) ++ddx;
          while (ddx > 0 && ddx * ddx + dy * dy > r2) --ddx;
          const int lo = max(0, xs - ddx), hi = min(g.nx - 1, e + ddx);
          const long long row = (long long)zz * plane + (long long)yy * g.nx;
          for (int off = 0; lo + off <= hi; off += 32) {
            const int xx = lo + off + lane;
            const bool ok = xx <= hi;
            const bool m = ok && mask[row + xx];
            const bool before = ok && xx > lo && mask[row + xx - 1];
            if (m && !before) link::unite(lab, (int)vs, (int)(row + xx));
          }
        }
      }
    }
  }
}

// Every mask voxel points at its root afterwards, and counts[chunk] holds the
// roots of each chunk of kChunk voxels (a block per chunk, four consecutive
// voxels per thread). The walks only read: halving paths here could overwrite
// a voxel's final root with an older ancestor read before it. A voxel is a
// root exactly when its walk ends at itself, whatever other threads write.
__global__ void __launch_bounds__(link::kChunkThreads) k_cc_compress(const uint8_t* __restrict__ mask, int* lab,
                                                                     long long n, int* __restrict__ counts) {
  __shared__ int s_roots;
  if (threadIdx.x == 0) s_roots = 0;
  __syncthreads();
  const long long base = (long long)blockIdx.x * link::kChunk + 4LL * threadIdx.x;
  int c = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const long long v = base + k;
    if (v < n && mask[v]) {
      int x = (int)v, p = lab[x];
      while (p != x) {
        x = p;
        p = lab[x];
      }
      if (x == (int)v) ++c;
      else lab[v] = x;
    }
  }
  c = __reduce_add_sync(0xffffffffu, c);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(&s_roots, c);
  __syncthreads();
  if (threadIdx.x == 0) counts[blockIdx.x] = s_roots;
}

// Exclusive scan of a[0 .. len) in place by one block of 1024 threads, tile
// by tile; *total receives the sum.
__global__ void __launch_bounds__(1024) k_scan_block(int* a, long long len, int* total) {
  __shared__ int part[33];
  __shared__ int carry;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) carry = 0;
  __syncthreads();
  for (long long t0 = 0; t0 < len; t0 += 1024) {
    const long long i = t0 + tid;
    const int v = i < len ? a[i] : 0;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) part[warp] = x;
    __syncthreads();
    if (warp == 0) {
      const int w = part[lane];
      int wi = w;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, wi, o);
        if (lane >= o) wi += y;
      }
      part[lane] = wi - w;
      if (lane == 31) part[32] = wi;
    }
    __syncthreads();
    if (i < len) a[i] = carry + part[warp] + x - v;
    __syncthreads();
    if (tid == 0) carry += part[32];
    __syncthreads();
  }
  if (tid == 0) *total = carry;
}

// lab[root] = -(id) with ids 1, 2, ... in raster order of the roots.
__global__ void __launch_bounds__(link::kChunkThreads) k_cc_number(int* lab, long long n, const int* __restrict__ off) {
  __shared__ int part[33];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const long long base = (long long)blockIdx.x * link::kChunk + 4LL * tid;  // four consecutive voxels per thread
  bool root[4];
  int c = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const long long v = base + k;
    root[k] = v < n && lab[v] == (int)v;
    c += root[k] ? 1 : 0;
  }
  int x = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) part[warp] = x;
  __syncthreads();
  if (warp == 0) {
    const int w = part[lane];
    int wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += y;
    }
    part[lane] = wi - w;
  }
  __syncthreads();
  int id = off[blockIdx.x] + part[warp] + x - c;  // roots before this thread's first voxel
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if (root[k]) lab[base + k] = -(++id);
}

// Every mask voxel takes its root's id; roots hold -(id) (or +id once their
// own thread has passed), non-roots the root's index. Then the bounding box
// and voxel count of each detection, ext[7 * (id - 1) ...] = x_min, x_max,
// y_min, y_max, z_min, z_max, count: lanes of a warp with the same id
// (neighbours along x, mostly) combine their coordinates first, so a
// detection's seven words see one atomic per group.
__global__ void k_cc_final(int* lab, Geo g, int* ext) {
  const long long plane = (long long)g.nx * g.ny;
  const int lane = threadIdx.x & 31;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long v0 = blockIdx.x * (long long)blockDim.x + threadIdx.x - lane; v0 < g.n; v0 += stride) {
    const long long v = v0 + lane;
    int id = 0;
    if (v < g.n) {
      const int l = lab[v];
      if (l == link::kBackground) {
        id = 0;
      } else if (l < 0) {
        id = -l;
      } else {
        const int r = lab[l];
        id = r < 0 ? -r : r;
      }
      lab[v] = id;
    }
    if (__ballot_sync(0xffffffffu, id > 0) == 0u) continue;
    int x = 0, y = 0, z = 0;
    if (id > 0) {
      z = (int)(v / plane);
      const int rem = (int)(v - (long long)z * plane);
      y = rem / g.nx;
      x = rem - y * g.nx;
    }
    const unsigned peers = __match_any_sync(0xffffffffu, id);  // lanes of the same detection (or background)
    const int xmin = __reduce_min_sync(peers, x), xmax = __reduce_max_sync(peers, x);
    const int ymin = __reduce_min_sync(peers, y), ymax = __reduce_max_sync(peers, y);
    const int zmin = __reduce_min_sync(peers, z), zmax = __reduce_max_sync(peers, z);
    if (id > 0 && lane == __ffs(peers) - 1) {
      int* e = ext + 7LL * (id - 1);
      atomicMin(e + 0, xmin);
      atomicMax(e + 1, xmax);
      atomicMin(e + 2, ymin);
      atomicMax(e + 3, ymax);
      atomicMin(e + 4, zmin);
      atomicMax(e + 5, zmax);
      atomicAdd(e + 6, __popc(peers));
    }
  }
}

__global__ void k_cc_ext_init(int* ext, int ncomp) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ncomp; i += gridDim.x * blockDim.x) {
    int* e = ext + 7LL * i;
    e[0] = e[2] = e[4] = INT_MAX;
    e[1] = e[3] = e[5] = -1;
    e[6] = 0;
  }
}

__global__ void k_cc_keep(const int* __restrict__ ext, int ncomp, int min_xy, int min_z, int max_xy, int max_z,
                          int* keep) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ncomp; i += gridDim.x * blockDim.x) {
    const int* e = ext + 7LL * i;
    const int sx = e[1] - e[0] + 1, sy = e[3] - e[2] + 1, sz = e[5] - e[4] + 1;
    bool k = sx >= min_xy && sy >= min_xy && sz >= min_z;
    if (max_xy > 0) k = k && sx <= max_xy && sy <= max_xy;
    if (max_z > 0) k = k && sz <= max_z;
    keep[i] = k ? 1 : 0;
  }
}

// After the exclusive scan of the keep flags: the kept rows moved to the
// front of out (ids 1 .. kept), and new_id[i] = id of detection i + 1 or 0.
__global__ void k_cc_compact(const int* __restrict__ ext, const int* keep_flag, const int* __restrict__ keep_off,
                             int ncomp, int* out, int* new_id) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ncomp; i += gridDim.x * blockDim.x) {
    if (keep_flag[i]) {
      const int j = keep_off[i];
      for (int c = 0; c < 7; ++c) out[7LL * j + c] = ext[7LL * i + c];
      new_id[i] = j + 1;
    } else {
      new_id[i] = 0;
    }
  }
}

__global__ void k_cc_relabel(int* lab, long long n, const int* __restrict__ new_id) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
    const int id = lab[v];
    if (id > 0) lab[v] = new_id[id - 1];
  }
}

// ---------------------------------------------------------------------------
namespace {
inline int grid_for(long long n, int sms, int threads) {
  const long long want = (n + threads - 1) / threads;
  const long long cap = 16LL * sms;
  return (int)(want < 1 ? 1 : (want < cap ? want : cap));
}
}  // namespace

long long link_chunks(long long n) { return (n + link::kChunk - 1) / link::kChunk; }

cudaError_t launch_link_components(const uint8_t* mask, const long long dims[3], int r_xy, int r_z, int* lab,
                                   int* chunk_off, int* d_total, int sms, cudaStream_t s) {
  Geo g{(int)dims[0], (int)dims[1], (int)dims[2], dims[0] * dims[1] * dims[2], r_xy, r_z};
  const long long chunks = link_chunks(g.n);
  k_cc_init<<<grid_for(g.n, sms, 256), 256, 0, s>>>(mask, lab, g);
  k_cc_union<<<grid_for((g.n + 31) / 32 * 32, sms, 256), 256, 0, s>>>(mask, lab, g);
  k_cc_compress<<<(unsigned)chunks, link::kChunkThreads, 0, s>>>(mask, lab, g.n, chunk_off);
  k_scan_block<<<1, 1024, 0, s>>>(chunk_off, chunks, d_total);
  return cudaGetLastError();
}

cudaError_t launch_link_filter(const long long dims[3], int* lab, int* chunk_off, int ncomp, int min_xy, int min_z,
                               int max_xy, int max_z, int* ext, int* keep, int* ext_out, int* new_id, int* d_total,
                               int sms, cudaStream_t s) {
  Geo g{(int)dims[0], (int)dims[1], (int)dims[2], dims[0] * dims[1] * dims[2], 0, 0};
  const long long chunks = link_chunks(g.n);
  if (ncomp > 0) k_cc_ext_init<<<grid_for(ncomp, sms, 256), 256, 0, s>>>(ext, ncomp);
  k_cc_number<<<(unsigned)chunks, link::kChunkThreads, 0, s>>>(lab, g.n, chunk_off);
  k_cc_final<<<grid_for((g.n + 31) / 32 * 32, sms, 256), 256, 0, s>>>(lab, g, ext);
  if (ncomp <= 0) return cudaGetLastError();
  k_cc_keep<<<grid_for(ncomp, sms, 256), 256, 0, s>>>(ext, ncomp, min_xy, min_z, max_xy, max_z, keep);
  // keep flags are kept in new_id while keep becomes their exclusive scan
  cudaError_t e = cudaMemcpyAsync(new_id, keep, sizeof(int) * (size_t)ncomp, cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return e;
  k_scan_block<<<1, 1024, 0, s>>>(keep, ncomp, d_total);
  k_cc_compact<<<grid_for(ncomp, sms, 256), 256, 0, s>>>(ext, new_id, keep, ncomp, ext_out, new_id);
  k_cc_relabel<<<grid_for(g.n, sms, 256), 256, 0, s>>>(lab, g.n, new_id);
  return cudaGetLastError();
}

}  // namespace sc
