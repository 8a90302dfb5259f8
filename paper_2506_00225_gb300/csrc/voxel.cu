// voxel.cu -- the Exploration Map of Sec. 3.2: a voxel occupancy grid (5 cm
// voxels in the paper) updated from each depth frame, and the list of voxels
// the update newly freed, from which candidate positions are sampled.
//
// State: 2 bits per voxel packed 16 to a 32-bit word (bit 2j: seen free,
// bit 2j+1: seen occupied; occupied wins).  An update only sets bits, with
// warp-aggregated atomicOr, so its result does not depend on the thread
// schedule.  Voxel
// (x, y, z) has linear index (z ny + y) nx + x.
//
// Update: one thread per sampled pixel (every stride-th column and row).
// The pixel's depth d (camera-space z, as rendered) gives the point
// X = ((u + 1/2 - cx) d / fx, (v + 1/2 - cy) d / fy, d) in the camera; the
// segment from the camera centre to it is walked voxel by voxel (the
// grid traversal of Amanatides and Woo, 1987), clipped to the grid: every
// voxel it passes before the one holding the point is free, the one holding
// the point occupied.  Depths beyond max_depth are cut there and mark no
// occupied voxel; depths that are not positive and finite are skipped.
//
// New free voxels: free now (and not occupied) and unknown in the previous
// state.  Counted per CTA over fixed word ranges, scanned, then written in
// voxel index order: deterministic.
#include <cmath>

#include "gs_internal.cuh"

namespace gs {

constexpr int kVoxThreads = 256;
constexpr int kVoxWordsPerThread = 8;
constexpr int kVoxWordsPerCta = kVoxThreads * kVoxWordsPerThread;

struct VoxArgs {
  float ox, oy, oz, vs;  // grid origin (world) and voxel size
  int nx, ny, nz;
  float rt[9];           // camera-to-world rotation (R^T), row-major
  float cc[3];           // camera centre (world)
  float fx, fy, cx, cy;
  int width, height, stride, nu, nv;
  float max_depth;
};

// Sets one state bit of voxel vox.  The lanes of the warp that set bits of
// the same word at this point are grouped (they usually are: neighbouring
// pixels' rays pass the same voxels), their bits OR-ed, and one of them
// issues a single atomicOr whose result is not used (no wait).
__device__ __forceinline__ void set_bit(uint32_t *state, int64_t vox, uint32_t which) {
  const uint32_t bit = 1u << (2 * (uint32_t)(vox & 15) + which);
  const unsigned long long word = (unsigned long long)(vox >> 4);
  const uint32_t grp = __match_any_sync(__activemask(), word);
  const uint32_t bits = __reduce_or_sync(grp, bit);
  if (lane_id() == (uint32_t)(__ffs(grp) - 1)) atomicOr(state + word, bits);
}

__global__ void __launch_bounds__(kVoxThreads) k_voxel_update(VoxArgs a, uint32_t *state, const float *depth) {
  const int i = blockIdx.x * kVoxThreads + threadIdx.x;
  if (i >= a.nu * a.nv) return;
  const int u = (i % a.nu) * a.stride, v = (i / a.nu) * a.stride;
  const float d = depth[(size_t)v * a.width + u];
  if (!(d > 0.f) || !(d < INFINITY)) return;
  const bool hit = d <= a.max_depth;
  const float de = hit ? d : a.max_depth;
  const float xc = __fmul_rn(__fdiv_rn(__fsub_rn(__fadd_rn((float)u, 0.5f), a.cx), a.fx), de);
  const float yc = __fmul_rn(__fdiv_rn(__fsub_rn(__fadd_rn((float)v, 0.5f), a.cy), a.fy), de);
  const float zc = de;
  float p[3];
  for (int r = 0; r < 3; ++r)
    p[r] = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(a.rt[3 * r], xc), __fmul_rn(a.rt[3 * r + 1], yc)),
                               __fmul_rn(a.rt[3 * r + 2], zc)), a.cc[r]);
  // segment in grid units
  const float org[3] = {a.ox, a.oy, a.oz};
  const int n[3] = {a.nx, a.ny, a.nz};
  float s0[3], s1[3], dir[3];
  for (int r = 0; r < 3; ++r) {
    s0[r] = __fdiv_rn(__fsub_rn(a.cc[r], org[r]), a.vs);
    s1[r] = __fdiv_rn(__fsub_rn(p[r], org[r]), a.vs);
    dir[r] = __fsub_rn(s1[r], s0[r]);
  }
  // voxel holding the point (when it lies in the grid)
  int e[3];
  bool e_in = hit;
  for (int r = 0; r < 3; ++r) {
    e[r] = (int)floorf(s1[r]);
    e_in = e_in && s1[r] >= 0.f && e[r] < n[r];
  }
  auto lin = [&](const int *c) { return ((int64_t)c[2] * a.ny + c[1]) * a.nx + c[0]; };
  // clip the parameter range [0, 1] to the grid box [0, n]^3
  float t0 = 0.f, t1 = 1.f;
  for (int r = 0; r < 3; ++r) {
    if (dir[r] == 0.f) {
      if (s0[r] < 0.f || s0[r] >= (float)n[r]) t1 = -1.f;
    } else {
      const float ta = __fdiv_rn(-s0[r], dir[r]), tb = __fdiv_rn(__fsub_rn((float)n[r], s0[r]), dir[r]);
      t0 = fmaxf(t0, fminf(ta, tb));
      t1 = fminf(t1, fmaxf(ta, tb));
    }
  }
  if (t0 < t1) {
    // per axis: the voxel, the step direction and the parameter of the next
    // boundary crossing (recomputed from the start point at every step, so
    // no error accumulates along long rays)
    int c[3], step[3];
    float tmax[3];
    auto crossing = [&](int r) {
      return __fdiv_rn(__fsub_rn((float)(step[r] > 0 ? c[r] + 1 : c[r]), s0[r]), dir[r]);
    };
    for (int r = 0; r < 3; ++r) {
      const float x = __fadd_rn(s0[r], __fmul_rn(t0, dir[r]));
      c[r] = min(max((int)floorf(x), 0), n[r] - 1);
      step[r] = dir[r] > 0.f ? 1 : (dir[r] < 0.f ? -1 : 0);
      tmax[r] = step[r] ? crossing(r) : INFINITY;
    }
    const int limit = a.nx + a.ny + a.nz + 3;
    for (int it = 0; it < limit; ++it) {
      if (e_in && c[0] == e[0] && c[1] == e[1] && c[2] == e[2]) break;
      set_bit(state, lin(c), 0);
      const int ax = tmax[0] <= tmax[1] ? (tmax[0] <= tmax[2] ? 0 : 2) : (tmax[1] <= tmax[2] ? 1 : 2);
      if (!(tmax[ax] < t1)) break;
      c[ax] += step[ax];
      if (c[ax] < 0 || c[ax] >= n[ax]) break;
      tmax[ax] = crossing(ax);
    }
  }
  if (e_in) set_bit(state, lin(e), 1);
}

// newly freed voxels of word w: free, not occupied, and no bit before
__device__ __forceinline__ uint32_t new_free_bits(uint32_t cur, uint32_t prev) {
  const uint32_t free_only = cur & ~(cur >> 1) & 0x55555555u;
  const uint32_t unknown = ~(prev | (prev >> 1)) & 0x55555555u;
  return free_only & unknown;
}

__global__ void __launch_bounds__(kVoxThreads) k_voxel_new_count(int64_t words, const uint32_t *prev,
                                                                 const uint32_t *cur, uint32_t *counts) {
  __shared__ uint32_t tmp[33];
  const int64_t w0 = (int64_t)blockIdx.x * kVoxWordsPerCta + (int64_t)threadIdx.x * kVoxWordsPerThread;
  uint32_t c = 0;
  for (int j = 0; j < kVoxWordsPerThread; ++j)
    if (w0 + j < words) c += __popc(new_free_bits(cur[w0 + j], prev[w0 + j]));
  uint32_t total;
  block_exclusive_scan(c, tmp, &total);
  if (threadIdx.x == 0) counts[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kVoxThreads) k_voxel_new_emit(int64_t words, VoxArgs a, const uint32_t *prev,
                                                                const uint32_t *cur, const uint32_t *offsets,
                                                                float *centres, int64_t capacity) {
  __shared__ uint32_t tmp[33];
  const int64_t w0 = (int64_t)blockIdx.x * kVoxWordsPerCta + (int64_t)threadIdx.x * kVoxWordsPerThread;
  uint32_t c = 0;
  for (int j = 0; j < kVoxWordsPerThread; ++j)
    if (w0 + j < words) c += __popc(new_free_bits(cur[w0 + j], prev[w0 + j]));
  uint32_t total;
  uint64_t pos = (uint64_t)offsets[blockIdx.x] + block_exclusive_scan(c, tmp, &total);
  for (int j = 0; j < kVoxWordsPerThread; ++j) {
    if (w0 + j >= words) break;
    uint32_t b = new_free_bits(cur[w0 + j], prev[w0 + j]);
    while (b) {
      const int k = (__ffs(b) - 1) >> 1;
      b &= b - 1;
      if ((int64_t)pos < capacity) {
        const int64_t vox = (w0 + j) * 16 + k;
        const int x = (int)(vox % a.nx), y = (int)((vox / a.nx) % a.ny), z = (int)(vox / ((int64_t)a.nx * a.ny));
        centres[3 * pos] = a.ox + ((float)x + 0.5f) * a.vs;
        centres[3 * pos + 1] = a.oy + ((float)y + 0.5f) * a.vs;
        centres[3 * pos + 2] = a.oz + ((float)z + 0.5f) * a.vs;
      }
      ++pos;
    }
  }
}

static bool grid_ok(const gs_voxel_grid *g) {
  if (!g || !(g->voxel > 0.f) || g->nx < 1 || g->ny < 1 || g->nz < 1) return false;
  if (!std::isfinite(g->origin[0]) || !std::isfinite(g->origin[1]) || !std::isfinite(g->origin[2])) return false;
  return (int64_t)g->nx * g->ny * g->nz < (1ll << 40) && g->nx + g->ny + g->nz < (1 << 24);
}

static int64_t grid_words(const gs_voxel_grid *g) { return ((int64_t)g->nx * g->ny * g->nz + 15) / 16; }

static VoxArgs vox_args(const gs_voxel_grid *g) {
  VoxArgs a{};
  a.ox = g->origin[0]; a.oy = g->origin[1]; a.oz = g->origin[2]; a.vs = g->voxel;
  a.nx = g->nx; a.ny = g->ny; a.nz = g->nz;
  return a;
}

}  // namespace gs

using namespace gs;

extern "C" {

int64_t gs_voxel_words(const gs_voxel_grid *grid) { return grid_ok(grid) ? grid_words(grid) : -1; }

int64_t gs_voxel_scratch_words(const gs_voxel_grid *grid) {
  return grid_ok(grid) ? (grid_words(grid) + kVoxWordsPerCta - 1) / kVoxWordsPerCta + 1 : -1;
}

gs_status gs_voxel_update(const gs_voxel_grid *grid, uint32_t *state, const float *depth, const gs_camera *cam,
                          int stride, float max_depth, gs_stream_t stream) {
  if (!grid_ok(grid) || !state || !depth || !cam || stride < 1 || !(max_depth > 0.f)) return GS_ERR_ARG;
  if (cam->width < 1 || cam->height < 1 || !(cam->fx > 0.f) || !(cam->fy > 0.f)) return GS_ERR_ARG;
  VoxArgs a = vox_args(grid);
  // camera-to-world rotation and centre from [R|t] (in double, then float)
  const float *w = cam->w2c;
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c) a.rt[3 * r + c] = w[4 * c + r];
    double cc = 0.0;
    for (int c = 0; c < 3; ++c) cc -= (double)w[4 * c + r] * (double)w[4 * c + 3];
    a.cc[r] = (float)cc;
  }
  a.fx = cam->fx; a.fy = cam->fy; a.cx = cam->cx; a.cy = cam->cy;
  a.width = cam->width; a.height = cam->height; a.stride = stride;
  a.nu = (cam->width + stride - 1) / stride;
  a.nv = (cam->height + stride - 1) / stride;
  a.max_depth = max_depth;
  const int64_t rays = (int64_t)a.nu * a.nv;
  k_voxel_update<<<(unsigned)((rays + kVoxThreads - 1) / kVoxThreads), kVoxThreads, 0, (cudaStream_t)stream>>>(
      a, state, depth);
  return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

gs_status gs_voxel_new_free(const gs_voxel_grid *grid, const uint32_t *prev, const uint32_t *cur, uint32_t *scratch,
                            float *centres, int64_t capacity, uint32_t *count, gs_stream_t stream) {
  if (!grid_ok(grid) || !prev || !cur || !scratch || !count || capacity < 0 || (capacity > 0 && !centres))
    return GS_ERR_ARG;
  const int64_t words = grid_words(grid);
  const int64_t ctas = (words + kVoxWordsPerCta - 1) / kVoxWordsPerCta;
  if (ctas >= (1ll << 31)) return GS_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  k_voxel_new_count<<<(unsigned)ctas, kVoxThreads, 0, s>>>(words, prev, cur, scratch);
  if (cudaGetLastError() != cudaSuccess) return GS_ERR_CUDA;
  if (launch_scan_single(scratch, (uint32_t)ctas, count, 0xffffffffu, nullptr, s) != cudaSuccess) return GS_ERR_CUDA;
  k_voxel_new_emit<<<(unsigned)ctas, kVoxThreads, 0, s>>>(words, vox_args(grid), prev, cur, scratch, centres,
                                                         capacity);
  return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

}  // extern "C"
