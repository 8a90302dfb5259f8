// gs_internal.cuh -- workspace layout, device camera table and small device
// helpers shared by the kernels of the rasterizer library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gs.h"

namespace gs {

constexpr int kMaxViews = 256;
constexpr int kMaxK = 16;
constexpr int kMaxM = 1024;
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kMaxRadixPasses = 8;       // 64-bit keys at most
constexpr int kProjThreads = 256;
constexpr int kProjItems = 4;
constexpr int kProjBlock = kProjThreads * kProjItems;  // Gaussians per projection CTA
constexpr int kEmitCtasMax = 1024;   // chunks of the pair emission (2 per SM, capped; sizes the chunk totals)
constexpr int64_t kCandBitsDefault = 4ll << 30;  // contributor-bit bytes of a candidate layout (default)
constexpr int kEmitThreads = 256;

// Status bits in the workspace counters (1 << gs_status code).
constexpr uint32_t kStatusCapacity = 1u << GS_ERR_CAPACITY;
constexpr uint32_t kStatusTimeout = 1u << GS_ERR_TIMEOUT;

// Per-view camera as the kernels read it (written once per call into the
// workspace by k_setup_views).
struct DevCam {
  float fx, fy, cx, cy, near_plane;
  float r[9];
  float t[3];
  int width, height;
  int tiles_x, tiles_y;
  uint32_t tile_off;   // first global tile id of this view
};

// Kernel-parameter carrier for up to kMaxViews cameras (kernel parameters up
// to 32 KB are legal on sm_70+ with CUDA 12.1+; 256 * 84 B fits).
struct CamTable {
  DevCam cam[kMaxViews];
};

struct Counters {
  uint32_t status;
  uint32_t n_records;
  uint32_t n_pairs;
  uint32_t n_contrib;  // (pixel, Gaussian) contributions of the last forward render
  uint32_t tiles_done; // tickets of the tile pass that finishes the loss (0 between launches)
  uint32_t grp_records, grp_pairs;  // largest counts of the earlier view groups of a grouped call
};

// Host-computed workspace layout (offsets in bytes from the base pointer).
struct Layout {
  int n, k, m, n_views, tile_w, tile_h;
  int cam0_w, cam0_h;                      // first camera (the single view of mapping calls)
  int ppt;                                 // pixels per thread in the adjoint (1, 2 or 4)
  uint32_t spin_limit;                     // polls of one inter-CTA wait
  int64_t rcap, pcap, total_tiles, npix;  // npix: pixels of view 0 when n_views == 1
  int64_t proj_blocks;                     // projection CTAs per view
  int key_bits_depth;                      // bits of the (view, depth) record key
  int key_bits_tile;                       // bits of the global tile id
  size_t off_counters, off_cams, off_tile_off, off_blockcnt;
  size_t off_rec_uv, off_rec_conic, off_rec_depth, off_rec_rect, off_rec_gid, off_rec_view;
  size_t off_rec_box, off_rec_cd, off_rec_unc, off_rec_sem;
  size_t off_dkeys[2], off_dvals[2];
  size_t off_epart, off_rloc;
  size_t off_pkeys[2], off_pvals[2];
  size_t off_tickets, off_ghist, off_lb_depth, off_lb_pairs;
  size_t off_ranges;
  size_t off_tfinal, off_nlast;
  size_t off_grad2d;
  int nwc;                                 // 32-class sign words per plane (fused L1 mode)
  size_t off_codes, off_lpart;
  size_t off_semg;                         // mapping view: [n][k] objective gradient of sem_w (unscaled)
  size_t off_mask_off, off_masks;          // contributor bitmasks (mapping view; candidate views when they fit)
  size_t off_clast;                        // candidate views: last contributor per (tile, pixel)
  int64_t mask_units;                      // capacity in (tile, 64-pair batch) units (mapping view)
  int cand_batch;                          // Gaussians per batch of the candidate kernels (32, 64, 128)
  int cand_waves;                          // candidate waves the launch chain provides for
  int64_t cand_cap_units;                  // bit capacity in (tile, cand_batch) units (0: single pass)
  size_t off_cand_plan;                    // candidate waves
  size_t total;
};

struct WsPtrs {
  Counters *counters;
  DevCam *cams;
  uint32_t *tile_off;
  uint32_t *blockcnt;
  float2 *rec_uv;
  float4 *rec_conic;
  float *rec_depth;
  short4 *rec_rect;
  int32_t *rec_gid;
  int32_t *rec_view;
  short4 *rec_box;   // alpha box (pixels outside have alpha < 1/255), within rec_rect
  float4 *rec_cd;    // r, g, b, depth
  float *rec_unc;    // per-Gaussian uncertainty (0 when absent)
  int2 *rec_sem;     // [rcap][k] (class id, weight bits)
  unsigned long long *dkeys[2];
  uint32_t *dvals[2];
  uint32_t *epart;
  uint32_t *rloc;     // [rcap] pair offset of each depth-sorted record inside its emit chunk
  uint32_t *pkeys[2];
  uint32_t *pvals[2];
  uint32_t *tickets;                 // [2][kMaxRadixPasses] tile tickets (depth sort, pair sort)
  uint32_t *ghist;                   // [2][kMaxRadixPasses][256] digit histograms
  unsigned long long *lb_depth;      // look-back words of the depth sort
  unsigned long long *lb_pairs;      // look-back words of the pair sort
  uint2 *ranges;
  float *tfinal;
  uint32_t *nlast;
  float4 *grad2d;  // [rcap][2]: (du, dv, da, db), (dc, dopacity, dz, 0)
  uint32_t *codes; // [npix][1 + nwc] (nonzero, negative) word pairs: sign codes of the fused L1 mode
  uint32_t *mask_off;  // [tiles + 1] first (tile, batch) unit of each tile
  uint32_t *masks;     // [unit][2][tile pixels] contributor bits of each staged batch
  uint32_t *clast;     // [tiles][tile pixels] last contributor (candidate views)
  double *lpart;   // [tiles of view 0][3] per-tile L1 sums
  float *semg;     // [n][k] d(semantic term)/d(sem_w) of the fused Sec. 3.1 objective, before dL/dloss
  uint32_t *cand_plan;  // candidate waves: [waves][5] (first tile, end tile, first unit, two tickets)
};

// Host side (api.cu): device facts, queried per device and cached
// (thread-safe).  device_sms() is the multiprocessor count of the current
// device (0 when it cannot be queried); sm_grid(c) is c CTAs per SM for a
// grid-stride kernel (0 on failure); emit_chunks() is the chunk count of the
// pair emission (2 per SM, at most kEmitCtasMax); ensure_smem_limit raises
// the dynamic shared-memory limit of one kernel on the current device the
// first time that device launches it.
int device_sms();
unsigned sm_grid(int ctas_per_sm);
int emit_chunks();
cudaError_t ensure_smem_limit(const void *func, int bytes);

// Host side (api.cu): the camera table of a call (kernel parameter of the
// view setup), and the launch chains of gs_project and gs_bin_sort; `tab` is
// the caller's storage for the table (no heap use inside).
void fill_cam_table(const gs_camera *cams, int n_views, int tw, int th, CamTable *tab);
// `first` = false continues a grouped call: the device status is kept and
// the previous group's counts are folded into the group maxima.
gs_status run_project_with(const Layout &L, const WsPtrs &P, const gs_scene &sc, const gs_camera *cams,
                           CamTable *tab, cudaStream_t s, bool first = true);
gs_status run_bin_sort(const Layout &L, const WsPtrs &P, cudaStream_t s);

// Host side (api.cu).
bool make_layout(const gs_scene *scene, const gs_camera *cams, int n_views, const gs_config *cfg, Layout *L);
WsPtrs ws_ptrs(const Layout &L, void *ws);

// Number of radix passes over `bits` key bits.
inline int radix_passes(int bits) { return (bits + kRadixBits - 1) / kRadixBits; }
// Tiles of the radix-sort pass kernel for `capacity` elements.
int sort_tiles(int64_t capacity);

// ---------------------------------------------------------------------------
// Launchers implemented in the kernel translation units.
// ---------------------------------------------------------------------------
cudaError_t launch_setup_views(const CamTable &tab, int n_views, const WsPtrs &P, uint32_t total_tiles,
                               bool reset_status, cudaStream_t s);
cudaError_t launch_project(const Layout &L, const WsPtrs &P, const gs_scene &sc, cudaStream_t s);
cudaError_t launch_scan_single(uint32_t *data, uint32_t n, uint32_t *total_out, uint32_t capacity,
                               Counters *counters, cudaStream_t s);
cudaError_t launch_radix_sort_u64(const Layout &L, const WsPtrs &P, int bits, int *final_buf, cudaStream_t s);
cudaError_t launch_radix_sort_u32(const Layout &L, const WsPtrs &P, int bits, int *final_buf, cudaStream_t s);
cudaError_t launch_emit_pairs(const Layout &L, const WsPtrs &P, int dbuf, cudaStream_t s);
// first (tile, batch) unit of every tile: batches per tile, exclusive scan
cudaError_t launch_tile_batch_offsets(const uint2 *ranges, uint32_t ntiles, uint32_t *mask_off, Counters *counters,
                                      cudaStream_t s, int batch = 64);
cudaError_t launch_tile_ranges(const Layout &L, const WsPtrs &P, int pbuf, cudaStream_t s);
cudaError_t launch_render_fwd(const Layout &L, const WsPtrs &P, int pbuf, const gs_scene &sc, float *rgb,
                              float *depth, float *sil, float *sem, cudaStream_t s);
cudaError_t launch_render_fwd_l1(const Layout &L, const WsPtrs &P, int pbuf, const gs_scene &sc,
                                 const float *t_rgb, const float *t_depth, const float *t_sem, float *rgb,
                                 float *depth, float *sil, float *sem, float *loss, cudaStream_t s);
// loss_scale != nullptr selects the fused-loss adjoint (upstream from sign
// codes); objective = 1 takes the Sec. 3.1 objective's scales and no class codes
cudaError_t launch_render_bwd(const Layout &L, const WsPtrs &P, int pbuf, const gs_scene &sc, const float *d_rgb,
                              const float *d_depth, const float *d_sil, const float *d_sem, int sem_detach,
                              float *g_rgb, float *g_sem_w, cudaStream_t s, const float *loss_scale = nullptr,
                              int objective = 0);
// Fused Sec. 3.1 objective (render_paper.cu): whether the mapping view's
// class accumulator fits one shared-memory chunk; the forward (blend with the
// silhouette-masked geometry, semantic term and its sem_w gradient); the
// adjoint's g_sem_w += dL/dloss * semg.
bool objective_fits(const Layout &L, int k, int m);
cudaError_t launch_render_fwd_objective(const Layout &L, const WsPtrs &P, int pbuf, const gs_scene &sc,
                                        const float *t_rgb, const float *t_depth, const float *t_sem, float *rgb,
                                        float *depth, float *sil, float *loss, cudaStream_t s);
// Dense-semantic comparator (render_dense.cu): every Gaussian carries all
// m class probabilities (dense [n][m]); needs the contributor bits.
bool dense_supported(const Layout &L);
cudaError_t launch_render_fwd_dense(const Layout &L, const WsPtrs &P, int pbuf, const gs_scene &sc,
                                    const float *dense, float *rgb, float *depth, float *sil, float *sem,
                                    cudaStream_t s);
cudaError_t launch_add_semg(const WsPtrs &P, const gs_scene &sc, const float *loss_scale, float *g_sem_w,
                            cudaStream_t s);
cudaError_t launch_project_bwd(const Layout &L, const WsPtrs &P, const gs_scene &sc, float *g_means,
                               float *g_scales, float *g_quats, float *g_opacity, cudaStream_t s);
cudaError_t launch_candidates(const Layout &L, const WsPtrs &P, int pbuf, const gs_scene &sc, double *out,
                              cudaStream_t s);
// Work counters of the binned views (stats.cu): out[5] = n_eval, n_eval_box,
// n_contrib, n_touched, n_pixels; per_pixel (single view, or null): the
// (n_eval, n_contrib) pair of every pixel.
cudaError_t launch_work_stats(const Layout &L, const WsPtrs &P, int pbuf, const gs_scene &sc,
                              unsigned long long *out, uint32_t *per_pixel, cudaStream_t s);
cudaError_t launch_l1_loss(int64_t npix, int m, const float *rgb, const float *t_rgb, const float *depth,
                           const float *t_depth, const float *sem, const float *t_sem, float *d_rgb, float *d_depth,
                           float *d_sem, float *loss, double *partial, cudaStream_t s);
cudaError_t launch_mapping_loss(int64_t npix, int m, int k, const float *rgb, const float *t_rgb, const float *depth,
                                const float *t_depth, const float *sil, const float *sem, const float *t_sem,
                                float *d_rgb, float *d_depth, float *d_sem, float *loss, double *partial,
                                cudaStream_t s);

// Which of the two ping-pong buffers holds the sorted data after the passes.
inline int depth_sort_buffer(const Layout &L) { return radix_passes(L.key_bits_depth) & 1; }
inline int pair_sort_buffer(const Layout &L) { return radix_passes(L.key_bits_tile) & 1; }

}  // namespace gs

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------
#ifdef __CUDACC__
namespace gs {

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Inclusive warp scan of a u32.
__device__ __forceinline__ uint32_t warp_inclusive_scan(uint32_t v) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    uint32_t o = __shfl_up_sync(0xffffffffu, v, d);
    if ((int)lane_id() >= d) v += o;
  }
  return v;
}

// Exclusive block scan of one u32 per thread (blockDim.x a multiple of 32,
// at most 1024).  `tmp` needs 33 words of shared memory.  Returns the
// exclusive prefix; *total receives the block sum.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *tmp, uint32_t *total) {
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t inc = warp_inclusive_scan(v);
  if (lane == 31) tmp[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < nw ? tmp[lane] : 0u;
    uint32_t wi = warp_inclusive_scan(w);
    if (lane < nw) tmp[lane] = wi - w;
    if (lane == nw - 1) tmp[32] = wi;
  }
  __syncthreads();
  uint32_t r = tmp[warp] + inc - v;
  *total = tmp[32];
  __syncthreads();
  return r;
}

__device__ __forceinline__ void set_status(Counters *c, uint32_t bits) { atomicOr(&c->status, bits); }

}  // namespace gs
#endif
