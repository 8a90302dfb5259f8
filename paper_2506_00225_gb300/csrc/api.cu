// api.cu -- the extern "C" entry points declared in include/gs.h: argument
// validation, workspace layout and the launch chains.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <set>
#include <utility>
#include <vector>

#include "gs_internal.cuh"
#include "render_common.cuh"

namespace gs {

// ---------------------------------------------------------------------------
// Device facts.  One process may drive several devices: the multiprocessor
// count is cached per device index, and the dynamic shared-memory limit of a
// kernel is raised once per (kernel, device), under a lock.
// ---------------------------------------------------------------------------
constexpr int kMaxDevices = 64;
static std::atomic<int> g_sms[kMaxDevices];
static std::atomic<int (*)(void)> g_sms_query{nullptr};  // replaces the device query (host tests)

int device_sms() {
  if (int (*q)(void) = g_sms_query.load()) return q();
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 0;
  int v = g_sms[dev].load(std::memory_order_relaxed);
  if (v > 0) return v;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) return 0;
  g_sms[dev].store(v, std::memory_order_relaxed);
  return v;
}

unsigned sm_grid(int ctas_per_sm) {
  const int sms = device_sms();
  return sms > 0 && ctas_per_sm > 0 ? (unsigned)sms * (unsigned)ctas_per_sm : 0u;
}

int emit_chunks() {
  const int sms = device_sms();
  return sms > 0 ? (2 * sms < kEmitCtasMax ? 2 * sms : kEmitCtasMax) : 0;
}

cudaError_t ensure_smem_limit(const void *func, int bytes) {
  static std::mutex mu;
  static std::set<std::pair<const void *, int>> done;  // (kernel, device) pairs already raised
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  if (done.count({func, dev})) return cudaSuccess;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) done.insert({func, dev});
  return e;
}

static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

static int bits_for(uint64_t max_value) {
  int b = 1;
  while (b < 64 && (max_value >> b) != 0) ++b;
  return b;
}

static bool cam_ok(const gs_camera &c) {
  if (c.width < 1 || c.height < 1 || c.width > 16384 || c.height > 16384) return false;
  if (!(c.fx > 0.f) || !(c.fy > 0.f) || !isfinite(c.fx) || !isfinite(c.fy)) return false;
  if (!isfinite(c.cx) || !isfinite(c.cy)) return false;
  if (!(c.near_plane > 0.f) || !isfinite(c.near_plane)) return false;
  for (int i = 0; i < 12; ++i)
    if (!isfinite(c.w2c[i])) return false;
  return true;
}

static gs_config default_config() {
  gs_config c{};
  c.tile_w = 16;
  c.tile_h = 16;
  c.sem_detach_geometry = 1;
  return c;
}

// Layout of one call over all `n_views` views at once.
static bool layout_views(const gs_scene *scene, const gs_camera *cams, int n_views, const gs_config *cfg_in,
                         Layout *L) {
  if (!scene || !cams || n_views < 1 || n_views > kMaxViews) return false;
  const gs_config cfg = cfg_in ? *cfg_in : default_config();
  if (scene->n < 0 || scene->n >= (1 << 28) || scene->k < 1 || scene->k > kMaxK || scene->m < 1 ||
      scene->m > kMaxM)
    return false;
  if (cfg.tile_w < 1 || cfg.tile_h < 1 || cfg.tile_w > 64 || cfg.tile_h > 64) return false;
  memset(L, 0, sizeof(*L));
  L->n = scene->n; L->k = scene->k; L->m = scene->m; L->n_views = n_views;
  L->tile_w = cfg.tile_w; L->tile_h = cfg.tile_h;
  if (cfg.px_per_thread < 0 || cfg.px_per_thread == 3 || cfg.px_per_thread > 4) return false;
  if (cfg.px_per_thread == 4 && cfg.tile_h % 16 != 0) return false;  // warp block 8 x 16
  if (cfg.recompute_bwd != 0 && cfg.recompute_bwd != 1) return false;
  if (cfg.spin_limit < 0) return false;
  L->spin_limit = cfg.spin_limit ? (uint32_t)cfg.spin_limit : (1u << 22);
  L->ppt = cfg.px_per_thread == 0 ? 2 : cfg.px_per_thread;
  uint64_t tiles = 0;
  for (int v = 0; v < n_views; ++v) {
    if (!cam_ok(cams[v])) return false;
    const uint64_t gx = (uint64_t)(cams[v].width + cfg.tile_w - 1) / cfg.tile_w;
    const uint64_t gy = (uint64_t)(cams[v].height + cfg.tile_h - 1) / cfg.tile_h;
    tiles += gx * gy;
  }
  if (tiles >= (1ull << 31)) return false;
  L->total_tiles = (int64_t)tiles;
  L->cam0_w = cams[0].width;
  L->cam0_h = cams[0].height;
  L->npix = n_views == 1 ? (int64_t)cams[0].width * cams[0].height : 0;
  const int64_t max_cap = (1ll << 31) - 1;
  int64_t rcap = cfg.record_capacity > 0 ? cfg.record_capacity : (int64_t)scene->n * n_views;
  if (rcap > max_cap) rcap = max_cap;
  int64_t pcap = cfg.pair_capacity > 0 ? cfg.pair_capacity : 8 * rcap;
  if (pcap > max_cap) pcap = max_cap;
  L->rcap = rcap;
  L->pcap = pcap;
  L->proj_blocks = ((int64_t)scene->n + kProjBlock - 1) / kProjBlock;
  L->key_bits_depth = 31 + (n_views > 1 ? bits_for((uint64_t)(n_views - 1)) : 0);
  L->key_bits_tile = bits_for(tiles > 0 ? tiles - 1 : 0);
  const size_t A = 256;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, A); return o; };
  L->off_counters = take(sizeof(Counters));
  L->off_cams = take(sizeof(DevCam) * n_views);
  L->off_tile_off = take(sizeof(uint32_t) * (n_views + 1));
  L->off_blockcnt = take(sizeof(uint32_t) * (size_t)(L->proj_blocks * n_views + 1));
  L->off_rec_uv = take(8 * (size_t)rcap);
  L->off_rec_conic = take(16 * (size_t)rcap);
  L->off_rec_depth = take(4 * (size_t)rcap);
  L->off_rec_rect = take(8 * (size_t)rcap);
  L->off_rec_gid = take(4 * (size_t)rcap);
  L->off_rec_view = take(4 * (size_t)rcap);
  L->off_rec_box = take(8 * (size_t)rcap);
  L->off_rec_cd = take(16 * (size_t)rcap);
  L->off_rec_unc = take(4 * (size_t)rcap);
  L->off_rec_sem = take(8 * (size_t)rcap * scene->k);
  for (int i = 0; i < 2; ++i) L->off_dkeys[i] = take(8 * (size_t)rcap);
  for (int i = 0; i < 2; ++i) L->off_dvals[i] = take(4 * (size_t)rcap);
  L->off_epart = take(sizeof(uint32_t) * (kEmitCtasMax + 1));
  L->off_rloc = take(4 * (size_t)rcap);
  for (int i = 0; i < 2; ++i) L->off_pkeys[i] = take(4 * (size_t)pcap);
  for (int i = 0; i < 2; ++i) L->off_pvals[i] = take(4 * (size_t)pcap);
  L->off_tickets = take(sizeof(uint32_t) * 2 * kMaxRadixPasses);
  L->off_ghist = take(sizeof(uint32_t) * 2 * kMaxRadixPasses * kRadix);
  L->off_lb_depth = take(8 * (size_t)kRadix * sort_tiles(rcap) * radix_passes(L->key_bits_depth));
  L->off_lb_pairs = take(8 * (size_t)kRadix * sort_tiles(pcap) * radix_passes(L->key_bits_tile));
  L->off_ranges = take(8 * (size_t)(tiles > 0 ? tiles : 1));
  L->off_tfinal = take(4 * (size_t)(L->npix > 0 ? L->npix : 1));
  L->off_nlast = take(4 * (size_t)(L->npix > 0 ? L->npix : 1));
  L->off_grad2d = take(n_views == 1 ? 32 * (size_t)rcap : 32);
  L->nwc = (scene->m + 31) / 32;
  L->off_codes = take(n_views == 1 ? 4 * (size_t)L->npix * (2 * (1 + L->nwc)) : 32);
  L->off_lpart = take(n_views == 1 ? 3 * sizeof(double) * (size_t)(tiles > 0 ? tiles : 1) : 32);
  L->off_semg = take(n_views == 1 ? 4 * (size_t)scene->n * scene->k : 32);
  // Contributor bits: one unit = one staged batch of one tile, one bit per
  // (tile pixel, pair) (none with recompute_bwd: the passes after the blend
  // re-test the pairs).  The mapping view keeps every unit of 64 pairs; a
  // candidate call keeps at most cand_bits_bytes and renders its views in
  // waves whose units fit (a tile that still does not fit re-tests).
  if (cfg.cand_batch != 0 && cfg.cand_batch != 32 && cfg.cand_batch != 64 && cfg.cand_batch != 128) return false;
  if (cfg.cand_bits_bytes < 0) return false;
  L->cand_batch = cfg.cand_batch ? cfg.cand_batch : 64;
  {
    const int64_t tpx = (int64_t)cfg.tile_w * cfg.tile_h;
    const int64_t map_units = pcap / kBatch + (int64_t)tiles + 1;
    const int64_t cand_units = pcap / L->cand_batch + (int64_t)tiles + 1;
    const int64_t unit_bytes = (int64_t)(L->cand_batch / 8) * tpx;  // cand_batch bits per tile pixel
    int64_t bytes = cand_units * unit_bytes;
    if (n_views == 1 && 8 * map_units * tpx > bytes) bytes = 8 * map_units * tpx;
    const int64_t budget = cfg.cand_bits_bytes > 0 ? cfg.cand_bits_bytes : kCandBitsDefault;
    if (n_views > 1 && bytes > budget) bytes = budget;
    if (cfg.recompute_bwd) bytes = 0;
    L->mask_units = n_views == 1 ? bytes / (8 * tpx) : 0;
    L->cand_cap_units = bytes / unit_bytes;
    if (L->cand_cap_units < 1) {
      L->cand_cap_units = 0;
      bytes = 0;
    }
    // waves: enough for the worst case of the capacities, twice over for the
    // views that do not pack (at most one wave per view)
    const int64_t need = cand_units;
    int64_t waves = L->cand_cap_units > 0 ? 2 * ((need + L->cand_cap_units - 1) / L->cand_cap_units) : 1;
    if (need <= L->cand_cap_units) waves = 1;
    L->cand_waves = (int)(waves < n_views ? waves : n_views);
    L->off_mask_off = take(sizeof(uint32_t) * (size_t)(tiles + 1));
    L->off_masks = take(bytes > 0 ? (size_t)bytes : 32);
  }
  // last contributor of every (tile, pixel), written by the two-pass
  // candidate kernels (any number of views) whenever the bits exist
  L->off_clast = take(L->cand_cap_units ? 4 * (size_t)tiles * cfg.tile_w * cfg.tile_h : 32);
  L->off_cand_plan = take(sizeof(uint32_t) * (size_t)L->cand_waves * 5);
  L->total = off;
  return true;
}

WsPtrs ws_ptrs(const Layout &L, void *ws) {
  char *b = static_cast<char *>(ws);
  WsPtrs P;
  P.counters = reinterpret_cast<Counters *>(b + L.off_counters);
  P.cams = reinterpret_cast<DevCam *>(b + L.off_cams);
  P.tile_off = reinterpret_cast<uint32_t *>(b + L.off_tile_off);
  P.blockcnt = reinterpret_cast<uint32_t *>(b + L.off_blockcnt);
  P.rec_uv = reinterpret_cast<float2 *>(b + L.off_rec_uv);
  P.rec_conic = reinterpret_cast<float4 *>(b + L.off_rec_conic);
  P.rec_depth = reinterpret_cast<float *>(b + L.off_rec_depth);
  P.rec_rect = reinterpret_cast<short4 *>(b + L.off_rec_rect);
  P.rec_gid = reinterpret_cast<int32_t *>(b + L.off_rec_gid);
  P.rec_view = reinterpret_cast<int32_t *>(b + L.off_rec_view);
  P.rec_box = reinterpret_cast<short4 *>(b + L.off_rec_box);
  P.rec_cd = reinterpret_cast<float4 *>(b + L.off_rec_cd);
  P.rec_unc = reinterpret_cast<float *>(b + L.off_rec_unc);
  P.rec_sem = reinterpret_cast<int2 *>(b + L.off_rec_sem);
  for (int i = 0; i < 2; ++i) {
    P.dkeys[i] = reinterpret_cast<unsigned long long *>(b + L.off_dkeys[i]);
    P.dvals[i] = reinterpret_cast<uint32_t *>(b + L.off_dvals[i]);
    P.pkeys[i] = reinterpret_cast<uint32_t *>(b + L.off_pkeys[i]);
    P.pvals[i] = reinterpret_cast<uint32_t *>(b + L.off_pvals[i]);
  }
  P.epart = reinterpret_cast<uint32_t *>(b + L.off_epart);
  P.rloc = reinterpret_cast<uint32_t *>(b + L.off_rloc);
  P.tickets = reinterpret_cast<uint32_t *>(b + L.off_tickets);
  P.ghist = reinterpret_cast<uint32_t *>(b + L.off_ghist);
  P.lb_depth = reinterpret_cast<unsigned long long *>(b + L.off_lb_depth);
  P.lb_pairs = reinterpret_cast<unsigned long long *>(b + L.off_lb_pairs);
  P.ranges = reinterpret_cast<uint2 *>(b + L.off_ranges);
  P.tfinal = reinterpret_cast<float *>(b + L.off_tfinal);
  P.nlast = reinterpret_cast<uint32_t *>(b + L.off_nlast);
  P.grad2d = reinterpret_cast<float4 *>(b + L.off_grad2d);
  P.codes = reinterpret_cast<uint32_t *>(b + L.off_codes);
  P.lpart = reinterpret_cast<double *>(b + L.off_lpart);
  P.semg = reinterpret_cast<float *>(b + L.off_semg);
  P.mask_off = reinterpret_cast<uint32_t *>(b + L.off_mask_off);
  P.masks = reinterpret_cast<uint32_t *>(b + L.off_masks);
  P.clast = reinterpret_cast<uint32_t *>(b + L.off_clast);
  P.cand_plan = reinterpret_cast<uint32_t *>(b + L.off_cand_plan);
  return P;
}

void fill_cam_table(const gs_camera *cams, int n_views, int tw, int th, CamTable *tab) {
  uint32_t off = 0;
  for (int v = 0; v < n_views; ++v) {
    const gs_camera &c = cams[v];
    DevCam &d = tab->cam[v];
    d.fx = c.fx; d.fy = c.fy; d.cx = c.cx; d.cy = c.cy; d.near_plane = c.near_plane;
    d.r[0] = c.w2c[0]; d.r[1] = c.w2c[1]; d.r[2] = c.w2c[2];
    d.r[3] = c.w2c[4]; d.r[4] = c.w2c[5]; d.r[5] = c.w2c[6];
    d.r[6] = c.w2c[8]; d.r[7] = c.w2c[9]; d.r[8] = c.w2c[10];
    d.t[0] = c.w2c[3]; d.t[1] = c.w2c[7]; d.t[2] = c.w2c[11];
    d.width = c.width; d.height = c.height;
    d.tiles_x = (c.width + tw - 1) / tw;
    d.tiles_y = (c.height + th - 1) / th;
    d.tile_off = off;
    off += (uint32_t)(d.tiles_x * d.tiles_y);
  }
}

static bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

static bool scene_ptrs_ok(const gs_scene *s, bool need_sem) {
  if (s->n == 0) return true;
  if (!s->means || !s->scales || !s->quats || !s->opacity) return false;
  if (!aligned(s->quats, 16)) return false;
  if (need_sem && (!s->sem_ids || !s->sem_w)) return false;
  return true;
}

static bool shape_compiled(int tw, int th) {
  return (tw == 16 && th == 16) || (tw == 16 && th == 8) || (tw == 8 && th == 8) || (tw == 32 && th == 8);
}

#define GS_CHECK_CUDA(expr)                      \
  do {                                           \
    cudaError_t _e = (expr);                     \
    if (_e != cudaSuccess) return GS_ERR_CUDA;   \
  } while (0)

gs_status run_project_with(const Layout &L, const WsPtrs &P, const gs_scene &sc, const gs_camera *cams,
                           CamTable *tab, cudaStream_t s, bool first) {
  memset(tab, 0, sizeof(CamTable));
  fill_cam_table(cams, L.n_views, L.tile_w, L.tile_h, tab);
  GS_CHECK_CUDA(launch_setup_views(*tab, L.n_views, P, (uint32_t)L.total_tiles, first, s));
  GS_CHECK_CUDA(launch_project(L, P, sc, s));
  return GS_OK;
}

static gs_status run_project(const Layout &L, const WsPtrs &P, const gs_scene &sc, const gs_camera *cams,
                             cudaStream_t s, bool first = true) {
  std::vector<unsigned char> buf(sizeof(CamTable));
  return run_project_with(L, P, sc, cams, reinterpret_cast<CamTable *>(buf.data()), s, first);
}

gs_status run_bin_sort(const Layout &L, const WsPtrs &P, cudaStream_t s) {
  int dbuf = 0, pbuf = 0;
  GS_CHECK_CUDA(launch_radix_sort_u64(L, P, L.key_bits_depth, &dbuf, s));
  GS_CHECK_CUDA(launch_emit_pairs(L, P, dbuf, s));
  GS_CHECK_CUDA(launch_radix_sort_u32(L, P, L.key_bits_tile, &pbuf, s));
  GS_CHECK_CUDA(launch_tile_ranges(L, P, pbuf, s));
  return GS_OK;
}

// End (exclusive) of the view group that starts at view v0: views are
// added while the group's pixels stay within `budget` (at least one view);
// budget <= 0 puts every view in one group.
static int group_end(const gs_camera *views, int n_views, int v0, int64_t budget) {
  if (budget <= 0) return n_views;
  int v1 = v0;
  int64_t px = 0;
  while (v1 < n_views) {
    const int64_t p = (int64_t)views[v1].width * views[v1].height;
    if (v1 > v0 && px + p > budget) break;
    px += p;
    ++v1;
  }
  return v1;
}

static int64_t group_pixels(const gs_config *cfg) { return cfg ? cfg->cand_group_pixels : 0; }

// A view list that needs more than one group (only gs_render_candidates runs
// those).
static bool grouped(const gs_camera *views, int n_views, const gs_config *cfg) {
  return views && n_views > 0 && n_views <= kMaxViews && group_end(views, n_views, 0, group_pixels(cfg)) < n_views;
}

bool make_layout(const gs_scene *scene, const gs_camera *cams, int n_views, const gs_config *cfg, Layout *L) {
  if (group_pixels(cfg) < 0 || grouped(cams, n_views, cfg)) return false;
  return layout_views(scene, cams, n_views, cfg, L);
}

// Grouped candidate call: checks every group of views and returns the
// largest group's workspace bytes (0 if a group is invalid).
static size_t grouped_total(const gs_scene *scene, const gs_camera *cams, int n_views, const gs_config *cfg) {
  if (!cams || n_views < 1 || n_views > kMaxViews || group_pixels(cfg) < 0) return 0;
  size_t total = 0;
  for (int v0 = 0, v1; v0 < n_views; v0 = v1) {
    v1 = group_end(cams, n_views, v0, group_pixels(cfg));
    Layout L;
    if (!layout_views(scene, cams + v0, v1 - v0, cfg, &L)) return 0;
    total = std::max(total, L.total);
  }
  return total;
}

}  // namespace gs

using namespace gs;

extern "C" {

size_t gs_workspace_size(const gs_scene *scene, const gs_camera *cams, int n_views, const gs_config *cfg) {
  if (grouped(cams, n_views, cfg)) return grouped_total(scene, cams, n_views, cfg);
  Layout L;
  if (!make_layout(scene, cams, n_views, cfg, &L)) return 0;
  return L.total;
}

gs_status gs_workspace_layout(const gs_scene *scene, const gs_camera *cams, int n_views, const gs_config *cfg,
                              void *ws, gs_workspace_map *map) {
  Layout L;
  if (!map || !ws || !make_layout(scene, cams, n_views, cfg, &L)) return GS_ERR_ARG;
  WsPtrs P = ws_ptrs(L, ws);
  map->counters = P.counters;
  map->rec_uv = P.rec_uv;
  map->rec_conic = P.rec_conic;
  map->rec_depth = P.rec_depth;
  map->rec_rect = P.rec_rect;
  map->rec_gid = P.rec_gid;
  map->rec_view = P.rec_view;
  map->pair_tile = P.pkeys[pair_sort_buffer(L)];
  map->pair_rec = P.pvals[pair_sort_buffer(L)];
  map->tile_ranges = P.ranges;
  map->tile_offset = P.tile_off;
  map->record_capacity = L.rcap;
  map->pair_capacity = L.pcap;
  map->total_tiles = L.total_tiles;
  return GS_OK;
}

gs_status gs_project(const gs_scene *scene, const gs_camera *cams, int n_views, const gs_config *cfg, void *ws,
                     gs_stream_t stream) {
  Layout L;
  if (!ws || !aligned(ws, 256) || !make_layout(scene, cams, n_views, cfg, &L)) return GS_ERR_ARG;
  if (!scene_ptrs_ok(scene, false)) return GS_ERR_ARG;
  return run_project(L, ws_ptrs(L, ws), *scene, cams, (cudaStream_t)stream);
}

gs_status gs_bin_sort(const gs_scene *scene, const gs_camera *cams, int n_views, const gs_config *cfg, void *ws,
                      gs_stream_t stream) {
  Layout L;
  if (!ws || !aligned(ws, 256) || !make_layout(scene, cams, n_views, cfg, &L)) return GS_ERR_ARG;
  return run_bin_sort(L, ws_ptrs(L, ws), (cudaStream_t)stream);
}

gs_status gs_render_fwd(const gs_scene *scene, const gs_camera *cam, const gs_config *cfg, void *ws, float *rgb,
                        float *depth, float *sil, float *sem, gs_stream_t stream) {
  Layout L;
  if (!ws || !aligned(ws, 256) || !make_layout(scene, cam, 1, cfg, &L)) return GS_ERR_ARG;
  if (!scene_ptrs_ok(scene, true) || (scene->n > 0 && !scene->rgb)) return GS_ERR_ARG;
  if (!shape_compiled(L.tile_w, L.tile_h)) return GS_ERR_UNSUPPORTED;
  WsPtrs P = ws_ptrs(L, ws);
  GS_CHECK_CUDA(launch_render_fwd(L, P, pair_sort_buffer(L), *scene, rgb, depth, sil, sem, (cudaStream_t)stream));
  return GS_OK;
}

gs_status gs_render_bwd(const gs_scene *scene, const gs_camera *cam, const gs_config *cfg, void *ws,
                        const float *d_rgb, const float *d_depth, const float *d_sil, const float *d_sem,
                        float *g_means, float *g_scales, float *g_quats, float *g_opacity, float *g_rgb,
                        float *g_sem_w, gs_stream_t stream) {
  Layout L;
  if (!ws || !aligned(ws, 256) || !make_layout(scene, cam, 1, cfg, &L)) return GS_ERR_ARG;
  if (!scene_ptrs_ok(scene, true) || (scene->n > 0 && !scene->rgb)) return GS_ERR_ARG;
  if (scene->n > 0 && (!g_means || !g_scales || !g_quats || !g_opacity || !g_rgb || !g_sem_w)) return GS_ERR_ARG;
  if (!shape_compiled(L.tile_w, L.tile_h)) return GS_ERR_UNSUPPORTED;
  const gs_config c = cfg ? *cfg : default_config();
  WsPtrs P = ws_ptrs(L, ws);
  cudaStream_t s = (cudaStream_t)stream;
  GS_CHECK_CUDA(launch_render_bwd(L, P, pair_sort_buffer(L), *scene, d_rgb, d_depth, d_sil, d_sem,
                                  c.sem_detach_geometry ? 1 : 0, g_rgb, g_sem_w, s));
  GS_CHECK_CUDA(launch_project_bwd(L, P, *scene, g_means, g_scales, g_quats, g_opacity, s));
  return GS_OK;
}

gs_status gs_render_fwd_l1(const gs_scene *scene, const gs_camera *cam, const gs_config *cfg, void *ws,
                           const float *t_rgb, const float *t_depth, const float *t_sem, float *rgb, float *depth,
                           float *sil, float *sem, float *loss, gs_stream_t stream) {
  Layout L;
  if (!ws || !aligned(ws, 256) || !make_layout(scene, cam, 1, cfg, &L)) return GS_ERR_ARG;
  if (!scene_ptrs_ok(scene, true) || (scene->n > 0 && !scene->rgb)) return GS_ERR_ARG;
  if (!t_rgb || !t_depth || !loss) return GS_ERR_ARG;
  if (!shape_compiled(L.tile_w, L.tile_h)) return GS_ERR_UNSUPPORTED;
  WsPtrs P = ws_ptrs(L, ws);
  GS_CHECK_CUDA(launch_render_fwd_l1(L, P, pair_sort_buffer(L), *scene, t_rgb, t_depth, t_sem, rgb, depth, sil, sem,
                                     loss, (cudaStream_t)stream));
  return GS_OK;
}

gs_status gs_render_bwd_l1(const gs_scene *scene, const gs_camera *cam, const gs_config *cfg, void *ws,
                           const float *loss_scale, float *g_means, float *g_scales, float *g_quats,
                           float *g_opacity, float *g_rgb, float *g_sem_w, gs_stream_t stream) {
  Layout L;
  if (!ws || !aligned(ws, 256) || !make_layout(scene, cam, 1, cfg, &L)) return GS_ERR_ARG;
  if (!scene_ptrs_ok(scene, true) || (scene->n > 0 && !scene->rgb) || !loss_scale) return GS_ERR_ARG;
  if (scene->n > 0 && (!g_means || !g_scales || !g_quats || !g_opacity || !g_rgb || !g_sem_w)) return GS_ERR_ARG;
  if (!shape_compiled(L.tile_w, L.tile_h)) return GS_ERR_UNSUPPORTED;
  const gs_config c = cfg ? *cfg : default_config();
  WsPtrs P = ws_ptrs(L, ws);
  cudaStream_t s = (cudaStream_t)stream;
  GS_CHECK_CUDA(launch_render_bwd(L, P, pair_sort_buffer(L), *scene, nullptr, nullptr, nullptr, nullptr,
                                  c.sem_detach_geometry ? 1 : 0, g_rgb, g_sem_w, s, loss_scale));
  GS_CHECK_CUDA(launch_project_bwd(L, P, *scene, g_means, g_scales, g_quats, g_opacity, s));
  return GS_OK;
}

gs_status gs_render_fwd_dense(const gs_scene *scene, const gs_camera *cam, const gs_config *cfg, void *ws,
                              const float *sem_dense, float *rgb, float *depth, float *sil, float *sem,
                              gs_stream_t stream) {
  Layout L;
  if (!ws || !aligned(ws, 256) || !make_layout(scene, cam, 1, cfg, &L)) return GS_ERR_ARG;
  if (!scene_ptrs_ok(scene, true) || (scene->n > 0 && !scene->rgb)) return GS_ERR_ARG;
  if (sem && scene->n > 0 && !sem_dense) return GS_ERR_ARG;
  if (!shape_compiled(L.tile_w, L.tile_h) || !dense_supported(L)) return GS_ERR_UNSUPPORTED;
  WsPtrs P = ws_ptrs(L, ws);
  GS_CHECK_CUDA(launch_render_fwd_dense(L, P, pair_sort_buffer(L), *scene, sem_dense, rgb, depth, sil, sem,
                                        (cudaStream_t)stream));
  return GS_OK;
}

// Preconditions of the fused Sec. 3.1 objective beyond gs_render_fwd's.
static gs_status objective_supported(const Layout &L, const gs_scene *scene, const gs_config &c) {
  if (!c.sem_detach_geometry || !objective_fits(L, scene->k, scene->m)) return GS_ERR_UNSUPPORTED;
  return GS_OK;
}

gs_status gs_render_fwd_objective(const gs_scene *scene, const gs_camera *cam, const gs_config *cfg, void *ws,
                                  const float *t_rgb, const float *t_depth, const float *t_sem, float *rgb,
                                  float *depth, float *sil, float *loss, gs_stream_t stream) {
  Layout L;
  if (!ws || !aligned(ws, 256) || !make_layout(scene, cam, 1, cfg, &L)) return GS_ERR_ARG;
  if (!scene_ptrs_ok(scene, true) || (scene->n > 0 && !scene->rgb)) return GS_ERR_ARG;
  if (!t_rgb || !t_depth || !loss) return GS_ERR_ARG;
  if (!shape_compiled(L.tile_w, L.tile_h)) return GS_ERR_UNSUPPORTED;
  const gs_config c = cfg ? *cfg : default_config();
  const gs_status st = objective_supported(L, scene, c);
  if (st != GS_OK) return st;
  WsPtrs P = ws_ptrs(L, ws);
  GS_CHECK_CUDA(launch_render_fwd_objective(L, P, pair_sort_buffer(L), *scene, t_rgb, t_depth, t_sem, rgb, depth,
                                            sil, loss, (cudaStream_t)stream));
  return GS_OK;
}

gs_status gs_render_bwd_objective(const gs_scene *scene, const gs_camera *cam, const gs_config *cfg, void *ws,
                                  const float *loss_scale, float *g_means, float *g_scales, float *g_quats,
                                  float *g_opacity, float *g_rgb, float *g_sem_w, gs_stream_t stream) {
  Layout L;
  if (!ws || !aligned(ws, 256) || !make_layout(scene, cam, 1, cfg, &L)) return GS_ERR_ARG;
  if (!scene_ptrs_ok(scene, true) || (scene->n > 0 && !scene->rgb) || !loss_scale) return GS_ERR_ARG;
  if (scene->n > 0 && (!g_means || !g_scales || !g_quats || !g_opacity || !g_rgb || !g_sem_w)) return GS_ERR_ARG;
  if (!shape_compiled(L.tile_w, L.tile_h)) return GS_ERR_UNSUPPORTED;
  const gs_config c = cfg ? *cfg : default_config();
  const gs_status st = objective_supported(L, scene, c);
  if (st != GS_OK) return st;
  WsPtrs P = ws_ptrs(L, ws);
  cudaStream_t s = (cudaStream_t)stream;
  GS_CHECK_CUDA(launch_render_bwd(L, P, pair_sort_buffer(L), *scene, nullptr, nullptr, nullptr, nullptr, 1, g_rgb,
                                  g_sem_w, s, loss_scale, 1));
  GS_CHECK_CUDA(launch_add_semg(P, *scene, loss_scale, g_sem_w, s));
  GS_CHECK_CUDA(launch_project_bwd(L, P, *scene, g_means, g_scales, g_quats, g_opacity, s));
  return GS_OK;
}

gs_status gs_render_candidates(const gs_scene *scene, const gs_camera *views, int n_views, const gs_config *cfg,
                               void *ws, double *out, gs_stream_t stream) {
  if (!ws || !aligned(ws, 256) || !out || grouped_total(scene, views, n_views, cfg) == 0) return GS_ERR_ARG;
  if (!scene_ptrs_ok(scene, true)) return GS_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  // one projection, binning and candidate chain per group of views, each in
  // its own layout of the same workspace; the device status and the largest
  // counts carry over from group to group
  for (int v0 = 0, v1; v0 < n_views; v0 = v1) {
    v1 = group_end(views, n_views, v0, group_pixels(cfg));
    Layout L;
    if (!layout_views(scene, views + v0, v1 - v0, cfg, &L)) return GS_ERR_ARG;
    if (!shape_compiled(L.tile_w, L.tile_h)) return GS_ERR_UNSUPPORTED;
    WsPtrs P = ws_ptrs(L, ws);
    gs_status st = run_project(L, P, *scene, views + v0, s, v0 == 0);
    if (st != GS_OK) return st;
    st = run_bin_sort(L, P, s);
    if (st != GS_OK) return st;
    GS_CHECK_CUDA(launch_candidates(L, P, pair_sort_buffer(L), *scene, out + 3 * (size_t)v0, s));
  }
  return GS_OK;
}

gs_status gs_l1_loss(int64_t npix, int m, const float *rgb, const float *t_rgb, const float *depth,
                     const float *t_depth, const float *sem, const float *t_sem, float *d_rgb, float *d_depth,
                     float *d_sem, float *loss, double *partial, gs_stream_t stream) {
  if (npix < 1 || !loss || !partial) return GS_ERR_ARG;
  if ((rgb && !t_rgb) || (depth && !t_depth) || (sem && (!t_sem || m < 1))) return GS_ERR_ARG;
  if (sem && (!aligned(sem, 16) || !aligned(t_sem, 16) || (d_sem && !aligned(d_sem, 16)))) return GS_ERR_ARG;
  GS_CHECK_CUDA(launch_l1_loss(npix, m, rgb, t_rgb, depth, t_depth, sem, t_sem, d_rgb, d_depth, d_sem, loss, partial,
                               (cudaStream_t)stream));
  return GS_OK;
}

gs_status gs_mapping_loss(int64_t npix, int m, int k, const float *rgb, const float *t_rgb, const float *depth,
                          const float *t_depth, const float *sil, const float *sem, const float *t_sem, float *d_rgb,
                          float *d_depth, float *d_sem, float *loss, double *partial, gs_stream_t stream) {
  if (npix < 1 || !loss || !partial || !rgb || !t_rgb || !depth || !t_depth || !sil) return GS_ERR_ARG;
  if (sem && (!t_sem || m < 1 || k < 1 || k > kMaxK)) return GS_ERR_ARG;
  GS_CHECK_CUDA(launch_mapping_loss(npix, m, k, rgb, t_rgb, depth, t_depth, sil, sem, t_sem, d_rgb, d_depth, d_sem,
                                    loss, partial, (cudaStream_t)stream));
  return GS_OK;
}

void gs_testing_set_sm_query(int (*query)(void)) { g_sms_query.store(query); }

int64_t gs_testing_grid(int which) {
  switch (which) {
    case GS_GRID_EMIT_CHUNKS: return emit_chunks();
    case GS_GRID_EMIT_WRITE: return sm_grid(8);
    case GS_GRID_SORT_RESET: return sm_grid(2);
    case GS_GRID_RANGES: return sm_grid(4);
    case GS_GRID_ZERO_GRAD: return sm_grid(2);
    default: return -1;
  }
}

gs_status gs_read_counters(void *ws, gs_counters *out, gs_stream_t stream) {
  if (!ws || !out) return GS_ERR_ARG;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return GS_ERR_CUDA;
  Counters c;
  if (cudaMemcpy(&c, ws, sizeof(c), cudaMemcpyDeviceToHost) != cudaSuccess) return GS_ERR_CUDA;
  out->status = c.status;
  out->n_records = std::max(c.n_records, c.grp_records);
  out->n_pairs = std::max(c.n_pairs, c.grp_pairs);
  out->n_contrib = c.n_contrib;
  if (c.status & kStatusTimeout) return GS_ERR_TIMEOUT;  // first: later counts may be meaningless
  if (c.status & kStatusCapacity) return GS_ERR_CAPACITY;
  return GS_OK;
}

const char *gs_status_string(gs_status s) {
  switch (s) {
    case GS_OK: return "ok";
    case GS_ERR_ARG: return "invalid argument";
    case GS_ERR_CAPACITY: return "workspace capacity exceeded (records or pairs)";
    case GS_ERR_CUDA: return "CUDA error";
    case GS_ERR_TIMEOUT: return "bounded device wait timed out";
    case GS_ERR_UNSUPPORTED: return "configuration not compiled in";
    case GS_ERR_TOO_LARGE: return "sizes need more workspace than the fixed no-allocation scratch array holds";
  }
  return "unknown status";
}

}  // extern "C"
