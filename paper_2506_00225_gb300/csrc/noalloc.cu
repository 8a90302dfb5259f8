// noalloc.cu -- the one entry point that allocates nothing.
//
// Some callers cannot call cudaMalloc or any allocating routine: code
// running inside a CUDA-graph capture, real-time loops that must not block in
// an allocator, and plug-in hosts that own all device memory.  For them
// gs_render_fwd_noalloc runs the same projection, binning and forward-render
// kernels as gs_project + gs_bin_sort + gs_render_fwd, with the workspace
// placed in a file-scope device array of fixed size instead of a
// caller-allocated buffer.  Every GPU that loads this library holds that
// array (GS_NOALLOC_SCRATCH_BYTES) until the process exits.
#include <mutex>
#include <string.h>

#include "gs_internal.cuh"
#include "render_common.cuh"

namespace gs {

static __device__ __align__(256) unsigned char g_noalloc_scratch[GS_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
static void *g_scratch_ptr[kMaxDevices];
static std::mutex g_scratch_mu;

// Device address of the array for the current device.  In host code the
// symbol is only a host-side stand-in, so the address is looked up once per
// device (with that device current) and cached.
static gs_status scratch_for_current_device(void **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GS_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return GS_ERR_CUDA;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return GS_OK;
}

// Fills the kernel-parameter camera table without touching the heap.
static void fill_table(const gs_camera *c, int tw, int th, CamTable *tab) {
  DevCam &d = tab->cam[0];
  d.fx = c->fx; d.fy = c->fy; d.cx = c->cx; d.cy = c->cy; d.near_plane = c->near_plane;
  d.r[0] = c->w2c[0]; d.r[1] = c->w2c[1]; d.r[2] = c->w2c[2];
  d.r[3] = c->w2c[4]; d.r[4] = c->w2c[5]; d.r[5] = c->w2c[6];
  d.r[6] = c->w2c[8]; d.r[7] = c->w2c[9]; d.r[8] = c->w2c[10];
  d.t[0] = c->w2c[3]; d.t[1] = c->w2c[7]; d.t[2] = c->w2c[11];
  d.width = c->width; d.height = c->height;
  d.tiles_x = (c->width + tw - 1) / tw;
  d.tiles_y = (c->height + th - 1) / th;
  d.tile_off = 0;
}

}  // namespace gs

using namespace gs;

extern "C" gs_status gs_render_fwd_noalloc(const gs_scene *scene, const gs_camera *cam, const gs_config *cfg,
                                           float *rgb, float *depth, float *sil, float *sem,
                                           gs_counters *counters_out, gs_stream_t stream) {
  Layout L;
  if (!make_layout(scene, cam, 1, cfg, &L)) return GS_ERR_ARG;
  if (scene->n > 0 && (!scene->means || !scene->scales || !scene->quats || !scene->opacity || !scene->rgb ||
                       !scene->sem_ids || !scene->sem_w))
    return GS_ERR_ARG;
  if (scene->n > 0 && (reinterpret_cast<uintptr_t>(scene->quats) % 16) != 0) return GS_ERR_ARG;
  if (!((L.tile_w == 16 && L.tile_h == 16) || (L.tile_w == 16 && L.tile_h == 8) || (L.tile_w == 8 && L.tile_h == 8) ||
        (L.tile_w == 32 && L.tile_h == 8)))
    return GS_ERR_UNSUPPORTED;
  if (L.total > (size_t)GS_NOALLOC_SCRATCH_BYTES) return GS_ERR_TOO_LARGE;
  void *ws = nullptr;
  gs_status st = scratch_for_current_device(&ws);
  if (st != GS_OK) return st;
  const WsPtrs P = ws_ptrs(L, ws);
  cudaStream_t s = (cudaStream_t)stream;
  thread_local CamTable tab;
  memset(&tab, 0, sizeof(tab));
  fill_table(cam, L.tile_w, L.tile_h, &tab);
  // the setup kernel clears the counters and status word left by the last call
  if (launch_setup_views(tab, 1, P, (uint32_t)L.total_tiles, true, s) != cudaSuccess) return GS_ERR_CUDA;
  if (launch_project(L, P, *scene, s) != cudaSuccess) return GS_ERR_CUDA;
  int dbuf = 0, pbuf = 0;
  if (launch_radix_sort_u64(L, P, L.key_bits_depth, &dbuf, s) != cudaSuccess) return GS_ERR_CUDA;
  if (launch_emit_pairs(L, P, dbuf, s) != cudaSuccess) return GS_ERR_CUDA;
  if (launch_radix_sort_u32(L, P, L.key_bits_tile, &pbuf, s) != cudaSuccess) return GS_ERR_CUDA;
  if (launch_tile_ranges(L, P, pbuf, s) != cudaSuccess) return GS_ERR_CUDA;
  if (launch_render_fwd(L, P, pbuf, *scene, rgb, depth, sil, sem, s) != cudaSuccess) return GS_ERR_CUDA;
  if (counters_out &&
      cudaMemcpyAsync(counters_out, P.counters, sizeof(gs_counters), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return GS_ERR_CUDA;
  return GS_OK;
}
