// noalloc.cu -- the one entry point that allocates nothing.
//
// Some callers cannot call cudaMalloc or any allocating routine: plug-in
// hosts that own all device memory and hand none to their plug-ins, and
// real-time loops that must never block in an allocator (cudaMalloc and
// cudaFree may synchronise the device).  For them
// gs_render_fwd_noalloc runs the same projection, binning and forward-render
// kernels as gs_project + gs_bin_sort + gs_render_fwd, with the workspace
// placed in a file-scope device array of fixed size instead of a
// caller-allocated buffer.  Every GPU that loads this library holds that
// array (GS_NOALLOC_SCRATCH_BYTES) until the process exits.
#include <mutex>

#include "gs_internal.cuh"
#include "render_common.cuh"

namespace gs {

static __device__ __align__(256) unsigned char g_noalloc_scratch[GS_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
static void *g_scratch_ptr[kMaxDevices];
static std::mutex g_scratch_mu;

// Device address of the array for the current device.  In host code the
// symbol is only a host-side stand-in, so the address is looked up once per
// device (with that device current) and cached for the life of the process;
// it belongs to the device's primary context and does not survive a
// cudaDeviceReset of that device.
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
  // the same launch chains as gs_project, gs_bin_sort and gs_render_fwd; the
  // camera table lives in thread-local storage, not on the heap, and the
  // setup kernel clears the counters and status word left by the last call
  thread_local CamTable tab;
  st = run_project_with(L, P, *scene, cam, &tab, s);
  if (st != GS_OK) return st;
  st = run_bin_sort(L, P, s);
  if (st != GS_OK) return st;
  if (launch_render_fwd(L, P, pair_sort_buffer(L), *scene, rgb, depth, sil, sem, s) != cudaSuccess)
    return GS_ERR_CUDA;
  if (counters_out &&
      cudaMemcpyAsync(counters_out, P.counters, sizeof(gs_counters), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return GS_ERR_CUDA;
  return GS_OK;
}
