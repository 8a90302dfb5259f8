// stats.cu -- work counters of the blend passes, for the roofline figures.
//
// A separate pass over the binned views of a workspace (after gs_project and
// gs_bin_sort) that applies the per-pixel compositing rules of Eq. 1 once
// more and counts, per pixel: the (pixel, Gaussian) pairs whose pixel
// rectangle holds the pixel, up to and including the pair that stops it
// (the evaluations of the brute-force definition, N_eval); the subset of
// those inside the Gaussian's alpha box (the pairs the blend kernels
// evaluate; outside it alpha < 1/255 for sure); the contributions; and the
// classes of the composited Eq. 3 distribution above the 0.001 clip floor of
// Eq. 7 (the logarithms the candidate pass takes).  Decisions use the same
// instructions as the blend kernels.  It is not on the timed path: one CTA
// per (view, tile), batches staged with CTA barriers, class rows in shared
// memory (class chunks re-walk the pairs).
#include "gs_internal.cuh"
#include "render_common.cuh"

namespace gs {

struct StatsArgs {
  const uint2 *ranges;
  const uint32_t *pvals;
  RecPtrs rec;
  const short4 *rect;
  const DevCam *cams;
  const uint32_t *tile_off;
  int n_views, k, m;
  const Counters *counters;
  int mchunk, mstride, nchunks;
  unsigned long long *out;  // n_eval, n_eval_box, n_contrib, n_touched, n_pixels
  uint32_t *per_pixel;      // single view: (n_eval, n_contrib) of every pixel, or null
};

__host__ __device__ inline size_t stats_batch_bytes(int k) { return (size_t)kBatch * (16 + 8 + 8 + 8 + 8 * k); }

template <int TW, int TH>
__global__ void __launch_bounds__(TW *TH) k_work_stats(StatsArgs a) {
  using FP = Footprint<TW, TH>;
  constexpr int THREADS = FP::kThreads;
  extern __shared__ float4 smem4[];
  char *base = reinterpret_cast<char *>(smem4);
  float4 *s_co = reinterpret_cast<float4 *>(base);
  float2 *s_uv = reinterpret_cast<float2 *>(base + kBatch * 16);
  short4 *s_rect = reinterpret_cast<short4 *>(base + kBatch * 24);
  short4 *s_box = reinterpret_cast<short4 *>(base + kBatch * 32);
  int2 *s_sem = reinterpret_cast<int2 *>(base + kBatch * 40);
  float *sP = reinterpret_cast<float *>(base + stats_batch_bytes(a.k));
  __shared__ unsigned long long red[5];
  if (a.counters->status & kStatusTimeout) return;

  const uint32_t tile = blockIdx.x;
  int lo = 0, hi = a.n_views;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (a.tile_off[mid] <= tile) lo = mid; else hi = mid;
  }
  const DevCam &c = a.cams[lo];
  const uint32_t local = tile - c.tile_off;
  const int ox = (int)(local % (uint32_t)c.tiles_x) * TW, oy = (int)(local / (uint32_t)c.tiles_x) * TH;
  const uint2 rg = a.ranges[tile];
  const int px = ox + FP::lx(), py = oy + FP::ly(0);
  const bool inside = px < c.width && py < c.height;
  const float fpx = (float)px + 0.5f, fpy = (float)py + 0.5f;
  float *myP = sP + threadIdx.x * a.mstride;
  const int k = a.k;
  if (threadIdx.x < 5) red[threadIdx.x] = 0ull;

  unsigned long long ne = 0, nb = 0, nc = 0, nt = 0;
  for (int ch = 0; ch < a.nchunks; ++ch) {
    const int c_lo = ch * a.mchunk, c_hi = min(a.m, c_lo + a.mchunk), mc = c_hi - c_lo;
    for (int q = 0; q < mc; ++q) myP[q] = 0.f;
    float T = 1.f;
    bool done = !inside;
    for (uint32_t b = rg.x; b < rg.y; b += kBatch) {
      const int n = (int)min((uint32_t)kBatch, rg.y - b);
      __syncthreads();
      for (int t = threadIdx.x; t < n; t += THREADS) {
        const uint32_t r = a.pvals[b + t];
        s_co[t] = __ldg(a.rec.co + r);
        s_uv[t] = __ldg(a.rec.uv + r);
        s_rect[t] = __ldg(a.rect + r);
        s_box[t] = __ldg(a.rec.box + r);
        for (int l = 0; l < k; ++l) s_sem[t * k + l] = __ldg(a.rec.sem + (size_t)r * k + l);
      }
      __syncthreads();
      for (int j = 0; j < n && !done; ++j) {
        const short4 rc = s_rect[j];
        if (px < rc.x || px > rc.y || py < rc.z || py > rc.w) continue;
        if (ch == 0) ++ne;
        const short4 bx = s_box[j];
        if (px < bx.x || px > bx.y || py < bx.z || py > bx.w) continue;
        if (ch == 0) ++nb;
        float alpha, G, araw, dx, dy;
        if (!gauss_alpha(s_uv[j], s_co[j], fpx, fpy, alpha, G, araw, dx, dy)) continue;
        const float Tn = __fmul_rn(T, __fsub_rn(1.f, alpha));
        if (Tn < kTStop) { done = true; break; }
        const float w = __fmul_rn(alpha, T);
        for (int l = 0; l < k; ++l) {
          const int id = s_sem[j * k + l].x - c_lo;
          if ((unsigned)id < (unsigned)mc) myP[id] = fmaf(w, __int_as_float(s_sem[j * k + l].y), myP[id]);
        }
        if (ch == 0) ++nc;
        T = Tn;
      }
      if (__syncthreads_count(done) == THREADS) break;
    }
    if (inside)
      for (int q = 0; q < mc; ++q) nt += myP[q] > 0.001f ? 1ull : 0ull;
  }
  if (a.per_pixel && inside) {
    const size_t pix = (size_t)py * c.width + px;
    a.per_pixel[2 * pix] = (uint32_t)ne;
    a.per_pixel[2 * pix + 1] = (uint32_t)nc;
  }
  atomicAdd(&red[0], ne);
  atomicAdd(&red[1], nb);
  atomicAdd(&red[2], nc);
  atomicAdd(&red[3], nt);
  atomicAdd(&red[4], inside ? 1ull : 0ull);
  __syncthreads();
  if (threadIdx.x < 5 && red[threadIdx.x]) atomicAdd(a.out + threadIdx.x, red[threadIdx.x]);
}

__global__ void k_zero_u64(unsigned long long *p, int n) {
  if ((int)threadIdx.x < n) p[threadIdx.x] = 0ull;
}

template <int TW, int TH>
static cudaError_t launch_stats_shape(const StatsArgs &a, uint32_t grid, size_t smem, cudaStream_t s) {
  {
    const cudaError_t e = ensure_smem_limit((const void *)k_work_stats<TW, TH>, (int)kSmemBudget);
    if (e != cudaSuccess) return e;
  }
  k_work_stats<TW, TH><<<grid, TW * TH, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_work_stats(const Layout &L, const WsPtrs &P, int pbuf, const gs_scene &sc,
                              unsigned long long *out, uint32_t *per_pixel, cudaStream_t s) {
  k_zero_u64<<<1, 32, 0, s>>>(out, 5);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  StatsArgs a{};
  a.ranges = P.ranges;
  a.pvals = P.pvals[pbuf];
  a.rec = rec_ptrs(P);
  a.rect = P.rec_rect;
  a.cams = P.cams;
  a.tile_off = P.tile_off;
  a.n_views = L.n_views; a.k = sc.k; a.m = sc.m;
  a.counters = P.counters;
  a.out = out;
  a.per_pixel = per_pixel;
  const int threads = L.tile_w * L.tile_h;
  chunk_classes(sc.m, threads, sc.k, true, &a.mchunk, &a.mstride, &a.nchunks,
                stats_batch_bytes(sc.k) - batch_smem_bytes(sc.k));
  const size_t smem = stats_batch_bytes(sc.k) + (size_t)threads * a.mstride * sizeof(float);
  const uint32_t grid = (uint32_t)L.total_tiles;
  if (grid == 0) return cudaSuccess;
  if (L.tile_w == 16 && L.tile_h == 16) return launch_stats_shape<16, 16>(a, grid, smem, s);
  if (L.tile_w == 16 && L.tile_h == 8) return launch_stats_shape<16, 8>(a, grid, smem, s);
  if (L.tile_w == 8 && L.tile_h == 8) return launch_stats_shape<8, 8>(a, grid, smem, s);
  if (L.tile_w == 32 && L.tile_h == 8) return launch_stats_shape<32, 8>(a, grid, smem, s);
  return cudaErrorInvalidConfiguration;
}

}  // namespace gs

using namespace gs;

extern "C" gs_status gs_count_work(const gs_scene *scene, const gs_camera *cams, int n_views, const gs_config *cfg,
                                   void *ws, gs_work_counts *out, uint32_t *per_pixel, gs_stream_t stream) {
  Layout L;
  if (!ws || !out || (reinterpret_cast<uintptr_t>(ws) % 256) != 0 || !make_layout(scene, cams, n_views, cfg, &L))
    return GS_ERR_ARG;
  if (reinterpret_cast<uintptr_t>(out) % 8 != 0 || (per_pixel && n_views != 1)) return GS_ERR_ARG;
  if (scene->n > 0 && (!scene->sem_ids || !scene->sem_w)) return GS_ERR_ARG;
  if (!((L.tile_w == 16 && L.tile_h == 16) || (L.tile_w == 16 && L.tile_h == 8) || (L.tile_w == 8 && L.tile_h == 8) ||
        (L.tile_w == 32 && L.tile_h == 8)))
    return GS_ERR_UNSUPPORTED;
  const WsPtrs P = ws_ptrs(L, ws);
  if (launch_work_stats(L, P, pair_sort_buffer(L), *scene, reinterpret_cast<unsigned long long *>(out), per_pixel,
                        (cudaStream_t)stream) != cudaSuccess)
    return GS_ERR_CUDA;
  return GS_OK;
}
