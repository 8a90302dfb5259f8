// candidates.cu -- batched candidate-view rendering for next-best-view
// scoring (Sec. 3.2).
//
// One launch covers every (view, tile) of all candidate views (mixed
// resolutions share one projection and one binning pass).  Per pixel it
// composites the silhouette (Eq. 1, z_i = 1), the per-Gaussian scalar
// uncertainty (Eq. 1, z_i = u_i) and the sparse semantic map (Eq. 3), then
// computes the entropy (Eq. 4) of the map clipped to [0.001, 1] and
// renormalised (Eq. 7) as H = ln Z - (sum_m p_m ln p_m) / Z, with
// Z = sum_m p_m; classes at the clip floor are counted rather than
// logged one by one.  Per-view sums of U and H and the number of pixels with
// S = 0 (Eq. 6) are reduced per CTA and added to the view's accumulators in
// double precision.  No per-pixel map is written.
#include "gs_internal.cuh"
#include "render_common.cuh"

namespace gs {

struct CandArgs {
  const uint2 *ranges;
  const uint32_t *pvals;
  RecPtrs rec;
  const float *unc;
  const DevCam *cams;
  const uint32_t *tile_off;
  int n_views, k, m;
  double *out;
  int mchunk, mstride, nchunks;
};

constexpr float kClipLo = 0.001f;

template <int TW, int TH>
__global__ void __launch_bounds__(TW *TH) k_candidates(CandArgs a) {
  using FP = Footprint<TW, TH>;
  constexpr int THREADS = FP::kThreads;
  extern __shared__ float4 smem4[];
  BatchSmem bs = batch_smem(smem4, a.k);
  float *sP = bs.tail;
  __shared__ float red_u[THREADS / 32], red_h[THREADS / 32];
  __shared__ uint32_t red_n[THREADS / 32];

  const uint32_t tile = blockIdx.x;
  // view of this tile: last v with tile_off[v] <= tile
  int lo = 0, hi = a.n_views;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (a.tile_off[mid] <= tile) lo = mid; else hi = mid;
  }
  const int v = lo;
  const DevCam &c = a.cams[v];
  const uint32_t local = tile - c.tile_off;
  const int ox = (int)(local % (uint32_t)c.tiles_x) * TW, oy = (int)(local / (uint32_t)c.tiles_x) * TH;
  const uint2 rg = a.ranges[tile];
  const int px = ox + FP::lx(), py = oy + FP::ly(0);
  const bool inside = px < c.width && py < c.height;
  const float fpx = (float)px + 0.5f, fpy = (float)py + 0.5f;
  float *myP = sP + threadIdx.x * a.mstride;
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
  const int k = a.k;
  const bool use_unc = a.unc != nullptr;

  float T = 1.f, U = 0.f, Z = 0.f, Aacc = 0.f;
  uint32_t nfloor = 0;
  for (int ch = 0; ch < a.nchunks; ++ch) {
    const int c_lo = ch * a.mchunk, c_hi = min(a.m, c_lo + a.mchunk), mc = c_hi - c_lo;
    for (int i = 0; i < mc; ++i) myP[i] = 0.f;
    T = 1.f; U = 0.f;
    bool done = !inside;
    for (uint32_t b = rg.x; b < rg.y; b += kBatch) {
      const int n = (int)min((uint32_t)kBatch, rg.y - b);
      __syncthreads();
      for (int t = threadIdx.x; t < n; t += THREADS)
        stage_record<TW, TH>(a.rec, a.pvals[b + t], t, k, ox, oy, bs, true, use_unc);
      __syncthreads();
      if (!__all_sync(0xffffffffu, done)) {
        for (int base = 0; base < n; base += 32) {
          const int jj = base + (int)lane;
          uint32_t vis = __ballot_sync(0xffffffffu, jj < n && ((bs.wmask[jj] >> warp) & 1u));
          while (vis) {
            const int j = base + __ffs(vis) - 1;
            vis &= vis - 1;
            if (done || !box_holds(bs.box[j], px, py)) continue;
            float alpha, G, araw, dx, dy;
            if (!gauss_alpha(bs.uv[j], bs.co[j], fpx, fpy, alpha, G, araw, dx, dy)) continue;
            const float Tn = __fmul_rn(T, __fsub_rn(1.f, alpha));
            if (Tn < kTStop) { done = true; continue; }
            const float w = __fmul_rn(alpha, T);
            U = fmaf(w, bs.cd[j].x, U);
            const int2 *sp = bs.sem + j * k;
            for (int l = 0; l < k; ++l) {
              const int2 e = sp[l];
              const int id = e.x - c_lo;
              if ((unsigned)id < (unsigned)mc) myP[id] = fmaf(w, __int_as_float(e.y), myP[id]);
            }
            T = Tn;
          }
        }
      }
      if (__syncthreads_count(done) == THREADS) break;
    }
    if (inside) {
      for (int i = 0; i < mc; ++i) {
        const float p = myP[i];
        if (p > kClipLo) {
          const float ph = p < 1.f ? p : 1.f;
          Z += ph;
          Aacc = fmaf(ph, logf(ph), Aacc);
        } else {
          ++nfloor;
        }
      }
    }
  }
  float h = 0.f, u = 0.f;
  uint32_t ns = 0;
  if (inside) {
    const float zf = kClipLo * (float)nfloor;
    Z += zf;
    Aacc = fmaf(zf, logf(kClipLo), Aacc);
    h = logf(Z) - Aacc / Z;
    u = use_unc ? U : 0.f;
    ns = (T == 1.f) ? 1u : 0u;
  }
  // block reduction
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    h += __shfl_xor_sync(0xffffffffu, h, o);
    u += __shfl_xor_sync(0xffffffffu, u, o);
    ns += __shfl_xor_sync(0xffffffffu, ns, o);
  }
  if (lane == 0) { red_h[warp] = h; red_u[warp] = u; red_n[warp] = ns; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sh = 0.0, su = 0.0;
    uint32_t sn = 0;
    for (int w = 0; w < THREADS / 32; ++w) { sh += red_h[w]; su += red_u[w]; sn += red_n[w]; }
    atomicAdd(a.out + 3 * v, su);
    atomicAdd(a.out + 3 * v + 1, sh);
    atomicAdd(a.out + 3 * v + 2, (double)sn);
  }
}

__global__ void k_zero_doubles(double *p, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = 0.0;
}

template <int TW, int TH>
static cudaError_t launch_cand_shape(const CandArgs &a, uint32_t grid, size_t smem, cudaStream_t s) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_candidates<TW, TH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kSmemBudget);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  k_candidates<TW, TH><<<grid, TW * TH, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_candidates(const Layout &L, const WsPtrs &P, int pbuf, const gs_scene &sc, double *out,
                              cudaStream_t s) {
  k_zero_doubles<<<(3 * L.n_views + 255) / 256, 256, 0, s>>>(out, 3 * L.n_views);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  CandArgs a{};
  a.ranges = P.ranges;
  a.pvals = P.pvals[pbuf];
  a.rec = rec_ptrs(P);
  a.unc = sc.geo_unc;
  a.cams = P.cams; a.tile_off = P.tile_off;
  a.n_views = L.n_views; a.k = sc.k; a.m = sc.m;
  a.out = out;
  const int threads = L.tile_w * L.tile_h;
  chunk_classes(sc.m, threads, sc.k, true, &a.mchunk, &a.mstride, &a.nchunks);
  const size_t smem = batch_smem_bytes(sc.k) + (size_t)threads * a.mstride * sizeof(float);
  const uint32_t grid = (uint32_t)L.total_tiles;
  if (grid == 0) return cudaSuccess;
  if (L.tile_w == 16 && L.tile_h == 16) return launch_cand_shape<16, 16>(a, grid, smem, s);
  if (L.tile_w == 16 && L.tile_h == 8) return launch_cand_shape<16, 8>(a, grid, smem, s);
  if (L.tile_w == 8 && L.tile_h == 8) return launch_cand_shape<8, 8>(a, grid, smem, s);
  if (L.tile_w == 32 && L.tile_h == 8) return launch_cand_shape<32, 8>(a, grid, smem, s);
  return cudaErrorInvalidConfiguration;
}

}  // namespace gs
