// render_fwd.cu -- forward tile blend: Eq. 1 (colour, depth, silhouette) and
// Eq. 3 (sparse top-k semantics), supplement "Sparse Rendering".
//
// One CTA per screen tile, one thread per pixel, each warp an 8 x 4 pixel
// block.  The tile's depth-sorted pair range is walked in batches staged in
// shared memory; for every staged Gaussian the stager records which warps'
// blocks meet its alpha box (the pixels where alpha can reach 1/255), and
// each warp visits only those Gaussians.  A thread composites a Gaussian
// whose box holds its pixel, front to back, and stops before the Gaussian
// that would take the transmittance below 1e-4; the CTA leaves when every
// pixel is done (__syncthreads_count).  Semantic probabilities are scattered
// into a per-pixel M-class accumulator in shared memory (k adds per
// contributor instead of M, the point of the sparse representation), then
// written out with coalesced stores.  When M does not fit, classes are
// processed in chunks of 32-class multiples, recompositing per chunk.
//
// Fused mean-L1 mode (L1 = true): the rendered colour, depth and semantic
// distribution are compared with the targets inside the tile; the kernel
// keeps per-tile sums of |rendered - target| and, per value, two bits
// (nonzero, negative) of the sign of the difference for the adjoint.  The
// tile's target rows are prefetched into L2 with bulk-copy prefetches when
// the CTA starts, so the comparison reads them from L2.
#include "gs_internal.cuh"
#include "render_common.cuh"

namespace gs {

// L2 prefetch of [p, p + bytes) clipped to 16-byte granules inside
// [base, base + total).
__device__ __forceinline__ void prefetch_l2(const void *base, size_t total, const void *p, size_t bytes) {
  const uintptr_t b = reinterpret_cast<uintptr_t>(base);
  const uintptr_t lo = (reinterpret_cast<uintptr_t>(p) + 15) & ~(uintptr_t)15;
  uintptr_t hi = (reinterpret_cast<uintptr_t>(p) + bytes) & ~(uintptr_t)15;
  const uintptr_t end = (b + total) & ~(uintptr_t)15;
  if (hi > end) hi = end;
  if (lo < b || hi <= lo) return;
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(lo), "r"((uint32_t)(hi - lo)) : "memory");
}

template <int TW, int TH, bool L1, int PPT>
__global__ void __launch_bounds__(TW *TH / PPT) k_render_fwd(FwdArgs a) {
  using FP = Footprint<TW, TH, PPT>;
  constexpr int THREADS = FP::kThreads;
  constexpr int WARPS = FP::kWarps;
  constexpr int NPIX = FP::kPix;
  extern __shared__ float4 smem4[];
  BatchSmem bs = batch_smem(smem4, a.k);
  float *sP = bs.tail;
  __shared__ float red[3][WARPS];

  const int tile = blockIdx.x;
  const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
  const int ox = tx * TW, oy = ty * TH;
  const uint2 rg = a.ranges[tile];
  const int lx = FP::lx();
  const int px = ox + lx;
  const float fpx = (float)px + 0.5f;
  int py[PPT];
  bool inside[PPT];
  float fpy[PPT];
  float *myP[PPT];
#pragma unroll
  for (int i = 0; i < PPT; ++i) {
    const int ly = FP::ly(i);
    py[i] = oy + ly;
    inside[i] = px < a.width && py[i] < a.height;
    fpy[i] = (float)py[i] + 0.5f;
    myP[i] = sP + (ly * TW + lx) * a.mstride;
  }
  const bool acc_sem = a.sem != nullptr || (L1 && a.t_sem != nullptr);
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
  const int cw = code_words(a.nwc);
  const int k = a.k;
  float l1_sem = 0.f;

  if (L1 && a.t_sem && (int)threadIdx.x < TH) {
    const int y = oy + (int)threadIdx.x;
    if (y < a.height) {
      const int vw = min(TW, a.width - ox);
      prefetch_l2(a.t_sem, (size_t)a.width * a.height * a.m * 4, a.t_sem + ((size_t)y * a.width + ox) * a.m,
                  (size_t)vw * a.m * 4);
    }
  }

  float T[PPT], cr[PPT], cg[PPT], cb[PPT], cd[PPT];
  uint32_t last[PPT];
  uint32_t ncontrib = 0;
  for (int c = 0; c < a.nchunks; ++c) {
    const int c_lo = c * a.mchunk, c_hi = min(a.m, c_lo + a.mchunk);
    const int mc = c_hi - c_lo;
    bool done[PPT];
#pragma unroll
    for (int i = 0; i < PPT; ++i) {
      if (acc_sem)
        for (int q = 0; q < mc; ++q) myP[i][q] = 0.f;
      T[i] = 1.f; cr[i] = cg[i] = cb[i] = cd[i] = 0.f; last[i] = 0;
      done[i] = !inside[i];
    }
    ncontrib = 0;
    for (uint32_t b = rg.x; b < rg.y; b += kBatch) {
      const int n = (int)min((uint32_t)kBatch, rg.y - b);
      __syncthreads();
      for (int t = threadIdx.x; t < n; t += THREADS)
        stage_record<TW, TH, PPT>(a.rec, a.pvals[b + t], t, k, ox, oy, bs, acc_sem, false);
      __syncthreads();
      bool all_done = true;
#pragma unroll
      for (int i = 0; i < PPT; ++i) all_done = all_done && done[i];
      if (!__all_sync(0xffffffffu, all_done)) {
        for (int base = 0; base < n; base += 32) {
          const int jj = base + (int)lane;
          uint32_t vis = __ballot_sync(0xffffffffu, jj < n && ((bs.wmask[jj] >> warp) & 1u));
          while (vis) {
            const int j = base + __ffs(vis) - 1;
            vis &= vis - 1;
            const int2 bb = bs.box[j];
            bool hold[PPT];
            bool any = false;
#pragma unroll
            for (int i = 0; i < PPT; ++i) {
              hold[i] = !done[i] && box_holds(bb, px, py[i]);
              any = any || hold[i];
            }
            if (!any) continue;
            const float2 uv = bs.uv[j];
            const float4 co = bs.co[j];
            const float4 cdp = bs.cd[j];
#pragma unroll
            for (int i = 0; i < PPT; ++i) {
              if (!hold[i]) continue;
              float alpha, G, araw, dx, dy;
              if (!gauss_alpha(uv, co, fpx, fpy[i], alpha, G, araw, dx, dy)) continue;
              const float Tn = __fmul_rn(T[i], __fsub_rn(1.f, alpha));
              if (Tn < kTStop) { done[i] = true; continue; }
              const float w = __fmul_rn(alpha, T[i]);
              cr[i] = fmaf(w, cdp.x, cr[i]); cg[i] = fmaf(w, cdp.y, cg[i]); cb[i] = fmaf(w, cdp.z, cb[i]);
              cd[i] = fmaf(w, cdp.w, cd[i]);
              if (acc_sem) {
                const int2 *sp = bs.sem + j * k;
                for (int l = 0; l < k; ++l) {
                  const int2 e = sp[l];
                  const int id = e.x - c_lo;
                  if ((unsigned)id < (unsigned)mc) myP[i][id] = fmaf(w, __int_as_float(e.y), myP[i][id]);
                }
              }
              T[i] = Tn;
              last[i] = b - rg.x + j + 1;
              ++ncontrib;
            }
          }
        }
      }
      bool my_done = true;
#pragma unroll
      for (int i = 0; i < PPT; ++i) my_done = my_done && done[i];
      if (__syncthreads_count(my_done) == THREADS) break;
    }
    if (acc_sem) {
      __syncthreads();
      const int vw = min(TW, a.width - ox);
      if (a.sem) {
        for (int r = 0; r < TH; ++r) {
          const int y = oy + r;
          if (y >= a.height) break;
          float *dst = a.sem + ((size_t)y * a.width + ox) * a.m + c_lo;
          const float *src = sP + (r * TW) * a.mstride;
          for (int e = threadIdx.x; e < vw * mc; e += THREADS) {
            const int p = e / mc, cl = e - p * mc;
            dst[(size_t)p * a.m + cl] = src[p * a.mstride + cl];
          }
        }
      }
      if (L1 && a.t_sem) {
        // each warp takes kG pixels x kWG 32-class words per round: all kG*kWG
        // coalesced target reads (L2 hits after the prefetch) are issued before
        // any is consumed; ballots assemble the sign words
        constexpr int kG = 4, kWG = 4;
        const int w_lo = c_lo >> 5, w_hi = (c_hi + 31) >> 5;
        for (int p0 = (int)warp * kG; p0 < NPIX; p0 += WARPS * kG) {
          for (int wb = w_lo; wb < w_hi; wb += kWG) {
            float tv[kG][kWG];
            const float *row[kG];
            bool okp[kG];
#pragma unroll
            for (int g = 0; g < kG; ++g) {
              const int p = p0 + g;
              const int qx = ox + p % TW, qy = oy + p / TW;
              okp[g] = qx < a.width && qy < a.height;
              row[g] = a.t_sem + (okp[g] ? ((size_t)qy * a.width + qx) * a.m : 0);
#pragma unroll
              for (int u = 0; u < kWG; ++u) {
                const int mcl = (wb + u) * 32 + (int)lane;
                tv[g][u] = (okp[g] && mcl < c_hi) ? __ldcs(row[g] + mcl) : 0.f;
              }
            }
#pragma unroll
            for (int g = 0; g < kG; ++g) {
              if (!okp[g]) continue;  // uniform over the warp
              const int p = p0 + g;
#pragma unroll
              for (int u = 0; u < kWG; ++u) {
                const int wd = wb + u;
                if (wd >= w_hi) break;
                const int mcl = wd * 32 + (int)lane;
                float d = 0.f;
                if (mcl < c_hi) d = sP[p * a.mstride + (mcl - c_lo)] - tv[g][u];
                const uint32_t nz = __ballot_sync(0xffffffffu, d != 0.f);
                const uint32_t ng = __ballot_sync(0xffffffffu, d < 0.f);
                l1_sem += fabsf(d);
                if (lane == 0) {
                  uint32_t *cp = a.codes + (size_t)((row[g] - a.t_sem) / a.m) * cw;
                  cp[1 + wd] = nz;
                  cp[2 + a.nwc + wd] = ng;
                }
              }
            }
          }
        }
      }
      __syncthreads();  // the next chunk reuses the accumulator rows
    }
  }
  {
    // diagnostics: total contributions (one atomic per warp)
    uint32_t nc = ncontrib;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nc += __shfl_xor_sync(0xffffffffu, nc, o);
    if (lane == 0 && nc) atomicAdd(&a.counters->n_contrib, nc);
  }
  float l1_rgb = 0.f, l1_d = 0.f;
#pragma unroll
  for (int i = 0; i < PPT; ++i) {
    if (!inside[i]) continue;
    const size_t pix = (size_t)py[i] * a.width + px;
    if (a.rgb_out) { a.rgb_out[3 * pix] = cr[i]; a.rgb_out[3 * pix + 1] = cg[i]; a.rgb_out[3 * pix + 2] = cb[i]; }
    if (a.depth_out) a.depth_out[pix] = cd[i];
    if (a.sil_out) a.sil_out[pix] = 1.f - T[i];
    a.tfinal[pix] = T[i];
    a.nlast[pix] = last[i];
    if (L1) {
      const float d0 = cr[i] - a.t_rgb[3 * pix], d1 = cg[i] - a.t_rgb[3 * pix + 1], d2 = cb[i] - a.t_rgb[3 * pix + 2];
      const float d3 = cd[i] - a.t_depth[pix];
      const uint32_t nz = (d0 != 0.f ? 1u : 0u) | (d1 != 0.f ? 2u : 0u) | (d2 != 0.f ? 4u : 0u) | (d3 != 0.f ? 8u : 0u);
      const uint32_t ng = (d0 < 0.f ? 1u : 0u) | (d1 < 0.f ? 2u : 0u) | (d2 < 0.f ? 4u : 0u) | (d3 < 0.f ? 8u : 0u);
      uint32_t *cp = a.codes + pix * cw;
      cp[0] = nz;
      cp[1 + a.nwc] = ng;
      if (!a.t_sem)
        for (int wd = 0; wd < a.nwc; ++wd) { cp[1 + wd] = 0u; cp[2 + a.nwc + wd] = 0u; }
      l1_rgb += fabsf(d0) + fabsf(d1) + fabsf(d2);
      l1_d += fabsf(d3);
    }
  }
  if (L1) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      l1_rgb += __shfl_xor_sync(0xffffffffu, l1_rgb, o);
      l1_d += __shfl_xor_sync(0xffffffffu, l1_d, o);
      l1_sem += __shfl_xor_sync(0xffffffffu, l1_sem, o);
    }
    if (lane == 0) { red[0][warp] = l1_rgb; red[1][warp] = l1_d; red[2][warp] = l1_sem; }
    __syncthreads();
    if (threadIdx.x < 3) {
      double s = 0.0;
      for (int w = 0; w < WARPS; ++w) s += red[threadIdx.x][w];
      a.lpart[3 * (size_t)tile + threadIdx.x] = s;
    }
  }
}

// loss = sum|d rgb| / (3 npix) + sum|d depth| / npix + sum|d sem| / (npix m)
__global__ void k_l1_tiles_final(const double *lpart, int ntiles, double npix, double m, int has_sem, float *loss) {
  __shared__ double red[3][32];
  double s[3] = {0.0, 0.0, 0.0};
  for (int t = threadIdx.x; t < ntiles; t += blockDim.x)
    for (int i = 0; i < 3; ++i) s[i] += lpart[3 * (size_t)t + i];
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s[i] += __shfl_xor_sync(0xffffffffu, s[i], o);
    if ((threadIdx.x & 31) == 0) red[i][threadIdx.x >> 5] = s[i];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t[3] = {0.0, 0.0, 0.0};
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
      for (int i = 0; i < 3; ++i) t[i] += red[i][w];
    double l = t[0] / (3.0 * npix) + t[1] / npix;
    if (has_sem) l += t[2] / (npix * m);
    *loss = (float)l;
  }
}

template <int TW, int TH, bool L1, int PPT>
static cudaError_t launch_fwd_shape(const FwdArgs &a, int grid, size_t smem, cudaStream_t s) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_render_fwd<TW, TH, L1, PPT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBudget);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  k_render_fwd<TW, TH, L1, PPT><<<grid, TW * TH / PPT, smem, s>>>(a);
  return cudaGetLastError();
}

template <bool L1, int PPT>
static cudaError_t dispatch_fwd_ppt(int tw, int th, const FwdArgs &a, int grid, size_t smem, cudaStream_t s) {
  if (tw == 16 && th == 16) return launch_fwd_shape<16, 16, L1, PPT>(a, grid, smem, s);
  if (tw == 16 && th == 8) return launch_fwd_shape<16, 8, L1, PPT>(a, grid, smem, s);
  if (tw == 8 && th == 8) return launch_fwd_shape<8, 8, L1, PPT>(a, grid, smem, s);
  if (tw == 32 && th == 8) return launch_fwd_shape<32, 8, L1, PPT>(a, grid, smem, s);
  return cudaErrorInvalidConfiguration;
}

template <bool L1>
static cudaError_t dispatch_fwd(const Layout &L, const FwdArgs &a, int grid, size_t smem, cudaStream_t s) {
  if (L.ppt == 2) return dispatch_fwd_ppt<L1, 2>(L.tile_w, L.tile_h, a, grid, smem, s);
  return dispatch_fwd_ppt<L1, 1>(L.tile_w, L.tile_h, a, grid, smem, s);
}

static FwdArgs fwd_args(const Layout &L, const WsPtrs &P, int pbuf, const gs_scene &sc) {
  FwdArgs a{};
  a.ranges = P.ranges;
  a.pvals = P.pvals[pbuf];
  a.rec = rec_ptrs(P);
  a.k = sc.k; a.m = sc.m;
  a.width = L.cam0_w; a.height = L.cam0_h;
  a.tiles_x = (L.cam0_w + L.tile_w - 1) / L.tile_w;
  a.tfinal = P.tfinal; a.nlast = P.nlast;
  a.counters = P.counters;
  return a;
}

cudaError_t launch_render_fwd(const Layout &L, const WsPtrs &P, int pbuf, const gs_scene &sc, float *rgb,
                              float *depth, float *sil, float *sem, cudaStream_t s) {
  FwdArgs a = fwd_args(L, P, pbuf, sc);
  const int tiles_y = (L.cam0_h + L.tile_h - 1) / L.tile_h;
  a.rgb_out = rgb; a.depth_out = depth; a.sil_out = sil; a.sem = sem;
  const int npix = L.tile_w * L.tile_h;  // accumulator rows: one per pixel of the tile
  chunk_classes(sc.m, npix, sc.k, sem != nullptr, &a.mchunk, &a.mstride, &a.nchunks);
  const size_t smem = batch_smem_bytes(sc.k) + (sem ? (size_t)npix * a.mstride * sizeof(float) : 0);
  const int grid = a.tiles_x * tiles_y;
  if (grid == 0) return cudaSuccess;
  return dispatch_fwd<false>(L, a, grid, smem, s);
}

cudaError_t launch_render_fwd_l1(const Layout &L, const WsPtrs &P, int pbuf, const gs_scene &sc,
                                 const float *t_rgb, const float *t_depth, const float *t_sem, float *rgb,
                                 float *depth, float *sil, float *sem, float *loss, cudaStream_t s) {
  FwdArgs a = fwd_args(L, P, pbuf, sc);
  const int tiles_y = (L.cam0_h + L.tile_h - 1) / L.tile_h;
  a.rgb_out = rgb; a.depth_out = depth; a.sil_out = sil; a.sem = sem;
  a.t_rgb = t_rgb; a.t_depth = t_depth; a.t_sem = t_sem;
  a.codes = P.codes;
  a.nwc = L.nwc;
  a.lpart = P.lpart;
  const bool acc = sem != nullptr || t_sem != nullptr;
  const int npix = L.tile_w * L.tile_h;
  chunk_classes(sc.m, npix, sc.k, acc, &a.mchunk, &a.mstride, &a.nchunks);
  const size_t smem = batch_smem_bytes(sc.k) + (acc ? (size_t)npix * a.mstride * sizeof(float) : 0);
  const int grid = a.tiles_x * tiles_y;
  if (grid == 0) return cudaSuccess;
  cudaError_t e = dispatch_fwd<true>(L, a, grid, smem, s);
  if (e != cudaSuccess) return e;
  k_l1_tiles_final<<<1, 1024, 0, s>>>(P.lpart, grid, (double)L.npix, (double)sc.m, t_sem ? 1 : 0, loss);
  return cudaGetLastError();
}

}  // namespace gs
