// render_fwd.cu -- forward tile blend: Eq. 1 (colour, depth, silhouette) and
// Eq. 3 (sparse top-k semantics), supplement "Sparse Rendering".
//
// One CTA per screen tile, one thread per pixel.  The tile's depth-sorted
// pair range is walked in batches staged in shared memory; each thread
// composites the Gaussians whose pixel rectangle holds its pixel, front to
// back, and stops before the Gaussian that would take the transmittance
// below 1e-4.  The CTA leaves the loop when every pixel is done
// (__syncthreads_count).  Semantic probabilities are scattered into a
// per-pixel M-class accumulator in shared memory (k adds per contributor
// instead of M, the point of the sparse representation), then written out
// with coalesced stores.  When M does not fit the shared-memory budget the
// classes are processed in chunks of 32-class multiples, recompositing per
// chunk.
//
// Fused mean-L1 mode (L1 = true): the rendered colour, depth and semantic
// distribution are compared with the targets inside the tile; the kernel
// keeps per-tile sums of |rendered - target| and, per value, two bits
// (nonzero, negative) of the sign of the difference for the adjoint.  The
// semantic map itself need not be written.
#include "gs_internal.cuh"
#include "render_common.cuh"

namespace gs {

template <int TW, int TH, bool L1>
__global__ void __launch_bounds__(TW *TH) k_render_fwd(FwdArgs a) {
  constexpr int THREADS = TW * TH;
  constexpr int WARPS = THREADS / 32;
  extern __shared__ float4 smem4[];
  BatchSmem bs = batch_smem(smem4, a.k);
  float *sP = bs.tail;
  __shared__ float red[3][WARPS];

  const int tile = blockIdx.x;
  const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
  const uint2 rg = a.ranges[tile];
  const int lx = threadIdx.x % TW, ly = threadIdx.x / TW;
  const int px = tx * TW + lx, py = ty * TH + ly;
  const bool inside = px < a.width && py < a.height;
  const float fpx = (float)px + 0.5f, fpy = (float)py + 0.5f;
  const bool acc_sem = a.sem != nullptr || (L1 && a.t_sem != nullptr);
  float *myP = sP + threadIdx.x * a.mstride;
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
  const int cw = code_words(a.nwc);
  float l1_sem = 0.f;

  float T = 1.f, cr = 0.f, cg = 0.f, cb = 0.f, cd = 0.f;
  uint32_t last = 0, ncontrib = 0;
  for (int c = 0; c < a.nchunks; ++c) {
    const int c_lo = c * a.mchunk, c_hi = min(a.m, c_lo + a.mchunk);
    const int mc = c_hi - c_lo;
    if (acc_sem)
      for (int i = 0; i < mc; ++i) myP[i] = 0.f;
    T = 1.f; cr = cg = cb = cd = 0.f; last = 0; ncontrib = 0;
    bool done = !inside;
    for (uint32_t b = rg.x; b < rg.y; b += kBatch) {
      const int n = (int)min((uint32_t)kBatch, rg.y - b);
      __syncthreads();
      if ((int)threadIdx.x < n) load_batch_entry(a.rec, a.pvals[b + threadIdx.x], threadIdx.x, a.k, bs, a.rgb,
                                                 a.sem_ids, a.sem_w, nullptr);
      __syncthreads();
      if (!done) {
        for (int j = 0; j < n; ++j) {
          const int2 rr = bs.rect[j];
          if (!rect_holds(rr, px, py)) continue;
          const float2 uv = bs.uv[j];
          const float4 co = bs.co[j];
          float alpha, G, araw, dx, dy;
          if (!gauss_alpha(uv, co, fpx, fpy, alpha, G, araw, dx, dy)) continue;
          const float Tn = __fmul_rn(T, __fsub_rn(1.f, alpha));
          if (Tn < kTStop) { done = true; break; }
          const float w = __fmul_rn(alpha, T);
          const float4 cdp = bs.cd[j];
          cr = fmaf(w, cdp.x, cr); cg = fmaf(w, cdp.y, cg); cb = fmaf(w, cdp.z, cb); cd = fmaf(w, cdp.w, cd);
          if (acc_sem) {
            const int *sid = bs.sid + j * a.k;
            const float *sw = bs.sw + j * a.k;
            for (int l = 0; l < a.k; ++l) {
              const int id = sid[l] - c_lo;
              if ((unsigned)id < (unsigned)mc) myP[id] = fmaf(w, sw[l], myP[id]);
            }
          }
          T = Tn;
          last = b - rg.x + j + 1;
          ++ncontrib;
        }
      }
      if (__syncthreads_count(done) == THREADS) break;
    }
    if (acc_sem) {
      __syncthreads();
      const int x0 = tx * TW;
      const int vw = min(TW, a.width - x0);
      if (a.sem) {
        for (int r = 0; r < TH; ++r) {
          const int y = ty * TH + r;
          if (y >= a.height) break;
          float *dst = a.sem + ((size_t)y * a.width + x0) * a.m + c_lo;
          const float *src = sP + (r * TW) * a.mstride;
          for (int e = threadIdx.x; e < vw * mc; e += THREADS) {
            const int p = e / mc, cl = e - p * mc;
            dst[(size_t)p * a.m + cl] = src[p * a.mstride + cl];
          }
        }
      }
      if (L1 && a.t_sem) {
        // one warp per (pixel, 32-class word): coalesced target reads, ballots
        // assemble the sign words
        const int w_lo = c_lo >> 5, nwt = (c_hi + 31) / 32 - w_lo;
        for (int task = warp; task < THREADS * nwt; task += WARPS) {
          const int p = task / nwt, wd = w_lo + task % nwt;
          const int qx = x0 + p % TW, qy = ty * TH + p / TW;
          if (qx >= a.width || qy >= a.height) continue;
          const size_t pix = (size_t)qy * a.width + qx;
          const int mcl = wd * 32 + (int)lane;
          const bool valid = mcl < c_hi;
          float d = 0.f;
          if (valid) d = sP[p * a.mstride + (mcl - c_lo)] - __ldcs(a.t_sem + pix * a.m + mcl);
          const uint32_t nz = __ballot_sync(0xffffffffu, d != 0.f);
          const uint32_t ng = __ballot_sync(0xffffffffu, d < 0.f);
          l1_sem += fabsf(d);
          if (lane == 0) {
            uint32_t *cp = a.codes + pix * cw;
            cp[1 + wd] = nz;
            cp[1 + a.nwc + 1 + wd] = ng;
          }
        }
      }
      __syncthreads();  // the next chunk reuses the accumulator rows
    }
  }
  {
    // diagnostics: total contributions (one atomic per CTA)
    uint32_t nc = ncontrib;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nc += __shfl_xor_sync(0xffffffffu, nc, o);
    if (lane == 0 && nc) atomicAdd(&a.counters->n_contrib, nc);
  }
  float l1_rgb = 0.f, l1_d = 0.f;
  if (inside) {
    const size_t pix = (size_t)py * a.width + px;
    if (a.rgb_out) { a.rgb_out[3 * pix] = cr; a.rgb_out[3 * pix + 1] = cg; a.rgb_out[3 * pix + 2] = cb; }
    if (a.depth_out) a.depth_out[pix] = cd;
    if (a.sil_out) a.sil_out[pix] = 1.f - T;
    a.tfinal[pix] = T;
    a.nlast[pix] = last;
    if (L1) {
      const float d0 = cr - a.t_rgb[3 * pix], d1 = cg - a.t_rgb[3 * pix + 1], d2 = cb - a.t_rgb[3 * pix + 2];
      const float d3 = cd - a.t_depth[pix];
      const uint32_t nz = (d0 != 0.f ? 1u : 0u) | (d1 != 0.f ? 2u : 0u) | (d2 != 0.f ? 4u : 0u) | (d3 != 0.f ? 8u : 0u);
      const uint32_t ng = (d0 < 0.f ? 1u : 0u) | (d1 < 0.f ? 2u : 0u) | (d2 < 0.f ? 4u : 0u) | (d3 < 0.f ? 8u : 0u);
      uint32_t *cp = a.codes + pix * cw;
      cp[0] = nz;
      cp[1 + a.nwc] = ng;
      if (!a.t_sem)
        for (int wd = 0; wd < a.nwc; ++wd) { cp[1 + wd] = 0u; cp[2 + a.nwc + wd] = 0u; }
      l1_rgb = fabsf(d0) + fabsf(d1) + fabsf(d2);
      l1_d = fabsf(d3);
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

template <int TW, int TH, bool L1>
static cudaError_t launch_fwd_shape(const FwdArgs &a, int grid, size_t smem, cudaStream_t s) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_render_fwd<TW, TH, L1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kSmemBudget);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  k_render_fwd<TW, TH, L1><<<grid, TW * TH, smem, s>>>(a);
  return cudaGetLastError();
}

template <bool L1>
static cudaError_t dispatch_fwd(int tw, int th, const FwdArgs &a, int grid, size_t smem, cudaStream_t s) {
  if (tw == 16 && th == 16) return launch_fwd_shape<16, 16, L1>(a, grid, smem, s);
  if (tw == 16 && th == 8) return launch_fwd_shape<16, 8, L1>(a, grid, smem, s);
  if (tw == 8 && th == 8) return launch_fwd_shape<8, 8, L1>(a, grid, smem, s);
  if (tw == 32 && th == 8) return launch_fwd_shape<32, 8, L1>(a, grid, smem, s);
  return cudaErrorInvalidConfiguration;
}

static FwdArgs fwd_args(const Layout &L, const WsPtrs &P, int pbuf, const gs_scene &sc) {
  FwdArgs a{};
  a.ranges = P.ranges;
  a.pvals = P.pvals[pbuf];
  a.rec = rec_ptrs(P);
  a.rgb = sc.rgb; a.sem_ids = sc.sem_ids; a.sem_w = sc.sem_w;
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
  const int threads = L.tile_w * L.tile_h;
  chunk_classes(sc.m, threads, sc.k, sem != nullptr, &a.mchunk, &a.mstride, &a.nchunks);
  const size_t smem = batch_smem_bytes(sc.k) + (sem ? (size_t)threads * a.mstride * sizeof(float) : 0);
  const int grid = a.tiles_x * tiles_y;
  if (grid == 0) return cudaSuccess;
  return dispatch_fwd<false>(L.tile_w, L.tile_h, a, grid, smem, s);
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
  const int threads = L.tile_w * L.tile_h;
  chunk_classes(sc.m, threads, sc.k, acc, &a.mchunk, &a.mstride, &a.nchunks);
  const size_t smem = batch_smem_bytes(sc.k) + (acc ? (size_t)threads * a.mstride * sizeof(float) : 0);
  const int grid = a.tiles_x * tiles_y;
  if (grid == 0) return cudaSuccess;
  cudaError_t e = dispatch_fwd<true>(L.tile_w, L.tile_h, a, grid, smem, s);
  if (e != cudaSuccess) return e;
  k_l1_tiles_final<<<1, 1024, 0, s>>>(P.lpart, grid, (double)L.npix, (double)sc.m, t_sem ? 1 : 0, loss);
  return cudaGetLastError();
}

}  // namespace gs
