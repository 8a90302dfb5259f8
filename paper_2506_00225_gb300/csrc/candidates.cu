// candidates.cu -- batched candidate-view rendering for next-best-view
// scoring (Sec. 3.2).
//
// One launch chain covers every (view, tile) of all candidate views (mixed
// resolutions share one projection and one binning pass).  Per pixel it
// composites the silhouette (Eq. 1, z_i = 1), the per-Gaussian scalar
// uncertainty (Eq. 1, z_i = u_i) and the sparse semantic map (Eq. 3), then
// computes the entropy (Eq. 4) of the map clipped to [0.001, 1] and
// renormalised (Eq. 7) as H = ln Z - (sum_m p_m ln p_m) / Z, with
// Z = sum_m p_m; classes at the clip floor are counted rather than
// logged one by one.  Per-view sums of U and H and the number of pixels with
// S = 0 (Eq. 6) are reduced per CTA and added to the view's accumulators in
// double precision.  No per-pixel map is written.  The per-class logarithms
// use the hardware approximation (__logf: a few ulp on (0.001, 1]); the
// per-view sums stay within 1e-5 relative of the oracle's libm result.
//
// When the workspace holds contributor bits, two passes run (as for the
// mapping view): k_cand_blend composites U and S, records the last
// contributor and one bit per (pixel, staged Gaussian) that contributed;
// k_cand_sem walks only those bits to build the class distribution, class
// chunk by class chunk, and reduces the entropy.  Otherwise the single-pass
// k_candidates re-blends every chunk.
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
  const Counters *counters;
  int mchunk, mstride, nchunks;
  // two-pass mode
  const uint32_t *mask_off;
  uint32_t *masks;
  uint32_t mask_units;
  uint32_t *clast;
};

// View of a global tile id: last v with tile_off[v] <= tile.
__device__ __forceinline__ int view_of(const uint32_t *tile_off, int n_views, uint32_t tile) {
  int lo = 0, hi = n_views;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (tile_off[mid] <= tile) lo = mid; else hi = mid;
  }
  return lo;
}

// Per-view double sums of one float per thread (block reduction, then one
// atomic per CTA).
template <int THREADS>
__device__ __forceinline__ void add_view_sum(float v, double *dst) {
  __shared__ float red[THREADS / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane_id() == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < THREADS / 32; ++w) s += red[w];
    atomicAdd(dst, s);
  }
}

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
  if (a.counters->status & kStatusTimeout) return;  // the binning is incomplete

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
          Aacc = fmaf(ph, __logf(ph), Aacc);  // hardware log2 approximation (ph in (0.001, 1])
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

// Pass 1: U and S of Eq. 1 with the same per-pair rules as the mapping
// blend (alpha box, 1/255 skip, 1e-4 stop); writes the last contributor and
// the contributor bits of every staged batch; adds sum U and N_S per view.
template <int TW, int TH>
__global__ void __launch_bounds__(TW *TH) k_cand_blend(CandArgs a) {
  using FP = Footprint<TW, TH>;
  constexpr int THREADS = FP::kThreads;
  constexpr int WARPS = FP::kWarps;
  constexpr int NPIX = FP::kPix;
  extern __shared__ float4 smem4[];
  BatchSmem bs = batch_smem(smem4, 0);
  __shared__ uint32_t lmask[kBatch * WARPS];  // per staged Gaussian: its lanes of each warp
  if (a.counters->status & kStatusTimeout) return;
  const uint32_t tile = blockIdx.x;
  const int v = view_of(a.tile_off, a.n_views, tile);
  const DevCam &c = a.cams[v];
  const uint32_t local = tile - c.tile_off;
  const int ox = (int)(local % (uint32_t)c.tiles_x) * TW, oy = (int)(local / (uint32_t)c.tiles_x) * TH;
  const uint2 rg = a.ranges[tile];
  const int lx = FP::lx(), ly = FP::ly(0);
  const int px = ox + lx, py = oy + ly, lp = ly * TW + lx;
  const bool inside = px < c.width && py < c.height;
  const float fpx = (float)px + 0.5f, fpy = (float)py + 0.5f;
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
  const uint32_t unit0 = a.mask_off[tile];
  const bool use_unc = a.unc != nullptr;

  float T = 1.f, U = 0.f;
  uint32_t last = 0;
  bool done = !inside;
  uint32_t bi = 0;
  for (uint32_t b = rg.x; b < rg.y; b += kBatch, ++bi) {
    const int n = (int)min((uint32_t)kBatch, rg.y - b);
    __syncthreads();
    for (int t = threadIdx.x; t < n; t += THREADS) {
      const uint32_t r = a.pvals[b + t];
      stage_record<TW, TH>(a.rec, r, t, 0, ox, oy, bs, false, use_unc);
      lane_masks<TW, TH>(__ldg(a.rec.box + r), ox, oy, lmask + t * WARPS);
    }
    __syncthreads();
    uint32_t bits[2] = {0u, 0u};
    if (!__all_sync(0xffffffffu, done)) {
      for (int base = 0; base < n; base += 32) {
        const int jj = base + (int)lane;
        uint32_t vis = __ballot_sync(0xffffffffu, jj < n && lmask[jj * WARPS + warp] != 0u);
        while (vis) {
          const int bit = __ffs(vis) - 1;
          vis &= vis - 1;
          const int j = base + bit;
          if (done || !((lmask[j * WARPS + warp] >> lane) & 1u)) continue;
          float alpha, G, araw, dx, dy;
          if (!gauss_alpha(bs.uv[j], bs.co[j], fpx, fpy, alpha, G, araw, dx, dy)) continue;
          const float Tn = __fmul_rn(T, __fsub_rn(1.f, alpha));
          if (Tn < kTStop) { done = true; continue; }
          const float w = __fmul_rn(alpha, T);
          U = fmaf(w, bs.cd[j].x, U);
          T = Tn;
          bits[base >> 5] |= 1u << bit;
        }
      }
    }
    if (bits[1]) last = b - rg.x + 32 + (32 - __clz(bits[1]));
    else if (bits[0]) last = b - rg.x + (32 - __clz(bits[0]));
    if (unit0 + bi < a.mask_units) {
      uint32_t *mw = a.masks + (size_t)(unit0 + bi) * 2 * NPIX;
      mw[lp] = bits[0];
      mw[NPIX + lp] = bits[1];
    }
    if (__syncthreads_count(done) == THREADS) break;
  }
  a.clast[(size_t)tile * NPIX + lp] = last;
  add_view_sum<THREADS>(inside && use_unc ? U : 0.f, a.out + 3 * v);
  add_view_sum<THREADS>(inside && T == 1.f ? 1.f : 0.f, a.out + 3 * v + 2);
}

// Pass 2: the class distribution from the contributor bits (warp-uniform
// walk over the union of the warp's bits, alpha recomputed bit-identically,
// k adds per contributor into per-thread rows), one class chunk at a time,
// and the clipped, renormalised entropy per pixel.
template <int TW, int TH, int K>
__global__ void __launch_bounds__(TW *TH, 2) k_cand_sem(CandArgs a) {
  using FP = Footprint<TW, TH>;
  constexpr int THREADS = FP::kThreads;
  constexpr int NPIX = FP::kPix;
  extern __shared__ float4 smem4[];
  const int k = a.k;
  char *sbase = reinterpret_cast<char *>(smem4);
  const size_t bbytes = sem_batch_bytes(k);
  float *sP = reinterpret_cast<float *>(sbase + 2 * bbytes);
  __shared__ uint32_t s_maxlast;
  if (a.counters->status & kStatusTimeout) return;

  const uint32_t tile = blockIdx.x;
  const int v = view_of(a.tile_off, a.n_views, tile);
  const DevCam &c = a.cams[v];
  const uint32_t local = tile - c.tile_off;
  const int ox = (int)(local % (uint32_t)c.tiles_x) * TW, oy = (int)(local / (uint32_t)c.tiles_x) * TH;
  const uint2 rg = a.ranges[tile];
  const int lx = FP::lx(), ly = FP::ly(0);
  const int px = ox + lx, py = oy + ly, lp = ly * TW + lx;
  const bool inside = px < c.width && py < c.height;
  const float fpx = (float)px + 0.5f, fpy = (float)py + 0.5f;
  float *myP = sP + threadIdx.x * a.mstride;
  const uint32_t unit0 = a.mask_off[tile];

  const uint32_t last = a.clast[(size_t)tile * NPIX + lp];
  if (threadIdx.x == 0) s_maxlast = 0;
  __syncthreads();
  if (last) atomicMax(&s_maxlast, last);
  __syncthreads();
  const int nbatch = (int)((s_maxlast + kBatch - 1) / kBatch);

  auto buf_uv = [&](int q) { return reinterpret_cast<float2 *>(sbase + q * bbytes); };
  auto buf_co = [&](int q) { return reinterpret_cast<float4 *>(sbase + q * bbytes + kBatch * 8); };
  auto buf_sem = [&](int q) { return reinterpret_cast<int2 *>(sbase + q * bbytes + kBatch * 32); };
  auto batch_n = [&](int bi) { return (int)min((uint32_t)kBatch, rg.y - (rg.x + (uint32_t)bi * kBatch)); };
  auto issue = [&](int bi, uint32_t r) {
    const int q = bi & 1, t = threadIdx.x;
    cp_async8(buf_uv(q) + t, a.rec.uv + r);
    cp_async16(buf_co(q) + t, a.rec.co + r);
    const int2 *src = a.rec.sem + (size_t)r * k;
    for (int l = 0; l < k; ++l) cp_async8(buf_sem(q) + t * k + l, src + l);
  };

  float Z = 0.f, Aacc = 0.f;
  uint32_t nfloor = 0;
  for (int ch = 0; ch < a.nchunks; ++ch) {
    const int c_lo = ch * a.mchunk, c_hi = min(a.m, c_lo + a.mchunk), mc = c_hi - c_lo;
    for (int q = 0; q < mc; ++q) myP[q] = 0.f;
    float T = 1.f;
    const int t = threadIdx.x;
    if (nbatch > 0 && t < batch_n(0)) issue(0, a.pvals[rg.x + t]);
    cp_async_commit();
    uint32_t pv = (nbatch > 1 && t < batch_n(1)) ? a.pvals[rg.x + kBatch + t] : 0u;
    cp_async_wait_all();
    __syncthreads();
    for (int bi = 0; bi < nbatch; ++bi) {
      if (bi + 1 < nbatch && t < batch_n(bi + 1)) issue(bi + 1, pv);
      cp_async_commit();
      if (bi + 2 < nbatch && t < batch_n(bi + 2)) pv = a.pvals[rg.x + (uint32_t)(bi + 2) * kBatch + t];
      const uint32_t b0 = (uint32_t)bi * kBatch;
      uint32_t mine[2] = {0u, 0u};
      if (b0 < last) {
        const uint32_t *mw = a.masks + (size_t)(unit0 + bi) * 2 * NPIX;
        mine[0] = mw[lp];
        mine[1] = mw[NPIX + lp];
      }
      const float2 *suv = buf_uv(bi & 1);
      const float4 *sco = buf_co(bi & 1);
      const int2 *ssem = buf_sem(bi & 1);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        uint32_t un = __reduce_or_sync(0xffffffffu, mine[h]);
        while (un) {
          const int jb = __ffs(un) - 1;
          un &= un - 1;
          const int j = h * 32 + jb;
          float alpha = 0.f, G, araw, dx, dy;
          gauss_alpha(suv[j], sco[j], fpx, fpy, alpha, G, araw, dx, dy);
          const bool on = (mine[h] >> jb) & 1u;
          const float w = on ? __fmul_rn(alpha, T) : 0.f;
          if (on) T = __fmul_rn(T, __fsub_rn(1.f, alpha));
          scatter_classes<K>(myP, ssem + j * k, k, c_lo, mc, w);
        }
      }
      cp_async_wait_all();
      __syncthreads();
    }
    if (inside) {
      for (int q = 0; q < mc; ++q) {
        const float p = myP[q];
        if (p > kClipLo) {
          const float ph = p < 1.f ? p : 1.f;
          Z += ph;
          Aacc = fmaf(ph, __logf(ph), Aacc);  // hardware log2 approximation (ph in (0.001, 1])
        } else {
          ++nfloor;
        }
      }
    }
    __syncthreads();  // the next chunk reuses the rows
  }
  float h = 0.f;
  if (inside) {
    const float zf = kClipLo * (float)nfloor;
    Z += zf;
    Aacc = fmaf(zf, logf(kClipLo), Aacc);
    h = logf(Z) - Aacc / Z;
  }
  add_view_sum<THREADS>(h, a.out + 3 * v + 1);
}

__global__ void k_zero_doubles(double *p, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = 0.0;
}

template <int TW, int TH>
static cudaError_t launch_cand_shape(const CandArgs &a, uint32_t grid, size_t smem, cudaStream_t s) {
  {
    const cudaError_t e = ensure_smem_limit((const void *)k_candidates<TW, TH>, (int)kSmemBudget);
    if (e != cudaSuccess) return e;
  }
  k_candidates<TW, TH><<<grid, TW * TH, smem, s>>>(a);
  return cudaGetLastError();
}

template <int TW, int TH, int K>
static cudaError_t launch_cand_sem(const CandArgs &a, uint32_t grid, size_t smem, cudaStream_t s) {
  {
    const cudaError_t e = ensure_smem_limit((const void *)k_cand_sem<TW, TH, K>, (int)kSmemBudget);
    if (e != cudaSuccess) return e;
  }
  k_cand_sem<TW, TH, K><<<grid, TW * TH, smem, s>>>(a);
  return cudaGetLastError();
}

template <int TW, int TH>
static cudaError_t launch_cand_two_pass(const CandArgs &a, uint32_t grid, size_t smem_sem, cudaStream_t s) {
  k_cand_blend<TW, TH><<<grid, TW * TH, batch_smem_bytes(0), s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (a.k == 3) return launch_cand_sem<TW, TH, 3>(a, grid, smem_sem, s);
  if (a.k == 8) return launch_cand_sem<TW, TH, 8>(a, grid, smem_sem, s);
  return launch_cand_sem<TW, TH, 0>(a, grid, smem_sem, s);
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
  a.counters = P.counters;
  const int threads = L.tile_w * L.tile_h;
  const uint32_t grid = (uint32_t)L.total_tiles;
  if (grid == 0) return cudaSuccess;
  if (L.mask_units > 0) {
    // two passes: batch offsets of every tile, blend + bits, classes + entropy
    a.mask_off = P.mask_off;
    a.masks = P.masks;
    a.mask_units = (uint32_t)L.mask_units;
    a.clast = P.clast;
    e = launch_tile_batch_offsets(P.ranges, grid, P.mask_off, P.counters, s);
    if (e != cudaSuccess) return e;
    const size_t fixed = 2 * sem_batch_bytes(sc.k), base = batch_smem_bytes(sc.k);
    chunk_classes(sc.m, threads, sc.k, true, &a.mchunk, &a.mstride, &a.nchunks, fixed > base ? fixed - base : 0);
    const size_t smem = fixed + (size_t)threads * a.mstride * sizeof(float);
    if (L.tile_w == 16 && L.tile_h == 16) return launch_cand_two_pass<16, 16>(a, grid, smem, s);
    if (L.tile_w == 16 && L.tile_h == 8) return launch_cand_two_pass<16, 8>(a, grid, smem, s);
    if (L.tile_w == 8 && L.tile_h == 8) return launch_cand_two_pass<8, 8>(a, grid, smem, s);
    if (L.tile_w == 32 && L.tile_h == 8) return launch_cand_two_pass<32, 8>(a, grid, smem, s);
    return cudaErrorInvalidConfiguration;
  }
  chunk_classes(sc.m, threads, sc.k, true, &a.mchunk, &a.mstride, &a.nchunks);
  const size_t smem = batch_smem_bytes(sc.k) + (size_t)threads * a.mstride * sizeof(float);
  if (L.tile_w == 16 && L.tile_h == 16) return launch_cand_shape<16, 16>(a, grid, smem, s);
  if (L.tile_w == 16 && L.tile_h == 8) return launch_cand_shape<16, 8>(a, grid, smem, s);
  if (L.tile_w == 8 && L.tile_h == 8) return launch_cand_shape<8, 8>(a, grid, smem, s);
  if (L.tile_w == 32 && L.tile_h == 8) return launch_cand_shape<32, 8>(a, grid, smem, s);
  return cudaErrorInvalidConfiguration;
}

}  // namespace gs
