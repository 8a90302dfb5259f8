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
// chunk by class chunk, and reduces the entropy.  Both are persistent: their
// CTAs take (view, tile) work items by ticket, in tile order.
// The bits are bounded: the views are rendered in waves whose bits fit the
// workspace (planned on the device from the tile pair counts), and a tile
// whose bits do not fit re-tests its pairs in the class pass.  The staged
// batch size B (32, 64 or 128 Gaussians) is a template parameter chosen by
// the autotuner.  Without bits (recompute_bwd) the single-pass k_candidates
// re-blends every class chunk.
#include "gs_internal.cuh"
#include "render_common.cuh"

namespace gs {

// Candidate waves in the workspace: [waves][5] = first tile, end tile,
// first bit unit, ticket of the blend pass, ticket of the class pass.
struct CandPlan {
  uint32_t *wave;
  int waves;
};

inline CandPlan cand_plan(const Layout &L, const WsPtrs &P) { return CandPlan{P.cand_plan, L.cand_waves}; }

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
  uint32_t cap_units;  // bit capacity of a wave in (tile, batch) units
  uint32_t *clast;
  CandPlan plan;
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

// add_view_sum over the pixels of a tile as the one-pixel-per-thread
// kernels add them (same 32-pixel groups, same butterfly, same order of the
// group sums), whatever the thread mapping of the caller: px[p] is the
// value of tile pixel p (raster order).  Every thread of the CTA calls it.
template <int TW, int TH, int THREADS>
__device__ __forceinline__ void add_view_sum_pixels(const float *px, double *dst) {
  using F1 = Footprint<TW, TH, 1>;
  constexpr int G = F1::kWarps;  // 32-pixel groups
  __shared__ float red[G];
  __syncthreads();  // px is complete
  for (int w = threadIdx.x >> 5; w < G; w += THREADS / 32) {
    const int l = (int)lane_id();
    const int lx = (w % F1::kWX) * 8 + (l & 7), ly = (w / F1::kWX) * 4 + (l >> 3);
    float v = px[ly * TW + lx];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (l == 0) red[w] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < G; ++w) s += red[w];
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

// Next tile of a persistent candidate pass: the CTA takes a ticket of the
// wave's tile range (tile order: a view's tiles run together and share its
// records in L2); false when the wave is exhausted.
__device__ __forceinline__ bool next_tile(const CandPlan &p, int wave, int which, uint32_t *s_item,
                                          uint32_t &tile, uint32_t &unit_base) {
  __syncthreads();  // the previous tile's shared memory is no longer read
  if (threadIdx.x == 0) *s_item = atomicAdd(p.wave + 5 * wave + 3 + which, 1u);
  __syncthreads();
  tile = p.wave[5 * wave] + *s_item;
  if (tile >= p.wave[5 * wave + 1]) return false;
  unit_base = p.wave[5 * wave + 2];
  return true;
}

// Pass 1: U and S of Eq. 1 with the same per-pair rules as the mapping
// blend (alpha box, 1/255 skip, 1e-4 stop); writes the last contributor and
// the contributor bits of every staged batch of B pairs (when the tile's
// bits fit the wave's capacity); adds sum U and N_S per view.  Each warp
// works through the tile's pairs on its own, 32 at a time: a lane per pair
// tests the pair's alpha box against the warp's 8 x 4 block, the pairs
// that reach it are staged (packed) in the warp's shared memory and blended
// in order.  A warp stops at a batch boundary once all its pixels are done,
// so every batch a pixel can still read in pass 2 has its bits written.
// Shared memory of one warp of the candidate blend: 32 staging slots (conic
// + opacity, uncertainty, mean, and per row group the lanes the pair reaches).
__host__ __device__ inline size_t cand_blend_warp_bytes(int ppt) { return 32 * (16 + 16 + 8 + 4 * (size_t)ppt); }
constexpr int kCandBlendPpt = 2;  // pixels per thread of the candidate blend

// PPT pixels per thread, one column, rows 4 apart: they share every staged
// load and the x offset of every Gaussian (as in the mapping blend pass).
template <int TW, int TH, int B, int PPT>
__global__ void __launch_bounds__(TW *TH / PPT) k_cand_blend(CandArgs a, int wave) {
  using FP = Footprint<TW, TH, PPT>;
  constexpr int THREADS = FP::kThreads;
  constexpr int NPIX = FP::kPix;
  constexpr int NW = B / 32;  // contributor words per pixel and batch
  extern __shared__ float4 smem4[];
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
  char *wb = reinterpret_cast<char *>(smem4) + warp * cand_blend_warp_bytes(PPT);
  float4 *w_co = reinterpret_cast<float4 *>(wb);
  float4 *w_cd = w_co + 32;  // uncertainty in .x
  float2 *w_uv = reinterpret_cast<float2 *>(w_co + 64);
  uint32_t *w_lm = reinterpret_cast<uint32_t *>(w_uv + 32);  // [row group][slot]: lanes each staged pair reaches
  __shared__ uint32_t s_item;
  __shared__ float s_px[2][NPIX];  // per-pixel uncertainty sum and empty flag of the current tile
  if (a.counters->status & kStatusTimeout) return;
  const int lx = FP::lx();
  const bool use_unc = a.unc != nullptr;
  uint32_t tile, unit_base;
  while (next_tile(a.plan, wave, 0, &s_item, tile, unit_base)) {
    const int v = view_of(a.tile_off, a.n_views, tile);
    const DevCam &c = a.cams[v];
    const uint32_t local = tile - c.tile_off;
    const int ox = (int)(local % (uint32_t)c.tiles_x) * TW, oy = (int)(local / (uint32_t)c.tiles_x) * TH;
    const int bx0 = ox + (int)(warp % FP::kWX) * 8, by0 = oy + (int)(warp / FP::kWX) * FP::kBH;  // the warp's block
    const uint2 rg = a.ranges[tile];
    const int px = ox + lx;
    const float fpx = (float)px + 0.5f;
    const uint32_t unit0 = a.mask_off[tile] - unit_base;
    const bool store = unit0 + (rg.y - rg.x + B - 1) / B <= a.cap_units;

    int lp[PPT];
    float fpy[PPT], T[PPT], U[PPT];
    uint32_t last[PPT];
    bool inside[PPT], done[PPT];
#pragma unroll
    for (int i = 0; i < PPT; ++i) {
      const int ly = FP::ly(i);
      lp[i] = ly * TW + lx;
      fpy[i] = (float)(oy + ly) + 0.5f;
      inside[i] = px < c.width && oy + ly < c.height;
      done[i] = !inside[i];
      T[i] = 1.f; U[i] = 0.f;
      last[i] = 0;
    }
    auto all_done = [&]() {
      bool d = true;
#pragma unroll
      for (int i = 0; i < PPT; ++i) d = d && done[i];
      return d;
    };
    // groups up to the end of the last batch: the empty groups of a partial
    // batch still write their (zero) bits, which pass 2 reads
    const uint32_t gend = rg.x + (rg.y - rg.x + B - 1) / B * B;
    for (uint32_t g0 = rg.x; g0 < gend; g0 += 32) {
      const uint32_t rel = g0 - rg.x, bi = rel / B, h = (rel % B) / 32;
      const int n = g0 < rg.y ? (int)min(32u, rg.y - g0) : 0;
      // the group's pairs that reach the warp's block, per row group
      uint32_t r = 0u, lm[PPT];
      bool reach = false;
#pragma unroll
      for (int i = 0; i < PPT; ++i) lm[i] = 0u;
      if ((int)lane < n) {
        r = a.pvals[g0 + lane];
        const short4 bx = __ldg(a.rec.box + r);
#pragma unroll
        for (int i = 0; i < PPT; ++i) {
          lm[i] = block_lane_mask(bx, bx0, by0 + 4 * i);
          reach = reach || lm[i] != 0u;
        }
      }
      const uint32_t vis = __ballot_sync(0xffffffffu, reach);
      uint32_t bits[PPT];
#pragma unroll
      for (int i = 0; i < PPT; ++i) bits[i] = 0u;
      if (vis && !__all_sync(0xffffffffu, all_done())) {
        __syncwarp();  // the previous group's slots are no longer read
        if (reach) {
          const int slot = __popc(vis & lanemask_lt());
          w_co[slot] = __ldg(a.rec.co + r);
          w_uv[slot] = __ldg(a.rec.uv + r);
          float4 cd = __ldg(a.rec.cd + r);
          if (use_unc) cd.x = __ldg(a.rec.unc + r);
          w_cd[slot] = cd;
#pragma unroll
          for (int i = 0; i < PPT; ++i) w_lm[i * 32 + slot] = lm[i];
        }
        __syncwarp();
        uint32_t rem = vis;
        int slot = 0;
        while (rem) {
          const int bit = __ffs(rem) - 1;
          rem &= rem - 1;
          const int sl = slot++;
          const float2 uv = w_uv[sl];
          const float4 co = w_co[sl];
#pragma unroll
          for (int i = 0; i < PPT; ++i) {
            if (done[i] || !((w_lm[i * 32 + sl] >> lane) & 1u)) continue;
            float alpha, G, araw, dx, dy;
            if (!gauss_alpha(uv, co, fpx, fpy[i], alpha, G, araw, dx, dy)) continue;
            const float Tn = __fmul_rn(T[i], __fsub_rn(1.f, alpha));
            if (Tn < kTStop) { done[i] = true; continue; }
            const float w = __fmul_rn(alpha, T[i]);
            U[i] = fmaf(w, w_cd[sl].x, U[i]);
            T[i] = Tn;
            bits[i] |= 1u << bit;
          }
        }
      }
#pragma unroll
      for (int i = 0; i < PPT; ++i) {
        if (bits[i]) last[i] = rel + (32 - __clz(bits[i]));
        if (store) a.masks[((size_t)(unit0 + bi) * NW + h) * NPIX + lp[i]] = bits[i];
      }
      // stop at a batch boundary once every pixel of the warp is done
      if (h == NW - 1 && __all_sync(0xffffffffu, all_done())) break;
    }
#pragma unroll
    for (int i = 0; i < PPT; ++i) {
      a.clast[(size_t)tile * NPIX + lp[i]] = last[i];
      s_px[0][lp[i]] = inside[i] && use_unc ? U[i] : 0.f;
      s_px[1][lp[i]] = inside[i] && T[i] == 1.f ? 1.f : 0.f;
    }
    add_view_sum_pixels<TW, TH, THREADS>(s_px[0], a.out + 3 * v);
    add_view_sum_pixels<TW, TH, THREADS>(s_px[1], a.out + 3 * v + 2);
  }
}

// Pass 2: the class distribution from the contributor bits (warp-uniform
// walk over the union of the warp's bits, alpha recomputed bit-identically,
// k adds per contributor into per-thread rows), one class chunk at a time,
// and the clipped, renormalised entropy per pixel.  A tile without stored
// bits re-tests its pairs up to each pixel's last contributor (alpha box,
// alpha), which selects the same contributors.
__host__ __device__ inline size_t cand_sem_batch_bytes(int k, int B) { return (size_t)B * (8 + 16 + 8 + 8 * k); }

template <int TW, int TH, int K, int B>
__global__ void __launch_bounds__(TW *TH, 2) k_cand_sem(CandArgs a, int wave) {
  using FP = Footprint<TW, TH>;
  constexpr int THREADS = FP::kThreads;
  constexpr int NPIX = FP::kPix;
  constexpr int NW = B / 32;
  extern __shared__ float4 smem4[];
  const int k = a.k;
  char *sbase = reinterpret_cast<char *>(smem4);
  const size_t bbytes = cand_sem_batch_bytes(k, B);
  float *sP = reinterpret_cast<float *>(sbase + 2 * bbytes);
  __shared__ uint32_t s_maxlast, s_item;
  if (a.counters->status & kStatusTimeout) return;
  const int lx = FP::lx(), ly = FP::ly(0), lp = ly * TW + lx;
  float *myP = sP + threadIdx.x * a.mstride;

  auto buf_co = [&](int q) { return reinterpret_cast<float4 *>(sbase + q * bbytes); };
  auto buf_uv = [&](int q) { return reinterpret_cast<float2 *>(sbase + q * bbytes + B * 16); };
  auto buf_box = [&](int q) { return reinterpret_cast<short4 *>(sbase + q * bbytes + B * 24); };
  auto buf_sem = [&](int q) { return reinterpret_cast<int2 *>(sbase + q * bbytes + B * 32); };

  uint32_t tile, unit_base;
  while (next_tile(a.plan, wave, 1, &s_item, tile, unit_base)) {
    const int v = view_of(a.tile_off, a.n_views, tile);
    const DevCam &c = a.cams[v];
    const uint32_t local = tile - c.tile_off;
    const int ox = (int)(local % (uint32_t)c.tiles_x) * TW, oy = (int)(local / (uint32_t)c.tiles_x) * TH;
    const uint2 rg = a.ranges[tile];
    const int px = ox + lx, py = oy + ly;
    const bool inside = px < c.width && py < c.height;
    const float fpx = (float)px + 0.5f, fpy = (float)py + 0.5f;
    const uint32_t unit0 = a.mask_off[tile] - unit_base;
    const bool stored = unit0 + (rg.y - rg.x + B - 1) / B <= a.cap_units;

    const uint32_t last = a.clast[(size_t)tile * NPIX + lp];
    if (threadIdx.x == 0) s_maxlast = 0;
    __syncthreads();
    if (last) atomicMax(&s_maxlast, last);
    __syncthreads();
    const int nbatch = (int)((s_maxlast + B - 1) / B);
    auto batch_n = [&](int bi) { return (int)min((uint32_t)B, rg.y - (rg.x + (uint32_t)bi * B)); };
    // thread t stages slots t, t + THREADS, ... (PER of them) of a batch
    constexpr int PER = (B + THREADS - 1) / THREADS;
    auto issue = [&](int bi, const uint32_t (&r)[PER]) {
      const int q = bi & 1;
#pragma unroll
      for (int u = 0; u < PER; ++u) {
        const int t = threadIdx.x + u * THREADS;
        if (t >= batch_n(bi)) break;
        cp_async16(buf_co(q) + t, a.rec.co + r[u]);
        cp_async8(buf_uv(q) + t, a.rec.uv + r[u]);
        if (!stored) cp_async8(buf_box(q) + t, a.rec.box + r[u]);
        const int2 *src = a.rec.sem + (size_t)r[u] * k;
        for (int l = 0; l < k; ++l) cp_async8(buf_sem(q) + l * B + t, src + l);  // entry-major
      }
    };
    // repeated-id marks of this thread's slots of batch bi, once they landed
    auto mark = [&](int bi) {
      if constexpr (K >= 4) {
#pragma unroll
        for (int u = 0; u < PER; ++u) {
          const int t = threadIdx.x + u * THREADS;
          if (bi >= nbatch || t >= batch_n(bi)) break;
          mark_repeated_ids<K>(buf_sem(bi & 1) + t, B);
        }
      }
    };
    // pair indices of batch bi for this thread's slots
    auto fetch = [&](int bi, uint32_t (&r)[PER]) {
#pragma unroll
      for (int u = 0; u < PER; ++u) {
        const int t = threadIdx.x + u * THREADS;
        r[u] = (bi < nbatch && t < batch_n(bi)) ? a.pvals[rg.x + (uint32_t)bi * B + t] : 0u;
      }
    };

    float Z = 0.f, Aacc = 0.f;
    uint32_t nfloor = 0;
    for (int ch = 0; ch < a.nchunks; ++ch) {
      const int c_lo = ch * a.mchunk, c_hi = min(a.m, c_lo + a.mchunk), mc = c_hi - c_lo;
      for (int q = 0; q < mc; ++q) myP[q] = 0.f;
      float T = 1.f;
      uint32_t pv[PER];
      fetch(0, pv);
      if (nbatch > 0) issue(0, pv);
      cp_async_commit();
      fetch(1, pv);
      // contributor words of the next batch, loaded one batch ahead
      uint32_t mnext[NW];
      auto load_bits = [&](int bi, uint32_t (&m)[NW]) {
#pragma unroll
        for (int h = 0; h < NW; ++h) m[h] = 0u;
        if (stored && bi < nbatch && (uint32_t)bi * B < last) {
          const uint32_t *mw = a.masks + (size_t)(unit0 + bi) * NW * NPIX;
#pragma unroll
          for (int h = 0; h < NW; ++h) m[h] = mw[h * NPIX + lp];
        }
      };
      load_bits(0, mnext);
      cp_async_wait_all();
      mark(0);
      __syncthreads();
      for (int bi = 0; bi < nbatch; ++bi) {
        if (bi + 1 < nbatch) issue(bi + 1, pv);
        cp_async_commit();
        fetch(bi + 2, pv);
        const uint32_t b0 = (uint32_t)bi * B;
        uint32_t mine[NW];
#pragma unroll
        for (int h = 0; h < NW; ++h) mine[h] = mnext[h];
        load_bits(bi + 1, mnext);
        const float2 *suv = buf_uv(bi & 1);
        const float4 *sco = buf_co(bi & 1);
        const int2 *ssem = buf_sem(bi & 1);
        if (b0 < last && !stored) {
          // no stored bits: re-test the pairs before the last contributor
          const short4 *sbox = buf_box(bi & 1);
          const int n = min(batch_n(bi), (int)(last - b0));
          for (int j = 0; j < n; ++j) {
            const short4 bx = sbox[j];
            if (px < bx.x || px > bx.y || py < bx.z || py > bx.w) continue;
            float alpha, G, araw, dx, dy;
            if (gauss_alpha(suv[j], sco[j], fpx, fpy, alpha, G, araw, dx, dy)) mine[j >> 5] |= 1u << (j & 31);
          }
        }
#pragma unroll
        for (int h = 0; h < NW; ++h) {
          uint32_t un = __reduce_or_sync(0xffffffffu, mine[h]);
          while (un) {
            const int jb = __ffs(un) - 1;
            un &= un - 1;
            const int j = h * 32 + jb;
            // branch-free alpha (a contributor has power <= 0; other lanes get w = 0)
            const float2 uv_ = suv[j];
            const float4 co_ = sco[j];
            const float dx = __fsub_rn(uv_.x, fpx), dy = __fsub_rn(uv_.y, fpy);
            const float q_ = __fmaf_rn(co_.x, __fmul_rn(dx, dx), __fmul_rn(co_.z, __fmul_rn(dy, dy)));
            const float power = __fmaf_rn(-0.5f, q_, -__fmul_rn(co_.y, __fmul_rn(dx, dy)));
            const float araw = __fmul_rn(co_.w, __expf(power));
            const float alpha = araw < kAlphaMax ? araw : kAlphaMax;
            const bool on = (mine[h] >> jb) & 1u;
            const float w = on ? __fmul_rn(alpha, T) : 0.f;
            if (on) T = __fmul_rn(T, __fsub_rn(1.f, alpha));
            scatter_classes_marked<K>(myP, ssem + j, k, c_lo, mc, w, B);
          }
        }
        cp_async_wait_all();
        mark(bi + 1);
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
}

// Plan of the candidate waves (one CTA): the bit units of every view (its
// tiles' batch counts, from the exclusive scan mask_off), greedy waves of
// consecutive views whose units fit the capacity (a view larger than the
// capacity forms its own wave; its tiles that do not fit re-test), the
// waves' tile ranges, first units and cleared tickets.
__global__ void k_cand_plan(const uint32_t *__restrict__ mask_off, const uint32_t *__restrict__ tile_off,
                            int n_views, uint32_t cap_units, CandPlan p) {
  __shared__ uint32_t s_units[kMaxViews];
  const int t = threadIdx.x;
  if (t < n_views) s_units[t] = mask_off[tile_off[t + 1]] - mask_off[tile_off[t]];
  __syncthreads();
  if (t != 0) return;
  int w = 0;
  uint32_t used = 0;
  const uint32_t total_tiles = tile_off[n_views];
  p.wave[0] = 0u;
  for (int v = 0; v < n_views; ++v) {
    if (used > 0 && used + s_units[v] > cap_units && w + 1 < p.waves) {
      p.wave[5 * w + 1] = tile_off[v];
      ++w;
      p.wave[5 * w] = tile_off[v];
      used = 0;
    }
    used += s_units[v];
  }
  p.wave[5 * w + 1] = total_tiles;
  for (int i = w + 1; i < p.waves; ++i) p.wave[5 * i] = p.wave[5 * i + 1] = total_tiles;
  for (int i = 0; i < p.waves; ++i) {
    p.wave[5 * i + 2] = mask_off[p.wave[5 * i]];
    p.wave[5 * i + 3] = p.wave[5 * i + 4] = 0u;
  }
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

// CTAs per SM of a persistent candidate pass (occupancy of the kernel with
// its dynamic shared memory), cached per (kernel, shared memory, device).
static int resident_ctas(const void *func, int threads, size_t smem) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, func, threads, smem) != cudaSuccess || n < 1) n = 1;
  return n;
}

template <int TW, int TH, int K, int B>
static cudaError_t launch_cand_waves(const CandArgs &a, size_t smem_blend, size_t smem_sem, int waves,
                                     cudaStream_t s) {
  const void *fb = (const void *)k_cand_blend<TW, TH, B, kCandBlendPpt>;
  const void *fs = (const void *)k_cand_sem<TW, TH, K, B>;
  cudaError_t e = ensure_smem_limit(fs, (int)kSmemBudget);
  if (e != cudaSuccess) return e;
  const int sms = device_sms();
  if (sms < 1) return cudaErrorInvalidDevice;
  const unsigned gb = (unsigned)(sms * resident_ctas(fb, TW * TH / kCandBlendPpt, smem_blend));
  const unsigned gs = (unsigned)(sms * resident_ctas(fs, TW * TH, smem_sem));
  for (int w = 0; w < waves; ++w) {
    k_cand_blend<TW, TH, B, kCandBlendPpt><<<gb, TW * TH / kCandBlendPpt, smem_blend, s>>>(a, w);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_cand_sem<TW, TH, K, B><<<gs, TW * TH, smem_sem, s>>>(a, w);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <int TW, int TH, int B>
static cudaError_t launch_cand_two_pass(const CandArgs &a, size_t smem_blend, size_t smem_sem, int waves,
                                        cudaStream_t s) {
  if (a.k == 3) return launch_cand_waves<TW, TH, 3, B>(a, smem_blend, smem_sem, waves, s);
  if (a.k == 8) return launch_cand_waves<TW, TH, 8, B>(a, smem_blend, smem_sem, waves, s);
  return launch_cand_waves<TW, TH, 0, B>(a, smem_blend, smem_sem, waves, s);
}

template <int TW, int TH>
static cudaError_t launch_cand_batch(int batch, const CandArgs &a, size_t smem_blend, size_t smem_sem, int waves,
                                     cudaStream_t s) {
  if (batch == 32) return launch_cand_two_pass<TW, TH, 32>(a, smem_blend, smem_sem, waves, s);
  if (batch == 128) return launch_cand_two_pass<TW, TH, 128>(a, smem_blend, smem_sem, waves, s);
  return launch_cand_two_pass<TW, TH, 64>(a, smem_blend, smem_sem, waves, s);
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
  if (L.cand_cap_units > 0) {
    // two passes over the waves: batch offsets of every tile, the wave
    // plan, then blend + bits, classes + entropy
    const int B = L.cand_batch;
    a.mask_off = P.mask_off;
    a.masks = P.masks;
    a.cap_units = (uint32_t)L.cand_cap_units;
    a.clast = P.clast;
    a.plan = cand_plan(L, P);
    e = launch_tile_batch_offsets(P.ranges, grid, P.mask_off, P.counters, s, B);
    if (e != cudaSuccess) return e;
    k_cand_plan<<<1, kMaxViews, 0, s>>>(P.mask_off, P.tile_off, L.n_views, a.cap_units, a.plan);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t fixed = 2 * cand_sem_batch_bytes(sc.k, B);
    {
      // class rows beside the two batch buffers, within the two-CTAs budget
      const int max_stride = (int)((kSmemBudget - fixed) / ((size_t)threads * sizeof(float)));
      const int st = (sc.m & 1) ? sc.m : sc.m + 1;
      if (st <= max_stride) {
        a.mchunk = sc.m; a.mstride = st; a.nchunks = 1;
      } else {
        const int c = ((max_stride - 1) / 32) * 32;
        a.mchunk = c; a.mstride = c + 1; a.nchunks = (sc.m + c - 1) / c;
      }
    }
    const size_t smem_sem = fixed + (size_t)threads * a.mstride * sizeof(float);
    const size_t smem_blend = (size_t)(threads / kCandBlendPpt / 32) * cand_blend_warp_bytes(kCandBlendPpt);
    if (L.tile_w == 16 && L.tile_h == 16) return launch_cand_batch<16, 16>(B, a, smem_blend, smem_sem, L.cand_waves, s);
    if (L.tile_w == 16 && L.tile_h == 8) return launch_cand_batch<16, 8>(B, a, smem_blend, smem_sem, L.cand_waves, s);
    if (L.tile_w == 8 && L.tile_h == 8) return launch_cand_batch<8, 8>(B, a, smem_blend, smem_sem, L.cand_waves, s);
    if (L.tile_w == 32 && L.tile_h == 8) return launch_cand_batch<32, 8>(B, a, smem_blend, smem_sem, L.cand_waves, s);
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
