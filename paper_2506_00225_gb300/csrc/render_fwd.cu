// render_fwd.cu -- forward tile blend: Eq. 1 (colour, depth, silhouette) and
// Eq. 3 (sparse top-k semantics), supplement "Sparse Rendering".
//
// Two passes over each screen tile (one CTA per tile, one thread per pixel,
// each warp an 8 x 4 pixel block):
//
// Pass 1 (k_blend) walks the tile's depth-sorted pair range in batches
// staged in shared memory.  For every staged Gaussian the stager records
// which warps' blocks meet its alpha box (the pixels where alpha can reach
// 1/255), and each warp visits only those Gaussians.  A thread composites a
// Gaussian whose box holds its pixel, front to back, and stops before the
// Gaussian that would take the transmittance below 1e-4.  Besides colour,
// depth, silhouette, the final transmittance and the last contributor, it
// writes one bit per (pixel, staged Gaussian) that contributed.  Pass 1 keeps
// no per-pixel class accumulator, so many CTAs share an SM.
//
// Pass 2 (k_semantic) rebuilds Eq. 3: it walks only each pixel's
// contributor bits, recomputes alpha with the same function (bit-identical)
// and the transmittance from the contributors alone, and scatters the k
// (class, weight) pairs into a per-pixel M-class accumulator in shared memory
// (k adds per contributor instead of M, the point of the sparse
// representation).  Then it writes the semantic map, or, in the fused mean-L1
// mode, compares it with the target map (read from L2 after a bulk prefetch)
// and keeps per-value sign bits and per-tile sums.  When M does not fit,
// classes are processed in chunks of 32-class multiples.
#include "gs_internal.cuh"
#include "render_common.cuh"

namespace gs {

// Per tile: number of staged batches (of `batch` pairs) of its pair range.
__global__ void k_tile_batches(const uint2 *__restrict__ ranges, uint32_t ntiles, uint32_t *units, uint32_t batch) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < ntiles) units[t] = (ranges[t].y - ranges[t].x + batch - 1) / batch;
}

// Shared memory of one warp of the blend pass: 32 staging slots (conic +
// opacity, colour + depth, mean, and per row group the lanes the Gaussian
// reaches).
__host__ __device__ inline size_t blend_warp_bytes(int ppt) { return 32 * (16 + 16 + 8 + 4 * (size_t)ppt); }

template <int TW, int TH, bool L1, int PPT>
__global__ void __launch_bounds__(TW *TH / PPT) k_blend(FwdArgs a) {
  using FP = Footprint<TW, TH, PPT>;
  constexpr int THREADS = FP::kThreads;
  constexpr int WARPS = FP::kWarps;
  constexpr int NPIX = FP::kPix;
  extern __shared__ float4 smem4[];
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
  char *wb = reinterpret_cast<char *>(smem4) + warp * blend_warp_bytes(PPT);
  float4 *w_co = reinterpret_cast<float4 *>(wb);
  float4 *w_cd = w_co + 32;
  float2 *w_uv = reinterpret_cast<float2 *>(w_co + 64);
  uint32_t *w_lm = reinterpret_cast<uint32_t *>(w_uv + 32);  // [row group][slot]
  __shared__ float red[2][WARPS];
  if (a.counters->status & kStatusTimeout) return;  // the binning is incomplete

  const int tile = blockIdx.x;
  const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
  const int ox = tx * TW, oy = ty * TH;
  const uint2 rg = a.ranges[tile];
  const int lx = FP::lx();
  const int px = ox + lx;
  const float fpx = (float)px + 0.5f;
  const uint32_t unit0 = a.masks ? a.mask_off[tile] : 0u;
  const int bx0 = ox + (int)(warp % FP::kWX) * 8, by0 = oy + (int)(warp / FP::kWX) * FP::kBH;  // the warp's block

  // PPT pixels per thread, one column, rows 4 apart: they share every
  // staged load and the x offset of every Gaussian
  int py[PPT], lp[PPT];
  float fpy[PPT], T[PPT], cr[PPT], cg[PPT], cb[PPT], cd[PPT];
  uint32_t last[PPT];
  bool inside[PPT], done[PPT];
#pragma unroll
  for (int i = 0; i < PPT; ++i) {
    const int ly = FP::ly(i);
    py[i] = oy + ly;
    lp[i] = ly * TW + lx;
    fpy[i] = (float)py[i] + 0.5f;
    inside[i] = px < a.width && py[i] < a.height;
    done[i] = !inside[i];
    T[i] = 1.f; cr[i] = cg[i] = cb[i] = cd[i] = 0.f;
    last[i] = 0;
  }
  uint32_t ncontrib = 0;
  auto all_done = [&]() {
    bool d = true;
#pragma unroll
    for (int i = 0; i < PPT; ++i) d = d && done[i];
    return d;
  };
  // Every warp works through the tile's pairs on its own, 32 at a time: a
  // lane per pair tests the pair's alpha box against the warp's block (per
  // row group), the pairs that reach it are staged (packed) and composited in
  // order.  The warp stops at a batch boundary once all its pixels are done;
  // the groups up to the end of the last batch write their bits (zero when
  // empty), so every batch a pixel can still read has its bits.
  const uint32_t gend = rg.x + (rg.y - rg.x + kBatch - 1) / kBatch * kBatch;
  for (uint32_t g0 = rg.x; g0 < gend; g0 += 32) {
    const uint32_t rel = g0 - rg.x, bi = rel / kBatch, h = (rel % kBatch) / 32;
    const int n = g0 < rg.y ? (int)min(32u, rg.y - g0) : 0;
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
        w_cd[slot] = __ldg(a.rec.cd + r);
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
          const float4 cdp = w_cd[sl];
          cr[i] = fmaf(w, cdp.x, cr[i]); cg[i] = fmaf(w, cdp.y, cg[i]); cb[i] = fmaf(w, cdp.z, cb[i]);
          cd[i] = fmaf(w, cdp.w, cd[i]);
          T[i] = Tn;
          bits[i] |= 1u << bit;
        }
      }
    }
    // last contributor, contribution count and this group's bits
#pragma unroll
    for (int i = 0; i < PPT; ++i) {
      if (bits[i]) last[i] = rel + (32 - __clz(bits[i]));
      ncontrib += __popc(bits[i]);
      if (a.masks && unit0 + bi < a.mask_units)
        a.masks[((size_t)(unit0 + bi) * 2 + h) * NPIX + lp[i]] = bits[i];
    }
    if (h == 1 && __all_sync(0xffffffffu, all_done())) break;
  }
  {
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
      const int cw = code_words(a.nwc);
      const float d0 = cr[i] - a.t_rgb[3 * pix], d1 = cg[i] - a.t_rgb[3 * pix + 1];
      const float d2 = cb[i] - a.t_rgb[3 * pix + 2], d3 = cd[i] - a.t_depth[pix];
      // Sec. 3.1 objective mode: only pixels with S > 0.99 count
      const bool keep = !a.objective || 1.f - T[i] > kSilMinLoss;
      const uint32_t nz = keep ? ((d0 != 0.f ? 1u : 0u) | (d1 != 0.f ? 2u : 0u) | (d2 != 0.f ? 4u : 0u) |
                                  (d3 != 0.f ? 8u : 0u)) : 0u;
      const uint32_t ng = (d0 < 0.f ? 1u : 0u) | (d1 < 0.f ? 2u : 0u) | (d2 < 0.f ? 4u : 0u) | (d3 < 0.f ? 8u : 0u);
      uint2 *cp = reinterpret_cast<uint2 *>(a.codes + pix * cw);
      cp[0] = make_uint2(nz, ng);
      if (!a.t_sem)
        for (int wd = 0; wd < a.nwc; ++wd) cp[1 + wd] = make_uint2(0u, 0u);
      if (keep) {
        l1_rgb += fabsf(d0) + fabsf(d1) + fabsf(d2);
        l1_d += fabsf(d3);
      }
    }
  }
  if (L1) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      l1_rgb += __shfl_xor_sync(0xffffffffu, l1_rgb, o);
      l1_d += __shfl_xor_sync(0xffffffffu, l1_d, o);
    }
    if (lane == 0) { red[0][warp] = l1_rgb; red[1][warp] = l1_d; }
    __syncthreads();
    if (threadIdx.x < 3) {
      double s = 0.0;
      if (threadIdx.x < 2)
        for (int w = 0; w < WARPS; ++w) s += red[threadIdx.x][w];
      a.lpart[3 * (size_t)tile + threadIdx.x] = s;  // [2] (semantic) is set by pass 2
    }
  }
}

// Class chunking for pass 2, whose fixed part is two batch buffers.
static void sem_chunks(int m, int npix, int k, bool acc, FwdArgs &a) {
  const size_t fixed = 2 * sem_batch_bytes(k), base = batch_smem_bytes(k);
  chunk_classes(m, npix, k, acc, &a.mchunk, &a.mstride, &a.nchunks, fixed > base ? fixed - base : 0);
}

template <int TW, int TH, bool L1, int K>
__global__ void __launch_bounds__(TW *TH, 2) k_semantic(FwdArgs a) {
  using FP = Footprint<TW, TH, 1>;
  constexpr int THREADS = FP::kThreads;
  constexpr int WARPS = FP::kWarps;
  constexpr int NPIX = FP::kPix;
  extern __shared__ float4 smem4[];
  const int k = a.k;
  // two batch buffers, then the accumulator rows
  char *sbase = reinterpret_cast<char *>(smem4);
  const size_t bbytes = sem_batch_bytes(k);
  float *sP = reinterpret_cast<float *>(sbase + 2 * bbytes);
  __shared__ float red[WARPS];
  __shared__ uint32_t s_maxlast;
  if (a.counters->status & kStatusTimeout) return;

  const int tile = blockIdx.x;
  const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
  const int ox = tx * TW, oy = ty * TH;
  const uint2 rg = a.ranges[tile];
  const int lx = FP::lx(), ly = FP::ly(0);
  const int px = ox + lx, py = oy + ly;
  const int lp = ly * TW + lx;
  const bool inside = px < a.width && py < a.height;
  const float fpx = (float)px + 0.5f, fpy = (float)py + 0.5f;
  float *myP = sP + threadIdx.x * a.mstride;  // accumulator row of this thread's pixel
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
  const uint32_t unit0 = a.masks ? a.mask_off[tile] : 0u;
  const int cw = code_words(a.nwc);

  // fused mean-L1 without a semantic map output: the accumulator rows start
  // as the target rows and the contributions are subtracted, so they end as
  // target - rendered and the comparison needs no second read of the target
  const bool tmode = L1 && a.t_sem && !a.sem;
  if (L1 && a.t_sem && !tmode && (int)threadIdx.x < TH) {
    // warm L2 with the tile's target rows while the accumulation runs
    const int y = oy + (int)threadIdx.x;
    if (y < a.height) {
      const int vw = min(TW, a.width - ox);
      prefetch_l2(a.t_sem, (size_t)a.width * a.height * a.m * 4, a.t_sem + ((size_t)y * a.width + ox) * a.m,
                  (size_t)vw * a.m * 4);
    }
  }
  const uint32_t last = inside ? a.nlast[(size_t)py * a.width + px] : 0u;
  if (threadIdx.x == 0) s_maxlast = 0;
  __syncthreads();
  if (last) atomicMax(&s_maxlast, last);
  __syncthreads();
  const uint32_t maxlast = s_maxlast;
  const int nbatch = (int)((maxlast + kBatch - 1) / kBatch);
  float l1_sem = 0.f;

  auto buf_uv = [&](int q) { return reinterpret_cast<float2 *>(sbase + q * bbytes); };
  auto buf_co = [&](int q) { return reinterpret_cast<float4 *>(sbase + q * bbytes + kBatch * 8); };
  auto buf_box = [&](int q) { return reinterpret_cast<short4 *>(sbase + q * bbytes + kBatch * 24); };
  auto buf_sem = [&](int q) { return reinterpret_cast<int2 *>(sbase + q * bbytes + kBatch * 32); };
  auto batch_n = [&](int bi) { return (int)min((uint32_t)kBatch, rg.y - (rg.x + (uint32_t)bi * kBatch)); };
  auto issue = [&](int bi, uint32_t r) {  // thread t < n copies record r into slot t of buffer bi & 1
    const int q = bi & 1, t = threadIdx.x;
    cp_async8(buf_uv(q) + t, a.rec.uv + r);
    cp_async16(buf_co(q) + t, a.rec.co + r);
    if (!a.masks) cp_async8(buf_box(q) + t, a.rec.box + r);
    const int2 *src = a.rec.sem + (size_t)r * k;
    for (int l = 0; l < k; ++l) cp_async8(buf_sem(q) + l * kBatch + t, src + l);  // entry-major
  };

  for (int c = 0; c < a.nchunks; ++c) {
    const int c_lo = c * a.mchunk, c_hi = min(a.m, c_lo + a.mchunk);
    const int mc = c_hi - c_lo;
    if (tmode) {
      // each warp copies whole target rows of its pixels (coalesced 128-byte
      // runs), lanes over classes; rows of pixels outside the image start at 0
      for (int p = (int)warp; p < NPIX; p += WARPS) {
        float *row = sP + FP::thread_of(p) * a.mstride;
        const int qx = ox + p % TW, qy = oy + p / TW;
        if (qx < a.width && qy < a.height) {
          const float *src = a.t_sem + ((size_t)qy * a.width + qx) * a.m + c_lo;
          for (int e = (int)lane; e < mc; e += 32) cp_async4(row + e, src + e);
        } else {
          for (int e = (int)lane; e < mc; e += 32) row[e] = 0.f;
        }
      }
    } else {
      for (int q = 0; q < mc; ++q) myP[q] = 0.f;
    }
    float T = 1.f;
    // pipeline: copies of batch bi + 1 fly while batch bi is processed; the
    // pair indices are fetched one batch further ahead
    const int t = threadIdx.x;
    if (nbatch > 0 && t < batch_n(0)) issue(0, a.pvals[rg.x + t]);
    cp_async_commit();
    uint32_t pv = (nbatch > 1 && t < batch_n(1)) ? a.pvals[rg.x + kBatch + t] : 0u;
    // contributor words of the next batch, loaded one batch ahead (their
    // latency overlaps the walk of the current batch)
    uint32_t mn0 = 0u, mn1 = 0u;
    if (a.masks && nbatch > 0 && last > 0u) {
      const uint32_t *mw = a.masks + (size_t)unit0 * 2 * NPIX;
      mn0 = mw[lp];
      mn1 = mw[NPIX + lp];
    }
    cp_async_wait_all();
    if (nbatch > 0 && t < batch_n(0)) mark_repeated_ids<K>(buf_sem(0) + t, kBatch);
    __syncthreads();
    for (int bi = 0; bi < nbatch; ++bi) {
      if (bi + 1 < nbatch && t < batch_n(bi + 1)) issue(bi + 1, pv);
      cp_async_commit();
      if (bi + 2 < nbatch && t < batch_n(bi + 2)) pv = a.pvals[rg.x + (uint32_t)(bi + 2) * kBatch + t];
      const uint32_t b0 = (uint32_t)bi * kBatch;
      // warp-uniform walk over the union of the warp's contributor bits: the
      // Gaussian's entries are broadcast reads, lanes that it does not touch
      // add zero weight, and the accumulator rows are indexed by thread so
      // that the 32 lanes' adds to one class fall in 32 distinct banks
      uint32_t mine[2] = {0u, 0u};
      const float2 *suv = buf_uv(bi & 1);
      const float4 *sco = buf_co(bi & 1);
      const int2 *ssem = buf_sem(bi & 1);
      if (a.masks) {
        mine[0] = mn0;
        mine[1] = mn1;
        mn0 = mn1 = 0u;
        if (bi + 1 < nbatch && b0 + kBatch < last) {
          const uint32_t *mw = a.masks + (size_t)(unit0 + bi + 1) * 2 * NPIX;
          mn0 = mw[lp];
          mn1 = mw[NPIX + lp];
        }
      }
      if (!a.masks) {
        // recomputation: contributors are the pairs up to the last one
        // whose pixel box holds the pixel and whose alpha passes 1/255.
        // First the pairs whose box meets the warp's pixel block (two slots
        // per lane); the others fail every pixel's box test.
        const short4 *sbox = buf_box(bi & 1);
        const int nb = batch_n(bi);
        const int bx0 = __reduce_min_sync(0xffffffffu, px), bx1 = __reduce_max_sync(0xffffffffu, px);
        const int by0 = __reduce_min_sync(0xffffffffu, py), by1 = __reduce_max_sync(0xffffffffu, py);
        uint32_t meets[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int j = h * 32 + (int)lane;
          const short4 bx = sbox[j];  // slots past nb hold stale boxes: masked out
          meets[h] = __ballot_sync(0xffffffffu, j < nb && bx.x <= bx1 && bx.y >= bx0 && bx.z <= by1 && bx.w >= by0);
        }
        if (b0 < last) {
          const int n = min(nb, (int)(last - b0));
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int lim = n - 32 * h;
            uint32_t cand = lim >= 32 ? meets[h] : (lim > 0 ? meets[h] & ((1u << lim) - 1u) : 0u);
            while (cand) {
              const int jb = __ffs(cand) - 1;
              cand &= cand - 1u;
              const short4 bx = sbox[h * 32 + jb];
              if (px < bx.x || px > bx.y || py < bx.z || py > bx.w) continue;
              float alpha, G, araw, dx, dy;
              if (gauss_alpha(suv[h * 32 + jb], sco[h * 32 + jb], fpx, fpy, alpha, G, araw, dx, dy))
                mine[h] |= 1u << jb;
            }
          }
        }
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
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
          float w = on ? __fmul_rn(alpha, T) : 0.f;
          if (tmode) w = -w;
          if (on) T = __fmul_rn(T, __fsub_rn(1.f, alpha));
          scatter_classes_marked<K>(myP, ssem + j, k, c_lo, mc, w, kBatch);
        }
      }
      cp_async_wait_all();
      if (bi + 1 < nbatch && t < batch_n(bi + 1)) mark_repeated_ids<K>(buf_sem((bi + 1) & 1) + t, kBatch);
      __syncthreads();
    }
    __syncthreads();
    const int vw = min(TW, a.width - ox);
    if (a.sem) {
      for (int r = 0; r < TH; ++r) {
        const int y = oy + r;
        if (y >= a.height) break;
        float *dst = a.sem + ((size_t)y * a.width + ox) * a.m + c_lo;
        for (int e = threadIdx.x; e < vw * mc; e += THREADS) {
          const int p = e / mc, cl = e - p * mc;
          dst[(size_t)p * a.m + cl] = sP[FP::thread_of(r * TW + p) * a.mstride + cl];
        }
      }
    }
    if (tmode) {
      // each thread reads its own pixel's row (target - rendered; odd stride,
      // conflict-free) and assembles the sign words 32 classes at a time
      if (inside) {
        uint2 *cp = reinterpret_cast<uint2 *>(a.codes + ((size_t)py * a.width + px) * cw);
        for (int wd = c_lo >> 5; wd < (c_hi + 31) >> 5; ++wd) {
          const float *v = myP + (wd * 32 - c_lo);
          uint32_t nz = 0u, ng = 0u;
          float s = 0.f;
          if (wd * 32 + 32 <= c_hi) {
#pragma unroll
            for (int b = 0; b < 32; ++b) {
              nz |= (v[b] != 0.f ? 1u : 0u) << b;
              ng |= (v[b] > 0.f ? 1u : 0u) << b;  // rendered < target
              s += fabsf(v[b]);
            }
          } else {
            for (int b = 0; b < c_hi - wd * 32; ++b) {
              nz |= (v[b] != 0.f ? 1u : 0u) << b;
              ng |= (v[b] > 0.f ? 1u : 0u) << b;
              s += fabsf(v[b]);
            }
          }
          l1_sem += s;
          cp[1 + wd] = make_uint2(nz, ng);
        }
      }
    } else if (L1 && a.t_sem) {
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
              if (mcl < c_hi) d = sP[FP::thread_of(p) * a.mstride + (mcl - c_lo)] - tv[g][u];
              const uint32_t nz = __ballot_sync(0xffffffffu, d != 0.f);
              const uint32_t ng = __ballot_sync(0xffffffffu, d < 0.f);
              l1_sem += fabsf(d);
              if (lane == 0)
                reinterpret_cast<uint2 *>(a.codes + (size_t)((row[g] - a.t_sem) / a.m) * cw)[1 + wd] =
                    make_uint2(nz, ng);
            }
          }
        }
      }
    }
    __syncthreads();  // the next chunk reuses the accumulator rows
  }
  if (L1 && a.t_sem) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) l1_sem += __shfl_xor_sync(0xffffffffu, l1_sem, o);
    if (lane == 0) red[warp] = l1_sem;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < WARPS; ++w) s += red[w];
      a.lpart[3 * (size_t)tile + 2] = s;
    }
    finish_loss<THREADS>(a, 0, gridDim.x);
  }
}

// loss = sum|d rgb| / (3 npix) + sum|d depth| / npix + sum|d sem| / (npix m)
// Mean-L1 mode: rgb / (3 npix) + depth / npix + sem / (npix m).  Sec. 3.1
// objective mode (objective != 0): 0.5 rgb + depth (sums over the silhouette
// mask) + sem / npix (mean of the per-pixel semantic terms).
__global__ void k_l1_tiles_final(const double *lpart, int ntiles, double npix, double m, int has_sem, int objective,
                                 float *loss) {
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
    double l;
    if (objective) {
      l = 0.5 * t[0] + t[1];
      if (has_sem) l += t[2] / npix;
    } else {
      l = t[0] / (3.0 * npix) + t[1] / npix;
      if (has_sem) l += t[2] / (npix * m);
    }
    *loss = (float)l;
  }
}

template <int TW, int TH, bool L1, int K>
static cudaError_t launch_semantic(const FwdArgs &a, int grid, size_t smem, cudaStream_t s) {
  {
    const cudaError_t e = ensure_smem_limit((const void *)k_semantic<TW, TH, L1, K>, (int)kSmemBudget);
    if (e != cudaSuccess) return e;
  }
  k_semantic<TW, TH, L1, K><<<grid, TW * TH, smem, s>>>(a);
  return cudaGetLastError();
}

template <int TW, int TH, bool L1>
static cudaError_t launch_shape(const FwdArgs &a, int grid, size_t smem_sem, bool run_sem, cudaStream_t s) {
  if (a.blend_ppt == 2) k_blend<TW, TH, L1, 2><<<grid, TW * TH / 2, (TW * TH / 64) * blend_warp_bytes(2), s>>>(a);
  else k_blend<TW, TH, L1, 1><<<grid, TW * TH, (TW * TH / 32) * blend_warp_bytes(1), s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !run_sem) return e;
  // the common top-k sizes get an unrolled scatter
  if (a.k == 3) return launch_semantic<TW, TH, L1, 3>(a, grid, smem_sem, s);
  if (a.k == 8) return launch_semantic<TW, TH, L1, 8>(a, grid, smem_sem, s);
  return launch_semantic<TW, TH, L1, 0>(a, grid, smem_sem, s);
}

template <bool L1>
static cudaError_t dispatch_fwd(const Layout &L, const FwdArgs &a, int grid, size_t smem_sem, bool run_sem,
                                cudaStream_t s) {
  if (L.tile_w == 16 && L.tile_h == 16) return launch_shape<16, 16, L1>(a, grid, smem_sem, run_sem, s);
  if (L.tile_w == 16 && L.tile_h == 8) return launch_shape<16, 8, L1>(a, grid, smem_sem, run_sem, s);
  if (L.tile_w == 8 && L.tile_h == 8) return launch_shape<8, 8, L1>(a, grid, smem_sem, run_sem, s);
  if (L.tile_w == 32 && L.tile_h == 8) return launch_shape<32, 8, L1>(a, grid, smem_sem, run_sem, s);
  return cudaErrorInvalidConfiguration;
}

FwdArgs fwd_args(const Layout &L, const WsPtrs &P, int pbuf, const gs_scene &sc) {
  FwdArgs a{};
  a.ranges = P.ranges;
  a.pvals = P.pvals[pbuf];
  a.rec = rec_ptrs(P);
  a.k = sc.k; a.m = sc.m;
  a.width = L.cam0_w; a.height = L.cam0_h;
  a.tiles_x = (L.cam0_w + L.tile_w - 1) / L.tile_w;
  a.tfinal = P.tfinal; a.nlast = P.nlast;
  a.counters = P.counters;
  a.mask_off = L.mask_units ? P.mask_off : nullptr;
  a.masks = L.mask_units ? P.masks : nullptr;
  a.mask_units = (uint32_t)L.mask_units;
  a.codes = P.codes;
  a.nwc = L.nwc;
  a.lpart = P.lpart;
  a.blend_ppt = L.ppt >= 2 ? 2 : 1;  // every compiled tile height is a multiple of 8
  return a;
}

// First (tile, batch) unit of every tile: batches per tile, exclusive scan.
cudaError_t launch_tile_batch_offsets(const uint2 *ranges, uint32_t ntiles, uint32_t *mask_off, Counters *counters,
                                      cudaStream_t s, int batch) {
  k_tile_batches<<<(ntiles + 255) / 256, 256, 0, s>>>(ranges, ntiles, mask_off, (uint32_t)batch);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // mask_off[ntiles] receives the total
  return launch_scan_single(mask_off, ntiles, mask_off + ntiles, 0xffffffffu, counters, s);
}

static cudaError_t launch_mask_offsets(const Layout &L, const WsPtrs &P, int grid, cudaStream_t s) {
  if (!L.mask_units) return cudaSuccess;
  return launch_tile_batch_offsets(P.ranges, (uint32_t)grid, P.mask_off, P.counters, s);
}

cudaError_t launch_render_fwd(const Layout &L, const WsPtrs &P, int pbuf, const gs_scene &sc, float *rgb,
                              float *depth, float *sil, float *sem, cudaStream_t s) {
  FwdArgs a = fwd_args(L, P, pbuf, sc);
  const int tiles_y = (L.cam0_h + L.tile_h - 1) / L.tile_h;
  a.rgb_out = rgb; a.depth_out = depth; a.sil_out = sil; a.sem = sem;
  const int npix = L.tile_w * L.tile_h;  // accumulator rows: one per pixel of the tile
  sem_chunks(sc.m, npix, sc.k, sem != nullptr, a);
  const size_t smem = 2 * sem_batch_bytes(sc.k) + (sem ? (size_t)npix * a.mstride * sizeof(float) : 0);
  const int grid = a.tiles_x * tiles_y;
  if (grid == 0) return cudaSuccess;
  cudaError_t e = launch_mask_offsets(L, P, grid, s);
  if (e != cudaSuccess) return e;
  return dispatch_fwd<false>(L, a, grid, smem, sem != nullptr, s);
}

cudaError_t launch_render_fwd_l1(const Layout &L, const WsPtrs &P, int pbuf, const gs_scene &sc,
                                 const float *t_rgb, const float *t_depth, const float *t_sem, float *rgb,
                                 float *depth, float *sil, float *sem, float *loss, cudaStream_t s) {
  FwdArgs a = fwd_args(L, P, pbuf, sc);
  const int tiles_y = (L.cam0_h + L.tile_h - 1) / L.tile_h;
  a.rgb_out = rgb; a.depth_out = depth; a.sil_out = sil; a.sem = sem;
  a.t_rgb = t_rgb; a.t_depth = t_depth; a.t_sem = t_sem;
  const bool acc = sem != nullptr || t_sem != nullptr;
  const int npix = L.tile_w * L.tile_h;
  sem_chunks(sc.m, npix, sc.k, acc, a);
  const size_t smem = 2 * sem_batch_bytes(sc.k) + (acc ? (size_t)npix * a.mstride * sizeof(float) : 0);
  const int grid = a.tiles_x * tiles_y;
  if (grid == 0) return cudaSuccess;
  cudaError_t e = launch_mask_offsets(L, P, grid, s);
  if (e != cudaSuccess) return e;
  a.loss = loss;
  a.npix_d = (double)L.npix;
  e = dispatch_fwd<true>(L, a, grid, smem, acc, s);
  if (e != cudaSuccess) return e;
  if (t_sem) return cudaSuccess;  // the semantic pass's last tile wrote the loss
  return launch_loss_final(P.lpart, grid, (double)L.npix, (double)sc.m, 0, 0, loss, s);
}

cudaError_t launch_blend_objective(const Layout &L, const FwdArgs &a, int grid, cudaStream_t s) {
  return dispatch_fwd<true>(L, a, grid, 0, false, s);
}

cudaError_t launch_blend_plain(const Layout &L, const FwdArgs &a, int grid, cudaStream_t s) {
  return dispatch_fwd<false>(L, a, grid, 0, false, s);
}

cudaError_t launch_loss_final(const double *lpart, int ntiles, double npix, double m, int has_sem, int objective,
                              float *loss, cudaStream_t s) {
  k_l1_tiles_final<<<1, 1024, 0, s>>>(lpart, ntiles, npix, m, has_sem, objective, loss);
  return cudaGetLastError();
}

}  // namespace gs
