// render_objective.cu -- the mapping step's Sec. 3.1 objective fused into the
// render passes: silhouette-masked depth / colour L1 (summed over pixels) and
// the entropy-masked Hellinger + cosine semantic term (Eq. 4, Eq. 5; averaged
// over pixels), with neither the H x W x M semantic map nor its gradient ever
// written to memory.
//
// Pass 1 is the blend pass in its fused-loss form with the silhouette mask
// (sign codes of the masked depth / colour errors and their per-tile sums).
// The semantic pass below, one CTA per tile, then
//   (1) accumulates each pixel's class distribution P from the contributor
//       bits of pass 1 (Eq. 3), in a per-pixel shared-memory row, exactly as
//       the plain semantic pass does;
//   (2) one thread per pixel: reads its target distribution Q (warmed into
//       L2 for the whole tile when the CTA starts), forms the entropy mask,
//       the Hellinger distance, the cosine and the pixel's term, and
//       overwrites its row with d term / d P_m divided by the pixel count
//       (the same arithmetic and summation order as the objective on
//       rendered maps);
//   (3) walks the contributors again, recomputing w = alpha T, and adds
//       sum_p w * dP_p[id] into the objective's gradient of every (Gaussian,
//       entry) weight: a transposed warp sum, one atomic per entry and warp.
// The semantic term reaches the semantic weights only (Sec. 3.1: the
// geometry does not follow the semantic loss), so the adjoint of the blend
// needs no class data: it takes the depth / colour signs from the codes and
// adds dL/dloss times the gradient of (3) to the weights' gradient.
// Requires the contributor bits (not the recompute mode) and a class count
// whose accumulator fits one shared-memory chunk.
#include "gs_internal.cuh"
#include "render_common.cuh"
#include "objective_math.cuh"

namespace gs {

template <int TW, int TH, int K>
__global__ void __launch_bounds__(TW *TH, 2) k_sem_objective(FwdArgs a, float log_k, float inv_n) {
  using FP = Footprint<TW, TH, 1>;
  constexpr int WARPS = FP::kWarps;
  constexpr int NPIX = FP::kPix;
  extern __shared__ float4 smem4[];
  const int k = a.k, m = a.m;
  char *sbase = reinterpret_cast<char *>(smem4);
  const size_t bbytes = sem_batch_bytes(k);
  float *sP = reinterpret_cast<float *>(sbase + 2 * bbytes);
  __shared__ double red[WARPS];
  __shared__ uint32_t s_maxlast;
  __shared__ uint8_t s_keep[NPIX];  // raster pixel of the tile: its semantic term is kept
  if (a.counters->status & kStatusTimeout) return;  // the binning is incomplete

  const int tile = blockIdx.x;
  const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
  const int ox = tx * TW, oy = ty * TH;
  const uint2 rg = a.ranges[tile];
  const int lx = FP::lx(), ly = FP::ly(0);
  const int px = ox + lx, py = oy + ly;
  const int lp = ly * TW + lx;
  const bool inside = px < a.width && py < a.height;
  const float fpx = (float)px + 0.5f, fpy = (float)py + 0.5f;
  float *myP = sP + threadIdx.x * a.mstride;
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
  const uint32_t unit0 = a.mask_off[tile];

  if ((int)threadIdx.x < TH) {
    // warm L2 with the tile's target rows while the class accumulation runs
    const int y = oy + (int)threadIdx.x;
    if (y < a.height) {
      const int vw = min(TW, a.width - ox);
      prefetch_l2(a.t_sem, (size_t)a.width * a.height * m * 4, a.t_sem + ((size_t)y * a.width + ox) * m,
                  (size_t)vw * m * 4);
    }
  }
  const uint32_t last = inside ? a.nlast[(size_t)py * a.width + px] : 0u;
  if (threadIdx.x == 0) s_maxlast = 0;
  __syncthreads();
  if (last) atomicMax(&s_maxlast, last);
  __syncthreads();
  const int nbatch = (int)((s_maxlast + kBatch - 1) / kBatch);

  // batch buffer: mean, conic, Gaussian id (in the 8-byte slot that holds
  // the pixel box in the recompute mode), k (class, weight) entries
  auto buf_uv = [&](int q) { return reinterpret_cast<float2 *>(sbase + q * bbytes); };
  auto buf_co = [&](int q) { return reinterpret_cast<float4 *>(sbase + q * bbytes + kBatch * 8); };
  auto buf_gid = [&](int q) { return reinterpret_cast<int *>(sbase + q * bbytes + kBatch * 24); };
  auto buf_sem = [&](int q) { return reinterpret_cast<int2 *>(sbase + q * bbytes + kBatch * 32); };
  auto batch_n = [&](int bi) { return (int)min((uint32_t)kBatch, rg.y - (rg.x + (uint32_t)bi * kBatch)); };
  auto issue = [&](int bi, uint32_t r) {
    const int q = bi & 1, t = threadIdx.x;
    cp_async8(buf_uv(q) + t, a.rec.uv + r);
    cp_async16(buf_co(q) + t, a.rec.co + r);
    cp_async4(buf_gid(q) + t, a.rec.gid + r);
    const int2 *src = a.rec.sem + (size_t)r * k;
    for (int l = 0; l < k; ++l) cp_async8(buf_sem(q) + l * kBatch + t, src + l);  // entry-major
  };
  // One front-to-back walk over the tile's batches (copies of batch bi + 1
  // in flight while bi is processed); a thread that is not live takes no
  // contributor bits.  For every Gaussian j in the union of
  // the warp's contributor bits: f(gid, on, w, entries) with on = the lane's
  // pixel takes the Gaussian, w = alpha T there and 0 elsewhere (a
  // warp-uniform call).
  auto walk = [&](bool live, auto &&f) {
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
      if (live && b0 < last) {
        const uint32_t *mw = a.masks + (size_t)(unit0 + bi) * 2 * NPIX;
        mine[0] = mw[lp];
        mine[1] = mw[NPIX + lp];
      }
      const float2 *suv = buf_uv(bi & 1);
      const float4 *sco = buf_co(bi & 1);
      const int *sgid = buf_gid(bi & 1);
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
          f(sgid[j], on, w, ssem + j);  // entry l at [l * kBatch]
        }
      }
      cp_async_wait_all();
      __syncthreads();
    }
  };

  // (1) the rendered class distribution P of this thread's pixel
  for (int c = 0; c < m; ++c) myP[c] = 0.f;
  walk(true, [&](int, bool, float w, const int2 *e) { scatter_classes_ilp<K>(myP, e, k, 0, m, w, kBatch); });

  // (2) per pixel: the semantic term, and d term / d P (over the pixel
  // count) in place of P.  Thread per pixel: its own row (shared memory,
  // odd stride: conflict-free) and its target row (global, two classes per
  // 8-byte load when the row allows; consecutive classes share a 32-byte
  // sector, so most reads hit L1).  A class where both distributions are 0
  // adds exactly nothing to the sums and has a zero gradient (its row entry
  // is already 0), so only the others do the arithmetic.  Pixels outside
  // the entropy mask keep their row (pass 3 skips them).
  double term_sum = 0.0;
  {
    const float *q = a.t_sem + (inside ? ((size_t)py * a.width + px) * m : 0);
    const bool pairs = (reinterpret_cast<uintptr_t>(q) & 7) == 0;
    const int m2 = pairs ? (m & ~3) : 0;  // classes read as 8-byte pairs, four per step
    float st[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    if (inside) {
#pragma unroll 4
      for (int c = 0; c < m2; c += 4) {
        const float2 q0 = __ldg(reinterpret_cast<const float2 *>(q + c));
        const float2 q1 = __ldg(reinterpret_cast<const float2 *>(q + c + 2));
        const float qv[4] = {q0.x, q0.y, q1.x, q1.y};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float pv = myP[c + u];
          if (qv[u] != 0.f || pv != 0.f) class_sums(qv[u], pv, st);
        }
      }
      for (int c = m2; c < m; ++c) {
        const float qv = __ldg(q + c), pv = myP[c];
        if (qv != 0.f || pv != 0.f) class_sums(qv, pv, st);
      }
    }
    const PixelTerm t = pixel_term(st, inside, log_k);
    s_keep[lp] = t.keep;
    if (t.keep) {
      term_sum = (double)t.value;
#pragma unroll 4
      for (int c = 0; c < m2; c += 4) {
        const float2 q0 = __ldg(reinterpret_cast<const float2 *>(q + c));
        const float2 q1 = __ldg(reinterpret_cast<const float2 *>(q + c + 2));
        const float qv[4] = {q0.x, q0.y, q1.x, q1.y};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float pv = myP[c + u];
          if (qv[u] != 0.f || pv != 0.f) myP[c + u] = class_grad(qv[u], pv, class_roots(qv[u], pv), t, inv_n);
        }
      }
      for (int c = m2; c < m; ++c) {
        const float qv = __ldg(q + c), pv = myP[c];
        if (qv != 0.f || pv != 0.f) myP[c] = class_grad(qv, pv, class_roots(qv, pv), t, inv_n);
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) term_sum += __shfl_xor_sync(0xffffffffu, term_sum, o);
  if (lane == 0) red[warp] = term_sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < WARPS; ++w) s += red[w];
    a.lpart[3 * (size_t)tile + 2] = s;
  }
  finish_loss<TW * TH>(a, 1, gridDim.x);

  // (3) d(objective)/d(weight l of Gaussian g) = sum_p w_gp dP_p[id_gl]:
  // lanes hold their pixel's products, a transposed warp sum leaves the
  // total of entry l on lane l (one or two contributing lanes add directly).
  // Pixels outside the entropy mask have a zero gradient row: they skip.
  const int nl = K > 0 ? K : k;
  walk(s_keep[lp] != 0, [&](int gid, bool on, float w, const int2 *e) {
    if (__popc(__ballot_sync(0xffffffffu, on)) <= 2) {
      // one or two lanes: their products go straight to the atomics
      if (on) {
#pragma unroll
        for (int l = 0; l < (K > 0 ? K : 16); ++l) {
          if (K == 0 && l >= nl) break;
          const int2 en = e[l * kBatch];
          const float v = (unsigned)en.x < (unsigned)m ? w * myP[en.x] : 0.f;
          if (v != 0.f) atomicAdd(a.semg + (size_t)gid * k + l, v);
        }
      }
      return;
    }
    if constexpr (K > 0 && K <= 4) {
      // few entries: K independent butterfly sums (5K shuffles) beat the
      // 16-slot transposed reduction
      float v[K];
#pragma unroll
      for (int l = 0; l < K; ++l) {
        const int2 en = e[l * kBatch];
        v[l] = (unsigned)en.x < (unsigned)m ? w * myP[en.x] : 0.f;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int l = 0; l < K; ++l) v[l] += __shfl_xor_sync(0xffffffffu, v[l], o);
      float tot = v[0];
#pragma unroll
      for (int l = 1; l < K; ++l)
        if ((int)lane == l) tot = v[l];
      if ((int)lane < K && tot != 0.f) atomicAdd(a.semg + (size_t)gid * k + lane, tot);
    } else {
      float v[16];
#pragma unroll
      for (int l = 0; l < 16; ++l) v[l] = 0.f;
#pragma unroll
      for (int l = 0; l < (K > 0 ? K : 16); ++l) {
        if (K == 0 && l >= nl) break;
        const int2 en = e[l * kBatch];
        if ((unsigned)en.x < (unsigned)m) v[l] = w * myP[en.x];
      }
      const float tot = warp_reduce_scatter<16>(v);
      if ((int)lane < nl && tot != 0.f) atomicAdd(a.semg + (size_t)gid * k + lane, tot);
    }
  });
}

__global__ void k_zero_f32(float *p, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    p[i] = 0.f;
}

// g[i] += (*scale) * src[i]
__global__ void k_add_scaled(float *g, const float *src, const float *scale, size_t n) {
  const float s = *scale;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float v = src[i];
    if (v != 0.f) g[i] = fmaf(s, v, g[i]);
  }
}

static unsigned elementwise_grid(size_t n) {
  const size_t b = (n + 255) / 256, cap = sm_grid(4);
  return (unsigned)(b < cap ? b : cap);
}

template <int TW, int TH, int K>
static cudaError_t launch_sem_objective(const FwdArgs &a, int grid, size_t smem, float log_k, float inv_n,
                                        cudaStream_t s) {
  {
    const cudaError_t e = ensure_smem_limit((const void *)k_sem_objective<TW, TH, K>, (int)kSmemBudget);
    if (e != cudaSuccess) return e;
  }
  k_sem_objective<TW, TH, K><<<grid, TW * TH, smem, s>>>(a, log_k, inv_n);
  return cudaGetLastError();
}

template <int TW, int TH>
static cudaError_t dispatch_sem_objective(const FwdArgs &a, int grid, size_t smem, float log_k, float inv_n,
                                          cudaStream_t s) {
  if (a.k == 3) return launch_sem_objective<TW, TH, 3>(a, grid, smem, log_k, inv_n, s);
  if (a.k == 8) return launch_sem_objective<TW, TH, 8>(a, grid, smem, log_k, inv_n, s);
  return launch_sem_objective<TW, TH, 0>(a, grid, smem, log_k, inv_n, s);
}

static void objective_chunks(int m, int npix, int k, int *mchunk, int *mstride, int *nchunks) {
  const size_t fixed = 2 * sem_batch_bytes(k), base = batch_smem_bytes(k);
  chunk_classes(m, npix, k, true, mchunk, mstride, nchunks, fixed > base ? fixed - base : 0);
}

bool objective_fits(const Layout &L, int k, int m) {
  if (!L.mask_units || L.npix <= 0 || k > 16) return false;
  int mchunk, mstride, nchunks;
  objective_chunks(m, L.tile_w * L.tile_h, k, &mchunk, &mstride, &nchunks);
  return nchunks == 1;
}

cudaError_t launch_render_fwd_objective(const Layout &L, const WsPtrs &P, int pbuf, const gs_scene &sc,
                                        const float *t_rgb, const float *t_depth, const float *t_sem, float *rgb,
                                        float *depth, float *sil, float *loss, cudaStream_t s) {
  FwdArgs a = fwd_args(L, P, pbuf, sc);
  const int tiles_y = (L.cam0_h + L.tile_h - 1) / L.tile_h;
  a.rgb_out = rgb; a.depth_out = depth; a.sil_out = sil; a.sem = nullptr;
  a.t_rgb = t_rgb; a.t_depth = t_depth; a.t_sem = t_sem;
  a.objective = 1;
  a.semg = P.semg;
  a.nwc = 0;  // codes hold the depth / colour word pair only
  const int npix = L.tile_w * L.tile_h;
  objective_chunks(sc.m, npix, sc.k, &a.mchunk, &a.mstride, &a.nchunks);
  if (a.nchunks != 1) return cudaErrorInvalidValue;
  const size_t smem = 2 * sem_batch_bytes(sc.k) + (size_t)npix * a.mstride * sizeof(float);
  const int grid = a.tiles_x * tiles_y;
  const size_t ng = (size_t)sc.n * sc.k;
  if (ng) {
    k_zero_f32<<<elementwise_grid(ng), 256, 0, s>>>(P.semg, ng);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (grid == 0) return cudaSuccess;
  cudaError_t e = launch_tile_batch_offsets(P.ranges, (uint32_t)grid, P.mask_off, P.counters, s);
  if (e != cudaSuccess) return e;
  e = launch_blend_objective(L, a, grid, s);
  if (e != cudaSuccess) return e;
  a.loss = loss;
  a.npix_d = (double)L.npix;
  if (t_sem) {
    const float log_k = logf((float)sc.k), inv_n = 1.f / (float)L.npix;
    if (L.tile_w == 16 && L.tile_h == 16) e = dispatch_sem_objective<16, 16>(a, grid, smem, log_k, inv_n, s);
    else if (L.tile_w == 16 && L.tile_h == 8) e = dispatch_sem_objective<16, 8>(a, grid, smem, log_k, inv_n, s);
    else if (L.tile_w == 8 && L.tile_h == 8) e = dispatch_sem_objective<8, 8>(a, grid, smem, log_k, inv_n, s);
    else if (L.tile_w == 32 && L.tile_h == 8) e = dispatch_sem_objective<32, 8>(a, grid, smem, log_k, inv_n, s);
    else e = cudaErrorInvalidConfiguration;
    return e;  // the semantic pass's last tile wrote the loss
  }
  return launch_loss_final(P.lpart, grid, (double)L.npix, (double)sc.m, 0, 1, loss, s);
}

cudaError_t launch_add_semg(const WsPtrs &P, const gs_scene &sc, const float *loss_scale, float *g_sem_w,
                            cudaStream_t s) {
  const size_t ng = (size_t)sc.n * sc.k;
  if (!g_sem_w || ng == 0) return cudaSuccess;
  k_add_scaled<<<elementwise_grid(ng), 256, 0, s>>>(g_sem_w, P.semg, loss_scale, ng);
  return cudaGetLastError();
}

}  // namespace gs
