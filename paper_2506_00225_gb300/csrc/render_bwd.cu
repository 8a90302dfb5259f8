// render_bwd.cu -- adjoint of the tile blend and of the projection.
//
// Sec. 3.1: the rendering is differentiable and the map is optimised end to
// end; Sec. 3.1 "Semantic Loss" (last paragraph) and Sec. 6: the semantic
// loss only updates semantic attributes (sem_detach_geometry).
//
// Per pixel, the contributors of Eq. 1 are revisited back to front starting
// from the last contributor recorded by the forward pass.  With
// w_i = alpha_i T_i and g_i = dL/dC . c_i + dL/dD d_i + dL/dS
// (+ sum_l dL/dP[id_il] p_il when semantics reach geometry):
//   dL/dc_i = dL/dC w_i,  dL/dd_i = dL/dD w_i,  dL/dp_il = dL/dP[id_il] w_i,
//   dL/dalpha_i = T_i g_i - (sum_{j>i} w_j g_j) / (1 - alpha_i),
// and T_i = T_{i+1} / (1 - alpha_i) is recovered from the stored final
// transmittance, so no per-pixel lists are kept.  alpha = o exp(power) below
// the 0.99 cap passes its gradient to opacity, the conic and the 2D mean.
// Per-Gaussian sums over the pixels of a warp are shuffle-reduced before one
// atomic per warp; a second kernel chains the 2D gradients through the
// projection to means, scales and quaternions.
#include "gs_internal.cuh"
#include "render_common.cuh"

namespace gs {

struct BwdArgs {
  const uint2 *ranges;
  const uint32_t *pvals;
  RecPtrs rec;
  int k, m, width, height, tiles_x;
  const float *tfinal;
  const uint32_t *nlast;
  const float *d_rgb, *d_depth, *d_sil, *d_sem;
  int sem_detach;
  const Counters *counters;
  float4 *grad2d;
  float *g_rgb, *g_sem_w;
  // fused mean-L1 mode: upstream gradients decoded from sign codes
  const uint32_t *codes;
  int nwc;
  const float *loss_scale;  // device dL/dloss
  int objective;            // Sec. 3.1 objective: 0.5 / 1 weights of colour / depth sums, no class codes
  double npix;
  const uint32_t *mask_off;  // contributor bitmasks of the forward pass
  const uint32_t *masks;
};

__device__ __forceinline__ float sign_code(uint32_t nz, uint32_t ng, int bit, float s) {
  return ((nz >> bit) & 1u) ? (((ng >> bit) & 1u) ? -s : s) : 0.f;
}

// Per contributing (pixel, Gaussian) the thread forms NV values
//   0..6  du, dv, da, db, dc, dopacity, ddepth   (2D gradients of the record)
//   7..9  drgb                                   (colour of the Gaussian)
//   10..  dsem_w (k values)
// which a transposed warp reduction sums over the warp's 32 pixels; each lane
// then adds one of the totals with a single scalar atomic.
// K > 0 fixes the top-k count at compile time (exact unrolling of the
// per-class terms); the reduction width follows: 16 values for K <= 6,
// else 32.
template <int TW, int TH, bool CODES, int K, int PPT>
__global__ void __launch_bounds__(TW *TH / PPT) k_render_bwd(BwdArgs a) {
  constexpr int NV = (K > 0 && K <= 6) ? 16 : 32;
  constexpr int NL = K > 0 ? K : NV - 10;  // per-class value slots walked
  using FP = Footprint<TW, TH, PPT>;
  extern __shared__ float4 smem4[];
  BatchSmem bs = batch_smem(smem4, a.k);
  __shared__ uint32_t s_maxnl;
  if (a.counters->status & kStatusTimeout) return;  // the binning is incomplete

  const int tile = blockIdx.x;
  const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
  const int ox = tx * TW, oy = ty * TH;
  const uint2 rg = a.ranges[tile];
  const int lx = FP::lx();
  const int px = ox + lx;
  const float fpx = (float)px + 0.5f;
  const int k = a.k;
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
  // warp-uniform: every lane takes the same branches around the shuffles
  const bool has_dsem = (CODES && !a.objective) || a.d_sem != nullptr;
  float s_sem = 0.f;

  int py[PPT];
  float fpy[PPT], T[PPT], acc[PPT], dR[PPT], dG[PPT], dB[PPT], dD[PPT], dS[PPT];
  uint32_t nl[PPT];
  const float *dP[PPT];
  uint2 *myc[PPT];  // CODES: this pixel's (nonzero, negative) class sign word pairs (odd stride)
  uint32_t my_max = 0;
#pragma unroll
  for (int i = 0; i < PPT; ++i) {
    const int ly = FP::ly(i);
    py[i] = oy + ly;
    fpy[i] = (float)py[i] + 0.5f;
    T[i] = 1.f; acc[i] = 0.f; dR[i] = dG[i] = dB[i] = dD[i] = dS[i] = 0.f;
    nl[i] = 0;
    dP[i] = nullptr;
    myc[i] = reinterpret_cast<uint2 *>(bs.tail) + (ly * TW + lx) * (a.nwc | 1);
    if (px < a.width && py[i] < a.height) {
      const size_t pix = (size_t)py[i] * a.width + px;
      T[i] = a.tfinal[pix];
      nl[i] = a.nlast[pix];
      if (CODES) {
        const float ls = *a.loss_scale;
        const float s_rgb = a.objective ? 0.5f * ls : (float)(ls / (3.0 * a.npix));
        const float s_d = a.objective ? ls : (float)(ls / a.npix);
        s_sem = (float)(ls / (a.npix * a.m));
        const uint2 *cp = reinterpret_cast<const uint2 *>(a.codes + pix * code_words(a.nwc));
        const uint32_t nz = cp[0].x, ng = cp[0].y;
        dR[i] = sign_code(nz, ng, 0, s_rgb); dG[i] = sign_code(nz, ng, 1, s_rgb); dB[i] = sign_code(nz, ng, 2, s_rgb);
        dD[i] = sign_code(nz, ng, 3, s_d);
        for (int wd = 0; wd < a.nwc; ++wd) myc[i][wd] = cp[1 + wd];
      } else {
        if (a.d_rgb) { dR[i] = a.d_rgb[3 * pix]; dG[i] = a.d_rgb[3 * pix + 1]; dB[i] = a.d_rgb[3 * pix + 2]; }
        if (a.d_depth) dD[i] = a.d_depth[pix];
        if (a.d_sil) dS[i] = a.d_sil[pix];
        if (a.d_sem) dP[i] = a.d_sem + pix * a.m;
      }
      my_max = max(my_max, nl[i]);
    }
  }
  if (threadIdx.x == 0) s_maxnl = 0;
  __syncthreads();
  if (my_max) atomicMax(&s_maxnl, my_max);
  __syncthreads();
  const uint32_t maxnl = s_maxnl;
  const int my_idx = reduced_index<NV>();

  // the forward's batches, last to first (batch bi covers rg.x + 64 bi ...)
  for (int bi = maxnl ? (int)((maxnl - 1) / kBatch) : -1; bi >= 0; --bi) {
    const uint32_t lo = rg.x + (uint32_t)bi * kBatch;
    const int n = (int)min((uint32_t)kBatch, rg.y - lo);
    __syncthreads();
    for (int t = threadIdx.x; t < n; t += FP::kThreads)
      stage_record<TW, TH, PPT>(a.rec, a.pvals[lo + t], t, k, ox, oy, bs, has_dsem, false);
    __syncthreads();
    // contributor bits of this batch: written by the forward pass 1, or
    // re-tested (pairs up to the last contributor whose pixel box holds the
    // pixel and whose alpha passes 1/255)
    uint32_t mb[PPT][2];
    if (a.masks) {
      const uint32_t unit = a.mask_off[tile] + (uint32_t)bi;
      const uint32_t *mw = a.masks + (size_t)unit * 2 * FP::kPix;
#pragma unroll
      for (int i = 0; i < PPT; ++i) {
        const int lp = FP::ly(i) * TW + lx;
        const bool ok = px < a.width && py[i] < a.height;
        mb[i][0] = ok ? mw[lp] : 0u;
        mb[i][1] = ok ? mw[FP::kPix + lp] : 0u;
      }
    } else {
#pragma unroll
      for (int i = 0; i < PPT; ++i) {
        mb[i][0] = mb[i][1] = 0u;
        const uint32_t b0 = (uint32_t)bi * kBatch;
        const int nj = nl[i] > b0 ? min(n, (int)(nl[i] - b0)) : 0;
        for (int j = 0; j < nj; ++j) {
          if (!((bs.wmask[j] >> warp) & 1u) || !box_holds(bs.box[j], px, py[i])) continue;
          float al, G_, ar, dx_, dy_;
          if (gauss_alpha(bs.uv[j], bs.co[j], fpx, fpy[i], al, G_, ar, dx_, dy_)) mb[i][j >> 5] |= 1u << (j & 31);
        }
      }
    }
    for (int h = 1; h >= 0; --h) {
      uint32_t mine = 0u;
#pragma unroll
      for (int i = 0; i < PPT; ++i) mine |= mb[i][h];
      uint32_t vis = __reduce_or_sync(0xffffffffu, mine);
      while (vis) {
        const int bit = 31 - __clz(vis);
        vis &= ~(1u << bit);
        const int j = h * 32 + bit;
        const float2 uv = bs.uv[j];
        const float4 co = bs.co[j];
        bool contrib[PPT];
        float alpha[PPT], G[PPT], araw[PPT], dx[PPT], dy[PPT];
        bool any = false;
#pragma unroll
        for (int i = 0; i < PPT; ++i) {
          contrib[i] = (mb[i][h] >> bit) & 1u;
          if (contrib[i]) gauss_alpha(uv, co, fpx, fpy[i], alpha[i], G[i], araw[i], dx[i], dy[i]);
          any = any || contrib[i];
        }
        float v[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) v[q] = 0.f;
        const float4 cdp = bs.cd[j];
        const int2 *sp = bs.sem + j * k;
#pragma unroll
        for (int i = 0; i < PPT; ++i) {
          if (!contrib[i]) continue;
          const float om = 1.f - alpha[i];
          const float inv_om = __fdividef(1.f, om);  // approximate: 2 ulp, well inside the gradient bar
          const float Ti = T[i] * inv_om;
          const float w = alpha[i] * Ti;
          float gi = dR[i] * cdp.x + dG[i] * cdp.y + dB[i] * cdp.z + dD[i] * cdp.w + dS[i];
          if (has_dsem) {
            float gs = 0.f;
#pragma unroll
            for (int l = 0; l < NL; ++l) {
              if (K > 0 || l < k) {
                const int2 e = sp[l];
                float dp = 0.f;
                if ((unsigned)e.x < (unsigned)a.m) {
                  if (CODES) {
                    const uint2 cw = myc[i][e.x >> 5];
                    dp = sign_code(cw.x, cw.y, e.x & 31, s_sem);
                  } else {
                    dp = __ldg(dP[i] + e.x);
                  }
                }
                v[10 + l] = fmaf(dp, w, v[10 + l]);
                gs = fmaf(dp, __int_as_float(e.y), gs);
              }
            }
            if (!a.sem_detach) gi += gs;
          }
          v[7] = fmaf(dR[i], w, v[7]); v[8] = fmaf(dG[i], w, v[8]); v[9] = fmaf(dB[i], w, v[9]);
          v[6] = fmaf(dD[i], w, v[6]);
          const float dalpha = Ti * gi - acc[i] * inv_om;
          acc[i] = fmaf(w, gi, acc[i]);
          T[i] = Ti;
          if (araw[i] < kAlphaMax) {
            v[5] = fmaf(dalpha, G[i], v[5]);
            const float dpow = dalpha * araw[i];
            const float ddx = dx[i], ddy = dy[i];
            v[2] = fmaf(dpow, -0.5f * ddx * ddx, v[2]);
            v[3] = fmaf(dpow, -ddx * ddy, v[3]);
            v[4] = fmaf(dpow, -0.5f * ddy * ddy, v[4]);
            v[0] = fmaf(dpow, -(co.x * ddx + co.y * ddy), v[0]);
            v[1] = fmaf(dpow, -(co.z * ddy + co.y * ddx), v[1]);
          }
        }
        if (NV == 32 && __popc(__ballot_sync(0xffffffffu, any)) <= 2) {
          // with the wide (32-value) reduction, one or two lanes touched by
          // this Gaussian add their values directly
          if (any) {
            float *g2 = reinterpret_cast<float *>(a.grad2d) + 8 * (size_t)bs.rec[j];
#pragma unroll
            for (int q = 0; q < 7; ++q)
              if (v[q] != 0.f) atomicAdd(g2 + q, v[q]);
            if (a.g_rgb) {
              float *gr = a.g_rgb + 3 * (size_t)bs.gid[j];
#pragma unroll
              for (int q = 0; q < 3; ++q)
                if (v[7 + q] != 0.f) atomicAdd(gr + q, v[7 + q]);
            }
            if (has_dsem && a.g_sem_w) {
              float *gw = a.g_sem_w + (size_t)bs.gid[j] * k;
#pragma unroll
              for (int l = 0; l < NL; ++l)
                if ((K > 0 || l < k) && v[10 + l] != 0.f) atomicAdd(gw + l, v[10 + l]);
            }
          }
          continue;
        }
        const float tot = warp_reduce_scatter<NV>(v);
        if (my_idx == (int)lane || NV == 32) {
          // lanes 0..15 (NV = 16) or all lanes (NV = 32) own one value each
          if (my_idx < 7) {
            if (tot != 0.f) atomicAdd(reinterpret_cast<float *>(a.grad2d) + 8 * (size_t)bs.rec[j] + my_idx, tot);
          } else if (my_idx < 10) {
            if (a.g_rgb && tot != 0.f) atomicAdd(a.g_rgb + 3 * (size_t)bs.gid[j] + (my_idx - 7), tot);
          } else if (my_idx < 10 + k) {
            if (has_dsem && a.g_sem_w && tot != 0.f) atomicAdd(a.g_sem_w + (size_t)bs.gid[j] * k + (my_idx - 10), tot);
          }
        }
      }
    }
  }
}

__global__ void k_zero_grad2d(float4 *g, const Counters *cnt, uint32_t rcap) {
  const uint32_t n = 2 * min(cnt->n_records, rcap);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    g[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

template <int TW, int TH, bool CODES, int K, int PPT>
static cudaError_t launch_bwd_shape(const BwdArgs &a, int grid, size_t smem, cudaStream_t s) {
  {  // the sign words of large class counts need more than 48 KB
    const cudaError_t e = ensure_smem_limit((const void *)k_render_bwd<TW, TH, CODES, K, PPT>, (int)kSmemBudget);
    if (e != cudaSuccess) return e;
  }
  k_render_bwd<TW, TH, CODES, K, PPT><<<grid, TW * TH / PPT, smem, s>>>(a);
  return cudaGetLastError();
}

template <bool CODES, int K, int PPT>
static cudaError_t dispatch_bwd_shape(int tw, int th, const BwdArgs &a, int grid, size_t smem, cudaStream_t s) {
  if (tw == 16 && th == 16) return launch_bwd_shape<16, 16, CODES, K, PPT>(a, grid, smem, s);
  if (tw == 16 && th == 8) return launch_bwd_shape<16, 8, CODES, K, PPT>(a, grid, smem, s);
  if (tw == 8 && th == 8) return launch_bwd_shape<8, 8, CODES, K, PPT>(a, grid, smem, s);
  if (tw == 32 && th == 8) return launch_bwd_shape<32, 8, CODES, K, PPT>(a, grid, smem, s);
  return cudaErrorInvalidConfiguration;
}

template <bool CODES>
static cudaError_t dispatch_bwd(const Layout &L, const BwdArgs &a, int grid, size_t smem, cudaStream_t s) {
  if (L.ppt == 4) {
    if (L.tile_w != 16 || L.tile_h != 16) return cudaErrorInvalidConfiguration;
    if (a.k == 3) return launch_bwd_shape<16, 16, CODES, 3, 4>(a, grid, smem, s);
    if (a.k == 8) return launch_bwd_shape<16, 16, CODES, 8, 4>(a, grid, smem, s);
    return launch_bwd_shape<16, 16, CODES, 0, 4>(a, grid, smem, s);
  }
  if (L.ppt == 2) {
    if (a.k == 3) return dispatch_bwd_shape<CODES, 3, 2>(L.tile_w, L.tile_h, a, grid, smem, s);
    if (a.k == 8) return dispatch_bwd_shape<CODES, 8, 2>(L.tile_w, L.tile_h, a, grid, smem, s);
    return dispatch_bwd_shape<CODES, 0, 2>(L.tile_w, L.tile_h, a, grid, smem, s);
  }
  if (a.k == 3) return dispatch_bwd_shape<CODES, 3, 1>(L.tile_w, L.tile_h, a, grid, smem, s);
  if (a.k == 8) return dispatch_bwd_shape<CODES, 8, 1>(L.tile_w, L.tile_h, a, grid, smem, s);
  return dispatch_bwd_shape<CODES, 0, 1>(L.tile_w, L.tile_h, a, grid, smem, s);
}

cudaError_t launch_render_bwd(const Layout &L, const WsPtrs &P, int pbuf, const gs_scene &sc, const float *d_rgb,
                              const float *d_depth, const float *d_sil, const float *d_sem, int sem_detach,
                              float *g_rgb, float *g_sem_w, cudaStream_t s, const float *loss_scale,
                              int objective) {
  k_zero_grad2d<<<sm_grid(2), 256, 0, s>>>(P.grad2d, P.counters, (uint32_t)L.rcap);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  BwdArgs a{};
  a.ranges = P.ranges;
  a.pvals = P.pvals[pbuf];
  a.rec = rec_ptrs(P);
  a.k = sc.k; a.m = sc.m;
  a.width = L.cam0_w; a.height = L.cam0_h;
  a.tiles_x = (L.cam0_w + L.tile_w - 1) / L.tile_w;
  const int tiles_y = (L.cam0_h + L.tile_h - 1) / L.tile_h;
  a.tfinal = P.tfinal; a.nlast = P.nlast;
  a.d_rgb = d_rgb; a.d_depth = d_depth; a.d_sil = d_sil; a.d_sem = d_sem;
  a.sem_detach = sem_detach;
  a.counters = P.counters;
  a.grad2d = P.grad2d;
  a.g_rgb = g_rgb; a.g_sem_w = g_sem_w;
  a.mask_off = L.mask_units ? P.mask_off : nullptr;
  a.masks = L.mask_units ? P.masks : nullptr;
  const int grid = a.tiles_x * tiles_y;
  if (grid == 0) return cudaSuccess;
  if (loss_scale) {
    a.codes = P.codes;
    a.nwc = objective ? 0 : L.nwc;
    a.loss_scale = loss_scale;
    a.npix = (double)L.npix;
    a.objective = objective;
    const size_t smem = batch_smem_bytes(sc.k) + (size_t)L.tile_w * L.tile_h * (a.nwc | 1) * 8;
    return dispatch_bwd<true>(L, a, grid, smem, s);
  }
  const size_t smem = batch_smem_bytes(sc.k);
  return dispatch_bwd<false>(L, a, grid, smem, s);
}

// ---------------------------------------------------------------------------
// Projection adjoint: (du, dv, dconic, ddepth) of each record -> means,
// linear scales, quaternions; dopacity -> opacity.
// ---------------------------------------------------------------------------
__global__ void k_project_bwd(gs_scene sc, const DevCam *cams, const int32_t *__restrict__ rgid,
                              const int32_t *__restrict__ rview, const float4 *__restrict__ grad2d,
                              const Counters *cnt, uint32_t rcap, float *g_means, float *g_scales, float *g_quats,
                              float *g_opacity) {
  const uint32_t count = min(cnt->n_records, rcap);
  const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= count) return;
  const int g = rgid[r];
  const DevCam c = cams[rview[r]];
  const float4 ga = grad2d[2 * (size_t)r], gb = grad2d[2 * (size_t)r + 1];
  const float du = ga.x, dv = ga.y, dca = ga.z, dcb = ga.w, dcc = gb.x, dop = gb.y, dz = gb.z;
  const float m0 = sc.means[3 * g], m1 = sc.means[3 * g + 1], m2 = sc.means[3 * g + 2];
  const float s[3] = {sc.scales[3 * g], sc.scales[3 * g + 1], sc.scales[3 * g + 2]};
  const float4 q = reinterpret_cast<const float4 *>(sc.quats)[g];
  const float *V = c.r;
  const float tx = V[0] * m0 + V[1] * m1 + V[2] * m2 + c.t[0];
  const float ty = V[3] * m0 + V[4] * m1 + V[5] * m2 + c.t[1];
  const float tz = V[6] * m0 + V[7] * m1 + V[8] * m2 + c.t[2];
  const float qn = sqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
  const float w = q.x / qn, x = q.y / qn, y = q.z / qn, z = q.w / qn;
  float R[9];
  R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z); R[2] = 2.f * (x * z + w * y);
  R[3] = 2.f * (x * y + w * z); R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
  R[6] = 2.f * (x * z - w * y); R[7] = 2.f * (y * z + w * x); R[8] = 1.f - 2.f * (x * x + y * y);
  float Mq[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) Mq[i * 3 + j] = R[i * 3 + j] * s[j];
  float S[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) S[i * 3 + j] = Mq[i * 3] * Mq[j * 3] + Mq[i * 3 + 1] * Mq[j * 3 + 1] + Mq[i * 3 + 2] * Mq[j * 3 + 2];
  const float limx = 1.3f * ((0.5f * (float)c.width) / c.fx);
  const float limy = 1.3f * ((0.5f * (float)c.height) / c.fy);
  const float rx = tx / tz, ry = ty / tz;
  const bool clx = rx < -limx || rx > limx, cly = ry < -limy || ry > limy;
  const float rxc = fminf(limx, fmaxf(-limx, rx)), ryc = fminf(limy, fmaxf(-limy, ry));
  const float tz2 = tz * tz, tz3 = tz2 * tz;
  const float J00 = c.fx / tz, J02 = -(c.fx * rxc * tz) / tz2;
  const float J11 = c.fy / tz, J12 = -(c.fy * ryc * tz) / tz2;
  float T[6];
  for (int j = 0; j < 3; ++j) {
    T[j] = J00 * V[j] + J02 * V[6 + j];
    T[3 + j] = J11 * V[3 + j] + J12 * V[6 + j];
  }
  float U[6];
  for (int a = 0; a < 2; ++a)
    for (int j = 0; j < 3; ++j) U[a * 3 + j] = T[a * 3] * S[j] + T[a * 3 + 1] * S[3 + j] + T[a * 3 + 2] * S[6 + j];
  const float A = U[0] * T[0] + U[1] * T[1] + U[2] * T[2] + 0.3f;
  const float B = U[0] * T[3] + U[1] * T[4] + U[2] * T[5];
  const float C = U[3] * T[3] + U[4] * T[4] + U[5] * T[5] + 0.3f;
  const float det = A * C - B * B;
  const float inv = 1.f / det, inv2 = inv * inv;
  // conic = inverse of [[A, B], [B, C]]
  const float dinv = dca * C - dcb * B + dcc * A;
  const float dA = dcc * inv - dinv * C * inv2;
  const float dB = -dcb * inv + 2.f * dinv * B * inv2;
  const float dC = dca * inv - dinv * A * inv2;
  // Sigma2 = T S T^T
  float ST0[3], ST1[3];
  for (int i = 0; i < 3; ++i) {
    ST0[i] = S[i * 3] * T[0] + S[i * 3 + 1] * T[1] + S[i * 3 + 2] * T[2];
    ST1[i] = S[i * 3] * T[3] + S[i * 3 + 1] * T[4] + S[i * 3 + 2] * T[5];
  }
  float dT[6];
  for (int i = 0; i < 3; ++i) {
    dT[i] = 2.f * dA * ST0[i] + dB * ST1[i];
    dT[3 + i] = 2.f * dC * ST1[i] + dB * ST0[i];
  }
  // dL/dS (full) -> dL/dM = (G + G^T) M for S = M M^T
  float Gm[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      Gm[i * 3 + j] = dA * T[i] * T[j] + dB * T[i] * T[3 + j] + dC * T[3 + i] * T[3 + j];
  float gs[3] = {0.f, 0.f, 0.f}, dR[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      float acc = 0.f;
      for (int l = 0; l < 3; ++l) acc += (Gm[i * 3 + l] + Gm[l * 3 + i]) * Mq[l * 3 + j];
      gs[j] += acc * R[i * 3 + j];
      dR[i * 3 + j] = acc * s[j];
    }
  const float dw = 2.f * (-z * dR[1] + y * dR[2] + z * dR[3] - x * dR[5] - y * dR[6] + x * dR[7]);
  const float dx = 2.f * (y * dR[1] + z * dR[2] + y * dR[3] - 2.f * x * dR[4] - w * dR[5] + z * dR[6] + w * dR[7] -
                          2.f * x * dR[8]);
  const float dy = 2.f * (-2.f * y * dR[0] + x * dR[1] + w * dR[2] + x * dR[3] + z * dR[5] - w * dR[6] + z * dR[7] -
                          2.f * y * dR[8]);
  const float dzq = 2.f * (-2.f * z * dR[0] - w * dR[1] + x * dR[2] + w * dR[3] - 2.f * z * dR[4] + y * dR[5] +
                           x * dR[6] + y * dR[7]);
  const float dot = w * dw + x * dx + y * dy + z * dzq;
  // T = J W
  const float dJ00 = dT[0] * V[0] + dT[1] * V[1] + dT[2] * V[2];
  const float dJ02 = dT[0] * V[6] + dT[1] * V[7] + dT[2] * V[8];
  const float dJ11 = dT[3] * V[3] + dT[4] * V[4] + dT[5] * V[5];
  const float dJ12 = dT[3] * V[6] + dT[4] * V[7] + dT[5] * V[8];
  float dtx = 0.f, dty = 0.f, dtz = dz;
  dtz += dJ00 * (-c.fx / tz2) + dJ11 * (-c.fy / tz2);
  if (!clx) { dtx += dJ02 * (-c.fx / tz2); dtz += dJ02 * (2.f * c.fx * tx / tz3); }
  else { dtz += dJ02 * (c.fx * rxc / tz2); }
  if (!cly) { dty += dJ12 * (-c.fy / tz2); dtz += dJ12 * (2.f * c.fy * ty / tz3); }
  else { dtz += dJ12 * (c.fy * ryc / tz2); }
  dtx += du * c.fx / tz;
  dty += dv * c.fy / tz;
  dtz += -du * c.fx * tx / tz2 - dv * c.fy * ty / tz2;
  // t = R m + t_c; one record per Gaussian for a single view, but keep the
  // update atomic so several views can accumulate into the same gradients.
  atomicAdd(g_means + 3 * g, V[0] * dtx + V[3] * dty + V[6] * dtz);
  atomicAdd(g_means + 3 * g + 1, V[1] * dtx + V[4] * dty + V[7] * dtz);
  atomicAdd(g_means + 3 * g + 2, V[2] * dtx + V[5] * dty + V[8] * dtz);
  for (int j = 0; j < 3; ++j) atomicAdd(g_scales + 3 * g + j, gs[j]);
  atomicAdd(g_quats + 4 * g, (dw - w * dot) / qn);
  atomicAdd(g_quats + 4 * g + 1, (dx - x * dot) / qn);
  atomicAdd(g_quats + 4 * g + 2, (dy - y * dot) / qn);
  atomicAdd(g_quats + 4 * g + 3, (dzq - z * dot) / qn);
  atomicAdd(g_opacity + g, dop);
}

cudaError_t launch_project_bwd(const Layout &L, const WsPtrs &P, const gs_scene &sc, float *g_means,
                               float *g_scales, float *g_quats, float *g_opacity, cudaStream_t s) {
  const uint32_t grid = (uint32_t)((L.rcap + 255) / 256);
  if (grid == 0) return cudaSuccess;
  k_project_bwd<<<grid, 256, 0, s>>>(sc, P.cams, P.rec_gid, P.rec_view, P.grad2d, P.counters, (uint32_t)L.rcap,
                                     g_means, g_scales, g_quats, g_opacity);
  return cudaGetLastError();
}

}  // namespace gs
