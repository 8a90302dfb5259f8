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
  int warp_bytes;            // shared memory of one warp: staging slots + reduction rows
};

__device__ __forceinline__ float sign_code(uint32_t nz, uint32_t ng, int bit, float s) {
  return ((nz >> bit) & 1u) ? (((ng >> bit) & 1u) ? -s : s) : 0.f;
}

// +w, -w or 0 for the class bit at left shift sh = 31 - bit of a (nonzero,
// negative) sign-code word pair: all-ones / zero mask from the nonzero bit,
// sign from the negative bit (a zero code may come out as -0.0, which adds
// nothing).
__device__ __forceinline__ float signed_weight(uint2 cw, uint32_t sh, float w) {
  const uint32_t nzm = (uint32_t)((int32_t)(cw.x << sh) >> 31);
  const uint32_t sg = (cw.y << sh) & 0x80000000u;
  return __uint_as_float((__float_as_uint(w) & nzm) ^ sg);
}

// Per warp, the staged Gaussians of one half batch (32 pairs): the records
// the warp's pixels visit, in pair order (mask mode: only the visited ones,
// packed; recomputation: all of them, slot = position in the half), with
// the base addresses of their gradient entries.
constexpr int kSlots = 32;
constexpr int kRedStride = 36;  // reduction row stride (floats): 16-byte rows, conflict-free reads and writes

__host__ __device__ inline size_t warp_stage_bytes(int k) {
  return (size_t)kSlots * (16 + 16 + 8 + 8 + 24 + 8 * k);
}

__host__ __device__ inline size_t bwd_warp_bytes(int k) {
  return (warp_stage_bytes(k) + (size_t)(10 + k) * kRedStride * 4 + 15) & ~(size_t)15;
}

struct WarpStage {
  float4 *co, *cd;   // conic + opacity; colour + depth
  float2 *uv;
  short4 *box;       // alpha box (recomputation mode)
  float **dst;       // [slot][3]: 2D gradients of the record, colour and class-weight gradients of the Gaussian
  int2 *sem;         // [k][slot] (class id, weight bits)
};

__device__ __forceinline__ WarpStage warp_stage(char *p, int k) {
  WarpStage w;
  w.co = reinterpret_cast<float4 *>(p); p += kSlots * 16;
  w.cd = reinterpret_cast<float4 *>(p); p += kSlots * 16;
  w.uv = reinterpret_cast<float2 *>(p); p += kSlots * 8;
  w.box = reinterpret_cast<short4 *>(p); p += kSlots * 8;
  w.dst = reinterpret_cast<float **>(p); p += kSlots * 24;
  w.sem = reinterpret_cast<int2 *>(p);
  return w;
}

// The adjoint of the tile blend, one CTA per tile.  Every warp owns an
// 8 x (4 PPT) pixel block and works through the tile's pairs on its own
// (no CTA barrier after the set-up): half batch by half batch, last to
// first, it stages the Gaussians its pixels' contributor bits name, then
// walks them back to front.  Per visited Gaussian every lane evaluates its
// PPT pixels without branches (a pixel the Gaussian did not reach adds
// exact zeros), forming
//   0, 1   sum dpow dx, sum dpow dy   (-> du, dv with the conic)
//   2..4   sum dpow dx dx, dx dy, dy dy (-> the conic gradient)
//   5      dopacity,  6  ddepth,  7..9  drgb,  10..  dsem_w (k values)
// with dpow = dalpha o G; the warp sums them through a transposed
// shared-memory exchange (each lane writes its values as a column, a lane
// per value reads its row back) and one lane per value adds the warp total
// with a single atomic.  SEMG: the semantic upstream gradient also reaches
// the geometry (sem_detach_geometry = 0).  K > 0 fixes the top-k count.
template <int TW, int TH, bool CODES, int K, int PPT, bool SEMG>
__global__ void __launch_bounds__(TW *TH / PPT) k_render_bwd(BwdArgs a) {
  constexpr int NVMAX = 10 + (K > 0 ? K : kMaxK);
  constexpr int KMAX = K > 0 ? K : kMaxK;
  using FP = Footprint<TW, TH, PPT>;
  constexpr int THREADS = FP::kThreads;
  constexpr int NPIX = FP::kPix;
  extern __shared__ float4 smem4[];
  if (a.counters->status & kStatusTimeout) return;  // the binning is incomplete

  const int k = K > 0 ? K : a.k;
  const int nv = 10 + k;
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
  char *wbase = reinterpret_cast<char *>(smem4) + (size_t)warp * a.warp_bytes;
  const WarpStage st = warp_stage(wbase, k);
  float *red = reinterpret_cast<float *>(wbase + warp_stage_bytes(k));
  // this thread's class sign words, [word][pixel i][thread] (conflict-free);
  // word nwc is zero (invalid class ids point there)
  uint2 *mycodes = reinterpret_cast<uint2 *>(reinterpret_cast<char *>(smem4) + (size_t)FP::kWarps * a.warp_bytes) +
                   threadIdx.x;

  const int tile = blockIdx.x;
  const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
  const int ox = tx * TW, oy = ty * TH;
  const uint2 rg = a.ranges[tile];
  const int lx = FP::lx();
  const int px = ox + lx;
  const float fpx = (float)px + 0.5f;
  // warp-uniform: every lane takes the same branches around the exchanges
  const bool has_dsem = (CODES && !a.objective) || a.d_sem != nullptr;
  const bool recompute = a.masks == nullptr;
  // fused-loss scales of the decoded signs (the class entries are scaled by
  // the lane that issues their atomic)
  float s_rgb = 0.f, s_d = 0.f, s_sem = 1.f;
  if (CODES) {
    const float ls = *a.loss_scale;
    s_rgb = a.objective ? 0.5f * ls : (float)(ls / (3.0 * a.npix));
    s_d = a.objective ? ls : (float)(ls / a.npix);
    s_sem = (float)(ls / (a.npix * a.m));
  }

  int py[PPT], lp[PPT];
  float fpy[PPT], T[PPT], acc[PPT], dR[PPT], dG[PPT], dB[PPT], dD[PPT], dS[PPT];
  uint32_t nl[PPT];
  const float *dP[PPT];
  bool ok[PPT];
  uint32_t my_max = 0;
#pragma unroll
  for (int i = 0; i < PPT; ++i) {
    const int ly = FP::ly(i);
    py[i] = oy + ly;
    lp[i] = ly * TW + lx;
    fpy[i] = (float)py[i] + 0.5f;
    T[i] = 1.f; acc[i] = 0.f; dR[i] = dG[i] = dB[i] = dD[i] = dS[i] = 0.f;
    nl[i] = 0;
    dP[i] = a.d_sem;
    ok[i] = px < a.width && py[i] < a.height;
    if (CODES && has_dsem) mycodes[(a.nwc * PPT + i) * THREADS] = make_uint2(0u, 0u);
    if (ok[i]) {
      const size_t pix = (size_t)py[i] * a.width + px;
      T[i] = a.tfinal[pix];
      nl[i] = a.nlast[pix];
      if (CODES) {
        const uint2 *cp = reinterpret_cast<const uint2 *>(a.codes + pix * code_words(a.nwc));
        const uint32_t nz = cp[0].x, ng = cp[0].y;
        dR[i] = sign_code(nz, ng, 0, s_rgb); dG[i] = sign_code(nz, ng, 1, s_rgb); dB[i] = sign_code(nz, ng, 2, s_rgb);
        dD[i] = sign_code(nz, ng, 3, s_d);
        for (int wd = 0; wd < a.nwc; ++wd) mycodes[(wd * PPT + i) * THREADS] = cp[1 + wd];
      } else {
        if (a.d_rgb) { dR[i] = a.d_rgb[3 * pix]; dG[i] = a.d_rgb[3 * pix + 1]; dB[i] = a.d_rgb[3 * pix + 2]; }
        if (a.d_depth) dD[i] = a.d_depth[pix];
        if (a.d_sil) dS[i] = a.d_sil[pix];
        if (a.d_sem) dP[i] = a.d_sem + pix * a.m;
      }
      my_max = max(my_max, nl[i]);
    }
  }
  // the warp's last contributor bounds its walk
  const uint32_t wmax = __reduce_max_sync(0xffffffffu, my_max);
  const uint32_t unit0 = recompute ? 0u : a.mask_off[tile];
  // value q of this lane after the exchange (lane = q + 16 h for up to 16
  // values, else lane = q) and its constant part of the final scaling
  const bool narrow = NVMAX <= 16 || nv <= 16;
  const int q = narrow ? (int)(lane & 15) : (int)lane;
  const bool issue = narrow ? (lane < 16 && q < nv) : q < nv;
  const int q_cls = q < 7 ? 0 : (q < 10 ? 1 : 2);
  const int q_off = q < 7 ? q : (q < 10 ? q - 7 : q - 10);
  const float q_scale = (q == 2 || q == 4) ? -0.5f : (q == 3 ? -1.f : (q >= 10 ? (CODES ? s_sem : 1.f) : 1.f));

  auto stage = [&](uint32_t r, int slot, bool use_box) {
    st.uv[slot] = __ldg(a.rec.uv + r);
    st.co[slot] = __ldg(a.rec.co + r);
    st.cd[slot] = __ldg(a.rec.cd + r);
    if (use_box) st.box[slot] = __ldg(a.rec.box + r);
    const int gid = __ldg(a.rec.gid + r);
    st.dst[3 * slot] = reinterpret_cast<float *>(a.grad2d) + 8 * (size_t)r;
    st.dst[3 * slot + 1] = a.g_rgb ? a.g_rgb + 3 * (size_t)gid : nullptr;
    st.dst[3 * slot + 2] = (has_dsem && a.g_sem_w) ? a.g_sem_w + (size_t)gid * k : nullptr;
    if (has_dsem) {
      const int2 *src = a.rec.sem + (size_t)r * k;
      for (int l = 0; l < k; ++l) st.sem[l * kSlots + slot] = __ldg(src + l);  // lanes: consecutive slots
    }
  };

  for (int bi = wmax ? (int)((wmax - 1) / kBatch) : -1; bi >= 0; --bi) {
    const uint32_t b0 = (uint32_t)bi * kBatch;
    const uint32_t lo = rg.x + b0;
    const int n = (int)min((uint32_t)kBatch, rg.y - lo);
    for (int h = 1; h >= 0; --h) {
      const int nh = min(n - h * kSlots, kSlots);
      if (nh <= 0) continue;
      const uint32_t hb = b0 + (uint32_t)h * kSlots;  // first pair of the half, within the tile
      // contributor bits of this half for the thread's pixels
      uint32_t mine[PPT];
      uint32_t any = 0u;
      if (!recompute) {
        const uint32_t *mw = a.masks + (size_t)(unit0 + (uint32_t)bi) * 2 * NPIX + (size_t)h * NPIX;
#pragma unroll
        for (int i = 0; i < PPT; ++i) {
          // pairs from the pixel's last contributor on are none of its own
          mine[i] = (ok[i] && hb < nl[i]) ? mw[lp[i]] : 0u;
          any |= mine[i];
        }
      } else {
        // recomputation: stage every pair of the half, then each pixel
        // re-tests the pairs before its last contributor (alpha box, alpha)
        __syncwarp();
        if ((int)lane < nh) stage(a.pvals[lo + h * kSlots + lane], lane, true);
        __syncwarp();
        // pairs whose pixel box meets the warp's pixel block (one test per
        // lane); the others fail every pixel's box test below
        int bx0 = px, bx1 = px, by0 = py[0], by1 = py[0];
#pragma unroll
        for (int i = 1; i < PPT; ++i) { by0 = min(by0, py[i]); by1 = max(by1, py[i]); }
        bx0 = __reduce_min_sync(0xffffffffu, bx0); bx1 = __reduce_max_sync(0xffffffffu, bx1);
        by0 = __reduce_min_sync(0xffffffffu, by0); by1 = __reduce_max_sync(0xffffffffu, by1);
        const short4 lb = st.box[lane];  // slots past nh hold stale boxes: masked out
        const uint32_t meets = __ballot_sync(0xffffffffu, (int)lane < nh && lb.x <= bx1 && lb.y >= bx0 &&
                                                               lb.z <= by1 && lb.w >= by0);
#pragma unroll
        for (int i = 0; i < PPT; ++i) {
          mine[i] = 0u;
          const int nj = nl[i] > hb ? min(nh, (int)(nl[i] - hb)) : 0;
          uint32_t cand = nj >= 32 ? meets : meets & ((1u << nj) - 1u);
          while (cand) {
            const int j = __ffs(cand) - 1;
            cand &= cand - 1u;
            const short4 bx = st.box[j];
            if (px < bx.x || px > bx.y || py[i] < bx.z || py[i] > bx.w) continue;
            float al, G_, ar, dx_, dy_;
            if (gauss_alpha(st.uv[j], st.co[j], fpx, fpy[i], al, G_, ar, dx_, dy_)) mine[i] |= 1u << j;
          }
          any |= mine[i];
        }
      }
      const uint32_t vis = __reduce_or_sync(0xffffffffu, any);
      if (!vis) continue;
      if (!recompute) {
        // stage the visited Gaussians, packed in pair order
        __syncwarp();
        if ((vis >> lane) & 1u) stage(a.pvals[lo + h * kSlots + lane], __popc(vis & lanemask_lt()), false);
        __syncwarp();
      }
      int s = __popc(vis);
      uint32_t rem = vis;
      while (rem) {
        const int bit = 31 - __clz(rem);
        rem ^= 1u << bit;
        --s;
        const int slot = recompute ? bit : s;
        const float2 uv = st.uv[slot];
        const float4 co = st.co[slot];
        const float4 cdp = st.cd[slot];
        // per class: the sign-word address and shift (CODES) or the class id
        const uint2 *cwp[KMAX];
        uint32_t csh[KMAX];
        int cid[KMAX];
        float cw8[KMAX];
        bool cvalid[KMAX];
        if (has_dsem) {
#pragma unroll
          for (int l = 0; l < KMAX; ++l) {
            if (K > 0 || l < k) {
              const int2 e = st.sem[l * kSlots + slot];
              cvalid[l] = (unsigned)e.x < (unsigned)a.m;
              cid[l] = cvalid[l] ? e.x : 0;
              cwp[l] = mycodes + (cvalid[l] ? (e.x >> 5) : a.nwc) * (PPT * THREADS);
              csh[l] = 31u - ((uint32_t)e.x & 31u);
              cw8[l] = __int_as_float(e.y);
            }
          }
        }
        float v[NVMAX];
        bool first = true, anyc = false;
#pragma unroll
        for (int i = 0; i < PPT; ++i) {
          const bool c = (mine[i] >> bit) & 1u;
          anyc = anyc || c;
          if (!__any_sync(0xffffffffu, c)) continue;  // uniform: no pixel of this row group
          // alpha at the pixel, with the forward's instructions; pixels the
          // Gaussian did not reach get w = dalpha = 0 (all terms exact zeros)
          const float dx = __fsub_rn(uv.x, fpx), dy = __fsub_rn(uv.y, fpy[i]);
          const float qf = __fmaf_rn(co.x, __fmul_rn(dx, dx), __fmul_rn(co.z, __fmul_rn(dy, dy)));
          const float power = __fmaf_rn(-0.5f, qf, -__fmul_rn(co.y, __fmul_rn(dx, dy)));
          const float G = __expf(power);
          const float araw = __fmul_rn(co.w, G);
          const float alpha = araw < kAlphaMax ? araw : kAlphaMax;
          const float inv_om = __fdividef(1.f, 1.f - alpha);  // approximate: 2 ulp, well inside the gradient bar
          const float Ti = T[i] * inv_om;
          const float w = c ? alpha * Ti : 0.f;
          T[i] = c ? Ti : T[i];
          float gi = dR[i] * cdp.x + dG[i] * cdp.y + dB[i] * cdp.z + dD[i] * cdp.w + dS[i];
          float vs[KMAX];
          if (has_dsem) {
            float gs = 0.f;
#pragma unroll
            for (int l = 0; l < KMAX; ++l) {
              if (K > 0 || l < k) {
                if (CODES) {
                  const uint2 cw = cwp[l][i * THREADS];
                  vs[l] = signed_weight(cw, csh[l], w);
                  if (SEMG) gs += signed_weight(cw, csh[l], cw8[l]);
                } else {
                  const float dp = cvalid[l] ? __ldg(dP[i] + cid[l]) : 0.f;
                  vs[l] = dp * w;
                  if (SEMG) gs = fmaf(dp, cw8[l], gs);
                }
              }
            }
            if (SEMG) gi = CODES ? fmaf(s_sem, gs, gi) : gi + gs;
          }
          const float dal = (c && araw < kAlphaMax) ? Ti * gi - acc[i] * inv_om : 0.f;
          acc[i] = fmaf(w, gi, acc[i]);
          const float dpow = dal * araw;
          const float ax = dpow * dx, ay = dpow * dy;
          if (first) {
            v[0] = ax; v[1] = ay; v[2] = ax * dx; v[3] = ax * dy; v[4] = ay * dy;
            v[5] = dal * G; v[6] = dD[i] * w; v[7] = dR[i] * w; v[8] = dG[i] * w; v[9] = dB[i] * w;
#pragma unroll
            for (int l = 0; l < KMAX; ++l)
              if (K > 0 || l < k) v[10 + l] = has_dsem ? vs[l] : 0.f;
          } else {
            v[0] += ax; v[1] += ay; v[2] = fmaf(ax, dx, v[2]); v[3] = fmaf(ax, dy, v[3]); v[4] = fmaf(ay, dy, v[4]);
            v[5] = fmaf(dal, G, v[5]); v[6] = fmaf(dD[i], w, v[6]);
            v[7] = fmaf(dR[i], w, v[7]); v[8] = fmaf(dG[i], w, v[8]); v[9] = fmaf(dB[i], w, v[9]);
#pragma unroll
            for (int l = 0; l < KMAX; ++l)
              if ((K > 0 || l < k) && has_dsem) v[10 + l] += vs[l];
          }
          first = false;
        }
        if (first) continue;  // unreachable: the Gaussian is a contributor of some pixel of the warp
        if (NVMAX > 16 && __popc(__ballot_sync(0xffffffffu, anyc)) <= 2) {
          // one or two lanes touched: they add their own values directly
          if (anyc) {
#pragma unroll
            for (int qq = 0; qq < NVMAX; ++qq) {
              if (qq >= nv) break;
              const int cls = qq < 7 ? 0 : (qq < 10 ? 1 : 2);
              const int off = qq < 7 ? qq : (qq < 10 ? qq - 7 : qq - 10);
              float val = v[qq];
              if (qq == 0) val = -(co.x * v[0] + co.y * v[1]);
              else if (qq == 1) val = -(co.z * v[1] + co.y * v[0]);
              else if (qq == 2 || qq == 4) val = -0.5f * v[qq];
              else if (qq == 3) val = -v[qq];
              else if (qq >= 10 && CODES) val = v[qq] * s_sem;
              float *base = st.dst[3 * slot + cls];
              if (base && val != 0.f) red_add_global(base + off, val);
            }
          }
          continue;
        }
        // transposed exchange: value q of every lane in row q
        __syncwarp();
#pragma unroll
        for (int qq = 0; qq < NVMAX; ++qq)
          if (qq < nv) red[qq * kRedStride + lane] = v[qq];
        __syncwarp();
        float tot = 0.f;
        if (narrow) {
          if (q < nv) {
            const float4 *r4 = reinterpret_cast<const float4 *>(red + q * kRedStride + 16 * (lane >> 4));
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const float4 x = r4[u];
              tot += (x.x + x.y) + (x.z + x.w);
            }
          }
          tot += __shfl_xor_sync(0xffffffffu, tot, 16);
        } else if (q < nv) {
          const float4 *r4 = reinterpret_cast<const float4 *>(red + q * kRedStride);
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const float4 x = r4[u];
            tot += (x.x + x.y) + (x.z + x.w);
          }
        }
        // lanes 0, 1 combine the two sums with the conic: du, dv
        const float other = __shfl_xor_sync(0xffffffffu, tot, 1);
        const float c1 = q == 0 ? -co.x : (q == 1 ? -co.z : q_scale);
        const float c2 = q < 2 ? -co.y : 0.f;
        const float val = fmaf(c1, tot, c2 * other);
        float *base = st.dst[3 * slot + q_cls];
        if (issue && base && val != 0.f) red_add_global(base + q_off, val);
      }
    }
  }
}

__global__ void k_zero_grad2d(float4 *g, const Counters *cnt, uint32_t rcap) {
  const uint32_t n = 2 * min(cnt->n_records, rcap);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    g[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

constexpr int kBwdSmemMax = 227 * 1024;  // opt-in dynamic shared memory per CTA

template <int TW, int TH, bool CODES, int K, int PPT, bool SEMG>
static cudaError_t launch_bwd_shape(const BwdArgs &a, int grid, size_t smem, cudaStream_t s) {
  if (smem > (size_t)kBwdSmemMax) return cudaErrorInvalidConfiguration;
  {
    const cudaError_t e =
        ensure_smem_limit((const void *)k_render_bwd<TW, TH, CODES, K, PPT, SEMG>, kBwdSmemMax);
    if (e != cudaSuccess) return e;
  }
  k_render_bwd<TW, TH, CODES, K, PPT, SEMG><<<grid, TW * TH / PPT, smem, s>>>(a);
  return cudaGetLastError();
}

template <bool CODES, int K, int PPT, bool SEMG>
static cudaError_t dispatch_bwd_shape(int tw, int th, const BwdArgs &a, int grid, size_t smem, cudaStream_t s) {
  if (tw == 16 && th == 16) return launch_bwd_shape<16, 16, CODES, K, PPT, SEMG>(a, grid, smem, s);
  if (tw == 16 && th == 8) return launch_bwd_shape<16, 8, CODES, K, PPT, SEMG>(a, grid, smem, s);
  if (tw == 8 && th == 8) return launch_bwd_shape<8, 8, CODES, K, PPT, SEMG>(a, grid, smem, s);
  if (tw == 32 && th == 8) return launch_bwd_shape<32, 8, CODES, K, PPT, SEMG>(a, grid, smem, s);
  return cudaErrorInvalidConfiguration;
}

template <bool CODES, int PPT>
static cudaError_t dispatch_bwd_k(const Layout &L, const BwdArgs &a, bool semg, int grid, size_t smem,
                                  cudaStream_t s) {
  // semantics reaching the geometry (not the paper's setting) take the generic-k kernel
  if (semg) return dispatch_bwd_shape<CODES, 0, PPT, true>(L.tile_w, L.tile_h, a, grid, smem, s);
  if (a.k == 3) return dispatch_bwd_shape<CODES, 3, PPT, false>(L.tile_w, L.tile_h, a, grid, smem, s);
  if (a.k == 8) return dispatch_bwd_shape<CODES, 8, PPT, false>(L.tile_w, L.tile_h, a, grid, smem, s);
  return dispatch_bwd_shape<CODES, 0, PPT, false>(L.tile_w, L.tile_h, a, grid, smem, s);
}

template <bool CODES>
static cudaError_t dispatch_bwd(const Layout &L, const BwdArgs &a, bool semg, int grid, size_t smem,
                                cudaStream_t s) {
  if (L.ppt == 4) {
    if (L.tile_w != 16 || L.tile_h != 16) return cudaErrorInvalidConfiguration;
    if (semg) return launch_bwd_shape<16, 16, CODES, 0, 4, true>(a, grid, smem, s);
    if (a.k == 3) return launch_bwd_shape<16, 16, CODES, 3, 4, false>(a, grid, smem, s);
    if (a.k == 8) return launch_bwd_shape<16, 16, CODES, 8, 4, false>(a, grid, smem, s);
    return launch_bwd_shape<16, 16, CODES, 0, 4, false>(a, grid, smem, s);
  }
  if (L.ppt == 2) return dispatch_bwd_k<CODES, 2>(L, a, semg, grid, smem, s);
  return dispatch_bwd_k<CODES, 1>(L, a, semg, grid, smem, s);
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
  a.counters = P.counters;
  a.grad2d = P.grad2d;
  a.g_rgb = g_rgb; a.g_sem_w = g_sem_w;
  a.mask_off = L.mask_units ? P.mask_off : nullptr;
  a.masks = L.mask_units ? P.masks : nullptr;
  a.warp_bytes = (int)bwd_warp_bytes(sc.k);
  const int grid = a.tiles_x * tiles_y;
  if (grid == 0) return cudaSuccess;
  const int threads = L.tile_w * L.tile_h / L.ppt;
  const size_t warps_bytes = (size_t)(threads / 32) * a.warp_bytes;
  // the semantic upstream gradient reaches the geometry only when asked for
  // and when there is one
  if (loss_scale) {
    a.codes = P.codes;
    a.nwc = objective ? 0 : L.nwc;
    a.loss_scale = loss_scale;
    a.npix = (double)L.npix;
    a.objective = objective;
    const bool semg = !sem_detach && !objective;
    // per thread and pixel: the class sign words plus one zero word
    const size_t smem = warps_bytes + (a.nwc ? (size_t)threads * L.ppt * (a.nwc + 1) * 8 : 0);
    return dispatch_bwd<true>(L, a, semg, grid, smem, s);
  }
  const bool semg = !sem_detach && d_sem != nullptr;
  return dispatch_bwd<false>(L, a, semg, grid, warps_bytes, s);
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
