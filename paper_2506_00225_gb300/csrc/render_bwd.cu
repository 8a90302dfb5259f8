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
  const float *rgb;
  const int32_t *sem_ids;
  const float *sem_w;
  int k, m, width, height, tiles_x;
  const float *tfinal;
  const uint32_t *nlast;
  const float *d_rgb, *d_depth, *d_sil, *d_sem;
  int sem_detach;
  float4 *grad2d;
  float *g_rgb, *g_sem_w;
  // fused mean-L1 mode: upstream gradients decoded from sign codes
  const uint32_t *codes;
  int nwc;
  const float *loss_scale;  // device dL/dloss
  double npix;
};

__device__ __forceinline__ float sign_code(uint32_t nz, uint32_t ng, int bit, float s) {
  return ((nz >> bit) & 1u) ? (((ng >> bit) & 1u) ? -s : s) : 0.f;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <int TW, int TH, bool CODES>
__global__ void __launch_bounds__(TW *TH) k_render_bwd(BwdArgs a) {
  extern __shared__ float4 smem4[];
  BatchSmem bs = batch_smem(smem4, a.k);
  __shared__ uint32_t s_maxnl;
  // CODES: per-thread copy of its pixel's class sign words (odd stride)
  uint32_t *myc = reinterpret_cast<uint32_t *>(bs.tail) + threadIdx.x * (2 * a.nwc + 1);

  const int tile = blockIdx.x;
  const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
  const uint2 rg = a.ranges[tile];
  const int lx = threadIdx.x % TW, ly = threadIdx.x / TW;
  const int px = tx * TW + lx, py = ty * TH + ly;
  const bool inside = px < a.width && py < a.height;
  const float fpx = (float)px + 0.5f, fpy = (float)py + 0.5f;
  const size_t pix = inside ? (size_t)py * a.width + px : 0;
  const int k = a.k;
  // warp-uniform: every lane takes the same branches around the shuffles
  const bool has_dsem = CODES || a.d_sem != nullptr;
  float s_sem = 0.f;

  float T = 1.f, dR = 0.f, dG = 0.f, dB = 0.f, dD = 0.f, dS = 0.f;
  uint32_t nl = 0;
  const float *dP = nullptr;
  if (inside) {
    T = a.tfinal[pix];
    nl = a.nlast[pix];
    if (CODES) {
      const float ls = *a.loss_scale;
      const float s_rgb = (float)(ls / (3.0 * a.npix)), s_d = (float)(ls / a.npix);
      s_sem = (float)(ls / (a.npix * a.m));
      const uint32_t *cp = a.codes + pix * code_words(a.nwc);
      const uint32_t nz = cp[0], ng = cp[1 + a.nwc];
      dR = sign_code(nz, ng, 0, s_rgb); dG = sign_code(nz, ng, 1, s_rgb); dB = sign_code(nz, ng, 2, s_rgb);
      dD = sign_code(nz, ng, 3, s_d);
      for (int wd = 0; wd < a.nwc; ++wd) { myc[wd] = cp[1 + wd]; myc[a.nwc + wd] = cp[2 + a.nwc + wd]; }
    } else {
      if (a.d_rgb) { dR = a.d_rgb[3 * pix]; dG = a.d_rgb[3 * pix + 1]; dB = a.d_rgb[3 * pix + 2]; }
      if (a.d_depth) dD = a.d_depth[pix];
      if (a.d_sil) dS = a.d_sil[pix];
      if (a.d_sem) dP = a.d_sem + pix * a.m;
    }
  }
  if (threadIdx.x == 0) s_maxnl = 0;
  __syncthreads();
  if (nl) atomicMax(&s_maxnl, nl);
  __syncthreads();
  const uint32_t maxnl = s_maxnl;
  float acc = 0.f;  // sum over later contributors of w_j g_j

  for (uint32_t hi = rg.x + maxnl; hi > rg.x;) {
    const uint32_t lo = hi - min((uint32_t)kBatch, hi - rg.x);
    const int n = (int)(hi - lo);
    __syncthreads();
    if ((int)threadIdx.x < n) load_batch_entry(a.rec, a.pvals[lo + threadIdx.x], threadIdx.x, k, bs, a.rgb,
                                               a.sem_ids, a.sem_w, nullptr);
    __syncthreads();
    for (int j = n - 1; j >= 0; --j) {
      const uint32_t idx = lo - rg.x + j;
      bool contrib = inside && idx < nl && rect_holds(bs.rect[j], px, py);
      float alpha = 0.f, G = 0.f, araw = 0.f, dx = 0.f, dy = 0.f;
      if (contrib) contrib = gauss_alpha(bs.uv[j], bs.co[j], fpx, fpy, alpha, G, araw, dx, dy);
      float v[7];  // du, dv, da, db, dc, dopacity, ddepth
      float vc[3];
      float vs[kMaxK];
#pragma unroll
      for (int i = 0; i < 7; ++i) v[i] = 0.f;
      vc[0] = vc[1] = vc[2] = 0.f;
#pragma unroll
      for (int l = 0; l < kMaxK; ++l) vs[l] = 0.f;
      if (contrib) {
        const float4 co = bs.co[j];
        const float4 cdp = bs.cd[j];
        const float om = 1.f - alpha;
        const float Ti = T / om;
        const float w = alpha * Ti;
        float gi = dR * cdp.x + dG * cdp.y + dB * cdp.z + dD * cdp.w + dS;
        if (has_dsem) {
          const int *sid = bs.sid + j * k;
          const float *sw = bs.sw + j * k;
          float gs = 0.f;
#pragma unroll
          for (int l = 0; l < kMaxK; ++l) {
            if (l < k && (unsigned)sid[l] < (unsigned)a.m) {
              float dp;
              if (CODES) {
                const int wd = sid[l] >> 5, bit = sid[l] & 31;
                dp = sign_code(myc[wd], myc[a.nwc + wd], bit, s_sem);
              } else {
                dp = __ldg(dP + sid[l]);
              }
              vs[l] = dp * w;
              gs = fmaf(dp, sw[l], gs);
            }
          }
          if (!a.sem_detach) gi += gs;
        }
        vc[0] = dR * w; vc[1] = dG * w; vc[2] = dB * w;
        v[6] = dD * w;
        const float dalpha = Ti * gi - acc / om;
        acc = fmaf(w, gi, acc);
        T = Ti;
        if (araw < kAlphaMax) {
          v[5] = dalpha * G;
          const float dpow = dalpha * araw;
          v[2] = dpow * (-0.5f * dx * dx);
          v[3] = dpow * (-dx * dy);
          v[4] = dpow * (-0.5f * dy * dy);
          v[0] = dpow * (-(co.x * dx + co.y * dy));
          v[1] = dpow * (-(co.z * dy + co.y * dx));
        }
      }
      if (__any_sync(0xffffffffu, contrib)) {
#pragma unroll
        for (int i = 0; i < 7; ++i) v[i] = warp_sum(v[i]);
#pragma unroll
        for (int i = 0; i < 3; ++i) vc[i] = warp_sum(vc[i]);
        if (has_dsem) {
#pragma unroll
          for (int l = 0; l < kMaxK; ++l)
            if (l < k) vs[l] = warp_sum(vs[l]);
        }
        if (lane_id() == 0) {
          const int r = bs.rec[j], g = bs.gid[j];
          atomicAdd(a.grad2d + 2 * (size_t)r, make_float4(v[0], v[1], v[2], v[3]));
          atomicAdd(a.grad2d + 2 * (size_t)r + 1, make_float4(v[4], v[5], v[6], 0.f));
          if (a.g_rgb) {
            atomicAdd(a.g_rgb + 3 * (size_t)g, vc[0]);
            atomicAdd(a.g_rgb + 3 * (size_t)g + 1, vc[1]);
            atomicAdd(a.g_rgb + 3 * (size_t)g + 2, vc[2]);
          }
          if (has_dsem && a.g_sem_w)
            for (int l = 0; l < k; ++l) atomicAdd(a.g_sem_w + (size_t)g * k + l, vs[l]);
        }
      }
    }
    hi = lo;
  }
}

__global__ void k_zero_grad2d(float4 *g, const Counters *cnt, uint32_t rcap) {
  const uint32_t n = 2 * min(cnt->n_records, rcap);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    g[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

template <int TW, int TH, bool CODES>
static cudaError_t launch_bwd_shape(const BwdArgs &a, int grid, size_t smem, cudaStream_t s) {
  k_render_bwd<TW, TH, CODES><<<grid, TW * TH, smem, s>>>(a);
  return cudaGetLastError();
}

template <bool CODES>
static cudaError_t dispatch_bwd(int tw, int th, const BwdArgs &a, int grid, size_t smem, cudaStream_t s) {
  if (tw == 16 && th == 16) return launch_bwd_shape<16, 16, CODES>(a, grid, smem, s);
  if (tw == 16 && th == 8) return launch_bwd_shape<16, 8, CODES>(a, grid, smem, s);
  if (tw == 8 && th == 8) return launch_bwd_shape<8, 8, CODES>(a, grid, smem, s);
  if (tw == 32 && th == 8) return launch_bwd_shape<32, 8, CODES>(a, grid, smem, s);
  return cudaErrorInvalidConfiguration;
}

cudaError_t launch_render_bwd(const Layout &L, const WsPtrs &P, int pbuf, const gs_scene &sc, const float *d_rgb,
                              const float *d_depth, const float *d_sil, const float *d_sem, int sem_detach,
                              float *g_rgb, float *g_sem_w, cudaStream_t s, const float *loss_scale) {
  k_zero_grad2d<<<2 * 152, 256, 0, s>>>(P.grad2d, P.counters, (uint32_t)L.rcap);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  BwdArgs a{};
  a.ranges = P.ranges;
  a.pvals = P.pvals[pbuf];
  a.rec = rec_ptrs(P);
  a.rgb = sc.rgb; a.sem_ids = sc.sem_ids; a.sem_w = sc.sem_w;
  a.k = sc.k; a.m = sc.m;
  a.width = L.cam0_w; a.height = L.cam0_h;
  a.tiles_x = (L.cam0_w + L.tile_w - 1) / L.tile_w;
  const int tiles_y = (L.cam0_h + L.tile_h - 1) / L.tile_h;
  a.tfinal = P.tfinal; a.nlast = P.nlast;
  a.d_rgb = d_rgb; a.d_depth = d_depth; a.d_sil = d_sil; a.d_sem = d_sem;
  a.sem_detach = sem_detach;
  a.grad2d = P.grad2d;
  a.g_rgb = g_rgb; a.g_sem_w = g_sem_w;
  const int grid = a.tiles_x * tiles_y;
  if (grid == 0) return cudaSuccess;
  if (loss_scale) {
    a.codes = P.codes;
    a.nwc = L.nwc;
    a.loss_scale = loss_scale;
    a.npix = (double)L.npix;
    const size_t smem = batch_smem_bytes(sc.k) + (size_t)L.tile_w * L.tile_h * (2 * L.nwc + 1) * 4;
    return dispatch_bwd<true>(L.tile_w, L.tile_h, a, grid, smem, s);
  }
  const size_t smem = batch_smem_bytes(sc.k);
  return dispatch_bwd<false>(L.tile_w, L.tile_h, a, grid, smem, s);
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
