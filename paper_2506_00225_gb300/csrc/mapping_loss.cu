// mapping_loss.cu -- the mapping objective of Sec. 3.1 on rendered maps, and
// its gradient with respect to them.
//
// Geometry and colour (the objective after Eq. 1): pixels with silhouette
// above 0.99 contribute |D - D*| + 0.5 sum_c |C_c - C*_c|; these terms are
// summed.  Semantics ("Semantic Loss", Eq. 4, Eq. 5): for the target class
// distribution Q of a pixel and the rendered one P, the entropy mask
// M_H = [H(Q) < ln k], the Hellinger distance
// D = sqrt(0.5 sum_m (sqrt(Q_m + e) - sqrt(max(P_m, 0) + e))^2) and the cosine
// similarity cos = Q.P / (|Q| |P|) give M_H (0.8 D + 0.2 (1 - cos)); this term
// is averaged over the pixels and added.  e = 1e-12 keeps the square roots
// differentiable at 0; a zero distance or norm gives a zero gradient for its
// term.
//
// A warp takes 4 consecutive pixels at a time: lanes 0-3 their geometry,
// all lanes their classes (c = lane + 32 i, held in registers up to 128
// classes, so that the four pixels' loads and warp sums overlap), then the
// lanes write the class gradients (coalesced).  Per-CTA partial sums in
// double, reduced by one CTA: deterministic.
#include "gs_internal.cuh"
#include "objective_math.cuh"

namespace gs {

constexpr int kMlThreads = 256;
constexpr int kMlMaxCtas = GS_MAPPING_LOSS_PARTIALS / 2;  // two partial sums per CTA
constexpr int kMlG = 4;  // pixels per warp round
constexpr float kSilMin = 0.99f;
constexpr float kWColour = 0.5f;

__global__ void __launch_bounds__(kMlThreads) k_mapping_loss(int64_t npix, int m, float log_k, const float *rgb,
                                                             const float *t_rgb, const float *depth,
                                                             const float *t_depth, const float *sil,
                                                             const float *sem, const float *t_sem, float *d_rgb,
                                                             float *d_depth, float *d_sem, double *partial) {
  const uint32_t lane = lane_id();
  const int64_t warp0 = ((int64_t)blockIdx.x * kMlThreads + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * kMlThreads) >> 5;
  const float inv_n = 1.f / (float)npix;
  double geo = 0.0, semt = 0.0;
  for (int64_t p0 = warp0 * kMlG; p0 < npix; p0 += nwarps * kMlG) {
    // geometry and colour: lane g < 4 takes pixel p0 + g
    if (lane < kMlG && p0 + lane < npix) {
      const int64_t p = p0 + lane;
      const float mg = sil[p] > kSilMin ? 1.f : 0.f;
      const float ed = depth[p] - t_depth[p];
      float l = fabsf(ed);
      if (d_depth) d_depth[p] = ed > 0.f ? mg : (ed < 0.f ? -mg : 0.f);
      for (int c = 0; c < 3; ++c) {
        const float ec = rgb[3 * p + c] - t_rgb[3 * p + c];
        l += kWColour * fabsf(ec);
        if (d_rgb) d_rgb[3 * p + c] = ec > 0.f ? kWColour * mg : (ec < 0.f ? -kWColour * mg : 0.f);
      }
      geo += (double)(mg * l);
    }
    if (!sem) continue;
    if (m <= 32 * kObjMI) {
      float qv[kMlG][kObjMI], pv[kMlG][kObjMI], st[kMlG][5];
      ClassRoots rt[kMlG][kObjMI];
      bool ok[kMlG];
#pragma unroll
      for (int g = 0; g < kMlG; ++g) {
        ok[g] = p0 + g < npix;
        const int64_t base = ok[g] ? (p0 + g) * m : 0;
#pragma unroll
        for (int i = 0; i < kObjMI; ++i) {
          const int c = (int)lane + 32 * i;
          const bool in = ok[g] && c < m;
          qv[g][i] = in ? t_sem[base + c] : 0.f;
          pv[g][i] = in ? sem[base + c] : 0.f;
        }
      }
#pragma unroll
      for (int g = 0; g < kMlG; ++g) {
#pragma unroll
        for (int j = 0; j < 5; ++j) st[g][j] = 0.f;
#pragma unroll
        for (int i = 0; i < kObjMI; ++i) rt[g][i] = class_sums(qv[g][i], pv[g][i], st[g]);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int g = 0; g < kMlG; ++g)
#pragma unroll
          for (int j = 0; j < 5; ++j) st[g][j] += __shfl_xor_sync(0xffffffffu, st[g][j], o);
#pragma unroll
      for (int g = 0; g < kMlG; ++g) {
        const PixelTerm t = pixel_term(st[g], ok[g], log_k);
        if (lane == 0 && t.keep) semt += (double)t.value;
        if (d_sem && ok[g]) {
          float *gr = d_sem + (p0 + g) * m;
#pragma unroll
          for (int i = 0; i < kObjMI; ++i) {
            const int c = (int)lane + 32 * i;
            if (c < m) gr[c] = t.keep ? class_grad(qv[g][i], pv[g][i], rt[g][i], t, inv_n) : 0.f;
          }
        }
      }
    } else {
      for (int g = 0; g < kMlG && p0 + g < npix; ++g) {
        const int64_t p = p0 + g;
        const float *q = t_sem + p * m, *pr = sem + p * m;
        float st[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
        for (int c = (int)lane; c < m; c += 32) class_sums(q[c], pr[c], st);
        warp_sum5(st);
        const PixelTerm t = pixel_term(st, true, log_k);
        if (lane == 0 && t.keep) semt += (double)t.value;
        if (d_sem) {
          float *gr = d_sem + p * m;
          for (int c = (int)lane; c < m; c += 32) {
            gr[c] = t.keep ? class_grad(q[c], pr[c], class_roots(q[c], pr[c]), t, inv_n) : 0.f;
          }
        }
      }
    }
  }
  __shared__ double red[2][kMlThreads / 32];
  // lanes 0-3 hold geometry sums, lane 0 the semantic sum
#pragma unroll
  for (int o = 2; o > 0; o >>= 1) geo += __shfl_xor_sync(0xffffffffu, geo, o);
  if (lane == 0) { red[0][threadIdx.x >> 5] = geo; red[1][threadIdx.x >> 5] = semt; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < kMlThreads / 32; ++w) { a += red[0][w]; b += red[1][w]; }
    partial[2 * blockIdx.x] = a;
    partial[2 * blockIdx.x + 1] = b;
  }
}

__global__ void k_mapping_loss_final(const double *partial, int n, double npix, float *loss) {
  __shared__ double red[2][32];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) { a += partial[2 * i]; b += partial[2 * i + 1]; }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = a; red[1][threadIdx.x >> 5] = b; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { s0 += red[0][w]; s1 += red[1][w]; }
    *loss = (float)(s0 + s1 / npix);
  }
}

cudaError_t launch_mapping_loss(int64_t npix, int m, int k, const float *rgb, const float *t_rgb, const float *depth,
                                const float *t_depth, const float *sil, const float *sem, const float *t_sem,
                                float *d_rgb, float *d_depth, float *d_sem, float *loss, double *partial,
                                cudaStream_t s) {
  // four CTAs per SM, within the caller's partial-sum scratch
  const unsigned ctas = min(sm_grid(4), (unsigned)kMlMaxCtas);
  if (ctas == 0) return cudaErrorInvalidDevice;
  k_mapping_loss<<<ctas, kMlThreads, 0, s>>>(npix, m, logf((float)k), rgb, t_rgb, depth, t_depth, sil, sem, t_sem,
                                                d_rgb, d_depth, d_sem, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_mapping_loss_final<<<1, 256, 0, s>>>(partial, (int)ctas, (double)npix, loss);
  return cudaGetLastError();
}

}  // namespace gs
