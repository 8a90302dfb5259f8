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
// One warp per pixel: lanes stride over the classes, warp sums give the
// pixel's entropy, distance, norms and dot product, then the lanes write the
// class gradients (coalesced).  Per-CTA partial sums in double, reduced by one
// CTA: deterministic.
#include "gs_internal.cuh"

namespace gs {

constexpr int kMlThreads = 256;
constexpr int kMlCtas = 4 * 152;
constexpr float kSilMin = 0.99f;
constexpr float kWColour = 0.5f;
constexpr float kLamHd = 0.8f, kLamCos = 0.2f;
constexpr float kEpsSqrt = 1e-12f, kEpsDiv = 1e-12f;

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

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
  for (int64_t p = warp0; p < npix; p += nwarps) {
    // geometry and colour (lane 0)
    if (lane == 0) {
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
    // semantics: warp sums over the classes
    const float *q = t_sem + p * m, *pr = sem + p * m;
    float hq = 0.f, s2 = 0.f, qq = 0.f, pp = 0.f, qp = 0.f;
    for (int c = (int)lane; c < m; c += 32) {
      const float qv = q[c], pv = pr[c];
      if (qv > 0.f) hq -= qv * logf(qv);
      const float d = sqrtf(fmaxf(qv, 0.f) + kEpsSqrt) - sqrtf(fmaxf(pv, 0.f) + kEpsSqrt);
      s2 = fmaf(d, d, s2);
      qq = fmaf(qv, qv, qq);
      pp = fmaf(pv, pv, pp);
      qp = fmaf(qv, pv, qp);
    }
    hq = warp_sum(hq); s2 = warp_sum(s2); qq = warp_sum(qq); pp = warp_sum(pp); qp = warp_sum(qp);
    const bool keep = hq < log_k;
    const float dist = sqrtf(0.5f * s2);
    const float den = sqrtf(qq) * sqrtf(pp);
    const float cosv = den > kEpsDiv ? qp / den : 0.f;
    if (lane == 0 && keep) semt += (double)(kLamHd * dist + kLamCos * (1.f - cosv));
    if (d_sem) {
      float *g = d_sem + p * m;
      for (int c = (int)lane; c < m; c += 32) {
        float gv = 0.f;
        if (keep) {
          const float qv = q[c], pv = pr[c];
          float dhd = 0.f;
          if (dist > kEpsDiv && pv >= 0.f) {
            const float sp = sqrtf(pv + kEpsSqrt), sq = sqrtf(fmaxf(qv, 0.f) + kEpsSqrt);
            dhd = (sp - sq) / (4.f * dist * sp);
          }
          float dcos = 0.f;
          if (den > kEpsDiv) dcos = qv / den - cosv * pv / fmaxf(pp, kEpsDiv);
          gv = (kLamHd * dhd - kLamCos * dcos) * inv_n;
        }
        g[c] = gv;
      }
    }
  }
  __shared__ double red[2][kMlThreads / 32];
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
  k_mapping_loss<<<kMlCtas, kMlThreads, 0, s>>>(npix, m, logf((float)k), rgb, t_rgb, depth, t_depth, sil, sem, t_sem,
                                                d_rgb, d_depth, d_sem, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_mapping_loss_final<<<1, 256, 0, s>>>(partial, kMlCtas, (double)npix, loss);
  return cudaGetLastError();
}

}  // namespace gs
