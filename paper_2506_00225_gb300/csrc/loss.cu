// loss.cu -- mean-L1 mapping loss and its gradient in one pass over the
// rendered and target images (colour, depth, semantic map).  Sec. 3.1 Eq. 2
// uses L1 colour and depth terms; the semantic map gets an L1 term as well.
// Deterministic: per-CTA partial sums in double, reduced by one CTA.
#include "gs_internal.cuh"

namespace gs {

constexpr int kLossMaxCtas = 2048;  // partial sums the caller's scratch holds (one per CTA)
constexpr int kLossThreads = 256;

__device__ __forceinline__ float l1_term(float x, float t, float scale, float &grad) {
  const float d = x - t;
  grad = d > 0.f ? scale : (d < 0.f ? -scale : 0.f);
  return fabsf(d);
}

__global__ void __launch_bounds__(kLossThreads) k_l1_partial(int64_t npix, int m, const float *rgb,
                                                             const float *t_rgb, const float *depth,
                                                             const float *t_depth, const float *sem,
                                                             const float *t_sem, float *d_rgb, float *d_depth,
                                                             float *d_sem, double *partial) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  double acc = 0.0;
  if (rgb) {
    const int64_t n = 3 * npix;
    const float sc = 1.f / (float)n;
    float s = 0.f;
    for (int64_t i = tid; i < n; i += stride) {
      float g;
      s += l1_term(rgb[i], t_rgb[i], sc, g);
      if (d_rgb) d_rgb[i] = g;
    }
    acc += (double)s / (double)n;
  }
  if (depth) {
    const int64_t n = npix;
    const float sc = 1.f / (float)n;
    float s = 0.f;
    for (int64_t i = tid; i < n; i += stride) {
      float g;
      s += l1_term(depth[i], t_depth[i], sc, g);
      if (d_depth) d_depth[i] = g;
    }
    acc += (double)s / (double)n;
  }
  if (sem) {
    const int64_t n = npix * m;
    const float sc = 1.f / (float)n;
    float s = 0.f;
    const int64_t n4 = n / 4;
    const float4 *x4 = reinterpret_cast<const float4 *>(sem);
    const float4 *t4 = reinterpret_cast<const float4 *>(t_sem);
    float4 *g4 = reinterpret_cast<float4 *>(d_sem);
    for (int64_t i = tid; i < n4; i += stride) {
      const float4 x = __ldcs(x4 + i), t = __ldcs(t4 + i);
      float4 g;
      s += l1_term(x.x, t.x, sc, g.x) + l1_term(x.y, t.y, sc, g.y) + l1_term(x.z, t.z, sc, g.z) +
           l1_term(x.w, t.w, sc, g.w);
      if (d_sem) __stcs(g4 + i, g);
    }
    for (int64_t i = 4 * n4 + tid; i < n; i += stride) {
      float g;
      s += l1_term(sem[i], t_sem[i], sc, g);
      if (d_sem) d_sem[i] = g;
    }
    acc += (double)s / (double)n;
  }
  // block reduction in double
  __shared__ double red[kLossThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kLossThreads / 32; ++w) s += red[w];
    partial[blockIdx.x] = s;
  }
}

__global__ void k_l1_final(const double *partial, int n, float *loss) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += partial[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    *loss = (float)t;
  }
}

cudaError_t launch_l1_loss(int64_t npix, int m, const float *rgb, const float *t_rgb, const float *depth,
                           const float *t_depth, const float *sem, const float *t_sem, float *d_rgb, float *d_depth,
                           float *d_sem, float *loss, double *partial, cudaStream_t s) {
  // two CTAs per SM, within the caller's partial-sum scratch
  const unsigned ctas = min(sm_grid(2), (unsigned)kLossMaxCtas);
  if (ctas == 0) return cudaErrorInvalidDevice;
  k_l1_partial<<<ctas, kLossThreads, 0, s>>>(npix, m, rgb, t_rgb, depth, t_depth, sem, t_sem, d_rgb, d_depth, d_sem,
                                             partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_l1_final<<<1, 256, 0, s>>>(partial, (int)ctas, loss);
  return cudaGetLastError();
}

}  // namespace gs
