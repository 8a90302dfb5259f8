// topk.cu -- the sparse semantic representation's initialisation and update
// (Sec. 3.1 "Sparse Semantic Representation"): a new Gaussian keeps the k
// classes of highest probability of its first observed distribution; later
// observations update those k probabilities with the ids fixed.
//
// One warp per Gaussian: lanes stride over the M classes of its observed row
// (coalesced), k rounds of a warp arg-max pick the classes (larger
// probability first, the lower class id on ties; NaN counts as -inf), so the
// result does not depend on the thread schedule.
#include <cmath>

#include "gs_internal.cuh"

namespace gs {

constexpr int kTopkThreads = 256;

struct Cand {
  float v;
  int c;
};

// a before b: larger value, then lower class id (c < 0: no candidate)
__device__ __forceinline__ bool better(Cand a, Cand b) {
  if (a.c < 0) return false;
  if (b.c < 0) return true;
  return a.v > b.v || (a.v == b.v && a.c < b.c);
}

__global__ void __launch_bounds__(kTopkThreads) k_topk_init(int64_t n, int m, int k, const float *__restrict__ probs,
                                                             const int64_t *__restrict__ rows, int32_t *ids,
                                                             float *w) {
  const uint32_t lane = lane_id();
  const int64_t warp0 = ((int64_t)blockIdx.x * kTopkThreads + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * kTopkThreads) >> 5;
  int taken[kMaxK];
  for (int64_t g = warp0; g < n; g += nwarps) {
    const int64_t row = rows ? rows[g] : g;
    const float *p = probs + row * m;
    for (int r = 0; r < k; ++r) {
      Cand best{0.f, -1};
      for (int c = (int)lane; c < m; c += 32) {
        bool used = false;
        for (int q = 0; q < r; ++q) used |= taken[q] == c;
        if (used) continue;
        float v = __ldg(p + c);
        if (v != v) v = -INFINITY;
        const Cand cd{v, c};
        if (better(cd, best)) best = cd;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const Cand other{__shfl_xor_sync(0xffffffffu, best.v, o), __shfl_xor_sync(0xffffffffu, best.c, o)};
        if (better(other, best)) best = other;
      }
      taken[r] = best.c;
      if (lane == 0) {
        ids[g * k + r] = best.c;
        w[g * k + r] = __ldg(p + best.c);
      }
    }
  }
}

__global__ void k_topk_gather(int64_t n, int m, int k, const float *__restrict__ probs,
                              const int64_t *__restrict__ rows, const int32_t *__restrict__ ids, float *w) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n * k; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t g = i / k;
    const int64_t row = rows ? rows[g] : g;
    const int c = ids[i];
    if ((unsigned)c < (unsigned)m) w[i] = __ldg(probs + row * m + c);
  }
}

static unsigned grid_for(int64_t items, int per_cta) {
  const int64_t b = (items + per_cta - 1) / per_cta, cap = sm_grid(8);
  return (unsigned)(b < cap ? (b > 0 ? b : 1) : cap);
}

}  // namespace gs

using namespace gs;

extern "C" {

gs_status gs_topk_init(int64_t n, int m, int k, const float *probs, const int64_t *rows, int32_t *ids, float *w,
                       gs_stream_t stream) {
  if (n < 0 || m < 1 || k < 1 || k > kMaxK || k > m) return GS_ERR_ARG;
  if (n == 0) return GS_OK;
  if (!probs || !ids || !w) return GS_ERR_ARG;
  k_topk_init<<<grid_for(n, kTopkThreads / 32), kTopkThreads, 0, (cudaStream_t)stream>>>(n, m, k, probs, rows, ids,
                                                                                          w);
  return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

gs_status gs_topk_gather(int64_t n, int m, int k, const float *probs, const int64_t *rows, const int32_t *ids,
                         float *w, gs_stream_t stream) {
  if (n < 0 || m < 1 || k < 1 || k > kMaxK) return GS_ERR_ARG;
  if (n == 0) return GS_OK;
  if (!probs || !ids || !w) return GS_ERR_ARG;
  k_topk_gather<<<grid_for(n * k, 256), 256, 0, (cudaStream_t)stream>>>(n, m, k, probs, rows, ids, w);
  return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

}  // extern "C"
