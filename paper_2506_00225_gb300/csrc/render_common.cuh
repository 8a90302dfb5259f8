// render_common.cuh -- pieces shared by the forward, backward and candidate
// blend kernels: shared-memory batch staging of a tile's sorted Gaussians,
// the pixel-rectangle test and the per-pixel opacity rule.
#pragma once

#include "gs_internal.cuh"

namespace gs {

constexpr int kBatch = 64;                       // Gaussians staged per batch
constexpr float kTStop = 0.0001f;                // transmittance stop
constexpr float kAlphaMin = 1.0f / 255.0f;       // skip threshold
constexpr float kAlphaMax = 0.99f;               // opacity cap
constexpr size_t kSmemBudget = 112 * 1024;       // per CTA: two 256-thread CTAs per SM

struct RecPtrs {
  const float2 *uv;
  const float4 *co;
  const float *depth;
  const short4 *rect;
  const int32_t *gid;
};

inline RecPtrs rec_ptrs(const WsPtrs &P) { return RecPtrs{P.rec_uv, P.rec_conic, P.rec_depth, P.rec_rect, P.rec_gid}; }

// Shared-memory view of one staged batch (struct-of-arrays) plus the tail
// region after it (per-pixel class accumulators).
struct BatchSmem {
  float4 *co;   // conic a, b, c, opacity
  float4 *cd;   // colour r, g, b, depth (candidates: uncertainty in .x)
  float2 *uv;   // 2D mean
  int2 *rect;   // packed pixel rectangle (x0 | x1 << 16, y0 | y1 << 16)
  int *gid;
  int *rec;
  int *sid;     // [kBatch][k] class ids
  float *sw;    // [kBatch][k] class weights
  float *tail;
};

__host__ __device__ inline size_t batch_smem_bytes(int k) {
  size_t b = (size_t)kBatch * (16 + 16 + 8 + 8 + 4 + 4) + (size_t)kBatch * k * 8;
  return (b + 15) & ~(size_t)15;
}

__device__ __forceinline__ BatchSmem batch_smem(float4 *base, int k) {
  BatchSmem s;
  char *p = reinterpret_cast<char *>(base);
  s.co = reinterpret_cast<float4 *>(p); p += kBatch * 16;
  s.cd = reinterpret_cast<float4 *>(p); p += kBatch * 16;
  s.uv = reinterpret_cast<float2 *>(p); p += kBatch * 8;
  s.rect = reinterpret_cast<int2 *>(p); p += kBatch * 8;
  s.gid = reinterpret_cast<int *>(p); p += kBatch * 4;
  s.rec = reinterpret_cast<int *>(p); p += kBatch * 4;
  s.sid = reinterpret_cast<int *>(p); p += kBatch * k * 4;
  s.sw = reinterpret_cast<float *>(p);
  s.tail = reinterpret_cast<float *>(reinterpret_cast<char *>(base) + batch_smem_bytes(k));
  return s;
}

// Stage record r in batch slot `slot`.  If unc != nullptr the .x of the
// colour/depth slot carries unc[gid] instead of red.
__device__ __forceinline__ void load_batch_entry(const RecPtrs &rec, uint32_t r, int slot, int k,
                                                 const BatchSmem &bs, const float *__restrict__ rgb,
                                                 const int32_t *__restrict__ sem_ids,
                                                 const float *__restrict__ sem_w, const float *__restrict__ unc) {
  const int g = __ldg(rec.gid + r);
  bs.uv[slot] = __ldg(rec.uv + r);
  bs.co[slot] = __ldg(rec.co + r);
  const short4 rc = __ldg(rec.rect + r);
  bs.rect[slot] = make_int2((int)(uint16_t)rc.x | ((int)(uint16_t)rc.y << 16),
                            (int)(uint16_t)rc.z | ((int)(uint16_t)rc.w << 16));
  const float d = __ldg(rec.depth + r);
  if (unc) {
    bs.cd[slot] = make_float4(__ldg(unc + g), 0.f, 0.f, d);
  } else {
    bs.cd[slot] = make_float4(__ldg(rgb + 3 * g), __ldg(rgb + 3 * g + 1), __ldg(rgb + 3 * g + 2), d);
  }
  bs.gid[slot] = g;
  bs.rec[slot] = (int)r;
  if (sem_ids) {
    for (int l = 0; l < k; ++l) {
      bs.sid[slot * k + l] = __ldg(sem_ids + (size_t)g * k + l);
      bs.sw[slot * k + l] = __ldg(sem_w + (size_t)g * k + l);
    }
  }
}

__device__ __forceinline__ bool rect_holds(int2 rr, int px, int py) {
  const int x0 = rr.x & 0xffff, x1 = (int)((unsigned)rr.x >> 16);
  const int y0 = rr.y & 0xffff, y1 = (int)((unsigned)rr.y >> 16);
  return px >= x0 && px <= x1 && py >= y0 && py <= y1;
}

// The per-pixel opacity of one Gaussian at pixel centre (fpx, fpy):
// alpha = min(0.99, o exp(-0.5 d^T conic d)), d = mean - centre.  Evaluated
// with one rounding per operation (no contraction) so the skip / stop
// decisions match a plain IEEE evaluation of the same expression.  Returns
// false when the Gaussian is skipped (power > 0 or alpha < 1/255).
__device__ __forceinline__ bool gauss_alpha(float2 uv, float4 co, float fpx, float fpy, float &alpha, float &G,
                                            float &araw, float &dx, float &dy) {
  dx = __fsub_rn(uv.x, fpx);
  dy = __fsub_rn(uv.y, fpy);
  const float t1 = __fmul_rn(dx, dx), t2 = __fmul_rn(dy, dy), t3 = __fmul_rn(dx, dy);
  const float s = __fadd_rn(__fmul_rn(co.x, t1), __fmul_rn(co.z, t2));
  const float power = __fsub_rn(__fmul_rn(-0.5f, s), __fmul_rn(co.y, t3));
  if (power > 0.f) return false;
  G = expf(power);
  araw = __fmul_rn(co.w, G);
  alpha = araw < kAlphaMax ? araw : kAlphaMax;
  return !(alpha < kAlphaMin);
}

// Class chunking of the per-pixel accumulator: the stride is odd so that
// threads of a warp adding to the same class hit distinct banks; when M does
// not fit, chunks are multiples of 32 classes (one sign word per 32 classes
// never straddles two chunks).  `extra` bytes of shared memory are reserved.
inline void chunk_classes(int m, int threads, int k, bool has_sem, int *mchunk, int *mstride, int *nchunks,
                          size_t extra = 0) {
  if (!has_sem) { *mchunk = m; *mstride = 0; *nchunks = 1; return; }
  const size_t avail = kSmemBudget - batch_smem_bytes(k) - extra;
  const int max_stride = (int)(avail / ((size_t)threads * sizeof(float)));
  const int s = (m & 1) ? m : m + 1;
  if (s <= max_stride) { *mchunk = m; *mstride = s; *nchunks = 1; return; }
  const int c = ((max_stride - 1) / 32) * 32;
  *mchunk = c;
  *mstride = c + 1;
  *nchunks = (m + c - 1) / c;
}

struct FwdArgs {
  const uint2 *ranges;
  const uint32_t *pvals;
  RecPtrs rec;
  const float *rgb;
  const int32_t *sem_ids;
  const float *sem_w;
  int k, m, width, height, tiles_x;
  float *rgb_out, *depth_out, *sil_out, *sem;
  float *tfinal;
  uint32_t *nlast;
  int mchunk, mstride, nchunks;
  // fused mean-L1 mode
  const float *t_rgb, *t_depth, *t_sem;
  uint32_t *codes;   // per pixel: 2 planes (nonzero, negative) x (1 head word + nwc class words)
  int nwc;           // class words per plane = ceil(m / 32) when t_sem is given, else 0
  double *lpart;     // per tile: sum|d rgb|, sum|d depth|, sum|d sem|
  Counters *counters;
};

// Per-pixel sign-code layout of the fused L1 mode.
__host__ __device__ inline int code_words(int nwc) { return 2 * (1 + nwc); }

}  // namespace gs
