// objective_math.cuh -- per-pixel arithmetic of the Sec. 3.1 semantic term
// (entropy mask of Eq. 4, Hellinger distance of Eq. 5, cosine similarity)
// and its gradient with respect to the rendered distribution, shared by the
// objective on rendered maps and the fused render pass so that both take
// the same decisions in the same float32 operations.  Lanes of a warp hold
// the classes c = lane + 32 i of one pixel; the caller sums st[] over the
// warp (xor butterfly) between class_sums and pixel_term.
#pragma once

#include "gs_internal.cuh"

namespace gs {

constexpr float kObjLamHd = 0.8f, kObjLamCos = 0.2f;
constexpr float kObjEpsSqrt = 1e-12f, kObjEpsDiv = 1e-12f;
constexpr int kObjMI = 4;  // class registers per lane of the cached paths (m <= 128)

// Per-class values kept between the sums and the gradient: sqrt(Q_c + e) and
// 1 / sqrt(max(P_c, 0) + e), from the reciprocal square root (x rsqrt(x)
// for the root; a few ulp, far inside the objective's tolerances).
struct ClassRoots {
  float sq, rp;
};

// Per-class contributions to a pixel's sums: entropy of Q (fast log: its
// absolute error stays below 1e-5 over a pixel, well off the ln k
// threshold's rounding band), squared Hellinger difference, |Q|^2, |P|^2,
// Q.P (st[0..4]).
__device__ __forceinline__ ClassRoots class_roots(float qv, float pv) {
  const float xq = fmaxf(qv, 0.f) + kObjEpsSqrt;
  return ClassRoots{xq * rsqrtf(xq), rsqrtf(fmaxf(pv, 0.f) + kObjEpsSqrt)};
}

__device__ __forceinline__ ClassRoots class_sums(float qv, float pv, float (&st)[5]) {
  if (qv > 0.f) st[0] -= qv * __logf(qv);
  const ClassRoots r = class_roots(qv, pv);
  const float d = r.sq - (fmaxf(pv, 0.f) + kObjEpsSqrt) * r.rp;
  st[1] = fmaf(d, d, st[1]);
  st[2] = fmaf(qv, qv, st[2]);
  st[3] = fmaf(pv, pv, st[3]);
  st[4] = fmaf(qv, pv, st[4]);
  return r;
}

struct PixelTerm {
  bool keep;    // entropy mask (and pixel inside the image)
  bool hd, cs;  // Hellinger distance / cosine denominators above the floor
  float value;  // 0.8 D_HD + 0.2 (1 - cos)
  float inv4d;  // 1 / (4 D_HD)
  float inv_den, cos_pp;  // 1 / (|Q| |P|), cos / |P|^2
};

// The pixel's term from its warp-summed class sums (Eq. 4 mask, Eq. 5
// Hellinger distance, cosine similarity), with the per-pixel factors of
// its gradient.
__device__ __forceinline__ PixelTerm pixel_term(const float (&st)[5], bool ok, float log_k) {
  PixelTerm t;
  t.keep = ok && st[0] < log_k;
  const float dist = sqrtf(0.5f * st[1]);
  const float den = sqrtf(st[2]) * sqrtf(st[3]);
  t.hd = dist > kObjEpsDiv;
  t.cs = den > kObjEpsDiv;
  const float cosv = t.cs ? st[4] / den : 0.f;
  t.value = kObjLamHd * dist + kObjLamCos * (1.f - cosv);
  t.inv4d = t.hd ? 1.f / (4.f * dist) : 0.f;
  t.inv_den = t.cs ? 1.f / den : 0.f;
  t.cos_pp = t.cs ? cosv / fmaxf(st[3], kObjEpsDiv) : 0.f;
  return t;
}

// d term / d P_c over the pixel count, for a kept pixel:
// 0.8 (1 - sqrt(Q_c) / sqrt(P_c)) / (4 D_HD) - 0.2 (Q_c / (|Q||P|) - cos P_c / |P|^2).
__device__ __forceinline__ float class_grad(float qv, float pv, ClassRoots r, const PixelTerm &t, float inv_n) {
  const float dhd = (t.hd && pv >= 0.f) ? (1.f - r.sq * r.rp) * t.inv4d : 0.f;
  const float dcos = t.cs ? fmaf(qv, t.inv_den, -pv * t.cos_pp) : 0.f;
  return (kObjLamHd * dhd - kObjLamCos * dcos) * inv_n;
}

// Warp sum of the five class sums (xor butterfly: every lane gets the totals).
__device__ __forceinline__ void warp_sum5(float (&st)[5]) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int j = 0; j < 5; ++j) st[j] += __shfl_xor_sync(0xffffffffu, st[j], o);
}

}  // namespace gs
