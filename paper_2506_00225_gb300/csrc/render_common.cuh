// render_common.cuh -- pieces shared by the forward, backward and candidate
// blend kernels: warp footprints inside a tile, shared-memory batch staging
// of a tile's sorted Gaussians with per-warp visibility masks, the per-pixel
// opacity rule and a transposed warp reduction.
#pragma once

#include "gs_internal.cuh"

namespace gs {

constexpr int kBatch = 64;                       // Gaussians staged per batch
constexpr float kTStop = 0.0001f;                // transmittance stop
constexpr float kAlphaMin = 1.0f / 255.0f;       // skip threshold
constexpr float kAlphaMax = 0.99f;               // opacity cap
constexpr float kSilMinLoss = 0.99f;             // silhouette threshold of the Sec. 3.1 objective
constexpr size_t kSmemBudget = 112 * 1024;       // per CTA: two 256-thread CTAs per SM

// Each warp owns an 8 x (4 PPT) pixel block of the tile; lane l sits at
// column l % 8 and rows l / 8 + 4 i (i < PPT) of its block, so a thread
// handles PPT pixels that share every staged load.
template <int TW, int TH, int PPT = 1>
struct Footprint {
  static constexpr int kPix = TW * TH;
  static constexpr int kThreads = kPix / PPT;
  static constexpr int kWarps = kThreads / 32;
  static constexpr int kBH = 4 * PPT;  // warp block height
  static constexpr int kWX = TW / 8;   // warp blocks per tile row
  static_assert(TW % 8 == 0 && TH % kBH == 0, "tile must be a multiple of the warp block");
  // tile-local pixel i of this thread
  __device__ static int lx() { return ((threadIdx.x >> 5) % kWX) * 8 + (threadIdx.x & 7); }
  __device__ static int ly(int i) { return ((threadIdx.x >> 5) / kWX) * kBH + ((threadIdx.x & 31) >> 3) + 4 * i; }
  // thread holding tile-local pixel p (raster order); PPT = 1 only
  __device__ static int thread_of(int p) {
    const int x = p % TW, y = p / TW;
    return ((y >> 2) * kWX + (x >> 3)) * 32 + (y & 3) * 8 + (x & 7);
  }
  // bit w set when box [bx0,bx1] x [by0,by1] (tile-local pixels) meets warp w's block
  __device__ static uint32_t warp_mask(int bx0, int bx1, int by0, int by1) {
    uint32_t m = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
      const int x0 = (w % kWX) * 8, y0 = (w / kWX) * kBH;
      if (bx0 <= x0 + 7 && bx1 >= x0 && by0 <= y0 + kBH - 1 && by1 >= y0) m |= 1u << w;
    }
    return m;
  }
};

// Fire-and-forget float add to global memory through a generic pointer that
// holds a global address (as staged in shared memory): the reduction the
// compiler cannot emit for a generic atomicAdd without a returned value.
__device__ __forceinline__ void red_add_global(float *p, float v) {
  asm volatile("red.global.add.f32 [%0], %1;" ::"l"(__cvta_generic_to_global(p)), "f"(v) : "memory");
}

struct RecPtrs {
  const float2 *uv;
  const float4 *co;    // conic a, b, c, opacity
  const short4 *box;   // alpha box
  const float4 *cd;    // r, g, b, depth
  const float *unc;
  const int2 *sem;     // [k] (id, weight bits)
  const int32_t *gid;
};

inline RecPtrs rec_ptrs(const WsPtrs &P) {
  return RecPtrs{P.rec_uv, P.rec_conic, P.rec_box, P.rec_cd, P.rec_unc, P.rec_sem, P.rec_gid};
}

// Shared-memory view of one staged batch (struct of arrays) plus the tail
// region after it.
struct BatchSmem {
  float4 *co;
  float4 *cd;      // r, g, b, depth (candidates: uncertainty in .x)
  float2 *uv;
  int2 *box;       // packed alpha box (x0 | x1 << 16, y0 | y1 << 16), image pixels
  int2 *sem;       // [kBatch][k]
  uint32_t *wmask; // warps whose block meets the box
  int *gid;
  int *rec;
  float *tail;
};

__host__ __device__ inline size_t batch_smem_bytes(int k) {
  size_t b = (size_t)kBatch * (16 + 16 + 8 + 8 + 4 + 4 + 4) + (size_t)kBatch * k * 8;
  return (b + 15) & ~(size_t)15;
}

__device__ __forceinline__ BatchSmem batch_smem(float4 *base, int k) {
  BatchSmem s;
  char *p = reinterpret_cast<char *>(base);
  s.co = reinterpret_cast<float4 *>(p); p += kBatch * 16;
  s.cd = reinterpret_cast<float4 *>(p); p += kBatch * 16;
  s.uv = reinterpret_cast<float2 *>(p); p += kBatch * 8;
  s.box = reinterpret_cast<int2 *>(p); p += kBatch * 8;
  s.sem = reinterpret_cast<int2 *>(p); p += (size_t)kBatch * k * 8;
  s.wmask = reinterpret_cast<uint32_t *>(p); p += kBatch * 4;
  s.gid = reinterpret_cast<int *>(p); p += kBatch * 4;
  s.rec = reinterpret_cast<int *>(p);
  s.tail = reinterpret_cast<float *>(reinterpret_cast<char *>(base) + batch_smem_bytes(k));
  return s;
}

// Stage record r in batch slot `slot` of the tile whose top-left pixel is
// (ox, oy).  With use_unc the .x of the colour slot carries the uncertainty.
template <int TW, int TH, int PPT = 1>
__device__ __forceinline__ void stage_record(const RecPtrs &rec, uint32_t r, int slot, int k, int ox, int oy,
                                             const BatchSmem &bs, bool use_sem, bool use_unc) {
  const short4 b = __ldg(rec.box + r);
  bs.uv[slot] = __ldg(rec.uv + r);
  bs.co[slot] = __ldg(rec.co + r);
  float4 cd = __ldg(rec.cd + r);
  if (use_unc) cd.x = __ldg(rec.unc + r);
  bs.cd[slot] = cd;
  bs.box[slot] = make_int2((int)(uint16_t)b.x | ((int)(uint16_t)b.y << 16),
                           (int)(uint16_t)b.z | ((int)(uint16_t)b.w << 16));
  bs.wmask[slot] = b.x > b.y ? 0u : Footprint<TW, TH, PPT>::warp_mask(b.x - ox, b.y - ox, b.z - oy, b.w - oy);
  bs.gid[slot] = __ldg(rec.gid + r);
  bs.rec[slot] = (int)r;
  if (use_sem) {
    const int2 *src = rec.sem + (size_t)r * k;
    for (int l = 0; l < k; ++l) bs.sem[slot * k + l] = __ldg(src + l);
  }
}

// Lane masks of a staged record for every warp of a tile: bit l of
// masks[(w PPT + i) stride] is set when lane l's i-th pixel of warp w lies in
// the record's alpha box (image pixels b; tile origin ox, oy).  A warp's lanes
// hold an 8 x 4 PPT block, lane l at column l % 8 and rows l / 8 + 4 i.  With
// the staged records consecutive (stride = batch size), the threads staging
// consecutive records write consecutive words (no bank conflicts).
// Lanes of an 8 x 4 pixel block at (x0, y0) (lane l at column l % 8, row
// l / 8) whose pixel lies in the box b = (x_lo, x_hi, y_lo, y_hi).
__device__ __forceinline__ uint32_t block_lane_mask(short4 b, int x0, int y0) {
  const int cl = max((int)b.x - x0, 0), ch = min((int)b.y - x0, 7);
  const int rl = max((int)b.z - y0, 0), rh = min((int)b.w - y0, 3);
  if (cl > ch || rl > rh) return 0u;
  const uint32_t cols = (0xffu >> (7 - ch)) & (0xffu << cl);
  const uint32_t rows = (0xffffffffu >> (8 * (3 - rh))) & (0xffffffffu << (8 * rl));
  return (cols * 0x01010101u) & rows;
}

template <int TW, int TH, int PPT = 1>
__device__ __forceinline__ void lane_masks(short4 b, int ox, int oy, uint32_t *masks, int stride) {
  using FP = Footprint<TW, TH, PPT>;
#pragma unroll
  for (int w = 0; w < FP::kWarps; ++w) {
#pragma unroll
    for (int i = 0; i < PPT; ++i)  // rows 4 i .. 4 i + 3 of warp w's block
      masks[(w * PPT + i) * stride] =
          block_lane_mask(b, ox + (w % FP::kWX) * 8, oy + (w / FP::kWX) * FP::kBH + 4 * i);
  }
}

// Pixel inside the packed box (x0 | x1 << 16, y0 | y1 << 16).
__device__ __forceinline__ bool box_holds(int2 bb, int px, int py) {
  const int x0 = bb.x & 0xffff, x1 = (int)((unsigned)bb.x >> 16);
  const int y0 = bb.y & 0xffff, y1 = (int)((unsigned)bb.y >> 16);
  return (unsigned)(px - x0) <= (unsigned)(x1 - x0) && (unsigned)(py - y0) <= (unsigned)(y1 - y0);
}

// The per-pixel opacity of one Gaussian at pixel centre (fpx, fpy):
// alpha = min(0.99, o exp(-0.5 d^T conic d)), d = mean - centre, evaluated
// in a fixed fused order (the same instructions in every kernel, so the
// forward, backward and candidate kernels take identical decisions).
// Returns false when skipped (power > 0 or alpha < 1/255).
__device__ __forceinline__ bool gauss_alpha(float2 uv, float4 co, float fpx, float fpy, float &alpha, float &G,
                                            float &araw, float &dx, float &dy) {
  dx = __fsub_rn(uv.x, fpx);
  dy = __fsub_rn(uv.y, fpy);
  const float q = __fmaf_rn(co.x, __fmul_rn(dx, dx), __fmul_rn(co.z, __fmul_rn(dy, dy)));
  const float power = __fmaf_rn(-0.5f, q, -__fmul_rn(co.y, __fmul_rn(dx, dy)));
  if (power > 0.f) return false;
  G = __expf(power);
  araw = __fmul_rn(co.w, G);
  alpha = araw < kAlphaMax ? araw : kAlphaMax;
  return !(alpha < kAlphaMin);
}

// Transposed warp sum of NV values per lane (NV = 16 or 32): exchange halves
// of the value set at each butterfly level, so NV - 1 (+1 for NV = 16)
// shuffles replace 5 NV.  Afterwards lane l holds the warp total of value
// reduced_index<NV>() (l & 15 for NV = 16, l for NV = 32).
template <int NV>
__device__ __forceinline__ float warp_reduce_scatter(float (&v)[NV]) {
  const uint32_t lane = lane_id();
  if constexpr (NV == 32) {
    const bool hi = lane & 16;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const float send = hi ? v[i] : v[i + 16];
      const float keep = hi ? v[i + 16] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
  }
  {
    const bool hi = lane & 8;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float send = hi ? v[i] : v[i + 8];
      const float keep = hi ? v[i + 8] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
  }
  {
    const bool hi = lane & 4;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float send = hi ? v[i] : v[i + 4];
      const float keep = hi ? v[i + 4] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
  }
  {
    const bool hi = lane & 2;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const float send = hi ? v[i] : v[i + 2];
      const float keep = hi ? v[i + 2] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
    }
  }
  {
    const bool hi = lane & 1;
    const float send = hi ? v[0] : v[1];
    const float keep = hi ? v[1] : v[0];
    v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 1);
  }
  if constexpr (NV == 16) v[0] += __shfl_xor_sync(0xffffffffu, v[0], 16);
  return v[0];
}

template <int NV>
__device__ __forceinline__ int reduced_index() {
  return NV == 32 ? (int)lane_id() : (int)(lane_id() & 15);
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

// L2 prefetch of [p, p + bytes) clipped to 16-byte granules inside
// [base, base + total).
__device__ __forceinline__ void prefetch_l2(const void *base, size_t total, const void *p, size_t bytes) {
  const uintptr_t b = reinterpret_cast<uintptr_t>(base);
  const uintptr_t lo = (reinterpret_cast<uintptr_t>(p) + 15) & ~(uintptr_t)15;
  uintptr_t hi = (reinterpret_cast<uintptr_t>(p) + bytes) & ~(uintptr_t)15;
  const uintptr_t end = (b + total) & ~(uintptr_t)15;
  if (hi > end) hi = end;
  if (lo < b || hi <= lo) return;
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(lo), "r"((uint32_t)(hi - lo)) : "memory");
}

// Asynchronous global -> shared copies (sm_80+ cp.async), used to stage the
// next batch while the current one is processed.
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
               "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
               "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
               "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Shared-memory layout of one pass-2 batch buffer: mean, conic, pixel box
// (recomputation mode), k sem pairs.
__host__ __device__ inline size_t sem_batch_bytes(int k) {
  return (size_t)kBatch * (8 + 16 + 8) + (size_t)kBatch * k * 8;
}

// Adds w * weight to the accumulator slot of each of the Gaussian's k
// (class, weight) entries that falls in the class chunk [c_lo, c_lo + mc).
// Entry l of the Gaussian is e[l * es] (staged entry-major: the threads that
// stage consecutive Gaussians write consecutive words).  K > 0 fixes k at
// compile time.
template <int K>
__device__ __forceinline__ void scatter_classes(float *row, const int2 *e, int k, int c_lo, int mc, float w,
                                                int es) {
  const int n = K > 0 ? K : k;
#pragma unroll
  for (int l = 0; l < n; ++l) {
    const int2 v = e[l * es];
    const int id = v.x - c_lo;
    if ((unsigned)id < (unsigned)mc) row[id] = fmaf(w, __int_as_float(v.y), row[id]);
  }
}

// The same adds with the k = 3 read-modify-writes in flight together: all
// three slots are read before any is written, and an id repeated within the
// Gaussian takes the earlier entry's result as its input, so every slot ends
// with the roundings and the order of scatter_classes.  Straight-line code
// (no branch on the ids).  Other k take scatter_classes.
template <int K>
__device__ __forceinline__ void scatter_classes_ilp(float *row, const int2 *e, int k, int c_lo, int mc, float w,
                                                    int es) {
  if constexpr (K == 3) {
    const int2 e0 = e[0], e1 = e[es], e2 = e[2 * es];
    const int i0 = e0.x - c_lo, i1 = e1.x - c_lo, i2 = e2.x - c_lo;
    const bool k0 = (unsigned)i0 < (unsigned)mc, k1 = (unsigned)i1 < (unsigned)mc, k2 = (unsigned)i2 < (unsigned)mc;
    const float o0 = k0 ? row[i0] : 0.f, o1 = k1 ? row[i1] : 0.f, o2 = k2 ? row[i2] : 0.f;
    const float n0 = fmaf(w, __int_as_float(e0.y), o0);
    const float n1 = fmaf(w, __int_as_float(e1.y), i1 == i0 ? n0 : o1);
    const float n2 = fmaf(w, __int_as_float(e2.y), i2 == i1 ? n1 : (i2 == i0 ? n0 : o2));
    if (k0) row[i0] = n0;
    if (k1) row[i1] = n1;
    if (k2) row[i2] = n2;
  } else {
    scatter_classes<K>(row, e, k, c_lo, mc, w, es);
  }
}

// Staged-entry mark for k >= 4: the thread that staged a Gaussian's k
// (class, weight) entries, once its copies have landed, sets bit 31 of the
// first id when two of the ids are equal (valid ids are non-negative, so the
// bit is free).  scatter_classes_marked reads it.
template <int K>
__device__ __forceinline__ void mark_repeated_ids(int2 *e, int es) {
  if constexpr (K >= 4) {
    int id[K];
#pragma unroll
    for (int a = 0; a < K; ++a) id[a] = e[a * es].x;
    bool rep = false;
#pragma unroll
    for (int a = 1; a < K; ++a)
#pragma unroll
      for (int b = 0; b < a; ++b) rep |= id[a] == id[b];
    if (rep) e[0].x = (int)((uint32_t)e[0].x | 0x80000000u);
  }
}

// scatter_classes over entries marked by mark_repeated_ids: a Gaussian
// without repeated ids (the warp-uniform common case) has all K
// read-modify-writes in flight together; one with repeated ids takes them
// one after another.  Either way each slot ends as in scatter_classes.
// k = 3 takes scatter_classes_ilp (needs no mark).
template <int K>
__device__ __forceinline__ void scatter_classes_marked(float *row, const int2 *e, int k, int c_lo, int mc, float w,
                                                       int es) {
  if constexpr (K >= 4) {
    int2 v[K];
#pragma unroll
    for (int l = 0; l < K; ++l) v[l] = e[l * es];
    if (v[0].x >= 0) {
      float o[K];
#pragma unroll
      for (int l = 0; l < K; ++l) {
        const int id = v[l].x - c_lo;
        o[l] = (unsigned)id < (unsigned)mc ? row[id] : 0.f;
      }
#pragma unroll
      for (int l = 0; l < K; ++l) {
        const int id = v[l].x - c_lo;
        if ((unsigned)id < (unsigned)mc) row[id] = fmaf(w, __int_as_float(v[l].y), o[l]);
      }
    } else {
      v[0].x = (int)((uint32_t)v[0].x & 0x7fffffffu);
#pragma unroll
      for (int l = 0; l < K; ++l) {
        const int id = v[l].x - c_lo;
        if ((unsigned)id < (unsigned)mc) row[id] = fmaf(w, __int_as_float(v[l].y), row[id]);
      }
    }
  } else {
    scatter_classes_ilp<K>(row, e, k, c_lo, mc, w, es);
  }
}

struct FwdArgs {
  const uint2 *ranges;
  const uint32_t *pvals;
  RecPtrs rec;
  int k, m, width, height, tiles_x;
  float *rgb_out, *depth_out, *sil_out, *sem;
  float *tfinal;
  uint32_t *nlast;
  int mchunk, mstride, nchunks;
  int objective;     // 1: Sec. 3.1 objective (silhouette-masked geometry; semantic term by k_sem_objective)
  float *semg;       // objective mode: d(objective)/d(sem_w) [n][k], accumulated by the semantic pass
  // fused mean-L1 mode
  const float *t_rgb, *t_depth, *t_sem;
  uint32_t *codes;   // per pixel: (nonzero, negative) word pairs: head (rgb, depth bits), then nwc class words
  int nwc;           // class words per plane = ceil(m / 32)
  double *lpart;     // per tile: sum|d rgb|, sum|d depth|, sum|d sem|
  float *loss;       // written by the last tile of the semantic pass (fused-loss modes)
  int blend_ppt;     // pixels per thread of the blend pass (1 or 2)
  double npix_d;     // pixels of the view
  Counters *counters;
  // contributor bitmasks (pass 1 writes, pass 2 and the adjoint read)
  const uint32_t *mask_off;
  uint32_t *masks;
  uint32_t mask_units;
};

// The fused-loss semantic passes end each tile with this: the tile's three
// sums are written; the CTA that takes the last of the ntiles tickets adds
// all tiles' sums (a fixed order: deterministic) and writes the loss, then
// leaves the ticket counter at 0 for the next launch.  Mean-L1 mode: rgb / (3 npix) +
// depth / npix + sem / (npix m); Sec. 3.1 objective mode: 0.5 rgb + depth
// (sums over the silhouette mask) + sem / npix.  No CTA waits on another.
template <int THREADS>
__device__ __forceinline__ void finish_loss(const FwdArgs &a, int objective, uint32_t ntiles) {
  constexpr int WARPS = THREADS / 32;
  __shared__ int s_last;
  __shared__ double s_red[3][WARPS];
  if (threadIdx.x == 0) {
    __threadfence();  // this tile's sums before the ticket
    s_last = atomicAdd(&a.counters->tiles_done, 1u) == ntiles - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double s[3] = {0.0, 0.0, 0.0};
  for (uint32_t t = threadIdx.x; t < ntiles; t += THREADS)
    for (int i = 0; i < 3; ++i) s[i] += __ldcg(a.lpart + 3 * (size_t)t + i);
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s[i] += __shfl_xor_sync(0xffffffffu, s[i], o);
    if ((threadIdx.x & 31) == 0) s_red[i][threadIdx.x >> 5] = s[i];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t[3] = {0.0, 0.0, 0.0};
    for (int w = 0; w < WARPS; ++w)
      for (int i = 0; i < 3; ++i) t[i] += s_red[i][w];
    const double l = objective ? 0.5 * t[0] + t[1] + t[2] / a.npix_d
                               : t[0] / (3.0 * a.npix_d) + t[1] / a.npix_d + t[2] / (a.npix_d * a.m);
    *a.loss = (float)l;
    a.counters->tiles_done = 0u;
  }
}

// Per-pixel sign-code layout of the fused L1 mode.
__host__ __device__ inline int code_words(int nwc) { return 2 * (1 + nwc); }

// Host side (render_fwd.cu): the blend arguments of the mapping view, the
// blend pass alone (fused-loss or plain form), and the per-tile loss
// reduction.
FwdArgs fwd_args(const Layout &L, const WsPtrs &P, int pbuf, const gs_scene &sc);
cudaError_t launch_blend_objective(const Layout &L, const FwdArgs &a, int grid, cudaStream_t s);
cudaError_t launch_blend_plain(const Layout &L, const FwdArgs &a, int grid, cudaStream_t s);
cudaError_t launch_loss_final(const double *lpart, int ntiles, double npix, double m, int has_sem, int objective,
                              float *loss, cudaStream_t s);

}  // namespace gs
