// project.cu -- per-(view, Gaussian) EWA projection, visibility compaction
// (count / scan / emit passes for several views, one look-back pass for a
// single view) and the single-CTA exclusive scan used for compaction offsets.
//
// Sec. 3.1 "Gaussian Mapping" (transform to camera space, project to the
// image plane); the EWA projection with 0.3 px^2 dilation, 3-sigma radius and
// frustum clamp is the 3DGS prior art the paper adopts via SplaTAM.
//
// This translation unit is compiled with -fmad=false: every expression below
// is evaluated as written (one rounding per operation), so the pixel and tile
// rectangles -- and therefore the tile lists -- are reproducible bit for bit.
#include "gs_internal.cuh"

namespace gs {

struct Proj {
  float u, v, ca, cb, cc, depth;
  int x0, x1, y0, y1;
  float A, C;  // dilated 2D covariance diagonal (for the alpha box)
};

// Pixel box outside which alpha < 1/255 for sure: the axis-aligned box of the
// ellipse q(d) <= 2 ln(255 o) (half-extents sqrt(2 ln(255 o) Sigma_xx),
// sqrt(.. Sigma_yy)), widened by 0.1 % plus one pixel, clipped to the pixel
// rectangle.  Inside the rectangle but outside this box every pixel would be
// skipped by the alpha < 1/255 rule, so the blend kernels may skip it without
// evaluating alpha; tile lists still use the pixel rectangle.  Empty when
// x0 > x1.
__device__ __forceinline__ short4 alpha_box(const Proj &p, float opacity) {
  if (!(opacity >= 1.f / 255.f)) return make_short4(1, 0, 1, 0);
  const float L = 2.f * logf(255.f * opacity);
  const float hx = sqrtf(fmaxf(L, 0.f) * p.A) * 1.001f + 1.f;
  const float hy = sqrtf(fmaxf(L, 0.f) * p.C) * 1.001f + 1.f;
  const float bx0 = fmaxf((float)p.x0, floorf(p.u - 0.5f - hx)), bx1 = fminf((float)p.x1, ceilf(p.u - 0.5f + hx));
  const float by0 = fmaxf((float)p.y0, floorf(p.v - 0.5f - hy)), by1 = fminf((float)p.y1, ceilf(p.v - 0.5f + hy));
  if (!(bx0 <= bx1) || !(by0 <= by1)) return make_short4(1, 0, 1, 0);
  return make_short4((short)bx0, (short)bx1, (short)by0, (short)by1);
}

// Projects one Gaussian into camera `c`; returns false when culled.
__device__ __forceinline__ bool project_gaussian(float mx, float my, float mz, float sx, float sy, float sz,
                                                 float4 q, const DevCam &c, Proj &o) {
  const float tx = ((c.r[0] * mx + c.r[1] * my) + c.r[2] * mz) + c.t[0];
  const float ty = ((c.r[3] * mx + c.r[4] * my) + c.r[5] * mz) + c.t[1];
  const float tz = ((c.r[6] * mx + c.r[7] * my) + c.r[8] * mz) + c.t[2];
  if (!(isfinite(tx) && isfinite(ty) && isfinite(tz))) return false;
  if (!(tz > c.near_plane)) return false;
  const float n2 = ((q.x * q.x + q.y * q.y) + q.z * q.z) + q.w * q.w;
  if (!(n2 > 0.f) || !isfinite(n2)) return false;
  const float qn = sqrtf(n2);
  const float w = q.x / qn, x = q.y / qn, y = q.z / qn, z = q.w / qn;
  const float xx = x * x, yy = y * y, zz = z * z, xy = x * y, xz = x * z, yz = y * z;
  const float wx = w * x, wy = w * y, wz = w * z;
  const float R0 = 1.f - 2.f * (yy + zz), R1 = 2.f * (xy - wz), R2 = 2.f * (xz + wy);
  const float R3 = 2.f * (xy + wz), R4 = 1.f - 2.f * (xx + zz), R5 = 2.f * (yz - wx);
  const float R6 = 2.f * (xz - wy), R7 = 2.f * (yz + wx), R8 = 1.f - 2.f * (xx + yy);
  // M = R diag(s)
  const float M0 = R0 * sx, M1 = R1 * sy, M2 = R2 * sz;
  const float M3 = R3 * sx, M4 = R4 * sy, M5 = R5 * sz;
  const float M6 = R6 * sx, M7 = R7 * sy, M8 = R8 * sz;
  // Sigma3 = M M^T (rows i <= j)
  const float s00 = (M0 * M0 + M1 * M1) + M2 * M2;
  const float s01 = (M0 * M3 + M1 * M4) + M2 * M5;
  const float s02 = (M0 * M6 + M1 * M7) + M2 * M8;
  const float s11 = (M3 * M3 + M4 * M4) + M5 * M5;
  const float s12 = (M3 * M6 + M4 * M7) + M5 * M8;
  const float s22 = (M6 * M6 + M7 * M7) + M8 * M8;
  // pinhole Jacobian at the frustum-clamped mean
  const float limx = 1.3f * ((0.5f * (float)c.width) / c.fx);
  const float limy = 1.3f * ((0.5f * (float)c.height) / c.fy);
  const float rx = tx / tz, ry = ty / tz;
  const float rxc = rx < -limx ? -limx : (rx > limx ? limx : rx);
  const float ryc = ry < -limy ? -limy : (ry > limy ? limy : ry);
  const float txc = rxc * tz, tyc = ryc * tz;
  const float tz2 = tz * tz;
  const float J00 = c.fx / tz;
  const float J02 = -(c.fx * txc) / tz2;
  const float J11 = c.fy / tz;
  const float J12 = -(c.fy * tyc) / tz2;
  // T = J W
  const float T0 = J00 * c.r[0] + J02 * c.r[6];
  const float T1 = J00 * c.r[1] + J02 * c.r[7];
  const float T2 = J00 * c.r[2] + J02 * c.r[8];
  const float T3 = J11 * c.r[3] + J12 * c.r[6];
  const float T4 = J11 * c.r[4] + J12 * c.r[7];
  const float T5 = J11 * c.r[5] + J12 * c.r[8];
  // U = T Sigma3 (Sigma3 column j = (s0j, s1j, s2j) with the mirrored entries)
  const float U0 = (T0 * s00 + T1 * s01) + T2 * s02;
  const float U1 = (T0 * s01 + T1 * s11) + T2 * s12;
  const float U2 = (T0 * s02 + T1 * s12) + T2 * s22;
  const float U3 = (T3 * s00 + T4 * s01) + T5 * s02;
  const float U4 = (T3 * s01 + T4 * s11) + T5 * s12;
  const float U5 = (T3 * s02 + T4 * s12) + T5 * s22;
  const float A = ((U0 * T0 + U1 * T1) + U2 * T2) + 0.3f;
  const float B = (U0 * T3 + U1 * T4) + U2 * T5;
  const float C = ((U3 * T3 + U4 * T4) + U5 * T5) + 0.3f;
  if (!(isfinite(A) && isfinite(B) && isfinite(C))) return false;
  const float det = A * C - B * B;
  if (!(det > 0.f)) return false;
  const float inv = 1.f / det;
  o.ca = C * inv;
  o.cb = -B * inv;
  o.cc = A * inv;
  const float mid = 0.5f * (A + C);
  const float disc = mid * mid - det;
  const float lam = mid + sqrtf(disc > 0.1f ? disc : 0.1f);
  const float rad = ceilf(3.f * sqrtf(lam));
  o.u = (c.fx * tx) / tz + c.cx;
  o.v = (c.fy * ty) / tz + c.cy;
  if (!(isfinite(o.u) && isfinite(o.v))) return false;
  float xlo = ceilf((o.u - 0.5f) - rad);
  float xhi = floorf((o.u - 0.5f) + rad);
  float ylo = ceilf((o.v - 0.5f) - rad);
  float yhi = floorf((o.v - 0.5f) + rad);
  if (xlo < 0.f) xlo = 0.f;
  if (ylo < 0.f) ylo = 0.f;
  if (xhi > (float)(c.width - 1)) xhi = (float)(c.width - 1);
  if (yhi > (float)(c.height - 1)) yhi = (float)(c.height - 1);
  if (!(xlo <= xhi) || !(ylo <= yhi)) return false;
  o.x0 = (int)xlo; o.x1 = (int)xhi; o.y0 = (int)ylo; o.y1 = (int)yhi;
  o.depth = tz;
  o.A = A;
  o.C = C;
  return true;
}

__global__ void k_setup_views(CamTable tab, int n_views, DevCam *cams, uint32_t *tile_off, uint32_t total_tiles,
                              Counters *counters, int reset_status) {
  int i = threadIdx.x;
  if (i < n_views) {
    cams[i] = tab.cam[i];
    tile_off[i] = tab.cam[i].tile_off;
  }
  if (i == 0) {
    tile_off[n_views] = total_tiles;
    if (reset_status) {
      counters->status = 0u;
      counters->grp_records = 0u;
      counters->grp_pairs = 0u;
    } else {
      counters->grp_records = max(counters->grp_records, counters->n_records);
      counters->grp_pairs = max(counters->grp_pairs, counters->n_pairs);
    }
    counters->n_records = 0u;
    counters->n_pairs = 0u;
    counters->n_contrib = 0u;
    counters->tiles_done = 0u;
  }
}

// Loads Gaussian g's projection inputs.
struct GIn {
  float mx, my, mz, sx, sy, sz;
  float4 q;
};
__device__ __forceinline__ GIn load_gaussian(const gs_scene &sc, int g) {
  GIn r;
  r.mx = __ldg(sc.means + 3 * g); r.my = __ldg(sc.means + 3 * g + 1); r.mz = __ldg(sc.means + 3 * g + 2);
  r.sx = __ldg(sc.scales + 3 * g); r.sy = __ldg(sc.scales + 3 * g + 1); r.sz = __ldg(sc.scales + 3 * g + 2);
  r.q = __ldg(reinterpret_cast<const float4 *>(sc.quats) + g);
  return r;
}

// The Gaussians of one projection block are read once and projected for a
// group of up to kViewsPerCta views (grid.y runs over the view groups).
constexpr int kViewsPerCta = 16;

// Pass 1: count visible Gaussians per (view, projection block).
__global__ void __launch_bounds__(kProjThreads) k_project_count(gs_scene sc, const DevCam *cams, int nb, int n_views,
                                                                uint32_t *blockcnt) {
  // per view: a warp sum, then one shared-memory add per warp (the counts
  // are totals, so no scan and no barrier per view)
  __shared__ uint32_t s_cnt[kViewsPerCta];
  const int b = blockIdx.x;
  const int v0 = blockIdx.y * kViewsPerCta, v1 = min(n_views, v0 + kViewsPerCta);
  if ((int)threadIdx.x < kViewsPerCta) s_cnt[threadIdx.x] = 0u;
  __syncthreads();
  const int g0 = b * kProjBlock + threadIdx.x * kProjItems;
  GIn in[kProjItems];
#pragma unroll
  for (int i = 0; i < kProjItems; ++i)
    if (g0 + i < sc.n) in[i] = load_gaussian(sc, g0 + i);
  for (int v = v0; v < v1; ++v) {
    const DevCam c = cams[v];
    uint32_t cnt = 0;
#pragma unroll
    for (int i = 0; i < kProjItems; ++i) {
      if (g0 + i < sc.n) {
        Proj p;
        cnt += project_gaussian(in[i].mx, in[i].my, in[i].mz, in[i].sx, in[i].sy, in[i].sz, in[i].q, c, p) ? 1u
                                                                                                          : 0u;
      }
    }
    cnt = __reduce_add_sync(0xffffffffu, cnt);
    if (lane_id() == 0 && cnt) atomicAdd(&s_cnt[v - v0], cnt);
  }
  __syncthreads();
  if ((int)threadIdx.x < v1 - v0) blockcnt[(v0 + threadIdx.x) * nb + b] = s_cnt[threadIdx.x];
}

// Writes visible record r (Gaussian g projected into view v) and its
// (view, depth) sort key.
__device__ __forceinline__ void write_record(const gs_scene &sc, const WsPtrs &P, uint32_t r, int g, int v,
                                             const Proj &p) {
  const float op = __ldg(sc.opacity + g);
  P.rec_uv[r] = make_float2(p.u, p.v);
  P.rec_conic[r] = make_float4(p.ca, p.cb, p.cc, op);
  P.rec_depth[r] = p.depth;
  P.rec_rect[r] = make_short4((short)p.x0, (short)p.x1, (short)p.y0, (short)p.y1);
  P.rec_gid[r] = g;
  P.rec_view[r] = v;
  // blend record: alpha box, colour + depth, uncertainty, sparse semantics
  P.rec_box[r] = alpha_box(p, op);
  P.rec_cd[r] = make_float4(sc.rgb ? __ldg(sc.rgb + 3 * g) : 0.f, sc.rgb ? __ldg(sc.rgb + 3 * g + 1) : 0.f,
                            sc.rgb ? __ldg(sc.rgb + 3 * g + 2) : 0.f, p.depth);
  P.rec_unc[r] = sc.geo_unc ? __ldg(sc.geo_unc + g) : 0.f;
  if (sc.sem_ids)
    for (int l = 0; l < sc.k; ++l)
      P.rec_sem[(size_t)r * sc.k + l] = make_int2(__ldg(sc.sem_ids + (size_t)g * sc.k + l),
                                                  __float_as_int(__ldg(sc.sem_w + (size_t)g * sc.k + l)));
  P.dkeys[0][r] = ((unsigned long long)v << 31) | (unsigned long long)__float_as_uint(p.depth);
  P.dvals[0][r] = r;
}

// Pass 2: recompute (bit-identical) and write compacted records in
// (view, Gaussian index) order, plus the (view, depth) sort keys.
__global__ void __launch_bounds__(kProjThreads) k_project_emit(gs_scene sc, const DevCam *cams, int nb, int n_views,
                                                               const uint32_t *blockoff, uint32_t rcap,
                                                               WsPtrs P) {
  __shared__ uint32_t tmp[33];
  const int b = blockIdx.x;
  const int v0 = blockIdx.y * kViewsPerCta, v1 = min(n_views, v0 + kViewsPerCta);
  const int g0 = b * kProjBlock + threadIdx.x * kProjItems;
  GIn in[kProjItems];
#pragma unroll
  for (int i = 0; i < kProjItems; ++i)
    if (g0 + i < sc.n) in[i] = load_gaussian(sc, g0 + i);
  for (int v = v0; v < v1; ++v) {
    const DevCam c = cams[v];
    Proj p[kProjItems];
    bool vis[kProjItems];
    uint32_t cnt = 0;
#pragma unroll
    for (int i = 0; i < kProjItems; ++i) {
      vis[i] = false;
      if (g0 + i < sc.n)
        vis[i] = project_gaussian(in[i].mx, in[i].my, in[i].mz, in[i].sx, in[i].sy, in[i].sz, in[i].q, c, p[i]);
      cnt += vis[i] ? 1u : 0u;
    }
    uint32_t total;
    uint32_t rank = blockoff[v * nb + b] + block_exclusive_scan(cnt, tmp, &total);
#pragma unroll
    for (int i = 0; i < kProjItems; ++i) {
      if (!vis[i]) continue;
      const uint32_t r = rank++;
      if (r < rcap) write_record(sc, P, r, g0 + i, v, p[i]);
    }
  }
}

// Single-view projection in one pass (the mapping view): each CTA takes a
// block ticket, projects its Gaussians, publishes its visible count and
// looks back over the blocks ticketed before it (decoupled look-back) for
// its offset, then writes its records -- the same records, in the same
// (Gaussian index) order, as the count / scan / emit passes, without the
// count pass and the scan.  A look-back word holds a flag in its top two
// bits (aggregate or inclusive prefix published) and a count below, so the
// path is taken for n < 2^30.  A CTA only waits on blocks whose tickets were
// taken earlier (their CTAs are running); every wait is bounded and, if the
// bound is hit, raises the timeout status instead of hanging (later kernels
// then skip their work).  The block ticketed last writes the record count.
constexpr uint32_t kPjFlagA = 1u << 30;  // block count published
constexpr uint32_t kPjFlagP = 2u << 30;  // inclusive prefix published
constexpr uint32_t kPjVal = kPjFlagA - 1u;

__global__ void __launch_bounds__(kProjThreads) k_project_single(gs_scene sc, const DevCam *cams, int nb,
                                                                 uint32_t rcap, uint32_t *lookback,
                                                                 uint32_t *ticket, uint32_t spin_limit,
                                                                 WsPtrs P) {
  __shared__ uint32_t tmp[33];
  __shared__ uint32_t s_b, s_off;
  if (threadIdx.x == 0) s_b = atomicAdd(ticket, 1u);
  __syncthreads();
  const int b = (int)s_b;
  const int g0 = b * kProjBlock + threadIdx.x * kProjItems;
  GIn in[kProjItems];
#pragma unroll
  for (int i = 0; i < kProjItems; ++i)
    if (g0 + i < sc.n) in[i] = load_gaussian(sc, g0 + i);
  const DevCam c = cams[0];
  Proj p[kProjItems];
  bool vis[kProjItems];
  uint32_t cnt = 0;
#pragma unroll
  for (int i = 0; i < kProjItems; ++i) {
    vis[i] = false;
    if (g0 + i < sc.n)
      vis[i] = project_gaussian(in[i].mx, in[i].my, in[i].mz, in[i].sx, in[i].sy, in[i].sz, in[i].q, c, p[i]);
    cnt += vis[i] ? 1u : 0u;
  }
  uint32_t total;
  const uint32_t ex = block_exclusive_scan(cnt, tmp, &total);
  if (threadIdx.x < 32) {
    // warp 0 looks back 32 blocks at a time (lane i reads block j - i):
    // the newest blocks' counts are added up to the first inclusive prefix;
    // an unpublished word stops the step there and is read again (a bounded
    // wait).  Blocks before block 0 read as an empty prefix.
    const uint32_t lane = threadIdx.x;
    uint32_t excl = 0u;
    if (b == 0) {
      if (lane == 0) atomicExch(lookback, kPjFlagP | total);
    } else {
      if (lane == 0) atomicExch(lookback + b, kPjFlagA | total);
      int j = b - 1;
      uint32_t spins = 0;
      while (true) {
        const int idx = j - (int)lane;
        const uint32_t w = idx >= 0 ? *reinterpret_cast<volatile uint32_t *>(lookback + idx) : (uint32_t)kPjFlagP;
        const uint32_t flag = w & ~kPjVal;
        const uint32_t zero = __ballot_sync(0xffffffffu, flag == 0u);
        const uint32_t pre = __ballot_sync(0xffffffffu, flag == kPjFlagP);
        const int first_zero = zero ? __ffs(zero) - 1 : 32, first_p = pre ? __ffs(pre) - 1 : 32;
        const int upto = first_p < first_zero ? first_p + 1 : first_zero;  // lanes whose counts are taken
        uint32_t v = (int)lane < upto ? (w & kPjVal) : 0u;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        excl += v;
        if (first_p < first_zero) break;
        j -= upto;
        if (first_zero < 32) {
          if (++spins > spin_limit) {
            if (lane == 0) set_status(P.counters, kStatusTimeout);
            break;
          }
          __nanosleep(32);
        }
      }
      if (lane == 0) atomicExch(lookback + b, kPjFlagP | ((excl + total) & kPjVal));
    }
    if (lane == 0) {
      s_off = excl;
      if (b == nb - 1) {
        P.counters->n_records = excl + total;
        if (excl + total > rcap) set_status(P.counters, kStatusCapacity);
      }
    }
  }
  __syncthreads();
  uint32_t rank = s_off + ex;
#pragma unroll
  for (int i = 0; i < kProjItems; ++i) {
    if (!vis[i]) continue;
    const uint32_t r = rank++;
    if (r < rcap) write_record(sc, P, r, g0 + i, 0, p[i]);
  }
}

// Exclusive scan of n u32 in place by one CTA of 1024 threads (each thread
// owns a contiguous segment).  Writes the sum to *total_out and raises the
// capacity status when it exceeds `capacity`.
__global__ void __launch_bounds__(1024) k_scan_single(uint32_t *data, uint32_t n, uint32_t *total_out,
                                                      uint32_t capacity, Counters *counters) {
  __shared__ uint32_t tmp[33];
  const uint32_t per = (n + blockDim.x - 1) / blockDim.x;
  const uint32_t lo = min(n, threadIdx.x * per), hi = min(n, lo + per);
  uint32_t s = 0;
  for (uint32_t i = lo; i < hi; ++i) s += data[i];
  uint32_t total;
  uint32_t run = block_exclusive_scan(s, tmp, &total);
  for (uint32_t i = lo; i < hi; ++i) {
    uint32_t x = data[i];
    data[i] = run;
    run += x;
  }
  if (threadIdx.x == 0) {
    if (total_out) *total_out = total;
    if (total > capacity) set_status(counters, kStatusCapacity);
  }
}

cudaError_t launch_setup_views(const CamTable &tab, int n_views, const WsPtrs &P, uint32_t total_tiles,
                               bool reset_status, cudaStream_t s) {
  k_setup_views<<<1, kMaxViews, 0, s>>>(tab, n_views, P.cams, P.tile_off, total_tiles, P.counters,
                                        reset_status ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_scan_single(uint32_t *data, uint32_t n, uint32_t *total_out, uint32_t capacity,
                               Counters *counters, cudaStream_t s) {
  k_scan_single<<<1, 1024, 0, s>>>(data, n, total_out, capacity, counters);
  return cudaGetLastError();
}

cudaError_t launch_project(const Layout &L, const WsPtrs &P, const gs_scene &sc, cudaStream_t s) {
  const int nb = (int)L.proj_blocks;
  const int grid = nb * L.n_views;
  if (grid == 0) return cudaSuccess;
  if (L.n_views == 1 && (int64_t)sc.n < (int64_t)kPjVal) {
    // blockcnt holds nb + 1 words: the look-back words, then the ticket
    cudaError_t e = cudaMemsetAsync(P.blockcnt, 0, sizeof(uint32_t) * ((size_t)nb + 1), s);
    if (e != cudaSuccess) return e;
    k_project_single<<<nb, kProjThreads, 0, s>>>(sc, P.cams, nb, (uint32_t)L.rcap, P.blockcnt, P.blockcnt + nb,
                                                 L.spin_limit, P);
    return cudaGetLastError();
  }
  const dim3 g2(nb, (L.n_views + kViewsPerCta - 1) / kViewsPerCta);
  k_project_count<<<g2, kProjThreads, 0, s>>>(sc, P.cams, nb, L.n_views, P.blockcnt);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = launch_scan_single(P.blockcnt, (uint32_t)grid, &P.counters->n_records, (uint32_t)L.rcap, P.counters, s);
  if (e != cudaSuccess) return e;
  k_project_emit<<<g2, kProjThreads, 0, s>>>(sc, P.cams, nb, L.n_views, P.blockcnt, (uint32_t)L.rcap, P);
  return cudaGetLastError();
}

}  // namespace gs
