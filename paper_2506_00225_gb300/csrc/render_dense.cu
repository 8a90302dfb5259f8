// render_dense.cu -- the dense-semantic comparator of the supplement's
// "Sparse Rendering" and "Runtime Analysis": every Gaussian carries a full
// distribution over all M classes and Eq. 3 blends all of them, the
// representation the paper's sparse top-k form replaces.
//
// Same passes as the sparse forward: the blend pass (colour, depth,
// silhouette, contributor bits) is shared; the semantic pass below walks the
// contributor bits like the sparse one, but for every contributor adds
// w * p_c for all classes c.  A thread keeps 32 classes of its pixel in
// registers; the tile walks its contributors once per 32-class chunk, with
// the staged Gaussians' chunk of probabilities (read by Gaussian id straight
// from the caller's [n][m] array) double-buffered in shared memory and read
// as float4 broadcasts.  A dense class that is 0 adds exactly 0 (fmaf with a
// zero product), so a dense array holding only the top-k entries renders the
// same bits as the sparse path.
#include "gs_internal.cuh"
#include "render_common.cuh"

namespace gs {

constexpr int kDenseCh = 32;  // classes per chunk (per-thread registers)

// Shared memory of one dense batch buffer: mean, conic, kDenseCh
// probabilities of each staged Gaussian.
__host__ __device__ inline size_t dense_batch_bytes() { return (size_t)kBatch * (8 + 16 + 4 * kDenseCh); }

template <int TW, int TH>
__global__ void __launch_bounds__(TW *TH) k_semantic_dense(FwdArgs a, const float *__restrict__ dense) {
  using FP = Footprint<TW, TH, 1>;
  constexpr int THREADS = FP::kThreads;
  constexpr int NPIX = FP::kPix;
  constexpr int CPR = kDenseCh / 4;             // float4 per staged row
  constexpr int TPR = THREADS / kBatch;         // copying threads per staged row
  static_assert(THREADS % kBatch == 0 && kDenseCh % TPR == 0, "copy split");
  extern __shared__ float4 smem4[];
  const int m = a.m;
  char *sbase = reinterpret_cast<char *>(smem4);
  const size_t bbytes = dense_batch_bytes();
  __shared__ uint32_t s_maxlast;
  if (a.counters->status & kStatusTimeout) return;  // the binning is incomplete

  const int tile = blockIdx.x;
  const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
  const int ox = tx * TW, oy = ty * TH;
  const uint2 rg = a.ranges[tile];
  const int lx = FP::lx(), ly = FP::ly(0);
  const int px = ox + lx, py = oy + ly;
  const int lp = ly * TW + lx;
  const bool inside = px < a.width && py < a.height;
  const float fpx = (float)px + 0.5f, fpy = (float)py + 0.5f;
  const uint32_t unit0 = a.mask_off[tile];

  const uint32_t last = inside ? a.nlast[(size_t)py * a.width + px] : 0u;
  if (threadIdx.x == 0) s_maxlast = 0;
  __syncthreads();
  if (last) atomicMax(&s_maxlast, last);
  __syncthreads();
  const int nbatch = (int)((s_maxlast + kBatch - 1) / kBatch);

  auto buf_uv = [&](int q) { return reinterpret_cast<float2 *>(sbase + q * bbytes); };
  auto buf_co = [&](int q) { return reinterpret_cast<float4 *>(sbase + q * bbytes + kBatch * 8); };
  auto buf_pr = [&](int q) { return reinterpret_cast<float *>(sbase + q * bbytes + kBatch * 24); };
  auto batch_n = [&](int bi) { return (int)min((uint32_t)kBatch, rg.y - (rg.x + (uint32_t)bi * kBatch)); };

  for (int c0 = 0; c0 < m; c0 += kDenseCh) {
    const int mc = min(kDenseCh, m - c0);
    // batch bi into buffer bi & 1: thread t stages the mean and conic of
    // slot t (t < n) and part t % TPR of row t / TPR's probability chunk;
    // classes past the chunk's end read as 0
    auto issue = [&](int bi) {
      const int q = bi & 1, t = threadIdx.x, n = batch_n(bi);
      const uint32_t base = rg.x + (uint32_t)bi * kBatch;
      if (t < n) {
        const uint32_t r = a.pvals[base + t];
        cp_async8(buf_uv(q) + t, a.rec.uv + r);
        cp_async16(buf_co(q) + t, a.rec.co + r);
      }
      const int row = t / TPR, part = t % TPR;
      if (row < n) {
        const int g = __ldg(a.rec.gid + a.pvals[base + row]);
        const float *src = dense + (size_t)g * m + c0;
        float *dst = buf_pr(q) + row * kDenseCh;
#pragma unroll
        for (int e = part * (kDenseCh / TPR); e < (part + 1) * (kDenseCh / TPR); ++e) {
          if (e < mc) cp_async4(dst + e, src + e);
          else dst[e] = 0.f;
        }
      }
    };
    float acc[kDenseCh];
#pragma unroll
    for (int c = 0; c < kDenseCh; ++c) acc[c] = 0.f;
    float T = 1.f;
    if (nbatch > 0) issue(0);
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
    for (int bi = 0; bi < nbatch; ++bi) {
      if (bi + 1 < nbatch) issue(bi + 1);
      cp_async_commit();
      const uint32_t b0 = (uint32_t)bi * kBatch;
      uint32_t mine[2] = {0u, 0u};
      if (b0 < last) {
        const uint32_t *mw = a.masks + (size_t)(unit0 + bi) * 2 * NPIX;
        mine[0] = mw[lp];
        mine[1] = mw[NPIX + lp];
      }
      const float2 *suv = buf_uv(bi & 1);
      const float4 *sco = buf_co(bi & 1);
      const float4 *spr = reinterpret_cast<const float4 *>(buf_pr(bi & 1));
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        uint32_t un = __reduce_or_sync(0xffffffffu, mine[h]);
        while (un) {
          const int jb = __ffs(un) - 1;
          un &= un - 1;
          const int j = h * 32 + jb;
          float alpha = 0.f, G, araw, dx, dy;
          gauss_alpha(suv[j], sco[j], fpx, fpy, alpha, G, araw, dx, dy);
          const bool on = (mine[h] >> jb) & 1u;
          const float w = on ? __fmul_rn(alpha, T) : 0.f;
          if (on) T = __fmul_rn(T, __fsub_rn(1.f, alpha));
#pragma unroll
          for (int v = 0; v < CPR; ++v) {
            const float4 p = spr[j * CPR + v];
            acc[4 * v] = fmaf(w, p.x, acc[4 * v]);
            acc[4 * v + 1] = fmaf(w, p.y, acc[4 * v + 1]);
            acc[4 * v + 2] = fmaf(w, p.z, acc[4 * v + 2]);
            acc[4 * v + 3] = fmaf(w, p.w, acc[4 * v + 3]);
          }
        }
      }
      cp_async_wait_all();
      __syncthreads();
    }
    if (inside) {
      float *dst = a.sem + ((size_t)py * a.width + px) * m + c0;
#pragma unroll
      for (int c = 0; c < kDenseCh; ++c)
        if (c < mc) dst[c] = acc[c];
    }
    __syncthreads();  // the next chunk reuses the batch buffers
  }
}

template <int TW, int TH>
static cudaError_t launch_dense_shape(const FwdArgs &a, const float *dense, int grid, cudaStream_t s) {
  const size_t smem = 2 * dense_batch_bytes();
  k_semantic_dense<TW, TH><<<grid, TW * TH, smem, s>>>(a, dense);
  return cudaGetLastError();
}

bool dense_supported(const Layout &L) { return L.mask_units > 0 && L.npix > 0; }

cudaError_t launch_render_fwd_dense(const Layout &L, const WsPtrs &P, int pbuf, const gs_scene &sc,
                                    const float *dense, float *rgb, float *depth, float *sil, float *sem,
                                    cudaStream_t s) {
  FwdArgs a = fwd_args(L, P, pbuf, sc);
  const int tiles_y = (L.cam0_h + L.tile_h - 1) / L.tile_h;
  a.rgb_out = rgb; a.depth_out = depth; a.sil_out = sil; a.sem = sem;
  const int grid = a.tiles_x * tiles_y;
  if (grid == 0) return cudaSuccess;
  cudaError_t e = launch_tile_batch_offsets(P.ranges, (uint32_t)grid, P.mask_off, P.counters, s);
  if (e != cudaSuccess) return e;
  e = launch_blend_plain(L, a, grid, s);
  if (e != cudaSuccess || !sem) return e;
  if (L.tile_w == 16 && L.tile_h == 16) return launch_dense_shape<16, 16>(a, dense, grid, s);
  if (L.tile_w == 16 && L.tile_h == 8) return launch_dense_shape<16, 8>(a, dense, grid, s);
  if (L.tile_w == 8 && L.tile_h == 8) return launch_dense_shape<8, 8>(a, dense, grid, s);
  if (L.tile_w == 32 && L.tile_h == 8) return launch_dense_shape<32, 8>(a, dense, grid, s);
  return cudaErrorInvalidConfiguration;
}

}  // namespace gs
