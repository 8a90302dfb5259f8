// explore.cu -- candidate management around the candidate renders (Sec. 3.2):
// the scoring tail of Eq. 6-8 on the device, and the host-side generation
// of candidate poses (positions on a v1-spaced lattice over newly freed
// space, v2 viewing directions from a Fibonacci lattice on the sphere).
//
// Scoring, per call over the V candidates given (one CTA, fixed reduction
// order: deterministic):
//   I_geo^v = softmax_v(log N_S^v) = N_S^v / sum_u N_S^u        (Eq. 6)
//   I_sem^v = softmax_v(sum_p H^v(p))                            (Eq. 7)
//   I^v     = (1 - softmax_v(l^v)) I_geo^v I_sem^v,  l^v = |T^v - T^t|   (Eq. 8)
// with the per-view sums of gs_render_candidates, softmaxes taken with the
// maximum subtracted, in double.  A view whose N_S is below prune_frac of its
// pixels is dropped from the pool (keep = 0); the best view is the largest
// I^v among the kept ones.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <vector>

#include "gs_internal.cuh"

namespace gs {

constexpr int kScoreThreads = 256;

// Block-wide reduction of one double per thread (sum or max), result on
// every thread.  `sh` holds kScoreThreads / 32 doubles.
template <bool MAX>
__device__ double block_reduce(double v, double *sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double u = __shfl_xor_sync(0xffffffffu, v, o);
    v = MAX ? fmax(v, u) : v + u;
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = sh[0];
  for (int w = 1; w < kScoreThreads / 32; ++w) r = MAX ? fmax(r, sh[w]) : r + sh[w];
  return r;
}

__global__ void __launch_bounds__(kScoreThreads) k_score_candidates(int V, const double *__restrict__ sums,
                                                                     const int32_t *__restrict__ npix,
                                                                     const float *__restrict__ pos,
                                                                     const float *__restrict__ cur,
                                                                     double prune_frac, double *scores,
                                                                     int32_t *keep, int32_t *best) {
  __shared__ double sh[kScoreThreads / 32];
  __shared__ double sbv[kScoreThreads];
  __shared__ int sbi[kScoreThreads];
  const int t = threadIdx.x;
  const double cx = cur[0], cy = cur[1], cz = cur[2];
  auto dist = [&](int v) {
    const double dx = (double)pos[3 * v] - cx, dy = (double)pos[3 * v + 1] - cy, dz = (double)pos[3 * v + 2] - cz;
    return sqrt(dx * dx + dy * dy + dz * dz);
  };
  // pass 1: sum of N_S, maxima of sum H and of the distance
  double ns = 0.0, hmax = -INFINITY, lmax = -INFINITY;
  for (int v = t; v < V; v += kScoreThreads) {
    ns += sums[3 * v + 2];
    hmax = fmax(hmax, sums[3 * v + 1]);
    lmax = fmax(lmax, dist(v));
  }
  ns = block_reduce<false>(ns, sh);
  hmax = block_reduce<true>(hmax, sh);
  lmax = block_reduce<true>(lmax, sh);
  // pass 2: softmax denominators
  double eh = 0.0, el = 0.0;
  for (int v = t; v < V; v += kScoreThreads) {
    eh += exp(sums[3 * v + 1] - hmax);
    el += exp(dist(v) - lmax);
  }
  eh = block_reduce<false>(eh, sh);
  el = block_reduce<false>(el, sh);
  // pass 3: scores, pool flags, and the best kept view of this thread
  double bv = -1.0;
  int bi = -1;
  for (int v = t; v < V; v += kScoreThreads) {
    const double nsv = sums[3 * v + 2];
    const double igeo = ns > 0.0 ? nsv / ns : 0.0;
    const double isem = exp(sums[3 * v + 1] - hmax) / eh;
    const double mov = 1.0 - exp(dist(v) - lmax) / el;
    const double iv = mov * igeo * isem;
    scores[4 * v] = iv;
    scores[4 * v + 1] = igeo;
    scores[4 * v + 2] = isem;
    scores[4 * v + 3] = mov;
    const int k = nsv >= prune_frac * (double)npix[v] ? 1 : 0;
    keep[v] = k;
    if (k && iv > bv) { bv = iv; bi = v; }  // ascending v: ties keep the lower index
  }
  sbv[t] = bv;
  sbi[t] = bi;
  __syncthreads();
  for (int s = kScoreThreads / 2; s > 0; s >>= 1) {
    if (t < s) {
      const double ov = sbv[t + s];
      const int oi = sbi[t + s];
      if (oi >= 0 && (sbi[t] < 0 || ov > sbv[t] || (ov == sbv[t] && oi < sbi[t]))) {
        sbv[t] = ov;
        sbi[t] = oi;
      }
    }
    __syncthreads();
  }
  if (t == 0) *best = sbi[0];
}

cudaError_t launch_score_candidates(int V, const double *sums, const int32_t *npix, const float *pos,
                                    const float *cur, double prune_frac, double *scores, int32_t *keep,
                                    int32_t *best, cudaStream_t s) {
  k_score_candidates<<<1, kScoreThreads, 0, s>>>(V, sums, npix, pos, cur, prune_frac, scores, keep, best);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Host: candidate generation
// ---------------------------------------------------------------------------

// Direction i of an n-point Fibonacci lattice on the unit sphere: heights
// z_i = 1 - (2 i + 1) / n equally spaced, azimuth advancing by the golden
// angle pi (3 - sqrt 5) per point.
void fibonacci_direction(int i, int n, double d[3]) {
  const double golden = 3.14159265358979323846 * (3.0 - std::sqrt(5.0));
  const double z = 1.0 - (2.0 * i + 1.0) / (double)n;
  const double r = std::sqrt(std::max(0.0, 1.0 - z * z));
  const double phi = golden * (double)i;
  d[0] = r * std::cos(phi);
  d[1] = r * std::sin(phi);
  d[2] = z;
}

// World-to-camera [R|t] of a camera at p looking along the unit vector d
// (OpenCV axes: rows right, down, forward), right = d x up with up = +z
// (+y when d is within 1e-6 of vertical).
void look_along(const double p[3], const double d[3], float w2c[12]) {
  double up[3] = {0.0, 0.0, 1.0};
  if (std::fabs(d[2]) > 1.0 - 1e-6) { up[1] = 1.0; up[2] = 0.0; }
  double rt[3] = {d[1] * up[2] - d[2] * up[1], d[2] * up[0] - d[0] * up[2], d[0] * up[1] - d[1] * up[0]};
  const double rn = std::sqrt(rt[0] * rt[0] + rt[1] * rt[1] + rt[2] * rt[2]);
  for (double &x : rt) x /= rn;
  const double dn[3] = {d[1] * rt[2] - d[2] * rt[1], d[2] * rt[0] - d[0] * rt[2], d[0] * rt[1] - d[1] * rt[0]};
  const double *rows[3] = {rt, dn, d};
  for (int r = 0; r < 3; ++r) {
    double tr = 0.0;
    for (int c = 0; c < 3; ++c) {
      w2c[4 * r + c] = (float)rows[r][c];
      tr -= rows[r][c] * p[c];
    }
    w2c[4 * r + 3] = (float)tr;
  }
}

}  // namespace gs

using namespace gs;

extern "C" {

gs_status gs_score_candidates(int n_views, const double *sums, const int32_t *npix, const float *positions,
                              const float *current, double prune_frac, double *scores, int32_t *keep,
                              int32_t *best, gs_stream_t stream) {
  if (n_views < 1 || !sums || !npix || !positions || !current || !scores || !keep || !best) return GS_ERR_ARG;
  if (!(prune_frac >= 0.0 && prune_frac <= 1.0)) return GS_ERR_ARG;
  if (launch_score_candidates(n_views, sums, npix, positions, current, prune_frac, scores, keep, best,
                              (cudaStream_t)stream) != cudaSuccess)
    return GS_ERR_CUDA;
  return GS_OK;
}

gs_status gs_candidate_poses(int n_positions, const float *positions, int n_dirs, int width, int height, float fx,
                             float fy, float near_plane, gs_camera *out) {
  if (n_positions < 0 || n_dirs < 1 || (n_positions > 0 && (!positions || !out))) return GS_ERR_ARG;
  if (width < 1 || height < 1 || !(fx > 0.f) || !(fy > 0.f) || !(near_plane > 0.f)) return GS_ERR_ARG;
  for (int p = 0; p < n_positions; ++p) {
    const double pos[3] = {positions[3 * p], positions[3 * p + 1], positions[3 * p + 2]};
    for (int i = 0; i < n_dirs; ++i) {
      gs_camera &c = out[(size_t)p * n_dirs + i];
      memset(&c, 0, sizeof(c));
      c.width = width;
      c.height = height;
      c.fx = fx;
      c.fy = fy;
      c.cx = (float)(width / 2.0);
      c.cy = (float)(height / 2.0);
      c.near_plane = near_plane;
      double d[3];
      fibonacci_direction(i, n_dirs, d);
      look_along(pos, d, c.w2c);
    }
  }
  return GS_OK;
}

int64_t gs_candidate_positions(int64_t n_voxels, const float *centres, float step, int n_heights,
                               const float *heights, float band, float *out, int64_t capacity) {
  if (n_voxels < 0 || (n_voxels > 0 && !centres) || !(step > 0.f) || n_heights < 1 || !heights || !(band >= 0.f))
    return -1;
  if (capacity < 0 || (capacity > 0 && !out)) return -1;
  // lattice points (i step, j step, height h) with a voxel centre in the
  // square cell around (i, j) whose height lies within band of h
  std::vector<std::array<int64_t, 3>> cells;
  cells.reserve((size_t)n_voxels);
  for (int64_t q = 0; q < n_voxels; ++q) {
    const double x = centres[3 * q], y = centres[3 * q + 1], z = centres[3 * q + 2];
    for (int h = 0; h < n_heights; ++h) {
      if (std::fabs(z - (double)heights[h]) > (double)band) continue;
      cells.push_back({(int64_t)std::floor(x / step + 0.5), (int64_t)std::floor(y / step + 0.5), (int64_t)h});
    }
  }
  std::sort(cells.begin(), cells.end());
  cells.erase(std::unique(cells.begin(), cells.end()), cells.end());
  const int64_t n = (int64_t)cells.size();
  for (int64_t i = 0; i < std::min(n, capacity); ++i) {
    out[3 * i] = (float)((double)cells[i][0] * step);
    out[3 * i + 1] = (float)((double)cells[i][1] * step);
    out[3 * i + 2] = heights[cells[i][2]];
  }
  return n;
}

}  // extern "C"
