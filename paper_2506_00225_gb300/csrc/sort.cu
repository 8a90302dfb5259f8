// sort.cu -- front-to-back binning (Sec. 3.1 "sorting them front-to-back";
// supplement "Sparse Rendering": each tile renders its frustum Gaussians in
// batches).
//
// Order produced: (view, tile, depth bits, Gaussian index), obtained in two
// stable sorts:
//   1. visible records (compacted in (view, gid) order) sorted by
//      (view, depth bits) -- LSD radix over 31 + view bits;
//   2. one pair per tile of each record's tile rectangle, emitted in that
//      depth order, stably sorted by global tile id -- LSD radix over the tile
//      bits only.
// Stability carries the depth order (and the gid tie-break) into each tile.
//
// The radix sort is a reduce-then-scan LSD sort with 8-bit digits and a
// fixed grid: per pass, (1) per-CTA digit histograms, (2) one-CTA exclusive
// scan of the digit-major histogram matrix, (3) per-CTA stable scatter using
// warp match-based ranking.  There are no inter-CTA waits; element counts
// are read from device memory, so the whole sort is graph-capturable.
#include "gs_internal.cuh"

namespace gs {

template <typename K>
__device__ __forceinline__ uint32_t digit_of(K key, int shift) {
  return (uint32_t)(key >> shift) & (kRadix - 1);
}

__device__ __forceinline__ void chunk_range(uint32_t count, uint32_t &begin, uint32_t &end) {
  const uint32_t tiles = (count + kSortTile - 1) / kSortTile;
  const uint32_t per = (tiles + gridDim.x - 1) / gridDim.x;
  begin = min(count, blockIdx.x * per * kSortTile);
  end = min(count, begin + per * kSortTile);
}

template <typename K>
__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const K *__restrict__ keys, const uint32_t *count_p,
                                                             uint32_t cap, int shift, uint32_t *hist) {
  __shared__ uint32_t h[kSortThreads / 32][kRadix];
  const uint32_t warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < (kSortThreads / 32) * kRadix; i += kSortThreads) (&h[0][0])[i] = 0;
  __syncthreads();
  const uint32_t count = min(*count_p, cap);
  uint32_t begin, end;
  chunk_range(count, begin, end);
  for (uint32_t i = begin + threadIdx.x; i < end; i += kSortThreads) atomicAdd(&h[warp][digit_of(keys[i], shift)], 1u);
  __syncthreads();
  for (int d = threadIdx.x; d < kRadix; d += kSortThreads) {
    uint32_t s = 0;
#pragma unroll
    for (int w = 0; w < kSortThreads / 32; ++w) s += h[w][d];
    hist[d * gridDim.x + blockIdx.x] = s;
  }
}

template <typename K>
__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(const K *__restrict__ keys_in,
                                                                const uint32_t *__restrict__ vals_in,
                                                                K *__restrict__ keys_out, uint32_t *__restrict__ vals_out,
                                                                const uint32_t *count_p, uint32_t cap, int shift,
                                                                const uint32_t *__restrict__ hist) {
  constexpr int kWarps = kSortThreads / 32;
  __shared__ uint32_t digit_off[kRadix];
  __shared__ uint32_t wcnt[kWarps][kRadix];
  __shared__ uint32_t tile_tot[kRadix];
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
  const uint32_t count = min(*count_p, cap);
  uint32_t begin, end;
  chunk_range(count, begin, end);
  for (int d = threadIdx.x; d < kRadix; d += kSortThreads) digit_off[d] = hist[d * gridDim.x + blockIdx.x];
  const uint32_t lt = lanemask_lt();
  for (uint32_t base = begin; base < end; base += kSortTile) {
    for (int i = threadIdx.x; i < kWarps * kRadix; i += kSortThreads) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    K key[kSortItems];
    uint32_t val[kSortItems], dig[kSortItems], loc[kSortItems];
#pragma unroll
    for (int i = 0; i < kSortItems; ++i) {
      const uint32_t idx = base + warp * (32 * kSortItems) + i * 32 + lane;
      const bool ok = idx < end;
      key[i] = ok ? keys_in[idx] : (K)0;
      val[i] = ok ? vals_in[idx] : 0u;
      dig[i] = ok ? digit_of(key[i], shift) : (uint32_t)kRadix;
    }
#pragma unroll
    for (int i = 0; i < kSortItems; ++i) {
      const uint32_t peers = __match_any_sync(0xffffffffu, dig[i]);
      const uint32_t rank = __popc(peers & lt);
      const bool leader = (peers & lt) == 0u;
      uint32_t b = 0;
      if (dig[i] < (uint32_t)kRadix) b = wcnt[warp][dig[i]];
      loc[i] = b + rank;
      __syncwarp();
      if (leader && dig[i] < (uint32_t)kRadix) wcnt[warp][dig[i]] = b + __popc(peers);
      __syncwarp();
    }
    __syncthreads();
    // exclusive scan over warps, per digit
    for (int d = threadIdx.x; d < kRadix; d += kSortThreads) {
      uint32_t run = 0;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) {
        const uint32_t c = wcnt[w][d];
        wcnt[w][d] = run;
        run += c;
      }
      tile_tot[d] = run;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kSortItems; ++i) {
      if (dig[i] < (uint32_t)kRadix) {
        const uint32_t pos = digit_off[dig[i]] + wcnt[warp][dig[i]] + loc[i];
        keys_out[pos] = key[i];
        vals_out[pos] = val[i];
      }
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += kSortThreads) digit_off[d] += tile_tot[d];
    __syncthreads();
  }
}

template <typename K>
static cudaError_t radix_sort(K *keys[2], uint32_t *vals[2], const uint32_t *count_p, uint32_t cap, int bits,
                              uint32_t *hist, Counters *counters, cudaStream_t s) {
  const int passes = radix_passes(bits);
  for (int p = 0; p < passes; ++p) {
    const int src = p & 1, dst = src ^ 1;
    const int shift = p * kRadixBits;
    k_radix_hist<K><<<kSortCtas, kSortThreads, 0, s>>>(keys[src], count_p, cap, shift, hist);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = launch_scan_single(hist, (uint32_t)(kRadix * kSortCtas), nullptr, 0xffffffffu, counters, s);
    if (e != cudaSuccess) return e;
    k_radix_scatter<K><<<kSortCtas, kSortThreads, 0, s>>>(keys[src], vals[src], keys[dst], vals[dst], count_p, cap,
                                                         shift, hist);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_radix_sort_u64(const Layout &L, const WsPtrs &P, int bits, int *final_buf, cudaStream_t s) {
  unsigned long long *k[2] = {P.dkeys[0], P.dkeys[1]};
  uint32_t *v[2] = {P.dvals[0], P.dvals[1]};
  *final_buf = radix_passes(bits) & 1;
  return radix_sort<unsigned long long>(k, v, &P.counters->n_records, (uint32_t)L.rcap, bits, P.hist, P.counters, s);
}

cudaError_t launch_radix_sort_u32(const Layout &L, const WsPtrs &P, int bits, int *final_buf, cudaStream_t s) {
  uint32_t *k[2] = {P.pkeys[0], P.pkeys[1]};
  uint32_t *v[2] = {P.pvals[0], P.pvals[1]};
  *final_buf = radix_passes(bits) & 1;
  return radix_sort<uint32_t>(k, v, &P.counters->n_pairs, (uint32_t)L.pcap, bits, P.hist, P.counters, s);
}

// ---------------------------------------------------------------------------
// Pair emission in depth order.
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t record_ntiles(short4 r, int tw, int th) {
  return (uint32_t)((r.y / tw - r.x / tw + 1) * (r.w / th - r.z / th + 1));
}

__device__ __forceinline__ void emit_chunk(uint32_t count, uint32_t &begin, uint32_t &end) {
  const uint32_t per = (count + gridDim.x - 1) / gridDim.x;
  begin = min(count, blockIdx.x * per);
  end = min(count, begin + per);
}

__global__ void __launch_bounds__(kEmitThreads) k_emit_count(const uint32_t *__restrict__ sorted_rec,
                                                             const short4 *__restrict__ rect, const Counters *cnt,
                                                             uint32_t rcap, int tw, int th, uint32_t *epart) {
  __shared__ uint32_t tmp[33];
  const uint32_t count = min(cnt->n_records, rcap);
  uint32_t begin, end;
  emit_chunk(count, begin, end);
  uint32_t s = 0;
  for (uint32_t q = begin + threadIdx.x; q < end; q += kEmitThreads) s += record_ntiles(rect[sorted_rec[q]], tw, th);
  uint32_t total;
  block_exclusive_scan(s, tmp, &total);
  if (threadIdx.x == 0) epart[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kEmitThreads) k_emit_write(const uint32_t *__restrict__ sorted_rec,
                                                             const short4 *__restrict__ rect,
                                                             const int32_t *__restrict__ rview,
                                                             const DevCam *__restrict__ cams, const Counters *cnt,
                                                             uint32_t rcap, uint32_t pcap, int tw, int th,
                                                             const uint32_t *__restrict__ epart,
                                                             uint32_t *__restrict__ pkeys,
                                                             uint32_t *__restrict__ pvals) {
  __shared__ uint32_t tmp[33];
  const uint32_t count = min(cnt->n_records, rcap);
  uint32_t begin, end;
  emit_chunk(count, begin, end);
  uint32_t run = epart[blockIdx.x];
  for (uint32_t q0 = begin; q0 < end; q0 += kEmitThreads) {
    const uint32_t q = q0 + threadIdx.x;
    uint32_t r = 0, nt = 0;
    short4 rc = make_short4(0, 0, 0, 0);
    if (q < end) {
      r = sorted_rec[q];
      rc = rect[r];
      nt = record_ntiles(rc, tw, th);
    }
    uint32_t total;
    uint32_t pos = run + block_exclusive_scan(nt, tmp, &total);
    run += total;
    if (nt) {
      const DevCam &c = cams[rview[r]];
      const int tx0 = rc.x / tw, tx1 = rc.y / tw, ty0 = rc.z / th, ty1 = rc.w / th;
      for (int ty = ty0; ty <= ty1; ++ty)
        for (int tx = tx0; tx <= tx1; ++tx) {
          if (pos < pcap) {
            pkeys[pos] = c.tile_off + (uint32_t)(ty * c.tiles_x + tx);
            pvals[pos] = r;
          }
          ++pos;
        }
    }
  }
}

cudaError_t launch_emit_pairs(const Layout &L, const WsPtrs &P, int dbuf, cudaStream_t s) {
  k_emit_count<<<kEmitCtas, kEmitThreads, 0, s>>>(P.dvals[dbuf], P.rec_rect, P.counters, (uint32_t)L.rcap, L.tile_w,
                                                  L.tile_h, P.epart);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = launch_scan_single(P.epart, (uint32_t)kEmitCtas, &P.counters->n_pairs, (uint32_t)L.pcap, P.counters, s);
  if (e != cudaSuccess) return e;
  k_emit_write<<<kEmitCtas, kEmitThreads, 0, s>>>(P.dvals[dbuf], P.rec_rect, P.rec_view, P.cams, P.counters,
                                                  (uint32_t)L.rcap, (uint32_t)L.pcap, L.tile_w, L.tile_h, P.epart,
                                                  P.pkeys[0], P.pvals[0]);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Per-tile [start, end) ranges by binary search over the sorted tile ids.
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t lower_bound_u32(const uint32_t *a, uint32_t n, uint32_t x) {
  uint32_t lo = 0, hi = n;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (a[mid] < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__global__ void k_tile_ranges(const uint32_t *__restrict__ pkeys, const Counters *cnt, uint32_t pcap,
                              uint32_t total_tiles, uint2 *ranges) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total_tiles) return;
  const uint32_t k = min(cnt->n_pairs, pcap);
  ranges[t] = make_uint2(lower_bound_u32(pkeys, k, t), lower_bound_u32(pkeys, k, t + 1));
}

cudaError_t launch_tile_ranges(const Layout &L, const WsPtrs &P, int pbuf, cudaStream_t s) {
  const uint32_t T = (uint32_t)L.total_tiles;
  if (T == 0) return cudaSuccess;
  k_tile_ranges<<<(T + 255) / 256, 256, 0, s>>>(P.pkeys[pbuf], P.counters, (uint32_t)L.pcap, T, P.ranges);
  return cudaGetLastError();
}

}  // namespace gs
