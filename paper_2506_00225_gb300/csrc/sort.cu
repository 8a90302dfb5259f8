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
// Radix sort: 8-bit digits, one histogram kernel for all digit passes (for
// the tile sort the pair emission counts the digits itself), then one
// kernel per pass.  Each CTA takes a tile ticket from an atomic counter,
// ranks its keys stably (warp match + per-warp counters), publishes its
// per-digit counts and looks back over earlier tiles for their prefixes
// (decoupled look-back).  A CTA only waits on tiles whose tickets were taken
// earlier, i.e. by CTAs already running; every wait is bounded and, if the
// bound is hit, raises the timeout status instead of hanging.  Keys are then
// reordered in shared memory so that the global writes of each digit run are
// contiguous.  Element counts are read from device memory, so the sort is
// graph-capturable.
#include "gs_internal.cuh"

namespace gs {

constexpr int kOsThreads = 256;
constexpr int kOsWarps = kOsThreads / 32;
// keys per thread of one sort tile, by element capacity: small sorts get
// small tiles (more CTAs in flight, shorter per-tile latency), large ones
// large tiles (fewer look-back steps, bounded look-back storage)
inline int os_items(int64_t capacity) { return capacity <= (1 << 20) ? 8 : 16; }
constexpr unsigned long long kFlagA = 1ull << 62;   // tile aggregate published
constexpr unsigned long long kFlagP = 2ull << 62;   // inclusive prefix published
constexpr unsigned long long kValMask = (1ull << 62) - 1;
constexpr int kLookWindow = 8;                       // predecessors read per look-back step

int sort_tiles(int64_t capacity) {
  const int64_t tile = (int64_t)kOsThreads * os_items(capacity);
  return (int)((capacity + tile - 1) / tile);
}

template <typename K>
__device__ __forceinline__ uint32_t digit_of(K key, int shift) {
  return (uint32_t)(key >> shift) & (kRadix - 1);
}

// Clears the tickets, the global histograms and the look-back words of the
// tiles the current element count needs.
__global__ void k_os_reset(const uint32_t *count_p, uint32_t cap, int passes, uint32_t *tickets, uint32_t *ghist,
                           unsigned long long *lookback, uint32_t lb_tiles, uint32_t tile_keys) {
  const uint32_t count = min(*count_p, cap);
  const uint32_t tiles = (count + tile_keys - 1) / tile_keys;
  const size_t words = (size_t)tiles * kRadix;
  const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (size_t)gridDim.x * blockDim.x;
  if (tid < (size_t)passes) tickets[tid] = 0u;
  if (tid < (size_t)passes * kRadix) ghist[tid] = 0u;
  for (int p = 0; p < passes; ++p) {
    unsigned long long *lb = lookback + (size_t)p * lb_tiles * kRadix;
    for (size_t i = tid; i < words; i += stride) lb[i] = 0ull;
  }
}

// Digit histograms of every pass in one read of the keys.  Each thread
// loads kHistItems keys before counting them (loads in flight); a warp's
// equal digits are merged with one shared-memory add.
constexpr int kHistItems = 4;

template <typename K>
__global__ void __launch_bounds__(256) k_os_hist(const K *__restrict__ keys, const uint32_t *count_p, uint32_t cap,
                                                 int passes, uint32_t *ghist) {
  __shared__ uint32_t h[kMaxRadixPasses][kRadix];
  for (int i = threadIdx.x; i < kMaxRadixPasses * kRadix; i += blockDim.x) (&h[0][0])[i] = 0u;
  __syncthreads();
  const uint32_t count = min(*count_p, cap);
  const uint32_t lt = lanemask_lt();
  const uint32_t stride = gridDim.x * blockDim.x * kHistItems;
  // uniform trip count so that every lane takes part in the match; item it
  // of a thread is element base + it * blockDim.x + threadIdx.x (coalesced)
  for (uint32_t base = blockIdx.x * blockDim.x * kHistItems; base < count; base += stride) {
    K k[kHistItems];
    bool ok[kHistItems];
#pragma unroll
    for (int it = 0; it < kHistItems; ++it) {
      const uint32_t i = base + it * blockDim.x + threadIdx.x;
      ok[it] = i < count;
      k[it] = ok[it] ? keys[i] : (K)0;
    }
#pragma unroll
    for (int it = 0; it < kHistItems; ++it) {
      for (int p = 0; p < passes; ++p) {
        const uint32_t d = ok[it] ? digit_of(k[it], p * kRadixBits) : (uint32_t)kRadix;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        if (ok[it] && (peers & lt) == 0u) atomicAdd(&h[p][d], (uint32_t)__popc(peers));
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < passes * kRadix; i += blockDim.x) {
    const uint32_t v = (&h[0][0])[i];
    if (v) atomicAdd(ghist + i, v);
  }
}

template <typename K, int ITEMS>
__global__ void __launch_bounds__(kOsThreads, sizeof(K) == 4 ? 3 : 2) k_os_pass(const K *__restrict__ keys_in,
                                                        const uint32_t *__restrict__ vals_in,
                                                        K *__restrict__ keys_out, uint32_t *__restrict__ vals_out,
                                                        const uint32_t *count_p, uint32_t cap, int shift,
                                                        const uint32_t *__restrict__ ghist,
                                                        unsigned long long *lookback, uint32_t *ticket,
                                                        Counters *counters, uint32_t spin_limit) {
  constexpr int kTile = kOsThreads * ITEMS;
  extern __shared__ unsigned long long os_smem[];
  K *skey = reinterpret_cast<K *>(os_smem);
  uint32_t *sval = reinterpret_cast<uint32_t *>(skey + kTile);
  __shared__ uint32_t wcnt[kOsWarps][kRadix];
  __shared__ uint32_t tile_pre[kRadix];
  __shared__ uint32_t out_base[kRadix];
  __shared__ uint32_t scan_tmp[33];
  __shared__ uint32_t s_tile;

  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5, d = threadIdx.x;
  const uint32_t count = min(*count_p, cap);
  if (threadIdx.x == 0) s_tile = atomicAdd(ticket, 1u);
  for (int i = threadIdx.x; i < kOsWarps * kRadix; i += kOsThreads) (&wcnt[0][0])[i] = 0u;
  __syncthreads();
  const uint32_t t = s_tile;
  const uint32_t base = t * kTile;
  if (base >= count) return;  // uniform: tiles past the data
  const uint32_t n_tile = min((uint32_t)kTile, count - base);

  // stable ranking: warp-striped items, in index order within each warp
  const uint32_t lt = lanemask_lt();
  // per item one word: its digit (kRadix past the tile's end) in the high
  // half and its rank among the warp's equal digits in the low half (fewer
  // live registers: more CTAs per SM)
  K key[ITEMS];
  uint32_t val[ITEMS], dl[ITEMS];
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const uint32_t off = warp * (32 * ITEMS) + i * 32 + lane;
    const bool ok = off < n_tile;
    key[i] = ok ? keys_in[base + off] : (K)0;
    val[i] = ok ? vals_in[base + off] : 0u;
    dl[i] = (ok ? digit_of(key[i], shift) : (uint32_t)kRadix) << 16;
  }
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const uint32_t di = dl[i] >> 16;
    const uint32_t peers = __match_any_sync(0xffffffffu, di);
    uint32_t b = 0;
    if (di < (uint32_t)kRadix) b = wcnt[warp][di];
    dl[i] |= b + __popc(peers & lt);
    __syncwarp();
    if ((peers & lt) == 0u && di < (uint32_t)kRadix) wcnt[warp][di] = b + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // per digit: exclusive prefix over warps, tile count
  uint32_t run = 0;
#pragma unroll
  for (int w = 0; w < kOsWarps; ++w) {
    const uint32_t c = wcnt[w][d];
    wcnt[w][d] = run;
    run += c;
  }
  const uint32_t tile_count = run;
  // publish this tile's aggregate, then look back for the exclusive prefix
  unsigned long long *lb = lookback + (size_t)t * kRadix;
  if (t == 0) {
    atomicExch(lb + d, kFlagP | (unsigned long long)tile_count);
  } else {
    atomicExch(lb + d, kFlagA | (unsigned long long)tile_count);
  }
  unsigned long long excl = 0ull;
  if (t > 0) {
    // the look-back reads kLookWindow predecessors at a time (their loads in
    // flight together) and walks them newest first: aggregates are added,
    // an inclusive prefix ends the walk, and an unpublished word (flag 0)
    // stops the window there to be read again (a bounded wait)
    int j = (int)t - 1;
    uint32_t spins = 0;
    bool done = false;
    while (!done) {
      unsigned long long v[kLookWindow];
#pragma unroll
      for (int i = 0; i < kLookWindow; ++i)
        v[i] = j - i >= 0 ? *reinterpret_cast<volatile unsigned long long *>(lookback + (size_t)(j - i) * kRadix + d)
                          : (unsigned long long)kFlagP;  // before tile 0: an empty inclusive prefix
      int taken = 0;
      bool blocked = false;
#pragma unroll
      for (int i = 0; i < kLookWindow; ++i) {
        if (done || blocked) continue;
        const unsigned long long flag = v[i] & ~kValMask;
        if (flag == 0ull) {
          blocked = true;
          continue;
        }
        excl += v[i] & kValMask;
        ++taken;
        if (flag == kFlagP) done = true;
      }
      j -= taken;
      if (blocked && !done) {
        if (++spins > spin_limit) { set_status(counters, kStatusTimeout); break; }
        __nanosleep(32);
      }
    }
    atomicExch(lb + d, kFlagP | (excl + tile_count));
  }
  // global start of digit d: all keys with a smaller digit + earlier tiles
  const uint32_t gpre = block_exclusive_scan(ghist[d], scan_tmp, &run);
  const uint32_t tpre = block_exclusive_scan(tile_count, scan_tmp, &run);
  tile_pre[d] = tpre;
  out_base[d] = gpre + (uint32_t)excl;
  __syncthreads();
  // local reorder by digit (stable), then contiguous global writes
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const uint32_t di = dl[i] >> 16;
    if (di < (uint32_t)kRadix) {
      const uint32_t lp = tile_pre[di] + wcnt[warp][di] + (dl[i] & 0xffffu);
      skey[lp] = key[i];
      sval[lp] = val[i];
    }
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < n_tile; i += kOsThreads) {
    const K k = skey[i];
    const uint32_t dd = digit_of(k, shift);
    const uint32_t pos = out_base[dd] + (i - tile_pre[dd]);
    keys_out[pos] = k;
    vals_out[pos] = sval[i];
  }
}

template <typename K, int ITEMS>
static cudaError_t os_passes(K *keys[2], uint32_t *vals[2], const uint32_t *count_p, uint32_t cap, int passes,
                             uint32_t *tickets, uint32_t *ghist, unsigned long long *lookback, uint32_t lb_tiles,
                             Counters *counters, uint32_t spin_limit, cudaStream_t s) {
  const size_t smem = (size_t)kOsThreads * ITEMS * (sizeof(K) + sizeof(uint32_t));
  {
    const cudaError_t e = ensure_smem_limit((const void *)k_os_pass<K, ITEMS>, (int)smem);
    if (e != cudaSuccess) return e;
  }
  for (int p = 0; p < passes; ++p) {
    const int src = p & 1, dst = src ^ 1;
    k_os_pass<K, ITEMS><<<lb_tiles, kOsThreads, smem, s>>>(keys[src], vals[src], keys[dst], vals[dst], count_p, cap,
                                                          p * kRadixBits, ghist + p * kRadix,
                                                          lookback + (size_t)p * lb_tiles * kRadix, tickets + p,
                                                          counters, spin_limit);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Clears the tickets, histograms and look-back words of a sort of at most
// `cap` elements (the element count is read on the device).
static cudaError_t os_reset(const uint32_t *count_p, uint32_t cap, int passes, uint32_t *tickets, uint32_t *ghist,
                            unsigned long long *lookback, cudaStream_t s) {
  const uint32_t lb_tiles = (uint32_t)sort_tiles(cap);
  if (passes < 1 || passes > kMaxRadixPasses || lb_tiles == 0) return cudaErrorInvalidValue;
  k_os_reset<<<sm_grid(2), 256, 0, s>>>(count_p, cap, passes, tickets, ghist, lookback, lb_tiles,
                                     (uint32_t)(kOsThreads * os_items(cap)));
  return cudaGetLastError();
}

// hist_ready: the reset and the digit histograms were done by the producer
// of the keys (the pair emission), so only the passes run here.
template <typename K>
static cudaError_t os_sort(K *keys[2], uint32_t *vals[2], const uint32_t *count_p, uint32_t cap, int bits,
                           uint32_t *tickets, uint32_t *ghist, unsigned long long *lookback, Counters *counters,
                           uint32_t spin_limit, cudaStream_t s, bool hist_ready = false) {
  const int passes = radix_passes(bits);
  const uint32_t lb_tiles = (uint32_t)sort_tiles(cap);
  const int items = os_items(cap);
  if (passes < 1 || passes > kMaxRadixPasses || lb_tiles == 0) return cudaErrorInvalidValue;
  if (!hist_ready) {
    cudaError_t e = os_reset(count_p, cap, passes, tickets, ghist, lookback, s);
    if (e != cudaSuccess) return e;
    k_os_hist<K><<<sm_grid(2), 256, 0, s>>>(keys[0], count_p, cap, passes, ghist);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (items == 8)
    return os_passes<K, 8>(keys, vals, count_p, cap, passes, tickets, ghist, lookback, lb_tiles, counters,
                           spin_limit, s);
  return os_passes<K, 16>(keys, vals, count_p, cap, passes, tickets, ghist, lookback, lb_tiles, counters,
                          spin_limit, s);
}

cudaError_t launch_radix_sort_u64(const Layout &L, const WsPtrs &P, int bits, int *final_buf, cudaStream_t s) {
  unsigned long long *k[2] = {P.dkeys[0], P.dkeys[1]};
  uint32_t *v[2] = {P.dvals[0], P.dvals[1]};
  *final_buf = radix_passes(bits) & 1;
  return os_sort<unsigned long long>(k, v, &P.counters->n_records, (uint32_t)L.rcap, bits, P.tickets, P.ghist,
                                     P.lb_depth, P.counters, L.spin_limit, s);
}

cudaError_t launch_radix_sort_u32(const Layout &L, const WsPtrs &P, int bits, int *final_buf, cudaStream_t s) {
  uint32_t *k[2] = {P.pkeys[0], P.pkeys[1]};
  uint32_t *v[2] = {P.pvals[0], P.pvals[1]};
  *final_buf = radix_passes(bits) & 1;
  // the pair emission has reset this sort and counted its digits
  return os_sort<uint32_t>(k, v, &P.counters->n_pairs, (uint32_t)L.pcap, bits, P.tickets + kMaxRadixPasses,
                           P.ghist + kMaxRadixPasses * kRadix, P.lb_pairs, P.counters, L.spin_limit, s, true);
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

// Pass 1: per chunk of depth-sorted records, the exclusive prefix of their
// tile counts inside the chunk (rloc) and the chunk total (epart).
__global__ void __launch_bounds__(kEmitThreads) k_emit_count(const uint32_t *__restrict__ sorted_rec,
                                                             const short4 *__restrict__ rect, const Counters *cnt,
                                                             uint32_t rcap, int tw, int th, uint32_t *epart,
                                                             uint32_t *rloc) {
  __shared__ uint32_t tmp[33];
  if (cnt->status & kStatusTimeout) return;  // the depth order may hold stale entries
  const uint32_t count = min(cnt->n_records, rcap);
  uint32_t begin, end;
  emit_chunk(count, begin, end);
  uint32_t run = 0;
  for (uint32_t q0 = begin; q0 < end; q0 += kEmitThreads) {
    const uint32_t q = q0 + threadIdx.x;
    const uint32_t nt = q < end ? record_ntiles(rect[sorted_rec[q]], tw, th) : 0u;
    uint32_t total;
    const uint32_t ex = block_exclusive_scan(nt, tmp, &total);
    if (q < end) rloc[q] = run + ex;
    run += total;
  }
  if (threadIdx.x == 0) epart[blockIdx.x] = run;
}

// Record (position in the depth order) of pair p of the emission: the chunk
// c (largest with epart[c] <= p), then the largest q of the chunk with
// rloc[q] <= p - epart[c].  Records with no tile are never selected.
__device__ __forceinline__ uint32_t find_record(uint32_t p, uint32_t count, uint32_t per, int n_chunks,
                                                const uint32_t *s_epart, const uint32_t *__restrict__ rloc) {
  int lo = 0, hi = n_chunks - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (s_epart[mid] <= p) lo = mid; else hi = mid - 1;
  }
  const uint32_t local = p - s_epart[lo];
  uint32_t qlo = (uint32_t)lo * per, qhi = min(count, qlo + per) - 1;
  while (qlo < qhi) {
    const uint32_t mid = (qlo + qhi + 1) >> 1;
    if (__ldg(rloc + mid) <= local) qlo = mid; else qhi = mid - 1;
  }
  return qlo;
}

// First pair of depth-order record q in the whole emission (chunk q / per).
__device__ __forceinline__ uint32_t pair_start(uint32_t q, uint32_t per, const uint32_t *s_epart,
                                               const uint32_t *__restrict__ rloc) {
  return s_epart[q / per] + __ldg(rloc + q);
}

// Global tile id of the j-th tile (row-major) of record r's tile rectangle.
// TW, TH > 0 fix the tile shape at compile time (the divisions become
// shifts); 0 takes tw, th.  Rectangle coordinates are non-negative.
template <int TW, int TH>
__device__ __forceinline__ uint32_t pair_tile(uint32_t r, uint32_t j, const short4 *__restrict__ rect,
                                              const int32_t *__restrict__ rview, const DevCam *__restrict__ cams,
                                              int tw, int th) {
  const uint32_t w = TW > 0 ? (uint32_t)TW : (uint32_t)tw, h = TH > 0 ? (uint32_t)TH : (uint32_t)th;
  const short4 rc = __ldg(rect + r);
  const DevCam &c = cams[__ldg(rview + r)];
  const int tx0 = (int)((uint32_t)rc.x / w), gw = (int)((uint32_t)rc.y / w) - tx0 + 1;
  const int ty0 = (int)((uint32_t)rc.z / h);
  const int ty = ty0 + (int)(j / (uint32_t)gw), tx = tx0 + (int)(j % (uint32_t)gw);
  return c.tile_off + (uint32_t)(ty * c.tiles_x + tx);
}

// Pass 2, balanced over pairs.  A CTA takes blocks of kEmitBlock consecutive
// pairs; two threads find the records of the block's first and last pair
// (search over the chunk totals, then over the chunk's rloc), the block's
// records' first pairs are staged in shared memory, and every pair finds its
// record by a binary search there -- one chain of dependent global loads
// per block instead of one per pair.  Consecutive threads write consecutive
// pairs, and the output equals the depth-ordered, row-major-within-record
// emission.  The same kernel counts the 8-bit digits of the tile ids for the
// tile sort that follows: a warp's 32 consecutive pairs mostly come in runs
// of equal digits (the tiles of one record), so each run adds its length
// with one shared-memory atomic, and each CTA adds its counts to the global
// histograms at the end.
constexpr int kEmitHistPasses = 4;                          // 32-bit tile ids
constexpr int kEmitItems = 8;                               // pairs per thread and block
constexpr int kEmitBlock = kEmitThreads * kEmitItems;       // pairs per CTA block
template <int TW, int TH>
__global__ void __launch_bounds__(kEmitThreads) k_emit_write(const uint32_t *__restrict__ sorted_rec,
                                                             const short4 *__restrict__ rect,
                                                             const int32_t *__restrict__ rview,
                                                             const DevCam *__restrict__ cams, const Counters *cnt,
                                                             uint32_t rcap, uint32_t pcap, int tw, int th,
                                                             const uint32_t *__restrict__ epart,
                                                             const uint32_t *__restrict__ rloc,
                                                             uint32_t *__restrict__ pkeys,
                                                             uint32_t *__restrict__ pvals, int hist_passes,
                                                             uint32_t *__restrict__ ghist, int n_chunks) {
  __shared__ uint32_t s_epart[kEmitCtasMax];
  __shared__ uint32_t s_hist[kEmitHistPasses * kRadix];
  __shared__ uint32_t s_start[kEmitBlock];  // first pair of records qa, qa + 1, ...
  __shared__ uint32_t s_q[2];
  if (cnt->status & kStatusTimeout) return;
  for (int i = threadIdx.x; i < n_chunks; i += kEmitThreads) s_epart[i] = epart[i];
  for (int i = threadIdx.x; i < kEmitHistPasses * kRadix; i += kEmitThreads) s_hist[i] = 0u;
  __syncthreads();
  const uint32_t count = min(cnt->n_records, rcap);
  const uint32_t npairs = min(cnt->n_pairs, pcap);
  const uint32_t per = (count + n_chunks - 1) / n_chunks;
  const uint32_t lane = lane_id();
  for (uint32_t P0 = blockIdx.x * (uint32_t)kEmitBlock; P0 < npairs; P0 += gridDim.x * (uint32_t)kEmitBlock) {
    const uint32_t P1 = min(npairs, P0 + (uint32_t)kEmitBlock);
    if (threadIdx.x < 2) s_q[threadIdx.x] = find_record(threadIdx.x ? P1 - 1 : P0, count, per, n_chunks, s_epart, rloc);
    __syncthreads();
    const uint32_t qa = s_q[0], nrec = s_q[1] - qa + 1;
    // more records than staging slots only with records of no tile
    const bool staged = nrec <= (uint32_t)kEmitBlock;
    if (staged)
      for (uint32_t i = threadIdx.x; i < nrec; i += kEmitThreads) s_start[i] = pair_start(qa + i, per, s_epart, rloc);
    __syncthreads();
    uint32_t rec[kEmitItems], jj[kEmitItems], key[kEmitItems];
#pragma unroll
    for (int it = 0; it < kEmitItems; ++it) {
      const uint32_t p = P0 + it * kEmitThreads + threadIdx.x;
      rec[it] = 0u; jj[it] = 0u;
      if (p < P1) {
        if (staged) {
          int lo = 0, hi = (int)nrec - 1;
          while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_start[mid] <= p) lo = mid; else hi = mid - 1;
          }
          rec[it] = qa + (uint32_t)lo;
          jj[it] = p - s_start[lo];
        } else {
          rec[it] = find_record(p, count, per, n_chunks, s_epart, rloc);
          jj[it] = p - pair_start(rec[it], per, s_epart, rloc);
        }
      }
    }
#pragma unroll
    for (int it = 0; it < kEmitItems; ++it)
      if (P0 + it * kEmitThreads + threadIdx.x < P1) rec[it] = __ldg(sorted_rec + rec[it]);
#pragma unroll
    for (int it = 0; it < kEmitItems; ++it) {
      const uint32_t p = P0 + it * kEmitThreads + threadIdx.x;
      key[it] = 0xffffffffu;
      if (p < P1) {
        key[it] = pair_tile<TW, TH>(rec[it], jj[it], rect, rview, cams, tw, th);
        pkeys[p] = key[it];
        pvals[p] = rec[it];
      }
    }
    // lanes of a warp hold consecutive pairs of each item
#pragma unroll
    for (int it = 0; it < kEmitItems; ++it) {
      const bool ok = P0 + it * kEmitThreads + threadIdx.x < P1;
      for (int q = 0; q < hist_passes; ++q) {
        // lanes past the end carry digit kRadix, which starts a run and is not counted
        const uint32_t d = ok ? (key[it] >> (q * kRadixBits)) & (kRadix - 1) : (uint32_t)kRadix;
        const uint32_t prev = __shfl_up_sync(0xffffffffu, d, 1);
        const bool start = lane == 0 || prev != d;
        const uint32_t starts = __ballot_sync(0xffffffffu, start);
        if (start && d < (uint32_t)kRadix) {
          const uint32_t after = lane == 31 ? 0u : starts & (0xffffffffu << (lane + 1));
          const uint32_t end = after ? (uint32_t)(__ffs(after) - 1) : 32u;
          atomicAdd(&s_hist[q * kRadix + d], end - lane);
        }
      }
    }
    __syncthreads();  // s_q and s_start are rewritten by the next block
  }
  if (hist_passes > 0) {
    __syncthreads();
    for (int i = threadIdx.x; i < hist_passes * kRadix; i += kEmitThreads)
      if (s_hist[i]) atomicAdd(ghist + i, s_hist[i]);
  }
}

cudaError_t launch_emit_pairs(const Layout &L, const WsPtrs &P, int dbuf, cudaStream_t s) {
  // chunk count: the same in the count pass (its grid), the scan and the write pass
  const int n_chunks = emit_chunks();
  if (n_chunks < 1) return cudaErrorInvalidDevice;
  k_emit_count<<<n_chunks, kEmitThreads, 0, s>>>(P.dvals[dbuf], P.rec_rect, P.counters, (uint32_t)L.rcap, L.tile_w,
                                                  L.tile_h, P.epart, P.rloc);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = launch_scan_single(P.epart, (uint32_t)n_chunks, &P.counters->n_pairs, (uint32_t)L.pcap, P.counters, s);
  if (e != cudaSuccess) return e;
  // the tile sort's reset, then the emission counts its digits
  const int passes = radix_passes(L.key_bits_tile);
  if (passes > kEmitHistPasses) return cudaErrorInvalidValue;
  uint32_t *ghist = P.ghist + kMaxRadixPasses * kRadix;
  e = os_reset(&P.counters->n_pairs, (uint32_t)L.pcap, passes, P.tickets + kMaxRadixPasses, ghist, P.lb_pairs, s);
  if (e != cudaSuccess) return e;
  const int tw = L.tile_w, th = L.tile_h;
  auto kern = tw == 16 && th == 16 ? k_emit_write<16, 16>
            : tw == 16 && th == 8  ? k_emit_write<16, 8>
            : tw == 8 && th == 8   ? k_emit_write<8, 8>
            : tw == 32 && th == 8  ? k_emit_write<32, 8>
                                   : k_emit_write<0, 0>;
  kern<<<sm_grid(8), kEmitThreads, 0, s>>>(P.dvals[dbuf], P.rec_rect, P.rec_view, P.cams, P.counters,
                                           (uint32_t)L.rcap, (uint32_t)L.pcap, tw, th, P.epart, P.rloc, P.pkeys[0],
                                           P.pvals[0], passes, ghist, n_chunks);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Per-tile [start, end) ranges from the sorted tile ids: every pair that
// starts or ends a run writes its tile's bound; tiles with no pair keep the
// empty range written first.
// ---------------------------------------------------------------------------

__global__ void k_ranges_clear(uint2 *ranges, uint32_t total_tiles) {
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < total_tiles; t += gridDim.x * blockDim.x)
    ranges[t] = make_uint2(0u, 0u);
}

// Each thread takes 4 consecutive sorted tile ids (one 16-byte load when
// the group is whole) plus its neighbours, and writes the bounds of the runs
// that start or end there.
__global__ void k_ranges_mark(const uint32_t *__restrict__ pkeys, const Counters *cnt, uint32_t pcap,
                              uint32_t total_tiles, uint2 *ranges) {
  const uint32_t k = min(cnt->n_pairs, pcap);
  for (uint32_t i0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x); i0 < k; i0 += 4 * gridDim.x * blockDim.x) {
    uint32_t t[6];
    t[0] = i0 > 0 ? pkeys[i0 - 1] : 0xffffffffu;
    if (i0 + 4 <= k) {
      const uint4 v = *reinterpret_cast<const uint4 *>(pkeys + i0);
      t[1] = v.x; t[2] = v.y; t[3] = v.z; t[4] = v.w;
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) t[1 + j] = i0 + j < k ? pkeys[i0 + j] : 0xffffffffu;
    }
    t[5] = i0 + 4 < k ? pkeys[i0 + 4] : 0xffffffffu;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint32_t i = i0 + j, tt = t[1 + j];
      if (i >= k || tt >= total_tiles) continue;
      if (t[j] != tt) ranges[tt].x = i;
      if (t[2 + j] != tt) ranges[tt].y = i + 1;
    }
  }
}

cudaError_t launch_tile_ranges(const Layout &L, const WsPtrs &P, int pbuf, cudaStream_t s) {
  const uint32_t T = (uint32_t)L.total_tiles;
  if (T == 0) return cudaSuccess;
  const unsigned g4 = sm_grid(4);
  if (g4 == 0) return cudaErrorInvalidDevice;
  k_ranges_clear<<<min((T + 255) / 256, g4), 256, 0, s>>>(P.ranges, T);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_ranges_mark<<<g4, 256, 0, s>>>(P.pkeys[pbuf], P.counters, (uint32_t)L.pcap, T, P.ranges);
  return cudaGetLastError();
}

}  // namespace gs
