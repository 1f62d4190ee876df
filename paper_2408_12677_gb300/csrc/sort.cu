// Tile binning (Sec. III-B.3: screen tiles, per-tile depth order):
//   1. LSD radix sort of the Gaussians by the float32 bit pattern of their
//      camera depth (z > 0, so the bits order like the values),
//   2. duplication: each depth-sorted Gaussian writes one (tile, id) pair per
//      covered tile, at offsets from an exclusive scan of the tile counts,
//   3. stable LSD radix sort of the pairs by tile id only (ceil(log2 T) bits),
//   4. per-tile [start, end) ranges.
// Sorting depth once over N Gaussians and then only the tile bits over the P
// pairs gives the same (tile, depth, id) order as one 64-bit key sort over P
// at a fraction of the passes over the pair array.
//
// The radix sort is reduce-then-scan with a fixed grid: each block owns a
// contiguous chunk; an upsweep builds per-block digit histograms, one block
// scans them digit-major, and a downsweep ranks every item stably (warp
// match + per-warp digit counts) and scatters it.  No block ever waits on
// another block.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace gs {

namespace {

constexpr int kRadix = 256;
constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kScanThreads = 1024;

__device__ __forceinline__ uint32_t read_n(const uint32_t* n_dev, uint32_t n_host) {
  return n_dev ? *n_dev : n_host;
}

__global__ void __launch_bounds__(kSortThreads) radix_upsweep(const uint32_t* __restrict__ keys,
                                                              const uint32_t* n_dev, uint32_t n_host, int shift,
                                                              uint32_t mask, uint32_t* __restrict__ ghist, int G) {
  __shared__ uint32_t h[kRadix];
  h[threadIdx.x] = 0;
  __syncthreads();
  const uint32_t n = read_n(n_dev, n_host);
  const uint32_t chunk = (n + G - 1) / G;
  const uint64_t beg64 = (uint64_t)blockIdx.x * chunk;
  const uint32_t beg = (uint32_t)(beg64 < n ? beg64 : (uint64_t)n);
  const uint32_t end = (uint32_t)(beg64 + chunk < n ? beg64 + chunk : (uint64_t)n);
  // lanes with the same digit add their count with one shared atomic (keys
  // in a run share the high digits: per-lane atomics would serialise)
  const uint32_t lane = threadIdx.x & 31;
  for (uint32_t base = beg; base < end; base += kSortThreads) {
    const uint32_t i = base + threadIdx.x;
    const uint32_t d = i < end ? (keys[i] >> shift) & mask : 0xFFFFFFFFu;
    const uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
    if (d != 0xFFFFFFFFu && lane == (uint32_t)(__ffs(peers) - 1)) atomicAdd(&h[d], (uint32_t)__popc(peers));
  }
  __syncthreads();
  ghist[threadIdx.x * G + blockIdx.x] = h[threadIdx.x];
}

// exclusive scan of a value per thread over a 256-thread block; *total gets the sum
__device__ __forceinline__ uint32_t block256_exclusive_scan(uint32_t v, uint32_t* total) {
  __shared__ uint32_t s_w[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, off);
    if (lane >= off) x += y;
  }
  if (lane == 31) s_w[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < 8 ? s_w[lane] : 0u;
#pragma unroll
    for (int off = 1; off < 8; off <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, w, off);
      if (lane >= off) w += y;
    }
    if (lane < 8) s_w[lane] = w;
  }
  __syncthreads();
  const uint32_t prefix = warp > 0 ? s_w[warp - 1] : 0u;
  *total = s_w[7];
  __syncthreads();
  return prefix + x - v;
}

// Row scan of the digit-major histogram: block d turns hist[d][0..G) into its
// exclusive prefix over blocks and writes the digit total to totals[d].
__global__ void __launch_bounds__(kSortThreads) radix_rowscan(uint32_t* __restrict__ ghist, int G,
                                                              uint32_t* __restrict__ totals) {
  uint32_t* row = ghist + (size_t)blockIdx.x * G;
  const int per = (G + kSortThreads - 1) / kSortThreads;
  const int beg = min(G, (int)threadIdx.x * per), end = min(G, beg + per);
  uint32_t sum = 0;
  for (int i = beg; i < end; ++i) sum += row[i];
  uint32_t total;
  uint32_t run = block256_exclusive_scan(sum, &total);
  for (int i = beg; i < end; ++i) {
    const uint32_t v = row[i];
    row[i] = run;
    run += v;
  }
  if (threadIdx.x == 0) totals[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kSortThreads) radix_downsweep(
    const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin, uint32_t* __restrict__ kout,
    uint32_t* __restrict__ vout, const uint32_t* n_dev, uint32_t n_host, int shift, uint32_t mask,
    const uint32_t* __restrict__ ghist, const uint32_t* __restrict__ totals, int G) {
  __shared__ uint32_t s_off[kRadix];
  __shared__ uint32_t s_wc[kSortWarps][kRadix];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint32_t all;
  const uint32_t digit_base = block256_exclusive_scan(totals[tid], &all);
  s_off[tid] = digit_base + ghist[tid * G + blockIdx.x];
  for (int w = 0; w < kSortWarps; ++w) s_wc[w][tid] = 0;
  const uint32_t n = read_n(n_dev, n_host);
  const uint32_t chunk = (n + G - 1) / G;
  const uint64_t beg64 = (uint64_t)blockIdx.x * chunk;
  const uint32_t beg = (uint32_t)(beg64 < n ? beg64 : (uint64_t)n);
  const uint32_t end = (uint32_t)(beg64 + chunk < n ? beg64 + chunk : (uint64_t)n);
  const uint32_t lt_mask = (1u << lane) - 1u;
  __syncthreads();
  for (uint32_t base = beg; base < end; base += kSortThreads) {
    const uint32_t i = base + tid;
    const bool valid = i < end;
    uint32_t k = 0, v = 0, d = 0xFFFFFFFFu;
    if (valid) {
      k = kin[i];
      v = vin ? vin[i] : i;
      d = (k >> shift) & mask;
    }
    const uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
    const uint32_t rank = __popc(peers & lt_mask);
    if (valid && rank == 0) s_wc[warp][d] = __popc(peers);
    __syncthreads();
    {
      uint32_t run = s_off[tid];
#pragma unroll
      for (int w = 0; w < kSortWarps; ++w) {
        uint32_t c = s_wc[w][tid];
        s_wc[w][tid] = run;
        run += c;
      }
      s_off[tid] = run;
    }
    __syncthreads();
    if (valid) {
      const uint32_t pos = s_wc[warp][d] + rank;
      kout[pos] = k;
      vout[pos] = v;
    }
    __syncthreads();
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) s_wc[w][tid] = 0;
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// duplication
// ---------------------------------------------------------------------------
constexpr int kDupThreads = 256;
constexpr int kDupItems = 4;  // per thread, consecutive
constexpr int kDupChunk = kDupThreads * kDupItems;

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* total) {
  static_assert(kDupThreads == 256, "block scan is written for 256 threads");
  return block256_exclusive_scan(v, total);
}

__global__ void __launch_bounds__(kDupThreads) dup_count_kernel(int n, const uint32_t* __restrict__ sorted_ids,
                                                                const uint32_t* __restrict__ tiles,
                                                                uint32_t* __restrict__ block_sums) {
  const int base = blockIdx.x * kDupChunk + threadIdx.x * kDupItems;
  uint32_t s = 0;
#pragma unroll
  for (int j = 0; j < kDupItems; ++j)
    if (base + j < n) s += tiles[sorted_ids[base + j]];
  uint32_t total;
  block_exclusive_scan(s, &total);
  if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

// exclusive scan of the block sums (one block), total to n_pairs
__global__ void __launch_bounds__(kScanThreads) dup_scan_kernel(uint32_t* __restrict__ sums, int len,
                                                                uint32_t capacity, uint32_t* __restrict__ n_pairs,
                                                                unsigned long long* __restrict__ n_full) {
  __shared__ unsigned long long s[kScanThreads];
  const int per = (len + kScanThreads - 1) / kScanThreads;
  const int beg = min(len, (int)threadIdx.x * per), end = min(len, beg + per);
  unsigned long long sum = 0;
  for (int i = beg; i < end; ++i) sum += sums[i];
  s[threadIdx.x] = sum;
  __syncthreads();
  for (int off = 1; off < kScanThreads; off <<= 1) {
    unsigned long long v = threadIdx.x >= (unsigned)off ? s[threadIdx.x - off] : 0ull;
    __syncthreads();
    s[threadIdx.x] += v;
    __syncthreads();
  }
  unsigned long long run = s[threadIdx.x] - sum;
  for (int i = beg; i < end; ++i) {
    unsigned long long v = sums[i];
    sums[i] = (uint32_t)(run < 0xFFFFFFFFull ? run : 0xFFFFFFFFull);
    run += v;
  }
  if (threadIdx.x == kScanThreads - 1) {
    unsigned long long tot = s[kScanThreads - 1];
    *n_full = tot;
    *n_pairs = (uint32_t)(tot < (unsigned long long)capacity ? tot : (unsigned long long)capacity);
  }
}

// Writes the pairs of the block's kDupChunk consecutive (depth-sorted) items
// at the offsets of the scan.  The block's pairs are spread over all its
// threads -- pair k of the block goes to thread k mod 256, its item found by
// a binary search over the block's exclusive prefix in shared memory -- so a
// Gaussian covering thousands of tiles does not serialise one thread, and
// consecutive threads write consecutive slots.
__global__ void __launch_bounds__(kDupThreads) dup_write_kernel(
    int n, const uint32_t* __restrict__ sorted_ids, const uint32_t* __restrict__ tiles,
    const ushort4* __restrict__ rects, const __grid_constant__ TileMap map,
    const uint32_t* __restrict__ block_offsets, uint32_t* __restrict__ tile_keys, uint32_t* __restrict__ vals,
    uint32_t capacity, uint32_t* overflow) {
  __shared__ uint32_t s_excl[kDupChunk];
  __shared__ uint32_t s_id[kDupChunk];
  const int base = blockIdx.x * kDupChunk + threadIdx.x * kDupItems;
  uint32_t cnt[kDupItems];
  uint32_t id[kDupItems];
  uint32_t s = 0;
#pragma unroll
  for (int j = 0; j < kDupItems; ++j) {
    id[j] = base + j < n ? sorted_ids[base + j] : 0u;
    cnt[j] = base + j < n ? tiles[id[j]] : 0u;
    s += cnt[j];
  }
  uint32_t total;
  uint32_t run = block_exclusive_scan(s, &total);
#pragma unroll
  for (int j = 0; j < kDupItems; ++j) {
    s_excl[threadIdx.x * kDupItems + j] = run;
    s_id[threadIdx.x * kDupItems + j] = id[j];
    run += cnt[j];
  }
  __syncthreads();
  const uint64_t off0 = (uint64_t)block_offsets[blockIdx.x];
  bool over = false;
  for (uint32_t k = threadIdx.x; k < total; k += kDupThreads) {
    // the item owning pair k: the last o with s_excl[o] <= k (items with no
    // pairs share their successor's prefix and are never the last such o)
    int o = 0;
#pragma unroll
    for (int step = kDupChunk / 2; step > 0; step >>= 1)
      if (s_excl[o + step] <= k) o += step;
    const uint32_t g = s_id[o];
    const ushort4 r = rects[g];
    const uint32_t local = k - s_excl[o];
    const uint32_t width = (uint32_t)(r.z - r.x);
    const uint32_t ty = r.y + local / width, tx = r.x + local % width;
    const int v = map.views == 1 ? 0 : (int)(g / (uint32_t)map.n_per_view);
    const uint64_t off = off0 + k;
    if (off < capacity) {
      tile_keys[off] = map.tile_base[v] + ty * (uint32_t)map.tiles_x[v] + tx;
      vals[off] = g;
    } else {
      over = true;
    }
  }
  if (over) atomicOr(overflow, 1u);
}

__global__ void tile_ranges_kernel(const uint32_t* __restrict__ keys, const uint32_t* n_dev, uint32_t n_host,
                                   uint2* __restrict__ ranges) {
  const uint32_t n = read_n(n_dev, n_host);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t k = keys[i];
    if (i == 0 || keys[i - 1] != k) ranges[k].x = i;
    if (i + 1 == n || keys[i + 1] != k) ranges[k].y = i + 1;
  }
}

__global__ void export_keys_kernel(const uint32_t* __restrict__ tiles, const uint32_t* __restrict__ ids,
                                   const uint32_t* __restrict__ depth_key, uint32_t P, uint64_t* __restrict__ keys,
                                   uint32_t* __restrict__ ids_out) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x) {
    const uint32_t g = ids[i];
    keys[i] = ((uint64_t)tiles[i] << 32) | (uint64_t)depth_key[g];
    ids_out[i] = g;
  }
}

// one block per tile writes the keys of its range
__global__ void export_keys_ranges_kernel(const uint2* __restrict__ ranges, const uint32_t* __restrict__ ids,
                                          const uint32_t* __restrict__ depth_key, uint64_t* __restrict__ keys,
                                          uint32_t* __restrict__ ids_out) {
  const uint2 r = ranges[blockIdx.x];
  for (uint32_t i = r.x + threadIdx.x; i < r.y; i += blockDim.x) {
    const uint32_t g = ids[i];
    keys[i] = ((uint64_t)blockIdx.x << 32) | (uint64_t)depth_key[g];
    ids_out[i] = g;
  }
}

int sort_blocks(uint32_t n, int num_sms, int max_blocks) {
  // at least four rounds of 256 items per block; at most eight blocks per SM
  // (one resident wave of 2048 threads per SM)
  int g = (int)std::min<uint64_t>(((uint64_t)n + 1023) / 1024, (uint64_t)std::max(1, 8 * num_sms));
  return std::max(1, std::min(g, max_blocks));
}

}  // namespace

int radix_sort_pairs(SortBuffers& b, const uint32_t* in_k, const uint32_t* in_v, uint32_t n_max,
                     const uint32_t* n_dev, int bits, int num_sms, cudaStream_t s, int64_t* launches) {
  const bool in_place = in_k == b.keys[0];
  if (n_max == 0 || bits <= 0) return in_place ? 0 : -1;
  const int G = sort_blocks(n_max, num_sms, b.max_blocks);
  const uint32_t* ck = in_k;
  const uint32_t* cv = in_v;
  int out = in_place ? 1 : 0, last = -1;
  for (int shift = 0; shift < bits; shift += 8) {
    const int nb = std::min(8, bits - shift);
    const uint32_t mask = (1u << nb) - 1u;
    radix_upsweep<<<G, kSortThreads, 0, s>>>(ck, n_dev, n_max, shift, mask, b.hist, G);
    radix_rowscan<<<kRadix, kSortThreads, 0, s>>>(b.hist, G, b.hist + (size_t)kRadix * G);
    radix_downsweep<<<G, kSortThreads, 0, s>>>(ck, cv, b.keys[out], b.vals[out], n_dev, n_max, shift, mask, b.hist,
                                               b.hist + (size_t)kRadix * G, G);
    if (launches) *launches += 3;
    ck = b.keys[out];
    cv = b.vals[out];
    last = out;
    out ^= 1;
  }
  return last;
}

int dup_blocks(int n) { return (n + kDupChunk - 1) / kDupChunk; }

void launch_dup_count_scan(const DupArgs& a, cudaStream_t s, int64_t* launches) {
  const int nb = dup_blocks(a.n);
  if (nb == 0) {
    cudaMemsetAsync(a.n_pairs, 0, sizeof(uint32_t), s);
    cudaMemsetAsync(a.n_pairs_full, 0, sizeof(unsigned long long), s);
    return;
  }
  dup_count_kernel<<<nb, kDupThreads, 0, s>>>(a.n, a.sorted_ids, a.tiles_touched, a.block_sums);
  dup_scan_kernel<<<1, kScanThreads, 0, s>>>(a.block_sums, nb, a.capacity, a.n_pairs, a.n_pairs_full);
  if (launches) *launches += 2;
}

void launch_dup_write(const DupArgs& a, cudaStream_t s, int64_t* launches) {
  const int nb = dup_blocks(a.n);
  if (nb == 0) return;
  dup_write_kernel<<<nb, kDupThreads, 0, s>>>(a.n, a.sorted_ids, a.tiles_touched, a.rects, a.map,
                                              a.block_sums, a.tile_keys, a.vals, a.capacity, a.overflow);
  if (launches) *launches += 1;
}

void launch_tile_ranges(const uint32_t* sorted_tiles, const uint32_t* n_dev, uint32_t n_max, uint2* ranges,
                        int n_tiles, int num_sms, cudaStream_t s, int64_t* launches) {
  cudaMemsetAsync(ranges, 0, sizeof(uint2) * (size_t)n_tiles, s);
  if (n_max == 0) return;
  int g = (int)std::min<uint64_t>(((uint64_t)n_max + 255) / 256, (uint64_t)(8 * num_sms));
  tile_ranges_kernel<<<std::max(g, 1), 256, 0, s>>>(sorted_tiles, n_dev, n_max, ranges);
  if (launches) *launches += 1;
}

void launch_export_keys_ranges(const uint2* ranges, int n_tiles, const uint32_t* sorted_ids,
                               const uint32_t* depth_key_by_id, uint32_t P, uint64_t* keys, uint32_t* ids,
                               cudaStream_t s) {
  if (P == 0 || n_tiles == 0) return;
  export_keys_ranges_kernel<<<n_tiles, 128, 0, s>>>(ranges, sorted_ids, depth_key_by_id, keys, ids);
}

void launch_export_keys(const uint32_t* sorted_tiles, const uint32_t* sorted_ids, const uint32_t* depth_key_by_id,
                        uint32_t P, uint64_t* keys, uint32_t* ids, cudaStream_t s) {
  if (P == 0) return;
  int g = (int)std::min<uint32_t>((P + 255) / 256, 1024u);
  export_keys_kernel<<<g, 256, 0, s>>>(sorted_tiles, sorted_ids, depth_key_by_id, P, keys, ids);
}

}  // namespace gs
