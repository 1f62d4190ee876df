// Tile binning by counting scatter and per-tile sort (Sec. III-B.3: screen
// tiles, Gaussians sorted by depth in each tile):
//   1. count:   every (Gaussian, tile) pair of a Gaussian's tile rectangle adds
//               one to its tile's counter,
//   2. scan:    exclusive scan of the tile counters -> list offsets (and the
//               total pair count and the longest list),
//   3. scatter: every pair takes a slot of its tile's list with an atomic
//               cursor and writes its Gaussian id,
//   4. sort:    each tile's list is sorted by the 64-bit key (float32 depth
//               bits << 32 | id) with a bitonic network: by one warp in
//               registers up to 512 entries, by a CTA in shared memory beyond.
// The per-tile keys are unique, so the result is exactly the (tile, depth, id)
// order of a stable sort and does not depend on the scatter's atomic order.
// Counting and scattering expand the rectangles warp-cooperatively, so a
// Gaussian covering thousands of tiles is spread over the whole warp.
#include "common.cuh"
#include "internal.h"

namespace gs {

namespace {

constexpr int kBinThreads = 256;
constexpr int kBinWarps = kBinThreads / 32;
constexpr int kScanThreads = 1024;
constexpr int kSortThreads = 128;
constexpr int kSortWarps = kSortThreads / 32;  // tiles per CTA of the per-tile sort
constexpr int kWarpSortMax = 512;              // lists up to this length are sorted by one warp

// Global tile of tile (tx, ty) of the view that item `it` belongs to.
struct ItemTiles {
  uint32_t base, stride;  // tile_base[v], tiles_x[v]
};
__device__ __forceinline__ ItemTiles item_tiles(const TileMap& map, uint32_t it) {
  if (map.views == 1) return ItemTiles{0u, (uint32_t)map.tiles_x[0]};
  const int v = (int)(it / (uint32_t)map.n_per_view);
  return ItemTiles{map.tile_base[v], (uint32_t)map.tiles_x[v]};
}

// Calls f(item, global tile, active) for every tile of every item's
// rectangle.  Items with more than kBigTiles tiles come from the queue
// the projection built (see the end); the others are expanded by their
// block, 256 consecutive items at a time: a block scan of their tile counts
// gives each item's first pair, and the block's threads take consecutive
// pairs (owner found by binary search over the prefix in shared memory), so
// one large splat is spread over the whole block and large splats clustered
// in one region are averaged over 256 items.
// `active` is the mask of lanes of the calling warp that call f together.
template <bool SMALL = true, class F>
__device__ __forceinline__ void for_each_pair(int n, const ushort4* __restrict__ rects,
                                              const uint32_t* __restrict__ tiles, const TileMap& map,
                                              const uint32_t* __restrict__ big_queue,
                                              const uint32_t* __restrict__ big_len, F f) {
  __shared__ uint32_t s_excl[kBinThreads];
  __shared__ ushort4 s_rect[kBinThreads];
  __shared__ ItemTiles s_map[kBinThreads];
  __shared__ uint32_t s_wsum[kBinWarps];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int base = blockIdx.x * kBinThreads; SMALL && base < n; base += gridDim.x * kBinThreads) {
    const int g = base + threadIdx.x;
    uint32_t cnt = g < n ? tiles[g] : 0u;
    if (cnt > kBigTiles) cnt = 0;  // expanded from the queue below
    const ushort4 r = g < n ? rects[g] : make_ushort4(0, 0, 0, 0);
    uint32_t incl = cnt;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, off);
      if (lane >= off) incl += y;
    }
    __syncthreads();  // previous round done with the shared arrays
    if (lane == 31) s_wsum[w] = incl;
    __syncthreads();
    uint32_t wpre = 0, total = 0;
#pragma unroll
    for (int k = 0; k < kBinWarps; ++k) {
      const uint32_t sk = s_wsum[k];
      wpre += k < w ? sk : 0u;
      total += sk;
    }
    s_excl[threadIdx.x] = wpre + incl - cnt;
    s_rect[threadIdx.x] = r;
    s_map[threadIdx.x] = item_tiles(map, (uint32_t)min(g, n - 1));
    __syncthreads();
    for (uint32_t k0 = 0; k0 < total; k0 += kBinThreads) {
      const uint32_t k = k0 + threadIdx.x;
      const unsigned active = __ballot_sync(0xFFFFFFFFu, k < total);
      if (k >= total) break;
      int o = 0;
#pragma unroll
      for (int step = kBinThreads / 2; step > 0; step >>= 1)
        if (s_excl[o + step] <= k) o += step;
      const ushort4 ro = s_rect[o];
      const ItemTiles mt = s_map[o];
      const uint32_t local = k - s_excl[o];
      const uint32_t width = (uint32_t)(ro.z - ro.x);
      const uint32_t ty = ro.y + local / width, tx = ro.x + local % width;
      f(base + o, mt.base + ty * mt.stride + tx, active);
    }
  }
  // large splats: warp w of the grid expands queued items w, w + W, ...
  // spreading each one's tiles over its lanes (no shared cursor: one address
  // hit by every warp would serialise)
  const uint32_t nbig = *big_len;
  const uint32_t gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t item = gwarp; item < nbig; item += nwarps) {
    const uint32_t g = big_queue[item];
    const ushort4 ro = rects[g];
    const uint32_t cnt = tiles[g];
    const ItemTiles mt = item_tiles(map, g);
    const uint32_t width = (uint32_t)(ro.z - ro.x);
    for (uint32_t k0 = 0; k0 < cnt; k0 += 32) {
      const uint32_t k = k0 + lane;
      const unsigned active = __ballot_sync(0xFFFFFFFFu, k < cnt);
      if (k >= cnt) break;
      const uint32_t ty = ro.y + k / width, tx = ro.x + k % width;
      f((int)g, mt.base + ty * mt.stride + tx, active);
    }
  }
}

// Every (item, tile) pair adds one to its tile's counter (when the
// projection has not counted them itself, as for gs_bin_tiles).
__global__ void __launch_bounds__(kBinThreads) tile_count_kernel(const __grid_constant__ TileBinArgs a) {
  pdl_enter();
  for_each_pair<true>(a.n, a.rects, a.tiles, a.map, a.big_queue, a.big_len,
                       [&](int, uint32_t t, unsigned active) {
                         // (the checked build counts a tile beyond the grid into tile 0, reported)
                         warp_agg_inc(a.counts, in_bounds(t < (uint32_t)a.n_tiles) ? t : 0u, active);
                       });
}

// Length class of a tile list for the visit order, four per octave: 0 for
// an empty list, else 4 floor(log2 c) + (the two bits after c's leading one)
// + 1, so classes grow with the length and tiles within 19% of each other's
// length share one.  kLenClasses classes (kLenClasses is also the "no tile"
// sentinel; the raster passes' bucket-mode visit order uses the same classes).
__device__ __forceinline__ int length_class(uint32_t c) {
  if (!c) return 0;
  const int lead = 31 - __clz(c);
  const int frac = lead >= 2 ? (int)((c >> (lead - 2)) & 3u) : (int)((c << (2 - lead)) & 3u);
  return 4 * lead + frac + 1;
}

// offsets = exclusive scan of counts (clamped to 32 bits), cursors = offsets;
// stats[0] = total pairs, stats[1] = longest list; n_pairs = min(total, capacity).
// order (if non-null) = the tiles by descending length class, the order in
// which the raster passes visit them (longest lists first, so that the
// slowest tiles do not start last).
__global__ void __launch_bounds__(kScanThreads) tile_scan_kernel(int T, const uint32_t* __restrict__ counts,
                                                                 uint32_t* __restrict__ offsets,
                                                                 uint32_t* __restrict__ cursors, uint32_t capacity,
                                                                 uint32_t* __restrict__ n_pairs,
                                                                 unsigned long long* __restrict__ stats,
                                                                 uint32_t* __restrict__ order) {
  pdl_enter();
  __shared__ unsigned long long s[kScanThreads];
  __shared__ uint32_t s_max[32];
  const int per = (T + kScanThreads - 1) / kScanThreads;
  const int beg = min(T, (int)threadIdx.x * per), end = min(T, beg + per);
  unsigned long long sum = 0;
  uint32_t mx = 0;
  for (int i = beg; i < end; ++i) {
    const uint32_t c = counts[i];
    sum += c;
    mx = max(mx, c);
  }
  s[threadIdx.x] = sum;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) mx = max(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, off));
  if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = mx;
  __syncthreads();
  for (int off = 1; off < kScanThreads; off <<= 1) {
    const unsigned long long v = threadIdx.x >= (unsigned)off ? s[threadIdx.x - off] : 0ull;
    __syncthreads();
    s[threadIdx.x] += v;
    __syncthreads();
  }
  unsigned long long run = s[threadIdx.x] - sum;
  for (int i = beg; i < end; ++i) {
    const uint32_t o = (uint32_t)(run < 0xFFFFFFFFull ? run : 0xFFFFFFFFull);
    offsets[i] = o;
    cursors[i] = o;
    run += counts[i];
  }
  if (threadIdx.x == 0) {
    uint32_t m = 0;
    for (int k = 0; k < kScanThreads / 32; ++k) m = max(m, s_max[k]);
    const unsigned long long tot = s[kScanThreads - 1];
    stats[0] = tot;
    stats[1] = m;
    *n_pairs = (uint32_t)(tot < (unsigned long long)capacity ? tot : (unsigned long long)capacity);
  }
  if (!order) return;
  // counting sort of the tiles by length class, descending; lanes of a warp
  // with the same class are aggregated into one atomic
  __shared__ uint32_t s_cls[kLenClasses];
  const int lane = threadIdx.x & 31;
  if (threadIdx.x < kLenClasses) s_cls[threadIdx.x] = 0;
  __syncthreads();
  for (int i0 = 0; i0 < T; i0 += kScanThreads) {
    const int i = i0 + threadIdx.x;
    const int c = i < T ? length_class(counts[i]) : kLenClasses;
    const unsigned peers = __match_any_sync(0xFFFFFFFFu, c);
    if (c < kLenClasses && lane == __ffs(peers) - 1) atomicAdd(&s_cls[c], (uint32_t)__popc(peers));
  }
  __syncthreads();
  if (threadIdx.x < 32) class_starts_desc(s_cls);
  __syncthreads();
  for (int i0 = 0; i0 < T; i0 += kScanThreads) {
    const int i = i0 + threadIdx.x;
    const int c = i < T ? length_class(counts[i]) : kLenClasses;
    const unsigned peers = __match_any_sync(0xFFFFFFFFu, c);
    const int leader = __ffs(peers) - 1;
    uint32_t base = 0;
    if (c < kLenClasses && lane == leader) base = atomicAdd(&s_cls[c], (uint32_t)__popc(peers));
    base = __shfl_sync(peers, base, leader);
    if (c < kLenClasses) order[base + __popc(peers & ((1u << lane) - 1u))] = (uint32_t)i;
  }
}

// Multi-block form of tile_scan_kernel for many tiles (batches of views):
//   up:   block b sums the counts of its kScanTiles tiles, takes their
//         maximum and the histogram of their length classes;
//   mid:  one block: the total (stats, n_pairs), the longest list and the
//         start of each length class in the visit order (descending);
//   down: block b adds up the earlier blocks' sums and class histograms (in
//         block order) for its bases, then writes offsets, cursors and the
//         visit order of its tiles.
// aux per block: {sum lo, sum hi, max, hist[kLenClasses]}; aux_tail: class starts[kLenClasses].
constexpr int kScanTiles = 1024;
constexpr int kScanAux = 3 + kLenClasses;

__global__ void __launch_bounds__(256) tile_scan_up_kernel(int T, const uint32_t* __restrict__ counts,
                                                           uint32_t* __restrict__ aux) {
  pdl_enter();
  __shared__ uint32_t s_hist[kLenClasses];
  __shared__ unsigned long long s_sum[8];
  __shared__ uint32_t s_max[8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (threadIdx.x < kLenClasses) s_hist[threadIdx.x] = 0;
  __syncthreads();
  unsigned long long sum = 0;
  uint32_t mx = 0;
  const int i0 = blockIdx.x * kScanTiles;
#pragma unroll
  for (int j = 0; j < kScanTiles / 256; ++j) {
    const int i = i0 + j * 256 + threadIdx.x;
    const uint32_t c = i < T ? counts[i] : 0u;
    sum += c;
    mx = max(mx, c);
    const int cls = i < T ? length_class(c) : kLenClasses;
    const unsigned peers = __match_any_sync(0xFFFFFFFFu, cls);
    if (cls < kLenClasses && lane == __ffs(peers) - 1) atomicAdd(&s_hist[cls], (uint32_t)__popc(peers));
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    sum += __shfl_xor_sync(0xFFFFFFFFu, sum, off);
    mx = max(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, off));
  }
  if (lane == 0) {
    s_sum[wid] = sum;
    s_max[wid] = mx;
  }
  __syncthreads();
  uint32_t* out = aux + (size_t)kScanAux * blockIdx.x;
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    uint32_t m = 0;
    for (int w = 0; w < 8; ++w) {
      t += s_sum[w];
      m = max(m, s_max[w]);
    }
    out[0] = (uint32_t)t;
    out[1] = (uint32_t)(t >> 32);
    out[2] = m;
  }
  if (threadIdx.x < kLenClasses) out[3 + threadIdx.x] = s_hist[threadIdx.x];
}

__global__ void __launch_bounds__(64) tile_scan_mid_kernel(int nb, const uint32_t* __restrict__ aux,
                                                           uint32_t* __restrict__ aux_tail, uint32_t capacity,
                                                           uint32_t* __restrict__ n_pairs,
                                                           unsigned long long* __restrict__ stats) {
  pdl_enter();
  __shared__ uint32_t s_tot[kLenClasses];
  for (int c = threadIdx.x; c < kLenClasses; c += blockDim.x) {
    uint32_t t = 0;
    for (int b = 0; b < nb; ++b) t += aux[(size_t)kScanAux * b + 3 + c];
    s_tot[c] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long tot = 0;
    uint32_t m = 0;
    for (int b = 0; b < nb; ++b) {
      const uint32_t* a = aux + (size_t)kScanAux * b;
      tot += (unsigned long long)a[0] | ((unsigned long long)a[1] << 32);
      m = max(m, a[2]);
    }
    stats[0] = tot;
    stats[1] = m;
    *n_pairs = (uint32_t)(tot < (unsigned long long)capacity ? tot : (unsigned long long)capacity);
  }
  if (threadIdx.x < 32) {  // longest class first
    class_starts_desc(s_tot);
    __syncwarp();
    for (int c = threadIdx.x; c < kLenClasses; c += 32) aux_tail[c] = s_tot[c];
  }
}

__global__ void __launch_bounds__(256) tile_scan_down_kernel(int T, const uint32_t* __restrict__ counts,
                                                             const uint32_t* __restrict__ aux,
                                                             const uint32_t* __restrict__ aux_tail,
                                                             uint32_t* __restrict__ offsets,
                                                             uint32_t* __restrict__ cursors,
                                                             uint32_t* __restrict__ order) {
  pdl_enter();
  constexpr int PER = kScanTiles / 256;  // consecutive tiles per thread
  __shared__ unsigned long long s_scan[256];
  __shared__ unsigned long long s_base;
  __shared__ uint32_t s_cls[kLenClasses];
  const int b = blockIdx.x, lane = threadIdx.x & 31;
  static_assert(kLenClasses < 255, "thread 255 sums the bases");
  if (threadIdx.x < kLenClasses) {  // start of this block's tiles within each length class
    uint32_t o = aux_tail[threadIdx.x];
    for (int k = 0; k < b; ++k) o += aux[(size_t)kScanAux * k + 3 + threadIdx.x];
    s_cls[threadIdx.x] = o;
  } else if (threadIdx.x == 255) {
    unsigned long long o = 0;
    for (int k = 0; k < b; ++k) {
      const uint32_t* a = aux + (size_t)kScanAux * k;
      o += (unsigned long long)a[0] | ((unsigned long long)a[1] << 32);
    }
    s_base = o;
  }
  const int i0 = b * kScanTiles + threadIdx.x * PER;
  uint32_t c[PER];
  unsigned long long sum = 0;
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    c[j] = i0 + j < T ? counts[i0 + j] : 0u;
    sum += c[j];
  }
  s_scan[threadIdx.x] = sum;
  __syncthreads();
  for (int off = 1; off < 256; off <<= 1) {
    const unsigned long long v = threadIdx.x >= (unsigned)off ? s_scan[threadIdx.x - off] : 0ull;
    __syncthreads();
    s_scan[threadIdx.x] += v;
    __syncthreads();
  }
  unsigned long long run = s_base + s_scan[threadIdx.x] - sum;
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    if (i0 + j < T) {
      const uint32_t o = (uint32_t)(run < 0xFFFFFFFFull ? run : 0xFFFFFFFFull);
      offsets[i0 + j] = o;
      cursors[i0 + j] = o;
    }
    run += c[j];
  }
  if (!order) return;
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    const int i = i0 + j;
    const int cls = i < T ? length_class(c[j]) : kLenClasses;
    const unsigned peers = __match_any_sync(0xFFFFFFFFu, cls);
    const int leader = __ffs(peers) - 1;
    uint32_t base = 0;
    if (cls < kLenClasses && lane == leader) base = atomicAdd(&s_cls[cls], (uint32_t)__popc(peers));
    base = __shfl_sync(peers, base, leader);
    if (cls < kLenClasses) order[base + __popc(peers & ((1u << lane) - 1u))] = (uint32_t)i;
  }
}

__global__ void __launch_bounds__(kBinThreads) tile_scatter_kernel(const __grid_constant__ TileBinArgs a) {
  pdl_enter();
  bool over = false;
  for_each_pair(a.n, a.rects, a.tiles, a.map, a.big_queue, a.big_len,
                [&](int g, uint32_t t, unsigned active) {
                  const uint32_t pos = warp_agg_inc(a.cursors, in_bounds(t < (uint32_t)a.n_tiles) ? t : 0u, active);
                  if (pos < a.capacity)
                    a.ids[pos] = (uint32_t)g;
                  else
                    over = true;
                });
  if (over) atomicOr(a.overflow, 1u);
}

// Bitonic network over the 32 KEYS keys of one warp, sorted ascending.
// Blocked layout: lane l holds elements KEYS l .. KEYS l + KEYS - 1, so the
// compare-exchanges of partner distance j < KEYS stay inside a lane (no
// shuffle) and only the log2(32) largest distances of each merge level cross
// lanes.  Element e is the lower index of its pair when (e & j) == 0 and its
// block ascends when (e & k) == 0.
template <int KEYS>
__device__ __forceinline__ void warp_bitonic(unsigned long long (&x)[KEYS], int lane) {
  constexpr int M = 32 * KEYS;
#pragma unroll
  for (int k = 2; k <= M; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      if (j < KEYS) {
#pragma unroll
        for (int i = 0; i < KEYS; ++i) {
          if ((i & j) == 0) {
            const int p = i | j;
            // (e & k) for e = KEYS lane + i: i's bit when k < KEYS, else the lane's
            const bool up = k < KEYS ? ((i & k) == 0) : (((lane * KEYS) & k) == 0);
            const unsigned long long a = x[i], b = x[p];
            const bool sw = (a > b) == up;
            x[i] = sw ? b : a;
            x[p] = sw ? a : b;
          }
        }
      } else {
        const int d = j / KEYS;  // partner lane distance
        const bool keep_min = ((lane & d) == 0) == (((lane * KEYS) & k) == 0);
#pragma unroll
        for (int i = 0; i < KEYS; ++i) {
          const unsigned long long y = __shfl_xor_sync(0xFFFFFFFFu, x[i], d);
          x[i] = ((x[i] < y) == keep_min) ? x[i] : y;
        }
      }
    }
  }
}

// One warp sorts the list of n <= 32 KEYS ids at ids[off ..] by the key
// (depth bits << 32 | id), padded with all-ones keys to 32 KEYS.
template <int KEYS>
__device__ __forceinline__ void warp_sort_list(uint32_t* __restrict__ ids, const uint32_t* __restrict__ zkey,
                                               uint32_t off, uint32_t n, uint32_t n_items, int lane) {
  unsigned long long x[KEYS];
#pragma unroll
  for (int i = 0; i < KEYS; ++i) {
    const uint32_t e = (uint32_t)(lane * KEYS + i);
    x[i] = ~0ull;
    if (e < n) {
      const uint32_t g = ids[off + e];
      x[i] = in_bounds(g < n_items) ? ((unsigned long long)zkey[g] << 32) | g : ~0ull;
    }
  }
  warp_bitonic<KEYS>(x, lane);
#pragma unroll
  for (int i = 0; i < KEYS; ++i) {
    const uint32_t e = (uint32_t)(lane * KEYS + i);
    if (e < n) ids[off + e] = (uint32_t)x[i];
  }
}

// Per-tile sort of the lists by the 64-bit key (depth bits << 32 | id).  A
// CTA takes kSortWarps consecutive tiles, one warp each: lists of up to
// kWarpSortMax entries are sorted by that warp in registers (warp_bitonic,
// no barriers); longer ones (up to CAP) are queued in the CTA and then
// sorted one after the other by the whole CTA with a bitonic network in
// shared memory.  The last binning kernel: it also zeroes each tile's counter
// (and block 0 the large-splat queue length, and the two raster job counters
// when given), leaving them zero for the next passes.  In bucket mode each
// warp also files its tile under its length class (see TileBinArgs).
template <int CAP>
__global__ void __launch_bounds__(kSortThreads) tile_sort_kernel(const uint32_t* __restrict__ offsets,
                                                                 uint32_t* __restrict__ counts,
                                                                 uint32_t* __restrict__ ids,
                                                                 const uint32_t* __restrict__ zkey,
                                                                 uint2* __restrict__ ranges, uint32_t n_tiles,
                                                                 uint32_t capacity, uint32_t* __restrict__ overflow,
                                                                 uint32_t* __restrict__ big_len,
                                                                 uint32_t* __restrict__ raster_work,
                                                                 uint32_t n_items, uint32_t bucket_cap,
                                                                 uint32_t* __restrict__ cls_count,
                                                                 uint32_t* __restrict__ cls_tiles,
                                                                 uint32_t cls_stride) {
  pdl_enter();
  const bool buckets = cls_count != nullptr;  // the lists are per-tile buckets (see TileBinArgs)
  __shared__ unsigned long long s[CAP];
  __shared__ uint2 s_long[kSortWarps];  // (offset, length) of the CTA's lists longer than kWarpSortMax
  __shared__ uint32_t s_nlong;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    s_nlong = 0u;
    if (blockIdx.x == 0) {
      *big_len = 0u;
      if (raster_work) raster_work[0] = raster_work[1] = 0u;  // the raster passes' job counters
    }
  }
  __syncthreads();
  const uint32_t t = blockIdx.x * kSortWarps + warp;
  if (t < n_tiles) {
    uint32_t n = counts[t];
    const uint32_t off = buckets ? t * bucket_cap : offsets[t];
    __syncwarp();  // every lane has read counts[t]
    if (buckets && n > bucket_cap) n = bucket_cap;  // its bucket overflowed (flagged by the projection)
    const bool fits = buckets || (unsigned long long)off + n <= (unsigned long long)capacity;
    if (lane == 0) {
      counts[t] = 0u;
      if (buckets) {  // file the tile under its length class (empty ones too: their pixels are composited)
        const int c = length_class(n);
        cls_tiles[(size_t)c * cls_stride + atomicAdd(&cls_count[c], 1u)] = t;
      }
      uint2 rg = (n && fits) ? make_uint2(off, off + n) : make_uint2(0u, 0u);
      if (fits && n > (uint32_t)CAP) {
        atomicOr(overflow, 2u);
        rg = make_uint2(0u, 0u);
      } else if (fits && n > (uint32_t)kWarpSortMax) {
        s_long[atomicAdd(&s_nlong, 1u)] = make_uint2(off, n);
      }
      ranges[t] = rg;
    }
    if (fits && n > 1 && n <= (uint32_t)kWarpSortMax) {
      if (n <= 256) warp_sort_list<8>(ids, zkey, off, n, n_items, lane);
      else warp_sort_list<16>(ids, zkey, off, n, n_items, lane);
    }
  }
  __syncthreads();
  const uint32_t n_long = s_nlong;
  for (uint32_t q = 0; q < n_long; ++q) {
    const uint32_t off = s_long[q].x, n = s_long[q].y;
    uint32_t m = 2;
    while (m < n) m <<= 1;
    for (uint32_t i = threadIdx.x; i < m; i += kSortThreads) {
      unsigned long long key = ~0ull;
      if (i < n) {
        const uint32_t g = ids[off + i];
        key = in_bounds(g < n_items) ? ((unsigned long long)zkey[g] << 32) | g : ~0ull;
      }
      s[i] = key;
    }
    __syncthreads();
    for (uint32_t k = 2; k <= m; k <<= 1) {
      for (uint32_t j = k >> 1; j > 0; j >>= 1) {
        for (uint32_t i = threadIdx.x; i < m; i += kSortThreads) {
          const uint32_t ixj = i ^ j;
          if (ixj > i) {
            const unsigned long long a = s[i], b = s[ixj];
            const bool up = (i & k) == 0;
            if ((a > b) == up) {
              s[i] = b;
              s[ixj] = a;
            }
          }
        }
        __syncthreads();
      }
    }
    for (uint32_t i = threadIdx.x; i < n; i += kSortThreads) ids[off + i] = (uint32_t)s[i];
    __syncthreads();  // s is reused by the next long list
  }
}

int bin_grid(int n, int num_sms) {
  const int blocks = (n + kBinThreads - 1) / kBinThreads;
  return max(1, min(blocks, 16 * max(num_sms, 1)));
}

}  // namespace

int tile_sort_capacity() { return kTileSortCap; }

int64_t tile_scan_aux_size(int64_t n_tiles) { return (int64_t)kScanAux * ((n_tiles + kScanTiles - 1) / kScanTiles + 2); }

void launch_tile_count_scan(const TileBinArgs& a, cudaStream_t s, int64_t* launches) {
  if (!a.counted) {
    cudaMemsetAsync(a.counts, 0, sizeof(uint32_t) * (size_t)a.n_tiles, s);
    if (a.n > 0) {
      launch_pdl(tile_count_kernel, bin_grid(a.n, a.num_sms), kBinThreads, 0, s, a);
      if (launches) *launches += 1;
    }
  }
  if (a.n_tiles <= 4 * kScanThreads || !a.scan_aux) {  // one block is enough
    launch_pdl(tile_scan_kernel, 1, kScanThreads, 0, s, a.n_tiles, a.counts, a.offsets, a.cursors, a.capacity,
               a.n_pairs, a.stats, a.order);
    if (launches) *launches += 1;
  } else {
    const int nb = (a.n_tiles + kScanTiles - 1) / kScanTiles;
    uint32_t* tail = a.scan_aux + (size_t)kScanAux * nb;
    launch_pdl(tile_scan_up_kernel, nb, 256, 0, s, a.n_tiles, a.counts, a.scan_aux);
    launch_pdl(tile_scan_mid_kernel, 1, 64, 0, s, nb, a.scan_aux, tail, a.capacity, a.n_pairs, a.stats);
    launch_pdl(tile_scan_down_kernel, nb, 256, 0, s, a.n_tiles, a.counts, a.scan_aux, tail, a.offsets, a.cursors,
               a.order);
    if (launches) *launches += 3;
  }
}

void launch_tile_scatter(const TileBinArgs& a, cudaStream_t s, int64_t* launches) {
  if (a.n > 0) {
    launch_pdl(tile_scatter_kernel, bin_grid(a.n, a.num_sms), kBinThreads, 0, s, a);
    if (launches) *launches += 1;
  }
}

void launch_tile_sort(const TileBinArgs& a, cudaStream_t s, int64_t* launches) {
  const int grid = (a.n_tiles + kSortWarps - 1) / kSortWarps;
  const bool buckets = a.bucket_ids != nullptr;
  launch_pdl(tile_sort_kernel<kTileSortCap>, grid, kSortThreads, 0, s, a.offsets, a.counts,
             buckets ? a.bucket_ids : a.ids, a.zkey, a.ranges, (uint32_t)a.n_tiles, a.capacity, a.overflow,
             const_cast<uint32_t*>(a.big_len), a.raster_work, (uint32_t)a.n, a.bucket_cap,
             buckets ? a.cls_count : nullptr,
             a.cls_tiles, a.cls_stride);
  if (launches) *launches += 1;
}

cudaError_t tilebin_bind_bounds(uint32_t* word) { return bind_bounds_word(word); }

}  // namespace gs
