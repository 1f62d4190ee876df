// Per-frame seeding of new Gaussians on the device (Sec. III-B.2, Eq. 10):
// the contrast quadtree over the RGB frame, then the back-projection of the
// leaf centres that the map does not cover yet.
//
// Quadtree, one level per launch: root cells of max_size px on a grid over
// the image (clipped at the border), then the children of the cells the
// previous level split.  A group of L lanes (L = 32 for cells of 8 px and up,
// 16 / 4 for 4 / 2 px cells, 1 where no cell can split) takes one cell, sums
// its pixels' values and squares per channel in double and reduces them over
// the group; the cell splits into its four (clipped, non-empty) quadrants
// when the mean over the channels of the variances exceeds var_thr, its side
// exceeds min_size and it holds more than one pixel, and is a leaf otherwise.
// The cell and leaf lists grow through device counters with one atomic per
// warp and list, and each level's grid is the largest number of cells the
// level can have, so no level needs a host round trip.
#include "internal.h"
#include "seed.cuh"

namespace gs {

namespace {

constexpr int kQtWarps = 8;  // warps per CTA

// level 0: cell w is root cell w of the grid; later levels: cells_in[w]
template <int L>
__global__ void __launch_bounds__(32 * kQtWarps) qt_level_kernel(
    const float* __restrict__ rgb, int W, int H, int size, int min_size, double var_thr, bool root, int grid_x,
    uint32_t n_root, const int2* __restrict__ cells_in, const uint32_t* __restrict__ n_in,
    int2* __restrict__ cells_out, uint32_t* __restrict__ n_out, int4* __restrict__ leaves,
    uint32_t* __restrict__ n_leaves) {
  constexpr int kCells = 32 / L;  // cells per warp
  const int lane = threadIdx.x & 31, sub = lane % L;
  const uint32_t first = (blockIdx.x * kQtWarps + (threadIdx.x >> 5)) * kCells;
  const uint32_t n = root ? n_root : *n_in;
  if (first >= n) return;  // whole warps only: the shuffles below name all 32 lanes
  const uint32_t w = first + lane / L;
  const bool live = w < n;
  int2 cell = make_int2(0, 0);
  if (live)
    cell = root ? make_int2((int)(w % (uint32_t)grid_x) * size, (int)(w / (uint32_t)grid_x) * size) : cells_in[w];
  const int x0 = cell.x, y0 = cell.y;
  const int x1 = min(x0 + size, W), y1 = min(y0 + size, H);
  const int cw = x1 - x0, area = live ? cw * (y1 - y0) : 0;
  const bool may_split = size > min_size && area > 1;
  double s1[3] = {0.0, 0.0, 0.0}, s2[3] = {0.0, 0.0, 0.0};
  if (may_split) {
    const size_t HW = (size_t)W * H;
    for (int p = sub; p < area; p += L) {
      const size_t pix = (size_t)(y0 + p / cw) * W + x0 + p % cw;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const double x = (double)rgb[c * HW + pix];
        s1[c] += x;
        s2[c] = fma(x, x, s2[c]);
      }
    }
  }
  if (L > 1 && size > min_size) {  // uniform over the launch
#pragma unroll
    for (int off = L / 2; off > 0; off >>= 1)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        s1[c] += __shfl_xor_sync(0xFFFFFFFFu, s1[c], off);
        s2[c] += __shfl_xor_sync(0xFFFFFFFFu, s2[c], off);
      }
  }
  const bool leader = live && sub == 0;
  bool split = false;
  if (leader && may_split) {
    double var = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double m1 = s1[c] / area, m2 = s2[c] / area;
      var += fmax(m2 - m1 * m1, 0.0);
    }
    split = var / 3.0 > var_thr;
  }
  // leaves: one atomic per warp
  const bool is_leaf = leader && !split;
  const unsigned lb = __ballot_sync(0xFFFFFFFFu, is_leaf);
  if (lb) {
    const int src = __ffs(lb) - 1;
    uint32_t base = 0;
    if (lane == src) base = atomicAdd(n_leaves, (uint32_t)__popc(lb));
    base = __shfl_sync(0xFFFFFFFFu, base, src);
    if (is_leaf) leaves[base + __popc(lb & ((1u << lane) - 1u))] = make_int4(x0, y0, cw, y1 - y0);
  }
  // children: a warp scan of the counts, one atomic per warp
  // the quadrants that are not clipped away: (0, 0) always, the right ones
  // if x0 + half < W, the lower ones if y0 + half < H
  const int half = size / 2;
  const bool right = x0 + half < W, lower = y0 + half < H;
  const int nc = split ? (1 + right) * (1 + lower) : 0;
  if (__ballot_sync(0xFFFFFFFFu, nc > 0)) {
    int incl = nc;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int v = __shfl_up_sync(0xFFFFFFFFu, incl, off);
      if (lane >= off) incl += v;
    }
    uint32_t base = 0;
    if (lane == 31) base = atomicAdd(n_out, (uint32_t)incl);
    base = __shfl_sync(0xFFFFFFFFu, base, 31);
    if (split) {
      int2* o = cells_out + base + (uint32_t)(incl - nc);
      *o++ = make_int2(x0, y0);
      if (right) *o++ = make_int2(x0 + half, y0);
      if (lower) *o++ = make_int2(x0, y0 + half);
      if (right && lower) *o = make_int2(x0 + half, y0 + half);
    }
  }
}

// Eq. 10 for every leaf with valid depth (and alpha below the threshold):
// one thread per leaf, the seeded ones compacted through a counter
__global__ void __launch_bounds__(256) qt_seed_kernel(const __grid_constant__ SeedArgs a,
                                                      const int4* __restrict__ leaves, uint32_t n_leaves,
                                                      uint32_t* __restrict__ n_seeded) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_leaves) return;
  const int4 L = leaves[i];
  float ux, uy;
  const size_t pix = leaf_pixel(a, L, &ux, &uy);
  const float z = a.depth[pix];
  if (!(z > 0.f)) return;
  if (a.alpha && !(a.alpha[pix] < a.alpha_thr)) return;
  const uint32_t k = atomicAdd(n_seeded, 1u);
  if (k >= a.capacity) return;
  float p[3];
  leaf_point(a, ux, uy, z, p);
  write_seed(a, k, L, pix, p, z);
}

}  // namespace

int64_t quadtree_scratch_cells(int W, int H) { return (int64_t)W * H + 4; }

int launch_quadtree(const float* rgb, int W, int H, int max_size, int min_size, double var_thr, int2* cells_a,
                    int2* cells_b, uint32_t* counters, int4* leaves, cudaStream_t s) {
  // counters: [0] leaves, [1 + level] cells of the next level
  int levels = 0;
  for (int sz = max_size; sz >= min_size && sz >= 1; sz /= 2) ++levels;
  cudaMemsetAsync(counters, 0, sizeof(uint32_t) * (size_t)(levels + 2), s);
  int2* in = cells_b;
  int2* out = cells_a;
  int size = max_size;
  for (int l = 0; l < levels; ++l, size /= 2) {
    const int gx = (W + size - 1) / size, gy = (H + size - 1) / size;
    const int64_t max_cells = (int64_t)gx * gy;
    // lanes per cell: enough for the cell's pixels, 1 where nothing is summed
    const int lanes = size <= min_size ? 1 : size >= 8 ? 32 : size * size;
    const int64_t per_block = (int64_t)kQtWarps * (32 / lanes);
    const int blocks = (int)((max_cells + per_block - 1) / per_block);
    const uint32_t n_root = (uint32_t)max_cells;
    auto* k = lanes == 32 ? qt_level_kernel<32> : lanes == 16 ? qt_level_kernel<16> : lanes == 4 ? qt_level_kernel<4>
                                                                                                 : qt_level_kernel<1>;
    k<<<blocks, 32 * kQtWarps, 0, s>>>(rgb, W, H, size, min_size, var_thr, l == 0, gx, n_root, in, counters + l, out,
                                       counters + 1 + l, leaves, counters);
    int2* tmp = in;
    in = out;
    out = tmp;
  }
  return levels;
}

void launch_seed(const float* rgb, const float* depth, const float* alpha, float alpha_thr, int W, int H,
                 const float K4[4], const float R[9], const float t[3], int sh_degree, const int4* leaves,
                 uint32_t n_leaves, float* means, float* log_scales, float* quats, float* logits, float* sh,
                 uint32_t capacity, uint32_t* n_seeded, cudaStream_t s) {
  cudaMemsetAsync(n_seeded, 0, sizeof(uint32_t), s);
  if (n_leaves == 0) return;
  const SeedArgs a = make_seed_args(rgb, depth, alpha, alpha_thr, W, H, K4, R, t, sh_degree, means, log_scales,
                                    quats, logits, sh, capacity);
  qt_seed_kernel<<<(n_leaves + 255) / 256, 256, 0, s>>>(a, leaves, n_leaves, n_seeded);
}

}  // namespace gs
