// Per-frame seeding of new Gaussians on the device (Sec. III-B.2, Eq. 10):
// the contrast quadtree over the RGB frame, then the back-projection of the
// leaf centres that the map does not cover yet.
//
// Quadtree, one level per launch: root cells of max_size px on a grid over
// the image (clipped at the border), then the children of the cells the
// previous level split.  A cell splits into its four (clipped, non-empty)
// quadrants when the mean over the channels of the variances of its pixels
// exceeds var_thr, its side exceeds min_size and it holds more than one
// pixel, and is a leaf otherwise.
//
// The per-channel sums of the values and their squares (double) come from a
// sum pyramid built bottom-up before the top-down pass: level l holds, for
// every aligned 2^l x 2^l cell (clipped at the border), the sums of its
// pixels, level 1 from the pixels and level l from the four cells of level
// l - 1.  Every level is one thread per cell, so the work is W H (1 + 1/4 +
// ...) double additions spread over the whole GPU instead of one pass over
// the pixels per quadtree level.  The top-down pass is one thread per cell;
// leaves and children are appended with one atomic per warp and list, and
// each level's grid is the largest number of cells the level can have, so no
// level needs a host round trip.
#include "common.cuh"
#include "internal.h"
#include "seed.cuh"

namespace gs {

namespace {

constexpr int kQtThreads = 256;

struct Sums {
  double s1[3], s2[3];
};

__device__ __forceinline__ void store_sums(double* __restrict__ out, const Sums& a) {
  double2* o = reinterpret_cast<double2*>(out);
  o[0] = make_double2(a.s1[0], a.s1[1]);
  o[1] = make_double2(a.s1[2], a.s2[0]);
  o[2] = make_double2(a.s2[1], a.s2[2]);
}

__device__ __forceinline__ void add_sums(const double* __restrict__ in, Sums& a) {
  const double2* q = reinterpret_cast<const double2*>(in);
  const double2 x = q[0], y = q[1], z = q[2];
  a.s1[0] += x.x;
  a.s1[1] += x.y;
  a.s1[2] += y.x;
  a.s2[0] += y.y;
  a.s2[1] += z.x;
  a.s2[2] += z.y;
}

// level 1: the 2 x 2 cells' sums from the pixels
__global__ void __launch_bounds__(kQtThreads) qt_pyr_base_kernel(const float* __restrict__ rgb, int W, int H,
                                                                 int W1, int H1, double* __restrict__ out) {
  const int64_t c = blockIdx.x * (int64_t)kQtThreads + threadIdx.x;
  if (c >= (int64_t)W1 * H1) return;
  const int i = (int)(c % W1), j = (int)(c / W1);
  const size_t HW = (size_t)W * H;
  Sums a = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};
#pragma unroll
  for (int d = 0; d < 4; ++d) {
    const int x = 2 * i + (d & 1), y = 2 * j + (d >> 1);
    if (x < W && y < H) {
      const size_t p = (size_t)y * W + x;
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) {
        const double v = (double)rgb[ch * HW + p];
        a.s1[ch] += v;
        a.s2[ch] = fma(v, v, a.s2[ch]);
      }
    }
  }
  store_sums(out + 6 * c, a);
}

// level l from level l - 1 (Wp x Hp cells)
__global__ void __launch_bounds__(kQtThreads) qt_pyr_up_kernel(const double* __restrict__ in, int Wp, int Hp,
                                                               int Wl, int Hl, double* __restrict__ out) {
  const int64_t c = blockIdx.x * (int64_t)kQtThreads + threadIdx.x;
  if (c >= (int64_t)Wl * Hl) return;
  const int i = (int)(c % Wl), j = (int)(c / Wl);
  Sums a = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};
#pragma unroll
  for (int d = 0; d < 4; ++d) {
    const int x = 2 * i + (d & 1), y = 2 * j + (d >> 1);
    if (x < Wp && y < Hp) add_sums(in + 6 * ((size_t)y * Wp + x), a);
  }
  store_sums(out + 6 * c, a);
}

// top-down level: cell w is root cell w of the grid (root) or cells_in[w];
// sums: the pyramid level of this cell size (Wl cells per row), unused when
// no cell of the level can split
__global__ void __launch_bounds__(kQtThreads) qt_level_kernel(
    const double* __restrict__ sums, int Wl, int W, int H, int size, int min_size, double var_thr, bool root,
    int grid_x, uint32_t n_root, const int2* __restrict__ cells_in, const uint32_t* __restrict__ n_in,
    int2* __restrict__ cells_out, uint32_t* __restrict__ n_out, int4* __restrict__ leaves,
    uint32_t* __restrict__ n_leaves) {
  const int lane = threadIdx.x & 31;
  const uint32_t w = blockIdx.x * kQtThreads + threadIdx.x;
  const uint32_t n = root ? n_root : *n_in;
  if (w - lane >= n) return;  // whole warps only: the warp collectives below name all 32 lanes
  const bool live = w < n;
  int2 cell = make_int2(0, 0);
  if (live)
    cell = root ? make_int2((int)(w % (uint32_t)grid_x) * size, (int)(w / (uint32_t)grid_x) * size) : cells_in[w];
  const int x0 = cell.x, y0 = cell.y;
  const int x1 = min(x0 + size, W), y1 = min(y0 + size, H);
  const int cw = x1 - x0, area = cw * (y1 - y0);
  bool split = false;
  if (live && size > min_size && area > 1) {
    Sums a = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};
    add_sums(sums + 6 * ((size_t)(y0 / size) * Wl + x0 / size), a);
    // mean over the channels of the variances, compared without a division:
    // sum_c max(A s2_c - s1_c^2, 0) > 3 var_thr A^2
    const double A = (double)area;
    double d = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) d += fmax(A * a.s2[c] - a.s1[c] * a.s1[c], 0.0);
    split = d > 3.0 * var_thr * A * A;
  }
  // leaves: one atomic per warp
  const bool is_leaf = live && !split;
  const unsigned lb = __ballot_sync(0xFFFFFFFFu, is_leaf);
  if (lb) {
    const int src = __ffs(lb) - 1;
    uint32_t base = 0;
    if (lane == src) base = atomicAdd(n_leaves, (uint32_t)__popc(lb));
    base = __shfl_sync(0xFFFFFFFFu, base, src);
    if (is_leaf) leaves[base + __popc(lb & ((1u << lane) - 1u))] = make_int4(x0, y0, cw, y1 - y0);
  }
  // children (the quadrants that are not clipped away): a warp scan of the
  // counts, one atomic per warp
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
  bool seeds = false;
  int4 L = make_int4(0, 0, 1, 1);
  float ux = 0.f, uy = 0.f, z = 0.f;
  size_t pix = 0;
  if (i < n_leaves) {
    L = leaves[i];
    pix = leaf_pixel(a, L, &ux, &uy);
    z = a.depth[pix];
    seeds = z > 0.f && !(a.alpha && !(a.alpha[pix] < a.alpha_thr));
  }
  const unsigned m = __ballot_sync(0xFFFFFFFFu, seeds);
  if (!seeds) return;
  const uint32_t k = warp_agg_inc(n_seeded, 0u, m);  // one atomic per warp
  if (k >= a.capacity) return;
  float p[3];
  leaf_point(a, ux, uy, z, p);
  write_seed(a, k, L, pix, p, z);
}

}  // namespace

int64_t quadtree_scratch_cells(int W, int H) { return (int64_t)W * H + 4; }

// doubles of the sum pyramid for cells of 2 .. max_size px
int64_t quadtree_pyramid_doubles(int W, int H, int max_size) {
  int64_t n = 0;
  for (int l = 1, sz = 2; sz <= max_size; ++l, sz *= 2)
    n += 6 * (int64_t)((W + sz - 1) / sz) * ((H + sz - 1) / sz);
  return n;
}

int launch_quadtree(const float* rgb, int W, int H, int max_size, int min_size, double var_thr, int2* cells_a,
                    int2* cells_b, uint32_t* counters, int4* leaves, double* pyramid, cudaStream_t s) {
  // counters: [0] leaves, [1 + level] cells of the next level
  int levels = 0;
  for (int sz = max_size; sz >= min_size && sz >= 1; sz /= 2) ++levels;
  int launches = 0;
  cudaMemsetAsync(counters, 0, sizeof(uint32_t) * (size_t)(levels + 2), s);
  // sum pyramid up to the largest cell size that can split (sizes > min_size)
  const double* level_sums[13] = {nullptr};
  int level_w[13] = {0};
  double* at = pyramid;
  int Wp = W, Hp = H;
  // (levels 1 .. log2(max_size); none when no cell can split)
  for (int l = 1, sz = 2; max_size > min_size && sz <= max_size && l < 13; ++l, sz *= 2) {
    const int Wl = (W + sz - 1) / sz, Hl = (H + sz - 1) / sz;
    const int64_t cells = (int64_t)Wl * Hl;
    const unsigned blocks = (unsigned)((cells + kQtThreads - 1) / kQtThreads);
    if (l == 1)
      qt_pyr_base_kernel<<<blocks, kQtThreads, 0, s>>>(rgb, W, H, Wl, Hl, at);
    else
      qt_pyr_up_kernel<<<blocks, kQtThreads, 0, s>>>(level_sums[l - 1], Wp, Hp, Wl, Hl, at);
    ++launches;
    level_sums[l] = at;
    level_w[l] = Wl;
    at += 6 * cells;
    Wp = Wl;
    Hp = Hl;
  }
  int2* in = cells_b;
  int2* out = cells_a;
  int size = max_size;
  for (int l = 0; l < levels; ++l, size /= 2) {
    const int gx = (W + size - 1) / size, gy = (H + size - 1) / size;
    const int64_t max_cells = (int64_t)gx * gy;
    int lv = 0;
    while ((1 << lv) < size) ++lv;
    const double* sums = size > min_size ? level_sums[lv] : nullptr;
    const int blocks = (int)((max_cells + kQtThreads - 1) / kQtThreads);
    qt_level_kernel<<<blocks, kQtThreads, 0, s>>>(sums, level_w[lv], W, H, size, min_size, var_thr, l == 0, gx,
                                                  (uint32_t)max_cells, in, counters + l, out, counters + 1 + l,
                                                  leaves, counters);
    ++launches;
    int2* tmp = in;
    in = out;
    out = tmp;
  }
  return launches;
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
