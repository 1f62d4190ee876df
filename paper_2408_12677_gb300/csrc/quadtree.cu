// Per-frame seeding of new Gaussians on the device (Sec. III-B.2, Eq. 10):
// the contrast quadtree over the RGB frame, then the back-projection of the
// leaf centres that the map does not cover yet.
//
// Quadtree, one level per launch: root cells of max_size px on a grid over
// the image (clipped at the border), then the children of the cells the
// previous level split.  One warp per cell sums its pixels' values and
// squares per channel in double; the cell splits into its four (clipped,
// non-empty) quadrants when the mean over the channels of the variances
// exceeds var_thr, its side exceeds min_size and it holds more than one
// pixel, and is a leaf otherwise.  The cell and leaf lists grow through
// device counters, and each level's grid is the largest number of cells the
// level can have, so no level needs a host round trip.
#include "internal.h"

namespace gs {

namespace {

constexpr int kQtWarps = 8;  // warps (cells) per CTA

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, off);
  return v;
}

// level 0: cell w is root cell w of the grid; later levels: cells_in[w]
__global__ void __launch_bounds__(32 * kQtWarps) qt_level_kernel(
    const float* __restrict__ rgb, int W, int H, int size, int min_size, double var_thr, bool root, int grid_x,
    const int2* __restrict__ cells_in, const uint32_t* __restrict__ n_in, int2* __restrict__ cells_out,
    uint32_t* __restrict__ n_out, int4* __restrict__ leaves, uint32_t* __restrict__ n_leaves) {
  const uint32_t w = blockIdx.x * kQtWarps + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  int2 cell;
  if (root) {
    if (w >= (uint32_t)grid_x * (uint32_t)((H + size - 1) / size)) return;
    cell = make_int2((int)(w % (uint32_t)grid_x) * size, (int)(w / (uint32_t)grid_x) * size);
  } else {
    if (w >= *n_in) return;
    cell = cells_in[w];
  }
  const int x0 = cell.x, y0 = cell.y;
  const int x1 = min(x0 + size, W), y1 = min(y0 + size, H);
  const int cw = x1 - x0, area = cw * (y1 - y0);
  const size_t HW = (size_t)W * H;
  double s1[3] = {0.0, 0.0, 0.0}, s2[3] = {0.0, 0.0, 0.0};
  for (int p = lane; p < area; p += 32) {
    const size_t pix = (size_t)(y0 + p / cw) * W + x0 + p % cw;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double x = (double)rgb[c * HW + pix];
      s1[c] += x;
      s2[c] = fma(x, x, s2[c]);
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    s1[c] = warp_sum_d(s1[c]);
    s2[c] = warp_sum_d(s2[c]);
  }
  if (lane != 0) return;
  double var = 0.0;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double m1 = s1[c] / area, m2 = s2[c] / area;
    var += fmax(m2 - m1 * m1, 0.0);
  }
  var /= 3.0;
  if (size > min_size && area > 1 && var > var_thr) {
    const int half = size / 2;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int cx = x0 + (q & 1) * half, cy = y0 + (q >> 1) * half;
      if (cx < W && cy < H) cells_out[atomicAdd(n_out, 1u)] = make_int2(cx, cy);
    }
  } else {
    leaves[atomicAdd(n_leaves, 1u)] = make_int4(x0, y0, cw, y1 - y0);
  }
}

struct SeedArgs {
  const float *rgb, *depth, *alpha;
  float alpha_thr;
  int W, H;
  double fx, fy, cx, cy;
  double R[9], t[3];
  int sh_degree;
  float *means, *log_scales, *quats, *logits, *sh;
  uint32_t capacity;
};

// Eq. 10 for every leaf with valid depth (and alpha below the threshold):
// one thread per leaf, the seeded ones compacted through a counter
__global__ void __launch_bounds__(256) qt_seed_kernel(const __grid_constant__ SeedArgs a,
                                                      const int4* __restrict__ leaves, uint32_t n_leaves,
                                                      uint32_t* __restrict__ n_seeded) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_leaves) return;
  const int4 L = leaves[i];
  const double ux = L.x + 0.5 * L.z, uy = L.y + 0.5 * L.w;
  const int pi = min((int)floor(ux), a.W - 1), pj = min((int)floor(uy), a.H - 1);
  const size_t pix = (size_t)pj * a.W + pi;
  const float z = a.depth[pix];
  if (!(z > 0.f)) return;
  if (a.alpha && !(a.alpha[pix] < a.alpha_thr)) return;
  const uint32_t k = atomicAdd(n_seeded, 1u);
  if (k >= a.capacity) return;
  const double zd = (double)z;
  const double pc[3] = {(ux - a.cx) * zd / a.fx, (uy - a.cy) * zd / a.fy, zd};
  const double q[3] = {pc[0] - a.t[0], pc[1] - a.t[1], pc[2] - a.t[2]};
#pragma unroll
  for (int c = 0; c < 3; ++c)
    a.means[3 * (size_t)k + c] = (float)(a.R[c] * q[0] + a.R[3 + c] * q[1] + a.R[6 + c] * q[2]);  // R^T q
  const float ls = (float)log(0.5 * hypot((double)L.z, (double)L.w) * zd / a.fx);
#pragma unroll
  for (int c = 0; c < 3; ++c) a.log_scales[3 * (size_t)k + c] = ls;
  a.quats[4 * (size_t)k] = 1.f;
  a.quats[4 * (size_t)k + 1] = 0.f;
  a.quats[4 * (size_t)k + 2] = 0.f;
  a.quats[4 * (size_t)k + 3] = 0.f;
  a.logits[k] = 0.f;
  const int K = (a.sh_degree + 1) * (a.sh_degree + 1);
  float* sh = a.sh + (size_t)k * 3 * K;
  const size_t HW = (size_t)a.W * a.H;
  constexpr double kInvY00 = 3.5449077018110318;  // 1 / Y_00 = 2 sqrt(pi)
#pragma unroll
  for (int c = 0; c < 3; ++c) sh[c] = (float)(((double)a.rgb[c * HW + pix] - 0.5) * kInvY00);
  for (int e = 3; e < 3 * K; ++e) sh[e] = 0.f;
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
    const int blocks = (int)((max_cells + kQtWarps - 1) / kQtWarps);
    qt_level_kernel<<<blocks, 32 * kQtWarps, 0, s>>>(rgb, W, H, size, min_size, var_thr, l == 0, gx, in,
                                                     counters + l, out, counters + 1 + l, leaves, counters);
    int2* tmp = in;
    in = out;
    out = tmp;
  }
  return levels;
}

void launch_seed(const float* rgb, const float* depth, const float* alpha, float alpha_thr, int W, int H,
                 const double K4[4], const double R[9], const double t[3], int sh_degree, const int4* leaves,
                 uint32_t n_leaves, float* means, float* log_scales, float* quats, float* logits, float* sh,
                 uint32_t capacity, uint32_t* n_seeded, cudaStream_t s) {
  cudaMemsetAsync(n_seeded, 0, sizeof(uint32_t), s);
  if (n_leaves == 0) return;
  SeedArgs a;
  a.rgb = rgb;
  a.depth = depth;
  a.alpha = alpha;
  a.alpha_thr = alpha_thr;
  a.W = W;
  a.H = H;
  a.fx = K4[0];
  a.fy = K4[1];
  a.cx = K4[2];
  a.cy = K4[3];
  for (int k = 0; k < 9; ++k) a.R[k] = R[k];
  for (int k = 0; k < 3; ++k) a.t[k] = t[k];
  a.sh_degree = sh_degree;
  a.means = means;
  a.log_scales = log_scales;
  a.quats = quats;
  a.logits = logits;
  a.sh = sh;
  a.capacity = capacity;
  qt_seed_kernel<<<(n_leaves + 255) / 256, 256, 0, s>>>(a, leaves, n_leaves, n_seeded);
}

}  // namespace gs
