// L1 photometric + depth loss with image gradients (Eq. 12 plus a depth
// term), the dense Adam update over the flat parameter buffer, and small
// export helpers.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace gs {

namespace {

constexpr int kLossThreads = 256;
constexpr int kLossItems = 8;  // pixels per thread

__device__ __forceinline__ float sgn(float x) { return (float)((x > 0.f) - (x < 0.f)); }

// Block b of a batched launch belongs to the view v with
// block_base[v] <= b < block_base[v + 1] and covers that view's pixels
// [(b - block_base[v]) * kLossThreads * kLossItems, ...).
__device__ __forceinline__ int loss_view_of(const LossArgs& a, int b) {
  int v = 0;
  for (int k = 1; k < a.views; ++k)
    if (b >= a.v[k].block_base) v = k;
  return v;
}

// Pass 1: per pixel |residuals| and sign gradients; per-block partial sums
// (|colour residual| sum, |depth residual| sum over valid pixels, valid count).
__global__ void __launch_bounds__(kLossThreads) loss_partials_kernel(const __grid_constant__ LossArgs a,
                                                                     float* __restrict__ partials) {
  const LossView& lv = a.v[loss_view_of(a, blockIdx.x)];
  const int npix = lv.npix;
  const float* __restrict__ color = lv.color;
  const float* __restrict__ depth = lv.depth;
  const float* __restrict__ trgb = lv.trgb;
  const float* __restrict__ tdep = lv.tdep;
  float* __restrict__ dLdc = lv.dLdc;
  float* __restrict__ dLdd = lv.dLdd;
  const float gscale_c = a.w_color / (3.f * (float)npix);
  float sc = 0.f, sd = 0.f, nv = 0.f;
  const int base = (blockIdx.x - lv.block_base) * kLossThreads * kLossItems + threadIdx.x;
#pragma unroll
  for (int j = 0; j < kLossItems; ++j) {
    const int p = base + j * kLossThreads;
    if (p >= npix) break;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float r = color[(size_t)c * npix + p] - trgb[(size_t)c * npix + p];
      sc += fabsf(r);
      dLdc[(size_t)c * npix + p] = gscale_c * sgn(r);
    }
    const float td = tdep[p];
    const bool valid = td > 0.f;
    const float rd = depth[p] - td;
    sd += valid ? fabsf(rd) : 0.f;
    nv += valid ? 1.f : 0.f;
    dLdd[p] = valid ? sgn(rd) : 0.f;
  }
  __shared__ float red[3][kLossThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int off = 16; off > 0; off >>= 1) {
    sc += __shfl_xor_sync(0xFFFFFFFFu, sc, off);
    sd += __shfl_xor_sync(0xFFFFFFFFu, sd, off);
    nv += __shfl_xor_sync(0xFFFFFFFFu, nv, off);
  }
  if (lane == 0) {
    red[0][wid] = sc;
    red[1][wid] = sd;
    red[2][wid] = nv;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    float s = 0.f;
    for (int w = 0; w < kLossThreads / 32; ++w) s += red[threadIdx.x][w];
    partials[3 * blockIdx.x + threadIdx.x] = s;
  }
}

// Pass 2 (one block of 256): per view, a fixed-order reduction of its
// partials -> L_v and the depth-gradient scale w_depth / n_valid (scale[v]);
// loss = sum of L_v in view order.  Each thread sums a strided subset in
// order, then a fixed tree combines them, so the result does not depend on
// scheduling.
// The finalize step by one block of 256 threads (every thread calls it).
__device__ __forceinline__ void loss_finalize_block(const LossArgs& a, const float* __restrict__ partials,
                                                    float* __restrict__ scale) {
  __shared__ float red[3][256];
  float total = 0.f;
  for (int v = 0; v < a.views; ++v) {
    const int b0 = a.v[v].block_base;
    const int b1 = v + 1 < a.views ? a.v[v + 1].block_base : a.n_blocks;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f;
    for (int b = b0 + threadIdx.x; b < b1; b += 256) {
      a0 += partials[3 * b];
      a1 += partials[3 * b + 1];
      a2 += partials[3 * b + 2];
    }
    __syncthreads();  // previous view done with red
    red[0][threadIdx.x] = a0;
    red[1][threadIdx.x] = a1;
    red[2][threadIdx.x] = a2;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
      if ((int)threadIdx.x < s) {
        red[0][threadIdx.x] += red[0][threadIdx.x + s];
        red[1][threadIdx.x] += red[1][threadIdx.x + s];
        red[2][threadIdx.x] += red[2][threadIdx.x + s];
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      const float nv = red[2][0] > 0.f ? red[2][0] : 1.f;
      total += a.w_color * red[0][0] / (3.f * (float)a.v[v].npix) + a.w_depth * red[1][0] / nv;
      scale[v] = a.w_depth / nv;
    }
  }
  if (threadIdx.x == 0) a.loss[0] = total;
}

__global__ void __launch_bounds__(256) loss_finalize_kernel(const __grid_constant__ LossArgs a,
                                                            const float* __restrict__ partials,
                                                            float* __restrict__ scale) {
  loss_finalize_block(a, partials, scale);
}

// Pass 3: dL/dD = scale[v] * sign, same block layout as pass 1
__global__ void __launch_bounds__(kLossThreads) scale_kernel(const __grid_constant__ LossArgs a,
                                                             const float* __restrict__ scale) {
  const int v = loss_view_of(a, blockIdx.x);
  const LossView& lv = a.v[v];
  const float sv = scale[v];
  float* __restrict__ dLdd = lv.dLdd;
  const int base = (blockIdx.x - lv.block_base) * kLossThreads * kLossItems + threadIdx.x;
#pragma unroll
  for (int j = 0; j < kLossItems; ++j) {
    const int p = base + j * kLossThreads;
    if (p >= lv.npix) break;
    dLdd[p] *= sv;
  }
}

// Loss of the fused forward pass, phase 1: block b sums, in a fixed order,
// the (tile, 8 x 8 block) partials [lo, lo + kTileLossChunk) of one view
// into partials[3 b ..] (the layout of loss_partials_kernel's output, so
// loss_finalize_kernel finishes the job).  View v owns blocks
// [block_base[v], block_base[v + 1]) and job partials [4 tile_base[v], 4 tile_base[v + 1]).
constexpr int kTileLossChunk = kLossThreads * kLossItems;

struct TileLossArgs {
  int views;
  int block_base[kMaxViews + 1];
  uint32_t job_base[kMaxViews + 1];
  const float* jobs;
};

// One launch: every block sums its chunk of the per-(tile, block) partials;
// the last block to finish (a ticket counter, reset by that block) then
// finalises the loss and the depth scales over all blocks' partials in block
// order (so the result does not depend on which block is last), and, given
// `step`, advances the device Adam step counter of the training step.
static_assert(kLossThreads == 256, "the finalize step is written for 256 threads");
__global__ void __launch_bounds__(kLossThreads) loss_tiles_kernel(const __grid_constant__ TileLossArgs t,
                                                                  const __grid_constant__ LossArgs la,
                                                                  float* __restrict__ partials,
                                                                  float* __restrict__ scale,
                                                                  uint32_t* __restrict__ ticket,
                                                                  long long* __restrict__ step) {
  pdl_enter();
  int v = 0;
  for (int k = 1; k < t.views; ++k)
    if ((int)blockIdx.x >= t.block_base[k]) v = k;
  const uint32_t lo = t.job_base[v] + (uint32_t)(blockIdx.x - t.block_base[v]) * kTileLossChunk;
  const uint32_t hi = min(lo + (uint32_t)kTileLossChunk, t.job_base[v + 1]);
  float sc = 0.f, sd = 0.f, nv = 0.f;
#pragma unroll
  for (int j = 0; j < kLossItems; ++j) {
    const uint32_t i = lo + threadIdx.x + j * kLossThreads;
    if (i < hi) {
      sc += t.jobs[3 * (size_t)i];
      sd += t.jobs[3 * (size_t)i + 1];
      nv += t.jobs[3 * (size_t)i + 2];
    }
  }
  __shared__ float red[3][kLossThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int off = 16; off > 0; off >>= 1) {
    sc += __shfl_xor_sync(0xFFFFFFFFu, sc, off);
    sd += __shfl_xor_sync(0xFFFFFFFFu, sd, off);
    nv += __shfl_xor_sync(0xFFFFFFFFu, nv, off);
  }
  if (lane == 0) {
    red[0][wid] = sc;
    red[1][wid] = sd;
    red[2][wid] = nv;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    float s = 0.f;
    for (int w = 0; w < kLossThreads / 32; ++w) s += red[threadIdx.x][w];
    partials[3 * blockIdx.x + threadIdx.x] = s;
  }
  __shared__ bool s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();  // this block's partials are visible before its ticket
    s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  loss_finalize_block(la, partials, scale);
  if (threadIdx.x == 0) {
    *ticket = 0u;
    if (step) *step += 1;
  }
}

// ---------------------------------------------------------------------------
// Adam
// ---------------------------------------------------------------------------
struct AdamGroups {
  int64_t e_means, e_scales, e_quats, e_opac;  // group ends (exclusive) in floats
  int sh_stride;                              // 3 K
  float lr[6];
  const long long* step_dev;  // device step counter (bias corrections on the device) or null
  float log_b1, log_b2;
};

// Bias corrections from the device step counter when there is one:
// 1 - beta^t = -expm1(t log beta).
__device__ __forceinline__ void device_steps(const AdamGroups& g, float& ss, float& isb2) {
  if (!g.step_dev) return;
  const float t = (float)*g.step_dev;
  ss = 1.f / -expm1f(t * g.log_b1);
  isb2 = rsqrtf(-expm1f(t * g.log_b2));
}

__device__ __forceinline__ float adam_lr(const AdamGroups& g, int64_t i) {
  if (i < g.e_means) return g.lr[0];
  if (i < g.e_scales) return g.lr[1];
  if (i < g.e_quats) return g.lr[2];
  if (i < g.e_opac) return g.lr[3];
  return ((i - g.e_opac) % g.sh_stride) < 3 ? g.lr[4] : g.lr[5];
}

__device__ __forceinline__ void adam_one(float& p, float g, float& m, float& v, float lr, float b1, float b2,
                                         float eps, float ss, float isb2) {
  adam_apply(p, g, m, v, lr, b1, b2, eps, ss, isb2);
}

__global__ void __launch_bounds__(256) adam_kernel(int64_t total, float4* __restrict__ p4, float4* __restrict__ g4,
                                                   float4* __restrict__ m4, float4* __restrict__ v4, AdamGroups grp,
                                                   float b1, float b2, float eps, float ss, float isb2, bool zero) {
  device_steps(grp, ss, isb2);
  const int64_t nvec = total >> 2;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nvec; q += (int64_t)gridDim.x * blockDim.x) {
    float4 p = p4[q], g = g4[q], m = m4[q], v = v4[q];
    const int64_t i = q << 2;
    adam_one(p.x, g.x, m.x, v.x, adam_lr(grp, i), b1, b2, eps, ss, isb2);
    adam_one(p.y, g.y, m.y, v.y, adam_lr(grp, i + 1), b1, b2, eps, ss, isb2);
    adam_one(p.z, g.z, m.z, v.z, adam_lr(grp, i + 2), b1, b2, eps, ss, isb2);
    adam_one(p.w, g.w, m.w, v.w, adam_lr(grp, i + 3), b1, b2, eps, ss, isb2);
    p4[q] = p;
    m4[q] = m;
    v4[q] = v;
    if (zero) g4[q] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

__global__ void adam_tail_kernel(int64_t start, int64_t total, float* __restrict__ p, float* __restrict__ g,
                                 float* __restrict__ m, float* __restrict__ v, AdamGroups grp, float b1, float b2,
                                 float eps, float ss, float isb2, bool zero) {
  device_steps(grp, ss, isb2);
  const int64_t i = start + threadIdx.x;
  if (i < total) {
    adam_one(p[i], g[i], m[i], v[i], adam_lr(grp, i), b1, b2, eps, ss, isb2);
    if (zero) g[i] = 0.f;
  }
}

__global__ void adam_scalar_kernel(int64_t total, float* __restrict__ p, float* __restrict__ g,
                                   float* __restrict__ m, float* __restrict__ v, AdamGroups grp, float b1, float b2,
                                   float eps, float ss, float isb2, bool zero) {
  device_steps(grp, ss, isb2);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    adam_one(p[i], g[i], m[i], v[i], adam_lr(grp, i), b1, b2, eps, ss, isb2);
    if (zero) g[i] = 0.f;
  }
}

__global__ void export_projection_kernel(int n, const float4* __restrict__ feat, const uint32_t* __restrict__ tiles,
                                         float* mean2d, float* cov2d, float* depth, float* rgb, float* opacity,
                                         int32_t* tiles_out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 f0 = feat[3 * i], f1 = feat[3 * i + 1], f2 = feat[3 * i + 2];
  if (mean2d) {
    mean2d[2 * i] = f0.x + f0.z;
    mean2d[2 * i + 1] = f0.y + f0.w;
  }
  if (cov2d) {
    // i0 = S/sqrt(a), k = b/a, i1 = S sqrt(a/det): a = S^2/i0^2, b = k a, c = (det + b^2)/a
    const float S2sq = kS2 * kS2;
    const float a = f1.x != 0.f ? S2sq / (f1.x * f1.x) : 0.f;
    const float b = f1.y * a;
    const float det = f1.z != 0.f ? S2sq * a / (f1.z * f1.z) : 0.f;
    cov2d[3 * i] = a;
    cov2d[3 * i + 1] = b;
    cov2d[3 * i + 2] = a != 0.f ? (det + b * b) / a : 0.f;
  }
  if (depth) depth[i] = f2.w;
  if (rgb) {
    rgb[3 * i] = f2.x;
    rgb[3 * i + 1] = f2.y;
    rgb[3 * i + 2] = f2.z;
  }
  if (opacity) opacity[i] = exp2f(f1.w);
  if (tiles_out) tiles_out[i] = (int32_t)tiles[i];
}

}  // namespace

int loss_blocks(int npix) { return (npix + kLossThreads * kLossItems - 1) / (kLossThreads * kLossItems); }

void launch_loss(const LossArgs& a, float* partials, cudaStream_t s, int64_t* launches) {
  if (a.n_blocks <= 0) return;
  float* scale = partials + 3 * a.n_blocks;
  loss_partials_kernel<<<a.n_blocks, kLossThreads, 0, s>>>(a, partials);
  loss_finalize_kernel<<<1, 256, 0, s>>>(a, partials, scale);
  scale_kernel<<<a.n_blocks, kLossThreads, 0, s>>>(a, scale);
  if (launches) *launches += 3;
}

void launch_loss_tiles_finalize(const RasterArgs& a, float w_depth, float* loss, float* depth_scale,
                                float* partials, uint32_t* ticket, long long* step, cudaStream_t s,
                                int64_t* launches) {
  TileLossArgs t;
  LossArgs la;
  t.views = la.views = a.views;
  t.jobs = a.loss_partials;
  la.w_color = a.w_color;
  la.w_depth = w_depth;
  la.loss = loss;
  int blocks = 0;
  for (int v = 0; v < a.views; ++v) {
    const uint32_t j0 = 4 * a.v[v].tile_base;
    const uint32_t j1 = 4 * (v + 1 < a.views ? a.v[v + 1].tile_base : a.n_tiles);
    t.block_base[v] = blocks;
    t.job_base[v] = j0;
    t.job_base[v + 1] = j1;
    la.v[v] = LossView{a.v[v].width * a.v[v].height, blocks, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    blocks += (int)((j1 - j0 + kTileLossChunk - 1) / kTileLossChunk);
  }
  t.block_base[a.views] = blocks;
  la.n_blocks = blocks;
  if (blocks == 0) {
    if (step) launch_step_increment(step, s);
    return;
  }
  launch_pdl(loss_tiles_kernel, blocks, kLossThreads, 0, s, t, la, partials, depth_scale, ticket, step);
  if (launches) *launches += 1;
}

void launch_adam(float* p, float* g, float* m, float* v, int64_t n_gauss, int sh_degree, const float lr[6],
                 float beta1, float beta2, float eps, float step_size_scale, float inv_sqrt_bc2, bool zero,
                 const long long* step_dev, cudaStream_t s) {
  const int K = (sh_degree + 1) * (sh_degree + 1);
  AdamGroups grp;
  grp.e_means = 3 * n_gauss;
  grp.e_scales = 6 * n_gauss;
  grp.e_quats = 10 * n_gauss;
  grp.e_opac = 11 * n_gauss;
  grp.sh_stride = 3 * K;
  for (int k = 0; k < 6; ++k) grp.lr[k] = lr[k];
  grp.step_dev = step_dev;
  grp.log_b1 = logf(beta1);
  grp.log_b2 = logf(beta2);
  const int64_t total = n_gauss * (11 + 3 * K);
  if (total == 0) return;
  const bool aligned = ((((uintptr_t)p) | ((uintptr_t)g) | ((uintptr_t)m) | ((uintptr_t)v)) & 15) == 0;
  if (aligned) {
    const int64_t nvec = total >> 2;
    if (nvec > 0) {
      int64_t blocks = std::min<int64_t>((nvec + 255) / 256, 152 * 16);
      adam_kernel<<<(int)blocks, 256, 0, s>>>(total, (float4*)p, (float4*)g, (float4*)m, (float4*)v, grp, beta1,
                                              beta2, eps, step_size_scale, inv_sqrt_bc2, zero);
    }
    if (total & 3)
      adam_tail_kernel<<<1, 4, 0, s>>>(nvec << 2, total, p, g, m, v, grp, beta1, beta2, eps, step_size_scale,
                                       inv_sqrt_bc2, zero);
  } else {
    int64_t blocks = std::min<int64_t>((total + 255) / 256, 152 * 16);
    adam_scalar_kernel<<<(int)blocks, 256, 0, s>>>(total, p, g, m, v, grp, beta1, beta2, eps, step_size_scale,
                                                   inv_sqrt_bc2, zero);
  }
}

void launch_export_projection(int n, const float4* feat, const uint32_t* tiles, float* mean2d, float* cov2d,
                              float* depth, float* rgb, float* opacity, int32_t* tiles_out, cudaStream_t s) {
  if (n <= 0) return;
  export_projection_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, feat, tiles, mean2d, cov2d, depth, rgb, opacity,
                                                           tiles_out);
}

namespace {

// non-finite floats (NaN, +-Inf) of x[0, n): per-thread counts, a warp sum,
// one atomic per warp
__global__ void __launch_bounds__(256) count_nonfinite_kernel(const float* __restrict__ x, int64_t n,
                                                              unsigned long long* __restrict__ out) {
  unsigned c = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    c += isfinite(x[i]) ? 0u : 1u;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, off);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, (unsigned long long)c);
}

}  // namespace

void launch_count_nonfinite(const float* x, int64_t n, unsigned long long* out, int num_sms, cudaStream_t s) {
  cudaMemsetAsync(out, 0, sizeof(unsigned long long), s);
  if (n <= 0) return;
  const int64_t want = (n + 255) / 256;
  const int blocks = (int)std::min<int64_t>(want, 8 * (int64_t)std::max(num_sms, 1));
  count_nonfinite_kernel<<<blocks, 256, 0, s>>>(x, n, out);
}

}  // namespace gs
