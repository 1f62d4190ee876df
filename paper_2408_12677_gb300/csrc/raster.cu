// Tile rasterizer, forward (Eq. 11, front to back with early stop on
// transmittance) and backward (back to front from the stored last
// contributor, transmittance recomputed from the stored final T).
//
// One CTA of 256 threads per tile, one pixel per thread.  The tile's
// depth-sorted list is staged in shared memory 256 Gaussians at a time (one
// gathered 48 B record per thread, converted to tile-local coordinates so the
// per-pixel offsets keep float32 precision).  The backward pass reduces each
// Gaussian's gradient over the warp with shuffles, over the CTA with shared
// atomics, and adds it to global memory once per tile with float4 atomics.
#include "common.cuh"
#include "internal.h"

namespace gs {

namespace {

constexpr int kThreads = 256;
constexpr int kBatch = 256;

template <int TW, int TH>
__global__ void __launch_bounds__(kThreads) raster_fwd_kernel(RasterParams rp, const uint2* __restrict__ ranges,
                                                              const uint32_t* __restrict__ ids,
                                                              const float4* __restrict__ feat,
                                                              float* __restrict__ color, float* __restrict__ depth,
                                                              float* __restrict__ alpha,
                                                              float* __restrict__ T_final,
                                                              int32_t* __restrict__ last_out,
                                                              unsigned long long* __restrict__ counters) {
  static_assert(TW * TH == kThreads, "one pixel per thread");
  __shared__ float4 s_a[kBatch];  // mu_local.x, mu_local.y, i0, k
  __shared__ float4 s_b[kBatch];  // i1, log2o, z, -
  __shared__ float4 s_c[kBatch];  // r, g, b, -
  const int tile = blockIdx.x;
  const int tx = tile % rp.tiles_x, ty = tile / rp.tiles_x;
  const int lx = threadIdx.x % TW, ly = threadIdx.x / TW;
  const int px = tx * TW + lx, py = ty * TH + ly;
  const bool inside = px < rp.width && py < rp.height;
  const float plx = (float)lx + 0.5f, ply = (float)ly + 0.5f;
  const float ox = (float)(tx * TW), oy = (float)(ty * TH);
  const uint2 r = ranges[tile];
  const int n = (int)(r.y - r.x);

  float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f, D = 0.f;
  int last = 0;
  uint32_t n_blend = 0, n_visit = 0;
  bool done = !inside;
  for (int b = 0; b < n; b += kBatch) {
    if (__syncthreads_count(done) == kThreads) break;
    const int i = b + threadIdx.x;
    if (i < n) {
      const uint32_t g = ids[r.x + i];
      const float4* fg = feat + 3 * (size_t)g;
      const float4 f0 = fg[0], f1 = fg[1], f2 = fg[2];
      s_a[threadIdx.x] = make_float4(__fadd_rn(__fsub_rn(f0.x, ox), f0.z), __fadd_rn(__fsub_rn(f0.y, oy), f0.w),
                                     f1.x, f1.y);
      s_b[threadIdx.x] = make_float4(f1.z, f1.w, f2.w, 0.f);
      s_c[threadIdx.x] = make_float4(f2.x, f2.y, f2.z, 0.f);
    }
    __syncthreads();
    if (!done) {
      const int cnt = min(kBatch, n - b);
      for (int j = 0; j < cnt; ++j) {
        const float4 a = s_a[j];
        const float4 bb = s_b[j];
        PixEval e;
        ++n_visit;
        if (!eval_splat(a, bb.x, bb.y, plx, ply, rp.qmax_s, rp.log2_alpha_min, e)) continue;
        const float al = fminf(rp.alpha_max, e.araw);
        const float test_T = __fmul_rn(T, __fsub_rn(1.f, al));
        if (test_T < rp.t_eps) {
          done = true;
          break;
        }
        const float4 c = s_c[j];
        const float w = al * T;
        C0 = fmaf(w, c.x, C0);
        C1 = fmaf(w, c.y, C1);
        C2 = fmaf(w, c.z, C2);
        D = fmaf(w, bb.z, D);
        T = test_T;
        last = b + j + 1;
        ++n_blend;
      }
    }
  }
  if (counters) {
    unsigned long long vb = n_blend, vv = n_visit;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      vb += __shfl_xor_sync(0xFFFFFFFFu, vb, off);
      vv += __shfl_xor_sync(0xFFFFFFFFu, vv, off);
    }
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(&counters[0], vb);
      atomicAdd(&counters[1], vv);
    }
  }
  if (inside) {
    const size_t HW = (size_t)rp.width * rp.height;
    const size_t p = (size_t)py * rp.width + px;
    if (color) {
      color[p] = C0 + T * rp.bg[0];
      color[HW + p] = C1 + T * rp.bg[1];
      color[2 * HW + p] = C2 + T * rp.bg[2];
    }
    if (depth) depth[p] = D;
    if (alpha) alpha[p] = 1.f - T;
    T_final[p] = T;
    last_out[p] = last;
  }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, off);
  return v;
}

// per-Gaussian gradient record accumulated in shared memory: 12 floats,
// {mu_x, mu_y, i0, k} {i1, opacity, z, -} {r, g, b, -}
template <int TW, int TH>
__global__ void __launch_bounds__(kThreads) raster_bwd_kernel(
    RasterParams rp, const uint2* __restrict__ ranges, const uint32_t* __restrict__ ids,
    const float4* __restrict__ feat, const float* __restrict__ T_final, const int32_t* __restrict__ last_in,
    const float* __restrict__ dLdc, const float* __restrict__ dLdd, const float* __restrict__ dLda,
    float4* __restrict__ g2d) {
  static_assert(TW * TH == kThreads, "one pixel per thread");
  __shared__ float4 s_a[kBatch];
  __shared__ float4 s_b[kBatch];  // i1, log2o, z, opacity
  __shared__ float4 s_c[kBatch];
  __shared__ uint32_t s_id[kBatch];
  __shared__ float s_acc[kBatch][12];
  __shared__ int s_maxlast;
  const int tile = blockIdx.x;
  const int tx = tile % rp.tiles_x, ty = tile / rp.tiles_x;
  const int lx = threadIdx.x % TW, ly = threadIdx.x / TW;
  const int px = tx * TW + lx, py = ty * TH + ly;
  const bool inside = px < rp.width && py < rp.height;
  const float plx = (float)lx + 0.5f, ply = (float)ly + 0.5f;
  const float ox = (float)(tx * TW), oy = (float)(ty * TH);
  const uint2 r = ranges[tile];
  const int lane = threadIdx.x & 31;

  const size_t HW = (size_t)rp.width * rp.height;
  const size_t p = (size_t)py * rp.width + px;
  float T = 1.f, dC0 = 0.f, dC1 = 0.f, dC2 = 0.f, dD = 0.f, dA = 0.f;
  int my_last = 0;
  if (inside) {
    T = T_final[p];
    my_last = last_in[p];
    dC0 = dLdc[p];
    dC1 = dLdc[HW + p];
    dC2 = dLdc[2 * HW + p];
    dD = dLdd[p];
    dA = dLda ? dLda[p] : 0.f;
  }
  const float T_fin = T;
  // U = sum over Gaussians behind of w_j (c_j . dC + z_j dD) + T_final (bg . dC)
  float U = T_fin * (rp.bg[0] * dC0 + rp.bg[1] * dC1 + rp.bg[2] * dC2);
  const float dA_T = dA * T_fin;

  if (threadIdx.x == 0) s_maxlast = 0;
  __syncthreads();
  if (my_last > 0) atomicMax(&s_maxlast, my_last);
  __syncthreads();
  const int max_last = s_maxlast;

  for (int hi = max_last; hi > 0; hi -= kBatch) {
    const int lo = max(0, hi - kBatch);
    const int cnt = hi - lo;
    __syncthreads();
    if (threadIdx.x < cnt) {
      const uint32_t g = ids[r.x + lo + threadIdx.x];
      const float4* fg = feat + 3 * (size_t)g;
      const float4 f0 = fg[0], f1 = fg[1], f2 = fg[2];
      s_a[threadIdx.x] = make_float4(__fadd_rn(__fsub_rn(f0.x, ox), f0.z), __fadd_rn(__fsub_rn(f0.y, oy), f0.w),
                                     f1.x, f1.y);
      s_b[threadIdx.x] = make_float4(f1.z, f1.w, f2.w, ex2_approx(f1.w));
      s_c[threadIdx.x] = make_float4(f2.x, f2.y, f2.z, 0.f);
      s_id[threadIdx.x] = g;
    }
    for (int k = threadIdx.x; k < kBatch * 12; k += kThreads) (&s_acc[0][0])[k] = 0.f;
    __syncthreads();
    for (int jj = cnt - 1; jj >= 0; --jj) {
      const int idx = lo + jj;
      float v[10];
#pragma unroll
      for (int k = 0; k < 10; ++k) v[k] = 0.f;
      bool contrib = false;
      if (idx < my_last) {
        const float4 a = s_a[jj];
        const float4 bb = s_b[jj];
        PixEval e;
        if (eval_splat(a, bb.x, bb.y, plx, ply, rp.qmax_s, rp.log2_alpha_min, e)) {
          contrib = true;
          const float al = fminf(rp.alpha_max, e.araw);
          const float one_m = 1.f - al;
          const float inv1m = 1.f / one_m;
          const float Ti = T * inv1m;  // transmittance in front of this Gaussian
          const float w = al * Ti;
          const float4 c = s_c[jj];
          v[7] = w * dC0;
          v[8] = w * dC1;
          v[9] = w * dC2;
          v[6] = w * dD;
          const float cdot = c.x * dC0 + c.y * dC1 + c.z * dC2 + bb.z * dD;
          // d/d alpha_i: colour/depth T_i c_i - (sum behind)/(1 - alpha_i); alpha image + T_final/(1 - alpha_i)
          const float g_alpha = Ti * cdot - (U - dA_T) * inv1m;
          U = fmaf(w, cdot, U);
          T = Ti;
          if (e.araw <= rp.alpha_max) {
            v[5] = g_alpha * e.araw / bb.w;           // d alpha / d opacity = G
            const float gq = -g_alpha * e.araw * kLn2;  // d alpha / d q' = -ln2 alpha
            // q' = t0^2 + t1^2, t0 = i0 dx, t1 = i1 (dy - k dx), dx = plx - mu_x
            const float two_t0 = 2.f * e.t0, two_t1 = 2.f * e.t1;
            const float dq_ddx = two_t0 * a.z - two_t1 * bb.x * a.w;
            const float dq_ddy = two_t1 * bb.x;
            v[0] = -gq * dq_ddx;
            v[1] = -gq * dq_ddy;
            v[2] = gq * two_t0 * e.dx;
            v[3] = -gq * two_t1 * bb.x * e.dx;
            v[4] = gq * two_t1 * e.w;
          }
        }
      }
      const unsigned m = __ballot_sync(0xFFFFFFFFu, contrib);
      if (m == 0) continue;
      if (__popc(m) == 1) {
        if (contrib) {
#pragma unroll
          for (int k = 0; k < 10; ++k) atomicAdd(&s_acc[jj][k], v[k]);
        }
      } else {
#pragma unroll
        for (int k = 0; k < 10; ++k) v[k] = warp_sum(v[k]);
        if (lane == 0) {
#pragma unroll
          for (int k = 0; k < 10; ++k) atomicAdd(&s_acc[jj][k], v[k]);
        }
      }
    }
    __syncthreads();
    if (threadIdx.x < cnt) {
      const float* acc = s_acc[threadIdx.x];
      bool nz = false;
#pragma unroll
      for (int k = 0; k < 10; ++k) nz |= acc[k] != 0.f;
      if (nz) {
        float4* dst = g2d + 3 * (size_t)s_id[threadIdx.x];
        atomicAdd(dst, make_float4(acc[0], acc[1], acc[2], acc[3]));
        atomicAdd(dst + 1, make_float4(acc[4], acc[5], acc[6], 0.f));
        atomicAdd(dst + 2, make_float4(acc[7], acc[8], acc[9], 0.f));
      }
    }
  }
}

RasterParams make_params(const RasterArgs& a) {
  RasterParams rp;
  rp.width = a.width;
  rp.height = a.height;
  rp.tile_w = a.tile_w;
  rp.tile_h = a.tile_h;
  rp.tiles_x = a.tiles_x;
  rp.tiles_y = a.tiles_y;
  for (int c = 0; c < 3; ++c) rp.bg[c] = a.bg[c];
  rp.alpha_max = a.alpha_max;
  rp.log2_alpha_min = log2f(a.alpha_min);
  rp.qmax_s = 9.f * kHalfLog2e;
  rp.t_eps = a.t_eps;
  return rp;
}

}  // namespace

bool raster_shape_supported(int tw, int th) {
  return (tw == 16 && th == 16) || (tw == 8 && th == 32) || (tw == 32 && th == 8);
}

void launch_raster_fwd(const RasterArgs& a, float* color, float* depth, float* alpha, float* T_final,
                       int32_t* last, unsigned long long* counters, cudaStream_t s) {
  const int nt = a.tiles_x * a.tiles_y;
  if (nt == 0) return;
  RasterParams rp = make_params(a);
  if (a.tile_w == 16)
    raster_fwd_kernel<16, 16><<<nt, kThreads, 0, s>>>(rp, a.ranges, a.ids, a.feat, color, depth, alpha, T_final, last,
                                                      counters);
  else if (a.tile_w == 8)
    raster_fwd_kernel<8, 32><<<nt, kThreads, 0, s>>>(rp, a.ranges, a.ids, a.feat, color, depth, alpha, T_final, last,
                                                      counters);
  else
    raster_fwd_kernel<32, 8><<<nt, kThreads, 0, s>>>(rp, a.ranges, a.ids, a.feat, color, depth, alpha, T_final, last,
                                                      counters);
}

void launch_raster_bwd(const RasterArgs& a, const float* T_final, const int32_t* last, const float* dL_dcolor,
                       const float* dL_ddepth, const float* dL_dalpha, float4* g2d, cudaStream_t s) {
  const int nt = a.tiles_x * a.tiles_y;
  if (nt == 0) return;
  RasterParams rp = make_params(a);
  if (a.tile_w == 16)
    raster_bwd_kernel<16, 16><<<nt, kThreads, 0, s>>>(rp, a.ranges, a.ids, a.feat, T_final, last, dL_dcolor,
                                                      dL_ddepth, dL_dalpha, g2d);
  else if (a.tile_w == 8)
    raster_bwd_kernel<8, 32><<<nt, kThreads, 0, s>>>(rp, a.ranges, a.ids, a.feat, T_final, last, dL_dcolor,
                                                     dL_ddepth, dL_dalpha, g2d);
  else
    raster_bwd_kernel<32, 8><<<nt, kThreads, 0, s>>>(rp, a.ranges, a.ids, a.feat, T_final, last, dL_dcolor,
                                                     dL_ddepth, dL_dalpha, g2d);
}

}  // namespace gs
