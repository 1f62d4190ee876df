// Tile rasterizer, forward (Eq. 11, front to back with early stop on
// transmittance) and backward (back to front from the stored last
// contributor, transmittance recomputed from the stored final T).
//
// One CTA of 128 threads per tile; each warp owns an 8 x 8 pixel block, each
// thread two pixels of it (rows y and y + 4).  The tile's depth-sorted list is
// staged in shared memory 256 Gaussians at a time (gathered 48 B records,
// converted to tile-local coordinates so the per-pixel offsets keep float32
// precision); each Gaussian's support bounding box is tested against the four
// warp blocks and every warp walks only its own compacted list.  The backward
// pass sums each Gaussian's gradient over the warp (direct shared atomics when
// at most two lanes contribute, else a transposed shuffle reduction), over the
// CTA in shared memory, and adds it to global memory once per tile with
// float4 atomics.
#include "common.cuh"
#include "internal.h"

namespace gs {

namespace {

constexpr int kThreads = 128;  // 4 warps, each owns an 8 x 8 pixel block, 2 pixels per thread
constexpr int kBatch = 256;    // Gaussians staged in shared memory per step
constexpr unsigned kFull = 0xFFFFFFFFu;

// Stage one list entry: features in tile-local coordinates and the mask of
// warps whose 8 x 8 block meets the splat's support bounding box.  The box
// holds every pixel the per-pixel test can accept: q' <= min(qmax, log2 o -
// log2 alpha_min) is the ellipse (i0 dx)^2 + (i1 (dy - k dx))^2 <= R2, whose
// half-extents are sqrt(R2) / i0 and sqrt(R2) sqrt(k^2 / i0^2 + 1 / i1^2);
// the widening covers float32 rounding of the test.
template <int WX>
__device__ __forceinline__ void stage_entry(const float4* __restrict__ feat, uint32_t g, float ox, float oy,
                                            const RasterParams& rp, float4& sa, float4& sb, float4& sc,
                                            uint32_t& mask) {
  const float4* fg = feat + 3 * (size_t)g;
  const float4 f0 = fg[0], f1 = fg[1], f2 = fg[2];
  const float mlx = __fadd_rn(__fsub_rn(f0.x, ox), f0.z);
  const float mly = __fadd_rn(__fsub_rn(f0.y, oy), f0.w);
  sa = make_float4(mlx, mly, f1.x, f1.y);
  sb = make_float4(f1.z, f1.w, f2.w, ex2_approx(-f1.w));  // .w = 1 / opacity
  sc = make_float4(f2.x, f2.y, f2.z, 0.f);
  mask = 0;
  const float R2 = fminf(rp.qmax_s, f1.w - rp.log2_alpha_min);
  if (R2 > 0.f && f1.x > 0.f && f1.z > 0.f) {
    const float Rr = sqrtf(R2) * 1.0001f + 1e-4f;
    const float inv0 = 1.f / f1.x, inv1 = 1.f / f1.z;
    const float ex = Rr * inv0 + 1e-3f;
    const float ey = Rr * sqrtf(f1.y * f1.y * inv0 * inv0 + inv1 * inv1) + 1e-3f;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      const float x0 = (float)((w % WX) * 8) + 0.5f, y0 = (float)((w / WX) * 8) + 0.5f;
      if (mlx + ex >= x0 && mlx - ex <= x0 + 7.f && mly + ey >= y0 && mly - ey <= y0 + 7.f) mask |= 1u << w;
    }
  }
}

// Compact the batch entries whose mask has bit `w` into list[0..count).
__device__ __forceinline__ int build_list(const uint32_t* s_mask, int cnt, int w, uint8_t* list) {
  const int lane = threadIdx.x & 31;
  int count = 0;
  for (int base = 0; base < cnt; base += 32) {
    const int j = base + lane;
    const bool on = j < cnt && ((s_mask[j] >> w) & 1u);
    const unsigned bal = __ballot_sync(kFull, on);
    if (on) list[count + __popc(bal & ((1u << lane) - 1u))] = (uint8_t)j;
    count += __popc(bal);
  }
  __syncwarp();
  return count;
}

template <int TW, int TH, bool COUNT>
__global__ void __launch_bounds__(kThreads) raster_fwd_kernel(RasterParams rp, const uint2* __restrict__ ranges,
                                                              const uint32_t* __restrict__ ids,
                                                              const float4* __restrict__ feat,
                                                              float* __restrict__ color, float* __restrict__ depth,
                                                              float* __restrict__ alpha,
                                                              float* __restrict__ T_final,
                                                              int32_t* __restrict__ last_out,
                                                              unsigned long long* __restrict__ counters) {
  constexpr int WX = TW / 8;
  static_assert((TW / 8) * (TH / 8) == kThreads / 32, "four 8x8 warp blocks per tile");
  __shared__ float4 s_a[kBatch];  // mu_local.x, mu_local.y, i0, k
  __shared__ float4 s_b[kBatch];  // i1, log2o, z, 1/opacity
  __shared__ float4 s_c[kBatch];  // r, g, b, -
  __shared__ uint32_t s_mask[kBatch];
  __shared__ uint8_t s_list[kThreads / 32][kBatch];
  const int tile = blockIdx.x;
  const int tx = tile % rp.tiles_x, ty = tile / rp.tiles_x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int lx = (warp % WX) * 8 + (lane & 7), ly0 = (warp / WX) * 8 + (lane >> 3), ly1 = ly0 + 4;
  const int px = tx * TW + lx, py0 = ty * TH + ly0, py1 = ty * TH + ly1;
  const bool in0 = px < rp.width && py0 < rp.height, in1 = px < rp.width && py1 < rp.height;
  const float plx = (float)lx + 0.5f, ply0 = (float)ly0 + 0.5f, ply1 = (float)ly1 + 0.5f;
  const float ox = (float)(tx * TW), oy = (float)(ty * TH);
  const uint2 r = ranges[tile];
  const int n = (int)(r.y - r.x);

  float T0 = 1.f, R0 = 0.f, G0 = 0.f, B0 = 0.f, D0 = 0.f;
  float T1 = 1.f, R1 = 0.f, G1 = 0.f, B1 = 0.f, D1 = 0.f;
  int last0 = 0, last1 = 0;
  uint32_t n_blend = 0, n_visit = 0;
  bool done0 = !in0, done1 = !in1;
  for (int b = 0; b < n; b += kBatch) {
    if (__syncthreads_count(done0 && done1) == kThreads) break;
#pragma unroll
    for (int s = threadIdx.x; s < kBatch; s += kThreads) {
      if (b + s < n) stage_entry<WX>(feat, ids[r.x + b + s], ox, oy, rp, s_a[s], s_b[s], s_c[s], s_mask[s]);
    }
    __syncthreads();
    const int cnt = min(kBatch, n - b);
    const int count = build_list(s_mask, cnt, warp, s_list[warp]);
    for (int q = 0; q < count; ++q) {
      if ((q & 7) == 0 && __all_sync(kFull, done0 && done1)) break;
      const int j = s_list[warp][q];
      const float4 a = s_a[j];
      const float4 bb = s_b[j];
      PixEval e;
      if (!done0) {
        if (COUNT) ++n_visit;
        if (eval_splat(a, bb.x, bb.y, plx, ply0, rp.qmax_s, rp.log2_alpha_min, e)) {
          const float al = fminf(rp.alpha_max, e.araw);
          const float test_T = __fmul_rn(T0, __fsub_rn(1.f, al));
          if (test_T < rp.t_eps) {
            done0 = true;
          } else {
            const float4 c = s_c[j];
            const float w = al * T0;
            R0 = fmaf(w, c.x, R0);
            G0 = fmaf(w, c.y, G0);
            B0 = fmaf(w, c.z, B0);
            D0 = fmaf(w, bb.z, D0);
            T0 = test_T;
            last0 = b + j + 1;
            if (COUNT) ++n_blend;
          }
        }
      }
      if (!done1) {
        if (COUNT) ++n_visit;
        if (eval_splat(a, bb.x, bb.y, plx, ply1, rp.qmax_s, rp.log2_alpha_min, e)) {
          const float al = fminf(rp.alpha_max, e.araw);
          const float test_T = __fmul_rn(T1, __fsub_rn(1.f, al));
          if (test_T < rp.t_eps) {
            done1 = true;
          } else {
            const float4 c = s_c[j];
            const float w = al * T1;
            R1 = fmaf(w, c.x, R1);
            G1 = fmaf(w, c.y, G1);
            B1 = fmaf(w, c.z, B1);
            D1 = fmaf(w, bb.z, D1);
            T1 = test_T;
            last1 = b + j + 1;
            if (COUNT) ++n_blend;
          }
        }
      }
    }
  }
  if (COUNT) {
    unsigned long long vb = n_blend, vv = n_visit;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      vb += __shfl_xor_sync(kFull, vb, off);
      vv += __shfl_xor_sync(kFull, vv, off);
    }
    if (lane == 0) {
      atomicAdd(&counters[0], vb);
      atomicAdd(&counters[1], vv);
    }
  }
  const size_t HW = (size_t)rp.width * rp.height;
  if (in0) {
    const size_t p = (size_t)py0 * rp.width + px;
    if (color) {
      color[p] = R0 + T0 * rp.bg[0];
      color[HW + p] = G0 + T0 * rp.bg[1];
      color[2 * HW + p] = B0 + T0 * rp.bg[2];
    }
    if (depth) depth[p] = D0;
    if (alpha) alpha[p] = 1.f - T0;
    T_final[p] = T0;
    last_out[p] = last0;
  }
  if (in1) {
    const size_t p = (size_t)py1 * rp.width + px;
    if (color) {
      color[p] = R1 + T1 * rp.bg[0];
      color[HW + p] = G1 + T1 * rp.bg[1];
      color[2 * HW + p] = B1 + T1 * rp.bg[2];
    }
    if (depth) depth[p] = D1;
    if (alpha) alpha[p] = 1.f - T1;
    T_final[p] = T1;
    last_out[p] = last1;
  }
}

// Sum the 10 values v[0..9] over the warp with exchanges that halve the number
// of values each lane carries (xor 16: 10 -> 5, xor 8: 5 -> 3, xor 4: 3 -> 2,
// xor 2: 2 -> 1) and a final xor-1 step (12 shuffles instead of 50).  The
// even lane l then holds the total of value vidx(l) and adds it to dst.
__device__ __forceinline__ void warp_transpose_add10(float (&v)[10], float* dst) {
  const int lane = threadIdx.x & 31;
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4, b1 = lane & 2;
  float u[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) {  // keep v[i] (b4 = 0) or v[i + 5] (b4 = 1)
    const float send = b4 ? v[i] : v[i + 5];
    const float keep = b4 ? v[i + 5] : v[i];
    u[i] = keep + __shfl_xor_sync(kFull, send, 16);
  }
  float w3[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {  // keep u[0..2] (b3 = 0) or u[3..4], 0 (b3 = 1)
    const float hi = i < 2 ? u[i + 3] : 0.f;
    const float send = b3 ? u[i] : hi;
    const float keep = b3 ? hi : u[i];
    w3[i] = keep + __shfl_xor_sync(kFull, send, 8);
  }
  float w2[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) {  // keep w3[0..1] (b2 = 0) or w3[2], 0 (b2 = 1)
    const float hi = i < 1 ? w3[i + 2] : 0.f;
    const float send = b2 ? w3[i] : hi;
    const float keep = b2 ? hi : w3[i];
    w2[i] = keep + __shfl_xor_sync(kFull, send, 4);
  }
  float x;
  {
    const float send = b1 ? w2[0] : w2[1];
    const float keep = b1 ? w2[1] : w2[0];
    x = keep + __shfl_xor_sync(kFull, send, 2);
  }
  x += __shfl_xor_sync(kFull, x, 1);
  // value held: 5 b4 + i3 with i3 = 3 b3 + 2 b2 + b1 among the five kept at
  // xor 16; lanes with b2 and (b3 or b1) hold the zero pads
  const int i3 = (b3 ? 3 : 0) + (b2 ? 2 : 0) + (b1 ? 1 : 0);
  const bool valid = !(b2 && (b3 || b1));
  if (!(lane & 1) && valid) atomicAdd(&dst[(b4 ? 5 : 0) + i3], x);
}

// Back-to-front step of one pixel for one Gaussian: updates the pixel's
// running transmittance T and "colour behind" U and adds the Gaussian's
// gradient record (mu 2, factor 3, opacity, z, rgb 3) to v.
__device__ __forceinline__ bool bwd_pixel(const float4& a, const float4& bb, const float4* s_c, int j, float plx,
                                          float ply, const RasterParams& rp, float& T, float& U, float dC0, float dC1,
                                          float dC2, float dD, float dA_T, float (&v)[10]) {
  PixEval e;
  if (!eval_splat(a, bb.x, bb.y, plx, ply, rp.qmax_s, rp.log2_alpha_min, e)) return false;
  const float al = fminf(rp.alpha_max, e.araw);
  const float inv1m = __frcp_rn(1.f - al);
  const float Ti = T * inv1m;  // transmittance in front of this Gaussian
  const float w = al * Ti;
  const float4 c = s_c[j];
  v[7] += w * dC0;
  v[8] += w * dC1;
  v[9] += w * dC2;
  v[6] += w * dD;
  const float cdot = c.x * dC0 + c.y * dC1 + c.z * dC2 + bb.z * dD;
  // d/d alpha_i: colour/depth T_i c_i - (sum behind)/(1 - alpha_i); alpha image + T_final/(1 - alpha_i)
  const float g_alpha = Ti * cdot - (U - dA_T) * inv1m;
  U = fmaf(w, cdot, U);
  T = Ti;
  if (e.araw <= rp.alpha_max) {
    v[5] += g_alpha * e.araw * bb.w;             // d alpha / d opacity = G = alpha / opacity
    const float gq = -g_alpha * e.araw * kLn2;  // d alpha / d q' = -ln2 alpha
    // q' = t0^2 + t1^2, t0 = i0 dx, t1 = i1 (dy - k dx), dx = plx - mu_x
    const float two_t0 = 2.f * e.t0, two_t1 = 2.f * e.t1;
    const float dq_ddx = two_t0 * a.z - two_t1 * bb.x * a.w;
    const float dq_ddy = two_t1 * bb.x;
    v[0] -= gq * dq_ddx;
    v[1] -= gq * dq_ddy;
    v[2] += gq * two_t0 * e.dx;
    v[3] -= gq * two_t1 * bb.x * e.dx;
    v[4] += gq * two_t1 * e.w;
  }
  return true;
}

template <int TW, int TH>
__global__ void __launch_bounds__(kThreads) raster_bwd_kernel(
    RasterParams rp, const uint2* __restrict__ ranges, const uint32_t* __restrict__ ids,
    const float4* __restrict__ feat, const float* __restrict__ T_final, const int32_t* __restrict__ last_in,
    const float* __restrict__ dLdc, const float* __restrict__ dLdd, const float* __restrict__ dLda,
    float4* __restrict__ g2d) {
  constexpr int WX = TW / 8;
  static_assert((TW / 8) * (TH / 8) == kThreads / 32, "four 8x8 warp blocks per tile");
  __shared__ float4 s_a[kBatch];
  __shared__ float4 s_b[kBatch];  // i1, log2o, z, 1/opacity
  __shared__ float4 s_c[kBatch];
  __shared__ uint32_t s_mask[kBatch];
  __shared__ uint32_t s_id[kBatch];
  __shared__ uint8_t s_list[kThreads / 32][kBatch];
  __shared__ float s_acc[kBatch][12];
  __shared__ int s_maxlast;
  const int tile = blockIdx.x;
  const int tx = tile % rp.tiles_x, ty = tile / rp.tiles_x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int lx = (warp % WX) * 8 + (lane & 7), ly0 = (warp / WX) * 8 + (lane >> 3), ly1 = ly0 + 4;
  const int px = tx * TW + lx, py0 = ty * TH + ly0, py1 = ty * TH + ly1;
  const bool in0 = px < rp.width && py0 < rp.height, in1 = px < rp.width && py1 < rp.height;
  const float plx = (float)lx + 0.5f, ply0 = (float)ly0 + 0.5f, ply1 = (float)ly1 + 0.5f;
  const float ox = (float)(tx * TW), oy = (float)(ty * TH);
  const uint2 r = ranges[tile];
  const size_t HW = (size_t)rp.width * rp.height;

  // per-pixel state (two pixels per thread)
  float T0 = 1.f, c00 = 0.f, c01 = 0.f, c02 = 0.f, d0 = 0.f, a0 = 0.f;
  float T1 = 1.f, c10 = 0.f, c11 = 0.f, c12 = 0.f, d1 = 0.f, a1 = 0.f;
  int last0 = 0, last1 = 0;
  if (in0) {
    const size_t p = (size_t)py0 * rp.width + px;
    T0 = T_final[p];
    last0 = last_in[p];
    c00 = dLdc[p];
    c01 = dLdc[HW + p];
    c02 = dLdc[2 * HW + p];
    d0 = dLdd[p];
    a0 = dLda ? dLda[p] : 0.f;
  }
  if (in1) {
    const size_t p = (size_t)py1 * rp.width + px;
    T1 = T_final[p];
    last1 = last_in[p];
    c10 = dLdc[p];
    c11 = dLdc[HW + p];
    c12 = dLdc[2 * HW + p];
    d1 = dLdd[p];
    a1 = dLda ? dLda[p] : 0.f;
  }
  // U = sum over Gaussians behind of w_j (c_j . dC + z_j dD) + T_final (bg . dC)
  float U0 = T0 * (rp.bg[0] * c00 + rp.bg[1] * c01 + rp.bg[2] * c02);
  float U1 = T1 * (rp.bg[0] * c10 + rp.bg[1] * c11 + rp.bg[2] * c12);
  const float dAT0 = a0 * T0, dAT1 = a1 * T1;

  int wmax = max(last0, last1);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) wmax = max(wmax, __shfl_xor_sync(kFull, wmax, off));
  if (threadIdx.x == 0) s_maxlast = 0;
  __syncthreads();
  if (lane == 0 && wmax > 0) atomicMax(&s_maxlast, wmax);
  __syncthreads();
  const int max_last = s_maxlast;

  for (int hi = max_last; hi > 0; hi -= kBatch) {
    const int lo = max(0, hi - kBatch);
    const int cnt = hi - lo;
    __syncthreads();
#pragma unroll
    for (int s = threadIdx.x; s < kBatch; s += kThreads) {
      if (s < cnt) {
        const uint32_t g = ids[r.x + lo + s];
        s_id[s] = g;
        stage_entry<WX>(feat, g, ox, oy, rp, s_a[s], s_b[s], s_c[s], s_mask[s]);
      }
    }
    for (int k = threadIdx.x; k < kBatch * 12; k += kThreads) (&s_acc[0][0])[k] = 0.f;
    __syncthreads();
    const int count = build_list(s_mask, cnt, warp, s_list[warp]);
    for (int q = count - 1; q >= 0; --q) {
      const int j = s_list[warp][q];
      const int idx = lo + j;
      if (idx >= wmax) continue;  // behind every pixel's last contributor in this warp
      const float4 a = s_a[j];
      const float4 bb = s_b[j];
      float v[10];
#pragma unroll
      for (int k = 0; k < 10; ++k) v[k] = 0.f;
      bool contrib = false;
      if (idx < last0) contrib |= bwd_pixel(a, bb, s_c, j, plx, ply0, rp, T0, U0, c00, c01, c02, d0, dAT0, v);
      if (idx < last1) contrib |= bwd_pixel(a, bb, s_c, j, plx, ply1, rp, T1, U1, c10, c11, c12, d1, dAT1, v);
      const unsigned m = __ballot_sync(kFull, contrib);
      if (m == 0) continue;
      if (__popc(m) <= 2) {
        if (contrib) {
#pragma unroll
          for (int k = 0; k < 10; ++k) atomicAdd(&s_acc[j][k], v[k]);
        }
      } else {
        warp_transpose_add10(v, s_acc[j]);
      }
    }
    __syncthreads();
#pragma unroll
    for (int s = threadIdx.x; s < kBatch; s += kThreads) {
      if (s < cnt) {
        const float* acc = s_acc[s];
        bool nz = false;
#pragma unroll
        for (int k = 0; k < 10; ++k) nz |= acc[k] != 0.f;
        if (nz) {
          float4* dst = g2d + 3 * (size_t)s_id[s];
          atomicAdd(dst, make_float4(acc[0], acc[1], acc[2], acc[3]));
          atomicAdd(dst + 1, make_float4(acc[4], acc[5], acc[6], 0.f));
          atomicAdd(dst + 2, make_float4(acc[7], acc[8], acc[9], 0.f));
        }
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
#define GS_FWD(TW_, TH_, C_)                                                                               \
  raster_fwd_kernel<TW_, TH_, C_><<<nt, kThreads, 0, s>>>(rp, a.ranges, a.ids, a.feat, color, depth, alpha, T_final, \
                                                         last, counters)
  if (counters) {
    if (a.tile_w == 16) GS_FWD(16, 16, true);
    else if (a.tile_w == 8) GS_FWD(8, 32, true);
    else GS_FWD(32, 8, true);
  } else {
    if (a.tile_w == 16) GS_FWD(16, 16, false);
    else if (a.tile_w == 8) GS_FWD(8, 32, false);
    else GS_FWD(32, 8, false);
  }
#undef GS_FWD
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
