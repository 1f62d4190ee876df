// Projection of 3D Gaussians to 2D splats (Eq. 2-5) and its backward pass,
// including the gradient w.r.t. the camera pose.
#include <type_traits>

#include "common.cuh"
#include "internal.h"

namespace gs {

namespace {

__device__ __forceinline__ void quat_rotmat(float w, float x, float y, float z, float R[3][3]) {
  R[0][0] = 1.f - 2.f * (y * y + z * z);
  R[0][1] = 2.f * (x * y - w * z);
  R[0][2] = 2.f * (x * z + w * y);
  R[1][0] = 2.f * (x * y + w * z);
  R[1][1] = 1.f - 2.f * (x * x + z * z);
  R[1][2] = 2.f * (y * z - w * x);
  R[2][0] = 2.f * (x * z - w * y);
  R[2][1] = 2.f * (y * z + w * x);
  R[2][2] = 1.f - 2.f * (x * x + y * y);
}

// Everything of the forward projection that the backward pass needs again,
// in float32.
struct Geo {
  float x, y, z, rz;
  float xt, yt;      // clamped J positions x~, y~
  bool cx_, cy_;     // clamp active
  float qn[4], qlen;
  float Rq[3][3];
  float s[3];
  float B[3][3];     // Rq diag(s)
  float A[3][3];     // W B
  float j00, j02, j11, j12;
  float m0[3], m1[3];
  float a, b, c, det;
  float i0, k, i1;
};

__device__ __forceinline__ void geometry(const CamView& cv, float dilation, float px, float py, float pz,
                                         const float* q4, const float* ls, float x, float y, float z, Geo& g) {
  g.x = x;
  g.y = y;
  g.z = z;
  g.rz = 1.f / z;
  const float limx = 1.3f * (float)cv.width / (2.f * cv.fx);
  const float limy = 1.3f * (float)cv.height / (2.f * cv.fy);
  float xr = x * g.rz, yr = y * g.rz;
  g.cx_ = (xr < -limx) || (xr > limx);
  g.cy_ = (yr < -limy) || (yr > limy);
  g.xt = fminf(fmaxf(xr, -limx), limx) * z;
  g.yt = fminf(fmaxf(yr, -limy), limy) * z;
  float qq = q4[0] * q4[0] + q4[1] * q4[1] + q4[2] * q4[2] + q4[3] * q4[3];
  float inv = rsqrtf(qq);
  g.qlen = qq * inv;
  for (int j = 0; j < 4; ++j) g.qn[j] = q4[j] * inv;
  quat_rotmat(g.qn[0], g.qn[1], g.qn[2], g.qn[3], g.Rq);
  for (int j = 0; j < 3; ++j) g.s[j] = expf(ls[j]);
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) g.B[r][c] = g.Rq[r][c] * g.s[c];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c)
      g.A[r][c] = cv.R[3 * r + 0] * g.B[0][c] + cv.R[3 * r + 1] * g.B[1][c] + cv.R[3 * r + 2] * g.B[2][c];
  g.j00 = cv.fx * g.rz;
  g.j02 = -cv.fx * g.xt * g.rz * g.rz;
  g.j11 = cv.fy * g.rz;
  g.j12 = -cv.fy * g.yt * g.rz * g.rz;
  for (int c = 0; c < 3; ++c) {
    g.m0[c] = g.j00 * g.A[0][c] + g.j02 * g.A[2][c];
    g.m1[c] = g.j11 * g.A[1][c] + g.j12 * g.A[2][c];
  }
  float n0 = g.m0[0] * g.m0[0] + g.m0[1] * g.m0[1] + g.m0[2] * g.m0[2];
  float n1 = g.m1[0] * g.m1[0] + g.m1[1] * g.m1[1] + g.m1[2] * g.m1[2];
  g.a = n0 + dilation;
  g.c = n1 + dilation;
  g.b = g.m0[0] * g.m1[0] + g.m0[1] * g.m1[1] + g.m0[2] * g.m1[2];
  // det of the dilated covariance without cancellation (Lagrange identity):
  // |m0 x m1|^2 + dil (|m0|^2 + |m1|^2) + dil^2, where
  // m0 x m1 = det(A) A^-1 (j0 x j1) = diag(s1 s2, s0 s2, s0 s1) Rq^T W^T (fx fy / z^3)(x~, y~, z)
  float v[3];
  for (int r = 0; r < 3; ++r) v[r] = cv.R[r] * g.xt + cv.R[3 + r] * g.yt + cv.R[6 + r] * z;  // W^T (x~, y~, z)
  float u[3];
  for (int c = 0; c < 3; ++c) u[c] = g.Rq[0][c] * v[0] + g.Rq[1][c] * v[1] + g.Rq[2][c] * v[2];
  float f = cv.fx * cv.fy * g.rz * g.rz * g.rz;
  float c0 = g.s[1] * g.s[2] * u[0] * f, c1 = g.s[0] * g.s[2] * u[1] * f, c2 = g.s[0] * g.s[1] * u[2] * f;
  g.det = c0 * c0 + c1 * c1 + c2 * c2 + dilation * (n0 + n1) + dilation * dilation;
  g.i0 = kS2 * rsqrtf(g.a);
  g.k = g.b / g.a;
  g.i1 = kS2 * sqrtf(g.a / g.det);
}

__device__ __forceinline__ void cp_async4(float* smem, const float* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

constexpr int kFwdThreads = 128;

// 16-byte asynchronous copy (both addresses 16-byte aligned)
__device__ __forceinline__ void cp_async16(float* smem, const float* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
// Stages len floats from src (4-byte aligned, sh = (address / 4) mod 4) to
// dst[sh .. sh + len): 4-byte copies up to the first 16-byte boundary and
// after the last, 16-byte copies in between (dst 16-byte aligned).
__device__ __forceinline__ void stage_slice16(float* dst, const float* src, int len, int sh, int t, int nthreads) {
  const int head = min((4 - sh) & 3, len);
  const int nvec = (len - head) >> 2;
  const int tail0 = head + 4 * nvec;
  if (t < head) cp_async4(dst + sh + t, src + t);
  for (int c = t; c < nvec; c += nthreads) cp_async16(dst + sh + head + 4 * c, src + head + 4 * c);
  if (t < len - tail0) cp_async4(dst + sh + tail0 + t, src + tail0 + t);
}

// tiles a block's shared counters cover (the bounding box of its rectangles)
constexpr int kCountBox = 1024;

// Bucket mode: takes slot `slot` of tile t's bucket for item `item` (a slot
// beyond the bucket's capacity sets bit 4 of *overflow instead).
__device__ __forceinline__ void bucket_put(uint32_t* __restrict__ bids, uint32_t cap, uint32_t* __restrict__ overflow,
                                           uint32_t t, uint32_t slot, uint32_t item) {
  if (slot < cap)
    bids[(size_t)t * cap + slot] = item;
  else
    atomicOr(overflow, 4u);
}

// Adds the tiles of the block's rectangles [x0, x1) x [y0, y1) of one view
// (those of at most kBigTiles tiles: ns = their tile count, 0 for the others
// and for threads without an item) to the global per-tile counters.  When
// the block's rectangles lie in a box of at most kCountBox tiles they are
// counted in shared memory (s_cnt) first and each touched tile's counter
// gets one atomic add; otherwise each (item, tile) pair adds 1 directly.
// Bucket mode (bids non-null): the same counting reserves each touched
// tile's run of slots (the atomic returns its start), then every pair takes
// the next slot of its tile's run and writes `item` there.
// Called by every thread of the block (it synchronises the block).
__device__ __forceinline__ void block_count_tiles(uint32_t* __restrict__ counts, uint32_t tile_base, int tiles_x,
                                                  int x0, int y0, int x1, int y1, uint32_t ns,
                                                  uint32_t* __restrict__ s_cnt, int* __restrict__ s_box,
                                                  uint32_t* __restrict__ bids, uint32_t cap,
                                                  uint32_t* __restrict__ overflow, uint32_t item) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int W = kFwdThreads / 32;
  unsigned bx0 = ns ? (unsigned)x0 : 0xFFFFu, by0 = ns ? (unsigned)y0 : 0xFFFFu;
  unsigned bx1 = ns ? (unsigned)x1 : 0u, by1 = ns ? (unsigned)y1 : 0u;
  bx0 = __reduce_min_sync(0xFFFFFFFFu, bx0);
  by0 = __reduce_min_sync(0xFFFFFFFFu, by0);
  bx1 = __reduce_max_sync(0xFFFFFFFFu, bx1);
  by1 = __reduce_max_sync(0xFFFFFFFFu, by1);
  if (lane == 0) {
    s_box[4 * warp] = (int)bx0;
    s_box[4 * warp + 1] = (int)by0;
    s_box[4 * warp + 2] = (int)bx1;
    s_box[4 * warp + 3] = (int)by1;
  }
  __syncthreads();  // also: every thread is done with what s_cnt held before
  int X0 = s_box[0], Y0 = s_box[1], X1 = s_box[2], Y1 = s_box[3];
#pragma unroll
  for (int w = 1; w < W; ++w) {
    X0 = min(X0, s_box[4 * w]);
    Y0 = min(Y0, s_box[4 * w + 1]);
    X1 = max(X1, s_box[4 * w + 2]);
    Y1 = max(Y1, s_box[4 * w + 3]);
  }
  const int bw = X1 - X0, bh = Y1 - Y0;
  const int w = x1 - x0;
  if (bw <= 0 || bh <= 0 || bw * bh > kCountBox) {  // block-uniform
    for (uint32_t k = 0; k < ns; ++k) {
      const uint32_t t = tile_base + (uint32_t)(y0 + (int)k / w) * (uint32_t)tiles_x + (uint32_t)(x0 + (int)k % w);
      if (bids)
        bucket_put(bids, cap, overflow, t, atomicAdd(&counts[t], 1u), item);
      else
        atomicAdd(&counts[t], 1u);
    }
    __syncthreads();  // s_box is read before the next call rewrites it
    return;
  }
  const int area = bw * bh;
  for (int c = threadIdx.x; c < area; c += kFwdThreads) s_cnt[c] = 0u;
  __syncthreads();
  int tx = x0, ty = y0;
  for (uint32_t k = 0; k < ns; ++k) {
    atomicAdd(&s_cnt[(ty - Y0) * bw + (tx - X0)], 1u);
    if (++tx == x1) {
      tx = x0;
      ++ty;
    }
  }
  __syncthreads();
  for (int c = threadIdx.x; c < area; c += kFwdThreads) {
    const uint32_t v = s_cnt[c];
    if (v) {
      uint32_t* cnt = &counts[tile_base + (uint32_t)(Y0 + c / bw) * (uint32_t)tiles_x + (uint32_t)(X0 + c % bw)];
      if (bids)
        s_cnt[c] = atomicAdd(cnt, v);  // the start of the block's run in the tile's bucket
      else
        atomicAdd(cnt, v);
    }
  }
  __syncthreads();
  if (bids) {
    tx = x0;
    ty = y0;
    for (uint32_t k = 0; k < ns; ++k) {
      bucket_put(bids, cap, overflow, tile_base + (uint32_t)ty * (uint32_t)tiles_x + (uint32_t)tx,
                 atomicAdd(&s_cnt[(ty - Y0) * bw + (tx - X0)], 1u), item);
      if (++tx == x1) {
        tx = x0;
        ++ty;
      }
    }
  }
  __syncthreads();  // s_cnt and s_box are reused by the next view
}

// One thread per Gaussian: its parameters are read once and projected into
// every view of the batch (item v * n + i for view v).
template <int D>
__global__ void __launch_bounds__(kFwdThreads) project_fwd_kernel(const __grid_constant__ ProjectArgs a,
                                                                  float4* __restrict__ feat,
                                                                  uint32_t* __restrict__ depth_key,
                                                                  uint32_t* __restrict__ tiles_touched,
                                                                  ushort4* __restrict__ rects) {
  constexpr int K = (D + 1) * (D + 1);
  constexpr int NS = 3 * K;
  constexpr int RS = (NS % 2 == 0) ? NS + 1 : NS;  // odd row stride: conflict-free per-thread rows
  __shared__ float s_sh[kFwdThreads * RS];
  pdl_enter();
  __shared__ float s_p[kFwdThreads * 11];  // means (3B) | log-scales (3B) | quats (4B) | logits (B)
  if (blockIdx.x == 0) {  // per-pass counters the later kernels accumulate into
    if (a.nvalid && threadIdx.x < (unsigned)a.views) a.nvalid[threadIdx.x] = 0u;
    if (a.cls_count)
      for (int c = threadIdx.x; c < kLenClasses; c += kFwdThreads) a.cls_count[c] = 0u;
    if (a.step_inc && threadIdx.x == 0) *a.step_inc += 1;
  }
  // the block's slices of every parameter array are contiguous: stage them
  // all at once with coalesced asynchronous copies
  const int base = blockIdx.x * kFwdThreads;
  const int cnt = min(kFwdThreads, a.n - base);
  {
    constexpr int B = kFwdThreads;
    const float* src[4] = {a.means + 3 * (size_t)base, a.log_scales + 3 * (size_t)base, a.quats + 4 * (size_t)base,
                           a.logits + (size_t)base};
    const int so[4] = {0, 3 * B, 6 * B, 10 * B};
    const int len[4] = {3 * cnt, 3 * cnt, 4 * cnt, cnt};
#pragma unroll
    for (int r = 0; r < 4; ++r)
      for (int e = threadIdx.x; e < len[r]; e += B) cp_async4(&s_p[so[r] + e], src[r] + e);
    for (int e = threadIdx.x; e < cnt * NS; e += B) {
      const int gi = e / NS;
      cp_async4(&s_sh[gi * RS + (e - gi * NS)], a.sh + (size_t)base * NS + e);
    }
    cp_async_commit();
    cp_async_wait<0>();
  }
  __syncthreads();
  const int i = base + threadIdx.x;
  const bool valid = i < a.n;  // threads without an item stay for the block's tile counting
  __shared__ int s_box[4 * (kFwdThreads / 32)];
  uint32_t* s_cnt = reinterpret_cast<uint32_t*>(s_p);  // s_p is in registers before it is reused
  static_assert(kFwdThreads * 11 >= kCountBox, "the counters fit in the staging buffer");
  const int t = valid ? threadIdx.x : 0;
  const float px = s_p[3 * t], py = s_p[3 * t + 1], pz = s_p[3 * t + 2];
  const float ls[3] = {s_p[3 * kFwdThreads + 3 * t], s_p[3 * kFwdThreads + 3 * t + 1],
                       s_p[3 * kFwdThreads + 3 * t + 2]};
  const float q4[4] = {s_p[6 * kFwdThreads + 4 * t], s_p[6 * kFwdThreads + 4 * t + 1],
                       s_p[6 * kFwdThreads + 4 * t + 2], s_p[6 * kFwdThreads + 4 * t + 3]};
  const float logit = s_p[10 * kFwdThreads + t];
  const float o = 1.f / (1.f + expf(-logit));
  const float log2o = log2f(o);
  // support of the blend test: q <= min(9, 2 ln(o / alpha_min)), widened a
  // little so that float32 rounding of the per-pixel test stays inside
  const float Q = fminf(9.f, 2.f * logf(o / a.alpha_min));
  const float* shp = s_sh + threadIdx.x * RS;

  for (int v = 0; v < a.views; ++v) {
    const CamView& cv = a.cv[v];
    const size_t it = (size_t)v * a.n + i;
    int x0 = 0, y0 = 0, x1 = 0, y1 = 0;
    if (valid) {
    // camera-space position and pixel mean in double-float (the float32 error
    // of W p + t alone would move mu by ~1e-3 px at 1-2 m)
    df Z = df_dot3_plus(cv.R[6], cv.R[7], cv.R[8], px, py, pz, cv.t[2]);
    const float z = Z.hi;
    if (!(z > a.near_z)) {
      depth_key[it] = 0xFFFFFFFFu;
      tiles_touched[it] = 0;
      rects[it] = make_ushort4(0, 0, 0, 0);
      feat[3 * it] = make_float4(0.f, 0.f, 0.f, 0.f);
      feat[3 * it + 1] = make_float4(0.f, 0.f, 0.f, -1e30f);
      feat[3 * it + 2] = make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
      df X = df_dot3_plus(cv.R[0], cv.R[1], cv.R[2], px, py, pz, cv.t[0]);
      df Y = df_dot3_plus(cv.R[3], cv.R[4], cv.R[5], px, py, pz, cv.t[1]);
      df mux = df_add(df_mul_f(df_div(X, Z), cv.fx), df{cv.cx, 0.f});
      df muy = df_add(df_mul_f(df_div(Y, Z), cv.fy), df{cv.cy, 0.f});

      Geo g;
      geometry(cv, a.dilation, px, py, pz, q4, ls, X.hi, Y.hi, z, g);

      if (Q > 0.f && g.det > 0.f) {
        float Qw = Q * 1.0001f + 1e-4f;
        float ex = sqrtf(Qw * g.a) * 1.00001f + 1e-3f;
        float ey = sqrtf(Qw * (g.b * g.b + g.det) / g.a) * 1.00001f + 1e-3f;
        tile_rect(mux.hi, muy.hi, ex, ey, 1.f / (float)a.tile_w, 1.f / (float)a.tile_h, a.tiles_x[v], a.tiles_y[v],
                  x0, y0, x1, y1);
      }
      const uint32_t nt = (uint32_t)(x1 - x0) * (uint32_t)(y1 - y0);
      tiles_touched[it] = nt;
      rects[it] = make_ushort4((unsigned short)x0, (unsigned short)y0, (unsigned short)x1, (unsigned short)y1);
      depth_key[it] = __float_as_uint(z);
      if (nt > kBigTiles) a.big_queue[atomicAdd(a.big_len, 1u)] = (uint32_t)it;

      // view-dependent colour
      float dx = px - cv.C[0], dy = py - cv.C[1], dz = pz - cv.C[2];
      float inv = rsqrtf(dx * dx + dy * dy + dz * dz);
      float Yb[16];
      sh_basis(D, dx * inv, dy * inv, dz * inv, Yb);
      float rgb[3] = {0.5f, 0.5f, 0.5f};
#pragma unroll
      for (int k = 0; k < K; ++k) {
        rgb[0] += Yb[k] * shp[3 * k];
        rgb[1] += Yb[k] * shp[3 * k + 1];
        rgb[2] += Yb[k] * shp[3 * k + 2];
      }
      feat[3 * it] = make_float4(mux.hi, muy.hi, mux.lo, muy.lo);
      feat[3 * it + 1] = make_float4(g.i0, g.k, g.i1, log2o);
      feat[3 * it + 2] = make_float4(fmaxf(rgb[0], 0.f), fmaxf(rgb[1], 0.f), fmaxf(rgb[2], 0.f), z);
    }
    }
    // tile counts: the small rectangles per block in shared memory, each
    // large one (queued above for the scatter) by its whole warp
    if (a.counts) {
      const uint32_t nt = (uint32_t)(x1 - x0) * (uint32_t)(y1 - y0);
      block_count_tiles(a.counts, a.tile_base[v], a.tiles_x[v], x0, y0, x1, y1, nt <= kBigTiles ? nt : 0u, s_cnt,
                        s_box, a.bucket_ids, a.bucket_cap, a.overflow, (uint32_t)it);
      unsigned big = __ballot_sync(0xFFFFFFFFu, nt > kBigTiles);
      const int lane = threadIdx.x & 31;
      while (big) {
        const int src = __ffs(big) - 1;
        big &= big - 1;
        const uint32_t bx = (uint32_t)__shfl_sync(0xFFFFFFFFu, x0, src);
        const uint32_t by = (uint32_t)__shfl_sync(0xFFFFFFFFu, y0, src);
        const uint32_t bw = (uint32_t)__shfl_sync(0xFFFFFFFFu, x1 - x0, src);
        const uint32_t bn = __shfl_sync(0xFFFFFFFFu, nt, src);
        const uint32_t bit = (uint32_t)__shfl_sync(0xFFFFFFFFu, (uint32_t)it, src);
        for (uint32_t k = lane; k < bn; k += 32) {
          const uint32_t t = a.tile_base[v] + (by + k / bw) * (uint32_t)a.tiles_x[v] + bx + k % bw;
          if (a.bucket_ids)
            bucket_put(a.bucket_ids, a.bucket_cap, a.overflow, t, atomicAdd(&a.counts[t], 1u), bit);
          else
            atomicAdd(&a.counts[t], 1u);
        }
      }
    }
  }
}

__global__ void bin_prepare_kernel(int n, const float* __restrict__ mean2d, const float* __restrict__ extent,
                                   const float* __restrict__ depth, float inv_tw, float inv_th, int tiles_x,
                                   int tiles_y, uint32_t* __restrict__ depth_key, uint32_t* __restrict__ tiles,
                                   ushort4* __restrict__ rects, uint32_t* __restrict__ big_queue,
                                   uint32_t* __restrict__ big_len) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int x0, y0, x1, y1;
  tile_rect(mean2d[2 * i], mean2d[2 * i + 1], extent[2 * i], extent[2 * i + 1], inv_tw, inv_th, tiles_x, tiles_y,
            x0, y0, x1, y1);
  const uint32_t nt = (uint32_t)(x1 - x0) * (uint32_t)(y1 - y0);
  tiles[i] = nt;
  rects[i] = make_ushort4((unsigned short)x0, (unsigned short)y0, (unsigned short)x1, (unsigned short)y1);
  depth_key[i] = __float_as_uint(depth[i]);
  if (nt > kBigTiles) big_queue[atomicAdd(big_len, 1u)] = (uint32_t)i;
}

constexpr int kBwdThreads = 128;

// Gradient of one Gaussian's parameters from its gradient record G0..G2
// (the raster backward pass's six exponent / opacity sums, depth, rgb 3),
// plus its share of the pose-twist gradient.  SH gradients are returned in factored form: the
// gradient of coefficient (k, c) is Y[k] * graw[c].
template <int D>
struct GaussGrad {
  float gm[3], gls[3], gq[4], glogit;
  float Y[16], graw[3];
  float pose[6];
};

template <int D>
__device__ __forceinline__ void gaussian_grad(const CamView& cv, float dilation, const float (&p)[3],
                                              const float (&q4)[4], const float (&ls)[3], float logit,
                                              const float* __restrict__ shp, float4 G0, float4 G1, float4 G2,
                                              GaussGrad<D>& out) {
  constexpr int K = (D + 1) * (D + 1);
  float pc[3];
  for (int r = 0; r < 3; ++r) pc[r] = cv.R[3 * r] * p[0] + cv.R[3 * r + 1] * p[1] + cv.R[3 * r + 2] * p[2] + cv.t[r];
  Geo g;
  geometry(cv, dilation, p[0], p[1], p[2], q4, ls, pc[0], pc[1], pc[2], g);
  // The raster backward pass leaves, per Gaussian, sums over its pixels of
  // ga = dL/dalpha * alpha times {t0, t1, t0 dx, t1 dx, t1 w, 1}
  // (q' = t0^2 + t1^2, t0 = i0 dx, t1 = i1 w, w = dy - k dx, dx = u - mu_x,
  // dalpha/dq' = -ln2 alpha, dalpha/do = alpha / o): the gradients of the
  // mean and the factored conic follow with the Gaussian's constants.
  constexpr float kTwoLn2 = 2.f * kLn2;
  const float gmx = kTwoLn2 * (g.i0 * G0.x - g.i1 * g.k * G0.y);
  const float gmy = kTwoLn2 * g.i1 * G0.y;
  const float gi0 = -kTwoLn2 * G0.z;
  const float gk = kTwoLn2 * g.i1 * G0.w;
  const float gi1 = -kTwoLn2 * G1.x;
  const float gdep = G1.z;

  // opacity: dL/do = sum ga / o, d o / d logit = o (1 - o)
  const float o = 1.f / (1.f + expf(-logit));
  out.glogit = G1.y * (1.f - o);

  // colour: SH coefficients and view direction
  float dv[3] = {p[0] - cv.C[0], p[1] - cv.C[1], p[2] - cv.C[2]};
  const float inv = rsqrtf(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
  const float d[3] = {dv[0] * inv, dv[1] * inv, dv[2] * inv};
  sh_basis(D, d[0], d[1], d[2], out.Y);
  float raw[3] = {0.5f, 0.5f, 0.5f};
#pragma unroll
  for (int k = 0; k < K; ++k)
#pragma unroll
    for (int c = 0; c < 3; ++c) raw[c] += out.Y[k] * shp[3 * k + c];
  out.graw[0] = raw[0] > 0.f ? G2.x : 0.f;
  out.graw[1] = raw[1] > 0.f ? G2.y : 0.f;
  out.graw[2] = raw[2] > 0.f ? G2.z : 0.f;
  float cw[16];
#pragma unroll
  for (int k = 0; k < K; ++k)
    cw[k] = shp[3 * k] * out.graw[0] + shp[3 * k + 1] * out.graw[1] + shp[3 * k + 2] * out.graw[2];
  float gd[3];
  sh_basis_vjp(D, d[0], d[1], d[2], cw, gd[0], gd[1], gd[2]);
  const float dd = d[0] * gd[0] + d[1] * gd[1] + d[2] * gd[2];
  const float gv[3] = {(gd[0] - d[0] * dd) * inv, (gd[1] - d[1] * dd) * inv, (gd[2] - d[2] * dd) * inv};
  float gp[3] = {gv[0], gv[1], gv[2]};
  const float gC[3] = {-gv[0], -gv[1], -gv[2]};

  // (i0, k, i1) -> dilated covariance entries (a, b, c)
  const float ga = -gi0 * g.i0 / (2.f * g.a) - gk * g.k / g.a - gi1 * g.i1 * g.b * g.b / (2.f * g.a * g.det);
  const float gb = gk / g.a + gi1 * g.i1 * g.b / g.det;
  const float gc = -gi1 * g.i1 * g.a / (2.f * g.det);
  // covariance = M M^T + dil I, rows m0, m1 of M = J A
  float Gm0[3], Gm1[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    Gm0[c] = 2.f * ga * g.m0[c] + gb * g.m1[c];
    Gm1[c] = gb * g.m0[c] + 2.f * gc * g.m1[c];
  }
  float gj00 = 0.f, gj02 = 0.f, gj11 = 0.f, gj12 = 0.f;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    gj00 += Gm0[c] * g.A[0][c];
    gj02 += Gm0[c] * g.A[2][c];
    gj11 += Gm1[c] * g.A[1][c];
    gj12 += Gm1[c] * g.A[2][c];
  }
  float GA[3][3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    GA[0][c] = g.j00 * Gm0[c];
    GA[1][c] = g.j11 * Gm1[c];
    GA[2][c] = g.j02 * Gm0[c] + g.j12 * Gm1[c];
  }
  // J and the mean -> camera-space position
  const float rz = g.rz, rz2 = rz * rz, rz3 = rz2 * rz;
  float gpc[3] = {0.f, 0.f, 0.f};
  gpc[2] += -cv.fx * rz2 * gj00 - cv.fy * rz2 * gj11;
  if (!g.cx_) {
    gpc[0] += -cv.fx * rz2 * gj02;
    gpc[2] += 2.f * cv.fx * g.x * rz3 * gj02;
  } else {
    gpc[2] += cv.fx * g.xt * rz3 * gj02;
  }
  if (!g.cy_) {
    gpc[1] += -cv.fy * rz2 * gj12;
    gpc[2] += 2.f * cv.fy * g.y * rz3 * gj12;
  } else {
    gpc[2] += cv.fy * g.yt * rz3 * gj12;
  }
  gpc[0] += gmx * cv.fx * rz;
  gpc[1] += gmy * cv.fy * rz;
  gpc[2] += -(gmx * cv.fx * g.x + gmy * cv.fy * g.y) * rz2 + gdep;

  // A = W B, B = Rq diag(s)
  float GW[3][3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) GW[r][c] = GA[r][0] * g.B[c][0] + GA[r][1] * g.B[c][1] + GA[r][2] * g.B[c][2];
  float GR[3][3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float gs_ = 0.f;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const float GBrc = cv.R[r] * GA[0][c] + cv.R[3 + r] * GA[1][c] + cv.R[6 + r] * GA[2][c];  // (W^T GA)[r][c]
      GR[r][c] = GBrc * g.s[c];
      gs_ += GBrc * g.Rq[r][c];
    }
    out.gls[c] = gs_ * g.s[c];
  }
  // rotation matrix -> normalised quaternion -> raw quaternion
  const float w = g.qn[0], x = g.qn[1], y = g.qn[2], z = g.qn[3];
  float gqn[4];
  gqn[0] = 2.f * (-z * GR[0][1] + y * GR[0][2] + z * GR[1][0] - x * GR[1][2] - y * GR[2][0] + x * GR[2][1]);
  gqn[1] = 2.f * (y * GR[0][1] + z * GR[0][2] + y * GR[1][0] - 2.f * x * GR[1][1] - w * GR[1][2] + z * GR[2][0] +
                  w * GR[2][1] - 2.f * x * GR[2][2]);
  gqn[2] = 2.f * (-2.f * y * GR[0][0] + x * GR[0][1] + w * GR[0][2] + x * GR[1][0] + z * GR[1][2] - w * GR[2][0] +
                  z * GR[2][1] - 2.f * y * GR[2][2]);
  gqn[3] = 2.f * (-2.f * z * GR[0][0] - w * GR[0][1] + x * GR[0][2] + w * GR[1][0] - 2.f * z * GR[1][1] +
                  y * GR[1][2] + x * GR[2][0] + y * GR[2][1]);
  const float dq = g.qn[0] * gqn[0] + g.qn[1] * gqn[1] + g.qn[2] * gqn[2] + g.qn[3] * gqn[3];
#pragma unroll
  for (int j = 0; j < 4; ++j) out.gq[j] = (gqn[j] - g.qn[j] * dq) / g.qlen;

  // p_c = W p + t
#pragma unroll
  for (int c = 0; c < 3; ++c) gp[c] += cv.R[c] * gpc[0] + cv.R[3 + c] * gpc[1] + cv.R[6 + c] * gpc[2];
#pragma unroll
  for (int c = 0; c < 3; ++c) out.gm[c] = gp[c];

  // pose: total dL/dW and dL/dt of this Gaussian, then the left-perturbation twist
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) GW[r][c] += gpc[r] * p[c] - cv.t[r] * gC[c];
  float gt[3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
    gt[r] = gpc[r] - (cv.R[3 * r] * gC[0] + cv.R[3 * r + 1] * gC[1] + cv.R[3 * r + 2] * gC[2]);
  float Am[3][3];  // GW W^T
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      Am[r][c] = GW[r][0] * cv.R[3 * c] + GW[r][1] * cv.R[3 * c + 1] + GW[r][2] * cv.R[3 * c + 2];
  out.pose[0] = gt[0];
  out.pose[1] = gt[1];
  out.pose[2] = gt[2];
  out.pose[3] = Am[2][1] - Am[1][2] + (cv.t[1] * gt[2] - cv.t[2] * gt[1]);
  out.pose[4] = Am[0][2] - Am[2][0] + (cv.t[2] * gt[0] - cv.t[0] * gt[2]);
  out.pose[5] = Am[1][0] - Am[0][1] + (cv.t[0] * gt[1] - cv.t[1] * gt[0]);
}

__device__ __forceinline__ bool nonzero_record(const float4& G0, const float4& G1, const float4& G2) {
  return (G0.x != 0.f) | (G0.y != 0.f) | (G0.z != 0.f) | (G0.w != 0.f) | (G1.x != 0.f) | (G1.y != 0.f) |
         (G1.z != 0.f) | (G2.x != 0.f) | (G2.y != 0.f) | (G2.z != 0.f);
}

// The consumer of a gradient record leaves it zero for the next backward
// pass (the raster backward pass only adds to records).
__device__ __forceinline__ void zero_record(float4* rec) {
  const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
  rec[0] = z;
  rec[1] = z;
  rec[2] = z;
}

// deterministic per-block sum of the pose gradient into out[0..5]; every
// thread of the block calls it
__device__ __forceinline__ void block_pose_partial(const float (&pose)[6], float* __restrict__ out) {
  __shared__ float red[kBwdThreads / 32][6];  // blocks of up to kBwdThreads threads
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
  __syncthreads();  // an earlier call is done reading red
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    float v = pose[k];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (lane == 0) red[wid][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    float s = 0.f;
    for (int w = 0; w < nw; ++w) s += red[w][threadIdx.x];
    out[threadIdx.x] = s;
  }
}

// One thread per Gaussian: the gradient records of its items in every view
// are turned into parameter gradients, summed over the views and added to
// the gradient arrays.
template <int D>
__global__ void __launch_bounds__(kBwdThreads) project_bwd_kernel(const __grid_constant__ ProjectArgs a,
                                                                  float4* __restrict__ g2d,
                                                                  float* __restrict__ gm, float* __restrict__ gls,
                                                                  float* __restrict__ gq, float* __restrict__ glog,
                                                                  float* __restrict__ gsh,
                                                                  float* __restrict__ pose_partials) {
  pdl_enter();
  constexpr int K = (D + 1) * (D + 1);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = i < a.n;
  float p[3] = {0.f, 0.f, 0.f}, q4[4] = {1.f, 0.f, 0.f, 0.f}, ls[3] = {0.f, 0.f, 0.f}, logit = 0.f;
  if (live) {
    for (int c = 0; c < 3; ++c) {
      p[c] = a.means[3 * i + c];
      ls[c] = a.log_scales[3 * i + c];
    }
    for (int j = 0; j < 4; ++j) q4[j] = a.quats[4 * i + j];
    logit = a.logits[i];
  }
  float am[3] = {0.f, 0.f, 0.f}, als[3] = {0.f, 0.f, 0.f}, aq[4] = {0.f, 0.f, 0.f, 0.f}, alog = 0.f;
  bool any = false;
  for (int v = 0; v < a.views; ++v) {
    float pose[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (live) {
      const size_t it = (size_t)v * a.n + i;
      const float4 G0 = g2d[3 * it], G1 = g2d[3 * it + 1], G2 = g2d[3 * it + 2];
      if (nonzero_record(G0, G1, G2)) {
        zero_record(g2d + 3 * it);
        any = true;
        GaussGrad<D> gg;
        gaussian_grad<D>(a.cv[v], a.dilation, p, q4, ls, logit, a.sh + (size_t)i * K * 3, G0, G1, G2, gg);
        alog += gg.glogit;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          am[c] += gg.gm[c];
          als[c] += gg.gls[c];
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) aq[j] += gg.gq[j];
        float* gshp = gsh + (size_t)i * K * 3;
#pragma unroll
        for (int k = 0; k < K; ++k)
#pragma unroll
          for (int c = 0; c < 3; ++c) gshp[3 * k + c] += gg.Y[k] * gg.graw[c];
#pragma unroll
        for (int k = 0; k < 6; ++k) pose[k] = gg.pose[k];
      }
    }
    if (pose_partials) block_pose_partial(pose, pose_partials + ((size_t)blockIdx.x * a.views + v) * 6);
  }
  if (live && any) {
    glog[i] += alog;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      gm[3 * i + c] += am[c];
      gls[3 * i + c] += als[c];
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) gq[4 * i + j] += aq[j];
  }
}

// Bias corrections from the device step counter: 1 - beta^t = -expm1(t log beta),
// accurate also for small t where 1 - powf(beta, t) would cancel.
__device__ __forceinline__ void device_bias_corrections(AdamArgs& ad) {
  if (!ad.step_dev) return;
  const float t = (float)*ad.step_dev;
  ad.step_scale = 1.f / -expm1f(t * ad.log_beta1);
  ad.inv_sqrt_bc2 = rsqrtf(-expm1f(t * ad.log_beta2));
}

__global__ void step_increment_kernel(long long* step) {
  pdl_enter();
  *step += 1;
}

__device__ __forceinline__ void adam_update(float& p, float g, float& m, float& v, float lr, const AdamArgs& ad) {
  adam_apply(p, g, m, v, lr, ad.beta1, ad.beta2, ad.eps, ad.step_scale, ad.inv_sqrt_bc2);
}

// Backward of the projection fused with the Adam step, for one optimisation
// iteration on a batch of views.  A block (one warp) owns 32 consecutive
// Gaussians:
//   1. its slices of the parameter array and of the two Adam moments (each
//      slice contiguous in the flat layout) are copied to shared memory with
//      cp.async, the parameters as a first group and the moments as a second,
//      so the moment loads stay in flight during step 2;
//   2. one thread per Gaussian turns its gradient records (one per view)
//      into parameter gradients summed over the views, kept in shared memory;
//   3. coalesced sweeps apply Adam to every float and store p, m, v.
// No gradient buffer is written or read.  With one view the SH gradient is
// kept in factored form (Y_k * graw_c) and the SH moments are staged too;
// with several views the SH gradients are summed in shared memory rows and
// the SH moments are staged as well, beside the summed rows.  Blocks of one
// warp (27 KB for one view, 8 blocks per SM) let the staging, gradient and
// sweep phases of different blocks overlap.
template <bool MULTI>
constexpr int fused_threads() { return 32; }
static_assert(fused_threads<false>() == 32 && fused_threads<true>() == 32,
              "the fused loss reduction takes one warp per block");

template <int D>
struct FusedSmem {
  static constexpr int K = (D + 1) * (D + 1);
  static constexpr int NS = 3 * K;
  static constexpr int RS = (NS % 2 == 0) ? NS + 1 : NS;  // odd row stride: conflict-free per-thread rows
  static constexpr int B = fused_threads<false>();
  float p[B * 11], m[B * 11], v[B * 11];  // means (3B) | log-scales (3B) | quats (4B) | logits (B)
  float g[B * 11];                        // gradients, same layout
  float sp[B * RS], sm[B * NS + 4], sv[B * NS + 4];  // SH moments at their slice's offset within 16 B
  float Y[B][K + 1];
  float graw[B][4];
};

template <int D>
struct FusedSmemMulti {
  static constexpr int K = (D + 1) * (D + 1);
  static constexpr int NS = 3 * K;
  static constexpr int RS = (NS % 2 == 0) ? NS + 1 : NS;
  static constexpr int B = fused_threads<true>();
  float p[B * 11], m[B * 11], v[B * 11];
  float g[B * 11];
  float sp[B * RS];  // SH parameters, one row per Gaussian
  float gs[B * RS];  // SH gradients summed over the views, same rows
  float sm[B * NS + 4], sv[B * NS + 4];  // SH moments
};

// The training step's loss reduction (see LossFoldArgs), by one warp per
// reduction block: kLossChunk / 32 partials per lane in a fixed order, then
// over the warp; the warp completing the last block sums the blocks per
// view (per lane, then over the warp).  Warp-uniform.
__device__ __forceinline__ void fused_loss_reduce(const LossFoldArgs& L) {
  const int lane = threadIdx.x & 31;
  for (int lb = blockIdx.x; lb < L.blocks; lb += gridDim.x) {
    int v = 0;
    for (int k = 1; k < L.views; ++k)
      if (lb >= L.block_base[k]) v = k;
    const uint32_t lo = L.job_base[v] + (uint32_t)(lb - L.block_base[v]) * kLossChunk;
    const uint32_t hi = min(lo + (uint32_t)kLossChunk, L.job_base[v + 1]);
    float sc = 0.f, sd = 0.f, nv = 0.f;
#pragma unroll 8
    for (uint32_t i = lo + lane; i < hi; i += 32) {
      sc += L.partials[3 * (size_t)i];
      sd += L.partials[3 * (size_t)i + 1];
      nv += L.partials[3 * (size_t)i + 2];
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      sc += __shfl_xor_sync(0xFFFFFFFFu, sc, off);
      sd += __shfl_xor_sync(0xFFFFFFFFu, sd, off);
      nv += __shfl_xor_sync(0xFFFFFFFFu, nv, off);
    }
    uint32_t last = 0u;
    if (lane == 0) {
      L.blk[3 * lb] = sc;
      L.blk[3 * lb + 1] = sd;
      L.blk[3 * lb + 2] = nv;
      __threadfence();  // this block's sums are visible before its ticket
      last = atomicAdd(L.ticket, 1u) == (uint32_t)L.blocks - 1u ? 1u : 0u;
    }
    if (!__shfl_sync(0xFFFFFFFFu, last, 0)) continue;
    __threadfence();
    float total = 0.f;
    for (int w = 0; w < L.views; ++w) {
      float s0 = 0.f, s1 = 0.f, s2 = 0.f;
      for (int b = L.block_base[w] + lane; b < L.block_base[w + 1]; b += 32) {
        s0 += __ldcg(&L.blk[3 * b]);
        s1 += __ldcg(&L.blk[3 * b + 1]);
        s2 += __ldcg(&L.blk[3 * b + 2]);
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        s0 += __shfl_xor_sync(0xFFFFFFFFu, s0, off);
        s1 += __shfl_xor_sync(0xFFFFFFFFu, s1, off);
        s2 += __shfl_xor_sync(0xFFFFFFFFu, s2, off);
      }
      const float nvw = s2 > 0.f ? s2 : 1.f;
      total += L.w_color * s0 / (3.f * L.npix[w]) + L.w_depth * s1 / nvw;
      if (lane == 0) L.scale[w] = L.w_depth / nvw;
    }
    if (lane == 0) {
      *L.out = total;
      *L.ticket = 0u;
    }
  }
}

template <int D, bool MULTI>
__global__ void __launch_bounds__(fused_threads<MULTI>()) project_bwd_adam_kernel(const __grid_constant__ ProjectArgs a,
                                                                         float4* __restrict__ g2d,
                                                                         float* __restrict__ P, float* __restrict__ M,
                                                                         float* __restrict__ V, AdamArgs ad,
                                                                         float* __restrict__ pose_partials,
                                                                         const __grid_constant__ LossFoldArgs L) {
  pdl_enter();
  if (L.out && threadIdx.x < 32) fused_loss_reduce(L);  // blocks of one warp: the whole block
  device_bias_corrections(ad);
  using S = typename std::conditional<MULTI, FusedSmemMulti<D>, FusedSmem<D>>::type;
  constexpr int K = S::K, NS = S::NS, RS = S::RS, B = S::B;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  S& sm = *reinterpret_cast<S*>(smem_raw);
  const int64_t N = a.n;
  const int base = blockIdx.x * B;
  const int cnt = min(B, a.n - base);
  const int t = threadIdx.x;
  const int64_t g0[4] = {3 * (int64_t)base, 3 * N + 3 * (int64_t)base, 6 * N + 4 * (int64_t)base, 10 * N + base};
  const int so[4] = {0, 3 * B, 6 * B, 10 * B};
  const int len[4] = {3 * cnt, 3 * cnt, 4 * cnt, cnt};
  const int64_t gsh = 11 * N + (int64_t)base * NS;

  // 1. asynchronous staging: parameters (group 0), then Adam moments (group 1)
#pragma unroll
  for (int r = 0; r < 4; ++r)
    for (int e = t; e < len[r]; e += B) cp_async4(&sm.p[so[r] + e], P + g0[r] + e);
  for (int e = t; e < cnt * NS; e += B) {
    const int gi = e / NS;
    cp_async4(&sm.sp[gi * RS + (e - gi * NS)], P + gsh + e);
  }
  cp_async_commit();
#pragma unroll
  for (int r = 0; r < 4; ++r)
    for (int e = t; e < len[r]; e += B) {
      cp_async4(&sm.m[so[r] + e], M + g0[r] + e);
      cp_async4(&sm.v[so[r] + e], V + g0[r] + e);
    }
  // SH moments: 16-byte copies over the 16-byte aligned interior of each
  // slice, staged at the slice's own offset within 16 bytes (shM, shV)
  const int shM = (int)(((uintptr_t)(M + gsh) >> 2) & 3u), shV = (int)(((uintptr_t)(V + gsh) >> 2) & 3u);
  stage_slice16(sm.sm, M + gsh, cnt * NS, shM, t, B);
  stage_slice16(sm.sv, V + gsh, cnt * NS, shV, t, B);
  cp_async_commit();
  float4 G0 = make_float4(0.f, 0.f, 0.f, 0.f), G1 = G0, G2 = G0;
  if (t < cnt) {
    const int64_t i = base + t;
    G0 = g2d[3 * i];
    G1 = g2d[3 * i + 1];
    G2 = g2d[3 * i + 2];
    if (nonzero_record(G0, G1, G2)) zero_record(g2d + 3 * i);
  }
  cp_async_wait<1>();
  __syncthreads();

  // 2. per-Gaussian gradients
  float pq[3], ls[3], q4[4];
  if (t < cnt) {
    for (int c = 0; c < 3; ++c) {
      pq[c] = sm.p[3 * t + c];
      ls[c] = sm.p[3 * B + 3 * t + c];
    }
    for (int j = 0; j < 4; ++j) q4[j] = sm.p[6 * B + 4 * t + j];
  }
  float am[3] = {0.f, 0.f, 0.f}, als[3] = {0.f, 0.f, 0.f}, aq[4] = {0.f, 0.f, 0.f, 0.f}, alog = 0.f;
  if constexpr (MULTI) {
    if (t < cnt)
      for (int e = 0; e < NS; ++e) sm.gs[t * RS + e] = 0.f;
  }
  for (int v = 0; v < (MULTI ? a.views : 1); ++v) {  // the one-view variant runs for one view only
    float pose[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (t < cnt) {
      if (v > 0) {
        const int64_t it = (int64_t)v * N + base + t;
        G0 = g2d[3 * it];
        G1 = g2d[3 * it + 1];
        G2 = g2d[3 * it + 2];
        if (nonzero_record(G0, G1, G2)) zero_record(g2d + 3 * it);
      }
      GaussGrad<D> gg;
      const bool nz = nonzero_record(G0, G1, G2);
      if (nz) {
        gaussian_grad<D>(a.cv[v], a.dilation, pq, q4, ls, sm.p[10 * B + t], sm.sp + t * RS, G0, G1, G2, gg);
        alog += gg.glogit;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          am[c] += gg.gm[c];
          als[c] += gg.gls[c];
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) aq[j] += gg.gq[j];
#pragma unroll
        for (int k = 0; k < 6; ++k) pose[k] = gg.pose[k];
      }
      if constexpr (MULTI) {
        if (nz) {
#pragma unroll
          for (int k = 0; k < K; ++k)
#pragma unroll
            for (int c = 0; c < 3; ++c) sm.gs[t * RS + 3 * k + c] += gg.Y[k] * gg.graw[c];
        }
      } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) sm.graw[t][c] = nz ? gg.graw[c] : 0.f;
#pragma unroll
        for (int k = 0; k < K; ++k) sm.Y[t][k] = nz ? gg.Y[k] : 0.f;
      }
    }
    if (pose_partials) block_pose_partial(pose, pose_partials + ((size_t)blockIdx.x * a.views + v) * 6);
  }
  if (t < cnt) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      sm.g[3 * t + c] = am[c];
      sm.g[3 * B + 3 * t + c] = als[c];
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) sm.g[6 * B + 4 * t + j] = aq[j];
    sm.g[10 * B + t] = alog;
  }
  cp_async_wait<0>();
  __syncthreads();

  // 3. Adam sweeps (dense: zero gradients still update the moments)
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const float lr = ad.lr[r];
    for (int e = t; e < len[r]; e += B) {
      const int l = so[r] + e;
      float p = sm.p[l], m = sm.m[l], v = sm.v[l];
      adam_update(p, sm.g[l], m, v, lr, ad);
      const int64_t f = g0[r] + e;
      P[f] = p;
      M[f] = m;
      V[f] = v;
    }
  }
  if constexpr (B == 32) {
    // a warp per block: walk the SH rows, lane t on columns t, t + 32, ...
    // (coalesced rows, and each lane's coefficient (k, c) fixed per column)
#pragma unroll
    for (int c0 = 0; c0 < NS; c0 += B) {
      const int rr = c0 + t;
      if (rr < NS) {
        const int k = rr / 3, c = rr - 3 * k;
        const float lr = k == 0 ? ad.lr[4] : ad.lr[5];
        for (int gi = 0; gi < cnt; ++gi) {
          const int e = gi * NS + rr;
          float p = sm.sp[gi * RS + rr], m = sm.sm[shM + e], v = sm.sv[shV + e];
          float g;
          if constexpr (MULTI)
            g = sm.gs[gi * RS + rr];
          else
            g = sm.Y[gi][k] * sm.graw[gi][c];
          adam_update(p, g, m, v, lr, ad);
          const int64_t f = gsh + e;
          P[f] = p;
          M[f] = m;
          V[f] = v;
        }
      }
    }
  } else {
    for (int e = t; e < cnt * NS; e += B) {
      const int gi = e / NS, rr = e - gi * NS;
      const int k = rr / 3, c = rr - 3 * k;
      const int64_t f = gsh + e;
      float p = sm.sp[gi * RS + rr], m = sm.sm[shM + e], v = sm.sv[shV + e], g;
      if constexpr (MULTI)
        g = sm.gs[gi * RS + rr];
      else
        g = sm.Y[gi][k] * sm.graw[gi][c];
      adam_update(p, g, m, v, k == 0 ? ad.lr[4] : ad.lr[5], ad);
      P[f] = p;
      M[f] = m;
      V[f] = v;
    }
  }
}

// one block per view: dL_dpose[v] += sum over blocks b of partials[b][v]
__global__ void pose_reduce_kernel(const float* __restrict__ partials, int nblocks, int views,
                                   float* __restrict__ out) {
  __shared__ float red[32][6];
  const int v = blockIdx.x;
  float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
    for (int k = 0; k < 6; ++k) acc[k] += partials[((size_t)b * views + v) * 6 + k];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int k = 0; k < 6; ++k) {
    float x = acc[k];
    for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
    if (lane == 0) red[wid][k] = x;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    float s = 0.f;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) s += red[w][threadIdx.x];
    out[6 * v + threadIdx.x] += s;
  }
}

}  // namespace

void launch_project_fwd(const ProjectArgs& a, float4* feat, uint32_t* depth_key, uint32_t* tiles_touched,
                        ushort4* rects, cudaStream_t s) {
  if (a.n <= 0) return;
  const int nb = (a.n + kFwdThreads - 1) / kFwdThreads;
  switch (a.sh_degree) {
    case 0: launch_pdl(project_fwd_kernel<0>, nb, kFwdThreads, 0, s, a, feat, depth_key, tiles_touched, rects); break;
    case 1: launch_pdl(project_fwd_kernel<1>, nb, kFwdThreads, 0, s, a, feat, depth_key, tiles_touched, rects); break;
    case 2: launch_pdl(project_fwd_kernel<2>, nb, kFwdThreads, 0, s, a, feat, depth_key, tiles_touched, rects); break;
    default: launch_pdl(project_fwd_kernel<3>, nb, kFwdThreads, 0, s, a, feat, depth_key, tiles_touched, rects); break;
  }
}

void launch_bin_prepare(int n, const float* mean2d, const float* extent, const float* depth, int tile_w, int tile_h,
                        int tiles_x, int tiles_y, uint32_t* depth_key, uint32_t* tiles_touched, ushort4* rects,
                        uint32_t* big_queue, uint32_t* big_len, cudaStream_t s) {
  if (n <= 0) return;
  bin_prepare_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, mean2d, extent, depth, 1.f / (float)tile_w,
                                                     1.f / (float)tile_h, tiles_x, tiles_y, depth_key,
                                                     tiles_touched, rects, big_queue, big_len);
}

int project_bwd_blocks(int n) { return n > 0 ? (n + kBwdThreads - 1) / kBwdThreads : 0; }

int launch_project_bwd(const ProjectArgs& a, float4* g2d, float* g_means, float* g_log_scales, float* g_quats,
                       float* g_logits, float* g_sh, float* pose_partials, cudaStream_t s) {
  const int nb = project_bwd_blocks(a.n);
  if (nb == 0) return 0;
  switch (a.sh_degree) {
    case 0: launch_pdl(project_bwd_kernel<0>, nb, kBwdThreads, 0, s, a, g2d, g_means, g_log_scales, g_quats, g_logits, g_sh, pose_partials); break;
    case 1: launch_pdl(project_bwd_kernel<1>, nb, kBwdThreads, 0, s, a, g2d, g_means, g_log_scales, g_quats, g_logits, g_sh, pose_partials); break;
    case 2: launch_pdl(project_bwd_kernel<2>, nb, kBwdThreads, 0, s, a, g2d, g_means, g_log_scales, g_quats, g_logits, g_sh, pose_partials); break;
    default: launch_pdl(project_bwd_kernel<3>, nb, kBwdThreads, 0, s, a, g2d, g_means, g_log_scales, g_quats, g_logits, g_sh, pose_partials); break;
  }
  return nb;
}

int launch_project_bwd_adam(const ProjectArgs& a, float4* g2d, float* params, float* m, float* v,
                            const AdamArgs& ad, float* pose_partials, cudaStream_t s, const LossFoldArgs* loss) {
  if (a.n <= 0) return 0;
  const int bt = a.views == 1 ? fused_threads<false>() : fused_threads<true>();
  const int nb = (a.n + bt - 1) / bt;
  LossFoldArgs L{};
  if (loss) L = *loss;
#define GS_FUSED(D_, M_, S_)                                                                                  \
  launch_pdl(project_bwd_adam_kernel<D_, M_>, nb, fused_threads<M_>(), sizeof(S_<D_>), s, a, g2d, params, m, v, ad, \
             pose_partials, L)
  if (a.views == 1) {
    switch (a.sh_degree) {
      case 0: GS_FUSED(0, false, FusedSmem); break;
      case 1: GS_FUSED(1, false, FusedSmem); break;
      case 2: GS_FUSED(2, false, FusedSmem); break;
      default: GS_FUSED(3, false, FusedSmem); break;
    }
  } else {
    switch (a.sh_degree) {
      case 0: GS_FUSED(0, true, FusedSmemMulti); break;
      case 1: GS_FUSED(1, true, FusedSmemMulti); break;
      case 2: GS_FUSED(2, true, FusedSmemMulti); break;
      default: GS_FUSED(3, true, FusedSmemMulti); break;
    }
  }
#undef GS_FUSED
  return nb;
}

void init_project_kernels() {
#define GS_ATTR(D_, M_, S_)                                                                           \
  cudaFuncSetAttribute(project_bwd_adam_kernel<D_, M_>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                       (int)sizeof(S_<D_>))
  GS_ATTR(0, false, FusedSmem);
  GS_ATTR(1, false, FusedSmem);
  GS_ATTR(2, false, FusedSmem);
  GS_ATTR(3, false, FusedSmem);
  GS_ATTR(0, true, FusedSmemMulti);
  GS_ATTR(1, true, FusedSmemMulti);
  GS_ATTR(2, true, FusedSmemMulti);
  GS_ATTR(3, true, FusedSmemMulti);
#undef GS_ATTR
}

void launch_step_increment(long long* step, cudaStream_t s) { launch_pdl(step_increment_kernel, 1, 1, 0, s, step); }

void launch_pose_reduce(const float* partials, int nblocks, int views, float* dL_dpose, cudaStream_t s) {
  if (nblocks <= 0 || views <= 0) return;
  pose_reduce_kernel<<<views, 256, 0, s>>>(partials, nblocks, views, dL_dpose);
}

}  // namespace gs
