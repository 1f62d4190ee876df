// Shared device helpers of the GB300 Gaussian-splatting path: constants,
// the projected-feature layout, double-float arithmetic, the real SH basis,
// hardware exp2 / reciprocal and the warp-aggregated counter increment.
#pragma once

#include <cstdint>
#include <utility>

#include <cuda_runtime.h>

namespace gs {

// ---------------------------------------------------------------------------
// Projected feature record, 3 x float4 = 48 B per Gaussian (written by the
// projection kernel, gathered by the raster kernels):
//   f0 = {mu_x_hi, mu_y_hi, mu_x_lo, mu_y_lo}   double-float pixel mean
//   f1 = {i0, k, i1, log2(opacity)}             factored inverse covariance
//   f2 = {r, g, b, z}                           decoded colour, camera depth
// The 2D Gaussian exponent is evaluated as
//   q' = (i0 dx)^2 + (i1 (dy - k dx))^2 = 0.5 log2(e) * (u - mu)^T Sigma^-1 (u - mu)
// with i0 = S / sqrt(a), k = b / a, i1 = S sqrt(a / det), S^2 = 0.5 log2(e),
// for the dilated covariance [[a, b], [b, c]] (Eq. 5).  This is a Cholesky
// factorisation of the conic: a sum of two squares, so q' keeps full float32
// relative accuracy even for very elongated splats, where the usual
// a dx^2 + 2 b dx dy + c dy^2 form cancels.  exp(-q/2) becomes 2^(-q').
// ---------------------------------------------------------------------------
constexpr float kS2 = 0.8493218002880191f;        // sqrt(0.5 * log2(e))
constexpr float kHalfLog2e = 0.7213475204444817f;  // 0.5 * log2(e)
constexpr float kLn2 = 0.6931471805599453f;

// Real SH basis constants (Condon-Shortley phase), from
//   Y_{l,+-m} = sqrt(2 - [m==0]) K_l^m (-1)^m (d^m P_l / dz^m)(z) {Re,Im}(x + i y)^m,
//   K_l^m = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!), with the Legendre derivative
//   factors folded in.
constexpr float kSH0 = 0.28209479177387814f;   // K_0^0
constexpr float kSH1 = 0.4886025119029199f;    // sqrt(3 / (4 pi))
constexpr float kSH20 = 0.31539156525252005f;  // K_2^0 / 2          * (3z^2 - 1)
constexpr float kSH21 = 1.0925484305920792f;   // 3 sqrt(2) K_2^1     * z {x, y}
constexpr float kSH22 = 0.5462742152960396f;   // 3 sqrt(2) K_2^2     * (x^2 - y^2), 2xy
constexpr float kSH30 = 0.3731763325901154f;   // K_3^0 / 2          * (5z^3 - 3z)
constexpr float kSH31 = 0.4570457994644658f;   // 1.5 sqrt(2) K_3^1   * (5z^2 - 1) {x, y}
constexpr float kSH32 = 1.4453057213202773f;   // 15 sqrt(2) K_3^2    * z (x^2 - y^2), 2xyz
constexpr float kSH33 = 0.5900435899266436f;   // 15 sqrt(2) K_3^3    * (x^3 - 3xy^2), (3x^2y - y^3)

struct RasterParams {
  int width, height, tile_w, tile_h, tiles_x, tiles_y;
  float bg[3];
  float alpha_max;
  float log2_alpha_min;  // log2(alpha_min)
  float qmax_s;          // 9 * 0.5 log2(e): the 3-sigma bound on q'
  float t_eps;
};

// ---------------------------------------------------------------------------
// double-float helpers (error-free transformations, no contraction)
// ---------------------------------------------------------------------------
struct df {
  float hi, lo;
};

__device__ __forceinline__ df df_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, err};
}
__device__ __forceinline__ df df_fast_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df df_two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ df df_add(df a, df b) {
  df s = df_two_sum(a.hi, b.hi);
  float lo = __fadd_rn(__fadd_rn(a.lo, b.lo), s.lo);
  return df_fast_two_sum(s.hi, lo);
}
__device__ __forceinline__ df df_mul_f(df a, float b) {
  df p = df_two_prod(a.hi, b);
  return df_fast_two_sum(p.hi, __fmaf_rn(a.lo, b, p.lo));
}
__device__ __forceinline__ df df_div(df a, df b) {
  float q1 = __fdiv_rn(a.hi, b.hi);
  df r = df_add(a, df_mul_f(b, -q1));
  float q2 = __fdiv_rn(r.hi, b.hi);
  return df_fast_two_sum(q1, q2);
}
// sum_j W[j] * p[j] + t, exactly rounded to double-float
__device__ __forceinline__ df df_dot3_plus(float w0, float w1, float w2, float p0, float p1, float p2, float t) {
  df acc = df_two_prod(w0, p0);
  acc = df_add(acc, df_two_prod(w1, p1));
  acc = df_add(acc, df_two_prod(w2, p2));
  return df_add(acc, df{t, 0.f});
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// sqrt(x) by the hardware approximation (PTX sqrt.approx, about 1 ulp).
__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// One Adam update of one float, shared by every Adam kernel so that the
// fused and the standalone updates agree bit for bit:
//   m = b1 m + (1 - b1) g,  v = b2 v + (1 - b2) g^2,
//   p -= lr ss m / (sqrt(v) isb2 + eps),  ss = 1 / (1 - b1^t), isb2 = 1 / sqrt(1 - b2^t).
// The square root and the division are the hardware approximations (within
// 2 ulp; the denominator is at least eps, a normal number).
__device__ __forceinline__ void adam_apply(float& p, float g, float& m, float& v, float lr, float b1, float b2,
                                           float eps, float ss, float isb2) {
  m = b1 * m + (1.f - b1) * g;
  v = b2 * v + (1.f - b2) * g * g;
  p -= __fdividef(lr * ss * m, sqrt_approx(v) * isb2 + eps);
}

// 1 / x by the hardware reciprocal (PTX rcp.approx: relative error within
// 2^-23 for normal x), one instruction instead of the IEEE-rounded
// division sequence; used where x is a normal number far from overflow.
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// ---------------------------------------------------------------------------
// real SH basis up to degree 3 (16 values) and its gradient w.r.t. the
// (unnormalised-treated) direction components
// ---------------------------------------------------------------------------
__device__ __forceinline__ void sh_basis(int deg, float x, float y, float z, float* Y) {
  Y[0] = kSH0;
  if (deg < 1) return;
  Y[1] = -kSH1 * y;
  Y[2] = kSH1 * z;
  Y[3] = -kSH1 * x;
  if (deg < 2) return;
  float xx = x * x, yy = y * y, zz = z * z;
  Y[4] = 2.f * kSH22 * x * y;
  Y[5] = -kSH21 * y * z;
  Y[6] = kSH20 * (3.f * zz - 1.f);
  Y[7] = -kSH21 * x * z;
  Y[8] = kSH22 * (xx - yy);
  if (deg < 3) return;
  Y[9] = -kSH33 * (3.f * xx * y - yy * y);
  Y[10] = 2.f * kSH32 * x * y * z;
  Y[11] = -kSH31 * y * (5.f * zz - 1.f);
  Y[12] = kSH30 * (5.f * zz * z - 3.f * z);
  Y[13] = -kSH31 * x * (5.f * zz - 1.f);
  Y[14] = kSH32 * z * (xx - yy);
  Y[15] = -kSH33 * (xx * x - 3.f * x * yy);
}

// d/d(x, y, z) of sum_k c_k Y_k(x, y, z) for per-basis weights c[k]
__device__ __forceinline__ void sh_basis_vjp(int deg, float x, float y, float z, const float* c, float& gx,
                                             float& gy, float& gz) {
  gx = gy = gz = 0.f;
  if (deg < 1) return;
  gy += -kSH1 * c[1];
  gz += kSH1 * c[2];
  gx += -kSH1 * c[3];
  if (deg < 2) return;
  float xx = x * x, yy = y * y, zz = z * z;
  gx += 2.f * kSH22 * y * c[4];
  gy += 2.f * kSH22 * x * c[4];
  gy += -kSH21 * z * c[5];
  gz += -kSH21 * y * c[5];
  gz += kSH20 * 6.f * z * c[6];
  gx += -kSH21 * z * c[7];
  gz += -kSH21 * x * c[7];
  gx += kSH22 * 2.f * x * c[8];
  gy += -kSH22 * 2.f * y * c[8];
  if (deg < 3) return;
  gx += -kSH33 * 6.f * x * y * c[9];
  gy += -kSH33 * (3.f * xx - 3.f * yy) * c[9];
  gx += 2.f * kSH32 * y * z * c[10];
  gy += 2.f * kSH32 * x * z * c[10];
  gz += 2.f * kSH32 * x * y * c[10];
  gy += -kSH31 * (5.f * zz - 1.f) * c[11];
  gz += -kSH31 * y * 10.f * z * c[11];
  gz += kSH30 * (15.f * zz - 3.f) * c[12];
  gx += -kSH31 * (5.f * zz - 1.f) * c[13];
  gz += -kSH31 * x * 10.f * z * c[13];
  gx += kSH32 * z * 2.f * x * c[14];
  gy += -kSH32 * z * 2.f * y * c[14];
  gz += kSH32 * (xx - yy) * c[14];
  gx += -kSH33 * (3.f * xx - 3.f * yy) * c[15];
  gy += kSH33 * 6.f * x * y * c[15];
}

// ---------------------------------------------------------------------------
// tile rectangle of a support box (integer contract, float32 arithmetic)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void tile_rect(float mx, float my, float ex, float ey, float inv_tw, float inv_th,
                                          int tiles_x, int tiles_y, int& x0, int& y0, int& x1, int& y1) {
  if (!(ex > 0.f && ey > 0.f)) {
    x0 = y0 = x1 = y1 = 0;
    return;
  }
  float lx = floorf(__fmul_rn(__fsub_rn(mx, ex), inv_tw));
  float hx = __fadd_rn(floorf(__fmul_rn(__fadd_rn(mx, ex), inv_tw)), 1.f);
  float ly = floorf(__fmul_rn(__fsub_rn(my, ey), inv_th));
  float hy = __fadd_rn(floorf(__fmul_rn(__fadd_rn(my, ey), inv_th)), 1.f);
  float TX = (float)tiles_x, TY = (float)tiles_y;
  x0 = (int)fminf(fmaxf(lx, 0.f), TX);
  x1 = (int)fminf(fmaxf(hx, 0.f), TX);
  y0 = (int)fminf(fmaxf(ly, 0.f), TY);
  y1 = (int)fminf(fmaxf(hy, 0.f), TY);
  if (x1 <= x0 || y1 <= y0) x0 = y0 = x1 = y1 = 0;
}

// ---------------------------------------------------------------------------
// per-pixel evaluation shared by the forward and backward raster kernels;
// the skip decisions must be bit-identical in both, hence explicit rounding
// intrinsics (no contraction differences between the two call sites).
// a = {mu_local_x, mu_local_y, i0, k}, i1, log2o
// ---------------------------------------------------------------------------

// Warp-aggregated atomic add of 1 per active lane to counter[t]: lanes with the
// same t are grouped, the group leader adds the group size once, and each
// lane gets old value + its rank in the group (neighbouring Gaussians tend to
// share tiles, so plain per-lane atomics would serialise on one address).
__device__ __forceinline__ uint32_t warp_agg_inc(uint32_t* __restrict__ counter, uint32_t t, unsigned active) {
  const unsigned peers = __match_any_sync(active, t);
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(peers) - 1;
  uint32_t base = 0;
  if (lane == leader) base = atomicAdd(&counter[t], (uint32_t)__popc(peers));
  base = __shfl_sync(peers, base, leader);
  return base + __popc(peers & ((1u << lane) - 1u));
}

// ---------------------------------------------------------------------------
// Bounds-checked build (compiled with -DGS_CHECKED into libgsplat_checked.so):
// every index read from memory (list ids, tile ranges, tile numbers computed
// from rectangles, record ids) is checked before it is used; a violation
// sets the context's bounds word (gs_sync_status reports GS_ERR_BOUNDS) and
// the access is skipped or redirected to a valid dummy, never trapped.  The
// normal build compiles the checks away.  Each translation unit has its own
// copy of the word's address, bound by bind_bounds_word().
// ---------------------------------------------------------------------------
#ifdef GS_CHECKED
static __device__ uint32_t* gs_bounds_word = nullptr;
#endif
__device__ __forceinline__ bool in_bounds(bool ok) {
#ifdef GS_CHECKED
  if (!ok && gs_bounds_word) atomicOr(gs_bounds_word, 1u);
  return ok;
#else
  (void)ok;
  return true;
#endif
}
static inline cudaError_t bind_bounds_word(uint32_t* word) {
#ifdef GS_CHECKED
  return cudaMemcpyToSymbol(gs_bounds_word, &word, sizeof(word));
#else
  (void)word;
  return cudaSuccess;
#endif
}

// ---------------------------------------------------------------------------
// Programmatic dependent launch.  The kernels of an iteration form one chain
// on one stream; launched with launch_pdl, a kernel's CTAs may be scheduled
// while the previous kernel drains its last CTAs (and, in a CUDA graph, the
// launch gap between them shrinks).  Every chained kernel starts with
// pdl_wait(), which returns once the previous kernel has completed and its
// memory is visible (a no-op for a kernel launched without the attribute),
// and then calls pdl_trigger(), which allows the next kernel to be scheduled
// as soon as SMs free up.  Nothing before pdl_wait() touches memory, so the
// results are those of plain stream order.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;\n" :::); }
__device__ __forceinline__ void pdl_enter() {
  pdl_wait();
  pdl_trigger();
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

}  // namespace gs
