// Eq. 10 for one quadtree leaf: the back-projection of its centre and the
// initial parameters of the Gaussian placed there (Sec. III-B.2).  Shared by
// the rendered-alpha seeding (quadtree.cu) and the voxel-weight seeding
// (tsdf.cu).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace gs {

struct SeedArgs {
  const float *rgb, *depth, *alpha;
  float alpha_thr;
  int W, H;
  float fx, fy, cx, cy;
  float R[9], t[3];  // world-to-camera, R row-major
  int sh_degree;
  float *means, *log_scales, *quats, *logits, *sh;
  uint32_t capacity;
};

// Centre pixel of leaf L (pixel centres at integer + 0.5): the pixel holding
// u = (x0 + w/2, y0 + h/2) (exact in float32), clamped to the image.
__device__ __forceinline__ size_t leaf_pixel(const SeedArgs& a, int4 L, float* ux, float* uy) {
  *ux = (float)L.x + 0.5f * (float)L.z;
  *uy = (float)L.y + 0.5f * (float)L.w;
  const int pi = min((int)floorf(*ux), a.W - 1), pj = min((int)floorf(*uy), a.H - 1);
  return (size_t)pj * a.W + pi;
}

// p_w = R^T (((u_x - cx) z / fx, (u_y - cy) z / fy, z) - t) in float32 with
// a fixed order of correctly rounded operations (no contraction), so that
// the voxel it falls in is decided identically by any IEEE float32
// evaluation in the same order.
__device__ __forceinline__ void leaf_point(const SeedArgs& a, float ux, float uy, float z, float p[3]) {
  const float q0 = __fsub_rn(__fdiv_rn(__fmul_rn(__fsub_rn(ux, a.cx), z), a.fx), a.t[0]);
  const float q1 = __fsub_rn(__fdiv_rn(__fmul_rn(__fsub_rn(uy, a.cy), z), a.fy), a.t[1]);
  const float q2 = __fsub_rn(z, a.t[2]);
#pragma unroll
  for (int c = 0; c < 3; ++c)
    p[c] = __fadd_rn(__fadd_rn(__fmul_rn(a.R[c], q0), __fmul_rn(a.R[3 + c], q1)), __fmul_rn(a.R[6 + c], q2));
}

// Row k of the output arrays: mean p, log-scale log(d) with d the
// back-projected half diagonal sqrt(w^2 + h^2) / 2 * z / fx on all axes,
// identity rotation, opacity 0.5 (logit 0), SH DC so that the decoded colour
// is the pixel colour, higher bands 0.
__device__ __forceinline__ void write_seed(const SeedArgs& a, uint32_t k, int4 L, size_t pix, const float p[3],
                                           float z) {
#pragma unroll
  for (int c = 0; c < 3; ++c) a.means[3 * (size_t)k + c] = p[c];
  const float ls = logf(0.5f * hypotf((float)L.z, (float)L.w) * z / a.fx);
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
  constexpr float kInvY00 = 3.5449077018110318f;  // 1 / Y_00 = 2 sqrt(pi)
#pragma unroll
  for (int c = 0; c < 3; ++c) sh[c] = (a.rgb[c * HW + pix] - 0.5f) * kInvY00;
  for (int e = 3; e < 3 * K; ++e) sh[e] = 0.f;
}

// SeedArgs from the camera intrinsics K4 = (fx, fy, cx, cy) and the pose
inline SeedArgs make_seed_args(const float* rgb, const float* depth, const float* alpha, float alpha_thr, int W,
                               int H, const float K4[4], const float R[9], const float t[3], int sh_degree,
                               float* means, float* log_scales, float* quats, float* logits, float* sh,
                               uint32_t capacity) {
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
  return a;
}

}  // namespace gs
