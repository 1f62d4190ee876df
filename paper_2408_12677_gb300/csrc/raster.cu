// Tile rasterizer, forward (Eq. 11, front to back with early stop on
// transmittance) and backward (back to front from the stored last
// contributor, transmittance recomputed from the stored final T).
//
// One CTA of 128 threads per tile; each warp owns an 8 x 8 pixel block of it,
// each thread two pixels (rows y and y + 4), and the four warps run
// independently (no block barriers).  A warp walks the tile's depth-sorted
// list in chunks of 32 entries with the next chunk's 48 B records already in
// flight, converts the records to tile-local coordinates (so per-pixel offsets
// keep float32 precision), keeps the entries whose support bounding box meets
// its block (ballot) and evaluates only those.  The backward pass adds each
// Gaussian's gradient to its global record with per-lane vector atomics when
// few lanes contribute, else after a transposed shuffle reduction over the
// warp with one warp-wide atomic.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace gs {

namespace {

constexpr int kThreads = 128;  // 4 independent warps per CTA, one 8 x 8 pixel block each
// Backward pass: when at most this many lanes contribute to a Gaussian, each
// adds its ten values with three 16-byte vector atomics (3 issue slots)
// instead of the warp reduction (about 45); the kernel is issue-bound, and
// up to this many lanes the L2 atomic units keep up (at 32 they saturate).
constexpr int kAtomicLanes = 16;
constexpr unsigned kFull = 0xFFFFFFFFu;

// One list entry in tile-local coordinates:
//   a = {mu_x, mu_y, i0, k}, b = {i1, log2 opacity, z, support radius r2},
//   c = {r, g, b, mask of the warp block's halves the support box meets}
struct Entry {
  float4 a, b, c;
};

// A list entry's item id; the checked build redirects an id beyond the
// records to record 0 (and reports it), the normal build passes it through.
__device__ __forceinline__ uint32_t checked_id(uint32_t g, uint32_t n_items) {
  return in_bounds(g < n_items) ? g : 0u;
}

// Asynchronous copy of one 48 B record into shared memory (3 x 16 B cp.async).
__device__ __forceinline__ void cp_record(float4* dst, const float4* __restrict__ feat, uint32_t g) {
  const float4* src = feat + 3 * (size_t)g;
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
#pragma unroll
  for (int k = 0; k < 3; ++k)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d + 16u * k), "l"(src + k) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// Converts a gathered record to tile-local coordinates and tests the splat's
// support bounding box against the two halves of the warp's 8 x 8 block:
// rows [by, by + 4) (bit 0, the lanes' first pixels) and [by + 4, by + 8)
// (bit 1, their second pixels), columns [bx, bx + 8).  The box holds every
// pixel the per-pixel test can accept: q' <= min(qmax, log2 o - log2 alpha_min)
// is the ellipse (i0 dx)^2 + (i1 (dy - k dx))^2 <= R2, with half-extents
// sqrt(R2) / i0 and sqrt(R2) sqrt(k^2 / i0^2 + 1 / i1^2); the widening covers
// float32 rounding of the test.  Returns the mask of halves hit (0 = none);
// the mask is warp-uniform per entry, so a half it excludes costs the warp
// nothing.
__device__ __forceinline__ unsigned make_entry(float4 f0, float4 f1, float4 f2, float ox, float oy, float bx, float by,
                                               const RasterParams& rp, Entry& e) {
  const float mlx = __fadd_rn(__fsub_rn(f0.x, ox), f0.z);
  const float mly = __fadd_rn(__fsub_rn(f0.y, oy), f0.w);
  const float R2 = fminf(rp.qmax_s, __fsub_rn(f1.w, rp.log2_alpha_min));
  e.a = make_float4(mlx, mly, f1.x, f1.y);
  e.b = make_float4(f1.z, f1.w, f2.w, R2);
  unsigned m = 0u;
  if (R2 > 0.f && f1.x > 0.f && f1.z > 0.f) {
    const float Rr = sqrtf(R2) * 1.0001f + 1e-4f;
    const float inv0 = rcp_approx(f1.x), inv1 = rcp_approx(f1.z);
    const float ex = Rr * inv0 + 1e-3f;
    const float ey = Rr * sqrtf(f1.y * f1.y * inv0 * inv0 + inv1 * inv1) + 1e-3f;
    if (mlx + ex >= bx + 0.5f && mlx - ex <= bx + 7.5f) {
      const float y0 = mly - ey, y1 = mly + ey;
      m = ((y1 >= by + 0.5f && y0 <= by + 3.5f) ? 1u : 0u) | ((y1 >= by + 4.5f && y0 <= by + 7.5f) ? 2u : 0u);
    }
  }
  e.c = make_float4(f2.x, f2.y, f2.z, __uint_as_float(m));
  return m;
}

// Tile, view and pixel origin of visit k: k indexes the tile visit order (or
// the tiles directly), global tiles map to views by tile_base.
struct TileJob {
  int v;          // view
  int ox, oy;     // pixel origin of the tile within the view
  uint2 range;
  uint32_t tile;  // global tile id
};
template <int TW, int TH>
__device__ __forceinline__ TileJob tile_job_of(const RasterArgs& a, uint32_t tile) {
  int v = 0;
  for (int k = 1; k < a.views; ++k)
    if (tile >= a.v[k].tile_base) v = k;
  const int lt = (int)(tile - a.v[v].tile_base);
  const int tx = lt % a.v[v].tiles_x, ty = lt / a.v[v].tiles_x;
  uint2 r = __ldg(&a.ranges[tile]);
  if (!in_bounds(r.x <= r.y && r.y <= a.n_ids)) r = make_uint2(0u, 0u);  // checked build: an empty list
  return TileJob{v, tx * TW, ty * TH, r, tile};
}
template <int TW, int TH>
__device__ __forceinline__ TileJob tile_job(const RasterArgs& a, uint32_t k) {
  return tile_job_of<TW, TH>(a, a.order ? __ldg(&a.order[k]) : k);
}

// Bucket mode: loads the class counts into s_start (kLenClasses + 1 words)
// as s_start[c] = tiles of class c or longer (s_start[kLenClasses] = 0);
// called by every thread of the CTA (it synchronises the CTA).
__device__ __forceinline__ void load_class_starts(const RasterArgs& a, uint32_t* __restrict__ s_start) {
  if (threadIdx.x < 32) {
    constexpr int PER = (kLenClasses + 31) / 32;
    uint32_t cnt[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int c = (int)threadIdx.x + 32 * i;
      cnt[i] = c < kLenClasses ? __ldg(&a.cls_count[c]) : 0u;
    }
#pragma unroll
    for (int i = 0; i < PER; ++i)
      if ((int)threadIdx.x + 32 * i < kLenClasses) s_start[threadIdx.x + 32 * i] = cnt[i];
    __syncwarp();
    class_starts_desc(s_start);  // s_start[c] = tiles of the classes above c
    __syncwarp();
#pragma unroll
    for (int i = 0; i < PER; ++i)
      if ((int)threadIdx.x + 32 * i < kLenClasses) s_start[threadIdx.x + 32 * i] += cnt[i];
    if (threadIdx.x == 0) s_start[kLenClasses] = 0u;
  }
  __syncthreads();
}

// Bucket mode: the tile of visit k, the (k - tiles of longer classes)-th of
// its class, c the largest class with s_start[c] > k (s_start is
// non-increasing and s_start[0] is the tile count, which exceeds k).
__device__ __forceinline__ uint32_t class_visit_tile(const RasterArgs& a, const uint32_t* __restrict__ s_start,
                                                     uint32_t k) {
  int c = 0;
#pragma unroll
  for (int step = 128; step > 0; step >>= 1)
    if (c + step < kLenClasses && s_start[c + step] > k) c += step;
  return __ldg(&a.cls_tiles[(size_t)c * a.cls_stride + (k - s_start[c + 1])]);
}

// Front-to-back step of one pixel for one list entry (Eq. 11 with the skip
// and stop rules), without branches: a pixel that is done, outside the
// support or would drop T below t_eps adds a weight of exactly 0.
template <bool COUNT>
__device__ __forceinline__ void blend_slot(const float4& a, const float4& bb, const float4& c, float plx, float ply,
                                           const RasterParams& rp, int idx1, bool on, float& T, float& R, float& G,
                                           float& B, float& D, int& last, bool& done, uint32_t& n_visit,
                                           uint32_t& n_blend) {
  const float dx = __fsub_rn(plx, a.x);
  const float dy = __fsub_rn(ply, a.y);
  const float t0 = __fmul_rn(a.z, dx);
  const float t1 = __fmul_rn(bb.x, __fmaf_rn(-a.w, dx, dy));
  const float q = __fmaf_rn(t0, t0, __fmul_rn(t1, t1));
  const bool pass = on && !done && q <= bb.w;
  const float al = fminf(rp.alpha_max, ex2_approx(__fsub_rn(bb.y, q)));
  const float test_T = __fmul_rn(T, __fsub_rn(1.f, al));
  const bool stop = pass && test_T < rp.t_eps;
  const bool add = pass && !stop;
  const float w = add ? al * T : 0.f;
  R = fmaf(w, c.x, R);
  G = fmaf(w, c.y, G);
  B = fmaf(w, c.z, B);
  D = fmaf(w, bb.z, D);
  T = add ? test_T : T;
  last = add ? idx1 : last;
  if (COUNT) {
    n_visit += (on && !done) ? 1u : 0u;
    n_blend += add ? 1u : 0u;
  }
  done = done || stop;
}

// Two floats in one 64-bit register pair, for the packed FP32 instructions
// add / sub / mul / fma .rn.f32x2: each rounds both halves exactly as the
// scalar instruction would, and takes one issue slot for two operations per
// lane (the FMA pipe itself does not get wider: 124 FMA lanes per SM per
// clock either way, measured; the gain is issue slots in issue-bound code).
typedef unsigned long long f2x;
__device__ __forceinline__ f2x f2_pack(float lo, float hi) {
  f2x r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ f2x f2_bcast(float x) { return f2_pack(x, x); }
__device__ __forceinline__ float f2_lo(f2x r) { return __uint_as_float((unsigned)(r & 0xFFFFFFFFull)); }
__device__ __forceinline__ float f2_hi(f2x r) { return __uint_as_float((unsigned)(r >> 32)); }
__device__ __forceinline__ f2x f2_sub(f2x a, f2x b) {
  f2x d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2x f2_mul(f2x a, f2x b) {
  f2x d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2x f2_fma(f2x a, f2x b, f2x c) {
  f2x d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// Forward pass of one 8 x 8 pixel block (quadrant `quad` of global tile
// `tile`) by one warp; buf is the warp's shared staging buffer, s_raw the
// two shared slots per lane that its Gaussians' records land in (cp.async).
template <int TW, int TH, bool COUNT, bool LOSS>
__device__ __forceinline__ void fwd_job(const RasterArgs& a, const RasterParams& rp, uint32_t tile, int quad,
                                        Entry* __restrict__ buf, float4 (*__restrict__ s_raw)[32][3],
                                        float* __restrict__ T_final_all,
                                        int32_t* __restrict__ last_all, unsigned long long* __restrict__ counters) {
  constexpr int WX = TW / 8;
  const TileJob job = tile_job_of<TW, TH>(a, tile);
  const RasterView& vw = a.v[job.v];
  const int width = vw.width, height = vw.height;
  const uint32_t* __restrict__ ids = a.ids;
  const float4* __restrict__ feat = a.feat;
  const int lane = threadIdx.x & 31;
  const int bxi = (quad % WX) * 8, byi = (quad / WX) * 8;
  const int lx = bxi + (lane & 7), ly0 = byi + (lane >> 3), ly1 = ly0 + 4;
  const int px = job.ox + lx, py0 = job.oy + ly0, py1 = job.oy + ly1;
  const bool in0 = px < width && py0 < height, in1 = px < width && py1 < height;
  const float plx = (float)lx + 0.5f, ply0 = (float)ly0 + 0.5f, ply1 = (float)ly1 + 0.5f;
  const float ox = (float)job.ox, oy = (float)job.oy, bx = (float)bxi, by = (float)byi;
  const uint2 r = job.range;
  const int n = (int)(r.y - r.x);
  __syncwarp();  // the warp's previous job is done with buf

  float T0 = 1.f, R0 = 0.f, G0 = 0.f, B0 = 0.f, D0 = 0.f;
  float T1 = 1.f, R1 = 0.f, G1 = 0.f, B1 = 0.f, D1 = 0.f;
  int last0 = 0, last1 = 0;
  uint32_t n_blend = 0, n_visit = 0;
  bool done0 = !in0, done1 = !in1;
  const f2x PLY = f2_pack(ply0, ply1), ONE2 = f2_pack(1.f, 1.f);

  // software pipeline: chunk c's records in shared memory, chunk c + 32's in
  // flight (cp.async), the ids of chunk c + 64 in a register
  int cur = 0;
  if (lane < n) cp_record(s_raw[0][lane], feat, checked_id(__ldg(&ids[r.x + lane]), a.n_items));
  cp_commit();
  uint32_t g2 = 32 + lane < n ? checked_id(__ldg(&ids[r.x + 32 + lane]), a.n_items) : 0u;
  for (int c0 = 0; c0 < n; c0 += 32, cur ^= 1) {
    if (__all_sync(kFull, done0 && done1)) break;
    if (c0 + 32 + lane < n) cp_record(s_raw[cur ^ 1][lane], feat, g2);
    cp_commit();
    if (c0 + 64 + lane < n) g2 = checked_id(__ldg(&ids[r.x + c0 + 64 + lane]), a.n_items);
    cp_wait_prev();
    const bool have = c0 + lane < n;
    Entry e;
    const float4* raw = s_raw[cur][lane];
    const bool hit = have && make_entry(raw[0], raw[1], raw[2], ox, oy, bx, by, rp, e) != 0u;
    __syncwarp();
    if (hit) buf[lane] = e;
    unsigned bal = __ballot_sync(kFull, hit);
    __syncwarp();
    while (bal) {
      const int j = __ffs(bal) - 1;
      bal &= bal - 1;
      const float4 a = buf[j].a;
      const float4 bb = buf[j].b;
      const float4 c = buf[j].c;
      const unsigned halves = __float_as_uint(c.w);
      // branch-free per pixel: every lane evaluates, predicates decide
      // (a blend of weight 0 leaves R, G, B, D unchanged)
      // both rows as straight-line code (independent chains; a row outside the
      // support box runs with weight 0)
      // a half the support box misses (warp-uniform) is skipped
      if (halves == 3u) {
        // blend_slot for both rows at once, element for element the same
        // operations (packed f32x2)
        const float dx = __fsub_rn(plx, a.x);
        const float t0 = __fmul_rn(a.z, dx);
        const f2x DY = f2_sub(PLY, f2_bcast(a.y));
        const f2x WQ = f2_fma(f2_bcast(-a.w), f2_bcast(dx), DY);
        const f2x TQ = f2_mul(f2_bcast(bb.x), WQ);
        const f2x Q = f2_fma(f2_bcast(t0), f2_bcast(t0), f2_mul(TQ, TQ));
        const bool pass0 = !done0 && f2_lo(Q) <= bb.w, pass1 = !done1 && f2_hi(Q) <= bb.w;
        const f2x ARG = f2_sub(f2_bcast(bb.y), Q);
        const f2x AL = f2_pack(fminf(rp.alpha_max, ex2_approx(f2_lo(ARG))), fminf(rp.alpha_max, ex2_approx(f2_hi(ARG))));
        const f2x TT = f2_pack(T0, T1);
        const f2x TEST = f2_mul(TT, f2_sub(ONE2, AL));
        const bool stop0 = pass0 && f2_lo(TEST) < rp.t_eps, stop1 = pass1 && f2_hi(TEST) < rp.t_eps;
        const bool add0 = pass0 && !stop0, add1 = pass1 && !stop1;
        const f2x WW = f2_mul(AL, TT);
        const f2x W = f2_pack(add0 ? f2_lo(WW) : 0.f, add1 ? f2_hi(WW) : 0.f);
        const f2x RR = f2_fma(W, f2_bcast(c.x), f2_pack(R0, R1));
        const f2x GG = f2_fma(W, f2_bcast(c.y), f2_pack(G0, G1));
        const f2x BB = f2_fma(W, f2_bcast(c.z), f2_pack(B0, B1));
        const f2x DZ = f2_fma(W, f2_bcast(bb.z), f2_pack(D0, D1));
        R0 = f2_lo(RR);
        R1 = f2_hi(RR);
        G0 = f2_lo(GG);
        G1 = f2_hi(GG);
        B0 = f2_lo(BB);
        B1 = f2_hi(BB);
        D0 = f2_lo(DZ);
        D1 = f2_hi(DZ);
        T0 = add0 ? f2_lo(TEST) : T0;
        T1 = add1 ? f2_hi(TEST) : T1;
        last0 = add0 ? c0 + j + 1 : last0;
        last1 = add1 ? c0 + j + 1 : last1;
        if (COUNT) {
          n_visit += (done0 ? 0u : 1u) + (done1 ? 0u : 1u);
          n_blend += (add0 ? 1u : 0u) + (add1 ? 1u : 0u);
        }
        done0 = done0 || stop0;
        done1 = done1 || stop1;
      } else if (halves == 1u) {
        blend_slot<COUNT>(a, bb, c, plx, ply0, rp, c0 + j + 1, true, T0, R0, G0, B0, D0, last0, done0, n_visit,
                          n_blend);
      } else {
        blend_slot<COUNT>(a, bb, c, plx, ply1, rp, c0 + j + 1, true, T1, R1, G1, B1, D1, last1, done1, n_visit,
                          n_blend);
      }
    }
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
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
  const size_t HW = (size_t)width * height;
  float* __restrict__ color = vw.color;
  float* __restrict__ depth = vw.depth;
  float* __restrict__ alpha = vw.alpha;
  float* __restrict__ T_final = T_final_all + vw.pix_base;
  int32_t* __restrict__ last_out = last_all + vw.pix_base;
  if (in0) {
    const size_t p = (size_t)py0 * width + px;
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
    const size_t p = (size_t)py1 * width + px;
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
  if constexpr (LOSS) {
    // L1 loss epilogue (Eq. 12 plus the depth term): the same residuals,
    // signs and colour scale as the separate loss kernels, per-block sums
    const float gscale_c = a.w_color / (3.f * (float)HW);
    float sc = 0.f, sd = 0.f, nv = 0.f;
    const float* __restrict__ trgb = vw.trgb;
    const float* __restrict__ tdep = vw.tdep;
    float* __restrict__ ldc = vw.loss_dc;
    float* __restrict__ ldd = vw.loss_dd;
    auto score = [&](size_t p, float T, float Rc, float Gc, float Bc, float D) {
      const float col[3] = {Rc + T * rp.bg[0], Gc + T * rp.bg[1], Bc + T * rp.bg[2]};
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float r = col[c] - __ldg(&trgb[(size_t)c * HW + p]);
        sc += fabsf(r);
        ldc[(size_t)c * HW + p] = gscale_c * (float)((r > 0.f) - (r < 0.f));
      }
      const float td = __ldg(&tdep[p]);
      const bool valid = td > 0.f;
      const float rd = D - td;
      sd += valid ? fabsf(rd) : 0.f;
      nv += valid ? 1.f : 0.f;
      ldd[p] = valid ? (float)((rd > 0.f) - (rd < 0.f)) : 0.f;
    };
    if (in0) score((size_t)py0 * width + px, T0, R0, G0, B0, D0);
    if (in1) score((size_t)py1 * width + px, T1, R1, G1, B1, D1);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      sc += __shfl_xor_sync(kFull, sc, off);
      sd += __shfl_xor_sync(kFull, sd, off);
      nv += __shfl_xor_sync(kFull, nv, off);
    }
    if (lane == 0) {
      float* part = a.loss_partials + 3 * (4 * (size_t)job.tile + quad);
      part[0] = sc;
      part[1] = sd;
      part[2] = nv;
      if (a.nvalid) atomicAdd(&a.nvalid[job.v], (uint32_t)nv);  // an integer: exact in any order
    }
  }
}

// Pulls the next (tile visit, quadrant) job for the calling warp from the
// device counter `work`: jobs 4k .. 4k + 3 are the four quadrants of visit
// k, so warps take the tiles in visit order (longest lists first) and a warp
// that finishes early takes new work instead of waiting for the other
// quadrants of its tile.  Returns false when all jobs are taken.
__device__ __forceinline__ bool next_job(uint32_t* __restrict__ work, uint32_t n_jobs, uint32_t& job) {
  uint32_t j = 0;
  if ((threadIdx.x & 31) == 0) j = atomicAdd(work, 1u);
  job = __shfl_sync(kFull, j, 0);
  return job < n_jobs;
}

// The tile of forward visit k: from the class lists in bucket mode (the warp
// on block 0 of the visit also records it in the flat order the backward
// pass reads), else from the flat order, else tile k.
__device__ __forceinline__ uint32_t fwd_visit_tile(const RasterArgs& a, const uint32_t* __restrict__ s_start,
                                                   uint32_t k, int quad) {
  if (!a.cls_count) return a.order ? a.order[k] : k;
  const uint32_t tile = class_visit_tile(a, s_start, k);
  if (quad == 0 && (threadIdx.x & 31) == 0) a.order_out[k] = tile;
  return tile;
}

// PERSIST = false: one CTA per tile visit, warp w on quadrant w.  Otherwise
// a persistent grid whose warps pull jobs from `work` with next_job.
template <int TW, int TH, bool COUNT, bool LOSS, bool PERSIST>
__global__ void __launch_bounds__(kThreads, 7) raster_fwd_kernel(const __grid_constant__ RasterArgs a, RasterParams rp,
                                                              float* __restrict__ T_final_all,
                                                              int32_t* __restrict__ last_all,
                                                              unsigned long long* __restrict__ counters,
                                                              uint32_t* __restrict__ work) {
  pdl_enter();
  static_assert((TW / 8) * (TH / 8) == kThreads / 32, "four 8x8 warp blocks per tile");
  __shared__ Entry s_e[kThreads / 32][32];
  __shared__ __align__(16) float4 s_rawf[kThreads / 32][2][32][3];
  __shared__ uint32_t s_start[kLenClasses + 1];  // bucket mode: tiles of class c or longer
  const int warp = threadIdx.x >> 5;
  if (a.cls_count) load_class_starts(a, s_start);  // CTA-uniform
  if constexpr (!PERSIST) {
    fwd_job<TW, TH, COUNT, LOSS>(a, rp, fwd_visit_tile(a, s_start, blockIdx.x, warp), warp, s_e[warp], s_rawf[warp],
                                 T_final_all, last_all, counters);
  } else {
    const uint32_t n_jobs = 4u * a.n_tiles;
    uint32_t job;
    while (next_job(work, n_jobs, job)) {
      const int quad = (int)(job & 3u);
      fwd_job<TW, TH, COUNT, LOSS>(a, rp, fwd_visit_tile(a, s_start, job >> 2, quad), quad, s_e[warp], s_rawf[warp],
                                   T_final_all, last_all, counters);
    }
  }
}

// float offset of gradient value k (the six exponent / opacity sums, depth |
// rgb 3) in the 12-float record {s0, s1, s2, s3} {s4, s5, depth, -} {r, g, b, -}
__device__ __forceinline__ int rec_off(int k) { return k < 7 ? k : k + 1; }

// Sum the 10 values v[0..9] over the warp with exchanges that halve the number
// of values each lane carries (xor 16: 10 -> 5, xor 8: 5 -> 3, xor 4: 3 -> 2,
// xor 2: 2 -> 1) and a final xor-1 step (12 shuffles instead of 50), then add
// the totals to the record: even lanes hold distinct values, so this is one
// warp-wide scalar atomic add.
__device__ __forceinline__ void warp_reduce_add10(float (&v)[10], float* __restrict__ rec) {
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
  if (!(lane & 1) && valid) atomicAdd(&rec[rec_off((b4 ? 5 : 0) + i3)], x);
}

// Back-to-front step of one pixel for one Gaussian (pixel_q, then bwd_body):
// updates the pixel's running transmittance T and "colour behind" U and adds
// the Gaussian's gradient sums to v.  With ga = dL/dalpha * alpha (unclamped alpha) the
// exponent and opacity gradients are linear in
//   v[0] = sum ga t0, v[1] = sum ga t1, v[2] = sum ga t0 dx,
//   v[3] = sum ga t1 dx, v[4] = sum ga t1 w, v[5] = sum ga
// (t0 = i0 dx, t1 = i1 w, w = dy - k dx): the Gaussian's constants (i0, i1,
// k, ln 2, 1 / opacity) are applied once per Gaussian in the projection
// backward pass.  v[6] = sum w dD (depth), v[7..9] = sum w dC (colour).
// Exponent of one pixel for one entry: q' = t0^2 + t1^2 and its parts.
struct PixQ {
  float dx, t0, wq, t1, q;
  bool pass;  // inside the support and in front of the pixel's last contributor
};
__device__ __forceinline__ PixQ pixel_q(const float4& a, const float4& bb, float plx, float ply, bool behind_last) {
  PixQ r;
  r.dx = __fsub_rn(plx, a.x);
  const float dy = __fsub_rn(ply, a.y);
  r.t0 = __fmul_rn(a.z, r.dx);
  r.wq = __fmaf_rn(-a.w, r.dx, dy);
  r.t1 = __fmul_rn(bb.x, r.wq);
  r.q = __fmaf_rn(r.t0, r.t0, __fmul_rn(r.t1, r.t1));
  r.pass = behind_last && r.q <= bb.w;
  return r;
}

// The rest of the back-to-front step, without branches: a lane whose pixel
// does not take part runs it with weight 0 and leaves T, U and v unchanged.
// FIRST: the entry's first pixel row of the lane writes the ten sums instead
// of adding to them (no zeroing of v per entry; a zero term may then be
// stored as -0, which adds like +0).
template <bool FIRST>
__device__ __forceinline__ void bwd_body(const PixQ& e, const float4& bb, const float4& c, const RasterParams& rp,
                                         float& T, float& U, float dC0, float dC1, float dC2, float dD, float dA_T,
                                         float (&v)[10]) {
  const float araw = ex2_approx(__fsub_rn(bb.y, e.q));
  const float al = fminf(rp.alpha_max, araw);
  const float inv1m = rcp_approx(1.f - al);  // 1 - alpha in [0.01, 1)
  const float Ti = T * inv1m;  // transmittance in front of this Gaussian
  const float w = e.pass ? al * Ti : 0.f;
  v[7] = FIRST ? w * dC0 : fmaf(w, dC0, v[7]);
  v[8] = FIRST ? w * dC1 : fmaf(w, dC1, v[8]);
  v[9] = FIRST ? w * dC2 : fmaf(w, dC2, v[9]);
  v[6] = FIRST ? w * dD : fmaf(w, dD, v[6]);
  const float cdot = c.x * dC0 + c.y * dC1 + c.z * dC2 + bb.z * dD;
  // d/d alpha_i: colour/depth T_i c_i - (sum behind)/(1 - alpha_i); alpha image + T_final/(1 - alpha_i)
  const float g_alpha = Ti * cdot - (U - dA_T) * inv1m;
  U = fmaf(w, cdot, U);
  T = e.pass ? Ti : T;
  const float ga = (e.pass && araw <= rp.alpha_max) ? g_alpha * araw : 0.f;  // the 0.99 clamp has zero gradient
  const float gt0 = ga * e.t0, gt1 = ga * e.t1;
  v[0] = FIRST ? gt0 : v[0] + gt0;
  v[1] = FIRST ? gt1 : v[1] + gt1;
  v[2] = FIRST ? gt0 * e.dx : fmaf(gt0, e.dx, v[2]);
  v[3] = FIRST ? gt1 * e.dx : fmaf(gt1, e.dx, v[3]);
  v[4] = FIRST ? gt1 * e.wq : fmaf(gt1, e.wq, v[4]);
  v[5] = FIRST ? ga : v[5] + ga;
}

// Backward pass of one 8 x 8 pixel block (quadrant `quad` of the tile of
// visit k) by one warp, with the warp's shared staging buffers.
template <int TW, int TH>
__device__ __forceinline__ void bwd_job(const RasterArgs& a, const RasterParams& rp, uint32_t k, int quad,
                                        Entry* __restrict__ buf, uint32_t* __restrict__ bid,
                                        float4 (*__restrict__ s_raw)[32][3], uint32_t (*__restrict__ s_gid)[32],
                                        const float* __restrict__ T_final_all,
                                        const int32_t* __restrict__ last_all, float* __restrict__ g2d) {
  constexpr int WX = TW / 8;
  const TileJob job = tile_job<TW, TH>(a, k);
  const RasterView& vw = a.v[job.v];
  const int width = vw.width, height = vw.height;
  const uint32_t* __restrict__ ids = a.ids;
  const float4* __restrict__ feat = a.feat;
  const float* __restrict__ T_final = T_final_all + vw.pix_base;
  const int32_t* __restrict__ last_in = last_all + vw.pix_base;
  const float* __restrict__ dLdc = vw.dLdc;
  const float* __restrict__ dLdd = vw.dLdd;
  const float* __restrict__ dLda = vw.dLda;
  const float dscale = a.nvalid ? a.w_depth / (float)max(a.nvalid[job.v], 1u)
                                : (a.depth_scale ? a.depth_scale[job.v] : 1.f);
  const int lane = threadIdx.x & 31;
  const int bxi = (quad % WX) * 8, byi = (quad / WX) * 8;
  const int lx = bxi + (lane & 7), ly0 = byi + (lane >> 3), ly1 = ly0 + 4;
  const int px = job.ox + lx, py0 = job.oy + ly0, py1 = job.oy + ly1;
  const bool in0 = px < width && py0 < height, in1 = px < width && py1 < height;
  const float plx = (float)lx + 0.5f, ply0 = (float)ly0 + 0.5f, ply1 = (float)ly1 + 0.5f;
  const float ox = (float)job.ox, oy = (float)job.oy, bx = (float)bxi, by = (float)byi;
  const uint2 r = job.range;
  const size_t HW = (size_t)width * height;
  __syncwarp();  // the warp's previous job is done with the buffers

  // per-pixel state (two pixels per thread)
  float T0 = 1.f, c00 = 0.f, c01 = 0.f, c02 = 0.f, d0 = 0.f, a0 = 0.f;
  float T1 = 1.f, c10 = 0.f, c11 = 0.f, c12 = 0.f, d1 = 0.f, a1 = 0.f;
  int last0 = 0, last1 = 0;
  if (in0) {
    const size_t p = (size_t)py0 * width + px;
    T0 = T_final[p];
    last0 = last_in[p];
    c00 = dLdc[p];
    c01 = dLdc[HW + p];
    c02 = dLdc[2 * HW + p];
    d0 = dLdd[p] * dscale;
    a0 = dLda ? dLda[p] : 0.f;
  }
  if (in1) {
    const size_t p = (size_t)py1 * width + px;
    T1 = T_final[p];
    last1 = last_in[p];
    c10 = dLdc[p];
    c11 = dLdc[HW + p];
    c12 = dLdc[2 * HW + p];
    d1 = dLdd[p] * dscale;
    a1 = dLda ? dLda[p] : 0.f;
  }
  // U = sum over Gaussians behind of w_j (c_j . dC + z_j dD) + T_final (bg . dC)
  float U0 = T0 * (rp.bg[0] * c00 + rp.bg[1] * c01 + rp.bg[2] * c02);
  float U1 = T1 * (rp.bg[0] * c10 + rp.bg[1] * c11 + rp.bg[2] * c12);
  const float dAT0 = a0 * T0, dAT1 = a1 * T1;

  int wmax = max(last0, last1);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) wmax = max(wmax, __shfl_xor_sync(kFull, wmax, off));
  if (wmax == 0) return;

  // walk the list back to front in chunks of 32: chunk c in shared memory,
  // chunk c - 32 in flight (cp.async), the ids of chunk c - 64 in a register
  int c0 = ((wmax - 1) >> 5) << 5;
  int cur = 0;
  if (c0 + lane < wmax) {
    const uint32_t g = checked_id(ids[r.x + c0 + lane], a.n_items);
    s_gid[0][lane] = g;
    cp_record(s_raw[0][lane], feat, g);
  }
  cp_commit();
  uint32_t g2 = c0 >= 32 ? checked_id(ids[r.x + c0 - 32 + lane], a.n_items) : 0u;
  for (; c0 >= 0; c0 -= 32, cur ^= 1) {
    if (c0 >= 32) {
      s_gid[cur ^ 1][lane] = g2;
      cp_record(s_raw[cur ^ 1][lane], feat, g2);
    }
    cp_commit();
    if (c0 >= 64) g2 = checked_id(ids[r.x + c0 - 64 + lane], a.n_items);
    cp_wait_prev();
    const bool have = c0 + lane < wmax;
    Entry e;
    const float4* raw = s_raw[cur][lane];
    const bool hit = have && make_entry(raw[0], raw[1], raw[2], ox, oy, bx, by, rp, e) != 0u;
    __syncwarp();
    if (hit) {
      buf[lane] = e;
      bid[lane] = s_gid[cur][lane];
    }
    unsigned bal = __ballot_sync(kFull, hit);
    __syncwarp();
    while (bal) {
      const int j = 31 - __clz(bal);
      bal &= ~(1u << j);
      const int idx = c0 + j;
      const float4 a = buf[j].a;
      const float4 bb = buf[j].b;
      const float4 cc = buf[j].c;
      float v[10];  // written by the first row's step
      const unsigned halves = __float_as_uint(cc.w);
      // both pixel rows' exponents first, then the rows' steps as straight-line
      // code (independent chains); skipped when no lane of the warp takes part
      // a half the support box misses (warp-uniform) is skipped
      bool contrib;
      if (halves == 3u) {
        const PixQ e0 = pixel_q(a, bb, plx, ply0, idx < last0);
        const PixQ e1 = pixel_q(a, bb, plx, ply1, idx < last1);
        contrib = e0.pass || e1.pass;
        if (!__any_sync(kFull, contrib)) continue;
        bwd_body<true>(e0, bb, cc, rp, T0, U0, c00, c01, c02, d0, dAT0, v);
        bwd_body<false>(e1, bb, cc, rp, T1, U1, c10, c11, c12, d1, dAT1, v);
      } else if (halves == 1u) {
        const PixQ e0 = pixel_q(a, bb, plx, ply0, idx < last0);
        contrib = e0.pass;
        if (!__any_sync(kFull, contrib)) continue;
        bwd_body<true>(e0, bb, cc, rp, T0, U0, c00, c01, c02, d0, dAT0, v);
      } else {
        const PixQ e1 = pixel_q(a, bb, plx, ply1, idx < last1);
        contrib = e1.pass;
        if (!__any_sync(kFull, contrib)) continue;
        bwd_body<true>(e1, bb, cc, rp, T1, U1, c10, c11, c12, d1, dAT1, v);
      }
      const unsigned m = __ballot_sync(kFull, contrib);
      if (m == 0) continue;
      float* rec = g2d + 12 * (size_t)bid[j];
      if (__popc(m) <= kAtomicLanes) {
        if (contrib) {
          // three 16-byte vector atomics per lane (red.global.add.v4.f32)
          float4* r4 = reinterpret_cast<float4*>(rec);
          atomicAdd(r4, make_float4(v[0], v[1], v[2], v[3]));
          atomicAdd(r4 + 1, make_float4(v[4], v[5], v[6], 0.f));
          atomicAdd(r4 + 2, make_float4(v[7], v[8], v[9], 0.f));
        }
      } else {
        warp_reduce_add10(v, rec);
      }
    }
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// PERSIST = false: one CTA per tile visit, warp w on quadrant w.  Otherwise
// a persistent grid whose warps pull jobs from `work` with next_job.
template <int TW, int TH, bool PERSIST>
__global__ void __launch_bounds__(kThreads, 6) raster_bwd_kernel(const __grid_constant__ RasterArgs a,
                                                                 RasterParams rp,
                                                                 const float* __restrict__ T_final_all,
                                                                 const int32_t* __restrict__ last_all,
                                                                 float* __restrict__ g2d,
                                                                 uint32_t* __restrict__ work) {
  pdl_enter();
  static_assert((TW / 8) * (TH / 8) == kThreads / 32, "four 8x8 warp blocks per tile");
  __shared__ Entry s_e[kThreads / 32][32];
  __shared__ uint32_t s_id[kThreads / 32][32];
  __shared__ __align__(16) float4 s_raw[kThreads / 32][2][32][3];
  __shared__ uint32_t s_gid[kThreads / 32][2][32];
  const int warp = threadIdx.x >> 5;
  if constexpr (!PERSIST) {
    bwd_job<TW, TH>(a, rp, blockIdx.x, warp, s_e[warp], s_id[warp], s_raw[warp], s_gid[warp], T_final_all,
                    last_all, g2d);
  } else {
    const uint32_t n_jobs = 4u * a.n_tiles;
    uint32_t job;
    while (next_job(work, n_jobs, job))
      bwd_job<TW, TH>(a, rp, job >> 2, (int)(job & 3u), s_e[warp], s_id[warp], s_raw[warp], s_gid[warp],
                      T_final_all, last_all, g2d);
  }
}

RasterParams make_params(const RasterArgs& a) {
  RasterParams rp;
  rp.width = rp.height = 0;  // per view, from the view table
  rp.tile_w = a.tile_w;
  rp.tile_h = a.tile_h;
  rp.tiles_x = rp.tiles_y = 0;
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

namespace {

// Persistent grid: as many CTAs as fit on the GPU at once (occupancy of the
// kernel x SMs; per_sm caches the occupancy query of one kernel), at most one
// per tile visit.
template <class K>
int persistent_grid(K kernel, int& per_sm, int n_tiles, int num_sms) {
  if (per_sm == 0) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, kThreads, 0) != cudaSuccess || b < 1) b = 1;
    per_sm = b;
  }
  return std::max(1, std::min(n_tiles, per_sm * std::max(num_sms, 1)));
}

template <int TW, int TH, bool COUNT, bool LOSS>
void fwd_shape(const RasterArgs& a, const RasterParams& rp, float* T_final, int32_t* last,
               unsigned long long* counters, cudaStream_t s) {
  const int nt = (int)a.n_tiles;
  if (a.work) {
    static int per_sm = 0;
    auto* k = raster_fwd_kernel<TW, TH, COUNT, LOSS, true>;
    launch_pdl(k, persistent_grid(k, per_sm, nt, a.num_sms), kThreads, 0, s, a, rp, T_final, last, counters, a.work);
  } else {
    launch_pdl(raster_fwd_kernel<TW, TH, COUNT, LOSS, false>, nt, kThreads, 0, s, a, rp, T_final, last, counters,
               (uint32_t*)nullptr);
  }
}

template <bool COUNT, bool LOSS>
void fwd_shapes(const RasterArgs& a, const RasterParams& rp, float* T_final, int32_t* last,
                unsigned long long* counters, cudaStream_t s) {
  if (a.tile_w == 16) fwd_shape<16, 16, COUNT, LOSS>(a, rp, T_final, last, counters, s);
  else if (a.tile_w == 8) fwd_shape<8, 32, COUNT, LOSS>(a, rp, T_final, last, counters, s);
  else fwd_shape<32, 8, COUNT, LOSS>(a, rp, T_final, last, counters, s);
}

template <int TW, int TH>
void bwd_shape(const RasterArgs& a, const RasterParams& rp, const float* T_final, const int32_t* last, float* g2d,
               cudaStream_t s) {
  const int nt = (int)a.n_tiles;
  if (a.work) {
    static int per_sm = 0;
    auto* k = raster_bwd_kernel<TW, TH, true>;
    launch_pdl(k, persistent_grid(k, per_sm, nt, a.num_sms), kThreads, 0, s, a, rp, T_final, last, g2d, a.work);
  } else {
    launch_pdl(raster_bwd_kernel<TW, TH, false>, nt, kThreads, 0, s, a, rp, T_final, last, g2d, (uint32_t*)nullptr);
  }
}

}  // namespace

void launch_raster_fwd(const RasterArgs& a, float* T_final, int32_t* last, unsigned long long* counters,
                       cudaStream_t s) {
  if (a.n_tiles == 0) return;
  const RasterParams rp = make_params(a);
  if (a.work && a.zero_work) cudaMemsetAsync(a.work, 0, sizeof(uint32_t), s);
  const bool loss = a.loss_partials != nullptr;
  if (counters) {
    if (loss) fwd_shapes<true, true>(a, rp, T_final, last, counters, s);
    else fwd_shapes<true, false>(a, rp, T_final, last, counters, s);
  } else {
    if (loss) fwd_shapes<false, true>(a, rp, T_final, last, counters, s);
    else fwd_shapes<false, false>(a, rp, T_final, last, counters, s);
  }
}

void launch_raster_bwd(const RasterArgs& a, const float* T_final, const int32_t* last, float4* g2d, cudaStream_t s) {
  if (a.n_tiles == 0) return;
  const RasterParams rp = make_params(a);
  if (a.work && a.zero_work) cudaMemsetAsync(a.work, 0, sizeof(uint32_t), s);
  if (a.tile_w == 16) bwd_shape<16, 16>(a, rp, T_final, last, (float*)g2d, s);
  else if (a.tile_w == 8) bwd_shape<8, 32>(a, rp, T_final, last, (float*)g2d, s);
  else bwd_shape<32, 8>(a, rp, T_final, last, (float*)g2d, s);
}

cudaError_t raster_bind_bounds(uint32_t* word) { return bind_bounds_word(word); }

}  // namespace gs
