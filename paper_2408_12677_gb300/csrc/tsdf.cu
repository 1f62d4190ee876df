// TSDF fusion (Sec. III-B.1, Eq. 6-9) on a voxel-hashed grid, and the
// voxel-weight novelty check of the per-frame seeding (Sec. III-B.2).
//
// The grid is single resolution: voxels of side s in blocks of 8^3 (the leaf
// blocks of the octree the paper builds on).  Instead of an octree the blocks
// are found through an open-addressing hash table (linear probing) keyed by
// the packed block coordinates; a block's voxels live in a pool slot of 512
// float2 (tsdf, weight), x fastest, so one warp reads 256 contiguous bytes.
//
// One frame is two launches:
//  * allocation: one CTA per 16 x 16 pixel tile samples every pixel's ray in
//    the +-eps band and collects the distinct block keys of its tile in a
//    shared-memory set first (neighbouring rays hit the same blocks), so the
//    global table sees one probe per (tile, block) instead of one per sample.
//    New keys take the next pool slot; every bucket the frame touches is
//    listed once through a per-bucket frame stamp.
//  * integration: a persistent grid walks the touched list, a CTA per block,
//    a thread per two voxels: Eq. 6-9 with the running average of Eq. 9.
// The integer decisions (block of a sample, pixel of a voxel, whether a voxel
// is updated) use float32 with a fixed order of correctly rounded operations
// (no contraction), the tsdf arithmetic plain float32.
#include <algorithm>
#include <cfloat>
#include <cmath>

#include "common.cuh"
#include "internal.h"
#include "seed.cuh"

namespace gs {

namespace {

constexpr unsigned long long kEmptyKey = ~0ull;
constexpr int kKeyBias = 1 << 20;  // block coordinates in [-2^20, 2^20)
constexpr int kAllocTile = 16;
constexpr int kAllocThreads = kAllocTile * kAllocTile;
constexpr int kIntegrateThreads = 256;
constexpr int kVoxels = 512;

struct Band {
  float c[kTsdfMaxSamples];  // camera-depth offsets of the samples from D
  int n;                     // samples
};

__device__ __forceinline__ bool pack_key(const int b[3], unsigned long long* key) {
#pragma unroll
  for (int a = 0; a < 3; ++a)
    if (b[a] < -kKeyBias || b[a] >= kKeyBias) return false;
  *key = ((unsigned long long)(b[0] + kKeyBias) << 42) | ((unsigned long long)(b[1] + kKeyBias) << 21) |
         (unsigned long long)(b[2] + kKeyBias);
  return true;
}

__device__ __forceinline__ void unpack_key(unsigned long long key, int b[3]) {
  b[0] = (int)((key >> 42) & 0x1FFFFF) - kKeyBias;
  b[1] = (int)((key >> 21) & 0x1FFFFF) - kKeyBias;
  b[2] = (int)(key & 0x1FFFFF) - kKeyBias;
}

// the finaliser of the splitmix64 generator (Steele, Lea and Flood, 2014)
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// bucket of `key`, inserting it (with the next pool slot) if absent; -1 if
// the table has no free bucket
__device__ int64_t insert_key(const TsdfGrid& g, unsigned long long key) {
  const unsigned long long mask = (unsigned long long)g.table_size - 1;
  unsigned long long h = mix64(key) & mask;
  for (int64_t p = 0; p < g.table_size; ++p, h = (h + 1) & mask) {
    unsigned long long cur = __ldcg(g.keys + h);
    if (cur == kEmptyKey) {
      cur = atomicCAS(g.keys + h, kEmptyKey, key);
      if (cur == kEmptyKey) {
        g.slots[h] = (int32_t)atomicAdd(g.counters + 0, 1u);
        return (int64_t)h;
      }
    }
    if (cur == key) return (int64_t)h;
  }
  return -1;
}

// bucket of `key` or -1 (read-only: the table does not change during the call)
__device__ int64_t find_key(const TsdfGrid& g, unsigned long long key) {
  const unsigned long long mask = (unsigned long long)g.table_size - 1;
  unsigned long long h = mix64(key) & mask;
  for (int64_t p = 0; p < g.table_size; ++p, h = (h + 1) & mask) {
    const unsigned long long cur = g.keys[h];
    if (cur == key) return (int64_t)h;
    if (cur == kEmptyKey) return -1;
  }
  return -1;
}

__device__ __forceinline__ float block_of(float p, float side, bool* ok) {
  const float f = floorf(__fdiv_rn(p, side));
  *ok = *ok && fabsf(f) < (float)kKeyBias;  // also rejects NaN
  return f;
}

__global__ void __launch_bounds__(kAllocThreads) tsdf_alloc_kernel(const __grid_constant__ TsdfGrid g,
                                                                   const float* __restrict__ depth,
                                                                   const __grid_constant__ TsdfCamera c,
                                                                   const __grid_constant__ Band band,
                                                                   uint32_t frame, int set_size) {
  extern __shared__ unsigned long long s_set[];
  for (int e = threadIdx.x; e < set_size; e += kAllocThreads) s_set[e] = kEmptyKey;
  __syncthreads();
  const int i = blockIdx.x * kAllocTile + (threadIdx.x % kAllocTile);
  const int j = blockIdx.y * kAllocTile + (threadIdx.x / kAllocTile);
  float D = 0.f;
  if (i < c.W && j < c.H) D = depth[(size_t)j * c.W + i];
  const bool valid = D > 0.f && D <= FLT_MAX;
  const float xn = __fdiv_rn(__fsub_rn(__fadd_rn((float)i, 0.5f), c.cx), c.fx);
  const float yn = __fdiv_rn(__fsub_rn(__fadd_rn((float)j, 0.5f), c.cy), c.fy);
  const float side = __fmul_rn(8.f, g.voxel_size);
  const unsigned lane = threadIdx.x & 31;
  // every lane runs all samples (invalid ones carry the empty key) so that
  // the warp can merge equal keys before they reach shared memory: the rays
  // of a warp mostly sample the same few blocks
  for (int k = 0; k < band.n; ++k) {
    unsigned long long key = kEmptyKey;
    const float z = __fadd_rn(D, band.c[k]);
    if (valid && z > 0.f) {
      const float d0 = __fsub_rn(__fmul_rn(xn, z), c.t[0]);
      const float d1 = __fsub_rn(__fmul_rn(yn, z), c.t[1]);
      const float d2 = __fsub_rn(z, c.t[2]);
      bool ok = true;
      int b[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const float pw = __fadd_rn(__fadd_rn(__fmul_rn(c.R[a], d0), __fmul_rn(c.R[3 + a], d1)),
                                   __fmul_rn(c.R[6 + a], d2));
        b[a] = (int)block_of(pw, side, &ok);
      }
      if (!ok || !pack_key(b, &key)) key = kEmptyKey;
    }
    const unsigned peers = __match_any_sync(0xFFFFFFFFu, key);
    if (key == kEmptyKey || lane != (unsigned)(__ffs(peers) - 1)) continue;
    // the set holds at most kAllocThreads * band.n keys in >= twice as many
    // entries, so the probe always ends
    unsigned h = (unsigned)mix64(key) & (unsigned)(set_size - 1);
    for (int p = 0; p < set_size; ++p, h = (h + 1) & (unsigned)(set_size - 1)) {
      const unsigned long long cur = *(volatile unsigned long long*)(s_set + h);
      if (cur == key) break;
      if (cur == kEmptyKey) {
        const unsigned long long prev = atomicCAS(s_set + h, kEmptyKey, key);
        if (prev == kEmptyKey || prev == key) break;
      }
    }
  }
  __syncthreads();
  const uint32_t touched_cap = (uint32_t)(g.table_size / 2);
  for (int e = threadIdx.x; e < set_size; e += kAllocThreads) {
    const unsigned long long key = s_set[e];
    if (key == kEmptyKey) continue;
    const int64_t h = insert_key(g, key);
    if (h < 0) {
      atomicAdd(g.counters + 2, 1u);
      continue;
    }
    if (atomicExch(g.stamps + h, frame) != frame) {
      const uint32_t idx = atomicAdd(g.counters + 1, 1u);
      if (idx < touched_cap)
        g.touched[idx] = (uint32_t)h;
      else
        atomicAdd(g.counters + 2, 1u);
    }
  }
}

__global__ void __launch_bounds__(kIntegrateThreads) tsdf_integrate_kernel(const __grid_constant__ TsdfGrid g,
                                                                           const float* __restrict__ depth,
                                                                           const __grid_constant__ TsdfCamera c,
                                                                           int64_t min_slot) {
  const uint32_t n = min(__ldcg(g.counters + 1), (uint32_t)(g.table_size / 2));
  const float s = g.voxel_size, eps = g.truncation, wmax = g.max_weight;
  const float Wf = (float)c.W, Hf = (float)c.H;
  uint32_t updated = 0;
  for (uint32_t it = blockIdx.x; it < n; it += gridDim.x) {
    const uint32_t h = g.touched[it];
    const int64_t slot = g.slots[h];
    if (slot >= g.capacity || slot < min_slot) continue;
    int b[3];
    unpack_key(g.keys[h], b);
    float2* vox = reinterpret_cast<float2*>(g.voxels) + (size_t)slot * kVoxels;
#pragma unroll
    for (int r = 0; r < kVoxels / kIntegrateThreads; ++r) {
      const int v = threadIdx.x + r * kIntegrateThreads;
      const float px = __fmul_rn(__fadd_rn((float)(8 * b[0] + (v & 7)), 0.5f), s);
      const float py = __fmul_rn(__fadd_rn((float)(8 * b[1] + ((v >> 3) & 7)), 0.5f), s);
      const float pz = __fmul_rn(__fadd_rn((float)(8 * b[2] + (v >> 6)), 0.5f), s);
      const float xc = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(c.R[0], px), __fmul_rn(c.R[1], py)),
                                           __fmul_rn(c.R[2], pz)), c.t[0]);
      const float yc = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(c.R[3], px), __fmul_rn(c.R[4], py)),
                                           __fmul_rn(c.R[5], pz)), c.t[1]);
      const float zc = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(c.R[6], px), __fmul_rn(c.R[7], py)),
                                           __fmul_rn(c.R[8], pz)), c.t[2]);
      if (!(zc > 0.f)) continue;
      const float u = __fadd_rn(__fmul_rn(c.fx, __fdiv_rn(xc, zc)), c.cx);
      const float w = __fadd_rn(__fmul_rn(c.fy, __fdiv_rn(yc, zc)), c.cy);
      if (!(u >= 0.f && u < Wf && w >= 0.f && w < Hf)) continue;
      const float D = __ldg(depth + (size_t)(int)floorf(w) * c.W + (int)floorf(u));
      if (!(D > 0.f)) continue;
      const float sdf = __fsub_rn(D, zc);
      if (!(sdf >= -eps)) continue;
      // Eq. 7-9
      const float x = sdf > 0.f ? fminf(1.f, sdf / eps) : fmaxf(-1.f, sdf / eps);
      const float2 o = vox[v];
      const float w1 = fminf(wmax, o.y + 1.f);
      const float tn = g.fusion == 0 ? (o.x * o.y + x * w1) / (o.y + w1) : (o.x * o.y + x) / (o.y + 1.f);
      vox[v] = make_float2(tn, w1);
      ++updated;
    }
  }
  // updated voxels, one atomic per warp
  for (int off = 16; off > 0; off >>= 1) updated += __shfl_xor_sync(0xFFFFFFFFu, updated, off);
  if ((threadIdx.x & 31) == 0 && updated) atomicAdd(g.counters + 3, updated);
}

__global__ void tsdf_rehash_kernel(const __grid_constant__ TsdfGrid from, const __grid_constant__ TsdfGrid to) {
  const unsigned long long mask = (unsigned long long)to.table_size - 1;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < from.table_size;
       e += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long key = from.keys[e];
    if (key == kEmptyKey) continue;
    unsigned long long h = mix64(key) & mask;
    for (int64_t p = 0; p < to.table_size; ++p, h = (h + 1) & mask) {
      if (atomicCAS(to.keys + h, kEmptyKey, key) == kEmptyKey) {
        to.slots[h] = from.slots[e];
        break;
      }
    }
  }
}

// voxel (and its pool index) holding world point p: floor(p / s) in float32
__device__ __forceinline__ int64_t voxel_index(const TsdfGrid& g, const float p[3]) {
  int b[3], l[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float f = floorf(__fdiv_rn(p[a], g.voxel_size));
    if (!(fabsf(f) < 8.f * (float)kKeyBias)) return -1;
    const int v = (int)f;
    l[a] = v & 7;
    b[a] = (v - l[a]) / 8;
  }
  unsigned long long key;
  if (!pack_key(b, &key)) return -1;
  const int64_t h = find_key(g, key);
  if (h < 0) return -1;
  const int64_t slot = g.slots[h];
  if (slot >= g.capacity) return -1;
  return slot * kVoxels + l[0] + 8 * l[1] + 64 * l[2];
}

__global__ void tsdf_query_kernel(const __grid_constant__ TsdfGrid g, const float* __restrict__ points, int64_t n,
                                  float* __restrict__ tsdf, float* __restrict__ weight) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float p[3] = {points[3 * i], points[3 * i + 1], points[3 * i + 2]};
  const int64_t v = voxel_index(g, p);
  const float2 o = v >= 0 ? reinterpret_cast<const float2*>(g.voxels)[v] : make_float2(0.f, 0.f);
  if (tsdf) tsdf[i] = o.x;
  if (weight) weight[i] = o.y;
}

// novelty check: a leaf whose Eq. 10 point lies in a voxel of weight 1 bids
// for that voxel with its key y0 W + x0 (smallest wins)
__global__ void __launch_bounds__(256) tsdf_claim_kernel(const __grid_constant__ SeedArgs a,
                                                         const __grid_constant__ TsdfGrid g,
                                                         const int4* __restrict__ leaves, uint32_t n_leaves,
                                                         int64_t* __restrict__ leaf_claim) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_leaves) return;
  const int4 L = leaves[i];
  float ux, uy;
  const size_t pix = leaf_pixel(a, L, &ux, &uy);
  const float z = a.depth[pix];
  int64_t v = -1;
  if (z > 0.f) {
    float p[3];
    leaf_point(a, ux, uy, z, p);
    v = voxel_index(g, p);
    if (v >= 0 && reinterpret_cast<const float2*>(g.voxels)[v].y == 1.f)
      atomicMin(g.claims + v, (uint32_t)L.y * (uint32_t)a.W + (uint32_t)L.x);
    else
      v = -1;
  }
  leaf_claim[i] = v;
}

// the winners seed (Eq. 10) and give their voxel's claim back
__global__ void __launch_bounds__(256) tsdf_seed_kernel(const __grid_constant__ SeedArgs a,
                                                        const __grid_constant__ TsdfGrid g,
                                                        const int4* __restrict__ leaves, uint32_t n_leaves,
                                                        const int64_t* __restrict__ leaf_claim,
                                                        uint32_t* __restrict__ n_seeded) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t v = i < n_leaves ? leaf_claim[i] : -1;
  int4 L = make_int4(0, 0, 1, 1);
  bool wins = false;
  if (v >= 0) {
    L = leaves[i];
    wins = g.claims[v] == (uint32_t)L.y * (uint32_t)a.W + (uint32_t)L.x;
  }
  const unsigned m = __ballot_sync(0xFFFFFFFFu, wins);
  if (!wins) return;
  g.claims[v] = 0xFFFFFFFFu;
  const uint32_t k = warp_agg_inc(n_seeded, 0u, m);  // one atomic per warp
  if (k >= a.capacity) return;
  float ux, uy;
  const size_t pix = leaf_pixel(a, L, &ux, &uy);
  const float z = a.depth[pix];
  float p[3];
  leaf_point(a, ux, uy, z, p);
  write_seed(a, k, L, pix, p, z);
}

Band make_band(float eps, float s) {
  Band b;
  b.n = tsdf_band_steps(eps, s) + 1;
  const double e = (double)eps;
  const int n = b.n - 1;
  for (int k = 0; k < kTsdfMaxSamples; ++k) b.c[k] = k <= n ? (float)(-e + (double)k * (2.0 * e / n)) : 0.f;
  return b;
}

int set_entries(int samples) {
  int e = 1;
  while (e < 2 * kAllocThreads * samples) e <<= 1;
  return e;
}

}  // namespace

int tsdf_band_steps(float eps, float s) {
  return std::max(1, (int)std::ceil((double)eps / (2.0 * (double)s) - 1e-6));
}

int64_t tsdf_alloc_smem_bytes(float eps, float s) {
  return (int64_t)set_entries(tsdf_band_steps(eps, s) + 1) * (int64_t)sizeof(unsigned long long);
}

void launch_tsdf_alloc(const TsdfGrid& g, const float* depth, const TsdfCamera& c, uint32_t frame, cudaStream_t s) {
  const Band band = make_band(g.truncation, g.voxel_size);
  const int set = set_entries(band.n);
  // per device and cheap: set on every launch
  cudaFuncSetAttribute(tsdf_alloc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)(set_entries(kTsdfMaxSamples) * sizeof(unsigned long long)));
  const dim3 grid((c.W + kAllocTile - 1) / kAllocTile, (c.H + kAllocTile - 1) / kAllocTile);
  tsdf_alloc_kernel<<<grid, kAllocThreads, set * sizeof(unsigned long long), s>>>(g, depth, c, band, frame, set);
}

void launch_tsdf_integrate(const TsdfGrid& g, const float* depth, const TsdfCamera& c, int64_t min_slot,
                           int num_sms, cudaStream_t s) {
  // 8 CTAs of 256 threads per SM walk the touched list
  tsdf_integrate_kernel<<<8 * num_sms, kIntegrateThreads, 0, s>>>(g, depth, c, min_slot);
}

void launch_tsdf_rehash(const TsdfGrid& from, const TsdfGrid& to, int num_sms, cudaStream_t s) {
  tsdf_rehash_kernel<<<8 * num_sms, 256, 0, s>>>(from, to);
}

void launch_tsdf_query(const TsdfGrid& g, const float* points, int64_t n, float* tsdf, float* weight,
                       cudaStream_t s) {
  if (n <= 0) return;
  tsdf_query_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(g, points, n, tsdf, weight);
}

void launch_tsdf_seed(const TsdfGrid& g, const float* rgb, const float* depth, int W, int H, const float K4[4],
                      const float R[9], const float t[3], int sh_degree, const int4* leaves, uint32_t n_leaves,
                      int64_t* leaf_claim, float* means, float* log_scales, float* quats, float* logits, float* sh,
                      uint32_t capacity, uint32_t* n_seeded, cudaStream_t s) {
  cudaMemsetAsync(n_seeded, 0, sizeof(uint32_t), s);
  if (n_leaves == 0) return;
  const SeedArgs a = make_seed_args(rgb, depth, nullptr, 0.f, W, H, K4, R, t, sh_degree, means, log_scales, quats,
                                    logits, sh, capacity);
  const unsigned blocks = (n_leaves + 255) / 256;
  tsdf_claim_kernel<<<blocks, 256, 0, s>>>(a, g, leaves, n_leaves, leaf_claim);
  tsdf_seed_kernel<<<blocks, 256, 0, s>>>(a, g, leaves, n_leaves, leaf_claim, n_seeded);
}

}  // namespace gs
