// Host-side launchers shared between the translation units of libgsplat.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace gs {

struct CamView {
  float fx, fy, cx, cy;
  int width, height;
  float R[9], t[3];
  float C[3];  // camera centre in the world frame, -R^T t
};

// A call renders up to kMaxViews views of one Gaussian map.  Every per-item
// array (projected features, depth keys, tile rectangles, gradient records)
// holds V * n items, item i = v * n + g being Gaussian g seen from view v,
// and the views' tiles are laid end to end: view v owns the global tiles
// [tile_base[v], tile_base[v + 1]), row-major within the view.
constexpr int kMaxViews = 16;

struct TileMap {
  int views;
  int n_per_view;                     // n: Gaussians per view
  int tiles_x[kMaxViews];
  uint32_t tile_base[kMaxViews + 1];  // tile_base[views] = total tiles
};

// Gaussians covering more than this many tiles are queued and expanded by
// whole warps spread over the grid in the binning kernels instead of by the
// block that owns them (large splats cluster, which would leave a few blocks
// running long).
constexpr uint32_t kBigTiles = 32;

struct ProjectArgs {
  uint32_t* big_queue;  // items with more than kBigTiles tiles
  uint32_t* big_len;    // queue length (zeroed before the launch)
  int n;                // Gaussians
  int views;
  const float *means, *log_scales, *quats, *logits, *sh;
  int sh_degree;
  float near_z, dilation, alpha_min;
  int tile_w, tile_h;
  CamView cv[kMaxViews];
  int tiles_x[kMaxViews], tiles_y[kMaxViews];
  uint32_t tile_base[kMaxViews];  // first global tile of each view
  uint32_t* counts;               // per global tile (zeroed, nullable): the projection adds every
                                  // item's tiles
  uint32_t* nvalid = nullptr;     // per view (nullable): zeroed by the projection (block 0)
  // per-tile buckets (nullable; graph-mode binning): every (item, tile) pair
  // is written straight to bucket_ids[tile * bucket_cap + slot], slot taken
  // from the tile's counter (a pair beyond the capacity sets bit 4 of
  // *overflow instead); block 0 zeroes the length-class counters the
  // per-tile sort then fills
  uint32_t* bucket_ids = nullptr;
  uint32_t bucket_cap = 0;
  uint32_t* overflow = nullptr;
  uint32_t* cls_count = nullptr;
  // training step (nullable): block 0 advances the device Adam step that
  // the iteration's fused backward + Adam reads
  long long* step_inc = nullptr;
};

// projection (Eq. 2-5) -> features, depth keys, tile rects, tile counts
void launch_project_fwd(const ProjectArgs& a, float4* feat, uint32_t* depth_key, uint32_t* tiles_touched,
                        ushort4* rects, cudaStream_t s);
// binning-only front end: rects/keys from given mean2d / extent / depth
void launch_bin_prepare(int n, const float* mean2d, const float* extent, const float* depth, int tile_w, int tile_h,
                        int tiles_x, int tiles_y, uint32_t* depth_key, uint32_t* tiles_touched, ushort4* rects,
                        uint32_t* big_queue, uint32_t* big_len, cudaStream_t s);
// g2d [V * n, 12] -> parameter gradients summed over the views (+=) and,
// if pose_partials is non-null, per-block pose partials [blocks][V][6]
int launch_project_bwd(const ProjectArgs& a, float4* g2d, float* g_means, float* g_log_scales,
                       float* g_quats, float* g_logits, float* g_sh, float* pose_partials, cudaStream_t s);
// dL_dpose[v][k] += sum over blocks of partials[b][v][k]
void launch_pose_reduce(const float* partials, int nblocks, int views, float* dL_dpose, cudaStream_t s);

// Adam hyper-parameters as the kernels use them
struct AdamArgs {
  float lr[6];  // means, log-scales, quaternions, opacity, SH DC, SH rest
  float beta1, beta2, eps;
  float step_scale;    // 1 / (1 - beta1^t), when step_dev is null
  float inv_sqrt_bc2;  // 1 / sqrt(1 - beta2^t), when step_dev is null
  const long long* step_dev;  // device step counter (bias corrections computed on the device), or null
  float log_beta1, log_beta2;  // log(beta) for the device-side bias corrections
};
// The training step's loss reduction, done by the fused backward + Adam
// kernel's first blocks before their own work (out nullable): reduction
// block b (of `blocks`; view v's from block_base[v]) sums kLossChunk
// consecutive (tile, 8 x 8 block) partials {|colour residual|, |depth
// residual| over valid targets, valid count} of one view, starting at
// job_base[v] + (b - block_base[v]) kLossChunk, into blk[3 b + k] in a fixed
// order; the block completing the last one (ticket: 0 between launches)
// sums them per view into *out and the depth scales scale[v].
struct LossFoldArgs {
  const float* partials;
  float* blk;
  float* out;
  float* scale;
  uint32_t* ticket;
  float w_color, w_depth;
  int views, blocks;
  int block_base[kMaxViews + 1];
  uint32_t job_base[kMaxViews + 1];
  float npix[kMaxViews];
};
constexpr int kLossChunk = 2048;
// device step counter: *step += 1
void launch_step_increment(long long* step, cudaStream_t s);
// set once per context: shared-memory limits of the fused kernel
void init_project_kernels();
// fused projection backward + Adam over the flat buffer (gradients summed
// over the views, one step)
int launch_project_bwd_adam(const ProjectArgs& a, float4* g2d, float* params, float* m, float* v,
                            const AdamArgs& ad, float* pose_partials, cudaStream_t s,
                            const LossFoldArgs* loss = nullptr);
int project_bwd_blocks(int n);

// Stable radix sort of (u32 key, u32 value) pairs on the low `bits` bits.
// The first pass reads (in_k, in_v) -- in_v == nullptr means value = index --
// and later passes ping-pong between the two buffers of `b`.  If in_k is
// b.keys[0] the sort runs in place.  Returns the index (0 or 1) of the buffer
// holding the result, or -1 if no pass ran and the input is the result.
// n is read from n_dev when non-null (grid sized from n_max).
struct SortBuffers {
  uint32_t* keys[2];
  uint32_t* vals[2];
  uint32_t* hist;   // scratch, >= 256 * (max_blocks + 1): per-block digit counts, then digit totals
  int max_blocks;
};
int radix_sort_pairs(SortBuffers& b, const uint32_t* in_k, const uint32_t* in_v, uint32_t n_max,
                     const uint32_t* n_dev, int bits, int num_sms, cudaStream_t s, int64_t* launches);

// pair generation: per depth-sorted Gaussian, its tiles in row-major order
struct DupArgs {
  int n;
  const uint32_t* sorted_ids;
  const uint32_t* tiles_touched;
  const ushort4* rects;
  TileMap map;
  uint32_t* block_sums;  // scratch >= dup_blocks(n) + 1
  uint32_t* n_pairs;     // device total (clamped to capacity for the kernels)
  unsigned long long* n_pairs_full;  // device total before clamping
  uint32_t* tile_keys;
  uint32_t* vals;
  uint32_t capacity;
  uint32_t* overflow;
};
int dup_blocks(int n);
void launch_dup_count_scan(const DupArgs& a, cudaStream_t s, int64_t* launches);
void launch_dup_write(const DupArgs& a, cudaStream_t s, int64_t* launches);

// counting-scatter binning with per-tile sorts (lists of at most kTileSortCap)
constexpr int kTileSortCap = 4096;
// graph-mode binning: entries of a tile's bucket (the projection writes the
// pairs straight into per-tile buckets, no scan and no scatter), a power of
// two from kBucketCapMin to kBucketCapMax (the per-tile sort's limit) chosen
// per context
constexpr uint32_t kBucketCapMin = 1024;
constexpr uint32_t kBucketCapMax = 4096;
static_assert(kBucketCapMax <= (uint32_t)kTileSortCap, "a full bucket is sorted by the per-tile sort");
// length classes of the raster passes' visit order (four per octave)
constexpr int kLenClasses = 129;

// Turns the class counts cls[0 .. kLenClasses) into the first visit position
// of each class, longest class first (cls[c] = sum of the counts of the
// classes above c); run by one warp.
__device__ __forceinline__ void class_starts_desc(uint32_t* cls) {
  constexpr int PER = (kLenClasses + 31) / 32;
  const int lane = threadIdx.x & 31;
  // lane l takes classes kLenClasses - 1 - (PER l .. PER l + PER - 1)
  uint32_t v[PER], sum = 0;
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    const int c = kLenClasses - 1 - (PER * lane + j);
    v[j] = c >= 0 ? cls[c] : 0u;
    sum += v[j];
  }
  uint32_t incl = sum;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, off);
    if (lane >= off) incl += y;
  }
  uint32_t run = incl - sum;
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    const int c = kLenClasses - 1 - (PER * lane + j);
    if (c >= 0) cls[c] = run;
    run += v[j];
  }
}
struct TileBinArgs {
  int n;                      // items (views x Gaussians)
  const ushort4* rects;       // per item tile rectangle (view-local tile coordinates)
  const uint32_t* tiles;      // per item tile count
  const uint32_t* zkey;       // per item float32 depth bits
  TileMap map;
  int n_tiles, num_sms;
  uint32_t* counts;           // per tile
  uint32_t* offsets;          // per tile
  uint32_t* cursors;          // per tile
  uint32_t* ids;              // per pair: item (output, sorted per tile)
  uint2* ranges;              // per tile (output)
  uint32_t capacity;          // pair slots in ids
  uint32_t* n_pairs;          // device: min(total, capacity)
  unsigned long long* stats;  // device: [0] total pairs, [1] longest list
  uint32_t* overflow;         // device flag: 1 = pairs over capacity, 2 = list over kTileSortCap
  const uint32_t* big_queue;  // items with more than kBigTiles tiles
  const uint32_t* big_len;    // queue length (the per-tile sort zeroes it, and the counts, when done)
  uint32_t* order;            // per tile (output, nullable): visit order, longest lists first
  bool counted;               // counts already hold every item's tiles (the projection counted them)
  uint32_t* scan_aux;         // scratch of tile_scan_aux_size(n_tiles) words for the multi-block scan
  uint32_t* raster_work = nullptr;  // nullable: the forward and backward raster job counters, zeroed by the sort
  // bucket mode (nullable): the lists are the projection's per-tile buckets
  // (bucket_ids, tile t's list at t * bucket_cap, its length in counts[t]);
  // the sort files each tile under its length class (class 0: empty),
  // cls_tiles[c * cls_stride + i] for i < cls_count[c], from which the
  // forward raster pass takes its visit order (see RasterArgs)
  uint32_t* bucket_ids = nullptr;
  uint32_t bucket_cap = 0;
  uint32_t* cls_count = nullptr;
  uint32_t* cls_tiles = nullptr;
  uint32_t cls_stride = 0;
};
int tile_sort_capacity();
int64_t tile_scan_aux_size(int64_t n_tiles);
void launch_tile_count_scan(const TileBinArgs& a, cudaStream_t s, int64_t* launches);
void launch_tile_scatter(const TileBinArgs& a, cudaStream_t s, int64_t* launches);
void launch_tile_sort(const TileBinArgs& a, cudaStream_t s, int64_t* launches);

void launch_tile_ranges(const uint32_t* sorted_tiles, const uint32_t* n_dev, uint32_t n_max, uint2* ranges,
                        int n_tiles, int num_sms, cudaStream_t s, int64_t* launches);

// raster passes: one CTA per global tile, visited in `order` when given
// (the tile list sorted by descending list length) else in index order
struct RasterView {
  int width, height, tiles_x;
  uint32_t tile_base;  // first global tile of the view
  int64_t pix_base;    // first pixel of the view in the T_final / last buffers
  float *color, *depth, *alpha;           // forward outputs (each nullable)
  const float *dLdc, *dLdd, *dLda;        // backward inputs (dLda nullable)
  // forward with the fused loss: targets in, image gradients out (dLdd
  // unscaled: the sign of the depth residual, 0 where the target is invalid)
  const float *trgb, *tdep;
  float *loss_dc, *loss_dd;
};
struct RasterArgs {
  int views, tile_w, tile_h;
  uint32_t n_tiles;
  float bg[3];
  float alpha_max, alpha_min, t_eps;
  const uint2* ranges;
  const uint32_t* ids;
  const float4* feat;
  uint32_t n_ids, n_items;  // entries of ids, records of feat (bounds of the checked build)
  const uint32_t* order;  // nullable
  uint32_t* work;         // nullable: job counter of the persistent form
  bool zero_work;         // the launcher zeroes *work first (it is not known to be 0)
  int num_sms;
  // fused loss (forward): per (tile, 8 x 8 block) partial sums {|colour
  // residual|, |depth residual| over valid targets, valid count} at
  // loss_partials[3 (4 tile + block) + i]; null = no loss
  float* loss_partials;
  float w_color;
  // backward: dL/dD = dLdd * depth_scale[v] when non-null (the scale the
  // fused loss finalises on the device)
  const float* depth_scale;
  // fused loss: the forward pass adds each warp block's count of valid
  // target depths to nvalid[v] (exact integers); given to the backward pass,
  // dL/dD = dLdd * w_depth / max(nvalid[v], 1), the same scale the loss
  // reduction computes (it takes precedence over depth_scale)
  uint32_t* nvalid;
  float w_depth;
  // bucket-mode visit order (forward pass, nullable): the tiles of length
  // class c are cls_tiles[c * cls_stride + i] for i < cls_count[c]; visit k
  // takes the longest classes first (each CTA turns the class counts into
  // class starts once), and the warp that takes block 0 of visit k writes
  // its tile to order_out[k], the flat order the backward pass reads
  const uint32_t* cls_count;
  const uint32_t* cls_tiles;
  uint32_t cls_stride;
  uint32_t* order_out;
  RasterView v[kMaxViews];
};
bool raster_shape_supported(int tw, int th);
// bounds-checked build: point the translation unit's kernels at the
// context's bounds word (no-op in the normal build)
cudaError_t raster_bind_bounds(uint32_t* word);
cudaError_t tilebin_bind_bounds(uint32_t* word);
void launch_raster_fwd(const RasterArgs& a, float* T_final, int32_t* last, unsigned long long* counters,
                       cudaStream_t s);
// loss from the forward pass's per-block partials: loss = sum over views of
// w_color sum|rc| / (3 npix_v) + w_depth sum|rd| / nvalid_v; depth_scale[v] =
// w_depth / nvalid_v (fixed summation order)
// partials: scratch of >= 3 * (4 n_tiles / 2048 + views) floats; ticket: a
// device word that is 0 between launches (one launch; its last block
// finalises and resets it); step (nullable): the device Adam step counter,
// advanced by one after the loss is final
void launch_loss_tiles_finalize(const RasterArgs& a, float w_depth, float* loss, float* depth_scale,
                                float* partials, uint32_t* ticket, long long* step, cudaStream_t s,
                                int64_t* launches);
void launch_raster_bwd(const RasterArgs& a, const float* T_final, const int32_t* last, float4* g2d, cudaStream_t s);

// loss and optimiser: per view v, L_v = w_color mean |C - C^| + w_depth
// mean over valid target depths |D - D^|; loss = sum over views of L_v
struct LossView {
  int npix;
  int block_base;  // first partials block of the view
  const float *color, *depth, *trgb, *tdep;
  float *dLdc, *dLdd;
};
struct LossArgs {
  int views, n_blocks;
  float w_color, w_depth;
  float* loss;
  LossView v[kMaxViews];
};
int loss_blocks(int npix);
// partials: >= 3 * n_blocks + kMaxViews floats
void launch_loss(const LossArgs& a, float* partials, cudaStream_t s, int64_t* launches);
// step_dev non-null: bias corrections from the device step counter instead
// of step_size_scale / inv_sqrt_bc2
void launch_adam(float* p, float* g, float* m, float* v, int64_t n_gauss, int sh_degree, const float lr[6],
                 float beta1, float beta2, float eps, float step_size_scale, float inv_sqrt_bc2, bool zero_grads,
                 const long long* step_dev, cudaStream_t s);

// TSDF grid (Sec. III-B.1): hash table of 8^3-voxel blocks over a slot pool.
// Mirrors gs_tsdf_grid; counters: [0] blocks (next slot), [1] buckets
// touched by the last allocation, [2] insert / list failures, [3] voxels
// updated.
struct TsdfGrid {
  unsigned long long* keys;  // [table_size], ~0 = free
  int32_t* slots;            // [table_size]
  uint32_t* stamps;          // [table_size] last frame that touched the bucket
  float* voxels;             // [capacity][512] float2 (tsdf, weight)
  uint32_t* claims;          // [capacity][512], ~0 between calls
  uint32_t* touched;         // [table_size / 2] buckets
  uint32_t* counters;        // [4]
  int64_t table_size, capacity;
  float voxel_size, truncation, max_weight;
  int fusion;  // 0: Eq. 9 as printed, 1: unit measurement weight
};

struct TsdfCamera {
  float fx, fy, cx, cy;
  int W, H;
  float R[9], t[3];  // world-to-camera, R row-major
};

constexpr int kTsdfMaxSamples = 16;  // band samples per ray
int tsdf_band_steps(float eps, float s);
int64_t tsdf_alloc_smem_bytes(float eps, float s);
void launch_tsdf_alloc(const TsdfGrid& g, const float* depth, const TsdfCamera& c, uint32_t frame, cudaStream_t s);
void launch_tsdf_integrate(const TsdfGrid& g, const float* depth, const TsdfCamera& c, int64_t min_slot,
                           int num_sms, cudaStream_t s);
void launch_tsdf_rehash(const TsdfGrid& from, const TsdfGrid& to, int num_sms, cudaStream_t s);
void launch_tsdf_query(const TsdfGrid& g, const float* points, int64_t n, float* tsdf, float* weight,
                       cudaStream_t s);
// claim + seed kernels over the leaves; leaf_claim: n_leaves scratch words
void launch_tsdf_seed(const TsdfGrid& g, const float* rgb, const float* depth, int W, int H, const float K4[4],
                      const float R[9], const float t[3], int sh_degree, const int4* leaves, uint32_t n_leaves,
                      int64_t* leaf_claim, float* means, float* log_scales, float* quats, float* logits, float* sh,
                      uint32_t capacity, uint32_t* n_seeded, cudaStream_t s);

// per-frame seeding (quadtree + Eq. 10); counters: >= levels + 2 words;
// cells_a / cells_b / leaves: quadtree_scratch_cells(W, H) entries each;
// pyramid: quadtree_pyramid_doubles(W, H, max_size) doubles.  Returns the
// number of kernels launched.
int64_t quadtree_scratch_cells(int W, int H);
int64_t quadtree_pyramid_doubles(int W, int H, int max_size);
int launch_quadtree(const float* rgb, int W, int H, int max_size, int min_size, double var_thr, int2* cells_a,
                    int2* cells_b, uint32_t* counters, int4* leaves, double* pyramid, cudaStream_t s);
// K4 = (fx, fy, cx, cy); R, t world-to-camera
void launch_seed(const float* rgb, const float* depth, const float* alpha, float alpha_thr, int W, int H,
                 const float K4[4], const float R[9], const float t[3], int sh_degree, const int4* leaves,
                 uint32_t n_leaves, float* means, float* log_scales, float* quats, float* logits, float* sh,
                 uint32_t capacity, uint32_t* n_seeded, cudaStream_t s);

// debug/introspection
void launch_export_projection(int n, const float4* feat, const uint32_t* tiles, float* mean2d, float* cov2d,
                              float* depth, float* rgb, float* opacity, int32_t* tiles_out, cudaStream_t s);
void launch_export_keys(const uint32_t* sorted_tiles, const uint32_t* sorted_ids, const uint32_t* depth_key_by_id,
                        uint32_t P, uint64_t* keys, uint32_t* ids, cudaStream_t s);
// same, taking the tile of each pair from the per-tile ranges
void launch_export_keys_ranges(const uint2* ranges, int n_tiles, const uint32_t* sorted_ids,
                               const uint32_t* depth_key_by_id, uint32_t P, uint64_t* keys, uint32_t* ids,
                               cudaStream_t s);

// out (device) = number of non-finite floats in x[0, n)
void launch_count_nonfinite(const float* x, int64_t n, unsigned long long* out, int num_sms, cudaStream_t s);

}  // namespace gs
