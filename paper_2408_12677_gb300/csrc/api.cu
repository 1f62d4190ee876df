// C ABI of libgsplat: context and scratch management, argument checks and
// the orchestration of the projection, binning, raster, loss and Adam
// kernels.  See include/gsplat.h for the contract of every entry point.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/gsplat.h"
#include "common.cuh"
#include "internal.h"

using namespace gs;

// the forward state is matched by comparing these structs byte for byte
static_assert(sizeof(gs_camera) == 24 && sizeof(gs_viewmat) == 48 && sizeof(gs_raster_cfg) == 44,
              "ABI structs without padding");

struct gs_ctx {
  int device = 0;
  int num_sms = 0;
  std::string err;
  bool sync = true;
  int64_t launches = 0;
  int fail_alloc = 0;  // > 0: the fail_alloc-th next scratch growth fails (GS_ERR_OOM)
  unsigned long long* d_count = nullptr;  // gs_count_nonfinite

  // per-Gaussian scratch
  int64_t cap_n = 0;
  float4* feat = nullptr;
  uint32_t* zkey = nullptr;  // per-Gaussian depth key (float32 bits of z)
  uint32_t* dkey[2] = {nullptr, nullptr};
  uint32_t* dval[2] = {nullptr, nullptr};
  uint32_t* tiles = nullptr;
  ushort4* rects = nullptr;
  float4* g2d = nullptr;
  uint32_t* dup_sums = nullptr;
  float* pose_partials = nullptr;
  // per-pair scratch
  int64_t cap_p = 0;
  uint32_t* pk[2] = {nullptr, nullptr};
  uint32_t* pv[2] = {nullptr, nullptr};
  // radix histograms
  uint32_t* hist = nullptr;
  int hist_blocks = 0;
  // per-tile / per-pixel scratch
  int64_t cap_t = 0;
  uint2* ranges = nullptr;
  uint32_t* tcount = nullptr;   // per-tile pair counts
  uint32_t* toffset = nullptr;  // per-tile list offsets
  uint32_t* tcursor = nullptr;  // per-tile scatter cursors
  uint32_t* torder = nullptr;   // raster visit order of the tiles (longest lists first)
  uint32_t* scan_aux = nullptr;  // multi-block tile scan scratch
  uint32_t* bigq = nullptr;     // ids of Gaussians covering more than kBigTiles tiles
  uint32_t* d_bigmeta = nullptr;  // [0] length of the large-splat queue, [1] / [2] forward / backward raster
                                  // job counters, [3] ticket of the fused-loss reduction (0 between launches)
  bool counts_zero = false;       // the tile counters and the large-splat queue length are 0 (the per-tile
                                  // sort, the last binning kernel, zeroes them)
  bool fwd_work_zero = false;     // the forward / backward raster job counters are 0 (the per-tile sort zeroes
  bool bwd_work_zero = false;     // both; a raster launch uses its counter up)
  bool g2d_zero = false;          // the gradient records are all 0 (their consumers clear what they read)
  unsigned long long* d_binstats = nullptr;  // [0] total pairs, [1] longest tile list
  long long* d_step = nullptr;               // device Adam step counter (step = 0 calls)
  int64_t cap_px = 0;
  float* T_final = nullptr;
  int32_t* last = nullptr;
  float* loss_partials = nullptr;
  float* tune_img = nullptr;  // zero image gradients for the autotuner
  float* dl_img = nullptr;    // per pixel: dL/dcolor (3 planes) and the depth residual sign (fused loss)
  float* tile_loss = nullptr;  // per (tile, 8 x 8 block): fused-loss partial sums (3 floats)
  float* d_dscale = nullptr;   // per view: depth-gradient scale of the fused loss
  uint32_t* d_nvalid = nullptr;  // per view: target depths > 0 seen by the fused-loss forward pass
  // per-frame seeding scratch
  int64_t cap_qt = 0;
  int2* qt_cells[2] = {nullptr, nullptr};
  int4* qt_leaves = nullptr;
  int64_t* qt_claim = nullptr;  // per leaf: the voxel it bids for (TSDF seeding)
  double* qt_pyr = nullptr;     // quadtree sum pyramid
  int64_t cap_pyr = 0;
  uint32_t* qt_counters = nullptr;
  int64_t cap_tune = 0;
  // device scalars and their host mirror
  uint32_t* d_npairs = nullptr;
  unsigned long long* d_npairs_full = nullptr;
  uint32_t* d_overflow = nullptr;
  uint32_t* d_bounds = nullptr;  // set by the checked build's kernels on an out-of-bounds index
  unsigned long long* h_pinned = nullptr;
  // eval counters (blended, visited) and per-stage event profiling
  bool counting = false;
  unsigned long long* d_evals = nullptr;
  bool profiling = false;
  struct Ev {
    int stage;
    cudaEvent_t a, b;
  };
  std::vector<Ev> evs;
  size_t ev_used = 0;

  // state of the last forward pass: what it was computed from (the
  // backward pass must be given the same) and its token
  bool have_state = false;
  uint64_t serial = 0;       // forward passes started on this context
  uint64_t state_token = 0;  // token of the held state (0 = none)
  gs_gaussians st_g{};
  gs_camera st_cam[kMaxViews] = {};
  gs_viewmat st_view[kMaxViews] = {};
  gs_raster_cfg st_cfg{};
  int64_t st_n = 0;
  int st_views = 0;
  int st_w[kMaxViews] = {}, st_h[kMaxViews] = {};
  int st_tw = 0, st_th = 0;
  int64_t st_tiles = 0;
  int64_t st_pairs = 0;
  int st_pair_buf = 0;
  bool st_ordered = false;  // torder holds the visit order of the last forward pass
  // Graph-mode (no-sync) binning into per-tile buckets: the projection writes
  // each pair straight into its tile's bucket (bucket_cap entries), the
  // per-tile sort sorts the buckets in place and files every tile under its
  // length class (cls_count / cls_tiles); the forward raster pass takes its
  // visit order from the classes and records it in torder for the backward
  // pass, so the scan and the scatter drop out of the iteration.  Used in
  // no-sync mode while every sync-mode pass of the context has seen every
  // list at most half a bucket long (longest_seen, bucket_ok: a context that
  // renders several views or maps must not take one view's short lists for
  // another's); a bucket overflow clears bucket_ok for good (reported as
  // GS_ERR_CAPACITY).
  uint32_t* bids = nullptr;       // bids_words >= cap_bt * bucket_cap
  int64_t bids_words = 0;
  uint32_t bucket_cap = 0;        // entries per tile bucket: a power of two in [kBucketCapMin, kBucketCapMax]
  uint32_t* cls_count = nullptr;  // kLenClasses
  uint32_t* cls_tiles = nullptr;  // kLenClasses * cap_bt
  int64_t cap_bt = 0;
  int64_t longest_seen = 0;
  bool bucket_ok = false;
  bool st_buckets = false;        // the last forward pass binned into the buckets
  bool order_tiles = true;  // compute and use the visit order
  bool persistent = true;   // raster passes as persistent grids pulling (tile, quadrant) jobs
  int st_sh = 0;
  TileMap st_map{};
  int64_t st_pix_base[kMaxViews] = {};
};

namespace {

// Records a CUDA event pair around the launches of one stage when profiling.
struct StageTimer {
  gs_ctx* c;
  cudaStream_t s;
  size_t idx = (size_t)-1;
  StageTimer(gs_ctx* ctx, int stage, cudaStream_t stream) : c(ctx), s(stream) {
    if (!c->profiling) return;
    if (c->ev_used == c->evs.size()) {
      gs_ctx::Ev e{stage, nullptr, nullptr};
      if (cudaEventCreate(&e.a) != cudaSuccess || cudaEventCreate(&e.b) != cudaSuccess) return;
      c->evs.push_back(e);
    }
    idx = c->ev_used++;
    c->evs[idx].stage = stage;
    cudaEventRecord(c->evs[idx].a, s);
  }
  ~StageTimer() {
    if (idx != (size_t)-1) cudaEventRecord(c->evs[idx].b, s);
  }
};

gs_status fail(gs_ctx* c, gs_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

gs_status cuda_fail(gs_ctx* c, cudaError_t e, const char* where) {
  return fail(c, e == cudaErrorMemoryAllocation ? GS_ERR_OOM : GS_ERR_CUDA,
              std::string(where) + ": " + cudaGetErrorString(e));
}

#define GS_CUDA(ctx, call)                                  \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
  } while (0)

#define GS_CHECK_LAUNCH(ctx, where)                           \
  do {                                                        \
    cudaError_t e_ = cudaGetLastError();                      \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, where);   \
  } while (0)

template <class T>
cudaError_t regrow(T** p, int64_t count) {
  if (*p) cudaFree(*p);
  *p = nullptr;
  if (count <= 0) return cudaSuccess;
  return cudaMalloc((void**)p, sizeof(T) * (size_t)count);
}

int64_t grow_target(int64_t need, int64_t have) { return std::max<int64_t>(need + need / 4 + 1024, have); }

// A scratch group that fails to grow mid-way has freed some of its old
// buffers: its capacity drops to 0 so the next call allocates the whole
// group again.
#define GS_GROW(ctx, cap_field, call)       \
  do {                                      \
    cudaError_t e_ = (call);                \
    if (e_ != cudaSuccess) {                \
      (ctx)->cap_field = 0;                 \
      (ctx)->have_state = false;            \
      return cuda_fail(ctx, e_, #call);     \
    }                                       \
  } while (0)

// the failure injected by gs_ctx_inject_alloc_failure, checked before a
// scratch group grows (the group keeps its current buffers)
bool injected_alloc_failure(gs_ctx* c) { return c->fail_alloc > 0 && --c->fail_alloc == 0; }

// RAII NVTX range around an ABI call (a no-op unless a profiler is attached)
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

gs_status ensure_n(gs_ctx* c, int64_t n) {
  if (n <= c->cap_n) return GS_OK;
  if (injected_alloc_failure(c)) return fail(c, GS_ERR_OOM, "injected allocation failure");
  const int64_t cap = grow_target(n, c->cap_n);
  GS_CUDA(c, cudaSetDevice(c->device));
  GS_CUDA(c, cudaDeviceSynchronize());
  GS_GROW(c, cap_n, regrow(&c->feat, 3 * cap));
  GS_GROW(c, cap_n, regrow(&c->zkey, cap));
  for (int k = 0; k < 2; ++k) {
    GS_GROW(c, cap_n, regrow(&c->dkey[k], cap));
    GS_GROW(c, cap_n, regrow(&c->dval[k], cap));
  }
  GS_GROW(c, cap_n, regrow(&c->tiles, cap));
  GS_GROW(c, cap_n, regrow(&c->rects, cap));
  GS_GROW(c, cap_n, regrow(&c->bigq, cap));
  GS_GROW(c, cap_n, regrow(&c->g2d, 3 * cap));
  c->g2d_zero = false;
  GS_GROW(c, cap_n, regrow(&c->dup_sums, (int64_t)dup_blocks((int)cap) + 1));
  // per (block, view) pose partials: blocks(n) * V <= blocks(V n) + V, for
  // blocks of 64 or more Gaussians
  GS_GROW(c, cap_n, regrow(&c->pose_partials, 6 * ((cap + 31) / 32 + kMaxViews + 1)));
  c->cap_n = cap;
  c->have_state = false;
  return GS_OK;
}

gs_status ensure_pairs(gs_ctx* c, int64_t p) {
  if (p <= c->cap_p) return GS_OK;
  if (injected_alloc_failure(c)) return fail(c, GS_ERR_OOM, "injected allocation failure");
  if (p > 0xFFFFFFF0ll) return fail(c, GS_ERR_CAPACITY, "more than 2^32 - 16 (tile, Gaussian) pairs");
  const int64_t cap = std::min<int64_t>(grow_target(p, c->cap_p), 0xFFFFFFF0ll);
  GS_CUDA(c, cudaSetDevice(c->device));
  GS_CUDA(c, cudaDeviceSynchronize());
  for (int k = 0; k < 2; ++k) {
    GS_GROW(c, cap_p, regrow(&c->pk[k], cap));
    GS_GROW(c, cap_p, regrow(&c->pv[k], cap));
  }
  c->cap_p = cap;
  c->have_state = false;
  return GS_OK;
}

// Bucket storage for t tiles of `entries` each (see bids); synchronises
// when it grows.
gs_status ensure_buckets(gs_ctx* c, int64_t t, uint32_t entries) {
  const int64_t tiles = t <= c->cap_bt ? c->cap_bt : grow_target(t, c->cap_bt);
  if (tiles == c->cap_bt && tiles * (int64_t)entries <= c->bids_words) {
    c->bucket_cap = entries;
    return GS_OK;
  }
  if (injected_alloc_failure(c)) return fail(c, GS_ERR_OOM, "injected allocation failure");
  GS_CUDA(c, cudaDeviceSynchronize());
  c->bids_words = 0;
  GS_GROW(c, cap_bt, regrow(&c->bids, tiles * (int64_t)entries));
  c->bids_words = tiles * (int64_t)entries;
  if (tiles != c->cap_bt) GS_GROW(c, cap_bt, regrow(&c->cls_tiles, tiles * (int64_t)kLenClasses));
  if (!c->cls_count) GS_GROW(c, cap_bt, regrow(&c->cls_count, (int64_t)kLenClasses));
  c->cap_bt = tiles;
  c->bucket_cap = entries;
  return GS_OK;
}

gs_status ensure_tiles(gs_ctx* c, int64_t t) {
  if (t <= c->cap_t) return GS_OK;
  if (injected_alloc_failure(c)) return fail(c, GS_ERR_OOM, "injected allocation failure");
  GS_CUDA(c, cudaDeviceSynchronize());
  const int64_t cap = grow_target(t, c->cap_t);
  GS_GROW(c, cap_t, regrow(&c->ranges, cap));
  GS_GROW(c, cap_t, regrow(&c->tcount, cap));
  c->counts_zero = false;
  GS_GROW(c, cap_t, regrow(&c->toffset, cap));
  GS_GROW(c, cap_t, regrow(&c->tcursor, cap));
  GS_GROW(c, cap_t, regrow(&c->torder, cap));
  GS_GROW(c, cap_t, regrow(&c->scan_aux, tile_scan_aux_size(cap)));
  GS_GROW(c, cap_t, regrow(&c->tile_loss, 12 * cap));
  c->cap_t = cap;
  c->have_state = false;
  return GS_OK;
}

gs_status ensure_px(gs_ctx* c, int64_t npx) {
  if (npx <= c->cap_px) return GS_OK;
  if (injected_alloc_failure(c)) return fail(c, GS_ERR_OOM, "injected allocation failure");
  GS_CUDA(c, cudaDeviceSynchronize());
  const int64_t cap = grow_target(npx, c->cap_px);
  GS_GROW(c, cap_px, regrow(&c->T_final, cap));
  GS_GROW(c, cap_px, regrow(&c->last, cap));
  GS_GROW(c, cap_px, regrow(&c->dl_img, 4 * cap));
  // per-block partials (blocks of every view: <= blocks(total) + views) and per-view scales
  const int64_t lb = loss_blocks((int)std::min<int64_t>(cap, INT32_MAX - 4096));
  GS_GROW(c, cap_px, regrow(&c->loss_partials, 3 * (lb + kMaxViews) + kMaxViews + 4));
  c->cap_px = cap;
  c->have_state = false;
  return GS_OK;
}

int bits_for(int64_t n) {
  int b = 0;
  while (b < 40 && (int64_t(1) << b) < n) ++b;
  return b;
}

bool finite_pos(float v) { return std::isfinite(v) && v > 0.f; }

gs_status check_cam(gs_ctx* c, const gs_camera* cam) {
  if (!cam) return fail(c, GS_ERR_INVALID_ARG, "camera is NULL");
  if (cam->width < 1 || cam->height < 1) return fail(c, GS_ERR_INVALID_ARG, "camera width/height must be >= 1");
  if ((int64_t)cam->width * cam->height > (int64_t)1 << 30)
    return fail(c, GS_ERR_INVALID_ARG, "image larger than 2^30 pixels");
  if (!finite_pos(cam->fx) || !finite_pos(cam->fy) || !std::isfinite(cam->cx) || !std::isfinite(cam->cy))
    return fail(c, GS_ERR_INVALID_ARG, "camera intrinsics must be finite with fx, fy > 0");
  return GS_OK;
}

gs_status check_cfg(gs_ctx* c, const gs_raster_cfg* cfg) {
  if (!cfg) return fail(c, GS_ERR_INVALID_ARG, "raster cfg is NULL");
  if (!raster_shape_supported(cfg->tile_w, cfg->tile_h))
    return fail(c, GS_ERR_INVALID_ARG, "tile shape must be 16x16, 8x32 or 32x8");
  if (cfg->batch != 32) return fail(c, GS_ERR_INVALID_ARG, "batch (list entries per warp round) must be 32");
  if (!(cfg->alpha_max > 0.f && cfg->alpha_max < 1.f) || !(cfg->alpha_min > 0.f && cfg->alpha_min < cfg->alpha_max) ||
      !(cfg->t_eps > 0.f && cfg->t_eps < 1.f) || !(cfg->dilation >= 0.f) || !std::isfinite(cfg->near_z))
    return fail(c, GS_ERR_INVALID_ARG, "raster thresholds out of range");
  return GS_OK;
}

gs_status check_gauss(gs_ctx* c, const gs_gaussians* g) {
  if (!g) return fail(c, GS_ERR_INVALID_ARG, "gaussians is NULL");
  if (g->n < 0 || g->n >= ((int64_t)1 << 31)) return fail(c, GS_ERR_INVALID_ARG, "n out of range");
  if (g->sh_degree < 0 || g->sh_degree > 3) return fail(c, GS_ERR_INVALID_ARG, "sh_degree must be 0..3");
  if (g->n > 0 && (!g->means || !g->log_scales || !g->quats || !g->opacity_logits || !g->sh))
    return fail(c, GS_ERR_INVALID_ARG, "a Gaussian parameter pointer is NULL");
  return GS_OK;
}

CamView make_camview(const gs_camera* cam, const gs_viewmat* v) {
  CamView cv;
  cv.fx = cam->fx;
  cv.fy = cam->fy;
  cv.cx = cam->cx;
  cv.cy = cam->cy;
  cv.width = cam->width;
  cv.height = cam->height;
  for (int k = 0; k < 9; ++k) cv.R[k] = v->R[k];
  for (int k = 0; k < 3; ++k) cv.t[k] = v->t[k];
  for (int c = 0; c < 3; ++c) {
    double s = 0.0;
    for (int r = 0; r < 3; ++r) s += (double)v->R[3 * r + c] * (double)v->t[r];
    cv.C[c] = (float)(-s);
  }
  return cv;
}

gs_status ensure_hist(gs_ctx* c) {
  const int want = 8 * std::max(c->num_sms, 1);
  if (c->hist && c->hist_blocks >= want) return GS_OK;
  GS_CUDA(c, regrow(&c->hist, (int64_t)256 * (want + 1)));
  c->hist_blocks = want;
  return GS_OK;
}

// Radix binning (used when a tile list is longer than the per-tile sort holds):
// depth sort of the n items (keys in zkey, ids implicit), duplication into
// pairs, pair sort by global tile, tile ranges.  On success c->st_pairs /
// st_pair_buf describe the sorted pair list.
gs_status bin_and_sort_radix(gs_ctx* c, int n, const TileMap& map, cudaStream_t s) {
  const int64_t T = (int64_t)map.tile_base[map.views];
  if (c->sync) GS_CUDA(c, cudaMemsetAsync(c->d_overflow, 0, sizeof(uint32_t), s));
  SortBuffers sb;
  sb.keys[0] = c->dkey[0];
  sb.keys[1] = c->dkey[1];
  sb.vals[0] = c->dval[0];
  sb.vals[1] = c->dval[1];
  sb.hist = c->hist;
  sb.max_blocks = c->hist_blocks;
  int dcur;
  {
    StageTimer t(c, GS_STAGE_DEPTH_SORT, s);
    dcur = radix_sort_pairs(sb, c->zkey, nullptr, (uint32_t)n, nullptr, 32, c->num_sms, s, &c->launches);
  }
  const uint32_t* sorted_ids = dcur >= 0 ? c->dval[dcur] : c->dval[0];

  DupArgs da;
  da.n = n;
  da.sorted_ids = sorted_ids;
  da.tiles_touched = c->tiles;
  da.rects = c->rects;
  da.map = map;
  da.block_sums = c->dup_sums;
  da.n_pairs = c->d_npairs;
  da.n_pairs_full = c->d_npairs_full;
  da.tile_keys = nullptr;
  da.vals = nullptr;
  da.capacity = (uint32_t)std::min<int64_t>(c->cap_p, 0xFFFFFFF0ll);
  da.overflow = c->d_overflow;
  // phase 1: counts and scan
  {
    StageTimer t(c, GS_STAGE_DUPLICATE, s);
    launch_dup_count_scan(da, s, &c->launches);
  }
  GS_CHECK_LAUNCH(c, "duplicate count/scan");
  int64_t P = -1;
  if (c->sync) {
    GS_CUDA(c, cudaMemcpyAsync(c->h_pinned, c->d_npairs_full, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    GS_CUDA(c, cudaStreamSynchronize(s));
    P = (int64_t)*c->h_pinned;
    gs_status st = ensure_pairs(c, std::max<int64_t>(P, 1));
    if (st != GS_OK) return st;
    da.capacity = (uint32_t)std::min<int64_t>(c->cap_p, 0xFFFFFFF0ll);
  } else if (c->cap_p == 0) {
    return fail(c, GS_ERR_CAPACITY, "no-sync mode needs reserved pair capacity (gs_ctx_reserve)");
  }
  da.tile_keys = c->pk[0];
  da.vals = c->pv[0];
  {
    StageTimer t(c, GS_STAGE_DUPLICATE, s);
    launch_dup_write(da, s, &c->launches);
  }
  GS_CHECK_LAUNCH(c, "duplicate write");

  SortBuffers pb;
  pb.keys[0] = c->pk[0];
  pb.keys[1] = c->pk[1];
  pb.vals[0] = c->pv[0];
  pb.vals[1] = c->pv[1];
  pb.hist = c->hist;
  pb.max_blocks = c->hist_blocks;
  const uint32_t n_max = c->sync ? (uint32_t)P : (uint32_t)c->cap_p;
  const uint32_t* n_dev = c->sync ? nullptr : c->d_npairs;
  int pcur;
  {
    StageTimer t(c, GS_STAGE_PAIR_SORT, s);
    pcur = radix_sort_pairs(pb, c->pk[0], c->pv[0], n_max, n_dev, bits_for(T), c->num_sms, s, &c->launches);
  }
  {
    StageTimer t(c, GS_STAGE_RANGES, s);
    launch_tile_ranges(c->pk[pcur], n_dev, n_max, c->ranges, (int)T, c->num_sms, s, &c->launches);
  }
  GS_CHECK_LAUNCH(c, "pair sort / ranges");
  c->st_pairs = c->sync ? P : -1;
  c->st_pair_buf = pcur;
  c->st_buckets = false;
  return GS_OK;
}

// Graph-mode binning into the per-tile buckets the projection filled: one
// per-tile sort, which also files the tiles under their length classes.
gs_status bin_buckets(gs_ctx* c, int n, const TileMap& map, cudaStream_t s) {
  TileBinArgs tb;
  tb.n = n;
  tb.rects = c->rects;
  tb.tiles = c->tiles;
  tb.zkey = c->zkey;
  tb.map = map;
  tb.n_tiles = (int)map.tile_base[map.views];
  tb.num_sms = c->num_sms;
  tb.counts = c->tcount;
  tb.offsets = nullptr;
  tb.cursors = nullptr;
  tb.ids = nullptr;
  tb.ranges = c->ranges;
  tb.capacity = 0;
  tb.n_pairs = c->d_npairs;
  tb.stats = c->d_binstats;
  tb.overflow = c->d_overflow;
  tb.big_queue = c->bigq;
  tb.big_len = c->d_bigmeta;
  tb.order = nullptr;
  tb.counted = true;
  tb.scan_aux = nullptr;
  tb.raster_work = c->persistent ? c->d_bigmeta + 1 : nullptr;
  tb.bucket_ids = c->bids;
  tb.bucket_cap = c->bucket_cap;
  tb.cls_count = c->cls_count;
  tb.cls_tiles = c->cls_tiles;
  tb.cls_stride = (uint32_t)c->cap_bt;
  {
    StageTimer t(c, GS_STAGE_PAIR_SORT, s);
    launch_tile_sort(tb, s, &c->launches);
  }
  GS_CHECK_LAUNCH(c, "tile sort (buckets)");
  c->counts_zero = true;
  if (tb.raster_work) c->fwd_work_zero = c->bwd_work_zero = true;
  c->st_pairs = -1;
  c->st_pair_buf = 0;
  c->st_ordered = true;
  c->st_buckets = true;
  return GS_OK;
}

// Counting-scatter binning with per-tile sorts: count, scan (one host read of
// the totals in sync mode), scatter, sort.  Falls back to the radix path when
// some tile list is longer than the per-tile sort holds.  counted: the
// projection already added every item's tiles to the (zeroed) tile
// counters.
gs_status bin_and_sort(gs_ctx* c, int n, const TileMap& map, cudaStream_t s, bool counted) {
  const int64_t T = (int64_t)map.tile_base[map.views];
  if (c->sync) GS_CUDA(c, cudaMemsetAsync(c->d_overflow, 0, sizeof(uint32_t), s));
  TileBinArgs tb;
  tb.n = n;
  tb.rects = c->rects;
  tb.tiles = c->tiles;
  tb.zkey = c->zkey;
  tb.map = map;
  tb.n_tiles = (int)T;
  tb.num_sms = c->num_sms;
  tb.counts = c->tcount;
  tb.offsets = c->toffset;
  tb.cursors = c->tcursor;
  tb.ids = nullptr;
  tb.ranges = c->ranges;
  tb.capacity = c->sync ? 0xFFFFFFF0u : (uint32_t)std::min<int64_t>(c->cap_p, 0xFFFFFFF0ll);
  tb.n_pairs = c->d_npairs;
  tb.stats = c->d_binstats;
  tb.overflow = c->d_overflow;
  tb.big_queue = c->bigq;
  tb.big_len = c->d_bigmeta;
  tb.order = c->order_tiles ? c->torder : nullptr;
  tb.counted = counted;
  tb.scan_aux = c->scan_aux;
  c->st_ordered = false;
  {
    StageTimer t(c, GS_STAGE_DUPLICATE, s);
    launch_tile_count_scan(tb, s, &c->launches);
  }
  GS_CHECK_LAUNCH(c, "tile count/scan");
  int64_t P = -1;
  if (c->sync) {
    GS_CUDA(c, cudaMemcpyAsync(c->h_pinned, c->d_binstats, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    GS_CUDA(c, cudaStreamSynchronize(s));
    P = (int64_t)c->h_pinned[0];
    const int64_t longest = (int64_t)c->h_pinned[1];
    // graph-mode passes may bin into buckets while every list any sync pass
    // has seen fits half of one; a bucket holds twice the longest of them,
    // rounded up to a power of two (at least kBucketCapMin)
    c->longest_seen = std::max(c->longest_seen, longest);
    int64_t entries = kBucketCapMin;
    while (entries < 2 * c->longest_seen && entries < (int64_t)kBucketCapMax) entries *= 2;
    c->bucket_ok = c->longest_seen <= entries / 2 && T * entries < ((int64_t)1 << 32) &&
                   ensure_buckets(c, T, (uint32_t)entries) == GS_OK &&
                   c->cap_bt * (int64_t)kLenClasses < ((int64_t)1 << 32);
    if (longest > tile_sort_capacity()) return bin_and_sort_radix(c, n, map, s);
    gs_status st = ensure_pairs(c, std::max<int64_t>(P, 1));
    if (st != GS_OK) return st;
    tb.capacity = (uint32_t)std::min<int64_t>(c->cap_p, 0xFFFFFFF0ll);
  } else if (c->cap_p == 0) {
    return fail(c, GS_ERR_CAPACITY, "no-sync mode needs reserved pair capacity (gs_ctx_reserve)");
  }
  tb.ids = c->pv[0];
  {
    StageTimer t(c, GS_STAGE_DUPLICATE, s);
    launch_tile_scatter(tb, s, &c->launches);
  }
  tb.raster_work = c->persistent ? c->d_bigmeta + 1 : nullptr;
  {
    StageTimer t(c, GS_STAGE_PAIR_SORT, s);
    launch_tile_sort(tb, s, &c->launches);
  }
  GS_CHECK_LAUNCH(c, "tile scatter/sort");
  c->counts_zero = true;
  if (tb.raster_work) c->fwd_work_zero = c->bwd_work_zero = true;
  c->st_pairs = P;
  c->st_pair_buf = 0;
  c->st_ordered = tb.order != nullptr;
  c->st_buckets = false;
  return GS_OK;
}

}  // namespace

extern "C" {

gs_status gs_raster_cfg_default(gs_raster_cfg* cfg) {
  if (!cfg) return GS_ERR_INVALID_ARG;
  cfg->tile_w = 16;
  cfg->tile_h = 16;
  cfg->batch = 32;
  cfg->bg[0] = cfg->bg[1] = cfg->bg[2] = 0.f;
  cfg->near_z = 0.2f;
  cfg->alpha_max = 0.99f;
  cfg->alpha_min = 1.f / 255.f;
  cfg->t_eps = 1e-4f;
  cfg->dilation = 0.3f;
  return GS_OK;
}

gs_status gs_adam_cfg_default(gs_adam_cfg* cfg) {
  if (!cfg) return GS_ERR_INVALID_ARG;
  cfg->lr_means = 1.6e-4f;
  cfg->lr_log_scales = 5e-3f;
  cfg->lr_quats = 1e-3f;
  cfg->lr_opacity = 5e-2f;
  cfg->lr_sh_dc = 2.5e-3f;
  cfg->lr_sh_rest = 1.25e-4f;
  cfg->beta1 = 0.9f;
  cfg->beta2 = 0.999f;
  cfg->eps = 1e-15f;
  cfg->zero_grads = 0;
  return GS_OK;
}

gs_status gs_ctx_create(gs_ctx** out, int device, int64_t pair_capacity) {
  if (!out) return GS_ERR_INVALID_ARG;
  *out = nullptr;
  if (device < 0 || pair_capacity < 0) return GS_ERR_INVALID_ARG;
  gs_ctx* c = new gs_ctx();
  c->device = device;
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_npairs, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_npairs_full, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_overflow, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_binstats, 2 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_step, sizeof(long long));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_dscale, kMaxViews * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_nvalid, kMaxViews * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMemset(c->d_nvalid, 0, kMaxViews * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_bigmeta, 4 * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMemset(c->d_bigmeta, 0, 4 * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMemset(c->d_step, 0, sizeof(long long));
  if (e == cudaSuccess) init_project_kernels();
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_evals, 2 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(c->d_evals, 0, 2 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(c->d_overflow, 0, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_bounds, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMemset(c->d_bounds, 0, sizeof(uint32_t));
  if (e == cudaSuccess) e = raster_bind_bounds(c->d_bounds);
  if (e == cudaSuccess) e = tilebin_bind_bounds(c->d_bounds);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&c->h_pinned, 4 * sizeof(unsigned long long));
  if (e != cudaSuccess) {
    gs_ctx_destroy(c);
    return e == cudaErrorMemoryAllocation ? GS_ERR_OOM : GS_ERR_CUDA;
  }
  if (ensure_hist(c) != GS_OK || (pair_capacity > 0 && ensure_pairs(c, pair_capacity) != GS_OK)) {
    gs_ctx_destroy(c);
    return GS_ERR_OOM;
  }
  *out = c;
  return GS_OK;
}

gs_status gs_ctx_destroy(gs_ctx* c) {
  if (!c) return GS_ERR_INVALID_ARG;
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  cudaFree(c->feat);
  cudaFree(c->zkey);
  for (int k = 0; k < 2; ++k) {
    cudaFree(c->dkey[k]);
    cudaFree(c->dval[k]);
    cudaFree(c->pk[k]);
    cudaFree(c->pv[k]);
  }
  cudaFree(c->tiles);
  cudaFree(c->rects);
  cudaFree(c->g2d);
  cudaFree(c->dup_sums);
  cudaFree(c->pose_partials);
  cudaFree(c->hist);
  cudaFree(c->ranges);
  cudaFree(c->tcount);
  cudaFree(c->toffset);
  cudaFree(c->tcursor);
  cudaFree(c->torder);
  cudaFree(c->scan_aux);
  cudaFree(c->bigq);
  cudaFree(c->d_bigmeta);
  cudaFree(c->d_bounds);
  cudaFree(c->d_binstats);
  cudaFree(c->d_step);
  cudaFree(c->T_final);
  cudaFree(c->last);
  cudaFree(c->loss_partials);
  cudaFree(c->tune_img);
  cudaFree(c->dl_img);
  cudaFree(c->tile_loss);
  cudaFree(c->d_dscale);
  cudaFree(c->d_nvalid);
  cudaFree(c->bids);
  cudaFree(c->cls_count);
  cudaFree(c->cls_tiles);
  cudaFree(c->qt_cells[0]);
  cudaFree(c->qt_cells[1]);
  cudaFree(c->qt_leaves);
  cudaFree(c->qt_claim);
  cudaFree(c->qt_pyr);
  cudaFree(c->d_count);
  cudaFree(c->qt_counters);
  cudaFree(c->d_npairs);
  cudaFree(c->d_npairs_full);
  cudaFree(c->d_overflow);
  cudaFree(c->d_evals);
  for (auto& ev : c->evs) {
    cudaEventDestroy(ev.a);
    cudaEventDestroy(ev.b);
  }
  if (c->h_pinned) cudaFreeHost(c->h_pinned);
  delete c;
  return GS_OK;
}

const char* gs_last_error(const gs_ctx* c) { return c ? c->err.c_str() : "null context"; }

gs_status gs_ctx_reserve(gs_ctx* c, int64_t n_gaussians, int64_t n_pixels, int64_t n_pairs) {
  if (!c) return GS_ERR_INVALID_ARG;
  if (n_gaussians < 0 || n_pixels < 0 || n_pairs < 0) return fail(c, GS_ERR_INVALID_ARG, "negative reserve size");
  GS_CUDA(c, cudaSetDevice(c->device));
  gs_status s = GS_OK;
  if (n_gaussians > 0 && (s = ensure_n(c, n_gaussians)) != GS_OK) return s;
  if (n_pixels > 0 && (s = ensure_px(c, n_pixels)) != GS_OK) return s;
  if (n_pixels > 0 && (s = ensure_tiles(c, (n_pixels + 63) / 64 + 1024)) != GS_OK) return s;
  if (n_pairs > 0 && (s = ensure_pairs(c, n_pairs)) != GS_OK) return s;
  return GS_OK;
}

gs_status gs_ctx_set_adam_step(gs_ctx* c, int64_t step) {
  if (!c || step < 0) return GS_ERR_INVALID_ARG;
  GS_CUDA(c, cudaSetDevice(c->device));
  GS_CUDA(c, cudaDeviceSynchronize());
  const long long v = (long long)step;
  GS_CUDA(c, cudaMemcpy(c->d_step, &v, sizeof(v), cudaMemcpyHostToDevice));
  return GS_OK;
}

gs_status gs_ctx_set_sync(gs_ctx* c, int sync) {
  if (!c) return GS_ERR_INVALID_ARG;
  c->sync = sync != 0;
  return GS_OK;
}

gs_status gs_ctx_set_tile_order(gs_ctx* c, int on) {
  if (!c) return GS_ERR_INVALID_ARG;
  c->order_tiles = on != 0;
  return GS_OK;
}

gs_status gs_ctx_set_persistent(gs_ctx* c, int on) {
  if (!c) return GS_ERR_INVALID_ARG;
  c->persistent = on != 0;
  return GS_OK;
}

gs_status gs_sync_status(gs_ctx* c, gs_stream_t stream) {
  if (!c) return GS_ERR_INVALID_ARG;
  GS_CUDA(c, cudaSetDevice(c->device));
  cudaStream_t s = (cudaStream_t)stream;
  GS_CUDA(c, cudaMemcpyAsync(c->h_pinned + 1, c->d_overflow, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  GS_CUDA(c, cudaMemcpyAsync(c->h_pinned + 2, c->d_npairs_full, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  GS_CUDA(c, cudaMemcpyAsync(c->h_pinned + 3, c->d_bounds, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  GS_CUDA(c, cudaStreamSynchronize(s));
  if ((uint32_t)(c->h_pinned[3] & 0xFFFFFFFFull)) {
    GS_CUDA(c, cudaMemsetAsync(c->d_bounds, 0, sizeof(uint32_t), s));
    GS_CUDA(c, cudaStreamSynchronize(s));
    c->have_state = false;
    return fail(c, GS_ERR_BOUNDS, "an index was out of bounds (bounds-checked build); the results since are invalid");
  }
  const uint32_t ov = (uint32_t)(c->h_pinned[1] & 0xFFFFFFFFull);
  if (ov & 4u) {  // a tile bucket overflowed: graph-mode passes go back to the counting-scatter binning
    GS_CUDA(c, cudaMemsetAsync(c->d_overflow, 0, sizeof(uint32_t), s));
    GS_CUDA(c, cudaStreamSynchronize(s));
    c->have_state = false;
    c->bucket_ok = false;
    c->longest_seen = std::numeric_limits<int64_t>::max();
    return fail(c, GS_ERR_CAPACITY, "a tile list outgrew its bucket (" + std::to_string(c->bucket_cap) +
                                        " entries) in graph-mode binning; recapture to bin by counting and scatter");
  }
  if (ov) {
    GS_CUDA(c, cudaMemsetAsync(c->d_overflow, 0, sizeof(uint32_t), s));
    GS_CUDA(c, cudaStreamSynchronize(s));
    c->have_state = false;
    return fail(c, GS_ERR_CAPACITY, "pair buffer overflow: needed " + std::to_string(c->h_pinned[2]) + " pairs");
  }
  return GS_OK;
}

gs_status gs_get_stats(gs_ctx* c, gs_stats* out) {
  if (!c || !out) return GS_ERR_INVALID_ARG;
  out->n_pairs = c->st_pairs;
  out->pair_capacity = c->cap_p;
  out->kernel_launches = c->launches;
  out->n_tiles = c->st_tiles;
  out->evals_blended = 0;
  out->evals_tiled = 0;
  if (c->counting) {
    unsigned long long h[2] = {0, 0};
    GS_CUDA(c, cudaSetDevice(c->device));
    GS_CUDA(c, cudaDeviceSynchronize());
    GS_CUDA(c, cudaMemcpy(h, c->d_evals, sizeof(h), cudaMemcpyDeviceToHost));
    out->evals_blended = (int64_t)h[0];
    out->evals_tiled = (int64_t)h[1];
  }
  return GS_OK;
}

gs_status gs_set_eval_counting(gs_ctx* c, int counting) {
  if (!c) return GS_ERR_INVALID_ARG;
  GS_CUDA(c, cudaSetDevice(c->device));
  GS_CUDA(c, cudaDeviceSynchronize());
  GS_CUDA(c, cudaMemset(c->d_evals, 0, 2 * sizeof(unsigned long long)));
  c->counting = counting != 0;
  return GS_OK;
}

gs_status gs_set_profiling(gs_ctx* c, int profiling) {
  if (!c) return GS_ERR_INVALID_ARG;
  GS_CUDA(c, cudaSetDevice(c->device));
  GS_CUDA(c, cudaDeviceSynchronize());
  c->ev_used = 0;
  c->profiling = profiling != 0;
  return GS_OK;
}

gs_status gs_profile_read(gs_ctx* c, double* ms, int64_t* count) {
  if (!c || !ms || !count) return GS_ERR_INVALID_ARG;
  GS_CUDA(c, cudaSetDevice(c->device));
  GS_CUDA(c, cudaDeviceSynchronize());
  for (int k = 0; k < GS_NUM_STAGES; ++k) {
    ms[k] = 0.0;
    count[k] = 0;
  }
  for (size_t i = 0; i < c->ev_used; ++i) {
    float t = 0.f;
    GS_CUDA(c, cudaEventElapsedTime(&t, c->evs[i].a, c->evs[i].b));
    ms[c->evs[i].stage] += t;
    count[c->evs[i].stage] += 1;
  }
  c->ev_used = 0;
  return GS_OK;
}

}  // extern "C"

namespace {

// ---------------------------------------------------------------------------
// Batched internals: every render entry point runs through these with
// V >= 1 views of one Gaussian map (the single-view calls are V = 1).
// ---------------------------------------------------------------------------

struct ViewLayout {
  int V = 0;
  int64_t items = 0, pixels = 0, tiles = 0;
  TileMap map{};
  int tiles_y[kMaxViews] = {};
  int64_t pix_base[kMaxViews] = {};
};

gs_status check_views(gs_ctx* c, int32_t V, const gs_camera* cams, const gs_viewmat* views) {
  if (V < 1 || V > kMaxViews) return fail(c, GS_ERR_INVALID_ARG, "n_views must be in [1, 16]");
  if (!cams || !views) return fail(c, GS_ERR_INVALID_ARG, "cameras / viewmats array is NULL");
  for (int v = 0; v < V; ++v) {
    gs_status st = check_cam(c, &cams[v]);
    if (st != GS_OK) return st;
  }
  return GS_OK;
}

gs_status layout_views(gs_ctx* c, int64_t n, int V, const gs_camera* cams, const gs_raster_cfg* cfg, ViewLayout& L) {
  L.V = V;
  L.items = (int64_t)V * n;
  if (L.items >= ((int64_t)1 << 31)) return fail(c, GS_ERR_INVALID_ARG, "views x Gaussians must be < 2^31");
  L.map.views = V;
  L.map.n_per_view = (int)n;
  int64_t tiles = 0, pixels = 0;
  for (int v = 0; v < V; ++v) {
    const int tx = (cams[v].width + cfg->tile_w - 1) / cfg->tile_w;
    const int ty = (cams[v].height + cfg->tile_h - 1) / cfg->tile_h;
    if (tx > 65535 || ty > 65535) return fail(c, GS_ERR_INVALID_ARG, "too many tiles per axis");
    L.map.tiles_x[v] = tx;
    L.tiles_y[v] = ty;
    L.map.tile_base[v] = (uint32_t)tiles;
    L.pix_base[v] = pixels;
    tiles += (int64_t)tx * ty;
    pixels += (int64_t)cams[v].width * cams[v].height;
  }
  if (tiles >= ((int64_t)1 << 31) || pixels >= ((int64_t)1 << 31))
    return fail(c, GS_ERR_INVALID_ARG, "a batch must have < 2^31 tiles and pixels");
  for (int v = V; v <= kMaxViews; ++v) {
    if (v < kMaxViews) L.map.tiles_x[v] = 1;
    L.map.tile_base[v] = (uint32_t)tiles;
  }
  L.tiles = tiles;
  L.pixels = pixels;
  return GS_OK;
}

ProjectArgs project_args(const gs_gaussians* g, int V, const gs_camera* cams, const gs_viewmat* views,
                         const gs_raster_cfg* cfg, const TileMap& map, const int* tiles_y) {
  ProjectArgs pa;
  pa.big_queue = nullptr;
  pa.big_len = nullptr;
  pa.n = (int)g->n;
  pa.views = V;
  pa.means = g->means;
  pa.log_scales = g->log_scales;
  pa.quats = g->quats;
  pa.logits = g->opacity_logits;
  pa.sh = g->sh;
  pa.sh_degree = g->sh_degree;
  pa.near_z = cfg->near_z;
  pa.dilation = cfg->dilation;
  pa.alpha_min = cfg->alpha_min;
  pa.tile_w = cfg->tile_w;
  pa.tile_h = cfg->tile_h;
  for (int v = 0; v < kMaxViews; ++v) {
    if (v < V) {
      pa.cv[v] = make_camview(&cams[v], &views[v]);
      pa.tiles_x[v] = map.tiles_x[v];
      pa.tiles_y[v] = tiles_y[v];
    } else {
      pa.cv[v] = CamView{};
      pa.tiles_x[v] = pa.tiles_y[v] = 0;
    }
    pa.tile_base[v] = map.tile_base[v];
  }
  pa.counts = nullptr;
  return pa;
}

RasterArgs raster_args(gs_ctx* c, const gs_raster_cfg* cfg) {
  RasterArgs ra;
  ra.views = c->st_views;
  ra.tile_w = cfg->tile_w;
  ra.tile_h = cfg->tile_h;
  ra.n_tiles = (uint32_t)c->st_tiles;
  for (int k = 0; k < 3; ++k) ra.bg[k] = cfg->bg[k];
  ra.alpha_max = cfg->alpha_max;
  ra.alpha_min = cfg->alpha_min;
  ra.t_eps = cfg->t_eps;
  ra.ranges = c->ranges;
  ra.ids = c->st_buckets ? c->bids : c->pv[c->st_pair_buf];
  ra.feat = c->feat;
  ra.n_ids = (uint32_t)std::min<int64_t>(c->st_buckets ? c->cap_bt * (int64_t)c->bucket_cap : c->cap_p, 0xFFFFFFFFll);
  ra.n_items = (uint32_t)(c->st_n * c->st_views);
  ra.order = c->st_ordered ? c->torder : nullptr;
  ra.work = c->persistent ? c->d_bigmeta + 1 : nullptr;  // the forward counter; the backward pass uses [2]
  ra.zero_work = true;
  ra.num_sms = c->num_sms;
  ra.loss_partials = nullptr;
  ra.w_color = 0.f;
  ra.depth_scale = nullptr;
  ra.nvalid = nullptr;
  ra.w_depth = 0.f;
  ra.cls_count = nullptr;
  ra.cls_tiles = nullptr;
  ra.cls_stride = 0;
  ra.order_out = nullptr;
  for (int v = 0; v < kMaxViews; ++v) {
    RasterView& rv = ra.v[v];
    const bool live = v < c->st_views;
    rv.width = live ? c->st_w[v] : 0;
    rv.height = live ? c->st_h[v] : 0;
    rv.tiles_x = c->st_map.tiles_x[v];
    rv.tile_base = c->st_map.tile_base[v];
    rv.pix_base = live ? c->st_pix_base[v] : 0;
    rv.color = rv.depth = rv.alpha = nullptr;
    rv.dLdc = rv.dLdd = rv.dLda = nullptr;
    rv.trgb = rv.tdep = nullptr;
    rv.loss_dc = rv.loss_dd = nullptr;
  }
  return ra;
}

// Fused loss of a training step: targets per view and the colour weight; the
// image gradients go to the context's dl_img, the partial sums to tile_loss.
struct FusedLoss {
  const float* const* trgb;
  const float* const* tdep;
  float w_color;
  long long* step;  // nullable: the device Adam step, advanced by the projection
};

gs_status render_fwd_views(gs_ctx* c, const gs_gaussians* g, int32_t V, const gs_camera* cams,
                           const gs_viewmat* views, const gs_raster_cfg* cfg, float* const* color,
                           float* const* depth, float* const* alpha, cudaStream_t s,
                           const FusedLoss* fl = nullptr) {
  gs_status st;
  if ((st = check_gauss(c, g)) != GS_OK || (st = check_views(c, V, cams, views)) != GS_OK ||
      (st = check_cfg(c, cfg)) != GS_OK)
    return st;
  ViewLayout L;
  if ((st = layout_views(c, g->n, V, cams, cfg, L)) != GS_OK) return st;
  GS_CUDA(c, cudaSetDevice(c->device));
  const int n_items = (int)L.items;
  if (c->sync) {
    if ((st = ensure_n(c, std::max(n_items, 1))) != GS_OK || (st = ensure_px(c, L.pixels)) != GS_OK ||
        (st = ensure_tiles(c, L.tiles)) != GS_OK)
      return st;
  } else if (n_items > c->cap_n || L.pixels > c->cap_px || L.tiles > c->cap_t) {
    return fail(c, GS_ERR_CAPACITY, "no-sync mode: reserve items/pixels first (gs_ctx_reserve)");
  }
  c->have_state = false;
  c->state_token = 0;
  c->serial += 1;

  ProjectArgs pa = project_args(g, V, cams, views, cfg, L.map, L.tiles_y);
  pa.big_queue = c->bigq;
  pa.big_len = c->d_bigmeta;
  pa.counts = c->tcount;  // the projection counts every rectangle's tiles
  pa.nvalid = fl ? c->d_nvalid : nullptr;  // zeroed by the projection for the fused loss's count
  pa.step_inc = fl ? fl->step : nullptr;
  const bool buckets = !c->sync && c->bucket_ok && (int64_t)L.tiles <= c->cap_bt;
  if (buckets) {  // and writes every pair into its tile's bucket
    pa.bucket_ids = c->bids;
    pa.bucket_cap = c->bucket_cap;
    pa.overflow = c->d_overflow;
    pa.cls_count = c->cls_count;
  }
  if (!c->counts_zero) {  // else the last per-tile sort left them zero
    // every counter of the allocation, so that a later pass over more tiles
    // also starts from zeros
    GS_CUDA(c, cudaMemsetAsync(c->d_bigmeta, 0, sizeof(uint32_t), s));
    GS_CUDA(c, cudaMemsetAsync(c->tcount, 0, sizeof(uint32_t) * (size_t)c->cap_t, s));
  }
  c->counts_zero = false;
  {
    StageTimer t(c, GS_STAGE_PROJECT_FWD, s);
    launch_project_fwd(pa, c->feat, c->zkey, c->tiles, c->rects, s);
  }
  if (g->n > 0) c->launches += 1;
  GS_CHECK_LAUNCH(c, "project_fwd");

  if ((st = buckets ? bin_buckets(c, n_items, L.map, s) : bin_and_sort(c, n_items, L.map, s, true)) != GS_OK)
    return st;

  c->st_n = g->n;
  c->st_views = V;
  for (int v = 0; v < V; ++v) {
    c->st_w[v] = cams[v].width;
    c->st_h[v] = cams[v].height;
    c->st_pix_base[v] = L.pix_base[v];
  }
  c->st_tw = cfg->tile_w;
  c->st_th = cfg->tile_h;
  c->st_tiles = L.tiles;
  c->st_map = L.map;
  c->st_sh = g->sh_degree;

  RasterArgs ra = raster_args(c, cfg);
  for (int v = 0; v < V; ++v) {
    ra.v[v].color = color ? color[v] : nullptr;
    ra.v[v].depth = depth ? depth[v] : nullptr;
    ra.v[v].alpha = alpha ? alpha[v] : nullptr;
  }
  if (fl) {
    ra.loss_partials = c->tile_loss;
    ra.nvalid = c->d_nvalid;
    ra.w_color = fl->w_color;
    for (int v = 0; v < V; ++v) {
      const int64_t np = (int64_t)cams[v].width * cams[v].height;
      ra.v[v].trgb = fl->trgb[v];
      ra.v[v].tdep = fl->tdep[v];
      ra.v[v].loss_dc = c->dl_img + 4 * L.pix_base[v];
      ra.v[v].loss_dd = c->dl_img + 4 * L.pix_base[v] + 3 * np;
    }
  }
  if (c->st_buckets) {  // visit order from the sort's class lists, recorded for the backward pass
    ra.order = nullptr;
    ra.cls_count = c->cls_count;
    ra.cls_tiles = c->cls_tiles;
    ra.cls_stride = (uint32_t)c->cap_bt;
    ra.order_out = c->torder;
  }
  ra.zero_work = !c->fwd_work_zero;
  {
    StageTimer t(c, GS_STAGE_RASTER_FWD, s);
    launch_raster_fwd(ra, c->T_final, c->last, c->counting ? c->d_evals : nullptr, s);
  }
  c->fwd_work_zero = false;
  c->launches += 1;
  GS_CHECK_LAUNCH(c, "raster_fwd");
  c->st_g = *g;
  for (int v = 0; v < V; ++v) {
    c->st_cam[v] = cams[v];
    c->st_view[v] = views[v];
  }
  c->st_cfg = *cfg;
  c->state_token = c->serial;
  c->have_state = true;
  return GS_OK;
}

gs_status check_bwd_views(gs_ctx* c, const gs_gaussians* g, int32_t V, const gs_camera* cams,
                          const gs_viewmat* views, const gs_raster_cfg* cfg, const float* const* dL_dcolor,
                          const float* const* dL_ddepth) {
  gs_status st;
  if ((st = check_gauss(c, g)) != GS_OK || (st = check_views(c, V, cams, views)) != GS_OK ||
      (st = check_cfg(c, cfg)) != GS_OK)
    return st;
  if (!dL_dcolor || !dL_ddepth) return fail(c, GS_ERR_INVALID_ARG, "dL_dcolor and dL_ddepth are required");
  for (int v = 0; v < V; ++v)
    if (!dL_dcolor[v] || !dL_ddepth[v]) return fail(c, GS_ERR_INVALID_ARG, "dL_dcolor and dL_ddepth are required");
  if (!c->have_state) return fail(c, GS_ERR_STATE, "no forward state on this context (run the forward pass first)");
  const gs_gaussians& h = c->st_g;
  const bool same_map = h.means == g->means && h.log_scales == g->log_scales && h.quats == g->quats &&
                        h.opacity_logits == g->opacity_logits && h.sh == g->sh && h.n == g->n &&
                        h.sh_degree == g->sh_degree;
  if (!same_map || c->st_views != V)
    return fail(c, GS_ERR_STATE, "the held forward state is of other Gaussian arrays or another view count");
  for (int v = 0; v < V; ++v)
    if (std::memcmp(&c->st_cam[v], &cams[v], sizeof(gs_camera)) != 0 ||
        std::memcmp(&c->st_view[v], &views[v], sizeof(gs_viewmat)) != 0)
      return fail(c, GS_ERR_STATE, "the held forward state is of another camera or pose (view " + std::to_string(v) + ")");
  if (std::memcmp(&c->st_cfg, cfg, sizeof(gs_raster_cfg)) != 0)
    return fail(c, GS_ERR_STATE, "the held forward state is of another raster configuration");
  return GS_OK;
}

// raster backward into the context's per-item gradient records
gs_status raster_backward(gs_ctx* c, const gs_raster_cfg* cfg, const float* const* dL_dcolor,
                          const float* const* dL_ddepth, const float* const* dL_dalpha, cudaStream_t s,
                          const float* depth_scale = nullptr, const float* nvalid_w_depth = nullptr) {
  // the records are zero unless a backward pass ran without its consumer (or
  // the buffer is new): then clear the whole buffer once
  if (!c->g2d_zero) GS_CUDA(c, cudaMemsetAsync(c->g2d, 0, sizeof(float4) * 3 * (size_t)c->cap_n, s));
  RasterArgs ra = raster_args(c, cfg);
  if (ra.work) ra.work = c->d_bigmeta + 2;
  ra.zero_work = !c->bwd_work_zero;
  ra.depth_scale = depth_scale;
  if (nvalid_w_depth) {  // the fused loss: dL/dD scale w_depth / (valid target depths) per view
    ra.nvalid = c->d_nvalid;
    ra.w_depth = *nvalid_w_depth;
  }
  for (int v = 0; v < c->st_views; ++v) {
    ra.v[v].dLdc = dL_dcolor[v];
    ra.v[v].dLdd = dL_ddepth[v];
    ra.v[v].dLda = dL_dalpha ? dL_dalpha[v] : nullptr;
  }
  c->g2d_zero = false;  // until a consumer has read (and cleared) the records
  {
    StageTimer t(c, GS_STAGE_RASTER_BWD, s);
    launch_raster_bwd(ra, c->T_final, c->last, c->g2d, s);
  }
  c->bwd_work_zero = false;
  c->launches += 1;
  GS_CHECK_LAUNCH(c, "raster_bwd");
  return GS_OK;
}

// The training step's loss, reduced by the fused backward + Adam kernel
// (LossFoldArgs): the caller's loss word and the weights.
struct LossFold {
  float* loss;
  float w_color, w_depth;
};

gs_status check_adam(gs_ctx* c, const gs_adam_cfg* cfg, int64_t step, bool allow_device_step = false) {
  if (!cfg || step < (allow_device_step ? 0 : 1)) return fail(c, GS_ERR_INVALID_ARG, "Adam: bad cfg or step");
  if (!(cfg->beta1 >= 0.f && cfg->beta1 < 1.f && cfg->beta2 >= 0.f && cfg->beta2 < 1.f && cfg->eps >= 0.f))
    return fail(c, GS_ERR_INVALID_ARG, "Adam: betas must be in [0, 1), eps >= 0");
  return GS_OK;
}

AdamArgs adam_args(const gs_adam_cfg* cfg, int64_t step) {
  AdamArgs ad;
  ad.lr[0] = cfg->lr_means;
  ad.lr[1] = cfg->lr_log_scales;
  ad.lr[2] = cfg->lr_quats;
  ad.lr[3] = cfg->lr_opacity;
  ad.lr[4] = cfg->lr_sh_dc;
  ad.lr[5] = cfg->lr_sh_rest;
  ad.beta1 = cfg->beta1;
  ad.beta2 = cfg->beta2;
  ad.eps = cfg->eps;
  ad.step_dev = nullptr;
  ad.log_beta1 = (float)std::log((double)cfg->beta1);
  ad.log_beta2 = (float)std::log((double)cfg->beta2);
  ad.step_scale = ad.inv_sqrt_bc2 = 1.f;
  if (step > 0) {
    const double bc1 = 1.0 - std::pow((double)cfg->beta1, (double)step);
    const double bc2 = 1.0 - std::pow((double)cfg->beta2, (double)step);
    ad.step_scale = (float)(1.0 / bc1);
    ad.inv_sqrt_bc2 = (float)(1.0 / std::sqrt(bc2));
  }
  return ad;
}

gs_status render_bwd_adam_views(gs_ctx* c, const gs_gaussians* g, int32_t V, const gs_camera* cams,
                                const gs_viewmat* views, const gs_raster_cfg* cfg, const float* const* dL_dcolor,
                                const float* const* dL_ddepth, const float* const* dL_dalpha, float* params,
                                float* m, float* v, const gs_adam_cfg* adam, int64_t step, float* dL_dpose,
                                cudaStream_t s, const float* depth_scale = nullptr, bool step_advanced = false,
                                const float* nvalid_w_depth = nullptr, const LossFold* lf = nullptr) {
  // lf: the training step's loss, reduced by the fused kernel's first blocks
  gs_status st;
  if ((st = check_bwd_views(c, g, V, cams, views, cfg, dL_dcolor, dL_ddepth)) != GS_OK) return st;
  if ((st = check_adam(c, adam, step, true)) != GS_OK) return st;
  const int64_t n = g->n;
  if (n > 0 && (!params || !m || !v)) return fail(c, GS_ERR_INVALID_ARG, "params, m and v are required");
  if (n > 0 && (g->means != params || g->log_scales != params + 3 * n || g->quats != params + 6 * n ||
                g->opacity_logits != params + 10 * n || g->sh != params + 11 * n))
    return fail(c, GS_ERR_INVALID_ARG, "the Gaussian arrays must be the flat parameter buffer's blocks");
  GS_CUDA(c, cudaSetDevice(c->device));
  if (n == 0) return GS_OK;
  if ((st = raster_backward(c, cfg, dL_dcolor, dL_ddepth, dL_dalpha, s, depth_scale, nvalid_w_depth)) != GS_OK)
    return st;
  const ProjectArgs pa = project_args(g, V, cams, views, cfg, c->st_map, c->st_map.tiles_x);
  {
    StageTimer t(c, GS_STAGE_PROJECT_BWD, s);
    AdamArgs ad = adam_args(adam, step);
    if (step == 0) {
      if (!step_advanced) {  // (the training step's projection has advanced it)
        launch_step_increment(c->d_step, s);
        c->launches += 1;
      }
      ad.step_dev = c->d_step;
    }
    LossFoldArgs L{};
    if (lf) {  // the forward pass's loss partials (per tile and 8 x 8 block)
      L.partials = c->tile_loss;
      L.blk = c->loss_partials;
      L.out = lf->loss;
      L.scale = c->d_dscale;
      L.ticket = c->d_bigmeta + 3;
      L.w_color = lf->w_color;
      L.w_depth = lf->w_depth;
      L.views = c->st_views;
      int blocks = 0;
      for (int k = 0; k < c->st_views; ++k) {
        const int64_t t1 = k + 1 < c->st_views ? (int64_t)c->st_map.tile_base[k + 1] : c->st_tiles;
        L.block_base[k] = blocks;
        L.job_base[k] = 4u * c->st_map.tile_base[k];
        L.job_base[k + 1] = (uint32_t)(4 * t1);
        L.npix[k] = (float)c->st_w[k] * (float)c->st_h[k];
        blocks += (int)((4 * (t1 - (int64_t)c->st_map.tile_base[k]) + kLossChunk - 1) / kLossChunk);
      }
      L.block_base[c->st_views] = blocks;
      L.blocks = blocks;
    }
    const int nb = launch_project_bwd_adam(pa, c->g2d, params, m, v, ad, dL_dpose ? c->pose_partials : nullptr, s,
                                           lf ? &L : nullptr);
    c->launches += 1;
    if (dL_dpose) {
      launch_pose_reduce(c->pose_partials, nb, V, dL_dpose, s);
      c->launches += 1;
    }
  }
  GS_CHECK_LAUNCH(c, "project_bwd_adam");
  c->g2d_zero = true;  // the consumer clears the records it reads
  return GS_OK;
}

gs_status render_bwd_views(gs_ctx* c, const gs_gaussians* g, int32_t V, const gs_camera* cams,
                           const gs_viewmat* views, const gs_raster_cfg* cfg, const float* const* dL_dcolor,
                           const float* const* dL_ddepth, const float* const* dL_dalpha, const gs_grads* grads,
                           float* dL_dpose, cudaStream_t s) {
  gs_status st;
  if ((st = check_bwd_views(c, g, V, cams, views, cfg, dL_dcolor, dL_ddepth)) != GS_OK) return st;
  if (!grads) return fail(c, GS_ERR_INVALID_ARG, "grads is NULL");
  if (g->n > 0 && (!grads->means || !grads->log_scales || !grads->quats || !grads->opacity_logits || !grads->sh))
    return fail(c, GS_ERR_INVALID_ARG, "a gradient pointer is NULL");
  GS_CUDA(c, cudaSetDevice(c->device));
  if (g->n == 0) return GS_OK;
  if ((st = raster_backward(c, cfg, dL_dcolor, dL_ddepth, dL_dalpha, s)) != GS_OK) return st;
  const ProjectArgs pa = project_args(g, V, cams, views, cfg, c->st_map, c->st_map.tiles_x);
  {
    StageTimer t(c, GS_STAGE_PROJECT_BWD, s);
    const int nb = launch_project_bwd(pa, c->g2d, grads->means, grads->log_scales, grads->quats,
                                      grads->opacity_logits, grads->sh, dL_dpose ? c->pose_partials : nullptr, s);
    c->launches += 1;
    if (dL_dpose) {
      launch_pose_reduce(c->pose_partials, nb, V, dL_dpose, s);
      c->launches += 1;
    }
  }
  GS_CHECK_LAUNCH(c, "project_bwd");
  c->g2d_zero = true;  // the consumer clears the records it reads
  return GS_OK;
}

gs_status loss_views(gs_ctx* c, int32_t V, const gs_camera* cams, const float* const* color,
                     const float* const* depth, const float* const* target_rgb, const float* const* target_depth,
                     float w_color, float w_depth, float* loss, float* const* dL_dcolor, float* const* dL_ddepth,
                     cudaStream_t s) {
  if (V < 1 || V > kMaxViews) return fail(c, GS_ERR_INVALID_ARG, "n_views must be in [1, 16]");
  if (!cams) return fail(c, GS_ERR_INVALID_ARG, "cameras array is NULL");
  if (!color || !depth || !target_rgb || !target_depth || !loss || !dL_dcolor || !dL_ddepth)
    return fail(c, GS_ERR_INVALID_ARG, "loss: NULL pointer");
  if (!std::isfinite(w_color) || !std::isfinite(w_depth)) return fail(c, GS_ERR_INVALID_ARG, "non-finite weight");
  LossArgs la;
  la.views = V;
  la.w_color = w_color;
  la.w_depth = w_depth;
  la.loss = loss;
  int64_t pixels = 0, blocks = 0;
  for (int v = 0; v < V; ++v) {
    gs_status st = check_cam(c, &cams[v]);
    if (st != GS_OK) return st;
    if (!color[v] || !depth[v] || !target_rgb[v] || !target_depth[v] || !dL_dcolor[v] || !dL_ddepth[v])
      return fail(c, GS_ERR_INVALID_ARG, "loss: NULL image pointer");
    const int64_t npx = (int64_t)cams[v].width * cams[v].height;
    la.v[v] = LossView{(int)npx, (int)blocks, color[v], depth[v], target_rgb[v], target_depth[v], dL_dcolor[v],
                       dL_ddepth[v]};
    pixels += npx;
    blocks += loss_blocks((int)npx);
  }
  if (pixels >= ((int64_t)1 << 31)) return fail(c, GS_ERR_INVALID_ARG, "a batch must have < 2^31 pixels");
  la.n_blocks = (int)blocks;
  GS_CUDA(c, cudaSetDevice(c->device));
  gs_status st;
  if (c->sync) {
    if ((st = ensure_px(c, pixels)) != GS_OK) return st;
  } else if (pixels > c->cap_px) {
    return fail(c, GS_ERR_CAPACITY, "no-sync mode: reserve pixels first");
  }
  {
    StageTimer t(c, GS_STAGE_LOSS, s);
    launch_loss(la, c->loss_partials, s, &c->launches);
  }
  GS_CHECK_LAUNCH(c, "loss");
  return GS_OK;
}

// One optimisation iteration: forward pass with the loss fused into the
// compositing epilogue, the loss finalised on the device (with the per-view
// depth-gradient scales), then the backward pass fused with the Adam step,
// reading the image gradients from the context.
gs_status train_step_views(gs_ctx* c, const gs_gaussians* g, int32_t V, const gs_camera* cams,
                           const gs_viewmat* views, const gs_raster_cfg* cfg, const float* const* target_rgb,
                           const float* const* target_depth, float w_color, float w_depth, float* loss,
                           float* params, float* m, float* v, const gs_adam_cfg* adam, int64_t step,
                           float* const* color, float* const* depth, float* const* alpha, cudaStream_t s) {
  if (V < 1 || V > kMaxViews) return fail(c, GS_ERR_INVALID_ARG, "n_views must be in [1, 16]");
  if (!cams || !target_rgb || !target_depth || !loss)
    return fail(c, GS_ERR_INVALID_ARG, "train step: NULL cameras, targets or loss");
  for (int k = 0; k < V; ++k)
    if (!target_rgb[k] || !target_depth[k]) return fail(c, GS_ERR_INVALID_ARG, "train step: NULL target image");
  if (!std::isfinite(w_color) || !std::isfinite(w_depth)) return fail(c, GS_ERR_INVALID_ARG, "non-finite weight");
  gs_status st;
  if ((st = check_adam(c, adam, step, true)) != GS_OK) return st;
  // The device step counter (step = 0) is advanced by the projection, and
  // the loss is reduced by the fused backward + Adam kernel's first blocks
  // before their own work: the backward raster pass takes its depth scale
  // from the forward pass's count of valid target depths, so only the
  // reported loss needs the reduction.  Without Gaussians neither kernel
  // runs, and one kernel reduces the loss and advances the step.
  const FusedLoss fl{target_rgb, target_depth, w_color, step == 0 && g->n > 0 ? c->d_step : nullptr};
  if ((st = render_fwd_views(c, g, V, cams, views, cfg, color, depth, alpha, s, &fl)) != GS_OK) return st;
  if (g->n == 0) {
    RasterArgs ra = raster_args(c, cfg);
    ra.loss_partials = c->tile_loss;
    ra.w_color = w_color;
    {
      StageTimer t(c, GS_STAGE_LOSS, s);
      launch_loss_tiles_finalize(ra, w_depth, loss, c->d_dscale, c->loss_partials, c->d_bigmeta + 3,
                                 step == 0 ? c->d_step : nullptr, s, &c->launches);
    }
    GS_CHECK_LAUNCH(c, "loss finalize");
  }
  const LossFold lf{loss, w_color, w_depth};
  const float* dlc[kMaxViews];
  const float* dld[kMaxViews];
  for (int k = 0; k < V; ++k) {
    const int64_t np = (int64_t)cams[k].width * cams[k].height;
    dlc[k] = c->dl_img + 4 * c->st_pix_base[k];
    dld[k] = c->dl_img + 4 * c->st_pix_base[k] + 3 * np;
  }
  return render_bwd_adam_views(c, g, V, cams, views, cfg, dlc, dld, nullptr, params, m, v, adam, step, nullptr, s,
                               nullptr, /*step_advanced=*/true, &w_depth, &lf);
}

}  // namespace

extern "C" {

gs_status gs_train_step(gs_ctx* c, const gs_gaussians* g, const gs_camera* cam, const gs_viewmat* view,
                        const gs_raster_cfg* cfg, const float* target_rgb, const float* target_depth,
                        float w_color, float w_depth, float* loss, float* params, float* m, float* v,
                        const gs_adam_cfg* adam, int64_t step, gs_stream_t stream) {
  NvtxRange nvtx_("gs_train_step");
  if (!c) return GS_ERR_INVALID_ARG;
  if (!cam || !view) return fail(c, GS_ERR_INVALID_ARG, "camera / viewmat is NULL");
  return train_step_views(c, g, 1, cam, view, cfg, &target_rgb, &target_depth, w_color, w_depth, loss, params, m, v,
                          adam, step, nullptr, nullptr, nullptr, (cudaStream_t)stream);
}

gs_status gs_train_step_batched(gs_ctx* c, const gs_gaussians* g, int32_t n_views, const gs_camera* cams,
                                const gs_viewmat* views, const gs_raster_cfg* cfg, const float* const* target_rgb,
                                const float* const* target_depth, float w_color, float w_depth, float* loss,
                                float* params, float* m, float* v, const gs_adam_cfg* adam, int64_t step,
                                float* const* color, float* const* depth, float* const* alpha,
                                gs_stream_t stream) {
  NvtxRange nvtx_("gs_train_step_batched");
  if (!c) return GS_ERR_INVALID_ARG;
  return train_step_views(c, g, n_views, cams, views, cfg, target_rgb, target_depth, w_color, w_depth, loss, params,
                          m, v, adam, step, color, depth, alpha, (cudaStream_t)stream);
}

gs_status gs_render_fwd(gs_ctx* c, const gs_gaussians* g, const gs_camera* cam, const gs_viewmat* view,
                        const gs_raster_cfg* cfg, float* color, float* depth, float* alpha, gs_stream_t stream) {
  NvtxRange nvtx_("gs_render_fwd");
  if (!c) return GS_ERR_INVALID_ARG;
  if (!cam || !view) return fail(c, GS_ERR_INVALID_ARG, "camera / viewmat is NULL");
  return render_fwd_views(c, g, 1, cam, view, cfg, &color, &depth, &alpha, (cudaStream_t)stream);
}

gs_status gs_render_fwd_batched(gs_ctx* c, const gs_gaussians* g, int32_t n_views, const gs_camera* cams,
                                const gs_viewmat* views, const gs_raster_cfg* cfg, float* const* color,
                                float* const* depth, float* const* alpha, gs_stream_t stream) {
  NvtxRange nvtx_("gs_render_fwd_batched");
  if (!c) return GS_ERR_INVALID_ARG;
  return render_fwd_views(c, g, n_views, cams, views, cfg, color, depth, alpha, (cudaStream_t)stream);
}

gs_status gs_render_bwd_adam(gs_ctx* c, const gs_gaussians* g, const gs_camera* cam, const gs_viewmat* view,
                             const gs_raster_cfg* cfg, const float* dL_dcolor, const float* dL_ddepth,
                             const float* dL_dalpha, float* params, float* m, float* v, const gs_adam_cfg* adam,
                             int64_t step, float* dL_dpose, gs_stream_t stream) {
  NvtxRange nvtx_("gs_render_bwd_adam");
  if (!c) return GS_ERR_INVALID_ARG;
  if (!cam || !view) return fail(c, GS_ERR_INVALID_ARG, "camera / viewmat is NULL");
  return render_bwd_adam_views(c, g, 1, cam, view, cfg, &dL_dcolor, &dL_ddepth, &dL_dalpha, params, m, v, adam, step,
                               dL_dpose, (cudaStream_t)stream);
}

gs_status gs_render_bwd_adam_batched(gs_ctx* c, const gs_gaussians* g, int32_t n_views, const gs_camera* cams,
                                     const gs_viewmat* views, const gs_raster_cfg* cfg,
                                     const float* const* dL_dcolor, const float* const* dL_ddepth,
                                     const float* const* dL_dalpha, float* params, float* m, float* v,
                                     const gs_adam_cfg* adam, int64_t step, float* dL_dpose, gs_stream_t stream) {
  NvtxRange nvtx_("gs_render_bwd_adam_batched");
  if (!c) return GS_ERR_INVALID_ARG;
  return render_bwd_adam_views(c, g, n_views, cams, views, cfg, dL_dcolor, dL_ddepth, dL_dalpha, params, m, v, adam,
                               step, dL_dpose, (cudaStream_t)stream);
}

gs_status gs_render_bwd(gs_ctx* c, const gs_gaussians* g, const gs_camera* cam, const gs_viewmat* view,
                        const gs_raster_cfg* cfg, const float* dL_dcolor, const float* dL_ddepth,
                        const float* dL_dalpha, const gs_grads* grads, float* dL_dpose, gs_stream_t stream) {
  NvtxRange nvtx_("gs_render_bwd");
  if (!c) return GS_ERR_INVALID_ARG;
  if (!cam || !view) return fail(c, GS_ERR_INVALID_ARG, "camera / viewmat is NULL");
  return render_bwd_views(c, g, 1, cam, view, cfg, &dL_dcolor, &dL_ddepth, &dL_dalpha, grads, dL_dpose,
                          (cudaStream_t)stream);
}

gs_status gs_render_bwd_batched(gs_ctx* c, const gs_gaussians* g, int32_t n_views, const gs_camera* cams,
                                const gs_viewmat* views, const gs_raster_cfg* cfg, const float* const* dL_dcolor,
                                const float* const* dL_ddepth, const float* const* dL_dalpha,
                                const gs_grads* grads, float* dL_dpose, gs_stream_t stream) {
  NvtxRange nvtx_("gs_render_bwd_batched");
  if (!c) return GS_ERR_INVALID_ARG;
  return render_bwd_views(c, g, n_views, cams, views, cfg, dL_dcolor, dL_ddepth, dL_dalpha, grads, dL_dpose,
                          (cudaStream_t)stream);
}

gs_status gs_loss_l1(gs_ctx* c, const gs_camera* cam, const float* color, const float* depth,
                     const float* target_rgb, const float* target_depth, float w_color, float w_depth, float* loss,
                     float* dL_dcolor, float* dL_ddepth, gs_stream_t stream) {
  NvtxRange nvtx_("gs_loss_l1");
  if (!c) return GS_ERR_INVALID_ARG;
  if (!cam) return fail(c, GS_ERR_INVALID_ARG, "camera is NULL");
  return loss_views(c, 1, cam, &color, &depth, &target_rgb, &target_depth, w_color, w_depth, loss, &dL_dcolor,
                    &dL_ddepth, (cudaStream_t)stream);
}

gs_status gs_loss_l1_batched(gs_ctx* c, int32_t n_views, const gs_camera* cams, const float* const* color,
                             const float* const* depth, const float* const* target_rgb,
                             const float* const* target_depth, float w_color, float w_depth, float* loss,
                             float* const* dL_dcolor, float* const* dL_ddepth, gs_stream_t stream) {
  NvtxRange nvtx_("gs_loss_l1_batched");
  if (!c) return GS_ERR_INVALID_ARG;
  return loss_views(c, n_views, cams, color, depth, target_rgb, target_depth, w_color, w_depth, loss, dL_dcolor,
                    dL_ddepth, (cudaStream_t)stream);
}

gs_status gs_adam_step(gs_ctx* c, float* params, float* grads, float* m, float* v, int64_t n,
                       int32_t sh_degree, const gs_adam_cfg* cfg, int64_t step, gs_stream_t stream) {
  NvtxRange nvtx_("gs_adam_step");
  if (!c) return GS_ERR_INVALID_ARG;
  if (!cfg || step < 0 || n < 0 || sh_degree < 0 || sh_degree > 3)
    return fail(c, GS_ERR_INVALID_ARG, "gs_adam_step: bad cfg, step, n or sh_degree");
  if (n > 0 && (!params || !grads || !m || !v)) return fail(c, GS_ERR_INVALID_ARG, "gs_adam_step: NULL pointer");
  if (!(cfg->beta1 >= 0.f && cfg->beta1 < 1.f && cfg->beta2 >= 0.f && cfg->beta2 < 1.f && cfg->eps >= 0.f))
    return fail(c, GS_ERR_INVALID_ARG, "gs_adam_step: betas must be in [0, 1), eps >= 0");
  GS_CUDA(c, cudaSetDevice(c->device));
  cudaStream_t s = (cudaStream_t)stream;
  const float lr[6] = {cfg->lr_means, cfg->lr_log_scales, cfg->lr_quats, cfg->lr_opacity, cfg->lr_sh_dc, cfg->lr_sh_rest};
  {
    StageTimer t(c, GS_STAGE_ADAM, s);
    if (step == 0) {  // device-side step counter (graph-capturable)
      launch_step_increment(c->d_step, s);
      c->launches += 1;
      launch_adam(params, grads, m, v, n, sh_degree, lr, cfg->beta1, cfg->beta2, cfg->eps, 1.f, 1.f,
                  cfg->zero_grads != 0, c->d_step, s);
    } else {
      const double bc1 = 1.0 - std::pow((double)cfg->beta1, (double)step);
      const double bc2 = 1.0 - std::pow((double)cfg->beta2, (double)step);
      launch_adam(params, grads, m, v, n, sh_degree, lr, cfg->beta1, cfg->beta2, cfg->eps, (float)(1.0 / bc1),
                  (float)(1.0 / std::sqrt(bc2)), cfg->zero_grads != 0, nullptr, s);
    }
  }
  if (n > 0) c->launches += 1;
  GS_CHECK_LAUNCH(c, "adam");
  return GS_OK;
}

gs_status gs_autotune(gs_ctx* c, const gs_gaussians* g, int32_t n_views, const gs_camera* cams,
                      const gs_viewmat* views, gs_raster_cfg* cfg, int32_t reps, float* ms, gs_stream_t stream) {
  NvtxRange nvtx_("gs_autotune");
  if (!c) return GS_ERR_INVALID_ARG;
  gs_status st;
  if ((st = check_gauss(c, g)) != GS_OK || (st = check_views(c, n_views, cams, views)) != GS_OK ||
      (st = check_cfg(c, cfg)) != GS_OK)
    return st;
  if (reps < 1 || reps > 1000) return fail(c, GS_ERR_INVALID_ARG, "gs_autotune: reps must be in [1, 1000]");
  GS_CUDA(c, cudaSetDevice(c->device));
  cudaStream_t s = (cudaStream_t)stream;
  int64_t pixels = 0;
  for (int v = 0; v < n_views; ++v) pixels += (int64_t)cams[v].width * cams[v].height;
  if (4 * pixels > c->cap_tune) {  // dL/dcolor (3 planes) + dL/ddepth per view, all zero
    GS_CUDA(c, cudaDeviceSynchronize());
    GS_CUDA(c, regrow(&c->tune_img, 4 * pixels));
    GS_CUDA(c, cudaMemset(c->tune_img, 0, sizeof(float) * 4 * (size_t)pixels));
    c->cap_tune = 4 * pixels;
  }
  const float* dlc[kMaxViews];
  const float* dld[kMaxViews];
  int64_t off = 0;
  for (int v = 0; v < n_views; ++v) {
    const int64_t np = (int64_t)cams[v].width * cams[v].height;
    dlc[v] = c->tune_img + off;
    dld[v] = c->tune_img + off + 3 * np;
    off += 4 * np;
  }
  static const int kShapes[GS_AUTOTUNE_CANDIDATES][2] = {{16, 16}, {8, 32}, {32, 8}};
  const bool was_sync = c->sync;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  GS_CUDA(c, cudaEventCreate(&e0));
  GS_CUDA(c, cudaEventCreate(&e1));
  float best = 0.f;
  int best_k = -1;
  st = GS_OK;
  for (int k = 0; k < GS_AUTOTUNE_CANDIDATES && st == GS_OK; ++k) {
    gs_raster_cfg cand = *cfg;
    cand.tile_w = kShapes[k][0];
    cand.tile_h = kShapes[k][1];
    // untimed pass in sync mode sizes the buffers for this tile shape
    c->sync = true;
    st = render_fwd_views(c, g, n_views, cams, views, &cand, nullptr, nullptr, nullptr, s);
    if (st == GS_OK) st = raster_backward(c, &cand, dlc, dld, nullptr, s);
    if (st != GS_OK) break;
    c->sync = false;  // timed passes: no host synchronisation, same inputs so the same pair count
    cudaEventRecord(e0, s);
    for (int r = 0; r < reps && st == GS_OK; ++r) {
      st = render_fwd_views(c, g, n_views, cams, views, &cand, nullptr, nullptr, nullptr, s);
      if (st == GS_OK) st = raster_backward(c, &cand, dlc, dld, nullptr, s);
    }
    cudaEventRecord(e1, s);
    if (st != GS_OK) break;
    cudaError_t e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (e != cudaSuccess) {
      st = cuda_fail(c, e, "gs_autotune timing");
      break;
    }
    t /= (float)reps;
    if (ms) ms[k] = t;
    if (best_k < 0 || t < best) {
      best = t;
      best_k = k;
    }
  }
  c->sync = was_sync;
  c->have_state = false;  // the stored state is the last candidate's, not the chosen one
  c->state_token = 0;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != GS_OK) return st;
  cfg->tile_w = kShapes[best_k][0];
  cfg->tile_h = kShapes[best_k][1];
  return GS_OK;
}

namespace {

bool pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }

gs_status qt_prepare(gs_ctx* c, int W, int H, int max_size, int min_size, float var_thr) {
  if (W < 1 || H < 1 || (int64_t)W * H > ((int64_t)1 << 30))
    return fail(c, GS_ERR_INVALID_ARG, "quadtree: image size out of range");
  if (!pow2(max_size) || !pow2(min_size) || min_size > max_size || max_size > 4096)
    return fail(c, GS_ERR_INVALID_ARG, "quadtree: cell sizes must be powers of two, 1 <= min <= max <= 4096");
  if (!std::isfinite(var_thr) || var_thr < 0.f) return fail(c, GS_ERR_INVALID_ARG, "quadtree: bad threshold");
  const int64_t need = quadtree_scratch_cells(W, H);
  if (need > c->cap_qt) {
    GS_CUDA(c, cudaDeviceSynchronize());
    GS_CUDA(c, regrow(&c->qt_cells[0], need));
    GS_CUDA(c, regrow(&c->qt_cells[1], need));
    GS_CUDA(c, regrow(&c->qt_leaves, need));
    GS_CUDA(c, regrow(&c->qt_claim, need));
    if (!c->qt_counters) GS_CUDA(c, cudaMalloc((void**)&c->qt_counters, 32 * sizeof(uint32_t)));
    c->cap_qt = need;
  }
  const int64_t need_pyr = quadtree_pyramid_doubles(W, H, max_size);
  if (need_pyr > c->cap_pyr) {
    GS_CUDA(c, cudaDeviceSynchronize());
    GS_CUDA(c, regrow(&c->qt_pyr, need_pyr));
    c->cap_pyr = need_pyr;
  }
  return GS_OK;
}

// quadtree over rgb [3, H, W]; returns the leaf count (host) after one synchronisation
gs_status qt_run(gs_ctx* c, const float* rgb, int W, int H, int max_size, int min_size, float var_thr,
                 uint32_t* n_leaves, cudaStream_t s) {
  gs_status st = qt_prepare(c, W, H, max_size, min_size, var_thr);
  if (st != GS_OK) return st;
  c->launches += launch_quadtree(rgb, W, H, max_size, min_size, (double)var_thr, c->qt_cells[0], c->qt_cells[1],
                                 c->qt_counters, c->qt_leaves, c->qt_pyr, s);
  GS_CHECK_LAUNCH(c, "quadtree");
  GS_CUDA(c, cudaMemcpyAsync(c->h_pinned, c->qt_counters, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  GS_CUDA(c, cudaStreamSynchronize(s));
  *n_leaves = (uint32_t)(c->h_pinned[0] & 0xFFFFFFFFull);
  return GS_OK;
}

}  // namespace

gs_status gs_quadtree_leaves(gs_ctx* c, const float* rgb, int32_t width, int32_t height, float var_thr,
                             int32_t max_size, int32_t min_size, int32_t* leaves, int64_t capacity, int64_t* n_leaves,
                             gs_stream_t stream) {
  NvtxRange nvtx_("gs_quadtree_leaves");
  if (!c) return GS_ERR_INVALID_ARG;
  if (!rgb || !n_leaves || capacity < 0) return fail(c, GS_ERR_INVALID_ARG, "gs_quadtree_leaves: bad arguments");
  GS_CUDA(c, cudaSetDevice(c->device));
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t nl = 0;
  gs_status st = qt_run(c, rgb, width, height, max_size, min_size, var_thr, &nl, s);
  if (st != GS_OK) return st;
  *n_leaves = nl;
  if ((int64_t)nl > capacity) return fail(c, GS_ERR_CAPACITY, "gs_quadtree_leaves: output capacity too small");
  if (nl > 0) {
    if (!leaves) return fail(c, GS_ERR_INVALID_ARG, "gs_quadtree_leaves: NULL output");
    GS_CUDA(c, cudaMemcpyAsync(leaves, c->qt_leaves, sizeof(int4) * nl, cudaMemcpyDeviceToDevice, s));
  }
  GS_CUDA(c, cudaStreamSynchronize(s));
  return GS_OK;
}

gs_status gs_seed_quadtree(gs_ctx* c, const float* rgb, const float* depth, const float* alpha, float alpha_thr,
                           const gs_camera* cam, const gs_viewmat* view, int32_t sh_degree, float var_thr,
                           int32_t max_size, int32_t min_size, float* means, float* log_scales, float* quats,
                           float* opacity_logits, float* sh, int64_t capacity, int64_t* n_seeded,
                           gs_stream_t stream) {
  NvtxRange nvtx_("gs_seed_quadtree");
  if (!c) return GS_ERR_INVALID_ARG;
  gs_status st;
  if ((st = check_cam(c, cam)) != GS_OK) return st;
  if (!view || !rgb || !depth || !n_seeded || capacity < 0 || sh_degree < 0 || sh_degree > 3)
    return fail(c, GS_ERR_INVALID_ARG, "gs_seed_quadtree: bad arguments");
  if (capacity > 0 && (!means || !log_scales || !quats || !opacity_logits || !sh))
    return fail(c, GS_ERR_INVALID_ARG, "gs_seed_quadtree: NULL output array");
  if (capacity > 0xFFFFFFF0ll) return fail(c, GS_ERR_INVALID_ARG, "gs_seed_quadtree: capacity too large");
  GS_CUDA(c, cudaSetDevice(c->device));
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t nl = 0;
  if ((st = qt_run(c, rgb, cam->width, cam->height, max_size, min_size, var_thr, &nl, s)) != GS_OK) return st;
  const float K4[4] = {cam->fx, cam->fy, cam->cx, cam->cy};
  float R[9], t[3];
  for (int k = 0; k < 9; ++k) R[k] = view->R[k];
  for (int k = 0; k < 3; ++k) t[k] = view->t[k];
  uint32_t* n_dev = c->qt_counters + 24;
  launch_seed(rgb, depth, alpha, alpha_thr, cam->width, cam->height, K4, R, t, sh_degree, c->qt_leaves, nl, means,
              log_scales, quats, opacity_logits, sh, (uint32_t)capacity, n_dev, s);
  if (nl > 0) c->launches += 1;
  GS_CHECK_LAUNCH(c, "seed");
  GS_CUDA(c, cudaMemcpyAsync(c->h_pinned, n_dev, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  GS_CUDA(c, cudaStreamSynchronize(s));
  const int64_t n = (int64_t)(c->h_pinned[0] & 0xFFFFFFFFull);
  *n_seeded = n;
  if (n > capacity) return fail(c, GS_ERR_CAPACITY, "gs_seed_quadtree: more new Gaussians than capacity");
  return GS_OK;
}

namespace {

gs_status check_grid(gs_ctx* c, const gs_tsdf_grid* g) {
  if (!g) return fail(c, GS_ERR_INVALID_ARG, "tsdf grid is NULL");
  if (!g->keys || !g->slots || !g->stamps || !g->voxels || !g->claims || !g->touched || !g->counters)
    return fail(c, GS_ERR_INVALID_ARG, "tsdf grid: NULL array");
  if (g->table_size < 2 || g->table_size > ((int64_t)1 << 32) || (g->table_size & (g->table_size - 1)))
    return fail(c, GS_ERR_INVALID_ARG, "tsdf grid: table_size must be a power of two in [2, 2^32]");
  if (g->capacity < 1 || g->capacity > INT32_MAX) return fail(c, GS_ERR_INVALID_ARG, "tsdf grid: bad capacity");
  if (!finite_pos(g->voxel_size) || !finite_pos(g->truncation))
    return fail(c, GS_ERR_INVALID_ARG, "tsdf grid: voxel_size and truncation must be finite and > 0");
  if ((double)g->truncation / (double)g->voxel_size > 1e6 ||
      tsdf_band_steps(g->truncation, g->voxel_size) + 1 > GS_TSDF_MAX_SAMPLES)
    return fail(c, GS_ERR_INVALID_ARG, "tsdf grid: truncation too wide for the band samples (eps <= 30 s)");
  if (!(g->max_weight >= 1.f) || !std::isfinite(g->max_weight))
    return fail(c, GS_ERR_INVALID_ARG, "tsdf grid: max_weight must be finite and >= 1");
  if (g->fusion != 0 && g->fusion != 1) return fail(c, GS_ERR_INVALID_ARG, "tsdf grid: fusion must be 0 or 1");
  return GS_OK;
}

TsdfGrid to_internal(const gs_tsdf_grid* g) {
  TsdfGrid t;
  t.keys = reinterpret_cast<unsigned long long*>(g->keys);
  t.slots = g->slots;
  t.stamps = g->stamps;
  t.voxels = g->voxels;
  t.claims = g->claims;
  t.touched = g->touched;
  t.counters = g->counters;
  t.table_size = g->table_size;
  t.capacity = g->capacity;
  t.voxel_size = g->voxel_size;
  t.truncation = g->truncation;
  t.max_weight = g->max_weight;
  t.fusion = g->fusion;
  return t;
}

TsdfCamera tsdf_camera(const gs_camera* cam, const gs_viewmat* view) {
  TsdfCamera t;
  t.fx = cam->fx;
  t.fy = cam->fy;
  t.cx = cam->cx;
  t.cy = cam->cy;
  t.W = cam->width;
  t.H = cam->height;
  for (int k = 0; k < 9; ++k) t.R[k] = view->R[k];
  for (int k = 0; k < 3; ++k) t.t[k] = view->t[k];
  return t;
}

bool finite_view(const gs_viewmat* v) {
  for (int k = 0; k < 9; ++k)
    if (!std::isfinite(v->R[k])) return false;
  for (int k = 0; k < 3; ++k)
    if (!std::isfinite(v->t[k])) return false;
  return true;
}

}  // namespace

gs_status gs_tsdf_integrate(gs_ctx* c, const gs_tsdf_grid* grid, const float* depth, const gs_camera* cam,
                            const gs_viewmat* view, uint32_t frame, int64_t min_slot, gs_stream_t stream) {
  NvtxRange nvtx_("gs_tsdf_integrate");
  if (!c) return GS_ERR_INVALID_ARG;
  gs_status st;
  if ((st = check_grid(c, grid)) != GS_OK || (st = check_cam(c, cam)) != GS_OK) return st;
  if (!depth || !view || !finite_view(view) || frame == 0 || min_slot < 0 || min_slot > grid->capacity)
    return fail(c, GS_ERR_INVALID_ARG, "gs_tsdf_integrate: bad arguments");
  GS_CUDA(c, cudaSetDevice(c->device));
  cudaStream_t s = (cudaStream_t)stream;
  const TsdfGrid g = to_internal(grid);
  const TsdfCamera tc = tsdf_camera(cam, view);
  if (min_slot == 0) {
    GS_CUDA(c, cudaMemsetAsync(grid->counters + 1, 0, 2 * sizeof(uint32_t), s));
    launch_tsdf_alloc(g, depth, tc, frame, s);
    GS_CHECK_LAUNCH(c, "tsdf allocation");
    c->launches += 1;
  }
  launch_tsdf_integrate(g, depth, tc, min_slot, c->num_sms, s);
  GS_CHECK_LAUNCH(c, "tsdf integration");
  c->launches += 1;
  return GS_OK;
}

gs_status gs_tsdf_counters(gs_ctx* c, const gs_tsdf_grid* grid, int64_t* out, gs_stream_t stream) {
  if (!c) return GS_ERR_INVALID_ARG;
  gs_status st;
  if ((st = check_grid(c, grid)) != GS_OK) return st;
  if (!out) return fail(c, GS_ERR_INVALID_ARG, "gs_tsdf_counters: NULL output");
  GS_CUDA(c, cudaSetDevice(c->device));
  cudaStream_t s = (cudaStream_t)stream;
  GS_CUDA(c, cudaMemcpyAsync(c->h_pinned, grid->counters, 4 * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  GS_CUDA(c, cudaStreamSynchronize(s));
  const uint32_t* h = reinterpret_cast<const uint32_t*>(c->h_pinned);
  for (int k = 0; k < 4; ++k) out[k] = h[k];
  if (out[2] > 0) return fail(c, GS_ERR_CAPACITY, "tsdf: hash table or touched list full (grow table_size)");
  if (out[0] > grid->capacity) return fail(c, GS_ERR_CAPACITY, "tsdf: more blocks than pool slots (grow capacity)");
  return GS_OK;
}

gs_status gs_tsdf_rehash(gs_ctx* c, const gs_tsdf_grid* from, const gs_tsdf_grid* to, gs_stream_t stream) {
  if (!c) return GS_ERR_INVALID_ARG;
  gs_status st;
  if ((st = check_grid(c, from)) != GS_OK || (st = check_grid(c, to)) != GS_OK) return st;
  if (from->keys == to->keys || from->slots == to->slots)
    return fail(c, GS_ERR_INVALID_ARG, "gs_tsdf_rehash: the tables must not overlap");
  GS_CUDA(c, cudaSetDevice(c->device));
  launch_tsdf_rehash(to_internal(from), to_internal(to), c->num_sms, (cudaStream_t)stream);
  GS_CHECK_LAUNCH(c, "tsdf rehash");
  c->launches += 1;
  return GS_OK;
}

gs_status gs_tsdf_query(gs_ctx* c, const gs_tsdf_grid* grid, const float* points, int64_t n, float* tsdf,
                        float* weight, gs_stream_t stream) {
  if (!c) return GS_ERR_INVALID_ARG;
  gs_status st;
  if ((st = check_grid(c, grid)) != GS_OK) return st;
  if (n < 0 || (n > 0 && !points)) return fail(c, GS_ERR_INVALID_ARG, "gs_tsdf_query: bad arguments");
  GS_CUDA(c, cudaSetDevice(c->device));
  launch_tsdf_query(to_internal(grid), points, n, tsdf, weight, (cudaStream_t)stream);
  GS_CHECK_LAUNCH(c, "tsdf query");
  if (n > 0) c->launches += 1;
  return GS_OK;
}

gs_status gs_seed_tsdf(gs_ctx* c, const float* rgb, const float* depth, const gs_tsdf_grid* grid,
                       const gs_camera* cam, const gs_viewmat* view, int32_t sh_degree, float var_thr,
                       int32_t max_size, int32_t min_size, float* means, float* log_scales, float* quats,
                       float* opacity_logits, float* sh, int64_t capacity, int64_t* n_seeded, gs_stream_t stream) {
  NvtxRange nvtx_("gs_seed_tsdf");
  if (!c) return GS_ERR_INVALID_ARG;
  gs_status st;
  if ((st = check_cam(c, cam)) != GS_OK || (st = check_grid(c, grid)) != GS_OK) return st;
  if (!view || !finite_view(view) || !rgb || !depth || !n_seeded || capacity < 0 || sh_degree < 0 || sh_degree > 3)
    return fail(c, GS_ERR_INVALID_ARG, "gs_seed_tsdf: bad arguments");
  if (capacity > 0 && (!means || !log_scales || !quats || !opacity_logits || !sh))
    return fail(c, GS_ERR_INVALID_ARG, "gs_seed_tsdf: NULL output array");
  if (capacity > 0xFFFFFFF0ll) return fail(c, GS_ERR_INVALID_ARG, "gs_seed_tsdf: capacity too large");
  GS_CUDA(c, cudaSetDevice(c->device));
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t nl = 0;
  if ((st = qt_run(c, rgb, cam->width, cam->height, max_size, min_size, var_thr, &nl, s)) != GS_OK) return st;
  const float K4[4] = {cam->fx, cam->fy, cam->cx, cam->cy};
  float R[9], t[3];
  for (int k = 0; k < 9; ++k) R[k] = view->R[k];
  for (int k = 0; k < 3; ++k) t[k] = view->t[k];
  uint32_t* n_dev = c->qt_counters + 24;
  launch_tsdf_seed(to_internal(grid), rgb, depth, cam->width, cam->height, K4, R, t, sh_degree, c->qt_leaves, nl,
                   c->qt_claim, means, log_scales, quats, opacity_logits, sh, (uint32_t)capacity, n_dev, s);
  if (nl > 0) c->launches += 2;
  GS_CHECK_LAUNCH(c, "tsdf seed");
  GS_CUDA(c, cudaMemcpyAsync(c->h_pinned, n_dev, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  GS_CUDA(c, cudaStreamSynchronize(s));
  const int64_t n = (int64_t)(c->h_pinned[0] & 0xFFFFFFFFull);
  *n_seeded = n;
  if (n > capacity) return fail(c, GS_ERR_CAPACITY, "gs_seed_tsdf: more new Gaussians than capacity");
  return GS_OK;
}

gs_status gs_bin_tiles(gs_ctx* c, int64_t n, const float* mean2d, const float* extent, const float* depth,
                       int32_t width, int32_t height, int32_t tile_w, int32_t tile_h, uint64_t* keys, uint32_t* ids,
                       uint32_t* ranges, int64_t pair_capacity, int64_t* n_pairs, gs_stream_t stream) {
  NvtxRange nvtx_("gs_bin_tiles");
  if (!c) return GS_ERR_INVALID_ARG;
  if (n < 0 || n >= ((int64_t)1 << 31) || width < 1 || height < 1 || !n_pairs || pair_capacity < 0)
    return fail(c, GS_ERR_INVALID_ARG, "gs_bin_tiles: bad sizes");
  if (!raster_shape_supported(tile_w, tile_h)) return fail(c, GS_ERR_INVALID_ARG, "unsupported tile shape");
  if (n > 0 && (!mean2d || !extent || !depth)) return fail(c, GS_ERR_INVALID_ARG, "gs_bin_tiles: NULL input");
  if (!ranges) return fail(c, GS_ERR_INVALID_ARG, "gs_bin_tiles: NULL ranges");
  const int tiles_x = (width + tile_w - 1) / tile_w, tiles_y = (height + tile_h - 1) / tile_h;
  if (tiles_x > 65535 || tiles_y > 65535) return fail(c, GS_ERR_INVALID_ARG, "too many tiles per axis");
  cudaStream_t s = (cudaStream_t)stream;
  GS_CUDA(c, cudaSetDevice(c->device));
  const bool was_sync = c->sync;
  c->sync = true;
  gs_status st;
  const int64_t T = (int64_t)tiles_x * tiles_y;
  if ((st = ensure_n(c, std::max<int64_t>(n, 1))) != GS_OK || (st = ensure_tiles(c, T)) != GS_OK) {
    c->sync = was_sync;
    return st;
  }
  c->have_state = false;
  GS_CUDA(c, cudaMemsetAsync(c->d_bigmeta, 0, sizeof(uint32_t), s));
  // the count kernel zeroes the T counters it uses; the others stay as they were
  const bool counters_were_zero = c->counts_zero;
  c->counts_zero = false;
  launch_bin_prepare((int)n, mean2d, extent, depth, tile_w, tile_h, tiles_x, tiles_y, c->zkey, c->tiles, c->rects,
                     c->bigq, c->d_bigmeta, s);
  if (n > 0) c->launches += 1;
  TileMap map{};
  map.views = 1;
  map.n_per_view = (int)n;
  map.tiles_x[0] = tiles_x;
  for (int v = 1; v <= kMaxViews; ++v) map.tile_base[v] = (uint32_t)T;
  st = bin_and_sort(c, (int)n, map, s, false);
  c->counts_zero = c->counts_zero && counters_were_zero;
  c->sync = was_sync;
  if (st != GS_OK) return st;
  const int64_t P = c->st_pairs;
  *n_pairs = P;
  GS_CUDA(c, cudaMemcpyAsync(ranges, c->ranges, sizeof(uint2) * (size_t)T, cudaMemcpyDeviceToDevice, s));
  if (P > pair_capacity) {
    GS_CUDA(c, cudaStreamSynchronize(s));
    return fail(c, GS_ERR_CAPACITY, "gs_bin_tiles: output capacity too small");
  }
  if (P > 0) {
    if (!keys || !ids) return fail(c, GS_ERR_INVALID_ARG, "gs_bin_tiles: NULL keys/ids");
    launch_export_keys_ranges(c->ranges, (int)T, c->pv[c->st_pair_buf], c->zkey, (uint32_t)P, keys, ids, s);
    c->launches += 1;
  }
  GS_CHECK_LAUNCH(c, "bin export");
  GS_CUDA(c, cudaStreamSynchronize(s));
  return GS_OK;
}

gs_status gs_get_projection(gs_ctx* c, float* mean2d, float* cov2d, float* depth, float* rgb, float* opacity,
                            int32_t* tiles, gs_stream_t stream) {
  if (!c) return GS_ERR_INVALID_ARG;
  if (!c->have_state) return fail(c, GS_ERR_STATE, "no forward pass on this context");
  GS_CUDA(c, cudaSetDevice(c->device));
  launch_export_projection((int)(c->st_n * c->st_views), c->feat, c->tiles, mean2d, cov2d, depth, rgb, opacity, tiles,
                           (cudaStream_t)stream);
  if (c->st_n > 0) c->launches += 1;
  GS_CHECK_LAUNCH(c, "export projection");
  return GS_OK;
}

gs_status gs_get_tile_ranges(gs_ctx* c, uint32_t* ranges, int64_t n_tiles, gs_stream_t stream) {
  if (!c) return GS_ERR_INVALID_ARG;
  if (!c->have_state) return fail(c, GS_ERR_STATE, "no forward pass on this context");
  if (!ranges || n_tiles != c->st_tiles)
    return fail(c, GS_ERR_INVALID_ARG, "gs_get_tile_ranges: ranges is NULL or n_tiles is not the forward pass's");
  GS_CUDA(c, cudaSetDevice(c->device));
  GS_CUDA(c, cudaMemcpyAsync(ranges, c->ranges, sizeof(uint2) * (size_t)n_tiles, cudaMemcpyDeviceToDevice,
                             (cudaStream_t)stream));
  return GS_OK;
}

gs_status gs_get_tile_order(gs_ctx* c, uint32_t* order, int64_t n_tiles, gs_stream_t stream) {
  if (!c) return GS_ERR_INVALID_ARG;
  if (!c->have_state) return fail(c, GS_ERR_STATE, "no forward pass on this context");
  if (!c->st_ordered) return fail(c, GS_ERR_STATE, "the last forward pass visited the tiles in index order");
  if (!order || n_tiles != c->st_tiles)
    return fail(c, GS_ERR_INVALID_ARG, "gs_get_tile_order: order is NULL or n_tiles is not the forward pass's");
  GS_CUDA(c, cudaSetDevice(c->device));
  GS_CUDA(c, cudaMemcpyAsync(order, c->torder, sizeof(uint32_t) * (size_t)n_tiles, cudaMemcpyDeviceToDevice,
                             (cudaStream_t)stream));
  return GS_OK;
}

gs_status gs_state_token(const gs_ctx* c, uint64_t* token) {
  if (!c || !token) return GS_ERR_INVALID_ARG;
  *token = c->have_state ? c->state_token : 0;
  return GS_OK;
}

int gs_bounds_checked(void) {
#ifdef GS_CHECKED
  return 1;
#else
  return 0;
#endif
}

gs_status gs_ctx_inject_bounds_fault(gs_ctx* c) {
  if (!c) return GS_ERR_INVALID_ARG;
  GS_CUDA(c, cudaSetDevice(c->device));
  GS_CUDA(c, cudaMemset(c->d_bounds, 0xFF, sizeof(uint32_t)));
  return GS_OK;
}

gs_status gs_ctx_inject_alloc_failure(gs_ctx* c, int32_t after) {
  if (!c || after < 0) return GS_ERR_INVALID_ARG;
  c->fail_alloc = after;
  return GS_OK;
}

gs_status gs_count_nonfinite(gs_ctx* c, const float* x, int64_t n, int64_t* count, gs_stream_t stream) {
  if (!c) return GS_ERR_INVALID_ARG;
  NvtxRange nvtx_("gs_count_nonfinite");
  if (n < 0 || !count || (n > 0 && !x)) return fail(c, GS_ERR_INVALID_ARG, "gs_count_nonfinite: bad arguments");
  GS_CUDA(c, cudaSetDevice(c->device));
  if (!c->d_count) GS_CUDA(c, cudaMalloc((void**)&c->d_count, sizeof(unsigned long long)));
  cudaStream_t s = (cudaStream_t)stream;
  launch_count_nonfinite(x, n, c->d_count, c->num_sms, s);
  if (n > 0) c->launches += 1;
  GS_CHECK_LAUNCH(c, "count non-finite");
  GS_CUDA(c, cudaMemcpyAsync(c->h_pinned, c->d_count, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  GS_CUDA(c, cudaStreamSynchronize(s));
  *count = (int64_t)c->h_pinned[0];
  if (*count > 0) return fail(c, GS_ERR_NONFINITE, "non-finite values found");
  return GS_OK;
}

}  // extern "C"
