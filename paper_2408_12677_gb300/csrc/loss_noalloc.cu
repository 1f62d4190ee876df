// gs_loss_l1_noalloc: the L1 loss of gs_loss_l1 without any device
// allocation, for callers that are not allowed to call cudaMalloc.
//
// gs_loss_l1 keeps its per-block partial sums in scratch that a context grows
// with cudaMalloc.  Some callers cannot allocate on the device at that point:
// a process that has handed all of the GPU's memory to its own pool (where a
// raw cudaMalloc fails or fragments the pool), or a latency-critical loop that
// must not pay for an allocation and the implicit synchronisation it brings.
// This variant takes its scratch from a fixed array compiled into the
// library instead, so it allocates nothing: every GPU that loads libgsplat
// holds this array (about 96 KB) until the process exits.
#include <mutex>

#include "../../include/gsplat.h"
#include "internal.h"

namespace {

constexpr int64_t kMaxPixels = GS_LOSS_NOALLOC_MAX_PIXELS;
constexpr int kScratchFloats = 3 * ((int)(kMaxPixels / 2048)) + 4;  // partials of <= kMaxPixels / 2048 blocks + scale
constexpr int kMaxDevices = 64;

}  // namespace

// The scratch shared by every call on a device: per-block partial sums of the
// loss followed by the depth-gradient scale.  Each call rewrites every value
// it later reads, so no state carries over from one call to the next.
static __device__ __align__(256) float gs_loss_noalloc_scratch[kScratchFloats];

namespace {

std::mutex g_setup_mu;
float* g_scratch[kMaxDevices] = {};  // device address of the array, per device

// Once per device, with that device current: the host-side name of the
// array is only a stand-in, so fetch the array's device address.
cudaError_t scratch_for(int dev, float** out) {
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, gs_loss_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch[dev] = static_cast<float*>(p);
  }
  *out = g_scratch[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" gs_status gs_loss_l1_noalloc(const gs_camera* cam, const float* color, const float* depth,
                                        const float* target_rgb, const float* target_depth, float w_color,
                                        float w_depth, float* loss, float* dL_dcolor, float* dL_ddepth,
                                        gs_stream_t stream) {
  if (!cam || cam->width < 1 || cam->height < 1) return GS_ERR_INVALID_ARG;
  if (!color || !depth || !target_rgb || !target_depth || !loss || !dL_dcolor || !dL_ddepth) return GS_ERR_INVALID_ARG;
  const int64_t npix = (int64_t)cam->width * cam->height;
  if (npix > kMaxPixels) return GS_ERR_CAPACITY;
  if (3 * (int64_t)gs::loss_blocks((int)npix) + 1 > kScratchFloats) return GS_ERR_CAPACITY;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return GS_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return GS_ERR_INVALID_ARG;
  float* scratch = nullptr;
  if (scratch_for(dev, &scratch) != cudaSuccess) return GS_ERR_CUDA;
  gs::LossArgs la;
  la.views = 1;
  la.n_blocks = gs::loss_blocks((int)npix);
  la.w_color = w_color;
  la.w_depth = w_depth;
  la.loss = loss;
  la.v[0] = gs::LossView{(int)npix, 0, color, depth, target_rgb, target_depth, dL_dcolor, dL_ddepth};
  gs::launch_loss(la, scratch, (cudaStream_t)stream, nullptr);
  return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}
