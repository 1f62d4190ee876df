// Issue-rate probes of the two ALU pipes the raster passes run on: FP32 FMA
// and the MUFU exp2 (ex2.approx).  They give the measured denominators of
// the raster passes' ALU roofline (the passes are neither HBM- nor tensor-
// bound: per (pixel, Gaussian) pair they evaluate a 2x2 quadratic form, one
// exp2 and a blend or its gradient).
//
// Each kernel runs, per thread, eight independent dependency chains of one
// instruction kind in a fully occupied grid, so the pipe, not the latency of
// a chain, bounds it.  Thread 0 of block 0 reads the SM cycle counter and the
// global nanosecond timer around its own loop, which gives the SM clock the
// probe ran at.
#include <cstdint>

#include "../../include/gsplat.h"
#include <cuda_runtime.h>

namespace gs {
namespace {

constexpr int kPeakThreads = 256;
constexpr int kChains = 8;

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// clk[0..1] = (cycles, ns) of block 0's thread 0 (clk[2..3] for the exp2
// probe); sink receives a value only if the chains end on `magic` (never),
// so that the compiler keeps them.
__global__ void __launch_bounds__(kPeakThreads) fma_probe_kernel(float b, float c, int iters, float magic,
                                                                 unsigned long long* clk, float* sink) {
  float x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = (float)(threadIdx.x + k) * 1e-3f;
  uint64_t c0 = 0, t0 = 0;
  const bool timer = blockIdx.x == 0 && threadIdx.x == 0;
  if (timer) {
    t0 = global_ns();
    c0 = clock64();
  }
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 16; ++r) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) x[k] = __fmaf_rn(x[k], b, c);
    }
  }
  if (timer) {
    const uint64_t c1 = clock64(), t1 = global_ns();
    clk[0] = c1 - c0;
    clk[1] = t1 - t0;
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  if (s == magic) sink[0] = s;
}

__device__ __forceinline__ float ex2_neg(float x) {
  float y;
  asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-x));
  return y;
}

__global__ void __launch_bounds__(kPeakThreads) ex2_probe_kernel(int iters, float magic, unsigned long long* clk,
                                                                 float* sink) {
  float x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = (float)(threadIdx.x + k) * 1e-3f;
  uint64_t c0 = 0, t0 = 0;
  const bool timer = blockIdx.x == 0 && threadIdx.x == 0;
  if (timer) {
    t0 = global_ns();
    c0 = clock64();
  }
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 16; ++r) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) x[k] = ex2_neg(x[k]);  // x -> 2^-x stays in (0, 1]
    }
  }
  if (timer) {
    const uint64_t c1 = clock64(), t1 = global_ns();
    clk[2] = c1 - c0;
    clk[3] = t1 - t0;
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  if (s == magic) sink[0] = s;
}

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" gs_status gs_measure_alu_peaks(int device, int32_t iters, gs_alu_peaks* out) {
  if (!out || device < 0 || iters < 1 || iters > (1 << 24)) return GS_ERR_INVALID_ARG;
  *out = gs_alu_peaks{};
  if (cudaSetDevice(device) != cudaSuccess) return GS_ERR_CUDA;
  int sms = 0, per_sm = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms < 1)
    return GS_ERR_CUDA;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_probe_kernel, kPeakThreads, 0) != cudaSuccess ||
      per_sm < 1)
    return GS_ERR_CUDA;
  int per_sm_ex2 = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_ex2, ex2_probe_kernel, kPeakThreads, 0) != cudaSuccess ||
      per_sm_ex2 < 1)
    return GS_ERR_CUDA;
  unsigned long long* clk = nullptr;
  float* sink = nullptr;
  cudaEvent_t e[4] = {};
  cudaError_t err = cudaMalloc((void**)&clk, 4 * sizeof(unsigned long long));
  if (err == cudaSuccess) err = cudaMalloc((void**)&sink, sizeof(float));
  for (int k = 0; k < 4 && err == cudaSuccess; ++k) err = cudaEventCreate(&e[k]);
  const int grid_f = sms * per_sm, grid_e = sms * per_sm_ex2;
  const int iters_e = iters / 4 > 0 ? iters / 4 : 1;  // the exp2 pipe is several times narrower
  if (err == cudaSuccess) {
    // warm-up launches (clock ramp, module load), then the timed ones
    fma_probe_kernel<<<grid_f, kPeakThreads>>>(0.999f, 1e-7f, iters / 8 + 1, -1.f, clk, sink);
    ex2_probe_kernel<<<grid_e, kPeakThreads>>>(iters_e / 8 + 1, -1.f, clk, sink);
    cudaEventRecord(e[0]);
    fma_probe_kernel<<<grid_f, kPeakThreads>>>(0.999f, 1e-7f, iters, -1.f, clk, sink);
    cudaEventRecord(e[1]);
    cudaEventRecord(e[2]);
    ex2_probe_kernel<<<grid_e, kPeakThreads>>>(iters_e, -1.f, clk, sink);
    cudaEventRecord(e[3]);
    err = cudaGetLastError();
  }
  if (err == cudaSuccess) err = cudaDeviceSynchronize();
  float ms_f = 0.f, ms_e = 0.f;
  unsigned long long h[4] = {0, 0, 0, 0};
  if (err == cudaSuccess) err = cudaEventElapsedTime(&ms_f, e[0], e[1]);
  if (err == cudaSuccess) err = cudaEventElapsedTime(&ms_e, e[2], e[3]);
  if (err == cudaSuccess) err = cudaMemcpy(h, clk, sizeof(h), cudaMemcpyDeviceToHost);
  for (int k = 0; k < 4; ++k)
    if (e[k]) cudaEventDestroy(e[k]);
  cudaFree(clk);
  cudaFree(sink);
  if (err != cudaSuccess) return GS_ERR_CUDA;
  const double fmas = (double)iters * 16.0 * kChains * (double)grid_f * kPeakThreads;
  const double ex2s = (double)iters_e * 16.0 * kChains * (double)grid_e * kPeakThreads;
  out->num_sms = sms;
  out->fma_ms = ms_f;
  out->ex2_ms = ms_e;
  out->fma_tflops = ms_f > 0.f ? 2.0 * fmas / (ms_f * 1e-3) / 1e12 : 0.0;
  out->ex2_gops = ms_e > 0.f ? ex2s / (ms_e * 1e-3) / 1e9 : 0.0;
  out->fma_sm_mhz = h[1] ? (double)h[0] / (double)h[1] * 1e3 : 0.0;
  out->ex2_sm_mhz = h[3] ? (double)h[2] / (double)h[3] * 1e3 : 0.0;
  out->fma_per_sm_clk = (out->fma_sm_mhz > 0.0 && ms_f > 0.f)
                            ? fmas / (ms_f * 1e-3) / (out->fma_sm_mhz * 1e6) / sms : 0.0;
  out->ex2_per_sm_clk = (out->ex2_sm_mhz > 0.0 && ms_e > 0.f)
                            ? ex2s / (ms_e * 1e-3) / (out->ex2_sm_mhz * 1e6) / sms : 0.0;
  return GS_OK;
}
