// Measured ALU peaks of the GPU (FP32 and FP64 fused multiply-add), the
// denominators a reader can set beside the derived unit-count peak of the
// synthesis roofline. Every thread of a full grid runs kChains independent FMA
// chains, so the FMA pipes never wait on a dependency; a data-dependent store
// that never happens in practice keeps the chains live.
#include <cstdint>

#include "msrc.h"
#include "msrc_internal.h"

namespace msrc {
namespace {

constexpr int kPeakThreads = 256;
constexpr int kChains = 16;

template <typename T>
__global__ void __launch_bounds__(kPeakThreads) k_fma_peak(T* out, T b, T c, int iters) {
  T a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = T(threadIdx.x + i) * T(1e-3);
  for (int it = 0; it < iters; it += 4) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int i = 0; i < kChains; ++i) a[i] = fma(a[i], b, c);
  }
  T s = T(0);
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  if (s == T(-1.25e30)) out[0] = s;
}

// Best of `reps` timed launches after one warm-up; TFLOP/s at 2 flops per FMA.
template <typename T>
cudaError_t time_peak(void* scratch, cudaStream_t st, int iters, double* tflops) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int blocks = sms * (2048 / kPeakThreads);
  cudaEvent_t e0, e1;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess) return e;
  if ((e = cudaEventCreate(&e1)) != cudaSuccess) { cudaEventDestroy(e0); return e; }
  const T b = T(0.999999), c = T(1e-6);
  float best = 0.0f;
  for (int r = 0; r < 6 && e == cudaSuccess; ++r) {
    cudaEventRecord(e0, st);
    k_fma_peak<T><<<blocks, kPeakThreads, 0, st>>>(static_cast<T*>(scratch), b, c, iters);
    cudaEventRecord(e1, st);
    e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && r > 0 && (best == 0.0f || ms < best)) best = ms;
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return e;
  const double flops = 2.0 * double(blocks) * kPeakThreads * kChains * double(iters);
  *tflops = flops / (double(best) * 1e-3) / 1e12;
  return cudaSuccess;
}

}  // namespace
}  // namespace msrc

extern "C" msrc_status msrc_measure_alu_peaks(void* scratch_dev, void* stream, double* fp32_tflops,
                                              double* fp64_tflops) {
  if (!scratch_dev || !fp32_tflops || !fp64_tflops) {
    msrc::set_last_error("null scratch or output");
    return MSRC_ERR_INVALID_ARG;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // a few milliseconds of work per launch for either type on this GPU class
  cudaError_t e = msrc::time_peak<float>(scratch_dev, st, 1 << 14, fp32_tflops);
  if (e == cudaSuccess) e = msrc::time_peak<double>(scratch_dev, st, 1 << 8, fp64_tflops);
  if (e != cudaSuccess) {
    msrc::set_last_error(cudaGetErrorString(e));
    return MSRC_ERR_CUDA;
  }
  return MSRC_OK;
}
