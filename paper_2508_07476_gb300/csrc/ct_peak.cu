// Measurement support, not part of the method: the device's FP32 FMA rate.
//
// The benchmark states the FP32 roofline of the stencil formulation against a
// measured rate rather than one derived from unit counts and a nominal clock.
// Every thread runs kChains independent FMA chains (enough independent work
// to cover the pipe's latency at full occupancy), so the kernel is bound by
// FFMA issue alone; its operands come from the kernel parameters, and the
// result is stored only when it equals a value it never takes, so the
// compiler keeps every FMA.
#include <cuda_runtime.h>

#include "ct.h"
#include "ct_launch.h"

namespace ct {
ct_status set_error(ct_status st, const char* fmt, ...);
}

namespace {

constexpr int kChains = 16;
constexpr int kPeakThreads = 256;

__global__ void __launch_bounds__(kPeakThreads) k_ffma_rate(int64_t iters, float b, float c, float* sink) {
  float a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = (float)(threadIdx.x + i);
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = fmaf(a[i], b, c);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  if (s == -1.2345f) sink[blockIdx.x] = s;
}

}  // namespace

extern "C" ct_status ct_fp32_fma_rate(int64_t iterations, double* fma_per_s, int32_t* sm_count, double* ms) {
  if (!fma_per_s || iterations < 1) return ct::set_error(CT_ERR_INVALID, "bad argument");
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return ct::set_error(CT_ERR_NO_DEVICE, "no CUDA device is available");
  }
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
      (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ffma_rate, kPeakThreads, 0)) != cudaSuccess)
    return ct::set_error(CT_ERR_CUDA, "device query: %s", cudaGetErrorString(e));
  const int grid = sms * per_sm;  // one full wave: every SM at full occupancy
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float elapsed = 0.f;
  if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) == cudaSuccess &&
      (e = cudaEventCreate(&e0)) == cudaSuccess && (e = cudaEventCreate(&e1)) == cudaSuccess) {
    k_ffma_rate<<<grid, kPeakThreads, 0, st>>>(iterations / 8 + 1, 0.999f, 1e-3f, nullptr);  // warm-up
    e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) {
      k_ffma_rate<<<grid, kPeakThreads, 0, st>>>(iterations, 0.999f, 1e-3f, nullptr);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&elapsed, e0, e1);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  if (e != cudaSuccess) return ct::set_error(CT_ERR_CUDA, "FMA rate kernel: %s", cudaGetErrorString(e));
  const double fmas = (double)grid * kPeakThreads * (double)iterations * kChains;
  *fma_per_s = fmas / (elapsed * 1e-3);
  if (sm_count) *sm_count = sms;
  if (ms) *ms = elapsed;
  return CT_OK;
}
