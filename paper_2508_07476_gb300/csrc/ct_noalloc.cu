// ct_eig_smallest_noalloc: the eigen stage without any device allocation.
//
// ct_eig_smallest keeps its list of near-degenerate voxels in scratch memory
// that the plan allocates.  Some callers cannot allocate at all once they are
// running: a host framework that owns every byte of device memory through its
// own pool, a service that forbids allocation after start-up because
// cudaMalloc may synchronise the device and stall other work, or code that
// must not fail half-way for lack of memory.  This entry point serves them: it
// needs no plan and keeps its scratch (a counter and the re-solve list) in a
// fixed-size array that lives in the library's device image, so a call never
// allocates, frees or asks another library to allocate.
//
// The array is loaded with the module on every device that uses the library
// and stays resident until the process exits.  The first call on a device,
// with that device current, looks its address up once (cudaGetSymbolAddress);
// make that first call before any stream capture.  Every call shares the one
// array and the array keeps the last call's contents: the counters are zeroed
// on the stream at the start of each call, and calls that overlap on the GPU
// (on different streams, or different host threads) race on the list.
#include <cuda_runtime.h>

#include <mutex>

#include "ct.h"
#include "ct_launch.h"

namespace ct {
ct_status set_error(ct_status st, const char* fmt, ...);
}

namespace {

constexpr int64_t kMaxVoxels = (int64_t)1 << 20;  // voxels per call (list capacity)
constexpr size_t kTotalOffset = 8;                 // unsigned long long running total
constexpr size_t kListOffset = 256;                // int64_t list[kMaxVoxels]
constexpr size_t kScratchBytes = kListOffset + sizeof(int64_t) * kMaxVoxels;  // 8 MiB + 256 B

static __device__ __align__(256) unsigned char g_eig_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once).
ct_status scratch_address(unsigned char** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return ct::set_error(CT_ERR_NO_DEVICE, "no CUDA device is available: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return ct::set_error(CT_ERR_UNSUPPORTED, "device index %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_eig_scratch);
    if (e != cudaSuccess)
      return ct::set_error(CT_ERR_CUDA, "scratch address lookup failed: %s", cudaGetErrorString(e));
    g_addr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_addr[dev];
  return CT_OK;
}

}  // namespace

extern "C" ct_status ct_eig_smallest_noalloc(const float* d_S, int64_t n, float* d_evals, float* d_evec,
                                             int32_t precision, void* stream) {
  if (!d_S || !d_evec) return ct::set_error(CT_ERR_INVALID, "NULL argument");
  if (precision != CT_PREC_FP32 && precision != CT_PREC_MIXED) return ct::set_error(CT_ERR_INVALID, "bad precision");
  if (n < 0) return ct::set_error(CT_ERR_INVALID, "n must be >= 0");
  if (n > kMaxVoxels)
    return ct::set_error(CT_ERR_INVALID, "n = %lld exceeds the %lld voxels one call can take (static scratch limit)",
                         (long long)n, (long long)kMaxVoxels);
  if (n == 0) return CT_OK;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || count == 0) {
    cudaGetLastError();
    return ct::set_error(CT_ERR_NO_DEVICE, "no CUDA device is available");
  }
  unsigned char* base = nullptr;
  ct_status rc = scratch_address(&base);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  ct::Fallback fb;
  fb.count = reinterpret_cast<int*>(base);
  fb.total = reinterpret_cast<unsigned long long*>(base + kTotalOffset);
  fb.list = reinterpret_cast<int64_t*>(base + kListOffset);
  fb.cap = kMaxVoxels;
  cudaError_t e = cudaMemsetAsync(base, 0, kListOffset, st);
  bool mixed = precision == CT_PREC_MIXED;
  if (e == cudaSuccess) e = ct::launch_eig_only(d_S, n, d_evals, d_evec, mixed, fb, st);
  if (e == cudaSuccess) e = ct::launch_eig_only_fallback(d_S, n, d_evals, d_evec, mixed, fb, n, st);
  if (e != cudaSuccess) return ct::set_error(CT_ERR_CUDA, "eigen launch failed: %s", cudaGetErrorString(e));
  return CT_OK;
}
