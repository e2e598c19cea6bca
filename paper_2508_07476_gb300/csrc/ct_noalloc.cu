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
// The array belongs to this file's module of the library.  Under CUDA's lazy
// module loading the module, and with it the array's 8 MiB, is loaded on a
// device by the first call there, which also looks the array's address up
// once (cudaGetSymbolAddress, with that device current) and may synchronise
// the device while loading: make that first call at start-up, before any
// stream capture.  The array then stays resident until the process exits.
// The address is kept per device together with the identity of the CUDA
// context it belongs to; after a device reset the next call looks it up again
// in the new context.  Every call shares the one array and the array keeps the
// last call's contents: the counters are zeroed on the stream at the start of
// each call, and calls that overlap on the GPU (on different streams, or
// different host threads) race on the list.
#include <cuda.h>  // CUcontext; the two context queries are fetched from the driver at run time
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
struct Cached {
  unsigned long long ctx_id;  // identity of the context the address belongs to (0: unknown)
  unsigned char* addr;
};
Cached g_addr[kMaxDevices] = {};

using CtxGetCurrent = CUresult (*)(CUcontext*);
using CtxGetId = CUresult (*)(CUcontext, unsigned long long*);

// Unique identity of the calling thread's current context (0 when there is
// none yet or the driver cannot say).  Context identities are never reused
// within a process, unlike context handles.
unsigned long long current_context_id() {
  static const CtxGetCurrent get_current = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    return cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
                   q == cudaDriverEntryPointSuccess
               ? reinterpret_cast<CtxGetCurrent>(p)
               : nullptr;
  }();
  static const CtxGetId get_id = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    return cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
                   q == cudaDriverEntryPointSuccess
               ? reinterpret_cast<CtxGetId>(p)
               : nullptr;
  }();
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
    return 0;
  return id;
}

// Device address of the scratch array on the current device, looked up once
// per device and context.
ct_status scratch_address(unsigned char** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return ct::set_error(CT_ERR_NO_DEVICE, "no CUDA device is available: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return ct::set_error(CT_ERR_UNSUPPORTED, "device index %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_mu);
  Cached& c = g_addr[dev];
  const unsigned long long id = current_context_id();
  if (!c.addr || id != c.ctx_id) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_eig_scratch);  // with no context yet, this creates the primary one
    if (e != cudaSuccess)
      return ct::set_error(CT_ERR_CUDA, "scratch address lookup failed: %s", cudaGetErrorString(e));
    c.addr = static_cast<unsigned char*>(p);
    c.ctx_id = id ? id : current_context_id();
  }
  *out = c.addr;
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
  bool mixed = precision == CT_PREC_MIXED;
  fb.gap = ct::degenerate_gap(mixed);
  cudaError_t e = cudaMemsetAsync(base, 0, kListOffset, st);
  if (e == cudaSuccess) e = ct::launch_eig_only(d_S, n, d_evals, d_evec, mixed, fb, st);
  if (e == cudaSuccess) e = ct::launch_eig_only_fallback(d_S, n, d_evals, d_evec, mixed, fb, n, st);
  if (e != cudaSuccess) return ct::set_error(CT_ERR_CUDA, "eigen launch failed: %s", cudaGetErrorString(e));
  return CT_OK;
}
