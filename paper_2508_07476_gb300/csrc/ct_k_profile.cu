// Transmural HA profile: histogram of the helical angle against normalised
// wall depth (the paper's analysis module plots this profile from the HA map
// of Figure 1(c)).  A reduction over the pipeline's HA output, privatised per
// CTA in shared memory and flushed once per CTA with 64-bit atomics.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

#include "ct.h"

namespace ct {
ct_status set_error(ct_status st, const char* fmt, ...);
}

namespace {

constexpr int kProfThreads = 256;
constexpr int kProfMaxBins = 16384;  // 64 KB of shared uint32 counters

struct ProfDev {
  float c[3], a[3];
  float r_in, inv_w;
  int nd, nh;
  int64_t lo[3];
  int n0, n1, n2;
};

template <int TYPE>
__device__ __forceinline__ float decode_ha(const void* ha, int64_t i, bool& ok) {
  if (TYPE == CT_OUT_F32) {
    const float v = __ldg(reinterpret_cast<const float*>(ha) + i);
    ok = isfinite(v);
    return v;
  } else if (TYPE == CT_OUT_F16) {
    const float v = __half2float(reinterpret_cast<const __half*>(ha)[i]);
    ok = isfinite(v);
    return v;
  } else {
    const int code = __ldg(reinterpret_cast<const uint8_t*>(ha) + i);
    ok = code != 0;
    return (float)code * (180.f / 256.f) - 90.f;
  }
}

template <int TYPE>
__global__ void __launch_bounds__(kProfThreads) k_transmural(const void* __restrict__ ha,
                                                             const uint8_t* __restrict__ mask, ProfDev P,
                                                             unsigned long long* __restrict__ hist) {
  extern __shared__ uint32_t sh[];
  const int nb = P.nd * P.nh;
  for (int k = threadIdx.x; k < nb; k += kProfThreads) sh[k] = 0u;
  __syncthreads();
  const int64_t rows = (int64_t)P.n1 * P.n2;
  for (int64_t row = blockIdx.x; row < rows; row += gridDim.x) {
    const int yr = (int)(row % P.n1), zr = (int)(row / P.n1);
    const float dy = (float)(P.lo[1] + yr) - P.c[1], dz = (float)(P.lo[2] + zr) - P.c[2];
    const int64_t base = row * P.n0;
    for (int xr = threadIdx.x; xr < P.n0; xr += kProfThreads) {
      const int64_t i = base + xr;
      int bin = -1;
      bool ok = mask == nullptr || __ldg(mask + i) != 0;
      if (ok) {
        const float h = decode_ha<TYPE>(ha, i, ok);
        const float dx = (float)(P.lo[0] + xr) - P.c[0];
        const float t = dx * P.a[0] + dy * P.a[1] + dz * P.a[2];
        const float rx = dx - t * P.a[0], ry = dy - t * P.a[1], rz = dz - t * P.a[2];
        const float d = (sqrtf(rx * rx + ry * ry + rz * rz) - P.r_in) * P.inv_w;
        if (ok && d >= 0.f && d < 1.f) {
          const int kd = min((int)(d * (float)P.nd), P.nd - 1);
          const int kh = min(max((int)((h + 90.f) * ((float)P.nh / 180.f)), 0), P.nh - 1);
          bin = kd * P.nh + kh;
        }
      }
      // neighbouring voxels mostly share a bin: one shared-memory atomic per distinct bin of the warp
      const unsigned same = __match_any_sync(__activemask(), bin);
      if (bin >= 0 && (threadIdx.x & 31) == __ffs(same) - 1) atomicAdd(&sh[bin], (uint32_t)__popc(same));
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < nb; k += kProfThreads)
    if (sh[k]) atomicAdd(hist + k, (unsigned long long)sh[k]);
}

}  // namespace

extern "C" ct_status ct_transmural_profile(const ct_profile_spec* spec, const int64_t vol_dims[3],
                                           const int64_t lo[3], const int64_t n[3], const void* d_ha,
                                           const uint8_t* d_mask, uint64_t* d_hist, void* stream) {
  if (!spec || !vol_dims || !lo || !n || !d_ha || !d_hist) return ct::set_error(CT_ERR_INVALID, "NULL argument");
  for (int k = 0; k < 3; ++k)
    if (vol_dims[k] < 1 || n[k] < 1 || lo[k] < 0 || lo[k] + n[k] > vol_dims[k] || vol_dims[k] > (1 << 24))
      return ct::set_error(CT_ERR_INVALID, "box outside the volume");
  if (n[0] > (1 << 30) || n[1] * n[2] > ((int64_t)1 << 40)) return ct::set_error(CT_ERR_INVALID, "box too large");
  if (spec->n_depth < 1 || spec->n_ha < 1 || (int64_t)spec->n_depth * spec->n_ha > kProfMaxBins)
    return ct::set_error(CT_ERR_INVALID, "n_depth * n_ha must be in [1, %d]", kProfMaxBins);
  if (!(spec->r_out > spec->r_in) || !std::isfinite(spec->r_in) || !std::isfinite(spec->r_out))
    return ct::set_error(CT_ERR_INVALID, "r_out must exceed r_in");
  if (spec->ha_type != CT_OUT_F32 && spec->ha_type != CT_OUT_F16 && spec->ha_type != CT_OUT_U8Q)
    return ct::set_error(CT_ERR_INVALID, "unknown HA encoding %d", spec->ha_type);
  if (spec->reserved != 0) return ct::set_error(CT_ERR_INVALID, "reserved must be 0");
  const double an = std::sqrt(spec->lv_axis[0] * spec->lv_axis[0] + spec->lv_axis[1] * spec->lv_axis[1] +
                              spec->lv_axis[2] * spec->lv_axis[2]);
  if (!(an > 0.0) || !std::isfinite(an)) return ct::set_error(CT_ERR_INVALID, "axis must be finite and non-zero");
  ProfDev P;
  for (int k = 0; k < 3; ++k) {
    P.c[k] = (float)spec->lv_center[k];
    P.a[k] = (float)(spec->lv_axis[k] / an);
    P.lo[k] = lo[k];
  }
  P.r_in = (float)spec->r_in;
  P.inv_w = (float)(1.0 / (spec->r_out - spec->r_in));
  P.nd = spec->n_depth;
  P.nh = spec->n_ha;
  P.n0 = (int)n[0];
  P.n1 = (int)n[1];
  P.n2 = (int)n[2];
  const int64_t rows = n[1] * n[2];
  const int grid = (int)(rows < 152 * 4 ? rows : 152 * 4);
  const size_t smem = sizeof(uint32_t) * (size_t)P.nd * P.nh;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  unsigned long long* h = reinterpret_cast<unsigned long long*>(d_hist);
  switch (spec->ha_type) {
    case CT_OUT_F32:
      e = cudaFuncSetAttribute(k_transmural<CT_OUT_F32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess) k_transmural<CT_OUT_F32><<<grid, kProfThreads, smem, st>>>(d_ha, d_mask, P, h);
      break;
    case CT_OUT_F16:
      e = cudaFuncSetAttribute(k_transmural<CT_OUT_F16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess) k_transmural<CT_OUT_F16><<<grid, kProfThreads, smem, st>>>(d_ha, d_mask, P, h);
      break;
    default:
      e = cudaFuncSetAttribute(k_transmural<CT_OUT_U8Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess) k_transmural<CT_OUT_U8Q><<<grid, kProfThreads, smem, st>>>(d_ha, d_mask, P, h);
      break;
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return ct::set_error(CT_ERR_CUDA, "profile launch failed: %s", cudaGetErrorString(e));
  return CT_OK;
}
