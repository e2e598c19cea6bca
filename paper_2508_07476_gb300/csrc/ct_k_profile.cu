// Transmural HA profile: histogram of the helical angle against normalised
// wall depth (the paper's analysis module plots this profile from the HA map
// of Figure 1(c)).  A reduction over the pipeline's HA output, privatised per
// CTA in shared memory and flushed once per CTA with 64-bit atomics.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
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

// 8 consecutive HA values from one 16- (or 32-) byte aligned load.
template <int TYPE>
__device__ __forceinline__ void load8(const void* ha, int64_t i, float h[8], bool ok[8]) {
  if (TYPE == CT_OUT_F32) {
    const float4* p = reinterpret_cast<const float4*>(reinterpret_cast<const float*>(ha) + i);
    const float4 a = __ldg(p), b = __ldg(p + 1);
    h[0] = a.x; h[1] = a.y; h[2] = a.z; h[3] = a.w; h[4] = b.x; h[5] = b.y; h[6] = b.z; h[7] = b.w;
#pragma unroll
    for (int k = 0; k < 8; ++k) ok[k] = isfinite(h[k]);
  } else if (TYPE == CT_OUT_F16) {
    const uint4 q = __ldg(reinterpret_cast<const uint4*>(reinterpret_cast<const __half*>(ha) + i));
    const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&w[k]));
      h[2 * k] = f.x;
      h[2 * k + 1] = f.y;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) ok[k] = isfinite(h[k]);
  } else {
    const uint2 q = __ldg(reinterpret_cast<const uint2*>(reinterpret_cast<const uint8_t*>(ha) + i));
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int code = ((k < 4 ? q.x : q.y) >> (8 * (k & 3))) & 0xff;
      ok[k] = code != 0;
      h[k] = (float)code * (180.f / 256.f) - 90.f;
    }
  }
}

// Each thread takes 8 consecutive voxels of a row (one vector load of HA and
// of the mask when the rows allow it: VEC), counts runs of equal bins itself
// and adds a run to the CTA's shared histogram when its bin changes; at the
// end of the 8 the warp's lanes that end in the same bin add their runs with
// one atomic.  Grid-stride over the 8-voxel segments.
template <int TYPE, bool VEC>
__global__ void __launch_bounds__(kProfThreads) k_transmural(const void* __restrict__ ha,
                                                             const uint8_t* __restrict__ mask, ProfDev P,
                                                             unsigned long long* __restrict__ hist) {
  extern __shared__ uint32_t sh[];
  const int nb = P.nd * P.nh;
  for (int k = threadIdx.x; k < nb; k += kProfThreads) sh[k] = 0u;
  __syncthreads();
  const int segs_row = (P.n0 + 7) / 8;
  const int64_t nseg = (int64_t)segs_row * P.n1 * P.n2;
  for (int64_t b = (int64_t)blockIdx.x * kProfThreads; b < nseg; b += (int64_t)gridDim.x * kProfThreads) {
    const int64_t s = b + threadIdx.x;
    int cur = -1;
    uint32_t cnt = 0;
    if (s < nseg) {
      const int64_t row = s / segs_row;
      const int x0 = (int)(s - row * segs_row) * 8;
      const int yr = (int)(row % P.n1), zr = (int)(row / P.n1);
      const float dy = (float)(P.lo[1] + yr) - P.c[1], dz = (float)(P.lo[2] + zr) - P.c[2];
      const int64_t i0 = row * P.n0 + x0;
      const int nk = min(8, P.n0 - x0);
      float h[8];
      bool ok[8];
      uint8_t m8[8];
      if (VEC) {  // whole 8-voxel segments on aligned rows
        load8<TYPE>(ha, i0, h, ok);
        if (mask) {
          const uint2 q = __ldg(reinterpret_cast<const uint2*>(mask + i0));
#pragma unroll
          for (int k = 0; k < 8; ++k) m8[k] = ((k < 4 ? q.x : q.y) >> (8 * (k & 3))) & 0xff;
        }
      } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          ok[k] = false;
          h[k] = 0.f;
          m8[k] = 0;
          if (k < nk) {
            h[k] = decode_ha<TYPE>(ha, i0 + k, ok[k]);
            if (mask) m8[k] = __ldg(mask + i0 + k);
          }
        }
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        if (k >= nk) break;
        int bin = -1;
        if (ok[k] && (mask == nullptr || m8[k] != 0)) {
          const float dx = (float)(P.lo[0] + x0 + k) - P.c[0];
          const float t = dx * P.a[0] + dy * P.a[1] + dz * P.a[2];
          const float rx = dx - t * P.a[0], ry = dy - t * P.a[1], rz = dz - t * P.a[2];
          const float d = (sqrtf(rx * rx + ry * ry + rz * rz) - P.r_in) * P.inv_w;
          if (d >= 0.f && d < 1.f) {
            const int kd = min((int)(d * (float)P.nd), P.nd - 1);
            const int kh = min(max((int)((h[k] + 90.f) * ((float)P.nh / 180.f)), 0), P.nh - 1);
            bin = kd * P.nh + kh;
          }
        }
        if (bin == cur) {
          ++cnt;
        } else {
          if (cur >= 0) atomicAdd(&sh[cur], cnt);
          cur = bin;
          cnt = 1;
        }
      }
    }
    // the last runs: lanes ending in the same bin add them with one atomic
    const unsigned same = __match_any_sync(0xffffffffu, cur);
    const uint32_t total = __reduce_add_sync(same, cnt);
    if (cur >= 0 && (int)(threadIdx.x & 31) == __ffs(same) - 1) atomicAdd(&sh[cur], total);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < nb; k += kProfThreads)
    if (sh[k]) atomicAdd(hist + k, (unsigned long long)sh[k]);
}

template <int TYPE>
cudaError_t launch_profile(const void* ha, const uint8_t* mask, const ProfDev& P, unsigned long long* hist, int grid,
                           size_t smem, bool vec, cudaStream_t st) {
  cudaError_t e;
  if (vec) {
    e = cudaFuncSetAttribute(k_transmural<TYPE, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) k_transmural<TYPE, true><<<grid, kProfThreads, smem, st>>>(ha, mask, P, hist);
  } else {
    e = cudaFuncSetAttribute(k_transmural<TYPE, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) k_transmural<TYPE, false><<<grid, kProfThreads, smem, st>>>(ha, mask, P, hist);
  }
  return e == cudaSuccess ? cudaGetLastError() : e;
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
  const int64_t segs = (n[0] + 7) / 8 * n[1] * n[2];
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
  const int64_t want = (int64_t)sms * 4;  // four CTAs of 256 threads per SM
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (segs + kProfThreads - 1) / kProfThreads));
  const size_t smem = sizeof(uint32_t) * (size_t)P.nd * P.nh;
  // vector loads: rows of whole 8-voxel segments on 16-byte aligned arrays
  const bool vec = n[0] % 8 == 0 && (uintptr_t)d_ha % 16 == 0 && (d_mask == nullptr || (uintptr_t)d_mask % 8 == 0);
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  unsigned long long* h = reinterpret_cast<unsigned long long*>(d_hist);
  switch (spec->ha_type) {
    case CT_OUT_F32: e = launch_profile<CT_OUT_F32>(d_ha, d_mask, P, h, grid, smem, vec, st); break;
    case CT_OUT_F16: e = launch_profile<CT_OUT_F16>(d_ha, d_mask, P, h, grid, smem, vec, st); break;
    default: e = launch_profile<CT_OUT_U8Q>(d_ha, d_mask, P, h, grid, smem, vec, st); break;
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return ct::set_error(CT_ERR_CUDA, "profile launch failed: %s", cudaGetErrorString(e));
  return CT_OK;
}
