// Streamline tractography through the fibre field (Figure 1(d); Architecture,
// "tractography"): from each seed, classical RK4 through the sign-aligned,
// trilinearly interpolated orientation field, forwards and backwards, with
// the stopping rules stated in include/ct.h.  One thread per track: the
// tracks are independent and their cells are read through the L1/L2 caches.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

#include "ct.h"

namespace ct {
ct_status set_error(ct_status st, const char* fmt, ...);
}

namespace {

struct TrackDev {
  int n[3];
  float h, fa_min, cos_turn;
  int max_steps;
};

struct Cell {
  int64_t i000;  // linear index of the cell's lowest corner
  float t[3];
};

__device__ __forceinline__ bool cell_of(const TrackDev& T, const float q[3], Cell& c) {
  int i[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (!(q[a] >= 0.f && q[a] <= (float)(T.n[a] - 1))) return false;
    i[a] = min((int)floorf(q[a]), T.n[a] - 2);
    c.t[a] = q[a] - (float)i[a];
  }
  c.i000 = ((int64_t)i[2] * T.n[1] + i[1]) * T.n[0] + i[0];
  return true;
}

__device__ __forceinline__ int64_t corner(const TrackDev& T, const Cell& c, int k) {
  return c.i000 + (k & 1) + ((k >> 1) & 1) * (int64_t)T.n[0] + ((k >> 2) & 1) * (int64_t)T.n[0] * T.n[1];
}

__device__ __forceinline__ float weight(const Cell& c, int k) {
  return ((k & 1) ? c.t[0] : 1.f - c.t[0]) * (((k >> 1) & 1) ? c.t[1] : 1.f - c.t[1]) *
         (((k >> 2) & 1) ? c.t[2] : 1.f - c.t[2]);
}

// dir(q; r): the cell's 8 vectors aligned with r, trilinear weights, normalised.
__device__ bool direction(const float* __restrict__ vec, int64_t nv, const TrackDev& T, const float q[3],
                          const float r[3], float o[3]) {
  Cell c;
  if (!cell_of(T, q, c)) return false;
  float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int64_t i = corner(T, c, k);
    float u0 = __ldg(vec + i), u1 = __ldg(vec + nv + i), u2 = __ldg(vec + 2 * nv + i);
    if (!(isfinite(u0) && isfinite(u1) && isfinite(u2))) return false;
    if (u0 * r[0] + u1 * r[1] + u2 * r[2] < 0.f) { u0 = -u0; u1 = -u1; u2 = -u2; }
    const float w = weight(c, k);
    s0 = fmaf(w, u0, s0);
    s1 = fmaf(w, u1, s1);
    s2 = fmaf(w, u2, s2);
  }
  const float n2 = s0 * s0 + s1 * s1 + s2 * s2;
  if (!(n2 > 0.f)) return false;
  const float inv = rsqrtf(n2);
  o[0] = s0 * inv; o[1] = s1 * inv; o[2] = s2 * inv;
  return true;
}

__device__ float trilinear(const float* __restrict__ f, const TrackDev& T, const float q[3]) {
  Cell c;
  if (!cell_of(T, q, c)) return nanf("");
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s = fmaf(weight(c, k), __ldg(f + corner(T, c, k)), s);
  return s;
}

__device__ __forceinline__ int64_t nearest(const TrackDev& T, const float q[3]) {
  const int x = (int)floorf(q[0] + 0.5f), y = (int)floorf(q[1] + 0.5f), z = (int)floorf(q[2] + 0.5f);
  return ((int64_t)z * T.n[1] + y) * T.n[0] + x;
}

__global__ void __launch_bounds__(128) k_track(const float* __restrict__ vec, const float* __restrict__ fa,
                                               const uint8_t* __restrict__ mask, const float* __restrict__ seeds,
                                               int64_t n_seeds, TrackDev T, float* __restrict__ points,
                                               int32_t* __restrict__ count) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= 2 * n_seeds) return;
  const int64_t seed = g >> 1;
  const bool backward = g & 1;
  const int64_t nv = (int64_t)T.n[0] * T.n[1] * T.n[2];
  float* out = points + g * (int64_t)(T.max_steps + 1) * 3;
  float p[3] = {seeds[3 * seed], seeds[3 * seed + 1], seeds[3 * seed + 2]};
#pragma unroll
  for (int a = 0; a < 3; ++a)
    if (!(p[a] >= 0.f && p[a] <= (float)(T.n[a] - 1))) {
      count[g] = 0;
      return;
    }
  out[0] = p[0]; out[1] = p[1]; out[2] = p[2];
  int cnt = 1;
  const int64_t i0 = nearest(T, p);
  float ref[3] = {__ldg(vec + i0), __ldg(vec + nv + i0), __ldg(vec + 2 * nv + i0)};
  float d[3];
  const bool start = isfinite(ref[0]) && isfinite(ref[1]) && isfinite(ref[2]) &&
                     (ref[0] != 0.f || ref[1] != 0.f || ref[2] != 0.f) && direction(vec, nv, T, p, ref, d);
  if (start) {
    if (backward) { d[0] = -d[0]; d[1] = -d[1]; d[2] = -d[2]; }
    const float h = T.h, hh = 0.5f * T.h;
    for (int step = 0; step < T.max_steps; ++step) {
      float k1[3], k2[3], k3[3], k4[3], q[3];
      if (!direction(vec, nv, T, p, d, k1)) break;
#pragma unroll
      for (int a = 0; a < 3; ++a) q[a] = fmaf(hh, k1[a], p[a]);
      if (!direction(vec, nv, T, q, k1, k2)) break;
#pragma unroll
      for (int a = 0; a < 3; ++a) q[a] = fmaf(hh, k2[a], p[a]);
      if (!direction(vec, nv, T, q, k2, k3)) break;
#pragma unroll
      for (int a = 0; a < 3; ++a) q[a] = fmaf(h, k3[a], p[a]);
      if (!direction(vec, nv, T, q, k3, k4)) break;
      float s[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) s[a] = k1[a] + 2.f * k2[a] + 2.f * k3[a] + k4[a];
      const float n2 = s[0] * s[0] + s[1] * s[1] + s[2] * s[2];
      if (!(n2 > 0.f)) break;
      const float inv = rsqrtf(n2);
      const float dn[3] = {s[0] * inv, s[1] * inv, s[2] * inv};
      if (dn[0] * d[0] + dn[1] * d[1] + dn[2] * d[2] < T.cos_turn) break;
#pragma unroll
      for (int a = 0; a < 3; ++a) q[a] = fmaf(h * (1.f / 6.f), s[a], p[a]);
      bool inside = true;
#pragma unroll
      for (int a = 0; a < 3; ++a) inside = inside && q[a] >= 0.f && q[a] <= (float)(T.n[a] - 1);
      if (!inside) break;
      if (mask && __ldg(mask + nearest(T, q)) == 0) break;
      if (fa && !(trilinear(fa, T, q) >= T.fa_min)) break;
      float* o = out + 3 * cnt;
      o[0] = q[0]; o[1] = q[1]; o[2] = q[2];
      ++cnt;
#pragma unroll
      for (int a = 0; a < 3; ++a) { p[a] = q[a]; d[a] = dn[a]; }
    }
  }
  count[g] = cnt;
}

}  // namespace

extern "C" ct_status ct_track(const ct_track_params* params, const int64_t vol_dims[3], const float* d_vec,
                              const float* d_fa, const uint8_t* d_mask, const float* d_seeds, int64_t n_seeds,
                              float* d_points, int32_t* d_count, void* stream) {
  if (!params || !vol_dims || !d_vec || (n_seeds > 0 && (!d_seeds || !d_points || !d_count)))
    return ct::set_error(CT_ERR_INVALID, "NULL argument");
  if (n_seeds < 0 || n_seeds > ((int64_t)1 << 30)) return ct::set_error(CT_ERR_INVALID, "n_seeds out of range");
  for (int a = 0; a < 3; ++a)
    if (vol_dims[a] < 2 || vol_dims[a] > (1 << 24)) return ct::set_error(CT_ERR_INVALID, "every dims must be in [2, 2^24]");
  if (!(params->step > 0.0) || !std::isfinite(params->step)) return ct::set_error(CT_ERR_INVALID, "step must be > 0");
  if (params->max_steps < 1 || params->max_steps > (1 << 20))
    return ct::set_error(CT_ERR_INVALID, "max_steps must be in [1, 2^20]");
  if (!std::isfinite(params->fa_min) || !std::isfinite(params->max_turn_deg))
    return ct::set_error(CT_ERR_INVALID, "fa_min and max_turn_deg must be finite");
  if (params->reserved != 0) return ct::set_error(CT_ERR_INVALID, "reserved must be 0");
  if (n_seeds == 0) return CT_OK;
  TrackDev T;
  for (int a = 0; a < 3; ++a) T.n[a] = (int)vol_dims[a];
  T.h = (float)params->step;
  T.fa_min = (float)params->fa_min;
  T.cos_turn = (float)std::cos(params->max_turn_deg * 3.14159265358979323846 / 180.0);
  T.max_steps = params->max_steps;
  const int64_t tracks = 2 * n_seeds;
  const int64_t grid = (tracks + 127) / 128;
  if (grid > 0x7fffffff) return ct::set_error(CT_ERR_INVALID, "too many seeds");
  k_track<<<(unsigned)grid, 128, 0, (cudaStream_t)stream>>>(d_vec, d_fa, d_mask, d_seeds, n_seeds, T, d_points,
                                                             d_count);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return ct::set_error(CT_ERR_CUDA, "track launch failed: %s", cudaGetErrorString(e));
  return CT_OK;
}
