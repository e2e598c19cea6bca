// Seeded synthetic heart-wall volumes generated on the device.
//
// Large workloads (batches of crops, volumes of tens of gigavoxels streamed
// chunk by chunk) are generated where they are consumed.  This file holds no
// part of the orientation method: it is the device implementation of the
// generator that synth.py implements for the host, from the same definitions,
// so that a box generated here equals the same box generated there:
//   * SplitMix64 (Steele, Lea & Flood 2014) keyed by (seed, stream, counter),
//     53-bit uniforms in (0, 1), Box-Muller normals;
//   * an annulus about a centre and axis, rods along the local helix direction
//     f0 = cos(HA) e_t + sin(HA) e_z (HA linear from r_in to r_out): one stripe
//     family along r, one along a helical phase taken about local origins on a
//     (theta, h) lattice of spacing 2T and blended with smoothstep weights;
//   * optional radial warp by C1 value noise (out-of-plane tilt of the rods);
//   * Gaussian or Poisson-like noise, clamping and round-half-even to uint16.
// The FP64 form is the definition and matches the host generator voxel for
// voxel (up to the last bit of a transcendental).  The FP32 form
// (CT_SYNTH_FP32) evaluates the same construction in FP32, with 24-bit
// uniforms, for inputs of tens of gigavoxels generated inside a timed stream;
// it agrees with the FP64 form to about one intensity unit.
// The lattice values of the IA field that a block row touches are drawn once
// per block into shared memory (same counters, same blend order).
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

#include "ct.h"

namespace ct {
ct_status set_error(ct_status st, const char* fmt, ...);
}

namespace {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;
constexpr double kPi = 3.14159265358979323846;

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z ^= z >> 30;
  z *= 0xBF58476D1CE4E5B9ull;
  z ^= z >> 27;
  z *= 0x94D049BB133111EBull;
  z ^= z >> 31;
  return z;
}

__device__ __forceinline__ double uniform01(uint64_t key, uint64_t counter) {
  uint64_t bits = mix64(key + (counter + 1ull) * kGamma) >> 11;
  return ((double)bits + 0.5) * (1.0 / 9007199254740992.0);
}

// 24-bit uniforms of the same SplitMix64 outputs, for the FP32 form.
__device__ __forceinline__ float uniform01f(uint64_t key, uint64_t counter) {
  uint32_t bits = (uint32_t)(mix64(key + (counter + 1ull) * kGamma) >> 40);
  return ((float)bits + 0.5f) * (1.0f / 16777216.0f);
}

// Arithmetic of the two forms.  FP64 is the definition (the host generator's
// arithmetic); FP32 is a faster approximation of it for large streamed inputs.
template <typename R>
struct M;
template <>
struct M<double> {
  static __device__ __forceinline__ double normal(uint64_t key, uint64_t counter) {
    double u1 = uniform01(key, 2ull * counter);
    double u2 = uniform01(key, 2ull * counter + 1ull);
    return sqrt(-2.0 * log(u1)) * cos(2.0 * kPi * u2);
  }
  // cos(2 pi a / T)
  static __device__ __forceinline__ double cos2pi(double a, double T) { return cos(2.0 * kPi * a / T); }
  static __device__ __forceinline__ double wrap(double d) { return atan2(sin(d), cos(d)); }
  static __device__ __forceinline__ double atan2_(double y, double x) { return atan2(y, x); }
  static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
  static __device__ __forceinline__ double floor_(double x) { return floor(x); }
  static __device__ __forceinline__ double rint_(double x) { return rint(x); }
  static __device__ __forceinline__ void sincos_(double x, double* s, double* c) {
    *s = sin(x);
    *c = cos(x);
  }
};
template <>
struct M<float> {
  static __device__ __forceinline__ float normal(uint64_t key, uint64_t counter) {
    float u1 = uniform01f(key, 2ull * counter);
    float u2 = uniform01f(key, 2ull * counter + 1ull);
    return sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
  }
  static __device__ __forceinline__ float cos2pi(float a, float T) { return cospif(2.0f * a / T); }
  static __device__ __forceinline__ float wrap(float d) { return d - 6.28318530717958647692f * rintf(d * 0.159154943091895335769f); }
  static __device__ __forceinline__ float atan2_(float y, float x) { return atan2f(y, x); }
  static __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
  static __device__ __forceinline__ float floor_(float x) { return floorf(x); }
  static __device__ __forceinline__ float rint_(float x) { return rintf(x); }
  static __device__ __forceinline__ void sincos_(float x, float* s, float* c) { sincosf(x, s, c); }
};

template <typename R>
__device__ __forceinline__ R smootherstep(R t) {
  return t * t * t * (t * (t * R(6) - R(15)) + R(10));
}

struct SynthDev {
  double c[3], a[3], u[3], w[3];
  double r_in, r_out, period, ha_in, ha_out, background, amplitude, noise_level;
  double ia_amp, ia_corr;
  int noise_kind, use_ia;
  double dth;  // angular lattice step
  uint64_t key_noise, key_ia;
  int64_t dims[3];
};

// Lattice values of the IA field that one block row can touch: x columns
// cx0 .. cx0 + ncol - 1 (ncol <= kLatCols), two y and two z lattice rows.
constexpr int kSynthThreads = 128;
constexpr int kLatCols = 36;

__device__ __forceinline__ uint64_t lattice_counter(int64_t ix, int64_t iy, int64_t iz) {
  return (uint64_t)(((iz + 4) * 4096 + (iy + 4)) * 4096 + (ix + 4));
}

template <typename R>
__global__ void __launch_bounds__(kSynthThreads) k_synth(SynthDev S, int64_t lo0, int64_t lo1, int64_t lo2, int n0,
                                                         int n1, int n2, uint16_t* vol, uint8_t* mask) {
  using Mr = M<R>;
  __shared__ R lat[2][2][kLatCols];
  const int64_t row = (int64_t)blockIdx.z * gridDim.y + blockIdx.y;
  if (row >= (int64_t)n1 * n2) return;  // block-uniform
  const int i = blockIdx.x * kSynthThreads + threadIdx.x;
  const bool active = i < n0;
  const int64_t X = lo0 + (active ? i : n0 - 1), Y = lo1 + row % n1, Z = lo2 + row / n1;
  const R x = (R)X, y = (R)Y, z = (R)Z;
  const R cx = (R)S.c[0], cy = (R)S.c[1], cz = (R)S.c[2];
  const R ax = (R)S.a[0], ay = (R)S.a[1], az = (R)S.a[2];
  const R dx = x - cx, dy = y - cy, dz = z - cz;
  const R h = dx * ax + dy * ay + dz * az;
  const R rx = dx - h * ax, ry = dy - h * ay, rz = dz - h * az;
  R r = Mr::sqrt_(rx * rx + ry * ry + rz * rz);
  const bool inside = r >= (R)S.r_in && r <= (R)S.r_out;
  const int64_t o = ((int64_t)(Z - lo2) * n1 + (Y - lo1)) * n0 + i;
  if (!vol) {  // mask only (block-uniform)
    if (active) mask[o] = inside ? 1 : 0;
    return;
  }
  if (S.use_ia) {
    // C1 value noise of N(0,1) lattice values at spacing ia_corr, quintic blend.
    const R L = (R)S.ia_corr;
    const R fx = x / L, fy = y / L, fz = z / L;
    const R flx = Mr::floor_(fx), fly = Mr::floor_(fy), flz = Mr::floor_(fz);
    const R tx = smootherstep(fx - flx), ty = smootherstep(fy - fly), tz = smootherstep(fz - flz);
    // The lattice columns of this block row (same floor as every voxel takes).
    const int64_t xa = lo0 + (int64_t)blockIdx.x * kSynthThreads;
    const int64_t xb = lo0 + min((int64_t)n0, (int64_t)(blockIdx.x + 1) * kSynthThreads) - 1;
    const int64_t cx0 = (int64_t)Mr::floor_((R)xa / L);
    const int ncol = (int)((int64_t)Mr::floor_((R)xb / L) - cx0) + 2;
    const bool table = ncol <= kLatCols;  // block-uniform
    const int64_t iy = (int64_t)fly, iz = (int64_t)flz;
    if (table) {
      for (int e = threadIdx.x; e < 4 * ncol; e += kSynthThreads) {
        const int c = e % ncol, q = e / ncol;
        lat[q >> 1][q & 1][c] = Mr::normal(S.key_ia, lattice_counter(cx0 + c, iy + (q & 1), iz + (q >> 1)));
      }
      __syncthreads();
    }
    const int64_t ix = (int64_t)flx;
    R acc = R(0);
    for (int ddz = 0; ddz < 2; ++ddz) {
      const R wz = ddz ? tz : R(1) - tz;
      for (int ddy = 0; ddy < 2; ++ddy) {
        const R wy = ddy ? ty : R(1) - ty;
        for (int ddx = 0; ddx < 2; ++ddx) {
          const R wx = ddx ? tx : R(1) - tx;
          const R g = table ? lat[ddz][ddy][ix - cx0 + ddx] : Mr::normal(S.key_ia, lattice_counter(ix + ddx, iy + ddy, iz + ddz));
          acc = acc + wx * wy * wz * g;
        }
      }
    }
    const R delta = (R)S.ia_amp * acc;
    r = r - delta > R(0) ? r - delta : R(0);
  }
  if (!active) return;
  const R ux = (R)S.u[0], uy = (R)S.u[1], uz = (R)S.u[2];
  const R wx_ = (R)S.w[0], wy_ = (R)S.w[1], wz_ = (R)S.w[2];
  const R theta = Mr::atan2_(rx * wx_ + ry * wy_ + rz * wz_, rx * ux + ry * uy + rz * uz);
  R t = (r - (R)S.r_in) / ((R)S.r_out - (R)S.r_in);
  t = t < R(0) ? R(0) : (t > R(1) ? R(1) : t);
  const R ha = ((R)S.ha_in + t * ((R)S.ha_out - (R)S.ha_in)) * (R)(kPi / 180.0);
  const R T = (R)S.period, L2 = R(2) * T;
  const R dth = (R)S.dth;
  const R gs = (theta + (R)kPi) / dth;
  const R g0 = Mr::floor_(gs);
  R fs = gs - g0;
  fs = fs * fs * (R(3) - R(2) * fs);
  const R hs = h / L2;
  const R h0 = Mr::floor_(hs);
  R fh = hs - h0;
  fh = fh * fh * (R(3) - R(2) * fh);
  R sha, cha;
  Mr::sincos_(ha, &sha, &cha);
  R helical = R(0);
  for (int ds = 0; ds < 2; ++ds) {
    const R ws = ds ? fs : R(1) - fs;
    const R th_j = (g0 + (R)ds) * dth - (R)kPi;
    const R dtheta = Mr::wrap(theta - th_j);
    for (int dh = 0; dh < 2; ++dh) {
      const R wh = dh ? fh : R(1) - fh;
      const R h_j = (h0 + (R)dh) * L2;
      const R phi2 = cha * (h - h_j) - sha * r * dtheta;
      helical = helical + ws * wh * Mr::cos2pi(phi2, T);
    }
  }
  const R grating = Mr::cos2pi(r, T) + helical;
  const R bg = (R)S.background;
  const R clean = bg + (inside ? R(0.5) * (R)S.amplitude * grating : R(0));
  const uint64_t gidx = ((uint64_t)Z * (uint64_t)S.dims[1] + (uint64_t)Y) * (uint64_t)S.dims[0] + (uint64_t)X;
  const R nrm = Mr::normal(S.key_noise, gidx);
  const R lvl = (R)S.noise_level;
  const R sd = S.noise_kind == 0 ? lvl : lvl * Mr::sqrt_(bg * (clean > R(0) ? clean : R(0)));
  R v = clean + sd * nrm;
  v = v < R(0) ? R(0) : (v > R(65535) ? R(65535) : v);
  vol[o] = (uint16_t)Mr::rint_(v);
  if (mask) mask[o] = inside ? 1 : 0;
}

uint64_t host_mix64(uint64_t z) {
  z ^= z >> 30;
  z *= 0xBF58476D1CE4E5B9ull;
  z ^= z >> 27;
  z *= 0x94D049BB133111EBull;
  z ^= z >> 31;
  return z;
}

}  // namespace

extern "C" ct_status ct_synth_annulus(const ct_synth_spec* spec, const int64_t vol_dims[3], const int64_t lo[3],
                                      const int64_t n[3], uint16_t* d_vol, uint8_t* d_mask, void* stream) {
  if (!spec || !vol_dims || !lo || !n || (!d_vol && !d_mask))
    return ct::set_error(CT_ERR_INVALID, "NULL argument");
  for (int k = 0; k < 3; ++k)
    if (vol_dims[k] < 1 || n[k] < 1 || lo[k] < 0 || lo[k] + n[k] > vol_dims[k])
      return ct::set_error(CT_ERR_INVALID, "box outside the volume");
  if (n[0] > (1 << 30) || n[1] * n[2] > INT32_MAX)
    return ct::set_error(CT_ERR_INVALID, "box too large");
  if (!(spec->r_out > spec->r_in) || (spec->ia_std_deg > 0.0 && !(spec->ia_corr > 0.0)) || !(spec->period > 0.0) || spec->noise_kind < 0 || spec->noise_kind > 1 ||
      (spec->flags & ~CT_SYNTH_FP32) != 0)
    return ct::set_error(CT_ERR_INVALID, "bad annulus spec");
  double an = std::sqrt(spec->axis[0] * spec->axis[0] + spec->axis[1] * spec->axis[1] + spec->axis[2] * spec->axis[2]);
  if (!(an > 0.0)) return ct::set_error(CT_ERR_INVALID, "axis must not be zero");
  SynthDev S;
  for (int k = 0; k < 3; ++k) {
    S.c[k] = spec->center[k];
    S.a[k] = spec->axis[k] / an;
    S.dims[k] = vol_dims[k];
  }
  // plane basis: reference x (or y when the axis is close to x), Gram-Schmidt, w = a x u
  double ref[3] = {1.0, 0.0, 0.0};
  if (!(std::fabs(S.a[0]) < 0.9)) { ref[0] = 0.0; ref[1] = 1.0; }
  double ra = ref[0] * S.a[0] + ref[1] * S.a[1] + ref[2] * S.a[2];
  double u[3] = {ref[0] - ra * S.a[0], ref[1] - ra * S.a[1], ref[2] - ra * S.a[2]};
  double un = std::sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  for (int k = 0; k < 3; ++k) S.u[k] = u[k] / un;
  S.w[0] = S.a[1] * S.u[2] - S.a[2] * S.u[1];
  S.w[1] = S.a[2] * S.u[0] - S.a[0] * S.u[2];
  S.w[2] = S.a[0] * S.u[1] - S.a[1] * S.u[0];
  S.r_in = spec->r_in;
  S.r_out = spec->r_out;
  S.period = spec->period;
  S.ha_in = spec->ha_in_deg;
  S.ha_out = spec->ha_out_deg;
  S.background = spec->background;
  S.amplitude = spec->amplitude;
  S.noise_kind = spec->noise_kind;
  S.noise_level = spec->noise_level;
  S.use_ia = spec->ia_std_deg > 0.0;
  S.ia_corr = spec->ia_corr;
  S.ia_amp = std::tan(spec->ia_std_deg * 3.14159265358979323846 / 180.0) * spec->ia_corr / 1.3;
  const double r_mid = 0.5 * (spec->r_in + spec->r_out);
  const double L2 = 2.0 * spec->period;
  int n_sec = (int)std::nearbyint(2.0 * 3.14159265358979323846 * r_mid / L2);  // half-even, like the host
  if (n_sec < 4) n_sec = 4;
  S.dth = 2.0 * 3.14159265358979323846 / n_sec;
  S.key_noise = host_mix64(spec->seed * 0x632BE59BD9B4E019ull + 1ull * 0x8CB92BA72F3D8DD7ull);
  S.key_ia = host_mix64(spec->seed * 0x632BE59BD9B4E019ull + 7ull * 0x8CB92BA72F3D8DD7ull);
  const int64_t rows = n[1] * n[2];
  const int gy = (int)(rows < 65535 ? rows : 65535);
  dim3 grid((unsigned)((n[0] + kSynthThreads - 1) / kSynthThreads), (unsigned)gy, (unsigned)((rows + gy - 1) / gy));
  if (spec->flags & CT_SYNTH_FP32)
    k_synth<float><<<grid, kSynthThreads, 0, (cudaStream_t)stream>>>(S, lo[0], lo[1], lo[2], (int)n[0], (int)n[1],
                                                                     (int)n[2], d_vol, d_mask);
  else
    k_synth<double><<<grid, kSynthThreads, 0, (cudaStream_t)stream>>>(S, lo[0], lo[1], lo[2], (int)n[0], (int)n[1],
                                                                      (int)n[2], d_vol, d_mask);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return ct::set_error(CT_ERR_CUDA, "generator launch failed: %s", cudaGetErrorString(e));
  return CT_OK;
}
