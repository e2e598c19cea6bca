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
// Everything is FP64, as on the host.
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

__device__ __forceinline__ uint64_t stream_key(uint64_t seed, uint64_t stream) {
  return mix64(seed * 0x632BE59BD9B4E019ull + stream * 0x8CB92BA72F3D8DD7ull);
}

__device__ __forceinline__ double uniform01(uint64_t key, uint64_t counter) {
  uint64_t bits = mix64(key + (counter + 1ull) * kGamma) >> 11;
  return ((double)bits + 0.5) * (1.0 / 9007199254740992.0);
}

__device__ __forceinline__ double normal(uint64_t key, uint64_t counter) {
  double u1 = uniform01(key, 2ull * counter);
  double u2 = uniform01(key, 2ull * counter + 1ull);
  return sqrt(-2.0 * log(u1)) * cos(2.0 * kPi * u2);
}

__device__ __forceinline__ double smootherstep(double t) { return t * t * t * (t * (t * 6.0 - 15.0) + 10.0); }

struct SynthDev {
  double c[3], a[3], u[3], w[3];
  double r_in, r_out, period, ha_in, ha_out, background, amplitude, noise_level;
  double ia_amp, ia_corr;
  int noise_kind, use_ia;
  double dth;  // angular lattice step
  uint64_t key_noise, key_ia;
  int64_t dims[3];
};

__device__ double value_noise(const SynthDev& S, double px, double py, double pz) {
  const double L = S.ia_corr;
  const double fx = px / L, fy = py / L, fz = pz / L;
  const double flx = floor(fx), fly = floor(fy), flz = floor(fz);
  const double tx = smootherstep(fx - flx), ty = smootherstep(fy - fly), tz = smootherstep(fz - flz);
  const int64_t ix = (int64_t)flx + 4, iy = (int64_t)fly + 4, iz = (int64_t)flz + 4;
  double out = 0.0;
  for (int dz = 0; dz < 2; ++dz) {
    const double wz = dz ? tz : 1.0 - tz;
    for (int dy = 0; dy < 2; ++dy) {
      const double wy = dy ? ty : 1.0 - ty;
      for (int dx = 0; dx < 2; ++dx) {
        const double wx = dx ? tx : 1.0 - tx;
        const int64_t idx = ((iz + dz) * 4096 + (iy + dy)) * 4096 + (ix + dx);
        out = out + wx * wy * wz * normal(S.key_ia, (uint64_t)idx);
      }
    }
  }
  return out;
}

__global__ void k_synth(SynthDev S, int64_t lo0, int64_t lo1, int64_t lo2, int n0, int n1, int n2, uint16_t* vol,
                        uint8_t* mask) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n0) return;
  const int row = blockIdx.z * gridDim.y + blockIdx.y;
  if (row >= n1 * n2) return;
  const int64_t X = lo0 + i, Y = lo1 + row % n1, Z = lo2 + row / n1;
  const double x = (double)X, y = (double)Y, z = (double)Z;
  const double dx = x - S.c[0], dy = y - S.c[1], dz = z - S.c[2];
  const double h = dx * S.a[0] + dy * S.a[1] + dz * S.a[2];
  const double rx = dx - h * S.a[0], ry = dy - h * S.a[1], rz = dz - h * S.a[2];
  double r = sqrt(rx * rx + ry * ry + rz * rz);
  const bool inside = r >= S.r_in && r <= S.r_out;
  if (S.use_ia) {
    const double delta = S.ia_amp * value_noise(S, x, y, z);
    r = fmax(r - delta, 0.0);
  }
  const double theta = atan2(rx * S.w[0] + ry * S.w[1] + rz * S.w[2], rx * S.u[0] + ry * S.u[1] + rz * S.u[2]);
  double t = (r - S.r_in) / (S.r_out - S.r_in);
  t = t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t);
  const double ha = (S.ha_in + t * (S.ha_out - S.ha_in)) * (kPi / 180.0);
  const double T = S.period, L2 = 2.0 * T;
  const double gs = (theta + kPi) / S.dth;
  const double g0 = floor(gs);
  double fs = gs - g0;
  fs = fs * fs * (3.0 - 2.0 * fs);
  const double hs = h / L2;
  const double h0 = floor(hs);
  double fh = hs - h0;
  fh = fh * fh * (3.0 - 2.0 * fh);
  const double sha = sin(ha), cha = cos(ha);
  double helical = 0.0;
  for (int ds = 0; ds < 2; ++ds) {
    const double ws = ds ? fs : 1.0 - fs;
    const double th_j = (g0 + ds) * S.dth - kPi;
    const double dd = theta - th_j;
    const double dtheta = atan2(sin(dd), cos(dd));
    for (int dh = 0; dh < 2; ++dh) {
      const double wh = dh ? fh : 1.0 - fh;
      const double h_j = (h0 + dh) * L2;
      const double phi2 = cha * (h - h_j) - sha * r * dtheta;
      helical = helical + ws * wh * cos(2.0 * kPi * phi2 / T);
    }
  }
  const double grating = cos(2.0 * kPi * r / T) + helical;
  const double clean = S.background + (inside ? 0.5 * S.amplitude * grating : 0.0);
  const uint64_t gidx = ((uint64_t)Z * (uint64_t)S.dims[1] + (uint64_t)Y) * (uint64_t)S.dims[0] + (uint64_t)X;
  const double nrm = normal(S.key_noise, gidx);
  const double std = S.noise_kind == 0 ? S.noise_level : S.noise_level * sqrt(S.background * fmax(clean, 0.0));
  double v = clean + std * nrm;
  v = v < 0.0 ? 0.0 : (v > 65535.0 ? 65535.0 : v);
  const int64_t o = ((int64_t)(Z - lo2) * n1 + (Y - lo1)) * n0 + i;
  vol[o] = (uint16_t)rint(v);
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
  if (!spec || !vol_dims || !lo || !n || !d_vol) return ct::set_error(CT_ERR_INVALID, "NULL argument");
  for (int k = 0; k < 3; ++k)
    if (vol_dims[k] < 1 || n[k] < 1 || lo[k] < 0 || lo[k] + n[k] > vol_dims[k])
      return ct::set_error(CT_ERR_INVALID, "box outside the volume");
  if (n[0] > (1 << 30) || n[1] * n[2] > ((int64_t)65535 * 65535))
    return ct::set_error(CT_ERR_INVALID, "box too large");
  if (!(spec->r_out > spec->r_in) || !(spec->period > 0.0) || spec->noise_kind < 0 || spec->noise_kind > 1)
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
  dim3 grid((unsigned)((n[0] + 127) / 128), (unsigned)gy, (unsigned)((rows + gy - 1) / gy));
  k_synth<<<grid, 128, 0, (cudaStream_t)stream>>>(S, lo[0], lo[1], lo[2], (int)n[0], (int)n[1], (int)n[2], d_vol,
                                                    d_mask);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return ct::set_error(CT_ERR_CUDA, "generator launch failed: %s", cudaGetErrorString(e));
  return CT_OK;
}
