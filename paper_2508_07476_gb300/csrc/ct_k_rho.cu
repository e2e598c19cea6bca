// Integration-scale smoothing of the six tensor components (Figure 1b:
// structure tensor), as three separable passes with "nearest" handling of the
// product field at the global volume edges.
//
//  * x pass: a CTA stages 4 haloed rows of all six components in shared
//    memory; each thread computes 8 consecutive outputs of one row from a
//    register window filled by 16-byte shared loads (one load per 28 FMAs at
//    R = 24).  Results leave through shared memory as coalesced stores.
//  * y and z passes: one thread per (column, component) walks the pass axis
//    with a register window of the last 2R+1 inputs plus D prefetched ones;
//    each step costs one coalesced load, 2R+1 FMAs and one coalesced store, and
//    no halo is re-read except at segment starts.
#include "ct_common.cuh"
#include "ct_launch.h"

namespace ct {

int rho_kernel_radius(int r) {
  static const int radii[] = {4, 6, 8, 12, 16, 24, 32, 36};
  for (int v : radii)
    if (r <= v) return v;
  return -1;
}

// ----------------------------------------------------------------- x pass
constexpr int kRxOut = 128;  // outputs per row per CTA
constexpr int kRxRows = 4;   // rows per CTA
constexpr int kRxPer = 8;    // outputs per thread
constexpr int kRxThreads = 6 * kRxRows * (kRxOut / kRxPer);  // 384

template <int RR>
__global__ void __launch_bounds__(kRxThreads)
    k_rho_x(const float* __restrict__ in, Box ib, int dimx, float* __restrict__ out, Box ob, const Taps taps) {
  constexpr int W = kRxOut + 2 * RR;  // staged row length (multiple of 4 for even RR)
  static_assert(W % 4 == 0, "row stride must allow 16-byte loads");
  __shared__ __align__(16) float sin_[6][kRxRows][W];
  __shared__ __align__(16) float sout[6][kRxRows][kRxOut];

  const int t = threadIdx.x;
  const int x0 = ob.lo[0] + blockIdx.y * kRxOut;
  const int nrows = ob.n[1] * ob.n[2];
  const int row0 = blockIdx.x * kRxRows;
  const int64_t nib = box_vox(ib), nob = box_vox(ob);

  // stage: element e -> (comp, row, col)
  for (int e = t; e < 6 * kRxRows * W; e += kRxThreads) {
    const int col = e % W;
    const int row = (e / W) % kRxRows;
    const int comp = e / (W * kRxRows);
    const int r = min(row0 + row, nrows - 1);
    const int y = ob.lo[1] + r % ob.n[1], z = ob.lo[2] + r / ob.n[1];
    const int gx = clamp_to(x0 - RR + col, dimx, ib.lo[0], ib.n[0]);
    sin_[comp][row][col] = __ldg(in + comp * nib + box_index(ib, gx, y, z));
  }
  __syncthreads();
  {
    const int comp = t / (kRxRows * (kRxOut / kRxPer));
    const int row = (t / (kRxOut / kRxPer)) % kRxRows;
    const int seg = t % (kRxOut / kRxPer);
    const float* src = &sin_[comp][row][seg * kRxPer];
    float win[kRxPer + 2 * RR];
#pragma unroll
    for (int j = 0; j < (kRxPer + 2 * RR) / 4; ++j) {
      float4 v = *reinterpret_cast<const float4*>(src + 4 * j);
      win[4 * j] = v.x;
      win[4 * j + 1] = v.y;
      win[4 * j + 2] = v.z;
      win[4 * j + 3] = v.w;
    }
    float acc[kRxPer];
#pragma unroll
    for (int i = 0; i < kRxPer; ++i) {
      float a0 = 0.f, a1 = 0.f;
#pragma unroll
      for (int k = 0; k <= 2 * RR; k += 2) a0 = fmaf(taps.w[k], win[i + k], a0);
#pragma unroll
      for (int k = 1; k <= 2 * RR; k += 2) a1 = fmaf(taps.w[k], win[i + k], a1);
      acc[i] = a0 + a1;
    }
    float4* dst = reinterpret_cast<float4*>(&sout[comp][row][seg * kRxPer]);
    dst[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
    dst[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
  }
  __syncthreads();
  for (int e = t; e < 6 * kRxRows * kRxOut; e += kRxThreads) {
    const int col = e % kRxOut;
    const int row = (e / kRxOut) % kRxRows;
    const int comp = e / (kRxOut * kRxRows);
    const int r = row0 + row;
    const int x = x0 + col;
    if (r < nrows && x < ob.lo[0] + ob.n[0]) {
      const int y = ob.lo[1] + r % ob.n[1], z = ob.lo[2] + r / ob.n[1];
      out[comp * nob + box_index(ob, x, y, z)] = sout[comp][row][col];
    }
  }
}

// ------------------------------------------------------ y / z streaming pass
constexpr int kStreamD = 4;  // prefetch distance (steps)

template <int RR>
__global__ void __launch_bounds__(256)
    k_rho_stream(const float* __restrict__ in, Box ib, int dim_axis, float* __restrict__ out, Box ob, int axis,
                 int seg, const Taps taps) {
  constexpr int P = 2 * RR + 1;
  constexpr int Q = P + kStreamD;
  const int other = 3 - axis;  // the non-x cross axis
  const int x = ob.lo[0] + blockIdx.x * 32 + threadIdx.x;
  const int cross = blockIdx.y * blockDim.y + threadIdx.y;  // (comp, other) pair
  const int n_other = ob.n[other];
  if (cross >= 6 * n_other) return;
  const int comp = cross / n_other;
  const int o = ob.lo[other] + cross % n_other;
  const int p0 = ob.lo[axis] + blockIdx.z * seg;  // first output position on the axis
  const int L = min(seg, ob.lo[axis] + ob.n[axis] - p0);
  if (L <= 0) return;
  const bool xok = x < ob.lo[0] + ob.n[0];
  const int xi = xok ? x : ob.lo[0] + ob.n[0] - 1;

  // input: fixed (x, other), varying axis coordinate
  const int64_t nib = box_vox(ib);
  int ci[3];
  ci[0] = xi;
  ci[other] = o;
  ci[axis] = ib.lo[axis];
  const float* base = in + comp * nib + box_index(ib, ci[0], ci[1], ci[2]);
  const int64_t istride = axis == 1 ? (int64_t)ib.n[0] : (int64_t)ib.n[0] * ib.n[1];
  const int alo = ib.lo[axis], an = ib.n[axis];
  auto ld = [&](int step) -> float {  // input step j <-> position p0 - RR + j
    int p = clamp_to(p0 - RR + step, dim_axis, alo, an);
    return __ldg(base + (int64_t)(p - alo) * istride);
  };

  const int64_t nob = box_vox(ob);
  int co[3];
  co[0] = xi;
  co[other] = o;
  co[axis] = p0;
  float* obase = out + comp * nob + box_index(ob, co[0], co[1], co[2]);
  const int64_t ostride = axis == 1 ? (int64_t)ob.n[0] : (int64_t)ob.n[0] * ob.n[1];

  float win[Q];
#pragma unroll
  for (int j = 0; j < Q - 1; ++j) win[j] = ld(j);
  win[Q - 1] = 0.f;

  for (int b = 0; b < L; b += Q) {
#pragma unroll
    for (int u = 0; u < Q; ++u) {
      const int s = b + u;
      if (s >= L) break;
      win[(u + Q - 1) % Q] = ld(s + Q - 1);
      float a0 = 0.f, a1 = 0.f;
#pragma unroll
      for (int k = 0; k < P; k += 2) a0 = fmaf(taps.w[k], win[(u + k) % Q], a0);
#pragma unroll
      for (int k = 1; k < P; k += 2) a1 = fmaf(taps.w[k], win[(u + k) % Q], a1);
      if (xok) obase[(int64_t)s * ostride] = a0 + a1;
    }
  }
}

template <int RR>
static cudaError_t launch_rho_x_r(const float* in, const Box& ib, const int dims[3], float* out, const Box& ob,
                                  const Taps& taps, cudaStream_t st) {
  dim3 grid((ob.n[1] * ob.n[2] + kRxRows - 1) / kRxRows, (ob.n[0] + kRxOut - 1) / kRxOut);
  k_rho_x<RR><<<grid, kRxThreads, 0, st>>>(in, ib, dims[0], out, ob, taps);
  return cudaGetLastError();
}

cudaError_t launch_rho_x(const float* in, const Box& ib, const int dims[3], float* out, const Box& ob,
                         const Taps& taps, int rk, cudaStream_t st) {
  if (box_vox(ob) == 0) return cudaSuccess;
  if ((ob.n[0] + kRxOut - 1) / kRxOut > 65535) return cudaErrorInvalidValue;
  switch (rk) {
    case 4: return launch_rho_x_r<4>(in, ib, dims, out, ob, taps, st);
    case 6: return launch_rho_x_r<6>(in, ib, dims, out, ob, taps, st);
    case 8: return launch_rho_x_r<8>(in, ib, dims, out, ob, taps, st);
    case 12: return launch_rho_x_r<12>(in, ib, dims, out, ob, taps, st);
    case 16: return launch_rho_x_r<16>(in, ib, dims, out, ob, taps, st);
    case 24: return launch_rho_x_r<24>(in, ib, dims, out, ob, taps, st);
    case 32: return launch_rho_x_r<32>(in, ib, dims, out, ob, taps, st);
    case 36: return launch_rho_x_r<36>(in, ib, dims, out, ob, taps, st);
    default: return cudaErrorInvalidValue;
  }
}

template <int RR>
static cudaError_t launch_stream_r(const float* in, const Box& ib, const int dims[3], float* out, const Box& ob,
                                   int axis, const Taps& taps, cudaStream_t st) {
  const int other = 3 - axis;
  const int n_axis = ob.n[axis];
  // segment the walk so that the grid has enough CTAs to fill the GPU
  int64_t cols = (int64_t)((ob.n[0] + 31) / 32) * 32 * 6 * ob.n[other];
  int nseg = 1;
  while (nseg < 16 && cols * nseg < (int64_t)152 * 2048 * 4 && n_axis / (nseg * 2) >= 4 * (2 * RR + 1)) nseg *= 2;
  int seg = (n_axis + nseg - 1) / nseg;
  dim3 block(32, 8);
  dim3 grid((ob.n[0] + 31) / 32, (6 * ob.n[other] + 7) / 8, (n_axis + seg - 1) / seg);
  if (grid.y > 65535 || grid.z > 65535) return cudaErrorInvalidValue;
  k_rho_stream<RR><<<grid, block, 0, st>>>(in, ib, dims[axis], out, ob, axis, seg, taps);
  return cudaGetLastError();
}

cudaError_t launch_rho_stream(const float* in, const Box& ib, const int dims[3], float* out, const Box& ob, int axis,
                              const Taps& taps, int rk, cudaStream_t st) {
  if (box_vox(ob) == 0) return cudaSuccess;
  if (axis != 1 && axis != 2) return cudaErrorInvalidValue;
  switch (rk) {
    case 4: return launch_stream_r<4>(in, ib, dims, out, ob, axis, taps, st);
    case 6: return launch_stream_r<6>(in, ib, dims, out, ob, axis, taps, st);
    case 8: return launch_stream_r<8>(in, ib, dims, out, ob, axis, taps, st);
    case 12: return launch_stream_r<12>(in, ib, dims, out, ob, axis, taps, st);
    case 16: return launch_stream_r<16>(in, ib, dims, out, ob, axis, taps, st);
    case 24: return launch_stream_r<24>(in, ib, dims, out, ob, axis, taps, st);
    case 32: return launch_stream_r<32>(in, ib, dims, out, ob, axis, taps, st);
    case 36: return launch_stream_r<36>(in, ib, dims, out, ob, axis, taps, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ct
