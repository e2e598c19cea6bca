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
// Tile shape (compile-time tunables): outputs per row, rows per CTA, outputs per thread.
#ifndef CT_RX_OUT
#define CT_RX_OUT 128
#endif
#ifndef CT_RX_ROWS
#define CT_RX_ROWS 4
#endif
#ifndef CT_RX_PER
#define CT_RX_PER 8
#endif
#ifndef CT_RX_MINB
#define CT_RX_MINB 1
#endif
constexpr int kRxOut = CT_RX_OUT;
constexpr int kRxRows = CT_RX_ROWS;
constexpr int kRxPer = CT_RX_PER;
constexpr int kRxThreads = 6 * kRxRows * (kRxOut / kRxPer);

template <int RR>
__global__ void __launch_bounds__(kRxThreads, CT_RX_MINB)
    k_rho_x(const float* __restrict__ in, Box ib, int dimx, float* __restrict__ out, Box ob, const Taps taps) {
  constexpr int W = kRxOut + 2 * RR;  // staged row length (multiple of 4 for even RR)
  static_assert(W % 4 == 0, "row stride must allow 16-byte loads");
  __shared__ __align__(16) float sin_[6][kRxRows][W];
  __shared__ __align__(16) float sout[6][kRxRows][kRxOut];
  __shared__ int64_t rin[kRxRows], rout[kRxRows];  // row offsets (component 0) in the input / output arrays
  __shared__ int rvalid[kRxRows];

  const int t = threadIdx.x;
  const int x0 = ob.lo[0] + blockIdx.y * kRxOut;
  const int nrows = ob.n[1] * ob.n[2];
  const int row0 = blockIdx.x * kRxRows;
  const int64_t nib = box_vox(ib), nob = box_vox(ob);
  if (t < kRxRows) {
    const int r = min(row0 + t, nrows - 1);
    const int y = ob.lo[1] + r % ob.n[1], z = ob.lo[2] + r / ob.n[1];
    rin[t] = box_index(ib, ib.lo[0], y, z);
    rout[t] = box_index(ob, ob.lo[0], y, z);
    rvalid[t] = row0 + t < nrows;
  }
  __syncthreads();

  // stage in 16-byte chunks: q -> (comp, row, 4 columns).  A chunk that lies
  // inside the volume and the input array, on a 16-byte boundary, is one
  // vector load; a chunk that needs clamping takes four scalar loads.
  constexpr int QW = W / 4;
  const int xlo_ok = max(0, ib.lo[0]), xhi_ok = min(dimx, ib.lo[0] + ib.n[0]);  // [xlo_ok, xhi_ok) loadable as is
  for (int q = t; q < 6 * kRxRows * QW; q += kRxThreads) {
    const int cq = q % QW;
    const int row = (q / QW) % kRxRows;
    const int comp = q / (QW * kRxRows);
    const int gx0 = x0 - RR + 4 * cq;
    const float* rowp = in + comp * nib + rin[row] - ib.lo[0];
    float4 v;
    if (gx0 >= xlo_ok && gx0 + 3 < xhi_ok && ((reinterpret_cast<uintptr_t>(rowp + gx0) & 15) == 0)) {
      v = __ldg(reinterpret_cast<const float4*>(rowp + gx0));
    } else {
      v.x = __ldg(rowp + clamp_to(gx0, dimx, ib.lo[0], ib.n[0]));
      v.y = __ldg(rowp + clamp_to(gx0 + 1, dimx, ib.lo[0], ib.n[0]));
      v.z = __ldg(rowp + clamp_to(gx0 + 2, dimx, ib.lo[0], ib.n[0]));
      v.w = __ldg(rowp + clamp_to(gx0 + 3, dimx, ib.lo[0], ib.n[0]));
    }
    *reinterpret_cast<float4*>(&sin_[comp][row][4 * cq]) = v;
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
#pragma unroll
    for (int i = 0; i < kRxPer / 4; ++i) dst[i] = make_float4(acc[4 * i], acc[4 * i + 1], acc[4 * i + 2], acc[4 * i + 3]);
  }
  __syncthreads();
  const int xend = ob.lo[0] + ob.n[0];
  constexpr int QO = kRxOut / 4;
  for (int q = t; q < 6 * kRxRows * QO; q += kRxThreads) {
    const int cq = q % QO;
    const int row = (q / QO) % kRxRows;
    const int comp = q / (QO * kRxRows);
    if (!rvalid[row]) continue;
    const int x = x0 + 4 * cq;
    float* dst = out + comp * nob + rout[row] + (x - ob.lo[0]);
    const float4 v = *reinterpret_cast<const float4*>(&sout[comp][row][4 * cq]);
    if (x + 3 < xend && ((reinterpret_cast<uintptr_t>(dst) & 15) == 0)) {
      *reinterpret_cast<float4*>(dst) = v;
    } else {
      if (x < xend) dst[0] = v.x;
      if (x + 1 < xend) dst[1] = v.y;
      if (x + 2 < xend) dst[2] = v.z;
      if (x + 3 < xend) dst[3] = v.w;
    }
  }
}

// ------------------------------------------------------ y / z streaming pass
// One thread per (x, component, cross-row) column walks the pass axis in
// blocks of kT outputs.  A block's outputs come from a register window of
// kT + 2R inputs; between blocks the window slides by kT (2R register moves
// per kT (2R+1) FMAs), so the code of one block is small and no halo is
// re-read.  Inputs arrive through a per-thread shared-memory ring two blocks
// deep, filled by cp.async one block ahead of use.  Offsets inside one
// component plane are 32-bit (planes are limited to 2^31 voxels).
constexpr int kStreamThreads = 256;


// A CTA spans blockDim.x consecutive x (a multiple of 32) and blockDim.y
// (component, cross-row) pairs, so the accesses of one step form contiguous runs.
#ifndef CT_RZ_CHAINS
#define CT_RZ_CHAINS 2
#endif
#ifndef CT_RZ_MINB
#define CT_RZ_MINB 1
#endif
template <int RR, int kT, typename BLK>
__device__ __forceinline__ void rho_stream_body(const float* __restrict__ in, Box ib, int dim_axis,
                                                float* __restrict__ out, Box ob, int axis, int seg, const Taps taps,
                                                const BLK blk) {
  constexpr int P = 2 * RR + 1;
  constexpr int WN = kT + 2 * RR;
  __shared__ float ring[2 * kT][kStreamThreads];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int other = 3 - axis;  // the non-x cross axis
  const int x = ob.lo[0] + blk.x() * blockDim.x + threadIdx.x;
  const int n_other = other == 1 ? ob.n[1] : ob.n[2];
  const bool cok = blk.y() * blockDim.y + threadIdx.y < 6 * n_other;
  const int cross = min(blk.y() * blockDim.y + threadIdx.y, 6 * n_other - 1);  // (comp, other) pair
  const int comp = cross / n_other;
  const int o = (other == 1 ? ob.lo[1] : ob.lo[2]) + cross % n_other;
  const int a_lo = axis == 1 ? ob.lo[1] : ob.lo[2], a_n = axis == 1 ? ob.n[1] : ob.n[2];
  const int p0 = a_lo + blk.z() * seg;  // first output position on the axis
  const int L = min(seg, a_lo + a_n - p0);
  if (L <= 0) return;
  const bool xok = x < ob.lo[0] + ob.n[0] && cok;
  const int xi = min(x, ob.lo[0] + ob.n[0] - 1);

  // input column: fixed (x, other); element offset of axis position a is (a - alo) * istride
  const int alo = axis == 1 ? ib.lo[1] : ib.lo[2], an = axis == 1 ? ib.n[1] : ib.n[2];
  const int yb = axis == 1 ? ib.lo[1] : o;
  const int zb = axis == 1 ? o : ib.lo[2];
  const float* base = in + comp * box_vox(ib) + box_index(ib, xi, yb, zb);
  const int istride = axis == 1 ? ib.n[0] : ib.n[0] * ib.n[1];
  const int qlo = max(0, alo) - alo, qhi = min(dim_axis - 1, alo + an - 1) - alo;  // clamp range, relative
  const int q0 = p0 - RR - alo;  // relative position of input step 0
  auto src = [&](int step) -> const float* { return base + min(max(q0 + step, qlo), qhi) * istride; };

  const int yo = axis == 1 ? p0 : o;
  const int zo = axis == 1 ? o : p0;
  float* obase = out + comp * box_vox(ob) + box_index(ob, xi, yo, zo);
  const int ostride = axis == 1 ? ob.n[0] : ob.n[0] * ob.n[1];

  const uint32_t ring0 = (uint32_t)__cvta_generic_to_shared(&ring[0][tid]);
  constexpr uint32_t kSlot = kStreamThreads * sizeof(float);

  float win[WN];
#pragma unroll
  for (int j = 0; j < 2 * RR; ++j) win[j] = __ldg(src(j));
  // blocks 0 and 1: steps 2R + t, t < 2 kT, into ring slot t
#pragma unroll
  for (int h = 0; h < 2; ++h) {
#pragma unroll
    for (int t = 0; t < kT; ++t) cp_async4(ring0 + (h * kT + t) * kSlot, src(2 * RR + h * kT + t));
    cp_async_commit();
  }
  const int nb = (L + kT - 1) / kT;
  for (int bk = 0; bk < nb; ++bk) {
    cp_async_wait<1>();  // block bk has landed (block bk + 1 may still be in flight)
    const int half = (bk & 1) * kT;
#pragma unroll
    for (int t = 0; t < kT; ++t) win[2 * RR + t] = ring[half + t][tid];
    const int s0 = bk * kT;
#if CT_RZ_CHAINS == 1
    // one chain per output: the kT outputs of the block are the independent work
#pragma unroll
    for (int i = 0; i < kT; ++i) {
      float a = taps.w[0] * win[i];
#pragma unroll
      for (int k = 1; k < P; ++k) a = fmaf(taps.w[k], win[i + k], a);
      if (xok && s0 + i < L) obase[(s0 + i) * ostride] = a;
    }
#elif CT_RZ_CHAINS == 2
#pragma unroll
    for (int i = 0; i < kT; ++i) {
      float a0 = taps.w[0] * win[i], a1 = taps.w[1] * win[i + 1];
#pragma unroll
      for (int k = 2; k < P; k += 2) {
        a0 = fmaf(taps.w[k], win[i + k], a0);
        if (k + 1 < P) a1 = fmaf(taps.w[k + 1], win[i + k + 1], a1);
      }
      if (xok && s0 + i < L) obase[(s0 + i) * ostride] = a0 + a1;
    }
#else
#pragma unroll
    for (int i = 0; i < kT; ++i) {
      float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll
      for (int k = 0; k < P; k += 4) {
        a0 = fmaf(taps.w[k], win[i + k], a0);
        if (k + 1 < P) a1 = fmaf(taps.w[k + 1], win[i + k + 1], a1);
        if (k + 2 < P) a2 = fmaf(taps.w[k + 2], win[i + k + 2], a2);
        if (k + 3 < P) a3 = fmaf(taps.w[k + 3], win[i + k + 3], a3);
      }
      if (xok && s0 + i < L) obase[(s0 + i) * ostride] = (a0 + a1) + (a2 + a3);
    }
#endif
    // refill the slots just consumed with block bk + 2 (their values are in registers)
#pragma unroll
    for (int t = 0; t < kT; ++t) cp_async4(ring0 + (half + t) * kSlot, src(2 * RR + (bk + 2) * kT + t));
    cp_async_commit();
#pragma unroll
    for (int j = 0; j < 2 * RR; ++j) win[j] = win[j + kT];
  }
  cp_async_wait<0>();
}

template <int RR, int kT>
__global__ void __launch_bounds__(kStreamThreads, CT_RZ_MINB)
    k_rho_stream(const float* __restrict__ in, Box ib, int dim_axis, float* __restrict__ out, Box ob, int axis,
                 int seg, const Taps taps) {
  rho_stream_body<RR, kT>(in, ib, dim_axis, out, ob, axis, seg, taps, HwBlock{});
}

// The z pass over a batch of volumes in one persistent launch (MultiTable).
template <int RR, int kT>
__global__ void __launch_bounds__(kStreamThreads, CT_RZ_MINB)
    k_rho_z_multi(const RzItem* __restrict__ items, const MultiTable T, const Taps taps) {
  for_each_vblock(T, [&](int i, const VBlock& v) {
    const RzItem it = items[i];  // a local copy: the body keeps its fields in registers
    rho_stream_body<RR, kT>(it.in, it.ib, it.dim_axis, it.out, it.ob, 2, it.seg, taps, v);
  });
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

// The walk's segment length (enough CTAs to fill the GPU) and the CTA shape
// (warps along x: the widest that leaves the fewest idle columns).
static int stream_seg(const Box& ob, int axis, int RR) {
  const int other = 3 - axis;
  const int n_axis = ob.n[axis];
  int64_t cols = (int64_t)((ob.n[0] + 31) / 32) * 32 * 6 * ob.n[other];
  int nseg = 1;
  while (nseg < 16 && cols * nseg < (int64_t)152 * 1024 * 8 && n_axis / (nseg * 2) >= 4 * (2 * RR + 1)) nseg *= 2;
  return (n_axis + nseg - 1) / nseg;
}

dim3 rho_stream_block(const Box& ob, int axis) {
  (void)axis;
  int wx = 1;
  for (int w = 2; w <= kStreamThreads / 32; w *= 2) {
    const int span = 32 * w, best = 32 * wx;
    if (32 * (w / 2) >= ob.n[0]) break;  // a narrower CTA already covers the row
    if ((ob.n[0] + span - 1) / span * span <= (ob.n[0] + best - 1) / best * best) wx = w;
  }
  return dim3(32 * wx, kStreamThreads / (32 * wx));
}

template <int RR>
static cudaError_t launch_stream_r(const float* in, const Box& ib, const int dims[3], float* out, const Box& ob,
                                   int axis, const Taps& taps, int block_t, cudaStream_t st) {
  const int other = 3 - axis;
  const int n_axis = ob.n[axis];
  if (box_vox(ib) >= ((int64_t)1 << 31) || box_vox(ob) >= ((int64_t)1 << 31)) return cudaErrorInvalidValue;
  const int seg = stream_seg(ob, axis, RR);
  const dim3 block = rho_stream_block(ob, axis);
  dim3 grid((ob.n[0] + block.x - 1) / block.x, (6 * ob.n[other] + block.y - 1) / block.y, (n_axis + seg - 1) / seg);
  if (grid.y > 65535 || grid.z > 65535) return cudaErrorInvalidValue;
  if (block_t == 8)
    k_rho_stream<RR, 8><<<grid, block, 0, st>>>(in, ib, dims[axis], out, ob, axis, seg, taps);
  else
    k_rho_stream<RR, 16><<<grid, block, 0, st>>>(in, ib, dims[axis], out, ob, axis, seg, taps);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- batches
uint3 rho_z_item(int rk, int block_t, dim3 block, RzItem& it) {
  (void)block_t;
  (void)rk;
  it.seg = it.ob.n[2];  // unsplit: the batch's items fill the GPU, and a segment recomputes its warm-up
  return make_uint3((it.ob.n[0] + block.x - 1) / block.x, (6 * it.ob.n[1] + block.y - 1) / block.y, 1);
}

template <int RR>
static cudaError_t z_multi_r(const RzItem* items, const MultiTable& T, int64_t blocks, dim3 block, const Taps& taps,
                             int block_t, cudaStream_t st) {
  if (block_t == 8) {
    const int grid = persistent_grid(k_rho_z_multi<RR, 8>, kStreamThreads, 0, blocks);
    k_rho_z_multi<RR, 8><<<grid, block, 0, st>>>(items, T, taps);
  } else {
    const int grid = persistent_grid(k_rho_z_multi<RR, 16>, kStreamThreads, 0, blocks);
    k_rho_z_multi<RR, 16><<<grid, block, 0, st>>>(items, T, taps);
  }
  return cudaGetLastError();
}

cudaError_t launch_rho_z_multi(const RzItem* items, const MultiTable& T, int64_t blocks, dim3 block,
                               const Taps& taps, int rk, int block_t, cudaStream_t st) {
  switch (rk) {
    case 4: return z_multi_r<4>(items, T, blocks, block, taps, block_t, st);
    case 6: return z_multi_r<6>(items, T, blocks, block, taps, block_t, st);
    case 8: return z_multi_r<8>(items, T, blocks, block, taps, block_t, st);
    case 12: return z_multi_r<12>(items, T, blocks, block, taps, block_t, st);
    case 16: return z_multi_r<16>(items, T, blocks, block, taps, block_t, st);
    case 24: return z_multi_r<24>(items, T, blocks, block, taps, block_t, st);
    case 32: return z_multi_r<32>(items, T, blocks, block, taps, block_t, st);
    case 36: return z_multi_r<36>(items, T, blocks, block, taps, block_t, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_rho_stream(const float* in, const Box& ib, const int dims[3], float* out, const Box& ob, int axis,
                              const Taps& taps, int rk, int block_t, cudaStream_t st) {
  if (box_vox(ob) == 0) return cudaSuccess;
  if (axis != 1 && axis != 2) return cudaErrorInvalidValue;
  switch (rk) {
    case 4: return launch_stream_r<4>(in, ib, dims, out, ob, axis, taps, block_t, st);
    case 6: return launch_stream_r<6>(in, ib, dims, out, ob, axis, taps, block_t, st);
    case 8: return launch_stream_r<8>(in, ib, dims, out, ob, axis, taps, block_t, st);
    case 12: return launch_stream_r<12>(in, ib, dims, out, ob, axis, taps, block_t, st);
    case 16: return launch_stream_r<16>(in, ib, dims, out, ob, axis, taps, block_t, st);
    case 24: return launch_stream_r<24>(in, ib, dims, out, ob, axis, taps, block_t, st);
    case 32: return launch_stream_r<32>(in, ib, dims, out, ob, axis, taps, block_t, st);
    case 36: return launch_stream_r<36>(in, ib, dims, out, ob, axis, taps, block_t, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ct
