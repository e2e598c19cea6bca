// The x and y passes of the integration-scale smoothing (Figure 1b) fused in
// one y-streaming kernel, so the x-smoothed field never goes to HBM.
//
// A CTA owns kXT output columns (x) of one (z, component) row and walks y.
// Input rows of the product field arrive kTB at a time through a cp.async
// ring of kStages stages; all threads apply the x pass to those kTB rows
// (each thread kTB consecutive outputs of one row, register-blocked from
// 16-byte shared loads), the results go to shared memory, and each thread
// appends its own column's kTB values to a register window of kTB + 2R rows
// that applies the y pass.  Shared row strides are padded so that the eight
// lanes of a 16-byte access phase hit distinct banks.
#include <cstring>

#include "ct_common.cuh"
#include "ct_launch.h"

namespace ct {

#ifndef CT_XY_TB
#define CT_XY_TB 16
#endif
#ifndef CT_XY_MINB
#define CT_XY_MINB 2
#endif
#ifndef CT_XY_CHAINS
#define CT_XY_CHAINS 2
#endif
constexpr int kStages = 3;      // cp.async ring depth (blocks)
static_assert(CT_XY_TB == 8 || CT_XY_TB == 16, "rows per block");

// XT output columns per CTA (= threads): 256, or 128 for widths that 256
// would cover with a mostly idle last CTA.
template <int RR, int XT>
struct XYGeom {
  // rows per block: 8 for the widest kernels, whose y window would not fit
  // the register budget of 16 warps per SM with 16
  static constexpr int TB = RR >= 32 ? 8 : CT_XY_TB;
  static constexpr int kTB = TB;
  static constexpr int kXT = XT;
  static constexpr int XW = kXT + 2 * RR;                      // staged row width (x pass: 8 per thread)
  static constexpr int XS = XW + ((4 - XW % 8) + 8) % 8;       // padded stride, = 4 (mod 8)
  static constexpr int SXS = kXT + 4;                          // x-pass output row stride
  static constexpr int QW = XW / 4;                            // 16-byte chunks per staged row
  static constexpr int W = (2 * RR + kTB - 1) / kTB;           // warm-up blocks
  static constexpr int PAD = W * kTB - 2 * RR;                 // extra leading rows
  static constexpr int WN = kTB + 2 * RR;                      // y window
};

__device__ __forceinline__ void cp_async16(uint32_t smem_dst, const float* gsrc) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_dst), "l"(gsrc) : "memory");
}

template <int RR, int XT, bool SAMEXY, typename BLK>
__device__ __forceinline__ void rho_xy_body(const float* __restrict__ in, const Box& ib, int dimx, int dimy,
                                            float* __restrict__ out, const Box& ob, int seg, const Taps& tx,
                                            const Taps& ty, const BLK blk) {
  using G = XYGeom<RR, XT>;
  constexpr int kTB = G::TB;
  constexpr int kXT = XT;
  const Taps& TY = SAMEXY ? tx : ty;  // isotropic runs read one tap set
  extern __shared__ __align__(16) float smem[];
  float* stage = smem;                              // [kStages][kTB][XS]
  float* sx = smem + kStages * kTB * G::XS;         // [kTB][SXS]

  const int t = threadIdx.x;
  const int x0 = ob.lo[0] + blk.x() * kXT;
  const int xend = ob.lo[0] + ob.n[0];
  const int comp = blk.y() / ob.n[2];
  const int z = ob.lo[2] + blk.y() % ob.n[2];
  const int p0 = ob.lo[1] + blk.z() * seg;
  const int L = min(seg, ob.lo[1] + ob.n[1] - p0);
  if (L <= 0) return;

  // input rows: row j of the walk is y = p0 - RR - PAD + j, clamped
  const float* plane = in + comp * box_vox(ib) + (int64_t)(z - ib.lo[2]) * ib.n[0] * ib.n[1];
  const int ylo = max(0, ib.lo[1]), yhi = min(dimy - 1, ib.lo[1] + ib.n[1] - 1);
  const int xlo_ok = max(0, ib.lo[0]), xhi_ok = min(dimx, ib.lo[0] + ib.n[0]);
  const int nblocks = G::W + (L + kTB - 1) / kTB;
  const uint32_t stage0 = (uint32_t)__cvta_generic_to_shared(stage);

  // This thread's 16-byte chunks of a staged block: chunk q = t + kXT i is row
  // q / QW, columns 4 (q % QW) .. +3.  Column-dependent parts are fixed for the
  // walk; a chunk is copied by cp.async when it lies inside the input box and
  // rows are 16-byte aligned, else element by element with clamping.
  constexpr int NQ = (kTB * G::QW + kXT - 1) / kXT;
  int q_row[NQ], q_col[NQ];
  bool q_fast[NQ];
  const bool rows_aligned = (ib.n[0] % 4) == 0 && ((reinterpret_cast<uintptr_t>(plane) & 15) == 0);
#pragma unroll
  for (int i = 0; i < NQ; ++i) {
    const int q = t + kXT * i;
    q_row[i] = q < kTB * G::QW ? q / G::QW : -1;
    const int gx0 = x0 - RR + 4 * (q % G::QW);
    q_col[i] = gx0;
    q_fast[i] = rows_aligned && gx0 >= xlo_ok && gx0 + 3 < xhi_ok && ((gx0 - ib.lo[0]) % 4) == 0;
  }
  auto issue = [&](int b) {  // stage block b (kTB rows) into ring slot b % kStages
    const int slot = (b % kStages) * kTB * G::XS;
#pragma unroll
    for (int i = 0; i < NQ; ++i) {
      if (q_row[i] < 0) continue;
      const int rr = q_row[i];
      const int y = min(max(p0 - RR - G::PAD + b * kTB + rr, ylo), yhi);
      const float* row = plane + (y - ib.lo[1]) * ib.n[0] - ib.lo[0];
      const int so = slot + rr * G::XS + (q_col[i] - (x0 - RR));
      if (q_fast[i]) {
        cp_async16(stage0 + (uint32_t)so * 4u, row + q_col[i]);
      } else {
        float* d = stage + so;
        const int gx0 = q_col[i];
        d[0] = __ldg(row + clamp_to(gx0, dimx, ib.lo[0], ib.n[0]));
        d[1] = __ldg(row + clamp_to(gx0 + 1, dimx, ib.lo[0], ib.n[0]));
        d[2] = __ldg(row + clamp_to(gx0 + 2, dimx, ib.lo[0], ib.n[0]));
        d[3] = __ldg(row + clamp_to(gx0 + 3, dimx, ib.lo[0], ib.n[0]));
      }
    }
  };

  // y window of this thread's column
  float win[G::WN];
#pragma unroll
  for (int j = 0; j < G::WN; ++j) win[j] = 0.f;
  // x pass: each thread computes 8 consecutive outputs of one row per 256 outputs;
  // with 16-row blocks it takes two rows (xr and xr + 8)
  const int xr = t % 8;
  const int xseg = t / 8;
  const bool xok = x0 + t < xend;
  float* obase = out + comp * box_vox(ob) + box_index(ob, min(x0 + t, xend - 1), p0, z);
  const int ostride = ob.n[0];

#pragma unroll
  for (int b = 0; b < kStages - 1; ++b) {
    if (b < nblocks) issue(b);
    cp_async_commit();
  }
  for (int b = 0; b < nblocks; ++b) {
    cp_async_wait<kStages - 2>();  // block b has landed (this thread's copies)
    __syncthreads();               // ... and everyone's; slot (b-1) % kStages is free again
    if (b + kStages - 1 < nblocks) issue(b + kStages - 1);
    cp_async_commit();
    // x pass: 8 outputs of row xr (+ 8 r), columns xseg*8 .. +7
#pragma unroll
    for (int r8 = 0; r8 < kTB / 8; ++r8) {
      const int row = xr + 8 * r8;
      const float* src = stage + (b % kStages) * kTB * G::XS + row * G::XS + xseg * 8;
      float acc[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) acc[i] = 0.f;
#pragma unroll
      for (int j4 = 0; j4 < (8 + 2 * RR + 3) / 4; ++j4) {
        const float4 v4 = *reinterpret_cast<const float4*>(src + 4 * j4);
        const float vv[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int j = 4 * j4 + e;  // input index; contributes to outputs i with 0 <= j - i <= 2R
#pragma unroll
          for (int i = 0; i < 8; ++i)
            if (j - i >= 0 && j - i <= 2 * RR) acc[i] = fmaf(tx.w[j - i], vv[e], acc[i]);
        }
      }
      float4* d = reinterpret_cast<float4*>(sx + row * G::SXS + xseg * 8);
      d[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
      d[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
    }
    __syncthreads();  // x-pass rows complete
    // y pass: slide the window by kTB and append this column's new rows
#pragma unroll
    for (int j = 0; j < 2 * RR; ++j) win[j] = win[j + kTB];
#pragma unroll
    for (int r = 0; r < kTB; ++r) win[2 * RR + r] = sx[r * G::SXS + t];
    if (b >= G::W) {
      const int m = (b - G::W) * kTB;  // first output row of this block, relative to p0
#if CT_XY_CHAINS == 1
#pragma unroll
      for (int i = 0; i < kTB; ++i) {
        float a = TY.w[0] * win[i];
#pragma unroll
        for (int k = 1; k <= 2 * RR; ++k) a = fmaf(TY.w[k], win[i + k], a);
        if (xok && m + i < L) obase[(m + i) * ostride] = a;
      }
#elif CT_XY_CHAINS == 2
#pragma unroll
      for (int i = 0; i < kTB; ++i) {
        float a0 = TY.w[0] * win[i], a1 = TY.w[1] * win[i + 1];
#pragma unroll
        for (int k = 2; k <= 2 * RR; k += 2) {
          a0 = fmaf(TY.w[k], win[i + k], a0);
          if (k + 1 <= 2 * RR) a1 = fmaf(TY.w[k + 1], win[i + k + 1], a1);
        }
        if (xok && m + i < L) obase[(m + i) * ostride] = a0 + a1;
      }
#else
#pragma unroll
      for (int i = 0; i < kTB; ++i) {
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll
        for (int k = 0; k <= 2 * RR; k += 4) {
          a0 = fmaf(TY.w[k], win[i + k], a0);
          if (k + 1 <= 2 * RR) a1 = fmaf(TY.w[k + 1], win[i + k + 1], a1);
          if (k + 2 <= 2 * RR) a2 = fmaf(TY.w[k + 2], win[i + k + 2], a2);
          if (k + 3 <= 2 * RR) a3 = fmaf(TY.w[k + 3], win[i + k + 3], a3);
        }
        if (xok && m + i < L) obase[(m + i) * ostride] = (a0 + a1) + (a2 + a3);
      }
#endif
    }
  }
  cp_async_wait<0>();
}

// The single-item kernel keeps its own copy of the body: compiled through the
// body function (taps passed on as copies of the kernel's parameters) it ran
// 19% slower on the uneven crops.
template <int RR, int XT, bool SAMEXY>
__global__ void __launch_bounds__(XT, CT_XY_MINB * 256 / XT)
    k_rho_xy(const float* __restrict__ in, Box ib, int dimx, int dimy, float* __restrict__ out, Box ob, int seg,
             const Taps tx, const Taps ty) {
  using G = XYGeom<RR, XT>;
  constexpr int kTB = G::TB;
  constexpr int kXT = XT;
  const Taps& TY = SAMEXY ? tx : ty;  // isotropic runs read one tap set
  extern __shared__ __align__(16) float smem[];
  float* stage = smem;                              // [kStages][kTB][XS]
  float* sx = smem + kStages * kTB * G::XS;         // [kTB][SXS]

  const int t = threadIdx.x;
  const int x0 = ob.lo[0] + blockIdx.x * kXT;
  const int xend = ob.lo[0] + ob.n[0];
  const int comp = blockIdx.y / ob.n[2];
  const int z = ob.lo[2] + blockIdx.y % ob.n[2];
  const int p0 = ob.lo[1] + blockIdx.z * seg;
  const int L = min(seg, ob.lo[1] + ob.n[1] - p0);
  if (L <= 0) return;

  // input rows: row j of the walk is y = p0 - RR - PAD + j, clamped
  const float* plane = in + comp * box_vox(ib) + (int64_t)(z - ib.lo[2]) * ib.n[0] * ib.n[1];
  const int ylo = max(0, ib.lo[1]), yhi = min(dimy - 1, ib.lo[1] + ib.n[1] - 1);
  const int xlo_ok = max(0, ib.lo[0]), xhi_ok = min(dimx, ib.lo[0] + ib.n[0]);
  const int nblocks = G::W + (L + kTB - 1) / kTB;
  const uint32_t stage0 = (uint32_t)__cvta_generic_to_shared(stage);

  // This thread's 16-byte chunks of a staged block: chunk q = t + kXT i is row
  // q / QW, columns 4 (q % QW) .. +3.  Column-dependent parts are fixed for the
  // walk; a chunk is copied by cp.async when it lies inside the input box and
  // rows are 16-byte aligned, else element by element with clamping.
  constexpr int NQ = (kTB * G::QW + kXT - 1) / kXT;
  int q_row[NQ], q_col[NQ];
  bool q_fast[NQ];
  const bool rows_aligned = (ib.n[0] % 4) == 0 && ((reinterpret_cast<uintptr_t>(plane) & 15) == 0);
#pragma unroll
  for (int i = 0; i < NQ; ++i) {
    const int q = t + kXT * i;
    q_row[i] = q < kTB * G::QW ? q / G::QW : -1;
    const int gx0 = x0 - RR + 4 * (q % G::QW);
    q_col[i] = gx0;
    q_fast[i] = rows_aligned && gx0 >= xlo_ok && gx0 + 3 < xhi_ok && ((gx0 - ib.lo[0]) % 4) == 0;
  }
  auto issue = [&](int b) {  // stage block b (kTB rows) into ring slot b % kStages
    const int slot = (b % kStages) * kTB * G::XS;
#pragma unroll
    for (int i = 0; i < NQ; ++i) {
      if (q_row[i] < 0) continue;
      const int rr = q_row[i];
      const int y = min(max(p0 - RR - G::PAD + b * kTB + rr, ylo), yhi);
      const float* row = plane + (y - ib.lo[1]) * ib.n[0] - ib.lo[0];
      const int so = slot + rr * G::XS + (q_col[i] - (x0 - RR));
      if (q_fast[i]) {
        cp_async16(stage0 + (uint32_t)so * 4u, row + q_col[i]);
      } else {
        float* d = stage + so;
        const int gx0 = q_col[i];
        d[0] = __ldg(row + clamp_to(gx0, dimx, ib.lo[0], ib.n[0]));
        d[1] = __ldg(row + clamp_to(gx0 + 1, dimx, ib.lo[0], ib.n[0]));
        d[2] = __ldg(row + clamp_to(gx0 + 2, dimx, ib.lo[0], ib.n[0]));
        d[3] = __ldg(row + clamp_to(gx0 + 3, dimx, ib.lo[0], ib.n[0]));
      }
    }
  };

  // y window of this thread's column
  float win[G::WN];
#pragma unroll
  for (int j = 0; j < G::WN; ++j) win[j] = 0.f;
  // x pass: each thread computes 8 consecutive outputs of one row per 256 outputs;
  // with 16-row blocks it takes two rows (xr and xr + 8)
  const int xr = t % 8;
  const int xseg = t / 8;
  const bool xok = x0 + t < xend;
  float* obase = out + comp * box_vox(ob) + box_index(ob, min(x0 + t, xend - 1), p0, z);
  const int ostride = ob.n[0];

#pragma unroll
  for (int b = 0; b < kStages - 1; ++b) {
    if (b < nblocks) issue(b);
    cp_async_commit();
  }
  for (int b = 0; b < nblocks; ++b) {
    cp_async_wait<kStages - 2>();  // block b has landed (this thread's copies)
    __syncthreads();               // ... and everyone's; slot (b-1) % kStages is free again
    if (b + kStages - 1 < nblocks) issue(b + kStages - 1);
    cp_async_commit();
    // x pass: 8 outputs of row xr (+ 8 r), columns xseg*8 .. +7
#pragma unroll
    for (int r8 = 0; r8 < kTB / 8; ++r8) {
      const int row = xr + 8 * r8;
      const float* src = stage + (b % kStages) * kTB * G::XS + row * G::XS + xseg * 8;
      float acc[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) acc[i] = 0.f;
#pragma unroll
      for (int j4 = 0; j4 < (8 + 2 * RR + 3) / 4; ++j4) {
        const float4 v4 = *reinterpret_cast<const float4*>(src + 4 * j4);
        const float vv[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int j = 4 * j4 + e;  // input index; contributes to outputs i with 0 <= j - i <= 2R
#pragma unroll
          for (int i = 0; i < 8; ++i)
            if (j - i >= 0 && j - i <= 2 * RR) acc[i] = fmaf(tx.w[j - i], vv[e], acc[i]);
        }
      }
      float4* d = reinterpret_cast<float4*>(sx + row * G::SXS + xseg * 8);
      d[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
      d[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
    }
    __syncthreads();  // x-pass rows complete
    // y pass: slide the window by kTB and append this column's new rows
#pragma unroll
    for (int j = 0; j < 2 * RR; ++j) win[j] = win[j + kTB];
#pragma unroll
    for (int r = 0; r < kTB; ++r) win[2 * RR + r] = sx[r * G::SXS + t];
    if (b >= G::W) {
      const int m = (b - G::W) * kTB;  // first output row of this block, relative to p0
#if CT_XY_CHAINS == 1
#pragma unroll
      for (int i = 0; i < kTB; ++i) {
        float a = TY.w[0] * win[i];
#pragma unroll
        for (int k = 1; k <= 2 * RR; ++k) a = fmaf(TY.w[k], win[i + k], a);
        if (xok && m + i < L) obase[(m + i) * ostride] = a;
      }
#elif CT_XY_CHAINS == 2
#pragma unroll
      for (int i = 0; i < kTB; ++i) {
        float a0 = TY.w[0] * win[i], a1 = TY.w[1] * win[i + 1];
#pragma unroll
        for (int k = 2; k <= 2 * RR; k += 2) {
          a0 = fmaf(TY.w[k], win[i + k], a0);
          if (k + 1 <= 2 * RR) a1 = fmaf(TY.w[k + 1], win[i + k + 1], a1);
        }
        if (xok && m + i < L) obase[(m + i) * ostride] = a0 + a1;
      }
#else
#pragma unroll
      for (int i = 0; i < kTB; ++i) {
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll
        for (int k = 0; k <= 2 * RR; k += 4) {
          a0 = fmaf(TY.w[k], win[i + k], a0);
          if (k + 1 <= 2 * RR) a1 = fmaf(TY.w[k + 1], win[i + k + 1], a1);
          if (k + 2 <= 2 * RR) a2 = fmaf(TY.w[k + 2], win[i + k + 2], a2);
          if (k + 3 <= 2 * RR) a3 = fmaf(TY.w[k + 3], win[i + k + 3], a3);
        }
        if (xok && m + i < L) obase[(m + i) * ostride] = (a0 + a1) + (a2 + a3);
      }
#endif
    }
  }
  cp_async_wait<0>();
}

// The same over a batch of volumes in one persistent launch (MultiTable).
template <int RR, int XT, bool SAMEXY>
__global__ void __launch_bounds__(XT, CT_XY_MINB * 256 / XT)
    k_rho_xy_multi(const RxyItem* __restrict__ items, const MultiTable T, const __grid_constant__ Taps tx,
                   const __grid_constant__ Taps ty) {
  for_each_vblock(T, [&](int i, const VBlock& v) {
    const RxyItem it = items[i];  // a local copy: the body keeps its fields in registers
    rho_xy_body<RR, XT, SAMEXY>(it.in, it.ib, it.dimx, it.dimy, it.out, it.ob, it.seg, tx, ty, v);
  });
}

template <int RR, int XT>
static cudaError_t launch_xy_rt(const float* in, const Box& ib, const int dims[3], float* out, const Box& ob,
                                const Taps& tx, const Taps& ty, cudaStream_t st) {
  using G = XYGeom<RR, XT>;
  constexpr int kTB = G::TB;
  const size_t smem = sizeof(float) * (kStages * kTB * G::XS + kTB * G::SXS);
  const int64_t rows = (int64_t)6 * ob.n[2];
  if (rows > 65535) return cudaErrorInvalidValue;
  const int64_t ctas = (int64_t)((ob.n[0] + XT - 1) / XT) * rows;
  int nseg = 1;
  while (nseg < 16 && ctas * nseg < (int64_t)152 * 2 * 4 * (256 / XT) && ob.n[1] / (nseg * 2) >= 8 * kTB) nseg *= 2;
  const int seg = (ob.n[1] + nseg - 1) / nseg;
  dim3 grid((ob.n[0] + XT - 1) / XT, (unsigned)rows, (ob.n[1] + seg - 1) / seg);
  if (std::memcmp(&tx, &ty, sizeof(Taps)) == 0)
    k_rho_xy<RR, XT, true><<<grid, XT, smem, st>>>(in, ib, dims[0], dims[1], out, ob, seg, tx, ty);
  else
    k_rho_xy<RR, XT, false><<<grid, XT, smem, st>>>(in, ib, dims[0], dims[1], out, ob, seg, tx, ty);
  return cudaGetLastError();
}

// 128-column CTAs when they leave fewer idle columns than 256-column ones.
static bool narrow_xy(int n0) {
  const int w256 = (n0 + 255) / 256 * 256 - n0, w128 = (n0 + 127) / 128 * 128 - n0;
  return w128 < w256;
}

template <int RR>
static cudaError_t launch_xy_r(const float* in, const Box& ib, const int dims[3], float* out, const Box& ob,
                               const Taps& tx, const Taps& ty, cudaStream_t st) {
  if (box_vox(ib) >= ((int64_t)1 << 31) || box_vox(ob) >= ((int64_t)1 << 31)) return cudaErrorInvalidValue;
  return narrow_xy(ob.n[0]) ? launch_xy_rt<RR, 128>(in, ib, dims, out, ob, tx, ty, st)
                            : launch_xy_rt<RR, 256>(in, ib, dims, out, ob, tx, ty, st);
}

template <int RR, int XT>
static cudaError_t prepare_xy_rt() {
  using G = XYGeom<RR, XT>;
  const int smem = (int)(sizeof(float) * (kStages * G::TB * G::XS + G::TB * G::SXS));
  cudaError_t e = cudaFuncSetAttribute(k_rho_xy<RR, XT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_rho_xy<RR, XT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_rho_xy_multi<RR, XT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_rho_xy_multi<RR, XT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  return e;
}

template <int RR>
static cudaError_t prepare_xy_r() {
  cudaError_t e = prepare_xy_rt<RR, 256>();
  if (e == cudaSuccess) e = prepare_xy_rt<RR, 128>();
  return e;
}

cudaError_t prepare_rho_xy_kernels() {
  cudaError_t e = prepare_xy_r<4>();
  if (e == cudaSuccess) e = prepare_xy_r<6>();
  if (e == cudaSuccess) e = prepare_xy_r<8>();
  if (e == cudaSuccess) e = prepare_xy_r<12>();
  if (e == cudaSuccess) e = prepare_xy_r<16>();
  if (e == cudaSuccess) e = prepare_xy_r<24>();
  if (e == cudaSuccess) e = prepare_xy_r<32>();
  if (e == cudaSuccess) e = prepare_xy_r<36>();
  return e;
}

// ---------------------------------------------------------------- batches
int rho_xy_width(int n0) { return narrow_xy(n0) ? 128 : 256; }

// A batch item's walk along y is never split into segments: the batch's items
// fill the GPU, and every segment would recompute its 2R warm-up rows.
template <int RR, int XT>
static uint3 xy_item(RxyItem& it) {
  const Box& ob = it.ob;
  it.seg = ob.n[1];
  return make_uint3((ob.n[0] + XT - 1) / XT, (unsigned)(6 * ob.n[2]), 1);
}

template <int RR>
static uint3 xy_item_r(int xt, RxyItem& it) {
  return xt == 128 ? xy_item<RR, 128>(it) : xy_item<RR, 256>(it);
}

uint3 rho_xy_item(int rk, int xt, RxyItem& it) {
  switch (rk) {
    case 4: return xy_item_r<4>(xt, it);
    case 6: return xy_item_r<6>(xt, it);
    case 8: return xy_item_r<8>(xt, it);
    case 12: return xy_item_r<12>(xt, it);
    case 16: return xy_item_r<16>(xt, it);
    case 24: return xy_item_r<24>(xt, it);
    case 32: return xy_item_r<32>(xt, it);
    default: return xy_item_r<36>(xt, it);
  }
}

template <int RR, int XT>
static cudaError_t xy_multi_t(const RxyItem* items, const MultiTable& T, int64_t blocks, const Taps& tx,
                              const Taps& ty, cudaStream_t st) {
  using G = XYGeom<RR, XT>;
  const size_t smem = sizeof(float) * (kStages * G::TB * G::XS + G::TB * G::SXS);
  if (std::memcmp(&tx, &ty, sizeof(Taps)) == 0) {
    const int grid = persistent_grid(k_rho_xy_multi<RR, XT, true>, XT, smem, blocks);
    k_rho_xy_multi<RR, XT, true><<<grid, XT, smem, st>>>(items, T, tx, ty);
  } else {
    const int grid = persistent_grid(k_rho_xy_multi<RR, XT, false>, XT, smem, blocks);
    k_rho_xy_multi<RR, XT, false><<<grid, XT, smem, st>>>(items, T, tx, ty);
  }
  return cudaGetLastError();
}

template <int RR>
static cudaError_t xy_multi_r(const RxyItem* items, const MultiTable& T, int64_t blocks, const Taps& tx,
                              const Taps& ty, int xt, cudaStream_t st) {
  return xt == 128 ? xy_multi_t<RR, 128>(items, T, blocks, tx, ty, st) : xy_multi_t<RR, 256>(items, T, blocks, tx, ty, st);
}

cudaError_t launch_rho_xy_multi(const RxyItem* items, const MultiTable& T, int64_t blocks, const Taps& tx,
                                const Taps& ty, int rk, int xt, cudaStream_t st) {
  switch (rk) {
    case 4: return xy_multi_r<4>(items, T, blocks, tx, ty, xt, st);
    case 6: return xy_multi_r<6>(items, T, blocks, tx, ty, xt, st);
    case 8: return xy_multi_r<8>(items, T, blocks, tx, ty, xt, st);
    case 12: return xy_multi_r<12>(items, T, blocks, tx, ty, xt, st);
    case 16: return xy_multi_r<16>(items, T, blocks, tx, ty, xt, st);
    case 24: return xy_multi_r<24>(items, T, blocks, tx, ty, xt, st);
    case 32: return xy_multi_r<32>(items, T, blocks, tx, ty, xt, st);
    case 36: return xy_multi_r<36>(items, T, blocks, tx, ty, xt, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_rho_xy(const float* in, const Box& ib, const int dims[3], float* out, const Box& ob,
                          const Taps& tx, const Taps& ty, int rk, cudaStream_t st) {
  if (box_vox(ob) == 0) return cudaSuccess;
  switch (rk) {
    case 4: return launch_xy_r<4>(in, ib, dims, out, ob, tx, ty, st);
    case 6: return launch_xy_r<6>(in, ib, dims, out, ob, tx, ty, st);
    case 8: return launch_xy_r<8>(in, ib, dims, out, ob, tx, ty, st);
    case 12: return launch_xy_r<12>(in, ib, dims, out, ob, tx, ty, st);
    case 16: return launch_xy_r<16>(in, ib, dims, out, ob, tx, ty, st);
    case 24: return launch_xy_r<24>(in, ib, dims, out, ob, tx, ty, st);
    case 32: return launch_xy_r<32>(in, ib, dims, out, ob, tx, ty, st);
    case 36: return launch_xy_r<36>(in, ib, dims, out, ob, tx, ty, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ct
