// Gradient at noise scale sigma and the six tensor products (Figure 1b;
// Architecture, "orientation") as two streaming kernels:
//
//   k_grad_xy  the x and y passes of the three gradient components, per
//              z-plane: F0 = w_y c_x I, F1 = c_y w_x I, F2 = w_y w_x I;
//   k_grad_z   the z pass (g_x = w_z F0, g_y = w_z F1, g_z = c_z F2), the
//              FP16 rounding of the mixed form and the six products g_a g_b.
//
// Both walk an axis with per-thread register windows (y in the first, z in
// the second), so neither computes the halo rows of a 2-D tile.  The three
// partial fields cross HBM once (12 B written and read per voxel); the
// gradient itself never does.
//
// Every pass folds the +k / -k taps (sums for the smoothing taps w,
// differences for the derivative taps c), so a constant volume gives an
// exactly zero gradient.
#include "ct_common.cuh"
#include "ct_launch.h"

namespace ct {

// ---------------------------------------------------------------- x and y
// The arithmetic runs on FP32 pairs (packed add / fma: one instruction, two
// lanes, each rounded as the scalar operation would be):
//   x pass  the staged rows hold every voxel twice, (v, v), so that one packed
//           fma forms (v[m+k] - v[m-k], v[m+k] + v[m-k]) and another adds tap k
//           of both filters to the pair (c_x I, w_x I) of an output;
//   y pass  the window holds those pairs, so that the two smoothing outputs
//           (w_y c_x I, w_y w_x I) share one packed add and one packed fma per
//           tap; the derivative output (c_y w_x I) stays scalar.
// Every output takes the same operations in the same order as the scalar
// form, so its value is the same to the bit.
#ifndef CT_GXY_TB
#define CT_GXY_TB 0  // rows per block, 0: by radius (tuning choice)
#endif
#ifndef CT_GXY_XH
#define CT_GXY_XH 0  // x-pass outputs per sub-pass, 0: by radius (tuning choice)
#endif
template <int RS, int XT>
struct GXYGeom {
  static constexpr int TB = CT_GXY_TB > 0 ? CT_GXY_TB : RS <= 8 ? 16 : 8;  // rows per block (window registers)
  static constexpr int XA = (RS + 7) / 8 * 8;              // staged columns left of the first output
  static constexpr int CW = XT + 2 * XA;                   // staged row width in voxels (a multiple of 8)
  static constexpr int QW = CW / 8;                        // 8-voxel chunks per staged row
  static constexpr int NQ = (TB * QW + XT - 1) / XT;       // chunks per thread per block
  static constexpr int XS = 2 * CW + 4;                    // staged row stride (floats, each voxel twice), = 4 (mod 8)
  static constexpr int SXS = 2 * XT + 4;                   // x-pass output row stride (floats, (c, w) pairs)
  static constexpr int W = (2 * RS + TB - 1) / TB;         // warm-up blocks
  static constexpr int PAD = W * TB - 2 * RS;              // extra leading rows
  static constexpr int WN = TB + 2 * RS;                   // y window
  static constexpr int OFF = XA - RS;                      // first needed staged column of output 0
  static constexpr int XH = CT_GXY_XH > 0 ? CT_GXY_XH : RS <= 6 ? 8 : 4;  // x-pass outputs per sub-pass (registers)
  static constexpr int B2 = OFF / 2 * 2, O2 = OFF % 2;     // 16-byte aligned start (2 voxels), remainder
  static constexpr int NV = (XH + 2 * RS + O2 + 1) / 2;    // float4 loads (2 voxel pairs each) per sub-pass
  static constexpr size_t SMEM = sizeof(float) * (TB * XS + TB * SXS);
};

// 8 uint16 (one 16-byte chunk) -> 8 floats, exact.
__device__ __forceinline__ void u16x8_to_f32(const uint4 q, float* f) {
  const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    f[2 * k] = (float)(w[k] & 0xffffu);
    f[2 * k + 1] = (float)(w[k] >> 16);
  }
}

template <int RS, int XT, typename BLK>
__device__ __forceinline__ void grad_xy_body(const uint16_t* __restrict__ vol, const Box& vb, int dimx, int dimy,
                                             float* __restrict__ F, const Box& ab, int seg, const Taps& tx,
                                             const Taps& ty, const BLK blk) {
  using G = GXYGeom<RS, XT>;
  constexpr int TB = G::TB;
  extern __shared__ __align__(16) float gsm[];
  float* stage = gsm;                  // [TB][XS] staged rows, (v, v) per voxel
  float* sx = gsm + TB * G::XS;        // [TB][SXS] x-pass rows, (c_x I, w_x I) per voxel
  const int t = threadIdx.x;
  const int x0 = ab.lo[0] + blk.x() * XT;
  const int xend = ab.lo[0] + ab.n[0];
  const int z = ab.lo[2] + blk.y();
  const int p0 = ab.lo[1] + blk.z() * seg;
  const int L = min(seg, ab.lo[1] + ab.n[1] - p0);
  if (L <= 0) return;
  const uint16_t* plane = vol + (int64_t)(z - vb.lo[2]) * vb.n[0] * vb.n[1];
  const int ylo = max(0, vb.lo[1]), yhi = min(dimy - 1, vb.lo[1] + vb.n[1] - 1);
  const int xlo_ok = max(0, vb.lo[0]), xhi_ok = min(dimx, vb.lo[0] + vb.n[0]);
  const int nblocks = G::W + (L + TB - 1) / TB;
  const bool aligned = (vb.n[0] % 8) == 0 && ((reinterpret_cast<uintptr_t>(vol) & 15) == 0);
  // this thread's 16-byte chunks of a block: chunk q = t + XT i is row q % TB,
  // columns x0 - XA + 8 (q / TB) .. +7 (the 8 lanes of a shared-memory phase
  // then write 8 different rows); loaded whole when inside the box and
  // aligned, else element by element with clamping
  int q_row[G::NQ], q_col[G::NQ];
  bool q_fast[G::NQ];
#pragma unroll
  for (int i = 0; i < G::NQ; ++i) {
    const int q = t + XT * i;
    q_row[i] = q < TB * G::QW ? q % TB : -1;
    q_col[i] = x0 - G::XA + 8 * (q / TB);
    q_fast[i] = aligned && q_col[i] >= xlo_ok && q_col[i] + 7 < xhi_ok && ((q_col[i] - vb.lo[0]) % 8) == 0;
  }
  uint4 pre[G::NQ];
  auto load_block = [&](int b) {  // block b's chunks into registers
#pragma unroll
    for (int i = 0; i < G::NQ; ++i) {
      if (q_row[i] < 0) continue;
      const int y = min(max(p0 - RS - G::PAD + b * TB + q_row[i], ylo), yhi);
      const uint16_t* row = plane + (int64_t)(y - vb.lo[1]) * vb.n[0] - vb.lo[0];
      if (q_fast[i]) {
        pre[i] = __ldg(reinterpret_cast<const uint4*>(row + q_col[i]));
      } else {
        uint32_t h[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) h[e] = __ldg(row + clamp_to(q_col[i] + e, dimx, vb.lo[0], vb.n[0]));
        pre[i] = make_uint4(h[0] | (h[1] << 16), h[2] | (h[3] << 16), h[4] | (h[5] << 16), h[6] | (h[7] << 16));
      }
    }
  };
  auto store_block = [&]() {  // registers -> staged rows, every voxel twice
#pragma unroll
    for (int i = 0; i < G::NQ; ++i) {
      if (q_row[i] < 0) continue;
      float f[8];
      u16x8_to_f32(pre[i], f);
      float4* d = reinterpret_cast<float4*>(stage + q_row[i] * G::XS + 2 * (q_col[i] - (x0 - G::XA)));
#pragma unroll
      for (int e = 0; e < 4; ++e) d[e] = make_float4(f[2 * e], f[2 * e], f[2 * e + 1], f[2 * e + 1]);
    }
  };
  // y window of this thread's column: (c_x I, w_x I) rows
  float2 wp[G::WN];
#pragma unroll
  for (int j = 0; j < G::WN; ++j) wp[j] = make_float2(0.f, 0.f);
  const int xr = t % 8;
  const int xseg = t / 8;
  const bool xok = x0 + t < xend;
  const int64_t nab = box_vox(ab);
  float* obase = F + box_index(ab, min(x0 + t, xend - 1), p0, z);
  const int ostride = ab.n[0];
  const float2 cw0 = make_float2(0.f, tx.w[RS]);  // centre tap of (c_x, w_x)
  const float2 sgn = make_float2(-1.f, 1.f);
  const float2 wy0 = make_float2(ty.w[RS], ty.w[RS]);
  load_block(0);
  for (int b = 0; b < nblocks; ++b) {
    store_block();                           // the staged rows were last read before the previous barrier
    if (b + 1 < nblocks) load_block(b + 1);  // in flight during this block's passes
    __syncthreads();                         // staged rows complete; x-pass rows free
    // x pass: 8 outputs of row xr (+ 8 r), columns xseg*8 .. +7, in sub-passes of XH
#pragma unroll
    for (int r8 = 0; r8 < TB / 8; ++r8) {
      const int row = xr + 8 * r8;
#pragma unroll
      for (int h = 0; h < 8; h += G::XH) {
        const float* src = stage + row * G::XS + 2 * (8 * xseg + h + G::B2);
        float2 d[2 * G::NV];  // (v, v) of voxels B2 + h + j
#pragma unroll
        for (int j4 = 0; j4 < G::NV; ++j4) {
          const float4 q = *reinterpret_cast<const float4*>(src + 4 * j4);
          d[2 * j4] = make_float2(q.x, q.y);
          d[2 * j4 + 1] = make_float2(q.z, q.w);
        }
        float2 acc[G::XH];  // (c_x I, w_x I)
#pragma unroll
        for (int i = 0; i < G::XH; ++i) {
          const int m = G::O2 + i + RS;  // centre of output h + i in d
          acc[i] = __fmul2_rn(cw0, d[m]);
#pragma unroll
          for (int k = 1; k <= RS; ++k) {
            const float2 dk = __ffma2_rn(d[m - k], sgn, d[m + k]);  // (v+ - v-, v+ + v-)
            acc[i] = __ffma2_rn(make_float2(tx.c[RS + k], tx.w[RS + k]), dk, acc[i]);
          }
        }
        float4* o = reinterpret_cast<float4*>(sx + row * G::SXS + 2 * (8 * xseg + h));
#pragma unroll
        for (int i = 0; i < G::XH; i += 2) o[i / 2] = make_float4(acc[i].x, acc[i].y, acc[i + 1].x, acc[i + 1].y);
      }
    }
    __syncthreads();  // x-pass rows complete
    // y pass: slide the window by TB, append this column's rows
#pragma unroll
    for (int j = 0; j < 2 * RS; ++j) wp[j] = wp[j + TB];
#pragma unroll
    for (int r = 0; r < TB; ++r) wp[2 * RS + r] = *reinterpret_cast<const float2*>(sx + r * G::SXS + 2 * t);
    if (b >= G::W) {
      const int m0 = (b - G::W) * TB;  // first output row of this block, relative to p0
#pragma unroll
      for (int i = 0; i < TB; ++i) {
        const int m = i + RS;
        float2 f02 = __fmul2_rn(wy0, wp[m]);  // (w_y c_x I, w_y w_x I)
        float f1 = 0.f;
#pragma unroll
        for (int k = 1; k <= RS; ++k) {
          f02 = __ffma2_rn(make_float2(ty.w[RS + k], ty.w[RS + k]), __fadd2_rn(wp[m + k], wp[m - k]), f02);
          f1 = fmaf(ty.c[RS + k], wp[m + k].y - wp[m - k].y, f1);
        }
        if (xok && m0 + i < L) {
          float* o = obase + (int64_t)(m0 + i) * ostride;
          o[0] = f02.x;
          o[nab] = f1;
          o[2 * nab] = f02.y;
        }
      }
    }
  }
}

// The single-item kernel keeps its own copy of the body (through the body
// function it ran 6% slower).
template <int RS, int XT>
__global__ void __launch_bounds__(XT, 512 / XT)
    k_grad_xy(const uint16_t* __restrict__ vol, Box vb, int dimx, int dimy, float* __restrict__ F, Box ab, int seg,
              const Taps tx, const Taps ty) {
  using G = GXYGeom<RS, XT>;
  constexpr int TB = G::TB;
  extern __shared__ __align__(16) float gsm[];
  float* stage = gsm;                  // [TB][XS] staged rows, (v, v) per voxel
  float* sx = gsm + TB * G::XS;        // [TB][SXS] x-pass rows, (c_x I, w_x I) per voxel
  const int t = threadIdx.x;
  const int x0 = ab.lo[0] + blockIdx.x * XT;
  const int xend = ab.lo[0] + ab.n[0];
  const int z = ab.lo[2] + blockIdx.y;
  const int p0 = ab.lo[1] + blockIdx.z * seg;
  const int L = min(seg, ab.lo[1] + ab.n[1] - p0);
  if (L <= 0) return;
  const uint16_t* plane = vol + (int64_t)(z - vb.lo[2]) * vb.n[0] * vb.n[1];
  const int ylo = max(0, vb.lo[1]), yhi = min(dimy - 1, vb.lo[1] + vb.n[1] - 1);
  const int xlo_ok = max(0, vb.lo[0]), xhi_ok = min(dimx, vb.lo[0] + vb.n[0]);
  const int nblocks = G::W + (L + TB - 1) / TB;
  const bool aligned = (vb.n[0] % 8) == 0 && ((reinterpret_cast<uintptr_t>(vol) & 15) == 0);
  // this thread's 16-byte chunks of a block: chunk q = t + XT i is row q % TB,
  // columns x0 - XA + 8 (q / TB) .. +7 (the 8 lanes of a shared-memory phase
  // then write 8 different rows); loaded whole when inside the box and
  // aligned, else element by element with clamping
  int q_row[G::NQ], q_col[G::NQ];
  bool q_fast[G::NQ];
#pragma unroll
  for (int i = 0; i < G::NQ; ++i) {
    const int q = t + XT * i;
    q_row[i] = q < TB * G::QW ? q % TB : -1;
    q_col[i] = x0 - G::XA + 8 * (q / TB);
    q_fast[i] = aligned && q_col[i] >= xlo_ok && q_col[i] + 7 < xhi_ok && ((q_col[i] - vb.lo[0]) % 8) == 0;
  }
  uint4 pre[G::NQ];
  auto load_block = [&](int b) {  // block b's chunks into registers
#pragma unroll
    for (int i = 0; i < G::NQ; ++i) {
      if (q_row[i] < 0) continue;
      const int y = min(max(p0 - RS - G::PAD + b * TB + q_row[i], ylo), yhi);
      const uint16_t* row = plane + (int64_t)(y - vb.lo[1]) * vb.n[0] - vb.lo[0];
      if (q_fast[i]) {
        pre[i] = __ldg(reinterpret_cast<const uint4*>(row + q_col[i]));
      } else {
        uint32_t h[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) h[e] = __ldg(row + clamp_to(q_col[i] + e, dimx, vb.lo[0], vb.n[0]));
        pre[i] = make_uint4(h[0] | (h[1] << 16), h[2] | (h[3] << 16), h[4] | (h[5] << 16), h[6] | (h[7] << 16));
      }
    }
  };
  auto store_block = [&]() {  // registers -> staged rows, every voxel twice
#pragma unroll
    for (int i = 0; i < G::NQ; ++i) {
      if (q_row[i] < 0) continue;
      float f[8];
      u16x8_to_f32(pre[i], f);
      float4* d = reinterpret_cast<float4*>(stage + q_row[i] * G::XS + 2 * (q_col[i] - (x0 - G::XA)));
#pragma unroll
      for (int e = 0; e < 4; ++e) d[e] = make_float4(f[2 * e], f[2 * e], f[2 * e + 1], f[2 * e + 1]);
    }
  };
  // y window of this thread's column: (c_x I, w_x I) rows
  float2 wp[G::WN];
#pragma unroll
  for (int j = 0; j < G::WN; ++j) wp[j] = make_float2(0.f, 0.f);
  const int xr = t % 8;
  const int xseg = t / 8;
  const bool xok = x0 + t < xend;
  const int64_t nab = box_vox(ab);
  float* obase = F + box_index(ab, min(x0 + t, xend - 1), p0, z);
  const int ostride = ab.n[0];
  const float2 cw0 = make_float2(0.f, tx.w[RS]);  // centre tap of (c_x, w_x)
  const float2 sgn = make_float2(-1.f, 1.f);
  const float2 wy0 = make_float2(ty.w[RS], ty.w[RS]);
  load_block(0);
  for (int b = 0; b < nblocks; ++b) {
    store_block();                           // the staged rows were last read before the previous barrier
    if (b + 1 < nblocks) load_block(b + 1);  // in flight during this block's passes
    __syncthreads();                         // staged rows complete; x-pass rows free
    // x pass: 8 outputs of row xr (+ 8 r), columns xseg*8 .. +7, in sub-passes of XH
#pragma unroll
    for (int r8 = 0; r8 < TB / 8; ++r8) {
      const int row = xr + 8 * r8;
#pragma unroll
      for (int h = 0; h < 8; h += G::XH) {
        const float* src = stage + row * G::XS + 2 * (8 * xseg + h + G::B2);
        float2 d[2 * G::NV];  // (v, v) of voxels B2 + h + j
#pragma unroll
        for (int j4 = 0; j4 < G::NV; ++j4) {
          const float4 q = *reinterpret_cast<const float4*>(src + 4 * j4);
          d[2 * j4] = make_float2(q.x, q.y);
          d[2 * j4 + 1] = make_float2(q.z, q.w);
        }
        float2 acc[G::XH];  // (c_x I, w_x I)
#pragma unroll
        for (int i = 0; i < G::XH; ++i) {
          const int m = G::O2 + i + RS;  // centre of output h + i in d
          acc[i] = __fmul2_rn(cw0, d[m]);
#pragma unroll
          for (int k = 1; k <= RS; ++k) {
            const float2 dk = __ffma2_rn(d[m - k], sgn, d[m + k]);  // (v+ - v-, v+ + v-)
            acc[i] = __ffma2_rn(make_float2(tx.c[RS + k], tx.w[RS + k]), dk, acc[i]);
          }
        }
        float4* o = reinterpret_cast<float4*>(sx + row * G::SXS + 2 * (8 * xseg + h));
#pragma unroll
        for (int i = 0; i < G::XH; i += 2) o[i / 2] = make_float4(acc[i].x, acc[i].y, acc[i + 1].x, acc[i + 1].y);
      }
    }
    __syncthreads();  // x-pass rows complete
    // y pass: slide the window by TB, append this column's rows
#pragma unroll
    for (int j = 0; j < 2 * RS; ++j) wp[j] = wp[j + TB];
#pragma unroll
    for (int r = 0; r < TB; ++r) wp[2 * RS + r] = *reinterpret_cast<const float2*>(sx + r * G::SXS + 2 * t);
    if (b >= G::W) {
      const int m0 = (b - G::W) * TB;  // first output row of this block, relative to p0
#pragma unroll
      for (int i = 0; i < TB; ++i) {
        const int m = i + RS;
        float2 f02 = __fmul2_rn(wy0, wp[m]);  // (w_y c_x I, w_y w_x I)
        float f1 = 0.f;
#pragma unroll
        for (int k = 1; k <= RS; ++k) {
          f02 = __ffma2_rn(make_float2(ty.w[RS + k], ty.w[RS + k]), __fadd2_rn(wp[m + k], wp[m - k]), f02);
          f1 = fmaf(ty.c[RS + k], wp[m + k].y - wp[m - k].y, f1);
        }
        if (xok && m0 + i < L) {
          float* o = obase + (int64_t)(m0 + i) * ostride;
          o[0] = f02.x;
          o[nab] = f1;
          o[2 * nab] = f02.y;
        }
      }
    }
  }
}

// The same over a batch of volumes in one persistent launch (MultiTable).
template <int RS, int XT>
__global__ void __launch_bounds__(XT, 512 / XT)
    k_grad_xy_multi(const GxyItem* __restrict__ items, const MultiTable T, const __grid_constant__ Taps tx,
                    const __grid_constant__ Taps ty) {
  for_each_vblock(T, [&](int i, const VBlock& v) {
    const GxyItem it = items[i];  // a local copy: the body keeps its fields in registers
    grad_xy_body<RS, XT>(it.vol, it.vb, it.dimx, it.dimy, it.F, it.ab, it.seg, tx, ty, v);
  });
}

// ---------------------------------------------------------------- z pass
// One thread per (x, y) column of the output box walks z.  The three partial
// fields arrive by 4-byte cp.async into a shared ring of P = 2R+1 steps
// (dynamic shared memory, P * 3 KB), issued kGzAhead steps ahead; ring slots
// and register windows are indexed statically because the step loop is
// unrolled by P.
constexpr int kGzThreads = 256;

// Scale of each product g_a g_b (1 / (spacing_a spacing_b)); `unit` when all are 1.
struct ProdScale {
  float s[6];
  int unit;
};
#ifndef CT_GZ_AHEAD
#define CT_GZ_AHEAD 8
#endif
#ifndef CT_GZ_MINB
#define CT_GZ_MINB 2
#endif
constexpr int kGzAhead = CT_GZ_AHEAD;

// 2^-8 keeps every possible gradient of uint16 data inside FP16's range while
// leaving gradients down to 2^-6 intensity units normal.
constexpr float kGzHalfScale = 1.0f / 256.0f;

// GOUT: write the gradient itself (3 planes: FP16 holding g * 2^-8 in the
// mixed form, FP32 otherwise) for a consumer that forms the products, instead
// of the six products.
template <int RS, bool MIXED, bool GOUT, typename BLK>
__device__ __forceinline__ void grad_z_body(const float* __restrict__ F, const Box& ab, void* __restrict__ Jv,
                                            const Box& ob, int seg, const Taps& taps, const ProdScale& ps,
                                            const BLK blk) {
  constexpr int P = 2 * RS + 1;
  constexpr int AH = kGzAhead < P ? kGzAhead : P - 1;  // steps in flight (the ring holds P)
  // [P] steps of (F0, F1) pairs [kGzThreads][2], then F2 [kGzThreads]: the x and y
  // components run as FP32 pairs (one packed add and fma per tap for both)
  extern __shared__ __align__(16) float gz_ring[];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int x = ob.lo[0] + blk.x() * blockDim.x + threadIdx.x;
  const int yr = blk.y() * blockDim.y + threadIdx.y;
  const bool ok = x < ob.lo[0] + ob.n[0] && yr < ob.n[1];
  const int xi = min(x, ob.lo[0] + ob.n[0] - 1);
  const int y = ob.lo[1] + min(yr, ob.n[1] - 1);
  const int p0 = ob.lo[2] + blk.z() * seg;  // first output plane
  const int L = min(seg, ob.lo[2] + ob.n[2] - p0);
  if (L <= 0) return;
  const int nsteps = L + 2 * RS;

  // input column (xi, y) of the partial fields; step s reads plane p0 - RS + s,
  // clamped to the planes the fields cover (the volume's edges, or the halo)
  const int64_t nab = box_vox(ab);
  const float* base = F + box_index(ab, xi, y, ab.lo[2]);
  const int plane = ab.n[0] * ab.n[1];
  const int q0 = p0 - RS - ab.lo[2];
  auto src = [&](int s) -> const float* { return base + (int64_t)min(max(q0 + s, 0), ab.n[2] - 1) * plane; };
  const uint32_t ring01 = (uint32_t)__cvta_generic_to_shared(gz_ring + 2 * tid);
  const uint32_t ring2 = (uint32_t)__cvta_generic_to_shared(gz_ring + 2 * kGzThreads + tid);
  constexpr uint32_t kStep = 3 * kGzThreads * sizeof(float);
  auto issue = [&](int s, int slot) {
    if (s < nsteps) {
      const float* p = src(s);
      cp_async4(ring01 + slot * kStep, p);
      cp_async4(ring01 + slot * kStep + 4, p + nab);
      cp_async4(ring2 + slot * kStep, p + 2 * nab);
    }
    cp_async_commit();
  };
#pragma unroll
  for (int s = 0; s < AH; ++s) issue(s, s);

  const int64_t nob = box_vox(ob);
  float* J = static_cast<float*>(Jv);
  __half* Jh = static_cast<__half*>(Jv);
  const int64_t obase_i = box_index(ob, xi, y, p0);
  float* obase = J + obase_i;
  const int ostride = ob.n[0] * ob.n[1];
  float2 w01[P];
  float w2[P];
#pragma unroll
  for (int i = 0; i < P; ++i) {
    w01[i] = make_float2(0.f, 0.f);
    w2[i] = 0.f;
  }

  for (int base_s = 0; base_s < nsteps; base_s += P) {
#pragma unroll
    for (int u = 0; u < P; ++u) {
      const int s = base_s + u;
      if (s >= nsteps) continue;
      cp_async_wait<AH - 1>();  // step s has landed (this thread's own copies)
      w01[u] = *reinterpret_cast<const float2*>(gz_ring + 3 * u * kGzThreads + 2 * tid);
      w2[u] = gz_ring[(3 * u + 2) * kGzThreads + tid];
      issue(s + AH, (u + AH) % P);  // into the slot of step s + AH - P, consumed already
      if (s >= 2 * RS) {
        const int c = (u + P - RS) % P;  // window slot of the output plane
        // (gx, gy) as a pair: each lane rounds as the scalar fmaf / add would
        float2 gxy = __fmul2_rn(make_float2(taps.w[RS], taps.w[RS]), w01[c]);
        float gz = 0.f;
#pragma unroll
        for (int k = 1; k <= RS; ++k) {
          const int sp = (u + P - RS + k) % P, sm = (u + P - RS - k) % P;
          gxy = __ffma2_rn(make_float2(taps.w[RS + k], taps.w[RS + k]), __fadd2_rn(w01[sp], w01[sm]), gxy);
          gz = fmaf(taps.c[RS + k], w2[sp] - w2[sm], gz);
        }
        float gx = gxy.x, gy = gxy.y;
        if (GOUT) {  // the gradient itself, held in FP16 (scaled) in the mixed form
          if (ok) {
            const int64_t o = obase_i + (int64_t)(s - 2 * RS) * ostride;
            if (MIXED) {
              Jh[o] = __float2half_rn(gx * kGzHalfScale);
              Jh[o + nob] = __float2half_rn(gy * kGzHalfScale);
              Jh[o + 2 * nob] = __float2half_rn(gz * kGzHalfScale);
            } else {
              J[o] = gx;
              J[o + nob] = gy;
              J[o + 2 * nob] = gz;
            }
          }
          continue;
        }
        if (MIXED) {  // gradient held in FP16 (scaled), products formed exactly in FP32
          gx = __half2float(__float2half_rn(gx * kGzHalfScale)) * (1.0f / kGzHalfScale);
          gy = __half2float(__float2half_rn(gy * kGzHalfScale)) * (1.0f / kGzHalfScale);
          gz = __half2float(__float2half_rn(gz * kGzHalfScale)) * (1.0f / kGzHalfScale);
        }
        if (ok) {
          float* o = obase + (int64_t)(s - 2 * RS) * ostride;
          if (ps.unit) {
            o[0] = gx * gx;
            o[nob] = gy * gy;
            o[2 * nob] = gz * gz;
            o[3 * nob] = gx * gy;
            o[4 * nob] = gx * gz;
            o[5 * nob] = gy * gz;
          } else {  // physical units: component ab divided by spacing_a spacing_b
            o[0] = (gx * gx) * ps.s[0];
            o[nob] = (gy * gy) * ps.s[1];
            o[2 * nob] = (gz * gz) * ps.s[2];
            o[3 * nob] = (gx * gy) * ps.s[3];
            o[4 * nob] = (gx * gz) * ps.s[4];
            o[5 * nob] = (gy * gz) * ps.s[5];
          }
        }
      }
    }
  }
  cp_async_wait<0>();
}

template <int RS, bool MIXED, bool GOUT>
__global__ void __launch_bounds__(kGzThreads, CT_GZ_MINB > 0 ? CT_GZ_MINB : (RS <= 8 ? 3 : 2))
    k_grad_z(const float* __restrict__ F, const __grid_constant__ Box ab, void* __restrict__ Jv,
             const __grid_constant__ Box ob, int seg,
             const __grid_constant__ Taps taps, const __grid_constant__ ProdScale ps) {
  grad_z_body<RS, MIXED, GOUT>(F, ab, Jv, ob, seg, taps, ps, HwBlock{});
}

// The same (the six products) over a batch of volumes in one persistent launch,
// blocks of kGzMultiX x (kGzThreads / kGzMultiX) threads.
constexpr int kGzMultiX = 128;
template <int RS, bool MIXED>
__global__ void __launch_bounds__(kGzThreads, CT_GZ_MINB > 0 ? CT_GZ_MINB : (RS <= 8 ? 3 : 2))
    k_grad_z_multi(const GzItem* __restrict__ items, const MultiTable T, const __grid_constant__ Taps taps,
                   const __grid_constant__ ProdScale ps) {
  for_each_vblock(T, [&](int i, const VBlock& v) {
    const GzItem it = items[i];  // a local copy: the body keeps its fields in registers
    grad_z_body<RS, MIXED, false>(it.F, it.ab, it.J, it.ob, it.seg, taps, ps, v);
  });
}

// ---------------------------------------------------------------- launch
#ifndef CT_GXY_XT
#define CT_GXY_XT 128  // columns (threads) per gradient x/y CTA (tuning choice)
#endif
template <int RS, int XT>
static cudaError_t set_xy_attr() {
  return cudaFuncSetAttribute(k_grad_xy<RS, XT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)GXYGeom<RS, XT>::SMEM);
}

template <int RS>
static size_t gz_smem() {
  return sizeof(float) * (2 * RS + 1) * 3 * kGzThreads;
}

template <int RS>
static cudaError_t prepare_gs() {
  cudaError_t e = set_xy_attr<RS, CT_GXY_XT>();
  const int sm = (int)gz_smem<RS>();
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_grad_xy_multi<RS, CT_GXY_XT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)GXYGeom<RS, CT_GXY_XT>::SMEM);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_grad_z_multi<RS, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_grad_z_multi<RS, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_grad_z<RS, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_grad_z<RS, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_grad_z<RS, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_grad_z<RS, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  return e;
}

int sigma_kernel_radius(int r) {
  static const int radii[] = {2, 3, 4, 6, 8, 12};
  for (int v : radii)
    if (r <= v) return v;
  return -1;
}

cudaError_t prepare_grad_split_kernels() {
  cudaError_t e = prepare_gs<2>();
  if (e == cudaSuccess) e = prepare_gs<3>();
  if (e == cudaSuccess) e = prepare_gs<4>();
  if (e == cudaSuccess) e = prepare_gs<6>();
  if (e == cudaSuccess) e = prepare_gs<8>();
  if (e == cudaSuccess) e = prepare_gs<12>();
  return e;
}

// The box of the partial fields for gradient outputs over ob: ob grown by RS
// in z and clipped to the volume and to the input box.
Box grad_partial_box(const Box& ob, const Box& vb, int rs, int dimz) {
  Box a = ob;
  const int lo = max(max(0, vb.lo[2]), ob.lo[2] - rs);
  const int hi = min(min(dimz, vb.lo[2] + vb.n[2]), ob.lo[2] + ob.n[2] + rs);
  a.lo[2] = lo;
  a.n[2] = hi - lo;
  return a;
}

template <int RS, int XT>
static cudaError_t launch_gxy_t(const uint16_t* vol, const Box& vb, const int dims[3], float* F, const Box& ab,
                                const Taps& tx, const Taps& ty, cudaStream_t st) {
  using G = GXYGeom<RS, XT>;
  if (ab.n[2] > 65535) return cudaErrorInvalidValue;
  const int64_t ctas = (int64_t)((ab.n[0] + XT - 1) / XT) * ab.n[2];
  int nseg = 1;
  while (nseg < 16 && ctas * nseg < (int64_t)152 * 2 * 4 * (256 / XT) && ab.n[1] / (nseg * 2) >= 8 * G::TB) nseg *= 2;
  const int seg = (ab.n[1] + nseg - 1) / nseg;
  dim3 grid((ab.n[0] + XT - 1) / XT, ab.n[2], (ab.n[1] + seg - 1) / seg);
  k_grad_xy<RS, XT><<<grid, XT, G::SMEM, st>>>(vol, vb, dims[0], dims[1], F, ab, seg, tx, ty);
  return cudaGetLastError();
}

// 128-column CTAs at every width: four CTAs of 4 warps per SM wait at their
// barriers independently (512^3: 0.62 ms, against 0.67 with two CTAs of 256
// columns, the same 16 warps per SM)
template <int RS>
static cudaError_t launch_gxy_r(const uint16_t* vol, const Box& vb, const int dims[3], float* F, const Box& ab,
                                const Taps& tx, const Taps& ty, cudaStream_t st) {
  return launch_gxy_t<RS, CT_GXY_XT>(vol, vb, dims, F, ab, tx, ty, st);
}

template <int RS>
static cudaError_t launch_gz_r(const float* F, const Box& ab, void* J, const Box& ob, const Taps& taps,
                               const ProdScale& ps, bool mixed, bool gout, cudaStream_t st) {
  // warps along x: the widest that leaves the fewest idle columns
  int wx = 1;
  for (int w = 2; w <= kGzThreads / 32; w *= 2) {
    const int span = 32 * w, best = 32 * wx;
    if (32 * (w / 2) >= ob.n[0]) break;
    if ((ob.n[0] + span - 1) / span * span <= (ob.n[0] + best - 1) / best * best) wx = w;
  }
  dim3 block(32 * wx, kGzThreads / (32 * wx));
  const int64_t cols = (int64_t)((ob.n[0] + block.x - 1) / block.x) * ((ob.n[1] + block.y - 1) / block.y);
  int nseg = 1;
  while (nseg < 16 && cols * nseg < (int64_t)152 * 2 * 4 && ob.n[2] / (nseg * 2) >= 4 * (2 * RS + 1)) nseg *= 2;
  const int seg = (ob.n[2] + nseg - 1) / nseg;
  dim3 grid((ob.n[0] + block.x - 1) / block.x, (ob.n[1] + block.y - 1) / block.y, (ob.n[2] + seg - 1) / seg);
  if (grid.y > 65535 || grid.z > 65535) return cudaErrorInvalidValue;
  if (gout) {
    if (mixed)
      k_grad_z<RS, true, true><<<grid, block, gz_smem<RS>(), st>>>(F, ab, J, ob, seg, taps, ps);
    else
      k_grad_z<RS, false, true><<<grid, block, gz_smem<RS>(), st>>>(F, ab, J, ob, seg, taps, ps);
  } else if (mixed) {
    k_grad_z<RS, true, false><<<grid, block, gz_smem<RS>(), st>>>(F, ab, J, ob, seg, taps, ps);
  } else {
    k_grad_z<RS, false, false><<<grid, block, gz_smem<RS>(), st>>>(F, ab, J, ob, seg, taps, ps);
  }
  return cudaGetLastError();
}

cudaError_t launch_grad_xy(const uint16_t* vol, const Box& vb, const int dims[3], float* F, const Box& ab,
                           const Taps& tx, const Taps& ty, int rk, cudaStream_t st) {
  if (box_vox(ab) == 0) return cudaSuccess;
  if (box_vox(ab) >= ((int64_t)1 << 31)) return cudaErrorInvalidValue;
  switch (rk) {
    case 2: return launch_gxy_r<2>(vol, vb, dims, F, ab, tx, ty, st);
    case 3: return launch_gxy_r<3>(vol, vb, dims, F, ab, tx, ty, st);
    case 4: return launch_gxy_r<4>(vol, vb, dims, F, ab, tx, ty, st);
    case 6: return launch_gxy_r<6>(vol, vb, dims, F, ab, tx, ty, st);
    case 8: return launch_gxy_r<8>(vol, vb, dims, F, ab, tx, ty, st);
    case 12: return launch_gxy_r<12>(vol, vb, dims, F, ab, tx, ty, st);
    default: return cudaErrorInvalidValue;
  }
}

// ---------------------------------------------------------------- batches
// A batch item's walk is never split into segments: the batch's items fill
// the GPU, and every segment would recompute its warm-up rows.
template <int RS>
static uint3 gxy_item(GxyItem& it) {
  constexpr int XT = CT_GXY_XT;
  const Box& ab = it.ab;
  it.seg = ab.n[1];
  return make_uint3((ab.n[0] + XT - 1) / XT, ab.n[2], 1);
}

uint3 grad_xy_item(int rk, GxyItem& it) {
  switch (rk) {
    case 2: return gxy_item<2>(it);
    case 3: return gxy_item<3>(it);
    case 4: return gxy_item<4>(it);
    case 6: return gxy_item<6>(it);
    case 8: return gxy_item<8>(it);
    default: return gxy_item<12>(it);
  }
}

template <int RS>
static cudaError_t gxy_multi(const GxyItem* items, const MultiTable& T, int64_t blocks, const Taps& tx,
                             const Taps& ty, cudaStream_t st) {
  using G = GXYGeom<RS, CT_GXY_XT>;
  const int grid = persistent_grid(k_grad_xy_multi<RS, CT_GXY_XT>, CT_GXY_XT, G::SMEM, blocks);
  k_grad_xy_multi<RS, CT_GXY_XT><<<grid, CT_GXY_XT, G::SMEM, st>>>(items, T, tx, ty);
  return cudaGetLastError();
}

cudaError_t launch_grad_xy_multi(const GxyItem* items, const MultiTable& T, int64_t blocks, const Taps& tx,
                                 const Taps& ty, int rk, cudaStream_t st) {
  switch (rk) {
    case 2: return gxy_multi<2>(items, T, blocks, tx, ty, st);
    case 3: return gxy_multi<3>(items, T, blocks, tx, ty, st);
    case 4: return gxy_multi<4>(items, T, blocks, tx, ty, st);
    case 6: return gxy_multi<6>(items, T, blocks, tx, ty, st);
    case 8: return gxy_multi<8>(items, T, blocks, tx, ty, st);
    case 12: return gxy_multi<12>(items, T, blocks, tx, ty, st);
    default: return cudaErrorInvalidValue;
  }
}

template <int RS>
static uint3 gz_item(GzItem& it) {
  const Box& ob = it.ob;
  const dim3 block(kGzMultiX, kGzThreads / kGzMultiX);
  it.seg = ob.n[2];  // unsplit (see gxy_item)
  return make_uint3((ob.n[0] + block.x - 1) / block.x, (ob.n[1] + block.y - 1) / block.y, 1);
}

uint3 grad_z_item(int rk, GzItem& it) {
  switch (rk) {
    case 2: return gz_item<2>(it);
    case 3: return gz_item<3>(it);
    case 4: return gz_item<4>(it);
    case 6: return gz_item<6>(it);
    case 8: return gz_item<8>(it);
    default: return gz_item<12>(it);
  }
}

template <int RS>
static cudaError_t gz_multi(const GzItem* items, const MultiTable& T, int64_t blocks, const Taps& tz,
                            const ProdScale& ps, bool mixed, cudaStream_t st) {
  const dim3 block(kGzMultiX, kGzThreads / kGzMultiX);
  if (mixed) {
    const int grid = persistent_grid(k_grad_z_multi<RS, true>, kGzThreads, gz_smem<RS>(), blocks);
    k_grad_z_multi<RS, true><<<grid, block, gz_smem<RS>(), st>>>(items, T, tz, ps);
  } else {
    const int grid = persistent_grid(k_grad_z_multi<RS, false>, kGzThreads, gz_smem<RS>(), blocks);
    k_grad_z_multi<RS, false><<<grid, block, gz_smem<RS>(), st>>>(items, T, tz, ps);
  }
  return cudaGetLastError();
}

cudaError_t launch_grad_z_multi(const GzItem* items, const MultiTable& T, int64_t blocks, const Taps& tz,
                                const float scale[6], int rk, bool mixed, cudaStream_t st) {
  ProdScale ps;
  ps.unit = 1;
  for (int k = 0; k < 6; ++k) {
    ps.s[k] = scale[k];
    ps.unit = ps.unit && scale[k] == 1.f;
  }
  switch (rk) {
    case 2: return gz_multi<2>(items, T, blocks, tz, ps, mixed, st);
    case 3: return gz_multi<3>(items, T, blocks, tz, ps, mixed, st);
    case 4: return gz_multi<4>(items, T, blocks, tz, ps, mixed, st);
    case 6: return gz_multi<6>(items, T, blocks, tz, ps, mixed, st);
    case 8: return gz_multi<8>(items, T, blocks, tz, ps, mixed, st);
    case 12: return gz_multi<12>(items, T, blocks, tz, ps, mixed, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_grad_z(const float* F, const Box& ab, void* J, const Box& ob, const Taps& tz,
                          const float scale[6], int rk, bool mixed, bool gout, cudaStream_t st) {
  if (box_vox(ob) == 0) return cudaSuccess;
  if (box_vox(ab) >= ((int64_t)1 << 31) || box_vox(ob) >= ((int64_t)1 << 31)) return cudaErrorInvalidValue;
  ProdScale ps;
  ps.unit = 1;
  for (int k = 0; k < 6; ++k) {
    ps.s[k] = scale[k];
    ps.unit = ps.unit && scale[k] == 1.f;
  }
  switch (rk) {
    case 2: return launch_gz_r<2>(F, ab, J, ob, tz, ps, mixed, gout, st);
    case 3: return launch_gz_r<3>(F, ab, J, ob, tz, ps, mixed, gout, st);
    case 4: return launch_gz_r<4>(F, ab, J, ob, tz, ps, mixed, gout, st);
    case 6: return launch_gz_r<6>(F, ab, J, ob, tz, ps, mixed, gout, st);
    case 8: return launch_gz_r<8>(F, ab, J, ob, tz, ps, mixed, gout, st);
    case 12: return launch_gz_r<12>(F, ab, J, ob, tz, ps, mixed, gout, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ct
