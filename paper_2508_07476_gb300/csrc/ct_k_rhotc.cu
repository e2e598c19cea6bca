// The integration-scale smoothing (Figure 1b) as a 1-D pass along one axis on
// the tensor cores (tcgen05, TF32 operands, FP32 accumulation): a banded
// Toeplitz product per tile instead of the FP32 stencil.
//
// A tile is M = 128 lines (for y / z: consecutive x of one (component, other)
// row; for x: 128 consecutive (component, z, y) rows) by N = NT outputs along
// the axis (NT = 64, or 32 for the largest radius).  With the window of
// W = NT + 2 RA input positions of a tile (RA = the radius rounded up to a
// multiple of 4, so that W is a multiple of 8),
//   D[m][n] = sum_k A[m][k] B[n][k],   A[m][k] = in(line m, first - RA + k),
//   B[n][k] = w[k - n - (RA - R)] (zero off the band of 2R + 1 taps),
// one M x N x W product.  Each operand is split into a TF32 head and the FP32
// remainder (a = a_hi + a_lo): the taps' heads are rounded to TF32, the data's
// heads truncated (the low 13 mantissa bits cleared: one logic operation instead
// of a conversion, on the producers' path), and
//   D = A_hi B_hi + A_hi B_lo + A_lo B_hi
// keeps every product within about 2^-19 of its value (|A_lo| < 2^-10 |A|,
// read by the MMA to 11 significant bits; the dropped A_lo B_lo is below
// 2^-21), far inside the FP32 stage tolerances.
//
// A_hi and A_lo live in tensor memory (lane m = line m, one column per
// position), each a ring of WR = W + NT columns indexed by position mod WR.
// Tiles advance by NT positions, so staging tile t writes the slots of
// positions that only tiles up to t - 2 read: a tile can be staged while its
// predecessor's product runs.  A k-step of 8 positions starts on a multiple of
// 8 and never straddles the wrap.  B_hi / B_lo are fixed for the launch and
// staged once per CTA in shared memory (K-major core matrices of 8 outputs x
// 4 positions).
//
// The CTA is warp-specialised, one CTA per SM holding all 512 tensor-memory
// columns.  Producer warps own the 128 lines (x form: four warps, one line per
// thread; y / z forms: eight warps, two per lane quadrant, each with half of
// every chunk's positions).  NT-position chunks of their lines are copied into
// shared memory several chunks ahead, in one stream that runs on across work
// units: in the y / z forms by the producers themselves with cp.async
// (16-byte copies when the boxes are 16-byte aligned); in the x form, where
// each line is a row, by four copy warps, one per producer warp, with tensor
// (TMA) or bulk copies completing on per-slice mbarriers, refilled once the
// producer warp releases the slice.  The producers split a landed chunk, write
// both rings and arrive on the tile's "staged" mbarrier.  An MMA warp waits on
// it, issues the 3 W / 8 MMAs (one elected lane, the loop in warp-uniform
// control flow) into one of two accumulators and commits them to that
// accumulator's mbarrier.  Four epilogue warps wait on it, read their 32
// lanes of D, free the accumulator (a third mbarrier) and store the outputs;
// in the x form an epilogue thread writes its row of outputs by a tensor or
// bulk store, and unaligned or clamped pieces go through coalesced
// per-element copies and a padded shared-memory transpose.
// Every wait is bounded; a CTA that gives up raises a flag that ends the other
// roles' waits, drains its MMAs and releases the tensor memory.
#include <cuda.h>  // CUtensorMap and its enums; the encoder is fetched from the driver at run time

#include <algorithm>
#include <cstring>

#include "ct_common.cuh"
#include "ct_launch.h"

namespace ct {

namespace {

constexpr int kTcLines = 128;  // = M: TMEM lane m holds line m
// Warp roles: producer warps 0 .. NP-1, epilogue warps NP .. NP+3, the MMA warp
// NP+4.  The x form has one producer thread per line (NP = 4), and four copy
// warps NP+5 .. NP+8: copy warp w fills the chunk slices of producer warp
// w % 4 (its 32 rows), so that no producer waits for a copy to be issued and
// each producer / copy pair runs on its own.  The y / z forms split each
// chunk's positions between two producer warps per lane quadrant (NP = 8: warp
// w stages positions [(w / 4) NT / 2, + NT / 2) of the lines 32 (w % 4) ..),
// which halves each producer thread's work per tile, and copy their own parts.
#ifndef CT_TC_PCOPY
#define CT_TC_PCOPY 1  // tuning: the products (first) pass with copy warps too (0: its producers copy)
#endif
template <bool XAXIS, int PROD = 0>
struct TcRoles {
  static constexpr int NP = XAXIS ? 4 : 8;
  static constexpr bool COPY = XAXIS || (CT_TC_PCOPY && PROD != 0);  // copy warps NP+5 .. NP+8
  static constexpr int THREADS = 32 * (NP + 5 + (COPY ? 4 : 0));
  static constexpr int MMA_WARP = NP + 4;
};
constexpr int kTcNB = 4;                       // mbarriers per hand-off, used by tiles g mod 4 in turn
#ifndef CT_TC_NT64_MAX_R
#define CT_TC_NT64_MAX_R 36  // tuning: largest radius instance with 64-output tiles
#endif
#ifndef CT_TC_XSTAGES
#define CT_TC_XSTAGES 3  // tuning: x form, chunk stages in flight (with the copy warps 3 beat 2: 0.95 vs 1.04 ms)
#endif
#ifndef CT_TC_PSTAGES
#define CT_TC_PSTAGES 5  // tuning: products pass from the FP16 gradient, chunk stages (at most what fits)
#endif
#ifndef CT_TC_YZSTAGES
#define CT_TC_YZSTAGES 4  // tuning: y / z forms (plain and FP16 products), chunk stages in flight
#endif
#ifndef CT_TC_XEPI
#define CT_TC_XEPI 1  // tuning: x form, output buffers per epilogue warp (2: a tile's store overlaps the next)
#endif
#ifndef CT_TC_BIG_RING
#define CT_TC_BIG_RING 1  // tuning: 0 restarts a W + NT ring at every work unit
#endif
constexpr uint32_t kTcWaitLimit = 1u << 20;    // mbarrier polls before a CTA gives up (and drain limit)
constexpr uint32_t kTcSuspendNs = 500;         // a waiting thread sleeps up to this long per poll

template <int RR>
struct TcGeom {
  static constexpr int RA = (RR + 3) / 4 * 4;    // window margin: W is a multiple of 8
  // outputs per tile (MMA N): 64, which at R = 36 leaves room for one
  // accumulator only (CT_TC_NT64_MAX_R = 32 keeps two there with 32-output tiles)
  static constexpr int NT = RR <= CT_TC_NT64_MAX_R ? 64 : 32;
  static constexpr int W = NT + 2 * RA;          // window positions of a tile
  static constexpr int KCB = W / 4;              // core-matrix columns of B
  static constexpr int KS = W / 8;               // k-steps per tile
  static constexpr int P = (2 * RA + NT - 1) / NT;  // NT-position chunks that fill the ring
  // The ring runs on across work units (window positions numbered globally)
  // when it can hold the last two windows of one unit plus the halo and first
  // tile of the next, beside two accumulators: then no unit start waits for
  // the previous unit's last products.  Otherwise it restarts at every unit,
  // after those products (at R = 24 the longer ring would leave room for one
  // accumulator only, which measured slower: 1.21 / 1.17 vs 1.12 / 1.13 ms
  // for the y / z passes at 512^3).
  static constexpr bool BIG = CT_TC_BIG_RING && P == 1 && 2 * (W + NT + 2 * RA) + 2 * NT <= 512;
  static constexpr int WR = BIG ? W + NT + 2 * RA : W + NT;  // ring positions
  static constexpr int ND = 2 * WR + 2 * NT <= 512 ? 2 : 1;   // accumulators
  static constexpr int LO = WR;                              // tensor memory: A_hi ring, A_lo ring, ND D
  static constexpr int DCOL = 2 * WR;
  static constexpr int TCOLS = 512;  // one CTA per SM holds all of it
  static_assert(DCOL + ND * NT <= TCOLS && WR % 8 == 0, "tensor memory");
  static constexpr int B_BYTES = NT * W * 4;
  // FP16-gradient chunk stages that fit beside B (one 128-line x NT-position chunk of two FP16 components)
  static constexpr int P2FIT = (232448 - 1024 - 2 * B_BYTES) / (NT * kTcLines * 4);
  static constexpr int XS = NT + 4;  // x-form chunk row: 16-byte aligned, conflict-free by line
  static constexpr int TE = NT + 4;  // x-form output row: 16-byte aligned, float4 writes conflict-free
  static constexpr int ROW_BYTES = kTcLines * 8;
  // x form: each warp owns one 1024-byte-aligned slice of a chunk stage or of the
  // output buffer, whichever layout a chunk uses (32 padded rows of XS floats, or
  // NT / 32 swizzled 32 x 32 boxes), so that every hand-off stays within the warp
  static constexpr int WS = (32 * XS * 4 + 1023) / 1024 * 1024;
  // one chunk: y / z [NT positions][128 lines] (products: two such arrays of
  // gradient components, FP32 or FP16); x four warp slices
  static constexpr int raw_floats(bool xaxis, int prod = 0) {
    return xaxis ? 4 * WS / 4 : (prod == 1 ? 2 * NT * kTcLines : NT * kTcLines);
  }
  // chunks in flight (FP32 gradient pairs: two, the most that fit beside B)
  static constexpr int stages(bool xaxis, int prod = 0) {
    return xaxis ? CT_TC_XSTAGES
                 : (prod == 1 ? 2
                              : (prod == 2 ? (CT_TC_PSTAGES < P2FIT ? CT_TC_PSTAGES : P2FIT) : CT_TC_YZSTAGES));
  }
  static_assert((2 * B_BYTES) % 1024 == 0 && NT * 32 * 4 <= WS && TE == XS, "x-form slices");
  static constexpr int need(bool xaxis, int prod = 0) {
    return 1024 + 2 * B_BYTES + stages(xaxis, prod) * raw_floats(xaxis, prod) * 4 +
           (xaxis ? 4 * CT_TC_XEPI * WS + 2 * ROW_BYTES : 0);  // + slack to align the base to 1024 bytes
  }
  // dynamic shared memory requested: at least half an SM's (233472 bytes,
  // 1 KB reserved per CTA), so that one CTA, holding all the tensor memory,
  // is resident per SM
  static constexpr int smem(bool xaxis, int prod = 0) {
    return need(xaxis, prod) > 233472 / 2 ? need(xaxis, prod) : 233472 / 2;
  }
  static_assert(need(false, 1) <= 232448 && need(false, 2) <= 232448 && need(true) <= 232448, "shared memory");
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp_async16(uint32_t smem_dst, const float* gsrc) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_dst), "l"(gsrc) : "memory");
}

// Bulk copy global -> shared on the TMA engine, completing `bytes` on an mbarrier.
__device__ __forceinline__ void bulk_g2s(uint32_t smem_dst, const float* gsrc, uint32_t bytes, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(smem_dst),
      "l"(gsrc), "r"(bytes), "r"(mbar)
      : "memory");
}

// Bulk copy shared -> global (bulk group of the issuing thread).
__device__ __forceinline__ void bulk_s2g(float* gdst, uint32_t smem_src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n" ::"l"(gdst), "r"(smem_src), "r"(bytes)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}


// Tensor (TMA) copies of a 3-D box (x, row, component), completing on an mbarrier / bulk group.
__device__ __forceinline__ void tma_load3(uint32_t smem_dst, const CUtensorMap* map, int x, int y, int z,
                                          uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n" ::
          "r"(smem_dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(mbar)
      : "memory");
}

__device__ __forceinline__ void tma_store3(const CUtensorMap* map, int x, int y, int z, uint32_t smem_src) {
  asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];\n" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(x), "r"(y), "r"(z), "r"(smem_src)
               : "memory");
}

// Byte offset of float x (0..31) of row r (0..31) in a 32 x 32 box stored with
// the 128-byte swizzle (16-byte chunk index XOR row mod 8; 1024-byte aligned).
__device__ __forceinline__ int swz(int r, int x) { return r * 128 + ((((x >> 2) ^ r) & 7) << 4) + ((x & 3) << 2); }

// Shared-memory matrix descriptor: K-major, no swizzle; lbo = byte stride of
// core matrices along K, sbo = along M/N.
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor: D FP32, A and B TF32, both K-major, then N and M.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// The TF32 head of a data value: x with its low 13 mantissa bits cleared (an
// exact TF32 value; x - head is exact in FP32).
__device__ __forceinline__ float tf32_head(float x) { return __uint_as_float(__float_as_uint(x) & 0xffffe000u); }

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// float index of element (row r, k) of a K-major no-swizzle operand with kc core columns
__host__ __device__ __forceinline__ int core_index(int r, int k, int kc) {
  return ((r >> 3) * kc + (k >> 2)) * 32 + (r & 7) * 4 + (k & 3);
}

// One k-step of the split product into D, issued by one elected lane of a
// warp that runs this in uniform control flow (operands stay warp-uniform):
// D (+)= A_hi B_hi + A_hi B_lo + A_lo B_hi, with A_hi / A_lo from tensor memory.
__device__ __forceinline__ void mma_kstep(uint32_t d, uint32_t a_hi, uint32_t a_lo, uint64_t b_hi, uint64_t b_lo,
                                          uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p, q, e;\nelect.sync _|e, 0xffffffff;\nsetp.ne.b32 p, %6, 0;\nsetp.eq.b32 q, 0, 0;\n"
      "@e tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %3, %5, p;\n"
      "@e tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %4, %5, q;\n"
      "@e tcgen05.mma.cta_group::1.kind::tf32 [%0], [%2], %3, %5, q;\n}\n" ::"r"(d),
      "r"(a_hi), "r"(a_lo), "l"(b_hi), "l"(b_lo), "r"(idesc), "r"(acc));
}

// Commit the MMAs the elected lane issued to an mbarrier (same lane as mma_kstep).
__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile(
      "{\n.reg .pred e;\nelect.sync _|e, 0xffffffff;\n"
      "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n}\n" ::"r"(mbar)
      : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t mbar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(mbar), "r"(parity), "r"(kTcSuspendNs)
      : "memory");
  return done != 0;
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  for (uint32_t i = 0; i < kTcWaitLimit; ++i)
    if (mbar_try(mbar, parity)) return true;
  return false;
}

// Bounded wait (at most `limit` polls) that also gives up once another thread
// of the CTA has raised *abort.
__device__ __forceinline__ bool mbar_wait_or_abort(uint32_t mbar, uint32_t parity, const volatile int* abort,
                                                   uint32_t limit = kTcWaitLimit) {
  for (uint32_t i = 0; i < limit; ++i) {
    if (mbar_try(mbar, parity)) return true;
    if (*abort) return false;
  }
  return false;
}

__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const float v[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
               "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
               "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
               "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
               : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float v[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

// One unit's geometry as seen by line m: the segment, and the line's input
// (relative position 0) and output (position a_lo) addresses with their strides.
struct TcUnit {
  int p0, nt;  // first tile start (absolute, a multiple of NT), tiles
  const float* src;
  float* dst;
  int64_t istride, ostride;
  bool lok;           // line m exists
  bool wfull = true;  // y / z: all 32 lines of this thread's warp exist (16-byte copies read 4 lines)
  // products form: element offsets of the line's relative position 0 in the
  // planes of gradient components a and b of the unit's component g_a g_b
  int64_t ga = 0, gb = 0;
  int comp = 0;
  // x form with tensor maps: the warp's first row as (row, component) of the
  // output view (computed once per unit: 64-bit divisions are long)
  int orow = 0, ocomp = 0;
};

// The products form's inputs: gradient planes (FP32, or FP16 holding g * 2^-8)
// and the factor of each product (1 / (spacing_a spacing_b); `unit` when all 1).
struct TcProd {
  float s[6];
  int unit;
};

// component k of the tensor = g_a g_b with a = kProdA[k], b = kProdB[k] (xx yy zz xy xz yz)
__host__ __device__ constexpr int prod_a(int k) { return k < 3 ? k : (k < 5 ? 0 : 1); }
__host__ __device__ constexpr int prod_b(int k) { return k < 3 ? k : (k == 3 ? 1 : 2); }

template <int PROD>
struct GradT {
  using T = float;
  static constexpr float kBScale = 1.0f;
  // the product g_a g_b
  static __device__ __forceinline__ float prod(float a, float b) { return a * b; }
};
template <>
struct GradT<2> {
  using T = __half;
  // The mixed form's gradient is FP16 holding g * 2^-8.  The product of two
  // FP16 values is exact in FP32, so one mixed-precision FMA (FP16 operands,
  // FP32 result, + 0) gives (g_a 2^-8)(g_b 2^-8) exactly; the missing 2^16 is
  // carried by the taps (B scaled by 2^16, which scales every product of the
  // pass exactly), so D is the same as from the restored products.
  static constexpr float kBScale = 65536.0f;
  static __device__ __forceinline__ float prod(__half a, __half b) {
    float r;
    asm("fma.rn.f32.f16 %0, %1, %2, %3;" : "=f"(r) : "h"(__half_as_ushort(a)), "h"(__half_as_ushort(b)), "f"(0.0f));
    return r;
  }
};

// One 1-D pass of the integration-scale Gaussian along `axis` (0, 1 or 2; XAXIS
// selects the row-transposing x form): out (6 planes over ob) from in (6 planes
// over ib), positions clamped to the volume [0, dim_axis) and to ib.  Work
// unit = (line group, segment of `seg` outputs, a multiple of NT).  Tiles
// start at absolute multiples of NT along the axis, so that an output's taps
// meet the same k-steps whatever box it is computed in: chunked runs
// reproduce the whole-volume result bit for bit.  vec: bit 0, the input box
// allows 16-byte copies; bit 1 (x form), the output rows start on 16-byte
// boundaries; bits 2 / 3 (x form), tin / tout map the 128-row groups as
// (x, row, component) boxes of the input / output (all checked on the host).
//
// PROD (y / z form only): the input is not the 6 tensor planes but the 3
// gradient planes (1: FP32, 2: FP16 holding g * 2^-8), and the producers form
// each component's product g_a g_b (times its factor) from the two staged
// gradient chunks before splitting it, with the same FP32 operations the
// gradient kernel would have used to store it: the product field never
// crosses HBM.  Work units then take the six components of one line group
// in turn, so that the group's gradient lines are read from L2 after the
// first component.
template <int RR, bool XAXIS, int PROD>
__global__ void __launch_bounds__(TcRoles<XAXIS, PROD>::THREADS, 1)
    k_rho_tc(const float* __restrict__ in, Box ib, int dim_axis, float* __restrict__ out, Box ob, int axis, int seg,
             int vec, const __grid_constant__ Taps taps, const __grid_constant__ CUtensorMap tin,
             const __grid_constant__ CUtensorMap tout, const TcCtl ctl, const TcProd pr) {
  static_assert(!(XAXIS && PROD), "the products form is a y / z form");
  using G = TcGeom<RR>;
  using GT = typename GradT<PROD>::T;
  constexpr int NT = G::NT;
  constexpr int S = G::stages(XAXIS, PROD);
  constexpr int RAWF = G::raw_floats(XAXIS, PROD);
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  float* sBhi = reinterpret_cast<float*>(smem);
  float* sBlo = reinterpret_cast<float*>(smem + G::B_BYTES);
  float* sRaw = reinterpret_cast<float*>(smem + 2 * G::B_BYTES);
  unsigned char* xs = smem + 2 * G::B_BYTES + S * RAWF * 4;  // x form only
  float* sTe = reinterpret_cast<float*>(xs);
  const float** sSrc = reinterpret_cast<const float**>(xs + 4 * CT_TC_XEPI * G::WS);
  float** sDst = reinterpret_cast<float**>(xs + 4 * CT_TC_XEPI * G::WS + G::ROW_BYTES);
  __shared__ __align__(8) uint64_t bar_xfull[8][4];   // copy warps: slice q of chunk stage s has landed
  __shared__ __align__(8) uint64_t bar_xempty[8][4];  // copy warps: the producers of slice q have read stage s
  __shared__ __align__(8) uint64_t bar_staged[kTcNB];  // the producers have staged tile g
  __shared__ __align__(8) uint64_t bar_mma[kTcNB];     // tile g's product is in D[g % ND]
  __shared__ __align__(8) uint64_t bar_dfree[kTcNB];   // the epilogue has read tile g's D
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  using RL = TcRoles<XAXIS, PROD>;
  const int role = w < RL::NP ? 0 : (w < RL::NP + 4 ? 1 : (w == RL::MMA_WARP ? 2 : 3));  // producer, epilogue,
                                                                                          // MMA, copy (x form)
  const int m = tid & (kTcLines - 1);            // line / TMEM lane (roles 0 and 1)
  const int wq = w & 3;                          // lane quadrant of this warp

  // B = the banded Toeplitz matrix of the taps, split into TF32 head and remainder
  for (int e = tid; e < NT * G::W; e += RL::THREADS) {
    const int n = e / G::W, k = e % G::W;
    const int j = k - n - (G::RA - RR);
    const float v = (j >= 0 && j <= 2 * RR) ? taps.w[j] * GradT<PROD>::kBScale : 0.f;
    const float hi = tf32_round(v);
    const int c = core_index(n, k, G::KCB);
    sBhi[c] = hi;
    sBlo[c] = v - hi;
  }
  if (tid == 0) {
    for (int a = 0; a < S; ++a)
      for (int q = 0; q < 4; ++q) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 32;" ::"r"(smem_u32(&bar_xfull[a][q])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar_xempty[a][q])),
                     "r"(RL::NP / 4));  // the producer warps of lane quadrant q
      }
    for (int a = 0; a < kTcNB; ++a) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar_staged[a])), "n"(32 * RL::NP));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_mma[a])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar_dfree[a])), "n"(kTcLines));
    }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (w == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "n"(G::TCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tm = tmem_base;
  const uint32_t tlane = tm + ((uint32_t)(wq * 32) << 16);  // this warp's 32 lanes
  // mbarriers of tile g, and the parity of its phase
  auto staged_bar = [&](uint32_t g) { return smem_u32(&bar_staged[g % kTcNB]); };
  auto mma_bar = [&](uint32_t g) { return smem_u32(&bar_mma[g % kTcNB]); };
  auto dfree_bar = [&](uint32_t g) { return smem_u32(&bar_dfree[g % kTcNB]); };
  auto par = [](uint32_t g) { return (g / kTcNB) & 1u; };

  // line groups and segments
  const int a_lo = ob.lo[axis], a_end = ob.lo[axis] + ob.n[axis];
  const int a_first = a_lo & ~(NT - 1);  // first tile start (a_lo >= 0)
  const int other = XAXIS ? 1 : 3 - axis;
  const int64_t n_rows = XAXIS ? 6 * (int64_t)ob.n[1] * ob.n[2] : 0;
  const int ngx = (ob.n[0] + kTcLines - 1) / kTcLines;
  const int64_t n_groups = XAXIS ? (n_rows + kTcLines - 1) / kTcLines : 6 * (int64_t)ob.n[other] * ngx;
  const int64_t n_units = n_groups * ((a_end - a_first + seg - 1) / seg);
  const int alo = ib.lo[axis], an = ib.n[axis];
  const int qlo = max(0, alo) - alo, qhi = min(dim_axis - 1, alo + an - 1) - alo;  // clamp range, relative
  // x form with tensor maps: a group's rows are contiguous rows of the (x, row, component) views
  const int64_t rows_pc = (int64_t)ob.n[1] * ob.n[2];                  // output rows per component
  const int64_t row_off = (int64_t)(ob.lo[2] - ib.lo[2]) * ib.n[1];    // input row of output row 0

  auto decode = [&](int64_t unit) {
    TcUnit U;
    const int sgi = (int)(unit / n_groups);
    const int64_t grp = unit % n_groups;
    U.p0 = a_first + sgi * seg;
    U.nt = (min(seg, a_end - U.p0) + NT - 1) / NT;
    U.istride = U.ostride = 1;
    if (XAXIS) {
      const int64_t r = grp * kTcLines + m;
      U.lok = r < n_rows;
      const int64_t rc = U.lok ? r : n_rows - 1;
      const int yy = ob.lo[1] + (int)(rc % ob.n[1]);
      const int64_t t2 = rc / ob.n[1];
      const int zz = ob.lo[2] + (int)(t2 % ob.n[2]);
      const int comp = (int)(t2 / ob.n[2]);
      U.src = in + comp * box_vox(ib) + box_index(ib, ib.lo[0], yy, zz);
      U.dst = out + comp * box_vox(ob) + box_index(ob, a_lo, yy, zz);
      if (vec & 12) {
        const int64_t r0 = grp * kTcLines + 32 * (m >> 5);  // the warp's first row
        U.orow = (int)(r0 % rows_pc);
        U.ocomp = (int)(r0 / rows_pc);
      }
    } else {
      // plain: groups by (component, other, x group), x group fastest; products:
      // component fastest (the six components of a line group in turn)
      const int xg = PROD ? (int)((grp / 6) % ngx) : (int)(grp % ngx);
      const int64_t co = PROD ? (grp / 6) / ngx : grp / ngx;
      const int comp = PROD ? (int)(grp % 6) : (int)(co / ob.n[other]);
      const int o = ob.lo[other] + (int)(PROD ? co : co % ob.n[other]);
      const int x = ob.lo[0] + xg * kTcLines + m;
      U.lok = x < ob.lo[0] + ob.n[0];
      U.wfull = xg * kTcLines + 32 * (m >> 5) + 32 <= ob.n[0];
      const int xi = min(x, ob.lo[0] + ob.n[0] - 1);
      const int yb = axis == 1 ? ib.lo[1] : o, zb = axis == 1 ? o : ib.lo[2];
      U.src = in + comp * box_vox(ib) + box_index(ib, xi, yb, zb);
      if (PROD) {
        U.comp = comp;
        U.ga = prod_a(comp) * box_vox(ib) + box_index(ib, xi, yb, zb);
        U.gb = prod_b(comp) * box_vox(ib) + box_index(ib, xi, yb, zb);
      }
      U.istride = axis == 1 ? ib.n[0] : (int64_t)ib.n[0] * ib.n[1];
      const int yo = axis == 1 ? a_lo : o, zo = axis == 1 ? o : a_lo;
      U.dst = out + comp * box_vox(ob) + box_index(ob, xi, yo, zo);
      U.ostride = axis == 1 ? ob.n[0] : (int64_t)ob.n[0] * ob.n[1];
    }
    return U;
  };

  uint32_t g = 0;          // tiles this thread's role has handled (every role counts the same sequence)
  uint32_t committed = 0;  // MMA warp: tiles whose MMAs it has committed
  // a producer warp's positions of each chunk: [p_lo, p_lo + NTP)
  constexpr int NTP = XAXIS ? NT : NT / 2;
  const int p_lo = XAXIS ? 0 : (w >> 2) * NTP;
  // The copy stream (y / z producers, x copy warps): chunk ic of unit iu (window
  // positions NT ic for ic < P, then tile ic - P's NT), one cp.async group per
  // chunk, stage k mod S
  int64_t iu = blockIdx.x;
  int ic = 0, iC = 0, iq0 = 0;
  TcUnit IU;
  auto enter = [&](int64_t u) {
    iu = u;
    ic = 0;
    if (u >= n_units) return;
    IU = decode(u);
    iC = G::P + IU.nt;
    iq0 = IU.p0 - G::RA - alo;
    if (XAXIS) {
      __syncwarp();  // the warp's copies of the previous unit have been issued
      sSrc[m] = IU.src;
      __syncwarp();
    }
  };
  // y / z forms: positions [plo, plo + NTP) of chunk rb (relative input position
  // qs of its position 0; inside: no position needs clamping) for this thread's
  // lines
  auto stage_yz = [&](float* rb, int qs, bool inside, int plo) {
    if (PROD) {
      // the two gradient components of the unit's product (one for xx, yy, zz)
      const GT* gbase = reinterpret_cast<const GT*>(in);
      GT* sa = reinterpret_cast<GT*>(rb);
      GT* sb = sa + NT * kTcLines;
      const bool two = prod_a(IU.comp) != prod_b(IU.comp);
      if ((vec & 1) && IU.wfull) {
        // 16-byte copies of LPC consecutive lines, within the warp's own 32 lines:
        // lane -> line group qd of the warp, positions pg + PPI i, each clamped
        // to the box (a copy holds one position of its lines)
        constexpr int LPC = 16 / (int)sizeof(GT), GPW = 32 / LPC, PPI = 32 / GPW;
        const int qd = lane % GPW, pg = lane / GPW;
        const GT* pa = gbase + IU.ga + (LPC * qd - lane);
        const GT* pb = gbase + IU.gb + (LPC * qd - lane);
#pragma unroll
        for (int i = 0; i < NTP / PPI; ++i) {
          const int pos = plo + pg + PPI * i;
          const int64_t q = (int64_t)(inside ? qs + pos : min(max(qs + pos, qlo), qhi)) * IU.istride;
          const int so = pos * kTcLines + 32 * wq + LPC * qd;
          cp_async16(smem_u32(sa + so), reinterpret_cast<const float*>(pa + q));
          if (two) cp_async16(smem_u32(sb + so), reinterpret_cast<const float*>(pb + q));
        }
      } else if (IU.lok) {  // this thread's own line, position by position (clamped to the box)
#pragma unroll 4
        for (int j = plo; j < plo + NTP; ++j) {
          const int64_t q = (int64_t)min(max(qs + j, qlo), qhi) * IU.istride;
          if (PROD == 1) {  // FP32: asynchronous 4-byte copies
            cp_async4(smem_u32(sa + j * kTcLines + m), reinterpret_cast<const float*>(gbase + IU.ga + q));
            if (two)
              cp_async4(smem_u32(sb + j * kTcLines + m), reinterpret_cast<const float*>(gbase + IU.gb + q));
          } else {  // FP16: below the 4-byte copy size, loaded and stored here
            sa[j * kTcLines + m] = gbase[IU.ga + q];
            if (two) sb[j * kTcLines + m] = gbase[IU.gb + q];
          }
        }
      }
    } else if ((vec & 1) && IU.wfull) {  // 16 bytes (4 lines) per copy, within the warp's
                                   // own 32 lines (the stage hand-off is warp-local):
                                   // lane -> lines 32 wq + 4 (lane % 8).., positions
                                   // lane / 8 + 4 i, each clamped to the box; a warp
                                   // with lines past the box copies its own line below
      const int qd = lane & 7, pg = lane >> 3;
      const float* p = IU.src + (4 * qd - lane);
#pragma unroll
      for (int i = 0; i < NTP / 4; ++i) {
        const int pos = plo + pg + 4 * i;
        const int64_t q = (int64_t)(inside ? qs + pos : min(max(qs + pos, qlo), qhi)) * IU.istride;
        cp_async16(smem_u32(rb + pos * kTcLines + 32 * wq + 4 * qd), p + q);
      }
    } else if (!IU.lok) {
      // a line past the box: its products are never stored and every line's
      // row of the product is its own, so it stages nothing
    } else if (inside) {
      const float* p = IU.src + qs * IU.istride;
#pragma unroll
      for (int j = plo; j < plo + NTP; ++j) cp_async4(smem_u32(rb + j * kTcLines + m), p + j * IU.istride);
    } else {
#pragma unroll
      for (int j = plo; j < plo + NTP; ++j)
        cp_async4(smem_u32(rb + j * kTcLines + m), IU.src + min(max(qs + j, qlo), qhi) * IU.istride);
    }
  };
  uint32_t k_issue = 0;
  auto issue_next = [&]() {
    if (iu < n_units) {
      float* rb = sRaw + (k_issue % S) * RAWF;
      const int qs = iq0 + (ic < G::P ? NT * ic : 2 * G::RA + NT * (ic - G::P));
      const bool inside = qs >= qlo && qs + NT - 1 <= qhi;  // no clamping in this chunk
      if (XAXIS) {
        const uint32_t cb = smem_u32(&bar_xfull[k_issue % S][wq]);
        const int a = max(qs, qlo), b = min(qs + NT - 1, qhi);  // the chunk's part inside the box
        if ((vec & 4) && inside) {  // two swizzled 32 x 32 boxes per slice, issued by one lane
          if (lane == 0) {
            mbar_arrive_tx(cb, NT * 32 * 4);
#pragma unroll
            for (int h = 0; h < NT / 32; ++h)
              tma_load3(smem_u32(reinterpret_cast<unsigned char*>(rb) + wq * G::WS + h * 4096), &tin,
                        qs + 32 * h, (int)row_off + IU.orow, IU.ocomp, cb);
          } else {
            mbar_arrive(cb);
          }
        } else if ((vec & 1) && b >= a) {  // one bulk copy of that part of this thread's own row; the reader
                                    // replicates the edge (start and length stay multiples of 4)
          mbar_arrive_tx(cb, (b - a + 1) * 4);
          bulk_g2s(smem_u32(rb + wq * (G::WS / 4) + lane * G::XS + (a - qs)), IU.src + a, (b - a + 1) * 4, cb);
        } else {
#pragma unroll
          for (int h = 0; h < NT / 32; ++h) {
            const int rel = min(max(qs + 32 * h + lane, qlo), qhi);
#pragma unroll
            for (int i = 0; i < 32; ++i)
              cp_async4(smem_u32(rb + wq * (G::WS / 4) + i * G::XS + 32 * h + lane), sSrc[32 * wq + i] + rel);
          }
          // this thread's arrival once its copies have landed
          asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(cb) : "memory");
        }
      } else if (RL::COPY) {  // a copy warp of the products pass: both halves of its lines' positions
        stage_yz(rb, qs, inside, 0);
        stage_yz(rb, qs, inside, NTP);
        const uint32_t cb = smem_u32(&bar_xfull[k_issue % S][wq]);
        if (PROD == 2 && !((vec & 1) && IU.wfull))
          mbar_arrive(cb);  // FP16 element copies are plain stores: a plain arrival releases them
        else  // this thread's arrival once its copies have landed
          asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(cb) : "memory");
      } else {
        stage_yz(rb, qs, inside, p_lo);
      }
      if (++ic == iC) enter(iu + gridDim.x);
    }
    cp_async_commit();
    ++k_issue;
  };
  if (role == 0) {
    if (!RL::COPY) {
      enter(blockIdx.x);
#pragma unroll 1
      for (int i = 0; i < S; ++i) issue_next();
    }
    uint32_t k = 0;  // chunks consumed
    bool go = true;
    int gbase = 0;  // ring position of this unit's window position 0 (continuous ring: runs on)
    int ws1 = 0, ws2 = 0, ws3 = 0, ws4 = 0;  // continuous ring: window starts of tiles g-1 .. g-4
    for (int64_t unit = blockIdx.x; unit < n_units && go; unit += gridDim.x) {
      const TcUnit CU = decode(unit);
      const int nt = CU.nt;
      const float fprod = PROD ? (CU.comp < 3 ? (CU.comp == 0 ? pr.s[0] : CU.comp == 1 ? pr.s[1] : pr.s[2])
                                              : (CU.comp == 3 ? pr.s[3] : CU.comp == 4 ? pr.s[4] : pr.s[5]))
                               : 1.f;  // selected without indexing the parameter (no stack copy)
      if (!G::BIG) gbase = 0;
      const int q0u = CU.p0 - G::RA - alo;  // relative input position of window position 0
      for (int c = 0; c < G::P + nt; ++c, ++k) {
        if (!RL::COPY) {
          cp_async_wait<S - 1>();  // chunk k has landed
          __syncwarp();            // and so have the other lanes' copies (each warp copies only its own lines)
        }
        // x form: the copy warp's copies of this warp's slice of chunk k have
        // landed (never waited for with the short limit: a copy warp that gives
        // up raises the abort flag)
        if (RL::COPY && !__all_sync(0xffffffffu, mbar_wait_or_abort(smem_u32(&bar_xfull[k % S][wq]), (k / S) & 1u,
                                                                 &abort_flag))) {
          abort_flag = 1;
          go = false;
          break;
        }
        const float* rb = sRaw + (k % S) * RAWF;
        float v[NTP];
        if (XAXIS) {
          const int qs = q0u + (c < G::P ? NT * c : 2 * G::RA + NT * (c - G::P));
          const int jlo = max(0, qlo - qs), jhi = min(NT - 1, qhi - qs);
          const bool tma = (vec & 4) && jlo == 0 && jhi == NT - 1;
#pragma unroll
          for (int j = 0; j < NT; j += 4) {
            const float* src4 = tma ? reinterpret_cast<const float*>(reinterpret_cast<const unsigned char*>(rb) +
                                                                   wq * G::WS + (j / 32) * 4096 + swz(lane, j & 31))
                                    : rb + wq * (G::WS / 4) + lane * G::XS + j;
            const float4 f = *reinterpret_cast<const float4*>(src4);
            v[j] = f.x;
            v[j + 1] = f.y;
            v[j + 2] = f.z;
            v[j + 3] = f.w;
          }
          if (!tma && (vec & 1) && jhi >= jlo) {  // a bulk chunk: positions outside the box take the edge value
            if (jlo > 0 || jhi < NT - 1) {
              const float* row = rb + wq * (G::WS / 4) + lane * G::XS;
              const float elo = row[jlo], ehi = row[jhi];
#pragma unroll
              for (int j = 0; j < NT; ++j) v[j] = j < jlo ? elo : (j > jhi ? ehi : v[j]);
            }
          }
        } else if (PROD) {
          const GT* sa = reinterpret_cast<const GT*>(rb);
          const GT* sb = prod_a(CU.comp) != prod_b(CU.comp) ? sa + NT * kTcLines : sa;
          const float f = fprod;
#pragma unroll
          for (int j = 0; j < NTP; ++j) {
            const float ab = GradT<PROD>::prod(sa[(p_lo + j) * kTcLines + m], sb[(p_lo + j) * kTcLines + m]);
            v[j] = pr.unit ? ab : ab * f;
          }
        } else {
#pragma unroll
          for (int j = 0; j < NTP; ++j) v[j] = rb[(p_lo + j) * kTcLines + m];
        }
        if (RL::COPY) {
          // the copy warp refills the slice (x: with bulk / tensor copies, the
          // async proxy: this warp's reads are ordered before them by a proxy
          // fence, without which a refill overtook the reads of a work unit's
          // first chunk), then the warp releases the slice
          if (XAXIS) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          __syncwarp();
          if (lane == 0) mbar_arrive(smem_u32(&bar_xempty[k % S][wq]));
        } else {
          __syncwarp();  // every lane has read the stage before it is refilled
          issue_next();
        }
        const int t = c - G::P;  // tile of this chunk (< 0: ring fill)
        const int q = c < G::P ? NT * c : 2 * G::RA + NT * t;
        const int nw = c < G::P ? min(NT, 2 * G::RA - q) : NT;  // positions written (a fill chunk: its halo part)
        bool ok = true;
        if (G::BIG) {
          // the slots of positions [gbase + q, + nw) last held positions WR lower: wait for the
          // latest tile whose window starts below their end (window starts increase; it is
          // never more than four tiles back)
          const int lim = gbase + q + nw - G::WR;
          int back = 0;
          if (g >= 1 && ws1 < lim)
            back = 1;
          else if (g >= 2 && ws2 < lim)
            back = 2;
          else if (g >= 3 && ws3 < lim)
            back = 3;
          else if (g >= 4 && ws4 < lim)
            back = 4;
          if (back) ok = mbar_wait_or_abort(mma_bar(g - back), par(g - back), &abort_flag, ctl.wait_limit);
        } else if (c == 0) {  // the ring restarts: every MMA of the previous unit must have read it
          if (g >= 1) ok = mbar_wait_or_abort(mma_bar(g - 1), par(g - 1), &abort_flag, ctl.wait_limit);
          if (g >= 2) ok = mbar_wait_or_abort(mma_bar(g - 2), par(g - 2), &abort_flag, ctl.wait_limit) && ok;
        } else if (t >= 2) {  // tile t's positions take the slots that only tiles up to t - 2 read
          ok = mbar_wait_or_abort(mma_bar(g - 2), par(g - 2), &abort_flag, ctl.wait_limit);
        }
        if (!__all_sync(0xffffffffu, ok)) {  // the whole warp gives up together
          abort_flag = 1;
          go = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // split and write both rings (slots mod WR)
#pragma unroll
        for (int cc = 0; cc < NTP / 8; ++cc) {
          if (p_lo + 8 * cc >= nw) break;  // uniform across the warp
          const int slot = (gbase + q + p_lo + 8 * cc) % G::WR;
          float hi[8], lo[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            hi[j] = tf32_head(v[8 * cc + j]);
            lo[j] = v[8 * cc + j] - hi[j];
          }
          tmem_st8(tlane + slot, hi);
          tmem_st8(tlane + G::LO + slot, lo);
        }
        if (t < 0) continue;
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        mbar_arrive(staged_bar(g));
        ws4 = ws3;
        ws3 = ws2;
        ws2 = ws1;
        ws1 = gbase + NT * t;
        ++g;
      }
      gbase += 2 * G::RA + NT * nt;
    }
    if (!RL::COPY) {
      cp_async_wait<0>();  // no cp.async copy is left in flight
      __syncwarp();
    }
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");  // nor a store to tensor memory
  } else if (role == 2) {
    const uint64_t bhi_d = umma_desc(smem_u32(sBhi), 128, G::KCB * 128);
    const uint64_t blo_d = umma_desc(smem_u32(sBlo), 128, G::KCB * 128);
    constexpr uint32_t kIdesc = idesc_tf32(kTcLines, NT);
    bool go = true;
    int gbase = 0;
    for (int64_t unit = blockIdx.x; unit < n_units && go; unit += gridDim.x) {
      const int nt = decode(unit).nt;
      if (!G::BIG) gbase = 0;
      for (int t = 0; t < nt; ++t, ++g) {
        // the tile is staged, and D[g % ND] has been read (tile g - ND)
        bool ok = mbar_wait_or_abort(staged_bar(g), par(g), &abort_flag, ctl.wait_limit);
        if (ok && g >= G::ND) ok = mbar_wait_or_abort(dfree_bar(g - G::ND), par(g - G::ND), &abort_flag, ctl.wait_limit);
        if (!__all_sync(0xffffffffu, ok)) {
          abort_flag = 1;
          go = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d = tm + G::DCOL + (g % G::ND) * NT;
        int slot = (gbase + NT * t) % G::WR;
#pragma unroll
        for (int ks = 0; ks < G::KS; ++ks) {
          const uint64_t bo = (uint64_t)(ks * 16);  // 256 bytes per k-step, in 16-byte units
          mma_kstep(d, tm + slot, tm + G::LO + slot, bhi_d + bo, blo_d + bo, kIdesc, ks > 0);
          slot = slot + 8 >= G::WR ? slot + 8 - G::WR : slot + 8;
        }
        mma_commit(mma_bar(g));
        committed = g + 1;
      }
      gbase += 2 * G::RA + NT * nt;
    }
  } else if (RL::COPY && role == 3) {
    // A copy warp: slice wq of chunk k (the lines of lane quadrant wq) into stage
    // k mod S once the quadrant's producer warps have read the slice's previous
    // chunk there
    enter(blockIdx.x);
    while (iu < n_units) {
      const uint32_t k = k_issue;
      if (k >= (uint32_t)S &&
          !__all_sync(0xffffffffu, mbar_wait_or_abort(smem_u32(&bar_xempty[k % S][wq]), ((k / S) - 1) & 1u,
                                                      &abort_flag, ctl.wait_limit))) {
        abort_flag = 1;
        break;
      }
      issue_next();
    }
    // every issued chunk's copies have landed before the CTA releases its memory
    // (a slice is refilled only after its previous chunk was read, so at most
    // the last S chunks can still be in flight)
    for (uint32_t j = k_issue > (uint32_t)S ? k_issue - S : 0; j < k_issue; ++j)
      mbar_wait(smem_u32(&bar_xfull[j % S][wq]), (j / S) & 1u);
  } else {
    bool go = true;
    for (int64_t unit = blockIdx.x; unit < n_units && go; unit += gridDim.x) {
      const TcUnit U = decode(unit);
      if (XAXIS) {
        __syncwarp();  // the warp's previous unit is done with its table
        sDst[m] = U.lok ? U.dst : nullptr;
        __syncwarp();
      }
      for (int t = 0; t < U.nt; ++t, ++g) {
        if (!__all_sync(0xffffffffu, mbar_wait_or_abort(mma_bar(g), par(g), &abort_flag, ctl.wait_limit))) {
          abort_flag = 1;
          go = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        float r[NT];
#pragma unroll
        for (int h = 0; h < NT / 32; ++h) tmem_ld32(tlane + G::DCOL + (g % G::ND) * NT + 32 * h, r + 32 * h);
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        mbar_arrive(dfree_bar(g));
        const int pt = U.p0 + NT * t;  // absolute position of output 0 of the tile
        const int nlo = max(0, a_lo - pt), nhi = min(NT, a_end - pt);  // stored outputs [nlo, nhi)
        const int64_t off = pt - a_lo;
        if (XAXIS) {
          // this thread's bulk stores of the tile that used this buffer last have read
          // their source (with two buffers, the previous tile's may still be reading)
          asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(CT_TC_XEPI - 1) : "memory");
          __syncwarp();  // and the warp's transposed stores have read theirs
          const int eslice = wq * CT_TC_XEPI + (CT_TC_XEPI == 2 ? (int)(g & 1) : 0);
          if ((vec & 8) && nlo == 0 && nhi == NT) {  // a whole tile: two swizzled box stores per warp
            unsigned char* eb = reinterpret_cast<unsigned char*>(sTe) + eslice * G::WS;
#pragma unroll
            for (int n = 0; n < NT; n += 4)
              *reinterpret_cast<float4*>(eb + (n / 32) * 4096 + swz(lane, n & 31)) =
                  make_float4(r[n], r[n + 1], r[n + 2], r[n + 3]);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) {
#pragma unroll
              for (int h = 0; h < NT / 32; ++h)
                tma_store3(&tout, pt - ob.lo[0] + 32 * h, U.orow, U.ocomp, smem_u32(eb + h * 4096));
              asm volatile("cp.async.bulk.commit_group;" ::: "memory");
            }
            continue;
          }
          float* er = sTe + eslice * (G::WS / 4);  // this warp's slice: its 32 rows at stride TE
#pragma unroll
          for (int n = 0; n < NT; n += 4)
            *reinterpret_cast<float4*>(er + lane * G::TE + n) = make_float4(r[n], r[n + 1], r[n + 2], r[n + 3]);
          if ((vec & 2) && nlo == 0 && nhi == NT) {  // a whole aligned tile: one bulk store per row
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            if (U.lok) bulk_s2g(U.dst + off, smem_u32(er + lane * G::TE), NT * 4);
          } else {
            __syncwarp();
#pragma unroll 4
            for (int i = 0; i < 32; ++i) {
              float* rd = sDst[32 * wq + i];
              if (rd) {
#pragma unroll
                for (int h = 0; h < NT / 32; ++h) {
                  const int n = 32 * h + lane;
                  if (n >= nlo && n < nhi) rd[off + n] = er[i * G::TE + n];
                }
              }
            }
          }
        } else if (U.lok) {
          float* d = U.dst + off * U.ostride;
          if (nlo == 0 && nhi == NT) {
#pragma unroll
            for (int n = 0; n < NT; ++n) d[n * U.ostride] = r[n];
          } else {
#pragma unroll
            for (int n = 0; n < NT; ++n)
              if (n >= nlo && n < nhi) d[n * U.ostride] = r[n];
          }
        }
      }
    }
  }
  if (XAXIS && role == 1) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");  // stores complete
  // a CTA that gave up waits once more (bounded) for the last product it
  // committed before it releases the tensor memory, and reports itself
  __syncthreads();
  if (abort_flag && w == RL::MMA_WARP) {
    if (committed >= 1) mbar_wait(mma_bar(committed - 1), par(committed - 1));
    if (lane == 0 && ctl.timeouts) atomicAdd(ctl.timeouts, 1u);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (w == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm), "n"(G::TCOLS));
}

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// The driver's tensor-map encoder (nullptr if the driver does not offer it).
EncodeTiled tensor_map_encoder() {
  static const EncodeTiled fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return (EncodeTiled) nullptr;
    return reinterpret_cast<EncodeTiled>(p);
  }();
  return fn;
}

// 6 planes over box b seen as (x, row = (z, y) flattened, component), in 32 x 32
// boxes with the 128-byte swizzle.  False if the encoder refuses.
bool rows_map(CUtensorMap* map, const float* base, const Box& b) {
  const EncodeTiled enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)b.n[0], (cuuint64_t)b.n[1] * b.n[2], 6};
  const cuuint64_t strides[2] = {(cuuint64_t)b.n[0] * 4, (cuuint64_t)box_vox(b) * 4};
  const cuuint32_t box[3] = {32, 32, 1}, estr[3] = {1, 1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int RR, bool XAXIS, int PROD>
struct TcLaunch {
  static bool ready;
  static cudaError_t prepare() {
    if (ready) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_rho_tc<RR, XAXIS, PROD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         TcGeom<RR>::smem(XAXIS, PROD));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_rho_tc<RR, XAXIS, PROD>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    ready = true;
    return cudaSuccess;
  }
  static cudaError_t run(const float* in, const Box& ib, const int dims[3], float* out, const Box& ob, int axis,
                         const Taps& taps, const TcCtl& ctl, const TcProd& pr, cudaStream_t st) {
    using G = TcGeom<RR>;
    cudaError_t e = prepare();
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    // one CTA per SM (it holds all of the SM's tensor memory)
    const int a_n = ob.lo[axis] + ob.n[axis] - (ob.lo[axis] & ~(G::NT - 1));  // aligned extent
    const int64_t groups = axis == 0 ? (6 * (int64_t)ob.n[1] * ob.n[2] + kTcLines - 1) / kTcLines
                                     : 6 * (int64_t)ob.n[3 - axis] * ((ob.n[0] + kTcLines - 1) / kTcLines);
    // outputs per unit: long enough to amortise the ring fill, short enough to spread
    // (a power of two from NT to 512, so that units start on tile boundaries)
    int seg = 512;
    while (ctl.seg_cap > 0 && seg > ctl.seg_cap && seg > G::NT) seg /= 2;
    while (seg > G::NT && groups * ((a_n + seg - 1) / seg) < 2 * sms) seg /= 2;
    const int64_t units = groups * ((a_n + seg - 1) / seg);
    const int grid = (int)std::min<int64_t>(units, sms);
    // 16-byte copies: the input rows start on 16-byte boundaries, and so do
    // the copied pieces (y / z: groups of 4 lines, 8 for FP16 gradients, in
    // warps whose 32 lines all lie in the box; x: the windows)
    const int lq = PROD == 2 ? 8 : 4;  // elements per 16 bytes
    const bool rows16 = ((uintptr_t)in % 16) == 0 && ib.n[0] % lq == 0;
    const bool vin = axis == 0 ? rows16 && ib.lo[0] % 4 == 0 : rows16 && (ob.lo[0] - ib.lo[0]) % lq == 0;
    const bool vout = axis == 0 && ((uintptr_t)out % 16) == 0 && ob.n[0] % 4 == 0 && ob.lo[0] % 4 == 0;
    int flags = (vin ? 1 : 0) | (vout ? 2 : 0);
    // x form: tensor maps when each 128-row group is 128 consecutive rows of one component,
    // in the input box (its y extent is the output's) and in the output box
    CUtensorMap tin, tout;
    std::memset(&tin, 0, sizeof tin);
    std::memset(&tout, 0, sizeof tout);
    if (axis == 0 && ((int64_t)ob.n[1] * ob.n[2]) % kTcLines == 0) {
      if (vin && ob.lo[1] == ib.lo[1] && ob.n[1] == ib.n[1] && rows_map(&tin, in, ib)) flags |= 4;
      if (vout && rows_map(&tout, out, ob)) flags |= 8;
    }
    k_rho_tc<RR, XAXIS, PROD><<<grid, TcRoles<XAXIS, PROD>::THREADS, G::smem(XAXIS, PROD), st>>>(in, ib, dims[axis], out, ob,
                                                                                           axis, seg,
                                                                              flags, taps, tin, tout, ctl, pr);
    return cudaGetLastError();
  }
};
template <int RR, bool XAXIS, int PROD>
bool TcLaunch<RR, XAXIS, PROD>::ready = false;

template <int RR>
cudaError_t run_tc(const float* in, const Box& ib, const int dims[3], float* out, const Box& ob, int axis,
                   const Taps& taps, const TcCtl& ctl, int prod, const TcProd& pr, cudaStream_t st) {
  if (axis == 0) return TcLaunch<RR, true, 0>::run(in, ib, dims, out, ob, axis, taps, ctl, pr, st);
  if (prod == 1) return TcLaunch<RR, false, 1>::run(in, ib, dims, out, ob, axis, taps, ctl, pr, st);
  if (prod == 2) return TcLaunch<RR, false, 2>::run(in, ib, dims, out, ob, axis, taps, ctl, pr, st);
  return TcLaunch<RR, false, 0>::run(in, ib, dims, out, ob, axis, taps, ctl, pr, st);
}

template <int RR>
cudaError_t prepare_tc() {
  cudaError_t e = TcLaunch<RR, true, 0>::prepare();
  if (e == cudaSuccess) e = TcLaunch<RR, false, 0>::prepare();
  if (e == cudaSuccess) e = TcLaunch<RR, false, 1>::prepare();
  if (e == cudaSuccess) e = TcLaunch<RR, false, 2>::prepare();
  return e;
}

cudaError_t dispatch_tc(const float* in, const Box& ib, const int dims[3], float* out, const Box& ob, int axis,
                        const Taps& taps, int rk, const TcCtl& ctl, int prod, const TcProd& pr, cudaStream_t st) {
  if (box_vox(ob) == 0) return cudaSuccess;
  if (axis < 0 || axis > 2 || (prod && axis == 0)) return cudaErrorInvalidValue;
  switch (rk) {
    case 4: return run_tc<4>(in, ib, dims, out, ob, axis, taps, ctl, prod, pr, st);
    case 6: return run_tc<6>(in, ib, dims, out, ob, axis, taps, ctl, prod, pr, st);
    case 8: return run_tc<8>(in, ib, dims, out, ob, axis, taps, ctl, prod, pr, st);
    case 12: return run_tc<12>(in, ib, dims, out, ob, axis, taps, ctl, prod, pr, st);
    case 16: return run_tc<16>(in, ib, dims, out, ob, axis, taps, ctl, prod, pr, st);
    case 24: return run_tc<24>(in, ib, dims, out, ob, axis, taps, ctl, prod, pr, st);
    case 32: return run_tc<32>(in, ib, dims, out, ob, axis, taps, ctl, prod, pr, st);
    case 36: return run_tc<36>(in, ib, dims, out, ob, axis, taps, ctl, prod, pr, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t prepare_rho_tc_kernels() {
  cudaError_t e = prepare_tc<4>();
  if (e == cudaSuccess) e = prepare_tc<6>();
  if (e == cudaSuccess) e = prepare_tc<8>();
  if (e == cudaSuccess) e = prepare_tc<12>();
  if (e == cudaSuccess) e = prepare_tc<16>();
  if (e == cudaSuccess) e = prepare_tc<24>();
  if (e == cudaSuccess) e = prepare_tc<32>();
  if (e == cudaSuccess) e = prepare_tc<36>();
  return e;
}

cudaError_t launch_rho_tc(const float* in, const Box& ib, const int dims[3], float* out, const Box& ob, int axis,
                          const Taps& taps, int rk, const TcCtl& ctl, cudaStream_t st) {
  TcProd pr;
  std::memset(&pr, 0, sizeof pr);
  return dispatch_tc(in, ib, dims, out, ob, axis, taps, rk, ctl, 0, pr, st);
}

cudaError_t launch_rho_tc_products(const void* g, bool half, const Box& ib, const int dims[3], float* out,
                                   const Box& ob, int axis, const Taps& taps, const float scale[6], int rk,
                                   const TcCtl& ctl, cudaStream_t st) {
  TcProd pr;
  pr.unit = 1;
  for (int k = 0; k < 6; ++k) {
    pr.s[k] = scale[k];
    pr.unit = pr.unit && scale[k] == 1.f;
  }
  return dispatch_tc(static_cast<const float*>(g), ib, dims, out, ob, axis, taps, rk, ctl, half ? 2 : 1, pr, st);
}

// The tensor cores take volumes whose x extent is a multiple of 4 (16-byte rows;
// a ragged last line group copies its lines past the box not at all).
bool rho_tc_volume_aligned(int nx, int axis) { return (void)axis, nx % 4 == 0; }

}  // namespace ct
