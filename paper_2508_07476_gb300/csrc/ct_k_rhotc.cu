// The integration-scale smoothing (Figure 1b) as a 1-D pass along one axis on
// the tensor cores (tcgen05, TF32 operands, FP32 accumulation): a banded
// Toeplitz product per tile instead of the FP32 stencil.
//
// A tile is M = 128 lines (for y / z: consecutive x of one (component, other)
// row; for x: 128 consecutive (component, z, y) rows) by N = 32 outputs along
// the axis.  With the window of W = 32 + 2 RA input positions of a tile (RA =
// the radius rounded up to a multiple of 4, so that W is a multiple of 8),
//   D[m][n] = sum_k A[m][k] B[n][k],   A[m][k] = in(line m, first - RA + k),
//   B[n][k] = w[k - n - (RA - R)] (zero off the band of 2R + 1 taps),
// one M x N x W product.  Each operand is split into a TF32 head and the FP32
// remainder (a = a_hi + a_lo, a_hi = a rounded to TF32), and
//   D = A_hi B_hi + A_hi B_lo + A_lo B_hi
// keeps every product within about 2^-20 of its value (the MMA reads the
// remainders to 11 significant bits; the dropped A_lo B_lo is below 2^-22),
// comparable with the FP32 stencil's own rounding.
//
// A_hi lives in tensor memory (lane m = line m, one column per position) and
// A_lo in shared memory (K-major core matrices of 8 lines x 4 positions);
// both are rings of W columns indexed by position mod W.  Since tiles advance
// by 32 positions and the ring holds one window, each tile writes only its 32
// new positions, into the slots of the 32 its predecessor no longer needs; a
// k-step of 8 positions starts on a multiple of 8 and never straddles the
// wrap.  B_hi / B_lo are fixed for the launch and staged once per CTA.
//
// Per tile: every thread splits its 32 new values (loaded during the previous
// tile's product) and writes them to the rings; one thread issues the
// 3 W / 8 MMAs and commits them to an mbarrier; the next tile's loads go out;
// after the (bounded) wait every warp reads its 32 lanes of D and stores the
// outputs.  For x the loads and stores go through a padded shared-memory
// transpose so that global accesses stay coalesced.  A CTA walks whole
// segments of a line group (persistent grid), so the ring is filled once per
// segment.
#include <algorithm>

#include "ct_common.cuh"
#include "ct_launch.h"

namespace ct {

namespace {

constexpr int kTcThreads = 128;              // = M: thread / TMEM lane m owns line m
constexpr int kTcNT = 32;                    // outputs per tile along the axis (MMA N)
constexpr uint32_t kTcWaitLimit = 1u << 20;  // mbarrier polls before a CTA gives up
constexpr uint32_t kTcSuspendNs = 500;       // a waiting thread sleeps up to this long per poll

// CTAs that gave up waiting for their MMAs (read and cleared by tc_timeouts()).
__device__ unsigned int g_tc_timeouts = 0;

template <int RR>
struct TcGeom {
  static constexpr int RA = (RR + 3) / 4 * 4;  // window margin: W is a multiple of 8
  static constexpr int W = kTcNT + 2 * RA;     // ring / window positions
  static constexpr int KC = W / 4;             // core-matrix columns of a K-major operand
  static constexpr int KS = W / 8;             // k-steps per tile
  static constexpr int TCOLS = W + kTcNT <= 128 ? 128 : 256;  // tensor-memory columns held
  static constexpr int DCOL = TCOLS - kTcNT;                  // accumulator columns
  static constexpr int MAX_CTAS = 512 / TCOLS;                // CTAs per SM that fit in TMEM
  static constexpr int ALO_BYTES = kTcThreads * W * 4;
  static constexpr int B_BYTES = kTcNT * W * 4;
  static constexpr int T_STRIDE = 33;  // padded row of the x-pass transpose
  static constexpr int T_BYTES = kTcThreads * T_STRIDE * 4;
  static constexpr int ROW_BYTES = kTcThreads * 8 * 2;  // x form: each row's input and output pointers
  static constexpr int need(bool xaxis) { return ALO_BYTES + 2 * B_BYTES + (xaxis ? T_BYTES + ROW_BYTES : 0); }
  // dynamic shared memory requested: at least enough that no more than
  // MAX_CTAS CTAs fit on an SM (233472 bytes, 1 KB reserved per CTA)
  static constexpr int smem(bool xaxis) {
    return need(xaxis) > 233472 / (MAX_CTAS + 1) ? need(xaxis) : 233472 / (MAX_CTAS + 1);
  }
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

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

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// float index of element (row r, k) of a K-major no-swizzle operand with kc core columns
__host__ __device__ __forceinline__ int core_index(int r, int k, int kc) {
  return ((r >> 3) * kc + (k >> 2)) * 32 + (r & 7) * 4 + (k & 3);
}

__device__ __forceinline__ void mma_ts(uint32_t d, uint32_t a_tmem, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
      "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_ss(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  for (uint32_t i = 0; i < kTcWaitLimit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity), "r"(kTcSuspendNs)
        : "memory");
    if (done) return true;
  }
  return false;
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

// One 1-D pass of the integration-scale Gaussian along `axis` (0, 1 or 2; XAXIS
// selects the row-transposing x form): out (6 planes over ob) from in (6 planes
// over ib), positions clamped to the volume [0, dim_axis) and to ib.  Work
// unit = (line group, segment of `seg` outputs, a multiple of 32).  Tiles
// start at absolute multiples of 32 along the axis, so that an output's taps
// meet the same k-steps whatever box it is computed in: chunked runs
// reproduce the whole-volume result bit for bit.
template <int RR, bool XAXIS>
__global__ void __launch_bounds__(kTcThreads, 3)
    k_rho_tc(const float* __restrict__ in, Box ib, int dim_axis, float* __restrict__ out, Box ob, int axis, int seg,
             const __grid_constant__ Taps taps) {
  using G = TcGeom<RR>;
  extern __shared__ __align__(128) unsigned char smem[];
  float* sAlo = reinterpret_cast<float*>(smem);
  float* sBhi = reinterpret_cast<float*>(smem + G::ALO_BYTES);
  float* sBlo = reinterpret_cast<float*>(smem + G::ALO_BYTES + G::B_BYTES);
  float* sT = reinterpret_cast<float*>(smem + G::ALO_BYTES + 2 * G::B_BYTES);
  const float** sSrc = reinterpret_cast<const float**>(smem + G::ALO_BYTES + 2 * G::B_BYTES + G::T_BYTES);
  float** sDst = reinterpret_cast<float**>(smem + G::ALO_BYTES + 2 * G::B_BYTES + G::T_BYTES + kTcThreads * 8);
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  const int m = threadIdx.x, w = m >> 5, lane = m & 31;

  // B = the banded Toeplitz matrix of the taps, split into TF32 head and remainder
  for (int e = m; e < kTcNT * G::W; e += kTcThreads) {
    const int n = e / G::W, k = e % G::W;
    const int j = k - n - (G::RA - RR);
    const float v = (j >= 0 && j <= 2 * RR) ? taps.w[j] : 0.f;
    const float hi = tf32_round(v);
    const int c = core_index(n, k, G::KC);
    sBhi[c] = hi;
    sBlo[c] = v - hi;
  }
  const uint32_t mbar_a = smem_u32(&mbar);
  if (m == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar_a));
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
  const uint32_t tlane = tm + ((uint32_t)(w * 32) << 16);  // this warp's 32 lanes
  constexpr uint32_t kC = G::KC * 128;                     // byte stride of 8-row core groups
  const uint64_t bhi_d = umma_desc(smem_u32(sBhi), 128, kC);
  const uint64_t blo_d = umma_desc(smem_u32(sBlo), 128, kC);
  const uint64_t alo_d = umma_desc(smem_u32(sAlo), 128, kC);
  constexpr uint32_t kIdesc = idesc_tf32(kTcThreads, kTcNT);

  // line groups and segments
  const int a_lo = ob.lo[axis], a_end = ob.lo[axis] + ob.n[axis];
  const int a_first = a_lo & ~(kTcNT - 1);  // first tile start (a_lo >= 0)
  const int other = XAXIS ? 1 : 3 - axis;
  const int64_t n_rows = XAXIS ? 6 * (int64_t)ob.n[1] * ob.n[2] : 0;
  const int ngx = (ob.n[0] + kTcThreads - 1) / kTcThreads;
  const int64_t n_groups = XAXIS ? (n_rows + kTcThreads - 1) / kTcThreads : 6 * (int64_t)ob.n[other] * ngx;
  const int64_t n_units = n_groups * ((a_end - a_first + seg - 1) / seg);
  const int alo = ib.lo[axis], an = ib.n[axis];
  const int qlo = max(0, alo) - alo, qhi = min(dim_axis - 1, alo + an - 1) - alo;  // clamp range, relative

  uint32_t parity = 0;
  bool ok = true;    // CTA-uniform: cleared only from a barrier's vote
  bool mine = true;  // this thread's waits all completed
  for (int64_t unit = blockIdx.x; unit < n_units && ok; unit += gridDim.x) {
    const int sgi = (int)(unit / n_groups);
    const int64_t grp = unit % n_groups;
    const int p0 = a_first + sgi * seg;  // first tile start of the segment
    const int L = min(seg, a_end - p0);
    const int nt = (L + kTcNT - 1) / kTcNT;
    const float* src;  // this thread's line at relative position 0 (stride istride)
    float* dst;        // this thread's line at output position a_lo (stride ostride)
    int64_t istride = 1, ostride = 1;
    bool lok;
    if (XAXIS) {
      const int64_t r = grp * kTcThreads + m;
      lok = r < n_rows;
      const int64_t rc = lok ? r : n_rows - 1;
      const int yy = ob.lo[1] + (int)(rc % ob.n[1]);
      const int64_t t2 = rc / ob.n[1];
      const int zz = ob.lo[2] + (int)(t2 % ob.n[2]);
      const int comp = (int)(t2 / ob.n[2]);
      src = in + comp * box_vox(ib) + box_index(ib, ib.lo[0], yy, zz);
      dst = out + comp * box_vox(ob) + box_index(ob, a_lo, yy, zz);
      __syncwarp();  // the warp's previous unit is done with the table
      sSrc[m] = src;
      sDst[m] = lok ? dst : nullptr;
      __syncwarp();
    } else {
      const int xg = (int)(grp % ngx);
      const int64_t co = grp / ngx;
      const int comp = (int)(co / ob.n[other]);
      const int o = ob.lo[other] + (int)(co % ob.n[other]);
      const int x = ob.lo[0] + xg * kTcThreads + m;
      lok = x < ob.lo[0] + ob.n[0];
      const int xi = min(x, ob.lo[0] + ob.n[0] - 1);
      const int yb = axis == 1 ? ib.lo[1] : o, zb = axis == 1 ? o : ib.lo[2];
      src = in + comp * box_vox(ib) + box_index(ib, xi, yb, zb);
      istride = axis == 1 ? ib.n[0] : (int64_t)ib.n[0] * ib.n[1];
      const int yo = axis == 1 ? a_lo : o, zo = axis == 1 ? o : a_lo;
      dst = out + comp * box_vox(ob) + box_index(ob, xi, yo, zo);
      ostride = axis == 1 ? ob.n[0] : (int64_t)ob.n[0] * ob.n[1];
    }
    const int q0 = p0 - G::RA - alo;  // relative input position of window position 0

    // pf: 32 consecutive window positions from q (y / z: of this thread's line;
    // x: position q + lane of each of the warp's 32 rows)
    float pf[32];
    auto load32 = [&](int q) {
      const int qs = q0 + q;
      if (XAXIS) {
        const int rel = min(max(qs + lane, qlo), qhi);
#pragma unroll
        for (int i = 0; i < 32; ++i) pf[i] = __ldg(sSrc[32 * w + i] + rel);
      } else if (qs >= qlo && qs + 31 <= qhi) {  // inside the input box: no clamping
        const float* p = src + qs * istride;
#pragma unroll
        for (int j = 0; j < 32; ++j) pf[j] = __ldg(p + j * istride);
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) pf[j] = __ldg(src + min(max(qs + j, qlo), qhi) * istride);
      }
    };
    // split positions q .. q + 31 and write them to the rings (slots mod W)
    auto stage32 = [&](int q) {
      float v[32];
      if (XAXIS) {
#pragma unroll
        for (int i = 0; i < 32; ++i) sT[(32 * w + i) * G::T_STRIDE + lane] = pf[i];
        __syncwarp();
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = sT[m * G::T_STRIDE + j];
        __syncwarp();
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = pf[j];
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int slot = (q + 8 * c) % G::W;
        float hi[8], lo[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          hi[j] = tf32_round(v[8 * c + j]);
          lo[j] = v[8 * c + j] - hi[j];
        }
        tmem_st8(tlane + slot, hi);
        float4* d = reinterpret_cast<float4*>(sAlo + core_index(m, slot, G::KC));
        d[0] = make_float4(lo[0], lo[1], lo[2], lo[3]);
        d[8] = make_float4(lo[4], lo[5], lo[6], lo[7]);  // next core column: +32 floats
      }
    };

    // fill the ring with the first 2 RA positions, then fetch tile 0's
    for (int q = 0; q < 2 * G::RA; q += 32) {
      load32(q);
      stage32(q);
    }
    load32(2 * G::RA);
    int base = 0;  // ring slot of the current tile's first window position
    for (int t = 0; t < nt; ++t) {
      stage32(2 * G::RA + kTcNT * t);
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      if (!__syncthreads_and(mine)) {
        ok = false;
        break;
      }
      if (m == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        int slot = base;
#pragma unroll
        for (int ks = 0; ks < G::KS; ++ks) {
          const uint64_t bo = (uint64_t)(ks * 16);   // 256 bytes per k-step, in 16-byte units
          const uint64_t ao = (uint64_t)(slot * 2);  // slot / 4 core columns of 128 bytes
          mma_ts(tm + G::DCOL, tm + slot, bhi_d + bo, kIdesc, ks > 0);
          mma_ts(tm + G::DCOL, tm + slot, blo_d + bo, kIdesc, 1);
          mma_ss(tm + G::DCOL, alo_d + ao, bhi_d + bo, kIdesc, 1);
          slot = slot + 8 >= G::W ? slot + 8 - G::W : slot + 8;
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar_a)
                     : "memory");
      }
      if (t + 1 < nt) load32(2 * G::RA + kTcNT * (t + 1));
      mine = mbar_wait(mbar_a, parity) && mine;
      parity ^= 1u;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      float r[32];
      tmem_ld32(tlane + G::DCOL, r);
      const int pt = p0 + kTcNT * t;  // absolute position of output 0 of the tile
      const int nlo = max(0, a_lo - pt), nhi = min(kTcNT, a_end - pt);  // stored outputs [nlo, nhi)
      const int64_t off = pt - a_lo;
      if (XAXIS) {
#pragma unroll
        for (int n = 0; n < 32; ++n) sT[m * G::T_STRIDE + n] = r[n];
        __syncwarp();
        const bool col = lane >= nlo && lane < nhi;
#pragma unroll 8
        for (int i = 0; i < 32; ++i) {
          float* rd = sDst[32 * w + i];
          if (rd && col) rd[off + lane] = sT[(32 * w + i) * G::T_STRIDE + lane];
        }
        __syncwarp();
      } else if (lok) {
        float* d = dst + off * ostride;
        if (nlo == 0 && nhi == kTcNT) {
#pragma unroll
          for (int n = 0; n < 32; ++n) d[n * ostride] = r[n];
        } else {
#pragma unroll
          for (int n = 0; n < 32; ++n)
            if (n >= nlo && n < nhi) d[n * ostride] = r[n];
        }
      }
      base = base + kTcNT >= G::W ? base + kTcNT - G::W : base + kTcNT;
    }
  }
  // a CTA whose MMAs did not complete waits once more (bounded) before it
  // releases the tensor memory they write, and reports itself
  ok = __syncthreads_and(ok && mine);
  if (!ok) {
    mbar_wait(mbar_a, parity ^ 1u);
    if (m == 0) atomicAdd(&g_tc_timeouts, 1u);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (w == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm), "n"(G::TCOLS));
}

template <int RR, bool XAXIS>
struct TcLaunch {
  static int ctas_per_sm;  // resident CTAs per SM (0 until prepared)
  static cudaError_t prepare() {
    if (ctas_per_sm > 0) return cudaSuccess;
    const int smem = TcGeom<RR>::smem(XAXIS);
    cudaError_t e = cudaFuncSetAttribute(k_rho_tc<RR, XAXIS>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_rho_tc<RR, XAXIS>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_rho_tc<RR, XAXIS>);
    int dev = 0, smem_sm = 0, regs_sm = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    if (e != cudaSuccess) return e;
    // resident CTAs: shared memory (1 KB reserved per CTA), registers (allocated
    // in units of 8 per thread) and tensor memory, whichever binds first
    const int by_smem = smem_sm / (smem + (int)fa.sharedSizeBytes + 1024);
    const int by_regs = regs_sm / (((fa.numRegs + 7) / 8 * 8) * kTcThreads);
    ctas_per_sm = std::max(1, std::min(std::min(by_smem, by_regs), TcGeom<RR>::MAX_CTAS));
    return cudaSuccess;
  }
  static cudaError_t run(const float* in, const Box& ib, const int dims[3], float* out, const Box& ob, int axis,
                         const Taps& taps, cudaStream_t st) {
    cudaError_t e = prepare();
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int64_t cap = (int64_t)sms * ctas_per_sm;
    const int a_n = ob.lo[axis] + ob.n[axis] - (ob.lo[axis] & ~(kTcNT - 1));  // aligned extent
    const int64_t groups = axis == 0 ? (6 * (int64_t)ob.n[1] * ob.n[2] + kTcThreads - 1) / kTcThreads
                                     : 6 * (int64_t)ob.n[3 - axis] * ((ob.n[0] + kTcThreads - 1) / kTcThreads);
    int seg = 512;  // outputs per unit: long enough to amortise the ring fill, short enough to spread
    while (seg > kTcNT && groups * ((a_n + seg - 1) / seg) < 2 * cap) seg /= 2;
    const int64_t units = groups * ((a_n + seg - 1) / seg);
    const int grid = (int)std::min<int64_t>(units, cap);
    k_rho_tc<RR, XAXIS><<<grid, kTcThreads, TcGeom<RR>::smem(XAXIS), st>>>(in, ib, dims[axis], out, ob, axis, seg,
                                                                          taps);
    return cudaGetLastError();
  }
};
template <int RR, bool XAXIS>
int TcLaunch<RR, XAXIS>::ctas_per_sm = 0;

template <int RR>
cudaError_t run_tc(const float* in, const Box& ib, const int dims[3], float* out, const Box& ob, int axis,
                   const Taps& taps, cudaStream_t st) {
  return axis == 0 ? TcLaunch<RR, true>::run(in, ib, dims, out, ob, axis, taps, st)
                   : TcLaunch<RR, false>::run(in, ib, dims, out, ob, axis, taps, st);
}

template <int RR>
cudaError_t prepare_tc() {
  cudaError_t e = TcLaunch<RR, true>::prepare();
  return e == cudaSuccess ? TcLaunch<RR, false>::prepare() : e;
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
                          const Taps& taps, int rk, cudaStream_t st) {
  if (box_vox(ob) == 0) return cudaSuccess;
  if (axis < 0 || axis > 2) return cudaErrorInvalidValue;
  switch (rk) {
    case 4: return run_tc<4>(in, ib, dims, out, ob, axis, taps, st);
    case 6: return run_tc<6>(in, ib, dims, out, ob, axis, taps, st);
    case 8: return run_tc<8>(in, ib, dims, out, ob, axis, taps, st);
    case 12: return run_tc<12>(in, ib, dims, out, ob, axis, taps, st);
    case 16: return run_tc<16>(in, ib, dims, out, ob, axis, taps, st);
    case 24: return run_tc<24>(in, ib, dims, out, ob, axis, taps, st);
    case 32: return run_tc<32>(in, ib, dims, out, ob, axis, taps, st);
    case 36: return run_tc<36>(in, ib, dims, out, ob, axis, taps, st);
    default: return cudaErrorInvalidValue;
  }
}

unsigned int tc_timeouts(bool reset) {
  unsigned int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_tc_timeouts, sizeof v) != cudaSuccess) return 0;
  if (reset && v) {
    const unsigned int z = 0;
    cudaMemcpyToSymbol(g_tc_timeouts, &z, sizeof z);
  }
  return v;
}

}  // namespace ct
