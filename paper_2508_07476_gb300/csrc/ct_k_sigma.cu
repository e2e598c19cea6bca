// Gradient at noise scale sigma and the six tensor products (Figure 1b;
// Architecture, "orientation"), fused in one z-streaming kernel so that the
// gradient never leaves the SM.
//
// A CTA owns a 32 x 16 (x, y) tile of output columns and walks a z segment.
// For every input plane it stages the haloed plane in shared memory, applies
// the x pass (smoothing w and derivative c, each +k/-k pair folded) and the y
// pass (three fields) in shared memory, and feeds the three results into
// per-thread register windows of 2R+1 planes that apply the z pass.  The
// window index is static because the plane loop is unrolled by the window
// length.  Output: the products g_a g_b as 6 FP32 planes.
#include "ct_common.cuh"
#include "ct_launch.h"

namespace ct {

constexpr int kSigTX = 32;
#ifndef CT_SIG_TY
#define CT_SIG_TY 16
#endif
constexpr int kSigTY = CT_SIG_TY;
constexpr int kSigThreads = kSigTX * kSigTY;
#ifndef CT_SIG_PREFETCH
#define CT_SIG_PREFETCH 4
#endif
constexpr int kSigPrefetch = CT_SIG_PREFETCH;  // planes ahead for the L2 prefetch hint
#ifndef CT_SIG_ZSEG
#define CT_SIG_ZSEG 256
#endif

template <int RS>
struct SigmaGeom {
  static constexpr int RX = kSigTX + 2 * RS;  // raw plane columns
  static constexpr int RY = kSigTY + 2 * RS;  // raw plane rows
  static constexpr int NRAW = RX * RY;
  static constexpr int NLOAD = (NRAW + kSigThreads - 1) / kSigThreads;
  static constexpr int NPAIR = RY * (kSigTX / 2);  // x-pass work items (2 columns each)
  static constexpr int P = 2 * RS + 1;             // z window
  // cp.async staging of interior tiles: rows of CW uint16 from x0 - XA (16-byte chunks)
  static constexpr int XA = (RS + 7) / 8 * 8;
  static constexpr int CW = kSigTX + 2 * XA;
  static constexpr int NCH = RY * (CW / 8);  // 16-byte chunks per plane
  // dynamic shared memory: raw[2][RY][RX] f32 | pwc[2][RY][TX] f32x2 | ring[3][RY][CW] u16
  static constexpr size_t RAW_B = sizeof(float) * 2 * RY * RX;
  static constexpr size_t PWC_B = sizeof(float2) * 2 * RY * kSigTX;
  static constexpr size_t RING_B = sizeof(uint16_t) * 3 * RY * CW;
  static constexpr size_t SMEM = RAW_B + PWC_B + RING_B;
};

// 2^-8 keeps every possible gradient of uint16 data inside FP16's range while
// leaving gradients down to 2^-6 intensity units normal.
constexpr float kHalfScale = 1.0f / 256.0f;

template <int RS, bool MIXED>
__global__ void __launch_bounds__(kSigThreads, 512 / kSigThreads)
    k_grad_products(const uint16_t* __restrict__ vol, Box vb, int dimx, int dimy, int dimz, float* __restrict__ J,
                    Box ob, int zseg, const Taps taps) {
  using G = SigmaGeom<RS>;
  extern __shared__ __align__(16) unsigned char sig_smem[];
  auto raw = reinterpret_cast<float(*)[G::RY][G::RX]>(sig_smem);
  auto pwc = reinterpret_cast<float2(*)[G::RY][kSigTX]>(sig_smem + G::RAW_B);  // x pass: (smoothed, derivative)
  auto ring = reinterpret_cast<uint16_t(*)[G::RY][G::CW]>(sig_smem + G::RAW_B + G::PWC_B);  // cp.async landing

  const int t = threadIdx.x;
  const int tx = t % kSigTX, ty = t / kSigTX;
  const int x0 = ob.lo[0] + blockIdx.x * kSigTX;
  const int y0 = ob.lo[1] + blockIdx.y * kSigTY;
  const int zs = ob.lo[2] + blockIdx.z * zseg;
  const int ze = min(zs + zseg, ob.lo[2] + ob.n[2]);
  const int nsteps = (ze - zs) + 2 * RS;
  const int64_t nob = box_vox(ob);

  // per-thread raw-plane load slots: (row, col) -> clamped global (x, y)
  int64_t loff[G::NLOAD];
  bool lval[G::NLOAD];
#pragma unroll
  for (int i = 0; i < G::NLOAD; ++i) {
    int e = t + i * kSigThreads;
    lval[i] = e < G::NRAW;
    int row = lval[i] ? e / G::RX : 0, col = lval[i] ? e % G::RX : 0;
    int gx = clamp_to(x0 - RS + col, dimx, vb.lo[0], vb.n[0]);
    int gy = clamp_to(y0 - RS + row, dimy, vb.lo[1], vb.n[1]);
    loff[i] = (int64_t)(gy - vb.lo[1]) * vb.n[0] + (gx - vb.lo[0]);
  }
  const int64_t plane = (int64_t)vb.n[0] * vb.n[1];
  auto plane_base = [&](int s) -> int64_t {
    int gz = clamp_to(zs - RS + s, dimz, vb.lo[2], vb.n[2]);
    return (int64_t)(gz - vb.lo[2]) * plane;
  };

  // Interior tiles (no clamping in x or y, 16-byte aligned rows) stream their
  // raw planes with cp.async two planes ahead; edge tiles load through registers.
  const bool interior = x0 - G::XA >= max(0, vb.lo[0]) && x0 + kSigTX + G::XA <= min(dimx, vb.lo[0] + vb.n[0]) &&
                        y0 - RS >= max(0, vb.lo[1]) && y0 + kSigTY + RS <= min(dimy, vb.lo[1] + vb.n[1]) &&
                        (vb.n[0] % 8) == 0 && ((x0 - G::XA - vb.lo[0]) % 8) == 0 &&
                        ((reinterpret_cast<uintptr_t>(vol) & 15) == 0);
  const uint32_t ring0 = (uint32_t)__cvta_generic_to_shared(&ring[0][0][0]);
  // Fixed per-thread parts of the per-plane work: this thread's 16-byte chunk
  // of a staged plane (source offset within a plane, landing offset within a
  // ring slot), the ring elements it converts, and the line it prefetches.
  const int ich_row = t / (G::CW / 8), ich_cq = t % (G::CW / 8);
  const int64_t ich_src = (int64_t)(y0 - RS + ich_row - vb.lo[1]) * vb.n[0] + (x0 - G::XA - vb.lo[0]) + 8 * ich_cq;
  const uint32_t ich_dst = (uint32_t)(ich_row * G::CW + 8 * ich_cq) * 2u;
  int cv_src[G::NLOAD];  // element of a ring slot converted into raw element t + i * threads (-1: none)
#pragma unroll
  for (int i = 0; i < G::NLOAD; ++i) {
    const int e = t + i * kSigThreads;
    cv_src[i] = lval[i] ? (e / G::RX) * G::CW + (e % G::RX) + G::XA - RS : -1;
  }
  int64_t pf_off = -1;  // first or last column of one staged row
  if (t < 2 * G::RY) {
    const int gx = clamp_to(x0 - RS + ((t & 1) ? G::RX - 1 : 0), dimx, vb.lo[0], vb.n[0]);
    const int gy = clamp_to(y0 - RS + (t >> 1), dimy, vb.lo[1], vb.n[1]);
    pf_off = (int64_t)(gy - vb.lo[1]) * vb.n[0] + (gx - vb.lo[0]);
  }
  auto issue_plane = [&](int s) {  // cp.async of plane s into ring slot s % 3
    if (s < nsteps && t < G::NCH) {
      const uint16_t* src = vol + plane_base(s) + ich_src;
      const uint32_t dst = ring0 + (uint32_t)((s % 3) * G::RY * G::CW) * 2u + ich_dst;
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
    }
    cp_async_commit();
  };
  auto convert_plane = [&](int s, int slot_raw) {  // ring slot s % 3 -> raw[slot_raw] as float
    const uint16_t* rs = &ring[s % 3][0][0];
    float* rd = &raw[slot_raw][0][0];
#pragma unroll
    for (int i = 0; i < G::NLOAD; ++i)
      if (cv_src[i] >= 0) rd[t + i * kSigThreads] = (float)rs[cv_src[i]];
  };

  // x pass of the staged plane in raw[rb] into pwc[rb]: smoothing and derivative
  auto xpass_item = [&](int rb, int item) {
    {
      const int row = item / (kSigTX / 2);
      const int c0 = 2 * (item % (kSigTX / 2));
      const float* rr = &raw[rb][row][c0];
      float xv[2 * RS + 2];
#pragma unroll
      for (int k = 0; k < RS + 1; ++k) {
        float2 v2 = *reinterpret_cast<const float2*>(rr + 2 * k);
        xv[2 * k] = v2.x;
        xv[2 * k + 1] = v2.y;
      }
      float sw0 = taps.w[RS] * xv[RS], sw1 = taps.w[RS] * xv[RS + 1];
      float sc0 = 0.f, sc1 = 0.f;
#pragma unroll
      for (int k = 1; k <= RS; ++k) {
        sw0 = fmaf(taps.w[RS + k], xv[RS + k] + xv[RS - k], sw0);
        sw1 = fmaf(taps.w[RS + k], xv[RS + 1 + k] + xv[RS + 1 - k], sw1);
        sc0 = fmaf(taps.c[RS + k], xv[RS + k] - xv[RS - k], sc0);
        sc1 = fmaf(taps.c[RS + k], xv[RS + 1 + k] - xv[RS + 1 - k], sc1);
      }
      *reinterpret_cast<float4*>(&pwc[rb][row][c0]) = make_float4(sw0, sc0, sw1, sc1);
    }
  };
  // One item per thread when the items match the threads exactly (straight-line
  // code the compiler can interleave with the y and z passes), else a loop.
  auto xpass = [&](int rb) {
    if constexpr (G::NPAIR == kSigThreads) {
      xpass_item(rb, t);
    } else {
      for (int item = t; item < G::NPAIR; item += kSigThreads) xpass_item(rb, item);
    }
  };
  float pre[G::NLOAD];
  auto load_pre = [&](int s) {  // edge tiles: plane s into registers
    const int64_t bs = plane_base(s);
#pragma unroll
    for (int i = 0; i < G::NLOAD; ++i) pre[i] = lval[i] ? (float)__ldg(vol + bs + loff[i]) : 0.f;
  };
  auto store_pre = [&](int rb) {
#pragma unroll
    for (int i = 0; i < G::NLOAD; ++i)
      if (lval[i]) (&raw[rb][0][0])[t + i * kSigThreads] = pre[i];
  };

  // Software pipeline, one barrier per plane: step s runs the x pass of plane
  // s + 1 and the y and z passes of plane s (independent work), stages plane
  // s + 2 and issues the copy of plane s + 4.
  if (interior) {
    issue_plane(0);
    issue_plane(1);
    issue_plane(2);
    cp_async_wait<1>();
    __syncthreads();
    convert_plane(0, 0);
    if (1 < nsteps) convert_plane(1, 1);
    __syncthreads();
    xpass(0);
    issue_plane(3);  // into the slot of plane 0
    cp_async_wait<1>();
    __syncthreads();
  } else {
    load_pre(0);
    store_pre(0);
    if (1 < nsteps) {
      load_pre(1);
      store_pre(1);
    }
    if (2 < nsteps) load_pre(2);
    __syncthreads();
    xpass(0);
    __syncthreads();
  }

  // z windows of the three y-pass results: (c_x w_y), (w_x c_y), (w_x w_y)
  float wgx[G::P], wgy[G::P], wgz[G::P];
#pragma unroll
  for (int i = 0; i < G::P; ++i) { wgx[i] = 0.f; wgy[i] = 0.f; wgz[i] = 0.f; }

  const int ox = x0 + tx, oy = y0 + ty;
  const bool store_ok = ox < ob.lo[0] + ob.n[0] && oy < ob.lo[1] + ob.n[1];
  const int64_t out_xy = (int64_t)(oy - ob.lo[1]) * ob.n[0] + (ox - ob.lo[0]);

  for (int base = 0; base < nsteps; base += G::P) {
#pragma unroll
    for (int u = 0; u < G::P; ++u) {
      const int s = base + u;
      if (s >= nsteps) continue;
      const int b = s & 1;
      if (s + 1 < nsteps) xpass(b ^ 1);
      // y pass of plane s for this thread's column
      const float2 c0v = pwc[b][ty + RS][tx];
      float qww = taps.w[RS] * c0v.x;
      float qcw = taps.w[RS] * c0v.y;
      float qwc = 0.f;
#pragma unroll
      for (int k = 1; k <= RS; ++k) {
        const float2 pp = pwc[b][ty + RS + k][tx], pm = pwc[b][ty + RS - k][tx];
        qww = fmaf(taps.w[RS + k], pp.x + pm.x, qww);
        qwc = fmaf(taps.c[RS + k], pp.x - pm.x, qwc);
        qcw = fmaf(taps.w[RS + k], pp.y + pm.y, qcw);
      }
      // push into the z windows (slot u: base is a multiple of P)
      wgx[u] = qcw;
      wgy[u] = qwc;
      wgz[u] = qww;
      if (s >= 2 * RS) {
        // window slot of offset k (-RS..RS) relative to the output plane
        float gx = taps.w[RS] * wgx[(u + G::P - RS) % G::P];
        float gy = taps.w[RS] * wgy[(u + G::P - RS) % G::P];
        float gz = 0.f;
#pragma unroll
        for (int k = 1; k <= RS; ++k) {
          const int sp = (u + G::P - RS + k) % G::P;
          const int sm = (u + G::P - RS - k) % G::P;
          gx = fmaf(taps.w[RS + k], wgx[sp] + wgx[sm], gx);
          gy = fmaf(taps.w[RS + k], wgy[sp] + wgy[sm], gy);
          gz = fmaf(taps.c[RS + k], wgz[sp] - wgz[sm], gz);
        }
        if (MIXED) {  // gradient held in FP16 (scaled), products formed exactly in FP32
          gx = __half2float(__float2half_rn(gx * kHalfScale)) * (1.0f / kHalfScale);
          gy = __half2float(__float2half_rn(gy * kHalfScale)) * (1.0f / kHalfScale);
          gz = __half2float(__float2half_rn(gz * kHalfScale)) * (1.0f / kHalfScale);
        }
        const int oz = zs + s - 2 * RS;
        if (store_ok) {
          const int64_t o = (int64_t)(oz - ob.lo[2]) * ob.n[0] * ob.n[1] + out_xy;
          J[o] = gx * gx;
          J[nob + o] = gy * gy;
          J[2 * nob + o] = gz * gz;
          J[3 * nob + o] = gx * gy;
          J[4 * nob + o] = gx * gz;
          J[5 * nob + o] = gy * gz;
        }
      }
      // stage plane s + 2 into raw[b] (last read by the x pass of plane s)
      if (interior) {
        if (s + 2 < nsteps) convert_plane(s + 2, b);
        issue_plane(s + 4);  // into the slot of plane s + 1, converted one step ago
      } else {
        if (s + 2 < nsteps) store_pre(b);
        if (s + 3 < nsteps) load_pre(s + 3);
      }
      if (kSigPrefetch > 0 && s + kSigPrefetch < nsteps && pf_off >= 0)  // warm L2 for a later plane (a hint)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(vol + plane_base(s + kSigPrefetch) + pf_off));
      if (interior) cp_async_wait<1>();  // plane s + 3 landed (this thread's chunks)
      __syncthreads();
    }
  }
  cp_async_wait<0>();
}

template <int RS>
static cudaError_t launch_grad_rs(const uint16_t* vol, const Box& vb, const int dims[3], float* J, const Box& ob,
                                  const Taps& taps, bool mixed, cudaStream_t st) {
  using G = SigmaGeom<RS>;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_grad_products<RS, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)G::SMEM);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_grad_products<RS, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)G::SMEM);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int zseg = CT_SIG_ZSEG;
  dim3 grid((ob.n[0] + kSigTX - 1) / kSigTX, (ob.n[1] + kSigTY - 1) / kSigTY, (ob.n[2] + zseg - 1) / zseg);
  if (mixed)
    k_grad_products<RS, true><<<grid, kSigThreads, G::SMEM, st>>>(vol, vb, dims[0], dims[1], dims[2], J, ob, zseg,
                                                                   taps);
  else
    k_grad_products<RS, false><<<grid, kSigThreads, G::SMEM, st>>>(vol, vb, dims[0], dims[1], dims[2], J, ob, zseg,
                                                                    taps);
  return cudaGetLastError();
}

template <int RS>
static cudaError_t prepare_rs() {
  using G = SigmaGeom<RS>;
  cudaError_t e = cudaFuncSetAttribute(k_grad_products<RS, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)G::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_grad_products<RS, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM);
  return e;
}

cudaError_t prepare_sigma_kernels() {
  cudaError_t e = prepare_rs<2>();
  if (e == cudaSuccess) e = prepare_rs<3>();
  if (e == cudaSuccess) e = prepare_rs<4>();
  if (e == cudaSuccess) e = prepare_rs<6>();
  if (e == cudaSuccess) e = prepare_rs<8>();
  if (e == cudaSuccess) e = prepare_rs<12>();
  return e;
}

int sigma_kernel_radius(int r) {
  static const int radii[] = {2, 3, 4, 6, 8, 12};
  for (int v : radii)
    if (r <= v) return v;
  return -1;
}

cudaError_t launch_grad_products(const uint16_t* vol, const Box& vb, const int dims[3], float* J, const Box& ob,
                                 const Taps& taps, int rk, bool mixed, cudaStream_t st) {
  if (box_vox(ob) == 0) return cudaSuccess;
  switch (rk) {
    case 2: return launch_grad_rs<2>(vol, vb, dims, J, ob, taps, mixed, st);
    case 3: return launch_grad_rs<3>(vol, vb, dims, J, ob, taps, mixed, st);
    case 4: return launch_grad_rs<4>(vol, vb, dims, J, ob, taps, mixed, st);
    case 6: return launch_grad_rs<6>(vol, vb, dims, J, ob, taps, mixed, st);
    case 8: return launch_grad_rs<8>(vol, vb, dims, J, ob, taps, mixed, st);
    case 12: return launch_grad_rs<12>(vol, vb, dims, J, ob, taps, mixed, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ct
