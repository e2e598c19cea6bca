// The last smoothing pass (rho along z) fused with the eigen-decomposition and
// the cardiac descriptors (Figure 1b,c), so the finished tensor never goes to
// HBM.
//
// A CTA owns 32 x-columns of one (y) row for all six components (192 threads,
// one warp per component) and walks a z segment in blocks of kZT outputs, with
// the register window and cp.async ring of the streaming pass.  After each
// block the six components of the kZT x 32 voxels sit in shared memory; after
// one barrier every thread solves two of those voxels and writes their outputs.
// Near-degenerate voxels go to a compact list that carries their tensor (it is
// not stored anywhere else); if the list is full the voxel is re-solved in
// place.
#include "ct_common.cuh"
#include "ct_launch.h"

namespace ct {

constexpr int kZX = 32;               // x columns per CTA
constexpr int kZT = 12;               // z outputs per block
constexpr int kZThreads = 6 * kZX;    // 192
static_assert((kZT * kZX) % kZThreads == 0, "voxels of a block must split evenly");
constexpr int kZVox = (kZT * kZX) / kZThreads;  // voxels per thread per block (2)

// Robust re-solve (FP32 Jacobi, or FP64 closed form / Jacobi in the mixed form).
__device__ __noinline__ void resolve_voxel(const Sym3<float>& s, bool mixed, float l[3], float v[3]) {
  if (mixed) {
    Sym3<double> sd{(double)s.a, (double)s.b, (double)s.c, (double)s.d, (double)s.e, (double)s.f};
    double ld[3], vd[3];
    if (!eig_closed<double>(sd, ld, vd)) eig_jacobi<double>(sd, ld, vd);
    for (int k = 0; k < 3; ++k) {
      l[k] = (float)ld[k];
      v[k] = (float)vd[k];
    }
  } else {
    eig_jacobi<float>(s, l, v);
  }
  float nv = rsqrtf(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  v[0] *= nv; v[1] *= nv; v[2] *= nv;
}

// TY: compile-time encoding of all outputs (CT_OUT_F32 = 0), or -1 for the
// run-time encodings in `o`.
template <int TY = -1>
__device__ __forceinline__ void emit(const EigOut& o, int64_t oi, bool inside, const Frame& F, int x, int y, int z,
                                     const float l[3], float v[3], float fill) {
  const int64_t n = box_vox(o.ab);
  if (!inside) {
    if (o.vec) {
      store_val<TY>(o.vec, oi, o.vec_t, fill);
      store_val<TY>(o.vec, n + oi, o.vec_t, fill);
      store_val<TY>(o.vec, 2 * n + oi, o.vec_t, fill);
    }
    store_angle<TY>(o.ha, oi, o.ang_t, fill, false);
    store_angle<TY>(o.ia, oi, o.ang_t, fill, false);
    store_val<TY>(o.fa, oi, o.fa_t, fill);
    return;
  }
  float ha, ia;
  const bool framed = ha_ia(F, x, y, z, v, ha, ia);
  if (!framed) orient_largest(v);
  if (o.vec) {
    store_val<TY>(o.vec, oi, o.vec_t, v[0]);
    store_val<TY>(o.vec, n + oi, o.vec_t, v[1]);
    store_val<TY>(o.vec, 2 * n + oi, o.vec_t, v[2]);
  }
  store_angle<TY>(o.ha, oi, o.ang_t, framed ? ha : fill, framed);
  store_angle<TY>(o.ia, oi, o.ang_t, framed ? ia : fill, framed);
  store_val<TY>(o.fa, oi, o.fa_t, fa_of(l));
}

#ifndef CT_ZE_MINB
#define CT_ZE_MINB 1
#endif
template <int RR, int TY>
__global__ void __launch_bounds__(kZThreads, CT_ZE_MINB)
    k_rho_z_eig(const float* __restrict__ in, Box ib, int dimz, Box ob, const uint8_t* __restrict__ mask, Box mb,
                Frame F, float fill, EigOut o, bool mixed, FallbackS fb, int seg, const Taps taps) {
  constexpr int P = 2 * RR + 1;
  constexpr int WN = kZT + 2 * RR;
  __shared__ float ring[2 * kZT][kZThreads];
  __shared__ float sS[2][kZT][6][kZX];
  const int tid = threadIdx.x;
  const int xl = tid % kZX, comp = tid / kZX;
  const int xt0 = ob.lo[0] + blockIdx.x * kZX;  // first x of the CTA
  const int xend = ob.lo[0] + ob.n[0];
  const int y = ob.lo[1] + blockIdx.y;
  const int p0 = ob.lo[2] + blockIdx.z * seg;
  const int L = min(seg, ob.lo[2] + ob.n[2] - p0);
  if (L <= 0) return;
  const int xi = min(xt0 + xl, xend - 1);

  const float* base = in + comp * box_vox(ib) + box_index(ib, xi, y, ib.lo[2]);
  const int istride = ib.n[0] * ib.n[1];
  const int qlo = max(0, ib.lo[2]) - ib.lo[2], qhi = min(dimz - 1, ib.lo[2] + ib.n[2] - 1) - ib.lo[2];
  const int q0 = p0 - RR - ib.lo[2];
  auto src = [&](int step) -> const float* { return base + min(max(q0 + step, qlo), qhi) * istride; };
  const uint32_t ring0 = (uint32_t)__cvta_generic_to_shared(&ring[0][tid]);
  constexpr uint32_t kSlot = kZThreads * sizeof(float);

  float win[WN];
#pragma unroll
  for (int j = 0; j < 2 * RR; ++j) win[j] = __ldg(src(j));
#pragma unroll
  for (int h = 0; h < 2; ++h) {
#pragma unroll
    for (int t = 0; t < kZT; ++t) cp_async4(ring0 + (h * kZT + t) * kSlot, src(2 * RR + h * kZT + t));
    cp_async_commit();
  }
  const int nb = (L + kZT - 1) / kZT;
  for (int bk = 0; bk < nb; ++bk) {
    cp_async_wait<1>();
    const int half = (bk & 1) * kZT;
#pragma unroll
    for (int t = 0; t < kZT; ++t) win[2 * RR + t] = ring[half + t][tid];
    float (*dst)[6][kZX] = sS[bk & 1];
#pragma unroll
    for (int i = 0; i < kZT; ++i) {
      float acc = taps.w[0] * win[i];
#pragma unroll
      for (int k = 1; k < P; ++k) acc = fmaf(taps.w[k], win[i + k], acc);
      dst[i][comp][xl] = acc;
    }
#pragma unroll
    for (int t = 0; t < kZT; ++t) cp_async4(ring0 + (half + t) * kSlot, src(2 * RR + (bk + 2) * kZT + t));
    cp_async_commit();
#pragma unroll
    for (int j = 0; j < 2 * RR; ++j) win[j] = win[j + kZT];
    __syncthreads();  // the block's tensors are complete
#pragma unroll 1
    for (int h = 0; h < kZVox; ++h) {
      const int vi = tid + h * kZThreads;
      const int t = vi / kZX, xv = vi % kZX;
      const int x = xt0 + xv, z = p0 + bk * kZT + t;
      if (bk * kZT + t >= L || x >= xend) continue;
      const bool inside = mask == nullptr || __ldg(mask + box_index(mb, x, y, z)) != 0;
      float l[3] = {0.f, 0.f, 0.f}, v[3] = {1.f, 0.f, 0.f};
      if (inside) {
        Sym3<float> s{dst[t][0][xv], dst[t][1][xv], dst[t][2][xv], dst[t][3][xv], dst[t][4][xv], dst[t][5][xv]};
        if (!eig_closed<float>(s, l, v)) {
          atomicAdd(fb.total, 1ull);
          const int slot = atomicAdd(fb.count, 1);
          if (slot < fb.cap) {
            fb.idx[slot] = box_index(ob, x, y, z);
            float* e = fb.S + 6 * (int64_t)slot;
            e[0] = s.a; e[1] = s.b; e[2] = s.c; e[3] = s.d; e[4] = s.e; e[5] = s.f;
          } else {
            resolve_voxel(s, mixed, l, v);
          }
        }
      }
      emit<TY>(o, box_index(o.ab, x, y, z), inside, F, x, y, z, l, v, fill);
    }
  }
  cp_async_wait<0>();
}

__global__ void __launch_bounds__(128)
    k_fallback_s(Box ob, Frame F, float fill, EigOut o, bool mixed, FallbackS fb) {
  const int64_t cnt = min((int64_t)*fb.count, fb.cap);
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < cnt; j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = fb.idx[j];
    const int x = ob.lo[0] + (int)(i % ob.n[0]);
    const int y = ob.lo[1] + (int)((i / ob.n[0]) % ob.n[1]);
    const int z = ob.lo[2] + (int)(i / ((int64_t)ob.n[0] * ob.n[1]));
    const float* e = fb.S + 6 * j;
    Sym3<float> s{e[0], e[1], e[2], e[3], e[4], e[5]};
    float l[3], v[3];
    resolve_voxel(s, mixed, l, v);
    emit(o, box_index(o.ab, x, y, z), true, F, x, y, z, l, v, fill);
  }
}

template <int RR>
static cudaError_t launch_rzeig_r(const float* in, const Box& ib, const int dims[3], const Box& ob,
                                  const uint8_t* mask, const Box& mb, const Frame& F, float fill, const EigOut& o,
                                  bool mixed, const FallbackS& fb, const Taps& taps, cudaStream_t st) {
  if (box_vox(ib) >= ((int64_t)1 << 31)) return cudaErrorInvalidValue;
  const int64_t ctas = (int64_t)((ob.n[0] + kZX - 1) / kZX) * ob.n[1];
  int nseg = 1;
  while (nseg < 16 && ctas * nseg < (int64_t)152 * 3 * 4 && ob.n[2] / (nseg * 2) >= 4 * (2 * RR + 1)) nseg *= 2;
  const int seg = (ob.n[2] + nseg - 1) / nseg;
  dim3 grid((ob.n[0] + kZX - 1) / kZX, ob.n[1], (ob.n[2] + seg - 1) / seg);
  if (grid.y > 65535 || grid.z > 65535) return cudaErrorInvalidValue;
  if (o.vec_t == 0 && o.ang_t == 0 && o.fa_t == 0)
    k_rho_z_eig<RR, 0><<<grid, kZThreads, 0, st>>>(in, ib, dims[2], ob, mask, mb, F, fill, o, mixed, fb, seg, taps);
  else
    k_rho_z_eig<RR, -1><<<grid, kZThreads, 0, st>>>(in, ib, dims[2], ob, mask, mb, F, fill, o, mixed, fb, seg, taps);
  return cudaGetLastError();
}

cudaError_t launch_rho_z_eig(const float* in, const Box& ib, const int dims[3], const Box& ob, const uint8_t* mask,
                             const Box& mb, const Frame& F, float fill, const EigOut& o, bool mixed,
                             const FallbackS& fb, const Taps& taps, int rk, cudaStream_t st) {
  if (box_vox(ob) == 0) return cudaSuccess;
  switch (rk) {
    case 4: return launch_rzeig_r<4>(in, ib, dims, ob, mask, mb, F, fill, o, mixed, fb, taps, st);
    case 6: return launch_rzeig_r<6>(in, ib, dims, ob, mask, mb, F, fill, o, mixed, fb, taps, st);
    case 8: return launch_rzeig_r<8>(in, ib, dims, ob, mask, mb, F, fill, o, mixed, fb, taps, st);
    case 12: return launch_rzeig_r<12>(in, ib, dims, ob, mask, mb, F, fill, o, mixed, fb, taps, st);
    case 16: return launch_rzeig_r<16>(in, ib, dims, ob, mask, mb, F, fill, o, mixed, fb, taps, st);
    case 24: return launch_rzeig_r<24>(in, ib, dims, ob, mask, mb, F, fill, o, mixed, fb, taps, st);
    case 32: return launch_rzeig_r<32>(in, ib, dims, ob, mask, mb, F, fill, o, mixed, fb, taps, st);
    case 36: return launch_rzeig_r<36>(in, ib, dims, ob, mask, mb, F, fill, o, mixed, fb, taps, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_fallback_s(const Box& ob, const Frame& F, float fill, const EigOut& o, bool mixed,
                              const FallbackS& fb, int64_t max_items, cudaStream_t st) {
  if (max_items <= 0) return cudaSuccess;
  int64_t b = (max_items + 127) / 128;
  int grid = (int)(b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : b));
  k_fallback_s<<<grid, 128, 0, st>>>(ob, F, fill, o, mixed, fb);
  return cudaGetLastError();
}

}  // namespace ct
