// Eigen-decomposition of the structure tensor and the cardiac descriptors
// (Figure 1b: smallest-eigenvalue eigenvector as the fibre direction;
// Figure 1c: HA, IA, FA in the cylindrical left-ventricle frame; Figure 1a:
// optional myocardial mask).
//
// Every voxel first takes the FP32 closed form (trigonometric roots of the
// characteristic cubic, cross product of two rows of S - l1 I).  Voxels whose
// two smallest eigenvalues nearly coincide, where that form loses half of its
// digits, are appended to a compact list and re-solved by a second kernel:
// FP32 cyclic Jacobi in the FP32 form, FP64 closed form (FP64 Jacobi if that
// too is near-degenerate) in the mixed form.  The list keeps the re-solve off
// the common path, so no warp diverges into it.
#include <algorithm>

#include "ct.h"
#include "ct_common.cuh"
#include "ct_launch.h"

namespace ct {

__device__ __forceinline__ Sym3<float> load_sym(const float* S, int64_t n, int64_t i) {
  Sym3<float> s;
  s.a = __ldg(S + i);
  s.b = __ldg(S + n + i);
  s.c = __ldg(S + 2 * n + i);
  s.d = __ldg(S + 3 * n + i);
  s.e = __ldg(S + 4 * n + i);
  s.f = __ldg(S + 5 * n + i);
  return s;
}

// Robust re-solve of one voxel.
__device__ __forceinline__ void resolve(const Sym3<float>& s, bool mixed, float l[3], float v[3]) {
  if (mixed) {
    Sym3<double> sd{(double)s.a, (double)s.b, (double)s.c, (double)s.d, (double)s.e, (double)s.f};
    double ld[3], vd[3];
    if (!eig_closed<double>(sd, ld, vd, kDegenerateGap64)) eig_jacobi<double>(sd, ld, vd);
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

// Outputs of one voxel: oriented vector, HA, IA, FA (or fill outside the mask).
// VT / AT / FT: compile-time encodings of the vector / angle / FA outputs, or
// -1 to take them from `o` at run time.
template <int VT = -1, int AT = -1, int FT = -1, typename IT = int64_t, bool PLAIN = false>
__device__ __forceinline__ void write_voxel(const EigOut& o, IT oi, bool inside, const Frame& F, int x, int y,
                                            int z, const float l[3], float v[3], float fill) {
  const IT n = (IT)box_vox(o.ab);
  if (!inside) {
    store_val<VT, IT>(o.vec, oi, o.vec_t, fill);
    if (o.vec) {
      store_val<VT, IT>(o.vec, n + oi, o.vec_t, fill);
      store_val<VT, IT>(o.vec, 2 * n + oi, o.vec_t, fill);
    }
    store_angle<AT, IT>(o.ha, oi, o.ang_t, fill, false);
    store_angle<AT, IT>(o.ia, oi, o.ang_t, fill, false);
    store_val<FT, IT>(o.fa, oi, o.fa_t, fill);
    return;
  }
  float ha, ia;
  bool framed = ha_ia<PLAIN>(F, x, y, z, v, ha, ia);
  if (!framed) orient_largest(v);
  if (o.vec) {
    store_val<VT, IT>(o.vec, oi, o.vec_t, v[0]);
    store_val<VT, IT>(o.vec, n + oi, o.vec_t, v[1]);
    store_val<VT, IT>(o.vec, 2 * n + oi, o.vec_t, v[2]);
  }
  store_angle<AT, IT>(o.ha, oi, o.ang_t, framed ? ha : fill, framed);
  store_angle<AT, IT>(o.ia, oi, o.ang_t, framed ? ia : fill, framed);
  store_val<FT, IT>(o.fa, oi, o.fa_t, fa_of(l));
}

__device__ __forceinline__ void push_fallback(const Fallback& fb, int64_t i) {
  int slot = atomicAdd(fb.count, 1);
  if (slot < fb.cap) fb.list[slot] = i;
  atomicAdd(fb.total, 1ull);
}

// One thread per voxel on a 3D grid (x from the thread index, y and z from the
// block index, rows beyond 65535 folded into blockIdx.z), so no index division.
// 8 CTAs of 256 threads per SM (32 registers): the kernel streams HBM and
// needs every resident warp to cover its latency.
#ifndef CT_EIG_MINB
#define CT_EIG_MINB 8
#endif
template <int VT, int AT, int FT>
__global__ void __launch_bounds__(256, CT_EIG_MINB)
    k_eig_angles(const float* __restrict__ S, Box sb, Box ob, const uint8_t* __restrict__ mask, Box mb, Frame F,
                 float fill, EigOut o, bool mixed, Fallback fb) {
  const int x = ob.lo[0] + blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= ob.lo[0] + ob.n[0]) return;
  const int row = blockIdx.z * gridDim.y + blockIdx.y;  // y + ny * z within ob
  if (row >= ob.n[1] * ob.n[2]) return;
  const int yr = row % ob.n[1], zr = row / ob.n[1];  // one division per thread, 32-bit
  const int y = ob.lo[1] + yr, z = ob.lo[2] + zr;
  const bool inside = mask == nullptr || __ldg(mask + box_index(mb, x, y, z)) != 0;
  float l[3] = {0.f, 0.f, 0.f}, v[3] = {1.f, 0.f, 0.f};
  if (inside) {
    const Sym3<float> s = load_sym(S, box_vox(sb), box_index(sb, x, y, z));
    if (!eig_closed<float>(s, l, v, fb.gap)) push_fallback(fb, ((int64_t)zr * ob.n[1] + yr) * ob.n[0] + (x - ob.lo[0]));
  }
  write_voxel<VT, AT, FT>(o, box_index(o.ab, x, y, z), inside, F, x, y, z, l, v, fill);
}

// The same for boxes whose planes fit 32-bit indices and whose rows fit the
// grid's y and z: (y, z) from the block index, every index in 32 bits.
__device__ __forceinline__ int box_index32(const Box& b, int x, int y, int z) {
  return ((z - b.lo[2]) * b.n[1] + (y - b.lo[1])) * b.n[0] + (x - b.lo[0]);
}

template <int VT, int AT, int FT, bool PLAIN, typename BLK>
__device__ __forceinline__ void eig32_body(const float* __restrict__ S, Box sb, Box ob,
                                           const uint8_t* __restrict__ mask, Box mb, const Frame& F, float fill,
                                           const EigOut& o, const Fallback& fb, const BLK blk) {
  const int x = ob.lo[0] + blk.x() * blockDim.x + threadIdx.x;
  if (x >= ob.lo[0] + ob.n[0]) return;
  const int y = ob.lo[1] + blk.y(), z = ob.lo[2] + blk.z();
  const bool inside = mask == nullptr || __ldg(mask + box_index32(mb, x, y, z)) != 0;
  float l[3] = {0.f, 0.f, 0.f}, v[3] = {1.f, 0.f, 0.f};
  if (inside) {
    const int ns = sb.n[0] * sb.n[1] * sb.n[2];
    const int si = box_index32(sb, x, y, z);
    Sym3<float> s;
    s.a = __ldg(S + si);
    s.b = __ldg(S + ns + si);
    s.c = __ldg(S + 2 * ns + si);
    s.d = __ldg(S + 3 * ns + si);
    s.e = __ldg(S + 4 * ns + si);
    s.f = __ldg(S + 5 * ns + si);
    if (!eig_closed<float>(s, l, v, fb.gap))
      push_fallback(fb, ((int64_t)blk.z() * ob.n[1] + blk.y()) * ob.n[0] + (x - ob.lo[0]));
  }
  write_voxel<VT, AT, FT, int, PLAIN>(o, box_index32(o.ab, x, y, z), inside, F, x, y, z, l, v, fill);
}

template <int VT, int AT, int FT, bool PLAIN>
__global__ void __launch_bounds__(256, CT_EIG_MINB)
    k_eig_angles32(const float* __restrict__ S, Box sb, Box ob, const uint8_t* __restrict__ mask, Box mb, Frame F,
                   float fill, EigOut o, bool mixed, Fallback fb) {
  (void)mixed;
  eig32_body<VT, AT, FT, PLAIN>(S, sb, ob, mask, mb, F, fill, o, fb, HwBlock{});
}

// The masked form: a CTA of kEigThreads threads takes kEigSpan consecutive
// voxels of one row (voxel x0 + t + kEigThreads k for thread t, so that the
// mask loads and the fill stores stay coalesced), writes the fill outputs of
// those outside the mask at once and lists the inside ones in shared memory,
// in x order (warp ballots; every warp scans the per-warp counts itself).
// The eigen solve then runs over the list, so that only the last warp of a row
// segment has idle lanes, where a warp per 32 voxels would idle wherever the
// wall boundary cuts it.  Each voxel's arithmetic is that of k_eig_angles32;
// only the thread that does it differs.
// Two-warp CTAs over 512 voxels: 32 CTAs per SM, whose barriers and list
// phases interleave (512^3: 0.97 ms, against 1.09 for 256 threads x 2 voxels,
// 1.01 for 128 x 4, 0.99 for 64 x 4, 1.04 for 64 x 16)
#ifndef CT_EIG_THREADS
#define CT_EIG_THREADS 64
#endif
#ifndef CT_EIG_SPAN_K
#define CT_EIG_SPAN_K 8
#endif
#ifndef CT_EIG_ILP
#define CT_EIG_ILP 1
#endif
constexpr int kEigThreads = CT_EIG_THREADS;        // threads per CTA (tuning choice)
constexpr int kEigSpanK = CT_EIG_SPAN_K;           // voxels per thread per segment (tuning choice)
constexpr int kEigSpan = kEigThreads * kEigSpanK;  // voxels per segment
constexpr int kEigIlp = CT_EIG_ILP;                // list entries per thread whose tensors load together (tuning choice)
constexpr int kEigWarps = kEigThreads / 32;
static_assert(kEigWarps * kEigSpanK <= 32, "one warp scans the per-warp counts");
static_assert(kEigSpan <= 65536, "list entries are 16-bit");

template <int VT, int AT, int FT, bool PLAIN, typename BLK>
__device__ __forceinline__ void eig_compact_body(const float* __restrict__ S, Box sb, Box ob,
                                                 const uint8_t* __restrict__ mask, Box mb, const Frame& F, float fill,
                                                 const EigOut& o, const Fallback& fb, const BLK blk) {
  constexpr int NC = kEigWarps * kEigSpanK;
  __shared__ uint16_t list[kEigSpan];
  __shared__ int cnt[NC];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int x0 = ob.lo[0] + blk.x() * kEigSpan;
  const int xend = ob.lo[0] + ob.n[0];
  const int y = ob.lo[1] + blk.y(), z = ob.lo[2] + blk.z();
  unsigned in_bits[kEigSpanK];
#pragma unroll
  for (int k = 0; k < kEigSpanK; ++k) {
    const int x = x0 + t + kEigThreads * k;
    const bool valid = x < xend;
    const bool inside = valid && __ldg(mask + box_index32(mb, x, y, z)) != 0;
    if (valid && !inside) {
      float l[3] = {0.f, 0.f, 0.f}, v[3] = {1.f, 0.f, 0.f};
      write_voxel<VT, AT, FT, int, PLAIN>(o, box_index32(o.ab, x, y, z), false, F, x, y, z, l, v, fill);
    }
    in_bits[k] = __ballot_sync(0xffffffffu, inside);
    if (lane == 0) cnt[k * kEigWarps + warp] = __popc(in_bits[k]);
  }
  __syncthreads();
  // every warp scans the counts, in (k, warp) order = x order, itself
  const int c = lane < NC ? cnt[lane] : 0;
  int incl = c;
#pragma unroll
  for (int d = 1; d < NC; d <<= 1) {
    const int u = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += u;
  }
  const int total = __shfl_sync(0xffffffffu, incl, NC - 1);
  const unsigned below = (1u << lane) - 1u;
#pragma unroll
  for (int k = 0; k < kEigSpanK; ++k) {
    const int base = __shfl_sync(0xffffffffu, incl - c, k * kEigWarps + warp);
    if (in_bits[k] >> lane & 1u) list[base + __popc(in_bits[k] & below)] = (uint16_t)(t + kEigThreads * k);
  }
  __syncthreads();
  const int ns = sb.n[0] * sb.n[1] * sb.n[2];
  for (int i0 = t; i0 < total; i0 += kEigThreads * kEigIlp) {
    int xs[kEigIlp];
    Sym3<float> s[kEigIlp];
#pragma unroll
    for (int u = 0; u < kEigIlp; ++u) {
      const int i = i0 + kEigThreads * u;
      xs[u] = x0 + list[i < total ? i : i0];
      const int si = box_index32(sb, xs[u], y, z);
      s[u].a = __ldg(S + si);
      s[u].b = __ldg(S + ns + si);
      s[u].c = __ldg(S + 2 * ns + si);
      s[u].d = __ldg(S + 3 * ns + si);
      s[u].e = __ldg(S + 4 * ns + si);
      s[u].f = __ldg(S + 5 * ns + si);
    }
#pragma unroll
    for (int u = 0; u < kEigIlp; ++u) {
      if (i0 + kEigThreads * u >= total) break;
      const int x = xs[u];
      float l[3], v[3];
      if (!eig_closed<float>(s[u], l, v, fb.gap))
        push_fallback(fb, ((int64_t)blk.z() * ob.n[1] + blk.y()) * ob.n[0] + (x - ob.lo[0]));
      write_voxel<VT, AT, FT, int, PLAIN>(o, box_index32(o.ab, x, y, z), true, F, x, y, z, l, v, fill);
    }
  }
}

template <int VT, int AT, int FT, bool PLAIN>
__global__ void __launch_bounds__(kEigThreads, CT_EIG_MINB * 256 / kEigThreads)
    k_eig_angles_compact(const float* __restrict__ S, Box sb, Box ob, const uint8_t* __restrict__ mask, Box mb,
                         Frame F, float fill, EigOut o, bool mixed, Fallback fb) {
  (void)mixed;
  eig_compact_body<VT, AT, FT, PLAIN>(S, sb, ob, mask, mb, F, fill, o, fb, HwBlock{});
}

// The eigen stage over a batch of volumes in one persistent launch: masked
// items through the compacted form (kEigThreads per CTA), unmasked ones one
// voxel per thread (kEigMultiThreads per CTA); the encodings and the plain
// frame are the batch's (the plan's).
constexpr int kEigMultiThreads = 256;
template <int VT, int AT, int FT, bool PLAIN, bool COMPACT>
__global__ void __launch_bounds__(COMPACT ? kEigThreads : kEigMultiThreads,
                                  COMPACT ? CT_EIG_MINB * 256 / kEigThreads : CT_EIG_MINB)
    k_eig_multi(const EigItem* __restrict__ items, const MultiTable T, float fill) {
  for_each_vblock<COMPACT ? 4 : 16>(T, [&](int i, const VBlock& v) {
    const EigItem& it = items[i];
    if (COMPACT)
      eig_compact_body<VT, AT, FT, PLAIN>(it.S, it.sb, it.ob, it.mask, it.mb, it.F, fill, it.o, it.fb, v);
    else
      eig32_body<VT, AT, FT, PLAIN>(it.S, it.sb, it.ob, it.mask, it.mb, it.F, fill, it.o, it.fb, v);
  });
}

__global__ void __launch_bounds__(128)
    k_eig_angles_fallback(const float* __restrict__ S, Box sb, Box ob, const uint8_t* __restrict__ mask, Box mb,
                          Frame F, float fill, EigOut o, bool mixed, Fallback fb) {
  const int64_t cnt = min((int64_t)*fb.count, fb.cap);
  const int64_t ns = box_vox(sb);
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < cnt; j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = fb.list[j];
    const int x = ob.lo[0] + (int)(i % ob.n[0]);
    const int y = ob.lo[1] + (int)((i / ob.n[0]) % ob.n[1]);
    const int z = ob.lo[2] + (int)(i / ((int64_t)ob.n[0] * ob.n[1]));
    Sym3<float> s = load_sym(S, ns, box_index(sb, x, y, z));
    float l[3], v[3];
    resolve(s, mixed, l, v);
    write_voxel(o, box_index(o.ab, x, y, z), true, F, x, y, z, l, v, fill);
  }
}

// The re-solve of a batch: blockIdx.y = item, each item's listed voxels grid-strided.
__global__ void __launch_bounds__(128)
    k_eig_fallback_multi(const EigItem* __restrict__ items, float fill, bool mixed) {
  const EigItem& it = items[blockIdx.y];
  const int64_t cnt = min((int64_t)*it.fb.count, it.fb.cap);
  const int64_t ns = box_vox(it.sb);
  const Box ob = it.ob;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < cnt; j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = it.fb.list[j];
    const int x = ob.lo[0] + (int)(i % ob.n[0]);
    const int y = ob.lo[1] + (int)((i / ob.n[0]) % ob.n[1]);
    const int z = ob.lo[2] + (int)(i / ((int64_t)ob.n[0] * ob.n[1]));
    Sym3<float> s = load_sym(it.S, ns, box_index(it.sb, x, y, z));
    float l[3], v[3];
    resolve(s, mixed, l, v);
    write_voxel(it.o, box_index(it.o.ab, x, y, z), true, it.F, x, y, z, l, v, fill);
  }
}

// The re-solve launches: the listed voxels are few (the list's length is read
// on the device), so a few CTAs per SM stride over it; a grid sized by the box
// would mostly start CTAs that find nothing (batches launch one per item).
static int fallback_grid(int64_t max_items) {
  static const int sms = [] {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    return cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && n > 0 ? n : 152;
  }();
  const int64_t b = (max_items + 127) / 128;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, 4 * sms));
}

static int grid_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  const int64_t cap = 152 * 64;  // grid-stride beyond this
  return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

cudaError_t launch_eig_angles(const float* S, const Box& sb, const Box& ob, const uint8_t* mask, const Box& mb,
                              const Frame& F, float fill, const EigOut& o, bool mixed, const Fallback& fb,
                              bool compact, cudaStream_t st) {
  int64_t n = box_vox(ob);
  if (n == 0) return cudaSuccess;
  const int rows = ob.n[1] * ob.n[2];
  const int gy = rows < 65535 ? rows : 65535;
  // 128-thread rows where 256 would leave more columns idle (e.g. width 384)
  const int nt = ((ob.n[0] + 127) / 128 * 128 - ob.n[0]) < ((ob.n[0] + 255) / 256 * 256 - ob.n[0]) ? 128 : 256;
  dim3 grid((ob.n[0] + nt - 1) / nt, gy, (rows + gy - 1) / gy);
  // 32-bit indices and a (x, y, z) grid when every plane set fits
  const int64_t lim = ((int64_t)1 << 31) - 1;
  if (ob.n[1] <= 65535 && ob.n[2] <= 65535 && 6 * box_vox(sb) <= lim && 3 * box_vox(o.ab) <= lim &&
      box_vox(mb) <= lim) {
    dim3 g3((ob.n[0] + nt - 1) / nt, ob.n[1], ob.n[2]);
    // unit voxels and a fixed centre take the plain frame
    const bool plain = F.sp[0] == 1.f && F.sp[1] == 1.f && F.sp[2] == 1.f && F.centres == nullptr;
    if (mask != nullptr && compact) {
      dim3 gc((ob.n[0] + kEigSpan - 1) / kEigSpan, ob.n[1], ob.n[2]);
      if (o.vec_t == CT_OUT_F32 && o.ang_t == CT_OUT_F32 && o.fa_t == CT_OUT_F32) {
        if (plain)
          k_eig_angles_compact<0, 0, 0, true><<<gc, kEigThreads, 0, st>>>(S, sb, ob, mask, mb, F, fill, o, mixed, fb);
        else
          k_eig_angles_compact<0, 0, 0, false><<<gc, kEigThreads, 0, st>>>(S, sb, ob, mask, mb, F, fill, o, mixed, fb);
      } else if (o.vec_t == CT_OUT_F16 && o.ang_t == CT_OUT_F16 && o.fa_t == CT_OUT_F16) {
        if (plain)
          k_eig_angles_compact<1, 1, 1, true><<<gc, kEigThreads, 0, st>>>(S, sb, ob, mask, mb, F, fill, o, mixed, fb);
        else
          k_eig_angles_compact<1, 1, 1, false><<<gc, kEigThreads, 0, st>>>(S, sb, ob, mask, mb, F, fill, o, mixed, fb);
      } else if (o.ang_t == CT_OUT_U8Q && o.fa_t == CT_OUT_F16) {
        k_eig_angles_compact<-1, 2, 1, false><<<gc, kEigThreads, 0, st>>>(S, sb, ob, mask, mb, F, fill, o, mixed, fb);
      } else {
        k_eig_angles_compact<-1, -1, -1, false><<<gc, kEigThreads, 0, st>>>(S, sb, ob, mask, mb, F, fill, o, mixed, fb);
      }
      return cudaGetLastError();
    }
    if (o.vec_t == CT_OUT_F32 && o.ang_t == CT_OUT_F32 && o.fa_t == CT_OUT_F32) {
      if (plain)
        k_eig_angles32<0, 0, 0, true><<<g3, nt, 0, st>>>(S, sb, ob, mask, mb, F, fill, o, mixed, fb);
      else
        k_eig_angles32<0, 0, 0, false><<<g3, nt, 0, st>>>(S, sb, ob, mask, mb, F, fill, o, mixed, fb);
    } else if (o.vec_t == CT_OUT_F16 && o.ang_t == CT_OUT_F16 && o.fa_t == CT_OUT_F16) {
      if (plain)
        k_eig_angles32<1, 1, 1, true><<<g3, nt, 0, st>>>(S, sb, ob, mask, mb, F, fill, o, mixed, fb);
      else
        k_eig_angles32<1, 1, 1, false><<<g3, nt, 0, st>>>(S, sb, ob, mask, mb, F, fill, o, mixed, fb);
    } else if (o.ang_t == CT_OUT_U8Q && o.fa_t == CT_OUT_F16) {
      k_eig_angles32<-1, 2, 1, false><<<g3, nt, 0, st>>>(S, sb, ob, mask, mb, F, fill, o, mixed, fb);
    } else {
      k_eig_angles32<-1, -1, -1, false><<<g3, nt, 0, st>>>(S, sb, ob, mask, mb, F, fill, o, mixed, fb);
    }
    return cudaGetLastError();
  }
  // the encodings of the common configurations are compiled in; others are read at run time
  if (o.vec_t == CT_OUT_F32 && o.ang_t == CT_OUT_F32 && o.fa_t == CT_OUT_F32)
    k_eig_angles<0, 0, 0><<<grid, nt, 0, st>>>(S, sb, ob, mask, mb, F, fill, o, mixed, fb);
  else if (o.vec_t == CT_OUT_F16 && o.ang_t == CT_OUT_F16 && o.fa_t == CT_OUT_F16)
    k_eig_angles<1, 1, 1><<<grid, nt, 0, st>>>(S, sb, ob, mask, mb, F, fill, o, mixed, fb);
  else if (o.ang_t == CT_OUT_U8Q && o.fa_t == CT_OUT_F16)
    k_eig_angles<-1, 2, 1><<<grid, nt, 0, st>>>(S, sb, ob, mask, mb, F, fill, o, mixed, fb);
  else
    k_eig_angles<-1, -1, -1><<<grid, nt, 0, st>>>(S, sb, ob, mask, mb, F, fill, o, mixed, fb);
  return cudaGetLastError();
}

cudaError_t launch_eig_angles_fallback(const float* S, const Box& sb, const Box& ob, const uint8_t* mask,
                                       const Box& mb, const Frame& F, float fill, const EigOut& o, bool mixed,
                                       const Fallback& fb, int64_t max_items, cudaStream_t st) {
  if (max_items <= 0) return cudaSuccess;
  k_eig_angles_fallback<<<fallback_grid(max_items), 128, 0, st>>>(S, sb, ob, mask, mb, F, fill, o, mixed, fb);
  return cudaGetLastError();
}

// ------------------------------------------------------------ batches
bool eig_item_ok(const EigItem& it) {
  const int64_t lim = ((int64_t)1 << 31) - 1;
  return it.ob.n[1] <= 65535 && it.ob.n[2] <= 65535 && 6 * box_vox(it.sb) <= lim && 3 * box_vox(it.o.ab) <= lim &&
         box_vox(it.mb) <= lim;
}

uint3 eig_item_grid(bool compact, const EigItem& it) {
  const Box& ob = it.ob;
  return compact ? make_uint3((ob.n[0] + kEigSpan - 1) / kEigSpan, ob.n[1], ob.n[2])
                 : make_uint3((ob.n[0] + kEigMultiThreads - 1) / kEigMultiThreads, ob.n[1], ob.n[2]);
}

template <int VT, int AT, int FT, bool PLAIN, bool COMPACT>
static cudaError_t eig_multi_t(const EigItem* items, const MultiTable& T, int64_t blocks, float fill,
                               cudaStream_t st) {
  constexpr int threads = COMPACT ? kEigThreads : kEigMultiThreads;
  const int grid = persistent_grid(k_eig_multi<VT, AT, FT, PLAIN, COMPACT>, threads, 0, blocks);
  k_eig_multi<VT, AT, FT, PLAIN, COMPACT><<<grid, threads, 0, st>>>(items, T, fill);
  return cudaGetLastError();
}

template <bool COMPACT>
static cudaError_t eig_multi_c(const EigItem* items, const MultiTable& T, int64_t blocks, int vt, int at, int ft,
                               bool plain, float fill, cudaStream_t st) {
  if (vt == CT_OUT_F32 && at == CT_OUT_F32 && ft == CT_OUT_F32)
    return plain ? eig_multi_t<0, 0, 0, true, COMPACT>(items, T, blocks, fill, st)
                 : eig_multi_t<0, 0, 0, false, COMPACT>(items, T, blocks, fill, st);
  if (vt == CT_OUT_F16 && at == CT_OUT_F16 && ft == CT_OUT_F16)
    return plain ? eig_multi_t<1, 1, 1, true, COMPACT>(items, T, blocks, fill, st)
                 : eig_multi_t<1, 1, 1, false, COMPACT>(items, T, blocks, fill, st);
  if (at == CT_OUT_U8Q && ft == CT_OUT_F16) return eig_multi_t<-1, 2, 1, false, COMPACT>(items, T, blocks, fill, st);
  return eig_multi_t<-1, -1, -1, false, COMPACT>(items, T, blocks, fill, st);
}

cudaError_t launch_eig_multi(const EigItem* items, const MultiTable& T, int64_t blocks, bool compact, int vt, int at,
                             int ft, bool plain, float fill, cudaStream_t st) {
  return compact ? eig_multi_c<true>(items, T, blocks, vt, at, ft, plain, fill, st)
                 : eig_multi_c<false>(items, T, blocks, vt, at, ft, plain, fill, st);
}

cudaError_t launch_eig_fallback_multi(const EigItem* items, int n_items, int64_t max_per_item, float fill, bool mixed,
                                      cudaStream_t st) {
  if (n_items <= 0 || max_per_item <= 0) return cudaSuccess;
  dim3 grid((unsigned)std::min<int64_t>((max_per_item + 127) / 128, 64), (unsigned)n_items);
  k_eig_fallback_multi<<<grid, 128, 0, st>>>(items, fill, mixed);
  return cudaGetLastError();
}

// ------------------------------------------------------------ stage kernels
__global__ void __launch_bounds__(256)
    k_eig_only(const float* __restrict__ S, int64_t n, float* __restrict__ evals, float* __restrict__ evec,
               bool mixed, Fallback fb) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    Sym3<float> s = load_sym(S, n, i);
    float l[3], v[3];
    if (!eig_closed<float>(s, l, v, fb.gap)) push_fallback(fb, i);
    orient_largest(v);
    if (evals) {
      evals[i] = l[0];
      evals[n + i] = l[1];
      evals[2 * n + i] = l[2];
    }
    evec[i] = v[0];
    evec[n + i] = v[1];
    evec[2 * n + i] = v[2];
  }
}

__global__ void __launch_bounds__(128)
    k_eig_only_fallback(const float* __restrict__ S, int64_t n, float* __restrict__ evals, float* __restrict__ evec,
                        bool mixed, Fallback fb) {
  const int64_t cnt = min((int64_t)*fb.count, fb.cap);
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < cnt; j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = fb.list[j];
    Sym3<float> s = load_sym(S, n, i);
    float l[3], v[3];
    resolve(s, mixed, l, v);
    orient_largest(v);
    if (evals) {
      evals[i] = l[0];
      evals[n + i] = l[1];
      evals[2 * n + i] = l[2];
    }
    evec[i] = v[0];
    evec[n + i] = v[1];
    evec[2 * n + i] = v[2];
  }
}

__global__ void __launch_bounds__(256)
    k_angles_only(const float* __restrict__ evec, const float* __restrict__ evals, Box ob,
                  const uint8_t* __restrict__ mask, Frame F, float fill, EigOut o) {
  const int64_t n = box_vox(ob);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int x = ob.lo[0] + (int)(i % ob.n[0]);
    const int y = ob.lo[1] + (int)((i / ob.n[0]) % ob.n[1]);
    const int z = ob.lo[2] + (int)(i / ((int64_t)ob.n[0] * ob.n[1]));
    const bool inside = mask == nullptr || __ldg(mask + i) != 0;
    float l[3] = {__ldg(evals + i), __ldg(evals + n + i), __ldg(evals + 2 * n + i)};
    float v[3] = {__ldg(evec + i), __ldg(evec + n + i), __ldg(evec + 2 * n + i)};
    write_voxel(o, i, inside, F, x, y, z, l, v, fill);
  }
}

cudaError_t launch_eig_only(const float* S, int64_t n, float* evals, float* evec, bool mixed, const Fallback& fb,
                            cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_eig_only<<<grid_for(n, 256), 256, 0, st>>>(S, n, evals, evec, mixed, fb);
  return cudaGetLastError();
}

cudaError_t launch_eig_only_fallback(const float* S, int64_t n, float* evals, float* evec, bool mixed,
                                     const Fallback& fb, int64_t max_items, cudaStream_t st) {
  if (max_items <= 0) return cudaSuccess;
  k_eig_only_fallback<<<fallback_grid(max_items), 128, 0, st>>>(S, n, evals, evec, mixed, fb);
  return cudaGetLastError();
}

cudaError_t launch_angles_only(const float* evec, const float* evals, const Box& ob, const uint8_t* mask,
                               const Frame& F, float fill, const EigOut& o, cudaStream_t st) {
  int64_t n = box_vox(ob);
  if (n == 0) return cudaSuccess;
  k_angles_only<<<grid_for(n, 256), 256, 0, st>>>(evec, evals, ob, mask, F, fill, o);
  return cudaGetLastError();
}

}  // namespace ct
