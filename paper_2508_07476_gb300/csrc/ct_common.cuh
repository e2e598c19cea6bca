// Device-side building blocks shared by the library's kernels (not by the oracle).
//
// Sources: the structure tensor, its smallest-eigenvalue eigenvector and the
// HA / IA / FA descriptors are the stages of Figure 1(b,c) and of the
// "orientation" module (Architecture); chunking with padding is described under
// Implementation.  The paper gives no formulas; the definitions used are the
// textbook ones stated in include/ct.h.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace ct {

constexpr int kMaxRadius = 36;               // largest supported tap radius
constexpr int kMaxTaps = 2 * kMaxRadius + 1;

// Taps of one scale, passed by value as a kernel parameter so that each FMA
// reads its weight from the constant bank.  w: sampled normalised Gaussian;
// c: derivative-correlation taps c_k = (k / s^2) w_k; entries beyond the
// actual radius are zero (a zero tap adds an exact +0 and changes nothing).
struct Taps {
  float w[kMaxTaps];
  float c[kMaxTaps];
};

// A box of the global volume: lo (x, y, z) and extent n (x, y, z).
struct Box {
  int lo[3];
  int n[3];
};

__host__ __device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

__host__ __device__ __forceinline__ int64_t box_vox(const Box& b) { return (int64_t)b.n[0] * b.n[1] * b.n[2]; }

// Linear index of global voxel (x, y, z) in an array covering box b.
__device__ __forceinline__ int64_t box_index(const Box& b, int x, int y, int z) {
  return ((int64_t)(z - b.lo[2]) * b.n[1] + (y - b.lo[1])) * b.n[0] + (x - b.lo[0]);
}

// Global coordinate p + k clamped to the volume [0, dim) and then to the array
// box [lo, lo + n) (the second clamp only matters for lanes whose outputs are
// discarded: for every stored output the first clamp already lands inside the
// array, which the host validates).
__device__ __forceinline__ int clamp_to(int p, int dim, int lo, int n) {
  return clampi(clampi(p, 0, dim - 1), lo, lo + n - 1);
}

// ---------------------------------------------------------------------------
// Persistent multi-item launches.  A stage kernel's body reads its block index
// and grid size from a VBlock instead of blockIdx / gridDim: the single-item
// kernel passes its own, and a persistent launch over a batch of items (the
// blocks of item i numbered first[i] .. first[i+1] - 1 in one sequence, its
// grid grids[i]) runs the body once per block it takes from a device counter,
// so that all items of the batch share one launch and the SMs stay busy
// across items of any size.  The counter is zeroed before the launch; every
// CTA stops once the counter passes the last block (no CTA waits on another).
struct VBlock {
  uint3 idx;
  uint3 dim;
  __device__ __forceinline__ unsigned x() const { return idx.x; }
  __device__ __forceinline__ unsigned y() const { return idx.y; }
  __device__ __forceinline__ unsigned z() const { return idx.z; }
};

// The launch's own block index, read where it is used (the single-item kernels
// compile as if the body read blockIdx itself).
struct HwBlock {
  __device__ __forceinline__ unsigned x() const { return blockIdx.x; }
  __device__ __forceinline__ unsigned y() const { return blockIdx.y; }
  __device__ __forceinline__ unsigned z() const { return blockIdx.z; }
};

// Per-launch table of a multi-item launch (device pointers).
struct MultiTable {
  const int64_t* first;  // n + 1 block offsets
  const uint3* grids;    // n grids
  int n;
  unsigned long long* counter;
};

// CLAIM: blocks taken per counter increment (consecutive ones), so that the
// counter's round trip is paid once per CLAIM blocks of short-lived kernels.
template <int CLAIM = 1, typename F>
__device__ __forceinline__ void for_each_vblock(const MultiTable& T, F&& f) {
  __shared__ long long s_next;
  const int64_t total = T.first[T.n];
  for (;;) {
    if (threadIdx.x == 0 && threadIdx.y == 0 && threadIdx.z == 0)
      s_next = (long long)atomicAdd(T.counter, (unsigned long long)CLAIM) ;
    __syncthreads();
    const int64_t b0 = s_next;
    __syncthreads();  // every thread has read it before it is overwritten
    if (b0 >= total) break;
    int lo = 0, hi = T.n - 1;  // the item whose blocks hold b0: the last with first <= b0
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (T.first[mid] <= b0) lo = mid;
      else hi = mid - 1;
    }
    for (int c = 0; c < CLAIM; ++c) {
      const int64_t b = b0 + c;
      if (b >= total) break;
      while (lo + 1 < T.n && T.first[lo + 1] <= b) ++lo;  // the claim may run into the next item
      const uint3 g = T.grids[lo];
      int64_t r = b - T.first[lo];
      VBlock v;
      v.dim = g;
      v.idx.x = (unsigned)(r % g.x);
      r /= g.x;
      v.idx.y = (unsigned)(r % g.y);
      v.idx.z = (unsigned)(r / g.y);
      f(lo, v);
      __syncthreads();  // the block's shared memory is free for the next one
    }
  }
}

// Asynchronous 4-byte global -> shared copies (cp.async), grouped per commit.
__device__ __forceinline__ void cp_async4(uint32_t smem_dst, const float* gsrc) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_dst), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// atan2(y, x) on the closed right half-plane (x >= 0), in radians.  The ratio
// a = min(|y|, x) / max(|y|, x) is reduced by the addition formula
// atan(a) = pi/6 + atan((sqrt3 a - 1) / (sqrt3 + a)) when a > 2 - sqrt3, so the
// argument u of Gregory's series u - u^3/3 + u^5/5 - u^7/7 + u^9/9 stays within
// |u| <= 2 - sqrt3, where the first omitted term is below 5e-8; |y| > x uses
// atan(a) = pi/2 - atan(1/a).  One division; the result is within a few 1e-7
// rad of atan2 (angles are reported to far coarser than that).
__device__ __forceinline__ float atan2_right(float y, float x) {
  const float ay = fabsf(y);
  const bool swap = ay > x;
  const float n = swap ? x : ay, d = swap ? ay : x;  // 0 <= n <= d
  const bool red = n > 0.26794919243112270f * d;
  const float nn = red ? fmaf(1.7320508075688772f, n, -d) : n;
  const float dd = red ? fmaf(1.7320508075688772f, d, n) : d;
  const float u = d > 0.f ? __fdividef(nn, dd) : 0.f;
  const float t = __fmul_rn(u, u);
  float p = fmaf(t, 1.f / 9.f, -1.f / 7.f);
  p = fmaf(t, p, 1.f / 5.f);
  p = fmaf(t, p, -1.f / 3.f);
  p = fmaf(t, p, 1.f);
  float r = fmaf(u, p, red ? 0.52359877559829887f : 0.f);
  r = swap ? 1.5707963267948966f - r : r;
  return copysignf(r, y);
}

// ---------------------------------------------------------------------------
// Eigen-decomposition of a symmetric 3x3 tensor s = (xx, yy, zz, xy, xz, yz).
// ---------------------------------------------------------------------------

// Near-degeneracy threshold: the smallest pair of eigenvalues closer than this
// fraction of the spread (l3 - l1) is re-solved, since the trigonometric form
// loses about half of its digits as the two smallest eigenvalues meet.  On
// FP32 input its direction error is at its floor (~0.03 deg) from a gap of
// 2e-2 of the spread up, 0.044 deg at 1e-2, 0.5 deg at 3e-3.
constexpr float kDegenerateGap = 2e-2f;
// The mixed form lists from 1e-2: its tensor already carries the FP16-held
// gradient's error (about 1e-3 of the trace), which at such gaps turns the
// direction by far more than the FP32 closed form's own 0.044 deg, so an FP64
// re-solve there would not change the result's accuracy, only its cost (FP64
// runs at a small fraction of the FP32 rate).
constexpr float kDegenerateGapMixed = 1e-2f;
// The same for the FP64 closed form (the mixed form's re-solve).  Near a double
// root an error eps in det(B) / 2 moves l1 by about eps p^2 / gap and the null
// vector by that over the gap, eps (p / gap)^2: at a gap of 1e-4 of the spread
// and eps = 1.1e-16 that is ~1e-8, far below the FP32 outputs' resolution,
// so only voxels closer than that go on to FP64 Jacobi.
constexpr double kDegenerateGap64 = 1e-4;

template <typename T>
struct Sym3 {
  T a, b, c, d, e, f;  // xx, yy, zz, xy, xz, yz
};

// Eigenvector of eigenvalue lam: the largest of the three cross products of
// the rows of (S - lam I).  Returns the squared norm of the chosen product
// before normalisation (0 when S - lam I has rank <= 1).
template <typename T>
__device__ __forceinline__ T null_vector(const Sym3<T>& s, T lam, T v[3]) {
  T r0x = s.a - lam, r0y = s.d, r0z = s.e;
  T r1x = s.d, r1y = s.b - lam, r1z = s.f;
  T r2x = s.e, r2y = s.f, r2z = s.c - lam;
  T x01 = r0y * r1z - r0z * r1y, y01 = r0z * r1x - r0x * r1z, z01 = r0x * r1y - r0y * r1x;
  T x02 = r0y * r2z - r0z * r2y, y02 = r0z * r2x - r0x * r2z, z02 = r0x * r2y - r0y * r2x;
  T x12 = r1y * r2z - r1z * r2y, y12 = r1z * r2x - r1x * r2z, z12 = r1x * r2y - r1y * r2x;
  T n01 = x01 * x01 + y01 * y01 + z01 * z01;
  T n02 = x02 * x02 + y02 * y02 + z02 * z02;
  T n12 = x12 * x12 + y12 * y12 + z12 * z12;
  T bx = x01, by = y01, bz = z01, bn = n01;
  if (n02 > bn) { bx = x02; by = y02; bz = z02; bn = n02; }
  if (n12 > bn) { bx = x12; by = y12; bz = z12; bn = n12; }
  if (bn > T(0)) {
    T inv = T(1) / sqrt(bn);
    v[0] = bx * inv; v[1] = by * inv; v[2] = bz * inv;
  } else {
    v[0] = T(1); v[1] = T(0); v[2] = T(0);
  }
  return bn;
}

// Closed-form eigenvalues (trigonometric solution of the characteristic cubic,
// O. K. Smith, Comm. ACM 4(4), 1961) and the smallest-eigenvalue eigenvector.
// With B = (S - qI)/p, q = tr/3, p^2 = |S - qI|_F^2 / 6 and phi = acos(det(B)/2)/3:
//   l3 = q + 2p cos(phi),  l1 = q + 2p cos(phi + 2pi/3) = q - p (cos(phi) + sqrt(3) sin(phi)),
//   l2 = 3q - l1 - l3.
// Eigenvalues ascending in l[0..2].  Returns true when the result is well
// conditioned, false when the voxel should be re-solved.  The FP32 form takes
// sin/cos of phi (in [0, pi/3]) from the hardware approximations and the
// reciprocal square roots from rsqrt; the errors they add, a few 1e-7 of p,
// are far below what the re-solve threshold leaves between l1 and l2.
// The FP32 form lists the voxel for a re-solve when l2 - l1 < gap (l3 - l1).
template <typename T>
__device__ __forceinline__ bool eig_closed(const Sym3<T>& s, T l[3], T v[3], T gap);

template <>
__device__ __forceinline__ bool eig_closed<float>(const Sym3<float>& s, float l[3], float v[3], float gap) {
  const float q = (s.a + s.b + s.c) * (1.f / 3.f);
  const float aq = s.a - q, bq = s.b - q, cq = s.c - q;
  const float p1 = s.d * s.d + s.e * s.e + s.f * s.f;
  const float p2 = aq * aq + bq * bq + cq * cq + 2.f * p1;
  if (p2 == 0.f) {  // isotropic (including the zero tensor): every vector is an eigenvector
    l[0] = l[1] = l[2] = q;
    v[0] = 1.f; v[1] = 0.f; v[2] = 0.f;
    return true;
  }
  const float p6 = p2 * (1.f / 6.f);
  const float ip = rsqrtf(p6);
  const float p = p6 * ip;
  const float B00 = aq * ip, B11 = bq * ip, B22 = cq * ip, B01 = s.d * ip, B02 = s.e * ip, B12 = s.f * ip;
  const float det = B00 * (B11 * B22 - B12 * B12) - B01 * (B01 * B22 - B12 * B02) + B02 * (B01 * B12 - B11 * B02);
  const float r = fminf(fmaxf(0.5f * det, -1.f), 1.f);
  const float phi = acosf(r) * (1.f / 3.f);
  float sp, cp;
  __sincosf(phi, &sp, &cp);
  float l3 = q + 2.f * p * cp;
  float l1 = q - p * (cp + 1.7320508075688772f * sp);
  float l2 = 3.f * q - l1 - l3;
  if (l2 < l1) { float t = l1; l1 = l2; l2 = t; }
  if (l3 < l2) { float t = l2; l2 = l3; l3 = t; }
  l[0] = l1; l[1] = l2; l[2] = l3;
  // null vector of S - l1 I: the largest cross product of two of its rows
  const float r0x = s.a - l1, r0y = s.d, r0z = s.e;
  const float r1x = s.d, r1y = s.b - l1, r1z = s.f;
  const float r2x = s.e, r2y = s.f, r2z = s.c - l1;
  const float x01 = r0y * r1z - r0z * r1y, y01 = r0z * r1x - r0x * r1z, z01 = r0x * r1y - r0y * r1x;
  const float x02 = r0y * r2z - r0z * r2y, y02 = r0z * r2x - r0x * r2z, z02 = r0x * r2y - r0y * r2x;
  const float x12 = r1y * r2z - r1z * r2y, y12 = r1z * r2x - r1x * r2z, z12 = r1x * r2y - r1y * r2x;
  const float n01 = x01 * x01 + y01 * y01 + z01 * z01;
  const float n02 = x02 * x02 + y02 * y02 + z02 * z02;
  const float n12 = x12 * x12 + y12 * y12 + z12 * z12;
  float bx = x01, by = y01, bz = z01, bn = n01;
  if (n02 > bn) { bx = x02; by = y02; bz = z02; bn = n02; }
  if (n12 > bn) { bx = x12; by = y12; bz = z12; bn = n12; }
  if (bn > 0.f) {
    const float inv = rsqrtf(bn);
    v[0] = bx * inv; v[1] = by * inv; v[2] = bz * inv;
  } else {
    v[0] = 1.f; v[1] = 0.f; v[2] = 0.f;
  }
  return (l2 - l1) >= gap * (l3 - l1) && bn > 0.f;
}

// FP64 version (the re-solve of the mixed form): library acos / sincos / sqrt,
// l1 from the same sin and cos as l3 (one sincos instead of two cos).
template <>
__device__ __forceinline__ bool eig_closed<double>(const Sym3<double>& s, double l[3], double v[3], double gap) {
  const double q = (s.a + s.b + s.c) / 3.0;
  const double aq = s.a - q, bq = s.b - q, cq = s.c - q;
  const double p1 = s.d * s.d + s.e * s.e + s.f * s.f;
  const double p2 = aq * aq + bq * bq + cq * cq + 2.0 * p1;
  if (p2 == 0.0) {
    l[0] = l[1] = l[2] = q;
    v[0] = 1.0; v[1] = 0.0; v[2] = 0.0;
    return true;
  }
  const double p = sqrt(p2 / 6.0);
  const double ip = 1.0 / p;
  const double B00 = aq * ip, B11 = bq * ip, B22 = cq * ip, B01 = s.d * ip, B02 = s.e * ip, B12 = s.f * ip;
  const double det = B00 * (B11 * B22 - B12 * B12) - B01 * (B01 * B22 - B12 * B02) + B02 * (B01 * B12 - B11 * B02);
  const double r = fmin(fmax(0.5 * det, -1.0), 1.0);
  const double phi = acos(r) / 3.0;
  double sp, cp;
  sincos(phi, &sp, &cp);
  double l3 = q + 2.0 * p * cp;
  double l1 = q - p * (cp + 1.7320508075688772935 * sp);
  double l2 = 3.0 * q - l1 - l3;
  if (l2 < l1) { double t = l1; l1 = l2; l2 = t; }
  if (l3 < l2) { double t = l2; l2 = l3; l3 = t; }
  l[0] = l1; l[1] = l2; l[2] = l3;
  const double bn = null_vector(s, l1, v);
  return (l2 - l1) >= gap * (l3 - l1) && bn > 0.0;
}

// Cyclic Jacobi (Golub & Van Loan, Matrix Computations, section 8.5) on a
// symmetric 3x3: the robust re-solve for near-degenerate voxels.  Eigenvalues
// ascending; v = eigenvector of the smallest.
template <typename T>
__device__ __noinline__ void eig_jacobi(const Sym3<T>& s, T l[3], T v[3]) {
  T A[3][3] = {{s.a, s.d, s.e}, {s.d, s.b, s.f}, {s.e, s.f, s.c}};
  T Q[3][3] = {{T(1), T(0), T(0)}, {T(0), T(1), T(0)}, {T(0), T(0), T(1)}};
  T fro = T(0);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) fro += A[i][j] * A[i][j];
  fro = sqrt(fro);
  const T tol = (sizeof(T) == 8 ? T(1e-15) : T(1e-7)) * fro;
  for (int sweep = 0; sweep < 32; ++sweep) {
    T off = sqrt(T(2) * (A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2]));
    if (off <= tol || off == T(0)) break;
    for (int p = 0; p < 2; ++p) {
      for (int qq = p + 1; qq < 3; ++qq) {
        if (A[p][qq] == T(0)) continue;
        T tau = (A[qq][qq] - A[p][p]) / (T(2) * A[p][qq]);
        T t = (tau >= T(0) ? T(1) : T(-1)) / (fabs(tau) + sqrt(T(1) + tau * tau));
        T cs = T(1) / sqrt(T(1) + t * t), sn = t * cs;
        for (int k = 0; k < 3; ++k) {
          T akp = A[k][p], akq = A[k][qq];
          A[k][p] = cs * akp - sn * akq;
          A[k][qq] = sn * akp + cs * akq;
        }
        for (int k = 0; k < 3; ++k) {
          T apk = A[p][k], aqk = A[qq][k];
          A[p][k] = cs * apk - sn * aqk;
          A[qq][k] = sn * apk + cs * aqk;
        }
        for (int k = 0; k < 3; ++k) {
          T qkp = Q[k][p], qkq = Q[k][qq];
          Q[k][p] = cs * qkp - sn * qkq;
          Q[k][qq] = sn * qkp + cs * qkq;
        }
      }
    }
  }
  T d0 = A[0][0], d1 = A[1][1], d2 = A[2][2];
  int i0 = 0, i1 = 1, i2 = 2;
  if (d1 < d0) { T t = d0; d0 = d1; d1 = t; int u = i0; i0 = i1; i1 = u; }
  if (d2 < d1) { T t = d1; d1 = d2; d2 = t; int u = i1; i1 = i2; i2 = u; }
  if (d1 < d0) { T t = d0; d0 = d1; d1 = t; int u = i0; i0 = i1; i1 = u; }
  l[0] = d0; l[1] = d1; l[2] = d2;
  v[0] = Q[0][i0]; v[1] = Q[1][i0]; v[2] = Q[2][i0];
  (void)i2;
}

// Fractional anisotropy from eigenvalues clamped at zero; 0 for the zero tensor.
// The square root is taken as q rsqrt(q) (within a few 1e-7 of it), since FA
// is reported to far coarser than that.
// Every operation is explicit (fmaf, __fmul_rn), so that each kernel that
// inlines it rounds the same way.
__device__ __forceinline__ float fa_of(const float l[3]) {
  const float l1 = fmaxf(l[0], 0.f), l2 = fmaxf(l[1], 0.f), l3 = fmaxf(l[2], 0.f);
  const float den = fmaf(l1, l1, fmaf(l2, l2, __fmul_rn(l3, l3)));
  if (den == 0.f) return 0.f;
  const float d12 = l1 - l2, d23 = l2 - l3, d31 = l3 - l1;
  const float num = fmaf(d12, d12, fmaf(d23, d23, __fmul_rn(d31, d31)));
  const float q = __fdividef(0.5f * num, den);
  return q > 0.f ? __fmul_rn(q, rsqrtf(q)) : 0.f;
}

// Cylindrical left-ventricle frame (unit axis, centre), per launch.
struct Frame {
  float c[3];
  float a[3];                      // unit
  float sp[3];                     // voxel size: position = (x sp0, y sp1, z sp2)
  const float* centres = nullptr;  // per-slice LV centre (cx, cy) on the device, or none
};

// HA / IA (degrees) of v at voxel (x, y, z) (global indices; the frame is in
// the units of the voxel size); orients v so that v.e_t > 0.  Every operation
// is explicit (fmaf, __fmul_rn), so that each kernel that inlines it (and
// encodes its angles) rounds the same way.
// Returns false on the axis, where the frame does not exist.
// PLAIN: unit voxels and a fixed centre, known at compile time (the same
// arithmetic as the general form with spacing 1, without its work).
template <bool PLAIN = false>
__device__ __forceinline__ bool ha_ia(const Frame& F, int x, int y, int z, float v[3], float& ha, float& ia) {
  const float px = PLAIN ? (float)x : __fmul_rn((float)x, F.sp[0]);
  const float py = PLAIN ? (float)y : __fmul_rn((float)y, F.sp[1]);
  const float pz = PLAIN ? (float)z : __fmul_rn((float)z, F.sp[2]);
  float cx = F.c[0], cy = F.c[1], cz = F.c[2];
  if (!PLAIN && F.centres) {  // this slice's centre on the centreline
    cx = __ldg(F.centres + 2 * z);
    cy = __ldg(F.centres + 2 * z + 1);
    cz = pz;
  }
  const float dx = px - cx, dy = py - cy, dz = pz - cz;
  const float h = fmaf(dx, F.a[0], fmaf(dy, F.a[1], __fmul_rn(dz, F.a[2])));
  float rx = fmaf(-h, F.a[0], dx), ry = fmaf(-h, F.a[1], dy), rz = fmaf(-h, F.a[2], dz);
  const float rr = fmaf(rx, rx, fmaf(ry, ry, __fmul_rn(rz, rz)));
  if (rr == 0.f) return false;
  const float inv = rsqrtf(rr);
  rx = __fmul_rn(rx, inv); ry = __fmul_rn(ry, inv); rz = __fmul_rn(rz, inv);
  const float tx = fmaf(F.a[1], rz, -__fmul_rn(F.a[2], ry)), ty = fmaf(F.a[2], rx, -__fmul_rn(F.a[0], rz)),
              tz = fmaf(F.a[0], ry, -__fmul_rn(F.a[1], rx));
  float vr = fmaf(v[0], rx, fmaf(v[1], ry, __fmul_rn(v[2], rz)));
  float vt = fmaf(v[0], tx, fmaf(v[1], ty, __fmul_rn(v[2], tz)));
  float vz = fmaf(v[0], F.a[0], fmaf(v[1], F.a[1], __fmul_rn(v[2], F.a[2])));
  if (vt < 0.f || (vt == 0.f && vz < 0.f)) {
    vr = -vr; vt = -vt; vz = -vz;
    v[0] = -v[0]; v[1] = -v[1]; v[2] = -v[2];
  }
  const float rad2deg = 57.295779513082320877f;
  ha = __fmul_rn(atan2_right(vz, vt), rad2deg);
  const float pp = fmaf(vt, vt, __fmul_rn(vz, vz));  // IA = asin(vr) as the angle of v out of the (e_t, e_z) plane
  ia = __fmul_rn(atan2_right(vr, pp > 0.f ? __fmul_rn(pp, rsqrtf(pp)) : 0.f), rad2deg);
  return true;
}

// Largest-magnitude component positive (orientation where no frame exists).
__device__ __forceinline__ void orient_largest(float v[3]) {
  int m = 0;
  if (fabsf(v[1]) > fabsf(v[m])) m = 1;
  if (fabsf(v[2]) > fabsf(v[m])) m = 2;
  if (v[m] < 0.f) { v[0] = -v[0]; v[1] = -v[1]; v[2] = -v[2]; }
}

// Output encodings (CT_OUT_F32 = 0, CT_OUT_F16 = 1, CT_OUT_U8Q = 2).  TYPE is a
// compile-time encoding, or -1 for the run-time one in `type`.
template <int TYPE = -1, typename IT = int64_t>
__device__ __forceinline__ void store_val(void* base, IT i, int type, float val) {
  if (base == nullptr) return;
  const int ty = TYPE >= 0 ? TYPE : type;
  if (ty == 0) {
    reinterpret_cast<float*>(base)[i] = val;
  } else if (ty == 1) {
    reinterpret_cast<__half*>(base)[i] = __float2half_rn(val);
  }
}

template <int TYPE = -1, typename IT = int64_t>
__device__ __forceinline__ void store_angle(void* base, IT i, int type, float deg, bool valid) {
  if (base == nullptr) return;
  const int ty = TYPE >= 0 ? TYPE : type;
  if (ty == 2) {
    uint8_t code = 0;
    if (valid) code = (uint8_t)(((int)rintf(__fmul_rn(__fadd_rn(deg, 90.f), 256.f / 180.f))) & 255);
    reinterpret_cast<uint8_t*>(base)[i] = code;
  } else {
    store_val<TYPE, IT>(base, i, ty, deg);
  }
}

}  // namespace ct
