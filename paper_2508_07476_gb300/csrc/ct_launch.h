// Host-side entry points of the kernels (internal to the library).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ct_common.cuh"

namespace ct {

// Set the shared-memory attributes of every kernel instantiation (once per process,
// before any launch may be captured into a graph).
cudaError_t prepare_rho_xy_kernels();
cudaError_t prepare_grad_split_kernels();

// Instantiated radius that serves radius r (zero taps pad the difference), or -1.
int sigma_kernel_radius(int r);
int rho_kernel_radius(int r);

// The gradient and its products: launch_grad_xy writes the x/y-filtered partial
// fields (3 planes over ab = grad_partial_box(ob, vb, R, dims[2])) of vol;
// launch_grad_z takes their z pass and writes J (6 FP32 planes over ob), or
// with gout the gradient g (3 planes over ob: FP16 holding g * 2^-8 in the
// mixed form, FP32 otherwise) for launch_rho_tc_products to form J from.
Box grad_partial_box(const Box& ob, const Box& vb, int rs, int dimz);
// tx / ty / tz: the taps of each axis (anisotropic voxels); scale: the factor of
// each product (1 / (spacing_a spacing_b), xx yy zz xy xz yz).
cudaError_t launch_grad_xy(const uint16_t* vol, const Box& vb, const int dims[3], float* F, const Box& ab,
                           const Taps& tx, const Taps& ty, int rk, cudaStream_t st);
cudaError_t launch_grad_z(const float* F, const Box& ab, void* J, const Box& ob, const Taps& tz,
                          const float scale[6], int rk, bool mixed, bool gout, cudaStream_t st);

// rho pass along x: out (6 planes over ob) from in (6 planes over ib).
cudaError_t launch_rho_x(const float* in, const Box& ib, const int dims[3], float* out, const Box& ob,
                         const Taps& taps, int rk, cudaStream_t st);

// rho passes along x and y fused: out (6 planes over ob) from in (6 planes over ib).
cudaError_t launch_rho_xy(const float* in, const Box& ib, const int dims[3], float* out, const Box& ob,
                          const Taps& tx, const Taps& ty, int rk, cudaStream_t st);

// rho pass along axis 1 (y) or 2 (z), streaming register windows of block_t (8 or 16) outputs.
cudaError_t launch_rho_stream(const float* in, const Box& ib, const int dims[3], float* out, const Box& ob, int axis,
                              const Taps& taps, int rk, int block_t, cudaStream_t st);

// rho pass along axis 0, 1 or 2 on the tensor cores (banded Toeplitz product,
// TF32 split operands, FP32 accumulation): same contract as launch_rho_x /
// launch_rho_stream.  prepare_rho_tc_kernels sets the shared-memory
// attributes (call before any capture).  Every CTA that gives up a bounded
// wait (ctl.wait_limit polls on another role; copies are waited for up to a
// fixed limit) stops, drains its copies and products, releases its tensor
// memory and adds 1 to *ctl.timeouts (a device word of the caller's plan).
struct TcCtl {
  unsigned int* timeouts;
  uint32_t wait_limit;
  int seg_cap;  // outputs per work unit at most (0: 512); the work is then spread over the SMs
};
cudaError_t prepare_rho_tc_kernels();
cudaError_t launch_rho_tc(const float* in, const Box& ib, const int dims[3], float* out, const Box& ob, int axis,
                          const Taps& taps, int rk, const TcCtl& ctl, cudaStream_t st);
// The same pass along axis 1 or 2 reading the gradient instead of the tensor:
// g (3 planes over ib: FP16 holding g * 2^-8 when half, else FP32, as
// launch_grad_z writes them with gout) -> out (6 planes over ob) = the pass of
// the products g_a g_b * scale[k], each formed as launch_grad_z forms it.
cudaError_t launch_rho_tc_products(const void* g, bool half, const Box& ib, const int dims[3], float* out,
                                   const Box& ob, int axis, const Taps& taps, const float scale[6], int rk,
                                   const TcCtl& ctl, cudaStream_t st);
// Whether a volume nx voxels wide suits launch_rho_tc along axis: 16-byte copies
// of its rows (x extent a multiple of 4).
bool rho_tc_volume_aligned(int nx, int axis);

// ---------------------------------------------------------------- batches
// One persistent launch per stage over a batch of volumes (MultiTable, in
// ct_common.cuh): the item's arguments as the single-item launch takes them;
// *_item fills the item's launch shape (seg: the whole walk, unsplit, since
// the batch's items fill the GPU) and returns its grid; the blocks compute
// every output with the same operations as the single launch, so a batch
// reproduces every item's results bit for bit; launch_*_multi runs the stage
// over a device table of items (grid: the SMs times the blocks each holds, at
// most `blocks`).
struct GxyItem {
  const uint16_t* vol;
  Box vb;
  int dimx, dimy;
  float* F;
  Box ab;
  int seg;
};
struct GzItem {
  const float* F;
  Box ab;
  float* J;
  Box ob;
  int seg;
};
struct RxyItem {
  const float* in;
  Box ib;
  int dimx, dimy;
  float* out;
  Box ob;
  int seg;
};
struct RzItem {
  const float* in;
  Box ib;
  int dim_axis;
  float* out;
  Box ob;
  int seg;
};
uint3 grad_xy_item(int rk, GxyItem& it);
cudaError_t launch_grad_xy_multi(const GxyItem* items, const MultiTable& T, int64_t blocks, const Taps& tx,
                                 const Taps& ty, int rk, cudaStream_t st);
uint3 grad_z_item(int rk, GzItem& it);
cudaError_t launch_grad_z_multi(const GzItem* items, const MultiTable& T, int64_t blocks, const Taps& tz,
                                const float scale[6], int rk, bool mixed, cudaStream_t st);
// the fused x / y stencil at the CTA width `xt` (128 or 256; rho_xy_width picks it as the single launch does)
int rho_xy_width(int n0);
uint3 rho_xy_item(int rk, int xt, RxyItem& it);
cudaError_t launch_rho_xy_multi(const RxyItem* items, const MultiTable& T, int64_t blocks, const Taps& tx,
                                const Taps& ty, int rk, int xt, cudaStream_t st);
// the z stencil (axis 2), block_t outputs per thread block; the block shape
// of an item: rho_stream_block (the single launch's), fixed per batch launch
uint3 rho_z_item(int rk, int block_t, dim3 block, RzItem& it);
dim3 rho_stream_block(const Box& ob, int axis);
cudaError_t launch_rho_z_multi(const RzItem* items, const MultiTable& T, int64_t blocks, dim3 block,
                               const Taps& taps, int rk, int block_t, cudaStream_t st);

// Persistent grid of a multi-item launch: the SMs times the CTAs each holds.
template <typename K>
int persistent_grid(K kernel, int threads, size_t smem, int64_t blocks) {
  int dev = 0, sms = 1, per = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem) != cudaSuccess || per < 1) per = 1;
  const int64_t g = (int64_t)per * sms;
  return (int)(blocks < g ? (blocks > 0 ? blocks : 1) : g);
}

struct EigOut {
  void* vec;
  void* ha;
  void* ia;
  void* fa;
  int vec_t, ang_t, fa_t;
  Box ab;  // box covered by the output arrays
};

struct Fallback {
  float gap = kDegenerateGap;  // listing threshold of the arithmetic form (degenerate_gap)
  int* count;                 // device counter of listed voxels (reset per launch)
  unsigned long long* total;  // device running total (for statistics)
  int64_t* list;
  int64_t cap;
};

// The near-degeneracy listing threshold of an arithmetic form (FP32 / mixed).
inline float degenerate_gap(bool mixed) { return mixed ? kDegenerateGapMixed : kDegenerateGap; }

// One item of a batched eigen stage (the arguments of launch_eig_angles).
struct EigItem {
  const float* S;
  Box sb, ob;
  const uint8_t* mask;
  Box mb;
  Frame F;
  EigOut o;
  Fallback fb;
};
// Whether an item suits the batched eigen kernels (32-bit indices, rows in the grid).
bool eig_item_ok(const EigItem& it);
uint3 eig_item_grid(bool compact, const EigItem& it);
cudaError_t launch_eig_multi(const EigItem* items, const MultiTable& T, int64_t blocks, bool compact, int vt, int at,
                             int ft, bool plain, float fill, cudaStream_t st);
// The re-solve of every item's listed voxels (at most max_per_item each) in one launch.
cudaError_t launch_eig_fallback_multi(const EigItem* items, int n_items, int64_t max_per_item, float fill, bool mixed,
                                      cudaStream_t st);

// Per-voxel eigen-solve + HA/IA/FA over ob from S (6 planes over sb); mask
// array (nullable) covers mb.  Near-degenerate voxels are appended to fb.
// compact: with a mask, each row segment lists its inside voxels first and
// solves them with full warps (the same arithmetic per voxel).
cudaError_t launch_eig_angles(const float* S, const Box& sb, const Box& ob, const uint8_t* mask, const Box& mb,
                              const Frame& F, float fill, const EigOut& o, bool mixed, const Fallback& fb,
                              bool compact, cudaStream_t st);
// Re-solve the listed voxels (FP32 Jacobi, or FP64 in the mixed form) and rewrite their outputs.
cudaError_t launch_eig_angles_fallback(const float* S, const Box& sb, const Box& ob, const uint8_t* mask,
                                       const Box& mb, const Frame& F, float fill, const EigOut& o, bool mixed,
                                       const Fallback& fb, int64_t max_items, cudaStream_t st);

// Stage kernels: eigen only (evals + unoriented evec), and angles only.
cudaError_t launch_eig_only(const float* S, int64_t n, float* evals, float* evec, bool mixed, const Fallback& fb,
                            cudaStream_t st);
cudaError_t launch_eig_only_fallback(const float* S, int64_t n, float* evals, float* evec, bool mixed,
                                     const Fallback& fb, int64_t max_items, cudaStream_t st);
cudaError_t launch_angles_only(const float* evec, const float* evals, const Box& ob, const uint8_t* mask,
                               const Frame& F, float fill, const EigOut& o, cudaStream_t st);

}  // namespace ct
