// C ABI of the library (include/ct.h): plans, argument validation, the stage
// calls, and the fused, chunked hot path with its host streaming runtime.
//
// Padded chunks (Implementation): an output box needs the input grown by
// R(sigma) + R(rho) on every side, clipped to the volume; with "nearest"
// handling at the global edges only, a chunked run reproduces the
// whole-volume result exactly.
#include <cuda_runtime.h>
#include <dlfcn.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "ct.h"
#include "ct_launch.h"

using namespace ct;

namespace {

thread_local std::string g_err;

ct_status fail(ct_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

ct_status cuda_fail(cudaError_t e, const char* what) {
  return fail(e == cudaErrorMemoryAllocation ? CT_ERR_OOM : CT_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CT_CUDA(call, what)                        \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

bool device_present() {
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return n > 0;
}

int radius_of(double s, double trunc) { return (int)std::floor(trunc * s + 0.5); }

// Sampled normalised Gaussian (w) and derivative-correlation taps (c) of scale
// s, centred in an array of instantiated radius rk; taps beyond R are zero.
Taps make_taps(double s, double trunc, int rk) {
  Taps t;
  std::memset(&t, 0, sizeof t);
  int R = radius_of(s, trunc);
  double sum = 0.0;
  for (int k = -R; k <= R; ++k) sum += std::exp(-(double)k * k / (2.0 * s * s));
  for (int k = -R; k <= R; ++k) {
    double w = std::exp(-(double)k * k / (2.0 * s * s)) / sum;
    t.w[k + rk] = (float)w;
    t.c[k + rk] = (float)((double)k / (s * s) * w);
  }
  return t;
}

Box make_box(const int64_t lo[3], const int64_t n[3]) {
  Box b;
  for (int a = 0; a < 3; ++a) {
    b.lo[a] = (int)lo[a];
    b.n[a] = (int)n[a];
  }
  return b;
}

// b grown by r[a] along axis a (anisotropic voxels give each axis its radius),
// clipped to the volume
Box grow_clip3(const Box& b, const int r[3], const int dims[3]) {
  Box o;
  for (int a = 0; a < 3; ++a) {
    int lo = std::max(0, b.lo[a] - r[a]);
    int hi = std::min(dims[a] - 1, b.lo[a] + b.n[a] - 1 + r[a]);
    o.lo[a] = lo;
    o.n[a] = hi - lo + 1;
  }
  return o;
}

bool inside(const Box& outer, const Box& inner) {
  for (int a = 0; a < 3; ++a)
    if (inner.lo[a] < outer.lo[a] || inner.lo[a] + inner.n[a] > outer.lo[a] + outer.n[a]) return false;
  return true;
}

bool valid_box(const int64_t lo[3], const int64_t n[3], const int dims[3]) {
  for (int a = 0; a < 3; ++a)
    if (lo[a] < 0 || n[a] < 1 || lo[a] + n[a] > dims[a]) return false;
  return true;
}

// Voxel size with 0 meaning 1.
void spacing_of(const ct_params& p, double sp[3]) {
  for (int a = 0; a < 3; ++a) sp[a] = p.spacing[a] > 0.0 ? p.spacing[a] : 1.0;
}

Frame make_frame(const double c[3], const double a[3], const double sp[3], const float* centres) {
  Frame F;
  double an = std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
  for (int k = 0; k < 3; ++k) {
    F.c[k] = (float)c[k];
    F.a[k] = (float)(a[k] / an);
    F.sp[k] = (float)sp[k];
  }
  F.centres = centres;
  return F;
}

// Per-axis scales: s / spacing[a] voxels along axis a.  The kernels of a pass
// are instantiated at the largest radius over the axes they filter; shorter
// tap sets are zero-padded to it.
struct Scale {
  double sigma, rho;
  int rs[3], rr[3];  // radii per axis
  int rks, rkr;      // instantiated radii
  Taps ts[3], tr[3];
  float ss[6];       // 1 / (spacing_a spacing_b) per tensor component: S in physical units
  int halo[3];       // rs + rr per axis
};

}  // namespace

struct ct_plan_s {
  ct_params p;
  int dims[3];
  double sp[3] = {1.0, 1.0, 1.0};  // voxel size (0 in the params means 1)
  float* d_centres = nullptr;      // LV centreline on the device (dims[2] pairs), or none
  int device = 0;
  // Scratch slots: slots 0 and 1 serve the two streams of host streaming;
  // batches of device items use up to kSlots streams, one slot each.
  static constexpr int kSlots = 8;
  cudaStream_t st[kSlots] = {};
  cudaEvent_t ev[kSlots] = {};
  float* buf[kSlots][2] = {};
  int64_t buf_cap[kSlots] = {};  // voxels per buffer
  int* fb_count[kSlots] = {};
  unsigned long long* fb_total = nullptr;  // running count of re-solved voxels
  int64_t* fb_list[kSlots] = {};
  int64_t fb_cap[kSlots] = {};
  // device word counting the tensor-core CTAs of this plan that gave up a
  // bounded wait (read and cleared by ct_plan_sync)
  unsigned int* d_timeouts = nullptr;
  uint32_t tc_wait_limit = 1u << 20;  // mbarrier polls before such a CTA gives up
  // streams that calls of this plan enqueued work on since the last sync,
  // each with an event recorded after that work (ct_plan_sync waits for these)
  std::vector<std::pair<cudaStream_t, cudaEvent_t>> marks;
  // device staging for host-resident items
  uint16_t* d_in[2] = {nullptr, nullptr};
  uint8_t* d_mask[2] = {nullptr, nullptr};
  void* d_out[2] = {nullptr, nullptr};
  void* h_in[2] = {nullptr, nullptr};
  void* h_out[2] = {nullptr, nullptr};
  size_t in_cap[2] = {0, 0}, out_cap[2] = {0, 0}, hin_cap[2] = {0, 0}, hout_cap[2] = {0, 0};
  // batches: graph of the multi-stream launch sequence, keyed by the item list
  int batch_streams = 4;
  bool batch_graph = true;
  // persistent batches (run_persistent_waves): device items on the FP32
  // stencil chain run as one persistent launch per stage and tap set, in waves
  // whose scratch fits batch_bytes of the arena.  Off by default: on the
  // 200-crop workload the graph of per-item launches is faster (the batched
  // bodies index through an item table and lose the per-shape constants)
  bool batch_persistent = false;
  int64_t batch_bytes = int64_t(48) << 30;
  void* arena = nullptr;
  size_t arena_cap = 0;
  void* tables = nullptr;
  size_t tables_cap = 0;
  cudaEvent_t wev[kSlots] = {};  // fork / join of a wave's chains
  cudaStream_t gst = nullptr;   // origin stream of the captured graph
  cudaEvent_t gev[2] = {nullptr, nullptr};
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  uint64_t graph_key = 0;
  int64_t graph_launches = 0, graph_voxels = 0;
  bool capturing = false;
  ct_stats stats;
  std::mutex mu;
  int stream_block = 16;  // outputs per thread block of the y / z passes (tuning choice)
  int tc_rho = 7;           // rho passes on the tensor cores: bit a for axis a (tuning choice)
  int tc_min_r = 24;        // ... for rho radii of at least this (tuning choice)
  int64_t tc_min_vox = int64_t(1) << 24;  // ... on volumes of at least this many voxels (tuning choice)
  bool tc_any_box = false;  // ... or on every volume (tuning choice)
  bool tc_products = true;  // with all three passes there: products formed in the first (tuning choice)
  bool eig_compact = true;  // masked eigen stage over compacted inside voxels (tuning choice)
  int64_t slab_bytes = int64_t(4) << 30;  // host streaming: device bytes of one slab's buffers at most
  // Autotuned choices (ct_autotune), read from the tuning cache at plan
  // creation: this GPU's entries, one per (precision, instantiated radii,
  // x-extent class, size class) of a volume.  A choice applies to every box of
  // a volume alike (the key is the volume's), so chunks still reproduce it.
  struct TuneEntry {
    int precision, rs, rr, xclass, vlog2;
    int rho_path;      // 0: FP32 stencils; 1: tensor cores, products in the gradient kernel;
                       // 2: tensor cores, products formed in the first pass
    int seg_cap;       // tensor-core outputs per work unit at most (0: the default)
    int stream_block;  // stencil y / z outputs per thread block (0: the default)
    int eig_compact;   // masked eigen stage over compacted voxels (-1: the default)
    double ms;
  };
  std::vector<TuneEntry> tune;
  bool tune_forced = false;           // a CT_TUNE_* setting of the rho path set: the cache is not used
  const TuneEntry* trial = nullptr;   // ct_autotune's candidate under test
  // per-kernel timing (ct_plan_profile)
  bool profile = false;
  struct Rec {
    const char* name;
    cudaEvent_t a, b;
  };
  std::vector<Rec> recs;
};

namespace {

ct_status check_params(const ct_params* p) {
  if (!p) return fail(CT_ERR_INVALID, "params is NULL");
  if (!(p->sigma > 0.0) || !std::isfinite(p->sigma)) return fail(CT_ERR_INVALID, "sigma must be finite and > 0");
  if (!(p->rho > 0.0) || !std::isfinite(p->rho)) return fail(CT_ERR_INVALID, "rho must be finite and > 0");
  if (p->truncate < 0.0 || !std::isfinite(p->truncate)) return fail(CT_ERR_INVALID, "truncate must be >= 0");
  for (int k = 0; k < 3; ++k) {
    if (!std::isfinite(p->lv_center[k])) return fail(CT_ERR_INVALID, "lv_center must be finite");
    if (!std::isfinite(p->lv_axis[k])) return fail(CT_ERR_INVALID, "lv_axis must be finite");
  }
  if (p->lv_axis[0] == 0.0 && p->lv_axis[1] == 0.0 && p->lv_axis[2] == 0.0)
    return fail(CT_ERR_INVALID, "lv_axis must not be the zero vector");
  if (p->precision != CT_PREC_FP32 && p->precision != CT_PREC_MIXED) return fail(CT_ERR_INVALID, "bad precision");
  if (p->vec_type != CT_OUT_F32 && p->vec_type != CT_OUT_F16) return fail(CT_ERR_INVALID, "bad vec_type");
  if (p->angle_type < CT_OUT_F32 || p->angle_type > CT_OUT_U8Q) return fail(CT_ERR_INVALID, "bad angle_type");
  if (p->fa_type != CT_OUT_F32 && p->fa_type != CT_OUT_F16) return fail(CT_ERR_INVALID, "bad fa_type");
  if (p->flags != 0) return fail(CT_ERR_INVALID, "flags must be 0");
  for (int k = 0; k < 3; ++k)
    if (p->chunk[k] < 0) return fail(CT_ERR_INVALID, "chunk sizes must be >= 0");
  for (int k = 0; k < 3; ++k)
    if (!(p->spacing[k] >= 0.0) || !std::isfinite(p->spacing[k]))
      return fail(CT_ERR_INVALID, "spacing must be finite and >= 0 (0 = 1)");
  return CT_OK;
}

double trunc_of(const ct_params& p) { return p.truncate > 0.0 ? p.truncate : 4.0; }

ct_status make_scale(const ct_params& p, double sigma, double rho, Scale* s) {
  double tr = trunc_of(p), sp[3];
  spacing_of(p, sp);
  s->sigma = sigma;
  s->rho = rho;
  int ms = 0, mr = 0;
  for (int a = 0; a < 3; ++a) {
    s->rs[a] = radius_of(sigma / sp[a], tr);
    s->rr[a] = radius_of(rho / sp[a], tr);
    if (s->rs[a] < 1 || s->rr[a] < 1) return fail(CT_ERR_INVALID, "truncate * scale must give a radius >= 1");
    ms = std::max(ms, s->rs[a]);
    mr = std::max(mr, s->rr[a]);
    s->halo[a] = s->rs[a] + s->rr[a];
  }
  s->rks = sigma_kernel_radius(ms);
  s->rkr = rho_kernel_radius(mr);
  if (s->rks < 0) return fail(CT_ERR_UNSUPPORTED, "sigma radius %d exceeds 12", ms);
  if (s->rkr < 0) return fail(CT_ERR_UNSUPPORTED, "rho radius %d exceeds 36", mr);
  for (int a = 0; a < 3; ++a) {
    s->ts[a] = make_taps(sigma / sp[a], tr, s->rks);
    s->tr[a] = make_taps(rho / sp[a], tr, s->rkr);
  }
  static const int ca[6] = {0, 1, 2, 0, 0, 1}, cb[6] = {0, 1, 2, 1, 2, 2};
  for (int k = 0; k < 6; ++k) s->ss[k] = (float)(1.0 / (sp[ca[k]] * sp[cb[k]]));
  return CT_OK;
}

size_t elem_size(int type) { return type == CT_OUT_F32 ? 4 : (type == CT_OUT_F16 ? 2 : 1); }

ct_status ensure_device(void** ptr, size_t* cap, size_t need, const char* what) {
  if (*cap >= need && *ptr) return CT_OK;
  if (*ptr) cudaFree(*ptr);
  *ptr = nullptr;
  *cap = 0;
  CT_CUDA(cudaMalloc(ptr, std::max<size_t>(need, 256)), what);
  *cap = need;
  return CT_OK;
}

ct_status ensure_fallback(ct_plan P, int slot, int64_t vox) {
  if (!P->fb_count[slot]) CT_CUDA(cudaMalloc(&P->fb_count[slot], sizeof(int)), "counter allocation");
  if (!P->fb_total) {
    CT_CUDA(cudaMalloc(&P->fb_total, sizeof(unsigned long long)), "counter allocation");
    CT_CUDA(cudaMemset(P->fb_total, 0, sizeof(unsigned long long)), "counter reset");
  }
  if (P->fb_cap[slot] < vox) {
    if (P->fb_list[slot]) cudaFree(P->fb_list[slot]);
    P->fb_list[slot] = nullptr;
    P->fb_cap[slot] = 0;
    CT_CUDA(cudaMalloc(&P->fb_list[slot], sizeof(int64_t) * vox), "re-solve list allocation");
    P->fb_cap[slot] = vox;
  }
  return CT_OK;
}

ct_status ensure_scratch(ct_plan P, int slot, int64_t vox) {
  if (P->buf_cap[slot] < vox) {
    for (int k = 0; k < 2; ++k) {
      if (P->buf[slot][k]) cudaFree(P->buf[slot][k]);
      P->buf[slot][k] = nullptr;
    }
    P->buf_cap[slot] = 0;
    for (int k = 0; k < 2; ++k) CT_CUDA(cudaMalloc(&P->buf[slot][k], sizeof(float) * 6 * vox), "scratch allocation");
    P->buf_cap[slot] = vox;
  }
  return ensure_fallback(P, slot, vox);
}

Fallback fallback_of(ct_plan P, int slot) {
  Fallback fb;
  fb.count = P->fb_count[slot];
  fb.total = P->fb_total;
  fb.list = P->fb_list[slot];
  fb.cap = P->fb_cap[slot];
  fb.gap = degenerate_gap(P->p.precision == CT_PREC_MIXED);
  return fb;
}

// Remember that this plan enqueued work on stream st: an event recorded after
// it lets ct_plan_sync wait for exactly the plan's work.
ct_status mark(ct_plan P, cudaStream_t st) {
  for (auto& m : P->marks)
    if (m.first == st) {
      CT_CUDA(cudaEventRecord(m.second, st), "event record");
      return CT_OK;
    }
  cudaEvent_t ev = nullptr;
  CT_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "event creation");
  cudaError_t e = cudaEventRecord(ev, st);
  if (e != cudaSuccess) {
    cudaEventDestroy(ev);
    return cuda_fail(e, "event record");
  }
  P->marks.push_back({st, ev});
  return CT_OK;
}

// Wait for the plan's work (its own streams and those its calls used); then
// report a tensor-core CTA that gave up a bounded wait as CT_ERR_TIMEOUT.
ct_status sync_plan(ct_plan P) {
  cudaError_t e = cudaSuccess;
  for (auto& m : P->marks)
    if (e == cudaSuccess) e = cudaEventSynchronize(m.second);
  for (int k = 0; k < ct_plan_s::kSlots && e == cudaSuccess; ++k)
    if (P->st[k]) e = cudaStreamSynchronize(P->st[k]);
  if (e == cudaSuccess && P->gst) e = cudaStreamSynchronize(P->gst);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "device work");
  unsigned int n = 0;
  e = cudaMemcpyAsync(&n, P->d_timeouts, sizeof n, cudaMemcpyDeviceToHost, P->st[0]);
  if (e == cudaSuccess) e = cudaStreamSynchronize(P->st[0]);
  if (e == cudaSuccess && n) e = cudaMemsetAsync(P->d_timeouts, 0, sizeof n, P->st[0]);
  if (e == cudaSuccess && n) e = cudaStreamSynchronize(P->st[0]);
  if (e != cudaSuccess) return cuda_fail(e, "timeout word read");
  if (n)
    return fail(CT_ERR_TIMEOUT, "%u tensor-core CTAs gave up a bounded wait (their outputs are invalid)", n);
  return CT_OK;
}

// Launch `call` (a cudaError_t expression) bracketed by timing events when profiling.
#define CT_LAUNCH(P, st, name, call, what)                                  \
  do {                                                                      \
    cudaEvent_t a_ = nullptr, b_ = nullptr;                                 \
    const bool prof_ = (P)->profile && !(P)->capturing;                     \
    if (prof_) {                                                            \
      cudaEventCreate(&a_);                                                 \
      cudaEventCreate(&b_);                                                 \
      cudaEventRecord(a_, st);                                              \
    }                                                                       \
    cudaError_t e2_ = (call);                                               \
    if (prof_) {                                                            \
      cudaEventRecord(b_, st);                                              \
      (P)->recs.push_back({name, a_, b_});                                  \
    }                                                                       \
    if (e2_ != cudaSuccess) return cuda_fail(e2_, what);                    \
    (P)->stats.launches += 1;                                               \
  } while (0)

int x_class(int nx) { return nx % 8 == 0 ? 8 : (nx % 4 == 0 ? 4 : 1); }

int vox_log2(const int dims[3]) {
  const int64_t v = (int64_t)dims[0] * dims[1] * dims[2];
  int l = 0;
  while (l < 62 && (int64_t(1) << (l + 1)) <= v) ++l;
  return l;
}

// The autotuned choice for a volume of size dims at scale sc (nullptr: the
// defaults): the entry of the same precision, radii and x-extent class whose
// size class is nearest, within a factor of two either way.
const ct_plan_s::TuneEntry* tuned(const ct_plan P, const Scale& sc, const int dims[3]) {
  if (P->trial) return P->trial;
  if (P->tune_forced) return nullptr;
  const int xc = x_class(dims[0]), vl = vox_log2(dims);
  const ct_plan_s::TuneEntry* best = nullptr;
  for (const auto& t : P->tune) {
    if (t.precision != P->p.precision || t.rs != sc.rks || t.rr != sc.rkr || t.xclass != xc) continue;
    if (std::abs(t.vlog2 - vl) > 1) continue;
    if (!best || std::abs(t.vlog2 - vl) < std::abs(best->vlog2 - vl)) best = &t;
  }
  return best;
}

// Whether the rho pass along axis of a volume dims[] runs on the tensor cores:
// a function of the plan, the volume's extent and the scale, never of the box,
// so that every chunk and sub-box of a volume takes the same arithmetic as the
// whole and their results agree bit for bit.  Those passes are bound by HBM at
// 48 B per voxel with 16-byte copies (x extents that are multiples of 4) and
// several times slower otherwise; the FP32 stencils cost 6 (2R+1) FMAs per
// voxel and pass, so below R ~ 17 they are the faster, and on small volumes
// the persistent passes' start-up outweighs them (one step: 200^3 0.87 ms on
// the tensor cores against 0.72 on the stencils; 256^3 0.98 against 1.12;
// 384^3 2.70 against 3.34; 400^3 3.91 against 4.23; 200 uneven crops, all on
// the tensor cores where the extent allows, 167 ms against 164).  tc_any_box
// drops the extent and size conditions (tests drive every copy path with it).
bool use_tc(const ct_plan P, const Scale& sc, const int dims[3], int axis) {
  if (const auto* t = tuned(P, sc, dims)) return t->rho_path > 0;
  const int64_t vox = (int64_t)dims[0] * dims[1] * dims[2];
  return (P->tc_rho >> axis & 1) && sc.rkr >= P->tc_min_r &&
         (P->tc_any_box || (rho_tc_volume_aligned(dims[0], axis) && vox >= P->tc_min_vox));
}

// The structure tensor S (6 planes over ob) of vol (covering vb): the gradient
// at sigma, its products and the three rho passes (Figure 1b).  S goes to
// S_out when given (the stage API), else to a scratch buffer; *S_res tells
// which.  Two chains, chosen per plan and volume, never per box, so that
// chunks and sub-boxes of a volume reproduce it bit for bit:
//   - every rho pass on the tensor cores (and products in the first pass,
//     the plan's default): the gradient g (FP16 in the mixed form) goes to
//     HBM instead of the six products; the z pass forms the products as it
//     stages them, then the y and x passes follow:
//       grad_xy -> B, grad_z: g -> A, z: S_z -> B, y: S_zy -> A, x: S -> out;
//   - otherwise the products J and the x, y passes (tensor cores per axis, or
//     the fused FP32 stencil), then the z pass:
//       grad_xy -> B, grad_z: J -> A, x / y -> B or A, z -> out.
ct_status smooth_chain(ct_plan P, const Scale& sc, const int dims[3], const uint16_t* vol, const Box& vb,
                       const Box& ob, int slot, bool mixed, cudaStream_t st, float* S_out, float** S_res) {
  const Box G = grow_clip3(ob, sc.rr, dims);
  // the gradient keeps its 3 partial planes (over G grown in z) in B
  const Box Ab = grad_partial_box(G, vb, sc.rks, dims[2]);
  const int64_t need = std::max<int64_t>(box_vox(G), (box_vox(Ab) + 1) / 2);
  ct_status rc = ensure_scratch(P, slot, need);
  if (rc) return rc;
  float* A = P->buf[slot][0];
  float* B = P->buf[slot][1];
  const auto* tuning = tuned(P, sc, dims);
  const TcCtl ctl{P->d_timeouts, P->tc_wait_limit, tuning ? tuning->seg_cap : 0};
  const int sblock = tuning && tuning->stream_block ? tuning->stream_block : P->stream_block;
  CT_LAUNCH(P, st, "grad_xy", launch_grad_xy(vol, vb, dims, B, Ab, sc.ts[0], sc.ts[1], sc.rks, st),
            "gradient x/y kernel launch");
  const bool tcx = use_tc(P, sc, dims, 0), tcy = use_tc(P, sc, dims, 1), tcz = use_tc(P, sc, dims, 2);
  if (tcx && tcy && tcz && (tuning ? tuning->rho_path == 2 : P->tc_products)) {
    Box Bz = G, Bzy = G;
    Bz.lo[2] = Bzy.lo[2] = ob.lo[2];
    Bz.n[2] = Bzy.n[2] = ob.n[2];
    Bzy.lo[1] = ob.lo[1];
    Bzy.n[1] = ob.n[1];
    float* S = S_out ? S_out : B;
    CT_LAUNCH(P, st, mixed ? "grad_z_g16" : "grad_z_g32",
              launch_grad_z(B, Ab, A, G, sc.ts[2], sc.ss, sc.rks, mixed, true, st), "gradient z kernel launch");
    CT_LAUNCH(P, st, mixed ? "rho_z_tc_g16" : "rho_z_tc_g32",
              launch_rho_tc_products(A, mixed, G, dims, B, Bz, 2, sc.tr[2], sc.ss, sc.rkr, ctl, st),
              "rho z kernel launch");
    CT_LAUNCH(P, st, "rho_y_tc", launch_rho_tc(B, Bz, dims, A, Bzy, 1, sc.tr[1], sc.rkr, ctl, st),
              "rho y kernel launch");
    CT_LAUNCH(P, st, "rho_x_tc", launch_rho_tc(A, Bzy, dims, S, ob, 0, sc.tr[0], sc.rkr, ctl, st),
              "rho x kernel launch");
    *S_res = S;
    return CT_OK;
  }
  Box Bx = G, Bxy = G;
  Bx.lo[0] = Bxy.lo[0] = ob.lo[0];
  Bx.n[0] = Bxy.n[0] = ob.n[0];
  Bxy.lo[1] = ob.lo[1];
  Bxy.n[1] = ob.n[1];
  CT_LAUNCH(P, st, "grad_z", launch_grad_z(B, Ab, A, G, sc.ts[2], sc.ss, sc.rks, mixed, false, st),
            "gradient z kernel launch");
  // x and y on the tensor cores together, or as one fused FP32 stencil; a mask
  // that selects one of the two axes (tuning, tests) runs them as separate passes
  const bool one_axis = (P->tc_rho & 3) == 1 || (P->tc_rho & 3) == 2;
  float* Sxy;
  if ((tcx && tcy) || (one_axis && (tcx || tcy))) {
    if (tcx)
      CT_LAUNCH(P, st, "rho_x_tc", launch_rho_tc(A, G, dims, B, Bx, 0, sc.tr[0], sc.rkr, ctl, st),
                "rho x kernel launch");
    else
      CT_LAUNCH(P, st, "rho_x", launch_rho_x(A, G, dims, B, Bx, sc.tr[0], sc.rkr, st), "rho x kernel launch");
    if (tcy)
      CT_LAUNCH(P, st, "rho_y_tc", launch_rho_tc(B, Bx, dims, A, Bxy, 1, sc.tr[1], sc.rkr, ctl, st),
                "rho y kernel launch");
    else
      CT_LAUNCH(P, st, "rho_y", launch_rho_stream(B, Bx, dims, A, Bxy, 1, sc.tr[1], sc.rkr, sblock, st),
                "rho y kernel launch");
    Sxy = A;
  } else {
    CT_LAUNCH(P, st, "rho_xy", launch_rho_xy(A, G, dims, B, Bxy, sc.tr[0], sc.tr[1], sc.rkr, st), "rho xy kernel launch");
    Sxy = B;
  }
  float* S = S_out ? S_out : (Sxy == A ? B : A);
  if (tcz)
    CT_LAUNCH(P, st, "rho_z_tc", launch_rho_tc(Sxy, Bxy, dims, S, ob, 2, sc.tr[2], sc.rkr, ctl, st),
              "rho z kernel launch");
  else
    CT_LAUNCH(P, st, "rho_z", launch_rho_stream(Sxy, Bxy, dims, S, ob, 2, sc.tr[2], sc.rkr, sblock, st),
              "rho z kernel launch");
  *S_res = S;
  return CT_OK;
}

// The whole smoothing chain into S (6 planes over ob): the stage API.
ct_status tensor_stages(ct_plan P, const Scale& sc, const int dims[3], const uint16_t* vol, const Box& vb,
                        const Box& ob, float* S_out, int slot, bool mixed, cudaStream_t st) {
  float* S = nullptr;
  return smooth_chain(P, sc, dims, vol, vb, ob, slot, mixed, st, S_out, &S);
}

ct_status eig_stage(ct_plan P, const float* S, const Box& ob, const uint8_t* mask, const Box& mb, const Frame& F,
                    const EigOut& o, int slot, bool mixed, bool compact, cudaStream_t st);

// The fused hot path (Figure 1b, c): gradient and products, the three rho
// passes into the free scratch buffer, then eigen + angles + mask + encode and
// the re-solve of the listed voxels.  Outputs in arrays covering o.ab.
ct_status fused_stages(ct_plan P, const Scale& sc, const int dims[3], const uint16_t* vol, const Box& vb,
                       const Box& ob, const uint8_t* mask, const Box& mb, const Frame& F, const EigOut& o, int slot,
                       bool mixed, cudaStream_t st) {
  float* S = nullptr;
  ct_status rc = smooth_chain(P, sc, dims, vol, vb, ob, slot, mixed, st, nullptr, &S);
  if (rc) return rc;
  const auto* t = tuned(P, sc, dims);
  return eig_stage(P, S, ob, mask, mb, F, o, slot, mixed, t && t->eig_compact >= 0 ? t->eig_compact != 0 : P->eig_compact,
                   st);
}

// Eigen + angles over ob from S (over ob); outputs in arrays covering o.ab.
ct_status eig_stage(ct_plan P, const float* S, const Box& ob, const uint8_t* mask, const Box& mb, const Frame& F,
                    const EigOut& o, int slot, bool mixed, bool compact, cudaStream_t st) {
  Fallback fb = fallback_of(P, slot);
  CT_CUDA(cudaMemsetAsync(fb.count, 0, sizeof(int), st), "counter reset");
  CT_LAUNCH(P, st, "eig_angles",
            launch_eig_angles(S, ob, ob, mask, mb, F, P->p.fill_value, o, mixed, fb, compact, st),
            "eigen kernel launch");
  CT_LAUNCH(P, st, "eig_resolve",
            launch_eig_angles_fallback(S, ob, ob, mask, mb, F, P->p.fill_value, o, mixed, fb, box_vox(ob), st),
            "re-solve kernel launch");
  return CT_OK;
}

// ------------------------------------------------------------ tuning cache
// A JSON array, one object per line, written by ct_autotune:
//   {"gpu": "<device name>", "precision": p, "rs": R_sigma, "rr": R_rho,
//    "xclass": 8|4|1, "vox_log2": l, "rho_path": 0|1|2, "seg_cap": n,
//    "stream_block": n, "eig_compact": -1|0|1, "ms": t}
struct CacheLine {
  std::string gpu;
  ct_plan_s::TuneEntry e;
};

std::string default_cache_path() {
  Dl_info info;
  if (dladdr(reinterpret_cast<void*>(&ct_radius), &info) && info.dli_fname) {
    const std::string so = info.dli_fname;  // <package>/_build/libct_gb300.so
    const size_t k = so.rfind('/');
    return (k == std::string::npos ? std::string(".") : so.substr(0, k)) + "/../tuning/tune_cache.json";
  }
  return "";
}

// CT_TUNE_CACHE names the cache ("" disables it); else the package's own.
std::string cache_path() {
  if (const char* e = std::getenv("CT_TUNE_CACHE")) return e;
  return default_cache_path();
}

std::string gpu_name(int dev) {
  cudaDeviceProp pr;
  if (cudaGetDeviceProperties(&pr, dev) != cudaSuccess) {
    cudaGetLastError();
    return "";
  }
  return pr.name;
}

bool json_num(const std::string& line, const char* key, double* v) {
  const std::string k = std::string("\"") + key + "\":";
  const size_t p = line.find(k);
  if (p == std::string::npos) return false;
  const char* b = line.c_str() + p + k.size();
  char* end = nullptr;
  *v = std::strtod(b, &end);
  return end != b;
}

bool json_str(const std::string& line, const char* key, std::string* v) {
  const std::string k = std::string("\"") + key + "\":";
  size_t p = line.find(k);
  if (p == std::string::npos) return false;
  p = line.find('"', p + k.size());
  if (p == std::string::npos) return false;
  const size_t q = line.find('"', p + 1);
  if (q == std::string::npos) return false;
  *v = line.substr(p + 1, q - p - 1);
  return true;
}

std::vector<CacheLine> read_cache(const std::string& path) {
  std::vector<CacheLine> out;
  std::ifstream f(path);
  std::string line;
  while (f && std::getline(f, line)) {
    if (line.find('{') == std::string::npos) continue;
    CacheLine c;
    double v[10];
    static const char* keys[10] = {"precision", "rs", "rr", "xclass", "vox_log2", "rho_path", "seg_cap",
                                   "stream_block", "eig_compact", "ms"};
    bool ok = json_str(line, "gpu", &c.gpu);
    for (int k = 0; k < 10 && ok; ++k) ok = json_num(line, keys[k], &v[k]);
    if (!ok) continue;
    c.e = {(int)v[0], (int)v[1], (int)v[2], (int)v[3], (int)v[4], (int)v[5], (int)v[6], (int)v[7], (int)v[8], v[9]};
    out.push_back(c);
  }
  return out;
}

bool same_key(const ct_plan_s::TuneEntry& a, const ct_plan_s::TuneEntry& b) {
  return a.precision == b.precision && a.rs == b.rs && a.rr == b.rr && a.xclass == b.xclass && a.vlog2 == b.vlog2;
}

bool write_cache(const std::string& path, const std::vector<CacheLine>& lines) {
  const std::string tmp = path + ".tmp";
  {
    std::ofstream f(tmp);
    if (!f) return false;
    f << "[\n";
    for (size_t i = 0; i < lines.size(); ++i) {
      const auto& e = lines[i].e;
      char buf[512];
      std::snprintf(buf, sizeof buf,
                    "{\"gpu\": \"%s\", \"precision\": %d, \"rs\": %d, \"rr\": %d, \"xclass\": %d, "
                    "\"vox_log2\": %d, \"rho_path\": %d, \"seg_cap\": %d, \"stream_block\": %d, "
                    "\"eig_compact\": %d, \"ms\": %.4f}",
                    lines[i].gpu.c_str(), e.precision, e.rs, e.rr, e.xclass, e.vlog2, e.rho_path, e.seg_cap,
                    e.stream_block, e.eig_compact, e.ms);
      f << buf << (i + 1 < lines.size() ? ",\n" : "\n");
    }
    f << "]\n";
    if (!f) return false;
  }
  return std::rename(tmp.c_str(), path.c_str()) == 0;
}

}  // namespace

extern "C" {

int32_t ct_radius(double s, double truncate) {
  if (!(s > 0.0) || !(truncate >= 0.0)) return -1;
  return radius_of(s, truncate > 0.0 ? truncate : 4.0);
}

const char* ct_last_error(void) { return g_err.c_str(); }

ct_status ct_plan_create(const ct_params* params, const int64_t vol_dims[3], ct_plan* out) {
  if (!out) return fail(CT_ERR_INVALID, "out is NULL");
  *out = nullptr;
  ct_status rc = check_params(params);
  if (rc) return rc;
  if (!vol_dims) return fail(CT_ERR_INVALID, "vol_dims is NULL");
  for (int k = 0; k < 3; ++k)
    if (vol_dims[k] < 1 || vol_dims[k] > (1 << 20)) return fail(CT_ERR_INVALID, "vol_dims must be in [1, 2^20]");
  Scale sc;
  if ((rc = make_scale(*params, params->sigma, params->rho, &sc))) return rc;
  if (!device_present()) return fail(CT_ERR_NO_DEVICE, "no CUDA device is available");
  {
    cudaError_t e = prepare_rho_xy_kernels();
    if (e == cudaSuccess) e = prepare_grad_split_kernels();
    if (e == cudaSuccess) e = prepare_rho_tc_kernels();
    if (e != cudaSuccess) return cuda_fail(e, "kernel attribute set-up");
  }
  ct_plan P = new (std::nothrow) ct_plan_s();
  if (!P) return fail(CT_ERR_OOM, "plan allocation failed");
  P->p = *params;
  P->p.lv_centres = nullptr;  // the caller's array is copied below, not kept
  for (int k = 0; k < 3; ++k) P->dims[k] = (int)vol_dims[k];
  spacing_of(*params, P->sp);
  if (params->lv_centres) {
    std::vector<float> c((size_t)2 * P->dims[2]);
    for (size_t i = 0; i < c.size(); ++i) {
      if (!std::isfinite(params->lv_centres[i])) {
        delete P;
        return fail(CT_ERR_INVALID, "lv_centres must be finite");
      }
      c[i] = (float)params->lv_centres[i];
    }
    cudaError_t e = cudaMalloc(&P->d_centres, sizeof(float) * c.size());
    if (e == cudaSuccess) e = cudaMemcpy(P->d_centres, c.data(), sizeof(float) * c.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      if (P->d_centres) cudaFree(P->d_centres);
      delete P;
      return cuda_fail(e, "centreline copy");
    }
  }
  std::memset(&P->stats, 0, sizeof P->stats);
  if (const char* e = std::getenv("CT_TUNE_STREAM_BLOCK")) P->stream_block = std::atoi(e) == 8 ? 8 : 16;
  if (const char* e = std::getenv("CT_TUNE_TC_RHO")) P->tc_rho = std::atoi(e) & 7;
  if (const char* e = std::getenv("CT_TUNE_TC_ANY_BOX")) P->tc_any_box = std::atoi(e) != 0;
  if (const char* e = std::getenv("CT_TUNE_TC_MIN_VOX")) P->tc_min_vox = std::max<int64_t>(0, std::atoll(e));
  if (const char* e = std::getenv("CT_TUNE_EIG_COMPACT")) P->eig_compact = std::atoi(e) != 0;
  if (const char* e = std::getenv("CT_TUNE_SLAB_BYTES")) P->slab_bytes = std::max<int64_t>(0, std::atoll(e));
  if (const char* e = std::getenv("CT_TUNE_TC_MIN_R")) P->tc_min_r = std::max(0, std::atoi(e));
  if (const char* e = std::getenv("CT_TUNE_BATCH_STREAMS"))
    P->batch_streams = std::max(1, std::min(ct_plan_s::kSlots, std::atoi(e)));
  if (const char* e = std::getenv("CT_TUNE_BATCH_GRAPH")) P->batch_graph = std::atoi(e) != 0;
  if (const char* e = std::getenv("CT_TUNE_BATCH_PERSISTENT")) P->batch_persistent = std::atoi(e) != 0;
  if (const char* e = std::getenv("CT_TUNE_BATCH_BYTES")) P->batch_bytes = std::max<int64_t>(1, std::atoll(e));
  if (const char* e = std::getenv("CT_TUNE_TC_WAIT_LIMIT")) P->tc_wait_limit = (uint32_t)std::max(0, std::atoi(e));
  if (const char* e = std::getenv("CT_TUNE_TC_PRODUCTS")) P->tc_products = std::atoi(e) != 0;
  for (const char* k : {"CT_TUNE_TC_RHO", "CT_TUNE_TC_MIN_R", "CT_TUNE_TC_MIN_VOX", "CT_TUNE_TC_ANY_BOX",
                        "CT_TUNE_TC_PRODUCTS", "CT_TUNE_STREAM_BLOCK", "CT_TUNE_EIG_COMPACT"})
    if (std::getenv(k)) P->tune_forced = true;
  cudaGetDevice(&P->device);
  if (!P->tune_forced) {
    const std::string path = cache_path(), gpu = gpu_name(P->device);
    if (!path.empty())
      for (const auto& c : read_cache(path))
        if (c.gpu == gpu) P->tune.push_back(c.e);
  }
  {
    cudaError_t e = cudaMalloc(&P->d_timeouts, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemset(P->d_timeouts, 0, sizeof(unsigned int));
    if (e != cudaSuccess) {
      ct_plan_destroy(P);
      return cuda_fail(e, "timeout word allocation");
    }
  }
  for (int k = 0; k < 2; ++k) {
    cudaError_t e = cudaStreamCreateWithFlags(&P->st[k], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->ev[k], cudaEventDisableTiming);
    if (e != cudaSuccess) {
      ct_plan_destroy(P);
      return cuda_fail(e, "stream creation");
    }
  }
  *out = P;
  return CT_OK;
}

ct_status ct_plan_destroy(ct_plan P) {
  if (!P) return CT_OK;
  cudaDeviceSynchronize();
  if (P->d_centres) cudaFree(P->d_centres);
  if (P->d_timeouts) cudaFree(P->d_timeouts);
  for (auto& m : P->marks) cudaEventDestroy(m.second);
  if (P->graph_exec) cudaGraphExecDestroy(P->graph_exec);
  if (P->graph) cudaGraphDestroy(P->graph);
  if (P->gst) cudaStreamDestroy(P->gst);
  if (P->arena) cudaFree(P->arena);
  if (P->tables) cudaFree(P->tables);
  for (int k = 0; k < ct_plan_s::kSlots; ++k)
    if (P->wev[k]) cudaEventDestroy(P->wev[k]);
  for (int k = 0; k < 2; ++k)
    if (P->gev[k]) cudaEventDestroy(P->gev[k]);
  for (int s = 0; s < ct_plan_s::kSlots; ++s) {
    for (int k = 0; k < 2; ++k)
      if (P->buf[s][k]) cudaFree(P->buf[s][k]);
    if (P->fb_count[s]) cudaFree(P->fb_count[s]);
    if (P->fb_list[s]) cudaFree(P->fb_list[s]);
    if (s < 2) {
      if (P->d_in[s]) cudaFree(P->d_in[s]);
      if (P->d_mask[s]) cudaFree(P->d_mask[s]);
      if (P->d_out[s]) cudaFree(P->d_out[s]);
      if (P->h_in[s]) cudaFreeHost(P->h_in[s]);
      if (P->h_out[s]) cudaFreeHost(P->h_out[s]);
    }
    if (P->st[s]) cudaStreamDestroy(P->st[s]);
    if (P->ev[s]) cudaEventDestroy(P->ev[s]);
  }
  if (P->fb_total) cudaFree(P->fb_total);
  for (auto& r : P->recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  delete P;
  return CT_OK;
}

ct_status ct_structure_tensor(ct_plan P, const uint16_t* d_vol, const int64_t in_lo[3], const int64_t in_n[3],
                              const int64_t out_lo[3], const int64_t out_n[3], float* d_S, void* stream) {
  if (!P) return fail(CT_ERR_INVALID, "plan is NULL");
  if (!d_vol || !d_S || !in_lo || !in_n || !out_lo || !out_n) return fail(CT_ERR_INVALID, "NULL argument");
  if (!valid_box(in_lo, in_n, P->dims)) return fail(CT_ERR_INVALID, "input box outside the volume");
  if (!valid_box(out_lo, out_n, P->dims)) return fail(CT_ERR_INVALID, "output box outside the volume");
  std::lock_guard<std::mutex> lk(P->mu);
  Scale sc;
  ct_status rc = make_scale(P->p, P->p.sigma, P->p.rho, &sc);
  if (rc) return rc;
  Box ib = make_box(in_lo, in_n), ob = make_box(out_lo, out_n);
  if (!inside(ib, grow_clip3(ob, sc.halo, P->dims)))
    return fail(CT_ERR_INVALID, "input box must contain the output box grown by R(sigma)+R(rho) = (%d, %d, %d) (clipped)",
                sc.halo[0], sc.halo[1], sc.halo[2]);
  rc = tensor_stages(P, sc, P->dims, d_vol, ib, ob, d_S, 0, P->p.precision == CT_PREC_MIXED,
                     (cudaStream_t)stream);
  if (rc) return rc;
  P->stats.voxels += box_vox(ob);
  return mark(P, (cudaStream_t)stream);
}

ct_status ct_eig_smallest(ct_plan P, const float* d_S, int64_t n, float* d_evals, float* d_evec, void* stream) {
  if (!P) return fail(CT_ERR_INVALID, "plan is NULL");
  if (!d_S || !d_evec) return fail(CT_ERR_INVALID, "NULL argument");
  if (n < 0) return fail(CT_ERR_INVALID, "n must be >= 0");
  if (n == 0) return CT_OK;
  std::lock_guard<std::mutex> lk(P->mu);
  cudaStream_t st = (cudaStream_t)stream;
  ct_status rc = ensure_fallback(P, 0, n);
  if (rc) return rc;
  Fallback fb = fallback_of(P, 0);
  bool mixed = P->p.precision == CT_PREC_MIXED;
  CT_CUDA(cudaMemsetAsync(fb.count, 0, sizeof(int), st), "counter reset");
  CT_LAUNCH(P, st, "eig_only", launch_eig_only(d_S, n, d_evals, d_evec, mixed, fb, st), "eigen kernel launch");
  CT_LAUNCH(P, st, "eig_only_resolve", launch_eig_only_fallback(d_S, n, d_evals, d_evec, mixed, fb, n, st),
            "re-solve kernel launch");
  return mark(P, st);
}

ct_status ct_angles(ct_plan P, const float* d_evec, const float* d_evals, const int64_t out_lo[3],
                    const int64_t out_n[3], const uint8_t* d_mask, void* d_vec, void* d_ha, void* d_ia, void* d_fa,
                    void* stream) {
  if (!P) return fail(CT_ERR_INVALID, "plan is NULL");
  if (!d_evec || !d_evals || !out_lo || !out_n) return fail(CT_ERR_INVALID, "NULL argument");
  if (!valid_box(out_lo, out_n, P->dims)) return fail(CT_ERR_INVALID, "output box outside the volume");
  std::lock_guard<std::mutex> lk(P->mu);
  Box ob = make_box(out_lo, out_n);
  EigOut o{d_vec, d_ha, d_ia, d_fa, P->p.vec_type, P->p.angle_type, P->p.fa_type, ob};
  Frame F = make_frame(P->p.lv_center, P->p.lv_axis, P->sp, P->d_centres);
  cudaStream_t st = (cudaStream_t)stream;
  CT_LAUNCH(P, st, "angles_only", launch_angles_only(d_evec, d_evals, ob, d_mask, F, P->p.fill_value, o, st),
            "angles kernel launch");
  return mark(P, st);
}

}  // extern "C"

namespace {

// Chunk grid over dims with chunk sizes (0 = whole extent).
std::vector<Box> chunk_grid(const int dims[3], const int64_t chunk[3]) {
  int cs[3];
  for (int a = 0; a < 3; ++a) cs[a] = chunk[a] > 0 ? (int)std::min<int64_t>(chunk[a], dims[a]) : dims[a];
  std::vector<Box> out;
  for (int z = 0; z < dims[2]; z += cs[2])
    for (int y = 0; y < dims[1]; y += cs[1])
      for (int x = 0; x < dims[0]; x += cs[0]) {
        Box b;
        b.lo[0] = x; b.lo[1] = y; b.lo[2] = z;
        b.n[0] = std::min(cs[0], dims[0] - x);
        b.n[1] = std::min(cs[1], dims[1] - y);
        b.n[2] = std::min(cs[2], dims[2] - z);
        out.push_back(b);
      }
  return out;
}

// 3D copy of box `b` between an array covering `arr` (x-fastest, element size
// esz) and a dense array covering exactly `b`.
cudaError_t copy_box(const void* src, void* dst, const Box& arr, const Box& b, size_t esz, bool to_device,
                     cudaStream_t st) {
  cudaMemcpy3DParms p;
  std::memset(&p, 0, sizeof p);
  cudaPitchedPtr whole = make_cudaPitchedPtr(const_cast<void*>(to_device ? src : dst), esz * arr.n[0], arr.n[0],
                                             arr.n[1]);
  cudaPitchedPtr dense = make_cudaPitchedPtr(const_cast<void*>(to_device ? dst : src), esz * b.n[0], b.n[0], b.n[1]);
  cudaPos pos = make_cudaPos(esz * (b.lo[0] - arr.lo[0]), b.lo[1] - arr.lo[1], b.lo[2] - arr.lo[2]);
  if (to_device) {
    p.srcPtr = whole;
    p.srcPos = pos;
    p.dstPtr = dense;
    p.kind = cudaMemcpyHostToDevice;
  } else {
    p.srcPtr = dense;
    p.dstPtr = whole;
    p.dstPos = pos;
    p.kind = cudaMemcpyDeviceToHost;
  }
  p.extent = make_cudaExtent(esz * b.n[0], b.n[1], b.n[2]);
  return cudaMemcpy3DAsync(&p, st);
}

struct ItemCtx {
  Scale sc;
  Frame F;
  int dims[3];
  Box whole;
};

ct_status item_ctx(ct_plan P, const ct_item& it, ItemCtx* c) {
  for (int k = 0; k < 3; ++k) {
    if (it.dims[k] < 1 || it.dims[k] > (1 << 20)) return fail(CT_ERR_INVALID, "item dims must be in [1, 2^20]");
    c->dims[k] = (int)it.dims[k];
    c->whole.lo[k] = 0;
    c->whole.n[k] = (int)it.dims[k];
  }
  if (!it.vol) return fail(CT_ERR_INVALID, "item volume is NULL");
  double sig = it.sigma > 0.0 ? it.sigma : P->p.sigma;
  double rho = it.rho > 0.0 ? it.rho : P->p.rho;
  ct_status rc = make_scale(P->p, sig, rho, &c->sc);
  if (rc) return rc;
  bool own_axis = it.lv_axis[0] != 0.0 || it.lv_axis[1] != 0.0 || it.lv_axis[2] != 0.0;
  for (int k = 0; k < 3; ++k)
    if (!std::isfinite(it.lv_center[k]) || !std::isfinite(it.lv_axis[k]))
      return fail(CT_ERR_INVALID, "item frame must be finite");
  // an item with its own frame has no centreline (the plan's belongs to the plan's volume)
  c->F = own_axis ? make_frame(it.lv_center, it.lv_axis, P->sp, nullptr)
                  : make_frame(P->p.lv_center, P->p.lv_axis, P->sp, P->d_centres);
  return CT_OK;
}

// Output planes per item: (pointer, element size, planes).
struct OutPlanes {
  void* ptr[4];
  size_t esz[4];
  int planes[4];
};

OutPlanes out_planes(ct_plan P, const ct_item& it) {
  OutPlanes o;
  o.ptr[0] = it.vec; o.esz[0] = elem_size(P->p.vec_type); o.planes[0] = 3;
  o.ptr[1] = it.ha; o.esz[1] = elem_size(P->p.angle_type); o.planes[1] = 1;
  o.ptr[2] = it.ia; o.esz[2] = elem_size(P->p.angle_type); o.planes[2] = 1;
  o.ptr[3] = it.fa; o.esz[3] = elem_size(P->p.fa_type); o.planes[3] = 1;
  return o;
}

ct_status run_device_item(ct_plan P, const ct_item& it, cudaStream_t st) {
  ItemCtx c;
  ct_status rc = item_ctx(P, it, &c);
  if (rc) return rc;
  bool mixed = P->p.precision == CT_PREC_MIXED;
  for (const Box& ob : chunk_grid(c.dims, P->p.chunk)) {
    EigOut o{it.vec, it.ha, it.ia, it.fa, P->p.vec_type, P->p.angle_type, P->p.fa_type, c.whole};
    if ((rc = fused_stages(P, c.sc, c.dims, it.vol, c.whole, ob, it.mask, c.whole, c.F, o, 0, mixed, st))) return rc;
    P->stats.voxels += box_vox(ob);
  }
  return CT_OK;
}

ct_status ensure_stream(ct_plan P, int k) {
  if (!P->st[k]) {
    CT_CUDA(cudaStreamCreateWithFlags(&P->st[k], cudaStreamNonBlocking), "stream creation");
    CT_CUDA(cudaEventCreateWithFlags(&P->ev[k], cudaEventDisableTiming), "event creation");
  }
  return CT_OK;
}

uint64_t fnv1a(uint64_t h, const void* data, size_t n) {
  const unsigned char* p = static_cast<const unsigned char*>(data);
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}

// ---------------------------------------------------------- persistent batches
// The stencil-chain items of a batch run as one persistent launch per stage
// and tap set (template radius and taps) over every item of a wave: the CTAs
// take (item, block) work from a device counter, so items of any size share
// the SMs.  The items of one tap set form a chain (gradient x/y, gradient z,
// rho x/y, rho z) that runs in order on one of the plan's streams, chains side
// by side; the eigen stage of the whole wave follows them.  A wave holds the items whose scratch (the two tensor
// buffers and the re-solve list) fits the plan's batch_bytes; waves reuse the
// arena in stream order.  Every item's blocks, launch shape and arithmetic are
// those of its single launch, so a batch reproduces each item alone bit for
// bit.  The launch records (tables in device memory, uploaded before any
// capture) are built here; run_persistent_waves enqueues them.
struct MultiRec {
  int kind;          // 0 grad_xy, 1 grad_z, 2 rho_xy, 3 rho_z, 4 eigen (compact), 5 eigen (per voxel)
  int chain;         // stencil stages: the chain (tap sets) whose four launches run in order on one stream
  int rk, xt, block_t;
  bool plain;
  dim3 block;
  Taps t0, t1;
  float ss[6];
  size_t items_off, first_off, grids_off, counter_off;
  int n;
  int64_t blocks;
};

struct WaveRec {
  std::vector<MultiRec> launches;
  size_t counters_off = 0, n_counters = 0;  // per-launch work counters, zeroed per wave
  size_t fbc_off = 0, n_fbc = 0;            // re-solve list counters
  size_t eig_items_off = 0;                 // every eigen item of the wave, contiguous
  int n_eig = 0;
  int n_chains = 0;
  int64_t max_vox = 0;
};

struct HostTable {
  std::vector<unsigned char> bytes;
  template <typename T>
  size_t put(const T* p, size_t n) {
    const size_t off = (bytes.size() + 15) / 16 * 16;
    bytes.resize(off + sizeof(T) * n);
    if (n) std::memcpy(bytes.data() + off, p, sizeof(T) * n);
    return off;
  }
  size_t zeros(size_t nbytes) {
    const size_t off = (bytes.size() + 15) / 16 * 16;
    bytes.resize(off + nbytes, 0);
    return off;
  }
};

// Group the wave's items of one stage by a key and append one launch record per group.
template <typename Item, typename KeyEq, typename Fill>
void add_groups(HostTable& H, WaveRec& W, std::vector<Item>& items, std::vector<uint3>& grids,
                std::vector<MultiRec>& proto, KeyEq same, Fill fill) {
  std::vector<bool> done(items.size(), false);
  for (size_t i = 0; i < items.size(); ++i) {
    if (done[i]) continue;
    std::vector<Item> gi;
    std::vector<uint3> gg;
    std::vector<int64_t> first(1, 0);
    for (size_t j = i; j < items.size(); ++j) {
      if (done[j] || !same(proto[i], proto[j])) continue;
      done[j] = true;
      gi.push_back(items[j]);
      gg.push_back(grids[j]);
      first.push_back(first.back() + (int64_t)grids[j].x * grids[j].y * grids[j].z);
    }
    MultiRec r = proto[i];
    r.n = (int)gi.size();
    r.blocks = first.back();
    r.items_off = H.put(gi.data(), gi.size());
    r.first_off = H.put(first.data(), first.size());
    r.grids_off = H.put(gg.data(), gg.size());
    r.counter_off = 0;  // set when the wave's counters are laid out
    fill(r);
    W.launches.push_back(r);
  }
}

bool same_taps(const Taps& a, const Taps& b) { return std::memcmp(&a, &b, sizeof(Taps)) == 0; }

// Scratch of one item in a persistent wave: A, B (6 planes each of need voxels) and its re-solve list.
int64_t item_scratch_bytes(const ItemCtx& c) {
  const Box G = grow_clip3(c.whole, c.sc.rr, c.dims);
  const Box Ab = grad_partial_box(G, c.whole, c.sc.rks, c.dims[2]);
  const int64_t need = std::max<int64_t>(box_vox(G), (box_vox(Ab) + 1) / 2);
  return 2 * (int64_t)sizeof(float) * 6 * need + (int64_t)sizeof(int64_t) * box_vox(c.whole) + 1024;
}

// Build the waves of the items listed in `which` (indices into items / ctx).
ct_status build_persistent_waves(ct_plan P, const ct_item* items, const std::vector<ItemCtx>& ctx,
                                 const std::vector<int>& which, std::vector<WaveRec>* waves, HostTable* H,
                                 size_t* arena_need) {
  const bool mixed = P->p.precision == CT_PREC_MIXED;
  *arena_need = 0;
  size_t k = 0;
  while (k < which.size()) {
    // the wave: items in order while their scratch fits the budget (one at least)
    std::vector<int> wv;
    int64_t bytes = 0;
    while (k < which.size()) {
      const int64_t b = item_scratch_bytes(ctx[which[k]]);
      if (!wv.empty() && bytes + b > P->batch_bytes) break;
      wv.push_back(which[k]);
      bytes += b;
      ++k;
    }
    *arena_need = std::max(*arena_need, (size_t)bytes);
    WaveRec W;
    std::vector<GxyItem> gxy;
    std::vector<GzItem> gz;
    std::vector<RxyItem> rxy;
    std::vector<RzItem> rz;
    std::vector<EigItem> eig;
    std::vector<uint3> g_gxy, g_gz, g_rxy, g_rz, g_eig;
    std::vector<MultiRec> p_gxy, p_gz, p_rxy, p_rz, p_eig;
    // the chain of each item: equal radii, taps, product scales and z-block outputs
    std::vector<int> chain_of;
    std::vector<int> chain_rep;  // an item of each chain
    for (int idx : wv) {
      const ItemCtx& c = ctx[idx];
      const auto* t = tuned(P, c.sc, c.dims);
      const int bt = t && t->stream_block ? t->stream_block : P->stream_block;
      int found = -1;
      for (size_t q = 0; q < chain_rep.size() && found < 0; ++q) {
        const ItemCtx& d = ctx[chain_rep[q]];
        const auto* td = tuned(P, d.sc, d.dims);
        const int btd = td && td->stream_block ? td->stream_block : P->stream_block;
        bool eq = c.sc.rks == d.sc.rks && c.sc.rkr == d.sc.rkr && bt == btd &&
                  std::memcmp(c.sc.ss, d.sc.ss, sizeof c.sc.ss) == 0;
        for (int a = 0; a < 3 && eq; ++a) eq = same_taps(c.sc.ts[a], d.sc.ts[a]) && same_taps(c.sc.tr[a], d.sc.tr[a]);
        if (eq) found = (int)q;
      }
      if (found < 0) {
        found = (int)chain_rep.size();
        chain_rep.push_back(idx);
      }
      chain_of.push_back(found);
    }
    size_t off = 0;  // arena offset of the next item's scratch
    int item_no = 0;
    for (int idx : wv) {
      const int chain = chain_of[item_no++];
      const ItemCtx& c = ctx[idx];
      const ct_item& it = items[idx];
      const Box ob = c.whole;
      const Box G = grow_clip3(ob, c.sc.rr, c.dims);
      const Box Ab = grad_partial_box(G, ob, c.sc.rks, c.dims[2]);
      Box Bxy = G;
      Bxy.lo[0] = ob.lo[0];
      Bxy.n[0] = ob.n[0];
      Bxy.lo[1] = ob.lo[1];
      Bxy.n[1] = ob.n[1];
      const int64_t need = std::max<int64_t>(box_vox(G), (box_vox(Ab) + 1) / 2);
      // arena pointers are offsets until the arena exists: stored relative, fixed up below
      const size_t a_off = off, b_off = a_off + sizeof(float) * 6 * need, l_off = b_off + sizeof(float) * 6 * need;
      off = (l_off + sizeof(int64_t) * box_vox(ob) + 255) / 256 * 256;
      float* A = reinterpret_cast<float*>(a_off);
      float* B = reinterpret_cast<float*>(b_off);
      MultiRec base;
      std::memset(&base, 0, sizeof base);
      base.block = dim3(1, 1, 1);
      base.chain = chain;
      {
        GxyItem x{it.vol, ob, c.dims[0], c.dims[1], B, Ab, 0};
        g_gxy.push_back(grad_xy_item(c.sc.rks, x));
        gxy.push_back(x);
        MultiRec r = base;
        r.kind = 0;
        r.rk = c.sc.rks;
        r.t0 = c.sc.ts[0];
        r.t1 = c.sc.ts[1];
        p_gxy.push_back(r);
      }
      {
        GzItem x{B, Ab, A, G, 0};
        g_gz.push_back(grad_z_item(c.sc.rks, x));
        gz.push_back(x);
        MultiRec r = base;
        r.kind = 1;
        r.rk = c.sc.rks;
        r.t0 = c.sc.ts[2];
        std::memcpy(r.ss, c.sc.ss, sizeof r.ss);
        p_gz.push_back(r);
      }
      {
        RxyItem x{A, G, c.dims[0], c.dims[1], B, Bxy, 0};
        const int xt = rho_xy_width(Bxy.n[0]);  // the single launch's CTA width (items of each width in one launch)
        g_rxy.push_back(rho_xy_item(c.sc.rkr, xt, x));
        rxy.push_back(x);
        MultiRec r = base;
        r.kind = 2;
        r.rk = c.sc.rkr;
        r.xt = xt;
        r.t0 = c.sc.tr[0];
        r.t1 = c.sc.tr[1];
        p_rxy.push_back(r);
      }
      const auto* t = tuned(P, c.sc, c.dims);
      {
        RzItem x{B, Bxy, c.dims[2], A, ob, 0};
        MultiRec r = base;
        r.kind = 3;
        r.rk = c.sc.rkr;
        r.block_t = t && t->stream_block ? t->stream_block : P->stream_block;
        r.block = rho_stream_block(ob, 2);  // the single launch's CTA shape (items of each shape in one launch)
        r.t0 = c.sc.tr[2];
        g_rz.push_back(rho_z_item(c.sc.rkr, r.block_t, r.block, x));
        rz.push_back(x);
        p_rz.push_back(r);
      }
      {
        Fallback fb;
        fb.count = nullptr;  // set below to the wave's counter slot
        fb.total = P->fb_total;
        fb.list = reinterpret_cast<int64_t*>(l_off);
        fb.cap = box_vox(ob);
        fb.gap = degenerate_gap(P->p.precision == CT_PREC_MIXED);
        EigOut o{it.vec, it.ha, it.ia, it.fa, P->p.vec_type, P->p.angle_type, P->p.fa_type, ob};
        EigItem x{A, ob, ob, it.mask, ob, c.F, o, fb};
        const bool compact = it.mask && (t && t->eig_compact >= 0 ? t->eig_compact != 0 : P->eig_compact);
        MultiRec r = base;
        r.kind = compact ? 4 : 5;
        r.plain = c.F.sp[0] == 1.f && c.F.sp[1] == 1.f && c.F.sp[2] == 1.f && c.F.centres == nullptr;
        g_eig.push_back(eig_item_grid(compact, x));
        eig.push_back(x);
        p_eig.push_back(r);
      }
      W.max_vox = std::max(W.max_vox, box_vox(ob));
    }
    // re-solve counters: one int per eigen item, in the table (zeroed per wave)
    W.n_fbc = eig.size();
    W.fbc_off = H->zeros(sizeof(int) * W.n_fbc);
    for (size_t i = 0; i < eig.size(); ++i)
      eig[i].fb.count = reinterpret_cast<int*>(W.fbc_off + sizeof(int) * i);  // table offset, fixed up below
    // order the eigen items by kernel form so that the re-solve can take them all contiguously
    std::vector<size_t> order(eig.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](size_t a, size_t b) { return p_eig[a].kind < p_eig[b].kind || (p_eig[a].kind == p_eig[b].kind && p_eig[a].plain > p_eig[b].plain); });
    {
      std::vector<EigItem> e2;
      std::vector<uint3> g2;
      std::vector<MultiRec> p2;
      for (size_t i : order) {
        e2.push_back(eig[i]);
        g2.push_back(g_eig[i]);
        p2.push_back(p_eig[i]);
      }
      eig.swap(e2);
      g_eig.swap(g2);
      p_eig.swap(p2);
    }
    // the four stages' launches of each chain, in stage order
    const auto same_chain = [](const MultiRec& a, const MultiRec& b) { return a.chain == b.chain; };
    add_groups(*H, W, gxy, g_gxy, p_gxy, same_chain, [](MultiRec&) {});
    add_groups(*H, W, gz, g_gz, p_gz, same_chain, [](MultiRec&) {});
    add_groups(*H, W, rxy, g_rxy, p_rxy, [](const MultiRec& a, const MultiRec& b) { return a.chain == b.chain && a.xt == b.xt; },
               [](MultiRec&) {});
    add_groups(*H, W, rz, g_rz, p_rz,
               [](const MultiRec& a, const MultiRec& b) {
                 return a.chain == b.chain && a.block.x == b.block.x && a.block.y == b.block.y &&
                        a.block_t == b.block_t;
               },
               [](MultiRec&) {});
    W.n_chains = (int)chain_rep.size();
    // the eigen items in groups of equal kernel form, and all of them once more,
    // contiguous, for the wave's re-solve
    W.n_eig = (int)eig.size();
    W.eig_items_off = H->put(eig.data(), eig.size());
    add_groups(*H, W, eig, g_eig, p_eig,
               [](const MultiRec& a, const MultiRec& b) { return a.kind == b.kind && a.plain == b.plain; },
               [](MultiRec& r) { r.chain = -1; });
    W.n_counters = W.launches.size();
    W.counters_off = H->zeros(sizeof(unsigned long long) * W.n_counters);
    for (size_t g = 0; g < W.launches.size(); ++g)
      W.launches[g].counter_off = W.counters_off + sizeof(unsigned long long) * g;
    waves->push_back(W);
  }
  (void)mixed;
  return CT_OK;
}

// Replace the arena and table offsets stored in the table's item records by
// device addresses (the records hold offsets until the buffers exist).
void fix_up_eig(EigItem* x, uintptr_t arena, uintptr_t tables) {
  x->S = reinterpret_cast<const float*>(arena + reinterpret_cast<uintptr_t>(x->S));
  x->fb.list = reinterpret_cast<int64_t*>(arena + reinterpret_cast<uintptr_t>(x->fb.list));
  x->fb.count = reinterpret_cast<int*>(tables + reinterpret_cast<uintptr_t>(x->fb.count));
}

void fix_up_tables(HostTable& H, const std::vector<WaveRec>& waves, uintptr_t arena, uintptr_t tables) {
  for (const WaveRec& W : waves) {
    for (int i = 0; i < W.n_eig; ++i)
      fix_up_eig(reinterpret_cast<EigItem*>(H.bytes.data() + W.eig_items_off) + i, arena, tables);
    for (const MultiRec& r : W.launches) {
      unsigned char* p = H.bytes.data() + r.items_off;
      for (int i = 0; i < r.n; ++i) {
        switch (r.kind) {
          case 0: {
            GxyItem* x = reinterpret_cast<GxyItem*>(p) + i;
            x->F = reinterpret_cast<float*>(arena + reinterpret_cast<uintptr_t>(x->F));
            break;
          }
          case 1: {
            GzItem* x = reinterpret_cast<GzItem*>(p) + i;
            x->F = reinterpret_cast<const float*>(arena + reinterpret_cast<uintptr_t>(x->F));
            x->J = reinterpret_cast<float*>(arena + reinterpret_cast<uintptr_t>(x->J));
            break;
          }
          case 2: {
            RxyItem* x = reinterpret_cast<RxyItem*>(p) + i;
            x->in = reinterpret_cast<const float*>(arena + reinterpret_cast<uintptr_t>(x->in));
            x->out = reinterpret_cast<float*>(arena + reinterpret_cast<uintptr_t>(x->out));
            break;
          }
          case 3: {
            RzItem* x = reinterpret_cast<RzItem*>(p) + i;
            x->in = reinterpret_cast<const float*>(arena + reinterpret_cast<uintptr_t>(x->in));
            x->out = reinterpret_cast<float*>(arena + reinterpret_cast<uintptr_t>(x->out));
            break;
          }
          default:
            fix_up_eig(reinterpret_cast<EigItem*>(p) + i, arena, tables);
            break;
        }
      }
    }
  }
}

// Enqueue the waves: the chains of a wave spread over the plan's first K
// streams (forked from and joined back into stream 0), then the wave's eigen
// stage and re-solve on stream 0 (the tables and arena are in place).
ct_status run_persistent_waves(ct_plan P, const std::vector<WaveRec>& waves, int K) {
  const bool mixed = P->p.precision == CT_PREC_MIXED;
  const uintptr_t tb = reinterpret_cast<uintptr_t>(P->tables);
  cudaStream_t st0 = P->st[0];
  for (const WaveRec& W : waves) {
    CT_CUDA(cudaMemsetAsync(reinterpret_cast<void*>(tb + W.counters_off), 0, sizeof(unsigned long long) * W.n_counters,
                            st0),
            "counter reset");
    CT_CUDA(cudaMemsetAsync(reinterpret_cast<void*>(tb + W.fbc_off), 0, sizeof(int) * W.n_fbc, st0), "counter reset");
    const int ks = std::max(1, std::min(K, W.n_chains));
    CT_CUDA(cudaEventRecord(P->wev[0], st0), "event record");
    for (int k = 1; k < ks; ++k) CT_CUDA(cudaStreamWaitEvent(P->st[k], P->wev[0], 0), "stream wait");
    bool joined = false;
    for (const MultiRec& r : W.launches) {
      if (r.chain < 0 && !joined) {  // the eigen stage: every chain has finished
        for (int k = 1; k < ks; ++k) {
          CT_CUDA(cudaEventRecord(P->wev[k], P->st[k]), "event record");
          CT_CUDA(cudaStreamWaitEvent(st0, P->wev[k], 0), "stream wait");
        }
        joined = true;
      }
      cudaStream_t st = r.chain >= 0 ? P->st[r.chain % ks] : st0;
      MultiTable T;
      T.first = reinterpret_cast<const int64_t*>(tb + r.first_off);
      T.grids = reinterpret_cast<const uint3*>(tb + r.grids_off);
      T.n = r.n;
      T.counter = reinterpret_cast<unsigned long long*>(tb + r.counter_off);
      const void* items = reinterpret_cast<const void*>(tb + r.items_off);
      switch (r.kind) {
        case 0:
          CT_LAUNCH(P, st, "grad_xy_batch",
                    launch_grad_xy_multi(static_cast<const GxyItem*>(items), T, r.blocks, r.t0, r.t1, r.rk, st),
                    "batched gradient x/y launch");
          break;
        case 1:
          CT_LAUNCH(P, st, "grad_z_batch",
                    launch_grad_z_multi(static_cast<const GzItem*>(items), T, r.blocks, r.t0, r.ss, r.rk, mixed, st),
                    "batched gradient z launch");
          break;
        case 2:
          CT_LAUNCH(P, st, "rho_xy_batch",
                    launch_rho_xy_multi(static_cast<const RxyItem*>(items), T, r.blocks, r.t0, r.t1, r.rk, r.xt, st),
                    "batched rho xy launch");
          break;
        case 3:
          CT_LAUNCH(P, st, "rho_z_batch",
                    launch_rho_z_multi(static_cast<const RzItem*>(items), T, r.blocks, r.block, r.t0, r.rk, r.block_t,
                                       st),
                    "batched rho z launch");
          break;
        default:
          CT_LAUNCH(P, st, "eig_batch",
                    launch_eig_multi(static_cast<const EigItem*>(items), T, r.blocks, r.kind == 4, P->p.vec_type,
                                     P->p.angle_type, P->p.fa_type, r.plain, P->p.fill_value, st),
                    "batched eigen launch");
          break;
      }
    }
    CT_LAUNCH(P, st0, "eig_resolve_batch",
              launch_eig_fallback_multi(reinterpret_cast<const EigItem*>(tb + W.eig_items_off), W.n_eig, W.max_vox,
                                        P->p.fill_value, mixed, st0),
              "batched re-solve launch");
  }
  return CT_OK;
}

// A batch of device-resident volumes (uneven sizes, per-item scales and
// frames): items go round-robin onto up to kSlots streams, each with its own
// scratch slot, so that small volumes run side by side.  The whole
// multi-stream launch sequence is captured once into a CUDA graph (cached
// under a hash of the item list and the plan's settings) and replayed with a
// single graph launch; with graphs off, every item is launched in turn on the
// caller's stream.
ct_status run_device_batch(ct_plan P, const ct_item* items, int n, cudaStream_t user) {
  bool mixed = P->p.precision == CT_PREC_MIXED;
  std::vector<ItemCtx> ctx(n);
  ct_status rc;
  for (int i = 0; i < n; ++i)
    if ((rc = item_ctx(P, items[i], &ctx[i]))) return rc;
  if (!P->batch_graph && !P->batch_persistent) {
    for (int i = 0; i < n; ++i) {
      const ItemCtx& c = ctx[i];
      EigOut o{items[i].vec, items[i].ha, items[i].ia, items[i].fa, P->p.vec_type, P->p.angle_type, P->p.fa_type,
               c.whole};
      if ((rc = fused_stages(P, c.sc, c.dims, items[i].vol, c.whole, c.whole, items[i].mask, c.whole, c.F, o, 0,
                             mixed, user)))
        return rc;
      P->stats.voxels += box_vox(c.whole);
    }
    return CT_OK;
  }
  const int K = std::max(1, std::min(std::min(P->batch_streams, ct_plan_s::kSlots), n));
  // persistent batches: the items on the stencil chain (the tensor-core chain
  // keeps its own per-item launches) go through run_persistent_waves on
  // stream 0; the others round-robin over the remaining streams
  std::vector<int> pers, rest;
  for (int i = 0; i < n; ++i) {
    const ItemCtx& c = ctx[i];
    bool ok = P->batch_persistent && !use_tc(P, c.sc, c.dims, 0) && !use_tc(P, c.sc, c.dims, 1) &&
              !use_tc(P, c.sc, c.dims, 2);
    if (ok) {
      EigOut o{items[i].vec, items[i].ha, items[i].ia, items[i].fa, P->p.vec_type, P->p.angle_type, P->p.fa_type,
               c.whole};
      EigItem e{nullptr, c.whole, c.whole, items[i].mask, c.whole, c.F, o, Fallback{}};
      const Box G = grow_clip3(c.whole, c.sc.rr, c.dims);
      ok = eig_item_ok(e) && box_vox(grad_partial_box(G, c.whole, c.sc.rks, c.dims[2])) < (int64_t(1) << 31) &&
           6 * box_vox(G) < (int64_t(1) << 31) && c.whole.n[2] <= 65535 && 6 * c.whole.n[2] <= 65535;
    }
    (ok ? pers : rest).push_back(i);
  }
  const int k0 = pers.empty() || K == 1 ? 0 : 1;  // first stream of the per-item launches
  const int kn = std::max(1, K - k0);
  // scratch of every slot sized for its largest item, before any capture
  std::vector<int64_t> gmax(K, 0);
  int64_t total = 0;
  for (int i = 0; i < n; ++i) total += box_vox(ctx[i].whole);
  for (size_t r = 0; r < rest.size(); ++r) {
    const int i = rest[r], k = k0 + (int)(r % kn);
    gmax[k] = std::max(gmax[k], box_vox(grow_clip3(ctx[i].whole, ctx[i].sc.rr, ctx[i].dims)));
  }
  for (int k = 0; k < K; ++k) {
    if ((rc = ensure_stream(P, k))) return rc;
    if (gmax[k] > 0 && (rc = ensure_scratch(P, k, gmax[k]))) return rc;
  }
  for (int k = 0; k < K && !pers.empty(); ++k)
    if (!P->wev[k]) CT_CUDA(cudaEventCreateWithFlags(&P->wev[k], cudaEventDisableTiming), "event creation");
  if (!pers.empty() && !P->fb_total) {
    CT_CUDA(cudaMalloc(&P->fb_total, sizeof(unsigned long long)), "counter allocation");
    CT_CUDA(cudaMemset(P->fb_total, 0, sizeof(unsigned long long)), "counter reset");
  }
  if (!P->gst) {
    CT_CUDA(cudaStreamCreateWithFlags(&P->gst, cudaStreamNonBlocking), "stream creation");
    for (int k = 0; k < 2; ++k) CT_CUDA(cudaEventCreateWithFlags(&P->gev[k], cudaEventDisableTiming), "event creation");
  }
  if (!P->batch_graph) {
    // persistent launches without a graph (their kernels then carry the plan's
    // timing events): tables built and uploaded on every call, the waves and the
    // per-item sequences forked from and joined back into the caller's stream
    std::vector<WaveRec> waves;
    if (!pers.empty()) {
      HostTable H;
      size_t arena_need = 0;
      CT_CUDA(cudaStreamSynchronize(user), "stream sync");  // the arena and tables may be in use
      for (int k = 0; k < K; ++k) CT_CUDA(cudaStreamSynchronize(P->st[k]), "stream sync");
      if ((rc = build_persistent_waves(P, items, ctx, pers, &waves, &H, &arena_need))) return rc;
      if ((rc = ensure_device(&P->arena, &P->arena_cap, arena_need, "batch scratch"))) return rc;
      if ((rc = ensure_device(&P->tables, &P->tables_cap, H.bytes.size(), "batch tables"))) return rc;
      fix_up_tables(H, waves, reinterpret_cast<uintptr_t>(P->arena), reinterpret_cast<uintptr_t>(P->tables));
      CT_CUDA(cudaMemcpy(P->tables, H.bytes.data(), H.bytes.size(), cudaMemcpyHostToDevice), "batch table upload");
    }
    if (!P->gst) {
      CT_CUDA(cudaStreamCreateWithFlags(&P->gst, cudaStreamNonBlocking), "stream creation");
      for (int k = 0; k < 2; ++k)
        CT_CUDA(cudaEventCreateWithFlags(&P->gev[k], cudaEventDisableTiming), "event creation");
    }
    CT_CUDA(cudaEventRecord(P->gev[0], user), "event record");
    for (int k = 0; k < K; ++k) CT_CUDA(cudaStreamWaitEvent(P->st[k], P->gev[0], 0), "stream wait");
    if (!waves.empty() && (rc = run_persistent_waves(P, waves, K))) return rc;
    for (size_t r = 0; r < rest.size(); ++r) {
      const int i = rest[r], k = k0 + (int)(r % kn);
      const ItemCtx& c = ctx[i];
      EigOut o{items[i].vec, items[i].ha, items[i].ia, items[i].fa, P->p.vec_type, P->p.angle_type, P->p.fa_type,
               c.whole};
      if ((rc = fused_stages(P, c.sc, c.dims, items[i].vol, c.whole, c.whole, items[i].mask, c.whole, c.F, o, k, mixed,
                             P->st[k])))
        return rc;
    }
    for (int k = 0; k < K; ++k) {
      CT_CUDA(cudaEventRecord(P->ev[k], P->st[k]), "event record");
      CT_CUDA(cudaStreamWaitEvent(user, P->ev[k], 0), "stream wait");
    }
    P->stats.voxels += total;
    return CT_OK;
  }
  uint64_t key = 1469598103934665603ull;
  key = fnv1a(key, items, sizeof(ct_item) * (size_t)n);
  key = fnv1a(key, &P->p, sizeof(ct_params));
  key = fnv1a(key, &K, sizeof K);
  key = fnv1a(key, &P->batch_persistent, sizeof P->batch_persistent);
  key = fnv1a(key, &P->batch_bytes, sizeof P->batch_bytes);
  if (!P->graph_exec || P->graph_key != key) {
    if (P->graph_exec) cudaGraphExecDestroy(P->graph_exec);
    if (P->graph) cudaGraphDestroy(P->graph);
    P->graph_exec = nullptr;
    P->graph = nullptr;
    // the persistent waves' tables and scratch arena, in place before the capture
    std::vector<WaveRec> waves;
    if (!pers.empty()) {
      HostTable H;
      size_t arena_need = 0;
      if ((rc = build_persistent_waves(P, items, ctx, pers, &waves, &H, &arena_need))) return rc;
      if ((rc = ensure_device(&P->arena, &P->arena_cap, arena_need, "batch scratch"))) return rc;
      if ((rc = ensure_device(&P->tables, &P->tables_cap, H.bytes.size(), "batch tables"))) return rc;
      fix_up_tables(H, waves, reinterpret_cast<uintptr_t>(P->arena), reinterpret_cast<uintptr_t>(P->tables));
      CT_CUDA(cudaMemcpy(P->tables, H.bytes.data(), H.bytes.size(), cudaMemcpyHostToDevice), "batch table upload");
    }
    const int64_t launches0 = P->stats.launches;
    CT_CUDA(cudaStreamBeginCapture(P->gst, cudaStreamCaptureModeRelaxed), "graph capture");
    P->capturing = true;
    cudaError_t e = cudaEventRecord(P->gev[0], P->gst);
    for (int k = 0; k < K && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(P->st[k], P->gev[0], 0);
    rc = CT_OK;
    if (e == cudaSuccess && !waves.empty()) rc = run_persistent_waves(P, waves, K);
    for (size_t r = 0; r < rest.size() && e == cudaSuccess && rc == CT_OK; ++r) {
      const int i = rest[r], k = k0 + (int)(r % kn);
      const ItemCtx& c = ctx[i];
      EigOut o{items[i].vec, items[i].ha, items[i].ia, items[i].fa, P->p.vec_type, P->p.angle_type, P->p.fa_type,
               c.whole};
      rc = fused_stages(P, c.sc, c.dims, items[i].vol, c.whole, c.whole, items[i].mask, c.whole, c.F, o, k, mixed,
                        P->st[k]);
    }
    for (int k = 0; k < K && e == cudaSuccess; ++k) {
      e = cudaEventRecord(P->ev[k], P->st[k]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(P->gst, P->ev[k], 0);
    }
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(P->gst, &g);
    P->capturing = false;
    if (rc) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return cuda_fail(e, "graph capture");
    }
    e = cudaGraphInstantiate(&P->graph_exec, g, 0);
    if (e != cudaSuccess) {
      cudaGraphDestroy(g);
      P->graph_exec = nullptr;
      return cuda_fail(e, "graph instantiation");
    }
    P->graph = g;
    P->graph_key = key;
    P->graph_launches = P->stats.launches - launches0;
    P->stats.launches = launches0;
    P->graph_voxels = total;
  }
  CT_CUDA(cudaEventRecord(P->gev[1], user), "event record");
  CT_CUDA(cudaStreamWaitEvent(P->gst, P->gev[1], 0), "stream wait");
  CT_CUDA(cudaGraphLaunch(P->graph_exec, P->gst), "graph launch");
  CT_CUDA(cudaEventRecord(P->gev[1], P->gst), "event record");
  CT_CUDA(cudaStreamWaitEvent(user, P->gev[1], 0), "stream wait");
  P->stats.launches += P->graph_launches;
  P->stats.voxels += P->graph_voxels;
  return CT_OK;
}

// Host-resident item.  Chunks that share their y / z extents (a run along x)
// share one slab of copies: the slab's haloed input box comes over in one 3D
// copy (rows of the whole run, not of one chunk, and no x halo copied twice),
// each chunk of the run is computed from it into the slab's output planes,
// and those go back in one copy per plane.  Slabs alternate between the plan's
// two streams, so the copies of one overlap the kernels of the other; stream
// order protects each slot's buffers.  Every chunk's arithmetic is that of a
// chunk on its own, so the results equal the whole volume's bit for bit.
ct_status run_host_item(ct_plan P, const ct_item& it) {
  ItemCtx c;
  ct_status rc = item_ctx(P, it, &c);
  if (rc) return rc;
  bool mixed = P->p.precision == CT_PREC_MIXED;
  OutPlanes op = out_planes(P, it);
  size_t out_bytes_per_vox = 0;
  for (int k = 0; k < 4; ++k)
    if (op.ptr[k]) out_bytes_per_vox += op.esz[k] * op.planes[k];
  std::vector<Box> chunks = chunk_grid(c.dims, P->p.chunk);
  // z slabs: a short first slab (a quarter of its z extent, at least 8 planes),
  // so that the first device-to-host copies start early (512^3 in 128-plane
  // slabs: 20.9 -> 19.0 ms; a ramp doubling up to the slab height measured 20.1)
  if (chunks.size() >= 2 && chunks[0].n[2] >= 16 && chunks[0].n[0] == c.dims[0] && chunks[0].n[1] == c.dims[1]) {
    Box head = chunks[0], rest = chunks[0];
    head.n[2] = std::max(8, chunks[0].n[2] / 4);
    rest.lo[2] += head.n[2];
    rest.n[2] -= head.n[2];
    chunks[0] = rest;
    chunks.insert(chunks.begin(), head);
  }
  int64_t nwhole = box_vox(c.whole);
  // device bytes of a slab's buffers (haloed input, mask, outputs), kept under
  // the plan's slab_bytes per slot by ending a run early
  auto slab_bytes = [&](const Box& b) {
    const Box g = grow_clip3(b, c.sc.halo, c.dims);
    return (int64_t)sizeof(uint16_t) * box_vox(g) + (int64_t)(1 + out_bytes_per_vox) * box_vox(b);
  };
  int slab = 0;
  for (size_t g0 = 0; g0 < chunks.size(); ++slab) {
    size_t g1 = g0 + 1;  // the run: consecutive chunks with the same y / z extents, adjacent in x
    while (g1 < chunks.size() && chunks[g1].lo[1] == chunks[g0].lo[1] && chunks[g1].n[1] == chunks[g0].n[1] &&
           chunks[g1].lo[2] == chunks[g0].lo[2] && chunks[g1].n[2] == chunks[g0].n[2] &&
           chunks[g1].lo[0] == chunks[g1 - 1].lo[0] + chunks[g1 - 1].n[0]) {
      Box wider = chunks[g0];
      wider.n[0] = chunks[g1].lo[0] + chunks[g1].n[0] - wider.lo[0];
      if (slab_bytes(wider) > P->slab_bytes) break;
      ++g1;
    }
    const int slot = slab & 1;
    cudaStream_t st = P->st[slot];
    Box ob = chunks[g0];  // the slab's output box
    ob.n[0] = chunks[g1 - 1].lo[0] + chunks[g1 - 1].n[0] - ob.lo[0];
    Box ib = grow_clip3(ob, c.sc.halo, c.dims);
    int64_t niv = box_vox(ib), nov = box_vox(ob);
    size_t in_bytes = (sizeof(uint16_t) * niv + 255) / 256 * 256;
    size_t mask_bytes = it.mask ? (size_t)nov : 0;
    size_t out_bytes = out_bytes_per_vox * nov;
    if ((rc = ensure_device((void**)&P->d_in[slot], &P->in_cap[slot], in_bytes + mask_bytes, "device input")))
      return rc;
    if ((rc = ensure_device(&P->d_out[slot], &P->out_cap[slot], std::max<size_t>(out_bytes, 1), "device output")))
      return rc;
    CT_CUDA(copy_box(it.vol, P->d_in[slot], c.whole, ib, sizeof(uint16_t), true, st), "host to device copy");
    uint8_t* dmask = nullptr;
    if (it.mask) {
      dmask = (uint8_t*)P->d_in[slot] + in_bytes;
      CT_CUDA(copy_box(it.mask, dmask, c.whole, ob, 1, true, st), "host to device copy");
    }
    P->stats.h2d_bytes += (int64_t)(sizeof(uint16_t) * niv + mask_bytes);
    // device outputs: dense planes over the slab, in the order vec(3), ha, ia, fa
    uint8_t* dptr = (uint8_t*)P->d_out[slot];
    void* dout[4] = {nullptr, nullptr, nullptr, nullptr};
    for (int k = 0; k < 4; ++k) {
      if (!op.ptr[k]) continue;
      dout[k] = dptr;
      dptr += nov * op.esz[k] * op.planes[k];
    }
    EigOut o{dout[0], dout[1], dout[2], dout[3], P->p.vec_type, P->p.angle_type, P->p.fa_type, ob};
    for (size_t ci = g0; ci < g1; ++ci)
      if ((rc = fused_stages(P, c.sc, c.dims, P->d_in[slot], ib, chunks[ci], dmask, ob, c.F, o, slot, mixed, st)))
        return rc;
    for (int k = 0; k < 4; ++k) {
      if (!op.ptr[k]) continue;
      for (int pl = 0; pl < op.planes[k]; ++pl) {
        const uint8_t* src = (const uint8_t*)dout[k] + (size_t)pl * nov * op.esz[k];
        uint8_t* dst = (uint8_t*)op.ptr[k] + (size_t)pl * nwhole * op.esz[k];
        CT_CUDA(copy_box(src, dst, c.whole, ob, op.esz[k], false, st), "device to host copy");
      }
    }
    P->stats.d2h_bytes += (int64_t)out_bytes;
    P->stats.voxels += nov;
    g0 = g1;
  }
  for (int s = 0; s < 2; ++s) CT_CUDA(cudaStreamSynchronize(P->st[s]), "chunked run");
  return CT_OK;
}

}  // namespace

extern "C" {

ct_status ct_run_chunks(ct_plan P, const ct_item* items, int32_t n_items, int32_t items_on_host, void* stream) {
  if (!P) return fail(CT_ERR_INVALID, "plan is NULL");
  if (n_items < 0 || (n_items > 0 && !items)) return fail(CT_ERR_INVALID, "bad item list");
  if (items_on_host != 0 && items_on_host != 1) return fail(CT_ERR_INVALID, "items_on_host must be 0 or 1");
  std::lock_guard<std::mutex> lk(P->mu);
  ct_status rc;
  if (!items_on_host && n_items > 1) {
    rc = run_device_batch(P, items, n_items, (cudaStream_t)stream);
    if (rc) return rc;
  } else {
    for (int i = 0; i < n_items; ++i) {
      rc = items_on_host ? run_host_item(P, items[i]) : run_device_item(P, items[i], (cudaStream_t)stream);
      if (rc) return rc;
    }
  }
  if (items_on_host) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "chunked run");
    return sync_plan(P);  // the outputs are in host memory: report a wait that ran out now
  }
  return n_items > 0 ? mark(P, (cudaStream_t)stream) : CT_OK;
}

ct_status ct_run_box(ct_plan P, const uint16_t* d_vol, const int64_t in_lo[3], const int64_t in_n[3],
                     const int64_t out_lo[3], const int64_t out_n[3], const uint8_t* d_mask, void* d_vec, void* d_ha,
                     void* d_ia, void* d_fa, void* stream) {
  if (!P) return fail(CT_ERR_INVALID, "plan is NULL");
  if (!d_vol || !in_lo || !in_n || !out_lo || !out_n) return fail(CT_ERR_INVALID, "NULL argument");
  if (!valid_box(in_lo, in_n, P->dims)) return fail(CT_ERR_INVALID, "input box outside the volume");
  if (!valid_box(out_lo, out_n, P->dims)) return fail(CT_ERR_INVALID, "output box outside the volume");
  std::lock_guard<std::mutex> lk(P->mu);
  Scale sc;
  ct_status rc = make_scale(P->p, P->p.sigma, P->p.rho, &sc);
  if (rc) return rc;
  Box ib = make_box(in_lo, in_n), ob = make_box(out_lo, out_n);
  if (!inside(ib, grow_clip3(ob, sc.halo, P->dims)))
    return fail(CT_ERR_INVALID, "input box must contain the output box grown by R(sigma)+R(rho) = (%d, %d, %d) (clipped)",
                sc.halo[0], sc.halo[1], sc.halo[2]);
  Frame F = make_frame(P->p.lv_center, P->p.lv_axis, P->sp, P->d_centres);
  EigOut o{d_vec, d_ha, d_ia, d_fa, P->p.vec_type, P->p.angle_type, P->p.fa_type, ob};
  rc = fused_stages(P, sc, P->dims, d_vol, ib, ob, d_mask, ob, F, o, 0, P->p.precision == CT_PREC_MIXED,
                    (cudaStream_t)stream);
  if (rc) return rc;
  P->stats.voxels += box_vox(ob);
  return mark(P, (cudaStream_t)stream);
}

ct_status ct_plan_sync(ct_plan P) {
  if (!P) return fail(CT_ERR_INVALID, "plan is NULL");
  std::lock_guard<std::mutex> lk(P->mu);
  return sync_plan(P);
}

ct_status ct_plan_stats(ct_plan P, ct_stats* out, int32_t reset) {
  if (!P || !out) return fail(CT_ERR_INVALID, "NULL argument");
  std::lock_guard<std::mutex> lk(P->mu);
  ct_status rc = sync_plan(P);
  if (rc) return rc;
  *out = P->stats;
  unsigned long long total = 0;
  if (P->fb_total) CT_CUDA(cudaMemcpy(&total, P->fb_total, sizeof total, cudaMemcpyDeviceToHost), "counter read");
  out->fallback_voxels = (int64_t)total;
  if (reset) {
    std::memset(&P->stats, 0, sizeof P->stats);
    if (P->fb_total) CT_CUDA(cudaMemset(P->fb_total, 0, sizeof(unsigned long long)), "counter reset");
  }
  return CT_OK;
}

ct_status ct_plan_profile(ct_plan P, int32_t enable) {
  if (!P) return fail(CT_ERR_INVALID, "plan is NULL");
  std::lock_guard<std::mutex> lk(P->mu);
  P->profile = enable != 0;
  return CT_OK;
}

ct_status ct_plan_kernel_times(ct_plan P, ct_kernel_time* out, int32_t capacity, int32_t* count) {
  if (!P || !count || (capacity > 0 && !out)) return fail(CT_ERR_INVALID, "NULL argument");
  std::lock_guard<std::mutex> lk(P->mu);
  std::vector<ct_kernel_time> acc;
  cudaError_t err = cudaSuccess;
  for (auto& r : P->recs) {
    float ms = 0.f;
    cudaError_t e = cudaEventSynchronize(r.b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.a, r.b);
    if (e != cudaSuccess && err == cudaSuccess) err = e;
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
    size_t k = 0;
    while (k < acc.size() && std::strcmp(acc[k].name, r.name) != 0) ++k;
    if (k == acc.size()) {
      ct_kernel_time t;
      std::memset(&t, 0, sizeof t);
      std::snprintf(t.name, sizeof t.name, "%s", r.name);
      acc.push_back(t);
    }
    acc[k].launches += 1;
    acc[k].total_ms += ms;
  }
  P->recs.clear();
  if (err != cudaSuccess) return cuda_fail(err, "kernel timing");
  int32_t n = 0;
  for (size_t k = 0; k < acc.size() && n < capacity; ++k) out[n++] = acc[k];
  *count = n;
  return CT_OK;
}

namespace {

// Device buffers of one autotuning run, freed on every exit.
struct TuneBuffers {
  void* p[6] = {};
  ~TuneBuffers() {
    for (void* q : p)
      if (q) cudaFree(q);
  }
};

}  // namespace

ct_status ct_autotune(const ct_params* params, const int64_t vol_dims[3], const int64_t chunk[3], int32_t masked,
                      const char* cache_file, ct_tune_result* out) {
  if (!out || !vol_dims) return fail(CT_ERR_INVALID, "NULL argument");
  ct_status rc = check_params(params);
  if (rc) return rc;
  int dims[3];
  for (int k = 0; k < 3; ++k) {
    if (vol_dims[k] < 1 || vol_dims[k] > (1 << 20)) return fail(CT_ERR_INVALID, "vol_dims must be in [1, 2^20]");
    dims[k] = (int)vol_dims[k];
  }
  Scale sc;
  if ((rc = make_scale(*params, params->sigma, params->rho, &sc))) return rc;
  // the timed box: the whole volume, or a chunk of the given size at its centre
  // with its halo (the input box), as ct_run_chunks would process it
  Box ob;
  for (int k = 0; k < 3; ++k) {
    const int c = chunk && chunk[k] > 0 ? (int)std::min<int64_t>(chunk[k], dims[k]) : dims[k];
    ob.lo[k] = (dims[k] - c) / 2;
    ob.n[k] = c;
  }
  const Box ib = grow_clip3(ob, sc.halo, dims);
  const int64_t vox = box_vox(ib);
  if (vox > (int64_t(1) << 30)) return fail(CT_ERR_INVALID, "the timed box and its halo hold at most 2^30 voxels");
  int64_t in_lo[3], in_n[3], out_lo[3], out_n[3];
  for (int k = 0; k < 3; ++k) {
    in_lo[k] = ib.lo[k];
    in_n[k] = ib.n[k];
    out_lo[k] = ob.lo[k];
    out_n[k] = ob.n[k];
  }
  if (!device_present()) return fail(CT_ERR_NO_DEVICE, "no CUDA device is available");
  int dev = 0;
  CT_CUDA(cudaGetDevice(&dev), "device query");
  // a seeded annulus of the volume's size (the benchmark's construction, scaled)
  TuneBuffers buf;
  const size_t esz_v = elem_size(params->vec_type), esz_a = elem_size(params->angle_type),
               esz_f = elem_size(params->fa_type);
  const int64_t ovox = box_vox(ob);
  CT_CUDA(cudaMalloc(&buf.p[0], sizeof(uint16_t) * vox), "volume allocation");
  if (masked) CT_CUDA(cudaMalloc(&buf.p[1], ovox), "mask allocation");
  CT_CUDA(cudaMalloc(&buf.p[2], esz_v * 3 * ovox), "output allocation");
  CT_CUDA(cudaMalloc(&buf.p[3], esz_a * ovox), "output allocation");
  CT_CUDA(cudaMalloc(&buf.p[4], esz_a * ovox), "output allocation");
  CT_CUDA(cudaMalloc(&buf.p[5], esz_f * ovox), "output allocation");
  ct_synth_spec sp;
  std::memset(&sp, 0, sizeof sp);
  const double m = std::min(dims[0], std::min(dims[1], dims[2]));
  for (int k = 0; k < 3; ++k) sp.center[k] = (dims[k] - 1) / 2.0;
  sp.axis[0] = std::sin(10.0 * M_PI / 180.0);
  sp.axis[2] = std::cos(10.0 * M_PI / 180.0);
  sp.r_in = 0.2 * m;
  sp.r_out = 0.42 * m;
  sp.period = 6.0;
  sp.ha_in_deg = 60.0;
  sp.ha_out_deg = -60.0;
  sp.background = 1000.0;
  sp.amplitude = 800.0;
  sp.noise_kind = 0;
  sp.noise_level = 50.0;
  sp.flags = CT_SYNTH_FP32;
  sp.seed = 11;
  cudaStream_t st = nullptr;
  CT_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "stream creation");
  struct StreamGuard {
    cudaStream_t s;
    ~StreamGuard() { cudaStreamDestroy(s); }
  } sg{st};
  if ((rc = ct_synth_annulus(&sp, vol_dims, in_lo, in_n, (uint16_t*)buf.p[0], nullptr, st))) return rc;
  if (masked && (rc = ct_synth_annulus(&sp, vol_dims, out_lo, out_n, nullptr, (uint8_t*)buf.p[1], st))) return rc;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CT_CUDA(cudaEventCreate(&e0), "event creation");
  CT_CUDA(cudaEventCreate(&e1), "event creation");
  struct EventGuard {
    cudaEvent_t a, b;
    ~EventGuard() {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
    }
  } eg{e0, e1};
  // one candidate: the whole volume as one padded box, best of 3 after a warm-up
  auto measure = [&](const ct_plan_s::TuneEntry* cand, double* ms) -> ct_status {
    ct_plan P = nullptr;
    ct_status r = ct_plan_create(params, vol_dims, &P);
    if (r) return r;
    P->tune.clear();
    P->tune_forced = true;
    P->trial = cand;
    double best = 1e30;
    for (int it = 0; it < 4 && r == CT_OK; ++it) {
      cudaEventRecord(e0, st);
      r = ct_run_box(P, (const uint16_t*)buf.p[0], in_lo, in_n, out_lo, out_n, (const uint8_t*)buf.p[1], buf.p[2],
                     buf.p[3], buf.p[4], buf.p[5], st);
      cudaEventRecord(e1, st);
      if (r == CT_OK) r = ct_plan_sync(P);
      float t = 0.f;
      if (r == CT_OK && cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) r = cuda_fail(cudaGetLastError(), "timing");
      if (it > 0) best = std::min(best, (double)t);
    }
    ct_plan_destroy(P);
    *ms = best;
    return r;
  };
  std::memset(out, 0, sizeof *out);
  if ((rc = measure(nullptr, &out->default_ms))) return rc;
  const int xc = x_class(dims[0]), vl = vox_log2(dims);
  std::vector<ct_plan_s::TuneEntry> cands;
  auto entry = [&](int path, int seg, int sb, int ec) {
    return ct_plan_s::TuneEntry{params->precision, sc.rks, sc.rkr, xc, vl, path, seg, sb, ec, 0.0};
  };
  if (xc >= 4)  // the tensor-core passes' 16-byte copies want x extents that are multiples of 4
    for (int path : {2, 1})
      for (int seg : {512, 256, 128}) cands.push_back(entry(path, seg, 0, -1));
  for (int sb : {16, 8}) cands.push_back(entry(0, 0, sb, -1));
  ct_plan_s::TuneEntry best = cands[0];
  best.ms = 1e30;
  for (auto& c : cands) {
    if ((rc = measure(&c, &c.ms))) return rc;
    if (c.ms < best.ms) best = c;
  }
  int n_timed = (int)cands.size() + 1;
  if (masked) {  // the eigen stage's form, on the best path
    ct_plan_s::TuneEntry pick = best;
    pick.ms = 1e30;
    for (int ec : {1, 0}) {
      ct_plan_s::TuneEntry c = best;
      c.eig_compact = ec;
      if ((rc = measure(&c, &c.ms))) return rc;
      ++n_timed;
      if (c.ms < pick.ms) pick = c;
    }
    best = pick;
  }
  out->rho_path = best.rho_path;
  out->seg_cap = best.seg_cap;
  out->stream_block = best.stream_block;
  out->eig_compact = best.eig_compact;
  out->ms = best.ms;
  out->candidates = n_timed;
  if (cache_file && *cache_file) {
    std::vector<CacheLine> lines = read_cache(cache_file);
    const std::string gpu = gpu_name(dev);
    bool replaced = false;
    for (auto& l : lines)
      if (l.gpu == gpu && same_key(l.e, best)) {
        l.e = best;
        replaced = true;
      }
    if (!replaced) lines.push_back(CacheLine{gpu, best});
    if (!write_cache(cache_file, lines)) return fail(CT_ERR_INVALID, "cannot write the tuning cache %s", cache_file);
  }
  return CT_OK;
}

}  // extern "C"

namespace ct {
// Record a message for ct_last_error from another translation unit of the library.
ct_status set_error(ct_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}
}  // namespace ct
