/*
 * ct.h -- C ABI of the GB300 structure-tensor orientation library.
 *
 * The library computes, per voxel of a 3D image volume, the orientation of the
 * local fibre texture and the cardiac descriptors derived from it (Summary;
 * Figure 1; Architecture, "orientation"):
 *   1. the image gradient by Gaussian-derivative filters at noise scale sigma,
 *   2. the structure tensor: the six products g_a g_b smoothed by a Gaussian
 *      at integration scale rho,
 *   3. its eigen-decomposition; the eigenvector of the SMALLEST eigenvalue is
 *      the fibre direction ("third eigenvector", Figure 1b),
 *   4. helical angle (HA), intrusion angle (IA) and fractional anisotropy (FA)
 *      in a cylindrical frame about a given left-ventricle centre and axis
 *      (Figure 1c), under an optional myocardial mask (Figure 1a),
 * over whole volumes or padded chunks of them (Implementation).
 *
 * Definitions (the paper prints no formulas; these are the textbook ones):
 *   taps      R(s) = floor(truncate * s + 0.5); w_k = exp(-k^2/2s^2) / sum_j exp(-j^2/2s^2),
 *             c_k = (k / s^2) w_k, k = -R..R
 *   gradient  g_x(p) = sum_{i,j,k} c_i w_j w_k I(p + (i,j,k)), cyclically for y, z
 *   tensor    S_ab(p) = sum_{i,j,k} w_i w_j w_k g_a g_b (p + (i,j,k))   (rho taps)
 *   edges     a coordinate beyond the GLOBAL volume is clamped to the edge voxel,
 *             both for the image and for the product field
 *   frame     e_z = axis/|axis|, r = (p - c) - ((p - c).e_z) e_z, e_r = r/|r|, e_t = e_z x e_r
 *   angles    v oriented so that v.e_t > 0 (v.e_z >= 0 if v.e_t = 0);
 *             HA = atan2(v.e_z, v.e_t), IA = asin(v.e_r), in degrees
 *   FA        sqrt(1/2) |(l1-l2, l2-l3, l3-l1)| / |(l1, l2, l3)| with l clamped to >= 0;
 *             0 when all eigenvalues are 0
 *
 * Conventions
 *   - Volumes are uint16 [nz][ny][nx], x fastest; masks uint8 0/1 in the same layout.
 *   - Dimensions, positions and boxes are (x, y, z) in voxel units; a box is
 *     (lo[3], n[3]) in GLOBAL voxel indices of the plan's volume.
 *   - Multi-component fields are SoA planes: component k of box voxel i at
 *     plane k * nvox + i (nvox = n[0]*n[1]*n[2], i in x-fastest order).
 *     Tensor planes: (xx, yy, zz, xy, xz, yz).  Vector planes: (x, y, z).
 *   - Every function returns a ct_status; none aborts or throws.  On error,
 *     ct_last_error() gives a message for the calling thread.
 *   - Device pointers must be allocated on the plan's device, aligned to their
 *     element size.  Stream arguments are cudaStream_t passed as void* (NULL =
 *     the legacy default stream); stage calls are asynchronous on that stream.
 *   - The caller owns every input and output buffer; the plan owns its scratch
 *     memory, streams and staging buffers and frees them in ct_plan_destroy.
 *   - Asynchronous device errors surface as CT_ERR_CUDA from the next call
 *     that synchronises (ct_run_chunks with host items, ct_plan_sync,
 *     ct_plan_stats).  Every wait of a kernel on another part of itself is
 *     bounded; a kernel whose wait runs out stops, drains its own copies and
 *     releases what it holds, leaving the context usable, and the next of
 *     those calls returns CT_ERR_TIMEOUT (the outputs of the work since the
 *     previous synchronising call are then invalid).
 *   - There is no CPU fallback: without a usable CUDA device every compute
 *     call returns CT_ERR_NO_DEVICE.
 */
#ifndef CT_H
#define CT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t ct_status;
#define CT_OK 0
#define CT_ERR_INVALID (-1)     /* bad argument: the message names it */
#define CT_ERR_OOM (-2)         /* device or pinned host allocation failed */
#define CT_ERR_CUDA (-3)        /* a CUDA call or kernel failed */
#define CT_ERR_TIMEOUT (-4)     /* a bounded wait ran out */
#define CT_ERR_NO_DEVICE (-5)   /* no usable CUDA device */
#define CT_ERR_UNSUPPORTED (-6) /* valid request outside what the kernels implement */

/* Arithmetic of the path. */
#define CT_PREC_FP32 0  /* FP32 gradient, tensor and eigen-solve (FP32 Jacobi re-solve
                           for near-degenerate voxels: l2 - l1 < 2e-2 (l3 - l1)) */
#define CT_PREC_MIXED 1 /* gradient held in FP16 (scaled by 2^-8), products and sums in
                           FP32, FP32 closed-form eigen-solve with an FP64 re-solve for
                           near-degenerate voxels (l2 - l1 < 1e-2 (l3 - l1): beyond that
                           the FP16-held gradient, not the solver, bounds the direction) */

/* Output encodings. */
#define CT_OUT_F32 0
#define CT_OUT_F16 1
#define CT_OUT_U8Q 2 /* angles only: code = round((deg + 90) * 256 / 180) mod 256,
                        bin 180/256 deg; masked / undefined voxels get code 0 */

typedef struct ct_params {
  double sigma;        /* noise scale of the gradient, > 0 (units of `spacing`) */
  double rho;          /* integration scale of the tensor smoothing, > 0 (units of `spacing`) */
  double truncate;     /* radius factor; 0 selects 4.0 */
  double lv_center[3]; /* left-ventricle centre (x, y, z) in the units of `spacing`, finite */
  double lv_axis[3];   /* left-ventricle axis (x, y, z); need not be unit; not zero */
  int32_t precision;   /* CT_PREC_* */
  int32_t vec_type;    /* CT_OUT_F32 or CT_OUT_F16 */
  int32_t angle_type;  /* CT_OUT_F32, CT_OUT_F16 or CT_OUT_U8Q */
  int32_t fa_type;     /* CT_OUT_F32 or CT_OUT_F16 */
  float fill_value;    /* value written outside the mask (all outputs) and for HA/IA on
                          the axis; NaN is the usual choice */
  int32_t flags;       /* reserved, must be 0 */
  int64_t chunk[3];    /* ct_run_chunks chunk size (x, y, z); 0 = whole extent */
  /*
   * Anisotropic voxels (the paper is silent; the textbook reading): voxel size
   * (x, y, z), each >= 0 and finite, 0 meaning 1 (all zero = voxel units).
   * Scale s along axis a is s / spacing[a] voxels (its own radius), the
   * gradient and so S are in physical units (component a divided by
   * spacing[a]) and positions are (x spacing[0], y spacing[1], z spacing[2]).
   */
  double spacing[3];
  /*
   * Optional LV centreline (NULL = the fixed lv_center): vol_dims[2] pairs
   * (cx, cy), slice z's centre being (cx, cy, z spacing[2]); copied by
   * ct_plan_create.  Frames then vary along the axis.
   */
  const double* lv_centres;
} ct_params;

typedef struct ct_plan_s* ct_plan;

/*
 * Create a plan for volumes of global size vol_dims (x, y, z) on the current
 * CUDA device.  Validates params (CT_ERR_INVALID) and the supported radius
 * range (R(sigma) <= 12, R(rho) <= 36 at truncate 4, else CT_ERR_UNSUPPORTED).
 * Scratch memory is allocated lazily by the first call that needs it.
 */
ct_status ct_plan_create(const ct_params* params, const int64_t vol_dims[3], ct_plan* out);
ct_status ct_plan_destroy(ct_plan plan);

/*
 * Stage: structure tensor (Figure 1b).  d_vol holds the input box (in_lo,
 * in_n) of the plan's volume as a dense uint16 [in_n.z][in_n.y][in_n.x]
 * array.  d_S receives the 6 FP32 tensor planes over the output box (out_lo,
 * out_n).  The output box grown by R(sigma) + R(rho) on every side (per axis
 * with anisotropic voxels: the radii of sigma / spacing[a] and rho /
 * spacing[a]) and then clipped to the volume must lie inside the input box
 * (that is the halo a padded chunk needs); CT_ERR_INVALID otherwise.  S is in
 * the units of the spacing (voxel units by default).
 */
ct_status ct_structure_tensor(ct_plan plan, const uint16_t* d_vol, const int64_t in_lo[3], const int64_t in_n[3],
                              const int64_t out_lo[3], const int64_t out_n[3], float* d_S, void* stream);

/*
 * Stage: eigen-decomposition of n tensors (Figure 1b: the fibre direction is
 * the structure tensor's third eigenvector, the one of the smallest
 * eigenvalue; Implementation: eigen-decomposition of the structure tensor).
 * d_S holds 6 FP32 planes of n tensors; d_evals (nullable) receives the 3
 * eigenvalues ascending; d_evec receives the unit eigenvector of the smallest
 * eigenvalue (3 planes), its sign chosen so that the largest-magnitude
 * component is positive.  Uses the plan's precision.  Plan scratch holds the
 * list of near-degenerate tensors re-solved after the closed form.
 */
ct_status ct_eig_smallest(ct_plan plan, const float* d_S, int64_t n, float* d_evals, float* d_evec, void* stream);

/*
 * Stage: HA, IA, FA (Figure 1c: helix and intrusion angles of the fibre
 * direction in the left ventricle's cylindrical frame, and fractional
 * anisotropy; Summary) over the box (out_lo, out_n) from the smallest
 * eigenvectors and the eigenvalues (3 FP32 planes each, box-shaped), in the
 * plan's frame.  d_mask (nullable) is a box-shaped uint8 array; 0 = outside.
 * Outputs (each nullable) use the plan's encodings: d_vec 3 planes of the
 * oriented fibre vector (v.e_t > 0; largest-magnitude component positive where
 * no frame exists), d_ha, d_ia, d_fa one plane each.
 */
ct_status ct_angles(ct_plan plan, const float* d_evec, const float* d_evals, const int64_t out_lo[3],
                    const int64_t out_n[3], const uint8_t* d_mask, void* d_vec, void* d_ha, void* d_ia, void* d_fa,
                    void* stream);

/* One volume for the fused path. */
typedef struct ct_item {
  const uint16_t* vol;  /* uint16 [dims.z][dims.y][dims.x] */
  const uint8_t* mask;  /* nullable, same layout */
  int64_t dims[3];      /* (x, y, z) */
  double sigma, rho;    /* <= 0: the plan's values */
  double lv_center[3];  /* frame of this item ... */
  double lv_axis[3];    /* ... all-zero axis: the plan's centre and axis */
  void* vec;            /* outputs, nullable, plan encodings, planes over the whole item */
  void* ha;
  void* ia;
  void* fa;
} ct_item;

/*
 * Fused hot path (Implementation: volumes processed chunk by chunk with
 * padding so that chunks match the whole; independent jobs for many volumes;
 * Figure 1b, c for the stages): the whole pipeline for each item.
 * items_on_host = 0: every
 * pointer of the items is a device pointer and the work is enqueued on
 * `stream` (returns without waiting).  items_on_host = 1: pointers are host
 * pointers (pinned or pageable; pinned copies run at the link's rate); the
 * volume is processed in chunks of the plan's chunk size with a halo of
 * R(sigma) + R(rho).  The chunks of one run along x share a slab of copies
 * (its haloed input box in, its output box out, straight between the caller's
 * arrays and the plan's device buffers, up to 4 GiB of them per slab), slabs
 * alternating between two streams; the call returns when every output is in
 * host memory.  Results do not depend on the chunking.
 */
ct_status ct_run_chunks(ct_plan plan, const ct_item* items, int32_t n_items, int32_t items_on_host, void* stream);

/*
 * Fused hot path for one padded chunk of the plan's volume (Implementation:
 * chunks with padding): d_vol holds the input box (in_lo, in_n) as a dense
 * uint16 array; every output is written for the output box (out_lo, out_n)
 * into dense box-shaped arrays (plan encodings; each nullable); d_mask
 * (nullable) is a box-shaped uint8 array over the output box.  The output box
 * grown by R(sigma) + R(rho) and clipped to the volume must lie inside the
 * input box.  Asynchronous on `stream`; results equal those of the
 * whole-volume run.
 */
ct_status ct_run_box(ct_plan plan, const uint16_t* d_vol, const int64_t in_lo[3], const int64_t in_n[3],
                     const int64_t out_lo[3], const int64_t out_n[3], const uint8_t* d_mask, void* d_vec, void* d_ha,
                     void* d_ia, void* d_fa, void* stream);

/*
 * Wait for the plan's work: its own streams and, on each stream a call of the
 * plan enqueued work on, that work (other work on those streams or the
 * device is not waited for).  Reports asynchronous errors (CT_ERR_CUDA) and a
 * kernel of the plan whose bounded wait ran out since the last sync
 * (CT_ERR_TIMEOUT; the wait limit is a plan setting, CT_TUNE_TC_WAIT_LIMIT
 * polls, default 2^20).
 */
ct_status ct_plan_sync(ct_plan plan);

typedef struct ct_stats {
  int64_t voxels;          /* output voxels processed */
  int64_t fallback_voxels; /* voxels re-solved by the near-degenerate path */
  int64_t launches;        /* kernels launched */
  int64_t h2d_bytes;       /* bytes copied host -> device by ct_run_chunks */
  int64_t d2h_bytes;       /* bytes copied device -> host by ct_run_chunks */
} ct_stats;

/* Counters since creation or the last reset (synchronises the plan). */
ct_status ct_plan_stats(ct_plan plan, ct_stats* out, int32_t reset);

/*
 * Eigen stage for callers that cannot allocate device memory: frameworks that
 * own all device memory through their own pools, services that forbid
 * allocation once running (cudaMalloc may synchronise the device), code that
 * must not fail for lack of memory half-way through.  The paper has no
 * counterpart; this is a property of the library, not of the method.
 * Same arguments and results as ct_eig_smallest (bit for bit: the same kernels),
 * without a plan: precision is CT_PREC_FP32 or CT_PREC_MIXED.  The re-solve
 * list lives in a fixed 8 MiB array of the library's device image, so at most
 * 2^20 tensors per call; larger n is CT_ERR_INVALID, checked before any CUDA
 * call.  No call allocates.  The array is part of a module that CUDA loads
 * lazily: the FIRST call on a device loads it (claiming its 8 MiB on that
 * device, where it stays until exit, and possibly synchronising the device)
 * and looks its address up.  Make that first call at start-up, before any
 * stream capture.  The address is kept per device and CUDA context; after a
 * device reset the next call looks it up again (and loads the module again).
 * All calls share the array: each call clears its counters on `stream`, and
 * calls that overlap on the GPU race on it.
 */
ct_status ct_eig_smallest_noalloc(const float* d_S, int64_t n, float* d_evals, float* d_evec, int32_t precision,
                                  void* stream);

/*
 * Seeded synthetic volume on the device (test and benchmark input; not part of
 * the method).  Same definition, voxel for voxel, as the host generator of
 * the Python package: an annulus about `center` / `axis` with rods along the
 * local helix direction (HA linear from ha_in_deg at r_in to ha_out_deg at
 * r_out, stripe period `period`), optional smooth out-of-plane tilt
 * (ia_std_deg, ia_corr), noise (noise_kind 0: Gaussian of std noise_level;
 * 1: std = noise_level * sqrt(background * clean)), SplitMix64 keyed by `seed`
 * and the global voxel index.  Writes the box (lo, n) of a volume of size
 * vol_dims as dense uint16 (and the annulus mask, nullable) on `stream`;
 * with d_vol NULL only the mask is written (it needs no arithmetic beyond the
 * radius).  flags: 0 = FP64 arithmetic (the definition); CT_SYNTH_FP32 = the same
 * construction in FP32 with 24-bit uniforms (about one intensity unit from
 * the FP64 form, far faster on this GPU's FP32 pipes).  Other bits, a zero
 * axis, r_out <= r_in, period <= 0 or ia_corr <= 0 with ia_std_deg > 0 are
 * CT_ERR_INVALID.
 */
#define CT_SYNTH_FP32 1
typedef struct ct_synth_spec {
  double center[3];
  double axis[3];
  double r_in, r_out, period, ha_in_deg, ha_out_deg;
  double background, amplitude;
  int32_t noise_kind;
  int32_t flags;
  double noise_level;
  double ia_std_deg, ia_corr;
  uint64_t seed;
} ct_synth_spec;

ct_status ct_synth_annulus(const ct_synth_spec* spec, const int64_t vol_dims[3], const int64_t lo[3],
                           const int64_t n[3], uint16_t* d_vol, uint8_t* d_mask, void* stream);

/*
 * Per-kernel timing.  While enabled, the plan records a CUDA event pair on the
 * launching stream around every kernel it launches; ct_plan_kernel_times
 * synchronises, adds the elapsed times up per kernel name, returns them
 * (at most `capacity` entries, *count = entries written) and clears them.
 */
typedef struct ct_kernel_time {
  char name[32];
  int64_t launches;
  double total_ms;
} ct_kernel_time;

ct_status ct_plan_profile(ct_plan plan, int32_t enable);
ct_status ct_plan_kernel_times(ct_plan plan, ct_kernel_time* out, int32_t capacity, int32_t* count);

/*
 * Transmural HA profile: the histogram of helical angle against normalised
 * wall depth, the regional statistic the paper's analysis module plots
 * (Architecture: "analysis", transmural profile of Figure 1(c)'s HA map).
 * It reads the HA output of the pipeline, so it runs after ct_run_chunks /
 * ct_angles on the same box; it is a reduction, not part of the per-voxel path.
 *
 * For every voxel of the box (lo, n) of a volume of size vol_dims (x, y, z):
 *   depth d = (r - r_in) / (r_out - r_in), r = distance of the voxel centre
 *   from the axis line through lv_center along lv_axis (voxel units, FP32);
 *   the voxel counts when the mask (nullable, uint8 over the box) is non-zero,
 *   HA is valid (finite; for CT_OUT_U8Q a code other than 0) and 0 <= d < 1;
 *   then d_hist[kd * n_ha + kh] += 1 with kd = floor(d * n_depth) and
 *   kh = floor((HA + 90) * n_ha / 180) clamped to [0, n_ha - 1].
 * d_ha: dense over the box, encoding ha_type (CT_OUT_F32, CT_OUT_F16,
 * CT_OUT_U8Q: code c decodes to c * 180/256 - 90).  d_hist: device
 * uint64 [n_depth][n_ha], accumulated into (the caller zeroes it).
 * n_depth * n_ha must be in [1, 16384]; r_out > r_in; non-zero axis;
 * reserved 0.  Asynchronous on `stream`.
 */
typedef struct ct_profile_spec {
  double lv_center[3];
  double lv_axis[3];
  double r_in, r_out;
  int32_t n_depth, n_ha;
  int32_t ha_type;
  int32_t reserved;
} ct_profile_spec;

ct_status ct_transmural_profile(const ct_profile_spec* spec, const int64_t vol_dims[3], const int64_t lo[3],
                                const int64_t n[3], const void* d_ha, const uint8_t* d_mask, uint64_t* d_hist,
                                void* stream);

/*
 * Streamline tractography through the fibre field (Figure 1(d); Architecture,
 * "tractography").  The paper gives no integration scheme or stopping rule;
 * this is the textbook one:
 *   - direction at a point q: the 8 voxel vectors of q's interpolation cell
 *     (corner i0 = min(floor(q), n - 2) per axis, weights trilinear), each
 *     negated when it points against a reference direction r (the field is an
 *     orientation: +v and -v are the same fibre), summed and normalised;
 *     invalid when q lies outside [0, n-1] on an axis, a corner vector is not
 *     finite, or the sum vanishes;
 *   - one step from p along the current direction d: classical RK4 with
 *     k1 = dir(p; d), k2 = dir(p + h/2 k1; k1), k3 = dir(p + h/2 k2; k2),
 *     k4 = dir(p + h k3; k3), p' = p + h (k1 + 2 k2 + 2 k3 + k4) / 6 and the
 *     new direction d' = normalise(k1 + 2 k2 + 2 k3 + k4);
 *   - the track stops before p' when a direction is invalid, when d' turns
 *     from d by more than max_turn_deg, when p' is outside the volume, when
 *     the mask (nullable) is 0 at p's nearest voxel floor(p' + 1/2), or when
 *     FA (nullable; trilinear, not aligned) at p' is below fa_min;
 *   - from each seed two tracks: the forward one starts along
 *     dir(seed; v at the seed's nearest voxel), the backward one along its
 *     negation (neither starts when that voxel's vector is zero or not
 *     finite, or dir is invalid); max_steps steps at most.
 * d_vec: 3 FP32 planes [z][y][x] over the volume (the pipeline's vector
 * output; NaN fill stops tracks), d_fa: 1 FP32 plane or NULL, d_mask: uint8
 * or NULL, d_seeds: n_seeds x (x, y, z) FP32 voxel coordinates.
 * Outputs: d_points: FP32 [n_seeds][2][max_steps + 1][3] (point 0 is the
 * seed), d_count: int32 [n_seeds][2] points written per track (0 when the
 * seed is outside the volume, 1 when it cannot start).  Every dims >= 2;
 * step > 0; max_steps >= 1; reserved 0.  Asynchronous on `stream`.
 */
typedef struct ct_track_params {
  double step;
  double fa_min;
  double max_turn_deg;
  int32_t max_steps;
  int32_t reserved;
} ct_track_params;

ct_status ct_track(const ct_track_params* params, const int64_t vol_dims[3], const float* d_vec, const float* d_fa,
                   const uint8_t* d_mask, const float* d_seeds, int64_t n_seeds, float* d_points, int32_t* d_count,
                   void* stream);

/*
 * Autotuner of the kernel choices (the paper gives none: the integration-scale
 * smoothing's formulation and schedule are this library's).  For volumes of
 * size vol_dims at the scales and precision of `params`, it times on the
 * current device, on a seeded synthetic annulus of that size (with the
 * annulus mask when `masked`), one padded-box call per candidate over the
 * whole volume, or over a chunk of size `chunk` (nullable; 0 = whole extent)
 * at the volume's centre with its halo, as ct_run_chunks processes chunks: the rho passes as FP32 stencils (8 or 16 outputs per y / z thread
 * block) or on the tensor cores (products formed in the gradient kernel or in
 * the first pass; work units of at most 512, 256 or 128 outputs), then, when
 * masked, the eigen stage over compacted voxels or a thread per voxel.  Best
 * of 3 runs after a warm-up, CUDA events.  *out gets the best choice, its
 * time and that of the built-in choices.  With cache_file (nullable) the
 * choice is stored there under the device's name and the key (precision,
 * instantiated radii R(sigma) and R(rho), x extent class: a multiple of 8, of
 * 4, or neither; floor(log2(voxels))), replacing an entry of the same key.
 * Plans read the cache at creation (CT_TUNE_CACHE names it, "" disables it;
 * default: tuning/tune_cache.json beside the library's package directory)
 * and apply the entry of their precision, radii and x class whose size class
 * is nearest to a volume's, within one either way; the choice is made per
 * volume, so chunks of a volume reproduce it bit for bit.  Any CT_TUNE_*
 * setting of these choices in the environment disables the cache for a plan.
 * Synchronous; allocates its own device buffers (the timed box and its halo:
 * at most 2^30 voxels).
 */
typedef struct ct_tune_result {
  int32_t rho_path;     /* 0 FP32 stencils; 1 tensor cores, products in the gradient kernel;
                           2 tensor cores, products formed in the first pass */
  int32_t seg_cap;      /* tensor-core outputs per work unit at most (0: not tuned) */
  int32_t stream_block; /* stencil outputs per y / z thread block (0: not tuned) */
  int32_t eig_compact;  /* 1 compacted, 0 a thread per voxel, -1 not tuned (unmasked) */
  double ms;            /* best time of one run */
  double default_ms;    /* time with the built-in choices */
  int32_t candidates;   /* configurations timed */
  int32_t reserved;
} ct_tune_result;

ct_status ct_autotune(const ct_params* params, const int64_t vol_dims[3], const int64_t chunk[3], int32_t masked,
                      const char* cache_file, ct_tune_result* out);

/*
 * Measurement support (not part of the method): the device's FP32 FMA rate.
 * A kernel of independent FMA chains fills every SM of the current device
 * (the SM count read from the device) for `iterations` steps of 16 FMAs per
 * thread, timed with CUDA events; *fma_per_s = FMAs / elapsed time, *sm_count
 * (nullable) the device's SM count, *ms (nullable) the elapsed time.  The
 * benchmark states the FP32 roofline against this rate.  Synchronous.
 */
ct_status ct_fp32_fma_rate(int64_t iterations, double* fma_per_s, int32_t* sm_count, double* ms);

/* Message for the calling thread's last non-OK status ("" if none). */
const char* ct_last_error(void);

/* Radius R = floor(truncate * s + 0.5) as the library computes it (-1 if invalid). */
int32_t ct_radius(double s, double truncate);

#ifdef __cplusplus
}
#endif
#endif /* CT_H */
