/*
 * hhffbp.h -- C ABI of the GB300 HHFFBPA library.
 *
 * Fast factorized backprojection for near-range handheld SAR (HHFFBPA) and the
 * direct backprojection it approximates, from "A Fast and Accurate 3-D
 * Reconstruction Algorithm for Near-Range Microwave Imaging with Handheld
 * Synthetic Aperture Radar".  All compute runs in hand-written CUDA kernels for
 * sm_103a; the host side only validates, plans and launches.
 *
 * Conventions shared by every entry point
 *   - Status: every function returns an int status, HH_OK (0) on success.
 *   - Trajectory: host float64[n_pos][3] (x', y', z') in metres, copied by the call.
 *   - Frequencies: host float64[n_f] in Hz, strictly increasing and equidistant
 *     (relative tolerance 1e-9); k = 2 pi f / c with c = 299 792 458 m/s.
 *   - Echo: complex64[n_pos][n_f] (interleaved re, im; row = position in
 *     trajectory order), the monostatic samples s(p', k) of Sec. II-A, Eq. (1).
 *   - Image: complex64[nz][ny][nx] (x fastest); voxel (a, b, c) is the point
 *     (x0 + a dx, y0 + b dy, z0 + c dz).
 *   - Echo and image pointers may be device pointers (used in place) or host
 *     pointers (copied to/from device inside the call, on the call's stream);
 *     page-locked host memory makes those copies asynchronous.
 *   - cuda_stream: a cudaStream_t (NULL = legacy default stream).  Imaging calls
 *     are asynchronous on that stream and enqueue no host synchronisation.
 *   - The caller owns echo and image buffers; a plan owns its device workspace.
 */
#ifndef HHFFBP_H
#define HHFFBP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define HH_OK 0
#define HH_ERR_ARG 1              /* null pointer, size <= 0, bad grid/config, D not in front of the aperture */
#define HH_ERR_FREQ_NONUNIFORM 2  /* frequencies not equidistant/increasing */
#define HH_ERR_OOM 3              /* device or host allocation failed */
#define HH_ERR_CUDA 4             /* a CUDA call failed; see hh_last_cuda_error() */
#define HH_ERR_PLAN_NONCONVERGED 5 /* reserved: preimage solver failure rate too high */
#define HH_ERR_DEVICE_FLAG 6      /* a kernel raised an error counter (see hhffbp_plan_counters) */
#define HH_ERR_UNIMPLEMENTED 7
#define HH_ERR_HOST_ONLY 8        /* the plan was built with HH_FLAG_HOST_ONLY and holds no device state */
#define HH_ERR_SCRATCH_LIMIT 9    /* the problem needs more than the fixed workspace of bpa_form_image_noalloc */

/* ---- plan flags --------------------------------------------------------- */
#define HH_FLAG_HOST_ONLY 1u      /* build tree and sampling grids on the host only (no CUDA calls) */
#define HH_FLAG_FP32_REFS 2u      /* precision study: take the per-tile reference ranges and phases (direct BPA)
                                     and the tile references of the merges in FP32 instead of FP64 */

/* Output grid D (Sec. V: the final image grid). */
typedef struct {
    double x0, y0, z0;  /* first voxel centre, metres */
    double dx, dy, dz;  /* spacings, metres, > 0 */
    int32_t nx, ny, nz; /* voxel counts, > 0 */
} hh_grid;

/* Algorithm configuration.  The paper leaves the factorisation depth, the
 * interpolation kernel and the range oversampling open (Sec. IV); these fields
 * choose them. */
typedef struct {
    int32_t leaf_size;    /* positions per level-1 subarray: the tree depth is the largest d with
                             2^d * leaf_size <= n_pos (leaves hold leaf_size .. 2*leaf_size-1) */
    int32_t merge_factor; /* 2: pairwise merges as in Sec. III; 4: two binary levels per merge */
    float eta;            /* lattice density per (u, v, n) unit before the per-axis spectral-extent
                             scaling, >= 1 (1 = the unity sampling rate of Sec. III) */
    int32_t taps;         /* interpolation taps per axis: 4 or 6 */
    int32_t range_os;     /* range oversampling: N_fft = next power of two >= range_os * n_f */
    uint32_t flags;       /* HH_FLAG_* */
} hh_config;

/* Plan summary. */
typedef struct {
    int32_t n_levels;          /* materialised levels including the root (1 = no factorisation) */
    int32_t depth_leaves;      /* binary depth of the leaves */
    int64_t n_nodes;           /* materialised nodes including the root */
    int64_t level_nodes[32];   /* nodes per level, leaves first */
    int64_t level_samples[32]; /* lattice samples per level (the root: the grid's voxel count) */
    int64_t workspace_bytes;   /* device bytes owned by the plan */
    int64_t n_fft;             /* range FFT length */
    int64_t gate_start;        /* first stored range bin */
    int64_t gate_bins;         /* stored range bins per position */
    double dR;                 /* range bin spacing pi / (N_fft dk), metres */
    double kc;                 /* centre wavenumber (k_min + k_max) / 2, rad/m */
} hh_plan_info;

typedef struct hh_plan hh_plan;

/* Defaults: leaf_size 32, merge_factor 4, eta 2, taps 6, range_os 16, flags 0. */
int hhffbp_default_config(hh_config* cfg);

/*
 * hhffbp_interp_weights -- the interpolation weights the merge kernels use, evaluated on
 * the host exactly as the kernels do (FP32 polynomials of x = 2 tau - 1, degree 8, fitted
 * to the least-squares fractional-delay weights for lattice density eta; Sec. IV-A leaves
 * the interpolator open).  tau: host float64 [n] in [0, 1); out: host float64 [n][taps],
 * weight q for the sample at offset q - (taps/2 - 1) from floor(index).  taps: 4 or 6.
 * Errors: HH_ERR_ARG.
 */
int hhffbp_interp_weights(int32_t taps, double eta, const double* tau, int64_t n, double* out);

/*
 * hhffbp_plan -- build the subarray tree and the compressed sampling grids
 * (Sec. IV-A: 2^(M-1) level-1 subarrays; uniform grids in (u, v, n) of
 * Eq. eq_uvw_xyz per subarray), allocate the device workspace and upload the
 * descriptors on cuda_stream.  May synchronise the stream.  The plan depends on
 * the trajectory and is rebuilt per scan (Sec. III: no reusable
 * precalculation).  *out receives the plan (NULL on error).
 * Errors: HH_ERR_ARG, HH_ERR_FREQ_NONUNIFORM, HH_ERR_OOM, HH_ERR_CUDA.
 */
int hhffbp_plan(const double* traj_xyz, int64_t n_pos, const double* freqs_hz, int32_t n_f, const hh_grid* grid,
                const hh_config* cfg, void* cuda_stream, hh_plan** out);

/*
 * hhffbp_plan_update_positions -- replace the plan's positions (host float64 [n_pos][3],
 * trajectory order) and keep everything else: tree, subarray rectangles and design planes,
 * sampling grids, range gate.  Later calls image (and differentiate) the moved positions
 * with that plan held fixed, as an autofocus iteration does for small corrections of an
 * uncertain track (the paper builds one plan per scan, Sec. III).  Moves that carry a range
 * outside the stored gate are counted (hhffbp_plan_counters).  Synchronises cuda_stream.
 * Errors: HH_ERR_ARG (null, non-finite), HH_ERR_CUDA.
 */
int hhffbp_plan_update_positions(hh_plan* plan, const double* traj_xyz, void* cuda_stream);

/* Release a plan and its device workspace (NULL is accepted). */
int hhffbp_plan_destroy(hh_plan* plan);

/* Fill *info from the plan. */
int hhffbp_plan_info(const hh_plan* plan, hh_plan_info* info);

/*
 * hhffbp_plan_export -- copy the plan's tree and grid descriptors to host arrays
 * (for comparison with an independent implementation).  Any pointer may be NULL.
 *   perm[n_pos]         position index of each tree slot (members of a node are contiguous)
 *   nodes_i[n_nodes][10] {level, depth, t, begin, end, child0, nchild, N_u, N_v, N_n}
 *   nodes_d[n_nodes][11] {x'min, x'max, y'min, y'max, lo_u, lo_v, lo_n, eta_u, eta_v, eta_n, zbar}
 *   scalars[5]          {zbar (mean height of all positions), k_min, k_max, zh_floor (least
 *                        height of a feasible sampling point above its subarray's plane),
 *                        zh_mid (height of D's centre above zbar: the solver's fallback depth)}
 * Nodes are ordered by level (leaves first, the root last).
 */
int hhffbp_plan_export(const hh_plan* plan, int64_t* perm, int64_t* nodes_i, double* nodes_d, double* scalars);

/*
 * hhffbp_form_image -- HHFFBPA image of one scan (Sec. IV-A, Fig. 4):
 *   range compression (Eq. eq2_rangecompression), level-1 subimages by BPA on
 *   each subarray's grid with spatial downconversion (Eqs. eq_sdc_mul,
 *   eq_sdc_phi), then per level interpolation of the compressed child subimages
 *   onto the parent grid, remodulation and coherent summation, and finally the
 *   same onto the Cartesian voxels of D.  echo: complex64[n_pos][n_f];
 *   image: complex64[nz][ny][nx] written in full.  Asynchronous on cuda_stream;
 *   allocates nothing.
 * Errors: HH_ERR_ARG (null), HH_ERR_HOST_ONLY, HH_ERR_CUDA.
 */
int hhffbp_form_image(const hh_plan* plan, const void* echo_c64, void* image_c64, void* cuda_stream);

/*
 * hhffbp_plan_counters -- synchronise the plan's last stream and read the device
 * counters of the last form_image: out[0] exact-fallback evaluations, out[1]
 * infeasible lattice samples, out[2] preimage solver failures, out[3] range
 * lookups outside the stored gate (must be 0), out[4] other kernel errors (must
 * be 0), out[5] position updates spent in exact fallbacks, out[6] exact fallbacks
 * evaluated after their merge (queued in groups), out[7] groups evaluated in place
 * because the queue was full.  Returns HH_ERR_DEVICE_FLAG when out[3] or out[4] is
 * non-zero.
 */
int hhffbp_plan_counters(const hh_plan* plan, int64_t out[8]);

/*
 * hhffbp_plan_level_counts -- synchronise and return, for the last form_image,
 * the number of lattice samples evaluated at each level (only the samples the
 * image needs are evaluated; the last level is the voxel count), for
 * min(max_levels, n_levels) levels, leaves first.  out[5] of
 * hhffbp_plan_counters holds the member positions summed by exact fallbacks.
 */
int hhffbp_plan_level_counts(const hh_plan* plan, int64_t* evaluated, int32_t max_levels);

/*
 * hhffbp_plan_tile_fill -- diagnostic: synchronise and histogram, for non-root level
 * `level` of the last form_image, the launch tiles (8 x 8 x 4 lattice samples) by the
 * number of their samples the image needed: hist[k] = tiles with k needed samples,
 * k = 0 .. 256 (hist has 257 entries).  Allocates, and synchronises cuda_stream.
 * Errors: HH_ERR_ARG (null, level out of range), HH_ERR_HOST_ONLY, HH_ERR_CUDA.
 */
int hhffbp_plan_tile_fill(const hh_plan* plan, int32_t level, int64_t* hist, void* cuda_stream);

/*
 * hhffbp_plan_profile -- when enable != 0, hhffbp_form_image records a CUDA
 * event on its stream before and after every stage (range compression, demand
 * passes, level-1 subimages, each merge level, the final level, and the host
 * copies), for hhffbp_plan_stage_times.  Costs one event record per stage.
 */
int hhffbp_plan_profile(hh_plan* plan, int enable);

/*
 * hhffbp_plan_stage_times -- synchronise and return the stage durations of the
 * last profiled hhffbp_form_image: ms[i] (milliseconds), kind[i] (HH_STAGE_*)
 * and level[i] (materialised level the stage works on, -1 when none), for
 * i < *n_out <= max_n.  Any output pointer but n_out may be NULL.
 */
#define HH_STAGE_RC 0
#define HH_STAGE_NEED_FINAL 1
#define HH_STAGE_NEED_LEVEL 2
#define HH_STAGE_LEAF 3
#define HH_STAGE_MERGE 4
#define HH_STAGE_FINAL 5
#define HH_STAGE_H2D 6
#define HH_STAGE_D2H 7
int hhffbp_plan_stage_times(const hh_plan* plan, float* ms, int32_t* kind, int32_t* level, int32_t max_n,
                            int32_t* n_out);

/*
 * bpa_form_image -- direct time-domain backprojection on range-compressed data
 * (Eqs. eq2_rangecompression and eq2_bpatimedomain):
 *   f(p) = sum_i exp(+j 2 k_c R_i) [(1 - t) P_i[m0] + t P_i[m0 + 1]],
 *   R_i = ||p - p'_i||, m0 = floor(R_i / dR), t = R_i / dR - m0,
 * with P_i the centred zero-padded IFFT of s(p'_i, k) (N_fft from cfg->range_os).
 * Only cfg->range_os is used.  Workspace (the range profiles) is allocated and
 * freed stream-ordered on cuda_stream.  Asynchronous on cuda_stream.
 * Errors: HH_ERR_ARG, HH_ERR_FREQ_NONUNIFORM, HH_ERR_OOM, HH_ERR_CUDA.
 */
int bpa_form_image(const double* traj_xyz, int64_t n_pos, const double* freqs_hz, int32_t n_f, const hh_grid* grid,
                   const hh_config* cfg, const void* echo_c64, void* image_c64, void* cuda_stream);

/*
 * bpa_traj_gradient -- gradient of a real loss of the direct BPA image with
 * respect to the positions (the paper forms images only; this differentiates
 * the sum of Eq. eq2_bpatimedomain term by term).  With g the image gradient
 * (grad_image_c64, device complex64 [nz][ny][nx], dL = Re sum_p conj(g_p) df_p):
 *   dL/dp'_i = sum_p Re[conj(g_p) exp(+j 2 k_c R_i) (j 2 k_c lerp_i + (P_i[m0+1] - P_i[m0]) / dR)]
 *              (p'_i - p) / R_i,
 * with R_i, m0, lerp_i as in bpa_form_image (the range profiles do not depend on
 * the positions; the lerp is differentiated within its bin).  grad_traj:
 * device float64 [n_pos][3], overwritten.  traj_xyz, freqs_hz: host float64;
 * echo_c64: device or host complex64 [n_pos][n_f].  Only cfg->range_os is used.
 * Workspace is allocated and freed stream-ordered.  Asynchronous on cuda_stream.
 * Errors: HH_ERR_ARG (null pointers, host gradient buffers), HH_ERR_FREQ_NONUNIFORM,
 * HH_ERR_OOM, HH_ERR_CUDA.
 */
int bpa_traj_gradient(const double* traj_xyz, int64_t n_pos, const double* freqs_hz, int32_t n_f,
                      const hh_grid* grid, const hh_config* cfg, const void* echo_c64, const void* grad_image_c64,
                      double* grad_traj, void* cuda_stream);

/*
 * bpa_adjoint -- adjoint of bpa_form_image (reprojection: image -> echoes), the linear
 * map's conjugate transpose:
 *   s_i[n] = sum_m exp(-j theta_n m) sum_p x(p) exp(-j 2 k_c R_i) w_m(R_i / dR),
 * theta_n = 2 pi (n - (N_f - 1)/2) / N_fft, w_m the linear-interpolation weights of bin m
 * (Eqs. eq2_rangecompression, eq2_bpatimedomain transposed; the paper forms images
 * only).  image_c64: device complex64 [nz][ny][nx]; echo_c64: device complex64
 * [n_pos][n_f], overwritten.  traj_xyz, freqs_hz: host float64.  Only cfg->range_os is
 * used.  Workspace is allocated and freed stream-ordered.  Asynchronous on cuda_stream.
 * Errors: HH_ERR_ARG (null or host buffers), HH_ERR_FREQ_NONUNIFORM, HH_ERR_OOM, HH_ERR_CUDA.
 */
int bpa_adjoint(const double* traj_xyz, int64_t n_pos, const double* freqs_hz, int32_t n_f, const hh_grid* grid,
                const hh_config* cfg, const void* image_c64, void* echo_c64, void* cuda_stream);

/*
 * bpa_form_image_noalloc -- bpa_form_image for callers that cannot allocate
 * memory during the call: code that runs under a device-memory budget fixed at
 * start-up, or a caller whose memory pool already owns every free byte of the
 * device.  The paper has no counterpart: it is an interface variant of the same
 * computation (Eqs. eq2_rangecompression and eq2_bpatimedomain), with the same
 * arguments and results as bpa_form_image.
 *
 * Workspace: a fixed device array of HH_NOALLOC_SCRATCH_BYTES per device,
 * reserved when the library's module is loaded; the call makes no device or
 * host allocation.  It holds the counters, the twiddle table (16 n_fft bytes),
 * the trajectory (24 n_pos bytes) and the range profiles (16 n_pos gate_n bytes,
 * gate_n = range bins spanned by all voxel-position distances, <= n_fft), each
 * rounded up to 256 bytes.  Larger problems return HH_ERR_SCRATCH_LIMIT before
 * any device work.  The first call on a device looks the workspace's address up
 * (and may load the module); the cached address does not survive cudaDeviceReset.
 *
 * echo_c64 and image_c64 must be device (or managed) memory of the current
 * device (no host staging, which would need a buffer); traj_xyz and freqs_hz
 * are host arrays, copied to the workspace on cuda_stream.  Asynchronous on
 * cuda_stream.  Calls that overlap in time on the same device (any streams or
 * host threads) share the workspace and race: serialise them.  The device
 * counters are cleared but not read back (no synchronisation): the gate covers
 * every voxel-position distance, so no lookup falls outside it.
 * Errors: HH_ERR_ARG (also for host or foreign-device echo/image),
 * HH_ERR_FREQ_NONUNIFORM, HH_ERR_SCRATCH_LIMIT, HH_ERR_CUDA.
 */
#define HH_NOALLOC_SCRATCH_BYTES (64ull << 20)
int bpa_form_image_noalloc(const double* traj_xyz, int64_t n_pos, const double* freqs_hz, int32_t n_f,
                           const hh_grid* grid, const hh_config* cfg, const void* echo_c64, void* image_c64,
                           void* cuda_stream);

/*
 * hhffbp_plan_preimages -- diagnostic: run the device preimage solver of the
 * sampling grids (the xyz point whose (u, v, n) of Eq. eq_uvw_xyz equals a
 * target; Sec. IV-A converts uniform (u, v, n) grids to xyz grids this way) on
 * n host targets float64[n][3] of non-root node `node` (export order).  out:
 * host float64[n][4] = absolute (x, y, z) and 1.0 when feasible (converged with
 * height above the node's design plane >= the plan's floor), else 0.0.
 * Allocates, and synchronises cuda_stream.
 */
int hhffbp_plan_preimages(const hh_plan* plan, int64_t node, const double* targets, int64_t n, double* out,
                          void* cuda_stream);

/*
 * hhffbp_adjoint -- the adjoint (conjugate transpose) of hhffbp_form_image as a linear map of
 * the echo: reprojection of an image to echoes.  The paper forms images only; this is the
 * recursion of Sec. III / Sec. IV-A (Fig. 4) transposed step by step: the final level's
 * interpolation scattered into the root's children, the merges top down (the phase factors
 * conjugated, the same footprints and the same exact fallbacks as the forward), the leaf
 * backprojections (Eq. eq2_bpatimedomain) transposed into range bins, and the range
 * compression (Eq. eq2_rangecompression) transposed.  The forward's demand passes run again
 * (the plan's workspace is reused); no forward value is needed.
 * image_c64: complex64 [nz][ny][nx]; echo_c64: complex64 [n_pos][n_f], overwritten; either
 * may be device or host memory (host buffers are staged on the stream).  Asynchronous on
 * cuda_stream.  Sums use atomics: results are not bit-reproducible between calls.  Device
 * counters as for hhffbp_form_image (hhffbp_plan_counters).
 * Errors: HH_ERR_ARG, HH_ERR_HOST_ONLY, HH_ERR_CUDA.
 */
int hhffbp_adjoint(const hh_plan* plan, const void* image_c64, void* echo_c64, void* cuda_stream);

/*
 * hhffbp_traj_gradient -- gradient with respect to the positions of a real loss L of the
 * HHFFBPA image, with the plan held fixed (tree, sampling grids, preimages and subarray
 * phases of the plan's trajectory; only the backprojection terms of the leaves and of the
 * exact fallbacks move with the positions -- the paper forms images only, so this
 * differentiates its recursion, Sec. III / Sec. IV-A, term by term).  With g the image
 * gradient (grad_image_c64, device complex64 [nz][ny][nx], dL = Re sum_p conj(g_p) df_p), the
 * adjoint traversal of hhffbp_adjoint carries to every such term, the value y at point p of
 * member i, and member i receives
 *   dL/dp'_i += Re[conj(y) exp(+j 2 k_c R) (j 2 k_c lerp_i + (P_i[m0+1] - P_i[m0]) / dR)] (p'_i - p) / R
 * (as bpa_traj_gradient, with the range profiles of echo_c64).  grad_traj: device float64
 * [n_pos][3] (trajectory order), overwritten.  echo_c64: device or host complex64
 * [n_pos][n_f].  Asynchronous on cuda_stream; sums use atomics (not bit-reproducible).
 * Errors: HH_ERR_ARG (null pointers, host gradient buffers), HH_ERR_HOST_ONLY, HH_ERR_CUDA.
 */
int hhffbp_traj_gradient(const hh_plan* plan, const void* echo_c64, const void* grad_image_c64, double* grad_traj,
                         void* cuda_stream);

/*
 * Batched imaging of many independent scans (uneven lengths and grids; one plan each) by one
 * CUDA graph launch.  The paper images one scan at a time (Sec. IV); this batches its method.
 *   hhffbp_batch_create(plans, n_plans, n_streams, &batch): plans stay owned by the caller and
 *     must outlive the batch; scan i runs on branch i mod n_streams of the graph, so that
 *     independent scans execute concurrently.
 *   hhffbp_batch_form_images(batch, echos, images, stream): echos[i] / images[i] are device
 *     complex64 buffers of scan i (as for hhffbp_form_image).  The first call, and any call
 *     whose buffers differ from the previous call's, records every scan's hhffbp_form_image
 *     into a graph (relaxed stream capture on private streams: make it before the caller
 *     starts a capture of its own); every call then launches the graph once on `stream`.
 *     Device counters per plan as usual (hhffbp_plan_counters synchronises `stream`).
 *   hhffbp_batch_destroy(batch) (NULL accepted).
 * Errors: HH_ERR_ARG (null, host buffers, n <= 0), HH_ERR_HOST_ONLY, HH_ERR_OOM, HH_ERR_CUDA.
 */
typedef struct hh_batch hh_batch;
int hhffbp_batch_create(hh_plan* const* plans, int32_t n_plans, int32_t n_streams, hh_batch** out);
int hhffbp_batch_form_images(hh_batch* batch, const void* const* echos, void* const* images, void* cuda_stream);
int hhffbp_batch_destroy(hh_batch* batch);

/*
 * hh_mip -- maximum-intensity projection of a complex image (the display of the paper's
 * reconstructions, Sec. V): out = max |f| along one axis of image_c64 (device complex64
 * [nz][ny][nx]): axis 0 over z -> out [ny][nx], axis 1 over y -> out [nz][nx], axis 2 over
 * x -> out [nz][ny] (device float32).  Asynchronous on cuda_stream.
 * Errors: HH_ERR_ARG (null or host buffers, sizes <= 0, axis not 0..2), HH_ERR_CUDA.
 */
int hh_mip(const void* image_c64, int32_t nx, int32_t ny, int32_t nz, int32_t axis, float* out, void* cuda_stream);

/*
 * hh_release_cached_memory -- free the device blocks that destroyed plans left
 * in the library's cache (plans reuse them instead of calling cudaMalloc; at
 * most 64 GiB stay cached, and an allocation failure first empties the cache of
 * that device).  Call when no plan is being created or destroyed.
 */
int hh_release_cached_memory(void);

/* Human-readable status text (static string). */
const char* hh_status_string(int status);

/* Last CUDA error code recorded by the library in this thread (0 = none). */
int hh_last_cuda_error(void);

/*
 * hh_mufu_throughput -- measure the special-function unit's rate on the current device
 * for the approximate functions of the backprojection update (Eq. 3: one reciprocal
 * square root for the range, one sine and one cosine for the carrier phase), the bound
 * of every kernel that sums (sample, position) updates.
 *   op        HH_MUFU_RSQRT, HH_MUFU_SIN, HH_MUFU_COS, or HH_MUFU_UPDATE_MIX (one
 *             rsqrt feeding one sine and one cosine, three results per step).
 *   iters     steps per dependency chain (1 .. 2^20); the grid holds 2048 threads per
 *             SM with eight chains each.  iters = 4096 takes about 2 ms.
 *   mufu_ops  out: MUFU results computed by the timed launch.
 *   ms        out: its duration (CUDA events on cuda_stream, after one untimed launch).
 * Synchronises the stream.  Errors: HH_ERR_ARG (null outputs, op or iters out of range),
 * HH_ERR_CUDA.
 */
#define HH_MUFU_RSQRT 0
#define HH_MUFU_SIN 1
#define HH_MUFU_COS 2
#define HH_MUFU_UPDATE_MIX 3
int hh_mufu_throughput(int32_t op, int32_t iters, void* cuda_stream, int64_t* mufu_ops, float* ms);

/* Diagnostic: kernel launches the library has issued in this process so far (all
 * threads, every entry point).  The difference across a region counts the library's own
 * kernels launched there.  No error. */
long long hh_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* HHFFBP_H */
