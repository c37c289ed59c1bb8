/*
 * gftorf.h -- C ABI of the GB300 (sm_103a) raw C-ToF Gaussian splatting path
 * of "Time of the Flight of the Gaussians" (arXiv 2505.05356).
 *
 * The library renders time-varying 3D Gaussians into raw continuous-wave
 * time-of-flight samples (Eq. 4: each Gaussian contributes
 * (s r_k / d_k^2) sin(psi_k + phi_j) o_k G2D_k T_k^2, psi_k = 4 pi d_k f / c,
 * with T_k squared for the round trip, plus q_bg T_N) at every modulation
 * frequency f and phase offset phi_j, plus one ambient channel
 * (sum_k (s r_k / d_k^2) o_k G2D_k T_k^2 + bg T_N), and differentiates it
 * (Eq. S3 opacity recursion with squared transmittance).
 *
 * Pipeline per batch of frames (three calls):
 *   gftorf_preprocess  -- deform each Gaussian to the frame's time
 *                         x(t) = mu + c1 t + c2 t^2 + c3 t^3 (+ delta_b),
 *                         project (EWA, 3DGS convention), depth, tile bounds,
 *                         C-ToF features (Sec. 3, Eq. 3/4 terms).
 *   gftorf_render_fwd  -- depth radix sort, tile-key duplication, stable tile
 *                         sort, per-tile ranges, then front-to-back
 *                         compositing of Eq. 4 per pixel.
 *   gftorf_render_bwd  -- back-to-front re-walk (Eq. S3), 2D gradients with
 *                         warp-reduced atomics, chain rule to the Gaussian
 *                         parameters, summed over frames.
 *
 * Conventions shared by every entry point:
 *   - All array arguments are DEVICE pointers unless stated otherwise, owned
 *     by the caller.  The library never allocates or frees memory; all its
 *     scratch lives in a caller-allocated workspace (see
 *     gftorf_workspace_size).  Nothing synchronises the stream unless stated.
 *   - `stream` is a cudaStream_t passed as void*.  All work is enqueued on it
 *     in order, so the calls can be captured in a CUDA graph.
 *   - Scalar type of all parameter, output and gradient arrays is
 *     dims->dtype: GFTORF_F32 (float) or GFTORF_F64 (double).
 *   - Errors: invalid arguments return immediately with GFTORF_ERR_ARG (no
 *     work enqueued).  Errors found on the device (tile-instance capacity
 *     exceeded) are recorded in a status word inside the workspace; the
 *     affected work is skipped without out-of-bounds access; read the word
 *     with gftorf_read_device_status.  No entry point aborts or traps.
 *   - Pixel (x, y) samples the image plane at (x + 0.5, y + 0.5); a point
 *     p (camera frame) projects to (fx p_x / p_z + cx, fy p_y / p_z + cy).
 *   - Outputs are channel-major: out[frame][channel][y][x]; channels are the
 *     F*P raw samples, frequency-major (f0 phi0, f0 phi1, ..., f1 phi0, ...),
 *     then the ambient channel, then (GFTORF_FLAG_PHASOR) Re, Im of the
 *     phasor of each frequency, then (GFTORF_FLAG_DEPTH) the mean depth;
 *     C = F*P + 1 (+ 2F) (+ 1).
 */
#ifndef GFTORF_H
#define GFTORF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GFTORF_MAX_FREQ 4
#define GFTORF_MAX_OFFSETS 8
#define GFTORF_MAX_FRAMES 64
#define GFTORF_MAX_SH 16

typedef enum {
  GFTORF_OK = 0,
  GFTORF_ERR_ARG = 1,         /* invalid argument (host-side check)          */
  GFTORF_ERR_CAPACITY = 2,    /* more tile instances than dims.max_instances */
  GFTORF_ERR_TIMEOUT = 3,     /* a bounded device wait gave up               */
  GFTORF_ERR_CUDA = 4,        /* a CUDA launch or runtime call failed        */
  GFTORF_ERR_UNSUPPORTED = 5, /* valid but unsupported configuration         */
  GFTORF_ERR_WORKSPACE = 6    /* workspace missing, misaligned or too small  */
} gftorf_status;

typedef enum { GFTORF_F32 = 0, GFTORF_F64 = 1 } gftorf_dtype;

/* gftorf_dims.flags.  By default the pipeline drops (Gaussian, tile) pairs
 * where alpha = o G cannot reach alpha_min at any pixel centre of the tile:
 * preprocess shrinks each tile rectangle to the bounding box of that
 * ellipse, and the compositing kernels skip the remaining non-intersecting
 * records while staging them.  Those pairs are skipped by every pixel anyway,
 * so outputs are the same; this flag turns the culling off (lists then hold
 * every tile of the 3-sigma rectangle, as gftorf_sort_footprints does). */
#define GFTORF_FLAG_NO_TILE_CULL 1
/* gftorf_dims.flags: the forward also counts the (pixel, Gaussian) pairs it
 * evaluates (each pixel: the staged entries up to and including the one that
 * stops it), readable with gftorf_read_counters.  Same outputs; a separate
 * kernel instantiation, for measurement. */
#define GFTORF_FLAG_COUNT_PAIRS 2
/* gftorf_dims.flags: extra output channels after the raw samples and the
 * ambient channel.  PHASOR adds, per frequency, the real and imaginary part
 * of the C-ToF phasor of Eq. 3, p = p_bg T_N + sum 2 A_k exp(i psi_k)
 * alpha_k T_k^2 (two channels, background from bg).  DEPTH adds the mean
 * depth of Eq. 5, sum d_k alpha_k T_k with the ONE-WAY transmittance and no
 * background term (its bg entry is ignored, its dL/dbg is 0). */
#define GFTORF_FLAG_PHASOR 4
#define GFTORF_FLAG_DEPTH 8

/* Static problem shape.  One workspace serves one dims value. */
typedef struct {
  int32_t n_gaussians;   /* N in [0, 2^30)                                  */
  int32_t n_frames;      /* B in [1, GFTORF_MAX_FRAMES]                     */
  int32_t width, height; /* image size in pixels, >= 1                      */
  int32_t tile_w, tile_h;/* one of 8x8, 16x16, 16x32, 32x32, 64x32, 64x64
                            (w x h): the binning tile; a 64x32 or 64x64
                            tile's list is composited by two or four CTAs
                            of 32x32 pixels                               */
  int32_t n_freq;        /* F in [1, GFTORF_MAX_FREQ]                       */
  int32_t n_offsets;     /* P in [1, GFTORF_MAX_OFFSETS]                    */
  int32_t dtype;         /* gftorf_dtype                                    */
  int32_t render_mode;   /* 0: one CTA per (frame, tile);
                            1: persistent CTAs over a (frame, tile) queue   */
  int32_t pixels_per_thread; /* compositing pixels per thread: 1, 2 or 4
                            (0: 2, or 4 for 32- and 64-wide tiles, which
                            take only 4);
                            tile_w * tile_h / it must be >= 32.  Results do
                            not depend on it, nor on the tile shape.        */
  int32_t flags;         /* GFTORF_FLAG_* bits, 0 for the defaults         */
  int32_t n_sh;          /* reflectivity model (Sec. 3): 0 = the scalar
                            gaussians.amplitude; 1, 4, 9 or 16 = real
                            spherical harmonics of degree 0..3 in
                            gaussians.sh (see gftorf_gaussians)             */
  int32_t reserved;      /* must be 0                                       */
  int64_t max_instances; /* capacity of the (Gaussian, tile) instance list,
                            summed over the batch                           */
} gftorf_dims;

/* One frame (host struct): pinhole camera with a rigid world->camera
 * transform [R | t] (R orthonormal, row-major 3x4), near-plane cull distance (> 0)
 * on the view depth, and the frame's time t for the deformation.  Sec. 3:
 * emitter co-located with the camera, so d_k is the distance from the
 * Gaussian centre to the optical centre o = -R^T t.
 *   phase_offset_rad: added to every sensor phase offset in this frame.  An
 *     asynchronously captured raw sequence (Sec. 3: each raw frame at its own
 *     time) is a batch with n_offsets = 1, sensor offset 0 and the frame's
 *     own offset here.  0 for synchronous capture.
 *   interp_t0, interp_t1: Eq. 7 piecewise-linear motion.  With
 *     interp_t0 < interp_t1 the positions at `time` are the linear
 *     interpolation of the deformed positions at the two timesteps,
 *     x = ((t1 - t) x(t0) + (t - t0) x(t1)) / (t1 - t0), plus delta_b;
 *     with interp_t0 == interp_t1 (e.g. both 0) x = x(time) + delta_b.
 *     interp_t0 > interp_t1 is an error. */
typedef struct {
  float fx, fy, cx, cy;
  float world_to_cam[12];
  float near_plane;
  float time;
  float phase_offset_rad;
  float interp_t0, interp_t1;
} gftorf_frame;

/* C-ToF sensor (Sec. 2): modulation frequencies f (Hz), phase offsets phi_j
 * of the reference signal (rad, shared by all frequencies), source
 * intensity s.  Raw sample j of frequency f is A sin(psi_f + phi_j). */
typedef struct {
  float freq_hz[GFTORF_MAX_FREQ];
  float offset_rad[GFTORF_MAX_OFFSETS];
  float source_intensity;
} gftorf_sensor;

/* Screen-space constants of the 3DGS rasterizer the paper builds on
 * (Sec. 4, implementation details).  Defaults: dilation 0.3 (added to the 2D
 * covariance diagonal), alpha_max 0.99 (alpha = min(alpha_max, o G)),
 * alpha_min 1/255 (smaller alphas are skipped), t_min 1e-4 (the walk stops
 * before a Gaussian that would take the one-way T below it), guard 1.3
 * (lateral clamp of the EWA Jacobian, in units of the half field of view),
 * sigma_cut 3 (footprint radius in standard deviations). */
typedef struct {
  float dilation, alpha_max, alpha_min, t_min, guard, sigma_cut;
} gftorf_consts;

/* Gaussian parameters (device pointers, dims.dtype, N rows):
 *   means[N][3]; coeffs[N][3][3] = (c1, c2, c3) each xyz, or NULL (static);
 *   scales[N][3] (linear, > 0); quats[N][4] (w, x, y, z; normalised inside);
 *   opacity[N] in (0, 1]; amplitude[N] = reflectivity r_k (dims.n_sh == 0;
 *   unused, may be NULL, otherwise);
 *   delta[B][N][3] per-frame displacement added to x(t), or NULL;
 *   sh[N][dims.n_sh] (dims.n_sh > 0, else unused): view-dependent
 *   reflectivity r_k = max(0, 0.5 + sum_l sh_l Y_l(w)) (Sec. 3: r_k held
 *   as spherical harmonic coefficients; 0.5 offset and clamp as in the 3DGS
 *   colour model), w the unit vector from the frame's optical centre to
 *   x(t) in world coordinates, Y_l the orthonormal real spherical harmonics
 *   without the Condon-Shortley phase, ordered by degree and, within a
 *   degree, by order m = -l..l (Y_1: y, z, x). */
typedef struct {
  const void *means, *coeffs, *scales, *quats, *opacity, *amplitude, *delta;
  const void* sh;
} gftorf_gaussians;

/* Gradient outputs (device pointers, dims.dtype; each may be NULL to skip),
 * same layouts as the inputs; bg[B][C].  They are OVERWRITTEN, not
 * accumulated.  With dims.n_sh > 0 the amplitude gradient is 0. */
typedef struct {
  void *means, *coeffs, *scales, *quats, *opacity, *amplitude, *delta, *bg;
  void* sh;
} gftorf_gradients;

/* Bytes of workspace needed for `dims` (0 if dims is invalid).  The
 * workspace must be 256-byte aligned device memory owned by the caller; the
 * library keeps everything between gftorf_preprocess and gftorf_render_bwd
 * there (projected records, sort buffers, tile ranges, per-pixel final
 * transmittance and last-contributor index, 2D gradients). */
size_t gftorf_workspace_size(const gftorf_dims* dims);

/* Deformation + projection + C-ToF features for all frames (Sec. 3, Eq. 3/4
 * terms; deformation x(t) = mu + c1 t + c2 t^2 + c3 t^3 + delta_b, or its
 * Eq. 7 interpolation, see gftorf_frame).
 * frames: HOST array of dims->n_frames entries; sensor, consts: HOST.
 * Resets the device status word. */
gftorf_status gftorf_preprocess(const gftorf_dims* dims,
                                const gftorf_gaussians* gaussians,
                                const gftorf_frame* frames,
                                const gftorf_sensor* sensor,
                                const gftorf_consts* consts, void* workspace,
                                size_t workspace_bytes, void* stream);

/* Binning and compositing (Eq. 4).  bg[B][C] device; out[B][C][H][W] device.
 * Needs a preceding gftorf_preprocess on the same workspace. */
gftorf_status gftorf_render_fwd(const gftorf_dims* dims, const void* bg,
                                void* out, void* workspace,
                                size_t workspace_bytes, void* stream);

/* Backward of gftorf_render_fwd (Eq. S3 recursion; chain rule through the
 * projection and deformation, summed over frames in a fixed order).
 * gaussians: the same parameters the batch was preprocessed with (re-read
 * to recompute the projection instead of storing it); dL_dout[B][C][H][W]
 * and bg[B][C] device.  Needs the gftorf_render_fwd of the same batch to be
 * the last render on this workspace. */
gftorf_status gftorf_render_bwd(const gftorf_dims* dims,
                                const gftorf_gaussians* gaussians,
                                const void* bg, const void* dL_dout,
                                const gftorf_gradients* grads, void* workspace,
                                size_t workspace_bytes, void* stream);

/* The stages of gftorf_render_fwd and gftorf_render_bwd, callable one by
 * one (same arguments and requirements as the combined calls):
 *   gftorf_render_fwd = gftorf_bin + gftorf_composite_fwd
 *   gftorf_render_bwd = gftorf_zero_grad_buffers + gftorf_composite_bwd
 *                       + gftorf_preprocess_bwd
 * gftorf_bin: depth radix sort, tile-key duplication, stable tile sort and
 *   per-(frame, tile) ranges of the preprocessed batch.
 * gftorf_composite_fwd: Eq. 4 compositing over the binned lists.
 * gftorf_zero_grad_buffers: clears the workspace's per-(frame, Gaussian) 2D
 *   gradient rows and grads->bg (if non-NULL) before a backward.
 * gftorf_composite_bwd: Eq. S3 re-walk; accumulates 2D gradients in the
 *   workspace and dL/dbg into grads->bg (if non-NULL).
 * gftorf_preprocess_bwd: chain rule from the 2D gradients to the parameter
 *   gradients of `grads` (except bg), overwriting them. */
gftorf_status gftorf_bin(const gftorf_dims* dims, void* workspace,
                         size_t workspace_bytes, void* stream);
gftorf_status gftorf_composite_fwd(const gftorf_dims* dims, const void* bg,
                                   void* out, void* workspace,
                                   size_t workspace_bytes, void* stream);
gftorf_status gftorf_zero_grad_buffers(const gftorf_dims* dims,
                                       const gftorf_gradients* grads,
                                       void* workspace, size_t workspace_bytes,
                                       void* stream);
gftorf_status gftorf_composite_bwd(const gftorf_dims* dims, const void* bg,
                                   const void* dL_dout,
                                   const gftorf_gradients* grads,
                                   void* workspace, size_t workspace_bytes,
                                   void* stream);
gftorf_status gftorf_preprocess_bwd(const gftorf_dims* dims,
                                    const gftorf_gaussians* gaussians,
                                    const gftorf_gradients* grads,
                                    void* workspace, size_t workspace_bytes,
                                    void* stream);

/* Binning alone, from caller-given screen-space footprints (device arrays
 * [B][N]: u, v float32 centre, radius int32 (<= 0: not visible), z float32
 * view depth > 0).  Tile rectangle, in single precision:
 *   [floor((u-r)/tw), floor((u+r)/tw)+1) x [floor((v-r)/th), floor((v+r)/th)+1)
 * clamped to the grid.  Every covered tile emits the 64-bit key
 * ((b*tiles + tile) << 32) | bits(z) with value g; the pairs are sorted by
 * key, equal keys by g.  Writes keys[M], values[M] (device, capacity
 * dims->max_instances), ranges[B*tiles][2] = [start, end) (empty tiles get
 * [k, k), k the count in the tiles before), and *count (device int64).
 * Uses dims->n_gaussians, n_frames, width, height, tile_w, tile_h,
 * max_instances. */
gftorf_status gftorf_sort_footprints(const gftorf_dims* dims, const float* u,
                                     const float* v, const int32_t* radius,
                                     const float* z, uint64_t* keys,
                                     uint32_t* values, uint32_t* ranges,
                                     int64_t* count, void* workspace,
                                     size_t workspace_bytes, void* stream);

/* gftorf_sort_footprints without a workspace argument, for callers that
 * cannot allocate device memory themselves: code running where cudaMalloc is
 * not available or not allowed (inside a region being captured into a CUDA
 * graph, a host callback, a plugin that may only touch buffers it was
 * handed).  The paper has no counterpart; it is a packaging convenience.
 * Same arguments, results and bit-exact ordering as gftorf_sort_footprints.
 * Its scratch is a fixed 32 MiB device array inside the library, so:
 *   - the 32 MiB are reserved on a device at the latest by the first call
 *     made there (with lazy module loading, CUDA creates the array when the
 *     library's device code first loads on that device, so a failure to get
 *     the memory shows up as GFTORF_ERR_CUDA from that call) and stay
 *     reserved until the process exits;
 *   - problems whose binning scratch (about 32 B per (frame, Gaussian) plus
 *     4 B per instance of dims->max_instances plus per-tile counters) does
 *     not fit return GFTORF_ERR_WORKSPACE before any work is enqueued;
 *   - the first call on a device looks up the array's device address (with
 *     that device current); make that first call before any stream capture;
 *   - all calls share the one array: calls whose GPU work overlaps (other
 *     streams, other host threads) race and corrupt each other's results;
 *   - a capacity overflow is seen as *count > dims->max_instances (the lists
 *     are then left empty); the device status word of a workspace is not
 *     involved.
 * It allocates nothing: no cudaMalloc, no cudaFree, no allocating library
 * call. */
gftorf_status gftorf_sort_footprints_noalloc(const gftorf_dims* dims,
                                             const float* u, const float* v,
                                             const int32_t* radius,
                                             const float* z, uint64_t* keys,
                                             uint32_t* values, uint32_t* ranges,
                                             int64_t* count, void* stream);

/* Copy the current batch's sorted tile instances out of the workspace:
 * keys[M] (as in gftorf_sort_footprints), values[M], ranges[B*tiles][2],
 * *count (all device; keys may be NULL).  For inspection and tests. */
gftorf_status gftorf_export_tile_lists(const gftorf_dims* dims, uint64_t* keys,
                                       uint32_t* values, uint32_t* ranges,
                                       int64_t* count, void* workspace,
                                       size_t workspace_bytes, void* stream);

/* Copy per-pixel state of the last forward: t_final[B][H][W] (dims.dtype),
 * n_last[B][H][W] (uint32: index within the tile list of the last composited
 * Gaussian, plus one).  Device pointers; either may be NULL. */
gftorf_status gftorf_export_pixel_state(const gftorf_dims* dims, void* t_final,
                                        uint32_t* n_last, void* workspace,
                                        size_t workspace_bytes, void* stream);

/* Synchronises `stream`, then returns the device status word written since
 * the last gftorf_preprocess (GFTORF_OK or GFTORF_ERR_CAPACITY /
 * GFTORF_ERR_TIMEOUT) and, if count is non-NULL, the batch's instance count
 * (host int64). */
gftorf_status gftorf_read_device_status(const gftorf_dims* dims,
                                        void* workspace, size_t workspace_bytes,
                                        int64_t* count, void* stream);

/* Number of CUDA kernels this library has enqueued so far in this process
 * (host-side counter; a captured graph's replays are not counted again). */
int64_t gftorf_kernel_launches(void);

/* Synchronises `stream`; counters[0] = tile instances of the last binning,
 * counters[1] = (pixel, Gaussian) pairs the last forward evaluated: per
 * pixel, the entries of its tile's list up to and including the one that
 * stops it; counters[2] = the part of counters[1] in records that can reach
 * alpha_min in the rows of the pixel's warp (the compositing kernels skip the
 * others for the whole warp; the results do not depend on it).  Both are 0
 * unless dims->flags has GFTORF_FLAG_COUNT_PAIRS.  counters: HOST int64[3]. */
gftorf_status gftorf_read_counters(const gftorf_dims* dims, void* workspace,
                                   size_t workspace_bytes, int64_t* counters,
                                   void* stream);

/* Throughput probes: the rooflines of the compositing kernels (Eq. 4 forward,
 * Eq. S3 backward) are FP32 issue (each evaluated (pixel, Gaussian) pair is a
 * short chain of FP32 multiply-adds, compares and selects) and, for the one
 * base-2 exponential per pair, the multi-function unit.  This enqueues one
 * launch of 8 CTAs x 256 threads per SM, each thread running 8 independent
 * chains of `iters` operations:
 *   GFTORF_PROBE_FFMA: x <- x a + b (FP32 fused multiply-add);
 *   GFTORF_PROBE_EX2:  x <- 2^-x (ex2.approx.ftz.f32, the instruction the
 *                      compositing kernels use).
 * *lane_ops (HOST int64) receives the lane operations the launch performs;
 * time the launch with events on `stream` to get the rate.  sink: device
 * float[1], never written in practice (it keeps the loops live).  iters must
 * be a positive multiple of 16.  Not part of the method: measurement only. */
#define GFTORF_PROBE_FFMA 0
#define GFTORF_PROBE_EX2 1
gftorf_status gftorf_probe_throughput(int32_t kind, int32_t iters, float* sink,
                                      int64_t* lane_ops, void* stream);

/* ---- Optimisation loop (Sec. 4: raw-quad L2 loss, Adam with betas (0.9,
 * 0.999) and epsilon 1e-15, a fresh random background every iteration) ----
 * Three calls that, with the render calls above, make one fitting iteration
 * that needs no host round trip (so it can be captured in a CUDA graph):
 *   gftorf_train_begin -> gftorf_preprocess -> gftorf_render_fwd ->
 *   gftorf_l2_loss -> gftorf_render_bwd -> gftorf_adam_step.
 * All FP32. */

/* Device-resident loop state: caller-owned device memory, 8-byte aligned,
 * all zero before the first iteration. */
typedef struct {
  int64_t step;        /* iterations begun: Adam's t                         */
  double loss;         /* the current iteration's loss (gftorf_l2_loss adds) */
  int64_t reserved[2];
} gftorf_train_state;

/* Starts an iteration: state->step += 1, state->loss = 0 and, if bg is not
 * NULL, a fresh background bg[n_bg] (device) uniform in [-1, 1): value i of
 * iteration s is 2u - 1, u = (top 24 bits of the k-th output of SplitMix64
 * seeded with `seed`) * 2^-24, k = (s - 1) n_bg + i + 1.  One CTA;
 * n_bg <= 65536. */
gftorf_status gftorf_train_begin(gftorf_train_state* state, float* bg, int64_t n_bg,
                                 uint64_t seed, void* stream);

/* The same for a shard of a batch whose frames are split over processes:
 * bg[n_bg] receives values [bg_offset, bg_offset + n_bg) of the iteration's
 * bg_stride values (k = (s - 1) bg_stride + bg_offset + i + 1), the slice the
 * whole batch's draw would give these frames.  gftorf_train_begin is the
 * case bg_offset = 0, bg_stride = n_bg.  GFTORF_ERR_ARG unless
 * 0 <= bg_offset, bg_offset + n_bg <= bg_stride <= 2^40. */
gftorf_status gftorf_train_begin_shard(gftorf_train_state* state, float* bg, int64_t n_bg,
                                       uint64_t seed, int64_t bg_offset, int64_t bg_stride,
                                       void* stream);

/* Raw-sample L2 loss of a rendered batch (the L_q term of Eq. 9, without
 * SSIM): L = mean over frames, raw channels c < n_freq * n_offsets and
 * pixels of (out - target)^2.  out, target, dL_dout: device [B][C][H][W]
 * (C as for gftorf_render_fwd); dL_dout gets 2 (out - target) / M on the raw
 * channels and 0 on the others (ambient, phasor, depth); L is added to
 * state->loss.  dims->dtype must be GFTORF_F32. */
gftorf_status gftorf_l2_loss(const gftorf_dims* dims, const float* out, const float* target,
                             float* dL_dout, gftorf_train_state* state, void* stream);

/* The same with the mean taken over `count` raw samples instead of this
 * batch's M: for a shard of frames, count = the whole batch's raw samples,
 * so that the shards' losses and gradients add up to the whole batch's.
 * GFTORF_ERR_ARG unless count >= 1 and finite. */
gftorf_status gftorf_l2_loss_scaled(const gftorf_dims* dims, const float* out,
                                    const float* target, float* dL_dout,
                                    gftorf_train_state* state, double count, void* stream);

#define GFTORF_MAX_ADAM_GROUPS 12

/* One parameter group of gftorf_adam_step: n values at param (updated in
 * place), their gradient, Adam's first and second moments m, v (updated in
 * place, zero before the first step), the learning rate, and the box
 * [lo, hi] the updated values are clamped to (use +-INFINITY for none).
 * Device pointers, FP32; grad may alias nothing else in the call. */
typedef struct {
  float* param;
  const float* grad;
  float* m;
  float* v;
  int64_t n;
  float lr, lo, hi;
} gftorf_adam_group;

/* Adam (Kingma and Ba 2015, Algorithm 1) at t = max(1, state->step) over up to
 * GFTORF_MAX_ADAM_GROUPS groups (HOST array) in one launch:
 *   m = b1 m + (1 - b1) g;  v = b2 v + (1 - b2) g^2;
 *   p = clamp(p - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps), lo, hi). */
gftorf_status gftorf_adam_step(const gftorf_adam_group* groups, int n_groups, float beta1,
                               float beta2, float eps, const gftorf_train_state* state,
                               void* stream);

/* ---- Deformation MLP (Sec. 4, "MLP") on the tensor cores ----
 * delta_x[b][g] = MLP(gamma(means[g] * inv_scale), gamma(times[b])): the
 * positions rescaled by inv_scale (the paper uses 1 / d_u, the unambiguous
 * range), positional encoding gamma(p) = (p, sin(2^l pi p), cos(2^l pi p),
 * l = 0..9) laid out as [x_0..2, (sin x_0..2, cos x_0..2) for l = 0..9, t,
 * (sin t, cos t) for l = 0..9] (84 values, zero-padded to
 * GFTORF_MLP_INPUT), GFTORF_MLP_DEPTH hidden layers of GFTORF_MLP_WIDTH
 * units with ReLU, a linear head to the 3 components.  The output feeds
 * gftorf_gaussians.delta; its gradient grads.delta feeds the backward.
 * Parameters: one packed FP32 device vector of gftorf_mlp_param_count()
 * values, [W_0 (256 x 128), b_0, W_1 (256 x 256), b_1, ..., W_7, b_7,
 * W_head (3 x 256), b_head (3)], each W row-major (out, in).  Matrix
 * products run in BF16 on the tensor cores with FP32 accumulation (weights,
 * encoded inputs, hidden activations and back-propagated pre-activation
 * gradients rounded to BF16); biases, the output and the encoding's gradient
 * stay FP32.  The workspace (caller-owned device memory, 256-byte aligned,
 * gftorf_mlp_workspace_size bytes) keeps the activations from the forward
 * for the backward.  n_frames in [1, GFTORF_MAX_FRAMES], n_gaussians x
 * n_frames below 2^27 (GFTORF_ERR_ARG otherwise; workspace size 0); times:
 * HOST array of n_frames values. */
#define GFTORF_MLP_WIDTH 256
#define GFTORF_MLP_DEPTH 8
#define GFTORF_MLP_INPUT 128

size_t gftorf_mlp_param_count(void);
size_t gftorf_mlp_workspace_size(int32_t n_gaussians, int32_t n_frames);

/* delta[B][N][3] (device, FP32) for the packed parameters theta (device)
 * and means[N][3] (device).  GFTORF_ERR_UNSUPPORTED when the driver offers
 * no tensor-map encoder. */
gftorf_status gftorf_mlp_forward(int32_t n_gaussians, int32_t n_frames, const float* theta,
                                 const float* means, const float* times, float inv_scale,
                                 float* delta, void* workspace, size_t workspace_bytes,
                                 void* stream);

/* Backward of the last gftorf_mlp_forward on this workspace (same
 * arguments): d_theta (packed like theta) and d_means[N][3] (the path
 * through the encoding, summed over frames) are OVERWRITTEN from
 * d_delta[B][N][3]. */
gftorf_status gftorf_mlp_backward(int32_t n_gaussians, int32_t n_frames, const float* theta,
                                  const float* means, const float* times, float inv_scale,
                                  const float* d_delta, float* d_theta, float* d_means,
                                  void* workspace, size_t workspace_bytes, void* stream);

/* Inference forward of the same network (rendering a fitted scene): all
 * layers of a 128-row tile in one CTA, the activations kept in shared memory
 * (bit-identical outputs to gftorf_mlp_forward, nothing kept for a
 * backward).  Workspace: gftorf_mlp_infer_workspace_size() bytes (weights
 * only), 256-byte aligned; same other arguments as gftorf_mlp_forward. */
size_t gftorf_mlp_infer_workspace_size(void);
gftorf_status gftorf_mlp_infer(int32_t n_gaussians, int32_t n_frames, const float* theta,
                               const float* means, const float* times, float inv_scale,
                               float* delta, void* workspace, size_t workspace_bytes,
                               void* stream);

/* Copy an intermediate of the last gftorf_mlp_forward / _backward on this
 * workspace into dst (device), rows m = b N + g, for inspection and tests:
 * what = 0: the encoded input (BF16 bits, [B N][GFTORF_MLP_INPUT]);
 * 1: hidden activation H_layer (BF16 bits, [B N][GFTORF_MLP_WIDTH]);
 * 2: back-propagated pre-activation gradient dZ_layer of the last backward
 *    (BF16 bits, [B N][GFTORF_MLP_WIDTH]);
 * 3: gradient of the encoded input (FP32, [B N][GFTORF_MLP_INPUT]).
 * layer in [0, GFTORF_MLP_DEPTH) for what = 1, 2. */
gftorf_status gftorf_mlp_export(int32_t n_gaussians, int32_t n_frames, int32_t what,
                                int32_t layer, void* dst, void* workspace,
                                size_t workspace_bytes, void* stream);

/* Test hooks, process-wide.  Mode 1 (fault injection without a GPU fault):
 * the MLP kernels' load warps issue no copies, so every CTA's bounded waits
 * (50 ms each in this mode, about 2 s otherwise) run out, record
 * GFTORF_ERR_TIMEOUT in the MLP status word and the kernels return with the
 * context usable (outputs undefined); for small problems only.  Mode 2: the
 * training forward and the backward's chain of dZ run one GEMM per layer
 * instead of the fused kernels (activations, masks and dZ bit-identical,
 * bias-gradient sums in another order; for cross-checks).  Mode 0: normal
 * operation. */
void gftorf_mlp_debug_inject(int32_t mode);

/* Synchronises `stream`; GFTORF_OK or GFTORF_ERR_TIMEOUT if a bounded wait
 * of the last MLP call ran out. */
gftorf_status gftorf_mlp_read_status(void* workspace, size_t workspace_bytes, void* stream);

/* Static description of a status code. */
const char* gftorf_status_string(gftorf_status status);

/* ABI version (major * 100 + minor). */
int32_t gftorf_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GFTORF_H */
