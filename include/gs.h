/*
 * libgs — C ABI of the joint pose-appearance training step of GloSplat
 * (arXiv 2603.04847): differentiable 3D Gaussian splatting with camera poses
 * as parameters, fused with the explicit feature-track reprojection term.
 *
 * The step (Algorithm 1, one iteration, for a batch of views B):
 *   gs_project        EWA projection + SH colour + tile rectangle per
 *                     (view, Gaussian)                       ("Rasterize")
 *   gs_sort_tiles     scan, per-tile duplication, depth-key radix sort and
 *                     per-tile ranges                        ("Rasterize")
 *   gs_render_fwd     front-to-back alpha compositing        ("Rasterize")
 *   gs_photo_loss     Eq. 5 with its SSIM term: loss and dL/dimage
 *   sfm_ba_assemble   Eq. 4: the normal-equation blocks of one LM iteration
 *   sfm_ba_schur, sfm_ba_solve_cameras, sfm_ba_back_substitute   Eq. 4:
 *                     point elimination, camera solve, back-substitution
 *                     (sfm_ba_pair_lists + sfm_ba_schur_pairs: the
 *                     elimination summed by camera pairs, no atomics)
 *   gs_mcmc_relocate, gs_mcmc_grow, gs_mcmc_noise, gs_mcmc_reset_moments
 *                     the MCMC densification (Sec. 3.3)
 *   gs_render_bwd     L1 gradient of Eq. 5 (fused) + compositing backward
 *                     + projection backward with pose gradient (its halves
 *                     gs_raster_bwd[_zeroed] and gs_project_bwd[_clearing])
 *                     (Algorithm 1 "Backpropagate"; Sec. 3.3: poses are
 *                     optimised by both losses)
 *   track_reproj_fwd_bwd   Eq. 6: Huber reprojection of the separate track
 *                     points, loss and Jacobians w.r.t. points and poses
 *   pose_se3_update   T_i = T_i^(0) (+) dT_i (Algorithm 1) with the SE(3)
 *                     gradient map and the Adam step on the pose deltas
 *   gs_adam_update    Adam on Gaussian / track-point parameter arrays
 *                     (Algorithm 1 "Update Gaussians", "Update track
 *                     points"; Sec. 3.3 learning rates)
 *
 * Conventions shared by every entry point
 *   - All array arguments are DEVICE pointers owned by the caller, unless a
 *     field says "host".  Arrays are dense, row-major, 4-byte floats unless
 *     stated; float arrays read with 16-byte vector loads must be 16-byte
 *     aligned (checked: GS_ERR_ARG).
 *   - No entry point allocates memory.  Scratch comes from a caller buffer
 *     `ws` whose size the matching *_workspace() query returns.
 *   - Every entry point is asynchronous on `stream` (a cudaStream_t; NULL =
 *     the legacy default stream), returns a gs_status and never throws.
 *     On failure gs_last_error() (thread-local) describes the cause.
 *   - Conditions found on the device (instance capacity overflow,
 *     non-finite inputs) are OR-ed into the caller's device word `status`
 *     (GS_FLAG_*), so a captured CUDA graph can be checked after a replay.
 *   - Camera model: world-to-camera x_c = R x + t, pinhole intrinsics
 *     (fx, fy, cx, cy), pi(X) = (fx X/Z + cx, fy Y/Z + cy) (Sec. 3.2, the
 *     projection pi of Eq. 4; Appendix E "Projection function").  Pixel
 *     (u, v) has its centre at (u + 0.5, v + 0.5).
 *   - Pose tangent: g = (dL/d rho, dL/d phi) for T <- Exp((rho, phi)) T at
 *     0 (left perturbation, translation first), accumulated in double.
 */
#ifndef GS_H
#define GS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int gs_status;
enum {
  GS_OK = 0,
  GS_ERR_ARG = 1,         /* invalid argument (null, size, alignment)      */
  GS_ERR_CAPACITY = 2,    /* host-detected capacity problem                */
  GS_ERR_CUDA = 3,        /* a CUDA runtime call or launch failed          */
  GS_ERR_NONFINITE = 4,   /* host-detected non-finite scalar argument      */
  GS_ERR_UNSUPPORTED = 5  /* valid but unsupported configuration           */
};

/* Bits OR-ed into the device status word. */
enum {
  GS_FLAG_CAPACITY = 1,   /* more tile instances than `capacity`: the sort
                             and renders ran on a truncated list; re-run
                             with a larger capacity                      */
  GS_FLAG_NONFINITE = 2,  /* a Gaussian had a non-finite parameter and was
                             treated as invisible                         */
  GS_FLAG_SORT_STALL = 4, /* a sort block gave up waiting (after 2^20
                             polls) for a predecessor block's digit
                             counts: the sort stopped there, every tile
                             list is empty and the renders show only the
                             background                                   */
  GS_FLAG_NOT_SPD = 8     /* a bundle-adjustment camera system had a pivot
                             <= 0: its step was set to zero              */
};

#define GS_ABI_VERSION 5
#define GS_MAX_BATCH 64   /* views per call */
#define GS_MAX_BA_CAMERAS 4096 /* cameras of one sfm_ba_solve_cameras call */

typedef struct CUstream_st* gs_stream; /* = cudaStream_t */

/* Gaussian parameters, raw (pre-activation): scale = exp(log_scale),
 * opacity = sigmoid(opacity_logit), rotation = quat / |quat| with quat =
 * (w, x, y, z).  SH colour of degree sh_degree (<= 3) in the real basis of
 * the original 3DGS renderer, K = (sh_degree + 1)^2 coefficients per colour
 * channel, colour = max(0, 0.5 + sum_k sh[k] Y_k(dir)) with dir from the
 * camera centre to the mean (Sec. 3.3 "Implementation": SH up to degree 3). */
typedef struct gs_gaussians {
  int32_t n;                  /* number of Gaussians N                     */
  int32_t sh_degree;          /* 0..3                                       */
  const float* mean;          /* [N,3]                                      */
  const float* log_scale;     /* [N,3]                                      */
  const float* quat;          /* [N,4]   16-byte aligned                    */
  const float* opacity_logit; /* [N]                                        */
  const float* sh;            /* [N,K,3]                                    */
} gs_gaussians;

/* Gradients w.r.t. the raw parameters, same layouts; ACCUMULATED (+=). */
typedef struct gs_gaussian_grads {
  float* mean;
  float* log_scale;
  float* quat;
  float* opacity_logit;
  float* sh;
} gs_gaussian_grads;

/* All cameras of the scene (Algorithm 1 REQUIRE: intrinsics K_i, poses). */
typedef struct gs_cameras {
  int32_t n_cams;             /* V                                          */
  const int32_t* wh;          /* [V,2] width, height in pixels              */
  const float* K;             /* [V,4] fx, fy, cx, cy                       */
  const float* Rt;            /* [V,12] world-to-camera R (row-major), t    */
  float near_plane;           /* splats/points with z < near are culled     */
  float far_plane;            /* splats with z > far are culled             */
} gs_cameras;

/* A batch of views rendered together (Algorithm 1 "Sample image indices").
 * Slot b renders camera views[b].  Per-slot images are packed one after
 * another: pixel (u, v) of slot b is element px_offset[b] + v * W + u of
 * every per-pixel buffer; its tiles are global tiles tile_offset[b] ..
 * tile_offset[b+1]-1, row-major within the view.
 * n_pixels and n_tiles are host-side sizes of the batch's per-pixel and
 * per-tile buffers: px_offset[B] <= n_pixels and tile_offset[B] <= n_tiles.
 * They are equal for a batch laid out on the host; a batch whose views
 * change on the device between calls (gs_batch_layout) gives its capacity,
 * and the kernels then read the views' own extent from px_offset[B] and
 * tile_offset[B].  A slot with no tiles (tile_offset[b+1] == tile_offset[b])
 * is skipped. */
typedef struct gs_batch {
  int32_t B;                  /* 1..GS_MAX_BATCH                            */
  int32_t tile;               /* tile edge in pixels: 16 or 32              */
  const int32_t* views;       /* [B]   device                               */
  const int64_t* px_offset;   /* [B+1] device                               */
  const int32_t* tile_offset; /* [B+1] device                               */
  int64_t n_pixels;           /* per-pixel buffer size, >= px_offset[B]     */
  int32_t n_tiles;            /* per-tile buffer size, >= tile_offset[B]    */
  int32_t _pad;
} gs_batch;

/* Per-(slot, Gaussian) screen-space records, index r = b * N + j. */
typedef struct gs_projected {
  float* splat;     /* [B*N,12]: mean2d x, y, opacity, depth | conic a, b,
                       c, q_max | colour r, g, b, 0.  16-byte aligned.
                       q = a dx^2 + 2 b dx dy + c dy^2; alpha >= 1/255 iff
                       q <= q_max = 2 ln(255 opacity) (below the clamp)   */
  uint16_t* rect;   /* [B*N,4] tile rectangle x0, y0, x1, y1 (inclusive,
                       tile units, within the view)                      */
  uint32_t* n_tiles;/* [B*N]   tiles touched; 0 = invisible in that view   */
  uint32_t* depth_key; /* [B*N] depth sort key: float bits of the camera
                       depth if visible (positive floats order like their
                       bits), 0xffffffff if not                          */
} gs_projected;

/* Adam hyperparameters.  `step` points to a DEVICE int32 holding the
 * 1-based step number t used for bias correction (advance it with
 * gs_step_advance, so a captured graph stays valid across replays). */
typedef struct gs_adam {
  float lr, beta1, beta2, eps;
  const int32_t* step;
} gs_adam;

/* Launch tuning, process-wide (chosen by an autotuner; results do not
 * depend on it).  render_fwd_batch, render_bwd_batch: splat records staged
 * in shared memory per round by the compositing forward and backward (64,
 * 128 or 256 each); sort_blocks_per_sm: grid of the sort's grid-stride
 * kernels (histogram, zeroing, ranges), in 2048-thread units per SM (1..8).
 * sort_spin_limit: polls of an unpublished predecessor after which a radix
 * block gives up waiting (GS_FLAG_SORT_STALL): 0 = the default 2^20; a
 * negative value -n is a test hook in which no predecessor is ever seen
 * published, so every wait gives up after n polls (n >= 1).
 * Not synchronised: set it while no other thread calls the library. */
typedef struct gs_tuning {
  int32_t render_fwd_batch;
  int32_t render_bwd_batch;
  int32_t sort_blocks_per_sm;
  int32_t sort_spin_limit;
} gs_tuning;

/* One parameter array of gs_adam_update_groups (learning rate per group). */
typedef struct gs_adam_group {
  float* p;
  const float* g;
  float* m;
  float* v;
  int64_t n;
  float lr;
  int32_t _pad;
} gs_adam_group;

/* Double-precision counterparts of gs_gaussians, gs_gaussian_grads,
 * gs_cameras and gs_projected, for the FP64 instantiation of the projection
 * and compositing kernels (the *_f64 entry points): the same fields, the
 * same layouts, with double elements.  quat and splat must be 16-byte
 * aligned. */
typedef struct gs_gaussians_f64 {
  int32_t n;
  int32_t sh_degree;
  const double* mean;
  const double* log_scale;
  const double* quat;
  const double* opacity_logit;
  const double* sh;
} gs_gaussians_f64;

typedef struct gs_gaussian_grads_f64 {
  double* mean;
  double* log_scale;
  double* quat;
  double* opacity_logit;
  double* sh;
} gs_gaussian_grads_f64;

typedef struct gs_cameras_f64 {
  int32_t n_cams;
  const int32_t* wh;
  const double* K;
  const double* Rt;
  double near_plane;
  double far_plane;
} gs_cameras_f64;

typedef struct gs_projected_f64 {
  double* splat;     /* [B*N,12], the layout of gs_projected.splat */
  uint16_t* rect;
  uint32_t* n_tiles;
  uint32_t* depth_key; /* float bits of the camera depth rounded to float */
} gs_projected_f64;

/* ---------------------------------------------------------------------- */

int gs_abi_version(void);
gs_status gs_set_tuning(const gs_tuning* t);
gs_status gs_get_tuning(gs_tuning* t);
const char* gs_last_error(void);
/* sizeof of the ABI structs, for bindings to verify their layout:
 * 0 gs_gaussians, 1 gs_gaussian_grads, 2 gs_cameras, 3 gs_batch,
 * 4 gs_projected, 5 gs_adam, 6 gs_tuning, 7 gs_adam_group,
 * 8 gs_gaussians_f64, 9 gs_gaussian_grads_f64, 10 gs_cameras_f64,
 * 11 gs_projected_f64.  Returns 0 for an unknown id. */
size_t gs_struct_size(int which);
/* Number of streaming multiprocessors of the current device (0 on error). */
int gs_device_sm_count(void);

/*
 * gs_project — EWA splatting of every Gaussian into every view of the batch
 * (the rasterizer of Sec. 3.3, "Implementation"; the mean follows pi of
 * Sec. 3.2).  Per (slot b, Gaussian j): x_c = R mu + t, culled if z is
 * outside [near, far]; 2-D covariance J R Sigma R^T J^T + 0.3 I with the
 * Jacobian J of pi at x_c (x/z, y/z clamped to 1.3 half-fields of view);
 * conic = its inverse; colour from SH; tile rectangle of the pixels whose
 * alpha can reach 1/255 (1/64 px of margin).  Writes out->splat, ->rect
 * and ->n_tiles for all B*N records (n_tiles = 0 when culled).
 * Non-finite parameters set GS_FLAG_NONFINITE and cull the Gaussian.
 */
gs_status gs_project(const gs_gaussians* g, const gs_cameras* cams,
                     const gs_batch* batch, const gs_projected* out,
                     int32_t* status, gs_stream stream);

/*
 * gs_sort_tiles — per-tile duplication and depth ordering.  A stable sort
 * of the B*N records r = b*N + j by camera depth (ties in record order),
 * an exclusive scan of n_tiles in that order, one instance (global tile, r)
 * per covered tile, and a stable sort of the instances by tile id, so that
 * every tile's list is ordered by (depth, j).  Outputs: tiles[i], vals[i] =
 * tile id and record of sorted instance i; ranges[2*t], ranges[2*t+1] =
 * [start, end) of global tile t (0, 0 when empty).  The full instance count
 * (saturated at 2^32 - 1) is written to n_instances (device) and never read
 * back by the library, so the call can be captured in a CUDA graph.  If it
 * exceeds `capacity`, GS_FLAG_CAPACITY is set and only the first `capacity`
 * instances (in depth order) are sorted and rendered; re-run with more.
 * tiles/vals: [capacity] uint32 (tiles 16-byte aligned); ranges:
 * [2 * batch->n_tiles]; ws: see query (256-byte aligned).  Reads the
 * depth_key and n_tiles arrays gs_project wrote.  Each radix pass is one
 * kernel whose blocks wait (bounded) on the counts of the blocks before
 * them; a wait that runs out sets GS_FLAG_SORT_STALL.
 */
gs_status gs_sort_tiles_workspace(int32_t n_gaussians, const gs_batch* batch,
                                  size_t capacity, size_t* ws_bytes);
gs_status gs_sort_tiles(int32_t n_gaussians, const gs_cameras* cams,
                        const gs_batch* batch,
                        const gs_projected* proj, uint32_t* tiles,
                        uint32_t* vals, size_t capacity, uint32_t* ranges,
                        uint32_t* n_instances, void* ws, size_t ws_bytes,
                        int32_t* status, gs_stream stream);

/*
 * gs_render_fwd — front-to-back alpha compositing (Algorithm 1,
 * "Rasterize").  For each pixel, over its tile's list: alpha = min(0.99,
 * o exp(-q/2)); splats with alpha < 1/255 are skipped; the pixel stops
 * before the splat that would take its transmittance T below 1e-4;
 * C = sum c alpha T + T_final bg.  Writes image [n_pixels,3],
 * T_final [n_pixels] and n_contrib [n_pixels] (position in the tile list,
 * plus one, of the last splat added; 0 if none).  bg: [3] device.
 * n_added [n_pixels] (may be NULL) receives the number of splats added per
 * pixel (a diagnostic: the work count of the compositing).
 */
gs_status gs_render_fwd(const gs_batch* batch, const gs_cameras* cams,
                        const gs_projected* proj, const uint32_t* vals,
                        const uint32_t* ranges, const float* bg, float* image,
                        float* T_final, uint32_t* n_contrib, uint32_t* n_added,
                        gs_stream stream);

/*
 * gs_render_bwd — backward of gs_project + gs_render_fwd.
 * dL/dimage is either v_image [n_pixels,3] or, when v_image is NULL, the L1
 * term of Eq. 5 computed in place: l1_weight * sign(image - target) /
 * (3 W_b H_b) per slot (sign(0) = 0); then loss (device double, may be
 * NULL) += l1_weight * sum |image - target| / (3 W_b H_b).
 * Compositing is recomputed back to front from T_final (nothing else is
 * stored per pixel); per-splat gradients are reduced inside each tile's
 * thread block before one atomic add per splat; then the projection
 * backward accumulates dL/d(raw parameters) into dg and the per-camera pose
 * tangent into g_pose_tangent [V,6] (double, +=) for cameras views[b].
 * ws: see query (holds the screen-space gradients and block partials).
 */
gs_status gs_render_bwd_workspace(int32_t n_gaussians, const gs_batch* batch,
                                  size_t* ws_bytes);
gs_status gs_render_bwd(const gs_gaussians* g, const gs_cameras* cams,
                        const gs_batch* batch, const gs_projected* proj,
                        const uint32_t* vals, const uint32_t* ranges,
                        const float* bg, const float* image,
                        const float* T_final, const uint32_t* n_contrib,
                        const float* v_image, const float* target,
                        float l1_weight, double* loss,
                        const gs_gaussian_grads* dg, double* g_pose_tangent,
                        void* ws, size_t ws_bytes, gs_stream stream);

/*
 * gs_render_bwd_det, gs_raster_bwd_det — the same backward (Algorithm 1,
 * "Backpropagate"; arguments and rules of gs_render_bwd / gs_raster_bwd)
 * with results that do not depend on the order in which tiles run: two
 * calls on the same inputs give bit-identical gradients and loss.  Each
 * (record, tile) instance writes its sums into a slot of its own; the
 * per-record sums are then formed in a fixed order (the record's tiles in
 * row-major order of its tile rectangle), and the fused L1 loss is summed
 * over the tiles in tile order.  capacity and n_instances: the instance
 * capacity given to gs_sort_tiles and the count it wrote (device); when
 * the lists do not hold every instance (GS_FLAG_CAPACITY or
 * GS_FLAG_SORT_STALL raised by the sort) all screen-space gradients are
 * zero.  ws: gs_render_bwd_det_workspace() bytes, 256-byte aligned
 * (its start is laid out like gs_render_bwd's workspace, so gs_project_bwd
 * takes it too).  Slower than gs_render_bwd (the slots are written and read
 * once: 36 bytes per instance each way) and the workspace grows with the
 * capacity.
 */
gs_status gs_render_bwd_det_workspace(int32_t n_gaussians, const gs_batch* batch,
                                      size_t capacity, size_t* ws_bytes);
gs_status gs_raster_bwd_det(const gs_gaussians* g, const gs_cameras* cams,
                            const gs_batch* batch, const gs_projected* proj,
                            const uint32_t* vals, const uint32_t* ranges,
                            const uint32_t* n_instances, const float* bg, const float* image,
                            const float* T_final, const uint32_t* n_contrib,
                            const float* v_image, const float* target,
                            float l1_weight, double* loss, size_t capacity,
                            void* ws, size_t ws_bytes, gs_stream stream);
gs_status gs_render_bwd_det(const gs_gaussians* g, const gs_cameras* cams,
                            const gs_batch* batch, const gs_projected* proj,
                            const uint32_t* vals, const uint32_t* ranges,
                            const uint32_t* n_instances, const float* bg, const float* image,
                            const float* T_final, const uint32_t* n_contrib,
                            const float* v_image, const float* target,
                            float l1_weight, double* loss, size_t capacity,
                            const gs_gaussian_grads* dg, double* g_pose_tangent,
                            void* ws, size_t ws_bytes, gs_stream stream);

/*
 * gs_photo_loss — the photometric loss of Eq. 5 (Algorithm 1, "L_photo")
 * of every slot of the batch, and its gradient with respect to the rendered
 * image, to be passed to gs_render_bwd / gs_raster_bwd as v_image:
 *   loss += sum_b [ l1_weight * mean_b |image - target|
 *                   + ssim_weight * (1 - mean_b SSIM(image, target)) ]
 * with mean_b over the 3 W_b H_b values of slot b; the paper's weights are
 * l1_weight = 1 - lambda_SSIM = 0.8, ssim_weight = lambda_SSIM = 0.2.
 * v_image [n_pixels,3] = dL/dimage, overwritten (sign(0) = 0 in the L1
 * part).  SSIM is the index of Wang et al. (2004) as 3DGS trains with it
 * (the paper fixes only its weight): per colour channel, an 11x11 Gaussian
 * window of sigma 1.5 whose 1-D taps sum to 1, C1 = 0.01^2, C2 = 0.03^2,
 * zero padding outside the view (the window is not renormalised there).
 * image, target: [n_pixels,3] in the batch's pixel layout (slot b's W_b x
 * H_b pixels, row-major, from px_offset[b]); loss: device double, may be
 * NULL.  ws: gs_photo_loss_workspace() bytes, 4-byte aligned (nine floats
 * per pixel, the per-pixel factors of the SSIM gradient, and a list of the
 * batch's 32x32 pixel blocks).  GS_ERR_ARG for a NULL image, target or
 * v_image, a negative or non-finite weight, or a short or misaligned
 * workspace; GS_ERR_UNSUPPORTED above (2^31 - 1) / 3 pixels in the batch.
 */
gs_status gs_photo_loss_workspace(const gs_batch* batch, size_t* ws_bytes);
gs_status gs_photo_loss(const gs_cameras* cams, const gs_batch* batch,
                        const float* image, const float* target,
                        float l1_weight, float ssim_weight, double* loss,
                        float* v_image, void* ws, size_t ws_bytes,
                        gs_stream stream);

/*
 * The two halves of gs_render_bwd, callable separately (same arguments and
 * workspace; gs_render_bwd == gs_raster_bwd then gs_project_bwd):
 *  gs_raster_bwd   zeroes the screen-space gradient records in ws, then runs
 *                  the compositing backward (fused L1 when v_image is NULL)
 *                  and accumulates per-record gradients of (mean2d, conic,
 *                  opacity, colour) into ws;
 *  gs_project_bwd  chains those records through the projection into dg and
 *                  g_pose_tangent.
 */
gs_status gs_raster_bwd(const gs_gaussians* g, const gs_cameras* cams,
                        const gs_batch* batch, const gs_projected* proj,
                        const uint32_t* vals, const uint32_t* ranges,
                        const float* bg, const float* image,
                        const float* T_final, const uint32_t* n_contrib,
                        const float* v_image, const float* target,
                        float l1_weight, double* loss, void* ws,
                        size_t ws_bytes, gs_stream stream);
/*
 * gs_raster_bwd_zeroed — gs_raster_bwd without its first step: the caller
 * has already zeroed the screen-space records, the first
 * B * n_gaussians * 12 floats of ws (for instance with gs_zero on another
 * stream, overlapping earlier work, and ordered before this call).
 */
gs_status gs_raster_bwd_zeroed(const gs_gaussians* g, const gs_cameras* cams,
                               const gs_batch* batch, const gs_projected* proj,
                               const uint32_t* vals, const uint32_t* ranges,
                               const float* bg, const float* image,
                               const float* T_final, const uint32_t* n_contrib,
                               const float* v_image, const float* target,
                               float l1_weight, double* loss, void* ws,
                               size_t ws_bytes, gs_stream stream);
gs_status gs_project_bwd(const gs_gaussians* g, const gs_cameras* cams,
                         const gs_batch* batch, const gs_projected* proj,
                         const gs_gaussian_grads* dg, double* g_pose_tangent,
                         void* ws, size_t ws_bytes, gs_stream stream);
/*
 * gs_project_bwd_clearing — gs_project_bwd (same arguments and results)
 * that also leaves the screen-space records zero behind it: each record is
 * zeroed right after it is read, all B * n_gaussians of them.  A following
 * gs_raster_bwd_zeroed on the same workspace then needs no clearing pass
 * (the first one after allocation still does).  FP32.
 */
gs_status gs_project_bwd_clearing(const gs_gaussians* g, const gs_cameras* cams,
                                  const gs_batch* batch,
                                  const gs_projected* proj,
                                  const gs_gaussian_grads* dg,
                                  double* g_pose_tangent, void* ws,
                                  size_t ws_bytes, gs_stream stream);

/*
 * track_reproj_fwd_bwd — Eq. 6 for the observations of the batch's views
 * (Algorithm 1, "Joint BA loss on track points").  Observations are
 * bucketed by camera: those of camera i are obs [view_obs_offset[i],
 * view_obs_offset[i+1]); observation o sees track point obs_point[o] at
 * pixel obs_xy[o] (continuous coordinates, pixel centres at +0.5).
 * For each: X_c = R_i X + t_i; masked (counted in n_masked) if Z_c <= near;
 * r = pi_i(X) - x; rho = |r|^2 if |r| <= delta else 2 delta |r| - delta^2.
 * loss (device double) += sum rho; grad_X [n_points,3] += weight * d rho/dX;
 * g_pose_tangent [V,6] (double) += weight * d rho / d(pose tangent).
 * n_masked (device uint32, may be NULL) += masked count.
 */
gs_status track_reproj_workspace(const gs_batch* batch, size_t* ws_bytes);
gs_status track_reproj_fwd_bwd(const float* X, int32_t n_points,
                               const int32_t* obs_point, const float* obs_xy,
                               const int64_t* view_obs_offset,
                               const gs_cameras* cams, const gs_batch* batch,
                               float delta, float weight, double* loss,
                               float* grad_X, double* g_pose_tangent,
                               uint32_t* n_masked, void* ws, size_t ws_bytes,
                               gs_stream stream);

/*
 * track_reproj_fwd_bwd_det — the same term (arguments, workspace and rules
 * of track_reproj_fwd_bwd) with results that do not depend on the order in
 * which threads run, given that no track point has two observations in one
 * camera (a track sees each image once): the slots are processed one
 * launch after another in slot order, each block and warp keeps its own
 * sums, and the loss and pose sums are formed in block order.  Two calls
 * on the same inputs give bit-identical loss, grad_X and g_pose_tangent.
 * 3 B launches instead of 2 (per slot: the kernel, the pose sums and the
 * loss sum).
 */
gs_status track_reproj_fwd_bwd_det(const float* X, int32_t n_points,
                                   const int32_t* obs_point, const float* obs_xy,
                                   const int64_t* view_obs_offset,
                                   const gs_cameras* cams, const gs_batch* batch,
                                   float delta, float weight, double* loss,
                                   float* grad_X, double* g_pose_tangent,
                                   uint32_t* n_masked, void* ws, size_t ws_bytes,
                                   gs_stream stream);

/*
 * track_reproj_fwd_bwd_static — the same computation as track_reproj_fwd_bwd
 * with the same arguments except `ws`/`ws_bytes`: it allocates nothing and
 * needs no workspace from the caller.  The paper has no counterpart; this
 * entry point exists for callers that cannot allocate device memory when they
 * run the track term: real-time loops that must not risk the implicit device
 * synchronisation an allocation can cause, plug-ins that live inside a host
 * framework's memory pool and may not allocate outside it, and processes that
 * reserve all device memory up front.
 * Its scratch (the per-block pose partials) is a 1 MiB array in device
 * memory owned by the library; every GPU that loads the library keeps it
 * until the process exits.  A batch whose partials need more than 1 MiB
 * (2 x SM count x B x 48 bytes; never on GPUs with up to 170 SMs) is
 * rejected with GS_ERR_CAPACITY.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current and
 * caches it; make that first call before any stream capture.  All calls
 * share the one array and it keeps the last call's contents (every call
 * overwrites all the partials it reads, so nothing needs clearing): calls
 * that overlap on the GPU, on different streams or devices sharing the
 * process, race on it and must be serialised by the caller.
 */
gs_status track_reproj_fwd_bwd_static(const float* X, int32_t n_points,
                                      const int32_t* obs_point,
                                      const float* obs_xy,
                                      const int64_t* view_obs_offset,
                                      const gs_cameras* cams,
                                      const gs_batch* batch, float delta,
                                      float weight, double* loss,
                                      float* grad_X, double* g_pose_tangent,
                                      uint32_t* n_masked, gs_stream stream);

/*
 * sfm_ba_assemble — the iteratively reweighted Gauss-Newton blocks of one
 * Levenberg-Marquardt iteration of the SfM bundle adjustment of Eq. 4
 * (Sec. 3.2, "Bundle Adjustment"), over n_obs observations o = (camera
 * obs_cam[o], point obs_point[o], pixel obs_xy[o]) with the residual
 * r = pi_i(X_k) - x (pi of Eq. 4, poses and intrinsics from cams) and the
 * Huber weight w = rho'(|r|^2) (rho as for Eq. 6: s for s <= delta^2, else
 * 2 delta sqrt(s) - delta^2).  Pose derivatives are taken with respect to
 * a left perturbation T <- Exp(d) T, d = (rho, phi).  Accumulated (+=), in
 * double precision:
 *   U  [V,36]  sum w Jp^T Jp per camera (row-major 6x6)
 *   Vp [P,9]   sum w JX^T JX per point (row-major 3x3)
 *   gc [V,6]   sum w Jp^T r per camera;   gp [P,3]  sum w JX^T r per point
 *   objective  sum rho(|r|^2) (device double, may be NULL)
 * and written per observation: Wo [n_obs,18] = w Jp^T JX (row-major 6x3).
 * An observation whose camera depth is <= cams->near_plane, or whose camera
 * or point index is out of range, contributes nothing (its Wo row is zero).
 * All arrays are device memory owned by the caller; the arithmetic is
 * double precision.  GS_ERR_ARG for null arrays or negative sizes.
 */
gs_status sfm_ba_assemble(const float* X, int32_t n_points,
                          const gs_cameras* cams, const int32_t* obs_point,
                          const int32_t* obs_cam, const float* obs_xy,
                          int64_t n_obs, float delta, double* U, double* Vp,
                          double* gc, double* gp, double* Wo,
                          double* objective, gs_stream stream);

/*
 * sfm_ba_schur — eliminates the points from the damped normal equations of
 * one LM iteration of Eq. 4 (the blocks of sfm_ba_assemble):
 *   S [6V,6V] = U_d - sum_k W_ik V_k^-1 W_jk^T   (row-major; S is
 *               symmetric and only its lower triangle is formed, which is
 *               all sfm_ba_solve_cameras reads; the rest is not meaningful),
 *   rhs [6V]  = -gc + sum_k W_ik V_k^-1 gp_k      (written),
 *   Vinv [P,9] = V_k^-1 of the damped point blocks (written),
 * with the Marquardt damping A_d = A + lambda diag(A) of every camera block
 * U_i and point block V_k; a block with no observation (all zero) is taken
 * as the identity with a zero right-hand side.  The observations of point
 * k are point_obs[point_obs_offset[k] .. point_obs_offset[k+1]), a CSR list
 * the caller builds (offsets non-decreasing, [P+1]); entries outside
 * [0, n_obs) and cameras outside [0, V) are skipped.  No camera is singled
 * out: a caller holds camera 0 fixed by solving without its six rows and
 * columns.  lambda_dev (device double, may be NULL): when given, the
 * damping is read from it on the device and lambda is ignored (the LM loop
 * of sfm_ba_lm_accept).  Double precision; device arrays owned by the
 * caller.
 */
gs_status sfm_ba_schur(int32_t n_cams, int32_t n_points, int64_t n_obs,
                       const double* U, const double* Vp, const double* gc,
                       const double* gp, const double* Wo,
                       const int32_t* obs_cam, const int64_t* point_obs_offset,
                       const int32_t* point_obs, double lambda,
                       const double* lambda_dev, double* S, double* rhs,
                       double* Vinv, gs_stream stream);

/*
 * sfm_ba_pair_lists — HOST-side plan of the elimination by camera pairs
 * (sfm_ba_schur_pairs), built once per problem: the observation structure
 * does not change between LM iterations.  All pointers are host memory.
 * Inputs as for sfm_ba_schur (obs_cam [n_obs], the CSR point lists
 * point_obs_offset [n_points+1], point_obs).  An incidence (k, a, b) is an
 * ordered pair of observations a, b of point k whose cameras satisfy
 * obs_cam[b] <= obs_cam[a] (entries outside [0, n_obs) and cameras outside
 * [0, n_cams) are skipped); incidences are grouped by camera pair (ca, cb)
 * in order of (ca, cb), within a pair in order of k, then of a's and b's
 * positions in the point's list, and each pair's list is cut into chunks of
 * at most `chunk` (> 0) incidences.  Outputs:
 *   n_inc, n_pairs, n_chunks   the sizes (always written);
 *   inc [n_inc,3] (k, a, b), pair_cams [n_pairs,2] (ca, cb),
 *   pair_chunks [n_pairs+1] (the chunks of pair p are
 *   [pair_chunks[p], pair_chunks[p+1])), chunk_start [n_chunks+1] (the
 *   incidences of chunk j are [chunk_start[j], chunk_start[j+1])): written
 *   only when all four are non-NULL, so a first call with them NULL sizes
 *   the arrays.  GS_ERR_ARG for null inputs, negative sizes or chunk <= 0.
 */
gs_status sfm_ba_pair_lists(int32_t n_cams, int32_t n_points, int64_t n_obs,
                            const int32_t* obs_cam,
                            const int64_t* point_obs_offset,
                            const int32_t* point_obs, int32_t chunk,
                            int64_t* n_inc, int32_t* n_pairs,
                            int32_t* n_chunks, int32_t* inc,
                            int32_t* pair_cams, int32_t* pair_chunks,
                            int64_t* chunk_start);

/*
 * sfm_ba_schur_pairs_workspace — bytes of device workspace that
 * sfm_ba_schur_pairs needs for n_obs observations and n_chunks chunks
 * (per observation W V^-1 and W V^-1 g; per chunk its 42 partial sums).
 */
gs_status sfm_ba_schur_pairs_workspace(int64_t n_obs, int32_t n_chunks,
                                       size_t* bytes);

/*
 * sfm_ba_schur_pairs — the elimination of sfm_ba_schur (same S lower
 * triangle, rhs and Vinv, same damping and same conventions), summed by
 * camera pairs from the plan of sfm_ba_pair_lists (its arrays copied to the
 * device as they are) instead of with atomics: every entry of S and rhs is
 * formed in one fixed order, so the result is bit-reproducible; it equals
 * sfm_ba_schur's up to the order of the FP64 sums.  ws: device workspace
 * of sfm_ba_schur_pairs_workspace(n_obs, n_chunks) bytes.  GS_ERR_ARG for
 * null arrays, negative sizes or a small workspace.
 */
gs_status sfm_ba_schur_pairs(int32_t n_cams, int32_t n_points, int64_t n_obs,
                             const double* U, const double* Vp,
                             const double* gc, const double* gp,
                             const double* Wo, const int32_t* obs_cam,
                             const int64_t* point_obs_offset,
                             const int32_t* point_obs, const int32_t* inc,
                             const int32_t* pair_cams, int32_t n_pairs,
                             const int32_t* pair_chunks,
                             const int64_t* chunk_start, int32_t n_chunks,
                             double lambda, const double* lambda_dev,
                             double* S, double* rhs, double* Vinv, void* ws,
                             size_t ws_bytes, gs_stream stream);

/*
 * sfm_ba_lm_accept — the accept / reject decision of one LM iteration of
 * Eq. 4, on the device (so that a whole iteration can be captured in a
 * CUDA graph and replayed without reading anything back).  objective [2]
 * (device double): the robust objective at the current parameters and at
 * the trial ones (sfm_ba_apply_step, then sfm_ba_objective into
 * objective + 1).  If the trial one is lower: Rt [V,12] <- Rt_trial,
 * X [P,3] <- X_trial, objective[0] <- objective[1], *lambda (device double,
 * the damping read by sfm_ba_schur through lambda_dev) /= 10 and
 * *n_accepted += 1 (device int32, may be NULL); else *lambda *= 10.  With
 * n_iter (device int32, may be NULL): history[*n_iter] <- objective[0]
 * while *n_iter < history_len (history may be NULL), then *n_iter += 1.
 */
gs_status sfm_ba_lm_accept(int32_t n_cams, int32_t n_points, double* objective,
                           double* lambda, float* Rt, float* X,
                           const float* Rt_trial, const float* X_trial,
                           int32_t* n_accepted, double* history,
                           int32_t history_len, int32_t* n_iter,
                           gs_stream stream);

/*
 * sfm_ba_back_substitute — the points' step once the cameras' step
 * dc [V,6] is known: dp_k = V_k^-1 (-gp_k - sum_i W_ik^T dc_i), dp [P,3]
 * written (Vinv from sfm_ba_schur; a point with no observation gets 0).
 * Same observation lists and skipping rules as sfm_ba_schur.
 */
/*
 * sfm_ba_solve_cameras — solves the reduced camera system of sfm_ba_schur
 * with camera 0 held fixed: S' dc' = rhs' over cameras 1..V-1, S' being S
 * without camera 0's six rows and columns.  S is overwritten (its lower
 * triangle below camera 0 holds the Cholesky factor of S', and camera 0's
 * rows are scratch: the reciprocals of the factor's diagonal among them);
 * dc [V,6] is written, row 0 zero.  The factorization
 * is tiled (32 x 32 tiles): per tile column one launch factors the
 * diagonal tile, one solves the tiles below it and one updates the
 * trailing tiles, a block per tile, so the O(n^3 / 6) flops (n = 6 (V - 1))
 * spread over the SMs; 3 ceil(n / 32) + 2 launches in all, none of which
 * synchronises with the host (the triangular solves keep the n unknowns in
 * one block's shared memory: up to GS_MAX_BA_CAMERAS cameras, else
 * GS_ERR_UNSUPPORTED).  A pivot <= 0 leaves dc zero and ORs
 * GS_FLAG_NOT_SPD into the device word *status (may be NULL).
 */
gs_status sfm_ba_solve_cameras(int32_t n_cams, double* S, const double* rhs,
                               double* dc, int32_t* status, gs_stream stream);

/*
 * sfm_ba_objective — the objective of Eq. 4 alone, sum rho(|r|^2) over the
 * observations (same readings and skipping rules as sfm_ba_assemble),
 * added (+=) to the device double *objective.
 */
gs_status sfm_ba_objective(const float* X, int32_t n_points,
                           const gs_cameras* cams, const int32_t* obs_point,
                           const int32_t* obs_cam, const float* obs_xy,
                           int64_t n_obs, float delta, double* objective,
                           gs_stream stream);

/*
 * sfm_ba_apply_step — the trial parameters of an LM step: T_i' =
 * Exp(dc_i) T_i (left perturbation, translation first, computed in double
 * and stored as float into Rt_out [V,12]) and X_k' = X_k + dp_k (X_out
 * [P,3]).  Outputs must not alias the inputs.
 */
gs_status sfm_ba_apply_step(int32_t n_cams, int32_t n_points, const float* Rt,
                            const float* X, const double* dc, const double* dp,
                            float* Rt_out, float* X_out, gs_stream stream);

gs_status sfm_ba_back_substitute(int32_t n_cams, int32_t n_points,
                                 int64_t n_obs, const double* Vinv,
                                 const double* Vp, const double* gp,
                                 const double* Wo, const int32_t* obs_cam,
                                 const int64_t* point_obs_offset,
                                 const int32_t* point_obs, const double* dc,
                                 double* dp, gs_stream stream);

/*
 * pose_se3_update — pose composition of Algorithm 1 (T_i = T_i^(0) (+)
 * dT_i, read as T_i = Exp(xi_i) T_i^(0), xi = (rho, phi)) and the pose
 * step ("Update poses"; Sec. 3.3: Adam, learning rate 1e-5).  For every
 * camera: g_xi = Jl(xi)^T g_tangent with the closed-form SE(3) left
 * Jacobian; if hp is not NULL, one Adam step on xi with g_xi (moments m,
 * v); then Rt_out = Exp(xi) T0.  Computed in double per camera.
 * T0, Rt_out: [V,12]; xi, g_xi (may be NULL), m, v: [V,6] float;
 * g_tangent: [V,6] double.
 */
gs_status pose_se3_update(int32_t n_cams, const float* T0, float* xi,
                          const double* g_tangent, float* g_xi, float* m,
                          float* v, const gs_adam* hp, float* Rt_out,
                          gs_stream stream);

/*
 * FP64 instantiation of the projection and compositing: the same kernels as
 * gs_project, gs_sort_tiles, gs_render_fwd, gs_raster_bwd, gs_project_bwd
 * and gs_render_bwd (same algorithm, same order of operations, same
 * arguments and rules) computing in double, for checking the differentiable
 * path against finite differences at double precision (Algorithm 1,
 * "Backpropagate").  Per-pixel buffers (image, T_final, v_image, target,
 * bg) are double; the tile lists are shared with the FP32 path (the depth
 * key is the float rounding of the double depth, so depths within float
 * rounding of each other keep index order).  The compositing kernels stage
 * 64 splats per round whatever the tuning says.  The workspace of
 * gs_render_bwd_f64 holds double screen-space records.
 */
gs_status gs_project_f64(const gs_gaussians_f64* g, const gs_cameras_f64* cams,
                         const gs_batch* batch, const gs_projected_f64* out,
                         int32_t* status, gs_stream stream);
gs_status gs_sort_tiles_f64(int32_t n_gaussians, const gs_cameras_f64* cams,
                            const gs_batch* batch,
                            const gs_projected_f64* proj, uint32_t* tiles,
                            uint32_t* vals, size_t capacity, uint32_t* ranges,
                            uint32_t* n_instances, void* ws, size_t ws_bytes,
                            int32_t* status, gs_stream stream);
gs_status gs_render_fwd_f64(const gs_batch* batch, const gs_cameras_f64* cams,
                            const gs_projected_f64* proj, const uint32_t* vals,
                            const uint32_t* ranges, const double* bg,
                            double* image, double* T_final, uint32_t* n_contrib,
                            uint32_t* n_added, gs_stream stream);
gs_status gs_render_bwd_workspace_f64(int32_t n_gaussians,
                                      const gs_batch* batch, size_t* ws_bytes);
gs_status gs_raster_bwd_f64(const gs_gaussians_f64* g,
                            const gs_cameras_f64* cams, const gs_batch* batch,
                            const gs_projected_f64* proj, const uint32_t* vals,
                            const uint32_t* ranges, const double* bg,
                            const double* image, const double* T_final,
                            const uint32_t* n_contrib, const double* v_image,
                            const double* target, double l1_weight,
                            double* loss, void* ws, size_t ws_bytes,
                            gs_stream stream);
gs_status gs_project_bwd_f64(const gs_gaussians_f64* g,
                             const gs_cameras_f64* cams, const gs_batch* batch,
                             const gs_projected_f64* proj,
                             const gs_gaussian_grads_f64* dg,
                             double* g_pose_tangent, void* ws, size_t ws_bytes,
                             gs_stream stream);
gs_status gs_render_bwd_f64(const gs_gaussians_f64* g,
                            const gs_cameras_f64* cams, const gs_batch* batch,
                            const gs_projected_f64* proj, const uint32_t* vals,
                            const uint32_t* ranges, const double* bg,
                            const double* image, const double* T_final,
                            const uint32_t* n_contrib, const double* v_image,
                            const double* target, double l1_weight,
                            double* loss, const gs_gaussian_grads_f64* dg,
                            double* g_pose_tangent, void* ws, size_t ws_bytes,
                            gs_stream stream);
/* pose_se3_update_f64 — pose_se3_update on double arrays (T0, xi, g_xi, m,
 * v, Rt_out), for the FP64 path. */
gs_status pose_se3_update_f64(int32_t n_cams, const double* T0, double* xi,
                              const double* g_tangent, double* g_xi, double* m,
                              double* v, const gs_adam* hp, double* Rt_out,
                              gs_stream stream);

/* gs_adam_update — one Adam step on n floats p with gradient g and
 * moments m, v (Kingma & Ba, bias-corrected with t = *hp->step). */
gs_status gs_adam_update(float* p, const float* g, float* m, float* v,
                         int64_t n, const gs_adam* hp, gs_stream stream);

/* gs_adam_update_groups — gs_adam_update on up to 8 arrays in one launch,
 * each with its own learning rate (hp->lr is ignored). */
gs_status gs_adam_update_groups(const gs_adam_group* groups, int32_t n_groups,
                                const gs_adam* hp, gs_stream stream);

/*
 * gs_mcmc_relocate — the relocation step of the MCMC densification the
 * paper trains with (Sec. 3.3; Algorithm 1 "Relocate / add Gaussians"),
 * with the cited method's rules, in place on the N Gaussians' parameters
 * (same layouts as gs_gaussians):
 *  - a Gaussian is dead when sigmoid(opacity_logit) <= 0.005;
 *  - the dead one of rank r (index order among the dead) draws a live
 *    source with the uniform u[r] in [0,1): the first j whose cumulative
 *    live opacity exceeds u[r] times the total (dead ranks >= n_u, or no
 *    live Gaussian, are left as they are; src -1);
 *  - a source drawn c times and its copies become N = c + 1 identical
 *    Gaussians with opacity o_N = 1 - (1 - o)^(1/N) and scales
 *    s o / sum_{m=1..N} C(N,m) (-1)^(m-1) o_N^m / sqrt(m);
 *    (o_N, then bounded to [0.005, 1 - 2^-23], the scale taking the
 *    unbounded o_N: a copy is never born dead and its logit stays finite);
 *  - each dead Gaussian then copies its source's (reset) parameters.
 * A draw always lands on a live Gaussian.  src [N] (int32) gets each
 * Gaussian's source or -1; n_dead (device uint32, may be NULL) the number
 * of dead Gaussians.  The Adam moments are not touched: the cited method
 * restarts them for every relocated Gaussian and its source, which
 * gs_mcmc_reset_moments(N, src, N, 0, ...) does.  ws: gs_mcmc_workspace(N)
 * bytes.  GS_ERR_ARG for null arrays, negative sizes or a short workspace.
 */
gs_status gs_mcmc_workspace(int32_t n, size_t* ws_bytes);
gs_status gs_mcmc_relocate(int32_t n, int32_t sh_degree, float* mean,
                           float* log_scale, float* quat, float* opacity_logit,
                           float* sh, const double* u, int32_t n_u,
                           int32_t* src, uint32_t* n_dead, void* ws,
                           size_t ws_bytes, gs_stream stream);

/*
 * gs_mcmc_grow — the growth step of the same densification (Sec. 3.3, "max
 * 3M Gaussians"; Algorithm 1 "Relocate / add Gaussians"), with the cited
 * method's rule: n_add new Gaussians are appended after the n existing ones
 * (the caller picks n_add; the cited rule is min(cap, floor(1.05 n)) - n).
 * New Gaussian k draws a live source with the uniform u[k] in [0,1) exactly
 * as gs_mcmc_relocate draws for a dead one; a source drawn c times has its
 * opacity and scales reset for N = c + 1 as there; row n + k then copies
 * its source's reset parameters.  The parameter arrays must hold n + n_add
 * rows (rows n.. are overwritten); u [n_add] double; src [n_add] (int32)
 * gets each new Gaussian's source (-1 when none is live, the row then left
 * as it was).  ws: gs_mcmc_workspace(n) bytes.  Restart the moments with
 * gs_mcmc_reset_moments(n + n_add, src, n_add, n, ...).
 */
gs_status gs_mcmc_grow(int32_t n, int32_t n_add, int32_t sh_degree, float* mean,
                       float* log_scale, float* quat, float* opacity_logit,
                       float* sh, const double* u, int32_t* src, void* ws,
                       size_t ws_bytes, gs_stream stream);

/*
 * gs_mcmc_reset_moments — zeroes the Adam moments (m and v of up to 8
 * gs_adam_group entries; p, g and lr are not read) of the Gaussians that a
 * relocation or a growth step wrote, as the cited method restarts them: for
 * every k < n_src with src[k] >= 0, rows row0 + k and src[k].  Each group
 * holds n_rows rows of n / n_rows floats.  GS_ERR_ARG for more than 8
 * groups, a group size that is not a multiple of n_rows, or row0 + n_src >
 * n_rows.
 */
gs_status gs_mcmc_reset_moments(int32_t n_rows, const int32_t* src,
                                int32_t n_src, int32_t row0,
                                const gs_adam_group* groups, int32_t n_groups,
                                gs_stream stream);

/*
 * gs_mcmc_noise — the cited method's noise on the means (the MCMC
 * exploration term): mean += noise_lr * sigmoid(-100 (o - 0.005)) *
 * Sigma eta, Sigma = R diag(exp(log_scale))^2 R^T, eta [N,3] given
 * (standard normal draws).  Computed in float; quat 16-byte aligned.
 */
gs_status gs_mcmc_noise(int32_t n, float* mean, const float* log_scale,
                        const float* quat, const float* opacity_logit,
                        const float* eta, float noise_lr, gs_stream stream);

/* gs_step_advance — *step += 1 on the device. */
gs_status gs_step_advance(int32_t* step, gs_stream stream);

/* gs_gather_view_pixels — for every slot b of the batch, copies the
 * per-pixel data of camera views[b] from a dataset buffer holding all
 * cameras (camera v's pixels start at element src_px_offset[v], [V+1]) into
 * slot b's place in a batch-packed buffer (px_offset[b]); `channels` floats
 * per pixel.  Used to fetch a batch's target images (Algorithm 1, "Sample
 * image indices") without the host reading the view ids, so a captured step
 * stays valid when only the device copy of views changes. */
gs_status gs_gather_view_pixels(const float* src, const int64_t* src_px_offset,
                                const gs_cameras* cams, const gs_batch* batch,
                                int32_t channels, float* dst, gs_stream stream);

/* gs_batch_layout — the batch's offsets from its view ids, on the device
 * (Algorithm 1, "Sample image indices", for a batch whose views are chosen
 * on the device or swapped between replays of a captured step):
 *   px_offset[b + 1] = px_offset[b] + W_v H_v,
 *   tile_offset[b + 1] = tile_offset[b] + ceil(W_v / T) ceil(H_v / T)
 * for v = batch->views[b], T = batch->tile, px_offset[0] = tile_offset[0]
 * = 0.  px_offset [B+1] (8-byte aligned) and tile_offset [B+1] are device
 * arrays, normally the batch's own.  batch->n_pixels and batch->n_tiles are
 * the capacity: the first slot whose pixels or tiles would exceed it, and
 * every later slot, gets zero pixels and tiles (so they are not rendered)
 * and GS_FLAG_CAPACITY is OR-ed into *status (may be NULL). */
gs_status gs_batch_layout(const gs_cameras* cams, const gs_batch* batch,
                          int64_t* px_offset, int32_t* tile_offset,
                          int32_t* status, gs_stream stream);

/* gs_zero — set `bytes` bytes at ptr to zero on the stream. */
gs_status gs_zero(void* ptr, size_t bytes, gs_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* GS_H */
