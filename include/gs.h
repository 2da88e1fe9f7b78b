/*
 * gs.h — C ABI of the GB300 (sm_103a) differentiable 3D-Gaussian rasterizer.
 *
 * The library renders a map of 3D Gaussians (mean, covariance, opacity and colour:
 * the scene model of Sec. II-A of "Real-time Photorealistic Mapping for Situational
 * Awareness in Robot Teleoperation") from K camera poses and differentiates the
 * result back to the Gaussians and the poses, which is what the mapping optimiser
 * (render I1 of Fig. 3) and render-based pose tracking (Sec. II-B) call every
 * iteration. The paper names this renderer but does not write it out; the reading
 * implemented here is the tile-based EWA splatting rasterizer:
 *
 *   gs_project      per (view, Gaussian): 2D mean, conic, depth, radius, tile rectangle
 *   gs_bin_sort     prefix sum of tiles touched, one (tile, Gaussian) pair per tile an item
 *                   touches, stored as the key (tile << 32 | Gaussian id) with its emission
 *                   index as the value, put in the order of the (tile << 32 | depth bits)
 *                   keys by stable onesweep LSD radix sorts; per-tile [start, end) ranges
 *   gs_raster_fwd   front-to-back alpha compositing of colour, depth, transmittance
 *   gs_loss_l1      photometric L1(RGB) + lambda L1(depth) and its image gradient
 *   gs_raster_bwd   reverse of the compositing into per-(Gaussian, tile) gradients
 *   gs_project_bwd  reverse of the projection into means, log-scales, quaternions,
 *                   opacity logits, colours and the se(3) camera poses
 *
 * Conventions shared by every call
 * --------------------------------
 * - Pointers named d_* and every array argument are DEVICE pointers unless the
 *   comment says "host". Arrays are C-contiguous, structure of arrays.
 * - `stream` is a cudaStream_t passed as void*; NULL means the legacy default stream.
 *   Every call except gs_read_status only enqueues work on `stream` and returns.
 * - The library never allocates device memory. The caller owns every buffer and
 *   provides one opaque workspace `ws` of at least gs_workspace_size() bytes,
 *   256-byte aligned. The workspace carries state from gs_project through
 *   gs_project_bwd; calls on one workspace must be ordered on one stream.
 * - Synchronous errors (bad arguments, undersized workspace, launch failure) are
 *   returned as gs_status_t and nothing is enqueued. Errors found on the device
 *   (pair capacity exceeded, a bounded wait that gave up, non-finite input) set
 *   bits of a device error word inside `ws`; gs_read_status returns it. Kernels
 *   never trap.
 * - Gradient outputs are ACCUMULATED (+=). The caller zeroes them; summing over
 *   several calls or views is how batches accumulate.
 * - Images: rgb is [K,3,H,W] (planar), depth / T_final / last are [K,H,W]; pixel
 *   (i, j) is sampled at its centre (i + 0.5, j + 0.5).
 */
#ifndef GS_H_
#define GS_H_

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define GS_API __attribute__((visibility("default")))
#else
#define GS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GS_OK = 0,
  GS_ERR_INVALID_ARG = 1,          /* null pointer, size out of range, misaligned ws */
  GS_ERR_WORKSPACE_TOO_SMALL = 2,  /* ws_bytes < gs_workspace_size() */
  GS_ERR_CAPACITY_OVERFLOW = 3,    /* returned by gs_read_status when the device word says so */
  GS_ERR_DEVICE_TIMEOUT = 4,       /* returned by gs_read_status: a bounded device wait gave up */
  GS_ERR_CUDA = 5,                 /* a CUDA runtime call or kernel launch failed */
  GS_ERR_NONFINITE = 6,            /* returned by gs_read_status: non-finite input seen */
  GS_ERR_SIZE_LIMIT = 7,           /* n exceeds a fixed maximum (gs_sort_pairs_noalloc) */
  GS_ERR_INDEX_CHECK = 8           /* returned by gs_read_status: an index check of the debug build
                                      failed (GS_DEVERR_BOUNDS; the access was skipped) */
} gs_status_t;

/* Bits of the device error word (gs_read_status). */
#define GS_DEVERR_PAIR_OVERFLOW 0x1u /* more (Gaussian, tile) pairs than pair_capacity */
#define GS_DEVERR_TIMEOUT 0x2u       /* a decoupled look-back spin hit its iteration cap */
#define GS_DEVERR_NONFINITE 0x4u     /* a mean, scale, quaternion, logit or colour was NaN/Inf */
#define GS_DEVERR_BOUNDS 0x8u        /* debug builds only (GS_DEBUG): a data-dependent index failed its
                                        bounds check; the access was skipped */

typedef enum { GS_F32 = 0, GS_BF16 = 1, GS_F16 = 2 } gs_dtype_t;

/* How a Gaussian's `rgb` array is read (gs_config_t.color_mode).
 * GS_COLOR_RGB: rgb is [N,3], the colour itself, used as is (degree-0 appearance).
 * GS_COLOR_SH:  rgb is [N,(D+1)^2,3], D = gs_config_t.sh_degree in 0..3: RGB coefficient
 *   triples of the real spherical harmonics (Condon-Shortley phase; band l, then m = -l..l),
 *   evaluated per view at the unit direction from the camera centre -R^T t to the mean
 *   (Sec. II-A: view-dependent colour). colour = max(sum_i Y_i f_i + 1/2, 0); at D = 0 this is
 *   the SH0 mapping f_0 / (2 sqrt(pi)) + 1/2. Gradients: zero where the clamp is active; the
 *   direction's gradient reaches the means and the pose translation (rho). */
typedef enum { GS_COLOR_RGB = 0, GS_COLOR_SH = 1 } gs_color_mode_t;

/* One pinhole camera, 64 bytes. R, t map world to camera: p_c = R p + t, with the
 * camera looking along +z, x right and y down. Pixel u = fx x/z + cx, v = fy y/z + cy. */
typedef struct {
  float fx, fy, cx, cy;
  float R[9]; /* row-major */
  float t[3];
} gs_camera_t;

typedef struct {
  int32_t width, height;  /* image size shared by all K views, 1..16384 */
  int32_t tile;           /* tile side in pixels; must be 16 */
  int32_t num_views;      /* K, 1..1024 */
  int64_t num_gaussians;  /* N, 0..2^31-1 */
  int64_t pair_capacity;  /* max (Gaussian, tile) pairs held by the workspace, <= 2^30 - 1 */
  float near_plane;       /* Gaussians with camera depth <= near_plane are culled (0.2) */
  float lambda_depth;     /* depth weight of gs_loss_l1 (0.1) */
  int32_t fwd_px_per_thread;  /* pixels per thread of gs_raster_fwd: 1, 2 or 4; 0 = library default */
  int32_t bwd_px_per_thread;  /* pixels per thread of gs_raster_bwd: 1, 2 or 4; 0 = library default.
                                 Every choice takes the same skip/stop decisions: forward outputs are
                                 bit-identical, gradients differ only in FP32 summation order. */
  int32_t fwd_chunk;          /* splats staged in shared memory per step of gs_raster_fwd: 64, 128 or
                                 256; 0 = library default (128). Outputs do not depend on it. */
  int32_t bwd_chunk;          /* the same for gs_raster_bwd: 32, 64 or 128; 0 = default (64).
                                 Gradients do not depend on it. */
  int32_t color_mode;         /* gs_color_mode_t; 0 = GS_COLOR_RGB */
  int32_t sh_degree;          /* 0..3 with GS_COLOR_SH (ignored with GS_COLOR_RGB) */
  int32_t raster_blocks_per_sm; /* cap on the resident blocks per multiprocessor of the compositing
                                   kernels (gs_raster_fwd*, gs_raster_bwd): 1..32; 0 = as many as
                                   fit. Enforced by padding each block's dynamic shared memory;
                                   outputs do not depend on it. */
} gs_config_t;

/* Gaussian attributes. means may be F32 or BF16/F16 (means_dtype); the other four
 * arrays share `dtype`. All arithmetic is FP32 whatever the storage type. */
typedef struct {
  const void* means;          /* [N,3] world position */
  const void* log_scales;     /* [N,3] log of the per-axis standard deviation */
  const void* quats;          /* [N,4] (w,x,y,z), any non-zero length */
  const void* opacity_logits; /* [N]   opacity = sigmoid(logit) */
  const void* rgb;            /* [N,3] colour (GS_COLOR_RGB), or [N,(D+1)^2,3] spherical-harmonic
                                 coefficients (GS_COLOR_SH, see gs_color_mode_t) */
  gs_dtype_t dtype;
  gs_dtype_t means_dtype;
} gs_gaussians_t;

/* Gradient outputs of gs_project_bwd, FP32, accumulated (+=) or stored (overwrite); any array
 * may be NULL (skipped). */
typedef struct {
  float* means;          /* [N,3] */
  float* log_scales;     /* [N,3] */
  float* quats;          /* [N,4] w.r.t. the stored (unnormalised) quaternion */
  float* opacity_logits; /* [N] */
  float* rgb;            /* [N,3], or [N,(D+1)^2,3] with GS_COLOR_SH (the shape of the rgb input) */
  float* pose;           /* [K,6] (rho, phi): left perturbation T <- Exp(xi) T at xi = 0 */
  int32_t overwrite;     /* 0: accumulate into the arrays (+=); 1: store the gradients (=), so the
                            caller need not zero them first */
} gs_grads_t;

/* Byte offsets of the workspace sub-buffers (for inspection and tests). */
typedef struct {
  size_t total;          /* == gs_workspace_size() */
  size_t status;         /* u32 error word, u32 num_pairs (clamped), u64 total pairs, u64 evals,
                            u32[8] sort tile counters, u64 evals that blended a splat */
  size_t proj_uv;        /* float4 [K*N]: u_hi, u_lo, v_hi, v_lo (u = u_hi + u_lo) */
  size_t proj_conic;     /* float4 [K*N]: conic A, B, C (Sigma2^-1 entries 00, 01, 11), depth z */
  size_t proj_tiles;     /* int4 [K*N]: -, x0 | x1 << 16, y0 | y1 << 16, tiles emitted */
  size_t proj_depth_key; /* u32 [K*N]: binary32 bits of the camera depth (sort key low word) */
  size_t proj_radius;    /* i32 [K*N]: pixel radius */
  size_t color_opacity;  /* float4 [N]: r, g, b, opacity; [K*N] (view-major) with GS_COLOR_SH of
                            degree >= 1, whose colours depend on the view */
  size_t keys_sorted;    /* u64 [pair_capacity], valid prefix num_pairs, after gs_bin_sort:
                            (global tile id << 32) | Gaussian id */
  size_t vals_sorted;    /* u32 [pair_capacity]: emission index of each sorted pair (pairs of an
                            item occupy [pair offset, pair offset + tiles emitted)) */
  size_t ranges;         /* u32 [K*Tx*Ty][2]: [start, end) of each global tile ([0, 0) when empty) */
  size_t pair_grads;     /* float [pair_capacity][12]: per-pair gradients of gs_raster_bwd, valid
                            where the pair's bit in pair_valid is set (other pairs: zero) */
  int32_t sort_passes;   /* 8-bit LSD passes of the pair sort over the tile bits: ceil(ceil(log2(K*Tx*Ty)) / 8) */
  int32_t tiles_x, tiles_y;
  int32_t bin_sort_launches; /* kernels one gs_bin_sort launches */
  size_t pair_valid;     /* u32 [ceil(pair_capacity / 32)]: bit (slot & 31) of word slot / 32 is set
                            when gs_raster_bwd wrote the record of the pair with that slot */
  size_t live_mask;      /* u32 [ceil(K*N / 32)]: bit (i & 31) of word i / 32 is set when item
                            i = k*N + g emits at least one pair (is live). The proj_* records above
                            are written for live items only */
  int32_t project_launches;     /* kernels one gs_project launches */
  int32_t project_bwd_launches; /* kernels one gs_project_bwd launches when it stores (overwrite) parameter
                                   gradients and the pose gradient */
  size_t live_off;       /* u32 [K*N]: first pair index of each live item, the items taken in
                            increasing k*N + g order (entry j: the j-th live item); valid prefix:
                            the number of live items. The pairs of a live item occupy the slots
                            [first, first + tiles emitted) */
} gs_ws_layout_t;

/* ---------------------------------------------------------------- sizing / status */

/* Workspace bytes for `cfg` (host call, no device work). */
GS_API gs_status_t gs_workspace_size(const gs_config_t* cfg, size_t* bytes);

/* Sub-buffer offsets of the workspace for `cfg` (host call). */
GS_API gs_status_t gs_workspace_layout(const gs_config_t* cfg, gs_ws_layout_t* out);

/* Synchronises `stream`, then reads the device error word, the pair count and the
 * eval count (Gaussian-pixel evaluations of the last gs_raster_fwd_stats) into host
 * memory. Any pointer may be NULL. Returns GS_OK, or the first device error in the
 * order CAPACITY_OVERFLOW, DEVICE_TIMEOUT, NONFINITE, or GS_ERR_CUDA. */
GS_API gs_status_t gs_read_status(const gs_config_t* cfg, const void* ws, size_t ws_bytes, uint32_t* err_word,
                           int64_t* num_pairs, int64_t* evals, void* stream);

/* ---------------------------------------------------------------- the hot path */

/* Projection (Sec. II-A: Gaussians "defined by their mean, covariance and opacity").
 * For every view k < K and Gaussian g < N, with p_c = R p + t, Sigma = Rq S S^T Rq^T
 * (Rq from the normalised quaternion, S = diag(exp(log_scale))), J the perspective
 * Jacobian at p_c with x/z, y/z clamped to 1.3 * (W/2)/fx and 1.3 * (H/2)/fy:
 *   Sigma2 = J R Sigma R^T J^T + 0.3 I,   conic = Sigma2^-1,
 *   radius = ceil(3 sqrt(lambda_max)),     lambda_max = mid + sqrt(max(0.1, ((a-c)/2)^2 + b^2)),
 *   rect   = tiles whose 16x16 square meets [u - r, u + r] x [v - r, v + r],
 * culling z <= near_plane and empty rectangles. Of the rectangle, an item emits (row by
 * row) only the tiles whose square of pixel centres, widened by 0.05 px + 0.2% of the
 * ellipse's half-extent, meets the ellipse d^T Sigma2^-1 d <= 2 (l + 0.02 |l| + 1.5e-4),
 * l = ln(255 opacity): outside it the opacity stays below 1/255, so the skipped pairs
 * could never be composited. The depth key, culls, radius, rectangle and emitted tiles
 * are computed in binary32 in one fixed operation order (every step rounded once, with a
 * deterministic exp and log built from + - * / sqrt and fma), so they are reproducible bit
 * for bit. d_cams: K cameras. */
GS_API gs_status_t gs_project(const gs_config_t* cfg, const gs_gaussians_t* gaussians, const gs_camera_t* d_cams, void* ws,
                       size_t ws_bytes, void* stream);

/* Binning: sorts the (view, Gaussian) pairs of every tile by depth. Result: one pair per
 * emitted (view, Gaussian, tile), in the order of a stable sort of the keys
 * ((k*Tx*Ty + ty*Tx + tx) << 32) | depth bits emitted in (k, g) order (equal keys keep
 * (k, g) order), plus per-tile [start, end) ranges. Each sorted pair is stored as key =
 * ((k*Tx*Ty + ty*Tx + tx) << 32) | g and value = its emission index (the slot of its
 * gradient record). Computed as: a stable onesweep radix sort of the K*N items on their
 * 32-bit depth keys, an exclusive scan of tiles emitted in that order, emission in that
 * order, and a stable onesweep radix sort of the pairs on the tile bits only. The pair count stays on the device; more than pair_capacity pairs sets
 * GS_DEVERR_PAIR_OVERFLOW and only the first pair_capacity pairs are emitted. Consumes the
 * state of the preceding gs_project on the same workspace (call it once per gs_project). */
GS_API gs_status_t gs_bin_sort(const gs_config_t* cfg, void* ws, size_t ws_bytes, void* stream);

/* Forward compositing (render I1/I2 of Fig. 3). Per pixel, front to back over its
 * tile's sorted list: power = -0.5 d^T conic d with d = mean2D - pixel (skip if > 0),
 * alpha = min(0.99, opacity exp(power)) (skip if < 1/255), stop before a Gaussian whose
 * T (1 - alpha) < 1e-4, otherwise C += rgb alpha T, D += z alpha T, T *= 1 - alpha.
 * Background 0; D is the un-normalised expected depth. Writes rgb [K,3,H,W],
 * depth, T_final [K,H,W] and last [K,H,W] = 1 + list position of the last composited
 * Gaussian (0 if none); each may be NULL except what gs_raster_bwd will need. */
GS_API gs_status_t gs_raster_fwd(const gs_config_t* cfg, void* ws, size_t ws_bytes, float* rgb, float* depth,
                          float* T_final, int32_t* last, void* stream);

/* gs_raster_fwd with the same decisions and outputs that also counts, into the status
 * block read by gs_read_status, the Gaussian-pixel evaluations (list entries examined,
 * including the entry that stops a pixel) and those that blended a splat. For measurement:
 * the counting costs time, so gs_raster_fwd does not count. */
GS_API gs_status_t gs_raster_fwd_stats(const gs_config_t* cfg, void* ws, size_t ws_bytes, float* rgb, float* depth,
                                float* T_final, int32_t* last, void* stream);

/* gs_raster_fwd with gs_loss_l1 fused into its epilogue: the same rgb, depth, T_final and
 * last (bit for bit), the same dL/drgb and dL/ddepth images (bit for bit), and the loss L in
 * d_loss[0] summed per tile then over tiles in tile order (equal to gs_loss_l1's value up to
 * FP32 summation order). rgb and depth must not be NULL. */
GS_API gs_status_t gs_raster_fwd_l1(const gs_config_t* cfg, void* ws, size_t ws_bytes, float* rgb, float* depth,
                             float* T_final, int32_t* last, const float* rgb_target, const float* depth_target,
                             float* dL_drgb, float* dL_ddepth, float* d_loss, void* stream);

/* gs_raster_fwd_l1 and then gs_raster_bwd (dL_dT = NULL) in one launch: each tile's block runs
 * the backward pass of its tile as soon as its forward and loss are done, from the loss gradient,
 * colour, depth and last contributor of its pixels held in registers (no wait for every tile's
 * forward, no reload of those images). Writes everything both calls write: rgb, depth, T_final,
 * last, dL/drgb, dL/ddepth, d_loss and the per-pair gradient records that gs_project_bwd
 * consumes; bit for bit the results of the two calls when gs_config_t.bwd_px_per_thread equals
 * fwd_px_per_thread (the backward phase runs with the forward's pixels per thread). rgb, depth,
 * the targets, the gradient images and d_loss must not be NULL (else GS_ERR_INVALID_ARG); T_final
 * and last may be. The mapping step's form of the forward and backward compositing (Sec. II-B). */
GS_API gs_status_t gs_raster_fwd_l1_bwd(const gs_config_t* cfg, void* ws, size_t ws_bytes, float* rgb, float* depth,
                                         float* T_final, int32_t* last, const float* rgb_target,
                                         const float* depth_target, float* dL_drgb, float* dL_ddepth, float* d_loss,
                                         void* stream);

/* gs_raster_fwd occluded by an external surface (the digital twin's virtual objects; the
 * viewer composites the map against them): ext_depth [K,H,W] (camera depth of the surface per
 * pixel, +inf or very large = none), ext_rgb [K,3,H,W] (its colour; NULL = black). Per pixel
 * the depth-sorted list is composited until the first Gaussian at or behind the surface (not
 * composited), then the surface shows through the remaining transmittance:
 * rgb += T ext_rgb, depth += T ext_depth. T_final and last are those of the occluded pixel. */
GS_API gs_status_t gs_raster_fwd_occluded(const gs_config_t* cfg, void* ws, size_t ws_bytes, float* rgb, float* depth,
                                   float* T_final, int32_t* last, const float* ext_depth, const float* ext_rgb,
                                   void* stream);

/* Photometric loss of a mapping step: L = sum_k [ mean|R - R*| over 3HW + lambda
 * mean|D - D*| over HW ], sign(0) = 0. Writes dL/drgb [K,3,H,W], dL/ddepth [K,H,W] and
 * the scalar L to d_loss[0] (device). rgb/depth are the forward outputs. */
GS_API gs_status_t gs_loss_l1(const gs_config_t* cfg, const float* rgb, const float* depth, const float* rgb_target,
                       const float* depth_target, float* dL_drgb, float* dL_ddepth, float* d_loss, void* ws,
                       size_t ws_bytes, void* stream);

/* Backward compositing (the splat-wise back-propagation the mapping optimiser needs,
 * Sec. II-B). Inputs: the forward outputs rgb, depth, T_final, last and the upstream
 * gradients dL/drgb, dL/ddepth, dL/dT_final (dL_dT may be NULL = 0). For each
 * composited Gaussian i of a pixel, with S the colour/depth accumulated behind it:
 *   dC/dc_i = alpha_i T_i,  dC/dalpha_i = c_i T_i - S / (1 - alpha_i),
 *   dT_final/dalpha_i = -T_final / (1 - alpha_i); the 0.99 clamp passes no gradient.
 * Writes one gradient record per sorted pair into the workspace (mean2D, conic,
 * depth, opacity, colour), summed over the tile's pixels; gs_project_bwd consumes it. */
GS_API gs_status_t gs_raster_bwd(const gs_config_t* cfg, void* ws, size_t ws_bytes, const float* rgb, const float* depth,
                          const float* T_final, const int32_t* last, const float* dL_drgb, const float* dL_ddepth,
                          const float* dL_dT, void* stream);

/* Backward projection: sums each (view, Gaussian)'s pair records in a fixed order
 * (deterministic, no atomics) and applies the chain rule of gs_project to the means,
 * log-scales, quaternions (through the normalisation), opacity logits, colours and
 * the pose of each view (rho, phi), accumulating into `grads`. */
GS_API gs_status_t gs_project_bwd(const gs_config_t* cfg, const gs_gaussians_t* gaussians, const gs_camera_t* d_cams,
                           void* ws, size_t ws_bytes, const gs_grads_t* grads, void* stream);

/* Screen-space gradients of the last gs_raster_bwd, summed per (view, Gaussian): for
 * inspection and densification statistics. Outputs (overwritten, any may be NULL):
 * d_mean2d [K*N,2], d_conic [K*N,3], d_depth [K*N], d_opacity [N] (w.r.t. the
 * opacity, not the logit), d_rgb [N,3]. */
GS_API gs_status_t gs_screen_grads(const gs_config_t* cfg, const void* ws, size_t ws_bytes, float* d_mean2d, float* d_conic,
                            float* d_depth, float* d_opacity, float* d_rgb, void* stream);

/* Pose update of render-based tracking (GS-SLAM variants that localise by optimising the
 * camera pose against the rendered map, Sec. II-B). For each of the K views: one Adam step
 * on the se(3) increment xi = (rho, phi) from the pose gradient of gs_project_bwd,
 * xi = -(lr * m_hat / (sqrt(v_hat) + eps)) with lr_rho for rho and lr_phi for phi, then the
 * left update T <- Exp(xi) T (rotation re-orthonormalised). d_cams [K] is updated in place;
 * d_pose_grad [K,6] is read and, if zero_grad != 0, cleared for the next accumulation;
 * d_state [K,16] floats (m[6], v[6], step count, 3 unused) must be zeroed before the first
 * step. Device-only: suitable for capture in a CUDA graph. */
GS_API gs_status_t gs_pose_adam_step(gs_camera_t* d_cams, float* d_pose_grad, float* d_state, int32_t K,
                                     float lr_rho, float lr_phi, float beta1, float beta2, float eps, int32_t zero_grad,
                                     void* stream);

/* ---------------------------------------------------------------- sort primitive */

/* Temporary bytes for gs_sort_pairs on n pairs (host call). */
GS_API gs_status_t gs_sort_pairs_tmp_size(int64_t n, size_t* bytes);

/* Stable LSD radix sort (8-bit digits, one onesweep pass per digit) of n (key, value)
 * pairs on the low key_bits (1..64) bits of the keys, in place. tmp: caller-owned
 * scratch of gs_sort_pairs_tmp_size(n) bytes. n <= 2^30 - 1. */
GS_API gs_status_t gs_sort_pairs(uint64_t* keys, uint32_t* vals, int64_t n, int32_t key_bits, void* tmp, size_t tmp_bytes,
                          uint32_t* d_err_word, void* stream);

/* Diagnostic of the device-side error path (no counterpart in the paper): one 8-bit pass
 * of the pair sort on n >= 7680 pairs with the first onesweep tile withheld, so the next
 * tile's bounded look-back wait (about a second) runs out and sets GS_DEVERR_TIMEOUT in the
 * device word d_err_word. The kernel then finishes normally; keys and vals are left in an
 * unspecified order (all writes in bounds). tmp: gs_sort_pairs_tmp_size(n) bytes. */
GS_API gs_status_t gs_sort_diag_withheld_tile(uint64_t* keys, uint32_t* vals, int64_t n, void* tmp, size_t tmp_bytes,
                                              uint32_t* d_err_word, void* stream);

/* ---------------------------------------------------------------- the mapping loop */

/* Learning rates per parameter group and Adam's constants. */
typedef struct {
  float lr_means, lr_log_scales, lr_quats, lr_opacity, lr_rgb;
  float beta1, beta2, eps;
  int32_t color_width;  /* colour scalars per Gaussian: 3 for GS_COLOR_RGB, 3 (D+1)^2 for SH
                           coefficients of degree D; 0 = 3 */
} gs_adam_t;

/* Floats of the Adam state of N Gaussians whose colour has color_width scalars (0 = 3): m and v
 * (11 + color_width values per Gaussian each, grouped as means [N,3], log-scales [N,3],
 * quaternions [N,4], opacity logits [N], colours [N,color_width]) and the step count. The
 * caller zeroes it before the first step. */
GS_API gs_status_t gs_map_adam_state_size(int64_t N, int32_t color_width, int64_t* floats);

/* One Adam step (Kingma & Ba; bias-corrected) of the mapping optimiser (Sec. II-B: the map is
 * updated from the comparison of rendered images with the key-frames) on the FP32 master arrays
 * of N Gaussians, from the gradients in `grads` (FP32, the five parameter arrays; pose is
 * ignored). The step count lives in the state, so the call can be replayed from a CUDA graph.
 * storage (optional, NULL = none): reduced-storage arrays (its dtype / means_dtype) that receive
 * the updated values rounded to nearest, for the next render; an array equal to its master is
 * skipped. */
GS_API gs_status_t gs_map_adam_step(int64_t N, float* means, float* log_scales, float* quats, float* opacity_logits,
                             float* rgb /* [N, hp->color_width] */, const gs_grads_t* grads, float* state,
                             const gs_adam_t* hp, const gs_gaussians_t* storage, void* stream);

/* Scratch bytes of gs_keyframe_insert for a width x height frame sampled every `stride` pixels. */
GS_API gs_status_t gs_keyframe_tmp_size(int32_t width, int32_t height, int32_t stride, size_t* bytes);

/* New Gaussians from one RGB-D key-frame (the map grows from the key-frames, Sec. II-B; how is
 * not in the paper, so this rule is proposed): every stride-th pixel in x and y whose depth is
 * > near_plane and, when T (the current map's transmittance image, [H,W], may be NULL) is
 * given, whose T is > t_min, becomes one Gaussian: the pixel centre back-projected to its
 * depth through the camera *d_cam (device; world = R^T (p_c - t)), isotropic log-scale ln(scale_factor * stride *
 * depth / ((fx + fy) / 2)), quaternion (1, 0, 0, 0), opacity logit logit0, colour = rgb
 * ([3,H,W]) at the pixel. They are written in row-major pixel order to FP32 arrays at
 * indices [first, first + count), count <= capacity - first (excess pixels are dropped), and
 * count is stored to *d_count (device). tmp: gs_keyframe_tmp_size bytes of device scratch. */
GS_API gs_status_t gs_keyframe_insert(const gs_camera_t* d_cam, const float* rgb, const float* depth, const float* T,
                               int32_t width, int32_t height, int32_t stride, float near_plane, float t_min,
                               float scale_factor, float logit0, float* means, float* log_scales, float* quats,
                               float* opacity_logits, float* colours, int64_t first, int64_t capacity,
                               uint32_t* d_count, void* tmp, size_t tmp_bytes, void* stream);

/* ---------------------------------------------------------------- map-accuracy metrics
 *
 * Sec. IV measures a map by the PSNR and SSIM of its rendered views against the key-frames (and
 * its generation speed by the time a new frame takes to reach its final PSNR / SSIM). The
 * paper gives no formula; these are the standard definitions of the splatting literature:
 *   PSNR of an image = 10 log10(R^2 / MSE) over its C*H*W values (+inf when MSE = 0);
 *   SSIM (Wang et al. 2004) per pixel and channel under an 11 x 11 Gaussian window (sigma 1.5,
 *   taps normalised to sum 1) over zero-padded planes, C1 = (0.01 R)^2, C2 = (0.03 R)^2; an
 *   image's SSIM is the mean of its map.
 * x, y: device FP32 images [images, channels, height, width], contiguous. R = data_range > 0.
 * Results are deterministic (fixed-order reductions). images <= 65535, images * channels <=
 * 65535, height and width <= 65536, else GS_ERR_INVALID_ARG. */

/* Device scratch bytes of gs_psnr / gs_ssim for these dimensions. */
GS_API gs_status_t gs_metrics_tmp_size(int32_t images, int32_t channels, int32_t height, int32_t width, size_t* bytes);

/* psnr: device float [images]. tmp: gs_metrics_tmp_size bytes of device scratch. */
GS_API gs_status_t gs_psnr(const float* x, const float* y, int32_t images, int32_t channels, int32_t height,
                           int32_t width, float data_range, float* psnr, void* tmp, size_t tmp_bytes, void* stream);

/* ssim: device float [images] (mean SSIM); ssim_map: device float [images, channels, height,
 * width] or NULL (not written). tmp: gs_metrics_tmp_size bytes of device scratch. */
GS_API gs_status_t gs_ssim(const float* x, const float* y, int32_t images, int32_t channels, int32_t height,
                           int32_t width, float data_range, float* ssim, float* ssim_map, void* tmp, size_t tmp_bytes,
                           void* stream);

/* ---------------------------------------------------------------- shared map over CUDA IPC
 *
 * Sec. III (Fig. 5) runs the map optimiser and the interactive viewer as two processes on one
 * GPU, each with its own renderer, both reading the Gaussian map where it lives in GPU memory
 * through CUDA IPC. The exporting process shares a device range (e.g. one buffer holding the
 * five Gaussian arrays) and an interprocess event; the importing process maps the range and
 * orders its reads after the exporter's updates with the event.
 *
 * Ordering rule: the exporter records the event on its stream after an update of the map
 * (gs_ipc_event_record); the importer enqueues gs_ipc_stream_wait before a render, which then
 * starts after the last update recorded before that wait was enqueued. The exporter is never
 * held back: an update enqueued after that record may run while the importer reads, so a
 * render can mix two consecutive updates (the paper does not say how its processes
 * synchronise; this is the non-blocking reading). Both processes must use the same GPU. */

typedef struct { uint8_t bytes[128]; } gs_ipc_mem_handle_t;  /* opaque; plain bytes, may be sent
                                                                between processes as is */
typedef struct { uint8_t bytes[64]; } gs_ipc_event_handle_t; /* opaque; plain bytes */

/* Shares bytes [d_ptr, d_ptr + bytes) of a device allocation made with cudaMalloc (d_ptr may
 * point inside it). GS_ERR_INVALID_ARG if the range leaves the allocation; GS_ERR_CUDA if CUDA
 * refuses (e.g. memory from a virtual-memory or managed allocator). The exporter keeps the
 * allocation alive while importers use it. */
GS_API gs_status_t gs_ipc_export(const void* d_ptr, size_t bytes, gs_ipc_mem_handle_t* out);

/* In another process: maps the shared range; *d_ptr receives its address in this process and
 * *bytes (may be NULL) its size. A handle cannot be imported by the process that exported it. */
GS_API gs_status_t gs_ipc_import(const gs_ipc_mem_handle_t* handle, void** d_ptr, size_t* bytes);

/* Unmaps a range from gs_ipc_import (d_ptr as returned by it). */
GS_API gs_status_t gs_ipc_release(void* d_ptr);

/* Creates an interprocess event (cudaEvent_t, timing disabled) in *event and its handle. */
GS_API gs_status_t gs_ipc_event_create(void** event, gs_ipc_event_handle_t* out);

/* In another process: opens the event of a handle; *event is a cudaEvent_t of this process. */
GS_API gs_status_t gs_ipc_event_open(const gs_ipc_event_handle_t* handle, void** event);

/* Records the event on `stream` (exporter: after an update of the map). */
GS_API gs_status_t gs_ipc_event_record(void* event, void* stream);

/* Makes `stream` wait for the event's last record (importer: before a render). */
GS_API gs_status_t gs_ipc_stream_wait(void* stream, void* event);

/* Destroys an event from gs_ipc_event_create or gs_ipc_event_open. */
GS_API gs_status_t gs_ipc_event_destroy(void* event);

/* Largest n accepted by gs_sort_pairs_noalloc. */
#define GS_SORT_NOALLOC_MAX_PAIRS 1048576

/* The paper has no counterpart to this call: it serves callers that cannot allocate.
 *
 * Same result as gs_sort_pairs (stable LSD radix sort of n pairs on the low key_bits
 * bits, in place), but the call needs no temporary buffer from the caller and allocates
 * nothing: its scratch is one fixed device array inside the library, sized for
 * GS_SORT_NOALLOC_MAX_PAIRS pairs (about 14 MB), which every GPU that loads the library
 * keeps until the process exits. It is for code that cannot call cudaMalloc where it
 * sorts, such as a renderer plugin whose buffers belong to a host application, or a
 * real-time loop that cannot take cudaMalloc's device synchronisation and latency.
 *
 * - n > GS_SORT_NOALLOC_MAX_PAIRS returns GS_ERR_SIZE_LIMIT and enqueues nothing.
 * - All calls share the one scratch array: calls whose GPU work overlaps (other streams,
 *   other host threads on the same device) race and must be serialised by the caller.
 * - Every call made outside a stream capture looks up the array's device address
 *   (cudaGetSymbolAddress) with the current device, so a context re-created after
 *   cudaDeviceReset is followed; a call inside a capture reuses the last address looked up on
 *   that device. Make the first call on a device before any stream capture (a call captured
 *   with no earlier call on its device returns GS_ERR_CUDA).
 * - d_err_word (device, may be NULL) receives GS_DEVERR_TIMEOUT if a look-back wait gave up. */
GS_API gs_status_t gs_sort_pairs_noalloc(uint64_t* keys, uint32_t* vals, int64_t n, int32_t key_bits,
                                         uint32_t* d_err_word, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GS_H_ */
