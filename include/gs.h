/*
 * gs.h -- C-ABI of the GB300 (sm_103a) differentiable tile-based 3D Gaussian
 * Splatting mapping step.
 *
 * The method: a map of anisotropic 3D Gaussians (opacity, rotation, location,
 * scale, colour) is rendered with the differentiable tile-based rasteriser of
 * 3DGS and optimised by gradient descent on the photometric loss of Eq. 2
 * (paper Sec. III-B, "Dense Reconstruction"); rendering projects the Gaussians
 * onto the camera plane, sorts them by depth and blends them front to back
 * (paper Sec. II, 3DGS paragraph); the optimiser is the default 3DGS one, Adam
 * (paper Sec. IV-A, "Experimental Setup").  One mapping iteration is
 *
 *   gs_project -> gs_bin_sort -> gs_render_fwd -> gs_loss_l1_ssim
 *              -> gs_render_bwd -> gs_adam_step
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Pointers named *_dev, and every array argument not marked host, are
 *   device memory owned by the caller.  The library allocates nothing, keeps
 *   no pointer across calls and never synchronises, except gs_read_counters.
 * - Every call enqueues asynchronously on `stream` (a cudaStream_t passed as
 *   void*; NULL = the legacy default stream), so a whole iteration can be
 *   captured in one CUDA graph.
 * - Argument errors are reported synchronously (GS_ERR_INVALID, nothing is
 *   enqueued); launch failures as GS_ERR_CUDA.  Errors found on the device
 *   (instance-buffer overflow, non-finite parameters) set bits of a status
 *   word inside the workspace, read with gs_read_counters after the stream
 *   has been synchronised.  There is no CPU fallback.
 * - All arithmetic is FP32, except the projected 2D means, which are carried
 *   as an unevaluated sum of two floats (about 48 significant bits).
 *
 * Map layout (SoA, row-major, float32):
 *   means[n][3], log_scales[n][3], quats[n][4] as (w, x, y, z) (need not be
 *   normalised), opacity_logits[n], sh[K][n][3] with K = (sh_degree+1)^2,
 *   coefficient-major so that each coefficient plane is contiguous.
 * Images: planar [channels][height][width] per view, views packed back to
 *   back in view order (gs_plan_view gives the offsets).  Per-pixel maps
 *   (final_T, last_idx) are [height][width] per view, packed the same way.
 */
#ifndef GS_GB300_H
#define GS_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GS_MAX_VIEWS 64
#define GS_MAX_GROUPS 8
#define GS_PLAN_WORDS 1536

typedef enum {
    GS_OK = 0,
    GS_ERR_INVALID = -1,     /* bad argument; nothing was enqueued */
    GS_ERR_CUDA = -2,        /* a CUDA launch or copy failed */
    GS_ERR_CAPACITY = -3,    /* a capacity given to gs_plan_init is too small */
    GS_ERR_UNSUPPORTED = -4, /* configuration outside what the kernels handle */
    GS_ERR_TIMEOUT = -5      /* reserved: a bounded device wait gave up */
} gs_status;

/* Bits of the device status word (gs_counters.status). */
#define GS_DEV_CAPACITY 1u  /* more (Gaussian, tile) instances than instance_capacity;
                               the surplus was dropped and the render is incomplete */
#define GS_DEV_NONFINITE 2u /* a Gaussian with a non-finite parameter was culled */
#define GS_DEV_SPAN_POOL 4u /* tight rects: the row spans of boxes taller than 16 tile rows
                               did not all fit the plan's span pool; the boxes that missed
                               it kept all their tiles (images and gradients unchanged, the
                               instance lists longer than the geometric set) */

/* One camera.  x_cam = R x_world + t with R row-major (world -> camera), the
 * camera looking along +z with y down; pixel (px, py) is sampled at its
 * integer coordinates in the frame where a camera point projects to
 * (fx x/z + cx, fy y/z + cy).  channels is 3 (RGB) or 1 (the mean of the
 * three composited channels). */
typedef struct {
    float R[9];
    float t[3];
    float fx, fy, cx, cy;
    int32_t width, height, channels, reserved;
} gs_view;

/* The Gaussian map (device pointers, layout above). */
typedef struct {
    const float *means, *log_scales, *quats, *opacity_logits, *sh;
    int32_t n, sh_degree; /* sh_degree in 0..3 */
} gs_map;

/* Gradients, same layouts as gs_map (device pointers). */
typedef struct {
    float *means, *log_scales, *quats, *opacity_logits, *sh;
} gs_map_grad;

/* Rasteriser configuration.  Readings of what the paper leaves open:
 *   tile_w x tile_h in {8x8, 16x16, 32x8} (other powers of two with
 *     tile_w*tile_h in [64, 256] are accepted);
 *   smem_batch: Gaussians staged per shared-memory batch, 32..256, a
 *     multiple of 32;
 *   pixels_per_thread: 0 (automatic) or 1, 2, 4, 8 consecutive pixels of a
 *     tile row handled by one thread; tile_w must be a multiple of it and the
 *     tile must keep at least one full warp of threads;
 *   smem_batch_bwd, pixels_per_thread_bwd: the same two choices for the
 *     backward (gs_render_bwd*); 0 = as for the forward;
 *   near_z: Gaussians whose camera depth is not above near_z are culled
 *     (default reading 0.2 m);
 *   bg: background colour, entering the image as T_final * bg;
 *   density_stats: nonzero makes the pixel adjoint also sum, per (view,
 *     Gaussian), the per-pixel contributions to dL/dmean2d by absolute value
 *     (GS_BUF_ABSGRAD), the statistic of the density control below;
 *   deterministic: nonzero makes the pixel adjoint bit-reproducible (no
 *     paper counterpart): each (Gaussian, tile) pair's partial sums are
 *     stored in its own slot, indexed by the pair's emission position, and
 *     summed per Gaussian in emission order by a second kernel, instead of
 *     float atomics; needs one warp per tile in the backward (tile_w *
 *     tile_h / pixels_per_thread_bwd == 32, GS_ERR_UNSUPPORTED otherwise);
 *   tight_rect: nonzero (recommended) cuts each Gaussian's 3-sigma square
 *     tile rect to the tiles that meet the axis-aligned box of the ellipse
 *     outside which alpha = o exp(power) < 1/255, with the level widened by
 *     1% + 0.01 against FP32 rounding (a Gaussian with o < 0.999/255 gets no
 *     tile), and then each tile row of that box to the tiles whose pixel
 *     rectangle meets the ellipse: the kept tiles are the tiles of the square
 *     rect that meet the widened ellipse, for every box shape (GS_BUF_RECT
 *     keeps the box; GS_BUF_TOUCHED counts the tiles).  The spans of a box of
 *     more than 16 tile rows live in a span pool of the workspace
 *     (GS_DEV_SPAN_POOL if it runs out).  Only (Gaussian, tile) pairs that
 *     every pixel would skip are dropped: images and gradients are
 *     unchanged, the instance lists (and so last_idx) shorter.
 *   recompute: k > 0 makes a recompute (checkpointing) plan: the workspace
 *     holds the projection and binning of at most k views, and nothing of
 *     them is kept from the forward to the backward -- only the images,
 *     final_T and last_idx, which the caller owns.  The views go through it
 *     in passes of k (the last one fewer; gs_plan_view_pass); the backward of
 *     a pass re-runs its gs_project and gs_bin_sort (deterministic: the same
 *     buffers bit for bit) before gs_render_bwd*.  The SSIM maps of
 *     gs_loss_l1_ssim share their bytes with that region, so the loss
 *     overwrites it.  instance_capacity is then the capacity of one pass.
 *     Against a plan holding all V views, the workspace shrinks by about
 *     (V - k) x (200 B per Gaussian + 16 B per instance of a view) plus the
 *     loss maps; k = 4 keeps the projection reading each Gaussian once per
 *     4 views, as in a plan without recompute.
 * The tile shape changes which pixels a Gaussian can reach (its 3-sigma
 * rect is counted in whole tiles), hence the image; the batch sizes, pixels
 * per thread, tight_rect and recompute change only the speed and memory. */
typedef struct {
    int32_t tile_w, tile_h, smem_batch, pixels_per_thread;
    int32_t smem_batch_bwd, pixels_per_thread_bwd;
    float near_z;
    float bg[3];
    int32_t density_stats;
    int32_t deterministic;
    int32_t tight_rect;
    int32_t recompute;
} gs_config;

/* A plan: the sizes, tile grids and workspace layout of one batch of views.
 * Caller-owned plain memory filled by gs_plan_init; opaque otherwise. */
typedef struct {
    uint64_t words[GS_PLAN_WORDS];
} gs_plan;

/* Device-side counters copied back by gs_read_counters. */
typedef struct {
    uint32_t status;           /* GS_DEV_* bits since the last gs_project */
    uint32_t n_instances;      /* (Gaussian, tile) instances binned (<= capacity) */
    uint64_t n_instances_raw;  /* instances requested before clamping to capacity */
    float loss;                /* last value written by gs_loss_l1_ssim */
    uint32_t reserved[3];
} gs_counters;

/* Fills *plan for n_views views (sizes taken from views_host, a HOST array;
 * poses are read later from device copies, so they may change between
 * calls), at most n_capacity Gaussians and instance_capacity (Gaussian,
 * tile) instances.  Returns GS_ERR_INVALID for a bad view size, channel
 * count or count, GS_ERR_UNSUPPORTED for a tile shape or batch outside the
 * supported set. */
gs_status gs_plan_init(gs_plan *plan, const gs_config *cfg, int32_t n_views,
                       const gs_view *views_host, int32_t n_capacity, int64_t instance_capacity);

/* Bytes of device workspace the plan needs (256-byte aligned base). */
size_t gs_plan_workspace_bytes(const gs_plan *plan);

/* Recompute plans (gs_config.recompute = k; the recompute-from-saved-
 * transmittance checkpointing mode, no paper counterpart).
 * gs_plan_passes: the number of passes of a plan, ceil(n_views / k) (1 for a
 * plan without recompute or for a pass; 0 for an invalid plan).
 * gs_plan_view_pass: fills *pass with the plan of pass p, the views
 * [p k, min((p + 1) k, n_views)) of `plan`, sharing its workspace layout.
 * The per-view calls -- gs_project, gs_bin_sort, gs_render_fwd,
 * gs_render_bwd, gs_render_bwd_pixels, gs_project_bwd, gs_densify_stats --
 * take pass plans (a recompute plan with at most k views is its own pass):
 * they read the poses views_dev[p k ...] of the same views_dev array and
 * write the images, final_T, last_idx and dL of those views at their
 * offsets in the packed buffers.  gs_loss_l1_ssim takes the whole plan.
 * Parameter gradients accumulate over passes with accumulate = 1.  The
 * device status word is reset by the gs_project of pass 0 only, so it
 * gathers the bits of all passes; the instance count (gs_read_counters) is
 * that of the last pass.  The calls that need every view at once
 * (gs_project_bwd_groups, gs_project_bwd_adam, gs_visibility) accept a
 * recompute plan only when it has a single pass.  GS_ERR_INVALID if plan is
 * not a recompute plan made by gs_plan_init or p is out of range; pass may
 * be plan itself. */
int32_t gs_plan_passes(const gs_plan *plan);
gs_status gs_plan_view_pass(const gs_plan *plan, int32_t p, gs_plan *pass);

/* Offsets of view v inside packed images (values: channels*H*W units) and
 * per-pixel maps (pixels: H*W units), its first global tile id and grid. */
gs_status gs_plan_view(const gs_plan *plan, int32_t v, int64_t *value_offset,
                       int64_t *pixel_offset, int32_t *tile_offset, int32_t *tiles_x,
                       int32_t *tiles_y);

/* Totals over all views: values (sum C*H*W), pixels (sum H*W), tiles. */
gs_status gs_plan_totals(const gs_plan *plan, int64_t *total_values, int64_t *total_pixels,
                         int32_t *total_tiles);

/* Location of an intermediate buffer inside the workspace, for inspection
 * and testing: id is one of GS_BUF_*; *offset and *bytes in bytes. */
enum {
    GS_BUF_COUNTERS = 0, /* gs_counters-like header (device side) */
    GS_BUF_PROJ = 1,     /* [V*n] x 12 floats: mean hi (2), mean lo (2),
                            conic a,b,c, opacity, r, g, b, depth */
    GS_BUF_RECT = 2,     /* [V*n] x 4 uint16: tile rect x0, y0, x1, y1 (x1, y1 exclusive) */
    GS_BUF_TOUCHED = 3,  /* [V*n] uint32: tiles touched (0 = culled); with tight rects the
                            tiles of the row spans, at most the rect area */
    GS_BUF_RADIUS = 4,   /* [V*n] int32: ceil(3 sqrt(lambda_max)) */
    GS_BUF_DEPTH_ORDER = 5, /* [V*n] uint32: view*n + index of the pairs with a tile,
                               sorted by (depth, view, index), in the first entries
                               (as many as such pairs); the rest unspecified */
    GS_BUF_TILE_KEYS = 6,   /* [instance_capacity] uint32: sorted global tile ids */
    GS_BUF_TILE_VALUES = 7, /* [instance_capacity] uint32: view*n + index per instance */
    GS_BUF_RANGES = 8,      /* [total_tiles] x 2 uint32: [begin, end) of each tile */
    GS_BUF_GRAD2D = 9,      /* [V*n] x 9 floats: dmean2d (2), dconic (3), dopacity,
                               dcolour (3) accumulated by gs_render_bwd */
    GS_BUF_ABSGRAD = 10,    /* [V*n] x 2 floats: sum over pixels of |dL_p/dmean2d| per
                               component (only with density_stats) */
    GS_BUF_COUNT = 16
};
gs_status gs_plan_buffer(const gs_plan *plan, int32_t id, size_t *offset, size_t *bytes);

/* A1: projection (paper Sec. II: each Gaussian mapped onto the image plane;
 * Sec. III-B original 3DGS rasteriser).  For every (view, Gaussian): camera
 * transform, cull at near_z or on non-finite input, 3D covariance from the
 * normalised quaternion and exp(log_scales), EWA 2D covariance with the
 * Jacobian clamped to 1.3x the image extent and a 0.3 px^2 dilation, conic,
 * radius ceil(3 sqrt(lambda_max)), tile rect, SH colour
 * max(0, sum_k Y_k(dir) c_k + 0.5) and opacity sigmoid(logit).
 * views_dev: device array of n_views gs_view (sizes must match the plan).
 * Resets the device status word. */
gs_status gs_project(const gs_plan *plan, const gs_map *map, const gs_view *views_dev, void *ws,
                     void *stream);

/* A2-A4: binning.  Deterministic (tile, depth, index) order: a stable LSD
 * radix sort whose depth digits run once per (view, Gaussian) with a tile
 * (the first pass drops the culled pairs) before the instances are emitted,
 * followed by stable passes over the tile-id digits
 * of the instances; then per-tile [begin, end) ranges.  n = map->n of the
 * preceding gs_project.  The instance count stays on the device (no host
 * synchronisation); overflow sets GS_DEV_CAPACITY. */
gs_status gs_bin_sort(const gs_plan *plan, int32_t n, void *ws, void *stream);

/* A5: forward compositing (paper Sec. II: blending in depth order, front first).
 * Per pixel, front to back over its tile's list: power = -(a dx^2 + c dy^2)/2
 * - b dx dy, skipped when > 0; alpha = min(0.99, o e^power), skipped when
 * < 1/255; the Gaussian that would take T below 1e-4 stops the pixel and is
 * not added.  Writes images (packed planar), final_T and last_idx (one past
 * the list position of the last blended Gaussian, 0 if none).  Of ws it
 * writes only the tile-queue counter of its persistent launch. */
gs_status gs_render_fwd(const gs_plan *plan, void *ws, float *images, float *final_T,
                        int32_t *last_idx, void *stream);

/* A6: photometric loss, Eq. 2 read as
 *   L_v = (1 - lambda) mean|I - I_gt| + lambda (1 - mean SSIM(I, I_gt))
 * (11x11 Gaussian window, sigma 1.5, zero padding, C1 = 0.01^2, C2 = 0.03^2,
 * per channel, means over the C*H*W values of view v), and
 *   L = view_weight * sum_v L_v
 * (view_weight = 1/n_views gives the mean over the plan's views; a loop of
 * single-view plans passes 1/V to reproduce a V-view mean).  Writes L to
 * loss_dev[0] (device float) and dL/dimages (packed like images).  Uses the
 * workspace for the SSIM partial maps.  lambda must lie in [0, 1] and
 * view_weight be positive, else GS_ERR_INVALID. */
gs_status gs_loss_l1_ssim(const gs_plan *plan, const float *images, const float *targets,
                          float lambda, float view_weight, float *loss_dev, float *dL_dimages,
                          void *ws, void *stream);

/* A7-A8: backward.  The pixel adjoint walks each pixel's list back to front
 * from last_idx, recovering T_i = T_{i+1} / (1 - alpha_i) from final_T,
 * reduces each Gaussian's screen-space gradient over a warp with shuffles and
 * adds it atomically; the projection adjoint then maps it to the parameter
 * gradients, summed over views.  accumulate = 0 overwrites grads, 1 adds.
 * Equivalent to gs_render_bwd_pixels followed by gs_project_bwd. */
gs_status gs_render_bwd(const gs_plan *plan, const gs_map *map, const gs_view *views_dev,
                        void *ws, const float *final_T, const int32_t *last_idx,
                        const float *dL_dimages, const gs_map_grad *grads, int32_t accumulate,
                        void *stream);

/* gs_loss_l1_ssim without a workspace, for callers that cannot allocate
 * device memory: code that runs where cudaMalloc is unavailable or forbidden
 * (inside a fixed, pre-reserved memory budget, a host callback, or a real-time
 * thread that must not block on the allocator) and that has no workspace of
 * its own to lend.  The paper has no counterpart to this entry point.
 *
 * Same arguments, arithmetic and results as gs_loss_l1_ssim, minus ws: its
 * scratch (SSIM partial maps, per-block loss partials, the loss) is
 * a fixed array compiled into the library, about 12.6 MB, which every GPU
 * that has loaded the library's device code holds until the process exits.
 * Limits: the plan's images may hold at most 2^20 values in total (sum of
 * C*H*W; e.g. one 640x480 RGB view) and at most 8192 loss tiles of 32x32;
 * larger plans are rejected with GS_ERR_CAPACITY before anything is
 * enqueued.
 *
 * Every call looks up the array's device address on the current device
 * (cudaGetSymbolAddress, a host-side lookup), so no address outlives a device
 * reset.  The first call on each device may load the library's device code
 * and with it reserve the array: make that first call before any stream
 * capture and before the caller's memory budget starts.  Apart from that
 * loading, nothing is allocated, by this call or any library routine it
 * uses.  All calls share the one array and it keeps the last call's contents
 * (every call overwrites what it reads): calls that overlap on
 * the GPU -- on different streams, or from several threads -- race on the
 * scratch and corrupt each other's results; order them on one stream. */
gs_status gs_loss_l1_ssim_noalloc(const gs_plan *plan, const float *images, const float *targets,
                                  float lambda, float view_weight, float *loss_dev,
                                  float *dL_dimages, void *stream);

/* A7 alone: the pixel adjoint of gs_render_bwd, leaving the per-view
 * screen-space gradients (dmean2d, dconic, dopacity, dcolour) in the
 * workspace buffer GS_BUF_GRAD2D (zeroed first). */
gs_status gs_render_bwd_pixels(const gs_plan *plan, void *ws, const float *final_T,
                               const int32_t *last_idx, const float *dL_dimages, void *stream);

/* A8 alone: the projection adjoint of gs_render_bwd, mapping the
 * screen-space gradients in GS_BUF_GRAD2D to parameter gradients summed over
 * the plan's views (accumulate = 0 overwrites grads, 1 adds).  The map and
 * views must be those of the preceding gs_project. */
gs_status gs_project_bwd(const gs_plan *plan, const gs_map *map, const gs_view *views_dev,
                         const void *ws, const gs_map_grad *grads, int32_t accumulate,
                         void *stream);

/* A8 + A9 fused: the projection adjoint of gs_project_bwd followed, in the
 * same kernels, by one Adam step (as gs_adam_step) on every Gaussian, so the
 * parameter gradients are never written to and read back from memory.
 * map: the parameters of the preceding gs_project (read); params: where the
 * updated parameters go (normally the same arrays as map, updated in place);
 * m, v: Adam moments in the gs_map layout; grads_acc (nullable): gradients
 * of other views to add first (a loop of single-view plans passes its
 * accumulated gradients here on its last view); grads_out (nullable): receives
 * the total gradient.  group_lr_host: 6 HOST floats, the learning rates of
 * means, log-scales, quaternions, opacity logits, SH coefficient 0 and SH
 * coefficients 1.. .  *step_dev is incremented first; bias corrections as in
 * gs_adam_step.  Same results, bit for bit, as gs_project_bwd into a zeroed
 * gradient plus gs_adam_step.  Slower than those two calls on a GB300 (one
 * kernel needs the adjoint's registers for both phases, which halves its
 * occupancy: 0.47 ms against 0.12 + 0.27 ms at 1M Gaussians of SH degree 3):
 * for callers that cannot hold a gradient buffer; otherwise use
 * gs_project_bwd_groups and gs_adam_step_groups. */
gs_status gs_project_bwd_adam(const gs_plan *plan, const gs_map *map, const gs_view *views_dev,
                              void *ws, const gs_map_grad *params, const gs_map_grad *m,
                              const gs_map_grad *v, const gs_map_grad *grads_acc,
                              const gs_map_grad *grads_out, const float *group_lr_host,
                              float beta1, float beta2, float eps, int32_t *step_dev,
                              void *stream);

/* A9: Adam (paper Sec. IV-A, default 3DGS optimiser) over one contiguous
 * parameter buffer of n_floats split into n_groups contiguous groups:
 * group g covers [group_offsets_host[g], group_offsets_host[g+1]) with
 * learning rate group_lr_host[g] (HOST arrays of n_groups+1 and n_groups).
 * n_floats must be below 2^31 (GS_ERR_UNSUPPORTED otherwise).
 * *step_dev (device int32) is incremented first, then
 *   m = b1 m + (1-b1) g;  v = b2 v + (1-b2) g^2;
 *   p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps),  t = *step_dev. */
gs_status gs_adam_step(float *params, const float *grads, float *m, float *v, int64_t n_floats,
                       int32_t n_groups, const int64_t *group_offsets_host,
                       const float *group_lr_host, float beta1, float beta2, float eps,
                       int32_t *step_dev, void *stream);

/* A8 + A9 without the known zeros (no paper counterpart; the same results
 * as gs_project_bwd with accumulate = 0 followed by gs_adam_step).  The
 * Gaussians form groups of GS_GRAD_GROUP consecutive indices; a group none
 * of whose Gaussians touches a tile in any view of the last gs_project has
 * an all-zero gradient.
 * gs_project_bwd_groups: the projection adjoint, writing the gradients of the
 * other groups only (those of the zero groups are left as they were) and
 * group_vis[k] = 1 or 0 (device uint8 [ceil(n / GS_GRAD_GROUP)]) for
 * written or not.
 * gs_adam_step_groups: gs_adam_step with the groups, strides and planes of
 * gs_adam_step_sparse, reading the gradient only where group_vis is 1 and
 * taking it as zero elsewhere; the floats after a group's last whole plane
 * (padding, zero) are left as they are, as gs_adam_step leaves them. */
#define GS_GRAD_GROUP 32
gs_status gs_project_bwd_groups(const gs_plan *plan, const gs_map *map, const gs_view *views_dev,
                                const void *ws, const gs_map_grad *grads, uint8_t *group_vis,
                                void *stream);
gs_status gs_adam_step_groups(float *params, const float *grads, float *m, float *v,
                              int64_t n_floats, int32_t n_groups,
                              const int64_t *group_offsets_host, const float *group_lr_host,
                              const int32_t *group_stride_host, int32_t n_gauss,
                              const uint8_t *group_vis, float beta1, float beta2, float eps,
                              int32_t *step_dev, void *stream);

/* Visibility of the last gs_project: vis[i] = 1 (device uint8 [n]) if
 * Gaussian i touches a tile in any view of the plan, else 0. */
gs_status gs_visibility(const gs_plan *plan, int32_t n, const void *ws, uint8_t *vis,
                        void *stream);

/* A9 variant, visibility-masked ("sparse") Adam -- no counterpart in the
 * paper, whose optimiser is the dense 3DGS Adam: the floats of Gaussians
 * with vis[i] == 0 are neither read nor written (their moments do not decay
 * and their parameters do not move); visible ones get exactly the dense
 * update with the shared step t.  Float j of group k (offsets as in
 * gs_adam_step) belongs to Gaussian ((j - off_k) mod (stride_k n_gauss)) /
 * stride_k, with group_stride_host[k] the floats per Gaussian per plane (3
 * for means, log-scales and each SH plane, 4 for quaternions, 1 for
 * opacities; only 1, 3 and 4 are accepted, GS_ERR_UNSUPPORTED otherwise); a
 * group holds whole planes of stride_k n_gauss floats (at most 64 planes in
 * all), and floats after its last whole plane (padding) are skipped.  The
 * four buffers must be 16-byte aligned (GS_ERR_INVALID otherwise). */
gs_status gs_adam_step_sparse(float *params, const float *grads, float *m, float *v,
                              int64_t n_floats, int32_t n_groups,
                              const int64_t *group_offsets_host, const float *group_lr_host,
                              const int32_t *group_stride_host, int32_t n_gauss,
                              const uint8_t *vis, float beta1, float beta2, float eps,
                              int32_t *step_dev, void *stream);

/* ---------------------------------------------------------------------------
 * Adaptive density control (paper Sec. III-B): periodically, Gaussians with a
 * high homodirectional view-space position gradient (the AbsGS criterion) are
 * cloned when small and split in two when large, with the original 3DGS
 * parameters, and Gaussians of low opacity are pruned.
 *
 * Readings: the statistic of a Gaussian is the mean, over the (iteration,
 * view) pairs in which it touches a tile, of |(W/2 h_x, H/2 h_y)|, where
 * (h_x, h_y) sums over pixels the absolute per-pixel contributions to
 * dL/dmean2d (pixel units; W/2, H/2 convert to normalised device
 * coordinates).  Category, in this order: PRUNE if sigmoid(opacity_logit) <
 * min_opacity; CLONE if statistic >= grad_threshold and the largest scale
 * exp(max log_scale) <= percent_dense * extent; SPLIT if statistic >=
 * grad_threshold otherwise; else KEEP.  Output order: kept Gaussians (KEEP
 * and the originals of CLONE) by index, clones by index, then two children
 * per SPLIT by index; child c of Gaussian i: mean + R(q/|q|) (s * xi_ic)
 * with xi = samples[i][c][0..2] (standard normal draws, supplied by the
 * caller), log-scales - log(split_shrink), rotation, opacity and SH copied.
 * Adam moments: kept Gaussians keep theirs, new ones start at zero.
 * ------------------------------------------------------------------------- */
typedef struct {
    float grad_threshold; /* 3DGS-style NDC gradient threshold (0.0004) */
    float percent_dense;  /* clone/split boundary as a fraction of extent (0.01) */
    float min_opacity;    /* prune below (0.005) */
    float split_shrink;   /* children scales divided by this (1.6) */
    float extent;         /* scene extent */
    int32_t reserved[3];
} gs_densify_config;

/* Adds this iteration's statistic: for each (view, Gaussian) of the plan with
 * tiles touched > 0, accum[i] += |(W/2 h_x, H/2 h_y)| and denom[i] += 1
 * (device float arrays of n).  Needs a plan with density_stats and a
 * preceding gs_render_bwd / gs_render_bwd_pixels. */
gs_status gs_densify_stats(const gs_plan *plan, int32_t n, const void *ws, float *accum,
                           float *denom, void *stream);

/* Bytes of device scratch gs_densify_count / gs_densify_apply need for n
 * Gaussians. */
size_t gs_densify_scratch_bytes(int32_t n);

/* Categorises every Gaussian of map and writes counts_dev[0..3] (device int32)
 * = (kept, cloned, split, 0); the new map holds kept + cloned + 2 split
 * Gaussians.  The per-block counts stay in scratch for gs_densify_apply. */
gs_status gs_densify_count(const gs_map *map, const float *accum, const float *denom,
                           const gs_densify_config *cfg, void *scratch, int32_t *counts_dev,
                           void *stream);

/* Writes the new map (dst: n_out Gaussians, SH planes [K][n_out][3]) and its
 * moments (dst_m, dst_v; src_m/src_v the moments of map) from the same
 * inputs given to gs_densify_count and its scratch.  samples: device floats
 * [map->n][2][3].  n_out must equal kept + cloned + 2 split (checked on the
 * device: GS_DEV_CAPACITY is not used; a mismatch writes nothing past
 * n_out and sets counts_dev[3] = 1 if counts_dev is given). counts_dev: [4]. */
gs_status gs_densify_apply(const gs_map *map, const gs_map_grad *src_m, const gs_map_grad *src_v,
                           const float *accum, const float *denom, const float *samples,
                           const gs_densify_config *cfg, const void *scratch, int32_t n_out,
                           gs_map_grad *dst, gs_map_grad *dst_m, gs_map_grad *dst_v,
                           int32_t *counts_dev, void *stream);

/* One level of the Gaussian pyramid of a target (paper Sec. III-B: training
 * starts on smoothed, down-sampled keyframe images and moves to finer
 * levels).  src: [channels][height][width]; dst: [channels][ceil(height/2)]
 * [ceil(width/2)].  Reading: the 5-tap binomial [1, 4, 6, 4, 1]/16 along each
 * axis, mirrored borders without repeating the edge pixel, every second
 * pixel kept from 0; a view of the next level has half its focal lengths
 * and principal point. */
gs_status gs_pyr_down(const float *src, int32_t channels, int32_t height, int32_t width,
                      float *dst, void *stream);

/* ---------------------------------------------------------------------------
 * Point-cloud densification (paper Sec. III-A): tracked pixels are chosen
 * DSO-style (per block the pixel of largest gradient above a threshold,
 * repeated with lower thresholds on larger blocks), and points in flat,
 * untracked regions are added at the mean depth of the vertices of their
 * triangle in the Delaunay triangulation of the tracked pixels.
 * ------------------------------------------------------------------------- */

/* Delaunay triangulation of n distinct points with integer coordinates in
 * [0, 2^20) (HOST arrays: xy_host[n][2]; tri_host[tri_capacity][3] receives
 * counter-clockwise vertex indices).  Exact predicates; on co-circular
 * points one of the valid triangulations.  Synchronous host code (no GPU
 * work).  *n_tri is set to the triangle count (2n - h - 2 for h points on
 * the hull boundary; 0 if all points are collinear or n < 3);
 * GS_ERR_CAPACITY if it exceeds tri_capacity (the first tri_capacity are
 * written), GS_ERR_INVALID for duplicate or out-of-range points. */
gs_status gs_delaunay(const int32_t *xy_host, int32_t n, int32_t *tri_host, int32_t tri_capacity,
                      int32_t *n_tri);

/* DSO-style selection on a [height][width] gray image: grad_sq receives the
 * squared central-difference gradient (zero on the one-pixel border) and
 * selected the pass (k + 1) in which each pixel was chosen, else 0.  Pass k
 * (k < passes <= 8) divides the image into blocks of block * 2^k pixels
 * (partial blocks at the right and bottom edges included); a block without
 * an earlier selection takes its first pixel (raster order) of largest
 * squared gradient if that reaches threshold_sq_host[k] (HOST array). */
gs_status gs_select_pixels(const float *gray, int32_t height, int32_t width, int32_t block,
                           int32_t passes, const float *threshold_sq_host, float *grad_sq,
                           int32_t *selected, void *stream);

/* Mean-depth interpolation on the grid pixels (gx * grid, gy * grid): a
 * pixel not selected and with grad_sq < flat_sq that lies in a triangle of
 * tri[n_tri][3] (counter-clockwise indices into xy[][2] pixel coordinates;
 * closed triangles, the lowest index wins on shared edges) gets the mean of
 * the three vertex depths in out[ceil(height/grid)][ceil(width/grid)],
 * every other grid pixel 0.  owner: int32 scratch of the same size.  All
 * device arrays. */
gs_status gs_interp_depth(const int32_t *tri, int32_t n_tri, const int32_t *xy,
                          const float *depth, const float *grad_sq, const int32_t *selected,
                          int32_t height, int32_t width, int32_t grid, float flat_sq,
                          int32_t *owner, float *out, void *stream);

/* Copies the device counters of the workspace to *out (host) and waits for
 * `stream`. */
gs_status gs_read_counters(const gs_plan *plan, const void *ws, gs_counters *out, void *stream);

/* A static string naming a status. */
const char *gs_status_string(gs_status s);

#ifdef __cplusplus
}
#endif
#endif /* GS_GB300_H */
