/*
 * gsta.h -- C ABI of the GSta training hot path on GB300 (sm_103a).
 *
 * One 3-D Gaussian splatting optimisation step with GSta's gradient-norm
 * freezing ("GSta: Efficient Training Scheme with Siestaed Gaussians for
 * Monocular 3D Scene Reconstruction", arXiv 2504.06716):
 *
 *   gs_project      Sec. 3.1, Eq. 1   EWA projection + SH colour
 *   gs_sort         Sec. 3.1          per-tile depth order ("sorted order")
 *   gs_render_fwd   Sec. 3.1, Eq. 2   front-to-back alpha compositing
 *   gs_loss         Sec. 3.1, Eq. 3   0.8 L1 + 0.2 D-SSIM and dL/dC
 *   gs_render_bwd   Sec. 3.2.4        analytic backward, frozen Gaussians skipped
 *                                     (= gs_raster_bwd then gs_project_bwd)
 *   gs_freeze_update Sec. 3.2.1, Eqs. 4-6  freeze map and active list
 *   gs_adam_masked  Sec. 3.2.4        Adam over the unfrozen Gaussians only
 *   gs_psnr         Sec. 3.2.2, Eq. 7 PSNR for the early-stop check
 *
 * Conventions shared by every call
 * --------------------------------
 * - Pointers named *_dev, and every array argument unless stated otherwise,
 *   are DEVICE pointers owned by the caller. The library allocates nothing
 *   and keeps no pointer after a call returns. Scratch memory is passed in
 *   as a workspace whose size the matching *_workspace_bytes() call gives.
 * - Every call is asynchronous on `stream` (a cudaStream_t; NULL = legacy
 *   default stream). None synchronises the host except gs_get_device_error.
 * - Arguments are validated on the host before any launch; a bad argument
 *   returns GS_ERR_INVALID_ARG and launches nothing. A launch failure
 *   returns GS_ERR_CUDA. Problems found on the device (sort capacity
 *   exceeded, non-finite loss) set bits of a sticky per-device error word,
 *   read and cleared by gs_get_device_error.
 * - Calls on one stream run in order; the library holds no handle, so calls
 *   on different streams are independent as long as their buffers are.
 *
 * Data layout
 * -----------
 * Parameters P: float [n][64], one 256-byte row per Gaussian (AoS):
 *   0-2 mean xyz, 3-5 log scale, 6-9 rotation quaternion (w, x, y, z, not
 *   normalised), 10 opacity logit, 11 + 3c + ch SH coefficient c = 0..15 of
 *   channel ch = 0..2; floats 59-63 are padding and must hold zeros.
 *   Gradients G and the Adam moments m, v have the same layout.
 * Projected splats: float [n][12] (48 bytes per Gaussian):
 *   0 mean_x, 1 mean_y (pixels), 2-4 conic a, b, c (inverse 2-D covariance
 *   [[a, b], [b, c]]), 5 opacity, 6-8 rgb, 9 camera depth, 10 radius (int32
 *   bits; 0 = culled), 11 tiles touched (int32 bits).
 * Images: float [3][H][W]. Raster gradients grad2d: float [n][12]:
 *   0-1 dL/dmean2d, 2-4 dL/dconic (a, b, c), 5 dL/dopacity, 6-8 dL/drgb.
 * Pixel (i, j) is evaluated at coordinates (i, j); tile size 8, 16 or 32.
 */
#ifndef GSTA_H
#define GSTA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GS_OK = 0,
    GS_ERR_INVALID_ARG = 1,  /* host-side validation failed; nothing launched */
    GS_ERR_CUDA = 2,         /* a CUDA launch or copy failed */
    GS_ERR_CAPACITY = 3,     /* device flag: sort entries exceeded the capacity */
    GS_ERR_NONFINITE = 4,    /* device flag: a non-finite loss value */
    GS_ERR_TIMEOUT = 5,      /* device flag: a bounded wait gave up */
    GS_ERR_DEVICE_FLAG = 6   /* gs_get_device_error found flags set */
} gs_status;

/* Device error word bits. */
#define GS_FLAG_CAPACITY 1u
#define GS_FLAG_NONFINITE 2u
#define GS_FLAG_TIMEOUT 4u /* reserved: no kernel of this library waits on another block or a flag */
#define GS_FLAG_BADJOB 8u /* a batch job whose camera differs from the batch's size or tile */

typedef void *gs_stream_t; /* a cudaStream_t */

/* Pinhole camera, passed by host pointer and copied at launch.
 * Camera space is x right, y down, z forward: p_cam = R p_world + t.
 * Readings of the renderer the paper cites (Sec. 3.1, EWA splatting) but does
 * not write out: Gaussians with p_cam.z <= znear are culled; `dilation` is
 * added to both diagonal entries of the 2-D covariance; tan-space
 * coordinates are clamped to 1.3x the half field of view inside the
 * Jacobian; the background colour fills the transmittance left over. */
typedef struct {
    int32_t width, height; /* image size in pixels */
    int32_t tile;          /* tile edge: 8, 16 or 32 */
    int32_t pad0;
    float fx, fy, cx, cy;  /* focal lengths and principal point, pixels */
    float R[9];            /* world -> camera rotation, row-major */
    float t[3];            /* world -> camera translation */
    float campos[3];       /* camera centre, world space (SH view direction) */
    float znear;           /* near cull plane (0.2) */
    float dilation;        /* 2-D covariance dilation (0.3) */
    float bg[3];           /* background colour */
} gs_camera;

/* Sec. 3.1, Eq. 1 and the SH colour of Sec. 3.1. For every Gaussian i < n:
 * projects its mean and covariance (R(q/|q|) diag(exp(2 s)) R^T through the
 * camera Jacobian), inverts the 2-D covariance into a conic, takes
 * radius = ceil(3 sqrt(largest eigenvalue)) and the tiles it touches
 *   x in [floor((mean_x - r)/tile), floor((mean_x + r)/tile)] (same for y,
 *   clipped to the grid; decided in float32),
 * opacity = sigmoid(logit), and colour = max(0, sum_c k_c Y_c(d) + 1/2)
 * over the real SH basis (Condon-Shortley phase) of degree `sh_degree`
 * (0..3) at d = (mean - campos)/|mean - campos|.
 * P [n][64] in, splats [n][12] out (culled Gaussians get radius 0 and
 * tiles 0). n may be 0. Errors: INVALID_ARG (null pointer with n > 0, bad
 * camera or degree), CUDA. */
int gs_project(const float *P, int64_t n, int32_t sh_degree, const gs_camera *cam, float *splats,
               gs_stream_t stream);

/* Opacity activations: sigmoid of the parameter (Sec. 3.1), or its absolute
 * value -- the finetuning stage's activation (Sec. 4.1, a trick taken from
 * Taming 3DGS): opacities may then exceed 1 (alpha is still capped at 0.99),
 * which turns capped Gaussians into opaque ones. */
#define GS_OPACITY_SIGMOID 0
#define GS_OPACITY_ABS 1
/* Flag of the same argument (or-ed in): float 59 of each parameter row is the
 * volume-mask logit m of Sec. 3.3 ("Pruning with Volume Masking"). The hard
 * mask M = 1[sigmoid(m) > 0.01] (m > logit(0.01) = -4.59512 in float32)
 * multiplies opacity and scales: a Gaussian with M = 0 is culled. */
#define GS_VOLUME_MASK 2

/* gs_project with the parameterisation chosen: opacity_act is
 * GS_OPACITY_SIGMOID or GS_OPACITY_ABS, optionally or-ed with GS_VOLUME_MASK;
 * gs_project is this with GS_OPACITY_SIGMOID. Errors as gs_project, and
 * INVALID_ARG for other flag bits. */
int gs_project_ex(const float *P, int64_t n, int32_t sh_degree, int32_t opacity_act, const gs_camera *cam,
                  float *splats, gs_stream_t stream);

/* Workspace of the per-tile depth order (Sec. 3.1, the sort below).
 * Bytes of workspace gs_sort needs for n Gaussians and `capacity` entries
 * on a width x height image with this tile size (0 for invalid sizes). */
size_t gs_sort_workspace_bytes(int64_t n, int64_t capacity, int32_t width, int32_t height, int32_t tile);

/* Sec. 3.1 ("blended in a sorted order"). Lists, for every tile, the
 * Gaussians that tile lists, in ascending order of (float32 camera depth,
 * Gaussian index): a tile of a Gaussian's rectangle lists it only if the box
 * of the tile's pixel centres holds a point where d^T Q d (Q the conic) is
 * at most tau + 1e-3 (1 + tau), tau = 2 ln(255 opacity) -- elsewhere alpha is
 * below 1/255 at every pixel of the tile, so images and gradients are those
 * of the whole rectangle (the tiles count in the splat record is the
 * rectangle's, an upper bound). Decided in float32 with every operation
 * rounded; ln by the atanh series (x = m 2^e, ln m = 2 atanh((m-1)/(m+1))).
 * Out: vals [capacity] (Gaussian index per entry), ranges [tiles][2]
 * (start, end) into vals, (0, 0) for an empty tile, count_dev [1] int64 =
 * total entries P. If P > capacity, entries are dropped (the lists become
 * subsets), ranges are clipped to the capacity, count_dev still holds P,
 * and GS_FLAG_CAPACITY is raised. Workspace: ws of ws_bytes >=
 * gs_sort_workspace_bytes(...), 256-byte aligned. Errors: INVALID_ARG
 * (sizes, tile, workspace too small), CUDA. */
int gs_sort(const float *splats, int64_t n, const gs_camera *cam, void *ws, size_t ws_bytes, int64_t capacity,
            uint32_t *vals, uint32_t *ranges, int64_t *count_dev, gs_stream_t stream);

/* Sec. 3.1, Eq. 2, C = sum_i c_i a_i prod_{j<i}(1 - a_j) per pixel over its
 * tile's list, with a_i = min(0.99, o_i exp(-0.5 d^T Q d)), d = mean - pixel;
 * entries with a positive exponent or a_i < 1/255 are skipped and the ray
 * stops before the entry that would take T below 1e-4; C += T bg.
 * Out: image [3][H][W], t_final [H][W] (T left over), n_last [H][W] (list
 * entries up to and including the last contributor). Errors: INVALID_ARG,
 * CUDA. */
int gs_render_fwd(const float *splats, const uint32_t *vals, const uint32_t *ranges, const gs_camera *cam,
                  float *image, float *t_final, int32_t *n_last, gs_stream_t stream);

/* Launch shape of the two rasteriser kernels (the autotuner's knobs; the
 * results do not depend on it). NULL selects the built-in default for the
 * camera's tile size. */
typedef struct {
    int32_t pixels_per_thread; /* pixels each thread composites: 1, 2, or 4 (tiles of 16 and 32) */
    int32_t batch;             /* splats staged per shared-memory batch: 32, 64, 128 or 256 */
} gs_raster_config;

/* Sec. 3.1, Eq. 2: gs_render_fwd with an explicit launch shape (cfg may be
 * NULL). */
int gs_render_fwd_cfg(const float *splats, const uint32_t *vals, const uint32_t *ranges, const gs_camera *cam,
                      const gs_raster_config *cfg, float *image, float *t_final, int32_t *n_last, gs_stream_t stream);

/* Workspace of the Eq. 3 loss: bytes gs_loss needs for an H x W image. */
size_t gs_loss_workspace_bytes(int32_t H, int32_t W);

/* Sec. 3.1, Eq. 3, L = (1 - lambda) L1 + lambda (1 - SSIM), lambda = 0.2 in
 * the paper. L1 and SSIM are means over the 3 H W values; SSIM per channel
 * with an 11x11 Gaussian window (sigma 1.5), zero padding, C1 = 0.01^2,
 * C2 = 0.03^2; the windows run as separable 1-D passes (the fused SSIM of
 * Sec. 3.3). Out: loss_dev [1] float, dl_dimage [3][H][W] (d|x-y|/dx at
 * x = y taken as 0). A non-finite loss or gradient value raises
 * GS_FLAG_NONFINITE.
 * Errors: INVALID_ARG, CUDA. */
int gs_loss(const float *image, const float *gt, int32_t H, int32_t W, float lambda, void *ws, size_t ws_bytes,
            float *loss_dev, float *dl_dimage, gs_stream_t stream);

/* Sec. 3.2.4, first half: the rasteriser backward. Recomputes each pixel's
 * transmittance back to front from t_final over the same lists and adds,
 * for every Gaussian that is not frozen, dL/d{mean2d, conic, opacity, rgb}
 * into grad2d [n][12]. Frozen Gaussians (frozen[i] != 0; frozen may be NULL)
 * still occlude but receive nothing. grad2d must be zero on entry for
 * every Gaussian in the lists (gs_project_bwd leaves it so).
 * Errors: INVALID_ARG, CUDA. */
int gs_raster_bwd(const float *splats, const uint32_t *vals, const uint32_t *ranges, const gs_camera *cam,
                  const float *t_final, const int32_t *n_last, const float *dl_dimage, const uint8_t *frozen,
                  float *grad2d, gs_stream_t stream);

/* Sec. 3.2.4: gs_raster_bwd with an explicit launch shape (cfg may be
 * NULL). */
int gs_raster_bwd_cfg(const float *splats, const uint32_t *vals, const uint32_t *ranges, const gs_camera *cam,
                      const gs_raster_config *cfg, const float *t_final, const int32_t *n_last,
                      const float *dl_dimage, const uint8_t *frozen, float *grad2d, gs_stream_t stream);

/* Sec. 3.1 and Sec. 3.2.4 with the frozen splats behind a tile's last
 * unfrozen one left out of the backward. A frozen Gaussian takes no
 * gradient (Sec. 3.2.4); the backward visits the splats behind an unfrozen
 * one only to rebuild the transmittance in front of it and the colour
 * blended behind it, so the forward records those: gs_render_fwd_resume is
 * gs_render_fwd_cfg that also writes, for each tile, resume_pos [tiles]
 * (int32) = 1 + the list position of the last splat with frozen[i] == 0 the
 * tile's walk passed (0 if none; frozen may be NULL: nothing frozen), and
 * for each pixel resume [H][W][4] (float, 16-byte aligned) = (T after that
 * splat, the colour blended behind it). gs_raster_bwd_resume is
 * gs_raster_bwd_cfg that starts each tile's walk there from that state,
 * given the buffers of the forward of the same lists and freeze map; its
 * gradients equal gs_raster_bwd_cfg's up to float32 rounding (the state is
 * carried forward instead of recovered backward). resume and resume_pos are
 * both NULL (no record: the plain calls) or both given. Errors: INVALID_ARG
 * (also one of the two NULL, resume misaligned), CUDA. */
int gs_render_fwd_resume(const float *splats, const uint32_t *vals, const uint32_t *ranges, const gs_camera *cam,
                         const gs_raster_config *cfg, const uint8_t *frozen, float *image, float *t_final,
                         int32_t *n_last, float *resume, int32_t *resume_pos, gs_stream_t stream);
int gs_raster_bwd_resume(const float *splats, const uint32_t *vals, const uint32_t *ranges, const gs_camera *cam,
                         const gs_raster_config *cfg, const float *t_final, const int32_t *n_last,
                         const float *dl_dimage, const uint8_t *frozen, const float *resume,
                         const int32_t *resume_pos, float *grad2d, gs_stream_t stream);

/* Several scenes in one launch. The paper trains one scene at a time and
 * has no counterpart; each job computes what gs_render_fwd (Sec. 3.1,
 * Eq. 2) or gs_raster_bwd (Sec. 3.2.4) computes for one view.
 * One rendering job of a batch: a view of one scene (all pointers device,
 * the camera by value). Used by the batch calls below. */
typedef struct {
    const float *splats;     /* [n][12] of the job's scene, projected for this view */
    const uint32_t *vals;    /* the view's sorted lists (gs_sort) */
    const uint32_t *ranges;  /* [tiles][2] */
    float *image;            /* [3][H][W] out (forward) */
    float *t_final;          /* [H][W] out (forward), in (backward) */
    int32_t *n_last;         /* [H][W] out (forward), in (backward) */
    const float *dl_dimage;  /* [3][H][W] in (backward) */
    const uint8_t *frozen;   /* [n] or NULL (backward) */
    float *grad2d;           /* [n][12] accumulated (backward) */
    gs_camera cam;
} gs_raster_job;

/* gs_render_fwd for n_jobs jobs in ONE persistent launch: resident CTAs take
 * (job, tile) items from a device counter (queue_dev, one uint32 of device
 * memory, reset by the call) until all jobs are done, so jobs of uneven cost
 * balance without one launch per job. jobs_dev is a DEVICE array; every job
 * must have this width, height and tile (a job that does not is skipped and
 * raises GS_FLAG_BADJOB). Results equal gs_render_fwd per job. The grid is
 * the number of CTAs that fit on the device at once. Errors: INVALID_ARG,
 * CUDA. */
int gs_render_fwd_batch(const gs_raster_job *jobs_dev, int32_t n_jobs, int32_t width, int32_t height, int32_t tile,
                        const gs_raster_config *cfg, uint32_t *queue_dev, gs_stream_t stream);

/* Sec. 3.2.4 per job: gs_raster_bwd for n_jobs jobs in one persistent launch, as above. Jobs of
 * one scene may share grad2d (their terms add up). */
int gs_raster_bwd_batch(const gs_raster_job *jobs_dev, int32_t n_jobs, int32_t width, int32_t height, int32_t tile,
                        const gs_raster_config *cfg, uint32_t *queue_dev, gs_stream_t stream);

/* Sec. 3.2.4, second half, and the statistics of Sec. 3.2.1: chain rule from
 * grad2d to the 59 parameters for the Gaussians act[0 .. *n_active_dev).
 * Writes full rows of G [n][64] for those Gaussians (zeros if culled in this
 * view), zeroes their grad2d rows, and for each visible one adds
 *   acc_xyz += |dL/dmean2d| in normalised device units (x W/2, y H/2),
 *   acc_rgb += |dL/d k_0| over the three channels, cnt += 1.
 * Rows of G for other Gaussians are not touched. acc_xyz, acc_rgb, cnt may
 * be NULL together. Errors: INVALID_ARG, CUDA. */
int gs_project_bwd(const float *P, int64_t n, int32_t sh_degree, const gs_camera *cam, const float *splats,
                   const int32_t *act, const int32_t *n_active_dev, float *grad2d, float *G, float *acc_xyz,
                   float *acc_rgb, int32_t *cnt, gs_stream_t stream);

/* Sec. 3.2.4: gs_project_bwd that ADDS its gradient rows into G instead of writing them
 * (several views of one scene in one optimiser step: call gs_project_bwd for
 * the first view, this for the others). */
int gs_project_bwd_accum(const float *P, int64_t n, int32_t sh_degree, const gs_camera *cam, const float *splats,
                         const int32_t *act, const int32_t *n_active_dev, float *grad2d, float *G, float *acc_xyz,
                         float *acc_rgb, int32_t *cnt, gs_stream_t stream);

/* One window of gradient statistics (as gs_project_bwd keeps them): acc_xyz,
 * acc_rgb float [n], cnt int32 [n]; max_radius int32 [n] or NULL -- the
 * largest screen radius (px) of the Gaussian in the views counted. */
typedef struct {
    float *acc_xyz;
    float *acc_rgb;
    int32_t *cnt;
    int32_t *max_radius;
} gs_grad_stats;

/* gs_project_bwd (accumulate = 0) or gs_project_bwd_accum (accumulate != 0)
 * that updates n_sets (0..2) statistics windows at once -- the freeze window
 * of Sec. 3.2.1 and the densification window of Sec. 4.1 have different
 * lengths. sets: host array of n_sets. Errors: INVALID_ARG, CUDA. */
int gs_project_bwd_stats(const float *P, int64_t n, int32_t sh_degree, const gs_camera *cam, const float *splats,
                         const int32_t *act, const int32_t *n_active_dev, float *grad2d, float *G, int32_t accumulate,
                         const gs_grad_stats *sets, int32_t n_sets, gs_stream_t stream);

/* Sec. 3.2.4 under the activations of Sec. 4.1 (absolute-value opacity) and
 * Sec. 3.3 (volume mask): gs_project_bwd_stats for the parameterisation `opacity_act` (as in
 * gs_project_ex): dL/dx = dL/dopacity * sigmoid'(x), or * sign(x) (0 at
 * x = 0) under GS_OPACITY_ABS. Under GS_VOLUME_MASK the mask logit's
 * gradient, G[i][59], is the straight-through one, (dL/dM + mask_loss) *
 * sigmoid'(m) with dL/dM = dL/dopacity * opacity + sum_b dL/dlog s_b for a
 * visible Gaussian (0 otherwise), where mask_loss >= 0 is the derivative of
 * the mask term lambda_m mean_i sigmoid(m_i) of the loss with respect to one
 * sigmoid(m_i) (lambda_m / N); it reaches every Gaussian of the active list.
 * The other entry points take the sigmoid and no mask. */
int gs_project_bwd_ex(const float *P, int64_t n, int32_t sh_degree, int32_t opacity_act, float mask_loss,
                      const gs_camera *cam, const float *splats, const int32_t *act, const int32_t *n_active_dev,
                      float *grad2d, float *G, int32_t accumulate, const gs_grad_stats *sets, int32_t n_sets,
                      gs_stream_t stream);

/* Sec. 3.2.4, the backward of Algorithm 1's rasterisation step:
 * gs_raster_bwd followed by gs_project_bwd on the same stream. */
int gs_render_bwd(const float *P, int64_t n, int32_t sh_degree, const gs_camera *cam, const float *splats,
                  const uint32_t *vals, const uint32_t *ranges, const float *t_final, const int32_t *n_last,
                  const float *dl_dimage, const uint8_t *frozen, const int32_t *act, const int32_t *n_active_dev,
                  float *grad2d, float *G, float *acc_xyz, float *acc_rgb, int32_t *cnt, gs_stream_t stream);

/* One iteration of Algorithm 1's inner body for one view, in one call:
 * gs_project_ex, gs_sort, gs_render_fwd_resume, gs_loss, gs_raster_bwd_resume,
 * gs_project_bwd_ex (statistics windows `stats`), gs_adam_masked -- the
 * same kernels, enqueued from native code instead of one binding call
 * each. Everything the step touches is described by gs_step (device
 * pointers, sizes, launch shapes); the view's camera, its target image gt
 * [3][H][W] (device), the group learning rates lr (host, [n_lr]) and the
 * Adam step (>= 1) are the per-iteration arguments. Returns the first
 * non-OK status of the sequence (nothing after it is enqueued). */
typedef struct {
    /* Gaussians: P, G, m, v [n][64]; splats, grad2d [n][12] */
    float *P, *G, *m, *v, *splats, *grad2d;
    int64_t n;
    int32_t sh_degree;
    int32_t opacity_act;              /* GS_OPACITY_*, optionally | GS_VOLUME_MASK */
    float mask_loss;                  /* volume mask: lambda_m / N (see gs_project_bwd_ex) */
    int32_t n_lr;                     /* learning-rate groups in lr: 6, or 7 (the mask logit); 0 reads as 6 */
    const uint8_t *frozen;            /* [n] or NULL */
    const int32_t *act;               /* unfrozen list [n], its length in n_active_dev [1] */
    const int32_t *n_active_dev;
    gs_grad_stats stats[2];           /* statistics windows of the projection backward */
    int32_t n_stats;                  /* 0..2 */
    /* the view's buffers: sort workspace and lists, image, loss */
    void *sort_ws;
    size_t sort_ws_bytes;
    int64_t capacity;
    uint32_t *vals, *ranges;
    int64_t *count_dev;
    float *image, *t_final;
    int32_t *n_last;
    float *dl_dimage;
    void *loss_ws;
    size_t loss_ws_bytes;
    float *loss_dev;
    float lambda_ssim;                /* 0.2 */
    /* rasteriser launch shapes; pixels_per_thread 0 takes the default */
    gs_raster_config fwd, bwd;
    float b1, b2, eps;                /* Adam */
    /* optional cudaEvent_t pair (NULL: none) recorded on the stream just
     * before and just after the rasteriser backward, to time it in place */
    void *bwd_events[2];
    /* optional: the view's resume record ([H][W][4] float, [tiles] int32,
     * see gs_render_fwd_resume); both NULL runs the plain rasteriser calls */
    float *resume;
    int32_t *resume_pos;
} gs_step;

int gs_train_step(const gs_step *s, const gs_camera *cam, const float *gt, const float *lr, int64_t step,
                  gs_stream_t stream);

/* Progressive training and blur (Sec. 3.3, "Progressive Training", "Blur";
 * Sec. 4.1: resolution from scale 0.175 to 1 and a decaying blur until
 * iteration 6K). gs_resize_area: src [C][H][W] -> dst [C][H2][W2], the area
 * average over the same extent of the image plane -- with pixel j spanning
 * [j - 1/2, j + 1/2), target pixel i covers source [i W / W2 - 1/2,
 * (i + 1) W / W2 - 1/2) (same in y), each source pixel weighted by its
 * overlap; the matching camera has fx' = fx W2 / W and cx' = (cx + 1/2) W2 /
 * W - 1/2. gs_blur: dst = src convolved with a 5 x 5 Gaussian of standard
 * deviation sigma (pixels), its weights renormalised over the taps inside
 * the image; a plain copy when sigma < GS_BLUR_SIGMA_MIN. Device pointers,
 * dst distinct from src. Errors: INVALID_ARG, CUDA. */
#define GS_BLUR_SIGMA_MIN 0.1f
int gs_resize_area(const float *src, int32_t C, int32_t W, int32_t H, float *dst, int32_t W2, int32_t H2,
                   gs_stream_t stream);
int gs_blur(const float *src, int32_t C, int32_t W, int32_t H, float sigma, float *dst, gs_stream_t stream);

/* Significance pruning (Sec. 3.3, "Pruning with Significance of Gaussians",
 * after LightGaussian; Sec. 4.1: at 4K and 7K). gs_hit_counts ADDS to hits_dev
 * [n] (uint32), for every pixel of this view, 1 to each Gaussian the pixel
 * blends (the forward's own decisions up to n_last). gs_significance_mark
 * scores score_i = hits_i * o_i * (V_i / V_q)^beta with V_i = exp(s_0 + s_1 +
 * s_2) (float32) and V_q the volume of rank floor(quantile n) - 1 in
 * ascending (volume, index) order, o the opacity under opacity_act, and sets
 * mark [n] to 1 for the floor(fraction n) Gaussians of lowest (score, index),
 * 0 elsewhere (gs_densify_plan's prune_mark). Workspace:
 * gs_significance_workspace_bytes(n), 256-byte aligned. Errors: INVALID_ARG,
 * CUDA. */
int gs_hit_counts(const float *splats, const uint32_t *vals, const uint32_t *ranges, const gs_camera *cam,
                  const int32_t *n_last, uint32_t *hits_dev, gs_stream_t stream);
size_t gs_significance_workspace_bytes(int64_t n);
int gs_significance_mark(int64_t n, const float *P, const uint32_t *hits, int32_t opacity_act, float beta,
                         float quantile, float fraction, uint8_t *mark, void *ws, size_t ws_bytes, gs_stream_t stream);

/* Workspace of the Sec. 3.2.1 freeze update: bytes gs_freeze_update needs
 * for n Gaussians. */
size_t gs_freeze_workspace_bytes(int64_t n);

/* Sec. 3.2.1, Eqs. 4-6, with the cadence of Sec. 4.1. mode:
 *   0 update: frozen[i] |= cnt[i] > 0 && acc_xyz[i]/cnt[i] < eps_xyz
 *                                     && acc_rgb[i]/cnt[i] < eps_rgb
 *             (float32 division and strict comparisons; the map only grows);
 *   1 reset : frozen[i] = 0 for all i;
 *   2 clear : the map is kept;
 *   3 list  : the map and the statistics are kept (for a set the
 *             densification rearranged; gs_freeze_update_noalloc takes 0-2).
 * Modes 0-2 zero acc_xyz, acc_rgb, cnt; every mode writes the unfrozen
 * indices in ascending order to act [n] and their number to n_active_dev [1].
 * Errors: INVALID_ARG (mode, sizes, workspace), CUDA. */
int gs_freeze_update(int64_t n, float *acc_xyz, float *acc_rgb, int32_t *cnt, uint8_t *frozen, float eps_xyz,
                     float eps_rgb, int32_t mode, int32_t *act, int32_t *n_active_dev, void *ws, size_t ws_bytes,
                     gs_stream_t stream);

/* Freeze strategies of the ablation (Sec. 5, "Freezing strategies" and
 * "Gradient information"; Table 3). A Gaussian is eligible when it is not
 * frozen and cnt[i] > 0; with avg_x = acc_xyz[i]/cnt[i] and avg_r =
 * acc_rgb[i]/cnt[i] (float32 division), an update freezes the eligible
 *   GS_FREEZE_RULE    with avg_x < eps_xyz && avg_r < eps_rgb (Eq. 4: the
 *                     same decision as gs_freeze_update mode 0),
 *   GS_FREEZE_XYZ     with avg_x < eps_xyz (positional gradients only),
 *   GS_FREEZE_RANDOM  with u[i] < fraction (u [n]: the caller's uniform
 *                     draws in [0, 1); each eligible Gaussian is frozen with
 *                     probability `fraction`),
 *   GS_FREEZE_MINGRAD the k = floor(fraction * m) of the m eligible with the
 *                     smallest (score, index), score = max(avg_x / eps_xyz,
 *                     avg_r / eps_rgb) in float32 (the rule's own measure,
 *                     with a rank cut instead of the thresholds; NaN orders
 *                     last), k computed in double.
 * Then, as mode 0 of gs_freeze_update: the map only grows, acc_xyz,
 * acc_rgb, cnt are zeroed, act / n_active_dev rebuilt. fraction in [0, 1]
 * for RANDOM and MINGRAD; eps > 0 for MINGRAD; u may be NULL except for
 * RANDOM. Workspace: ws of ws_bytes >= gs_freeze_select_workspace_bytes(n),
 * 256-byte aligned. Errors: INVALID_ARG, CUDA. */
#define GS_FREEZE_RULE 0
#define GS_FREEZE_XYZ 1
#define GS_FREEZE_RANDOM 2
#define GS_FREEZE_MINGRAD 3
size_t gs_freeze_select_workspace_bytes(int64_t n);
int gs_freeze_select(int64_t n, float *acc_xyz, float *acc_rgb, int32_t *cnt, uint8_t *frozen, float eps_xyz,
                     float eps_rgb, int32_t strategy, float fraction, const float *u, int32_t *act,
                     int32_t *n_active_dev, void *ws, size_t ws_bytes, gs_stream_t stream);

/* gs_freeze_update without a workspace argument. The paper has no
 * counterpart: this exists for callers that cannot allocate device memory
 * where they make the call -- for example a host that owns every device
 * buffer and hands this library only the inputs and outputs, or a loop that
 * must not call cudaMalloc because an allocation can synchronise the whole
 * device. Its scratch (one count per 1024 Gaussians) is a fixed 256 KB array
 * inside the library that every GPU which loads the library keeps until the
 * process exits; it allows n <= 67,108,864 and returns GS_ERR_INVALID_ARG for
 * more. The first call on a device, made with that device current, looks up
 * the array's device address (cudaGetSymbolAddress) and keeps it for that
 * device's context; after a device reset (a new context) the next call looks
 * it up again. Make the first call on a device, and the first after a reset,
 * before any stream capture. All calls share the one array: each call writes
 * every entry it reads before reading it, so nothing has to be cleared
 * between calls, but calls whose executions overlap on the GPU (other
 * streams, other host threads) race on it and must be ordered by the caller.
 * Allocates nothing (no cudaMalloc, no library allocator). Arguments,
 * results and errors are those of gs_freeze_update; GS_ERR_CUDA also if the
 * address lookup fails. */
int gs_freeze_update_noalloc(int64_t n, float *acc_xyz, float *acc_rgb, int32_t *cnt, uint8_t *frozen,
                             float eps_xyz, float eps_rgb, int32_t mode, int32_t *act, int32_t *n_active_dev,
                             gs_stream_t stream);

/* Sec. 3.2.4 (the optimiser only updates Gaussians that are not frozen).
 * Adam at global step `step` >= 1 for the rows act[0 .. *n_active_dev) of
 * P, with gradient G and moments m, v (all [n][64]):
 *   m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
 *   p -= lr_group * (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps).
 * lr is a HOST array of 6 group rates: xyz (floats 0-2), scale (3-5),
 * rotation (6-9), opacity (10), SH DC (11-13), SH rest (14-58). Other rows
 * are not read or written. Errors: INVALID_ARG, CUDA. */
int gs_adam_masked(float *P, const float *G, float *m, float *v, int64_t n, const int32_t *act,
                   const int32_t *n_active_dev, const float *lr, float b1, float b2, float eps, int64_t step,
                   gs_stream_t stream);

/* Sec. 3.2.4 with the volume masks of Sec. 3.3: gs_adam_masked with
 * n_groups (6 or 7) learning rates: a seventh, lr[6], is the rate of
 * float 59, the volume-mask logit (0 with six). */
int gs_adam_masked_groups(float *P, const float *G, float *m, float *v, int64_t n, const int32_t *act,
                          const int32_t *n_active_dev, const float *lr, int32_t n_groups, float b1, float b2,
                          float eps, int64_t step, gs_stream_t stream);

/* ---------------------------------------------------------------------
 * Learned freeze predictor. The paper has no learned component: these
 * calls build a small network that proposes Gaussians the gradient-norm
 * rule (Sec. 3.2.1, Eqs. 4-6) is about to freeze, so they can be frozen
 * earlier; the rule stays in force and judges the proposals.
 * --------------------------------------------------------------------- */
#define GS_MLP_IN 16
#define GS_MLP_HIDDEN 64
#define GS_MLP_PARAMS 5313 /* W1[16][64] b1[64] W2[64][64] b2[64] W3[64] b3 */
#define GS_MLP_WEIGHTS 5184 /* bf16 copies of W1, W2, W3 */

/* Statistics boundary update of the predictor state state[n][12] (float32):
 * 0-3 xyz-norm EMA history (newest first), 4-7 rgb history, 8 xyz EMA,
 * 9 rgb EMA, 10 visible iterations, 11 boundaries spent frozen. For each
 * Gaussian with cnt > 0: EMA = 0.5 EMA + 0.5 acc/cnt, views += cnt; frozen
 * count += frozen[i] (frozen may be NULL); the histories shift and take the
 * EMA at the front. Call before gs_freeze_update clears the statistics.
 * Errors: INVALID_ARG, CUDA. */
int gs_pred_history(int64_t n, const float *acc_xyz, const float *acc_rgb, const int32_t *cnt, const uint8_t *frozen,
                    float *state, gs_stream_t stream);

/* The 16 predictor features of every Gaussian, as bfloat16 X[n][16]:
 * 0-3 and 4-7 log10(history / eps_xyz | eps_rgb) clamped to [-8, 8] (norms
 * floored at 1e-30), 8 sigmoid(opacity logit), 9 largest and 10 smallest
 * log-scale, 11 ln(1 + visible iterations), 12 k / K, 13-14 log10 of the
 * current window's average norms over the thresholds (0 if never visible),
 * 15 min(boundaries spent frozen, 8) / 8. P [n][64], state [n][12].
 * Errors: INVALID_ARG, CUDA. */
int gs_pred_features(int64_t n, const float *P, const float *acc_xyz, const float *acc_rgb, const int32_t *cnt,
                     const float *state, int32_t k, int32_t K, float eps_xyz, float eps_rgb, uint16_t *X,
                     gs_stream_t stream);

/* Inference p[i] = sigmoid(relu(relu(X W1 + b1) W2 + b2) . W3 + b3) on the
 * tensor cores (bf16 inputs X[n][16] and weights wb[5184], the first hidden
 * layer rounded to bf16, float32 accumulation; biases from params[5313]).
 * Errors: INVALID_ARG, CUDA. */
int gs_mlp_fwd(int64_t n, const uint16_t *X, const uint16_t *wb, const float *params, float *p, gs_stream_t stream);

/* Gradient of the weighted binary cross-entropy
 *   L = inv_wsum * sum_i w_i (softplus(z_i) - y_i z_i)   (w NULL: all 1)
 * over the 5313 parameters, ADDED into grad[5313] (zero it first); the loss
 * is added into *loss_dev if loss_dev is not NULL. The forward is the
 * inference above computed in float32; gradients pass through the bf16
 * roundings as the identity. Errors: INVALID_ARG, CUDA. */
int gs_mlp_grad(int64_t n, const uint16_t *X, const float *y, const float *w, float inv_wsum, const uint16_t *wb,
                const float *params, float *grad, float *loss_dev, gs_stream_t stream);

/* Adam step on the float32 parameters (bias-corrected at `step` >= 1) that
 * also refreshes the bf16 weight copies wb. Errors: INVALID_ARG, CUDA. */
int gs_mlp_adam(float *params, const float *grad, float *m, float *v, uint16_t *wb, float lr, float b1, float b2,
                float eps, int64_t step, gs_stream_t stream);

/* wb = bf16(W1, W2, W3) of params. Errors: INVALID_ARG, CUDA. */
int gs_mlp_refresh(const float *params, uint16_t *wb, gs_stream_t stream);

/* Freezes every Gaussian with prob[i] > tau (the map only grows; the
 * statistics are not touched) and rebuilds act / n_active_dev as
 * gs_freeze_update does. Workspace as gs_freeze_workspace_bytes(n).
 * Errors: INVALID_ARG, CUDA. */
int gs_freeze_apply(int64_t n, const float *prob, float tau, uint8_t *frozen, int32_t *act, int32_t *n_active_dev,
                    void *ws, size_t ws_bytes, gs_stream_t stream);

/* Sec. 3.2.4 for graph replay (the paper has no counterpart of the device-side
 * step): gs_adam_masked with the step counter and the six group learning rates in
 * device memory: *step_dev is advanced by one and the bias correction taken
 * at the new value, and the rates are read from lr_dev [6] (same order as
 * gs_adam_masked's lr) when the kernel runs, so a captured CUDA graph can
 * replay the update step after step while the host changes the rates
 * between replays. scratch_dev: two floats of device memory.
 * Errors: INVALID_ARG, CUDA. */
int gs_adam_masked_devstep(float *P, const float *G, float *m, float *v, int64_t n, const int32_t *act,
                           const int32_t *n_active_dev, const float *lr_dev, float b1, float b2, float eps,
                           int64_t *step_dev, float *scratch_dev, gs_stream_t stream);

/* Measurement support (the paper has no counterpart): classifies the
 * (pixel, splat) pairs of every pixel's tile list with the forward's own
 * decisions, up to its last contributor (n_last, as left by gs_render_fwd)
 * or, if that is less, 1 + the tile's last unfrozen entry among the first
 * max(n_last over the tile) -- the pairs gs_raster_bwd_resume walks, or a
 * lower bound of them; with frozen NULL, every pair up to the last
 * contributor (gs_raster_bwd's walk) -- and ADDS the counts to counts_dev
 * [3] (uint64, device): [0] blended by an unfrozen splat, [1] blended by a
 * frozen splat, [2] skipped (positive exponent or alpha < 1/255). A
 * benchmark weighs them by their arithmetic to state the backward's
 * algorithmic work. Errors: INVALID_ARG, CUDA. */
int gs_raster_pair_counts(const float *splats, const uint32_t *vals, const uint32_t *ranges, const gs_camera *cam,
                          const int32_t *n_last, const uint8_t *frozen, uint64_t *counts_dev, gs_stream_t stream);

/* ---------------------------------------------------------------------
 * Adaptive densification and pruning (Sec. 4.1: thresholds and cadence;
 * the clone / split / prune rules are those of 3DGS, which the paper builds
 * on) and opacity reset. Thresholds at the current iteration, compared in
 * float32; sizes and opacities in the log / logit domain.
 * --------------------------------------------------------------------- */
typedef struct {
    float eps_xyz;           /* average |dL/dmean2d| (NDC) threshold */
    float eps_rgb;           /* average |dL/dk0| threshold */
    int32_t use_rgb;         /* the diffuse-colour criterion on this step */
    float log_clone_max;     /* log(0.01 extent): largest log-scale that clones */
    float logit_min_opacity; /* logit(0.005): below it, pruned */
    int32_t prune_big;       /* screen / world size pruning active */
    int32_t max_screen_radius; /* px (20): larger originals are pruned */
    float log_max_world;     /* log(0.1 extent): larger Gaussians are pruned */
    float log_split_div;     /* log(1.6): children's log-scales are this much smaller */
    int32_t mask_prune;      /* also prune Gaussians whose volume mask is off ... */
    float mask_logit_min;    /* ... mask logit (float 59) <= this (logit(0.01)) */
    const uint8_t *prune_mark; /* device [n] or NULL: also prune where nonzero (significance) */
} gs_densify_params;

/* Bytes of workspace the densification of n Gaussians needs. */
size_t gs_densify_workspace_bytes(int64_t n);

/* Decides, for each of the n Gaussians (P [n][64], the densification
 * window's statistics: average = acc / cnt over cnt > 0, max_radius may be
 * NULL), candidate = average xyz >= eps_xyz (or, with use_rgb, average rgb
 * >= eps_rgb); clone if its largest log-scale <= log_clone_max, else split;
 * prune when logit < logit_min_opacity, or (mask_prune) the volume-mask
 * logit P[i][59] <= mask_logit_min, or prune_mark[i] != 0, or (prune_big)
 * largest screen radius
 * > max_screen_radius (originals only) or largest log-scale > log_max_world
 * (a child's log-scale is smaller by log_split_div). Writes counts_dev [4]
 * (int64, device): surviving originals, surviving clones, surviving children
 * (two per split original whose children survive), split originals (the
 * number of z draws gs_densify_apply needs). Keeps the decisions in ws for
 * gs_densify_apply. Errors: INVALID_ARG, CUDA. */
int gs_densify_plan(int64_t n, const float *P, const gs_grad_stats *stats, const gs_densify_params *prm, void *ws,
                    size_t ws_bytes, int64_t *counts_dev, gs_stream_t stream);

/* Further per-Gaussian state gs_densify_apply moves with the Gaussians:
 * rows of row_bytes (a multiple of 4) from src [n] to dst [capacity]; copied
 * for survivors, zero for new Gaussians (device pointers, 4-byte aligned). */
typedef struct {
    const void *src;
    void *dst;
    int32_t row_bytes;
} gs_densify_carry;

/* Writes the densified set planned in ws: rows of P_out / m_out / v_out
 * [capacity][64], frozen_out [capacity] and of each carried array (carry:
 * host array of n_carry <= 8, may be NULL with 0): the
 * surviving originals in index order (all state copied), then the surviving
 * clones (exact copies of P), then the surviving children, two per split
 * original in its order: mean + R(q/|q|)(exp(log_s) * z_k) with z [splits][2][3]
 * (device, N(0, 1) draws of the split originals in index order, child 0
 * first), log-scales minus log_split_div, the rest of P copied. New rows have
 * zero m, v and carried state and are not frozen. Writes nothing if the
 * total exceeds `capacity`. The output buffers must not overlap the inputs.
 * Errors: INVALID_ARG, CUDA. */
int gs_densify_apply(int64_t n, const float *P, const float *m, const float *v, const uint8_t *frozen,
                     const gs_densify_carry *carry, int32_t n_carry, const gs_densify_params *prm, const float *z,
                     const void *ws, size_t ws_bytes, int64_t capacity, float *P_out, float *m_out, float *v_out,
                     uint8_t *frozen_out, gs_stream_t stream);

/* 3DGS opacity reset: P[i][10] = min(P[i][10], logit_cap) (logit_cap =
 * logit(0.01)) and the opacity's Adam moments m, v [i][10] set to 0, for
 * every Gaussian i < n that is not frozen (frozen [n] may be NULL: all of
 * them, as 3DGS resets; passing the freeze map leaves frozen Gaussians as
 * they are, like every other parameter update). Errors: INVALID_ARG, CUDA. */
int gs_opacity_reset(int64_t n, float *P, float *m, float *v, float logit_cap, const uint8_t *frozen,
                     gs_stream_t stream);

/* Entry into the absolute-value opacity (Sec. 4.1, finetuning stage): for
 * all i < n, P[i][10] = o = sigmoid(P[i][10]) -- the same expression, in
 * float32, that gs_project evaluates, so |new parameter| is bit for bit the
 * opacity rendered before. The opacity's Adam moments m, v [i][10]:
 * GS_MOMENTS_ZERO restarts them; GS_MOMENTS_RESCALE carries them over to the
 * new parameterisation, whose gradient is the old one over s = o (1 - o):
 * m /= s, v /= s^2 (s floored at 1e-12). slope_sum_dev (device, one float,
 * or NULL): the sum of s over the n Gaussians is ADDED to it (float atomics,
 * summation order unspecified) -- s is how far an Adam step of the logit
 * moved the opacity, for a caller that keeps that step size under |x|.
 * Errors: INVALID_ARG, CUDA. */
#define GS_MOMENTS_ZERO 0
#define GS_MOMENTS_RESCALE 1
int gs_opacity_to_abs(int64_t n, float *P, float *m, float *v, int32_t moments, float *slope_sum_dev,
                      gs_stream_t stream);

/* Workspace of the Eq. 7 PSNR: bytes gs_psnr needs for S images of H x W. */
size_t gs_psnr_workspace_bytes(int32_t S, int32_t H, int32_t W);

/* Sec. 3.2.2, Eq. 7 input: psnr[s] = 10 log10(1 / MSE) of clamp(image, 0, 1)
 * against gt over the 3 H W values of image s (MSE floored at 1e-10).
 * images, gts [S][3][H][W]; psnr_dev [S] float. Errors: INVALID_ARG, CUDA. */
int gs_psnr(const float *images, const float *gts, int32_t S, int32_t H, int32_t W, void *ws, size_t ws_bytes,
            float *psnr_dev, gs_stream_t stream);

/* Library plumbing below (errors, accounting, version): the paper has no
 * counterpart.
 * Synchronises `stream`, then reads and clears the current device's error
 * word into *flags_host (GS_FLAG_* bits). Returns GS_OK when no bit was set,
 * GS_ERR_DEVICE_FLAG otherwise, GS_ERR_CUDA on a CUDA failure. */
int gs_get_device_error(uint32_t *flags_host, gs_stream_t stream);

/* Static text for a gs_status value. */
const char *gs_status_string(int status);

/* Number of kernels this library has launched in this process, over all
 * devices and streams (a monotone counter for accounting; host-side only). */
uint64_t gs_launch_count(void);

/* Library version, major * 10000 + minor * 100 + patch. */
int gs_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GSTA_H */
