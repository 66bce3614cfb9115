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
#define GS_FLAG_TIMEOUT 4u

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

/* Bytes of workspace gs_sort needs for n Gaussians and `capacity` entries. */
size_t gs_sort_workspace_bytes(int64_t n, int64_t capacity, int32_t width, int32_t height, int32_t tile);

/* Sec. 3.1 ("blended in a sorted order"). Lists, for every tile, the
 * Gaussians whose tile rectangle holds it, in ascending order of
 * (float32 camera depth, Gaussian index). Equivalent to a stable sort of the
 * 64-bit keys (tile << 32 | depth bits) generated in Gaussian order.
 * Out: vals [capacity] (Gaussian index per entry), ranges [tiles][2]
 * (start, end) into vals, count_dev [1] int64 = total entries P.
 * If P > capacity, the entries past the capacity are dropped, ranges are
 * clipped to the capacity, count_dev still holds P, and GS_FLAG_CAPACITY is
 * raised. Workspace: ws of ws_bytes >= gs_sort_workspace_bytes(...).
 * Errors: INVALID_ARG (sizes, tile, workspace too small), CUDA. */
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
    int32_t pixels_per_thread; /* pixels each thread composites: 1 or 2 */
    int32_t batch;             /* splats staged per shared-memory batch: 32, 64, 128 or 256 */
} gs_raster_config;

/* gs_render_fwd with an explicit launch shape (cfg may be NULL). */
int gs_render_fwd_cfg(const float *splats, const uint32_t *vals, const uint32_t *ranges, const gs_camera *cam,
                      const gs_raster_config *cfg, float *image, float *t_final, int32_t *n_last, gs_stream_t stream);

/* Bytes of workspace gs_loss needs for an H x W image. */
size_t gs_loss_workspace_bytes(int32_t H, int32_t W);

/* Sec. 3.1, Eq. 3, L = (1 - lambda) L1 + lambda (1 - SSIM), lambda = 0.2 in
 * the paper. L1 and SSIM are means over the 3 H W values; SSIM per channel
 * with an 11x11 Gaussian window (sigma 1.5), zero padding, C1 = 0.01^2,
 * C2 = 0.03^2; the windows run as separable 1-D passes (the fused SSIM of
 * Sec. 3.3). Out: loss_dev [1] float, dl_dimage [3][H][W] (d|x-y|/dx at
 * x = y taken as 0). A non-finite loss raises GS_FLAG_NONFINITE.
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

/* gs_raster_bwd with an explicit launch shape (cfg may be NULL). */
int gs_raster_bwd_cfg(const float *splats, const uint32_t *vals, const uint32_t *ranges, const gs_camera *cam,
                      const gs_raster_config *cfg, const float *t_final, const int32_t *n_last,
                      const float *dl_dimage, const uint8_t *frozen, float *grad2d, gs_stream_t stream);

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

/* gs_raster_bwd followed by gs_project_bwd on the same stream. */
int gs_render_bwd(const float *P, int64_t n, int32_t sh_degree, const gs_camera *cam, const float *splats,
                  const uint32_t *vals, const uint32_t *ranges, const float *t_final, const int32_t *n_last,
                  const float *dl_dimage, const uint8_t *frozen, const int32_t *act, const int32_t *n_active_dev,
                  float *grad2d, float *G, float *acc_xyz, float *acc_rgb, int32_t *cnt, gs_stream_t stream);

/* Bytes of workspace gs_freeze_update needs for n Gaussians. */
size_t gs_freeze_workspace_bytes(int64_t n);

/* Sec. 3.2.1, Eqs. 4-6, with the cadence of Sec. 4.1. mode:
 *   0 update: frozen[i] |= cnt[i] > 0 && acc_xyz[i]/cnt[i] < eps_xyz
 *                                     && acc_rgb[i]/cnt[i] < eps_rgb
 *             (float32 division and strict comparisons; the map only grows);
 *   1 reset : frozen[i] = 0 for all i;
 *   2 clear : the map is kept.
 * Every mode zeroes acc_xyz, acc_rgb, cnt and writes the unfrozen indices in
 * ascending order to act [n] and their number to n_active_dev [1].
 * Errors: INVALID_ARG (mode, sizes, workspace), CUDA. */
int gs_freeze_update(int64_t n, float *acc_xyz, float *acc_rgb, int32_t *cnt, uint8_t *frozen, float eps_xyz,
                     float eps_rgb, int32_t mode, int32_t *act, int32_t *n_active_dev, void *ws, size_t ws_bytes,
                     gs_stream_t stream);

/* gs_freeze_update without a workspace argument. The paper has no
 * counterpart: this exists for callers that cannot allocate device memory
 * where they make the call -- for example a host that owns every device
 * buffer and hands this library only the inputs and outputs, or a loop that
 * must not call cudaMalloc because an allocation can synchronise the whole
 * device. Its scratch (one count per 1024 Gaussians) is a fixed 256 KB array
 * inside the library that every GPU which loads the library keeps until the
 * process exits; it allows n <= 67,108,864 and returns GS_ERR_INVALID_ARG for
 * more. The first call on a device, made with that device current, looks up
 * the array's device address (cudaGetSymbolAddress); make that first call
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

/* Bytes of workspace gs_psnr needs for S images of H x W. */
size_t gs_psnr_workspace_bytes(int32_t S, int32_t H, int32_t W);

/* Sec. 3.2.2, Eq. 7 input: psnr[s] = 10 log10(1 / MSE) of clamp(image, 0, 1)
 * against gt over the 3 H W values of image s (MSE floored at 1e-10).
 * images, gts [S][3][H][W]; psnr_dev [S] float. Errors: INVALID_ARG, CUDA. */
int gs_psnr(const float *images, const float *gts, int32_t S, int32_t H, int32_t W, void *ws, size_t ws_bytes,
            float *psnr_dev, gs_stream_t stream);

/* Synchronises `stream`, then reads and clears the current device's error
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
