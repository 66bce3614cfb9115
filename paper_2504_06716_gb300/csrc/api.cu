// C-ABI entry points that compose kernels or report state.
#include <atomic>

#include "common.cuh"

namespace gs {
static std::atomic<unsigned long long> g_launches{0};
void note_launches(int k) { g_launches.fetch_add((unsigned long long)k, std::memory_order_relaxed); }
uint32_t take_sort_flags();
uint32_t take_loss_flags();
uint32_t take_render_flags();
}  // namespace gs

using namespace gs;

extern "C" int gs_render_bwd(const float *P, int64_t n, int32_t sh_degree, const gs_camera *cam, const float *splats,
                             const uint32_t *vals, const uint32_t *ranges, const float *t_final, const int32_t *n_last,
                             const float *dl_dimage, const uint8_t *frozen, const int32_t *act,
                             const int32_t *n_active_dev, float *grad2d, float *G, float *acc_xyz, float *acc_rgb,
                             int32_t *cnt, gs_stream_t stream) {
    if (n < 0 || sh_degree < 0 || sh_degree > 3 || !camera_ok(cam)) return GS_ERR_INVALID_ARG;
    int st = gs_raster_bwd(splats, vals, ranges, cam, t_final, n_last, dl_dimage, frozen, grad2d, stream);
    if (st != GS_OK) return st;
    return gs_project_bwd(P, n, sh_degree, cam, splats, act, n_active_dev, grad2d, G, acc_xyz, acc_rgb, cnt, stream);
}

extern "C" int gs_train_step(const gs_step *s, const gs_camera *cam, const float *gt, const float *lr, int64_t step,
                             gs_stream_t stream) {
    if (!s || !cam || !gt || !lr || step < 1 || s->n_stats < 0 || s->n_stats > 2) return GS_ERR_INVALID_ARG;
    const gs_raster_config *fwd = s->fwd.pixels_per_thread ? &s->fwd : nullptr;
    const gs_raster_config *bwd = s->bwd.pixels_per_thread ? &s->bwd : nullptr;
    int st = gs_project_ex(s->P, s->n, s->sh_degree, s->opacity_act, cam, s->splats, stream);
    if (st == GS_OK)
        st = gs_sort(s->splats, s->n, cam, s->sort_ws, s->sort_ws_bytes, s->capacity, s->vals, s->ranges,
                     s->count_dev, stream);
    if (st == GS_OK)
        st = gs_render_fwd_resume(s->splats, s->vals, s->ranges, cam, fwd, s->frozen, s->image, s->t_final, s->n_last,
                                  s->resume, s->resume_pos, stream);
    if (st == GS_OK)
        st = gs_loss(s->image, gt, cam->height, cam->width, s->lambda_ssim, s->loss_ws, s->loss_ws_bytes, s->loss_dev,
                     s->dl_dimage, stream);
    cudaStream_t cs = as_stream(stream);
    if (st == GS_OK && s->bwd_events[0] && cudaEventRecord(static_cast<cudaEvent_t>(s->bwd_events[0]), cs) != cudaSuccess)
        st = GS_ERR_CUDA;
    if (st == GS_OK)
        st = gs_raster_bwd_resume(s->splats, s->vals, s->ranges, cam, bwd, s->t_final, s->n_last, s->dl_dimage,
                                  s->frozen, s->resume, s->resume_pos, s->grad2d, stream);
    if (st == GS_OK && s->bwd_events[1] && cudaEventRecord(static_cast<cudaEvent_t>(s->bwd_events[1]), cs) != cudaSuccess)
        st = GS_ERR_CUDA;
    if (st == GS_OK)
        st = gs_project_bwd_ex(s->P, s->n, s->sh_degree, s->opacity_act, s->mask_loss, cam, s->splats, s->act,
                               s->n_active_dev, s->grad2d, s->G, 0, s->stats, s->n_stats, stream);
    if (st == GS_OK)
        st = gs_adam_masked_groups(s->P, s->G, s->m, s->v, s->n, s->act, s->n_active_dev, lr,
                                   s->n_lr ? s->n_lr : 6, s->b1, s->b2, s->eps, step, stream);
    return st;
}

extern "C" int gs_get_device_error(uint32_t *flags_host, gs_stream_t stream) {
    if (!flags_host) return GS_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(as_stream(stream)) != cudaSuccess) return GS_ERR_CUDA;
    uint32_t f = take_sort_flags() | take_loss_flags() | take_render_flags();
    if (cudaGetLastError() != cudaSuccess) return GS_ERR_CUDA;
    *flags_host = f;
    return f ? GS_ERR_DEVICE_FLAG : GS_OK;
}

extern "C" const char *gs_status_string(int status) {
    switch (status) {
        case GS_OK: return "ok";
        case GS_ERR_INVALID_ARG: return "invalid argument";
        case GS_ERR_CUDA: return "CUDA error";
        case GS_ERR_CAPACITY: return "sort capacity exceeded";
        case GS_ERR_NONFINITE: return "non-finite value";
        case GS_ERR_TIMEOUT: return "bounded wait timed out";
        case GS_ERR_DEVICE_FLAG: return "device error flag set";
        default: return "unknown status";
    }
}

extern "C" int gs_version(void) { return 100; }

extern "C" uint64_t gs_launch_count(void) { return (uint64_t)g_launches.load(std::memory_order_relaxed); }
