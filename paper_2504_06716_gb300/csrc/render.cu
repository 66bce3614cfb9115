// Tile rasteriser: front-to-back alpha compositing (Sec. 3.1, Eq. 2) and its
// backward (Sec. 3.2.4), which skips the gradient work of frozen Gaussians.
//
// One CTA per screen tile, one thread per pixel. The tile's sorted splat list
// is staged through shared memory in batches (one record per thread), so
// every thread reads each splat as a shared-memory broadcast. No tensor
// cores: the work is a per-pixel exponential and a handful of FMAs.
//
// The backward walks each list back to front and recovers the transmittance
// in front of every splat from the value the forward left over, so no
// per-pixel list is stored. A warp's 32 pixels see the same splat at the
// same time; their nine gradient terms are summed with warp shuffles, then
// added once per warp into a shared accumulator, and the accumulator goes
// to global memory with one atomic per value per tile.
#include "common.cuh"

namespace gs {
namespace {

constexpr int kBatch = 256;

template <int TS>
__global__ void __launch_bounds__(TS * TS) k_render_fwd(const float *__restrict__ splats,
                                                        const uint32_t *__restrict__ vals,
                                                        const uint32_t *__restrict__ ranges, DevCam cam,
                                                        float *__restrict__ image, float *__restrict__ t_final,
                                                        int32_t *__restrict__ n_last) {
    constexpr int NT = TS * TS;
    constexpr int B = NT < kBatch ? NT : kBatch;
    __shared__ float4 s_xyab[B];
    __shared__ float4 s_cocg[B];
    __shared__ float s_blue[B];
    const int tile = blockIdx.x;
    const int tx = tile % cam.tiles_x, ty = tile / cam.tiles_x;
    const int px = tx * TS + (int)(threadIdx.x % TS), py = ty * TS + (int)(threadIdx.x / TS);
    const bool inside = px < cam.W && py < cam.H;
    const uint32_t start = ranges[2 * tile], end = ranges[2 * tile + 1];
    const float fpx = (float)px, fpy = (float)py;
    float T = 1.f, c0 = 0.f, c1 = 0.f, c2 = 0.f;
    int last = 0;
    bool done = !inside;
    for (uint32_t base = start; base < end; base += B) {
        if (__syncthreads_count(done) == NT) break;
        if (threadIdx.x < B && base + threadIdx.x < end) {
            const float4 *r = reinterpret_cast<const float4 *>(splats + (int64_t)vals[base + threadIdx.x] * kSplat);
            s_xyab[threadIdx.x] = __ldg(r);
            s_cocg[threadIdx.x] = __ldg(r + 1);
            s_blue[threadIdx.x] = __ldg(reinterpret_cast<const float *>(r + 2));
        }
        __syncthreads();
        const int cnt = (int)min((uint32_t)B, end - base);
        for (int j = 0; j < cnt && !done; ++j) {
            const float4 xa = s_xyab[j], co = s_cocg[j];
            const float dx = __fsub_rn(xa.x, fpx), dy = __fsub_rn(xa.y, fpy);
            const float power = splat_power(dx, dy, xa.z, xa.w, co.x);
            if (power > 0.f) continue;
            const float alpha = fminf(kAlphaMax, __fmul_rn(co.y, __expf(power)));
            if (alpha < kAlphaMin) continue;
            const float tn = __fmul_rn(T, __fsub_rn(1.f, alpha));
            if (tn < kTMin) { done = true; break; }
            const float w = alpha * T;
            c0 += co.z * w;
            c1 += co.w * w;
            c2 += s_blue[j] * w;
            T = tn;
            last = (int)(base - start) + j + 1;
        }
    }
    if (inside) {
        const int64_t pix = (int64_t)py * cam.W + px, HW = (int64_t)cam.W * cam.H;
        image[pix] = c0 + T * cam.bg[0];
        image[HW + pix] = c1 + T * cam.bg[1];
        image[2 * HW + pix] = c2 + T * cam.bg[2];
        t_final[pix] = T;
        n_last[pix] = last;
    }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

template <int TS>
__global__ void __launch_bounds__(TS * TS) k_raster_bwd(const float *__restrict__ splats,
                                                        const uint32_t *__restrict__ vals,
                                                        const uint32_t *__restrict__ ranges, DevCam cam,
                                                        const float *__restrict__ t_final,
                                                        const int32_t *__restrict__ n_last,
                                                        const float *__restrict__ dl_dimage,
                                                        const uint8_t *__restrict__ frozen,
                                                        float *__restrict__ grad2d) {
    constexpr int NT = TS * TS;
    constexpr int B = NT < kBatch ? NT : kBatch;
    __shared__ float4 s_xyab[B];
    __shared__ float4 s_cocg[B];
    __shared__ float s_blue[B];
    __shared__ uint32_t s_gid[B];
    __shared__ int s_frz[B];
    __shared__ float s_acc[9][B];
    __shared__ int s_maxlast;
    const int tile = blockIdx.x;
    const int tx = tile % cam.tiles_x, ty = tile / cam.tiles_x;
    const int px = tx * TS + (int)(threadIdx.x % TS), py = ty * TS + (int)(threadIdx.x / TS);
    const bool inside = px < cam.W && py < cam.H;
    const uint32_t start = ranges[2 * tile];
    const float fpx = (float)px, fpy = (float)py;
    const int64_t pix = (int64_t)py * cam.W + px, HW = (int64_t)cam.W * cam.H;

    float T = 1.f, dC0 = 0.f, dC1 = 0.f, dC2 = 0.f;
    int nl = 0;
    if (inside) {
        T = t_final[pix];
        nl = n_last[pix];
        dC0 = dl_dimage[pix];
        dC1 = dl_dimage[HW + pix];
        dC2 = dl_dimage[2 * HW + pix];
    }
    const float Tf = T;
    const float bgdot = cam.bg[0] * dC0 + cam.bg[1] * dC1 + cam.bg[2] * dC2;
    float S0 = 0.f, S1 = 0.f, S2 = 0.f;  // colour behind the current splat, per unit transmittance
    float la = 0.f, lc0 = 0.f, lc1 = 0.f, lc2 = 0.f;  // alpha and colour of the splat behind

    if (threadIdx.x == 0) s_maxlast = 0;
    __syncthreads();
    if (nl > 0) atomicMax(&s_maxlast, nl);
    __syncthreads();
    const uint32_t rend = start + (uint32_t)s_maxlast;
    const int lane = threadIdx.x & 31;

    for (int64_t bend = rend; bend > (int64_t)start; bend -= B) {
        const int64_t bstart = bend - B > (int64_t)start ? bend - B : (int64_t)start;
        const int cnt = (int)(bend - bstart);
        if ((int)threadIdx.x < cnt) {
            const uint32_t g = vals[bstart + threadIdx.x];
            const float4 *r = reinterpret_cast<const float4 *>(splats + (int64_t)g * kSplat);
            s_xyab[threadIdx.x] = __ldg(r);
            s_cocg[threadIdx.x] = __ldg(r + 1);
            s_blue[threadIdx.x] = __ldg(reinterpret_cast<const float *>(r + 2));
            s_gid[threadIdx.x] = g;
            s_frz[threadIdx.x] = frozen ? (int)frozen[g] : 0;
        }
        if ((int)threadIdx.x < B) {
#pragma unroll
            for (int q = 0; q < 9; ++q) s_acc[q][threadIdx.x] = 0.f;
        }
        __syncthreads();
        for (int j = cnt - 1; j >= 0; --j) {
            const int pos = (int)(bstart - (int64_t)start) + j;  // position in the tile list
            const float4 xa = s_xyab[j], co = s_cocg[j];
            const float blue = s_blue[j];
            const float dx = __fsub_rn(xa.x, fpx), dy = __fsub_rn(xa.y, fpy);
            const float power = splat_power(dx, dy, xa.z, xa.w, co.x);
            const float G = __expf(power);
            const float oG = __fmul_rn(co.y, G);
            const float alpha = fminf(kAlphaMax, oG);
            const bool contrib = pos < nl && power <= 0.f && alpha >= kAlphaMin;
            float g0 = 0.f, g1 = 0.f, g2 = 0.f, g3 = 0.f, g4 = 0.f, g5 = 0.f, g6 = 0.f, g7 = 0.f, g8 = 0.f;
            if (contrib) {
                const float om = 1.f - alpha;
                T = __fdividef(T, om);  // transmittance in front of this splat
                S0 = la * lc0 + (1.f - la) * S0;
                S1 = la * lc1 + (1.f - la) * S1;
                S2 = la * lc2 + (1.f - la) * S2;
                if (!s_frz[j]) {
                    const float dA = T * (dC0 * (co.z - S0) + dC1 * (co.w - S1) + dC2 * (blue - S2)) -
                                     __fdividef(Tf, om) * bgdot;
                    const float wT = alpha * T;
                    g6 = wT * dC0;
                    g7 = wT * dC1;
                    g8 = wT * dC2;
                    if (!(oG > kAlphaMax)) {
                        const float dpow = dA * oG;
                        g5 = dA * G;
                        g2 = -0.5f * dx * dx * dpow;
                        g3 = -dx * dy * dpow;
                        g4 = -0.5f * dy * dy * dpow;
                        g0 = -(xa.z * dx + xa.w * dy) * dpow;
                        g1 = -(xa.w * dx + co.x * dy) * dpow;
                    }
                }
                la = alpha;
                lc0 = co.z;
                lc1 = co.w;
                lc2 = blue;
            }
            if (!s_frz[j] && __any_sync(kFull, contrib)) {
                g0 = warp_sum(g0); g1 = warp_sum(g1); g2 = warp_sum(g2);
                g3 = warp_sum(g3); g4 = warp_sum(g4); g5 = warp_sum(g5);
                g6 = warp_sum(g6); g7 = warp_sum(g7); g8 = warp_sum(g8);
                if (lane == 0) {
                    atomicAdd(&s_acc[0][j], g0); atomicAdd(&s_acc[1][j], g1); atomicAdd(&s_acc[2][j], g2);
                    atomicAdd(&s_acc[3][j], g3); atomicAdd(&s_acc[4][j], g4); atomicAdd(&s_acc[5][j], g5);
                    atomicAdd(&s_acc[6][j], g6); atomicAdd(&s_acc[7][j], g7); atomicAdd(&s_acc[8][j], g8);
                }
            }
        }
        __syncthreads();
        if ((int)threadIdx.x < cnt && !s_frz[threadIdx.x]) {
            float *dst = grad2d + (int64_t)s_gid[threadIdx.x] * kG2d;
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                const float v = s_acc[q][threadIdx.x];
                if (v != 0.f) atomicAdd(dst + q, v);
            }
        }
        __syncthreads();
    }
}

template <int TS>
int launch_fwd(const float *splats, const uint32_t *vals, const uint32_t *ranges, const DevCam &dc, float *image,
               float *t_final, int32_t *n_last, cudaStream_t s) {
    k_render_fwd<TS><<<dc.tiles_x * dc.tiles_y, TS * TS, 0, s>>>(splats, vals, ranges, dc, image, t_final, n_last);
    note_launches(1);
    return launch_status();
}

template <int TS>
int launch_bwd(const float *splats, const uint32_t *vals, const uint32_t *ranges, const DevCam &dc,
               const float *t_final, const int32_t *n_last, const float *dl, const uint8_t *frozen, float *grad2d,
               cudaStream_t s) {
    k_raster_bwd<TS><<<dc.tiles_x * dc.tiles_y, TS * TS, 0, s>>>(splats, vals, ranges, dc, t_final, n_last, dl,
                                                                  frozen, grad2d);
    note_launches(1);
    return launch_status();
}

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" int gs_render_fwd(const float *splats, const uint32_t *vals, const uint32_t *ranges, const gs_camera *cam,
                             float *image, float *t_final, int32_t *n_last, gs_stream_t stream) {
    if (!camera_ok(cam) || !ranges || !image || !t_final || !n_last) return GS_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(splats) & 15) return GS_ERR_INVALID_ARG;
    DevCam dc = make_cam(cam);
    cudaStream_t s = as_stream(stream);
    switch (dc.tile) {
        case 8: return launch_fwd<8>(splats, vals, ranges, dc, image, t_final, n_last, s);
        case 16: return launch_fwd<16>(splats, vals, ranges, dc, image, t_final, n_last, s);
        default: return launch_fwd<32>(splats, vals, ranges, dc, image, t_final, n_last, s);
    }
}

extern "C" int gs_raster_bwd(const float *splats, const uint32_t *vals, const uint32_t *ranges, const gs_camera *cam,
                             const float *t_final, const int32_t *n_last, const float *dl_dimage,
                             const uint8_t *frozen, float *grad2d, gs_stream_t stream) {
    if (!camera_ok(cam) || !ranges || !t_final || !n_last || !dl_dimage || !grad2d) return GS_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(splats) & 15) return GS_ERR_INVALID_ARG;
    DevCam dc = make_cam(cam);
    cudaStream_t s = as_stream(stream);
    switch (dc.tile) {
        case 8: return launch_bwd<8>(splats, vals, ranges, dc, t_final, n_last, dl_dimage, frozen, grad2d, s);
        case 16: return launch_bwd<16>(splats, vals, ranges, dc, t_final, n_last, dl_dimage, frozen, grad2d, s);
        default: return launch_bwd<32>(splats, vals, ranges, dc, t_final, n_last, dl_dimage, frozen, grad2d, s);
    }
}
