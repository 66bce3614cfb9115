// Image-space schedules of the Trick-GS additions (Sec. 3.3, "Progressive
// Training" and "Blur"): the target image at a reduced resolution (area
// average over the same extent of the image plane) and its Gaussian blur.
// Both are small memory-bound passes over one image per iteration.
#include "common.cuh"

namespace gs {
namespace {

// Area average: target pixel i of n2 covers source [i n / n2 - 1/2,
// (i + 1) n / n2 - 1/2); in units of 1 / (2 n2) every bound is an integer,
// so the overlaps (the weights) are exact integers summing to 2 n.
__device__ __forceinline__ int overlap(int i, int j, int n, int n2) {
    const int a = 2 * i * n - n2, b = 2 * (i + 1) * n - n2;       // target interval
    const int lo = (2 * j - 1) * n2, hi = (2 * j + 1) * n2;         // source pixel j
    const int ov = min(b, hi) - max(a, lo);
    return ov > 0 ? ov : 0;
}

__global__ void __launch_bounds__(256) k_resize_area(const float *__restrict__ src, int C, int W, int H,
                                                     float *__restrict__ dst, int W2, int H2) {
    const int64_t total = (int64_t)C * H2 * W2;
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < total;
         o += (int64_t)gridDim.x * blockDim.x) {
        const int x2 = (int)(o % W2), y2 = (int)((o / W2) % H2), c = (int)(o / ((int64_t)W2 * H2));
        const int jx0 = (int)(((int64_t)x2 * W) / W2), jx1 = min(W - 1, (int)(((int64_t)(x2 + 1) * W) / W2));
        const int jy0 = (int)(((int64_t)y2 * H) / H2), jy1 = min(H - 1, (int)(((int64_t)(y2 + 1) * H) / H2));
        const float *s = src + (int64_t)c * H * W;
        float acc = 0.f;
        for (int jy = jy0; jy <= jy1; ++jy) {
            const int wy = overlap(y2, jy, H, H2);
            if (!wy) continue;
            float row = 0.f;
            for (int jx = jx0; jx <= jx1; ++jx) {
                const int wx = overlap(x2, jx, W, W2);
                if (wx) row += (float)wx * __ldg(s + (int64_t)jy * W + jx);
            }
            acc += (float)wy * row;
        }
        dst[o] = acc / ((float)(2 * W) * (float)(2 * H));
    }
}

struct Taps {
    float w[5];  // w[2 + d] = exp(-d^2 / (2 sigma^2)), d = -2 .. 2
};

// 5 x 5 Gaussian with the weights renormalised over the taps inside the image
// (separable: the normaliser is the product of the in-image row and column sums).
__global__ void __launch_bounds__(256) k_blur5(const float *__restrict__ src, int C, int W, int H, Taps t,
                                               float *__restrict__ dst) {
    const int64_t total = (int64_t)C * H * W;
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < total;
         o += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(o % W), y = (int)((o / W) % H), c = (int)(o / ((int64_t)W * H));
        const float *s = src + (int64_t)c * H * W;
        float acc = 0.f, sx = 0.f, sy = 0.f;
#pragma unroll
        for (int d = -2; d <= 2; ++d) {
            if (x + d >= 0 && x + d < W) sx += t.w[2 + d];
            if (y + d >= 0 && y + d < H) sy += t.w[2 + d];
        }
#pragma unroll
        for (int dy = -2; dy <= 2; ++dy) {
            const int yy = y + dy;
            if (yy < 0 || yy >= H) continue;
            float row = 0.f;
#pragma unroll
            for (int dx = -2; dx <= 2; ++dx) {
                const int xx = x + dx;
                if (xx >= 0 && xx < W) row += t.w[2 + dx] * __ldg(s + (int64_t)yy * W + xx);
            }
            acc += t.w[2 + dy] * row;
        }
        dst[o] = acc / (sx * sy);
    }
}

unsigned grid_of(int64_t total) {
    const int64_t b = (total + 255) / 256;
    return (unsigned)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" int gs_resize_area(const float *src, int32_t C, int32_t W, int32_t H, float *dst, int32_t W2, int32_t H2,
                              gs_stream_t stream) {
    if (C <= 0 || W <= 0 || H <= 0 || W2 <= 0 || H2 <= 0 || W > 16384 || H > 16384 || W2 > 16384 || H2 > 16384)
        return GS_ERR_INVALID_ARG;
    if (!src || !dst || src == dst) return GS_ERR_INVALID_ARG;
    const int64_t total = (int64_t)C * H2 * W2;
    k_resize_area<<<grid_of(total), 256, 0, as_stream(stream)>>>(src, C, W, H, dst, W2, H2);
    note_launches(1);
    return launch_status();
}

extern "C" int gs_blur(const float *src, int32_t C, int32_t W, int32_t H, float sigma, float *dst,
                       gs_stream_t stream) {
    if (C <= 0 || W <= 0 || H <= 0 || !(sigma >= 0.f) || !src || !dst || src == dst) return GS_ERR_INVALID_ARG;
    const int64_t total = (int64_t)C * H * W;
    cudaStream_t s = as_stream(stream);
    if (sigma < GS_BLUR_SIGMA_MIN) {
        if (cudaMemcpyAsync(dst, src, sizeof(float) * (size_t)total, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return GS_ERR_CUDA;
        return GS_OK;
    }
    Taps t;
    for (int d = -2; d <= 2; ++d) t.w[2 + d] = (float)exp(-(double)(d * d) / (2.0 * (double)sigma * (double)sigma));
    k_blur5<<<grid_of(total), 256, 0, s>>>(src, C, W, H, t, dst);
    note_launches(1);
    return launch_status();
}
