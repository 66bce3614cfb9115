// Shared device helpers for the GSta kernels (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gsta.h"

namespace gs {

constexpr int kRow = 64;    // floats per parameter row (59 used)
constexpr int kSplat = 12;  // floats per projected splat record
constexpr int kG2d = 12;    // floats per raster-gradient row (9 used)
constexpr unsigned kFull = 0xffffffffu;

// Kernel-argument copy of gs_camera plus derived constants.
struct DevCam {
    int W, H, tile, tiles_x, tiles_y;
    float fx, fy, cx, cy;
    float R[9], t[3], campos[3];
    float znear, dilation;
    float bg[3];
    float limx, limy;  // 1.3 x tan(half field of view), the Jacobian clamp
};

inline bool tile_ok(int t) { return t == 8 || t == 16 || t == 32; }

inline bool camera_ok(const gs_camera *c) {
    if (!c) return false;
    if (c->width <= 0 || c->height <= 0 || c->width > 16384 || c->height > 16384) return false;
    if (!tile_ok(c->tile)) return false;
    if (!(c->fx > 0.f) || !(c->fy > 0.f)) return false;
    if (!(c->znear >= 0.f) || !(c->dilation >= 0.f)) return false;
    return true;
}

__host__ __device__ inline DevCam make_cam(const gs_camera *c) {
    DevCam d;
    d.W = c->width;
    d.H = c->height;
    d.tile = c->tile;
    d.tiles_x = (c->width + c->tile - 1) / c->tile;
    d.tiles_y = (c->height + c->tile - 1) / c->tile;
    d.fx = c->fx; d.fy = c->fy; d.cx = c->cx; d.cy = c->cy;
    for (int i = 0; i < 9; ++i) d.R[i] = c->R[i];
    for (int i = 0; i < 3; ++i) { d.t[i] = c->t[i]; d.campos[i] = c->campos[i]; d.bg[i] = c->bg[i]; }
    d.znear = c->znear;
    d.dilation = c->dilation;
    d.limx = 1.3f * 0.5f * (float)c->width / c->fx;
    d.limy = 1.3f * 0.5f * (float)c->height / c->fy;
    return d;
}

inline cudaStream_t as_stream(gs_stream_t s) { return reinterpret_cast<cudaStream_t>(s); }

// Adds k to the library-wide count of kernel launches (gs_launch_count).
void note_launches(int k);

inline int launch_status() { return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA; }

// Two float32 values in one 64-bit register pair, and the packed FP32
// instructions of sm_100 and later (add/sub/mul/fma .rn .f32x2): each half is
// rounded exactly as the scalar __fadd_rn / __fsub_rn / __fmul_rn / __fmaf_rn
// of the same operands, and one instruction issues both.
typedef unsigned long long f32x2;

__device__ __forceinline__ f32x2 f2_pack(float lo, float hi) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ void f2_unpack(f32x2 v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

__device__ __forceinline__ f32x2 f2_sub(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

__device__ __forceinline__ f32x2 f2_mul(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

__device__ __forceinline__ f32x2 f2_fma(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// Programmatic dependent launch: a kernel started by launch_chained may be
// scheduled while the kernel before it in the stream is still finishing, so
// that its launch overlaps that kernel's last blocks. It must call
// wait_prior_grid() before anything else: griddepcontrol.wait returns once
// the grids it depends on have completed and their memory operations are
// visible (at once when it was launched without a dependency).
__device__ __forceinline__ void wait_prior_grid() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline void launch_chained(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t s, Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

inline unsigned grid_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

// Tile rectangle of a splat, decided in float32 with explicitly rounded
// operations: x0 = floor((mx - r) / tile), x1 = floor((mx + r) / tile),
// clipped to the grid. Writes the half-open rectangle; returns the count.
__device__ __forceinline__ int tile_rect(float mx, float my, int r, int tile, int tx, int ty, int &x0, int &y0,
                                         int &x1, int &y1) {
    float inv = 1.0f / (float)tile;  // exact: tile is a power of two
    float fr = (float)r;
    float fx0 = floorf(__fmul_rn(__fsub_rn(mx, fr), inv));
    float fx1 = floorf(__fmul_rn(__fadd_rn(mx, fr), inv));
    float fy0 = floorf(__fmul_rn(__fsub_rn(my, fr), inv));
    float fy1 = floorf(__fmul_rn(__fadd_rn(my, fr), inv));
    fx0 = fmaxf(fx0, 0.0f);
    fy0 = fmaxf(fy0, 0.0f);
    fx1 = fminf(fx1, (float)(tx - 1));
    fy1 = fminf(fy1, (float)(ty - 1));
    if (fx0 > fx1 || fy0 > fy1) {
        x0 = y0 = x1 = y1 = 0;
        return 0;
    }
    x0 = (int)fx0;
    y0 = (int)fy0;
    x1 = (int)fx1 + 1;
    y1 = (int)fy1 + 1;
    return (x1 - x0) * (y1 - y0);
}

// Opacity from its parameter under the sigmoid activation; one definition
// for the projection and for the switch to the absolute-value activation,
// which must reproduce it bit for bit.
__device__ __forceinline__ float opacity_sigmoid(float x) { return 1.f / (1.f + expf(-x)); }

// Exponent of the 2-D Gaussian at offset (dx, dy), -0.5 (a dx^2 + c dy^2) -
// b dx dy, as a quadratic in dy whose coefficients depend on dx only:
// power = (c2 dy + c1) dy + c0 with c2 = -c/2, c1 = -b dx, c0 = -a dx^2 / 2.
// A thread's pixels share a column, so per splat it forms the row once and
// pays two fused multiply-adds per pixel. Every kernel rounds it the same
// way (explicit intrinsics), so forward and backward take identical skip
// decisions.
struct SplatRow {
    float c0, c1, c2;
};

__device__ __forceinline__ SplatRow splat_row(float dx, float a, float b, float c) {
    SplatRow r;
    r.c0 = __fmul_rn(__fmul_rn(-0.5f, a), __fmul_rn(dx, dx));
    r.c1 = __fmul_rn(-b, dx);
    r.c2 = __fmul_rn(-0.5f, c);
    return r;
}

__device__ __forceinline__ float splat_power(const SplatRow &r, float dy) {
    return __fmaf_rn(__fmaf_rn(r.c2, dy, r.c1), dy, r.c0);
}

constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaMax = 0.99f;
constexpr float kTMin = 1e-4f;

// Block-wide exclusive scan of one int per thread (blockDim.x <= 1024, a
// multiple of 32). Returns the exclusive prefix; *total gets the block sum.
// `warp_sums` must hold 32 ints of shared memory.
__device__ __forceinline__ int block_exclusive_scan(int v, int *warp_sums, int *total) {
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = lane < nwarps ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(kFull, w, o);
            if (lane >= o) w += y;
        }
        warp_sums[lane] = w;  // inclusive prefix over warps
    }
    __syncthreads();
    int before = warp > 0 ? warp_sums[warp - 1] : 0;
    *total = warp_sums[nwarps - 1];
    __syncthreads();
    return before + x - v;
}

}  // namespace gs
