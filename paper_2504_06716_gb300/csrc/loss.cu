// Training loss L = (1 - lambda) L1 + lambda (1 - SSIM) and dL/dimage
// (Sec. 3.1, Eq. 3), and the PSNR of Eq. 7's early-stop check (Sec. 3.2.2).
//
// SSIM uses the 11x11 Gaussian window (sigma 1.5) as two 1-D passes in
// shared memory (Sec. 3.3, "Accelerated SSIM loss calculation"): one kernel
// builds the five window moments of a 32x32 tile plus its 5-pixel halo and
// emits the SSIM map's three partial-derivative maps; a second kernel runs
// the same separable window over those maps (the window is symmetric, so it
// is its own adjoint) and combines them with the L1 term into dL/dimage.
// Block partial sums are reduced in a fixed order, so the loss is
// deterministic.
#include "common.cuh"

namespace gs {

__device__ uint32_t g_loss_flags;

namespace {

constexpr int kT = 32;            // output tile edge
constexpr int kR = 5;             // window radius
constexpr int kE = kT + 2 * kR;   // tile edge with halo
constexpr int kLossThreads = 256;
constexpr int kLoadRows = kLossThreads / kE;  // haloed rows loaded per round (6; threads 252-255 idle)

struct Win {
    float w[11];
};

// Each pass gives a thread kV = 4 consecutive outputs, so that it reads the
// kV + 10 inputs of their windows once from shared memory instead of
// 11 per output. Horizontal items: (row of the haloed tile, 4 columns);
// vertical items: (column, 4 rows), one per thread, a warp on 32 columns.
constexpr int kV = 4;
constexpr int kSeg = kT / kV;              // 8 segments per row / column
constexpr int kHItems = kE * kSeg;         // 336 horizontal items
static_assert(kT * kSeg == kLossThreads, "one vertical item per thread");

// The loss from the per-block partial sums (L1 sum, SSIM sum), by the last
// block to finish: every thread sums a fixed stride of them in double, then a
// fixed-shape tree, so the result does not depend on the block order.
__device__ void loss_from_parts(const float2 *part, int nparts, int64_t N, float lambda, float *loss,
                                double *scratch /* shared, 2 * kLossThreads */) {
    double *r1 = scratch, *r2 = scratch + kLossThreads;
    double a = 0.0, b = 0.0;
    for (int k = threadIdx.x; k < nparts; k += kLossThreads) {
        const float2 v = __ldcg(part + k);
        a += (double)v.x;
        b += (double)v.y;
    }
    r1[threadIdx.x] = a;
    r2[threadIdx.x] = b;
    __syncthreads();
    for (int w = kLossThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            r1[threadIdx.x] += r1[threadIdx.x + w];
            r2[threadIdx.x] += r2[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double L = (1.0 - lambda) * r1[0] / (double)N + lambda * (1.0 - r2[0] / (double)N);
        const float Lf = (float)L;
        if (!isfinite(Lf)) atomicOr(&g_loss_flags, GS_FLAG_NONFINITE);
        *loss = Lf;
    }
}

__global__ void __launch_bounds__(kLossThreads) k_ssim_fwd(const float *__restrict__ img,
                                                          const float *__restrict__ gt, int H, int W, Win win,
                                                          float *__restrict__ mapA, float *__restrict__ mapB,
                                                          float *__restrict__ mapC, float2 *__restrict__ part,
                                                          unsigned int *__restrict__ done, float lambda,
                                                          float *__restrict__ loss) {
    __shared__ float sx[kE][kE + 1], sy[kE][kE + 1];
    __shared__ __align__(16) float h[5][kE][kT + 1];  // also the last block's reduction scratch
    __shared__ float red[2][kLossThreads / 32];
    __shared__ bool last;
    static_assert(sizeof(h) >= 2 * kLossThreads * sizeof(double), "scratch fits");
    wait_prior_grid();
    const int ch = blockIdx.z;
    const int64_t HW = (int64_t)H * W;
    const float *x = img + ch * HW, *y = gt + ch * HW;
    const int oy = blockIdx.y * kT - kR, ox = blockIdx.x * kT - kR;
    {   // thread t loads column t % kE of rows t / kE, + kLoadRows, ...: all its loads in flight together
        const int c = (int)threadIdx.x % kE, r0 = (int)threadIdx.x / kE;
        const int gx = ox + c;
        const bool col_in = gx >= 0 && gx < W;
        if (r0 < kLoadRows) {
#pragma unroll
            for (int r = r0; r < kE; r += kLoadRows) {
                const int gy = oy + r;
                const bool in = col_in && gy >= 0 && gy < H;
                const int64_t o = (int64_t)gy * W + gx;
                sx[r][c] = in ? __ldg(x + o) : 0.f;
                sy[r][c] = in ? __ldg(y + o) : 0.f;
            }
        }
    }
    __syncthreads();
    // horizontal: window sums of x, y, x^2, y^2, x y along the rows
    for (int it = threadIdx.x; it < kHItems; it += kLossThreads) {
        const int r = it / kSeg, c0 = (it % kSeg) * kV;
        float a[kV], b[kV], aa[kV], bb[kV], ab[kV];
#pragma unroll
        for (int v = 0; v < kV; ++v) a[v] = b[v] = aa[v] = bb[v] = ab[v] = 0.f;
#pragma unroll
        for (int q = 0; q < kV + 10; ++q) {
            const float xv = sx[r][c0 + q], yv = sy[r][c0 + q];
            const float xx = xv * xv, yy = yv * yv, xy = xv * yv;
#pragma unroll
            for (int v = 0; v < kV; ++v) {
                const int t = q - v;  // tap of input q in output v's window
                if (t >= 0 && t < 11) {
                    const float w = win.w[t];
                    a[v] += w * xv; b[v] += w * yv; aa[v] += w * xx; bb[v] += w * yy; ab[v] += w * xy;
                }
            }
        }
#pragma unroll
        for (int v = 0; v < kV; ++v) {
            h[0][r][c0 + v] = a[v]; h[1][r][c0 + v] = b[v]; h[2][r][c0 + v] = aa[v];
            h[3][r][c0 + v] = bb[v]; h[4][r][c0 + v] = ab[v];
        }
    }
    __syncthreads();
    // vertical, then the SSIM map and its partial derivatives
    const float C1 = 0.01f * 0.01f, C2 = 0.03f * 0.03f;
    float l1 = 0.f, ss = 0.f;
    {
        const int c = threadIdx.x % kT, r0 = (threadIdx.x / kT) * kV;
        float mx[kV], my[kV], xx[kV], yy[kV], xy[kV];
#pragma unroll
        for (int v = 0; v < kV; ++v) mx[v] = my[v] = xx[v] = yy[v] = xy[v] = 0.f;
#pragma unroll
        for (int q = 0; q < kV + 10; ++q) {
            const float h0 = h[0][r0 + q][c], h1 = h[1][r0 + q][c], h2 = h[2][r0 + q][c];
            const float h3 = h[3][r0 + q][c], h4 = h[4][r0 + q][c];
#pragma unroll
            for (int v = 0; v < kV; ++v) {
                const int t = q - v;
                if (t >= 0 && t < 11) {
                    const float w = win.w[t];
                    mx[v] += w * h0; my[v] += w * h1; xx[v] += w * h2; yy[v] += w * h3; xy[v] += w * h4;
                }
            }
        }
#pragma unroll
        for (int v = 0; v < kV; ++v) {
            const int r = r0 + v;
            const int gy = blockIdx.y * kT + r, gx = blockIdx.x * kT + c;
            if (gy >= H || gx >= W) continue;
            const float vx = xx[v] - mx[v] * mx[v], vy = yy[v] - my[v] * my[v], cxy = xy[v] - mx[v] * my[v];
            const float n1 = 2.f * mx[v] * my[v] + C1, n2 = 2.f * cxy + C2;
            const float d1 = mx[v] * mx[v] + my[v] * my[v] + C1, d2 = vx + vy + C2;
            // d1 >= C1 and d2 >= C2 (up to rounding of the variances): the map
            // and its partials are formed without dividing by n1 or n2, which
            // may be zero (m / n2 = n1 / (d1 d2), m / n1 = n2 / (d1 d2))
            const float rd1 = __fdividef(1.f, d1), rd2 = __fdividef(1.f, d2);  // d1, d2 in [1e-4, 3]
            const float qd = rd1 * rd2;
            const float m_n1 = n2 * qd, m_n2 = n1 * qd;
            const float m = n1 * m_n1;
            ss += m;
            l1 += fabsf(sx[r + kR][c + kR] - sy[r + kR][c + kR]);
            // partials of the map value w.r.t. the window means of x, x^2 and x*y
            const int64_t p = ch * HW + (int64_t)gy * W + gx;
            mapA[p] = 2.f * my[v] * (m_n1 - m_n2) + 2.f * mx[v] * m * (rd2 - rd1);
            mapB[p] = -m * rd2;
            mapC[p] = 2.f * m_n2;
        }
    }
    // block sums
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        l1 += __shfl_xor_sync(kFull, l1, o);
        ss += __shfl_xor_sync(kFull, ss, o);
    }
    if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = l1; red[1][threadIdx.x >> 5] = ss; }
    __syncthreads();
    const unsigned int nblk = gridDim.x * gridDim.y * gridDim.z;
    if (threadIdx.x == 0) {
        float a = 0.f, b = 0.f;
        for (int w = 0; w < kLossThreads / 32; ++w) { a += red[0][w]; b += red[1][w]; }
        int64_t blk = ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        part[blk] = make_float2(a, b);
        __threadfence();  // the partial is visible before this block is counted
        last = atomicAdd(done, 1u) == nblk - 1;
    }
    __syncthreads();
    if (last) {
        __threadfence();
        loss_from_parts(part, (int)nblk, 3 * HW, lambda, loss, reinterpret_cast<double *>(&h[0][0][0]));
    }
}

__global__ void __launch_bounds__(kLossThreads, 5) k_ssim_bwd(const float *__restrict__ img,
                                                          const float *__restrict__ gt, int H, int W, Win win,
                                                          float lambda, const float *__restrict__ mapA,
                                                          const float *__restrict__ mapB,
                                                          const float *__restrict__ mapC, float *__restrict__ dl) {
    __shared__ float sm[3][kE][kE + 1];
    __shared__ float h[3][kE][kT + 1];
    wait_prior_grid();
    const int ch = blockIdx.z;
    const int64_t HW = (int64_t)H * W;
    const int oy = blockIdx.y * kT - kR, ox = blockIdx.x * kT - kR;
    const float *a = mapA + ch * HW, *b = mapB + ch * HW, *c = mapC + ch * HW;
    {
        const int q = (int)threadIdx.x % kE, r0 = (int)threadIdx.x / kE;
        const int gx = ox + q;
        const bool col_in = gx >= 0 && gx < W;
        if (r0 < kLoadRows) {
#pragma unroll
            for (int r = r0; r < kE; r += kLoadRows) {
                const int gy = oy + r;
                const bool in = col_in && gy >= 0 && gy < H;
                const int64_t o = (int64_t)gy * W + gx;
                sm[0][r][q] = in ? __ldg(a + o) : 0.f;
                sm[1][r][q] = in ? __ldg(b + o) : 0.f;
                sm[2][r][q] = in ? __ldg(c + o) : 0.f;
            }
        }
    }
    __syncthreads();
    for (int it = threadIdx.x; it < kHItems; it += kLossThreads) {
        const int r = it / kSeg, c0 = (it % kSeg) * kV;
        float s0[kV], s1[kV], s2[kV];
#pragma unroll
        for (int v = 0; v < kV; ++v) s0[v] = s1[v] = s2[v] = 0.f;
#pragma unroll
        for (int q = 0; q < kV + 10; ++q) {
            const float m0 = sm[0][r][c0 + q], m1 = sm[1][r][c0 + q], m2 = sm[2][r][c0 + q];
#pragma unroll
            for (int v = 0; v < kV; ++v) {
                const int t = q - v;
                if (t >= 0 && t < 11) {
                    const float w = win.w[t];
                    s0[v] += w * m0; s1[v] += w * m1; s2[v] += w * m2;
                }
            }
        }
#pragma unroll
        for (int v = 0; v < kV; ++v) { h[0][r][c0 + v] = s0[v]; h[1][r][c0 + v] = s1[v]; h[2][r][c0 + v] = s2[v]; }
    }
    __syncthreads();
    const float invN = 1.f / (3.f * (float)HW);
    const int cc = threadIdx.x % kT, r0 = (threadIdx.x / kT) * kV;
    float s0[kV], s1[kV], s2[kV];
#pragma unroll
    for (int v = 0; v < kV; ++v) s0[v] = s1[v] = s2[v] = 0.f;
#pragma unroll
    for (int q = 0; q < kV + 10; ++q) {
        const float h0 = h[0][r0 + q][cc], h1 = h[1][r0 + q][cc], h2 = h[2][r0 + q][cc];
#pragma unroll
        for (int v = 0; v < kV; ++v) {
            const int t = q - v;
            if (t >= 0 && t < 11) {
                const float w = win.w[t];
                s0[v] += w * h0; s1[v] += w * h1; s2[v] += w * h2;
            }
        }
    }
#pragma unroll
    for (int v = 0; v < kV; ++v) {
        const int gy = blockIdx.y * kT + r0 + v, gx = blockIdx.x * kT + cc;
        if (gy >= H || gx >= W) continue;
        const int64_t p = ch * HW + (int64_t)gy * W + gx;
        const float xv = __ldg(img + p), yv = __ldg(gt + p);
        const float d = xv - yv;
        const float sg = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
        const float dssim = s0[v] + 2.f * xv * s1[v] + yv * s2[v];
        const float g = ((1.f - lambda) * sg - lambda * dssim) * invN;
        if (!isfinite(g)) atomicOr(&g_loss_flags, GS_FLAG_NONFINITE);
        dl[p] = g;
    }
}

// ---- PSNR ----
constexpr int kPsnrThreads = 256;
constexpr int kPsnrBlocks = 64;  // partial sums per image

__global__ void __launch_bounds__(kPsnrThreads) k_psnr_partial(const float *__restrict__ img,
                                                              const float *__restrict__ gt, int64_t N,
                                                              float *__restrict__ part) {
    __shared__ float red[kPsnrThreads / 32];
    const int s = blockIdx.y;
    const float *x = img + s * N, *y = gt + s * N;
    float acc = 0.f;
    for (int64_t k = (int64_t)blockIdx.x * kPsnrThreads + threadIdx.x; k < N; k += (int64_t)kPsnrBlocks * kPsnrThreads) {
        float v = fminf(fmaxf(__ldg(x + k), 0.f), 1.f) - __ldg(y + k);
        acc += v * v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float a = 0.f;
        for (int w = 0; w < kPsnrThreads / 32; ++w) a += red[w];
        part[(int64_t)s * kPsnrBlocks + blockIdx.x] = a;
    }
}

__global__ void k_psnr_final(const float *__restrict__ part, int64_t N, float *__restrict__ psnr) {
    const int s = blockIdx.x;
    if (threadIdx.x != 0) return;
    double se = 0.0;
    for (int b = 0; b < kPsnrBlocks; ++b) se += (double)part[(int64_t)s * kPsnrBlocks + b];
    double mse = se / (double)N;
    if (mse < 1e-10) mse = 1e-10;
    psnr[s] = (float)(10.0 * log10(1.0 / mse));
}

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct LossGrid {
    dim3 grid;
    int nparts;
};

inline LossGrid loss_grid(int H, int W) {
    LossGrid g;
    g.grid = dim3((unsigned)((W + kT - 1) / kT), (unsigned)((H + kT - 1) / kT), 3);
    g.nparts = (int)(g.grid.x * g.grid.y * g.grid.z);
    return g;
}

Win make_window() {
    Win w;
    double g[11], s = 0.0;
    for (int i = 0; i < 11; ++i) {
        g[i] = exp(-(double)((i - 5) * (i - 5)) / (2.0 * 1.5 * 1.5));
        s += g[i];
    }
    for (int i = 0; i < 11; ++i) w.w[i] = (float)(g[i] / s);
    return w;
}

}  // namespace

uint32_t take_loss_flags() {
    uint32_t f = 0, z = 0;
    cudaMemcpyFromSymbol(&f, g_loss_flags, sizeof(f));
    cudaMemcpyToSymbol(g_loss_flags, &z, sizeof(z));
    return f;
}

}  // namespace gs

using namespace gs;

extern "C" size_t gs_loss_workspace_bytes(int32_t H, int32_t W) {
    if (H <= 0 || W <= 0) return 0;
    size_t maps = 3 * (size_t)3 * H * W * sizeof(float);
    return align256(maps) + align256(sizeof(float2) * (size_t)loss_grid(H, W).nparts) + 256;
}

extern "C" int gs_loss(const float *image, const float *gt, int32_t H, int32_t W, float lambda, void *ws,
                       size_t ws_bytes, float *loss_dev, float *dl_dimage, gs_stream_t stream) {
    if (H <= 0 || W <= 0 || H > 16384 || W > 16384 || !(lambda >= 0.f && lambda <= 1.f)) return GS_ERR_INVALID_ARG;
    if (!image || !gt || !ws || !loss_dev || !dl_dimage) return GS_ERR_INVALID_ARG;
    if (ws_bytes < gs_loss_workspace_bytes(H, W) || (reinterpret_cast<uintptr_t>(ws) & 255)) return GS_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    const int64_t HW = (int64_t)H * W;
    float *mapA = static_cast<float *>(ws);
    float *mapB = mapA + 3 * HW, *mapC = mapB + 3 * HW;
    float2 *part = reinterpret_cast<float2 *>(static_cast<char *>(ws) + align256(9 * (size_t)HW * sizeof(float)));
    LossGrid g = loss_grid(H, W);
    unsigned int *done = reinterpret_cast<unsigned int *>(reinterpret_cast<char *>(part) +
                                                          align256(sizeof(float2) * (size_t)g.nparts));
    Win win = make_window();
    if (cudaMemsetAsync(done, 0, sizeof(unsigned int), s) != cudaSuccess) return GS_ERR_CUDA;
    launch_chained(k_ssim_fwd, g.grid, kLossThreads, s, image, gt, H, W, win, mapA, mapB, mapC, part, done, lambda,
                   loss_dev);
    launch_chained(k_ssim_bwd, g.grid, kLossThreads, s, image, gt, H, W, win, lambda, mapA, mapB, mapC, dl_dimage);
    note_launches(2);
    return launch_status();
}

extern "C" size_t gs_psnr_workspace_bytes(int32_t S, int32_t H, int32_t W) {
    (void)H; (void)W;
    if (S <= 0) return 0;
    return align256(sizeof(float) * (size_t)S * kPsnrBlocks);
}

extern "C" int gs_psnr(const float *images, const float *gts, int32_t S, int32_t H, int32_t W, void *ws,
                       size_t ws_bytes, float *psnr_dev, gs_stream_t stream) {
    if (S < 0 || H <= 0 || W <= 0) return GS_ERR_INVALID_ARG;
    if (S == 0) return GS_OK;
    if (!images || !gts || !ws || !psnr_dev || ws_bytes < gs_psnr_workspace_bytes(S, H, W)) return GS_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    const int64_t N = 3 * (int64_t)H * W;
    float *part = static_cast<float *>(ws);
    k_psnr_partial<<<dim3(kPsnrBlocks, (unsigned)S), kPsnrThreads, 0, s>>>(images, gts, N, part);
    k_psnr_final<<<(unsigned)S, 32, 0, s>>>(part, N, psnr_dev);
    note_launches(2);
    return launch_status();
}
