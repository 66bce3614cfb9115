// Learned freeze predictor: per-Gaussian gradient-norm history, features,
// a 16 -> 64 -> 64 -> 1 MLP with bfloat16 weights and float32 accumulation
// (inference on tensor cores), its training gradient and Adam. The paper has
// no learned component; the predictor proposes Gaussians the gradient-norm
// rule of Sec. 3.2.1 (Eqs. 4-6) is about to freeze, so they can be frozen
// earlier. Definitions (shared with the oracle by their statement):
//
// state [n][12]: 0-3 xyz-norm EMA history (newest first), 4-7 rgb history,
//   8 xyz EMA, 9 rgb EMA, 10 visible iterations, 11 boundaries spent frozen.
//   At each statistics boundary: if cnt > 0, EMA = 0.5 EMA + 0.5 acc/cnt and
//   views += cnt; frozen count += frozen; histories shift, EMA at the front.
// features [n][16] (bf16): 0-3 / 4-7 log10(history / eps) clamped to
//   [-8, 8] (norms floored at 1e-30), 8 sigmoid(logit), 9 max and 10 min
//   log-scale, 11 ln(1 + views), 12 k / K, 13-14 log10(window average /
//   eps) (average 0 if never visible), 15 min(frozen count, 8) / 8.
// MLP: a1 = X W1 + b1, h1 = relu(a1) rounded to bf16, a2 = h1 W2 + b2,
//   h2 = relu(a2), z = h2 . W3 + b3, p = sigmoid(z). Inputs and W1, W2, W3
//   are bf16; biases and accumulation float32.
// params (float32, 5313): W1 [16][64] | b1 [64] | W2 [64][64] | b2 [64] |
//   W3 [64] | b3 [1]  (weights input-major). wb (bf16, 5184): W1 | W2 | W3.
#include <cuda_bf16.h>

#include "common.cuh"

namespace gs {
namespace {

constexpr int kIn = 16, kH = 64;
constexpr int oW1 = 0, oB1 = oW1 + kIn * kH, oW2 = oB1 + kH, oB2 = oW2 + kH * kH, oW3 = oB2 + kH, oB3 = oW3 + kH;
constexpr int kNParam = oB3 + 1;            // 5313
constexpr int kNWb = kIn * kH + kH * kH + kH;  // 5184 bf16 weights
constexpr int wbW1 = 0, wbW2 = kIn * kH, wbW3 = kIn * kH + kH * kH;

__device__ __forceinline__ float log_ratio(float v, float eps) {
    float r = log10f(fmaxf(v, 1e-30f) / eps);
    return fminf(fmaxf(r, -8.f), 8.f);
}

__global__ void k_pred_history(int64_t n, const float *__restrict__ acc_xyz, const float *__restrict__ acc_rgb,
                               const int32_t *__restrict__ cnt, const uint8_t *__restrict__ frozen,
                               float *__restrict__ state) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float *s = state + 12 * i;
    float h[12];
#pragma unroll
    for (int j = 0; j < 12; ++j) h[j] = s[j];
    const int c = cnt[i];
    if (c > 0) {
        const float cf = (float)c;
        h[8] = 0.5f * h[8] + 0.5f * (acc_xyz[i] / cf);
        h[9] = 0.5f * h[9] + 0.5f * (acc_rgb[i] / cf);
        h[10] += cf;
    }
    if (frozen && frozen[i]) h[11] += 1.f;
#pragma unroll
    for (int j = 3; j > 0; --j) {
        h[j] = h[j - 1];
        h[4 + j] = h[4 + j - 1];
    }
    h[0] = h[8];
    h[4] = h[9];
#pragma unroll
    for (int j = 0; j < 12; ++j) s[j] = h[j];
}

__global__ void k_pred_features(int64_t n, const float *__restrict__ P, const float *__restrict__ acc_xyz,
                                const float *__restrict__ acc_rgb, const int32_t *__restrict__ cnt,
                                const float *__restrict__ state, float kfrac, float ex, float er,
                                __nv_bfloat16 *__restrict__ X) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float *s = state + 12 * i;
    const float4 r0 = __ldg(reinterpret_cast<const float4 *>(P + i * kRow));
    const float4 r1 = __ldg(reinterpret_cast<const float4 *>(P + i * kRow) + 1);
    const float4 r2 = __ldg(reinterpret_cast<const float4 *>(P + i * kRow) + 2);
    float f[16];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        f[j] = log_ratio(s[j], ex);
        f[4 + j] = log_ratio(s[4 + j], er);
    }
    f[8] = 1.f / (1.f + expf(-r2.z));
    f[9] = fmaxf(r0.w, fmaxf(r1.x, r1.y));
    f[10] = fminf(r0.w, fminf(r1.x, r1.y));
    f[11] = log1pf(s[10]);
    f[12] = kfrac;
    const int c = cnt[i];
    const float ax = c > 0 ? acc_xyz[i] / (float)c : 0.f, ar = c > 0 ? acc_rgb[i] / (float)c : 0.f;
    f[13] = log_ratio(ax, ex);
    f[14] = log_ratio(ar, er);
    f[15] = fminf(s[11], 8.f) / 8.f;
    __nv_bfloat162 *out = reinterpret_cast<__nv_bfloat162 *>(X + i * kIn);
#pragma unroll
    for (int j = 0; j < 8; ++j) out[j] = __floats2bfloat162_rn(f[2 * j], f[2 * j + 1]);
}

// ---- inference: mma.sync m16n8k16 bf16 -> f32 ----
__device__ __forceinline__ void mma16816(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}

__device__ __forceinline__ uint32_t pack_raw(__nv_bfloat16 lo, __nv_bfloat16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// A fragments of one 16-row tile (rows beyond n read as zero).
__device__ __forceinline__ void load_tile(const __nv_bfloat16 *__restrict__ X, int64_t n, int64_t tile, int g, int t,
                                          uint32_t (&a)[4]) {
    const int64_t r0 = tile * 16 + g, r1 = r0 + 8;
    const uint32_t *x0 = reinterpret_cast<const uint32_t *>(X + r0 * kIn);
    const uint32_t *x1 = reinterpret_cast<const uint32_t *>(X + r1 * kIn);
    a[0] = r0 < n ? __ldg(x0 + t) : 0u;
    a[1] = r1 < n ? __ldg(x1 + t) : 0u;
    a[2] = r0 < n ? __ldg(x0 + 4 + t) : 0u;
    a[3] = r1 < n ? __ldg(x1 + 4 + t) : 0u;
}

// One warp per 16-row tile, tiles strided over the grid; each warp has the
// features of its next two tiles in flight while it computes the current
// one (the kernel is bound by reading 32 B per row). Fragment layouts of
// m16n8k16 (lane = 4 g + t): A rows g, g+8 / columns 2t, 2t+1, 2t+8, 2t+9;
// B columns g / rows 2t, 2t+1, 2t+8, 2t+9; C rows g, g+8 / columns 2t, 2t+1.
// The layer-1 accumulators of n-tiles 2s and 2s+1 are exactly the A fragment
// of layer 2's k-step s, so the hidden layer never leaves registers. Layer
// 1's B fragments and W3 stay in registers; layer 2's (64 per lane) are read
// from shared memory, packed per lane, to keep the register count low.
__global__ void __launch_bounds__(128, 4) k_mlp_fwd(int64_t n, const __nv_bfloat16 *__restrict__ X,
                                                    const __nv_bfloat16 *__restrict__ wb,
                                                    const float *__restrict__ prm, float *__restrict__ p) {
    __shared__ __nv_bfloat16 sW[kNWb];
    __shared__ float sB[kH * 2 + 1];
    __shared__ uint2 sB2[4][8][32];  // [k-step][n-tile][lane]
    for (int k = threadIdx.x; k < kNWb; k += blockDim.x) sW[k] = wb[k];
    for (int k = threadIdx.x; k < kH; k += blockDim.x) {
        sB[k] = prm[oB1 + k];
        sB[kH + k] = prm[oB2 + k];
    }
    if (threadIdx.x == 0) sB[2 * kH] = prm[oB3];
    __syncthreads();
    for (int e = threadIdx.x; e < 4 * 8 * 32; e += blockDim.x) {
        const int st = e >> 8, nt = (e >> 5) & 7, ln = e & 31;
        const int col = 8 * nt + (ln >> 2), k0 = 16 * st + 2 * (ln & 3);
        sB2[st][nt][ln] = make_uint2(pack_raw(sW[wbW2 + k0 * kH + col], sW[wbW2 + (k0 + 1) * kH + col]),
                                     pack_raw(sW[wbW2 + (k0 + 8) * kH + col], sW[wbW2 + (k0 + 9) * kH + col]));
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    uint32_t b1[8][2];
    float w3[8][2];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const int col = 8 * nt + g;
        b1[nt][0] = pack_raw(sW[wbW1 + (2 * t) * kH + col], sW[wbW1 + (2 * t + 1) * kH + col]);
        b1[nt][1] = pack_raw(sW[wbW1 + (2 * t + 8) * kH + col], sW[wbW1 + (2 * t + 9) * kH + col]);
        w3[nt][0] = __bfloat162float(sW[wbW3 + 8 * nt + 2 * t]);
        w3[nt][1] = __bfloat162float(sW[wbW3 + 8 * nt + 2 * t + 1]);
    }
    const float b3 = sB[2 * kH];
    const int64_t tiles = (n + 15) / 16;
    const int warp = threadIdx.x >> 5, warps = blockDim.x >> 5;
    const int64_t stride = (int64_t)gridDim.x * warps;
    int64_t tile = (int64_t)blockIdx.x * warps + warp;
    uint32_t a[4], na[4];
    load_tile(X, n, tile, g, t, a);
    load_tile(X, n, tile + stride, g, t, na);
    for (; tile < tiles; tile += stride) {
        uint32_t nna[4];
        load_tile(X, n, tile + 2 * stride, g, t, nna);
        uint32_t ha[4][4];  // relu(h1) as bf16 A fragments of layer 2
#pragma unroll
        for (int st = 0; st < 4; ++st) {
            float h[2][4];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int nt = 2 * st + q;
                const float c0 = sB[8 * nt + 2 * t], c1 = sB[8 * nt + 2 * t + 1];
                h[q][0] = c0; h[q][1] = c1; h[q][2] = c0; h[q][3] = c1;
                mma16816(h[q], a[0], a[1], a[2], a[3], b1[nt][0], b1[nt][1]);
            }
            ha[st][0] = pack_bf16(fmaxf(h[0][0], 0.f), fmaxf(h[0][1], 0.f));
            ha[st][1] = pack_bf16(fmaxf(h[0][2], 0.f), fmaxf(h[0][3], 0.f));
            ha[st][2] = pack_bf16(fmaxf(h[1][0], 0.f), fmaxf(h[1][1], 0.f));
            ha[st][3] = pack_bf16(fmaxf(h[1][2], 0.f), fmaxf(h[1][3], 0.f));
        }
        float z0 = 0.f, z1 = 0.f;
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const float c0 = sB[kH + 8 * nt + 2 * t], c1 = sB[kH + 8 * nt + 2 * t + 1];
            float acc[4] = {c0, c1, c0, c1};
#pragma unroll
            for (int st = 0; st < 4; ++st) {
                const uint2 bb = sB2[st][nt][lane];
                mma16816(acc, ha[st][0], ha[st][1], ha[st][2], ha[st][3], bb.x, bb.y);
            }
            z0 += fmaxf(acc[0], 0.f) * w3[nt][0] + fmaxf(acc[1], 0.f) * w3[nt][1];
            z1 += fmaxf(acc[2], 0.f) * w3[nt][0] + fmaxf(acc[3], 0.f) * w3[nt][1];
        }
        z0 += __shfl_xor_sync(kFull, z0, 1);
        z0 += __shfl_xor_sync(kFull, z0, 2);
        z1 += __shfl_xor_sync(kFull, z1, 1);
        z1 += __shfl_xor_sync(kFull, z1, 2);
        const int64_t r0 = tile * 16 + g, r1 = r0 + 8;
        if (t == 0) {
            if (r0 < n) p[r0] = 1.f / (1.f + expf(-(z0 + b3)));
            if (r1 < n) p[r1] = 1.f / (1.f + expf(-(z1 + b3)));
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            a[k] = na[k];
            na[k] = nna[k];
        }
    }
}

// ---- training gradient (float32 on CUDA cores, rows staged in shared memory) ----
constexpr int kTR = 32;  // rows per tile
constexpr int kGradThreads = 256;

struct GradSmem {
    float W1[kIn * kH], W2[kH * kH], W3[kH], b1[kH], b2[kH], b3;
    float X[kTR][kIn], a1[kTR][kH], h1[kTR][kH], a2[kTR][kH], h2[kTR][kH], dh2[kTR][kH], dh1[kTR][kH];
    float z[kTR], dz[kTR], loss[kGradThreads / 32];
};

__global__ void __launch_bounds__(kGradThreads) k_mlp_grad(int64_t n, const __nv_bfloat16 *__restrict__ X,
                                                           const float *__restrict__ y, const float *__restrict__ w,
                                                           float inv_wsum, const __nv_bfloat16 *__restrict__ wb,
                                                           const float *__restrict__ prm, float *__restrict__ grad,
                                                           float *__restrict__ loss) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    GradSmem &S = *reinterpret_cast<GradSmem *>(smem_raw);
    const int tid = threadIdx.x;
    for (int k = tid; k < kIn * kH; k += kGradThreads) S.W1[k] = __bfloat162float(wb[wbW1 + k]);
    for (int k = tid; k < kH * kH; k += kGradThreads) S.W2[k] = __bfloat162float(wb[wbW2 + k]);
    for (int k = tid; k < kH; k += kGradThreads) {
        S.W3[k] = __bfloat162float(wb[wbW3 + k]);
        S.b1[k] = prm[oB1 + k];
        S.b2[k] = prm[oB2 + k];
    }
    if (tid == 0) S.b3 = prm[oB3];
    // per-thread gradient accumulators: thread owns W2 entries tid + 256 q (16),
    // W1 entries tid + 256 q (4), and for tid < 64: b1, b2, W3 entry tid.
    float gW2[16] = {0}, gW1[4] = {0}, gb1 = 0.f, gb2 = 0.f, gW3 = 0.f, gb3 = 0.f, lsum = 0.f;
    __syncthreads();
    const int64_t tiles = (n + kTR - 1) / kTR;
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int64_t base = tile * kTR;
        for (int k = tid; k < kTR * kIn; k += kGradThreads) {
            const int r = k / kIn, c = k % kIn;
            S.X[r][c] = base + r < n ? __bfloat162float(X[(base + r) * kIn + c]) : 0.f;
        }
        __syncthreads();
        for (int k = tid; k < kTR * kH; k += kGradThreads) {  // layer 1
            const int r = k / kH, j = k % kH;
            float s = S.b1[j];
#pragma unroll
            for (int c = 0; c < kIn; ++c) s += S.X[r][c] * S.W1[c * kH + j];
            S.a1[r][j] = s;
            S.h1[r][j] = __bfloat162float(__float2bfloat16_rn(fmaxf(s, 0.f)));
        }
        __syncthreads();
        for (int k = tid; k < kTR * kH; k += kGradThreads) {  // layer 2
            const int r = k / kH, j = k % kH;
            float s = S.b2[j];
#pragma unroll 16
            for (int c = 0; c < kH; ++c) s += S.h1[r][c] * S.W2[c * kH + j];
            S.a2[r][j] = s;
            S.h2[r][j] = fmaxf(s, 0.f);
        }
        __syncthreads();
        if (tid < kTR) {  // output, loss and dL/dz
            const int r = tid;
            float z = S.b3;
            for (int j = 0; j < kH; ++j) z += S.h2[r][j] * S.W3[j];
            float dz = 0.f;
            if (base + r < n) {
                const float yy = y[base + r], wi = (w ? w[base + r] : 1.f) * inv_wsum;
                const float sp = z > 0.f ? z + log1pf(expf(-z)) : log1pf(expf(z));
                lsum += wi * (sp - yy * z);
                dz = wi * (1.f / (1.f + expf(-z)) - yy);
            }
            S.dz[r] = dz;
        }
        __syncthreads();
        for (int k = tid; k < kTR * kH; k += kGradThreads) {
            const int r = k / kH, j = k % kH;
            S.dh2[r][j] = S.a2[r][j] > 0.f ? S.dz[r] * S.W3[j] : 0.f;
        }
        __syncthreads();
        for (int k = tid; k < kTR * kH; k += kGradThreads) {
            const int r = k / kH, c = k % kH;
            float s = 0.f;
#pragma unroll 16
            for (int j = 0; j < kH; ++j) s += S.dh2[r][j] * S.W2[c * kH + j];
            S.dh1[r][c] = S.a1[r][c] > 0.f ? s : 0.f;
        }
        __syncthreads();
        // weight-gradient contributions of this tile
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int e = tid + kGradThreads * q, c = e / kH, j = e % kH;
            float s = 0.f;
            for (int r = 0; r < kTR; ++r) s += S.h1[r][c] * S.dh2[r][j];
            gW2[q] += s;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = tid + kGradThreads * q, c = e / kH, j = e % kH;
            float s = 0.f;
            for (int r = 0; r < kTR; ++r) s += S.X[r][c] * S.dh1[r][j];
            gW1[q] += s;
        }
        if (tid < kH) {
            float s1 = 0.f, s2 = 0.f, s3 = 0.f;
            for (int r = 0; r < kTR; ++r) {
                s1 += S.dh1[r][tid];
                s2 += S.dh2[r][tid];
                s3 += S.dz[r] * S.h2[r][tid];
            }
            gb1 += s1; gb2 += s2; gW3 += s3;
        }
        if (tid == 0)
            for (int r = 0; r < kTR; ++r) gb3 += S.dz[r];
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) atomicAdd(grad + oW2 + tid + kGradThreads * q, gW2[q]);
#pragma unroll
    for (int q = 0; q < 4; ++q) atomicAdd(grad + oW1 + tid + kGradThreads * q, gW1[q]);
    if (tid < kH) {
        atomicAdd(grad + oB1 + tid, gb1);
        atomicAdd(grad + oB2 + tid, gb2);
        atomicAdd(grad + oW3 + tid, gW3);
    }
    if (tid == 0) atomicAdd(grad + oB3, gb3);
    if (loss && tid < kTR) {
        float l = lsum;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(kFull, l, o);
        if (tid == 0) atomicAdd(loss, l);
    }
}

__global__ void k_mlp_adam(float *__restrict__ prm, const float *__restrict__ grad, float *__restrict__ m,
                           float *__restrict__ v, __nv_bfloat16 *__restrict__ wb, float lr, float b1, float b2,
                           float eps, float inv_bc1, float inv_sqrt_bc2) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= kNParam) return;
    const float g = grad[k];
    const float mm = b1 * m[k] + (1.f - b1) * g, vv = b2 * v[k] + (1.f - b2) * g * g;
    m[k] = mm;
    v[k] = vv;
    const float p = prm[k] - lr * (mm * inv_bc1) / (sqrtf(vv) * inv_sqrt_bc2 + eps);
    prm[k] = p;
    int o = -1;  // position of this parameter among the bf16 weights
    if (k < oB1) o = wbW1 + (k - oW1);
    else if (k >= oW2 && k < oB2) o = wbW2 + (k - oW2);
    else if (k >= oW3 && k < oB3) o = wbW3 + (k - oW3);
    if (o >= 0) wb[o] = __float2bfloat16_rn(p);
}

__global__ void k_mlp_refresh(const float *__restrict__ prm, __nv_bfloat16 *__restrict__ wb) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= kNParam) return;
    int o = -1;
    if (k < oB1) o = wbW1 + (k - oW1);
    else if (k >= oW2 && k < oB2) o = wbW2 + (k - oW2);
    else if (k >= oW3 && k < oB3) o = wbW3 + (k - oW3);
    if (o >= 0) wb[o] = __float2bfloat16_rn(prm[k]);
}

int g_sms = 0;
int sms() {
    if (!g_sms) {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        g_sms = v > 0 ? v : 152;
    }
    return g_sms;
}

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" int gs_pred_history(int64_t n, const float *acc_xyz, const float *acc_rgb, const int32_t *cnt,
                               const uint8_t *frozen, float *state, gs_stream_t stream) {
    if (n < 0) return GS_ERR_INVALID_ARG;
    if (n == 0) return GS_OK;
    if (!acc_xyz || !acc_rgb || !cnt || !state) return GS_ERR_INVALID_ARG;
    k_pred_history<<<grid_for(n, 256), 256, 0, as_stream(stream)>>>(n, acc_xyz, acc_rgb, cnt, frozen, state);
    note_launches(1);
    return launch_status();
}

extern "C" int gs_pred_features(int64_t n, const float *P, const float *acc_xyz, const float *acc_rgb,
                                const int32_t *cnt, const float *state, int32_t k, int32_t K, float eps_xyz,
                                float eps_rgb, uint16_t *X, gs_stream_t stream) {
    if (n < 0 || K <= 0 || !(eps_xyz > 0.f) || !(eps_rgb > 0.f)) return GS_ERR_INVALID_ARG;
    if (n == 0) return GS_OK;
    if (!P || !acc_xyz || !acc_rgb || !cnt || !state || !X) return GS_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(P) & 15) || (reinterpret_cast<uintptr_t>(X) & 3)) return GS_ERR_INVALID_ARG;
    k_pred_features<<<grid_for(n, 256), 256, 0, as_stream(stream)>>>(
        n, P, acc_xyz, acc_rgb, cnt, state, (float)k / (float)K, eps_xyz, eps_rgb,
        reinterpret_cast<__nv_bfloat16 *>(X));
    note_launches(1);
    return launch_status();
}

extern "C" int gs_mlp_fwd(int64_t n, const uint16_t *X, const uint16_t *wb, const float *params, float *p,
                          gs_stream_t stream) {
    if (n < 0) return GS_ERR_INVALID_ARG;
    if (n == 0) return GS_OK;
    if (!X || !wb || !params || !p || (reinterpret_cast<uintptr_t>(X) & 3)) return GS_ERR_INVALID_ARG;
    const int64_t tiles = (n + 15) / 16;
    int64_t blocks = (tiles + 3) / 4;
    if (blocks > (int64_t)sms() * 4) blocks = (int64_t)sms() * 4;  // one resident wave
    k_mlp_fwd<<<(unsigned)blocks, 128, 0, as_stream(stream)>>>(n, reinterpret_cast<const __nv_bfloat16 *>(X),
                                                               reinterpret_cast<const __nv_bfloat16 *>(wb), params, p);
    note_launches(1);
    return launch_status();
}

extern "C" int gs_mlp_grad(int64_t n, const uint16_t *X, const float *y, const float *w, float inv_wsum,
                           const uint16_t *wb, const float *params, float *grad, float *loss_dev, gs_stream_t stream) {
    if (n < 0 || !(inv_wsum > 0.f)) return GS_ERR_INVALID_ARG;
    if (n == 0) return GS_OK;
    if (!X || !y || !wb || !params || !grad) return GS_ERR_INVALID_ARG;
    if (cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(GradSmem)) !=
        cudaSuccess)
        return GS_ERR_CUDA;
    const int64_t tiles = (n + kTR - 1) / kTR;
    int64_t blocks = tiles < (int64_t)sms() * 2 ? tiles : (int64_t)sms() * 2;
    k_mlp_grad<<<(unsigned)blocks, kGradThreads, sizeof(GradSmem), as_stream(stream)>>>(
        n, reinterpret_cast<const __nv_bfloat16 *>(X), y, w, inv_wsum, reinterpret_cast<const __nv_bfloat16 *>(wb),
        params, grad, loss_dev);
    note_launches(1);
    return launch_status();
}

extern "C" int gs_mlp_adam(float *params, const float *grad, float *m, float *v, uint16_t *wb, float lr, float b1,
                           float b2, float eps, int64_t step, gs_stream_t stream) {
    if (!params || !grad || !m || !v || !wb || step < 1 || !(lr >= 0.f) || !(b1 >= 0.f && b1 < 1.f) ||
        !(b2 >= 0.f && b2 < 1.f) || !(eps >= 0.f))
        return GS_ERR_INVALID_ARG;
    const double bc1 = 1.0 - pow((double)b1, (double)step), bc2 = 1.0 - pow((double)b2, (double)step);
    k_mlp_adam<<<grid_for(kNParam, 256), 256, 0, as_stream(stream)>>>(
        params, grad, m, v, reinterpret_cast<__nv_bfloat16 *>(wb), lr, b1, b2, eps, (float)(1.0 / bc1),
        (float)(1.0 / sqrt(bc2)));
    note_launches(1);
    return launch_status();
}

extern "C" int gs_mlp_refresh(const float *params, uint16_t *wb, gs_stream_t stream) {
    if (!params || !wb) return GS_ERR_INVALID_ARG;
    k_mlp_refresh<<<grid_for(kNParam, 256), 256, 0, as_stream(stream)>>>(params,
                                                                        reinterpret_cast<__nv_bfloat16 *>(wb));
    note_launches(1);
    return launch_status();
}
