// Freeze map and active list (Sec. 3.2.1, Eqs. 4-6) and Adam restricted to
// the unfrozen Gaussians (Sec. 3.2.4).
//
// The freeze update is a stream compaction: each Gaussian's new state is
// decided in place, per-block counts are scanned, and the unfrozen indices
// are written in ascending order. Adam then runs over that compacted list
// only; with the 256-byte parameter rows, every active Gaussian is 15 whole
// 16-byte vectors of P, G, m and v, so the traffic is proportional to the
// number of unfrozen Gaussians whatever the freeze pattern.
#include <algorithm>

#include "common.cuh"

namespace gs {
namespace {

constexpr int kFB = 1024;  // Gaussians per freeze block

__device__ __forceinline__ bool decide(int mode, uint8_t fr, float ax, float ar, int32_t c, float ex, float er) {
    if (mode == 1) return false;
    if (fr) return true;
    if (mode == 0 && c > 0) {
        float cf = (float)c;
        return __fdiv_rn(ax, cf) < ex && __fdiv_rn(ar, cf) < er;
    }
    return false;
}

__global__ void __launch_bounds__(kFB) k_freeze_mark(int64_t n, float *__restrict__ acc_xyz,
                                                    float *__restrict__ acc_rgb, int32_t *__restrict__ cnt,
                                                    uint8_t *__restrict__ frozen, float ex, float er, int mode,
                                                    int32_t *__restrict__ part) {
    int64_t i = (int64_t)blockIdx.x * kFB + threadIdx.x;
    int active = 0;
    if (i < n) {
        bool f = decide(mode, frozen[i], acc_xyz[i], acc_rgb[i], cnt[i], ex, er);
        frozen[i] = f ? 1 : 0;
        if (mode != 3) {  // 3: list only, the statistics are kept
            acc_xyz[i] = 0.f;
            acc_rgb[i] = 0.f;
            cnt[i] = 0;
        }
        active = !f;
    }
    int c = __syncthreads_count(active);
    if (threadIdx.x == 0) part[blockIdx.x] = c;
}

__global__ void __launch_bounds__(1024) k_freeze_scan(int32_t *__restrict__ part, int nb,
                                                      int32_t *__restrict__ n_active) {
    __shared__ int ws[32];
    int carry = 0;
    for (int base = 0; base < nb; base += 1024) {
        int j = base + threadIdx.x;
        int v = j < nb ? part[j] : 0, tot;
        int ex = block_exclusive_scan(v, ws, &tot);
        if (j < nb) part[j] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) *n_active = carry;
}

__global__ void __launch_bounds__(kFB) k_freeze_emit(int64_t n, const uint8_t *__restrict__ frozen,
                                                    const int32_t *__restrict__ part, int32_t *__restrict__ act) {
    __shared__ int ws[32];
    int64_t i = (int64_t)blockIdx.x * kFB + threadIdx.x;
    int a = (i < n) && !frozen[i];
    int tot;
    int r = block_exclusive_scan(a, ws, &tot);
    if (a) act[part[blockIdx.x] + r] = (int32_t)i;
}

// Freezes every Gaussian whose predicted probability exceeds tau (the map
// only grows); the gradient statistics are left to the rule.
__global__ void __launch_bounds__(kFB) k_freeze_mark_pred(int64_t n, const float *__restrict__ prob, float tau,
                                                         uint8_t *__restrict__ frozen, int32_t *__restrict__ part) {
    int64_t i = (int64_t)blockIdx.x * kFB + threadIdx.x;
    int active = 0;
    if (i < n) {
        const bool f = frozen[i] || prob[i] > tau;
        frozen[i] = f ? 1 : 0;
        active = !f;
    }
    int c = __syncthreads_count(active);
    if (threadIdx.x == 0) part[blockIdx.x] = c;
}

// ---- Ablation strategies (Sec. 5, "Freezing strategies" and "Gradient
// information"): which eligible Gaussians (unfrozen, seen in the window) an
// update freezes. ----

// Radix-select state: the 64-bit key of rank k - 1 among the eligible
// (score bits << 32 | index), found one 8-bit digit per pass.
struct SelState {
    unsigned long long prefix;  // digits chosen so far
    unsigned long long m;       // eligible count
    long long k;                // how many to freeze
    long long r;                // rank still to find inside the current prefix
};

constexpr unsigned long long kNoKey = ~0ull;

// Average gradient norm over the window, as the Eq. 4 rule reads it.
__device__ __forceinline__ float window_avg(float acc, int32_t c) { return __fdiv_rn(acc, (float)c); }

// Per Gaussian: the mingrad key (eligible only) and the eligible count.
__global__ void __launch_bounds__(kFB) k_sel_keys(int64_t n, const float *__restrict__ acc_xyz,
                                                 const float *__restrict__ acc_rgb, const int32_t *__restrict__ cnt,
                                                 const uint8_t *__restrict__ frozen, float ex, float er,
                                                 unsigned long long *__restrict__ keys, SelState *st) {
    int64_t i = (int64_t)blockIdx.x * kFB + threadIdx.x;
    int elig = 0;
    if (i < n) {
        unsigned long long key = kNoKey;
        const int32_t c = cnt[i];
        if (!frozen[i] && c > 0) {
            // score: the larger of the two averages in units of their
            // thresholds (the rule freezes exactly when it is below 1)
            const float sx = __fdiv_rn(window_avg(acc_xyz[i], c), ex);
            const float sr = __fdiv_rn(window_avg(acc_rgb[i], c), er);
            const float sc = sx > sr ? sx : sr;
            key = ((unsigned long long)__float_as_uint(sc) << 32) | (unsigned long long)i;
            elig = 1;
        }
        keys[i] = key;
    }
    const int c = __syncthreads_count(elig);
    if (threadIdx.x == 0 && c) atomicAdd(&st->m, (unsigned long long)c);
}

// Histogram of digit `shift` over the keys whose higher digits equal the
// chosen prefix.
__global__ void __launch_bounds__(1024) k_sel_hist(int64_t n, const unsigned long long *__restrict__ keys, int shift,
                                                  const SelState *st, uint32_t *__restrict__ hist) {
    __shared__ uint32_t h[256];
    for (int b = threadIdx.x; b < 256; b += blockDim.x) h[b] = 0;
    __syncthreads();
    const unsigned long long hi = shift == 56 ? 0ull : st->prefix >> (shift + 8);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long key = keys[i];
        if (key == kNoKey) continue;
        if (shift != 56 && (key >> (shift + 8)) != hi) continue;
        atomicAdd(&h[(key >> shift) & 255u], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < 256; b += blockDim.x)
        if (h[b]) atomicAdd(&hist[b], h[b]);
}

// Picks the digit holding rank r, narrows the prefix and clears the
// histogram for the next pass. At the first pass it also fixes
// k = floor(fraction * m).
__global__ void k_sel_pick(int shift, double fraction, SelState *st, uint32_t *__restrict__ hist) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = hist[threadIdx.x];
    hist[threadIdx.x] = 0;
    __syncthreads();
    if (threadIdx.x == 0) {
        if (shift == 56) {
            st->k = (long long)floor(fraction * (double)st->m);
            st->r = st->k - 1;
        }
        if (st->k > 0) {
            long long r = st->r;
            int b = 0;
            while (b < 255 && r >= (long long)h[b]) r -= h[b++];
            st->r = r;
            st->prefix |= (unsigned long long)b << shift;
        }
    }
}

// New freeze state under `strategy` (GS_FREEZE_*), statistics zeroed,
// per-block unfrozen counts.
__global__ void __launch_bounds__(kFB) k_freeze_mark_strat(int64_t n, float *__restrict__ acc_xyz,
                                                          float *__restrict__ acc_rgb, int32_t *__restrict__ cnt,
                                                          uint8_t *__restrict__ frozen, float ex, float er,
                                                          int strategy, float fraction, const float *__restrict__ u,
                                                          const unsigned long long *__restrict__ keys,
                                                          const SelState *st, int32_t *__restrict__ part) {
    int64_t i = (int64_t)blockIdx.x * kFB + threadIdx.x;
    int active = 0;
    if (i < n) {
        bool f = frozen[i] != 0;
        const int32_t c = cnt[i];
        if (!f && c > 0) {
            switch (strategy) {
                case GS_FREEZE_RULE:
                    f = window_avg(acc_xyz[i], c) < ex && window_avg(acc_rgb[i], c) < er;
                    break;
                case GS_FREEZE_XYZ: f = window_avg(acc_xyz[i], c) < ex; break;
                case GS_FREEZE_RANDOM: f = u[i] < fraction; break;
                default: f = st->k > 0 && keys[i] <= st->prefix; break;
            }
        }
        frozen[i] = f ? 1 : 0;
        acc_xyz[i] = 0.f;
        acc_rgb[i] = 0.f;
        cnt[i] = 0;
        active = !f;
    }
    int c = __syncthreads_count(active);
    if (threadIdx.x == 0) part[blockIdx.x] = c;
}

// ---- Significance pruning (Sec. 3.3, "Pruning with Significance of
// Gaussians", after LightGaussian): score_i = hits_i o_i (V_i / V_q)^beta,
// V_i = exp(s_0 + s_1 + s_2) the product of the scales, V_q the volume of
// rank floor(q n); the floor(fraction n) lowest (score, index) are marked. ----

// Keys of the volumes (all Gaussians count).
__global__ void __launch_bounds__(kFB) k_sig_vol_keys(int64_t n, const float *__restrict__ P,
                                                     unsigned long long *__restrict__ keys, SelState *st) {
    const int64_t i = (int64_t)blockIdx.x * kFB + threadIdx.x;
    if (i < n) {
        const float *r = P + i * kRow;
        const float vol = expf(r[3] + r[4] + r[5]);
        keys[i] = ((unsigned long long)__float_as_uint(vol) << 32) | (unsigned long long)i;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) st->m = (unsigned long long)n;
}

// Keys of the scores, the volume normaliser read from the first selection.
__global__ void __launch_bounds__(kFB) k_sig_score_keys(int64_t n, const float *__restrict__ P,
                                                       const uint32_t *__restrict__ hits, float beta, int abs_act,
                                                       const SelState *vq, unsigned long long *__restrict__ keys,
                                                       SelState *st) {
    const int64_t i = (int64_t)blockIdx.x * kFB + threadIdx.x;
    if (i < n) {
        const float *r = P + i * kRow;
        const float vol = expf(r[3] + r[4] + r[5]);
        const float v_q = __uint_as_float((uint32_t)(vq->prefix >> 32));
        const float o = abs_act ? fabsf(r[10]) : opacity_sigmoid(r[10]);
        const float v = v_q > 0.f ? powf(vol / v_q, beta) : 1.f;
        const float score = (float)hits[i] * o * v;
        keys[i] = ((unsigned long long)__float_as_uint(score) << 32) | (unsigned long long)i;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) st->m = (unsigned long long)n;
}

__global__ void __launch_bounds__(kFB) k_sig_mark(int64_t n, const unsigned long long *__restrict__ keys,
                                                 const SelState *st, uint8_t *__restrict__ mark) {
    const int64_t i = (int64_t)blockIdx.x * kFB + threadIdx.x;
    if (i < n) mark[i] = (st->k > 0 && keys[i] <= st->prefix) ? 1 : 0;
}

// Group rates: lr[0..5] for xyz, scale, rotation, opacity, SH DC, SH rest;
// lr[6] for float 59 (the volume-mask logit, 0 when it is not trained). The
// kernel reads them at constant indices only: indexing a parameter array by
// a run-time value makes every thread copy the whole struct to local memory.
struct AdamArgs {
    float lr[7];
    float b1, b2, eps, step_size_scale, inv_sqrt_bc2;
};

constexpr int kChunks = 15;  // 16-byte vectors per row holding the 59 parameters

// Step counter kept on the device (for CUDA-graph replay): advances it and
// stores 1 / (1 - b1^t) and 1 / sqrt(1 - b2^t) for the update that follows.
__global__ void k_adam_step(int64_t *__restrict__ step, float b1, float b2, float *__restrict__ scales) {
    const int64_t t = *step + 1;
    *step = t;
    scales[0] = (float)(1.0 / (1.0 - pow((double)b1, (double)t)));
    scales[1] = (float)(1.0 / sqrt(1.0 - pow((double)b2, (double)t)));
}

// Rate of float f (0..59) of a row from the group rates l0..l6 (see AdamArgs).
__device__ __forceinline__ float lr_of(int f, float l0, float l1, float l2, float l3, float l4, float l5,
                                       float l6) {
    return f < 3 ? l0 : f < 6 ? l1 : f < 10 ? l2 : f < 11 ? l3 : f < 14 ? l4 : f < 59 ? l5 : l6;
}

__global__ void __launch_bounds__(256) k_adam(float *__restrict__ P, const float *__restrict__ G,
                                              float *__restrict__ m, float *__restrict__ v,
                                              const int32_t *__restrict__ act, const int32_t *__restrict__ n_active,
                                              AdamArgs a, const float *__restrict__ scales,
                                              const float *__restrict__ lr_dev) {
    wait_prior_grid();
    const float step_size_scale = scales ? scales[0] : a.step_size_scale;
    const float inv_sqrt_bc2 = scales ? scales[1] : a.inv_sqrt_bc2;
    float l0 = a.lr[0], l1 = a.lr[1], l2 = a.lr[2], l3 = a.lr[3], l4 = a.lr[4], l5 = a.lr[5], l6 = a.lr[6];
    if (lr_dev) {  // group rates from device memory (changed between graph replays)
        l0 = lr_dev[0];
        l1 = lr_dev[1];
        l2 = lr_dev[2];
        l3 = lr_dev[3];
        l4 = lr_dev[4];
        l5 = lr_dev[5];
        l6 = 0.f;
    }
    const float b1 = a.b1, b2 = a.b2, eps = a.eps;
    const int64_t total = (int64_t)(*n_active) * kChunks;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = idx / kChunks;
        const int c = (int)(idx - k * kChunks);
        const int64_t off = (int64_t)act[k] * kRow + 4 * c;
        float4 p4 = *reinterpret_cast<float4 *>(P + off);
        const float4 g4 = __ldg(reinterpret_cast<const float4 *>(G + off));
        float4 m4 = *reinterpret_cast<float4 *>(m + off);
        float4 v4 = *reinterpret_cast<float4 *>(v + off);
        float pp[4] = {p4.x, p4.y, p4.z, p4.w}, gg[4] = {g4.x, g4.y, g4.z, g4.w};
        float mm[4] = {m4.x, m4.y, m4.z, m4.w}, vv[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float g = gg[e];
            mm[e] = b1 * mm[e] + (1.f - b1) * g;
            vv[e] = b2 * vv[e] + (1.f - b2) * g * g;
            const float lr = lr_of(4 * c + e, l0, l1, l2, l3, l4, l5, l6);
            pp[e] -= lr * step_size_scale * mm[e] / (sqrtf(vv[e]) * inv_sqrt_bc2 + eps);
        }
        *reinterpret_cast<float4 *>(P + off) = make_float4(pp[0], pp[1], pp[2], pp[3]);
        *reinterpret_cast<float4 *>(m + off) = make_float4(mm[0], mm[1], mm[2], mm[3]);
        *reinterpret_cast<float4 *>(v + off) = make_float4(vv[0], vv[1], vv[2], vv[3]);
    }
}

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

int g_num_sms = 0;

int num_sms() {
    if (g_num_sms == 0) {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        g_num_sms = v > 0 ? v : 152;
    }
    return g_num_sms;
}

int g_adam_per_sm = 0;

// Blocks of k_adam that fit on the GPU at once: its grid-stride loop then runs
// in a single wave, each block's share of the rows the same.
int64_t adam_grid(int64_t n) {
    if (g_adam_per_sm == 0) {
        int v = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_adam, 256, 0) != cudaSuccess || v < 1) v = 4;
        g_adam_per_sm = v;
    }
    int64_t blocks = (n * kChunks + 255) / 256;
    const int64_t cap = (int64_t)num_sms() * g_adam_per_sm;
    return blocks < cap ? blocks : cap;
}

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" size_t gs_freeze_workspace_bytes(int64_t n) {
    if (n < 0) return 0;
    int64_t nb = (n + kFB - 1) / kFB;
    return align256(sizeof(int32_t) * (size_t)(nb > 0 ? nb : 1));
}

extern "C" int gs_freeze_update(int64_t n, float *acc_xyz, float *acc_rgb, int32_t *cnt, uint8_t *frozen,
                                float eps_xyz, float eps_rgb, int32_t mode, int32_t *act, int32_t *n_active_dev,
                                void *ws, size_t ws_bytes, gs_stream_t stream) {
    if (n < 0 || n > INT32_MAX || mode < 0 || mode > 3 || !n_active_dev) return GS_ERR_INVALID_ARG;
    if (n > 0 && (!acc_xyz || !acc_rgb || !cnt || !frozen || !act)) return GS_ERR_INVALID_ARG;
    if (!ws || ws_bytes < gs_freeze_workspace_bytes(n)) return GS_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    int nb = (int)((n + kFB - 1) / kFB);
    int32_t *part = static_cast<int32_t *>(ws);
    if (nb > 0)
        k_freeze_mark<<<nb, kFB, 0, s>>>(n, acc_xyz, acc_rgb, cnt, frozen, eps_xyz, eps_rgb, mode, part);
    k_freeze_scan<<<1, 1024, 0, s>>>(part, nb, n_active_dev);
    if (nb > 0) k_freeze_emit<<<nb, kFB, 0, s>>>(n, frozen, part, act);
    note_launches(nb > 0 ? 3 : 1);
    return launch_status();
}

extern "C" int gs_freeze_apply(int64_t n, const float *prob, float tau, uint8_t *frozen, int32_t *act,
                               int32_t *n_active_dev, void *ws, size_t ws_bytes, gs_stream_t stream) {
    if (n < 0 || n > INT32_MAX || !n_active_dev || !(tau >= 0.f && tau <= 1.f)) return GS_ERR_INVALID_ARG;
    if (n > 0 && (!prob || !frozen || !act)) return GS_ERR_INVALID_ARG;
    if (!ws || ws_bytes < gs_freeze_workspace_bytes(n)) return GS_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    int nb = (int)((n + kFB - 1) / kFB);
    int32_t *part = static_cast<int32_t *>(ws);
    if (nb > 0) k_freeze_mark_pred<<<nb, kFB, 0, s>>>(n, prob, tau, frozen, part);
    k_freeze_scan<<<1, 1024, 0, s>>>(part, nb, n_active_dev);
    if (nb > 0) k_freeze_emit<<<nb, kFB, 0, s>>>(n, frozen, part, act);
    note_launches(nb > 0 ? 3 : 1);
    return launch_status();
}

namespace {
// Workspace of gs_freeze_select: block counts | selection state | histogram
// | keys [n].
struct SelLayout {
    size_t part, state, hist, keys, total;
};

SelLayout sel_layout(int64_t n) {
    SelLayout L;
    const int64_t nb = (n + kFB - 1) / kFB;
    L.part = 0;
    L.state = align256(sizeof(int32_t) * (size_t)(nb > 0 ? nb : 1));
    L.hist = L.state + 256;
    L.keys = L.hist + align256(256 * sizeof(uint32_t));
    L.total = L.keys + align256(sizeof(unsigned long long) * (size_t)(n > 0 ? n : 1));
    return L;
}
}  // namespace

extern "C" size_t gs_freeze_select_workspace_bytes(int64_t n) {
    if (n < 0 || n > INT32_MAX) return 0;
    return sel_layout(n).total;
}

extern "C" int gs_freeze_select(int64_t n, float *acc_xyz, float *acc_rgb, int32_t *cnt, uint8_t *frozen,
                                float eps_xyz, float eps_rgb, int32_t strategy, float fraction, const float *u,
                                int32_t *act, int32_t *n_active_dev, void *ws, size_t ws_bytes, gs_stream_t stream) {
    if (n < 0 || n > INT32_MAX || !n_active_dev || strategy < GS_FREEZE_RULE || strategy > GS_FREEZE_MINGRAD)
        return GS_ERR_INVALID_ARG;
    if (n > 0 && (!acc_xyz || !acc_rgb || !cnt || !frozen || !act)) return GS_ERR_INVALID_ARG;
    if ((strategy == GS_FREEZE_RANDOM || strategy == GS_FREEZE_MINGRAD) && !(fraction >= 0.f && fraction <= 1.f))
        return GS_ERR_INVALID_ARG;
    if (strategy == GS_FREEZE_RANDOM && n > 0 && !u) return GS_ERR_INVALID_ARG;
    if (strategy == GS_FREEZE_MINGRAD && !(eps_xyz > 0.f && eps_rgb > 0.f)) return GS_ERR_INVALID_ARG;
    const SelLayout L = sel_layout(n);
    if (!ws || ws_bytes < L.total || (reinterpret_cast<uintptr_t>(ws) & 255)) return GS_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    char *w = static_cast<char *>(ws);
    int32_t *part = reinterpret_cast<int32_t *>(w + L.part);
    SelState *st = reinterpret_cast<SelState *>(w + L.state);
    uint32_t *hist = reinterpret_cast<uint32_t *>(w + L.hist);
    unsigned long long *keys = reinterpret_cast<unsigned long long *>(w + L.keys);
    const int nb = (int)((n + kFB - 1) / kFB);
    int launches = nb > 0 ? 3 : 1;
    if (strategy == GS_FREEZE_MINGRAD && nb > 0) {
        if (cudaMemsetAsync(w + L.state, 0, L.keys - L.state, s) != cudaSuccess) return GS_ERR_CUDA;
        k_sel_keys<<<nb, kFB, 0, s>>>(n, acc_xyz, acc_rgb, cnt, frozen, eps_xyz, eps_rgb, keys, st);
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int hb = (int)std::min<int64_t>(nb, 2 * (int64_t)(sms > 0 ? sms : 152));
        for (int shift = 56; shift >= 0; shift -= 8) {
            k_sel_hist<<<hb, 1024, 0, s>>>(n, keys, shift, st, hist);
            k_sel_pick<<<1, 256, 0, s>>>(shift, (double)fraction, st, hist);
        }
        launches += 17;
    }
    if (nb > 0)
        k_freeze_mark_strat<<<nb, kFB, 0, s>>>(n, acc_xyz, acc_rgb, cnt, frozen, eps_xyz, eps_rgb, strategy, fraction,
                                               u, keys, st, part);
    k_freeze_scan<<<1, 1024, 0, s>>>(part, nb, n_active_dev);
    if (nb > 0) k_freeze_emit<<<nb, kFB, 0, s>>>(n, frozen, part, act);
    note_launches(launches);
    return launch_status();
}

namespace {
// Radix selection of the key of rank floor(fraction * m) - 1 into st.
void select_rank(int64_t n, const unsigned long long *keys, double fraction, SelState *st, uint32_t *hist,
                 cudaStream_t s) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t nb = (n + kFB - 1) / kFB;
    const int hb = (int)std::min<int64_t>(nb, 2 * (int64_t)(sms > 0 ? sms : 152));
    for (int shift = 56; shift >= 0; shift -= 8) {
        k_sel_hist<<<hb, 1024, 0, s>>>(n, keys, shift, st, hist);
        k_sel_pick<<<1, 256, 0, s>>>(shift, fraction, st, hist);
    }
    note_launches(16);
}

struct SigLayout {
    size_t st1, st2, hist, keys, total;
};

SigLayout sig_layout(int64_t n) {
    SigLayout L;
    L.st1 = 0;
    L.st2 = 256;
    L.hist = 512;
    L.keys = L.hist + align256(256 * sizeof(uint32_t));
    L.total = L.keys + align256(sizeof(unsigned long long) * (size_t)(n > 0 ? n : 1));
    return L;
}
}  // namespace

extern "C" size_t gs_significance_workspace_bytes(int64_t n) {
    if (n < 0 || n > INT32_MAX) return 0;
    return sig_layout(n).total;
}

extern "C" int gs_significance_mark(int64_t n, const float *P, const uint32_t *hits, int32_t opacity_act,
                                    float beta, float quantile, float fraction, uint8_t *mark, void *ws,
                                    size_t ws_bytes, gs_stream_t stream) {
    if (n < 0 || n > INT32_MAX || !(beta >= 0.f) || !(quantile > 0.f && quantile <= 1.f) ||
        !(fraction >= 0.f && fraction <= 1.f) || (opacity_act & ~(GS_OPACITY_ABS | GS_VOLUME_MASK)))
        return GS_ERR_INVALID_ARG;
    if (n == 0) return GS_OK;
    if (!P || !hits || !mark) return GS_ERR_INVALID_ARG;
    const SigLayout L = sig_layout(n);
    if (!ws || ws_bytes < L.total || (reinterpret_cast<uintptr_t>(ws) & 255)) return GS_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    char *w = static_cast<char *>(ws);
    SelState *st1 = reinterpret_cast<SelState *>(w + L.st1), *st2 = reinterpret_cast<SelState *>(w + L.st2);
    uint32_t *hist = reinterpret_cast<uint32_t *>(w + L.hist);
    unsigned long long *keys = reinterpret_cast<unsigned long long *>(w + L.keys);
    if (cudaMemsetAsync(w, 0, L.keys, s) != cudaSuccess) return GS_ERR_CUDA;
    const int nb = (int)((n + kFB - 1) / kFB);
    k_sig_vol_keys<<<nb, kFB, 0, s>>>(n, P, keys, st1);
    select_rank(n, keys, (double)quantile, st1, hist, s);
    k_sig_score_keys<<<nb, kFB, 0, s>>>(n, P, hits, beta, opacity_act & GS_OPACITY_ABS, st1, keys, st2);
    select_rank(n, keys, (double)fraction, st2, hist, s);
    k_sig_mark<<<nb, kFB, 0, s>>>(n, keys, st2, mark);
    note_launches(3);
    return launch_status();
}

extern "C" int gs_adam_masked_groups(float *P, const float *G, float *m, float *v, int64_t n, const int32_t *act,
                                     const int32_t *n_active_dev, const float *lr, int32_t n_groups, float b1,
                                     float b2, float eps, int64_t step, gs_stream_t stream) {
    if (n < 0 || step < 1 || !lr || !n_active_dev || (n_groups != 6 && n_groups != 7)) return GS_ERR_INVALID_ARG;
    if (!(b1 >= 0.f && b1 < 1.f) || !(b2 >= 0.f && b2 < 1.f) || !(eps >= 0.f)) return GS_ERR_INVALID_ARG;
    if (n == 0) return GS_OK;
    if (!P || !G || !m || !v || !act) return GS_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(P) | reinterpret_cast<uintptr_t>(G) | reinterpret_cast<uintptr_t>(m) |
         reinterpret_cast<uintptr_t>(v)) & 15)
        return GS_ERR_INVALID_ARG;
    AdamArgs a;
    for (int k = 0; k < 6; ++k) a.lr[k] = lr[k];
    a.lr[6] = n_groups == 7 ? lr[6] : 0.f;  // the volume-mask logit
    double bc1 = 1.0 - pow((double)b1, (double)step), bc2 = 1.0 - pow((double)b2, (double)step);
    a.b1 = b1;
    a.b2 = b2;
    a.eps = eps;
    a.step_size_scale = (float)(1.0 / bc1);
    a.inv_sqrt_bc2 = (float)(1.0 / sqrt(bc2));
    const int64_t blocks = adam_grid(n);
    launch_chained(k_adam, (unsigned)blocks, 256, as_stream(stream), P, G, m, v, act, n_active_dev, a,
                   static_cast<float *>(nullptr), static_cast<float *>(nullptr));
    note_launches(1);
    return launch_status();
}

extern "C" int gs_adam_masked(float *P, const float *G, float *m, float *v, int64_t n, const int32_t *act,
                              const int32_t *n_active_dev, const float *lr, float b1, float b2, float eps,
                              int64_t step, gs_stream_t stream) {
    return gs_adam_masked_groups(P, G, m, v, n, act, n_active_dev, lr, 6, b1, b2, eps, step, stream);
}

extern "C" int gs_adam_masked_devstep(float *P, const float *G, float *m, float *v, int64_t n, const int32_t *act,
                                      const int32_t *n_active_dev, const float *lr_dev, float b1, float b2, float eps,
                                      int64_t *step_dev, float *scratch_dev, gs_stream_t stream) {
    if (n < 0 || !lr_dev || !n_active_dev || !step_dev || !scratch_dev) return GS_ERR_INVALID_ARG;
    if (!(b1 >= 0.f && b1 < 1.f) || !(b2 >= 0.f && b2 < 1.f) || !(eps >= 0.f)) return GS_ERR_INVALID_ARG;
    if (n == 0) return GS_OK;
    if (!P || !G || !m || !v || !act) return GS_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(P) | reinterpret_cast<uintptr_t>(G) | reinterpret_cast<uintptr_t>(m) |
         reinterpret_cast<uintptr_t>(v)) & 15)
        return GS_ERR_INVALID_ARG;
    AdamArgs a;
    for (int k = 0; k < 7; ++k) a.lr[k] = 0.f;  // taken from lr_dev on the device
    a.b1 = b1;
    a.b2 = b2;
    a.eps = eps;
    a.step_size_scale = 1.f;
    a.inv_sqrt_bc2 = 1.f;
    cudaStream_t s = as_stream(stream);
    k_adam_step<<<1, 1, 0, s>>>(step_dev, b1, b2, scratch_dev);
    const int64_t blocks = adam_grid(n);
    k_adam<<<(unsigned)blocks, 256, 0, s>>>(P, G, m, v, act, n_active_dev, a, scratch_dev, lr_dev);
    note_launches(2);
    return launch_status();
}

// ---------------------------------------------------------------------------
// gs_freeze_update_noalloc: the same freeze update with its scratch (one count
// per block of 1024 Gaussians) in a fixed array inside the library, for
// callers that cannot allocate device memory where they call it.
// ---------------------------------------------------------------------------
#include <cuda.h>  // CUcontext / CUresult types; the two driver calls are fetched through the runtime

#include <mutex>

namespace gs {
namespace {

constexpr int kNoAllocBlocks = 65536;  // 256 KB of counts: n <= 65536 * 1024
static __device__ __align__(256) int32_t g_freeze_scratch[kNoAllocBlocks];

constexpr int kMaxDevices = 256;
std::mutex g_scratch_mu;
int32_t *g_scratch_ptr[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};

typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);

// Id of the context current on this thread, 0 if it cannot be read. A device
// reset replaces the primary context by one with a new id, so an address
// cached under the old id is looked up again instead of being reused.
unsigned long long current_context_id() {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q;
        void *f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(f);
    });
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

// Device address of g_freeze_scratch in the current device's current context,
// looked up on the first call there (and again after a device reset; on every
// call if the context id cannot be read). Returns nullptr if the lookup fails.
int32_t *scratch_on_current_device() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    const unsigned long long id = current_context_id();
    if (!g_scratch_ptr[dev] || id == 0 || id != g_scratch_ctx[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_freeze_scratch) != cudaSuccess) return nullptr;
        g_scratch_ptr[dev] = static_cast<int32_t *>(p);
        g_scratch_ctx[dev] = current_context_id();  // the lookup made the context current if it was not
    }
    return g_scratch_ptr[dev];
}

}  // namespace
}  // namespace gs

extern "C" int gs_freeze_update_noalloc(int64_t n, float *acc_xyz, float *acc_rgb, int32_t *cnt, uint8_t *frozen,
                                        float eps_xyz, float eps_rgb, int32_t mode, int32_t *act,
                                        int32_t *n_active_dev, gs_stream_t stream) {
    if (n < 0 || n > (int64_t)kNoAllocBlocks * kFB || mode < 0 || mode > 2 || !n_active_dev)
        return GS_ERR_INVALID_ARG;
    if (n > 0 && (!acc_xyz || !acc_rgb || !cnt || !frozen || !act)) return GS_ERR_INVALID_ARG;
    int32_t *part = scratch_on_current_device();
    if (!part) return GS_ERR_CUDA;
    // Every count the scan reads is written by k_freeze_mark in the same call,
    // so nothing left in the array by an earlier call needs clearing.
    cudaStream_t s = as_stream(stream);
    int nb = (int)((n + kFB - 1) / kFB);
    if (nb > 0)
        k_freeze_mark<<<nb, kFB, 0, s>>>(n, acc_xyz, acc_rgb, cnt, frozen, eps_xyz, eps_rgb, mode, part);
    k_freeze_scan<<<1, 1024, 0, s>>>(part, nb, n_active_dev);
    if (nb > 0) k_freeze_emit<<<nb, kFB, 0, s>>>(n, frozen, part, act);
    note_launches(nb > 0 ? 3 : 1);
    return launch_status();
}
