// Adaptive densification, pruning and opacity reset.
//
// The paper keeps 3DGS's densification and changes its thresholds and
// cadence (Sec. 4.1); the clone / split / prune rules are 3DGS's:
//   candidate : the window's average |dL/dmean2d| (NDC units) >= eps_xyz,
//               or, on a diffuse-colour step, average |dL/dk0| >= eps_rgb;
//   clone     : a candidate whose largest log-scale <= log_clone_max
//               (an identical copy is appended);
//   split     : any other candidate: two children at mean + R(q)(s * z_k),
//               z_k ~ N(0, I3) given by the caller, log-scales minus
//               log_split_div, all else copied; the original is removed;
//   prune     : logit(opacity) < logit_min_opacity (originals, clones and
//               children); with prune_big also largest screen radius >
//               max_screen_radius (originals) and largest log-scale >
//               log_max_world (all).
// Output rows: surviving originals in index order, then surviving clones,
// then surviving children (two per split original, child 0 first), in the
// order of their originals. New Gaussians get zero Adam moments, are not
// frozen, and zero carried state. All comparisons in float32, thresholds in
// the log / logit domain.
#include "common.cuh"

namespace gs {
namespace {

constexpr int kDB = 256;  // Gaussians per block

// flag bits
constexpr uint8_t kKeep = 1, kClone = 2, kSplit = 4, kChild = 8;

__device__ __forceinline__ uint8_t den_flags(const float *__restrict__ P, const gs_grad_stats st,
                                             const gs_densify_params &p, int64_t i) {
    const float *r = P + i * kRow;
    const int32_t c = st.cnt[i];
    bool cand = false;
    if (c > 0) {
        const float fc = (float)c;
        const float ax = __fdiv_rn(st.acc_xyz[i], fc), ar = __fdiv_rn(st.acc_rgb[i], fc);
        cand = ax >= p.eps_xyz || (p.use_rgb && ar >= p.eps_rgb);
    }
    const float smax = fmaxf(fmaxf(r[3], r[4]), r[5]);
    const bool clone = cand && smax <= p.log_clone_max;
    const bool split = cand && !clone;
    // low opacity, or a volume mask that is off (its logit at most logit(0.01))
    const bool low = r[10] < p.logit_min_opacity || (p.mask_prune && !(r[59] > p.mask_logit_min)) ||
                     (p.prune_mark && p.prune_mark[i]);
    bool big_world = false, big_child = false, big_screen = false;
    if (p.prune_big) {
        big_world = smax > p.log_max_world;
        big_child = __fsub_rn(smax, p.log_split_div) > p.log_max_world;
        big_screen = st.max_radius && st.max_radius[i] > p.max_screen_radius;
    }
    uint8_t f = 0;
    if (!split && !low && !big_world && !big_screen) f |= kKeep;
    if (clone && !low && !big_world) f |= kClone;
    if (split) f |= kSplit;
    if (split && !low && !big_child) f |= kChild;
    return f;
}

struct Quad {  // four counts: kept originals, kept clones, splits, split originals with kept children
    uint32_t v[4];
};

__device__ __forceinline__ Quad quad_of(uint8_t f) {
    return Quad{{(uint32_t)((f & kKeep) != 0), (uint32_t)((f & kClone) != 0), (uint32_t)((f & kSplit) != 0),
                 (uint32_t)((f & kChild) != 0)}};
}

// Block-wide exclusive scan of four counts at once.
__device__ __forceinline__ Quad block_scan4(Quad q, Quad *total) {
    __shared__ uint32_t ws[4][kDB / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    Quad incl = q;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, incl.v[k], o);
            if (lane >= o) incl.v[k] += y;
        }
        if (lane == 31) ws[k][warp] = incl.v[k];
    }
    __syncthreads();
    Quad ex;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        uint32_t before = 0, all = 0;
        for (int w = 0; w < kDB / 32; ++w) {
            if (w < warp) before += ws[k][w];
            all += ws[k][w];
        }
        ex.v[k] = before + incl.v[k] - q.v[k];
        total->v[k] = all;
    }
    __syncthreads();
    return ex;
}

__global__ void __launch_bounds__(kDB) k_den_plan(int64_t n, const float *__restrict__ P, gs_grad_stats st,
                                                  gs_densify_params p, uint8_t *__restrict__ flags,
                                                  uint32_t *__restrict__ part, int nb) {
    const int64_t i = (int64_t)blockIdx.x * kDB + threadIdx.x;
    uint8_t f = 0;
    if (i < n) {
        f = den_flags(P, st, p, i);
        flags[i] = f;
    }
    Quad tot;
    block_scan4(quad_of(f), &tot);
    if (threadIdx.x == 0)
        for (int k = 0; k < 4; ++k) part[(int64_t)k * nb + blockIdx.x] = tot.v[k];
}

// Exclusive scan of the four rows of part [4][nb] in place (one block per
// row); totals[4] = the row sums.
__global__ void __launch_bounds__(1024) k_den_scan(uint32_t *__restrict__ part, int nb, uint32_t *__restrict__ totals,
                                                   int64_t *__restrict__ counts) {
    __shared__ int ws[32];
    uint32_t *row = part + (int64_t)blockIdx.x * nb;
    uint32_t carry = 0;
    for (int base = 0; base < nb; base += 1024) {
        const int j = base + threadIdx.x;
        const int v = j < nb ? (int)row[j] : 0;
        int tot;
        const int ex = block_exclusive_scan(v, ws, &tot);
        if (j < nb) row[j] = carry + (uint32_t)ex;
        carry += (uint32_t)tot;
    }
    if (threadIdx.x == 0) {
        totals[blockIdx.x] = carry;
        // counts: kept originals, kept clones, children, splits
        const int64_t slot[4] = {0, 1, 3, 2};
        counts[slot[blockIdx.x]] = blockIdx.x == 3 ? 2 * (int64_t)carry : (int64_t)carry;
    }
}

// Rotation of the unit quaternion (w, x, y, z) times a vector.
__device__ __forceinline__ void quat_rotate(float w, float x, float y, float z, const float v[3], float out[3]) {
    out[0] = (1.f - 2.f * (y * y + z * z)) * v[0] + 2.f * (x * y - w * z) * v[1] + 2.f * (x * z + w * y) * v[2];
    out[1] = 2.f * (x * y + w * z) * v[0] + (1.f - 2.f * (x * x + z * z)) * v[1] + 2.f * (y * z - w * x) * v[2];
    out[2] = 2.f * (x * z - w * y) * v[0] + 2.f * (y * z + w * x) * v[1] + (1.f - 2.f * (x * x + y * y)) * v[2];
}

__device__ __forceinline__ void copy_row(const float *__restrict__ src, float *__restrict__ dst) {
    const float4 *s4 = reinterpret_cast<const float4 *>(src);
    float4 *d4 = reinterpret_cast<float4 *>(dst);
#pragma unroll
    for (int c = 0; c < kRow / 4; ++c) d4[c] = s4[c];
}

__device__ __forceinline__ void zero_row(float *__restrict__ dst) {
    float4 *d4 = reinterpret_cast<float4 *>(dst);
#pragma unroll
    for (int c = 0; c < kRow / 4; ++c) d4[c] = make_float4(0.f, 0.f, 0.f, 0.f);
}

constexpr int kMaxCarry = 8;

struct ApplyOut {
    float *P, *m, *v;
    uint8_t *frozen;
    const uint32_t *csrc[kMaxCarry];
    uint32_t *cdst[kMaxCarry];
    int cwords[kMaxCarry];  // 4-byte words per row
    int ncarry;
};

__device__ __forceinline__ void write_new(int64_t o, const ApplyOut &out) {
    zero_row(out.m + o * kRow);
    zero_row(out.v + o * kRow);
    out.frozen[o] = 0;
    for (int c = 0; c < out.ncarry; ++c)
        for (int k = 0; k < out.cwords[c]; ++k) out.cdst[c][o * out.cwords[c] + k] = 0u;
}

__global__ void __launch_bounds__(kDB) k_den_apply(int64_t n, const float *__restrict__ P, const float *__restrict__ m,
                                                   const float *__restrict__ v, const uint8_t *__restrict__ frozen,
                                                   gs_densify_params p,
                                                   const float *__restrict__ z, const uint8_t *__restrict__ flags,
                                                   const uint32_t *__restrict__ part, int nb,
                                                   const uint32_t *__restrict__ totals, int64_t capacity,
                                                   ApplyOut out) {
    const int64_t i = (int64_t)blockIdx.x * kDB + threadIdx.x;
    const uint8_t f = i < n ? flags[i] : 0;
    Quad tot;
    const Quad ex = block_scan4(quad_of(f), &tot);
    const uint64_t kept = totals[0], clones = totals[1];
    if (kept + clones + 2ull * totals[3] > (uint64_t)capacity) return;  // checked by the host as well
    if (i >= n || f == 0) return;
    const float *src = P + i * kRow;
    if (f & kKeep) {
        const int64_t o = part[blockIdx.x] + ex.v[0];
        copy_row(src, out.P + o * kRow);
        copy_row(m + i * kRow, out.m + o * kRow);
        copy_row(v + i * kRow, out.v + o * kRow);
        out.frozen[o] = frozen ? frozen[i] : 0;
        for (int c = 0; c < out.ncarry; ++c)
            for (int k = 0; k < out.cwords[c]; ++k) out.cdst[c][o * out.cwords[c] + k] = out.csrc[c][i * out.cwords[c] + k];
    }
    if (f & kClone) {
        const int64_t o = (int64_t)kept + part[(int64_t)nb + blockIdx.x] + ex.v[1];
        copy_row(src, out.P + o * kRow);
        write_new(o, out);
    }
    if (f & kChild) {
        const int64_t rank = part[2 * (int64_t)nb + blockIdx.x] + ex.v[2];  // among all split originals
        const int64_t o0 = (int64_t)kept + (int64_t)clones + 2 * ((int64_t)part[3 * (int64_t)nb + blockIdx.x] + ex.v[3]);
        const float qw = src[6], qx = src[7], qy = src[8], qz = src[9];
        const float inv = rsqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
        const float s[3] = {expf(src[3]), expf(src[4]), expf(src[5])};
        for (int c = 0; c < 2; ++c) {
            const int64_t o = o0 + c;
            float *dst = out.P + o * kRow;
            copy_row(src, dst);
            const float *zz = z + (rank * 2 + c) * 3;
            const float sv[3] = {s[0] * zz[0], s[1] * zz[1], s[2] * zz[2]};
            float d[3];
            quat_rotate(qw * inv, qx * inv, qy * inv, qz * inv, sv, d);
            dst[0] = src[0] + d[0];
            dst[1] = src[1] + d[1];
            dst[2] = src[2] + d[2];
            dst[3] = __fsub_rn(src[3], p.log_split_div);
            dst[4] = __fsub_rn(src[4], p.log_split_div);
            dst[5] = __fsub_rn(src[5], p.log_split_div);
            write_new(o, out);
        }
    }
}

__global__ void k_opacity_reset(int64_t n, float *__restrict__ P, float *__restrict__ m, float *__restrict__ v,
                                float cap, const uint8_t *__restrict__ frozen) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || (frozen && frozen[i])) return;
    P[i * kRow + 10] = fminf(P[i * kRow + 10], cap);
    m[i * kRow + 10] = 0.f;
    v[i * kRow + 10] = 0.f;
}

// rescale: the moments carried into the new parameterisation -- its gradient
// is the old one divided by s = sigmoid'(x) = o (1 - o), so m / s and v / s^2
// (s floored at 1e-12); else the moments restart at zero.
__global__ void __launch_bounds__(256) k_opacity_to_abs(int64_t n, float *__restrict__ P, float *__restrict__ m,
                                                        float *__restrict__ v, int rescale,
                                                        float *__restrict__ slope_sum) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float slope = 0.f;
    if (i < n) {
        const float o = opacity_sigmoid(P[i * kRow + 10]);
        slope = o * (1.f - o);
        P[i * kRow + 10] = o;
        if (rescale) {
            const float is = 1.f / fmaxf(slope, 1e-12f);
            m[i * kRow + 10] *= is;
            v[i * kRow + 10] *= is * is;
        } else {
            m[i * kRow + 10] = 0.f;
            v[i * kRow + 10] = 0.f;
        }
    }
    if (slope_sum) {  // sum of sigmoid'(x) = o (1 - o) over the Gaussians
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) slope += __shfl_xor_sync(0xffffffffu, slope, off);
        if ((threadIdx.x & 31) == 0 && slope != 0.f) atomicAdd(slope_sum, slope);
    }
}

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct DenWs {
    uint8_t *flags;
    uint32_t *part, *totals;
    size_t bytes;
};

inline DenWs den_layout(char *base, int64_t n) {
    DenWs w;
    const int64_t nb = (n + kDB - 1) / kDB > 0 ? (n + kDB - 1) / kDB : 1;
    size_t off = 0;
    auto take = [&](size_t bytes) -> char * {
        char *p = base ? base + off : nullptr;
        off += align256(bytes);
        return p;
    };
    w.flags = (uint8_t *)take((size_t)(n > 0 ? n : 1));
    w.part = (uint32_t *)take(4 * 4 * (size_t)nb);
    w.totals = (uint32_t *)take(4 * 4);
    w.bytes = off;
    return w;
}

bool params_ok(const gs_densify_params *p) {
    return p && p->eps_xyz >= 0.f && p->eps_rgb >= 0.f && p->max_screen_radius >= 0;
}

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" size_t gs_densify_workspace_bytes(int64_t n) {
    if (n < 0) return 0;
    return den_layout(nullptr, n).bytes;
}

extern "C" int gs_densify_plan(int64_t n, const float *P, const gs_grad_stats *stats, const gs_densify_params *prm,
                               void *ws, size_t ws_bytes, int64_t *counts_dev, gs_stream_t stream) {
    if (n < 0 || n > INT32_MAX || !stats || !params_ok(prm) || !counts_dev) return GS_ERR_INVALID_ARG;
    const DenWs w = den_layout(static_cast<char *>(ws), n);
    if (!ws || ws_bytes < w.bytes || (reinterpret_cast<uintptr_t>(ws) & 255)) return GS_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    if (n == 0) {
        if (cudaMemsetAsync(counts_dev, 0, 4 * sizeof(int64_t), s) != cudaSuccess) return GS_ERR_CUDA;
        if (cudaMemsetAsync(w.totals, 0, 4 * sizeof(uint32_t), s) != cudaSuccess) return GS_ERR_CUDA;
        return GS_OK;
    }
    if (!P || !stats->acc_xyz || !stats->acc_rgb || !stats->cnt) return GS_ERR_INVALID_ARG;
    const int nb = (int)((n + kDB - 1) / kDB);
    k_den_plan<<<nb, kDB, 0, s>>>(n, P, *stats, *prm, w.flags, w.part, nb);
    k_den_scan<<<4, 1024, 0, s>>>(w.part, nb, w.totals, counts_dev);
    note_launches(2);
    return launch_status();
}

extern "C" int gs_densify_apply(int64_t n, const float *P, const float *m, const float *v, const uint8_t *frozen,
                                const gs_densify_carry *carry, int32_t n_carry, const gs_densify_params *prm,
                                const float *z, const void *ws, size_t ws_bytes, int64_t capacity, float *P_out,
                                float *m_out, float *v_out, uint8_t *frozen_out, gs_stream_t stream) {
    if (n < 0 || n > INT32_MAX || capacity < 0 || !params_ok(prm) || n_carry < 0 || n_carry > kMaxCarry ||
        (n_carry > 0 && !carry))
        return GS_ERR_INVALID_ARG;
    const DenWs w = den_layout(const_cast<char *>(static_cast<const char *>(ws)), n);
    if (!ws || ws_bytes < w.bytes) return GS_ERR_INVALID_ARG;
    if (n == 0) return GS_OK;
    if (!P || !m || !v || !P_out || !m_out || !v_out || !frozen_out) return GS_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(P) | reinterpret_cast<uintptr_t>(m) | reinterpret_cast<uintptr_t>(v) |
         reinterpret_cast<uintptr_t>(P_out) | reinterpret_cast<uintptr_t>(m_out) |
         reinterpret_cast<uintptr_t>(v_out)) & 15)
        return GS_ERR_INVALID_ARG;
    ApplyOut out{};
    out.P = P_out; out.m = m_out; out.v = v_out; out.frozen = frozen_out; out.ncarry = n_carry;
    for (int c = 0; c < n_carry; ++c) {
        const gs_densify_carry &k = carry[c];
        if (!k.src || !k.dst || k.row_bytes <= 0 || (k.row_bytes & 3) ||
            ((reinterpret_cast<uintptr_t>(k.src) | reinterpret_cast<uintptr_t>(k.dst)) & 3))
            return GS_ERR_INVALID_ARG;
        out.csrc[c] = static_cast<const uint32_t *>(k.src);
        out.cdst[c] = static_cast<uint32_t *>(k.dst);
        out.cwords[c] = k.row_bytes / 4;
    }
    const int nb = (int)((n + kDB - 1) / kDB);
    k_den_apply<<<nb, kDB, 0, as_stream(stream)>>>(n, P, m, v, frozen, *prm, z, w.flags, w.part, nb, w.totals,
                                                   capacity, out);
    note_launches(1);
    return launch_status();
}

extern "C" int gs_opacity_reset(int64_t n, float *P, float *m, float *v, float logit_cap, const uint8_t *frozen,
                                gs_stream_t stream) {
    if (n < 0) return GS_ERR_INVALID_ARG;
    if (n == 0) return GS_OK;
    if (!P || !m || !v) return GS_ERR_INVALID_ARG;
    k_opacity_reset<<<grid_for(n, 256), 256, 0, as_stream(stream)>>>(n, P, m, v, logit_cap, frozen);
    note_launches(1);
    return launch_status();
}

extern "C" int gs_opacity_to_abs(int64_t n, float *P, float *m, float *v, int32_t moments, float *slope_sum_dev,
                                 gs_stream_t stream) {
    if (n < 0 || (moments != GS_MOMENTS_ZERO && moments != GS_MOMENTS_RESCALE)) return GS_ERR_INVALID_ARG;
    if (n == 0) return GS_OK;
    if (!P || !m || !v) return GS_ERR_INVALID_ARG;
    k_opacity_to_abs<<<grid_for(n, 256), 256, 0, as_stream(stream)>>>(n, P, m, v, moments == GS_MOMENTS_RESCALE,
                                                                       slope_sum_dev);
    note_launches(1);
    return launch_status();
}
