// Tile rasteriser: front-to-back alpha compositing (Sec. 3.1, Eq. 2) and its
// backward (Sec. 3.2.4), which skips the gradient work of frozen Gaussians.
//
// One CTA per screen tile, two pixels per thread. The tile's sorted splat
// list is staged through shared memory in batches, so every thread reads
// each splat as a shared-memory broadcast. No tensor
// cores: the work is a per-pixel exponential and a handful of FMAs.
//
// The backward walks each list back to front and recovers the transmittance
// in front of every splat from the value the forward left over, so no
// per-pixel list is stored. A warp's 32 pixels see the same splat at the
// same time; their nine gradient terms are summed with a recursive-halving
// warp reduction, added once per warp into a shared accumulator, and the
// accumulator goes to global memory with one atomic per value per tile.
#include "common.cuh"

static_assert(sizeof(gs_camera) == 112, "gs_camera layout");
static_assert(sizeof(gs_raster_job) == 184, "gs_raster_job layout");

namespace gs {
namespace {


// A thread owns PPT pixels of its tile, (x, y + k TS/PPT) for k < PPT. Each
// splat staged in shared memory is loaded once per PPT evaluations, and the
// per-pixel update is written with selects instead of branches so the PPT
// independent chains interleave.
//
// With resume given, the walk also records where the backward may start:
// resume_pos[tile] = 1 + the list position of the last unfrozen splat it
// passed (0 if none), and per pixel resume = (T after that splat, the colour
// blended behind it), so that the backward skips the frozen splats behind
// every unfrozen one: they carry no gradient, and the state they would
// rebuild is this one.
template <int TS, int PPT, int B>
__device__ __forceinline__ void render_tile(const float *__restrict__ splats, const uint32_t *__restrict__ vals,
                                            const uint32_t *__restrict__ ranges, const DevCam &cam,
                                            float *__restrict__ image, float *__restrict__ t_final,
                                            int32_t *__restrict__ n_last, int tile,
                                            const uint8_t *__restrict__ frozen = nullptr,
                                            float4 *__restrict__ resume = nullptr,
                                            int32_t *__restrict__ resume_pos = nullptr) {
    constexpr int NT = TS * TS / PPT;  // threads; B = splats per staged batch
    // With an even number of pixels per thread, the pixels go in pairs through
    // the packed FP32 instructions (f2_*), and each splat is staged with every
    // value duplicated into both halves of a 64-bit pair.
    constexpr bool kPair = PPT % 2 == 0;
    constexpr int NP = kPair ? PPT / 2 : 1;
    __shared__ float4 s_xyab[kPair ? 1 : B];
    __shared__ float4 s_cocg[kPair ? 1 : B];
    __shared__ float s_blue[kPair ? 1 : B];
    __shared__ ulonglong2 s_pk[kPair ? 4 * B : 1];  // (mx, my), (-a/2, -b), (-c/2, o), (r, g), each duplicated
    __shared__ f32x2 s_pb[kPair ? B : 1];           // (blue, blue)
    __shared__ int s_lu;  // the batch's last unfrozen splat (-1: none)
    __shared__ int s_upos;
    const int tx = tile % cam.tiles_x, ty = tile / cam.tiles_x;
    const int px = tx * TS + (int)(threadIdx.x % TS);
    const uint32_t start = ranges[2 * tile], end = ranges[2 * tile + 1];
    const float fpx = (float)px;
    float fpy[PPT], T[PPT], c0[PPT], c1[PPT], c2[PPT];
    int last[PPT], py[PPT];
    bool done[PPT];
    float uT[PPT], u0[PPT], u1[PPT], u2[PPT];  // T and colour after the last unfrozen splat passed
    int upos = 0;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        py[k] = ty * TS + (int)(threadIdx.x / TS) + k * (TS / PPT);
        fpy[k] = (float)py[k];
        T[k] = 1.f;
        c0[k] = c1[k] = c2[k] = 0.f;
        last[k] = 0;
        done[k] = !(px < cam.W && py[k] < cam.H);
        uT[k] = 1.f;
        u0[k] = u1[k] = u2[k] = 0.f;
    }
    // packed state of pixel pairs (2h, 2h + 1); the scalar arrays are brought up
    // to date from it where they are read (the resume record and the end)
    f32x2 T2[NP], r2[NP], g2[NP], b2[NP], fpy2[NP];
    const f32x2 fpx2 = f2_pack(fpx, fpx), one2 = f2_pack(1.f, 1.f);
#pragma unroll
    for (int h = 0; h < NP; ++h) {
        T2[h] = one2;
        r2[h] = g2[h] = b2[h] = f2_pack(0.f, 0.f);
        fpy2[h] = kPair ? f2_pack(fpy[2 * h], fpy[(2 * h + 1) % PPT]) : 0ull;
    }
    auto to_scalar = [&]() {
        if constexpr (kPair) {
#pragma unroll
            for (int h = 0; h < NP; ++h) {
                f2_unpack(T2[h], T[2 * h], T[2 * h + 1]);
                f2_unpack(r2[h], c0[2 * h], c0[2 * h + 1]);
                f2_unpack(g2[h], c1[2 * h], c1[2 * h + 1]);
                f2_unpack(b2[h], c2[2 * h], c2[2 * h + 1]);
            }
        }
    };
    if (resume) {  // a uniform branch
        if (threadIdx.x == 0) s_upos = 0;
        __syncthreads();
    }
    if (threadIdx.x == 0) s_lu = -1;  // ordered before the staging's atomics by the loop's first barrier
    for (uint32_t base = start; base < end; base += B) {
        bool all = true;
#pragma unroll
        for (int k = 0; k < PPT; ++k) all = all && done[k];
        if (__syncthreads_count(all) == NT) break;
        for (int q = threadIdx.x; q < B; q += NT) {
            if (base + q < end) {
                // staged with -a/2 and -c/2 in place of a and c: the row coefficients of
                // splat_row, rounded once here instead of once per thread
                const uint32_t g = vals[base + q];
                const float4 *r = reinterpret_cast<const float4 *>(splats + (int64_t)g * kSplat);
                float4 xa = __ldg(r), co = __ldg(r + 1);
                const float blue = __ldg(reinterpret_cast<const float *>(r + 2));
                xa.z = __fmul_rn(-0.5f, xa.z);
                co.x = __fmul_rn(-0.5f, co.x);
                if constexpr (kPair) {
                    s_pk[4 * q] = make_ulonglong2(f2_pack(xa.x, xa.x), f2_pack(xa.y, xa.y));
                    s_pk[4 * q + 1] = make_ulonglong2(f2_pack(xa.z, xa.z), f2_pack(-xa.w, -xa.w));
                    s_pk[4 * q + 2] = make_ulonglong2(f2_pack(co.x, co.x), f2_pack(co.y, co.y));
                    s_pk[4 * q + 3] = make_ulonglong2(f2_pack(co.z, co.z), f2_pack(co.w, co.w));
                    s_pb[q] = f2_pack(blue, blue);
                } else {
                    s_xyab[q] = xa;
                    s_cocg[q] = co;
                    s_blue[q] = blue;
                }
                if (resume && !(frozen && frozen[g])) atomicMax(&s_lu, q);
            }
        }
        __syncthreads();
        const int cnt = (int)min((uint32_t)B, end - base);
        // One splat of the batch for this thread's pixels; false once they are all done.
        auto blend = [&](int j) -> bool {
            const float4 xa = s_xyab[j], co = s_cocg[j];
            const float blue = s_blue[j];
            const float dx = __fsub_rn(xa.x, fpx);
            SplatRow row;  // splat_row's coefficients from the staged halves
            row.c0 = __fmul_rn(xa.z, __fmul_rn(dx, dx));
            row.c1 = __fmul_rn(-xa.w, dx);
            row.c2 = co.x;
            bool alive = false;
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                const float dy = __fsub_rn(xa.y, fpy[k]);
                const float power = splat_power(row, dy);
                const float alpha = fminf(kAlphaMax, __fmul_rn(co.y, __expf(power)));
                const float tn = __fmul_rn(T[k], __fsub_rn(1.f, alpha));
                const bool use = !done[k] && power <= 0.f && alpha >= kAlphaMin;
                const bool stop = use && tn < kTMin;
                const bool add = use && !stop;
                const float w = add ? alpha * T[k] : 0.f;
                c0[k] += co.z * w;
                c1[k] += co.w * w;
                c2[k] += blue * w;
                T[k] = add ? tn : T[k];
                last[k] = add ? (int)(base - start) + j + 1 : last[k];
                done[k] = done[k] || stop;
                alive = alive || !done[k];
            }
            return alive;
        };
        // The same for a pair of pixels per packed instruction: every rounded
        // operation is the scalar one's, so the results are bit for bit those of
        // blend (the exponential stays scalar).
        auto blend2 = [&](int j) -> bool {
            const ulonglong2 q0 = s_pk[4 * j], q1 = s_pk[4 * j + 1], q2 = s_pk[4 * j + 2], q3 = s_pk[4 * j + 3];
            const f32x2 qb = s_pb[j];
            const f32x2 dx2 = f2_sub(q0.x, fpx2);
            const f32x2 rc0 = f2_mul(q1.x, f2_mul(dx2, dx2)), rc1 = f2_mul(q1.y, dx2);
            bool alive = false;
#pragma unroll
            for (int h = 0; h < NP; ++h) {
                const int ka = 2 * h, kb = (2 * h + 1) % PPT;
                const f32x2 dy2 = f2_sub(q0.y, fpy2[h]);
                const f32x2 pw2 = f2_fma(f2_fma(q2.x, dy2, rc1), dy2, rc0);
                float pa, pb;
                f2_unpack(pw2, pa, pb);
                float oa, ob;
                f2_unpack(f2_mul(q2.y, f2_pack(__expf(pa), __expf(pb))), oa, ob);
                const float aa = fminf(kAlphaMax, oa), ab = fminf(kAlphaMax, ob);
                const f32x2 al2 = f2_pack(aa, ab);
                float tna, tnb, ata, atb, Ta, Tb;
                f2_unpack(f2_mul(T2[h], f2_sub(one2, al2)), tna, tnb);
                f2_unpack(f2_mul(al2, T2[h]), ata, atb);
                f2_unpack(T2[h], Ta, Tb);
                const bool usea = !done[ka] && pa <= 0.f && aa >= kAlphaMin;
                const bool useb = !done[kb] && pb <= 0.f && ab >= kAlphaMin;
                const bool stopa = usea && tna < kTMin, stopb = useb && tnb < kTMin;
                const bool adda = usea && !stopa, addb = useb && !stopb;
                const f32x2 w2 = f2_pack(adda ? ata : 0.f, addb ? atb : 0.f);
                r2[h] = f2_fma(q3.x, w2, r2[h]);
                g2[h] = f2_fma(q3.y, w2, g2[h]);
                b2[h] = f2_fma(qb, w2, b2[h]);
                T2[h] = f2_pack(adda ? tna : Ta, addb ? tnb : Tb);
                const int idx = (int)(base - start) + j + 1;
                last[ka] = adda ? idx : last[ka];
                last[kb] = addb ? idx : last[kb];
                done[ka] = done[ka] || stopa;
                done[kb] = done[kb] || stopb;
                alive = alive || !done[ka] || !done[kb];
            }
            return alive;
        };
        auto step = [&](int jj) -> bool {
            if constexpr (kPair) return blend2(jj);
            else return blend(jj);
        };
        // with resume, the loop runs in two parts around the batch's last unfrozen
        // splat, recording the state after it; no test per splat
        const int lu = resume ? s_lu : -1;
        int j = 0;
        bool alive = true;
        if (lu >= 0) {
            for (; j <= lu && alive; ++j) alive = step(j);
            if (alive || j == lu + 1) {  // reached the state after splat lu
                to_scalar();
#pragma unroll
                for (int k = 0; k < PPT; ++k) {
                    uT[k] = T[k];
                    u0[k] = c0[k];
                    u1[k] = c1[k];
                    u2[k] = c2[k];
                }
                upos = (int)(base - start) + lu + 1;
            }
        }
        for (; j < cnt && alive; ++j) alive = step(j);
        __syncthreads();
        if (threadIdx.x == 0) s_lu = -1;  // read by every thread before the barrier above
    }
    to_scalar();
    if (resume) {
        // A thread leaves the splat loop once its own pixels are done, so it may
        // have stopped before the tile's last unfrozen splat: its pixels are then
        // done at that position too, with their final T and nothing blended behind.
        if (upos > 0) atomicMax(&s_upos, upos);
        __syncthreads();
        const int umax = s_upos;
        if (upos < umax) {
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                uT[k] = T[k];
                u0[k] = c0[k];
                u1[k] = c1[k];
                u2[k] = c2[k];
            }
        }
        upos = umax;
    }
    const int64_t HW = (int64_t)cam.W * cam.H;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        if (px < cam.W && py[k] < cam.H) {
            const int64_t pix = (int64_t)py[k] * cam.W + px;
            image[pix] = c0[k] + T[k] * cam.bg[0];
            image[HW + pix] = c1[k] + T[k] * cam.bg[1];
            image[2 * HW + pix] = c2[k] + T[k] * cam.bg[2];
            t_final[pix] = T[k];
            n_last[pix] = last[k];
            if (resume)
                resume[pix] = make_float4(uT[k], __fsub_rn(c0[k], u0[k]), __fsub_rn(c1[k], u1[k]),
                                          __fsub_rn(c2[k], u2[k]));
        }
    }
    if (resume && threadIdx.x == 0) resume_pos[tile] = upos;
}

template <int TS, int PPT, int B>
__global__ void __launch_bounds__(TS * TS / PPT) k_render_fwd(const float *__restrict__ splats,
                                                              const uint32_t *__restrict__ vals,
                                                              const uint32_t *__restrict__ ranges, DevCam cam,
                                                              float *__restrict__ image, float *__restrict__ t_final,
                                                              int32_t *__restrict__ n_last,
                                                              const uint8_t *__restrict__ frozen,
                                                              float4 *__restrict__ resume,
                                                              int32_t *__restrict__ resume_pos) {
    wait_prior_grid();
    render_tile<TS, PPT, B>(splats, vals, ranges, cam, image, t_final, n_last, blockIdx.x, frozen, resume,
                            resume_pos);
}

// Sum of nine per-lane values over a warp by recursive halving: at each of
// the five xor levels a lane keeps half of its remaining slots and adds the
// partner's copy of them (5 + 3 + 2 + 1 + 1 = 12 shuffles instead of 45).
// On return, lane L holds the warp total of value kSlotOf[(L >> 1) & 15]
// (-1: none); lanes L and L ^ 1 hold the same total.
__device__ __constant__ int8_t kSlotOf[16] = {0, 1, 2, -1, 3, 4, -1, -1, 5, 6, 7, -1, 8, -1, -1, -1};

__device__ __forceinline__ float warp_sum9(const float (&g)[9], int lane) {
    const bool h4 = lane & 16, h3 = lane & 8, h2 = lane & 4, h1 = lane & 2;
    float r[5];
#pragma unroll
    for (int j = 0; j < 5; ++j) {  // keep values 0-4 (lower half) or 5-8 (upper half)
        const float lo = g[j], hi = j < 4 ? g[5 + j] : 0.f;
        const float mine = h4 ? hi : lo, other = h4 ? lo : hi;
        r[j] = mine + __shfl_xor_sync(kFull, other, 16);
    }
    float s[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {  // keep slots 0-2 or 3-4
        const float lo = r[j], hi = j < 2 ? r[3 + j] : 0.f;
        const float mine = h3 ? hi : lo, other = h3 ? lo : hi;
        s[j] = mine + __shfl_xor_sync(kFull, other, 8);
    }
    float u[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {  // keep slots 0-1 or 2
        const float lo = s[j], hi = j < 1 ? s[2 + j] : 0.f;
        const float mine = h2 ? hi : lo, other = h2 ? lo : hi;
        u[j] = mine + __shfl_xor_sync(kFull, other, 4);
    }
    float w = (h1 ? u[1] : u[0]) + __shfl_xor_sync(kFull, h1 ? u[0] : u[1], 2);
    return w + __shfl_xor_sync(kFull, w, 1);
}

// Backward state of one pixel: recovered transmittance T, dL/dC, and the
// colour blended behind the current splat, kept only as G = dL/dC . sum over
// the splats k behind it of c_k alpha_k T_k (all dL/dalpha needs): a splat
// with alpha and T in front of it has dL/dalpha = T dL/dC . c - (G + T_final
// dL/dC . bg) / (1 - alpha), and adds dL/dC . c alpha T to G.
struct PixBwd {
    float T, Tf, dC0, dC1, dC2, bgdot;
    float G;
    int nl;
};

// One (pixel, splat) step of the backward blend. The exponent's derivatives
// with respect to the 2-D mean and conic are dx/dy polynomials; the thread's
// pixels share dx, so only the dy moments of dL/dpower are summed here
// (g[0] += dpow, g[1] += dy dpow, g[2] += dy^2 dpow) and geo_grads() turns
// them into the five gradients once per splat. FRZ: the splat is frozen, so
// only the pixel's state moves (a separate instantiation, so that a frozen
// splat issues none of the gradient instructions).
template <bool FRZ>
__device__ __forceinline__ bool pix_bwd(PixBwd &p, int pos, const SplatRow &row, float dy, const float4 &co,
                                        float blue, float (&g)[9]) {
    const float power = splat_power(row, dy);
    const float G = __expf(power);
    const float oG = __fmul_rn(co.y, G);
    const float alpha = fminf(kAlphaMax, oG);
    if (!(pos < p.nl && power <= 0.f && alpha >= kAlphaMin)) return false;
    const float om = 1.f - alpha;
    p.T = __fdividef(p.T, om);  // transmittance in front of this splat
    const float dcc = p.dC0 * co.z + p.dC1 * co.w + p.dC2 * blue;
    if (!FRZ) {
        const float dA = p.T * dcc - __fdividef(fmaf(p.Tf, p.bgdot, p.G), om);
        const float wT = alpha * p.T;
        g[6] += wT * p.dC0;
        g[7] += wT * p.dC1;
        g[8] += wT * p.dC2;
        if (!(oG > kAlphaMax)) {
            const float dpow = dA * oG;
            const float ydp = dy * dpow;
            g[5] += dA * G;
            g[0] += dpow;
            g[1] += ydp;
            g[2] += dy * ydp;
        }
    }
    p.G = fmaf(dcc * alpha, p.T, p.G);
    return true;
}

// dy moments (s0, s1, s2) of dL/dpower -> gradients of the 2-D mean and
// conic for power = -0.5 (a dx^2 + c dy^2) - b dx dy, dx = mean_x - px.
__device__ __forceinline__ void geo_grads(float (&g)[9], float dx, float a, float b, float c) {
    const float s0 = g[0], s1 = g[1], s2 = g[2];
    const float xs0 = dx * s0;
    g[0] = -(a * xs0 + b * s1);
    g[1] = -(b * xs0 + c * s1);
    g[2] = -0.5f * dx * xs0;
    g[3] = -dx * s1;
    g[4] = -0.5f * s2;
}

// The walk starts from the pixel's final state (T = T_final, nothing behind),
// or, with resume, from the state the forward recorded after the tile's last
// unfrozen splat (T there, and the colour blended behind it).
__device__ __forceinline__ void pix_load(PixBwd &p, bool inside, int64_t pix, int64_t HW, const float *t_final,
                                         const int32_t *n_last, const float *dl, const float4 *resume,
                                         const DevCam &cam) {
    p.T = 1.f; p.dC0 = p.dC1 = p.dC2 = 0.f; p.nl = 0;
    p.G = 0.f;
    if (inside) {
        p.T = t_final[pix];
        p.nl = n_last[pix];
        p.dC0 = dl[pix];
        p.dC1 = dl[HW + pix];
        p.dC2 = dl[2 * HW + pix];
    }
    p.Tf = p.T;
    p.bgdot = cam.bg[0] * p.dC0 + cam.bg[1] * p.dC1 + cam.bg[2] * p.dC2;
    if (inside && resume) {
        const float4 r = resume[pix];
        p.T = r.x;
        p.G = p.dC0 * r.y + p.dC1 * r.z + p.dC2 * r.w;
    }
}

template <int TS, int PPT, int B>
__device__ __forceinline__ void raster_bwd_tile(const float *__restrict__ splats, const uint32_t *__restrict__ vals,
                                                const uint32_t *__restrict__ ranges, const DevCam &cam,
                                                const float *__restrict__ t_final, const int32_t *__restrict__ n_last,
                                                const float *__restrict__ dl_dimage, const uint8_t *__restrict__ frozen,
                                                float *__restrict__ grad2d, int tile,
                                                const float4 *__restrict__ resume = nullptr,
                                                const int32_t *__restrict__ resume_pos = nullptr) {
    constexpr int NT = TS * TS / PPT;
    __shared__ float4 s_xyab[B];
    __shared__ float4 s_cocg[B];
    __shared__ float s_blue[B];
    __shared__ uint32_t s_gid[B];
    __shared__ int s_frz[B];
    __shared__ float s_acc[9][B];
    __shared__ int s_maxlast;
    const int tx = tile % cam.tiles_x, ty = tile / cam.tiles_x;
    const int px = tx * TS + (int)(threadIdx.x % TS);
    const uint32_t start = ranges[2 * tile];
    const float fpx = (float)px;
    const int64_t HW = (int64_t)cam.W * cam.H;
    PixBwd p[PPT];
    float fpy[PPT];
    int nlmax = 0;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const int py = ty * TS + (int)(threadIdx.x / TS) + k * (TS / PPT);
        fpy[k] = (float)py;
        pix_load(p[k], px < cam.W && py < cam.H, (int64_t)py * cam.W + px, HW, t_final, n_last, dl_dimage, resume,
                 cam);
        nlmax = max(nlmax, p[k].nl);
    }
    if (threadIdx.x == 0) s_maxlast = 0;
    __syncthreads();
    if (nlmax > 0) atomicMax(&s_maxlast, nlmax);
    __syncthreads();
    // with resume, the frozen splats behind the last unfrozen one are skipped
    const uint32_t rend = start + (uint32_t)(resume ? min(s_maxlast, resume_pos[tile]) : s_maxlast);
    const int lane = threadIdx.x & 31;
    const int slot = kSlotOf[(lane >> 1) & 15];
    const bool writer = slot >= 0 && !(lane & 1);

    for (int64_t bend = rend; bend > (int64_t)start; bend -= B) {
        const int64_t bstart = bend - B > (int64_t)start ? bend - B : (int64_t)start;
        const int cnt = (int)(bend - bstart);
        for (int q = threadIdx.x; q < B; q += NT) {
            if (q < cnt) {
                const uint32_t g = vals[bstart + q];
                const float4 *r = reinterpret_cast<const float4 *>(splats + (int64_t)g * kSplat);
                // -a/2 and -c/2 in place of a and c, as in the forward (exact halves;
                // geo_grads gets a and c back by an exact doubling)
                float4 xa = __ldg(r), co = __ldg(r + 1);
                xa.z = __fmul_rn(-0.5f, xa.z);
                co.x = __fmul_rn(-0.5f, co.x);
                s_xyab[q] = xa;
                s_cocg[q] = co;
                s_blue[q] = __ldg(reinterpret_cast<const float *>(r + 2));
                s_gid[q] = g;
                s_frz[q] = frozen ? (int)frozen[g] : 0;
            }
#pragma unroll
            for (int k = 0; k < 9; ++k) s_acc[k][q] = 0.f;
        }
        __syncthreads();
        for (int j = cnt - 1; j >= 0; --j) {
            const int pos = (int)(bstart - (int64_t)start) + j;  // position in the tile list
            const float4 xa = s_xyab[j], co = s_cocg[j];
            const float blue = s_blue[j];
            const bool frz = s_frz[j] != 0;  // the same for every thread: a uniform branch
            const float dx = __fsub_rn(xa.x, fpx);
            SplatRow row;  // splat_row's coefficients from the staged halves
            row.c0 = __fmul_rn(xa.z, __fmul_rn(dx, dx));
            row.c1 = __fmul_rn(-xa.w, dx);
            row.c2 = co.x;
            float g[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            if (frz) {
#pragma unroll
                for (int k = 0; k < PPT; ++k) pix_bwd<true>(p[k], pos, row, __fsub_rn(xa.y, fpy[k]), co, blue, g);
            } else {
                bool c = false;
#pragma unroll
                for (int k = 0; k < PPT; ++k)
                    c |= pix_bwd<false>(p[k], pos, row, __fsub_rn(xa.y, fpy[k]), co, blue, g);
                if (__any_sync(kFull, c)) {
                    geo_grads(g, dx, -2.f * xa.z, xa.w, -2.f * co.x);
                    const float tot = warp_sum9(g, lane);
                    if (writer) atomicAdd(&s_acc[slot][j], tot);
                }
            }
        }
        __syncthreads();
        for (int q = threadIdx.x; q < cnt; q += NT) {
            if (!s_frz[q]) {
                float *dst = grad2d + (int64_t)s_gid[q] * kG2d;
#pragma unroll
                for (int k = 0; k < 9; ++k) {
                    const float v = s_acc[k][q];
                    if (v != 0.f) atomicAdd(dst + k, v);
                }
            }
        }
        __syncthreads();
    }
}

template <int TS, int PPT, int B>
__global__ void __launch_bounds__(TS * TS / PPT) k_raster_bwd(const float *__restrict__ splats,
                                                              const uint32_t *__restrict__ vals,
                                                              const uint32_t *__restrict__ ranges, DevCam cam,
                                                              const float *__restrict__ t_final,
                                                              const int32_t *__restrict__ n_last,
                                                              const float *__restrict__ dl_dimage,
                                                              const uint8_t *__restrict__ frozen,
                                                              float *__restrict__ grad2d,
                                                              const float4 *__restrict__ resume,
                                                              const int32_t *__restrict__ resume_pos) {
    wait_prior_grid();
    raster_bwd_tile<TS, PPT, B>(splats, vals, ranges, cam, t_final, n_last, dl_dimage, frozen, grad2d, blockIdx.x,
                                resume, resume_pos);
}

// ---- measurement support: the (pixel, splat) pairs the backward visits ----
// Per Gaussian, the pixels of this view it is blended into (the "hits" of
// significance pruning, Sec. 3.3): one CTA per tile, one thread per pixel,
// all threads at the same list position at once, one atomic per warp and
// position with the number of its pixels that blend the splat there.
__global__ void k_hit_counts(const float *__restrict__ splats, const uint32_t *__restrict__ vals,
                             const uint32_t *__restrict__ ranges, DevCam cam, const int32_t *__restrict__ n_last,
                             uint32_t *__restrict__ hits) {
    __shared__ int s_max;
    if (threadIdx.x == 0) s_max = 0;
    __syncthreads();
    const int tile = blockIdx.x, TS = cam.tile;
    const int px = (tile % cam.tiles_x) * TS + (int)(threadIdx.x % TS);
    const int py = (tile / cam.tiles_x) * TS + (int)(threadIdx.x / TS);
    const bool inside = px < cam.W && py < cam.H;
    const int nl = inside ? n_last[(int64_t)py * cam.W + px] : 0;
    if (nl > 0) atomicMax(&s_max, nl);
    __syncthreads();
    const int jmax = s_max;
    const uint32_t start = ranges[2 * tile];
    const float fpx = (float)px, fpy = (float)py;
    const int lane = threadIdx.x & 31;
    for (int j = 0; j < jmax; ++j) {
        const uint32_t g = vals[start + j];
        bool hit = false;
        if (j < nl) {
            const float4 *r = reinterpret_cast<const float4 *>(splats + (int64_t)g * kSplat);
            const float4 xa = __ldg(r), co = __ldg(r + 1);
            const float power = splat_power(splat_row(__fsub_rn(xa.x, fpx), xa.z, xa.w, co.x), __fsub_rn(xa.y, fpy));
            const float alpha = fminf(kAlphaMax, __fmul_rn(co.y, __expf(power)));
            hit = power <= 0.f && alpha >= kAlphaMin;
        }
        const unsigned b = __ballot_sync(kFull, hit);
        if (lane == 0 && b) atomicAdd(hits + g, (uint32_t)__popc(b));
    }
}

// One CTA per tile, one thread per pixel, walking the pixel's list with the
// forward's own decisions up to where the resuming backward walks it: the
// pixel's last contributor, or with a freeze map 1 + the tile's last unfrozen
// entry among those the tile's deepest contributor reaches, if that is less
// (a lower bound of the backward's walk, which may go on to the deepest
// contributor when an unfrozen entry lies further on in the list).
__device__ __forceinline__ bool pair_blended(const float *__restrict__ splats, uint32_t g, float fpx, float fpy) {
    const float4 *r = reinterpret_cast<const float4 *>(splats + (int64_t)g * kSplat);
    const float4 xa = __ldg(r), co = __ldg(r + 1);
    const float power = splat_power(splat_row(__fsub_rn(xa.x, fpx), xa.z, xa.w, co.x), __fsub_rn(xa.y, fpy));
    const float alpha = fminf(kAlphaMax, __fmul_rn(co.y, __expf(power)));
    return power <= 0.f && alpha >= kAlphaMin;
}

__global__ void k_pair_counts(const float *__restrict__ splats, const uint32_t *__restrict__ vals,
                              const uint32_t *__restrict__ ranges, DevCam cam, const int32_t *__restrict__ n_last,
                              const uint8_t *__restrict__ frozen, unsigned long long *__restrict__ counts) {
    __shared__ unsigned long long s_c[3];
    __shared__ int s_maxnl, s_lu;
    if (threadIdx.x < 3) s_c[threadIdx.x] = 0ull;
    if (threadIdx.x == 0) { s_maxnl = 0; s_lu = -1; }
    __syncthreads();
    const int tile = blockIdx.x, TS = cam.tile;
    const int px = (tile % cam.tiles_x) * TS + (int)(threadIdx.x % TS);
    const int py = (tile / cam.tiles_x) * TS + (int)(threadIdx.x / TS);
    const bool inside = px < cam.W && py < cam.H;
    const int nl = inside ? n_last[(int64_t)py * cam.W + px] : 0;
    const uint32_t start = ranges[2 * tile];
    if (nl > 0) atomicMax(&s_maxnl, nl);
    __syncthreads();
    if (frozen) {
        for (int j = (int)threadIdx.x; j < s_maxnl; j += (int)blockDim.x)
            if (!frozen[vals[start + j]]) atomicMax(&s_lu, j);
        __syncthreads();
    }
    const int upto = frozen ? min(nl, s_lu + 1) : nl;
    uint32_t c[3] = {0u, 0u, 0u};
    const float fpx = (float)px, fpy = (float)py;
    for (int j = 0; j < upto; ++j) {
        const uint32_t g = vals[start + j];
        if (pair_blended(splats, g, fpx, fpy))
            ++c[frozen && frozen[g] ? 1 : 0];
        else
            ++c[2];
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        unsigned long long v = c[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
        if ((threadIdx.x & 31) == 0 && v) atomicAdd(&s_c[k], v);
    }
    __syncthreads();
    if (threadIdx.x < 3 && s_c[threadIdx.x]) atomicAdd(counts + threadIdx.x, s_c[threadIdx.x]);
}

// ---- many views of many scenes in one persistent launch ----
// CTAs pull (job, tile) items from a device counter until the batch is done,
// so jobs of uneven cost (scenes of different sizes) share the GPU without a
// per-job launch. Every job of a batch has the same image size and tile.
__device__ __forceinline__ int next_item(uint32_t *queue, int *s_item) {
    __syncthreads();  // every thread is done with the previous item's shared memory
    if (threadIdx.x == 0) *s_item = (int)atomicAdd(queue, 1u);
    __syncthreads();
    return *s_item;
}

__device__ uint32_t g_render_flags;

// A job whose camera does not have the batch's image size and tile would
// index its tile ranges and images with the wrong grid: it is skipped and
// GS_FLAG_BADJOB raised (uniform across the CTA: every thread reads the same job).
__device__ __forceinline__ bool job_ok(const DevCam &cam, int W, int H, int TS) {
    if (cam.W == W && cam.H == H && cam.tile == TS) return true;
    if (threadIdx.x == 0) atomicOr(&g_render_flags, GS_FLAG_BADJOB);
    return false;
}

template <int TS, int PPT, int B>
__global__ void __launch_bounds__(TS * TS / PPT) k_render_fwd_batch(const gs_raster_job *__restrict__ jobs,
                                                                    int W, int H, int tiles_per_job, int total,
                                                                    uint32_t *__restrict__ queue) {
    __shared__ int s_item;
    for (int item = next_item(queue, &s_item); item < total; item = next_item(queue, &s_item)) {
        const gs_raster_job &j = jobs[item / tiles_per_job];
        const DevCam cam = make_cam(&j.cam);
        if (!job_ok(cam, W, H, TS)) continue;
        render_tile<TS, PPT, B>(j.splats, j.vals, j.ranges, cam, j.image, j.t_final, j.n_last, item % tiles_per_job);
    }
}

template <int TS, int PPT, int B>
__global__ void __launch_bounds__(TS * TS / PPT) k_raster_bwd_batch(const gs_raster_job *__restrict__ jobs,
                                                                    int W, int H, int tiles_per_job, int total,
                                                                    uint32_t *__restrict__ queue) {
    __shared__ int s_item;
    for (int item = next_item(queue, &s_item); item < total; item = next_item(queue, &s_item)) {
        const gs_raster_job &j = jobs[item / tiles_per_job];
        const DevCam cam = make_cam(&j.cam);
        if (!job_ok(cam, W, H, TS)) continue;
        raster_bwd_tile<TS, PPT, B>(j.splats, j.vals, j.ranges, cam, j.t_final, j.n_last, j.dl_dimage, j.frozen,
                                    j.grad2d, item % tiles_per_job);
    }
}

// Launch shape used when the caller gives none: pixels per thread and batch
// size of each kernel by tile size (timed on GB300; the autotuner may pick
// another per workload).
inline void default_config(int tile, bool bwd, int &ppt, int &batch) {
    if (tile == 8) { ppt = 1; batch = 64; return; }
    if (tile == 16) { ppt = bwd ? 2 : 1; batch = 256; return; }
    ppt = 2;
    batch = 256;
}

struct FwdArgs {
    const float *splats;
    const uint32_t *vals, *ranges;
    DevCam cam;
    float *image, *t_final;
    int32_t *n_last;
    const uint8_t *frozen;
    float4 *resume;
    int32_t *resume_pos;
};

struct BwdArgs {
    const float *splats;
    const uint32_t *vals, *ranges;
    DevCam cam;
    const float *t_final;
    const int32_t *n_last;
    const float *dl;
    const uint8_t *frozen;
    float *grad2d;
    const float4 *resume;
    const int32_t *resume_pos;
};

template <int TS, int PPT, int B>
void launch(const FwdArgs &a, cudaStream_t s) {
    launch_chained(k_render_fwd<TS, PPT, B>, a.cam.tiles_x * a.cam.tiles_y, TS * TS / PPT, s, a.splats, a.vals,
                   a.ranges, a.cam, a.image, a.t_final, a.n_last, a.frozen, a.resume, a.resume_pos);
}

template <int TS, int PPT, int B>
void launch(const BwdArgs &a, cudaStream_t s) {
    launch_chained(k_raster_bwd<TS, PPT, B>, a.cam.tiles_x * a.cam.tiles_y, TS * TS / PPT, s, a.splats, a.vals,
                   a.ranges, a.cam, a.t_final, a.n_last, a.dl, a.frozen, a.grad2d, a.resume, a.resume_pos);
}

struct BatchArgs {
    const gs_raster_job *jobs;
    int W, H, tiles_per_job, total;
    uint32_t *queue;
    bool bwd;
};

template <class K>
int resident_ctas(K kernel, int threads) {
    int per_sm = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    return (sms > 0 ? sms : 152) * per_sm;
}

template <int TS, int PPT, int B>
void launch(const BatchArgs &a, cudaStream_t s) {
    constexpr int NT = TS * TS / PPT;
    if (a.bwd) {
        const int grid = resident_ctas(k_raster_bwd_batch<TS, PPT, B>, NT);
        k_raster_bwd_batch<TS, PPT, B><<<grid, NT, 0, s>>>(a.jobs, a.W, a.H, a.tiles_per_job, a.total, a.queue);
    } else {
        const int grid = resident_ctas(k_render_fwd_batch<TS, PPT, B>, NT);
        k_render_fwd_batch<TS, PPT, B><<<grid, NT, 0, s>>>(a.jobs, a.W, a.H, a.tiles_per_job, a.total, a.queue);
    }
}

template <int TS, int PPT, class A>
void by_batch(int batch, const A &a, cudaStream_t s) {
    switch (batch) {
        case 32: launch<TS, PPT, 32>(a, s); break;
        case 64: launch<TS, PPT, 64>(a, s); break;
        case 128: launch<TS, PPT, 128>(a, s); break;
        default: launch<TS, PPT, 256>(a, s); break;
    }
}

template <class A>
int dispatch(int tile, int ppt, int batch, const A &a, cudaStream_t s) {
    switch (tile * 10 + ppt) {
        case 81: by_batch<8, 1>(batch, a, s); break;
        case 82: by_batch<8, 2>(batch, a, s); break;
        case 161: by_batch<16, 1>(batch, a, s); break;
        case 162: by_batch<16, 2>(batch, a, s); break;
        case 164: by_batch<16, 4>(batch, a, s); break;
        case 321: by_batch<32, 1>(batch, a, s); break;
        case 324: by_batch<32, 4>(batch, a, s); break;
        default: by_batch<32, 2>(batch, a, s); break;
    }
    note_launches(1);
    return launch_status();
}

// Four pixels per thread only where a tile still fills whole warps (16, 32).
inline bool config_ok(const gs_raster_config *c, int tile) {
    return !c || ((c->pixels_per_thread == 1 || c->pixels_per_thread == 2 ||
                   (c->pixels_per_thread == 4 && tile >= 16)) &&
                  (c->batch == 32 || c->batch == 64 || c->batch == 128 || c->batch == 256));
}

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" int gs_render_fwd_resume(const float *splats, const uint32_t *vals, const uint32_t *ranges,
                                    const gs_camera *cam, const gs_raster_config *cfg, const uint8_t *frozen,
                                    float *image, float *t_final, int32_t *n_last, float *resume,
                                    int32_t *resume_pos, gs_stream_t stream) {
    if (!camera_ok(cam) || !config_ok(cfg, cam->tile) || !ranges || !image || !t_final || !n_last)
        return GS_ERR_INVALID_ARG;
    if ((resume == nullptr) != (resume_pos == nullptr)) return GS_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(splats) | reinterpret_cast<uintptr_t>(resume)) & 15) return GS_ERR_INVALID_ARG;
    FwdArgs a{splats, vals, ranges, make_cam(cam), image, t_final, n_last, frozen, reinterpret_cast<float4 *>(resume),
              resume_pos};
    int ppt, batch;
    default_config(a.cam.tile, false, ppt, batch);
    if (cfg) { ppt = cfg->pixels_per_thread; batch = cfg->batch; }
    return dispatch(a.cam.tile, ppt, batch, a, as_stream(stream));
}

extern "C" int gs_render_fwd_cfg(const float *splats, const uint32_t *vals, const uint32_t *ranges,
                                 const gs_camera *cam, const gs_raster_config *cfg, float *image, float *t_final,
                                 int32_t *n_last, gs_stream_t stream) {
    return gs_render_fwd_resume(splats, vals, ranges, cam, cfg, nullptr, image, t_final, n_last, nullptr, nullptr,
                                stream);
}

extern "C" int gs_render_fwd(const float *splats, const uint32_t *vals, const uint32_t *ranges, const gs_camera *cam,
                             float *image, float *t_final, int32_t *n_last, gs_stream_t stream) {
    return gs_render_fwd_cfg(splats, vals, ranges, cam, nullptr, image, t_final, n_last, stream);
}

extern "C" int gs_raster_bwd_resume(const float *splats, const uint32_t *vals, const uint32_t *ranges,
                                    const gs_camera *cam, const gs_raster_config *cfg, const float *t_final,
                                    const int32_t *n_last, const float *dl_dimage, const uint8_t *frozen,
                                    const float *resume, const int32_t *resume_pos, float *grad2d,
                                    gs_stream_t stream) {
    if (!camera_ok(cam) || !config_ok(cfg, cam->tile) || !ranges || !t_final || !n_last || !dl_dimage || !grad2d)
        return GS_ERR_INVALID_ARG;
    if ((resume == nullptr) != (resume_pos == nullptr)) return GS_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(splats) | reinterpret_cast<uintptr_t>(resume)) & 15) return GS_ERR_INVALID_ARG;
    BwdArgs a{splats, vals, ranges, make_cam(cam), t_final, n_last, dl_dimage, frozen, grad2d,
              reinterpret_cast<const float4 *>(resume), resume_pos};
    int ppt, batch;
    default_config(a.cam.tile, true, ppt, batch);
    if (cfg) { ppt = cfg->pixels_per_thread; batch = cfg->batch; }
    return dispatch(a.cam.tile, ppt, batch, a, as_stream(stream));
}

extern "C" int gs_raster_bwd_cfg(const float *splats, const uint32_t *vals, const uint32_t *ranges,
                                 const gs_camera *cam, const gs_raster_config *cfg, const float *t_final,
                                 const int32_t *n_last, const float *dl_dimage, const uint8_t *frozen, float *grad2d,
                                 gs_stream_t stream) {
    return gs_raster_bwd_resume(splats, vals, ranges, cam, cfg, t_final, n_last, dl_dimage, frozen, nullptr, nullptr,
                                grad2d, stream);
}

extern "C" int gs_raster_bwd(const float *splats, const uint32_t *vals, const uint32_t *ranges, const gs_camera *cam,
                             const float *t_final, const int32_t *n_last, const float *dl_dimage,
                             const uint8_t *frozen, float *grad2d, gs_stream_t stream) {
    return gs_raster_bwd_cfg(splats, vals, ranges, cam, nullptr, t_final, n_last, dl_dimage, frozen, grad2d, stream);
}

static int batch_common(const gs_raster_job *jobs_dev, int32_t n_jobs, int32_t width, int32_t height, int32_t tile,
                        const gs_raster_config *cfg, uint32_t *queue_dev, gs_stream_t stream, bool bwd) {
    if (!jobs_dev || !queue_dev || n_jobs < 0 || width <= 0 || height <= 0 || !tile_ok(tile) ||
        !config_ok(cfg, tile))
        return GS_ERR_INVALID_ARG;
    if (n_jobs == 0) return GS_OK;
    const int64_t tiles = (int64_t)((width + tile - 1) / tile) * ((height + tile - 1) / tile);
    if (tiles * n_jobs > INT32_MAX) return GS_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    if (cudaMemsetAsync(queue_dev, 0, sizeof(uint32_t), s) != cudaSuccess) return GS_ERR_CUDA;
    BatchArgs a{jobs_dev, width, height, (int)tiles, (int)(tiles * n_jobs), queue_dev, bwd};
    int ppt, batch;
    default_config(tile, bwd, ppt, batch);
    if (cfg) { ppt = cfg->pixels_per_thread; batch = cfg->batch; }
    return dispatch(tile, ppt, batch, a, s);
}

extern "C" int gs_render_fwd_batch(const gs_raster_job *jobs_dev, int32_t n_jobs, int32_t width, int32_t height,
                                   int32_t tile, const gs_raster_config *cfg, uint32_t *queue_dev, gs_stream_t stream) {
    return batch_common(jobs_dev, n_jobs, width, height, tile, cfg, queue_dev, stream, false);
}

extern "C" int gs_raster_bwd_batch(const gs_raster_job *jobs_dev, int32_t n_jobs, int32_t width, int32_t height,
                                   int32_t tile, const gs_raster_config *cfg, uint32_t *queue_dev, gs_stream_t stream) {
    return batch_common(jobs_dev, n_jobs, width, height, tile, cfg, queue_dev, stream, true);
}

namespace gs {
uint32_t take_render_flags() {
    uint32_t f = 0, z = 0;
    cudaMemcpyFromSymbol(&f, g_render_flags, sizeof(f));
    cudaMemcpyToSymbol(g_render_flags, &z, sizeof(z));
    return f;
}
}  // namespace gs

extern "C" int gs_raster_pair_counts(const float *splats, const uint32_t *vals, const uint32_t *ranges,
                                     const gs_camera *cam, const int32_t *n_last, const uint8_t *frozen,
                                     uint64_t *counts_dev, gs_stream_t stream) {
    if (!camera_ok(cam) || !splats || !vals || !ranges || !n_last || !counts_dev) return GS_ERR_INVALID_ARG;
    const DevCam dc = make_cam(cam);
    k_pair_counts<<<dc.tiles_x * dc.tiles_y, dc.tile * dc.tile, 0, as_stream(stream)>>>(
        splats, vals, ranges, dc, n_last, frozen, reinterpret_cast<unsigned long long *>(counts_dev));
    note_launches(1);
    return launch_status();
}

extern "C" int gs_hit_counts(const float *splats, const uint32_t *vals, const uint32_t *ranges, const gs_camera *cam,
                             const int32_t *n_last, uint32_t *hits_dev, gs_stream_t stream) {
    if (!camera_ok(cam) || !splats || !vals || !ranges || !n_last || !hits_dev) return GS_ERR_INVALID_ARG;
    const DevCam dc = make_cam(cam);
    k_hit_counts<<<dc.tiles_x * dc.tiles_y, dc.tile * dc.tile, 0, as_stream(stream)>>>(splats, vals, ranges, dc,
                                                                                      n_last, hits_dev);
    note_launches(1);
    return launch_status();
}
