// Per-tile depth order of splats (Sec. 3.1: colours are blended "in a sorted
// order").
//
// The result equals a stable sort of the 64-bit keys (tile << 32 | depth
// bits) generated in Gaussian order, but no (Gaussian, tile) entry is ever
// sorted:
//   1. compact the visible Gaussians (ascending index) and LSD-radix-sort
//      them by the bits of their float32 depth (4 passes of 8 bits over the
//      visible Gaussians only; stable, so equal depths keep index order);
//   2. in that depth order, emit one entry per super-tile (8 x 8 tiles) a
//      Gaussian's tile rectangle meets -- about one per Gaussian -- and
//      stable-sort those few entries by super-tile id (1-2 radix passes);
//   3. split each super-tile's depth-ordered list into chunks of 256; per
//      chunk, every entry's 64-bit mask of the tiles that list it (see the
//      tile membership rule below) and one warp ballot
//      per tile give the entry's rank among the chunk's entries of that tile;
//      a scan over the chunks of a super-tile and one over the tile counts
//      give every tile's start (the ranges) and every entry's final place,
//      written once: in depth order, then index order, inside each tile.
// All counts live on the device; nothing waits on the host.
#include "common.cuh"

namespace gs {

__device__ uint32_t g_sort_flags;

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 4;
constexpr int kSortBlock = kSortThreads * kSortItems;  // keys per radix block
constexpr int kMaxRadixBits = 9;                       // digits of up to 9 bits (512 buckets) per pass
constexpr int kMaxRadix = 1 << kMaxRadixBits;
constexpr int kScanBlock = 1024;                       // elements per scan block

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

template <typename T>
__device__ __forceinline__ T block_scan_excl(T v, T *warp_sums, T *total) {
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        T w = lane < nwarps ? warp_sums[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(kFull, w, o);
            if (lane >= o) w += y;
        }
        warp_sums[lane] = w;
    }
    __syncthreads();
    T before = warp > 0 ? warp_sums[warp - 1] : T(0);
    *total = warp_sums[nwarps - 1];
    __syncthreads();
    return before + x - v;
}

__device__ __forceinline__ bool splat_visible(const float *splats, int64_t i) {
    return __float_as_int(__ldg(splats + i * kSplat + 11)) > 0;
}

// ---- stage 1a: compaction of visible Gaussians ----
// Also zeroes the sort's counters: `zero` [nzero] words and *total_exact.
__global__ void __launch_bounds__(kScanBlock) k_count_visible(const float *__restrict__ splats, int64_t n,
                                                             uint32_t *__restrict__ part, uint32_t *__restrict__ zero,
                                                             int64_t nzero,
                                                             unsigned long long *__restrict__ total_exact) {
    wait_prior_grid();
    int64_t i = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
    for (int64_t z = i; z < nzero; z += (int64_t)gridDim.x * kScanBlock) zero[z] = 0u;
    if (i == 0) *total_exact = 0ull;
    int f = (i < n) && splat_visible(splats, i);
    int c = __syncthreads_count(f);
    if (threadIdx.x == 0) part[blockIdx.x] = (uint32_t)c;
}

// Exclusive scan of part[0..nb) in place by one block; total to *total. With
// clip given: *clip = min(total, capacity), and the capacity flag if the
// total exceeds it (the super-tile entries kept).
template <typename T>
__global__ void __launch_bounds__(1024) k_scan_parts(T *__restrict__ part, int nb, T *__restrict__ total,
                                                     uint32_t *__restrict__ clip, int64_t capacity) {
    wait_prior_grid();
    __shared__ T ws[32];
    T carry = 0;
    for (int base = 0; base < nb; base += 1024) {
        int j = base + threadIdx.x;
        T v = j < nb ? part[j] : T(0), tot;
        T ex = block_scan_excl<T>(v, ws, &tot);
        if (j < nb) part[j] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) {
        *total = carry;
        if (clip) {
            const unsigned long long Q = (unsigned long long)carry;
            *clip = (uint32_t)(Q > (unsigned long long)capacity ? capacity : Q);
            if (Q > (unsigned long long)capacity) atomicOr(&g_sort_flags, GS_FLAG_CAPACITY);
        }
    }
}

// ---- LSD radix pass: histogram, per-digit row scan, stable scatter ----
// The number of keys lives on the device; the three kernels derive the same
// block count nbd from it and loop over those blocks with whatever grid the
// host launched (sized for the device, not for the worst case). hist is
// [radix][nbd].
__device__ __forceinline__ int radix_blocks(const uint32_t *count) {
    return (int)((*count + kSortBlock - 1) / kSortBlock);
}

__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const uint32_t *__restrict__ keys,
                                                            const uint32_t *__restrict__ count, int shift, int bits,
                                                            uint32_t *__restrict__ hist) {
    wait_prior_grid();
    __shared__ uint32_t h[kMaxRadix];
    const int radix = 1 << bits;
    const uint32_t mask = (uint32_t)radix - 1u;
    const uint32_t n = *count;
    const int nbd = radix_blocks(count);
    for (int b = blockIdx.x; b < nbd; b += gridDim.x) {
        for (int d = threadIdx.x; d < radix; d += kSortThreads) h[d] = 0;
        __syncthreads();
        const int64_t base = (int64_t)b * kSortBlock;
#pragma unroll
        for (int r = 0; r < kSortItems; ++r) {
            int64_t i = base + r * kSortThreads + threadIdx.x;
            if (i < n) atomicAdd(&h[(keys[i] >> shift) & mask], 1u);
        }
        __syncthreads();
        for (int d = threadIdx.x; d < radix; d += kSortThreads) hist[(int64_t)d * nbd + b] = h[d];
        __syncthreads();
    }
}

__global__ void __launch_bounds__(1024) k_radix_rowscan(uint32_t *__restrict__ hist, const uint32_t *__restrict__ count,
                                                        uint32_t *__restrict__ digit_total) {
    wait_prior_grid();
    __shared__ uint32_t ws[32];
    const int nb = radix_blocks(count);
    uint32_t *row = hist + (int64_t)blockIdx.x * nb;
    uint32_t carry = 0;
    for (int base = 0; base < nb; base += 1024) {
        int j = base + threadIdx.x;
        uint32_t v = j < nb ? row[j] : 0u, tot;
        uint32_t ex = block_scan_excl<uint32_t>(v, ws, &tot);
        if (j < nb) row[j] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) digit_total[blockIdx.x] = carry;
}

// Where a one-pass sort by super-tile id leaves each super-tile's entries:
// its digit's range of the output. Given (chunk_base non-null), block 0 of
// the pass writes the chunk plan from the digit totals: chunk_base [ns + 1]
// (exclusive scan of ceil(len / chunk)) and chunk_rec (per chunk: its
// super-tile, first entry, the segment's end and the super-tile's first
// chunk).
struct SegPlan {
    uint32_t *chunk_base;
    uint4 *chunk_rec;
    int ns, chunk;
};

__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(const uint32_t *__restrict__ kin,
                                                               const uint32_t *__restrict__ vin,
                                                               uint32_t *__restrict__ kout, uint32_t *__restrict__ vout,
                                                               const uint32_t *__restrict__ count, int shift, int bits,
                                                               const uint32_t *__restrict__ hist,
                                                               const uint32_t *__restrict__ digit_total, SegPlan sp) {
    wait_prior_grid();
    constexpr int kWarps = kSortThreads / 32;
    constexpr int kPer = kMaxRadix / kSortThreads;  // buckets per thread (consecutive)
    __shared__ uint32_t run[kMaxRadix];
    __shared__ uint32_t wc[kWarps][kMaxRadix];
    __shared__ uint32_t ws[32];
    const uint32_t n = *count;
    const int nbd = radix_blocks(count);
    const bool plan = sp.chunk_base && blockIdx.x == 0;
    if ((int)blockIdx.x >= nbd && !plan) return;
    const int radix = 1 << bits;
    const uint32_t mask = (uint32_t)radix - 1u;
    const int t = threadIdx.x, warp = t >> 5;
    // exclusive scan of the bucket totals: thread t owns buckets kPer t .. kPer t + kPer - 1
    uint32_t dtot[kPer], own = 0u, tot;
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
        const int d = kPer * t + q;
        dtot[q] = d < radix ? digit_total[d] : 0u;
        own += dtot[q];
    }
    uint32_t dbase[kPer];
    dbase[0] = block_scan_excl<uint32_t>(own, ws, &tot);
#pragma unroll
    for (int q = 1; q < kPer; ++q) dbase[q] = dbase[q - 1] + dtot[q - 1];
    if (plan) {  // block-uniform
        uint32_t nc[kPer], ncown = 0u, nctot;
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const int d = kPer * t + q;
            nc[q] = d < sp.ns ? (dtot[q] + (uint32_t)sp.chunk - 1u) / (uint32_t)sp.chunk : 0u;
            ncown += nc[q];
        }
        uint32_t cb = block_scan_excl<uint32_t>(ncown, ws, &nctot);
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const int d = kPer * t + q;
            if (d < sp.ns) {
                sp.chunk_base[d] = cb;
                for (uint32_t c = 0; c < nc[q]; ++c)
                    sp.chunk_rec[cb + c] = make_uint4((uint32_t)d, dbase[q] + c * (uint32_t)sp.chunk,
                                                      dbase[q] + dtot[q], cb);
            }
            cb += nc[q];
        }
        if (t == 0) sp.chunk_base[sp.ns] = nctot;
        if ((int)blockIdx.x >= nbd) return;
    }
    for (int b = blockIdx.x; b < nbd; b += gridDim.x) {
        const int64_t base = (int64_t)b * kSortBlock;
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const int d = kPer * t + q;
            if (d < radix) run[d] = dbase[q] + hist[(int64_t)d * nbd + b];
        }
        // all of the block's keys and values in flight at once; then ranked
        // and written a sub-block of kSortThreads at a time, in order
        uint32_t kr[kSortItems], vr[kSortItems];
#pragma unroll
        for (int r = 0; r < kSortItems; ++r) {
            const int64_t i = base + r * kSortThreads + t;
            kr[r] = i < n ? kin[i] : 0u;
            vr[r] = i < n ? vin[i] : 0u;
        }
#pragma unroll
        for (int r = 0; r < kSortItems; ++r) {
            int64_t i = base + r * kSortThreads + t;
            bool valid = i < n;
            uint32_t key = kr[r];
            uint32_t d = valid ? ((key >> shift) & mask) : 0xffffu;
            unsigned peers = __match_any_sync(kFull, d);
            unsigned lrank = __popc(peers & lanemask_lt());
            for (int e = t; e < radix; e += kSortThreads) {
#pragma unroll
                for (int w = 0; w < kWarps; ++w) wc[w][e] = 0u;
            }
            __syncthreads();
            if (valid && lrank == 0) wc[warp][d] = (uint32_t)__popc(peers);
            __syncthreads();
            for (int e = t; e < radix; e += kSortThreads) {
                uint32_t c = run[e];
#pragma unroll
                for (int w = 0; w < kWarps; ++w) {
                    uint32_t x = wc[w][e];
                    wc[w][e] = c;
                    c += x;
                }
                run[e] = c;
            }
            __syncthreads();
            if (valid) {
                uint32_t pos = wc[warp][d] + lrank;
                kout[pos] = key;
                vout[pos] = vr[r];
            }
            __syncthreads();
        }
    }
}

// Blocks of 256 threads the device holds at once (grids of the loops above).
int64_t resident_blocks() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return (int64_t)(sms > 0 ? sms : 152) * 8;
}

__global__ void k_zero_u32(uint32_t *__restrict__ p, int64_t n) {
    wait_prior_grid();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = 0u;
}

// ---- stage 2: super-tile entries in depth order ----
constexpr int kSuper = 8;       // a super-tile is kSuper x kSuper tiles (64 = one bit each)
constexpr int kChunk = 256;     // super-tile list entries per chunk (one per thread)

__device__ __forceinline__ int splat_rect(const float *splats, uint32_t g, const DevCam &cam, int &x0, int &y0,
                                          int &x1, int &y1) {
    const float *r = splats + (int64_t)g * kSplat;
    int rad = __float_as_int(__ldg(r + 10));
    if (rad <= 0) { x0 = y0 = x1 = y1 = 0; return 0; }
    return tile_rect(__ldg(r), __ldg(r + 1), rad, cam.tile, cam.tiles_x, cam.tiles_y, x0, y0, x1, y1);
}

__device__ __forceinline__ int super_rect(int x0, int y0, int x1, int y1, int &sx0, int &sy0, int &sx1, int &sy1) {
    sx0 = x0 / kSuper; sy0 = y0 / kSuper;
    sx1 = (x1 - 1) / kSuper + 1; sy1 = (y1 - 1) / kSuper + 1;
    return (sx1 - sx0) * (sy1 - sy0);
}

// ---- tile membership ----
// A tile of a splat's 3-sigma rectangle lists the splat only if the box of its
// pixel centres [X, X + T - 1] x [Y, Y + T - 1] holds a point where the
// conic's quadratic form q = a dx^2 + 2 b dx dy + c dy^2 is at most
// tau + 1e-3 (1 + tau), tau = 2 ln(255 o): elsewhere alpha = o exp(-q/2) is
// below the 1/255 floor of Eq. 2 at every pixel of the tile, so leaving the
// splat out changes no image and no gradient. A splat with 255 o < 1 is
// listed nowhere. Decided in single precision, every operation rounded
// (explicit intrinsics, no contraction); the 1e-3 relative margin makes the
// lists a superset of the tiles that hold a pixel centre with alpha >= 1/255
// exactly, so float32 rounding never drops a contribution.

// ln x for x >= 1: x = m 2^e, m in [1, 2); ln m = 2 atanh(s), s = (m-1)/(m+1),
// by the series 2 s (1 + s^2/3 + ... + s^14/15).
__device__ __forceinline__ float ln_f32(float x) {
    const uint32_t b = __float_as_uint(x);
    const int e = (int)((b >> 23) & 0xffu) - 127;
    const float m = __uint_as_float((b & 0x007fffffu) | 0x3f800000u);
    const float s = __fdiv_rn(__fsub_rn(m, 1.f), __fadd_rn(m, 1.f));
    const float s2 = __fmul_rn(s, s);
    float p = 0.0666666667f;
    p = __fadd_rn(__fmul_rn(p, s2), 0.0769230769f);
    p = __fadd_rn(__fmul_rn(p, s2), 0.0909090909f);
    p = __fadd_rn(__fmul_rn(p, s2), 0.111111111f);
    p = __fadd_rn(__fmul_rn(p, s2), 0.142857143f);
    p = __fadd_rn(__fmul_rn(p, s2), 0.2f);
    p = __fadd_rn(__fmul_rn(p, s2), 0.333333333f);
    p = __fadd_rn(__fmul_rn(p, s2), 1.f);
    return __fadd_rn(__fmul_rn((float)e, 0.693147181f), __fmul_rn(__fmul_rn(2.f, s), p));
}

// The bound on q with its margin; negative when the splat is listed nowhere.
__device__ __forceinline__ float tile_tau(float opacity) {
    const float x = __fmul_rn(255.f, opacity);
    if (!(x >= 1.f)) return -1.f;
    const float tau = __fmul_rn(2.f, ln_f32(x));
    return __fadd_rn(tau, __fmul_rn(1e-3f, __fadd_rn(1.f, tau)));
}

__device__ __forceinline__ float quad_f32(float a, float b, float c, float dx, float dy) {
    return __fadd_rn(__fadd_rn(__fmul_rn(__fmul_rn(a, dx), dx), __fmul_rn(__fmul_rn(__fmul_rn(2.f, b), dx), dy)),
                     __fmul_rn(__fmul_rn(c, dy), dy));
}

struct SplatShape {
    float mx, my, a, b, c, tau, bc, ba;  // bc = b / c, ba = b / a
};

__device__ __forceinline__ SplatShape splat_shape(const float *splats, uint32_t g) {
    const float4 *r = reinterpret_cast<const float4 *>(splats + (int64_t)g * kSplat);
    const float4 p0 = __ldg(r), p1 = __ldg(r + 1);
    SplatShape sh;
    sh.mx = p0.x; sh.my = p0.y; sh.a = p0.z; sh.b = p0.w; sh.c = p1.x;
    sh.tau = tile_tau(p1.y);
    sh.bc = __fdiv_rn(sh.b, sh.c);
    sh.ba = __fdiv_rn(sh.b, sh.a);
    return sh;
}

// Whether tile (x, y) lists the splat: the box minimum of q is 0 when the mean
// lies inside, else the least of the four edges' clamped one-dimensional
// minima (on x = X at y = my - (b/c)(X - mx), on y = Y at x = mx - (b/a)(Y - my)).
__device__ __forceinline__ bool tile_hit(const SplatShape &sh, int tile, int x, int y) {
    if (sh.tau < 0.f) return false;
    const float x0 = (float)(x * tile), x1 = (float)(x * tile + tile - 1);
    const float y0 = (float)(y * tile), y1 = (float)(y * tile + tile - 1);
    if (sh.mx >= x0 && sh.mx <= x1 && sh.my >= y0 && sh.my <= y1) return true;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float ex = k ? x1 : x0, ey = k ? y1 : y0;
        const float dx = __fsub_rn(ex, sh.mx);
        const float yo = __fsub_rn(sh.my, __fmul_rn(sh.bc, dx));
        const float yy = yo < y0 ? y0 : (yo > y1 ? y1 : yo);
        if (quad_f32(sh.a, sh.b, sh.c, dx, __fsub_rn(yy, sh.my)) <= sh.tau) return true;
        const float dy = __fsub_rn(ey, sh.my);
        const float xo = __fsub_rn(sh.mx, __fmul_rn(sh.ba, dy));
        const float xx = xo < x0 ? x0 : (xo > x1 ? x1 : xo);
        if (quad_f32(sh.a, sh.b, sh.c, __fsub_rn(xx, sh.mx), dy) <= sh.tau) return true;
    }
    return false;
}

// The tiles a splat may be listed in: its 3-sigma rectangle, narrowed to the
// bounding box of the ellipse q <= tau when that box is provably wide
// enough. tile_hit evaluates q = a dx^2 + 2 b dx dy + c dy^2 (float32) only
// at points of a tile's pixel-centre box, and min over dy of q is
// dx^2 det / c (det = a c - b^2), so q > tau wherever |dx| >= sqrt(tau c /
// det). The rounding error of q is at most 4 u kappa q (u = 2^-24) with
// kappa = (a + |b| + c)(a + c) / det >= (|a| dx^2 + 2 |b dx dy| + c dy^2) / q,
// and det carries a relative error of about 2 u kappa; for kappa <= 1e4 both
// stay below 0.3%, well inside the 4% that the factor 1.02 on the box's half
// widths leaves (plus a pixel). Ill-conditioned conics keep the rectangle.
// So every tile dropped here fails tile_hit: the lists are unchanged.
__device__ __forceinline__ int cand_rect(const float *splats, uint32_t g, const DevCam &cam, float tau, int &x0,
                                         int &y0, int &x1, int &y1) {
    if (!splat_rect(splats, g, cam, x0, y0, x1, y1)) return 0;
    const float *r = splats + (int64_t)g * kSplat;
    const float mx = __ldg(r), my = __ldg(r + 1), a = __ldg(r + 2), b = __ldg(r + 3), c = __ldg(r + 4);
    const float det = a * c - b * b;
    if (!(tau >= 0.f) || !(det > 0.f) || !(a > 0.f) || !(c > 0.f)) return 1;
    const float kappa = (a + fabsf(b) + c) * (a + c) / det;
    if (!(kappa <= 1e4f)) return 1;
    const float hx = sqrtf(tau * c / det) * 1.02f + 1.f;
    const float hy = sqrtf(tau * a / det) * 1.02f + 1.f;
    const float inv = 1.f / (float)cam.tile;  // exact: a power of two
    x0 = max(x0, (int)floorf((mx - hx) * inv));
    x1 = min(x1, (int)floorf((mx + hx) * inv) + 1);
    y0 = max(y0, (int)floorf((my - hy) * inv));
    y1 = min(y1, (int)floorf((my + hy) * inv) + 1);
    if (x0 >= x1 || y0 >= y1) {
        x0 = y0 = x1 = y1 = 0;
        return 0;
    }
    return 1;
}

// The tile tests' constants and the candidate rectangle of a visible
// Gaussian, computed once per sort (k_emit_visible) and read by the
// depth-ordered passes and the chunk kernels: cull[2 g] = (tau, b / c, b / a,
// 0), cull[2 g + 1] = (x0 | y0 << 16, x1 | y1 << 16, 0, 0) as integers, the
// empty rectangle when no tile can list the splat (255 o < 1).
__device__ __forceinline__ void write_cull(const float *splats, uint32_t g, const DevCam &cam, float4 *cull) {
    const SplatShape sh = splat_shape(splats, g);
    int x0 = 0, y0 = 0, x1 = 0, y1 = 0;
    if (!(sh.tau >= 0.f) || !cand_rect(splats, g, cam, sh.tau, x0, y0, x1, y1)) x0 = y0 = x1 = y1 = 0;
    cull[2 * (int64_t)g] = make_float4(sh.tau, sh.bc, sh.ba, 0.f);
    reinterpret_cast<uint4 *>(cull)[2 * (int64_t)g + 1] =
        make_uint4((uint32_t)x0 | ((uint32_t)y0 << 16), (uint32_t)x1 | ((uint32_t)y1 << 16), 0u, 0u);
}

// Tile coordinates are below 2^16 (images of at most 16384 pixels a side).
__device__ __forceinline__ bool cull_rect(const float4 *cull, uint32_t g, int &x0, int &y0, int &x1, int &y1) {
    const uint4 r = __ldg(reinterpret_cast<const uint4 *>(cull) + 2 * (int64_t)g + 1);
    x0 = (int)(r.x & 0xffffu);
    y0 = (int)(r.x >> 16);
    x1 = (int)(r.y & 0xffffu);
    y1 = (int)(r.y >> 16);
    return x0 < x1 && y0 < y1;
}

// The depth keys and indices of the visible Gaussians, ascending index, and
// their cull records.
__global__ void __launch_bounds__(kScanBlock) k_emit_visible(const float *__restrict__ splats, int64_t n,
                                                            const uint32_t *__restrict__ part, DevCam cam,
                                                            uint32_t *__restrict__ keys, uint32_t *__restrict__ vals,
                                                            float4 *__restrict__ cull) {
    wait_prior_grid();
    __shared__ int ws[32];
    int64_t i = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
    int f = (i < n) && splat_visible(splats, i);
    int tot;
    int r = block_scan_excl<int>(f, ws, &tot);
    if (f) {
        uint32_t pos = part[blockIdx.x] + (uint32_t)r;
        keys[pos] = __float_as_uint(__ldg(splats + i * kSplat + 9));
        vals[pos] = (uint32_t)i;
        write_cull(splats, (uint32_t)i, cam, cull);
    }
}

// Per block of depth-ordered Gaussians: its super-tile entries (part_s).
// Only splats some tile can list (255 o >= 1) get entries.
__device__ __forceinline__ unsigned long long super_entries(const float4 *cull, uint32_t g, int &sx0, int &sy0,
                                                            int &sx1, int &sy1) {
    int x0, y0, x1, y1;
    if (!cull_rect(cull, g, x0, y0, x1, y1)) return 0ull;
    return (unsigned long long)super_rect(x0, y0, x1, y1, sx0, sy0, sx1, sy1);
}

__global__ void __launch_bounds__(kScanBlock) k_count_entries(const float4 *__restrict__ cull,
                                                             const uint32_t *__restrict__ order,
                                                             const uint32_t *__restrict__ n_vis,
                                                             unsigned long long *__restrict__ part_s) {
    wait_prior_grid();
    __shared__ unsigned long long ws[32];
    int64_t k = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
    int sx0, sy0, sx1, sy1;
    const unsigned long long cs = k < *n_vis ? super_entries(cull, order[k], sx0, sy0, sx1, sy1) : 0ull;
    unsigned long long tot;
    block_scan_excl<unsigned long long>(cs, ws, &tot);
    if (threadIdx.x == 0) part_s[blockIdx.x] = tot;
}

// Only when the super-tile entries alone overflowed the capacity (then the
// tile counts miss the dropped ones): P counted splat by splat, tile by tile.
// The tiles that list splat g, counted one by one.
__device__ __forceinline__ unsigned long long exact_tiles(const float *splats, uint32_t g, const DevCam &cam) {
    int x0, y0, x1, y1;
    const SplatShape sh = splat_shape(splats, g);
    if (sh.tau < 0.f || !cand_rect(splats, g, cam, sh.tau, x0, y0, x1, y1)) return 0ull;
    unsigned long long m = 0ull;
    for (int y = y0; y < y1; ++y)
        for (int x = x0; x < x1; ++x) m += tile_hit(sh, cam.tile, x, y) ? 1ull : 0ull;
    return m;
}

// A warp's sum of v added to *total (every lane of the warp calls it).
__device__ __forceinline__ void warp_add_total(unsigned long long v, unsigned long long *total) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(total, v);
}

__global__ void __launch_bounds__(256) k_count_exact(const float *__restrict__ splats,
                                                    const uint32_t *__restrict__ order,
                                                    const uint32_t *__restrict__ n_vis, DevCam cam,
                                                    const unsigned long long *__restrict__ total_s, int64_t capacity,
                                                    unsigned long long *__restrict__ total_exact) {
    wait_prior_grid();
    if (*total_s <= (unsigned long long)capacity) return;
    unsigned long long mine = 0ull;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < *n_vis;
         k += (int64_t)gridDim.x * blockDim.x)
        mine += exact_tiles(splats, order[k], cam);
    warp_add_total(mine, total_exact);
}

// count_dev = P, the number of entries: the sum of the tile counts, or the
// exact count above when the super-tile entries overflowed.
__global__ void k_finish_count(const unsigned long long *__restrict__ total_t,
                               const unsigned long long *__restrict__ total_s,
                               const unsigned long long *__restrict__ total_exact, int64_t capacity,
                               int64_t *__restrict__ count_dev) {
    wait_prior_grid();
    const unsigned long long P = *total_s > (unsigned long long)capacity ? *total_exact : *total_t;
    *count_dev = (int64_t)P;
    if (P > (unsigned long long)capacity) atomicOr(&g_sort_flags, GS_FLAG_CAPACITY);
}

__global__ void __launch_bounds__(kScanBlock) k_emit_super(const float *__restrict__ splats,
                                                          const float4 *__restrict__ cull,
                                                          const uint32_t *__restrict__ order,
                                                          const uint32_t *__restrict__ n_vis, DevCam cam,
                                                          int supers_x, const unsigned long long *__restrict__ part_s,
                                                          const unsigned long long *__restrict__ total_s,
                                                          int64_t capacity, uint32_t *__restrict__ skeys,
                                                          uint32_t *__restrict__ svals,
                                                          unsigned long long *__restrict__ total_exact) {
    wait_prior_grid();
    __shared__ unsigned long long ws[32];
    int64_t k = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
    int sx0 = 0, sy0 = 0, sx1 = 0, sy1 = 0;
    uint32_t g = 0;
    unsigned long long c = 0ull;
    if (k < *n_vis) {
        g = order[k];
        c = super_entries(cull, g, sx0, sy0, sx1, sy1);
    }
    unsigned long long tot;
    unsigned long long off = part_s[blockIdx.x] + block_scan_excl<unsigned long long>(c, ws, &tot);
    if (*total_s > (unsigned long long)capacity)  // the super-tile entries overflowed: P counted tile by tile
        warp_add_total(c ? exact_tiles(splats, g, cam) : 0ull, total_exact);
    if (c == 0) return;
    for (int y = sy0; y < sy1; ++y)
        for (int x = sx0; x < sx1; ++x) {
            if (off >= (unsigned long long)capacity) return;
            skeys[off] = (uint32_t)(y * supers_x + x);
            svals[off] = g;
            ++off;
        }
}

// Segments of the super-tile-sorted list: seg_lo / seg_hi [ns] (zero for an
// empty super-tile; both arrays zeroed before).
__global__ void __launch_bounds__(256) k_seg_mark(const uint32_t *__restrict__ skeys,
                                                 const uint32_t *__restrict__ count, uint32_t *__restrict__ seg_lo,
                                                 uint32_t *__restrict__ seg_hi) {
    wait_prior_grid();
    const uint32_t n = *count;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t k = skeys[e];
        if (e == 0 || skeys[e - 1] != k) seg_lo[k] = (uint32_t)e;
        if (e == (int64_t)n - 1 || skeys[e + 1] != k) seg_hi[k] = (uint32_t)(e + 1);
    }
}

// One block: chunk bases, chunk_base [ns + 1] (exclusive scan of
// ceil(len / kChunk)), and the record of every chunk, chunk_rec [chunks] (as
// the one-pass radix writes them).
__global__ void __launch_bounds__(1024) k_super_plan(const uint32_t *__restrict__ seg_lo,
                                                     const uint32_t *__restrict__ seg_hi, int ns,
                                                     uint32_t *__restrict__ chunk_base,
                                                     uint4 *__restrict__ chunk_rec) {
    wait_prior_grid();
    __shared__ uint32_t ws[32];
    uint32_t carry = 0;
    for (int base = 0; base < ns; base += 1024) {
        const int j = base + threadIdx.x;
        const uint32_t nc = j < ns ? (seg_hi[j] - seg_lo[j] + kChunk - 1) / kChunk : 0u;
        uint32_t tot;
        const uint32_t ex = block_scan_excl<uint32_t>(nc, ws, &tot);
        if (j < ns) {
            chunk_base[j] = carry + ex;
            for (uint32_t c = 0; c < nc; ++c)
                chunk_rec[carry + ex + c] = make_uint4((uint32_t)j, seg_lo[j] + c * kChunk, seg_hi[j], carry + ex);
        }
        carry += tot;
    }
    if (threadIdx.x == 0) chunk_base[ns] = carry;
}

// Shared part of the chunk kernels for chunk c: this thread's entry and the
// mask of the tiles of the super-tile that list it.
struct ChunkCtx {
    int s, sx, sy;
    uint32_t first;  // the super-tile's first chunk
    uint32_t g;
    unsigned long long mask;
};

// Scratch of the tile tests (shared memory, one slot per thread): hit
// masks as two 32-bit halves, the entry's shape and its candidate
// rectangle packed as lx0 | ly0 << 3 | w << 6 | ceil(512 / w) << 10.
struct TestScratch {
    uint32_t *hit;  // [2 * kChunk]
    float4 *shape;  // [2 * kChunk]
    uint32_t *rect; // [kChunk]
};

// With masks_in NULL the masks are computed by the tile test (and stored to
// masks_out when given); else they are read.
__device__ __forceinline__ void chunk_load(ChunkCtx &cx, uint32_t c, const float *__restrict__ splats,
                                           const float4 *__restrict__ cull,
                                           const uint32_t *__restrict__ svals,
                                           const uint4 *__restrict__ chunk_rec, int supers_x,
                                           const DevCam &cam, const TestScratch &sc,
                                           const unsigned long long *__restrict__ masks_in,
                                           unsigned long long *__restrict__ masks_out) {
    __syncthreads();  // the previous chunk's shared data is no longer read
    const uint4 cr = chunk_rec[c];
    cx.s = (int)cr.x;
    cx.first = cr.w;
    cx.sx = cx.s % supers_x;
    cx.sy = cx.s / supers_x;
    const uint32_t e = cr.y + threadIdx.x;
    const bool valid = e < cr.z;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    cx.mask = 0ull;
    cx.g = valid ? svals[e] : 0u;
    if (masks_in) {
        if (valid) cx.mask = masks_in[e];
        return;
    }
    // candidate tiles: the entry's rectangle inside this super-tile, w x h
    // tiles from (lx0, ly0) in the super-tile's own tile coordinates
    int lx0 = 0, ly0 = 0, w = 0, h = 0;
    SplatShape sh{};
    int x0, y0, x1, y1;
    if (valid) {  // every listed entry's splat has tau >= 0 and a candidate rectangle
        const float *r = splats + (int64_t)cx.g * kSplat;
        const float4 p0 = __ldg(reinterpret_cast<const float4 *>(r));
        const float4 c0 = __ldg(cull + 2 * (int64_t)cx.g);
        sh.mx = p0.x; sh.my = p0.y; sh.a = p0.z; sh.b = p0.w;
        sh.c = __ldg(r + 4);
        sh.tau = c0.x; sh.bc = c0.y; sh.ba = c0.z;
        if (cull_rect(cull, cx.g, x0, y0, x1, y1)) {
            lx0 = max(x0 - cx.sx * kSuper, 0);
            ly0 = max(y0 - cx.sy * kSuper, 0);
            w = max(min(x1 - cx.sx * kSuper, kSuper) - lx0, 0);
            h = max(min(y1 - cx.sy * kSuper, kSuper) - ly0, 0);
        }
    }
    const int cnt = w * h;
    sc.shape[2 * threadIdx.x] = make_float4(sh.mx, sh.my, sh.a, sh.b);
    sc.shape[2 * threadIdx.x + 1] = make_float4(sh.c, sh.tau, sh.bc, sh.ba);
    // k / w = (k * ceil(512 / w)) >> 9 exactly for k < 64, w <= 8
    sc.rect[threadIdx.x] = cnt ? (uint32_t)(lx0 | (ly0 << 3) | (w << 6) | (((512 + w - 1) / w) << 10)) : 0u;
    sc.hit[2 * threadIdx.x] = 0u;
    sc.hit[2 * threadIdx.x + 1] = 0u;
    // the warp's (entry, tile) candidates, spread evenly over its lanes
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    const int excl = incl - cnt, total = __shfl_sync(kFull, incl, 31);
    __syncwarp();
    for (int base = 0; base < total; base += 32) {
        const int j = base + lane;
        int i = 0;  // owner: the last lane whose first candidate index is <= j
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const int ex = __shfl_sync(kFull, excl, i + step);
            if (ex <= j) i += step;
        }
        const int k = j - __shfl_sync(kFull, excl, i);
        if (j < total) {
            const int o = warp * 32 + i;
            const uint32_t pk = sc.rect[o];
            const int ow = (int)((pk >> 6) & 15u);
            const int q = (k * (int)(pk >> 10)) >> 9, r = k - q * ow;
            const int t = ((int)((pk >> 3) & 7u) + q) * kSuper + (int)(pk & 7u) + r;
            const float4 s0 = sc.shape[2 * o], s1 = sc.shape[2 * o + 1];
            SplatShape os;
            os.mx = s0.x; os.my = s0.y; os.a = s0.z; os.b = s0.w;
            os.c = s1.x; os.tau = s1.y; os.bc = s1.z; os.ba = s1.w;
            if (tile_hit(os, cam.tile, cx.sx * kSuper + (t & 7), cx.sy * kSuper + (t >> 3)))
                atomicOr(&sc.hit[2 * o + (t >> 5)], 1u << (t & 31));  // native 32-bit
        }
    }
    __syncwarp();
    cx.mask = ((unsigned long long)sc.hit[2 * threadIdx.x + 1] << 32) | sc.hit[2 * threadIdx.x];
    if (valid && masks_out) masks_out[e] = cx.mask;
}

// 32 x 32 bit-matrix transpose across a warp: lane i holds row i (bit j =
// M[i][j]); on return lane j holds column j (bit i = M[i][j]) -- for every
// slot j at once what __ballot_sync of bit j would give. Swaps the
// off-diagonal blocks of 16, 8, 4, 2 and 1 bits.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x, int lane) {
    const uint32_t m16 = 0x0000FFFFu, m8 = 0x00FF00FFu, m4 = 0x0F0F0F0Fu, m2 = 0x33333333u, m1 = 0x55555555u;
#define GS_TSTEP(S, M)                                                                  \
    {                                                                                   \
        const uint32_t p = __shfl_xor_sync(kFull, x, S);                                \
        x = (lane & S) ? ((x & ~(M)) | ((p >> S) & (M))) : ((x & (M)) | ((p & (M)) << S)); \
    }
    GS_TSTEP(16, m16)
    GS_TSTEP(8, m8)
    GS_TSTEP(4, m4)
    GS_TSTEP(2, m2)
    GS_TSTEP(1, m1)
#undef GS_TSTEP
    return x;
}

// Global tile id of slot t of super-tile (sx, sy).
__device__ __forceinline__ int slot_tile(int t, int sx, int sy, int tiles_x) {
    return (sy * kSuper + (t >> 3)) * tiles_x + sx * kSuper + (t & 7);
}

__global__ void __launch_bounds__(kChunk) k_chunk_counts(const float *__restrict__ splats,
                                                        const float4 *__restrict__ cull,
                                                        const uint32_t *__restrict__ svals,
                                                        const uint32_t *__restrict__ chunk_base,
                                                        const uint4 *__restrict__ chunk_rec, int ns,
                                                        int supers_x, DevCam cam, uint32_t *__restrict__ counts,
                                                        uint32_t *__restrict__ tile_count,
                                                        unsigned long long *__restrict__ masks) {
    wait_prior_grid();
    __shared__ uint32_t hit_mask[2 * kChunk];  // per entry, low and high halves
    __shared__ float4 shape[2 * kChunk];
    __shared__ uint32_t rect[kChunk];
    __shared__ uint32_t cnt[kChunk / 32][64];  // per warp and slot: the warp's entries that the slot's tile lists
    const TestScratch sc{hit_mask, shape, rect};
    const uint32_t nc = chunk_base[ns];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (uint32_t c = blockIdx.x; c < nc; c += gridDim.x) {
        ChunkCtx cx;
        chunk_load(cx, c, splats, cull, svals, chunk_rec, supers_x, cam, sc, nullptr, masks);
        cnt[warp][lane] = (uint32_t)__popc(warp_transpose32((uint32_t)cx.mask, lane));
        cnt[warp][lane + 32] = (uint32_t)__popc(warp_transpose32((uint32_t)(cx.mask >> 32), lane));
        __syncthreads();
        if (threadIdx.x < 64) {
            const int t = threadIdx.x;
            uint32_t n = 0u;
#pragma unroll
            for (int w = 0; w < kChunk / 32; ++w) n += cnt[w][t];
            counts[(int64_t)c * 64 + t] = n;
            if (n) atomicAdd(tile_count + slot_tile(t, cx.sx, cx.sy, cam.tiles_x), n);
        }
    }
}

// Tile starts (exclusive scan of the tile counts over tile ids) and the
// ranges, clipped to the capacity: per-block sums, a scan of those, then each
// block scans its own tiles from its offset; block 0 of the last step also
// sets count_dev = P, the sum of the tile counts, or the exact count when the
// super-tile entries overflowed (and the capacity flag if P exceeds it).
__global__ void __launch_bounds__(kScanBlock) k_tile_sums(const uint32_t *__restrict__ tile_count, int64_t tiles,
                                                         unsigned long long *__restrict__ part) {
    wait_prior_grid();
    __shared__ unsigned long long ws[32];
    const int64_t j = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
    unsigned long long tot;
    block_scan_excl<unsigned long long>(j < tiles ? tile_count[j] : 0ull, ws, &tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanBlock) k_tile_starts(const uint32_t *__restrict__ tile_count, int64_t tiles,
                                                           const unsigned long long *__restrict__ part,
                                                           int64_t capacity,
                                                           const unsigned long long *__restrict__ total_t,
                                                           const unsigned long long *__restrict__ total_s,
                                                           const unsigned long long *__restrict__ total_exact,
                                                           unsigned long long *__restrict__ tile_start,
                                                           uint32_t *__restrict__ ranges,
                                                           int64_t *__restrict__ count_dev) {
    wait_prior_grid();
    __shared__ unsigned long long ws[32];
    const int64_t j = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
    const unsigned long long n = j < tiles ? tile_count[j] : 0ull;
    unsigned long long tot;
    const unsigned long long st = part[blockIdx.x] + block_scan_excl<unsigned long long>(n, ws, &tot);
    const unsigned long long cap = (unsigned long long)capacity;
    if (j < tiles) {
        const unsigned long long en = st + n;
        tile_start[j] = st;
        // an empty tile has the range (0, 0)
        ranges[2 * j] = n ? (uint32_t)(st < cap ? st : cap) : 0u;
        ranges[2 * j + 1] = n ? (uint32_t)(en < cap ? en : cap) : 0u;
    }
    if (j == 0) {
        const unsigned long long P = *total_s > cap ? *total_exact : *total_t;
        *count_dev = (int64_t)P;
        if (P > cap) atomicOr(&g_sort_flags, GS_FLAG_CAPACITY);
    }
}

__global__ void __launch_bounds__(kChunk) k_expand(const float *__restrict__ splats, const uint32_t *__restrict__ svals,
                                                  const uint32_t *__restrict__ chunk_base,
                                                  const uint4 *__restrict__ chunk_rec, int ns, int supers_x,
                                                  DevCam cam, const uint32_t *__restrict__ counts,
                                                  const unsigned long long *__restrict__ tile_start, int64_t capacity,
                                                  const unsigned long long *__restrict__ masks,
                                                  uint32_t *__restrict__ vals) {
    wait_prior_grid();
    constexpr int kW = kChunk / 32;
    __shared__ uint32_t ballots[kW][64];                 // per (warp, slot): lanes whose entry the tile lists
    __shared__ uint32_t before[kChunk / 64][64];         // partial sums of earlier chunks' counts
    __shared__ unsigned long long base[kW][64];         // start of (warp, slot) in the final list
    const uint32_t nc = chunk_base[ns];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    for (uint32_t c = blockIdx.x; c < nc; c += gridDim.x) {
        ChunkCtx cx;
        chunk_load(cx, c, splats, nullptr, svals, chunk_rec, supers_x, cam, TestScratch{}, masks, nullptr);
        const uint32_t lo = (uint32_t)cx.mask, hi = (uint32_t)(cx.mask >> 32);
        ballots[warp][lane] = warp_transpose32(lo, lane);
        ballots[warp][lane + 32] = warp_transpose32(hi, lane);
        {   // entries of each slot in the super-tile's earlier chunks: 4 threads per slot,
            // four independent sums so that the loads overlap
            constexpr int kQ = kChunk / 64;
            const int t = threadIdx.x & 63, q = threadIdx.x >> 6;
            uint32_t n0 = 0u, n1 = 0u, n2 = 0u, n3 = 0u;
            uint32_t c2 = cx.first + q;
            for (; c2 + 3 * kQ < c; c2 += 4 * kQ) {
                n0 += counts[(int64_t)c2 * 64 + t];
                n1 += counts[(int64_t)(c2 + kQ) * 64 + t];
                n2 += counts[(int64_t)(c2 + 2 * kQ) * 64 + t];
                n3 += counts[(int64_t)(c2 + 3 * kQ) * 64 + t];
            }
            for (; c2 < c; c2 += kQ) n0 += counts[(int64_t)c2 * 64 + t];
            before[q][t] = (n0 + n1) + (n2 + n3);
        }
        __syncthreads();
        if (threadIdx.x < 64) {
            const int t = threadIdx.x;
            const bool inside = cx.sx * kSuper + (t & 7) < cam.tiles_x && cx.sy * kSuper + (t >> 3) < cam.tiles_y;
            unsigned long long run = 0ull;
            if (inside) {
                run = tile_start[slot_tile(t, cx.sx, cx.sy, cam.tiles_x)];
#pragma unroll
                for (int q = 0; q < kChunk / 64; ++q) run += before[q][t];
            }
#pragma unroll
            for (int w = 0; w < kW; ++w) {
                base[w][t] = run;
                run += (unsigned long long)__popc(ballots[w][t]);
            }
        }
        __syncthreads();
        // An entry's position in tile t's list: the warp's start there plus the
        // lanes before it that tile t lists. Written slot by slot over the
        // slots some lane has (a warp's entries of one tile go to consecutive
        // words) or, when that takes more rounds, each lane over its own slots.
        const unsigned long long any = ((unsigned long long)__reduce_or_sync(kFull, hi) << 32) |
                                       __reduce_or_sync(kFull, lo);
        const int by_slot = __popcll(any), by_lane = (int)__reduce_max_sync(kFull, (unsigned)__popcll(cx.mask));
        for (unsigned long long u = by_lane < by_slot ? cx.mask : any; u; u &= u - 1ull) {
            const int t = __ffsll((long long)u) - 1;
            if ((cx.mask >> t) & 1ull) {
                const unsigned long long pos =
                    base[warp][t] + (unsigned long long)__popc(ballots[warp][t] & lt);
                if (pos < (unsigned long long)capacity) vals[pos] = cx.g;
            }
        }
    }
}

// ---- workspace ----
struct SortWs {
    uint32_t *keys[2], *vals[2];  // visible Gaussians: depth keys and indices
    uint32_t *skeys[2], *svals1;  // super-tile entries; the other value buffer is the output
    uint32_t *hist, *digit_total, *part32;
    unsigned long long *part_s, *total_s, *total_t, *total_exact;
    unsigned long long *masks;                 // [capacity] tile mask of each super-tile entry
    unsigned long long *tile_part;             // [tile blocks]
    float4 *cull;                              // [2 n] cull record of each visible Gaussian
    uint32_t *n_vis, *sclip;
    uint32_t *seg_lo, *seg_hi, *chunk_base;    // [ns], [ns], [ns + 1]
    uint32_t *tile_count;                      // [tiles]
    unsigned long long *tile_start;            // [tiles]
    uint32_t *chunk_counts;                    // [max chunks][64]
    uint4 *chunk_rec;                          // [max chunks]
    size_t bytes;
};

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

inline int64_t max_chunks(int64_t cap, int64_t ns) { return (cap + kChunk - 1) / kChunk + ns + 1; }

inline SortWs sort_layout(char *base, int64_t n, int64_t cap, int64_t tiles, int64_t ns) {
    SortWs w;
    int64_t nbN = (n + kSortBlock - 1) / kSortBlock, nbC = (cap + kSortBlock - 1) / kSortBlock;
    int64_t nbMax = nbN > nbC ? nbN : nbC;
    if (nbMax < 1) nbMax = 1;
    int64_t nbS = (n + kScanBlock - 1) / kScanBlock;
    if (nbS < 1) nbS = 1;
    size_t off = 0;
    auto take = [&](size_t bytes) -> char * {
        char *p = base ? base + off : nullptr;
        off += align256(bytes);
        return p;
    };
    for (int k = 0; k < 2; ++k) w.keys[k] = (uint32_t *)take(4 * (size_t)n);
    for (int k = 0; k < 2; ++k) w.vals[k] = (uint32_t *)take(4 * (size_t)n);
    for (int k = 0; k < 2; ++k) w.skeys[k] = (uint32_t *)take(4 * (size_t)cap);
    w.svals1 = (uint32_t *)take(4 * (size_t)cap);
    w.hist = (uint32_t *)take(4 * (size_t)kMaxRadix * (size_t)nbMax);
    w.digit_total = (uint32_t *)take(4 * (size_t)kMaxRadix);
    w.part32 = (uint32_t *)take(4 * (size_t)nbS);
    w.part_s = (unsigned long long *)take(8 * (size_t)nbS);
    w.total_s = (unsigned long long *)take(8);
    w.total_t = (unsigned long long *)take(8);
    w.total_exact = (unsigned long long *)take(8);
    w.masks = (unsigned long long *)take(8 * (size_t)cap);
    w.cull = (float4 *)take(32 * (size_t)n);
    w.n_vis = (uint32_t *)take(4);
    w.sclip = (uint32_t *)take(4);
    // zeroed together before each sort: segment bounds, then tile counts
    w.seg_lo = (uint32_t *)take(4 * (size_t)(2 * ns + tiles));
    w.seg_hi = w.seg_lo ? w.seg_lo + ns : nullptr;
    w.tile_count = w.seg_lo ? w.seg_lo + 2 * ns : nullptr;
    w.chunk_base = (uint32_t *)take(4 * (size_t)(ns + 1));
    w.chunk_rec = (uint4 *)take(16 * (size_t)max_chunks(cap, ns));
    w.tile_part = (unsigned long long *)take(8 * (size_t)((tiles + kScanBlock - 1) / kScanBlock));
    w.tile_start = (unsigned long long *)take(8 * (size_t)tiles);
    w.chunk_counts = (uint32_t *)take(4 * 64 * (size_t)max_chunks(cap, ns));
    w.bytes = off;
    return w;
}

struct SuperGrid {
    int supers_x, supers_y;
    int64_t tiles, ns;
};

inline SuperGrid super_grid(int32_t width, int32_t height, int32_t tile) {
    SuperGrid g;
    const int tx = (width + tile - 1) / tile, ty = (height + tile - 1) / tile;
    g.supers_x = (tx + kSuper - 1) / kSuper;
    g.supers_y = (ty + kSuper - 1) / kSuper;
    g.tiles = (int64_t)tx * ty;
    g.ns = (int64_t)g.supers_x * g.supers_y;
    return g;
}

// One full LSD sort of (keys, vals) over *count (bounded by `bound`) on `bits`
// low bits; buffers ping-pong between index `in` and 1 - in. The last pass
// writes the segment plan sp (if given). Returns the index holding the result.
int radix_sort(uint32_t *const keys[2], uint32_t *const vals[2], int in, const uint32_t *count, int64_t bound,
               int total_bits, const SortWs &w, cudaStream_t s, SegPlan sp = SegPlan{}) {
    if (total_bits <= 0) return in;
    // 8-bit digits, or one pass of up to kMaxRadixBits when that suffices
    int npass = total_bits <= kMaxRadixBits ? 1 : (total_bits + 7) / 8;
    int per = (total_bits + npass - 1) / npass;
    const int64_t nb = (bound + kSortBlock - 1) / kSortBlock, cap = resident_blocks();
    const int grid = (int)(nb < 1 ? 1 : (nb < cap ? nb : cap));
    int shift = 0;
    for (int p = 0; p < npass; ++p) {
        int bits = per < total_bits - shift ? per : total_bits - shift;
        launch_chained(k_radix_hist, grid, kSortThreads, s, keys[in], count, shift, bits, w.hist);
        launch_chained(k_radix_rowscan, 1 << bits, 1024, s, w.hist, count, w.digit_total);
        launch_chained(k_radix_scatter, grid, kSortThreads, s, keys[in], vals[in], keys[1 - in], vals[1 - in], count,
                       shift, bits, w.hist, w.digit_total, p == npass - 1 ? sp : SegPlan{});
        note_launches(3);
        in = 1 - in;
        shift += bits;
    }
    return in;
}

int ceil_log2(int64_t x) {
    int b = 0;
    while ((int64_t(1) << b) < x) ++b;
    return b;
}

}  // namespace

uint32_t take_sort_flags() {
    uint32_t f = 0, z = 0;
    cudaMemcpyFromSymbol(&f, g_sort_flags, sizeof(f));
    cudaMemcpyToSymbol(g_sort_flags, &z, sizeof(z));
    return f;
}

}  // namespace gs

using namespace gs;

extern "C" size_t gs_sort_workspace_bytes(int64_t n, int64_t capacity, int32_t width, int32_t height, int32_t tile) {
    if (n < 0 || capacity < 0 || width <= 0 || height <= 0 || !tile_ok(tile)) return 0;
    const SuperGrid sg = super_grid(width, height, tile);
    return sort_layout(nullptr, n, capacity, sg.tiles, sg.ns).bytes;
}

extern "C" int gs_sort(const float *splats, int64_t n, const gs_camera *cam, void *ws, size_t ws_bytes,
                       int64_t capacity, uint32_t *vals, uint32_t *ranges, int64_t *count_dev, gs_stream_t stream) {
    if (n < 0 || n > INT32_MAX || capacity < 0 || capacity > INT32_MAX || !camera_ok(cam)) return GS_ERR_INVALID_ARG;
    if (!ranges || !count_dev || (n > 0 && !splats) || (capacity > 0 && !vals)) return GS_ERR_INVALID_ARG;
    const SuperGrid sg = super_grid(cam->width, cam->height, cam->tile);
    SortWs w = sort_layout(static_cast<char *>(ws), n, capacity, sg.tiles, sg.ns);
    if (!ws || ws_bytes < w.bytes) return GS_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(ws) & 255) return GS_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    DevCam dc = make_cam(cam);
    const int64_t tiles = sg.tiles;
    const int ns = (int)sg.ns;
    const int nbS = (int)((n + kScanBlock - 1) / kScanBlock);

    if (n == 0 || capacity == 0) {
        k_zero_u32<<<grid_for(2 * tiles, 256), 256, 0, s>>>(ranges, 2 * tiles);
        note_launches(1);
        if (n == 0) {
            cudaMemsetAsync(count_dev, 0, sizeof(int64_t), s);
            return launch_status();
        }
    }
    // stage 1: visible Gaussians by depth (the first kernel also zeroes the
    // segment bounds, tile counts and exact count)
    launch_chained(k_count_visible, nbS, kScanBlock, s, splats, n, w.part32, w.seg_lo, 2 * sg.ns + tiles,
                   w.total_exact);
    launch_chained(k_scan_parts<uint32_t>, 1, 1024, s, w.part32, nbS, w.n_vis, nullptr, 0);
    launch_chained(k_emit_visible, nbS, kScanBlock, s, splats, n, w.part32, dc, w.keys[0], w.vals[0], w.cull);
    note_launches(3);
    int cur = radix_sort(w.keys, w.vals, 0, w.n_vis, n, 32, w, s);
    // stage 2: super-tile entries in depth order, stable-sorted by super-tile
    launch_chained(k_count_entries, nbS, kScanBlock, s, w.cull, w.vals[cur], w.n_vis, w.part_s);
    launch_chained(k_scan_parts<unsigned long long>, 1, 1024, s, w.part_s, nbS, w.total_s, w.sclip, capacity);
    note_launches(2);
    if (capacity == 0) {
        cudaMemsetAsync(w.total_t, 0, sizeof(unsigned long long), s);
        launch_chained(k_count_exact, (unsigned)resident_blocks(), 256, s, splats, w.vals[cur], w.n_vis, dc, w.total_s,
                       capacity, w.total_exact);
        launch_chained(k_finish_count, 1, 1, s, w.total_t, w.total_s, w.total_exact, capacity, count_dev);
        note_launches(2);
        return launch_status();
    }
    const int sbits = ceil_log2(sg.ns);
    const int npass = sbits <= 0 ? 0 : (sbits <= kMaxRadixBits ? 1 : (sbits + 7) / 8);
    uint32_t *sk[2] = {w.skeys[0], w.skeys[1]};
    uint32_t *sv[2] = {w.svals1, vals};  // the sorted list must end in svals1: vals is written from it
    const int start = npass % 2;
    launch_chained(k_emit_super, nbS, kScanBlock, s, splats, w.cull, w.vals[cur], w.n_vis, dc, sg.supers_x, w.part_s,
                   w.total_s, capacity, sk[start], sv[start], w.total_exact);
    note_launches(1);
    // one pass: its digit ranges are the segments, written by the pass itself
    const SegPlan sp{w.chunk_base, w.chunk_rec, ns, kChunk};
    // ends in skeys[0] / svals1
    radix_sort(sk, sv, start, w.sclip, capacity, sbits, w, s, npass == 1 ? sp : SegPlan{});
    // stage 3: per-tile lists
    const int64_t chunks = max_chunks(capacity, sg.ns), resident = resident_blocks();
    const unsigned cgrid = (unsigned)(chunks < resident ? chunks : resident);
    if (npass != 1) {
        launch_chained(k_seg_mark, (unsigned)resident, 256, s, w.skeys[0], w.sclip, w.seg_lo, w.seg_hi);
        launch_chained(k_super_plan, 1, 1024, s, w.seg_lo, w.seg_hi, ns, w.chunk_base, w.chunk_rec);
        note_launches(2);
    }
    launch_chained(k_chunk_counts, cgrid, kChunk, s, splats, w.cull, w.svals1, w.chunk_base, w.chunk_rec, ns,
                   sg.supers_x, dc, w.chunk_counts, w.tile_count, w.masks);
    const int tb = (int)((tiles + kScanBlock - 1) / kScanBlock);
    launch_chained(k_tile_sums, tb, kScanBlock, s, w.tile_count, tiles, w.tile_part);
    launch_chained(k_scan_parts<unsigned long long>, 1, 1024, s, w.tile_part, tb, w.total_t, nullptr, 0);
    launch_chained(k_tile_starts, tb, kScanBlock, s, w.tile_count, tiles, w.tile_part, capacity, w.total_t, w.total_s,
                   w.total_exact, w.tile_start, ranges, count_dev);
    note_launches(2);
    launch_chained(k_expand, cgrid, kChunk, s, splats, w.svals1, w.chunk_base, w.chunk_rec, ns, sg.supers_x, dc,
                   w.chunk_counts, w.tile_start, capacity, w.masks, vals);
    note_launches(3);
    return launch_status();
}
