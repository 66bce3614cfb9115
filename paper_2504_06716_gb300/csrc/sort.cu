// Per-tile depth order of splats (Sec. 3.1: colours are blended "in a sorted
// order").
//
// The result equals a stable sort of the 64-bit keys (tile << 32 | depth
// bits) generated in Gaussian order, but it is computed in two cheaper
// stages instead of one 45-bit sort over every (Gaussian, tile) entry:
//   1. compact the visible Gaussians (ascending index) and LSD-radix-sort
//      them by the bits of their float32 depth (4 passes of 8 bits over the
//      visible Gaussians only; stable, so equal depths keep index order);
//   2. emit every Gaussian's tile entries in that depth order and
//      LSD-radix-sort the entries by tile id only (ceil(log2 tiles) bits, 1-2
//      passes); stability keeps depth order, then index order, inside a tile.
// All counts live on the device; nothing waits on the host.
#include "common.cuh"

namespace gs {

__device__ uint32_t g_sort_flags;

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 4;
constexpr int kSortBlock = kSortThreads * kSortItems;  // keys per radix block
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
__global__ void __launch_bounds__(kScanBlock) k_count_visible(const float *__restrict__ splats, int64_t n,
                                                             uint32_t *__restrict__ part) {
    int64_t i = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
    int f = (i < n) && splat_visible(splats, i);
    int c = __syncthreads_count(f);
    if (threadIdx.x == 0) part[blockIdx.x] = (uint32_t)c;
}

// Exclusive scan of part[0..nb) in place by one block; total to *total.
template <typename T>
__global__ void __launch_bounds__(1024) k_scan_parts(T *__restrict__ part, int nb, T *__restrict__ total) {
    __shared__ T ws[32];
    T carry = 0;
    for (int base = 0; base < nb; base += 1024) {
        int j = base + threadIdx.x;
        T v = j < nb ? part[j] : T(0), tot;
        T ex = block_scan_excl<T>(v, ws, &tot);
        if (j < nb) part[j] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void __launch_bounds__(kScanBlock) k_emit_visible(const float *__restrict__ splats, int64_t n,
                                                            const uint32_t *__restrict__ part,
                                                            uint32_t *__restrict__ keys, uint32_t *__restrict__ vals) {
    __shared__ int ws[32];
    int64_t i = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
    int f = (i < n) && splat_visible(splats, i);
    int tot;
    int r = block_scan_excl<int>(f, ws, &tot);
    if (f) {
        uint32_t pos = part[blockIdx.x] + (uint32_t)r;
        keys[pos] = __float_as_uint(__ldg(splats + i * kSplat + 9));
        vals[pos] = (uint32_t)i;
    }
}

// ---- LSD radix pass: histogram, per-digit row scan, stable scatter ----
__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const uint32_t *__restrict__ keys,
                                                            const uint32_t *__restrict__ count, int shift, int bits,
                                                            uint32_t *__restrict__ hist, int nb) {
    __shared__ uint32_t h[256];
    const int radix = 1 << bits;
    const uint32_t mask = (uint32_t)radix - 1u;
    h[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t n = *count;
    const int64_t base = (int64_t)blockIdx.x * kSortBlock;
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        int64_t i = base + r * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & mask], 1u);
    }
    __syncthreads();
    if ((int)threadIdx.x < radix) hist[(int64_t)threadIdx.x * nb + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(1024) k_radix_rowscan(uint32_t *__restrict__ hist, int nb,
                                                        uint32_t *__restrict__ digit_total) {
    __shared__ uint32_t ws[32];
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

__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(const uint32_t *__restrict__ kin,
                                                               const uint32_t *__restrict__ vin,
                                                               uint32_t *__restrict__ kout, uint32_t *__restrict__ vout,
                                                               const uint32_t *__restrict__ count, int shift, int bits,
                                                               const uint32_t *__restrict__ hist,
                                                               const uint32_t *__restrict__ digit_total, int nb) {
    constexpr int kWarps = kSortThreads / 32;
    __shared__ uint32_t run[256];
    __shared__ uint32_t wc[kWarps][256];
    __shared__ uint32_t ws[32];
    const uint32_t n = *count;
    const int64_t base = (int64_t)blockIdx.x * kSortBlock;
    if (base >= n) return;
    const int radix = 1 << bits;
    const uint32_t mask = (uint32_t)radix - 1u;
    const int t = threadIdx.x, warp = t >> 5;
    uint32_t tot;
    uint32_t dt = t < radix ? digit_total[t] : 0u;
    uint32_t dbase = block_scan_excl<uint32_t>(dt, ws, &tot);
    if (t < radix) run[t] = dbase + hist[(int64_t)t * nb + blockIdx.x];
#pragma unroll 1
    for (int r = 0; r < kSortItems; ++r) {
        int64_t i = base + r * kSortThreads + t;
        bool valid = i < n;
        uint32_t key = valid ? kin[i] : 0u;
        uint32_t d = valid ? ((key >> shift) & mask) : 0xffffu;
        unsigned peers = __match_any_sync(kFull, d);
        unsigned lrank = __popc(peers & lanemask_lt());
        if (t < radix) {
#pragma unroll
            for (int w = 0; w < kWarps; ++w) wc[w][t] = 0u;
        }
        __syncthreads();
        if (valid && lrank == 0) wc[warp][d] = (uint32_t)__popc(peers);
        __syncthreads();
        if (t < radix) {
            uint32_t c = run[t];
#pragma unroll
            for (int w = 0; w < kWarps; ++w) {
                uint32_t x = wc[w][t];
                wc[w][t] = c;
                c += x;
            }
            run[t] = c;
        }
        __syncthreads();
        if (valid) {
            uint32_t pos = wc[warp][d] + lrank;
            kout[pos] = key;
            vout[pos] = vin[i];
        }
        __syncthreads();
    }
}

// ---- stage 2: tile entries in depth order ----
__device__ __forceinline__ int splat_rect(const float *splats, uint32_t g, const DevCam &cam, int &x0, int &y0,
                                          int &x1, int &y1) {
    const float *r = splats + (int64_t)g * kSplat;
    int rad = __float_as_int(__ldg(r + 10));
    if (rad <= 0) { x0 = y0 = x1 = y1 = 0; return 0; }
    return tile_rect(__ldg(r), __ldg(r + 1), rad, cam.tile, cam.tiles_x, cam.tiles_y, x0, y0, x1, y1);
}

__global__ void __launch_bounds__(kScanBlock) k_count_entries(const float *__restrict__ splats,
                                                             const uint32_t *__restrict__ order,
                                                             const uint32_t *__restrict__ n_vis, DevCam cam,
                                                             unsigned long long *__restrict__ part) {
    __shared__ unsigned long long ws[32];
    int64_t k = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
    int x0, y0, x1, y1;
    unsigned long long c = k < *n_vis ? (unsigned long long)splat_rect(splats, order[k], cam, x0, y0, x1, y1) : 0ull;
    unsigned long long tot;
    block_scan_excl<unsigned long long>(c, ws, &tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void k_finish_count(const unsigned long long *__restrict__ total, int64_t capacity,
                               int64_t *__restrict__ count_dev, uint32_t *__restrict__ pclip) {
    unsigned long long P = *total;
    *count_dev = (int64_t)P;
    if (P > (unsigned long long)capacity) {
        *pclip = (uint32_t)capacity;
        atomicOr(&g_sort_flags, GS_FLAG_CAPACITY);
    } else {
        *pclip = (uint32_t)P;
    }
}

__global__ void __launch_bounds__(kScanBlock) k_emit_entries(const float *__restrict__ splats,
                                                            const uint32_t *__restrict__ order,
                                                            const uint32_t *__restrict__ n_vis, DevCam cam,
                                                            const unsigned long long *__restrict__ part,
                                                            int64_t capacity, uint32_t *__restrict__ tkeys,
                                                            uint32_t *__restrict__ tvals) {
    __shared__ unsigned long long ws[32];
    int64_t k = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
    int x0 = 0, y0 = 0, x1 = 0, y1 = 0;
    uint32_t g = 0;
    unsigned long long c = 0;
    if (k < *n_vis) {
        g = order[k];
        c = (unsigned long long)splat_rect(splats, g, cam, x0, y0, x1, y1);
    }
    unsigned long long tot;
    unsigned long long off = part[blockIdx.x] + block_scan_excl<unsigned long long>(c, ws, &tot);
    if (c == 0 || off >= (unsigned long long)capacity) return;
    for (int y = y0; y < y1; ++y)
        for (int x = x0; x < x1; ++x) {
            if (off >= (unsigned long long)capacity) return;
            tkeys[off] = (uint32_t)(y * cam.tiles_x + x);
            tvals[off] = g;
            ++off;
        }
}

__global__ void k_zero_u32(uint32_t *__restrict__ p, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = 0u;
}

__global__ void __launch_bounds__(256) k_ranges_mark(const uint32_t *__restrict__ tkeys,
                                                    const uint32_t *__restrict__ pclip,
                                                    uint32_t *__restrict__ ranges) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t P = *pclip;
    if (k >= P) return;
    uint32_t t = tkeys[k];
    if (k == 0 || tkeys[k - 1] != t) ranges[2 * (int64_t)t] = (uint32_t)k;
    if (k == (int64_t)P - 1 || tkeys[k + 1] != t) ranges[2 * (int64_t)t + 1] = (uint32_t)(k + 1);
}

// ---- workspace ----
struct SortWs {
    uint32_t *keys[2], *vals[2];  // visible Gaussians: depth keys and indices
    uint32_t *tkeys[2], *tvals1;  // tile entries; the other value buffer is the output
    uint32_t *hist, *digit_total, *part32;
    unsigned long long *part64, *total64;
    uint32_t *n_vis, *pclip;
    size_t bytes;
};

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

inline SortWs sort_layout(char *base, int64_t n, int64_t cap) {
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
    for (int k = 0; k < 2; ++k) w.tkeys[k] = (uint32_t *)take(4 * (size_t)cap);
    w.tvals1 = (uint32_t *)take(4 * (size_t)cap);
    w.hist = (uint32_t *)take(4 * 256 * (size_t)nbMax);
    w.digit_total = (uint32_t *)take(4 * 256);
    w.part32 = (uint32_t *)take(4 * (size_t)nbS);
    w.part64 = (unsigned long long *)take(8 * (size_t)nbS);
    w.total64 = (unsigned long long *)take(8);
    w.n_vis = (uint32_t *)take(4);
    w.pclip = (uint32_t *)take(4);
    w.bytes = off;
    return w;
}

// One full LSD sort of (keys, vals) over *count (bounded by `bound`) on `bits`
// low bits; buffers ping-pong between index `in` and 1 - in. Returns the
// index holding the result.
int radix_sort(uint32_t *const keys[2], uint32_t *const vals[2], int in, const uint32_t *count, int64_t bound,
               int total_bits, const SortWs &w, cudaStream_t s) {
    if (total_bits <= 0) return in;
    int npass = (total_bits + 7) / 8;
    int per = (total_bits + npass - 1) / npass;
    int nb = (int)((bound + kSortBlock - 1) / kSortBlock);
    if (nb < 1) nb = 1;
    int shift = 0;
    for (int p = 0; p < npass; ++p) {
        int bits = per < total_bits - shift ? per : total_bits - shift;
        k_radix_hist<<<nb, kSortThreads, 0, s>>>(keys[in], count, shift, bits, w.hist, nb);
        k_radix_rowscan<<<1 << bits, 1024, 0, s>>>(w.hist, nb, w.digit_total);
        k_radix_scatter<<<nb, kSortThreads, 0, s>>>(keys[in], vals[in], keys[1 - in], vals[1 - in], count, shift,
                                                    bits, w.hist, w.digit_total, nb);
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
    (void)width; (void)height; (void)tile;
    if (n < 0 || capacity < 0) return 0;
    return sort_layout(nullptr, n, capacity).bytes;
}

extern "C" int gs_sort(const float *splats, int64_t n, const gs_camera *cam, void *ws, size_t ws_bytes,
                       int64_t capacity, uint32_t *vals, uint32_t *ranges, int64_t *count_dev, gs_stream_t stream) {
    if (n < 0 || n > INT32_MAX || capacity < 0 || capacity > INT32_MAX || !camera_ok(cam)) return GS_ERR_INVALID_ARG;
    if (!ranges || !count_dev || (n > 0 && !splats) || (capacity > 0 && !vals)) return GS_ERR_INVALID_ARG;
    SortWs w = sort_layout(static_cast<char *>(ws), n, capacity);
    if (!ws || ws_bytes < w.bytes) return GS_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(ws) & 255) return GS_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    DevCam dc = make_cam(cam);
    const int64_t tiles = (int64_t)dc.tiles_x * dc.tiles_y;
    const int nbS = (int)((n + kScanBlock - 1) / kScanBlock);

    k_zero_u32<<<grid_for(2 * tiles, 256), 256, 0, s>>>(ranges, 2 * tiles);
    note_launches(1);
    if (n == 0) {
        cudaMemsetAsync(count_dev, 0, sizeof(int64_t), s);
        return launch_status();
    }
    // stage 1: visible Gaussians by depth
    k_count_visible<<<nbS, kScanBlock, 0, s>>>(splats, n, w.part32);
    k_scan_parts<uint32_t><<<1, 1024, 0, s>>>(w.part32, nbS, w.n_vis);
    k_emit_visible<<<nbS, kScanBlock, 0, s>>>(splats, n, w.part32, w.keys[0], w.vals[0]);
    note_launches(3);
    int cur = radix_sort(w.keys, w.vals, 0, w.n_vis, n, 32, w, s);
    // stage 2: tile entries in depth order, then by tile id
    k_count_entries<<<nbS, kScanBlock, 0, s>>>(splats, w.vals[cur], w.n_vis, dc, w.part64);
    k_scan_parts<unsigned long long><<<1, 1024, 0, s>>>(w.part64, nbS, w.total64);
    k_finish_count<<<1, 1, 0, s>>>(w.total64, capacity, count_dev, w.pclip);
    note_launches(3);
    const int tbits = ceil_log2(tiles);
    const int npass = (tbits + 7) / 8;
    uint32_t *tk[2] = {w.tkeys[0], w.tkeys[1]};
    uint32_t *tv[2] = {vals, w.tvals1};
    const int start = (npass % 2 == 0) ? 0 : 1;  // so that the last pass lands in `vals`
    if (capacity > 0) {
        k_emit_entries<<<nbS, kScanBlock, 0, s>>>(splats, w.vals[cur], w.n_vis, dc, w.part64, capacity, tk[start],
                                                  tv[start]);
        int fin = radix_sort(tk, tv, start, w.pclip, capacity, tbits, w, s);
        k_ranges_mark<<<grid_for(capacity, 256), 256, 0, s>>>(tk[fin], w.pclip, ranges);
        note_launches(2);
    }
    return launch_status();
}
