// Tile binning and per-tile depth sorting (App. C.2).
//
// The canonical result is the list of (tile, Gaussian) pairs ordered by the 64-bit key
// (global_tile << 32) | float_bits(depth), ties by flat index c*N + n.  Instead of one
// radix sort over K 64-bit keys, the same order is reached in two stable stages:
//   1. a 32-bit LSD radix sort of the C*N (camera, Gaussian) pairs by depth bits
//      (invisible pairs get key 0xFFFFFFFF and emit nothing);
//   2. emission of every pair's tiles in that depth order, followed by a stable LSD
//      radix sort of the K intersections by tile id alone (ceil(log2 T) bits).
// Stability carries the depth order (and the index tie-break) into each tile's list.
// Stage 2 moves 8 bytes per intersection per pass over ~2 passes instead of 12 bytes
// over 6 passes.  Every kernel reads the data-dependent counts from device memory, so
// the host never synchronises and the whole call can be captured in a CUDA graph.
#include "gs_internal.cuh"

namespace gs {

constexpr int kSortThreads = 256;  // 8 warps
constexpr int kSortIPT = 8;        // items per thread per sub-tile
constexpr int kSubTile = kSortThreads * kSortIPT;
constexpr int kRadix = 256;

__device__ __forceinline__ void block_range(int n, int G, int b, int &beg, int &end) {
    int tiles = (n + kSubTile - 1) / kSubTile;
    int per = tiles / G, rem = tiles % G;
    int t0 = b * per + min(b, rem);
    int t1 = t0 + per + (b < rem ? 1 : 0);
    beg = min(n, t0 * kSubTile);
    end = min(n, t1 * kSubTile);
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Per-block digit histogram: hist[d * G + b].
__global__ void __launch_bounds__(kSortThreads) radix_upsweep(const uint32_t *__restrict__ keys,
                                                              const int *__restrict__ n_dev, int n_host, int shift,
                                                              unsigned mask, int *__restrict__ hist) {
    __shared__ int s_h[kSortThreads / 32][kRadix];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < (kSortThreads / 32) * kRadix; i += kSortThreads) (&s_h[0][0])[i] = 0;
    __syncthreads();
    const int n = n_dev ? *n_dev : n_host;
    int beg, end;
    block_range(n, gridDim.x, blockIdx.x, beg, end);
    for (int base = beg; base < end; base += kSortThreads * 4) {
        uint32_t k[4];
        bool ok[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            int i = base + u * kSortThreads + threadIdx.x;
            ok[u] = i < end;
            k[u] = ok[u] ? keys[i] : 0u;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            unsigned valid = __ballot_sync(0xffffffffu, ok[u]);
            if (ok[u]) {
                unsigned d = (k[u] >> shift) & mask;
                unsigned peers = __match_any_sync(valid, d);
                if ((__ffs(peers) - 1) == lane) atomicAdd(&s_h[warp][d], __popc(peers));
            }
        }
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += kSortThreads) {
        int s = 0;
#pragma unroll
        for (int w = 0; w < kSortThreads / 32; ++w) s += s_h[w][d];
        hist[d * gridDim.x + blockIdx.x] = s;
    }
}

// Exclusive scan of hist[0 .. total) in place (digit-major order), one CTA of 1024 threads.
__global__ void __launch_bounds__(1024) scan_hist(int *__restrict__ hist, int total) {
    __shared__ int s_w[32];
    const int per = (total + 1023) / 1024;
    const int b = threadIdx.x * per, e = min(total, b + per);
    int sum = 0;
    for (int i = b; i < e; ++i) sum += hist[i];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int v = s_w[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        s_w[lane] = v;
    }
    __syncthreads();
    int run = x - sum + (warp > 0 ? s_w[warp - 1] : 0);
    for (int i = b; i < e; ++i) {
        int v = hist[i];
        hist[i] = run;
        run += v;
    }
}

// Stable scatter of one LSD pass.  Items of a sub-tile are owned warp-striped (warp w
// takes a contiguous run, lane order inside), ranks inside a warp come from
// __match_any_sync, and per-digit warp prefixes make the scatter stable.
__global__ void __launch_bounds__(kSortThreads) radix_downsweep(
    const uint32_t *__restrict__ keys_in, const int *__restrict__ vals_in, uint32_t *__restrict__ keys_out,
    int *__restrict__ vals_out, const int *__restrict__ n_dev, int n_host, int shift, unsigned mask,
    const int *__restrict__ hist) {
    constexpr int W = kSortThreads / 32;
    __shared__ int s_warp[W][kRadix];
    __shared__ int s_base[kRadix];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n = n_dev ? *n_dev : n_host;
    int beg, end;
    block_range(n, gridDim.x, blockIdx.x, beg, end);
    for (int d = threadIdx.x; d < kRadix; d += kSortThreads) s_base[d] = hist[d * gridDim.x + blockIdx.x];
    const unsigned lt = lanemask_lt();
    for (int t0 = beg; t0 < end; t0 += kSubTile) {
        for (int i = threadIdx.x; i < W * kRadix; i += kSortThreads) (&s_warp[0][0])[i] = 0;
        __syncthreads();
        const int wbase = t0 + warp * 32 * kSortIPT;
        uint32_t k[kSortIPT];
        int v[kSortIPT], rank[kSortIPT];
        unsigned dg[kSortIPT];
#pragma unroll
        for (int j = 0; j < kSortIPT; ++j) {
            int i = wbase + j * 32 + lane;
            bool ok = i < end;
            k[j] = ok ? keys_in[i] : 0u;
            v[j] = ok ? vals_in[i] : 0;
            dg[j] = ok ? ((k[j] >> shift) & mask) : 0xffffffffu;
        }
#pragma unroll
        for (int j = 0; j < kSortIPT; ++j) {
            bool ok = dg[j] != 0xffffffffu;
            unsigned valid = __ballot_sync(0xffffffffu, ok);
            rank[j] = 0;
            if (ok) {
                unsigned d = dg[j];
                unsigned peers = __match_any_sync(valid, d);
                int before = s_warp[warp][d];
                __syncwarp(valid);
                if ((__ffs(peers) - 1) == lane) s_warp[warp][d] = before + __popc(peers);
                rank[j] = before + __popc(peers & lt);
            }
            __syncwarp();
        }
        __syncthreads();
        for (int d = threadIdx.x; d < kRadix; d += kSortThreads) {
            int run = s_base[d];
#pragma unroll
            for (int w = 0; w < W; ++w) {
                int c = s_warp[w][d];
                s_warp[w][d] = run;
                run += c;
            }
            s_base[d] = run;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kSortIPT; ++j) {
            if (dg[j] != 0xffffffffu) {
                int pos = s_warp[warp][dg[j]] + rank[j];
                if ((unsigned)pos < (unsigned)n) {  // holds by construction; guards the scatter
                    keys_out[pos] = k[j];
                    vals_out[pos] = v[j];
                }
            }
        }
        __syncthreads();
    }
}

// Stage 1 keys: depth bits of visible (camera, Gaussian) pairs, 0xFFFFFFFF otherwise.
__global__ void depth_keys_kernel(int CN, const float *__restrict__ depths, const int *__restrict__ radii,
                                  uint32_t *__restrict__ keys, int *__restrict__ vals) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= CN) return;
    keys[i] = radii[i] > 0 ? __float_as_uint(depths[i]) : 0xffffffffu;
    vals[i] = i;
}

__device__ __forceinline__ bool tile_rect(const CamSet &cs, int N, int i, const float2 *__restrict__ means2d,
                                          const int *__restrict__ radii, int &c, int &tx0, int &tx1, int &ty0,
                                          int &ty1) {
    if ((unsigned)i >= (unsigned)(cs.C * N)) return false;
    int r = radii[i];
    if (r <= 0) return false;
    c = i / N;
    const CamDev &cam = cs.cam[c];
    float2 m = means2d[i];
    int x0, x1, y0, y1;
    if (!pixel_box(m.x, m.y, r, cam.W, cam.H, x0, x1, y0, y1)) return false;
    const int t = cs.tile;
    tx0 = x0 / t;
    tx1 = x1 / t;
    ty0 = y0 / t;
    ty1 = y1 / t;
    return true;
}

// Tiles touched by each pair, in depth order.
__global__ void count_tiles_kernel(int CN, int N, const __grid_constant__ CamSet cs, const int *__restrict__ order,
                                   const float2 *__restrict__ means2d, const int *__restrict__ radii,
                                   int *__restrict__ counts) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= CN) return;
    int i = order[j], c, tx0, tx1, ty0, ty1;  // tile_rect range-checks i
    counts[j] = tile_rect(cs, N, i, means2d, radii, c, tx0, tx1, ty0, ty1) ? (tx1 - tx0 + 1) * (ty1 - ty0 + 1) : 0;
}

// Block sums of counts (same partition as the sort kernels).
__global__ void __launch_bounds__(kSortThreads) count_reduce_kernel(int CN, const int *__restrict__ counts,
                                                                   long long *__restrict__ partials) {
    int beg, end;
    block_range(CN, gridDim.x, blockIdx.x, beg, end);
    long long s = 0;
    for (int i = beg + threadIdx.x; i < end; i += kSortThreads) s += counts[i];
    __shared__ long long s_w[kSortThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        for (int w = 0; w < kSortThreads / 32; ++w) t += s_w[w];
        partials[blockIdx.x] = t;
    }
}

// Exclusive scan of the G partials; K = total; n_eff = min(K, capacity).
__global__ void partial_scan_kernel(int G, long long *__restrict__ partials, long long capacity,
                                    long long *__restrict__ K_out, int *__restrict__ n_eff) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    long long run = 0;
    for (int b = 0; b < G; ++b) {
        long long v = partials[b];
        partials[b] = run;
        run += v;
    }
    *K_out = run;
    *n_eff = (int)(run < capacity ? run : capacity);
}

// Exclusive offsets of counts inside each block, then emission of (tile, index) pairs.
__global__ void __launch_bounds__(kSortThreads) emit_kernel(int CN, int N, const __grid_constant__ CamSet cs,
                                                           const int *__restrict__ order,
                                                           const int *__restrict__ counts,
                                                           const long long *__restrict__ partials,
                                                           const float2 *__restrict__ means2d,
                                                           const int *__restrict__ radii, long long capacity,
                                                           uint32_t *__restrict__ tkeys, int *__restrict__ tvals) {
    int beg, end;
    block_range(CN, gridDim.x, blockIdx.x, beg, end);
    __shared__ long long s_w[kSortThreads / 32];
    __shared__ long long s_carry;
    if (threadIdx.x == 0) s_carry = partials[blockIdx.x];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int base = beg; base < end; base += kSortThreads) {
        int j = base + threadIdx.x;
        int cnt = j < end ? counts[j] : 0;
        long long x = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            long long y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_w[warp] = x;
        __syncthreads();
        long long wpre = 0, tot = 0;
        for (int w = 0; w < kSortThreads / 32; ++w) {
            if (w < warp) wpre += s_w[w];
            tot += s_w[w];
        }
        long long off = s_carry + wpre + x - cnt;
        if (cnt > 0) {
            int i = order[j], c, tx0, tx1, ty0, ty1;
            tile_rect(cs, N, i, means2d, radii, c, tx0, tx1, ty0, ty1);
            const CamDev &cam = cs.cam[c];
            long long p = off;
            for (int ty = ty0; ty <= ty1; ++ty) {
                uint32_t rowbase = (uint32_t)(cam.tile_offset + ty * cam.tiles_x);
                for (int tx = tx0; tx <= tx1; ++tx, ++p) {
                    if (p < capacity) {
                        tkeys[p] = rowbase + (uint32_t)tx;
                        tvals[p] = i;
                    }
                }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) s_carry += tot;
        __syncthreads();
    }
}

__global__ void empty_result_kernel(long long *__restrict__ K_out, int *__restrict__ n_eff) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        *K_out = 0;
        *n_eff = 0;
    }
}

__global__ void zero_ranges_kernel(int T, int2 *__restrict__ ranges) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < T) ranges[t] = make_int2(0, 0);
}

__global__ void ranges_kernel(const int *__restrict__ n_dev, int T, int CN, const uint32_t *__restrict__ tkeys,
                              const int *__restrict__ vals, const float *__restrict__ depths,
                              int2 *__restrict__ ranges, unsigned long long *__restrict__ keys64) {
    const int n = *n_dev;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        uint32_t t = tkeys[p];
        if (t >= (uint32_t)T) continue;  // holds by construction
        if (p == 0 || tkeys[p - 1] != t) ranges[t].x = p;
        if (p == n - 1 || tkeys[p + 1] != t) ranges[t].y = p + 1;
        if (keys64) {
            int v = vals[p];
            keys64[p] = ((unsigned long long)t << 32) | ((unsigned)v < (unsigned)CN ? __float_as_uint(depths[v]) : 0u);
        }
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

static inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int sort_grid_blocks();  // defined in gs_abi.cu (4 CTAs per SM of the current device)

static int tile_bits(long long T) {
    int b = 1;
    while ((1ll << b) < T) ++b;
    return b;
}

BinSortLayout binsort_layout(long long CN, long long Kcap, int G) {
    BinSortLayout L;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o += align256(bytes);
        return at;
    };
    L.dk0 = take(CN * 4);
    L.dk1 = take(CN * 4);
    L.dv0 = take(CN * 4);
    L.dv1 = take(CN * 4);
    L.counts = take(CN * 4);
    L.partials = take((size_t)(G + 1) * 8);
    L.misc = take(64);
    L.hist = take((size_t)kRadix * G * 4);
    L.tk0 = take(Kcap * 4);
    L.tk1 = take(Kcap * 4);
    L.tvB = take(Kcap * 4);
    L.total = o;
    return L;
}

static cudaError_t radix_pass(const uint32_t *kin, const int *vin, uint32_t *kout, int *vout, const int *n_dev,
                              int n_host, int shift, int bits, int *hist, int G, cudaStream_t st) {
    unsigned mask = (bits >= 32) ? 0xffffffffu : ((1u << bits) - 1u);
    radix_upsweep<<<G, kSortThreads, 0, st>>>(kin, n_dev, n_host, shift, mask, hist);
    note_launch();
    scan_hist<<<1, 1024, 0, st>>>(hist, kRadix * G);
    note_launch();
    radix_downsweep<<<G, kSortThreads, 0, st>>>(kin, vin, kout, vout, n_dev, n_host, shift, mask, hist);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_binsort(const CamSet &cs, int N, const float *means2d, const float *depths, const int *radii,
                           long long Kcap, unsigned long long *keys64, int *values, int *tile_ranges,
                           long long *K_out, void *ws, cudaStream_t st) {
    const int C = cs.C;
    const long long CN = (long long)C * N;
    const int G = sort_grid_blocks();
    BinSortLayout L = binsort_layout(CN, Kcap, G);
    char *w = (char *)ws;
    uint32_t *dk0 = (uint32_t *)(w + L.dk0), *dk1 = (uint32_t *)(w + L.dk1);
    int *dv0 = (int *)(w + L.dv0), *dv1 = (int *)(w + L.dv1);
    int *counts = (int *)(w + L.counts);
    long long *partials = (long long *)(w + L.partials);
    int *n_eff = (int *)(w + L.misc);
    int *hist = (int *)(w + L.hist);
    uint32_t *tk0 = (uint32_t *)(w + L.tk0), *tk1 = (uint32_t *)(w + L.tk1);
    int *tvB = (int *)(w + L.tvB);

    const int cn = (int)CN;
    const int eb = (cn + 255) / 256;
    if (cn == 0) {
        empty_result_kernel<<<1, 32, 0, st>>>(K_out, n_eff);
        note_launch();
        zero_ranges_kernel<<<(cs.total_tiles + 255) / 256, 256, 0, st>>>(cs.total_tiles, (int2 *)tile_ranges);
        note_launch();
        return cudaGetLastError();
    }
    // stage 1: depth order of all (camera, Gaussian) pairs
    depth_keys_kernel<<<eb, 256, 0, st>>>(cn, depths, radii, dk0, dv0);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    for (int pass = 0; pass < 4; ++pass) {
        bool even = (pass % 2) == 0;
        e = radix_pass(even ? dk0 : dk1, even ? dv0 : dv1, even ? dk1 : dk0, even ? dv1 : dv0, nullptr, cn, 8 * pass,
                       8, hist, G, st);
        if (e != cudaSuccess) return e;
    }
    const int *order = dv0;  // after 4 passes the sorted pairs are back in (dk0, dv0)
    // stage 2: emission in depth order, then a stable sort by tile id
    count_tiles_kernel<<<eb, 256, 0, st>>>(cn, N, cs, order, (const float2 *)means2d, radii, counts);
    note_launch();
    count_reduce_kernel<<<G, kSortThreads, 0, st>>>(cn, counts, partials);
    note_launch();
    partial_scan_kernel<<<1, 32, 0, st>>>(G, partials, Kcap, K_out, n_eff);
    note_launch();
    const int bits = tile_bits(cs.total_tiles);
    const int passes = (bits + 7) / 8;
    // choose buffers so that the last pass writes into the caller's `values`
    uint32_t *kA = tk0, *kB = tk1;
    int *vA = (passes % 2 == 0) ? values : tvB;
    int *vB = (passes % 2 == 0) ? tvB : values;
    emit_kernel<<<G, kSortThreads, 0, st>>>(cn, N, cs, order, counts, partials, (const float2 *)means2d, radii, Kcap,
                                            kA, vA);
    note_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    for (int pass = 0; pass < passes; ++pass) {
        int b = min(8, bits - 8 * pass);
        e = radix_pass(kA, vA, kB, vB, n_eff, 0, 8 * pass, b, hist, G, st);
        if (e != cudaSuccess) return e;
        uint32_t *tk = kA;
        kA = kB;
        kB = tk;
        int *tv = vA;
        vA = vB;
        vB = tv;
    }
    // (kA, vA) now hold the sorted list; vA == values
    zero_ranges_kernel<<<(cs.total_tiles + 255) / 256, 256, 0, st>>>(cs.total_tiles, (int2 *)tile_ranges);
    note_launch();
    ranges_kernel<<<G, 256, 0, st>>>(n_eff, cs.total_tiles, cn, kA, vA, depths, (int2 *)tile_ranges, keys64);
    note_launch();
    return cudaGetLastError();
}

}  // namespace gs
