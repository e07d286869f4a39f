// Tile binning and per-tile depth sorting (App. C.2).
//
// The canonical result is the list of (tile, Gaussian) pairs ordered by the 64-bit key
// (global_tile << 32) | float_bits(depth), ties by flat index c*N + n.  Instead of one
// radix sort over K 64-bit keys, the same order is reached in two stable stages:
//   1. a 32-bit LSD radix sort of the C*N (camera, Gaussian) pairs by depth bits
//      (invisible pairs get key 0xFFFFFFFF, sort last and emit nothing);
//   2. emission of every pair's tiles in that depth order, followed by a stable LSD
//      radix sort of the K intersections by tile id alone (ceil(log2 T) bits, in passes
//      of at most 7 bits so each digit's run of a sorted block is long).
// Stability carries the depth order (and the index tie-break) into each tile's list.
//
// Each LSD pass is a reduce-then-scan over blocks of 4096 items: a histogram kernel
// writes every block's digit counts into a digit-major matrix, two small kernels turn the
// matrix into each (digit, block) pair's global start, and a persistent scatter kernel
// ranks each block stably in shared memory (atomic-OR peer masks within a warp, warp
// prefixes across the CTA), reorders it by digit in place and stores each digit's run
// contiguously.  The scatter streams its blocks into shared memory with 1-D bulk copies
// (TMA) double-buffered behind an mbarrier, so the next block is in flight while the
// current one is ranked.  No CTA waits on another CTA; the only waits are on the CTA's
// own bulk copies, and they are bounded (a timeout raises an error flag that the call
// reports as K_out = -1).
//
// Emission is balanced by output slot, not by pair: the output is cut into chunks of
// 1024 slots, a pass over the pairs records which pair starts each chunk, and a CTA
// fills a chunk with every thread writing 4 consecutive slots (staged through shared
// memory so the global stores are contiguous).  Pairs that cover thousands of tiles (big
// Gaussians close to the camera, all at the front of the depth order) therefore cost
// no more than many small ones.
//
// Every kernel reads the data-dependent counts (K) from device memory, so the host never
// synchronises and the whole call can be captured in a CUDA graph.
#include <stdlib.h>

#include "gs_internal.cuh"

namespace gs {

constexpr int kRadix = 256;
constexpr int kSortThreads = 256;        // histogram CTA (== kRadix)
constexpr int kSortIPT = 16;             // items per histogram thread
constexpr int kSortBlock = kSortThreads * kSortIPT;  // items per block of a pass
constexpr int kChunk = 1024;             // emission chunk (output slots)
constexpr int kEmitThreads = 256;
constexpr int kSlotsPerThread = kChunk / kEmitThreads;
static_assert(kSlotsPerThread == 4, "emission stores a thread's slots as one 16-byte store");
constexpr long long kWaitSpins = 1ll << 22;  // bound on a wait for a bulk copy

// misc region layout (ints)
constexpr int kMiscNeff = 0;
constexpr int kMiscErr = 1;
constexpr int kMiscRowsum = 64;                // [kMaxPasses][kRadix] digit totals of every pass
constexpr int kMaxPasses = 8;                  // 4 depth passes + up to 4 tile passes
constexpr int kFusedRowsumCols = 1024;         // passes of up to this many blocks sum digits by atomics
constexpr int kMiscInts = kMiscRowsum + kMaxPasses * kRadix;

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Exclusive scan of one int per thread over a CTA of NT threads; also returns the total.
template <int NT = 256>
__device__ __forceinline__ int block_exclusive_scan(int x, int &total, int *s_tmp /* >= NT/32 ints */) {
    constexpr int W = NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_tmp[warp] = inc;
    __syncthreads();
    int wpre = 0;
    total = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        int v = s_tmp[w];
        if (w < warp) wpre += v;
        total += v;
    }
    __syncthreads();
    return wpre + inc - x;
}

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------

__global__ void zero_ints_kernel(int n, int *__restrict__ p) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) p[t] = 0;
}

__global__ void empty_result_kernel(long long *__restrict__ K_out, int *__restrict__ n_eff) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        *K_out = 0;
        *n_eff = 0;
    }
}


// ---------------------------------------------------------------------------
// stage 1 keys
// ---------------------------------------------------------------------------

// Depth key of every (camera, Gaussian) pair.  A pair that touches no pixel (radius 0, or
// a pixel box that is empty after clipping to the image) gets 0xFFFFFFFF and so sorts
// after every pair with tiles: in depth order, every pair before the first such key has at
// least one tile, which the emission relies on.
__global__ void __launch_bounds__(256) depth_keys_kernel(int CN, int N, const __grid_constant__ CamSet cs,
                                                         const float2 *__restrict__ means2d,
                                                         const float *__restrict__ depths,
                                                         const int *__restrict__ radii, uint32_t *__restrict__ keys,
                                                         int *__restrict__ vals, int *__restrict__ misc) {
    if (blockIdx.x == 0)  // the sort's counters, digit totals and error flag start at zero
        for (int i = threadIdx.x; i < kMiscInts; i += blockDim.x) misc[i] = 0;
    // four consecutive pairs per thread: 16-byte loads of radii, depths and means, 16-byte stores
    const int i0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (i0 >= CN) return;
    const bool vec = ((reinterpret_cast<uintptr_t>(radii) | reinterpret_cast<uintptr_t>(depths) |
                       reinterpret_cast<uintptr_t>(means2d)) & 15) == 0;  // (caller arrays: usually aligned)
    if (vec && i0 + 4 <= CN) {  // i0 is a multiple of 4: 16-byte loads and stores
        const int4 r = *reinterpret_cast<const int4 *>(radii + i0);
        const float4 d = *reinterpret_cast<const float4 *>(depths + i0);
        const float4 m01 = *reinterpret_cast<const float4 *>(means2d + i0);
        const float4 m23 = *reinterpret_cast<const float4 *>(means2d + i0 + 2);
        const int rr[4] = {r.x, r.y, r.z, r.w};
        const float dd[4] = {d.x, d.y, d.z, d.w};
        const float2 mm[4] = {make_float2(m01.x, m01.y), make_float2(m01.z, m01.w), make_float2(m23.x, m23.y),
                              make_float2(m23.z, m23.w)};
        uint32_t k[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            bool ok = rr[u] > 0;
            if (ok) {
                const CamDev &cam = cs.cam[(i0 + u) / N];
                int x0, x1, y0, y1;
                ok = pixel_box(mm[u].x, mm[u].y, rr[u], cam.W, cam.H, x0, x1, y0, y1);
            }
            k[u] = ok ? __float_as_uint(dd[u]) : 0xffffffffu;
        }
        *reinterpret_cast<uint4 *>(keys + i0) = make_uint4(k[0], k[1], k[2], k[3]);
        *reinterpret_cast<int4 *>(vals + i0) = make_int4(i0, i0 + 1, i0 + 2, i0 + 3);
        return;
    }
    for (int i = i0; i < min(CN, i0 + 4); ++i) {  // the ragged end, or unaligned inputs
        const int r = radii[i];
        bool ok = r > 0;
        if (ok) {
            const CamDev &cam = cs.cam[i / N];
            const float2 m = means2d[i];
            int x0, x1, y0, y1;
            ok = pixel_box(m.x, m.y, r, cam.W, cam.H, x0, x1, y0, y1);
        }
        keys[i] = ok ? __float_as_uint(depths[i]) : 0xffffffffu;
        vals[i] = i;
    }
}

// ---------------------------------------------------------------------------
// one stable LSD pass as reduce-then-scan: no CTA waits on another
// ---------------------------------------------------------------------------

// Digit counts of every kSortBlock-item block: hist[d * cols + b] (digit-major), and, when
// rowsum is given, the pass's digit totals rowsum[d] by atomic adds (zeroed before the sort;
// used for passes of few blocks, where the adds to one counter do not queue up).
__global__ void __launch_bounds__(kSortThreads) block_hist_kernel(const uint32_t *__restrict__ keys,
                                                                const int *__restrict__ n_dev, int n_host, int shift,
                                                                int bits, int cols, int *__restrict__ hist,
                                                                int *__restrict__ rowsum) {
    constexpr int W = kSortThreads / 32;
    __shared__ int s_h[W][kRadix];
    const int warp = threadIdx.x >> 5;
    const int n = n_dev ? *n_dev : n_host;
    const int b = blockIdx.x;
    const int t0 = b * kSortBlock;
    if (t0 >= n) return;  // uniform
    for (int i = threadIdx.x; i < W * kRadix; i += kSortThreads) (&s_h[0][0])[i] = 0;
    __syncthreads();
    const unsigned mask = (1u << bits) - 1u;
    const int end = min(n, t0 + kSortBlock);
    uint4 q[kSortIPT / 4];  // all loads in flight before the first atomic
#pragma unroll
    for (int r = 0; r < kSortIPT / 4; ++r) {
        const int i0 = t0 + (r * kSortThreads + threadIdx.x) * 4;  // 16-byte aligned: keys are 256-byte aligned
        if (i0 + 3 < end) {
            q[r] = *reinterpret_cast<const uint4 *>(keys + i0);
        } else {
            q[r].x = i0 + 0 < end ? keys[i0 + 0] : 0u;
            q[r].y = i0 + 1 < end ? keys[i0 + 1] : 0u;
            q[r].z = i0 + 2 < end ? keys[i0 + 2] : 0u;
            q[r].w = i0 + 3 < end ? keys[i0 + 3] : 0u;
        }
    }
#pragma unroll
    for (int r = 0; r < kSortIPT / 4; ++r) {
        const int i0 = t0 + (r * kSortThreads + threadIdx.x) * 4;
        if (i0 + 0 < end) atomicAdd(&s_h[warp][(q[r].x >> shift) & mask], 1);
        if (i0 + 1 < end) atomicAdd(&s_h[warp][(q[r].y >> shift) & mask], 1);
        if (i0 + 2 < end) atomicAdd(&s_h[warp][(q[r].z >> shift) & mask], 1);
        if (i0 + 3 < end) atomicAdd(&s_h[warp][(q[r].w >> shift) & mask], 1);
    }
    __syncthreads();
    const int d = threadIdx.x;  // kSortThreads == kRadix
    int c = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) c += s_h[w][d];
    hist[(size_t)d * cols + b] = c;
    if (rowsum && c) atomicAdd(&rowsum[d], c);
}

// Row sums of the digit-major count matrix over its first nb = ceil(n / kSortBlock) columns.
__global__ void __launch_bounds__(kSortThreads) hist_rowsum_kernel(const int *__restrict__ n_dev, int n_host, int cols,
                                                                 const int *__restrict__ hist, int *__restrict__ rowsum) {
    __shared__ int s_tmp[8];
    const int n = n_dev ? *n_dev : n_host;
    const int nb = (n + kSortBlock - 1) / kSortBlock;
    const int *row = hist + (size_t)blockIdx.x * cols;
    int s = 0;
    for (int b = threadIdx.x; b < nb; b += kSortThreads) s += row[b];
    int tot;
    block_exclusive_scan(s, tot, s_tmp);
    if (threadIdx.x == 0) rowsum[blockIdx.x] = tot;
}

// hist[d * cols + b] <- global start of digit d for block b:
// sum_{d' < d} rowsum[d'] + sum_{b' < b} hist[d * cols + b'].
// Rows of up to 256 * MAXSEG blocks: every thread loads its whole segment into registers (all
// loads in flight at once) and rewrites it from there.
template <int MAXSEG>
__global__ void __launch_bounds__(kSortThreads) hist_scan_reg_kernel(const int *__restrict__ n_dev, int n_host,
                                                                   int cols, const int *__restrict__ rowsum,
                                                                   int *__restrict__ hist) {
    __shared__ int s_tmp[8];
    const int n = n_dev ? *n_dev : n_host;
    const int nb = (n + kSortBlock - 1) / kSortBlock;
    const int d = blockIdx.x;
    int *row = hist + (size_t)d * cols;
    const int seg = (nb + kSortThreads - 1) / kSortThreads;  // <= MAXSEG (checked by the host)
    const int b0 = threadIdx.x * seg, b1 = min(nb, b0 + seg);
    int v[MAXSEG];
#pragma unroll
    for (int k = 0; k < MAXSEG; ++k) v[k] = b0 + k < b1 ? row[b0 + k] : 0;
    const int pre = threadIdx.x < d ? rowsum[threadIdx.x] : 0;
    int s = 0;
#pragma unroll
    for (int k = 0; k < MAXSEG; ++k) s += v[k];
    int base, tot;
    block_exclusive_scan(pre, base, s_tmp);
    int run = base + block_exclusive_scan(s, tot, s_tmp);
#pragma unroll
    for (int k = 0; k < MAXSEG; ++k) {
        if (b0 + k < b1) row[b0 + k] = run;
        run += v[k];
    }
}

__global__ void __launch_bounds__(kSortThreads) hist_scan_kernel(const int *__restrict__ n_dev, int n_host, int cols,
                                                               const int *__restrict__ rowsum, int *__restrict__ hist) {
    __shared__ int s_tmp[8];
    const int n = n_dev ? *n_dev : n_host;
    const int nb = (n + kSortBlock - 1) / kSortBlock;
    const int d = blockIdx.x;
    int base;
    block_exclusive_scan(threadIdx.x < d ? rowsum[threadIdx.x] : 0, base, s_tmp);
    int *row = hist + (size_t)d * cols;
    // each thread scans a contiguous segment of the row
    const int seg = (nb + kSortThreads - 1) / kSortThreads;
    const int b0 = threadIdx.x * seg, b1 = min(nb, b0 + seg);
    int s = 0;
    for (int b = b0; b < b1; ++b) s += row[b];
    int tot;
    int run = base + block_exclusive_scan(s, tot, s_tmp);
    for (int b = b0; b < b1; ++b) {
        const int v = row[b];
        row[b] = run;
        run += v;
    }
}

// --- bulk copies (TMA, 1-D) into shared memory with mbarrier completion -------------

__device__ __forceinline__ unsigned smem_addr(const void *p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// 1-D bulk copy global -> shared (both 16-byte aligned, bytes a multiple of 16).
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for a bulk copy; false (and the error flag raised) when the copy never lands.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, unsigned parity, int *err) {
    for (long long it = 0; it < kWaitSpins; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
    }
    atomicExch(err, 1);
    return false;
}

constexpr int kTmaThreads = 512;
constexpr int kTmaWarps = kTmaThreads / 32;
constexpr int kTmaIPT = kSortBlock / kTmaThreads;  // items per scatter thread
constexpr size_t kTmaSmem = 2ull * kSortBlock * 8          // double-buffered keys + values (reordered in place)
                            + 2ull * kTmaWarps * kRadix * 4  // per-warp digit counts, per-warp peer masks
                            + 2ull * kRadix * 4              // local starts, shifts
                            + 128;                           // barriers, scratch

// Stable scatter of one pass by persistent CTAs (two per SM): the next block's keys and
// values are bulk-copied into the other shared-memory buffer while the current block is
// ranked and stored, so DRAM latency hides behind the ranking instead of stalling it.
// The ranked block is reordered by digit into its own input buffer (the items are held in
// registers across the barrier), so each CTA needs no separate reorder buffer.
__global__ void __launch_bounds__(kTmaThreads, 2) scatter_tma_kernel(const uint32_t *__restrict__ keys_in,
                                                                     const int *__restrict__ vals_in,
                                                                     uint32_t *__restrict__ keys_out,
                                                                     int *__restrict__ vals_out,
                                                                     const int *__restrict__ n_dev, int n_host,
                                                                     int shift, int bits, int cols,
                                                                     const int *__restrict__ hist,
                                                                     int *__restrict__ err) {
    constexpr int W = kTmaWarps;
    extern __shared__ __align__(128) unsigned char smem[];
    uint32_t *s_in_k = reinterpret_cast<uint32_t *>(smem);              // [2][kSortBlock]
    int *s_in_v = reinterpret_cast<int *>(s_in_k + 2 * kSortBlock);      // [2][kSortBlock]
    int(*s_warp)[kRadix] = reinterpret_cast<int(*)[kRadix]>(s_in_v + 2 * kSortBlock);
    unsigned(*s_peer)[kRadix] = reinterpret_cast<unsigned(*)[kRadix]>(&s_warp[W][0]);
    int *s_local = reinterpret_cast<int *>(&s_peer[W][0]);
    int *s_shift = s_local + kRadix;
    unsigned long long *s_bar = reinterpret_cast<unsigned long long *>(s_shift + kRadix);  // [2]
    int *s_tmp = reinterpret_cast<int *>(s_bar + 2);                                       // [W]

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n = n_dev ? *n_dev : n_host;
    const int nb = (n + kSortBlock - 1) / kSortBlock;
    const unsigned mask = (1u << bits) - 1u;
    if (blockIdx.x >= nb) return;  // uniform
    if (threadIdx.x == 0) {
        mbar_init(&s_bar[0], 1);
        mbar_init(&s_bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // issue the bulk copies of block `blk` into buffer `buf` (thread 0); the ragged tail of
    // the last block (fewer than 4 items past a 16-byte boundary) is loaded after the wait
    auto issue = [&](int blk, int buf) {
        const int t0 = blk * kSortBlock;
        const int items = min(kSortBlock, n - t0);
        const unsigned bytes = (unsigned)(items & ~3) * 4u;
        mbar_expect_tx(&s_bar[buf], 2u * bytes);
        if (bytes) {
            bulk_g2s(s_in_k + buf * kSortBlock, keys_in + t0, bytes, &s_bar[buf]);
            bulk_g2s(s_in_v + buf * kSortBlock, vals_in + t0, bytes, &s_bar[buf]);
        }
    };
    if (threadIdx.x == 0) issue(blockIdx.x, 0);
    const unsigned lt = lanemask_lt();
    int it = 0;
    for (int blk = blockIdx.x; blk < nb; blk += gridDim.x, ++it) {
        const int buf = it & 1;
        const int t0 = blk * kSortBlock;
        const int items = min(kSortBlock, n - t0);
        // prefetch the next block into the other buffer: the previous iteration ended with a
        // proxy fence by every thread and a CTA barrier after its last access to that buffer
        const int next = blk + gridDim.x;
        if (threadIdx.x == 0 && next < nb) issue(next, buf ^ 1);
        for (int i = threadIdx.x; i < W * kRadix; i += kTmaThreads) {
            (&s_warp[0][0])[i] = 0;
            if (it == 0) (&s_peer[0][0])[i] = 0u;  // the ranking leaves every peer mask at zero again
        }
        const bool landed = mbar_wait_bounded(&s_bar[buf], (unsigned)(it >> 1) & 1u, err);
        uint32_t *ik = s_in_k + buf * kSortBlock;
        int *iv = s_in_v + buf * kSortBlock;
        // ragged tail (< 4 items) with plain loads
        const int body = items & ~3;
        if (threadIdx.x < items - body) {
            ik[body + threadIdx.x] = keys_in[t0 + body + threadIdx.x];
            iv[body + threadIdx.x] = vals_in[t0 + body + threadIdx.x];
        }
        if (!__syncthreads_and(landed)) {
            // a copy never arrived: give up on this CTA's remaining blocks (the error flag is set);
            // wait, bounded, for the copy still in flight before shared memory is released
            if (threadIdx.x == 0 && next < nb) mbar_wait_bounded(&s_bar[buf ^ 1], (unsigned)((it + 1) >> 1) & 1u, err);
            return;
        }
        // stable rank inside each warp (warp w owns items [w*32*kTmaIPT, (w+1)*32*kTmaIPT))
        uint32_t kk[kTmaIPT];
        int vv[kTmaIPT], rank[kTmaIPT];
#pragma unroll
        for (int j = 0; j < kTmaIPT; ++j) {
            const int li = warp * 32 * kTmaIPT + j * 32 + lane;
            const bool ok = li < items;
            kk[j] = ok ? ik[li] : 0u;
            vv[j] = ok ? iv[li] : 0;
            const unsigned d = ok ? ((kk[j] >> shift) & mask) : 0u;
            if (ok) atomicOr(&s_peer[warp][d], 1u << lane);
            __syncwarp();
            const unsigned peers = ok ? s_peer[warp][d] : 0u;
            const int before = ok ? s_warp[warp][d] : 0;
            __syncwarp();
            if (ok && (__ffs(peers) - 1) == lane) {
                s_warp[warp][d] = before + __popc(peers);
                s_peer[warp][d] = 0u;
            }
            rank[j] = before + __popc(peers & lt);
            __syncwarp();
        }
        __syncthreads();
        {
            const int d = threadIdx.x;
            int run = 0;
            if (d < kRadix) {
                int c[W];  // all W counts in flight before the prefix is written back
#pragma unroll
                for (int w = 0; w < W; ++w) c[w] = s_warp[w][d];
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    s_warp[w][d] = run;
                    run += c[w];
                }
            }
            int tot;
            const int local = block_exclusive_scan<kTmaThreads>(run, tot, s_tmp);
            if (d < kRadix) {
                s_local[d] = local;
                s_shift[d] = hist[(size_t)d * cols + blk] - local;
            }
        }
        __syncthreads();
        // every item of the block is in registers: reorder by digit into the input buffer
#pragma unroll
        for (int j = 0; j < kTmaIPT; ++j) {
            const int li = warp * 32 * kTmaIPT + j * 32 + lane;
            if (li < items) {
                const unsigned d = (kk[j] >> shift) & mask;
                const int lp = s_local[d] + s_warp[warp][d] + rank[j];
                if ((unsigned)lp < (unsigned)kSortBlock) {  // holds by construction
                    ik[lp] = kk[j];
                    iv[lp] = vv[j];
                }
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < items; i += kTmaThreads) {
            const uint32_t k = ik[i];
            const int pos = i + s_shift[(k >> shift) & mask];
            if ((unsigned)pos < (unsigned)n) {  // holds by construction; guards the scatter
                keys_out[pos] = k;
                vals_out[pos] = iv[i];
            }
        }
        // order this iteration's generic-proxy accesses to the buffer before the bulk copy
        // that refills it two iterations on
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// stage 2: tile counts, offsets, chunk starts, balanced emission
// ---------------------------------------------------------------------------

// Tile rectangle of pair i from its radius r and 2D mean m (false when it touches no tile).
__device__ __forceinline__ bool tile_rect_of(const CamSet &cs, int N, int i, int r, float2 m, int &c, int &tx0,
                                             int &tx1, int &ty0, int &ty1) {
    if ((unsigned)i >= (unsigned)(cs.C * N) || r <= 0) return false;
    c = i / N;
    const CamDev &cam = cs.cam[c];
    int x0, x1, y0, y1;
    if (!pixel_box(m.x, m.y, r, cam.W, cam.H, x0, x1, y0, y1)) return false;
    const int t = cs.tile;
    tx0 = x0 / t;
    tx1 = x1 / t;
    ty0 = y0 / t;
    ty1 = y1 / t;
    return true;
}

constexpr int kPairsPerThread = 4;                            // consecutive pairs per thread
constexpr int kPairsPerCta = 256 * kPairsPerThread;           // pairs per CTA of the count/offset kernels

// Tiles touched by each pair, in depth order, their sum per CTA, and each pair's tile
// rectangle packed as (tx0 | ty0 << 16, width | camera << 16) for the emission.  A thread
// owns kPairsPerThread consecutive pairs: all their indices, then all their radii and means
// are requested before any is used, so the two dependent gathers overlap.
__global__ void __launch_bounds__(256) count_tiles_kernel(int CN, int N, int T, int *__restrict__ tile_ranges,
                                                          const __grid_constant__ CamSet cs,
                                                          const int *__restrict__ order,
                                                          const float2 *__restrict__ means2d,
                                                          const int *__restrict__ radii, int *__restrict__ counts,
                                                          int2 *__restrict__ rects, long long *__restrict__ partials) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 2 * T; i += gridDim.x * blockDim.x)
        tile_ranges[i] = 0;  // empty tiles read (0, 0); the ranges kernel fills the others later
    __shared__ long long s_w[8];
    const int j0 = blockIdx.x * kPairsPerCta + threadIdx.x * kPairsPerThread;
    int id[kPairsPerThread], r[kPairsPerThread];
    float2 m[kPairsPerThread];
    if (j0 + kPairsPerThread <= CN) {  // j0 is a multiple of 4 and order 16-byte aligned
        const int4 v = *reinterpret_cast<const int4 *>(order + j0);
        id[0] = v.x, id[1] = v.y, id[2] = v.z, id[3] = v.w;
    } else {
#pragma unroll
        for (int u = 0; u < kPairsPerThread; ++u) id[u] = j0 + u < CN ? order[j0 + u] : -1;
    }
#pragma unroll
    for (int u = 0; u < kPairsPerThread; ++u) {
        const bool ok = (unsigned)id[u] < (unsigned)CN;
        r[u] = ok ? radii[id[u]] : 0;
        m[u] = ok ? means2d[id[u]] : make_float2(0.f, 0.f);
    }
    int cnt[kPairsPerThread];
    int2 rc[kPairsPerThread];
#pragma unroll
    for (int u = 0; u < kPairsPerThread; ++u) {
        int c = 0, tx0 = 0, tx1 = 0, ty0 = 0, ty1 = 0;
        const bool ok = tile_rect_of(cs, N, id[u], r[u], m[u], c, tx0, tx1, ty0, ty1);
        cnt[u] = ok ? (tx1 - tx0 + 1) * (ty1 - ty0 + 1) : 0;
        rc[u] = make_int2(tx0 | (ty0 << 16), (ok ? tx1 - tx0 + 1 : 1) | (c << 16));
    }
    if (j0 + kPairsPerThread <= CN) {
        *reinterpret_cast<int4 *>(counts + j0) = make_int4(cnt[0], cnt[1], cnt[2], cnt[3]);
        *reinterpret_cast<int4 *>(rects + j0) = make_int4(rc[0].x, rc[0].y, rc[1].x, rc[1].y);
        *reinterpret_cast<int4 *>(rects + j0 + 2) = make_int4(rc[2].x, rc[2].y, rc[3].x, rc[3].y);
    } else {
#pragma unroll
        for (int u = 0; u < kPairsPerThread; ++u)
            if (j0 + u < CN) {
                counts[j0 + u] = cnt[u];
                rects[j0 + u] = rc[u];
            }
    }
    long long sum = (long long)cnt[0] + cnt[1] + cnt[2] + cnt[3];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        for (int w = 0; w < 8; ++w) t += s_w[w];
        partials[blockIdx.x] = t;
    }
}

// Exclusive scan of the per-CTA partials (one CTA); K = total; n_eff = min(K, capacity).
// Each thread owns a contiguous segment: it sums it, the CTA scans the segment sums, and the
// thread rewrites its segment from its exclusive start (one pass, no per-round barriers).
__global__ void __launch_bounds__(1024) partial_scan_kernel(int G, long long *__restrict__ partials,
                                                            long long capacity, long long *__restrict__ K_out,
                                                            int *__restrict__ n_eff) {
    __shared__ long long s_w[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int per = (G + 1023) / 1024;
    const int b0 = min(G, threadIdx.x * per), b1 = min(G, b0 + per);
    long long sum = 0;
    for (int b = b0; b < b1; ++b) sum += partials[b];
    long long x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    long long wpre = 0, tot = 0;
    for (int w = 0; w < 32; ++w) {
        if (w < warp) wpre += s_w[w];
        tot += s_w[w];
    }
    long long run = wpre + x - sum;
    for (int b = b0; b < b1; ++b) {
        const long long v = partials[b];
        partials[b] = run;
        run += v;
    }
    if (threadIdx.x == 0) {
        *K_out = tot;
        *n_eff = (int)(tot < capacity ? tot : capacity);
    }
}

// Exclusive offsets of every pair, and for each emission chunk the pair holding its first
// slot (chunk_start[c] = j when c * kChunk falls in [offsets[j], offsets[j] + counts[j])).
__global__ void __launch_bounds__(256) offsets_kernel(int CN, const int *__restrict__ counts,
                                                      const long long *__restrict__ partials,
                                                      const int *__restrict__ n_eff, long long *__restrict__ offsets,
                                                      int *__restrict__ chunk_start) {
    __shared__ long long s_w[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int j0 = blockIdx.x * kPairsPerCta + threadIdx.x * kPairsPerThread;
    int cnt[kPairsPerThread];
    if (j0 + kPairsPerThread <= CN) {
        const int4 v = *reinterpret_cast<const int4 *>(counts + j0);
        cnt[0] = v.x, cnt[1] = v.y, cnt[2] = v.z, cnt[3] = v.w;
    } else {
#pragma unroll
        for (int u = 0; u < kPairsPerThread; ++u) cnt[u] = j0 + u < CN ? counts[j0 + u] : 0;
    }
    const long long mine = (long long)cnt[0] + cnt[1] + cnt[2] + cnt[3];
    long long x = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    long long wpre = 0;
    for (int w = 0; w < warp; ++w) wpre += s_w[w];
    long long off = partials[blockIdx.x] + wpre + x - mine;
    const long long limit = *n_eff;
#pragma unroll
    for (int u = 0; u < kPairsPerThread; ++u) {
        const int j = j0 + u;
        if (j >= CN) break;
        offsets[j] = off;
        if (cnt[u] > 0 && off < limit) {
            const long long end = min(off + cnt[u], limit);
            for (long long c = (off + kChunk - 1) / kChunk; c * kChunk < end; ++c) chunk_start[c] = j;
        }
        off += cnt[u];
    }
}

// Balanced emission of (tile id, pair index) in depth order into [0, n_eff).
__global__ void __launch_bounds__(kEmitThreads) emit_kernel(
    int CN, const __grid_constant__ CamSet cs, const int *__restrict__ order, const int2 *__restrict__ rects,
    const long long *__restrict__ offsets, const int *__restrict__ chunk_start, const int *__restrict__ n_eff,
    uint32_t *__restrict__ tkeys, int *__restrict__ tvals) {
    // at most one pair per slot: every pair before the first tile-less one has >= 1 tile, and
    // tile-less pairs (offset n_eff or beyond) are never inside a chunk
    constexpr int P = kChunk;
    __shared__ int s_off[P + 1];  // first slot of each pair, relative to the chunk
    __shared__ int s_base[P];     // global tile id of the rectangle's first tile
    __shared__ int s_wt[P];       // rectangle width | the camera's tiles per row << 16
    __shared__ int s_id[P];
    const int n = *n_eff;
    const int nchunks = (n + kChunk - 1) / kChunk;
    for (int ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {  // normally one chunk per CTA
        const long long k0 = (long long)ch * kChunk;
        const int len = (int)min((long long)kChunk, n - k0);
        const int j0 = chunk_start[ch];
        // the pairs of this chunk: j0, j0 + 1, ... while their first slot is inside the chunk
        // (offsets are non-decreasing, so they form a prefix and a count gives their number);
        // they end at the pair holding the next chunk's first slot, so only those are read
        const int j_end = (ch + 1 < nchunks) ? chunk_start[ch + 1] : CN - 1;
        const int cand = min(P, j_end - j0 + 1);
        int np = 0;
        for (int s0 = 0; s0 < cand; s0 += kEmitThreads) {
            const int s = s0 + threadIdx.x;
            const int j = j0 + s;
            const long long off = (j < CN) ? offsets[j] : (1ll << 62);
            const bool in = off < k0 + len;
            if (in) {
                const int2 rc = rects[j];
                const CamDev &cam = cs.cam[rc.y >> 16];
                s_off[s] = (int)(off - k0);  // negative for the pair that straddles into the chunk
                s_base[s] = cam.tile_offset + (rc.x >> 16) * cam.tiles_x + (rc.x & 0xffff);
                s_wt[s] = (rc.y & 0xffff) | (cam.tiles_x << 16);
                s_id[s] = order[j];
            }
            np += __syncthreads_count(in);
        }
        if (threadIdx.x == 0) s_off[np] = 1 << 30;
        __syncthreads();
        // each thread fills kSlotsPerThread consecutive slots and stores them as one 16-byte
        // store per array (consecutive threads, consecutive 16-byte pieces)
        const int q0 = threadIdx.x * kSlotsPerThread;
        if (q0 < len) {
            int lo = 0, hi = np - 1;  // last pair whose first slot is <= q0
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (s_off[mid] <= q0) lo = mid;
                else hi = mid - 1;
            }
            int p = lo;
            // position (kx, ky) of slot q0 in its pair's tile rectangle: one division, then the
            // following slots step through the rectangle (a new pair starts at its corner)
            int w = s_wt[p] & 0xffff, tx = s_wt[p] >> 16;
            const int kk = q0 - s_off[p];
            const int ky = kk / w;
            int kx = kk - ky * w;
            int tile = s_base[p] + ky * tx + kx;
            uint32_t key[kSlotsPerThread];
            int val[kSlotsPerThread];
#pragma unroll
            for (int u = 0; u < kSlotsPerThread; ++u) {
                const int q = q0 + u;
                if (u > 0 && q < len) {
                    if (q >= s_off[p + 1]) {
                        while (q >= s_off[p + 1]) ++p;
                        w = s_wt[p] & 0xffff;
                        tx = s_wt[p] >> 16;
                        kx = 0;
                        tile = s_base[p];
                    } else if (++kx == w) {
                        kx = 0;
                        tile += tx - w + 1;  // first tile of the next row of the rectangle
                    } else {
                        ++tile;
                    }
                }
                key[u] = (uint32_t)tile;
                val[u] = s_id[p];
            }
            if (q0 + kSlotsPerThread <= len) {  // k0 and q0 are multiples of 4: 16-byte aligned
                *reinterpret_cast<uint4 *>(tkeys + k0 + q0) = make_uint4(key[0], key[1], key[2], key[3]);
                *reinterpret_cast<int4 *>(tvals + k0 + q0) = make_int4(val[0], val[1], val[2], val[3]);
            } else {
#pragma unroll
                for (int u = 0; u < kSlotsPerThread; ++u)
                    if (q0 + u < len) {
                        tkeys[k0 + q0 + u] = key[u];
                        tvals[k0 + q0 + u] = val[u];
                    }
            }
        }
        __syncthreads();  // the next chunk reuses the shared arrays
    }
}

// Tile boundaries of the sorted list; each thread looks at 4 consecutive entries.
__global__ void ranges_kernel(const int *__restrict__ n_dev, int T, int CN, const uint32_t *__restrict__ tkeys,
                              const int *__restrict__ vals, const float *__restrict__ depths,
                              int2 *__restrict__ ranges, unsigned long long *__restrict__ keys64,
                              const int *__restrict__ err, long long *__restrict__ K_out) {
    // a timed-out bulk-copy wait in any pass (never expected) is reported through K_out
    if (blockIdx.x == 0 && threadIdx.x == 0 && *err) *K_out = -1;
    const int n = *n_dev;
    const int nq = (n + 3) / 4;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
        const int p0 = 4 * q;
        uint32_t t[6];
        t[0] = p0 > 0 ? tkeys[p0 - 1] : 0xffffffffu;
        if (p0 + 3 < n) {
            uint4 v = *reinterpret_cast<const uint4 *>(tkeys + p0);
            t[1] = v.x; t[2] = v.y; t[3] = v.z; t[4] = v.w;
        } else {
#pragma unroll
            for (int u = 0; u < 4; ++u) t[1 + u] = p0 + u < n ? tkeys[p0 + u] : 0xffffffffu;
        }
        t[5] = p0 + 4 < n ? tkeys[p0 + 4] : 0xffffffffu;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int p = p0 + u;
            if (p >= n) break;
            const uint32_t tt = t[1 + u];
            if (tt >= (uint32_t)T) continue;  // holds by construction
            if (t[u] != tt) ranges[tt].x = p;
            if (t[2 + u] != tt) ranges[tt].y = p + 1;
            if (keys64) {
                const int v = vals[p];
                keys64[p] = ((unsigned long long)tt << 32) |
                            ((unsigned)v < (unsigned)CN ? __float_as_uint(depths[v]) : 0u);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// launch order of the compositing kernels: longest tile lists first
// ---------------------------------------------------------------------------

// Bucket of a list length: 0 for an empty list, else 1 + 2 floor(log2 len) + the bit below
// the leading one (half-octave buckets, at most 63).
__device__ __forceinline__ int length_bucket(int len) {
    if (len <= 0) return 0;
    const int l = 31 - __clz(len);
    const int half = l > 0 ? (len >> (l - 1)) & 1 : 0;
    return 1 + 2 * l + half;
}

// One CTA: counting sort of the tiles by bucket, buckets in descending order.
__global__ void __launch_bounds__(1024) tile_order_kernel(int T, const int2 *__restrict__ ranges,
                                                          int *__restrict__ order) {
    __shared__ int s_cnt[64];
    __shared__ int s_cur[64];
    if (threadIdx.x < 64) s_cnt[threadIdx.x] = 0;
    if (threadIdx.x < 4) order[T + threadIdx.x] = 0;  // work counters of persistent compositing launches
    __syncthreads();
    for (int t = threadIdx.x; t < T; t += blockDim.x) {
        const int2 r = ranges[t];
        atomicAdd(&s_cnt[length_bucket(r.y - r.x)], 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int b = 63; b >= 0; --b) {
            s_cur[b] = run;
            run += s_cnt[b];
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < T; t += blockDim.x) {
        const int2 r = ranges[t];
        const int pos = atomicAdd(&s_cur[length_bucket(r.y - r.x)], 1);
        if ((unsigned)pos < (unsigned)T) order[pos] = t;  // holds by construction
    }
}

cudaError_t launch_tile_order(int T, const int *tile_ranges, int *order, cudaStream_t st) {
    if (T <= 0) return cudaSuccess;
    tile_order_kernel<<<1, 1024, 0, st>>>(T, (const int2 *)tile_ranges, order);
    note_launch();
    return cudaGetLastError();
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
    (void)G;
    BinSortLayout L;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o += align256(bytes);
        return at;
    };
    const long long cnb = (CN + 255) / 256;
    const long long max_items = CN > Kcap ? CN : Kcap;
    const long long cols = (max_items + kSortBlock - 1) / kSortBlock;
    L.dk0 = take(CN * 4);
    L.dk1 = take(CN * 4);
    L.dv0 = take(CN * 4);
    L.dv1 = take(CN * 4);
    L.counts = take(CN * 4);
    L.rects = take(CN * 8);
    L.offsets = take(CN * 8);
    L.chunk_start = take(((Kcap + kChunk - 1) / kChunk + 1) * 4);
    L.partials = take((size_t)(cnb + 1) * 8);
    L.misc = take((size_t)kMiscInts * 4);
    L.matrix = take((size_t)(cols > 0 ? cols : 1) * kRadix * 4);
    L.tk0 = take(Kcap * 4);
    L.tk1 = take(Kcap * 4);
    L.tvB = take(Kcap * 4);
    L.total = o;
    return L;
}

// One stable LSD pass by reduce-then-scan over blocks of kSortBlock items.
static cudaError_t rts_pass(const uint32_t *kin, const int *vin, uint32_t *kout, int *vout, const int *n_dev,
                            int n_host, long long max_items, int shift, int bits, int *matrix, int *rowsum, int *err,
                            cudaStream_t st) {
    const int cols = (int)((max_items + kSortBlock - 1) / kSortBlock);
    if (cols <= 0) return cudaSuccess;
    const bool fused = cols <= kFusedRowsumCols;
    block_hist_kernel<<<cols, kSortThreads, 0, st>>>(kin, n_dev, n_host, shift, bits, cols, matrix,
                                                     fused ? rowsum : nullptr);
    note_launch();
    if (!fused) {
        hist_rowsum_kernel<<<kRadix, kSortThreads, 0, st>>>(n_dev, n_host, cols, matrix, rowsum);
        note_launch();
    }
    if (cols <= kSortThreads * 4)
        hist_scan_reg_kernel<4><<<kRadix, kSortThreads, 0, st>>>(n_dev, n_host, cols, rowsum, matrix);
    else if (cols <= kSortThreads * 32)
        hist_scan_reg_kernel<32><<<kRadix, kSortThreads, 0, st>>>(n_dev, n_host, cols, rowsum, matrix);
    else
        hist_scan_kernel<<<kRadix, kSortThreads, 0, st>>>(n_dev, n_host, cols, rowsum, matrix);
    note_launch();
    cudaError_t e =
        ensure_smem((const void *)scatter_tma_kernel, (int)kTmaSmem);
    if (e != cudaSuccess) return e;
    const int persistent = 2 * sort_grid_blocks() / 4;  // two CTAs per SM
    scatter_tma_kernel<<<cols < persistent ? cols : persistent, kTmaThreads, kTmaSmem, st>>>(
        kin, vin, kout, vout, n_dev, n_host, shift, bits, cols, matrix, err);
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
    int2 *rects = (int2 *)(w + L.rects);
    long long *offsets = (long long *)(w + L.offsets);
    int *chunk_start = (int *)(w + L.chunk_start);
    long long *partials = (long long *)(w + L.partials);
    int *misc = (int *)(w + L.misc);
    int *n_eff = misc + kMiscNeff;
    int *err = misc + kMiscErr;
    int *matrix = (int *)(w + L.matrix);
    int *rowsum = misc + kMiscRowsum;
    uint32_t *tk0 = (uint32_t *)(w + L.tk0), *tk1 = (uint32_t *)(w + L.tk1);
    int *tvB = (int *)(w + L.tvB);

    const int cn = (int)CN;
    const int T = cs.total_tiles;
    if (cn == 0) {
        empty_result_kernel<<<1, 32, 0, st>>>(K_out, n_eff);
        note_launch();
        zero_ints_kernel<<<(2 * T + 255) / 256, 256, 0, st>>>(2 * T, tile_ranges);
        note_launch();
        return cudaGetLastError();
    }
    const int bits = tile_bits(T);
    const int tpasses = (bits + 6) / 7;                // passes of at most 7 bits
    const int tdigit = (bits + tpasses - 1) / tpasses;  // equal digit widths
    // stage 1: depth order of all (camera, Gaussian) pairs
    const int eb = (cn + 1023) / 1024;  // four pairs per thread
    depth_keys_kernel<<<eb, 256, 0, st>>>(cn, N, cs, (const float2 *)means2d, depths, radii, dk0, dv0, misc);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    for (int pass = 0; pass < 4; ++pass) {
        const bool even = (pass % 2) == 0;
        e = rts_pass(even ? dk0 : dk1, even ? dv0 : dv1, even ? dk1 : dk0, even ? dv1 : dv0, nullptr, cn, cn, 8 * pass,
                     8, matrix, rowsum + pass * kRadix, err, st);
        if (e != cudaSuccess) return e;
    }
    const int *order = dv0;  // after 4 passes the sorted pairs are back in (dk0, dv0)
    // stage 2: tile counts, offsets, balanced emission, stable sort by tile id
    const int pb = (cn + kPairsPerCta - 1) / kPairsPerCta;  // CTAs of the count and offset kernels
    count_tiles_kernel<<<pb, 256, 0, st>>>(cn, N, T, tile_ranges, cs, order, (const float2 *)means2d, radii, counts,
                                           rects, partials);
    note_launch();
    partial_scan_kernel<<<1, 1024, 0, st>>>(pb, partials, Kcap, K_out, n_eff);
    note_launch();
    offsets_kernel<<<pb, 256, 0, st>>>(cn, counts, partials, n_eff, offsets, chunk_start);
    note_launch();
    // choose buffers so that the last pass writes into the caller's `values`
    uint32_t *kA = tk0, *kB = tk1;
    int *vA = (tpasses % 2 == 0) ? values : tvB;
    int *vB = (tpasses % 2 == 0) ? tvB : values;
    if (Kcap > 0) {
        const long long chunks = (Kcap + kChunk - 1) / kChunk;
        const long long emit_blocks = chunks < 2ll * G ? chunks : 2ll * G;  // persistent: 8 CTAs per SM
        emit_kernel<<<(unsigned)emit_blocks, kEmitThreads, 0, st>>>(cn, cs, order, rects, offsets, chunk_start, n_eff,
                                                                    kA, vA);
        note_launch();
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    for (int pass = 0; pass < tpasses; ++pass) {
        e = rts_pass(kA, vA, kB, vB, n_eff, 0, Kcap, tdigit * pass, tdigit, matrix, rowsum + (4 + pass) * kRadix, err,
                     st);
        if (e != cudaSuccess) return e;
        uint32_t *tk = kA;
        kA = kB;
        kB = tk;
        int *tv = vA;
        vA = vB;
        vB = tv;
    }
    // (kA, vA) now hold the sorted list; vA == values
    // one thread per 4 entries of the largest possible list (threads past the real count exit)
    const long long rq = (Kcap + 3) / 4;
    ranges_kernel<<<(unsigned)((rq + 255) / 256 > 0 ? (rq + 255) / 256 : 1), 256, 0, st>>>(
        n_eff, T, cn, kA, vA, depths, (int2 *)tile_ranges, keys64, err, K_out);
    note_launch();
    return cudaGetLastError();
}

}  // namespace gs
