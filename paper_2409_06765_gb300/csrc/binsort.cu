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
// Each LSD pass is one "onesweep" kernel: the global digit counts of every pass are
// known up front (a histogram kernel for the depth keys, the emission kernel for the
// tile keys), a CTA takes the next 4096-item block by ticket, ranks it stably (per-bit
// ballots inside a warp, warp prefixes across the CTA), publishes its per-digit counts
// and finds its per-digit offsets by decoupled look-back over the blocks before it, then
// reorders the block by digit in shared memory so the global stores of each digit's run
// are contiguous.  A CTA only ever waits on blocks whose tickets came earlier, i.e. on
// CTAs that are already running, and every wait is bounded: on a timeout the CTA raises
// an error flag (reported as K_out = -1) instead of waiting forever.
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
#include "gs_internal.cuh"

namespace gs {

constexpr int kRadix = 256;
constexpr int kMaxPasses = 8;            // 4 depth passes + up to 4 tile passes
constexpr int kOsThreads = 256;          // onesweep CTA (== kRadix)
constexpr int kOsIPT = 16;               // items per thread
constexpr int kOsBlock = kOsThreads * kOsIPT;
constexpr int kChunk = 1024;             // emission chunk (output slots)
constexpr int kEmitThreads = 256;
constexpr int kSlotsPerThread = kChunk / kEmitThreads;
constexpr long long kLookbackSpins = 1ll << 22;
constexpr unsigned long long kFlagAggregate = 1ull << 62;
constexpr unsigned long long kFlagPrefix = 2ull << 62;
constexpr unsigned long long kValueMask = (1ull << 62) - 1;

// misc region layout (ints)
constexpr int kMiscNeff = 0;
constexpr int kMiscErr = 1;
constexpr int kMiscTickets = 8;                          // [kMaxPasses]
constexpr int kMiscHist = 64;                            // [kMaxPasses][kRadix] global digit counts
constexpr int kMiscBase = kMiscHist + kMaxPasses * kRadix;  // [kMaxPasses][kRadix] exclusive digit starts
constexpr int kMiscInts = kMiscBase + kMaxPasses * kRadix;

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Lanes of the warp (within `valid`) whose digit equals this lane's: one ballot per digit
// bit, so the cost does not depend on how many distinct digits the warp holds.  Every lane
// of the warp must call it (lanes outside `valid` pass any digit).
__device__ __forceinline__ unsigned digit_peers(unsigned d, unsigned valid, int bits) {
    unsigned p = valid;
#pragma unroll 1
    for (int b = 0; b < bits; ++b) {
        const bool set = (d >> b) & 1u;
        const unsigned m = __ballot_sync(0xffffffffu, set);
        p &= set ? m : ~m;
    }
    return p;
}

// Exclusive scan of one int per thread over a CTA of 256 threads; also returns the total.
__device__ __forceinline__ int block_exclusive_scan(int x, int &total, int *s_tmp /* >= 8 ints */) {
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
    for (int w = 0; w < 8; ++w) {
        int v = s_tmp[w];
        if (w < warp) wpre += v;
        total += v;
    }
    __syncthreads();
    return wpre + inc - x;
}

__device__ __forceinline__ unsigned long long load_volatile_u64(const unsigned long long *p) {
    return *reinterpret_cast<const volatile unsigned long long *>(p);
}

__device__ __forceinline__ void store_volatile_u64(unsigned long long *p, unsigned long long v) {
    *reinterpret_cast<volatile unsigned long long *>(p) = v;
}

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------

__global__ void zero_ints_kernel(int n, int *__restrict__ p) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) p[t] = 0;
}

// Zeroes the look-back words of the blocks a pass will use (n from the device when given).
__global__ void zero_lookback_kernel(const int *__restrict__ n_dev, int n_host, unsigned long long *__restrict__ lb,
                                     int *__restrict__ ticket) {
    const int n = n_dev ? *n_dev : n_host;
    const long long words = (long long)((n + kOsBlock - 1) / kOsBlock) * kRadix;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < words;
         t += (long long)gridDim.x * blockDim.x)
        lb[t] = 0ull;
    if (blockIdx.x == 0 && threadIdx.x == 0) *ticket = 0;
}

// Exclusive digit starts of every pass from the global digit counts (one CTA of 256).
__global__ void digit_base_kernel(const int *__restrict__ hist, int *__restrict__ base, int passes) {
    __shared__ int s_tmp[8];
    for (int p = 0; p < passes; ++p) {
        int tot;
        const int ex = block_exclusive_scan(hist[p * kRadix + threadIdx.x], tot, s_tmp);
        base[p * kRadix + threadIdx.x] = ex;
    }
}

__global__ void empty_result_kernel(long long *__restrict__ K_out, int *__restrict__ n_eff) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        *K_out = 0;
        *n_eff = 0;
    }
}

// Reports a look-back timeout (never expected) through K_out.
__global__ void report_error_kernel(const int *__restrict__ err, long long *__restrict__ K_out) {
    if (threadIdx.x == 0 && blockIdx.x == 0 && *err) *K_out = -1;
}

// ---------------------------------------------------------------------------
// stage 1 keys + the digit histograms of all four depth passes
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(256) depth_keys_kernel(int CN, const float *__restrict__ depths,
                                                         const int *__restrict__ radii, uint32_t *__restrict__ keys,
                                                         int *__restrict__ vals, int *__restrict__ hist) {
    __shared__ int s_h[4][kRadix];
    for (int i = threadIdx.x; i < 4 * kRadix; i += blockDim.x) (&s_h[0][0])[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int stride = gridDim.x * blockDim.x;
    const int n_iter = (CN + stride - 1) / stride;
    for (int it = 0; it < n_iter; ++it) {
        const int i = it * stride + blockIdx.x * blockDim.x + threadIdx.x;
        const bool ok = i < CN;
        uint32_t key = 0xffffffffu;
        if (ok) {
            key = radii[i] > 0 ? __float_as_uint(depths[i]) : 0xffffffffu;
            keys[i] = key;
            vals[i] = i;
        }
        // invisible pairs all carry the same key: count them per warp, not per lane
        const unsigned inv = __ballot_sync(0xffffffffu, ok && key == 0xffffffffu);
        if (ok && key != 0xffffffffu) {
#pragma unroll
            for (int p = 0; p < 4; ++p) atomicAdd(&s_h[p][(key >> (8 * p)) & 0xffu], 1);
        }
        if (lane == 0 && inv) {
#pragma unroll
            for (int p = 0; p < 4; ++p) atomicAdd(&s_h[p][0xff], __popc(inv));
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 4 * kRadix; i += blockDim.x) {
        const int v = (&s_h[0][0])[i];
        if (v) atomicAdd(&hist[i], v);
    }
}

// ---------------------------------------------------------------------------
// one stable LSD pass (onesweep)
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(kOsThreads) onesweep_kernel(
    const uint32_t *__restrict__ keys_in, const int *__restrict__ vals_in, uint32_t *__restrict__ keys_out,
    int *__restrict__ vals_out, const int *__restrict__ n_dev, int n_host, int shift, int bits,
    const int *__restrict__ digit_base, unsigned long long *__restrict__ lookback, int *__restrict__ ticket,
    int *__restrict__ err) {
    constexpr int W = kOsThreads / 32;
    __shared__ int s_block;
    __shared__ int s_warp[W][kRadix];   // per-warp digit counts, then per-warp offsets inside the block's digit
    __shared__ int s_local[kRadix];     // start of each digit in the block reordered by digit
    __shared__ int s_shift[kRadix];     // global position - local position, per digit
    __shared__ int s_tmp[W];
    // the reorder buffer; during ranking its first W * kRadix words hold the per-warp lane
    // masks of each digit (zero between uses)
    __shared__ uint32_t s_keys[kOsBlock];
    __shared__ int s_vals[kOsBlock];
    unsigned(*s_peer)[kRadix] = reinterpret_cast<unsigned(*)[kRadix]>(s_keys);
    static_assert(W * kRadix <= kOsBlock, "lane masks must fit in the reorder buffer");
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n = n_dev ? *n_dev : n_host;
    const int nblocks = (n + kOsBlock - 1) / kOsBlock;
    const unsigned mask = (1u << bits) - 1u;
    if (threadIdx.x == 0) s_block = atomicAdd(ticket, 1);
    for (int i = threadIdx.x; i < W * kRadix; i += kOsThreads) {
        (&s_warp[0][0])[i] = 0;
        (&s_peer[0][0])[i] = 0u;
    }
    __syncthreads();
    const int blk = s_block;
    if (blk >= nblocks) return;  // uniform: the grid is sized for the capacity, n may be smaller
    const int t0 = blk * kOsBlock;
    const int items = min(kOsBlock, n - t0);

    // load (warp-striped: warp w owns a contiguous run, lanes in order) and rank
    const int wbase = t0 + warp * 32 * kOsIPT;
    uint32_t k[kOsIPT];
    int v[kOsIPT], rank[kOsIPT];
    unsigned dg[kOsIPT];
#pragma unroll
    for (int j = 0; j < kOsIPT; ++j) {
        const int i = wbase + j * 32 + lane;
        const bool ok = i < n;
        k[j] = ok ? keys_in[i] : 0u;
        v[j] = ok ? vals_in[i] : 0;
        dg[j] = ok ? ((k[j] >> shift) & mask) : 0xffffffffu;
    }
    // stable rank inside the warp: lanes holding the same digit find each other by OR-ing
    // their lane bit into the warp's word for that digit, the lowest of them advances the
    // warp's count and clears the word
    const unsigned lt = lanemask_lt();
#pragma unroll
    for (int j = 0; j < kOsIPT; ++j) {
        const bool ok = dg[j] != 0xffffffffu;
        const unsigned d = ok ? dg[j] : 0u;
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

    // per digit: block count, publish, look back, global start
    {
        const int d = threadIdx.x;  // kOsThreads == kRadix
        int run = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const int c = s_warp[w][d];
            s_warp[w][d] = run;
            run += c;
        }
        long long excl = 0;
        if (d <= (int)mask) {
            unsigned long long *mine = lookback + (size_t)blk * kRadix + d;
            if (blk == 0) {
                store_volatile_u64(mine, kFlagPrefix | (unsigned long long)run);
            } else {
                store_volatile_u64(mine, kFlagAggregate | (unsigned long long)run);
                // sum the counts of the blocks before, back to the nearest one whose inclusive
                // prefix is known; a block not yet published is waited for (bounded)
                long long spins = 0;
                for (int b = blk - 1; b >= 0; --b) {
                    const unsigned long long *other = lookback + (size_t)b * kRadix + d;
                    unsigned long long w = load_volatile_u64(other);
                    while ((w & (kFlagAggregate | kFlagPrefix)) == 0ull) {
                        if (++spins > kLookbackSpins) {
                            atomicExch(err, 1);
                            break;
                        }
                        __nanosleep(20);
                        w = load_volatile_u64(other);
                    }
                    excl += (long long)(w & kValueMask);
                    if ((w & kFlagPrefix) || spins > kLookbackSpins) break;
                }
                store_volatile_u64(mine, kFlagPrefix | (unsigned long long)(excl + run));
            }
        }
        int tot;
        const int local = block_exclusive_scan(run, tot, s_tmp);
        s_local[d] = local;
        s_shift[d] = (int)(digit_base[d] + excl) - local;
    }
    __syncthreads();
    // reorder the block by digit in shared memory
#pragma unroll
    for (int j = 0; j < kOsIPT; ++j) {
        if (dg[j] != 0xffffffffu) {
            const int lp = s_local[dg[j]] + s_warp[warp][dg[j]] + rank[j];
            if ((unsigned)lp < (unsigned)kOsBlock) {  // holds by construction
                s_keys[lp] = k[j];
                s_vals[lp] = v[j];
            }
        }
    }
    __syncthreads();
    // contiguous stores of every digit's run
    for (int i = threadIdx.x; i < items; i += kOsThreads) {
        const uint32_t kk = s_keys[i];
        const int pos = i + s_shift[(kk >> shift) & mask];
        if ((unsigned)pos < (unsigned)n) {  // holds by construction; guards the scatter
            keys_out[pos] = kk;
            vals_out[pos] = s_vals[i];
        }
    }
}

// ---------------------------------------------------------------------------
// stage 2: tile counts, offsets, chunk starts, balanced emission
// ---------------------------------------------------------------------------

__device__ __forceinline__ bool tile_rect(const CamSet &cs, int N, int i, const float2 *__restrict__ means2d,
                                          const int *__restrict__ radii, int &c, int &tx0, int &tx1, int &ty0,
                                          int &ty1) {
    if ((unsigned)i >= (unsigned)(cs.C * N)) return false;
    const int r = radii[i];
    if (r <= 0) return false;
    c = i / N;
    const CamDev &cam = cs.cam[c];
    const float2 m = means2d[i];
    int x0, x1, y0, y1;
    if (!pixel_box(m.x, m.y, r, cam.W, cam.H, x0, x1, y0, y1)) return false;
    const int t = cs.tile;
    tx0 = x0 / t;
    tx1 = x1 / t;
    ty0 = y0 / t;
    ty1 = y1 / t;
    return true;
}

// Tiles touched by each pair, in depth order, their sum per CTA, and each pair's tile
// rectangle packed as (tx0 | ty0 << 16, width | camera << 16) for the emission.
__global__ void __launch_bounds__(256) count_tiles_kernel(int CN, int N, const __grid_constant__ CamSet cs,
                                                          const int *__restrict__ order,
                                                          const float2 *__restrict__ means2d,
                                                          const int *__restrict__ radii, int *__restrict__ counts,
                                                          int2 *__restrict__ rects, long long *__restrict__ partials) {
    __shared__ long long s_w[8];
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    int cnt = 0;
    if (j < CN) {
        int c = 0, tx0 = 0, tx1 = 0, ty0 = 0, ty1 = 0;
        const bool ok = tile_rect(cs, N, order[j], means2d, radii, c, tx0, tx1, ty0, ty1);
        cnt = ok ? (tx1 - tx0 + 1) * (ty1 - ty0 + 1) : 0;
        counts[j] = cnt;
        rects[j] = make_int2(tx0 | (ty0 << 16), (ok ? tx1 - tx0 + 1 : 1) | (c << 16));
    }
    long long s = cnt;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        for (int w = 0; w < 8; ++w) t += s_w[w];
        partials[blockIdx.x] = t;
    }
}

// Exclusive scan of the per-CTA partials (one CTA); K = total; n_eff = min(K, capacity).
__global__ void __launch_bounds__(1024) partial_scan_kernel(int G, long long *__restrict__ partials,
                                                            long long capacity, long long *__restrict__ K_out,
                                                            int *__restrict__ n_eff) {
    __shared__ long long s_w[32];
    __shared__ long long s_carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int b0 = 0; b0 < G; b0 += 1024) {
        const int b = b0 + threadIdx.x;
        const long long v = b < G ? partials[b] : 0;
        long long x = v;
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
        if (b < G) partials[b] = s_carry + wpre + x - v;
        __syncthreads();
        if (threadIdx.x == 0) s_carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const long long run = s_carry;
        *K_out = run;
        *n_eff = (int)(run < capacity ? run : capacity);
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
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int cnt = j < CN ? counts[j] : 0;
    long long x = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    long long wpre = 0;
    for (int w = 0; w < warp; ++w) wpre += s_w[w];
    if (j >= CN) return;
    const long long off = partials[blockIdx.x] + wpre + x - cnt;
    offsets[j] = off;
    const long long limit = *n_eff;
    if (cnt > 0 && off < limit) {
        const long long end = min(off + cnt, limit);
        for (long long c = (off + kChunk - 1) / kChunk; c * kChunk < end; ++c) chunk_start[c] = j;
    }
}

// Balanced emission of (tile id, pair index) in depth order into [0, n_eff), plus the global
// digit counts of the tile passes (digit p = bits [digit_bits p, digit_bits (p+1)) of the id).
__global__ void __launch_bounds__(kEmitThreads) emit_kernel(
    int CN, const __grid_constant__ CamSet cs, const int *__restrict__ order, const int2 *__restrict__ rects,
    const long long *__restrict__ offsets, const int *__restrict__ chunk_start, const int *__restrict__ n_eff,
    uint32_t *__restrict__ tkeys, int *__restrict__ tvals, int tile_passes, int digit_bits, int *__restrict__ hist) {
    constexpr int P = kChunk;  // at most one pair per slot: every pair in the chunk has >= 1 tile
    __shared__ int s_off[P + 1];  // first slot of each pair, relative to the chunk
    __shared__ int s_xy[P];       // tx0 | ty0 << 16
    __shared__ int s_wc[P];       // rectangle width | camera << 16
    __shared__ int s_id[P];
    __shared__ uint32_t s_key[kChunk + kChunk / 32];
    __shared__ int s_val[kChunk + kChunk / 32];
    __shared__ int s_h[4][kRadix];
    __shared__ int s_np;
    for (int i = threadIdx.x; i < 4 * kRadix; i += kEmitThreads) (&s_h[0][0])[i] = 0;
    const int n = *n_eff;
    const int nchunks = (n + kChunk - 1) / kChunk;
    const unsigned dmask = (1u << digit_bits) - 1u;
    for (int ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {  // normally one chunk per CTA
        const long long k0 = (long long)ch * kChunk;
        const int len = (int)min((long long)kChunk, n - k0);
        const int j0 = chunk_start[ch];
        if (threadIdx.x == 0) s_np = 0;
        __syncthreads();
        // the pairs of this chunk: j0, j0 + 1, ... while their first slot is inside the chunk
        for (int s = threadIdx.x; s < P; s += kEmitThreads) {
            const int j = j0 + s;
            const long long off = (j < CN) ? offsets[j] : (1ll << 62);
            if (off < k0 + len) {
                const int2 rc = rects[j];
                s_off[s] = (int)(off - k0);  // negative for the pair that straddles into the chunk
                s_xy[s] = rc.x;
                s_wc[s] = rc.y;
                s_id[s] = order[j];
                atomicMax(&s_np, s + 1);
            }
        }
        __syncthreads();
        const int np = s_np;
        if (threadIdx.x == 0) s_off[np] = 1 << 30;
        __syncthreads();
        // each thread fills kSlotsPerThread consecutive slots
        const int q0 = threadIdx.x * kSlotsPerThread;
        if (q0 < len) {
            int lo = 0, hi = np - 1;  // last pair whose first slot is <= q0
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (s_off[mid] <= q0) lo = mid;
                else hi = mid - 1;
            }
            int p = lo;
#pragma unroll
            for (int u = 0; u < kSlotsPerThread; ++u) {
                const int q = q0 + u;
                if (q >= len) break;
                while (q >= s_off[p + 1]) ++p;
                const int kk = q - s_off[p];
                const int w = s_wc[p] & 0xffff, cam = s_wc[p] >> 16;
                const int tx0 = s_xy[p] & 0xffff, ty0 = s_xy[p] >> 16;
                const int ky = kk / w;
                const uint32_t tile = (uint32_t)(cs.cam[cam].tile_offset + (ty0 + ky) * cs.cam[cam].tiles_x + tx0 +
                                                 (kk - ky * w));
                s_key[q + (q >> 5)] = tile;  // padded: one bank shift per 32 slots
                s_val[q + (q >> 5)] = s_id[p];
#pragma unroll
                for (int pass = 0; pass < 4; ++pass)
                    if (pass < tile_passes) atomicAdd(&s_h[pass][(tile >> (digit_bits * pass)) & dmask], 1);
            }
        }
        __syncthreads();
        for (int q = threadIdx.x; q < len; q += kEmitThreads) {
            tkeys[k0 + q] = s_key[q + (q >> 5)];
            tvals[k0 + q] = s_val[q + (q >> 5)];
        }
        __syncthreads();
    }
    __syncthreads();
    for (int i = threadIdx.x; i < tile_passes * kRadix; i += kEmitThreads) {
        const int v = (&s_h[0][0])[i];
        if (v) atomicAdd(&hist[i], v);
    }
}

// Tile boundaries of the sorted list; each thread looks at 4 consecutive entries.
__global__ void ranges_kernel(const int *__restrict__ n_dev, int T, int CN, const uint32_t *__restrict__ tkeys,
                              const int *__restrict__ vals, const float *__restrict__ depths,
                              int2 *__restrict__ ranges, unsigned long long *__restrict__ keys64) {
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
    const long long os_blocks = (max_items + kOsBlock - 1) / kOsBlock;
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
    L.lookback = take((size_t)(os_blocks > 0 ? os_blocks : 1) * kRadix * 8);
    L.tk0 = take(Kcap * 4);
    L.tk1 = take(Kcap * 4);
    L.tvB = take(Kcap * 4);
    L.total = o;
    return L;
}

static cudaError_t onesweep_pass(const uint32_t *kin, const int *vin, uint32_t *kout, int *vout, const int *n_dev,
                                 int n_host, long long max_items, int shift, int bits, const int *base,
                                 unsigned long long *lookback, int *ticket, int *err, int G, cudaStream_t st) {
    zero_lookback_kernel<<<G, 256, 0, st>>>(n_dev, n_host, lookback, ticket);
    note_launch();
    const long long blocks = (max_items + kOsBlock - 1) / kOsBlock;
    if (blocks > 0) {
        onesweep_kernel<<<(unsigned)blocks, kOsThreads, 0, st>>>(kin, vin, kout, vout, n_dev, n_host, shift, bits,
                                                                 base, lookback, ticket, err);
        note_launch();
    }
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
    int *tickets = misc + kMiscTickets;
    int *hist = misc + kMiscHist;
    int *base = misc + kMiscBase;
    unsigned long long *lookback = (unsigned long long *)(w + L.lookback);
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
    // counters, histograms, error flag
    zero_ints_kernel<<<(kMiscInts + 255) / 256, 256, 0, st>>>(kMiscInts, misc);
    note_launch();
    // stage 1: depth order of all (camera, Gaussian) pairs
    const int eb = (cn + 255) / 256;
    depth_keys_kernel<<<G, 256, 0, st>>>(cn, depths, radii, dk0, dv0, hist);
    note_launch();
    digit_base_kernel<<<1, kRadix, 0, st>>>(hist, base, 4);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    for (int pass = 0; pass < 4; ++pass) {
        const bool even = (pass % 2) == 0;
        e = onesweep_pass(even ? dk0 : dk1, even ? dv0 : dv1, even ? dk1 : dk0, even ? dv1 : dv0, nullptr, cn, cn,
                          8 * pass, 8, base + pass * kRadix, lookback, tickets + pass, err, G, st);
        if (e != cudaSuccess) return e;
    }
    const int *order = dv0;  // after 4 passes the sorted pairs are back in (dk0, dv0)
    // stage 2: tile counts, offsets, balanced emission, stable sort by tile id
    count_tiles_kernel<<<eb, 256, 0, st>>>(cn, N, cs, order, (const float2 *)means2d, radii, counts, rects, partials);
    note_launch();
    partial_scan_kernel<<<1, 1024, 0, st>>>(eb, partials, Kcap, K_out, n_eff);
    note_launch();
    offsets_kernel<<<eb, 256, 0, st>>>(cn, counts, partials, n_eff, offsets, chunk_start);
    note_launch();
    // choose buffers so that the last pass writes into the caller's `values`
    uint32_t *kA = tk0, *kB = tk1;
    int *vA = (tpasses % 2 == 0) ? values : tvB;
    int *vB = (tpasses % 2 == 0) ? tvB : values;
    int *thist = hist + 4 * kRadix;
    int *tbase = base + 4 * kRadix;
    if (Kcap > 0) {
        const long long chunks = (Kcap + kChunk - 1) / kChunk;
        const long long emit_blocks = chunks < 2ll * G ? chunks : 2ll * G;  // persistent: 8 CTAs per SM
        emit_kernel<<<(unsigned)emit_blocks, kEmitThreads, 0, st>>>(cn, cs, order, rects, offsets, chunk_start, n_eff,
                                                                    kA, vA, tpasses, tdigit, thist);
        note_launch();
    }
    digit_base_kernel<<<1, kRadix, 0, st>>>(thist, tbase, tpasses);
    note_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    for (int pass = 0; pass < tpasses; ++pass) {
        e = onesweep_pass(kA, vA, kB, vB, n_eff, 0, Kcap, tdigit * pass, tdigit, tbase + pass * kRadix, lookback,
                          tickets + 4 + pass, err, G, st);
        if (e != cudaSuccess) return e;
        uint32_t *tk = kA;
        kA = kB;
        kB = tk;
        int *tv = vA;
        vA = vB;
        vB = tv;
    }
    // (kA, vA) now hold the sorted list; vA == values
    zero_ints_kernel<<<(2 * T + 255) / 256, 256, 0, st>>>(2 * T, tile_ranges);
    note_launch();
    ranges_kernel<<<G, 256, 0, st>>>(n_eff, T, cn, kA, vA, depths, (int2 *)tile_ranges, keys64);
    note_launch();
    report_error_kernel<<<1, 32, 0, st>>>(err, K_out);
    note_launch();
    return cudaGetLastError();
}

}  // namespace gs
