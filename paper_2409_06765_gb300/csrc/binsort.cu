// Tile binning and per-tile depth sorting (App. C.2).
//
// The canonical result is the list of (tile, Gaussian) pairs ordered by the 64-bit key
// (global_tile << 32) | float_bits(depth), ties by flat index c*N + n.  Instead of one
// radix sort over K 64-bit keys, the same order is reached in two stable stages:
//   1. a stable LSD radix sort of the C*N (camera, Gaussian) pairs by the 32 depth bits, in
//      four passes of 8 bits.  The first pass also drops the pairs that touch no pixel (key
//      0xFFFFFFFF), so the later passes and stage 2 see only the visible ones;
//   2. the K intersections in that depth order, sorted stably by tile id alone.  A pair's
//      intersections are the tiles of its tile rectangle, so the list of "slots" in depth
//      order is defined by the pairs' tile counts and rectangles.  When the tile ids fit one
//      digit of at most 11 bits (up to 2048 tiles: one 1080p view at 32x32 tiles), a single
//      counting pass regenerates every slot from a 16-byte pair record, once to count and
//      once to place, and writes only the final values: no K-sized key or value array
//      exists.  More tiles take further LSD passes over materialised (tile, value) arrays.
// Stability carries the depth order (and the index tie-break) into each tile's list.
//
// Every pass is reduce-then-scan over blocks of items (4096 for the depth passes, 16384
// for the tile passes): a histogram kernel writes each block's digit counts into a
// digit-major matrix (and adds the digit totals), a scan kernel turns the matrix into each
// (digit, block)'s global start, and a rank kernel places the block.  The rank kernel
// gives each of its 16 warps a contiguous segment of the block: the warps first count
// their digits into per-warp 16-bit counters (shared atomics), the CTA turns the counters
// into per-warp prefixes, and each warp then walks its segment in order, ranking 32 items
// at a time among equal digits, so equal digits keep their input order.  The ranking uses
// per-warp peer masks for the 8-bit depth digits (match.any for the last, skewed one) and,
// in the single tile pass, the window's pairs one after another (a pair's slots are
// distinct tiles).  The depth passes reorder each block by digit in shared memory and write
// contiguous runs; the tile pass writes each slot straight to its place (runs of a block
// over 2048 tiles are too short to coalesce).  No CTA waits on another CTA and nothing
// waits on the device.
//
// Every kernel reads the data-dependent counts (visible pairs, K) from device memory, so
// the host never synchronises and the whole call can be captured in a CUDA graph.
#include <stdlib.h>

#include "gs_internal.cuh"

namespace gs {

constexpr int kMaxDigitBits = 11;
constexpr int kMaxDigits = 1 << kMaxDigitBits;
constexpr int kDepthWarps = 16;                         // warps of a depth-pass CTA
constexpr int kDepthSeg = 256;                          // items per warp segment, depth passes
constexpr int kDepthBlock = kDepthWarps * kDepthSeg;    // 4096
constexpr int kTileWarps = 16;                          // warps of a tile-pass CTA
constexpr int kTileSeg = 1024;                          // slots per warp segment, tile passes
constexpr int kTileBlock = kTileWarps * kTileSeg;       // 16384
constexpr int kDepthDigitBits = 8;                      // digit width of the depth passes
constexpr int kDepthPasses = (32 + kDepthDigitBits - 1) / kDepthDigitBits;
constexpr int kMaxTilePasses = 4;                       // up to 2^28 tiles (the ABI's limit) in 8-bit passes
constexpr int kMaxPasses = kDepthPasses + kMaxTilePasses;
constexpr int kPeerDigits = 256;  // digits up to which the rank kernel ranks by peer masks

// misc region layout (ints)
constexpr int kMiscNeff = 0;   // slots actually emitted: min(K, capacity)
constexpr int kMiscNvis = 2;   // visible pairs (depth keys other than 0xFFFFFFFF)
constexpr int kMiscRowsum = 64;                         // [kMaxPasses][kMaxDigits] digit totals
constexpr int kMiscInts = kMiscRowsum + kMaxPasses * kMaxDigits;
constexpr unsigned kInvisible = 0xffffffffu;

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

__global__ void zero_ints_kernel(int n, int *__restrict__ p) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) p[t] = 0;
}

__global__ void empty_result_kernel(long long *__restrict__ K_out, int *__restrict__ misc) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        *K_out = 0;
        misc[kMiscNeff] = 0;
        misc[kMiscNvis] = 0;
    }
}

// ---------------------------------------------------------------------------
// stage 1 keys
// ---------------------------------------------------------------------------

// The tile rectangle of a pair whose clipped pixel box is [x0, x1] x [y0, y1]: (global id of
// its first tile, width | height << 16) in tiles; t = 1 << ts pixels per tile edge.
__device__ __forceinline__ int2 tile_rect(const CamDev &cam, int ts, int x0, int x1, int y0, int y1) {
    const int tx0 = x0 >> ts, tx1 = x1 >> ts, ty0 = y0 >> ts, ty1 = y1 >> ts;  // (x0, y0 >= 0 after clipping)
    return make_int2(cam.tile_offset + ty0 * cam.tiles_x + tx0, (tx1 - tx0 + 1) | ((ty1 - ty0 + 1) << 16));
}

// Depth key of every (camera, Gaussian) pair.  A pair that touches no pixel (radius 0, or
// a pixel box that is empty after clipping to the image) gets 0xFFFFFFFF; the first depth
// pass drops those, so every pair that reaches stage 2 has at least one tile.  The tile
// rectangle of every visible pair goes to rect[] in pair order (coalesced, while the radius and
// mean are at hand), so the depth-ordered count kernel gathers one 8-byte record per pair.
__global__ void __launch_bounds__(256) depth_keys_kernel(int CN, int N, const __grid_constant__ CamSet cs,
                                                         const float2 *__restrict__ means2d,
                                                         const float *__restrict__ depths,
                                                         const int *__restrict__ radii, uint32_t *__restrict__ keys,
                                                         int *__restrict__ vals, int2 *__restrict__ rect,
                                                         int *__restrict__ misc) {
    // the sort's counters and digit totals start at zero (spread over the grid)
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kMiscInts; i += gridDim.x * blockDim.x) misc[i] = 0;
    // four consecutive pairs per thread: 16-byte loads of radii, depths and means, 16-byte stores
    const int i0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (i0 >= CN) return;
    const int ts = __ffs(cs.tile) - 1;  // tile edges are powers of two
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
        int2 rc[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            bool ok = rr[u] > 0;
            rc[u] = make_int2(0, 0);
            if (ok) {
                const CamDev &cam = cs.cam[(i0 + u) / N];
                int x0, x1, y0, y1;
                ok = pixel_box(mm[u].x, mm[u].y, rr[u], cam.W, cam.H, x0, x1, y0, y1);
                if (ok) rc[u] = tile_rect(cam, ts, x0, x1, y0, y1);
            }
            k[u] = ok ? __float_as_uint(dd[u]) : kInvisible;
        }
        *reinterpret_cast<uint4 *>(keys + i0) = make_uint4(k[0], k[1], k[2], k[3]);
        *reinterpret_cast<int4 *>(vals + i0) = make_int4(i0, i0 + 1, i0 + 2, i0 + 3);
        // rect is 256-byte aligned (a workspace region) and i0 a multiple of 4: 16-byte stores
        *reinterpret_cast<int4 *>(rect + i0) = make_int4(rc[0].x, rc[0].y, rc[1].x, rc[1].y);
        *reinterpret_cast<int4 *>(rect + i0 + 2) = make_int4(rc[2].x, rc[2].y, rc[3].x, rc[3].y);
        return;
    }
    for (int i = i0; i < min(CN, i0 + 4); ++i) {  // the ragged end, or unaligned inputs
        const int r = radii[i];
        bool ok = r > 0;
        int2 rc = make_int2(0, 0);
        if (ok) {
            const CamDev &cam = cs.cam[i / N];
            const float2 m = means2d[i];
            int x0, x1, y0, y1;
            ok = pixel_box(m.x, m.y, r, cam.W, cam.H, x0, x1, y0, y1);
            if (ok) rc = tile_rect(cam, ts, x0, x1, y0, y1);
        }
        keys[i] = ok ? __float_as_uint(depths[i]) : kInvisible;
        vals[i] = i;
        rect[i] = rc;
    }
}

// ---------------------------------------------------------------------------
// item sources of a pass: an array of (key, value), or the slots of the pair table
// ---------------------------------------------------------------------------

// A source hands out its items in windows of 32 (one per lane).  The loads of a group of G
// windows are issued together (load_group) before any of them is decoded (decode), so each
// warp keeps several windows' memory requests in flight instead of waiting for one at a time.
// Item indices are below 2^31 (C*N < 2^31 and K_capacity <= GS_MAX_INTERSECTIONS).

// Items [w0, w0 + 32) of a (key, value) array; `want_val` skips the value loads.
struct ArraySrc {
    static constexpr int G = 8;
    static constexpr bool kPairRank = false;
    const uint32_t *keys;
    const int *vals;
    struct Raw {
        uint32_t key;
        int val;
    };
    __device__ __forceinline__ void load_group(int w0, int n, int lane, bool want_val, Raw (&r)[G]) const {
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int q = w0 + 32 * g + lane;
            r[g].key = q < n ? keys[q] : kInvisible;
            r[g].val = (q < n && want_val) ? vals[q] : 0;
        }
    }
    // (every lane is its own pair: the ranking by pairs is not used with this source)
    __device__ __forceinline__ void decode(const Raw &r, int w0, int n, int lane, bool &valid, uint32_t &key,
                                           int &val, int &pair) const {
        valid = w0 + lane < n;
        key = r.key;
        val = r.val;
        pair = lane;
    }
};

// Slots [w0, w0 + 32) of the intersection list in depth order (w0 a multiple of 32).  Pair j
// (in depth order, j < npairs) owns slots [off_j, off_j + count_j) and covers a rectangle of
// tiles; slot k of the pair is the rectangle's tile k in row-major order.  The pair table
// holds one 16-byte record per pair: (off_j, global id of the first tile, rectangle width |
// tiles per camera row << 16, flat index c*N + n).  Per window w: win_start[w] is the pair
// holding slot 32 w, and bit b of win_bits[w] is set when a pair starts at slot 32 w + b
// (b >= 1).  The lane of slot 32 w + l belongs to pair win_start[w] + `pair`, with `pair` the
// number of bits set in 1..l; it loads that pair's record itself.  `pair` numbers the pairs of
// the window in slot order; a pair's slots are distinct tiles, so when the digit is the whole
// tile id, lanes of one pair never share a digit.
struct EmitSrc {
    static constexpr int G = 4;
    static constexpr bool kPairRank = true;
    const int4 *pairs;
    const int *win_start;
    const unsigned *win_bits;
    struct Raw {
        int4 rec;
        unsigned bits;
    };
    __device__ __forceinline__ void load_group(int w0, int n, int lane, bool want_val, Raw (&r)[G]) const {
        (void)want_val;
        int pc[G];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int wg = w0 + 32 * g;
            const bool in = wg < n;
            pc[g] = in ? win_start[wg >> 5] : 0;
            r[g].bits = in ? win_bits[wg >> 5] : 0u;
        }
        const unsigned le = 0xffffffffu >> (31 - lane);
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const bool in = w0 + 32 * g + lane < n;
            r[g].rec = in ? pairs[pc[g] + __popc(r[g].bits & le)] : make_int4(0, 0, 1, 0);
        }
    }
    __device__ __forceinline__ void decode(const Raw &r, int w0, int n, int lane, bool &valid, uint32_t &key,
                                           int &val, int &pair) const {
        pair = __popc(r.bits & (0xffffffffu >> (31 - lane)));
        val = r.rec.w;
        valid = w0 + lane < n;
        const int k = valid ? w0 + lane - r.rec.x : 0;  // slot of the pair: row-major in its rectangle
        const int w = max(r.rec.z & 0xffff, 1), tx = r.rec.z >> 16;
        // k / w from an approximate reciprocal and one branch-free correction step: the
        // quotient is below 4096 (tile rows of a camera) and the float estimate of
        // (k + 0.5) / w, whose fraction is at least 0.5 / w from an integer, is off by less
        // than one, so floor() lands on the quotient or next to it
        int ky = __float2int_rz(((float)k + 0.5f) * rcp_approx((float)w));
        int kx = k - ky * w;
        const int adj = (kx < 0) ? -1 : (kx >= w ? 1 : 0);
        ky += adj;
        kx -= adj * w;
        key = valid ? (uint32_t)(r.rec.y + ky * tx + kx) : kInvisible;
    }
};

// ---------------------------------------------------------------------------
// one stable LSD pass: histogram, scan, rank + place (no CTA waits on another)
// ---------------------------------------------------------------------------

__device__ __forceinline__ int pass_items(const int *n_dev, int n_host) { return n_dev ? *n_dev : n_host; }

// Digit counts of every block of WARPS * SEG items: hist[d * cols + b] (digit-major), and the
// pass's digit totals rowsum[d] by atomic adds (zeroed before the sort).  With `drop`, items
// whose key is 0xFFFFFFFF are left out, and the number of items kept is added to *n_kept
// (zeroed before the sort).
template <class Src, int WARPS, int SEG>
__global__ void __launch_bounds__(32 * WARPS) rank_hist_kernel(const Src src, const int *__restrict__ n_dev,
                                                             int n_host, int shift, int bits, int cols,
                                                             int *__restrict__ hist, int *__restrict__ rowsum,
                                                             int drop, int *__restrict__ n_kept) {
    constexpr int NT = 32 * WARPS;
    __shared__ int s_h[kMaxDigits];
    __shared__ int s_kept;
    const int n = pass_items(n_dev, n_host);
    const int b = blockIdx.x;
    const int t0 = b * (WARPS * SEG);
    if (t0 >= n) return;  // uniform
    const int nd = 1 << bits;
    const unsigned mask = (unsigned)nd - 1u;
    for (int d = threadIdx.x; d < nd; d += NT) s_h[d] = 0;
    if (threadIdx.x == 0) s_kept = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int s0 = t0 + warp * SEG;
    const int s1 = min(s0 + SEG, n);
    int kept = 0;
    for (int w0 = s0; w0 < s1; w0 += 32 * Src::G) {
        typename Src::Raw raw[Src::G];
        src.load_group(w0, s1, lane, false, raw);
#pragma unroll
        for (int g = 0; g < Src::G; ++g) {
            const int wg = w0 + 32 * g;
            if (wg >= s1) break;  // uniform over the warp
            bool valid;
            uint32_t key;
            int val, pair;
            src.decode(raw[g], wg, s1, lane, valid, key, val, pair);
            if (drop && key == kInvisible) valid = false;
            if (valid) {
                atomicAdd(&s_h[(key >> shift) & mask], 1);
                ++kept;
            }
        }
    }
    if (drop) {
        kept = __reduce_add_sync(0xffffffffu, kept);
        if (lane == 0 && kept) atomicAdd(&s_kept, kept);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < nd; d += NT) {
        const int c = s_h[d];
        hist[(size_t)d * cols + b] = c;
        if (c) atomicAdd(&rowsum[d], c);
    }
    if (drop && threadIdx.x == 0 && s_kept) atomicAdd(n_kept, s_kept);
}

// hist[d * cols + b] <- global start of digit d for block b:
// sum_{d' < d} rowsum[d'] + sum_{b' < b} hist[d * cols + b'].  One CTA per digit; rows of up
// to 256 * MAXSEG blocks are loaded into registers (all loads in flight at once).  With
// `ranges` (a single tile pass, where digits are tiles), digit d < T also gets its tile range
// (start, end), or (0, 0) when empty.
template <int MAXSEG>
__global__ void __launch_bounds__(256) rank_scan_kernel(const int *__restrict__ n_dev, int n_host,
                                                        int block_items, int cols, const int *__restrict__ rowsum,
                                                        int *__restrict__ hist, int2 *__restrict__ ranges, int T) {
    __shared__ int s_tmp[8];
    const int n = pass_items(n_dev, n_host);
    const int nb = (int)(((long long)n + block_items - 1) / block_items);
    const int d = blockIdx.x;
    // start of digit d: the digit totals below d (kMaxDigits / 256 = 8 per thread)
    int pre = 0;
#pragma unroll
    for (int k = 0; k < kMaxDigits / 256; ++k) {
        const int e = threadIdx.x * (kMaxDigits / 256) + k;
        pre += e < d ? rowsum[e] : 0;
    }
    int base;
    block_exclusive_scan(pre, base, s_tmp);
    if (ranges && d < T && threadIdx.x == 0) {
        const int c = rowsum[d];
        ranges[d] = c ? make_int2(base, base + c) : make_int2(0, 0);
    }
    int *row = hist + (size_t)d * cols;
    const int seg = (nb + 255) / 256;
    const int b0 = threadIdx.x * seg, b1 = min(nb, b0 + seg);
    if (seg <= MAXSEG) {
        int v[MAXSEG > 0 ? MAXSEG : 1];
#pragma unroll
        for (int k = 0; k < MAXSEG; ++k) v[k] = b0 + k < b1 ? row[b0 + k] : 0;
        int s = 0;
#pragma unroll
        for (int k = 0; k < MAXSEG; ++k) s += v[k];
        int tot;
        int run = base + block_exclusive_scan(s, tot, s_tmp);
#pragma unroll
        for (int k = 0; k < MAXSEG; ++k) {
            if (b0 + k < b1) row[b0 + k] = run;
            run += v[k];
        }
    } else {
        int s = 0;
        for (int bb = b0; bb < b1; ++bb) s += row[bb];
        int tot;
        int run = base + block_exclusive_scan(s, tot, s_tmp);
        for (int bb = b0; bb < b1; ++bb) {
            const int v = row[bb];
            row[bb] = run;
            run += v;
        }
    }
}

// Shared memory of the rank kernel for a block of `block` items and nd digits: the reordered
// block (keys and values), per-warp 16-bit digit counters, the block's digit starts in the
// output and in the block, and (for digits up to kPeerDigits, when not ranking by pairs)
// per-warp peer masks.
__host__ __device__ constexpr size_t rank_smem_bytes(int block, int warps, int nd, bool peers, bool reorder) {
    return (reorder ? (size_t)block * 8 : 0) + (size_t)warps * nd * 2 + (size_t)nd * 8 +
           (peers ? (size_t)warps * kPeerDigits * 4 : 0);
}

// Stable placement of one block.  (i) every warp counts its segment's digits into its own
// 16-bit counters; (ii) the counters become per-warp prefixes and the block's digit totals are
// scanned; (iii) every warp walks its segment in order (loading or generating the items again)
// and ranks 32 items at a time among equal digits -- by the window's pairs (whole tile ids as
// digits), by peer masks (up to kPeerDigits digits) or by match.any -- placing each item in
// shared memory at its position within the block, so the block ends up sorted by digit;
// (iv) the block is written out as one contiguous run per digit.  Without REORDER, (iii) writes
// every item straight to its final position and (iv) is skipped: with many digits (2048 tiles)
// the runs of a block are too short to coalesce, and the buffer would cost occupancy.
template <class Src, int WARPS, int SEG, bool REORDER>
__global__ void __launch_bounds__(32 * WARPS) rank_scatter_kernel(const Src src, const int *__restrict__ n_dev,
                                                                int n_host, int shift, int bits, int cols,
                                                                const int *__restrict__ hist,
                                                                uint32_t *__restrict__ keys_out,
                                                                int *__restrict__ vals_out, int drop,
                                                                int pair_rank, int no_peers) {
    constexpr int NT = 32 * WARPS;
    constexpr int BLOCK = WARPS * SEG;
    static_assert(SEG % (32 * 8) == 0 && WARPS % 8 == 0 && BLOCK <= 65535,
                  "per-warp 16-bit counters, cleared 16 bytes at a time; groups of up to 8 windows");
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_tmp[WARPS];
    __shared__ int s_kept;
    const int n = pass_items(n_dev, n_host);
    const int b = blockIdx.x;
    const int t0 = b * BLOCK;
    if (t0 >= n) return;  // uniform
    const int nd = 1 << bits;
    const unsigned mask = (unsigned)nd - 1u;
    const bool by_pairs = Src::kPairRank && pair_rank;
    const bool by_peers = !by_pairs && !no_peers && nd <= kPeerDigits;
    constexpr int RB = REORDER ? BLOCK : 0;
    uint32_t *s_ok = reinterpret_cast<uint32_t *>(smem);                       // [RB] reordered keys
    int *s_ov = reinterpret_cast<int *>(s_ok + RB);                             // [RB] reordered values
    unsigned short *s_c16 = reinterpret_cast<unsigned short *>(s_ov + RB);     // [WARPS][nd]
    unsigned *s_c32 = reinterpret_cast<unsigned *>(s_c16);
    int *s_start = reinterpret_cast<int *>(s_c16 + WARPS * nd);                // [nd] start in the output
    int *s_local = s_start + nd;                                               // [nd] start in the block
    unsigned *s_peer = reinterpret_cast<unsigned *>(s_local + nd);             // [WARPS][kPeerDigits]
    {
        uint4 *z = reinterpret_cast<uint4 *>(s_c16);
        for (int i = threadIdx.x; i < WARPS * nd / 8; i += NT) z[i] = make_uint4(0u, 0u, 0u, 0u);
        for (int d = threadIdx.x; d < nd; d += NT) s_start[d] = hist[(size_t)d * cols + b];
        if (by_peers)
            for (int i = threadIdx.x; i < WARPS * kPeerDigits; i += NT) s_peer[i] = 0u;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int s0 = t0 + warp * SEG;
    const int s1 = min(s0 + SEG, n);
    unsigned short *my = s_c16 + warp * nd;
    // (i) per-warp digit counts
    for (int w0 = s0; w0 < s1; w0 += 32 * Src::G) {
        typename Src::Raw raw[Src::G];
        src.load_group(w0, s1, lane, false, raw);
#pragma unroll
        for (int g = 0; g < Src::G; ++g) {
            const int wg = w0 + 32 * g;
            if (wg >= s1) break;  // uniform over the warp
            bool valid;
            uint32_t key;
            int val, pair;
            src.decode(raw[g], wg, s1, lane, valid, key, val, pair);
            if (drop && key == kInvisible) valid = false;
            if (valid) {
                const int c = warp * nd + (int)((key >> shift) & mask);
                atomicAdd(&s_c32[c >> 1], 1u << ((c & 1) * 16));
            }
        }
    }
    __syncthreads();
    // (ii) counters -> per-warp prefixes (warp w's items of digit d come after those of warps < w);
    // the block's digit totals -> their exclusive scan s_local (each thread a contiguous run of digits)
    {
        const int per = (nd + NT - 1) / NT;
        const int d0 = min(nd, (int)threadIdx.x * per), d1 = min(nd, d0 + per);
        int sum = 0;
        for (int d = d0; d < d1; ++d) {
            int run = 0;
#pragma unroll
            for (int w = 0; w < WARPS; ++w) {
                const int c = s_c16[w * nd + d];
                s_c16[w * nd + d] = (unsigned short)run;
                run += c;
            }
            s_local[d] = run;  // the digit's total for now
            sum += run;
        }
        int tot;
        int pre = block_exclusive_scan<NT>(sum, tot, s_tmp);
        for (int d = d0; d < d1; ++d) {
            const int c = s_local[d];
            s_local[d] = pre;
            pre += c;
        }
        if (threadIdx.x == 0) s_kept = tot;
    }
    __syncthreads();
    // (iii) each warp walks its segment in order and places its items in the block's digit order
    const unsigned lt = lanemask_lt();
    for (int w0 = s0; w0 < s1; w0 += 32 * Src::G) {
        typename Src::Raw raw[Src::G];
        src.load_group(w0, s1, lane, true, raw);
#pragma unroll
        for (int g = 0; g < Src::G; ++g) {
            const int wg = w0 + 32 * g;
            if (wg >= s1) break;  // uniform over the warp
            bool valid;
            uint32_t key;
            int val, pair;
            src.decode(raw[g], wg, s1, lane, valid, key, val, pair);
            if (drop && key == kInvisible) valid = false;
            unsigned d;
            int rank;
            if (by_pairs) {
                // the window's pairs one after the other: lanes of one pair hold distinct tiles
                d = (key >> shift) & mask;
                const int np = __reduce_max_sync(0xffffffffu, valid ? pair : 0) + 1;
                rank = 0;
                for (int p = 0; p < np; ++p) {
                    const int c = my[d];  // (every lane reads its own digit's counter)
                    if (valid && pair == p) {
                        rank = c;
                        my[d] = (unsigned short)(c + 1);
                    }
                    __syncwarp();
                }
            } else if (by_peers) {
                d = (key >> shift) & mask;
                unsigned *pm = s_peer + warp * kPeerDigits + d;
                if (valid) atomicOr(pm, 1u << lane);
                __syncwarp();
                const unsigned peers = valid ? *pm : 0u;
                const int before = valid ? (int)my[d] : 0;
                __syncwarp();
                if (valid && lane == __ffs(peers) - 1) {
                    my[d] = (unsigned short)(before + __popc(peers));
                    *pm = 0u;  // left at zero for the next window
                }
                __syncwarp();
                rank = before + __popc(peers & lt);
            } else {
                d = valid ? ((key >> shift) & mask) : (0x10000u + lane);  // invalid lanes match no one
                const unsigned peers = __match_any_sync(0xffffffffu, d);
                const int before = valid ? (int)my[d] : 0;
                __syncwarp();
                if (valid && lane == __ffs(peers) - 1) my[d] = (unsigned short)(before + __popc(peers));
                __syncwarp();
                rank = before + __popc(peers & lt);
            }
            if (valid) {
                if (REORDER) {
                    const int lp = s_local[d] + rank;
                    if ((unsigned)lp < (unsigned)BLOCK) {  // holds by construction
                        s_ok[lp] = key;
                        s_ov[lp] = val;
                    }
                } else {
                    const int pos = s_start[d] + rank;
                    if ((unsigned)pos < (unsigned)n) {  // holds by construction
                        if (keys_out) keys_out[pos] = key;
                        vals_out[pos] = val;
                    }
                }
            }
        }
    }
    if (!REORDER) return;
    __syncthreads();
    // (iv) the block in digit order: consecutive threads write consecutive slots of each run
    const int kept = s_kept;
    for (int i = threadIdx.x; i < kept; i += NT) {
        const uint32_t key = s_ok[i];
        const int d = (int)((key >> shift) & mask);
        const int pos = s_start[d] + (i - s_local[d]);
        if ((unsigned)pos < (unsigned)n) {  // holds by construction
            if (keys_out) keys_out[pos] = key;
            vals_out[pos] = s_ov[i];
        }
    }
}

// ---------------------------------------------------------------------------
// stage 2: tile counts, offsets and window starts of the visible pairs in depth order
// ---------------------------------------------------------------------------

constexpr int kPairsPerThread = 4;                            // consecutive pairs per thread
constexpr int kPairsPerCta = 256 * kPairsPerThread;           // pairs per CTA of the count/offset kernels

// Tiles touched by each visible pair, in depth order, their sum per CTA, and each pair's tile
// rectangle packed as (global id of its first tile, width | tiles per camera row << 16), from
// the pair-order rectangles of the depth-key kernel.  A thread owns kPairsPerThread consecutive
// pairs: all their indices, then all their rectangles are requested before any is used.  The
// pairs of a warp belong to any of the cameras, so the row length is read from a copy in shared
// memory.  Also zeroes the tile ranges when a later pass fills only the non-empty ones.
__global__ void __launch_bounds__(256) count_tiles_kernel(int CN, int N, int T, int *__restrict__ tile_ranges,
                                                          int nwin, unsigned *__restrict__ win_bits,
                                                          const __grid_constant__ CamSet cs,
                                                          const int *__restrict__ order, const int *__restrict__ nvis,
                                                          const int2 *__restrict__ rect, int *__restrict__ counts,
                                                          int2 *__restrict__ rects, long long *__restrict__ partials) {
    if (tile_ranges)
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 2 * T; i += gridDim.x * blockDim.x)
            tile_ranges[i] = 0;  // empty tiles read (0, 0); the ranges kernel fills the others later
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nwin; i += gridDim.x * blockDim.x)
        win_bits[i] = 0u;  // the offsets kernel ORs in the pair starts
    __shared__ long long s_w[8];
    __shared__ int s_tx[kMaxCams];  // tiles per row of each camera
    for (int c = threadIdx.x; c < cs.C; c += blockDim.x) s_tx[c] = cs.cam[c].tiles_x;
    __syncthreads();
    const int nv = *nvis;
    const int j0 = blockIdx.x * kPairsPerCta + threadIdx.x * kPairsPerThread;
    int id[kPairsPerThread];
    int2 pr[kPairsPerThread];
    if (j0 + kPairsPerThread <= nv) {  // j0 is a multiple of 4 and order 16-byte aligned
        const int4 v = *reinterpret_cast<const int4 *>(order + j0);
        id[0] = v.x, id[1] = v.y, id[2] = v.z, id[3] = v.w;
    } else {
#pragma unroll
        for (int u = 0; u < kPairsPerThread; ++u) id[u] = j0 + u < nv ? order[j0 + u] : -1;
    }
#pragma unroll
    for (int u = 0; u < kPairsPerThread; ++u)
        pr[u] = (unsigned)id[u] < (unsigned)CN ? rect[id[u]] : make_int2(0, 0);
    int cnt[kPairsPerThread];
    int2 rc[kPairsPerThread];
#pragma unroll
    for (int u = 0; u < kPairsPerThread; ++u) {
        // (the pairs in `order` are the visible ones: each has a rectangle of >= 1 tile)
        const int w = pr[u].y & 0xffff, h = pr[u].y >> 16;
        cnt[u] = w * h;
        rc[u] = cnt[u] > 0 ? make_int2(pr[u].x, w | (s_tx[id[u] / N] << 16)) : make_int2(0, 1);
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
                                                            int *__restrict__ misc) {
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
        misc[kMiscNeff] = (int)(tot < capacity ? tot : capacity);
    }
}

// Exclusive slot offsets of every visible pair, written with the pair's tile rectangle and
// flat index as one 16-byte record (offsets clamped to n_eff, below 2^31), and for each window
// of 32 slots the pair holding its first slot (win_start[w] = j when 32 w falls in
// [off_j, off_j + count_j)).
__global__ void __launch_bounds__(256) offsets_kernel(int CN, const int *__restrict__ counts,
                                                      const int2 *__restrict__ rects, const int *__restrict__ order,
                                                      const long long *__restrict__ partials,
                                                      const int *__restrict__ misc, int4 *__restrict__ pairs,
                                                      int *__restrict__ win_start, unsigned *__restrict__ win_bits) {
    __shared__ long long s_w[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int j0 = blockIdx.x * kPairsPerCta + threadIdx.x * kPairsPerThread;
    const int nv = misc[kMiscNvis];
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
    const long long limit = misc[kMiscNeff];
#pragma unroll
    for (int u = 0; u < kPairsPerThread; ++u) {
        const int j = j0 + u;
        if (j >= nv) break;
        const int2 rc = rects[j];
        pairs[j] = make_int4((int)min(off, limit), rc.x, rc.y, order[j]);
        if (cnt[u] > 0 && off < limit) {
            const long long end = min(off + cnt[u], limit);
            for (long long w = (off + 31) >> 5; (w << 5) < end; ++w) win_start[w] = j;
            if (off & 31) atomicOr(&win_bits[off >> 5], 1u << (off & 31));  // starts inside a window
        }
        off += cnt[u];
    }
}

// 64-bit keys (tile << 32 | depth bits) of the sorted list, from the tile ranges and values:
// one warp per tile (only when the caller asks for the keys).
__global__ void __launch_bounds__(256) keys64_kernel(int T, int CN, const int2 *__restrict__ ranges,
                                                     const int *__restrict__ vals, const float *__restrict__ depths,
                                                     unsigned long long *__restrict__ keys64) {
    const int t = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (t >= T) return;
    const int2 r = ranges[t];
    for (int p = r.x + (threadIdx.x & 31); p < r.y; p += 32) {
        const int v = vals[p];
        keys64[p] = ((unsigned long long)t << 32) | ((unsigned)v < (unsigned)CN ? __float_as_uint(depths[v]) : 0u);
    }
}

// Tile boundaries of a list sorted by materialised tile keys (the passes of more than 2048
// tiles); each thread looks at 4 consecutive entries.
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

static int tile_bits(long long T) {
    int b = 1;
    while ((1ll << b) < T) ++b;
    return b;
}

// One counting pass over whole tile ids up to 2048 tiles; beyond, LSD passes of at most 8 bits
// (peer-mask ranking, blocks reordered in shared memory, like the depth passes).
static int tile_passes(long long T) {
    const int b = tile_bits(T);
    return b <= kMaxDigitBits ? 1 : (b + kDepthDigitBits - 1) / kDepthDigitBits;
}

BinSortLayout binsort_layout(long long CN, long long Kcap, long long T) {
    BinSortLayout L;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o += align256(bytes);
        return at;
    };
    const long long cnb = (CN + kPairsPerCta - 1) / kPairsPerCta;
    // digit-major count matrix: the largest (digits x blocks) of any pass
    const long long cols_d = (CN + kDepthBlock - 1) / kDepthBlock;
    const long long m_depth = cols_d * (1 << kDepthDigitBits);
    const long long m_tile = tile_passes(T) == 1 ? (Kcap + kTileBlock - 1) / kTileBlock * (long long)kMaxDigits
                                                 : (Kcap + kDepthBlock - 1) / kDepthBlock * (1ll << kDepthDigitBits);
    const long long mat = m_depth > m_tile ? m_depth : m_tile;
    L.dk0 = take(CN * 4);
    L.dk1 = take(CN * 4);
    L.dv0 = take(CN * 4);
    L.dv1 = take(CN * 4);
    L.counts = take(CN * 4);
    L.rects = take(CN * 8);
    L.offsets = take(CN * 16);  // one 16-byte record per visible pair
    L.win_start = take(((Kcap + 31) / 32 + 1) * 4);
    L.win_bits = take(((Kcap + 31) / 32 + 1) * 4);
    L.partials = take((size_t)(cnb + 1) * 8);
    L.misc = take((size_t)kMiscInts * 4);
    L.matrix = take((size_t)(mat > 0 ? mat : 1) * 4);
    // (tile, value) arrays of the list exist only when the tile ids need more than one pass
    const bool multi = tile_passes(T) > 1;
    L.tk0 = multi ? take(Kcap * 4) : 0;
    L.tk1 = multi ? take(Kcap * 4) : 0;
    L.tvB = multi ? take(Kcap * 4) : 0;
    L.total = o;
    return L;
}

// One stable LSD pass (histogram, scan, rank + place) over blocks of WARPS * SEG items.
// `skewed`: most items share a few digits (the top bits of positive float depths), where lanes
// OR-ing into one peer mask serialise and match.any ranks faster.
template <class Src, int WARPS, int SEG, bool REORDER>
static cudaError_t rank_pass(const Src &src, const int *n_dev, int n_host, long long max_items, int shift, int bits,
                             int *matrix, int *rowsum, int drop, int *n_kept, uint32_t *kout, int *vout,
                             int2 *ranges, int T, cudaStream_t st, bool skewed = false) {
    constexpr int block = WARPS * SEG;
    const int cols = (int)((max_items + block - 1) / block);
    if (cols <= 0) return cudaSuccess;
    rank_hist_kernel<Src, WARPS, SEG><<<cols, 32 * WARPS, 0, st>>>(src, n_dev, n_host, shift, bits, cols, matrix,
                                                                  rowsum, drop, n_kept);
    note_launch();
    const int nd = 1 << bits;
    if (cols <= 256 * 4)
        rank_scan_kernel<4><<<nd, 256, 0, st>>>(n_dev, n_host, block, cols, rowsum, matrix, ranges, T);
    else if (cols <= 256 * 32)
        rank_scan_kernel<32><<<nd, 256, 0, st>>>(n_dev, n_host, block, cols, rowsum, matrix, ranges, T);
    else
        rank_scan_kernel<0><<<nd, 256, 0, st>>>(n_dev, n_host, block, cols, rowsum, matrix, ranges, T);
    note_launch();
    // ranking by pairs needs every digit to be a whole tile id: one pass over all tile bits
    const int pair_rank = (shift == 0 && ranges != nullptr) ? 1 : 0;
    const bool peers = !(Src::kPairRank && pair_rank) && !skewed && nd <= kPeerDigits;
    const int smem = (int)rank_smem_bytes(block, WARPS, nd, peers, REORDER);
    const int smem_max = (int)rank_smem_bytes(block, WARPS, kMaxDigits, true, REORDER);
    cudaError_t e = ensure_smem((const void *)rank_scatter_kernel<Src, WARPS, SEG, REORDER>, smem_max);
    if (e != cudaSuccess) return e;
    rank_scatter_kernel<Src, WARPS, SEG, REORDER><<<cols, 32 * WARPS, smem, st>>>(
        src, n_dev, n_host, shift, bits, cols, matrix, kout, vout, drop, pair_rank, skewed ? 1 : 0);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_binsort(const CamSet &cs, int N, const float *means2d, const float *depths, const int *radii,
                           long long Kcap, unsigned long long *keys64, int *values, int *tile_ranges,
                           long long *K_out, void *ws, cudaStream_t st) {
    const int C = cs.C;
    const long long CN = (long long)C * N;
    const int T = cs.total_tiles;
    BinSortLayout L = binsort_layout(CN, Kcap, T);
    char *w = (char *)ws;
    uint32_t *dk0 = (uint32_t *)(w + L.dk0), *dk1 = (uint32_t *)(w + L.dk1);
    int *dv0 = (int *)(w + L.dv0), *dv1 = (int *)(w + L.dv1);
    int *counts = (int *)(w + L.counts);
    int2 *rects = (int2 *)(w + L.rects);
    int4 *pairs = (int4 *)(w + L.offsets);
    int *win_start = (int *)(w + L.win_start);
    unsigned *win_bits = (unsigned *)(w + L.win_bits);
    const int nwin = (int)((Kcap + 31) / 32 + 1);
    long long *partials = (long long *)(w + L.partials);
    int *misc = (int *)(w + L.misc);
    int *n_eff = misc + kMiscNeff;
    int *n_vis = misc + kMiscNvis;
    int *matrix = (int *)(w + L.matrix);
    int *rowsum = misc + kMiscRowsum;

    const int cn = (int)CN;
    if (cn == 0) {
        empty_result_kernel<<<1, 32, 0, st>>>(K_out, misc);
        note_launch();
        zero_ints_kernel<<<(2 * T + 255) / 256, 256, 0, st>>>(2 * T, tile_ranges);
        note_launch();
        return cudaGetLastError();
    }
    // stage 1: depth order of the visible (camera, Gaussian) pairs
    const int eb = (cn + 1023) / 1024;  // four pairs per thread
    // (the pair-order rectangles live in the 16-byte pair-record region until the offsets kernel
    // overwrites it; the count kernel reads them before)
    int2 *prect = (int2 *)(w + L.offsets);
    depth_keys_kernel<<<eb, 256, 0, st>>>(cn, N, cs, (const float2 *)means2d, depths, radii, dk0, dv0, prect, misc);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    {
        // passes of kDepthDigitBits bits (the last takes the rest); the first drops the pairs
        // without tiles
        uint32_t *kin = dk0, *kout = dk1;
        int *vin = dv0, *vout = dv1;
        int shift = 0;
        for (int pass = 0; pass < kDepthPasses; ++pass) {
            const ArraySrc src{kin, vin};
            const int width = min(kDepthDigitBits, 32 - shift);
            // (the last pass writes only the values: the sorted keys are not read again)
            e = rank_pass<ArraySrc, kDepthWarps, kDepthSeg, true>(
                src, pass ? n_vis : nullptr, cn, cn, shift, width, matrix, rowsum + pass * kMaxDigits, pass == 0,
                n_vis, pass + 1 < kDepthPasses ? kout : nullptr, vout, nullptr, 0, st, pass + 1 == kDepthPasses);
            if (e != cudaSuccess) return e;
            shift += width;
            uint32_t *tk = kin;
            kin = kout;
            kout = tk;
            int *tv = vin;
            vin = vout;
            vout = tv;
        }
    }
    const int *order = (kDepthPasses % 2) ? dv1 : dv0;  // where the last depth pass wrote
    // stage 2: tile counts, offsets, then the tile passes over the slots in depth order
    const int passes = tile_passes(T);
    const int bits = tile_bits(T);
    const int pb = (cn + kPairsPerCta - 1) / kPairsPerCta;  // CTAs of the count and offset kernels
    count_tiles_kernel<<<pb, 256, 0, st>>>(cn, N, T, passes > 1 ? tile_ranges : nullptr, nwin, win_bits, cs, order,
                                           n_vis, prect, counts, rects, partials);
    note_launch();
    partial_scan_kernel<<<1, 1024, 0, st>>>(pb, partials, Kcap, K_out, misc);
    note_launch();
    offsets_kernel<<<pb, 256, 0, st>>>(cn, counts, rects, order, partials, misc, pairs, win_start, win_bits);
    note_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (Kcap <= 0) {  // nothing can be written: ranges stay zero
        if (passes == 1) {
            zero_ints_kernel<<<(2 * T + 255) / 256, 256, 0, st>>>(2 * T, tile_ranges);
            note_launch();
        }
        return cudaGetLastError();
    }
    const EmitSrc emit{pairs, win_start, win_bits};

    int2 *ranges = (int2 *)tile_ranges;
    if (passes == 1) {
        // one counting pass: slots -> values, tile ranges from the digit totals
        e = rank_pass<EmitSrc, kTileWarps, kTileSeg, false>(emit, n_eff, 0, Kcap, 0, bits, matrix,
                                                            rowsum + kDepthPasses * kMaxDigits, 0, nullptr, nullptr,
                                                            values, ranges, T, st);
        if (e != cudaSuccess) return e;
        if (keys64) {
            keys64_kernel<<<(T + 7) / 8, 256, 0, st>>>(T, cn, ranges, values, depths, keys64);
            note_launch();
        }
        return cudaGetLastError();
    }
    // several passes over materialised (tile, value) arrays; the last one writes `values`
    uint32_t *tk0 = (uint32_t *)(w + L.tk0), *tk1 = (uint32_t *)(w + L.tk1);
    int *tvB = (int *)(w + L.tvB);
    const int dw = (bits + passes - 1) / passes;  // <= 8 bits
    uint32_t *kout = tk0;
    int *vout = ((passes - 1) % 2 == 0) ? values : tvB;
    e = rank_pass<EmitSrc, kDepthWarps, kDepthSeg, true>(emit, n_eff, 0, Kcap, 0, dw, matrix,
                                                         rowsum + kDepthPasses * kMaxDigits, 0, nullptr, kout, vout,
                                                         nullptr, 0, st);
    if (e != cudaSuccess) return e;
    for (int pass = 1; pass < passes; ++pass) {
        const int width = min(dw, bits - pass * dw);
        const ArraySrc src{kout, vout};
        uint32_t *k2 = (kout == tk0) ? tk1 : tk0;
        int *v2 = (vout == values) ? tvB : values;
        e = rank_pass<ArraySrc, kDepthWarps, kDepthSeg, true>(src, n_eff, 0, Kcap, pass * dw, width, matrix,
                                                              rowsum + (kDepthPasses + pass) * kMaxDigits, 0, nullptr,
                                                              k2, v2, nullptr, 0, st);
        if (e != cudaSuccess) return e;
        kout = k2;
        vout = v2;
    }
    // (kout, vout) hold the sorted list; vout == values
    const long long rq = (Kcap + 3) / 4;
    ranges_kernel<<<(unsigned)((rq + 255) / 256 > 0 ? (rq + 255) / 256 : 1), 256, 0, st>>>(
        n_eff, T, cn, kout, vout, depths, ranges, keys64);
    note_launch();
    return cudaGetLastError();
}

}  // namespace gs
