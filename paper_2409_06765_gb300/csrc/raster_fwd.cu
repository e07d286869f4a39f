// Front-to-back alpha compositing (App. C.2), one CTA per tile.
//
// The CTA walks its tile's depth-sorted list in batches: each batch of Gaussians is
// gathered once (by index, from the projected splat arrays) into shared memory, then
// every pixel of the tile reads the batch as broadcasts.  A thread owns PPT pixels of one
// column.  Each warp first tests 32 staged entries at a time against its band of pixels
// (box overlap, and the minimum of sigma over the band against ln(opacity / alpha_min):
// entries failing it cannot reach alpha_min there) and walks only the hits, in list
// order.  Pixels stop at the transmittance floor; a warp whose pixels have all stopped
// leaves the batch, and the CTA stops when all of its pixels have (__syncthreads_count).
#include "gs_internal.cuh"


namespace gs {

struct BgConst {
    float v[GS_MAX_CHANNELS];
};

template <int TILE, int PPT, int CHC, bool COUNT>
__global__ void __launch_bounds__(RasterShape<TILE, PPT>::kThreads) raster_fwd_kernel(
    const __grid_constant__ CamSet cs, RasterConsts rc, int ch, int batch, const int2 *__restrict__ ranges,
    const int *__restrict__ values, const int *__restrict__ radii, const float2 *__restrict__ means2d,
    const float *__restrict__ conics, const float *__restrict__ opac, const float *__restrict__ colors,
    const __grid_constant__ BgConst bg, float *__restrict__ image, float *__restrict__ final_T,
    int *__restrict__ last_contrib, unsigned long long *__restrict__ blend_count) {
    using S = RasterShape<TILE, PPT>;
    constexpr int THREADS = S::kThreads;
    constexpr int C4 = (CHC + 3) / 4;
    extern __shared__ __align__(16) unsigned char smem[];

    __shared__ int s_next;
    for (int round = 0;; ++round) {
    int gt;
    if (rc.work) {  // persistent: tiles in tile_order, heaviest first, until none is left
        const int i = next_work_item(rc.work, &s_next);
        if (i >= cs.total_tiles) break;
        gt = rc.tile_order[i];
        if ((unsigned)gt >= (unsigned)cs.total_tiles) continue;  // uniform over the CTA
    } else {
        if (round > 0) break;
        gt = tile_of_block(rc, cs.total_tiles);
        if (gt < 0) break;  // uniform over the CTA
    }
    const int c = camera_of_tile(cs, gt);
    const CamDev &cam = cs.cam[c];
    const int local = gt - cam.tile_offset;
    const int tx0 = (local % cam.tiles_x) * TILE, ty0 = (local / cam.tiles_x) * TILE;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // this warp's band of pixels and this thread's column / first row in it
    int wx0, wx1, wy0, wy1, px, py0;
    warp_band<S>(tx0, ty0, warp, lane, wx0, wx1, wy0, wy1, px, py0);
    const float fx = (float)px + 0.5f;
    int last[PPT];
    bool done[PPT];
    float T[PPT], acc[PPT][CHC];
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        done[k] = !(px < cam.W && py0 + k < cam.H);
        T[k] = 1.f;
        last[k] = 0;
#pragma unroll
        for (int q = 0; q < CHC; ++q) acc[k][q] = 0.f;
    }
    const int2 rg = ranges[gt];
    const int cn_total = cs.C * cs.N;
    unsigned long long blends = 0;
    const float amax = rc.alpha_max, amin = rc.alpha_min, tmin = rc.T_min;

    const int n_shared = rc.colors_shared ? cs.N : 0;
    const StagedBatch sb = staged_batch<C4>(smem, batch);
    const float4 *s_g = sb.g, *s_h = sb.h, *s_c = sb.c;
    const int4 *s_b = sb.b;

    for (int start = rg.x; start < rg.y; start += batch) {
        bool tdone = true;
#pragma unroll
        for (int k = 0; k < PPT; ++k) tdone &= done[k];
        if (__syncthreads_count(tdone) == THREADS) break;
        const int cnt = min(batch, rg.y - start);
        stage_batch<THREADS, C4>(sb, values, start, 1, cnt, cn_total, n_shared, ch, means2d, conics, opac, radii,
                                 colors, amin);
        __syncthreads();
        for (int base = 0; base < cnt; base += 32) {
            bool wdone = true;
#pragma unroll
            for (int k = 0; k < PPT; ++k) wdone &= done[k];
            if (__all_sync(0xffffffffu, wdone)) break;
            // entries of this group of 32 that can blend somewhere in the warp's band
            const int jl = base + lane;
            bool hit = false;
            // (the blend-counting variant keeps every pair of the box, the definition it counts)
            if (jl < cnt)
                hit = COUNT ? box_hits(s_b[jl], wx0, wx1, wy0, wy1)
                            : may_blend(s_g[jl], s_h[jl], s_b[jl], wx0, wx1, wy0, wy1);
            unsigned m = __ballot_sync(0xffffffffu, hit);
            while (m) {
                const int j = base + __ffs(m) - 1;
                m &= m - 1;
                const int4 b = s_b[j];
                const float4 g = s_g[j];
                const float2 h = make_float2(s_h[j].x, s_h[j].y);
                const bool inx = (unsigned)(px - b.x) <= (unsigned)b.y;
                const float dx = fx - g.x;
                const GaussRow gr = gauss_row(dx, g.z, g.w, h.x);
                {
                    // the PPT pixels are independent chains: evaluate all of them without
                    // branches (the decisions become selects) so their latencies overlap
                    const int rel = start + j - rg.x + 1;
#pragma unroll
                    for (int k = 0; k < PPT; ++k) {
                        const bool act = !done[k] && inx && (unsigned)(py0 + k - b.z) <= (unsigned)b.w;
                        if (COUNT) blends += act ? 1 : 0;
                        const float dy = ((float)(py0 + k) + 0.5f) - g.y;
                        const float pe = gauss_exponent(gr, dy);  // -log2(e) sigma
                        const float e = ex2_approx(pe);
                        const bool neg = pe > 0.f;  // sigma < 0
                        const float alpha = fminf(amax, __fmul_rn(h.y, e));
                        const bool blend = act && !neg && !(alpha < amin);
                        const float Tn = __fmaf_rn(-T[k], alpha, T[k]);  // T (1 - alpha)
                        const bool stop = blend && Tn < tmin;
                        const bool take = blend && !stop;
                        const float w = take ? __fmul_rn(alpha, T[k]) : 0.f;
#pragma unroll
                        for (int q = 0; q < C4; ++q) {
                            const float4 v = s_c[j * C4 + q];
                            if (4 * q + 0 < CHC) acc[k][4 * q + 0] += v.x * w;
                            if (4 * q + 1 < CHC) acc[k][4 * q + 1] += v.y * w;
                            if (4 * q + 2 < CHC) acc[k][4 * q + 2] += v.z * w;
                            if (4 * q + 3 < CHC) acc[k][4 * q + 3] += v.w * w;
                        }
                        T[k] = take ? Tn : T[k];
                        last[k] = take ? rel : last[k];
                        done[k] = done[k] || stop;
                    }
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const int py = py0 + k;
        if (!(px < cam.W && py < cam.H)) continue;
        const size_t pix = (size_t)cam.pix_offset + (size_t)py * cam.W + px;
        float *out = image + pix * ch;
#pragma unroll
        for (int q = 0; q < CHC; ++q)
            if (q < ch) out[q] = acc[k][q] + T[k] * bg.v[q];
        final_T[pix] = T[k];
        last_contrib[pix] = last[k];
    }
    if (COUNT) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) blends += __shfl_down_sync(0xffffffffu, blends, o);
        if (lane == 0 && blends) atomicAdd(blend_count, blends);
    }
    __syncthreads();  // the next tile reuses the shared memory
    }
    if (rc.work) finish_work(rc.work);
}

// Shared memory of one compositing batch: geometry, conic/opacity/cut, box, colour (padded to float4).
size_t raster_fwd_smem(int batch, int chc) {
    return staged_batch_bytes(batch, (chc + 3) / 4);
}

template <int TILE, int PPT, int CHC, bool COUNT>
static cudaError_t launch_fwd_t(const CamSet &cs, const RasterConsts &rc, int ch, int batch, const int *ranges,
                                const int *values, const int *radii, const float *means2d, const float *conics,
                                const float *opac, const float *colors, const BgConst &bg, float *image,
                                float *final_T, int *last_contrib, unsigned long long *blend_count,
                                cudaStream_t st) {
    const size_t smem = raster_fwd_smem(batch, CHC);
    auto kern = raster_fwd_kernel<TILE, PPT, CHC, COUNT>;
    if (smem + 1024 > 48 * 1024) {  // dynamic + static shared memory above the default limit
        cudaError_t e = ensure_smem((const void *)kern, (int)smem);
        if (e != cudaSuccess) return e;
    }
    if (cs.total_tiles == 0) return cudaSuccess;
    const int grid = rc.work ? persistent_grid((const void *)kern, RasterShape<TILE, PPT>::kThreads, (int)smem,
                                               cs.total_tiles)
                             : cs.total_tiles;
    kern<<<grid, RasterShape<TILE, PPT>::kThreads, smem, st>>>(
        cs, rc, ch, batch, (const int2 *)ranges, values, radii, (const float2 *)means2d, conics, opac, colors, bg,
        image, final_T, last_contrib, blend_count);
    note_launch();
    return cudaGetLastError();
}

template <int TILE, int PPT, bool COUNT>
static cudaError_t dispatch_ch(int chc, const CamSet &cs, const RasterConsts &rc, int ch, int batch,
                               const int *ranges, const int *values, const int *radii, const float *means2d,
                               const float *conics, const float *opac, const float *colors, const BgConst &bg,
                               float *image, float *final_T, int *last_contrib, unsigned long long *cnt,
                               cudaStream_t st) {
#define GS_FWD_CASE(K)                                                                                              \
    case K:                                                                                                         \
        return launch_fwd_t<TILE, PPT, K, COUNT>(cs, rc, ch, batch, ranges, values, radii, means2d, conics, opac, colors, \
                                            bg, image, final_T, last_contrib, cnt, st);
    if constexpr (TILE == 16 && PPT == 1 && !COUNT) {
        switch (chc) {
            GS_FWD_CASE(1)
            GS_FWD_CASE(2)
            GS_FWD_CASE(3)
            GS_FWD_CASE(4)
            GS_FWD_CASE(8)
            GS_FWD_CASE(16)
            GS_FWD_CASE(32)
            GS_FWD_CASE(64)
        }
    } else {
        switch (chc) {
            GS_FWD_CASE(3)
            GS_FWD_CASE(4)
        }
    }
#undef GS_FWD_CASE
    return cudaErrorNotSupported;
}

// Pixels per thread compiled for a tile size (0 selects the default), or 0 when none.
int raster_pixels_per_thread(int tile, int ppt) {
    if (tile == 8) return (ppt == 0 || ppt == 1) ? 1 : 0;
    if (tile == 16) return ppt == 0 ? 1 : ((ppt == 1 || ppt == 2) ? ppt : 0);
    if (tile == 32) return ppt == 0 ? 4 : ((ppt == 2 || ppt == 4) ? ppt : 0);
    return 0;
}

// Smallest compiled channel capacity >= ch for a tile size and pixels per thread; 0 when
// none.  1..64 channels exist for 16x16 tiles with one pixel per thread; every other
// shape, the blend-counting and the absgrad variants exist for 3 and 4 channels.
int raster_channel_capacity(int tile, int ppt, int ch, bool restricted) {
    if (tile == 16 && ppt == 1 && !restricted) {
        const int caps[] = {1, 2, 3, 4, 8, 16, 32, 64};
        for (int c : caps)
            if (ch <= c) return c;
        return 0;
    }
    if (ch <= 3) return 3;
    if (ch <= 4) return 4;
    return 0;
}

cudaError_t launch_raster_fwd(const CamSet &cs, const RasterConsts &rc, int ch, int batch, int ppt, const int *ranges,
                              const int *values, const int *radii, const float *means2d, const float *conics,
                              const float *opac, const float *colors, const float *bg_host, float *image,
                              float *final_T, int *last_contrib, unsigned long long *blend_count, cudaStream_t st) {
    BgConst bg;
    for (int q = 0; q < GS_MAX_CHANNELS; ++q) bg.v[q] = (bg_host && q < ch) ? bg_host[q] : 0.f;
    const bool count = blend_count != nullptr;
    int chc = raster_channel_capacity(cs.tile, ppt, ch, count);
#define GS_FWD_TILE(T, P)                                                                                          \
    if (cs.tile == T && ppt == P)                                                                                  \
        return count ? dispatch_ch<T, P, true>(chc, cs, rc, ch, batch, ranges, values, radii, means2d, conics,      \
                                               opac, colors, bg, image, final_T, last_contrib, blend_count, st)     \
                     : dispatch_ch<T, P, false>(chc, cs, rc, ch, batch, ranges, values, radii, means2d, conics,     \
                                                opac, colors, bg, image, final_T, last_contrib, nullptr, st);
    GS_FWD_TILE(8, 1)
    GS_FWD_TILE(16, 1)
    GS_FWD_TILE(16, 2)
    GS_FWD_TILE(32, 2)
    GS_FWD_TILE(32, 4)
#undef GS_FWD_TILE
    return cudaErrorNotSupported;
}

}  // namespace gs
