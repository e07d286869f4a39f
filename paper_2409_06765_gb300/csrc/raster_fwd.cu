// Front-to-back alpha compositing (App. C.2), one CTA per tile.
//
// The CTA walks its tile's depth-sorted list in batches: each batch of Gaussians is
// gathered once (coalesced 4/8/16-byte loads by index) into shared memory, then every
// pixel of the tile reads the batch as broadcasts.  Pixels stop at the transmittance
// floor; a CTA stops as soon as all of its pixels have (__syncthreads_count), and a warp
// whose pixels have all stopped skips the compositing loop of a batch.  For 32x32
// tiles a thread owns four pixels of one column.
#include "gs_internal.cuh"

namespace gs {

struct BgConst {
    float v[GS_MAX_CHANNELS];
};

template <int TILE>
struct TileShape {
    static constexpr int kPixels = TILE * TILE;
    static constexpr int kThreads = kPixels >= 256 ? 256 : kPixels;
    static constexpr int kPPT = kPixels / kThreads;
};

// Shared-memory staging record of one Gaussian.
struct StagedGeom {
    float4 g;   // mx, my, conic a, conic b
    float2 h;   // conic c, opacity
};

template <int TILE, int CHC, bool COUNT>
__global__ void __launch_bounds__(TileShape<TILE>::kThreads) raster_fwd_kernel(
    const __grid_constant__ CamSet cs, RasterConsts rc, int ch, int batch, const int2 *__restrict__ ranges,
    const int *__restrict__ values, const int *__restrict__ radii, const float2 *__restrict__ means2d,
    const float *__restrict__ conics, const float *__restrict__ opac, const float *__restrict__ colors,
    const __grid_constant__ BgConst bg, float *__restrict__ image, float *__restrict__ final_T,
    int *__restrict__ last_contrib, unsigned long long *__restrict__ blend_count) {
    using S = TileShape<TILE>;
    constexpr int PPT = S::kPPT, THREADS = S::kThreads;
    constexpr int C4 = (CHC + 3) / 4;
    extern __shared__ __align__(16) unsigned char smem[];
    float4 *s_g = reinterpret_cast<float4 *>(smem);
    float2 *s_h = reinterpret_cast<float2 *>(s_g + batch);
    int4 *s_b = reinterpret_cast<int4 *>(s_h + batch);
    float4 *s_c = reinterpret_cast<float4 *>(s_b + batch);

    const int gt = blockIdx.x;
    const int c = camera_of_tile(cs, gt);
    const CamDev &cam = cs.cam[c];
    const int local = gt - cam.tile_offset;
    const int tx = local % cam.tiles_x, ty = local / cam.tiles_x;

    int px[PPT], py[PPT], last[PPT];
    bool done[PPT];
    float T[PPT], acc[PPT][CHC];
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        int lin = threadIdx.x + k * THREADS;
        px[k] = tx * TILE + lin % TILE;
        py[k] = ty * TILE + lin / TILE;
        done[k] = !(px[k] < cam.W && py[k] < cam.H);
        T[k] = 1.f;
        last[k] = 0;
#pragma unroll
        for (int q = 0; q < CHC; ++q) acc[k][q] = 0.f;
    }
    const int2 rg = ranges[gt];
    const int cn_total = cs.C * cs.N;
    unsigned long long blends = 0;
    const float amax = rc.alpha_max, amin = rc.alpha_min, tmin = rc.T_min;

    for (int start = rg.x; start < rg.y; start += batch) {
        bool tdone = true;
#pragma unroll
        for (int k = 0; k < PPT; ++k) tdone &= done[k];
        if (__syncthreads_count(tdone) == THREADS) break;
        const int cnt = min(batch, rg.y - start);
        for (int s = threadIdx.x; s < cnt; s += THREADS) {
            int id = values[start + s];
            if ((unsigned)id >= (unsigned)cn_total) id = 0;  // holds by construction (ids come from the sort)
            float2 m = means2d[id];
            int r = radii[id];
            int x0, x1, y0, y1;
            support_span(m.x, r, x0, x1);
            support_span(m.y, r, y0, y1);
            s_g[s] = make_float4(m.x, m.y, conics[3 * id], conics[3 * id + 1]);
            s_h[s] = make_float2(conics[3 * id + 2], opac[id]);
            s_b[s] = make_int4(x0, x1 - x0, y0, y1 - y0);
            const float *col = colors + (size_t)id * ch;
#pragma unroll
            for (int q = 0; q < C4; ++q) {
                float4 v;
                v.x = (4 * q + 0 < ch) ? col[4 * q + 0] : 0.f;
                v.y = (4 * q + 1 < ch) ? col[4 * q + 1] : 0.f;
                v.z = (4 * q + 2 < ch) ? col[4 * q + 2] : 0.f;
                v.w = (4 * q + 3 < ch) ? col[4 * q + 3] : 0.f;
                s_c[s * C4 + q] = v;
            }
        }
        __syncthreads();
        if (__all_sync(0xffffffffu, tdone)) continue;
        for (int j = 0; j < cnt; ++j) {
            const int4 b = s_b[j];
            const float4 g = s_g[j];
            const float2 h = s_h[j];
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                if (done[k]) continue;
                if ((unsigned)(px[k] - b.x) > (unsigned)b.y || (unsigned)(py[k] - b.z) > (unsigned)b.w) continue;
                if (COUNT) ++blends;
                const float dx = ((float)px[k] + 0.5f) - g.x;
                const float dy = ((float)py[k] + 0.5f) - g.y;
                const float sigma = mahalanobis_half(dx, dy, g.z, g.w, h.x);
                if (sigma < 0.f) continue;
                const float e = gauss_weight(sigma);
                const float alpha = fminf(amax, __fmul_rn(h.y, e));
                if (alpha < amin) continue;
                const float Tn = __fmul_rn(T[k], __fsub_rn(1.f, alpha));
                if (Tn < tmin) {
                    done[k] = true;
                    continue;
                }
                const float w = __fmul_rn(alpha, T[k]);
#pragma unroll
                for (int q = 0; q < C4; ++q) {
                    const float4 v = s_c[j * C4 + q];
                    if (4 * q + 0 < CHC) acc[k][4 * q + 0] += v.x * w;
                    if (4 * q + 1 < CHC) acc[k][4 * q + 1] += v.y * w;
                    if (4 * q + 2 < CHC) acc[k][4 * q + 2] += v.z * w;
                    if (4 * q + 3 < CHC) acc[k][4 * q + 3] += v.w * w;
                }
                T[k] = Tn;
                last[k] = start + j - rg.x + 1;
            }
        }
    }
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        if (!(px[k] < cam.W && py[k] < cam.H)) continue;
        const size_t pix = (size_t)cam.pix_offset + (size_t)py[k] * cam.W + px[k];
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
        if ((threadIdx.x & 31) == 0 && blends) atomicAdd(blend_count, blends);
    }
}

template <int TILE, int CHC, bool COUNT>
static cudaError_t launch_fwd_t(const CamSet &cs, const RasterConsts &rc, int ch, int batch, const int *ranges,
                                const int *values, const int *radii, const float *means2d, const float *conics,
                                const float *opac, const float *colors, const BgConst &bg, float *image,
                                float *final_T, int *last_contrib, unsigned long long *blend_count,
                                cudaStream_t st) {
    constexpr int C4 = (CHC + 3) / 4;
    size_t smem = (size_t)batch * (sizeof(float4) + sizeof(float2) + sizeof(int4) + C4 * sizeof(float4));
    auto kern = raster_fwd_kernel<TILE, CHC, COUNT>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    if (cs.total_tiles == 0) return cudaSuccess;
    kern<<<cs.total_tiles, TileShape<TILE>::kThreads, smem, st>>>(
        cs, rc, ch, batch, (const int2 *)ranges, values, radii, (const float2 *)means2d, conics, opac, colors,
        bg, image, final_T, last_contrib, blend_count);
    note_launch();
    return cudaGetLastError();
}

template <int TILE, bool COUNT>
static cudaError_t dispatch_ch(int chc, const CamSet &cs, const RasterConsts &rc, int ch, int batch,
                               const int *ranges, const int *values, const int *radii, const float *means2d,
                               const float *conics, const float *opac, const float *colors, const BgConst &bg,
                               float *image, float *final_T, int *last_contrib, unsigned long long *cnt,
                               cudaStream_t st) {
#define GS_FWD_CASE(K)                                                                                              \
    case K:                                                                                                         \
        return launch_fwd_t<TILE, K, COUNT>(cs, rc, ch, batch, ranges, values, radii, means2d, conics, opac, colors, \
                                            bg, image, final_T, last_contrib, cnt, st);
    if constexpr (TILE == 16 && !COUNT) {
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

// Smallest compiled channel capacity >= ch for a tile size; 0 when none.  The
// blend-counting variant exists for 3 and 4 channels only.
int raster_channel_capacity(int tile, int ch, bool count) {
    if (tile == 16 && !count) {
        const int caps[] = {1, 2, 3, 4, 8, 16, 32, 64};
        for (int c : caps)
            if (ch <= c) return c;
        return 0;
    }
    if (ch <= 3) return 3;
    if (ch <= 4) return 4;
    return 0;
}

cudaError_t launch_raster_fwd(const CamSet &cs, const RasterConsts &rc, int ch, int batch, const int *ranges,
                              const int *values, const int *radii, const float *means2d, const float *conics,
                              const float *opac, const float *colors, const float *bg_host, float *image,
                              float *final_T, int *last_contrib, unsigned long long *blend_count, cudaStream_t st) {
    BgConst bg;
    for (int q = 0; q < GS_MAX_CHANNELS; ++q) bg.v[q] = (bg_host && q < ch) ? bg_host[q] : 0.f;
    const bool count = blend_count != nullptr;
    int chc = raster_channel_capacity(cs.tile, ch, count);
#define GS_FWD_TILE(T)                                                                                             \
    if (cs.tile == T)                                                                                              \
        return count ? dispatch_ch<T, true>(chc, cs, rc, ch, batch, ranges, values, radii, means2d, conics, opac,   \
                                            colors, bg, image, final_T, last_contrib, blend_count, st)              \
                     : dispatch_ch<T, false>(chc, cs, rc, ch, batch, ranges, values, radii, means2d, conics, opac,  \
                                             colors, bg, image, final_T, last_contrib, nullptr, st);
    GS_FWD_TILE(8)
    GS_FWD_TILE(16)
    GS_FWD_TILE(32)
#undef GS_FWD_TILE
    return cudaErrorNotSupported;
}

}  // namespace gs
