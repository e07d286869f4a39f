// Backward of the compositing sum (App. D.1), one CTA per tile.
//
// Each pixel replays its list back to front from its last contributor: alpha is
// recomputed with the forward's exact arithmetic (so the same pairs are skipped),
// T_n = T_{n+1} / (1 - alpha_n) is recovered from the stored final T, and the suffix
// term sum_c g_c S_c is carried as one scalar per pixel.  Per Gaussian, the pixels of a
// warp are summed with shuffles (skipped when no lane of the warp touched it) and one
// lane adds the sums to global memory (float2 atomics for the mean and absgrad).  Only
// final T and the last-contributor index are stored by the forward, so memory stays
// O(pixels + Gaussians).
#include "gs_internal.cuh"

namespace gs {

struct BgConstB {
    float v[GS_MAX_CHANNELS];
};

template <int TILE>
struct TileShapeB {
    static constexpr int kPixels = TILE * TILE;
    static constexpr int kThreads = kPixels >= 256 ? 256 : kPixels;
    static constexpr int kPPT = kPixels / kThreads;
};

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <int TILE, int CHC, bool ABSG>
__global__ void __launch_bounds__(TileShapeB<TILE>::kThreads) raster_bwd_kernel(
    const __grid_constant__ CamSet cs, RasterConsts rc, int ch, int batch, const int2 *__restrict__ ranges,
    const int *__restrict__ values, const int *__restrict__ radii, const float2 *__restrict__ means2d,
    const float *__restrict__ conics, const float *__restrict__ opac, const float *__restrict__ colors,
    const __grid_constant__ BgConstB bg, const float *__restrict__ final_T, const int *__restrict__ last_contrib,
    const float *__restrict__ d_image, const float *__restrict__ d_alpha, float2 *__restrict__ d_means2d,
    float *__restrict__ d_conics, float *__restrict__ d_opac, float *__restrict__ d_colors,
    float2 *__restrict__ absgrad) {
    using S = TileShapeB<TILE>;
    constexpr int PPT = S::kPPT, THREADS = S::kThreads;
    constexpr int C4 = (CHC + 3) / 4;
    extern __shared__ __align__(16) unsigned char smem[];
    float4 *s_g = reinterpret_cast<float4 *>(smem);
    float2 *s_h = reinterpret_cast<float2 *>(s_g + batch);
    int4 *s_b = reinterpret_cast<int4 *>(s_h + batch);
    int *s_id = reinterpret_cast<int *>(s_b + batch);
    float4 *s_c = reinterpret_cast<float4 *>(s_id + batch);
    __shared__ int s_max;

    const int gt = blockIdx.x;
    const int c = camera_of_tile(cs, gt);
    const CamDev &cam = cs.cam[c];
    const int local = gt - cam.tile_offset;
    const int tx = local % cam.tiles_x, ty = local / cam.tiles_x;
    const int lane = threadIdx.x & 31;

    int px[PPT], py[PPT], last[PPT];
    float T[PPT], GS[PPT], g[PPT][CHC];
    int my_max = 0;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        int lin = threadIdx.x + k * THREADS;
        px[k] = tx * TILE + lin % TILE;
        py[k] = ty * TILE + lin / TILE;
        bool inside = px[k] < cam.W && py[k] < cam.H;
        size_t pix = inside ? (size_t)cam.pix_offset + (size_t)py[k] * cam.W + px[k] : 0;
        T[k] = inside ? final_T[pix] : 1.f;
        last[k] = inside ? last_contrib[pix] : 0;
        float gA = (inside && d_alpha) ? d_alpha[pix] : 0.f;
        float gb = 0.f;
#pragma unroll
        for (int q = 0; q < CHC; ++q) {
            g[k][q] = (inside && q < ch) ? d_image[pix * ch + q] : 0.f;
            gb += g[k][q] * bg.v[q];
        }
        // sum_c g_c S_c with S_N = T_N bg, minus the alpha-output term dL/dA T_N
        GS[k] = T[k] * (gb - gA);
        my_max = max(my_max, last[k]);
    }
    if (threadIdx.x == 0) s_max = 0;
    __syncthreads();
    const int wmax = __reduce_max_sync(0xffffffffu, my_max);
    if (lane == 0) atomicMax(&s_max, wmax);
    __syncthreads();
    const int2 rg = ranges[gt];
    const int count = min(s_max, rg.y - rg.x);  // last_contrib never exceeds the list length
    const int cn_total = cs.C * cs.N;
    const float amax = rc.alpha_max, amin = rc.alpha_min;

    for (int b0 = 0; b0 < count; b0 += batch) {
        const int cnt = min(batch, count - b0);
        // entries rg.x + count-1-b0-s, s = 0..cnt-1 (descending list positions)
        __syncthreads();
        for (int s = threadIdx.x; s < cnt; s += THREADS) {
            int id = values[rg.x + count - 1 - b0 - s];
            if ((unsigned)id >= (unsigned)cn_total) id = 0;  // holds by construction (ids come from the sort)
            float2 m = means2d[id];
            int r = radii[id];
            int x0, x1, y0, y1;
            support_span(m.x, r, x0, x1);
            support_span(m.y, r, y0, y1);
            s_id[s] = id;
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
        // the first entry of this batch that any pixel of this warp reaches
        const int jstart = max(0, (count - 1 - b0) - (wmax - 1));
        for (int j = jstart; j < cnt; ++j) {
            const int rel = count - 1 - b0 - j;  // 0-based position in the tile list
            const int4 bx = s_b[j];
            const float4 gg = s_g[j];
            const float2 hh = s_h[j];
            float dmx = 0.f, dmy = 0.f, dca = 0.f, dcb = 0.f, dcc = 0.f, dop = 0.f, dcol[CHC];
            float agx = 0.f, agy = 0.f;
#pragma unroll
            for (int q = 0; q < CHC; ++q) dcol[q] = 0.f;
            bool any = false;
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                if (rel >= last[k]) continue;
                if ((unsigned)(px[k] - bx.x) > (unsigned)bx.y || (unsigned)(py[k] - bx.z) > (unsigned)bx.w) continue;
                const float dx = ((float)px[k] + 0.5f) - gg.x;
                const float dy = ((float)py[k] + 0.5f) - gg.y;
                const float sigma = mahalanobis_half(dx, dy, gg.z, gg.w, hh.x);
                if (sigma < 0.f) continue;
                const float e = gauss_weight(sigma);
                const float oe = __fmul_rn(hh.y, e);
                const float alpha = fminf(amax, oe);
                if (alpha < amin) continue;
                any = true;
                const float ra = rcp_approx(1.f - alpha);
                const float Tn = T[k] * ra;  // transmittance in front of this Gaussian
                const float w = alpha * Tn;
                float gc = 0.f;
#pragma unroll
                for (int q4 = 0; q4 < C4; ++q4) {
                    const float4 v = s_c[j * C4 + q4];
                    const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int q = 4 * q4 + u;
                        if (q < CHC) {
                            gc += g[k][q] * vv[u];
                            dcol[q] += w * g[k][q];
                        }
                    }
                }
                float dalpha = gc * Tn - GS[k] * ra;
                GS[k] += gc * w;
                T[k] = Tn;
                if (oe > amax) dalpha = 0.f;  // alpha clamped: no gradient through it
                dop += e * dalpha;
                const float dsig = -oe * dalpha;
                // d sigma / d mu' = -conic D
                const float gx = -dsig * (gg.z * dx + gg.w * dy);
                const float gy = -dsig * (gg.w * dx + hh.x * dy);
                dmx += gx;
                dmy += gy;
                if (ABSG) {
                    agx += fabsf(gx);
                    agy += fabsf(gy);
                }
                dca += 0.5f * dsig * dx * dx;
                dcb += dsig * dx * dy;
                dcc += 0.5f * dsig * dy * dy;
            }
            if (!__any_sync(0xffffffffu, any)) continue;
            dmx = warp_sum(dmx);
            dmy = warp_sum(dmy);
            dca = warp_sum(dca);
            dcb = warp_sum(dcb);
            dcc = warp_sum(dcc);
            dop = warp_sum(dop);
#pragma unroll
            for (int q = 0; q < CHC; ++q) dcol[q] = warp_sum(dcol[q]);
            if (ABSG) {
                agx = warp_sum(agx);
                agy = warp_sum(agy);
            }
            if (lane == 0) {
                const int id = s_id[j];
                atomicAdd(d_means2d + id, make_float2(dmx, dmy));
                atomicAdd(d_conics + 3 * id, dca);
                atomicAdd(d_conics + 3 * id + 1, dcb);
                atomicAdd(d_conics + 3 * id + 2, dcc);
                atomicAdd(d_opac + id, dop);
#pragma unroll
                for (int q = 0; q < CHC; ++q)
                    if (q < ch) atomicAdd(d_colors + (size_t)id * ch + q, dcol[q]);
                if (ABSG) atomicAdd(absgrad + id, make_float2(agx, agy));
            }
        }
    }
}

template <int TILE, int CHC, bool ABSG>
static cudaError_t launch_bwd_t(const CamSet &cs, const RasterConsts &rc, int ch, int batch, const int *ranges,
                                const int *values, const int *radii, const float *means2d, const float *conics,
                                const float *opac, const float *colors, const BgConstB &bg, const float *final_T,
                                const int *last_contrib, const float *d_image, const float *d_alpha,
                                float *d_means2d, float *d_conics, float *d_opac, float *d_colors, float *absgrad,
                                cudaStream_t st) {
    constexpr int C4 = (CHC + 3) / 4;
    size_t smem = (size_t)batch * (sizeof(float4) + sizeof(float2) + sizeof(int4) + sizeof(int) + C4 * sizeof(float4));
    auto kern = raster_bwd_kernel<TILE, CHC, ABSG>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    if (cs.total_tiles == 0) return cudaSuccess;
    kern<<<cs.total_tiles, TileShapeB<TILE>::kThreads, smem, st>>>(
        cs, rc, ch, batch, (const int2 *)ranges, values, radii, (const float2 *)means2d, conics, opac, colors,
        bg, final_T, last_contrib, d_image, d_alpha, (float2 *)d_means2d, d_conics, d_opac, d_colors, (float2 *)absgrad);
    note_launch();
    return cudaGetLastError();
}

template <int TILE, bool ABSG>
static cudaError_t dispatch_bwd_ch(int chc, const CamSet &cs, const RasterConsts &rc, int ch, int batch,
                                   const int *ranges, const int *values, const int *radii, const float *means2d,
                                   const float *conics, const float *opac, const float *colors, const BgConstB &bg,
                                   const float *final_T, const int *last_contrib, const float *d_image,
                                   const float *d_alpha, float *d_means2d, float *d_conics, float *d_opac,
                                   float *d_colors, float *absgrad, cudaStream_t st) {
#define GS_BWD_CASE(K)                                                                                             \
    case K:                                                                                                        \
        return launch_bwd_t<TILE, K, ABSG>(cs, rc, ch, batch, ranges, values, radii, means2d, conics, opac, colors, \
                                           bg, final_T, last_contrib, d_image, d_alpha, d_means2d, d_conics, d_opac, \
                                           d_colors, absgrad, st);
    if constexpr (TILE == 16 && !ABSG) {
        switch (chc) {
            GS_BWD_CASE(1)
            GS_BWD_CASE(2)
            GS_BWD_CASE(3)
            GS_BWD_CASE(4)
            GS_BWD_CASE(8)
            GS_BWD_CASE(16)
            GS_BWD_CASE(32)
            GS_BWD_CASE(64)
        }
    } else {
        switch (chc) {
            GS_BWD_CASE(3)
            GS_BWD_CASE(4)
        }
    }
#undef GS_BWD_CASE
    return cudaErrorNotSupported;
}

int raster_channel_capacity(int tile, int ch, bool restricted);

cudaError_t launch_raster_bwd(const CamSet &cs, const RasterConsts &rc, int ch, int batch, const int *ranges,
                              const int *values, const int *radii, const float *means2d, const float *conics,
                              const float *opac, const float *colors, const float *bg_host, const float *final_T,
                              const int *last_contrib, const float *d_image, const float *d_alpha, float *d_means2d,
                              float *d_conics, float *d_opac, float *d_colors, float *absgrad, cudaStream_t st) {
    BgConstB bg;
    for (int q = 0; q < GS_MAX_CHANNELS; ++q) bg.v[q] = (bg_host && q < ch) ? bg_host[q] : 0.f;
    const bool absg = absgrad != nullptr;
    int chc = raster_channel_capacity(cs.tile, ch, absg);
#define GS_BWD_TILE(T)                                                                                            \
    if (cs.tile == T)                                                                                             \
        return absg ? dispatch_bwd_ch<T, true>(chc, cs, rc, ch, batch, ranges, values, radii, means2d, conics,      \
                                               opac, colors, bg, final_T, last_contrib, d_image, d_alpha,          \
                                               d_means2d, d_conics, d_opac, d_colors, absgrad, st)                 \
                    : dispatch_bwd_ch<T, false>(chc, cs, rc, ch, batch, ranges, values, radii, means2d, conics,     \
                                                opac, colors, bg, final_T, last_contrib, d_image, d_alpha,         \
                                                d_means2d, d_conics, d_opac, d_colors, nullptr, st);
    GS_BWD_TILE(8)
    GS_BWD_TILE(16)
    GS_BWD_TILE(32)
#undef GS_BWD_TILE
    return cudaErrorNotSupported;
}

}  // namespace gs
