// Backward of the compositing sum (App. D.2), one CTA per tile.
//
// Each pixel replays its list back to front from its last contributor: alpha is
// recomputed with the forward's exact arithmetic (same staging, same formulas, so the same
// pairs are skipped), T_n = T_{n+1} / (1 - alpha_n) is recovered from the stored final T,
// and the suffix term sum_c g_c S_c is carried as one scalar per pixel.  Only final T and
// the last-contributor index come from the forward, so memory stays O(pixels + Gaussians).
//
// Per Gaussian, a thread first sums its PPT pixels, then the warp sums its lanes with a
// transpose butterfly: at each step every lane trades half of its remaining values with
// its partner, so V values cost about V shuffles instead of 5 V, and the warp totals end
// up spread over the lanes -- the atomics of all V values leave in one instruction.
#include "gs_internal.cuh"


namespace gs {

struct BgConstB {
    float v[GS_MAX_CHANNELS];
};

__host__ __device__ constexpr int pow2_at_least(int v) { return v <= 1 ? 1 : 2 * pow2_at_least((v + 1) / 2); }

// Warp sum of VP values (VP a power of two <= 32).  On return lane l holds in v[0] the
// total of value l / (32 / VP); all lanes of that group hold the same total.
template <int VP>
__device__ __forceinline__ float transpose_sum(float (&v)[VP], int lane) {
#pragma unroll
    for (int n = VP / 2, o = 16; n >= 1; n >>= 1, o >>= 1) {
        const bool hi = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < n; ++i) {
            const float keep = hi ? v[i + n] : v[i];
            const float send = hi ? v[i] : v[i + n];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    float x = v[0];
#pragma unroll
    for (int o = 16 / VP; o >= 1; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Gradient slot of value index `idx` of Gaussian `id`:
// [mean x, mean y, conic a, conic b, conic c, opacity, (absgrad x, absgrad y), colour 0..ch-1]
template <bool ABSG>
__device__ __forceinline__ float *grad_slot(int idx, int id, int ch, int cmod, float *d_means2d, float *d_conics,
                                            float *d_opac, float *d_colors, float *absgrad) {
    if (idx < 2) return d_means2d + 2 * (size_t)id + idx;
    if (idx < 5) return d_conics + 3 * (size_t)id + (idx - 2);
    if (idx == 5) return d_opac + id;
    if (ABSG) {
        if (idx < 8) return absgrad + 2 * (size_t)id + (idx - 6);
        idx -= 2;
    }
    const int q = idx - 6;  // colour rows: per (camera, Gaussian), or per Gaussian (cmod = N) when shared
    return q < ch ? d_colors + (size_t)(cmod ? id % cmod : id) * ch + q : nullptr;
}

// Factor applied to the warp total of value `idx`: 1 / log2(e) for the mean (and absgrad)
// terms when they are summed in units of log2(e) (SG).
template <bool ABSG, bool SG>
__device__ __forceinline__ float total_scale(int idx) {
    if (idx == 2 || idx == 4) return 0.5f;  // dsig dx^2 and dsig dy^2 are summed unhalved
    return (SG && (idx < 2 || (ABSG && idx >= 6 && idx < 8))) ? kLn2 : 1.f;
}

// With the pre-scaled conic, the mean gradient of each pixel is either summed in units of
// log2(e) and rescaled once on the warp totals (4 pixels per thread), or computed from the
// conic recovered once per Gaussian (1 or 2 pixels per thread); each is the faster there.
template <int PPT>
__host__ __device__ constexpr bool scaled_grad() {
    return PPT >= 4;
}

// Reduces values [OFF, min(OFF + 32, V)) of v over the warp and adds them to global memory.
template <int V, int OFF, bool ABSG, bool SG>
__device__ __forceinline__ void reduce_chunks(const float (&v)[V], int lane, int id, int ch, int cmod, float *d_means2d,
                                              float *d_conics, float *d_opac, float *d_colors, float *absgrad) {
    if constexpr (OFF < V) {
        constexpr int n = (V - OFF) < 32 ? (V - OFF) : 32;
        constexpr int VP = pow2_at_least(n);
        float w[VP];
#pragma unroll
        for (int i = 0; i < VP; ++i) w[i] = (i < n) ? v[OFF + i] : 0.f;
        const float tot = transpose_sum<VP>(w, lane);
        constexpr int group = 32 / VP;
        const int idx = lane / group;
        if ((lane % group) == 0 && idx < n) {
            float *slot = grad_slot<ABSG>(OFF + idx, id, ch, cmod, d_means2d, d_conics, d_opac, d_colors, absgrad);
            if (slot) atomicAdd(slot, tot * total_scale<ABSG, SG>(OFF + idx));
        }
        reduce_chunks<V, OFF + 32, ABSG, SG>(v, lane, id, ch, cmod, d_means2d, d_conics, d_opac, d_colors, absgrad);
    }
}

#ifndef GS_BWD_SMEM_REDUCE
#define GS_BWD_SMEM_REDUCE 1
#endif

// The shared-memory reduction pays off where a warp covers few pixels per Gaussian (1 or 2 per
// thread: more reductions per blend); with 4 pixels per thread the butterfly is faster.
template <int PPT>
__host__ __device__ constexpr bool smem_reduce() {
    return GS_BWD_SMEM_REDUCE && PPT <= 2;
}

// Warp sum of the V values through a per-warp [8][32] shared transpose: for each group of 8
// values every lane stores its 8 values (value-major), then lane l sums value l / 4 over the 8
// lanes 8 (l % 4) .. 8 (l % 4) + 7 with two 16-byte loads and finishes with two shuffles, so a
// group costs 8 stores, 2 loads, 2 shuffles and 9 adds per lane instead of a shuffle butterfly
// with a select per value and step.  A group of at most two values uses plain butterflies.
template <int V, int OFF, bool ABSG, bool SG>
__device__ __forceinline__ void reduce_smem(const float (&v)[V], float *s_red, int lane, int id, int ch, int cmod,
                                            float *d_means2d, float *d_conics, float *d_opac, float *d_colors,
                                            float *absgrad) {
    if constexpr (OFF < V) {
        constexpr int n = (V - OFF) < 8 ? (V - OFF) : 8;
        if constexpr (n <= 2) {
#pragma unroll
            for (int i = 0; i < n; ++i) {
                float x = v[OFF + i];
#pragma unroll
                for (int o = 16; o >= 1; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
                if (lane == 8 * i) {
                    float *slot = grad_slot<ABSG>(OFF + i, id, ch, cmod, d_means2d, d_conics, d_opac, d_colors, absgrad);
                    if (slot) atomicAdd(slot, x * total_scale<ABSG, SG>(OFF + i));
                }
            }
        } else {
            __syncwarp();  // every lane has read the previous group
#pragma unroll
            for (int i = 0; i < n; ++i) s_red[i * 32 + lane] = v[OFF + i];
            __syncwarp();
            const int q = lane >> 2, c = lane & 3;
            float t = 0.f;
            if (q < n) {
                const float4 a = *reinterpret_cast<const float4 *>(s_red + q * 32 + 8 * c);
                const float4 b = *reinterpret_cast<const float4 *>(s_red + q * 32 + 8 * c + 4);
                t = ((a.x + a.y) + (a.z + a.w)) + ((b.x + b.y) + (b.z + b.w));
            }
            t += __shfl_xor_sync(0xffffffffu, t, 1);
            t += __shfl_xor_sync(0xffffffffu, t, 2);
            if (c == 0 && q < n) {
                float *slot = grad_slot<ABSG>(OFF + q, id, ch, cmod, d_means2d, d_conics, d_opac, d_colors, absgrad);
                if (slot) atomicAdd(slot, t * total_scale<ABSG, SG>(OFF + q));
            }
        }
        reduce_smem<V, OFF + 8, ABSG, SG>(v, s_red, lane, id, ch, cmod, d_means2d, d_conics, d_opac, d_colors,
                                          absgrad);
    }
}

template <int TILE, int PPT, int CHC, bool ABSG>
__global__ void __launch_bounds__(RasterShape<TILE, PPT>::kThreads) raster_bwd_kernel(
    const __grid_constant__ CamSet cs, RasterConsts rc, int ch, int batch, const int2 *__restrict__ ranges,
    const int *__restrict__ values, const int *__restrict__ radii, const float2 *__restrict__ means2d,
    const float *__restrict__ conics, const float *__restrict__ opac, const float *__restrict__ colors,
    const __grid_constant__ BgConstB bg, const float *__restrict__ final_T, const int *__restrict__ last_contrib,
    const float *__restrict__ d_image, const float *__restrict__ d_alpha, float *__restrict__ d_means2d,
    float *__restrict__ d_conics, float *__restrict__ d_opac, float *__restrict__ d_colors,
    float *__restrict__ absgrad) {
    using S = RasterShape<TILE, PPT>;
    constexpr int THREADS = S::kThreads;
    constexpr int C4 = (CHC + 3) / 4;
    constexpr int NA = ABSG ? 2 : 0;
    constexpr int V = 6 + NA + CHC;
    constexpr bool SG = scaled_grad<PPT>();
    // lanes with 2 or 4 pixels (one column) sum per-pixel moments; absgrad needs per-pixel terms
    constexpr bool MOMENTS = !ABSG && PPT >= 2;
    extern __shared__ __align__(16) unsigned char smem[];
    float *s_red = reinterpret_cast<float *>(smem + staged_batch_bytes(batch, C4)) + (threadIdx.x >> 5) * (8 * 32);
    __shared__ int s_max;

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
    int wx0, wx1, wy0, wy1, px, py0;
    warp_band<S>(tx0, ty0, warp, lane, wx0, wx1, wy0, wy1, px, py0);
    const float fx = (float)px + 0.5f;

    int last[PPT];
    float T[PPT], GS[PPT], g[PPT][CHC];
    int my_max = 0;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const int py = py0 + k;
        const bool inside = px < cam.W && py < cam.H;
        const size_t pix = inside ? (size_t)cam.pix_offset + (size_t)py * cam.W + px : 0;
        T[k] = inside ? final_T[pix] : 1.f;
        last[k] = inside ? last_contrib[pix] : 0;
        const float gA = (inside && d_alpha) ? d_alpha[pix] : 0.f;
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
    const int cmod = rc.colors_shared ? cs.N : 0;
    const float amax = rc.alpha_max, amin = rc.alpha_min;

    const StagedBatch sb = staged_batch<C4>(smem, batch);
    const float4 *s_g = sb.g, *s_h = sb.h, *s_c = sb.c;
    const int4 *s_b = sb.b;

    for (int b0 = 0; b0 < count; b0 += batch) {
        const int cnt = min(batch, count - b0);
        // entries rg.x + count-1-b0-s, s = 0..cnt-1 (descending list positions)
        __syncthreads();
        stage_batch<THREADS, C4>(sb, values, (long long)rg.x + count - 1 - b0, -1, cnt, cn_total, cmod, ch, means2d,
                                 conics, opac, radii, colors, amin);
        __syncthreads();
        // the first entry of this batch that any pixel of this warp reaches
        const int jstart = max(0, (count - 1 - b0) - (wmax - 1));
        for (int base = jstart & ~31; base < cnt; base += 32) {
            const int jl = base + lane;
            bool hit = false;
            if (jl >= jstart && jl < cnt) hit = may_blend(s_g[jl], s_h[jl], s_b[jl], wx0, wx1, wy0, wy1);
            unsigned m = __ballot_sync(0xffffffffu, hit);
            while (m) {
                const int j = base + __ffs(m) - 1;
                m &= m - 1;
                const int rel = count - 1 - b0 - j;  // 0-based position in the tile list
                const int4 bx = s_b[j];
                const float4 gg = s_g[j];
                const float4 hh4 = s_h[j];
                const bool inx = (unsigned)(px - bx.x) <= (unsigned)bx.y;
                const float dx = fx - gg.x;
                const float xx = __fmul_rn(dx, dx);
                const GaussRow gr = gauss_row(dx, gg.z, gg.w, hh4.x);
                // per Gaussian: the mean gradient of a pixel is dsig (+-) (Bx + Mx dy, By + My dy)
                const float Mx = SG ? gg.w : gg.w * -kLn2;
                const float My = SG ? 2.f * hh4.x : hh4.x * (-2.f * kLn2);
                const float Bx = SG ? 2.f * gg.z * dx : gg.z * (-2.f * kLn2) * dx;
                const float By = Mx * dx;
                float v[V];
#pragma unroll
                for (int i = 0; i < V; ++i) v[i] = 0.f;
                // (MOMENTS) the lane's pixels share dx: sum dsig, dsig dy and dsig dy^2 over them and
                // form the mean and conic terms once per Gaussian instead of per pixel:
                // sum gx = s (Mx S1 + Bx S0), sum dsig dx^2 = dx^2 S0, sum dsig dx dy = dx S1
                float S0 = 0.f, S1 = 0.f, S2 = 0.f;
                bool any = false;
                // the PPT pixels are independent chains: evaluate all of them without branches
                // (a pair that does not blend gets zero weight and zero dL/dalpha, so every
                // sum below adds an exact zero and T and S stay as they were)
#pragma unroll
                for (int k = 0; k < PPT; ++k) {
                    const bool act = rel < last[k] && inx && (unsigned)(py0 + k - bx.z) <= (unsigned)bx.w;
                    const float dy = ((float)(py0 + k) + 0.5f) - gg.y;
                    const float yy = __fmul_rn(dy, dy), xy = __fmul_rn(dx, dy);
                    const float pe = gauss_exponent(gr, dy);  // -log2(e) sigma
                    const float e = ex2_approx(pe);
                    const bool neg = pe > 0.f;  // sigma < 0
                    const float oe = __fmul_rn(hh4.y, e);
                    const float alpha = fminf(amax, oe);
                    const bool take = act && !neg && !(alpha < amin);
                    any = any || take;
                    const float ra = rcp_approx(1.f - alpha);
                    const float Tn = T[k] * ra;  // transmittance in front of this Gaussian
                    const float w = take ? alpha * Tn : 0.f;
                    float gc = 0.f;
#pragma unroll
                    for (int q4 = 0; q4 < C4; ++q4) {
                        const float4 cv = s_c[j * C4 + q4];
                        const float vv[4] = {cv.x, cv.y, cv.z, cv.w};
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int q = 4 * q4 + u;
                            if (q < CHC) {
                                gc += g[k][q] * vv[u];
                                v[6 + NA + q] += w * g[k][q];
                            }
                        }
                    }
                    // alpha clamped (oe > amax): no gradient through it
                    const float dalpha = (take && !(oe > amax)) ? gc * Tn - GS[k] * ra : 0.f;
                    GS[k] += gc * w;
                    T[k] = take ? Tn : T[k];
                    v[5] += e * dalpha;
                    const float dsig = -oe * dalpha;
                    // d sigma / d mu' = -conic D
                    // (with SG: -conic D = (2 a' dx + b' dy, b' dx + 2 c' dy) / log2(e) for the staged
                    // (a', b', c'), and the 1 / log2(e) is applied to the warp totals)
                    if constexpr (MOMENTS) {
                        S0 += dsig;
                        S1 += dsig * dy;
                        S2 += dsig * yy;
                    } else {
                        const float sd = SG ? dsig : -dsig;
                        const float gx = sd * (Mx * dy + Bx);
                        const float gy = sd * (My * dy + By);
                        v[0] += gx;
                        v[1] += gy;
                        if (ABSG) {
                            v[6] += fabsf(gx);
                            v[7] += fabsf(gy);
                        }
                        // d sigma / d conic = (dx^2 / 2, dx dy, dy^2 / 2): the halves are applied to the warp totals
                        v[2] += dsig * xx;
                        v[3] += dsig * xy;
                        v[4] += dsig * yy;
                    }
                }
                if constexpr (MOMENTS) {
                    const float s0 = SG ? S0 : -S0, s1 = SG ? S1 : -S1;
                    v[0] = Mx * s1 + Bx * s0;
                    v[1] = My * s1 + By * s0;
                    v[2] = xx * S0;
                    v[3] = dx * S1;
                    v[4] = S2;
                }
                if (!__any_sync(0xffffffffu, any)) continue;
                if constexpr (smem_reduce<PPT>())
                    reduce_smem<V, 0, ABSG, SG>(v, s_red, lane, __float_as_int(hh4.w), ch, cmod, d_means2d,
                                                d_conics, d_opac, d_colors, absgrad);
                else
                    reduce_chunks<V, 0, ABSG, SG>(v, lane, __float_as_int(hh4.w), ch, cmod, d_means2d, d_conics,
                                                  d_opac, d_colors, absgrad);
            }
        }
    }
    __syncthreads();  // the next tile reuses the shared memory
    }
    if (rc.work) finish_work(rc.work);
}

// staged batch (splat, box, colours) + (shared-memory reduction) one [8][32] float buffer per warp
size_t raster_bwd_smem(int batch, int chc, int threads, bool reduce_buffers) {
    return staged_batch_bytes(batch, (chc + 3) / 4) +
           (reduce_buffers ? (size_t)(threads / 32) * 8 * 32 * sizeof(float) : 0);
}

template <int TILE, int PPT, int CHC, bool ABSG>
static cudaError_t launch_bwd_t(const CamSet &cs, const RasterConsts &rc, int ch, int batch, const int *ranges,
                                const int *values, const int *radii, const float *means2d, const float *conics,
                                const float *opac, const float *colors, const BgConstB &bg, const float *final_T,
                                const int *last_contrib, const float *d_image, const float *d_alpha,
                                float *d_means2d, float *d_conics, float *d_opac, float *d_colors, float *absgrad,
                                cudaStream_t st) {
    const size_t smem = raster_bwd_smem(batch, CHC, RasterShape<TILE, PPT>::kThreads, smem_reduce<PPT>());
    auto kern = raster_bwd_kernel<TILE, PPT, CHC, ABSG>;
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
        final_T, last_contrib, d_image, d_alpha, d_means2d, d_conics, d_opac, d_colors, absgrad);
    note_launch();
    return cudaGetLastError();
}

template <int TILE, int PPT, bool ABSG>
static cudaError_t dispatch_bwd_ch(int chc, const CamSet &cs, const RasterConsts &rc, int ch, int batch,
                                   const int *ranges, const int *values, const int *radii, const float *means2d,
                                   const float *conics, const float *opac, const float *colors, const BgConstB &bg,
                                   const float *final_T, const int *last_contrib, const float *d_image,
                                   const float *d_alpha, float *d_means2d, float *d_conics, float *d_opac,
                                   float *d_colors, float *absgrad, cudaStream_t st) {
#define GS_BWD_CASE(K)                                                                                             \
    case K:                                                                                                        \
        return launch_bwd_t<TILE, PPT, K, ABSG>(cs, rc, ch, batch, ranges, values, radii, means2d, conics, opac, colors, \
                                           bg, final_T, last_contrib, d_image, d_alpha, d_means2d, d_conics, d_opac, \
                                           d_colors, absgrad, st);
    if constexpr (TILE == 16 && PPT == 1 && !ABSG) {
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

int raster_channel_capacity(int tile, int ppt, int ch, bool restricted);

cudaError_t launch_raster_bwd(const CamSet &cs, const RasterConsts &rc, int ch, int batch, int ppt, const int *ranges,
                              const int *values, const int *radii, const float *means2d, const float *conics,
                              const float *opac, const float *colors, const float *bg_host, const float *final_T,
                              const int *last_contrib, const float *d_image, const float *d_alpha, float *d_means2d,
                              float *d_conics, float *d_opac, float *d_colors, float *absgrad, cudaStream_t st) {
    BgConstB bg;
    for (int q = 0; q < GS_MAX_CHANNELS; ++q) bg.v[q] = (bg_host && q < ch) ? bg_host[q] : 0.f;
    const bool absg = absgrad != nullptr;
    int chc = raster_channel_capacity(cs.tile, ppt, ch, absg);
#define GS_BWD_TILE(T, P)                                                                                         \
    if (cs.tile == T && ppt == P)                                                                                 \
        return absg ? dispatch_bwd_ch<T, P, true>(chc, cs, rc, ch, batch, ranges, values, radii, means2d, conics,   \
                                                  opac, colors, bg, final_T, last_contrib, d_image, d_alpha,       \
                                                  d_means2d, d_conics, d_opac, d_colors, absgrad, st)              \
                    : dispatch_bwd_ch<T, P, false>(chc, cs, rc, ch, batch, ranges, values, radii, means2d, conics,  \
                                                   opac, colors, bg, final_T, last_contrib, d_image, d_alpha,      \
                                                   d_means2d, d_conics, d_opac, d_colors, nullptr, st);
    GS_BWD_TILE(8, 1)
    GS_BWD_TILE(16, 1)
    GS_BWD_TILE(16, 2)
    GS_BWD_TILE(32, 2)
    GS_BWD_TILE(32, 4)
#undef GS_BWD_TILE
    return cudaErrorNotSupported;
}

}  // namespace gs
