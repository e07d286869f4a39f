// Internal device-side definitions of libgs (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gs.h"

namespace gs {

// Host-side launch accounting behind gs_kernel_launches() (defined in gs_abi.cu).
void note_launch();

// Records the text gs_last_error() returns on this thread (defined in gs_abi.cu).
void set_last_error(const char *text);

// Raises a kernel's dynamic shared-memory limit to at least `bytes` on the current device.
// The attribute is set once per (device, kernel, size): setting it again on every call
// can stall the host until the device is idle, which would serialise eager launches.
cudaError_t ensure_smem(const void *kernel, int bytes);

// CTAs of `kernel` (threads, dynamic shared memory) that fit on the current device at once,
// capped at `work` items: the grid of a persistent launch.  Cached per (device, kernel, smem).
int persistent_grid(const void *kernel, int threads, int smem, int work);

constexpr int kMaxCams = GS_MAX_CAMERAS;

// Per-camera constants, passed to kernels by value (a __grid_constant__ CamSet).
struct CamDev {
    float R[9];        // world -> camera rotation, row-major
    float t[3];        // world -> camera translation
    float fx, fy, cx, cy;
    int W, H;
    int tiles_x, tiles_y;
    int tile_offset;   // first global tile of this camera
    int pix_offset;    // first pixel of this camera in packed per-pixel arrays
};

struct CamSet {
    int C;
    int N;             // Gaussians per camera (per-(camera, Gaussian) arrays are [C, N])
    int total_tiles;
    int total_pixels;
    int tile;
    CamDev cam[kMaxCams];
};

// Byte offsets of the tile_bin_sort workspace regions (see binsort.cu).
struct BinSortLayout {
    size_t dk0, dk1, dv0, dv1, counts, rects, offsets, win_start, win_bits, partials, misc, matrix, tk0, tk1, tvB, total;
};

struct RasterConsts {
    float eps2d, near_plane, alpha_min, alpha_max, T_min;
    int antialiased;
    int colors_shared;      // compositing: colour rows indexed by Gaussian n (shared by the cameras)
    const int *tile_order;  // compositing: CTA b renders tile tile_order[b] (NULL: tile b)
    int *work;              // persistent compositing: [next index, CTAs finished] (NULL: one CTA per tile)
};

// Persistent compositing: the next index into tile_order for this CTA (read by every thread),
// or total when the work is exhausted.  Uses one shared int of the caller.
__device__ __forceinline__ int next_work_item(int *work, int *s_next) {
    if (threadIdx.x == 0) *s_next = atomicAdd(work, 1);
    __syncthreads();
    const int i = *s_next;
    __syncthreads();
    return i;
}

// Persistent compositing: the last CTA to finish resets the counters for the next launch.
__device__ __forceinline__ void finish_work(int *work) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(work + 1, 1) == (int)gridDim.x - 1) {  // every CTA has taken its last index
            work[0] = 0;
            work[1] = 0;
        }
    }
}

// Sums v[0..V) over the CTA and adds the totals to dst[0..V) with one atomic each (thread
// k adds value k).  Every thread of the CTA must call it; s_red holds V * (warps) floats.
template <int V>
__device__ __forceinline__ void block_sum_atomic(float (&v)[V], float *dst, float *s_red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, warps = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < V; ++k) {
        float x = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) s_red[warp * V + k] = x;
    }
    __syncthreads();
    if (threadIdx.x < V) {
        float t = 0.f;
        for (int w = 0; w < warps; ++w) t += s_red[w * V + threadIdx.x];
        if (t != 0.f) atomicAdd(dst + threadIdx.x, t);
    }
    __syncthreads();
}

// Global tile rendered by this CTA of a compositing launch; -1 for an out-of-range entry of
// a caller-supplied order (the CTA then renders nothing).
__device__ __forceinline__ int tile_of_block(const RasterConsts &rc, int total_tiles) {
    const int t = rc.tile_order ? rc.tile_order[blockIdx.x] : (int)blockIdx.x;
    return (unsigned)t < (unsigned)total_tiles ? t : -1;
}

// Camera of a global tile: the last camera whose tile_offset <= gtile.
__device__ __forceinline__ int camera_of_tile(const CamSet &cs, int gtile) {
    int c = 0;
#pragma unroll 1
    for (int k = 1; k < cs.C; ++k)
        if (cs.cam[k].tile_offset <= gtile) c = k;
    return c;
}

// Pixel box of the support rule (inclusive pixel indices): pixel i supports a Gaussian
// with float32 mean m and integer radius r iff |i + 0.5 - m| <= r, i.e. i in
// [ceil(m - r - 0.5), floor(m + r - 0.5)].  Evaluated exactly without float64:
// with j = 2i + 1 the condition is ceil(2m) - 2r <= j <= floor(2m) + 2r, and 2m,
// ceil(2m), floor(2m) are exact in float32.  |2m| is clamped to 2^28, far outside
// any image, which keeps the integers in range without changing the clipped box.
__device__ __forceinline__ void support_span(float m, int r, int &lo, int &hi) {
    float m2 = fminf(fmaxf(2.f * m, -268435456.f), 268435456.f);
    int a = (int)ceilf(m2) - 2 * r;  // smallest admissible j
    int b = (int)floorf(m2) + 2 * r; // largest admissible j
    lo = a >> 1;                     // ceil((a - 1) / 2)
    hi = (b - 1) >> 1;               // floor((b - 1) / 2)
}

__device__ __forceinline__ bool pixel_box(float mx, float my, int r, int W, int H, int &x0, int &x1, int &y0,
                                          int &y1) {
    support_span(mx, r, x0, x1);
    support_span(my, r, y0, y1);
    x0 = max(x0, 0);
    y0 = max(y0, 0);
    x1 = min(x1, W - 1);
    y1 = min(y1, H - 1);
    return x0 <= x1 && y0 <= y1;
}

// Hardware exp2 / reciprocal approximations (MUFU).
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;

// The compositing kernels stage the conic pre-scaled,
// (a', b', c') = -log2(e) (a / 2, b, c / 2), so that the exponent of the Gaussian weight is
// p = -log2(e) sigma = a' dx^2 + b' dx dy + c' dy^2 and exp(-sigma) = 2^p.  A thread's pixels
// share dx (one column), so per Gaussian it forms a' dx^2 and b' dx once and per pixel
// evaluates p = (c' dy + b' dx) dy + a' dx^2 with two FMAs.  Forward and backward use these
// same explicitly rounded steps, so they obtain bit-identical weights.
struct GaussRow {
    float axx, bdx, c;
};
__device__ __forceinline__ GaussRow gauss_row(float dx, float a, float b, float c) {
    return GaussRow{__fmul_rn(a, __fmul_rn(dx, dx)), __fmul_rn(b, dx), c};
}
__device__ __forceinline__ float gauss_exponent(const GaussRow &r, float dy) {
    return __fmaf_rn(__fmaf_rn(r.c, dy, r.bdx), dy, r.axx);
}

// Launch shape of the compositing kernels: PPT pixels per thread stacked along y, so a
// tile of TILE x TILE pixels runs TILE*TILE/PPT threads and a warp covers a TILE-wide band
// of 32*PPT/TILE rows.
template <int TILE, int PPT>
struct RasterShape {
    static constexpr int kPPT = PPT;
    static constexpr int kThreads = TILE * TILE / PPT;
    // Each warp owns a band of kBandW x kBandH pixels: 8 columns x 4 lane rows, every lane
    // PPT consecutive pixels of its column.  Narrow, tall bands keep most lanes of a warp
    // inside the footprint of a small Gaussian (a 32 x 4 band would leave most of them idle).
    static constexpr int kBandW = 8;
    static constexpr int kBandH = 4 * PPT;
    static constexpr int kBandsX = TILE / kBandW;
    static_assert(kThreads >= 32 && kThreads <= 1024 && kThreads % 32 == 0, "bad raster shape");
    static_assert(TILE % kBandW == 0 && TILE % kBandH == 0 && kBandsX * (TILE / kBandH) == kThreads / 32,
                  "bands must tile the tile");
};

// Pixel band of warp `warp` of a tile whose corner is (tx0, ty0), and this lane's column and
// first row inside it.
template <class S>
__device__ __forceinline__ void warp_band(int tx0, int ty0, int warp, int lane, int &wx0, int &wx1, int &wy0,
                                          int &wy1, int &px, int &py0) {
    wx0 = tx0 + (warp % S::kBandsX) * S::kBandW;
    wy0 = ty0 + (warp / S::kBandsX) * S::kBandH;
    wx1 = wx0 + S::kBandW - 1;
    wy1 = wy0 + S::kBandH - 1;
    px = wx0 + (lane % S::kBandW);
    py0 = wy0 + (lane / S::kBandW) * S::kPPT;
}

// One Gaussian of a tile's list as both compositing kernels stage it in shared memory:
//   g   = (mean x, mean y, conic a, conic b)
//   h   = (conic c, opacity, sigma cut, id as int bits)
//   box = (x0, x1 - x0, y0, y1 - y0) of the (unclipped) pixel box
// The sigma cut is ln(opacity / alpha_min): beyond it alpha < alpha_min, so such pairs
// never blend; it is used only to skip work that would be skipped anyway.
__device__ __forceinline__ void make_splat(int id, float2 m, int r, float o, float ca, float cb, float cc,
                                           float alpha_min, float4 &g, float4 &h, int4 &box) {
    int x0, x1, y0, y1;
    support_span(m.x, r, x0, x1);
    support_span(m.y, r, y0, y1);
    const float cut = !(o >= alpha_min) ? -1.f : (alpha_min > 0.f ? __logf(o / alpha_min) : 3.0e38f);
    g = make_float4(m.x, m.y, -0.5f * kLog2e * ca, -kLog2e * cb);
    h = make_float4(-0.5f * kLog2e * cc, o, cut, __int_as_float(id));
    box = make_int4(x0, x1 - x0, y0, y1 - y0);
}

__device__ __forceinline__ void stage_splat(int id, const float2 *__restrict__ means2d,
                                            const float *__restrict__ conics, const float *__restrict__ opac,
                                            const int *__restrict__ radii, float alpha_min, float4 &g, float4 &h,
                                            int4 &box) {
    make_splat(id, means2d[id], radii[id], opac[id], conics[3 * id], conics[3 * id + 1], conics[3 * id + 2],
               alpha_min, g, h, box);
}

// One staged batch in shared memory: `batch` entries of g, h and box (see make_splat) and C4
// float4 colour slots per entry.
struct StagedBatch {
    float4 *g;
    float4 *h;
    int4 *b;
    float4 *c;
};

// The staged batch at the start of shared memory.
template <int C4>
__device__ __forceinline__ StagedBatch staged_batch(unsigned char *smem, int batch) {
    float4 *g = reinterpret_cast<float4 *>(smem);
    return StagedBatch{g, g + batch, reinterpret_cast<int4 *>(g + 2 * batch), g + 3 * batch};
}

// Bytes of a staged batch of `batch` entries with C4 colour slots each.
__host__ __device__ constexpr size_t staged_batch_bytes(int batch, int c4) {
    return (size_t)batch * (3 + c4) * sizeof(float4);
}

// Gathers `cnt` entries of a tile's list into `sb`: entry s is the Gaussian at list position
// pos0 + dir * s (dir = +1 front to back, -1 back to front).  Each thread of the CTA stages
// entries threadIdx.x, threadIdx.x + THREADS, ...
template <int THREADS, int C4>
__device__ __forceinline__ void stage_batch(const StagedBatch &sb, const int *__restrict__ values, long long pos0,
                                            int dir, int cnt, int cn_total, int n_shared, int ch,
                                            const float2 *__restrict__ means2d, const float *__restrict__ conics,
                                            const float *__restrict__ opac, const int *__restrict__ radii,
                                            const float *__restrict__ colors, float alpha_min) {
    for (int s = threadIdx.x; s < cnt; s += THREADS) {
        int id = values[pos0 + dir * s];
        if ((unsigned)id >= (unsigned)cn_total) id = 0;  // holds by construction (ids come from the sort)
        float4 g, h;
        int4 b;
        stage_splat(id, means2d, conics, opac, radii, alpha_min, g, h, b);
        sb.g[s] = g;
        sb.h[s] = h;
        sb.b[s] = b;
        const float *col = colors + (size_t)(n_shared ? id % n_shared : id) * ch;
#pragma unroll
        for (int q = 0; q < C4; ++q) {
            float4 v;
            v.x = (4 * q + 0 < ch) ? col[4 * q + 0] : 0.f;
            v.y = (4 * q + 1 < ch) ? col[4 * q + 1] : 0.f;
            v.z = (4 * q + 2 < ch) ? col[4 * q + 2] : 0.f;
            v.w = (4 * q + 3 < ch) ? col[4 * q + 3] : 0.f;
            sb.c[s * C4 + q] = v;
        }
    }
}

// Can the staged Gaussian blend at any pixel of the rectangle of pixel indices
// [rx0, rx1] x [ry0, ry1]?  False only when the pixel box misses the rectangle or when
// sigma exceeds the cut (plus a margin far above float32 rounding) on the whole
// rectangle of pixel centres; so a false answer never removes a pair that blends.
__device__ __forceinline__ bool box_hits(const int4 &b, int rx0, int rx1, int ry0, int ry1) {
    return !(b.x > rx1 || b.x + b.y < rx0 || b.z > ry1 || b.z + b.w < ry0);
}

__device__ __forceinline__ bool may_blend(const float4 &g, const float4 &h, const int4 &b, int rx0, int rx1, int ry0,
                                          int ry1) {
    if (!box_hits(b, rx0, rx1, ry0, ry1)) return false;
    if (!(h.z >= 0.f)) return false;
    // the minimum of sigma(p) = 1/2 (p-m)^T [[a,b],[b,c]] (p-m) over the rectangle of pixel
    // centres, taken as the maximum of the staged exponent p = a' dx^2 + b' dx dy + c' dy^2
    // = -log2(e) sigma (a', c' < 0: concave), which is on the boundary unless the mean is inside
    const float x0 = (float)rx0 + 0.5f - g.x, x1 = (float)rx1 + 0.5f - g.x;
    const float y0 = (float)ry0 + 0.5f - g.y, y1 = (float)ry1 + 0.5f - g.y;
    if (x0 <= 0.f && x1 >= 0.f && y0 <= 0.f && y1 >= 0.f) return true;
    const float a = g.z, bb = g.w, c = h.x;
    // (approximate reciprocals only place the maximising point; the margin below covers them)
    const float ia = rcp_approx(a), ic = rcp_approx(c);
    float best = -3.0e38f;
    // vertical edges: dx fixed, dp/ddy = b' dx + 2 c' dy = 0
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const float dx = e ? x1 : x0;
        const float bdx = bb * dx;
        const float dy = fminf(fmaxf(-0.5f * bdx * ic, y0), y1);
        best = fmaxf(best, fmaf(fmaf(c, dy, bdx), dy, a * dx * dx));
    }
    // horizontal edges: dy fixed, dp/ddx = 2 a' dx + b' dy = 0
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const float dy = e ? y1 : y0;
        const float bdy = bb * dy;
        const float dx = fminf(fmaxf(-0.5f * bdy * ia, x0), x1);
        best = fmaxf(best, fmaf(fmaf(a, dx, bdy), dx, c * dy * dy));
    }
    // sigma_min <= cut (1 + 1e-3) + 1e-3, a margin far above float32 rounding
    return best >= -(h.z * 1.001f + 1e-3f) * kLog2e;
}

}  // namespace gs
