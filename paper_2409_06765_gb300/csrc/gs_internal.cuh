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
    size_t dk0, dk1, dv0, dv1, counts, partials, misc, hist, tk0, tk1, tvB, total;
};

struct RasterConsts {
    float eps2d, near_plane, alpha_min, alpha_max, T_min;
    int antialiased;
};

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

// sigma = 1/2 D^T conic D for conic [[a,b],[b,c]], written with explicit roundings so the
// forward and the backward kernels obtain bit-identical values.
__device__ __forceinline__ float mahalanobis_half(float dx, float dy, float ca, float cb, float cc) {
    float xx = __fmul_rn(dx, dx);
    float yy = __fmul_rn(dy, dy);
    float xy = __fmul_rn(dx, dy);
    float s = __fmaf_rn(ca, xx, __fmul_rn(cc, yy));
    return __fmaf_rn(0.5f, s, __fmul_rn(cb, xy));
}

// exp(-sigma) = 2^(-sigma log2 e)
__device__ __forceinline__ float gauss_weight(float sigma) {
    return ex2_approx(__fmul_rn(-1.4426950408889634f, sigma));
}

}  // namespace gs
