// The extern "C" entry points declared in include/gs.h: argument validation, packing of
// the host camera array into the by-value kernel parameter block, and dispatch.
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <mutex>

#include "gs_internal.cuh"

namespace gs {

cudaError_t launch_project_fwd(const CamSet &, const RasterConsts &, int, const float *, const float *, const float *,
                               const float *, float *, float *, float *, int *, int *, float *, cudaStream_t);
cudaError_t launch_project_bwd(const CamSet &, const RasterConsts &, int, const float *, const float *, const float *,
                               const float *, const int *, const float *, const float *, const float *, const float *,
                               float *, float *, float *, float *, float *, cudaStream_t);
cudaError_t launch_sh_fwd(const CamSet &, int, int, const float *, const float *, const int *, float *, const float *,
                          cudaStream_t);
cudaError_t launch_sh_project_bwd(const CamSet &, const RasterConsts &, int, int, const float *, const float *,
                                  const float *, const float *, const float *, const int *, const float *,
                                  const float *, const float *, const float *, float *, float *, float *, float *,
                                  float *, cudaStream_t);
cudaError_t launch_project_sh_fwd(const CamSet &, const RasterConsts &, int, int, const float *, const float *,
                                  const float *, const float *, const float *, float *, float *, float *, int *, int *,
                                  float *, float *, cudaStream_t);
cudaError_t launch_sh_bwd(const CamSet &, int, int, const float *, const float *, const int *, const float *, float *,
                          float *, float *, float *, cudaStream_t);
cudaError_t launch_expected_depth(long long, const float *, int, int, const float *, float *, cudaStream_t);
cudaError_t launch_expected_depth_bwd(long long, const float *, int, int, const float *, const float *, float *,
                                      float *, cudaStream_t);
BinSortLayout binsort_layout(long long CN, long long Kcap, long long T);
cudaError_t launch_binsort(const CamSet &, int, const float *, const float *, const int *, long long,
                           unsigned long long *, int *, int *, long long *, void *, cudaStream_t);
cudaError_t launch_raster_fwd(const CamSet &, const RasterConsts &, int, int, int, const int *, const int *, const int *,
                              const float *, const float *, const float *, const float *, const float *, float *,
                              float *, int *, unsigned long long *, cudaStream_t);
cudaError_t launch_raster_bwd(const CamSet &, const RasterConsts &, int, int, int, const int *, const int *, const int *,
                              const float *, const float *, const float *, const float *, const float *,
                              const float *, const int *, const float *, const float *, float *, float *, float *,
                              float *, float *, cudaStream_t);
cudaError_t launch_probe(int, int, int, float *, double *, cudaStream_t);
cudaError_t launch_tile_order(int, const int *, int *, cudaStream_t);
int raster_channel_capacity(int tile, int ppt, int ch, bool restricted);
size_t raster_fwd_smem(int batch, int chc);
size_t raster_bwd_smem(int batch, int chc, int threads, bool reduce_buffers);
constexpr size_t kMaxSmemPerCta = 227 * 1024;  // opt-in dynamic shared memory of one CTA
int raster_pixels_per_thread(int tile, int ppt);

static std::atomic<unsigned long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

int persistent_grid(const void *kernel, int threads, int smem, int work) {
    struct Entry {
        int dev;
        const void *kernel;
        int smem;
        int ctas;
    };
    static std::mutex mu;
    static Entry table[256];
    static int used = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return work;
    int ctas = 0;
    {
        std::lock_guard<std::mutex> lock(mu);
        for (int i = 0; i < used; ++i)
            if (table[i].dev == dev && table[i].kernel == kernel && table[i].smem == smem) ctas = table[i].ctas;
    }
    if (ctas == 0) {
        int per_sm = 0, sms = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || per_sm <= 0) {
            cudaGetLastError();
            return work;  // fall back to one CTA per work item
        }
        ctas = per_sm * sms;
        std::lock_guard<std::mutex> lock(mu);
        if (used < 256) table[used++] = Entry{dev, kernel, smem, ctas};
    }
    return ctas < work ? ctas : work;
}

cudaError_t ensure_smem(const void *kernel, int bytes) {
    struct Entry {
        int dev;
        const void *kernel;
        int bytes;
    };
    static std::mutex mu;
    static Entry table[256];
    static int used = 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    for (int i = 0; i < used; ++i)
        if (table[i].dev == dev && table[i].kernel == kernel && table[i].bytes >= bytes) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    for (int i = 0; i < used; ++i)
        if (table[i].dev == dev && table[i].kernel == kernel) {
            table[i].bytes = bytes;
            return cudaSuccess;
        }
    if (used < 256) table[used++] = Entry{dev, kernel, bytes};
    return cudaSuccess;
}

}  // namespace gs

using namespace gs;

static thread_local char g_last_error[512] = "";

void gs::set_last_error(const char *text) { snprintf(g_last_error, sizeof(g_last_error), "%s", text); }

static gs_status fail_cuda(cudaError_t e, const char *where) {
    snprintf(g_last_error, sizeof(g_last_error), "%s: %s (%s)", where, cudaGetErrorName(e), cudaGetErrorString(e));
    return GS_ERR_CUDA;
}

static gs_status fail_arg(const char *what) {
    snprintf(g_last_error, sizeof(g_last_error), "invalid argument: %s", what);
    return GS_ERR_ARG;
}

static bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

static gs_status make_camset(const gs_camera *cams, int C, int tile, CamSet &cs) {
    if (!cams) return fail_arg("cams is NULL");
    if (C < 1 || C > GS_MAX_CAMERAS) return fail_arg("C must be in [1, GS_MAX_CAMERAS]");
    if (tile != 8 && tile != 16 && tile != 32) return fail_arg("tile must be 8, 16 or 32");
    memset(&cs, 0, sizeof(cs));
    cs.C = C;
    cs.tile = tile;
    long long tiles = 0, pixels = 0;
    for (int c = 0; c < C; ++c) {
        const gs_camera &g = cams[c];
        if (g.width < 1 || g.height < 1 || g.width > 32768 || g.height > 32768)
            return fail_arg("camera width/height must be in [1, 32768]");
        CamDev &d = cs.cam[c];
        for (int i = 0; i < 3; ++i) {
            for (int j = 0; j < 3; ++j) d.R[3 * i + j] = g.viewmat[4 * i + j];
            d.t[i] = g.viewmat[4 * i + 3];
        }
        d.fx = g.fx;
        d.fy = g.fy;
        d.cx = g.cx;
        d.cy = g.cy;
        d.W = g.width;
        d.H = g.height;
        d.tiles_x = (g.width + tile - 1) / tile;
        d.tiles_y = (g.height + tile - 1) / tile;
        d.tile_offset = (int)tiles;
        d.pix_offset = (int)pixels;
        tiles += (long long)d.tiles_x * d.tiles_y;
        pixels += (long long)g.width * g.height;
        if (tiles >= (1ll << 31) || pixels >= (1ll << 31)) return fail_arg("too many tiles or pixels in one call");
    }
    cs.total_tiles = (int)tiles;
    cs.total_pixels = (int)pixels;
    return GS_OK;
}

static gs_status check_params(const gs_params *p, RasterConsts &rc) {
    if (!p) return fail_arg("params is NULL");
    if (p->tile != 8 && p->tile != 16 && p->tile != 32) return fail_arg("tile must be 8, 16 or 32");
    if (raster_pixels_per_thread(p->tile, p->pixels_per_thread) == 0)
        return fail_arg("pixels_per_thread: 0, or 1 for 8x8 tiles, 1 or 2 for 16x16, 2 or 4 for 32x32");
    if (p->batch_depth < 32 || p->batch_depth > 1024 || (p->batch_depth % 32) != 0)
        return fail_arg("batch_depth must be a multiple of 32 in [32, 1024]");
    if (!(p->alpha_max > 0.f && p->alpha_max < 1.f)) return fail_arg("alpha_max must be in (0, 1)");
    if (!(p->alpha_min >= 0.f && p->alpha_min <= p->alpha_max)) return fail_arg("alpha_min must be in [0, alpha_max]");
    if (!(p->T_min > 0.f && p->T_min < 1.f)) return fail_arg("T_min must be in (0, 1)");
    if (!(p->eps2d >= 0.f)) return fail_arg("eps2d must be >= 0");
    if (!(p->near_plane > 0.f)) return fail_arg("near_plane must be > 0");
    rc.eps2d = p->eps2d;
    rc.near_plane = p->near_plane;
    rc.alpha_min = p->alpha_min;
    rc.alpha_max = p->alpha_max;
    rc.T_min = p->T_min;
    rc.antialiased = p->antialiased ? 1 : 0;
    rc.tile_order = nullptr;
    rc.work = nullptr;
    if (p->persistent != 0 && p->persistent != 1) return fail_arg("persistent must be 0 or 1");
    if (p->colors_shared != 0 && p->colors_shared != 1) return fail_arg("colors_shared must be 0 or 1");
    rc.colors_shared = p->colors_shared;
    return GS_OK;
}

static gs_status check_cn(int C, int N) {
    if (N < 0) return fail_arg("N must be >= 0");
    if ((long long)C * N >= (1ll << 31)) return fail_arg("C * N must be < 2^31");
    return GS_OK;
}

#define GS_TRY(x)                         \
    do {                                  \
        gs_status _s = (x);               \
        if (_s != GS_OK) return _s;       \
    } while (0)
#define GS_NONNULL(p)                              \
    do {                                           \
        if (!(p)) return fail_arg(#p " is NULL");  \
    } while (0)

extern "C" {

void gs_default_params(gs_params *p) {
    if (!p) return;
    p->tile = 16;
    p->batch_depth = 256;
    p->antialiased = 0;
    p->pixels_per_thread = 0;
    p->persistent = 0;
    p->colors_shared = 0;
    p->eps2d = 0.3f;
    p->near_plane = 0.01f;
    p->alpha_min = 1.f / 255.f;
    p->alpha_max = 0.99f;
    p->T_min = 1e-4f;
}

const char *gs_status_string(gs_status s) {
    switch (s) {
        case GS_OK: return "GS_OK";
        case GS_ERR_ARG: return "GS_ERR_ARG";
        case GS_ERR_CUDA: return "GS_ERR_CUDA";
        case GS_ERR_CAPACITY: return "GS_ERR_CAPACITY";
        case GS_ERR_UNSUPPORTED: return "GS_ERR_UNSUPPORTED";
        default: return "GS_ERR_UNKNOWN";
    }
}

const char *gs_last_error(void) { return g_last_error; }

uint64_t gs_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

int64_t gs_num_tiles(const gs_camera *cams, int32_t C, int32_t tile) {
    CamSet cs;
    if (make_camset(cams, C, tile, cs) != GS_OK) return -1;
    return cs.total_tiles;
}

gs_status gs_probe_peak(int32_t kind, int32_t blocks, int32_t iters, float *sink, double *ops, void *stream) {
    if (kind != 0 && kind != 1) return fail_arg("probe kind must be 0 (FFMA) or 1 (EX2)");
    if (blocks < 1 || iters < 1 || iters > (1 << 24)) return fail_arg("probe blocks >= 1, iters in [1, 2^24]");
    if (!sink || !ops) return fail_arg("probe sink and ops must be non-null");
    cudaError_t e = launch_probe(kind, blocks, iters, sink, ops, (cudaStream_t)stream);
    return e == cudaSuccess ? GS_OK : fail_cuda(e, "gs_probe_peak");
}

int64_t gs_num_pixels(const gs_camera *cams, int32_t C) {
    CamSet cs;
    if (make_camset(cams, C, 16, cs) != GS_OK) return -1;
    return cs.total_pixels;
}

gs_status gs_project(const gs_camera *cams, int32_t C, int32_t N, const float *means, const float *quats,
                     const float *log_scales, const float *opacity_logits, const gs_params *params, float *means2d,
                     float *depths, float *conics, int32_t *radii, int32_t *tiles_touched, float *opacities,
                     void *stream) {
    RasterConsts rc;
    CamSet cs;
    GS_TRY(check_params(params, rc));
    GS_TRY(make_camset(cams, C, params->tile, cs));
    GS_TRY(check_cn(C, N));
    cs.N = N;
    if (N == 0) return GS_OK;
    GS_NONNULL(means); GS_NONNULL(quats); GS_NONNULL(log_scales); GS_NONNULL(opacity_logits);
    GS_NONNULL(means2d); GS_NONNULL(depths); GS_NONNULL(conics); GS_NONNULL(radii); GS_NONNULL(tiles_touched);
    GS_NONNULL(opacities);
    if (!aligned(quats, 16)) return fail_arg("quats must be 16-byte aligned");
    if (!aligned(means2d, 8)) return fail_arg("means2d must be 8-byte aligned");
    cudaError_t e = launch_project_fwd(cs, rc, N, means, quats, log_scales, opacity_logits, means2d, depths, conics,
                                       radii, tiles_touched, opacities, (cudaStream_t)stream);
    return e == cudaSuccess ? GS_OK : fail_cuda(e, "gs_project");
}

gs_status gs_project_sh_eval(const gs_camera *cams, int32_t C, int32_t N, const gs_params *params,
                             int32_t sh_degree, const float *sh, const float *means, const float *quats,
                             const float *log_scales, const float *opacity_logits, float *means2d, float *depths,
                             float *conics, int32_t *radii, int32_t *tiles_touched, float *opacities, float *colors,
                             void *stream) {
    RasterConsts rc;
    CamSet cs;
    GS_TRY(check_params(params, rc));
    GS_TRY(make_camset(cams, C, params->tile, cs));
    GS_TRY(check_cn(C, N));
    cs.N = N;
    if (sh_degree < 0 || sh_degree > 3) return fail_arg("sh_degree must be in [0, 3]");
    if (N == 0) return GS_OK;
    GS_NONNULL(sh); GS_NONNULL(means); GS_NONNULL(quats); GS_NONNULL(log_scales); GS_NONNULL(opacity_logits);
    GS_NONNULL(means2d); GS_NONNULL(depths); GS_NONNULL(conics); GS_NONNULL(radii); GS_NONNULL(tiles_touched);
    GS_NONNULL(opacities); GS_NONNULL(colors);
    if (!aligned(quats, 16)) return fail_arg("quats must be 16-byte aligned");
    if (!aligned(means2d, 8)) return fail_arg("means2d must be 8-byte aligned");
    cudaError_t e = launch_project_sh_fwd(cs, rc, sh_degree, N, sh, means, quats, log_scales, opacity_logits, means2d,
                                          depths, conics, radii, tiles_touched, opacities, colors,
                                          (cudaStream_t)stream);
    return e == cudaSuccess ? GS_OK : fail_cuda(e, "gs_project_sh_eval");
}

gs_status gs_sh_eval(const gs_camera *cams, int32_t C, int32_t N, int32_t sh_degree, const float *sh,
                     const float *means, const int32_t *radii, float *colors, void *stream) {
    CamSet cs;
    GS_TRY(make_camset(cams, C, 16, cs));
    GS_TRY(check_cn(C, N));
    cs.N = N;
    if (sh_degree < 0 || sh_degree > 3) return fail_arg("sh_degree must be in [0, 3]");
    if (N == 0) return GS_OK;
    GS_NONNULL(sh); GS_NONNULL(means); GS_NONNULL(radii); GS_NONNULL(colors);
    cudaError_t e = launch_sh_fwd(cs, sh_degree, N, sh, means, radii, colors, nullptr, (cudaStream_t)stream);
    return e == cudaSuccess ? GS_OK : fail_cuda(e, "gs_sh_eval");
}

gs_status gs_sh_eval_depth(const gs_camera *cams, int32_t C, int32_t N, int32_t sh_degree, const float *sh,
                           const float *means, const int32_t *radii, const float *depths, float *colors_rgbd,
                           void *stream) {
    CamSet cs;
    GS_TRY(make_camset(cams, C, 16, cs));
    GS_TRY(check_cn(C, N));
    cs.N = N;
    if (sh_degree < 0 || sh_degree > 3) return fail_arg("sh_degree must be in [0, 3]");
    if (N == 0) return GS_OK;
    GS_NONNULL(sh); GS_NONNULL(means); GS_NONNULL(radii); GS_NONNULL(depths); GS_NONNULL(colors_rgbd);
    cudaError_t e = launch_sh_fwd(cs, sh_degree, N, sh, means, radii, colors_rgbd, depths, (cudaStream_t)stream);
    return e == cudaSuccess ? GS_OK : fail_cuda(e, "gs_sh_eval_depth");
}

gs_status gs_expected_depth(int64_t P, const float *image, int32_t channels, int32_t depth_channel,
                            const float *final_T, float *expected_depth, void *stream) {
    if (P < 0) return fail_arg("P must be >= 0");
    if (channels < 1 || depth_channel < 0 || depth_channel >= channels)
        return fail_arg("depth_channel must be in [0, channels)");
    if (P == 0) return GS_OK;
    GS_NONNULL(image); GS_NONNULL(final_T); GS_NONNULL(expected_depth);
    cudaError_t e = launch_expected_depth(P, image, channels, depth_channel, final_T, expected_depth,
                                          (cudaStream_t)stream);
    return e == cudaSuccess ? GS_OK : fail_cuda(e, "gs_expected_depth");
}

gs_status gs_expected_depth_bwd(int64_t P, const float *image, int32_t channels, int32_t depth_channel,
                                const float *final_T, const float *d_expected_depth, float *d_image, float *d_alpha,
                                void *stream) {
    if (P < 0) return fail_arg("P must be >= 0");
    if (channels < 1 || depth_channel < 0 || depth_channel >= channels)
        return fail_arg("depth_channel must be in [0, channels)");
    if (P == 0) return GS_OK;
    GS_NONNULL(image); GS_NONNULL(final_T); GS_NONNULL(d_expected_depth); GS_NONNULL(d_image); GS_NONNULL(d_alpha);
    cudaError_t e = launch_expected_depth_bwd(P, image, channels, depth_channel, final_T, d_expected_depth, d_image,
                                              d_alpha, (cudaStream_t)stream);
    return e == cudaSuccess ? GS_OK : fail_cuda(e, "gs_expected_depth_bwd");
}

int64_t gs_tile_bin_sort_workspace(const gs_camera *cams, int32_t C, int32_t N, const gs_params *params,
                                   int64_t K_capacity) {
    CamSet cs;
    if (!params || make_camset(cams, C, params->tile, cs) != GS_OK) return -1;
    if (N < 0 || K_capacity < 0 || K_capacity > GS_MAX_INTERSECTIONS || (long long)C * N >= (1ll << 31)) return -1;
    return (int64_t)binsort_layout((long long)C * N, K_capacity, cs.total_tiles).total;
}

gs_status gs_tile_bin_sort(const gs_camera *cams, int32_t C, int32_t N, const gs_params *params,
                           const float *means2d, const float *depths, const int32_t *radii, int64_t K_capacity,
                           uint64_t *keys, int32_t *values, int32_t *tile_ranges, int64_t *K_out, void *workspace,
                           size_t workspace_bytes, void *stream) {
    RasterConsts rc;
    CamSet cs;
    GS_TRY(check_params(params, rc));
    GS_TRY(make_camset(cams, C, params->tile, cs));
    GS_TRY(check_cn(C, N));
    cs.N = N;
    if (K_capacity < 0) return fail_arg("K_capacity must be >= 0");
    if (K_capacity > GS_MAX_INTERSECTIONS) {
        snprintf(g_last_error, sizeof(g_last_error),
                 "K_capacity %lld exceeds GS_MAX_INTERSECTIONS (2^31 - 1): list positions are int32; "
                 "render fewer cameras per call or use a larger tile",
                 (long long)K_capacity);
        return GS_ERR_CAPACITY;
    }
    if (cs.total_tiles >= (1 << 28)) return fail_arg("more than 2^28 tiles in one call");
    GS_NONNULL(tile_ranges); GS_NONNULL(K_out); GS_NONNULL(workspace);
    if (N > 0) {
        GS_NONNULL(means2d); GS_NONNULL(depths); GS_NONNULL(radii);
    }
    if (K_capacity > 0) GS_NONNULL(values);
    if (!aligned(workspace, 256)) return fail_arg("workspace must be 256-byte aligned");
    if (values && !aligned(values, 16)) return fail_arg("values must be 16-byte aligned");
    if (N > 0 && !aligned(means2d, 8)) return fail_arg("means2d must be 8-byte aligned");
    if (!aligned(tile_ranges, 8)) return fail_arg("tile_ranges must be 8-byte aligned");
    if (keys && !aligned(keys, 8)) return fail_arg("keys must be 8-byte aligned");
    size_t need = binsort_layout((long long)C * N, K_capacity, cs.total_tiles).total;
    if (workspace_bytes < need) {
        snprintf(g_last_error, sizeof(g_last_error), "workspace too small: %zu < %zu bytes", workspace_bytes, need);
        return GS_ERR_CAPACITY;
    }
    cudaError_t e = launch_binsort(cs, N, means2d, depths, radii, K_capacity, (unsigned long long *)keys, values,
                                   tile_ranges, (long long *)K_out, workspace, (cudaStream_t)stream);
    return e == cudaSuccess ? GS_OK : fail_cuda(e, "gs_tile_bin_sort");
}

gs_status gs_tile_order(const gs_camera *cams, int32_t C, const gs_params *params, const int32_t *tile_ranges,
                        int32_t *tile_order, void *stream) {
    RasterConsts rc;
    CamSet cs;
    GS_TRY(check_params(params, rc));
    GS_TRY(make_camset(cams, C, params->tile, cs));
    GS_NONNULL(tile_ranges); GS_NONNULL(tile_order);
    if (!aligned(tile_ranges, 8)) return fail_arg("tile_ranges must be 8-byte aligned");
    cudaError_t e = launch_tile_order(cs.total_tiles, tile_ranges, tile_order, (cudaStream_t)stream);
    return e == cudaSuccess ? GS_OK : fail_cuda(e, "gs_tile_order");
}

gs_status gs_rasterize_fwd(const gs_camera *cams, int32_t C, int32_t N, const gs_params *params, int32_t channels,
                           const int32_t *tile_ranges, const int32_t *values, const int32_t *radii,
                           const float *means2d, const float *conics, const float *opacities, const float *colors,
                           const float *background, float *image, float *final_T, int32_t *last_contrib,
                           int64_t *blend_count, const int32_t *tile_order, void *stream) {
    RasterConsts rc;
    CamSet cs;
    GS_TRY(check_params(params, rc));
    GS_TRY(make_camset(cams, C, params->tile, cs));
    GS_TRY(check_cn(C, N));
    cs.N = N;
    if (channels < 1 || channels > GS_MAX_CHANNELS) return fail_arg("channels must be in [1, GS_MAX_CHANNELS]");
    const int ppt = raster_pixels_per_thread(params->tile, params->pixels_per_thread);
    if (raster_channel_capacity(params->tile, ppt, channels, blend_count != nullptr) == 0) {
        snprintf(g_last_error, sizeof(g_last_error), "no kernel for tile %d with %d channels%s", params->tile,
                 channels, blend_count ? " and blend counting" : "");
        return GS_ERR_UNSUPPORTED;
    }
    {
        const size_t need = raster_fwd_smem(params->batch_depth,
                                            raster_channel_capacity(params->tile, ppt, channels, blend_count != nullptr));
        if (need > kMaxSmemPerCta) {
            snprintf(g_last_error, sizeof(g_last_error),
                     "batch_depth %d with %d channels needs %zu bytes of shared memory per CTA (at most %zu)",
                     params->batch_depth, channels, need, kMaxSmemPerCta);
            return GS_ERR_UNSUPPORTED;
        }
    }
    GS_NONNULL(tile_ranges); GS_NONNULL(image); GS_NONNULL(final_T); GS_NONNULL(last_contrib);
    if (N > 0) {
        GS_NONNULL(values); GS_NONNULL(radii); GS_NONNULL(means2d); GS_NONNULL(conics); GS_NONNULL(opacities);
        GS_NONNULL(colors);
        if (!aligned(means2d, 8)) return fail_arg("means2d must be 8-byte aligned");
    }
    if (!aligned(tile_ranges, 8)) return fail_arg("tile_ranges must be 8-byte aligned");
    if (blend_count && !aligned(blend_count, 8)) return fail_arg("blend_count must be 8-byte aligned");
    rc.tile_order = tile_order;
    if (params->persistent) {
        if (!tile_order) return fail_arg("a persistent launch needs the tile_order of gs_tile_order");
        rc.work = const_cast<int32_t *>(tile_order) + cs.total_tiles;  // counters 0, 1
    }
    cudaError_t e = launch_raster_fwd(cs, rc, channels, params->batch_depth, ppt, tile_ranges, values, radii, means2d,
                                      conics, opacities, colors, background, image, final_T, last_contrib,
                                      (unsigned long long *)blend_count, (cudaStream_t)stream);
    return e == cudaSuccess ? GS_OK : fail_cuda(e, "gs_rasterize_fwd");
}

gs_status gs_rasterize_bwd(const gs_camera *cams, int32_t C, int32_t N, const gs_params *params, int32_t channels,
                           const int32_t *tile_ranges, const int32_t *values, const int32_t *radii,
                           const float *means2d, const float *conics, const float *opacities, const float *colors,
                           const float *background, const float *final_T, const int32_t *last_contrib,
                           const float *d_image, const float *d_alpha, float *d_means2d, float *d_conics,
                           float *d_opacities, float *d_colors, float *absgrad, const int32_t *tile_order,
                           void *stream) {
    RasterConsts rc;
    CamSet cs;
    GS_TRY(check_params(params, rc));
    GS_TRY(make_camset(cams, C, params->tile, cs));
    GS_TRY(check_cn(C, N));
    cs.N = N;
    if (channels < 1 || channels > GS_MAX_CHANNELS) return fail_arg("channels must be in [1, GS_MAX_CHANNELS]");
    const int ppt = raster_pixels_per_thread(params->tile, params->pixels_per_thread);
    if (raster_channel_capacity(params->tile, ppt, channels, absgrad != nullptr) == 0) {
        snprintf(g_last_error, sizeof(g_last_error), "no backward kernel for tile %d with %d channels%s",
                 params->tile, channels, absgrad ? " and absgrad" : "");
        return GS_ERR_UNSUPPORTED;
    }
    {
        const size_t need = raster_bwd_smem(params->batch_depth,
                                            raster_channel_capacity(params->tile, ppt, channels, absgrad != nullptr),
                                            params->tile * params->tile / ppt, ppt <= 2);
        if (need > kMaxSmemPerCta) {
            snprintf(g_last_error, sizeof(g_last_error),
                     "batch_depth %d with %d channels needs %zu bytes of shared memory per CTA (at most %zu)",
                     params->batch_depth, channels, need, kMaxSmemPerCta);
            return GS_ERR_UNSUPPORTED;
        }
    }
    if (N == 0) return GS_OK;
    GS_NONNULL(tile_ranges); GS_NONNULL(values); GS_NONNULL(radii); GS_NONNULL(means2d); GS_NONNULL(conics);
    GS_NONNULL(opacities); GS_NONNULL(colors); GS_NONNULL(final_T); GS_NONNULL(last_contrib); GS_NONNULL(d_image);
    GS_NONNULL(d_means2d); GS_NONNULL(d_conics); GS_NONNULL(d_opacities); GS_NONNULL(d_colors);
    if (!aligned(means2d, 8) || !aligned(d_means2d, 8)) return fail_arg("means2d/d_means2d must be 8-byte aligned");
    if (absgrad && !aligned(absgrad, 8)) return fail_arg("absgrad must be 8-byte aligned");
    if (!aligned(tile_ranges, 8)) return fail_arg("tile_ranges must be 8-byte aligned");
    rc.tile_order = tile_order;
    if (params->persistent) {
        if (!tile_order) return fail_arg("a persistent launch needs the tile_order of gs_tile_order");
        rc.work = const_cast<int32_t *>(tile_order) + cs.total_tiles + 2;  // counters 2, 3
    }
    cudaError_t e = launch_raster_bwd(cs, rc, channels, params->batch_depth, ppt, tile_ranges, values, radii, means2d,
                                      conics, opacities, colors, background, final_T, last_contrib, d_image, d_alpha,
                                      d_means2d, d_conics, d_opacities, d_colors, absgrad, (cudaStream_t)stream);
    return e == cudaSuccess ? GS_OK : fail_cuda(e, "gs_rasterize_bwd");
}

gs_status gs_sh_eval_bwd(const gs_camera *cams, int32_t C, int32_t N, int32_t sh_degree, const float *sh,
                         const float *means, const int32_t *radii, const float *d_colors, float *d_sh,
                         float *d_means, float *d_viewmats, void *stream) {
    CamSet cs;
    GS_TRY(make_camset(cams, C, 16, cs));
    GS_TRY(check_cn(C, N));
    cs.N = N;
    if (sh_degree < 0 || sh_degree > 3) return fail_arg("sh_degree must be in [0, 3]");
    if (N == 0) return GS_OK;
    GS_NONNULL(sh); GS_NONNULL(means); GS_NONNULL(radii); GS_NONNULL(d_colors); GS_NONNULL(d_sh);
    GS_NONNULL(d_means);
    cudaError_t e =
        launch_sh_bwd(cs, sh_degree, N, sh, means, radii, d_colors, d_sh, d_means, nullptr, d_viewmats,
                      (cudaStream_t)stream);
    return e == cudaSuccess ? GS_OK : fail_cuda(e, "gs_sh_eval_bwd");
}

gs_status gs_sh_eval_depth_bwd(const gs_camera *cams, int32_t C, int32_t N, int32_t sh_degree, const float *sh,
                               const float *means, const int32_t *radii, const float *d_colors_rgbd, float *d_sh,
                               float *d_means, float *d_depths, float *d_viewmats, void *stream) {
    CamSet cs;
    GS_TRY(make_camset(cams, C, 16, cs));
    GS_TRY(check_cn(C, N));
    cs.N = N;
    if (sh_degree < 0 || sh_degree > 3) return fail_arg("sh_degree must be in [0, 3]");
    if (N == 0) return GS_OK;
    GS_NONNULL(sh); GS_NONNULL(means); GS_NONNULL(radii); GS_NONNULL(d_colors_rgbd); GS_NONNULL(d_sh);
    GS_NONNULL(d_means); GS_NONNULL(d_depths);
    cudaError_t e = launch_sh_bwd(cs, sh_degree, N, sh, means, radii, d_colors_rgbd, d_sh, d_means, d_depths,
                                  d_viewmats, (cudaStream_t)stream);
    return e == cudaSuccess ? GS_OK : fail_cuda(e, "gs_sh_eval_depth_bwd");
}

gs_status gs_project_bwd(const gs_camera *cams, int32_t C, int32_t N, const float *means, const float *quats,
                         const float *log_scales, const float *opacity_logits, const gs_params *params,
                         const int32_t *radii, const float *d_means2d, const float *d_conics, const float *d_opacities,
                         const float *d_depths, float *d_means, float *d_quats, float *d_log_scales,
                         float *d_opacity_logits, float *d_viewmats,
                         void *stream) {
    RasterConsts rc;
    CamSet cs;
    GS_TRY(check_params(params, rc));
    GS_TRY(make_camset(cams, C, params->tile, cs));
    GS_TRY(check_cn(C, N));
    cs.N = N;
    if (N == 0) return GS_OK;
    GS_NONNULL(means); GS_NONNULL(quats); GS_NONNULL(log_scales); GS_NONNULL(opacity_logits); GS_NONNULL(radii);
    GS_NONNULL(d_means2d); GS_NONNULL(d_conics); GS_NONNULL(d_opacities); GS_NONNULL(d_means); GS_NONNULL(d_quats);
    GS_NONNULL(d_log_scales); GS_NONNULL(d_opacity_logits);
    if (!aligned(quats, 16) || !aligned(d_quats, 16)) return fail_arg("quats/d_quats must be 16-byte aligned");
    if (!aligned(d_means2d, 8)) return fail_arg("d_means2d must be 8-byte aligned");
    cudaError_t e = launch_project_bwd(cs, rc, N, means, quats, log_scales, opacity_logits, radii, d_means2d, d_conics,
                                       d_opacities, d_depths, d_means, d_quats, d_log_scales, d_opacity_logits,
                                       d_viewmats, (cudaStream_t)stream);
    return e == cudaSuccess ? GS_OK : fail_cuda(e, "gs_project_bwd");
}

gs_status gs_sh_project_bwd(const gs_camera *cams, int32_t C, int32_t N, const gs_params *params, int32_t sh_degree,
                            const float *sh, const float *means, const float *quats, const float *log_scales,
                            const float *opacity_logits, const int32_t *radii, const float *d_colors,
                            const float *d_means2d, const float *d_conics, const float *d_opacities, float *d_sh,
                            float *d_means, float *d_quats, float *d_log_scales, float *d_opacity_logits,
                            void *stream) {
    RasterConsts rc;
    CamSet cs;
    GS_TRY(check_params(params, rc));
    GS_TRY(make_camset(cams, C, params->tile, cs));
    GS_TRY(check_cn(C, N));
    cs.N = N;
    if (C != 1) return fail_arg("gs_sh_project_bwd takes one camera (use gs_sh_eval_bwd + gs_project_bwd)");
    if (sh_degree < 0 || sh_degree > 3) return fail_arg("sh_degree must be in [0, 3]");
    if (N == 0) return GS_OK;
    GS_NONNULL(sh); GS_NONNULL(means); GS_NONNULL(quats); GS_NONNULL(log_scales); GS_NONNULL(opacity_logits);
    GS_NONNULL(radii); GS_NONNULL(d_colors); GS_NONNULL(d_means2d); GS_NONNULL(d_conics); GS_NONNULL(d_opacities);
    GS_NONNULL(d_sh); GS_NONNULL(d_means); GS_NONNULL(d_quats); GS_NONNULL(d_log_scales);
    GS_NONNULL(d_opacity_logits);
    if (!aligned(quats, 16) || !aligned(d_quats, 16)) return fail_arg("quats/d_quats must be 16-byte aligned");
    if (!aligned(d_means2d, 8)) return fail_arg("d_means2d must be 8-byte aligned");
    cudaError_t e = launch_sh_project_bwd(cs, rc, sh_degree, N, sh, means, quats, log_scales, opacity_logits, radii,
                                          d_colors, d_means2d, d_conics, d_opacities, d_sh, d_means, d_quats,
                                          d_log_scales, d_opacity_logits, (cudaStream_t)stream);
    return e == cudaSuccess ? GS_OK : fail_cuda(e, "gs_sh_project_bwd");
}

}  // extern "C"
