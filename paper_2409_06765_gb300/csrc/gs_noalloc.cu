// gs_tile_bin_sort_noalloc: the tile binning + depth sort of gs_tile_bin_sort, with its
// scratch memory taken from a fixed array compiled into this library instead of a
// caller-provided workspace.
//
// Who needs it: callers that cannot call cudaMalloc or any other allocator, for example
// a plug-in inside a host application whose own allocator owns every byte of device
// memory, a real-time render loop that must not hit the device-wide synchronisation an
// allocation or free can imply, or a thin language binding that has no device allocator
// at all.  They still own every input and output buffer; only the sort's scratch lives
// here.
//
// The array (GS_NOALLOC_SCRATCH_BYTES) is reserved on every GPU that loads this library
// and stays reserved until the process exits.  All calls share it: two calls whose work
// overlaps on the GPU (different streams, or different host threads on one device)
// race on it and corrupt each other's result, so serialise them.  It keeps whatever the
// last call left in it; the sort writes every scratch word before reading it, so
// nothing has to be cleared between calls.
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "gs_internal.cuh"

using gs::set_last_error;

static __device__ __align__(256) unsigned char g_sort_scratch[GS_NOALLOC_SCRATCH_BYTES];

// Device address of g_sort_scratch on the current device, looked up once per device.  In
// host code the symbol names a host-side shadow, never the device memory, so it is only
// ever used through this address.
static void *scratch_address(cudaError_t *err) {
    static std::mutex mu;
    static void *addr[64] = {nullptr};
    int dev = 0;
    *err = cudaGetDevice(&dev);
    if (*err != cudaSuccess) return nullptr;
    if (dev < 0 || dev >= 64) {
        *err = cudaErrorInvalidDevice;
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        *err = cudaGetSymbolAddress(&p, g_sort_scratch);
        if (*err != cudaSuccess) return nullptr;
        addr[dev] = p;
    }
    return addr[dev];
}

extern "C" GS_API gs_status gs_tile_bin_sort_noalloc(const gs_camera *cams, int32_t C, int32_t N,
                                                     const gs_params *params, const float *means2d,
                                                     const float *depths, const int32_t *radii, int64_t K_capacity,
                                                     uint64_t *keys, int32_t *values, int32_t *tile_ranges,
                                                     int64_t *K_out, void *stream) {
    if (!params || !cams || !tile_ranges || !K_out) return GS_ERR_ARG;
    if (C < 1 || C > GS_MAX_CAMERAS || N < 0 || (long long)C * N >= (1ll << 31)) return GS_ERR_ARG;
    if (K_capacity < 0) return GS_ERR_ARG;
    if (K_capacity > GS_MAX_INTERSECTIONS) return GS_ERR_CAPACITY;
    // the scratch this call would need, checked before anything is launched
    const int64_t need = gs_tile_bin_sort_workspace(cams, C, N, params, K_capacity);
    if (need < 0) return GS_ERR_ARG;
    char msg[256];
    if (need > (int64_t)GS_NOALLOC_SCRATCH_BYTES) {
        snprintf(msg, sizeof(msg),
                 "gs_tile_bin_sort_noalloc: these sizes need %lld bytes of scratch, the built-in array holds %lld",
                 (long long)need, (long long)GS_NOALLOC_SCRATCH_BYTES);
        set_last_error(msg);
        return GS_ERR_CAPACITY;
    }
    cudaError_t err;
    void *ws = scratch_address(&err);
    if (!ws) {
        snprintf(msg, sizeof(msg), "gs_tile_bin_sort_noalloc: cudaGetSymbolAddress failed: %s",
                 cudaGetErrorString(err));
        set_last_error(msg);
        return GS_ERR_CUDA;
    }
    // everything else (validation, launches) is the regular entry point with this workspace
    return gs_tile_bin_sort(cams, C, N, params, means2d, depths, radii, K_capacity, keys, values, tile_ranges, K_out,
                            ws, (size_t)GS_NOALLOC_SCRATCH_BYTES, stream);
}
