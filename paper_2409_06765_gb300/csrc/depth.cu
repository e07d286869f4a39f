// Depth rendering (App. A): the accumulated depth sum_n z_n alpha_n T_n is the compositing
// sum of a fourth feature channel that carries each Gaussian's camera-space depth (written
// by the SH kernel), so it needs no kernel of its own.  The expected depth divides it by the
// accumulated opacity sum_n alpha_n T_n = 1 - T_final; this file holds that division and its
// backward, one thread per pixel.
#include "gs_internal.cuh"

namespace gs {

__global__ void expected_depth_kernel(long long P, const float *__restrict__ image, int channels, int depth_ch,
                                      const float *__restrict__ final_T, float *__restrict__ out) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
        const float a = 1.f - final_T[p];
        out[p] = a > 0.f ? image[p * channels + depth_ch] / a : 0.f;
    }
}

// E = A / a:  dA += dE / a,  da += -dE A / a^2 = -dE E / a  (zero where a = 0).
__global__ void expected_depth_bwd_kernel(long long P, const float *__restrict__ image, int channels, int depth_ch,
                                          const float *__restrict__ final_T, const float *__restrict__ d_expected,
                                          float *__restrict__ d_image, float *__restrict__ d_alpha) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
        const float a = 1.f - final_T[p];
        if (!(a > 0.f)) continue;
        const float ia = 1.f / a;
        const float g = d_expected[p];
        const float E = image[p * channels + depth_ch] * ia;
        d_image[p * channels + depth_ch] += g * ia;
        d_alpha[p] += -g * E * ia;
    }
}

static unsigned grid_for(long long P) {
    const long long b = (P + 255) / 256;
    return (unsigned)(b < 65536 ? (b > 0 ? b : 1) : 65536);
}

cudaError_t launch_expected_depth(long long P, const float *image, int channels, int depth_ch, const float *final_T,
                                  float *out, cudaStream_t st) {
    if (P <= 0) return cudaSuccess;
    expected_depth_kernel<<<grid_for(P), 256, 0, st>>>(P, image, channels, depth_ch, final_T, out);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_expected_depth_bwd(long long P, const float *image, int channels, int depth_ch,
                                      const float *final_T, const float *d_expected, float *d_image, float *d_alpha,
                                      cudaStream_t st) {
    if (P <= 0) return cudaSuccess;
    expected_depth_bwd_kernel<<<grid_for(P), 256, 0, st>>>(P, image, channels, depth_ch, final_T, d_expected,
                                                           d_image, d_alpha);
    note_launch();
    return cudaGetLastError();
}

}  // namespace gs
