// gs_probe_peak: throughput microbenchmarks that give the compositing kernels a measured
// roofline.  The compositing arithmetic runs on the FP32 pipe (FFMA/FMUL/FADD/FMNMX, one
// lane operation per thread per instruction) and on the special-function unit (ex2 and
// rcp approximations), so the two ceilings are a stream of independent FFMAs and a
// stream of independent ex2.approx operations, each run over the whole GPU.
//
// Every thread keeps 8 independent dependency chains so that the pipe, not the latency
// of one chain, limits the rate; the chains' sum is stored (to a sink the caller owns)
// only when it equals an impossible value, so the compiler keeps the work and the stores
// never happen.
#include "gs_internal.cuh"

namespace gs {

constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 8;
constexpr int kProbeUnroll = 16;

__global__ void __launch_bounds__(kProbeThreads) probe_ffma_kernel(int iters, float a, float b,
                                                                   float *__restrict__ sink) {
    float x[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kProbeUnroll; ++u) {
#pragma unroll
            for (int c = 0; c < kProbeChains; ++c) x[c] = __fmaf_rn(x[c], a, b);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) s += x[c];
    if (s == -1.2345f) sink[0] = s;
}

__global__ void __launch_bounds__(kProbeThreads) probe_ex2_kernel(int iters, float a, float b,
                                                                  float *__restrict__ sink) {
    float x[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) x[c] = -(float)(threadIdx.x + c) * 1e-3f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kProbeUnroll; ++u) {
#pragma unroll
            for (int c = 0; c < kProbeChains; ++c) x[c] = ex2_approx(x[c]);  // stays in (0, 1]
        }
    }
    float s = a * b;
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) s += x[c];
    if (s == -1.2345f) sink[0] = s;
}

cudaError_t launch_probe(int kind, int blocks, int iters, float *sink, double *ops, cudaStream_t st) {
    const double per_thread = (double)iters * kProbeUnroll * kProbeChains;
    *ops = per_thread * (double)blocks * kProbeThreads;
    if (kind == 0)
        probe_ffma_kernel<<<blocks, kProbeThreads, 0, st>>>(iters, 0.999f, 1e-3f, sink);
    else
        probe_ex2_kernel<<<blocks, kProbeThreads, 0, st>>>(iters, 1.f, 0.f, sink);
    note_launch();
    return cudaGetLastError();
}

}  // namespace gs
