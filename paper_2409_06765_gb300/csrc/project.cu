// Projection of 3D Gaussians to 2D splats and its backward (App. C.1, App. D.3-D.4,
// App. E, App. A anti-aliasing).  One thread per Gaussian; each thread loops over
// the cameras of the call so the Gaussian's 44 bytes of parameters are read once.
#include "project_math.cuh"

namespace gs {

__global__ void __launch_bounds__(256) project_fwd_kernel(
    int N, const float *__restrict__ means, const float4 *__restrict__ quats, const float *__restrict__ log_scales,
    const float *__restrict__ logits, const __grid_constant__ CamSet cs, RasterConsts rc, float2 *__restrict__ means2d,
    float *__restrict__ depths, float *__restrict__ conics, int *__restrict__ radii, int *__restrict__ tiles_touched,
    float *__restrict__ opac) {
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    Gauss3 g;
    load_gauss(n, log_scales, quats, logits, g);
    float mean[3] = {means[3 * n], means[3 * n + 1], means[3 * n + 2]};
    const int tile = cs.tile;
    for (int c = 0; c < cs.C; ++c) {
        const CamDev &cam = cs.cam[c];
        size_t idx = (size_t)c * N + n;
        Splat2 sp;
        bool ok = splat_of(g, mean, cam, rc, sp);
        int r = ok ? radius_of(sp) : 0;
        int x0 = 0, x1 = -1, y0 = 0, y1 = -1;
        if (r > 0 && !pixel_box(sp.mx, sp.my, r, cam.W, cam.H, x0, x1, y0, y1)) r = 0;
        if (r == 0) {
            means2d[idx] = make_float2(0.f, 0.f);
            depths[idx] = 0.f;
            conics[3 * idx] = 0.f;
            conics[3 * idx + 1] = 0.f;
            conics[3 * idx + 2] = 0.f;
            radii[idx] = 0;
            tiles_touched[idx] = 0;
            opac[idx] = 0.f;
            continue;
        }
        means2d[idx] = make_float2(sp.mx, sp.my);
        depths[idx] = sp.t[2];
        conics[3 * idx] = sp.conic[0];
        conics[3 * idx + 1] = sp.conic[1];
        conics[3 * idx + 2] = sp.conic[2];
        radii[idx] = r;
        tiles_touched[idx] = (x1 / tile - x0 / tile + 1) * (y1 / tile - y0 / tile + 1);
        opac[idx] = g.o * sp.comp;
    }
}

#ifndef GS_PROJECT_BWD_MIN_BLOCKS
#define GS_PROJECT_BWD_MIN_BLOCKS 3  // 80 registers: the one-camera-ahead loads fit without much spilling
#endif
__global__ void __launch_bounds__(256, GS_PROJECT_BWD_MIN_BLOCKS) project_bwd_kernel(
    int N, const float *__restrict__ means, const float4 *__restrict__ quats, const float *__restrict__ log_scales,
    const float *__restrict__ logits, const __grid_constant__ CamSet cs, RasterConsts rc,
    const int *__restrict__ radii, const float2 *__restrict__ d_means2d, const float *__restrict__ d_conics,
    const float *__restrict__ d_opac, const float *__restrict__ d_depths, float *__restrict__ d_means,
    float4 *__restrict__ d_quats, float *__restrict__ d_log_scales, float *__restrict__ d_logits,
    float *__restrict__ d_viewmats) {
    __shared__ float s_red[8 * 12];
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = n < N;
    // every load of this Gaussian that does not depend on another is issued up front, so the
    // radii, the parameters and the d_means read-modify-write overlap instead of chaining
    Gauss3 g;
    float mean[3] = {0.f, 0.f, 0.f};
    float dm_in[3] = {0.f, 0.f, 0.f};
    if (valid) {
        mean[0] = means[3 * n];
        mean[1] = means[3 * n + 1];
        mean[2] = means[3 * n + 2];
        dm_in[0] = d_means[3 * n];
        dm_in[1] = d_means[3 * n + 1];
        dm_in[2] = d_means[3 * n + 2];
        load_gauss(n, log_scales, quats, logits, g);
    }
    bool any = false;
    if (valid)
        for (int c = 0; c < cs.C; ++c) any |= radii[(size_t)c * N + n] > 0;
    if (valid && !any) {
        d_quats[n] = make_float4(0.f, 0.f, 0.f, 0.f);
        d_log_scales[3 * n] = 0.f;
        d_log_scales[3 * n + 1] = 0.f;
        d_log_scales[3 * n + 2] = 0.f;
        d_logits[n] = 0.f;
    }
    const bool work = valid && any;
    if (!work && !d_viewmats) return;  // with a pose gradient every thread joins the CTA sums
    float dmu[3] = {0.f, 0.f, 0.f};
    float dSig[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // symmetric matrix gradient: xx, xy, xz, yy, yz, zz
    float d_o = 0.f;
    // a camera's radius and 2D gradients are requested one camera ahead (read whether or not
    // the pair is visible), so they arrive while the previous camera's chain runs
    struct Up {
        int r;
        float2 m;
        float a, b, c, op, dep;
    };
    auto fetch = [&](size_t idx) {
        Up u;
        u.r = radii[idx];
        u.m = d_means2d[idx];
        u.a = d_conics[3 * idx];
        u.b = d_conics[3 * idx + 1];
        u.c = d_conics[3 * idx + 2];
        u.op = d_opac[idx];
        u.dep = d_depths ? d_depths[idx] : 0.f;
        return u;
    };
    Up nxt{0, make_float2(0.f, 0.f), 0.f, 0.f, 0.f, 0.f, 0.f};
    if (work) nxt = fetch(n);
    for (int c = 0; c < cs.C; ++c) {
        const size_t idx = (size_t)c * N + n;
        const CamDev &cam = cs.cam[c];
        float pose[12] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // rows of [dR | dt]
        Splat2 sp;
        const Up cur = nxt;
        if (work && c + 1 < cs.C) nxt = fetch(idx + N);
        const bool vis = work && cur.r > 0;
        const float2 gm = cur.m;
        const float ga = cur.a, gb = cur.b, gc = cur.c, gop = cur.op, gdep = cur.dep;
        if (vis && splat_of(g, mean, cam, rc, sp)) {
            if (d_viewmats)
                splat_bwd<true>(g, mean, cam, rc, sp, gm, ga, gb, gc, gop, gdep, dmu, dSig, d_o, pose);
            else
                splat_bwd<false>(g, mean, cam, rc, sp, gm, ga, gb, gc, gop, gdep, dmu, dSig, d_o, pose);
        }
        if (d_viewmats) block_sum_atomic<12>(pose, d_viewmats + 16 * c, s_red);
    }
    if (!work) return;
    d_means[3 * n] = dm_in[0] + dmu[0];
    d_means[3 * n + 1] = dm_in[1] + dmu[1];
    d_means[3 * n + 2] = dm_in[2] + dmu[2];
    float dls[3], dl;
    float4 dq;
    gauss_bwd(g, dSig, d_o, dls, dq, dl);
    d_log_scales[3 * n] = dls[0];
    d_log_scales[3 * n + 1] = dls[1];
    d_log_scales[3 * n + 2] = dls[2];
    d_quats[n] = dq;
    d_logits[n] = dl;
}

cudaError_t launch_project_fwd(const CamSet &cs, const RasterConsts &rc, int N, const float *means,
                               const float *quats, const float *log_scales, const float *logits, float *means2d,
                               float *depths, float *conics, int *radii, int *tiles_touched, float *opac,
                               cudaStream_t st) {
    int blocks = (N + 255) / 256;
    project_fwd_kernel<<<blocks, 256, 0, st>>>(N, means, (const float4 *)quats, log_scales, logits, cs, rc,
                                                (float2 *)means2d, depths, conics, radii, tiles_touched, opac);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_project_bwd(const CamSet &cs, const RasterConsts &rc, int N, const float *means,
                               const float *quats, const float *log_scales, const float *logits, const int *radii,
                               const float *d_means2d, const float *d_conics, const float *d_opac,
                               const float *d_depths, float *d_means, float *d_quats, float *d_log_scales,
                               float *d_logits, float *d_viewmats, cudaStream_t st) {
    int blocks = (N + 255) / 256;
    project_bwd_kernel<<<blocks, 256, 0, st>>>(N, means, (const float4 *)quats, log_scales, logits, cs, rc, radii,
                                                (const float2 *)d_means2d, d_conics, d_opac, d_depths, d_means,
                                                (float4 *)d_quats, d_log_scales, d_logits, d_viewmats);
    note_launch();
    return cudaGetLastError();
}

}  // namespace gs
