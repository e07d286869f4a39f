// View-dependent colour from real spherical harmonics (App. C.1: c = SH(dir)) and its
// backward.  A CTA of 256 threads owns 256 consecutive Gaussians: their coefficients
// ([256, K, 3] floats, contiguous in HBM) are copied with 16-byte loads into shared
// memory at an odd row stride (no bank conflicts when each thread then reads its own
// row), and every thread loops over the cameras of the call.
#include <math.h>

#include "project_math.cuh"

namespace gs {

// Orthonormal real SH normalisation constants, from the closed form
// K_l^m = sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) times sqrt(2) for m != 0, folded
// with the Legendre polynomial coefficients.  Computed on the host in double.
struct ShConsts {
    float k0;                        // l = 0
    float k1;                        // l = 1
    float k2a, k2b, k2c;             // l = 2: m = +-1,-2 / 0 / 2
    float k3a, k3b, k3c, k3d, k3e;   // l = 3: +-3 / -2 / +-1 / 0 / 2
};

static ShConsts make_sh_consts() {
    const double pi = 3.14159265358979323846;
    ShConsts k;
    k.k0 = (float)(0.5 * sqrt(1.0 / pi));
    k.k1 = (float)sqrt(3.0 / (4.0 * pi));
    k.k2a = (float)(0.5 * sqrt(15.0 / pi));
    k.k2b = (float)(0.25 * sqrt(5.0 / pi));
    k.k2c = (float)(0.25 * sqrt(15.0 / pi));
    k.k3a = (float)(0.25 * sqrt(35.0 / (2.0 * pi)));
    k.k3b = (float)(0.5 * sqrt(105.0 / pi));
    k.k3c = (float)(0.25 * sqrt(21.0 / (2.0 * pi)));
    k.k3d = (float)(0.25 * sqrt(7.0 / pi));
    k.k3e = (float)(0.25 * sqrt(105.0 / pi));
    return k;
}

// Basis values, order m = -l..l within each degree (Condon-Shortley phase).
template <int DEG>
__device__ __forceinline__ void sh_eval_basis(const ShConsts &k, float x, float y, float z, float *Y) {
    Y[0] = k.k0;
    if (DEG >= 1) {
        Y[1] = -k.k1 * y;
        Y[2] = k.k1 * z;
        Y[3] = -k.k1 * x;
    }
    if (DEG >= 2) {
        float xx = x * x, yy = y * y, zz = z * z;
        Y[4] = k.k2a * x * y;
        Y[5] = -k.k2a * y * z;
        Y[6] = k.k2b * (2.f * zz - xx - yy);
        Y[7] = -k.k2a * x * z;
        Y[8] = k.k2c * (xx - yy);
        if (DEG >= 3) {
            Y[9] = -k.k3a * y * (3.f * xx - yy);
            Y[10] = k.k3b * x * y * z;
            Y[11] = -k.k3c * y * (4.f * zz - xx - yy);
            Y[12] = k.k3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
            Y[13] = -k.k3c * x * (4.f * zz - xx - yy);
            Y[14] = k.k3e * z * (xx - yy);
            Y[15] = -k.k3a * x * (xx - 3.f * yy);
        }
    }
}

// Accumulates g[k] * grad_{x,y,z} Y_k into d (the basis is a polynomial in x, y, z).
template <int DEG>
__device__ __forceinline__ void sh_basis_vjp(const ShConsts &k, float x, float y, float z, const float *g,
                                             float d[3]) {
    if (DEG >= 1) {
        d[1] += -k.k1 * g[1];
        d[2] += k.k1 * g[2];
        d[0] += -k.k1 * g[3];
    }
    if (DEG >= 2) {
        d[0] += k.k2a * y * g[4];
        d[1] += k.k2a * x * g[4];
        d[1] += -k.k2a * z * g[5];
        d[2] += -k.k2a * y * g[5];
        d[0] += -2.f * k.k2b * x * g[6];
        d[1] += -2.f * k.k2b * y * g[6];
        d[2] += 4.f * k.k2b * z * g[6];
        d[0] += -k.k2a * z * g[7];
        d[2] += -k.k2a * x * g[7];
        d[0] += 2.f * k.k2c * x * g[8];
        d[1] += -2.f * k.k2c * y * g[8];
        if (DEG >= 3) {
            float xx = x * x, yy = y * y, zz = z * z;
            d[0] += -k.k3a * 6.f * x * y * g[9];
            d[1] += -k.k3a * 3.f * (xx - yy) * g[9];
            d[0] += k.k3b * y * z * g[10];
            d[1] += k.k3b * x * z * g[10];
            d[2] += k.k3b * x * y * g[10];
            d[0] += k.k3c * 2.f * x * y * g[11];
            d[1] += -k.k3c * (4.f * zz - xx - 3.f * yy) * g[11];
            d[2] += -k.k3c * 8.f * y * z * g[11];
            d[0] += -k.k3d * 6.f * x * z * g[12];
            d[1] += -k.k3d * 6.f * y * z * g[12];
            d[2] += k.k3d * (6.f * zz - 3.f * xx - 3.f * yy) * g[12];
            d[0] += -k.k3c * (4.f * zz - 3.f * xx - yy) * g[13];
            d[1] += k.k3c * 2.f * x * y * g[13];
            d[2] += -k.k3c * 8.f * x * z * g[13];
            d[0] += k.k3e * 2.f * x * z * g[14];
            d[1] += -k.k3e * 2.f * y * z * g[14];
            d[2] += k.k3e * (xx - yy) * g[14];
            d[0] += -k.k3a * 3.f * (xx - yy) * g[15];
            d[1] += k.k3a * 6.f * x * y * g[15];
        }
    }
}

// Coefficient rows in shared memory, one per thread's Gaussian.  Rows whose length F is a
// multiple of 4 (degrees 1 and 3) are float4 rows at an odd float4 stride: each staging copy,
// each read or write of a thread's own row and each write-back is one 16-byte access, free of
// bank conflicts.  Other rows (degrees 0 and 2) are float rows at an odd float stride.
template <int F>
__host__ __device__ constexpr int row_stride() {
    return F % 4 == 0 ? ((F / 4) | 1) * 4 : (F | 1);
}

// fn(e, row[e]) for e = 0 .. F-1 in order (16-byte reads for float4 rows).
template <int F, class Fn>
__device__ __forceinline__ void row_for_each(const float *row, Fn &&fn) {
    if constexpr (F % 4 == 0) {
        const float4 *r4 = reinterpret_cast<const float4 *>(row);
#pragma unroll
        for (int j = 0; j < F / 4; ++j) {
            const float4 t = r4[j];
            fn(4 * j, t.x);
            fn(4 * j + 1, t.y);
            fn(4 * j + 2, t.z);
            fn(4 * j + 3, t.w);
        }
    } else {
#pragma unroll
        for (int e = 0; e < F; ++e) fn(e, row[e]);
    }
}

// row[e] = val(e), or row[e] += val(e) with ADD (16-byte accesses for float4 rows).
template <int F, bool ADD, class Fn>
__device__ __forceinline__ void row_write(float *row, Fn &&val) {
    if constexpr (F % 4 == 0) {
        float4 *r4 = reinterpret_cast<float4 *>(row);
#pragma unroll
        for (int j = 0; j < F / 4; ++j) {
            float4 o = make_float4(val(4 * j), val(4 * j + 1), val(4 * j + 2), val(4 * j + 3));
            if (ADD) {
                const float4 t = r4[j];
                o = make_float4(t.x + o.x, t.y + o.y, t.z + o.z, t.w + o.w);
            }
            r4[j] = o;
        }
    } else {
#pragma unroll
        for (int e = 0; e < F; ++e) row[e] = ADD ? row[e] + val(e) : val(e);
    }
}

// Copies the coefficient rows of Gaussians [n0, n0+cnt) into shared memory (row_stride<F>).
// NT threads each issue all their 16-byte loads before the first shared-memory store, so a
// thread keeps up to ceil(NT F / 4 / NT) loads in flight instead of waiting on each in turn.
// Rows whose flag in `ok` (shared memory, one per row) is zero are not read: their Gaussian is
// culled in every camera, so neither its colour nor its gradient uses the coefficients.
template <int F, int NT>
__device__ __forceinline__ void stage_rows(const float *__restrict__ src, int cnt, float *s, bool vec_ok,
                                           const unsigned char *ok) {
    constexpr int STRIDE = row_stride<F>();
    const int total = cnt * F;
    if constexpr (F % 4 == 0) {
        if (vec_ok) {  // one 16-byte load and one 16-byte store per float4 of a row
            constexpr int F4 = F / 4, S4 = STRIDE / 4;
            const int nvec = cnt * F4;
            const float4 *src4 = reinterpret_cast<const float4 *>(src);
            float4 *s4 = reinterpret_cast<float4 *>(s);
            float4 q[F4];
            unsigned take = 0u;  // bit j: load j is issued
#pragma unroll
            for (int j = 0; j < F4; ++j) {
                const int v = threadIdx.x + j * NT;
                if (v < nvec && ok[v / F4]) {
                    q[j] = src4[v];
                    take |= 1u << j;
                }
            }
#pragma unroll
            for (int j = 0; j < F4; ++j) {
                const int v = threadIdx.x + j * NT;
                if (take & (1u << j)) {
                    const int row = v / F4;
                    s4[row * S4 + (v - row * F4)] = q[j];
                }
            }
            return;
        }
    } else if (vec_ok) {
        constexpr int V = (NT * F / 4 + NT - 1) / NT;  // float4 loads per thread for a full chunk
        const int nvec = total / 4;
        const float4 *src4 = reinterpret_cast<const float4 *>(src);
        float4 q[V];
        unsigned take = 0u;  // bit j: load j is issued
#pragma unroll
        for (int j = 0; j < V; ++j) {
            const int v = threadIdx.x + j * NT;
            // a 16-byte load may straddle two rows when F is not a multiple of 4
            if (v < nvec && (ok[(4 * v) / F] | ok[(4 * v + 3) / F])) {
                q[j] = src4[v];
                take |= 1u << j;
            }
        }
#pragma unroll
        for (int j = 0; j < V; ++j) {
            const int v = threadIdx.x + j * NT;
            if (take & (1u << j)) {
                int e = 4 * v;
                s[(e / F) * STRIDE + e % F] = q[j].x;
                ++e;
                s[(e / F) * STRIDE + e % F] = q[j].y;
                ++e;
                s[(e / F) * STRIDE + e % F] = q[j].z;
                ++e;
                s[(e / F) * STRIDE + e % F] = q[j].w;
            }
        }
        for (int e = nvec * 4 + threadIdx.x; e < total; e += NT)
            if (ok[e / F]) s[(e / F) * STRIDE + e % F] = src[e];
        return;
    }
    for (int e = threadIdx.x; e < total; e += NT)
        if (ok[e / F]) s[(e / F) * STRIDE + e % F] = src[e];
}

// Writes the shared rows of Gaussians [n0, n0+cnt) back to dst (contiguous [cnt, F]).
template <int F, int NT>
__device__ __forceinline__ void store_rows(float *__restrict__ dst, int cnt, const float *s) {
    constexpr int STRIDE = row_stride<F>();
    const int total = cnt * F;
    const bool al = (reinterpret_cast<uintptr_t>(dst) & 15) == 0;
    if constexpr (F % 4 == 0) {
        if (al) {
            constexpr int F4 = F / 4, S4 = STRIDE / 4;
            float4 *dst4 = reinterpret_cast<float4 *>(dst);
            const float4 *s4 = reinterpret_cast<const float4 *>(s);
            for (int v = threadIdx.x; v < cnt * F4; v += NT) {
                const int row = v / F4;
                dst4[v] = s4[row * S4 + (v - row * F4)];
            }
            return;
        }
    } else if (al) {
        const int nvec = total / 4;
        float4 *dst4 = reinterpret_cast<float4 *>(dst);
        for (int v = threadIdx.x; v < nvec; v += NT) {
            int e = 4 * v;
            float4 o;
            o.x = s[(e / F) * STRIDE + e % F];
            ++e;
            o.y = s[(e / F) * STRIDE + e % F];
            ++e;
            o.z = s[(e / F) * STRIDE + e % F];
            ++e;
            o.w = s[(e / F) * STRIDE + e % F];
            dst4[v] = o;
        }
        for (int e = nvec * 4 + threadIdx.x; e < total; e += NT) dst[e] = s[(e / F) * STRIDE + e % F];
        return;
    }
    for (int e = threadIdx.x; e < total; e += NT) dst[e] = s[(e / F) * STRIDE + e % F];
}

// Copies the float4 rows flagged in `ok` with asynchronous 16-byte copies (global 16-byte
// aligned source, F a multiple of 4); the caller waits with cp.async.wait_all and a barrier.
template <int F, int NT>
__device__ __forceinline__ void stage_rows_async(const float *__restrict__ src, int cnt, float *s,
                                                 const unsigned char *ok) {
    constexpr int F4 = F / 4, S4 = row_stride<F>() / 4;
    const float4 *src4 = reinterpret_cast<const float4 *>(src);
    float4 *s4 = reinterpret_cast<float4 *>(s);
    for (int v = threadIdx.x; v < cnt * F4; v += NT) {
        const int row = v / F4;
        if (!ok[row]) continue;
        const unsigned dst = (unsigned)__cvta_generic_to_shared(s4 + row * S4 + (v - row * F4));
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src4 + v) : "memory");
    }
}

template <int DEG>
__global__ void __launch_bounds__(256) sh_fwd_kernel(int N, const float *__restrict__ sh,
                                                     const float *__restrict__ means, const int *__restrict__ radii,
                                                     const __grid_constant__ CamSet cs, ShConsts kc,
                                                     float *__restrict__ colors, const float *__restrict__ depths) {
    constexpr int K = (DEG + 1) * (DEG + 1), F = 3 * K, STRIDE = row_stride<F>();
    const int OS = depths ? 4 : 3;  // (r, g, b) or (r, g, b, depth) per (camera, Gaussian)
    extern __shared__ __align__(16) float s_coef[];
    int n0 = blockIdx.x * 256;
    int cnt = min(256, N - n0);
    int n = n0 + threadIdx.x;
    // this Gaussian's mean and first radius are requested before the coefficient rows, so
    // their latency overlaps the staging
    const bool valid = n < N;
    float mx = 0.f, my = 0.f, mz = 0.f;
    int r0 = 0;
    if (valid) {
        mx = means[3 * n];
        my = means[3 * n + 1];
        mz = means[3 * n + 2];
        r0 = radii[n];
    }
    __shared__ unsigned char s_ok[256];
    {
        bool seen = r0 > 0;
        for (int c = 1; c < cs.C && valid && !seen; ++c) seen = radii[(size_t)c * N + n] > 0;
        s_ok[threadIdx.x] = seen;
    }
    __syncthreads();
    const float *src = sh + (size_t)n0 * F;
    stage_rows<F, 256>(src, cnt, s_coef, (reinterpret_cast<uintptr_t>(src) & 15) == 0, s_ok);
    __syncthreads();
    if (!valid) return;
    const float *cf = s_coef + threadIdx.x * STRIDE;
    for (int c = 0; c < cs.C; ++c) {
        size_t idx = (size_t)c * N + n;
        float *out = colors + OS * idx;
        if ((c == 0 ? r0 : radii[idx]) <= 0) {
            out[0] = 0.f;
            out[1] = 0.f;
            out[2] = 0.f;
            if (depths) out[3] = 0.f;
            continue;
        }
        if (depths) out[3] = depths[idx];
        const float *R = cs.cam[c].R, *t = cs.cam[c].t;
        // camera centre = -R^T t
        float ox = -(R[0] * t[0] + R[3] * t[1] + R[6] * t[2]);
        float oy = -(R[1] * t[0] + R[4] * t[1] + R[7] * t[2]);
        float oz = -(R[2] * t[0] + R[5] * t[1] + R[8] * t[2]);
        float vx = mx - ox, vy = my - oy, vz = mz - oz;
        float il = rsqrtf(vx * vx + vy * vy + vz * vz);
        float Y[K];
        sh_eval_basis<DEG>(kc, vx * il, vy * il, vz * il, Y);
        float acc[3] = {0.5f, 0.5f, 0.5f};  // element e = 3 k + channel, k ascending per channel
        row_for_each<F>(cf, [&](int e, float v) { acc[e % 3] = fmaf(Y[e / 3], v, acc[e % 3]); });
        out[0] = fmaxf(acc[0], 0.f);
        out[1] = fmaxf(acc[1], 0.f);
        out[2] = fmaxf(acc[2], 0.f);
    }
}

// Backward: a CTA of kShBwdThreads threads owns as many consecutive Gaussians.  The
// coefficient gradients are accumulated over cameras in a second shared-memory row per
// thread (not in registers, which keeps occupancy up at degree 3) and leave through the
// same contiguous copy as the coefficients came in.
constexpr int kShBwdThreads = 128;

#ifndef GS_SH_PROJECT_BWD_MIN_BLOCKS
#define GS_SH_PROJECT_BWD_MIN_BLOCKS 5  // 96 registers, no spills: five 128-thread CTAs per SM
#endif

// ONECAM (a single camera): the gradient row of each Gaussian is written in place over its
// staged coefficient row once the row has been used, so a CTA needs half the shared memory
// and twice as many CTAs fit on an SM.  With several cameras the two rows per thread allow four
// 128-thread CTAs per SM (shared memory at degree 3), and the registers are held to that.
template <int DEG, bool ONECAM>
__global__ void __launch_bounds__(kShBwdThreads, ONECAM ? 5 : 4) sh_bwd_kernel(int N, const float *__restrict__ sh,
                                                               const float *__restrict__ means,
                                                               const int *__restrict__ radii,
                                                               const __grid_constant__ CamSet cs, ShConsts kc,
                                                               const float *__restrict__ d_colors,
                                                               float *__restrict__ d_sh, float *__restrict__ d_means,
                                                               float *__restrict__ d_depths,
                                                               float *__restrict__ d_viewmats) {
    constexpr int K = (DEG + 1) * (DEG + 1), F = 3 * K, STRIDE = row_stride<F>();
    const int IS = d_depths ? 4 : 3;  // d_colors rows: (r, g, b) or (r, g, b, depth)
    extern __shared__ __align__(16) float s_coef[];
    __shared__ float s_red[(kShBwdThreads / 32) * 12];
    float *s_grad = ONECAM ? s_coef : s_coef + kShBwdThreads * STRIDE;
    const int n0 = blockIdx.x * kShBwdThreads;
    const int cnt = min(kShBwdThreads, N - n0);
    const int n = n0 + threadIdx.x;
    const bool valid = n < N;
    // per-Gaussian inputs are requested before the coefficient rows, so their latency
    // overlaps the staging
    const float mx = valid ? means[3 * n] : 0.f, my = valid ? means[3 * n + 1] : 0.f,
                mz = valid ? means[3 * n + 2] : 0.f;
    const int r0 = valid ? radii[n] : 0;
    float g0[4] = {0.f, 0.f, 0.f, 0.f};
    if (valid) {  // (read for culled pairs too, so the load does not wait for the radius; unused there)
        g0[0] = d_colors[IS * (size_t)n];
        g0[1] = d_colors[IS * (size_t)n + 1];
        g0[2] = d_colors[IS * (size_t)n + 2];
        if (d_depths) g0[3] = d_colors[IS * (size_t)n + 3];
    }
    __shared__ unsigned char s_ok[kShBwdThreads];
    {
        bool seen = r0 > 0;
        for (int c = 1; c < cs.C && valid && !seen; ++c) seen = radii[(size_t)c * N + n] > 0;
        s_ok[threadIdx.x] = seen;
    }
    __syncthreads();
    const float *src = sh + (size_t)n0 * F;
    stage_rows<F, kShBwdThreads>(src, cnt, s_coef, (reinterpret_cast<uintptr_t>(src) & 15) == 0, s_ok);
    float *gr = s_grad + threadIdx.x * STRIDE;
    if (!ONECAM) row_write<F, false>(gr, [](int) { return 0.f; });
    __syncthreads();
    const float *cf = s_coef + threadIdx.x * STRIDE;
    float dm[3] = {0.f, 0.f, 0.f};
    // the next camera's radius and colour gradient are requested while this camera is worked
    // on (they are read whether or not the pair is visible), so each camera costs no round
    // trip to memory of its own
    int r_next = r0;
    float g_next[4] = {g0[0], g0[1], g0[2], g0[3]};
    for (int c = 0; c < cs.C; ++c) {  // every thread runs every camera (the pose sums are CTA-wide)
        const size_t idx = (size_t)c * N + n;
        float dv[3] = {0.f, 0.f, 0.f};  // gradient w.r.t. v = mu - centre for this camera
        const float *R = cs.cam[c].R, *t = cs.cam[c].t;
        const int rc = valid ? r_next : 0;
        const float gc[4] = {g_next[0], g_next[1], g_next[2], g_next[3]};
        if (valid && c + 1 < cs.C) {
            const size_t nx = idx + N;
            r_next = radii[nx];
            g_next[0] = d_colors[IS * nx];
            g_next[1] = d_colors[IS * nx + 1];
            g_next[2] = d_colors[IS * nx + 2];
            g_next[3] = d_depths ? d_colors[IS * nx + 3] : 0.f;
        }
        if (valid && d_depths) d_depths[idx] = rc > 0 ? gc[3] : 0.f;
        if (ONECAM && valid && rc <= 0) row_write<F, false>(gr, [](int) { return 0.f; });
        if (valid && rc > 0) {
            const float ox = -(R[0] * t[0] + R[3] * t[1] + R[6] * t[2]);
            const float oy = -(R[1] * t[0] + R[4] * t[1] + R[7] * t[2]);
            const float oz = -(R[2] * t[0] + R[5] * t[1] + R[8] * t[2]);
            const float vx = mx - ox, vy = my - oy, vz = mz - oz;
            const float il = rsqrtf(vx * vx + vy * vy + vz * vz);
            const float x = vx * il, y = vy * il, z = vz * il;
            float Y[K];
            sh_eval_basis<DEG>(kc, x, y, z, Y);
            // w_k = sum over channels of coeff_k,ch g_ch, where a channel clamped at 0 passes no
            // gradient.  With several cameras one pass over the staged row gives the colour and w
            // for unclamped channels, and only a pair with a clamped channel reads the row again
            // (a single camera keeps two passes: its in-place kernel has fewer registers to spare)
            float raw[3] = {0.5f, 0.5f, 0.5f};
            float w[K];
            if (ONECAM)
                row_for_each<F>(cf, [&](int e, float v) { raw[e % 3] = fmaf(Y[e / 3], v, raw[e % 3]); });
            else
                row_for_each<F>(cf, [&](int e, float v) {
                    raw[e % 3] = fmaf(Y[e / 3], v, raw[e % 3]);
                    w[e / 3] = e % 3 ? fmaf(v, gc[e % 3], w[e / 3]) : v * gc[0];
                });
            float g[3];
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) g[ch] = raw[ch] > 0.f ? gc[ch] : 0.f;
            if (ONECAM || !(raw[0] > 0.f && raw[1] > 0.f && raw[2] > 0.f))
                row_for_each<F>(cf, [&](int e, float v) { w[e / 3] = e % 3 ? fmaf(v, g[e % 3], w[e / 3]) : v * g[0]; });
            // (in place: every read of the row is above)
            row_write<F, !ONECAM>(gr, [&](int e) { return Y[e / 3] * g[e % 3]; });
            if (DEG > 0) {
                float dd[3] = {0.f, 0.f, 0.f};
                sh_basis_vjp<DEG>(kc, x, y, z, w, dd);
                // dir = v / |v|:  d v = (I - dir dir^T) d dir / |v|
                const float p = x * dd[0] + y * dd[1] + z * dd[2];
                dv[0] = (dd[0] - x * p) * il;
                dv[1] = (dd[1] - y * p) * il;
                dv[2] = (dd[2] - z * p) * il;
            }
        }
        dm[0] += dv[0];
        dm[1] += dv[1];
        dm[2] += dv[2];
        if (d_viewmats && DEG > 0) {
            // pose (App. A): centre = -R^T t, so dR_ij += t_i dv_j and dt_i += sum_j R_ij dv_j
            float pose[12];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
#pragma unroll
                for (int j = 0; j < 3; ++j) pose[4 * i + j] = t[i] * dv[j];
                pose[4 * i + 3] = R[3 * i] * dv[0] + R[3 * i + 1] * dv[1] + R[3 * i + 2] * dv[2];
            }
            block_sum_atomic<12>(pose, d_viewmats + 16 * c, s_red);
        }
    }
    if (valid) {
        d_means[3 * n] = dm[0];
        d_means[3 * n + 1] = dm[1];
        d_means[3 * n + 2] = dm[2];
    }
    __syncthreads();
    store_rows<F, kShBwdThreads>(d_sh + (size_t)n0 * F, cnt, s_grad);
}

// SH backward and projection backward of one camera in one kernel: the coefficient rows
// stream through shared memory as in sh_bwd_kernel (gradient rows written in place), and
// each thread runs the projection chain of its Gaussian (App. D.2-D.4) -- while its row is
// still arriving, when the rows are copied asynchronously (degrees 1 and 3) -- so d_means is
// written once and the Gaussian's parameters, radius and mean are read once for both.  Every
// per-Gaussian input of a visible Gaussian is requested before the coefficient rows.
template <int DEG>
__global__ void __launch_bounds__(kShBwdThreads, GS_SH_PROJECT_BWD_MIN_BLOCKS) sh_project_bwd_kernel(
    int N, const float *__restrict__ sh, const float *__restrict__ means, const float4 *__restrict__ quats,
    const float *__restrict__ log_scales, const float *__restrict__ logits, const int *__restrict__ radii,
    const __grid_constant__ CamSet cs, ShConsts kc, RasterConsts rc, const float *__restrict__ d_colors,
    const float2 *__restrict__ d_means2d, const float *__restrict__ d_conics, const float *__restrict__ d_opac,
    float *__restrict__ d_sh, float *__restrict__ d_means, float4 *__restrict__ d_quats,
    float *__restrict__ d_log_scales, float *__restrict__ d_logits) {
    constexpr int K = (DEG + 1) * (DEG + 1), F = 3 * K, STRIDE = row_stride<F>();
    extern __shared__ __align__(16) float s_coef[];
    __shared__ unsigned char s_ok[kShBwdThreads];
    const int n0 = blockIdx.x * kShBwdThreads;
    const int cnt = min(kShBwdThreads, N - n0);
    const int n = n0 + threadIdx.x;
    const bool valid = n < N;
    const int r0 = valid ? radii[n] : 0;
    const bool vis = r0 > 0;
    float mean[3] = {0.f, 0.f, 0.f};
    if (valid) {
        mean[0] = means[3 * n];
        mean[1] = means[3 * n + 1];
        mean[2] = means[3 * n + 2];
    }
    float g0[3] = {0.f, 0.f, 0.f};
    float2 gm = make_float2(0.f, 0.f);
    float ga = 0.f, gb = 0.f, gc = 0.f, gop = 0.f;
    float4 q = make_float4(1.f, 0.f, 0.f, 0.f);
    float ls0 = 0.f, ls1 = 0.f, ls2 = 0.f, lg = 0.f;
    if (vis) {
        g0[0] = d_colors[3 * (size_t)n];
        g0[1] = d_colors[3 * (size_t)n + 1];
        g0[2] = d_colors[3 * (size_t)n + 2];
        gm = d_means2d[n];
        ga = d_conics[3 * (size_t)n];
        gb = d_conics[3 * (size_t)n + 1];
        gc = d_conics[3 * (size_t)n + 2];
        gop = d_opac[n];
        q = quats[n];
        ls0 = log_scales[3 * (size_t)n];
        ls1 = log_scales[3 * (size_t)n + 1];
        ls2 = log_scales[3 * (size_t)n + 2];
        lg = logits[n];
    }
    s_ok[threadIdx.x] = vis;
    __syncthreads();
    const float *src = sh + (size_t)n0 * F;
    const bool aligned16 = (reinterpret_cast<uintptr_t>(src) & 15) == 0;
    const bool early = (F % 4 == 0) && aligned16;  // (uniform)
    if (early) {
        if constexpr (F % 4 == 0) stage_rows_async<F, kShBwdThreads>(src, cnt, s_coef, s_ok);
    } else {
        stage_rows<F, kShBwdThreads>(src, cnt, s_coef, aligned16, s_ok);
    }
    // the projection chain first: it needs no coefficient row, so with asynchronous copies it
    // runs while the rows arrive
    const CamDev &cam = cs.cam[0];
    float dmu[3] = {0.f, 0.f, 0.f}, dls[3] = {0.f, 0.f, 0.f}, dl = 0.f;
    float4 dq = make_float4(0.f, 0.f, 0.f, 0.f);
    if (vis) {
        Gauss3 gs3;
        gauss_from(q, ls0, ls1, ls2, lg, gs3);
        Splat2 sp;
        float dSig[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, d_o = 0.f, pose[12];
        if (splat_of(gs3, mean, cam, rc, sp))
            splat_bwd<false>(gs3, mean, cam, rc, sp, gm, ga, gb, gc, gop, 0.f, dmu, dSig, d_o, pose);
        gauss_bwd(gs3, dSig, d_o, dls, dq, dl);
    }
    if (early) asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();
    float *row = s_coef + threadIdx.x * STRIDE;  // coefficients, then (in place) their gradient
    float dm[3] = {0.f, 0.f, 0.f};
    if (vis) {
        const float *R = cam.R, *t = cam.t;
        const float ox = -(R[0] * t[0] + R[3] * t[1] + R[6] * t[2]);
        const float oy = -(R[1] * t[0] + R[4] * t[1] + R[7] * t[2]);
        const float oz = -(R[2] * t[0] + R[5] * t[1] + R[8] * t[2]);
        const float vx = mean[0] - ox, vy = mean[1] - oy, vz = mean[2] - oz;
        const float il = rsqrtf(vx * vx + vy * vy + vz * vz);
        const float x = vx * il, y = vy * il, z = vz * il;
        float Y[K];
        sh_eval_basis<DEG>(kc, x, y, z, Y);
        float raw[3] = {0.5f, 0.5f, 0.5f};
        row_for_each<F>(row, [&](int e, float v) { raw[e % 3] = fmaf(Y[e / 3], v, raw[e % 3]); });
        float g[3];
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) g[ch] = raw[ch] > 0.f ? g0[ch] : 0.f;  // the clamp at 0 passes no gradient
        float w[K];  // w_k = sum over channels of coeff_k,ch g_ch
        row_for_each<F>(row, [&](int e, float v) { w[e / 3] = e % 3 ? fmaf(v, g[e % 3], w[e / 3]) : v * g[0]; });
        // (in place: every read of the row is above)
        row_write<F, false>(row, [&](int e) { return Y[e / 3] * g[e % 3]; });
        if (DEG > 0) {
            float dd[3] = {0.f, 0.f, 0.f};
            sh_basis_vjp<DEG>(kc, x, y, z, w, dd);
            const float p = x * dd[0] + y * dd[1] + z * dd[2];
            dm[0] = (dd[0] - x * p) * il;
            dm[1] = (dd[1] - y * p) * il;
            dm[2] = (dd[2] - z * p) * il;
        }
    } else if (valid) {
        row_write<F, false>(row, [](int) { return 0.f; });
    }
    if (valid) {
        d_means[3 * n] = dm[0] + dmu[0];
        d_means[3 * n + 1] = dm[1] + dmu[1];
        d_means[3 * n + 2] = dm[2] + dmu[2];
        d_quats[n] = dq;
        d_log_scales[3 * n] = dls[0];
        d_log_scales[3 * n + 1] = dls[1];
        d_log_scales[3 * n + 2] = dls[2];
        d_logits[n] = dl;
    }
    __syncthreads();
    store_rows<F, kShBwdThreads>(d_sh + (size_t)n0 * F, cnt, s_coef);
}

constexpr int kProjShThreads = 64;  // Gaussians (threads) of a CTA of the fused forward (faster than 256)

// Could camera `cam` see a Gaussian with this mean and largest scale?  False only when the
// exact projection surely culls it: behind the near plane (the same test), or its pixel box,
// widened from an upper bound of the splat's radius, misses the image.  The bound uses
// lambda_max(T Sigma T^T) <= |T|_F^2 s_max^2 (T = J R_cw), plus the low-pass and margins far above
// float rounding.  Only the choice of which coefficient rows to copy early depends on it.
__device__ __forceinline__ bool maybe_visible(const float mean[3], float smax, const CamDev &cam,
                                              const RasterConsts &rc) {
    float t[3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
        t[i] = cam.R[3 * i] * mean[0] + cam.R[3 * i + 1] * mean[1] + cam.R[3 * i + 2] * mean[2] + cam.t[i];
    if (!(t[2] >= rc.near_plane)) return false;
    const float iz = 1.f / t[2];
    const float mx = cam.fx * t[0] * iz + cam.cx, my = cam.fy * t[1] * iz + cam.cy;
    const float j00 = cam.fx * iz, j02 = -cam.fx * t[0] * iz * iz;
    const float j11 = cam.fy * iz, j12 = -cam.fy * t[1] * iz * iz;
    float tf = 0.f;  // |T|_F^2
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float a = j00 * cam.R[k] + j02 * cam.R[6 + k], b = j11 * cam.R[3 + k] + j12 * cam.R[6 + k];
        tf += a * a + b * b;
    }
    const float r = 3.f * sqrtf(tf * smax * smax * 1.01f + rc.eps2d) * 1.01f + 2.f;
    if (!(r < 1.0e8f)) return true;  // (non-finite or huge: copy the row)
    return mx + r >= -1.f && mx - r <= (float)cam.W + 1.f && my + r >= -1.f && my - r <= (float)cam.H + 1.f;
}

// Projection and SH colours of the C cameras of a call in one kernel (App. C.1): each thread
// projects its Gaussian into every camera and writes the splats, and evaluates its colour per
// camera from its coefficient row, staged in shared memory (as sh_fwd_kernel does) for the
// Gaussians some camera may see.  With float4 rows (degrees 1 and 3) the row copies start
// before the projection, for the Gaussians a cheap conservative test keeps, so they arrive
// while the projection is computed; a row the test dropped but the projection needs (none, by
// construction) is read from global memory.  Otherwise the rows of the Gaussians the projection
// keeps are staged after it.  Parameters, mean and coefficients are read once for all cameras.
template <int DEG>
__global__ void __launch_bounds__(kProjShThreads) project_sh_fwd_kernel(
    int N, const float *__restrict__ sh, const float *__restrict__ means, const float4 *__restrict__ quats,
    const float *__restrict__ log_scales, const float *__restrict__ logits, const __grid_constant__ CamSet cs,
    ShConsts kc, RasterConsts rc, float2 *__restrict__ means2d, float *__restrict__ depths,
    float *__restrict__ conics, int *__restrict__ radii, int *__restrict__ tiles_touched, float *__restrict__ opac,
    float *__restrict__ colors) {
    constexpr int K = (DEG + 1) * (DEG + 1), F = 3 * K, STRIDE = row_stride<F>();
    extern __shared__ __align__(16) float s_coef[];
    __shared__ unsigned char s_ok[kProjShThreads];
    const int n0 = blockIdx.x * kProjShThreads;
    const int cnt = min(kProjShThreads, N - n0);
    const int n = n0 + threadIdx.x;
    const bool valid = n < N;
    const float *src = sh + (size_t)n0 * F;
    const bool early = (F % 4 == 0) && (reinterpret_cast<uintptr_t>(src) & 15) == 0;  // (uniform)
    float mean[3] = {0.f, 0.f, 0.f};
    Gauss3 g;
    if (valid) {
        mean[0] = means[3 * n];
        mean[1] = means[3 * n + 1];
        mean[2] = means[3 * n + 2];
        load_gauss(n, log_scales, quats, logits, g);
    }
    if (early) {
        bool maybe = false;
        if (valid) {
            const float smax = fmaxf(g.s[0], fmaxf(g.s[1], g.s[2]));
            for (int c = 0; c < cs.C && !maybe; ++c) maybe = maybe_visible(mean, smax, cs.cam[c], rc);
        }
        s_ok[threadIdx.x] = maybe;
        __syncthreads();
        if constexpr (F % 4 == 0) stage_rows_async<F, kProjShThreads>(src, cnt, s_coef, s_ok);
    }
    unsigned seen = 0u;  // bit c: camera c sees the Gaussian (C <= 32)
    if (valid) {
        const int tile = cs.tile;
        for (int c = 0; c < cs.C; ++c) {
            const CamDev &cam = cs.cam[c];
            const size_t idx = (size_t)c * N + n;
            Splat2 sp;
            const bool ok = splat_of(g, mean, cam, rc, sp);
            int r = ok ? radius_of(sp) : 0;
            int x0 = 0, x1 = -1, y0 = 0, y1 = -1;
            if (r > 0 && !pixel_box(sp.mx, sp.my, r, cam.W, cam.H, x0, x1, y0, y1)) r = 0;
            if (r > 0) {
                seen |= 1u << c;
                means2d[idx] = make_float2(sp.mx, sp.my);
                depths[idx] = sp.t[2];
                conics[3 * idx] = sp.conic[0];
                conics[3 * idx + 1] = sp.conic[1];
                conics[3 * idx + 2] = sp.conic[2];
                radii[idx] = r;
                tiles_touched[idx] = (x1 / tile - x0 / tile + 1) * (y1 / tile - y0 / tile + 1);
                opac[idx] = g.o * sp.comp;
            } else {
                means2d[idx] = make_float2(0.f, 0.f);
                depths[idx] = 0.f;
                conics[3 * idx] = 0.f;
                conics[3 * idx + 1] = 0.f;
                conics[3 * idx + 2] = 0.f;
                radii[idx] = 0;
                tiles_touched[idx] = 0;
                opac[idx] = 0.f;
            }
        }
    }
    if (early) {
        asm volatile("cp.async.wait_all;\n" ::: "memory");
    } else {
        s_ok[threadIdx.x] = seen != 0u;
        __syncthreads();
        stage_rows<F, kProjShThreads>(src, cnt, s_coef, (reinterpret_cast<uintptr_t>(src) & 15) == 0, s_ok);
    }
    __syncthreads();
    if (!valid) return;
    // the staged row, or (a row the conservative test dropped) the row in global memory
    const float *cf = s_ok[threadIdx.x] ? s_coef + threadIdx.x * STRIDE : sh + (size_t)n * F;
    for (int c = 0; c < cs.C; ++c) {
        float *out = colors + 3 * ((size_t)c * N + n);
        if (!(seen & (1u << c))) {
            out[0] = 0.f;
            out[1] = 0.f;
            out[2] = 0.f;
            continue;
        }
        const float *R = cs.cam[c].R, *t = cs.cam[c].t;
        // camera centre = -R^T t
        const float ox = -(R[0] * t[0] + R[3] * t[1] + R[6] * t[2]);
        const float oy = -(R[1] * t[0] + R[4] * t[1] + R[7] * t[2]);
        const float oz = -(R[2] * t[0] + R[5] * t[1] + R[8] * t[2]);
        const float vx = mean[0] - ox, vy = mean[1] - oy, vz = mean[2] - oz;
        const float il = rsqrtf(vx * vx + vy * vy + vz * vz);
        float Y[K];
        sh_eval_basis<DEG>(kc, vx * il, vy * il, vz * il, Y);
        float acc[3] = {0.5f, 0.5f, 0.5f};  // element e = 3 k + channel, k ascending per channel
        if (s_ok[threadIdx.x]) {
            row_for_each<F>(cf, [&](int e, float v) { acc[e % 3] = fmaf(Y[e / 3], v, acc[e % 3]); });
        } else {
#pragma unroll
            for (int e = 0; e < F; ++e) acc[e % 3] = fmaf(Y[e / 3], cf[e], acc[e % 3]);
        }
        out[0] = fmaxf(acc[0], 0.f);
        out[1] = fmaxf(acc[1], 0.f);
        out[2] = fmaxf(acc[2], 0.f);
    }
}

template <int DEG>
static cudaError_t launch_sh_fwd_t(const CamSet &cs, int N, const float *sh, const float *means, const int *radii,
                                   float *colors, const float *depths, cudaStream_t st) {
    constexpr int F = 3 * (DEG + 1) * (DEG + 1), STRIDE = row_stride<F>();
    size_t smem = 256 * STRIDE * sizeof(float);
    if (smem + 1024 > 48 * 1024) {  // dynamic + static shared memory above the default limit
        cudaError_t e = ensure_smem((const void *)sh_fwd_kernel<DEG>, (int)smem);
        if (e != cudaSuccess) return e;
    }
    sh_fwd_kernel<DEG><<<(N + 255) / 256, 256, smem, st>>>(N, sh, means, radii, cs, make_sh_consts(), colors, depths);
    note_launch();
    return cudaGetLastError();
}

template <int DEG>
static cudaError_t launch_sh_bwd_t(const CamSet &cs, int N, const float *sh, const float *means, const int *radii,
                                   const float *d_colors, float *d_sh, float *d_means, float *d_depths,
                                   float *d_viewmats, cudaStream_t st) {
    constexpr int F = 3 * (DEG + 1) * (DEG + 1), STRIDE = row_stride<F>();
    const bool one = cs.C == 1;
    size_t smem = (one ? 1 : 2) * kShBwdThreads * STRIDE * sizeof(float);
    auto kern = one ? sh_bwd_kernel<DEG, true> : sh_bwd_kernel<DEG, false>;
    if (smem + 1024 > 48 * 1024) {  // dynamic + static shared memory above the default limit
        cudaError_t e = ensure_smem((const void *)kern, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<(N + kShBwdThreads - 1) / kShBwdThreads, kShBwdThreads, smem, st>>>(
        N, sh, means, radii, cs, make_sh_consts(), d_colors, d_sh, d_means, d_depths, d_viewmats);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_sh_fwd(const CamSet &cs, int deg, int N, const float *sh, const float *means, const int *radii,
                          float *colors, const float *depths, cudaStream_t st) {
    switch (deg) {
        case 0: return launch_sh_fwd_t<0>(cs, N, sh, means, radii, colors, depths, st);
        case 1: return launch_sh_fwd_t<1>(cs, N, sh, means, radii, colors, depths, st);
        case 2: return launch_sh_fwd_t<2>(cs, N, sh, means, radii, colors, depths, st);
        default: return launch_sh_fwd_t<3>(cs, N, sh, means, radii, colors, depths, st);
    }
}

cudaError_t launch_sh_bwd(const CamSet &cs, int deg, int N, const float *sh, const float *means, const int *radii,
                          const float *d_colors, float *d_sh, float *d_means, float *d_depths, float *d_viewmats,
                          cudaStream_t st) {
    switch (deg) {
        case 0: return launch_sh_bwd_t<0>(cs, N, sh, means, radii, d_colors, d_sh, d_means, d_depths, d_viewmats, st);
        case 1: return launch_sh_bwd_t<1>(cs, N, sh, means, radii, d_colors, d_sh, d_means, d_depths, d_viewmats, st);
        case 2: return launch_sh_bwd_t<2>(cs, N, sh, means, radii, d_colors, d_sh, d_means, d_depths, d_viewmats, st);
        default: return launch_sh_bwd_t<3>(cs, N, sh, means, radii, d_colors, d_sh, d_means, d_depths, d_viewmats, st);
    }
}

template <int DEG>
static cudaError_t launch_project_sh_fwd_t(const CamSet &cs, const RasterConsts &rc, int N, const float *sh,
                                           const float *means, const float *quats, const float *log_scales,
                                           const float *logits, float *means2d, float *depths, float *conics,
                                           int *radii, int *tiles_touched, float *opac, float *colors,
                                           cudaStream_t st) {
    constexpr int F = 3 * (DEG + 1) * (DEG + 1), STRIDE = row_stride<F>();
    const size_t smem = kProjShThreads * STRIDE * sizeof(float);
    auto kern = project_sh_fwd_kernel<DEG>;
    if (smem + 1024 > 48 * 1024) {  // dynamic + static shared memory above the default limit
        cudaError_t e = ensure_smem((const void *)kern, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<(N + kProjShThreads - 1) / kProjShThreads, kProjShThreads, smem, st>>>(
        N, sh, means, (const float4 *)quats, log_scales, logits, cs,
                                             make_sh_consts(), rc, (float2 *)means2d, depths, conics, radii,
                                             tiles_touched, opac, colors);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_project_sh_fwd(const CamSet &cs, const RasterConsts &rc, int deg, int N, const float *sh,
                                  const float *means, const float *quats, const float *log_scales,
                                  const float *logits, float *means2d, float *depths, float *conics, int *radii,
                                  int *tiles_touched, float *opac, float *colors, cudaStream_t st) {
#define GS_PSF(D)                                                                                                  \
    return launch_project_sh_fwd_t<D>(cs, rc, N, sh, means, quats, log_scales, logits, means2d, depths, conics,   \
                                      radii, tiles_touched, opac, colors, st)
    switch (deg) {
        case 0: GS_PSF(0);
        case 1: GS_PSF(1);
        case 2: GS_PSF(2);
        default: GS_PSF(3);
    }
#undef GS_PSF
}

template <int DEG>
static cudaError_t launch_sh_project_bwd_t(const CamSet &cs, const RasterConsts &rc, int N, const float *sh,
                                           const float *means, const float *quats, const float *log_scales,
                                           const float *logits, const int *radii, const float *d_colors,
                                           const float *d_means2d, const float *d_conics, const float *d_opac,
                                           float *d_sh, float *d_means, float *d_quats, float *d_log_scales,
                                           float *d_logits, cudaStream_t st) {
    constexpr int F = 3 * (DEG + 1) * (DEG + 1), STRIDE = row_stride<F>();
    const size_t smem = kShBwdThreads * STRIDE * sizeof(float);
    auto kern = sh_project_bwd_kernel<DEG>;
    if (smem + 1024 > 48 * 1024) {  // dynamic + static shared memory above the default limit
        cudaError_t e = ensure_smem((const void *)kern, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<(N + kShBwdThreads - 1) / kShBwdThreads, kShBwdThreads, smem, st>>>(
        N, sh, means, (const float4 *)quats, log_scales, logits, radii, cs, make_sh_consts(), rc, d_colors,
        (const float2 *)d_means2d, d_conics, d_opac, d_sh, d_means, (float4 *)d_quats, d_log_scales, d_logits);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_sh_project_bwd(const CamSet &cs, const RasterConsts &rc, int deg, int N, const float *sh,
                                  const float *means, const float *quats, const float *log_scales,
                                  const float *logits, const int *radii, const float *d_colors,
                                  const float *d_means2d, const float *d_conics, const float *d_opac, float *d_sh,
                                  float *d_means, float *d_quats, float *d_log_scales, float *d_logits,
                                  cudaStream_t st) {
#define GS_SPB(D)                                                                                                \
    return launch_sh_project_bwd_t<D>(cs, rc, N, sh, means, quats, log_scales, logits, radii, d_colors, d_means2d, \
                                      d_conics, d_opac, d_sh, d_means, d_quats, d_log_scales, d_logits, st)
    switch (deg) {
        case 0: GS_SPB(0);
        case 1: GS_SPB(1);
        case 2: GS_SPB(2);
        default: GS_SPB(3);
    }
#undef GS_SPB
}

}  // namespace gs
