// Projection of a 3D Gaussian to a 2D splat and the pieces of its backward (App. C.1,
// App. D.2-D.4, App. E, App. A anti-aliasing), shared by the projection kernels and the
// fused SH + projection backward.
#pragma once

#include "gs_internal.cuh"

namespace gs {

struct Gauss3 {
    float s[3];     // exp(log_scale)
    float qn;       // |q|
    float q[4];     // q / |q|
    float R[9];     // R(q^)
    float Sig[6];   // Sigma: xx, xy, xz, yy, yz, zz
    float o;        // sigmoid(logit)
};

// Scale, rotation, covariance and opacity of a Gaussian from its raw parameters.
__device__ __forceinline__ void gauss_from(float4 q, float ls0, float ls1, float ls2, float logit, Gauss3 &g) {
    g.s[0] = __expf(ls0);
    g.s[1] = __expf(ls1);
    g.s[2] = __expf(ls2);
    g.qn = sqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
    float inv = 1.f / g.qn;
    float w = q.x * inv, x = q.y * inv, y = q.z * inv, z = q.w * inv;
    g.q[0] = w; g.q[1] = x; g.q[2] = y; g.q[3] = z;
    // App. E, Hamilton convention
    g.R[0] = 1.f - 2.f * (y * y + z * z);
    g.R[1] = 2.f * (x * y - w * z);
    g.R[2] = 2.f * (x * z + w * y);
    g.R[3] = 2.f * (x * y + w * z);
    g.R[4] = 1.f - 2.f * (x * x + z * z);
    g.R[5] = 2.f * (y * z - w * x);
    g.R[6] = 2.f * (x * z - w * y);
    g.R[7] = 2.f * (y * z + w * x);
    g.R[8] = 1.f - 2.f * (x * x + y * y);
    // Sigma = (R S)(R S)^T
    float M[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) M[3 * i + j] = g.R[3 * i + j] * g.s[j];
    g.Sig[0] = M[0] * M[0] + M[1] * M[1] + M[2] * M[2];
    g.Sig[1] = M[0] * M[3] + M[1] * M[4] + M[2] * M[5];
    g.Sig[2] = M[0] * M[6] + M[1] * M[7] + M[2] * M[8];
    g.Sig[3] = M[3] * M[3] + M[4] * M[4] + M[5] * M[5];
    g.Sig[4] = M[3] * M[6] + M[4] * M[7] + M[5] * M[8];
    g.Sig[5] = M[6] * M[6] + M[7] * M[7] + M[8] * M[8];
    g.o = 1.f / (1.f + __expf(-logit));
}

__device__ __forceinline__ void load_gauss(int n, const float *__restrict__ log_scales,
                                           const float4 *__restrict__ quats, const float *__restrict__ logits,
                                           Gauss3 &g) {
    gauss_from(quats[n], log_scales[3 * n + 0], log_scales[3 * n + 1], log_scales[3 * n + 2], logits[n], g);
}

struct Splat2 {
    float t[3];
    float T[6];      // J R_cw (2x3)
    float cov0[3];   // Sigma' before the low-pass
    float cov[3];    // Sigma' + eps I
    float conic[3];
    float mx, my;
    float comp;
};

// Returns false when culled (t_z < near) or degenerate.
__device__ __forceinline__ bool splat_of(const Gauss3 &g, const float mean[3], const CamDev &cam,
                                         const RasterConsts &rc, Splat2 &sp) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
        sp.t[i] = cam.R[3 * i] * mean[0] + cam.R[3 * i + 1] * mean[1] + cam.R[3 * i + 2] * mean[2] + cam.t[i];
    float tx = sp.t[0], ty = sp.t[1], tz = sp.t[2];
    if (!(tz >= rc.near_plane)) return false;
    float iz = 1.f / tz;
    sp.mx = cam.fx * tx * iz + cam.cx;
    sp.my = cam.fy * ty * iz + cam.cy;
    // J = [[fx/tz, 0, -fx tx/tz^2], [0, fy/tz, -fy ty/tz^2]];  T = J R_cw
    float j00 = cam.fx * iz, j02 = -cam.fx * tx * iz * iz;
    float j11 = cam.fy * iz, j12 = -cam.fy * ty * iz * iz;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        sp.T[k] = j00 * cam.R[k] + j02 * cam.R[6 + k];
        sp.T[3 + k] = j11 * cam.R[3 + k] + j12 * cam.R[6 + k];
    }
    // Sigma' = T Sigma T^T
    const float *S = g.Sig;
    float u0[3], u1[3];  // T Sigma rows
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const float *Tr = sp.T + 3 * r;
        float *u = r == 0 ? u0 : u1;
        u[0] = Tr[0] * S[0] + Tr[1] * S[1] + Tr[2] * S[2];
        u[1] = Tr[0] * S[1] + Tr[1] * S[3] + Tr[2] * S[4];
        u[2] = Tr[0] * S[2] + Tr[1] * S[4] + Tr[2] * S[5];
    }
    sp.cov0[0] = u0[0] * sp.T[0] + u0[1] * sp.T[1] + u0[2] * sp.T[2];
    sp.cov0[1] = u0[0] * sp.T[3] + u0[1] * sp.T[4] + u0[2] * sp.T[5];
    sp.cov0[2] = u1[0] * sp.T[3] + u1[1] * sp.T[4] + u1[2] * sp.T[5];
    sp.cov[0] = sp.cov0[0] + rc.eps2d;
    sp.cov[1] = sp.cov0[1];
    sp.cov[2] = sp.cov0[2] + rc.eps2d;
    float det = sp.cov[0] * sp.cov[2] - sp.cov[1] * sp.cov[1];
    if (!(det > 0.f)) return false;
    float idet = 1.f / det;
    sp.conic[0] = sp.cov[2] * idet;
    sp.conic[1] = -sp.cov[1] * idet;
    sp.conic[2] = sp.cov[0] * idet;
    sp.comp = 1.f;
    if (rc.antialiased) {
        float det0 = sp.cov0[0] * sp.cov0[2] - sp.cov0[1] * sp.cov0[1];
        sp.comp = sqrtf(fmaxf(det0 * idet, 0.f));
    }
    return true;
}

__device__ __forceinline__ int radius_of(const Splat2 &sp) {
    float m = 0.5f * (sp.cov[0] + sp.cov[2]);
    float det = sp.cov[0] * sp.cov[2] - sp.cov[1] * sp.cov[1];
    float lam = m + sqrtf(fmaxf(m * m - det, 0.f));
    float r = ceilf(3.f * sqrtf(lam));
    if (!(r > 0.f) || r > 1.0e7f) return 0;
    return (int)r;
}

// dR/dq_k at the unit quaternion (w, x, y, z), App. D.4 (the factor 2 included).
__device__ __forceinline__ void drot(const float q[4], const float dR[9], float dq[4]) {
    float w = q[0], x = q[1], y = q[2], z = q[3];
    // <dR, dR/dw>
    dq[0] = 2.f * (-z * dR[1] + y * dR[2] + z * dR[3] - x * dR[5] - y * dR[6] + x * dR[7]);
    dq[1] = 2.f * (y * dR[1] + z * dR[2] + y * dR[3] - 2.f * x * dR[4] - w * dR[5] + z * dR[6] + w * dR[7] -
                   2.f * x * dR[8]);
    dq[2] = 2.f * (-2.f * y * dR[0] + x * dR[1] + w * dR[2] + x * dR[3] + z * dR[5] - w * dR[6] + z * dR[7] -
                   2.f * y * dR[8]);
    dq[3] = 2.f * (-2.f * z * dR[0] - w * dR[1] + x * dR[2] + w * dR[3] - 2.f * z * dR[4] + y * dR[5] + x * dR[6] +
                   y * dR[7]);
}

// One camera's part of the projection backward: from the gradients of the splat's 2D mean
// (gm), conic (ga, gb, gc), opacity (gop) and camera depth (gdep), adds the gradients of the
// mean (dmu), of the 3D covariance (dSig: xx, xy, xz, yy, yz, zz) and of the sigmoid opacity
// (d_o); with POSE also fills pose[12], the rows of [dR_cw | dt_cw].
template <bool POSE>
__device__ __forceinline__ void splat_bwd(const Gauss3 &g, const float mean[3], const CamDev &cam,
                                          const RasterConsts &rc, const Splat2 &sp, float2 gm, float ga, float gb,
                                          float gc, float gop, float gdep, float dmu[3], float dSig[6], float &d_o,
                                          float pose[12]) {
    // conic scalars (a, b, c) -> matrix gradient dY = [[ga, gb/2], [gb/2, gc]];
    // dSigma' = -Y dY Y  (App. D.2)
    float Ya = sp.conic[0], Yb = sp.conic[1], Yc = sp.conic[2];
    float hb = 0.5f * gb;
    float m00 = Ya * ga + Yb * hb, m01 = Ya * hb + Yb * gc;
    float m10 = Yb * ga + Yc * hb, m11 = Yb * hb + Yc * gc;
    float G00 = -(m00 * Ya + m01 * Yb);
    float G01 = -(m00 * Yb + m01 * Yc);
    float G11 = -(m10 * Yb + m11 * Yc);
    d_o += gop * sp.comp;
    if (rc.antialiased && sp.comp > 0.f) {
        // comp = sqrt(det0/det1): gradient w.r.t. the entries (a, b, c) of Sigma'
        float a = sp.cov0[0], b = sp.cov0[1], cc = sp.cov0[2];
        float det0 = a * cc - b * b;
        float det1 = sp.cov[0] * sp.cov[2] - sp.cov[1] * sp.cov[1];
        float k = gop * g.o / (2.f * sp.comp) / (det1 * det1);
        G00 += k * (cc * det1 - det0 * sp.cov[2]);
        G11 += k * (a * det1 - det0 * sp.cov[0]);
        G01 += 0.5f * k * (2.f * b * det0 - 2.f * b * det1);
    }
    // Sigma' = T Sigma T^T:  dSigma = T^T G T;  dT = 2 G T Sigma (G, Sigma symmetric)
    const float *T = sp.T;
    float GT0[3], GT1[3];  // rows of G T
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        GT0[k] = G00 * T[k] + G01 * T[3 + k];
        GT1[k] = G01 * T[k] + G11 * T[3 + k];
    }
    // dSigma_ij += T0i GT0j + T1i GT1j
    dSig[0] += T[0] * GT0[0] + T[3] * GT1[0];
    dSig[1] += T[0] * GT0[1] + T[3] * GT1[1];
    dSig[2] += T[0] * GT0[2] + T[3] * GT1[2];
    dSig[3] += T[1] * GT0[1] + T[4] * GT1[1];
    dSig[4] += T[1] * GT0[2] + T[4] * GT1[2];
    dSig[5] += T[2] * GT0[2] + T[5] * GT1[2];
    const float *S = g.Sig;
    float dT[6];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float s0 = k == 0 ? S[0] : (k == 1 ? S[1] : S[2]);
        float s1 = k == 0 ? S[1] : (k == 1 ? S[3] : S[4]);
        float s2 = k == 0 ? S[2] : (k == 1 ? S[4] : S[5]);
        dT[k] = 2.f * (GT0[0] * s0 + GT0[1] * s1 + GT0[2] * s2);
        dT[3 + k] = 2.f * (GT1[0] * s0 + GT1[1] * s1 + GT1[2] * s2);
    }
    // T = J R_cw:  dJ = dT R_cw^T (only the non-constant entries of J are needed)
    const float *W = cam.R;
    float dJ00 = dT[0] * W[0] + dT[1] * W[1] + dT[2] * W[2];
    float dJ02 = dT[0] * W[6] + dT[1] * W[7] + dT[2] * W[8];
    float dJ11 = dT[3] * W[3] + dT[4] * W[4] + dT[5] * W[5];
    float dJ12 = dT[3] * W[6] + dT[4] * W[7] + dT[5] * W[8];
    float tx = sp.t[0], ty = sp.t[1], tz = sp.t[2];
    float iz = 1.f / tz, iz2 = iz * iz, iz3 = iz2 * iz;
    float fx = cam.fx, fy = cam.fy;
    float dtx = gm.x * fx * iz - dJ02 * fx * iz2;
    float dty = gm.y * fy * iz - dJ12 * fy * iz2;
    float dtz = -gm.x * fx * tx * iz2 - gm.y * fy * ty * iz2 - dJ00 * fx * iz2 + dJ02 * 2.f * fx * tx * iz3 -
                dJ11 * fy * iz2 + dJ12 * 2.f * fy * ty * iz3;
    dtz += gdep;
    // t = R_cw mu + t_cw:  dmu = R_cw^T dt
    dmu[0] += W[0] * dtx + W[3] * dty + W[6] * dtz;
    dmu[1] += W[1] * dtx + W[4] * dty + W[7] * dtz;
    dmu[2] += W[2] * dtx + W[5] * dty + W[8] * dtz;
    if (POSE) {
        // pose (App. A): dR_cw = J^T dT + dt mu^T,  dt_cw = dt, with
        // J = [[fx/tz, 0, -fx tx/tz^2], [0, fy/tz, -fy ty/tz^2]]
        const float dt3[3] = {dtx, dty, dtz};
        const float j02 = -fx * tx * iz2, j12 = -fy * ty * iz2;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            pose[j] = fx * iz * dT[j] + dt3[0] * mean[j];
            pose[4 + j] = fy * iz * dT[3 + j] + dt3[1] * mean[j];
            pose[8 + j] = j02 * dT[j] + j12 * dT[3 + j] + dt3[2] * mean[j];
        }
        pose[3] = dtx;
        pose[7] = dty;
        pose[11] = dtz;
    }
}

// The rest of the chain for one Gaussian: Sigma = (R S)(R S)^T, the quaternion
// normalisation, s = exp(log_scale) and o = sigmoid(logit).
__device__ __forceinline__ void gauss_bwd(const Gauss3 &g, const float dSig[6], float d_o, float d_log_scale[3],
                                          float4 &d_quat, float &d_logit) {
    // Sigma = M M^T, M = R S:  dM = 2 dSigma M;  dR = dM S;  dS_j = (R^T dM)_jj
    float D[9] = {dSig[0], dSig[1], dSig[2], dSig[1], dSig[3], dSig[4], dSig[2], dSig[4], dSig[5]};
    float dR[9], ds[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            float dMij = 2.f * (D[3 * i] * g.R[j] + D[3 * i + 1] * g.R[3 + j] + D[3 * i + 2] * g.R[6 + j]) * g.s[j];
            dR[3 * i + j] = dMij * g.s[j];
            ds[j] += g.R[3 * i + j] * dMij;
        }
    d_log_scale[0] = ds[0] * g.s[0];
    d_log_scale[1] = ds[1] * g.s[1];
    d_log_scale[2] = ds[2] * g.s[2];
    float dqh[4];
    drot(g.q, dR, dqh);
    float proj = g.q[0] * dqh[0] + g.q[1] * dqh[1] + g.q[2] * dqh[2] + g.q[3] * dqh[3];
    float iq = 1.f / g.qn;
    d_quat = make_float4((dqh[0] - g.q[0] * proj) * iq, (dqh[1] - g.q[1] * proj) * iq,
                             (dqh[2] - g.q[2] * proj) * iq, (dqh[3] - g.q[3] * proj) * iq);
    d_logit = d_o * g.o * (1.f - g.o);
}

}  // namespace gs
