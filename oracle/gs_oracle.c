/*
 * gs_oracle.c -- plain, slow FP64 CPU reference of the differentiable
 * tile-based Gaussian rasterizer of gsplat (arXiv 2409.06765).
 *
 * TEST INFRASTRUCTURE ONLY.  It is loaded by the test-suite, by the smoke
 * check and by the benchmark's CPU-baseline leg, never by the product path.
 * It shares no source, header, table or helper with the CUDA library.
 *
 * What it computes (paper sections in brackets):
 *   - activations and covariance: s~ = exp(s), o~ = sigmoid(logit),
 *     q^ = q/|q|, R(q^) [App. E, rotation matrix], Sigma = R S S^T R^T
 *     [gradient-flow figure];
 *   - world->camera t = R_cw mu + t_cw, pinhole mean mu' = (fx tx/tz + cx,
 *     fy ty/tz + cy) [App. E, pixel coordinates], EWA Jacobian J with the
 *     focal lengths [App. D.3, dJ/dt], Sigma' = J R_cw Sigma R_cw^T J^T
 *     [App. C.1], low-pass Sigma' + s I and the anti-aliased opacity
 *     compensation [App. A, anti-aliasing];
 *   - conic = (Sigma' + sI)^-1, radius ceil(3 sqrt(lambda_max)) and its
 *     axis-aligned pixel box [App. C.2];
 *   - real spherical-harmonics colour up to degree 3 along the view
 *     direction [App. C.1];
 *   - per-pixel front-to-back compositing over ALL visible Gaussians sorted
 *     by (depth, index), no tiles [App. C.2, discrete rendering sum];
 *   - the analytic backward [App. D.2-D.4];
 *   - the tile binning / sorting result by direct enumeration [App. C.2].
 *
 * Readings where the paper is silent (also listed in the design notes):
 *   alpha = min(0.99, o e^-sigma); alpha < 1/255 is skipped; a Gaussian that
 *   would push T below 1e-4 is excluded and ends the pixel; culled iff
 *   t_z < near; a Gaussian supports pixel (i,j) iff i is in
 *   [ceil(mu'x - r - 0.5), floor(mu'x + r - 0.5)] (same for j), so the image
 *   does not depend on the tile size; background C += T_final * bg.
 *
 * Compile: gcc -O2 -fopenmp -ffp-contract=off -shared -fPIC (no fast-math).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_EXPORT __attribute__((visibility("default")))

/* ------------------------------------------------------------------ */
/* small dense helpers (row-major)                                     */
/* ------------------------------------------------------------------ */

/* Rotation matrix of a unit quaternion (w,x,y,z), Hamilton convention [App. E]. */
static void quat_to_rot(const double q[4], double R[9]) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1.0 - 2.0 * (y * y + z * z);
    R[1] = 2.0 * (x * y - w * z);
    R[2] = 2.0 * (x * z + w * y);
    R[3] = 2.0 * (x * y + w * z);
    R[4] = 1.0 - 2.0 * (x * x + z * z);
    R[5] = 2.0 * (y * z - w * x);
    R[6] = 2.0 * (x * z - w * y);
    R[7] = 2.0 * (y * z + w * x);
    R[8] = 1.0 - 2.0 * (x * x + y * y);
}

/* C (m x n) = A (m x k) B (k x n) */
static void matmul(const double *A, const double *B, double *Cm, int m, int k, int n) {
    for (int i = 0; i < m; i++)
        for (int j = 0; j < n; j++) {
            double s = 0.0;
            for (int l = 0; l < k; l++) s += A[i * k + l] * B[l * n + j];
            Cm[i * n + j] = s;
        }
}

/* B (n x m) = A^T for A (m x n) */
static void transpose(const double *A, double *B, int m, int n) {
    for (int i = 0; i < m; i++)
        for (int j = 0; j < n; j++) B[j * m + i] = A[i * n + j];
}

static double sigmoid(double x) { return 1.0 / (1.0 + exp(-x)); }

/* ------------------------------------------------------------------ */
/* forward pieces shared by projection and its backward                */
/* ------------------------------------------------------------------ */

typedef struct {
    double s[3];      /* activated scales */
    double qn;        /* |q| */
    double qh[4];     /* normalised quaternion */
    double R[9];      /* R(q^) */
    double M[9];      /* R S */
    double Sig[9];    /* M M^T */
    double o;         /* sigmoid(logit) */
} gauss3d;

static void gauss3d_eval(const double *mean, const double *quat, const double *log_scale,
                         double logit, gauss3d *g) {
    (void)mean;
    for (int i = 0; i < 3; i++) g->s[i] = exp(log_scale[i]);
    double n2 = quat[0] * quat[0] + quat[1] * quat[1] + quat[2] * quat[2] + quat[3] * quat[3];
    g->qn = sqrt(n2);
    for (int i = 0; i < 4; i++) g->qh[i] = quat[i] / g->qn;
    quat_to_rot(g->qh, g->R);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) g->M[i * 3 + j] = g->R[i * 3 + j] * g->s[j];
    double Mt[9];
    transpose(g->M, Mt, 3, 3);
    matmul(g->M, Mt, g->Sig, 3, 3, 3);
    g->o = sigmoid(logit);
}

typedef struct {
    int visible;
    double t[3];       /* camera-space mean */
    double mu2[2];     /* pixel-space mean */
    double J[6];       /* 2x3 */
    double T[6];       /* J W, 2x3 */
    double cov0[3];    /* Sigma' before the low-pass (a, b, c) */
    double cov[3];     /* Sigma' + s I */
    double conic[3];   /* (Sigma' + s I)^-1 */
    double comp;       /* anti-aliasing compensation (1 in classic mode) */
    double opac;       /* o~ * comp */
    int radius;
    int box[4];        /* x0, x1, y0, y1 inclusive pixel indices */
} splat2d;

/* Pixel box of the support rule: i in [ceil(mx - r - 0.5), floor(mx + r - 0.5)] clipped to
 * the image.  Returns 0 when empty. */
static int pixel_box(double mx, double my, int r, int W, int H, int box[4]) {
    double x0 = ceil(mx - (double)r - 0.5), x1 = floor(mx + (double)r - 0.5);
    double y0 = ceil(my - (double)r - 0.5), y1 = floor(my + (double)r - 0.5);
    if (x0 < 0.0) x0 = 0.0;
    if (y0 < 0.0) y0 = 0.0;
    if (x1 > (double)(W - 1)) x1 = (double)(W - 1);
    if (y1 > (double)(H - 1)) y1 = (double)(H - 1);
    if (x0 > x1 || y0 > y1) {
        box[0] = 0; box[1] = -1; box[2] = 0; box[3] = -1;
        return 0;
    }
    box[0] = (int)x0; box[1] = (int)x1; box[2] = (int)y0; box[3] = (int)y1;
    return 1;
}

static void splat_eval(const gauss3d *g, const double *mean, const double *vm, const double *intr,
                       int W, int H, double eps2d, double near_plane, int antialiased, splat2d *sp) {
    const double Wr[9] = {vm[0], vm[1], vm[2], vm[4], vm[5], vm[6], vm[8], vm[9], vm[10]};
    const double tw[3] = {vm[3], vm[7], vm[11]};
    const double fx = intr[0], fy = intr[1], cx = intr[2], cy = intr[3];
    memset(sp, 0, sizeof(*sp));
    for (int i = 0; i < 3; i++)
        sp->t[i] = Wr[i * 3 + 0] * mean[0] + Wr[i * 3 + 1] * mean[1] + Wr[i * 3 + 2] * mean[2] + tw[i];
    double tx = sp->t[0], ty = sp->t[1], tz = sp->t[2];
    if (!(tz >= near_plane)) return; /* culled */
    sp->mu2[0] = fx * tx / tz + cx;
    sp->mu2[1] = fy * ty / tz + cy;
    sp->J[0] = fx / tz; sp->J[1] = 0.0;     sp->J[2] = -fx * tx / (tz * tz);
    sp->J[3] = 0.0;     sp->J[4] = fy / tz; sp->J[5] = -fy * ty / (tz * tz);
    matmul(sp->J, Wr, sp->T, 2, 3, 3);
    double TS[6], Tt[6], C2[4];
    matmul(sp->T, g->Sig, TS, 2, 3, 3);
    transpose(sp->T, Tt, 2, 3);
    matmul(TS, Tt, C2, 2, 3, 2);
    sp->cov0[0] = C2[0]; sp->cov0[1] = 0.5 * (C2[1] + C2[2]); sp->cov0[2] = C2[3];
    sp->cov[0] = sp->cov0[0] + eps2d; sp->cov[1] = sp->cov0[1]; sp->cov[2] = sp->cov0[2] + eps2d;
    double det = sp->cov[0] * sp->cov[2] - sp->cov[1] * sp->cov[1];
    if (!(det > 0.0)) return;
    sp->conic[0] = sp->cov[2] / det;
    sp->conic[1] = -sp->cov[1] / det;
    sp->conic[2] = sp->cov[0] / det;
    sp->comp = 1.0;
    if (antialiased) {
        double det0 = sp->cov0[0] * sp->cov0[2] - sp->cov0[1] * sp->cov0[1];
        double ratio = det0 / det;
        sp->comp = sqrt(ratio > 0.0 ? ratio : 0.0);
    }
    sp->opac = g->o * sp->comp;
    double m = 0.5 * (sp->cov[0] + sp->cov[2]);
    double disc = m * m - det;
    double lam = m + sqrt(disc > 0.0 ? disc : 0.0);
    double rr = ceil(3.0 * sqrt(lam));
    if (!(rr > 0.0) || rr > 1.0e7) return; /* a splat wider than 1e7 pixels is culled */
    sp->radius = (int)rr;
    if (!pixel_box(sp->mu2[0], sp->mu2[1], sp->radius, W, H, sp->box)) {
        sp->radius = 0;
        return;
    }
    sp->visible = 1;
}

/* ------------------------------------------------------------------ */
/* projection [App. C.1, App. E, App. A anti-aliasing]                  */
/* ------------------------------------------------------------------ */

ORC_EXPORT void orc_project(int N, const double *means, const double *quats, const double *log_scales,
                            const double *logits, const double *viewmat, const double *intr, int W, int H,
                            double eps2d, double near_plane, int antialiased,
                            double *means2d, double *depths, double *conics, double *cov2d, int *radii,
                            double *opac, int *boxes) {
#pragma omp parallel for schedule(static)
    for (int n = 0; n < N; n++) {
        gauss3d g;
        splat2d sp;
        gauss3d_eval(means + 3 * n, quats + 4 * n, log_scales + 3 * n, logits[n], &g);
        splat_eval(&g, means + 3 * n, viewmat, intr, W, H, eps2d, near_plane, antialiased, &sp);
        means2d[2 * n] = sp.mu2[0];
        means2d[2 * n + 1] = sp.mu2[1];
        depths[n] = sp.t[2];
        for (int k = 0; k < 3; k++) {
            conics[3 * n + k] = sp.conic[k];
            cov2d[3 * n + k] = sp.cov[k];
        }
        radii[n] = sp.visible ? sp.radius : 0;
        opac[n] = sp.opac;
        for (int k = 0; k < 4; k++) boxes[4 * n + k] = sp.box[k];
    }
}

/* ------------------------------------------------------------------ */
/* real spherical harmonics, degrees 0..3 [App. C.1, colour SH(dir)]    */
/*                                                                    */
/* Y_{l,m} = sqrt(2) Re Y_l^m (m>0), sqrt(2) Im Y_l^|m| (m<0), Y_l^0,   */
/* from the complex harmonics with the Condon-Shortley phase, written  */
/* as polynomials of the unit direction (x, y, z), order m = -l..l.     */
/* ------------------------------------------------------------------ */

static void sh_basis(int deg, double x, double y, double z, double *Y) {
    const double pi = 3.14159265358979323846;
    const double k0 = 0.5 * sqrt(1.0 / pi);
    const double k1 = sqrt(3.0 / (4.0 * pi));
    Y[0] = k0;
    if (deg < 1) return;
    Y[1] = -k1 * y;
    Y[2] = k1 * z;
    Y[3] = -k1 * x;
    if (deg < 2) return;
    const double k2a = 0.5 * sqrt(15.0 / pi);  /* m = +-1, -2 */
    const double k2b = 0.25 * sqrt(5.0 / pi);  /* m = 0 */
    const double k2c = 0.25 * sqrt(15.0 / pi); /* m = 2 */
    Y[4] = k2a * x * y;
    Y[5] = -k2a * y * z;
    Y[6] = k2b * (2.0 * z * z - x * x - y * y);
    Y[7] = -k2a * x * z;
    Y[8] = k2c * (x * x - y * y);
    if (deg < 3) return;
    const double k3a = 0.25 * sqrt(35.0 / (2.0 * pi)); /* m = +-3 */
    const double k3b = 0.5 * sqrt(105.0 / pi);         /* m = -2 */
    const double k3c = 0.25 * sqrt(21.0 / (2.0 * pi)); /* m = +-1 */
    const double k3d = 0.25 * sqrt(7.0 / pi);          /* m = 0 */
    const double k3e = 0.25 * sqrt(105.0 / pi);        /* m = 2 */
    Y[9] = -k3a * y * (3.0 * x * x - y * y);
    Y[10] = k3b * x * y * z;
    Y[11] = -k3c * y * (4.0 * z * z - x * x - y * y);
    Y[12] = k3d * z * (2.0 * z * z - 3.0 * x * x - 3.0 * y * y);
    Y[13] = -k3c * x * (4.0 * z * z - x * x - y * y);
    Y[14] = k3e * z * (x * x - y * y);
    Y[15] = -k3a * x * (x * x - 3.0 * y * y);
}

/* Gradient of each basis polynomial with respect to (x, y, z), dY[k*3 + axis]. */
static void sh_basis_grad(int deg, double x, double y, double z, double *dY) {
    const double pi = 3.14159265358979323846;
    int K = (deg + 1) * (deg + 1);
    for (int i = 0; i < 3 * K; i++) dY[i] = 0.0;
    if (deg < 1) return;
    const double k1 = sqrt(3.0 / (4.0 * pi));
    dY[3 * 1 + 1] = -k1;
    dY[3 * 2 + 2] = k1;
    dY[3 * 3 + 0] = -k1;
    if (deg < 2) return;
    const double k2a = 0.5 * sqrt(15.0 / pi);
    const double k2b = 0.25 * sqrt(5.0 / pi);
    const double k2c = 0.25 * sqrt(15.0 / pi);
    dY[3 * 4 + 0] = k2a * y;          dY[3 * 4 + 1] = k2a * x;
    dY[3 * 5 + 1] = -k2a * z;         dY[3 * 5 + 2] = -k2a * y;
    dY[3 * 6 + 0] = -2.0 * k2b * x;   dY[3 * 6 + 1] = -2.0 * k2b * y;  dY[3 * 6 + 2] = 4.0 * k2b * z;
    dY[3 * 7 + 0] = -k2a * z;         dY[3 * 7 + 2] = -k2a * x;
    dY[3 * 8 + 0] = 2.0 * k2c * x;    dY[3 * 8 + 1] = -2.0 * k2c * y;
    if (deg < 3) return;
    const double k3a = 0.25 * sqrt(35.0 / (2.0 * pi));
    const double k3b = 0.5 * sqrt(105.0 / pi);
    const double k3c = 0.25 * sqrt(21.0 / (2.0 * pi));
    const double k3d = 0.25 * sqrt(7.0 / pi);
    const double k3e = 0.25 * sqrt(105.0 / pi);
    /* Y9 = -k3a (3 x^2 y - y^3) */
    dY[3 * 9 + 0] = -k3a * 6.0 * x * y;
    dY[3 * 9 + 1] = -k3a * (3.0 * x * x - 3.0 * y * y);
    /* Y10 = k3b x y z */
    dY[3 * 10 + 0] = k3b * y * z; dY[3 * 10 + 1] = k3b * x * z; dY[3 * 10 + 2] = k3b * x * y;
    /* Y11 = -k3c (4 y z^2 - x^2 y - y^3) */
    dY[3 * 11 + 0] = -k3c * (-2.0 * x * y);
    dY[3 * 11 + 1] = -k3c * (4.0 * z * z - x * x - 3.0 * y * y);
    dY[3 * 11 + 2] = -k3c * (8.0 * y * z);
    /* Y12 = k3d (2 z^3 - 3 x^2 z - 3 y^2 z) */
    dY[3 * 12 + 0] = k3d * (-6.0 * x * z);
    dY[3 * 12 + 1] = k3d * (-6.0 * y * z);
    dY[3 * 12 + 2] = k3d * (6.0 * z * z - 3.0 * x * x - 3.0 * y * y);
    /* Y13 = -k3c (4 x z^2 - x^3 - x y^2) */
    dY[3 * 13 + 0] = -k3c * (4.0 * z * z - 3.0 * x * x - y * y);
    dY[3 * 13 + 1] = -k3c * (-2.0 * x * y);
    dY[3 * 13 + 2] = -k3c * (8.0 * x * z);
    /* Y14 = k3e (x^2 z - y^2 z) */
    dY[3 * 14 + 0] = k3e * 2.0 * x * z;
    dY[3 * 14 + 1] = -k3e * 2.0 * y * z;
    dY[3 * 14 + 2] = k3e * (x * x - y * y);
    /* Y15 = -k3a (x^3 - 3 x y^2) */
    dY[3 * 15 + 0] = -k3a * (3.0 * x * x - 3.0 * y * y);
    dY[3 * 15 + 1] = -k3a * (-6.0 * x * y);
}

ORC_EXPORT void orc_sh_basis(int deg, int P, const double *dirs, double *Y) {
    int K = (deg + 1) * (deg + 1);
    for (int p = 0; p < P; p++) sh_basis(deg, dirs[3 * p], dirs[3 * p + 1], dirs[3 * p + 2], Y + K * p);
}

ORC_EXPORT void orc_sh_basis_grad(int deg, int P, const double *dirs, double *dY) {
    int K = (deg + 1) * (deg + 1);
    for (int p = 0; p < P; p++)
        sh_basis_grad(deg, dirs[3 * p], dirs[3 * p + 1], dirs[3 * p + 2], dY + 3 * K * p);
}

/* Camera centre in world coordinates: -R_cw^T t_cw. */
static void camera_centre(const double *vm, double c[3]) {
    for (int i = 0; i < 3; i++) c[i] = -(vm[0 + i] * vm[3] + vm[4 + i] * vm[7] + vm[8 + i] * vm[11]);
}

/* colour = max(0, sum_k Y_k(dir) coeff_k + 0.5), dir = (mu - centre)/|mu - centre|. */
ORC_EXPORT void orc_sh_colors(int N, int deg, const double *sh, const double *means, const double *viewmat,
                              double *colors, double *raw) {
    int K = (deg + 1) * (deg + 1);
    double cc[3];
    camera_centre(viewmat, cc);
#pragma omp parallel for schedule(static)
    for (int n = 0; n < N; n++) {
        double v[3], Y[16];
        for (int i = 0; i < 3; i++) v[i] = means[3 * n + i] - cc[i];
        double len = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        sh_basis(deg, v[0] / len, v[1] / len, v[2] / len, Y);
        for (int ch = 0; ch < 3; ch++) {
            double s = 0.0;
            for (int k = 0; k < K; k++) s += Y[k] * sh[(n * K + k) * 3 + ch];
            s += 0.5;
            raw[3 * n + ch] = s;
            colors[3 * n + ch] = s > 0.0 ? s : 0.0;
        }
    }
}

/* d_viewmat (16, may be NULL) accumulates the pose gradient of the view direction [App. A,
   pose optimization]: the centre c = -R^T t, v = mu - c, so dL/dc = -dL/dv and
   dL/dR_ij += t_i dL/dv_j, dL/dt_i += sum_j R_ij dL/dv_j. */
ORC_EXPORT void orc_sh_bwd(int N, int deg, const double *sh, const double *means, const double *viewmat,
                           const double *d_colors, double *d_sh, double *d_means, double *d_viewmat) {
    int K = (deg + 1) * (deg + 1);
    double cc[3];
    camera_centre(viewmat, cc);
#pragma omp parallel for schedule(static)
    for (int n = 0; n < N; n++) {
        double v[3], Y[16], dY[48], dir[3], g[3];
        for (int i = 0; i < 3; i++) v[i] = means[3 * n + i] - cc[i];
        double len = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        for (int i = 0; i < 3; i++) dir[i] = v[i] / len;
        sh_basis(deg, dir[0], dir[1], dir[2], Y);
        sh_basis_grad(deg, dir[0], dir[1], dir[2], dY);
        for (int ch = 0; ch < 3; ch++) {
            double s = 0.5;
            for (int k = 0; k < K; k++) s += Y[k] * sh[(n * K + k) * 3 + ch];
            g[ch] = s > 0.0 ? d_colors[3 * n + ch] : 0.0; /* clamp at 0 passes no gradient */
        }
        double ddir[3] = {0.0, 0.0, 0.0};
        for (int k = 0; k < K; k++) {
            double w = 0.0;
            for (int ch = 0; ch < 3; ch++) {
                d_sh[(n * K + k) * 3 + ch] += Y[k] * g[ch];
                w += sh[(n * K + k) * 3 + ch] * g[ch];
            }
            for (int i = 0; i < 3; i++) ddir[i] += w * dY[3 * k + i];
        }
        /* d dir / d v = (I - dir dir^T) / |v| */
        double dd = dir[0] * ddir[0] + dir[1] * ddir[1] + dir[2] * ddir[2];
        double dv[3];
        for (int i = 0; i < 3; i++) {
            dv[i] = (ddir[i] - dir[i] * dd) / len;
            d_means[3 * n + i] += dv[i];
        }
        if (d_viewmat) {
            for (int i = 0; i < 3; i++) {
                for (int j = 0; j < 3; j++) {
#pragma omp atomic
                    d_viewmat[4 * i + j] += viewmat[4 * i + 3] * dv[j];
                }
                double r = viewmat[4 * i] * dv[0] + viewmat[4 * i + 1] * dv[1] + viewmat[4 * i + 2] * dv[2];
#pragma omp atomic
                d_viewmat[4 * i + 3] += r;
            }
        }
    }
}

/* ------------------------------------------------------------------ */
/* compositing [App. C.2]                                              */
/* ------------------------------------------------------------------ */

static const double *g_sort_depths; /* qsort has no context argument; guarded by a critical */

static int cmp_depth_index(const void *a, const void *b) {
    int ia = *(const int *)a, ib = *(const int *)b;
    double da = g_sort_depths[ia], db = g_sort_depths[ib];
    if (da < db) return -1;
    if (da > db) return 1;
    return (ia > ib) - (ia < ib);
}

/* Indices of visible Gaussians sorted by (depth, index). */
static int *depth_order(int N, const double *depths, const int *radii, int *count) {
    int *ord = (int *)malloc(sizeof(int) * (size_t)(N > 0 ? N : 1));
    int m = 0;
    for (int n = 0; n < N; n++)
        if (radii[n] > 0) ord[m++] = n;
#pragma omp critical(orc_sort)
    {
        g_sort_depths = depths;
        qsort(ord, (size_t)m, sizeof(int), cmp_depth_index);
    }
    *count = m;
    return ord;
}

typedef struct {
    int id;
    double alpha, T, G, dx, dy;
    int clamped;
} contrib;

/* Composite one pixel.  Fills up to 'cap' contributors into 'list' when non-NULL.
 * Returns the number of contributors; outputs colour, T_final and evaluated-pair count. */
static int composite_pixel(int px, int py, int M, const int *ord, const double *means2d,
                           const double *conics, const double *opac, const double *colors, int ch,
                           const int *boxes, const double *bg, double alpha_min, double alpha_max,
                           double T_min, double *out_col, double *out_T, long long *out_blends,
                           contrib *list) {
    double T = 1.0;
    int nc = 0;
    long long blends = 0;
    for (int c = 0; c < ch; c++) out_col[c] = 0.0;
    double pxc = px + 0.5, pyc = py + 0.5; /* pixel centre [App. E] */
    for (int j = 0; j < M; j++) {
        int n = ord[j];
        const int *b = boxes + 4 * n;
        if (px < b[0] || px > b[1] || py < b[2] || py > b[3]) continue;
        blends++;
        double dx = pxc - means2d[2 * n], dy = pyc - means2d[2 * n + 1];
        const double *Y = conics + 3 * n;
        double sigma = 0.5 * (Y[0] * dx * dx + Y[2] * dy * dy) + Y[1] * dx * dy;
        if (sigma < 0.0) continue;
        double G = exp(-sigma);
        double a = opac[n] * G;
        int clamped = 0;
        if (a > alpha_max) { a = alpha_max; clamped = 1; }
        if (a < alpha_min) continue;
        double Tn = T * (1.0 - a);
        if (Tn < T_min) break; /* excluded; the pixel is finished */
        for (int c = 0; c < ch; c++) out_col[c] += colors[(size_t)n * ch + c] * a * T;
        if (list) {
            list[nc].id = n; list[nc].alpha = a; list[nc].T = T; list[nc].G = G;
            list[nc].dx = dx; list[nc].dy = dy; list[nc].clamped = clamped;
        }
        nc++;
        T = Tn;
    }
    for (int c = 0; c < ch; c++) out_col[c] += T * (bg ? bg[c] : 0.0);
    *out_T = T;
    *out_blends = blends;
    return nc;
}

/* Render P pixels (linear indices y*W + x) or all pixels when pix == NULL. */
ORC_EXPORT void orc_render(int N, const double *means2d, const double *conics, const double *opac,
                           const double *colors, int ch, const double *depths, const int *radii,
                           const int *boxes, int W, int H, const double *bg, double alpha_min,
                           double alpha_max, double T_min, int P, const int *pix, double *out_col,
                           double *out_T, int *out_ncontrib, long long *out_blends) {
    int M;
    int *ord = depth_order(N, depths, radii, &M);
    int total = pix ? P : W * H;
#pragma omp parallel for schedule(dynamic, 16)
    for (int p = 0; p < total; p++) {
        int lin = pix ? pix[p] : p;
        int px = lin % W, py = lin / W;
        long long bl;
        out_ncontrib[p] = composite_pixel(px, py, M, ord, means2d, conics, opac, colors, ch, boxes, bg,
                                          alpha_min, alpha_max, T_min, out_col + (size_t)p * ch,
                                          out_T + p, &bl, NULL);
        out_blends[p] = bl;
    }
    free(ord);
}

/* Contributors of one pixel in front-to-back order: ids, alpha_n and T_n (before blending n). */
ORC_EXPORT int orc_render_trace(int N, const double *means2d, const double *conics, const double *opac,
                                const double *colors, int ch, const double *depths, const int *radii,
                                const int *boxes, int px, int py, const double *bg, double alpha_min,
                                double alpha_max, double T_min, int cap, int *ids, double *alphas,
                                double *Ts) {
    int M;
    int *ord = depth_order(N, depths, radii, &M);
    contrib *list = (contrib *)malloc(sizeof(contrib) * (size_t)(M > 0 ? M : 1));
    double col[64], T;
    long long bl;
    int nc = composite_pixel(px, py, M, ord, means2d, conics, opac, colors, ch, boxes, bg, alpha_min,
                             alpha_max, T_min, col, &T, &bl, list);
    for (int i = 0; i < nc && i < cap; i++) {
        ids[i] = list[i].id; alphas[i] = list[i].alpha; Ts[i] = list[i].T;
    }
    free(list);
    free(ord);
    return nc;
}

/* Every contributor multiplies T by (1 - alpha) <= 1 - alpha_min and T stays >= T_min, so a
 * pixel has at most log(T_min) / log(1 - alpha_min) + 1 contributors (and never more than M). */
static size_t contrib_bound(int M, double alpha_min, double T_min) {
    size_t cap = (size_t)(M > 0 ? M : 1);
    if (alpha_min > 0.0 && alpha_min < 1.0 && T_min > 0.0 && T_min < 1.0) {
        double b = ceil(log(T_min) / log1p(-alpha_min)) + 2.0;
        if (b < (double)cap) cap = (size_t)b;
    }
    return cap;
}

static void atomic_add(double *p, double v) {
#pragma omp atomic
    *p += v;
}

/* Backward of the compositing sum [App. D.2]: per pixel, back to front with
 * T_{n-1} = T_n / (1 - alpha_{n-1}) and the suffix S_n = sum_{m>n} c_m alpha_m T_m
 * (here S starts at T_final * bg so the background term is included).  Gradients
 * accumulate (+=) into per-Gaussian 2D buffers. */
ORC_EXPORT void orc_render_bwd(int N, const double *means2d, const double *conics, const double *opac,
                               const double *colors, int ch, const double *depths, const int *radii,
                               const int *boxes, int W, int H, const double *bg, double alpha_min,
                               double alpha_max, double T_min, int P, const int *pix, const double *d_col,
                               const double *d_alpha, double *d_means2d, double *d_conics, double *d_opac,
                               double *d_colors, double *absgrad) {
    int M;
    int *ord = depth_order(N, depths, radii, &M);
    int total = pix ? P : W * H;
    size_t cap = contrib_bound(M, alpha_min, T_min);
#pragma omp parallel
    {
        contrib *list = (contrib *)malloc(sizeof(contrib) * cap);
        double *S = (double *)malloc(sizeof(double) * (size_t)ch);
        double *col = (double *)malloc(sizeof(double) * (size_t)ch);
#pragma omp for schedule(dynamic, 16)
        for (int p = 0; p < total; p++) {
            int lin = pix ? pix[p] : p;
            int px = lin % W, py = lin / W;
            double Tf;
            long long bl;
            int nc = composite_pixel(px, py, M, ord, means2d, conics, opac, colors, ch, boxes, bg,
                                     alpha_min, alpha_max, T_min, col, &Tf, &bl, list);
            const double *g = d_col + (size_t)p * ch;
            double gA = d_alpha ? d_alpha[p] : 0.0;
            for (int c = 0; c < ch; c++) S[c] = Tf * (bg ? bg[c] : 0.0);
            for (int k = nc - 1; k >= 0; k--) {
                const contrib *e = list + k;
                int n = e->id;
                double a = e->alpha, T = e->T;
                const double *cn = colors + (size_t)n * ch;
                /* dC/dc_n = alpha_n T_n */
                for (int c = 0; c < ch; c++) atomic_add(&d_colors[(size_t)n * ch + c], a * T * g[c]);
                /* dC/dalpha_n = c_n T_n - S_n / (1 - alpha_n); alpha output A = 1 - T_final */
                double da = 0.0;
                for (int c = 0; c < ch; c++) da += g[c] * (cn[c] * T - S[c] / (1.0 - a));
                da += gA * Tf / (1.0 - a);
                for (int c = 0; c < ch; c++) S[c] += cn[c] * a * T;
                if (e->clamped) da = 0.0; /* alpha = alpha_max: no gradient */
                /* alpha = o G, G = exp(-sigma) */
                double d_o = e->G * da;
                double d_sigma = -opac[n] * e->G * da;
                const double *Y = conics + 3 * n;
                /* sigma = 1/2 D^T Y D, D = p - mu'  =>  d sigma / d mu' = -Y D */
                double gx = -d_sigma * (Y[0] * e->dx + Y[1] * e->dy);
                double gy = -d_sigma * (Y[1] * e->dx + Y[2] * e->dy);
                atomic_add(&d_means2d[2 * n], gx);
                atomic_add(&d_means2d[2 * n + 1], gy);
                if (absgrad) {
                    atomic_add(&absgrad[2 * n], fabs(gx));
                    atomic_add(&absgrad[2 * n + 1], fabs(gy));
                }
                /* d sigma / d(a, b, c) for Y = [[a, b], [b, c]] */
                atomic_add(&d_conics[3 * n], 0.5 * d_sigma * e->dx * e->dx);
                atomic_add(&d_conics[3 * n + 1], d_sigma * e->dx * e->dy);
                atomic_add(&d_conics[3 * n + 2], 0.5 * d_sigma * e->dy * e->dy);
                atomic_add(&d_opac[n], d_o);
            }
        }
        free(col);
        free(S);
        free(list);
    }
    free(ord);
}

/* ------------------------------------------------------------------ */
/* projection backward [App. D.3, D.4, gradient-flow figure]           */
/* ------------------------------------------------------------------ */

/* dR/dw, dR/dx, dR/dy, dR/dz at the unit quaternion (w,x,y,z) [App. D.4]. */
static void drot_dquat(const double q[4], double D[4][9]) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    double Dw[9] = {0, -z, y, z, 0, -x, -y, x, 0};
    double Dx[9] = {0, y, z, y, -2 * x, -w, z, w, -2 * x};
    double Dy[9] = {-2 * y, x, w, x, 0, z, -w, z, -2 * y};
    double Dz[9] = {-2 * z, -w, x, w, -2 * z, y, x, y, 0};
    for (int i = 0; i < 9; i++) {
        D[0][i] = 2 * Dw[i]; D[1][i] = 2 * Dx[i]; D[2][i] = 2 * Dy[i]; D[3][i] = 2 * Dz[i];
    }
}

/* Accumulates (+=) gradients of one camera into the 3D leaves.  d_depths may be NULL.
   d_viewmat (16, may be NULL) accumulates the pose gradient [App. A, pose optimization]:
   through t = R mu + t_w (dR += dt mu^T, dt_w += dt) and through T = J R in
   Sigma' = T Sigma T^T (dR += J^T dT). */
ORC_EXPORT void orc_project_bwd(int N, const double *means, const double *quats, const double *log_scales,
                                const double *logits, const double *viewmat, const double *intr, int W,
                                int H, double eps2d, double near_plane, int antialiased,
                                const double *d_means2d, const double *d_conics, const double *d_opac,
                                const double *d_depths, double *d_means, double *d_quats,
                                double *d_log_scales, double *d_logits, double *d_viewmat) {
    const double *vm = viewmat;
    const double Wr[9] = {vm[0], vm[1], vm[2], vm[4], vm[5], vm[6], vm[8], vm[9], vm[10]};
    const double fx = intr[0], fy = intr[1];
#pragma omp parallel for schedule(static)
    for (int n = 0; n < N; n++) {
        gauss3d g;
        splat2d sp;
        gauss3d_eval(means + 3 * n, quats + 4 * n, log_scales + 3 * n, logits[n], &g);
        splat_eval(&g, means + 3 * n, viewmat, intr, W, H, eps2d, near_plane, antialiased, &sp);
        if (!sp.visible) continue;
        const double *Y = sp.conic;
        /* conic scalars (a,b,c) -> symmetric matrix gradient of Y */
        double dYm[4] = {d_conics[3 * n], 0.5 * d_conics[3 * n + 1], 0.5 * d_conics[3 * n + 1],
                         d_conics[3 * n + 2]};
        double Ym[4] = {Y[0], Y[1], Y[1], Y[2]};
        /* d Sigma' = -Y dY Y   (dY/dx = -Y dSigma'/dx Y)  [App. D.2] */
        double t1[4], G2[4];
        matmul(Ym, dYm, t1, 2, 2, 2);
        matmul(t1, Ym, G2, 2, 2, 2);
        for (int i = 0; i < 4; i++) G2[i] = -G2[i];
        /* opacity: o_eff = o * comp */
        double d_oeff = d_opac[n];
        double d_o = d_oeff * sp.comp;
        if (antialiased && sp.comp > 0.0) {
            /* comp = sqrt(det0 / det1), det0 = ac - b^2 of Sigma', det1 of Sigma' + sI */
            double a = sp.cov0[0], b = sp.cov0[1], c = sp.cov0[2];
            double det0 = a * c - b * b;
            double det1 = sp.cov[0] * sp.cov[2] - sp.cov[1] * sp.cov[1];
            double dcomp = d_oeff * g.o;
            double k = dcomp / (2.0 * sp.comp) / (det1 * det1);
            double ga = k * (c * det1 - det0 * sp.cov[2]);
            double gc = k * (a * det1 - det0 * sp.cov[0]);
            double gb = k * (-2.0 * b * det1 + 2.0 * b * det0);
            G2[0] += ga; G2[3] += gc; G2[1] += 0.5 * gb; G2[2] += 0.5 * gb;
        }
        /* Sigma' = T Sigma T^T:  dSigma = T^T G T,  dT = G T Sigma^T + G^T T Sigma [App. D.3] */
        double Tt[6], GT[6], dSig[9], TS[6], dT[6], G2t[4], tmp[6];
        transpose(sp.T, Tt, 2, 3);
        matmul(G2, sp.T, GT, 2, 2, 3);
        matmul(Tt, GT, dSig, 3, 2, 3);
        double Sigt[9];
        transpose(g.Sig, Sigt, 3, 3);
        matmul(GT, Sigt, dT, 2, 3, 3);
        transpose(G2, G2t, 2, 2);
        matmul(sp.T, g.Sig, TS, 2, 3, 3);
        matmul(G2t, TS, tmp, 2, 2, 3);
        for (int i = 0; i < 6; i++) dT[i] += tmp[i];
        /* T = J R_cw:  dJ = dT R_cw^T */
        double Wt[9], dJ[6];
        transpose(Wr, Wt, 3, 3);
        matmul(dT, Wt, dJ, 2, 3, 3);
        double tx = sp.t[0], ty = sp.t[1], tz = sp.t[2];
        double tz2 = tz * tz, tz3 = tz2 * tz;
        double dt[3] = {0.0, 0.0, 0.0};
        /* through mu' = (fx tx/tz + cx, fy ty/tz + cy) [App. E] */
        double gmx = d_means2d[2 * n], gmy = d_means2d[2 * n + 1];
        dt[0] += gmx * fx / tz;
        dt[1] += gmy * fy / tz;
        dt[2] += -gmx * fx * tx / tz2 - gmy * fy * ty / tz2;
        /* through J: dJ/dtx, dJ/dty, dJ/dtz [App. D.3] */
        dt[0] += dJ[2] * (-fx / tz2);
        dt[1] += dJ[5] * (-fy / tz2);
        dt[2] += dJ[0] * (-fx / tz2) + dJ[2] * (2.0 * fx * tx / tz3) + dJ[4] * (-fy / tz2) +
                 dJ[5] * (2.0 * fy * ty / tz3);
        if (d_depths) dt[2] += d_depths[n];
        /* t = R_cw mu + t_cw:  dmu = R_cw^T dt */
        for (int i = 0; i < 3; i++)
            d_means[3 * n + i] += Wr[0 + i] * dt[0] + Wr[3 + i] * dt[1] + Wr[6 + i] * dt[2];
        if (d_viewmat) {
            /* J = [[fx/tz, 0, -fx tx/tz^2], [0, fy/tz, -fy ty/tz^2]];  dR = J^T dT + dt mu^T */
            double J[6] = {fx / tz, 0.0, -fx * tx / tz2, 0.0, fy / tz, -fy * ty / tz2};
            double Jt[6], dRw[9];
            transpose(J, Jt, 2, 3);
            matmul(Jt, dT, dRw, 3, 2, 3);
            for (int i = 0; i < 3; i++) {
                for (int j = 0; j < 3; j++) {
                    double v = dRw[3 * i + j] + dt[i] * means[3 * n + j];
#pragma omp atomic
                    d_viewmat[4 * i + j] += v;
                }
#pragma omp atomic
                d_viewmat[4 * i + 3] += dt[i];
            }
        }
        /* Sigma = M M^T:  dM = dSigma M + dSigma^T M [App. D.4] */
        double dSigt[9], dM[9], t2[9];
        transpose(dSig, dSigt, 3, 3);
        matmul(dSig, g.M, dM, 3, 3, 3);
        matmul(dSigt, g.M, t2, 3, 3, 3);
        for (int i = 0; i < 9; i++) dM[i] += t2[i];
        /* M = R S:  dR = dM S^T,  dS = R^T dM (diagonal) */
        double dR[9];
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) dR[i * 3 + j] = dM[i * 3 + j] * g.s[j];
        for (int j = 0; j < 3; j++) {
            double dsj = 0.0;
            for (int i = 0; i < 3; i++) dsj += g.R[i * 3 + j] * dM[i * 3 + j];
            d_log_scales[3 * n + j] += dsj * g.s[j]; /* s~ = exp(s) */
        }
        /* R(q^):  dq^_k = <dR, dR/dq^_k> */
        double D[4][9], dqh[4];
        drot_dquat(g.qh, D);
        for (int k2 = 0; k2 < 4; k2++) {
            double s = 0.0;
            for (int i = 0; i < 9; i++) s += dR[i] * D[k2][i];
            dqh[k2] = s;
        }
        /* q^ = q/|q|:  dq = (dq^ - q^ (q^ . dq^)) / |q| */
        double proj = 0.0;
        for (int k2 = 0; k2 < 4; k2++) proj += g.qh[k2] * dqh[k2];
        for (int k2 = 0; k2 < 4; k2++) d_quats[4 * n + k2] += (dqh[k2] - g.qh[k2] * proj) / g.qn;
        /* o~ = sigmoid(logit) */
        d_logits[n] += d_o * g.o * (1.0 - g.o);
    }
}

/* ------------------------------------------------------------------ */
/* tile binning and sorting by enumeration [App. C.2]                  */
/* ------------------------------------------------------------------ */

typedef struct {
    uint64_t key;
    int32_t value;
} kv;

static int cmp_kv(const void *a, const void *b) {
    const kv *x = (const kv *)a, *y = (const kv *)b;
    if (x->key < y->key) return -1;
    if (x->key > y->key) return 1;
    return (x->value > y->value) - (x->value < y->value);
}

static uint32_t f32_bits(float f) {
    uint32_t u;
    memcpy(&u, &f, sizeof(u));
    return u;
}

/* Inputs are the float32 projected means and depths and the integer radii of C cameras
 * ([C,N,2], [C,N], [C,N]).  Every (tile, Gaussian) pair whose tile contains a pixel of the
 * Gaussian's pixel box is listed with key = (global tile << 32) | bits(depth) and
 * value = c N + n, in (key, value) order.  Global tile ids run camera by camera, row-major.
 * Returns K; writes at most 'cap' pairs; ranges[2*t] = [start, end) (0,0 when empty). */
ORC_EXPORT long long orc_bin_sort(int C, int N, const float *means2d, const float *depths,
                                  const int *radii, const int *widths, const int *heights, int tile,
                                  long long cap, uint64_t *keys, int32_t *values, int32_t *ranges) {
    long long total_tiles = 0;
    long long *offs = (long long *)malloc(sizeof(long long) * (size_t)(C + 1));
    for (int c = 0; c < C; c++) {
        offs[c] = total_tiles;
        long long tx = (widths[c] + tile - 1) / tile, ty = (heights[c] + tile - 1) / tile;
        total_tiles += tx * ty;
    }
    offs[C] = total_tiles;
    long long K = 0;
    for (int pass = 0; pass < 2; pass++) {
        kv *buf = NULL;
        if (pass == 1) buf = (kv *)malloc(sizeof(kv) * (size_t)(K > 0 ? K : 1));
        long long k = 0;
        for (int c = 0; c < C; c++) {
            int W = widths[c], H = heights[c];
            long long tiles_x = (W + tile - 1) / tile;
            for (int n = 0; n < N; n++) {
                size_t i = (size_t)c * N + n;
                int r = radii[i];
                if (r <= 0) continue;
                int box[4];
                if (!pixel_box((double)means2d[2 * i], (double)means2d[2 * i + 1], r, W, H, box)) continue;
                for (int ty = box[2] / tile; ty <= box[3] / tile; ty++)
                    for (int tx = box[0] / tile; tx <= box[1] / tile; tx++) {
                        if (pass == 1) {
                            uint64_t gt = (uint64_t)(offs[c] + ty * tiles_x + tx);
                            buf[k].key = (gt << 32) | (uint64_t)f32_bits(depths[i]);
                            buf[k].value = (int32_t)i;
                        }
                        k++;
                    }
            }
        }
        if (pass == 0) {
            K = k;
            continue;
        }
        qsort(buf, (size_t)K, sizeof(kv), cmp_kv);
        for (long long t = 0; t < total_tiles; t++) { ranges[2 * t] = 0; ranges[2 * t + 1] = 0; }
        for (long long j = 0; j < K; j++) {
            if (j < cap) { keys[j] = buf[j].key; values[j] = buf[j].value; }
            long long t = (long long)(buf[j].key >> 32);
            if (j == 0 || (buf[j - 1].key >> 32) != (uint64_t)t) ranges[2 * t] = (int32_t)j;
            if (j == K - 1 || (buf[j + 1].key >> 32) != (uint64_t)t) ranges[2 * t + 1] = (int32_t)(j + 1);
        }
        free(buf);
    }
    free(offs);
    return K;
}

ORC_EXPORT int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* single-step exports used by the oracle's own pin tests              */
/* ------------------------------------------------------------------ */

/* R(q/|q|) [App. E]. */
ORC_EXPORT void orc_rotation(const double *q, double *R) {
    double n = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    double qh[4] = {q[0] / n, q[1] / n, q[2] / n, q[3] / n};
    quat_to_rot(qh, R);
}

/* dR/dw, dR/dx, dR/dy, dR/dz at a unit quaternion, 4 x 9 [App. D.4]. */
ORC_EXPORT void orc_drot(const double *q, double *D) {
    double M[4][9];
    drot_dquat(q, M);
    for (int k = 0; k < 4; k++)
        for (int i = 0; i < 9; i++) D[9 * k + i] = M[k][i];
}

/* Sigma = R S S^T R^T with S = diag(exp(log_scale)). */
ORC_EXPORT void orc_cov3d(const double *quat, const double *log_scale, double *Sig) {
    gauss3d g;
    double zero[3] = {0.0, 0.0, 0.0};
    gauss3d_eval(zero, quat, log_scale, 0.0, &g);
    for (int i = 0; i < 9; i++) Sig[i] = g.Sig[i];
}
