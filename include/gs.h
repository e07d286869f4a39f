/*
 * gs.h -- C ABI of libgs, a GB300 (sm_103a) implementation of the
 * differentiable tile-based Gaussian rasterizer described in
 * "gsplat: An Open-Source Library for Gaussian Splatting" (arXiv 2409.06765),
 * App. C (forward), App. D (backward), App. E (conventions), App. A
 * (anti-aliasing, depth, absgrad).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - All array arguments are DEVICE pointers to contiguous, row-major data
 *    (float32 / int32 / uint64) owned and allocated by the caller, except the
 *    camera array, the parameter struct and `background`, which live in HOST
 *    memory and are read during the call only.  The library never allocates
 *    device memory and never synchronises the stream: every call enqueues
 *    kernels on `stream` (a cudaStream_t, NULL = legacy default stream) and
 *    returns.  Device-side results (such as the intersection count) are valid
 *    once the stream reaches them.
 *  - Cameras: C cameras of possibly different sizes are rendered in one call.
 *    Per-(camera, Gaussian) arrays are laid out [C, N, ...].  Per-pixel arrays
 *    pack the cameras' images one after the other: camera c starts at pixel
 *    sum_{c'<c} H_c' * W_c', then rows of W_c pixels (y-major), then channels.
 *    Tiles are numbered globally: camera by camera, row-major within a camera.
 *  - Errors: host-side validation (NULL pointers, sizes, unsupported options)
 *    returns a negative gs_status and enqueues nothing.  A failed kernel launch
 *    returns GS_ERR_CUDA; gs_last_error() then describes it (per thread).
 *  - Gradient outputs of gs_rasterize_bwd are ACCUMULATED (+=) with atomics:
 *    the caller zeroes them first.  The per-Gaussian backward helpers state
 *    their own write/accumulate rule below.
 */
#ifndef GS_H_
#define GS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define GS_API __attribute__((visibility("default")))
#else
#define GS_API
#endif

typedef int32_t gs_status;
#define GS_OK 0
#define GS_ERR_ARG -1         /* invalid argument (NULL pointer, size, option) */
#define GS_ERR_CUDA -2        /* a CUDA launch or query failed; see gs_last_error() */
#define GS_ERR_CAPACITY -3    /* a caller-provided buffer is too small */
#define GS_ERR_UNSUPPORTED -5 /* option combination not compiled into this library */

#define GS_MAX_CAMERAS 32     /* cameras per call */
#define GS_MAX_CHANNELS 64    /* feature channels per Gaussian */
#define GS_MAX_INTERSECTIONS 2147483647ll /* (tile, Gaussian) pairs of one gs_tile_bin_sort call: list
                                             positions (values, tile_ranges) are int32 */

/* Pinhole camera [App. C.1, App. E].  viewmat maps world to camera coordinates
 * (x right, y down, z forward), row-major 4x4; its last row is ignored.  A camera
 * point t projects to the continuous pixel position (fx tx/tz + cx, fy ty/tz + cy),
 * pixel (i, j) having its centre at (i + 0.5, j + 0.5). */
typedef struct gs_camera {
    int32_t width, height;
    float viewmat[16];
    float fx, fy, cx, cy;
} gs_camera;

/* Rasterizer options.  gs_default_params() fills the values used throughout the
 * paper's classic mode: 16x16 tiles [App. C.2], low-pass s = 0.3 [App. A],
 * near plane 0.01, alpha in [1/255, 0.99], transmittance floor 1e-4. */
typedef struct gs_params {
    int32_t tile;         /* tile edge in pixels: 8, 16 or 32 */
    int32_t batch_depth;  /* Gaussians staged in shared memory per batch: 32..1024, multiple of 32.
                             A staged entry takes 48 bytes plus 16 per 4 channels; a batch beyond
                             the 227 KB of shared memory of one CTA (e.g. 1024 entries with 64
                             channels) returns GS_ERR_UNSUPPORTED. */
    int32_t antialiased;  /* 0: classic mode; 1: opacity * sqrt(|S'| / |S' + sI|) [App. A] */
    int32_t pixels_per_thread; /* pixels one compositing thread owns, stacked along y: 0 = default
                                  (1 for 8x8 and 16x16 tiles, 4 for 32x32); also 2 for 16x16, 2 or 4
                                  for 32x32.  Changes the schedule only, never the result. */
    float eps2d;          /* low-pass s added to the 2D covariance [App. A] */
    float near_plane;     /* a Gaussian is culled when its camera depth t_z < near_plane */
    float alpha_min;      /* a (pixel, Gaussian) pair with alpha < alpha_min is skipped */
    float alpha_max;      /* alpha = min(alpha_max, o * exp(-sigma)) */
    float T_min;          /* a Gaussian that would bring T below T_min is excluded and ends the pixel */
    int32_t persistent;   /* compositing launch: 0 = one CTA per tile; 1 = as many CTAs as fit on the GPU,
                             each taking the next tile of tile_order (heaviest first) until none is left;
                             needs the tile_order of gs_tile_order.  Changes the schedule only. */
    int32_t colors_shared; /* compositing: 0 = colors [C,N,ch], one row per (camera, Gaussian); 1 = colors
                              [N,ch] shared by every camera (N-D features, App. C), and the backward's
                              d_colors is [N,ch], accumulated over the cameras */
} gs_params;

GS_API void gs_default_params(gs_params *params);

/* Human-readable name of a status code (static storage). */
GS_API const char *gs_status_string(gs_status status);

/* Last CUDA error text recorded by a call of this thread ("" when none). */
GS_API const char *gs_last_error(void);

/* Number of tiles of C cameras at the given tile size (sum of ceil(W/t) ceil(H/t)). */
GS_API int64_t gs_num_tiles(const gs_camera *cams, int32_t C, int32_t tile);

/* Kernels this library has launched in this process so far (all threads, all devices):
 * a counter the host increments at every launch, for accounting only. */
GS_API uint64_t gs_kernel_launches(void);

/* Number of pixels of C cameras (sum of W * H). */
GS_API int64_t gs_num_pixels(const gs_camera *cams, int32_t C);

/* Throughput probe for the roofline of the compositing kernels (not part of the
 * method): launches `blocks` CTAs of 256 threads, each thread running 8 independent
 * chains of iters * 16 operations of one kind -- kind 0: FP32 FFMA, kind 1: the
 * special-function ex2 approximation.  *ops (host) receives the number of lane
 * operations launched; time the launch with events on `stream` to get ops/s.  `sink`
 * is one device float the kernel never actually writes (it keeps the work alive).
 * GS_ERR_ARG on a bad kind, blocks < 1 or iters outside [1, 2^24]. */
GS_API gs_status gs_probe_peak(int32_t kind, int32_t blocks, int32_t iters, float *sink, double *ops, void *stream);

/* ------------------------------------------------------------------------ */
/* gs_project -- App. C.1 (projection, EWA splatting), App. E (quaternion,   */
/* pixel coordinates), App. A (low-pass / anti-aliasing).                    */
/*                                                                          */
/* For each camera c and Gaussian n: s = exp(log_scales), o = sigmoid(logit),*/
/* R = R(q/|q|), Sigma = R diag(s)^2 R^T, t = R_cw mu + t_cw (cull when      */
/* t_z < near), mu' = (fx tx/tz + cx, fy ty/tz + cy), J the pinhole Jacobian */
/* [[fx/tz, 0, -fx tx/tz^2], [0, fy/tz, -fy ty/tz^2]], Sigma' = J R_cw Sigma */
/* R_cw^T J^T + eps2d I, conic = Sigma'^-1, radius r = ceil(3 sqrt(lambda_max)),*/
/* and the pixel box [ceil(mu'x - r - 0.5), floor(mu'x + r - 0.5)] x (same in */
/* y) clipped to the image.  A Gaussian is invisible (radius 0, no tiles) if  */
/* culled or if the box is empty.  Input limit of this library (not a rule   */
/* of the paper, whose 3-sigma radius has no bound): a splat whose radius    */
/* would exceed 1e7 pixels is culled too, which keeps the integer box        */
/* arithmetic (2r) inside int32; such a splat is 4 orders of magnitude wider */
/* than any image the ABI accepts.                                           */
/*                                                                          */
/* in : means [N,3], quats [N,4] (w,x,y,z, any norm > 0), log_scales [N,3],  */
/*      opacity_logits [N]                                                   */
/* out: means2d [C,N,2], depths [C,N] (= t_z), conics [C,N,3] (a,b,c of       */
/*      [[a,b],[b,c]]), radii [C,N] int32, tiles_touched [C,N] int32 (tiles   */
/*      containing a pixel of the box), opacities [C,N] (o, times the          */
/*      anti-aliasing factor when enabled).  Entries of invisible Gaussians     */
/*      are zero.                                                             */
/* ------------------------------------------------------------------------ */
GS_API gs_status gs_project(const gs_camera *cams, int32_t C, int32_t N, const float *means, const float *quats,
                     const float *log_scales, const float *opacity_logits, const gs_params *params,
                     float *means2d, float *depths, float *conics, int32_t *radii, int32_t *tiles_touched,
                     float *opacities, void *stream);

/* ------------------------------------------------------------------------ */
/* gs_sh_eval -- App. C.1: colour c = SH(dir), dir = (mu - centre)/|mu -     */
/* centre|, centre = -R_cw^T t_cw.  Real spherical harmonics of degree <= 3,  */
/* orthonormal, Condon-Shortley phase, coefficients ordered m = -l..l per l;  */
/* colour = max(0, sum_k Y_k(dir) coeff_k + 0.5).                             */
/*                                                                          */
/* in : sh [N, (degree+1)^2, 3], means [N,3], radii [C,N] (colours of         */
/*      invisible Gaussians are written as 0)                                 */
/* out: colors [C,N,3]                                                       */
/* ------------------------------------------------------------------------ */
GS_API gs_status gs_sh_eval(const gs_camera *cams, int32_t C, int32_t N, int32_t sh_degree, const float *sh,
                     const float *means, const int32_t *radii, float *colors, void *stream);

/* ------------------------------------------------------------------------ */
/* gs_project_sh_eval -- gs_project followed by gs_sh_eval in one kernel:    */
/* the same definitions (App. C.1), each Gaussian's parameters, mean and SH   */
/* coefficients read once for all C cameras, and the coefficients of         */
/* Gaussians that every camera culls not read.                               */
/* in : sh [N,K,3], means [N,3], quats [N,4] (16-byte aligned), log_scales    */
/*      [N,3], opacity_logits [N]                                            */
/* out: as gs_project (means2d 8-byte aligned), plus colors [C,N,3] as        */
/*      gs_sh_eval; all OVERWRITTEN (zeros for invisible pairs).              */
/* ------------------------------------------------------------------------ */
GS_API gs_status gs_project_sh_eval(const gs_camera *cams, int32_t C, int32_t N, const gs_params *params,
                                    int32_t sh_degree, const float *sh, const float *means, const float *quats,
                                    const float *log_scales, const float *opacity_logits, float *means2d,
                                    float *depths, float *conics, int32_t *radii, int32_t *tiles_touched,
                                    float *opacities, float *colors, void *stream);

/* ------------------------------------------------------------------------ */
/* gs_sh_eval_depth -- depth rendering (App. A): gs_sh_eval plus a fourth     */
/* feature channel holding each Gaussian's camera-space depth z, so that the  */
/* compositing of the 4 channels yields the accumulated depth                */
/* sum_n z_n alpha_n T_n beside the colour.                                   */
/*                                                                          */
/* in : as gs_sh_eval, plus depths [C,N] from gs_project                      */
/* out: colors_rgbd [C,N,4] = (r, g, b, z); zeros for invisible pairs         */
/* ------------------------------------------------------------------------ */
GS_API gs_status gs_sh_eval_depth(const gs_camera *cams, int32_t C, int32_t N, int32_t sh_degree, const float *sh,
                                  const float *means, const int32_t *radii, const float *depths,
                                  float *colors_rgbd, void *stream);

/* ------------------------------------------------------------------------ */
/* gs_expected_depth -- App. A: expected depth = accumulated depth divided   */
/* by the accumulated opacity sum_n alpha_n T_n = 1 - final_T; 0 where that   */
/* is 0.  One value per pixel.                                               */
/*                                                                          */
/* in : image [P, channels] (accumulated depth in channel depth_channel),     */
/*      final_T [P];  out: expected_depth [P]                                */
/* gs_expected_depth_bwd: ADDS the chain into d_image[:, depth_channel]      */
/*      (dE/dA = 1/a) and d_alpha (dE/da = -E/a), for gs_rasterize_bwd.       */
/* ------------------------------------------------------------------------ */
GS_API gs_status gs_expected_depth(int64_t P, const float *image, int32_t channels, int32_t depth_channel,
                                   const float *final_T, float *expected_depth, void *stream);
GS_API gs_status gs_expected_depth_bwd(int64_t P, const float *image, int32_t channels, int32_t depth_channel,
                                       const float *final_T, const float *d_expected_depth, float *d_image,
                                       float *d_alpha, void *stream);

/* ------------------------------------------------------------------------ */
/* gs_tile_bin_sort -- App. C.2: bin every visible Gaussian into the tiles   */
/* its pixel box touches and sort each tile's list by depth.                 */
/*                                                                          */
/* The result is the list of (tile, Gaussian) pairs in the order of the key  */
/* (global_tile << 32) | float_bits(depth), ties broken by the flat index     */
/* c*N + n.  The pixel box is recomputed here from means2d and radii with the */
/* rule of gs_project (in float64 from the float32 inputs).                  */
/*                                                                          */
/* in : means2d [C,N,2], depths [C,N], radii [C,N]                           */
/* out: values [K] int32 (flat index c*N + n; 16-byte aligned), tile_ranges   */
/*      [T,2] int32                                                          */
/*      ([start, end) into values; (0,0) for an empty tile; T = gs_num_tiles),*/
/*      keys [K] uint64 (optional, NULL to skip), K_out [1] int64 on the      */
/*      device = the number of pairs K.  When K > K_capacity only the first   */
/*      K_capacity slots are written, the lists are incomplete, and the       */
/*      caller must reallocate (K_out tells by how much) and call again.      */
/*      K_capacity above GS_MAX_INTERSECTIONS returns GS_ERR_CAPACITY: such   */
/*      a list does not fit the int32 positions; split the cameras over       */
/*      several calls or use a larger tile.                                   */
/* workspace: device scratch of at least gs_tile_bin_sort_workspace() bytes,  */
/*      256-byte aligned; its content on entry is ignored.  About 44 bytes    */
/*      per (camera, Gaussian) pair plus, per slot of K_capacity, under one   */
/*      byte with at most 2048 tiles (one 1080p view at 32x32 tiles: nothing  */
/*      of size K is materialised) and about 12.8 bytes beyond.              */
/* ------------------------------------------------------------------------ */
GS_API int64_t gs_tile_bin_sort_workspace(const gs_camera *cams, int32_t C, int32_t N, const gs_params *params,
                                   int64_t K_capacity);
GS_API gs_status gs_tile_bin_sort(const gs_camera *cams, int32_t C, int32_t N, const gs_params *params,
                           const float *means2d, const float *depths, const int32_t *radii, int64_t K_capacity,
                           uint64_t *keys, int32_t *values, int32_t *tile_ranges, int64_t *K_out,
                           void *workspace, size_t workspace_bytes, void *stream);

/* ------------------------------------------------------------------------ */
/* gs_tile_bin_sort_noalloc -- the same binning and sorting as               */
/* gs_tile_bin_sort, for callers that cannot allocate device memory (a       */
/* plug-in inside an application whose allocator owns all device memory, a   */
/* real-time loop that must not stall on an allocation, a binding with no    */
/* device allocator).  The paper has no counterpart: this is an interface    */
/* variant, not a step of the method.                                        */
/*                                                                          */
/* Same arguments, outputs and errors as gs_tile_bin_sort minus the           */
/* workspace: the scratch comes from a fixed array of                         */
/* GS_NOALLOC_SCRATCH_BYTES inside libgs, reserved on every GPU that loads   */
/* the library until the process exits.  A call whose scratch need           */
/* (gs_tile_bin_sort_workspace) exceeds it returns GS_ERR_CAPACITY and        */
/* launches nothing.  The first call on a device looks up the array's device */
/* address (cudaGetSymbolAddress); make that first call before any stream    */
/* capture.  All calls share the array: calls that overlap on the GPU (other */
/* streams, other host threads) race on it and must be serialised.  Nothing  */
/* in it needs clearing between calls.  Nothing is allocated by this call.   */
/* The looked-up address is cached per device ordinal for the life of the    */
/* process: it is not valid after cudaDeviceReset or in a context other than */
/* the device's primary context, so do not call this entry point there.     */
/* ------------------------------------------------------------------------ */
#define GS_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)
GS_API gs_status gs_tile_bin_sort_noalloc(const gs_camera *cams, int32_t C, int32_t N, const gs_params *params,
                                          const float *means2d, const float *depths, const int32_t *radii,
                                          int64_t K_capacity, uint64_t *keys, int32_t *values,
                                          int32_t *tile_ranges, int64_t *K_out, void *stream);

/* ------------------------------------------------------------------------ */
/* gs_tile_order -- a launch order for the compositing kernels (not a step   */
/* of the method; App. C.2 leaves the schedule open): tiles sorted by the    */
/* length of their list, longest first, in buckets of half an octave (ties   */
/* in any order).  Handing the heaviest tiles out first shortens the tail    */
/* of a launch whose per-tile work is uneven (clustered scenes, many views).  */
/*                                                                          */
/* in : tile_ranges [T,2] from gs_tile_bin_sort                              */
/* out: tile_order [T + 4] int32: a permutation of 0..T-1 (T = gs_num_tiles),*/
/*      then four work counters of the persistent compositing launches,      */
/*      zeroed here (each launch leaves them zero again when it ends)         */
/* One CTA, no scratch; never synchronises.                                  */
/* ------------------------------------------------------------------------ */
GS_API gs_status gs_tile_order(const gs_camera *cams, int32_t C, const gs_params *params,
                               const int32_t *tile_ranges, int32_t *tile_order, void *stream);

/* ------------------------------------------------------------------------ */
/* gs_rasterize_fwd -- App. C.2: for each pixel p (centre i+0.5, j+0.5) walk */
/* its tile's sorted list front to back; a Gaussian counts at p only if p is */
/* inside its pixel box; sigma = 1/2 D^T conic D with D = p - mu';           */
/* alpha = min(alpha_max, o exp(-sigma)); pairs with sigma < 0 or alpha <     */
/* alpha_min are skipped; if T (1 - alpha) < T_min the pixel stops without    */
/* that Gaussian; otherwise C += c alpha T and T *= 1 - alpha.  Finally       */
/* C += T * background.                                                      */
/*                                                                          */
/* in : tile_ranges, values (from gs_tile_bin_sort), radii [C,N],             */
/*      means2d [C,N,2], conics [C,N,3], opacities [C,N], colors [C,N,ch]     */
/*      ([N,ch] with params->colors_shared),                                 */
/*      background: host array of `channels` floats or NULL (zeros)          */
/* out: image [pixels, channels], final_T [pixels] (alpha = 1 - final_T),     */
/*      last_contrib [pixels] int32 = number of list entries of the pixel's   */
/*      tile up to and including its last contributor (read by the backward),*/
/*      blend_count (optional device int64, NULL to skip): += the number of   */
/*      (pixel, Gaussian) pairs whose alpha was evaluated.                    */
/* channels: 1..GS_MAX_CHANNELS; 1,2,3,4,8,16,32,64 use specialised kernels.  */
/* tile_order (optional device int32 [T + 4], NULL for 0..T-1): the order in */
/*      which tiles are handed to the GPU (gs_tile_order: heaviest first);    */
/*      a permutation of 0..T-1 followed by the persistent launches' work     */
/*      counters (required when params->persistent).  Results do not depend  */
/*      on it.                                                                */
/* ------------------------------------------------------------------------ */
GS_API gs_status gs_rasterize_fwd(const gs_camera *cams, int32_t C, int32_t N, const gs_params *params,
                           int32_t channels, const int32_t *tile_ranges, const int32_t *values,
                           const int32_t *radii, const float *means2d, const float *conics, const float *opacities,
                           const float *colors, const float *background, float *image, float *final_T,
                           int32_t *last_contrib, int64_t *blend_count, const int32_t *tile_order, void *stream);

/* ------------------------------------------------------------------------ */
/* gs_rasterize_bwd -- App. D.2: replay each pixel back to front from its    */
/* last contributor, recovering T_n = T_{n+1} / (1 - alpha_n) from final_T,  */
/* and accumulate per (camera, Gaussian):                                    */
/*   dL/dc_n     += alpha_n T_n dL/dC                                         */
/*   dL/dalpha_n  = <dL/dC, c_n T_n - S_n/(1 - alpha_n)> + dL/dA T_N/(1-alpha_n),*/
/*                  S_n = sum_{m>n} c_m alpha_m T_m + T_N background          */
/*                  (0 where alpha was clamped to alpha_max)                  */
/*   dL/do_n     += exp(-sigma) dL/dalpha_n                                   */
/*   dL/dmu'_n   += -dL/dsigma conic D,  dL/dsigma = -o exp(-sigma) dL/dalpha */
/*   dL/dconic_n += dL/dsigma (D_x^2/2, D_x D_y, D_y^2/2)  (for a, b, c)      */
/*   absgrad_n   += (|per-pixel dL/dmu'_x|, |per-pixel dL/dmu'_y|) [App. A]    */
/*                                                                          */
/* in : as gs_rasterize_fwd plus final_T, last_contrib from it, d_image       */
/*      [pixels, channels], d_alpha [pixels] or NULL                         */
/* out (accumulated, caller zeroes): d_means2d [C,N,2], d_conics [C,N,3],     */
/*      d_opacities [C,N], d_colors [C,N,channels] ([N,channels], summed over */
/*      the cameras, with params->colors_shared), absgrad [C,N,2] or NULL     */
/* tile_order: as for gs_rasterize_fwd.                                      */
/* ------------------------------------------------------------------------ */
GS_API gs_status gs_rasterize_bwd(const gs_camera *cams, int32_t C, int32_t N, const gs_params *params,
                           int32_t channels, const int32_t *tile_ranges, const int32_t *values,
                           const int32_t *radii, const float *means2d, const float *conics, const float *opacities,
                           const float *colors, const float *background, const float *final_T,
                           const int32_t *last_contrib, const float *d_image, const float *d_alpha,
                           float *d_means2d, float *d_conics, float *d_opacities, float *d_colors,
                           float *absgrad, const int32_t *tile_order,
                           void *stream);

/* ------------------------------------------------------------------------ */
/* gs_sh_eval_bwd -- backward of gs_sh_eval: d_sh[n] = sum_c Y(dir_c) *      */
/* d_colors[c,n] (masked where the clamp at 0 was active), and the gradient  */
/* through dir into the mean, d_means[n] = sum_c (I - dir dir^T)/|mu - centre|*/
/* sum_k grad Y_k(dir) <coeff_k, d_colors>.  Both outputs are OVERWRITTEN for */
/* every Gaussian (zeros where invisible in all cameras).                    */
/* ------------------------------------------------------------------------ */
GS_API gs_status gs_sh_eval_bwd(const gs_camera *cams, int32_t C, int32_t N, int32_t sh_degree, const float *sh,
                         const float *means, const int32_t *radii, const float *d_colors, float *d_sh,
                         float *d_means, float *d_viewmats, void *stream);

/* gs_sh_eval_depth_bwd: gs_sh_eval_bwd for (r, g, b, z) rows: the colour   */
/* part as gs_sh_eval_bwd, and d_depths [C,N] = the z channel's gradient      */
/* (OVERWRITTEN; 0 for invisible pairs), to be passed to gs_project_bwd.      */
GS_API gs_status gs_sh_eval_depth_bwd(const gs_camera *cams, int32_t C, int32_t N, int32_t sh_degree,
                                      const float *sh, const float *means, const int32_t *radii,
                                      const float *d_colors_rgbd, float *d_sh, float *d_means, float *d_depths,
                                      float *d_viewmats, void *stream);

/* ------------------------------------------------------------------------ */
/* gs_project_bwd -- App. D.3 / D.4 and the gradient-flow figure: from        */
/* d_means2d, d_conics, d_opacities (and optional d_depths, for depth         */
/* rendering) of every camera to the leaves: dSigma' = -Y dY Y,              */
/* dSigma = T^T dSigma' T and dT = dSigma' T Sigma^T + dSigma'^T T Sigma      */
/* (T = J R_cw), dJ -> dt, d mu = R_cw^T dt, dM = dSigma M + dSigma^T M,      */
/* dR = dM S, dS = diag(R^T dM), dq through dR/dq and the normalisation,     */
/* d log_scale = dS s, d logit = d o * o (1 - o).  Sums over the C cameras.   */
/* d_viewmats (optional, NULL to skip): pose gradient (App. A), ACCUMULATED  */
/* (+=) into [C,4,4] laid out like gs_camera.viewmat: rows 0-2 get           */
/* dR_cw = sum_n (J^T dT + dt mu^T) and dt_cw = sum_n dt (t = R_cw mu + t_cw, */
/* T = J R_cw); row 3 is left untouched.  gs_sh_eval_bwd / _depth_bwd add    */
/* the view-direction term (centre = -R_cw^T t_cw) into the same array.       */
/* d_means is ACCUMULATED (+=, so the SH term from gs_sh_eval_bwd adds up);   */
/* d_quats, d_log_scales and d_opacity_logits are OVERWRITTEN.               */
/* ------------------------------------------------------------------------ */
GS_API gs_status gs_project_bwd(const gs_camera *cams, int32_t C, int32_t N, const float *means, const float *quats,
                         const float *log_scales, const float *opacity_logits, const gs_params *params,
                         const int32_t *radii, const float *d_means2d, const float *d_conics,
                         const float *d_opacities, const float *d_depths, float *d_means, float *d_quats,
                         float *d_log_scales, float *d_opacity_logits, float *d_viewmats,
                                void *stream);

/* ------------------------------------------------------------------------ */
/* gs_sh_project_bwd -- gs_sh_eval_bwd followed by gs_project_bwd for ONE     */
/* camera (C == 1), without depth or pose gradients, in one kernel: the same  */
/* chain rule (App. C.1 differentiated; App. D.2-D.4), each Gaussian's        */
/* parameters, radius and mean read once, and d_means written once.           */
/* in : sh [N,K,3], means [N,3], quats [N,4] (16-byte aligned), log_scales    */
/*      [N,3], opacity_logits [N], radii [N], d_colors [N,3], d_means2d [N,2] */
/*      (8-byte aligned), d_conics [N,3], d_opacities [N]                     */
/* out: d_sh [N,K,3], d_means [N,3], d_quats [N,4] (16-byte aligned),        */
/*      d_log_scales [N,3], d_opacity_logits [N], all OVERWRITTEN (zeros for  */
/*      Gaussians the camera culls).  GS_ERR_ARG when C != 1.                 */
/* ------------------------------------------------------------------------ */
GS_API gs_status gs_sh_project_bwd(const gs_camera *cams, int32_t C, int32_t N, const gs_params *params,
                                   int32_t sh_degree, const float *sh, const float *means, const float *quats,
                                   const float *log_scales, const float *opacity_logits, const int32_t *radii,
                                   const float *d_colors, const float *d_means2d, const float *d_conics,
                                   const float *d_opacities, float *d_sh, float *d_means, float *d_quats,
                                   float *d_log_scales, float *d_opacity_logits, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GS_H_ */
