/*
 * libsop: Surface Octahedral Probes (SOPs) of ComGS (arXiv 2510.07729) on one
 * GB300 (sm_103a). C ABI.
 *
 * The library computes the two data-parallel halves of the SOP method:
 *   - the probe bake: every octahedral texel of every probe shoots a ray that
 *     is alpha-composited front to back through 3D Gaussians, giving the
 *     probe's occlusion O, indirect radiance L_in and depth D maps
 *     (Sec. 3.1.2 "SOPs ... initialised via ray tracing"; Sec. 3.2.2 occlusion
 *     caching; compositing of Eq. 1; unbiased depth D/W of Sec. 3.1);
 *   - the probe query + shading that replaces ray tracing: K nearest probes,
 *     back-face and distance weights (Eq. 4-6), per-direction bilinear
 *     octahedral fetches, and the Monte Carlo sum of the visibility-weighted
 *     BRDF against an environment map plus the interpolated indirect term
 *     (Eq. 2-3), or the shadow ratio S = L_o'/L_o (Eq. 7-9).
 *
 * Conventions for every entry point:
 *   - Every array pointer is DEVICE memory owned by the caller, unless the
 *     argument says "host". Arrays are C-contiguous float32 unless stated.
 *   - The library allocates no memory. Scratch space ("workspace") is passed
 *     in by the caller; its size comes from the matching *_workspace_bytes()
 *     query and the workspace pointer must be 256-byte aligned.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream). Work is
 *     enqueued asynchronously on it unless the entry point says it syncs.
 *   - Arguments are validated on the host before any launch. A non-OK status
 *     means nothing was launched (except SOP_ERR_CUDA, which reports a launch
 *     or runtime error); sop_last_error() then returns a message for the
 *     calling thread. No exception crosses this boundary.
 *   - Readings of points the paper leaves open (octahedral map formula,
 *     border rule, ray-Gaussian response, KNN tie-break, BRDF terms, light
 *     direction set, environment parameterisation) are stated beside the
 *     function that applies them.
 */
#ifndef SOP_H
#define SOP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
typedef enum {
    SOP_OK = 0,
    SOP_ERR_INVALID_ARG = 1, /* bad pointer, size, alignment or parameter  */
    SOP_ERR_CUDA = 2,        /* a CUDA launch or runtime call failed        */
    SOP_ERR_WORKSPACE = 3,   /* workspace missing, misaligned or too small  */
    SOP_ERR_UNSUPPORTED = 4, /* valid but not implemented (e.g. a dtype)    */
    SOP_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up          */
    SOP_ERR_DEVICE = 6       /* a device-side check failed (see message)    */
} sop_status;

/* Device status word. Problems that kernels meet while they run, and that no
 * host-side check can see before launch, set bits in one 32-bit word per
 * device (shared by every stream and thread that uses the library on it):
 *   SOP_DEVSTAT_NONFINITE      an input value was NaN or Inf: Gaussian
 *                              parameters (such a Gaussian is left out of
 *                              the bake), probe or shading-point positions
 *                              and normals, materials, view directions,
 *                              environment or atlas texels, upstream
 *                              gradients;
 *   SOP_DEVSTAT_BAKE_TRUNCATED a bake (or G-buffer) ray met more hits with
 *                              one t* than its 256-entry hit buffer holds,
 *                              could not split them further and stopped
 *                              there (its texel holds the partial
 *                              composite);
 *   SOP_DEVSTAT_INDEX          a caller-supplied index (probe ids, pixel
 *                              lists) was outside its range and skipped;
 *   SOP_DEVSTAT_CAPACITY       a fixed-capacity buffer overflowed and the
 *                              result was computed from part of its input
 *                              (the surrogate's near-field search found
 *                              more than 4,096 centres within r_near);
 *   SOP_DEVSTAT_TIMEOUT        a kernel's bounded wait for the tensor cores
 *                              (the surrogate network's completion
 *                              barrier) gave up; that launch's outputs are
 *                              not valid;
 *   SOP_DEVSTAT_GRID_COARSENED information, not an error: the bake's
 *                              binning grid was coarsened on the device
 *                              until the cell lists fit the workspace.
 * Entry points do not wait for their kernels, so these come back only
 * through sop_device_status(): it synchronises `stream`, writes the word to
 * *out_bits (host, may be NULL), clears it when `clear` is non-zero (an
 * atomic exchange on the device), and returns SOP_ERR_DEVICE with a message
 * naming the problems when any error bit (SOP_DEVSTAT_ERRORS) is set, else
 * SOP_OK. Bits stay set until a call clears them. The word's address is
 * looked up once per device: do not use the library across a
 * cudaDeviceReset() in the same process. */
#define SOP_DEVSTAT_NONFINITE 0x1u
#define SOP_DEVSTAT_BAKE_TRUNCATED 0x2u
#define SOP_DEVSTAT_INDEX 0x4u
#define SOP_DEVSTAT_CAPACITY 0x8u
#define SOP_DEVSTAT_TIMEOUT 0x10u
#define SOP_DEVSTAT_GRID_COARSENED 0x100u
#define SOP_DEVSTAT_ERRORS 0xffu
sop_status sop_device_status(void* stream, uint32_t* out_bits, int32_t clear);

/* Storage types of the probe atlas (Sec. 3.1.2 octahedral textures; the
 * reduced-precision atlas stores in bf16/fp16, accumulates in fp32). */
typedef enum { SOP_F32 = 0, SOP_BF16 = 1, SOP_F16 = 2, SOP_FP8E4M3 = 3 } sop_dtype;

/* Query output mode. SHADE: outgoing radiance of Eq. 3 with Eq. 4 lighting.
 * SHADOW: the ratio S = L_o'/L_o of Eq. 9 with the Lambertian Eq. 7-8 (the
 * diffuse factor cancels). */
typedef enum { SOP_MODE_SHADE = 0, SOP_MODE_SHADOW = 1 } sop_mode;

/* A set of n 3D Gaussians, structure of arrays, device memory:
 * mean [n,3], per-axis scale [n,3] (> 0), rotation quaternion [n,4] in
 * (w, x, y, z) order (need not be normalised), opacity [n] in [0,1],
 * colour rgb [n,3]. (Sec. 3.1: centre, quaternion, scaling; the colour is
 * the radiance a probe ray receives from the Gaussian.) */
typedef struct {
    const float* mean;
    const float* scale;
    const float* quat;
    const float* opacity;
    const float* rgb;
    int64_t n;
} sop_gaussians;

/* Probe atlas (caller-owned device memory). P probes, each an R x R
 * octahedral map stored with a one-texel border ("gutter"), i.e. (R+2)^2
 * texels per probe, probe-major, then row (v), then column (u):
 *   rgbo  [P][R+2][R+2][4]  indirect radiance RGB + occlusion O, dtype
 *                           rgbo_dtype (SOP_F32: 16 B/texel; SOP_BF16 or
 *                           SOP_F16: 8 B/texel);
 *   depth [P][R+2][R+2]     mean hit depth D, dtype depth_dtype (SOP_F32,
 *                           SOP_F16 or SOP_FP8E4M3, stored as D/depth_scale);
 *                           may be NULL when not needed.
 * Stored texel (jj, ii) for 1 <= ii, jj <= R is map texel (i = ii-1 along u,
 * j = jj-1 along v). Border texels copy the texel that the octahedral fold
 * makes their neighbour: crossing an edge mirrors the index along that edge,
 * corners take the diagonally opposite corner (the border rule of Majercik
 * et al. 2019, which keeps bilinear fetches continuous across the folds).
 * probe_pos [P,3] (and probe_nrm [P,3], informational) are device arrays.
 * The octahedral map is the one of Cigolle et al. 2014, z-up, world frame:
 * encode(d) = (p + 1)/2 with p = (d.x, d.y)/|d|_1 folded for d.z < 0. */
typedef struct {
    void* rgbo;
    void* depth;
    int32_t rgbo_dtype;
    int32_t depth_dtype;
    int32_t P;
    int32_t R;
    float depth_scale;
    const float* probe_pos;
    const float* probe_nrm;
} sop_atlas;

/* Bake parameters (paper silent; 3D Gaussian splatting conventions):
 * a Gaussian's response along a ray is its maximum, alpha = min(alpha_max,
 * o exp(-m^2/2)) with m the Mahalanobis distance at the maximising t*;
 * responses with t* <= t_near or alpha < alpha_min are skipped; compositing
 * stops once the transmittance falls below t_stop (0 = never).
 * Defaults: t_near 0, alpha_min 1/255, alpha_max 0.99, t_stop 1e-4.
 * grid_density: cells of the binning grid per Gaussian (an implementation
 * choice, not the method's: results do not depend on it), 0 (what
 * zero-initialised callers get) for the default of 0.35 cells per
 * Gaussian, else in [0.01, 2]; probe bakes run fastest near the default,
 * camera G-buffers near 0.06. sop_bake_bin and the traces that use its grid
 * take the same value. */
typedef struct {
    float t_near;
    float alpha_min;
    float alpha_max;
    float t_stop;
    float grid_density;
} sop_bake_params;

/* Query/shade parameters. K nearest probes (1..32), S light directions
 * (1..4096), mode (sop_mode), specular = the Disney "specular" level giving
 * F0 = 0.08 specular (1-m) + a m (0.5 gives F0 = 0.04), eps_snap = distance
 * below which a shading point counts as sitting on its nearest probe (the
 * blend is then one-hot on that probe; default 1e-6), env_layout = the
 * environment's layout (SOP_ENV_EQUIRECT: [He][We][3] equirectangular, z-up;
 * SOP_ENV_OCTAHEDRAL: [He][He][3] octahedral with the probe maps' mapping and
 * border rule, Sec. 4.1; zero-initialised callers get the equirectangular
 * layout), dir_world = 0: dirs_local is the local direction set (or NULL)
 * and the estimator is 2 pi / S sum (Eq. 3); 1: dirs_local is required and
 * holds S world directions with their density, [S][4] = (x, y, z, pdf), as
 * sop_env_importance_dirs writes them, shared by every point, and the
 * estimator is 1/S sum over the directions above the point's horizon of the
 * terms divided by pdf (Sec. 4.2); the adjoint and the allocation-free entry
 * point take dir_world = 0 only. radius = the fixed-radius neighbour search
 * of Sec. 3.2 (0, what zero-initialised callers get: no radius, the plain K
 * nearest): a point's neighbours are then the at most K nearest probes whose
 * quantised distance (positions rounded to multiples of 2^-20) is <= radius,
 * i.e. whose integer squared distance is <= floor((radius 2^20)^2); slots
 * left empty get index -1 and weight 0 in out_idx/out_w, the weights are
 * normalised over the probes found, and a point with none gets O = 0 and
 * L_in = 0 (the environment term alone). 0 <= radius <= 2048 (positions lie
 * within +-1024); every entry point, the adjoint included, takes it. */
#define SOP_ENV_EQUIRECT 0
#define SOP_ENV_OCTAHEDRAL 1
typedef struct {
    int32_t K;
    int32_t S;
    int32_t mode;
    float specular;
    float eps_snap;
    int32_t env_layout;
    int32_t dir_world;
    float radius;
} sop_shade_params;

/* Message for the last non-OK status returned to the calling thread
 * (thread-local, valid until the next call on that thread). */
const char* sop_last_error(void);

/* Library version string. */
const char* sop_version(void);

/* Bytes of the rgbo and depth planes of an atlas (either pointer may be
 * NULL). Returns SOP_ERR_INVALID_ARG for P < 1, R < 2 or an unknown dtype. */
sop_status sop_atlas_bytes(int32_t P, int32_t R, int32_t rgbo_dtype, int32_t depth_dtype,
                           size_t* rgbo_bytes, size_t* depth_bytes);

/* Pack compact probe maps into an atlas (conversion to the atlas dtypes and
 * the border rule described at sop_atlas). maps_rgb [P,R,R,3], maps_occ
 * [P,R,R], maps_depth [P,R,R] or NULL (depth plane then left untouched);
 * rows index v, columns index u. Asynchronous. */
sop_status sop_atlas_pack(const float* maps_rgb, const float* maps_occ, const float* maps_depth,
                          const sop_atlas* atlas, void* stream);

/* sop_atlas_pack for interleaved maps: maps_rgbo [P,R,R,4] = (L_in RGB, O)
 * per texel (the layout of the adjoint's probe-map gradient and of the
 * texture optimisation's parameters); the depth plane is left untouched.
 * Asynchronous. */
sop_status sop_atlas_pack_rgbo(const float* maps_rgbo, const sop_atlas* atlas, void* stream);

/* The canonical S light directions in the local frame (z along the normal),
 * written to out_dirs [S,3] (device): a Hammersley set with centred first
 * coordinate, z_i = (i + 1/2)/S, phi_i = 2 pi radical_inverse_base2(i),
 * uniform on the hemisphere (Sec. 3.1.2, Eq. 3 low-discrepancy rays).
 * Asynchronous. */
sop_status sop_hammersley(int32_t S, float* out_dirs, void* stream);

/* Resample an equirectangular environment env [He][We][3] (z-up) into an
 * octahedral one out [H][H][3] (Sec. 4.1: the estimated environment is
 * converted to an octahedral texture): texel (i, j) takes the bilinear
 * equirectangular value at its centre direction. 2 <= H <= 4096. Device
 * pointers; asynchronous. */
sop_status sop_env_to_octahedral(const float* env, int32_t He, int32_t We, float* out, int32_t H, void* stream);

/* Importance-sampled light directions for rendering (Sec. 4.2, Eq. PDF:
 * density H W I / (4 pi) over the octahedral environment's texels): from an
 * octahedral environment env [H][H][3], S world directions out [S][4] =
 * (x, y, z, pdf) for sop_query_shade with dir_world = 1. The intensity of a
 * texel is the float32 sum r + g + b; it is quantised to
 * q = max(1, floor(I / I_max 2^20)) so that the texel chosen is an exact
 * integer decision; sample i takes the texel whose cumulative interval holds
 * floor((2i + 1) Q / (2S)) (Q = sum q; stratified), in its centre direction,
 * with pdf = H^2 q / (4 pi Q) (texels taken as equal in solid angle, as the
 * equation does). 2 <= H <= 2048, 1 <= S <= 4096. ws: workspace of
 * sop_env_importance_workspace_bytes(H) bytes, 256-byte aligned. Device
 * pointers; asynchronous. */
size_t sop_env_importance_workspace_bytes(int32_t H);
sop_status sop_env_importance_dirs(const float* env, int32_t H, int32_t S, float* out, void* ws, size_t ws_bytes,
                                   void* stream);

/* Measurement utility (not part of the paper's method): reads the device
 * buffer buf [bytes] `reps` times with 16-byte loads from every SM, so that
 * the caller can time the read rate with events on `stream`: a buffer that
 * fits in L2 gives the L2-to-SM rate that bounds the query's footprint
 * gathers, a larger one the HBM rate. buf must be 16-byte aligned and bytes
 * a positive multiple of 16; sink is one device float that is written only
 * for one improbable checksum (it keeps the loads from being optimised
 * away). Nothing else is written. Asynchronous. */
sop_status sop_read_bandwidth_probe(const void* buf, size_t bytes, int32_t reps, float* sink, void* stream);

/* Workspace bytes for sop_bake / sop_bake_bin / sop_bake_trace on n
 * Gaussians (the size does not depend on P or R; they are only checked).
 * This is the minimum: it holds 24 grid cell entries per Gaussian plus
 * 65,536; a larger workspace holds more entries. */
size_t sop_bake_workspace_bytes(int64_t n_gauss, int32_t P, int32_t R);

/* Bake every texel of every probe of `atlas` (positions atlas->probe_pos)
 * against the Gaussians `g` and write the atlas (interior and border) in its
 * dtypes. Texel (i, j) looks along the octahedral decode of its centre
 * ((i + 1/2)/R, (j + 1/2)/R). Hits are composited in increasing (t*, Gaussian
 * index) order: T <- T (1 - alpha), L += T_before alpha rgb, D accumulates
 * T_before alpha t*. Outputs O = 1 - T, L_in = L, D = sum(T alpha t*) /
 * sum(T alpha) (0 when nothing is hit).
 * Implementation: Gaussians are binned by the bounding boxes of their
 * alpha_min ellipsoids into a uniform grid that each texel ray walks front
 * to back. Equivalent to sop_bake_bin followed by sop_bake_trace.
 * Asynchronous (no host synchronisation): the grid is sized on the device.
 * If the cell lists of the requested grid (grid_density) would overflow the
 * workspace's entry capacity, the grid is coarsened (1/16 of the cells, then
 * at most 2 cells, which always fit) and SOP_DEVSTAT_GRID_COARSENED is set
 * in the device status word; the result is the same, only slower. Gaussians
 * with non-finite parameters are left out and a ray that cannot split its
 * hits is stopped; both set device status bits (sop_device_status).
 * ws_bytes below sop_bake_workspace_bytes() gives SOP_ERR_WORKSPACE. */
sop_status sop_bake(const sop_gaussians* g, const sop_atlas* atlas, const sop_bake_params* params, void* ws,
                    size_t ws_bytes, void* stream);

/* First half of sop_bake: bin the Gaussians into the grid kept in `ws`.
 * Asynchronous (see sop_bake for the device-side sizing of the grid). */
sop_status sop_bake_bin(const sop_gaussians* g, const sop_bake_params* params, void* ws, size_t ws_bytes,
                        void* stream);

/* Second half of sop_bake: trace every texel of `atlas` through the grid
 * that sop_bake_bin left in `ws` (same g, params and ws_bytes). May be called
 * any number of times, for any probe set, after one binning. Asynchronous. */
sop_status sop_bake_trace(const sop_gaussians* g, const sop_atlas* atlas, const sop_bake_params* params, void* ws,
                          size_t ws_bytes, void* stream);

/* Work counters of the last sop_bake_trace on `ws` (synchronises stream);
 * `out` holds 4 values: out[0] = exact ray-Gaussian evaluations, out[1] =
 * composited hits, out[2] = status bits (bit 0: some ray met more hits at one
 * t* than its hit buffer holds and stopped there), out[3] = grid-cell
 * entries tested against rays (box tests). */
sop_status sop_bake_stats(const void* ws, size_t ws_bytes, int64_t n_gauss, int64_t* out, void* stream);

/* Workspace bytes for sop_query_shade / sop_query_shade_backward on M
 * points with this atlas (its P, R and rgbo_dtype) and a He x We
 * environment; 0 for invalid arguments. */
size_t sop_query_workspace_bytes(const sop_atlas* atlas, int64_t M, const sop_shade_params* params, int32_t He,
                                 int32_t We);

/* Probe query and shading of M points (Sec. 3.1.2 Eq. 2-6; Sec. 3.2.2 Eq. 7-9).
 * Inputs [M,3]: x (position), n (normal, normalised inside), wo (unit view
 * direction, towards the viewer); [M,3] albedo, [M] rough (> 0), [M] metal.
 * env [He,We,3]: equirectangular environment, z-up, row r at polar angle
 * (r+1/2)/He pi, column c at azimuth (c+1/2)/We 2pi - pi; bilinear, u wraps,
 * v clamps. dirs_local [S,3] or NULL (= sop_hammersley(S)).
 * Per point: the K nearest probes by the exact integer squared distance of
 * positions rounded to multiples of 2^-20 (|coordinates| < 1024), ties to the
 * lower probe index; weights w_s = 1/|d_k|, w_b = 0.5 (1 + d_k/|d_k| . n)
 * + 0.01, W_k = w_s w_b / sum (one-hot on the nearest probe when it is within
 * eps_snap). For every local direction l: w_i = l.x t + l.y b + l.z n with
 * the frame (t, b) of Duff et al. 2017; O and L_in are the W-blend of the K
 * probes' bilinear octahedral fetches at w_i; L_dir the environment.
 *   SHADE : out = 2pi/S sum_i f(wo, w_i) ((1 - O) L_dir + L_in) (n . w_i), with
 *           f the simplified Disney BRDF: (1-m) a/pi + D F G/(4 (n.w_i)
 *           max(n.wo, 1e-4)), GGX D with alpha = rough^2, Schlick-GGX G with
 *           k = (rough+1)^2/8, Schlick F from F0.
 *   SHADOW: out_c = sum L_dir,c (1 - O)(n . w_i) / sum L_dir,c (n . w_i)
 *           (1 where the denominator is < 1e-20).
 * out [M,3] float32. out_idx [M,K] int32 and out_w [M,K] float32 are
 * optional (NULL to skip): the neighbour indices in increasing distance and
 * their weights. P (R+1)^2 must not exceed 2^31 - 1 (the bilinear
 * footprints are indexed with 32-bit integers): SOP_ERR_INVALID_ARG
 * otherwise. Asynchronous. */
sop_status sop_query_shade(const float* x, const float* n, const float* wo, const float* albedo, const float* rough,
                           const float* metal, int64_t M, const sop_atlas* atlas, const float* env, int32_t He,
                           int32_t We, const float* dirs_local, const sop_shade_params* params, float* out,
                           int32_t* out_idx, float* out_w, void* ws, size_t ws_bytes, void* stream);

/* Adjoint of sop_query_shade in SOP_MODE_SHADE (the environment, the
 * materials and the SOP textures are the learnable quantities of the
 * paper's decomposition step, Sec. 3.1.2; Eq. 3-6). Given grad_out = dL/dC
 * [M,3], writes (overwriting) g_albedo [M,3], g_rough [M], g_metal [M] and
 * g_normal [M,3] (w.r.t. the raw, unnormalised input normal), and ADDS
 * dL/d(environment texel) into g_env [He,We,3] and dL/d(probe texel) into
 * g_maps [P,R,R,4] (compact maps: RGB radiance then occlusion, border texels
 * folded onto the texels they copy; 16-byte aligned). The caller zeroes the
 * accumulated arrays. Every per-direction term is recomputed rather than
 * stored; the K nearest probes do not depend on the differentiated inputs.
 * Bilinear fetches are piecewise linear: at a texel edge the gradient is
 * one of the one-sided derivatives. Accumulation uses float atomics, so sums
 * are order-nondeterministic. SOP_MODE_SHADOW returns SOP_ERR_UNSUPPORTED.
 * Same workspace as sop_query_shade. Asynchronous. */
sop_status sop_query_shade_backward(const float* x, const float* n, const float* wo, const float* albedo,
                                    const float* rough, const float* metal, int64_t M, const sop_atlas* atlas,
                                    const float* env, int32_t He, int32_t We, const float* dirs_local,
                                    const sop_shade_params* params, const float* grad_out, float* g_albedo,
                                    float* g_rough, float* g_metal, float* g_normal, float* g_env, float* g_maps,
                                    void* ws, size_t ws_bytes, void* stream);

/* ---- SOP texture optimisation (Sec. 3.1.2, the second reconstruction step:
 * L = L_pbr + lambda_lam L_lam + lambda_sops L_sops over the environment,
 * the materials and the SOP textures, with Adam). One step is: pack the maps
 * (sop_atlas_pack), shade (sop_query_shade), sop_l1_loss_grad, the adjoint
 * (sop_query_shade_backward) and one sop_adam_l1_step per parameter block.
 * L_pbr is read as the mean absolute error over the shaded RGB (the render
 * loss's SSIM term needs an image grid, which the shading points are not). */

/* dL/dC of L = mean |C - C_target| over n floats: grad[i] = sign(C_i -
 * C_target,i) / n (sign(0) = 0), written to grad [n] (device). If loss_sum is
 * not NULL, sum |C - C_target| is added to *loss_sum (one device float; the
 * caller zeroes it; float atomics, so the last bits depend on the order).
 * Asynchronous. */
sop_status sop_l1_loss_grad(const float* C, const float* C_target, int64_t n, float* grad, float* loss_sum,
                            void* stream);

/* Settings of one Adam step on a parameter block. The L1 regulariser
 * lam * |p - target| (target[i] if `target` is not NULL, else target_value)
 * adds lam * sign(p - target) to the gradient. Elements i with
 * i % period < split use lam[0], lo[0], hi[0], the others lam[1], lo[1],
 * hi[1] (e.g. period 4, split 3 for RGB + O texels); after the Adam update
 * (Kingma & Ba 2015, bias-corrected, step >= 1) each element is clamped to
 * [lo, hi]. */
typedef struct {
    float lr, beta1, beta2, eps;
    int32_t step;
    const float* target;
    float target_value;
    int32_t period, split;
    float lam[2], lo[2], hi[2];
} sop_adam_params;

/* One Adam step in place on p [n], with moments m [n], v [n] (caller-owned,
 * zero before the first step) and the gradient g [n] (NULL = zero, e.g. a
 * block that only the regulariser drives). All device pointers. Rejects
 * period < 1, split outside [0, period], step < 1, lr <= 0 or beta outside
 * [0, 1). Asynchronous. */
sop_status sop_adam_l1_step(float* p, const float* g, float* m, float* v, int64_t n, const sop_adam_params* params,
                            void* stream);

/* ---- Learned bake surrogate ------------------------------------------------
 * A small MLP predicts a probe texel's maps (O, D/depth_scale, RGB) from
 * features of the probe's neighbourhood along the texel's ray, to rebake
 * probes quickly after an object moves; the ray-traced sop_bake is its
 * fallback and its judge (the paper has no surrogate: it initialises SOPs
 * by ray tracing, Sec. 3.1.2 / 3.2.2).
 * Texel features (SOP_SURROGATE_FEATURES = 18 per texel, float32,
 * [P][R*R][18]), for the texel direction d (the octahedral decode of its
 * centre):
 *   [0..2]   d;
 *   [3..8]   near field: the probe's nearest Gaussians (at most
 *            SOP_SURROGATE_NEAR_CAP = 256 of the centres within r_near,
 *            nearest first by the integer squared distance of positions
 *            quantised to 2^-20, ties to the lower index), composited along
 *            the texel ray in that order with the bake's ray-Gaussian
 *            response: O_n = 1 - prod(1 - alpha), L_n (rgb) = sum T alpha
 *            rgb, D_n = sum T alpha t* / W_n (0 when W_n <= 1e-8),
 *            W_n = sum T alpha;
 *   [9..17]  far field: each Gaussian with opacity >= alpha_min carries
 *            the optical mass -ln(1 - min(o, alpha_max)) 2 pi s_2 s_3 (its
 *            two largest scales) into the cubic cell of its quantised
 *            centre (fixed-point sums; 128 cells along the longest axis of
 *            the centres' bounding box, edge h); along the ray from t0 (the
 *            last listed Gaussian's distance when the list is full, else
 *            r_near) the cells' extinction sigma = mass / h^3 gives the
 *            optical depth tau; the features are 1 - exp(-tau) at t0 + h
 *            {2, 4, 8, 16, 32} and at the end of the grid, then the
 *            emission-absorption colour sum exp(-tau) (1 - exp(-sigma dt))
 *            rgb_cell (the march stops once tau > 20).
 * Network: 18 -> 64 -> 64 -> 64 -> 5, ReLU, no output activation:
 * y = (O, D / depth_scale, R, G, B); written to an atlas as O clamped to
 * [0, 1], D and RGB clamped at 0. Parameters: one float32 vector of
 * sop_surrogate_param_count() values in the order W1 [64][18], b1 [64],
 * W2 [64][64], b2, W3 [64][64], b3, W4 [5][64], b4 [5] (row-major, out x
 * in). Every matrix operand (weights, features, activations, back-
 * propagated deltas) is used as bfloat16 (nearest-even) with float32
 * accumulation; all four layers run on the tensor cores. Training: mean
 * absolute error over the 5 outputs (an L1 loss, like the L1 texture
 * supervision of Sec. 3.1.2), Adam (0.9, 0.999, 1e-8, bias-corrected) on
 * float32 master weights. */
#define SOP_SURROGATE_FEATURES 18
#define SOP_SURROGATE_NEAR_CAP 256
typedef struct sop_surrogate sop_surrogate; /* opaque handle */
int32_t sop_surrogate_param_count(void);
/* Bytes of the device state a handle works on (master weights, Adam
 * moments, gradient, bf16 copy, step), caller-owned, 256-byte aligned. */
size_t sop_surrogate_state_bytes(void);
/* Make a handle over the caller's device state [state_bytes]: parameters
 * from `params` (device [count] float32) or, when NULL, He-uniform initial
 * weights (bound sqrt(6 / fan_in); weight i draws splitmix64(seed + i))
 * with zero biases; Adam moments and step zero. r_near (> 0, world units)
 * is the near-field radius of the features. The handle itself is one
 * small host allocation that sop_surrogate_destroy frees; the library
 * allocates no device memory. Asynchronous. */
sop_status sop_surrogate_create(void* state, size_t state_bytes, const float* params, uint64_t seed, float r_near,
                                sop_surrogate** out, void* stream);
sop_status sop_surrogate_destroy(sop_surrogate* net);
/* Parameters in and out (device [count] float32); set_params resets Adam.
 * get_grad: the gradient summed by the last training step. Asynchronous. */
sop_status sop_surrogate_set_params(sop_surrogate* net, const float* params, void* stream);
sop_status sop_surrogate_get_params(const sop_surrogate* net, float* params, void* stream);
sop_status sop_surrogate_get_grad(const sop_surrogate* net, float* grad, void* stream);
/* Checkpoint: save writes the master weights, Adam moments and step to
 * the file `path`; load reads such a file into the handle (bf16 copy
 * refreshed, gradient zeroed), so that training resumes exactly where the
 * save left it. Both synchronise `stream`. File format (little-endian):
 * "SOPSURR2" (8 bytes), int32 count, int32 step, then count float32
 * parameters, count float32 first moments, count float32 second moments.
 * SOP_ERR_INVALID_ARG for a missing, short or mismatched file. */
sop_status sop_surrogate_save(const sop_surrogate* net, const char* path, void* stream);
sop_status sop_surrogate_load(sop_surrogate* net, const char* path, void* stream);
/* The checkpoint format from and to host arrays (no GPU involved). */
sop_status sop_surrogate_file_write(const char* path, int32_t count, int32_t step, const float* params,
                                    const float* m, const float* v);
sop_status sop_surrogate_file_read(const char* path, int32_t count, int32_t* step, float* params, float* m,
                                   float* v);
/* Workspace of sop_surrogate_features / _train / _infer on n Gaussians, P
 * probes of side R (256-byte aligned). */
size_t sop_surrogate_workspace_bytes(int64_t n_gauss, int32_t P, int32_t R);
/* Texel features of P probes (probe_pos [P,3] device) against the
 * Gaussians: feats [P][R*R][18] float32 (device); near_list [P][256] int32
 * (device, -1 after the last) or NULL. bake params give alpha_min and
 * alpha_max. Asynchronous. */
sop_status sop_surrogate_features(const sop_surrogate* net, const sop_gaussians* g, const float* probe_pos,
                                  int32_t P, int32_t R, const sop_bake_params* params, float* feats,
                                  int32_t* near_list, void* ws, size_t ws_bytes, void* stream);
/* Workspace of sop_surrogate_train alone (drawn batches, per-CTA partial
 * gradients that are summed in a fixed order, so that training is
 * bit-reproducible); sop_surrogate_workspace_bytes() covers it too. */
size_t sop_surrogate_train_workspace_bytes(void);
/* `steps` Adam steps at learning rate lr, each on `batch` probes of
 * targets (P probes, baked maps of side R) with their features feats
 * [P][R*R][18]: the probes probe_ids [batch] (device) when given, else
 * drawn for each step as splitmix64(seed ^ (step 2^32 + i)) mod P (with
 * replacement; step = the handle's step count). out_loss (device [steps]
 * float32, or NULL) receives each step's mean absolute error before its
 * update. 1 <= batch <= 65536. ws: sop_surrogate_train_workspace_bytes().
 * The result is the same on every run. Asynchronous. */
sop_status sop_surrogate_train(sop_surrogate* net, const float* feats, const int32_t* probe_ids, int32_t batch,
                               const sop_atlas* targets, int32_t steps, float lr, uint64_t seed, float* out_loss,
                               void* ws, size_t ws_bytes, void* stream);
/* The network on given features: the maps of B probes (probe_ids [B]
 * device, or NULL for 0..B-1, indexing feats and `out`) written into the
 * atlas `out` (interior; border by the border rule when all of out's
 * probes are predicted, i.e. probe_ids NULL and B = out->P). Asynchronous. */
sop_status sop_surrogate_predict(const sop_surrogate* net, const float* feats, const int32_t* probe_ids, int32_t B,
                                 const sop_atlas* out, void* stream);
/* The learned rebake of every probe of `out` (positions out->probe_pos)
 * against the Gaussians g, with its spot check and fallback, all on the
 * device: bin the Gaussians (as sop_bake_bin), compute the features,
 * predict every probe into `out`; ray-trace n = max(1, ceil(spot_frac P))
 * probes (probe i of the sample is floor((i + u_i) P / n), u_i =
 * splitmix64(seed + i) / 2^64: distinct and spread over the probes) and
 * compare their O with the prediction: err = mean |dO| over their interior
 * texels. If err > tau (or is not finite) every probe of `out` is
 * ray-traced instead (fallback); the checked probes always keep their
 * traced maps. out_spot_err (device float) receives err, out_fell_back
 * (device int32) 1 after a fallback, else 0. 0 < spot_frac <= 1.
 * Asynchronous: no host synchronisation, the decision is taken on the
 * device. The spot check runs on a second stream of the library's (made
 * once per device, greatest priority) beside the features and the network;
 * it waits for the work queued on `stream` before the call, and work queued
 * on `stream` after the call waits for it. Calls from several host threads
 * are serialised while they are queued. Not to be called across a
 * cudaDeviceReset (the second stream does not survive it). */
sop_status sop_surrogate_infer(const sop_surrogate* net, const sop_gaussians* g, const sop_atlas* out,
                               const sop_bake_params* params, float spot_frac, float tau, uint64_t seed,
                               float* out_spot_err, int32_t* out_fell_back, void* ws, size_t ws_bytes, void* stream);
/* Spot-check helpers: out[0] = sum |O_a - O_b| and out[1] = sum of |RGB_a -
 * RGB_b| over the interior texels of n probe pairs (a_probes[i],
 * b_probes[i]; NULL = 0..n-1), written to device out[2]; indices outside
 * an atlas are skipped (SOP_DEVSTAT_INDEX). */
sop_status sop_atlas_compare(const sop_atlas* a, const int32_t* a_probes, const sop_atlas* b, const int32_t* b_probes,
                             int32_t n, float* out, void* stream);
/* Copy whole probes (all (R+2)^2 texels) src_probes[i] -> dst_probes[i]. */
sop_status sop_atlas_copy(const sop_atlas* src, const int32_t* src_probes, const sop_atlas* dst,
                          const int32_t* dst_probes, int32_t n, void* stream);

/* Allocation-free sop_query_shade. No counterpart in the paper: this entry
 * point exists for callers that cannot allocate device memory, for example
 * code running where cudaMalloc is unavailable or forbidden (a host
 * framework that owns all allocations, a capture or plugin context, an
 * embedded runtime without an allocator). It takes the same arguments as
 * sop_query_shade except the workspace, allocates nothing, and computes the
 * same result (same K nearest probes, weights and shading) by reading the
 * atlas and the environment in the caller's own layouts.
 * Scratch: one fixed array of SOP_NOALLOC_SCRATCH_BYTES (8 MiB) of device
 * memory inside the library, held on every GPU that loads the library until
 * the process exits. Limits: the probe grid, the direction table and one
 * chunk of 16,384 points' neighbour lists must fit it, which holds for up to
 * SOP_NOALLOC_MAX_PROBES probes at any K <= 32 and S <= 4096 (larger P is
 * rejected with SOP_ERR_INVALID_ARG and a message; use sop_query_shade).
 * The first call on a device looks up the array's address on that device
 * and keeps it for the life of the process, so make that first call before
 * any CUDA stream capture on the device, and do not call this entry point
 * after a cudaDeviceReset() in the same process (the library's device
 * memory is reloaded then, and the kept address would be stale).
 * Every call uses the same array and leaves its contents behind; calls that
 * overlap on the GPU (other streams or host threads) race on it and must be
 * serialised by the caller. Asynchronous on `stream`. */
#define SOP_NOALLOC_SCRATCH_BYTES (8u << 20)
#define SOP_NOALLOC_MAX_PROBES 65536
sop_status sop_query_shade_noalloc(const float* x, const float* n, const float* wo, const float* albedo,
                                   const float* rough, const float* metal, int64_t M, const sop_atlas* atlas,
                                   const float* env, int32_t He, int32_t We, const float* dirs_local,
                                   const sop_shade_params* params, float* out, int32_t* out_idx, float* out_w,
                                   void* stream);

/* ---- deferred front end (Sec. 3.1 multi-target rendering, Sec. 4.3) -------- */

/* Per-Gaussian materials, device: albedo [N][3], roughness [N], metallic [N]. */
typedef struct {
    const float* albedo;
    const float* rough;
    const float* metal;
} sop_materials;

/* Workspace bytes for sop_trace_gbuffer on n Gaussians: the bake's grid
 * (sop_bake_bin builds it; a larger workspace holds more cell entries). */
size_t sop_trace_workspace_bytes(int64_t n_gauss);

/* Multi-target rendering (Sec. 3.1, the alpha blending of G-buffers
 * B = sum_i T_i alpha_i b_i with b_i = {c, 1, d, n, a, r, m}) of the
 * Gaussians g along n_origins x n_dirs rays: ray p n_dirs + t starts at
 * origins[p] ([n_origins][3], device) and runs along dirs[t] ([n_dirs][4],
 * device, 16-byte aligned; x, y, z used as given, unit length expected).
 * Each Gaussian is evaluated as in the bake (point of maximum density t*,
 * alpha = min(alpha_max, o exp(-m^2/2)), kept when alpha >= alpha_min and
 * t* > t_near), hits are composited in increasing (t*, index) order until
 * T < t_stop; d = t*; the normal n is the Gaussian's local axis of smallest
 * scale (the first of equal ones), turned against the ray (n . d <= 0).
 * out [rays][16] float32, device, 16-byte aligned: C.rgb, W, N.xyz, D,
 * A.rgb, R, M, 0, 0, 0 (W = sum T alpha; D / W is the unbiased depth along
 * the ray). ws must hold the grid that sop_bake_bin built for the same g and
 * params (with the same ws_bytes). Asynchronous. */
sop_status sop_trace_gbuffer(const sop_gaussians* g, const sop_materials* m, const float* origins,
                             int32_t n_origins, const float* dirs, int64_t n_dirs, const sop_bake_params* params,
                             float* out, void* ws, size_t ws_bytes, void* stream);

/* Ray directions of a pinhole camera, W x H pixels, row 0 at the top: pixel
 * (i, j) looks along f + sx r + sy u, sx = ((i + 1/2)/W 2 - 1) tan(fov/2)
 * W/H, sy = (1 - (j + 1/2)/H 2) tan(fov/2), with f the unit direction from
 * eye to target, r = f x up normalised, u = r x f (up replaced by +y when
 * within 0.99 of f). eye, target, up: host float[3]; fov_y in degrees,
 * (0, 180). out [H W][4] device (unit x, y, z, 0), computed in double and
 * rounded once. Asynchronous. */
sop_status sop_pinhole_dirs(int32_t W, int32_t H, const float* eye, const float* target, const float* up,
                            float fov_y_deg, float* out, void* stream);

/* Directions of an equirectangular panorama (the 360 degree sweep of
 * Sec. 4.2), z-up, the environment map's parameterisation: pixel (i, j) of
 * W x H has azimuth (i + 1/2)/W 2 pi - pi and polar angle (j + 1/2)/H pi.
 * out [H W][4] device. Asynchronous. */
sop_status sop_panorama_dirs(int32_t W, int32_t H, float* out, void* stream);

/* Workspace bytes for sop_gbuffer_points on n_pix pixels. */
size_t sop_gbuffer_points_workspace_bytes(int64_t n_pix);

/* Shading points of a G-buffer (Sec. 4.3; the unbiased depth of Sec. 3.1):
 * pixel p of gbuf [n_pix][16] (device) is kept when W >= w_min, N != 0 and,
 * with `front` (another G-buffer of the same pixels, or NULL) kept at p,
 * when D/W < D'/W' (float32 quotients). Kept pixels are written in pixel
 * order: out_pix [k] (int64), out_x = origin + (D/W) d, out_n = N/|N|,
 * out_wo = -d, out_albedo = A/W ([k][3] each), out_rough = R/W,
 * out_metal = M/W ([k]); origin is a host float[3], dirs [n_pix][4] the
 * pixels' directions. out_count: one device int64, the number kept. Output
 * arrays hold n_pix entries at most. Asynchronous. */
sop_status sop_gbuffer_points(const float* gbuf, const float* front, int64_t n_pix, const float* origin,
                              const float* dirs, float w_min, int64_t* out_pix, float* out_x, float* out_n,
                              float* out_wo, float* out_albedo, float* out_rough, float* out_metal,
                              int64_t* out_count, void* ws, size_t ws_bytes, void* stream);

/* Depth compositing of the composed frame (Sec. 4.3): out [n_pix][3] =
 * the scene's traced colour C_s (scene_gbuf), multiplied at the scene's
 * shading points sc_pix [n_sc] by their shadow ratio shadow [n_sc][3]
 * (Eq. 9); then at the object's shading points obj_pix [n_obj] (the pixels
 * where it lies in front, from sop_gbuffer_points with front = scene_gbuf)
 * W_o obj_rgb + (1 - W_o) out, W_o the object's G-buffer weight. Pixel
 * lists hold distinct pixels; entries outside [0, n_pix) are skipped.
 * All device. Asynchronous. */
sop_status sop_depth_composite(const float* scene_gbuf, const float* obj_gbuf, int64_t n_pix, const int64_t* sc_pix,
                               const float* shadow, int64_t n_sc, const int64_t* obj_pix, const float* obj_rgb,
                               int64_t n_obj, float* out, void* stream);

/* ---- automatic placement of SOPs (Sec. 3.2) ---------------------------------- */

/* Workspace bytes for sop_place_probes on n points. */
size_t sop_place_probes_workspace_bytes(int64_t n_points);

/* Farthest point sampling of the surface points pts [n][3] (device; within
 * +-1024), then the offset of each chosen point along its normal (Sec. 3.2:
 * probes slightly off the surface). Distances are the exact integer squared
 * distances of positions quantised to 2^-20: the first point is `start`,
 * each next one maximises the smallest distance to the points already
 * chosen, ties to the lower index; the result is that of a sequential FPS
 * and the same on every run. out_idx [k] (int64, device): the chosen
 * points in order; out_pos [k][3] (device, or NULL): pts + offset nrm,
 * computed in double and rounded once (nrm [n][3] device, or NULL: no
 * offset). 1 <= k <= n, 0 <= start < n. Runs as one thread-block cluster
 * (16 CTAs where the device holds such a cluster, else 8) for all k
 * iterations. Asynchronous. */
sop_status sop_place_probes(const float* pts, const float* nrm, int64_t n_points, int32_t k, int64_t start,
                            float offset, int64_t* out_idx, float* out_pos, void* ws, size_t ws_bytes, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SOP_H */
