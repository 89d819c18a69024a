// C ABI of libsop: argument validation, workspace layout, launch sequencing.
#include <math.h>
#include <stdarg.h>
#include <stdlib.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <stdio.h>
#include <string.h>

#include "sop_device.cuh"
#include "sop_internal.h"

namespace {

thread_local char g_err[512] = "";

sop_status fail(sop_status st, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

sop_status cuda_status(cudaError_t e, const char* where)
{
    if (e == cudaSuccess) return SOP_OK;
    return fail(SOP_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

bool dtype_ok(int32_t dt, bool depth)
{
    if (dt == SOP_F32 || dt == SOP_BF16 || dt == SOP_F16) return true;
    return depth && dt == SOP_FP8E4M3;
}

size_t rgbo_texel_bytes(int32_t dt) { return dt == SOP_F32 ? 16 : 8; }
size_t depth_texel_bytes(int32_t dt) { return dt == SOP_F32 ? 4 : (dt == SOP_FP8E4M3 ? 1 : 2); }

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

sop_status check_atlas(const sop_atlas* a, bool need_depth)
{
    if (!a) return fail(SOP_ERR_INVALID_ARG, "atlas is NULL");
    if (a->P < 1) return fail(SOP_ERR_INVALID_ARG, "atlas P = %d < 1", a->P);
    if (a->R < 2 || a->R > 64) return fail(SOP_ERR_INVALID_ARG, "atlas R = %d outside [2, 64]", a->R);
    if (!dtype_ok(a->rgbo_dtype, false))
        return fail(SOP_ERR_UNSUPPORTED, "atlas rgbo dtype %d not supported (F32, BF16, F16)", a->rgbo_dtype);
    if (!a->rgbo || !aligned(a->rgbo, 16)) return fail(SOP_ERR_INVALID_ARG, "atlas rgbo NULL or not 16-byte aligned");
    if (!a->probe_pos) return fail(SOP_ERR_INVALID_ARG, "atlas probe_pos is NULL");
    if (need_depth && a->depth) {
        if (!dtype_ok(a->depth_dtype, true))
            return fail(SOP_ERR_UNSUPPORTED, "atlas depth dtype %d not supported", a->depth_dtype);
        if (!(a->depth_scale > 0.f) || !isfinite(a->depth_scale))
            return fail(SOP_ERR_INVALID_ARG, "atlas depth_scale must be finite and > 0");
    }
    return SOP_OK;
}

sop_status check_ws(void* ws, size_t ws_bytes, size_t need)
{
    if (need == 0) return SOP_OK;
    if (!ws) return fail(SOP_ERR_WORKSPACE, "workspace is NULL (%zu bytes needed)", need);
    if (!aligned(ws, 256)) return fail(SOP_ERR_WORKSPACE, "workspace not 256-byte aligned");
    if (ws_bytes < need) return fail(SOP_ERR_WORKSPACE, "workspace too small: %zu < %zu bytes", ws_bytes, need);
    return SOP_OK;
}

sop_status check_shade(const sop_shade_params* p, int32_t P)
{
    if (!p) return fail(SOP_ERR_INVALID_ARG, "params is NULL");
    if (p->K < 1 || p->K > 32) return fail(SOP_ERR_INVALID_ARG, "K = %d outside [1, 32]", p->K);
    if (p->K > P) return fail(SOP_ERR_INVALID_ARG, "K = %d exceeds the number of probes %d", p->K, P);
    if (p->S < 1 || p->S > 4096) return fail(SOP_ERR_INVALID_ARG, "S = %d outside [1, 4096]", p->S);
    if (p->mode != SOP_MODE_SHADE && p->mode != SOP_MODE_SHADOW)
        return fail(SOP_ERR_INVALID_ARG, "mode = %d is neither SHADE nor SHADOW", p->mode);
    if (!(p->eps_snap >= 0.f) || !isfinite(p->eps_snap)) return fail(SOP_ERR_INVALID_ARG, "eps_snap must be >= 0");
    if (!isfinite(p->specular)) return fail(SOP_ERR_INVALID_ARG, "specular must be finite");
    if (p->env_layout != SOP_ENV_EQUIRECT && p->env_layout != SOP_ENV_OCTAHEDRAL)
        return fail(SOP_ERR_INVALID_ARG, "env_layout = %d is neither EQUIRECT nor OCTAHEDRAL", p->env_layout);
    if (p->dir_world != 0 && p->dir_world != 1) return fail(SOP_ERR_INVALID_ARG, "dir_world must be 0 or 1");
    if (!(p->radius >= 0.f && p->radius <= 2048.f))
        return fail(SOP_ERR_INVALID_ARG, "radius = %g outside [0, 2048]", (double)p->radius);
    return SOP_OK;
}

// Largest integer squared distance (units of 2^-40) within a search radius:
// (radius 2^20)^2 has at most 48 significant bits, so the double square is
// exact and its floor is the bound. Radius 0 means no bound.
uint64_t radius_key(float radius)
{
    if (radius == 0.f) return UINT64_MAX;
    const double r = (double)radius * 1048576.0;
    return (uint64_t)floor(r * r);
}

}  // namespace

extern "C" {

const char* sop_last_error(void) { return g_err; }

const char* sop_version(void) { return "libsop 0.2 (sm_103a)"; }

sop_status sop_device_status(void* stream, uint32_t* out_bits, int32_t clear)
{
    uint32_t bits = 0;
    sop_status st = cuda_status(sop::status_take(&bits, clear != 0, (cudaStream_t)stream), "sop_device_status");
    if (st != SOP_OK) return st;
    if (out_bits) *out_bits = bits;
    if (bits & SOP_DEVSTAT_ERRORS) return fail(SOP_ERR_DEVICE, "device status 0x%x: %s", bits, sop::status_bits_message(bits));
    return SOP_OK;
}

sop_status sop_atlas_bytes(int32_t P, int32_t R, int32_t rgbo_dtype, int32_t depth_dtype, size_t* rgbo_bytes,
                           size_t* depth_bytes)
{
    if (P < 1 || R < 2 || R > 64) return fail(SOP_ERR_INVALID_ARG, "P = %d, R = %d invalid", P, R);
    if (!dtype_ok(rgbo_dtype, false) || !dtype_ok(depth_dtype, true))
        return fail(SOP_ERR_INVALID_ARG, "unknown dtype (%d, %d)", rgbo_dtype, depth_dtype);
    const size_t tex = (size_t)P * (R + 2) * (R + 2);
    if (rgbo_bytes) *rgbo_bytes = tex * rgbo_texel_bytes(rgbo_dtype);
    if (depth_bytes) *depth_bytes = tex * depth_texel_bytes(depth_dtype);
    return SOP_OK;
}

sop_status sop_atlas_pack(const float* maps_rgb, const float* maps_occ, const float* maps_depth,
                          const sop_atlas* atlas, void* stream)
{
    sop_status st = check_atlas(atlas, maps_depth != nullptr);
    if (st != SOP_OK) return st;
    if (!maps_rgb || !maps_occ) return fail(SOP_ERR_INVALID_ARG, "maps_rgb / maps_occ is NULL");
    return cuda_status(sop::launch_atlas_pack(maps_rgb, 3, maps_occ, 1, maps_depth, *atlas, (cudaStream_t)stream),
                       "sop_atlas_pack");
}

sop_status sop_atlas_pack_rgbo(const float* maps_rgbo, const sop_atlas* atlas, void* stream)
{
    sop_status st = check_atlas(atlas, false);
    if (st != SOP_OK) return st;
    if (!maps_rgbo) return fail(SOP_ERR_INVALID_ARG, "maps_rgbo is NULL");
    return cuda_status(sop::launch_atlas_pack(maps_rgbo, 4, maps_rgbo + 3, 4, nullptr, *atlas, (cudaStream_t)stream),
                       "sop_atlas_pack_rgbo");
}

sop_status sop_hammersley(int32_t S, float* out_dirs, void* stream)
{
    if (S < 1 || S > 4096) return fail(SOP_ERR_INVALID_ARG, "S = %d outside [1, 4096]", S);
    if (!out_dirs) return fail(SOP_ERR_INVALID_ARG, "out_dirs is NULL");
    return cuda_status(sop::launch_hammersley(S, out_dirs, (cudaStream_t)stream), "sop_hammersley");
}

sop_status sop_l1_loss_grad(const float* C, const float* C_target, int64_t n, float* grad, float* loss_sum,
                            void* stream)
{
    if (n < 0) return fail(SOP_ERR_INVALID_ARG, "n = %lld < 0", (long long)n);
    if (n > 0 && (!C || !C_target || !grad)) return fail(SOP_ERR_INVALID_ARG, "C, C_target or grad is NULL");
    return cuda_status(sop::launch_l1_grad(C, C_target, n, grad, loss_sum, (cudaStream_t)stream), "sop_l1_loss_grad");
}

sop_status sop_adam_l1_step(float* p, const float* g, float* m, float* v, int64_t n, const sop_adam_params* a,
                            void* stream)
{
    if (!a) return fail(SOP_ERR_INVALID_ARG, "params is NULL");
    if (n < 0) return fail(SOP_ERR_INVALID_ARG, "n = %lld < 0", (long long)n);
    if (n > 0 && (!p || !m || !v)) return fail(SOP_ERR_INVALID_ARG, "p, m or v is NULL");
    if (a->period < 1 || a->split < 0 || a->split > a->period)
        return fail(SOP_ERR_INVALID_ARG, "period = %d, split = %d: need period >= 1 and 0 <= split <= period",
                    a->period, a->split);
    if (a->step < 1) return fail(SOP_ERR_INVALID_ARG, "step = %d < 1", a->step);
    if (!(a->lr > 0.f) || !(a->beta1 >= 0.f && a->beta1 < 1.f) || !(a->beta2 >= 0.f && a->beta2 < 1.f) ||
        !(a->eps >= 0.f))
        return fail(SOP_ERR_INVALID_ARG, "lr must be > 0, beta1/beta2 in [0, 1), eps >= 0");
    return cuda_status(sop::launch_adam_l1(p, g, m, v, n, *a, (cudaStream_t)stream), "sop_adam_l1_step");
}

sop_status sop_env_to_octahedral(const float* env, int32_t He, int32_t We, float* out, int32_t H, void* stream)
{
    if (!env || !out) return fail(SOP_ERR_INVALID_ARG, "env or out is NULL");
    if (He < 1 || We < 1 || (int64_t)He * We > ((int64_t)1 << 28))
        return fail(SOP_ERR_INVALID_ARG, "environment size %d x %d invalid", He, We);
    if (H < 2 || H > 4096) return fail(SOP_ERR_INVALID_ARG, "H = %d outside [2, 4096]", H);
    return cuda_status(sop::launch_env_to_oct(env, He, We, out, H, (cudaStream_t)stream), "sop_env_to_octahedral");
}

size_t sop_env_importance_workspace_bytes(int32_t H)
{
    if (H < 2 || H > 2048) return 0;
    return sop::importance_ws_bytes(H);
}

sop_status sop_env_importance_dirs(const float* env, int32_t H, int32_t S, float* out, void* ws, size_t ws_bytes,
                                   void* stream)
{
    if (!env || !out) return fail(SOP_ERR_INVALID_ARG, "env or out is NULL");
    if (H < 2 || H > 2048) return fail(SOP_ERR_INVALID_ARG, "H = %d outside [2, 2048]", H);
    if (S < 1 || S > 4096) return fail(SOP_ERR_INVALID_ARG, "S = %d outside [1, 4096]", S);
    sop_status st = check_ws(ws, ws_bytes, sop::importance_ws_bytes(H));
    if (st != SOP_OK) return st;
    return cuda_status(sop::launch_importance_dirs(env, H, S, out, (char*)ws, (cudaStream_t)stream),
                       "sop_env_importance_dirs");
}

sop_status sop_read_bandwidth_probe(const void* buf, size_t bytes, int32_t reps, float* sink, void* stream)
{
    if (!buf || !sink) return fail(SOP_ERR_INVALID_ARG, "buf or sink is NULL");
    if (bytes < 16 || bytes % 16 != 0 || ((uintptr_t)buf & 15u) != 0)
        return fail(SOP_ERR_INVALID_ARG, "buf must be 16-byte aligned and bytes a positive multiple of 16");
    if (reps < 1) return fail(SOP_ERR_INVALID_ARG, "reps = %d < 1", reps);
    return cuda_status(sop::launch_read_probe(buf, bytes, reps, sink, (cudaStream_t)stream),
                       "sop_read_bandwidth_probe");
}

size_t sop_bake_workspace_bytes(int64_t n_gauss, int32_t P, int32_t R)
{
    if (n_gauss < 0 || P < 1 || R < 2) return 0;
    return sop::bake_layout(n_gauss, 0).total;
}

static sop_status check_bake_args(const sop_gaussians* g, const sop_bake_params* params)
{
    if (!g || !params) return fail(SOP_ERR_INVALID_ARG, "gaussians or params is NULL");
    if (g->n < 0 || g->n > (int64_t)INT32_MAX) return fail(SOP_ERR_INVALID_ARG, "n = %lld out of range", (long long)g->n);
    if (g->n > 0 && (!g->mean || !g->scale || !g->quat || !g->opacity || !g->rgb))
        return fail(SOP_ERR_INVALID_ARG, "a Gaussian array is NULL");
    if (!(params->alpha_min > 0.f) || !(params->alpha_max >= params->alpha_min) || !(params->alpha_max < 1.f) ||
        !(params->t_stop >= 0.f) || !(params->t_stop < 1.f) || !isfinite(params->t_near) ||
        !(params->grid_density == 0.f || (params->grid_density >= 0.01f && params->grid_density <= 2.f)))
        return fail(SOP_ERR_INVALID_ARG, "bake params out of range (need 0 < alpha_min <= alpha_max < 1, "
                                         "0 <= t_stop < 1, finite t_near, grid_density 0 or in [0.01, 2])");
    return SOP_OK;
}

// The layout with the largest cell-entry capacity that fits ws_bytes. The
// workspace must hold at least the default capacity (24 entries per Gaussian
// plus 65,536), which the device-side binning relies on: its last attempt,
// a grid of at most 2 cells, needs at most 2 entries per Gaussian.
static sop_status bake_fit(int64_t n, float density, void* ws, size_t ws_bytes, sop::BakeLayout& L)
{
    const sop::BakeLayout Lmin = sop::bake_layout(n, 0, density);
    sop_status st = check_ws(ws, ws_bytes, Lmin.total);
    if (st != SOP_OK) return st;
    const sop::BakeLayout L1 = sop::bake_layout(n, 1, density);
    int64_t cap = 1 + (int64_t)((ws_bytes - L1.total) / sop::kBakeEntryBytes);
    L = sop::bake_layout(n, cap, density);
    while (L.total > ws_bytes && L.entries_cap > Lmin.entries_cap) L = sop::bake_layout(n, L.entries_cap - 1, density);
    return check_ws(ws, ws_bytes, L.total);
}

sop_status sop_bake_bin(const sop_gaussians* g, const sop_bake_params* params, void* ws, size_t ws_bytes,
                        void* stream)
{
    sop_status st = check_bake_args(g, params);
    if (st != SOP_OK) return st;
    sop::BakeLayout L;
    if ((st = bake_fit(g->n, params->grid_density, ws, ws_bytes, L)) != SOP_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    char* w = (char*)ws;
    st = cuda_status(sop::launch_bake_bin(*g, params->alpha_min, L, w, s), "sop_bake_bin (binning)");
    if (st != SOP_OK) return st;
    return cuda_status(sop::launch_bake_fill(*g, L, w, s), "sop_bake_bin (fill)");
}

sop_status sop_bake_trace(const sop_gaussians* g, const sop_atlas* atlas, const sop_bake_params* params, void* ws,
                          size_t ws_bytes, void* stream)
{
    sop_status st = check_bake_args(g, params);
    if (st != SOP_OK) return st;
    if ((st = check_atlas(atlas, true)) != SOP_OK) return st;
    if ((int64_t)atlas->P * atlas->R * atlas->R > (int64_t)INT32_MAX)
        return fail(SOP_ERR_INVALID_ARG, "P * R^2 exceeds 2^31 texels");
    sop::BakeLayout L;
    if ((st = bake_fit(g->n, params->grid_density, ws, ws_bytes, L)) != SOP_OK) return st;
    return cuda_status(sop::launch_bake_trace(*atlas, *params, L, (char*)ws, (cudaStream_t)stream), "sop_bake_trace");
}

sop_status sop_bake(const sop_gaussians* g, const sop_atlas* atlas, const sop_bake_params* params, void* ws,
                    size_t ws_bytes, void* stream)
{
    sop_status st = check_bake_args(g, params);
    if (st != SOP_OK) return st;
    if ((st = check_atlas(atlas, true)) != SOP_OK) return st;
    if ((int64_t)atlas->P * atlas->R * atlas->R > (int64_t)INT32_MAX)
        return fail(SOP_ERR_INVALID_ARG, "P * R^2 exceeds 2^31 texels");
    if ((st = sop_bake_bin(g, params, ws, ws_bytes, stream)) != SOP_OK) return st;
    return sop_bake_trace(g, atlas, params, ws, ws_bytes, stream);
}

sop_status sop_bake_stats(const void* ws, size_t ws_bytes, int64_t n_gauss, int64_t* out, void* stream)
{
    if (!out) return fail(SOP_ERR_INVALID_ARG, "out is NULL");
    sop::BakeLayout L;
    sop_status st = bake_fit(n_gauss, 0.f, const_cast<void*>(ws), ws_bytes, L);
    if (st != SOP_OK) return st;
    unsigned long long v[5];
    cudaStream_t s = (cudaStream_t)stream;
    st = cuda_status(cudaMemcpyAsync(v, (const char*)ws + L.stats, sizeof(v), cudaMemcpyDeviceToHost, s),
                     "sop_bake_stats");
    if (st != SOP_OK) return st;
    st = cuda_status(cudaStreamSynchronize(s), "sop_bake_stats (sync)");
    if (st != SOP_OK) return st;
    out[0] = (int64_t)v[1];
    out[1] = (int64_t)v[2];
    out[2] = (int64_t)v[3];
    out[3] = (int64_t)v[4];
    return SOP_OK;
}

size_t sop_query_workspace_bytes(const sop_atlas* atlas, int64_t M, const sop_shade_params* params, int32_t He,
                                 int32_t We)
{
    if (!atlas || !params || atlas->P < 1 || atlas->R < 2 || M < 0 || He < 1 || We < 1 || params->K < 1 ||
        params->S < 1)
        return 0;
    return sop::query_layout(atlas->P, M, params->K, params->S, He, We, atlas->R, atlas->rgbo_dtype).total;
}

static sop_status query_common(const float* x, const float* n, const float* wo, const float* albedo, const float* rough,
                               const float* metal, int64_t M, const sop_atlas* atlas, const float* env, int32_t He,
                               int32_t We, const float* dirs_local, const sop_shade_params* params, void* ws,
                               size_t ws_bytes, sop::QueryArgs& a, sop::QueryLayout& L)
{
    sop_status st = check_atlas(atlas, false);
    if (st != SOP_OK) return st;
    st = check_shade(params, atlas->P);
    if (st != SOP_OK) return st;
    if (M < 0 || M > ((int64_t)1 << 36)) return fail(SOP_ERR_INVALID_ARG, "M = %lld out of range", (long long)M);
    // the shading kernels index the probes' bilinear footprints (P (R+1)^2 of
    // them) with 32-bit integers
    if ((int64_t)atlas->P * (atlas->R + 1) * (atlas->R + 1) > (int64_t)INT32_MAX)
        return fail(SOP_ERR_INVALID_ARG, "P * (R+1)^2 = %lld footprints exceeds 2^31 - 1",
                    (long long)atlas->P * (atlas->R + 1) * (atlas->R + 1));
    if (He < 1 || We < 1 || (int64_t)He * We > ((int64_t)1 << 28))
        return fail(SOP_ERR_INVALID_ARG, "environment size %d x %d invalid", He, We);
    if (params->env_layout == SOP_ENV_OCTAHEDRAL && (He != We || He < 2))
        return fail(SOP_ERR_INVALID_ARG, "an octahedral environment is square, H >= 2 (got %d x %d)", He, We);
    if (!env) return fail(SOP_ERR_INVALID_ARG, "env is NULL");
    if (params->dir_world && !dirs_local)
        return fail(SOP_ERR_INVALID_ARG, "dir_world = 1 needs the world directions [S][4] in dirs_local");
    if (M > 0 && (!x || !n || !wo || !albedo || !rough || !metal))
        return fail(SOP_ERR_INVALID_ARG, "a shading-point array is NULL");
    L = sop::query_layout(atlas->P, M, params->K, params->S, He, We, atlas->R, atlas->rgbo_dtype);
    st = check_ws(ws, ws_bytes, L.total);
    if (st != SOP_OK) return st;
    a = sop::QueryArgs{};
    a.x = x;
    a.n = n;
    a.wo = wo;
    a.albedo = albedo;
    a.rough = rough;
    a.metal = metal;
    a.M = M;
    a.rgbo = atlas->rgbo;
    a.rgbo_dtype = atlas->rgbo_dtype;
    a.P = atlas->P;
    a.R = atlas->R;
    a.probe_pos = atlas->probe_pos;
    a.env = env;
    a.He = He;
    a.We = We;
    a.dirs_local = dirs_local;
    a.K = params->K;
    a.S = params->S;
    a.mode = params->mode;
    a.env_layout = params->env_layout;
    a.dir_world = params->dir_world;
    a.specular = params->specular;
    const double e = (double)params->eps_snap * 1048576.0;
    a.snap_key = (uint64_t)floor(e * e);
    a.r2_key = radius_key(params->radius);
    return SOP_OK;
}

sop_status sop_query_shade(const float* x, const float* n, const float* wo, const float* albedo, const float* rough,
                           const float* metal, int64_t M, const sop_atlas* atlas, const float* env, int32_t He,
                           int32_t We, const float* dirs_local, const sop_shade_params* params, float* out,
                           int32_t* out_idx, float* out_w, void* ws, size_t ws_bytes, void* stream)
{
    sop::QueryArgs a;
    sop::QueryLayout L;
    sop_status st = query_common(x, n, wo, albedo, rough, metal, M, atlas, env, He, We, dirs_local, params, ws,
                                 ws_bytes, a, L);
    if (st != SOP_OK) return st;
    if (M > 0 && !out) return fail(SOP_ERR_INVALID_ARG, "out is NULL");
    a.out = out;
    a.out_idx = out_idx;
    a.out_w = out_w;
    cudaStream_t s = (cudaStream_t)stream;
    st = cuda_status(sop::launch_query_prep(a, L, (char*)ws, s), "sop_query_shade (prep)");
    if (st != SOP_OK) return st;
    return cuda_status(sop::launch_shade(a, L, (char*)ws, s), "sop_query_shade (shade)");
}

sop_status sop_query_shade_backward(const float* x, const float* n, const float* wo, const float* albedo,
                                    const float* rough, const float* metal, int64_t M, const sop_atlas* atlas,
                                    const float* env, int32_t He, int32_t We, const float* dirs_local,
                                    const sop_shade_params* params, const float* grad_out, float* g_albedo,
                                    float* g_rough, float* g_metal, float* g_normal, float* g_env, float* g_maps,
                                    void* ws, size_t ws_bytes, void* stream)
{
    sop::QueryArgs a;
    sop::QueryLayout L;
    sop_status st = query_common(x, n, wo, albedo, rough, metal, M, atlas, env, He, We, dirs_local, params, ws,
                                 ws_bytes, a, L);
    if (st != SOP_OK) return st;
    if (params && (params->env_layout != SOP_ENV_EQUIRECT || params->dir_world))
        return fail(SOP_ERR_UNSUPPORTED,
                    "the adjoint takes the equirectangular environment layout and local directions only");
    if (params->mode != SOP_MODE_SHADE)
        return fail(SOP_ERR_UNSUPPORTED, "sop_query_shade_backward: only SOP_MODE_SHADE has an adjoint");
    if (M > 0 && (!grad_out || !g_albedo || !g_rough || !g_metal || !g_normal))
        return fail(SOP_ERR_INVALID_ARG, "a per-point gradient array is NULL");
    if (!g_env || !g_maps) return fail(SOP_ERR_INVALID_ARG, "g_env / g_maps is NULL");
    if (!aligned(g_maps, 16)) return fail(SOP_ERR_INVALID_ARG, "g_maps must be 16-byte aligned");
    a.grad_out = grad_out;
    a.g_albedo = g_albedo;
    a.g_rough = g_rough;
    a.g_metal = g_metal;
    a.g_normal = g_normal;
    a.g_env = g_env;
    a.g_atlas = g_maps;
    cudaStream_t s = (cudaStream_t)stream;
    st = cuda_status(sop::launch_query_prep(a, L, (char*)ws, s), "sop_query_shade_backward (prep)");
    if (st != SOP_OK) return st;
    return cuda_status(sop::launch_adjoint(a, L, (char*)ws, s), "sop_query_shade_backward");
}

sop_status sop_query_shade_noalloc(const float* x, const float* n, const float* wo, const float* albedo,
                                   const float* rough, const float* metal, int64_t M, const sop_atlas* atlas,
                                   const float* env, int32_t He, int32_t We, const float* dirs_local,
                                   const sop_shade_params* params, float* out, int32_t* out_idx, float* out_w,
                                   void* stream)
{
    sop_status st = check_atlas(atlas, false);
    if (st != SOP_OK) return st;
    st = check_shade(params, atlas->P);
    if (st != SOP_OK) return st;
    if (params->env_layout != SOP_ENV_EQUIRECT || params->dir_world)
        return fail(SOP_ERR_UNSUPPORTED,
                    "sop_query_shade_noalloc takes the equirectangular environment layout and local directions only");
    const size_t need = sop::noalloc_required_bytes(atlas->P, params->K, params->S);
    if (atlas->P > SOP_NOALLOC_MAX_PROBES || need > sop::noalloc_scratch_bytes())
        return fail(SOP_ERR_INVALID_ARG,
                    "sop_query_shade_noalloc: P = %d, K = %d, S = %d need %zu bytes of scratch, more than the "
                    "fixed %zu (at most %d probes with K = 32 and S = 4096); use sop_query_shade with a workspace",
                    atlas->P, params->K, params->S, need, sop::noalloc_scratch_bytes(), SOP_NOALLOC_MAX_PROBES);
    if (M < 0 || M > ((int64_t)1 << 36)) return fail(SOP_ERR_INVALID_ARG, "M = %lld out of range", (long long)M);
    if (He < 1 || We < 1 || (int64_t)He * We > ((int64_t)1 << 28))
        return fail(SOP_ERR_INVALID_ARG, "environment size %d x %d invalid", He, We);
    if (!env) return fail(SOP_ERR_INVALID_ARG, "env is NULL");
    if (M > 0 && (!x || !n || !wo || !albedo || !rough || !metal || !out))
        return fail(SOP_ERR_INVALID_ARG, "a shading-point array is NULL");
    sop::QueryArgs a{};
    a.x = x;
    a.n = n;
    a.wo = wo;
    a.albedo = albedo;
    a.rough = rough;
    a.metal = metal;
    a.M = M;
    a.rgbo = atlas->rgbo;
    a.rgbo_dtype = atlas->rgbo_dtype;
    a.P = atlas->P;
    a.R = atlas->R;
    a.probe_pos = atlas->probe_pos;
    a.env = env;
    a.He = He;
    a.We = We;
    a.dirs_local = dirs_local;
    a.K = params->K;
    a.S = params->S;
    a.mode = params->mode;
    a.env_layout = params->env_layout;
    a.dir_world = params->dir_world;
    a.specular = params->specular;
    const double e = (double)params->eps_snap * 1048576.0;
    a.snap_key = (uint64_t)floor(e * e);
    a.r2_key = radius_key(params->radius);
    a.out = out;
    a.out_idx = out_idx;
    a.out_w = out_w;
    return cuda_status(sop::launch_query_noalloc(a, (cudaStream_t)stream), "sop_query_shade_noalloc");
}

// ---- learned bake surrogate ----------------------------------------------------
}  // extern "C"

struct sop_surrogate {
    uint32_t magic;
    char* state;
    float r_near;
};

namespace {

constexpr uint32_t kSurrMagic = 0x53555232u;  // "SUR2"
constexpr int32_t kMaxBatch = 65536;

sop_status check_net(const sop_surrogate* net)
{
    if (!net || net->magic != kSurrMagic) return fail(SOP_ERR_INVALID_ARG, "not a surrogate handle");
    return SOP_OK;
}

// the surrogate's workspace: a bake workspace (grid, records), the feature
// scratch, the features, a spot-check atlas for up to P probes, the sample
struct SurrRunLayout {
    size_t bake, feat, feats, spot_rgbo, spot_depth, spot_ids, spot_pos, sums, ids, total;
    sop::BakeLayout B;
};

SurrRunLayout surr_run_layout(int64_t n, int32_t P, int32_t R)
{
    SurrRunLayout L{};
    L.B = sop::bake_layout(n, 0, 0.f);
    const size_t tex = (size_t)P * (R + 2) * (R + 2);
    size_t o = 0;
    L.bake = o;       o = sop::align256(o + L.B.total);
    L.feat = o;       o = sop::align256(o + sop::surr_feat_layout(n, P, R).total);
    L.feats = o;      o = sop::align256(o + sizeof(float) * (size_t)P * R * R * sop::surr_n_features());
    L.spot_rgbo = o;  o = sop::align256(o + 16 * tex);
    L.spot_depth = o; o = sop::align256(o + 4 * tex);
    L.spot_ids = o;   o = sop::align256(o + sizeof(int32_t) * (size_t)P);
    L.spot_pos = o;   o = sop::align256(o + 3 * sizeof(float) * (size_t)P);
    L.sums = o;       o = sop::align256(o + 4 * sizeof(float));
    L.ids = o;        o = sop::align256(o + sizeof(int32_t) * (size_t)kMaxBatch);
    L.total = o;
    return L;
}

sop_status check_gauss(const sop_gaussians* g)
{
    if (!g) return fail(SOP_ERR_INVALID_ARG, "gaussians is NULL");
    if (g->n < 1 || g->n > (int64_t)INT32_MAX) return fail(SOP_ERR_INVALID_ARG, "n = %lld out of range", (long long)g->n);
    if (!g->mean || !g->scale || !g->quat || !g->opacity || !g->rgb)
        return fail(SOP_ERR_INVALID_ARG, "a Gaussian array is NULL");
    return SOP_OK;
}

// features of every probe of `atlas`-sized sets into the run workspace
// Two more streams for the rebake. The spot check needs the Gaussian records
// but not the features or the network, so it runs beside them on `s`, made
// with the greatest priority (its chain of small launches is short of
// parallelism; the features fill the GPU). The far field's grid and march
// run on `far`, beside the near field's composite. One pair per device, made
// on first use, with the events that fork and join them. The mutex keeps the
// events of overlapping calls from interleaving while they are enqueued.
struct SideStream {
    cudaStream_t s = nullptr, far = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr, list = nullptr, far_done = nullptr;
    bool tried = false, ok = false;
};
constexpr int kMaxDevices = 64;
std::mutex g_side_mu;
SideStream g_side[kMaxDevices];

// the current device's side stream, or NULL when it cannot be made (the
// rebake then runs on the caller's stream alone); call with g_side_mu held
SideStream* side_stream()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return nullptr;
    }
    SideStream& r = g_side[dev];
    if (!r.tried) {
        r.tried = true;
        int least = 0, greatest = 0;
        r.ok = cudaDeviceGetStreamPriorityRange(&least, &greatest) == cudaSuccess &&
               cudaStreamCreateWithPriority(&r.s, cudaStreamNonBlocking, greatest) == cudaSuccess &&
               cudaStreamCreateWithFlags(&r.far, cudaStreamNonBlocking) == cudaSuccess &&
               cudaEventCreateWithFlags(&r.fork, cudaEventDisableTiming) == cudaSuccess &&
               cudaEventCreateWithFlags(&r.join, cudaEventDisableTiming) == cudaSuccess &&
               cudaEventCreateWithFlags(&r.list, cudaEventDisableTiming) == cudaSuccess &&
               cudaEventCreateWithFlags(&r.far_done, cudaEventDisableTiming) == cudaSuccess;
        cudaGetLastError();  // a failed creation leaves no error for later calls
    }
    return r.ok ? &r : nullptr;
}

sop_status surr_feats_into(const sop_surrogate* net, const sop_gaussians* g, const float* probe_pos, int32_t P,
                           int32_t R, const sop_bake_params* bp, float* feats, int32_t* list, char* w,
                           const SurrRunLayout& L, cudaStream_t s, const char* what)
{
    sop_status st = cuda_status(sop::launch_bake_bin(*g, bp->alpha_min, L.B, w + L.bake, s), what);
    if (st != SOP_OK) return st;
    st = cuda_status(sop::launch_bake_fill(*g, L.B, w + L.bake, s), what);
    if (st != SOP_OK) return st;
    return cuda_status(sop::surr_features(*g, probe_pos, P, R, net->r_near, bp->alpha_min, bp->alpha_max,
                                          w + L.bake + L.B.rec, feats, list, w + L.feat, s),
                       what);
}

}  // namespace

extern "C" {

int32_t sop_surrogate_param_count(void) { return sop::surr_n_params(); }

size_t sop_surrogate_state_bytes(void) { return sop::surr_state_bytes(); }

sop_status sop_surrogate_create(void* state, size_t state_bytes, const float* params, uint64_t seed, float r_near,
                                sop_surrogate** out, void* stream)
{
    if (!out) return fail(SOP_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!state || !aligned(state, 256)) return fail(SOP_ERR_INVALID_ARG, "state is NULL or not 256-byte aligned");
    if (state_bytes < sop::surr_state_bytes())
        return fail(SOP_ERR_WORKSPACE, "state too small: %zu < %zu bytes", state_bytes, sop::surr_state_bytes());
    if (!(r_near > 0.f) || !isfinite(r_near) || r_near > 2048.f)
        return fail(SOP_ERR_INVALID_ARG, "r_near = %g must be in (0, 2048]", (double)r_near);
    sop_status st = cuda_status(sop::surr_set_params((char*)state, params, seed, (cudaStream_t)stream),
                                "sop_surrogate_create");
    if (st != SOP_OK) return st;
    sop_surrogate* net = new (std::nothrow) sop_surrogate;
    if (!net) return fail(SOP_ERR_INVALID_ARG, "out of host memory for the handle");
    net->magic = kSurrMagic;
    net->state = (char*)state;
    net->r_near = r_near;
    *out = net;
    return SOP_OK;
}

sop_status sop_surrogate_destroy(sop_surrogate* net)
{
    if (!net) return SOP_OK;
    sop_status st = check_net(net);
    if (st != SOP_OK) return st;
    net->magic = 0;
    delete net;
    return SOP_OK;
}

sop_status sop_surrogate_set_params(sop_surrogate* net, const float* params, void* stream)
{
    sop_status st = check_net(net);
    if (st != SOP_OK) return st;
    if (!params) return fail(SOP_ERR_INVALID_ARG, "params is NULL");
    return cuda_status(sop::surr_set_params(net->state, params, 0, (cudaStream_t)stream), "sop_surrogate_set_params");
}

sop_status sop_surrogate_get_params(const sop_surrogate* net, float* params, void* stream)
{
    sop_status st = check_net(net);
    if (st != SOP_OK) return st;
    if (!params) return fail(SOP_ERR_INVALID_ARG, "params is NULL");
    return cuda_status(sop::surr_get_params(net->state, params, (cudaStream_t)stream), "sop_surrogate_get_params");
}

sop_status sop_surrogate_get_grad(const sop_surrogate* net, float* grad, void* stream)
{
    sop_status st = check_net(net);
    if (st != SOP_OK) return st;
    if (!grad) return fail(SOP_ERR_INVALID_ARG, "grad is NULL");
    return cuda_status(sop::surr_get_grad(net->state, grad, (cudaStream_t)stream), "sop_surrogate_get_grad");
}

sop_status sop_surrogate_file_write(const char* path, int32_t count, int32_t step, const float* params,
                                    const float* m, const float* v)
{
    if (!path || !params || !m || !v || count < 1) return fail(SOP_ERR_INVALID_ARG, "bad checkpoint arguments");
    FILE* f = fopen(path, "wb");
    if (!f) return fail(SOP_ERR_INVALID_ARG, "cannot open %s for writing", path);
    bool ok = fwrite("SOPSURR2", 1, 8, f) == 8 && fwrite(&count, 4, 1, f) == 1 && fwrite(&step, 4, 1, f) == 1 &&
              fwrite(params, 4, (size_t)count, f) == (size_t)count && fwrite(m, 4, (size_t)count, f) == (size_t)count &&
              fwrite(v, 4, (size_t)count, f) == (size_t)count;
    ok = (fclose(f) == 0) && ok;
    if (!ok) return fail(SOP_ERR_INVALID_ARG, "writing %s failed", path);
    return SOP_OK;
}

sop_status sop_surrogate_file_read(const char* path, int32_t count, int32_t* step, float* params, float* m, float* v)
{
    if (!path || !step || !params || !m || !v || count < 1) return fail(SOP_ERR_INVALID_ARG, "bad checkpoint arguments");
    FILE* f = fopen(path, "rb");
    if (!f) return fail(SOP_ERR_INVALID_ARG, "cannot open %s", path);
    char magic[8];
    int32_t n = 0, st = 0;
    bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, "SOPSURR2", 8) == 0 && fread(&n, 4, 1, f) == 1 &&
              fread(&st, 4, 1, f) == 1;
    if (ok && n != count) {
        fclose(f);
        return fail(SOP_ERR_INVALID_ARG, "%s holds %d parameters, expected %d", path, n, count);
    }
    ok = ok && fread(params, 4, (size_t)count, f) == (size_t)count && fread(m, 4, (size_t)count, f) == (size_t)count &&
         fread(v, 4, (size_t)count, f) == (size_t)count;
    char extra;
    ok = ok && fread(&extra, 1, 1, f) == 0;
    fclose(f);
    if (!ok) return fail(SOP_ERR_INVALID_ARG, "%s is not a surrogate checkpoint of this size (bad header or length)",
                         path);
    *step = st;
    return SOP_OK;
}

sop_status sop_surrogate_save(const sop_surrogate* net, const char* path, void* stream)
{
    sop_status st = check_net(net);
    if (st != SOP_OK) return st;
    if (!path) return fail(SOP_ERR_INVALID_ARG, "path is NULL");
    const int n = sop::surr_n_params();
    float* buf = (float*)malloc(sizeof(float) * 3 * (size_t)n);
    if (!buf) return fail(SOP_ERR_INVALID_ARG, "out of host memory");
    int32_t step = 0;
    st = cuda_status(sop::surr_state_io(net->state, buf, buf + n, buf + 2 * n, &step, false, (cudaStream_t)stream),
                     "sop_surrogate_save");
    if (st == SOP_OK) st = sop_surrogate_file_write(path, n, step, buf, buf + n, buf + 2 * n);
    free(buf);
    return st;
}

sop_status sop_surrogate_load(sop_surrogate* net, const char* path, void* stream)
{
    sop_status st = check_net(net);
    if (st != SOP_OK) return st;
    const int n = sop::surr_n_params();
    float* buf = (float*)malloc(sizeof(float) * 3 * (size_t)n);
    if (!buf) return fail(SOP_ERR_INVALID_ARG, "out of host memory");
    int32_t step = 0;
    st = sop_surrogate_file_read(path, n, &step, buf, buf + n, buf + 2 * n);
    if (st == SOP_OK)
        st = cuda_status(sop::surr_state_io(net->state, buf, buf + n, buf + 2 * n, &step, true, (cudaStream_t)stream),
                         "sop_surrogate_load");
    free(buf);
    return st;
}

size_t sop_surrogate_workspace_bytes(int64_t n_gauss, int32_t P, int32_t R)
{
    if (n_gauss < 1 || P < 1 || R < 2 || R > 64) return 0;
    const size_t a = surr_run_layout(n_gauss, P, R).total, b = sop::surr_train_ws_bytes();
    return a > b ? a : b;
}

size_t sop_surrogate_train_workspace_bytes(void) { return sop::surr_train_ws_bytes(); }

sop_status sop_surrogate_features(const sop_surrogate* net, const sop_gaussians* g, const float* probe_pos,
                                  int32_t P, int32_t R, const sop_bake_params* params, float* feats,
                                  int32_t* near_list, void* ws, size_t ws_bytes, void* stream)
{
    sop_status st = check_net(net);
    if (st != SOP_OK) return st;
    if ((st = check_gauss(g)) != SOP_OK || (st = check_bake_args(g, params)) != SOP_OK) return st;
    if (!probe_pos || !feats) return fail(SOP_ERR_INVALID_ARG, "probe_pos / feats is NULL");
    if (P < 1 || R < 2 || R > 64) return fail(SOP_ERR_INVALID_ARG, "P = %d, R = %d invalid", P, R);
    const SurrRunLayout L = surr_run_layout(g->n, P, R);
    if ((st = check_ws(ws, ws_bytes, L.total)) != SOP_OK) return st;
    return surr_feats_into(net, g, probe_pos, P, R, params, feats, near_list, (char*)ws, L, (cudaStream_t)stream,
                           "sop_surrogate_features");
}

sop_status sop_surrogate_train(sop_surrogate* net, const float* feats, const int32_t* probe_ids, int32_t batch,
                               const sop_atlas* targets, int32_t steps, float lr, uint64_t seed, float* out_loss,
                               void* ws, size_t ws_bytes, void* stream)
{
    sop_status st = check_net(net);
    if (st != SOP_OK) return st;
    if ((st = check_atlas(targets, true)) != SOP_OK) return st;
    if (!feats) return fail(SOP_ERR_INVALID_ARG, "feats is NULL");
    if (batch < 1 || batch > kMaxBatch) return fail(SOP_ERR_INVALID_ARG, "batch = %d outside [1, %d]", batch, kMaxBatch);
    if (steps < 0) return fail(SOP_ERR_INVALID_ARG, "steps = %d < 0", steps);
    if (!(lr > 0.f) || !isfinite(lr)) return fail(SOP_ERR_INVALID_ARG, "lr must be finite and > 0");
    if ((st = check_ws(ws, ws_bytes, sop::surr_train_ws_bytes())) != SOP_OK) return st;
    return cuda_status(sop::surr_train_steps(net->state, feats, probe_ids, batch, targets->P, *targets, steps, lr, seed,
                                             out_loss, (char*)ws, (cudaStream_t)stream),
                       "sop_surrogate_train");
}

sop_status sop_surrogate_predict(const sop_surrogate* net, const float* feats, const int32_t* probe_ids, int32_t B,
                                 const sop_atlas* out, void* stream)
{
    sop_status st = check_net(net);
    if (st != SOP_OK) return st;
    if ((st = check_atlas(out, true)) != SOP_OK) return st;
    if (!feats) return fail(SOP_ERR_INVALID_ARG, "feats is NULL");
    if (B < 0 || (!probe_ids && B > out->P)) return fail(SOP_ERR_INVALID_ARG, "B = %d invalid", B);
    cudaStream_t s = (cudaStream_t)stream;
    st = cuda_status(sop::surr_infer(net->state, feats, probe_ids, B, out->P, *out, s), "sop_surrogate_predict");
    if (st != SOP_OK || probe_ids || B != out->P) return st;
    return cuda_status(sop::launch_gutter_fill(*out, s), "sop_surrogate_predict (border)");
}

sop_status sop_surrogate_infer(const sop_surrogate* net, const sop_gaussians* g, const sop_atlas* out,
                               const sop_bake_params* params, float spot_frac, float tau, uint64_t seed,
                               float* out_spot_err, int32_t* out_fell_back, void* ws, size_t ws_bytes, void* stream)
{
    sop_status st = check_net(net);
    if (st != SOP_OK) return st;
    if ((st = check_gauss(g)) != SOP_OK || (st = check_bake_args(g, params)) != SOP_OK) return st;
    if ((st = check_atlas(out, true)) != SOP_OK) return st;
    if (!(spot_frac > 0.f && spot_frac <= 1.f)) return fail(SOP_ERR_INVALID_ARG, "spot_frac must be in (0, 1]");
    if (!(tau >= 0.f) || !isfinite(tau)) return fail(SOP_ERR_INVALID_ARG, "tau must be finite and >= 0");
    if (!out_fell_back) return fail(SOP_ERR_INVALID_ARG, "out_fell_back is NULL");
    const int32_t P = out->P, R = out->R;
    const SurrRunLayout L = surr_run_layout(g->n, P, R);
    if ((st = check_ws(ws, ws_bytes, L.total)) != SOP_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    char* w = (char*)ws;
    float* feats = (float*)(w + L.feats);
    const int32_t n_spot = std::max(1, std::min(P, (int32_t)ceil((double)spot_frac * P)));
    int32_t* ids = (int32_t*)(w + L.spot_ids);
    float* pos = (float*)(w + L.spot_pos);
    sop_atlas spot = *out;
    spot.rgbo = w + L.spot_rgbo;
    spot.depth = out->depth ? w + L.spot_depth : nullptr;
    spot.P = n_spot;
    spot.probe_pos = pos;
    spot.probe_nrm = nullptr;
    // the Gaussian records, which both branches read
    if ((st = cuda_status(sop::launch_bake_prep(*g, params->alpha_min, L.B, w + L.bake, s),
                          "sop_surrogate_infer (records)")) != SOP_OK)
        return st;
    std::unique_lock<std::mutex> lock(g_side_mu);
    SideStream* side = side_stream();
    if (!side) lock.unlock();
    cudaStream_t b = side ? side->s : s;
    if (side && (st = cuda_status(cudaEventRecord(side->fork, s) == cudaSuccess
                                      ? cudaStreamWaitEvent(b, side->fork, 0)
                                      : cudaGetLastError(),
                                  "sop_surrogate_infer (fork)")) != SOP_OK)
        return st;
    // branch b: the binning grid, then the spot check's sample traced into
    // the workspace's atlas
    st = cuda_status(sop::launch_bake_grid(*g, L.B, w + L.bake, b), "sop_surrogate_infer (binning)");
    if (st == SOP_OK) st = cuda_status(sop::launch_bake_fill(*g, L.B, w + L.bake, b), "sop_surrogate_infer (binning)");
    if (st == SOP_OK)
        st = cuda_status(sop::launch_spot_pick(seed, P, n_spot, out->probe_pos, ids, pos, b),
                         "sop_surrogate_infer (sample)");
    if (st == SOP_OK)
        st = cuda_status(sop::launch_bake_trace(spot, *params, L.B, w + L.bake, b), "sop_surrogate_infer (spot bake)");
    // branch s: features and the prediction of every probe
    if (st == SOP_OK) {
        sop::SurrStreams ss{side ? side->far : nullptr, side ? side->fork : nullptr, side ? side->list : nullptr,
                            side ? side->far_done : nullptr};
        st = cuda_status(sop::surr_features(*g, out->probe_pos, P, R, net->r_near, params->alpha_min,
                                            params->alpha_max, w + L.bake + L.B.rec, feats, nullptr, w + L.feat, s,
                                            side ? &ss : nullptr),
                         "sop_surrogate_infer (features)");
    }
    if (st == SOP_OK)
        st = cuda_status(sop::surr_infer(net->state, feats, nullptr, P, P, *out, s), "sop_surrogate_infer (network)");
    if (st == SOP_OK) st = cuda_status(sop::launch_gutter_fill(*out, s), "sop_surrogate_infer (border)");
    // join (also after a failed launch, so that nothing of b outlives the call)
    if (side) {
        const sop_status sj = cuda_status(cudaEventRecord(side->join, b) == cudaSuccess
                                              ? cudaStreamWaitEvent(s, side->join, 0)
                                              : cudaGetLastError(),
                                          "sop_surrogate_infer (join)");
        lock.unlock();
        if (st == SOP_OK) st = sj;
    }
    if (st != SOP_OK) return st;
    float* sums = (float*)(w + L.sums);
    if ((st = cuda_status(sop::launch_atlas_compare(spot, nullptr, *out, ids, n_spot, sums, s),
                          "sop_surrogate_infer (compare)")) != SOP_OK)
        return st;
    if ((st = cuda_status(sop::launch_spot_decide(sums, 1.f / ((float)n_spot * R * R), tau, out_spot_err,
                                                  out_fell_back, s),
                          "sop_surrogate_infer (decision)")) != SOP_OK)
        return st;
    // fallback: every probe traced, only when the device decided so
    if ((st = cuda_status(sop::launch_bake_trace(*out, *params, L.B, w + L.bake, s, out_fell_back),
                          "sop_surrogate_infer (fallback bake)")) != SOP_OK)
        return st;
    return cuda_status(sop::launch_atlas_copy(spot, nullptr, *out, ids, n_spot, s), "sop_surrogate_infer (spot copy)");
}

sop_status sop_atlas_compare(const sop_atlas* a, const int32_t* a_probes, const sop_atlas* b, const int32_t* b_probes,
                             int32_t n, float* out, void* stream)
{
    sop_status st = check_atlas(a, false);
    if (st != SOP_OK) return st;
    if ((st = check_atlas(b, false)) != SOP_OK) return st;
    if (a->R != b->R) return fail(SOP_ERR_INVALID_ARG, "atlases of different R");
    if (n < 0 || !out) return fail(SOP_ERR_INVALID_ARG, "n < 0 or out is NULL");
    return cuda_status(sop::launch_atlas_compare(*a, a_probes, *b, b_probes, n, out, (cudaStream_t)stream),
                       "sop_atlas_compare");
}

sop_status sop_atlas_copy(const sop_atlas* src, const int32_t* src_probes, const sop_atlas* dst,
                          const int32_t* dst_probes, int32_t n, void* stream)
{
    sop_status st = check_atlas(src, false);
    if (st != SOP_OK) return st;
    if ((st = check_atlas(dst, false)) != SOP_OK) return st;
    if (src->R != dst->R || src->rgbo_dtype != dst->rgbo_dtype ||
        ((src->depth && dst->depth) && src->depth_dtype != dst->depth_dtype))
        return fail(SOP_ERR_INVALID_ARG, "atlases differ in R or dtype");
    if (n < 0) return fail(SOP_ERR_INVALID_ARG, "n < 0");
    return cuda_status(sop::launch_atlas_copy(*src, src_probes, *dst, dst_probes, n, (cudaStream_t)stream),
                       "sop_atlas_copy");
}

// ---- deferred front end ------------------------------------------------------

size_t sop_trace_workspace_bytes(int64_t n_gauss)
{
    if (n_gauss < 0) return 0;
    return sop::bake_layout(n_gauss, 0).total;
}

sop_status sop_trace_gbuffer(const sop_gaussians* g, const sop_materials* m, const float* origins,
                             int32_t n_origins, const float* dirs, int64_t n_dirs, const sop_bake_params* params,
                             float* out, void* ws, size_t ws_bytes, void* stream)
{
    sop_status st = check_bake_args(g, params);
    if (st != SOP_OK) return st;
    if (!m || (g->n > 0 && (!m->albedo || !m->rough || !m->metal)))
        return fail(SOP_ERR_INVALID_ARG, "materials NULL");
    if (n_origins < 1 || !origins) return fail(SOP_ERR_INVALID_ARG, "need at least one origin");
    if (n_dirs < 1 || n_dirs > (int64_t)INT32_MAX || !dirs || !aligned(dirs, 16))
        return fail(SOP_ERR_INVALID_ARG, "dirs: NULL, not 16-byte aligned, or n_dirs outside [1, 2^31)");
    if ((int64_t)n_origins * n_dirs > ((int64_t)1 << 36))
        return fail(SOP_ERR_INVALID_ARG, "n_origins * n_dirs exceeds 2^36 rays");
    if (!out || !aligned(out, 16)) return fail(SOP_ERR_INVALID_ARG, "out NULL or not 16-byte aligned");
    sop::BakeLayout L;
    if ((st = bake_fit(g->n, params->grid_density, ws, ws_bytes, L)) != SOP_OK) return st;
    return cuda_status(sop::launch_trace_gbuffer(*g, m->albedo, m->rough, m->metal, origins, n_origins, dirs, n_dirs,
                                                 *params, L, (char*)ws, out, (cudaStream_t)stream),
                       "sop_trace_gbuffer");
}

sop_status sop_pinhole_dirs(int32_t W, int32_t H, const float* eye, const float* target, const float* up,
                            float fov_y_deg, float* out, void* stream)
{
    if (W < 1 || H < 1 || (int64_t)W * H > (int64_t)INT32_MAX)
        return fail(SOP_ERR_INVALID_ARG, "image %d x %d invalid", W, H);
    if (!eye || !target || !up) return fail(SOP_ERR_INVALID_ARG, "eye, target or up is NULL");
    if (!(fov_y_deg > 0.f && fov_y_deg < 180.f)) return fail(SOP_ERR_INVALID_ARG, "fov_y outside (0, 180)");
    double f2 = 0.0, u2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        if (!isfinite(eye[a]) || !isfinite(target[a]) || !isfinite(up[a]))
            return fail(SOP_ERR_INVALID_ARG, "camera not finite");
        f2 += ((double)target[a] - eye[a]) * ((double)target[a] - eye[a]);
        u2 += (double)up[a] * up[a];
    }
    if (!(f2 > 0.0) || !(u2 > 0.0)) return fail(SOP_ERR_INVALID_ARG, "eye == target or up == 0");
    if (!out || !aligned(out, 16)) return fail(SOP_ERR_INVALID_ARG, "out NULL or not 16-byte aligned");
    return cuda_status(sop::launch_pinhole_dirs(W, H, eye, target, up, fov_y_deg, out, (cudaStream_t)stream),
                       "sop_pinhole_dirs");
}

sop_status sop_panorama_dirs(int32_t W, int32_t H, float* out, void* stream)
{
    if (W < 1 || H < 1 || (int64_t)W * H > (int64_t)INT32_MAX)
        return fail(SOP_ERR_INVALID_ARG, "panorama %d x %d invalid", W, H);
    if (!out || !aligned(out, 16)) return fail(SOP_ERR_INVALID_ARG, "out NULL or not 16-byte aligned");
    return cuda_status(sop::launch_panorama_dirs(W, H, out, (cudaStream_t)stream), "sop_panorama_dirs");
}

size_t sop_gbuffer_points_workspace_bytes(int64_t n_pix)
{
    if (n_pix < 0 || n_pix > (int64_t)INT32_MAX) return 0;
    return sop::points_ws_bytes(n_pix);
}

sop_status sop_gbuffer_points(const float* gbuf, const float* front, int64_t n_pix, const float* origin,
                              const float* dirs, float w_min, int64_t* out_pix, float* out_x, float* out_n,
                              float* out_wo, float* out_albedo, float* out_rough, float* out_metal,
                              int64_t* out_count, void* ws, size_t ws_bytes, void* stream)
{
    if (n_pix < 0 || n_pix > (int64_t)INT32_MAX) return fail(SOP_ERR_INVALID_ARG, "n_pix out of range");
    if (!out_count) return fail(SOP_ERR_INVALID_ARG, "out_count is NULL");
    if (!origin) return fail(SOP_ERR_INVALID_ARG, "origin is NULL");
    if (!(w_min > 0.f) || !isfinite(w_min)) return fail(SOP_ERR_INVALID_ARG, "w_min must be finite and > 0");
    if (n_pix > 0) {
        if (!gbuf || !aligned(gbuf, 16) || !dirs || !aligned(dirs, 16) || (front && !aligned(front, 16)))
            return fail(SOP_ERR_INVALID_ARG, "gbuf, front or dirs NULL or not 16-byte aligned");
        if (!out_pix || !out_x || !out_n || !out_wo || !out_albedo || !out_rough || !out_metal)
            return fail(SOP_ERR_INVALID_ARG, "an output array is NULL");
    }
    sop_status st = check_ws(ws, ws_bytes, sop::points_ws_bytes(n_pix));
    if (st != SOP_OK) return st;
    return cuda_status(sop::launch_gbuffer_points(gbuf, front, n_pix, origin, dirs, w_min, out_pix, out_x, out_n,
                                                  out_wo, out_albedo, out_rough, out_metal, out_count, (char*)ws,
                                                  (cudaStream_t)stream),
                       "sop_gbuffer_points");
}

sop_status sop_depth_composite(const float* scene_gbuf, const float* obj_gbuf, int64_t n_pix, const int64_t* sc_pix,
                               const float* shadow, int64_t n_sc, const int64_t* obj_pix, const float* obj_rgb,
                               int64_t n_obj, float* out, void* stream)
{
    if (n_pix < 0 || n_sc < 0 || n_obj < 0 || n_sc > n_pix || n_obj > n_pix)
        return fail(SOP_ERR_INVALID_ARG, "sizes out of range");
    if (n_pix > 0 && (!scene_gbuf || !aligned(scene_gbuf, 16) || !out))
        return fail(SOP_ERR_INVALID_ARG, "scene_gbuf or out NULL (or scene_gbuf not 16-byte aligned)");
    if (n_sc > 0 && (!sc_pix || !shadow)) return fail(SOP_ERR_INVALID_ARG, "sc_pix or shadow NULL");
    if (n_obj > 0 && (!obj_pix || !obj_rgb || !obj_gbuf || !aligned(obj_gbuf, 16)))
        return fail(SOP_ERR_INVALID_ARG, "obj_pix, obj_rgb or obj_gbuf NULL (or obj_gbuf not 16-byte aligned)");
    return cuda_status(sop::launch_depth_composite(scene_gbuf, obj_gbuf, n_pix, sc_pix, shadow, n_sc, obj_pix,
                                                   obj_rgb, n_obj, out, (cudaStream_t)stream),
                       "sop_depth_composite");
}

size_t sop_place_probes_workspace_bytes(int64_t n_points)
{
    if (n_points < 1 || n_points > (int64_t)INT32_MAX) return 0;
    return sop::fps_ws_bytes(n_points);
}

sop_status sop_place_probes(const float* pts, const float* nrm, int64_t n_points, int32_t k, int64_t start,
                            float offset, int64_t* out_idx, float* out_pos, void* ws, size_t ws_bytes, void* stream)
{
    if (n_points < 1 || n_points > (int64_t)INT32_MAX) return fail(SOP_ERR_INVALID_ARG, "n_points out of range");
    if (k < 1 || (int64_t)k > n_points) return fail(SOP_ERR_INVALID_ARG, "k = %d outside [1, n_points]", k);
    if (start < 0 || start >= n_points) return fail(SOP_ERR_INVALID_ARG, "start outside [0, n_points)");
    if (!pts || !out_idx) return fail(SOP_ERR_INVALID_ARG, "pts or out_idx is NULL");
    if (!isfinite(offset)) return fail(SOP_ERR_INVALID_ARG, "offset must be finite");
    sop_status st = check_ws(ws, ws_bytes, sop::fps_ws_bytes(n_points));
    if (st != SOP_OK) return st;
    return cuda_status(sop::launch_fps(pts, nrm, n_points, k, start, offset, out_idx, out_pos, (char*)ws,
                                       (cudaStream_t)stream),
                       "sop_place_probes");
}

}  // extern "C"
