// Host-side internal interface between the C ABI layer (sop_api.cu) and the
// kernel translation units. Not installed; not part of the ABI.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "sop.h"

namespace sop {

struct ProbeGrid;
struct GaussGrid;

// ---- query ----------------------------------------------------------------
struct QueryLayout {
    size_t grid_hdr, cell_start, cell_cnt, entries, env4, envq, quads, dirs, idx, w, perm, bucket, genv4, total;
    int32_t cells_cap, g_axis;
};
QueryLayout query_layout(int32_t P, int64_t M, int32_t K, int32_t S, int32_t He, int32_t We, int32_t R,
                         int32_t rgbo_dtype);

struct QueryArgs {
    const float *x, *n, *wo, *albedo, *rough, *metal;
    int64_t M;
    const void* rgbo;
    int32_t rgbo_dtype;
    int32_t P, R;
    const float* probe_pos;
    const float* env;
    int32_t He, We;
    const float* dirs_local;
    int32_t K, S, mode, env_layout, dir_world;
    float specular;
    uint64_t snap_key;
    uint64_t r2_key;  // fixed-radius search: keys above it are not neighbours (UINT64_MAX: no radius)
    float* out;
    int32_t* out_idx;
    float* out_w;
    // upstream gradient and gradient outputs (backward only)
    const float* grad_out;
    float *g_albedo, *g_rough, *g_metal, *g_normal, *g_env, *g_atlas;
};

// Enqueue the probe grid, nearest-probe search + weights, environment and
// direction tables (shared by forward and backward).
cudaError_t launch_query_prep(const QueryArgs& a, const QueryLayout& L, char* ws, cudaStream_t s);
cudaError_t launch_shade(const QueryArgs& a, const QueryLayout& L, char* ws, cudaStream_t s);
cudaError_t launch_adjoint(const QueryArgs& a, const QueryLayout& L, char* ws, cudaStream_t s);
cudaError_t launch_hammersley(int32_t S, float* out3, cudaStream_t s);
cudaError_t launch_read_probe(const void* buf, size_t bytes, int32_t reps, float* sink, cudaStream_t s);
cudaError_t launch_env_to_oct(const float* env, int32_t He, int32_t We, float* out, int32_t H, cudaStream_t s);
size_t importance_ws_bytes(int32_t H);
cudaError_t launch_importance_dirs(const float* env, int32_t H, int32_t S, float* out, char* ws, cudaStream_t s);

// SOP texture optimisation pieces (optimize.cu)
cudaError_t launch_l1_grad(const float* C, const float* Ct, int64_t n, float* grad, float* loss_sum, cudaStream_t s);
cudaError_t launch_adam_l1(float* p, const float* g, float* m, float* v, int64_t n, const sop_adam_params& a,
                           cudaStream_t s);

// the uniform grid of N sites (quantised positions and indices) that the
// site searches use, built in ws (sites_grid_bytes(N) bytes)
struct SitesGrid {
    const ProbeGrid* grid;
    const int32_t* cell_start;
    const int4* entries;
};
size_t sites_grid_bytes(int32_t N);
SitesGrid launch_sites_grid(const float* sites, int32_t N, char* ws, cudaStream_t s);

// allocation-free query (static device scratch, see query.cu)
size_t noalloc_scratch_bytes();
int64_t noalloc_chunk();
size_t noalloc_required_bytes(int32_t P, int32_t K, int32_t S);
cudaError_t launch_query_noalloc(const QueryArgs& a, cudaStream_t s);

// ---- atlas pack -------------------------------------------------------------
cudaError_t launch_atlas_pack(const float* rgb, int rgb_stride, const float* occ, int occ_stride, const float* depth,
                              const sop_atlas& atlas, cudaStream_t s);

// ---- bake -------------------------------------------------------------------
struct BakeLayout {
    size_t hdr, bbox, stats, rec, cell_start, cell_cnt, scan, dirs, ent, total;
    int64_t cells_cap, entries_cap;
};
// bytes per cell entry: quantised box and Gaussian index
constexpr size_t kBakeEntryBytes = 16;
// bake workspace layout for N Gaussians (independent of the atlas)
// density: grid cells per Gaussian (0: the default, 0.35)
BakeLayout bake_layout(int64_t N, int64_t entries_cap, float density = 0.f);
cudaError_t launch_bake_bin(const sop_gaussians& g, float alpha_min, const BakeLayout& L, char* ws, cudaStream_t s);
// launch_bake_bin in two parts: the Gaussian records (and the bounding box)
// and the binning grid built from them
cudaError_t launch_bake_prep(const sop_gaussians& g, float alpha_min, const BakeLayout& L, char* ws, cudaStream_t s);
cudaError_t launch_bake_grid(const sop_gaussians& g, const BakeLayout& L, char* ws, cudaStream_t s);
cudaError_t launch_bake_fill(const sop_gaussians& g, const BakeLayout& L, char* ws, cudaStream_t s);
// run_if: when not NULL, the launches do nothing unless *run_if != 0 (device)
// stats: the trace's counters, whose truncation bit goes to the status word
cudaError_t launch_gutter_fill(const sop_atlas& atlas, cudaStream_t s, const int32_t* run_if = nullptr,
                               const unsigned long long* stats = nullptr);
cudaError_t launch_bake_trace(const sop_atlas& atlas, const sop_bake_params& bp, const BakeLayout& L, char* ws,
                              cudaStream_t s, const int32_t* run_if = nullptr);

// ---- deferred front end (G-buffers, shading points, compositing) --------------
cudaError_t launch_trace_gbuffer(const sop_gaussians& g, const float* albedo, const float* rough, const float* metal,
                                 const float* origins, int32_t n_origins, const float* dirs, int64_t n_dirs,
                                 const sop_bake_params& bp, const BakeLayout& L, char* ws, float* out, cudaStream_t s);
cudaError_t launch_pinhole_dirs(int32_t W, int32_t H, const float* eye, const float* target, const float* up,
                                float fov_y_deg, float* out, cudaStream_t s);
cudaError_t launch_panorama_dirs(int32_t W, int32_t H, float* out, cudaStream_t s);
size_t points_ws_bytes(int64_t n_pix);
cudaError_t launch_gbuffer_points(const float* gbuf, const float* front, int64_t n, const float* origin,
                                  const float* dirs, float w_min, int64_t* pix, float* x, float* nrm, float* wo,
                                  float* albedo, float* rough, float* metal, int64_t* count, char* ws, cudaStream_t s);
cudaError_t launch_depth_composite(const float* scene_gbuf, const float* obj_gbuf, int64_t n, const int64_t* sc_pix,
                                   const float* shadow, int64_t n_sc, const int64_t* obj_pix, const float* obj_rgb,
                                   int64_t n_obj, float* out, cudaStream_t s);

// ---- automatic probe placement (FPS) ----------------------------------------------
size_t fps_ws_bytes(int64_t n);
cudaError_t launch_fps(const float* pts, const float* nrm, int64_t n, int32_t k, int64_t start, float offset,
                       int64_t* out_idx, float* out_pos, char* ws, cudaStream_t s);

// ---- learned bake surrogate ---------------------------------------------------
struct SurrState;
int surr_n_params();
int surr_n_features();
int surr_near_cap();
size_t surr_state_bytes();
// params NULL: He-uniform initial weights from `seed`; resets Adam
cudaError_t surr_set_params(char* state, const float* params, uint64_t seed, cudaStream_t s);
cudaError_t surr_get_params(const char* state, float* params, cudaStream_t s);
cudaError_t surr_get_grad(const char* state, float* grad, cudaStream_t s);
// host arrays <-> the state (master weights, Adam moments, step); synchronises
cudaError_t surr_state_io(char* state, float* master, float* m, float* v, int32_t* step, bool to_device,
                          cudaStream_t s);
struct SurrFeatLayout {
    size_t sites, tdirs, t0, fhdr, fmm, fctr, list, fbrick, facc, fcells, total;
};
// Streams of the features' two branches: the far field (grid, march) runs on
// `far`, after the event `fork` that the caller recorded on the main stream;
// `list` and `far_done` are recorded by surr_features (the near list done;
// the far march done, which the main stream then waits for).
struct SurrStreams {
    cudaStream_t far;
    cudaEvent_t fork, list, far_done;
};
SurrFeatLayout surr_feat_layout(int64_t N, int32_t P, int32_t R);
// features [P][R*R][18] of every texel; bake_rec: the Gaussian records of a
// binned bake workspace; list [P][near cap] or NULL
cudaError_t surr_features(const sop_gaussians& g, const float* probe_pos, int32_t P, int32_t R, float r_n,
                          float alpha_min, float alpha_max, const char* bake_rec, float* feats, int32_t* list,
                          char* ws, cudaStream_t s, const SurrStreams* ss = nullptr);
// `steps` Adam steps on B probes each (pid, or drawn from seed); ws holds
// surr_train_ws_bytes() (drawn ids, per-CTA gradient and loss sums)
size_t surr_train_ws_bytes();
cudaError_t surr_train_steps(char* state, const float* feats, const int32_t* pid, int32_t B, int32_t P,
                             const sop_atlas& tgt, int32_t steps, float lr, uint64_t seed, float* loss_out,
                             char* ws, cudaStream_t s);
cudaError_t surr_infer(const char* state, const float* feats, const int32_t* pid, int32_t B, int32_t P,
                       const sop_atlas& out, cudaStream_t s);
cudaError_t surr_loss_out(const char* state, float scale, float* out, cudaStream_t s);
cudaError_t launch_atlas_compare(const sop_atlas& a, const int32_t* ap, const sop_atlas& b, const int32_t* bp,
                                 int32_t n, float* out, cudaStream_t s);
cudaError_t launch_atlas_copy(const sop_atlas& src, const int32_t* sp, const sop_atlas& dst, const int32_t* dp,
                              int32_t n, cudaStream_t s);
cudaError_t launch_spot_pick(uint64_t seed, int32_t P, int32_t n, const float* probe_pos, int32_t* ids, float* pos,
                             cudaStream_t s);
cudaError_t launch_spot_decide(const float* sums, float inv_texels, float tau, float* err_out, int32_t* fell_back,
                               cudaStream_t s);

// ---- device status word (status.cu) -------------------------------------------
// Address of this device's status word (kernels atomicOr SOP_DEVSTAT_* bits
// into it), or NULL if it cannot be looked up; cached per device ordinal.
unsigned int* status_word();
// Synchronises s after reading (and, if clear, atomically clearing) the word.
cudaError_t status_take(uint32_t* host_out, bool clear, cudaStream_t s);
const char* status_bits_message(uint32_t bits);

inline size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

}  // namespace sop
