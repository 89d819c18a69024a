// SOP bake (Sec. 3.1.2 probe textures initialised by ray tracing; Sec. 3.2.2
// occlusion caching; compositing of Eq. 1; D/W depth of Sec. 3.1) for sm_103a.
//
// Every probe texel shoots one ray from the probe along the octahedral decode
// of the texel centre. A Gaussian's response along a ray is its maximum,
// alpha = min(alpha_max, o exp(-m^2/2)); responses with alpha >= alpha_min
// and t* > t_near are composited in increasing (t*, index) order.
//
// Design: the alpha_min cut-off bounds each Gaussian by a sphere of radius
// rho = s_max sqrt(2 ln(o / alpha_min)) (no point further away can reach
// alpha_min). The spheres are binned into a uniform grid (count, scan, fill).
// Each texel ray then walks the grid front to back (3D DDA). In each cell it
// keeps only hits whose t* lies inside the cell's t-interval, orders them by
// (t*, index) in a small local buffer (a cell with more hits than the buffer
// is rescanned past the last composited hit) and composites them. Cells
// partition the ray, so hits come out globally ordered and each once; the
// walk ends when the transmittance drops below t_stop. No per-ray hit lists.
//
// The hit evaluation avoids FP32 cancellation: the probe-to-centre offset is
// split exactly into hi + lo parts (two-sum), the closest-approach point is
// formed with an FMA, and m^2 is taken from the Mahalanobis norm of that
// small vector, so alpha carries ~1e-7 relative error even for far, thin
// Gaussians.
#include <stdlib.h>

#include "scan.cuh"
#include "sop_device.cuh"
#include "sop_internal.h"

namespace sop {

// Gaussian record: 5 float4 = 80 B.
//   r0 = (mu.xyz, rho)   rho < 0: never reaches alpha_min
//   r1..r3 = M = diag(1/s) R^T row-major (9) then opacity
//   r3.zw, r4.x = rgb; r4.yzw = half extents of the alpha_min ellipsoid's
//   axis-aligned box (used to bin the Gaussian into grid cells)
struct GRec {
    float4 r0, r1, r2, r3, r4;
};

constexpr float kMarginRel = 1e-4f;
constexpr int kMaxR = 64;

// Capacity of the binning grid: the grid gets about half of it, i.e.
// `density` cells per Gaussian when given (> 0), else 0.35 (a capacity of 70
// cells per 100 Gaussians).
constexpr int64_t kCellsPer100 = 70;
static int64_t cells_cap_for(int64_t N, float density)
{
    const int64_t c = density > 0.f ? (int64_t)(2.0 * (double)density * (double)N) : N * kCellsPer100 / 100;
    return c < 4096 ? 4096 : (c > (1 << 23) ? (1 << 23) : c);
}

// binning attempts of launch_bake_bin
constexpr int kBinAttempts = 3;

BakeLayout bake_layout(int64_t N, int64_t entries_cap, float density)
{
    BakeLayout L{};
    L.cells_cap = cells_cap_for(N, density);
    L.entries_cap = entries_cap > 0 ? entries_cap : 24 * N + 65536;
    size_t o = 0;
    L.hdr = o;        o = align256(o + sizeof(GaussGrid));
    L.bbox = o;       o = align256(o + 16 * sizeof(int32_t));
    L.stats = o;      o = align256(o + 8 * sizeof(unsigned long long));
    L.rec = o;        o = align256(o + sizeof(GRec) * (size_t)(N > 0 ? N : 1));
    L.cell_start = o; o = align256(o + sizeof(int32_t) * (size_t)(L.cells_cap + 1));
    L.cell_cnt = o;   o = align256(o + sizeof(int32_t) * (size_t)L.cells_cap);
    L.scan = o;       o = align256(o + sizeof(long long) * scan_scratch_count(L.cells_cap));
    L.dirs = o;       o = align256(o + sizeof(float4) * (size_t)kMaxR * kMaxR);
    L.ent = o;        o = align256(o + sizeof(uint4) * (size_t)L.entries_cap);
    L.total = o;
    return L;
}

// float <-> order-preserving int for atomic min/max of floats
__device__ __forceinline__ int32_t f2o(float f)
{
    int32_t i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float o2f(int32_t i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

__global__ void bbox_init_kernel(int32_t* bbox)
{
    if (threadIdx.x < 3) bbox[threadIdx.x] = f2o(FLT_MAX);
    else if (threadIdx.x < 6) bbox[threadIdx.x] = f2o(-FLT_MAX);
    else if (threadIdx.x < 8) bbox[threadIdx.x] = 0;  // [6]: binning status word
}

// Per-Gaussian record + bounding box of the (margin-expanded) spheres. A
// Gaussian with a non-finite parameter, a scale <= 0 or a zero quaternion is
// left out of the bake (rho < 0) and flagged in the device status word.
__global__ void gauss_prep_kernel(sop_gaussians g, float alpha_min, GRec* __restrict__ rec, int32_t* bbox,
                                  unsigned int* status)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
    if (i < g.n) {
        const float qw = g.quat[4 * i], qx = g.quat[4 * i + 1], qy = g.quat[4 * i + 2], qz = g.quat[4 * i + 3];
        const float qn = sqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
        const float w = qw / qn, x = qx / qn, y = qy / qn, z = qz / qn;
        // rotation matrix (columns = local axes in world space)
        const float R00 = 1.f - 2.f * (y * y + z * z), R01 = 2.f * (x * y - w * z), R02 = 2.f * (x * z + w * y);
        const float R10 = 2.f * (x * y + w * z), R11 = 1.f - 2.f * (x * x + z * z), R12 = 2.f * (y * z - w * x);
        const float R20 = 2.f * (x * z - w * y), R21 = 2.f * (y * z + w * x), R22 = 1.f - 2.f * (x * x + y * y);
        const float sx = g.scale[3 * i], sy = g.scale[3 * i + 1], sz = g.scale[3 * i + 2];
        const float ix = 1.f / sx, iy = 1.f / sy, iz = 1.f / sz;
        const float o = g.opacity[i];
        const float3 mu = load3(g.mean, i);
        const float c0 = g.rgb[3 * i], c1 = g.rgb[3 * i + 1], c2 = g.rgb[3 * i + 2];
        // a NaN anywhere makes the sum NaN; an Inf makes it Inf or NaN
        const bool ok = isfinite(mu.x + mu.y + mu.z + sx + sy + sz + qw + qx + qy + qz + o + c0 + c1 + c2) &&
                        sx > 0.f && sy > 0.f && sz > 0.f && qn > 0.f && isfinite(ix + iy + iz);
        if (!ok && status) atomicOr(status, SOP_DEVSTAT_NONFINITE);
        float rho = -1.f, ex = 0.f, ey = 0.f, ez = 0.f;
        if (ok && o >= alpha_min && o > 0.f) {
            // {x : o exp(-m^2(x)/2) >= alpha_min} is the ellipsoid m^2 <= kk^2
            const float kk = sqrtf(2.f * fmaxf(logf(o / alpha_min), 0.f));
            const float smax = fmaxf(sx, fmaxf(sy, sz));
            rho = smax * kk * (1.f + kMarginRel) + 1e-7f;
            // axis-aligned half extents: kk sqrt(Sigma_aa), Sigma = R diag(s^2) R^T
            const float sx2 = sx * sx, sy2 = sy * sy, sz2 = sz * sz;
            ex = kk * sqrtf(R00 * R00 * sx2 + R01 * R01 * sy2 + R02 * R02 * sz2) * (1.f + kMarginRel) + 1e-7f;
            ey = kk * sqrtf(R10 * R10 * sx2 + R11 * R11 * sy2 + R12 * R12 * sz2) * (1.f + kMarginRel) + 1e-7f;
            ez = kk * sqrtf(R20 * R20 * sx2 + R21 * R21 * sy2 + R22 * R22 * sz2) * (1.f + kMarginRel) + 1e-7f;
            ex = fminf(ex, rho);
            ey = fminf(ey, rho);
            ez = fminf(ez, rho);
        }
        GRec r;
        r.r0 = make_float4(mu.x, mu.y, mu.z, rho);
        // M = diag(1/s) R^T : row a = R[:, a] / s_a
        r.r1 = make_float4(R00 * ix, R10 * ix, R20 * ix, R01 * iy);
        r.r2 = make_float4(R11 * iy, R21 * iy, R02 * iz, R12 * iz);
        r.r3 = make_float4(R22 * iz, o, c0, c1);
        r.r4 = make_float4(c2, ex, ey, ez);
        rec[i] = r;
        if (rho >= 0.f) {
            lo[0] = mu.x - ex; lo[1] = mu.y - ey; lo[2] = mu.z - ez;
            hi[0] = mu.x + ex; hi[1] = mu.y + ey; hi[2] = mu.z + ez;
        }
    }
    // warp reduce then one atomic per warp
    for (int a = 0; a < 3; ++a) {
        for (int off = 16; off > 0; off >>= 1) {
            lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], off));
            hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], off));
        }
    }
    if ((threadIdx.x & 31) == 0) {
        for (int a = 0; a < 3; ++a) {
            if (lo[a] <= hi[a]) {
                atomicMin(&bbox[a], f2o(lo[a]));
                atomicMax(&bbox[3 + a], f2o(hi[a]));
            }
        }
    }
}

// Grid geometry from the bounding box: cubic cells, about cells_cap/2 of
// them over the box, never more than cells_cap. Binning attempt `level`
// (> 0: the previous attempt's cell lists did not fit the workspace) does
// nothing once an earlier attempt fitted.
__global__ void grid_setup_kernel(const int32_t* bbox, int64_t cells_cap, int32_t level, GaussGrid* grid,
                                  int32_t* cell_cnt)
{
    __shared__ GaussGrid G;
    if (level > 0 && grid->fits) return;
    if (threadIdx.x == 0) {
        float lo[3], hi[3], ext[3];
        bool empty = false;
        for (int a = 0; a < 3; ++a) {
            lo[a] = o2f(bbox[a]);
            hi[a] = o2f(bbox[3 + a]);
            if (!(lo[a] <= hi[a])) empty = true;
        }
        if (empty) {
            for (int a = 0; a < 3; ++a) { lo[a] = 0.f; hi[a] = 0.f; }
        }
        float emax = 0.f;
        for (int a = 0; a < 3; ++a) {
            // pad the box so boundary rounding never drops a sphere
            const float pad = 1e-5f * fmaxf(hi[a] - lo[a], 1e-3f) + 1e-6f;
            lo[a] -= pad;
            hi[a] += pad;
            ext[a] = hi[a] - lo[a];
            emax = fmaxf(emax, ext[a]);
        }
        // cell edge: volume / (cells_cap/2), clamped so that no axis needs
        // more than cbrt-balanced resolution
        const double vol = (double)ext[0] * ext[1] * ext[2];
        double h = cbrt(vol / (double)(cells_cap / 2));
        h = fmax(h, (double)emax / 1024.0);
        int64_t nc;
        int d[3];
        for (;;) {
            nc = 1;
            for (int a = 0; a < 3; ++a) {
                d[a] = (int)ceil(ext[a] / h);
                d[a] = d[a] < 1 ? 1 : d[a];
                nc *= d[a];
            }
            if (nc <= cells_cap) break;
            h *= 1.1;
        }
        for (int a = 0; a < 3; ++a) {
            G.origin[a] = lo[a];
            G.bmax[a] = hi[a];
            G.dims[a] = d[a];
        }
        G.h = (float)h;
        G.inv_h = (float)(1.0 / h);
        G.ncells = (int32_t)nc;
        G.n_entries = 0;
        G.fits = 0;
        G.level = level;
        *grid = G;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < G.ncells; c += blockDim.x) cell_cnt[c] = 0;
}

// A cell entry is the Gaussian's box as the walk tests it, in 16 bytes: the
// centre in 16-bit fixed point over the grid box (c = origin + q/65536 span),
// the half extents in fp16, rounded up and widened by the centre's
// quantisation error (so the box holds the alpha_min ellipsoid), and the
// Gaussian's index. Binning and the walk decode it with the same arithmetic.
__device__ __forceinline__ float qdecode(uint32_t q16, float span, float go)
{
    // q16 / 65536 exactly, from the bits of 1 + q16 / 65536
    return fmaf(__uint_as_float(0x3f800000u | (q16 << 7)) - 1.f, span, go);
}

__device__ __forceinline__ float hdecode(uint32_t h16)
{
    return __half2float(__ushort_as_half((unsigned short)h16));
}

__device__ __forceinline__ uint4 make_entry(const GaussGrid& G, float3 mu, float4 r4, int32_t gi)
{
    const float m[3] = {mu.x, mu.y, mu.z}, e[3] = {r4.y, r4.z, r4.w};
    uint32_t q[3], h[3];
    for (int a = 0; a < 3; ++a) {
        const float span = G.bmax[a] - G.origin[a];
        const float v = rintf((m[a] - G.origin[a]) / span * 65536.f);
        q[a] = (uint32_t)fminf(fmaxf(v, 0.f), 65535.f);
        const float c = qdecode(q[a], span, G.origin[a]);
        const float w = e[a] + fabsf(c - m[a]) + 1e-6f * (fabsf(m[a]) + span);
        h[a] = __half_as_ushort(__float2half_ru(w));
    }
    return make_uint4(q[0] | (q[1] << 16), q[2] | (h[0] << 16), h[1] | (h[2] << 16), (uint32_t)gi);
}

// Cells overlapped by the entry's box plus a margin. The margin is far
// larger than the rounding of the grid walk's cell boundaries and of the
// ray's entry into the box, so the cell in which the walk finds the box
// entry always lists the Gaussian.
__device__ __forceinline__ void cell_range(const GaussGrid& G, const uint4 en, int lo[3], int hi[3])
{
    float amax = 0.f;
    for (int a = 0; a < 3; ++a) amax = fmaxf(amax, fmaxf(fabsf(G.origin[a]), fabsf(G.bmax[a])));
    const float mg = 1e-3f * G.h + 16.f * FLT_EPSILON * amax;
    const float c[3] = {qdecode(en.x & 0xffffu, G.bmax[0] - G.origin[0], G.origin[0]),
                        qdecode(en.x >> 16, G.bmax[1] - G.origin[1], G.origin[1]),
                        qdecode(en.y & 0xffffu, G.bmax[2] - G.origin[2], G.origin[2])};
    const float e[3] = {hdecode(en.y >> 16) + mg, hdecode(en.z & 0xffffu) + mg, hdecode(en.z >> 16) + mg};
    for (int a = 0; a < 3; ++a) {
        lo[a] = min(max((int)floorf((c[a] - e[a] - G.origin[a]) * G.inv_h), 0), G.dims[a] - 1);
        hi[a] = min(max((int)floorf((c[a] + e[a] - G.origin[a]) * G.inv_h), 0), G.dims[a] - 1);
    }
}

__global__ void bin_count_kernel(int64_t N, const GRec* __restrict__ rec, const GaussGrid* __restrict__ gridp,
                                 int32_t* __restrict__ cell_cnt)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N || gridp->fits) return;
    const float4 r0 = rec[i].r0;
    if (r0.w < 0.f) return;
    const GaussGrid G = *gridp;
    int lo[3], hi[3];
    cell_range(G, make_entry(G, f3(r0.x, r0.y, r0.z), rec[i].r4, (int32_t)i), lo, hi);
    for (int z = lo[2]; z <= hi[2]; ++z)
        for (int y = lo[1]; y <= hi[1]; ++y)
            for (int x = lo[0]; x <= hi[0]; ++x) atomicAdd(&cell_cnt[(z * G.dims[1] + y) * G.dims[0] + x], 1);
}

// Exclusive scan of the cell counts in one CTA; total into grid->n_entries,
// and grid->fits = 1 when the total fits the entry capacity (an attempt
// after the first that fits marks the status word: the grid was coarsened).
// After the count pass of a binning attempt: whether the cell lists fit the
// entry capacity (the fill pass and later attempts read it).
struct BinScanFinal {
    GaussGrid* grid;
    int64_t entries_cap;
    unsigned int* status;
    __device__ void operator()(long long tot) const
    {
        const bool fit = tot <= entries_cap && tot < INT32_MAX;
        grid->n_entries = (int32_t)(tot < INT32_MAX ? tot : INT32_MAX);
        grid->fits = fit ? 1 : 0;
        if (fit && grid->level > 0 && status) atomicOr(status, SOP_DEVSTAT_GRID_COARSENED);
    }
};

__global__ void bin_fill_kernel(int64_t N, const GRec* __restrict__ rec, const GaussGrid* __restrict__ gridp,
                                const int32_t* __restrict__ cell_start, int32_t* __restrict__ cell_cnt,
                                uint4* __restrict__ ent)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N || !gridp->fits) return;
    const float4 r0 = rec[i].r0;
    if (r0.w < 0.f) return;
    const GaussGrid G = *gridp;
    const uint4 en = make_entry(G, f3(r0.x, r0.y, r0.z), rec[i].r4, (int32_t)i);
    int lo[3], hi[3];
    cell_range(G, en, lo, hi);
    for (int z = lo[2]; z <= hi[2]; ++z)
        for (int y = lo[1]; y <= hi[1]; ++y)
            for (int x = lo[0]; x <= hi[0]; ++x) {
                const int c = (z * G.dims[1] + y) * G.dims[0] + x;
                const int pos = cell_start[c] + atomicAdd(&cell_cnt[c], 1);
                ent[pos] = en;
            }
}

// Texel-centre directions, computed in fp64 and rounded once.
__global__ void texel_dirs_kernel(int R, float4* __restrict__ dirs)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= R * R) return;
    double d[3];
    oct_decode_centre_f64(R, t % R, t / R, d);
    dirs[t] = make_float4((float)d[0], (float)d[1], (float)d[2], 0.f);
}

// error-free a - b = hi + lo
__device__ __forceinline__ void two_diff(float a, float b, float& hi, float& lo)
{
    hi = a - b;
    const float bv = a - hi;
    const float av = hi + bv;
    lo = (a - av) + (bv - b);
}

struct TraceK {
    const GRec* rec;
    const GaussGrid* grid;
    const int32_t* cell_start;
    const uint4* ent;  // cell entries (quantised box and Gaussian index)
    const float4* dirs;
    const float* probe_pos;
    int32_t P, R;
    float t_near, alpha_min, alpha_max, t_stop;
    void* rgbo;       // atlas [P][R+2][R+2] in rgbo_dtype (interior written here)
    void* depth;      // atlas depth plane or NULL
    int32_t rgbo_dtype, depth_dtype;
    float inv_depth_scale;
    // stats[0]: next texel ray to trace; [1]: exact evaluations; [2]:
    // composited hits; [3] bit 0: a cell window could not be split; [4]: cell
    // entries tested
    unsigned long long* stats;
    // waiting hits plus candidates queued since the last composite that
    // make the walk stop to composite
    int32_t composite_at;
    // rays are origin p (of P) along direction t (of n_dirs): ray = p n_dirs + t
    int64_t n_dirs;
    // rays a warp takes from the counter at a time
    int32_t batch;
    // G-buffer mode (multi-target rendering): the Gaussians' orientation,
    // scales and materials, and the output [rays][4] float4
    const float *quat, *scale, *albedo, *rough, *metal;
    float4* gbuf;
    // device status word (SOP_DEVSTAT_* bits) or NULL
    unsigned int* status;
    // when not NULL, the launch does nothing unless *run_if != 0 (a decision
    // taken on the device, e.g. the surrogate's fallback)
    const int32_t* run_if;
};

// what a traced ray writes: the probe atlas texel (O, L_in, depth) or the
// G-buffer entry (C, W, N, D, A, R, M)
enum { kTraceAtlas = 0, kTraceGbuf = 1 };

constexpr int kWarpsPerCta = 8;
constexpr int kHitCap = 256;  // per-warp hit buffer (shared memory)
// the bitonic sort pads a buffer to the next power of two within kHitCap
static_assert((kHitCap & (kHitCap - 1)) == 0 && kHitCap >= 64, "kHitCap must be a power of two >= 64");

// order-preserving 64-bit key of (t*, Gaussian index)
__device__ __forceinline__ uint64_t hit_key(float t, int32_t g)
{
    const uint32_t o = (uint32_t)f2o(t) ^ 0x80000000u;
    return ((uint64_t)o << 32) | (uint32_t)g;
}

// Warp-uniform state of one texel ray, plus each lane's partial sums of the
// composited terms (reduced once per ray).
struct RayAcc {
    float T, L0, L1, L2, Dacc, Wacc;
    float N0, N1, N2, A0, A1, A2, Rg, Mg;  // G-buffer mode only
    int n_eval, n_comp, n_test;
    bool done;
};

// Unit normal of a Gaussian read as a surfel: its local axis of smallest
// scale (the first of equal ones), a column of R(q).
__device__ __forceinline__ float3 surfel_normal(const TraceK& k, const int32_t g)
{
    const float sx = __ldg(k.scale + 3 * g), sy = __ldg(k.scale + 3 * g + 1), sz = __ldg(k.scale + 3 * g + 2);
    int am = 0;
    float sm = sx;
    if (sy < sm) {
        am = 1;
        sm = sy;
    }
    if (sz < sm) am = 2;
    const float qw = __ldg(k.quat + 4 * g), qx = __ldg(k.quat + 4 * g + 1), qy = __ldg(k.quat + 4 * g + 2),
                qz = __ldg(k.quat + 4 * g + 3);
    const float qn = sqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
    const float w = qw / qn, x = qx / qn, y = qy / qn, z = qz / qn;
    if (am == 0) return f3(1.f - 2.f * (y * y + z * z), 2.f * (x * y + w * z), 2.f * (x * z - w * y));
    if (am == 1) return f3(2.f * (x * y - w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z + w * x));
    return f3(2.f * (x * z + w * y), 2.f * (y * z - w * x), 1.f - 2.f * (x * x + y * y));
}

// Exact responses of up to 32 queued candidates (one per lane). Hits are
// appended to the warp's buffer key/alp[0, n); n keeps counting past
// kHitCap, but nothing is written there.
__device__ __forceinline__ void eval_batch(const TraceK& k, const float3 o, const float3 d, int32_t* que, int& qn,
                                           uint64_t* key, float* alp, int& n, const int lane, RayAcc& acc)
{
    {
        const int take = qn < 32 ? qn : 32;
        acc.n_eval += take;
        bool hit = false;
        float ts = 0.f, al = 0.f;
        int32_t gi = 0;
        if (lane < take) {
            gi = que[lane];
            const GRec* gr = k.rec + gi;
            const float4 r0 = __ldg(&gr->r0), r1 = __ldg(&gr->r1), r2 = __ldg(&gr->r2), r3 = __ldg(&gr->r3);
            float hx, lx, hy, ly, hz, lz;
            two_diff(o.x, r0.x, hx, lx);
            two_diff(o.y, r0.y, hy, ly);
            two_diff(o.z, r0.z, hz, lz);
            const float u0 = fmaf(r1.x, hx, fmaf(r1.y, hy, r1.z * hz));
            const float u1 = fmaf(r1.w, hx, fmaf(r2.x, hy, r2.y * hz));
            const float u2 = fmaf(r2.z, hx, fmaf(r2.w, hy, r3.x * hz));
            const float w0 = fmaf(r1.x, d.x, fmaf(r1.y, d.y, r1.z * d.z));
            const float w1 = fmaf(r1.w, d.x, fmaf(r2.x, d.y, r2.y * d.z));
            const float w2 = fmaf(r2.z, d.x, fmaf(r2.w, d.y, r3.x * d.z));
            const float A = fmaf(w0, w0, fmaf(w1, w1, w2 * w2));
            const float B = fmaf(w0, u0, fmaf(w1, u1, w2 * u2));
            ts = -B / A;
            if (ts > k.t_near) {
                const float ex = fmaf(ts, d.x, hx) + lx, ey = fmaf(ts, d.y, hy) + ly, ez = fmaf(ts, d.z, hz) + lz;
                const float v0 = fmaf(r1.x, ex, fmaf(r1.y, ey, r1.z * ez));
                const float v1 = fmaf(r1.w, ex, fmaf(r2.x, ey, r2.y * ez));
                const float v2 = fmaf(r2.z, ex, fmaf(r2.w, ey, r3.x * ez));
                const float m2 = fmaf(v0, v0, fmaf(v1, v1, v2 * v2));
                const float resp = r3.y * expf(-0.5f * m2);
                if (resp >= k.alpha_min) {
                    hit = true;
                    al = fminf(resp, k.alpha_max);
                }
            }
        }
        __syncwarp();
        // drop the evaluated candidates (with take == 32 the sources lie at
        // 32 and above and the destinations below 32, so nothing overlaps)
        if (lane < qn - take) que[lane] = que[lane + take];
        qn -= take;
        __syncwarp();
        const unsigned m = __ballot_sync(0xffffffffu, hit);
        if (hit) {
            const int pos = n + __popc(m & ((1u << lane) - 1u));
            if (pos < kHitCap) {
                key[pos] = hit_key(ts, gi);
                alp[pos] = al;
            }
        }
        n += __popc(m);
        __syncwarp();
    }
}

// Sorts key/alp[0, n) (n <= kHitCap) by key: ranks for a few hits, a bitonic
// network over the lanes up to 32, a shared-memory bitonic network above.
__device__ __forceinline__ void sort_hits(uint64_t* key, float* alp, const int n, const int lane)
{
    __syncwarp();
    if (n > 32 && n <= 64) {
        // 64 elements in registers, two a lane: element lane (a) and
        // lane + 32 (b); a bitonic network whose j = 32 steps compare a lane's
        // own pair and whose others exchange over the lanes
        uint64_t ka = key[lane], kb = lane + 32 < n ? key[lane + 32] : ~0ull;
        float aa = alp[lane], ab = lane + 32 < n ? alp[lane + 32] : 0.f;
#pragma unroll 1
        for (int kk = 2; kk <= 64; kk <<= 1) {
#pragma unroll 1
            for (int j = kk >> 1; j > 0; j >>= 1) {
                if (j == 32) {
                    // (kk = 64: every pair ascending)
                    if (kb < ka) {
                        const uint64_t tk = ka;
                        ka = kb;
                        kb = tk;
                        const float ta = aa;
                        aa = ab;
                        ab = ta;
                    }
                    continue;
                }
                const bool lower = (lane & j) == 0;
                // element index lane (+ 32): ascending where (index & kk) == 0
                const bool up_a = (lane & kk) == 0;
                const bool up_b = ((lane + 32) & kk) == 0;
                const uint64_t koa = __shfl_xor_sync(0xffffffffu, ka, j);
                const float aoa = __shfl_xor_sync(0xffffffffu, aa, j);
                const uint64_t kob = __shfl_xor_sync(0xffffffffu, kb, j);
                const float aob = __shfl_xor_sync(0xffffffffu, ab, j);
                if ((lower == up_a) ? (koa < ka) : (koa > ka)) {
                    ka = koa;
                    aa = aoa;
                }
                if ((lower == up_b) ? (kob < kb) : (kob > kb)) {
                    kb = kob;
                    ab = aob;
                }
            }
        }
        key[lane] = ka;
        alp[lane] = aa;
        if (lane + 32 < n) {
            key[lane + 32] = kb;
            alp[lane + 32] = ab;
        }
    } else if (n > 64) {
        int P2 = 64;
        while (P2 < n) P2 <<= 1;
        for (int i = n + lane; i < P2; i += 32) {
            key[i] = ~0ull;
            alp[i] = 0.f;
        }
        __syncwarp();
        for (int kk = 2; kk <= P2; kk <<= 1) {
            for (int j = kk >> 1; j > 0; j >>= 1) {
                for (int i = lane; i < P2; i += 32) {
                    const int ixj = i ^ j;
                    if (ixj > i) {
                        const uint64_t a = key[i], b = key[ixj];
                        const bool up = (i & kk) == 0;
                        if ((a > b) == up) {
                            key[i] = b;
                            key[ixj] = a;
                            const float ta = alp[i];
                            alp[i] = alp[ixj];
                            alp[ixj] = ta;
                        }
                    }
                }
                __syncwarp();
            }
        }
    } else if (n > 1 && n <= 12) {
        // each lane's rank is the number of smaller keys
        const uint64_t kv = lane < n ? key[lane] : ~0ull;
        const float av = lane < n ? alp[lane] : 0.f;
        int rank = 0;
        for (int j = 0; j < n; ++j) rank += __shfl_sync(0xffffffffu, kv, j) < kv ? 1 : 0;
        __syncwarp();
        if (lane < n) {
            key[rank] = kv;
            alp[rank] = av;
        }
    } else if (n > 1) {
        uint64_t kv = lane < n ? key[lane] : ~0ull;
        float av = lane < n ? alp[lane] : 0.f;
#pragma unroll
        for (int kk = 2; kk <= 32; kk <<= 1) {
#pragma unroll
            for (int j = kk >> 1; j > 0; j >>= 1) {
                const uint64_t ko = __shfl_xor_sync(0xffffffffu, kv, j);
                const float ao = __shfl_xor_sync(0xffffffffu, av, j);
                const bool lower = (lane & j) == 0;
                const bool up = (lane & kk) == 0;
                // keep the smaller key on the lower lane of an ascending pair
                const bool tk = (lower == up) ? (ko < kv) : (ko > kv);
                if (tk) {
                    kv = ko;
                    av = ao;
                }
            }
        }
        if (lane < n) {
            key[lane] = kv;
            alp[lane] = av;
        }
    }
    __syncwarp();
}

// Composites the hits with t* < thr (every hit when `all`). They move to the
// scratch buffer dkey/dalp (the others close up, in order, at the front of
// key/alp, and n becomes their count), are sorted by (t*, index) and taken
// front to back, 32 at a time, with a prefix product of (1 - alpha). The
// ray stops once the transmittance falls below t_stop. In G-buffer mode each
// hit also adds its normal (turned against the ray direction d) and its
// materials.
template <int OUT>
__device__ __forceinline__ void composite_hits(const TraceK& k, uint64_t* key, float* alp, uint64_t* dkey,
                                               float* dalp, int& n, const bool all, const float thr, const int lane,
                                               RayAcc& acc, const float3 d)
{
    const unsigned below = (1u << lane) - 1u;
    int nd = 0, nr = 0;
    for (int i0 = 0; i0 < n; i0 += 32) {
        const int i = i0 + lane;
        const bool in = i < n;
        const uint64_t kv = in ? key[i] : 0ull;
        const float av = in ? alp[i] : 0.f;
        const float tv = o2f((int32_t)((uint32_t)(kv >> 32) ^ 0x80000000u));
        const bool due = in && (all || tv < thr);
        const unsigned dm = __ballot_sync(0xffffffffu, due), rm = __ballot_sync(0xffffffffu, in && !due);
        __syncwarp();
        if (due) {
            const int j = nd + __popc(dm & below);
            dkey[j] = kv;
            dalp[j] = av;
        } else if (in) {
            // j <= i: the chunk was read before any of it is overwritten
            const int j = nr + __popc(rm & below);
            key[j] = kv;
            alp[j] = av;
        }
        nd += __popc(dm);
        nr += __popc(rm);
        __syncwarp();
    }
    n = nr;
    if (nd == 0) return;
    sort_hits(dkey, dalp, nd, lane);
    int used = 0;
    for (int cb = 0; cb < nd && !acc.done; cb += 32) {
        const int h = cb + lane;
        const bool on = h < nd;
        const uint64_t kh = on ? dkey[h] : 0ull;
        const float th_hit = o2f((int32_t)((uint32_t)(kh >> 32) ^ 0x80000000u));
        const float a = on ? dalp[h] : 0.f;
        const int32_t gh = (int32_t)(uint32_t)(kh & 0xffffffffu);
        // inclusive prefix product of (1 - alpha)
        float pin = 1.f - a;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const float v = __shfl_up_sync(0xffffffffu, pin, off);
            if (lane >= off) pin *= v;
        }
        float pex = __shfl_up_sync(0xffffffffu, pin, 1);
        if (lane == 0) pex = 1.f;
        const float Tb = acc.T * pex, Ta = acc.T * pin;
        // first lane whose transmittance after its hit is below t_stop
        const unsigned stopm = __ballot_sync(0xffffffffu, on && Ta < k.t_stop);
        const int stop_lane = stopm ? __ffs(stopm) - 1 : 32;
        const bool use = on && lane <= stop_lane;
        const float w = use ? Tb * a : 0.f;
        if (use) {
            const float4 r3 = __ldg(&k.rec[gh].r3), r4 = __ldg(&k.rec[gh].r4);
            acc.L0 = fmaf(w, r3.z, acc.L0);
            acc.L1 = fmaf(w, r3.w, acc.L1);
            acc.L2 = fmaf(w, r4.x, acc.L2);
            acc.Dacc = fmaf(w, th_hit, acc.Dacc);
            acc.Wacc += w;
            if (OUT == kTraceGbuf) {
                const float3 nv = surfel_normal(k, gh);
                const float ws = dot3(nv, d) > 0.f ? -w : w;
                acc.N0 = fmaf(ws, nv.x, acc.N0);
                acc.N1 = fmaf(ws, nv.y, acc.N1);
                acc.N2 = fmaf(ws, nv.z, acc.N2);
                acc.A0 = fmaf(w, __ldg(k.albedo + 3 * gh), acc.A0);
                acc.A1 = fmaf(w, __ldg(k.albedo + 3 * gh + 1), acc.A1);
                acc.A2 = fmaf(w, __ldg(k.albedo + 3 * gh + 2), acc.A2);
                acc.Rg = fmaf(w, __ldg(k.rough + gh), acc.Rg);
                acc.Mg = fmaf(w, __ldg(k.metal + gh), acc.Mg);
            }
        }
        const int cnt = stop_lane < 32 ? stop_lane + 1 : min(32, nd - cb);
        used += cnt;
        acc.T = __shfl_sync(0xffffffffu, Ta, cnt - 1);
        if (stop_lane < 32) acc.done = true;
    }
    acc.n_comp += used;
    if (acc.done) n = 0;
    __syncwarp();
}

// Tests the cell entries [e0, e1) against the ray: the ray's entry E into
// the entry's box (not before the walk's start t0).
// Gaussians with E in [tl, th_e) are queued. Queued candidates are evaluated
// 32 at a time as the queue fills, and at the end while at least `least`
// remain. Entries are loaded 32 ahead of the ones being tested: pv holds
// entry pe + lane, and the last batch of the range loads the first one of
// the next range [nf, ne) (the next cell's, when the walk knows it). An
// entry's centre along axis a is go_a + span_a u (u = q / 65536, decoded as
// v = 1 + u from its bits), so its slab time (centre - o_a) / d_a is
// v qa_a + qb_a with the ray's qa = span iv and qb = (go - o) iv - qa: one
// FMA, the same in every cell.
__device__ __forceinline__ void scan_eval(const TraceK& k, const float3 o, const float3 iv, const float3 qa,
                                          const float3 qb, const float t0, const int e0, const int e1,
                                          const int nf, const int ne, const float tl, const float th_e,
                                          const int least, uint4& pv, int& pe, int32_t* que, int& qn,
                                          int& pend, uint64_t* key, float* alp, int& n, const int lane,
                                          RayAcc& acc, const float3 d)
{
    int eb = e0;
    if (eb < e1) acc.n_test += e1 - eb;
    if (eb < e1 && pe != eb) {
        pe = eb;
        if (eb + lane < e1) pv = __ldg(k.ent + eb + lane);
    }
    while (eb < e1 || (qn >= least && qn > 0)) {
        if (eb < e1) {
            const uint4 en = pv;
            const bool valid = eb + lane < e1;
            eb += 32;
            pe = eb < e1 ? eb : (ne > nf ? nf : -1);
            const int pl = eb < e1 ? e1 : ne;
            if (pe + lane < pl) pv = __ldg(k.ent + pe + lane);
            // box: slab entries/exits (c - o) iv -+ h |iv| per axis
            const float px = fmaf(__uint_as_float(0x3f800000u | ((en.x & 0xffffu) << 7)), qa.x, qb.x);
            const float py = fmaf(__uint_as_float(0x3f800000u | ((en.x >> 16) << 7)), qa.y, qb.y);
            const float pz = fmaf(__uint_as_float(0x3f800000u | ((en.y & 0xffffu) << 7)), qa.z, qb.z);
            const float qx = hdecode(en.y >> 16) * fabsf(iv.x), qy = hdecode(en.z & 0xffffu) * fabsf(iv.y),
                        qz = hdecode(en.z >> 16) * fabsf(iv.z);
            const float tin = fmaxf(fmaxf(px - qx, py - qy), pz - qz);
            const float tout = fminf(fminf(px + qx, py + qy), pz + qz);
            const float E = fmaxf(tin, t0);
            const bool pass = valid && tout >= E && E >= tl && E < th_e;
            const unsigned pm = __ballot_sync(0xffffffffu, pass);
            if (pass) que[qn + __popc(pm & ((1u << lane) - 1u))] = (int32_t)en.w;
            qn += __popc(pm);
            pend += __popc(pm);
            __syncwarp();
            if (qn < 32) continue;
        }
        eval_batch(k, o, d, que, qn, key, alp, n, lane, acc);
    }
}

// default of TraceK::composite_at
constexpr int kCompositeAt = 48;

// One warp per texel ray. Lanes share the grid walk (uniform control flow)
// and split each cell's entries. Every Gaussian is evaluated once per ray:
// in the cell window that holds the ray's entry into its axis-aligned box.
// Candidates queue across cells and are evaluated 32 at a time; their hits
// (t*, alpha) wait in the warp's shared buffer. Once enough have gathered,
// the buffer is sorted by (t*, index) and the hits whose t* the walk has
// passed are composited, so that hits are taken in (t*, index) order even
// when a box spans several cells. A cell whose entries alone could overflow
// the buffer is taken in halves of its window until each part fits.
// Binning fills each cell's entries in no fixed order, and which queued
// candidates have been evaluated at a cell's end depends on that order. So
// the decisions of when to composite and how to take a cell use only
// order-free counts: nw, the hits left waiting by the last composite, plus
// pend, the candidates queued since (an upper bound of hits + queue). At a
// composite the queue is always empty, so the set of hits composited, and
// with it every rounding, is the same on every run.
template <int OUT>
__global__ void __launch_bounds__(256, OUT == kTraceAtlas ? 4 : 3) trace_kernel(const TraceK k)
{
    __shared__ uint64_t s_key[kWarpsPerCta][kHitCap];
    __shared__ float s_alpha[kWarpsPerCta][kHitCap];
    __shared__ uint64_t s_dkey[kWarpsPerCta][kHitCap];
    __shared__ float s_dalpha[kWarpsPerCta][kHitCap];
    __shared__ int32_t s_que[kWarpsPerCta][64];
    if (k.run_if && __ldg(k.run_if) == 0) return;
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint64_t* key = s_key[wib];
    float* alp = s_alpha[wib];
    uint64_t* dkey = s_dkey[wib];
    float* dalp = s_dalpha[wib];
    int32_t* que = s_que[wib];
    const int64_t RR = k.n_dirs;
    const int64_t total = (int64_t)k.P * RR;
    const GaussGrid G = *k.grid;
    const float3 go = f3(G.origin[0], G.origin[1], G.origin[2]);
    const float3 sp = f3(G.bmax[0] - G.origin[0], G.bmax[1] - G.origin[1], G.bmax[2] - G.origin[2]);
    // persistent warps: each takes its next rays from a global counter, so
    // long rays (escaping the object) do not hold up short ones. Rays are
    // taken kBatch at a time (camera rays are mostly short: one counter
    // update per ray would serialise on it); the next batch's number is
    // fetched while the current batch is traced
    const int kBatch = k.batch;
    unsigned long long rr = 0;
    if (lane == 0) rr = atomicAdd(k.stats, (unsigned long long)kBatch);
    int64_t base = 0;
    int sub = kBatch;
    // work counters, summed over the warp's rays and added once at the end
    unsigned long long t_eval = 0, t_comp = 0, t_test = 0;
    for (;;) {
    if (sub == kBatch) {
        base = (int64_t)__shfl_sync(0xffffffffu, rr, 0);
        sub = 0;
        if (lane == 0 && base < total) rr = atomicAdd(k.stats, (unsigned long long)kBatch);
    }
    const int64_t ray = base + sub++;
    if (ray >= total) break;
    const int p = (int)(ray / RR), t = (int)(ray % RR);
    const float4 d4 = __ldg(k.dirs + t);
    const float3 d = f3(d4.x, d4.y, d4.z);
    const float3 o = load3(k.probe_pos, p);
    // a non-finite origin or direction is reported, and its ray traces
    // nothing (empty composite)
    const bool ray_ok = isfinite(o.x + o.y + o.z + d.x + d.y + d.z);
    if (!ray_ok && lane == 0 && k.status) atomicOr(k.status, SOP_DEVSTAT_NONFINITE);
    // reciprocal direction for the box entries (a zero component becomes a
    // tiny one: the slab along that axis is then all or nothing)
    const float3 iv = f3(1.f / (fabsf(d.x) > 1e-30f ? d.x : 1e-30f), 1.f / (fabsf(d.y) > 1e-30f ? d.y : 1e-30f),
                         1.f / (fabsf(d.z) > 1e-30f ? d.z : 1e-30f));
    // the box test's slab-time constants (see scan_eval)
    const float3 qa = f3(sp.x * iv.x, sp.y * iv.y, sp.z * iv.z);
    const float3 qb = f3((go.x - o.x) * iv.x - qa.x, (go.y - o.y) * iv.y - qa.y, (go.z - o.z) * iv.z - qa.z);
    RayAcc acc;
    acc.T = 1.f;
    acc.L0 = acc.L1 = acc.L2 = acc.Dacc = acc.Wacc = 0.f;
    acc.N0 = acc.N1 = acc.N2 = acc.A0 = acc.A1 = acc.A2 = acc.Rg = acc.Mg = 0.f;
    acc.n_eval = acc.n_comp = acc.n_test = 0;
    acc.done = false;
    int n = 0, qn = 0;  // hits in key/alp[0, n) (unsorted); candidates in que[0, qn)
    int nw = 0, pend = 0;  // hits waiting after the last composite; candidates queued since
    uint4 pv = make_uint4(0u, 0u, 0u, 0u);  // entry pe + lane, loaded ahead
    int pe = -1;

    // grid box entry/exit (slab test), per axis in scalars so that nothing
    // is indexed by a run-time axis (which would put it in local memory)
    const float gox = G.origin[0], goy = G.origin[1], goz = G.origin[2];
    const float gmx = G.bmax[0], gmy = G.bmax[1], gmz = G.bmax[2];
    const int gdx = G.dims[0], gdy = G.dims[1], gdz = G.dims[2];
    const float gh = G.h, gih = G.inv_h;
    float t0 = 0.f, t1 = FLT_MAX;
#define SOP_SLAB(OA, DA, IA, LO, HI)                                 \
    if (DA != 0.f) {                                                 \
        float ta = (LO - OA) * IA, tb = (HI - OA) * IA;              \
        if (ta > tb) {                                               \
            const float tmp = ta;                                    \
            ta = tb;                                                 \
            tb = tmp;                                                \
        }                                                            \
        t0 = fmaxf(t0, ta);                                          \
        t1 = fminf(t1, tb);                                          \
    } else if (OA < LO || OA > HI) {                                 \
        t1 = -1.f;                                                   \
    }
    SOP_SLAB(o.x, d.x, iv.x, gox, gmx)
    SOP_SLAB(o.y, d.y, iv.y, goy, gmy)
    SOP_SLAB(o.z, d.z, iv.z, goz, gmz)
#undef SOP_SLAB
    if (ray_ok && G.fits && G.n_entries > 0 && t0 <= t1) {
        int cx = min(max((int)floorf((o.x + t0 * d.x - gox) * gih), 0), gdx - 1);
        int cy = min(max((int)floorf((o.y + t0 * d.y - goy) * gih), 0), gdy - 1);
        int cz = min(max((int)floorf((o.z + t0 * d.z - goz) * gih), 0), gdz - 1);
        const int sx = d.x > 0.f ? 1 : (d.x < 0.f ? -1 : 0);
        const int sy = d.y > 0.f ? 1 : (d.y < 0.f ? -1 : 0);
        const int sz = d.z > 0.f ? 1 : (d.z < 0.f ? -1 : 0);
        // t at the next cell boundary along each axis, from the cell index
        // (no accumulated error; the bins' margin covers the rounding)
#define SOP_TNEXT(S, C, GO, OA, IA) ((S) == 0 ? FLT_MAX : ((GO) + ((C) + ((S) > 0 ? 1 : 0)) * gh - (OA)) * (IA))
        float tmx = SOP_TNEXT(sx, cx, gox, o.x, iv.x);
        float tmy = SOP_TNEXT(sy, cy, goy, o.y, iv.y);
        float tmz = SOP_TNEXT(sz, cz, goz, o.z, iv.z);
        float t_enter = t0;
        // entry range of the current cell; the next cell's range is loaded
        // one cell ahead
        int e0 = __ldg(k.cell_start + (cz * gdy + cy) * gdx + cx);
        int e1 = __ldg(k.cell_start + (cz * gdy + cy) * gdx + cx + 1);
        while (!acc.done) {
            const int ax = (tmx <= tmy && tmx <= tmz) ? 0 : (tmy <= tmz ? 1 : 2);
            const float tm = ax == 0 ? tmx : (ax == 1 ? tmy : tmz);
            float t_exit = fminf(tm, t1);
            if (t_exit < t_enter) t_exit = t_enter;
            // the last cell of the walk takes every box entry beyond it and
            // composites every waiting hit
            bool last = !(t_exit < t1);
            if (!last) {
                const int nx = ax == 0 ? cx + sx : (ax == 1 ? cy + sy : cz + sz);
                const int nd = ax == 0 ? gdx : (ax == 1 ? gdy : gdz);
                last = nx < 0 || nx >= nd;
            }
            int ne0 = 0, ne1 = 0;
            if (!last) {
                const int cn = (cz * gdy + cy) * gdx + cx + (ax == 0 ? sx : (ax == 1 ? sy * gdx : sz * gdx * gdy));
                ne0 = __ldg(k.cell_start + cn);
                ne1 = __ldg(k.cell_start + cn + 1);
            }
            // an empty cell with no composite due changes nothing: step on
            if (!(e0 == e1 && !last && nw + pend < k.composite_at)) {
                const float tl = t_enter;
                // mode 0: the cell cannot overflow the hit buffer; scan it, and
                //   composite once enough hits have gathered (or at the end).
                // mode 1: it could; first composite what lies before it, then go
                //   on in mode 0 if the cell now fits, else in
                // mode 2: take its window in parts [sl, sh), halving a part whose
                //   hits overflow the buffer.
                int mode = nw + pend + (e1 - e0) <= kHitCap ? 0 : 1;
                int from = mode == 0 ? e0 : e1, least = mode == 0 ? 32 : 1;
                float sl = tl, sh = t_exit;
                int splits = 0;
                for (;;) {
                    const bool sfin = last && !(sh < t_exit);
                    const float lo = mode == 2 ? sl : tl;
                    const float hi_e = (mode == 2 ? sfin : last) ? FLT_MAX : (mode == 2 ? sh : t_exit);
                    const int nb = n, pb = pend;
                    // in mode 0 the walk goes on to the next cell: load its first entries
                    scan_eval(k, o, iv, qa, qb, t0, from, e1, mode == 0 ? ne0 : 0, mode == 0 ? ne1 : 0, lo, hi_e, least,
                              pv, pe, que, qn, pend, key, alp, n, lane, acc, d);
                    if (mode == 0 && least == 32) {
                        if (!(last || nw + pend >= k.composite_at)) break;
                        from = e1;  // evaluate what is still queued, then composite
                        least = 1;
                        continue;
                    }
                    if (mode == 2 && n > kHitCap) {
                        n = nb;
                        pend = pb;
                        // halve the part; once it cannot shrink (the midpoint
                        // rounds onto sl: more hits than the buffer holds
                        // share one entry point) or after 40 halvings, stop
                        // the ray. The test comes before the part is taken:
                        // an empty part [sl, sl) would count as taken and
                        // restart the halving from t_exit without progress.
                        // Every part taken therefore advances sl strictly.
                        const float mid = sl + 0.5f * (sh - sl);
                        if (++splits > 40 || !(mid > sl)) {
                            // (the status word learns of it from stats[3]
                            // after the launch: kept out of this loop, its
                            // pointer would cost the walk registers)
                            if (lane == 0) atomicOr(k.stats + 3, 1ull);
                            acc.done = true;
                            break;
                        }
                        sh = mid;
                        continue;
                    }
                    composite_hits<OUT>(k, key, alp, dkey, dalp, n, mode == 0 ? last : (mode == 2 && sfin),
                                        mode == 0 ? t_exit : (mode == 1 ? tl : sh), lane, acc, d);
                    nw = n;
                    pend = 0;
                    if (acc.done || mode == 0) break;
                    if (mode == 2) {
                        if (!(sh < t_exit)) break;
                        sl = sh;
                        sh = t_exit;
                        splits = 0;
                    } else {
                        // the waiting hits are now those beyond tl: the cell may fit
                        mode = n + (e1 - e0) <= kHitCap ? 0 : 2;
                        least = mode == 0 ? 32 : 1;
                    }
                    from = e0;
                }
                if (acc.done || last) break;
            }
            e0 = ne0;
            e1 = ne1;
            // step one cell; the boundary is recomputed from the cell index
            // (no accumulated error)
            if (ax == 0) {
                cx += sx;
                tmx = SOP_TNEXT(sx, cx, gox, o.x, iv.x);
            } else if (ax == 1) {
                cy += sy;
                tmy = SOP_TNEXT(sy, cy, goy, o.y, iv.y);
            } else {
                cz += sz;
                tmz = SOP_TNEXT(sz, cz, goz, o.z, iv.z);
            }
            t_enter = t_exit;
        }
#undef SOP_TNEXT
    }
    float L0 = acc.L0, L1 = acc.L1, L2 = acc.L2, Dacc = acc.Dacc, Wacc = acc.Wacc;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        L0 += __shfl_xor_sync(0xffffffffu, L0, off);
        L1 += __shfl_xor_sync(0xffffffffu, L1, off);
        L2 += __shfl_xor_sync(0xffffffffu, L2, off);
        Dacc += __shfl_xor_sync(0xffffffffu, Dacc, off);
        Wacc += __shfl_xor_sync(0xffffffffu, Wacc, off);
    }
    if (OUT == kTraceGbuf) {
        float v[8] = {acc.N0, acc.N1, acc.N2, acc.A0, acc.A1, acc.A2, acc.Rg, acc.Mg};
#pragma unroll
        for (int c = 0; c < 8; ++c)
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v[c] += __shfl_xor_sync(0xffffffffu, v[c], off);
        if (lane == 0) {
            float4* o4 = k.gbuf + 4 * ray;
            o4[0] = make_float4(L0, L1, L2, Wacc);
            o4[1] = make_float4(v[0], v[1], v[2], Dacc);
            o4[2] = make_float4(v[3], v[4], v[5], v[6]);
            o4[3] = make_float4(v[7], 0.f, 0.f, 0.f);
        }
        t_eval += (unsigned long long)acc.n_eval;
        t_comp += (unsigned long long)acc.n_comp;
        t_test += (unsigned long long)acc.n_test;
        continue;
    }
    if (lane == 0) {
        // interior texel (t % R, t / R) of probe p, stored at (+1, +1)
        const int RS = k.R + 2;
        const int64_t ti = (int64_t)p * RS * RS + (int64_t)(t / k.R + 1) * RS + (t % k.R + 1);
        const float4 v = make_float4(L0, L1, L2, 1.f - acc.T);
        switch (k.rgbo_dtype) {
        case SOP_F32: reinterpret_cast<float4*>(k.rgbo)[ti] = v; break;
        case SOP_BF16: reinterpret_cast<uint2*>(k.rgbo)[ti] = Texel<SOP_BF16>::pack(v); break;
        default: reinterpret_cast<uint2*>(k.rgbo)[ti] = Texel<SOP_F16>::pack(v); break;
        }
        if (k.depth) {
            const float dv = (Wacc > 1e-8f ? Dacc / Wacc : 0.f) * k.inv_depth_scale;
            switch (k.depth_dtype) {
            case SOP_F32: reinterpret_cast<float*>(k.depth)[ti] = dv; break;
            case SOP_F16: reinterpret_cast<__half*>(k.depth)[ti] = __float2half_rn(dv); break;
            case SOP_BF16: reinterpret_cast<__nv_bfloat16*>(k.depth)[ti] = __float2bfloat16_rn(dv); break;
            default: reinterpret_cast<__nv_fp8_e4m3*>(k.depth)[ti] = __nv_fp8_e4m3(dv); break;
            }
        }
    }
    t_eval += (unsigned long long)acc.n_eval;
    t_comp += (unsigned long long)acc.n_comp;
    t_test += (unsigned long long)acc.n_test;
    }  // next ray
    if (lane == 0) {
        atomicAdd(k.stats + 1, t_eval);
        atomicAdd(k.stats + 2, t_comp);
        atomicAdd(k.stats + 4, t_test);
    }
}

cudaError_t launch_bake_bin(const sop_gaussians& g, float alpha_min, const BakeLayout& L, char* ws, cudaStream_t s)
{
    const cudaError_t e = launch_bake_prep(g, alpha_min, L, ws, s);
    return e != cudaSuccess ? e : launch_bake_grid(g, L, ws, s);
}

cudaError_t launch_bake_prep(const sop_gaussians& g, float alpha_min, const BakeLayout& L, char* ws, cudaStream_t s)
{
    int32_t* bbox = reinterpret_cast<int32_t*>(ws + L.bbox);
    GRec* rec = reinterpret_cast<GRec*>(ws + L.rec);
    bbox_init_kernel<<<1, 32, 0, s>>>(bbox);
    const unsigned nb = (unsigned)((g.n + 255) / 256);
    if (g.n > 0) gauss_prep_kernel<<<nb, 256, 0, s>>>(g, alpha_min, rec, bbox, status_word());
    return cudaGetLastError();
}

cudaError_t launch_bake_grid(const sop_gaussians& g, const BakeLayout& L, char* ws, cudaStream_t s)
{
    GaussGrid* grid = reinterpret_cast<GaussGrid*>(ws + L.hdr);
    int32_t* bbox = reinterpret_cast<int32_t*>(ws + L.bbox);
    GRec* rec = reinterpret_cast<GRec*>(ws + L.rec);
    int32_t* cstart = reinterpret_cast<int32_t*>(ws + L.cell_start);
    int32_t* ccnt = reinterpret_cast<int32_t*>(ws + L.cell_cnt);
    unsigned int* status = status_word();
    const int bs = 256;
    const unsigned nb = (unsigned)((g.n + bs - 1) / bs);
    // Binning attempts, decided on the device (no host read-back): the
    // requested grid; if its cell lists overflow the workspace, a grid with
    // 1/16 of the cells; then one of at most 2 cells, whose lists (at most
    // 2 entries per Gaussian) always fit, since the workspace holds at least
    // 24 per Gaussian. Attempts after a fitting one return at once.
    const int64_t caps[kBinAttempts] = {L.cells_cap, L.cells_cap / 16 > 64 ? L.cells_cap / 16 : 64, 2};
    for (int a = 0; a < kBinAttempts; ++a) {
        grid_setup_kernel<<<1, 1024, 0, s>>>(bbox, caps[a], a, grid, ccnt);
        if (g.n > 0) bin_count_kernel<<<nb, bs, 0, s>>>(g.n, rec, grid, ccnt);
        ScanArgs sa;
        sa.n = &grid->ncells;
        sa.skip = &grid->fits;
        sa.cnt = ccnt;
        sa.start = cstart;
        sa.scratch = reinterpret_cast<long long*>(ws + L.scan);
        launch_scan(sa, caps[a], BinScanFinal{grid, L.entries_cap, status}, s);
    }
    return cudaGetLastError();
}

// Border texels of an atlas copied from the texels the border rule names.
__global__ void gutter_fill_kernel(int32_t P, int32_t R, void* __restrict__ rgbo, int rgbo_bytes,
                                   void* __restrict__ depth, int depth_bytes, const int32_t* run_if,
                                   const unsigned long long* stats, unsigned int* status)
{
    if (run_if && __ldg(run_if) == 0) return;
    // a ray of the trace before this launch stopped early (stats[3] bit 0)
    if (blockIdx.x == 0 && threadIdx.x == 0 && stats && status && (stats[3] & 1ull))
        atomicOr(status, SOP_DEVSTAT_BAKE_TRUNCATED);
    const int RS = R + 2, NB = 4 * (R + 1);  // border texels per probe
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)P * NB) return;
    const int64_t p = i / NB;
    const int b = (int)(i % NB);
    int ii, jj;  // stored coordinates of this border texel
    if (b < RS) { ii = b; jj = 0; }
    else if (b < 2 * RS) { ii = b - RS; jj = RS - 1; }
    else if (b < 2 * RS + R) { ii = 0; jj = b - 2 * RS + 1; }
    else { ii = RS - 1; jj = b - 2 * RS - R + 1; }
    int si, sj;
    oct_wrap(R, ii - 1, jj - 1, si, sj);
    const int64_t dst = p * RS * RS + (int64_t)jj * RS + ii, src = p * RS * RS + (int64_t)(sj + 1) * RS + (si + 1);
    if (rgbo_bytes == 16) reinterpret_cast<float4*>(rgbo)[dst] = reinterpret_cast<const float4*>(rgbo)[src];
    else reinterpret_cast<uint2*>(rgbo)[dst] = reinterpret_cast<const uint2*>(rgbo)[src];
    if (depth) {
        if (depth_bytes == 4) reinterpret_cast<float*>(depth)[dst] = reinterpret_cast<const float*>(depth)[src];
        else if (depth_bytes == 2)
            reinterpret_cast<uint16_t*>(depth)[dst] = reinterpret_cast<const uint16_t*>(depth)[src];
        else reinterpret_cast<uint8_t*>(depth)[dst] = reinterpret_cast<const uint8_t*>(depth)[src];
    }
}

__global__ void trace_reset_kernel(unsigned long long* stats)
{
    if (threadIdx.x < 8) stats[threadIdx.x] = 0ull;
}

// the truncation bit of a G-buffer trace into the status word
__global__ void trace_status_kernel(const unsigned long long* stats, unsigned int* status)
{
    if (status && (stats[3] & 1ull)) atomicOr(status, SOP_DEVSTAT_BAKE_TRUNCATED);
}

cudaError_t launch_bake_fill(const sop_gaussians& g, const BakeLayout& L, char* ws, cudaStream_t s)
{
    GaussGrid* grid = reinterpret_cast<GaussGrid*>(ws + L.hdr);
    GRec* rec = reinterpret_cast<GRec*>(ws + L.rec);
    int32_t* cstart = reinterpret_cast<int32_t*>(ws + L.cell_start);
    int32_t* ccnt = reinterpret_cast<int32_t*>(ws + L.cell_cnt);
    uint4* ent = reinterpret_cast<uint4*>(ws + L.ent);
    const int bs = 256;
    if (g.n > 0)
        bin_fill_kernel<<<(unsigned)((g.n + bs - 1) / bs), bs, 0, s>>>(g.n, rec, grid, cstart, ccnt, ent);
    return cudaGetLastError();
}

// persistent grid: as many CTAs as fit on the device at once (fewer for a
// small launch)
template <int OUT>
static unsigned trace_blocks(int64_t rays)
{
    static int resident = 0;
    if (!resident) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, trace_kernel<OUT>, kWarpsPerCta * 32, 0);
        resident = (sms > 0 ? sms : 152) * (per_sm > 0 ? per_sm : 1);
    }
    const int64_t need = (rays + kWarpsPerCta - 1) / kWarpsPerCta;
    return (unsigned)(need < resident ? need : resident);
}

cudaError_t launch_bake_trace(const sop_atlas& atlas, const sop_bake_params& bp, const BakeLayout& L, char* ws,
                              cudaStream_t s, const int32_t* run_if)
{
    GaussGrid* grid = reinterpret_cast<GaussGrid*>(ws + L.hdr);
    const int R = atlas.R;
    float4* dirs = reinterpret_cast<float4*>(ws + L.dirs);
    unsigned long long* stats = reinterpret_cast<unsigned long long*>(ws + L.stats);
    trace_reset_kernel<<<1, 32, 0, s>>>(stats);
    texel_dirs_kernel<<<(R * R + 127) / 128, 128, 0, s>>>(R, dirs);
    TraceK k;
    k.rec = reinterpret_cast<GRec*>(ws + L.rec);
    k.grid = grid;
    k.cell_start = reinterpret_cast<int32_t*>(ws + L.cell_start);
    k.ent = reinterpret_cast<uint4*>(ws + L.ent);
    k.dirs = dirs;
    k.probe_pos = atlas.probe_pos;
    k.P = atlas.P;
    k.R = R;
    k.t_near = bp.t_near;
    k.alpha_min = bp.alpha_min;
    k.alpha_max = bp.alpha_max;
    k.t_stop = bp.t_stop;
    k.rgbo = atlas.rgbo;
    k.depth = atlas.depth;
    k.rgbo_dtype = atlas.rgbo_dtype;
    k.depth_dtype = atlas.depth_dtype;
    k.inv_depth_scale = 1.f / atlas.depth_scale;
    k.stats = stats;
    k.composite_at = kCompositeAt;
    k.n_dirs = (int64_t)R * R;
    k.batch = 1;
    k.quat = k.scale = k.albedo = k.rough = k.metal = nullptr;
    k.gbuf = nullptr;
    k.status = status_word();
    k.run_if = run_if;
    const int64_t rays = (int64_t)atlas.P * R * R;
    trace_kernel<kTraceAtlas><<<trace_blocks<kTraceAtlas>(rays), kWarpsPerCta * 32, 0, s>>>(k);
    return launch_gutter_fill(atlas, s, run_if, stats);
}

cudaError_t launch_trace_gbuffer(const sop_gaussians& g, const float* albedo, const float* rough, const float* metal,
                                 const float* origins, int32_t n_origins, const float* dirs, int64_t n_dirs,
                                 const sop_bake_params& bp, const BakeLayout& L, char* ws, float* out, cudaStream_t s)
{
    unsigned long long* stats = reinterpret_cast<unsigned long long*>(ws + L.stats);
    trace_reset_kernel<<<1, 32, 0, s>>>(stats);
    TraceK k;
    k.rec = reinterpret_cast<GRec*>(ws + L.rec);
    k.grid = reinterpret_cast<GaussGrid*>(ws + L.hdr);
    k.cell_start = reinterpret_cast<int32_t*>(ws + L.cell_start);
    k.ent = reinterpret_cast<uint4*>(ws + L.ent);
    k.dirs = reinterpret_cast<const float4*>(dirs);
    k.probe_pos = origins;
    k.P = n_origins;
    k.R = 0;
    k.t_near = bp.t_near;
    k.alpha_min = bp.alpha_min;
    k.alpha_max = bp.alpha_max;
    k.t_stop = bp.t_stop;
    k.rgbo = k.depth = nullptr;
    k.rgbo_dtype = k.depth_dtype = 0;
    k.inv_depth_scale = 1.f;
    k.stats = stats;
    k.composite_at = kCompositeAt;
    k.n_dirs = n_dirs;
    k.batch = 8;
    k.quat = g.quat;
    k.scale = g.scale;
    k.albedo = albedo;
    k.rough = rough;
    k.metal = metal;
    k.gbuf = reinterpret_cast<float4*>(out);
    k.status = status_word();
    k.run_if = nullptr;
    const int64_t rays = (int64_t)n_origins * n_dirs;
    if (rays == 0) return cudaGetLastError();
    trace_kernel<kTraceGbuf><<<trace_blocks<kTraceGbuf>(rays), kWarpsPerCta * 32, 0, s>>>(k);
    trace_status_kernel<<<1, 1, 0, s>>>(stats, k.status);
    return cudaGetLastError();
}

cudaError_t launch_gutter_fill(const sop_atlas& atlas, cudaStream_t s, const int32_t* run_if,
                               const unsigned long long* stats)
{
    const int64_t nbord = (int64_t)atlas.P * 4 * (atlas.R + 1);
    const int db = atlas.depth_dtype == SOP_F32 ? 4 : (atlas.depth_dtype == SOP_FP8E4M3 ? 1 : 2);
    gutter_fill_kernel<<<(unsigned)((nbord + 255) / 256), 256, 0, s>>>(
        atlas.P, atlas.R, atlas.rgbo, atlas.rgbo_dtype == SOP_F32 ? 16 : 8, atlas.depth, db, run_if, stats,
        stats ? status_word() : nullptr);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Atlas pack: compact maps -> gutter atlas in the storage dtypes.
// ---------------------------------------------------------------------------
template <int DT>
__global__ void atlas_pack_kernel(const float* __restrict__ rgb, int rgb_stride, const float* __restrict__ occ,
                                  int occ_stride, int32_t P, int32_t R, typename Texel<DT>::raw* __restrict__ out)
{
    const int RS = R + 2;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)P * RS * RS) return;
    const int p = (int)(i / (RS * RS)), r = (int)(i % (RS * RS));
    int si, sj;
    oct_wrap(R, r % RS - 1, r / RS - 1, si, sj);
    const int64_t src = (int64_t)p * R * R + (int64_t)sj * R + si;
    const float4 v = make_float4(rgb[src * rgb_stride], rgb[src * rgb_stride + 1], rgb[src * rgb_stride + 2],
                                 occ[src * occ_stride]);
    out[i] = Texel<DT>::pack(v);
}

template <int DT>
__global__ void depth_pack_kernel(const float* __restrict__ depth, int32_t P, int32_t R, float inv_scale,
                                  void* __restrict__ out)
{
    const int RS = R + 2;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)P * RS * RS) return;
    const int p = (int)(i / (RS * RS)), r = (int)(i % (RS * RS));
    int si, sj;
    oct_wrap(R, r % RS - 1, r / RS - 1, si, sj);
    const float v = depth[(int64_t)p * R * R + (int64_t)sj * R + si] * inv_scale;
    if (DT == SOP_F32) reinterpret_cast<float*>(out)[i] = v;
    else if (DT == SOP_F16) reinterpret_cast<__half*>(out)[i] = __float2half_rn(v);
    else if (DT == SOP_BF16) reinterpret_cast<__nv_bfloat16*>(out)[i] = __float2bfloat16_rn(v);
    else reinterpret_cast<__nv_fp8_e4m3*>(out)[i] = __nv_fp8_e4m3(v);
}

cudaError_t launch_atlas_pack(const float* rgb, int rgb_stride, const float* occ, int occ_stride, const float* depth,
                              const sop_atlas& atlas, cudaStream_t s)
{
    const int RS = atlas.R + 2;
    const int64_t n = (int64_t)atlas.P * RS * RS;
    const unsigned nb = (unsigned)((n + 255) / 256);
    switch (atlas.rgbo_dtype) {
    case SOP_F32:
        atlas_pack_kernel<SOP_F32><<<nb, 256, 0, s>>>(rgb, rgb_stride, occ, occ_stride, atlas.P, atlas.R,
                                                     reinterpret_cast<float4*>(atlas.rgbo));
        break;
    case SOP_BF16:
        atlas_pack_kernel<SOP_BF16><<<nb, 256, 0, s>>>(rgb, rgb_stride, occ, occ_stride, atlas.P, atlas.R,
                                                      reinterpret_cast<uint2*>(atlas.rgbo));
        break;
    case SOP_F16:
        atlas_pack_kernel<SOP_F16><<<nb, 256, 0, s>>>(rgb, rgb_stride, occ, occ_stride, atlas.P, atlas.R,
                                                     reinterpret_cast<uint2*>(atlas.rgbo));
        break;
    default: return cudaErrorInvalidValue;
    }
    if (depth && atlas.depth) {
        const float inv = 1.f / atlas.depth_scale;
        switch (atlas.depth_dtype) {
        case SOP_F32: depth_pack_kernel<SOP_F32><<<nb, 256, 0, s>>>(depth, atlas.P, atlas.R, inv, atlas.depth); break;
        case SOP_F16: depth_pack_kernel<SOP_F16><<<nb, 256, 0, s>>>(depth, atlas.P, atlas.R, inv, atlas.depth); break;
        case SOP_BF16: depth_pack_kernel<SOP_BF16><<<nb, 256, 0, s>>>(depth, atlas.P, atlas.R, inv, atlas.depth); break;
        case SOP_FP8E4M3:
            depth_pack_kernel<SOP_FP8E4M3><<<nb, 256, 0, s>>>(depth, atlas.P, atlas.R, inv, atlas.depth);
            break;
        default: return cudaErrorInvalidValue;
        }
    }
    return cudaGetLastError();
}

}  // namespace sop
