// SOP query + shade (Sec. 3.1.2 Eq. 2-6, Sec. 3.2.2 Eq. 7-9) for sm_103a.
//
// Kernels, in launch order:
//   probe_grid_kernel   one CTA: quantise probe positions to 2^-20, counting
//                       sort into a uniform grid of ~P cells;
//   knn_kernel          one thread per point: exact K nearest probes by
//                       integer squared distance (ring search with an exact
//                       integer stopping bound), then the Eq. 4-6 weights;
//   env_pack_kernel     environment to float4 with a wrapped column and
//                       clamped rows so the bilinear fetch needs no branches;
//   atlas_quad_kernel   bilinear footprints of the atlas (RGBO, SHADE mode)
//   / atlas_occ_quad_*  or occlusion alone (SHADOW mode reads only O);
//   dirs_kernel         local light directions (Hammersley in fp64 -> fp32);
//   shade_kernel        LANES threads per point split the S directions; per
//                       direction one octahedral encode (world-frame maps),
//                       4 texel fetches per probe from the L2-resident atlas,
//                       environment bilinear, BRDF, fp32 accumulation, and a
//                       shuffle reduction over the point's lanes.
#include <float.h>
#include <stdlib.h>

#include <mutex>

#include "scan.cuh"
#include "sop_device.cuh"
#include "sop_internal.h"

namespace sop {

QueryLayout query_layout(int32_t P, int64_t M, int32_t K, int32_t S, int32_t He, int32_t We, int32_t R,
                         int32_t rgbo_dtype)
{
    QueryLayout L{};
    int g = 1;
    while ((int64_t)g * g * g < P) ++g;
    L.g_axis = g;
    L.cells_cap = (g + 1) * (g + 1) * (g + 1);
    size_t o = 0;
    L.grid_hdr = o;   o = align256(o + sizeof(ProbeGrid));
    L.cell_start = o; o = align256(o + sizeof(int32_t) * (size_t)(L.cells_cap + 1));
    L.cell_cnt = o;   o = align256(o + sizeof(int32_t) * (size_t)L.cells_cap);
    L.entries = o;    o = align256(o + sizeof(int4) * (size_t)P);
    L.env4 = o;       o = align256(o + sizeof(float4) * (size_t)(He + 2) * (We + 1));
    L.envq = o;       o = align256(o + 64 * (size_t)(He + 1) * (We + 1));  // both layouts
    L.quads = o;      o = align256(o + (rgbo_dtype == SOP_F32 ? 64 : 32) * (size_t)P * (R + 1) * (R + 1));
    L.dirs = o;       o = align256(o + sizeof(float4) * (size_t)S);
    L.idx = o;        o = align256(o + sizeof(int32_t) * (size_t)M * K);
    L.w = o;          o = align256(o + sizeof(float) * (size_t)M * K);
    // adjoint only: points grouped by nearest probe, and the environment
    // gradient as float4 texels
    L.perm = o;       o = align256(o + sizeof(int32_t) * (size_t)M);
    L.bucket = o;     o = align256(o + sizeof(int32_t) * (size_t)(P + 1));
    L.genv4 = o;      o = align256(o + sizeof(float4) * (size_t)He * We);
    L.total = o;
    return L;
}

__device__ __forceinline__ int32_t quantise(float v) { return __float2int_rn(v * 1048576.0f); }

// Exact squared distance of two quantised points. Coordinates are below 2^30
// in magnitude (positions below 1024), so each difference fits 32 bits and
// each square is one 32x32 -> 64-bit multiply; the sum stays below 3 * 2^62.
__device__ __forceinline__ uint64_t qdist2(int32_t ax, int32_t ay, int32_t az, const int32_t q[3])
{
    const uint32_t dx = (uint32_t)abs(ax - q[0]), dy = (uint32_t)abs(ay - q[1]), dz = (uint32_t)abs(az - q[2]);
    return (uint64_t)dx * dx + (uint64_t)dy * dy + (uint64_t)dz * dz;
}

// Cubic cell edge (quantised units) for a box of extents ext[3]: the smallest
// edge whose grid, (ext/cs + 1) cells per axis, has at most `cap` cells. A
// flat site set (probes on a ground plane) then gets fine cells in its
// plane instead of the cbrt-per-axis split of a volume, which would put
// cbrt(P) sites in every cell of its one layer.
__device__ __forceinline__ int64_t grid_cell_edge(const int64_t ext[3], int64_t cap)
{
    int64_t emax = 0;
    for (int a = 0; a < 3; ++a) emax = ext[a] > emax ? ext[a] : emax;
    int64_t lo = 1, hi = emax + 1;  // hi: one cell per axis
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo) / 2;
        int64_t n = 1;
        for (int a = 0; a < 3 && n <= cap; ++a) n *= ext[a] / mid + 1;
        if (n <= cap) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// Probe grid (single CTA; P is small: thousands to ~1e5 probes).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) probe_grid_kernel(const float* __restrict__ probe_pos, int32_t P, int32_t g_axis,
                                                           ProbeGrid* grid, int32_t* cell_start, int32_t* cell_cnt,
                                                           int4* entries)
{
    __shared__ int32_t s_min[3], s_max[3];
    __shared__ int32_t s_part[1024];
    const int tid = threadIdx.x, nt = blockDim.x;
    if (tid < 3) {
        s_min[tid] = INT32_MAX;
        s_max[tid] = INT32_MIN;
    }
    __syncthreads();
    int32_t lmin[3] = {INT32_MAX, INT32_MAX, INT32_MAX}, lmax[3] = {INT32_MIN, INT32_MIN, INT32_MIN};
    for (int p = tid; p < P; p += nt)
        for (int a = 0; a < 3; ++a) {
            int32_t q = quantise(probe_pos[3 * p + a]);
            lmin[a] = min(lmin[a], q);
            lmax[a] = max(lmax[a], q);
        }
    for (int a = 0; a < 3; ++a) {
        atomicMin(&s_min[a], lmin[a]);
        atomicMax(&s_max[a], lmax[a]);
    }
    __syncthreads();
    // cell edge: the finest grid within (g+1)^3 cells, coarsened (cap
    // halved, at most 4 times) while there are fewer than 3 probes per
    // occupied cell. A volume-like set keeps the fine grid; a flat one (the
    // shadow probes on the ground), whose far query points need the K
    // nearest from a wide strip, gets cells of a few probes each.
    __shared__ ProbeGrid G;
    __shared__ int64_t s_cap;
    __shared__ int32_t s_occ;
    if (tid == 0) s_cap = (int64_t)(g_axis + 1) * (g_axis + 1) * (g_axis + 1);
    for (int it = 0;; ++it) {
        if (tid == 0) {
            int64_t ext[3];
            for (int a = 0; a < 3; ++a) ext[a] = (int64_t)s_max[a] - s_min[a];
            const int64_t cs = grid_cell_edge(ext, s_cap);
            G.cs = (int32_t)cs;
            int32_t nc = 1;
            for (int a = 0; a < 3; ++a) {
                G.qmin[a] = s_min[a];
                G.dims[a] = (int32_t)(ext[a] / cs) + 1;
                nc *= G.dims[a];
            }
            G.ncells = nc;
            s_occ = 0;
        }
        __syncthreads();
        for (int c = tid; c < G.ncells; c += nt) cell_cnt[c] = 0;
        __syncthreads();
        for (int p = tid; p < P; p += nt) {
            int c[3];
            for (int a = 0; a < 3; ++a) c[a] = (int)(((int64_t)quantise(probe_pos[3 * p + a]) - G.qmin[a]) / G.cs);
            if (atomicAdd(&cell_cnt[(c[2] * G.dims[1] + c[1]) * G.dims[0] + c[0]], 1) == 0) atomicAdd(&s_occ, 1);
        }
        __syncthreads();
        const bool again = it < 4 && (int64_t)P < 3 * (int64_t)s_occ && s_cap > 8;
        __syncthreads();
        if (!again) break;
        if (tid == 0) s_cap >>= 1;
    }
    if (tid == 0) *grid = G;
    const int nc = G.ncells;
    // exclusive scan of cell counts: contiguous chunk per thread + block scan
    const int chunk = (nc + nt - 1) / nt;
    const int c0 = tid * chunk, c1 = min(nc, c0 + chunk);
    int32_t sum = 0;
    for (int c = c0; c < c1; ++c) sum += cell_cnt[c];
    s_part[tid] = sum;
    __syncthreads();
    for (int off = 1; off < nt; off <<= 1) {
        int32_t v = (tid >= off) ? s_part[tid - off] : 0;
        __syncthreads();
        s_part[tid] += v;
        __syncthreads();
    }
    int32_t run = s_part[tid] - sum;
    for (int c = c0; c < c1; ++c) {
        int32_t v = cell_cnt[c];
        cell_start[c] = run;
        run += v;
        cell_cnt[c] = 0;
    }
    if (tid == nt - 1) cell_start[nc] = s_part[nt - 1];
    __syncthreads();
    for (int p = tid; p < P; p += nt) {
        int32_t q[3];
        int c[3];
        for (int a = 0; a < 3; ++a) {
            q[a] = quantise(probe_pos[3 * p + a]);
            c[a] = (int)(((int64_t)q[a] - G.qmin[a]) / G.cs);
        }
        int cell = (c[2] * G.dims[1] + c[1]) * G.dims[0] + c[0];
        int pos = cell_start[cell] + atomicAdd(&cell_cnt[cell], 1);
        entries[pos] = make_int4(q[0], q[1], q[2], p);
    }
}

// floor division for possibly negative numerators (positive divisor)
__device__ __forceinline__ int64_t floordiv(int64_t a, int64_t b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

// The search visits rings of cells (Chebyshev radius r in cell indices)
// around cc, the point's cell clamped into the grid. This is a lower bound on
// the squared quantised distance from the point q to every cell outside the
// cube of radius r: an unsearched cell lies in a slab beyond the cube along
// some axis b (below cc_b - r or above cc_b + r), at least d_b away along b,
// and, being inside the grid, at least out_a away along every other axis a
// (out_a: the point's distance outside the grid's extent on axis a; 0 for a
// point within it). The bound is the smallest d_b^2 + sum_{a != b} out_a^2
// over the slabs that hold cells; UINT64_MAX once the cube covers the grid.
// A site whose key is below it has been seen; sums that overflow 64 bits
// exceed every key and saturate.
__device__ __forceinline__ uint64_t unsearched_bound2(const ProbeGrid& G, const int32_t q[3], const int cc[3], int r)
{
    uint64_t out2[3], osum = 0;
    for (int a = 0; a < 3; ++a) {
        const int64_t lo = G.qmin[a], hi = lo + (int64_t)G.dims[a] * G.cs;
        const int64_t o = q[a] < lo ? lo - q[a] : (q[a] >= hi ? q[a] - hi + 1 : 0);
        out2[a] = (uint64_t)(o * o);
        osum += out2[a];
    }
    uint64_t best = UINT64_MAX;
    for (int b = 0; b < 3; ++b) {
        const uint64_t rest = osum - out2[b];
        // d^2 + rest, unless it exceeds 64 bits (then it bounds nothing)
        auto take = [&](uint64_t d) {
            if (__umul64hi(d, d) != 0) return;
            const uint64_t v = d * d + rest;
            if (v >= rest && v < best) best = v;
        };
        // cells of index <= cc_b - r - 1 end at qmin + (cc_b - r) cs
        if (cc[b] - r > 0) take((uint64_t)((int64_t)q[b] - (G.qmin[b] + (int64_t)(cc[b] - r) * G.cs)));
        // cells of index >= cc_b + r + 1 start at qmin + (cc_b + r + 1) cs
        if (cc[b] + r < G.dims[b] - 1) take((uint64_t)((G.qmin[b] + (int64_t)(cc[b] + r + 1) * G.cs) - (int64_t)q[b]));
    }
    return best;
}

// ---------------------------------------------------------------------------
// Exact K nearest probes + blend weights. One thread per point.
// ---------------------------------------------------------------------------
template <int KMAX>
__global__ void __launch_bounds__(128, KMAX <= 8 ? 8 : 1) knn_kernel(const float* __restrict__ x, const float* __restrict__ nrm, int64_t M,
                                                   int32_t K, uint64_t snap_key, uint64_t r2_key,
                                                   const ProbeGrid* __restrict__ gridp,
                                                   const int32_t* __restrict__ cell_start,
                                                   const int4* __restrict__ entries,
                                                   const float* __restrict__ probe_pos, int32_t* __restrict__ ws_idx,
                                                   float* __restrict__ ws_w, int32_t* __restrict__ user_idx,
                                                   float* __restrict__ user_w, unsigned int* status)
{
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    const ProbeGrid G = *gridp;
    float3 xp = load3(x, m);
    {
        // a non-finite position or normal is reported; the position is then
        // taken as the origin so that the search stays defined
        const float3 nr0 = load3(nrm, m);
        const bool okx = isfinite(xp.x + xp.y + xp.z);
        if ((!okx || !isfinite(nr0.x + nr0.y + nr0.z)) && status) atomicOr(status, SOP_DEVSTAT_NONFINITE);
        if (!okx) xp = f3(0.f, 0.f, 0.f);
    }
    const int32_t q[3] = {quantise(xp.x), quantise(xp.y), quantise(xp.z)};
    // rings are taken around the point's cell clamped into the grid
    int c[3];
    for (int a = 0; a < 3; ++a) {
        const int64_t ca = floordiv((int64_t)q[a] - G.qmin[a], G.cs);
        c[a] = (int)(ca < 0 ? 0 : (ca > G.dims[a] - 1 ? G.dims[a] - 1 : ca));
    }
    uint64_t bk[KMAX];
    int32_t bi[KMAX];
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
        bk[k] = UINT64_MAX;
        bi[k] = INT32_MAX;
    }
    for (int r = 0;; ++r) {
        const int zlo = max(c[2] - r, 0), zhi = min(c[2] + r, G.dims[2] - 1);
        const int ylo = max(c[1] - r, 0), yhi = min(c[1] + r, G.dims[1] - 1);
        for (int z = zlo; z <= zhi; ++z)
            for (int y = ylo; y <= yhi; ++y) {
                const bool face = (z == c[2] - r) || (z == c[2] + r) || (y == c[1] - r) || (y == c[1] + r);
                const int xs = face ? 1 : 2 * r;  // on a face row: every x; else only the two ends
                for (int xx = c[0] - r; xx <= c[0] + r; xx += (xs > 0 ? xs : 1)) {
                    if (xx < 0 || xx >= G.dims[0]) continue;
                    const int cell = (z * G.dims[1] + y) * G.dims[0] + xx;
                    const int e1 = __ldg(cell_start + cell + 1);
#pragma unroll 2
                    for (int e = __ldg(cell_start + cell); e < e1; ++e) {
                        const int4 en = __ldg(entries + e);
                        const uint64_t key = qdist2(en.x, en.y, en.z, q);
                        const int32_t id = en.w;
                        // keep the KMAX best (key, id) pairs within the radius
                        // sorted; the first K of them are the K nearest
                        const bool better = key <= r2_key &&
                                            (key < bk[KMAX - 1] || (key == bk[KMAX - 1] && id < bi[KMAX - 1]));
                        if (!better) continue;
                        // insert: every kept pair above the new one moves up a slot
                        bool lt[KMAX];
#pragma unroll
                        for (int k = 0; k < KMAX; ++k) lt[k] = key < bk[k] || (key == bk[k] && id < bi[k]);
#pragma unroll
                        for (int k = KMAX - 1; k > 0; --k) {
                            bk[k] = lt[k - 1] ? bk[k - 1] : (lt[k] ? key : bk[k]);
                            bi[k] = lt[k - 1] ? bi[k - 1] : (lt[k] ? id : bi[k]);
                        }
                        bk[0] = lt[0] ? key : bk[0];
                        bi[0] = lt[0] ? id : bi[0];
                    }
                }
            }
        // stop once no probe outside ring r can enter the best K, nor lie
        // within the radius
        // the K-th best key as a chain of selects: picking bk[K - 1] by the
        // run-time K would put bk in local memory
        uint64_t kth = bk[0];
#pragma unroll
        for (int k = 1; k < KMAX; ++k) kth = k < K ? bk[k] : kth;
        const uint64_t bnd = unsearched_bound2(G, q, c, r);
        if (bnd == UINT64_MAX || kth < bnd || r2_key < bnd) break;
    }
    // weights (Eq. 4-6)
    const float3 nr = load3(nrm, m);
    const float nl = sqrtf(dot3(nr, nr));
    const float3 nn = f3(nr.x / nl, nr.y / nl, nr.z / nl);
    float w[KMAX];
    float wsum = 0.f;
    // slots a radius search left empty keep bi = INT32_MAX: weight 0, and the
    // shading reads (with weight 0) the nearest probe found, or probe 0
    const bool snap = bi[0] != INT32_MAX && bk[0] <= snap_key;
    const int32_t fill = bi[0] != INT32_MAX ? bi[0] : 0;
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
        w[k] = 0.f;
        if (k < K && bi[k] != INT32_MAX) {
            const float3 pk = load3(probe_pos, bi[k]);
            const float3 d = pk - xp;
            const float dl = sqrtf(dot3(d, d));
            const float ws = 1.f / dl;
            const float wb = 0.5f * (1.f + dot3(d, nn) / dl) + 0.01f;
            w[k] = snap ? (k == 0 ? 1.f : 0.f) : ws * wb;
            wsum += w[k];
        }
    }
#pragma unroll
    for (int k = 0; k < KMAX; ++k)
        if (k < K) {
            const bool found = bi[k] != INT32_MAX;
            const float wk = (snap || !found) ? w[k] : w[k] / wsum;
            ws_idx[m * K + k] = found ? bi[k] : fill;
            ws_w[m * K + k] = wk;
            if (user_idx) user_idx[m * K + k] = found ? bi[k] : -1;
            if (user_w) user_w[m * K + k] = wk;
        }
}

// ---------------------------------------------------------------------------
// Environment table: float4 [(He+2)][(We+1)], stored row r+1 = row r (rows 0
// and He+1 repeat the first and last row: v clamps), stored column We =
// column 0 (u wraps).
// ---------------------------------------------------------------------------
__global__ void env_pack_kernel(const float* __restrict__ env, int32_t He, int32_t We, float4* __restrict__ env4,
                                unsigned int* status)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t n = (int64_t)(He + 2) * (We + 1);
    if (i >= n) return;
    const int rs = (int)(i / (We + 1)), cs = (int)(i % (We + 1));
    const int r = min(max(rs - 1, 0), He - 1), c = cs == We ? 0 : cs;
    const float* e = env + ((int64_t)r * We + c) * 3;
    if (!isfinite(e[0] + e[1] + e[2]) && status) atomicOr(status, SOP_DEVSTAT_NONFINITE);
    env4[i] = make_float4(e[0], e[1], e[2], 0.f);
}

// Environment footprints: for base (r0, c0), r0 in [0, He], c0 in [0, We),
// the 2x2 bilinear footprint of the padded table, RGB x 4 = 12 floats in a
// 64-byte slot: (e00, e01, e10, e11) with e01 = column c0+1, e10 = row r0+1.
__global__ void env_quad_kernel(const float4* __restrict__ env4, int32_t He, int32_t We, float4* __restrict__ envq)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)(He + 1) * We) return;
    const int r0 = (int)(i / We), c0 = (int)(i % We);
    const float4* p = env4 + (int64_t)r0 * (We + 1) + c0;
    const float4 a = p[0], b = p[1], c = p[We + 1], d = p[We + 2];
    float4* q = envq + 4 * i;
    q[0] = make_float4(a.x, a.y, a.z, b.x);
    q[1] = make_float4(b.y, b.z, c.x, c.y);
    q[2] = make_float4(c.z, d.x, d.y, d.z);
    q[3] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// Octahedral environment footprints (Sec. 4.1 layout, [H][H][3]): for base
// (a, b) in [0, H]^2, the texels (a-1+di, b-1+dj), di, dj in {0, 1}, through
// the probe maps' border rule, in the 64-byte slot format of env_quad_kernel
// (e00, e01 = next column, e10 = next row, e11).
__global__ void env_oct_quad_kernel(const float* __restrict__ env, int32_t H, float4* __restrict__ envq,
                                    unsigned int* status)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int HQ = H + 1;
    if (k >= (int64_t)HQ * HQ) return;
    const int b = (int)(k / HQ), a = (int)(k % HQ);
    float3 e[4];
    for (int q = 0; q < 4; ++q) {
        int si, sj;
        oct_wrap(H, a - 1 + (q & 1), b - 1 + (q >> 1), si, sj);
        const float* t = env + ((int64_t)sj * H + si) * 3;
        e[q] = f3(t[0], t[1], t[2]);
    }
    if (!isfinite(e[0].x + e[0].y + e[0].z) && status) atomicOr(status, SOP_DEVSTAT_NONFINITE);
    float4* o = envq + 4 * k;
    o[0] = make_float4(e[0].x, e[0].y, e[0].z, e[1].x);
    o[1] = make_float4(e[1].y, e[1].z, e[2].x, e[2].y);
    o[2] = make_float4(e[2].z, e[3].x, e[3].y, e[3].z);
    o[3] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// Atlas footprints: for probe p and base (a, b) in [0, R]^2 of the stored
// (gutter) map, the texels (a,b), (a+1,b), (a,b+1), (a+1,b+1) stored
// contiguously, so one bilinear fetch reads one aligned 32/64-byte block.
template <int DT>
__global__ void atlas_quad_kernel(const typename Texel<DT>::raw* __restrict__ atlas, int32_t P, int32_t R,
                                  typename Texel<DT>::raw* __restrict__ quads, unsigned int* status)
{
    const int RS = R + 2, RQ = R + 1;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)P * RQ * RQ) return;
    const int64_t pr = i / (RQ * RQ);
    const int r = (int)(i % (RQ * RQ));
    const int b = r / RQ, a = r % RQ;
    const typename Texel<DT>::raw* src = atlas + pr * RS * RS + (int64_t)b * RS + a;
    typename Texel<DT>::raw* dst = quads + 4 * i;
    // every interior texel is the first texel of one footprint
    if (!Texel<DT>::finite(src[0]) && status) atomicOr(status, SOP_DEVSTAT_NONFINITE);
    dst[0] = src[0];
    dst[1] = src[1];
    dst[2] = src[RS];
    dst[3] = src[RS + 1];
}

// Occlusion footprints for SHADOW mode, which reads only O (Eq. 8): the
// four O values of each footprint, as float4 (float32 atlas) or four
// 16-bit values in 8 bytes, so one probe fetch is one 128/64-bit load.
__global__ void atlas_occ_quad_f32_kernel(const float4* __restrict__ atlas, int32_t P, int32_t R,
                                          float4* __restrict__ quads, unsigned int* status)
{
    const int RS = R + 2, RQ = R + 1;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)P * RQ * RQ) return;
    const int64_t pr = i / (RQ * RQ);
    const int r = (int)(i % (RQ * RQ));
    const int b = r / RQ, a = r % RQ;
    const float4* src = atlas + pr * RS * RS + (int64_t)b * RS + a;
    if (!isfinite(src[0].w) && status) atomicOr(status, SOP_DEVSTAT_NONFINITE);
    quads[i] = make_float4(src[0].w, src[1].w, src[RS].w, src[RS + 1].w);
}

// 16-bit texels (R, G, B, O): O is the upper half of the second word.
template <int DT>
__global__ void atlas_occ_quad_16_kernel(const uint2* __restrict__ atlas, int32_t P, int32_t R,
                                         uint2* __restrict__ quads, unsigned int* status)
{
    const int RS = R + 2, RQ = R + 1;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)P * RQ * RQ) return;
    const int64_t pr = i / (RQ * RQ);
    const int r = (int)(i % (RQ * RQ));
    const int b = r / RQ, a = r % RQ;
    const uint2* src = atlas + pr * RS * RS + (int64_t)b * RS + a;
    if (!Texel<DT>::finite(src[0]) && status) atomicOr(status, SOP_DEVSTAT_NONFINITE);
    quads[i] = make_uint2((src[0].y >> 16) | (src[1].y & 0xffff0000u), (src[RS].y >> 16) | (src[RS + 1].y & 0xffff0000u));
}

__device__ __forceinline__ double radical_inverse2(uint32_t i) { return (double)__brev(i) * 2.3283064365386963e-10; }

// Local light directions: the caller's set, or the centred Hammersley set.
__global__ void dirs_kernel(int32_t S, const float* __restrict__ dirs_local, float4* __restrict__ out4,
                            float* __restrict__ out3)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= S) return;
    float3 d;
    if (dirs_local) {
        d = load3(dirs_local, i);
    } else {
        const double z = (i + 0.5) / S;
        const double phi = 6.283185307179586476925 * radical_inverse2((uint32_t)i);
        const double s = sqrt(1.0 - z * z);
        d = f3((float)(s * cos(phi)), (float)(s * sin(phi)), (float)z);
    }
    if (out4) out4[i] = make_float4(d.x, d.y, d.z, 0.f);
    if (out3) {
        out3[3 * i] = d.x;
        out3[3 * i + 1] = d.y;
        out3[3 * i + 2] = d.z;
    }
}

// Importance-sampled world directions (x, y, z, pdf) -> (x, y, z, 1/pdf).
__global__ void world_dirs_kernel(int32_t S, const float4* __restrict__ dirs_world, float4* __restrict__ out4)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= S) return;
    const float4 d = dirs_world[i];
    out4[i] = make_float4(d.x, d.y, d.z, 1.f / d.w);
}

// 256-bit read-only global load (sm_100+); p must be 32-byte aligned.
__device__ __forceinline__ void ldg256(const void* p, uint64_t& a, uint64_t& b, uint64_t& c, uint64_t& d)
{
    asm("ld.global.nc.v4.b64 {%0, %1, %2, %3}, [%4];"
        : "=l"(a), "=l"(b), "=l"(c), "=l"(d)
        : "l"(p));
}
__device__ __forceinline__ float lo32f(uint64_t v) { return __uint_as_float((uint32_t)v); }
__device__ __forceinline__ float hi32f(uint64_t v) { return __uint_as_float((uint32_t)(v >> 32)); }

// Bilinear environment lookup L_dir(w) (z-up equirectangular) from the
// footprint table: three 16-byte loads of one 64-byte slot.
__device__ __forceinline__ float3 env_lookup(const float4* __restrict__ envq, int He, int We, float3 w)
{
    const float th = atan2f(sqrtf(w.x * w.x + w.y * w.y), w.z);
    const float ph = atan2f(w.y, w.x);
    const float s = (ph + kPi) * kInv2Pi * We - 0.5f;
    const float t = th * kInvPi * He - 0.5f;
    const float fs = floorf(s), ft = floorf(t);
    const float a = s - fs, b = t - ft;
    int c0 = (int)fs;
    c0 = c0 < 0 ? c0 + We : c0;
    c0 = min(max(c0, 0), We - 1);
    const int r0 = min(max((int)ft + 1, 0), He);
    const float4* q = envq + 4 * ((int64_t)r0 * We + c0);
    uint64_t x0, x1, x2, x3;
    ldg256(q, x0, x1, x2, x3);
    const float4 q0 = make_float4(lo32f(x0), hi32f(x0), lo32f(x1), hi32f(x1));
    const float4 q1 = make_float4(lo32f(x2), hi32f(x2), lo32f(x3), hi32f(x3));
    const float4 q2 = __ldg(q + 2);
    const float w00 = (1.f - a) * (1.f - b), w01 = a * (1.f - b), w10 = (1.f - a) * b, w11 = a * b;
    return f3(w00 * q0.x + w01 * q0.w + w10 * q1.z + w11 * q2.y, w00 * q0.y + w01 * q1.x + w10 * q1.w + w11 * q2.z,
              w00 * q0.z + w01 * q1.y + w10 * q2.x + w11 * q2.w);
}

// Bilinear lookup of an octahedral environment (Sec. 4.1) at the octahedral
// coordinates uv of the direction (the probe maps' mapping: no atan2), from
// the footprint table of env_oct_quad_kernel.
__device__ __forceinline__ float3 env_oct_lookup(const float4* __restrict__ envq, int H, float2 uv)
{
    const float s = uv.x * H - 0.5f, t = uv.y * H - 0.5f;
    const float fs = floorf(s), ft = floorf(t);
    const float a = s - fs, b = t - ft;
    const int c0 = min(max((int)fs + 1, 0), H), r0 = min(max((int)ft + 1, 0), H);
    const float4* q = envq + 4 * ((int64_t)r0 * (H + 1) + c0);
    uint64_t x0, x1, x2, x3;
    ldg256(q, x0, x1, x2, x3);
    const float4 q0 = make_float4(lo32f(x0), hi32f(x0), lo32f(x1), hi32f(x1));
    const float4 q1 = make_float4(lo32f(x2), hi32f(x2), lo32f(x3), hi32f(x3));
    const float4 q2 = __ldg(q + 2);
    const float w00 = (1.f - a) * (1.f - b), w01 = a * (1.f - b), w10 = (1.f - a) * b, w11 = a * b;
    return f3(w00 * q0.x + w01 * q0.w + w10 * q1.z + w11 * q2.y, w00 * q0.y + w01 * q1.x + w10 * q1.w + w11 * q2.z,
              w00 * q0.z + w01 * q1.y + w10 * q2.x + w11 * q2.w);
}

// One bilinear footprint of the atlas: four texels as float4 (RGB, O).
template <int DT> struct Quad;
template <> struct Quad<SOP_F32> {
    static __device__ __forceinline__ void load(const void* base, int64_t qi, float4& t00, float4& t10, float4& t01,
                                                float4& t11)
    {
        const float4* p = reinterpret_cast<const float4*>(base) + 4 * qi;
        uint64_t a, b, c, d, e, f, g, h;
        ldg256(p, a, b, c, d);
        ldg256(p + 2, e, f, g, h);
        t00 = make_float4(lo32f(a), hi32f(a), lo32f(b), hi32f(b));
        t10 = make_float4(lo32f(c), hi32f(c), lo32f(d), hi32f(d));
        t01 = make_float4(lo32f(e), hi32f(e), lo32f(f), hi32f(f));
        t11 = make_float4(lo32f(g), hi32f(g), lo32f(h), hi32f(h));
    }
};
__device__ __forceinline__ float4 h4(uint32_t x, uint32_t y)
{
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&y));
    return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ float4 b4(uint32_t x, uint32_t y)
{
    return make_float4(__uint_as_float(x << 16), __uint_as_float(x & 0xffff0000u), __uint_as_float(y << 16),
                       __uint_as_float(y & 0xffff0000u));
}
template <> struct Quad<SOP_F16> {
    static __device__ __forceinline__ void load(const void* base, int64_t qi, float4& t00, float4& t10, float4& t01,
                                                float4& t11)
    {
        uint64_t a, b, c, d;
        ldg256(reinterpret_cast<const uint4*>(base) + 2 * qi, a, b, c, d);
        t00 = h4((uint32_t)a, (uint32_t)(a >> 32));
        t10 = h4((uint32_t)b, (uint32_t)(b >> 32));
        t01 = h4((uint32_t)c, (uint32_t)(c >> 32));
        t11 = h4((uint32_t)d, (uint32_t)(d >> 32));
    }
};
template <> struct Quad<SOP_BF16> {
    static __device__ __forceinline__ void load(const void* base, int64_t qi, float4& t00, float4& t10, float4& t01,
                                                float4& t11)
    {
        uint64_t a, b, c, d;
        ldg256(reinterpret_cast<const uint4*>(base) + 2 * qi, a, b, c, d);
        t00 = b4((uint32_t)a, (uint32_t)(a >> 32));
        t10 = b4((uint32_t)b, (uint32_t)(b >> 32));
        t01 = b4((uint32_t)c, (uint32_t)(c >> 32));
        t11 = b4((uint32_t)d, (uint32_t)(d >> 32));
    }
};

// One occlusion footprint: O at (a,b), (a+1,b), (a,b+1), (a+1,b+1).
template <int DT> struct OQuad;
template <> struct OQuad<SOP_F32> {
    static __device__ __forceinline__ float4 load(const void* base, int64_t qi)
    {
        return __ldg(reinterpret_cast<const float4*>(base) + qi);
    }
};
template <> struct OQuad<SOP_F16> {
    static __device__ __forceinline__ float4 load(const void* base, int64_t qi)
    {
        const uint2 v = __ldg(reinterpret_cast<const uint2*>(base) + qi);
        return h4(v.x, v.y);
    }
};
template <> struct OQuad<SOP_BF16> {
    static __device__ __forceinline__ float4 load(const void* base, int64_t qi)
    {
        const uint2 v = __ldg(reinterpret_cast<const uint2*>(base) + qi);
        return b4(v.x, v.y);
    }
};

// Geometry of one light direction at a point: the world direction (local
// direction l rotated into the frame (t, b, n)), its octahedral footprint
// (offset of the base texel in a probe's stored map) and bilinear weights.
struct DirTerms {
    float3 w;
    float2 uv;
    int off;
    float w00, w10, w01, w11;
};
// footprint part for a world direction w
__device__ __forceinline__ DirTerms footprint_terms(const float3 w, const float Rf, const int R, const int RQ)
{
    DirTerms d;
    d.w = w;
    const float2 uv = oct_encode(d.w);
    d.uv = uv;
    const float s = uv.x * Rf - 0.5f, t = uv.y * Rf - 0.5f;
    const float fi = floorf(s), fj = floorf(t);
    const float fu = s - fi, fv = t - fj;
    const int i0 = min(max((int)fi + 1, 0), R), j0 = min(max((int)fj + 1, 0), R);
    d.off = j0 * RQ + i0;
    d.w00 = (1.f - fu) * (1.f - fv);
    d.w10 = fu * (1.f - fv);
    d.w01 = (1.f - fu) * fv;
    d.w11 = fu * fv;
    return d;
}

__device__ __forceinline__ DirTerms dir_terms(const float4 l, const float3 tt, const float3 bb, const float3 n,
                                              const float Rf, const int R, const int RQ)
{
    return footprint_terms(f3(fmaf(l.x, tt.x, fmaf(l.y, bb.x, l.z * n.x)), fmaf(l.x, tt.y, fmaf(l.y, bb.y, l.z * n.y)),
                              fmaf(l.x, tt.z, fmaf(l.y, bb.z, l.z * n.z))),
                           Rf, R, RQ);
}

// Blended occlusion of one direction over a point's K probes (Eq. 5, applied
// to O): each footprint corner is blended over the probes, then the four
// corners are weighted once, O = sum_c w_c sum_k W_k O_k,c.
template <int DT, int KMAX>
__device__ __forceinline__ float shadow_blend(const void* quads, const int32_t* base, const float* W, const int K,
                                              const int off, const float w00, const float w10, const float w01,
                                              const float w11)
{
    float s00 = 0.f, s10 = 0.f, s01 = 0.f, s11 = 0.f;
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
        if (k < K) {
            const float4 q = OQuad<DT>::load(quads, (int64_t)(base[k] + off));
            s00 = fmaf(W[k], q.x, s00);
            s10 = fmaf(W[k], q.y, s10);
            s01 = fmaf(W[k], q.z, s01);
            s11 = fmaf(W[k], q.w, s11);
        }
    }
    return fmaf(w00, s00, fmaf(w10, s10, fmaf(w01, s01, w11 * s11)));
}

// SHADOW-mode warps whose points share a normal keep per-direction terms in
// shared memory (32 bytes a direction per warp) for S up to this
constexpr int kShadowTab = 128;

struct ShadeK {
    const float *n, *wo, *albedo, *rough, *metal;
    int64_t M;
    const void* rgbo;
    int32_t R, K, S, He, We;
    const float4* envq;
    int32_t env_layout;
    const void* quads;
    const float4* dirs;
    const int32_t* idx;
    const float* w;
    float specular;
    float* out;
    unsigned int* status;  // device status word or NULL
};

// ---------------------------------------------------------------------------
// Query + shade. LANES consecutive threads share one point and split its S
// directions; one warp covers 32/LANES points.
// ---------------------------------------------------------------------------
template <int DT, int KMAX, int MODE>
__global__ void __launch_bounds__(256, 4) shade_kernel(const ShadeK a, const int LANES)
{
    extern __shared__ float4 s_dirs[];
    for (int i = threadIdx.x; i < a.S; i += blockDim.x) s_dirs[i] = a.dirs[i];
    __syncthreads();
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t m = gid / LANES;
    const int sub = (int)(gid % LANES);
    const bool active = m < a.M;
    const int64_t mm = active ? m : 0;

    const float3 nr = load3(a.n, mm);
    const float nl = sqrtf(dot3(nr, nr));
    const float3 n = f3(nr.x / nl, nr.y / nl, nr.z / nl);
    float3 tt, bb;
    onb(n, tt, bb);
    const float3 wo = load3(a.wo, mm);
    const int RQ = a.R + 1;
    int32_t base[KMAX];
    float W[KMAX];
    int32_t ids[KMAX];
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
        const bool on = k < a.K;
        ids[k] = on ? __ldg(a.idx + mm * a.K + k) : INT32_MAX;
        W[k] = on ? __ldg(a.w + mm * a.K + k) : 0.f;
    }
    // visit the probes in index order: neighbouring points, which share most
    // of their probes, then read the same footprints at the same time
    if (KMAX <= 8)
#pragma unroll
    for (int i = 1; i < KMAX; ++i)
#pragma unroll
        for (int j = KMAX - 1; j >= i; --j) {
            const bool sw = ids[j - 1] > ids[j];
            const int32_t ti = ids[j - 1];
            const float tw = W[j - 1];
            ids[j - 1] = sw ? ids[j] : ids[j - 1];
            W[j - 1] = sw ? W[j] : W[j - 1];
            ids[j] = sw ? ti : ids[j];
            W[j] = sw ? tw : W[j];
        }
#pragma unroll
    for (int k = 0; k < KMAX; ++k) base[k] = (k < a.K) ? ids[k] * RQ * RQ : 0;
    // per-point BRDF constants
    float3 kd, F0;
    float a2 = 0.f, kk = 0.f, specV = 0.f, NdotV = 1.f;
    if (MODE == SOP_MODE_SHADE) {
        const float3 alb = load3(a.albedo, mm);
        const float r = __ldg(a.rough + mm), mt = __ldg(a.metal + mm);
        if (a.status && active && sub == 0 && !isfinite(alb.x + alb.y + alb.z + r + mt + wo.x + wo.y + wo.z))
            atomicOr(a.status, SOP_DEVSTAT_NONFINITE);
        const float dsc = (1.f - mt) * kInvPi;
        kd = f3(dsc * alb.x, dsc * alb.y, dsc * alb.z);
        const float f0d = 0.08f * a.specular * (1.f - mt);
        F0 = f3(f0d + alb.x * mt, f0d + alb.y * mt, f0d + alb.z * mt);
        const float al = r * r;
        a2 = al * al;
        kk = (r + 1.f) * (r + 1.f) * 0.125f;
        NdotV = fmaxf(dot3(n, wo), 1e-4f);
        const float G1V = NdotV / (NdotV * (1.f - kk) + kk);
        specV = G1V / (4.f * NdotV);
    }
    float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f, den0 = 0.f, den1 = 0.f, den2 = 0.f;
    const float Rf = (float)a.R;
    // SHADOW mode, every point of the warp on the same normal (bit for bit; a
    // planar receiver such as a ground plane): their light directions, and so
    // the footprint offsets, bilinear weights and environment terms of every
    // direction, coincide (Eq. 3 rotates one local set by the normal's frame).
    // The lanes then compute those once for the warp into shared memory, and
    // each point only gathers and blends its own probes.
    bool warp_dirs = false;
    if (MODE == SOP_MODE_SHADOW && a.S <= kShadowTab) {
        const unsigned full = 0xffffffffu;
        const unsigned bx = __float_as_uint(nr.x), by = __float_as_uint(nr.y), bz = __float_as_uint(nr.z);
        // every lane takes all three shuffles (no short-circuit: a lane that
        // skipped one would leave the others waiting at it)
        const unsigned x0 = __shfl_sync(full, bx, 0), y0 = __shfl_sync(full, by, 0), z0 = __shfl_sync(full, bz, 0);
        const bool same = (bx == x0) & (by == y0) & (bz == z0);
        warp_dirs = __all_sync(full, same);
    }
    if (MODE == SOP_MODE_SHADOW && warp_dirs) {
        float4* tab = s_dirs + a.S + (threadIdx.x >> 5) * 2 * a.S;
        for (int i = (int)(threadIdx.x & 31); i < a.S; i += 32) {
            const float4 l = s_dirs[i];
            const DirTerms d = dir_terms(l, tt, bb, n, Rf, a.R, RQ);
            const float3 Ld = a.env_layout == SOP_ENV_OCTAHEDRAL ? env_oct_lookup(a.envq, a.He, d.uv)
                                                                 : env_lookup(a.envq, a.He, a.We, d.w);
            const float NdotL = l.z;
            tab[i] = make_float4(__int_as_float(d.off), d.w00, d.w10, d.w01);
            tab[a.S + i] = make_float4(d.w11, Ld.x * NdotL, Ld.y * NdotL, Ld.z * NdotL);
        }
        __syncwarp();
        for (int i = sub; i < a.S; i += LANES) {
            const float4 ta = tab[i], tb = tab[a.S + i];
            const float vis =
                1.f - shadow_blend<DT, KMAX>(a.quads, base, W, a.K, __float_as_int(ta.x), ta.y, ta.z, ta.w, tb.x);
            acc0 = fmaf(tb.y, vis, acc0);
            acc1 = fmaf(tb.z, vis, acc1);
            acc2 = fmaf(tb.w, vis, acc2);
            den0 += tb.y;
            den1 += tb.z;
            den2 += tb.w;
        }
    } else
    for (int i = sub; i < a.S; i += LANES) {
        const float4 l = s_dirs[i];
        const DirTerms d = dir_terms(l, tt, bb, n, Rf, a.R, RQ);
        const float3 w = d.w;
        const int off = d.off;
        const float w00 = d.w00, w10 = d.w10, w01 = d.w01, w11 = d.w11;
        float4 pr = make_float4(0.f, 0.f, 0.f, 0.f);
        if (MODE == SOP_MODE_SHADOW) {
            pr.w = shadow_blend<DT, KMAX>(a.quads, base, W, a.K, off, w00, w10, w01, w11);
        } else
#pragma unroll
        for (int k = 0; k < KMAX; ++k) {
            if (k < a.K) {
                float4 t00, t10, t01, t11;
                Quad<DT>::load(a.quads, (int64_t)(base[k] + off), t00, t10, t01, t11);
                const float c00 = W[k] * w00, c10 = W[k] * w10, c01 = W[k] * w01, c11 = W[k] * w11;
                pr.x += c00 * t00.x + c10 * t10.x + c01 * t01.x + c11 * t11.x;
                pr.y += c00 * t00.y + c10 * t10.y + c01 * t01.y + c11 * t11.y;
                pr.z += c00 * t00.z + c10 * t10.z + c01 * t01.z + c11 * t11.z;
                pr.w += c00 * t00.w + c10 * t10.w + c01 * t01.w + c11 * t11.w;
            }
        }
        const float3 Ld = a.env_layout == SOP_ENV_OCTAHEDRAL ? env_oct_lookup(a.envq, a.He, d.uv)
                                                             : env_lookup(a.envq, a.He, a.We, w);
        const float NdotL = l.z;
        const float vis = 1.f - pr.w;
        if (MODE == SOP_MODE_SHADE) {
            float3 h = w + wo;
            const float hl2 = dot3(h, h);
            h = hl2 > 1e-30f ? rsqrtf(hl2) * h : n;
            const float NdotH = dot3(n, h), VdotH = dot3(wo, h);
            const float3 cr = cross3(n, h);
            const float sin2 = dot3(cr, cr);
            const float den = NdotH * NdotH * a2 + sin2;
            const float D = __fdividef(a2, kPi * den * den);
            const float spec = __fdividef(D * specV, NdotL * (1.f - kk) + kk);
            const float x1 = 1.f - VdotH, x2 = x1 * x1, fc = x2 * x2 * x1;
            const float f0 = kd.x + spec * (F0.x + (1.f - F0.x) * fc);
            const float f1 = kd.y + spec * (F0.y + (1.f - F0.y) * fc);
            const float f2 = kd.z + spec * (F0.z + (1.f - F0.z) * fc);
            acc0 += f0 * (vis * Ld.x + pr.x) * NdotL;
            acc1 += f1 * (vis * Ld.y + pr.y) * NdotL;
            acc2 += f2 * (vis * Ld.z + pr.z) * NdotL;
        } else {
            // the same terms, in the same order, as the shared-direction path
            const float L0 = Ld.x * NdotL, L1 = Ld.y * NdotL, L2 = Ld.z * NdotL;
            acc0 = fmaf(L0, vis, acc0);
            acc1 = fmaf(L1, vis, acc1);
            acc2 = fmaf(L2, vis, acc2);
            den0 += L0;
            den1 += L1;
            den2 += L2;
        }
    }
    for (int o = LANES / 2; o > 0; o >>= 1) {
        acc0 += __shfl_xor_sync(0xffffffffu, acc0, o);
        acc1 += __shfl_xor_sync(0xffffffffu, acc1, o);
        acc2 += __shfl_xor_sync(0xffffffffu, acc2, o);
        if (MODE == SOP_MODE_SHADOW) {
            den0 += __shfl_xor_sync(0xffffffffu, den0, o);
            den1 += __shfl_xor_sync(0xffffffffu, den1, o);
            den2 += __shfl_xor_sync(0xffffffffu, den2, o);
        }
    }
    if (active && sub == 0) {
        float* o = a.out + 3 * m;
        if (MODE == SOP_MODE_SHADE) {
            const float sc = 2.f * kPi / (float)a.S;
            o[0] = sc * acc0;
            o[1] = sc * acc1;
            o[2] = sc * acc2;
        } else {
            o[0] = den0 < 1e-20f ? 1.f : acc0 / den0;
            o[1] = den1 < 1e-20f ? 1.f : acc1 / den1;
            o[2] = den2 < 1e-20f ? 1.f : acc2 / den2;
        }
    }
}

// ---------------------------------------------------------------------------
// Query + shade over importance-sampled world directions (Sec. 4.2): the S
// directions, their octahedral footprints, bilinear weights, environment
// radiance and 1/pdf are the same for every point, so each CTA tabulates
// them once in shared memory (48 bytes a direction). Per point and direction
// there remain the horizon test, the gather of the K probe footprints and,
// in SHADE mode, the BRDF; terms are weighted by 1/pdf and the estimate is
// their sum over the directions above the horizon, divided by S.
// ---------------------------------------------------------------------------
template <int DT, int KMAX, int MODE>
__global__ void __launch_bounds__(256, 4) shade_world_kernel(const ShadeK a, const int LANES)
{
    extern __shared__ float4 s_tab[];  // [S][3]: (w, 1/pdf), (L_dir, off), (w00, w10, w01, w11)
    const float Rf = (float)a.R;
    const int RQ = a.R + 1;
    for (int i = threadIdx.x; i < a.S; i += blockDim.x) {
        const float4 l = a.dirs[i];
        const float3 w = f3(l.x, l.y, l.z);
        const DirTerms d = footprint_terms(w, Rf, a.R, RQ);
        const float3 Ld = a.env_layout == SOP_ENV_OCTAHEDRAL ? env_oct_lookup(a.envq, a.He, d.uv)
                                                             : env_lookup(a.envq, a.He, a.We, w);
        s_tab[3 * i] = l;
        s_tab[3 * i + 1] = make_float4(Ld.x, Ld.y, Ld.z, __int_as_float(d.off));
        s_tab[3 * i + 2] = make_float4(d.w00, d.w10, d.w01, d.w11);
    }
    __syncthreads();
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t m = gid / LANES;
    const int sub = (int)(gid % LANES);
    const bool active = m < a.M;
    const int64_t mm = active ? m : 0;
    const float3 nr = load3(a.n, mm);
    const float nl = sqrtf(dot3(nr, nr));
    const float3 n = f3(nr.x / nl, nr.y / nl, nr.z / nl);
    const float3 wo = load3(a.wo, mm);
    int32_t base[KMAX];
    float W[KMAX];
    int32_t ids[KMAX];
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
        const bool on = k < a.K;
        ids[k] = on ? __ldg(a.idx + mm * a.K + k) : INT32_MAX;
        W[k] = on ? __ldg(a.w + mm * a.K + k) : 0.f;
    }
    if (KMAX <= 8)
#pragma unroll
    for (int i = 1; i < KMAX; ++i)
#pragma unroll
        for (int j = KMAX - 1; j >= i; --j) {
            const bool sw = ids[j - 1] > ids[j];
            const int32_t ti = ids[j - 1];
            const float tw = W[j - 1];
            ids[j - 1] = sw ? ids[j] : ids[j - 1];
            W[j - 1] = sw ? W[j] : W[j - 1];
            ids[j] = sw ? ti : ids[j];
            W[j] = sw ? tw : W[j];
        }
#pragma unroll
    for (int k = 0; k < KMAX; ++k) base[k] = (k < a.K) ? ids[k] * RQ * RQ : 0;
    float3 kd, F0;
    float a2 = 0.f, kk = 0.f, specV = 0.f, NdotV = 1.f;
    if (MODE == SOP_MODE_SHADE) {
        const float3 alb = load3(a.albedo, mm);
        const float r = __ldg(a.rough + mm), mt = __ldg(a.metal + mm);
        if (a.status && active && sub == 0 && !isfinite(alb.x + alb.y + alb.z + r + mt + wo.x + wo.y + wo.z))
            atomicOr(a.status, SOP_DEVSTAT_NONFINITE);
        const float dsc = (1.f - mt) * kInvPi;
        kd = f3(dsc * alb.x, dsc * alb.y, dsc * alb.z);
        const float f0d = 0.08f * a.specular * (1.f - mt);
        F0 = f3(f0d + alb.x * mt, f0d + alb.y * mt, f0d + alb.z * mt);
        const float al = r * r;
        a2 = al * al;
        kk = (r + 1.f) * (r + 1.f) * 0.125f;
        NdotV = fmaxf(dot3(n, wo), 1e-4f);
        const float G1V = NdotV / (NdotV * (1.f - kk) + kk);
        specV = G1V / (4.f * NdotV);
    }
    float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f, den0 = 0.f, den1 = 0.f, den2 = 0.f;
    for (int i = sub; i < a.S; i += LANES) {
        const float4 ta = s_tab[3 * i], tb = s_tab[3 * i + 1], tc = s_tab[3 * i + 2];
        const float3 w = f3(ta.x, ta.y, ta.z);
        const float NdotL = dot3(n, w);
        if (!(NdotL > 0.f)) continue;  // below the horizon: no contribution
        const int off = __float_as_int(tb.w);
        if (MODE == SOP_MODE_SHADOW) {
            const float vis = 1.f - shadow_blend<DT, KMAX>(a.quads, base, W, a.K, off, tc.x, tc.y, tc.z, tc.w);
            const float c = NdotL * ta.w;
            const float L0 = tb.x * c, L1 = tb.y * c, L2 = tb.z * c;
            acc0 = fmaf(L0, vis, acc0);
            acc1 = fmaf(L1, vis, acc1);
            acc2 = fmaf(L2, vis, acc2);
            den0 += L0;
            den1 += L1;
            den2 += L2;
        } else {
            float4 pr = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int k = 0; k < KMAX; ++k) {
                if (k < a.K) {
                    float4 t00, t10, t01, t11;
                    Quad<DT>::load(a.quads, (int64_t)(base[k] + off), t00, t10, t01, t11);
                    const float c00 = W[k] * tc.x, c10 = W[k] * tc.y, c01 = W[k] * tc.z, c11 = W[k] * tc.w;
                    pr.x += c00 * t00.x + c10 * t10.x + c01 * t01.x + c11 * t11.x;
                    pr.y += c00 * t00.y + c10 * t10.y + c01 * t01.y + c11 * t11.y;
                    pr.z += c00 * t00.z + c10 * t10.z + c01 * t01.z + c11 * t11.z;
                    pr.w += c00 * t00.w + c10 * t10.w + c01 * t01.w + c11 * t11.w;
                }
            }
            const float vis = 1.f - pr.w;
            float3 h = w + wo;
            const float hl2 = dot3(h, h);
            h = hl2 > 1e-30f ? rsqrtf(hl2) * h : n;
            const float NdotH = dot3(n, h), VdotH = dot3(wo, h);
            const float3 cr = cross3(n, h);
            const float sin2 = dot3(cr, cr);
            const float den = NdotH * NdotH * a2 + sin2;
            const float D = __fdividef(a2, kPi * den * den);
            const float spec = __fdividef(D * specV, NdotL * (1.f - kk) + kk);
            const float x1 = 1.f - VdotH, x2 = x1 * x1, fc = x2 * x2 * x1;
            const float f0 = kd.x + spec * (F0.x + (1.f - F0.x) * fc);
            const float f1 = kd.y + spec * (F0.y + (1.f - F0.y) * fc);
            const float f2 = kd.z + spec * (F0.z + (1.f - F0.z) * fc);
            const float c = NdotL * ta.w;
            acc0 += f0 * (vis * tb.x + pr.x) * c;
            acc1 += f1 * (vis * tb.y + pr.y) * c;
            acc2 += f2 * (vis * tb.z + pr.z) * c;
        }
    }
    for (int o = LANES / 2; o > 0; o >>= 1) {
        acc0 += __shfl_xor_sync(0xffffffffu, acc0, o);
        acc1 += __shfl_xor_sync(0xffffffffu, acc1, o);
        acc2 += __shfl_xor_sync(0xffffffffu, acc2, o);
        if (MODE == SOP_MODE_SHADOW) {
            den0 += __shfl_xor_sync(0xffffffffu, den0, o);
            den1 += __shfl_xor_sync(0xffffffffu, den1, o);
            den2 += __shfl_xor_sync(0xffffffffu, den2, o);
        }
    }
    if (active && sub == 0) {
        float* o = a.out + 3 * m;
        if (MODE == SOP_MODE_SHADE) {
            const float sc = 1.f / (float)a.S;
            o[0] = sc * acc0;
            o[1] = sc * acc1;
            o[2] = sc * acc2;
        } else {
            o[0] = den0 < 1e-20f ? 1.f : acc0 / den0;
            o[1] = den1 < 1e-20f ? 1.f : acc1 / den1;
            o[2] = den2 < 1e-20f ? 1.f : acc2 / den2;
        }
    }
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
cudaError_t launch_hammersley(int32_t S, float* out3, cudaStream_t s)
{
    dirs_kernel<<<(S + 127) / 128, 128, 0, s>>>(S, nullptr, nullptr, out3);
    return cudaGetLastError();
}

cudaError_t launch_query_prep(const QueryArgs& a, const QueryLayout& L, char* ws, cudaStream_t s)
{
    ProbeGrid* grid = reinterpret_cast<ProbeGrid*>(ws + L.grid_hdr);
    int32_t* cstart = reinterpret_cast<int32_t*>(ws + L.cell_start);
    int32_t* ccnt = reinterpret_cast<int32_t*>(ws + L.cell_cnt);
    int4* ent = reinterpret_cast<int4*>(ws + L.entries);
    unsigned int* status = status_word();
    probe_grid_kernel<<<1, 1024, 0, s>>>(a.probe_pos, a.P, L.g_axis, grid, cstart, ccnt, ent);
    int32_t* idx = reinterpret_cast<int32_t*>(ws + L.idx);
    float* w = reinterpret_cast<float*>(ws + L.w);
    if (a.M > 0) {
        const int bs = 128;
        const unsigned nb = (unsigned)((a.M + bs - 1) / bs);
#define SOP_KNN(KM) \
    knn_kernel<KM><<<nb, bs, 0, s>>>(a.x, a.n, a.M, a.K, a.snap_key, a.r2_key, grid, cstart, ent, a.probe_pos, idx, w, \
                                     a.out_idx, a.out_w, status)
        if (a.K <= 4) SOP_KNN(4);
        else if (a.K <= 8) SOP_KNN(8);
        else if (a.K <= 16) SOP_KNN(16);
        else SOP_KNN(32);
#undef SOP_KNN
    }
    if (a.env_layout == SOP_ENV_OCTAHEDRAL) {
        const int64_t nq = (int64_t)(a.He + 1) * (a.He + 1);
        env_oct_quad_kernel<<<(unsigned)((nq + 255) / 256), 256, 0, s>>>(a.env, a.He,
                                                                         reinterpret_cast<float4*>(ws + L.envq), status);
    } else {
        const int64_t ne = (int64_t)(a.He + 2) * (a.We + 1);
        env_pack_kernel<<<(unsigned)((ne + 255) / 256), 256, 0, s>>>(a.env, a.He, a.We,
                                                                       reinterpret_cast<float4*>(ws + L.env4), status);
        const int64_t nq = (int64_t)(a.He + 1) * a.We;
        env_quad_kernel<<<(unsigned)((nq + 255) / 256), 256, 0, s>>>(reinterpret_cast<const float4*>(ws + L.env4),
                                                                       a.He, a.We,
                                                                       reinterpret_cast<float4*>(ws + L.envq));
    }
    const int64_t na = (int64_t)a.P * (a.R + 1) * (a.R + 1);
    const unsigned nba = (unsigned)((na + 255) / 256);
    if (a.mode == SOP_MODE_SHADOW) {
        // occlusion-only footprints (a quarter of the RGBO ones, same slot)
        if (a.rgbo_dtype == SOP_F32)
            atlas_occ_quad_f32_kernel<<<nba, 256, 0, s>>>(reinterpret_cast<const float4*>(a.rgbo), a.P, a.R,
                                                          reinterpret_cast<float4*>(ws + L.quads), status);
        else if (a.rgbo_dtype == SOP_BF16)
            atlas_occ_quad_16_kernel<SOP_BF16><<<nba, 256, 0, s>>>(reinterpret_cast<const uint2*>(a.rgbo), a.P, a.R,
                                                                   reinterpret_cast<uint2*>(ws + L.quads), status);
        else
            atlas_occ_quad_16_kernel<SOP_F16><<<nba, 256, 0, s>>>(reinterpret_cast<const uint2*>(a.rgbo), a.P, a.R,
                                                                  reinterpret_cast<uint2*>(ws + L.quads), status);
    } else switch (a.rgbo_dtype) {
    case SOP_F32:
        atlas_quad_kernel<SOP_F32><<<nba, 256, 0, s>>>(reinterpret_cast<const float4*>(a.rgbo), a.P, a.R,
                                                      reinterpret_cast<float4*>(ws + L.quads), status);
        break;
    case SOP_BF16:
        atlas_quad_kernel<SOP_BF16><<<nba, 256, 0, s>>>(reinterpret_cast<const uint2*>(a.rgbo), a.P, a.R,
                                                       reinterpret_cast<uint2*>(ws + L.quads), status);
        break;
    default:
        atlas_quad_kernel<SOP_F16><<<nba, 256, 0, s>>>(reinterpret_cast<const uint2*>(a.rgbo), a.P, a.R,
                                                      reinterpret_cast<uint2*>(ws + L.quads), status);
        break;
    }
    if (a.dir_world)
        world_dirs_kernel<<<(a.S + 127) / 128, 128, 0, s>>>(a.S, reinterpret_cast<const float4*>(a.dirs_local),
                                                            reinterpret_cast<float4*>(ws + L.dirs));
    else
        dirs_kernel<<<(a.S + 127) / 128, 128, 0, s>>>(a.S, a.dirs_local, reinterpret_cast<float4*>(ws + L.dirs),
                                                      nullptr);
    return cudaGetLastError();
}

template <int DT, int KMAX, int MODE>
static cudaError_t shade_launch(const ShadeK& k, int LANES, cudaStream_t s)
{
    const int bs = 256;
    const int64_t threads = k.M * LANES;
    const unsigned nb = (unsigned)((threads + bs - 1) / bs);
    size_t smem = sizeof(float4) * (size_t)k.S;
    // per-warp direction tables of the shared-normal SHADOW path (8 warps)
    if (MODE == SOP_MODE_SHADOW && k.S <= kShadowTab) smem += (size_t)(bs / 32) * 2 * sizeof(float4) * k.S;
    auto fn = shade_kernel<DT, KMAX, MODE>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    fn<<<nb, bs, smem, s>>>(k, LANES);
    return cudaGetLastError();
}

// Threads per shading point (they split the S directions).
// Measured on GB300, object workload: one thread per point for a float32
// atlas, two for 16-bit atlases; small point sets (the composition frame's
// 21,907 object pixels) take more lanes per point, up to 8, until the launch
// has about two waves of threads on the 152 SMs.
static int shade_lanes(int dtype, int64_t M)
{
    int l = dtype == SOP_F32 ? 1 : 2;
    while (l < 8 && M * l < (int64_t)2 * 152 * 1024) l *= 2;
    return l;
}

template <int DT, int KMAX, int MODE>
static cudaError_t shade_dispatch(const ShadeK& k, cudaStream_t s)
{
    return shade_launch<DT, KMAX, MODE>(k, shade_lanes(DT, k.M), s);
}

template <int DT, int MODE>
static cudaError_t shade_k(const ShadeK& k, cudaStream_t s)
{
    if (k.K <= 4) return shade_dispatch<DT, 4, MODE>(k, s);
    if (k.K <= 8) return shade_dispatch<DT, 8, MODE>(k, s);
    if (k.K <= 16) return shade_dispatch<DT, 16, MODE>(k, s);
    return shade_dispatch<DT, 32, MODE>(k, s);
}

template <int DT, int KMAX, int MODE>
static cudaError_t shade_world_launch(const ShadeK& k, cudaStream_t s)
{
    const int bs = 256, LANES = shade_lanes(DT, k.M);
    const int64_t threads = k.M * LANES;
    const unsigned nb = (unsigned)((threads + bs - 1) / bs);
    const size_t smem = 3 * sizeof(float4) * (size_t)k.S;
    auto fn = shade_world_kernel<DT, KMAX, MODE>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    fn<<<nb, bs, smem, s>>>(k, LANES);
    return cudaGetLastError();
}

template <int DT, int MODE>
static cudaError_t shade_world_k(const ShadeK& k, cudaStream_t s)
{
    if (k.K <= 4) return shade_world_launch<DT, 4, MODE>(k, s);
    if (k.K <= 8) return shade_world_launch<DT, 8, MODE>(k, s);
    if (k.K <= 16) return shade_world_launch<DT, 16, MODE>(k, s);
    return shade_world_launch<DT, 32, MODE>(k, s);
}

template <int DT>
static cudaError_t shade_mode(const ShadeK& k, int mode, bool world, cudaStream_t s)
{
    if (world)
        return mode == SOP_MODE_SHADE ? shade_world_k<DT, SOP_MODE_SHADE>(k, s) : shade_world_k<DT, SOP_MODE_SHADOW>(k, s);
    return mode == SOP_MODE_SHADE ? shade_k<DT, SOP_MODE_SHADE>(k, s) : shade_k<DT, SOP_MODE_SHADOW>(k, s);
}


cudaError_t launch_shade(const QueryArgs& a, const QueryLayout& L, char* ws, cudaStream_t s)
{
    if (a.M == 0) return cudaSuccess;
    ShadeK k;
    k.n = a.n;
    k.wo = a.wo;
    k.albedo = a.albedo;
    k.rough = a.rough;
    k.metal = a.metal;
    k.M = a.M;
    k.rgbo = a.rgbo;
    k.R = a.R;
    k.K = a.K;
    k.S = a.S;
    k.He = a.He;
    k.We = a.We;
    k.envq = reinterpret_cast<const float4*>(ws + L.envq);
    k.env_layout = a.env_layout;
    k.quads = ws + L.quads;
    k.dirs = reinterpret_cast<const float4*>(ws + L.dirs);
    k.idx = reinterpret_cast<const int32_t*>(ws + L.idx);
    k.w = reinterpret_cast<const float*>(ws + L.w);
    k.specular = a.specular;
    k.out = a.out;
    k.status = status_word();
    switch (a.rgbo_dtype) {
    case SOP_F32: return shade_mode<SOP_F32>(k, a.mode, a.dir_world != 0, s);
    case SOP_BF16: return shade_mode<SOP_BF16>(k, a.mode, a.dir_world != 0, s);
    case SOP_F16: return shade_mode<SOP_F16>(k, a.mode, a.dir_world != 0, s);
    default: return cudaErrorInvalidValue;
    }
}


// ---------------------------------------------------------------------------
// Multi-CTA build of the same quantised grid for large site sets (the
// single-CTA probe_grid_kernel is meant for thousands of probes).
// ---------------------------------------------------------------------------
__global__ void sites_bbox_kernel(const float* __restrict__ pos, int32_t N, int32_t* __restrict__ mm)
{
    int32_t lo[3] = {INT32_MAX, INT32_MAX, INT32_MAX}, hi[3] = {INT32_MIN, INT32_MIN, INT32_MIN};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        for (int a = 0; a < 3; ++a) {
            const int32_t q = quantise(pos[3 * i + a]);
            lo[a] = min(lo[a], q);
            hi[a] = max(hi[a], q);
        }
    for (int a = 0; a < 3; ++a) {
        for (int o = 16; o > 0; o >>= 1) {
            lo[a] = min(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
            hi[a] = max(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
        }
        if ((threadIdx.x & 31) == 0) {
            atomicMin(&mm[a], lo[a]);
            atomicMax(&mm[3 + a], hi[a]);
        }
    }
}

__global__ void sites_setup_kernel(int32_t* mm, int64_t cap, ProbeGrid* grid)
{
    if (threadIdx.x == 0) {
        ProbeGrid G;
        int64_t ext[3];
        for (int a = 0; a < 3; ++a) ext[a] = (int64_t)mm[3 + a] - mm[a];
        const int64_t cs = grid_cell_edge(ext, cap);
        G.cs = (int32_t)cs;
        int32_t nc = 1;
        for (int a = 0; a < 3; ++a) {
            G.qmin[a] = mm[a];
            G.dims[a] = (int32_t)(ext[a] / cs) + 1;
            nc *= G.dims[a];
        }
        G.ncells = nc;
        *grid = G;
    }
}

__global__ void sites_zero_kernel(int32_t* __restrict__ cnt, int64_t n, int32_t* mm)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) cnt[i] = 0;
    if (i < 3) mm[i] = INT32_MAX;
    else if (i < 6) mm[i] = INT32_MIN;
}

__device__ __forceinline__ int site_cell(const ProbeGrid& G, const float* pos, int64_t i, int32_t q[3])
{
    int c[3];
    for (int a = 0; a < 3; ++a) {
        q[a] = quantise(pos[3 * i + a]);
        c[a] = (int)(((int64_t)q[a] - G.qmin[a]) / G.cs);
    }
    return (c[2] * G.dims[1] + c[1]) * G.dims[0] + c[0];
}

__global__ void sites_count_kernel(const float* __restrict__ pos, int32_t N, const ProbeGrid* __restrict__ gp,
                                   int32_t* __restrict__ cnt)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const ProbeGrid G = *gp;
    int32_t q[3];
    atomicAdd(&cnt[site_cell(G, pos, i, q)], 1);
}

__global__ void sites_fill_kernel(const float* __restrict__ pos, int32_t N, const ProbeGrid* __restrict__ gp,
                                  const int32_t* __restrict__ start, int32_t* __restrict__ cnt, int4* __restrict__ ent)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const ProbeGrid G = *gp;
    int32_t q[3];
    const int cell = site_cell(G, pos, i, q);
    ent[start[cell] + atomicAdd(&cnt[cell], 1)] = make_int4(q[0], q[1], q[2], (int)i);
}

// ---------------------------------------------------------------------------
// K nearest sites (e.g. Gaussian centres) of M query points, exact, with the
// same integer keys and tie rule as the probe search.
// ---------------------------------------------------------------------------
size_t sites_grid_bytes(int32_t N)
{
    int g = 1;
    while ((int64_t)g * g * g < N) ++g;
    const int64_t cells = (int64_t)(g + 1) * (g + 1) * (g + 1);
    size_t o = align256(sizeof(ProbeGrid));
    o = align256(o + sizeof(int32_t) * (size_t)(cells + 1));
    o = align256(o + sizeof(int32_t) * (size_t)cells);
    o = align256(o + sizeof(int4) * (size_t)N);
    o = align256(o + 8 * sizeof(int32_t));
    o = align256(o + sizeof(long long) * scan_scratch_count(cells));
    return o;
}

// ---------------------------------------------------------------------------
// Read-bandwidth probe: every thread streams 16-byte loads over the buffer,
// `reps` times, on all SMs. A buffer that fits in L2 gives the L2-to-SM read
// rate that bounds the query's footprint gathers; a larger one the HBM rate.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(512) read_probe_kernel(const uint4* __restrict__ buf, int64_t n16, int32_t reps,
                                                          float* __restrict__ sink)
{
    uint32_t acc = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int r = 0; r < reps; ++r)
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride) {
            const uint4 v = __ldcg(buf + i);
            acc ^= v.x ^ v.y ^ v.z ^ v.w;
        }
    // a store the compiler cannot drop, taken only for one improbable value
    if (acc == 0x9e3779b9u) sink[0] = (float)acc;
}

cudaError_t launch_read_probe(const void* buf, size_t bytes, int32_t reps, float* sink, cudaStream_t s)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    read_probe_kernel<<<(unsigned)(sms > 0 ? sms : 152) * 4, 512, 0, s>>>(reinterpret_cast<const uint4*>(buf),
                                                                             (int64_t)(bytes / 16), reps, sink);
    return cudaGetLastError();
}

SitesGrid launch_sites_grid(const float* sites, int32_t N, char* ws, cudaStream_t s)
{
    int g = 1;
    while ((int64_t)g * g * g < N) ++g;
    const int64_t cells = (int64_t)(g + 1) * (g + 1) * (g + 1);
    size_t o = 0;
    SitesGrid r;
    ProbeGrid* grid = reinterpret_cast<ProbeGrid*>(ws + o);
    o = align256(sizeof(ProbeGrid));
    int32_t* cstart = reinterpret_cast<int32_t*>(ws + o);
    o = align256(o + sizeof(int32_t) * (size_t)(cells + 1));
    int32_t* ccnt = reinterpret_cast<int32_t*>(ws + o);
    o = align256(o + sizeof(int32_t) * (size_t)cells);
    int4* ent = reinterpret_cast<int4*>(ws + o);
    o = align256(o + sizeof(int4) * (size_t)N);
    int32_t* mm = reinterpret_cast<int32_t*>(ws + o);
    o = align256(o + 8 * sizeof(int32_t));
    long long* scan = reinterpret_cast<long long*>(ws + o);
    if (N <= 16384) {
        probe_grid_kernel<<<1, 1024, 0, s>>>(sites, N, g, grid, cstart, ccnt, ent);
    } else {
        const unsigned nb = (unsigned)((N + 255) / 256);
        sites_zero_kernel<<<(unsigned)((cells + 255) / 256), 256, 0, s>>>(ccnt, cells, mm);
        sites_bbox_kernel<<<nb < 1024 ? nb : 1024, 256, 0, s>>>(sites, N, mm);
        // about 4 sites per grid cell: the warp search pays per ring (a
        // round of dependent loads) far more than per candidate (32 lanes)
        const int64_t cap = N / 4 > 4096 ? N / 4 : 4096;
        sites_setup_kernel<<<1, 32, 0, s>>>(mm, cap < cells ? cap : cells, grid);
        sites_count_kernel<<<nb, 256, 0, s>>>(sites, N, grid, ccnt);
        ScanArgs sa;
        sa.n = &grid->ncells;
        sa.skip = nullptr;
        sa.cnt = ccnt;
        sa.start = cstart;
        sa.scratch = scan;
        launch_scan(sa, cap < cells ? cap : cells, ScanNoFinal{}, s);
        sites_fill_kernel<<<nb, 256, 0, s>>>(sites, N, grid, cstart, ccnt, ent);
    }
    r.grid = grid;
    r.cell_start = cstart;
    r.entries = ent;
    return r;
}


// ===========================================================================
// Allocation-free variant of the query + shade (sop_query_shade_noalloc).
//
// For callers that cannot allocate device memory themselves. Its scratch is
// one file-scope device array of kNoAllocScratchBytes, present on every GPU
// that loads the library until the process exits. Host code cannot pass the
// array's name to a kernel (on the host it is only a stand-in symbol), so the
// first call on each device looks up the array's device address with
// cudaGetSymbolAddress while that device is current, and later calls reuse
// it. The probe atlas and the environment are read in the caller's own
// layouts (no repacked copies), and points are processed in chunks of
// kNoAllocChunk so that the per-point neighbour lists fit the array. All
// calls share the array: calls that overlap on the GPU (other streams, other
// host threads) race on it.
// ===========================================================================
constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;
constexpr int64_t kNoAllocChunk = 16384;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

size_t noalloc_scratch_bytes() { return kNoAllocScratchBytes; }
int64_t noalloc_chunk() { return kNoAllocChunk; }

// Bilinear environment lookup straight from the caller's [He][We][3] array.
__device__ __forceinline__ float3 env_lookup_direct(const float* __restrict__ env, int He, int We, float3 w)
{
    const float th = atan2f(sqrtf(w.x * w.x + w.y * w.y), w.z);
    const float ph = atan2f(w.y, w.x);
    const float s = (ph + kPi) * kInv2Pi * We - 0.5f;
    const float t = th * kInvPi * He - 0.5f;
    const float fs = floorf(s), ft = floorf(t);
    const float a = s - fs, b = t - ft;
    int c0 = (int)fs;
    c0 = c0 < 0 ? c0 + We : c0;
    c0 = min(max(c0, 0), We - 1);
    const int c1 = c0 + 1 == We ? 0 : c0 + 1;
    const int r0 = min(max((int)ft, 0), He - 1), r1 = min(max((int)ft + 1, 0), He - 1);
    const float* e00 = env + ((int64_t)r0 * We + c0) * 3;
    const float* e01 = env + ((int64_t)r0 * We + c1) * 3;
    const float* e10 = env + ((int64_t)r1 * We + c0) * 3;
    const float* e11 = env + ((int64_t)r1 * We + c1) * 3;
    const float w00 = (1.f - a) * (1.f - b), w01 = a * (1.f - b), w10 = (1.f - a) * b, w11 = a * b;
    return f3(w00 * __ldg(e00) + w01 * __ldg(e01) + w10 * __ldg(e10) + w11 * __ldg(e11),
              w00 * __ldg(e00 + 1) + w01 * __ldg(e01 + 1) + w10 * __ldg(e10 + 1) + w11 * __ldg(e11 + 1),
              w00 * __ldg(e00 + 2) + w01 * __ldg(e01 + 2) + w10 * __ldg(e10 + 2) + w11 * __ldg(e11 + 2));
}

// Equirectangular -> octahedral environment (Sec. 4.1): texel (i, j) of the
// [H][H] map takes the bilinear equirectangular value at its centre
// direction (computed in double, rounded once).
__global__ void env_to_oct_kernel(const float* __restrict__ env, int32_t He, int32_t We, float* __restrict__ out,
                                  int32_t H)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (int64_t)H * H) return;
    double d[3];
    oct_decode_centre_f64(H, (int)(k % H), (int)(k / H), d);
    const float3 v = env_lookup_direct(env, He, We, f3((float)d[0], (float)d[1], (float)d[2]));
    out[3 * k] = v.x;
    out[3 * k + 1] = v.y;
    out[3 * k + 2] = v.z;
}

cudaError_t launch_env_to_oct(const float* env, int32_t He, int32_t We, float* out, int32_t H, cudaStream_t s)
{
    const int64_t n = (int64_t)H * H;
    env_to_oct_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(env, He, We, out, H);
    return cudaGetLastError();
}

struct ShadeDirectK {
    const float *n, *wo, *albedo, *rough, *metal;
    int64_t M;
    const void* rgbo;
    int32_t R, K, S, He, We;
    const float* env;
    const float4* dirs;
    const int32_t* idx;
    const float* w;
    float specular;
    float* out;
};

// One thread per point; texels read from the gutter atlas, four per probe.
template <int DT, int KMAX, int MODE>
__global__ void __launch_bounds__(256) shade_direct_kernel(const ShadeDirectK a)
{
    using TX = Texel<DT>;
    extern __shared__ float4 s_dirs[];
    for (int i = threadIdx.x; i < a.S; i += blockDim.x) s_dirs[i] = a.dirs[i];
    __syncthreads();
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= a.M) return;
    const float3 nr = load3(a.n, m);
    const float nl = sqrtf(dot3(nr, nr));
    const float3 n = f3(nr.x / nl, nr.y / nl, nr.z / nl);
    float3 tt, bb;
    onb(n, tt, bb);
    const float3 wo = load3(a.wo, m);
    const int RS = a.R + 2;
    const typename TX::raw* atlas = reinterpret_cast<const typename TX::raw*>(a.rgbo);
    int64_t base[KMAX];
    float W[KMAX];
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
        const bool on = k < a.K;
        base[k] = on ? (int64_t)__ldg(a.idx + m * a.K + k) * RS * RS : 0;
        W[k] = on ? __ldg(a.w + m * a.K + k) : 0.f;
    }
    float3 kd = f3(0.f, 0.f, 0.f), F0 = f3(0.f, 0.f, 0.f);
    float a2 = 0.f, kk = 0.f, specV = 0.f;
    if (MODE == SOP_MODE_SHADE) {
        const float3 alb = load3(a.albedo, m);
        const float r = __ldg(a.rough + m), mt = __ldg(a.metal + m);
        const float dsc = (1.f - mt) * kInvPi;
        kd = f3(dsc * alb.x, dsc * alb.y, dsc * alb.z);
        const float f0d = 0.08f * a.specular * (1.f - mt);
        F0 = f3(f0d + alb.x * mt, f0d + alb.y * mt, f0d + alb.z * mt);
        const float al = r * r;
        a2 = al * al;
        kk = (r + 1.f) * (r + 1.f) * 0.125f;
        const float NdotV = fmaxf(dot3(n, wo), 1e-4f);
        specV = (NdotV / (NdotV * (1.f - kk) + kk)) / (4.f * NdotV);
    }
    float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f, den0 = 0.f, den1 = 0.f, den2 = 0.f;
    const float Rf = (float)a.R;
    for (int i = 0; i < a.S; ++i) {
        const float4 l = s_dirs[i];
        const float3 w = f3(fmaf(l.x, tt.x, fmaf(l.y, bb.x, l.z * n.x)), fmaf(l.x, tt.y, fmaf(l.y, bb.y, l.z * n.y)),
                            fmaf(l.x, tt.z, fmaf(l.y, bb.z, l.z * n.z)));
        const float2 uv = oct_encode(w);
        const float s = uv.x * Rf - 0.5f, t = uv.y * Rf - 0.5f;
        const float fi = floorf(s), fj = floorf(t);
        const float fu = s - fi, fv = t - fj;
        const int i0 = min(max((int)fi + 1, 0), a.R), j0 = min(max((int)fj + 1, 0), a.R);
        const int off = j0 * RS + i0;
        const float w00 = (1.f - fu) * (1.f - fv), w10 = fu * (1.f - fv), w01 = (1.f - fu) * fv, w11 = fu * fv;
        float4 pr = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int k = 0; k < KMAX; ++k) {
            if (k < a.K) {
                const typename TX::raw* p = atlas + base[k] + off;
                const float4 t00 = TX::load(p), t10 = TX::load(p + 1), t01 = TX::load(p + RS), t11 = TX::load(p + RS + 1);
                const float c00 = W[k] * w00, c10 = W[k] * w10, c01 = W[k] * w01, c11 = W[k] * w11;
                pr.x += c00 * t00.x + c10 * t10.x + c01 * t01.x + c11 * t11.x;
                pr.y += c00 * t00.y + c10 * t10.y + c01 * t01.y + c11 * t11.y;
                pr.z += c00 * t00.z + c10 * t10.z + c01 * t01.z + c11 * t11.z;
                pr.w += c00 * t00.w + c10 * t10.w + c01 * t01.w + c11 * t11.w;
            }
        }
        const float3 Ld = env_lookup_direct(a.env, a.He, a.We, w);
        const float NdotL = l.z;
        const float vis = 1.f - pr.w;
        if (MODE == SOP_MODE_SHADE) {
            float3 h = w + wo;
            const float hl2 = dot3(h, h);
            h = hl2 > 1e-30f ? rsqrtf(hl2) * h : n;
            const float NdotH = dot3(n, h), VdotH = dot3(wo, h);
            const float3 cr = cross3(n, h);
            const float sin2 = dot3(cr, cr);
            const float den = NdotH * NdotH * a2 + sin2;
            const float D = __fdividef(a2, kPi * den * den);
            const float spec = __fdividef(D * specV, NdotL * (1.f - kk) + kk);
            const float x1 = 1.f - VdotH, x2 = x1 * x1, fc = x2 * x2 * x1;
            acc0 += (kd.x + spec * (F0.x + (1.f - F0.x) * fc)) * (vis * Ld.x + pr.x) * NdotL;
            acc1 += (kd.y + spec * (F0.y + (1.f - F0.y) * fc)) * (vis * Ld.y + pr.y) * NdotL;
            acc2 += (kd.z + spec * (F0.z + (1.f - F0.z) * fc)) * (vis * Ld.z + pr.z) * NdotL;
        } else {
            acc0 += Ld.x * vis * NdotL;
            acc1 += Ld.y * vis * NdotL;
            acc2 += Ld.z * vis * NdotL;
            den0 += Ld.x * NdotL;
            den1 += Ld.y * NdotL;
            den2 += Ld.z * NdotL;
        }
    }
    float* o = a.out + 3 * m;
    if (MODE == SOP_MODE_SHADE) {
        const float sc = 2.f * kPi / (float)a.S;
        o[0] = sc * acc0;
        o[1] = sc * acc1;
        o[2] = sc * acc2;
    } else {
        o[0] = den0 < 1e-20f ? 1.f : acc0 / den0;
        o[1] = den1 < 1e-20f ? 1.f : acc1 / den1;
        o[2] = den2 < 1e-20f ? 1.f : acc2 / den2;
    }
}

template <int DT, int KMAX, int MODE>
static cudaError_t shade_direct_launch(const ShadeDirectK& k, cudaStream_t s)
{
    const size_t smem = sizeof(float4) * (size_t)k.S;
    auto fn = shade_direct_kernel<DT, KMAX, MODE>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    fn<<<(unsigned)((k.M + 255) / 256), 256, smem, s>>>(k);
    return cudaGetLastError();
}

template <int DT, int MODE>
static cudaError_t shade_direct_k(const ShadeDirectK& k, cudaStream_t s)
{
    if (k.K <= 4) return shade_direct_launch<DT, 4, MODE>(k, s);
    if (k.K <= 8) return shade_direct_launch<DT, 8, MODE>(k, s);
    if (k.K <= 16) return shade_direct_launch<DT, 16, MODE>(k, s);
    return shade_direct_launch<DT, 32, MODE>(k, s);
}

template <int DT>
static cudaError_t shade_direct_mode(const ShadeDirectK& k, int mode, cudaStream_t s)
{
    return mode == SOP_MODE_SHADE ? shade_direct_k<DT, SOP_MODE_SHADE>(k, s) : shade_direct_k<DT, SOP_MODE_SHADOW>(k, s);
}

// Device address of the scratch array on the current device, looked up once
// per device (the lookup must run with that device current).
static cudaError_t noalloc_scratch_ptr(char** out)
{
    static std::mutex mu;
    static char* ptrs[256] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (!ptrs[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        ptrs[dev] = static_cast<char*>(p);
    }
    *out = ptrs[dev];
    return cudaSuccess;
}

// Scratch layout for P probes, S directions and K neighbours (per chunk).
static QueryLayout noalloc_layout(int32_t P, int32_t K, int32_t S)
{
    QueryLayout L{};
    int g = 1;
    while ((int64_t)g * g * g < P) ++g;
    L.g_axis = g;
    L.cells_cap = (g + 1) * (g + 1) * (g + 1);
    size_t o = 0;
    L.grid_hdr = o;   o = align256(o + sizeof(ProbeGrid));
    L.cell_start = o; o = align256(o + sizeof(int32_t) * (size_t)(L.cells_cap + 1));
    L.cell_cnt = o;   o = align256(o + sizeof(int32_t) * (size_t)L.cells_cap);
    L.entries = o;    o = align256(o + sizeof(int4) * (size_t)P);
    L.dirs = o;       o = align256(o + sizeof(float4) * (size_t)S);
    L.idx = o;        o = align256(o + sizeof(int32_t) * (size_t)kNoAllocChunk * K);
    L.w = o;          o = align256(o + sizeof(float) * (size_t)kNoAllocChunk * K);
    L.total = o;
    return L;
}

size_t noalloc_required_bytes(int32_t P, int32_t K, int32_t S) { return noalloc_layout(P, K, S).total; }

cudaError_t launch_query_noalloc(const QueryArgs& a, cudaStream_t s)
{
    char* ws = nullptr;
    cudaError_t e = noalloc_scratch_ptr(&ws);
    if (e != cudaSuccess) return e;
    const QueryLayout L = noalloc_layout(a.P, a.K, a.S);
    if (L.total > kNoAllocScratchBytes) return cudaErrorInvalidValue;  // checked by the caller first
    ProbeGrid* grid = reinterpret_cast<ProbeGrid*>(ws + L.grid_hdr);
    int32_t* cstart = reinterpret_cast<int32_t*>(ws + L.cell_start);
    int32_t* ccnt = reinterpret_cast<int32_t*>(ws + L.cell_cnt);
    int4* ent = reinterpret_cast<int4*>(ws + L.entries);
    float4* dirs = reinterpret_cast<float4*>(ws + L.dirs);
    int32_t* idx = reinterpret_cast<int32_t*>(ws + L.idx);
    float* w = reinterpret_cast<float*>(ws + L.w);
    // the grid build clears its own counters, so stale contents are harmless
    probe_grid_kernel<<<1, 1024, 0, s>>>(a.probe_pos, a.P, L.g_axis, grid, cstart, ccnt, ent);
    dirs_kernel<<<(a.S + 127) / 128, 128, 0, s>>>(a.S, a.dirs_local, dirs, nullptr);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    for (int64_t m0 = 0; m0 < a.M; m0 += kNoAllocChunk) {
        const int64_t mc = a.M - m0 < kNoAllocChunk ? a.M - m0 : kNoAllocChunk;
        const unsigned nb = (unsigned)((mc + 127) / 128);
        int32_t* uidx = a.out_idx ? a.out_idx + m0 * a.K : nullptr;
        float* uw = a.out_w ? a.out_w + m0 * a.K : nullptr;
#define SOP_KNN_NA(KM)                                                                                             \
    knn_kernel<KM><<<nb, 128, 0, s>>>(a.x + 3 * m0, a.n + 3 * m0, mc, a.K, a.snap_key, a.r2_key, grid, cstart, ent, \
                                      a.probe_pos, idx, w, uidx, uw, status_word())
        if (a.K <= 4) SOP_KNN_NA(4);
        else if (a.K <= 8) SOP_KNN_NA(8);
        else if (a.K <= 16) SOP_KNN_NA(16);
        else SOP_KNN_NA(32);
#undef SOP_KNN_NA
        ShadeDirectK k;
        k.n = a.n + 3 * m0;
        k.wo = a.wo + 3 * m0;
        k.albedo = a.albedo + 3 * m0;
        k.rough = a.rough + m0;
        k.metal = a.metal + m0;
        k.M = mc;
        k.rgbo = a.rgbo;
        k.R = a.R;
        k.K = a.K;
        k.S = a.S;
        k.He = a.He;
        k.We = a.We;
        k.env = a.env;
        k.dirs = dirs;
        k.idx = idx;
        k.w = w;
        k.specular = a.specular;
        k.out = a.out + 3 * m0;
        switch (a.rgbo_dtype) {
        case SOP_F32: e = shade_direct_mode<SOP_F32>(k, a.mode, s); break;
        case SOP_BF16: e = shade_direct_mode<SOP_BF16>(k, a.mode, s); break;
        case SOP_F16: e = shade_direct_mode<SOP_F16>(k, a.mode, s); break;
        default: e = cudaErrorInvalidValue;
        }
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

}  // namespace sop
