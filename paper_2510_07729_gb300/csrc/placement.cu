// Automatic placement of SOPs (Sec. 3.2) for sm_103a: farthest point
// sampling (FPS) of a surface point cloud, then an offset of the chosen
// points along their normals.
//
// Distances are exact integer squared distances of positions quantised to
// 2^-20 (the query's keys), so every choice is exact and matches a plain
// sequential FPS: the first point is `start`, each next one has the largest
// smallest key to the chosen ones, ties to the lower index.
//
// fps_cluster_kernel: one thread-block cluster of 16 CTAs (the non-portable
// size, where the device schedules it; else 8) runs all k iterations. CTA r
// owns a contiguous slice of the points; their quantised positions and
// current smallest keys live in its shared memory when the slice fits (else
// in the workspace). Per iteration every thread updates
// its points with the point just chosen and keeps its best (key, index); a
// warp then a CTA reduction gives the CTA's best, published in its shared
// memory (double-buffered by iteration parity); one cluster barrier; every
// thread reads the cluster's bests through distributed shared memory and
// takes the same winner. The barrier is the hardware cluster barrier, which
// every thread of the cluster reaches once per iteration.
#include <climits>
#include <cooperative_groups.h>

#include "sop_device.cuh"
#include "sop_internal.h"

namespace cg = cooperative_groups;

namespace sop {

constexpr int kFpsCtasMax = 16;
constexpr int kFpsThreads = 1024;
constexpr size_t kFpsPointBytes = sizeof(int4) + sizeof(unsigned long long);
constexpr size_t kFpsSmemMax = 220 * 1024;

struct FpsK {
    const float* pts;
    const float* nrm;
    int64_t n, chunk, start;
    int32_t k;
    float offset;
    int4* gq;                  // workspace slices when they do not fit in shared memory
    unsigned long long* gd;
    int use_smem;
    int64_t* out_idx;
    float* out_pos;
};

__device__ __forceinline__ int4 quant4(const float* p, int64_t i)
{
    // x 2^20 is exact in float; rintf rounds half to even
    return make_int4((int)rintf(__ldg(p + 3 * i) * 1048576.f), (int)rintf(__ldg(p + 3 * i + 1) * 1048576.f),
                     (int)rintf(__ldg(p + 3 * i + 2) * 1048576.f), 0);
}

__device__ __forceinline__ bool fps_better(unsigned long long ka, long long ia, unsigned long long kb, long long ib)
{
    return ka > kb || (ka == kb && ia < ib);
}

__global__ void __launch_bounds__(kFpsThreads) fps_cluster_kernel(const FpsK k)
{
    extern __shared__ __align__(16) unsigned char s_dyn[];
    __shared__ unsigned long long s_wkey[32];
    __shared__ long long s_widx[32];
    __shared__ unsigned long long s_ckey[2];
    __shared__ long long s_cidx[2];
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int n_ctas = (int)cl.num_blocks();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t lo = (int64_t)rank * k.chunk;
    const int64_t hi = min(k.n, lo + k.chunk);
    int4* q = k.use_smem ? reinterpret_cast<int4*>(s_dyn) : k.gq + lo;
    unsigned long long* dm =
        k.use_smem ? reinterpret_cast<unsigned long long*>(s_dyn + sizeof(int4) * (size_t)k.chunk) : k.gd + lo;
    for (int64_t i = lo + threadIdx.x; i < hi; i += kFpsThreads) {
        q[i - lo] = quant4(k.pts, i);
        dm[i - lo] = ULLONG_MAX;
    }
    __syncthreads();
    long long cur = k.start;
    for (int it = 0; it < k.k; ++it) {
        if (rank == 0 && threadIdx.x == 0) {
            k.out_idx[it] = cur;
            if (k.out_pos)
                for (int a = 0; a < 3; ++a) {
                    const double x = k.pts[3 * cur + a];
                    k.out_pos[3 * it + a] = (float)(k.nrm ? x + (double)k.offset * (double)k.nrm[3 * cur + a] : x);
                }
        }
        const int4 qc = quant4(k.pts, cur);
        unsigned long long bk = 0ull;
        long long bi = LLONG_MAX;
        for (int64_t i = lo + threadIdx.x; i < hi; i += kFpsThreads) {
            const int4 qi = q[i - lo];
            const long long dx = (long long)qi.x - qc.x, dy = (long long)qi.y - qc.y, dz = (long long)qi.z - qc.z;
            const unsigned long long key =
                (unsigned long long)(dx * dx) + (unsigned long long)(dy * dy) + (unsigned long long)(dz * dz);
            unsigned long long d = dm[i - lo];
            if (key < d) {
                d = key;
                dm[i - lo] = d;
            }
            if (fps_better(d, i, bk, bi)) {
                bk = d;
                bi = i;
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const unsigned long long ok = __shfl_xor_sync(0xffffffffu, bk, off);
            const long long oi = __shfl_xor_sync(0xffffffffu, bi, off);
            if (fps_better(ok, oi, bk, bi)) {
                bk = ok;
                bi = oi;
            }
        }
        if (lane == 0) {
            s_wkey[warp] = bk;
            s_widx[warp] = bi;
        }
        __syncthreads();
        const int buf = it & 1;
        if (warp == 0) {
            bk = s_wkey[lane];
            bi = s_widx[lane];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const unsigned long long ok = __shfl_xor_sync(0xffffffffu, bk, off);
                const long long oi = __shfl_xor_sync(0xffffffffu, bi, off);
                if (fps_better(ok, oi, bk, bi)) {
                    bk = ok;
                    bi = oi;
                }
            }
            if (lane == 0) {
                s_ckey[buf] = bk;
                s_cidx[buf] = bi;
            }
        }
        // every CTA's best of this iteration is published (and the warp
        // partials read) before anyone goes on
        cl.sync();
        unsigned long long gk = 0ull;
        long long gi = LLONG_MAX;
        for (int r = 0; r < n_ctas; ++r) {
            const unsigned long long rk = *cl.map_shared_rank(&s_ckey[buf], r);
            const long long ri = *cl.map_shared_rank(&s_cidx[buf], r);
            if (fps_better(rk, ri, gk, gi)) {
                gk = rk;
                gi = ri;
            }
        }
        cur = gi;
    }
    // no CTA leaves while another may still read its shared memory
    cl.sync();
}

size_t fps_ws_bytes(int64_t n) { return align256(sizeof(int4) * (size_t)n) + align256(8 * (size_t)n); }

cudaError_t launch_fps(const float* pts, const float* nrm, int64_t n, int32_t k, int64_t start, float offset,
                       int64_t* out_idx, float* out_pos, char* ws, cudaStream_t s)
{
    FpsK a;
    a.pts = pts;
    a.nrm = nrm;
    a.n = n;
    // the cluster: 16 CTAs where the device can hold such a cluster, else 8
    static int ctas = 0;
    if (!ctas) {
        ctas = 8;
        if (cudaFuncSetAttribute(fps_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
            cudaSuccess) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(kFpsCtasMax);
            cfg.blockDim = dim3(kFpsThreads);
            cfg.dynamicSmemBytes = kFpsSmemMax;
            cudaLaunchAttribute at;
            at.id = cudaLaunchAttributeClusterDimension;
            at.val.clusterDim.x = kFpsCtasMax;
            at.val.clusterDim.y = 1;
            at.val.clusterDim.z = 1;
            cfg.attrs = &at;
            cfg.numAttrs = 1;
            int nclusters = 0;
            cudaFuncSetAttribute(fps_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFpsSmemMax);
            if (cudaOccupancyMaxActiveClusters(&nclusters, fps_cluster_kernel, &cfg) == cudaSuccess && nclusters > 0)
                ctas = kFpsCtasMax;
        }
        cudaGetLastError();  // a refused query leaves the 8-CTA cluster
    }
    a.chunk = (n + ctas - 1) / ctas;
    a.start = start;
    a.k = k;
    a.offset = offset;
    a.gq = reinterpret_cast<int4*>(ws);
    a.gd = reinterpret_cast<unsigned long long*>(ws + align256(sizeof(int4) * (size_t)n));
    a.out_idx = out_idx;
    a.out_pos = out_pos;
    const size_t smem = kFpsPointBytes * (size_t)a.chunk;
    a.use_smem = smem <= kFpsSmemMax;
    const size_t dyn = a.use_smem ? smem : 0;
    cudaError_t e = cudaFuncSetAttribute(fps_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ctas);
    cfg.blockDim = dim3(kFpsThreads);
    cfg.dynamicSmemBytes = dyn;
    cfg.stream = s;
    cudaLaunchAttribute at;
    at.id = cudaLaunchAttributeClusterDimension;
    at.val.clusterDim.x = ctas;
    at.val.clusterDim.y = 1;
    at.val.clusterDim.z = 1;
    cfg.attrs = &at;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, fps_cluster_kernel, a);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace sop
