// Exclusive prefix sum of per-cell counts into cell offsets, over many CTAs
// (the grid builders' count -> start step). The number of cells lives on the
// device (the grid is set up there), so the host sizes the launches for an
// upper bound and CTAs past the real count return at once. Three launches:
//   scan_tile_sum_kernel: each CTA sums one tile of kScanTile counts;
//   scan_parts_kernel (one CTA): exclusive sum of the tile sums, the total,
//     and whether the pass runs at all (a device flag may say the cells are
//     already binned: the bake's later binning attempts);
//   scan_apply_kernel: each CTA scans its tile again, adds its tile's offset,
//     writes the starts and zeroes the counts (the fill pass counts again);
//     the CTA of the last tile writes start[n] and calls the finaliser with
//     the total.
// Counts are int32, sums int64 (the bake checks the total against its entry
// capacity); starts are clamped to INT32_MAX.
#pragma once
#include <cstdint>

namespace sop {

constexpr int kScanThreads = 1024;
constexpr int kScanPer = 4;
constexpr int kScanTile = kScanThreads * kScanPer;

// tiles (CTAs) for at most n cells, and the int64 scratch the scan needs
inline unsigned scan_tiles(int64_t n) { return (unsigned)((n + kScanTile - 1) / kScanTile); }
inline size_t scan_scratch_count(int64_t n) { return (size_t)scan_tiles(n) + 2; }

// scratch: [0] run flag (1: scan), [1] total, [2 + i] tile i's sum/offset
struct ScanArgs {
    const int32_t* n;     // number of cells (device)
    const int32_t* skip;  // when not NULL and *skip != 0 the pass does nothing
    int32_t* cnt;         // [n] counts (zeroed by the apply pass)
    int32_t* start;       // [n + 1] exclusive offsets
    long long* scratch;
};

// inclusive block sum of one value per thread; returns it and leaves the
// block total in *total (shared scratch of kScanThreads / 32 entries)
static __device__ __forceinline__ long long scan_block_inclusive(long long v, long long* warp_sums, long long* total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const long long u = __shfl_up_sync(0xffffffffu, v, off);
        if (lane >= off) v += u;
    }
    if (lane == 31) warp_sums[warp] = v;
    __syncthreads();
    if (warp == 0) {
        long long w = lane < kScanThreads / 32 ? warp_sums[lane] : 0;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const long long u = __shfl_up_sync(0xffffffffu, w, off);
            if (lane >= off) w += u;
        }
        if (lane < kScanThreads / 32) warp_sums[lane] = w;
    }
    __syncthreads();
    const long long r = v + (warp > 0 ? warp_sums[warp - 1] : 0);
    *total = warp_sums[kScanThreads / 32 - 1];
    return r;
}

static __global__ void __launch_bounds__(kScanThreads) scan_tile_sum_kernel(ScanArgs a)
{
    __shared__ long long s_w[kScanThreads / 32];
    if (a.skip && *a.skip) return;
    const int n = *a.n;
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    if (base >= n) return;
    long long v = 0;
#pragma unroll
    for (int e = 0; e < kScanPer; ++e) {
        const int64_t i = base + (int64_t)threadIdx.x * kScanPer + e;
        if (i < n) v += a.cnt[i];
    }
    long long tot;
    scan_block_inclusive(v, s_w, &tot);
    if (threadIdx.x == 0) a.scratch[2 + blockIdx.x] = tot;
}

static __global__ void __launch_bounds__(kScanThreads) scan_parts_kernel(ScanArgs a)
{
    __shared__ long long s_w[kScanThreads / 32];
    __shared__ long long s_carry;
    const bool run = !(a.skip && *a.skip);
    if (threadIdx.x == 0) {
        a.scratch[0] = run ? 1 : 0;
        s_carry = 0;
    }
    if (!run) return;
    const int n = *a.n;
    const int tiles = (int)((n + kScanTile - 1) / kScanTile);
    __syncthreads();
    for (int t0 = 0; t0 < tiles; t0 += kScanThreads) {
        const int t = t0 + threadIdx.x;
        const long long v = t < tiles ? a.scratch[2 + t] : 0;
        long long tot;
        const long long inc = scan_block_inclusive(v, s_w, &tot);
        const long long carry = s_carry;
        if (t < tiles) a.scratch[2 + t] = carry + inc - v;
        __syncthreads();
        if (threadIdx.x == 0) s_carry = carry + tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) a.scratch[1] = s_carry;
}

struct ScanNoFinal {
    __device__ void operator()(long long) const {}
};

template <class Fin>
static __global__ void __launch_bounds__(kScanThreads) scan_apply_kernel(ScanArgs a, Fin fin)
{
    __shared__ long long s_w[kScanThreads / 32];
    if (a.scratch[0] == 0) return;
    const int n = *a.n;
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    if (base >= n) {
        if (n == 0 && blockIdx.x == 0 && threadIdx.x == 0) {  // no cells: start[0] = 0
            a.start[0] = 0;
            fin(0ll);
        }
        return;
    }
    int32_t c[kScanPer];
    long long v = 0;
#pragma unroll
    for (int e = 0; e < kScanPer; ++e) {
        const int64_t i = base + (int64_t)threadIdx.x * kScanPer + e;
        c[e] = i < n ? a.cnt[i] : 0;
        v += c[e];
    }
    long long tot;
    long long run = scan_block_inclusive(v, s_w, &tot) - v + a.scratch[2 + blockIdx.x];
#pragma unroll
    for (int e = 0; e < kScanPer; ++e) {
        const int64_t i = base + (int64_t)threadIdx.x * kScanPer + e;
        if (i < n) {
            a.start[i] = (int32_t)(run < INT32_MAX ? run : INT32_MAX);
            a.cnt[i] = 0;
        }
        run += c[e];
    }
    if (base + kScanTile >= n && threadIdx.x == 0) {
        const long long total = a.scratch[1];
        a.start[n] = (int32_t)(total < INT32_MAX ? total : INT32_MAX);
        fin(total);
    }
}

// the three launches for at most n_max cells
template <class Fin>
inline void launch_scan(const ScanArgs& a, int64_t n_max, Fin fin, cudaStream_t s)
{
    const unsigned nb = scan_tiles(n_max > 0 ? n_max : 1);
    scan_tile_sum_kernel<<<nb, kScanThreads, 0, s>>>(a);
    scan_parts_kernel<<<1, kScanThreads, 0, s>>>(a);
    scan_apply_kernel<<<nb, kScanThreads, 0, s>>>(a, fin);
}

}  // namespace sop
