// The deferred steps around the G-buffer trace (Sec. 4.3, rendering; the
// G-buffers themselves are traced by trace_kernel<kTraceGbuf>) for sm_103a:
//   pinhole_dirs_kernel    per-pixel ray directions of a pinhole camera
//   panorama_dirs_kernel   per-pixel directions of an equirectangular
//                          panorama (the 360 degree sweep of Sec. 4.2)
//   points_*_kernel        the shading points of a G-buffer's kept pixels
//                          (position from the unbiased depth D/W of Sec. 3.1,
//                          normal N/|N|, materials per unit weight),
//                          compacted in pixel order: count per CTA, scan of
//                          the counts, write (deterministic)
//   comp_*_kernel          depth compositing: the scene colour, times its
//                          shadow ratio (Eq. 9), the relit object over it
// All are HBM streams of a few bytes per pixel.
#include <math.h>

#include "sop_device.cuh"
#include "sop_internal.h"

namespace sop {

// The camera's frame is set up on the host in double and rounded once; the
// per-pixel directions are FP32 (a few ulp of a unit vector).
struct CamK {
    float f[3], r[3], u[3];  // unit forward, right, up; r and u scaled by tan(fov/2) (aspect on r)
    float inv_w2, inv_h2;    // 2 / W, 2 / H
    int32_t W, H;
};

__global__ void pinhole_dirs_kernel(const CamK c, float4* __restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)c.W * c.H) return;
    const int px = (int)(i % c.W), py = (int)(i / c.W);
    const float sx = fmaf((float)px + 0.5f, c.inv_w2, -1.f);
    const float sy = fmaf(-((float)py + 0.5f), c.inv_h2, 1.f);
    const float v0 = fmaf(sy, c.u[0], fmaf(sx, c.r[0], c.f[0]));
    const float v1 = fmaf(sy, c.u[1], fmaf(sx, c.r[1], c.f[1]));
    const float v2 = fmaf(sy, c.u[2], fmaf(sx, c.r[2], c.f[2]));
    const float il = rsqrtf(fmaf(v0, v0, fmaf(v1, v1, v2 * v2)));
    out[i] = make_float4(v0 * il, v1 * il, v2 * il, 0.f);
}

// Equirectangular directions in FP32: sincospif of the polar and azimuthal
// angles in units of pi.
__global__ void panorama_dirs_kernel(int32_t W, int32_t H, float4* __restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)W * H) return;
    const int px = (int)(i % W), py = (int)(i / W);
    const float ph = (2.f * (float)px + 1.f - (float)W) / (float)W;  // azimuth / pi (exact numerator)
    const float th = (2.f * (float)py + 1.f) / (2.f * (float)H);        // polar angle / pi
    float st, ct, sp, cp;
    sincospif(th, &st, &ct);
    sincospif(ph, &sp, &cp);
    out[i] = make_float4(st * cp, st * sp, ct, 0.f);
}

struct PointsK {
    const float4* gbuf;   // [n][4]: (C, W), (N, D), (A, R), (M, -, -, -)
    const float4* front;  // another G-buffer that hides what lies behind it, or NULL
    const float4* dirs;
    int64_t n;
    float ox, oy, oz, w_min;
    int32_t* block_cnt;  // [blocks] counts, then exclusive offsets
    int64_t* pix;
    float *x, *nrm, *wo, *albedo, *rough, *metal;
    int64_t* count;
};

constexpr int kPointsBlock = 1024;

// kept: W >= w_min, N != 0, and in front of `front` where that one is kept
// (the unbiased depths compared as float32 quotients)
__device__ __forceinline__ bool point_kept(const PointsK& k, int64_t p)
{
    if (p >= k.n) return false;
    const float4 b0 = __ldg(k.gbuf + 4 * p), b1 = __ldg(k.gbuf + 4 * p + 1);
    if (!(b0.w >= k.w_min)) return false;
    if (!(b1.x != 0.f || b1.y != 0.f || b1.z != 0.f)) return false;
    if (k.front) {
        const float4 f0 = __ldg(k.front + 4 * p), f1 = __ldg(k.front + 4 * p + 1);
        if (f0.w >= k.w_min && !(b1.w / b0.w < f1.w / f0.w)) return false;
    }
    return true;
}

__global__ void __launch_bounds__(kPointsBlock) points_count_kernel(const PointsK k)
{
    const int64_t p = (int64_t)blockIdx.x * kPointsBlock + threadIdx.x;
    const int c = __syncthreads_count(point_kept(k, p));
    if (threadIdx.x == 0) k.block_cnt[blockIdx.x] = c;
}

// one CTA: exclusive offsets of the per-CTA counts, and the total
__global__ void __launch_bounds__(1024) points_scan_kernel(int32_t* __restrict__ cnt, int64_t nb,
                                                           int64_t* __restrict__ count)
{
    __shared__ int64_t s_part[1024];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int64_t chunk = (nb + nt - 1) / nt, c0 = tid * chunk, c1 = min(nb, c0 + chunk);
    int64_t sum = 0;
    for (int64_t b = c0; b < c1; ++b) sum += cnt[b];
    s_part[tid] = sum;
    __syncthreads();
    for (int off = 1; off < nt; off <<= 1) {
        const int64_t v = tid >= off ? s_part[tid - off] : 0;
        __syncthreads();
        s_part[tid] += v;
        __syncthreads();
    }
    int64_t run = s_part[tid] - sum;
    for (int64_t b = c0; b < c1; ++b) {
        const int32_t v = cnt[b];
        cnt[b] = (int32_t)run;  // offsets fit: fewer than 2^31 pixels
        run += v;
    }
    if (tid == nt - 1) *count = s_part[nt - 1];
}

__global__ void __launch_bounds__(kPointsBlock) points_write_kernel(const PointsK k)
{
    __shared__ int s_warp[kPointsBlock / 32];
    const int64_t p = (int64_t)blockIdx.x * kPointsBlock + threadIdx.x;
    const bool keep = point_kept(k, p);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    if (lane == 0) s_warp[wid] = __popc(m);
    __syncthreads();
    if (wid == 0) {
        int v = s_warp[lane];
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, v, off);
            if (lane >= off) v += u;
        }
        s_warp[lane] = v - s_warp[lane];  // exclusive
    }
    __syncthreads();
    if (!keep) return;
    const int64_t j = (int64_t)k.block_cnt[blockIdx.x] + s_warp[wid] + __popc(m & ((1u << lane) - 1u));
    const float4 b0 = __ldg(k.gbuf + 4 * p), b1 = __ldg(k.gbuf + 4 * p + 1), b2 = __ldg(k.gbuf + 4 * p + 2),
                 b3 = __ldg(k.gbuf + 4 * p + 3);
    const float4 d = __ldg(k.dirs + p);
    const float W = b0.w, t = b1.w / W;
    const float il = 1.f / sqrtf(b1.x * b1.x + b1.y * b1.y + b1.z * b1.z);
    k.pix[j] = p;
    k.x[3 * j] = fmaf(t, d.x, k.ox);
    k.x[3 * j + 1] = fmaf(t, d.y, k.oy);
    k.x[3 * j + 2] = fmaf(t, d.z, k.oz);
    k.nrm[3 * j] = b1.x * il;
    k.nrm[3 * j + 1] = b1.y * il;
    k.nrm[3 * j + 2] = b1.z * il;
    k.wo[3 * j] = -d.x;
    k.wo[3 * j + 1] = -d.y;
    k.wo[3 * j + 2] = -d.z;
    k.albedo[3 * j] = b2.x / W;
    k.albedo[3 * j + 1] = b2.y / W;
    k.albedo[3 * j + 2] = b2.z / W;
    k.rough[j] = b2.w / W;
    k.metal[j] = b3.x / W;
}

__global__ void comp_scene_kernel(const float4* __restrict__ sg, int64_t n, float* __restrict__ out)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const float4 c = __ldg(sg + 4 * p);
    out[3 * p] = c.x;
    out[3 * p + 1] = c.y;
    out[3 * p + 2] = c.z;
}

// pixel lists come from the compaction (distinct pixels); others are skipped
__global__ void comp_shadow_kernel(const int64_t* __restrict__ pix, const float* __restrict__ S, int64_t n_sc,
                                   int64_t n, float* __restrict__ out, unsigned int* status)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_sc) return;
    const int64_t p = pix[k];
    if (p < 0 || p >= n) {
        if (status) atomicOr(status, SOP_DEVSTAT_INDEX);
        return;
    }
    out[3 * p] *= S[3 * k];
    out[3 * p + 1] *= S[3 * k + 1];
    out[3 * p + 2] *= S[3 * k + 2];
}

__global__ void comp_object_kernel(const float4* __restrict__ og, const int64_t* __restrict__ pix,
                                   const float* __restrict__ rgb, int64_t n_obj, int64_t n, float* __restrict__ out,
                                   unsigned int* status)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_obj) return;
    const int64_t p = pix[k];
    if (p < 0 || p >= n) {
        if (status) atomicOr(status, SOP_DEVSTAT_INDEX);
        return;
    }
    const float a = __ldg(og + 4 * p).w;
    for (int c = 0; c < 3; ++c) out[3 * p + c] = fmaf(a, rgb[3 * k + c], (1.f - a) * out[3 * p + c]);
}

static unsigned blocks_for(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

cudaError_t launch_pinhole_dirs(int32_t W, int32_t H, const float* eye, const float* target, const float* up,
                                float fov_y_deg, float* out, cudaStream_t s)
{
    CamK c;
    double f[3], uu[3];
    for (int a = 0; a < 3; ++a) {
        f[a] = (double)target[a] - eye[a];
        uu[a] = up[a];
    }
    const double fl = sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
    for (int a = 0; a < 3; ++a) f[a] /= fl;
    const double ul = sqrt(uu[0] * uu[0] + uu[1] * uu[1] + uu[2] * uu[2]);
    // an up vector (nearly) along the view: take y instead
    if (fabs((f[0] * uu[0] + f[1] * uu[1] + f[2] * uu[2]) / ul) > 0.99) {
        uu[0] = 0.0;
        uu[1] = 1.0;
        uu[2] = 0.0;
    }
    double r[3] = {f[1] * uu[2] - f[2] * uu[1], f[2] * uu[0] - f[0] * uu[2], f[0] * uu[1] - f[1] * uu[0]};
    const double rl = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    for (int a = 0; a < 3; ++a) r[a] /= rl;
    const double u[3] = {r[1] * f[2] - r[2] * f[1], r[2] * f[0] - r[0] * f[2], r[0] * f[1] - r[1] * f[0]};
    const double th = tan((double)fov_y_deg * 3.14159265358979323846 / 360.0);
    const double aspect = (double)W / H;
    for (int a = 0; a < 3; ++a) {
        c.f[a] = (float)f[a];
        c.r[a] = (float)(r[a] * th * aspect);
        c.u[a] = (float)(u[a] * th);
    }
    c.inv_w2 = (float)(2.0 / W);
    c.inv_h2 = (float)(2.0 / H);
    c.W = W;
    c.H = H;
    pinhole_dirs_kernel<<<blocks_for((int64_t)W * H, 256), 256, 0, s>>>(c, reinterpret_cast<float4*>(out));
    return cudaGetLastError();
}

cudaError_t launch_panorama_dirs(int32_t W, int32_t H, float* out, cudaStream_t s)
{
    panorama_dirs_kernel<<<blocks_for((int64_t)W * H, 256), 256, 0, s>>>(W, H, reinterpret_cast<float4*>(out));
    return cudaGetLastError();
}

size_t points_ws_bytes(int64_t n_pix) { return align256(sizeof(int32_t) * (size_t)(blocks_for(n_pix, kPointsBlock) + 1)); }

cudaError_t launch_gbuffer_points(const float* gbuf, const float* front, int64_t n, const float* origin,
                                  const float* dirs, float w_min, int64_t* pix, float* x, float* nrm, float* wo,
                                  float* albedo, float* rough, float* metal, int64_t* count, char* ws, cudaStream_t s)
{
    PointsK k;
    k.gbuf = reinterpret_cast<const float4*>(gbuf);
    k.front = reinterpret_cast<const float4*>(front);
    k.dirs = reinterpret_cast<const float4*>(dirs);
    k.n = n;
    k.ox = origin[0];
    k.oy = origin[1];
    k.oz = origin[2];
    k.w_min = w_min;
    k.block_cnt = reinterpret_cast<int32_t*>(ws);
    k.pix = pix;
    k.x = x;
    k.nrm = nrm;
    k.wo = wo;
    k.albedo = albedo;
    k.rough = rough;
    k.metal = metal;
    k.count = count;
    const unsigned nb = blocks_for(n, kPointsBlock);
    if (nb == 0) {
        cudaMemsetAsync(count, 0, sizeof(int64_t), s);
        return cudaGetLastError();
    }
    points_count_kernel<<<nb, kPointsBlock, 0, s>>>(k);
    points_scan_kernel<<<1, 1024, 0, s>>>(k.block_cnt, nb, count);
    points_write_kernel<<<nb, kPointsBlock, 0, s>>>(k);
    return cudaGetLastError();
}

cudaError_t launch_depth_composite(const float* scene_gbuf, const float* obj_gbuf, int64_t n, const int64_t* sc_pix,
                                   const float* shadow, int64_t n_sc, const int64_t* obj_pix, const float* obj_rgb,
                                   int64_t n_obj, float* out, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    comp_scene_kernel<<<blocks_for(n, 256), 256, 0, s>>>(reinterpret_cast<const float4*>(scene_gbuf), n, out);
    unsigned int* status = status_word();
    if (n_sc > 0) comp_shadow_kernel<<<blocks_for(n_sc, 256), 256, 0, s>>>(sc_pix, shadow, n_sc, n, out, status);
    if (n_obj > 0)
        comp_object_kernel<<<blocks_for(n_obj, 256), 256, 0, s>>>(reinterpret_cast<const float4*>(obj_gbuf), obj_pix,
                                                                  obj_rgb, n_obj, n, out, status);
    return cudaGetLastError();
}

}  // namespace sop
