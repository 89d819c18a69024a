// Device-side building blocks of libsop (sm_103a). Internal header: every
// function is static inline, so each translation unit carries its own copy.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <float.h>
#include <stdint.h>

#include "sop.h"

namespace sop {

constexpr float kPi = 3.14159265358979323846f;
constexpr float kInvPi = 0.318309886183790671538f;
constexpr float kInv2Pi = 0.159154943091895335769f;

__device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return f3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ float3 cross3(float3 a, float3 b)
{
    return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float3 load3(const float* p, int64_t i)
{
    return f3(__ldg(p + 3 * i), __ldg(p + 3 * i + 1), __ldg(p + 3 * i + 2));
}

// ---------------------------------------------------------------------------
// Octahedral map (Sec. 3.1.2 octahedral textures; Cigolle et al. 2014 form,
// z-up, world frame). Unit direction -> uv in [0,1]^2.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 oct_encode(float3 d)
{
    float l1 = fabsf(d.x) + fabsf(d.y) + fabsf(d.z);
    const float inv = __fdividef(1.f, l1);
    float px = d.x * inv, py = d.y * inv;
    if (d.z < 0.f) {
        float qx = (1.f - fabsf(py)) * (px >= 0.f ? 1.f : -1.f);
        float qy = (1.f - fabsf(px)) * (py >= 0.f ? 1.f : -1.f);
        px = qx;
        py = qy;
    }
    return make_float2(0.5f * (px + 1.f), 0.5f * (py + 1.f));
}

// Double-precision decode of a texel centre (used once per call to build
// correctly rounded float direction tables).
__device__ __forceinline__ void oct_decode_centre_f64(int R, int i, int j, double* d)
{
    double px = 2.0 * ((i + 0.5) / R) - 1.0, py = 2.0 * ((j + 0.5) / R) - 1.0;
    double z = 1.0 - fabs(px) - fabs(py);
    if (z < 0.0) {
        double qx = (1.0 - fabs(py)) * (px >= 0.0 ? 1.0 : -1.0);
        double qy = (1.0 - fabs(px)) * (py >= 0.0 ? 1.0 : -1.0);
        px = qx;
        py = qy;
    }
    double n = sqrt(px * px + py * py + z * z);
    d[0] = px / n;
    d[1] = py / n;
    d[2] = z / n;
}

// Border rule for the gutter: texel index pair in [-1, R]^2 -> source texel.
__device__ __forceinline__ void oct_wrap(int R, int i, int j, int& si, int& sj)
{
    bool oi = (i < 0) || (i >= R), oj = (j < 0) || (j >= R);
    if (oi && oj) {
        si = (i < 0) ? R - 1 : 0;
        sj = (j < 0) ? R - 1 : 0;
    } else if (oi) {
        si = (i < 0) ? 0 : R - 1;
        sj = R - 1 - j;
    } else if (oj) {
        si = R - 1 - i;
        sj = (j < 0) ? 0 : R - 1;
    } else {
        si = i;
        sj = j;
    }
}

// Orthonormal frame (t, b) of unit n (Duff et al. 2017, branchless form).
__device__ __forceinline__ void onb(float3 n, float3& t, float3& b)
{
    float sg = n.z >= 0.f ? 1.f : -1.f;
    float a = -1.f / (sg + n.z);
    float c = n.x * n.y * a;
    t = f3(1.f + sg * n.x * n.x * a, sg * c, -sg * n.x);
    b = f3(c, sg + n.y * n.y * a, -n.y);
}

// ---------------------------------------------------------------------------
// Atlas texel storage.
// ---------------------------------------------------------------------------
template <int DT> struct Texel;
template <> struct Texel<SOP_F32> {
    using raw = float4;
    static __device__ __forceinline__ float4 load(const raw* p) { return __ldg(p); }
    static __device__ __forceinline__ raw pack(float4 v) { return v; }
    static __device__ __forceinline__ bool finite(raw v) { return isfinite(v.x + v.y + v.z + v.w); }
};
template <> struct Texel<SOP_BF16> {
    using raw = uint2;
    static __device__ __forceinline__ float4 load(const raw* p)
    {
        uint2 r = __ldg(p);
        return make_float4(__uint_as_float(r.x << 16), __uint_as_float(r.x & 0xffff0000u), __uint_as_float(r.y << 16),
                           __uint_as_float(r.y & 0xffff0000u));
    }
    static __device__ __forceinline__ raw pack(float4 v)
    {
        __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y), b = __floats2bfloat162_rn(v.z, v.w);
        return make_uint2(*reinterpret_cast<uint32_t*>(&a), *reinterpret_cast<uint32_t*>(&b));
    }
    // no half has its exponent field all ones (Inf or NaN)
    static __device__ __forceinline__ bool finite(raw v)
    {
        return ((v.x >> 16) & 0x7f80u) != 0x7f80u && (v.x & 0x7f80u) != 0x7f80u && ((v.y >> 16) & 0x7f80u) != 0x7f80u &&
               (v.y & 0x7f80u) != 0x7f80u;
    }
};
template <> struct Texel<SOP_F16> {
    using raw = uint2;
    static __device__ __forceinline__ float4 load(const raw* p)
    {
        uint2 r = __ldg(p);
        __half2 a = *reinterpret_cast<__half2*>(&r.x), b = *reinterpret_cast<__half2*>(&r.y);
        float2 fa = __half22float2(a), fb = __half22float2(b);
        return make_float4(fa.x, fa.y, fb.x, fb.y);
    }
    static __device__ __forceinline__ raw pack(float4 v)
    {
        __half2 a = __floats2half2_rn(v.x, v.y), b = __floats2half2_rn(v.z, v.w);
        return make_uint2(*reinterpret_cast<uint32_t*>(&a), *reinterpret_cast<uint32_t*>(&b));
    }
    // no half has its exponent field all ones (Inf or NaN)
    static __device__ __forceinline__ bool finite(raw v)
    {
        return ((v.x >> 16) & 0x7c00u) != 0x7c00u && (v.x & 0x7c00u) != 0x7c00u && ((v.y >> 16) & 0x7c00u) != 0x7c00u &&
               (v.y & 0x7c00u) != 0x7c00u;
    }
};

// Scratch-space header written by the probe-grid build and read by the
// nearest-probe search.
struct ProbeGrid {
    int32_t qmin[3];
    int32_t cs;      // cell edge in quantised units (2^-20)
    int32_t dims[3];
    int32_t ncells;
};

// Uniform grid over Gaussian bounding spheres, for the bake.
struct GaussGrid {
    float origin[3];
    float h;         // cell edge (world units)
    float inv_h;
    float bmax[3];   // bounding box max (origin is the min)
    int32_t dims[3];
    int32_t ncells;
    int32_t n_entries;
    int32_t fits;    // 1 once the cell lists fit the workspace's entry capacity
    int32_t level;   // binning attempt that fitted (0: the requested grid)
    int32_t pad;
};

}  // namespace sop
