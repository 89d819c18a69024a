// Importance-sampled light directions for rendering (Sec. 4.2, Eq. PDF:
// density H W I / (4 pi) over the texels of the octahedral environment).
//   imp_max_kernel     intensity I_t = r + g + b of every texel (float32, in
//                      this order) and its maximum (float bits as uint: the
//                      intensities are >= 0, so the order is that of uint);
//   imp_scan_kernel    one CTA: q_t = max(1, floor(I_t / I_max 2^20)) in
//                      double (the same decision on every machine), and the
//                      inclusive prefix sums C_t as int64;
//   imp_sample_kernel  sample i takes the texel whose interval [C_{t-1}, C_t)
//                      holds floor((2i + 1) Q / (2S)) (exact integers), its
//                      centre direction (double, rounded once) and density
//                      H^2 q_t / (4 pi Q).
#include <math.h>

#include "sop_device.cuh"
#include "sop_internal.h"

namespace sop {

__global__ void imp_reset_kernel(unsigned int* imax) { *imax = 0u; }

__global__ void imp_max_kernel(const float* __restrict__ env, int64_t T, unsigned int* __restrict__ imax)
{
    unsigned int best = 0u;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < T; t += (int64_t)gridDim.x * blockDim.x) {
        const float I = env[3 * t] + env[3 * t + 1] + env[3 * t + 2];
        const unsigned int b = __float_as_uint(fmaxf(I, 0.f));
        best = b > best ? b : best;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned int v = __shfl_xor_sync(0xffffffffu, best, o);
        best = v > best ? v : best;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(imax, best);
}

__device__ __forceinline__ int64_t imp_q(const float* __restrict__ env, int64_t t, double imax)
{
    const float I = env[3 * t] + env[3 * t + 1] + env[3 * t + 2];
    const int64_t q = imax > 0.0 ? (int64_t)floor((double)I / imax * 1048576.0) : 1;
    return q < 1 ? 1 : q;
}

// one CTA of 1024 threads: a contiguous chunk of texels per thread
__global__ void __launch_bounds__(1024) imp_scan_kernel(const float* __restrict__ env, int64_t T,
                                                        const unsigned int* __restrict__ imax_bits,
                                                        int64_t* __restrict__ cum)
{
    __shared__ int64_t s_part[1024];
    const int tid = threadIdx.x, nt = blockDim.x;
    const double imax = (double)__uint_as_float(*imax_bits);
    const int64_t chunk = (T + nt - 1) / nt, c0 = tid * chunk, c1 = min(T, c0 + chunk);
    int64_t sum = 0;
    for (int64_t t = c0; t < c1; ++t) sum += imp_q(env, t, imax);
    s_part[tid] = sum;
    __syncthreads();
    for (int off = 1; off < nt; off <<= 1) {
        const int64_t v = tid >= off ? s_part[tid - off] : 0;
        __syncthreads();
        s_part[tid] += v;
        __syncthreads();
    }
    int64_t run = s_part[tid] - sum;
    for (int64_t t = c0; t < c1; ++t) {
        run += imp_q(env, t, imax);
        cum[t] = run;
    }
}

__global__ void imp_sample_kernel(const int64_t* __restrict__ cum, int32_t H, int32_t S, float4* __restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= S) return;
    const int64_t T = (int64_t)H * H, Q = cum[T - 1];
    const int64_t target = (2 * (int64_t)i + 1) * Q / (2 * (int64_t)S);
    int64_t lo = 0, hi = T - 1;  // smallest t with cum[t] > target
    while (lo < hi) {
        const int64_t mid = (lo + hi) / 2;
        if (cum[mid] > target) hi = mid;
        else lo = mid + 1;
    }
    const int64_t q = cum[lo] - (lo > 0 ? cum[lo - 1] : 0);
    double d[3];
    oct_decode_centre_f64(H, (int)(lo % H), (int)(lo / H), d);
    const double pdf = (double)T * (double)q / (4.0 * 3.14159265358979323846 * (double)Q);
    out[i] = make_float4((float)d[0], (float)d[1], (float)d[2], (float)pdf);
}

size_t importance_ws_bytes(int32_t H)
{
    return align256(sizeof(unsigned int)) + align256(sizeof(int64_t) * (size_t)H * H);
}

cudaError_t launch_importance_dirs(const float* env, int32_t H, int32_t S, float* out, char* ws, cudaStream_t s)
{
    unsigned int* imax = reinterpret_cast<unsigned int*>(ws);
    int64_t* cum = reinterpret_cast<int64_t*>(ws + align256(sizeof(unsigned int)));
    const int64_t T = (int64_t)H * H;
    imp_reset_kernel<<<1, 1, 0, s>>>(imax);
    const int64_t nb = (T + 255) / 256;
    imp_max_kernel<<<(unsigned)(nb < 1024 ? nb : 1024), 256, 0, s>>>(env, T, imax);
    imp_scan_kernel<<<1, 1024, 0, s>>>(env, T, imax, cum);
    imp_sample_kernel<<<(unsigned)((S + 127) / 128), 128, 0, s>>>(cum, H, S, reinterpret_cast<float4*>(out));
    return cudaGetLastError();
}

}  // namespace sop
