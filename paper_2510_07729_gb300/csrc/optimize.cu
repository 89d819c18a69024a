// Pieces of one step of the SOP texture optimisation (Sec. 3.1.2, second
// reconstruction step: L = L_pbr + lambda_lam L_lam + lambda_sops L_sops,
// Adam) for sm_103a. The shading and its gradient come from the query and
// its adjoint; this file adds
//   l1_grad_kernel   dL/dC of the mean absolute error between the shaded
//                    colours and the target (and the summed |C - C_t|);
//   adam_l1_kernel   for one parameter block: add the gradient of an L1
//                    regulariser toward a target (array or value), take a
//                    bias-corrected Adam step, clamp to the block's range.
// Both are elementwise over grid-stride loops: HBM-bound streams.
#include <math.h>

#include "sop_device.cuh"
#include "sop_internal.h"

namespace sop {

__global__ void l1_grad_kernel(const float* __restrict__ C, const float* __restrict__ Ct, int64_t n, float inv_n,
                               float* __restrict__ grad, float* __restrict__ loss_sum)
{
    float s = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float d = C[i] - Ct[i];
        grad[i] = d > 0.f ? inv_n : (d < 0.f ? -inv_n : 0.f);
        s += fabsf(d);
    }
    if (loss_sum) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(loss_sum, s);
    }
}

struct AdamK {
    float lr, b1, b2, eps, bc1, bc2;  // bc: 1 - beta^t
    const float* target;
    float target_value;
    int32_t period, split;
    float lam[2], lo[2], hi[2];
};

__global__ void adam_l1_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                               float* __restrict__ v, int64_t n, const AdamK k)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        // elements i with i % period < split take the first set of settings
        const int set = (int)(i % k.period) < k.split ? 0 : 1;
        const float pi = p[i];
        const float tg = k.target ? k.target[i] : k.target_value;
        const float d = pi - tg;
        const float gt = (g ? g[i] : 0.f) + k.lam[set] * (d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f));
        const float mi = k.b1 * m[i] + (1.f - k.b1) * gt;
        const float vi = k.b2 * v[i] + (1.f - k.b2) * gt * gt;
        m[i] = mi;
        v[i] = vi;
        const float q = pi - k.lr * (mi / k.bc1) / (sqrtf(vi / k.bc2) + k.eps);
        p[i] = fminf(fmaxf(q, k.lo[set]), k.hi[set]);
    }
}

static unsigned stream_blocks(int64_t n)
{
    const int64_t b = (n + 255) / 256;
    return (unsigned)(b < 152 * 16 ? (b > 0 ? b : 1) : 152 * 16);
}

cudaError_t launch_l1_grad(const float* C, const float* Ct, int64_t n, float* grad, float* loss_sum, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    l1_grad_kernel<<<stream_blocks(n), 256, 0, s>>>(C, Ct, n, 1.f / (float)n, grad, loss_sum);
    return cudaGetLastError();
}

cudaError_t launch_adam_l1(float* p, const float* g, float* m, float* v, int64_t n, const sop_adam_params& a,
                           cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    AdamK k;
    k.lr = a.lr;
    k.b1 = a.beta1;
    k.b2 = a.beta2;
    k.eps = a.eps;
    // bias corrections in double, rounded once
    k.bc1 = (float)(1.0 - pow((double)a.beta1, (double)a.step));
    k.bc2 = (float)(1.0 - pow((double)a.beta2, (double)a.step));
    k.target = a.target;
    k.target_value = a.target_value;
    k.period = a.period;
    k.split = a.split;
    for (int j = 0; j < 2; ++j) {
        k.lam[j] = a.lam[j];
        k.lo[j] = a.lo[j];
        k.hi[j] = a.hi[j];
    }
    adam_l1_kernel<<<stream_blocks(n), 256, 0, s>>>(p, g, m, v, n, k);
    return cudaGetLastError();
}

}  // namespace sop
