// Learned bake surrogate for sm_103a: a small MLP that predicts a probe's
// octahedral maps (O, D/depth_scale, RGB) from the probe's 32 nearest
// Gaussians and the texel direction, so probes can be rebaked fast after an
// object moves. The ray-traced bake stays its fallback and its judge.
//
//   f_p (416)  = 32 nearest Gaussians (nearest first) x [(mu - p) * 10,
//                log(scale) + 5, opacity, rgb], then sin/cos of
//                pi 2^(f/3) p_axis for f = 0..15
//   h1 = relu(W1p f_p + W1d d_t + b1)   (the f_p part once per probe)
//   h2 = relu(W2 h1 + b2), h3 = relu(W3 h2 + b3), y = W4 h3 + b4 (5 outputs)
//
// Weights are used as bfloat16 with float32 accumulation; float32 master
// weights and Adam moments live in the caller's state buffer. The two
// 64x64 layers run on the tensor cores (mma.sync m16n8k16 bf16 -> f32) in
// the forward pass, in the back-propagation of deltas and in the weight
// gradients (sums over samples); the small layers (416 -> 64 per probe,
// 3 -> 64, 64 -> 5) are plain FP32 FMA.
#include "sop_device.cuh"
#include "sop_internal.h"

namespace sop {

constexpr int kNeigh = 32;
constexpr int kNFreq = 16;
constexpr int kFP = kNeigh * 10 + 6 * kNFreq;  // 416
constexpr int kHid = 64;
constexpr int kOut = 5;
// flat parameter blocks (row-major, out x in)
constexpr int oW1p = 0, oW1d = oW1p + kHid * kFP, ob1 = oW1d + kHid * 3, oW2 = ob1 + kHid, ob2 = oW2 + kHid * kHid,
              oW3 = ob2 + kHid, ob3 = oW3 + kHid * kHid, oW4 = ob3 + kHid, ob4 = oW4 + kOut * kHid,
              kNParam = ob4 + kOut;

// Caller-owned state: master weights, Adam moments, gradient accumulator,
// bf16 copy of the parameters (biases included, unused as bf16), step.
struct SurrState {
    size_t master, m, v, grad, wbf, step, loss, total;
};
SurrState surr_state_layout()
{
    SurrState S{};
    size_t o = 0;
    S.master = o; o = align256(o + sizeof(float) * kNParam);
    S.m = o;      o = align256(o + sizeof(float) * kNParam);
    S.v = o;      o = align256(o + sizeof(float) * kNParam);
    S.grad = o;   o = align256(o + sizeof(float) * kNParam);
    S.wbf = o;    o = align256(o + sizeof(uint16_t) * kNParam);
    S.step = o;   o = align256(o + sizeof(int32_t) * 4);
    S.loss = o;   o = align256(o + sizeof(float) * 4);
    S.total = o;
    return S;
}
int surr_n_params() { return kNParam; }
size_t surr_state_bytes() { return surr_state_layout().total; }

__device__ __forceinline__ uint16_t f2bf(float x)
{
    __nv_bfloat16 b = __float2bfloat16_rn(x);
    return *reinterpret_cast<uint16_t*>(&b);
}
__device__ __forceinline__ float bf2f(uint16_t u) { return __uint_as_float((uint32_t)u << 16); }
__device__ __forceinline__ float rbf(float x) { return bf2f(f2bf(x)); }

// bf16 copy of the master weights
__global__ void surr_to_bf16_kernel(const float* __restrict__ master, uint16_t* __restrict__ wbf)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kNParam) wbf[i] = f2bf(master[i]);
}

__global__ void surr_reset_kernel(float* m, float* v, int32_t* step)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kNParam) {
        m[i] = 0.f;
        v[i] = 0.f;
    }
    if (i == 0) step[0] = 0;
}

// Adam (Kingma & Ba 2015): beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected.
__global__ void surr_adam_kernel(float* __restrict__ master, float* __restrict__ m, float* __restrict__ v,
                                 const float* __restrict__ grad, uint16_t* __restrict__ wbf, const int32_t* step,
                                 float lr)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kNParam) return;
    const int t = step[0] + 1;
    const float g = grad[i];
    const float mi = 0.9f * m[i] + 0.1f * g;
    const float vi = 0.999f * v[i] + 0.001f * g * g;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / (1.f - powf(0.9f, (float)t)), vh = vi / (1.f - powf(0.999f, (float)t));
    const float w = master[i] - lr * mh / (sqrtf(vh) + 1e-8f);
    master[i] = w;
    wbf[i] = f2bf(w);
}

__global__ void surr_step_kernel(int32_t* step) { step[0] += 1; }

// Probe features from the 32 nearest Gaussians (idx [P,32], nearest first).
__global__ void surr_features_kernel(sop_gaussians g, const float* __restrict__ probe_pos, int32_t P,
                                     const int32_t* __restrict__ idx, float* __restrict__ feats)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)P * kFP) return;
    const int64_t p = i / kFP;
    const int f = (int)(i % kFP);
    // computed in double and rounded once, so that the bf16 rounding the
    // network applies to each feature sees the correctly rounded value
    const double pp[3] = {probe_pos[3 * p], probe_pos[3 * p + 1], probe_pos[3 * p + 2]};
    double v;
    if (f < kNeigh * 10) {
        const int j = f / 10, c = f % 10;
        const int64_t gi = idx[p * kNeigh + j];
        if (c < 3) v = ((double)g.mean[3 * gi + c] - pp[c]) * 10.0;
        else if (c < 6) v = log((double)g.scale[3 * gi + c - 3]) + 5.0;
        else if (c == 6) v = g.opacity[gi];
        else v = g.rgb[3 * gi + c - 7];
    } else {
        const int e = f - kNeigh * 10, ax = e / 32, r = e % 32, fr = r % 16;
        const double arg = pp[ax] * (3.14159265358979323846 * exp2((double)fr / 3.0));
        v = r < 16 ? sin(arg) : cos(arg);
    }
    feats[i] = (float)v;
}

// h1p[b] = W1p bf16(f_{pid[b]}) + b1, one thread per (probe, output).
__global__ void surr_l1_fwd_kernel(const float* __restrict__ feats, const int32_t* __restrict__ pid, int32_t B,
                                   const uint16_t* __restrict__ wbf, const float* __restrict__ master,
                                   float* __restrict__ h1p)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)B * kHid) return;
    const int64_t b = i / kHid;
    const int o = (int)(i % kHid);
    const int64_t p = pid ? pid[b] : b;
    const float* f = feats + p * kFP;
    const uint16_t* w = wbf + oW1p + o * kFP;
    float acc = 0.f;
    for (int k = 0; k < kFP; ++k) acc = fmaf(bf2f(w[k]), rbf(f[k]), acc);
    h1p[i] = acc + master[ob1 + o];
}

// dW1p[o][k] += sum_b dh1p[b][o] bf16(f_{pid[b]})[k], db1 via the texel kernel.
__global__ void surr_l1_bwd_kernel(const float* __restrict__ feats, const int32_t* __restrict__ pid, int32_t B,
                                   const float* __restrict__ dh1p, float* __restrict__ grad)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kHid * kFP) return;
    const int o = i / kFP, k = i % kFP;
    float acc = 0.f;
    for (int b = 0; b < B; ++b) {
        const int64_t p = pid ? pid[b] : b;
        acc = fmaf(dh1p[(int64_t)b * kHid + o], rbf(feats[p * kFP + k]), acc);
    }
    grad[oW1p + i] += acc;
}

// ---------------------------------------------------------------------------
// Tensor-core helpers: mma.sync m16n8k16, bf16 inputs, f32 accumulators.
// Fragment layout (g = lane / 4, t = lane % 4): A rows g and g+8, columns
// 2t, 2t+1 (+8); B rows (k) 2t, 2t+1 (+8), column g; C rows g, g+8, columns
// 2t, 2t+1. A bf16x2 register holds the lower column / row in its low half.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mma_bf16(float* c, const uint32_t* a, const uint32_t* b)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
__device__ __forceinline__ uint32_t pk(uint16_t lo, uint16_t hi) { return (uint32_t)lo | ((uint32_t)hi << 16); }
__device__ __forceinline__ uint32_t ld2(const uint16_t* p) { return *reinterpret_cast<const uint32_t*>(p); }

constexpr int kLD = 72;    // row stride of bf16 tiles in shared memory
constexpr int kCH = 128;   // samples per chunk (8 warps x 16 rows)

// out[16 rows of this warp] = act(in[rows] W^T + b): W is [64 out][kLD] bf16.
template <bool RELU_BF16>
__device__ __forceinline__ void layer_fwd(const uint16_t* in, const uint16_t* W, const float* bias, uint16_t* out,
                                          int row0, int lane)
{
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int k0 = 0; k0 < kHid; k0 += 16) {
            const uint32_t a[4] = {ld2(in + (row0 + g) * kLD + k0 + 2 * t), ld2(in + (row0 + g + 8) * kLD + k0 + 2 * t),
                                   ld2(in + (row0 + g) * kLD + k0 + 8 + 2 * t),
                                   ld2(in + (row0 + g + 8) * kLD + k0 + 8 + 2 * t)};
            const uint32_t b[2] = {ld2(W + (nt * 8 + g) * kLD + k0 + 2 * t), ld2(W + (nt * 8 + g) * kLD + k0 + 8 + 2 * t)};
            mma_bf16(c, a, b);
        }
        const int col = nt * 8 + 2 * t;
        const float b0 = bias[col], b1 = bias[col + 1];
        out[(row0 + g) * kLD + col] = f2bf(fmaxf(c[0] + b0, 0.f));
        out[(row0 + g) * kLD + col + 1] = f2bf(fmaxf(c[1] + b1, 0.f));
        out[(row0 + g + 8) * kLD + col] = f2bf(fmaxf(c[2] + b0, 0.f));
        out[(row0 + g + 8) * kLD + col + 1] = f2bf(fmaxf(c[3] + b1, 0.f));
    }
}

// acc[4 n-tiles][4] += D^T H over the chunk's rows: dW[m][n] = sum_s D[s][m] H[s][n]
// for the m-tile mt and n-tiles nt0..nt0+3 (D and H are [kCH][kLD] bf16).
__device__ __forceinline__ void wgrad(const uint16_t* D, const uint16_t* H, int mt, int nt0, float acc[4][4], int lane)
{
    const int g = lane >> 2, t = lane & 3, m0 = mt * 16;
#pragma unroll
    for (int k0 = 0; k0 < kCH; k0 += 16) {
        const int ka = k0 + 2 * t, kb = k0 + 8 + 2 * t;
        const uint32_t a[4] = {pk(D[ka * kLD + m0 + g], D[(ka + 1) * kLD + m0 + g]),
                               pk(D[ka * kLD + m0 + g + 8], D[(ka + 1) * kLD + m0 + g + 8]),
                               pk(D[kb * kLD + m0 + g], D[(kb + 1) * kLD + m0 + g]),
                               pk(D[kb * kLD + m0 + g + 8], D[(kb + 1) * kLD + m0 + g + 8])};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = (nt0 + j) * 8 + g;
            const uint32_t b[2] = {pk(H[ka * kLD + n], H[(ka + 1) * kLD + n]), pk(H[kb * kLD + n], H[(kb + 1) * kLD + n])};
            mma_bf16(acc[j], a, b);
        }
    }
}

// c[nt][4] = D[rows] W (back-propagation of deltas through a layer whose
// weights are W [out][in]: result[s][i] = sum_j D[s][j] W[j][i]).
__device__ __forceinline__ void delta_bwd(const uint16_t* D, const uint16_t* W, int row0, float c[8][4], int lane)
{
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) c[nt][0] = c[nt][1] = c[nt][2] = c[nt][3] = 0.f;
#pragma unroll
    for (int k0 = 0; k0 < kHid; k0 += 16) {
        const uint32_t a[4] = {ld2(D + (row0 + g) * kLD + k0 + 2 * t), ld2(D + (row0 + g + 8) * kLD + k0 + 2 * t),
                               ld2(D + (row0 + g) * kLD + k0 + 8 + 2 * t),
                               ld2(D + (row0 + g + 8) * kLD + k0 + 8 + 2 * t)};
        const int ka = k0 + 2 * t, kb = k0 + 8 + 2 * t;
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const int n = nt * 8 + g;
            const uint32_t b[2] = {pk(W[ka * kLD + n], W[(ka + 1) * kLD + n]), pk(W[kb * kLD + n], W[(kb + 1) * kLD + n])};
            mma_bf16(c[nt], a, b);
        }
    }
}

struct MlpK {
    const float* h1p;         // [B][64]
    const int32_t* pid;       // [B] atlas probe of each batch entry (NULL: identity)
    int32_t B, R;
    const float4* tdirs;      // [R*R] texel directions
    const uint16_t* wbf;      // bf16 parameters
    const float* master;      // f32 parameters (biases)
    // targets (train) or outputs (infer): an atlas
    void* rgbo;
    void* depth;
    int32_t rgbo_dtype, depth_dtype;
    float inv_count;          // 1 / (samples * 5) for the mean absolute error
    float* grad;              // train: gradient accumulator
    float* dh1p;              // train: [B][64]
    float* loss;              // train: sum of |y - target|
};

template <bool TRAIN>
__global__ void __launch_bounds__(256) surr_mlp_kernel(const MlpK k)
{
    extern __shared__ __align__(16) unsigned char smem[];
    uint16_t* sW2 = reinterpret_cast<uint16_t*>(smem);
    uint16_t* sW3 = sW2 + kHid * kLD;
    uint16_t* sH1 = sW3 + kHid * kLD;
    uint16_t* sH2 = sH1 + kCH * kLD;
    uint16_t* sH3 = sH2 + kCH * kLD;  // later holds D2
    uint16_t* sD3 = sH3 + kCH * kLD;
    float* fs = reinterpret_cast<float*>(sD3 + kCH * kLD);
    float* sW4 = fs;                  // [5][64]
    float* sb2 = sW4 + kOut * kHid;   // [64]
    float* sb3 = sb2 + kHid;          // [64]
    float* sb4 = sb3 + kHid;          // [8]
    float* sW1d = sb4 + 8;            // [64][3]
    float* sh1p = sW1d + kHid * 3;    // [64]
    float* sG4 = sh1p + kHid;         // [kCH][5]
    float* sDir = sG4 + kCH * kOut;   // [kCH][3] (bf16-rounded)
    float* gW4 = sDir + kCH * 3;      // [5][64]
    float* gb4 = gW4 + kOut * kHid;   // [8]
    float* gb3 = gb4 + 8;             // [64]
    float* gb2 = gb3 + kHid;          // [64]
    float* gW1d = gb2 + kHid;         // [64][3]
    float* gb1 = gW1d + kHid * 3;     // [64]
    float* sdh = gb1 + kHid;          // [64] per probe
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    for (int i = tid; i < kHid * kHid; i += blockDim.x) {
        const int r = i / kHid, c = i % kHid;
        sW2[r * kLD + c] = k.wbf[oW2 + i];
        sW3[r * kLD + c] = k.wbf[oW3 + i];
    }
    for (int i = tid; i < kOut * kHid; i += blockDim.x) sW4[i] = bf2f(k.wbf[oW4 + i]);
    for (int i = tid; i < kHid; i += blockDim.x) {
        sb2[i] = k.master[ob2 + i];
        sb3[i] = k.master[ob3 + i];
        for (int c = 0; c < 3; ++c) sW1d[3 * i + c] = bf2f(k.wbf[oW1d + 3 * i + c]);
        if (TRAIN) gb3[i] = gb2[i] = gb1[i] = sdh[i] = 0.f, gW1d[3 * i] = gW1d[3 * i + 1] = gW1d[3 * i + 2] = 0.f;
    }
    for (int i = tid; i < 8; i += blockDim.x) {
        sb4[i] = i < kOut ? k.master[ob4 + i] : 0.f;
        if (TRAIN) gb4[i] = 0.f;
    }
    if (TRAIN)
        for (int i = tid; i < kOut * kHid; i += blockDim.x) gW4[i] = 0.f;
    float acc3[4][4], acc2[4][4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc3[j][q] = acc2[j][q] = 0.f;
    float lsum = 0.f;
    const int RR = k.R * k.R, RS = k.R + 2;
    const int row0 = warp * 16, mt = warp & 3, nt0 = (warp >> 2) * 4;
    __syncthreads();

    for (int b = blockIdx.x; b < k.B; b += gridDim.x) {
        const int64_t p = k.pid ? k.pid[b] : b;
        for (int i = tid; i < kHid; i += blockDim.x) sh1p[i] = k.h1p[(int64_t)b * kHid + i];
        for (int s0 = 0; s0 < RR; s0 += kCH) {
            const int ns = min(kCH, RR - s0);
            __syncthreads();
            for (int i = tid; i < kCH * 3; i += blockDim.x) {
                const int s = i / 3, c = i % 3;
                float v = 0.f;
                if (s < ns) {
                    const float4 d = k.tdirs[s0 + s];
                    v = rbf(c == 0 ? d.x : (c == 1 ? d.y : d.z));
                }
                sDir[i] = v;
            }
            __syncthreads();
            // layer 1: h1 = relu(h1p + W1d d)
            for (int i = tid; i < kCH * kHid; i += blockDim.x) {
                const int s = i / kHid, o = i % kHid;
                float z = 0.f;
                if (s < ns)
                    z = sh1p[o] + sW1d[3 * o] * sDir[3 * s] + sW1d[3 * o + 1] * sDir[3 * s + 1] +
                        sW1d[3 * o + 2] * sDir[3 * s + 2];
                sH1[s * kLD + o] = f2bf(fmaxf(z, 0.f));
            }
            __syncthreads();
            layer_fwd<true>(sH1, sW2, sb2, sH2, row0, lane);
            __syncwarp();
            layer_fwd<true>(sH2, sW3, sb3, sH3, row0, lane);
            __syncthreads();
            // output layer (f32) and its loss gradient / the atlas write
            for (int i = tid; i < kCH * kOut; i += blockDim.x) {
                const int s = i / kOut, o = i % kOut;
                float y = sb4[o];
                for (int j = 0; j < kHid; ++j) y = fmaf(bf2f(sH3[s * kLD + j]), sW4[o * kHid + j], y);
                const int t = s0 + s;
                const int64_t ti = p * RS * RS + (int64_t)(t / k.R + 1) * RS + (t % k.R + 1);
                if (TRAIN) {
                    float g = 0.f;
                    if (s < ns) {
                        float tg;
                        if (o == 1) {
                            tg = 0.f;
                            if (k.depth) {
                                switch (k.depth_dtype) {
                                case SOP_F32: tg = reinterpret_cast<const float*>(k.depth)[ti]; break;
                                case SOP_F16: tg = __half2float(reinterpret_cast<const __half*>(k.depth)[ti]); break;
                                case SOP_BF16:
                                    tg = __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(k.depth)[ti]);
                                    break;
                                default: tg = float(reinterpret_cast<const __nv_fp8_e4m3*>(k.depth)[ti]); break;
                                }
                            }
                        } else {
                            float4 v;
                            if (k.rgbo_dtype == SOP_F32) v = reinterpret_cast<const float4*>(k.rgbo)[ti];
                            else if (k.rgbo_dtype == SOP_BF16) v = Texel<SOP_BF16>::load(reinterpret_cast<const uint2*>(k.rgbo) + ti);
                            else v = Texel<SOP_F16>::load(reinterpret_cast<const uint2*>(k.rgbo) + ti);
                            tg = o == 0 ? v.w : (o == 2 ? v.x : (o == 3 ? v.y : v.z));
                        }
                        const float df = y - tg;
                        lsum += fabsf(df);
                        g = (df > 0.f ? 1.f : (df < 0.f ? -1.f : 0.f)) * k.inv_count;
                    }
                    sG4[i] = g;
                } else if (s < ns) {
                    // write the prediction into the atlas interior
                    if (o == 1) {
                        if (k.depth) {
                            const float dv = fmaxf(y, 0.f);
                            switch (k.depth_dtype) {
                            case SOP_F32: reinterpret_cast<float*>(k.depth)[ti] = dv; break;
                            case SOP_F16: reinterpret_cast<__half*>(k.depth)[ti] = __float2half_rn(dv); break;
                            case SOP_BF16: reinterpret_cast<__nv_bfloat16*>(k.depth)[ti] = __float2bfloat16_rn(dv); break;
                            default: reinterpret_cast<__nv_fp8_e4m3*>(k.depth)[ti] = __nv_fp8_e4m3(dv); break;
                            }
                        }
                    } else {
                        sG4[i] = o == 0 ? fminf(fmaxf(y, 0.f), 1.f) : fmaxf(y, 0.f);
                    }
                }
            }
            __syncthreads();
            if (!TRAIN) {
                for (int s = tid; s < ns; s += blockDim.x) {
                    const int t = s0 + s;
                    const int64_t ti = p * RS * RS + (int64_t)(t / k.R + 1) * RS + (t % k.R + 1);
                    const float4 v = make_float4(sG4[s * kOut + 2], sG4[s * kOut + 3], sG4[s * kOut + 4], sG4[s * kOut]);
                    if (k.rgbo_dtype == SOP_F32) reinterpret_cast<float4*>(k.rgbo)[ti] = v;
                    else if (k.rgbo_dtype == SOP_BF16) reinterpret_cast<uint2*>(k.rgbo)[ti] = Texel<SOP_BF16>::pack(v);
                    else reinterpret_cast<uint2*>(k.rgbo)[ti] = Texel<SOP_F16>::pack(v);
                }
                continue;
            }
            // ---- backward (train) --------------------------------------------------
            // output layer: dW4 += G4^T H3, db4 += sum G4; D3 = bf16((G4 W4) * (h3 > 0))
            for (int i = tid; i < kOut * kHid; i += blockDim.x) {
                const int o = i / kHid, j = i % kHid;
                float a = 0.f;
                for (int s = 0; s < ns; ++s) a = fmaf(sG4[s * kOut + o], bf2f(sH3[s * kLD + j]), a);
                gW4[i] += a;
            }
            if (tid < kOut) {
                float a = 0.f;
                for (int s = 0; s < ns; ++s) a += sG4[s * kOut + tid];
                gb4[tid] += a;
            }
            for (int i = tid; i < kCH * kHid; i += blockDim.x) {
                const int s = i / kHid, j = i % kHid;
                float a = 0.f;
#pragma unroll
                for (int o = 0; o < kOut; ++o) a = fmaf(sG4[s * kOut + o], sW4[o * kHid + j], a);
                sD3[s * kLD + j] = f2bf(bf2f(sH3[s * kLD + j]) > 0.f ? a : 0.f);
            }
            __syncthreads();
            // layer 3: dW3 += D3^T H2 (tensor cores), db3; D2 = bf16((D3 W3) * (h2 > 0)) into sH3
            wgrad(sD3, sH2, mt, nt0, acc3, lane);
            if (tid < kHid) {
                float a = 0.f;
                for (int s = 0; s < ns; ++s) a += bf2f(sD3[s * kLD + tid]);
                gb3[tid] += a;
            }
            {
                float c[8][4];
                delta_bwd(sD3, sW3, row0, c, lane);
                const int g = lane >> 2, t = lane & 3;
#pragma unroll
                for (int nt = 0; nt < 8; ++nt) {
                    const int col = nt * 8 + 2 * t;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int r = row0 + g + (q >= 2 ? 8 : 0), cc = col + (q & 1);
                        sH3[r * kLD + cc] = f2bf(bf2f(sH2[r * kLD + cc]) > 0.f ? c[nt][q] : 0.f);
                    }
                }
            }
            __syncthreads();
            // layer 2: dW2 += D2^T H1, db2; D1 = (D2 W2) * (h1 > 0) in f32
            wgrad(sH3, sH1, mt, nt0, acc2, lane);
            if (tid < kHid) {
                float a = 0.f;
                for (int s = 0; s < ns; ++s) a += bf2f(sH3[s * kLD + tid]);
                gb2[tid] += a;
            }
            {
                float c[8][4];
                delta_bwd(sH3, sW2, row0, c, lane);
                const int g = lane >> 2, t = lane & 3;
                const int ra = row0 + g, rb = row0 + g + 8;
#pragma unroll
                for (int nt = 0; nt < 8; ++nt) {
                    const int col = nt * 8 + 2 * t;
                    float v[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int r = q >= 2 ? rb : ra, cc = col + (q & 1);
                        v[q] = bf2f(sH1[r * kLD + cc]) > 0.f ? c[nt][q] : 0.f;
                    }
                    // sums over this warp's 16 rows: d(h1p) and dW1d
                    float s0 = v[0] + v[2], s1 = v[1] + v[3];
                    float w0[3], w1[3];
#pragma unroll
                    for (int e = 0; e < 3; ++e) {
                        w0[e] = v[0] * sDir[3 * ra + e] + v[2] * sDir[3 * rb + e];
                        w1[e] = v[1] * sDir[3 * ra + e] + v[3] * sDir[3 * rb + e];
                    }
#pragma unroll
                    for (int off = 4; off < 32; off <<= 1) {
                        s0 += __shfl_xor_sync(0xffffffffu, s0, off);
                        s1 += __shfl_xor_sync(0xffffffffu, s1, off);
#pragma unroll
                        for (int e = 0; e < 3; ++e) {
                            w0[e] += __shfl_xor_sync(0xffffffffu, w0[e], off);
                            w1[e] += __shfl_xor_sync(0xffffffffu, w1[e], off);
                        }
                    }
                    if (g == 0) {
                        atomicAdd(&sdh[col], s0);
                        atomicAdd(&sdh[col + 1], s1);
#pragma unroll
                        for (int e = 0; e < 3; ++e) {
                            atomicAdd(&gW1d[3 * col + e], w0[e]);
                            atomicAdd(&gW1d[3 * (col + 1) + e], w1[e]);
                        }
                    }
                }
            }
        }
        if (TRAIN) {
            __syncthreads();
            for (int i = tid; i < kHid; i += blockDim.x) {
                k.dh1p[(int64_t)b * kHid + i] = sdh[i];
                gb1[i] += sdh[i];
                sdh[i] = 0.f;
            }
        }
    }
    if (TRAIN) {
        __syncthreads();
        // flush this CTA's gradient sums
        const int g = lane >> 2, t = lane & 3, m0 = mt * 16;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = (nt0 + j) * 8 + 2 * t;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int m = m0 + g + (q >= 2 ? 8 : 0), nn = n + (q & 1);
                atomicAdd(k.grad + oW3 + m * kHid + nn, acc3[j][q]);
                atomicAdd(k.grad + oW2 + m * kHid + nn, acc2[j][q]);
            }
        }
        for (int i = tid; i < kOut * kHid; i += blockDim.x) atomicAdd(k.grad + oW4 + i, gW4[i]);
        for (int i = tid; i < kHid; i += blockDim.x) {
            atomicAdd(k.grad + ob3 + i, gb3[i]);
            atomicAdd(k.grad + ob2 + i, gb2[i]);
            atomicAdd(k.grad + ob1 + i, gb1[i]);
            for (int e = 0; e < 3; ++e) atomicAdd(k.grad + oW1d + 3 * i + e, gW1d[3 * i + e]);
        }
        if (tid < kOut) atomicAdd(k.grad + ob4 + tid, gb4[tid]);
        for (int off = 16; off > 0; off >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, off);
        if (lane == 0) atomicAdd(k.loss, lsum);
    }
}

size_t surr_mlp_smem()
{
    return sizeof(uint16_t) * (2 * kHid * kLD + 4 * kCH * kLD) +
           sizeof(float) * (kOut * kHid + kHid + kHid + 8 + kHid * 3 + kHid + kCH * kOut + kCH * 3 + kOut * kHid + 8 +
                            kHid + kHid + kHid * 3 + kHid + kHid);
}

__global__ void surr_tdirs_kernel(int R, float4* __restrict__ dirs)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= R * R) return;
    double d[3];
    oct_decode_centre_f64(R, t % R, t / R, d);
    dirs[t] = make_float4((float)d[0], (float)d[1], (float)d[2], 0.f);
}

__global__ void zero_f32_kernel(float* p, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = 0.f;
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
cudaError_t surr_set_params(char* state, const float* params, cudaStream_t s)
{
    const SurrState S = surr_state_layout();
    cudaError_t e = cudaMemcpyAsync(state + S.master, params, sizeof(float) * kNParam, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    const unsigned nb = (kNParam + 255) / 256;
    surr_reset_kernel<<<nb, 256, 0, s>>>(reinterpret_cast<float*>(state + S.m), reinterpret_cast<float*>(state + S.v),
                                         reinterpret_cast<int32_t*>(state + S.step));
    surr_to_bf16_kernel<<<nb, 256, 0, s>>>(reinterpret_cast<const float*>(state + S.master),
                                           reinterpret_cast<uint16_t*>(state + S.wbf));
    return cudaGetLastError();
}

cudaError_t surr_get_params(const char* state, float* params, cudaStream_t s)
{
    const SurrState S = surr_state_layout();
    return cudaMemcpyAsync(params, state + S.master, sizeof(float) * kNParam, cudaMemcpyDeviceToDevice, s);
}

cudaError_t surr_get_grad(const char* state, float* grad, cudaStream_t s)
{
    const SurrState S = surr_state_layout();
    return cudaMemcpyAsync(grad, state + S.grad, sizeof(float) * kNParam, cudaMemcpyDeviceToDevice, s);
}

cudaError_t surr_features(const sop_gaussians& g, const float* probe_pos, int32_t P, float* feats, char* ws,
                          cudaStream_t s)
{
    int32_t* idx = reinterpret_cast<int32_t*>(ws);
    char* kws = ws + align256(sizeof(int32_t) * (size_t)P * kNeigh);
    cudaError_t e = launch_knn_sites(probe_pos, P, g.mean, (int32_t)g.n, kNeigh, idx, kws, s);
    if (e != cudaSuccess) return e;
    const int64_t n = (int64_t)P * kFP;
    surr_features_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(g, probe_pos, P, idx, feats);
    return cudaGetLastError();
}

size_t surr_features_ws_bytes(int64_t N, int32_t P)
{
    return align256(sizeof(int32_t) * (size_t)P * kNeigh) + knn_sites_bytes((int32_t)N, P, kNeigh);
}

// per-call scratch of train / infer: h1p, dh1p, texel directions
size_t surr_run_ws_bytes(int32_t B, int32_t R)
{
    return 2 * align256(sizeof(float) * (size_t)B * kHid) + align256(sizeof(float4) * (size_t)R * R);
}

static cudaError_t mlp_launch(bool train, const MlpK& k, cudaStream_t s)
{
    const size_t smem = surr_mlp_smem();
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned nb = (unsigned)(k.B < 2 * sms ? k.B : 2 * sms);
    if (train) {
        cudaError_t e = cudaFuncSetAttribute(surr_mlp_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        surr_mlp_kernel<true><<<nb, 256, smem, s>>>(k);
    } else {
        cudaError_t e = cudaFuncSetAttribute(surr_mlp_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        surr_mlp_kernel<false><<<nb, 256, smem, s>>>(k);
    }
    return cudaGetLastError();
}

cudaError_t surr_train_step(char* state, const float* feats, const int32_t* pid, int32_t B, const sop_atlas& tgt,
                            float lr, char* ws, cudaStream_t s)
{
    const SurrState S = surr_state_layout();
    float* h1p = reinterpret_cast<float*>(ws);
    float* dh1p = reinterpret_cast<float*>(ws + align256(sizeof(float) * (size_t)B * kHid));
    float4* tdirs = reinterpret_cast<float4*>(ws + 2 * align256(sizeof(float) * (size_t)B * kHid));
    float* grad = reinterpret_cast<float*>(state + S.grad);
    float* loss = reinterpret_cast<float*>(state + S.loss);
    const int R = tgt.R;
    zero_f32_kernel<<<(kNParam + 255) / 256, 256, 0, s>>>(grad, kNParam);
    zero_f32_kernel<<<1, 32, 0, s>>>(loss, 1);
    surr_tdirs_kernel<<<(R * R + 127) / 128, 128, 0, s>>>(R, tdirs);
    const uint16_t* wbf = reinterpret_cast<const uint16_t*>(state + S.wbf);
    const float* master = reinterpret_cast<const float*>(state + S.master);
    surr_l1_fwd_kernel<<<(unsigned)(((int64_t)B * kHid + 255) / 256), 256, 0, s>>>(feats, pid, B, wbf, master, h1p);
    MlpK k;
    k.h1p = h1p;
    k.pid = pid;
    k.B = B;
    k.R = R;
    k.tdirs = tdirs;
    k.wbf = wbf;
    k.master = master;
    k.rgbo = tgt.rgbo;
    k.depth = tgt.depth;
    k.rgbo_dtype = tgt.rgbo_dtype;
    k.depth_dtype = tgt.depth_dtype;
    k.inv_count = 1.f / ((float)B * R * R * kOut);
    k.grad = grad;
    k.dh1p = dh1p;
    k.loss = loss;
    cudaError_t e = mlp_launch(true, k, s);
    if (e != cudaSuccess) return e;
    surr_l1_bwd_kernel<<<(kHid * kFP + 255) / 256, 256, 0, s>>>(feats, pid, B, dh1p, grad);
    surr_adam_kernel<<<(kNParam + 255) / 256, 256, 0, s>>>(reinterpret_cast<float*>(state + S.master),
                                                           reinterpret_cast<float*>(state + S.m),
                                                           reinterpret_cast<float*>(state + S.v), grad,
                                                           reinterpret_cast<uint16_t*>(state + S.wbf),
                                                           reinterpret_cast<const int32_t*>(state + S.step), lr);
    surr_step_kernel<<<1, 1, 0, s>>>(reinterpret_cast<int32_t*>(state + S.step));
    return cudaGetLastError();
}

cudaError_t surr_infer(const char* state, const float* feats, const int32_t* pid, int32_t B, const sop_atlas& out,
                       char* ws, cudaStream_t s)
{
    const SurrState S = surr_state_layout();
    float* h1p = reinterpret_cast<float*>(ws);
    float4* tdirs = reinterpret_cast<float4*>(ws + 2 * align256(sizeof(float) * (size_t)B * kHid));
    const int R = out.R;
    surr_tdirs_kernel<<<(R * R + 127) / 128, 128, 0, s>>>(R, tdirs);
    const uint16_t* wbf = reinterpret_cast<const uint16_t*>(state + S.wbf);
    const float* master = reinterpret_cast<const float*>(state + S.master);
    surr_l1_fwd_kernel<<<(unsigned)(((int64_t)B * kHid + 255) / 256), 256, 0, s>>>(feats, pid, B, wbf, master, h1p);
    MlpK k{};
    k.h1p = h1p;
    k.pid = pid;
    k.B = B;
    k.R = R;
    k.tdirs = tdirs;
    k.wbf = wbf;
    k.master = master;
    k.rgbo = out.rgbo;
    k.depth = out.depth;
    k.rgbo_dtype = out.rgbo_dtype;
    k.depth_dtype = out.depth_dtype;
    return mlp_launch(false, k, s);
}


__global__ void surr_loss_kernel(const float* sum, float scale, float* out) { out[0] = sum[0] * scale; }

// ---------------------------------------------------------------------------
// Atlas helpers for the spot-check: compare and copy whole probes.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float4 texel_at(const sop_atlas& a, int64_t i)
{
    if (a.rgbo_dtype == SOP_F32) return reinterpret_cast<const float4*>(a.rgbo)[i];
    if (a.rgbo_dtype == SOP_BF16) return Texel<SOP_BF16>::load(reinterpret_cast<const uint2*>(a.rgbo) + i);
    return Texel<SOP_F16>::load(reinterpret_cast<const uint2*>(a.rgbo) + i);
}

// out[0] += sum |O_a - O_b|, out[1] += sum |RGB_a - RGB_b| over the interior
// texels of n probe pairs (a_probes[i], b_probes[i]).
__global__ void atlas_compare_kernel(sop_atlas a, const int32_t* ap, sop_atlas b, const int32_t* bp, int32_t n,
                                     float* out)
{
    const int R = a.R, RS = R + 2, RR = R * R;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float dO = 0.f, dC = 0.f;
    if (i < (int64_t)n * RR) {
        const int64_t q = i / RR;
        const int t = (int)(i % RR);
        const int64_t off = (int64_t)(t / R + 1) * RS + (t % R + 1);
        const float4 va = texel_at(a, (int64_t)(ap ? ap[q] : q) * RS * RS + off);
        const float4 vb = texel_at(b, (int64_t)(bp ? bp[q] : q) * RS * RS + off);
        dO = fabsf(va.w - vb.w);
        dC = fabsf(va.x - vb.x) + fabsf(va.y - vb.y) + fabsf(va.z - vb.z);
    }
    for (int o = 16; o > 0; o >>= 1) {
        dO += __shfl_xor_sync(0xffffffffu, dO, o);
        dC += __shfl_xor_sync(0xffffffffu, dC, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(out, dO);
        atomicAdd(out + 1, dC);
    }
}

// dst probe dp[i] <- src probe sp[i] (all (R+2)^2 texels; same dtypes)
__global__ void atlas_copy_kernel(sop_atlas src, const int32_t* sp, sop_atlas dst, const int32_t* dp, int32_t n)
{
    const int RS = src.R + 2, T = RS * RS;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)n * T) return;
    const int64_t q = i / T;
    const int t = (int)(i % T);
    const int64_t si = (int64_t)(sp ? sp[q] : q) * T + t, di = (int64_t)(dp ? dp[q] : q) * T + t;
    if (src.rgbo_dtype == SOP_F32) reinterpret_cast<float4*>(dst.rgbo)[di] = reinterpret_cast<const float4*>(src.rgbo)[si];
    else reinterpret_cast<uint2*>(dst.rgbo)[di] = reinterpret_cast<const uint2*>(src.rgbo)[si];
    if (src.depth && dst.depth) {
        if (src.depth_dtype == SOP_F32) reinterpret_cast<float*>(dst.depth)[di] = reinterpret_cast<const float*>(src.depth)[si];
        else if (src.depth_dtype == SOP_FP8E4M3) reinterpret_cast<uint8_t*>(dst.depth)[di] = reinterpret_cast<const uint8_t*>(src.depth)[si];
        else reinterpret_cast<uint16_t*>(dst.depth)[di] = reinterpret_cast<const uint16_t*>(src.depth)[si];
    }
}

cudaError_t launch_atlas_compare(const sop_atlas& a, const int32_t* ap, const sop_atlas& b, const int32_t* bp,
                                 int32_t n, float* out, cudaStream_t s)
{
    zero_f32_kernel<<<1, 32, 0, s>>>(out, 2);
    const int64_t m = (int64_t)n * a.R * a.R;
    if (m > 0) atlas_compare_kernel<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(a, ap, b, bp, n, out);
    return cudaGetLastError();
}

cudaError_t launch_atlas_copy(const sop_atlas& src, const int32_t* sp, const sop_atlas& dst, const int32_t* dp,
                              int32_t n, cudaStream_t s)
{
    const int64_t m = (int64_t)n * (src.R + 2) * (src.R + 2);
    if (m > 0) atlas_copy_kernel<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(src, sp, dst, dp, n);
    return cudaGetLastError();
}

cudaError_t surr_loss_out(const char* state, float scale, float* out, cudaStream_t s)
{
    const SurrState S = surr_state_layout();
    surr_loss_kernel<<<1, 1, 0, s>>>(reinterpret_cast<const float*>(state + S.loss), scale, out);
    return cudaGetLastError();
}

}  // namespace sop
