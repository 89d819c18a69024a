// Learned bake surrogate for sm_103a: a small MLP predicts each probe texel's
// maps (O, D/depth_scale, RGB) from 18 features of the probe's neighbourhood
// along that texel's ray, so that probes can be rebaked quickly after an
// object moves. The ray-traced bake stays its fallback and its judge. The
// paper has none of this: it initialises SOPs by ray tracing (Sec. 3.1.2)
// and caches occlusion (Sec. 3.2.2).
//
// Features of texel t of probe p (direction d_t, the octahedral decode of
// its centre):
//   d_t (3);
//   near field (6): the probe's nearest Gaussians (at most kNearCap, centres
//     within r_n, nearest first by the integer squared distance of positions
//     quantised to 2^-20, ties to the lower index), composited along the
//     texel ray in that order with the bake's ray-Gaussian response:
//     O_n = 1 - prod(1 - alpha), L_n rgb = sum T alpha rgb, D_n =
//     sum T alpha t* / W_n, W_n = sum T alpha;
//   far field (9): a coarse extinction grid (optical mass -ln(1 -
//     min(o, alpha_max)) 2 pi s_2 s_3 of each Gaussian in the cubic cell of
//     its quantised centre, fixed-point sums, kFarCells along the longest
//     axis) marched along the ray from t0 (the last listed Gaussian's
//     distance when the list is full, else r_n): 1 - exp(-tau) at t0 + h
//     {2, 4, 8, 16, 32} and at the end, and the emission-absorption colour.
// Network: 18 -> 64 -> 64 -> 64 -> 5, ReLU; every matrix operand (weights,
// features, activations, back-propagated deltas) rounded to bfloat16, sums
// in float32, all four layers on the tensor cores (mma.sync m16n8k16 bf16 ->
// f32) in the forward pass, the delta back-propagation and the weight
// gradients. Float32 master weights and Adam moments live in the caller's
// state buffer.
#include "sop_device.cuh"
#include "sop_internal.h"

namespace sop {

constexpr int kIn = 18;       // features per texel
constexpr int kInPad = 32;    // padded to two mma k-steps
constexpr int kHid = 64;
constexpr int kOut = 5;
constexpr int kNearCap = 256;     // near field: Gaussians per probe at most
constexpr int kCandCap = 4096;    // candidates sorted per probe
constexpr int kFarCells = 128;    // far field: cells along the longest axis
constexpr float kTauMax = 20.f;   // the far march stops beyond this depth
// flat parameter blocks (row-major, out x in)
constexpr int oW1 = 0, ob1 = oW1 + kHid * kIn, oW2 = ob1 + kHid, ob2 = oW2 + kHid * kHid, oW3 = ob2 + kHid,
              ob3 = oW3 + kHid * kHid, oW4 = ob3 + kHid, ob4 = oW4 + kOut * kHid, kNParam = ob4 + kOut;

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
int surr_n_features() { return kIn; }
int surr_near_cap() { return kNearCap; }

__device__ __forceinline__ uint16_t f2bf(float x)
{
    __nv_bfloat16 b = __float2bfloat16_rn(x);
    return *reinterpret_cast<uint16_t*>(&b);
}
__device__ __forceinline__ float bf2f(uint16_t u) { return __uint_as_float((uint32_t)u << 16); }

// ---------------------------------------------------------------------------
// state: bf16 copy, Adam, step
// ---------------------------------------------------------------------------
__global__ void surr_to_bf16_kernel(const float* __restrict__ master, uint16_t* __restrict__ wbf)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kNParam) wbf[i] = f2bf(master[i]);
}

__global__ void surr_reset_kernel(float* m, float* v, float* grad, int32_t* step)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kNParam) {
        m[i] = 0.f;
        v[i] = 0.f;
        grad[i] = 0.f;
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

__global__ void zero_f32_kernel(float* p, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = 0.f;
}

// splitmix64 (Steele, Lea & Flood 2014): the counter-based generator of the
// training batches and of the spot-check sample
__device__ __forceinline__ uint64_t splitmix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// He-uniform initial weights (bound sqrt(6 / fan_in)), zero biases, from the
// counter-based generator (weight i draws splitmix64(seed + i))
__global__ void surr_init_kernel(float* __restrict__ master, uint64_t seed)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kNParam) return;
    int fan = 0;
    if (i < ob1) fan = kIn;
    else if ((i >= oW2 && i < ob2) || (i >= oW3 && i < ob3) || (i >= oW4 && i < ob4)) fan = kHid;
    if (fan == 0) {
        master[i] = 0.f;
        return;
    }
    const double u = (double)(splitmix64(seed + (uint64_t)i) >> 11) * (1.0 / 9007199254740992.0);
    master[i] = (float)((2.0 * u - 1.0) * sqrt(6.0 / fan));
}

// ---------------------------------------------------------------------------
// Near field, in two launches of one CTA per probe. The list: the centres
// within r_n (integer keys) are gathered from the site grid into shared
// memory, the kNearCap-th key is selected and the candidates up to it are
// sorted by (key, index); the list and t0 (where the far field starts) go to
// memory. The composite: the listed Gaussians' terms are staged in shared
// memory and each thread composites them along its texels' rays. Between
// the two, the far march (which needs t0) can start.
// ---------------------------------------------------------------------------
struct NearK {
    const float* probe_pos;
    int32_t P, R;
    const ProbeGrid* grid;
    const int32_t* cell_start;
    const int4* ent;
    uint64_t r2key;       // floor((r_n 2^20)^2)
    int32_t r_q;          // ceil(r_n 2^20)
    float r_n;
    const float4* rec;    // the bake's Gaussian records, 5 float4 each
    const float4* tdirs;  // [R*R] texel directions
    float alpha_min, alpha_max;
    float* feats;         // [P][R*R][kIn]
    int32_t* list;        // [P][kNearCap]
    float* t0;            // [P]
    unsigned int* status;
};

__device__ __forceinline__ int32_t quantise_s(float v) { return __float2int_rn(v * 1048576.0f); }
__device__ __forceinline__ int64_t floordiv_s(int64_t a, int64_t b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

__device__ __forceinline__ void two_diff_s(float a, float b, float& hi, float& lo)
{
    hi = a - b;
    const float bv = a - hi;
    const float av = hi + bv;
    lo = (a - av) + (bv - b);
}

constexpr int kNearThreads = 256;
constexpr int kNearRec = 8;  // staged float4 per listed Gaussian
constexpr int kSelCap = 2 * kNearCap;  // candidates sorted after the selection of the list's last key
static_assert(kNearThreads == 256, "one histogram bin a thread");

__global__ void __launch_bounds__(kNearThreads) surr_near_list_kernel(const NearK k)
{
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t* ckey = reinterpret_cast<uint64_t*>(smem);                 // [kCandCap]
    int32_t* cidx = reinterpret_cast<int32_t*>(ckey + kCandCap);          // [kCandCap]
    // the selection ([kSelCap]) in the candidate arrays' tail, used while
    // the candidates leave it free
    uint64_t* skey = ckey + (kCandCap - kSelCap);
    int32_t* sidx = cidx + (kCandCap - kSelCap);
    __shared__ int32_t s_count, s_box[6], s_need, s_sel;
    __shared__ int32_t s_hist[256];
    __shared__ uint64_t s_prefix;
    const int tid = threadIdx.x, p = blockIdx.x;
    const float3 pp = load3(k.probe_pos, p);
    const int32_t q[3] = {quantise_s(pp.x), quantise_s(pp.y), quantise_s(pp.z)};
    const ProbeGrid G = *k.grid;
    if (tid == 0) {
        s_count = 0;
        for (int a = 0; a < 3; ++a) {
            const int64_t lo = floordiv_s((int64_t)q[a] - k.r_q - G.qmin[a], G.cs);
            const int64_t hi = floordiv_s((int64_t)q[a] + k.r_q - G.qmin[a], G.cs);
            s_box[a] = (int)(lo < 0 ? 0 : (lo > G.dims[a] - 1 ? G.dims[a] - 1 : lo));
            s_box[3 + a] = (int)(hi < 0 ? -1 : (hi > G.dims[a] - 1 ? G.dims[a] - 1 : hi));
        }
    }
    __syncthreads();
    // gather: each warp takes cells of the box in turn, its lanes the entries
    const int nx = s_box[3] - s_box[0] + 1, ny = s_box[4] - s_box[1] + 1, nz = s_box[5] - s_box[2] + 1;
    const int ncell = (nx > 0 && ny > 0 && nz > 0) ? nx * ny * nz : 0;
    const int warp = tid >> 5, lane = tid & 31;
    for (int c = warp; c < ncell; c += kNearThreads / 32) {
        const int cx = s_box[0] + c % nx, cy = s_box[1] + (c / nx) % ny, cz = s_box[2] + c / (nx * ny);
        const int cell = (cz * G.dims[1] + cy) * G.dims[0] + cx;
        const int e1 = __ldg(k.cell_start + cell + 1);
        for (int eb = __ldg(k.cell_start + cell); eb < e1; eb += 32) {
            const int e = eb + lane;
            bool in = false;
            uint64_t key = 0;
            int32_t gi = 0;
            if (e < e1) {
                const int4 en = __ldg(k.ent + e);
                const uint32_t dx = (uint32_t)abs(en.x - q[0]), dy = (uint32_t)abs(en.y - q[1]),
                               dz = (uint32_t)abs(en.z - q[2]);
                key = (uint64_t)dx * dx + (uint64_t)dy * dy + (uint64_t)dz * dz;
                gi = en.w;
                in = key <= k.r2key;
            }
            // one shared-memory atomic per warp and batch
            const unsigned m = __ballot_sync(0xffffffffu, in);
            int base = 0;
            if (m) {
                const int leader = __ffs(m) - 1;
                if (lane == leader) base = atomicAdd(&s_count, __popc(m));
                base = __shfl_sync(0xffffffffu, base, leader);
            }
            if (in) {
                const int pos = base + __popc(m & ((1u << lane) - 1u));
                if (pos < kCandCap) {
                    ckey[pos] = key;
                    cidx[pos] = gi;
                }
            }
        }
    }
    __syncthreads();
    const int total = s_count;
    const int n = total < kCandCap ? total : kCandCap;
    if (total > kCandCap && tid == 0 && k.status) atomicOr(k.status, SOP_DEVSTAT_CAPACITY);
    // The list is the first kNearCap candidates in (key, index) order. With
    // more candidates than that, the kNearCap-th smallest key K is found
    // first, 8 bits at a time from the top (a 256-bin histogram of the
    // candidates that match the digits found so far), and only the
    // candidates with key <= K are sorted: kNearCap of them, plus any others
    // equal to K (all candidates, should more than kSelCap share the key K
    // or more than kCandCap - kSelCap be found).
    uint64_t* lkey = ckey;
    int32_t* lidx = cidx;
    int nsort = n;
    if (n > kNearCap && n <= kCandCap - kSelCap) {
        const int bits = 64 - __clzll((long long)(k.r2key > 0 ? k.r2key : 1));
        if (tid == 0) {
            s_prefix = 0;
            s_need = kNearCap;
        }
        for (int sh = ((bits + 7) / 8 - 1) * 8; sh >= 0; sh -= 8) {
            s_hist[tid] = 0;
            __syncthreads();
            const uint64_t pre = s_prefix;
            for (int i = tid; i < n; i += kNearThreads) {
                const uint64_t kv = ckey[i];
                if (sh + 8 >= 64 || (kv >> (sh + 8)) == (pre >> (sh + 8))) atomicAdd(&s_hist[(kv >> sh) & 255], 1);
            }
            __syncthreads();
            if (tid < 32) {
                // lane l holds bins 8l .. 8l+7; the bin holding the need-th key
                int c[8], sum = 0;
#pragma unroll
                for (int b = 0; b < 8; ++b) {
                    c[b] = s_hist[8 * tid + b];
                    sum += c[b];
                }
                int incl = sum;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const int v = __shfl_up_sync(0xffffffffu, incl, off);
                    if (tid >= off) incl += v;
                }
                const int need = s_need, excl = incl - sum;
                if (excl < need && need <= incl) {
                    int r = need - excl, b = 0;
                    bool found = false;
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        if (!found) {
                            if (r <= c[q]) {
                                b = q;
                                found = true;
                            } else {
                                r -= c[q];
                            }
                        }
                    }
                    s_prefix = pre | ((uint64_t)(8 * tid + b) << sh);
                    s_need = r;
                }
            }
            __syncthreads();
        }
        const uint64_t K = s_prefix;
        if (tid == 0) s_sel = 0;
        __syncthreads();
        for (int i = tid; i < n; i += kNearThreads) {
            const uint64_t kv = ckey[i];
            if (kv <= K) {
                const int pos = atomicAdd(&s_sel, 1);
                if (pos < kSelCap) {
                    skey[pos] = kv;
                    sidx[pos] = cidx[i];
                }
            }
        }
        __syncthreads();
        if (s_sel <= kSelCap) {
            lkey = skey;
            lidx = sidx;
            nsort = s_sel;
        }
    }
    // bitonic sort by (key, index), padded to a power of two
    int n2 = 32;
    while (n2 < nsort) n2 <<= 1;
    for (int i = nsort + tid; i < n2; i += kNearThreads) {
        lkey[i] = UINT64_MAX;
        lidx[i] = INT32_MAX;
    }
    __syncthreads();
    for (int kk = 2; kk <= n2; kk <<= 1) {
        for (int j = kk >> 1; j > 0; j >>= 1) {
            for (int i = tid; i < n2; i += kNearThreads) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const uint64_t a = lkey[i], b = lkey[ixj];
                    const int32_t ia = lidx[i], ib = lidx[ixj];
                    const bool gt = a > b || (a == b && ia > ib);
                    if (gt == ((i & kk) == 0)) {
                        lkey[i] = b;
                        lkey[ixj] = a;
                        lidx[i] = ib;
                        lidx[ixj] = ia;
                    }
                }
            }
            __syncthreads();
        }
    }
    const int nl = n < kNearCap ? n : kNearCap;
    for (int i = tid; i < kNearCap; i += kNearThreads) k.list[(int64_t)p * kNearCap + i] = i < nl ? lidx[i] : -1;
    if (tid == 0) {
        // one square root per probe, in double, so that the far field's
        // start is the correctly rounded distance
        k.t0[p] = nl == kNearCap ? (float)(sqrt((double)lkey[kNearCap - 1]) * (1.0 / 1048576.0)) : k.r_n;
    }
}

// The near field's second part: the listed Gaussians' terms staged in
// shared memory, then one thread per texel composites them along its ray.
__global__ void __launch_bounds__(kNearThreads) surr_near_comp_kernel(const NearK k)
{
    extern __shared__ __align__(16) unsigned char smem[];
    float4* srec = reinterpret_cast<float4*>(smem);  // [kNearCap][kNearRec]
    __shared__ int32_t s_list[kNearCap];
    __shared__ int32_t s_nl;
    const int tid = threadIdx.x, p = blockIdx.x;
    const float3 pp = load3(k.probe_pos, p);
    if (tid == 0) s_nl = 0;
    __syncthreads();
    for (int i = tid; i < kNearCap; i += kNearThreads) {
        const int32_t g = k.list[(int64_t)p * kNearCap + i];
        s_list[i] = g;
        if (g >= 0) atomicMax(&s_nl, i + 1);
    }
    __syncthreads();
    const int nl = s_nl;
    // stage what each listed Gaussian contributes to every texel of this
    // probe, kNearRec float4 each:
    //   0: mu - p, rho (the alpha_min bounding sphere; < 0: never a hit)
    //   1: |mu - p|^2, rho^2 (1 + 1e-4) (-1 when rho < 0), h = p - mu (x, y)
    //   2: h (z), the low parts l of p - mu = h + l (error-free)
    //   3, 4, 5 (x): M = diag(1/s) R^T, row by row; 5 (yzw): u = M h
    //   6: opacity, rgb
    //   7 (x): Q, for a cheap test that a ray cannot reach alpha_min: the
    //     smallest m^2 along the ray is |u|^2 - B^2 / A (B = w.u, A = w.w,
    //     w = M d); above kk^2 = 2 ln(o / alpha_min) no point reaches
    //     alpha_min. With Q = |u|^2 (1 - 1e-3) - kk^2 - 1e-2, Q A > B^2 says
    //     so with a margin of 1e-3 |u|^2 A + 1e-2 A. The FP32 rounding of M
    //     and h moves |u|^2 A - B^2 by at most about 2^-23 (s_max / s_min)
    //     |u|^2 A, so the test only drops certain misses for any Gaussian
    //     with s_max / s_min below about 10^4.
    for (int j = tid; j < nl; j += kNearThreads) {
        const float4* r = k.rec + (int64_t)s_list[j] * 5;
        const float4 r0 = __ldg(r), r1 = __ldg(r + 1), r2 = __ldg(r + 2), r3 = __ldg(r + 3), r4 = __ldg(r + 4);
        const float dx = r0.x - pp.x, dy = r0.y - pp.y, dz = r0.z - pp.z;
        float hx, lx, hy, ly, hz, lz;
        two_diff_s(pp.x, r0.x, hx, lx);
        two_diff_s(pp.y, r0.y, hy, ly);
        two_diff_s(pp.z, r0.z, hz, lz);
        float4* o = srec + kNearRec * j;
        o[0] = make_float4(dx, dy, dz, r0.w);
        o[1] = make_float4(fmaf(dx, dx, fmaf(dy, dy, dz * dz)), r0.w < 0.f ? -1.f : r0.w * r0.w * 1.0001f, hx, hy);
        o[2] = make_float4(hz, lx, ly, lz);
        o[3] = r1;
        o[4] = r2;
        // u = M (h + l), the low part included
        o[5] = make_float4(r3.x, fmaf(r1.x, hx, fmaf(r1.y, hy, r1.z * hz)) + fmaf(r1.x, lx, fmaf(r1.y, ly, r1.z * lz)),
                           fmaf(r1.w, hx, fmaf(r2.x, hy, r2.y * hz)) + fmaf(r1.w, lx, fmaf(r2.x, ly, r2.y * lz)),
                           fmaf(r2.z, hx, fmaf(r2.w, hy, r3.x * hz)) + fmaf(r2.z, lx, fmaf(r2.w, ly, r3.x * lz)));
        o[6] = make_float4(r3.y, r3.z, r3.w, r4.x);
        const float u0 = o[5].y, u1 = o[5].z, u2 = o[5].w;
        const float uu = fmaf(u0, u0, fmaf(u1, u1, u2 * u2));
        const float kk2 = r0.w < 0.f ? 0.f : 2.f * fmaxf(logf(r3.y / k.alpha_min), 0.f);
        o[7] = make_float4(fmaf(uu, 1.f - 1e-3f, -kk2) - 1e-2f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
    const int RR = k.R * k.R;
    for (int t = tid; t < RR; t += kNearThreads) {
        const float4 d4 = __ldg(k.tdirs + t);
        const float3 d = f3(d4.x, d4.y, d4.z);
        float T = 1.f, L0 = 0.f, L1 = 0.f, L2 = 0.f, W = 0.f, Dacc = 0.f;
        for (int j = 0; j < nl; ++j) {
            const float4* q = srec + kNearRec * j;
            const float4 c0 = q[0], c1 = q[1];
            // lossless cull: a ray that misses the alpha_min bounding sphere
            // (margin included) cannot reach alpha_min; the texels of a warp
            // are neighbouring directions, so it is coherent
            const float pr = fmaf(c0.x, d.x, fmaf(c0.y, d.y, c0.z * d.z));
            if (c1.x - pr * pr > c1.y || pr < -c0.w) continue;
            const float4 c2 = q[2], c3 = q[3], c4 = q[4], c5 = q[5];
            // the response is largest at t* = -(w.u) / (w.w), w = M d
            const float w0 = fmaf(c3.x, d.x, fmaf(c3.y, d.y, c3.z * d.z));
            const float w1 = fmaf(c3.w, d.x, fmaf(c4.x, d.y, c4.y * d.z));
            const float w2 = fmaf(c4.z, d.x, fmaf(c4.w, d.y, c5.x * d.z));
            const float A = fmaf(w0, w0, fmaf(w1, w1, w2 * w2));
            const float B = fmaf(w0, c5.y, fmaf(w1, c5.z, w2 * c5.w));
            if (q[7].x * A > B * B) continue;  // certainly below alpha_min
            const float ts = __fdividef(-B, A);
            if (!(ts > 0.f)) continue;
            // m^2 at t*: M applied to the small offset e = h + l + t* d
            const float ex = fmaf(ts, d.x, c1.z) + c2.y, ey = fmaf(ts, d.y, c1.w) + c2.z,
                        ez = fmaf(ts, d.z, c2.x) + c2.w;
            const float v0 = fmaf(c3.x, ex, fmaf(c3.y, ey, c3.z * ez));
            const float v1 = fmaf(c3.w, ex, fmaf(c4.x, ey, c4.y * ez));
            const float v2 = fmaf(c4.z, ex, fmaf(c4.w, ey, c5.x * ez));
            const float4 c6 = q[6];
            const float resp = c6.x * expf(-0.5f * fmaf(v0, v0, fmaf(v1, v1, v2 * v2)));
            if (resp < k.alpha_min) continue;
            const float al = fminf(resp, k.alpha_max);
            const float w = T * al;
            L0 = fmaf(w, c6.y, L0);
            L1 = fmaf(w, c6.z, L1);
            L2 = fmaf(w, c6.w, L2);
            W += w;
            Dacc = fmaf(w, ts, Dacc);
            T *= 1.f - al;
        }
        float* f = k.feats + ((int64_t)p * RR + t) * kIn;
        f[0] = d.x;
        f[1] = d.y;
        f[2] = d.z;
        f[3] = 1.f - T;
        f[4] = L0;
        f[5] = L1;
        f[6] = L2;
        f[7] = W > 1e-8f ? Dacc / W : 0.f;
        f[8] = W;
    }
}

// ---------------------------------------------------------------------------
// Far field: grid geometry, fixed-point splat, per-cell (sigma, colour),
// and the DDA march of every texel ray.
// ---------------------------------------------------------------------------
struct FarGrid {
    int32_t qlo[3];
    int32_t hq;
    int32_t dims[3];
    int32_t ncells;
    float lo[3];
    float h;
};

__global__ void far_bbox_init_kernel(int32_t* mm)
{
    if (threadIdx.x < 3) mm[threadIdx.x] = INT32_MAX;
    else if (threadIdx.x < 6) mm[threadIdx.x] = INT32_MIN;
}

__device__ __forceinline__ bool far_massive(const sop_gaussians& g, int64_t i, float alpha_min)
{
    const float o = g.opacity[i];
    return o >= alpha_min && isfinite(g.mean[3 * i] + g.mean[3 * i + 1] + g.mean[3 * i + 2]);
}

__global__ void far_bbox_kernel(sop_gaussians g, float alpha_min, int32_t* mm)
{
    int32_t lo[3] = {INT32_MAX, INT32_MAX, INT32_MAX}, hi[3] = {INT32_MIN, INT32_MIN, INT32_MIN};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < g.n; i += (int64_t)gridDim.x * blockDim.x) {
        if (!far_massive(g, i, alpha_min)) continue;
        for (int a = 0; a < 3; ++a) {
            const int32_t qv = quantise_s(g.mean[3 * i + a]);
            lo[a] = min(lo[a], qv);
            hi[a] = max(hi[a], qv);
        }
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

__global__ void far_setup_kernel(const int32_t* mm, FarGrid* fg, unsigned long long* next_ray)
{
    if (threadIdx.x != 0) return;
    *next_ray = 0ull;  // the march's ray counter
    FarGrid F;
    if (mm[0] > mm[3]) {  // nothing carries mass
        for (int a = 0; a < 3; ++a) {
            F.qlo[a] = 0;
            F.dims[a] = 1;
            F.lo[a] = 0.f;
        }
        F.hq = 1;
        F.ncells = 1;
        F.h = 1.f / 1048576.f;
        *fg = F;
        return;
    }
    int64_t ext = 0;
    for (int a = 0; a < 3; ++a) ext = max(ext, (int64_t)mm[3 + a] - mm[a] + 1);
    const int64_t hq = (ext + kFarCells - 1) / kFarCells;
    int32_t nc = 1;
    for (int a = 0; a < 3; ++a) {
        F.qlo[a] = mm[a];
        F.dims[a] = (int32_t)(((int64_t)mm[3 + a] - mm[a]) / hq + 1);
        nc *= F.dims[a];
        F.lo[a] = (float)((double)mm[a] * (1.0 / 1048576.0));
    }
    F.hq = (int32_t)hq;
    F.ncells = nc;
    F.h = (float)((double)hq * (1.0 / 1048576.0));
    *fg = F;
}

__global__ void far_zero_kernel(const FarGrid* fg, unsigned long long* __restrict__ acc)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 4 * (int64_t)fg->ncells) acc[i] = 0ull;
}

// acc [cells][4]: mass and mass x rgb in units of 2^-40 (two's complement)
__global__ void far_splat_kernel(sop_gaussians g, float alpha_min, float alpha_max, const FarGrid* fg,
                                 unsigned long long* __restrict__ acc)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n || !far_massive(g, i, alpha_min)) return;
    const FarGrid F = *fg;
    const float s0 = g.scale[3 * i], s1 = g.scale[3 * i + 1], s2 = g.scale[3 * i + 2];
    const float prod2 = s0 * s1 * s2 / fminf(s0, fminf(s1, s2));
    const float mass = -log1pf(-fminf(g.opacity[i], alpha_max)) * 6.283185307179586f * prod2;
    if (!isfinite(mass)) return;
    int c[3];
    for (int a = 0; a < 3; ++a) c[a] = (quantise_s(g.mean[3 * i + a]) - F.qlo[a]) / F.hq;
    const int64_t cell = ((int64_t)c[2] * F.dims[1] + c[1]) * F.dims[0] + c[0];
    const float fix = 1099511627776.f;  // 2^40
    atomicAdd(acc + 4 * cell, (unsigned long long)__float2ll_rn(mass * fix));
    for (int k = 0; k < 3; ++k)
        atomicAdd(acc + 4 * cell + 1 + k, (unsigned long long)__float2ll_rn(mass * g.rgb[3 * i + k] * fix));
}

// per cell: (sigma = mass / h^3, mass-weighted colour), in FP32 from the
// fixed-point sums
__global__ void far_cells_kernel(const FarGrid* fg, const unsigned long long* __restrict__ acc,
                                 float4* __restrict__ cells)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const FarGrid F = *fg;
    if (i >= F.ncells) return;
    const float m = (float)(long long)acc[4 * i];
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (m > 0.f) {
        const float inv_m = 1.f / m;
        v.x = m * (9.094947017729282e-13f / (F.h * F.h * F.h));  // 2^-40 / h^3
        v.y = (float)(long long)acc[4 * i + 1] * inv_m;
        v.z = (float)(long long)acc[4 * i + 2] * inv_m;
        v.w = (float)(long long)acc[4 * i + 3] * inv_m;
    }
    cells[i] = v;
}

// Empty space: one bit per brick of kFarBrick^3 cells, set when a cell of
// the brick carries mass (a warp per 32 bricks, one word each).
constexpr int kFarBrick = 4;
constexpr int kFarBrickWords = (kFarCells / kFarBrick) * (kFarCells / kFarBrick) * (kFarCells / kFarBrick) / 32;

__global__ void far_bricks_kernel(const FarGrid* fg, const float4* __restrict__ cells, uint32_t* __restrict__ bits)
{
    const FarGrid F = *fg;
    const int bdx = (F.dims[0] + kFarBrick - 1) / kFarBrick, bdy = (F.dims[1] + kFarBrick - 1) / kFarBrick,
              bdz = (F.dims[2] + kFarBrick - 1) / kFarBrick;
    const int nb = bdx * bdy * bdz;
    const int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (w * 32 >= nb) return;
    const int b = w * 32 + lane;
    bool any = false;
    if (b < nb) {
        const int bx = b % bdx, by = (b / bdx) % bdy, bz = b / (bdx * bdy);
        for (int z = bz * kFarBrick; z < min((bz + 1) * kFarBrick, F.dims[2]); ++z)
            for (int y = by * kFarBrick; y < min((by + 1) * kFarBrick, F.dims[1]); ++y)
                for (int x = bx * kFarBrick; x < min((bx + 1) * kFarBrick, F.dims[0]); ++x)
                    any |= __ldg(&cells[((int64_t)z * F.dims[1] + y) * F.dims[0] + x].x) > 0.f;
    }
    const unsigned m = __ballot_sync(0xffffffffu, any);
    if (lane == 0) bits[w] = m;
}

// one thread per texel ray (scalars per axis and per checkpoint, so that
// nothing is indexed at run time and the walk stays in registers)
__device__ __forceinline__ void far_slab(float o, float d, float lo, float hi, float& ta, float& tb)
{
    if (d != 0.f) {
        float t1 = (lo - o) / d, t2 = (hi - o) / d;
        if (t1 > t2) {
            const float tmp = t1;
            t1 = t2;
            t2 = tmp;
        }
        ta = fmaxf(ta, t1);
        tb = fminf(tb, t2);
    } else if (o < lo || o >= hi) {
        tb = -INFINITY;
    }
}

__device__ __forceinline__ int far_cell0(float o, float d, float t, float lo, float h, int dim)
{
    const int ci = (int)floorf((fmaf(t, d, o) - lo) / h);
    return ci < 0 ? 0 : (ci >= dim ? dim - 1 : ci);
}

// the same boundary time with the reciprocal of the direction (the march:
// one division per axis and ray instead of one per step)
__device__ __forceinline__ float far_tn(int st, int c, float lo, float h, float o, float id)
{
    return st == 0 ? INFINITY : (fmaf((float)(c + (st > 0 ? 1 : 0)), h, lo) - o) * id;
}

__device__ __forceinline__ int far_cell_at(float o, float d, float t, float lo, float ih, int dim)
{
    const int ci = (int)floorf((fmaf(t, d, o) - lo) * ih);
    return ci < 0 ? 0 : (ci >= dim ? dim - 1 : ci);
}

__device__ __forceinline__ float far_tnext(int st, int c, float lo, float h, float o, float d)
{
    return st == 0 ? INFINITY : (lo + (float)(c + (st > 0 ? 1 : 0)) * h - o) / d;
}

// Texel rays of a warp differ widely in length (a ray into the object stops
// once tau > 20 within a few cells; one that leaves it crosses the box), so
// a warp that marched 32 fixed rays would idle most lanes behind its longest
// ray. The march is persistent instead: each lane holds one ray, and once
// kFarRefill lanes have finished (or none is left marching) the warp fetches
// that many new rays from a global counter. Every ray is still marched by one
// lane from start to end with the same arithmetic, so the result does not
// depend on which lane or warp took it.
constexpr int kFarRefill = 16;

__device__ __forceinline__ void far_write(float* __restrict__ feats, int64_t id, float tk0, float tk1, float tk2,
                                          float tk3, float tk4, float tau, float L0, float L1, float L2)
{
    float* f = feats + id * kIn + 9;
    f[0] = -expm1f(-tk0);
    f[1] = -expm1f(-tk1);
    f[2] = -expm1f(-tk2);
    f[3] = -expm1f(-tk3);
    f[4] = -expm1f(-tk4);
    f[5] = -expm1f(-tau);
    f[6] = L0;
    f[7] = L1;
    f[8] = L2;
}

__global__ void __launch_bounds__(256) far_march_kernel(const float* __restrict__ probe_pos, int32_t P, int32_t R,
                                                        const float* __restrict__ t0p, const float4* __restrict__ tdirs,
                                                        const FarGrid* __restrict__ fg,
                                                        const float4* __restrict__ cells, float* __restrict__ feats,
                                                        unsigned long long* __restrict__ next_ray,
                                                        const uint32_t* __restrict__ brick_bits)
{
    __shared__ uint32_t s_bits[kFarBrickWords];
    const int lane = threadIdx.x & 31;
    const int RR = R * R;
    const int64_t total = (int64_t)P * RR;
    const FarGrid F = *fg;
    const float h = F.h, ih = 1.f / F.h;
    // at most one step per cell along each axis: bounded by the dims
    const int max_steps = F.dims[0] + F.dims[1] + F.dims[2] + 3;
    const int bdx = (F.dims[0] + kFarBrick - 1) / kFarBrick, bdy = (F.dims[1] + kFarBrick - 1) / kFarBrick;
    const int nwords = (bdx * bdy * ((F.dims[2] + kFarBrick - 1) / kFarBrick) + 31) / 32;
    for (int i = threadIdx.x; i < nwords; i += blockDim.x) s_bits[i] = __ldg(brick_bits + i);
    __syncthreads();
    // the lane's ray
    int64_t id = -1;
    bool live = false, retired = false;
    float ox = 0.f, oy = 0.f, oz = 0.f, dx = 0.f, dy = 0.f, dz = 0.f, t0 = 0.f;
    float idx = 0.f, idy = 0.f, idz = 0.f;  // 1 / d (unused along an axis with d = 0)
    float tc = 0.f, tb = 0.f, tau = 0.f, L0 = 0.f, L1 = 0.f, L2 = 0.f;
    float ckn = 0.f;
    float tk0 = 0.f, tk1 = 0.f, tk2 = 0.f, tk3 = 0.f, tk4 = 0.f;  // tau at the checkpoints
    int cx = 0, cy = 0, cz = 0, sx = 0, sy = 0, sz = 0, kn = 0, it = 0;
    for (;;) {
        const unsigned want = __ballot_sync(0xffffffffu, !live && !retired);
        const unsigned marching = __ballot_sync(0xffffffffu, live);
        if (want == 0 && marching == 0) break;
        if (want != 0 && (marching == 0 || __popc(want) >= kFarRefill)) {
            // fetch a ray for every lane that wants one
            const int leader = __ffs(want) - 1;
            unsigned long long base = 0;
            if (lane == leader) base = atomicAdd(next_ray, (unsigned long long)__popc(want));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (want & (1u << lane)) {
                id = (int64_t)base + __popc(want & ((1u << lane) - 1u));
                if (id >= total) {
                    retired = true;
                } else {
                    const int p = (int)(id / RR), t = (int)(id % RR);
                    const float3 o = load3(probe_pos, p);
                    const float4 d = __ldg(tdirs + t);
                    ox = o.x;
                    oy = o.y;
                    oz = o.z;
                    dx = d.x;
                    dy = d.y;
                    dz = d.z;
                    idx = 1.f / dx;
                    idy = 1.f / dy;
                    idz = 1.f / dz;
                    t0 = __ldg(t0p + p);
                    tau = L0 = L1 = L2 = 0.f;
                    tk0 = tk1 = tk2 = tk3 = tk4 = -1.f;  // -1: not reached yet
                    kn = 0;
                    ckn = fmaf(2.f, h, t0);
                    it = 0;
                    float ta = t0;
                    tb = INFINITY;
                    far_slab(ox, dx, F.lo[0], F.lo[0] + F.dims[0] * h, ta, tb);
                    far_slab(oy, dy, F.lo[1], F.lo[1] + F.dims[1] * h, ta, tb);
                    far_slab(oz, dz, F.lo[2], F.lo[2] + F.dims[2] * h, ta, tb);
                    live = ta < tb;
                    if (live) {
                        cx = far_cell_at(ox, dx, ta, F.lo[0], ih, F.dims[0]);
                        cy = far_cell_at(oy, dy, ta, F.lo[1], ih, F.dims[1]);
                        cz = far_cell_at(oz, dz, ta, F.lo[2], ih, F.dims[2]);
                        sx = dx > 0.f ? 1 : (dx < 0.f ? -1 : 0);
                        sy = dy > 0.f ? 1 : (dy < 0.f ? -1 : 0);
                        sz = dz > 0.f ? 1 : (dz < 0.f ? -1 : 0);
                        tc = ta;
                    } else {
                        far_write(feats, id, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f);
                    }
                }
            }
            continue;
        }
        if (!live) continue;
        // One advance a lane, the same steps for all: the segment ends at the
        // boundary time of its exit cell along each axis, the current cell
        // or, when its brick of kFarBrick^3 cells carries no mass, the
        // brick's last cell along the ray (one jump across the brick). The
        // times come from the cell indices (the same expression the walk
        // takes), so the walk resumes in the next cell with the entry time
        // it would have had; across empty cells tau, the colour and the
        // checkpoints (which take tau there) do not change.
        const int bx = (unsigned)cx / kFarBrick, by = (unsigned)cy / kFarBrick, bz = (unsigned)cz / kFarBrick;
        const int bi = (bz * bdy + by) * bdx + bx;
        const bool empty = !((s_bits[bi >> 5] >> (bi & 31)) & 1u);
        const int lx = bx * kFarBrick, ly = by * kFarBrick, lz = bz * kFarBrick;
        const int hx = min(lx + kFarBrick - 1, F.dims[0] - 1), hy = min(ly + kFarBrick - 1, F.dims[1] - 1),
                  hz = min(lz + kFarBrick - 1, F.dims[2] - 1);
        const int ex = empty ? (sx > 0 ? hx : lx) : cx, ey = empty ? (sy > 0 ? hy : ly) : cy,
                  ez = empty ? (sz > 0 ? hz : lz) : cz;
        const float tnx = far_tn(sx, ex, F.lo[0], h, ox, idx), tny = far_tn(sy, ey, F.lo[1], h, oy, idy),
                    tnz = far_tn(sz, ez, F.lo[2], h, oz, idz);
        const int ax = (tnx <= tny && tnx <= tnz) ? 0 : (tny <= tnz ? 1 : 2);
        float te = fminf(ax == 0 ? tnx : (ax == 1 ? tny : tnz), tb);
        te = fmaxf(te, tc);
        float4 cv = make_float4(0.f, 0.f, 0.f, 0.f);
        if (!empty) cv = __ldg(cells + (cz * F.dims[1] + cy) * F.dims[0] + cx);  // < 2^21 cells
        // checkpoints inside this segment take tau at their position (they
        // are increasing: only the next one can be due)
        while (kn < 5 && ckn < te) {
            const float v = ckn <= tc ? tau : fmaf(cv.x, ckn - tc, tau);
            if (kn == 0) tk0 = v;
            else if (kn == 1) tk1 = v;
            else if (kn == 2) tk2 = v;
            else if (kn == 3) tk3 = v;
            else tk4 = v;
            ++kn;
            ckn = kn < 5 ? fmaf((float)(2 << kn), h, t0) : INFINITY;
        }
        if (cv.x > 0.f) {
            const float dtau = cv.x * (te - tc);
            const float a = __expf(-tau) * -expm1f(-dtau);
            L0 = fmaf(a, cv.y, L0);
            L1 = fmaf(a, cv.z, L1);
            L2 = fmaf(a, cv.w, L2);
            tau += dtau;
        }
        tc = te;
        bool end = !(te < tb);
        if (!end) {
            // the next cell: one beyond the exit cell along the exit axis; the
            // other axes stay, or after a jump follow the ray's position,
            // kept inside the brick it leaves
            int nx = cx, ny = cy, nz = cz;
            if (empty) {
                nx = min(max(far_cell_at(ox, dx, te, F.lo[0], ih, F.dims[0]), lx), hx);
                ny = min(max(far_cell_at(oy, dy, te, F.lo[1], ih, F.dims[1]), ly), hy);
                nz = min(max(far_cell_at(oz, dz, te, F.lo[2], ih, F.dims[2]), lz), hz);
            }
            if (ax == 0) nx = ex + sx;
            else if (ax == 1) ny = ey + sy;
            else nz = ez + sz;
            end = nx < 0 || nx >= F.dims[0] || ny < 0 || ny >= F.dims[1] || nz < 0 || nz >= F.dims[2];
            cx = nx;
            cy = ny;
            cz = nz;
        }
        ++it;
        if (end || it >= max_steps || !(tc < tb) || tau > kTauMax) {
            // checkpoints beyond the walk take its final depth
            far_write(feats, id, tk0 < 0.f ? tau : tk0, tk1 < 0.f ? tau : tk1, tk2 < 0.f ? tau : tk2,
                      tk3 < 0.f ? tau : tk3, tk4 < 0.f ? tau : tk4, tau, L0, L1, L2);
            live = false;
        }
    }
}

__global__ void surr_tdirs_kernel(int R, float4* __restrict__ dirs)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= R * R) return;
    double d[3];
    oct_decode_centre_f64(R, t % R, t / R, d);
    dirs[t] = make_float4((float)d[0], (float)d[1], (float)d[2], 0.f);
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

constexpr int kLD = 72;    // row stride of 64-wide bf16 tiles in shared memory
constexpr int kLDX = 40;   // row stride of the 32-wide (padded) feature tile
constexpr int kCH = 128;   // samples per chunk (8 warps x 16 rows)

// four 8x8 bf16 matrices from shared memory, one per register: lane i
// gives the address of row i % 8 of matrix i / 8 and receives, of each
// matrix, row lane / 4, columns 2 (lane % 4) and +1 (the mma fragment layout)
__device__ __forceinline__ void ldsm_x4(uint32_t* r, const uint16_t* row)
{
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(row);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a)
                 : "memory");
}

// out[16 rows of this warp] = relu(in[rows] W^T + b) in bf16: in is
// [kCH][LDI] with KD columns, W is [64 out][LDW] with KD columns (row
// strides of 16-byte multiples whose rows fall on distinct banks). Per
// k-step one ldmatrix gives the A fragments (rows +0/+8 by matrix bit 0,
// columns +0/+8 by bit 1) and one per pair of n-tiles the B fragments (k
// +0/+8 by bit 0, n +0/+8 by bit 1).
template <int KD, int LDI, int LDW>
__device__ __forceinline__ void layer_fwd(const uint16_t* in, const uint16_t* W, const float* bias, uint16_t* out,
                                          int row0, int lane)
{
    const int g = lane >> 2, t = lane & 3;
    const int mr = lane & 7, m0 = (lane >> 3) & 1, m1 = lane >> 4;
    float c[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) c[nt][0] = c[nt][1] = c[nt][2] = c[nt][3] = 0.f;
#pragma unroll
    for (int k0 = 0; k0 < KD; k0 += 16) {
        uint32_t a[4];
        ldsm_x4(a, in + (row0 + mr + 8 * m0) * LDI + k0 + 8 * m1);
#pragma unroll
        for (int np = 0; np < 4; ++np) {
            uint32_t b[4];
            ldsm_x4(b, W + (16 * np + mr + 8 * m1) * LDW + k0 + 8 * m0);
            mma_bf16(c[2 * np], a, b);
            mma_bf16(c[2 * np + 1], a, b + 2);
        }
    }
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const int col = nt * 8 + 2 * t;
        const float b0 = bias[col], b1 = bias[col + 1];
        *reinterpret_cast<uint32_t*>(out + (row0 + g) * kLD + col) =
            pk(f2bf(fmaxf(c[nt][0] + b0, 0.f)), f2bf(fmaxf(c[nt][1] + b1, 0.f)));
        *reinterpret_cast<uint32_t*>(out + (row0 + g + 8) * kLD + col) =
            pk(f2bf(fmaxf(c[nt][2] + b0, 0.f)), f2bf(fmaxf(c[nt][3] + b1, 0.f)));
    }
}

// y[16 rows of this warp][8] = H3[rows] W4^T + b4 in f32 (W4 padded to 8
// rows of zeros beyond the 5 outputs): one n-tile, four k-steps
__device__ __forceinline__ void out_fwd(const uint16_t* H3, const uint16_t* W4b, const float* b4, float* y, int row0,
                                        int lane)
{
    const int g = lane >> 2, t = lane & 3;
    float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int k0 = 0; k0 < kHid; k0 += 16) {
        const uint32_t a[4] = {ld2(H3 + (row0 + g) * kLD + k0 + 2 * t), ld2(H3 + (row0 + g + 8) * kLD + k0 + 2 * t),
                               ld2(H3 + (row0 + g) * kLD + k0 + 8 + 2 * t),
                               ld2(H3 + (row0 + g + 8) * kLD + k0 + 8 + 2 * t)};
        const uint32_t b[2] = {ld2(W4b + g * kLD + k0 + 2 * t), ld2(W4b + g * kLD + k0 + 8 + 2 * t)};
        mma_bf16(c, a, b);
    }
    const int col = 2 * t;
    y[(row0 + g) * 8 + col] = c[0] + b4[col];
    y[(row0 + g) * 8 + col + 1] = c[1] + b4[col + 1];
    y[(row0 + g + 8) * 8 + col] = c[2] + b4[col];
    y[(row0 + g + 8) * 8 + col + 1] = c[3] + b4[col + 1];
}

// acc[NT n-tiles][4] += D^T H over the chunk's rows: dW[m][n] = sum_s D[s][m]
// H[s][n], for the m-tile mt and n-tiles nt0..nt0+NT-1 (D is [kCH][kLD], H
// is [kCH][LDH]).
template <int NT, int LDH>
__device__ __forceinline__ void wgrad(const uint16_t* D, const uint16_t* H, int mt, int nt0, float acc[][4],
                                      int lane)
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
        for (int j = 0; j < NT; ++j) {
            const int n = (nt0 + j) * 8 + g;
            const uint32_t b[2] = {pk(H[ka * LDH + n], H[(ka + 1) * LDH + n]), pk(H[kb * LDH + n], H[(kb + 1) * LDH + n])};
            mma_bf16(acc[j], a, b);
        }
    }
}

// c[nt][4] = D[rows] W (back-propagation of deltas through a 64x64 layer
// whose weights are W [out][in]: result[s][i] = sum_j D[s][j] W[j][i]).
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

// the next layer's delta, bf16((c) * (activation > 0)), written over `out`
__device__ __forceinline__ void store_delta(float c[8][4], const uint16_t* act, uint16_t* out, int row0, int lane)
{
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const int col = nt * 8 + 2 * t;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int r = row0 + g + (q >= 2 ? 8 : 0), cc = col + (q & 1);
            out[r * kLD + cc] = f2bf(bf2f(act[r * kLD + cc]) > 0.f ? c[nt][q] : 0.f);
        }
    }
}

struct MlpK {
    const float* feats;       // [probes][R*R][kIn]
    const int32_t* pid;       // [B] probe of each batch entry (NULL: identity)
    int32_t B, R, P;
    const uint16_t* wbf;      // bf16 parameters
    const float* master;      // f32 parameters (biases)
    // targets (train) or outputs (infer): an atlas
    void* rgbo;
    void* depth;
    int32_t rgbo_dtype, depth_dtype;
    float inv_depth_scale;    // infer: D/depth_scale is what the net predicts (written as is)
    float inv_count;          // 1 / (samples * 5) for the mean absolute error
    float* grad_part;         // train: [gridDim][kNParam] this CTA's gradient sums
    float* loss_part;         // train: [gridDim] this CTA's sum of |y - target|
    unsigned int* status;
};

__device__ __forceinline__ float depth_at(const void* depth, int dt, int64_t ti)
{
    switch (dt) {
    case SOP_F32: return reinterpret_cast<const float*>(depth)[ti];
    case SOP_F16: return __half2float(reinterpret_cast<const __half*>(depth)[ti]);
    case SOP_BF16: return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(depth)[ti]);
    default: return float(reinterpret_cast<const __nv_fp8_e4m3*>(depth)[ti]);
    }
}

__device__ __forceinline__ void depth_put(void* depth, int dt, int64_t ti, float v)
{
    switch (dt) {
    case SOP_F32: reinterpret_cast<float*>(depth)[ti] = v; break;
    case SOP_F16: reinterpret_cast<__half*>(depth)[ti] = __float2half_rn(v); break;
    case SOP_BF16: reinterpret_cast<__nv_bfloat16*>(depth)[ti] = __float2bfloat16_rn(v); break;
    default: reinterpret_cast<__nv_fp8_e4m3*>(depth)[ti] = __nv_fp8_e4m3(v); break;
    }
}

__device__ __forceinline__ float4 texel_load(const void* rgbo, int dt, int64_t ti)
{
    if (dt == SOP_F32) return reinterpret_cast<const float4*>(rgbo)[ti];
    if (dt == SOP_BF16) return Texel<SOP_BF16>::load(reinterpret_cast<const uint2*>(rgbo) + ti);
    return Texel<SOP_F16>::load(reinterpret_cast<const uint2*>(rgbo) + ti);
}

__device__ __forceinline__ void texel_store(void* rgbo, int dt, int64_t ti, float4 v)
{
    if (dt == SOP_F32) reinterpret_cast<float4*>(rgbo)[ti] = v;
    else if (dt == SOP_BF16) reinterpret_cast<uint2*>(rgbo)[ti] = Texel<SOP_BF16>::pack(v);
    else reinterpret_cast<uint2*>(rgbo)[ti] = Texel<SOP_F16>::pack(v);
}

// A CTA's position in its share of the network's work: probe entry b of
// the batch (probe p, or -1 once the CTA is done) and its first texel s0.
struct MlpChunk {
    int b, s0;
    int64_t p;
};

// the first entry from c.b on (in steps of gridDim.x) with a valid probe id;
// invalid ids are reported and skipped
__device__ __forceinline__ void mlp_seek(const MlpK& k, MlpChunk& c, int tid)
{
    for (; c.b < k.B; c.b += gridDim.x) {
        const int64_t p = k.pid ? k.pid[c.b] : c.b;
        if (p >= 0 && p < k.P) {
            c.p = p;
            return;
        }
        if (tid == 0 && k.status) atomicOr(k.status, SOP_DEVSTAT_INDEX);
    }
    c.p = -1;
}

__device__ __forceinline__ void mlp_next(const MlpK& k, MlpChunk& c, int RR, int tid)
{
    c.s0 += kCH;
    if (c.s0 >= RR) {
        c.s0 = 0;
        c.b += gridDim.x;
        mlp_seek(k, c, tid);
    }
}

// A chunk's features (ns rows of kIn floats, contiguous) in registers: up
// to kFeatVec float4 a thread when the rows start on a 16-byte boundary.
constexpr int kFeatVec = (kCH * kIn / 4 + 255) / 256;
struct FeatRegs {
    float4 v[kFeatVec];
};

__device__ __forceinline__ const float* chunk_feats(const MlpK& k, const MlpChunk& c, int RR, int& nf)
{
    nf = min(kCH, RR - c.s0) * kIn;
    return k.feats + (c.p * RR + c.s0) * kIn;
}

__device__ __forceinline__ void feat_load(const MlpK& k, const MlpChunk& c, int RR, int tid, FeatRegs& r)
{
    int nf;
    const float* fp = chunk_feats(k, c, RR, nf);
    if ((reinterpret_cast<uintptr_t>(fp) & 15) != 0 || (nf & 3) != 0) return;  // feat_store reads them itself
#pragma unroll
    for (int q = 0; q < kFeatVec; ++q) {
        const int i = tid + 256 * q;
        if (i < nf / 4) r.v[q] = __ldg(reinterpret_cast<const float4*>(fp) + i);
    }
}

// the chunk's features as bf16 into the tile sX ([kCH][kLDX]; rows beyond
// the chunk zero)
__device__ __forceinline__ void feat_store(const MlpK& k, const MlpChunk& c, int RR, int tid, const FeatRegs& r,
                                           uint16_t* sX)
{
    int nf;
    const float* fp = chunk_feats(k, c, RR, nf);
    if ((reinterpret_cast<uintptr_t>(fp) & 15) == 0 && (nf & 3) == 0) {
#pragma unroll
        for (int q = 0; q < kFeatVec; ++q) {
            const int i = tid + 256 * q;
            if (i < nf / 4) {
                const float f[4] = {r.v[q].x, r.v[q].y, r.v[q].z, r.v[q].w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int n = 4 * i + e, s = n / kIn;
                    sX[s * kLDX + (n - s * kIn)] = f2bf(f[e]);
                }
            }
        }
    } else {
        for (int n = tid; n < nf; n += 256) {
            const int s = n / kIn;
            sX[s * kLDX + (n - s * kIn)] = f2bf(fp[n]);
        }
    }
    for (int i = nf + tid; i < kCH * kIn; i += 256) {
        const int s = i / kIn;
        sX[s * kLDX + (i - s * kIn)] = 0;
    }
}

// Training on mma.sync: the forward pass of each chunk (activations kept),
// the L1 loss gradient, and the backward pass (delta products and weight
// gradients on the tensor cores), summed into this CTA's gradient slot.
__global__ void __launch_bounds__(256) surr_mlp_train_kernel(const MlpK k)
{
    extern __shared__ __align__(16) unsigned char smem[];
    uint16_t* sW1 = reinterpret_cast<uint16_t*>(smem);  // [64][kLDX]
    uint16_t* sW2 = sW1 + kHid * kLDX;                  // [64][kLD]
    uint16_t* sW3 = sW2 + kHid * kLD;
    uint16_t* sX = sW3 + kHid * kLD;                    // [kCH][kLDX]
    uint16_t* sH1 = sX + kCH * kLDX;                    // [kCH][kLD]
    uint16_t* sH2 = sH1 + kCH * kLD;
    // h1..h3 and the deltas for the backward pass
    uint16_t* sH3 = sH2 + kCH * kLD;                    // (later D2)
    uint16_t* sD3 = sH3 + kCH * kLD;                    // (later D1)
    uint16_t* sW4b = sD3 + kCH * kLD;                   // [8][kLD] (rows 5..7 zero)
    float* fs = reinterpret_cast<float*>(sW4b + 8 * kLD);
    float* sW4 = fs;                  // [5][64]
    float* sb1 = sW4 + kOut * kHid;   // [64]
    float* sb2 = sb1 + kHid;
    float* sb3 = sb2 + kHid;
    float* sb4 = sb3 + kHid;          // [8]
    float* sG4 = sb4 + 8;             // [kCH][5]
    float* gW4 = sG4 + kCH * kOut;    // [5][64]
    float* gb4 = gW4 + kOut * kHid;   // [8]
    float* gb3 = gb4 + 8;             // [64]
    float* gb2 = gb3 + kHid;
    float* gb1 = gb2 + kHid;
    float* sY = gb1 + kHid;           // [kCH][8] outputs of the chunk
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    for (int i = tid; i < kHid * kLDX; i += blockDim.x) {
        const int r = i / kLDX, c = i % kLDX;
        sW1[i] = c < kIn ? k.wbf[oW1 + r * kIn + c] : (uint16_t)0;
    }
    for (int i = tid; i < kHid * kHid; i += blockDim.x) {
        const int r = i / kHid, c = i % kHid;
        sW2[r * kLD + c] = k.wbf[oW2 + i];
        sW3[r * kLD + c] = k.wbf[oW3 + i];
    }
    for (int i = tid; i < kOut * kHid; i += blockDim.x) {
        sW4[i] = bf2f(k.wbf[oW4 + i]);
        gW4[i] = 0.f;
    }
    for (int i = tid; i < 8 * kLD; i += blockDim.x) {
        const int r = i / kLD, c = i % kLD;
        sW4b[i] = (r < kOut && c < kHid) ? k.wbf[oW4 + r * kHid + c] : (uint16_t)0;
    }
    for (int i = tid; i < kHid; i += blockDim.x) {
        sb1[i] = k.master[ob1 + i];
        sb2[i] = k.master[ob2 + i];
        sb3[i] = k.master[ob3 + i];
        gb1[i] = gb2[i] = gb3[i] = 0.f;
    }
    for (int i = tid; i < 8; i += blockDim.x) {
        sb4[i] = i < kOut ? k.master[ob4 + i] : 0.f;
        gb4[i] = 0.f;
    }
    // weight-gradient accumulators of layers 1-3 (tensor cores): m-tile
    // warp & 3; n-tiles (warp >> 2) * 4 .. +3 of the 64-wide inputs, and
    // (warp >> 2) * 2 .. +1 of the 32-wide (padded) features
    float acc3[4][4], acc2[4][4], acc1[2][4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc3[j][q] = acc2[j][q] = 0.f;
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc1[j][q] = 0.f;
    float lsum = 0.f;
    const int RR = k.R * k.R, RS = k.R + 2;
    const int row0 = warp * 16, mt = warp & 3, nt0 = (warp >> 2) * 4, nx0 = (warp >> 2) * 2;
    __syncthreads();

    // the padding columns of the feature tile stay zero (chunks write only
    // the first kIn columns)
    for (int i = tid; i < kCH * (kLDX - kIn); i += blockDim.x)
        sX[(i / (kLDX - kIn)) * kLDX + kIn + i % (kLDX - kIn)] = 0;
    // the CTA's chunks: probe entries b = blockIdx.x, + gridDim.x, ... (each
    // in chunks of kCH texels)
    MlpChunk cur;
    cur.b = blockIdx.x;
    cur.s0 = 0;
    mlp_seek(k, cur, tid);
    FeatRegs pf;
    while (cur.p >= 0) {
        const int64_t p = cur.p;
        const int s0 = cur.s0;
        const int ns = min(kCH, RR - s0);
        __syncthreads();
        feat_load(k, cur, RR, tid, pf);
        feat_store(k, cur, RR, tid, pf, sX);
        mlp_next(k, cur, RR, tid);
        __syncthreads();
        {
            layer_fwd<kInPad, kLDX, kLDX>(sX, sW1, sb1, sH1, row0, lane);
            __syncwarp();
            layer_fwd<kHid, kLD, kLD>(sH1, sW2, sb2, sH2, row0, lane);
            __syncwarp();
            layer_fwd<kHid, kLD, kLD>(sH2, sW3, sb3, sH3, row0, lane);
            __syncwarp();
            out_fwd(sH3, sW4b, sb4, sY, row0, lane);
            __syncthreads();
            {
            // the loss gradient of the outputs (one block with the backward pass)
            for (int i = tid; i < kCH * kOut; i += blockDim.x) {
                const int s = i / kOut, o = i % kOut;
                const float y = sY[s * 8 + o];
                const int t = s0 + s;
                const int64_t ti = p * RS * RS + (int64_t)(t / k.R + 1) * RS + (t % k.R + 1);
                float g = 0.f;
                if (s < ns) {
                    float tg;
                    if (o == 1) {
                        tg = k.depth ? depth_at(k.depth, k.depth_dtype, ti) : 0.f;
                    } else {
                        const float4 v = texel_load(k.rgbo, k.rgbo_dtype, ti);
                        tg = o == 0 ? v.w : (o == 2 ? v.x : (o == 3 ? v.y : v.z));
                    }
                    const float df = y - tg;
                    lsum += fabsf(df);
                    g = (df > 0.f ? 1.f : (df < 0.f ? -1.f : 0.f)) * k.inv_count;
                }
                sG4[i] = g;
            }
            __syncthreads();
            // ---- backward ----------------------------------------------------------
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
            // layer 3: dW3 += D3^T H2, db3; D2 = bf16((D3 W3) * (h2 > 0)) into sH3
            wgrad<4, kLD>(sD3, sH2, mt, nt0, acc3, lane);
            if (tid < kHid) {
                float a = 0.f;
                for (int s = 0; s < ns; ++s) a += bf2f(sD3[s * kLD + tid]);
                gb3[tid] += a;
            }
            {
                float c[8][4];
                delta_bwd(sD3, sW3, row0, c, lane);
                store_delta(c, sH2, sH3, row0, lane);
            }
            __syncthreads();
            // layer 2: dW2 += D2^T H1, db2; D1 = bf16((D2 W2) * (h1 > 0)) into sD3
            wgrad<4, kLD>(sH3, sH1, mt, nt0, acc2, lane);
            if (tid < kHid) {
                float a = 0.f;
                for (int s = 0; s < ns; ++s) a += bf2f(sH3[s * kLD + tid]);
                gb2[tid] += a;
            }
            {
                float c[8][4];
                delta_bwd(sH3, sW2, row0, c, lane);
                // sD3 (D3) was last read before the barrier above
                store_delta(c, sH1, sD3, row0, lane);
            }
            __syncthreads();
            // layer 1: dW1 += D1^T X (padded columns give zero), db1
            wgrad<2, kLDX>(sD3, sX, mt, nx0, acc1, lane);
            if (tid < kHid) {
                float a = 0.f;
                for (int s = 0; s < ns; ++s) a += bf2f(sD3[s * kLD + tid]);
                gb1[tid] += a;
            }
            }
        }
    }
    {
        __syncthreads();
        // this CTA's gradient sums into its own slot (summed over the CTAs in
        // a fixed order by surr_grad_reduce_kernel: training is bit-
        // reproducible)
        float* gp = k.grad_part + (int64_t)blockIdx.x * kNParam;
        const int g = lane >> 2, t = lane & 3, m0 = mt * 16;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = (nt0 + j) * 8 + 2 * t;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int m = m0 + g + (q >= 2 ? 8 : 0), nn = n + (q & 1);
                gp[oW3 + m * kHid + nn] = acc3[j][q];
                gp[oW2 + m * kHid + nn] = acc2[j][q];
            }
        }
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int n = (nx0 + j) * 8 + 2 * t;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int m = m0 + g + (q >= 2 ? 8 : 0), nn = n + (q & 1);
                if (nn < kIn) gp[oW1 + m * kIn + nn] = acc1[j][q];
            }
        }
        for (int i = tid; i < kOut * kHid; i += blockDim.x) gp[oW4 + i] = gW4[i];
        for (int i = tid; i < kHid; i += blockDim.x) {
            gp[ob3 + i] = gb3[i];
            gp[ob2 + i] = gb2[i];
            gp[ob1 + i] = gb1[i];
        }
        if (tid < kOut) gp[ob4 + tid] = gb4[tid];
        for (int off = 16; off > 0; off >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, off);
        __shared__ float s_loss[8];
        if (lane == 0) s_loss[warp] = lsum;
        __syncthreads();
        if (tid == 0) {
            float l = 0.f;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) l += s_loss[w];
            k.loss_part[blockIdx.x] = l;
        }
    }
}

// ---------------------------------------------------------------------------
// Inference on the fifth-generation tensor cores (tcgen05). One CTA of 128
// threads takes chunks of kCH = 128 samples: each layer is one 128 x N x K
// product (M = 128 samples, N = 64 outputs, or 16 for the 5 outputs padded
// with zero rows; K = 32 padded features or 64), issued by one thread as
// K/16 tcgen05.mma of kind f16 (bf16 operands from shared memory, FP32
// accumulators in tensor memory), completed through an mbarrier. Each warp
// then reads its 32 samples' accumulators (tensor-memory lanes 32w..32w+31)
// with tcgen05.ld, adds the bias, applies ReLU and writes the bf16
// activations as the next layer's operand. The operands are K-major tiles
// of core matrices (8 rows x 8 bf16 = 128 contiguous bytes; along K 128 B
// apart, along the rows K/8 * 128 B apart), described to the MMA without
// swizzling. Waits give up after kTcSpin tries and report SOP_DEVSTAT_TIMEOUT.
// ---------------------------------------------------------------------------
constexpr int kTcThreads = 128;
constexpr int kTcCols = 128;    // tensor-memory columns: hidden layers 0-63, output layer 64-79
constexpr int kTcOutN = 16;     // the output layer's N (5 outputs and zero rows)
constexpr int kTcSpin = 1 << 24;
constexpr int kTcMaxCtas = 512 / kTcCols;  // CTAs an SM whose tensor memory fits

// element (r, k) of a K-major [rows][KK] tile of core matrices
__device__ __forceinline__ int tc_at(int r, int k, int KK) { return ((r >> 3) * (KK >> 3) + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7); }

__device__ __forceinline__ uint32_t tc_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start, K-direction core-matrix step
// (leading byte offset), row-direction step (stride byte offset), descriptor
// version 1, no swizzle
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor of kind f16: FP32 accumulator, bf16 A and B, both
// K-major, N and M
__host__ __device__ constexpr uint32_t tc_idesc(int n, int m)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// D[tmem] (+)= A[128 x K] B[N x K]^T, K/16 MMAs, then a commit to the mbarrier
// (one thread)
__device__ __forceinline__ void tc_layer(uint32_t tmem, const uint16_t* A, const uint16_t* B, int K, uint32_t idesc,
                                         uint64_t* mbar)
{
    const uint32_t a0 = tc_smem(A), b0 = tc_smem(B), sbo = (uint32_t)(K / 8) * 128u;
    for (int k0 = 0; k0 < K; k0 += 16) {
        const uint64_t da = tc_desc(a0 + (uint32_t)k0 * 16u, 128u, sbo), db = tc_desc(b0 + (uint32_t)k0 * 16u, 128u, sbo);
        const uint32_t acc = k0 > 0;
        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                     " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
                     "l"(da), "l"(db), "r"(idesc), "r"(acc));
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(tc_smem(mbar))
                 : "memory");
}

// waits for the mbarrier's phase `parity` to complete; false after kTcSpin tries
__device__ __forceinline__ bool tc_wait(uint64_t* mbar, uint32_t parity)
{
    uint32_t done = 0;
    for (int it = 0; it < kTcSpin && !done; ++it)
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done)
                     : "r"(tc_smem(mbar)), "r"(parity)
                     : "memory");
    return done != 0;
}

// 16 consecutive FP32 columns of this thread's tensor-memory lane
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float* v)
{
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// this thread's sample row: bias, ReLU, bf16 into the K-major [128][64] tile
__device__ __forceinline__ void tc_hidden_out(uint32_t tmem_row, const float* bias, uint16_t* H, int row)
{
#pragma unroll
    for (int c0 = 0; c0 < kHid; c0 += 16) {
        float v[16];
        tc_ld16(tmem_row + (uint32_t)c0, v);
        uint32_t w[8];
#pragma unroll
        for (int j = 0; j < 8; ++j)
            w[j] = pk(f2bf(fmaxf(v[2 * j] + bias[c0 + 2 * j], 0.f)), f2bf(fmaxf(v[2 * j + 1] + bias[c0 + 2 * j + 1], 0.f)));
        *reinterpret_cast<uint4*>(H + tc_at(row, c0, kHid)) = make_uint4(w[0], w[1], w[2], w[3]);
        *reinterpret_cast<uint4*>(H + tc_at(row, c0 + 8, kHid)) = make_uint4(w[4], w[5], w[6], w[7]);
    }
}

// orders this CTA's shared-memory writes before the tensor cores read them,
// and the tensor-memory reads before the next MMA
__device__ __forceinline__ void tc_sync()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// A chunk's features (ns rows of kIn floats, contiguous in memory) come into
// shared memory by one bulk asynchronous copy when they start on a 16-byte
// boundary and span whole 16 bytes (cp.async.bulk, completing on an
// mbarrier with its byte count); otherwise the threads read them.
__device__ __forceinline__ bool tc_bulk_ok(const MlpK& k, const MlpChunk& c, int RR)
{
    int nf;
    const float* fp = chunk_feats(k, c, RR, nf);
    return (reinterpret_cast<uintptr_t>(fp) & 15) == 0 && ((nf * 4) & 15) == 0;
}

// (one thread) the chunk's features into F, completing on mb
__device__ __forceinline__ void tc_bulk_issue(const MlpK& k, const MlpChunk& c, int RR, float* F, uint64_t* mb)
{
    int nf;
    const float* fp = chunk_feats(k, c, RR, nf);
    const uint32_t bytes = (uint32_t)nf * 4u;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc_smem(mb)), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     tc_smem(F)),
                 "l"(fp), "r"(bytes), "r"(tc_smem(mb))
                 : "memory");
}

// nf features (staged or in global memory) as bf16 into the K-major
// [kCH][kInPad] tile X; rows beyond them zero (the padding columns are
// zero from the start)
__device__ __forceinline__ void tc_feat_to_x(const float* src, int nf, int tid, uint16_t* X)
{
    for (int n = tid; n < nf; n += kTcThreads) {
        const int s = n / kIn;
        X[tc_at(s, n - s * kIn, kInPad)] = f2bf(src[n]);
    }
    for (int i = nf + tid; i < kCH * kIn; i += kTcThreads) {
        const int s = i / kIn;
        X[tc_at(s, i - s * kIn, kInPad)] = 0;
    }
}

constexpr size_t kTcSmem = sizeof(uint16_t) * ((size_t)kHid * kInPad + 2 * kHid * kHid + kTcOutN * kHid +
                                               (size_t)kCH * kInPad + (size_t)kCH * kHid) +
                           sizeof(float) * (3 * kHid + kTcOutN + kCH * kIn);
static_assert((sizeof(uint16_t) * ((size_t)kHid * kInPad + 2 * kHid * kHid + kTcOutN * kHid + (size_t)kCH * kInPad +
                                   (size_t)kCH * kHid) + sizeof(float) * (3 * kHid + kTcOutN)) % 16 == 0,
              "the staging buffer must start on a 16-byte boundary");
static_assert(kCH == 128 && kTcThreads == 128, "one sample a thread and tensor-memory lane");

__global__ void __launch_bounds__(kTcThreads) surr_mlp_tc_kernel(const MlpK k)
{
    // (unswizzled operands: 16-byte aligned starts suffice; every tile's size
    // is a multiple of 1 KB)
    extern __shared__ __align__(16) unsigned char smem[];
    uint16_t* W1 = reinterpret_cast<uint16_t*>(smem);  // [64][kInPad]
    uint16_t* W2 = W1 + kHid * kInPad;                  // [64][64]
    uint16_t* W3 = W2 + kHid * kHid;                    // [64][64]
    uint16_t* W4 = W3 + kHid * kHid;                    // [kTcOutN][64], rows beyond the 5 outputs zero
    uint16_t* X = W4 + kTcOutN * kHid;                  // [kCH][kInPad]
    // [kCH][64] activations: a layer's epilogue overwrites the tile its own
    // MMA read, which has completed by then
    uint16_t* H = X + kCH * kInPad;
    float* bias = reinterpret_cast<float*>(H + kCH * kHid);  // b1 | b2 | b3 | b4 (kTcOutN)
    float* F = bias + 3 * kHid + kTcOutN;                      // [kCH * kIn] the next chunk's features
    __shared__ __align__(8) uint64_t mbar;
    __shared__ __align__(8) uint64_t mbf;  // completion of the bulk copy into F
    __shared__ uint32_t s_tmem;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int row = 32 * warp + lane;  // this thread's sample of a chunk, and its tensor-memory lane
    for (int i = tid; i < kHid * kInPad; i += kTcThreads) {
        const int r = i / kInPad, c = i % kInPad;
        W1[tc_at(r, c, kInPad)] = c < kIn ? k.wbf[oW1 + r * kIn + c] : (uint16_t)0;
    }
    for (int i = tid; i < kHid * kHid; i += kTcThreads) {
        const int r = i / kHid, c = i % kHid;
        W2[tc_at(r, c, kHid)] = k.wbf[oW2 + i];
        W3[tc_at(r, c, kHid)] = k.wbf[oW3 + i];
    }
    for (int i = tid; i < kTcOutN * kHid; i += kTcThreads) {
        const int r = i / kHid, c = i % kHid;
        W4[tc_at(r, c, kHid)] = r < kOut ? k.wbf[oW4 + r * kHid + c] : (uint16_t)0;
    }
    for (int i = tid; i < kHid; i += kTcThreads) {
        bias[i] = k.master[ob1 + i];
        bias[kHid + i] = k.master[ob2 + i];
        bias[2 * kHid + i] = k.master[ob3 + i];
    }
    if (tid < kTcOutN) bias[3 * kHid + tid] = tid < kOut ? k.master[ob4 + tid] : 0.f;
    for (int i = tid; i < kCH * (kInPad - kIn); i += kTcThreads) {
        const int r = i / (kInPad - kIn), c = kIn + i % (kInPad - kIn);
        X[tc_at(r, c, kInPad)] = 0;
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc_smem(&mbar)), "r"(1));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc_smem(&mbf)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_smem(&s_tmem)),
                     "r"(kTcCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_sync();
    const uint32_t tmem = s_tmem;
    const uint32_t trow = tmem + ((uint32_t)(32 * warp) << 16);
    const int RR = k.R * k.R, RS = k.R + 2;
    uint32_t parity = 0, fpar = 0;  // phases of mbar and mbf
    bool ok = true, pend = false;   // a bulk copy into F not yet waited for
    MlpChunk cur;
    cur.b = blockIdx.x;
    cur.s0 = 0;
    mlp_seek(k, cur, tid);
    bool cur_bulk = cur.p >= 0 && tc_bulk_ok(k, cur, RR);
    if (cur_bulk) {
        if (tid == 0) tc_bulk_issue(k, cur, RR, F, &mbf);
        pend = true;
    }
    while (cur.p >= 0) {
        const int64_t p = cur.p;
        const int s0 = cur.s0;
        const int ns = min(kCH, RR - s0);
        int nf;
        const float* fp = chunk_feats(k, cur, RR, nf);
        if (cur_bulk) {
            ok = __syncthreads_and(tc_wait(&mbf, fpar)) && ok;
            fpar ^= 1u;
            pend = false;
            if (!ok) break;
            tc_feat_to_x(F, nf, tid, X);
        } else {
            tc_feat_to_x(fp, nf, tid, X);
        }
        // the next chunk's copy into F goes out after the first barrier
        // below (every thread has converted F by then), beside the layers
        MlpChunk nxt = cur;
        mlp_next(k, nxt, RR, tid);
        const bool nxt_bulk = nxt.p >= 0 && tc_bulk_ok(k, nxt, RR);
        // layers 1-3 (ReLU, bf16) and the output layer
        const uint16_t* Ws[4] = {W1, W2, W3, W4};
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            tc_sync();
            if (l == 0 && nxt_bulk) {
                if (tid == 0) tc_bulk_issue(k, nxt, RR, F, &mbf);
                pend = true;
            }
            if (tid == 0)
                tc_layer(l < 3 ? tmem : tmem + kHid, l == 0 ? X : H, Ws[l], l == 0 ? kInPad : kHid,
                         l < 3 ? tc_idesc(kHid, kCH) : tc_idesc(kTcOutN, kCH), &mbar);
            ok = __syncthreads_and(tc_wait(&mbar, parity)) && ok;
            parity ^= 1u;
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (l < 3) tc_hidden_out(trow, bias + l * kHid, H, row);
        }
        if (!ok) break;
        float y[16];
        tc_ld16(trow + kHid, y);
        if (row < ns) {
            const int t = s0 + row;
            const int64_t ti = p * RS * RS + (int64_t)(t / k.R + 1) * RS + (t % k.R + 1);
            const float* b4 = bias + 3 * kHid;
            if (k.depth) depth_put(k.depth, k.depth_dtype, ti, fmaxf(y[1] + b4[1], 0.f));
            texel_store(k.rgbo, k.rgbo_dtype, ti,
                        make_float4(fmaxf(y[2] + b4[2], 0.f), fmaxf(y[3] + b4[3], 0.f), fmaxf(y[4] + b4[4], 0.f),
                                    fminf(fmaxf(y[0] + b4[0], 0.f), 1.f)));
        }
        cur = nxt;
        cur_bulk = nxt_bulk;
    }
    if (!ok) {
        // a copy still in flight lands before the CTA leaves (bounded wait)
        if (pend) tc_wait(&mbf, fpar);
        if (tid == 0 && k.status) atomicOr(k.status, SOP_DEVSTAT_TIMEOUT);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols));
}

// grad[i] = sum over the CTAs, in CTA order, of their partial sums; loss
// likewise (thread 0)
__global__ void surr_grad_reduce_kernel(const float* __restrict__ part, const float* __restrict__ loss_part, int nb,
                                        float* __restrict__ grad, float* __restrict__ loss)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kNParam) {
        float a = 0.f;
        for (int b = 0; b < nb; ++b) a += part[(int64_t)b * kNParam + i];
        grad[i] = a;
    }
    if (i == 0) {
        float l = 0.f;
        for (int b = 0; b < nb; ++b) l += loss_part[b];
        loss[0] = l;
    }
}

size_t surr_mlp_smem()
{
    return sizeof(uint16_t) * (kHid * kLDX + 2 * kHid * kLD + kCH * kLDX + 4 * kCH * kLD + 8 * kLD) +
           sizeof(float) * (kOut * kHid + 3 * kHid + 8 + kCH * kOut + kOut * kHid + 8 + 3 * kHid + kCH * 8);
}

// batch probe ids of a training step: id i = splitmix64(seed ^ (step 2^32
// + i)) mod P (with replacement), step read from the state
__global__ void surr_pick_kernel(uint64_t seed, const int32_t* step, int32_t P, int32_t B, int32_t* ids)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B) return;
    const uint64_t r = splitmix64(seed ^ (((uint64_t)(uint32_t)step[0] << 32) | (uint32_t)i));
    ids[i] = (int32_t)(r % (uint64_t)P);
}

__global__ void surr_loss_kernel(const float* sum, float scale, float* out) { out[0] = sum[0] * scale; }

// ---------------------------------------------------------------------------
// Atlas helpers for the spot-check: compare and copy whole probes.
// ---------------------------------------------------------------------------
// out[0] += sum |O_a - O_b|, out[1] += sum |RGB_a - RGB_b| over the interior
// texels of n probe pairs (a_probes[i], b_probes[i]).
__global__ void atlas_compare_kernel(sop_atlas a, const int32_t* ap, sop_atlas b, const int32_t* bp, int32_t n,
                                     float* out, unsigned int* status)
{
    const int R = a.R, RS = R + 2, RR = R * R;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float dO = 0.f, dC = 0.f;
    if (i < (int64_t)n * RR) {
        const int64_t q = i / RR;
        const int t = (int)(i % RR);
        const int64_t off = (int64_t)(t / R + 1) * RS + (t % R + 1);
        const int64_t ia = ap ? ap[q] : q, ib = bp ? bp[q] : q;
        if (ia < 0 || ia >= a.P || ib < 0 || ib >= b.P) {
            if (status) atomicOr(status, SOP_DEVSTAT_INDEX);
        } else {
            const float4 va = texel_load(a.rgbo, a.rgbo_dtype, ia * RS * RS + off);
            const float4 vb = texel_load(b.rgbo, b.rgbo_dtype, ib * RS * RS + off);
            dO = fabsf(va.w - vb.w);
            dC = fabsf(va.x - vb.x) + fabsf(va.y - vb.y) + fabsf(va.z - vb.z);
        }
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
__global__ void atlas_copy_kernel(sop_atlas src, const int32_t* sp, sop_atlas dst, const int32_t* dp, int32_t n,
                                  unsigned int* status)
{
    const int RS = src.R + 2, T = RS * RS;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)n * T) return;
    const int64_t q = i / T;
    const int t = (int)(i % T);
    const int64_t ps = sp ? sp[q] : q, pd = dp ? dp[q] : q;
    if (ps < 0 || ps >= src.P || pd < 0 || pd >= dst.P) {
        if (status && t == 0) atomicOr(status, SOP_DEVSTAT_INDEX);
        return;
    }
    const int64_t si = ps * T + t, di = pd * T + t;
    if (src.rgbo_dtype == SOP_F32) reinterpret_cast<float4*>(dst.rgbo)[di] = reinterpret_cast<const float4*>(src.rgbo)[si];
    else reinterpret_cast<uint2*>(dst.rgbo)[di] = reinterpret_cast<const uint2*>(src.rgbo)[si];
    if (src.depth && dst.depth) {
        if (src.depth_dtype == SOP_F32) reinterpret_cast<float*>(dst.depth)[di] = reinterpret_cast<const float*>(src.depth)[si];
        else if (src.depth_dtype == SOP_FP8E4M3) reinterpret_cast<uint8_t*>(dst.depth)[di] = reinterpret_cast<const uint8_t*>(src.depth)[si];
        else reinterpret_cast<uint16_t*>(dst.depth)[di] = reinterpret_cast<const uint16_t*>(src.depth)[si];
    }
}

// The spot-check sample: n_spot of P probes, one per stratum: probe i is
// floor((i + u_i) P / n) with u_i = splitmix64(seed + i) / 2^64, so the
// sample is distinct, spread over the probe order and seeded; positions
// gathered for the trace.
__global__ void spot_pick_kernel(uint64_t seed, int32_t P, int32_t n, const float* __restrict__ probe_pos,
                                 int32_t* __restrict__ ids, float* __restrict__ pos)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double u = (double)(splitmix64(seed + (uint64_t)i) >> 11) * (1.0 / 9007199254740992.0);
    int64_t id = (int64_t)floor(((double)i + u) * (double)P / (double)n);
    id = id < 0 ? 0 : (id >= P ? P - 1 : id);
    ids[i] = (int32_t)id;
    for (int a = 0; a < 3; ++a) pos[3 * i + a] = probe_pos[3 * id + a];
}

// mean |dO| of the spot check and the fallback decision, on the device:
// err = sums[0] / texels; fell_back = err > tau (or not finite)
__global__ void spot_decide_kernel(const float* sums, float inv_texels, float tau, float* err_out,
                                   int32_t* fell_back)
{
    const float e = sums[0] * inv_texels;
    if (err_out) err_out[0] = e;
    fell_back[0] = (e > tau || !isfinite(e)) ? 1 : 0;
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
cudaError_t surr_set_params(char* state, const float* params, uint64_t seed, cudaStream_t s)
{
    const SurrState S = surr_state_layout();
    float* master = reinterpret_cast<float*>(state + S.master);
    const unsigned nb = (kNParam + 255) / 256;
    if (params) {
        cudaError_t e = cudaMemcpyAsync(master, params, sizeof(float) * kNParam, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return e;
    } else {
        surr_init_kernel<<<nb, 256, 0, s>>>(master, seed);
    }
    surr_reset_kernel<<<nb, 256, 0, s>>>(reinterpret_cast<float*>(state + S.m), reinterpret_cast<float*>(state + S.v),
                                         reinterpret_cast<float*>(state + S.grad),
                                         reinterpret_cast<int32_t*>(state + S.step));
    surr_to_bf16_kernel<<<nb, 256, 0, s>>>(master, reinterpret_cast<uint16_t*>(state + S.wbf));
    return cudaGetLastError();
}

cudaError_t surr_refresh_bf16(char* state, cudaStream_t s)
{
    const SurrState S = surr_state_layout();
    surr_to_bf16_kernel<<<(kNParam + 255) / 256, 256, 0, s>>>(reinterpret_cast<const float*>(state + S.master),
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

// ---- features ---------------------------------------------------------------
SurrFeatLayout surr_feat_layout(int64_t N, int32_t P, int32_t R)
{
    SurrFeatLayout L{};
    size_t o = 0;
    L.sites = o;  o = align256(o + sites_grid_bytes((int32_t)(N > 0 ? N : 1)));
    L.tdirs = o;  o = align256(o + sizeof(float4) * (size_t)R * R);
    L.t0 = o;     o = align256(o + sizeof(float) * (size_t)P);
    L.fhdr = o;   o = align256(o + sizeof(FarGrid));
    L.fmm = o;    o = align256(o + 8 * sizeof(int32_t));
    L.fctr = o;   o = align256(o + sizeof(unsigned long long));
    L.list = o;   o = align256(o + sizeof(int32_t) * (size_t)kNearCap * (size_t)(P > 0 ? P : 1));
    L.fbrick = o; o = align256(o + sizeof(uint32_t) * (size_t)kFarBrickWords);
    const size_t cells = (size_t)kFarCells * kFarCells * kFarCells;
    L.facc = o;   o = align256(o + 4 * sizeof(unsigned long long) * cells);
    L.fcells = o; o = align256(o + sizeof(float4) * cells);
    L.total = o;
    return L;
}


cudaError_t surr_features(const sop_gaussians& g, const float* probe_pos, int32_t P, int32_t R, float r_n,
                          float alpha_min, float alpha_max, const char* bake_rec, float* feats, int32_t* list,
                          char* ws, cudaStream_t s, const SurrStreams* ss)
{
    const SurrFeatLayout L = surr_feat_layout(g.n, P, R);
    unsigned int* status = status_word();
    // the far field's grid on the far stream (it reads only the Gaussians),
    // after the work queued on s before the call (ss->fork)
    cudaStream_t sf = ss ? ss->far : s;
    if (ss) {
        const cudaError_t e = cudaStreamWaitEvent(sf, ss->fork, 0);
        if (e != cudaSuccess) return e;
    }
    FarGrid* fg = reinterpret_cast<FarGrid*>(ws + L.fhdr);
    int32_t* mm = reinterpret_cast<int32_t*>(ws + L.fmm);
    unsigned long long* acc = reinterpret_cast<unsigned long long*>(ws + L.facc);
    float4* cells = reinterpret_cast<float4*>(ws + L.fcells);
    far_bbox_init_kernel<<<1, 32, 0, sf>>>(mm);
    const unsigned nb = (unsigned)((g.n + 255) / 256);
    if (g.n > 0) far_bbox_kernel<<<nb < 1024 ? nb : 1024, 256, 0, sf>>>(g, alpha_min, mm);
    unsigned long long* next_ray = reinterpret_cast<unsigned long long*>(ws + L.fctr);
    far_setup_kernel<<<1, 32, 0, sf>>>(mm, fg, next_ray);
    const int64_t maxc = (int64_t)kFarCells * kFarCells * kFarCells;
    far_zero_kernel<<<(unsigned)((4 * maxc + 255) / 256), 256, 0, sf>>>(fg, acc);
    if (g.n > 0) far_splat_kernel<<<nb, 256, 0, sf>>>(g, alpha_min, alpha_max, fg, acc);
    far_cells_kernel<<<(unsigned)((maxc + 255) / 256), 256, 0, sf>>>(fg, acc, cells);
    uint32_t* bricks = reinterpret_cast<uint32_t*>(ws + L.fbrick);
    far_bricks_kernel<<<(unsigned)((kFarBrickWords * 32 + 255) / 256), 256, 0, sf>>>(fg, cells, bricks);
    // the near list and t0 on s
    const SitesGrid sg = launch_sites_grid(g.mean, (int32_t)g.n, ws + L.sites, s);
    float4* tdirs = reinterpret_cast<float4*>(ws + L.tdirs);
    surr_tdirs_kernel<<<(R * R + 127) / 128, 128, 0, s>>>(R, tdirs);
    float* t0 = reinterpret_cast<float*>(ws + L.t0);
    NearK nk;
    nk.probe_pos = probe_pos;
    nk.P = P;
    nk.R = R;
    nk.grid = sg.grid;
    nk.cell_start = sg.cell_start;
    nk.ent = sg.entries;
    const double rq = (double)r_n * 1048576.0;
    nk.r2key = (uint64_t)floor(rq * rq);
    nk.r_q = (int32_t)ceil(rq);
    nk.r_n = r_n;
    nk.rec = reinterpret_cast<const float4*>(bake_rec);
    nk.tdirs = tdirs;
    nk.alpha_min = alpha_min;
    nk.alpha_max = alpha_max;
    nk.feats = feats;
    nk.list = list ? list : reinterpret_cast<int32_t*>(ws + L.list);
    nk.t0 = t0;
    nk.status = status;
    const size_t smem_list = (sizeof(uint64_t) + sizeof(int32_t)) * kCandCap;
    const size_t smem_comp = sizeof(float4) * kNearRec * kNearCap;
    cudaError_t e = cudaFuncSetAttribute(surr_near_list_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_list);
    if (e != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(surr_near_comp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem_comp)) != cudaSuccess)
        return e;
    if (P > 0) surr_near_list_kernel<<<P, kNearThreads, smem_list, s>>>(nk);
    // the far march on the far stream once t0 is known, beside the near
    // composite on s
    if (ss) {
        if ((e = cudaEventRecord(ss->list, s)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(sf, ss->list, 0)) != cudaSuccess) return e;
    }
    const int64_t rays = (int64_t)P * R * R;
    if (rays > 0) {
        // persistent: the CTAs that fit at once, never more than the rays need
        static int resident = 0;
        if (!resident) {
            int dev = 0, sms = 0, per_sm = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, far_march_kernel, 256, 0);
            resident = (sms > 0 ? sms : 152) * (per_sm > 0 ? per_sm : 1);
        }
        const int64_t need = (rays + 255) / 256;
        far_march_kernel<<<(unsigned)(need < resident ? need : resident), 256, 0, sf>>>(probe_pos, P, R, t0, tdirs,
                                                                                     fg, cells, feats, next_ray,
                                                                                     bricks);
    }
    if (P > 0) surr_near_comp_kernel<<<P, kNearThreads, smem_comp, s>>>(nk);
    if (ss) {
        if ((e = cudaEventRecord(ss->far_done, sf)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(s, ss->far_done, 0)) != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

// ---- network -----------------------------------------------------------------
// CTAs of a network launch: two per SM at most (kMaxMlpCtas)
constexpr int kMaxMlpCtas = 2 * 160;

static unsigned mlp_blocks(int32_t B)
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 152;
    }
    int nb = 2 * sms < kMaxMlpCtas ? 2 * sms : kMaxMlpCtas;
    return (unsigned)(B < nb ? B : nb);
}

static cudaError_t mlp_train_launch(const MlpK& k, unsigned nb, cudaStream_t s)
{
    const size_t smem = surr_mlp_smem();
    if (nb == 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(surr_mlp_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    surr_mlp_train_kernel<<<nb, 256, smem, s>>>(k);
    return cudaGetLastError();
}

size_t surr_train_ws_bytes()
{
    return align256(sizeof(int32_t) * 65536) + align256(sizeof(float) * (size_t)kMaxMlpCtas * kNParam) +
           align256(sizeof(float) * kMaxMlpCtas);
}

cudaError_t surr_train_steps(char* state, const float* feats, const int32_t* pid, int32_t B, int32_t P,
                             const sop_atlas& tgt, int32_t steps, float lr, uint64_t seed, float* loss_out,
                             char* ws, cudaStream_t s)
{
    const SurrState S = surr_state_layout();
    float* grad = reinterpret_cast<float*>(state + S.grad);
    float* loss = reinterpret_cast<float*>(state + S.loss);
    int32_t* step = reinterpret_cast<int32_t*>(state + S.step);
    const uint16_t* wbf = reinterpret_cast<const uint16_t*>(state + S.wbf);
    const float* master = reinterpret_cast<const float*>(state + S.master);
    int32_t* ids_ws = reinterpret_cast<int32_t*>(ws);
    float* part = reinterpret_cast<float*>(ws + align256(sizeof(int32_t) * 65536));
    float* lpart = reinterpret_cast<float*>(ws + align256(sizeof(int32_t) * 65536) +
                                            align256(sizeof(float) * (size_t)kMaxMlpCtas * kNParam));
    const int R = tgt.R;
    const unsigned nb = mlp_blocks(B);
    for (int it = 0; it < steps; ++it) {
        const int32_t* ids = pid;
        if (!ids) {
            surr_pick_kernel<<<(B + 255) / 256, 256, 0, s>>>(seed, step, P, B, ids_ws);
            ids = ids_ws;
        }
        MlpK k{};
        k.feats = feats;
        k.pid = ids;
        k.B = B;
        k.R = R;
        k.P = P;
        k.wbf = wbf;
        k.master = master;
        k.rgbo = tgt.rgbo;
        k.depth = tgt.depth;
        k.rgbo_dtype = tgt.rgbo_dtype;
        k.depth_dtype = tgt.depth_dtype;
        k.inv_count = 1.f / ((float)B * R * R * kOut);
        k.grad_part = part;
        k.loss_part = lpart;
        k.status = status_word();
        cudaError_t e = mlp_train_launch(k, nb, s);
        if (e != cudaSuccess) return e;
        surr_grad_reduce_kernel<<<(kNParam + 255) / 256, 256, 0, s>>>(part, lpart, (int)nb, grad, loss);
        if (loss_out) surr_loss_kernel<<<1, 1, 0, s>>>(loss, 1.f / ((float)B * R * R * kOut), loss_out + it);
        surr_adam_kernel<<<(kNParam + 255) / 256, 256, 0, s>>>(reinterpret_cast<float*>(state + S.master),
                                                               reinterpret_cast<float*>(state + S.m),
                                                               reinterpret_cast<float*>(state + S.v), grad,
                                                               reinterpret_cast<uint16_t*>(state + S.wbf), step, lr);
        surr_step_kernel<<<1, 1, 0, s>>>(step);
    }
    return cudaGetLastError();
}

cudaError_t surr_infer(const char* state, const float* feats, const int32_t* pid, int32_t B, int32_t P,
                       const sop_atlas& out, cudaStream_t s)
{
    const SurrState S = surr_state_layout();
    MlpK k{};
    k.feats = feats;
    k.pid = pid;
    k.B = B;
    k.R = out.R;
    k.P = P;
    k.wbf = reinterpret_cast<const uint16_t*>(state + S.wbf);
    k.master = reinterpret_cast<const float*>(state + S.master);
    k.rgbo = out.rgbo;
    k.depth = out.depth;
    k.rgbo_dtype = out.rgbo_dtype;
    k.depth_dtype = out.depth_dtype;
    k.status = status_word();
    // the CTAs that fit at once (57 KB of shared memory and 128 of the 512
    // tensor-memory columns each: four an SM)
    cudaError_t e = cudaFuncSetAttribute(surr_mlp_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
    if (e != cudaSuccess) return e;
    static int resident = 0;
    if (!resident) {
        // from the shared memory an SM holds (each CTA also takes 1 KB the
        // system reserves and its static variables), at most 4 (the tensor
        // memory's 512 columns)
        int dev = 0, sms = 0, smem_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        int per_sm = smem_sm > 0 ? (int)((size_t)smem_sm / (kTcSmem + 1024 + 128)) : 1;
        per_sm = per_sm < 1 ? 1 : (per_sm > kTcMaxCtas ? kTcMaxCtas : per_sm);
        resident = (sms > 0 ? sms : 152) * per_sm;
    }
    const unsigned nb = (unsigned)(B < resident ? B : resident);
    if (nb == 0) return cudaSuccess;
    surr_mlp_tc_kernel<<<nb, kTcThreads, kTcSmem, s>>>(k);
    return cudaGetLastError();
}

cudaError_t launch_atlas_compare(const sop_atlas& a, const int32_t* ap, const sop_atlas& b, const int32_t* bp,
                                 int32_t n, float* out, cudaStream_t s)
{
    zero_f32_kernel<<<1, 32, 0, s>>>(out, 2);
    const int64_t m = (int64_t)n * a.R * a.R;
    if (m > 0)
        atlas_compare_kernel<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(a, ap, b, bp, n, out, status_word());
    return cudaGetLastError();
}

cudaError_t launch_atlas_copy(const sop_atlas& src, const int32_t* sp, const sop_atlas& dst, const int32_t* dp,
                              int32_t n, cudaStream_t s)
{
    const int64_t m = (int64_t)n * (src.R + 2) * (src.R + 2);
    if (m > 0)
        atlas_copy_kernel<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(src, sp, dst, dp, n, status_word());
    return cudaGetLastError();
}

cudaError_t launch_spot_pick(uint64_t seed, int32_t P, int32_t n, const float* probe_pos, int32_t* ids, float* pos,
                             cudaStream_t s)
{
    spot_pick_kernel<<<(n + 127) / 128, 128, 0, s>>>(seed, P, n, probe_pos, ids, pos);
    return cudaGetLastError();
}

cudaError_t launch_spot_decide(const float* sums, float inv_texels, float tau, float* err_out, int32_t* fell_back,
                               cudaStream_t s)
{
    spot_decide_kernel<<<1, 1, 0, s>>>(sums, inv_texels, tau, err_out, fell_back);
    return cudaGetLastError();
}

cudaError_t surr_loss_out(const char* state, float scale, float* out, cudaStream_t s)
{
    const SurrState S = surr_state_layout();
    surr_loss_kernel<<<1, 1, 0, s>>>(reinterpret_cast<const float*>(state + S.loss), scale, out);
    return cudaGetLastError();
}

cudaError_t surr_state_io(char* state, float* master, float* m, float* v, int32_t* step, bool to_device,
                          cudaStream_t s)
{
    const SurrState S = surr_state_layout();
    const cudaMemcpyKind kind = to_device ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost;
    struct {
        size_t off;
        void* host;
        size_t bytes;
    } parts[4] = {{S.master, master, sizeof(float) * kNParam},
                  {S.m, m, sizeof(float) * kNParam},
                  {S.v, v, sizeof(float) * kNParam},
                  {S.step, step, sizeof(int32_t)}};
    for (auto& q : parts) {
        cudaError_t e = to_device ? cudaMemcpyAsync(state + q.off, q.host, q.bytes, kind, s)
                                  : cudaMemcpyAsync(q.host, state + q.off, q.bytes, kind, s);
        if (e != cudaSuccess) return e;
    }
    if (to_device) {
        zero_f32_kernel<<<(kNParam + 255) / 256, 256, 0, s>>>(reinterpret_cast<float*>(state + S.grad), kNParam);
        cudaError_t e = surr_refresh_bf16(state, s);
        if (e != cudaSuccess) return e;
    }
    return cudaStreamSynchronize(s);
}

}  // namespace sop
