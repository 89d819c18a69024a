// Hand-written adjoint of the SOP query/shade (SHADE mode) for sm_103a.
//
// The environment map, the materials and the SOP textures are the learnable
// quantities of the paper's decomposition step (Sec. 3.1.2, Eq. 3-6; the SOP
// textures are optimised under trace guidance). Given dL/dC [M,3] this kernel
// returns dL/d{albedo, roughness, metallic, raw normal} per point and
// accumulates dL/d{environment texels, probe texels}. Nothing of the forward
// pass is stored: every per-direction term is recomputed (frame, octahedral
// coordinates, K bilinear fetches, environment, BRDF), then pushed back
// through the same chain. Probe-texel gradients of border texels are folded
// back onto the texel the border copies, so the gradient is w.r.t. the
// compact [P][R][R] maps. Environment and probe gradients are scattered with
// float atomics (order-nondeterministic sums).
//
// Scatter traffic (bound by L2 atomics): the points are taken grouped by
// their nearest probe (a counting sort), so that a CTA's atomics go to few
// probes' texels; neighbouring points start their direction loops S/32
// apart (by point index), so that a warp's lanes do not update the same
// texels at the same step; the environment gradient is accumulated as float4 texels (4 vector
// atomics a direction instead of 12 scalar ones) and folded into g_env.
#include "sop_device.cuh"
#include "sop_internal.h"

namespace sop {

struct AdjK {
    const float *x, *n, *wo, *albedo, *rough, *metal;
    int64_t M;
    const void* rgbo;
    int32_t R, K, S, He, We;
    const float* env;
    const float4* dirs;
    const int32_t* idx;
    const float* w;
    const float* probe_pos;
    float specular;
    const float* grad_out;
    unsigned int* status;  // device status word or NULL
    float *g_albedo, *g_rough, *g_metal, *g_normal, *g_env;
    float4* g_maps;  // [P][R][R] (d rgb, d O)
    const int32_t* perm;  // order in which the points are taken
    float4* genv4;        // [He][We] environment gradient (rgb, -)
};

template <int DT, int KMAX>
__global__ void __launch_bounds__(128) adjoint_kernel(const AdjK a)
{
    using TX = Texel<DT>;
    extern __shared__ float4 s_dirs[];
    for (int i = threadIdx.x; i < a.S; i += blockDim.x) s_dirs[i] = a.dirs[i];
    __syncthreads();
    const int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // position in the grouped order
    if (pos >= a.M) return;
    const int64_t m = __ldg(a.perm + pos);

    const float3 nr = load3(a.n, m);
    const float nl = sqrtf(dot3(nr, nr));
    const float3 n = f3(nr.x / nl, nr.y / nl, nr.z / nl);
    float3 tt, bb;
    onb(n, tt, bb);
    const float3 wo = load3(a.wo, m);
    const float3 alb = load3(a.albedo, m);
    const float r = __ldg(a.rough + m), mt = __ldg(a.metal + m);
    const float3 go = load3(a.grad_out, m);
    if (a.status && !isfinite(go.x + go.y + go.z + alb.x + alb.y + alb.z + r + mt + wo.x + wo.y + wo.z))
        atomicOr(a.status, SOP_DEVSTAT_NONFINITE);
    const int RS = a.R + 2;
    const typename TX::raw* atlas = reinterpret_cast<const typename TX::raw*>(a.rgbo);
    int32_t pid[KMAX];
    float W[KMAX], gW[KMAX];
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
        const bool on = k < a.K;
        pid[k] = on ? __ldg(a.idx + m * a.K + k) : 0;
        W[k] = on ? __ldg(a.w + m * a.K + k) : 0.f;
        gW[k] = 0.f;
    }

    // per-point BRDF constants
    const float al = r * r, a2 = al * al, kk = (r + 1.f) * (r + 1.f) * 0.125f;
    const float NdotVraw = dot3(n, wo);
    const bool vclamp = NdotVraw < 1e-4f;
    const float NdotV = vclamp ? 1e-4f : NdotVraw;
    const float gvv = NdotV * (1.f - kk) + kk;
    const float G1V = NdotV / gvv;
    const float dG1V_dk = -NdotV * (1.f - NdotV) / (gvv * gvv);
    const float f0d = 0.08f * a.specular * (1.f - mt);
    const float F0[3] = {f0d + alb.x * mt, f0d + alb.y * mt, f0d + alb.z * mt};
    const float av[3] = {alb.x, alb.y, alb.z};
    const float gov[3] = {go.x, go.y, go.z};
    const float sc = 2.f * kPi / (float)a.S;
    // frame derivatives (Duff et al. 2017): dt/dn and db/dn, row = component
    const float sg = n.z >= 0.f ? 1.f : -1.f, aa = -1.f / (sg + n.z), a2n = aa * aa;
    const float dt[3][3] = {{2.f * sg * n.x * aa, 0.f, sg * n.x * n.x * a2n},
                            {sg * n.y * aa, sg * n.x * aa, sg * n.x * n.y * a2n},
                            {-sg, 0.f, 0.f}};
    const float db[3][3] = {{n.y * aa, n.x * aa, n.x * n.y * a2n}, {0.f, 2.f * n.y * aa, n.y * n.y * a2n},
                            {0.f, -1.f, 0.f}};
    float ga[3] = {0.f, 0.f, 0.f}, gr = 0.f, gm = 0.f, gn[3] = {0.f, 0.f, 0.f};
    const float Rf = (float)a.R;

    // neighbouring points (nearly the same frame) start their direction loops
    // S/32 apart, by their index, so that the lanes of a warp scatter into
    // other texels at each step instead of all into the same ones; the start
    // depends on the point alone, so each point's sums keep one order from
    // call to call whatever lane it lands in
    const int i_first = (int)(((m & 31) * (int64_t)a.S) >> 5);
    for (int ii = 0; ii < a.S; ++ii) {
        const int i = ii + i_first < a.S ? ii + i_first : ii + i_first - a.S;
        const float4 l = s_dirs[i];
        const float3 w = f3(fmaf(l.x, tt.x, fmaf(l.y, bb.x, l.z * n.x)), fmaf(l.x, tt.y, fmaf(l.y, bb.y, l.z * n.y)),
                            fmaf(l.x, tt.z, fmaf(l.y, bb.z, l.z * n.z)));
        const float NdotL = l.z;
        // ---- probe terms and their uv-derivatives ----------------------------
        const float2 uv = oct_encode(w);
        const float s = uv.x * Rf - 0.5f, t = uv.y * Rf - 0.5f;
        const float fi = floorf(s), fj = floorf(t);
        const float fu = s - fi, fv = t - fj;
        const int i0 = min(max((int)fi + 1, 0), a.R), j0 = min(max((int)fj + 1, 0), a.R);
        const int off = j0 * RS + i0;
        const float w00 = (1.f - fu) * (1.f - fv), w10 = fu * (1.f - fv), w01 = (1.f - fu) * fv, w11 = fu * fv;
        float4 pr = make_float4(0.f, 0.f, 0.f, 0.f), ps = pr, pt = pr;  // value, d/ds, d/dt
        float4 tk[KMAX];  // per-probe bilinear values (for dL/dW)
#pragma unroll
        for (int k = 0; k < KMAX; ++k) {
            tk[k] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (k < a.K) {
                const typename TX::raw* p = atlas + (int64_t)pid[k] * RS * RS + off;
                const float4 t00 = TX::load(p), t10 = TX::load(p + 1), t01 = TX::load(p + RS),
                             t11 = TX::load(p + RS + 1);
                const float4 v = make_float4(w00 * t00.x + w10 * t10.x + w01 * t01.x + w11 * t11.x,
                                             w00 * t00.y + w10 * t10.y + w01 * t01.y + w11 * t11.y,
                                             w00 * t00.z + w10 * t10.z + w01 * t01.z + w11 * t11.z,
                                             w00 * t00.w + w10 * t10.w + w01 * t01.w + w11 * t11.w);
                tk[k] = v;
                const float Wk = W[k];
                pr.x += Wk * v.x; pr.y += Wk * v.y; pr.z += Wk * v.z; pr.w += Wk * v.w;
                // d/ds = (1-fv)(t10-t00) + fv(t11-t01); d/dt = (1-fu)(t01-t00) + fu(t11-t10)
                ps.x += Wk * ((1.f - fv) * (t10.x - t00.x) + fv * (t11.x - t01.x));
                ps.y += Wk * ((1.f - fv) * (t10.y - t00.y) + fv * (t11.y - t01.y));
                ps.z += Wk * ((1.f - fv) * (t10.z - t00.z) + fv * (t11.z - t01.z));
                ps.w += Wk * ((1.f - fv) * (t10.w - t00.w) + fv * (t11.w - t01.w));
                pt.x += Wk * ((1.f - fu) * (t01.x - t00.x) + fu * (t11.x - t10.x));
                pt.y += Wk * ((1.f - fu) * (t01.y - t00.y) + fu * (t11.y - t10.y));
                pt.z += Wk * ((1.f - fu) * (t01.z - t00.z) + fu * (t11.z - t10.z));
                pt.w += Wk * ((1.f - fu) * (t01.w - t00.w) + fu * (t11.w - t10.w));
            }
        }
        const float O = pr.w;
        const float Lin[3] = {pr.x, pr.y, pr.z};
        // ---- environment and its direction derivative ------------------------
        const float rho2 = w.x * w.x + w.y * w.y, rho = sqrtf(rho2);
        const float th = atan2f(rho, w.z), ph = atan2f(w.y, w.x);
        const float es = (ph + kPi) * kInv2Pi * a.We - 0.5f, et = th * kInvPi * a.He - 0.5f;
        const float fes = floorf(es), fet = floorf(et);
        const float ea = es - fes, eb = et - fet;
        int c0 = (int)fes;
        c0 = c0 < 0 ? c0 + a.We : c0;
        c0 = min(max(c0, 0), a.We - 1);
        const int c1 = c0 + 1 == a.We ? 0 : c0 + 1;
        const int r0 = min(max((int)fet, 0), a.He - 1), r1 = min(max((int)fet + 1, 0), a.He - 1);
        const int64_t ei[4] = {((int64_t)r0 * a.We + c0) * 3, ((int64_t)r0 * a.We + c1) * 3,
                               ((int64_t)r1 * a.We + c0) * 3, ((int64_t)r1 * a.We + c1) * 3};
        const float ew[4] = {(1.f - ea) * (1.f - eb), ea * (1.f - eb), (1.f - ea) * eb, ea * eb};
        float Ld[3], dLs[3], dLt[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float e00 = __ldg(a.env + ei[0] + c), e01 = __ldg(a.env + ei[1] + c), e10 = __ldg(a.env + ei[2] + c),
                        e11 = __ldg(a.env + ei[3] + c);
            Ld[c] = ew[0] * e00 + ew[1] * e01 + ew[2] * e10 + ew[3] * e11;
            dLs[c] = (1.f - eb) * (e01 - e00) + eb * (e11 - e10);
            dLt[c] = (1.f - ea) * (e10 - e00) + ea * (e11 - e01);
        }
        // ds/dw, dt/dw
        float dsw[3] = {0.f, 0.f, 0.f}, dtw[3] = {0.f, 0.f, 0.f};
        if (rho2 > 0.f) {
            const float ks = a.We * kInv2Pi / rho2;
            dsw[0] = -ks * w.y;
            dsw[1] = ks * w.x;
            const float r2 = rho2 + w.z * w.z, kt = a.He * kInvPi / r2;
            dtw[0] = kt * w.z * w.x / rho;
            dtw[1] = kt * w.z * w.y / rho;
            dtw[2] = -kt * rho;
        }
        // ---- BRDF ---------------------------------------------------------------
        const float3 hv = w + wo;
        const float hl = sqrtf(dot3(hv, hv));
        const float3 h = hl > 1e-30f ? (1.f / hl) * hv : n;
        const float NdotH = dot3(n, h), VdotH = dot3(wo, h);
        const float3 cr = cross3(n, h);
        const float sin2 = dot3(cr, cr);
        const float den = NdotH * NdotH * a2 + sin2;
        const float D = a2 / (kPi * den * den);
        const float gl = NdotL * (1.f - kk) + kk;
        const float G1L = NdotL / gl;
        const float spec_t = D * G1L * G1V / (4.f * NdotL * NdotV);
        const float x1 = 1.f - VdotH, x2 = x1 * x1, fc = x2 * x2 * x1;
        const float dD_da2 = (den - 2.f * a2 * NdotH * NdotH) / (kPi * den * den * den);
        const float dG1L_dk = -NdotL * (1.f - NdotL) / (gl * gl);
        const float dspec_dr =
            (dD_da2 * 4.f * r * r * r * G1L * G1V + D * (dG1L_dk * G1V + G1L * dG1V_dk) * (r + 1.f) * 0.25f) /
            (4.f * NdotL * NdotV);
        const float Gc = G1L * G1V / (4.f * NdotL * NdotV);
        const float dD_dNH = -4.f * a2 * a2 * NdotH / (kPi * den * den * den);
        const float dD_ds2 = -2.f * a2 / (kPi * den * den * den);
        float GN = 0.f, GS = 0.f, GVH = 0.f, GNV = 0.f, gO = 0.f, gLin[3], gLd[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float F = F0[c] + (1.f - F0[c]) * fc;
            const float f = (1.f - mt) * av[c] * kInvPi + spec_t * F;
            const float Lmix = (1.f - O) * Ld[c] + Lin[c];
            const float gam = sc * gov[c] * NdotL;
            const float u = gam * Lmix;
            ga[c] += u * ((1.f - mt) * kInvPi + spec_t * (1.f - fc) * mt);
            gm += u * (-av[c] * kInvPi + spec_t * (1.f - fc) * (-0.08f * a.specular + av[c]));
            gr += u * dspec_dr * F;
            GN += u * F * Gc * dD_dNH;
            GS += u * F * Gc * dD_ds2;
            GVH += u * spec_t * (1.f - F0[c]) * (-5.f * x2 * x2);
            if (!vclamp) GNV += u * F * D * G1L / (4.f * NdotL) * (-(1.f - kk) / (gvv * gvv));
            gO += -gam * f * Ld[c];
            gLin[c] = gam * f;
            gLd[c] = gam * f * (1.f - O);
        }
        // ---- scatter: probe texels (folded through the border rule) and env ----
#pragma unroll
        for (int k = 0; k < KMAX; ++k) {
            // a zero weight (an empty slot of a radius search, or a probe
            // other than the one a snapped point sits on) scatters nothing
            if (k < a.K && W[k] != 0.f) {
                gW[k] += gO * tk[k].w + gLin[0] * tk[k].x + gLin[1] * tk[k].y + gLin[2] * tk[k].z;
                const float Wk = W[k];
                const float q[4] = {w00, w10, w01, w11};
#pragma unroll
                for (int qq = 0; qq < 4; ++qq) {
                    int si, sj;
                    oct_wrap(a.R, i0 - 1 + (qq & 1), j0 - 1 + (qq >> 1), si, sj);
                    const float c = Wk * q[qq];
                    atomicAdd(a.g_maps + ((int64_t)pid[k] * a.R + sj) * a.R + si,
                              make_float4(gLin[0] * c, gLin[1] * c, gLin[2] * c, gO * c));
                }
            }
        }
#pragma unroll
        for (int qq = 0; qq < 4; ++qq)
            atomicAdd(a.genv4 + ei[qq] / 3, make_float4(gLd[0] * ew[qq], gLd[1] * ew[qq], gLd[2] * ew[qq], 0.f));
        // ---- d/dw ---------------------------------------------------------------
        // octahedral coordinates: uv = (p + 1)/2, p = w.xy/|w|_1 (folded below)
        float gw[3];
        {
            const float gs_ = gO * ps.w + gLin[0] * ps.x + gLin[1] * ps.y + gLin[2] * ps.z;
            const float gt_ = gO * pt.w + gLin[0] * pt.x + gLin[1] * pt.y + gLin[2] * pt.z;
            const float gu = gs_ * Rf, gvv2 = gt_ * Rf;  // d/d(uv)
            const float ax_ = fabsf(w.x), ay_ = fabsf(w.y), az_ = fabsf(w.z);
            const float l1 = ax_ + ay_ + az_, il2 = 1.f / (l1 * l1);
            const float sx = w.x >= 0.f ? 1.f : -1.f, sy = w.y >= 0.f ? 1.f : -1.f, sz = w.z >= 0.f ? 1.f : -1.f;
            const float dpx[3] = {(l1 - ax_) * il2, -w.x * sy * il2, -w.x * sz * il2};
            const float dpy[3] = {-w.y * sx * il2, (l1 - ay_) * il2, -w.y * sz * il2};
            if (w.z < 0.f) {
                const float px = w.x / l1, py = w.y / l1;
                const float spx = px >= 0.f ? 1.f : -1.f, spy = py >= 0.f ? 1.f : -1.f;
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    gw[c] = 0.5f * (gu * (-spy * dpy[c] * spx) + gvv2 * (-spx * dpx[c] * spy));
            } else {
#pragma unroll
                for (int c = 0; c < 3; ++c) gw[c] = 0.5f * (gu * dpx[c] + gvv2 * dpy[c]);
            }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int j = 0; j < 3; ++j) gw[j] += gLd[c] * (dLs[c] * dsw[j] + dLt[c] * dtw[j]);
        // BRDF geometry through h, and directly through n
        const float hh[3] = {h.x, h.y, h.z}, nn[3] = {n.x, n.y, n.z}, vv[3] = {wo.x, wo.y, wo.z};
        float gh[3], gnd[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            gh[j] = GN * nn[j] + GS * 2.f * (hh[j] - NdotH * nn[j]) + GVH * vv[j];
            gnd[j] = GN * hh[j] + GS * 2.f * (nn[j] - NdotH * hh[j]) + GNV * vv[j];
        }
        if (hl > 1e-30f) {
            const float hg = hh[0] * gh[0] + hh[1] * gh[1] + hh[2] * gh[2];
#pragma unroll
            for (int j = 0; j < 3; ++j) gw[j] += (gh[j] - hg * hh[j]) / hl;
        }
        // w = l.x t(n) + l.y b(n) + l.z n
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            float v = l.z * gw[j] + gnd[j];
#pragma unroll
            for (int c = 0; c < 3; ++c) v += l.x * gw[c] * dt[c][j] + l.y * gw[c] * db[c][j];
            gn[j] += v;
        }
    }
    // blend weights W_k = w_s w_b / sum (Eq. 5-6) over the probes found (the
    // nonzero W: a found probe's weight is at least 0.01 w_s / sum): w_b moves
    // with the normal. A one-hot W (a point sitting on its nearest probe, or
    // a radius search that found one probe) and an all-zero one (none found)
    // do not depend on it; then W[1] == 0.
    const bool snapped = a.K > 1 && W[1] == 0.f;
    if (a.K > 1 && !snapped) {
        const float3 xp = load3(a.x, m);
        float U = 0.f, ws[KMAX], gdot = 0.f;
        float3 dh[KMAX];
#pragma unroll
        for (int k = 0; k < KMAX; ++k) {
            ws[k] = 0.f;
            dh[k] = f3(0.f, 0.f, 0.f);
            if (k < a.K && W[k] != 0.f) {
                const float3 d = load3(a.probe_pos, pid[k]) - xp;
                const float dl = sqrtf(dot3(d, d));
                ws[k] = 1.f / dl;
                dh[k] = (1.f / dl) * d;
                U += ws[k] * (0.5f * (1.f + dot3(dh[k], n)) + 0.01f);
                gdot += gW[k] * W[k];
            }
        }
#pragma unroll
        for (int k = 0; k < KMAX; ++k) {
            if (k < a.K && W[k] != 0.f) {
                const float gu = (gW[k] - gdot) / U;
                gn[0] += gu * ws[k] * 0.5f * dh[k].x;
                gn[1] += gu * ws[k] * 0.5f * dh[k].y;
                gn[2] += gu * ws[k] * 0.5f * dh[k].z;
            }
        }
    }
    // through n = n_raw / |n_raw|
    const float ng = gn[0] * n.x + gn[1] * n.y + gn[2] * n.z;
    a.g_normal[3 * m] = (gn[0] - ng * n.x) / nl;
    a.g_normal[3 * m + 1] = (gn[1] - ng * n.y) / nl;
    a.g_normal[3 * m + 2] = (gn[2] - ng * n.z) / nl;
    a.g_albedo[3 * m] = ga[0];
    a.g_albedo[3 * m + 1] = ga[1];
    a.g_albedo[3 * m + 2] = ga[2];
    a.g_rough[m] = gr;
    a.g_metal[m] = gm;
}

// ---- grouping of the points by nearest probe (counting sort) -----------------
__global__ void perm_count_kernel(const int32_t* __restrict__ idx, int32_t K, int64_t M, int32_t* __restrict__ bucket)
{
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m < M) atomicAdd(bucket + idx[m * K], 1);
}

__global__ void __launch_bounds__(1024) perm_scan_kernel(int32_t* __restrict__ bucket, int32_t P)
{
    __shared__ int32_t s_part[1024];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int chunk = (P + nt - 1) / nt, c0 = tid * chunk, c1 = min(P, c0 + chunk);
    int32_t sum = 0;
    for (int c = c0; c < c1; ++c) sum += bucket[c];
    s_part[tid] = sum;
    __syncthreads();
    for (int off = 1; off < nt; off <<= 1) {
        const int32_t v = tid >= off ? s_part[tid - off] : 0;
        __syncthreads();
        s_part[tid] += v;
        __syncthreads();
    }
    int32_t run = s_part[tid] - sum;
    for (int c = c0; c < c1; ++c) {
        const int32_t v = bucket[c];
        bucket[c] = run;
        run += v;
    }
}

__global__ void perm_fill_kernel(const int32_t* __restrict__ idx, int32_t K, int64_t M, int32_t* __restrict__ bucket,
                                 int32_t* __restrict__ perm)
{
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m < M) perm[atomicAdd(bucket + idx[m * K], 1)] = (int32_t)m;
}

__global__ void env_fold_kernel(const float4* __restrict__ genv4, int64_t n, float* __restrict__ g_env)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const float4 v = genv4[t];
    g_env[3 * t] += v.x;
    g_env[3 * t + 1] += v.y;
    g_env[3 * t + 2] += v.z;
}

template <int DT, int KMAX>
static cudaError_t adjoint_launch(const AdjK& k, cudaStream_t s)
{
    const size_t smem = sizeof(float4) * (size_t)k.S;
    auto fn = adjoint_kernel<DT, KMAX>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    fn<<<(unsigned)((k.M + 127) / 128), 128, smem, s>>>(k);
    return cudaGetLastError();
}

template <int DT>
static cudaError_t adjoint_k(const AdjK& k, cudaStream_t s)
{
    if (k.K <= 4) return adjoint_launch<DT, 4>(k, s);
    if (k.K <= 8) return adjoint_launch<DT, 8>(k, s);
    if (k.K <= 16) return adjoint_launch<DT, 16>(k, s);
    return adjoint_launch<DT, 32>(k, s);
}

cudaError_t launch_adjoint(const QueryArgs& a, const QueryLayout& L, char* ws, cudaStream_t s)
{
    if (a.M == 0) return cudaSuccess;
    AdjK k;
    k.x = a.x;
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
    k.env = a.env;
    k.dirs = reinterpret_cast<const float4*>(ws + L.dirs);
    k.idx = reinterpret_cast<const int32_t*>(ws + L.idx);
    k.w = reinterpret_cast<const float*>(ws + L.w);
    k.probe_pos = a.probe_pos;
    k.specular = a.specular;
    k.grad_out = a.grad_out;
    k.status = status_word();
    k.g_albedo = a.g_albedo;
    k.g_rough = a.g_rough;
    k.g_metal = a.g_metal;
    k.g_normal = a.g_normal;
    k.g_env = a.g_env;
    k.g_maps = reinterpret_cast<float4*>(a.g_atlas);
    int32_t* perm = reinterpret_cast<int32_t*>(ws + L.perm);
    int32_t* bucket = reinterpret_cast<int32_t*>(ws + L.bucket);
    k.perm = perm;
    k.genv4 = reinterpret_cast<float4*>(ws + L.genv4);

    cudaError_t e = cudaMemsetAsync(bucket, 0, sizeof(int32_t) * (size_t)(a.P + 1), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(k.genv4, 0, sizeof(float4) * (size_t)a.He * a.We, s);
    if (e != cudaSuccess) return e;
    const unsigned nb = (unsigned)((a.M + 255) / 256);
    perm_count_kernel<<<nb, 256, 0, s>>>(k.idx, a.K, a.M, bucket);
    perm_scan_kernel<<<1, 1024, 0, s>>>(bucket, a.P);
    perm_fill_kernel<<<nb, 256, 0, s>>>(k.idx, a.K, a.M, bucket, perm);
    switch (a.rgbo_dtype) {
    case SOP_F32: e = adjoint_k<SOP_F32>(k, s); break;
    case SOP_BF16: e = adjoint_k<SOP_BF16>(k, s); break;
    case SOP_F16: e = adjoint_k<SOP_F16>(k, s); break;
    default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    const int64_t ne = (int64_t)a.He * a.We;
    env_fold_kernel<<<(unsigned)((ne + 255) / 256), 256, 0, s>>>(k.genv4, ne, a.g_env);
    return cudaGetLastError();
}

}  // namespace sop
