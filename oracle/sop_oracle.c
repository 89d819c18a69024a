/*
 * FP64 CPU oracle for the Surface Octahedral Probe (SOP) bake and query/shade
 * of ComGS (arXiv 2510.07729).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may call, link or
 * load this file; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark use it. It shares no code, header or constant table
 * with the CUDA library: every step below is written out plainly, in double
 * precision, in the order the paper states it, with no blocking, fusion or
 * culling that the definition does not contain.
 *
 * Where the paper is silent the readings used are (each one also tested):
 *   - octahedral map: Cigolle et al. 2014 ("A Survey of Efficient
 *     Representations for Independent Unit Vectors"), z-up, world frame
 *     (Sec. 3.1.2 only names octahedral textures [Praun & Hoppe 2003]);
 *   - bilinear fetch across the octahedral folds: the DDGI border rule of
 *     Majercik et al. 2019 (the work the back-face weight of Sec. 3.1.2 cites);
 *   - ray-Gaussian response: the 3D Gaussian's maximum along the ray,
 *     alpha = min(alpha_max, o exp(-m^2/2)), kept when alpha >= alpha_min,
 *     composited front to back by Eq. 1 (T_i = prod (1 - alpha_j));
 *   - K nearest probes (Eq. 4) by an exact integer squared distance on
 *     positions quantised to 2^-20, ties to the lower probe index;
 *   - weights w_s = 1/|d_k| (Eq. 5), w_b = 0.5 (1 + d_k/|d_k| . n) + 0.01
 *     (Eq. 6) with n the shading normal, one-hot on the nearest probe when it
 *     coincides with the shading point;
 *   - S_r directions: Hammersley with centred first coordinate,
 *     z_i = (i + 1/2)/S, phi_i = 2 pi radical_inverse_2(i), uniform on the
 *     hemisphere, rotated by the branchless ONB of Duff et al. 2017;
 *   - "simplified Disney" BRDF (Sec. 3.1.2): Lambert (1-m) a/pi plus GGX
 *     specular D F G / (4 NdotL NdotV), alpha = r^2, Schlick-GGX k=(r+1)^2/8,
 *     F0 = 0.08 spec (1-m) + a m, Schlick Fresnel;
 *   - equirectangular environment, z-up, u = (phi + pi)/(2 pi),
 *     v = theta/pi, bilinear with u wrapping and v clamped; or (Sec. 4.1)
 *     an octahedral environment with the probe maps' mapping and border.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------ */
/* Octahedral map (Sec. 3.1.2, octahedral textures).                         */
/* ------------------------------------------------------------------------ */
static double sgn_nz(double v) { return v >= 0.0 ? 1.0 : -1.0; }

/* Unit direction -> uv in [0,1]^2. */
void orc_oct_encode(const double* d, double* uv)
{
    double l1 = fabs(d[0]) + fabs(d[1]) + fabs(d[2]);
    double px = d[0] / l1, py = d[1] / l1;
    if (d[2] < 0.0) {
        double qx = (1.0 - fabs(py)) * sgn_nz(px);
        double qy = (1.0 - fabs(px)) * sgn_nz(py);
        px = qx;
        py = qy;
    }
    uv[0] = 0.5 * (px + 1.0);
    uv[1] = 0.5 * (py + 1.0);
}

/* uv -> the point of the L1 unit octahedron (not normalised). */
void orc_oct_decode_l1(const double* uv, double* d)
{
    double px = 2.0 * uv[0] - 1.0, py = 2.0 * uv[1] - 1.0;
    double z = 1.0 - fabs(px) - fabs(py);
    if (z < 0.0) {
        double qx = (1.0 - fabs(py)) * sgn_nz(px);
        double qy = (1.0 - fabs(px)) * sgn_nz(py);
        px = qx;
        py = qy;
    }
    d[0] = px;
    d[1] = py;
    d[2] = z;
}

/* uv -> unit direction. */
void orc_oct_decode(const double* uv, double* d)
{
    orc_oct_decode_l1(uv, d);
    double n = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    d[0] /= n;
    d[1] /= n;
    d[2] /= n;
}

/* Texel (i = column along u, j = row along v) centre direction. */
void orc_texel_dir(int R, int i, int j, double* d)
{
    double uv[2] = {(i + 0.5) / R, (j + 0.5) / R};
    orc_oct_decode(uv, d);
}

/* Border rule: a texel index pair in [-1, R]^2 -> the texel it stands for.
 * Crossing an edge of the square mirrors the index along that edge; the
 * four corners map to the diagonally opposite corner. */
void orc_oct_wrap(int R, int i, int j, int* si, int* sj)
{
    int oi = (i < 0) || (i >= R), oj = (j < 0) || (j >= R);
    if (oi && oj) {
        *si = (i < 0) ? R - 1 : 0;
        *sj = (j < 0) ? R - 1 : 0;
    } else if (oi) {
        *si = (i < 0) ? 0 : R - 1;
        *sj = R - 1 - j;
    } else if (oj) {
        *si = R - 1 - i;
        *sj = (j < 0) ? 0 : R - 1;
    } else {
        *si = i;
        *sj = j;
    }
}

/* Bilinear read of a compact map [R][R][C] (row j, column i) at uv. */
void orc_oct_bilerp(const double* map, int R, int C, const double* uv, double* out)
{
    double s = uv[0] * R - 0.5, t = uv[1] * R - 0.5;
    double fi = floor(s), fj = floor(t);
    double fu = s - fi, fv = t - fj;
    int i0 = (int)fi, j0 = (int)fj;
    for (int c = 0; c < C; ++c) out[c] = 0.0;
    for (int dj = 0; dj < 2; ++dj)
        for (int di = 0; di < 2; ++di) {
            double w = (di ? fu : 1.0 - fu) * (dj ? fv : 1.0 - fv);
            int si, sj;
            orc_oct_wrap(R, i0 + di, j0 + dj, &si, &sj);
            const double* tex = map + ((size_t)sj * R + si) * C;
            for (int c = 0; c < C; ++c) out[c] += w * tex[c];
        }
}

/* ------------------------------------------------------------------------ */
/* Probe bake (Sec. 3.1.2 "initialised via ray tracing"; Sec. 3.2.2 occlusion */
/* caching; compositing of Eq. 1; depth normalisation D/W of Sec. 3.1).       */
/* ------------------------------------------------------------------------ */
typedef struct {
    double t, alpha;
    double dalpha, Tb; /* orc_bake_rays: bound of |d alpha|; transmittance before the hit */
    int64_t idx;
} orc_hit;

static int hit_cmp(const void* a, const void* b)
{
    const orc_hit* x = (const orc_hit*)a;
    const orc_hit* y = (const orc_hit*)b;
    if (x->t < y->t) return -1;
    if (x->t > y->t) return 1;
    return (x->idx < y->idx) ? -1 : (x->idx > y->idx);
}

/* Rotation matrix of a unit quaternion (w, x, y, z); columns are the
 * Gaussian's local axes in world space. */
static void quat_to_rot(const float* q4, double Rm[3][3])
{
    double w = q4[0], x = q4[1], y = q4[2], z = q4[3];
    double n = sqrt(w * w + x * x + y * y + z * z);
    w /= n; x /= n; y /= n; z /= n;
    Rm[0][0] = 1 - 2 * (y * y + z * z); Rm[0][1] = 2 * (x * y - w * z);     Rm[0][2] = 2 * (x * z + w * y);
    Rm[1][0] = 2 * (x * y + w * z);     Rm[1][1] = 1 - 2 * (x * x + z * z); Rm[1][2] = 2 * (y * z - w * x);
    Rm[2][0] = 2 * (x * z - w * y);     Rm[2][1] = 2 * (y * z + w * x);     Rm[2][2] = 1 - 2 * (x * x + y * y);
}

/* Flags a texel whose FP32 result may legitimately differ from this FP64
 * one because a floating-point comparison is within rounding of flipping. */
enum {
    ORC_FLAG_ALPHA_MIN = 1, /* a response within 1e-4 relative of alpha_min  */
    ORC_FLAG_ORDER = 2,     /* two kept hits whose t* differ by <= 1e-6 rel.  */
    ORC_FLAG_TNEAR = 4,     /* a t* within rounding of t_near                 */
    ORC_FLAG_TSTOP = 8,     /* transmittance within 1e-3 relative of T_stop   */
};

/* Bake n_rays texel rays. Ray r starts at probe probe_of[r] and points at the
 * centre of texel (ti[r], tj[r]) of an R x R map. Outputs per ray: RGB
 * indirect radiance L, occlusion O = 1 - T, depth D = sum(T a t*)/sum(T a)
 * (0 when nothing is hit) and ambiguity flags.
 *
 * Test allowance (out_sens [n_rays][5]: L0, L1, L2, O, D; NULL to skip): how
 * far each output may move when the ray direction carries an angular error
 * of up to eps_dir (an FP32 path holds the direction rounded to single
 * precision). At the point of maximum response m^2 is stationary in t, so
 * to first order only the rotation of the ray moves it: with e = M (p - mu
 * + t* d) the whitened offset there, dm^2 = 2 e . (t* M dd) and |dm^2| <=
 * 2 |e| t* |M|_2 eps_dir, |M|_2 = max 1/s; hence |d alpha| <= alpha |e| t*
 * max(1/s) eps_dir (0 where alpha is clamped at alpha_max). Each composited
 * hit's |d alpha| is carried to the outputs through their partial
 * derivatives in alpha (the later hits' transmittances hold 1 - alpha) and
 * summed in absolute value. A response within that |d alpha| of alpha_min
 * is flagged like one within 1e-4 relative of it. */
void orc_bake_rays(int64_t N, const float* mean, const float* scale, const float* quat,
                   const float* opacity, const float* rgb, const float* probe_pos, int R,
                   int64_t n_rays, const int32_t* probe_of, const int32_t* ti, const int32_t* tj,
                   double t_near, double alpha_min, double alpha_max, double t_stop,
                   double* out_rgb, double* out_occ, double* out_depth, int32_t* out_flags,
                   double eps_dir, double* out_sens)
{
    /* Per-Gaussian M = diag(1/s) R^T, so that m^2(x) = |M (x - mu)|^2. */
    double* Mg = (double*)malloc(sizeof(double) * 9 * (size_t)(N > 0 ? N : 1));
    double* Mn = (double*)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1)); /* |M|_2 = max 1/s */
    for (int64_t g = 0; g < N; ++g) {
        double Rm[3][3];
        quat_to_rot(quat + 4 * g, Rm);
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) Mg[9 * g + 3 * a + b] = Rm[b][a] / (double)scale[3 * g + a];
        Mn[g] = 0.0;
        for (int a = 0; a < 3; ++a)
            if (1.0 / (double)scale[3 * g + a] > Mn[g]) Mn[g] = 1.0 / (double)scale[3 * g + a];
    }
#pragma omp parallel
    {
        size_t cap = 1024;
        orc_hit* hits = (orc_hit*)malloc(sizeof(orc_hit) * cap);
#pragma omp for schedule(dynamic, 4)
        for (int64_t r = 0; r < n_rays; ++r) {
            const float* p = probe_pos + 3 * (size_t)probe_of[r];
            double d[3];
            orc_texel_dir(R, ti[r], tj[r], d);
            size_t nh = 0;
            int flags = 0;
            for (int64_t g = 0; g < N; ++g) {
                const double* M = Mg + 9 * g;
                double del[3] = {(double)p[0] - mean[3 * g], (double)p[1] - mean[3 * g + 1],
                                 (double)p[2] - mean[3 * g + 2]};
                double u[3], w[3];
                for (int a = 0; a < 3; ++a) {
                    u[a] = M[3 * a] * del[0] + M[3 * a + 1] * del[1] + M[3 * a + 2] * del[2];
                    w[a] = M[3 * a] * d[0] + M[3 * a + 1] * d[1] + M[3 * a + 2] * d[2];
                }
                double A = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
                double B = w[0] * u[0] + w[1] * u[1] + w[2] * u[2];
                double ts = -B / A;
                double m2 = 0.0;
                for (int a = 0; a < 3; ++a) {
                    double e = u[a] + ts * w[a];
                    m2 += e * e;
                }
                double resp = opacity[g] * exp(-0.5 * m2);
                double dl = sqrt(del[0] * del[0] + del[1] * del[1] + del[2] * del[2]);
                const double da = resp * sqrt(m2) * fabs(ts) * Mn[g] * eps_dir;
                if (fabs(resp - alpha_min) <= fmax(1e-4 * alpha_min, da) && ts > t_near) flags |= ORC_FLAG_ALPHA_MIN;
                if (resp >= alpha_min && fabs(ts - t_near) <= 1e-5 * (dl + 1e-3)) flags |= ORC_FLAG_TNEAR;
                if (ts <= t_near) continue;
                if (resp < alpha_min) continue;
                if (nh == cap) {
                    cap *= 2;
                    hits = (orc_hit*)realloc(hits, sizeof(orc_hit) * cap);
                }
                hits[nh].t = ts;
                hits[nh].alpha = resp < alpha_max ? resp : alpha_max;
                hits[nh].dalpha = resp < alpha_max ? da : 0.0;
                hits[nh].idx = g;
                ++nh;
            }
            qsort(hits, nh, sizeof(orc_hit), hit_cmp);
            double T = 1.0, L[3] = {0, 0, 0}, Dacc = 0.0, W = 0.0;
            size_t nc = 0; /* hits composited */
            for (size_t k = 0; k < nh; ++k) {
                nc = k + 1;
                if (k + 1 < nh && hits[k + 1].t - hits[k].t <= 1e-6 * fabs(hits[k + 1].t)) flags |= ORC_FLAG_ORDER;
                double wk = T * hits[k].alpha;
                hits[k].Tb = T;
                const float* c = rgb + 3 * hits[k].idx;
                L[0] += wk * c[0];
                L[1] += wk * c[1];
                L[2] += wk * c[2];
                Dacc += wk * hits[k].t;
                W += wk;
                T *= (1.0 - hits[k].alpha);
                if (t_stop > 0.0 && fabs(T - t_stop) <= 1e-3 * t_stop) flags |= ORC_FLAG_TSTOP;
                if (T < t_stop) break;
            }
            out_rgb[3 * r] = L[0];
            out_rgb[3 * r + 1] = L[1];
            out_rgb[3 * r + 2] = L[2];
            out_occ[r] = 1.0 - T;
            out_depth[r] = (W > 1e-8) ? Dacc / W : 0.0;
            out_flags[r] = flags;
            if (out_sens) {
                /* X = sum_k T_k a_k x_k with T_k = prod_{j<k} (1 - a_j):
                 * dX/da_k = T_k x_k - (sum_{j>k} T_j a_j x_j) / (1 - a_k);
                 * O = 1 - prod (1 - a_j): dO/da_k = T_end / (1 - a_k). The
                 * suffix sums run from the last composited hit down. */
                double sL[3] = {0, 0, 0}, sD = 0.0, sW = 0.0, sens[5] = {0, 0, 0, 0, 0};
                const double Dv = (W > 1e-8) ? Dacc / W : 0.0;
                for (size_t k = nc; k-- > 0;) {
                    const double a = hits[k].alpha, om = 1.0 - a, Tk = hits[k].Tb;
                    const double wk = Tk * a;
                    const float* c = rgb + 3 * hits[k].idx;
                    double dX[5];
                    for (int q = 0; q < 3; ++q) dX[q] = Tk * c[q] - sL[q] / om;
                    dX[3] = T / om;
                    const double dDacc = Tk * hits[k].t - sD / om, dW = Tk - sW / om;
                    dX[4] = (W > 1e-8) ? (dDacc - Dv * dW) / W : 0.0;
                    for (int q = 0; q < 5; ++q) sens[q] += fabs(dX[q]) * hits[k].dalpha;
                    for (int q = 0; q < 3; ++q) sL[q] += wk * c[q];
                    sD += wk * hits[k].t;
                    sW += wk;
                }
                for (int q = 0; q < 5; ++q) out_sens[5 * r + q] = sens[q];
            }
        }
        free(hits);
    }
    free(Mn);
    free(Mg);
}

/* ------------------------------------------------------------------------ */
/* Query: K nearest probes and blend weights (Sec. 3.1.2, Eq. 4-6).           */
/* ------------------------------------------------------------------------ */
static int64_t quantise(float v) { return (int64_t)nearbyint((double)v * 1048576.0); }

/* Exact K nearest probes of each point, by the integer squared distance of
 * positions quantised to 2^-20, ties to the lower probe index. With a
 * search radius (Sec. 3.2, fixed-radius neighbours) only probes whose key is
 * <= r2_key take part; slots left empty hold index -1 and key UINT64_MAX.
 * r2_key = UINT64_MAX is the plain K nearest. */
void orc_knn(int64_t M, const float* x, int32_t P, const float* probe_pos, int32_t K, uint64_t r2_key,
             int32_t* out_idx, uint64_t* out_key)
{
#pragma omp parallel for schedule(static)
    for (int64_t m = 0; m < M; ++m) {
        int64_t qx = quantise(x[3 * m]), qy = quantise(x[3 * m + 1]), qz = quantise(x[3 * m + 2]);
        int32_t* bi = out_idx + (size_t)m * K;
        uint64_t* bk = out_key + (size_t)m * K;
        int n = 0;
        for (int32_t p = 0; p < P; ++p) {
            int64_t dx = quantise(probe_pos[3 * p]) - qx;
            int64_t dy = quantise(probe_pos[3 * p + 1]) - qy;
            int64_t dz = quantise(probe_pos[3 * p + 2]) - qz;
            uint64_t key = (uint64_t)(dx * dx) + (uint64_t)(dy * dy) + (uint64_t)(dz * dz);
            if (key > r2_key) continue;
            /* insertion into the sorted list of the best K (key, index) */
            if (n == K && key >= bk[K - 1]) continue; /* equal key: larger index loses */
            int pos = (n < K) ? n++ : K - 1;
            while (pos > 0 && bk[pos - 1] > key) {
                bk[pos] = bk[pos - 1];
                bi[pos] = bi[pos - 1];
                --pos;
            }
            bk[pos] = key;
            bi[pos] = p;
        }
        for (int k = n; k < K; ++k) {
            bi[k] = -1;
            bk[k] = UINT64_MAX;
        }
    }
}

/* Normalised blend weights W_k = w_s w_b / sum_j w_s w_b (Eq. 4-6) for the
 * neighbours found by orc_knn. When the nearest probe's quantised squared
 * distance is <= snap_key the point sits on that probe: W is one-hot. Empty
 * slots (index -1) weigh 0; with no neighbour at all every W is 0. */
void orc_weights(int64_t M, const float* x, const float* n, const float* probe_pos, int32_t K,
                 const int32_t* idx, const uint64_t* key, uint64_t snap_key, double* out_w)
{
#pragma omp parallel for schedule(static)
    for (int64_t m = 0; m < M; ++m) {
        double* W = out_w + (size_t)m * K;
        const int32_t* id = idx + (size_t)m * K;
        if (id[0] < 0) {
            for (int k = 0; k < K; ++k) W[k] = 0.0;
            continue;
        }
        if (key[(size_t)m * K] <= snap_key) {
            for (int k = 0; k < K; ++k) W[k] = (k == 0) ? 1.0 : 0.0;
            continue;
        }
        double nn[3] = {n[3 * m], n[3 * m + 1], n[3 * m + 2]};
        double nl = sqrt(nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2]);
        double sum = 0.0;
        for (int k = 0; k < K; ++k) {
            W[k] = 0.0;
            if (id[k] < 0) continue;
            const float* p = probe_pos + 3 * (size_t)id[k];
            double d[3] = {(double)p[0] - x[3 * m], (double)p[1] - x[3 * m + 1], (double)p[2] - x[3 * m + 2]};
            double dl = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            double ws = 1.0 / dl;
            double wb = 0.5 * (1.0 + (d[0] * nn[0] + d[1] * nn[1] + d[2] * nn[2]) / (dl * nl)) + 0.01;
            W[k] = ws * wb;
            sum += W[k];
        }
        for (int k = 0; k < K; ++k) W[k] /= sum;
    }
}

/* ------------------------------------------------------------------------ */
/* Light directions, frame, environment and BRDF (Sec. 3.1.2, Eq. 2-3).        */
/* ------------------------------------------------------------------------ */
static double radical_inverse2(uint32_t i)
{
    double r = 0.0, f = 0.5;
    while (i) {
        if (i & 1u) r += f;
        f *= 0.5;
        i >>= 1;
    }
    return r;
}

/* The S_r local directions (z = cos theta about the normal). */
void orc_hammersley(int32_t S, double* out)
{
    for (int32_t i = 0; i < S; ++i) {
        double z = (i + 0.5) / S;
        double phi = 2.0 * M_PI * radical_inverse2((uint32_t)i);
        double s = sqrt(1.0 - z * z);
        out[3 * i] = s * cos(phi);
        out[3 * i + 1] = s * sin(phi);
        out[3 * i + 2] = z;
    }
}

/* Orthonormal frame (t, b, n) of a unit normal (Duff et al. 2017). */
void orc_onb(const double* n, double* t, double* b)
{
    double sg = n[2] >= 0.0 ? 1.0 : -1.0;
    double a = -1.0 / (sg + n[2]);
    double c = n[0] * n[1] * a;
    t[0] = 1.0 + sg * n[0] * n[0] * a;
    t[1] = sg * c;
    t[2] = -sg * n[0];
    b[0] = c;
    b[1] = sg + n[1] * n[1] * a;
    b[2] = -n[1];
}

/* Equirectangular environment lookup L_dir(w), bilinear, u wraps, v clamps. */
void orc_env_lookup(const float* env, int32_t He, int32_t We, const double* w, double* out)
{
    double theta = atan2(sqrt(w[0] * w[0] + w[1] * w[1]), w[2]);
    double phi = atan2(w[1], w[0]);
    double u = (phi + M_PI) / (2.0 * M_PI), v = theta / M_PI;
    double s = u * We - 0.5, t = v * He - 0.5;
    double fs = floor(s), ft = floor(t);
    double a = s - fs, b = t - ft;
    int c0 = (int)fs, r0 = (int)ft;
    out[0] = out[1] = out[2] = 0.0;
    for (int dr = 0; dr < 2; ++dr)
        for (int dc = 0; dc < 2; ++dc) {
            int r = r0 + dr, c = c0 + dc;
            r = r < 0 ? 0 : (r > He - 1 ? He - 1 : r);
            c = ((c % We) + We) % We;
            double wgt = (dc ? a : 1.0 - a) * (dr ? b : 1.0 - b);
            const float* e = env + ((size_t)r * We + c) * 3;
            out[0] += wgt * e[0];
            out[1] += wgt * e[1];
            out[2] += wgt * e[2];
        }
}

/* Octahedral environment lookup (Sec. 4.1: the estimated environment map is
 * converted to an octahedral texture): env [H][H][3] with the mapping and the
 * border rule of the probe maps (texel (i, j) = column i along u, row j
 * along v), bilinear. */
void orc_env_oct_lookup(const float* env, int32_t H, const double* w, double* out)
{
    double uv[2];
    orc_oct_encode(w, uv);
    double s = uv[0] * H - 0.5, t = uv[1] * H - 0.5;
    double fi = floor(s), fj = floor(t);
    double fu = s - fi, fv = t - fj;
    int i0 = (int)fi, j0 = (int)fj;
    out[0] = out[1] = out[2] = 0.0;
    for (int dj = 0; dj < 2; ++dj)
        for (int di = 0; di < 2; ++di) {
            double wgt = (di ? fu : 1.0 - fu) * (dj ? fv : 1.0 - fv);
            int si, sj;
            orc_oct_wrap(H, i0 + di, j0 + dj, &si, &sj);
            const float* e = env + ((size_t)sj * H + si) * 3;
            out[0] += wgt * e[0];
            out[1] += wgt * e[1];
            out[2] += wgt * e[2];
        }
}

/* L_dir(w) from the environment in its layout: 0 = equirectangular [He][We],
 * 1 = octahedral [He][He]. */
void orc_env_sample(const float* env, int32_t He, int32_t We, int32_t layout, const double* w, double* out)
{
    if (layout == 1) orc_env_oct_lookup(env, He, w, out);
    else orc_env_lookup(env, He, We, w, out);
}

/* Resample an equirectangular environment [He][We][3] into an octahedral one
 * [H][H][3]: each texel holds the bilinear equirectangular value at its
 * centre direction. */
void orc_env_to_oct(const float* env, int32_t He, int32_t We, int32_t H, double* out)
{
    for (int j = 0; j < H; ++j)
        for (int i = 0; i < H; ++i) {
            double d[3];
            orc_texel_dir(H, i, j, d);
            orc_env_lookup(env, He, We, d, out + ((size_t)j * H + i) * 3);
        }
}

/* Importance-sampled light directions (Sec. 4.2, Eq. PDF: density
 * H W I / (4 pi) over the octahedral environment's texels): S world
 * directions with their density, out [S][4] = (x, y, z, pdf). Readings: the
 * intensity of a texel is the float32 sum r + g + b; it is quantised to
 * q_t = max(1, floor(I_t / I_max 2^20)) (in double) so that the choice of a
 * texel is an exact integer decision; sample i takes the texel whose
 * cumulative interval [C_{t-1}, C_t) holds floor((2i + 1) Q / (2S)),
 * Q = sum q (stratified); its direction is the texel centre and its density
 * H^2 q_t / (4 pi Q) (texels of equal solid angle, as the equation takes). */
void orc_env_importance_dirs(const float* env, int32_t H, int32_t S, double* out)
{
    const int64_t T = (int64_t)H * H;
    float imax = 0.f;
    for (int64_t t = 0; t < T; ++t) {
        float I = env[3 * t] + env[3 * t + 1] + env[3 * t + 2];
        if (I > imax) imax = I;
    }
    int64_t* cum = (int64_t*)malloc(sizeof(int64_t) * (size_t)T);
    int64_t Q = 0;
    for (int64_t t = 0; t < T; ++t) {
        float I = env[3 * t] + env[3 * t + 1] + env[3 * t + 2];
        int64_t q = imax > 0.f ? (int64_t)floor((double)I / (double)imax * 1048576.0) : 1;
        if (q < 1) q = 1;
        Q += q;
        cum[t] = Q;
    }
    for (int32_t i = 0; i < S; ++i) {
        const int64_t target = (2 * (int64_t)i + 1) * Q / (2 * (int64_t)S);
        int64_t lo = 0, hi = T - 1;  /* smallest t with cum[t] > target */
        while (lo < hi) {
            const int64_t mid = (lo + hi) / 2;
            if (cum[mid] > target) hi = mid;
            else lo = mid + 1;
        }
        const int64_t q = cum[lo] - (lo > 0 ? cum[lo - 1] : 0);
        double d[3];
        orc_texel_dir(H, (int)(lo % H), (int)(lo / H), d);
        out[4 * i] = d[0];
        out[4 * i + 1] = d[1];
        out[4 * i + 2] = d[2];
        out[4 * i + 3] = (double)T * (double)q / (4.0 * M_PI * (double)Q);
    }
    free(cum);
}

/* GGX / Trowbridge-Reitz normal distribution D(h) for alpha = r^2, written
 * with sin^2 = |n x h|^2 so that it stays accurate near n . h = 1. */
double orc_ggx_D(double NdotH, double sin2, double rough)
{
    double al = rough * rough, a2 = al * al;
    double den = NdotH * NdotH * a2 + sin2;
    return a2 / (M_PI * den * den);
}

/* Schlick-GGX masking term of one direction, k = (r + 1)^2 / 8. */
double orc_smith_G1(double NdotX, double rough)
{
    double k = (rough + 1.0) * (rough + 1.0) / 8.0;
    return NdotX / (NdotX * (1.0 - k) + k);
}

/* Schlick Fresnel. */
double orc_fresnel(double F0, double VdotH) { return F0 + (1.0 - F0) * pow(1.0 - VdotH, 5.0); }

/* Simplified Disney BRDF value f(wo, wi) per channel (Sec. 3.1.2). */
void orc_brdf(const double* n, const double* wo, const double* wi, const double* albedo, double rough,
              double metal, double spec, double* f)
{
    double h[3] = {wi[0] + wo[0], wi[1] + wo[1], wi[2] + wo[2]};
    double hl = sqrt(h[0] * h[0] + h[1] * h[1] + h[2] * h[2]);
    if (hl < 1e-30) {
        h[0] = n[0]; h[1] = n[1]; h[2] = n[2];
    } else {
        h[0] /= hl; h[1] /= hl; h[2] /= hl;
    }
    double NdotL = n[0] * wi[0] + n[1] * wi[1] + n[2] * wi[2];
    double NdotV = n[0] * wo[0] + n[1] * wo[1] + n[2] * wo[2];
    if (NdotV < 1e-4) NdotV = 1e-4;
    double NdotH = n[0] * h[0] + n[1] * h[1] + n[2] * h[2];
    double VdotH = wo[0] * h[0] + wo[1] * h[1] + wo[2] * h[2];
    double cx = n[1] * h[2] - n[2] * h[1], cy = n[2] * h[0] - n[0] * h[2], cz = n[0] * h[1] - n[1] * h[0];
    double D = orc_ggx_D(NdotH, cx * cx + cy * cy + cz * cz, rough);
    double G = orc_smith_G1(NdotL, rough) * orc_smith_G1(NdotV, rough);
    for (int c = 0; c < 3; ++c) {
        double F0 = 0.08 * spec * (1.0 - metal) + albedo[c] * metal;
        double F = orc_fresnel(F0, VdotH);
        f[c] = (1.0 - metal) * albedo[c] / M_PI + D * F * G / (4.0 * NdotL * NdotV);
    }
}

/* ------------------------------------------------------------------------ */
/* Query + shade (Sec. 3.1.2 Eq. 2-6; shadow ratio of Sec. 3.2.2, Eq. 7-9).    */
/* ------------------------------------------------------------------------ */
enum { ORC_MODE_SHADE = 0, ORC_MODE_SHADOW = 1 };

/* One light direction's terms at a shading point (unit normal nn, view vo,
 * material a/rough/metal, K neighbours with weights W): O and L_in blended
 * from the probes' octahedral maps at w (Eq. 4), L_dir from the environment,
 * then
 *   shade : g[0..2] = f(wo, w) ((1 - O) L_dir + L_in) (n . w)     (Eq. 3, 4)
 *   shadow: g[0..2] = L_dir (1 - O) (n . w), g[3..5] = L_dir (n . w) (Eq. 7-8) */
static void sample_terms(const double* nn, const double* vo, const double* a, double rough, double metal, double spec,
                         int mode, const double* w, int32_t K, const int32_t* idx, const double* W, int32_t R,
                         const double* mrgb, const double* mocc, const float* env, int32_t He, int32_t We,
                         int32_t env_layout, double* g)
{
    size_t RR = (size_t)R * R;
    double uv[2];
    orc_oct_encode(w, uv);
    double O = 0.0, Lin[3] = {0, 0, 0};
    for (int k = 0; k < K; ++k) {
        if (idx[k] < 0) continue;
        double o1, l3[3];
        orc_oct_bilerp(mocc + RR * idx[k], R, 1, uv, &o1);
        orc_oct_bilerp(mrgb + 3 * RR * idx[k], R, 3, uv, l3);
        O += W[k] * o1;
        for (int c = 0; c < 3; ++c) Lin[c] += W[k] * l3[c];
    }
    double Ld[3];
    orc_env_sample(env, He, We, env_layout, w, Ld);
    double NdotL = nn[0] * w[0] + nn[1] * w[1] + nn[2] * w[2];
    if (mode == ORC_MODE_SHADE) {
        double f[3];
        orc_brdf(nn, vo, w, a, rough, metal, spec, f);
        for (int c = 0; c < 3; ++c) g[c] = f[c] * ((1.0 - O) * Ld[c] + Lin[c]) * NdotL;
    } else {
        for (int c = 0; c < 3; ++c) {
            g[c] = Ld[c] * (1.0 - O) * NdotL;
            g[3 + c] = Ld[c] * NdotL;
        }
    }
}

static void query_setup(int64_t M, const float* x, const float* n, int32_t P, const float* probe_pos, int32_t R,
                        const float* maps_rgb, const float* maps_occ, int32_t S, const double* dirs, int32_t dir_world,
                        int32_t K, uint64_t snap_key, uint64_t r2_key, int32_t* out_idx, double* out_w, double** dl,
                        double** mrgb, double** mocc)
{
    const size_t st = dir_world ? 4 : 3;
    *dl = (double*)malloc(sizeof(double) * st * (size_t)S);
    if (dirs) memcpy(*dl, dirs, sizeof(double) * st * (size_t)S);
    else orc_hammersley(S, *dl);
    size_t RR = (size_t)R * R;
    *mrgb = (double*)malloc(sizeof(double) * 3 * RR * (size_t)P);
    *mocc = (double*)malloc(sizeof(double) * RR * (size_t)P);
    for (size_t i = 0; i < 3 * RR * (size_t)P; ++i) (*mrgb)[i] = maps_rgb[i];
    for (size_t i = 0; i < RR * (size_t)P; ++i) (*mocc)[i] = maps_occ[i];
    uint64_t* key = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(M > 0 ? M : 1) * K);
    orc_knn(M, x, P, probe_pos, K, r2_key, out_idx, key);
    orc_weights(M, x, n, probe_pos, K, out_idx, key, snap_key, out_w);
    free(key);
}

/* World direction w of sample i and its Monte Carlo weight: a local
 * direction rotated into the frame (t, b, n) with weight 1 (the 2 pi / S
 * factor is applied at the end), or (dir_world) an importance-sampled world
 * direction with weight 1 / pdf, 0 below the point's horizon. */
static double sample_dir(const double* dl, int32_t dir_world, int32_t i, const double* t, const double* b,
                         const double* nn, double* w)
{
    if (dir_world) {
        const double* l = dl + 4 * (size_t)i;
        w[0] = l[0]; w[1] = l[1]; w[2] = l[2];
        return (nn[0] * w[0] + nn[1] * w[1] + nn[2] * w[2]) > 0.0 ? 1.0 / l[3] : 0.0;
    }
    const double* l = dl + 3 * (size_t)i;
    for (int c = 0; c < 3; ++c) w[c] = l[0] * t[c] + l[1] * b[c] + l[2] * nn[c];
    return 1.0;
}

static void point_frame(const float* n, const float* wo, const float* albedo, int64_t m, double* nn, double* vo,
                        double* a, double* t, double* b)
{
    nn[0] = n[3 * m]; nn[1] = n[3 * m + 1]; nn[2] = n[3 * m + 2];
    double nl = sqrt(nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2]);
    nn[0] /= nl; nn[1] /= nl; nn[2] /= nl;
    vo[0] = wo[3 * m]; vo[1] = wo[3 * m + 1]; vo[2] = wo[3 * m + 2];
    a[0] = albedo[3 * m]; a[1] = albedo[3 * m + 1]; a[2] = albedo[3 * m + 2];
    orc_onb(nn, t, b);
}

/* For each shading point: K nearest probes, weights, then the Monte Carlo sum
 * over the S directions of
 *   shade : C = 2pi/S sum f ((1 - O) L_dir + L_in) (n . w_i)      (Eq. 3, 4)
 *   shadow: S_c = sum L_dir (1 - O) (n . w_i) / sum L_dir (n . w_i) (Eq. 7-9)
 * with O and L_in blended from the probes' octahedral maps. maps_rgb is the
 * compact [P][R][R][3] radiance, maps_occ the [P][R][R] occlusion. dirs is the
 * local direction set [S][3]; NULL selects orc_hammersley(S). */
void orc_query_shade(int64_t M, const float* x, const float* n, const float* wo, const float* albedo,
                     const float* rough, const float* metal, int32_t P, const float* probe_pos, int32_t R,
                     const float* maps_rgb, const float* maps_occ, int32_t He, int32_t We, const float* env,
                     int32_t S, const double* dirs, int32_t K, int32_t mode, double spec, uint64_t snap_key,
                     uint64_t r2_key, int32_t env_layout, int32_t dir_world, double* out, int32_t* out_idx,
                     double* out_w)
{
    double *dl, *mrgb, *mocc;
    query_setup(M, x, n, P, probe_pos, R, maps_rgb, maps_occ, S, dirs, dir_world, K, snap_key, r2_key, out_idx, out_w,
                &dl, &mrgb, &mocc);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t m = 0; m < M; ++m) {
        double nn[3], vo[3], a[3], t[3], b[3];
        point_frame(n, wo, albedo, m, nn, vo, a, t, b);
        double acc[6] = {0, 0, 0, 0, 0, 0};
        for (int32_t i = 0; i < S; ++i) {
            double w[3], g[6];
            const double wt = sample_dir(dl, dir_world, i, t, b, nn, w);
            if (wt == 0.0) continue;
            sample_terms(nn, vo, a, rough[m], metal[m], spec, mode, w, K, out_idx + (size_t)m * K,
                         out_w + (size_t)m * K, R, mrgb, mocc, env, He, We, env_layout, g);
            for (int c = 0; c < (mode == ORC_MODE_SHADE ? 3 : 6); ++c) acc[c] += wt * g[c];
        }
        for (int c = 0; c < 3; ++c) {
            if (mode == ORC_MODE_SHADE) out[3 * m + c] = (dir_world ? 1.0 : 2.0 * M_PI) / S * acc[c];
            else out[3 * m + c] = (acc[3 + c] < 1e-20) ? 1.0 : acc[c] / acc[3 + c];
        }
    }
    free(mocc);
    free(mrgb);
    free(dl);
}

/* Test allowance for an FP32 evaluation of orc_query_shade: how far each
 * output may move when every light direction carries an angular error of
 * up to eps (the rounding of the frame, of the rotation into world space
 * and of atan2 in single precision). Each direction's terms are re-evaluated
 * at four directions rotated by eps about two axes normal to it; the largest
 * change per term is summed over directions (shadow: propagated through the
 * ratio). The environment and probe maps are piecewise bilinear, so this is
 * their local slope times eps; it is what separates a rough HDR environment,
 * where neighbouring texels differ by 10x, from a smooth one. */
void orc_query_shade_sensitivity(int64_t M, const float* x, const float* n, const float* wo, const float* albedo,
                                 const float* rough, const float* metal, int32_t P, const float* probe_pos, int32_t R,
                                 const float* maps_rgb, const float* maps_occ, int32_t He, int32_t We,
                                 const float* env, int32_t S, const double* dirs, int32_t K, int32_t mode, double spec,
                                 uint64_t snap_key, uint64_t r2_key, int32_t env_layout, int32_t dir_world, double eps,
                                 double* kappa)
{
    int32_t* idx = (int32_t*)malloc(sizeof(int32_t) * (size_t)(M > 0 ? M : 1) * K);
    double* W = (double*)malloc(sizeof(double) * (size_t)(M > 0 ? M : 1) * K);
    double *dl, *mrgb, *mocc;
    query_setup(M, x, n, P, probe_pos, R, maps_rgb, maps_occ, S, dirs, dir_world, K, snap_key, r2_key, idx, W, &dl,
                &mrgb, &mocc);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t m = 0; m < M; ++m) {
        double nn[3], vo[3], a[3], t[3], b[3];
        point_frame(n, wo, albedo, m, nn, vo, a, t, b);
        double acc[6] = {0, 0, 0, 0, 0, 0}, dev[6] = {0, 0, 0, 0, 0, 0};
        for (int32_t i = 0; i < S; ++i) {
            double w[3], g0[6];
            const double wt = sample_dir(dl, dir_world, i, t, b, nn, w);
            if (wt == 0.0) continue;
            sample_terms(nn, vo, a, rough[m], metal[m], spec, mode, w, K, idx + (size_t)m * K, W + (size_t)m * K, R,
                         mrgb, mocc, env, He, We, env_layout, g0);
            for (int c = 0; c < 6; ++c) g0[c] *= wt;
            /* two unit axes normal to w */
            double u1[3] = {w[1] * nn[2] - w[2] * nn[1], w[2] * nn[0] - w[0] * nn[2], w[0] * nn[1] - w[1] * nn[0]};
            double ul = sqrt(u1[0] * u1[0] + u1[1] * u1[1] + u1[2] * u1[2]);
            if (ul < 1e-12) { u1[0] = t[0]; u1[1] = t[1]; u1[2] = t[2]; ul = 1.0; }
            for (int c = 0; c < 3; ++c) u1[c] /= ul;
            double u2[3] = {w[1] * u1[2] - w[2] * u1[1], w[2] * u1[0] - w[0] * u1[2], w[0] * u1[1] - w[1] * u1[0]};
            double mx[6] = {0, 0, 0, 0, 0, 0};
            for (int j = 0; j < 4; ++j) {
                const double* u = (j < 2) ? u1 : u2;
                double sg = (j & 1) ? -eps : eps, wp[3], g1[6];
                for (int c = 0; c < 3; ++c) wp[c] = w[c] + sg * u[c];
                double wl = sqrt(wp[0] * wp[0] + wp[1] * wp[1] + wp[2] * wp[2]);
                for (int c = 0; c < 3; ++c) wp[c] /= wl;
                sample_terms(nn, vo, a, rough[m], metal[m], spec, mode, wp, K, idx + (size_t)m * K, W + (size_t)m * K,
                             R, mrgb, mocc, env, He, We, env_layout, g1);
                for (int c = 0; c < 6; ++c) g1[c] *= wt;
                for (int c = 0; c < 6; ++c) {
                    double d = fabs(g1[c] - g0[c]);
                    if (d > mx[c]) mx[c] = d;
                }
            }
            for (int c = 0; c < 6; ++c) {
                acc[c] += g0[c];
                dev[c] += mx[c];
            }
        }
        for (int c = 0; c < 3; ++c) {
            if (mode == ORC_MODE_SHADE) kappa[3 * m + c] = (dir_world ? 1.0 : 2.0 * M_PI) / S * dev[c];
            else if (acc[3 + c] < 1e-20) kappa[3 * m + c] = 0.0;
            else kappa[3 * m + c] = (dev[c] + fabs(acc[c] / acc[3 + c]) * dev[3 + c]) / acc[3 + c];
        }
    }
    free(mocc);
    free(mrgb);
    free(dl);
    free(W);
    free(idx);
}

/* ------------------------------------------------------------------------ */
/* Adjoint of the SHADE output (Sec. 3.1.2: environment, materials and SOP   */
/* textures are the learnable quantities of the decomposition; Eq. 3-6).     */
/* ------------------------------------------------------------------------ */

/* d uv / d w of orc_oct_encode (uv = (p + 1)/2), 2x3 row-major. */
static void oct_encode_jac(const double* w, double* J)
{
    double ax = fabs(w[0]), ay = fabs(w[1]), az = fabs(w[2]);
    double l1 = ax + ay + az;
    double sx = sgn_nz(w[0]), sy = sgn_nz(w[1]), sz = w[2] >= 0.0 ? 1.0 : -1.0;
    double px = w[0] / l1, py = w[1] / l1;
    /* dp/dw for p = w.xy / |w|_1 */
    double dpx[3] = {(l1 - ax) / (l1 * l1), -w[0] * sy / (l1 * l1), -w[0] * sz / (l1 * l1)};
    double dpy[3] = {-w[1] * sx / (l1 * l1), (l1 - ay) / (l1 * l1), -w[1] * sz / (l1 * l1)};
    if (w[2] < 0.0) {
        /* q = ((1 - |py|) sgn px, (1 - |px|) sgn py) */
        double spx = sgn_nz(px), spy = sgn_nz(py);
        for (int c = 0; c < 3; ++c) {
            double qx = -spy * dpy[c] * spx, qy = -spx * dpx[c] * spy;
            J[c] = 0.5 * qx;
            J[3 + c] = 0.5 * qy;
        }
    } else {
        for (int c = 0; c < 3; ++c) {
            J[c] = 0.5 * dpx[c];
            J[3 + c] = 0.5 * dpy[c];
        }
    }
}

/* Bilinear read of a compact [R][R][C] map with its uv-gradient and the
 * four (source texel, weight) pairs the read used. */
static void bilerp_grad(const double* map, int R, int C, const double* uv, double* out, double* duv, int* texel,
                        double* wt)
{
    double s = uv[0] * R - 0.5, t = uv[1] * R - 0.5;
    double fi = floor(s), fj = floor(t);
    double fu = s - fi, fv = t - fj;
    int i0 = (int)fi, j0 = (int)fj;
    const double* tx[4];
    for (int q = 0; q < 4; ++q) {
        int di = q & 1, dj = q >> 1, si, sj;
        orc_oct_wrap(R, i0 + di, j0 + dj, &si, &sj);
        texel[q] = sj * R + si;
        tx[q] = map + (size_t)texel[q] * C;
        wt[q] = (di ? fu : 1.0 - fu) * (dj ? fv : 1.0 - fv);
    }
    for (int c = 0; c < C; ++c) {
        out[c] = wt[0] * tx[0][c] + wt[1] * tx[1][c] + wt[2] * tx[2][c] + wt[3] * tx[3][c];
        duv[2 * c] = R * ((1.0 - fv) * (tx[1][c] - tx[0][c]) + fv * (tx[3][c] - tx[2][c]));
        duv[2 * c + 1] = R * ((1.0 - fu) * (tx[2][c] - tx[0][c]) + fu * (tx[3][c] - tx[1][c]));
    }
}

/* Environment read with dL/dw (3x3, row = channel) and the four
 * (texel, weight) pairs. */
static void env_grad(const float* env, int32_t He, int32_t We, const double* w, double* L, double* dL, int* texel,
                     double* wt)
{
    double rho2 = w[0] * w[0] + w[1] * w[1], rho = sqrt(rho2);
    double theta = atan2(rho, w[2]), phi = atan2(w[1], w[0]);
    double u = (phi + M_PI) / (2.0 * M_PI), v = theta / M_PI;
    double s = u * We - 0.5, t = v * He - 0.5;
    double fs = floor(s), ft = floor(t);
    double a = s - fs, b = t - ft;
    int c0 = (int)fs, r0 = (int)ft;
    const float* e[4];
    for (int q = 0; q < 4; ++q) {
        int dc = q & 1, dr = q >> 1;
        int r = r0 + dr, c = c0 + dc;
        r = r < 0 ? 0 : (r > He - 1 ? He - 1 : r);
        c = ((c % We) + We) % We;
        texel[q] = r * We + c;
        e[q] = env + (size_t)texel[q] * 3;
        wt[q] = (dc ? a : 1.0 - a) * (dr ? b : 1.0 - b);
    }
    /* ds/dw and dt/dw */
    double ds[3] = {0, 0, 0}, dt[3] = {0, 0, 0};
    if (rho2 > 0.0) {
        double k = We / (2.0 * M_PI);
        ds[0] = -k * w[1] / rho2;
        ds[1] = k * w[0] / rho2;
        double r2 = rho2 + w[2] * w[2], kt = He / M_PI;
        /* dtheta/dx = z x / (rho r2), dtheta/dy = z y / (rho r2), dtheta/dz = -rho / r2 */
        dt[0] = kt * w[2] * w[0] / (rho * r2);
        dt[1] = kt * w[2] * w[1] / (rho * r2);
        dt[2] = -kt * rho / r2;
    }
    for (int c = 0; c < 3; ++c) {
        L[c] = wt[0] * e[0][c] + wt[1] * e[1][c] + wt[2] * e[2][c] + wt[3] * e[3][c];
        double dLs = (1.0 - b) * (e[1][c] - e[0][c]) + b * (e[3][c] - e[2][c]);
        double dLt = (1.0 - a) * (e[2][c] - e[0][c]) + a * (e[3][c] - e[1][c]);
        for (int j = 0; j < 3; ++j) dL[3 * c + j] = dLs * ds[j] + dLt * dt[j];
    }
}

/* Gradients of L = sum_m grad_out[m] . C[m] (SHADE mode) with respect to
 * albedo [M,3], roughness [M], metallic [M], the raw normal [M,3] (these
 * four overwrite), the environment texels [He,We,3] and the compact probe
 * maps [P,R,R,3] radiance and [P,R,R] occlusion (these three accumulate).
 * The chain follows the forward pass term by term; NdotL is l_z, which does
 * not move with the normal. */
void orc_query_shade_grad(int64_t M, const float* x, const float* n, const float* wo, const float* albedo,
                          const float* rough, const float* metal, int32_t P, const float* probe_pos, int32_t R,
                          const float* maps_rgb, const float* maps_occ, int32_t He, int32_t We, const float* env,
                          int32_t S, const double* dirs, int32_t K, double spec, uint64_t snap_key, uint64_t r2_key,
                          const double* grad_out, double* g_albedo, double* g_rough, double* g_metal,
                          double* g_normal, double* g_env, double* g_maps_rgb, double* g_maps_occ,
                          double* abs_albedo, double* abs_rough, double* abs_metal, double* abs_normal)
{
    int32_t* idx = (int32_t*)malloc(sizeof(int32_t) * (size_t)(M > 0 ? M : 1) * K);
    double* W = (double*)malloc(sizeof(double) * (size_t)(M > 0 ? M : 1) * K);
    uint64_t* key = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(M > 0 ? M : 1) * K);
    double *dl, *mrgb, *mocc;
    query_setup(M, x, n, P, probe_pos, R, maps_rgb, maps_occ, S, dirs, 0, K, snap_key, r2_key, idx, W, &dl, &mrgb,
                &mocc);
    orc_knn(M, x, P, probe_pos, K, r2_key, idx, key);
    size_t RR = (size_t)R * R;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t m = 0; m < M; ++m) {
        double nn[3], vo[3], a[3], t[3], b[3];
        point_frame(n, wo, albedo, m, nn, vo, a, t, b);
        const int32_t* id = idx + (size_t)m * K;
        const double* Wk = W + (size_t)m * K;
        double r = rough[m], mt = metal[m];
        double al = r * r, a2 = al * al, kk = (r + 1.0) * (r + 1.0) / 8.0;
        double NdotVraw = nn[0] * vo[0] + nn[1] * vo[1] + nn[2] * vo[2];
        int vclamp = NdotVraw < 1e-4;
        double NdotV = vclamp ? 1e-4 : NdotVraw;
        double G1V = NdotV / (NdotV * (1.0 - kk) + kk);
        double F0[3];
        for (int c = 0; c < 3; ++c) F0[c] = 0.08 * spec * (1.0 - mt) + a[c] * mt;
        double ga[3] = {0, 0, 0}, gr = 0, gm = 0, gn[3] = {0, 0, 0}, gW[32];
        /* sums of the magnitudes of the per-direction terms (the scale of the
         * rounding error of each gradient, which may cancel to near zero) */
        double sa[3] = {0, 0, 0}, sr = 0, sm = 0, sn = 0;
        for (int k = 0; k < K; ++k) gW[k] = 0.0;
        const double sc = 2.0 * M_PI / S;
        for (int32_t i = 0; i < S; ++i) {
            const double* l = dl + 3 * i;
            double w[3];
            for (int c = 0; c < 3; ++c) w[c] = l[0] * t[c] + l[1] * b[c] + l[2] * nn[c];
            double NdotL = l[2];
            /* probe terms */
            double uv[2];
            orc_oct_encode(w, uv);
            double O = 0, Lin[3] = {0, 0, 0}, dO_duv[2] = {0, 0}, dLin_duv[6] = {0, 0, 0, 0, 0, 0};
            double ok[32], lk[32][3], dok[32][2], dlk[32][6], wto[32][4];
            int txo[32][4];
            for (int k = 0; k < K; ++k) {
                if (id[k] < 0) continue; /* empty slot of a radius search */
                double wt[4];
                int tx[4];
                bilerp_grad(mocc + RR * id[k], R, 1, uv, &ok[k], dok[k], tx, wt);
                bilerp_grad(mrgb + 3 * RR * id[k], R, 3, uv, lk[k], dlk[k], txo[k], wto[k]);
                O += Wk[k] * ok[k];
                for (int c = 0; c < 3; ++c) Lin[c] += Wk[k] * lk[k][c];
                for (int j = 0; j < 2; ++j) dO_duv[j] += Wk[k] * dok[k][j];
                for (int c = 0; c < 6; ++c) dLin_duv[c] += Wk[k] * dlk[k][c];
            }
            double Ld[3], dLd[9], ewt[4];
            int etx[4];
            env_grad(env, He, We, w, Ld, dLd, etx, ewt);
            /* BRDF pieces */
            double hv[3] = {w[0] + vo[0], w[1] + vo[1], w[2] + vo[2]};
            double hl = sqrt(hv[0] * hv[0] + hv[1] * hv[1] + hv[2] * hv[2]);
            double h[3];
            for (int c = 0; c < 3; ++c) h[c] = hl < 1e-30 ? nn[c] : hv[c] / hl;
            double NdotH = nn[0] * h[0] + nn[1] * h[1] + nn[2] * h[2];
            double VdotH = vo[0] * h[0] + vo[1] * h[1] + vo[2] * h[2];
            double cx = nn[1] * h[2] - nn[2] * h[1], cy = nn[2] * h[0] - nn[0] * h[2], cz = nn[0] * h[1] - nn[1] * h[0];
            double sin2 = cx * cx + cy * cy + cz * cz;
            double den = NdotH * NdotH * a2 + sin2;
            double D = a2 / (M_PI * den * den);
            double gl = NdotL * (1.0 - kk) + kk;
            double G1L = NdotL / gl;
            double spec_t = D * G1L * G1V / (4.0 * NdotL * NdotV);
            double x1 = 1.0 - VdotH, fc = pow(x1, 5.0);
            double f[3], F[3], Lmix[3], gam[3];
            for (int c = 0; c < 3; ++c) {
                F[c] = F0[c] + (1.0 - F0[c]) * fc;
                f[c] = (1.0 - mt) * a[c] / M_PI + spec_t * F[c];
                Lmix[c] = (1.0 - O) * Ld[c] + Lin[c];
                gam[c] = sc * grad_out[3 * m + c] * NdotL;
            }
            /* materials */
            double dD_da2 = (den - 2.0 * a2 * NdotH * NdotH) / (M_PI * den * den * den);
            double dG1L_dk = -NdotL * (1.0 - NdotL) / (gl * gl);
            double gvv = NdotV * (1.0 - kk) + kk;
            double dG1V_dk = -NdotV * (1.0 - NdotV) / (gvv * gvv);
            double dspec_dr = (dD_da2 * 4.0 * r * r * r * G1L * G1V +
                               D * (dG1L_dk * G1V + G1L * dG1V_dk) * (r + 1.0) / 4.0) /
                              (4.0 * NdotL * NdotV);
            double GN = 0, GS = 0, GVH = 0, GNV = 0; /* dL/d(NdotH), d(sin2), d(VdotH), d(NdotV) */
            double gOt = 0, gLin[3], gLd[3];
            for (int c = 0; c < 3; ++c) {
                double u = gam[c] * Lmix[c];
                double ta = u * ((1.0 - mt) / M_PI + spec_t * (1.0 - fc) * mt);
                double tm = u * (-a[c] / M_PI + spec_t * (1.0 - fc) * (-0.08 * spec + a[c]));
                double tr = u * dspec_dr * F[c];
                ga[c] += ta;
                gm += tm;
                gr += tr;
                sa[c] += fabs(ta);
                sm += fabs(tm);
                sr += fabs(tr);
                double fsp = F[c] * G1L * G1V / (4.0 * NdotL * NdotV);
                GN += u * fsp * (-4.0 * a2 * a2 * NdotH / (M_PI * den * den * den));
                GS += u * fsp * (-2.0 * a2 / (M_PI * den * den * den));
                GVH += u * spec_t * (1.0 - F0[c]) * (-5.0 * x1 * x1 * x1 * x1);
                if (!vclamp) {
                    double gv = NdotV * (1.0 - kk) + kk;
                    GNV += u * F[c] * D * G1L / (4.0 * NdotL) * (-(1.0 - kk) / (gv * gv));
                }
                gOt += -gam[c] * f[c] * Ld[c];
                gLin[c] = gam[c] * f[c];
                gLd[c] = gam[c] * f[c] * (1.0 - O);
            }
            /* texel scatter and weight gradients */
            for (int k = 0; k < K; ++k) {
                if (id[k] < 0) continue;
                gW[k] += gOt * ok[k] + gLin[0] * lk[k][0] + gLin[1] * lk[k][1] + gLin[2] * lk[k][2];
                for (int q = 0; q < 4; ++q) {
                    size_t tix = RR * id[k] + txo[k][q];
                    double wq = Wk[k] * wto[k][q];
#pragma omp atomic
                    g_maps_occ[tix] += gOt * wq;
                    for (int c = 0; c < 3; ++c) {
#pragma omp atomic
                        g_maps_rgb[3 * tix + c] += gLin[c] * wq;
                    }
                }
            }
            for (int q = 0; q < 4; ++q)
                for (int c = 0; c < 3; ++c) {
#pragma omp atomic
                    g_env[3 * (size_t)etx[q] + c] += gLd[c] * ewt[q];
                }
            /* d/dw */
            double gw[3] = {0, 0, 0}, guv[2];
            guv[0] = gOt * dO_duv[0] + gLin[0] * dLin_duv[0] + gLin[1] * dLin_duv[2] + gLin[2] * dLin_duv[4];
            guv[1] = gOt * dO_duv[1] + gLin[0] * dLin_duv[1] + gLin[1] * dLin_duv[3] + gLin[2] * dLin_duv[5];
            double J[6];
            oct_encode_jac(w, J);
            for (int j = 0; j < 3; ++j) gw[j] += guv[0] * J[j] + guv[1] * J[3 + j];
            for (int c = 0; c < 3; ++c)
                for (int j = 0; j < 3; ++j) gw[j] += gLd[c] * dLd[3 * c + j];
            /* BRDF geometry: through h (and directly through n) */
            double gh[3], gnd[3];
            for (int j = 0; j < 3; ++j) {
                gh[j] = GN * nn[j] + GS * 2.0 * (h[j] - NdotH * nn[j]) + GVH * vo[j];
                gnd[j] = GN * h[j] + GS * 2.0 * (nn[j] - NdotH * h[j]) + GNV * vo[j];
            }
            if (hl >= 1e-30) {
                double hg = h[0] * gh[0] + h[1] * gh[1] + h[2] * gh[2];
                for (int j = 0; j < 3; ++j) gw[j] += (gh[j] - hg * h[j]) / hl;
            }
            /* w = l.x t(n) + l.y b(n) + l.z n */
            double sg = nn[2] >= 0.0 ? 1.0 : -1.0, aa = -1.0 / (sg + nn[2]), a2n = aa * aa;
            double dt[3][3] = {{2.0 * sg * nn[0] * aa, 0.0, sg * nn[0] * nn[0] * a2n},
                               {sg * nn[1] * aa, sg * nn[0] * aa, sg * nn[0] * nn[1] * a2n},
                               {-sg, 0.0, 0.0}};
            double db[3][3] = {{nn[1] * aa, nn[0] * aa, nn[0] * nn[1] * a2n},
                               {0.0, 2.0 * nn[1] * aa, nn[1] * nn[1] * a2n},
                               {0.0, -1.0, 0.0}};
            double vn[3];
            for (int j = 0; j < 3; ++j) {
                double v = l[2] * gw[j] + gnd[j];
                for (int c = 0; c < 3; ++c) v += l[0] * gw[c] * dt[c][j] + l[1] * gw[c] * db[c][j];
                gn[j] += v;
                vn[j] = v;
            }
            sn += sqrt(vn[0] * vn[0] + vn[1] * vn[1] + vn[2] * vn[2]);
        }
        /* blend weights W_k = w_s w_b / sum (Eq. 4-6): w_b moves with n */
        if (id[0] >= 0 && key[(size_t)m * K] > snap_key) {
            double u[32], U = 0, ws[32], dh[32][3];
            for (int k = 0; k < K; ++k) {
                u[k] = ws[k] = 0.0;
                for (int j = 0; j < 3; ++j) dh[k][j] = 0.0;
                if (id[k] < 0) continue;
                const float* p = probe_pos + 3 * (size_t)id[k];
                double d[3] = {(double)p[0] - x[3 * m], (double)p[1] - x[3 * m + 1], (double)p[2] - x[3 * m + 2]};
                double dlen = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                ws[k] = 1.0 / dlen;
                for (int j = 0; j < 3; ++j) dh[k][j] = d[j] / dlen;
                u[k] = ws[k] * (0.5 * (1.0 + dh[k][0] * nn[0] + dh[k][1] * nn[1] + dh[k][2] * nn[2]) + 0.01);
                U += u[k];
            }
            double gu_dot = 0;
            for (int k = 0; k < K; ++k) gu_dot += gW[k] * Wk[k];
            for (int j = 0; j < K; ++j) {
                double gu = (gW[j] - gu_dot) / U; /* dL/du_j */
                for (int c = 0; c < 3; ++c) gn[c] += gu * ws[j] * 0.5 * dh[j][c];
                sn += fabs(gu * ws[j] * 0.5);
            }
        }
        /* through the normalisation n = n_raw / |n_raw| */
        double nr[3] = {n[3 * m], n[3 * m + 1], n[3 * m + 2]};
        double nl = sqrt(nr[0] * nr[0] + nr[1] * nr[1] + nr[2] * nr[2]);
        double ng = gn[0] * nn[0] + gn[1] * nn[1] + gn[2] * nn[2];
        for (int c = 0; c < 3; ++c) {
            g_normal[3 * m + c] = (gn[c] - ng * nn[c]) / nl;
            g_albedo[3 * m + c] = ga[c];
        }
        g_rough[m] = gr;
        g_metal[m] = gm;
        if (abs_albedo) {
            for (int c = 0; c < 3; ++c) abs_albedo[3 * m + c] = sa[c];
            abs_rough[m] = sr;
            abs_metal[m] = sm;
            abs_normal[m] = sn / nl;
        }
    }
    free(mocc);
    free(mrgb);
    free(dl);
    free(key);
    free(W);
    free(idx);
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Batched entry points for the tests (loops over the single-item routines).  */
/* ------------------------------------------------------------------------ */
void orc_oct_encode_n(int64_t n, const double* d, double* uv)
{
    for (int64_t i = 0; i < n; ++i) orc_oct_encode(d + 3 * i, uv + 2 * i);
}

void orc_oct_decode_n(int64_t n, const double* uv, double* d, int l1_only)
{
    for (int64_t i = 0; i < n; ++i) {
        if (l1_only) orc_oct_decode_l1(uv + 2 * i, d + 3 * i);
        else orc_oct_decode(uv + 2 * i, d + 3 * i);
    }
}

void orc_oct_bilerp_n(int64_t n, const double* map, int R, int C, const double* uv, double* out)
{
    for (int64_t i = 0; i < n; ++i) orc_oct_bilerp(map, R, C, uv + 2 * i, out + (size_t)C * i);
}

void orc_env_lookup_n(int64_t n, const float* env, int32_t He, int32_t We, const double* w, double* out)
{
    for (int64_t i = 0; i < n; ++i) orc_env_lookup(env, He, We, w + 3 * i, out + 3 * i);
}

void orc_env_oct_lookup_n(int64_t n, const float* env, int32_t H, const double* w, double* out)
{
    for (int64_t i = 0; i < n; ++i) orc_env_oct_lookup(env, H, w + 3 * i, out + 3 * i);
}

void orc_brdf_n(int64_t n, const double* nrm, const double* wo, const double* wi, const double* albedo,
                const double* rough, const double* metal, double spec, double* f)
{
    for (int64_t i = 0; i < n; ++i)
        orc_brdf(nrm + 3 * i, wo + 3 * i, wi + 3 * i, albedo + 3 * i, rough[i], metal[i], spec, f + 3 * i);
}

void orc_onb_n(int64_t n, const double* nrm, double* t, double* b)
{
    for (int64_t i = 0; i < n; ++i) orc_onb(nrm + 3 * i, t + 3 * i, b + 3 * i);
}
