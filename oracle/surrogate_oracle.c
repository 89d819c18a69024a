/*
 * FP64 oracle of the learned bake surrogate's texel features (test
 * infrastructure only; shares no code with the CUDA library).
 *
 * The paper has no surrogate: it initialises SOPs by ray tracing
 * (Sec. 3.1.2) and caches occlusion (Sec. 3.2.2). The surrogate predicts a
 * probe texel's maps from features that describe the probe's neighbourhood
 * along that texel's ray:
 *   near field: the probe's nearest Gaussians (at most KN, centres within
 *     r_n, nearest first by the integer squared distance of positions
 *     quantised to 2^-20, ties to the lower index; orc_knn computes the
 *     list), composited along the texel ray in list order with the bake's
 *     ray-Gaussian response (maximum along the ray, alpha = min(alpha_max,
 *     o exp(-m^2/2)), kept when t* > 0 and alpha >= alpha_min):
 *     O_n = 1 - prod(1 - alpha), L_n = sum T alpha rgb, W_n = sum T alpha,
 *     D_n = sum T alpha t* / W_n (0 when W_n <= 1e-8);
 *   far field: a coarse extinction field. Each Gaussian with opacity >=
 *     alpha_min carries the optical mass -ln(1 - min(o, alpha_max)) 2 pi
 *     s_2 s_3 (s_2, s_3 its two largest scales: the area of its footprint
 *     seen face on), deposited into the cubic cell holding its quantised
 *     centre, as fixed-point sums (units of 2^-40). The grid spans the
 *     bounding box of the quantised centres with G cells along its longest
 *     axis (edge hq quanta = ceil(extent / G)). Along the texel ray from t0
 *     (the distance of the list's last Gaussian when the list is full, else
 *     r_n), the walk through the cells accumulates tau += sigma dt
 *     (sigma = mass / h^3), and the colour
 *     L_f += exp(-tau) (1 - exp(-sigma dt)) rgb_cell (the mass-weighted mean
 *     colour), stopping once tau > 20. The features are 1 - exp(-tau) at
 *     t0 + h {2, 4, 8, 16, 32} and at the end, and L_f.
 * Everything here is plain FP64 except the fixed-point mass sums.
 */
#define _GNU_SOURCE
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

void orc_texel_dir(int R, int i, int j, double* d);

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif
static const double kQ = 1048576.0; /* 2^20 */
static const double kFix = 1099511627776.0; /* 2^40 */
static const double kEps32 = 5.9604644775390625e-08; /* 2^-24, the FP32 unit roundoff */

static int64_t quant(float v) { return (int64_t)nearbyint((double)v * kQ); }

static void rot_of(const float* q4, double Rm[3][3])
{
    double w = q4[0], x = q4[1], y = q4[2], z = q4[3];
    const double n = sqrt(w * w + x * x + y * y + z * z);
    w /= n; x /= n; y /= n; z /= n;
    Rm[0][0] = 1 - 2 * (y * y + z * z); Rm[0][1] = 2 * (x * y - w * z);     Rm[0][2] = 2 * (x * z + w * y);
    Rm[1][0] = 2 * (x * y + w * z);     Rm[1][1] = 1 - 2 * (x * x + z * z); Rm[1][2] = 2 * (y * z - w * x);
    Rm[2][0] = 2 * (x * z - w * y);     Rm[2][1] = 2 * (y * z + w * x);     Rm[2][2] = 1 - 2 * (x * x + y * y);
}

/* Near field of every texel of P probes. list [P][KN] holds Gaussian
 * indices (-1 ends a short list). out [P][R*R][6] = (O_n, L_n rgb, D_n,
 * W_n); flags [P][R*R]: 1 when a response lies within 1e-4 relative of
 * alpha_min or a t* within 1e-6 of 0 (a decision that FP32 may take the
 * other way). */
void orc_surr_near(int32_t P, const float* probe_pos, int32_t R, const float* mean, const float* scale,
                   const float* quat, const float* opacity, const float* rgb, const int32_t* list, int32_t KN,
                   double alpha_min, double alpha_max, double* out, int32_t* flags)
{
    const int RR = R * R;
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t p = 0; p < P; ++p) {
        const float* pp = probe_pos + 3 * (size_t)p;
        for (int t = 0; t < RR; ++t) {
            double d[3];
            orc_texel_dir(R, t % R, t / R, d);
            double T = 1.0, L[3] = {0, 0, 0}, W = 0.0, Dacc = 0.0;
            int fl = 0;
            for (int32_t k = 0; k < KN; ++k) {
                const int32_t g = list[(size_t)p * KN + k];
                if (g < 0) break;
                double Rm[3][3];
                rot_of(quat + 4 * (size_t)g, Rm);
                double u[3], w[3];
                const double del[3] = {(double)pp[0] - mean[3 * (size_t)g], (double)pp[1] - mean[3 * (size_t)g + 1],
                                       (double)pp[2] - mean[3 * (size_t)g + 2]};
                for (int a = 0; a < 3; ++a) {
                    /* row a of diag(1/s) R^T: column a of R over s_a */
                    const double s = scale[3 * (size_t)g + a];
                    u[a] = (Rm[0][a] * del[0] + Rm[1][a] * del[1] + Rm[2][a] * del[2]) / s;
                    w[a] = (Rm[0][a] * d[0] + Rm[1][a] * d[1] + Rm[2][a] * d[2]) / s;
                }
                const double A = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
                const double B = w[0] * u[0] + w[1] * u[1] + w[2] * u[2];
                const double ts = -B / A;
                double m2 = 0.0;
                for (int a = 0; a < 3; ++a) {
                    const double e = u[a] + ts * w[a];
                    m2 += e * e;
                }
                const double resp = opacity[g] * exp(-0.5 * m2);
                if (fabs(resp - alpha_min) <= 1e-4 * alpha_min && ts > 0.0) fl = 1;
                if (resp >= alpha_min && fabs(ts) <= 1e-6) fl = 1;
                if (!(ts > 0.0) || resp < alpha_min) continue;
                const double al = resp < alpha_max ? resp : alpha_max;
                const double wk = T * al;
                for (int c = 0; c < 3; ++c) L[c] += wk * rgb[3 * (size_t)g + c];
                W += wk;
                Dacc += wk * ts;
                T *= 1.0 - al;
            }
            double* o = out + ((size_t)p * RR + t) * 6;
            o[0] = 1.0 - T;
            o[1] = L[0];
            o[2] = L[1];
            o[3] = L[2];
            o[4] = W > 1e-8 ? Dacc / W : 0.0;
            o[5] = W;
            flags[(size_t)p * RR + t] = fl;
        }
    }
}

/* Geometry of the far-field grid: qlo [3] (quantised lower corner), hq
 * (cell edge in quanta) and dims [3], from the quantised centres of the
 * Gaussians that carry mass. Returns the number of cells (0: no mass). */
int64_t orc_surr_grid_dims(int64_t N, const float* mean, const float* opacity, double alpha_min, int32_t G,
                           int64_t* qlo, int64_t* hq, int32_t* dims)
{
    int64_t lo[3] = {INT64_MAX, INT64_MAX, INT64_MAX}, hi[3] = {INT64_MIN, INT64_MIN, INT64_MIN};
    int64_t n = 0;
    for (int64_t g = 0; g < N; ++g) {
        if (!(opacity[g] >= alpha_min)) continue;
        ++n;
        for (int a = 0; a < 3; ++a) {
            const int64_t q = quant(mean[3 * g + a]);
            if (q < lo[a]) lo[a] = q;
            if (q > hi[a]) hi[a] = q;
        }
    }
    if (n == 0) {
        qlo[0] = qlo[1] = qlo[2] = 0;
        *hq = 1;
        dims[0] = dims[1] = dims[2] = 1;
        return 0;
    }
    int64_t ext = 0;
    for (int a = 0; a < 3; ++a)
        if (hi[a] - lo[a] + 1 > ext) ext = hi[a] - lo[a] + 1;
    const int64_t h = (ext + G - 1) / G;
    int64_t cells = 1;
    for (int a = 0; a < 3; ++a) {
        qlo[a] = lo[a];
        dims[a] = (int32_t)((hi[a] - lo[a]) / h + 1);
        cells *= dims[a];
    }
    *hq = h;
    return cells;
}

/* Fixed-point optical mass and mass x rgb per cell (arrays of the size
 * orc_surr_grid_dims returned, zeroed here). */
void orc_surr_grid_fill(int64_t N, const float* mean, const float* scale, const float* opacity, const float* rgb,
                        double alpha_min, double alpha_max, const int64_t* qlo, int64_t hq, const int32_t* dims,
                        int64_t* mass_q, int64_t* col_q)
{
    const int64_t cells = (int64_t)dims[0] * dims[1] * dims[2];
    memset(mass_q, 0, sizeof(int64_t) * (size_t)cells);
    memset(col_q, 0, sizeof(int64_t) * 3 * (size_t)cells);
    for (int64_t g = 0; g < N; ++g) {
        const double o = opacity[g];
        if (!(o >= alpha_min)) continue;
        double s[3] = {scale[3 * g], scale[3 * g + 1], scale[3 * g + 2]};
        /* the two largest scales */
        double smin = s[0];
        if (s[1] < smin) smin = s[1];
        if (s[2] < smin) smin = s[2];
        const double prod2 = s[0] * s[1] * s[2] / smin;
        const double mass = -log1p(-(o < alpha_max ? o : alpha_max)) * 2.0 * M_PI * prod2;
        int64_t c[3];
        for (int a = 0; a < 3; ++a) c[a] = (quant(mean[3 * g + a]) - qlo[a]) / hq;
        const int64_t cell = (c[2] * dims[1] + c[1]) * dims[0] + c[0];
        mass_q[cell] += (int64_t)llrint(mass * kFix);
        for (int k = 0; k < 3; ++k) col_q[3 * cell + k] += (int64_t)llrint(mass * rgb[3 * g + k] * kFix);
    }
}

/* Far field of every texel of P probes, from t0[p] on. out [P][R*R][9] =
 * (1 - exp(-tau) at t0 + h {2, 4, 8, 16, 32} and at the end, L_f rgb).
 * sens [P][R*R] (may be NULL): the march's conditioning, for tests of an
 * FP32 march. A boundary time (B - o_a) / d_a taken in FP32 (B the cell
 * plane's coordinate) is off by about 2^-24 (|B| + |o_a|) / |d_a| + 2^-24 |t|,
 * and a segment [t, te] of a cell of extinction sigma moves tau by sigma
 * times the errors of its two ends: sens = sum of sigma (e(t) + e(te)) over
 * the segments, with e = 2^-24 ((|B| + |o_a|) / |d_a| + 2 |t|). A short
 * segment clipped off a dense cell's corner is the case it covers: tau is
 * sigma times a small difference of two large times. */
void orc_surr_far(int32_t P, const float* probe_pos, const double* t0, int32_t R, const int64_t* qlo, int64_t hq,
                  const int32_t* dims, const int64_t* mass_q, const int64_t* col_q, double* out, double* sens)
{
    static const double mult[5] = {2, 4, 8, 16, 32};
    const int RR = R * R;
    const double h = (double)hq / kQ, h3 = h * h * h;
    double lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
        lo[a] = (double)qlo[a] / kQ;
        hi[a] = lo[a] + dims[a] * h;
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t p = 0; p < P; ++p) {
        const double o[3] = {probe_pos[3 * (size_t)p], probe_pos[3 * (size_t)p + 1], probe_pos[3 * (size_t)p + 2]};
        for (int t = 0; t < RR; ++t) {
            double d[3];
            orc_texel_dir(R, t % R, t / R, d);
            double ck[5];
            for (int k = 0; k < 5; ++k) ck[k] = t0[p] + mult[k] * h;
            double tau_ck[6];
            int next = 0;
            double tau = 0.0, L[3] = {0, 0, 0};
            /* the part of the ray inside the grid box, from t0 on */
            double ta = t0[p], tb = INFINITY;
            double pm_in = 0.0, pm_out = 0.0, s_out = 0.0; /* conditioning (entry, exit planes; total) */
            for (int a = 0; a < 3; ++a) {
                if (d[a] != 0.0) {
                    double t1 = (lo[a] - o[a]) / d[a], t2 = (hi[a] - o[a]) / d[a];
                    double B1 = lo[a], B2 = hi[a];
                    if (t1 > t2) {
                        const double tmp = t1;
                        t1 = t2;
                        t2 = tmp;
                        B1 = hi[a];
                        B2 = lo[a];
                    }
                    if (t1 > ta) {
                        ta = t1;
                        pm_in = (fabs(B1) + fabs(o[a])) / fabs(d[a]);
                    }
                    if (t2 < tb) {
                        tb = t2;
                        pm_out = (fabs(B2) + fabs(o[a])) / fabs(d[a]);
                    }
                } else if (o[a] < lo[a] || o[a] >= hi[a]) {
                    tb = -INFINITY;
                }
            }
            if (ta < tb) {
                int c[3], st[3];
                double tnext[3], pm[3];
                for (int a = 0; a < 3; ++a) {
                    int ci = (int)floor((o[a] + ta * d[a] - lo[a]) / h);
                    c[a] = ci < 0 ? 0 : (ci >= dims[a] ? dims[a] - 1 : ci);
                    st[a] = d[a] > 0.0 ? 1 : (d[a] < 0.0 ? -1 : 0);
                    const double B = lo[a] + (c[a] + (st[a] > 0)) * h;
                    tnext[a] = st[a] == 0 ? INFINITY : (B - o[a]) / d[a];
                    pm[a] = st[a] == 0 ? 0.0 : (fabs(B) + fabs(o[a])) / fabs(d[a]);
                }
                /* conditioning: the rounding scale of the segment's start
                 * (the walk's start: the box's entry plane, or t0) */
                double e_start = kEps32 * (pm_in + 2.0 * fabs(ta)), s_acc = 0.0;
                double t = ta;
                while (t < tb && tau <= 20.0) {
                    int ax = 0;
                    if (tnext[1] < tnext[ax]) ax = 1;
                    if (tnext[2] < tnext[ax]) ax = 2;
                    double te = tnext[ax] < tb ? tnext[ax] : tb;
                    if (te < t) te = t;
                    const double e_end = kEps32 * ((tnext[ax] < tb ? pm[ax] : pm_out) + 2.0 * fabs(te));
                    const int64_t cell = ((int64_t)c[2] * dims[1] + c[1]) * dims[0] + c[0];
                    const double m = (double)mass_q[cell] / kFix;
                    const double sig = m / h3;
                    while (next < 5 && ck[next] < te) {
                        tau_ck[next] = ck[next] <= t ? tau : tau + sig * (ck[next] - t);
                        ++next;
                    }
                    s_acc += sig * (e_start + e_end);
                    e_start = e_end;
                    if (m > 0.0) {
                        const double dtau = sig * (te - t);
                        const double a = exp(-tau) * (1.0 - exp(-dtau));
                        for (int k = 0; k < 3; ++k) L[k] += a * ((double)col_q[3 * cell + k] / kFix) / m;
                        tau += dtau;
                    }
                    t = te;
                    if (!(te < tb)) break;
                    c[ax] += st[ax];
                    if (c[ax] < 0 || c[ax] >= dims[ax]) break;
                    const double B = lo[ax] + (c[ax] + (st[ax] > 0)) * h;
                    tnext[ax] = (B - o[ax]) / d[ax];
                    pm[ax] = (fabs(B) + fabs(o[ax])) / fabs(d[ax]);
                }
                s_out = s_acc;
            }
            if (sens) sens[(size_t)p * RR + t] = s_out;
            while (next < 5) tau_ck[next++] = tau;
            tau_ck[5] = tau;
            double* out_t = out + ((size_t)p * RR + t) * 9;
            for (int k = 0; k < 6; ++k) out_t[k] = 1.0 - exp(-tau_ck[k]);
            out_t[6] = L[0];
            out_t[7] = L[1];
            out_t[8] = L[2];
        }
    }
}
