/* FP64 CPU oracle of the deferred front end (test infrastructure only: the
 * tests, the smoke check and the benchmark's CPU-baseline leg use it; the
 * CUDA library never does).
 *
 *   orc_trace_gbuffer    multi-target rendering of Gaussians along general
 *                        rays (Sec. 3.1, the alpha blending of G-buffers:
 *                        B = sum_i T_i alpha_i b_i, b_i = {c, 1, d, n, a, r, m},
 *                        T_i = prod_{j<i} (1 - alpha_j)), brute force over
 *                        every Gaussian, hits ordered by (t*, index)
 *   orc_pinhole_dirs     per-pixel ray directions of a pinhole camera
 *   orc_panorama_dirs    per-pixel directions of an equirectangular panorama
 *                        (the 360 degree sweep of Sec. 4.2)
 *   orc_gbuffer_points   shading points of a G-buffer: position from the
 *                        unbiased depth D / W (Sec. 3.1), normal N / |N|,
 *                        materials per unit weight (Sec. 4.3)
 *   orc_fps              automatic placement of SOPs (Sec. 3.2): farthest
 *                        point sampling with exact integer keys, offset
 *                        along the normals
 *   orc_depth_composite  the composed frame: the scene colour times its
 *                        shadow ratio (Eq. 9), the relit object over it where
 *                        it is in front (Sec. 4.3, depth compositing)
 *
 * Readings where the paper is silent (its primitives are 2D surfels; these
 * are the 3D Gaussians of the bake):
 *   - the evaluation of a Gaussian along a ray is the bake's: the point of
 *     maximum density t* = -B/A, alpha = min(alpha_max, o exp(-m^2/2)),
 *     kept when alpha >= alpha_min and t* > t_near; d_i = t* (distance
 *     along the unit ray direction, so that x = o + (D/W) d);
 *   - the normal n_i is the Gaussian's local axis of smallest scale (the
 *     first of equal ones), turned to face the ray: n.d <= 0;
 *   - a pixel becomes a shading point when W >= w_min and N != 0; its
 *     materials are A/W, R/W, M/W;
 *   - the composed colour of a pixel is W_o C_o + (1 - W_o) S C_s where the
 *     object's shading point lies in front of the scene's (or the scene has
 *     none), else S C_s; S = 1 where the scene has no shading point. */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef struct {
    double t, alpha;
    int64_t idx;
} gb_hit;

static int gb_hit_cmp(const void* a, const void* b)
{
    const gb_hit* x = (const gb_hit*)a;
    const gb_hit* y = (const gb_hit*)b;
    if (x->t < y->t) return -1;
    if (x->t > y->t) return 1;
    return (x->idx < y->idx) ? -1 : (x->idx > y->idx);
}

/* rotation of the unit quaternion (w, x, y, z): column a = local axis a */
static void gb_rot(const float* q4, double Rm[3][3])
{
    double w = q4[0], x = q4[1], y = q4[2], z = q4[3];
    double n = sqrt(w * w + x * x + y * y + z * z);
    w /= n; x /= n; y /= n; z /= n;
    Rm[0][0] = 1 - 2 * (y * y + z * z); Rm[0][1] = 2 * (x * y - w * z);     Rm[0][2] = 2 * (x * z + w * y);
    Rm[1][0] = 2 * (x * y + w * z);     Rm[1][1] = 1 - 2 * (x * x + z * z); Rm[1][2] = 2 * (y * z - w * x);
    Rm[2][0] = 2 * (x * z - w * y);     Rm[2][1] = 2 * (y * z + w * x);     Rm[2][2] = 1 - 2 * (x * x + y * y);
}

/* flags, as the bake oracle's, plus one for the normal's turn */
enum {
    GB_FLAG_ALPHA_MIN = 1, /* a response within 1e-4 relative of alpha_min         */
    GB_FLAG_ORDER = 2,     /* two kept hits whose t* differ by <= 1e-6 relative     */
    GB_FLAG_TNEAR = 4,     /* a t* within rounding of t_near                        */
    GB_FLAG_TSTOP = 8,     /* transmittance within 1e-3 relative of T_stop          */
    GB_FLAG_GRAZING = 16,  /* a composited normal within 1e-4 of perpendicular to d */
};

/* n_rays rays given by id: origin id / n_dirs, direction id % n_dirs (the
 * float32 table dirs [n_dirs][4], used as given). Output per ray, 16 values:
 * C.rgb, W, N.xyz, D, A.rgb, R, M, 0, 0, 0. out_tie (or NULL), per ray and
 * value: how far any order of hits whose t* tie within 1e-6 relative (runs
 * of consecutive hits closer than that) can move the value: swapping two
 * adjacent hits i, j behind transmittance T changes B by
 * T alpha_i alpha_j (b_i - b_j), so a run starting behind T_run gets
 * 2 T_run sum over its pairs of alpha_i alpha_j |b_i - b_j|. */
void orc_trace_gbuffer(int64_t N, const float* mean, const float* scale, const float* quat, const float* opacity,
                       const float* rgb, const float* albedo, const float* rough, const float* metal,
                       const float* origins, int64_t n_dirs, const float* dirs, int64_t n_rays, const int64_t* rays,
                       double t_near, double alpha_min, double alpha_max, double t_stop, double* out,
                       int32_t* out_flags, double* out_tie)
{
    double* Mg = (double*)malloc(sizeof(double) * 9 * (size_t)(N > 0 ? N : 1));
    double* Ng = (double*)malloc(sizeof(double) * 3 * (size_t)(N > 0 ? N : 1));
    for (int64_t g = 0; g < N; ++g) {
        double Rm[3][3];
        gb_rot(quat + 4 * g, Rm);
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) Mg[9 * g + 3 * a + b] = Rm[b][a] / (double)scale[3 * g + a];
        const float* s = scale + 3 * g;
        int am = 0;
        if (s[1] < s[am]) am = 1;
        if (s[2] < s[am]) am = 2;
        for (int b = 0; b < 3; ++b) Ng[3 * g + b] = Rm[b][am];
    }
#pragma omp parallel
    {
        size_t cap = 1024;
        gb_hit* hits = (gb_hit*)malloc(sizeof(gb_hit) * cap);
        double* pay = (double*)malloc(sizeof(double) * 16 * cap); /* b_i of the composited hits */
        double* tb = (double*)malloc(sizeof(double) * cap);       /* transmittance before hit i */
#pragma omp for schedule(dynamic, 4)
        for (int64_t r = 0; r < n_rays; ++r) {
            const int64_t id = rays[r];
            const float* p = origins + 3 * (size_t)(id / n_dirs);
            const float* dv = dirs + 4 * (size_t)(id % n_dirs);
            const double d[3] = {dv[0], dv[1], dv[2]};
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
                if (fabs(resp - alpha_min) <= 1e-4 * alpha_min && ts > t_near) flags |= GB_FLAG_ALPHA_MIN;
                if (resp >= alpha_min && fabs(ts - t_near) <= 1e-5 * (dl + 1e-3)) flags |= GB_FLAG_TNEAR;
                if (ts <= t_near || resp < alpha_min) continue;
                if (nh == cap) {
                    cap *= 2;
                    hits = (gb_hit*)realloc(hits, sizeof(gb_hit) * cap);
                    pay = (double*)realloc(pay, sizeof(double) * 16 * cap);
                    tb = (double*)realloc(tb, sizeof(double) * cap);
                }
                hits[nh].t = ts;
                hits[nh].alpha = resp < alpha_max ? resp : alpha_max;
                hits[nh].idx = g;
                ++nh;
            }
            qsort(hits, nh, sizeof(gb_hit), gb_hit_cmp);
            double T = 1.0, B[16];
            memset(B, 0, sizeof(B));
            size_t used = 0;
            for (size_t k = 0; k < nh; ++k) {
                if (k + 1 < nh && hits[k + 1].t - hits[k].t <= 1e-6 * fabs(hits[k + 1].t)) flags |= GB_FLAG_ORDER;
                const int64_t g = hits[k].idx;
                const double wk = T * hits[k].alpha;
                const double* ng = Ng + 3 * g;
                const double nd = ng[0] * d[0] + ng[1] * d[1] + ng[2] * d[2];
                if (fabs(nd) < 1e-4) flags |= GB_FLAG_GRAZING;
                const double sg = nd > 0.0 ? -1.0 : 1.0;
                double* b = pay + 16 * k;
                memset(b, 0, 16 * sizeof(double));
                for (int c = 0; c < 3; ++c) {
                    b[c] = rgb[3 * g + c];
                    b[4 + c] = sg * ng[c];
                    b[8 + c] = albedo[3 * g + c];
                }
                b[3] = 1.0;
                b[7] = hits[k].t;
                b[11] = rough[g];
                b[12] = metal[g];
                for (int c = 0; c < 16; ++c) B[c] += wk * b[c];
                tb[k] = T;
                used = k + 1;
                T *= (1.0 - hits[k].alpha);
                if (t_stop > 0.0 && fabs(T - t_stop) <= 1e-3 * t_stop) flags |= GB_FLAG_TSTOP;
                if (T < t_stop) break;
            }
            memcpy(out + 16 * (size_t)r, B, sizeof(B));
            out_flags[r] = flags;
            if (out_tie) {
                double* a = out_tie + 16 * (size_t)r;
                memset(a, 0, 16 * sizeof(double));
                size_t s0 = 0;
                while (s0 < used) {
                    size_t s1 = s0 + 1; /* the run is [s0, s1) */
                    while (s1 < nh && hits[s1].t - hits[s1 - 1].t <= 1e-6 * fabs(hits[s1].t)) ++s1;
                    if (s1 > used) s1 = used;
                    for (size_t i = s0; i < s1; ++i)
                        for (size_t j = i + 1; j < s1; ++j) {
                            const double aa = 2.0 * tb[s0] * hits[i].alpha * hits[j].alpha;
                            for (int c = 0; c < 16; ++c) a[c] += aa * fabs(pay[16 * i + c] - pay[16 * j + c]);
                        }
                    s0 = s1 > s0 + 1 ? s1 : s0 + 1;
                }
            }
        }
        free(tb);
        free(pay);
        free(hits);
    }
    free(Ng);
    free(Mg);
}

/* Pinhole camera at eye looking at target, vertical field of view fov_y
 * (degrees), W x H pixels, row 0 at the top: the ray of pixel (i, j) points
 * along f + sx r + sy u with sx = ((i + 1/2)/W 2 - 1) tan(fov/2) W/H,
 * sy = (1 - (j + 1/2)/H 2) tan(fov/2), f the unit forward direction,
 * r = f x up / |f x up|, u = r x f (up = y when f is within 0.99 of it).
 * out [H*W][3], unit, row-major. */
void orc_pinhole_dirs(int32_t W, int32_t H, const double* eye, const double* target, const double* up,
                      double fov_y_deg, double* out)
{
    double f[3] = {target[0] - eye[0], target[1] - eye[1], target[2] - eye[2]};
    double fl = sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
    for (int c = 0; c < 3; ++c) f[c] /= fl;
    double uu[3] = {up[0], up[1], up[2]};
    double ul = sqrt(uu[0] * uu[0] + uu[1] * uu[1] + uu[2] * uu[2]);
    if (fabs((f[0] * uu[0] + f[1] * uu[1] + f[2] * uu[2]) / ul) > 0.99) {
        uu[0] = 0.0; uu[1] = 1.0; uu[2] = 0.0;
    }
    double r[3] = {f[1] * uu[2] - f[2] * uu[1], f[2] * uu[0] - f[0] * uu[2], f[0] * uu[1] - f[1] * uu[0]};
    double rl = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    for (int c = 0; c < 3; ++c) r[c] /= rl;
    double u[3] = {r[1] * f[2] - r[2] * f[1], r[2] * f[0] - r[0] * f[2], r[0] * f[1] - r[1] * f[0]};
    double th = tan(fov_y_deg * M_PI / 180.0 * 0.5);
    for (int32_t j = 0; j < H; ++j)
        for (int32_t i = 0; i < W; ++i) {
            double sx = ((i + 0.5) / W * 2.0 - 1.0) * th * ((double)W / H);
            double sy = (1.0 - (j + 0.5) / H * 2.0) * th;
            double v[3];
            for (int c = 0; c < 3; ++c) v[c] = f[c] + sx * r[c] + sy * u[c];
            double vl = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
            double* o = out + 3 * ((size_t)j * W + i);
            for (int c = 0; c < 3; ++c) o[c] = v[c] / vl;
        }
}

/* Equirectangular panorama, z-up, the environment map's parameterisation:
 * pixel (i, j) of W x H has azimuth (i + 1/2)/W 2 pi - pi and polar angle
 * (j + 1/2)/H pi. out [H*W][3]. */
void orc_panorama_dirs(int32_t W, int32_t H, double* out)
{
    for (int32_t j = 0; j < H; ++j)
        for (int32_t i = 0; i < W; ++i) {
            double ph = (i + 0.5) / W * 2.0 * M_PI - M_PI, th = (j + 0.5) / H * M_PI;
            double* o = out + 3 * ((size_t)j * W + i);
            o[0] = sin(th) * cos(ph);
            o[1] = sin(th) * sin(ph);
            o[2] = cos(th);
        }
}

/* Shading points of the n_pix pixels of a float32 G-buffer gbuf [n][16]
 * seen from origin along dirs [n][4]: pixel p is kept when W >= w_min and
 * N != 0 and, with a second G-buffer `front` given, when that one's W is
 * below w_min or its unbiased depth is larger (D/W < D'/W', decided in
 * float32 as the quotients of the stored values). Kept pixels, in pixel
 * order: out_pix, and out [k][14] = x (3), n (3), wo (3), albedo (3), rough,
 * metal with x = o + (D/W) d, n = N/|N|, wo = -d, materials / W. Returns
 * the count. */
int64_t orc_gbuffer_points(int64_t n_pix, const float* gbuf, const float* origin, const float* dirs, float w_min,
                           const float* front, int64_t* out_pix, double* out)
{
    int64_t k = 0;
    for (int64_t p = 0; p < n_pix; ++p) {
        const float* b = gbuf + 16 * (size_t)p;
        const float W = b[3];
        if (!(W >= w_min)) continue;
        const double nl = sqrt((double)b[4] * b[4] + (double)b[5] * b[5] + (double)b[6] * b[6]);
        if (!(nl > 0.0)) continue;
        if (front) {
            const float* f = front + 16 * (size_t)p;
            if (f[3] >= w_min) {
                const float dn = b[7] / W, df = f[7] / f[3];
                if (!(dn < df)) continue;
            }
        }
        const float* d = dirs + 4 * (size_t)p;
        const double t = (double)b[7] / W;
        double* o = out + 14 * (size_t)k;
        for (int c = 0; c < 3; ++c) {
            o[c] = origin[c] + t * d[c];
            o[3 + c] = b[4 + c] / nl;
            o[6 + c] = -(double)d[c];
            o[9 + c] = (double)b[8 + c] / W;
        }
        o[12] = (double)b[11] / W;
        o[13] = (double)b[12] / W;
        out_pix[k++] = p;
    }
    return k;
}

/* The composed frame out [n_pix][3] (see the header): scene colour C_s from
 * scene_gbuf, its shadow ratio shadow [n_sc][3] at pixels sc_pix, the
 * object's shaded colour obj_rgb [n_obj][3] and alpha W_o (from obj_gbuf)
 * at pixels obj_pix. */
void orc_depth_composite(int64_t n_pix, const float* scene_gbuf, const float* obj_gbuf, int64_t n_sc,
                         const int64_t* sc_pix, const float* shadow, int64_t n_obj, const int64_t* obj_pix,
                         const float* obj_rgb, double* out)
{
    for (int64_t p = 0; p < n_pix; ++p)
        for (int c = 0; c < 3; ++c) out[3 * p + c] = scene_gbuf[16 * (size_t)p + c];
    for (int64_t k = 0; k < n_sc; ++k)
        for (int c = 0; c < 3; ++c) out[3 * sc_pix[k] + c] *= shadow[3 * k + c];
    for (int64_t k = 0; k < n_obj; ++k) {
        const int64_t p = obj_pix[k];
        const double a = obj_gbuf[16 * (size_t)p + 3];
        for (int c = 0; c < 3; ++c) out[3 * p + c] = a * obj_rgb[3 * k + c] + (1.0 - a) * out[3 * p + c];
    }
}

/* Automatic placement of SOPs (Sec. 3.2): farthest point sampling of a
 * surface point cloud, then an offset along the normals. Distances are the
 * exact integer squared distances of positions quantised to 2^-20 (the
 * query's keys), so every choice is exact: the first point is `start`;
 * each next one maximises the smallest key to the points already chosen,
 * ties to the lower index. out_pos[i] = pts[idx] + offset * nrm[idx] (when
 * out_pos and nrm are given). */
static int64_t gb_quant(float v) { return (int64_t)nearbyint((double)v * 1048576.0); }

void orc_fps(int64_t n, const float* pts, const float* nrm, int32_t k, int64_t start, double offset,
             int64_t* out_idx, double* out_pos)
{
    int64_t* q = (int64_t*)malloc(sizeof(int64_t) * 3 * (size_t)(n > 0 ? n : 1));
    uint64_t* dmin = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) {
        for (int a = 0; a < 3; ++a) q[3 * i + a] = gb_quant(pts[3 * i + a]);
        dmin[i] = UINT64_MAX;
    }
    int64_t cur = start;
    for (int32_t it = 0; it < k; ++it) {
        out_idx[it] = cur;
        uint64_t best = 0;
        int64_t bi = -1;
        for (int64_t i = 0; i < n; ++i) {
            const int64_t dx = q[3 * i] - q[3 * cur], dy = q[3 * i + 1] - q[3 * cur + 1], dz = q[3 * i + 2] - q[3 * cur + 2];
            const uint64_t key = (uint64_t)(dx * dx) + (uint64_t)(dy * dy) + (uint64_t)(dz * dz);
            if (key < dmin[i]) dmin[i] = key;
            if (bi < 0 || dmin[i] > best) {
                best = dmin[i];
                bi = i;
            }
        }
        cur = bi;
    }
    if (out_pos)
        for (int32_t it = 0; it < k; ++it) {
            const int64_t i = out_idx[it];
            for (int a = 0; a < 3; ++a)
                out_pos[3 * it + a] = (double)pts[3 * i + a] + (nrm ? offset * (double)nrm[3 * i + a] : 0.0);
        }
    free(dmin);
    free(q);
}
