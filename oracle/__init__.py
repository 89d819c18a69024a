"""FP64 CPU oracle for the SOP bake and query/shade (test infrastructure).

Only the tests, the smoke check and the benchmark's CPU-baseline leg may
import this package. The product path (the CUDA library and its binding)
never does. The C source (sop_oracle.c) is compiled with gcc by `build()`
into oracle/_build/liboracle.so and driven here through ctypes; the
surrogate MLP part of the oracle is plain NumPy in `mlp.py`.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "sop_oracle.c")
SRCS = (SRC, os.path.join(HERE, "gbuffer_oracle.c"), os.path.join(HERE, "surrogate_oracle.c"))
LIB = os.path.join(HERE, "_build", "liboracle.so")

MODE_SHADE, MODE_SHADOW = 0, 1
ENV_EQUIRECT, ENV_OCTAHEDRAL = 0, 1
FLAG_ALPHA_MIN, FLAG_ORDER, FLAG_TNEAR, FLAG_TSTOP, FLAG_GRAZING = 1, 2, 4, 8, 16

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (IEEE double, no FMA contraction)."""
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(os.path.getmtime(f) for f in SRCS):
        return LIB
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]
    tmp = LIB + f".tmp{os.getpid()}"
    try:
        subprocess.run(base + ["-fopenmp", *SRCS, "-o", tmp, "-lm"], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + [*SRCS, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = C.CDLL(LIB)
        _lib.orc_num_threads.restype = C.c_int
        _lib.orc_gbuffer_points.restype = C.c_int64
        _lib.orc_surr_grid_dims.restype = C.c_int64
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _f32(a, shape_last=None):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return lib().orc_num_threads()


# ----------------------------------------------------------------------------
# octahedral map, frame, environment, BRDF
# ----------------------------------------------------------------------------
def oct_encode(d):
    d = _f64(d).reshape(-1, 3)
    uv = np.empty((len(d), 2))
    lib().orc_oct_encode_n(C.c_int64(len(d)), _p(d), _p(uv))
    return uv


def oct_decode(uv, l1_only=False):
    uv = _f64(uv).reshape(-1, 2)
    d = np.empty((len(uv), 3))
    lib().orc_oct_decode_n(C.c_int64(len(uv)), _p(uv), _p(d), C.c_int(1 if l1_only else 0))
    return d


def oct_wrap(R, i, j):
    si, sj = C.c_int(), C.c_int()
    lib().orc_oct_wrap(C.c_int(R), C.c_int(i), C.c_int(j), C.byref(si), C.byref(sj))
    return si.value, sj.value


def oct_bilerp(map_, uv):
    """map_: [R, R, C] float64 compact map; uv: [n, 2]."""
    map_ = _f64(map_)
    R, _, Ch = map_.shape
    uv = _f64(uv).reshape(-1, 2)
    out = np.empty((len(uv), Ch))
    lib().orc_oct_bilerp_n(C.c_int64(len(uv)), _p(map_), C.c_int(R), C.c_int(Ch), _p(uv), _p(out))
    return out


def hammersley(S):
    out = np.empty((S, 3))
    lib().orc_hammersley(C.c_int32(S), _p(out))
    return out


def onb(n):
    n = _f64(n).reshape(-1, 3)
    t, b = np.empty_like(n), np.empty_like(n)
    lib().orc_onb_n(C.c_int64(len(n)), _p(n), _p(t), _p(b))
    return t, b


def env_lookup(env, w):
    env = _f32(env)
    He, We, _ = env.shape
    w = _f64(w).reshape(-1, 3)
    out = np.empty((len(w), 3))
    lib().orc_env_lookup_n(C.c_int64(len(w)), _p(env), C.c_int32(He), C.c_int32(We), _p(w), _p(out))
    return out


def brdf(n, wo, wi, albedo, rough, metal, spec=0.5):
    n, wo, wi, albedo = (_f64(v).reshape(-1, 3) for v in (n, wo, wi, albedo))
    rough, metal = _f64(rough).reshape(-1), _f64(metal).reshape(-1)
    f = np.empty((len(n), 3))
    lib().orc_brdf_n(C.c_int64(len(n)), _p(n), _p(wo), _p(wi), _p(albedo), _p(rough), _p(metal),
                     C.c_double(spec), _p(f))
    return f


# ----------------------------------------------------------------------------
# bake
# ----------------------------------------------------------------------------
DEFAULT_BAKE = dict(t_near=0.0, alpha_min=1.0 / 255.0, alpha_max=0.99, t_stop=1e-4)


# angular error bound of a texel direction held in FP32 (rad): each unit
# component rounded once from double is off by at most 2^-25, so the vector
# by at most sqrt(3) 2^-25 < 2^-24
FP32_TEXEL_DIR_EPS = 2.0 ** -24


def bake_rays(gauss, probe_pos, R, probe_of, ti, tj, t_near=0.0, alpha_min=1.0 / 255.0,
              alpha_max=0.99, t_stop=1e-4, eps_dir=FP32_TEXEL_DIR_EPS, with_sens=False):
    """Bake the listed texel rays. Returns rgb [n,3], occ [n], depth [n], flags [n]
    and, with with_sens, the test allowance [n,5] (L0, L1, L2, O, D): each
    output's first-order bound under an angular error eps_dir of the ray
    direction (see orc_bake_rays)."""
    mean, scale, quat, op, rgb = (_f32(gauss[k]) for k in ("mean", "scale", "quat", "opacity", "rgb"))
    pp = _f32(probe_pos)
    probe_of, ti, tj = (np.ascontiguousarray(v, dtype=np.int32) for v in (probe_of, ti, tj))
    n = len(probe_of)
    o_rgb, o_occ, o_d = np.empty((n, 3)), np.empty(n), np.empty(n)
    o_fl = np.empty(n, np.int32)
    sens = np.empty((n, 5)) if with_sens else None
    lib().orc_bake_rays(C.c_int64(len(mean)), _p(mean), _p(scale), _p(quat), _p(op), _p(rgb), _p(pp),
                        C.c_int(R), C.c_int64(n), _p(probe_of), _p(ti), _p(tj), C.c_double(t_near),
                        C.c_double(alpha_min), C.c_double(alpha_max), C.c_double(t_stop),
                        _p(o_rgb), _p(o_occ), _p(o_d), _p(o_fl), C.c_double(eps_dir),
                        _p(sens) if with_sens else None)
    if with_sens:
        return o_rgb, o_occ, o_d, o_fl, sens
    return o_rgb, o_occ, o_d, o_fl


def bake(gauss, probe_pos, R, probes=None, with_sens=False, **kw):
    """Bake whole probes (all R*R texels). Returns maps [P',R,R,3], [P',R,R],
    [P',R,R] and flags [P',R,R] for the probes listed (default: all), and
    with with_sens the allowance [P',R,R,5] of bake_rays."""
    probes = np.arange(len(probe_pos)) if probes is None else np.asarray(probes)
    jj, ii = np.meshgrid(np.arange(R), np.arange(R), indexing="ij")
    po = np.repeat(probes, R * R)
    ti = np.tile(ii.reshape(-1), len(probes))
    tj = np.tile(jj.reshape(-1), len(probes))
    out = bake_rays(gauss, probe_pos, R, po, ti, tj, with_sens=with_sens, **kw)
    P = len(probes)
    res = (out[0].reshape(P, R, R, 3), out[1].reshape(P, R, R), out[2].reshape(P, R, R), out[3].reshape(P, R, R))
    return res + (out[4].reshape(P, R, R, 5),) if with_sens else res


# ----------------------------------------------------------------------------
# query / shade
# ----------------------------------------------------------------------------
def snap_key_for(eps_snap=1e-6):
    """Largest quantised squared distance (units of 2^-40) within eps_snap."""
    return int(np.floor((eps_snap * 1048576.0) ** 2))


UNBOUNDED = (1 << 64) - 1


def radius_key(radius=0.0):
    """Search radius (Sec. 3.2, fixed-radius neighbours) as a bound on the
    quantised squared distance: a probe takes part when its key is at most
    (r 2^20)^2, i.e. when its quantised distance is at most r; radius 0 is
    no bound. r is taken as float32; (r 2^20)^2 has at most 48 significant
    bits, so the double product is exact and its floor is the bound."""
    r = float(np.float32(radius))
    if r == 0.0:
        return UNBOUNDED
    rq = r * 1048576.0
    return int(np.floor(rq * rq))


def knn(x, probe_pos, K, radius=0.0):
    """K nearest probes (within the radius, if one is given): idx [M,K] with
    -1 in empty slots, key [M,K] (UINT64_MAX there)."""
    x, pp = _f32(x), _f32(probe_pos)
    M = len(x)
    idx = np.empty((M, K), np.int32)
    key = np.empty((M, K), np.uint64)
    lib().orc_knn(C.c_int64(M), _p(x), C.c_int32(len(pp)), _p(pp), C.c_int32(K), C.c_uint64(radius_key(radius)),
                  _p(idx), _p(key))
    return idx, key


def weights(x, n, probe_pos, idx, key, snap_key=None):
    x, n, pp = _f32(x), _f32(n), _f32(probe_pos)
    idx = np.ascontiguousarray(idx, np.int32)
    key = np.ascontiguousarray(key, np.uint64)
    M, K = idx.shape
    W = np.empty((M, K))
    sk = snap_key_for() if snap_key is None else snap_key
    lib().orc_weights(C.c_int64(M), _p(x), _p(n), _p(pp), C.c_int32(K), _p(idx), _p(key),
                      C.c_uint64(sk), _p(W))
    return W


def query_shade(x, n, wo, albedo, rough, metal, probe_pos, maps_rgb, maps_occ, env, K, S,
                mode=MODE_SHADE, spec=0.5, dirs=None, snap_key=None, env_layout=ENV_EQUIRECT, dir_world=False,
                radius=0.0):
    """FP64 query + shade. Returns out [M,3], idx [M,K], W [M,K]. dirs: the
    local direction set [S,3] (None: the centred Hammersley set), or with
    dir_world the importance-sampled world directions [S,4] (x, y, z, pdf).
    radius > 0 limits the neighbours to probes within it (idx -1, W 0 in
    the slots it leaves empty)."""
    x, n, wo, albedo, rough, metal = (_f32(v) for v in (x, n, wo, albedo, rough, metal))
    pp, mr, mo, env = _f32(probe_pos), _f32(maps_rgb), _f32(maps_occ), _f32(env)
    P, R = mr.shape[0], mr.shape[1]
    He, We, _ = env.shape
    M = len(x)
    out = np.empty((M, 3))
    idx = np.empty((M, K), np.int32)
    W = np.empty((M, K))
    dp = None if dirs is None else _f64(dirs)
    sk = snap_key_for() if snap_key is None else snap_key
    lib().orc_query_shade(C.c_int64(M), _p(x), _p(n), _p(wo), _p(albedo), _p(rough), _p(metal),
                          C.c_int32(P), _p(pp), C.c_int32(R), _p(mr), _p(mo), C.c_int32(He), C.c_int32(We),
                          _p(env), C.c_int32(S), None if dp is None else _p(dp), C.c_int32(K),
                          C.c_int32(mode), C.c_double(spec), C.c_uint64(sk), C.c_uint64(radius_key(radius)),
                          C.c_int32(env_layout), C.c_int32(1 if dir_world else 0), _p(out), _p(idx), _p(W))
    return out, idx, W


# angular error bound of one light direction in the FP32 path (rad): the
# rounding of the frame, the rotation into world space and of atan2
FP32_DIR_EPS = 2e-6


def query_shade_sensitivity(x, n, wo, albedo, rough, metal, probe_pos, maps_rgb, maps_occ, env, K, S,
                            mode=MODE_SHADE, spec=0.5, dirs=None, snap_key=None, eps=FP32_DIR_EPS,
                            env_layout=ENV_EQUIRECT, dir_world=False, radius=0.0):
    """Per-output allowance [M,3] for an FP32 evaluation (see the C docs)."""
    x, n, wo, albedo, rough, metal = (_f32(v) for v in (x, n, wo, albedo, rough, metal))
    pp, mr, mo, env = _f32(probe_pos), _f32(maps_rgb), _f32(maps_occ), _f32(env)
    P, R = mr.shape[0], mr.shape[1]
    He, We, _ = env.shape
    M = len(x)
    kap = np.empty((M, 3))
    dp = None if dirs is None else _f64(dirs)
    sk = snap_key_for() if snap_key is None else snap_key
    lib().orc_query_shade_sensitivity(
        C.c_int64(M), _p(x), _p(n), _p(wo), _p(albedo), _p(rough), _p(metal), C.c_int32(P), _p(pp), C.c_int32(R),
        _p(mr), _p(mo), C.c_int32(He), C.c_int32(We), _p(env), C.c_int32(S), None if dp is None else _p(dp),
        C.c_int32(K), C.c_int32(mode), C.c_double(spec), C.c_uint64(sk), C.c_uint64(radius_key(radius)),
        C.c_int32(env_layout), C.c_int32(1 if dir_world else 0), C.c_double(eps), _p(kap))
    return kap


def env_to_octahedral(env, H):
    """FP64 resampling of an equirectangular environment [He,We,3] into an
    octahedral one [H,H,3] (texel centre directions, bilinear)."""
    env = _f32(env)
    He, We, _ = env.shape
    out = np.empty((H, H, 3))
    lib().orc_env_to_oct(_p(env), C.c_int32(He), C.c_int32(We), C.c_int32(H), _p(out))
    return out


def env_importance_dirs(env, S):
    """Importance-sampled light directions [S,4] (x, y, z, pdf) from an
    octahedral environment [H,H,3] (see orc_env_importance_dirs)."""
    env = _f32(env)
    out = np.empty((S, 4))
    lib().orc_env_importance_dirs(_p(env), C.c_int32(env.shape[0]), C.c_int32(S), _p(out))
    return out


def env_oct_lookup(env, w):
    """FP64 bilinear lookup of an octahedral environment [H,H,3] at unit
    directions w [n,3] (the probe maps' mapping and border rule)."""
    env = _f32(env)
    w = _f64(w).reshape(-1, 3)
    out = np.empty((len(w), 3))
    lib().orc_env_oct_lookup_n(C.c_int64(len(w)), _p(env), C.c_int32(env.shape[0]), _p(w), _p(out))
    return out


def query_shade_grad(x, n, wo, albedo, rough, metal, probe_pos, maps_rgb, maps_occ, env, K, S, grad_out,
                     spec=0.5, dirs=None, snap_key=None, radius=0.0):
    """Analytic FP64 gradients of sum(grad_out * C) (SHADE mode). Returns a
    dict: albedo [M,3], rough [M], metal [M], normal [M,3] (w.r.t. the raw
    normal), env [He,We,3], maps_rgb [P,R,R,3], maps_occ [P,R,R], and the
    sums of the magnitudes of the per-direction terms of each per-point
    gradient (abs_albedo, abs_rough, abs_metal, abs_normal)."""
    x, n, wo, albedo, rough, metal = (_f32(v) for v in (x, n, wo, albedo, rough, metal))
    pp, mr, mo, env = _f32(probe_pos), _f32(maps_rgb), _f32(maps_occ), _f32(env)
    P, R = mr.shape[0], mr.shape[1]
    He, We, _ = env.shape
    M = len(x)
    go = _f64(grad_out).reshape(M, 3)
    out = dict(albedo=np.empty((M, 3)), rough=np.empty(M), metal=np.empty(M), normal=np.empty((M, 3)),
               env=np.zeros((He, We, 3)), maps_rgb=np.zeros((P, R, R, 3)), maps_occ=np.zeros((P, R, R)),
               abs_albedo=np.empty((M, 3)), abs_rough=np.empty(M), abs_metal=np.empty(M), abs_normal=np.empty(M))
    dp = None if dirs is None else _f64(dirs)
    sk = snap_key_for() if snap_key is None else snap_key
    lib().orc_query_shade_grad(
        C.c_int64(M), _p(x), _p(n), _p(wo), _p(albedo), _p(rough), _p(metal), C.c_int32(P), _p(pp), C.c_int32(R),
        _p(mr), _p(mo), C.c_int32(He), C.c_int32(We), _p(env), C.c_int32(S), None if dp is None else _p(dp),
        C.c_int32(K), C.c_double(spec), C.c_uint64(sk), C.c_uint64(radius_key(radius)), _p(go), _p(out["albedo"]), _p(out["rough"]),
        _p(out["metal"]), _p(out["normal"]), _p(out["env"]), _p(out["maps_rgb"]), _p(out["maps_occ"]),
        _p(out["abs_albedo"]), _p(out["abs_rough"]), _p(out["abs_metal"]), _p(out["abs_normal"]))
    return out


# ----------------------------------------------------------------------------
# deferred front end: G-buffers, shading points, depth compositing
# ----------------------------------------------------------------------------
GBUF_C, GBUF_W, GBUF_N, GBUF_D, GBUF_A, GBUF_R, GBUF_M = slice(0, 3), 3, slice(4, 7), 7, slice(8, 11), 11, 12


def trace_gbuffer(gauss, mats, origins, dirs, rays=None, t_near=0.0, alpha_min=1.0 / 255.0, alpha_max=0.99,
                  t_stop=1e-4, order_allowance=False):
    """FP64 multi-target rendering (see gbuffer_oracle.c). gauss: dict of
    mean/scale/quat/opacity/rgb; mats: albedo [N,3], rough [N], metal [N];
    origins [n_o,3]; dirs [n_d,4] (or [n_d,3]) float32 unit directions;
    rays: ray ids (origin id // n_d, direction id % n_d), default all.
    Returns (gbuf [n_rays,16], flags [n_rays]) and, with order_allowance,
    the per-value bound [n_rays,16] on what reordering tied hits can
    change."""
    g = {k: _f32(gauss[k]) for k in ("mean", "scale", "quat", "opacity", "rgb")}
    al, ro, me = _f32(mats["albedo"]), _f32(mats["rough"]), _f32(mats["metal"])
    org = _f32(origins).reshape(-1, 3)
    d = np.asarray(dirs, np.float32)
    if d.shape[-1] == 3:
        d = np.concatenate([d, np.zeros((len(d), 1), np.float32)], axis=1)
    d = np.ascontiguousarray(d)
    nd = len(d)
    rays = np.arange(len(org) * nd, dtype=np.int64) if rays is None else np.ascontiguousarray(rays, np.int64)
    out = np.empty((len(rays), 16))
    fl = np.empty(len(rays), np.int32)
    tie = np.empty((len(rays), 16))
    lib().orc_trace_gbuffer(C.c_int64(len(g["mean"])), _p(g["mean"]), _p(g["scale"]), _p(g["quat"]),
                            _p(g["opacity"]), _p(g["rgb"]), _p(al), _p(ro), _p(me), _p(org), C.c_int64(nd), _p(d),
                            C.c_int64(len(rays)), _p(rays), C.c_double(t_near), C.c_double(alpha_min),
                            C.c_double(alpha_max), C.c_double(t_stop), _p(out), _p(fl),
                            _p(tie) if order_allowance else None)
    return (out, fl, tie) if order_allowance else (out, fl)


def pinhole_dirs(W, H, eye, target, fov_y_deg, up=(0.0, 0.0, 1.0)):
    out = np.empty((H * W, 3))
    lib().orc_pinhole_dirs(C.c_int32(W), C.c_int32(H), _p(_f64(eye)), _p(_f64(target)), _p(_f64(up)),
                           C.c_double(fov_y_deg), _p(out))
    return out


def panorama_dirs(W, H):
    out = np.empty((H * W, 3))
    lib().orc_panorama_dirs(C.c_int32(W), C.c_int32(H), _p(out))
    return out


def gbuffer_points(gbuf, origin, dirs, w_min=0.5, front=None):
    """Shading points of a float32 G-buffer [n,16] (see gbuffer_oracle.c):
    returns (pix [k] int64, points dict x, n, wo, albedo, rough, metal)."""
    gb = _f32(gbuf)
    d = np.asarray(dirs, np.float32)
    if d.shape[-1] == 3:
        d = np.concatenate([d, np.zeros((len(d), 1), np.float32)], axis=1)
    d = np.ascontiguousarray(d)
    fr = None if front is None else _f32(front)
    n = len(gb)
    pix = np.empty(n, np.int64)
    out = np.empty((n, 14))
    k = lib().orc_gbuffer_points(C.c_int64(n), _p(gb), _p(_f32(origin)), _p(d), C.c_float(w_min),
                                 None if fr is None else _p(fr), _p(pix), _p(out))
    o = out[:k]
    return pix[:k], dict(x=o[:, 0:3], n=o[:, 3:6], wo=o[:, 6:9], albedo=o[:, 9:12], rough=o[:, 12], metal=o[:, 13])


def depth_composite(scene_gbuf, obj_gbuf, sc_pix, shadow, obj_pix, obj_rgb):
    sg, og = _f32(scene_gbuf), _f32(obj_gbuf)
    n = len(sg)
    out = np.empty((n, 3))
    lib().orc_depth_composite(C.c_int64(n), _p(sg), _p(og), C.c_int64(len(sc_pix)),
                              _p(np.ascontiguousarray(sc_pix, np.int64)), _p(_f32(shadow)), C.c_int64(len(obj_pix)),
                              _p(np.ascontiguousarray(obj_pix, np.int64)), _p(_f32(obj_rgb)), _p(out))
    return out


def fps(pts, k, start=0, nrm=None, offset=0.0):
    """Farthest point sampling with exact integer keys (see orc_fps):
    returns (idx [k] int64, positions [k,3] offset along nrm)."""
    p = _f32(pts).reshape(-1, 3)
    nr = None if nrm is None else _f32(nrm).reshape(-1, 3)
    idx = np.empty(k, np.int64)
    pos = np.empty((k, 3))
    lib().orc_fps(C.c_int64(len(p)), _p(p), None if nr is None else _p(nr), C.c_int32(k), C.c_int64(start),
                  C.c_double(offset), _p(idx), _p(pos))
    return idx, pos


# ----------------------------------------------------------------------------
# storage formats of the atlas depth plane
# ----------------------------------------------------------------------------
def fp8_e4m3_bits(x):
    """Bits of the FP8 E4M3 value nearest to each float32 x (1 sign bit, 4
    exponent bits with bias 7, 3 mantissa bits, subnormals below 2^-6, no
    infinities): ties to the even code, magnitudes beyond the largest
    finite value 448 saturate to it (NaN -> 0x7f). Written from the format's
    definition: the representable magnitudes are k 2^(e-3) for k = 8..15 and
    e = -6..8, and k 2^-9 for k = 0..7."""
    shape = np.shape(x)
    x = np.atleast_1d(np.asarray(x, np.float32)).astype(np.float64)
    s = np.signbit(x).astype(np.uint8) << 7
    a = np.abs(x)
    out = np.empty(a.shape, np.uint8)
    nan = np.isnan(a)
    # every magnitude at or above the largest finite value saturates to it
    a = np.minimum(np.where(nan, 0.0, a), 448.0)
    # the spacing of the representable values around a: 2^(e-3) for a in
    # [2^e, 2^(e+1)), e >= -6; 2^-9 below 2^-6
    e = np.floor(np.log2(np.maximum(a, 2.0 ** -6)))
    step = 2.0 ** (e - 3)
    q = a / step                      # exact: a power-of-two scaling
    k = np.floor(q)
    frac = q - k
    k = k + ((frac > 0.5) | ((frac == 0.5) & (np.mod(k, 2) == 1)))
    v = k * step                      # the rounded magnitude
    v = np.minimum(v, 448.0)
    # encode v: subnormal codes k for v < 2^-6, else exponent and mantissa
    sub = v < 2.0 ** -6
    ev = np.floor(np.log2(np.maximum(v, 2.0 ** -6)))
    mant = np.where(sub, v / 2.0 ** -9, v / 2.0 ** (ev - 3) - 8)
    code = np.where(sub, mant, (ev + 7) * 8 + mant)
    out[:] = code.astype(np.int64).astype(np.uint8)
    out = out | s
    out[nan] = 0x7F
    return out.reshape(shape)


# ----------------------------------------------------------------------------
# learned bake surrogate: texel features (surrogate_oracle.c)
# ----------------------------------------------------------------------------
SURR_KN = 256          # near field: at most this many nearest Gaussians
SURR_G = 128           # far field: cells along the longest axis
SURR_N_FEAT = 18       # direction (3), near (O, L rgb, D, W), far (6 x O, L rgb)


def surr_near_list(probe_pos, mean, r_n, KN=SURR_KN):
    """The near list of every probe: its at most KN nearest Gaussian centres
    within r_n (integer keys, ties to the lower index; -1 ends a short
    list), and t0, where the far field starts: the last listed Gaussian's
    distance when the list is full, else r_n."""
    idx, key = knn(probe_pos, mean, KN, radius=r_n)
    full = idx[:, KN - 1] >= 0
    t0 = np.where(full, np.sqrt(key[:, KN - 1].astype(np.float64)) / 1048576.0, float(r_n))
    return idx.astype(np.int32), t0


def surr_grid(gauss, alpha_min=1.0 / 255.0, alpha_max=0.99, G=SURR_G):
    """The far-field grid: (qlo [3], hq, dims [3], mass_q [cells], col_q
    [cells, 3]) with fixed-point sums in units of 2^-40."""
    mean, scale, op, rgb = (_f32(gauss[k]) for k in ("mean", "scale", "opacity", "rgb"))
    N = len(op)
    qlo = np.zeros(3, np.int64)
    hq = C.c_int64(0)
    dims = np.zeros(3, np.int32)
    cells = lib().orc_surr_grid_dims(C.c_int64(N), _p(mean), _p(op), C.c_double(alpha_min), C.c_int32(G), _p(qlo),
                                     C.byref(hq), _p(dims))
    n = max(int(cells), 1)
    mass = np.zeros(n, np.int64)
    col = np.zeros((n, 3), np.int64)
    if cells > 0:
        lib().orc_surr_grid_fill(C.c_int64(N), _p(mean), _p(scale), _p(op), _p(rgb), C.c_double(alpha_min),
                                 C.c_double(alpha_max), _p(qlo), C.c_int64(hq.value), _p(dims), _p(mass), _p(col))
    return qlo, int(hq.value), dims, mass, col


def surr_features(gauss, probe_pos, R, r_n, alpha_min=1.0 / 255.0, alpha_max=0.99, KN=SURR_KN, G=SURR_G,
                  near_list=None, far_sens=False):
    """FP64 texel features [P, R*R, 18] of every probe: the texel direction,
    the near field (O_n, L_n rgb, D_n, W_n) and the far field (1 - exp(-tau)
    at the 5 checkpoints and at the end, L_f rgb). Returns (feats, flags
    [P, R*R], near list [P, KN], t0 [P]), and with far_sens the far march's
    conditioning [P, R*R] (see surr_far)."""
    pp = _f32(probe_pos)
    P = len(pp)
    if near_list is None:
        lst, t0 = surr_near_list(pp, gauss["mean"], r_n, KN)
    else:
        lst, t0 = near_list
    mean, scale, quat, op, rgb = (_f32(gauss[k]) for k in ("mean", "scale", "quat", "opacity", "rgb"))
    near = np.empty((P, R * R, 6))
    flags = np.zeros((P, R * R), np.int32)
    lst = np.ascontiguousarray(lst, np.int32)
    lib().orc_surr_near(C.c_int32(P), _p(pp), C.c_int32(R), _p(mean), _p(scale), _p(quat), _p(op), _p(rgb),
                        _p(lst), C.c_int32(lst.shape[1]), C.c_double(alpha_min), C.c_double(alpha_max), _p(near),
                        _p(flags))
    far, sens = surr_far(pp, t0, R, *surr_grid(gauss, alpha_min, alpha_max, G), with_sens=True)
    dirs = np.array([_texel_dir(R, t % R, t // R) for t in range(R * R)])
    feats = np.concatenate([np.broadcast_to(dirs, (P, R * R, 3)), near, far], axis=-1)
    return (feats, flags, lst, t0, sens) if far_sens else (feats, flags, lst, t0)


def surr_far(probe_pos, t0, R, qlo, hq, dims, mass, col, with_sens=False):
    """The far-field features [P, R*R, 9] of every texel of the probes, from
    t0 [P] on, through a grid (qlo, hq, dims, fixed-point mass, col). With
    with_sens, also the march's conditioning [P, R*R]: how far tau can move
    when its cell boundary times are taken in FP32 (sum over the segments of
    sigma times the rounding scale of their two ends)."""
    pp = _f32(probe_pos)
    far = np.empty((len(pp), R * R, 9))
    sens = np.empty((len(pp), R * R)) if with_sens else None
    t0 = np.ascontiguousarray(t0, np.float64)
    qlo = np.ascontiguousarray(qlo, np.int64)
    dims = np.ascontiguousarray(dims, np.int32)
    mass = np.ascontiguousarray(mass, np.int64)
    col = np.ascontiguousarray(col, np.int64)
    lib().orc_surr_far(C.c_int32(len(pp)), _p(pp), _p(t0), C.c_int32(R), _p(qlo), C.c_int64(int(hq)), _p(dims),
                       _p(mass), _p(col), _p(far), _p(sens) if with_sens else None)
    return (far, sens) if with_sens else far


def _texel_dir(R, i, j):
    d = np.empty(3)
    lib().orc_texel_dir(C.c_int(R), C.c_int(i), C.c_int(j), _p(d))
    return d
