"""Seeded synthetic inputs for the SOP bake and query/shade workloads.

This module only *synthesises* inputs (Gaussian clouds, probe positions,
shading points, environment maps, synthetic probe atlases). It contains none
of the SOP method's arithmetic (no octahedral mapping, compositing, probe
blending or shading), so that the FP64 oracle and the CUDA path can both be fed
from it without sharing any method code.

The paper's datasets (SynCom, TensoIR, ...) are not available; these
generators stand in for them with the sizes and distributions of the five
workloads:

  tiny      2k isotropic Gaussians in a shell, 64 Fibonacci probes at 8x8,
            4096 points on the unit sphere, 16x32 lobed env, K=4, S=64
  object    200k anisotropic Gaussians on a union of 5 ellipsoids, 4096 FPS
            probes at 16x16 offset by 1% of the object size along the normal
            (placement of Sec. 3.1.2), an 800x800 pinhole view, 256x512
            log-normal env, K=8, S=128
  compose   the 'object' object on a ground plane with clutter (1.2M
            Gaussians total), 4096 object probes + 4096 shadow-region probes
            within 6x the object size (Sec. 4.1), 1920x1080 view, K=8, S=64
  diff      the 'object' scene seen from 4 cameras (adjoint workload)
  deferred  the composition rebuilt from flattened (surfel-like) Gaussians
            with per-Gaussian materials, for the G-buffer front end: the
            object (200k) and the scene (ground 700k, heights jittered, + clutter
            300k) traced
            separately from a 1920x1080 camera, the two probe sets of
            'compose'

Every array is float32 (int32 for indices) and C-contiguous.
"""
from __future__ import annotations

import copy
import functools

import numpy as np

F32 = np.float32
# vertical field of view of the 800x800 object views (camera at distance 3)
OBJECT_FOV = 28.0


# --------------------------------------------------------------------------
# small geometric helpers (input synthesis only)
# --------------------------------------------------------------------------
def _unit_vectors(rng, n):
    v = rng.standard_normal((n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def _random_rotations(rng, n):
    """Uniform random 3x3 rotations via QR of Gaussian matrices."""
    out = np.empty((n, 3, 3))
    for i in range(n):
        q, r = np.linalg.qr(rng.standard_normal((3, 3)))
        q = q * np.sign(np.diag(r))[None, :]
        if np.linalg.det(q) < 0:
            q[:, 0] = -q[:, 0]
        out[i] = q
    return out


def _random_quats(rng, n):
    """Uniform random unit quaternions, (w, x, y, z) order."""
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def fibonacci_sphere(n):
    i = np.arange(n, dtype=np.float64) + 0.5
    z = 1.0 - 2.0 * i / n
    phi = i * np.pi * (3.0 - np.sqrt(5.0))
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)


class Ellipsoids:
    """A union of oriented ellipsoids: centre c, semi-axes a, rotation Rm
    (columns = world directions of the local axes)."""

    def __init__(self, centres, axes, rots):
        self.c = np.asarray(centres, np.float64)
        self.a = np.asarray(axes, np.float64)
        self.R = np.asarray(rots, np.float64)

    def __len__(self):
        return len(self.c)

    def inside(self, x, exclude=None):
        """Boolean [n]: x strictly inside any ellipsoid (optionally skipping
        ellipsoid index array `exclude`, one per point)."""
        ins = np.zeros(len(x), bool)
        for e in range(len(self)):
            loc = (x - self.c[e]) @ self.R[e]
            r2 = np.sum((loc / self.a[e]) ** 2, axis=1)
            m = r2 < 1.0 - 1e-9
            if exclude is not None:
                m &= exclude != e
            ins |= m
        return ins

    def sample_surface(self, rng, n):
        """Area-uniform points on the union boundary with outward normals."""
        # area element of the map u -> a*u on the unit sphere is
        # prod(a) * ||u / a|| ; accept against the global maximum.
        wmax = max(np.prod(a) / np.min(a) for a in self.a)
        pts, nrm = [], []
        got = 0
        while got < n:
            m = max(4 * (n - got), 4096)
            e = rng.integers(0, len(self), m)
            u = _unit_vectors(rng, m)
            a = self.a[e]
            w = np.prod(a, axis=1) * np.linalg.norm(u / a, axis=1)
            keep = rng.random(m) * wmax < w
            e, u, a = e[keep], u[keep], a[keep]
            loc = u * a
            x = self.c[e] + np.einsum("nij,nj->ni", self.R[e], loc)
            g = np.einsum("nij,nj->ni", self.R[e], loc / (a * a))
            g /= np.linalg.norm(g, axis=1, keepdims=True)
            ok = ~self.inside(x, exclude=e)
            pts.append(x[ok])
            nrm.append(g[ok])
            got += int(ok.sum())
        return np.concatenate(pts)[:n], np.concatenate(nrm)[:n]

    def intersect(self, o, d):
        """First entering hit of rays from the single origin o (3,) along
        unit directions d [n,3] (t > 0). Returns t (inf on miss), ellipsoid
        id (-1 on miss) and the outward normal."""
        o = np.asarray(o, np.float64)
        n = len(d)
        tbest = np.full(n, np.inf)
        ebest = np.full(n, -1, np.int64)
        for e in range(len(self)):
            Me = self.R[e] / self.a[e][None, :]
            lo = (o - self.c[e]) @ Me
            ld = d @ Me
            A = np.einsum("ij,ij->i", ld, ld)
            B = ld @ lo
            C = float(lo @ lo) - 1.0
            disc = B * B - A * C
            hit = disc > 0
            t0 = (-B - np.sqrt(np.where(hit, disc, 0.0))) / A
            ok = hit & (t0 > 1e-9) & (t0 < tbest)
            tbest[ok] = t0[ok]
            ebest[ok] = e
        nrm = np.zeros((n, 3))
        h = ebest >= 0
        if h.any():
            x = o[None, :] + tbest[h, None] * d[h]
            e = ebest[h]
            loc = np.einsum("nji,nj->ni", self.R[e], x - self.c[e])
            g = np.einsum("nij,nj->ni", self.R[e], loc / self.a[e] ** 2)
            nrm[h] = g / np.linalg.norm(g, axis=1, keepdims=True)
        return tbest, ebest, nrm


def farthest_point_sampling(pts, k, start=0):
    """Greedy FPS: indices of k points of `pts` (float64 [n,3])."""
    X, Y, Z = (np.ascontiguousarray(pts[:, i]) for i in range(3))
    n = len(pts)
    sel = np.empty(k, np.int64)
    dmin = np.full(n, np.inf)
    d = np.empty(n)
    t = np.empty(n)
    cur = start
    for i in range(k):
        sel[i] = cur
        np.subtract(X, X[cur], out=d); np.multiply(d, d, out=d)
        np.subtract(Y, Y[cur], out=t); np.multiply(t, t, out=t); d += t
        np.subtract(Z, Z[cur], out=t); np.multiply(t, t, out=t); d += t
        np.minimum(dmin, d, out=dmin)
        cur = int(np.argmax(dmin))
    return sel


def pinhole_rays(cam_pos, look_at, width, height, fov_y_deg, up=(0.0, 0.0, 1.0)):
    """Per-pixel unit ray directions [H*W, 3] (row-major, row 0 at top)."""
    cam_pos = np.asarray(cam_pos, np.float64)
    fwd = np.asarray(look_at, np.float64) - cam_pos
    fwd /= np.linalg.norm(fwd)
    up = np.asarray(up, np.float64)
    if abs(np.dot(up, fwd)) > 0.99:
        up = np.array([0.0, 1.0, 0.0])
    right = np.cross(fwd, up)
    right /= np.linalg.norm(right)
    upv = np.cross(right, fwd)
    th = np.tan(np.deg2rad(fov_y_deg) * 0.5)
    jj, ii = np.meshgrid(np.arange(height), np.arange(width), indexing="ij")
    sx = ((ii + 0.5) / width * 2.0 - 1.0) * th * (width / height)
    sy = (1.0 - (jj + 0.5) / height * 2.0) * th
    d = fwd[None, :] + sx.reshape(-1, 1) * right[None, :] + sy.reshape(-1, 1) * upv[None, :]
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def equirect_texel_dirs(He, We):
    """Unit direction of every equirect texel centre, z-up: row r has polar
    angle (r+1/2)/He * pi, column c has azimuth (c+1/2)/We * 2pi - pi."""
    th = (np.arange(He) + 0.5) / He * np.pi
    ph = (np.arange(We) + 0.5) / We * 2.0 * np.pi - np.pi
    T, P = np.meshgrid(th, ph, indexing="ij")
    return np.stack([np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T)], axis=-1)


# --------------------------------------------------------------------------
# building blocks
# --------------------------------------------------------------------------
def gaussians_on_surface(rng, ells, n, scale_range=(0.002, 0.02), opacity_range=(0.2, 1.0)):
    mean, _ = ells.sample_surface(rng, n)
    lo, hi = np.log(scale_range[0]), np.log(scale_range[1])
    scale = np.exp(rng.uniform(lo, hi, (n, 3)))
    return dict(
        mean=mean.astype(F32),
        scale=scale.astype(F32),
        quat=_random_quats(rng, n).astype(F32),
        opacity=rng.uniform(*opacity_range, n).astype(F32),
        rgb=rng.uniform(0.0, 1.0, (n, 3)).astype(F32),
    )


def _quats_with_axis(rng, nrm):
    """Unit quaternions (w, x, y, z) whose rotation takes the local z axis
    to the unit vectors nrm [n,3], with a uniform random spin about it."""
    n = len(nrm)
    a = np.where(np.abs(nrm[:, :1]) < 0.9, np.array([[1.0, 0.0, 0.0]]), np.array([[0.0, 1.0, 0.0]]))
    t = np.cross(a, nrm)
    t /= np.linalg.norm(t, axis=1, keepdims=True)
    b = np.cross(nrm, t)
    ang = rng.uniform(0, 2 * np.pi, n)[:, None]
    t, b = np.cos(ang) * t + np.sin(ang) * b, -np.sin(ang) * t + np.cos(ang) * b
    Rm = np.stack([t, b, nrm], axis=2)  # columns: local axes in world space
    # rotation matrix to quaternion, through the largest of the four
    # candidate denominators (w, x, y, z) for accuracy
    m = Rm
    cand = np.stack([1.0 + m[:, 0, 0] + m[:, 1, 1] + m[:, 2, 2], 1.0 + m[:, 0, 0] - m[:, 1, 1] - m[:, 2, 2],
                     1.0 - m[:, 0, 0] + m[:, 1, 1] - m[:, 2, 2], 1.0 - m[:, 0, 0] - m[:, 1, 1] + m[:, 2, 2]], axis=1)
    k = np.argmax(cand, axis=1)
    r = np.sqrt(np.maximum(cand[np.arange(n), k], 1e-300))
    s21, s02, s10 = m[:, 2, 1] - m[:, 1, 2], m[:, 0, 2] - m[:, 2, 0], m[:, 1, 0] - m[:, 0, 1]
    a01, a02, a12 = m[:, 0, 1] + m[:, 1, 0], m[:, 0, 2] + m[:, 2, 0], m[:, 1, 2] + m[:, 2, 1]
    q = np.select([k[:, None] == 0, k[:, None] == 1, k[:, None] == 2, k[:, None] == 3],
                  [np.stack([r * r, s21, s02, s10], 1), np.stack([s21, r * r, a01, a02], 1),
                   np.stack([s02, a01, r * r, a12], 1), np.stack([s10, a02, a12, r * r], 1)])
    q = q / (2.0 * r[:, None])
    return q


def surfels(rng, mean, nrm, scale_range=(0.002, 0.02), flat=0.1, opacity_range=(0.2, 1.0)):
    """Flattened Gaussians at mean [n,3]: two tangent scales log-uniform in
    scale_range, the third (along nrm) `flat` times the smaller, opacity
    uniform, rgb uniform."""
    n = len(mean)
    lo, hi = np.log(scale_range[0]), np.log(scale_range[1])
    st = np.exp(rng.uniform(lo, hi, (n, 2)))
    scale = np.concatenate([st, flat * st.min(1, keepdims=True)], axis=1)
    return dict(mean=mean.astype(F32), scale=scale.astype(F32), quat=_quats_with_axis(rng, nrm).astype(F32),
                opacity=rng.uniform(*opacity_range, n).astype(F32), rgb=rng.uniform(0.0, 1.0, (n, 3)).astype(F32))


def concat_gaussians(*gs):
    return {k: np.ascontiguousarray(np.concatenate([g[k] for g in gs])) for k in gs[0]}


def materials(rng, m):
    return dict(
        albedo=rng.uniform(0.0, 1.0, (m, 3)).astype(F32),
        rough=rng.uniform(0.1, 1.0, m).astype(F32),
        metal=rng.uniform(0.0, 1.0, m).astype(F32),
    )


def env_lognormal(rng, He, We, sigma=1.5):
    return np.exp(rng.normal(0.0, sigma, (He, We, 3))).astype(F32)


def env_lobes(rng, He, We, n_lobes=3):
    """0.5 + sum_j a_j exp(lambda_j (w . mu_j - 1)) evaluated at texel centres."""
    mu = _unit_vectors(rng, n_lobes)
    lam = rng.uniform(5.0, 30.0, n_lobes)
    amp = rng.uniform(0.0, 2.0, (n_lobes, 3))
    w = equirect_texel_dirs(He, We)
    env = np.full((He, We, 3), 0.5)
    for j in range(n_lobes):
        env += amp[j][None, None, :] * np.exp(lam[j] * (w @ mu[j] - 1.0))[..., None]
    return env.astype(F32)


def synthetic_maps(rng, P, R):
    """Independent per-texel probe maps (a hard case for interpolation):
    RGB indirect radiance U(0, 0.5), occlusion U(0, 1), depth U(0.01, 2)."""
    return dict(
        rgb=rng.uniform(0.0, 0.5, (P, R, R, 3)).astype(F32),
        occ=rng.uniform(0.0, 1.0, (P, R, R)).astype(F32),
        depth=rng.uniform(0.01, 2.0, (P, R, R)).astype(F32),
    )


@functools.lru_cache(maxsize=2)
def _object(seed):
    """The 5-ellipsoid object: ellipsoids, 200k Gaussians, 4096 probes."""
    rng = np.random.default_rng(seed)
    ells = Ellipsoids(rng.uniform(-0.6, 0.6, (5, 3)), rng.uniform(0.2, 0.6, (5, 3)),
                      _random_rotations(rng, 5))
    g = gaussians_on_surface(rng, ells, 200_000)
    samp, snrm = ells.sample_surface(rng, 65_536)
    diag = float(np.linalg.norm(samp.max(0) - samp.min(0)))
    sel = farthest_point_sampling(samp, 4096)
    ppos = samp[sel] + 0.01 * diag * snrm[sel]
    return rng, ells, g, ppos, snrm[sel], samp, diag


def _view(rng, ells, cam_pos, W, H, fov):
    d = pinhole_rays(cam_pos, (0.0, 0.0, 0.0), W, H, fov)
    o = np.asarray(cam_pos, np.float64)
    t, e, nrm = ells.intersect(o, d)
    hit = e >= 0
    x = o[None, :] + t[hit, None] * d[hit]
    return x, nrm[hit], -d[hit], hit


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------
def make_tiny(seed=0):
    rng = np.random.default_rng(seed)
    N = 2000
    r = np.cbrt(rng.uniform(0.8 ** 3, 1.0, N))
    mean = _unit_vectors(rng, N) * r[:, None]
    s = np.exp(rng.uniform(np.log(0.005), np.log(0.03), N))
    g = dict(mean=mean.astype(F32),
             scale=np.repeat(s[:, None], 3, axis=1).astype(F32),
             quat=_random_quats(rng, N).astype(F32),
             opacity=rng.uniform(0.3, 1.0, N).astype(F32),
             rgb=rng.uniform(0.0, 1.0, (N, 3)).astype(F32))
    ppos = fibonacci_sphere(64)
    M = 4096
    x = _unit_vectors(rng, M)
    mat = materials(rng, M)
    env = env_lobes(rng, 16, 32)
    return dict(name="tiny", gauss=g, probe_pos=ppos.astype(F32), probe_nrm=ppos.astype(F32), R=8,
                x=x.astype(F32), n=x.astype(F32), wo=x.astype(F32), **mat, env=env, K=4, S=64)


def make_object(seed=1):
    rng, ells, g, ppos, pnrm, _, diag = _object(seed)
    # the cached scene's generator state is copied, so that every call draws
    # the same view, materials and environment
    rng = copy.deepcopy(rng)
    cam = _unit_vectors(rng, 1)[0] * 3.0
    x, n, wo, _ = _view(rng, ells, cam, 800, 800, OBJECT_FOV)
    mat = materials(rng, len(x))
    env = env_lognormal(rng, 256, 512)
    return dict(name="object", gauss=g, probe_pos=ppos.astype(F32), probe_nrm=pnrm.astype(F32), R=16,
                x=x.astype(F32), n=n.astype(F32), wo=wo.astype(F32), **mat, env=env, K=8, S=128,
                object_size=diag)


def make_diff(seed=3, views=4):
    """The 'object' scene with `views` cameras; concatenated points and a
    U(0,1)^3 target image for an L2 loss."""
    _, ells, g, ppos, pnrm, _, diag = _object(1)
    rng = np.random.default_rng(seed)
    xs, ns, wos = [], [], []
    for _ in range(views):
        cam = _unit_vectors(rng, 1)[0] * 3.0
        x, n, wo, _ = _view(rng, ells, cam, 800, 800, OBJECT_FOV)
        xs.append(x); ns.append(n); wos.append(wo)
    x, n, wo = np.concatenate(xs), np.concatenate(ns), np.concatenate(wos)
    mat = materials(rng, len(x))
    env = env_lognormal(rng, 256, 512)
    target = rng.uniform(0.0, 1.0, (len(x), 3)).astype(F32)
    return dict(name="diff", gauss=g, probe_pos=ppos.astype(F32), probe_nrm=pnrm.astype(F32), R=16,
                x=x.astype(F32), n=n.astype(F32), wo=wo.astype(F32), **mat, env=env, K=8, S=128,
                target=target, object_size=diag)


def make_compose(seed=2):
    """Object-scene composition at 1920x1080. Returns the object set (SHADE)
    and the scene set (SHADOW) with their own probes; both bake against the
    object Gaussians only (object self-occlusion, and the occlusion O' the
    object casts on the scene)."""
    _, obj_ells, gobj, opos, onrm, osamp, diag = _object(1)
    rng = np.random.default_rng(seed)
    lo, hi = osamp.min(0), osamp.max(0)
    size = float(np.max(hi - lo))
    zg = float(lo[2])
    cxy = 0.5 * (lo[:2] + hi[:2])
    half = 3.0 * size  # square of side 6x the object size
    # ground Gaussians: flat layer on z = zg
    ng = 700_000
    gm = np.empty((ng, 3))
    gm[:, :2] = cxy + rng.uniform(-half, half, (ng, 2))
    gm[:, 2] = zg
    s = np.exp(rng.uniform(np.log(0.002), np.log(0.02), (ng, 3)))
    ground = dict(mean=gm.astype(F32), scale=s.astype(F32), quat=_random_quats(rng, ng).astype(F32),
                  opacity=rng.uniform(0.2, 1.0, ng).astype(F32), rgb=rng.uniform(0, 1, (ng, 3)).astype(F32))
    # clutter: 30 small ellipsoids resting on the ground, away from the object
    nc = 30
    ax = rng.uniform(0.05, 0.15, (nc, 3))
    cc = np.empty((nc, 3))
    k = 0
    while k < nc:
        p = cxy + rng.uniform(-half, half, 2)
        if np.linalg.norm(p - cxy) > 0.75 * size:
            cc[k, :2] = p
            k += 1
    cc[:, 2] = zg + ax[:, 2]
    clutter_ells = Ellipsoids(cc, ax, np.repeat(np.eye(3)[None], nc, axis=0))
    clutter = gaussians_on_surface(rng, clutter_ells, 300_000)
    scene = concat_gaussians(ground, clutter, gobj)
    # shadow-region probes: FPS over ground samples in the square
    gs = np.empty((65_536, 3))
    gs[:, :2] = cxy + rng.uniform(-half, half, (65_536, 2))
    gs[:, 2] = zg
    gs = gs[~clutter_ells.inside(gs)]
    sel = farthest_point_sampling(gs, 4096)
    spos = gs[sel] + np.array([0.0, 0.0, 0.01 * diag])
    snrm = np.tile(np.array([0.0, 0.0, 1.0]), (4096, 1))
    # camera looking down at the object from 35 degrees elevation
    az = rng.uniform(0, 2 * np.pi)
    el = np.deg2rad(35.0)
    dist = 2.2 * size / np.tan(np.deg2rad(25.0))
    target = np.array([cxy[0], cxy[1], zg + 0.3 * size])
    cam = target + dist * np.array([np.cos(el) * np.cos(az), np.cos(el) * np.sin(az), np.sin(el)])
    d = pinhole_rays(cam, target, 1920, 1080, 50.0)
    o = cam[None, :]
    t_obj, e_obj, n_obj = obj_ells.intersect(cam, d)
    t_cl, e_cl, n_cl = clutter_ells.intersect(cam, d)
    t_gr = np.where(d[:, 2] < 0, (zg - cam[2]) / np.where(d[:, 2] < 0, d[:, 2], -1.0), np.inf)
    n_gr = np.tile(np.array([0.0, 0.0, 1.0]), (len(d), 1))
    t_sc = np.minimum(t_cl, t_gr)
    n_sc = np.where((t_cl < t_gr)[:, None], n_cl, n_gr)
    is_obj = t_obj < t_sc
    is_sc = (~is_obj) & np.isfinite(t_sc)
    xo = o + t_obj[is_obj, None] * d[is_obj]
    xs = o + t_sc[is_sc, None] * d[is_sc]
    mat_o = materials(rng, len(xo))
    mat_s = materials(rng, len(xs))
    env = env_lognormal(rng, 256, 512)
    shade = dict(probe_pos=opos.astype(F32), probe_nrm=onrm.astype(F32), x=xo.astype(F32),
                 n=n_obj[is_obj].astype(F32), wo=(-d[is_obj]).astype(F32), **mat_o)
    shadow = dict(probe_pos=spos.astype(F32), probe_nrm=snrm.astype(F32), x=xs.astype(F32),
                  n=n_sc[is_sc].astype(F32), wo=(-d[is_sc]).astype(F32), **mat_s)
    return dict(name="compose", gauss_object=gobj, gauss_scene=scene, shade=shade, shadow=shadow,
                R=16, K=8, S=64, env=env, pixels=1920 * 1080, object_size=diag)


@functools.lru_cache(maxsize=1)
def make_deferred(seed=5):
    """The composition workload for the deferred front end (G-buffers traced
    from the camera): the 'object' ellipsoids, probes and size, covered by
    200k surfels with per-Gaussian materials; a scene of 700k ground surfels
    (normal +z) in the square of side 6x the object size and 300k surfels on
    30 clutter ellipsoids; 4096 shadow-region probes by FPS over ground
    samples; a 1920x1080 camera looking down at the object from 35 degrees;
    a 256x512 log-normal environment. The scene does not contain the object:
    the two are traced separately and composed by depth."""
    _, obj_ells, _, opos, onrm, osamp, diag = _object(1)
    rng = np.random.default_rng(seed)
    m, nr = obj_ells.sample_surface(rng, 200_000)
    gobj = surfels(rng, m, nr)
    mobj = materials(rng, 200_000)
    lo, hi = osamp.min(0), osamp.max(0)
    size = float(np.max(hi - lo))
    zg = float(lo[2])
    cxy = 0.5 * (lo[:2] + hi[:2])
    half = 3.0 * size
    ng = 700_000
    gm = np.empty((ng, 3))
    gm[:, :2] = cxy + rng.uniform(-half, half, (ng, 2))
    # a reconstructed ground is not exactly planar: heights jitter by 0.5%
    # of the object size (exactly coplanar surfels would tie in depth)
    gm[:, 2] = zg + rng.normal(0.0, 5e-3 * size, ng)
    ground = surfels(rng, gm, np.tile(np.array([0.0, 0.0, 1.0]), (ng, 1)))
    nc = 30
    ax = rng.uniform(0.05, 0.15, (nc, 3))
    cc = np.empty((nc, 3))
    k = 0
    while k < nc:
        p = cxy + rng.uniform(-half, half, 2)
        if np.linalg.norm(p - cxy) > 0.75 * size:
            cc[k, :2] = p
            k += 1
    cc[:, 2] = zg + ax[:, 2]
    clutter_ells = Ellipsoids(cc, ax, np.repeat(np.eye(3)[None], nc, axis=0))
    m, nr = clutter_ells.sample_surface(rng, 300_000)
    scene = concat_gaussians(ground, surfels(rng, m, nr))
    mscene = materials(rng, len(scene["mean"]))
    gs = np.empty((65_536, 3))
    gs[:, :2] = cxy + rng.uniform(-half, half, (65_536, 2))
    gs[:, 2] = zg
    gs = gs[~clutter_ells.inside(gs)]
    sel = farthest_point_sampling(gs, 4096)
    spos = gs[sel] + np.array([0.0, 0.0, 0.01 * diag])
    az = rng.uniform(0, 2 * np.pi)
    el = np.deg2rad(35.0)
    dist = 2.2 * size / np.tan(np.deg2rad(25.0))
    target = np.array([cxy[0], cxy[1], zg + 0.3 * size])
    eye = target + dist * np.array([np.cos(el) * np.cos(az), np.cos(el) * np.sin(az), np.sin(el)])
    W, H, fov = 1920, 1080, 50.0
    d = pinhole_rays(eye, target, W, H, fov)
    dirs = np.concatenate([d, np.zeros((len(d), 1))], axis=1).astype(F32)
    env = env_lognormal(rng, 256, 512)
    return dict(name="deferred", gauss_object=gobj, mats_object=mobj, gauss_scene=scene, mats_scene=mscene,
                eye=eye.astype(F32), target=target, fov=fov, W=W, H=H, dirs=dirs,
                obj_probe_pos=opos.astype(F32), scene_probe_pos=spos.astype(F32), env=env, R=16, K=8, S=64,
                object_size=diag)


def subsample(rng, arrays, keys, m):
    """Pick m random rows (same rows for every key)."""
    n = len(arrays[keys[0]])
    idx = np.sort(rng.choice(n, size=min(m, n), replace=False))
    return idx, {k: np.ascontiguousarray(arrays[k][idx]) for k in keys}


def smooth_maps(rng, P, R):
    """Probe maps that vary slowly with the texel index (random phases per
    probe): O in [0.2, 0.8], RGB in [0.1, 0.4]."""
    jj, ii = np.meshgrid(np.arange(R) / R, np.arange(R) / R, indexing="ij")
    ph = rng.uniform(0, 2 * np.pi, (P, 4, 2))
    wave = lambda k: np.sin(2 * np.pi * ii[None] + ph[:, k, 0, None, None]) * \
        np.cos(2 * np.pi * jj[None] + ph[:, k, 1, None, None])  # noqa: E731
    occ = 0.5 + 0.3 * wave(3)
    rgb = np.stack([0.25 + 0.15 * wave(c) for c in range(3)], axis=-1)
    return dict(rgb=rgb.astype(F32), occ=occ.astype(F32),
                depth=np.full((P, R, R), 0.5, F32))


# --------------------------------------------------------------------------
# learned bake surrogate: initial parameters and training / evaluation scenes
# --------------------------------------------------------------------------
SURR_BLOCKS = [("W1", (64, 18)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)), ("W3", (64, 64)), ("b3", (64,)),
               ("W4", (5, 64)), ("b4", (5,))]


def surrogate_init(seed):
    """Initial surrogate parameters (flat float32, block order above):
    weights uniform in +-sqrt(6 / fan_in), biases zero."""
    rng = np.random.default_rng(seed)
    out = []
    for name, shp in SURR_BLOCKS:
        if name.startswith("b"):
            out.append(np.zeros(shp))
        else:
            b = np.sqrt(6.0 / shp[1])
            out.append(rng.uniform(-b, b, shp))
    return np.concatenate([o.reshape(-1) for o in out]).astype(F32)


def surrogate_scene(seed, n_gauss=200_000, n_probes=4096):
    """A randomised 'object'-style scene (5 random ellipsoids) with probes at
    random surface samples offset by 1% of the size along the normal."""
    rng = np.random.default_rng(seed)
    ells = Ellipsoids(rng.uniform(-0.6, 0.6, (5, 3)), rng.uniform(0.2, 0.6, (5, 3)), _random_rotations(rng, 5))
    g = gaussians_on_surface(rng, ells, n_gauss)
    samp, snrm = ells.sample_surface(rng, n_probes)
    diag = float(np.linalg.norm(g["mean"].max(0) - g["mean"].min(0)))
    ppos = samp + 0.01 * diag * snrm
    return dict(gauss=g, probe_pos=ppos.astype(F32), probe_nrm=snrm.astype(F32), R=16)


def moved_object(seed=4):
    """The 'object' scene after its first ellipsoid's Gaussians move by a
    U(-0.5, 0.5)^3 translation; 4,096 probes re-placed on the new surface
    (random samples, offset 1% of the size along the normal)."""
    _, ells, g, _, _, _, diag = _object(1)
    rng = np.random.default_rng(seed)
    shift = rng.uniform(-0.5, 0.5, 3)
    mean = g["mean"].astype(np.float64)
    # Gaussians of ellipsoid 0: those lying on its surface
    loc = (mean - ells.c[0]) @ ells.R[0]
    on0 = np.abs(np.sum((loc / ells.a[0]) ** 2, axis=1) - 1.0) < 1e-6
    mean[on0] += shift
    g2 = dict(g, mean=mean.astype(F32))
    moved = Ellipsoids(ells.c + np.where(np.arange(5)[:, None] == 0, shift, 0.0), ells.a, ells.R)
    samp, snrm = moved.sample_surface(rng, 4096)
    ppos = samp + 0.01 * diag * snrm
    out = dict(gauss=g2, probe_pos=ppos.astype(F32), probe_nrm=snrm.astype(F32), R=16, moved=int(on0.sum()),
               shift=shift)
    # a view of the moved object (drawn after the scene, which it leaves
    # unchanged): shading points, materials, a log-normal environment
    cam = _unit_vectors(rng, 1)[0] * 3.0
    x, n, wo, _ = _view(rng, moved, cam, 400, 400, OBJECT_FOV)
    out.update(x=x.astype(F32), n=n.astype(F32), wo=wo.astype(F32), **materials(rng, len(x)),
               env=env_lognormal(rng, 256, 512), K=8, S=128)
    return out
