"""Pins of the oracle's probe bake: texel rays composited front to back
through 3D Gaussians (Sec. 3.1.2 SOP initialisation by ray tracing, Eq. 1
transmittance, D/W depth of Sec. 3.1). The response of a Gaussian along a ray
is its maximum, alpha = min(0.99, o exp(-m^2/2)), kept if >= 1/255."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

AMIN = 1.0 / 255.0


def gset(mean, scale, quat=None, opacity=None, rgb=None):
    n = len(mean)
    return dict(mean=np.asarray(mean, np.float32).reshape(n, 3),
                scale=np.asarray(scale, np.float32).reshape(n, 3),
                quat=np.asarray(quat if quat is not None else [[1, 0, 0, 0]] * n, np.float32).reshape(n, 4),
                opacity=np.asarray(opacity if opacity is not None else [0.8] * n, np.float32).reshape(n),
                rgb=np.asarray(rgb if rgb is not None else [[0.2, 0.4, 0.6]] * n, np.float32).reshape(n, 3))


def ray(orc, R, i, j):
    return orc.oct_decode(np.array([[(i + 0.5) / R, (j + 0.5) / R]]))[0]


def one_texel(orc, g, R=8, i=3, j=5, probe=(0, 0, 0), **kw):
    rgb, occ, dep, fl = orc.bake_rays(g, np.array([probe], np.float32), R, [0], [i], [j], **kw)
    return rgb[0], occ[0], dep[0], fl[0]


def test_empty_scene(orc):
    g = gset(np.zeros((0, 3)), np.zeros((0, 3)))
    rgb, occ, dep, fl = orc.bake(g, np.zeros((2, 3), np.float32), 8)
    assert not rgb.any() and not occ.any() and not dep.any() and not fl.any()


@pytest.mark.parametrize("r_over_s", [0.0, 0.5, 1.3, 2.0, 3.0])
def test_single_isotropic_gaussian(orc, r_over_s):
    d = ray(orc, 8, 3, 5)
    perp = np.cross(d, [0.3, 0.1, 0.9]); perp /= np.linalg.norm(perp)
    s, t0, o = 0.05, 1.25, 0.7
    mu = t0 * d + r_over_s * s * perp
    g = gset([mu], [s, s, s], opacity=[o])
    rgb, occ, dep, _ = one_texel(orc, g)
    a = o * np.exp(-0.5 * r_over_s ** 2)
    if a < AMIN:
        assert occ == 0 and dep == 0
        return
    # centre stored in float32: compare against the float32 position
    mu32 = np.asarray(mu, np.float32).astype(np.float64)
    tt = mu32 @ d
    rr2 = mu32 @ mu32 - tt * tt
    a = min(0.99, np.float64(np.float32(o)) * np.exp(-0.5 * rr2 / np.float64(np.float32(s)) ** 2))
    assert occ == pytest.approx(a, rel=1e-12)
    assert dep == pytest.approx(tt, rel=1e-12)
    assert np.allclose(rgb, a * np.float32([0.2, 0.4, 0.6]), rtol=1e-12)


def test_single_anisotropic_gaussian_brute_force(orc):
    rng = np.random.default_rng(0)
    for trial in range(20):
        R, i, j = 16, int(rng.integers(16)), int(rng.integers(16))
        d = ray(orc, R, i, j)
        q = rng.standard_normal(4); q /= np.linalg.norm(q)
        s = np.exp(rng.uniform(np.log(0.02), np.log(0.2), 3))
        mu = rng.uniform(0.5, 2.0) * d + rng.normal(0, 0.05, 3)
        g = gset([mu], s, quat=[q], opacity=[0.9])
        rgb, occ, dep, _ = one_texel(orc, g, R=R, i=i, j=j)
        # independent route: scipy rotation (x, y, z, w order), dense sampling
        q32 = g["quat"][0].astype(np.float64)
        Rm = Rotation.from_quat([q32[1], q32[2], q32[3], q32[0]]).as_matrix()
        Sig = Rm @ np.diag(g["scale"][0].astype(np.float64) ** 2) @ Rm.T
        Si = np.linalg.inv(Sig)
        m32 = g["mean"][0].astype(np.float64)
        t = np.linspace(0, 4, 400001)
        e = t[:, None] * d[None, :] - m32[None, :]
        m2 = np.einsum("ni,ij,nj->n", e, Si, e)
        k = np.argmin(m2)
        tt = np.linspace(t[max(k - 2, 0)], t[min(k + 2, len(t) - 1)], 20001)
        e = tt[:, None] * d[None, :] - m32[None, :]
        m2 = np.einsum("ni,ij,nj->n", e, Si, e)
        k = np.argmin(m2)
        a = np.float64(np.float32(0.9)) * np.exp(-0.5 * m2[k])
        if a < AMIN * 1.001:
            continue
        assert occ == pytest.approx(min(a, 0.99), rel=1e-9)
        assert dep == pytest.approx(tt[k], abs=1e-6)


def test_two_gaussians_front_to_back(orc):
    d = ray(orc, 8, 2, 6)
    g = gset([1.0 * d, 2.0 * d], [[0.05] * 3, [0.08] * 3], opacity=[0.6, 0.5], rgb=[[1, 0, 0], [0, 0, 1]])
    rgb, occ, dep, _ = one_texel(orc, g, i=2, j=6)
    a1, a2 = np.float64(np.float32(0.6)), np.float64(np.float32(0.5))
    t1, t2 = np.asarray(g["mean"], np.float64) @ d
    assert np.allclose(rgb, [a1, 0, (1 - a1) * a2], rtol=1e-12)
    assert occ == pytest.approx(1 - (1 - a1) * (1 - a2), rel=1e-12)
    assert dep == pytest.approx((a1 * t1 + (1 - a1) * a2 * t2) / (a1 + (1 - a1) * a2), rel=1e-12)
    # array order does not matter, only depth along the ray
    g2 = {k: v[::-1].copy() for k, v in g.items()}
    rgb2, occ2, dep2, _ = one_texel(orc, g2, i=2, j=6)
    assert np.allclose(rgb2, rgb, rtol=1e-14) and occ2 == pytest.approx(occ) and dep2 == pytest.approx(dep)


def test_behind_probe_and_alpha_limits(orc):
    d = ray(orc, 8, 4, 4)
    # behind the probe: max-density point at t* < 0 -> not composited
    rgb, occ, dep, _ = one_texel(orc, gset([-1.0 * d], [[0.05] * 3], opacity=[0.9]), i=4, j=4)
    assert occ == 0 and not rgb.any()
    # opacity 1 on the ray: clamped to 0.99
    _, occ, _, _ = one_texel(orc, gset([1.0 * d], [[0.05] * 3], opacity=[1.0]), i=4, j=4)
    assert occ == pytest.approx(0.99, rel=1e-15)
    # just below / above the 1/255 cut-off
    for f, keep in [(0.999, False), (1.001, True)]:
        o = np.float32(AMIN * f)
        _, occ, _, _ = one_texel(orc, gset([1.0 * d], [[0.05] * 3], opacity=[o]), i=4, j=4)
        assert (occ > 0) == keep


def test_early_stop(orc):
    d = ray(orc, 8, 1, 1)
    g = gset([1.0 * d, 2.0 * d, 3.0 * d, 4.0 * d], [[0.05] * 3] * 4, opacity=[0.98] * 4,
             rgb=[[1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 1]])
    a = np.float64(np.float32(0.98))
    rgb, occ, _, _ = one_texel(orc, g, i=1, j=1, t_stop=1e-4)
    # T after three hits is (1-a)^3 = 8e-6 < 1e-4: the fourth is not composited
    assert occ == pytest.approx(1 - (1 - a) ** 3, rel=1e-12)
    assert rgb[0] == pytest.approx(a, rel=1e-14)  # only the first hit is red
    rgb0, occ0, _, _ = one_texel(orc, g, i=1, j=1, t_stop=0.0)
    assert occ0 == pytest.approx(1 - (1 - a) ** 4, rel=1e-12)
    assert rgb0[0] - rgb[0] == pytest.approx((1 - a) ** 3 * a, rel=1e-9)


def test_full_probe_sees_gaussian_in_its_texel(orc):
    R = 8
    for (i, j) in [(0, 0), (7, 0), (3, 4), (7, 7)]:
        d = ray(orc, R, i, j)
        g = gset([0.5 * d], [[0.01] * 3], opacity=[0.9])
        _, occ, _, _ = orc.bake(g, np.zeros((1, 3), np.float32), R)
        hit = np.argwhere(occ[0] > 0)
        assert hit.tolist() == [[j, i]]


def test_flags_mark_near_ties(orc):
    d = ray(orc, 8, 3, 3)
    g = gset([1.0 * d, 1.0 * d], [[0.05] * 3] * 2, opacity=[0.5, 0.5])
    _, _, _, fl = one_texel(orc, g, i=3, j=3)
    assert fl & orc.FLAG_ORDER
    g = gset([1.0 * d, 1.5 * d], [[0.05] * 3] * 2, opacity=[0.5, 0.5])
    _, _, _, fl = one_texel(orc, g, i=3, j=3)
    assert fl == 0


def test_direction_allowance_matches_finite_differences(orc):
    """The bake's test allowance (bake_rays with_sens) bounds each output's
    change under an angular error eps of the ray direction by the sum, over
    the composited hits, of the change that moving that hit alone by the
    worst first-order amount causes. For an isotropic Gaussian, turning the
    ray by eps about the probe moves the ray's closest point to the centre by
    t* eps, the same as moving the centre by t* eps towards the ray. So each
    hit's term is a central difference of the oracle's own outputs with that
    centre moved; their sum must reproduce the allowance. A Gaussian
    saturated at alpha_max contributes nothing of its own but scales the
    hits behind it."""
    R, i, j = 8, 3, 5
    d = ray(orc, R, i, j)
    rng = np.random.default_rng(7)
    ts, ms = [0.6, 0.9, 1.0, 1.3], [0.8, 1.4, 0.0, 2.1]
    ss, ops = [0.03, 0.05, 0.04, 0.02], [0.5, 0.7, 1.0, 0.9]
    mus = []
    for t, m, s in zip(ts, ms, ss):
        perp = np.cross(d, rng.standard_normal(3))
        perp /= np.linalg.norm(perp)
        mus.append(t * d + m * s * perp)
    rgb = rng.uniform(0.1, 1.0, (4, 3))
    eps = 1e-4

    def outs(means):
        g = gset(means, [[s, s, s] for s in ss], opacity=ops, rgb=rgb)
        o_rgb, o_occ, o_dep, fl, sens = orc.bake_rays(g, np.zeros((1, 3), np.float32), R, [0], [i], [j],
                                                     eps_dir=eps, with_sens=True)
        return np.concatenate([o_rgb[0], [o_occ[0], o_dep[0]]]), sens[0], fl[0]

    base, sens, fl = outs(mus)
    assert fl == 0
    assert base[3] > 0.99  # the saturated Gaussian is composited
    fd = np.zeros(5)
    for k in range(4):
        mu32 = np.asarray(mus[k], np.float32).astype(np.float64)
        tk = mu32 @ d
        off = mu32 - tk * d
        if np.linalg.norm(off) == 0:
            continue
        e_hat = off / np.linalg.norm(off)
        step = tk * eps * e_hat
        plus = [m if q != k else mu32 + step for q, m in enumerate(mus)]
        minus = [m if q != k else mu32 - step for q, m in enumerate(mus)]
        fd += np.abs(outs(plus)[0] - outs(minus)[0]) / 2
    assert sens[3] > 0 and sens[4] > 0
    np.testing.assert_allclose(sens, fd, rtol=1e-3)
