"""Pins of the FP64 oracle of the deferred front end (Sec. 3.1, the alpha
blending of G-buffers; Sec. 4.3, deferred shading and depth compositing):
closed forms for one and two Gaussians along a ray, the surfel normal and
its turn towards the ray, agreement with the bake oracle on the bake's own
rays, the camera and panorama conventions, and the shading-point and
compositing rules on G-buffers with known contents."""
import numpy as np
import pytest

from paper_2510_07729_gb300 import inputs as I

F = np.float32


def gauss(mean, scale, quat, opacity, rgb):
    return dict(mean=np.array(mean, F).reshape(-1, 3), scale=np.array(scale, F).reshape(-1, 3),
                quat=np.array(quat, F).reshape(-1, 4), opacity=np.array(opacity, F).reshape(-1),
                rgb=np.array(rgb, F).reshape(-1, 3))


def mats(n, seed=0):
    rng = np.random.default_rng(seed)
    return dict(albedo=rng.uniform(0, 1, (n, 3)).astype(F), rough=rng.uniform(0.1, 1, n).astype(F),
                metal=rng.uniform(0, 1, n).astype(F))


def unit(v):
    v = np.asarray(v, np.float64)
    return v / np.linalg.norm(v)


def test_empty_scene_is_zero(orc):
    g = gauss(np.zeros((0, 3)), np.zeros((0, 3)), np.zeros((0, 4)), [], np.zeros((0, 3)))
    out, fl = orc.trace_gbuffer(g, mats(0), [[0, 0, 0]], np.array([[0, 0, 1, 0], [1, 0, 0, 0]], F))
    assert np.all(out == 0.0) and np.all(fl == 0)


def test_one_isotropic_gaussian_closed_form(orc):
    """A ray from the origin along +x passing at distance r from the centre
    of an isotropic Gaussian (scale s, opacity o): alpha = o exp(-r^2/2s^2),
    t* = the centre's abscissa; every buffer is alpha times the Gaussian's
    value; its normal is local axis 0 (equal scales: the first), turned
    towards the ray."""
    s, o, r, cx = 0.05, 0.8, 0.03, 2.0
    q = unit([0.9, 0.1, -0.3, 0.2])
    g = gauss([cx, r, 0.0], [s, s, s], q, [o], [[0.2, 0.5, 0.9]])
    m = mats(1, 3)
    out, fl = orc.trace_gbuffer(g, m, [[0, 0, 0]], np.array([[1, 0, 0, 0]], F))
    a = float(F(o)) * np.exp(-0.5 * (float(F(r)) / float(F(s))) ** 2)
    b = out[0]
    assert fl[0] == 0
    assert b[3] == pytest.approx(a, rel=1e-12)
    np.testing.assert_allclose(b[0:3], a * g["rgb"][0], rtol=1e-12)
    assert b[7] / b[3] == pytest.approx(float(F(cx)), rel=1e-12)
    np.testing.assert_allclose(b[8:11], a * m["albedo"][0], rtol=1e-12)
    assert b[11] == pytest.approx(a * m["rough"][0], rel=1e-12)
    assert b[12] == pytest.approx(a * m["metal"][0], rel=1e-12)
    w, x, y, z = (float(v) for v in g["quat"][0] / np.linalg.norm(g["quat"][0].astype(np.float64)))
    ax0 = np.array([1 - 2 * (y * y + z * z), 2 * (x * y + w * z), 2 * (x * z - w * y)])
    ax0 = ax0 if ax0[0] <= 0 else -ax0  # faces the ray (d = +x)
    np.testing.assert_allclose(b[4:7], a * ax0, rtol=1e-12, atol=1e-15)


def test_two_gaussians_composite_front_to_back(orc):
    """Two Gaussians on the ray: B = a1 b1 + (1 - a1) a2 b2, the nearer one
    first whatever their index order."""
    g = gauss([[3.0, 0, 0], [1.0, 0, 0]], [[0.1] * 3, [0.1] * 3], [[1, 0, 0, 0]] * 2, [0.7, 0.4],
              [[1, 0, 0], [0, 1, 0]])
    m = mats(2, 4)
    out, _ = orc.trace_gbuffer(g, m, [[0, 0, 0]], np.array([[1, 0, 0, 0]], F))
    a1, a2 = 0.4, 0.7  # the nearer one (index 1) has opacity 0.4
    b = out[0]
    assert b[3] == pytest.approx(a1 + (1 - a1) * a2, rel=1e-7)
    np.testing.assert_allclose(b[0:3], [(1 - a1) * a2, a1, 0.0], rtol=1e-7, atol=1e-12)
    assert b[7] == pytest.approx(a1 * 1.0 + (1 - a1) * a2 * 3.0, rel=1e-7)
    np.testing.assert_allclose(b[8:11], a1 * m["albedo"][1] + (1 - a1) * a2 * m["albedo"][0], rtol=1e-6)
    # identity rotation, equal scales: axis 0 = +x, turned to face the ray
    np.testing.assert_allclose(b[4:7], [-b[3], 0.0, 0.0], rtol=1e-12)


def test_surfel_normal_faces_the_ray_from_either_side(orc):
    """A flattened Gaussian whose thin axis is n: rays from both sides see
    a normal of +-n, always against the ray; W is the same."""
    n = unit([0.3, -0.2, 0.93])
    q = I._quats_with_axis(np.random.default_rng(0), n[None])[0]
    g = gauss([0, 0, 0], [0.2, 0.1, 0.005], q, [0.9], [[1, 1, 1]])
    m = mats(1)
    d1, d2 = unit([0.1, 0.05, -1.0]), unit([-0.1, 0.0, 1.0])
    org = np.array([-2 * d1, -2 * d2], F)
    dirs = np.array([[*d1, 0], [*d2, 0]], F)
    out, fl = orc.trace_gbuffer(g, m, org, dirs, rays=[0, 3])  # origin 0 along d1, origin 1 along d2
    assert np.all(fl == 0)
    nq = np.asarray(n, np.float32).astype(np.float64)
    for k, d in enumerate(dirs[:, :3].astype(np.float64)):
        nn = out[k, 4:7] / out[k, 3]
        assert np.dot(nn, d) < 0
        assert abs(abs(np.dot(nn, nq)) - 1.0) < 1e-6


@pytest.mark.parametrize("scales,axis", [([0.005, 0.2, 0.1], 0), ([0.2, 0.005, 0.1], 1), ([0.2, 0.1, 0.005], 2),
                                         ([0.2, 0.01, 0.01], 1), ([0.01, 0.2, 0.01], 0)])
def test_normal_is_the_axis_of_smallest_scale(orc, scales, axis):
    """Identity rotation: the normal is +-e_axis for the axis of smallest
    scale (the first of equal ones), against the ray."""
    g = gauss([0, 0, 0], scales, [1, 0, 0, 0], [0.9], [[1, 1, 1]])
    d = unit([0.5, -0.6, 0.62])
    out, _ = orc.trace_gbuffer(g, mats(1), np.array([-3 * d], F), np.array([[*d, 0]], F))
    want = np.zeros(3)
    want[axis] = -np.sign(np.float32(d[axis]))
    np.testing.assert_allclose(out[0, 4:7] / out[0, 3], want, atol=1e-15)


def test_matches_the_bake_oracle_on_its_rays(orc):
    """Rays from the tiny workload's probes along their texel directions
    (rounded to float32): C, W and D/W agree with the bake oracle's
    L_in, O and depth to the direction's rounding."""
    c = I.make_tiny()
    R = c["R"]
    ti, tj = np.meshgrid(np.arange(R), np.arange(R), indexing="xy")
    ti, tj = ti.ravel().astype(np.int32), tj.ravel().astype(np.int32)
    dirs = np.empty((R * R, 4), F)
    dirs[:, :3] = orc.oct_decode(np.stack([(ti + 0.5) / R, (tj + 0.5) / R], 1)).astype(F)
    dirs[:, 3] = 0
    probes = [0, 17, 40]
    rays = np.concatenate([p * R * R + np.arange(R * R) for p in probes]).astype(np.int64)
    gb, fl = orc.trace_gbuffer(c["gauss"], mats(len(c["gauss"]["mean"])), c["probe_pos"], dirs, rays=rays)
    probe_of = np.repeat(np.array(probes, np.int32), R * R)
    rgb, occ, dep, bfl = orc.bake_rays(c["gauss"], c["probe_pos"], R, probe_of, np.tile(ti, len(probes)),
                                       np.tile(tj, len(probes)))
    ok = (fl & ~16) == 0
    ok &= bfl == 0
    assert ok.mean() > 0.9 and (gb[:, 3] > 0.1).mean() > 0.3
    np.testing.assert_allclose(gb[ok, 3], occ[ok], rtol=2e-5, atol=1e-7)
    np.testing.assert_allclose(gb[ok, 0:3], rgb[ok], rtol=2e-5, atol=1e-7)
    w = gb[:, 3] > 1e-3
    np.testing.assert_allclose(gb[ok & w, 7] / gb[ok & w, 3], dep[ok & w], rtol=1e-4, atol=1e-6)


def test_pinhole_convention(orc):
    """Unit rays; with an odd image the centre pixel looks at the target; the
    outermost pixel centres sit at the field of view minus half a pixel; the
    input generator's rays (an independent implementation) agree."""
    eye, target = np.array([1.0, -2.0, 0.5]), np.array([0.2, 0.1, -0.3])
    W, H, fov = 9, 5, 40.0
    d = orc.pinhole_dirs(W, H, eye, target, fov)
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-15)
    f = unit(target - eye)
    np.testing.assert_allclose(d[(H // 2) * W + W // 2], f, atol=1e-15)
    top, bot = d[0 * W + W // 2], d[(H - 1) * W + W // 2]
    ang = np.arccos(np.clip(np.dot(top, bot), -1, 1))
    th = np.tan(np.deg2rad(fov) / 2) * (1 - 1 / H)
    assert ang == pytest.approx(2 * np.arctan(th), rel=1e-12)
    np.testing.assert_allclose(d, I.pinhole_rays(eye, target, W, H, fov), atol=1e-14)
    # looking straight down along the up axis: the fallback up vector
    d2 = orc.pinhole_dirs(W, H, [0, 0, 3.0], [0, 0, 0], fov)
    np.testing.assert_allclose(d2, I.pinhole_rays([0, 0, 3.0], [0, 0, 0], W, H, fov), atol=1e-14)


def test_panorama_uses_the_environment_parameterisation(orc):
    """Looking up an environment map with a distinct value per texel at the
    direction of every panorama pixel returns that pixel's texel."""
    H, W = 8, 16
    d = orc.panorama_dirs(W, H)
    env = np.arange(H * W * 3, dtype=F).reshape(H, W, 3)
    got = orc.env_lookup(env, d)
    np.testing.assert_allclose(got, env.reshape(-1, 3), rtol=0, atol=1e-9)
    np.testing.assert_allclose(d, I.equirect_texel_dirs(H, W).reshape(-1, 3), atol=1e-15)


def make_gbuf(rng, n):
    gb = np.zeros((n, 16), F)
    W = rng.uniform(0, 1, n).astype(F)
    t = rng.uniform(0.5, 4, n)
    gb[:, 3] = W
    gb[:, 7] = (W * t).astype(F)
    gb[:, 4:7] = (rng.standard_normal((n, 3)) * W[:, None]).astype(F)
    gb[:, 8:11] = (rng.uniform(0, 1, (n, 3)) * W[:, None]).astype(F)
    gb[:, 11] = (rng.uniform(0.1, 1, n) * W).astype(F)
    gb[:, 12] = (rng.uniform(0, 1, n) * W).astype(F)
    gb[:, 0:3] = rng.uniform(0, 1, (n, 3)).astype(F)
    return gb


def test_gbuffer_points_rules(orc):
    rng = np.random.default_rng(1)
    n = 400
    gb = make_gbuf(rng, n)
    gb[0, 3] = F(0.5)  # exactly w_min: kept
    gb[1, 3] = np.nextafter(F(0.5), F(0))  # just below: dropped
    gb[2, 4:7] = 0  # no normal: dropped
    org = np.array([0.3, -0.1, 2.0], F)
    d = np.array([unit(v) for v in rng.standard_normal((n, 3))], F)
    pix, pts = orc.gbuffer_points(gb, org, d, 0.5)
    want = np.flatnonzero((gb[:, 3] >= F(0.5)) & (np.abs(gb[:, 4:7]).sum(1) > 0))
    assert np.array_equal(pix, want) and 0 in pix and 1 not in pix and 2 not in pix
    W = gb[pix, 3].astype(np.float64)
    t = gb[pix, 7] / W
    np.testing.assert_allclose(pts["x"], org + t[:, None] * d[pix], rtol=1e-15, atol=1e-15)
    np.testing.assert_allclose(np.linalg.norm(pts["n"], axis=1), 1.0, atol=1e-15)
    np.testing.assert_allclose(pts["wo"], -d[pix], atol=0)
    np.testing.assert_allclose(pts["albedo"], gb[pix, 8:11] / W[:, None], rtol=1e-15)
    # a G-buffer in front hides the pixels it covers nearer than their own
    front = make_gbuf(rng, n)
    pix2, _ = orc.gbuffer_points(gb, org, d, 0.5, front=front)
    fw = front[:, 3] >= F(0.5)
    near = (gb[:, 7] / gb[:, 3]).astype(F) < (front[:, 7] / front[:, 3]).astype(F)
    assert np.array_equal(pix2, want[(~fw[want]) | near[want]])


def test_depth_composite_rules(orc):
    rng = np.random.default_rng(2)
    n = 50
    sg, og = make_gbuf(rng, n), make_gbuf(rng, n)
    sc_pix = np.arange(0, 30)
    shadow = rng.uniform(0, 1, (30, 3)).astype(F)
    obj_pix = np.array([5, 31, 40])
    og[40, 3] = 1.0  # opaque object pixel
    obj_rgb = rng.uniform(0, 2, (3, 3)).astype(F)
    out = orc.depth_composite(sg, og, sc_pix, shadow, obj_pix, obj_rgb)
    # no object, no scene point: the scene colour as traced
    np.testing.assert_array_equal(out[45], sg[45, 0:3].astype(np.float64))
    # scene point, no object: colour times its shadow ratio
    np.testing.assert_allclose(out[7], sg[7, 0:3].astype(np.float64) * shadow[7], rtol=1e-15)
    # opaque object: its own colour
    np.testing.assert_allclose(out[40], obj_rgb[2], rtol=1e-15)
    # partial alpha over a shadowed scene pixel
    a = float(og[5, 3])
    want = a * obj_rgb[0].astype(np.float64) + (1 - a) * (sg[5, 0:3].astype(np.float64) * shadow[5])
    np.testing.assert_allclose(out[5], want, rtol=1e-14)


def test_order_allowance_bounds_a_swap_of_tied_hits(orc):
    """Two isotropic Gaussians with the same t* (mirror images across the
    ray; other orientations, so other normals): the
    oracle orders them by index, so swapping their indices swaps their
    order. The reported allowance is twice the change, T a1 a2 |b1 - b2|."""
    s, r = 0.05, 0.02
    g = gauss([[2.0, r, 0], [2.0, -r, 0]], [[s] * 3, [s] * 3], [[1, 0, 0, 0], [0.9, 0.3, 0.1, 0.2]],
              [0.8, 0.6], [[0.9, 0.1, 0.2], [0.1, 0.7, 0.5]])
    m = mats(2, 9)
    sw = {k: v[::-1].copy() for k, v in g.items()}
    msw = {k: v[::-1].copy() for k, v in m.items()}
    ray = np.array([[1, 0, 0, 0]], F)
    a, fa, ta = orc.trace_gbuffer(g, m, [[0, 0, 0]], ray, t_stop=0.0, order_allowance=True)
    b, fb, tb = orc.trace_gbuffer(sw, msw, [[0, 0, 0]], ray, t_stop=0.0, order_allowance=True)
    assert fa[0] & orc.FLAG_ORDER and fb[0] & orc.FLAG_ORDER
    diff = np.abs(a[0] - b[0])
    assert diff[0:3].max() > 1e-3  # the order matters for the colour
    assert a[0, 3] == pytest.approx(b[0, 3], rel=1e-15)  # not for W
    np.testing.assert_allclose(ta[0], 2 * diff, rtol=1e-9, atol=1e-15)
    np.testing.assert_allclose(tb[0], ta[0], rtol=1e-9, atol=1e-15)
    # hits that do not tie get no allowance
    far = gauss([[2.0, r, 0], [3.0, -r, 0]], [[s] * 3, [s] * 3], [[1, 0, 0, 0]] * 2, [0.8, 0.6],
                [[0.9, 0.1, 0.2], [0.1, 0.7, 0.5]])
    _, ff, tf = orc.trace_gbuffer(far, m, [[0, 0, 0]], ray, t_stop=0.0, order_allowance=True)
    assert ff[0] == 0 and not tf.any()
