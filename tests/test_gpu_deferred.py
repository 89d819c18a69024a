"""GPU parity of the deferred front end (Sec. 3.1 multi-target rendering,
Sec. 4.3 rendering) against the FP64 oracle, through the C ABI: camera and
panorama rays, the G-buffer trace (small scenes whole, the deferred
composition workload at full size on sampled rays), shading points,
depth compositing, and a whole composed frame at a small resolution."""
import numpy as np
import pytest
import torch

from paper_2510_07729_gb300 import inputs as I
from tests.tolerance import assert_close, excess

pytestmark = pytest.mark.gpu
F = np.float32


@pytest.fixture(scope="module")
def sop():
    from paper_2510_07729_gb300 import sop as S
    S.load()
    return S


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def tcuda(d):
    return {k: cuda(v) for k, v in d.items()}


def test_pinhole_dirs(sop, orc):
    for (W, H, eye, target, fov) in [(9, 5, (1.0, -2.0, 0.5), (0.2, 0.1, -0.3), 40.0),
                                     (640, 360, (0.0, 0.0, 3.0), (0.0, 0.0, 0.0), 50.0),
                                     (1920, 1080, (3.1, 2.2, 1.7), (0.1, -0.2, 0.05), 50.0)]:
        eye32, tg32 = np.array(eye, F), np.array(target, F)
        g = sop.pinhole_dirs(W, H, eye32, tg32, fov).cpu().numpy()
        o = orc.pinhole_dirs(W, H, eye32.astype(np.float64), tg32.astype(np.float64), float(F(fov)))
        assert np.all(g[:, 3] == 0)
        # the GPU's directions are FP32 (camera frame rounded once to float32,
        # two FMAs and a reciprocal square root per pixel): a few ulp of a
        # unit vector
        assert np.max(np.abs(g[:, :3] - o)) <= 8 * 2.0 ** -24


def test_panorama_dirs(sop, orc):
    for W, H in [(16, 8), (1024, 512)]:
        g = sop.panorama_dirs(W, H).cpu().numpy()
        o = orc.panorama_dirs(W, H)
        # FP32 angles in units of pi (one rounding each) and sincospif
        assert np.max(np.abs(g[:, :3] - o)) <= 8 * 2.0 ** -24


def compare_gbuf(orc, g, o, fl, what, extent, t_stop=1e-4):
    """Element-wise, as the bake: W (a product over hits) on rays with no
    decision near a threshold; the order-sensitive sums (C, D, A, R, M) also
    without near-equal t*; the normal also without a grazing hit. With an
    early stop (t_stop > 0) the order of near-equal hits decides which are
    composited, so W is then order-sensitive too."""
    dec_ok = (fl & (orc.FLAG_ALPHA_MIN | orc.FLAG_TNEAR | orc.FLAG_TSTOP)) == 0
    ok = dec_ok & ((fl & orc.FLAG_ORDER) == 0)
    w_ok = dec_ok if t_stop == 0 else ok
    assert_close(g[w_ok, 3], o[w_ok, 3], what=what + " W")
    assert_close(g[ok, 0:3], o[ok, 0:3], what=what + " C")
    assert_close(g[ok, 8:13], o[ok, 8:13], what=what + " A R M")
    assert_close(g[ok, 7], o[ok, 7], what=what + " D", absolute=4 * 2.0 ** -24 * extent * o[ok, 3])
    okn = ok & ((fl & orc.FLAG_GRAZING) == 0)
    assert_close(g[okn, 4:7], o[okn, 4:7], what=what + " N", absolute=2e-6 * o[okn, 3:4])
    assert np.all(g[:, 13:16] == 0)
    return int((~okn).sum())


def small_scene(seed=0):
    """Surfels on the unit sphere above a ground square, with materials."""
    rng = np.random.default_rng(seed)
    m, nr = I.Ellipsoids(np.zeros((1, 3)), np.ones((1, 3)), np.eye(3)[None]).sample_surface(rng, 3000)
    obj = I.surfels(rng, m, nr, scale_range=(0.02, 0.08))
    mo = I.materials(rng, 3000)
    gm = np.concatenate([rng.uniform(-3, 3, (6000, 2)), rng.normal(-1.0, 0.005, (6000, 1))], axis=1)
    scene = I.surfels(rng, gm, np.tile([0.0, 0.0, 1.0], (6000, 1)), scale_range=(0.03, 0.1))
    ms = I.materials(rng, 6000)
    return obj, mo, scene, ms


@pytest.mark.parametrize("t_stop", [0.0, 1e-4])
def test_trace_gbuffer_small(sop, orc, t_stop):
    obj, mo, scene, ms = small_scene()
    eye, target = np.array([2.5, -3.0, 1.5], F), np.array([0.0, 0.0, -0.3], F)
    W, H = 96, 64
    dirs = sop.pinhole_dirs(W, H, eye, target, 45.0)
    dn = dirs.cpu().numpy()
    for g, m, what in ((obj, mo, "object"), (scene, ms, "scene")):
        tr = sop.GbufferTracer(tcuda(g), tcuda(m), t_stop=t_stop)
        gb = tr.trace(cuda(eye[None]), dirs).cpu().numpy()
        o, fl = orc.trace_gbuffer(g, m, eye[None], dn, t_stop=t_stop)
        flagged = compare_gbuf(orc, gb, o, fl, what, extent=8.0, t_stop=t_stop)
        assert flagged <= 0.05 * len(fl)
        assert (o[:, 3] > 0.5).mean() > 0.1


def test_trace_gbuffer_several_origins(sop, orc):
    """Rays from several origins share one direction table (ray p n_d + t)."""
    c = I.make_tiny()
    g = c["gauss"]
    m = I.materials(np.random.default_rng(1), len(g["mean"]))
    dirs = sop.panorama_dirs(32, 16)
    org = c["probe_pos"][:5]
    tr = sop.GbufferTracer(tcuda(g), tcuda(m))
    gb = tr.trace(cuda(org), dirs).cpu().numpy()
    o, fl = orc.trace_gbuffer(g, m, org, dirs.cpu().numpy())
    compare_gbuf(orc, gb, o, fl, "tiny", extent=2.0)


def test_trace_gbuffer_empty_scene(sop):
    z = dict(mean=np.zeros((0, 3), F), scale=np.zeros((0, 3), F), quat=np.zeros((0, 4), F),
             opacity=np.zeros(0, F), rgb=np.zeros((0, 3), F))
    mz = dict(albedo=np.zeros((0, 3), F), rough=np.zeros(0, F), metal=np.zeros(0, F))
    tr = sop.GbufferTracer(tcuda(z), tcuda(mz))
    gb = tr.trace(cuda(np.zeros((1, 3), F)), sop.panorama_dirs(8, 4))
    assert not gb.any()


@pytest.fixture(scope="module")
def deferred():
    return I.make_deferred()


@pytest.mark.parametrize("part,n_samp", [("object", 1024), ("scene", 384)])
def test_deferred_full_size_sampled(sop, orc, deferred, part, n_samp):
    """The 1920x1080 deferred workload traced whole in the benchmark's
    launch configuration, sampled rays checked one by one. Surfels on one
    surface often tie in t* within rounding, so the order of tied hits is
    not unique: without an early stop, W (a product over the hits) is
    checked on every ray away from a threshold, and the other values
    within the oracle's allowance for reordering tied hits; with the
    benchmark's early stop, rays without ties are checked as usual."""
    d = deferred
    g, m = d["gauss_" + part], d["mats_" + part]
    rng = np.random.default_rng(7 if part == "object" else 8)
    for t_stop in (0.0, 1e-4):
        tr = sop.GbufferTracer(tcuda(g), tcuda(m), t_stop=t_stop)
        gb = tr.trace(cuda(d["eye"][None]), cuda(d["dirs"])).cpu().numpy()
        hit = np.flatnonzero(gb[:, 3] > 0)
        rays = np.sort(np.concatenate([rng.choice(hit, n_samp // 2, replace=False),
                                       rng.choice(len(gb), n_samp // 2, replace=False)]))
        o, fl, tie = orc.trace_gbuffer(g, m, d["eye"][None], d["dirs"], rays=rays, t_stop=t_stop,
                                       order_allowance=True)
        G = gb[rays]
        if t_stop == 0.0:
            dec_ok = (fl & (orc.FLAG_ALPHA_MIN | orc.FLAG_TNEAR)) == 0
            assert dec_ok.mean() > 0.97
            assert_close(G[dec_ok, 3], o[dec_ok, 3], what=part + " W")
            nok = dec_ok & ((fl & orc.FLAG_GRAZING) == 0)
            for sl, what, extra in ((slice(0, 3), " C", 0.0), (slice(8, 13), " A R M", 0.0),
                                    (slice(7, 8), " D", 4 * 2.0 ** -24 * 20.0),
                                    (slice(4, 7), " N", 2e-6)):
                rows = nok if what == " N" else dec_ok
                assert_close(G[rows, sl], o[rows, sl], what=part + what,
                             absolute=tie[rows, sl] + extra * o[rows, 3:4])
            assert (G[:, 3] > 0.5).sum() >= n_samp // 4
        else:
            flagged = compare_gbuf(orc, G, o, fl, part, extent=20.0, t_stop=t_stop)
            assert flagged <= 0.7 * len(rays)


def test_gbuffer_points(sop, orc):
    """Same float32 G-buffers on both sides: the kept pixels bit-exact (the
    decisions are float32 comparisons), the point values within rounding."""
    rng = np.random.default_rng(3)
    n = 5000
    gbs = []
    for _ in range(2):
        gb = np.zeros((n, 16), F)
        W = rng.uniform(0, 1, n).astype(F)
        W[::17] = 0.5
        gb[:, 3] = W
        gb[:, 7] = (W * rng.uniform(0.5, 4, n)).astype(F)
        gb[:, 4:7] = (rng.standard_normal((n, 3)) * W[:, None]).astype(F)
        gb[::23, 4:7] = 0
        gb[:, 8:11] = (rng.uniform(0, 1, (n, 3)) * W[:, None]).astype(F)
        gb[:, 11] = (rng.uniform(0.1, 1, n) * W).astype(F)
        gb[:, 12] = (rng.uniform(0, 1, n) * W).astype(F)
        gbs.append(gb)
    d = rng.standard_normal((n, 3))
    dirs = np.concatenate([d / np.linalg.norm(d, axis=1, keepdims=True), np.zeros((n, 1))], axis=1).astype(F)
    org = np.array([0.3, -0.1, 2.0], F)
    for front in (None, gbs[1]):
        pix, pts = sop.gbuffer_points(cuda(gbs[0]), org, cuda(dirs), 0.5, None if front is None else cuda(front))
        opix, opts = orc.gbuffer_points(gbs[0], org, dirs, 0.5, front=front)
        assert np.array_equal(pix.cpu().numpy(), opix)
        for k in ("x", "n", "wo", "albedo", "rough", "metal"):
            # x = o + t d may cancel: a few float32 ulps of |o| + t (t <= 4)
            ab = 4 * 2.0 ** -24 * (np.abs(org).max() + 4.0) if k == "x" else 0.0
            assert_close(pts[k].cpu().numpy(), opts[k], rtol=2e-6, what=k, absolute=ab)
    pix, _ = sop.gbuffer_points(cuda(gbs[0][:0]), org, cuda(dirs[:0]))
    assert pix.numel() == 0


def test_depth_composite(sop, orc):
    rng = np.random.default_rng(4)
    n = 3000
    sg = rng.uniform(0, 1, (n, 16)).astype(F)
    og = rng.uniform(0, 1, (n, 16)).astype(F)
    sc_pix = np.sort(rng.choice(n, 1200, replace=False)).astype(np.int64)
    obj_pix = np.sort(rng.choice(n, 400, replace=False)).astype(np.int64)
    shadow = rng.uniform(0, 1, (1200, 3)).astype(F)
    obj_rgb = rng.uniform(0, 2, (400, 3)).astype(F)
    g = sop.depth_composite(cuda(sg), cuda(og), cuda(sc_pix), cuda(shadow), cuda(obj_pix), cuda(obj_rgb))
    o = orc.depth_composite(sg, og, sc_pix, shadow, obj_pix, obj_rgb)
    assert_close(g.cpu().numpy(), o, rtol=1e-6, what="composite")


def test_composed_frame_small(sop, orc):
    """A whole composed frame: G-buffers of the object and the scene, the
    object's points in front SHADE-d with its probes, the scene's points
    SHADOW-ed with the shadow probes, depth compositing. Both sides run the
    same steps on their own values; pixels whose keep decision lies within
    rounding of a threshold in the oracle's G-buffers are left out."""
    obj, mo, scene, ms = small_scene(1)
    rng = np.random.default_rng(5)
    eye, target = np.array([2.5, -3.0, 1.5], F), np.array([0.0, 0.0, -0.3], F)
    W, H = 80, 48
    dirs_t = sop.pinhole_dirs(W, H, eye, target, 45.0)
    dirs = dirs_t.cpu().numpy()
    opos = (I.fibonacci_sphere(64) * 1.05).astype(F)
    spos = np.concatenate([rng.uniform(-3, 3, (64, 2)), np.full((64, 1), -0.97)], axis=1).astype(F)
    omaps, smaps = I.synthetic_maps(rng, 64, 8), I.synthetic_maps(rng, 64, 8)
    env = I.env_lobes(rng, 16, 32)
    K, S = 4, 32
    # oracle
    og, ofl = orc.trace_gbuffer(obj, mo, eye[None], dirs)
    sg, sfl = orc.trace_gbuffer(scene, ms, eye[None], dirs)
    og32, sg32 = og.astype(F), sg.astype(F)
    opix, opts = orc.gbuffer_points(og32, eye, dirs, 0.5, front=sg32)
    spix, spts = orc.gbuffer_points(sg32, eye, dirs, 0.5)
    f32 = lambda p: {k: np.ascontiguousarray(v, F) for k, v in p.items()}  # noqa: E731
    op, sp = f32(opts), f32(spts)
    orgb, _, _ = orc.query_shade(op["x"], op["n"], op["wo"], op["albedo"], op["rough"], op["metal"], opos,
                                 omaps["rgb"], omaps["occ"], env, K, S)
    osh, _, _ = orc.query_shade(sp["x"], sp["n"], sp["wo"], sp["albedo"], sp["rough"], sp["metal"], spos,
                                smaps["rgb"], smaps["occ"], env, K, S, mode=orc.MODE_SHADOW)
    ofr = orc.depth_composite(sg32, og32, spix, osh.astype(F), opix, orgb.astype(F))
    # GPU
    tro, trs = sop.GbufferTracer(tcuda(obj), tcuda(mo)), sop.GbufferTracer(tcuda(scene), tcuda(ms))
    ggo = tro.trace(cuda(eye[None]), dirs_t)
    ggs = trs.trace(cuda(eye[None]), dirs_t)
    gpix, gpts = sop.gbuffer_points(ggo, eye, dirs_t, 0.5, front=ggs)
    gspix, gspts = sop.gbuffer_points(ggs, eye, dirs_t, 0.5)

    def atlas(pp, maps):
        at = sop.make_atlas(cuda(pp), 8)
        sop.atlas_pack(cuda(maps["rgb"]), cuda(maps["occ"]), cuda(maps["depth"]), at)
        return at

    grgb = sop.query_shade(gpts["x"], gpts["n"], gpts["wo"], gpts["albedo"], gpts["rough"], gpts["metal"],
                           atlas(opos, omaps), cuda(env), K, S)
    gsh = sop.query_shade(gspts["x"], gspts["n"], gspts["wo"], gspts["albedo"], gspts["rough"], gspts["metal"],
                          atlas(spos, smaps), cuda(env), K, S, mode=sop.MODE_SHADOW)
    gfr = sop.depth_composite(ggs, ggo, gspix, gsh, gpix, grgb).cpu().numpy()
    # pixels with every decision away from rounding, in both G-buffers
    bad = (ofl != 0) | (sfl != 0)
    for gb in (og, sg):
        bad |= np.abs(gb[:, 3] - 0.5) < 1e-4
        nl = np.abs(gb[:, 4:7]).sum(1)
        bad |= (nl > 0) & (nl < 1e-6)
    both = (og[:, 3] > 0.4999) & (sg[:, 3] > 0.4999)
    dt = og[:, 7] / np.maximum(og[:, 3], 1e-30)
    ds = sg[:, 7] / np.maximum(sg[:, 3], 1e-30)
    bad |= both & (np.abs(dt - ds) < 1e-4 * np.minimum(dt, ds))
    assert bad.mean() < 0.05
    assert len(opix) > 50 and len(spix) > 500
    ok = ~bad
    assert np.array_equal(np.isin(np.arange(W * H), gpix.cpu().numpy())[ok], np.isin(np.arange(W * H), opix)[ok])
    # a point moved by the rounding of its G-buffer may pick another probe
    # set (keys quantised to 2^-20): a few pixels, each a different blend
    e = excess(gfr[ok], ofr[ok], rtol=1e-3).max(axis=1)
    assert (e > 1.0).mean() < 0.01, np.sort(e)[-10:]
