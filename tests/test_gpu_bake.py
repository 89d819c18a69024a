"""GPU parity of the probe bake (Sec. 3.1.2 ray-traced SOP initialisation,
Eq. 1 compositing, D/W depth) against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest
import torch

from paper_2510_07729_gb300 import inputs as I
from tests.tolerance import assert_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sop():
    from paper_2510_07729_gb300 import sop as S
    S.load()
    return S


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def gpu_bake(sop, g, probe_pos, R, **kw):
    at = sop.make_atlas(cuda(probe_pos), R)
    sop.bake({k: cuda(v) for k, v in g.items()}, at, **kw)
    torch.cuda.synchronize()
    rgb, occ, dep = at.interior()
    return rgb.cpu().numpy(), occ.cpu().numpy(), dep.cpu().numpy(), at


def compare(orc, g_rgb, g_occ, g_dep, o_rgb, o_occ, o_dep, flags, sens, what, extent=2.0):
    """Element-wise parity; `sens` is the oracle's allowance [..., 5] for
    the FP32 rounding of each texel direction (orc.bake with_sens)."""
    order_ok = (flags & orc.FLAG_ORDER) == 0
    dec_ok = (flags & (orc.FLAG_ALPHA_MIN | orc.FLAG_TNEAR | orc.FLAG_TSTOP)) == 0
    # occlusion is a product over hits: order-independent
    assert_close(g_occ[dec_ok], o_occ[dec_ok], what=what + " O", absolute=sens[..., 3][dec_ok])
    ok = order_ok & dec_ok
    assert_close(g_rgb[ok], o_rgb[ok], what=what + " L_in", absolute=sens[..., :3][ok])
    assert_close(g_dep[ok], o_dep[ok], what=what + " D", absolute=4 * 2.0 ** -24 * extent + sens[..., 4][ok])
    return int((~ok).sum())


@pytest.mark.parametrize("t_stop", [0.0, 1e-4])
def test_tiny_bake_parity(sop, orc, t_stop):
    c = I.make_tiny()
    g = c["gauss"]
    rgb, occ, dep, at = gpu_bake(sop, g, c["probe_pos"], c["R"], t_stop=t_stop)
    o_rgb, o_occ, o_dep, fl, sens = orc.bake(g, c["probe_pos"], c["R"], t_stop=t_stop, with_sens=True)
    flagged = compare(orc, rgb, occ, dep, o_rgb, o_occ, o_dep, fl, sens, "tiny")
    assert flagged <= 0.01 * fl.size
    assert occ.max() > 0.5  # the shell occludes


@pytest.mark.parametrize("R", [2, 64])
def test_tiny_bake_resolution_limits(sop, orc, R):
    """The smallest and largest octahedral resolutions the library accepts:
    the whole tiny scene baked (64 probes), 4 probes checked at 64 x 64."""
    c = I.make_tiny()
    g = c["gauss"]
    rgb, occ, dep, at = gpu_bake(sop, g, c["probe_pos"], R)
    probes = np.arange(64) if R == 2 else np.array([0, 17, 38, 63])
    o_rgb, o_occ, o_dep, fl, sens = orc.bake(g, c["probe_pos"], R, probes=probes, with_sens=True)
    flagged = compare(orc, rgb[probes], occ[probes], dep[probes], o_rgb, o_occ, o_dep, fl, sens, f"tiny R={R}")
    assert flagged <= 0.01 * fl.size
    assert occ.max() > 0.5
    a = at.rgbo.cpu().numpy()
    for jj in (0, 1, R, R + 1):
        for ii in range(R + 2):
            si, sj = orc.oct_wrap(R, ii - 1, jj - 1)
            assert np.array_equal(a[:, jj, ii], a[:, sj + 1, si + 1])


def test_bake_gutter_matches_interior(sop, orc):
    c = I.make_tiny()
    _, _, _, at = gpu_bake(sop, c["gauss"], c["probe_pos"], c["R"])
    a = at.rgbo.cpu().numpy()
    R = c["R"]
    for jj in range(R + 2):
        for ii in range(R + 2):
            si, sj = orc.oct_wrap(R, ii - 1, jj - 1)
            assert np.array_equal(a[:, jj, ii], a[:, sj + 1, si + 1])


def test_empty_and_single_gaussian(sop, orc):
    pp = np.zeros((2, 3), np.float32)
    pp[1] = [0.3, -0.2, 0.1]
    empty = dict(mean=np.zeros((0, 3), np.float32), scale=np.zeros((0, 3), np.float32),
                 quat=np.zeros((0, 4), np.float32), opacity=np.zeros(0, np.float32), rgb=np.zeros((0, 3), np.float32))
    rgb, occ, dep, _ = gpu_bake(sop, empty, pp, 8)
    assert not rgb.any() and not occ.any() and not dep.any()
    d = orc.oct_decode(np.array([[3.5 / 8, 5.5 / 8]]))[0]
    one = dict(mean=np.array([0.7 * d], np.float32), scale=np.array([[0.03, 0.05, 0.02]], np.float32),
               quat=np.array([[0.9, 0.1, -0.3, 0.2]], np.float32), opacity=np.array([0.8], np.float32),
               rgb=np.array([[0.1, 0.5, 0.9]], np.float32))
    rgb, occ, dep, _ = gpu_bake(sop, one, pp, 8)
    o_rgb, o_occ, o_dep, fl, sens = orc.bake(one, pp, 8, with_sens=True)
    assert (occ > 0).sum() >= 1
    compare(orc, rgb, occ, dep, o_rgb, o_occ, o_dep, fl, sens, "single")


def test_object_full_bake_sampled(sop, orc):
    """Full 'object' bake (200k Gaussians, 4096 probes at 16x16, default
    T_stop) in the benchmark's launch configuration; 16 sampled probes
    (4096 texel rays) checked against the oracle."""
    c = I.make_object()
    g = c["gauss"]
    rgb, occ, dep, _ = gpu_bake(sop, g, c["probe_pos"], c["R"])
    probes = np.sort(np.random.default_rng(21).choice(len(c["probe_pos"]), 16, replace=False))
    o_rgb, o_occ, o_dep, fl, sens = orc.bake(g, c["probe_pos"], c["R"], probes=probes, with_sens=True)
    flagged = compare(orc, rgb[probes], occ[probes], dep[probes], o_rgb, o_occ, o_dep, fl, sens, "object")
    assert flagged <= 0.05 * fl.size


def test_compose_full_bake_sampled(sop, orc):
    """The 1080p composition's bake in the benchmark's launch configuration:
    all 8,192 probes (4,096 on the object, 4,096 shadow-region probes on the
    ground) in one call against the object's 200k Gaussians. Sampled: 8
    random object probes, the 4 ground probes nearest the object (most of
    their upper hemisphere sees it) and 4 random ground probes."""
    c = I.make_compose()
    g = c["gauss_object"]
    po, ps = c["shade"]["probe_pos"], c["shadow"]["probe_pos"]
    pp = np.concatenate([po, ps])
    rgb, occ, dep, _ = gpu_bake(sop, g, pp, c["R"])
    rng = np.random.default_rng(22)
    centre = g["mean"].astype(np.float64).mean(0)
    near = np.argsort(np.linalg.norm(ps - centre, axis=1), kind="stable")[:4]
    far = rng.choice(np.setdiff1d(np.arange(len(ps)), near), 4, replace=False)
    probes = np.sort(np.concatenate([rng.choice(len(po), 8, replace=False), len(po) + near, len(po) + far]))
    o_rgb, o_occ, o_dep, fl, sens = orc.bake(g, pp, c["R"], probes=probes, with_sens=True)
    # the nearest ground probes do see the object
    assert o_occ[8:].max() > 0.5
    flagged = compare(orc, rgb[probes], occ[probes], dep[probes], o_rgb, o_occ, o_dep, fl, sens, "compose",
                      extent=float(c["object_size"]))
    assert flagged <= 0.05 * fl.size


def test_bake_reproducible(sop):
    """Binning fills each grid cell in no fixed order (atomics), yet the bake
    is bit-identical from run to run: re-binned into a fresh workspace, and
    traced again through a workspace that last traced another probe set."""
    c = I.make_object()
    g = {k: cuda(v) for k, v in c["gauss"].items()}
    pp = cuda(c["probe_pos"][:512])
    a = sop.make_atlas(pp, 16)
    sop.bake(g, a, workspace=sop.BakeWorkspace(len(c["gauss"]["mean"]), "cuda"))
    ws = sop.BakeWorkspace(len(c["gauss"]["mean"]), "cuda")
    other = sop.make_atlas(cuda(c["probe_pos"][1000:1064]), 16)
    sop.bake(g, other, workspace=ws)
    b = sop.make_atlas(pp, 16)
    sop.bake_trace(g, b, ws)
    torch.cuda.synchronize()
    assert torch.equal(a.rgbo, b.rgbo) and torch.equal(a.depth, b.depth)


def test_work_counters_tiny(sop, orc):
    """With no early stop every hit is composited, so the composited count
    equals the number of (texel ray, Gaussian) pairs with alpha >= 1/255 and
    t* > 0, counted here by brute force in float64; each Gaussian is
    evaluated at most once per ray, so evaluations do not exceed the box
    tests and are at least the hits."""
    c = I.make_tiny()
    g, pp, R = c["gauss"], c["probe_pos"], c["R"]
    at = sop.make_atlas(cuda(pp), R)
    ws = sop.BakeWorkspace(len(g["mean"]), "cuda")
    sop.bake({k: cuda(v) for k, v in g.items()}, at, t_stop=0.0, workspace=ws)
    n_eval, n_comp, status, n_test = sop.bake_stats(ws)
    assert status == 0
    ii, jj = np.meshgrid(np.arange(R), np.arange(R), indexing="xy")
    uv = np.stack([(ii.reshape(-1) + 0.5) / R, (jj.reshape(-1) + 0.5) / R], 1)
    dirs = orc.oct_decode(uv)  # [R*R, 3]
    mu = g["mean"].astype(np.float64)
    s = g["scale"].astype(np.float64)
    q = g["quat"].astype(np.float64)
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w_, x_, y_, z_ = q.T
    rot = np.stack([np.stack([1 - 2 * (y_ * y_ + z_ * z_), 2 * (x_ * y_ - w_ * z_), 2 * (x_ * z_ + w_ * y_)], -1),
                    np.stack([2 * (x_ * y_ + w_ * z_), 1 - 2 * (x_ * x_ + z_ * z_), 2 * (y_ * z_ - w_ * x_)], -1),
                    np.stack([2 * (x_ * z_ - w_ * y_), 2 * (y_ * z_ + w_ * x_), 1 - 2 * (x_ * x_ + y_ * y_)], -1)],
                   1)
    M = np.transpose(rot, (0, 2, 1)) / s[:, :, None]  # diag(1/s) R^T
    op = g["opacity"].astype(np.float64)
    hits = border = 0
    for p in pp.astype(np.float64):
        u = np.einsum("gab,gb->ga", M, p[None, :] - mu)  # [G, 3]
        w = np.einsum("gab,tb->tga", M, dirs)  # [T, G, 3]
        A = (w * w).sum(-1)
        B = (w * u[None]).sum(-1)
        ts = -B / A
        m2 = (u * u).sum(-1)[None] - B * B / A
        resp = op[None] * np.exp(-0.5 * m2)
        hit = (ts > 0) & (resp >= 1.0 / 255.0)
        hits += int(hit.sum())
        border += int(((np.abs(resp * 255.0 - 1.0) < 1e-5) | (np.abs(ts) < 1e-6)).sum())
    assert abs(n_comp - hits) <= border, (n_comp, hits, border)
    assert n_comp <= n_eval <= n_test
    assert n_eval <= len(mu) * len(pp) * R * R
