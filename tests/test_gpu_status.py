"""The device status word (include/sop.h, sop_device_status) on the GPU:
non-finite inputs, a bake ray that cannot split its hits, out-of-range
indices and the device-side coarsening of the bake's grid are reported after
the fact, and the results stay defined. No test here faults or hangs the GPU:
each problem is a value the kernels check."""
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
    S.device_status(clear=True, raise_on_error=False)
    return S


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def bake(sop, g, probe_pos, R, workspace=None, **kw):
    at = sop.make_atlas(cuda(probe_pos), R)
    sop.bake({k: cuda(v) for k, v in g.items()}, at, workspace=workspace, **kw)
    rgb, occ, dep = at.interior()
    return rgb.cpu().numpy(), occ.cpu().numpy(), dep.cpu().numpy()


def test_clean_bake_and_query_leave_the_word_clear(sop):
    c = I.make_tiny()
    bake(sop, c["gauss"], c["probe_pos"], c["R"])
    assert sop.device_status() == 0


def test_nonfinite_gaussian_is_reported_and_left_out(sop):
    c = I.make_tiny()
    g = {k: v.copy() for k, v in c["gauss"].items()}
    bad = 17
    g["opacity"][bad] = np.nan
    rgb, occ, dep = bake(sop, g, c["probe_pos"], c["R"], t_stop=0.0)
    with pytest.raises(sop.SopError) as ei:
        sop.device_status()
    assert ei.value.status == 6 and "non-finite" in str(ei.value)
    assert sop.device_status() == 0  # cleared by the call that raised
    # the same bake without that Gaussian (indices keep their order)
    g2 = {k: np.delete(v, bad, axis=0) for k, v in c["gauss"].items()}
    rgb2, occ2, dep2 = bake(sop, g2, c["probe_pos"], c["R"], t_stop=0.0)
    assert sop.device_status() == 0
    assert np.isfinite(rgb).all() and np.isfinite(occ).all() and np.isfinite(dep).all()
    assert_close(occ, occ2, what="O without the NaN Gaussian")
    assert_close(rgb, rgb2, what="L_in without the NaN Gaussian")


def test_nonfinite_query_inputs_are_reported(sop):
    c = I.make_tiny()
    at = sop.make_atlas(cuda(c["probe_pos"]), c["R"])
    sop.bake({k: cuda(v) for k, v in c["gauss"].items()}, at)
    pts = {k: cuda(c[k]) for k in ("x", "n", "wo", "albedo", "rough", "metal")}
    env = cuda(c["env"])
    ref = sop.query_shade(*pts.values(), at, env, c["K"], c["S"]).cpu().numpy()
    assert sop.device_status() == 0
    for key, row in (("x", 5), ("albedo", 9), ("n", 11)):
        bad = {k: v.clone() for k, v in pts.items()}
        bad[key][row, 0] = float("nan")
        out = sop.query_shade(*bad.values(), at, env, c["K"], c["S"]).cpu().numpy()
        bits = sop.device_status(raise_on_error=False)
        assert bits & sop.DEVSTAT_NONFINITE, key
        keep = np.arange(len(ref)) != row
        assert np.array_equal(out[keep], ref[keep]), key  # other points untouched
    env_bad = env.clone()
    env_bad[3, 4, 1] = float("inf")
    sop.query_shade(*pts.values(), at, env_bad, c["K"], c["S"])
    assert sop.device_status(raise_on_error=False) & sop.DEVSTAT_NONFINITE
    maps = at.rgbo.clone()
    at.rgbo[7, 3, 3, 3] = float("nan")
    sop.query_shade(*pts.values(), at, env, c["K"], c["S"], mode=sop.MODE_SHADOW)
    assert sop.device_status(raise_on_error=False) & sop.DEVSTAT_NONFINITE
    at.rgbo.copy_(maps)


def test_bake_truncation_is_reported(sop):
    # 300 identical Gaussians straight ahead of one probe: their hits share
    # one t*, more than the 256-entry hit buffer, and no split of the window
    # separates them, so the ray stops (bounded: at most 40 halvings)
    n = 300
    g = dict(mean=np.tile(np.array([[0.0, 0.0, 0.5]], np.float32), (n, 1)),
             scale=np.full((n, 3), 0.1, np.float32),
             quat=np.tile(np.array([[1.0, 0.0, 0.0, 0.0]], np.float32), (n, 1)),
             opacity=np.full(n, 0.05, np.float32), rgb=np.full((n, 3), 0.5, np.float32))
    pp = np.zeros((1, 3), np.float32)
    rgb, occ, dep = bake(sop, g, pp, 8, t_stop=0.0)
    bits = sop.device_status(raise_on_error=False)
    assert bits & sop.DEVSTAT_BAKE_TRUNCATED
    assert np.isfinite(occ).all() and np.isfinite(rgb).all()
    # the texels looking away from the Gaussians are not affected
    assert occ.min() == 0.0


def test_grid_coarsened_on_the_device_gives_the_same_bake(sop, orc):
    # 20,000 Gaussians whose boxes each span 2-3 cells of the default grid:
    # the requested grid's lists (about 770k entries) overflow the minimum
    # workspace (24 per Gaussian + 65,536 = 546k), and the device falls back
    # to the grid with 1/16 of the cells (about 146k entries; information
    # bit, not an error). At most about 95 boxes overlap at any point, so no
    # ray has more hits waiting than its 256-entry buffer holds.
    rng = np.random.default_rng(7)
    n = 20000
    s = np.exp(rng.uniform(np.log(0.02), np.log(0.035), n))
    g = dict(mean=rng.uniform(-0.5, 0.5, (n, 3)).astype(np.float32),
             scale=np.repeat(s[:, None], 3, axis=1).astype(np.float32),
             quat=rng.standard_normal((n, 4)).astype(np.float32),
             opacity=rng.uniform(0.05, 0.3, n).astype(np.float32),
             rgb=rng.uniform(0, 1, (n, 3)).astype(np.float32))
    # probes outside every box, looking in
    v = rng.standard_normal((6, 3))
    pp = (2.0 * v / np.linalg.norm(v, axis=1, keepdims=True)).astype(np.float32)
    R = 8
    ws = sop.BakeWorkspace(n, "cuda")
    rgb, occ, dep = bake(sop, g, pp, R, workspace=ws, t_stop=0.0)
    bits = sop.device_status()  # information only: no exception
    assert bits & sop.DEVSTAT_GRID_COARSENED
    big = sop.BakeWorkspace(n, "cuda", extra_bytes=16 * 1_000_000)
    rgb2, occ2, dep2 = bake(sop, g, pp, R, workspace=big, t_stop=0.0)
    assert not sop.device_status() & sop.DEVSTAT_GRID_COARSENED
    assert occ.max() > 0.5  # the rays cross the cloud
    assert_close(occ, occ2, what="O, coarsened grid")
    assert_close(rgb, rgb2, what="L_in, coarsened grid")
    o_rgb, o_occ, o_dep, fl = orc.bake(g, pp, R, t_stop=0.0)
    ok = (fl & (orc.FLAG_ALPHA_MIN | orc.FLAG_TNEAR | orc.FLAG_TSTOP)) == 0
    assert_close(occ[ok], o_occ[ok], what="O, coarsened grid vs oracle")


def test_out_of_range_pixel_index_is_reported(sop):
    n = 64
    sg = torch.rand((n, 16), device="cuda")
    og = torch.rand((n, 16), device="cuda")
    sc_pix = torch.tensor([0, 5, n + 3], dtype=torch.int64, device="cuda")
    shadow = torch.rand((3, 3), device="cuda")
    ob_pix = torch.tensor([1, -2], dtype=torch.int64, device="cuda")
    rgb = torch.rand((2, 3), device="cuda")
    out = sop.depth_composite(sg, og, sc_pix, shadow, ob_pix, rgb)
    assert sop.device_status(raise_on_error=False) & sop.DEVSTAT_INDEX
    assert torch.isfinite(out).all()
