"""GPU parity of the fixed-radius neighbour search (Sec. 3.2: at most K
nearest probes within a radius) through the query, the allocation-free
entry point and the adjoint, against the FP64 oracle, through the C ABI.
The probe selection is bit-exact, empty slots included (-1, weight 0)."""
import numpy as np
import pytest
import torch

from paper_2510_07729_gb300 import inputs as I
from tests.tolerance import assert_close

pytestmark = pytest.mark.gpu
KEYS = ("x", "n", "wo", "albedo", "rough", "metal")


@pytest.fixture(scope="module")
def sop():
    from paper_2510_07729_gb300 import sop as S
    S.load()
    return S


@pytest.fixture(scope="module")
def tiny():
    return I.make_tiny()


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def atlas(sop, pp, maps):
    at = sop.make_atlas(cuda(pp), maps["occ"].shape[1])
    sop.atlas_pack(cuda(maps["rgb"]), cuda(maps["occ"]), None, at)
    return at


def gpu(sop, pts, at, env, K, S, radius, mode=0, noalloc=False):
    f = sop.query_shade_noalloc if noalloc else sop.query_shade
    out = f(*[cuda(pts[k]) for k in KEYS], at, cuda(env), K, S, mode=mode, return_idx=True, radius=radius)
    torch.cuda.synchronize()
    return tuple(t.cpu().numpy() for t in out)


def orc_run(orc, pts, pp, maps, env, K, S, radius, mode=0):
    args = [pts[k] for k in KEYS] + [pp, maps["rgb"], maps["occ"], env, K, S]
    out, idx, W = orc.query_shade(*args, mode=mode, radius=radius)
    kap = orc.query_shade_sensitivity(*args, mode=mode, radius=radius)
    return out, idx, W, kap


def check(g, o, what):
    out, idx, w = g
    ro, ri, rw, kap = o
    assert np.array_equal(idx, ri), what  # bit-exact, -1 in the empty slots
    assert np.all(w[ri < 0] == 0.0), what
    assert_close(w, rw, what=what + " weights")
    assert_close(out, ro, what=what, absolute=kap)


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("K,radius", [(4, 0.2), (4, 0.3), (8, 0.35), (8, 0.5), (16, 0.4)])
def test_tiny_parity(sop, orc, tiny, K, radius, mode):
    c = tiny
    maps = I.synthetic_maps(np.random.default_rng(60 + K), 64, 8)
    at = atlas(sop, c["probe_pos"], maps)
    pts = {k: c[k] for k in KEYS}
    g = gpu(sop, pts, at, c["env"], K, 64, radius, mode)
    o = orc_run(orc, pts, c["probe_pos"], maps, c["env"], K, 64, radius, mode)
    cnt = (o[1] >= 0).sum(1)
    assert cnt.min() < K  # partial sets are exercised
    check(g, o, f"K={K} r={radius} mode={mode}")


def test_radius_holding_every_probe_is_bitwise_plain(sop, tiny):
    c = tiny
    maps = I.synthetic_maps(np.random.default_rng(61), 64, 8)
    at = atlas(sop, c["probe_pos"], maps)
    pts = {k: c[k] for k in KEYS}
    for mode in (0, 1):
        a = gpu(sop, pts, at, c["env"], 8, 64, 0.0, mode)
        b = gpu(sop, pts, at, c["env"], 8, 64, 100.0, mode)
        for u, v in zip(a, b):
            assert np.array_equal(u, v)


def test_no_probe_in_radius(sop, orc, tiny):
    c = tiny
    maps = I.synthetic_maps(np.random.default_rng(62), 64, 8)
    at = atlas(sop, c["probe_pos"], maps)
    pts = {k: c[k][:1000] for k in KEYS}
    for mode in (0, 1):
        g = gpu(sop, pts, at, c["env"], 4, 64, 1e-3, mode)
        assert np.all(g[1] == -1) and np.all(g[2] == 0.0)
        check(g, orc_run(orc, pts, c["probe_pos"], maps, c["env"], 4, 64, 1e-3, mode), f"empty mode={mode}")
        if mode == 1:
            assert np.all(g[0] == 1.0)


@pytest.mark.parametrize("M,K,S", [(1, 3, 37), (31, 32, 37), (4096 + 37, 3, 37), (4096 + 37, 32, 64)])
def test_ragged_sizes_and_K(sop, orc, tiny, M, K, S):
    c = tiny
    rng = np.random.default_rng(M + K)
    sel, pts = I.subsample(rng, {k: np.concatenate([c[k]] * 2) for k in KEYS}, list(KEYS), M)
    maps = I.synthetic_maps(rng, 64, 8)
    at = atlas(sop, c["probe_pos"], maps)
    g = gpu(sop, pts, at, c["env"], K, S, 0.45)
    check(g, orc_run(orc, pts, c["probe_pos"], maps, c["env"], K, S, 0.45), f"M={M} K={K}")


def test_noalloc_entry(sop, orc, tiny):
    c = tiny
    maps = I.synthetic_maps(np.random.default_rng(63), 64, 8)
    at = atlas(sop, c["probe_pos"], maps)
    pts = {k: c[k] for k in KEYS}
    for mode in (0, 1):
        g = gpu(sop, pts, at, c["env"], 8, 64, 0.35, mode, noalloc=True)
        check(g, orc_run(orc, pts, c["probe_pos"], maps, c["env"], 8, 64, 0.35, mode), f"noalloc mode={mode}")


def test_object_full_size_sampled(sop, orc):
    """The object workload (all points, K=8, S=128) in the query's launch
    configuration, with a radius at the median distance of the 4th nearest
    probe (so a point has anything from a few to 8 neighbours); 4096
    sampled points checked one by one."""
    c = I.make_object()
    rng = np.random.default_rng(64)
    s = rng.choice(len(c["x"]), 512, replace=False)
    d = np.linalg.norm(c["x"][s, None, :].astype(np.float64) - c["probe_pos"][None].astype(np.float64), axis=2)
    radius = float(np.float32(np.median(np.sort(d, axis=1)[:, 3])))
    maps = I.synthetic_maps(rng, len(c["probe_pos"]), 16)
    at = atlas(sop, c["probe_pos"], maps)
    out, idx, w = gpu(sop, {k: c[k] for k in KEYS}, at, c["env"], 8, 128, radius)
    sel, pts = I.subsample(np.random.default_rng(65), c, list(KEYS), 4096)
    o = orc_run(orc, pts, c["probe_pos"], maps, c["env"], 8, 128, radius)
    cnt = set((o[1] >= 0).sum(1).tolist())
    assert len(cnt) >= 5
    check((out[sel], idx[sel], w[sel]), o, "object")


def test_adjoint_with_partial_sets(sop, orc, tiny):
    """Smooth maps, tilted views, a radius that leaves points with 1 to 4
    of their K = 4 probes: every gradient as in the plain adjoint's smooth
    test (1e-4 relative, the per-term allowance of the FP32 directions,
    floors for the atomically summed env/probe gradients)."""
    c = tiny
    rng = np.random.default_rng(66)
    pts = {k: c[k] for k in KEYS}
    M = len(pts["n"])
    wo = pts["n"] + 0.4 * rng.standard_normal((M, 3)).astype(np.float32)
    wo /= np.linalg.norm(wo, axis=1, keepdims=True)
    pts["wo"] = np.where((np.sum(wo * pts["n"], 1) > 0.2)[:, None], wo, pts["n"]).astype(np.float32)
    maps = I.smooth_maps(rng, 64, 8)
    go = rng.standard_normal((M, 3))
    at = atlas(sop, c["probe_pos"], maps)
    radius = 0.35
    g = sop.query_shade_backward(*[cuda(pts[k]) for k in KEYS], at, cuda(c["env"]), 4, 64,
                                 cuda(go.astype(np.float32)), radius=radius)
    torch.cuda.synchronize()
    g = {k: v.cpu().numpy() for k, v in g.items()}
    o = orc.query_shade_grad(*[pts[k] for k in KEYS], c["probe_pos"], maps["rgb"], maps["occ"], c["env"], 4, 64,
                             go.astype(np.float32).astype(np.float64), radius=radius)
    idx, _ = orc.knn(pts["x"], c["probe_pos"], 4, radius=radius)
    assert len(set((idx >= 0).sum(1).tolist())) >= 3
    frac = 2e-4
    for k in ("albedo", "rough", "metal"):
        assert_close(g[k], o[k], rtol=1e-4, absolute=frac * o["abs_" + k], what=k)
    assert_close(g["normal"], o["normal"], rtol=1e-4, absolute=frac * o["abs_normal"][:, None], what="normal")
    assert_close(g["env"], o["env"], rtol=1e-4, floor=0, absolute=1e-6 * np.abs(o["env"]).max(), what="env")
    om = np.concatenate([o["maps_rgb"], o["maps_occ"][..., None]], axis=-1)
    assert_close(g["maps"], om, rtol=1e-4, floor=0, absolute=1e-6 * np.abs(om).max(), what="maps")
