"""Pins of the oracle's fixed-radius neighbour search (Sec. 3.2: the probes
N(x) of a shading point come from a fixed-radius nearest-neighbour search,
at most K of them, the nearest first): brute force with exact rational
arithmetic, the inclusive boundary, the two limits (a radius that holds
every probe is the plain K nearest; one that holds none leaves the
environment term alone), the reduction of a partial set to the plain K
nearest of its size, and the adjoint with partial sets against finite
differences."""
from fractions import Fraction

import numpy as np
import pytest

from paper_2510_07729_gb300 import inputs as I


@pytest.fixture(scope="module")
def tiny():
    return I.make_tiny()


def q(v):
    """Quantised coordinate: round half to even of v 2^20 (exact in double)."""
    return int(np.rint(np.float64(v) * 1048576.0))


def brute_frnn(x, pp, K, radius):
    r = Fraction(float(np.float32(radius))) * 1048576
    out = []
    for m in range(len(x)):
        qx = [q(x[m, a]) for a in range(3)]
        cand = []
        for p in range(len(pp)):
            key = sum((q(pp[p, a]) - qx[a]) ** 2 for a in range(3))
            if radius == 0 or key <= r * r:
                cand.append((key, p))
        cand.sort()
        ids = [p for _, p in cand[:K]]
        out.append(ids + [-1] * (K - len(ids)))
    return np.array(out, np.int32)


@pytest.mark.parametrize("K,radius", [(4, 0.2), (4, 0.3), (8, 0.35), (8, 0.5), (4, 0.0)])
def test_knn_radius_brute_force(orc, tiny, K, radius):
    x, pp = tiny["x"][:150], tiny["probe_pos"]
    idx, key = orc.knn(x, pp, K, radius=radius)
    want = brute_frnn(x, pp, K, radius)
    assert np.array_equal(idx, want)
    assert np.all(key[idx < 0] == np.uint64(2**64 - 1))
    if radius in (0.2, 0.3):  # partial sets of several sizes, empty ones at 0.2
        cnt = set((want >= 0).sum(1).tolist())
        assert len(cnt) >= 2 and (radius != 0.2 or 0 in cnt)


def test_radius_boundary_is_inclusive(orc):
    # dyadic positions: quantised distance exactly 2^18 = 0.25 2^20
    x = np.zeros((1, 3), np.float32)
    pp = np.array([[0.25, 0, 0], [0, 0.5, 0]], np.float32)
    idx, _ = orc.knn(x, pp, 2, radius=0.25)
    assert idx.tolist() == [[0, -1]]
    below = np.nextafter(np.float32(0.25), np.float32(0))
    idx, _ = orc.knn(x, pp, 2, radius=below)
    assert idx.tolist() == [[-1, -1]]
    idx, _ = orc.knn(x, pp, 2, radius=0.5)
    assert idx.tolist() == [[0, 1]]


def _shade(orc, tiny, maps, env, K, S, radius, mode=None, M=256, **kw):
    c = tiny
    sl = slice(0, M)
    args = (c["x"][sl], c["n"][sl], c["wo"][sl], kw.pop("albedo", c["albedo"][sl]), kw.pop("rough", c["rough"][sl]),
            kw.pop("metal", c["metal"][sl]), c["probe_pos"], maps["rgb"], maps["occ"], env, K, S)
    if mode is not None:
        kw["mode"] = mode
    return orc.query_shade(*args, radius=radius, **kw)


def test_radius_holding_every_probe_is_plain_knn(orc, tiny):
    rng = np.random.default_rng(3)
    maps = I.synthetic_maps(rng, 64, 8)
    env = I.env_lognormal(rng, 16, 32)
    for mode in (orc.MODE_SHADE, orc.MODE_SHADOW):
        a = _shade(orc, tiny, maps, env, 4, 32, 0.0, mode)
        b = _shade(orc, tiny, maps, env, 4, 32, 4.0, mode)
        for u, v in zip(a, b):
            assert np.array_equal(u, v)


def test_no_probe_in_radius_leaves_the_environment_alone(orc, tiny):
    """No neighbour: O = 0 and L_in = 0. Under a constant environment L the
    centred Hammersley set integrates the diffuse term (a/pi) L cos exactly
    to a L, whatever the (random) probe maps hold; with metal 0 the
    specular term does not depend on the albedo, so C(a) - C(0) is that
    diffuse part. The shadow ratio is 1."""
    rng = np.random.default_rng(4)
    maps = I.synthetic_maps(rng, 64, 8)
    L = np.array([0.7, 1.3, 2.1], np.float32)
    env = np.broadcast_to(L, (16, 32, 3)).copy()
    M = 128
    a = tiny["albedo"][:M]
    z = np.zeros(M, np.float32)
    out, idx, W = _shade(orc, tiny, maps, env, 4, 64, 1e-3, orc.MODE_SHADE, M=M, albedo=a, metal=z)
    o0, _, _ = _shade(orc, tiny, maps, env, 4, 64, 1e-3, orc.MODE_SHADE, M=M, albedo=0 * a, metal=z)
    assert np.all(idx == -1) and np.all(W == 0.0)
    np.testing.assert_allclose(out - o0, a.astype(np.float64) * L, rtol=1e-12)
    out, _, _ = _shade(orc, tiny, maps, env, 4, 64, 1e-3, orc.MODE_SHADOW, M=M)
    assert np.all(out == 1.0)


def test_single_probe_in_radius_is_that_probes_map(orc, tiny):
    """One neighbour: W = 1 on it. Constant maps per probe (O = c_p,
    L_in = e_p) and the same diffuse part give a (L (1 - c_k) + e_k)."""
    rng = np.random.default_rng(5)
    P, R = len(tiny["probe_pos"]), 8
    c = rng.uniform(0.1, 0.9, P).astype(np.float32)
    e = rng.uniform(0.0, 1.0, (P, 3)).astype(np.float32)
    maps = dict(occ=np.broadcast_to(c[:, None, None], (P, R, R)).copy(),
                rgb=np.broadcast_to(e[:, None, None, :], (P, R, R, 3)).copy())
    L = np.array([0.9, 1.1, 1.6], np.float32)
    env = np.broadcast_to(L, (16, 32, 3)).copy()
    M = 256
    a = tiny["albedo"][:M]
    z = np.zeros(M, np.float32)
    out, idx, W = _shade(orc, tiny, maps, env, 4, 64, 0.2, orc.MODE_SHADE, M=M, albedo=a, metal=z)
    o0, _, _ = _shade(orc, tiny, maps, env, 4, 64, 0.2, orc.MODE_SHADE, M=M, albedo=0 * a, metal=z)
    out = out - o0
    one = (idx >= 0).sum(1) == 1
    assert one.sum() > M // 3
    k = idx[one, 0]
    assert np.all(W[one, 0] == 1.0) and np.all(W[one, 1:] == 0.0)
    want = a[one].astype(np.float64) * (L * (1.0 - c[k, None].astype(np.float64)) + e[k])
    np.testing.assert_allclose(out[one], want, rtol=1e-12)


def test_partial_set_is_the_plain_knn_of_its_size(orc, tiny):
    """A point with n < K probes in the radius gets the weights, and the
    shading, of the plain n nearest (the in-radius probes are the n nearest):
    the empty slots are neither weighted nor normalised over."""
    rng = np.random.default_rng(6)
    maps = I.synthetic_maps(rng, 64, 8)
    env = I.env_lognormal(rng, 16, 32)
    M, K = 256, 4
    for mode in (orc.MODE_SHADE, orc.MODE_SHADOW):
        out, idx, W = _shade(orc, tiny, maps, env, K, 32, 0.3, mode, M=M)
        cnt = (idx >= 0).sum(1)
        for n in (1, 2, 3):
            sel = cnt == n
            assert sel.sum() > 0 or n == 3
            if not sel.any():
                continue
            o2, i2, w2 = _shade(orc, tiny, maps, env, n, 32, 0.0, mode, M=M)
            assert np.array_equal(idx[sel, :n], i2[sel])
            assert np.array_equal(W[sel, :n], w2[sel]) and np.all(W[sel, n:] == 0.0)
            assert np.array_equal(out[sel], o2[sel])


# ---- adjoint with partial neighbour sets ------------------------------------
@pytest.fixture(scope="module", params=[0.2, 0.35])
def gcase(tiny, request):
    rng = np.random.default_rng(32)
    M = 48
    maps = I.synthetic_maps(rng, 64, 8)
    env = I.env_lognormal(rng, 16, 32)
    pts = {k: np.ascontiguousarray(tiny[k][:M]) for k in ("x", "n", "wo", "albedo", "rough", "metal")}
    return dict(c=tiny, maps=maps, env=env, pts=pts, go=rng.standard_normal((M, 3)), K=4, S=32, radius=request.param,
                M=M)


def _loss(orc, cs, n=None, maps=None):
    p = cs["pts"]
    mp = maps or cs["maps"]
    out, _, _ = orc.query_shade(p["x"], p["n"] if n is None else n, p["wo"], p["albedo"], p["rough"], p["metal"],
                                cs["c"]["probe_pos"], mp["rgb"], mp["occ"], cs["env"], cs["K"], cs["S"],
                                radius=cs["radius"])
    return np.sum(out * cs["go"], axis=1)


def _grads(orc, cs, n=None):
    p = cs["pts"]
    return orc.query_shade_grad(p["x"], p["n"] if n is None else n, p["wo"], p["albedo"], p["rough"], p["metal"],
                                cs["c"]["probe_pos"], cs["maps"]["rgb"], cs["maps"]["occ"], cs["env"], cs["K"],
                                cs["S"], cs["go"], radius=cs["radius"])


def test_grad_with_partial_sets_matches_fd(orc, gcase):
    """Normal (through the weights of the in-radius probes only) by central
    differences at two step sizes, kinks excluded as in the plain case."""
    idx, _ = orc.knn(gcase["pts"]["x"], gcase["c"]["probe_pos"], gcase["K"], radius=gcase["radius"])
    cnt = set((idx >= 0).sum(1).tolist())
    # 0.2: empty and single sets; 0.35: one to three probes
    assert (0 in cnt) if gcase["radius"] == 0.2 else len(cnt) >= 3
    h = 2.0 ** -16
    n = (np.round(gcase["pts"]["n"].astype(np.float64) / h) * h).astype(np.float32)
    g = _grads(orc, gcase, n)["normal"]
    M = gcase["M"]
    ok_all, fds = np.ones(M, bool), []
    for comp in range(3):
        f = []
        for hh in (h, h / 4):
            up, dn = n.astype(np.float64), n.astype(np.float64)
            up[:, comp] += hh
            dn[:, comp] -= hh
            f.append((_loss(orc, gcase, up.astype(np.float32)) - _loss(orc, gcase, dn.astype(np.float32))) / (2 * hh))
        ok_all &= np.abs(f[0] - f[1]) < 1e-4 * np.abs(g).max()
        fds.append(f[1])
    fd = np.stack(fds, 1)
    assert ok_all.sum() >= M // 2
    assert np.max(np.abs(fd - g)[ok_all]) < 2e-3 * np.abs(g).max()


def test_map_grads_with_partial_sets_exact_by_linearity(orc, gcase):
    g = _grads(orc, gcase)
    idx, _ = orc.knn(gcase["pts"]["x"], gcase["c"]["probe_pos"], gcase["K"], radius=gcase["radius"])
    rng = np.random.default_rng(7)
    used = np.unique(idx[idx >= 0])
    unused = np.setdiff1d(np.arange(len(gcase["c"]["probe_pos"])), used)
    # probes outside every point's radius get no gradient
    assert np.all(g["maps_occ"][unused] == 0.0) and np.all(g["maps_rgb"][unused] == 0.0)
    for _ in range(10):
        p = int(rng.choice(used))
        i, j = rng.integers(8), rng.integers(8)
        a1, a2 = gcase["maps"]["occ"].copy(), gcase["maps"]["occ"].copy()
        a1[p, j, i] += 0.25
        a2[p, j, i] -= 0.25
        dh = float(a1[p, j, i]) - float(a2[p, j, i])
        m1, m2 = dict(gcase["maps"], occ=a1), dict(gcase["maps"], occ=a2)
        fd = (_loss(orc, gcase, maps=m1).sum() - _loss(orc, gcase, maps=m2).sum()) / dh
        assert fd == pytest.approx(g["maps_occ"][p, j, i], rel=1e-9, abs=1e-12)
