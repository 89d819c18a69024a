"""Pins of the oracle's hand-written adjoint of query/shade (SHADE mode)
against FP64 central finite differences of the oracle's own forward pass."""
import numpy as np
import pytest

from paper_2510_07729_gb300 import inputs as I

M = 48


@pytest.fixture(scope="module")
def case():
    c = I.make_tiny()
    rng = np.random.default_rng(31)
    maps = I.synthetic_maps(rng, 64, 8)
    env = I.env_lognormal(rng, 16, 32)
    pts = {k: np.ascontiguousarray(c[k][:M]) for k in ("x", "n", "wo", "albedo", "rough", "metal")}
    # tilt the view direction off the normal so every BRDF term is exercised
    wo = pts["n"] + 0.4 * rng.standard_normal((M, 3)).astype(np.float32)
    pts["wo"] = (wo / np.linalg.norm(wo, axis=1, keepdims=True)).astype(np.float32)
    pts["wo"] = np.where((np.sum(pts["wo"] * pts["n"], 1) > 0.2)[:, None], pts["wo"], pts["n"]).astype(np.float32)
    go = rng.standard_normal((M, 3))
    return dict(c=c, maps=maps, env=env, pts=pts, go=go, K=4, S=32)


def loss(orc, case, **over):
    p = dict(case["pts"])
    maps = dict(case["maps"])
    env = case["env"]
    for k, v in over.items():
        if k in p:
            p[k] = v
        elif k == "env":
            env = v
        else:
            maps[k] = v
    out, _, _ = orc.query_shade(p["x"], p["n"], p["wo"], p["albedo"], p["rough"], p["metal"], case["c"]["probe_pos"],
                                maps["rgb"], maps["occ"], env, case["K"], case["S"])
    return np.sum(out * case["go"], axis=1)


def grads(orc, case):
    p = case["pts"]
    return orc.query_shade_grad(p["x"], p["n"], p["wo"], p["albedo"], p["rough"], p["metal"], case["c"]["probe_pos"],
                                case["maps"]["rgb"], case["maps"]["occ"], case["env"], case["K"], case["S"],
                                case["go"])


def fd_per_point(orc, case, name, comp, h):
    """Central differences of each point's loss term w.r.t. one component;
    inputs are float32, so the perturbation is applied in float64 via a
    float64 copy rounded back only where it is exact (h is a power of 2)."""
    base = case["pts"][name].astype(np.float64)
    up, dn = base.copy(), base.copy()
    if base.ndim == 1:
        up += h
        dn -= h
    else:
        up[:, comp] += h
        dn[:, comp] -= h
    # keep the float32 path exact: the oracle reads float32 inputs
    assert np.array_equal(up.astype(np.float32).astype(np.float64), up)
    lu = loss(orc, case, **{name: up.astype(np.float32)})
    ld = loss(orc, case, **{name: dn.astype(np.float32)})
    return (lu - ld) / (up - dn).reshape(len(base), -1)[:, comp if base.ndim > 1 else 0]


@pytest.mark.parametrize("name,comps", [("albedo", [0, 1, 2]), ("rough", [0]), ("metal", [0])])
def test_material_grads_match_fd(orc, case, name, comps):
    g = grads(orc, case)[name]
    for comp in comps:
        # snap inputs to a multiple of h so that +-h is exact in float32
        h = 2.0 ** -12
        fd = fd_per_point(orc, dict(case, pts=dict(case["pts"], **{name: snap(case["pts"][name], h)})), name, comp, h)
        gg = grads(orc, dict(case, pts=dict(case["pts"], **{name: snap(case["pts"][name], h)})))[name]
        an = gg[:, comp] if gg.ndim > 1 else gg
        scale = np.abs(an).max()
        # the loss is smooth in the materials: O(h^2) difference error
        assert np.max(np.abs(fd - an)) < 1e-5 * scale, (name, comp)


def snap(a, h):
    return (np.round(a.astype(np.float64) / h) * h).astype(np.float32)


def test_normal_grad_matches_fd(orc, case):
    """Finite differences in the normal move every light direction, so they
    cross texel edges (bilinear kinks); points where two step sizes disagree
    are excluded, the rest must match."""
    h = 2.0 ** -16
    n = snap(case["pts"]["n"], h)
    cs = dict(case, pts=dict(case["pts"], n=n))
    g = grads(orc, cs)["normal"]
    ok_all = np.ones(M, bool)
    fds = []
    for comp in range(3):
        f1 = fd_per_point(orc, cs, "n", comp, h)
        f2 = fd_per_point(orc, cs, "n", comp, h / 4)
        scale = np.abs(g).max()
        ok = np.abs(f1 - f2) < 1e-4 * scale
        ok_all &= ok
        fds.append(f2)
    fd = np.stack(fds, 1)
    assert ok_all.sum() >= M // 2, "too many points at kinks"
    err = np.abs(fd - g)[ok_all]
    assert np.max(err) < 2e-3 * np.abs(g).max()


def test_env_and_map_grads_exact_by_linearity(orc, case):
    """The output is linear in environment and probe-map texels: a central
    difference of any size gives the derivative up to rounding."""
    g = grads(orc, case)
    rng = np.random.default_rng(5)
    He, We, _ = case["env"].shape
    for _ in range(12):
        r, c, ch = rng.integers(He), rng.integers(We), rng.integers(3)
        e1, e2 = case["env"].copy(), case["env"].copy()
        e1[r, c, ch] += 0.5
        e2[r, c, ch] -= 0.5
        dh = float(e1[r, c, ch]) - float(e2[r, c, ch])  # the float32 step actually taken
        fd = (loss(orc, case, env=e1).sum() - loss(orc, case, env=e2).sum()) / dh
        assert fd == pytest.approx(g["env"][r, c, ch], rel=1e-9, abs=1e-12)
    # texels actually read by the points (their nearest probes)
    idx, _ = orc.knn(case["pts"]["x"], case["c"]["probe_pos"], case["K"])
    for _ in range(12):
        p = int(rng.choice(idx.ravel()))
        i, j = rng.integers(8), rng.integers(8)
        for ch in range(4):
            m1, m2 = dict(case["maps"]), dict(case["maps"])
            key = "occ" if ch == 3 else "rgb"
            a1, a2 = case["maps"][key].copy(), case["maps"][key].copy()
            ix = (p, j, i) if ch == 3 else (p, j, i, ch)
            a1[ix] += 0.25
            a2[ix] -= 0.25
            want = g["maps_occ"][ix] if ch == 3 else g["maps_rgb"][ix]
            dh = float(a1[ix]) - float(a2[ix])
            fd = (loss(orc, case, **{key: a1}).sum() - loss(orc, case, **{key: a2}).sum()) / dh
            assert fd == pytest.approx(want, rel=1e-9, abs=1e-12)
