"""Pins of the oracle's octahedral map, border rule and bilinear fetch
(Sec. 3.1.2 octahedral textures; mapping of Cigolle et al. 2014; border rule
of Majercik et al. 2019). Each pin is a property fixed by the geometry of the
map, not a retyped formula."""
import numpy as np
import pytest


def centres(R):
    jj, ii = np.meshgrid(np.arange(R), np.arange(R), indexing="ij")
    return np.stack([(ii.ravel() + 0.5) / R, (jj.ravel() + 0.5) / R], axis=1)


@pytest.mark.parametrize("R", [4, 8, 16, 32])
def test_round_trip_exact_on_l1_octahedron(orc, R):
    uv = centres(R)
    d = orc.oct_decode(uv, l1_only=True)
    assert np.allclose(np.abs(d).sum(1), 1.0, rtol=0, atol=0)
    assert np.array_equal(orc.oct_encode(d), uv)  # dyadic texel centres: bit-exact


@pytest.mark.parametrize("R", [8, 16])
def test_round_trip_normalised(orc, R):
    uv = centres(R)
    back = orc.oct_encode(orc.oct_decode(uv))
    assert np.max(np.abs(back - uv)) < 8 * np.finfo(float).eps
    assert np.array_equal(np.floor(back * R), np.floor(uv * R))


def test_decode_unit_norm_and_encode_range(orc):
    rng = np.random.default_rng(0)
    uv = rng.random((20000, 2))
    d = orc.oct_decode(uv)
    assert np.max(np.abs(np.linalg.norm(d, axis=1) - 1.0)) < 1e-15
    v = rng.standard_normal((20000, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    e = orc.oct_encode(v)
    assert e.min() >= 0 and e.max() <= 1
    # encode is a bijection sphere -> square: decode(encode(v)) == v
    assert np.max(np.abs(orc.oct_decode(e) - v)) < 1e-14


def test_hemispheres_and_axes(orc):
    # +z maps to the square centre, -z to the four corners, the equator to
    # the inscribed diamond |2u-1| + |2v-1| = 1
    assert np.allclose(orc.oct_encode([0, 0, 1]), [[0.5, 0.5]])
    for c in [(0, 0), (1, 0), (0, 1), (1, 1)]:
        assert np.allclose(orc.oct_decode(np.array([c], float)), [[0, 0, -1]])
    rng = np.random.default_rng(1)
    ph = rng.uniform(-np.pi, np.pi, 1000)
    e = orc.oct_encode(np.stack([np.cos(ph), np.sin(ph), np.zeros_like(ph)], 1))
    assert np.allclose(np.abs(2 * e[:, 0] - 1) + np.abs(2 * e[:, 1] - 1), 1.0, atol=1e-15)


def test_decode_continuous_across_square_edges(orc):
    # the square's border folds onto itself: (0,v)~(0,1-v), (1,v)~(1,1-v),
    # (u,0)~(1-u,0), (u,1)~(1-u,1)
    rng = np.random.default_rng(2)
    t = rng.random(500)
    z, o = np.zeros_like(t), np.ones_like(t)
    for a, b in [((z, t), (z, 1 - t)), ((o, t), (o, 1 - t)), ((t, z), (1 - t, z)), ((t, o), (1 - t, o))]:
        da = orc.oct_decode(np.stack(a, 1))
        db = orc.oct_decode(np.stack(b, 1))
        assert np.max(np.abs(da - db)) < 1e-15


@pytest.mark.parametrize("R", [8, 16])
def test_wrap_maps_border_ring_onto_map(orc, R):
    for i in range(-1, R + 1):
        for j in range(-1, R + 1):
            si, sj = orc.oct_wrap(R, i, j)
            assert 0 <= si < R and 0 <= sj < R
            if 0 <= i < R and 0 <= j < R:
                assert (si, sj) == (i, j)


@pytest.mark.parametrize("R", [8, 16])
def test_wrap_is_the_geometric_neighbour(orc, R):
    # the texel standing in for a virtual neighbour across an edge is the one
    # whose centre is nearest (on the sphere) to where that neighbour would be
    for j in range(R):
        edge = np.array([[0.0, (j + 0.5) / R]])           # left edge point
        de = orc.oct_decode(edge)[0]
        cand = orc.oct_decode(centres(R))
        dist = np.arccos(np.clip(cand @ de, -1, 1))
        # interior texel (0, j) and the mirrored texel are the two nearest
        si, sj = orc.oct_wrap(R, -1, j)
        nearest = set(np.argsort(dist)[:2].tolist())
        assert {j * R + 0, sj * R + si} == nearest or np.isclose(
            dist[j * R], dist[sj * R + si])


def test_bilerp_at_centres_returns_texel(orc):
    rng = np.random.default_rng(3)
    R = 8
    m = rng.random((R, R, 4))
    out = orc.oct_bilerp(m, centres(R))
    assert np.array_equal(out, m.reshape(-1, 4))


def test_bilerp_continuous_across_seams(orc):
    rng = np.random.default_rng(4)
    R = 16
    m = rng.random((R, R, 3))
    t = rng.random(300)
    z, o = np.zeros_like(t), np.ones_like(t)
    for a, b in [((z, t), (z, 1 - t)), ((o, t), (o, 1 - t)), ((t, z), (1 - t, z)), ((t, o), (1 - t, o))]:
        va = orc.oct_bilerp(m, np.stack(a, 1))
        vb = orc.oct_bilerp(m, np.stack(b, 1))
        assert np.max(np.abs(va - vb)) < 1e-14
    # all four corners are the -z pole
    c = orc.oct_bilerp(m, np.array([[0, 0], [1, 0], [0, 1], [1, 1.0]]))
    assert np.max(np.abs(c - c[0])) < 1e-14
    # and just inside the corners the value approaches the corner value
    eps = 1e-9
    ci = orc.oct_bilerp(m, np.array([[eps, eps], [1 - eps, eps], [eps, 1 - eps], [1 - eps, 1 - eps]]))
    assert np.max(np.abs(ci - c[0])) < 1e-6


def test_bilerp_constant_and_linear_reproduction(orc):
    R = 8
    m = np.full((R, R, 2), 0.37)
    rng = np.random.default_rng(5)
    uv = rng.random((1000, 2))
    assert np.allclose(orc.oct_bilerp(m, uv), 0.37, rtol=0, atol=1e-15)
    # away from the border a map linear in the texel index is reproduced
    jj, ii = np.meshgrid(np.arange(R), np.arange(R), indexing="ij")
    lin = np.stack([ii, jj], -1).astype(float)
    uv = rng.uniform(0.5 / R, 1 - 0.5 / R, (1000, 2))
    assert np.allclose(orc.oct_bilerp(lin, uv), uv * R - 0.5, atol=1e-13)
