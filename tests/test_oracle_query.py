"""Pins of the oracle's probe query (Sec. 3.1.2, Eq. 4-6), light directions,
frame, environment lookup and BRDF (Eq. 2-3), and shadow ratio (Eq. 7-9)."""
import numpy as np
import pytest
from scipy.spatial import cKDTree

from paper_2510_07729_gb300 import inputs as I


def test_knn_matches_kdtree(orc):
    rng = np.random.default_rng(0)
    P, M, K = 500, 2000, 8
    pp = rng.uniform(-1, 1, (P, 3)).astype(np.float32)
    x = rng.uniform(-1, 1, (M, 3)).astype(np.float32)
    idx, key = orc.knn(x, pp, K)
    q = np.rint(pp.astype(np.float64) * 2 ** 20)
    qx = np.rint(x.astype(np.float64) * 2 ** 20)
    _, ref = cKDTree(q).query(qx, k=K)
    assert np.array_equal(idx, ref)
    assert np.all(np.diff(key.astype(np.float64), axis=1) >= 0)


def test_knn_ties_go_to_lower_index(orc):
    pp = np.array([[1, 0, 0], [0, 1, 0], [-1, 0, 0], [0, -1, 0], [0, 0, 1]], np.float32)
    x = np.zeros((1, 3), np.float32)
    idx, key = orc.knn(x, pp, 3)
    assert idx.tolist() == [[0, 1, 2]]
    assert key.tolist() == [[2 ** 40] * 3]
    # duplicated probe positions: the lower index first
    pp2 = np.array([[0.5, 0, 0], [0.1, 0, 0], [0.5, 0, 0], [0.1, 0, 0]], np.float32)
    idx, _ = orc.knn(x, pp2, 4)
    assert idx.tolist() == [[1, 3, 0, 2]]


def test_weights_sum_to_one_and_k1(orc):
    c = I.make_tiny()
    idx, key = orc.knn(c["x"], c["probe_pos"], 4)
    W = orc.weights(c["x"], c["n"], c["probe_pos"], idx, key)
    assert np.allclose(W.sum(1), 1.0, atol=1e-14)
    assert np.all(W > 0)
    idx1, key1 = orc.knn(c["x"], c["probe_pos"], 1)
    assert np.array_equal(orc.weights(c["x"], c["n"], c["probe_pos"], idx1, key1), np.ones((4096, 1)))


def test_weights_worked_example(orc):
    # probe A one unit along the normal, probe B two units against it:
    # w_s = (1, 1/2), w_b = (0.5*(1+1)+0.01, 0.5*(1-1)+0.01) = (1.01, 0.01)
    x = np.zeros((1, 3), np.float32)
    n = np.array([[0, 0, 1]], np.float32)
    pp = np.array([[0, 0, 1], [0, 0, -2]], np.float32)
    idx, key = orc.knn(x, pp, 2)
    W = orc.weights(x, n, pp, idx, key)
    assert np.allclose(W, [[1.01 / 1.015, 0.005 / 1.015]], rtol=1e-15)
    # unnormalised normal gives the same weights
    assert np.allclose(orc.weights(x, n * 3, pp, idx, key), W, rtol=1e-15)
    # perpendicular probe: w_b = 0.51
    pp = np.array([[1, 0, 0], [0, 0, 2]], np.float32)
    idx, key = orc.knn(x, pp, 2)
    W = orc.weights(x, n, pp, idx, key)
    assert np.allclose(W, [[0.51 / (0.51 + 0.505), 0.505 / (0.51 + 0.505)]], rtol=1e-15)


def test_snap_reproduces_probe_map(orc):
    c = I.make_tiny()
    rng = np.random.default_rng(1)
    maps = I.synthetic_maps(rng, 64, 8)
    k = np.array([3, 17, 40])
    x = c["probe_pos"][k]
    nrm = c["probe_nrm"][k]
    mat = {kk: c[kk][:3] for kk in ("albedo", "rough", "metal")}
    args = dict(wo=nrm, **mat, maps_rgb=maps["rgb"], maps_occ=maps["occ"], env=c["env"], S=64)
    full, idx, W = orc.query_shade(x, nrm, probe_pos=c["probe_pos"], K=4, **args)
    assert np.array_equal(W, np.eye(4)[[0, 0, 0]])
    assert idx[:, 0].tolist() == k.tolist()
    one, _, _ = orc.query_shade(x, nrm, probe_pos=c["probe_pos"][k[:, None]][:, 0] * 0 + c["probe_pos"][k],
                                K=1, **{**args, "maps_rgb": maps["rgb"][k], "maps_occ": maps["occ"][k]})
    assert np.allclose(full, one, rtol=1e-14, atol=0)


def test_hammersley_set(orc):
    for S in (16, 64, 128, 256):
        d = orc.hammersley(S)
        assert np.allclose(np.linalg.norm(d, axis=1), 1, atol=1e-15)
        assert np.all(d[:, 2] > 0)
        assert abs(d[:, 2].mean() - 0.5) < 1e-15  # centred strata
        assert np.allclose(np.sort(d[:, 2]), (np.arange(S) + 0.5) / S)
    # azimuths are 2 pi times the base-2 radical inverse of the index
    d = orc.hammersley(8)
    phi = np.mod(np.arctan2(d[:, 1], d[:, 0]), 2 * np.pi) / (2 * np.pi)
    phi[np.isclose(phi, 1.0)] = 0.0
    assert np.allclose(phi, [0, 0.5, 0.25, 0.75, 0.125, 0.625, 0.375, 0.875], atol=1e-15)


def test_onb_orthonormal_right_handed(orc):
    rng = np.random.default_rng(2)
    n = rng.standard_normal((5000, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    n[:3] = [[0, 0, 1], [0, 0, -1], [1e-9, 0, -1]]
    n[:3] /= np.linalg.norm(n[:3], axis=1, keepdims=True)
    t, b = orc.onb(n)
    for u, v in [(t, b), (t, n), (b, n)]:
        assert np.max(np.abs(np.sum(u * v, 1))) < 1e-12
    for u in (t, b):
        assert np.max(np.abs(np.linalg.norm(u, axis=1) - 1)) < 1e-12
    assert np.max(np.abs(np.cross(t, b) - n)) < 1e-12


def test_env_lookup(orc):
    He, We = 16, 32
    env = np.full((He, We, 3), 0.75, np.float32)
    rng = np.random.default_rng(3)
    w = rng.standard_normal((2000, 3))
    w /= np.linalg.norm(w, axis=1, keepdims=True)
    assert np.allclose(orc.env_lookup(env, w), 0.75, atol=1e-15)
    env = rng.random((He, We, 3)).astype(np.float32)
    dirs = I.equirect_texel_dirs(He, We).reshape(-1, 3)
    assert np.allclose(orc.env_lookup(env, dirs), env.reshape(-1, 3), atol=1e-12)
    # u wraps: just either side of the -x half plane (phi = +-pi)
    e = 1e-9
    a = orc.env_lookup(env, np.array([[-1, e, 0.3], [-1, -e, 0.3]]))
    assert np.max(np.abs(a[0] - a[1])) < 1e-6
    # poles: v clamps, so the pole value is the azimuthal average of row 0
    # bilinear in u between the two nearest columns at every azimuth
    top = orc.env_lookup(env, np.array([[0, 0, 1.0]]))
    assert np.all(top >= env[0].min(0) - 1e-12) and np.all(top <= env[0].max(0) + 1e-12)


@pytest.mark.parametrize("rough", [0.1, 0.3, 0.6, 1.0])
def test_ggx_D_normalised(orc, rough):
    import ctypes as C
    lib = orc.lib()
    lib.orc_ggx_D.restype = C.c_double
    # int D(h) (n.h) dw_h over the hemisphere = 1; quadrature in cos(theta)
    # with a mapping that resolves the peak at small roughness
    from numpy.polynomial.legendre import leggauss
    xg, wg = leggauss(400)
    a = rough * rough
    # substitute tan^2(theta) = a^2 s/(1-s): Gauss-Legendre in s over (0,1)
    s = 0.5 * (xg + 1)
    ws = 0.5 * wg
    t2 = a * a * s / (1 - s)
    c2 = 1 / (1 + t2)
    c = np.sqrt(c2)
    dt2_ds = a * a / (1 - s) ** 2
    # d(cos) = -(1/2) c^3 d(t2)
    dc = 0.5 * c ** 3 * dt2_ds
    D = np.array([lib.orc_ggx_D(C.c_double(ci), C.c_double(1 - ci * ci), C.c_double(rough)) for ci in c])
    total = 2 * np.pi * np.sum(ws * D * c * dc)
    assert abs(total - 1) < 1e-9


def test_brdf_reciprocity_and_lambert(orc):
    rng = np.random.default_rng(4)
    m = 3000
    n = np.tile([0, 0, 1.0], (m, 1))
    def hemi(k):
        v = rng.standard_normal((k, 3)); v[:, 2] = np.abs(v[:, 2]) + 0.05
        return v / np.linalg.norm(v, axis=1, keepdims=True)
    wo, wi = hemi(m), hemi(m)
    a = rng.random((m, 3)); r = rng.uniform(0.1, 1, m); mt = rng.random(m)
    f1 = orc.brdf(n, wo, wi, a, r, mt)
    f2 = orc.brdf(n, wi, wo, a, r, mt)
    assert np.allclose(f1, f2, rtol=1e-12)
    # metal=0: F0 does not depend on albedo, so the albedo-dependent part of
    # f is the Lambert lobe a/pi exactly
    z = np.zeros(m)
    f = orc.brdf(n, wo, wi, a, r, z) - orc.brdf(n, wo, wi, 0 * a, r, z)
    assert np.allclose(f, a / np.pi, rtol=1e-12, atol=1e-15)
    wz = np.tile([0, 0, 1.0], (m, 1))
    # normal incidence, metal=1: F = F0 = albedo, D at n.h=1 is 1/(pi a^2)
    wz = np.tile([0, 0, 1.0], (m, 1))
    f = orc.brdf(n, wz, wz, a, r, np.ones(m))
    # G1(1) = 1 for any k; D(n) = 1/(pi alpha^2) with alpha = r^2
    assert np.allclose(f, a * (1 / (np.pi * r ** 4) / 4)[:, None], rtol=1e-12)


def _const_setup(c, occ, lin, L, spec=0.0, metal0=True):
    P, R = 64, 8
    maps_rgb = np.full((P, R, R, 3), lin, np.float32)
    maps_occ = np.full((P, R, R), occ, np.float32)
    env = np.full((16, 32, 3), L, np.float32)
    metal = np.zeros_like(c["metal"]) if metal0 else c["metal"]
    return dict(wo=c["wo"], albedo=c["albedo"], rough=c["rough"], metal=metal, probe_pos=c["probe_pos"],
                maps_rgb=maps_rgb, maps_occ=maps_occ, env=env, K=4, S=64, spec=spec)


def _albedo_part(orc, c, setup):
    """Shade output minus the same with zero albedo (metal = 0): the
    diffuse term alone, since F0 does not depend on albedo then."""
    out, _, _ = orc.query_shade(c["x"], c["n"], **setup)
    z = dict(setup, albedo=np.zeros_like(c["albedo"]))
    out0, _, _ = orc.query_shade(c["x"], c["n"], **z)
    return out - out0


def test_lambertian_closed_form(orc):
    # unoccluded Lambertian point under a constant environment L: a * L
    # (2pi/S * sum a/pi * L * z_i with mean z_i = 1/2 exactly)
    c = I.make_tiny()
    d = _albedo_part(orc, c, _const_setup(c, 0.0, 0.0, 1.7))
    L = np.float64(np.float32(1.7))
    assert np.allclose(d, c["albedo"].astype(np.float64) * L, rtol=1e-12, atol=1e-14)
    d = _albedo_part(orc, c, _const_setup(c, 0.3, 0.25, 1.7))
    want = c["albedo"].astype(np.float64) * (L * (1 - np.float64(np.float32(0.3))) + np.float64(np.float32(0.25)))
    assert np.allclose(d, want, rtol=1e-12, atol=1e-14)


def test_shadow_ratio(orc):
    c = I.make_tiny()
    setup = _const_setup(c, 0.3, 0.0, 1.0, spec=0.5, metal0=False)
    out, _, _ = orc.query_shade(c["x"], c["n"], mode=orc.MODE_SHADOW, **setup)
    assert np.allclose(out, 1 - np.float32(0.3), rtol=1e-13)
    setup = _const_setup(c, 0.0, 0.0, 1.0)
    setup["env"] = c["env"]
    out, _, _ = orc.query_shade(c["x"], c["n"], mode=orc.MODE_SHADOW, **setup)
    assert np.allclose(out, 1.0, rtol=1e-14)
    # shadow ratio is invariant to the env's overall scale and in [0, 1]
    rng = np.random.default_rng(5)
    maps = I.synthetic_maps(rng, 64, 8)
    setup.update(maps_rgb=maps["rgb"], maps_occ=maps["occ"])
    a, _, _ = orc.query_shade(c["x"], c["n"], mode=orc.MODE_SHADOW, **setup)
    setup["env"] = c["env"] * 4.0
    b, _, _ = orc.query_shade(c["x"], c["n"], mode=orc.MODE_SHADOW, **setup)
    assert np.allclose(a, b, rtol=1e-13)
    assert a.min() >= 0 and a.max() <= 1


def test_shade_linear_in_env_and_probe_radiance(orc):
    c = I.make_tiny()
    rng = np.random.default_rng(6)
    maps = I.synthetic_maps(rng, 64, 8)
    base = dict(wo=c["wo"], albedo=c["albedo"], rough=c["rough"], metal=c["metal"], probe_pos=c["probe_pos"],
                maps_occ=maps["occ"], K=4, S=64)
    z = np.zeros_like(maps["rgb"])
    a, _, _ = orc.query_shade(c["x"], c["n"], maps_rgb=maps["rgb"], env=c["env"], **base)
    b, _, _ = orc.query_shade(c["x"], c["n"], maps_rgb=z, env=c["env"], **base)
    d, _, _ = orc.query_shade(c["x"], c["n"], maps_rgb=maps["rgb"], env=np.zeros_like(c["env"]), **base)
    assert np.allclose(a, b + d, rtol=1e-12, atol=1e-14)
    assert np.all(a >= 0)


def test_fp32_sensitivity_allowance(orc):
    """The FP32 allowance is linear in the angular error and much larger for
    a rough environment than for a smooth one."""
    c = I.make_tiny()
    rng = np.random.default_rng(7)
    maps = I.synthetic_maps(rng, 64, 8)
    args = (c["x"][:256], c["n"][:256], c["wo"][:256], c["albedo"][:256], c["rough"][:256], c["metal"][:256],
            c["probe_pos"], maps["rgb"], maps["occ"])
    k1 = orc.query_shade_sensitivity(*args, c["env"], 4, 64, eps=1e-6)
    k2 = orc.query_shade_sensitivity(*args, c["env"], 4, 64, eps=2e-6)
    assert np.allclose(k2, 2 * k1, rtol=0.02, atol=1e-15)
    rough = I.env_lognormal(rng, 16, 32)
    kr = orc.query_shade_sensitivity(*args, rough, 4, 64, eps=1e-6)
    out, _, _ = orc.query_shade(*args[:6], c["probe_pos"], maps["rgb"], maps["occ"], rough, 4, 64)
    assert np.median(kr / np.abs(out)) > 3 * np.median(k1 / np.abs(orc.query_shade(
        *args[:6], c["probe_pos"], maps["rgb"], maps["occ"], c["env"], 4, 64)[0]))
