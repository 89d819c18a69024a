"""Pins of the oracle's importance-sampled light directions (Sec. 4.2,
Eq. PDF: density H W I / (4 pi) over the octahedral environment) and of the
estimator that uses them."""
import numpy as np

from paper_2510_07729_gb300 import inputs as I


def test_constant_map_gives_the_uniform_density(orc):
    env = np.full((32, 32, 3), 0.4, np.float32)
    d = orc.env_importance_dirs(env, 300)
    np.testing.assert_allclose(d[:, 3], 1.0 / (4.0 * np.pi), rtol=1e-15)
    np.testing.assert_allclose(np.linalg.norm(d[:, :3], axis=1), 1.0, rtol=1e-15)


def test_samples_follow_the_intensity(orc):
    """Half of the texels three times brighter than the rest: three quarters
    of the stratified samples land in the bright half (integer CDF: to within
    one sample), each with density proportional to its texel's intensity."""
    H, S = 16, 400
    env = np.full((H, H, 3), 1.0, np.float32)
    env[: H // 2] = 3.0
    d = orc.env_importance_dirs(env, S)
    uv = orc.oct_encode(d[:, :3])
    bright = (np.floor(uv[:, 1] * H) < H // 2)
    assert abs(bright.sum() - 0.75 * S) <= 1
    T = H * H
    qb, qd = 2 ** 20, int(np.floor(np.float32(3.0) / np.float32(9.0) * 2 ** 20))  # quantised intensities
    Q = T // 2 * (qb + qd)
    pdf_bright, pdf_dim = T * qb / (4 * np.pi * Q), T * qd / (4 * np.pi * Q)
    np.testing.assert_allclose(d[bright, 3], pdf_bright, rtol=1e-12)
    np.testing.assert_allclose(d[~bright, 3], pdf_dim, rtol=1e-12)


def _lambert_part(orc, c, env, dirs, S):
    M = 64
    maps = dict(maps_rgb=np.zeros((64, 8, 8, 3), np.float32), maps_occ=np.zeros((64, 8, 8), np.float32))
    setup = dict(wo=c["wo"][:M], rough=c["rough"][:M], metal=np.zeros(M, np.float32), probe_pos=c["probe_pos"],
                 env=env, K=4, S=S, spec=0.0, env_layout=orc.ENV_OCTAHEDRAL, **maps)
    if dirs is not None:
        setup.update(dirs=dirs, dir_world=True)
    out, _, _ = orc.query_shade(c["x"][:M], c["n"][:M], albedo=c["albedo"][:M], **setup)
    out0, _, _ = orc.query_shade(c["x"][:M], c["n"][:M], albedo=np.zeros_like(c["albedo"][:M]), **setup)
    return out - out0


def test_lambertian_under_a_constant_map(orc):
    """(1/S) sum a/pi L cos+ / pdf with pdf = 1/(4 pi): 4 a L mean(cos+), and
    the mean of cos+ over the sphere is 1/4, so the estimate is a L. The
    samples sit at texel centres, one per texel here, and the equation takes
    the octahedral texels as equal in solid angle, which they are only
    roughly: a few percent per point, under 1.5% on average. A wrong factor
    (2 pi for 4 pi, a missing 1/pdf) would be off by 2x or more."""
    c = I.make_tiny()
    env = np.full((64, 64, 3), 1.3, np.float32)
    S = 4096
    got = _lambert_part(orc, c, env, orc.env_importance_dirs(env, S), S)
    want = np.float64(np.float32(1.3)) * c["albedo"][:64].astype(np.float64)
    np.testing.assert_allclose(got, want, rtol=5e-2)
    assert abs(got.sum() / want.sum() - 1.0) < 1.5e-2


def test_agrees_with_the_uniform_estimate(orc):
    """On a smooth, strongly varying map (lobes) the importance-sampled
    estimate of the unoccluded Lambertian term agrees with a dense uniform
    (Hammersley) estimate of the same integral."""
    c = I.make_tiny()
    eq = I.env_lobes(np.random.default_rng(7), 128, 256)
    env = orc.env_to_octahedral(eq, 64).astype(np.float32)
    a = _lambert_part(orc, c, env, orc.env_importance_dirs(env, 4096), 4096)
    b = _lambert_part(orc, c, env, None, 16384)
    assert np.abs(a - b).mean() / np.abs(b).mean() < 3e-2
