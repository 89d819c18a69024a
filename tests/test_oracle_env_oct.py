"""Pins of the oracle's octahedral environment (Sec. 4.1: the environment
map converted to an octahedral texture) used by the query's octahedral
layout."""
import numpy as np

from paper_2510_07729_gb300 import inputs as I


def test_constant_environment(orc):
    env = np.full((16, 16, 3), 0.7, np.float32)
    w = np.random.default_rng(0).standard_normal((200, 3))
    w /= np.linalg.norm(w, axis=1, keepdims=True)
    np.testing.assert_allclose(orc.env_oct_lookup(env, w), float(np.float32(0.7)), rtol=0, atol=1e-15)


def test_texel_centres_return_the_texel(orc):
    H = 8
    env = np.random.default_rng(1).uniform(0, 2, (H, H, 3)).astype(np.float32)
    jj, ii = np.meshgrid(np.arange(H), np.arange(H), indexing="ij")
    uv = np.stack([(ii.reshape(-1) + 0.5) / H, (jj.reshape(-1) + 0.5) / H], 1)
    d = orc.oct_decode(uv)
    got = orc.env_oct_lookup(env, d)
    np.testing.assert_allclose(got, env.reshape(-1, 3).astype(np.float64), rtol=0, atol=1e-12)


def test_conversion_of_a_smooth_environment(orc):
    """Resampling a smooth (lobe) environment into a fine octahedral texture
    and reading it back at random directions reproduces the equirectangular
    lookup up to the interpolation error of the two grids."""
    env = I.env_lobes(np.random.default_rng(2), 256, 512)
    oct_env = orc.env_to_octahedral(env, 512).astype(np.float32)
    w = np.random.default_rng(3).standard_normal((2000, 3))
    w /= np.linalg.norm(w, axis=1, keepdims=True)
    a = orc.env_oct_lookup(oct_env, w)
    b = orc.env_lookup(env, w)
    assert np.max(np.abs(a - b) / (np.abs(b) + 1e-3)) < 2e-2


def test_lambertian_closed_form_with_octahedral_environment(orc):
    """Unoccluded point under a constant octahedral environment L: the albedo
    part of the shading (output minus the same with zero albedo, metallic 0)
    is albedo * L, as with the equirectangular layout (the centred
    Hammersley set makes mean(cos) = 1/2 exact)."""
    c = I.make_tiny()
    maps = dict(maps_rgb=np.zeros((64, 8, 8, 3), np.float32), maps_occ=np.zeros((64, 8, 8), np.float32))
    env = np.full((16, 16, 3), 1.7, np.float32)
    setup = dict(wo=c["wo"], rough=c["rough"], metal=np.zeros_like(c["metal"]), probe_pos=c["probe_pos"], env=env,
                 K=4, S=64, spec=0.0, env_layout=orc.ENV_OCTAHEDRAL, **maps)
    out, _, _ = orc.query_shade(c["x"], c["n"], albedo=c["albedo"], **setup)
    out0, _, _ = orc.query_shade(c["x"], c["n"], albedo=np.zeros_like(c["albedo"]), **setup)
    L = np.float64(np.float32(1.7))
    assert np.allclose(out - out0, c["albedo"].astype(np.float64) * L, rtol=1e-12, atol=1e-14)
