"""GPU parity of importance-sampled rendering (Sec. 4.2, Eq. PDF over the
octahedral environment) against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest
import torch

from paper_2510_07729_gb300 import inputs as I
from tests.tolerance import assert_close

pytestmark = pytest.mark.gpu

PTS = ("x", "n", "wo", "albedo", "rough", "metal")


@pytest.fixture(scope="module")
def sop():
    from paper_2510_07729_gb300 import sop as S
    S.load()
    return S


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("H,S", [(64, 256), (256, 4096)])
def test_sampler_matches_oracle(sop, orc, H, S):
    """The texel of every sample is an exact integer decision on both sides:
    directions agree to float32 rounding, densities to float32 rounding."""
    env = orc.env_to_octahedral(I.env_lognormal(np.random.default_rng(H), 128, 256), H).astype(np.float32)
    got = sop.env_importance_dirs(cuda(env), S).cpu().numpy().astype(np.float64)
    want = orc.env_importance_dirs(env, S)
    assert np.max(np.abs(got[:, :3] - want[:, :3])) < 2e-7
    np.testing.assert_allclose(got[:, 3], want[:, 3], rtol=2e-7)


def _check(sop, orc, pts, probe_pos, maps, env_oct, K, S, mode, sample=None):
    at = sop.make_atlas(cuda(probe_pos), maps["occ"].shape[1])
    sop.atlas_pack(cuda(maps["rgb"]), cuda(maps["occ"]), cuda(maps["depth"]), at)
    gd = sop.env_importance_dirs(cuda(env_oct), S)
    out = sop.query_shade(*[cuda(pts[k]) for k in PTS], at, cuda(env_oct), K, S, mode=mode,
                          env_layout=sop.ENV_OCTAHEDRAL, dirs_world=gd).cpu().numpy()
    p = pts
    if sample is not None:
        sel, p = I.subsample(np.random.default_rng(sample), pts, list(PTS), 4096)
        out = out[sel]
    od = orc.env_importance_dirs(env_oct, S)
    args = [p[k] for k in PTS] + [probe_pos, maps["rgb"], maps["occ"], env_oct, K, S]
    kw = dict(mode=mode, env_layout=orc.ENV_OCTAHEDRAL, dirs=od, dir_world=True)
    ro, _, _ = orc.query_shade(*args, **kw)
    kap = orc.query_shade_sensitivity(*args, **kw)
    assert_close(out, ro, what=f"importance sampled, mode {mode}", absolute=kap)


@pytest.mark.parametrize("mode", [0, 1])
def test_importance_direction_count_limit(sop, orc, mode):
    """4,096 importance-sampled world directions (the library's maximum S;
    the world-direction kernel's table is 192 KB of shared memory) on 101
    points of the tiny workload."""
    c = I.make_tiny()
    pts = {k: c[k][:101] for k in PTS}
    env_oct = orc.env_to_octahedral(c["env"], 32).astype(np.float32)
    maps = I.synthetic_maps(np.random.default_rng(44 + mode), 64, 8)
    _check(sop, orc, pts, c["probe_pos"], maps, env_oct, c["K"], 4096, mode)


@pytest.mark.parametrize("mode", [0, 1])
def test_tiny_importance_sampled(sop, orc, mode):
    c = I.make_tiny()
    env_oct = orc.env_to_octahedral(c["env"], 32).astype(np.float32)
    maps = I.synthetic_maps(np.random.default_rng(40 + mode), 64, 8)
    _check(sop, orc, c, c["probe_pos"], maps, env_oct, c["K"], 256, mode)


def test_object_importance_sampled(sop, orc):
    c = I.make_object()
    env_oct = orc.env_to_octahedral(c["env"], 256).astype(np.float32)
    maps = I.synthetic_maps(np.random.default_rng(42), 4096, 16)
    _check(sop, orc, c, c["probe_pos"], maps, env_oct, c["K"], c["S"], 0, sample=43)


def test_compose_shadow_importance_sampled(sop, orc):
    c = I.make_compose()
    d = dict(c["shadow"])
    env_oct = orc.env_to_octahedral(c["env"], 128).astype(np.float32)
    maps = I.synthetic_maps(np.random.default_rng(44), 4096, 16)
    _check(sop, orc, d, d["probe_pos"], maps, env_oct, c["K"], c["S"], 1, sample=45)
