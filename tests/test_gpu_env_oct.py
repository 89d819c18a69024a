"""GPU parity of the octahedral environment layout (Sec. 4.1: the estimated
environment map is converted to an octahedral texture) against the FP64
oracle, through the C ABI."""
import ctypes as C

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


def _atlas(sop, probe_pos, maps):
    at = sop.make_atlas(cuda(probe_pos), maps["occ"].shape[1])
    sop.atlas_pack(cuda(maps["rgb"]), cuda(maps["occ"]), cuda(maps["depth"]), at)
    return at


def _run(sop, orc, pts, probe_pos, maps, env_oct, K, S, mode):
    at = _atlas(sop, probe_pos, maps)
    out, idx, _ = sop.query_shade(*[cuda(pts[k]) for k in PTS], at, cuda(env_oct), K, S, mode=mode, return_idx=True,
                                  env_layout=sop.ENV_OCTAHEDRAL)
    torch.cuda.synchronize()
    args = [pts[k] for k in PTS] + [probe_pos, maps["rgb"], maps["occ"], env_oct, K, S]
    ro, ri, _ = orc.query_shade(*args, mode=mode, env_layout=orc.ENV_OCTAHEDRAL)
    kap = orc.query_shade_sensitivity(*args, mode=mode, env_layout=orc.ENV_OCTAHEDRAL)
    assert np.array_equal(idx.cpu().numpy(), ri)
    return out.cpu().numpy(), ro, kap


def test_conversion_matches_oracle(sop, orc):
    env = I.env_lobes(np.random.default_rng(0), 64, 128)
    got = sop.env_to_octahedral(cuda(env), 32).cpu().numpy()
    want = orc.env_to_octahedral(env, 32)
    assert_close(got, want, what="env_to_octahedral")


@pytest.mark.parametrize("mode", [0, 1])
def test_tiny_octahedral_env(sop, orc, mode):
    c = I.make_tiny()
    env_oct = orc.env_to_octahedral(c["env"], 16).astype(np.float32)
    maps = I.synthetic_maps(np.random.default_rng(20 + mode), 64, 8)
    out, ro, kap = _run(sop, orc, c, c["probe_pos"], maps, env_oct, c["K"], c["S"], mode)
    assert_close(out, ro, what=f"tiny octahedral env, mode {mode}", absolute=kap)


def test_object_octahedral_env_sampled(sop, orc):
    """Full object view (K=8, S=128) with the log-normal environment
    resampled to a 256x256 octahedral map; 4096 sampled points checked."""
    c = I.make_object()
    env_oct = orc.env_to_octahedral(c["env"], 256).astype(np.float32)
    maps = I.synthetic_maps(np.random.default_rng(22), 4096, 16)
    at = _atlas(sop, c["probe_pos"], maps)
    out = sop.query_shade(*[cuda(c[k]) for k in PTS], at, cuda(env_oct), c["K"], c["S"],
                          env_layout=sop.ENV_OCTAHEDRAL).cpu().numpy()
    sel, pts = I.subsample(np.random.default_rng(23), c, list(PTS), 4096)
    args = [pts[k] for k in PTS] + [c["probe_pos"], maps["rgb"], maps["occ"], env_oct, c["K"], c["S"]]
    ro, _, _ = orc.query_shade(*args, env_layout=orc.ENV_OCTAHEDRAL)
    kap = orc.query_shade_sensitivity(*args, env_layout=orc.ENV_OCTAHEDRAL)
    assert_close(out[sel], ro, what="object octahedral env", absolute=kap)


def test_compose_shadow_octahedral_env(sop, orc):
    """The composition frame's scene pixels (planar receivers: per-warp
    direction tables) with an octahedral environment."""
    c = I.make_compose()
    d = dict(c["shadow"])
    env_oct = orc.env_to_octahedral(c["env"], 128).astype(np.float32)
    maps = I.synthetic_maps(np.random.default_rng(24), 4096, 16)
    at = _atlas(sop, d["probe_pos"], maps)
    out = sop.query_shade(*[cuda(d[k]) for k in PTS], at, cuda(env_oct), c["K"], c["S"], mode=1,
                          env_layout=sop.ENV_OCTAHEDRAL).cpu().numpy()
    sel, pts = I.subsample(np.random.default_rng(25), d, list(PTS), 4096)
    args = [pts[k] for k in PTS] + [d["probe_pos"], maps["rgb"], maps["occ"], env_oct, c["K"], c["S"]]
    ro, _, _ = orc.query_shade(*args, mode=1, env_layout=orc.ENV_OCTAHEDRAL)
    kap = orc.query_shade_sensitivity(*args, mode=1, env_layout=orc.ENV_OCTAHEDRAL)
    assert_close(out[sel], ro, what="compose shadow octahedral env", absolute=kap)


def test_adjoint_rejects_octahedral_env(sop):
    """The adjoint and the allocation-free entry point take the
    equirectangular layout only: SOP_ERR_UNSUPPORTED before any launch."""
    c = I.make_tiny()
    maps = I.synthetic_maps(np.random.default_rng(26), 64, 8)
    at = _atlas(sop, c["probe_pos"], maps)
    lib = sop.load()
    M = 8
    x, n, wo, alb, r, m = [cuda(c[k][:M]) for k in PTS]
    env = cuda(np.full((16, 16, 3), 0.5, np.float32))
    sp = sop.ShadeParams(4, 16, 0, 0.5, 1e-6, sop.ENV_OCTAHEDRAL)
    g = [torch.zeros((M, 3), device="cuda"), torch.zeros(M, device="cuda"), torch.zeros(M, device="cuda"),
         torch.zeros((M, 3), device="cuda"), torch.zeros((16, 16, 3), device="cuda"),
         torch.zeros((64, 8, 8, 4), device="cuda")]
    ws = torch.empty(1 << 24, dtype=torch.uint8, device="cuda")
    st = lib.sop_query_shade_backward(*[C.c_void_p(t.data_ptr()) for t in (x, n, wo, alb, r, m)], M,
                                      C.byref(at.c()), C.c_void_p(env.data_ptr()), 16, 16, None, C.byref(sp),
                                      C.c_void_p(x.data_ptr()), *[C.c_void_p(t.data_ptr()) for t in g],
                                      C.c_void_p(ws.data_ptr()), ws.numel(), None)
    assert st == 4
    out = torch.empty((M, 3), device="cuda")
    st = lib.sop_query_shade_noalloc(*[C.c_void_p(t.data_ptr()) for t in (x, n, wo, alb, r, m)], M,
                                     C.byref(at.c()), C.c_void_p(env.data_ptr()), 16, 16, None, C.byref(sp),
                                     C.c_void_p(out.data_ptr()), None, None, None)
    assert st == 4
