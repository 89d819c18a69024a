"""GPU parity of the query/shade path (Sec. 3.1.2 Eq. 2-6, Sec. 3.2.2
Eq. 7-9) against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest
import torch

from paper_2510_07729_gb300 import inputs as I
from tests.tolerance import assert_close, excess

pytestmark = pytest.mark.gpu

SOP = None


@pytest.fixture(scope="module")
def sop():
    from paper_2510_07729_gb300 import sop as S
    S.load()
    return S


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def tiny():
    return I.make_tiny()


@pytest.fixture(scope="module")
def obj():
    return I.make_object()


@pytest.fixture(scope="module")
def compose():
    return I.make_compose()


def atlas_from_maps(sop, probe_pos, maps, dtype=0):
    P, R = maps["occ"].shape[0], maps["occ"].shape[1]
    at = sop.make_atlas(cuda(probe_pos), R, rgbo_dtype=dtype)
    sop.atlas_pack(cuda(maps["rgb"]), cuda(maps["occ"]), cuda(maps["depth"]), at)
    return at


def run_gpu(sop, c, at, K, S, mode=0, pts=None, return_idx=True):
    p = pts if pts is not None else c
    out = sop.query_shade(cuda(p["x"]), cuda(p["n"]), cuda(p["wo"]), cuda(p["albedo"]), cuda(p["rough"]),
                          cuda(p["metal"]), at, cuda(c["env"]), K, S, mode=mode, return_idx=return_idx)
    torch.cuda.synchronize()
    if return_idx:
        return tuple(t.cpu().numpy() for t in out)
    return out.cpu().numpy()


def run_orc(orc, c, maps, probe_pos, K, S, mode=0, pts=None, env=None):
    p = pts if pts is not None else c
    return orc.query_shade(p["x"], p["n"], p["wo"], p["albedo"], p["rough"], p["metal"], probe_pos,
                           maps["rgb"], maps["occ"], c["env"] if env is None else env, K, S, mode=mode)


def kappa(orc, c, maps, probe_pos, K, S, mode=0, pts=None, env=None):
    p = pts if pts is not None else c
    return orc.query_shade_sensitivity(p["x"], p["n"], p["wo"], p["albedo"], p["rough"], p["metal"], probe_pos,
                                       maps["rgb"], maps["occ"], c["env"] if env is None else env, K, S, mode=mode)


def test_hammersley_matches_oracle(sop, orc):
    for S in (1, 7, 64, 128, 1000, 4096):
        g = sop.hammersley(S).cpu().numpy()
        o = orc.hammersley(S)
        assert np.array_equal(g, o.astype(np.float32))


@pytest.mark.parametrize("R", [2, 8, 16, 64])
def test_atlas_pack_gutter_exact(sop, orc, R):
    rng = np.random.default_rng(R)
    P = 5
    maps = I.synthetic_maps(rng, P, R)
    pp = rng.standard_normal((P, 3)).astype(np.float32)
    at = atlas_from_maps(sop, pp, maps)
    torch.cuda.synchronize()
    a = at.rgbo.cpu().numpy()
    dep = at.depth.cpu().numpy()
    for jj in range(R + 2):
        for ii in range(R + 2):
            si, sj = orc.oct_wrap(R, ii - 1, jj - 1)
            assert np.array_equal(a[:, jj, ii, :3], maps["rgb"][:, sj, si])
            assert np.array_equal(a[:, jj, ii, 3], maps["occ"][:, sj, si])
            assert np.array_equal(dep[:, jj, ii], maps["depth"][:, sj, si])


def test_tiny_parity(sop, orc, tiny):
    c = tiny
    maps = I.synthetic_maps(np.random.default_rng(10), 64, 8)
    at = atlas_from_maps(sop, c["probe_pos"], maps)
    out, idx, w = run_gpu(sop, c, at, c["K"], c["S"])
    ro, ri, rw = run_orc(orc, c, maps, c["probe_pos"], c["K"], c["S"])
    assert np.array_equal(idx, ri)  # bit-exact probe selection
    assert_close(w, rw, what="weights")
    assert_close(out, ro, what="shade")


@pytest.mark.parametrize("R", [2, 64])
@pytest.mark.parametrize("mode", [0, 1])
def test_tiny_parity_resolution_limits(sop, orc, tiny, R, mode):
    """The smallest and largest octahedral resolutions the library accepts
    (2 and 64 texels a side), SHADE and SHADOW, on the tiny workload."""
    c = tiny
    maps = I.synthetic_maps(np.random.default_rng(30 + R + mode), 64, R)
    at = atlas_from_maps(sop, c["probe_pos"], maps)
    out, idx, w = run_gpu(sop, c, at, c["K"], c["S"], mode=mode)
    ro, ri, rw = run_orc(orc, c, maps, c["probe_pos"], c["K"], c["S"], mode=mode)
    assert np.array_equal(idx, ri)
    kap = kappa(orc, c, maps, c["probe_pos"], c["K"], c["S"], mode=mode)
    assert_close(out, ro, what=f"R={R} mode {mode}", absolute=kap)


@pytest.mark.parametrize("mode", [0, 1])
def test_direction_count_limit(sop, orc, tiny, mode):
    """S = 4096, the most light directions the library accepts (a 64 KB
    direction table in shared memory), on 101 points of the tiny workload."""
    c = tiny
    M, S = 101, 4096
    pts = {k: c[k][:M] for k in ("x", "n", "wo", "albedo", "rough", "metal")}
    maps = I.synthetic_maps(np.random.default_rng(50 + mode), 64, 8)
    at = atlas_from_maps(sop, c["probe_pos"], maps)
    out, idx, _ = run_gpu(sop, c, at, 4, S, mode=mode, pts=pts)
    ro, ri, _ = run_orc(orc, c, maps, c["probe_pos"], 4, S, mode=mode, pts=pts)
    assert np.array_equal(idx, ri)
    kap = kappa(orc, c, maps, c["probe_pos"], 4, S, mode=mode, pts=pts)
    assert_close(out, ro, what=f"S={S} mode {mode}", absolute=kap)


def test_tiny_shadow_parity(sop, orc, tiny):
    c = tiny
    maps = I.synthetic_maps(np.random.default_rng(11), 64, 8)
    at = atlas_from_maps(sop, c["probe_pos"], maps)
    out, idx, _ = run_gpu(sop, c, at, c["K"], c["S"], mode=1)
    ro, ri, _ = run_orc(orc, c, maps, c["probe_pos"], c["K"], c["S"], mode=1)
    assert np.array_equal(idx, ri)
    assert_close(out, ro, what="shadow")


def round_bf16(a):
    """float32 -> nearest bfloat16 (ties to even), returned as float32."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


@pytest.mark.parametrize("dtype", [1, 2])
@pytest.mark.parametrize("mode", [0, 1])
def test_16bit_atlas_exact_maps(sop, orc, tiny, dtype, mode):
    """BF16 / FP16 atlases hold maps that are exact in that format: the GPU
    output (FP32 arithmetic) then meets the FP64 oracle on the same maps
    within the FP32 bound, in SHADE and SHADOW (occlusion-only footprints)
    modes."""
    c = tiny
    maps = I.synthetic_maps(np.random.default_rng(30 + dtype), 64, 8)
    rnd = round_bf16 if dtype == 1 else (lambda a: a.astype(np.float16).astype(np.float32))
    maps = {k: rnd(v) for k, v in maps.items()}
    at = atlas_from_maps(sop, c["probe_pos"], maps, dtype=dtype)
    out, idx, _ = run_gpu(sop, c, at, c["K"], c["S"], mode=mode)
    ro, ri, _ = run_orc(orc, c, maps, c["probe_pos"], c["K"], c["S"], mode=mode)
    assert np.array_equal(idx, ri)
    assert_close(out, ro, what=f"dtype {dtype} mode {mode}")


@pytest.mark.parametrize("S,dtype", [(64, 0), (128, 0), (130, 0), (64, 2), (128, 1)])
def test_shadow_shared_normal(sop, orc, tiny, S, dtype):
    """SHADOW mode on a planar receiver: warps whose points share a normal
    take their per-direction terms from a per-warp table (S <= 128); warps
    with one point off the plane, and S above the table's limit, take the
    per-point path. All match the FP64 oracle."""
    c = tiny
    rng = np.random.default_rng(40 + S)
    M = 32 * 40 + 7
    x = rng.uniform(-1.0, 1.0, (M, 3)).astype(np.float32)
    x[:, 2] = -1.05
    n = np.zeros((M, 3), np.float32)
    n[:, 2] = 1.0
    n[32 * 3 + 5] = np.array([0.3, 0.1, 0.95], np.float32)  # one warp is mixed
    pts = dict(x=x, n=n, wo=n.copy(), albedo=c["albedo"][:M], rough=c["rough"][:M], metal=c["metal"][:M])
    maps = I.synthetic_maps(rng, 64, 8)
    if dtype:  # maps exact in the atlas format (16-bit atlases: two lanes per point)
        rnd = round_bf16 if dtype == 1 else (lambda a: a.astype(np.float16).astype(np.float32))
        maps = {k: rnd(v) for k, v in maps.items()}
    at = atlas_from_maps(sop, c["probe_pos"], maps, dtype=dtype)
    out, idx, _ = run_gpu(sop, c, at, 4, S, mode=1, pts=pts)
    ro, ri, _ = run_orc(orc, c, maps, c["probe_pos"], 4, S, mode=1, pts=pts)
    assert np.array_equal(idx, ri)
    kap = kappa(orc, c, maps, c["probe_pos"], 4, S, mode=1, pts=pts)
    assert_close(out, ro, what=f"shadow S={S} dtype={dtype}", absolute=kap)


@pytest.mark.parametrize("M", [1, 31, 4096 + 37])
@pytest.mark.parametrize("K", [1, 3, 8, 32])
def test_ragged_sizes_and_K(sop, orc, tiny, M, K):
    c = tiny
    rng = np.random.default_rng(M * 100 + K)
    sel, pts = I.subsample(rng, {k: np.concatenate([c[k]] * 2) for k in ("x", "n", "wo", "albedo", "rough", "metal")},
                           ["x", "n", "wo", "albedo", "rough", "metal"], M)
    maps = I.synthetic_maps(rng, 64, 8)
    at = atlas_from_maps(sop, c["probe_pos"], maps)
    S = 37
    out, idx, w = run_gpu(sop, c, at, K, S, pts=pts)
    ro, ri, rw = run_orc(orc, c, maps, c["probe_pos"], K, S, pts=pts)
    assert np.array_equal(idx, ri)
    assert_close(w, rw, what="weights")
    assert_close(out, ro, what="shade")


def test_snap_and_axis_normals(sop, orc, tiny):
    c = tiny
    rng = np.random.default_rng(3)
    maps = I.synthetic_maps(rng, 64, 8)
    at = atlas_from_maps(sop, c["probe_pos"], maps)
    x = np.concatenate([c["probe_pos"][:8], c["x"][:8]])
    n = np.concatenate([c["probe_nrm"][:8], np.array([[0, 0, 1], [0, 0, -1], [1, 0, 0], [0, 1, 0], [0, -1, 0],
                                                       [-1, 0, 0], [0, 0, 3], [1e-8, 0, -1]], np.float32)])
    pts = dict(x=x, n=n.astype(np.float32), wo=np.abs(n).astype(np.float32) / np.linalg.norm(n, axis=1, keepdims=True),
               albedo=c["albedo"][:16], rough=c["rough"][:16], metal=c["metal"][:16])
    pts["wo"] = (pts["n"] / np.linalg.norm(pts["n"], axis=1, keepdims=True)).astype(np.float32)
    out, idx, w = run_gpu(sop, c, at, 4, 64, pts=pts)
    ro, ri, rw = run_orc(orc, c, maps, c["probe_pos"], 4, 64, pts=pts)
    assert np.array_equal(idx, ri)
    assert np.array_equal(w[:8], np.eye(4, dtype=np.float32)[[0] * 8])
    assert_close(out, ro, what="shade")


def test_empty_query(sop, tiny):
    c = tiny
    maps = I.synthetic_maps(np.random.default_rng(0), 64, 8)
    at = atlas_from_maps(sop, c["probe_pos"], maps)
    z = {k: c[k][:0] for k in ("x", "n", "wo", "albedo", "rough", "metal")}
    out = run_gpu(sop, c, at, 4, 64, pts=z, return_idx=False)
    assert out.shape == (0, 3)


def test_object_full_size_sampled(sop, orc, obj):
    """Full 'object' workload (all points, K=8, S=128) in the benchmark's
    launch configuration; 4096 sampled points checked one by one."""
    c = obj
    maps = I.synthetic_maps(np.random.default_rng(12), 4096, 16)
    at = atlas_from_maps(sop, c["probe_pos"], maps)
    out, idx, w = run_gpu(sop, c, at, c["K"], c["S"])
    sel, pts = I.subsample(np.random.default_rng(13), c, ["x", "n", "wo", "albedo", "rough", "metal"], 4096)
    ro, ri, rw = run_orc(orc, c, maps, c["probe_pos"], c["K"], c["S"], pts=pts)
    assert np.array_equal(idx[sel], ri)
    assert_close(w[sel], rw, what="weights")
    kap = kappa(orc, c, maps, c["probe_pos"], c["K"], c["S"], pts=pts)
    assert_close(out[sel], ro, what="shade", absolute=kap)


def test_object_geometry_smooth_env_strict(sop, orc, obj):
    """Same points and probes under a smooth environment (lobes): the plain
    1e-5 relative bound holds without any conditioning allowance."""
    c = dict(obj, env=I.env_lobes(np.random.default_rng(5), 256, 512))
    maps = I.synthetic_maps(np.random.default_rng(18), 4096, 16)
    at = atlas_from_maps(sop, c["probe_pos"], maps)
    out, idx, w = run_gpu(sop, c, at, c["K"], c["S"])
    sel, pts = I.subsample(np.random.default_rng(19), c, ["x", "n", "wo", "albedo", "rough", "metal"], 4096)
    ro, ri, rw = run_orc(orc, c, maps, c["probe_pos"], c["K"], c["S"], pts=pts)
    assert np.array_equal(idx[sel], ri)
    assert_close(out[sel], ro, what="shade")


def test_compose_full_size_sampled(sop, orc, compose):
    """1920x1080 composition: object pixels SHADE with the object probes,
    scene pixels SHADOW with the shadow-region probes (K=8, S=64)."""
    c = compose
    for part, mode, seed in (("shade", 0, 14), ("shadow", 1, 15)):
        d = dict(c[part], env=c["env"])
        maps = I.synthetic_maps(np.random.default_rng(seed), 4096, 16)
        at = atlas_from_maps(sop, d["probe_pos"], maps)
        out, idx, w = run_gpu(sop, d, at, c["K"], c["S"], mode=mode)
        sel, pts = I.subsample(np.random.default_rng(seed + 100), d, ["x", "n", "wo", "albedo", "rough", "metal"],
                               4096)
        ro, ri, rw = run_orc(orc, d, maps, d["probe_pos"], c["K"], c["S"], mode=mode, pts=pts)
        assert np.array_equal(idx[sel], ri)
        kap = kappa(orc, d, maps, d["probe_pos"], c["K"], c["S"], mode=mode, pts=pts)
        assert_close(out[sel], ro, what=part, absolute=kap)


@pytest.mark.parametrize("dtype,bound", [(1, 2e-2), (2, 2e-3)])
def test_reduced_precision_atlas_error(sop, orc, obj, dtype, bound):
    """BF16 / FP16 atlas storage with FP32 accumulation: relative L1 error of
    the shaded output against the FP64 oracle on the full-precision maps."""
    c = obj
    maps = I.synthetic_maps(np.random.default_rng(16), 4096, 16)
    at = atlas_from_maps(sop, c["probe_pos"], maps, dtype=dtype)
    out, idx, _ = run_gpu(sop, c, at, c["K"], c["S"])
    sel, pts = I.subsample(np.random.default_rng(17), c, ["x", "n", "wo", "albedo", "rough", "metal"], 4096)
    ro, ri, _ = run_orc(orc, c, maps, c["probe_pos"], c["K"], c["S"], pts=pts)
    assert np.array_equal(idx[sel], ri)
    rel = np.abs(out[sel] - ro).mean() / np.abs(ro).mean()
    assert rel < bound


def test_concurrent_queries_on_two_streams(sop, tiny):
    """Two independent queries (own points, atlas, output and workspace; the
    environment shared and read-only), a SHADE and a SHADOW call as in the
    composition frame, issued on two streams at once: each output is
    bit-identical to the same call issued alone (the library keeps no
    scratch of its own across sop_query_shade calls)."""
    c = tiny
    keys = ("x", "n", "wo", "albedo", "rough", "metal")
    env = cuda(c["env"])
    calls = []
    for seed, mode, sl in ((60, 0, slice(0, 2049)), (61, 1, slice(2049, 4096))):
        maps = I.synthetic_maps(np.random.default_rng(seed), 64, 8)
        at = atlas_from_maps(sop, c["probe_pos"], maps)
        pts = [cuda(c[k][sl]) for k in keys]
        M = pts[0].shape[0]
        ws = torch.empty(sop.query_workspace_bytes(at, M, 8, 256, env.shape[0], env.shape[1], mode),
                         dtype=torch.uint8, device="cuda")
        calls.append((pts, at, mode, ws, M))

    def run(pts, at, mode, ws, M, out):
        sop.query_shade(*pts, at, env, 8, 256, mode=mode, out=out, workspace=ws)

    alone = []
    for pts, at, mode, ws, M in calls:
        out = torch.empty((M, 3), dtype=torch.float32, device="cuda")
        run(pts, at, mode, ws, M, out)
        torch.cuda.synchronize()
        alone.append(out.clone())
    side = torch.cuda.Stream()
    main = torch.cuda.current_stream()
    for _ in range(3):
        outs = [torch.full((M, 3), float("nan"), device="cuda") for _, _, _, _, M in calls]
        side.wait_stream(main)
        with torch.cuda.stream(side):
            run(*calls[0], outs[0])
        run(*calls[1], outs[1])
        main.wait_stream(side)
        torch.cuda.synchronize()
        for a, b in zip(alone, outs):
            assert torch.equal(a, b)
    assert sop.device_status() == 0
