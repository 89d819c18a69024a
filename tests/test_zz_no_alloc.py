"""The allocation-free query entry point (sop_query_shade_noalloc).

Some callers cannot allocate device memory (a host framework that owns every
allocation, a plugin or capture context, an embedded runtime without an
allocator). For them the library offers a variant of sop_query_shade that
takes no workspace and uses a fixed scratch array compiled into the library.
These checks call it through the C ABI and compare it with the regular
entry point, twice in a row (the scratch array keeps the previous call's
contents, which must not leak into the next result). The file is named so
that pytest collects it last.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2510_07729_gb300 import inputs as I
from tests.tolerance import assert_close

pytestmark = pytest.mark.gpu


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def call_noalloc(lib, sop, pts, at, env, K, S, mode, out, idx, w):
    sp = sop.ShadeParams(K, S, mode, 0.5, 1e-6)
    d = at.c()
    M = pts[0].shape[0]
    st = lib.sop_query_shade_noalloc(*[C.c_void_p(t.data_ptr()) for t in pts], M, C.byref(d),
                                     C.c_void_p(env.data_ptr()), env.shape[0], env.shape[1], None, C.byref(sp),
                                     C.c_void_p(out.data_ptr()), C.c_void_p(idx.data_ptr()),
                                     C.c_void_p(w.data_ptr()), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, lib.sop_last_error().decode()


@pytest.mark.parametrize("workload,mode,dtype", [("tiny", 0, 0), ("object", 0, 0), ("object", 0, 2),
                                                  ("compose_shadow", 1, 0)])
def test_noalloc_matches_workspace_entry_point(workload, mode, dtype):
    from paper_2510_07729_gb300 import sop
    lib = sop.load()
    if workload == "tiny":
        c = I.make_tiny()
        pp, P, R, K, S, env = c["probe_pos"], 64, 8, c["K"], c["S"], c["env"]
        p = c
    elif workload == "object":
        c = I.make_object()
        pp, P, R, K, S, env = c["probe_pos"], 4096, 16, c["K"], c["S"], c["env"]
        p = c
    else:
        c = I.make_compose()
        p = c["shadow"]
        pp, P, R, K, S, env = p["probe_pos"], 4096, 16, c["K"], c["S"], c["env"]
    # more points than one scratch chunk, with a ragged tail
    keys = ("x", "n", "wo", "albedo", "rough", "metal")
    M = min(len(p["x"]), 3 * 16384 + 1001)
    pts = [cuda(p[k][:M]) for k in keys]
    maps = I.synthetic_maps(np.random.default_rng(40), P, R)
    at = sop.make_atlas(cuda(pp), R, rgbo_dtype=dtype)
    sop.atlas_pack(cuda(maps["rgb"]), cuda(maps["occ"]), cuda(maps["depth"]), at)
    envt = cuda(env)
    ref, ref_idx, ref_w = sop.query_shade(*pts, at, envt, K, S, mode=mode, return_idx=True)
    for _ in range(2):
        out = torch.full((M, 3), float("nan"), device="cuda")
        idx = torch.full((M, K), -1, dtype=torch.int32, device="cuda")
        w = torch.full((M, K), float("nan"), device="cuda")
        call_noalloc(lib, sop, pts, at, envt, K, S, mode, out, idx, w)
        torch.cuda.synchronize()
        assert torch.equal(idx, ref_idx)
        assert_close(w.cpu().numpy(), ref_w.cpu().numpy(), what="weights")
        assert_close(out.cpu().numpy(), ref.cpu().numpy(), what="noalloc vs workspace")


def test_noalloc_rejects_too_many_probes():
    from paper_2510_07729_gb300 import sop
    lib = sop.load()
    P = 65536 + 1
    pp = torch.zeros((P, 3), device="cuda")
    at = sop.make_atlas(pp, 2, with_depth=False)
    sp = sop.ShadeParams(4, 16, 0, 0.5, 1e-6)
    d = at.c()
    z = torch.zeros((1, 3), device="cuda")
    st = lib.sop_query_shade_noalloc(*[C.c_void_p(z.data_ptr())] * 6, 1, C.byref(d), C.c_void_p(z.data_ptr()), 1, 1,
                                     None, C.byref(sp), C.c_void_p(z.data_ptr()), None, None, None)
    assert st == 1
    assert "scratch" in lib.sop_last_error().decode()
