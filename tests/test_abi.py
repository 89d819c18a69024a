"""The C-ABI library builds for sm_103a, loads without a GPU, and exports
every function that include/sop.h declares (no compute calls here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "sop.h")).read()
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    # a declaration: return type, then the sop_ name and its parameter list
    names = re.findall(r"(?:^|;|\})\s*(?:const\s+)?[A-Za-z_][\w]*\s*\**\s*(sop_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_function():
    from paper_2510_07729_gb300 import build
    lib = ctypes.CDLL(build.build())
    names = declared_functions()
    assert len(names) >= 20, names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    for must in ("sop_bake", "sop_query_shade", "sop_query_shade_backward", "sop_surrogate_train_step",
                 "sop_surrogate_infer", "sop_query_shade_noalloc", "sop_last_error"):
        assert must in names


def test_host_side_queries_without_a_gpu():
    """Size queries and argument checks run on the host only."""
    from paper_2510_07729_gb300 import build
    lib = ctypes.CDLL(build.build())
    lib.sop_bake_workspace_bytes.restype = ctypes.c_size_t
    lib.sop_bake_workspace_bytes.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32]
    assert lib.sop_bake_workspace_bytes(200000, 4096, 16) > 200000 * 80
    assert lib.sop_bake_workspace_bytes(-1, 4096, 16) == 0
    lib.sop_hammersley.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
    assert lib.sop_hammersley(0, None, None) == 1  # SOP_ERR_INVALID_ARG, before any launch
    lib.sop_last_error.restype = ctypes.c_char_p
    assert b"S = 0" in lib.sop_last_error()
    lib.sop_read_bandwidth_probe.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int32, ctypes.c_void_p,
                                             ctypes.c_void_p]
    assert lib.sop_read_bandwidth_probe(None, 64, 1, None, None) == 1


def test_radius_checked_on_the_host():
    """A search radius outside [0, 2048] (or NaN) is refused before any
    device work, by every query entry point."""
    from paper_2510_07729_gb300 import sop as S
    lib = S.load()
    fake = 1 << 20  # never dereferenced: the argument checks come first
    at = S.AtlasDesc(fake, None, 0, 0, 64, 8, 1.0, fake, None)
    for r in (-1.0, float("nan"), 4096.0):
        sp = S.ShadeParams(4, 64, 0, 0.5, 1e-6, 0, 0, r)
        assert lib.sop_query_shade(fake, fake, fake, fake, fake, fake, 16, ctypes.byref(at), fake, 16, 32, None,
                                   ctypes.byref(sp), fake, None, None, fake, 1 << 30, None) == 1
        assert b"radius" in lib.sop_last_error()
        assert lib.sop_query_shade_noalloc(fake, fake, fake, fake, fake, fake, 16, ctypes.byref(at), fake, 16, 32,
                                           None, ctypes.byref(sp), fake, None, None, None) == 1
        assert b"radius" in lib.sop_last_error()
