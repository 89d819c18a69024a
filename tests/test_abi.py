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
    for must in ("sop_bake", "sop_query_shade", "sop_query_shade_backward", "sop_surrogate_create",
                 "sop_surrogate_destroy", "sop_surrogate_save", "sop_surrogate_load", "sop_surrogate_train",
                 "sop_surrogate_infer", "sop_query_shade_noalloc", "sop_device_status", "sop_last_error"):
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


def test_footprint_index_range_checked_on_the_host():
    """An atlas whose bilinear footprints (P (R+1)^2) overflow the shading
    kernels' 32-bit index is refused before any device work; one just
    inside the range passes the check (and then fails on the workspace)."""
    from paper_2510_07729_gb300 import sop as S
    lib = S.load()
    fake = 1 << 20
    sp = S.ShadeParams(4, 64, 0, 0.5, 1e-6, 0, 0, 0.0)
    for P, R, refused in ((508280, 64, False), (508281, 64, True), (7430739, 16, False), (7430740, 16, True)):
        assert (P * (R + 1) ** 2 > 2 ** 31 - 1) == refused
        at = S.AtlasDesc(fake, None, 0, 0, P, R, 1.0, fake, None)
        st = lib.sop_query_shade(fake, fake, fake, fake, fake, fake, 16, ctypes.byref(at), fake, 16, 32, None,
                                 ctypes.byref(sp), fake, None, None, fake, 64, None)
        # refused: SOP_ERR_INVALID_ARG; else the 64-byte workspace is too small
        assert st == (1 if refused else 3), (P, R, st, lib.sop_last_error())
        assert (b"footprints" in lib.sop_last_error()) == refused, lib.sop_last_error()


def test_front_end_and_placement_checks_on_the_host():
    """The deferred front end and the placement entry points refuse bad
    arguments before any device work (SOP_ERR_INVALID_ARG = 1, with a
    message), so these run without a GPU."""
    from paper_2510_07729_gb300 import sop as S
    lib = S.load()
    fake = 1 << 20  # 16-byte aligned, never dereferenced
    f3 = lambda *v: (ctypes.c_float * 3)(*v)  # noqa: E731
    # pinhole: empty image, degenerate camera, field of view out of range
    assert lib.sop_pinhole_dirs(0, 10, f3(0, 0, 1), f3(0, 0, 0), f3(0, 0, 1), 40.0, fake, None) == 1
    assert lib.sop_pinhole_dirs(8, 8, f3(0, 0, 1), f3(0, 0, 1), f3(0, 0, 1), 40.0, fake, None) == 1
    assert b"eye == target" in lib.sop_last_error()
    assert lib.sop_pinhole_dirs(8, 8, f3(0, 0, 1), f3(0, 0, 0), f3(0, 0, 1), 180.0, fake, None) == 1
    assert lib.sop_pinhole_dirs(8, 8, f3(0, 0, 1), f3(0, 0, 0), f3(0, 0, 1), 40.0, fake + 4, None) == 1
    assert lib.sop_panorama_dirs(16, 0, fake, None) == 1
    # G-buffer trace: no origin, unaligned directions, no materials
    g = S.Gaussians(fake, fake, fake, fake, fake, 10)
    m = S.Materials(fake, fake, fake)
    bp = S.BakeParams(0.0, 1.0 / 255.0, 0.99, 1e-4, 0.0)
    assert lib.sop_trace_gbuffer(ctypes.byref(g), ctypes.byref(m), fake, 0, fake, 4, ctypes.byref(bp), fake, fake,
                                 1 << 30, None) == 1
    assert lib.sop_trace_gbuffer(ctypes.byref(g), ctypes.byref(m), fake, 1, fake + 8, 4, ctypes.byref(bp), fake,
                                 fake, 1 << 30, None) == 1
    assert lib.sop_trace_gbuffer(ctypes.byref(g), None, fake, 1, fake, 4, ctypes.byref(bp), fake, fake, 1 << 30,
                                 None) == 1
    assert b"materials" in lib.sop_last_error()
    # shading points: non-positive threshold, missing outputs
    cnt = ctypes.c_void_p(fake)
    assert lib.sop_gbuffer_points(fake, None, 16, f3(0, 0, 0), fake, 0.0, fake, fake, fake, fake, fake, fake, fake,
                                  cnt, fake, 1 << 20, None) == 1
    assert lib.sop_gbuffer_points(fake, None, 16, f3(0, 0, 0), fake, 0.5, None, fake, fake, fake, fake, fake, fake,
                                  cnt, fake, 1 << 20, None) == 1
    # compositing: more points than pixels
    assert lib.sop_depth_composite(fake, fake, 4, fake, fake, 5, None, None, 0, fake, None) == 1
    # placement: k above n, start outside, non-finite offset
    assert lib.sop_place_probes(fake, None, 10, 11, 0, 0.0, fake, None, fake, 1 << 20, None) == 1
    assert lib.sop_place_probes(fake, None, 10, 4, 10, 0.0, fake, None, fake, 1 << 20, None) == 1
    assert lib.sop_place_probes(fake, None, 10, 4, 0, float("inf"), fake, None, fake, 1 << 20, None) == 1
    assert lib.sop_place_probes_workspace_bytes(0) == 0 and lib.sop_place_probes_workspace_bytes(100) > 0


def test_grid_density_checked_on_the_host():
    from paper_2510_07729_gb300 import sop as S
    lib = S.load()
    fake = 1 << 20
    g = S.Gaussians(fake, fake, fake, fake, fake, 10)
    for dens in (5.0, 0.001, -1.0, float("nan")):
        bp = S.BakeParams(0.0, 1.0 / 255.0, 0.99, 1e-4, dens)
        assert lib.sop_bake_bin(ctypes.byref(g), ctypes.byref(bp), fake, 1 << 30, None) == 1
        assert b"grid_density" in lib.sop_last_error()


def test_bake_workspace_minimum_checked_on_the_host():
    """sop_bake_bin sizes its grid on the device and relies on a workspace of
    at least sop_bake_workspace_bytes(): a smaller one is refused before any
    launch (SOP_ERR_WORKSPACE = 3), with the bytes needed in the message."""
    from paper_2510_07729_gb300 import sop as S
    lib = S.load()
    fake = 1 << 20
    n = 1000
    need = int(lib.sop_bake_workspace_bytes(n, 1, 2))
    g = S.Gaussians(fake, fake, fake, fake, fake, n)
    bp = S.BakeParams(0.0, 1.0 / 255.0, 0.99, 1e-4, 0.0)
    assert lib.sop_bake_bin(ctypes.byref(g), ctypes.byref(bp), fake, need - 256, None) == 3
    assert str(need).encode() in lib.sop_last_error()
    assert lib.sop_bake_bin(ctypes.byref(g), ctypes.byref(bp), fake + 128, need, None) == 3  # misaligned


def test_device_status_bits_decoded_on_the_host():
    """The device status word's bits as the header defines them, and their
    decoding by the binding (no GPU: the word itself is read on a GPU)."""
    from paper_2510_07729_gb300 import sop as S
    hdr = open(os.path.join(ROOT, "include", "sop.h")).read()
    for name, val in (("NONFINITE", S.DEVSTAT_NONFINITE), ("BAKE_TRUNCATED", S.DEVSTAT_BAKE_TRUNCATED),
                      ("INDEX", S.DEVSTAT_INDEX), ("CAPACITY", S.DEVSTAT_CAPACITY), ("TIMEOUT", S.DEVSTAT_TIMEOUT),
                      ("GRID_COARSENED", S.DEVSTAT_GRID_COARSENED), ("ERRORS", S.DEVSTAT_ERRORS)):
        m = re.search(r"#define SOP_DEVSTAT_%s (0x[0-9a-f]+)u" % name, hdr)
        assert m and int(m.group(1), 16) == val, name
    assert S.DEVSTAT_GRID_COARSENED & S.DEVSTAT_ERRORS == 0  # information, not an error
    assert S.devstat_names(0) == []
    assert S.devstat_names(S.DEVSTAT_NONFINITE | S.DEVSTAT_GRID_COARSENED) == ["nonfinite", "grid_coarsened"]
    assert S.devstat_names(0x7) == ["nonfinite", "bake_truncated", "index"]


def test_surrogate_arguments_checked_on_the_host():
    """The surrogate's entry points refuse bad arguments before any device
    work: no state, a bad near-field radius, a foreign handle, an empty
    batch, a spot fraction outside (0, 1]."""
    from paper_2510_07729_gb300 import sop as S
    lib = S.load()
    fake = 1 << 20
    h = ctypes.c_void_p()
    assert lib.sop_surrogate_create(None, 1 << 20, None, 0, ctypes.c_float(0.08), ctypes.byref(h), None) == 1
    assert lib.sop_surrogate_create(fake, 1 << 30, None, 0, ctypes.c_float(0.0), ctypes.byref(h), None) == 1
    assert b"r_near" in lib.sop_last_error()
    assert lib.sop_surrogate_create(fake, 16, None, 0, ctypes.c_float(0.08), ctypes.byref(h), None) == 3
    junk = (ctypes.c_uint32 * 16)()
    at = S.AtlasDesc(fake, None, 0, 0, 64, 8, 1.0, fake, None)
    assert lib.sop_surrogate_train(ctypes.byref(junk), fake, None, 64, ctypes.byref(at), 1, ctypes.c_float(1e-3), 0,
                                   None, fake, 1 << 30, None) == 1
    assert b"handle" in lib.sop_last_error()
    assert lib.sop_surrogate_destroy(ctypes.byref(junk)) == 1
    assert lib.sop_surrogate_destroy(None) == 0
    assert lib.sop_surrogate_workspace_bytes(0, 64, 8) == 0
    assert lib.sop_surrogate_workspace_bytes(1000, 64, 8) >= lib.sop_surrogate_train_workspace_bytes()
