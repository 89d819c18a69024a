"""Python binding of libsop (argument marshalling only).

Every function here passes torch CUDA tensors' device pointers and the
current CUDA stream to the C ABI declared in include/sop.h; all arithmetic
runs in the library's kernels. There is no fallback: if libsop.so is missing
or a call fails, an exception is raised.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field

import torch

from . import build as _build

SOP_F32, SOP_BF16, SOP_F16, SOP_FP8E4M3 = 0, 1, 2, 3
MODE_SHADE, MODE_SHADOW = 0, 1
ENV_EQUIRECT, ENV_OCTAHEDRAL = 0, 1
_STATUS = {0: "OK", 1: "INVALID_ARG", 2: "CUDA", 3: "WORKSPACE", 4: "UNSUPPORTED", 5: "TIMEOUT", 6: "DEVICE"}
# bits of the device status word (include/sop.h)
DEVSTAT_NONFINITE, DEVSTAT_BAKE_TRUNCATED, DEVSTAT_INDEX, DEVSTAT_GRID_COARSENED = 0x1, 0x2, 0x4, 0x100
DEVSTAT_CAPACITY, DEVSTAT_TIMEOUT = 0x8, 0x10
DEVSTAT_ERRORS = 0xff
_DEVSTAT_NAMES = {DEVSTAT_NONFINITE: "nonfinite", DEVSTAT_BAKE_TRUNCATED: "bake_truncated", DEVSTAT_INDEX: "index",
                  DEVSTAT_CAPACITY: "capacity", DEVSTAT_TIMEOUT: "timeout", DEVSTAT_GRID_COARSENED: "grid_coarsened"}


def devstat_names(bits):
    """Names of the device status bits set in `bits` (host-side decoding)."""
    return [name for b, name in sorted(_DEVSTAT_NAMES.items()) if bits & b]


class SopError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"libsop {_STATUS.get(status, status)}: {msg}")
        self.status = status


class Gaussians(C.Structure):
    _fields_ = [("mean", C.c_void_p), ("scale", C.c_void_p), ("quat", C.c_void_p), ("opacity", C.c_void_p),
                ("rgb", C.c_void_p), ("n", C.c_int64)]


class AtlasDesc(C.Structure):
    _fields_ = [("rgbo", C.c_void_p), ("depth", C.c_void_p), ("rgbo_dtype", C.c_int32), ("depth_dtype", C.c_int32),
                ("P", C.c_int32), ("R", C.c_int32), ("depth_scale", C.c_float), ("probe_pos", C.c_void_p),
                ("probe_nrm", C.c_void_p)]


class Materials(C.Structure):
    _fields_ = [("albedo", C.c_void_p), ("rough", C.c_void_p), ("metal", C.c_void_p)]


class BakeParams(C.Structure):
    _fields_ = [("t_near", C.c_float), ("alpha_min", C.c_float), ("alpha_max", C.c_float), ("t_stop", C.c_float),
                ("grid_density", C.c_float)]


class AdamParams(C.Structure):
    _fields_ = [("lr", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float),
                ("step", C.c_int32), ("target", C.c_void_p), ("target_value", C.c_float), ("period", C.c_int32),
                ("split", C.c_int32), ("lam", C.c_float * 2), ("lo", C.c_float * 2), ("hi", C.c_float * 2)]


class ShadeParams(C.Structure):
    _fields_ = [("K", C.c_int32), ("S", C.c_int32), ("mode", C.c_int32), ("specular", C.c_float),
                ("eps_snap", C.c_float), ("env_layout", C.c_int32), ("dir_world", C.c_int32), ("radius", C.c_float)]


_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libsop.so (building it first if asked and needed)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise ImportError(f"libsop.so not built ({_build.LIB}); run paper_2510_07729_gb300.build.build()")
    lib = C.CDLL(_build.LIB)
    vp, i32, i64, sz, f32 = C.c_void_p, C.c_int32, C.c_int64, C.c_size_t, C.c_float
    lib.sop_last_error.restype = C.c_char_p
    lib.sop_version.restype = C.c_char_p
    lib.sop_device_status.argtypes = [vp, C.POINTER(C.c_uint32), i32]
    lib.sop_atlas_bytes.argtypes = [i32, i32, i32, i32, C.POINTER(sz), C.POINTER(sz)]
    lib.sop_atlas_pack.argtypes = [vp, vp, vp, C.POINTER(AtlasDesc), vp]
    lib.sop_hammersley.argtypes = [i32, vp, vp]
    lib.sop_read_bandwidth_probe.argtypes = [vp, sz, i32, vp, vp]
    lib.sop_atlas_pack_rgbo.argtypes = [vp, C.POINTER(AtlasDesc), vp]
    lib.sop_env_to_octahedral.argtypes = [vp, i32, i32, vp, i32, vp]
    lib.sop_env_importance_workspace_bytes.argtypes = [i32]
    lib.sop_env_importance_workspace_bytes.restype = sz
    lib.sop_env_importance_dirs.argtypes = [vp, i32, i32, vp, vp, sz, vp]
    lib.sop_l1_loss_grad.argtypes = [vp, vp, i64, vp, vp, vp]
    lib.sop_adam_l1_step.argtypes = [vp, vp, vp, vp, i64, C.POINTER(AdamParams), vp]
    lib.sop_trace_workspace_bytes.argtypes = [i64]
    lib.sop_trace_workspace_bytes.restype = sz
    lib.sop_trace_gbuffer.argtypes = [C.POINTER(Gaussians), C.POINTER(Materials), vp, i32, vp, i64,
                                      C.POINTER(BakeParams), vp, vp, sz, vp]
    f3 = C.POINTER(C.c_float)
    lib.sop_pinhole_dirs.argtypes = [i32, i32, f3, f3, f3, C.c_float, vp, vp]
    lib.sop_panorama_dirs.argtypes = [i32, i32, vp, vp]
    lib.sop_gbuffer_points_workspace_bytes.argtypes = [i64]
    lib.sop_gbuffer_points_workspace_bytes.restype = sz
    lib.sop_gbuffer_points.argtypes = [vp, vp, i64, f3, vp, C.c_float, vp, vp, vp, vp, vp, vp, vp, vp, vp, sz, vp]
    lib.sop_depth_composite.argtypes = [vp, vp, i64, vp, vp, i64, vp, vp, i64, vp, vp]
    lib.sop_place_probes_workspace_bytes.argtypes = [i64]
    lib.sop_place_probes_workspace_bytes.restype = sz
    lib.sop_place_probes.argtypes = [vp, vp, i64, i32, i64, C.c_float, vp, vp, vp, sz, vp]
    lib.sop_bake_workspace_bytes.argtypes = [i64, i32, i32]
    lib.sop_bake_workspace_bytes.restype = sz
    lib.sop_bake.argtypes = [C.POINTER(Gaussians), C.POINTER(AtlasDesc), C.POINTER(BakeParams), vp, sz, vp]
    lib.sop_bake_bin.argtypes = [C.POINTER(Gaussians), C.POINTER(BakeParams), vp, sz, vp]
    lib.sop_bake_trace.argtypes = [C.POINTER(Gaussians), C.POINTER(AtlasDesc), C.POINTER(BakeParams), vp, sz, vp]
    lib.sop_bake_stats.argtypes = [vp, sz, i64, C.POINTER(i64), vp]
    lib.sop_query_workspace_bytes.argtypes = [C.POINTER(AtlasDesc), i64, C.POINTER(ShadeParams), i32, i32]
    lib.sop_query_workspace_bytes.restype = sz
    lib.sop_query_shade.argtypes = [vp, vp, vp, vp, vp, vp, i64, C.POINTER(AtlasDesc), vp, i32, i32, vp,
                                    C.POINTER(ShadeParams), vp, vp, vp, vp, sz, vp]
    lib.sop_query_shade_backward.argtypes = [vp, vp, vp, vp, vp, vp, i64, C.POINTER(AtlasDesc), vp, i32, i32, vp,
                                             C.POINTER(ShadeParams), vp, vp, vp, vp, vp, vp, vp, vp, sz, vp]
    lib.sop_query_shade_noalloc.argtypes = [vp, vp, vp, vp, vp, vp, i64, C.POINTER(AtlasDesc), vp, i32, i32, vp,
                                            C.POINTER(ShadeParams), vp, vp, vp, vp]
    lib.sop_surrogate_param_count.restype = i32
    lib.sop_surrogate_state_bytes.restype = sz
    pp_ = C.POINTER(C.c_void_p)
    lib.sop_surrogate_create.argtypes = [vp, sz, vp, C.c_uint64, f32, pp_, vp]
    lib.sop_surrogate_destroy.argtypes = [vp]
    lib.sop_surrogate_set_params.argtypes = [vp, vp, vp]
    lib.sop_surrogate_get_params.argtypes = [vp, vp, vp]
    lib.sop_surrogate_get_grad.argtypes = [vp, vp, vp]
    lib.sop_surrogate_save.argtypes = [vp, C.c_char_p, vp]
    lib.sop_surrogate_load.argtypes = [vp, C.c_char_p, vp]
    lib.sop_surrogate_file_write.argtypes = [C.c_char_p, i32, i32, vp, vp, vp]
    lib.sop_surrogate_file_read.argtypes = [C.c_char_p, i32, C.POINTER(i32), vp, vp, vp]
    lib.sop_surrogate_workspace_bytes.argtypes = [i64, i32, i32]
    lib.sop_surrogate_workspace_bytes.restype = sz
    lib.sop_surrogate_train_workspace_bytes.restype = sz
    lib.sop_surrogate_features.argtypes = [vp, C.POINTER(Gaussians), vp, i32, i32, C.POINTER(BakeParams), vp, vp, vp,
                                           sz, vp]
    lib.sop_surrogate_train.argtypes = [vp, vp, vp, i32, C.POINTER(AtlasDesc), i32, f32, C.c_uint64, vp, vp, sz, vp]
    lib.sop_surrogate_predict.argtypes = [vp, vp, vp, i32, C.POINTER(AtlasDesc), vp]
    lib.sop_surrogate_infer.argtypes = [vp, C.POINTER(Gaussians), C.POINTER(AtlasDesc), C.POINTER(BakeParams), f32,
                                        f32, C.c_uint64, vp, vp, vp, sz, vp]
    lib.sop_atlas_compare.argtypes = [C.POINTER(AtlasDesc), vp, C.POINTER(AtlasDesc), vp, i32, vp, vp]
    lib.sop_atlas_copy.argtypes = [C.POINTER(AtlasDesc), vp, C.POINTER(AtlasDesc), vp, i32, vp]
    for name in ("sop_surrogate_create", "sop_surrogate_destroy", "sop_surrogate_set_params",
                 "sop_surrogate_get_params", "sop_surrogate_get_grad", "sop_surrogate_save", "sop_surrogate_load",
                 "sop_surrogate_file_write", "sop_surrogate_file_read", "sop_surrogate_features",
                 "sop_surrogate_train", "sop_surrogate_predict", "sop_surrogate_infer", "sop_atlas_compare",
                 "sop_atlas_copy"):
        getattr(lib, name).restype = C.c_int
    for name in ("sop_device_status", "sop_atlas_bytes", "sop_atlas_pack", "sop_hammersley", "sop_bake", "sop_bake_bin", "sop_bake_trace",
                 "sop_bake_stats", "sop_query_shade",
                 "sop_query_shade_backward", "sop_query_shade_noalloc", "sop_read_bandwidth_probe",
                 "sop_atlas_pack_rgbo", "sop_l1_loss_grad", "sop_adam_l1_step", "sop_env_to_octahedral",
                 "sop_env_importance_dirs"):
        getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


def _check(st):
    if st != 0:
        raise SopError(st, load().sop_last_error().decode())


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("libsop takes CUDA tensors")
    if not t.is_contiguous():
        raise ValueError("libsop takes contiguous tensors")
    return C.c_void_p(t.data_ptr())


def _f32(t, shape=None):
    if t.dtype != torch.float32:
        raise TypeError(f"expected float32, got {t.dtype}")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"expected shape {tuple(shape)}, got {tuple(t.shape)}")
    return _ptr(t)


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ws(nbytes, device):
    # 256-byte aligned scratch from torch's caching allocator
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


_TORCH_DT = {SOP_F32: torch.float32, SOP_BF16: torch.bfloat16, SOP_F16: torch.float16,
             SOP_FP8E4M3: torch.float8_e4m3fn}


@dataclass
class Atlas:
    """Caller-owned probe atlas (see sop_atlas in include/sop.h)."""
    rgbo: torch.Tensor
    depth: torch.Tensor | None
    probe_pos: torch.Tensor
    probe_nrm: torch.Tensor | None
    rgbo_dtype: int = SOP_F32
    depth_dtype: int = SOP_F32
    depth_scale: float = 1.0
    desc: AtlasDesc = field(default=None, repr=False)

    @property
    def P(self):
        return self.probe_pos.shape[0]

    @property
    def R(self):
        return self.rgbo.shape[1] - 2

    def c(self):
        d = AtlasDesc()
        d.rgbo = self.rgbo.data_ptr()
        d.depth = self.depth.data_ptr() if self.depth is not None else None
        d.rgbo_dtype, d.depth_dtype = self.rgbo_dtype, self.depth_dtype
        d.P, d.R = self.P, self.R
        d.depth_scale = self.depth_scale
        d.probe_pos = self.probe_pos.data_ptr()
        d.probe_nrm = self.probe_nrm.data_ptr() if self.probe_nrm is not None else None
        self.desc = d
        return d

    def interior(self):
        """Interior texels as float32: rgb [P,R,R,3], occ [P,R,R], depth."""
        R = self.R
        v = self.rgbo.float()[:, 1:R + 1, 1:R + 1]
        dep = None
        if self.depth is not None:
            dep = self.depth.float()[:, 1:R + 1, 1:R + 1] * self.depth_scale
        return v[..., :3], v[..., 3], dep


def make_atlas(probe_pos, R, rgbo_dtype=SOP_F32, depth_dtype=SOP_F32, probe_nrm=None, depth_scale=1.0,
               with_depth=True):
    P = probe_pos.shape[0]
    dev = probe_pos.device
    rgbo = torch.empty((P, R + 2, R + 2, 4), dtype=_TORCH_DT[rgbo_dtype], device=dev)
    depth = torch.empty((P, R + 2, R + 2), dtype=_TORCH_DT[depth_dtype], device=dev) if with_depth else None
    return Atlas(rgbo, depth, probe_pos.contiguous(), probe_nrm, rgbo_dtype, depth_dtype, float(depth_scale))


def version() -> str:
    return load().sop_version().decode()


def device_status(clear=True, raise_on_error=True):
    """sop_device_status on the current stream (synchronises it): returns
    the device status bits; raises SopError (status DEVICE) when an error
    bit is set and raise_on_error."""
    bits = C.c_uint32(0)
    st = load().sop_device_status(_stream(), C.byref(bits), 1 if clear else 0)
    if st != 0 and (raise_on_error or st != 6):
        _check(st)
    return int(bits.value)


def atlas_bytes(P, R, rgbo_dtype=SOP_F32, depth_dtype=SOP_F32):
    a, b = C.c_size_t(), C.c_size_t()
    _check(load().sop_atlas_bytes(P, R, rgbo_dtype, depth_dtype, C.byref(a), C.byref(b)))
    return a.value, b.value


def atlas_pack(maps_rgb, maps_occ, maps_depth, atlas: Atlas):
    P, R = atlas.P, atlas.R
    d = atlas.c()
    _check(load().sop_atlas_pack(_f32(maps_rgb, (P, R, R, 3)), _f32(maps_occ, (P, R, R)),
                                 None if maps_depth is None else _f32(maps_depth, (P, R, R)), C.byref(d), _stream()))
    return atlas


def atlas_pack_rgbo(maps, atlas: Atlas):
    """Pack interleaved maps [P,R,R,4] (L_in RGB, O) into the atlas."""
    P, R = atlas.P, atlas.R
    d = atlas.c()
    _check(load().sop_atlas_pack_rgbo(_f32(maps, (P, R, R, 4)), C.byref(d), _stream()))
    return atlas


def env_to_octahedral(env, H):
    """sop_env_to_octahedral: an equirectangular environment [He,We,3] (device,
    float32) resampled into an octahedral one [H,H,3]."""
    He, We = env.shape[0], env.shape[1]
    out = torch.empty((H, H, 3), dtype=torch.float32, device=env.device)
    _check(load().sop_env_to_octahedral(_f32(env, (He, We, 3)), He, We, _ptr(out), H, _stream()))
    return out


def env_importance_dirs(env_oct, S):
    """sop_env_importance_dirs: S importance-sampled world directions [S,4]
    (x, y, z, pdf) from an octahedral environment [H,H,3] (device, float32),
    for query_shade(..., dirs_world=...)."""
    H = env_oct.shape[0]
    lib = load()
    ws = _ws(int(lib.sop_env_importance_workspace_bytes(H)), env_oct.device)
    out = torch.empty((S, 4), dtype=torch.float32, device=env_oct.device)
    _check(lib.sop_env_importance_dirs(_f32(env_oct, (H, H, 3)), H, S, _ptr(out), _ptr(ws), ws.numel(), _stream()))
    return out


def hammersley(S, device="cuda"):
    out = torch.empty((S, 3), dtype=torch.float32, device=device)
    _check(load().sop_hammersley(S, _ptr(out), _stream()))
    return out


def read_bandwidth_gbs(nbytes, reps, device="cuda", trials=5):
    """Read rate (GB/s) of sop_read_bandwidth_probe over a buffer of nbytes
    read `reps` times (best of `trials`, CUDA events on the current stream,
    after one untimed pass that also makes a small buffer L2-resident)."""
    buf = torch.ones(nbytes // 4, dtype=torch.float32, device=device)
    sink = torch.zeros(1, dtype=torch.float32, device=device)
    lib = load()
    _check(lib.sop_read_bandwidth_probe(_ptr(buf), buf.numel() * 4, 1, _ptr(sink), _stream()))
    best = float("inf")
    for _ in range(trials):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        _check(lib.sop_read_bandwidth_probe(_ptr(buf), buf.numel() * 4, reps, _ptr(sink), _stream()))
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return buf.numel() * 4 * reps / (best * 1e-3) / 1e9


def _gauss(g):
    n = g["mean"].shape[0]
    s = Gaussians()
    s.mean = g["mean"].data_ptr() if n else None
    s.scale = g["scale"].data_ptr() if n else None
    s.quat = g["quat"].data_ptr() if n else None
    s.opacity = g["opacity"].data_ptr() if n else None
    s.rgb = g["rgb"].data_ptr() if n else None
    s.n = n
    for k, shp in (("mean", (n, 3)), ("scale", (n, 3)), ("quat", (n, 4)), ("opacity", (n,)), ("rgb", (n, 3))):
        t = g[k]
        if n:
            _f32(t, shp)
    return s


# ----------------------------------------------------------------------------
# deferred front end: G-buffer trace, camera / panorama rays, shading points,
# depth compositing
# ----------------------------------------------------------------------------
def _f3(v):
    return (C.c_float * 3)(*[float(a) for a in v])


class GbufferTracer:
    """Multi-target rendering of one Gaussian set with per-Gaussian
    materials: bins the Gaussians once (sop_bake_bin), then traces any
    origins x directions (sop_trace_gbuffer) into [rays, 16] G-buffers
    (C.rgb, W, N.xyz, D, A.rgb, R, M, 0, 0, 0)."""

    def __init__(self, gauss, mats, t_near=0.0, alpha_min=1.0 / 255.0, alpha_max=0.99, t_stop=1e-4,
                 grid_density=0.06):
        self.gauss, self.mats = gauss, mats
        n = gauss["mean"].shape[0]
        # camera rays cross many cells they do not stop in: a coarser grid
        # than the probe bake's (0.35 cells per Gaussian) walks faster
        self.params = (t_near, alpha_min, alpha_max, t_stop, grid_density)
        self.ws = BakeWorkspace(n, gauss["mean"].device)
        bake_bin(gauss, self.ws, *self.params)
        for k, shp in (("albedo", (n, 3)), ("rough", (n,)), ("metal", (n,))):
            _f32(mats[k], shp)
        self.m = Materials(mats["albedo"].data_ptr() if n else None, mats["rough"].data_ptr() if n else None,
                           mats["metal"].data_ptr() if n else None)

    def trace(self, origins, dirs, out=None):
        """origins [n_o, 3], dirs [n_d, 4] float32 CUDA tensors; returns out
        [n_o * n_d, 16]."""
        lib = load()
        no, nd = origins.shape[0], dirs.shape[0]
        _f32(origins, (no, 3))
        _f32(dirs, (nd, 4))
        if out is None:
            out = torch.empty((no * nd, 16), dtype=torch.float32, device=dirs.device)
        _f32(out, (no * nd, 16))
        g = _gauss(self.gauss)
        bp = _bake_params(*self.params)
        _check(lib.sop_trace_gbuffer(C.byref(g), C.byref(self.m), _ptr(origins), no, _ptr(dirs), nd, C.byref(bp),
                                     _ptr(out), _ptr(self.ws.buf), self.ws.buf.numel(), _stream()))
        return out


def pinhole_dirs(W, H, eye, target, fov_y_deg, up=(0.0, 0.0, 1.0), device="cuda"):
    out = torch.empty((H * W, 4), dtype=torch.float32, device=device)
    _check(load().sop_pinhole_dirs(W, H, _f3(eye), _f3(target), _f3(up), float(fov_y_deg), _ptr(out), _stream()))
    return out


def panorama_dirs(W, H, device="cuda"):
    out = torch.empty((H * W, 4), dtype=torch.float32, device=device)
    _check(load().sop_panorama_dirs(W, H, _ptr(out), _stream()))
    return out


def gbuffer_points(gbuf, origin, dirs, w_min=0.5, front=None, count_only=False):
    """Shading points of a G-buffer [n, 16] (see sop_gbuffer_points):
    returns (pix [k] int64, dict x, n, wo, albedo [k,3], rough, metal [k]).
    Reads the count back (one synchronisation)."""
    lib = load()
    n = gbuf.shape[0]
    dev = gbuf.device
    _f32(gbuf, (n, 16))
    _f32(dirs, (n, 4))
    if front is not None:
        _f32(front, (n, 16))
    pix = torch.empty(n, dtype=torch.int64, device=dev)
    v3 = [torch.empty((n, 3), dtype=torch.float32, device=dev) for _ in range(4)]
    v1 = [torch.empty(n, dtype=torch.float32, device=dev) for _ in range(2)]
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    ws = _ws(lib.sop_gbuffer_points_workspace_bytes(n), dev)
    _check(lib.sop_gbuffer_points(_ptr(gbuf), _ptr(front), n, _f3(origin), _ptr(dirs), float(w_min), _ptr(pix),
                                  *[_ptr(t) for t in v3], *[_ptr(t) for t in v1], _ptr(cnt), _ptr(ws), ws.numel(),
                                  _stream()))
    k = int(cnt.item())
    pts = dict(x=v3[0][:k], n=v3[1][:k], wo=v3[2][:k], albedo=v3[3][:k], rough=v1[0][:k], metal=v1[1][:k])
    return pix[:k], pts


def depth_composite(scene_gbuf, obj_gbuf, sc_pix, shadow, obj_pix, obj_rgb, out=None):
    lib = load()
    n = scene_gbuf.shape[0]
    _f32(scene_gbuf, (n, 16))
    _f32(obj_gbuf, (n, 16))
    if out is None:
        out = torch.empty((n, 3), dtype=torch.float32, device=scene_gbuf.device)
    ns, no = sc_pix.shape[0], obj_pix.shape[0]
    for t in (sc_pix, obj_pix):
        if t.dtype != torch.int64:
            raise TypeError("pixel lists are int64")
    _f32(shadow, (ns, 3))
    _f32(obj_rgb, (no, 3))
    _check(lib.sop_depth_composite(_ptr(scene_gbuf), _ptr(obj_gbuf), n, _ptr(sc_pix) if ns else None,
                                   _ptr(shadow) if ns else None, ns, _ptr(obj_pix) if no else None,
                                   _ptr(obj_rgb) if no else None, no, _ptr(out), _stream()))
    return out


def place_probes(pts, k, nrm=None, offset=0.0, start=0):
    """Automatic placement (sop_place_probes): farthest point sampling of
    pts [n,3] with exact integer keys, offset along nrm [n,3]. Returns
    (idx [k] int64, positions [k,3])."""
    lib = load()
    n = pts.shape[0]
    _f32(pts, (n, 3))
    if nrm is not None:
        _f32(nrm, (n, 3))
    idx = torch.empty(k, dtype=torch.int64, device=pts.device)
    pos = torch.empty((k, 3), dtype=torch.float32, device=pts.device)
    ws = _ws(lib.sop_place_probes_workspace_bytes(n), pts.device)
    _check(lib.sop_place_probes(_ptr(pts), _ptr(nrm), n, k, start, float(offset), _ptr(idx), _ptr(pos), _ptr(ws),
                                ws.numel(), _stream()))
    return idx, pos


def bake_workspace_bytes(n_gauss, P, R):
    return int(load().sop_bake_workspace_bytes(n_gauss, P, R))


class BakeWorkspace:
    """Scratch for the bake of one Gaussian set (sop_bake_workspace_bytes;
    extra_bytes adds room for more grid cell entries)."""

    def __init__(self, n_gauss, device, extra_bytes=0):
        self.n = int(n_gauss)
        self.buf = _ws(bake_workspace_bytes(self.n, 1, 2) + int(extra_bytes), device)


def _bake_params(t_near, alpha_min, alpha_max, t_stop, grid_density=0.0):
    return BakeParams(t_near, alpha_min, alpha_max, t_stop, grid_density)


def bake_bin(gauss, workspace: BakeWorkspace, t_near=0.0, alpha_min=1.0 / 255.0, alpha_max=0.99, t_stop=1e-4,
             grid_density=0.0):
    """Bin the Gaussians into the grid kept in the workspace (asynchronous;
    the grid is coarsened on the device if its cell lists would overflow the
    workspace). grid_density: grid cells per Gaussian (0: the default, 0.35)."""
    lib = load()
    g = _gauss(gauss)
    bp = _bake_params(t_near, alpha_min, alpha_max, t_stop, grid_density)
    ws = workspace
    _check(lib.sop_bake_bin(C.byref(g), C.byref(bp), _ptr(ws.buf), ws.buf.numel(), _stream()))
    return ws


def bake_trace(gauss, atlas: Atlas, workspace: BakeWorkspace, t_near=0.0, alpha_min=1.0 / 255.0, alpha_max=0.99,
               t_stop=1e-4):
    """Trace every texel of the atlas through the binned grid (async)."""
    lib = load()
    g = _gauss(gauss)
    bp = _bake_params(t_near, alpha_min, alpha_max, t_stop)
    d = atlas.c()
    _check(lib.sop_bake_trace(C.byref(g), C.byref(d), C.byref(bp), _ptr(workspace.buf), workspace.buf.numel(),
                              _stream()))
    return atlas


def bake_stats(workspace: BakeWorkspace):
    """(exact evaluations, composited hits, status bits, cell entries tested)
    of the last trace."""
    out = (C.c_int64 * 4)()
    _check(load().sop_bake_stats(_ptr(workspace.buf), workspace.buf.numel(), workspace.n, out, _stream()))
    return int(out[0]), int(out[1]), int(out[2]), int(out[3])


_bake_ws = {}


def bake(gauss, atlas: Atlas, t_near=0.0, alpha_min=1.0 / 255.0, alpha_max=0.99, t_stop=1e-4, workspace=None):
    """Bake every texel of `atlas` against the Gaussians (dict of CUDA
    float32 tensors: mean, scale, quat, opacity, rgb): bin + trace.
    Asynchronous; device_status() reports non-finite inputs or truncated
    rays."""
    n = int(gauss["mean"].shape[0])
    dev = atlas.rgbo.device
    ws = workspace
    if ws is None:
        ws = _bake_ws.get((dev, n))
        if ws is None:
            _bake_ws.clear()
            ws = _bake_ws[(dev, n)] = BakeWorkspace(n, dev)
    bake_bin(gauss, ws, t_near, alpha_min, alpha_max, t_stop)
    bake_trace(gauss, atlas, ws, t_near, alpha_min, alpha_max, t_stop)
    return atlas


def query_workspace_bytes(atlas: Atlas, M, K, S, He, We, mode=MODE_SHADE):
    sp = ShadeParams(K, S, mode, 0.5, 1e-6)
    d = atlas.c()
    return int(load().sop_query_workspace_bytes(C.byref(d), M, C.byref(sp), He, We))


def query_shade(x, n, wo, albedo, rough, metal, atlas: Atlas, env, K, S, mode=MODE_SHADE, specular=0.5,
                eps_snap=1e-6, dirs_local=None, out=None, return_idx=False, workspace=None, env_layout=ENV_EQUIRECT,
                dirs_world=None, radius=0.0):
    """SOP query + shade of M points; returns out [M,3] (and idx [M,K] int32,
    W [M,K] float32 when return_idx). radius > 0: fixed-radius neighbours
    (at most K probes within it; idx -1 and W 0 in the empty slots)."""
    lib = load()
    M = x.shape[0]
    He, We = env.shape[0], env.shape[1]
    dev = x.device
    sp = ShadeParams(K, S, mode, specular, eps_snap, env_layout, 0 if dirs_world is None else 1, radius)
    if dirs_world is not None:
        dl = _f32(dirs_world, (S, 4))
    else:
        dl = None if dirs_local is None else _f32(dirs_local, (S, 3))
    d = atlas.c()
    if out is None:
        out = torch.empty((M, 3), dtype=torch.float32, device=dev)
    idx = torch.empty((M, K), dtype=torch.int32, device=dev) if return_idx else None
    w = torch.empty((M, K), dtype=torch.float32, device=dev) if return_idx else None
    need = int(lib.sop_query_workspace_bytes(C.byref(d), M, C.byref(sp), He, We))
    ws = workspace if workspace is not None else _ws(need, dev)
    for t, shp in ((x, (M, 3)), (n, (M, 3)), (wo, (M, 3)), (albedo, (M, 3)), (rough, (M,)), (metal, (M,)),
                   (env, (He, We, 3))):
        _f32(t, shp)
    _check(lib.sop_query_shade(_ptr(x), _ptr(n), _ptr(wo), _ptr(albedo), _ptr(rough), _ptr(metal), M, C.byref(d),
                               _ptr(env), He, We, dl,
                               C.byref(sp), _ptr(out), _ptr(idx), _ptr(w), _ptr(ws), ws.numel(), _stream()))
    if return_idx:
        return out, idx, w
    return out


def query_shade_backward(x, n, wo, albedo, rough, metal, atlas: Atlas, env, K, S, grad_out, g_env=None, g_maps=None,
                         specular=0.5, eps_snap=1e-6, dirs_local=None, workspace=None, radius=0.0):
    """sop_query_shade_backward (SHADE mode). Returns a dict of gradients:
    albedo, rough, metal, normal (fresh tensors) and env [He,We,3], maps
    [P,R,R,4] (accumulated into g_env / g_maps when given, else zeros)."""
    lib = load()
    M = x.shape[0]
    He, We = env.shape[0], env.shape[1]
    dev = x.device
    P, R = atlas.P, atlas.R
    sp = ShadeParams(K, S, MODE_SHADE, specular, eps_snap, ENV_EQUIRECT, 0, radius)
    d = atlas.c()
    g = dict(albedo=torch.empty((M, 3), dtype=torch.float32, device=dev),
             rough=torch.empty((M,), dtype=torch.float32, device=dev),
             metal=torch.empty((M,), dtype=torch.float32, device=dev),
             normal=torch.empty((M, 3), dtype=torch.float32, device=dev),
             env=g_env if g_env is not None else torch.zeros((He, We, 3), dtype=torch.float32, device=dev),
             maps=g_maps if g_maps is not None else torch.zeros((P, R, R, 4), dtype=torch.float32, device=dev))
    _f32(grad_out, (M, 3))
    _f32(g["env"], (He, We, 3))
    _f32(g["maps"], (P, R, R, 4))
    need = int(lib.sop_query_workspace_bytes(C.byref(d), M, C.byref(sp), He, We))
    ws = workspace if workspace is not None else _ws(need, dev)
    _check(lib.sop_query_shade_backward(
        _ptr(x), _ptr(n), _ptr(wo), _ptr(albedo), _ptr(rough), _ptr(metal), M, C.byref(d), _ptr(env), He, We,
        None if dirs_local is None else _f32(dirs_local, (S, 3)), C.byref(sp), _ptr(grad_out), _ptr(g["albedo"]),
        _ptr(g["rough"]), _ptr(g["metal"]), _ptr(g["normal"]), _ptr(g["env"]), _ptr(g["maps"]), _ptr(ws),
        ws.numel(), _stream()))
    return g


class SopQueryShade(torch.autograd.Function):
    """Differentiable SOP query + shade (SHADE mode) over compact probe maps.

    forward(x, n, wo, albedo, rough, metal, maps [P,R,R,4] (RGB, O), env
    [He,We,3], probe_pos [P,3], K, S) packs the maps into a float32 atlas and
    shades; backward calls the hand-written adjoint."""

    @staticmethod
    def forward(ctx, x, n, wo, albedo, rough, metal, maps, env, probe_pos, K, S):
        P, R = maps.shape[0], maps.shape[1]
        at = make_atlas(probe_pos, R, with_depth=False)
        atlas_pack_rgbo(maps.contiguous(), at)
        out = query_shade(x, n, wo, albedo, rough, metal, at, env, K, S)
        ctx.save_for_backward(x, n, wo, albedo, rough, metal, env)
        ctx.at, ctx.K, ctx.S = at, K, S
        return out

    @staticmethod
    def backward(ctx, grad_out):
        x, n, wo, albedo, rough, metal, env = ctx.saved_tensors
        g = query_shade_backward(x, n, wo, albedo, rough, metal, ctx.at, env, ctx.K, ctx.S,
                                 grad_out.contiguous().float())
        return None, g["normal"], None, g["albedo"], g["rough"], g["metal"], g["maps"], g["env"], None, None, None


def query_shade_noalloc(x, n, wo, albedo, rough, metal, atlas: Atlas, env, K, S, mode=MODE_SHADE, specular=0.5,
                        eps_snap=1e-6, dirs_local=None, out=None, return_idx=False, radius=0.0):
    """sop_query_shade_noalloc: the same query + shade without a workspace,
    for callers that cannot allocate device memory (the library's fixed
    scratch array is used instead; see include/sop.h)."""
    lib = load()
    M = x.shape[0]
    He, We = env.shape[0], env.shape[1]
    dev = x.device
    sp = ShadeParams(K, S, mode, specular, eps_snap, ENV_EQUIRECT, 0, radius)
    d = atlas.c()
    if out is None:
        out = torch.empty((M, 3), dtype=torch.float32, device=dev)
    idx = torch.empty((M, K), dtype=torch.int32, device=dev) if return_idx else None
    w = torch.empty((M, K), dtype=torch.float32, device=dev) if return_idx else None
    for t, shp in ((x, (M, 3)), (n, (M, 3)), (wo, (M, 3)), (albedo, (M, 3)), (rough, (M,)), (metal, (M,)),
                   (env, (He, We, 3))):
        _f32(t, shp)
    _check(lib.sop_query_shade_noalloc(_ptr(x), _ptr(n), _ptr(wo), _ptr(albedo), _ptr(rough), _ptr(metal), M,
                                       C.byref(d), _ptr(env), He, We,
                                       None if dirs_local is None else _f32(dirs_local, (S, 3)), C.byref(sp),
                                       _ptr(out), _ptr(idx), _ptr(w), _stream()))
    if return_idx:
        return out, idx, w
    return out


# ----------------------------------------------------------------------------
# learned bake surrogate
# ----------------------------------------------------------------------------
def _i32(t):
    if t is None:
        return None
    if t.dtype != torch.int32:
        raise TypeError(f"expected int32, got {t.dtype}")
    return _ptr(t)


class Surrogate:
    """The learned bake surrogate (sop_surrogate handle over a caller-owned
    device state). params: initial parameters (sop_surrogate_param_count()
    floats) or None for the library's seeded He-uniform initialisation;
    r_near: the near-field radius of the texel features."""

    N_FEATURES = 18
    NEAR_CAP = 256

    def __init__(self, params=None, device="cuda", r_near=0.08, seed=0):
        lib = load()
        self.n_params = int(lib.sop_surrogate_param_count())
        self.device = torch.device(device)
        self.state = _ws(int(lib.sop_surrogate_state_bytes()), self.device)
        self.r_near = float(r_near)
        p = None
        if params is not None:
            p = torch.as_tensor(params, dtype=torch.float32).to(self.device).contiguous()
            if p.numel() != self.n_params:
                raise ValueError(f"expected {self.n_params} parameters")
        h = C.c_void_p()
        _check(lib.sop_surrogate_create(_ptr(self.state), self.state.numel(), _ptr(p), C.c_uint64(seed),
                                        C.c_float(self.r_near), C.byref(h), _stream()))
        self._keep = p
        self.h = h
        self._ws = {}

    def __del__(self):
        try:
            if getattr(self, "h", None) and self.h.value:
                load().sop_surrogate_destroy(self.h)
                self.h = C.c_void_p()
        except Exception:
            pass

    def set_params(self, params):
        p = torch.as_tensor(params, dtype=torch.float32).to(self.device).contiguous()
        if p.numel() != self.n_params:
            raise ValueError(f"expected {self.n_params} parameters")
        _check(load().sop_surrogate_set_params(self.h, _ptr(p), _stream()))
        self._keep = p

    def params(self):
        out = torch.empty(self.n_params, dtype=torch.float32, device=self.device)
        _check(load().sop_surrogate_get_params(self.h, _ptr(out), _stream()))
        return out

    def grad(self):
        out = torch.empty(self.n_params, dtype=torch.float32, device=self.device)
        _check(load().sop_surrogate_get_grad(self.h, _ptr(out), _stream()))
        return out

    def save(self, path):
        _check(load().sop_surrogate_save(self.h, str(path).encode(), _stream()))

    def load_file(self, path):
        _check(load().sop_surrogate_load(self.h, str(path).encode(), _stream()))

    def workspace(self, n_gauss, P, R):
        key = (int(n_gauss), int(P), int(R))
        if key not in self._ws:
            self._ws.clear()
            self._ws[key] = _ws(int(load().sop_surrogate_workspace_bytes(*key)), self.device)
        return self._ws[key]

    def features(self, gauss, probe_pos, R, alpha_min=1.0 / 255.0, alpha_max=0.99, with_list=False):
        """Texel features [P, R*R, 18] (and the near lists [P, 256] int32)."""
        P = probe_pos.shape[0]
        g = _gauss(gauss)
        feats = torch.empty((P, R * R, self.N_FEATURES), dtype=torch.float32, device=self.device)
        lst = torch.empty((P, self.NEAR_CAP), dtype=torch.int32, device=self.device) if with_list else None
        ws = self.workspace(g.n, P, R)
        bp = _bake_params(0.0, alpha_min, alpha_max, 1e-4)
        _check(load().sop_surrogate_features(self.h, C.byref(g), _f32(probe_pos, (P, 3)), P, R, C.byref(bp),
                                             _ptr(feats), _ptr(lst), _ptr(ws), ws.numel(), _stream()))
        return (feats, lst) if with_list else feats

    def train(self, feats, targets: Atlas, steps=1, batch=64, lr=1e-3, seed=0, probe_ids=None, losses=None):
        """`steps` Adam steps on `batch` probes each (probe_ids [batch] int32,
        or drawn on the device from seed and the step count). losses: a
        device float32 tensor [steps] for each step's loss, or None."""
        d = targets.c()
        B = probe_ids.shape[0] if probe_ids is not None else batch
        if getattr(self, "_train_ws", None) is None:
            self._train_ws = _ws(int(load().sop_surrogate_train_workspace_bytes()), self.device)
        ws = self._train_ws
        _check(load().sop_surrogate_train(self.h, _ptr(feats), _i32(probe_ids), B, C.byref(d), steps, C.c_float(lr),
                                          C.c_uint64(seed), _ptr(losses), _ptr(ws), ws.numel(), _stream()))
        return losses

    def predict(self, feats, out: Atlas, probe_ids=None):
        B = probe_ids.shape[0] if probe_ids is not None else out.P
        d = out.c()
        _check(load().sop_surrogate_predict(self.h, _ptr(feats), _i32(probe_ids), B, C.byref(d), _stream()))
        return out

    def rebake(self, gauss, out: Atlas, spot_frac=0.01, tau=0.05, seed=0, alpha_min=1.0 / 255.0, alpha_max=0.99,
               t_stop=1e-4):
        """sop_surrogate_infer: the learned rebake of every probe of `out`
        with its spot check and fallback, decided on the device. Returns
        (spot-check mean |dO|, fell back) as device tensors."""
        g = _gauss(gauss)
        d = out.c()
        bp = _bake_params(0.0, alpha_min, alpha_max, t_stop)
        err = torch.empty(1, dtype=torch.float32, device=self.device)
        fell = torch.empty(1, dtype=torch.int32, device=self.device)
        ws = self.workspace(g.n, out.P, out.R)
        _check(load().sop_surrogate_infer(self.h, C.byref(g), C.byref(d), C.byref(bp), C.c_float(spot_frac),
                                          C.c_float(tau), C.c_uint64(seed), _ptr(err), _ptr(fell), _ptr(ws),
                                          ws.numel(), _stream()))
        return err, fell


def surrogate_file_write(path, step, params, m, v):
    """The checkpoint format from host arrays (no GPU)."""
    import numpy as np
    arrs = [np.ascontiguousarray(a, dtype=np.float32) for a in (params, m, v)]
    n = arrs[0].size
    _check(load(build_if_missing=False).sop_surrogate_file_write(
        str(path).encode(), n, int(step), *[a.ctypes.data_as(C.c_void_p) for a in arrs]))


def surrogate_file_read(path, n):
    """(step, params, m, v) of a checkpoint file of n parameters (no GPU)."""
    import numpy as np
    arrs = [np.empty(n, np.float32) for _ in range(3)]
    step = C.c_int32(0)
    _check(load(build_if_missing=False).sop_surrogate_file_read(
        str(path).encode(), n, C.byref(step), *[a.ctypes.data_as(C.c_void_p) for a in arrs]))
    return int(step.value), arrs[0], arrs[1], arrs[2]


def atlas_compare(a: Atlas, b: Atlas, a_probes=None, b_probes=None, n=None):
    """(sum |dO|, sum |dRGB|) over the interior texels of n probe pairs."""
    n = n if n is not None else (a_probes.shape[0] if a_probes is not None else a.P)
    out = torch.empty(2, dtype=torch.float32, device=a.rgbo.device)
    da, db = a.c(), b.c()
    _check(load().sop_atlas_compare(C.byref(da), _i32(a_probes), C.byref(db), _i32(b_probes), n, _ptr(out),
                                    _stream()))
    return out


def atlas_copy(src: Atlas, dst: Atlas, src_probes=None, dst_probes=None, n=None):
    n = n if n is not None else (src_probes.shape[0] if src_probes is not None else src.P)
    ds, dd = src.c(), dst.c()
    _check(load().sop_atlas_copy(C.byref(ds), _i32(src_probes), C.byref(dd), _i32(dst_probes), n, _stream()))


def l1_loss_grad(C_, C_target, grad=None, loss_sum=None):
    """sop_l1_loss_grad: grad = sign(C - C_target) / n; adds sum |C - C_target|
    to loss_sum (one float, zeroed by the caller) when given."""
    n = C_.numel()
    grad = grad if grad is not None else torch.empty_like(C_)
    _check(load().sop_l1_loss_grad(_f32(C_), _f32(C_target, tuple(C_.shape)), n, _ptr(grad),
                                   None if loss_sum is None else _ptr(loss_sum), _stream()))
    return grad


def adam_l1_step(p, g, m, v, step, lr, target=None, target_value=0.0, lam=(0.0, 0.0), lo=(-3.0e38, -3.0e38),
                 hi=(3.0e38, 3.0e38), period=1, split=1, beta1=0.9, beta2=0.999, eps=1e-8):
    """sop_adam_l1_step on one parameter block, in place."""
    a = AdamParams(lr, beta1, beta2, eps, step, None if target is None else _ptr(target), target_value, period, split,
                   (C.c_float * 2)(*lam), (C.c_float * 2)(*lo), (C.c_float * 2)(*hi))
    _check(load().sop_adam_l1_step(_ptr(p), None if g is None else _ptr(g), _ptr(m), _ptr(v), p.numel(), C.byref(a),
                                   _stream()))
    return p


class TextureOptimizer:
    """The second reconstruction step of Sec. 3.1.2: Adam on the environment
    map, the per-point albedo, roughness and metallic (lr 0.01) and the SOP
    textures {L_in, O} (lr 0.001) against L = L_pbr + lam_lam L_lam +
    lam_sops L_sops, with L_pbr the mean absolute error of the shaded RGB,
    L_lam = L1(R, 1) + L1(M, 0) and L_sops = L1(L_in, L_tr) + L1(O, O_tr)
    against the ray-traced maps. Parameters are clamped after each step
    (albedo, metallic, O to [0, 1]; roughness to [0.1, 1]; environment and
    L_in to [0, inf)). Every step runs in the library's kernels: pack, shade,
    loss gradient, adjoint, one fused regularise + Adam + clamp per block."""

    def __init__(self, albedo, rough, metal, env, maps, traced_maps, probe_pos, lr_mat=0.01, lr_sop=0.001,
                 lam_lam=0.001, lam_sops=1.0):
        self.p = {k: t.detach().float().contiguous().clone() for k, t in
                  dict(albedo=albedo, rough=rough, metal=metal, env=env, maps=maps).items()}
        self.m = {k: torch.zeros_like(t) for k, t in self.p.items()}
        self.v = {k: torch.zeros_like(t) for k, t in self.p.items()}
        self.traced = traced_maps.float().contiguous()
        self.lr_mat, self.lr_sop, self.lam_lam, self.lam_sops = lr_mat, lr_sop, lam_lam, lam_sops
        P, R = maps.shape[0], maps.shape[1]
        self.atlas = make_atlas(probe_pos, R, with_depth=False)
        self.g_env = torch.zeros_like(self.p["env"])
        self.g_maps = torch.zeros_like(self.p["maps"])
        self.loss_sum = torch.zeros(1, dtype=torch.float32, device=maps.device)
        self.t = 0
        self.ws = None

    def step(self, x, n, wo, target, K, S):
        """One step; returns the L_pbr of the shading before the update (a
        device scalar)."""
        p = self.p
        M = x.shape[0]
        atlas_pack_rgbo(p["maps"], self.atlas)
        He, We = p["env"].shape[0], p["env"].shape[1]
        if self.ws is None:
            self.ws = _ws(query_workspace_bytes(self.atlas, M, K, S, He, We), x.device)
        C_ = query_shade(x, n, wo, p["albedo"], p["rough"], p["metal"], self.atlas, p["env"], K, S, workspace=self.ws)
        self.loss_sum.zero_()
        gC = l1_loss_grad(C_, target, loss_sum=self.loss_sum)
        self.g_env.zero_()
        self.g_maps.zero_()
        g = query_shade_backward(x, n, wo, p["albedo"], p["rough"], p["metal"], self.atlas, p["env"], K, S, gC,
                                 g_env=self.g_env, g_maps=self.g_maps, workspace=self.ws)
        self.t += 1
        t, lm, ls = self.t, self.lr_mat, self.lr_sop
        inf = 3.0e38
        adam_l1_step(p["albedo"], g["albedo"], self.m["albedo"], self.v["albedo"], t, lm, lo=(0.0, 0.0), hi=(1.0, 1.0))
        lam = self.lam_lam / M
        adam_l1_step(p["rough"], g["rough"], self.m["rough"], self.v["rough"], t, lm, target_value=1.0, lam=(lam, lam),
                     lo=(0.1, 0.1), hi=(1.0, 1.0))
        adam_l1_step(p["metal"], g["metal"], self.m["metal"], self.v["metal"], t, lm, target_value=0.0, lam=(lam, lam),
                     lo=(0.0, 0.0), hi=(1.0, 1.0))
        adam_l1_step(p["env"], self.g_env, self.m["env"], self.v["env"], t, lm, lo=(0.0, 0.0), hi=(inf, inf))
        texels = p["maps"].shape[0] * p["maps"].shape[1] * p["maps"].shape[2]
        adam_l1_step(p["maps"], self.g_maps, self.m["maps"], self.v["maps"], t, ls, target=self.traced,
                     lam=(self.lam_sops / (3 * texels), self.lam_sops / texels), lo=(0.0, 0.0), hi=(inf, 1.0),
                     period=4, split=3)
        return self.loss_sum / (3 * M)
