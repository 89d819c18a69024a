"""Benchmark of the SOP hot path on GB300: probe bake + probe query/shade.

One step = one pass of the whole path over the 1920x1080 composition
workload (an object of 200,000 anisotropic Gaussians on a 1M-Gaussian
ground-and-clutter scene): sop_bake of all 8,192 probes (4,096 on the
object and 4,096 shadow-region probes on the ground, 16x16 each, 2,097,152
texel rays traced through the object's Gaussians: binning, grid walk,
compositing, atlas border) followed by the frame's two sop_query_shade
calls: the 21,907 object pixels in SHADE mode against the object probes and
the 2,051,693 scene pixels in SHADOW mode against the shadow-region probes
(K=8, S=64, 256x512 HDR environment). The two queries are independent and
are issued on two streams: the small SHADE call's launches run beside the
SHADOW call instead of before it. `value` is shaded point-directions per
second of that step; the bake's texels/s is reported beside it. The
object-reconstruction workload (4,096 probes, 418,111 points, K=8, S=128) is
timed the same way as a secondary line (`object_step`).

Usage (driver contract):
  python bench.py [--gpus N --steps K --warmup W] [--impl ours|reference]
Multi-GPU: one replica per rank (the path shards by independent probes and
points; no collective on the data path), weak scaling.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

L2_FLUSH_BYTES = 512 << 20
FP32_LANES_PER_SM = 128
N_SMS = 152


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="compose", choices=["compose", "object", "tiny"])
    ap.add_argument("--part", default="step",
                    choices=["step", "bake", "query", "compose", "optimize", "deferred", "surrogate"],
                    help="profiling aid: run only one half (the JSON line then covers that half), only the "
                         "1080p composition-frame query, or only the learned rebake (untrained network)")
    ap.add_argument("--probes", type=int, default=0, help="profiling aid: bake only the first N probes")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-surrogate", action="store_true", help="skip the learned-rebake measurement")
    ap.add_argument("--no-compose", action="store_true", help="skip the 1080p composition-frame query measurement")
    ap.add_argument("--no-optimize", action="store_true", help="skip the texture-optimisation step measurement")
    ap.add_argument("--no-deferred", action="store_true", help="skip the deferred (G-buffer) frame measurement")
    return ap.parse_args()


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                r = subprocess.run(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                    "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=5)
                if r.returncode == 0 and r.stdout.strip():
                    self.samples.append([v.strip() for v in r.stdout.strip().split(",")])
            except Exception:
                pass
            self._stop.wait(0.05)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if len(s) > 5 + i and
                          s[5 + i].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


# ----------------------------------------------------------------------------
# workload
# ----------------------------------------------------------------------------
def load_workload(name):
    """A workload: Gaussians, all probes (one atlas, baked in one call) and
    its query parts, each a point set with its mode and its slice of the
    atlas's probes."""
    from paper_2510_07729_gb300 import inputs as I
    keys = ("x", "n", "wo", "albedo", "rough", "metal")
    if name in ("object", "tiny"):
        c = I.make_object() if name == "object" else I.make_tiny()
        P = len(c["probe_pos"])
        return dict(name=name, gauss=c["gauss"], probe_pos=c["probe_pos"], R=c["R"], env=c["env"], K=c["K"],
                    S=c["S"], depth_scale=float(c.get("object_size", 2.0)),
                    parts=[dict(name="shade", mode=0, probes=(0, P), pts={k: c[k] for k in keys})],
                    label=f"{name}: {len(c['gauss']['mean'])} Gaussians, {P} probes {c['R']}x{c['R']}, "
                          f"{len(c['x'])} points SHADE, K={c['K']}, S={c['S']}, env {c['env'].shape[0]}x"
                          f"{c['env'].shape[1]}")
    c = I.make_compose()
    po, ps = c["shade"]["probe_pos"], c["shadow"]["probe_pos"]
    Po, Ps = len(po), len(ps)
    n_scene = len(c["gauss_scene"]["mean"])
    n_obj = len(c["gauss_object"]["mean"])
    return dict(name="compose", gauss=c["gauss_object"], probe_pos=np.concatenate([po, ps]), R=c["R"], env=c["env"],
                K=c["K"], S=c["S"], depth_scale=float(c["object_size"]),
                parts=[dict(name="shade", mode=0, probes=(0, Po), pts={k: c["shade"][k] for k in keys}),
                       dict(name="shadow", mode=1, probes=(Po, Po + Ps), pts={k: c["shadow"][k] for k in keys})],
                label=f"compose 1920x1080: object {n_obj} Gaussians in a {n_scene}-Gaussian scene; {Po} object + "
                      f"{Ps} shadow-region probes {c['R']}x{c['R']} baked against the object; "
                      f"{len(c['shade']['x'])} object pixels SHADE + {len(c['shadow']['x'])} scene pixels SHADOW, "
                      f"K={c['K']}, S={c['S']}, env {c['env'].shape[0]}x{c['env'].shape[1]}")


def atlas_view(sop, atlas, lo, hi):
    """The probes [lo, hi) of an atlas as an atlas of their own (views of the
    same memory: probe-major storage makes each slice contiguous)."""
    return sop.Atlas(atlas.rgbo[lo:hi], None if atlas.depth is None else atlas.depth[lo:hi],
                     atlas.probe_pos[lo:hi], None, atlas.rgbo_dtype, atlas.depth_dtype, atlas.depth_scale)


# algorithmic FP32 work of one shaded point-direction (K probes, SHADE mode):
# frame rotation 15, octahedral encode 12, texel coordinates 10, per probe
# 4 bilinear weights x 4 channels (16 FMA = 32 FLOP) + 4 weight products,
# environment uv 2 atan2 (~40) + bilinear 3x4 FMA (24) + weights 8, BRDF
# (half vector 12, dots 15, D 8, G 4, Fresnel 12, combine 12) and the
# accumulation 9.
# algorithmic FP32 work of the bake: a box test of one grid-cell entry
# against a ray (centre decode 3 add + 3 FMA = 9, offset from the probe 3,
# slab scaling 6, entries and exits 6, their max/min 4, the walk's start 1:
# ~29), an exact ray-Gaussian evaluation (the probe offset split into two
# parts 18, M*offset 15, M*direction 15, A and B 10, t* 2, closest point 9,
# M*point 15, m^2 5, response 4: ~93) and one composited hit (1 - alpha,
# transmittance, weight, 3 colour, depth and weight sums: ~15)
FLOP_PER_TEST = 29
FLOP_PER_EVAL = 93
FLOP_PER_COMPOSITE = 15


def measured_peaks():
    """(HBM GB/s, source) from the measured-peaks file at the repository
    root, else the fallback copy bandwidth of an earlier GB300 measurement."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


def traffic_for(kernel, workload, P):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on this workload with all of its probes and on the current source of the
    kernel (else None)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            tab = json.load(f)
    except (OSError, ValueError):
        return None
    e = tab.get(kernel)
    if not e or e.get("workload") != workload or e.get("probes") != P:
        return None
    src = os.path.join(ROOT, "paper_2510_07729_gb300", "csrc", e["source"])
    try:
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    if h != e.get("source_sha256_16"):
        return None
    return e.get("bytes")


def chosen_variant(sop, g, ppos, R, pargs, env, K, S, mode, out_ref, flush, steps):
    """The reduced-precision atlas (FP16 RGBO, FP32 accumulation): query
    throughput and its relative L1 difference from the FP32-atlas output."""
    import torch
    at16 = sop.make_atlas(ppos, R, rgbo_dtype=sop.SOP_F16, depth_dtype=sop.SOP_F16)
    sop.bake(g, at16)
    M = pargs[0].shape[0]
    out = torch.empty((M, 3), dtype=torch.float32, device=pargs[0].device)
    ws = torch.empty(sop.query_workspace_bytes(at16, M, K, S, env.shape[0], env.shape[1], mode), dtype=torch.uint8,
                     device=pargs[0].device)
    for _ in range(3):
        sop.query_shade(*pargs, at16, env, K, S, mode=mode, out=out, workspace=ws)
    ts = []
    for _ in range(steps):
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        sop.query_shade(*pargs, at16, env, K, S, mode=mode, out=out, workspace=ws)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    ms = float(np.mean(ts))
    rel = ((out - out_ref).abs().sum() / out_ref.abs().sum()).item()
    return {"atlas": "fp16 RGBO + fp16 depth, fp32 accumulation", "query_ms": round(ms, 4),
            "query_point_dirs_per_s": round(M * S / (ms * 1e-3), 1), "rel_l1_vs_fp32_atlas": rel}


def env_oct_variant(sop, atlas, pargs, env, K, S, mode, out_ref, flush, steps, H=256):
    """The query with the environment in the paper's octahedral layout
    (Sec. 4.1): the 256x512 equirectangular map resampled on the GPU to
    256x256; the lookup reuses the direction's octahedral coordinates (no
    atan2). Time and relative L1 difference from the equirectangular result
    (a resampling difference, not an error)."""
    import torch
    env_oct = sop.env_to_octahedral(env, H)
    M = pargs[0].shape[0]
    out = torch.empty((M, 3), dtype=torch.float32, device=pargs[0].device)
    ws = torch.empty(sop.query_workspace_bytes(atlas, M, K, S, H, H, mode), dtype=torch.uint8, device=out.device)

    def call():
        sop.query_shade(*pargs, atlas, env_oct, K, S, mode=mode, out=out, workspace=ws,
                        env_layout=sop.ENV_OCTAHEDRAL)

    for _ in range(3):
        call()
    ts = []
    for _ in range(steps):
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        call()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    ms = float(np.mean(ts))
    rel = ((out - out_ref).abs().sum() / out_ref.abs().sum()).item()
    return {"env": f"octahedral {H}x{H} (resampled from the equirectangular map)", "query_ms": round(ms, 4),
            "query_point_dirs_per_s": round(M * S / (ms * 1e-3), 1), "rel_l1_vs_equirect": rel}


def frnn_variant(sop, atlas, pargs, env, K, S, mode, out_ref, flush, steps, ppos):
    """The query with the fixed-radius neighbour search (Sec. 3.2; the paper
    does not give its radius): the radius is the median distance of the 4th
    nearest probe over 512 evenly spaced points, so a point keeps from one
    to K probes. Time, mean number of neighbours and relative L1 difference
    from the plain K nearest (a different blend, not an error)."""
    import torch
    x = pargs[0]
    M = x.shape[0]
    sub = x[torch.linspace(0, M - 1, 512, device=x.device).long()]
    d = torch.cdist(sub.double(), ppos.double()).sort(dim=1).values[:, 3]
    radius = float(np.float32(d.median().item()))
    out = torch.empty((M, 3), dtype=torch.float32, device=x.device)
    ws = torch.empty(sop.query_workspace_bytes(atlas, M, K, S, env.shape[0], env.shape[1], mode), dtype=torch.uint8,
                     device=x.device)
    _, idx, _ = sop.query_shade(*pargs, atlas, env, K, S, mode=mode, return_idx=True, radius=radius)
    n_mean = (idx >= 0).float().sum(1).mean().item()

    def call():
        sop.query_shade(*pargs, atlas, env, K, S, mode=mode, out=out, workspace=ws, radius=radius)

    for _ in range(3):
        call()
    ts = []
    for _ in range(steps):
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        call()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    ms = float(np.mean(ts))
    rel = ((out - out_ref).abs().sum() / out_ref.abs().sum()).item()
    return {"radius": radius, "neighbours_mean": round(n_mean, 3), "query_ms": round(ms, 4),
            "query_point_dirs_per_s": round(M * S / (ms * 1e-3), 1), "rel_l1_vs_knn": rel}


def rebake_only(sop, dev, flush, steps, warmup, n_probes=0, r_near=0.08):
    """Profiling aid: the learned rebake of the moved-object scene (its first
    n_probes probes, all when 0) with an untrained network and the fallback
    off (tau huge), so that every launch runs features, network and the
    spot check. The kernels' work does not depend on the weights."""
    import torch
    from paper_2510_07729_gb300 import inputs as I
    mv = I.moved_object()
    gt = {k: torch.from_numpy(np.ascontiguousarray(v)).to(dev) for k, v in mv["gauss"].items()}
    pp = mv["probe_pos"][:n_probes] if n_probes > 0 else mv["probe_pos"]
    pp = torch.from_numpy(np.ascontiguousarray(pp)).to(dev)
    net = sop.Surrogate(I.surrogate_init(0), device=dev, r_near=r_near)
    out = sop.make_atlas(pp, 16)
    for _ in range(warmup):
        net.rebake(gt, out, spot_frac=0.01, tau=1e30, seed=3)
    ts = []
    for _ in range(steps):
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        net.rebake(gt, out, spot_frac=0.01, tau=1e30, seed=3)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    ms = float(np.mean(ts)) if ts else 0.0
    texels = out.P * out.R * out.R
    return {"probes": out.P, "ms": round(ms, 4), "texels_per_s": round(texels / (ms * 1e-3), 1) if ms else 0.0}


def surrogate_variant(sop, dev, flush, steps, n_scenes=25, train_steps=30000, r_near=0.08):
    """The learned rebake after the object's first ellipsoid moves: train on
    ray-traced bakes of random scenes (untimed), then time the rebake of the
    moved scene's 4,096 probes (sop_surrogate_infer: binning, features,
    network, 1% spot check against the ray-traced bake, fallback when the
    check fails, all decided on the device) beside the plain bake, with the
    errors against the exact bake and the shading error they cause."""
    import torch
    from paper_2510_07729_gb300 import inputs as I

    def cu(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    net = sop.Surrogate(I.surrogate_init(0), device=dev, r_near=r_near)
    feats, atl = [], []
    for s in range(n_scenes):
        sc = I.surrogate_scene(1000 + s)
        gt = {k: cu(v) for k, v in sc["gauss"].items()}
        at = sop.make_atlas(cu(sc["probe_pos"]), 16)
        sop.bake(gt, at)
        atl.append(at)
        feats.append(net.features(gt, cu(sc["probe_pos"]), 16))
    rng = np.random.default_rng(0)
    chunk = 50
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for it in range(0, train_steps, chunk):
        j = int(rng.integers(n_scenes))
        net.train(feats[j], atl[j], steps=chunk, batch=64, lr=2e-3 if it < 0.7 * train_steps else 5e-4, seed=it)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    mv = I.moved_object()
    gt = {k: cu(v) for k, v in mv["gauss"].items()}
    pp = cu(mv["probe_pos"])
    exact = sop.make_atlas(pp, 16)
    bws = sop.BakeWorkspace(len(mv["gauss"]["mean"]), dev)
    out = sop.make_atlas(pp, 16)

    def timed(fn):
        for _ in range(2):
            fn()
        ts = []
        for _ in range(max(3, steps // 2)):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.mean(ts))

    t_plain = timed(lambda: sop.bake(gt, exact, workspace=bws))
    res = {}
    t_rebake = timed(lambda: res.update(r=net.rebake(gt, out, spot_frac=0.01, tau=0.05, seed=3)))
    err, fell = (t.item() for t in res["r"])
    fe = net.features(gt, pp, 16)
    pred = sop.make_atlas(pp, 16)
    net.predict(fe, pred)
    texels = 4096 * 256
    e_tr = sop.atlas_compare(exact, pred)[0].item() / texels
    e_out = sop.atlas_compare(exact, out)[0].item() / texels
    stale = sop.make_atlas(pp, 16)
    sop.bake({k: cu(v) for k, v in I.make_object()["gauss"].items()}, stale)
    e_st = sop.atlas_compare(exact, stale)[0].item() / texels
    f = fe.cpu().numpy()
    heur = 1 - (1 - f[..., 3]) * (1 - f[..., 14])
    e_heur = float(np.abs(heur - exact.interior()[1].cpu().numpy().reshape(4096, 256)).mean())
    t_feat = timed(lambda: net.features(gt, pp, 16))
    t_pred = timed(lambda: net.predict(fe, pred))
    pts = [cu(mv[k]) for k in ("x", "n", "wo", "albedo", "rough", "metal")]
    env = cu(mv["env"])
    C_exact = sop.query_shade(*pts, exact, env, mv["K"], mv["S"])
    C_out = sop.query_shade(*pts, out, env, mv["K"], mv["S"])
    rel = ((C_out - C_exact).abs().sum() / C_exact.abs().sum()).item()
    return {"what": "learned rebake (sop_surrogate_infer: binning, texel features, MLP, 1% spot check against the "
                    "ray-traced bake, fallback above mean |dO| 0.05, decided on the device) of 4,096 probes after the "
                    "object's first ellipsoid moved, against the plain ray-traced bake of the same probes",
            "train": f"{n_scenes} random scenes x 4096 probes, {train_steps} Adam steps of 64 probes "
                     f"({t_train:.1f} s)",
            "rebake_ms": round(t_rebake, 4), "plain_bake_ms": round(t_plain, 4),
            "rebake_texels_per_s": round(texels / (t_rebake * 1e-3), 1),
            "speedup_vs_plain": round(t_plain / t_rebake, 3), "fell_back": bool(fell),
            "mean_abs_dO": {"surrogate": round(e_tr, 5), "rebaked_atlas": round(e_out, 5),
                            "spot_check_estimate": round(err, 5), "stale_atlas": round(e_st, 5),
                            "features_without_network": round(e_heur, 5)},
            "shading_rel_l1_vs_exact_atlas": round(rel, 6),
            "parts_ms": {"features_with_binning": round(t_feat, 4), "network": round(t_pred, 4)}}


def l2_read_peak_gbs(dev):
    """L2 read bandwidth measured in this run: the library's read probe over
    a 64 MB buffer (resident in the 126 MB L2) read 40 times in one launch."""
    from paper_2510_07729_gb300 import sop
    return sop.read_bandwidth_gbs(64 << 20, 40, device=dev)


def query_demand(K, mode, texel_bytes, M, S, n_normals):
    """Algorithmic bytes that the SMs must receive from L2/L1 for M points
    with n_normals distinct normals: per point-direction the 4 texels of each
    of K probe footprints (RGBO in SHADE mode, O alone in SHADOW mode); per
    distinct (normal, direction) the 4 environment texels (RGB fp32), since
    points on one normal share their light directions."""
    per_texel = texel_bytes if mode == 0 else texel_bytes // 4
    return K * 4 * per_texel * M * S + 4 * 12 * n_normals * S


def deferred_frame_variant(sop, dev, flush, steps):
    """The whole composed 1920x1080 frame of the deferred front end (Sec. 4.3):
    camera rays; G-buffers of the object (200k surfels with materials) and
    of the scene (1M surfels) traced exactly (every Gaussian evaluated once
    per ray, hits in (t*, index) order); the object's shading points in
    front of the scene SHADE-d against the 4,096 object probes and the
    scene's points SHADOW-ed against the 4,096 shadow-region probes (K=8,
    S=64; both atlases baked from the object's Gaussians, untimed); depth
    compositing. Plus the 360 degree panorama (1024x512 G-buffer) at the
    object's placement through the scene (Sec. 4.2)."""
    import torch
    from paper_2510_07729_gb300 import inputs as I
    d = I.make_deferred()
    K, S, R, W, H = d["K"], d["S"], d["R"], d["W"], d["H"]

    def cu(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    go = {k: cu(v) for k, v in d["gauss_object"].items()}
    gs = {k: cu(v) for k, v in d["gauss_scene"].items()}
    tro = sop.GbufferTracer(go, {k: cu(v) for k, v in d["mats_object"].items()})
    trs = sop.GbufferTracer(gs, {k: cu(v) for k, v in d["mats_scene"].items()})
    env = cu(d["env"])
    at_o = sop.make_atlas(cu(d["obj_probe_pos"]), R)
    at_s = sop.make_atlas(cu(d["scene_probe_pos"]), R)
    sop.bake(go, at_o)
    sop.bake(go, at_s)
    eye = d["eye"]
    eye_t = cu(eye[None])
    n = W * H
    gb_o = torch.empty((n, 16), dtype=torch.float32, device=dev)
    gb_s = torch.empty((n, 16), dtype=torch.float32, device=dev)
    frame = torch.empty((n, 3), dtype=torch.float32, device=dev)
    ev = []

    def mark():
        e = torch.cuda.Event(enable_timing=True)
        e.record()
        ev.append(e)

    def render():
        ev.clear()
        mark()
        dirs = sop.pinhole_dirs(W, H, eye, d["target"], d["fov"], device=dev)
        tro.trace(eye_t, dirs, out=gb_o)
        mark()
        trs.trace(eye_t, dirs, out=gb_s)
        mark()
        pix_o, po = sop.gbuffer_points(gb_o, eye, dirs, 0.5, front=gb_s)
        pix_s, ps = sop.gbuffer_points(gb_s, eye, dirs, 0.5)
        mark()
        rgb = sop.query_shade(po["x"], po["n"], po["wo"], po["albedo"], po["rough"], po["metal"], at_o, env, K, S)
        sh = sop.query_shade(ps["x"], ps["n"], ps["wo"], ps["albedo"], ps["rough"], ps["metal"], at_s, env, K, S,
                             mode=sop.MODE_SHADOW)
        mark()
        sop.depth_composite(gb_s, gb_o, pix_s, sh, pix_o, rgb, out=frame)
        mark()
        return len(pix_o), len(pix_s)

    for _ in range(2):
        render()
    torch.cuda.synchronize()
    names = ("rays_and_object_gbuffer", "scene_gbuffer", "shading_points", "query_shade", "composite")
    tot, parts = [], {k: [] for k in names}
    for _ in range(steps):
        flush.fill_(1)
        n_o, n_s = render()
        torch.cuda.synchronize()
        tot.append(ev[0].elapsed_time(ev[-1]))
        for i, k in enumerate(names):
            parts[k].append(ev[i].elapsed_time(ev[i + 1]))
    ms = float(np.mean(tot))
    # panorama at the placement location through the scene
    pano = sop.panorama_dirs(1024, 512, device=dev)
    org = cu(np.array([[float(d["target"][0]), float(d["target"][1]), float(d["target"][2])]], np.float32))
    pg = torch.empty((1024 * 512, 16), dtype=torch.float32, device=dev)
    for _ in range(2):
        trs.trace(org, pano, out=pg)
    tp = []
    for _ in range(steps):
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        trs.trace(org, pano, out=pg)
        e1.record()
        torch.cuda.synchronize()
        tp.append(e0.elapsed_time(e1))
    covered = float((pg[:, 3] > 0.5).float().mean().item())
    # automatic placement (Sec. 3.2): G-buffers of the object from 8 views
    # around it, their shading points as the surface cloud, FPS of 4,096
    # probes offset by 1% of the object's size along the normals
    cams = [np.array([3.0 * np.cos(a) * np.cos(e), 3.0 * np.sin(a) * np.cos(e), 3.0 * np.sin(e)], np.float32)
            for a, e in zip(np.linspace(0, 2 * np.pi, 8, endpoint=False), [0.5, -0.3] * 4)]
    tpl, tfps, npts = [], [], 0
    for _ in range(max(1, steps // 2)):
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record()
        xs, ns = [], []
        for cam in cams:
            vd = sop.pinhole_dirs(512, 512, cam, np.zeros(3, np.float32), 40.0, device=dev)
            vg = tro.trace(cu(cam[None]), vd)
            _, vp = sop.gbuffer_points(vg, cam, vd, 0.5)
            xs.append(vp["x"])
            ns.append(vp["n"])
        cloud, cn = torch.cat(xs), torch.cat(ns)
        e1.record()
        sop.place_probes(cloud, 4096, nrm=cn, offset=0.01 * float(d["object_size"]))
        e2.record()
        torch.cuda.synchronize()
        npts = int(cloud.shape[0])
        tpl.append(e0.elapsed_time(e2))
        tfps.append(e1.elapsed_time(e2))
    return {"what": "composed 1920x1080 frame from G-buffers traced through 200k object and 1M scene surfels: "
                    "points, SHADE + SHADOW queries (K=8, S=64), depth compositing",
            "frame_ms": round(ms, 3), "fps": round(1000.0 / ms, 1),
            "parts_ms": {k: round(float(np.mean(v)), 3) for k, v in parts.items()},
            "object_points": n_o, "scene_points": n_s,
            "panorama_1024x512_ms": round(float(np.mean(tp)), 3), "panorama_covered": round(covered, 4),
            "placement": {"views": len(cams), "points": npts, "probes": 4096, "fps_ms": round(float(np.mean(tfps)), 3),
                          "views_and_fps_ms": round(float(np.mean(tpl)), 3)}}


def _rel_errors(gpu, ref):
    gpu, ref = np.asarray(gpu, np.float64), np.asarray(ref, np.float64)
    scale = np.maximum(np.abs(ref), 1e-3 * np.abs(ref).mean())
    return {"rel_l1": float(np.abs(gpu - ref).sum() / np.abs(ref).sum()),
            "max_rel": float((np.abs(gpu - ref) / scale).max())}


def compose_frame_variant(sop, dev, flush, steps, l2_gbs, hbm_gbs, peak_fp32, baked=None, n_shadow=4096,
                          n_shade=1024):
    """The 1920x1080 composition frame: the two sop_query_shade calls (object
    pixels SHADE against the 4,096 object probes, scene pixels SHADOW
    against the 4,096 shadow-region probes, K=8, S=64), timed for float32,
    bfloat16 and float16 atlases (each baked once, untimed), with the HBM,
    L2 and FP32 roofs of the frame. Every precision's output is compared
    with the FP64 oracle on a seeded sample of points (4,096 scene pixels,
    1,024 object pixels), the oracle shading with the float32 bake's maps;
    the depth plane's storage types (float32, float16, bfloat16, FP8 E4M3)
    are compared with the oracle's own bake of 16 sampled probes."""
    import torch

    import oracle
    W = load_workload("compose")
    K, S, R = W["K"], W["S"], W["R"]
    if baked is None:
        baked = StepState(sop, W, dev)
        baked.bake()
    states = {"fp32": baked}
    for dt, label in ((sop.SOP_BF16, "bf16"), (sop.SOP_F16, "fp16")):
        s = StepState(sop, W, dev, rgbo_dtype=dt, depth_dtype=dt)
        s.bake()
        states[label] = s
    parts = baked.parts
    normals = {q["name"]: len(np.unique(p["pts"]["n"], axis=0)) for q, p in zip(parts, W["parts"])}
    res = {"what": "1920x1080 composition frame: sop_query_shade of the object pixels (SHADE) and of the scene "
                   "pixels (SHADOW), K=8, S=64, 2x4,096 probes at 16x16",
           "points": {q["name"]: q["M"] for q in parts}, "distinct_normals": normals}
    tex_bytes = {"fp32": 16, "bf16": 8, "fp16": 8}
    for label, st in states.items():
        for _ in range(3):
            for q in st.parts:
                st.query(q)
        torch.cuda.synchronize()
        ts, tp = [], {q["name"]: [] for q in st.parts}
        for _ in range(steps):
            flush.fill_(1)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(st.parts) + 1)]
            ev[0].record()
            for i, q in enumerate(st.parts):
                st.query(q)
                ev[i + 1].record()
            torch.cuda.synchronize()
            ts.append(ev[0].elapsed_time(ev[-1]))
            for i, q in enumerate(st.parts):
                tp[q["name"]].append(ev[i].elapsed_time(ev[i + 1]))
        ms = float(np.mean(ts))
        pd = st.M * S
        fl = sum((flop_per_point_dir(K, q["mode"]) - FLOP_DIR_GEOMETRY) * q["M"] * S +
                 FLOP_DIR_GEOMETRY * normals[q["name"]] * S for q in st.parts)
        dem = sum(query_demand(K, q["mode"], tex_bytes[label], q["M"], S, normals[q["name"]]) for q in st.parts)
        hbm = 68 * st.M + st.atlas.rgbo.numel() * st.atlas.rgbo.element_size() + st.env.numel() * 4
        t_hbm, t_l2, t_alu = hbm / (hbm_gbs * 1e9), dem / (l2_gbs * 1e9), fl / (peak_fp32 * 1e12)
        bound = max((t_hbm, "hbm"), (t_l2, "l2"), (t_alu, "alu"))
        res[label] = {"frame_ms": round(ms, 4),
                      **{f"{q['name']}_ms": round(float(np.mean(tp[q["name"]])), 4) for q in st.parts},
                      "point_dirs_per_s": round(pd / (ms * 1e-3), 1),
                      "roofline": {"kernel": "shade_kernel (the frame's two sop_query_shade calls)",
                                   "bound": bound[1], "t_hbm_ms": round(t_hbm * 1e3, 4),
                                   "t_l2_ms": round(t_l2 * 1e3, 4), "t_alu_ms": round(t_alu * 1e3, 4),
                                   "frac": round(bound[0] * 1e3 / ms, 4), "l2_demand_bytes": int(dem),
                                   "hbm_bytes": int(hbm), "flop": int(fl)}}
    # errors against the FP64 oracle on sampled points (the oracle shades
    # with the float32 bake's maps; the 16-bit atlases round those maps)
    rng = np.random.default_rng(2024)
    prec = {}
    for iq, (q, part) in enumerate(zip(parts, W["parts"])):
        n = min(n_shadow if q["mode"] == 1 else n_shade, q["M"])
        sel = np.sort(rng.choice(q["M"], n, replace=False))
        lo, hi = part["probes"]
        rgb, occ, _ = q["at"].interior()
        ref, _, _ = oracle.query_shade(*[part["pts"][k][sel] for k in ("x", "n", "wo", "albedo", "rough", "metal")],
                                       W["probe_pos"][lo:hi], rgb.cpu().numpy(), occ.cpu().numpy(), W["env"], K, S,
                                       mode=q["mode"])
        selt = torch.from_numpy(sel).to(dev)
        for label, st in states.items():
            out = st.parts[iq]["out"][selt].cpu().numpy()
            prec.setdefault(label, {})[q["name"]] = _rel_errors(out, ref)
    for label in states:
        prec[label]["atlas"] = {"fp32": "float32 RGBO (16 B/texel)", "bf16": "bfloat16 RGBO (8 B/texel)",
                                "fp16": "float16 RGBO (8 B/texel)"}[label]
        prec[label]["frame_ms"] = res[label]["frame_ms"]
    prec["sample"] = (f"{n_shadow} scene pixels (SHADOW) and {n_shade} object pixels (SHADE), seeded; the oracle "
                      f"shades with the float32 bake's maps, so the 16-bit rows include the storage rounding")
    prec["depth"] = depth_precision(sop, W, dev)
    res["precision"] = prec
    res["chosen"] = {"atlas": "fp16 RGBO, fp32 accumulation", "frame_ms": res["fp16"]["frame_ms"],
                     "point_dirs_per_s": res["fp16"]["point_dirs_per_s"],
                     "speedup_vs_fp32_frame": round(res["fp32"]["frame_ms"] / res["fp16"]["frame_ms"], 4),
                     "error_vs_oracle": {k: v for k, v in prec["fp16"].items() if k in ("shade", "shadow")}}
    # the paper's rendering configuration: the environment as a 512x512
    # octahedral texture (Sec. 4.1) and S importance-sampled world directions
    # (Sec. 4.2, Eq. PDF) shared by all points, float32 atlas
    env_oct = sop.env_to_octahedral(baked.env, 512)
    dirs = sop.env_importance_dirs(env_oct, S)
    ref_mean = parts[1]["out"].mean().item()
    wsi = [torch.empty(sop.query_workspace_bytes(q["at"], q["M"], K, S, 512, 512, q["mode"]), dtype=torch.uint8,
                       device=dev) for q in parts]
    outs = [torch.empty_like(q["out"]) for q in parts]

    def call_is():
        for q, w, o in zip(parts, wsi, outs):
            sop.query_shade(*q["pts"], q["at"], env_oct, K, S, mode=q["mode"], out=o, workspace=w,
                            env_layout=sop.ENV_OCTAHEDRAL, dirs_world=dirs)

    for _ in range(3):
        call_is()
    torch.cuda.synchronize()
    ts = []
    for _ in range(steps):
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        call_is()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    ms = float(np.mean(ts))
    res["fp32_octahedral_importance"] = {
        "env": "octahedral 512x512 resampled from the equirectangular map; S importance-sampled world directions",
        "frame_ms": round(ms, 4), "point_dirs_per_s": round(baked.M * S / (ms * 1e-3), 1),
        "shadow_mean_vs_hammersley": round(float(outs[1].mean().item()) / ref_mean, 4)}
    res["peaks"] = {"l2_read_gbs": round(l2_gbs, 1), "l2_note": "measured in this run (sop_read_bandwidth_probe: "
                    "a 64 MB L2-resident buffer read 40 times, 16-byte loads on every SM)", "hbm_gbs": hbm_gbs,
                    "hbm_note": "MEASURED_PEAKS.json copy bandwidth", "fp32_tflops": round(peak_fp32, 1),
                    "fp32_note": "derived: 152 SMs x 128 lanes x 2 x 2.07 GHz"}
    return res


def depth_precision(sop, W, dev, n_probes=16):
    """The depth plane in each storage type (D / depth_scale, depth_scale =
    the object's bounding-box diagonal) against the FP64 oracle's bake of
    the same sampled probes (half object, half shadow-region), over the
    texels that hit something; texels the oracle flags as order- or
    threshold-ambiguous are left out."""
    import torch

    import oracle
    rng = np.random.default_rng(77)
    P = len(W["probe_pos"])
    sel = np.sort(np.concatenate([rng.choice(P // 2, n_probes // 2, replace=False),
                                  P // 2 + rng.choice(P - P // 2, n_probes - n_probes // 2, replace=False)]))
    pp = W["probe_pos"][sel]
    _, o_occ, o_dep, fl = oracle.bake(W["gauss"], pp, W["R"])
    ok = (fl == 0) & (o_occ > 0)
    g = {k: torch.from_numpy(np.ascontiguousarray(v)).to(dev) for k, v in W["gauss"].items()}
    ds = W["depth_scale"]
    out = {"probes": int(n_probes), "texels_compared": int(ok.sum()), "depth_scale": round(ds, 4),
           "note": "the query reads O and L_in only; the depth plane is the unbiased depth D/W of the bake"}
    for dt, label in ((sop.SOP_F32, "fp32"), (sop.SOP_F16, "fp16"), (sop.SOP_BF16, "bf16"),
                      (sop.SOP_FP8E4M3, "fp8_e4m3")):
        at = sop.make_atlas(torch.from_numpy(np.ascontiguousarray(pp)).to(dev), W["R"], depth_dtype=dt,
                            depth_scale=ds)
        sop.bake(g, at)
        _, _, dep = at.interior()
        d = dep.cpu().numpy().astype(np.float64)
        err = np.abs(d[ok] - o_dep[ok])
        out[label] = {"mean_abs_over_scale": float(err.mean() / ds), "max_abs_over_scale": float(err.max() / ds),
                      "mean_rel": float((err / np.maximum(o_dep[ok], 1e-6)).mean())}
    return out


# the part of flop_per_point_dir that depends only on the normal and the
# direction: frame rotation, octahedral encode, texel coordinates, environment
FLOP_DIR_GEOMETRY = 15 + 12 + 10 + 40 + 24 + 8


def flop_per_point_dir(K, mode):
    # SHADOW mode blends the occlusion alone: 4 FMA per probe (one per
    # footprint corner), then the 4 bilinear weights once (7)
    f = 15 + 12 + 10 + (K * (32 + 4) if mode == 0 else K * 8 + 7) + 40 + 24 + 8 + 9
    if mode == 0:
        f += 12 + 15 + 8 + 4 + 12 + 12
    return f


def reduce_max(vals, world, device):
    """Per-rank timings -> their maximum over ranks (the slowest rank sets
    the time of a weak-scaling step)."""
    if world <= 1:
        return [float(v) for v in vals]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in vals], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def whole_job_value(units_per_rank, ms_step, world):
    """Units processed by all ranks per second of the (max-over-ranks) step."""
    return world * units_per_rank / (ms_step * 1e-3)


class StepState:
    """Device state of one workload's step: Gaussians, the atlas of all its
    probes, and each query part's points, atlas view, output and workspace."""

    def __init__(self, sop, W, dev, n_probes=0, rgbo_dtype=0, depth_dtype=0):
        import torch

        def cu(a):
            return torch.from_numpy(np.ascontiguousarray(a)).to(dev)

        self.sop, self.W, self.dev = sop, W, dev
        self.g = {k: cu(v) for k, v in W["gauss"].items()}
        P_all = len(W["probe_pos"])
        self.P = P_all if n_probes <= 0 else min(n_probes, P_all)
        self.full = self.P == P_all
        self.ppos = cu(W["probe_pos"][:self.P])
        self.R, self.K, self.S = W["R"], W["K"], W["S"]
        self.env = cu(W["env"])
        self.atlas = sop.make_atlas(self.ppos, self.R, rgbo_dtype=rgbo_dtype, depth_dtype=depth_dtype,
                                    depth_scale=W["depth_scale"])
        self.bws = sop.BakeWorkspace(len(W["gauss"]["mean"]), dev)
        # the frame's queries are independent (own points, atlas slice,
        # output and workspace; the atlas and environment are read-only):
        # the smaller ones run on a second stream beside the largest
        self.side = torch.cuda.Stream(device=dev)
        self.parts = []
        for part in W["parts"]:
            q = dict(name=part["name"], mode=part["mode"], M=len(part["pts"]["x"]))
            q["pts"] = [cu(part["pts"][k]) for k in ("x", "n", "wo", "albedo", "rough", "metal")]
            if self.full:
                q["at"] = atlas_view(sop, self.atlas, *part["probes"])
                q["out"] = torch.empty((q["M"], 3), dtype=torch.float32, device=dev)
                q["ws"] = torch.empty(sop.query_workspace_bytes(q["at"], q["M"], self.K, self.S, self.env.shape[0],
                                                                self.env.shape[1], q["mode"]),
                                      dtype=torch.uint8, device=dev)
            self.parts.append(q)
        self.M = sum(q["M"] for q in self.parts)

    def bake(self):
        self.sop.bake_bin(self.g, self.bws)
        self.sop.bake_trace(self.g, self.atlas, self.bws)

    def query(self, q, **kw):
        self.sop.query_shade(*q["pts"], q["at"], self.env, self.K, self.S, mode=q["mode"], out=q["out"],
                             workspace=q["ws"], **kw)

    def step(self, evs, do_bake=True, do_query=True):
        import torch
        st = torch.cuda.current_stream()
        if do_bake:
            evs[0].record(st)
            self.sop.bake_bin(self.g, self.bws)
            evs[4].record(st)
            self.sop.bake_trace(self.g, self.atlas, self.bws)
            evs[1].record(st)
        if do_query:
            evs[2].record(st)
            big = max(self.parts, key=lambda q: q["M"])
            rest = [q for q in self.parts if q is not big]
            if rest:
                self.side.wait_stream(st)
                with torch.cuda.stream(self.side):
                    for q in rest:
                        self.query(q)
            self.query(big)
            if rest:
                st.wait_stream(self.side)
            evs[3].record(st)


def time_steps(state, flush, steps, warmup, do_bake, do_query, world=1, clock_index=None):
    """Times `steps` whole steps with CUDA events on the current stream (L2
    flushed before each, outside the events), after `warmup` untimed ones,
    with a barrier and a synchronisation on both sides; nvidia-smi clocks
    are sampled during the timed region when clock_index is given."""
    import contextlib

    import torch
    import torch.distributed as dist
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    for _ in range(warmup):
        flush.fill_(1)
        state.step([ev() for _ in range(5)], do_bake, do_query)
    torch.cuda.synchronize()
    records = []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(clock_index) if clock_index is not None else contextlib.nullcontext()
    t_wall0 = time.perf_counter()
    with clk:
        for _ in range(steps):
            flush.fill_(1)
            evs = [ev() for _ in range(5)]
            state.step(evs, do_bake, do_query)
            records.append(evs)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    r = {"bake": [e[0].elapsed_time(e[1]) for e in records] if do_bake else [0.0],
         "trace": [e[4].elapsed_time(e[1]) for e in records] if do_bake else [0.0],
         "query": [e[2].elapsed_time(e[3]) for e in records] if do_query else [0.0], "wall_s": t_wall}
    r["ms_step"] = float(np.sum(r["bake"]) + np.sum(r["query"])) / steps
    r["clocks"] = clk.summary() if clock_index is not None else None
    return r


def trace_roofline(sop, state, ms_trace, peak_fp32):
    """The bake's trace kernel against the FP32 ALU roof: its own work
    counters (box tests, exact evaluations, composited hits of the last
    trace on the workspace) x their FP32 operations / the CUDA-event time."""
    n_eval, n_comp, status, n_test = sop.bake_stats(state.bws)
    fl = n_test * FLOP_PER_TEST + n_eval * FLOP_PER_EVAL + n_comp * FLOP_PER_COMPOSITE
    ach = fl / (ms_trace * 1e-3) / 1e12
    rays = state.P * state.R * state.R
    return {"kernel": "trace_kernel (sop_bake_trace)", "bound": "alu", "achieved": round(ach, 3),
            "peak": round(peak_fp32, 1), "unit": "TFLOP/s", "frac": round(ach / peak_fp32, 4),
            "traffic": traffic_for("trace_kernel", state.W["name"], state.P),
            "work": {"rays": rays, "box_tests": n_test, "exact_evaluations": n_eval, "composited_hits": n_comp,
                     "per_ray": {"box_tests": round(n_test / rays, 2), "exact_evaluations": round(n_eval / rays, 2),
                                 "composited_hits": round(n_comp / rays, 2)},
                     "status_bits": status, "flop_per_box_test": FLOP_PER_TEST,
                     "flop_per_evaluation": FLOP_PER_EVAL, "flop_per_composite": FLOP_PER_COMPOSITE},
            "ms": round(ms_trace, 4),
            "peak_note": "FP32 FMA peak 152 SMs x 128 lanes x 2 x 2.07 GHz (derived from unit counts and the "
                         "maximum clock; the measured-peaks file holds no FP32 figure)"}


def object_step_variant(sop, dev, flush, steps, peak_fp32):
    """The object-reconstruction workload's step (bake of 4,096 probes +
    SHADE query of 418,111 points, K=8, S=128), timed like the headline
    step, with its trace roofline, the FP16-atlas query and the query
    variants of the paper (octahedral environment, fixed-radius search)."""
    W = load_workload("object")
    st = StepState(sop, W, dev)
    r = time_steps(st, flush, steps, 3, True, True)
    q = st.parts[0]
    mb, mq, mt = (float(np.mean(r[k])) for k in ("bake", "query", "trace"))
    pd = st.M * st.S
    res = {"workload": W["label"], "ms_per_step": round(r["ms_step"], 4),
           "point_dirs_per_s": round(pd / (r["ms_step"] * 1e-3), 1),
           "bake": {"ms": round(mb, 4), "texels_per_s": round(st.P * st.R * st.R / (mb * 1e-3), 1)},
           "query": {"ms": round(mq, 4), "point_dirs_per_s": round(pd / (mq * 1e-3), 1)},
           "roofline": trace_roofline(sop, st, mt, peak_fp32)}
    pargs = q["pts"]
    res["chosen"] = chosen_variant(sop, st.g, st.ppos, st.R, pargs, st.env, st.K, st.S, 0, q["out"], flush, steps)
    res["env_octahedral"] = env_oct_variant(sop, q["at"], pargs, st.env, st.K, st.S, 0, q["out"], flush, steps)
    res["frnn_query"] = frnn_variant(sop, q["at"], pargs, st.env, st.K, st.S, 0, q["out"], flush, steps, st.ppos)
    return res, st


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    from paper_2510_07729_gb300 import sop
    sop.load()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    peak_fp32 = N_SMS * FP32_LANES_PER_SM * 2 * 2.070e9 / 1e12
    if args.part == "compose":
        return compose_only(args, dev, sop)
    if args.part == "deferred":
        r = deferred_frame_variant(sop, dev, flush, args.steps)
        print(json.dumps({"metric": "composed deferred frames/s", "value": r["fps"], "unit": "frames/s",
                          "steps": args.steps, "higher_is_better": True, "detail": r}))
        return
    if args.part == "surrogate":
        r = rebake_only(sop, dev, flush, args.steps, args.warmup, args.probes)
        print(json.dumps({"metric": "learned rebake texels/s", "value": r["texels_per_s"], "unit": "texels/s",
                          "steps": args.steps, "higher_is_better": True, "detail": r}))
        return
    if args.part == "optimize":
        r = optimize_variant(sop, load_workload("object"), dev, flush, args.steps)
        print(json.dumps({"metric": "texture-optimisation step point-dirs/s", "value": r["point_dirs_per_s"],
                          "unit": "point-dirs/s", "steps": args.steps, "higher_is_better": True, "detail": r}))
        return
    W = load_workload(args.workload)
    st = StepState(sop, W, dev, n_probes=args.probes)
    do_bake = args.part in ("step", "bake")
    do_query = args.part in ("step", "query") and st.full
    if not do_bake:
        st.bake()  # query-only runs shade against a baked atlas
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    smi_index = vis.split(",")[local_rank] if vis else str(local_rank)
    r = time_steps(st, flush, args.steps, args.warmup, do_bake, do_query, world, smi_index)
    ms_step, mb, mq = reduce_max([r["ms_step"], float(np.mean(r["bake"])), float(np.mean(r["query"]))], world, dev)
    texels = st.P * st.R * st.R
    pd = st.M * st.S
    if args.part == "bake":
        units, unit_name = texels, "texels/s"
    else:
        units, unit_name = pd, "point-dirs/s"
    value = whole_job_value(units, ms_step, world)

    # e2e: public API from pinned host buffers, H2D + bake + queries + D2H each step
    e2e = None
    if not args.no_e2e and args.part == "step":
        e2e = measure_e2e(args, W, dev, sop, flush)

    roof = trace_roofline(sop, st, float(np.mean(r["trace"])), peak_fp32) if do_bake else None
    frame = objstep = surr = optim = defer = None
    if do_query and args.part == "step":
        if W["name"] == "compose" and not args.no_compose:
            frame = compose_frame_variant(sop, dev, flush, args.steps, l2_read_peak_gbs(dev), measured_peaks()[0],
                                          peak_fp32, baked=st)
        if W["name"] == "compose":
            objstep, _ = object_step_variant(sop, dev, flush, max(5, args.steps // 2), peak_fp32)
        if not args.no_surrogate:
            surr = surrogate_variant(sop, dev, flush, args.steps)
        if not args.no_optimize:
            optim = optimize_variant(sop, load_workload("object"), dev, flush, args.steps)
        if not args.no_deferred:
            defer = deferred_frame_variant(sop, dev, flush, args.steps)
    if roof is None and frame is not None:
        roof = frame["fp32"]["roofline"]

    line = {
        "metric": "SOP-shaded point-dirs/s (bake + query/shade step)" if args.part != "bake" else
        "probe-bake texels/s",
        "value": round(value, 1),
        "unit": unit_name,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_step, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded generators; the paper's SynCom/TensoIR scenes are not available)",
        "config": {"workload": W["label"], "part": args.part, "probes_baked": st.P,
                   "l2": "512 MB buffer written between timed steps", "parallelism": f"replicas x{world}"},
        "bake": {"ms": round(mb, 4), "texels_per_s": round(texels / (mb * 1e-3), 1) if do_bake else None},
        "query": {"ms": round(mq, 4), "point_dirs_per_s": round(pd / (mq * 1e-3), 1) if do_query else None,
                  "parts": {q["name"]: q["M"] for q in st.parts}},
        "wall_s_timed_region": round(r["wall_s"], 4),
        "gpu_launches": launches_per_step(do_bake, len(st.parts) if do_query else 0) * args.steps,
        "clocks": r["clocks"],
        "roofline": roof,
        "roofline_query": frame["fp32"]["roofline"] if frame else None,
        "precision": frame["precision"] if frame else None,
        "chosen": frame["chosen"] if frame else None,
        "chosen_bake": surr,
        "compose_frame_query": frame,
        "object_step": objstep,
        "deferred_frame": defer,
        "optimize_step": optim,
        "e2e": e2e,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.part == "step":
        line["cpu_baseline"] = cpu_baseline(W)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def optimize_variant(sop, W, dev, flush, steps):
    """One step of the SOP texture optimisation (the paper's second
    reconstruction step) on the object workload: pack the maps, shade the
    418,111 points (K=8, S=128), L1 gradient, adjoint, fused regularised Adam
    on the environment, materials and probe maps. Maps start from the
    ray-traced bake (which is also the L_sops target); the target image is
    U(0,1)^3 per point (seeded)."""
    import torch

    def cu(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    g = {k: cu(v) for k, v in W["gauss"].items()}
    pp = cu(W["probe_pos"])
    at = sop.make_atlas(pp, W["R"])
    sop.bake(g, at)
    rgb, occ, _ = at.interior()
    traced = torch.cat([rgb, occ[..., None]], dim=-1).contiguous()
    pts = {k: cu(v) for k, v in W["parts"][0]["pts"].items()}
    M = pts["x"].shape[0]
    target = cu(np.random.default_rng(11).uniform(0, 1, (M, 3)).astype(np.float32))
    opt = sop.TextureOptimizer(pts["albedo"], pts["rough"], pts["metal"], cu(W["env"]), traced.clone(), traced, pp)
    K, S = W["K"], W["S"]
    losses = []
    for _ in range(3):
        losses.append(opt.step(pts["x"], pts["n"], pts["wo"], target, K, S).item())
    torch.cuda.synchronize()
    ts = []
    for _ in range(steps):
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        opt.step(pts["x"], pts["n"], pts["wo"], target, K, S)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    losses.append(opt.step(pts["x"], pts["n"], pts["wo"], target, K, S).item())
    ms = float(np.mean(ts))
    return {"what": "SOP texture optimisation step (pack, shade, L1 gradient, adjoint, regularised Adam on "
                    "environment, materials and 4,096 probe maps) on the object view", "ms": round(ms, 4),
            "point_dirs_per_s": round(M * S / (ms * 1e-3), 1),
            "l_pbr": {"step_1": round(losses[0], 6), "after": round(losses[-1], 6), "steps": 4 + steps}}


def compose_only(args, dev, sop):
    """--part compose: the composition-frame query alone (profiling aid)."""
    import torch
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    peak_fp32 = N_SMS * FP32_LANES_PER_SM * 2 * 2.070e9 / 1e12
    r = compose_frame_variant(sop, dev, flush, args.steps, l2_read_peak_gbs(dev), measured_peaks()[0], peak_fp32)
    print(json.dumps({"metric": "composition-frame query point-dirs/s", "value": r["fp32"]["point_dirs_per_s"],
                      "unit": "point-dirs/s", "steps": args.steps, "higher_is_better": True, "detail": r}))


def launches_per_step(do_bake, n_queries):
    """This library's kernel launches in one step."""
    n = 0
    if do_bake:
        # binning: bbox init, Gaussian records, 3 attempts x (grid setup,
        # count, and the scan's tile sums, tile offsets and apply) decided on
        # the device, fill; trace: counter reset, texel directions, trace,
        # atlas border
        n += 2 + 3 * 5 + 1 + 4
    # per query: probe grid, nearest probes, environment table and
    # footprints, atlas footprints, directions, shade
    n += 7 * n_queries
    return n


def measure_e2e(args, W, dev, sop, flush):
    """The step through the public API from pinned host buffers: every step
    copies the Gaussians and probe positions (before the bake) and the
    points and environment (on a side stream while the bake runs) to the
    device, and reads every shaded output back."""
    import torch
    host = {}
    for k, v in W["gauss"].items():
        host["g_" + k] = torch.from_numpy(np.ascontiguousarray(v)).pin_memory()
    for i, part in enumerate(W["parts"]):
        for k, v in part["pts"].items():
            host[f"p{i}_{k}"] = torch.from_numpy(np.ascontiguousarray(v)).pin_memory()
    host["probe_pos"] = torch.from_numpy(np.ascontiguousarray(W["probe_pos"])).pin_memory()
    host["env"] = torch.from_numpy(np.ascontiguousarray(W["env"])).pin_memory()
    dbuf = {k: torch.empty_like(v, device=dev) for k, v in host.items()}
    R, K, S = W["R"], W["K"], W["S"]
    outs_h = [torch.empty((len(part["pts"]["x"]), 3), dtype=torch.float32).pin_memory() for part in W["parts"]]
    bi = sum(v.numel() * v.element_size() for v in host.values())
    bo = sum(o.numel() * o.element_size() for o in outs_h)
    M = sum(len(part["pts"]["x"]) for part in W["parts"])
    side = torch.cuda.Stream(device=dev)

    def one():
        main = torch.cuda.current_stream()
        for k in host:
            if k.startswith("g_") or k == "probe_pos":
                dbuf[k].copy_(host[k], non_blocking=True)
        side.wait_stream(main)
        with torch.cuda.stream(side):
            for k in host:
                if k.startswith("p") and k != "probe_pos" or k == "env":
                    dbuf[k].copy_(host[k], non_blocking=True)
        g = {k[2:]: dbuf[k] for k in dbuf if k.startswith("g_")}
        at = sop.make_atlas(dbuf["probe_pos"], R, depth_scale=W["depth_scale"])
        sop.bake(g, at)
        main.wait_stream(side)
        # as in the device-timed step: the smaller queries on the side
        # stream (after the bake), the largest on the main one
        big = int(np.argmax([len(part["pts"]["x"]) for part in W["parts"]]))
        side.wait_stream(main)
        for i, part in enumerate(W["parts"]):
            with torch.cuda.stream(main if i == big else side):
                o = sop.query_shade(*[dbuf[f"p{i}_{k}"] for k in ("x", "n", "wo", "albedo", "rough", "metal")],
                                    atlas_view(sop, at, *part["probes"]), dbuf["env"], K, S, mode=part["mode"])
                outs_h[i].copy_(o, non_blocking=True)
        main.wait_stream(side)

    for _ in range(2):
        one()
    torch.cuda.synchronize()
    ts = []
    for _ in range(max(3, args.steps // 2)):
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        one()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    ms = float(np.mean(ts))
    return {"value": round(M * S / (ms * 1e-3), 1), "unit": "point-dirs/s", "ms_per_step": round(ms, 4),
            "h2d_bytes_per_step": int(bi), "d2h_bytes_per_step": int(bo)}


def _oracle_step_seconds(W, rng, n_probes, n_points):
    """The FP64 oracle on a bounded sample of one step: n_probes probes of the
    bake and n_points points of each query part (at most), scaled to the
    whole step. Returns (seconds of the step, description)."""
    import oracle
    from paper_2510_07729_gb300 import inputs as I
    P, R, K, S = len(W["probe_pos"]), W["R"], W["K"], W["S"]
    probes = np.sort(rng.choice(P, min(n_probes, P), replace=False))
    t0 = time.perf_counter()
    oracle.bake(W["gauss"], W["probe_pos"], R, probes=probes)
    tb = time.perf_counter() - t0
    t_step = tb * (P / len(probes))
    desc = [f"bake of {len(probes)} probes ({len(probes) * R * R} rays, {tb:.2f} s)"]
    for part in W["parts"]:
        lo, hi = part["probes"]
        M = len(part["pts"]["x"])
        sel, pts = I.subsample(rng, part["pts"], ["x", "n", "wo", "albedo", "rough", "metal"], min(n_points, M))
        maps = I.synthetic_maps(rng, hi - lo, R)
        t0 = time.perf_counter()
        oracle.query_shade(pts["x"], pts["n"], pts["wo"], pts["albedo"], pts["rough"], pts["metal"],
                           W["probe_pos"][lo:hi], maps["rgb"], maps["occ"], W["env"], K, S, mode=part["mode"])
        tq = time.perf_counter() - t0
        t_step += tq * (M / len(sel))
        desc.append(f"{part['name']} query of {len(sel)} points x {S} dirs ({tq:.2f} s)")
    return t_step, " + ".join(desc) + ", scaled to the full step"


def cpu_baseline(W):
    """The FP64 oracle, as it stands, on a bounded sample of the same
    workload (16 probes of the bake, 4,096 points of each query part),
    scaled to the whole step."""
    import oracle
    t_step, desc = _oracle_step_seconds(W, np.random.default_rng(123), 16, 4096)
    M = sum(len(p["pts"]["x"]) for p in W["parts"])
    return {"value": round(M * W["S"] / t_step, 1), "unit": "point-dirs/s", "cores": oracle.num_threads(),
            "kind": "oracle", "sample": desc}


def run_reference(args, rank, world):
    """Reference arm: the FP64 oracle timed on the host cores, each step a
    bounded sample of the same workload (2 probes of the bake, 512 points of
    each query part, scaled to the step), in the same metric."""
    if rank != 0:
        return
    import oracle
    W = load_workload(args.workload)
    M = sum(len(p["pts"]["x"]) for p in W["parts"])
    rng = np.random.default_rng(7)
    for _ in range(args.warmup):
        _oracle_step_seconds(W, rng, 2, 512)
    ts = [_oracle_step_seconds(W, rng, 2, 512)[0] for _ in range(args.steps)]
    t = float(np.mean(ts))
    v = M * W["S"] / t
    line = {"impl": "reference", "metric": "SOP-shaded point-dirs/s (bake + query/shade step)", "value": round(v, 3),
            "unit": "point-dirs/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(t * 1e3, 3), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "config": {"workload": W["label"], "parallelism": "host cores"},
            "cpu_baseline": {"value": round(v, 3), "unit": "point-dirs/s", "cores": oracle.num_threads(),
                             "kind": "oracle",
                             "sample": "per step: bake of 2 probes + 512 points of each query part, scaled to the "
                                       "full step"},
            "e2e": {"value": round(v, 3), "unit": "point-dirs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
