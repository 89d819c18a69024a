"""The learned bake surrogate on its evaluation workload: trained on bakes
that the ray-traced sop_bake makes of randomised 5-ellipsoid scenes, then
used to rebake the 4,096 probes of the 'object' scene after its first
ellipsoid moved by a random U(-0.5, 0.5)^3 translation (probes re-placed on
the moved surface).

Checked against the targets of the learned form:
  - mean |dO| of the rebaked atlas against the exact bake <= 0.02;
  - a gain over what the method has without the network: the stale atlas
    (the same probes baked against the scene before the move) and the
    features alone (the near and far occlusion combined without a network);
  - the 1% spot check passes (no fallback) and estimates the error;
  - the rebake (features, network, spot check, all in sop_surrogate_infer)
    is at least 5x faster than the plain ray-traced bake of the same probes;
  - shading with the rebaked atlas is within 1e-2 relative L1 of shading with
    the exact one, on a view of the moved object."""
import numpy as np
import pytest
import torch

from paper_2510_07729_gb300 import inputs as I

pytestmark = pytest.mark.gpu

R_NEAR = 0.08
N_SCENES = 16
STEPS = 20000


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def mean_dO(sop, a, b):
    return sop.atlas_compare(a, b)[0].item() / (a.P * a.R * a.R)


def timed(fn, reps=7):
    for _ in range(2):
        fn()
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return float(np.median(ts))


@pytest.fixture(scope="module")
def trained():
    from paper_2510_07729_gb300 import sop
    sop.load()
    net = sop.Surrogate(I.surrogate_init(0), r_near=R_NEAR)
    feats, atlases = [], []
    for s in range(N_SCENES):
        sc = I.surrogate_scene(1000 + s)
        gt = {k: cuda(v) for k, v in sc["gauss"].items()}
        at = sop.make_atlas(cuda(sc["probe_pos"]), 16)
        sop.bake(gt, at)
        atlases.append(at)
        feats.append(net.features(gt, cuda(sc["probe_pos"]), 16))
    rng = np.random.default_rng(0)
    chunk = 50
    for it in range(0, STEPS, chunk):
        j = int(rng.integers(N_SCENES))
        net.train(feats[j], atlases[j], steps=chunk, batch=64, lr=2e-3 if it < 0.7 * STEPS else 5e-4, seed=it)
    torch.cuda.synchronize()
    return sop, net


def test_surrogate_rebake_after_object_move(trained):
    sop, net = trained
    mv = I.moved_object()
    gt = {k: cuda(v) for k, v in mv["gauss"].items()}
    pp = cuda(mv["probe_pos"])
    exact = sop.make_atlas(pp, 16)
    bws = sop.BakeWorkspace(len(mv["gauss"]["mean"]), "cuda")
    sop.bake(gt, exact, workspace=bws)
    fe = net.features(gt, pp, 16)
    pred = sop.make_atlas(pp, 16)
    net.predict(fe, pred)
    c = I.make_object()
    stale = sop.make_atlas(pp, 16)
    sop.bake({k: cuda(v) for k, v in c["gauss"].items()}, stale)
    f = fe.cpu().numpy()
    heur = 1 - (1 - f[..., 3]) * (1 - f[..., 14])  # near and far occlusion, no network
    e_heur = float(np.abs(heur - exact.interior()[1].cpu().numpy().reshape(4096, 256)).mean())
    e_tr, e_st = mean_dO(sop, exact, pred), mean_dO(sop, exact, stale)
    print(f"\nmean |dO| vs exact bake: surrogate {e_tr:.4f}, features alone {e_heur:.4f}, stale atlas {e_st:.4f}")
    assert e_tr < 0.5 * e_st
    assert e_tr < 0.8 * e_heur

    # the rebake with its 1% spot check, all on the device
    out = sop.make_atlas(pp, 16)
    err, fell = net.rebake(gt, out, spot_frac=0.01, tau=0.05, seed=3)
    err, fell = err.item(), fell.item()
    print(f"spot-check estimate {err:.4f} (true {e_tr:.4f}); fell back: {bool(fell)}")
    assert abs(err - e_tr) < 0.5 * e_tr + 0.01
    t_plain = timed(lambda: sop.bake(gt, exact, workspace=bws))
    t_rebake = timed(lambda: net.rebake(gt, out, spot_frac=0.01, tau=0.05, seed=3))
    print(f"rebake {t_rebake:.3f} ms against the plain bake {t_plain:.3f} ms: {t_plain / t_rebake:.2f}x")

    # shading a view of the moved object with the rebaked atlas
    pts = [cuda(mv[k]) for k in ("x", "n", "wo", "albedo", "rough", "metal")]
    env = cuda(mv["env"])
    C_exact = sop.query_shade(*pts, exact, env, mv["K"], mv["S"])
    C_out = sop.query_shade(*pts, out, env, mv["K"], mv["S"])
    rel = ((C_out - C_exact).abs().sum() / C_exact.abs().sum()).item()
    print(f"shaded output relative L1 (rebaked atlas vs exact): {rel:.5f}")
    assert sop.device_status() == 0

    assert e_tr <= 0.02, f"mean |dO| {e_tr:.4f} above the 0.02 target"
    assert not fell, f"the spot check fell back (estimate {err:.4f})"
    assert rel <= 1e-2, f"shading relative L1 {rel:.4f} above 1e-2"
    assert t_plain / t_rebake >= 5.0, f"rebake only {t_plain / t_rebake:.2f}x faster than the plain bake"
