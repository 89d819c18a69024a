"""The learned bake surrogate on its evaluation workload: trained on bakes
that the ray-traced sop_bake makes of randomised 5-ellipsoid scenes, then
used to rebake 4,096 probes of the 'object' scene after its first ellipsoid
moved by a random U(-0.5, 0.5)^3 translation. Reports (printed) and checks:
what training gains over the untrained network, how it compares with keeping
the stale atlas, the 1% spot-check's estimate of the error, the fallback, and
the error the rebaked atlas causes in the shaded output."""
import numpy as np
import pytest
import torch

from paper_2510_07729_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def mean_dO(sop, a, b):
    return sop.atlas_compare(a, b)[0].item() / (a.P * a.R * a.R)


def test_surrogate_rebake_after_object_move():
    from paper_2510_07729_gb300 import sop
    sop.load()
    surr = sop.Surrogate(I.surrogate_init(0))
    untrained = sop.Surrogate(I.surrogate_init(0))
    feats, atlases = [], []
    for s in range(8):
        sc = I.surrogate_scene(1000 + s)
        gt = {k: cuda(v) for k, v in sc["gauss"].items()}
        at = sop.make_atlas(cuda(sc["probe_pos"]), 16)
        sop.bake(gt, at)
        atlases.append(at)
        feats.append(surr.features(gt, cuda(sc["probe_pos"])))
    rng = np.random.default_rng(0)
    steps = 8000
    for it in range(steps):
        j = int(rng.integers(len(feats)))
        ids = cuda(np.sort(rng.choice(4096, 64, replace=False)).astype(np.int32))
        surr.train_step(feats[j], atlases[j], lr=2e-3 if it < 0.7 * steps else 5e-4, probe_ids=ids)

    mv = I.moved_object()
    gt = {k: cuda(v) for k, v in mv["gauss"].items()}
    pp = cuda(mv["probe_pos"])
    exact = sop.make_atlas(pp, 16)
    sop.bake(gt, exact)
    fe = surr.features(gt, pp)
    pred = sop.make_atlas(pp, 16)
    surr.infer(fe, pred)
    pred0 = sop.make_atlas(pp, 16)
    untrained.infer(fe, pred0)
    c = I.make_object()
    stale = sop.make_atlas(pp, 16)
    sop.bake({k: cuda(v) for k, v in c["gauss"].items()}, stale)
    e_tr, e_un, e_st = mean_dO(sop, exact, pred), mean_dO(sop, exact, pred0), mean_dO(sop, exact, stale)
    print(f"\nmean |dO| vs exact bake: trained {e_tr:.4f}, untrained {e_un:.4f}, stale atlas {e_st:.4f}")
    # training is what makes the network usable at all
    assert e_tr < 0.5 * e_un

    # rebake with a 1% spot-check: its estimate tracks the true error, and
    # above tau the result is exactly the ray-traced bake
    out = sop.make_atlas(pp, 16)
    err, fell = sop.surrogate_rebake(surr, gt, out, spot_frac=0.01, tau=0.05, seed=3)
    print(f"spot-check estimate {err:.4f} (true {e_tr:.4f}); fell back: {fell}")
    assert abs(err - e_tr) < 0.5 * e_tr + 0.01
    if fell:
        assert torch.equal(out.rgbo, exact.rgbo)
    else:
        assert mean_dO(sop, exact, out) <= e_tr + 1e-6

    # what the surrogate's atlas does to shading (rebaked object seen from the
    # 'object' camera; points of the moved scene are not regenerated, so this
    # is the probe-interpolated lighting error at the same points)
    pts = [cuda(c[k]) for k in ("x", "n", "wo", "albedo", "rough", "metal")]
    env = cuda(c["env"])
    C_exact = sop.query_shade(*pts, exact, env, 8, 128)
    C_pred = sop.query_shade(*pts, pred, env, 8, 128)
    rel = ((C_pred - C_exact).abs().sum() / C_exact.abs().sum()).item()
    print(f"shaded output relative L1 (surrogate atlas vs exact): {rel:.4f}")
    assert np.isfinite(rel)
