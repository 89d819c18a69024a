"""GPU parity of the learned bake surrogate (features, bf16 MLP forward,
hand-written backward, Adam) against the FP64 oracle (oracle/mlp.py), and
its rebake / spot-check / fallback flow, through the C ABI."""
import numpy as np
import pytest
import torch

from oracle import mlp
from paper_2510_07729_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sop():
    from paper_2510_07729_gb300 import sop as S
    S.load()
    return S


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def obj():
    return I.make_object()


def texel_dirs(orc, R):
    jj, ii = np.meshgrid(np.arange(R), np.arange(R), indexing="ij")
    return orc.oct_decode(np.stack([(ii.ravel() + 0.5) / R, (jj.ravel() + 0.5) / R], 1))


def params(seed=7):
    th = I.surrogate_init(seed).astype(np.float64)
    # nonzero biases so that every unit and output is exercised
    rng = np.random.default_rng(seed + 1)
    w = mlp.unflatten(th)
    for b in ("b1", "b2", "b3"):
        w[b][:] = rng.uniform(0.0, 0.3, w[b].shape)
    w["b4"][:] = [0.5, 0.4, 0.3, 0.3, 0.3]
    return mlp.flatten(w).astype(np.float32)


def test_features_match_oracle(sop, obj):
    g = obj["gauss"]
    pp = obj["probe_pos"][:48]
    surr = sop.Surrogate(params())
    f = surr.features({k: cuda(v) for k, v in g.items()}, cuda(pp)).cpu().numpy().astype(np.float64)
    ref, idx = mlp.probe_features(pp, g)
    # computed in double on both sides, rounded once to float32
    assert np.array_equal(f, ref.astype(np.float32).astype(np.float64))


def _tiny_setup(sop, obj, P=12, R=8):
    g = obj["gauss"]
    pp = obj["probe_pos"][:P]
    fp, _ = mlp.probe_features(pp, g)
    surr = sop.Surrogate(params())
    feats = surr.features({k: cuda(v) for k, v in g.items()}, cuda(pp))
    return g, pp, fp, surr, feats


def test_infer_matches_oracle_forward(sop, orc, obj):
    R = 8
    g, pp, fp, surr, feats = _tiny_setup(sop, obj)
    at = sop.make_atlas(cuda(pp), R)
    surr.infer(feats, at)
    torch.cuda.synchronize()
    rgb, occ, dep = (t.cpu().numpy() for t in at.interior())
    P = len(pp)
    dt = np.tile(texel_dirs(orc, R), (P, 1))
    pidx = np.repeat(np.arange(P), R * R)
    y, _ = mlp.forward(params().astype(np.float64), fp, dt, pidx)
    want_o = np.clip(y[:, 0], 0, 1).reshape(P, R, R)
    want_d = np.maximum(y[:, 1], 0).reshape(P, R, R)
    want_c = np.maximum(y[:, 2:], 0).reshape(P, R, R, 3)
    # bf16 operands: where an FP32 pre-activation and its FP64 counterpart
    # round to different bf16 values (a 2^-8 relative step on that operand),
    # the difference propagates through the later layers; elsewhere the two
    # agree to FP32 accumulation error
    for got, want in ((occ, want_o), (dep, want_d), (rgb, want_c)):
        scale = np.maximum(np.abs(want), 1e-2 * np.abs(want).mean())
        rel = np.abs(got - want) / scale
        assert np.median(rel) < 1e-4
        assert np.mean(rel > 1e-3) < 0.02
        assert np.max(rel) < 5e-2


def test_train_step_gradient_matches_oracle(sop, orc, obj):
    R = 8
    g, pp, fp, surr, feats = _tiny_setup(sop, obj)
    P = len(pp)
    maps = I.synthetic_maps(np.random.default_rng(60), P, R)
    maps["depth"] = (maps["depth"] * 0.25).astype(np.float32)
    tgt = sop.make_atlas(cuda(pp), R)
    sop.atlas_pack(cuda(maps["rgb"]), cuda(maps["occ"]), cuda(maps["depth"]), tgt)
    th0 = params()
    loss = surr.train_step(feats, tgt, lr=1e-3).item()
    gg = surr.grad().cpu().numpy().astype(np.float64)
    dt = np.tile(texel_dirs(orc, R), (P, 1))
    pidx = np.repeat(np.arange(P), R * R)
    target = np.concatenate([maps["occ"].reshape(-1, 1), maps["depth"].reshape(-1, 1),
                             maps["rgb"].reshape(-1, 3)], axis=1).astype(np.float64)
    l_o, g_o, _ = mlp.loss_and_grad(th0.astype(np.float64), fp, dt, pidx, target)
    assert loss == pytest.approx(l_o, rel=1e-3)
    wg, wo = mlp.unflatten(gg), mlp.unflatten(g_o)
    for name, _ in mlp.SHAPES:
        err = np.linalg.norm(wg[name] - wo[name]) / max(np.linalg.norm(wo[name]), 1e-12)
        assert err < 2e-2, (name, err)
    # first Adam step: -lr g / (|g| + eps) in every coordinate
    th1 = surr.params().cpu().numpy().astype(np.float64)
    want = th0 - 1e-3 * gg / (np.abs(gg) + 1e-8)
    assert np.max(np.abs(th1 - want)) < 2e-6


def test_training_reduces_loss(sop):
    scenes = [I.surrogate_scene(s, n_gauss=30_000, n_probes=256) for s in (70, 71)]
    surr = sop.Surrogate(I.surrogate_init(3))
    feats, atlases = [], []
    for sc in scenes:
        gt = {k: cuda(v) for k, v in sc["gauss"].items()}
        at = sop.make_atlas(cuda(sc["probe_pos"]), 16)
        sop.bake(gt, at)
        atlases.append(at)
        feats.append(surr.features(gt, cuda(sc["probe_pos"])))
    rng = np.random.default_rng(0)
    losses = []
    for it in range(400):
        j = it % 2
        ids = cuda(np.sort(rng.choice(256, 32, replace=False)).astype(np.int32))
        losses.append(surr.train_step(feats[j], atlases[j], lr=2e-3, probe_ids=ids).item())
    first, last = np.mean(losses[:20]), np.mean(losses[-20:])
    print(f"surrogate training loss {first:.4f} -> {last:.4f}")
    assert last < 0.75 * first


def test_rebake_fallback_and_spot_check(sop, obj):
    g = {k: cuda(v) for k, v in obj["gauss"].items()}
    pp = cuda(obj["probe_pos"][:512])
    exact = sop.make_atlas(pp, 16)
    sop.bake(g, exact)
    # corrupted surrogate: the spot-check must reject it and fall back
    bad = sop.Surrogate(params() * 50.0)
    out = sop.make_atlas(pp, 16)
    err, fell = sop.surrogate_rebake(bad, g, out, spot_frac=0.02, tau=0.05, seed=1)
    torch.cuda.synchronize()
    assert fell and err > 0.05
    assert torch.equal(out.rgbo, exact.rgbo) and torch.equal(out.depth, exact.depth)
    # accepted surrogate: the checked probes carry their exact bake
    ok = sop.Surrogate(params())
    out2 = sop.make_atlas(pp, 16)
    err2, fell2 = sop.surrogate_rebake(ok, g, out2, spot_frac=0.02, tau=10.0, seed=2)
    torch.cuda.synchronize()
    assert not fell2
    sel = np.sort(np.random.default_rng(2).choice(512, 11, replace=False))
    assert torch.equal(out2.rgbo[sel], exact.rgbo[sel])
    assert not torch.equal(out2.rgbo, exact.rgbo)
