"""GPU parity of the learned bake surrogate (sop_surrogate_*) through the C
ABI: its texel features against the FP64 feature oracle
(oracle/surrogate_oracle.c), its network (inference and one training step:
loss, gradient, Adam) against the FP64 network oracle (oracle/mlp.py) on the
same features and bf16-rounded operands, checkpoint save/load/resume, and
the rebake's spot check and fallback decided on the device."""
import numpy as np
import pytest
import torch

from oracle import mlp
from paper_2510_07729_gb300 import inputs as I
from tests.tolerance import assert_close

pytestmark = pytest.mark.gpu

R_NEAR = 0.08


@pytest.fixture(scope="module")
def sop():
    from paper_2510_07729_gb300 import sop as S
    S.load()
    return S


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def scene():
    # a surrogate training scene, cut down so the oracle finishes in seconds
    return I.surrogate_scene(1003, n_gauss=20000, n_probes=48)


def params(seed=0):
    th = I.surrogate_init(seed).astype(np.float64)
    w = mlp.unflatten(th)
    rng = np.random.default_rng(seed + 100)
    for k in ("b1", "b2", "b3", "b4"):
        w[k] = rng.uniform(-0.05, 0.05, w[k].shape)
    return mlp.flatten(w).astype(np.float32)


def check_near(gf, of, ok, what):
    """O_n, L_n, W_n at the FP32 bound; D_n with the bake's depth allowance:
    a t* next to the probe (B ~ 0) cannot be resolved better than a few ulp
    of the coordinates it comes from."""
    cols = [3, 4, 5, 6, 8]
    assert_close(gf[..., cols][ok], of[..., cols][ok], what=what)
    assert_close(gf[..., 7][ok], of[..., 7][ok], what=what + " D_n", absolute=4 * 2.0 ** -24 * 4.0)


def check_far(gf, of, sens, what):
    """The far field (FP32 march against FP64) at rtol 2e-5 plus twice the
    march's conditioning: a cell boundary time taken in FP32 is off by a few
    ulp of the coordinates it comes from, and a short segment clipped off a
    dense cell's corner turns that into a large relative change of tau
    (sigma times a small difference of two large times). The oracle sums
    sigma times those rounding scales over the segments; tau, the opacity
    features (their derivative in tau is at most 1) and the colour (cell
    colours at most 1) move by no more."""
    assert_close(gf[..., 9:], of[..., 9:], rtol=2e-5, what=what, absolute=2.0 * sens[..., None])


def test_features_match_oracle(sop, orc, scene):
    g = scene["gauss"]
    pp = scene["probe_pos"]
    R = 16
    net = sop.Surrogate(params(), r_near=R_NEAR)
    gf, lst = net.features({k: cuda(v) for k, v in g.items()}, cuda(pp), R, with_list=True)
    gf, lst = gf.cpu().numpy(), lst.cpu().numpy()
    of, flags, olst, t0, sens = orc.surr_features(g, pp, R, R_NEAR, far_sens=True)
    assert np.array_equal(lst, olst)  # the near lists: exact integer decisions
    assert (olst >= 0).sum(1).mean() > 30  # (this cut-down scene's lists are short)
    assert np.array_equal(gf[..., :3], of[..., :3].astype(np.float32))
    ok = flags == 0
    assert ok.mean() > 0.98
    check_near(gf, of, ok, "near field")
    check_far(gf, of, sens, "far field")


def test_features_full_scene_sampled(sop, orc):
    """The object-scale scene (200,000 Gaussians): 16 sampled probes of a
    full 4,096-probe feature pass against the oracle."""
    sc = I.surrogate_scene(1001)
    g, pp = sc["gauss"], sc["probe_pos"]
    R = 16
    net = sop.Surrogate(params(), r_near=R_NEAR)
    gf, lst = net.features({k: cuda(v) for k, v in g.items()}, cuda(pp), R, with_list=True)
    sel = np.random.default_rng(5).choice(len(pp), 16, replace=False)
    of, flags, olst, _, sens = orc.surr_features(g, pp[sel], R, R_NEAR, far_sens=True)
    gf, lst = gf.cpu().numpy()[sel], lst.cpu().numpy()[sel]
    assert np.array_equal(lst, olst)
    assert (olst[:, -1] >= 0).mean() > 0.5  # most lists are full (256 within r_near)
    ok = flags == 0
    check_near(gf, of, ok, "near field (object scene)")
    check_far(gf, of, sens, "far field (object scene)")


def _targets(sop, scene, R=16):
    g = {k: cuda(v) for k, v in scene["gauss"].items()}
    at = sop.make_atlas(cuda(scene["probe_pos"]), R)
    sop.bake(g, at)
    return g, at


def test_predict_matches_oracle_forward(sop, scene):
    th = params(1)
    net = sop.Surrogate(th, r_near=R_NEAR)
    g, _ = _targets(sop, scene)
    R = 16
    feats = net.features(g, cuda(scene["probe_pos"]), R)
    P = len(scene["probe_pos"])
    out = sop.make_atlas(cuda(scene["probe_pos"]), R)
    net.predict(feats, out)
    rgb, occ, dep = out.interior()
    x = feats.cpu().numpy().reshape(-1, mlp.N_IN).astype(np.float64)
    y, _ = mlp.forward(th.astype(np.float64), x)
    y = y.reshape(P, R, R, 5)
    want_o = np.clip(y[..., 0], 0, 1)
    want_rgb = np.maximum(y[..., 2:], 0)
    want_d = np.maximum(y[..., 1], 0)
    for got, want, name in ((occ.cpu().numpy(), want_o, "O"), (rgb.cpu().numpy(), want_rgb, "RGB"),
                            (dep.cpu().numpy(), want_d, "D")):
        err = np.abs(got - want) / np.maximum(np.abs(want), 1e-2)
        # float32 sums against exact ones, then a bf16 rounding of each
        # activation: a last-bit difference of a sum can move a bf16 value
        # by one ulp (2^-8 relative), which the next layer carries on
        assert np.median(err) < 1e-4, name
        assert (err > 1e-3).mean() < 0.02, name
        assert err.max() < 5e-2, name
    # the border follows the border rule
    a = out.rgbo.cpu().numpy()
    assert np.array_equal(a[:, 0, 1:R + 1], a[:, 1, R:0:-1])


def test_train_step_matches_oracle(sop, scene):
    """One Adam step on 6 given probes: the loss, the summed gradient of every
    parameter block and the update, against the FP64 network on the same
    features and targets."""
    th0 = params(2)
    net = sop.Surrogate(th0, r_near=R_NEAR)
    g, at = _targets(sop, scene)
    R = 16
    feats = net.features(g, cuda(scene["probe_pos"]), R)
    ids = np.array([3, 0, 17, 17, 40, 8], np.int32)
    losses = torch.zeros(1, device="cuda")
    net.train(feats, at, steps=1, lr=1e-3, probe_ids=cuda(ids), losses=losses)
    rgb, occ, dep = (t.cpu().numpy() for t in at.interior())
    tgt = np.concatenate([occ[..., None], dep[..., None], rgb], -1)[ids].reshape(-1, 5).astype(np.float64)
    x = feats.cpu().numpy()[ids].reshape(-1, mlp.N_IN).astype(np.float64)
    l_o, g_o, _ = mlp.loss_and_grad(th0.astype(np.float64), x, tgt)
    assert losses.item() == pytest.approx(l_o, rel=1e-4)
    gg = net.grad().cpu().numpy().astype(np.float64)
    wg, wo = mlp.unflatten(gg), mlp.unflatten(g_o)
    # both sides round activations and deltas to bf16; an FP32 sum that
    # differs from the FP64 one in its last bits can round to the neighbouring
    # bf16 value (2^-8 relative), which the later layers carry on. Measured on
    # three seeds: at most 1.9e-4 relative per block
    for name, _ in mlp.SHAPES:
        rel = np.linalg.norm(wg[name] - wo[name]) / max(np.linalg.norm(wo[name]), 1e-12)
        assert rel < 1e-3, (name, rel)
    # the Adam update, on the GPU's own gradient (first step: lr * sign)
    th1 = net.params().cpu().numpy().astype(np.float64)
    want, _, _ = mlp.adam(th0.astype(np.float64), np.zeros_like(gg), np.zeros_like(gg), gg, 1, lr=1e-3)
    assert np.allclose(th1, want, rtol=0, atol=2e-6)


def test_checkpoint_resume_is_exact(sop, scene, tmp_path):
    """Train 3 steps, save, train 2 more; a fresh handle loaded from the
    save and trained the same 2 steps (same seed: the batches are drawn
    from the seed and the restored step count) ends bit-identical."""
    g, at = _targets(sop, scene)
    R = 16
    a = sop.Surrogate(params(3), r_near=R_NEAR)
    feats = a.features(g, cuda(scene["probe_pos"]), R)
    a.train(feats, at, steps=3, batch=8, lr=2e-3, seed=9)
    path = tmp_path / "net.ckpt"
    a.save(path)
    a.train(feats, at, steps=2, batch=8, lr=2e-3, seed=9)
    b = sop.Surrogate(None, r_near=R_NEAR, seed=123)  # different start
    b.load_file(path)
    b.train(feats, at, steps=2, batch=8, lr=2e-3, seed=9)
    pa, pb = a.params().cpu().numpy(), b.params().cpu().numpy()
    assert np.array_equal(pa.view(np.uint32), pb.view(np.uint32))


def test_rebake_fallback_and_spot_check(sop, scene):
    """The device-side decision: tau = 0 forces the fallback, and the atlas
    is then the plain bake, bit for bit; a huge tau keeps the prediction,
    except the checked probes, which hold their traced maps; the reported
    error is the checked probes' mean |dO|."""
    g, exact = _targets(sop, scene)
    R = 16
    P = len(scene["probe_pos"])
    net = sop.Surrogate(params(4), r_near=R_NEAR)
    out = sop.make_atlas(cuda(scene["probe_pos"]), R)
    err, fell = net.rebake(g, out, spot_frac=0.1, tau=0.0, seed=11)
    assert fell.item() == 1 and err.item() > 0
    assert torch.equal(out.rgbo, exact.rgbo) and torch.equal(out.depth, exact.depth)
    out2 = sop.make_atlas(cuda(scene["probe_pos"]), R)
    err2, fell2 = net.rebake(g, out2, spot_frac=0.1, tau=1e9, seed=11)
    assert fell2.item() == 0 and err2.item() == pytest.approx(err.item(), rel=1e-6)
    pred = sop.make_atlas(cuda(scene["probe_pos"]), R)
    net.predict(net.features(g, cuda(scene["probe_pos"]), R), pred)
    n_spot = int(np.ceil(0.1 * P))
    same_as_exact = [torch.equal(out2.rgbo[p], exact.rgbo[p]) for p in range(P)]
    same_as_pred = [torch.equal(out2.rgbo[p], pred.rgbo[p]) for p in range(P)]
    assert sum(same_as_exact) >= n_spot
    assert sum(same_as_pred) == P - n_spot
    checked = [p for p in range(P) if not same_as_pred[p]]
    # one probe of each stratum of the probe order
    assert sorted(p * n_spot // P for p in checked) == list(range(n_spot))
    dO = (pred.rgbo[checked, 1:R + 1, 1:R + 1, 3] - exact.rgbo[checked, 1:R + 1, 1:R + 1, 3]).abs().mean().item()
    assert err2.item() == pytest.approx(dO, rel=1e-5)
    assert sop.device_status() == 0


def test_predict_unaligned_features(sop, scene):
    """The network reads a chunk's features by one bulk copy only when they
    start on a 16-byte boundary and span whole 16 bytes; other chunks are read
    by the threads. R = 15 (225 texels a probe: chunks of 128 and 97 whose
    starts alternate between aligned and not) and a feature array that starts
    one texel into its allocation take both paths; both match the FP64
    network on the same features."""
    th = params(6)
    net = sop.Surrogate(th, r_near=R_NEAR)
    R = 15
    g = {k: cuda(v) for k, v in scene["gauss"].items()}
    pp = cuda(scene["probe_pos"])
    P = len(scene["probe_pos"])
    feats = net.features(g, pp, R)
    # the same features, one texel into a larger buffer (72 bytes: not 16-aligned)
    buf = torch.zeros(P * R * R * mlp.N_IN + mlp.N_IN, device="cuda")
    shifted = buf[mlp.N_IN:].view(P, R * R, mlp.N_IN)
    shifted.copy_(feats)
    assert (shifted.data_ptr() % 16) != 0
    x = feats.cpu().numpy().reshape(-1, mlp.N_IN).astype(np.float64)
    y, _ = mlp.forward(th.astype(np.float64), x)
    want_o = np.clip(y[:, 0], 0, 1).reshape(P, R, R)
    for f in (feats, shifted):
        out = sop.make_atlas(pp, R)
        net.predict(f, out)
        occ = out.interior()[1].cpu().numpy()
        err = np.abs(occ - want_o) / np.maximum(np.abs(want_o), 1e-2)
        assert np.median(err) < 1e-4
        assert (err > 1e-3).mean() < 0.02
        assert err.max() < 5e-2
    assert sop.device_status() == 0


def test_rebake_from_two_host_threads(sop, scene):
    """sop_surrogate_infer shares one pair of side streams and events per
    device; calls from two host threads on two streams (each with its own
    handle, hence its own workspace) must each give the atlas of a call made
    alone, bit for bit."""
    import threading
    g, _ = _targets(sop, scene)
    R = 16
    pp = cuda(scene["probe_pos"])
    th = params(7)
    ref = sop.make_atlas(pp, R)
    sop.Surrogate(th, r_near=R_NEAR).rebake(g, ref, spot_frac=0.1, tau=1e9, seed=5)
    torch.cuda.synchronize()
    nets = [sop.Surrogate(th, r_near=R_NEAR) for _ in range(2)]
    outs = [sop.make_atlas(pp, R) for _ in range(2)]
    streams = [torch.cuda.Stream() for _ in range(2)]
    errors = []

    def run(i):
        try:
            with torch.cuda.stream(streams[i]):
                for _ in range(4):
                    nets[i].rebake(g, outs[i], spot_frac=0.1, tau=1e9, seed=5)
        except Exception as e:  # noqa: BLE001 - reported below
            errors.append(e)

    ts = [threading.Thread(target=run, args=(i,)) for i in range(2)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    torch.cuda.synchronize()
    assert not errors, errors
    for o in outs:
        assert torch.equal(o.rgbo, ref.rgbo) and torch.equal(o.depth, ref.depth)
    assert sop.device_status() == 0
