"""GPU parity of the SOP texture optimisation step (Sec. 3.1.2, second
step) against the FP64 oracle (oracle/optimize.py), through the C ABI."""
import numpy as np
import pytest
import torch

from paper_2510_07729_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sop():
    from paper_2510_07729_gb300 import sop as S
    S.load()
    return S


@pytest.fixture(scope="module")
def opt():
    from oracle import optimize
    return optimize


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def test_l1_loss_grad_kernel(sop, opt):
    rng = np.random.default_rng(0)
    C = rng.uniform(0, 1, (1000, 3)).astype(np.float32)
    Ct = rng.uniform(0, 1, (1000, 3)).astype(np.float32)
    Ct[:10] = C[:10]  # ties: zero subgradient
    loss = torch.zeros(1, device="cuda")
    g = sop.l1_loss_grad(cuda(C), cuda(Ct), loss_sum=loss).cpu().numpy()
    lo, go = opt.l1_loss_grad(C, Ct)
    assert np.array_equal(g, go.astype(np.float32))
    assert loss.item() / C.size == pytest.approx(lo, rel=1e-5)


@pytest.mark.parametrize("t", [1, 7])
def test_adam_kernel_matches_oracle(sop, opt, t):
    """Interleaved RGB + O block: regulariser toward per-element targets with
    two weights, Adam, clamps per channel group."""
    rng = np.random.default_rng(t)
    n = 4 * 3000
    p = rng.uniform(-0.2, 1.2, n).astype(np.float32)
    g = (rng.standard_normal(n) * 1e-3).astype(np.float32)
    m = (rng.standard_normal(n) * 1e-4).astype(np.float32)
    v = (rng.uniform(0, 1e-6, n)).astype(np.float32)
    tgt = rng.uniform(0, 1, n).astype(np.float32)
    lam = (2e-4, 5e-4)
    lo, hi = (0.0, 0.0), (3.0e38, 1.0)
    P, G, Mm, V = cuda(p), cuda(g), cuda(m), cuda(v)
    sop.adam_l1_step(P, G, Mm, V, t, 1e-3, target=cuda(tgt), lam=lam, lo=lo, hi=hi, period=4, split=3)
    rgb = (np.arange(n) % 4) < 3
    lam_e = np.where(rgb, lam[0], lam[1])
    gt = g.astype(np.float64) + lam_e * np.sign(p.astype(np.float64) - tgt)
    lo_e, hi_e = np.where(rgb, lo[0], lo[1]), np.where(rgb, np.inf, 1.0)
    po, mo, vo = opt.adam(p.astype(np.float64), gt, m.astype(np.float64), v.astype(np.float64), t, 1e-3, lo_e, hi_e)
    # the kernel's moments and bias corrections use the float32 betas it is
    # given; with those constants, each product and sum rounds to within a
    # few units of 2^-24 of the terms (the moments cancel when m and g
    # differ in sign)
    u = 2.0 ** -24
    b1, b2 = float(np.float32(0.9)), float(np.float32(0.999))
    c1, c2 = float(np.float32(1.0 - b1)), float(np.float32(1.0 - b2))
    me = b1 * m.astype(np.float64) + c1 * gt
    ve = b2 * v.astype(np.float64) + c2 * gt * gt
    m_gpu, v_gpu = Mm.cpu().numpy().astype(np.float64), V.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(m_gpu - me) <= 4 * u * (b1 * np.abs(m) + c1 * (np.abs(g) + lam_e)))
    assert np.all(np.abs(v_gpu - ve) <= 6 * u * (b2 * v + c2 * gt * gt))
    # the update from the kernel's own moments: a few ulp of p and of the step
    bc1, bc2 = float(np.float32(1 - b1 ** t)), float(np.float32(1 - b2 ** t))
    step = 1e-3 * (m_gpu / bc1) / (np.sqrt(v_gpu / bc2) + 1e-8)
    pe = np.clip(p.astype(np.float64) - step, lo_e, hi_e)
    assert np.all(np.abs(P.cpu().numpy() - pe) <= 4 * u * (np.abs(p) + np.abs(step)))
    # and the whole step against the oracle's moments, within the moments' rounding
    np.testing.assert_allclose(P.cpu().numpy(), po, rtol=0, atol=1e-6)


@pytest.fixture(scope="module")
def problem():
    c = I.make_tiny()
    rng = np.random.default_rng(9)
    M = 1024
    pts = {k: np.ascontiguousarray(c[k][:M]) for k in ("x", "n", "wo")}
    maps = I.synthetic_maps(rng, 64, 8)
    traced = I.synthetic_maps(rng, 64, 8)
    params = dict(albedo=c["albedo"][:M], rough=np.clip(c["rough"][:M], 0.15, 0.95).astype(np.float32),
                  metal=np.clip(c["metal"][:M], 0.05, 0.95).astype(np.float32), env=c["env"],
                  maps_rgb=maps["rgb"], maps_occ=maps["occ"])
    data = dict(pts, probe_pos=c["probe_pos"], K=4, S=32, target=rng.uniform(0, 1, (M, 3)).astype(np.float32),
                traced_rgb=traced["rgb"].astype(np.float64), traced_occ=traced["occ"].astype(np.float64))
    return params, data


def _gpu_optimizer(sop, params, data):
    maps = np.concatenate([params["maps_rgb"], params["maps_occ"][..., None]], axis=-1)
    traced = np.concatenate([data["traced_rgb"], data["traced_occ"][..., None]], axis=-1)
    return sop.TextureOptimizer(cuda(params["albedo"]), cuda(params["rough"]), cuda(params["metal"]),
                                cuda(params["env"]), cuda(maps), cuda(traced), cuda(data["probe_pos"]))


def test_first_step_matches_oracle(sop, opt, problem):
    """One step from the same float32 state: the L_pbr of the shading and the
    update of every block. At the first step Adam moves each element by
    lr g/(|g| + eps), so elements whose oracle gradient is at the noise
    level of the float32 adjoint (below 1e-5 of the block's largest) are
    left out; the rest must move like the oracle's within 1e-3 lr."""
    params, data = problem
    st = opt.init_state({k: np.asarray(v, np.float32).astype(np.float64) for k, v in params.items()})
    before = {k: st[k].copy() for k in opt.BLOCKS}
    loss, grads = opt.step(st, data)
    go = _gpu_optimizer(sop, params, data)
    x, n, wo = cuda(data["x"]), cuda(data["n"]), cuda(data["wo"])
    l_pbr = go.step(x, n, wo, cuda(data["target"]), data["K"], data["S"]).item()
    assert l_pbr == pytest.approx(loss["pbr"], rel=1e-5)
    gpu = {k: go.p[k].cpu().numpy().astype(np.float64) for k in ("albedo", "rough", "metal", "env")}
    gpu["maps_rgb"] = go.p["maps"][..., :3].cpu().numpy().astype(np.float64)
    gpu["maps_occ"] = go.p["maps"][..., 3].cpu().numpy().astype(np.float64)
    for k, (lr, _, _) in opt.BLOCKS.items():
        d_gpu, d_orc = gpu[k] - before[k], st[k] - before[k]
        g = np.abs(grads[k])
        keep = g > 1e-5 * g.max()
        assert keep.mean() > 0.5, k
        err = np.abs(d_gpu - d_orc)[keep]
        assert err.max() <= 1e-3 * lr + 1e-7, (k, err.max())


def test_loop_lowers_the_loss(sop, problem):
    params, data = problem
    go = _gpu_optimizer(sop, params, data)
    x, n, wo = cuda(data["x"]), cuda(data["n"]), cuda(data["wo"])
    tgt = cuda(data["target"])
    losses = [go.step(x, n, wo, tgt, data["K"], data["S"]).item() for _ in range(30)]
    assert losses[-1] < 0.95 * losses[0]
    r = go.p["rough"]
    assert float(r.min()) >= 0.1 and float(go.p["maps"][..., 3].max()) <= 1.0 and float(go.p["env"].min()) >= 0.0
