"""GPU parity of the automatic probe placement (Sec. 3.2: farthest point
sampling, offset along the normals) against the oracle, through the C ABI:
the chosen indices bit-exact (integer keys), the positions equal to the
oracle's double result rounded once."""
import numpy as np
import pytest
import torch

from paper_2510_07729_gb300 import inputs as I

pytestmark = pytest.mark.gpu
F = np.float32


@pytest.fixture(scope="module")
def sop():
    from paper_2510_07729_gb300 import sop as S
    S.load()
    return S


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def cloud(seed, n, dup=0):
    rng = np.random.default_rng(seed)
    pts = rng.uniform(-1, 1, (n, 3)).astype(F)
    if dup:
        pts[n // 2:n // 2 + dup] = pts[1]
    nrm = rng.standard_normal((n, 3))
    return pts, (nrm / np.linalg.norm(nrm, axis=1, keepdims=True)).astype(F)


@pytest.mark.parametrize("n,k,start,dup", [(1, 1, 0, 0), (9, 9, 4, 0), (1000, 1000, 0, 30), (65_536, 4096, 0, 0),
                                           (74_000, 300, 17, 5), (200_000, 512, 0, 0)])
def test_fps_matches_oracle(sop, orc, n, k, start, dup):
    """Slices in shared memory (up to ~75k points) and in the workspace
    (200k); fewer points than CTAs; duplicates (ties, and a covering radius
    that reaches zero when k = n)."""
    pts, nrm = cloud(n + k, n, dup)
    off = 0.03
    idx, pos = sop.place_probes(cuda(pts), k, nrm=cuda(nrm), offset=off, start=start)
    oi, op = orc.fps(pts, k, start=start, nrm=nrm, offset=float(F(off)))
    assert np.array_equal(idx.cpu().numpy(), oi)
    assert np.array_equal(pos.cpu().numpy(), op.astype(F))


def test_fps_on_a_surface_is_deterministic(sop, orc):
    """The object's 65,536 surface samples, 4,096 probes offset by 1% of the
    object's size: twice the same, and the oracle's."""
    _, _, _, _, _, samp, diag = I._object(1)
    rng = np.random.default_rng(0)
    pts = samp.astype(F)
    nrm = I._unit_vectors(rng, len(pts)).astype(F)
    a = sop.place_probes(cuda(pts), 4096, nrm=cuda(nrm), offset=0.01 * diag)
    b = sop.place_probes(cuda(pts), 4096, nrm=cuda(nrm), offset=0.01 * diag)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    oi, _ = orc.fps(pts, 4096)
    assert np.array_equal(a[0].cpu().numpy(), oi)
