"""Pins of the oracle's automatic probe placement (Sec. 3.2: farthest point
sampling of a surface point cloud, then an offset along the normals): a
worked example on a line, brute force with Python integers, agreement with
the input generator's independent float64 FPS, the monotone covering
radius, and the offset."""
import numpy as np
import pytest

from paper_2510_07729_gb300 import inputs as I


def q(v):
    return [int(np.rint(np.float64(a) * 1048576.0)) for a in v]


def brute_fps(pts, k, start=0):
    Q = [q(p) for p in pts]
    dmin = [None] * len(Q)
    cur, out, radii = start, [], []
    for _ in range(k):
        out.append(cur)
        for i, p in enumerate(Q):
            key = sum((a - b) ** 2 for a, b in zip(p, Q[cur]))
            dmin[i] = key if dmin[i] is None else min(dmin[i], key)
        best = max(dmin)
        radii.append(best)
        cur = dmin.index(best)  # the first (lowest index) of the largest
    return out, radii


def test_line_worked_example(orc):
    """Points 0, 1/16, ..., 10/16 on a line from 0: the far end, the middle,
    then the lowest of the tied points at distance 2/16, and so on."""
    pts = np.zeros((11, 3), np.float32)
    pts[:, 0] = np.arange(11) / 16.0
    idx, _ = orc.fps(pts, 7)
    assert idx.tolist() == [0, 10, 5, 2, 7, 1, 3]


@pytest.mark.parametrize("seed,n,k,start", [(0, 60, 60, 0), (1, 200, 37, 5), (2, 90, 90, 89)])
def test_brute_force(orc, seed, n, k, start):
    rng = np.random.default_rng(seed)
    pts = rng.uniform(-1, 1, (n, 3)).astype(np.float32)
    pts[n // 2:n // 2 + 5] = pts[3]  # duplicates: ties, and zero covering radius at the end
    idx, _ = orc.fps(pts, k, start=start)
    want, radii = brute_fps(pts, k, start)
    assert idx.tolist() == want
    assert all(a >= b for a, b in zip(radii, radii[1:]))  # the covering radius never grows


def test_agrees_with_float64_fps(orc):
    rng = np.random.default_rng(3)
    pts = rng.uniform(-1, 1, (3000, 3))
    idx, _ = orc.fps(pts.astype(np.float32), 200)
    ref = I.farthest_point_sampling(pts.astype(np.float32).astype(np.float64), 200)
    assert idx.tolist() == ref.tolist()


def test_offset_along_normals(orc):
    rng = np.random.default_rng(4)
    pts = rng.uniform(-1, 1, (500, 3)).astype(np.float32)
    nrm = rng.standard_normal((500, 3))
    nrm = (nrm / np.linalg.norm(nrm, axis=1, keepdims=True)).astype(np.float32)
    idx, pos = orc.fps(pts, 50, nrm=nrm, offset=0.03)
    np.testing.assert_array_equal(pos, pts[idx].astype(np.float64) + 0.03 * nrm[idx].astype(np.float64))
