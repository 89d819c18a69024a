"""Pins of the surrogate's texel-feature oracle (oracle/surrogate_oracle.c):
the near list against brute force, the near composite against the single-
and two-Gaussian closed forms, the far-field grid against mass conservation
and brute-force cell indices, and the march against homogeneous media and a
single occupied cell (closed forms of the optical depth and the colour)."""
import numpy as np
import pytest

Q = 2.0 ** 20
FIX = 2.0 ** 40


def _gauss(mean, scale, opacity, rgb, quat=None):
    n = len(mean)
    q = np.tile([1.0, 0.0, 0.0, 0.0], (n, 1)) if quat is None else quat
    return dict(mean=np.asarray(mean, np.float32), scale=np.asarray(scale, np.float32),
                quat=np.asarray(q, np.float32), opacity=np.asarray(opacity, np.float32),
                rgb=np.asarray(rgb, np.float32))


def test_near_list_is_brute_force(orc):
    rng = np.random.default_rng(0)
    mean = rng.uniform(-1, 1, (4000, 3)).astype(np.float32)
    mean[10] = mean[11]  # a duplicate: ties go to the lower index
    pp = np.vstack([mean[10] + 1e-3, rng.uniform(-1, 1, (20, 3))]).astype(np.float32)
    r_n, KN = 0.35, 64
    lst, t0 = orc.surr_near_list(pp, mean, r_n, KN)
    qm = np.rint(mean.astype(np.float64) * Q).astype(np.int64)
    for i, p in enumerate(pp):
        qp = np.rint(p.astype(np.float64) * Q).astype(np.int64)
        key = ((qm - qp) ** 2).sum(1)
        lim = np.floor((r_n * Q) ** 2)
        inside = np.nonzero(key <= lim)[0]
        order = inside[np.lexsort((inside, key[inside]))][:KN]
        want = np.full(KN, -1)
        want[:len(order)] = order
        assert np.array_equal(lst[i], want)
        full = len(order) == KN
        assert t0[i] == pytest.approx(np.sqrt(key[order[-1]]) / Q if full else r_n, rel=1e-15)
    assert lst[0][0] == 10 and lst[0][1] == 11


def test_near_single_gaussian_closed_form(orc):
    # isotropic Gaussian of scale s at perpendicular distance r from the ray
    # of the texel looking straight up (z), at height h: alpha = o exp(-r^2 /
    # 2 s^2), t* = h, L = alpha rgb
    R = 8
    d_up = orc._texel_dir(R, 3, 3)  # a texel near +z; use its own direction
    s, o, h, r = 0.05, 0.7, 0.4, 0.03
    perp = np.cross(d_up, [1.0, 0.0, 0.0])
    perp /= np.linalg.norm(perp)
    mu = h * d_up + r * perp
    g = _gauss([mu], [[s, s, s]], [o], [[0.2, 0.5, 0.9]])
    feats, flags, _, _ = orc.surr_features(g, np.zeros((1, 3), np.float32), R, r_n=1.0,
                                           near_list=(np.array([[0]], np.int32), np.array([1.0])))
    f = feats[0, 3 * R + 3]
    mu32 = g["mean"][0].astype(np.float64)
    t_star = mu32 @ d_up
    r32 = np.linalg.norm(mu32 - t_star * d_up)
    s32, o32 = float(np.float32(s)), float(np.float32(o))
    alpha = o32 * np.exp(-r32 ** 2 / (2 * s32 * s32))
    assert f[3] == pytest.approx(alpha, rel=1e-12)
    assert f[4:7] == pytest.approx(alpha * g["rgb"][0].astype(np.float64), rel=1e-12)
    assert f[7] == pytest.approx(t_star, rel=1e-12)
    assert f[8] == pytest.approx(alpha, rel=1e-12)


def test_near_composites_in_list_order(orc):
    # two Gaussians on the +z ray: listed far-first, the far one is
    # composited first (list order, not depth order)
    R = 4
    g = _gauss([[0, 0, 0.6], [0, 0, 0.3]], [[0.3] * 3] * 2, [0.5, 0.8], [[1, 0, 0], [0, 1, 0]])
    d = np.array([orc._texel_dir(R, i % R, i // R) for i in range(R * R)])
    t = int(np.argmax(d[:, 2]))
    feats, _, _, _ = orc.surr_features(g, np.zeros((1, 3), np.float32), R, r_n=1.0,
                                       near_list=(np.array([[0, 1]], np.int32), np.array([1.0])))
    f = feats[0, t]
    mu = g["mean"].astype(np.float64)
    s32 = float(np.float32(0.3))
    a = [float(g["opacity"][k]) * np.exp(-np.sum((mu[k] - (mu[k] @ d[t]) * d[t]) ** 2) / (2 * s32 ** 2))
         for k in (0, 1)]
    assert min(a) > 0.1
    assert f[3] == pytest.approx(1 - (1 - a[0]) * (1 - a[1]), rel=1e-12)
    assert f[4] == pytest.approx(a[0], rel=1e-12)               # red first
    assert f[5] == pytest.approx((1 - a[0]) * a[1], rel=1e-12)  # then green


def test_grid_conserves_mass_and_bins_by_integer_cells(orc):
    rng = np.random.default_rng(1)
    n = 3000
    g = _gauss(rng.uniform(-0.7, 0.9, (n, 3)), np.exp(rng.uniform(-6, -3, (n, 3))), rng.uniform(0.0, 1.0, n),
               rng.uniform(0, 1, (n, 3)))
    qlo, hq, dims, mass, col = orc.surr_grid(g, G=16)
    use = g["opacity"] >= 1.0 / 255.0
    s = np.sort(g["scale"].astype(np.float64), axis=1)
    m = -np.log1p(-np.minimum(g["opacity"].astype(np.float64), 0.99)) * 2 * np.pi * s[:, 1] * s[:, 2]
    m[~use] = 0.0
    assert abs(mass.sum() / FIX - m.sum()) <= n / FIX
    q = np.rint(g["mean"].astype(np.float64) * Q).astype(np.int64)
    assert max(dims) == 16 and hq == -(-(q[use].max(0) - q[use].min(0) + 1).max() // 16)
    c = (q - qlo) // hq
    cell = (c[:, 2] * dims[1] + c[:, 1]) * dims[0] + c[:, 0]
    want = np.zeros(int(np.prod(dims)))
    np.add.at(want, cell[use], np.rint(m[use] * FIX))
    assert np.array_equal(mass, want.astype(np.int64))


def _uniform_grid(dims, hq, qlo, m_per_cell, rgb):
    cells = int(np.prod(dims))
    mass = np.full(cells, int(round(m_per_cell * FIX)), np.int64)
    col = np.tile(np.rint(np.asarray(rgb) * m_per_cell * FIX).astype(np.int64), (cells, 1))
    return np.asarray(qlo, np.int64), hq, np.asarray(dims, np.int32), mass, col


def test_march_homogeneous_medium_closed_form(orc):
    # every cell carries the same mass: sigma constant, so tau(t) = sigma
    # (t - t0) inside the box; checkpoints and the colour follow in closed
    # form (L_f = rgb (1 - exp(-tau_total)))
    hq = 1 << 14  # h = 1/64
    dims = (64, 64, 64)
    qlo = (-(32 << 14),) * 3  # the box [-0.5, 0.5]^3
    h = hq / Q
    m = 0.3 * h ** 3  # sigma = 0.3
    grid = _uniform_grid(dims, hq, qlo, m, [0.25, 0.5, 1.0])
    R = 8
    t0 = 0.05
    far = orc.surr_far(np.zeros((1, 3), np.float32), np.array([t0]), R, *grid)[0]
    sig = grid[3][0] / FIX / h ** 3  # the fixed-point mass as stored
    assert sig == pytest.approx(0.3, rel=1e-6)  # one fixed-point quantum of the mass
    for t in range(R * R):
        d = orc._texel_dir(R, t % R, t // R)
        t_exit = np.min(0.5 / np.abs(d[np.abs(d) > 0]))
        for k, mult in enumerate((2, 4, 8, 16, 32)):
            tau = sig * (min(t0 + mult * h, t_exit) - t0)
            assert far[t, k] == pytest.approx(1 - np.exp(-tau), rel=1e-9, abs=1e-12)
        tau_tot = sig * (t_exit - t0)
        assert far[t, 5] == pytest.approx(1 - np.exp(-tau_tot), rel=1e-9)
        c_eff = grid[4][0] / grid[3][0]  # the stored mass-weighted colour
        assert far[t, 6:] == pytest.approx(c_eff * (1 - np.exp(-tau_tot)), rel=1e-9)


def test_march_single_cell_is_sigma_times_chord(orc):
    hq = 1 << 16  # h = 1/16
    dims = (8, 8, 8)
    qlo = (0, 0, 0)
    h = hq / Q
    cells = 512
    mass = np.zeros(cells, np.int64)
    col = np.zeros((cells, 3), np.int64)
    c = (3, 4, 5)
    cell = (c[2] * 8 + c[1]) * 8 + c[0]
    sigma = 2.0
    mass[cell] = int(round(sigma * h ** 3 * FIX))
    col[cell] = np.rint(np.array([1.0, 0.0, 0.5]) * sigma * h ** 3 * FIX).astype(np.int64)
    p = np.array([[0.21, 0.28, 0.2]], np.float32)  # just below the cell
    R = 16
    far = orc.surr_far(p, np.array([0.0]), R, np.array(qlo), hq, np.array(dims), mass, col)[0]
    lo = np.array(c) * h
    hi = lo + h
    hit = 0
    for t in range(R * R):
        d = orc._texel_dir(R, t % R, t // R)
        with np.errstate(divide="ignore", invalid="ignore"):
            t1 = (lo - p[0].astype(np.float64)) / d
            t2 = (hi - p[0].astype(np.float64)) / d
        ta = np.max(np.minimum(t1, t2))
        tb = np.min(np.maximum(t1, t2))
        chord = max(0.0, tb - max(ta, 0.0))
        m_exact = mass[cell] / FIX / h ** 3
        assert far[t, 5] == pytest.approx(1 - np.exp(-m_exact * chord), rel=1e-9, abs=1e-14)
        hit += chord > 0
    assert hit > 0


def test_march_conditioning_single_cell(orc):
    """The far march's conditioning (with_sens) for rays through one dense
    cell: sigma times the FP32 rounding scales of the entry and exit times,
    e(t) = 2^-24 ((|B| + |o_a|) / |d_a| + 2 |t|) with B the crossed face's
    coordinate; zero for rays that miss the cell. And it covers what it is
    for: the chord taken with FP32 boundary times (B - o_a) / d_a moves tau
    by less than it."""
    hq = 1 << 16  # h = 1/16
    dims = (8, 8, 8)
    h = hq / Q
    mass = np.zeros(512, np.int64)
    col = np.zeros((512, 3), np.int64)
    c = (3, 4, 5)
    cell = (c[2] * 8 + c[1]) * 8 + c[0]
    mass[cell] = int(round(40.0 * h ** 3 * FIX))
    p = np.array([[0.21, 0.28, 0.2]], np.float32)
    R = 16
    far, sens = orc.surr_far(p, np.array([0.0]), R, np.zeros(3, np.int64), hq, np.array(dims), mass, col,
                             with_sens=True)
    sig = mass[cell] / FIX / h ** 3
    eps = 2.0 ** -24
    o = p[0].astype(np.float64)
    lo = np.array(c) * h
    hi = lo + h
    hit = 0
    for t in range(R * R):
        d = orc._texel_dir(R, t % R, t // R)
        with np.errstate(divide="ignore", invalid="ignore"):
            t1 = (lo - o) / d
            t2 = (hi - o) / d
        tin, tout = np.minimum(t1, t2), np.maximum(t1, t2)
        a_in, a_out = int(np.argmax(tin)), int(np.argmin(tout))
        ta, tb = tin[a_in], tout[a_out]
        if not tb > max(ta, 0.0):
            assert sens[0, t] == 0.0
            continue
        hit += 1
        B_in = lo[a_in] if d[a_in] > 0 else hi[a_in]
        B_out = hi[a_out] if d[a_out] > 0 else lo[a_out]
        e_in = eps * ((abs(B_in) + abs(o[a_in])) / abs(d[a_in]) + 2 * abs(ta))
        e_out = eps * ((abs(B_out) + abs(o[a_out])) / abs(d[a_out]) + 2 * abs(tb))
        assert sens[0, t] == pytest.approx(sig * (e_in + e_out), rel=1e-12)
        # the chord from FP32 boundary times
        d32 = d.astype(np.float32)
        ta32 = (np.float32(B_in) - p[0][a_in]) / d32[a_in]
        tb32 = (np.float32(B_out) - p[0][a_out]) / d32[a_out]
        assert abs(sig * (float(tb32) - float(ta32)) - sig * (tb - ta)) <= sens[0, t]
    assert hit >= 8
