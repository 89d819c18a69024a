"""Pins of the oracle's specular lobe (Sec. 3.1.2, the "simplified Disney"
BRDF of Eq. 2, read as the Burley 2012 / Karis 2013 form).

Every value here is taken out of `orc_brdf` itself (the function the query
uses), in configurations where the other factors are known:

* mirror configuration: n = z, w_o and w_i symmetric about n, so h = n,
  n.h = 1 and v.h = n.l = n.v = mu. Then D = 1/(pi alpha^2) (pinned by the
  normalisation test of test_oracle_query.py) and
  f_spec = F(mu) G1(mu)^2 / (4 pi alpha^2 mu^2).
* metal = 1, albedo = 1 gives F = 1 (F0 = albedo), so G1 comes out alone;
  metal = 1, albedo = 0 gives F0 = 0, so the Schlick term comes out alone.

Each pin is set against mathematics independent of the oracle's formulas:
the exact Smith masking of the GGX slope distribution by numerical
integration, the cosine-weighted moment of (1 - mu)^5, the Fresnel
equations of a dielectric of refractive index 1.5. A wrong remap of k
(r^2/2, the image-based-lighting form), a wrong Schlick exponent or a wrong
dielectric F0 fails one of them.
"""
import numpy as np
import pytest
from scipy import integrate


def _mirror(mu):
    mu = np.atleast_1d(np.asarray(mu, np.float64))
    s = np.sqrt(1 - mu * mu)
    n = np.tile([0.0, 0.0, 1.0], (len(mu), 1))
    wo = np.stack([s, np.zeros_like(mu), mu], 1)
    wi = np.stack([-s, np.zeros_like(mu), mu], 1)
    return n, wo, wi


def _f(orc, mu, albedo, rough, metal, spec=0.5):
    n, wo, wi = _mirror(mu)
    m = len(n)
    a = np.broadcast_to(np.asarray(albedo, np.float64), (m, 3))
    return orc.brdf(n, wo, wi, a, np.full(m, rough), np.full(m, metal), spec)


def _g1_from_brdf(orc, mu, rough):
    """G1(mu) read out of f with F = 1 (metal 1, albedo 1), D = 1/(pi alpha^2)."""
    mu = np.atleast_1d(np.asarray(mu, np.float64))
    f = _f(orc, mu, [1.0, 1.0, 1.0], rough, 1.0)[:, 0]
    al = rough * rough
    return np.sqrt(f * 4 * np.pi * al * al * mu * mu)


def _smith_ggx_exact(mu, al):
    """Smith masking G1 = 1/(1 + Lambda) of the GGX slope distribution
    P22(x, y) = 1/(pi al^2 (1 + (x^2 + y^2)/al^2)^2), with
    Lambda = (1/c) int_c^inf (q - c) P2(q) dq, c = cot(theta), and P2 the
    marginal of P22 along the direction's azimuth, both by quadrature
    (Heitz 2014, "Understanding the Masking-Shadowing Function")."""
    c = mu / np.sqrt(1 - mu * mu)
    p22 = lambda y, x: 1.0 / (np.pi * al * al * (1 + (x * x + y * y) / (al * al)) ** 2)
    p2 = lambda x: integrate.quad(lambda y: p22(y, x), -np.inf, np.inf, epsabs=1e-13, epsrel=1e-12)[0]
    lam = integrate.quad(lambda x: (x - c) * p2(x), c, np.inf, limit=400, epsabs=1e-13, epsrel=1e-12)[0] / c
    return 1.0 / (1.0 + lam)


def _fresnel_dielectric(mu, eta=1.5):
    """Unpolarised reflectance of a smooth dielectric from the Fresnel
    equations (air to index eta), cos of the incidence angle mu."""
    st = np.sqrt(1 - mu * mu) / eta
    ct = np.sqrt(1 - st * st)
    rs = ((mu - eta * ct) / (mu + eta * ct)) ** 2
    rp = ((eta * mu - ct) / (eta * mu + ct)) ** 2
    return 0.5 * (rs + rp)


ROUGH = (0.1, 0.3, 0.5, 0.7, 1.0)


@pytest.mark.parametrize("rough", ROUGH)
def test_g1_grazing_slope_matches_smith_ggx(orc, rough):
    # Schlick's form mu/(mu(1-k)+k) has slope 1/k at grazing; exact Smith-GGX
    # has slope 2/alpha there, so k = alpha/2 matches it. With Karis's
    # remapped roughness alpha' = ((r+1)/2)^2 that is k = (r+1)^2/8. At
    # mu = 1e-3 both are within 1% of their grazing slope; k = r^2/2 is off
    # by the factor alpha'/r^2 (2.25 at r = 0.5, 30 at r = 0.1).
    ap = ((rough + 1) / 2) ** 2
    mu = 1e-3
    g_orc = _g1_from_brdf(orc, mu, rough)[0]
    g_ex = _smith_ggx_exact(mu, ap)
    assert abs(g_orc / g_ex - 1) < 1e-2, (g_orc, g_ex)
    if rough < 1.0:
        k_ibl = rough * rough / 2
        assert abs(mu / (mu * (1 - k_ibl) + k_ibl) / g_ex - 1) > 0.2


@pytest.mark.parametrize("rough", ROUGH)
def test_g1_within_schlick_error_of_smith_ggx(orc, rough):
    # Across the hemisphere Schlick's approximation of Smith-GGX (k = alpha'/2)
    # stays within 0.1 of it (the largest gap, 0.099, is at r = 0.1 near
    # mu = 0.25; exact at r = 1). The IBL remap k = r^2/2 misses by 0.17-0.48
    # at r <= 0.5.
    ap = ((rough + 1) / 2) ** 2
    mus = np.linspace(0.1, 0.95, 18)
    g_orc = _g1_from_brdf(orc, mus, rough)
    g_ex = np.array([_smith_ggx_exact(m, ap) for m in mus])
    assert np.max(np.abs(g_orc - g_ex)) < 0.1
    assert np.all(g_orc <= 1 + 1e-12) and np.all(np.diff(g_orc) > 0)
    g_one = _g1_from_brdf(orc, np.array([1.0 - 1e-12]), rough)[0]
    assert abs(g_one - 1) < 1e-9  # no masking at normal incidence


@pytest.mark.parametrize("rough", (0.2, 0.6))
def test_schlick_fresnel_cosine_moment(orc, rough):
    # With metal = 1, F0 = albedo per channel. Channels with F0 = 0, 0.3 and 1
    # give s(mu) = f[0]/f[2] = (1 - v.h)^5 and the affine form F0 + (1-F0) s.
    # The cosine-weighted hemispherical mean of (1 - mu)^p is 2/((p+1)(p+2)):
    # 1/21 for Schlick's p = 5 (1/15 for p = 4). Gauss-Legendre with 16 nodes
    # is exact for the degree-6 integrand.
    x, w = np.polynomial.legendre.leggauss(16)
    mu = 0.5 * (x + 1)
    f = _f(orc, mu, [0.0, 0.3, 1.0], rough, 1.0)
    s = f[:, 0] / f[:, 2]
    assert np.allclose(f[:, 1] / f[:, 2], 0.3 + 0.7 * s, rtol=1e-12, atol=1e-14)
    moment = np.sum(0.5 * w * s * 2 * mu)
    assert abs(moment - 1.0 / 21.0) < 1e-12
    # the full Fresnel factor's moment is F0 + (1 - F0)/21
    F = f[:, 1] / f[:, 2]
    assert abs(np.sum(0.5 * w * F * 2 * mu) - (0.3 + 0.7 / 21.0)) < 1e-12


def test_dielectric_f0_and_fresnel_equations(orc):
    # metal = 0, specular = 0.5: F0 is the normal-incidence reflectance of a
    # dielectric of index 1.5, ((1.5-1)/(1.5+1))^2 = 0.04. Read as
    # F(mu) = f(metal 0, albedo 0) / f(metal 1, albedo 1) in the mirror
    # configuration (same D and G). Schlick's curve stays within 0.036 of the
    # Fresnel equations for index 1.5 over the whole hemisphere (exponent 4
    # or 6 would miss by 0.10 or 0.055).
    rough = 0.4
    mu = np.linspace(1e-3, 1 - 1e-9, 400)
    F = _f(orc, mu, [0.0, 0.0, 0.0], rough, 0.0)[:, 0] / _f(orc, mu, [1.0, 1.0, 1.0], rough, 1.0)[:, 0]
    assert abs(F[-1] - ((1.5 - 1) / (1.5 + 1)) ** 2) < 1e-9
    assert np.max(np.abs(F - _fresnel_dielectric(mu))) < 0.036
    # normal incidence exactly (w_o = w_i = n): D = 1/(pi alpha^2), G = 1, so
    # f - (1-m) a/pi = F0 / (4 pi alpha^2); metal = 0 gives F0 = 0.04 for any
    # albedo, metal = 1 gives F0 = albedo, and the metallic blend is linear.
    n = np.tile([0.0, 0.0, 1.0], (3, 1))
    a = np.array([[0.2, 0.5, 0.9]] * 3)
    mt = np.array([0.0, 0.5, 1.0])
    f = orc.brdf(n, n, n, a, np.full(3, rough), mt)
    al = rough * rough
    F0 = (f - ((1 - mt)[:, None] * a / np.pi)) * 4 * np.pi * al * al
    assert np.allclose(F0[0], 0.04, rtol=1e-12)
    assert np.allclose(F0[2], a[2], rtol=1e-12)
    assert np.allclose(F0[1], 0.5 * (F0[0] + F0[2]), rtol=1e-12)
