"""Pins of the oracle's cosmology inputs (growth, sigma_8, transfer functions).

* Einstein-de Sitter: D = a and f = 1 exactly; v/psi = 100 a^{-1/2}.
* LambdaCDM growth against an independent ODE integration (scipy solve_ivp)
  of D'' + (3/a + E'/E) D' - 3 Om D / (2 a^5 E^2) = 0, and f against a
  numerical derivative of ln D.
* The variance integrator against the Gaussian-window power-law closed form
  sigma^2 = A Gamma((n+3)/2) / (4 pi^2 R^(n+3)).
* sigma(8) of the normalised P(k) re-integrated with a different rule.
* Transfer functions: T -> 1 at k -> 0, monotone decrease, the EH98
  sound-horizon fit near the measured Planck 2018 drag-epoch value
  (147.09 Mpc), and the zero-baryon EH shape close to BBKS.
"""
import math

import numpy as np
import pytest
from scipy import integrate, special

from oracle.cosmology import Cosmology
from tests.oracle_cases import BBKS, EH_NW, cosmology_from


def test_eds_growth_exact():
    c = Cosmology(1.0, 0.7, 1.0, 0.8, omega_l=0.0)
    for a in (0.01, 0.1, 0.5, 1.0):
        assert abs(c.growth_unnormalised(a) - a) < 1e-12 * a
        assert abs(c.growth(a) - a) < 1e-12 * a
        assert abs(c.growth_rate(a) - 1.0) < 1e-12
        assert abs(c.velocity_factor(a) - 100.0 / math.sqrt(a)) < 1e-10 / math.sqrt(a)


@pytest.mark.parametrize("om,ol", [(0.3, 0.7), (0.31, 0.69), (0.25, 0.6)])
def test_growth_against_ode(om, ol):
    c = Cosmology(om, 0.7, 1.0, 0.8, omega_l=ol)
    ok = 1.0 - om - ol

    def rhs(a, y):
        e2 = om / a ** 3 + ok / a ** 2 + ol
        dlne = (-3 * om / a ** 4 - 2 * ok / a ** 3) / (2 * e2)
        return [y[1], -(3 / a + dlne) * y[1] + 1.5 * om / (a ** 5 * e2) * y[0]]

    a0 = 1e-5  # matter dominated: D = a, D' = 1 up to O(a) curvature/Lambda terms
    sol = integrate.solve_ivp(rhs, (a0, 1.0), [a0, 1.0], rtol=1e-12, atol=1e-16,
                              dense_output=True, method="DOP853")
    for a in (0.01, 1 / 51.0, 1 / 101.0, 0.3, 0.7):
        d_ode = sol.sol(a)[0] / sol.sol(1.0)[0]
        assert abs(c.growth(a) - d_ode) < 1e-8 * d_ode
        f_ode = a * sol.sol(a)[1] / sol.sol(a)[0]
        assert abs(c.growth_rate(a) - f_ode) < 1e-8


def test_growth_rate_is_log_derivative():
    c = cosmology_from(BBKS)
    for a in (0.02, 0.5, 0.9):
        eps = 1e-4
        num = (math.log(c.growth(a * math.exp(eps))) - math.log(c.growth(a * math.exp(-eps)))) / (2 * eps)
        assert abs(num - c.growth_rate(a)) < 1e-7


@pytest.mark.parametrize("n", [-1.5, 0.0, 1.0])
def test_variance_gaussian_window_closed_form(n):
    c = cosmology_from(BBKS)
    amp, radius = 2.5, 5.0
    got = c.variance(lambda k: amp * k ** n, radius, window=lambda x: math.exp(-0.5 * x * x),
                     kmin=1e-8, kmax=1e2)
    want = amp * special.gamma((n + 3) / 2) / (4 * math.pi ** 2 * radius ** (n + 3))
    assert abs(got - want) < 1e-10 * want


@pytest.mark.parametrize("cfg", [BBKS, EH_NW])
def test_sigma8_reintegrated(cfg):
    c = cosmology_from(cfg)
    # composite Simpson in ln k on a dense grid: an integration rule unlike quad
    lnk = np.linspace(math.log(1e-6), math.log(1e3), 400001)
    k = np.exp(lnk)
    x = 8.0 * k
    w = np.where(x < 1e-2, 1 - x * x / 10, 3 * (np.sin(x) - x * np.cos(x)) / np.where(x < 1e-2, 1, x) ** 3)
    f = k ** 3 * c.power(k) * w * w / (2 * math.pi ** 2)
    var = integrate.simpson(f, x=lnk)
    assert abs(math.sqrt(var) - c.sigma_8) < 1e-9


@pytest.mark.parametrize("cfg", [BBKS, EH_NW])
def test_transfer_limits(cfg):
    c = cosmology_from(cfg)
    t = c.transfer_bbks if cfg["tf"] == "bbks" else c.transfer_eh_nowiggle
    assert abs(float(t(1e-7)) - 1.0) < 1e-4
    k = np.logspace(-5, 2, 400)
    tk = t(k)
    assert np.all(np.diff(tk) < 0) and np.all(tk > 0)


def test_eh_sound_horizon_near_planck():
    c = Cosmology(0.3111, 0.6766, 0.9665, 0.8102, tf="eh_nw", omega_b=0.04897)
    assert abs(c.eh_sound_horizon() - 147.09) / 147.09 < 0.03


def test_eh_zero_baryon_close_to_bbks():
    """With f_b -> 0 the EH shape (Gamma = Om h) describes the same CDM transfer as BBKS."""
    c = Cosmology(0.3, 0.7, 1.0, 0.8, tf="eh_nw", omega_b=1e-8, t_cmb=2.7)
    k = np.logspace(-3, 0, 200)
    rel = np.abs(c.transfer_eh_nowiggle(k) / c.transfer_bbks(k) - 1.0)
    assert rel.max() < 0.15


def test_power_scales_with_sigma8_squared():
    a = cosmology_from(BBKS)
    b = cosmology_from(dict(BBKS, sigma_8=1.6))
    k = np.array([0.01, 0.1, 1.0])
    np.testing.assert_allclose(b.power(k), 4.0 * a.power(k), rtol=1e-12)


def test_table_transfer_reproduces_analytic():
    """A tabulated P(k) sampled from the BBKS form gives the same normalised P."""
    a = cosmology_from(BBKS)
    tk = np.logspace(-5, 2.5, 4000)
    tab = Cosmology(0.3, 0.7, 0.96, 0.8, tf="table", tab_k=tk, tab_p=a.power(tk) * 3.0)
    k = np.array([0.01, 0.1, 1.0])
    np.testing.assert_allclose(tab.power(k), a.power(k), rtol=2e-4)


# ---------------------------------------------------------------------------
# Transfer-function coefficients, pinned by the series and asymptotes that the
# published formulas fix (derived by hand from BBKS eq. G3 and EH98 eq. 29,
# not by evaluating the formulas again):
#   BBKS, q -> 0:   T = 1 - (2.34/2 + 3.89/4) q
#                         + (2.34^2/3 + (2.34/2)(3.89/4) - 16.1^2/4 + (5/32) 3.89^2) q^2 + O(q^3)
#   BBKS, q -> oo:  T (2.34 q)(6.71 q) / ln(1 + 2.34 q) = 1 - 5.46^3 / (4 6.71^4 q) + O(q^-2)
#   EH98, q -> 0:   (1 - T0) / q^2 -> (14.2 + 731) / ln(2e)
#   EH98, q -> oo:  T0 q^2 14.2 / ln(2e + 1.8 q) = 1 - (731/62.5)/(14.2 q) + O(q^-2)
# A mistyped coefficient moves one of these limits.

def test_bbks_series_at_small_q():
    t = Cosmology.bbks_of_q
    c1 = 2.34 / 2 + 3.89 / 4
    c2 = 2.34 ** 2 / 3 + (2.34 / 2) * (3.89 / 4) - 16.1 ** 2 / 4 + (5 / 32) * 3.89 ** 2
    for q in (1e-6, 2e-6):  # the q^3 term (coefficient about 340) bounds the difference
        assert abs((1 - float(t(q))) / q - (c1 - c2 * q)) < 500 * q * q
    # second coefficient by Richardson extrapolation (removes the q^3 term)
    r = lambda q: (float(t(q)) - 1 + c1 * q) / q ** 2
    assert abs(2 * r(5e-6) - r(1e-5) - c2) < 1e-5 * abs(c2)


def test_bbks_asymptote_at_large_q():
    t = Cosmology.bbks_of_q
    d1 = -5.46 ** 3 / (4 * 6.71 ** 4)
    for q in (1e5, 1e6):
        g = float(t(q)) * (2.34 * q) * (6.71 * q) / math.log1p(2.34 * q)
        assert abs((g - 1) * q - d1) < 2e-5 * abs(d1) * (1e6 / q)


def test_eh_shape_series_at_small_q():
    t = Cosmology.eh_t0_of_q
    r = lambda q: (1 - float(t(q))) / q ** 2
    # r is linear in q near 0 (731/(1 + 62.5 q) and ln(2e + 1.8 q)): Richardson
    lim = 2 * r(5e-6) - r(1e-5)
    assert abs(lim - (14.2 + 731.0) / math.log(2 * math.e)) < 1e-6 * lim


def test_eh_shape_asymptote_at_large_q():
    t = Cosmology.eh_t0_of_q
    d1 = -(731.0 / 62.5) / 14.2
    for q in (1e6, 1e8):
        g = float(t(q)) * q * q * 14.2 / math.log(2 * math.e + 1.8 * q)
        assert abs((g - 1) * q - d1) < 1e-4 * abs(d1)


def test_eh_gamma_eff_limits():
    c = cosmology_from(EH_NW)
    gam = c.eh_gamma_eff(np.array([1e-8, 1e6]))
    fb = c.omega_b / c.omega_m
    assert abs(gam[0] / (c.omega_m * c.h) - 1) < 1e-12
    assert 0.5 < gam[1] / (c.omega_m * c.h) < 1.0  # alpha < 1 with baryons
    nob = Cosmology(0.31, 0.68, 0.965, 0.81, tf="eh_nw", omega_b=1e-12)
    g2 = nob.eh_gamma_eff(np.array([1e-8, 1e6]))
    assert np.allclose(g2, 0.31 * 0.68, rtol=1e-9) and fb > 0


@pytest.mark.parametrize("cfg", [BBKS, EH_NW])
def test_sigma8_certified_by_gauss_legendre(cfg):
    """sigma(8) of the normalised P(k) by composite 16-point Gauss-Legendre:
    4000 pieces in ln k below k = 1/R, then pieces of pi/(4R) in k up to
    1e3 h/Mpc (a quarter of the window's oscillation each), all vectorised:
    an integration entirely unlike the oracle's adaptive quadrature."""
    from scipy.special import roots_legendre
    c = cosmology_from(cfg)
    radius = 8.0
    x, w = roots_legendre(16)

    def gl(edges, f):
        lo, hi = edges[:-1, None], edges[1:, None]
        pts = 0.5 * (lo + hi) + 0.5 * (hi - lo) * x[None, :]
        return float(np.sum(0.5 * (hi - lo) * w[None, :] * f(pts)))

    def win2(xx):
        full = 3 * (np.sin(xx) - xx * np.cos(xx)) / np.where(xx < 1e-2, 1.0, xx) ** 3
        return np.where(xx < 1e-2, 1 - xx * xx / 10 + xx ** 4 / 280, full) ** 2

    kb = 1.0 / radius
    e1 = np.linspace(math.log(1e-6), math.log(kb), 4001)
    i1 = gl(e1, lambda l: np.exp(3 * l) * c.power(np.exp(l)) * win2(np.exp(l) * radius))
    e2 = np.append(np.arange(kb, 1e3, math.pi / (4 * radius)), 1e3)
    i2 = gl(e2, lambda k: k * k * c.power(k) * win2(k * radius))
    sigma = math.sqrt((i1 + i2) / (2 * math.pi ** 2))
    assert abs(sigma / c.sigma_8 - 1) < 1e-12


def test_variance_integration_has_no_quadrature_warnings():
    import warnings
    for cfg in (BBKS, EH_NW):
        c = cosmology_from(cfg)
        with warnings.catch_warnings():
            warnings.simplefilter("error")
            c.amplitude()
