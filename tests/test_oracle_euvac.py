"""Pins of the oracle's EUVAC heating (Sec. 2.2 and the appendix table)."""
import math
import os

import numpy as np
import pytest
from scipy import integrate

from oracle import euvac as E
from oracle import physics as P
from paper_2306_01085_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "euvac_table.txt")


def _golden():
    rows = []
    with open(GOLDEN) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            c = line.split()
            lo, _, hi = c[0].partition("-")
            rows.append((float(lo), float(hi or lo), float(c[1]), float(c[2])) + tuple(float(v) for v in c[3:7]))
    return rows


def test_table_matches_the_paper():
    g = _golden()
    assert len(g) == len(E.TABLE) == 37
    for (lo, hi, F, A, *phis), (tlo, thi, tF, tA, *tphis) in zip(g, E.TABLE):
        assert (lo, hi) == (tlo, thi)
        assert math.isclose(F * 1e13, tF, rel_tol=1e-12)      # printed exponent -13, 1e13 meant
        assert math.isclose(A, tA, rel_tol=1e-12)
        for a, b in zip(phis, tphis):                          # N2, O2, O, He
            assert math.isclose(a, b * 1e-22, rel_tol=1e-12, abs_tol=1e-40)


def _column(rt, chi):
    """Exact column along the ray to the Sun of an exponential atmosphere, in units of n H."""
    c = math.cos(chi)
    f = lambda s: math.exp(-(math.sqrt(rt * rt + s * s + 2 * rt * s * c) - rt))
    return integrate.quad(f, 0, np.inf, limit=400, epsabs=0, epsrel=1e-12)[0]


@pytest.mark.parametrize("rt", [100.0, 300.0, 600.0])
def test_chapman_against_quadrature(rt):
    """Day side: the Smith & Smith factor is the exact column to first order in 1/r~ (measured
    r~ x error <= 0.995); lit night side up to 100 degrees within 1 %."""
    for deg in (0, 30, 60, 80, 85, 89.9):
        chi = math.radians(deg)
        ch = float(E.chapman(rt, math.cos(chi), 1e9))
        assert abs(ch - _column(rt, chi)) <= 1.2 / rt * _column(rt, chi), deg
    for deg in (91, 95, 100):
        chi = math.radians(deg)
        ch = float(E.chapman(rt, math.cos(chi), 1e9))
        assert abs(ch - _column(rt, chi)) <= 1e-2 * _column(rt, chi), deg


def test_chapman_vertical_limit_terminator_and_shadow():
    for rt in (50.0, 200.0, 1000.0):
        ch = float(E.chapman(rt, 1.0, 1e9))
        assert 1.0 - 1.5 / rt <= ch <= 1.0
    eps = 1e-9
    day = float(E.chapman(400.0, eps, 1e9))
    night = float(E.chapman(400.0, -eps, 1e9))
    assert abs(day - night) <= 1e-6 * day
    assert abs(day - math.sqrt(math.pi * 400.0 / 2.0)) <= 1e-6 * day
    # 200 km above a 6471 km lower boundary, 170 degrees from the Sun: in the Earth's shadow
    assert np.isinf(E.chapman(400.0, math.cos(math.radians(170)), 6671.0 / 6471.0))
    # same point at 100 degrees: r sin(chi) above the lower boundary, lit
    assert np.isfinite(E.chapman(400.0, math.cos(math.radians(100)), 6671.0 / 6471.0))


def test_declination_and_flux_clamp():
    assert math.degrees(E.declination(172)) == pytest.approx(23.44, abs=0.05)
    assert math.degrees(E.declination(355)) == pytest.approx(-23.44, abs=0.05)
    assert abs(math.degrees(E.declination(80))) < 1.0
    assert abs(math.degrees(E.declination(266))) < 1.0
    assert all(abs(E.declination(d)) <= E.DELTA_0 + 1e-15 for d in range(1, 366))
    _, F, A, _ = E.bins()
    I0 = E.solar_flux(60.0, 60.0)
    assert np.allclose(I0, F * np.maximum(0.8, 1.0 - 20.0 * A))
    assert I0[5] == pytest.approx(0.8 * F[5])            # A = 0.138: 1 - 2.76 < 0.8
    assert np.allclose(E.solar_flux(150.0, 150.0, 2.0), E.solar_flux(150.0, 150.0) / 4.0)


def test_zenith_angle_formula_equals_the_rotating_frame_direction():
    """The paper's latitude / local-time formula against r_hat . s(t), s the direction heating()
    uses."""
    rng = np.random.default_rng(5)
    lat = rng.uniform(-1.5, 1.5, 50)
    lon = rng.uniform(-3.1, 3.1, 50)
    omega, tp = 7.292e-5, 12345.0
    for day in (80.0, 172.0, 300.0):
        delta = E.declination(day)
        ref = E.cos_zenith_latlon(lat, lon, tp, omega, delta)
        s = np.array(E.sun_direction(day, omega * tp))
        rhat = np.stack([np.cos(lat) * np.cos(lon), np.cos(lat) * np.sin(lon), np.sin(lat)])
        assert np.allclose(s @ rhat, ref, atol=1e-14)


def test_column_integrated_heating_is_the_absorbed_flux():
    """Overhead Sun over an isothermal exponential column (constant g): the height integral of
    q_euv equals eps sum_j I_0^j (h c / lambda_j)(1 - exp(-tau_j(bottom))) to the Chapman factor's
    first-order accuracy (r~ ~ 650 here, 0.2 %)."""
    T, m, g, R0 = 600.0, 16 * W.AMU, 9.0, 6471.0e3
    H = W.K_B * T / (m * g)
    n0 = 3e16
    z = np.linspace(0.0, 40 * H, 200001)
    n = n0 * np.exp(-z / H)
    I0 = E.solar_flux(150.0, 150.0)
    q = E.heating_dimensional(n * m, T * np.ones_like(z), R0 + z, np.ones_like(z), R0, m, g * np.ones_like(z), 0.25,
                              I0)
    total = integrate.trapezoid(q, z)
    lam, _, _, phi = E.bins()
    expect = 0.25 * np.sum(I0 * 6.62607015e-34 * 299792458.0 / lam * (1 - np.exp(-n0 * phi * H)))
    assert abs(total - expect) <= 3e-3 * expect


def test_heating_is_analytic_in_the_state():
    """Complex-step derivatives of the nondimensional heating in varrho and sqrt(rho) T agree with
    central differences (what the complex-step Jv of the residual relies on)."""
    d = W.shell_desc(n=2, nr=3, p=1, euvac=True, day=172.0)
    C = P.Coeffs(d)
    x = np.array([[592.5, -300.0, 20.0], [120.0, 610.0, -400.0], [-600.0, 50.0, 10.0]]).T
    u = np.zeros((5, 3))
    u[0] = [-1.0, -3.0, -6.0]
    u[4] = np.exp(0.5 * u[0]) * np.array([1.5, 3.0, 4.5])
    for k in (0, 4):
        du = np.zeros_like(u)
        du[k] = 1.0
        cs = E.heating(u + 1e-30j * du, x, 0.3, C).imag / 1e-30
        h = 1e-6
        fd = (E.heating(u + h * du, x, 0.3, C) - E.heating(u - h * du, x, 0.3, C)) / (2 * h)
        assert np.allclose(cs, fd, rtol=1e-6, atol=1e-20 + 1e-9 * np.abs(cs).max())
    assert np.all(E.heating(u, x, 0.3, C) >= 0)
