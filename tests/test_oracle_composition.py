"""Pins of the oracle's variable composition and transport (Sec. 2.1.1-2.1.2)."""
import math

import numpy as np
import pytest

from oracle import composition as CM
from oracle import euvac as E
from oracle import physics as P
from paper_2306_01085_gb300 import workloads as W

K_B, AMU = W.K_B, W.AMU


def _coeffs(a, b, nu=200.0, al=10.0):
    d = W.shell_desc(n=1, nr=2, p=1)
    d.comp, d.comp_a, d.comp_b, d.eddy_nu, d.eddy_alpha = 1, tuple(a), tuple(b), nu, al
    return P.Coeffs(d)


@pytest.mark.parametrize("k,mass,alpha", [(None, 16.0, 5.6e-4), (0, 28.0, 3.6e-4), (1, 32.0, 3.6e-4), (2, 4.0, 5.6e-4)])
def test_pure_constituents(k, mass, alpha):
    a = [0.0] * 6
    if k is not None:
        a[2 * k] = 1.0                       # chi_s = 1 (b = 0)
    C = _coeffs(a, [0.0] * 6)
    x = np.array([[3.0], [4.0], [12.0]])
    m, cv, gcv, kfac, chi = CM.mixture(x, C)
    assert m[0] == pytest.approx(mass / 16.0) and cv[0] == pytest.approx(16.0 / mass)
    assert kfac[0] == pytest.approx(alpha / 5.6e-4)
    assert np.all(gcv == 0) and chi.sum(0)[0] == pytest.approx(1.0)


def test_mixture_mass_and_derivatives():
    d = W.shell_desc(n=2, nr=3, p=2, composition=True)
    C = P.Coeffs(d)
    rng = np.random.default_rng(3)
    x = rng.normal(size=(3, 20))
    r = rng.uniform(d.r_inner, d.r_outer, 20)
    x = x / np.sqrt((x ** 2).sum(0)) * r
    m, cv, gcv, kfac, chi = CM.mixture(x, C)
    assert np.allclose(chi.sum(0), 1.0, atol=1e-14) and np.all(chi > -1e-15)
    # m = rho / sum_s (rho_s / m_s): number density of a unit mass of gas
    rho_s = chi * 1.0
    n_tot = sum(rho_s[s] / (CM.M_REL[s] * 16 * AMU) for s in range(4))
    assert np.allclose(m * 16 * AMU, 1.0 / n_tot, rtol=1e-13)
    # grad c_v against central differences of c_v along each axis
    h = 1e-4
    for dd in range(3):
        e = np.zeros_like(x)
        e[dd] = h
        fd = (CM.mixture(x + e, C)[1] - CM.mixture(x - e, C)[1]) / (2 * h)
        assert np.allclose(gcv[dd], fd, rtol=1e-6, atol=1e-12)


def test_transport_against_si_laws():
    """The nondimensional coefficients against the paper's SI laws divided by the references
    (mu0 = 6.5e-4 sqrt(T0 m_O/k), kappa0 = alpha_O T0^0.69, nu_0 = mu0/rho0, alpha_0 = kappa0/(rho0 c_p0))."""
    ref = W.shell_reference()
    C = _coeffs([0.3, 0.0, 0.1, 0.0, 0.05, 0.0], [0.0] * 6, nu=200.0, al=10.0)
    x = np.array([[1.0], [0.0], [0.0]])
    m, cv, _, kfac, chi = CM.mixture(x, C)
    T_si, rho_si = 640.0, 3.0e-9
    m_si = m[0] * ref.m_O
    mu_si = 6.5e-4 * math.sqrt(T_si * m_si / K_B) + rho_si * 200.0 * ref.mu0 / ref.rho0
    n = [chi[s, 0] / (CM.M_REL[s] * ref.m_O) for s in range(4)]
    alpha = [5.6e-4, 3.6e-4, 3.6e-4, 5.6e-4]
    kappa_m = sum(n[s] * alpha[s] for s in range(4)) / sum(n) * T_si ** 0.69
    cp_si = 2.5 * K_B / m_si                     # gamma/(gamma-1) k/m with gamma = 5/3
    cp0 = 2.5 * K_B / ref.m_O
    kappa_si = kappa_m + rho_si * cp_si * 10.0 * ref.kappa0 / (ref.rho0 * cp0)
    mu, kappa = CM.transport(np.array([T_si / ref.T0]), np.array([math.log(rho_si / ref.rho0)]), m, kfac, C)
    assert mu[0] == pytest.approx(mu_si / ref.mu0, rel=1e-12)
    assert kappa[0] == pytest.approx(kappa_si / ref.kappa0, rel=1e-12)


def test_multi_species_euvac_reduces_to_oxygen():
    """With pure-oxygen fits the four-absorber heating is the single-constituent one."""
    d1 = W.shell_desc(n=2, nr=3, p=1, euvac=True, day=172.0)
    d2 = W.shell_desc(n=2, nr=3, p=1, euvac=True, day=172.0)
    d2.comp = 1                               # a = b = 0: chi_O = 1
    C1, C2 = P.Coeffs(d1), P.Coeffs(d2)
    x = np.array([[592.5, -300.0, 20.0], [120.0, 610.0, -400.0], [-600.0, 50.0, 10.0]]).T
    u = np.zeros((5, 3))
    u[0] = [-1.0, -3.0, -6.0]
    u[4] = np.exp(0.5 * u[0]) * np.array([1.5, 3.0, 4.5])
    q1, q2 = E.heating(u, x, 0.3, C1), E.heating(u, x, 0.3, C2)
    assert np.allclose(q1, q2, rtol=1e-13, atol=0) and q1.max() > 0     # two points are in the shadow


def test_multi_species_column_absorption():
    """Overhead Sun over an isothermal column of fixed composition: the height integral of the
    heating is eps sum_j I0_j E_j (1 - exp(-tau_j)) with tau_j summed over the species, to the
    Chapman factor's first-order accuracy."""
    T, g, R0 = 700.0, 9.0, 6471.0e3
    frac = np.array([0.6, 0.3, 0.05, 0.05])                    # O, N2, O2, He mass fractions
    m = 1.0 / sum(frac[s] / (CM.M_REL[s] * 16 * AMU) for s in range(4))
    H = K_B * T / (m * g)
    z = np.linspace(0.0, 40 * H, 200001)
    rho = 2e-9 * np.exp(-z / H)
    n_s = [rho * frac[s] / (CM.M_REL[s] * 16 * AMU) for s in range(4)]
    phi_s = [E.bins(s)[3] for s in CM.SPECIES]
    I0 = E.solar_flux(150.0, 150.0)
    from scipy import integrate
    q = E.heating_absorbers(n_s, phi_s, T * np.ones_like(z), R0 + z, np.ones_like(z), R0, m, g * np.ones_like(z),
                            0.25, I0)
    total = integrate.trapezoid(q, z)
    lam = E.bins()[0]
    col = sum(n[0] * ph for n, ph in zip(n_s, phi_s)) * H
    expect = 0.25 * np.sum(I0 * 6.62607015e-34 * 299792458.0 / lam * (1 - np.exp(-col)))
    # the overhead Chapman factor is 1 - 1/r~ to first order, r~ = R0/H ~ 160 here
    assert abs(total - expect) <= 1.2 * H / R0 * expect
