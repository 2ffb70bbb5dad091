"""Pins of the arithmetic that the shared input module performs for both sides.

The input module states which problem is solved: the reference scales and nondimensional numbers of
Sec. 2.4 (Eq. nondimensional), the hydrostatic Bates base state of the shell workloads, the Sec. 3.3
cubed-sphere map with geometric radial layers, the variables of Sec. 2.3, and the seeded random
numbers. Both the oracle and the library read its output, so parity cannot see a mistake in it;
these tests pin each piece to something other than its own formula:

  * reference scales: the values the definitions give by hand (H0 = 10.93 km, a0 = 416.2 m/s,
    t0 = 26.26 s, Fr = 2.47e-3, Re = 5640, Pr = 24.2), and identities that follow from the
    definitions by algebra, not by restating them (a0^2 = gamma g0 H0, Re^2 = gamma Gr,
    Fr^2 = gamma (Omega t0)^2, Pr kappa0 / mu0 = the textbook c_p of a monatomic gas, 5 k_B / (2 m));
  * hydrostatic state: a closed form (isothermal column under inverse-square gravity) and an
    independent adaptive Runge-Kutta integration of d ln p / dr = -m g / (k_B T);
  * cubed sphere: node radii from the geometric layers, equal angles between the node directions
    of an equiangular panel, panel corners on the cube diagonals;
  * SplitMix64: the published output sequence of the reference generator.

Each pin is also shown to fail on a planted mistake (a dropped or wrong factor).
"""
import math

import numpy as np
import pytest
from scipy.integrate import solve_ivp

from paper_2306_01085_gb300 import workloads as W


# ----------------------------------------------------------------------------------------------
# reference scales (Sec. 2.4)
# ----------------------------------------------------------------------------------------------
def check_reference(ref, rtol=6e-4):
    """Hand values of the definitions at T0 = 200 K, m_O = 16 amu, g0 = 9.81 (6371/6471)^2 = 9.509 m/s^2,
    rho0 = 5e-7 kg/m^3, mu0 = 6.5e-4 sqrt(T0 m_O / k_B), kappa0 = 5.6e-4 T0^0.69."""
    problems = []
    for name, want in (("H0", 10.93e3), ("a0", 416.2), ("t0", 26.26), ("Fr", 2.472e-3), ("Re", 5640.0),
                       ("Pr", 24.17), ("g0", 9.509)):
        got = getattr(ref, name)
        if abs(got - want) > rtol * abs(want):
            problems.append(f"{name} = {got} (hand value {want})")
    gamma = W.GAMMA
    # a0^2 = gamma k T0 / m and H0 = k T0 / (m g0) give a0^2 = gamma g0 H0
    if abs(ref.a0 ** 2 - gamma * ref.g0 * ref.H0) > 1e-12 * ref.a0 ** 2:
        problems.append("a0^2 != gamma g0 H0")
    # Gr = g0 H0^3 rho0^2 / mu0^2 and Re = rho0 a0 H0 / mu0 give Re^2 = gamma Gr
    if abs(ref.Re ** 2 - gamma * ref.Gr) > 1e-12 * ref.Re ** 2:
        problems.append("Re^2 != gamma Gr")
    # Fr^2 = Omega^2 H0 / g0 = gamma (Omega t0)^2 with t0 = H0 / a0
    if abs(ref.Fr ** 2 - gamma * (W.OMEGA_EARTH * ref.t0) ** 2) > 1e-12 * ref.Fr ** 2:
        problems.append("Fr^2 != gamma (Omega t0)^2")
    # Pr = mu0 c_p / kappa0 with c_p of a monatomic gas = 5 k_B / (2 m) = 1299 J/(kg K) for O
    cp_mono = 2.5 * 1.380649e-23 / (16 * 1.66053906660e-27)
    if abs(ref.Pr * ref.kappa0 / ref.mu0 - cp_mono) > 1e-12 * cp_mono:
        problems.append("Pr kappa0 / mu0 != 5 k_B / (2 m_O)")
    if abs(cp_mono - 1299.0) > 0.5:
        problems.append("monatomic c_p")
    return problems


def test_reference_scales():
    assert check_reference(W.shell_reference()) == []


def test_reference_pins_catch_planted_mistakes():
    ref = W.shell_reference()
    planted = {
        "Gr with H0^2": dict(Gr=ref.Gr / ref.H0),
        "Fr without the square root": dict(Fr=ref.Fr ** 2),
        "H0 with m of O2": dict(H0=ref.H0 / 2.0, t0=ref.t0 / 2.0),
        "a0 without gamma": dict(a0=ref.a0 / math.sqrt(W.GAMMA)),
        "Pr with c_v": dict(Pr=ref.Pr / W.GAMMA),
        "g0 at the surface": dict(g0=9.81),
    }
    for name, change in planted.items():
        bad = W.Reference(**{**ref.__dict__, **change})
        assert check_reference(bad), name


def test_nondimensional_heating_scale():
    """The EUV shells' peak heating 1e-8 W/m^3 over the energy scale rho0 c_v0 T0 a0 / H0
    (= 2.968e-3 W/m^3 by hand) is 3.37e-6."""
    ref = W.shell_reference()
    d = W.shell_desc(n=2, nr=2, p=1, euv=True, ref=ref)
    assert abs(d.euv_amp - 1e-8 / 2.968e-3) < 2e-3 * d.euv_amp
    assert abs(d.euv_r_peak * ref.H0 - (W.R_EARTH + 300e3)) < 1e-6
    assert abs(d.euv_width * ref.H0 - 50e3) < 1e-6


# ----------------------------------------------------------------------------------------------
# hydrostatic base state
# ----------------------------------------------------------------------------------------------
R0 = W.R_EARTH + 100e3


def _ode_density(r_out, ref, temperature, gravity):
    """ln p by an adaptive 8th-order Runge-Kutta integration of d ln p/dr = -m g/(k_B T)."""
    m = ref.m_O

    def rhs(r, y):
        return [-m * gravity(r) / (W.K_B * temperature((r - W.R_EARTH) / 1e3))]

    sol = solve_ivp(rhs, (R0, float(r_out.max())), [0.0], method="DOP853", rtol=1e-13, atol=1e-14,
                    dense_output=True)
    lnp = sol.sol(r_out)[0]
    p0 = ref.rho0 * W.K_B * ref.T0 / m
    T = temperature((r_out - W.R_EARTH) / 1e3)
    return p0 * np.exp(lnp) * m / (W.K_B * T)


def bates_t(z_km):
    return 1000.0 - 800.0 * np.exp(-0.02 * (z_km - 100.0))


def inverse_square(r):
    return 9.81 * (W.R_EARTH / r) ** 2


RADII = R0 + np.array([0.0, 1.3e3, 2.5e3, 10e3, 47e3, 100e3, 250e3, 400e3, 500e3])


def test_bates_profile_values():
    assert abs(W.bates_temperature(100.0) - 200.0) < 1e-12
    assert abs(W.bates_temperature(600.0) - (1000.0 - 800.0 * math.exp(-10.0))) < 1e-9
    assert abs(W.bates_temperature(1e4) - 1000.0) < 1e-9


def test_hydrostatic_matches_independent_integration():
    ref = W.shell_reference()
    rho, T = W.bates_hydrostatic(RADII, ref)
    want = _ode_density(RADII, ref, bates_t, inverse_square)
    assert np.all(np.abs(rho / want - 1.0) < 1e-9)
    assert np.allclose(T, bates_t((RADII - W.R_EARTH) / 1e3), rtol=1e-14)
    assert abs(rho[0] - 5e-7) < 1e-20
    # rho(600 km) = 4.77e-12 kg/m^3 (the value the configuration's base state gives)
    assert abs(rho[-1] - 4.770e-12) < 2e-3 * 4.77e-12


def test_hydrostatic_isothermal_closed_form():
    """Constant T under g = g_s (R_E/r)^2: ln(p/p0) = -(m g_s R_E^2 / (k_B T)) (1/R0 - 1/r)."""
    ref = W.shell_reference()
    Tc = 640.0
    rho, _ = W.bates_hydrostatic(RADII, ref, temperature=lambda z: np.full_like(np.asarray(z, float), Tc))
    m = ref.m_O
    lnp = -(m * 9.81 * W.R_EARTH ** 2 / (W.K_B * Tc)) * (1.0 / R0 - 1.0 / RADII)
    want = ref.rho0 * ref.T0 / Tc * np.exp(lnp)
    assert np.all(np.abs(rho / want - 1.0) < 1e-12)


def test_hydrostatic_pins_catch_planted_mistakes():
    ref = W.shell_reference()
    want = _ode_density(RADII, ref, bates_t, inverse_square)
    planted = {
        "gravity without (R_E/r)^2": dict(gravity=lambda r: np.full_like(np.asarray(r, float), 9.81)),
        "temperature with a wrong decay rate": dict(temperature=lambda z: 1000.0 - 800.0 * np.exp(-0.021 * (z - 100.0))),
        "mass of O2": dict(),
    }
    for name, kw in planted.items():
        r2 = ref if name != "mass of O2" else W.Reference(**{**ref.__dict__, "m_O": 2 * ref.m_O})
        rho, _ = W.bates_hydrostatic(RADII, r2, **kw)
        assert np.max(np.abs(rho / want - 1.0)) > 1e-3, name


# ----------------------------------------------------------------------------------------------
# cubed-sphere map (Sec. 3.3)
# ----------------------------------------------------------------------------------------------
def check_shell_nodes(desc, X, tol=1e-12):
    """Node radii follow the layers (linear in the radial reference coordinate between interfaces
    r_k = r_in + h sum_{j<k} q^j, q the geometric ratio); on every panel the angles of the node
    directions about the panel's two axes step uniformly (equiangular map); panel corners lie on
    the cube diagonals."""
    problems = []
    n = desc.p + 1
    xi = W.gll_points(n)
    s = 0.5 * (1.0 + xi)
    q = solve_ratio(desc)
    rl = desc.r_inner + np.concatenate([[0.0], np.cumsum(desc.h_first * q ** np.arange(desc.nz))])
    nn, nz = desc.nx, desc.nz
    idx = np.arange(n ** 3)
    ia, ib, ic = idx % n, (idx // n) % n, idx // (n * n)
    rad = np.sqrt((X ** 2).sum(1))
    d_ang = 0.5 * math.pi / nn
    for P, (c, a, b) in enumerate(W.PANELS):
        c, a, b = np.array(c, float), np.array(a, float), np.array(b, float)
        for j in range(nn):
            for i in range(nn):
                for k in range(nz):
                    e = k + nz * (i + nn * (j + nn * P))
                    want_r = rl[k] + s[ic] * (rl[k + 1] - rl[k])
                    if np.max(np.abs(rad[e] - want_r)) > tol * rl[-1]:
                        problems.append(f"radius e={e}")
                    xc, xa, xb = X[e].T @ c, X[e].T @ a, X[e].T @ b
                    alpha = np.arctan2(xa, xc)
                    beta = np.arctan2(xb, xc)
                    if np.max(np.abs(alpha - (-0.25 * math.pi + (i + s[ia]) * d_ang))) > tol:
                        problems.append(f"alpha e={e}")
                    if np.max(np.abs(beta - (-0.25 * math.pi + (j + s[ib]) * d_ang))) > tol:
                        problems.append(f"beta e={e}")
    corners = X[:, :, [0, n - 1, n * (n - 1), n * n - 1]]          # inner-face corners
    cdir = corners / np.sqrt((corners ** 2).sum(1, keepdims=True))
    on_diag = np.abs(np.abs(cdir) - 1 / math.sqrt(3)).max(1) < 1e-12
    n_diag = int(on_diag.sum())
    if n_diag != 6 * 4 * nz:           # each panel has 4 corner cells x nz layers touching a cube corner
        problems.append(f"{n_diag} corner nodes on cube diagonals")
    return problems


def solve_ratio(desc):
    """Geometric ratio q with h_first (q^nz - 1)/(q - 1) = r_out - r_in, by Newton on the closed sum."""
    L, h, n = desc.r_outer - desc.r_inner, desc.h_first, desc.nz
    q = 1.5
    for _ in range(100):
        f = h * (q ** n - 1) / (q - 1) - L
        df = h * (n * q ** (n - 1) * (q - 1) - (q ** n - 1)) / (q - 1) ** 2
        q -= f / df
    return q


@pytest.mark.parametrize("n,nr,p", [(2, 3, 2), (3, 2, 3)])
def test_cubed_sphere_nodes(n, nr, p):
    desc = W.shell_desc(n=n, nr=nr, p=p)
    assert check_shell_nodes(desc, W.mesh_nodes(desc)) == []


def test_cubed_sphere_pins_catch_planted_mistakes():
    desc = W.shell_desc(n=2, nr=2, p=2)
    X = W.mesh_nodes(desc)
    # equidistant gnomonic map (tan uniform instead of the angle) on panel 0
    bad = X.copy()
    n = desc.p + 1
    s = 0.5 * (1.0 + W.gll_points(n))
    idx = np.arange(n ** 3)
    ia, ib = idx % n, (idx // n) % n
    for j in range(2):
        for i in range(2):
            for k in range(2):
                e = k + 2 * (i + 2 * j)
                ta = -1.0 + (i + s[ia]) * 1.0
                tb = -1.0 + (j + s[ib]) * 1.0
                dirv = np.stack([np.ones_like(ta), ta, tb])
                dirv /= np.sqrt((dirv ** 2).sum(0))
                bad[e] = dirv * np.sqrt((X[e] ** 2).sum(0))
    assert check_shell_nodes(desc, bad)
    # uniform instead of geometric layers
    d_uni = W.shell_desc(n=2, nr=2, p=2)
    d_uni.h_first = 0.0
    assert check_shell_nodes(desc, W.mesh_nodes(d_uni))


def test_gll_points_closed_forms():
    assert np.allclose(W.gll_points(3), [-1.0, 0.0, 1.0], atol=1e-15)
    assert np.allclose(W.gll_points(4), [-1.0, -1 / math.sqrt(5), 1 / math.sqrt(5), 1.0], atol=1e-15)
    assert np.allclose(W.gll_points(5), [-1.0, -math.sqrt(3 / 7), 0.0, math.sqrt(3 / 7), 1.0], atol=1e-15)


# ----------------------------------------------------------------------------------------------
# variables (Sec. 2.3) and random numbers
# ----------------------------------------------------------------------------------------------
def test_pack_state_variables():
    rho = np.array([[2.0, 0.25]])
    v = np.array([[[3.0, -1.0]], [[0.5, 2.0]], [[-4.0, 0.0]]])[:, 0][:, None, :]
    T = np.array([[1.5, 0.8]])
    u = W.pack_state(rho, v, T)
    assert np.allclose(u[0, 0], np.log(rho[0]))
    assert np.allclose(u[0, 1:4], np.sqrt(rho[0]) * v[:, 0])
    assert np.allclose(u[0, 4], np.sqrt(rho[0]) * T[0])


def test_isothermal_column_is_the_exact_hydrostatic_state():
    """d p/dz = -rho g with p = rho T / gamma and the nondimensional gravity g/gamma (Eq.
    fluxSWNondimensional with a = g/gamma): log rho = -g z / T."""
    z = np.linspace(0.0, 3.0, 7)
    x = np.zeros((1, 3, 7))
    x[0, 2] = z
    u = W.isothermal_column(x, T=1.7, g=0.9)
    rho = np.exp(u[0, 0])
    dp = np.gradient(rho * 1.7, z, edge_order=2)
    # pressure gradient balances the weight: d(rho T)/dz = -g rho (the gamma cancels)
    assert np.allclose(dp[1:-1], -0.9 * rho[1:-1], rtol=2e-2)
    assert np.allclose(np.log(rho), -0.9 * z / 1.7, atol=1e-15)


def test_splitmix64_reference_sequence():
    """SplitMix64 (Steele, Lea & Flood 2014) from state 1234567: the reference generator's first
    five outputs."""
    got = W.splitmix64(1234567, np.arange(5))
    want = [6457827717110365317, 3203168211198807973, 9817491932198370423, 4593380528125082431,
            16408922859458223821]
    assert [int(x) for x in got] == want
