"""EUV heating from the EUVAC flux model and Chapman optical depths, Sec. 2.2 (oracle; test
infrastructure only).

Discrete form of Eq. EUVcontinuous for the single constituent of the constant-composition model
(atomic oxygen, number density n = rho / m):

    q_euv = eps * n * sum_j phi_j I_0^j exp(-tau_j) h c / lambda_j,
    I_0^j = F_74113^j max{0.8, 1 + A_j (F10.7bar - 80)} / d^2,    F10.7bar = (F10.7 + F10.7_81) / 2,
    tau_j = n phi_j H Ch(r~, chi),   H = k_B T / (m g),   r~ = |r| / H,   y = sqrt(r~/2) |cos chi|,

with the Smith & Smith form of the Chapman factor for an isothermal exponential atmosphere,

    Ch = sqrt(pi r~ / 2) exp(y^2) erfc(y)                               cos chi > 0,
    Ch = sqrt(pi r~ / 2) [2 exp(r~ (1 - |sin chi|)) - exp(y^2) erfc(y)] cos chi <= 0, |sin chi| > R0/|r|,
    shadow (exp(-tau) = 0)                                              otherwise,

and the zenith angle from the solar declination delta, latitude theta and local time
phi~ = mod_2pi(phi_0 + omega t): cos chi = sin(delta) sin(theta) + cos(delta) cos(theta) cos(phi~ - pi),
delta = arcsin(sin(-delta_0) cos(2 pi/365.24 (N_d + 9) + 2 e sin(2 pi/365.24 (N_d - 3)))),
delta_0 = 23.44 deg, e = 0.0167.

Readings of the paper taken here: the flux column of the appendix table is printed as "x 10^-13
(m^-2 s^-1)"; photon fluxes of 10^13 m^-2 s^-1 are meant (EUVAC fluxes are 10^9 cm^-2 s^-1). The
photon energy of a wavelength band is taken at its centre, of a line at the line. Only the oxygen
cross sections enter (the model's single constituent); the exp(y^2) erfc(y) products are evaluated
as the scaled function erfcx(y). d = 1 (one astronomical unit) unless given.

The table is the paper's appendix table (Table EUVcrosssections), transcribed here.

Pinned by tests/test_oracle_euvac.py: the table against tests/golden/euvac_table.txt; the Chapman
factor against numerical quadrature of the column along the ray, its vertical limit and its
continuity at the terminator; the zenith-angle formula against the rotating-frame direction of the
Sun; the declination at the solstices and equinoxes; the flux clamp.
"""
import math

import numpy as np
from scipy import special as _sp

H_PLANCK = 6.62607015e-34     # J s
C_LIGHT = 299792458.0         # m / s
DELTA_0 = math.radians(23.44)
ECC = 0.0167

# wavelength band [A] (lo, hi; lo == hi for a line), F_74113 [1e13 m^-2 s^-1], A, and the cross
# sections [1e-22 m^2] of N2, O2, O, He
TABLE = [
    (50, 100, 1.200, 0.0100, 0.72, 1.316, 0.73, 0.144),
    (100, 150, 0.450, 0.0071, 2.261, 3.806, 1.839, 0.479),
    (150, 200, 4.800, 0.0134, 4.958, 7.509, 3.732, 1.157),
    (200, 250, 3.100, 0.0195, 8.392, 10.9, 5.202, 1.601),
    (256.3, 256.3, 0.460, 0.0028, 10.21, 13.37, 6.05, 2.121),
    (284.15, 284.15, 0.210, 0.1380, 10.9, 15.79, 7.08, 2.595),
    (250, 300, 1.679, 0.0265, 10.493, 14.387, 6.461, 2.321),
    (303.31, 303.31, 0.800, 0.0250, 11.67, 16.8, 7.68, 2.953),
    (303.78, 303.78, 6.900, 0.0033, 11.7, 16.81, 7.7, 2.962),
    (300, 350, 0.965, 0.0225, 13.857, 17.438, 8.693, 3.544),
    (368.07, 368.07, 0.650, 0.0066, 16.91, 18.32, 9.84, 4.268),
    (350, 400, 0.314, 0.0365, 16.395, 18.118, 9.687, 4.142),
    (400, 450, 0.383, 0.0074, 21.675, 20.31, 11.496, 5.447),
    (465.22, 465.22, 0.290, 0.0075, 23.16, 21.91, 11.93, 6.563),
    (450, 500, 0.285, 0.0202, 23.471, 23.101, 12.127, 7.208),
    (500, 550, 0.452, 0.0088, 24.501, 24.606, 12.059, 0.958),
    (554.37, 554.37, 0.720, 0.0033, 24.13, 26.04, 12.59, 0.0),
    (584.33, 584.33, 1.270, 0.0052, 22.4, 22.72, 13.09, 0.0),
    (550, 600, 0.357, 0.0037, 22.787, 26.61, 13.024, 0.0),
    (609.76, 609.76, 0.530, 0.0162, 22.79, 28.07, 13.4, 0.0),
    (629.73, 629.73, 1.590, 0.0033, 23.37, 32.06, 13.4, 0.0),
    (600, 650, 0.342, 0.0118, 23.339, 26.017, 13.365, 0.0),
    (650, 700, 0.230, 0.0043, 31.755, 21.919, 17.245, 0.0),
    (703.31, 703.31, 0.360, 0.0030, 26.54, 27.44, 11.46, 0.0),
    (700, 750, 0.141, 0.0047, 24.662, 28.535, 10.736, 0.0),
    (765.15, 765.15, 0.170, 0.0039, 120.49, 20.8, 4, 0.0),
    (770.41, 770.41, 0.260, 0.0128, 14.18, 18.91, 3.89, 0.0),
    (789.36, 789.36, 0.702, 0.0033, 16.487, 26.668, 3.749, 0.0),
    (750, 800, 0.758, 0.0048, 33.578, 22.145, 5.091, 0.0),
    (800, 850, 1.625, 0.0048, 16.992, 16.631, 3.498, 0.0),
    (850, 900, 3.537, 0.0057, 20.249, 8.562, 4.554, 0.0),
    (900, 950, 3.000, 0.0050, 9.68, 12.817, 1.315, 0.0),
    (977.02, 977.02, 4.400, 0.0039, 2.24, 18.73, 0.0, 0.0),
    (950, 1000, 1.475, 0.0044, 50.988, 21.108, 0.0, 0.0),
    (1025.72, 1025.72, 3.500, 0.0052, 0.0, 1.63, 0.0, 0.0),
    (1031.91, 1031.91, 2.100, 0.0053, 0.0, 1.05, 0.0, 0.0),
    (1000, 1050, 2.467, 0.0044, 0.0, 1.346, 0.0, 0.0),
]
SPECIES_COLUMNS = {"N2": 4, "O2": 5, "O": 6, "He": 7}


def bins(species="O"):
    """Arrays lambda [m] (band centre or line), F_74113 [m^-2 s^-1], A, phi_species [m^2]."""
    t = np.array(TABLE, dtype=float)
    lam = 0.5 * (t[:, 0] + t[:, 1]) * 1e-10
    return lam, t[:, 2] * 1e13, t[:, 3], t[:, SPECIES_COLUMNS[species]] * 1e-22


def solar_flux(f107, f107a, d=1.0):
    """I_0^j [m^-2 s^-1] of the EUVAC model."""
    _, F, A, _ = bins()
    fbar = 0.5 * (f107 + f107a)
    return F * np.maximum(0.8, 1.0 + A * (fbar - 80.0)) / d ** 2


def declination(day):
    """Solar declination [rad] on day of year N_d (1 = January 1st)."""
    w = 2.0 * math.pi / 365.24
    return math.asin(math.sin(-DELTA_0) * math.cos(w * (day + 9.0) + 2.0 * ECC * math.sin(w * (day - 3.0))))


def cos_zenith_latlon(lat, lon, t_phys, omega, delta):
    """cos chi from latitude, longitude [rad] and time [s], the paper's formula."""
    phit = np.mod(lon + omega * t_phys, 2.0 * math.pi)
    return math.sin(delta) * np.sin(lat) + math.cos(delta) * np.cos(lat) * np.cos(phit - math.pi)


def sun_direction(day, wt):
    """Unit vector to the Sun in the rotating frame after rotation angle wt = omega t: the point
    with cos(chi) = 1 is at latitude delta and local time pi (local noon)."""
    delta = declination(day)
    return (-math.cos(delta) * math.cos(wt), math.cos(delta) * math.sin(wt), math.sin(delta))


def chapman(rt, cchi, r_over_R0):
    """Chapman factor Ch(r~, chi); np.inf in the Earth's shadow. Elementwise over arrays."""
    rt, cchi = np.broadcast_arrays(np.asarray(rt), np.asarray(cchi))
    schi = np.sqrt(np.maximum(0.0, 1.0 - np.real(cchi) ** 2))
    y = np.sqrt(rt / 2.0) * np.abs(cchi)
    base = np.sqrt(np.pi * rt / 2.0)
    ex = _sp.erfcx(y)
    day = base * ex
    night = base * (2.0 * np.exp(np.where(np.real(cchi) > 0.0, 0.0, rt * (1.0 - schi))) - ex)
    lit_night = schi > 1.0 / np.asarray(r_over_R0)
    return np.where(np.real(cchi) > 0.0, day, np.where(lit_night, night, np.inf))


def heating_dimensional(rho, T, r, cchi, R0, m, g, eps, I0):
    """q_euv [W/m^3] at density rho [kg/m^3], temperature T [K], radius r [m], molecular mass m [kg],
    local gravity g [m/s^2]; R0 [m] is the radius of the lower boundary (the shadow test)."""
    lam, _, _, phi = bins()
    n = rho / m
    H = 1.380649e-23 * T / (m * g)
    ch = chapman(r / H, cchi, r / R0)
    q = 0.0
    for j in range(len(lam)):
        if phi[j] == 0.0:
            continue
        lit = np.isfinite(np.real(ch))
        tau = np.where(lit, n * phi[j] * H * np.where(lit, ch, 0.0), 0.0)
        q = q + np.where(lit, eps * n * phi[j] * I0[j] * np.exp(-tau) * H_PLANCK * C_LIGHT / lam[j], 0.0)
    return q


def heating_absorbers(n_s, phi_s, T, r, cchi, R0, m, g, eps, I0):
    """q_euv [W/m^3] for several absorbers: number densities n_s and cross-section arrays phi_s (per
    species, per band); every band is attenuated by the optical depth summed over the species."""
    lam = bins()[0]
    H = 1.380649e-23 * T / (m * g)
    ch = chapman(r / H, cchi, r / R0)
    lit = np.isfinite(np.real(ch))
    chl = np.where(lit, ch, 0.0)
    q = 0.0
    for j in range(len(lam)):
        absorb = sum(n * ph[j] for n, ph in zip(n_s, phi_s))
        if np.all(np.asarray(absorb) == 0):
            continue
        tau = absorb * H * chl
        q = q + np.where(lit, eps * absorb * I0[j] * np.exp(-tau) * H_PLANCK * C_LIGHT / lam[j], 0.0)
    return q


def heating(u, x, t, C):
    """Nondimensional EUVAC heating Q* (multiplied by e^{-varrho/2}/c_v in the energy source), in
    the scaling of the Gaussian heating, q* = q H0 / (rho0 c_v0 T0 a0), with H0 = k_B T0/(m g0),
    a0 = sqrt(gamma k_B T0/m), c_v0 = k_B/((gamma - 1) m) from the reference values."""
    kB = 1.380649e-23
    T0, rho0, m0, g0 = C.ref_T0, C.ref_rho0, C.ref_m, C.ref_g0
    H0 = kB * T0 / (m0 * g0)
    a0 = math.sqrt(C.gamma * kB * T0 / m0)
    cv0 = kB / ((C.gamma - 1.0) * m0)
    rho = rho0 * np.exp(u[0])
    T = T0 * u[4] * np.exp(-0.5 * u[0])
    r = np.sqrt(x[0] ** 2 + x[1] ** 2 + x[2] ** 2)
    g = g0 * (C.g_r0 / r) ** 2
    s = sun_direction(C.euv_day, C.euv_omega_t * t)
    cchi = np.clip((x[0] * s[0] + x[1] * s[1] + x[2] * s[2]) / r, -1.0, 1.0)
    I0 = solar_flux(C.euv_f107, C.euv_f107a, C.euv_dsun)
    if getattr(C, "comp", 0):
        from . import composition as CM
        mstar, _, _, _, chi = CM.mixture(x, C)
        n_s = [rho * chi[k] / (m0 * CM.M_REL[k]) for k in range(4)]
        phi_s = [bins(s)[3] for s in CM.SPECIES]
        q = heating_absorbers(n_s, phi_s, T, r * H0, cchi, C.g_r0 * H0, m0 * mstar, g, C.euv_eff, I0)
    else:
        q = heating_dimensional(rho, T, r * H0, cchi, C.g_r0 * H0, m0 * C.m, g, C.euv_eff, I0)
    return q * H0 / (rho0 * cv0 * T0 * a0)
