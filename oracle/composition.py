"""Chemically frozen variable composition and molecular + eddy transport, Sec. 2.1.1-2.1.2 (oracle;
test infrastructure only).

Species O, N2, O2 and He. The mass fractions of N2, O2 and He follow the paper's two-term fits in
the radius, chi_s = sum_{j=1,2} a_j^s exp(b_j^s |r|) (|r| nondimensional here), and chi_O = 1 - the
others. The mixture's molecular mass is m = [sum_s chi_s / m_s]^-1, so in the nondimensional
variables (masses in units of m_O) c_v* = 1/m* = sum_s chi_s / m_s*, with gamma fixed. Transport:

    mu_m = 6.5e-4 sqrt(T m / k)                       ->  mu_m*    = sqrt(T* m*),
    kappa_m = sum_s x_s alpha_s T^0.69                ->  kappa_m* = (sum_s x_s alpha_s / alpha_O) T*^0.69,
    mu = mu_m + rho nu_eddy, kappa = kappa_m + rho c_p alpha_eddy
                                                      ->  mu* = mu_m* + nu_e rho*,
                                                          kappa* = kappa_m* + alpha_e rho* / m*,

x_s = (chi_s/m_s) / sum_k (chi_k/m_k) the number fractions, alpha_N2 = alpha_O2 = 3.6e-4,
alpha_O = alpha_He = 5.6e-4, nu_e = nu_eddy/nu_0 = 200 and alpha_e = alpha_eddy/alpha_0 = 10
(nu_0, alpha_0 the reference molecular values, and c_p* = 1/m*). The energy equation gains
-(1/c_v)(sqrt(rho) T v - c_kappa kappa/(sqrt(rho) c_v) grad T) . grad c_v, with grad c_v from the
fits' radial derivative.

Readings of the paper taken here: the fit coefficients are inputs (the paper fits them to MSIS, which
is not available; the workloads carry synthetic ones); gamma stays 5/3; in this mode the paper's
transport laws replace the T^visc_exp law; the EUVAC optical depth of a band sums over the species
(photons are absorbed by every constituent).

Pinned by tests/test_oracle_composition.py: the mass fractions sum to one, the mixture mass of pure
constituents, c_v's radial derivative against central differences, the transport coefficients'
closed forms, the residual's reduction to the constant-composition one when the fits give pure
oxygen, and the extra energy source against the divergence it comes from.
"""
import numpy as np

SPECIES = ("O", "N2", "O2", "He")
M_REL = np.array([1.0, 28.0 / 16.0, 32.0 / 16.0, 4.0 / 16.0])   # m_s / m_O
ALPHA_REL = np.array([1.0, 3.6 / 5.6, 3.6 / 5.6, 1.0])          # alpha_s / alpha_O


def fractions(r, a, b):
    """Mass fractions (4, ...) at nondimensional radius r; a, b are (3, 2) for N2, O2, He."""
    r = np.asarray(r)
    others = [sum(a[s][j] * np.exp(b[s][j] * r) for j in range(2)) for s in range(3)]
    return np.stack([1.0 - others[0] - others[1] - others[2]] + others)


def dfractions(r, a, b):
    """d chi_s / d r (4, ...)."""
    r = np.asarray(r)
    others = [sum(a[s][j] * b[s][j] * np.exp(b[s][j] * r) for j in range(2)) for s in range(3)]
    return np.stack([-(others[0] + others[1] + others[2])] + others)


def mixture(x, C):
    """m*, c_v*, grad c_v* (3, ...), kappa factor sum_s x_s alpha_s/alpha_O, mass fractions (4, ...) at
    positions x (3, ...)."""
    r = np.sqrt(x[0] ** 2 + x[1] ** 2 + x[2] ** 2)
    chi = fractions(r, C.comp_a, C.comp_b)
    shape = (4,) + (1,) * (chi.ndim - 1)
    cv = (chi / M_REL.reshape(shape)).sum(0)
    m = 1.0 / cv
    xs = chi / M_REL.reshape(shape) / cv
    kfac = (xs * ALPHA_REL.reshape(shape)).sum(0)
    dcv = (dfractions(r, C.comp_a, C.comp_b) / M_REL.reshape(shape)).sum(0)
    gcv = np.stack([dcv * x[d] / r for d in range(3)])
    return m, cv, gcv, kfac, chi


def transport(T, u0, m, kfac, C):
    """mu*, kappa* with the molecular laws of Sec. 2.1.2 and the eddy offsets."""
    rho = np.exp(u0)
    mu = np.sqrt(T * m) + C.eddy_nu * rho
    kappa = kfac * T ** 0.69 + C.eddy_alpha * rho / m
    return mu, kappa
