"""Pointwise flux, source and stabilisation of the nondimensional model (oracle; test infrastructure).

Variables u = (varrho, sqrt(rho) v, sqrt(rho) T) with varrho = log(rho / rho0) (Sec. 2.3); q is the
LDG gradient, q[d, c] ~ d u_c / d x_d. All functions take arrays with trailing point axes:
u (5, ...), q (3, 5, ...), x (3, ...), and work for any numpy dtype (float64, complex128), so the
complex-step derivative of everything built on them is exact to rounding.

Reading of the paper taken here:
  * sqrt(rho) = exp(varrho / 2); v = u_{2:4} exp(-varrho/2); T = u_5 exp(-varrho/2).
  * grad v = exp(-varrho/2) (grad u_m - u_m grad(varrho) / 2), grad T likewise (chain rule on q).
  * Coefficients of Eq. fluxSWNondimensional: c_mu = 1/sqrt(gamma Gr), c_kappa = sqrt(gamma/Gr)/Pr,
    c_diss = (gamma - 1) sqrt(gamma/Gr).
  * c_v = 1/m with constant composition, so the grad(c_v) term of the energy source is zero.
  * The heating term is written Q*/(sqrt(rho) c_v) with Q* = q H0 / (rho0 c_v0 T0 a0), i.e. the
    paper's gamma (gamma - 1)/K factor is absorbed in the nondimensional amplitude.
  * mu* = kappa* = T*^visc_exp (visc_exp = 0: constant coefficients).

Parity pinned by tests/test_oracle_physics.py against the original Navier-Stokes system, Eq. NS1,
written in primitive variables (the reformulation must reproduce its time derivatives).
"""
import math

import numpy as np

from . import composition as _comp
from . import euvac as _euvac


class Coeffs:
    """Nondimensional numbers of one workload (Eq. nondimensional)."""

    def __init__(self, desc):
        g = desc.gamma
        self.gamma = g
        self.c_mu = 1.0 / math.sqrt(g * desc.grashof)
        self.c_kappa = math.sqrt(g / desc.grashof) / desc.prandtl
        self.c_diss = (g - 1.0) * math.sqrt(g / desc.grashof)
        self.m = desc.mass
        self.cv = 1.0 / desc.mass
        self.visc_exp = desc.visc_exp
        self.lam = desc.lambda0
        self.t_wall = desc.t_wall
        self.gravity_kind = desc.gravity_kind
        self.gvec = np.array(desc.gvec, dtype=np.float64)
        self.g_r0 = desc.g_r0
        self.omega = np.array(desc.omega, dtype=np.float64)
        self.Fr = desc.froude
        self.euv = desc.euv
        self.euv_amp = desc.euv_amp
        self.euv_sigma = desc.euv_sigma
        self.euv_r_peak = desc.euv_r_peak
        self.euv_width = desc.euv_width
        self.euv_omega_t = desc.euv_omega_t
        for k in ("euv_day", "euv_f107", "euv_f107a", "euv_eff", "euv_dsun", "ref_T0", "ref_rho0", "ref_m",
                  "ref_g0", "comp", "eddy_nu", "eddy_alpha"):
            setattr(self, k, getattr(desc, k))
        self.comp_a = np.array(desc.comp_a, dtype=np.float64).reshape(3, 2)
        self.comp_b = np.array(desc.comp_b, dtype=np.float64).reshape(3, 2)


def _mixture(x, C):
    """(m, c_v, grad c_v or None, kappa factor, mass fractions or None) at positions x."""
    if C.comp and x is not None:
        return _comp.mixture(x, C)
    return C.m, C.cv, None, 1.0, None


def _transport(T, C, u0=None, mix=None):
    if C.comp:
        return _comp.transport(T, u0, mix[0], mix[3], C)
    if C.visc_exp == 0.0:
        return np.ones_like(T), np.ones_like(T)
    mu = T ** C.visc_exp
    return mu, mu


def primitives(u, q, C):
    """sqrt(rho), 1/sqrt(rho), v, T, grad v [m, d], grad T [d], div v, strain eps [m, d]."""
    sr = np.exp(0.5 * u[0])
    isr = np.exp(-0.5 * u[0])
    v = u[1:4] * isr
    T = u[4] * isr
    gv = np.stack([np.stack([isr * (q[d, 1 + m] - 0.5 * u[1 + m] * q[d, 0]) for d in range(3)])
                   for m in range(3)])
    gT = np.stack([isr * (q[d, 4] - 0.5 * u[4] * q[d, 0]) for d in range(3)])
    div = gv[0, 0] + gv[1, 1] + gv[2, 2]
    eps = np.stack([np.stack([gv[m, d] + gv[d, m] - (2.0 / 3.0) * div * (1.0 if m == d else 0.0)
                              for d in range(3)]) for m in range(3)])
    return sr, isr, v, T, gv, gT, div, eps


def flux(u, q, C, viscous=True, x=None):
    """Physical flux F[c, d] of Eq. fluxSWNondimensional (left-hand divergence terms); x: positions
    (needed with variable composition)."""
    sr, isr, v, T, gv, gT, div, eps = primitives(u, q, C)
    mix = _mixture(x, C)
    mu, kappa = _transport(T, C, u[0], mix)
    p_coef = 1.0 / (C.gamma * mix[0])
    cv = mix[1]
    F = []
    F.append(np.stack([u[0] * v[d] for d in range(3)]))
    for m in range(3):
        row = []
        for d in range(3):
            val = u[1 + m] * v[d] + (p_coef * u[4] if m == d else 0.0 * u[4])
            if viscous:
                val = val - C.c_mu * mu * isr * eps[m, d]
            row.append(val)
        F.append(np.stack(row))
    row = []
    for d in range(3):
        val = u[4] * v[d]
        if viscous:
            val = val - C.c_kappa * kappa * isr / cv * gT[d]
        row.append(val)
    F.append(np.stack(row))
    return np.stack(F)


def acceleration(x, v, C):
    """a = g/gamma - (Fr^2/gamma) omega x (omega x r) - (2 Fr/sqrt(gamma)) omega x v (Sec. 2.4)."""
    if C.gravity_kind == 0:
        g = [C.gvec[d] * np.ones(x.shape[1:]) for d in range(3)]
    else:
        r = np.sqrt(x[0] ** 2 + x[1] ** 2 + x[2] ** 2)
        fac = -(C.g_r0 / r) ** 2 / r
        g = [fac * x[d] for d in range(3)]
    w = C.omega
    wx = np.stack([w[1] * x[2] - w[2] * x[1], w[2] * x[0] - w[0] * x[2], w[0] * x[1] - w[1] * x[0]])
    wwx = np.stack([w[1] * wx[2] - w[2] * wx[1], w[2] * wx[0] - w[0] * wx[2], w[0] * wx[1] - w[1] * wx[0]])
    wv = [w[1] * v[2] - w[2] * v[1], w[2] * v[0] - w[0] * v[2], w[0] * v[1] - w[1] * v[0]]
    return [g[d] / C.gamma - C.Fr ** 2 / C.gamma * wwx[d] - 2.0 * C.Fr / math.sqrt(C.gamma) * wv[d]
            for d in range(3)]


def euv_heating(x, t, C):
    """Nondimensional sub-solar Gaussian heating Q*(x, t) (zero when disabled).

    Q* = A exp(-chi^2 / (2 sigma^2)) exp(-ln 2 ((|r| - r_peak)/w)^2), cos chi = r_hat . s(t),
    s(t) = (cos(omega t), -sin(omega t), 0): the Sun fixed in the inertial frame seen from the
    rotating frame at equinox (declination 0), cf. the zenith-angle formula of Sec. 2.2.
    """
    r = np.sqrt(x[0] ** 2 + x[1] ** 2 + x[2] ** 2)
    if C.euv != 1:
        return np.zeros_like(r)
    sx, sy = math.cos(C.euv_omega_t * t), -math.sin(C.euv_omega_t * t)
    cchi = np.clip((x[0] * sx + x[1] * sy) / r, -1.0, 1.0)
    chi = np.arccos(cchi)
    return (C.euv_amp * np.exp(-chi ** 2 / (2.0 * C.euv_sigma ** 2))
            * np.exp(-math.log(2.0) * ((r - C.euv_r_peak) / C.euv_width) ** 2))


def source(u, q, x, t, C):
    """Source s(u, q) of Eq. fluxSWNondimensional (right-hand side)."""
    sr, isr, v, T, gv, gT, div, eps = primitives(u, q, C)
    mix = _mixture(x, C)
    mu, kappa = _transport(T, C, u[0], mix)
    mm, cv, gcv = mix[0], mix[1], mix[2]
    a = acceleration(x, v, C)
    s = [(u[0] - 1.0) * div]
    for m in range(3):
        eps_grad = eps[m, 0] * q[0, 0] + eps[m, 1] * q[1, 0] + eps[m, 2] * q[2, 0]
        s.append(sr * a[m] + 0.5 * div * u[1 + m] - 0.5 / (C.gamma * mm) * u[4] * q[m, 0]
                 + 0.5 * C.c_mu * mu * isr * eps_grad)
    gT_grad = gT[0] * q[0, 0] + gT[1] * q[1, 0] + gT[2] * q[2, 0]
    diss = sum(eps[m, d] * gv[m, d] for m in range(3) for d in range(3))
    heat = _euvac.heating(u, x, t, C) if C.euv == 2 else euv_heating(x, t, C)
    s4 = (heat * isr / cv
          + (1.5 - C.gamma) * u[4] * div
          + 0.5 * C.c_kappa * kappa * isr / cv * gT_grad
          + C.c_diss * mu * isr / cv * diss)
    if gcv is not None:
        # -(1/c_v) (sqrt(rho) T v - c_kappa kappa / (sqrt(rho) c_v) grad T) . grad c_v
        s4 = s4 - sum((u[4] * v[d] - C.c_kappa * kappa * isr / cv * gT[d]) * gcv[d] for d in range(3)) / cv
    s.append(s4)
    return np.stack(s)


def sigma(uhat, C, x=None):
    """Diagonal of sigma = sigma_c + sigma_d of Eq. LDG2, evaluated at the trace state uhat."""
    isr = np.exp(-0.5 * uhat[0])
    T = uhat[4] * isr
    mix = _mixture(x, C)
    mu, kappa = _transport(T, C, uhat[0], mix)
    lam = C.lam * np.ones_like(uhat[0])
    sm = lam + C.c_mu * mu * isr
    return np.stack([lam, sm, sm, sm, lam + C.c_kappa * kappa * isr / mix[1]])


def wall_state(u, C):
    """No-slip isothermal wall trace: (varrho, 0, 0, 0, exp(varrho/2) T_wall)."""
    z = 0.0 * u[0]
    return np.stack([u[0], z, z, z, np.exp(0.5 * u[0]) * C.t_wall])
