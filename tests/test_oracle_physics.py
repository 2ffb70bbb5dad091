"""Pin of the oracle's flux/source (Eq. fluxSWNondimensional) against the original system, Eq. NS1.

The paper derives the (varrho, sqrt(rho) v, sqrt(rho) T) flux form from the rotating-frame
Navier-Stokes equations NS1 with the ideal-gas law (Eq. eos) and Stokes stress (Eq. stress).
Here NS1 is written independently in primitive variables and nondimensionalised with the scales of
Sec. 2.4 (x ~ H0, v ~ a0, t ~ H0/a0, rho ~ rho0, T ~ T0, p ~ rho0 a0^2, a0^2 = gamma g0 H0):

  drho/dt = -div(rho v)
  rho (dv/dt + v.grad v) + grad p - c_mu div(mu eps) = rho a,                 p = rho T / (gamma m)
  rho c_v (dT/dt + v.grad T) + gamma (gamma-1) p div v
        = Q + c_kappa div(kappa grad T) + c_diss mu eps : grad v

with c_mu = mu0/(rho0 a0 H0) = 1/sqrt(gamma Gr), c_kappa = kappa0/(rho0 c_v0 a0 H0) =
sqrt(gamma/Gr)/Pr and c_diss = mu0 a0 / (rho0 c_v0 T0 H0) = (gamma-1) sqrt(gamma/Gr) (dimensional
analysis with c_v0 T0 = a0^2 / (gamma (gamma-1)) and Re^2 = gamma Gr).

For smooth analytic fields, du/dt = -div F(u, grad u) + s(u, grad u) from the oracle, converted to
(drho/dt, dv/dt, dT/dt) by the chain rule, must equal the right-hand sides above. A dropped term,
a wrong sign or a wrong coefficient in the oracle's flux or source breaks this identity.
"""
import math

import numpy as np
import pytest

from oracle import physics as P
from paper_2306_01085_gb300 import workloads as W

H_CS = 1e-30


def fields(x):
    """Primitive fields rho, v, T at points x (3, n); any dtype."""
    X, Y, Z = x
    rho = np.exp(0.3 * np.sin(0.7 * X + 1.3 * Y) - 0.2 * Z + 0.1 * np.cos(0.5 * Z * X))
    v = np.stack([0.1 * np.sin(X + Y - 0.3 * Z), 0.2 * np.cos(X - 0.6 * Y + 0.4 * Z), 0.05 * np.sin(0.9 * X * Y + 0.7 * Z)])
    T = 1.3 + 0.2 * np.cos(X - 0.8 * Z) + 0.1 * np.sin(0.6 * Y)
    return rho, v, T


def u_of(x):
    rho, v, T = fields(x)
    s = np.sqrt(rho)
    return np.stack([np.log(rho), s * v[0], s * v[1], s * v[2], s * T])


def cs_grad(fun, x):
    """Complex-step gradient of a vector function fun(x) -> (k, n): returns (3, k, n)."""
    out = []
    for d in range(3):
        xc = x.astype(np.complex128)
        xc[d] += 1j * H_CS
        out.append(fun(xc).imag / H_CS)
    return np.stack(out)


def fd_div(fun, x, h=1e-3):
    """4th-order central difference divergence: fun(x) -> (k, 3, n); returns (k, n)."""
    acc = 0.0
    for d in range(3):
        e = np.zeros_like(x)
        e[d] = h
        acc = acc + (-fun(x + 2 * e)[:, d] + 8 * fun(x + e)[:, d] - 8 * fun(x - e)[:, d]
                     + fun(x - 2 * e)[:, d]) / (12 * h)
    return acc


def flux_of(x, C):
    return P.flux(u_of(x), cs_grad(u_of, x), C, x=x)


def make_desc(kind):
    if kind == "shell_comp":
        d = make_desc("shell")
        d.comp = 1
        d.comp_a = (0.5, 0.1, 0.2, 0.05, 0.01, 0.0)     # N2, O2, He, varying over |r| in [1, 3]
        d.comp_b = (-0.8, -2.0, -1.0, -3.0, 1.0, 0.0)
        d.eddy_nu, d.eddy_alpha = 0.3, 0.2
        return d
    if kind == "box":
        d = W.box_desc(p=2, n=2, re=50.0, pr=0.7, visc_exp=0.0)
        d.gvec = (0.1, -0.2, -1.0)
    else:
        d = W.shell_desc(n=2, nr=2, p=2, euv=True)
        d.grashof = 30.0 ** 2 / d.gamma
        d.prandtl = 0.9
        d.froude = 0.3
        d.omega = (0.1, 0.2, 1.0)
        d.g_r0 = 1.5
        d.euv_amp = 0.2
        d.euv_r_peak = 2.0
        d.euv_width = 0.5
        d.euv_omega_t = 0.4
    return d


def _mix(y, d):
    """m, c_v and the kappa factor of the composition fits at y, written from Sec. 2.1.1-2.1.2."""
    r = np.sqrt((y ** 2).sum(0))
    ms = [1.0, 1.75, 2.0, 0.25]
    al = [1.0, 3.6 / 5.6, 3.6 / 5.6, 1.0]
    ch = [d.comp_a[2 * s] * np.exp(d.comp_b[2 * s] * r) + d.comp_a[2 * s + 1] * np.exp(d.comp_b[2 * s + 1] * r)
          for s in range(3)]
    chi = [1.0 - ch[0] - ch[1] - ch[2]] + ch
    moles = [chi[s] / ms[s] for s in range(4)]
    tot = moles[0] + moles[1] + moles[2] + moles[3]
    return 1.0 / tot, tot, sum(moles[s] * al[s] for s in range(4)) / tot


@pytest.mark.parametrize("kind", ["box", "shell", "shell_comp"])
def test_flux_form_reproduces_navier_stokes(kind):
    d = make_desc(kind)
    C = P.Coeffs(d)
    rng = np.random.default_rng(7)
    x = rng.uniform(0.5, 1.5, size=(3, 12))
    t = 0.7
    # oracle: du/dt = -div F + s
    u = u_of(x)
    q = cs_grad(u_of, x)
    dudt = -fd_div(lambda y: flux_of(y, C), x) + P.source(u, q, x, t, C)
    rho, v, T = fields(x)
    sr = np.sqrt(rho)
    drho = rho * dudt[0]
    dv = (dudt[1:4] - 0.5 * u[1:4] * dudt[0]) / sr
    dT = (dudt[4] - 0.5 * u[4] * dudt[0]) / sr

    # independent primitive-variable NS1
    g = d.gamma
    c_mu = 1.0 / math.sqrt(g * d.grashof)
    c_k = math.sqrt(g / d.grashof) / d.prandtl
    c_d = (g - 1.0) * math.sqrt(g / d.grashof)
    comp = kind == "shell_comp"

    def m_of(y):
        return _mix(y, d)[0] if comp else d.mass

    def cv_of(y):
        return _mix(y, d)[1] if comp else 1.0 / d.mass

    def visc(T_, y=None):
        if comp:
            return np.sqrt(T_ * m_of(y)) + d.eddy_nu * fields(y)[0]
        return T_ ** d.visc_exp if d.visc_exp else np.ones_like(T_)

    def cond(T_, y=None):
        if comp:
            return _mix(y, d)[2] * T_ ** 0.69 + d.eddy_alpha * fields(y)[0] / m_of(y)
        return visc(T_)

    m = m_of(x)
    cv = cv_of(x)

    def grad_v(y):
        return cs_grad(lambda z: fields(z)[1], y)            # [d, m] = d v_m / d x_d

    def eps_of(y):
        G = grad_v(y)
        div = G[0, 0] + G[1, 1] + G[2, 2]
        return np.stack([np.stack([G[dd, mm] + G[mm, dd] - (2 / 3) * div * (mm == dd) for dd in range(3)])
                         for mm in range(3)])                 # [m, d]

    def tau(y):
        return c_mu * visc(fields(y)[2], y) * eps_of(y)       # (3, 3, n)

    def heat(y):
        return (c_k * cond(fields(y)[2], y) * cs_grad(lambda z: fields(z)[2][None], y)[:, 0])[None]

    def mass_flux(y):
        r_, v_, _ = fields(y)
        return (r_ * v_)[None]

    Gv = grad_v(x)
    GT = cs_grad(lambda z: fields(z)[2][None], x)[:, 0]
    p_of = lambda z: (fields(z)[0] * fields(z)[2] / (g * m_of(z)))[None]
    Gp = cs_grad(p_of, x)[:, 0]
    div_v = Gv[0, 0] + Gv[1, 1] + Gv[2, 2]
    # acceleration a = g/gamma - Fr^2/gamma w x (w x r) - 2 Fr/sqrt(gamma) w x v
    if d.gravity_kind == 0:
        gv = np.array(d.gvec)[:, None] * np.ones_like(x)
    else:
        r = np.sqrt((x ** 2).sum(0))
        gv = -(d.g_r0 / r) ** 2 * x / r
    w = np.array(d.omega)[:, None]
    a = gv / g - d.froude ** 2 / g * np.cross(w, np.cross(w, x, axis=0), axis=0) \
        - 2 * d.froude / math.sqrt(g) * np.cross(w, v, axis=0)
    Q = P.euv_heating(x, t, C)

    drho_ref = -fd_div(mass_flux, x)[0]
    vgradv = np.einsum("dn,dmn->mn", v, Gv)
    dv_ref = -vgradv - Gp / rho + fd_div(tau, x) / rho + a
    eps = eps_of(x)
    dissip = np.einsum("mdn,dmn->n", visc(T, x)[None, None] * eps, Gv)
    # rho D(c_v T)/Dt with c_v(x): rho c_v DT/Dt + rho T v . grad c_v
    vgcv = np.einsum("dn,dn->n", v, cs_grad(lambda z: np.atleast_2d(cv_of(z) * np.ones(z.shape[1:])), x)[:, 0]) \
        if comp else 0.0
    dT_ref = -np.einsum("dn,dn->n", v, GT) + (
        Q - g * (g - 1) * (rho * T / (g * m)) * div_v + fd_div(heat, x)[0] + c_d * dissip
        - rho * T * vgcv) / (rho * cv)

    assert np.abs(drho - drho_ref).max() < 1e-8 * np.abs(drho_ref).max()
    assert np.abs(dv - dv_ref).max() < 1e-8 * np.abs(dv_ref).max()
    assert np.abs(dT - dT_ref).max() < 1e-8 * np.abs(dT_ref).max()


def test_euv_heating_shape():
    d = make_desc("shell")
    C = P.Coeffs(d)
    t = 0.0   # sub-solar point on +x
    pts = np.array([[2.0, 0.0, 0.0], [2.5, 0.0, 0.0], [0.0, 2.0, 0.0]]).T
    q = P.euv_heating(pts, t, C)
    assert abs(q[0] - d.euv_amp) < 1e-15
    assert abs(q[1] - 0.5 * d.euv_amp) < 1e-14                     # one half-width above the peak
    chi = math.pi / 2
    assert abs(q[2] - d.euv_amp * math.exp(-chi ** 2 / (2 * d.euv_sigma ** 2))) < 1e-15
    # the sub-solar point moves westward at the rotation rate
    t = math.pi / 2 / d.euv_omega_t
    q = P.euv_heating(np.array([[0.0], [-2.0], [0.0]]), t, C)
    assert abs(q[0] - d.euv_amp) < 1e-14


def test_sigma_and_wall_state():
    d = make_desc("shell")
    C = P.Coeffs(d)
    u = np.array([[-2.0], [0.1], [0.2], [0.3], [1.5 * math.exp(-1.0)]])
    s = P.sigma(u, C)
    T = 1.5
    mu = T ** d.visc_exp
    assert abs(s[0, 0] - d.lambda0) < 1e-15
    assert abs(s[1, 0] - (d.lambda0 + mu / math.sqrt(d.gamma * d.grashof) * math.exp(1.0))) < 1e-13
    assert abs(s[4, 0] - (d.lambda0 + mu * math.sqrt(d.gamma / d.grashof) / d.prandtl * math.exp(1.0)
                          * d.mass)) < 1e-13
    ub = P.wall_state(u, C)
    assert np.allclose(ub[:, 0], [-2.0, 0, 0, 0, math.exp(-1.0) * d.t_wall])
