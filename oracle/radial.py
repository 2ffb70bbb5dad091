"""Radial one-dimensional model (oracle; test infrastructure only).

Sec. 4.3 runs "the radial 1D thermospheric model": the same physics on a radial column of 28
elements of degree 2 with a geometric mesh from 2.5 km, stepped by DIRK(2,2). The paper does not
print its equations; the reading taken here is the spherically symmetric restriction of the 3D
problem:

  * fields depend on r only and the velocity is radial, u = (varrho, m = sqrt(rho) v_r, e = sqrt(rho) T);
    the rotating-frame accelerations are dropped (they are not spherically symmetric; the paper names
    Coriolis and horizontal winds as the 3D effects the 1D model lacks); gravity is radial;
  * the LDG weak form of Eq. DGformulation is kept with trial and test functions restricted to the
    symmetric subspace: scalars p(r), radial vectors p(r) r_hat and, for the gradient of the radial
    velocity, tensors a(r) r_hat r_hat + b(r) (I - r_hat r_hat). Integrals over the shell carry the
    measure r^2 dr (the 4 pi cancels). This gives, per element [r_L, r_R]:
      gradient:  (q, p)_{r^2} = -int u (r^2 p)' dr + [r^2 u_hat p]_L^R        (scalars, Q_rr)
                 (Q_tt, b)_{r^2} = int m b r dr                                (tangential part of grad m)
      residual:  (du/dt, w)_{r^2} = int (F_r w' + S w) r^2 dr - [r^2 F_hat w]_L^R,
                 S = s + 2 F_tt / r for the momentum (the tangential stress entering through
                 div(w r_hat) = w' + 2 w / r), S = s otherwise;
  * the flux and source are those of Eq. fluxSWNondimensional evaluated on the symmetric fields:
    grad v = v' r_hat r_hat + (v/r)(I - r_hat r_hat), eps_rr = (4/3)(v' - v/r), eps_tt = -eps_rr/2;
  * mu* = T*^visc_exp and kappa* = alpha0 T*^visc_exp with the column's conductivity factor alpha0
    (Sec. 4.3), EUVAC heating (Sec. 2.2) at the column's site with the column's efficiency epsilon;
  * boundaries as in 3D: wall at the bottom, outflow at the top; numerical flux of Eq. LDG2;
  * every integral uses the (p+1)-point Gauss rule of the element (the 1D counterpart of the
    (p+1)^3 Gauss rule of the shell), including the r^2 weight.

The element operators here are dense: element mass matrices with the r^2 weight solved by LU for
the gradient, nodal residuals tested against every Lagrange basis function. Jv is the complex-step
derivative. The implicit step is DIRK with Newton on the stage equations and a dense direct solve of
each Newton system (the Jacobian by complex-step columns).

Pinned by tests/test_oracle_radial.py: the 1D flux and source equal the 3D oracle physics at
symmetric states (projected on r_hat and on the tangential plane), free stream is exact on the
curved column, the isothermal hydrostatic column converges at rate >= p, complex-step Jv against
central differences, and the DIRK step against a direct solve.
"""
import math

import numpy as np

from . import euvac as _euvac
from . import quadrature as Q

BC_WALL, BC_OUTFLOW = 1, 2


class Coeffs:
    """Nondimensional numbers of a radial ensemble (Eq. nondimensional)."""

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
        self.g_r0 = desc.g_r0
        self.euv = desc.euv
        for k in ("euv_omega_t", "euv_day", "euv_f107", "euv_f107a", "euv_eff", "euv_dsun", "ref_T0",
                  "ref_rho0", "ref_m", "ref_g0"):
            setattr(self, k, getattr(desc, k))
        self.comp = 0


class RadialMesh:
    """Element radii, Gauss rule and Lagrange bases of the radial column mesh."""

    def __init__(self, desc, nodes_r):
        self.desc = desc
        self.n = n = desc.p + 1
        self.E = desc.n_elem
        self.xi, _ = Q.gll(n)
        self.xg, self.wg = Q.gauss(n)
        self.phi = Q.lagrange(self.xi, self.xg)                   # (g, i)
        self.dphi = Q.lagrange_deriv(self.xi, self.xg)            # (g, i) d/dxi
        self.phiL = Q.lagrange(self.xi, [-1.0])[0]                # (i,)
        self.phiR = Q.lagrange(self.xi, [1.0])[0]
        r = np.asarray(nodes_r, dtype=np.float64)                 # (E, n) node radii
        self.rL, self.rR = r[:, 0], r[:, -1]
        self.J = 0.5 * (self.rR - self.rL)                        # dr/dxi
        self.rg = np.einsum("gi,ei->eg", self.phi, r)             # Gauss-point radii
        self.W = self.wg[None, :] * self.J[:, None] * self.rg ** 2   # mass weights w J r^2
        self.M = np.einsum("eg,gi,gj->eij", self.W, self.phi, self.phi)


def _unit(lat, lon):
    return np.array([math.cos(lat) * math.cos(lon), math.cos(lat) * math.sin(lon), math.sin(lat)])


# ----------------------------------------------------------------------------------------------
# pointwise physics of the symmetric problem
# ----------------------------------------------------------------------------------------------
def primitives(u, q, r, C, alpha0):
    """sqrt(rho), 1/sqrt(rho), v, T, grad v (rr, tt), grad T, div v, eps (rr, tt), mu, kappa.
    q = (d varrho/dr, Q_rr, Q_tt, de/dr) with Q the symmetric gradient of m r_hat."""
    sr = np.exp(0.5 * u[0])
    isr = np.exp(-0.5 * u[0])
    v = u[1] * isr
    T = u[2] * isr
    gv_rr = isr * (q[1] - 0.5 * u[1] * q[0])
    gv_tt = isr * q[2]
    gT = isr * (q[3] - 0.5 * u[2] * q[0])
    div = gv_rr + 2.0 * gv_tt
    eps_rr = 2.0 * gv_rr - (2.0 / 3.0) * div
    eps_tt = 2.0 * gv_tt - (2.0 / 3.0) * div
    mu = T ** C.visc_exp if C.visc_exp != 0.0 else np.ones_like(T)
    kappa = alpha0 * mu
    return sr, isr, v, T, gv_rr, gv_tt, gT, div, eps_rr, eps_tt, mu, kappa


def flux(u, q, r, C, alpha0, viscous=True):
    """Radial fluxes (F_varrho, F_rr, F_e) and the tangential momentum flux F_tt."""
    sr, isr, v, T, gv_rr, gv_tt, gT, div, eps_rr, eps_tt, mu, kappa = primitives(u, q, r, C, alpha0)
    pc = 1.0 / (C.gamma * C.m)
    F0 = u[0] * v
    Frr = u[1] * v + pc * u[2]
    Ftt = pc * u[2]
    Fe = u[2] * v
    if viscous:
        cm = C.c_mu * mu * isr
        ck = C.c_kappa * kappa * isr / C.cv
        Frr = Frr - cm * eps_rr
        Ftt = Ftt - cm * eps_tt
        Fe = Fe - ck * gT
    return np.stack([F0, Frr, Fe]), Ftt


def heating(u, r, t, C, eps, site):
    """EUVAC heating Q* at radius r above the unit site direction, with efficiency eps."""
    if C.euv != 2:
        return 0.0 * u[0]
    u5 = np.stack([u[0], 0.0 * u[0], 0.0 * u[0], 0.0 * u[0], u[2]])
    x = np.stack([site[d] * r for d in range(3)])
    C5 = _C5(C, eps)
    return _euvac.heating(u5, x, t, C5)


class _C5:
    """The coefficient view that the EUVAC heating reads, with the column's efficiency."""

    def __init__(self, C, eps):
        self.__dict__.update(C.__dict__)
        self.euv_eff = eps


def source(u, q, r, t, C, alpha0, eps, site):
    """Source (s_varrho, s_m, s_e) of Eq. fluxSWNondimensional on the symmetric fields (radial
    momentum component; the tangential stress term enters the residual separately)."""
    sr, isr, v, T, gv_rr, gv_tt, gT, div, eps_rr, eps_tt, mu, kappa = primitives(u, q, r, C, alpha0)
    pc = 1.0 / (C.gamma * C.m)
    cm = C.c_mu * mu * isr
    ck = C.c_kappa * kappa * isr / C.cv
    a_r = -(C.g_r0 / r) ** 2 / C.gamma
    s0 = (u[0] - 1.0) * div
    s1 = sr * a_r + 0.5 * div * u[1] - 0.5 * pc * u[2] * q[0] + 0.5 * cm * eps_rr * q[0]
    diss = eps_rr * gv_rr + 2.0 * eps_tt * gv_tt
    s2 = (heating(u, r, t, C, eps, site) * isr / C.cv + (1.5 - C.gamma) * u[2] * div
          + 0.5 * ck * gT * q[0] + C.c_diss * mu * isr / C.cv * diss)
    return np.stack([s0, s1, s2])


def sigma(uh, C, alpha0):
    """Diagonal of sigma = sigma_c + sigma_d of Eq. LDG2 at the trace state."""
    isr = np.exp(-0.5 * uh[0])
    T = uh[2] * isr
    mu = T ** C.visc_exp if C.visc_exp != 0.0 else np.ones_like(T)
    kappa = alpha0 * mu
    lam = C.lam + 0.0 * uh[0]
    return np.stack([lam, lam + C.c_mu * mu * isr, lam + C.c_kappa * kappa * isr / C.cv])


def wall_state(u, C):
    return np.stack([u[0], 0.0 * u[0], np.exp(0.5 * u[0]) * C.t_wall])


# ----------------------------------------------------------------------------------------------
# discretisation of one column: u (3, E, n) nodal values
# ----------------------------------------------------------------------------------------------
def _traces(mesh, u):
    """Left and right end values (3, E) of each element (GLL nodes include the end points)."""
    return np.einsum("i,cei->ce", mesh.phiL, u), np.einsum("i,cei->ce", mesh.phiR, u)


def _uhat(mesh, u, C):
    """Trace u_hat at the E + 1 interfaces (3, E + 1): averages inside, boundary traces at the ends."""
    uL, uR = _traces(mesh, u)
    uh = np.zeros((3, mesh.E + 1), dtype=u.dtype)
    uh[:, 1:-1] = 0.5 * (uR[:, :-1] + uL[:, 1:])
    uh[:, 0] = wall_state(uL[:, 0], C) if mesh.desc.bc_lo == BC_WALL else uL[:, 0]
    uh[:, -1] = wall_state(uR[:, -1], C) if mesh.desc.bc_hi == BC_WALL else uR[:, -1]
    return uh


def gradient(mesh, u, C):
    """Nodal q (4, E, n) = (d varrho/dr, Q_rr, Q_tt, de/dr) from the LDG gradient equation."""
    E, n = mesh.E, mesh.n
    uh = _uhat(mesh, u, C)
    ug = np.einsum("gi,cei->ceg", mesh.phi, u)
    wJ = mesh.wg[None, :] * mesh.J[:, None]
    dphidr = mesh.dphi[None, :, :] / mesh.J[:, None, None]     # (e, g, i)
    q = np.zeros((4, E, n), dtype=u.dtype)
    for qi, c in ((0, 0), (1, 1), (3, 2)):
        # -int u (r^2 p)' dr = -int u (2 r p + r^2 p') dr, then the face terms r^2 u_hat p
        rhs = -np.einsum("eg,eg,gi->ei", wJ, ug[c] * 2.0 * mesh.rg, mesh.phi)
        rhs = rhs - np.einsum("eg,eg,egi->ei", wJ, ug[c] * mesh.rg ** 2, dphidr)
        rhs = rhs + (mesh.rR ** 2 * uh[c, 1:])[:, None] * mesh.phiR[None, :]
        rhs = rhs - (mesh.rL ** 2 * uh[c, :-1])[:, None] * mesh.phiL[None, :]
        q[qi] = np.linalg.solve(mesh.M, rhs[..., None])[..., 0]
    rhs = np.einsum("eg,eg,gi->ei", wJ, ug[1] * mesh.rg, mesh.phi)
    q[2] = np.linalg.solve(mesh.M, rhs[..., None])[..., 0]
    return q


def residual(mesh, u, t, C, params):
    """Nodal residual (3, E, n): int (F_r w' + S w) r^2 dr - [r^2 F_hat w] for one column with
    params = (epsilon, alpha0, latitude, longitude)."""
    eps, alpha0, lat, lon = params
    site = _unit(lat, lon)
    q = gradient(mesh, u, C)
    ug = np.einsum("gi,cei->ceg", mesh.phi, u)
    qg = np.einsum("gi,cei->ceg", mesh.phi, q)
    F, Ftt = flux(ug, qg, mesh.rg, C, alpha0)
    S = source(ug, qg, mesh.rg, t, C, alpha0, eps, site)
    S[1] = S[1] + 2.0 * Ftt / mesh.rg
    wJ = mesh.wg[None, :] * mesh.J[:, None]
    dphidr = mesh.dphi[None, :, :] / mesh.J[:, None, None]
    r = (np.einsum("eg,eg,ceg,egi->cei", wJ, mesh.rg ** 2, F, dphidr)
         + np.einsum("eg,eg,ceg,gi->cei", wJ, mesh.rg ** 2, S, mesh.phi))
    Fh = face_fluxes(mesh, u, q, C, alpha0)                    # (3, E + 1) radial numerical flux
    r = r - (mesh.rR ** 2)[None, :, None] * Fh[:, 1:, None] * mesh.phiR[None, None, :]
    r = r + (mesh.rL ** 2)[None, :, None] * Fh[:, :-1, None] * mesh.phiL[None, None, :]
    return r


def face_fluxes(mesh, u, q, C, alpha0):
    """Radial numerical flux F_hat . r_hat at the E + 1 interfaces (Eq. LDG2)."""
    uL, uR = _traces(mesh, u)
    qL, qR = _traces_q(mesh, q)
    E = mesh.E
    Fh = np.zeros((3, E + 1), dtype=u.dtype)
    rf = np.concatenate([mesh.rL, mesh.rR[-1:]])
    # interior: the element below (its right end) and the element above (its left end)
    a_u, a_q = uR[:, :-1], qR[:, :-1]
    b_u, b_q = uL[:, 1:], qL[:, 1:]
    Fa, _ = flux(a_u, a_q, rf[1:-1], C, alpha0)
    Fb, _ = flux(b_u, b_q, rf[1:-1], C, alpha0)
    uh = 0.5 * (a_u + b_u)
    sg = sigma(uh, C, alpha0)
    Fh[:, 1:-1] = 0.5 * (Fa + Fb) + sg * (0.5 * (a_u - b_u))
    # bottom (outward normal -r_hat): F_hat . n = F(u_b, q) . n + sigma(u_b)(u - u_b) for a wall
    u0, q0 = uL[:, 0], qL[:, 0]
    if mesh.desc.bc_lo == BC_WALL:
        ub = wall_state(u0, C)
        Fb0, _ = flux(ub, q0, rf[0], C, alpha0)
        Fh[:, 0] = Fb0 - sigma(ub, C, alpha0) * (u0 - ub)
    else:
        F0, _ = flux(u0, q0, rf[0], C, alpha0, viscous=False)
        Fh[:, 0] = F0
    # top (outward normal +r_hat)
    u1, q1 = uR[:, -1], qR[:, -1]
    if mesh.desc.bc_hi == BC_WALL:
        ub = wall_state(u1, C)
        F1, _ = flux(ub, q1, rf[-1], C, alpha0)
        Fh[:, -1] = F1 + sigma(ub, C, alpha0) * (u1 - ub)
    else:
        F1, _ = flux(u1, q1, rf[-1], C, alpha0, viscous=False)
        Fh[:, -1] = F1
    return Fh


def _traces_q(mesh, q):
    return np.einsum("i,cei->ce", mesh.phiL, q), np.einsum("i,cei->ce", mesh.phiR, q)


def jvp(mesh, u, v, t, C, params, h=1e-30):
    """Exact J v by complex step: Im r(u + i h v) / h."""
    uc = u.astype(np.complex128) + 1j * h * v
    return residual(mesh, uc, t, C, params).imag / h


def mass_apply(mesh, v):
    """(M v) with the r^2-weighted element mass matrices, per variable."""
    return np.einsum("eij,cej->cei", mesh.M, v)


def implicit_step(mesh, u_n, t, dt, C, params, stages=2, tol=1e-10, max_newton=20):
    """One DIRK step of M du/dt = r(u) for one column: Newton on each stage equation
    G(U) = M (U - u_n) - dt sum_{j<i} a_ij r(U_j) - dt a_ii r(U) = 0 with the exact Jacobian
    (complex-step columns) and a dense direct solve; stops when ||G||_2 <= tol ||G(U^0)||_2 or
    ||G||_2 <= 1e-14 ||M U||_2 (the rule of the shell's implicit step)."""
    from . import solver as S
    A, b, c = S.dirk_tableau(stages)
    Mu = mass_apply(mesh, u_n)
    R = []
    U = u_n.copy()
    n = U.size
    its = []
    for i in range(stages):
        known = Mu + sum(dt * A[i, j] * R[j] for j in range(i)) if i else Mu.copy()
        ti = t + c[i] * dt
        daii = dt * A[i, i]
        g0 = None
        for it in range(max_newton + 1):
            G = mass_apply(mesh, U) - known - daii * residual(mesh, U, ti, C, params)
            gn = np.linalg.norm(G)
            g0 = gn if g0 is None else g0
            if gn <= tol * g0 or gn <= 1e-14 * np.linalg.norm(mass_apply(mesh, U)):
                break
            Jm = np.zeros((n, n))
            for j in range(n):
                e = np.zeros(n)
                e[j] = 1.0
                ev = e.reshape(U.shape)
                Jm[:, j] = (mass_apply(mesh, ev) - daii * jvp(mesh, U, ev, ti, C, params)).ravel()
            U = U - np.linalg.solve(Jm, G.ravel()).reshape(U.shape)
        else:
            raise RuntimeError("Newton did not converge")
        its.append(it)
        R.append(residual(mesh, U, ti, C, params))
    return U, its
