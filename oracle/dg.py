"""LDG gradient, residual and Jacobian-vector product (oracle; test infrastructure only).

Semi-discrete form, Eq. DGformulation, with the LDG trace and flux of Eq. LDG2:

  (a)  (q_h, p) + (u_h, div p) - <u_hat, p.n> = 0                     for all p in Q_h
  (b)  (du_h/dt, w) = (F(u_h, q_h), grad w) - <F_hat.n, w> + (s(u_h, q_h), w)   for all w in W_h

  u_hat = (u + u^-)/2,  F_hat.n = (F(u, q) + F(u^-, q^-)).n / 2 + sigma (u - u_hat).

`residual` returns the right-hand side of (b) tested against every nodal basis function (r = M du/dt);
`gradient` returns the nodal q solving (a) with the dense element mass matrix (LU solve).
Integrals use the tensor Gauss rule; every element operator is a dense (n^3 x n^3) matrix built
from the basis definition. Boundary traces (reading of the boundary conditions of Sec. 2.5):
  wall     u_hat = (varrho, 0, 0, 0, exp(varrho/2) T_wall),
           F_hat.n = F(u_hat, q).n + sigma(u_hat) (u - u_hat)
  outflow  u_hat = u, F_hat.n = F_inviscid(u).n (adiabatic, zero viscous normal stress)
sigma is evaluated at u_hat on every face.

Jv: the complex-step derivative Im r(u + i h v) / h (h = 1e-30). Every operation on the state is
complex-analytic, so this is the exact directional derivative up to rounding.

Parity pinned by tests/test_oracle_dg.py: free stream, exact gradients of polynomials, discrete
conservation sum_i r = int s on periodic boxes, translation equivariance, consistency with the
strong form at rate >= p, hydrostatic convergence, central finite differences of the residual.
"""
import numpy as np

from . import physics as P

BC_WALL, BC_OUTFLOW = 1, 2


def _face_traces(mesh, arr, elems):
    """Values of a nodal field arr[e, c, i] at the face Gauss points: (len(elems), 6, C, Nf)."""
    a = arr[elems]
    return np.stack([np.einsum("fi,eci->ecf", mesh.phiF[f], a) for f in range(6)], axis=1)


def _neighbour_traces(mesh, traces_all, elems, f):
    """Neighbour's trace on face f of each element in elems, re-ordered to the element's own face
    points. traces_all is indexed by global element. Boundary faces return the own trace."""
    nb = mesh.nbr_elem[elems, f]
    nf = mesh.nbr_face[elems, f]
    own = traces_all[elems, f]
    out = own.copy()
    inter = np.nonzero(nb >= 0)[0]
    if len(inter):
        t = traces_all[nb[inter], nf[inter]]                   # (m, C, Nf) in the neighbour's order
        perm = mesh.nbr_pt[elems[inter], f]                    # (m, Nf)
        out[inter] = np.take_along_axis(t, perm[:, None, :], axis=2)
    return out


def _scatter(mesh, elems, values, shape, dtype):
    full = np.zeros(shape, dtype=dtype)
    full[elems] = values
    return full


def gradient(mesh, u, elems=None):
    """Nodal LDG gradient q[e, d, c, i] on the elements `elems` (all by default), Eq. DGformulation a."""
    C = P.Coeffs(mesh.desc)
    E_all = mesh.n_elem
    elems = np.arange(E_all) if elems is None else np.asarray(elems)
    need = np.union1d(elems, mesh.neighbours(elems))
    tr_need = _face_traces(mesh, u, need)
    traces = _scatter(mesh, need, tr_need, (E_all, 6, 5, mesh.Nf), u.dtype)
    uE = u[elems]
    uG = np.einsum("gi,eci->ecg", mesh.phi, uE)
    Wd = mesh.W[None, :] * mesh.detJ[elems]                           # (e, g)
    # -(u, d phi_i / d x_d) with d phi_i/d x_d = sum_a d phi_i / d xi_a  d xi_a / d x_d
    Y = np.einsum("eg,egad,ecg->ecadg", Wd, mesh.Jinv[elems], uG)
    rhs = -np.einsum("ecadg,gai->ecdi", Y, mesh.dphi)
    for f in range(6):
        own = traces[elems, f]
        nbr = _neighbour_traces(mesh, traces, elems, f)
        bc = mesh.bc[elems, f]
        uhat = 0.5 * (own + nbr)
        wall = bc == BC_WALL
        if np.any(wall):
            uhat[wall] = np.moveaxis(P.wall_state(np.moveaxis(own[wall], 0, 1), C), 0, 1)
        out = bc == BC_OUTFLOW
        if np.any(out):
            uhat[out] = own[out]
        # + <u_hat, phi_i n_d>
        rhs = rhs + np.einsum("f,edf,ecf,fi->ecdi", mesh.wF, mesh.nF[elems, f], uhat, mesh.phiF[f])
    M = np.einsum("eg,gi,gj->eij", Wd, mesh.phi, mesh.phi)
    b = rhs.reshape(len(elems), 15, mesh.Np).transpose(0, 2, 1)     # (e, i, c*3+d)
    sol = np.linalg.solve(M, b)                                        # (e, i, 15)
    q_cd = sol.transpose(0, 2, 1).reshape(len(elems), 5, 3, mesh.Np)
    return np.ascontiguousarray(q_cd.transpose(0, 2, 1, 3))          # (e, d, c, i)


def face_fluxes(mesh, u, q, elems, C):
    """F_hat . (n dS) at the face Gauss points of each element face: (len(elems), 6, 5, Nf)."""
    E_all = mesh.n_elem
    need = np.union1d(elems, mesh.neighbours(elems))
    tu = _scatter(mesh, need, _face_traces(mesh, u, need), (E_all, 6, 5, mesh.Nf), u.dtype)
    qflat = q.reshape(E_all, 15, mesh.Np)
    tq = _scatter(mesh, need, _face_traces(mesh, qflat, need), (E_all, 6, 15, mesh.Nf), q.dtype)
    out = []
    for f in range(6):
        u_own = np.moveaxis(tu[elems, f], 0, 1)                                  # (5, e, Nf)
        q_own = np.moveaxis(tq[elems, f].reshape(len(elems), 3, 5, mesh.Nf), 0, 2)  # (3, 5, e, Nf)
        u_nb = np.moveaxis(_neighbour_traces(mesh, tu, elems, f), 0, 1)
        q_nb = np.moveaxis(_neighbour_traces(mesh, tq, elems, f).reshape(len(elems), 3, 5, mesh.Nf), 0, 2)
        nds = np.moveaxis(mesh.nF[elems, f], 0, 1)                              # (3, e, Nf)
        xf = np.moveaxis(mesh.xF[elems, f], 0, 1)                               # (3, e, Nf)
        area = mesh.areaF[elems, f]                                              # (e, Nf)
        bc = mesh.bc[elems, f]
        # interior: central flux plus sigma (u - u_hat)
        uhat = 0.5 * (u_own + u_nb)
        Fo = P.flux(u_own, q_own, C, x=xf)
        Fn = P.flux(u_nb, q_nb, C, x=xf)
        fh = 0.5 * np.einsum("cdef,def->cef", Fo + Fn, nds) + P.sigma(uhat, C, xf) * (u_own - uhat) * area
        wall = bc == BC_WALL
        if np.any(wall):
            ub = P.wall_state(u_own[:, wall], C)
            Fb = P.flux(ub, q_own[:, :, wall], C, x=xf[:, wall])
            fh[:, wall] = (np.einsum("cdef,def->cef", Fb, nds[:, wall])
                           + P.sigma(ub, C, xf[:, wall]) * (u_own[:, wall] - ub) * area[wall])
        out_ = bc == BC_OUTFLOW
        if np.any(out_):
            Fi = P.flux(u_own[:, out_], q_own[:, :, out_], C, viscous=False, x=xf[:, out_])
            fh[:, out_] = np.einsum("cdef,def->cef", Fi, nds[:, out_])
        out.append(np.moveaxis(fh, 0, 1))
    return np.stack(out, axis=1)


def residual(mesh, u, q=None, t=0.0, elems=None):
    """Nodal residual r[e, c, i] = (F, grad phi_i) - <F_hat.n, phi_i> + (s, phi_i), Eq. DGformulation b.

    q: nodal gradient on all elements (None: computed from u by `gradient` where needed).
    """
    C = P.Coeffs(mesh.desc)
    E_all = mesh.n_elem
    elems = np.arange(E_all) if elems is None else np.asarray(elems)
    if q is None:
        need = np.union1d(elems, mesh.neighbours(elems))
        q = _scatter(mesh, need, gradient(mesh, u, need), (E_all, 3, 5, mesh.Np), u.dtype)
    uE, qE = u[elems], q[elems]
    uG = np.moveaxis(np.einsum("gi,eci->ecg", mesh.phi, uE), 0, 1)               # (5, e, g)
    qG = np.moveaxis(np.einsum("gi,edci->edcg", mesh.phi, qE), 0, 2)             # (3, 5, e, g)
    xG = np.moveaxis(mesh.xG[elems], 0, 1)                                        # (3, e, g)
    F = P.flux(uG, qG, C, x=xG)                                                   # (5, 3, e, g)
    s = P.source(uG, qG, xG, t, C)                                                # (5, e, g)
    Wd = mesh.W[None, :] * mesh.detJ[elems]
    # (F, grad phi_i): sum_g Wd sum_d F_cd sum_a dphi[g, a, i] Jinv[g, a, d]
    r = np.einsum("eg,cdeg,egad,gai->eci", Wd, F, mesh.Jinv[elems], mesh.dphi, optimize=True)
    r = r + np.einsum("eg,ceg,gi->eci", Wd, s, mesh.phi)
    fh = face_fluxes(mesh, u, q, elems, C)
    for f in range(6):
        r = r - np.einsum("f,ecf,fi->eci", mesh.wF, fh[:, f], mesh.phiF[f])
    return r


def jvp(mesh, u, v, t=0.0, elems=None, h=1e-30):
    """Exact J v by complex step: Im r(u + i h v) / h (Squire & Trapp 1998)."""
    uc = u.astype(np.complex128) + 1j * h * v
    return residual(mesh, uc, None, t, elems).imag / h


def mass_apply(mesh, v, elems=None):
    """(M v)_i = sum_j M_ij v_j with M_ij = (phi_i, phi_j) on each element."""
    elems = np.arange(mesh.n_elem) if elems is None else np.asarray(elems)
    Wd = mesh.W[None, :] * mesh.detJ[elems]
    vG = np.einsum("gj,ecj->ecg", mesh.phi, v[elems])
    return np.einsum("eg,ecg,gi->eci", Wd, vG, mesh.phi)


def mass_solve(mesh, v, elems=None):
    """M^{-1} v on each element: a dense solve with the element mass matrix (phi_i, phi_j)."""
    elems = np.arange(mesh.n_elem) if elems is None else np.asarray(elems)
    Wd = mesh.W[None, :] * mesh.detJ[elems]
    M = np.einsum("eg,gi,gj->eij", Wd, mesh.phi, mesh.phi)
    b = v[elems].transpose(0, 2, 1)                                   # (e, i, c)
    return np.ascontiguousarray(np.linalg.solve(M, b).transpose(0, 2, 1))
