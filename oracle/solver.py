"""Implicit time step of the semi-discrete system (oracle; test infrastructure only).

Sec. 3.1 integrates M du/dt = r(u) with diagonally implicit Runge-Kutta schemes (Alexander 1977);
Sec. 3.2 solves every stage by Newton's method, Eq. NewtonSolve, each Newton system by GMRES, and
needs only Jacobian-vector products. Stage i of an s-stage DIRK:

    M (U_i - u_n) = dt sum_{j <= i} a_ij r(U_j),      u_{n+1} = U_s (stiffly accurate),

so the Newton residual is G(U) = M (U - u_n) - dt sum_{j<i} a_ij r(U_j) - dt a_ii r(U) and its
Jacobian J_G v = M v - dt a_ii J_r v.

Readings of the paper taken here: Newton stops when ||G||_2 <= tol ||G(U^0)||_2 with U^0 the previous
stage value (absolute floor 1e-14 ||M U||_2); GMRES(restart) solves each Newton system to a
fixed relative tolerance eta; the block-Jacobi blocks are the exact diagonal blocks of J_G.

Parity pinned by tests/test_oracle_solver.py: the order conditions and observed orders of the
tableaux, GMRES against a dense solve, Newton against a dense-Jacobian Newton, diagonal blocks
against the full brute-force Jacobian.
"""
import math

import numpy as np

from . import dg as D


def dirk_tableau(stages):
    """Lower-triangular A, weights b, nodes c of the L-stable stiffly accurate DIRK with equal
    diagonal gamma, found from the order conditions (order = stages, stages in {2, 3}).

    2 stages: b = (1 - g, g), c = (g, 1); order 2 needs b.c = 1/2, i.e. g^2 - 2 g + 1/2 = 0,
              root g = 1 - 1/sqrt(2) in (0, 1).
    3 stages: unknowns g, a21, b1, b2 (c = (g, a21 + g, 1), b3 = g, last row of A = b) from
              b.1 = 1, b.c = 1/2, b.c^2 = 1/3, b.A.c = 1/6 by Newton's method; the L-stable root has
              g in (1/3, 1/2).
    """
    if stages == 1:
        return np.array([[1.0]]), np.array([1.0]), np.array([1.0])
    if stages == 2:
        g = 1.0 - 1.0 / math.sqrt(2.0)
        A = np.array([[g, 0.0], [1.0 - g, g]])
        return A, A[-1].copy(), A.sum(1)
    if stages != 3:
        raise ValueError("stages must be 1, 2 or 3")

    def build(x):
        g, a21, b1, b2 = x
        A = np.array([[g, 0, 0], [a21, g, 0], [b1, b2, g]])
        return A, A[-1], A.sum(1)

    def conditions(x):
        A, b, c = build(x)
        return np.array([b.sum() - 1, b @ c - 0.5, b @ c ** 2 - 1 / 3, b @ A @ c - 1 / 6])

    x = np.array([0.44, 0.28, 1.2, -0.64])
    for _ in range(50):
        f = conditions(x)
        J = np.zeros((4, 4))
        for k in range(4):
            e = np.zeros(4)
            e[k] = 1e-7
            J[:, k] = (conditions(x + e) - conditions(x - e)) / 2e-7
        dx = np.linalg.solve(J, -f)
        x = x + dx
        if np.abs(dx).max() < 1e-15:
            break
    A, b, c = build(x)
    return A, b.copy(), c


def gmres(matvec, rhs, x0=None, restart=30, tol=1e-3, max_restarts=10, precond=None):
    """Right-preconditioned restarted GMRES (Saad & Schultz 1986): solves A x = rhs to
    ||rhs - A x|| <= tol ||rhs||. Arnoldi by modified Gram-Schmidt, Givens rotations.
    Returns x and the total number of iterations."""
    n = rhs.size
    P = precond if precond is not None else (lambda v: v)
    x = np.zeros(n) if x0 is None else x0.copy()
    bnorm = np.linalg.norm(rhs)
    if bnorm == 0:
        return x, 0
    its = 0
    for _ in range(max_restarts):
        r = rhs - matvec(x)
        beta = np.linalg.norm(r)
        if beta <= tol * bnorm:
            return x, its
        V = np.zeros((restart + 1, n))
        H = np.zeros((restart + 1, restart))
        cs, sn = np.zeros(restart), np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        V[0] = r / beta
        k_done = 0
        for k in range(restart):
            w = matvec(P(V[k]))
            for j in range(k + 1):
                H[j, k] = np.dot(V[j], w)
                w = w - H[j, k] * V[j]
            H[k + 1, k] = np.linalg.norm(w)
            if H[k + 1, k] > 0:
                V[k + 1] = w / H[k + 1, k]
            for j in range(k):
                t = cs[j] * H[j, k] + sn[j] * H[j + 1, k]
                H[j + 1, k] = -sn[j] * H[j, k] + cs[j] * H[j + 1, k]
                H[j, k] = t
            den = math.hypot(H[k, k], H[k + 1, k])
            cs[k], sn[k] = H[k, k] / den, H[k + 1, k] / den
            H[k, k] = den
            H[k + 1, k] = 0.0
            g[k + 1] = -sn[k] * g[k]
            g[k] = cs[k] * g[k]
            its += 1
            k_done = k + 1
            if abs(g[k + 1]) <= tol * bnorm:
                break
        y = np.linalg.solve(np.triu(H[:k_done, :k_done]), g[:k_done])
        x = x + P(V[:k_done].T @ y)
        if abs(g[k_done]) <= tol * bnorm:
            r = rhs - matvec(x)
            if np.linalg.norm(r) <= tol * bnorm * 1.0000001 + 1e-300:
                return x, its
    raise RuntimeError("GMRES did not converge")


def stage_operator(mesh, U, t, dt_aii):
    """v -> J_G v = M v - dt a_ii J_r(U) v on flat vectors."""
    shape = U.shape

    def mv(v):
        v = v.reshape(shape)
        return (D.mass_apply(mesh, v) - dt_aii * D.jvp(mesh, U, v, t)).ravel()
    return mv


def newton_stage(mesh, U0, known, t, dt_aii, tol=1e-8, gmres_tol=1e-3, restart=30, max_newton=25,
                 precond_builder=None, history=None):
    """Solve G(U) = M U - known - dt a_ii r(U, t) = 0 by Newton-GMRES from U0."""
    U = U0.copy()
    g0 = None
    for it in range(max_newton + 1):
        G = D.mass_apply(mesh, U) - known - dt_aii * D.residual(mesh, U, None, t)
        gn = np.linalg.norm(G)
        if history is not None:
            history.append(gn)
        if g0 is None:
            g0 = gn
        floor = 1e-14 * np.linalg.norm(D.mass_apply(mesh, U))
        if gn <= tol * g0 or gn <= floor:
            return U, it
        P = precond_builder(U) if precond_builder else None
        dU, _ = gmres(stage_operator(mesh, U, t, dt_aii), -G.ravel(), restart=restart, tol=gmres_tol, precond=P)
        U = U + dU.reshape(U.shape)
    raise RuntimeError("Newton did not converge")


def implicit_step(mesh, u_n, t, dt, stages=3, tol=1e-8, gmres_tol=1e-3, restart=30, precond_builder=None,
                  stats=None):
    """One DIRK step u_n -> u_{n+1} of M du/dt = r(u) with Newton-GMRES on every stage."""
    A, b, c = dirk_tableau(stages)
    Mu = D.mass_apply(mesh, u_n)
    R = []
    U = u_n.copy()
    newton_its = []
    for i in range(stages):
        known = Mu + sum(dt * A[i, j] * R[j] for j in range(i)) if i else Mu.copy()
        ti = t + c[i] * dt
        pb = (lambda Uc, ti=ti, daii=dt * A[i, i]: precond_builder(Uc, ti, daii)) if precond_builder else None
        U, its = newton_stage(mesh, U, known, ti, dt * A[i, i], tol, gmres_tol, restart, precond_builder=pb)
        newton_its.append(its)
        R.append(D.residual(mesh, U, None, ti))
    if stats is not None:
        stats["newton"] = newton_its
    return U


def jacobian_columns(mesh, U, t, h=1e-30):
    """Full Jacobian of the residual by complex-step columns (tiny meshes only)."""
    n = U.size
    J = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        J[:, j] = D.jvp(mesh, U, e.reshape(U.shape), t, h=h).ravel()
    return J


def diagonal_blocks(mesh, U, t, dt_aii, elems=None):
    """Exact element diagonal blocks of J_G = M - dt a_ii J_r: B[e] is (5 Np x 5 Np) in the
    element's [var][node] ordering. Column j of B[e] is (J_G e_{e,j}) restricted to element e,
    computed on e and the elements its residual depends on. elems: the blocks to build (all by
    default); B[k] is then the block of elems[k]."""
    E, Np = mesh.n_elem, mesh.Np
    n = 5 * Np
    elems = list(range(E)) if elems is None else list(elems)
    B = np.zeros((len(elems), n, n))
    for k, e in enumerate(elems):
        for j in range(n):
            v = np.zeros_like(U)
            v[e].flat[j] = 1.0
            col = D.mass_apply(mesh, v, elems=[e])[0] - dt_aii * D.jvp(mesh, U, v, t, elems=[e])[0]
            B[k][:, j] = col.ravel()
    return B
