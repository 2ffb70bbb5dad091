"""Reduced-basis (RB) preconditioner and initial guess of Sec. 3.2 (oracle; test infrastructure only).

Sec. 3.2 preconditions each Newton system J dU = -G (Eq. NewtonSolve) with a low-rank
approximation of the Jacobian built on the reduced-basis space W_n spanned by the last n_rb Newton
updates, and uses the same space for the initial guess of GMRES. The construction itself is left to
the paper's references; the reading taken here:

  * W is any basis of the RB space (its span is all that matters), Z = J W its image under the
    stage Jacobian J = J_G (n_rb Jacobian-vector products, matrix-free);
  * the approximate Jacobian is exact on the RB space and equal to a base operator P0 on its
    orthogonal complement:
        J~ = P0 + (Z - P0 W) (W^T W)^{-1} W^T,
    with P0 the element mass matrix M (nothing assembled) or the exact diagonal blocks of J_G
    (block-Jacobi);
  * GMRES is right-preconditioned with J~^{-1};
  * the initial guess is the RB least-squares solution x0 = W a, a = argmin ||b - Z a||_2;
  * the RB space is the last n_rb Newton updates over all Newton iterations, stages and steps
    (a rolling window); with no update yet, J~ = P0 and x0 = 0.

Here J~ is formed as a dense matrix and J~ y = x is solved directly (small meshes only).

Pinned by tests/test_oracle_rb.py: J~^{-1} maps J w to w for w in the RB space; for a space that
is the whole vector space J~^{-1} is J^{-1} of the brute-force Jacobian; on the complement J~ is
P0; the result depends on the span only; the initial guess leaves a residual orthogonal to Z and
is exact when b lies in the span of Z.
"""
import numpy as np

from . import dg as D
from . import solver as S


def approximate_jacobian(W, Z, P0):
    """Dense J~ = P0 + (Z - P0 W)(W^T W)^{-1} W^T; W, Z are (n, r), P0 is (n, n)."""
    if W.shape[1] == 0:
        return P0.copy()
    return P0 + (Z - P0 @ W) @ np.linalg.solve(W.T @ W, W.T)


def initial_guess(W, Z, b):
    """x0 = W a with a minimising ||b - Z a||_2 (zero for an empty space)."""
    if W.shape[1] == 0:
        return np.zeros_like(b)
    a = np.linalg.lstsq(Z, b, rcond=None)[0]
    return W @ a


def mass_matrix(mesh):
    """Dense block-diagonal element mass matrix on flat vectors [e][c][i]."""
    E, Np = mesh.n_elem, mesh.Np
    n = E * 5 * Np
    M = np.zeros((n, n))
    for j in range(5 * Np):
        v = np.zeros((E, 5, Np))
        v.reshape(E, -1)[:, j] = 1.0
        col = D.mass_apply(mesh, v).reshape(E, -1)
        for e in range(E):
            M[e * 5 * Np:(e + 1) * 5 * Np, e * 5 * Np + j] = col[e]
    return M


def block_jacobi_matrix(mesh, U, t, dt_aii):
    """Dense block-diagonal matrix of the exact diagonal blocks of J_G."""
    B = S.diagonal_blocks(mesh, U, t, dt_aii)
    E, nb = B.shape[0], B.shape[1]
    P = np.zeros((E * nb, E * nb))
    for e in range(E):
        P[e * nb:(e + 1) * nb, e * nb:(e + 1) * nb] = B[e]
    return P


def stage_jacobian_times(mesh, U, t, dt_aii, W):
    """Z = J_G W column by column (matrix-free products)."""
    mv = S.stage_operator(mesh, U, t, dt_aii)
    return np.stack([mv(W[:, j]) for j in range(W.shape[1])], axis=1) if W.shape[1] else np.zeros_like(W)


def implicit_step(mesh, u_n, t, dt, window, n_rb=8, base="mass", stages=3, tol=1e-8, gmres_tol=1e-3,
                  restart=30, stats=None):
    """One DIRK step with RB-preconditioned Newton-GMRES. `window` is a list of flat Newton updates
    (oldest first) carried across calls; it is updated in place."""
    A, b, c = S.dirk_tableau(stages)
    Mu = D.mass_apply(mesh, u_n)
    R = []
    U = u_n.copy()
    its_newton, its_gmres = [], []
    for i in range(stages):
        known = Mu + sum(dt * A[i, j] * R[j] for j in range(i)) if i else Mu.copy()
        ti, daii = t + c[i] * dt, dt * A[i, i]
        g0 = None
        gm = 0
        for it in range(26):
            G = D.mass_apply(mesh, U) - known - daii * D.residual(mesh, U, None, ti)
            gn = np.linalg.norm(G)
            g0 = gn if g0 is None else g0
            if gn <= tol * g0 or gn <= 1e-14 * np.linalg.norm(D.mass_apply(mesh, U)):
                break
            if it == 25:
                raise RuntimeError("Newton did not converge")
            W = np.stack(window[-n_rb:], axis=1) if window else np.zeros((U.size, 0))
            Z = stage_jacobian_times(mesh, U, ti, daii, W)
            P0 = mass_matrix(mesh) if base == "mass" else block_jacobi_matrix(mesh, U, ti, daii)
            Jt = approximate_jacobian(W, Z, P0)
            rhs = -G.ravel()
            x0 = initial_guess(W, Z, rhs)
            dU, k = S.gmres(S.stage_operator(mesh, U, ti, daii), rhs, x0=x0, restart=restart, tol=gmres_tol,
                            precond=lambda v, Jt=Jt: np.linalg.solve(Jt, v))
            gm += k
            window.append(dU.copy())
            del window[:-n_rb]
            U = U + dU.reshape(U.shape)
        its_newton.append(it)
        its_gmres.append(gm)
        R.append(D.residual(mesh, U, None, ti))
    if stats is not None:
        stats["newton"], stats["gmres"] = its_newton, its_gmres
    return U
