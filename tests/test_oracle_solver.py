"""Pins of the oracle's DIRK tableaux, GMRES, Newton stage solve and diagonal blocks."""
import math

import numpy as np
import pytest

from oracle import dg as D
from oracle import mesh as OM
from oracle import solver as S
from paper_2306_01085_gb300 import workloads as W


@pytest.mark.parametrize("s", [2, 3])
def test_dirk_order_conditions_and_l_stability(s):
    A, b, c = S.dirk_tableau(s)
    assert np.allclose(np.triu(A, 1), 0) and np.allclose(np.diag(A), A[0, 0])
    assert np.allclose(A[-1], b) and np.allclose(A.sum(1), c)
    conds = [b.sum() - 1, b @ c - 0.5]
    if s == 3:
        conds += [b @ c ** 2 - 1 / 3, b @ A @ c - 1 / 6]
    assert np.abs(conds).max() < 1e-14
    g = A[0, 0]
    if s == 2:
        assert abs(g - (1 - 1 / math.sqrt(2))) < 1e-15
    else:
        # Alexander's gamma is the root of x^3 - 3x^2 + 3x/2 - 1/6 in (1/3, 1/2)
        assert abs(g ** 3 - 3 * g ** 2 + 1.5 * g - 1 / 6) < 1e-14 and 1 / 3 < g < 0.5
    # stability function R(z) = 1 + z b^T (I - z A)^{-1} 1 vanishes at infinity (L-stable)
    z = -1e9
    R = 1 + z * b @ np.linalg.solve(np.eye(s) - z * A, np.ones(s))
    assert abs(R) < 1e-6


@pytest.mark.parametrize("s", [2, 3])
def test_dirk_observed_order_on_linear_ode(s):
    """u' = lambda u (scalar, mass 1): the error at T = 1 falls as dt^s."""
    A, b, c = S.dirk_tableau(s)
    lam = -1.3
    errs = []
    for n in (20, 40, 80):
        dt = 1.0 / n
        u = 1.0
        for _ in range(n):
            K = np.linalg.solve(np.eye(s) - dt * lam * A, lam * u * np.ones(s))
            u = u + dt * b @ K
        errs.append(abs(u - math.exp(lam)))
    rate = math.log2(errs[1] / errs[2])
    assert abs(rate - s) < 0.1, errs


def test_gmres_matches_dense_solve():
    rng = np.random.default_rng(3)
    n = 80
    A = np.eye(n) * 2 + rng.standard_normal((n, n)) / math.sqrt(n)
    x_true = rng.standard_normal(n)
    b = A @ x_true
    x, its = S.gmres(lambda v: A @ v, b, restart=30, tol=1e-12, max_restarts=50)
    assert np.linalg.norm(x - x_true) < 1e-9 * np.linalg.norm(x_true)
    # right preconditioning by the exact inverse converges in one iteration
    Ainv = np.linalg.inv(A)
    x, its = S.gmres(lambda v: A @ v, b, restart=30, tol=1e-12, precond=lambda v: Ainv @ v)
    assert its <= 2 and np.linalg.norm(x - x_true) < 1e-9 * np.linalg.norm(x_true)


def _tiny():
    d = W.box_desc(p=1, n=2, bc_lo=W.BC_WALL, bc_hi=W.BC_OUTFLOW, visc_exp=0.69, re=30.0)
    m = OM.OracleMesh(d)
    u = W.box_state(m.X, seed=4, amp=0.02)
    return d, m, u


def test_newton_stage_matches_dense_newton():
    """Newton-GMRES (tight tolerances) and Newton with the dense complex-step Jacobian reach the
    same stage solution."""
    d, m, u = _tiny()
    dt_aii = 0.05
    known = D.mass_apply(m, u)
    U1, its = S.newton_stage(m, u, known, 0.0, dt_aii, tol=1e-12, gmres_tol=1e-10, restart=60)
    Mmat = np.zeros((u.size, u.size))
    for j in range(u.size):
        e = np.zeros(u.size)
        e[j] = 1
        Mmat[:, j] = D.mass_apply(m, e.reshape(u.shape)).ravel()
    U = u.copy()
    for _ in range(10):
        G = D.mass_apply(m, U) - known - dt_aii * D.residual(m, U)
        J = Mmat - dt_aii * S.jacobian_columns(m, U, 0.0)
        U = U - np.linalg.solve(J, G.ravel()).reshape(U.shape)
    assert np.abs(U1 - U).max() < 1e-10 * np.abs(U).max()
    assert its <= 6


def test_diagonal_blocks_match_full_jacobian():
    d, m, u = _tiny()
    dt_aii = 0.1
    B = S.diagonal_blocks(m, u, 0.0, dt_aii)
    n = 5 * m.Np
    J = S.jacobian_columns(m, u, 0.0)
    Mmat = np.zeros_like(J)
    for j in range(u.size):
        e = np.zeros(u.size)
        e[j] = 1
        Mmat[:, j] = D.mass_apply(m, e.reshape(u.shape)).ravel()
    JG = Mmat - dt_aii * J
    for e in range(m.n_elem):
        sl = slice(e * n, (e + 1) * n)
        assert np.abs(B[e] - JG[sl, sl]).max() < 1e-13 * np.abs(JG).max()
    # the neighbour-lifting path makes the exact block differ from the block with q frozen
    assert np.abs(JG[:n, n:]).max() > 0


def test_implicit_step_reduces_to_stage_equations():
    """The DIRK step with a tight Newton tolerance satisfies every stage equation."""
    d, m, u = _tiny()
    stats = {}
    dt = 0.05
    u1 = S.implicit_step(m, u, 0.0, dt, stages=2, tol=1e-11, gmres_tol=1e-9, restart=40, stats=stats)
    A, b, c = S.dirk_tableau(2)
    # recompute the stage values from u1 backwards is not possible; check the last stage instead:
    # M (u1 - u_n) = dt (a21 r(U1) + a22 r(u1)) with U1 solving stage 1
    known = D.mass_apply(m, u)
    U1, _ = S.newton_stage(m, u, known, c[0] * dt, dt * A[0, 0], tol=1e-11, gmres_tol=1e-9, restart=40)
    lhs = D.mass_apply(m, u1 - u)
    rhs = dt * (A[1, 0] * D.residual(m, U1, None, c[0] * dt) + A[1, 1] * D.residual(m, u1, None, c[1] * dt))
    assert np.abs(lhs - rhs).max() < 1e-9 * np.abs(lhs).max()
    assert len(stats["newton"]) == 2
