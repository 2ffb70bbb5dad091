"""Pins of the oracle's reduced-basis preconditioner and initial guess (Sec. 3.2)."""
import numpy as np
import pytest

from oracle import dg as OD
from oracle import mesh as OM
from oracle import rb as RB
from oracle import solver as OS
from paper_2306_01085_gb300 import workloads as W


@pytest.fixture(scope="module")
def problem():
    d = W.box_desc(p=1, n=2, bc_lo=W.BC_WALL, bc_hi=W.BC_OUTFLOW, visc_exp=0.69, re=30.0)
    om = OM.OracleMesh(d)
    U = W.state_for(d, om.X, 4)
    t, c = 0.0, 0.2
    n = U.size
    M = RB.mass_matrix(om)
    JG = M - c * OS.jacobian_columns(om, U, t)
    return om, U, t, c, n, M, JG


def _rand(seed, shape):
    return W.unit_vector(seed, shape) * np.sqrt(np.prod(shape))


def test_mass_matrix_matches_mass_apply(problem):
    om, U, t, c, n, M, JG = problem
    v = _rand(3, U.shape)
    assert np.allclose(M @ v.ravel(), OD.mass_apply(om, v).ravel(), rtol=0, atol=1e-14 * np.abs(M).max() * 10)


def test_exact_on_the_reduced_space(problem):
    """J~^{-1} (J w) = w for every w in the RB space, with a non-orthonormal basis."""
    om, U, t, c, n, M, JG = problem
    Wb = _rand(5, (n, 4)) + 0.5 * _rand(6, (n, 1))          # correlated columns
    Z = RB.stage_jacobian_times(om, U, t, c, Wb)
    assert np.allclose(Z, JG @ Wb, rtol=0, atol=1e-12 * np.abs(Z).max())
    Jt = RB.approximate_jacobian(Wb, Z, M)
    a = np.array([0.3, -1.0, 2.0, 0.7])
    y = np.linalg.solve(Jt, Z @ a)
    assert np.abs(y - Wb @ a).max() <= 1e-9 * np.abs(Wb @ a).max()


def test_whole_space_gives_the_jacobian(problem):
    """With a basis of the whole space the approximation is the brute-force Jacobian itself."""
    om, U, t, c, n, M, JG = problem
    Wb = _rand(7, (n, n))
    Z = JG @ Wb
    Jt = RB.approximate_jacobian(Wb, Z, M)
    assert np.abs(Jt - JG).max() <= 1e-9 * np.abs(JG).max()


def test_base_operator_on_the_complement(problem):
    om, U, t, c, n, M, JG = problem
    Wb = _rand(8, (n, 3))
    Z = JG @ Wb
    x = _rand(9, (n,))
    x = x - Wb @ np.linalg.solve(Wb.T @ Wb, Wb.T @ x)          # W^T x = 0
    for P0 in (M, RB.block_jacobi_matrix(om, U, t, c)):
        Jt = RB.approximate_jacobian(Wb, Z, P0)
        assert np.abs(Jt @ x - P0 @ x).max() <= 1e-11 * np.abs(P0 @ x).max()


def test_depends_on_the_span_only(problem):
    om, U, t, c, n, M, JG = problem
    Wb = _rand(10, (n, 3))
    Smix = np.array([[2.0, 0.1, -1.0], [0.0, 1.0, 0.5], [0.3, 0.0, 1.5]])
    J1 = RB.approximate_jacobian(Wb, JG @ Wb, M)
    J2 = RB.approximate_jacobian(Wb @ Smix, JG @ Wb @ Smix, M)
    assert np.abs(J1 - J2).max() <= 1e-10 * np.abs(J1).max()
    b = _rand(11, (n,))
    x1 = RB.initial_guess(Wb, JG @ Wb, b)
    x2 = RB.initial_guess(Wb @ Smix, JG @ Wb @ Smix, b)
    assert np.abs(x1 - x2).max() <= 1e-10 * np.abs(x1).max()


def test_initial_guess_is_the_least_squares_solution(problem):
    om, U, t, c, n, M, JG = problem
    Wb = _rand(12, (n, 5))
    Z = JG @ Wb
    b = _rand(13, (n,))
    x0 = RB.initial_guess(Wb, Z, b)
    a = np.linalg.solve(Wb.T @ Wb, Wb.T @ x0)
    r = b - Z @ a
    assert np.abs(Z.T @ r).max() <= 1e-10 * np.abs(Z).max() * np.abs(b).max() * np.sqrt(n)
    assert np.linalg.norm(r) < np.linalg.norm(b)
    astar = np.array([1.0, -2.0, 0.5, 0.0, 3.0])
    xs = RB.initial_guess(Wb, Z, Z @ astar)
    assert np.abs(xs - Wb @ astar).max() <= 1e-9 * np.abs(Wb @ astar).max()
    assert np.all(RB.initial_guess(np.zeros((n, 0)), np.zeros((n, 0)), b) == 0)


@pytest.mark.parametrize("base", ["mass", "bj"])
def test_rb_implicit_step_reaches_the_plain_step(problem, base):
    """The preconditioner changes only the Krylov iterations: two RB-preconditioned steps reach the
    plain (unpreconditioned) oracle steps to the Newton tolerance, and the rolling window holds the
    last updates."""
    om, U, t, c, n, M, JG = problem
    dt = 0.05
    ref = OS.implicit_step(om, U, 0.0, dt, stages=2, tol=1e-12, gmres_tol=1e-10, restart=40)
    ref = OS.implicit_step(om, ref, dt, dt, stages=2, tol=1e-12, gmres_tol=1e-10, restart=40)
    window = []
    st = {}
    u1 = RB.implicit_step(om, U, 0.0, dt, window, n_rb=4, base=base, stages=2, tol=1e-12, gmres_tol=1e-10,
                          restart=40)
    u2 = RB.implicit_step(om, u1, dt, dt, window, n_rb=4, base=base, stages=2, tol=1e-12, gmres_tol=1e-10,
                          restart=40, stats=st)
    assert np.abs(u2 - ref).max() <= 1e-9 * np.abs(ref).max()
    assert len(window) == 4
    assert all(k > 0 for k in st["gmres"])
