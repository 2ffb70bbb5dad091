"""Pins of the oracle's quadrature rules and Lagrange bases against closed forms and exactness."""
import math

import numpy as np
import pytest

from oracle import quadrature as Q


def test_gauss_closed_form_three_points():
    x, w = Q.gauss(3)
    assert np.allclose(x, [-math.sqrt(0.6), 0.0, math.sqrt(0.6)], atol=1e-15)
    assert np.allclose(w, [5 / 9, 8 / 9, 5 / 9], atol=1e-15)


def test_gll_closed_forms():
    x, w = Q.gll(3)
    assert np.allclose(x, [-1, 0, 1], atol=1e-15) and np.allclose(w, [1 / 3, 4 / 3, 1 / 3], atol=1e-15)
    x, w = Q.gll(4)
    a = 1 / math.sqrt(5)
    assert np.allclose(x, [-1, -a, a, 1], atol=1e-15)
    assert np.allclose(w, [1 / 6, 5 / 6, 5 / 6, 1 / 6], atol=1e-15)
    x, w = Q.gll(5)
    b = math.sqrt(3 / 7)
    assert np.allclose(x, [-1, -b, 0, b, 1], atol=1e-15)
    assert np.allclose(w, [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10], atol=1e-15)


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6])
def test_exactness_on_monomials(n):
    xg, wg = Q.gauss(n)
    for k in range(2 * n):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(wg, xg ** k) - exact) < 1e-14
    xl, wl = Q.gll(n)
    for k in range(2 * n - 2):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(wl, xl ** k) - exact) < 1e-14


@pytest.mark.parametrize("n", [2, 3, 5])
def test_lagrange_reproduces_polynomials(n):
    nodes, _ = Q.gll(n)
    x = np.linspace(-1, 1, 17)
    V = Q.lagrange(nodes, x)
    D = Q.lagrange_deriv(nodes, x)
    for k in range(n):
        assert np.allclose(V @ nodes ** k, x ** k, atol=1e-13)
        dk = k * x ** (k - 1) if k > 0 else 0 * x
        assert np.allclose(D @ nodes ** k, dk, atol=1e-12)


def test_basis3d_partition_of_unity_and_derivative():
    nodes, _ = Q.gll(4)
    pts = np.array([[0.1, -0.3, 0.7], [1.0, 0.2, -1.0], [0.0, 0.0, 0.0]])
    phi, dphi = Q.basis3d(nodes, pts)
    assert np.allclose(phi.sum(1), 1.0, atol=1e-14)
    assert np.allclose(dphi.sum(2), 0.0, atol=1e-12)
    # f = x^2 y z^3 sampled at nodes
    P = Q.tensor_points(nodes)
    f = P[:, 0] ** 2 * P[:, 1] * P[:, 2] ** 3
    assert np.allclose(phi @ f, pts[:, 0] ** 2 * pts[:, 1] * pts[:, 2] ** 3, atol=1e-13)
    assert np.allclose(dphi[:, 0] @ f, 2 * pts[:, 0] * pts[:, 1] * pts[:, 2] ** 3, atol=1e-12)
    assert np.allclose(dphi[:, 2] @ f, 3 * pts[:, 0] ** 2 * pts[:, 1] * pts[:, 2] ** 2, atol=1e-12)
