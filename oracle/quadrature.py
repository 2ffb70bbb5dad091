"""1D quadrature rules and Lagrange bases (oracle; test infrastructure only).

The discrete spaces W_h, Q_h of Sec. 3.1 hold polynomials of degree k on each element. They are
represented here by the tensor-product Lagrange basis on Gauss-Lobatto-Legendre (GLL) nodes, and
integrals are taken with the tensor-product Gauss-Legendre rule of k+1 points per direction.

Pinned by tests/test_oracle_quadrature.py: closed forms for k = 2, exactness on monomials,
Lagrange interpolation reproducing polynomials.
"""
import numpy as np
from numpy.polynomial import legendre as L


def gauss(n):
    """n-point Gauss-Legendre points and weights on [-1, 1] (library routine)."""
    x, w = L.leggauss(n)
    return np.asarray(x, dtype=np.float64), np.asarray(w, dtype=np.float64)


def gll(n):
    """n-point Gauss-Lobatto-Legendre points and weights on [-1, 1].

    Interior points are the roots of P'_{n-1}; weights 2 / (n (n-1) P_{n-1}(x)^2).
    """
    if n < 2:
        raise ValueError("GLL needs at least two points")
    N = n - 1
    c = np.zeros(N + 1)
    c[N] = 1.0
    inner = L.legroots(L.legder(c)) if N > 1 else np.array([])
    x = np.concatenate([[-1.0], np.sort(np.real(inner)), [1.0]])
    w = 2.0 / (N * (N + 1) * L.legval(x, c) ** 2)
    return x, w


def lagrange(nodes, x):
    """Matrix V[j, i] = l_i(x_j) of the Lagrange basis on `nodes` evaluated at points x."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = nodes.size
    V = np.ones((x.size, n))
    for i in range(n):
        for k in range(n):
            if k != i:
                V[:, i] *= (x - nodes[k]) / (nodes[i] - nodes[k])
    return V


def lagrange_deriv(nodes, x):
    """Matrix D[j, i] = l_i'(x_j): derivative of the product formula term by term."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = nodes.size
    D = np.zeros((x.size, n))
    for i in range(n):
        for k in range(n):
            if k == i:
                continue
            term = np.full(x.size, 1.0 / (nodes[i] - nodes[k]))
            for m in range(n):
                if m != i and m != k:
                    term *= (x - nodes[m]) / (nodes[i] - nodes[m])
            D[:, i] += term
    return D


def basis3d(nodes1d, pts):
    """Tensor-product nodal basis phi_i(xi) = l_a(xi_1) l_b(xi_2) l_c(xi_3), node i = a + n b + n^2 c.

    pts: (m, 3) reference points. Returns phi (m, n^3) and dphi (m, 3, n^3) with
    dphi[:, e, i] = d phi_i / d xi_e.
    """
    pts = np.asarray(pts, dtype=np.float64)
    n = len(nodes1d)
    V = [lagrange(nodes1d, pts[:, e]) for e in range(3)]
    D = [lagrange_deriv(nodes1d, pts[:, e]) for e in range(3)]
    # phi[m, c, b, a] = V3[m, c] V2[m, b] V1[m, a]  -> flattened index a + n b + n^2 c
    phi = np.einsum("mc,mb,ma->mcba", V[2], V[1], V[0]).reshape(-1, n ** 3)
    d1 = np.einsum("mc,mb,ma->mcba", V[2], V[1], D[0]).reshape(-1, n ** 3)
    d2 = np.einsum("mc,mb,ma->mcba", V[2], D[1], V[0]).reshape(-1, n ** 3)
    d3 = np.einsum("mc,mb,ma->mcba", D[2], V[1], V[0]).reshape(-1, n ** 3)
    return phi, np.stack([d1, d2, d3], axis=1)


def tensor_points(x1d):
    """All points (x_a, x_b, x_c) with flattened index a + n b + n^2 c, shape (n^3, 3)."""
    n = len(x1d)
    c, b, a = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    return np.stack([x1d[a.ravel()], x1d[b.ravel()], x1d[c.ravel()]], axis=1)


# Local faces of the reference hexahedron: (axis, side). Face parameters (s, t) are the two other
# reference coordinates in increasing axis order; face point index = i_s + n i_t.
FACES = [(0, -1.0), (0, 1.0), (1, -1.0), (1, 1.0), (2, -1.0), (2, 1.0)]


def face_points(x1d, face):
    """Reference coordinates (n^2, 3) of the tensor points of x1d on local face `face`."""
    axis, side = FACES[face]
    n = len(x1d)
    it, is_ = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    s = x1d[is_.ravel()]
    t = x1d[it.ravel()]
    others = [a for a in range(3) if a != axis]
    pts = np.zeros((n * n, 3))
    pts[:, axis] = side
    pts[:, others[0]] = s
    pts[:, others[1]] = t
    return pts
