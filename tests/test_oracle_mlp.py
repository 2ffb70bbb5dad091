"""Pins of the oracle's learned-preconditioner network: loss and hand-written gradients."""
import numpy as np
import pytest

from oracle import mlp as M


def _setup(seed=0, n_in=11, hidden=7, n=6, rank=2, nb=3):
    rng = np.random.default_rng(seed)
    flat = rng.standard_normal(sum(int(np.prod(s)) for _, s in M.shapes(n_in, hidden, n, rank))) * 0.3
    X = rng.standard_normal((nb, n_in))
    Bs = np.eye(n)[None] + 0.3 * rng.standard_normal((nb, n, n))
    return flat, X, Bs, (n_in, hidden, n, rank)


def test_gradients_match_central_differences():
    flat, X, Bs, dims = _setup()
    n_in, hidden, n, rank = dims
    p = M.unpack(flat, *dims)
    L, g = M.loss_and_grads(p, X, Bs, n, rank)
    gflat = M.flatten(g, *dims)
    h = 1e-6
    rng = np.random.default_rng(1)
    for k in rng.choice(flat.size, 60, replace=False):
        e = np.zeros_like(flat)
        e[k] = h
        fd = (M.loss(M.unpack(flat + e, *dims), X, Bs, n, rank) - M.loss(M.unpack(flat - e, *dims), X, Bs, n, rank)) / (2 * h)
        assert abs(fd - gflat[k]) <= 1e-7 * max(1.0, abs(fd)), (k, fd, gflat[k])
    assert abs(L - M.loss(p, X, Bs, n, rank)) < 1e-14


def test_zero_output_layer_is_the_identity_preconditioner():
    flat, X, Bs, dims = _setup()
    n_in, hidden, n, rank = dims
    p = M.unpack(flat.copy(), *dims)
    p["W3"][:] = 0.0
    p["b3"][:] = 0.0
    expect = ((Bs - np.eye(n)[None]) ** 2).sum() / (X.shape[0] * n)
    assert abs(M.loss(p, X, Bs, n, rank) - expect) < 1e-13


def test_exact_inverse_of_a_diagonal_block_gives_zero_loss():
    """A diagonal block diag(b) is inverted exactly by D = 1/b, U = V = 0 (output bias only)."""
    n_in, hidden, n, rank = 4, 5, 6, 2
    flat = np.zeros(sum(int(np.prod(s)) for _, s in M.shapes(n_in, hidden, n, rank)))
    p = M.unpack(flat, n_in, hidden, n, rank)
    b = np.linspace(0.5, 2.0, n)
    p["b3"][:n] = 1.0 / b - 1.0
    X = np.ones((2, n_in))
    Bs = np.stack([np.diag(b)] * 2)
    assert M.loss(p, X, Bs, n, rank) < 1e-28
    assert np.allclose(M.silu_grad(np.array([0.0])), 0.5)
