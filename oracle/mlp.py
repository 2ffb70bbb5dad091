"""Learned element preconditioner: network, loss and gradients (oracle; test infrastructure only).

The paper has no learned component; this is the library's learned right preconditioner. Per
element, a multilayer perceptron with two hidden layers and SiLU activations maps element features
x to o = W3 s(W2 s(W1 x + b1) + b2) + b3, s(z) = z / (1 + e^{-z}), read as

    D = 1 + o[:n],  U = o[n : n + n r] (n x r, row-major),  V = o[n + n r :] (n x r)

and P = diag(D) + U V^T approximates the inverse of the element's scaled diagonal block
Bs = S^{-1/2} B S^{-1/2} (S = diagonal of the element mass matrix). The loss of a batch of
samples (x_b, Bs_b) is

    L = (1 / nb) sum_b || Bs_b P_b - I ||_F^2 / n,

the residual of P as a RIGHT inverse, because GMRES is right-preconditioned: its operator is
J P, whose diagonal blocks are B P. Gradients (written out from the chain rule, no automatic
differentiation): with R = Bs P - I and G = dL/dP = (2 / (nb n)) Bs^T R,
    dL/dD = diag(G),  dL/dU = G V,  dL/dV = G^T U,
then back through the linear and SiLU layers, with s'(z) = sigma(z) (1 + z (1 - sigma(z))) and
sigma the logistic function.

Pinned by tests/test_oracle_mlp.py: gradients against central differences of the loss, the
identity case (zero output layer: P = I), the closed form of the loss for a diagonal block.
"""
import numpy as np


def shapes(n_in, hidden, n, rank):
    n_out = n + 2 * n * rank
    return [("W1", (hidden, n_in)), ("b1", (hidden,)), ("W2", (hidden, hidden)), ("b2", (hidden,)),
            ("W3", (n_out, hidden)), ("b3", (n_out,))]


def unpack(flat, n_in, hidden, n, rank):
    out, off = {}, 0
    for name, shp in shapes(n_in, hidden, n, rank):
        size = int(np.prod(shp))
        out[name] = flat[off:off + size].reshape(shp)
        off += size
    return out


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def silu(z):
    return z * sigmoid(z)


def silu_grad(z):
    s = sigmoid(z)
    return s * (1.0 + z * (1.0 - s))


def forward(p, X):
    z1 = X @ p["W1"].T + p["b1"]
    h1 = silu(z1)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = silu(z2)
    o = h2 @ p["W3"].T + p["b3"]
    return o, (z1, h1, z2, h2)


def split(o, n, rank):
    nb = o.shape[0]
    D = 1.0 + o[:, :n]
    U = o[:, n:n + n * rank].reshape(nb, n, rank)
    V = o[:, n + n * rank:].reshape(nb, n, rank)
    return D, U, V


def apply_inverse(D, U, V):
    """P = diag(D) + U V^T as dense matrices (nb, n, n)."""
    return np.einsum("bi,ij->bij", D, np.eye(D.shape[1])) + np.einsum("bir,bjr->bij", U, V)


def loss(p, X, Bs, n, rank):
    o, _ = forward(p, X)
    D, U, V = split(o, n, rank)
    R = Bs @ apply_inverse(D, U, V) - np.eye(n)[None]
    return float((R ** 2).sum() / (X.shape[0] * n))


def loss_and_grads(p, X, Bs, n, rank):
    nb = X.shape[0]
    o, (z1, h1, z2, h2) = forward(p, X)
    D, U, V = split(o, n, rank)
    R = Bs @ apply_inverse(D, U, V) - np.eye(n)[None]
    L = float((R ** 2).sum() / (nb * n))
    G = (2.0 / (nb * n)) * np.transpose(Bs, (0, 2, 1)) @ R
    dD = np.einsum("bii->bi", G)
    dU = G @ V
    dV = np.transpose(G, (0, 2, 1)) @ U
    do = np.concatenate([dD, dU.reshape(nb, -1), dV.reshape(nb, -1)], axis=1)
    g = {}
    g["W3"] = do.T @ h2
    g["b3"] = do.sum(0)
    dz2 = (do @ p["W3"]) * silu_grad(z2)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(0)
    dz1 = (dz2 @ p["W2"]) * silu_grad(z1)
    g["W1"] = dz1.T @ X
    g["b1"] = dz1.sum(0)
    return L, g


def flatten(g, n_in, hidden, n, rank):
    return np.concatenate([g[name].ravel() for name, _ in shapes(n_in, hidden, n, rank)])
