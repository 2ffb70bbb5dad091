"""The digit slicing that the tensor-core interpolation (DG_INTERP_TC) uses, restated in numpy and
checked against exact arithmetic: operator rows and data columns scaled to 53-bit integers and
written as seven balanced digits (six base-256 digits in [-128, 128] under a leading one of at most
33); the digit products of levels 0..7 summed per level; the levels combined in 64-bit integers
and rounded once. Pins: every digit is exact in FP16 (|d| <= 2048), every level sum stays below
2^24 (exact in the FP32 accumulators of the MMA), and the result is within 3e-15 of the largest
data value of its column, for the interpolation operator at p = 1..4 and random columns spanning
ten decades. A planted mistake (a dropped level) is caught."""
import math
from fractions import Fraction

import numpy as np
import pytest

L, LEVELS = 7, 8


def _lagrange(x, t):
    return np.array([np.prod([(t - x[m]) / (x[k] - x[m]) for m in range(len(x)) if m != k]) for k in range(len(x))])


def _operator(N):
    """Gauss values (B x B x B) and the six face traces, from the GLL nodes (numpy's own rules)."""
    eta, _ = np.polynomial.legendre.leggauss(N)
    c = np.zeros(N)
    c[-1] = 1.0
    xi = np.concatenate([[-1.0], np.sort(np.polynomial.legendre.Legendre(c).deriv().roots().real), [1.0]])
    B = np.array([_lagrange(xi, e) for e in eta])
    A3 = np.einsum("ia,jb,kc->kjicba", B, B, B).reshape(N ** 3, N ** 3)
    eL, eR = _lagrange(eta, -1.0), _lagrange(eta, 1.0)
    F = np.zeros((6 * N * N, N ** 3))
    for phi in range(6):
        ax, ev = phi >> 1, (eR if phi & 1 else eL)
        for f in range(N * N):
            s, t = f % N, f // N
            for j in range(N):
                i0 = j if ax == 0 else s
                i1 = s if ax == 0 else (j if ax == 1 else t)
                i2 = j if ax == 2 else t
                F[phi * N * N + f] += ev[j] * A3[i0 + N * (i1 + N * i2)]
    return np.vstack([A3, F])


def _digits(X):
    d = []
    X = X.copy()
    for _ in range(L - 1):
        lo = X & 0xFF
        lo = np.where(lo >= 128, lo - 256, lo)
        d.append(lo)
        X = (X - lo) >> 8
    d.append(X)
    return np.array(d[::-1])          # d[0] most significant


def _sliced_product(A, X, levels=LEVELS):
    fr = np.array([max(math.frexp(a)[1] for a in row if a != 0) for row in A])
    ec = np.array([max(math.frexp(x)[1] for x in col if x != 0) for col in X.T])
    Af = np.array([[int(np.rint(math.ldexp(a, int(53 - fr[r])))) for a in A[r]] for r in range(len(A))], dtype=np.int64)
    Xf = np.array([[int(np.rint(math.ldexp(X[k, c], int(53 - ec[c])))) for c in range(X.shape[1])]
                   for k in range(X.shape[0])], dtype=np.int64)
    Ad, Xd = _digits(Af), _digits(Xf)
    lev = np.zeros((LEVELS, A.shape[0], X.shape[1]), dtype=np.int64)
    for j in range(L):
        for i in range(L):
            if i + j < levels:
                lev[i + j] += Ad[j] @ Xd[i]
    T = np.zeros_like(lev[0])
    for lv in range(6):
        T = T * 256 + lev[lv]
    T = T + ((lev[6] * 256 + lev[7] + 32768) >> 16)
    out = np.array([[math.ldexp(float(T[r, c]), int(fr[r] + ec[c] - 50)) for c in range(X.shape[1])]
                    for r in range(A.shape[0])])
    return out, Ad, Xd, lev


def _exact(A, X):
    Af = [[Fraction(a) for a in row] for row in A]
    return np.array([[float(sum(Af[r][k] * Fraction(X[k, c]) for k in range(X.shape[0])))
                      for c in range(X.shape[1])] for r in range(len(A))])


@pytest.mark.parametrize("N", [2, 3, 4, 5])
def test_slicing_is_fp64_accurate(N):
    A = _operator(N)
    rng = np.random.default_rng(N)
    X = rng.normal(size=(N ** 3, 6)) * 10.0 ** rng.uniform(-5, 5, size=6)
    X[:, 0] = -11.0 + 0.01 * rng.normal(size=N ** 3)          # a log-density column
    out, Ad, Xd, lev = _sliced_product(A, X)
    assert np.abs(Ad).max() <= 2048 and np.abs(Xd).max() <= 2048   # exact in FP16
    assert np.abs(Ad[1:]).max() <= 128 and np.abs(Xd[1:]).max() <= 128
    assert np.abs(lev).max() < 2 ** 24                              # exact in FP32
    ref = _exact(A, X)
    err = np.abs(out - ref).max(axis=0) / np.abs(X).max(axis=0)
    assert np.all(err <= 3e-15), err


def test_a_dropped_level_is_caught():
    A = _operator(5)
    rng = np.random.default_rng(9)
    X = rng.normal(size=(125, 3))
    out, *_ = _sliced_product(A, X, levels=LEVELS - 2)             # levels 6 and 7 left out
    err = np.abs(out - _exact(A, X)).max(axis=0) / np.abs(X).max(axis=0)
    assert np.any(err > 3e-15), err
