"""Algorithmic FP64 operation counts of the pointwise physics, taken from the oracle's expressions.

The oracle's flux, source and stabilisation functions are evaluated at one point on a scalar type
that counts its arithmetic: +, -, * and / are one flop each (a fused multiply-add is two), and exp,
log, sqrt and pow are counted apart as transcendental calls. Primitives and transport
coefficients are shared between the flux and the source (evaluated once per point), as any
evaluation of the method would share them.

The exact tangent (the Jacobian-vector product's second plane) costs, per value operation, the
forward-mode rule: a +- b -> 1, a * c (c constant) -> 1, a * b -> 3, a / c -> 1, a / b -> 3,
exp -> 1 (y a'), log -> 1 (a'/a), sqrt -> 2 (a'/(2 y)), a**c -> 3 (c y / a a').
"""
import contextlib
import math

import numpy as np


class Tally:
    def __init__(self):
        self.flops = 0
        self.tangent = 0
        self.trans = 0

    def add(self, flops=0, tangent=0, trans=0):
        self.flops += flops
        self.tangent += tangent
        self.trans += trans


TALLY = Tally()


class C:
    """A counted real number."""

    def __init__(self, v):
        self.v = float(v)

    # binary arithmetic -----------------------------------------------------------------------
    def _bin(self, other, fn, tan_var, tan_const):
        if isinstance(other, C):
            TALLY.add(1, tan_var)
            return C(fn(self.v, other.v))
        TALLY.add(1, tan_const)
        return C(fn(self.v, float(other)))

    def __add__(self, o):
        return self._bin(o, lambda a, b: a + b, 1, 0)

    def __radd__(self, o):
        return self.__add__(o)

    def __sub__(self, o):
        return self._bin(o, lambda a, b: a - b, 1, 0)

    def __rsub__(self, o):
        TALLY.add(1, 0)
        return C(float(o) - self.v)

    def __mul__(self, o):
        if not isinstance(o, C) and float(o) == 0.0:
            return C(0.0)                       # a structural zero (the oracle's "0.0 * u") costs nothing
        return self._bin(o, lambda a, b: a * b, 3, 1)

    def __rmul__(self, o):
        return self.__mul__(o)

    def __truediv__(self, o):
        return self._bin(o, lambda a, b: a / b, 3, 1)

    def __rtruediv__(self, o):
        TALLY.add(1, 3)
        return C(float(o) / self.v)

    def __neg__(self):
        return C(-self.v)

    def __pow__(self, e):
        if float(e) == 2.0:
            TALLY.add(1, 3)
        else:
            TALLY.add(0, 3, 1)
        return C(self.v ** float(e))

    # transcendental functions (numpy calls these on object arrays) ---------------------------
    def exp(self):
        TALLY.add(0, 1, 1)
        return C(math.exp(self.v))

    def log(self):
        TALLY.add(0, 1, 1)
        return C(math.log(self.v))

    def sqrt(self):
        TALLY.add(0, 2, 1)
        return C(math.sqrt(self.v))

    def __float__(self):
        return self.v

    def __lt__(self, o):
        return self.v < float(o)

    def __gt__(self, o):
        return self.v > float(o)


def counted(x):
    """An object array of counted numbers with the shape of x."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty(x.shape, dtype=object)
    for idx in np.ndindex(x.shape):
        out[idx] = C(x[idx])
    return out


@contextlib.contextmanager
def shared_primitives(P):
    """Evaluate the oracle's primitives and transport coefficients once per (state, gradient)."""
    prim, trans = P.primitives, P._transport
    cache = {}

    def prim_once(u, q, Cf):
        key = ("p", id(u), id(q))
        if key not in cache:
            cache[key] = prim(u, q, Cf)
        return cache[key]

    def trans_once(T, Cf, u0=None, mix=None):
        key = ("t", id(T))
        if key not in cache:
            cache[key] = trans(T, Cf, u0, mix)
        return cache[key]

    P.primitives, P._transport = prim_once, trans_once
    try:
        yield
    finally:
        P.primitives, P._transport = prim, trans


def measure(fn):
    """(value flops, tangent flops, transcendental calls) of fn()."""
    global TALLY
    TALLY = Tally()
    fn()
    return TALLY.flops, TALLY.tangent, TALLY.trans
