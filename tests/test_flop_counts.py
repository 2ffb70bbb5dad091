"""The algorithmic FP64 flop counts that bench.py reports against the FP64 roofline are the counts of
the oracle's own pointwise expressions (tests/flopcount.py): flux and source at a volume Gauss
point, the numerical flux of Eq. LDG2 at an interior, wall and outflow face point, each for the
value and for the exact tangent. Static geometry (gravity and centrifugal terms from the
positions) is precomputed once per mesh and is not counted."""
import numpy as np
import pytest

import flopcount as FC
from oracle import physics as P
from paper_2306_01085_gb300 import workloads as W

import bench


def _state(rng, shift=0.0):
    u = FC.counted(np.array([-1.0 + shift, 0.01, 0.02, -0.01, 2.0 + shift]))
    q = FC.counted(rng.standard_normal((3, 5)) * 0.1)
    return u, q


def _flux_dot_n(u, q, Cf, n, viscous):
    with FC.shared_primitives(P):
        F = P.flux(u, q, Cf, viscous, None)
    return [sum(F[c, d] * n[d] for d in range(3)) for c in range(5)]


def counts(desc):
    Cf = P.Coeffs(desc)
    rng = np.random.default_rng(0)
    u, q = _state(rng)
    u2, q2 = _state(rng, 0.01)
    x = np.array([600.0, 10.0, 5.0])            # positions: static geometry, not counted
    n = np.array([0.3, 0.4, 0.5])
    area = 1.3

    def volume():
        with FC.shared_primitives(P):
            P.flux(u, q, Cf, True, None)
            P.source(u, q, x, 0.0, Cf)

    def interior():
        f1 = _flux_dot_n(u, q, Cf, n, True)
        f2 = _flux_dot_n(u2, q2, Cf, n, True)
        uh = np.array([0.5 * (u[c] + u2[c]) for c in range(5)], dtype=object)
        with FC.shared_primitives(P):
            sg = P.sigma(uh, Cf)
        return [0.5 * (f1[c] + f2[c]) + sg[c] * ((0.5 * area) * (u[c] - u2[c])) for c in range(5)]

    def wall():
        ub = P.wall_state(u, Cf)
        f = _flux_dot_n(ub, q, Cf, n, True)
        with FC.shared_primitives(P):
            sg = P.sigma(ub, Cf)
        return [f[c] + sg[c] * (area * (u[c] - ub[c])) for c in range(5)]

    def outflow():
        return _flux_dot_n(u, q, Cf, n, False)

    return {k: FC.measure(fn) for k, fn in (("volume_point", volume), ("face_interior", interior),
                                            ("face_wall", wall), ("face_outflow", outflow))}


def test_pointwise_counts_are_the_benchmark_constants():
    desc = W.CONFIGS[bench.CONFIG_NAME][0]()
    got = counts(desc)
    for k, (val, tan, trans) in got.items():
        assert (val, tan) == bench.PHYS_FLOPS[k], (k, val, tan)
        assert trans == bench.PHYS_TRANSCENDENTALS[k], (k, trans)


def test_counter_counts_a_known_expression():
    """x*y + exp(x)/y: 3 flops and one transcendental; tangent 3 (x*y) + 1 (+) + 1 (exp) + 3 (/)."""
    x, y = FC.C(0.3), FC.C(1.7)
    val, tan, trans = FC.measure(lambda: x * y + np.exp(x) / y)
    assert (val, tan, trans) == (3, 8, 1)


def test_kernel_flops_per_element_at_p4():
    """The per-element totals combine the pointwise counts with the sum-factorised contractions
    (per plane and Gauss point: reference fluxes 90, source weighting 5, weak derivative 30 N,
    face lifting 60, projection B^T 30 N; interpolation 30 N per plane and point plus 30 N per
    face point; the LDG gradient as counted for k_grad)."""
    k = bench.kernel_flops(5, n_elem=1, n_interior=0, n_wall=0, n_outflow=0)
    v = sum(bench.PHYS_FLOPS["volume_point"])
    assert k["k_volume"] == 125 * (v + 2 * (155 + 60 * 5))
    assert k["k_interp"] == 2 * 5 * (125 * 3 * 5 * 2 + 6 * 25 * 5 * 2)
    assert k["k_grad"] == bench.grad_flops_per_element(5)
