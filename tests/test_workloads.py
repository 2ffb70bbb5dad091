"""The benchmark workloads have the sizes the measurements quote: elements, degree and unknowns
(5 variables x (p + 1)^3 nodes per element), and the seeded inputs are reproducible."""
import numpy as np
import pytest

from paper_2306_01085_gb300 import workloads as W


@pytest.mark.parametrize("name,n_elem,p,n_dof", [
    ("box4_p2", 64, 2, 8_640),
    ("shell16x8_p4", 12_288, 4, 7_680_000),
    ("shell24x8_p2_euv", 27_648, 2, 3_732_480),
    ("shell24x8_p3_euv", 27_648, 3, 8_847_360),
    ("shell8x4_p3_euv", 1_536, 3, 491_520),
    ("shell32x16_p2_euv", 98_304, 2, 13_271_040),
    ("shell32x16_p2_euvac", 98_304, 2, 13_271_040),
    ("shell32x16_p2_comp", 98_304, 2, 13_271_040),
    ("shell48x16_p3_euv", 221_184, 3, 70_778_880),
    ("shell36x28_p3_euvac", 217_728, 3, 69_672_960),
])
def test_workload_sizes(name, n_elem, p, n_dof):
    d = W.CONFIGS[name][0]()
    assert d.p == p and d.n_elem == n_elem and d.n_dof == n_dof
    assert d.n_dof == 5 * n_elem * (p + 1) ** 3


def test_workload_flavours():
    assert W.CONFIGS["shell32x16_p2_euv"][0]().euv == W.EUV_GAUSS
    assert W.CONFIGS["shell32x16_p2_euvac"][0]().euv == W.EUV_EUVAC
    comp = W.CONFIGS["shell32x16_p2_comp"][0]()
    assert comp.euv == W.EUV_EUVAC and comp.comp == 1


def test_seeded_inputs_are_reproducible_and_distinct():
    d = W.CONFIGS["box4_p2"][0]()
    x = W.mesh_nodes(d)
    a, b, c = W.state_for(d, x, 3), W.state_for(d, x, 3), W.state_for(d, x, 4)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    v = W.unit_vector(7, a.shape)
    assert np.array_equal(v, W.unit_vector(7, a.shape)) and abs(np.linalg.norm(v) - 1.0) < 1e-14
