"""Pins of the oracle's meshes and isoparametric geometry (Sec. 3.1 curved elements, Sec. 3.3 shells)."""
import math

import numpy as np
import pytest

from oracle import mesh as OM
from paper_2306_01085_gb300 import workloads as W


def _shell(n=2, nr=2, p=2, h_first=0.0):
    d = W.shell_desc(n=n, nr=nr, p=p)
    d.h_first = h_first
    return d


def test_box_volume_normals_and_matching():
    d = W.box_desc(p=2, n=3)
    m = OM.OracleMesh(d)
    vol = (m.W[None, :] * m.detJ).sum()
    assert abs(vol - 1.0) < 1e-14
    assert np.allclose(m.detJ, (1 / 3 / 2) ** 3, rtol=1e-13)
    # periodic box: every face has a neighbour and the matched points coincide (mod 1)
    assert np.all(m.nbr_elem >= 0)
    assert m.match_err < 1e-12
    # neighbour of the neighbour is the element itself
    e2, f2 = m.nbr_elem, m.nbr_face
    idx = np.arange(m.n_elem)[:, None]
    assert np.all(e2[e2, f2] == idx) and np.all(f2[e2, f2] == np.arange(6)[None, :])


def test_box_wall_boundaries_classified():
    d = W.box_desc(p=1, n=2, bc_lo=W.BC_WALL, bc_hi=W.BC_OUTFLOW)
    m = OM.OracleMesh(d)
    assert (m.bc == 1).sum() == 4 and (m.bc == 2).sum() == 4
    # wall faces are the xi_3 = -1 faces of the bottom layer and point down
    for e, f in zip(*np.nonzero(m.bc == 1)):
        assert f == 4 and np.all(m.nF[e, f, 2] < 0)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_closed_surface_normal_sum_is_zero(p):
    """sum over the 6 faces of int n dS vanishes for every curved element (exact quadrature)."""
    m = OM.OracleMesh(_shell(n=2, nr=2, p=p, h_first=0.5))
    tot = np.einsum("x,efdx->ed", m.wF, m.nF)
    assert np.abs(tot).max() < 1e-9 * np.abs(m.nF).max()
    assert np.all(m.detJ > 0)


def test_outward_normals_on_shell():
    m = OM.OracleMesh(_shell(n=2, nr=2, p=3))
    for e in range(m.n_elem):
        for f in range(6):
            dirv = m.xF[e, f].mean(-1) - m.xG[e].mean(-1)
            assert np.dot(m.nF[e, f].sum(-1), dirv) > 0


def test_shell_volume_converges_with_p():
    errs = []
    for p in (1, 2, 3, 4):
        d = _shell(n=2, nr=1, p=p)
        m = OM.OracleMesh(d)
        vol = (m.W[None, :] * m.detJ).sum()
        exact = 4.0 / 3.0 * math.pi * (d.r_outer ** 3 - d.r_inner ** 3)
        errs.append(abs(vol - exact) / exact)
    assert errs[-1] < 1e-5 and errs[0] > errs[1] > errs[2] > errs[3]


def test_shell_matching_and_boundaries():
    m = OM.OracleMesh(_shell(n=2, nr=3, p=2, h_first=0.3))
    assert (m.bc == 1).sum() == 24 and (m.bc == 2).sum() == 24
    assert m.match_err < 1e-9
    inter = m.nbr_elem >= 0
    assert inter.sum() == m.n_elem * 6 - 48
    # matched face normals are opposite at matched points
    for e, f in zip(*np.nonzero(inter)):
        e2, f2 = m.nbr_elem[e, f], m.nbr_face[e, f]
        n2 = m.nF[e2, f2][:, m.nbr_pt[e, f]]
        assert np.allclose(m.nF[e, f], -n2, atol=1e-10 * np.abs(m.nF).max())


def test_radial_layers_geometric_growth():
    d = W.shell_desc(n=2, nr=8, p=2)
    r = W.radial_layers(d.r_inner, d.r_outer, d.nz, d.h_first)
    h = np.diff(r)
    assert abs(h[0] - d.h_first) < 1e-12 * d.r_outer
    assert abs(r[-1] - d.r_outer) < 1e-12 and np.allclose(h[1:] / h[:-1], h[1] / h[0], rtol=1e-9)
    # growth ratio for 8 layers of a 500 km shell with a 2.5 km first layer
    assert abs(h[1] / h[0] - 1.9206) < 1e-3
