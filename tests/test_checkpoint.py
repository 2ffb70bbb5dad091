"""Checkpoint files (paper_2306_01085_gb300.checkpoint): the state, the mesh description, time, step
counter, input nodes and network parameters come back exactly; mismatched or foreign files are
refused."""
import numpy as np
import pytest

from paper_2306_01085_gb300 import checkpoint as CK
from paper_2306_01085_gb300 import workloads as W


def test_round_trip(tmp_path):
    d = W.shell_desc(n=3, nr=2, p=2, euv=True)
    d.h_first = 0.0
    rng = np.random.default_rng(4)
    u = rng.normal(size=(d.n_elem, 5, d.n_p))
    nodes = rng.normal(size=(d.n_elem, 3, d.n_p))
    params = rng.normal(size=1000).astype(np.float32)
    f = tmp_path / "c.npz"
    CK.save(f, d, u, 12.5, 7, nodes=nodes, mlp=(256, 16, params))
    back = CK.load(f)
    assert back["desc"] == d
    assert np.array_equal(back["u"], u) and back["u"].dtype == np.float64
    assert back["t"] == 12.5 and back["step"] == 7
    assert np.array_equal(back["nodes"], nodes)
    h, r, p = back["mlp"]
    assert (h, r) == (256, 16) and np.array_equal(p, params)


def test_without_optional_parts(tmp_path):
    d = W.box_desc(p=1, n=2)
    u = np.zeros((d.n_elem, 5, d.n_p))
    CK.save(tmp_path / "c.npz", d, u, 0.0, 0)
    back = CK.load(tmp_path / "c.npz")
    assert back["nodes"] is None and back["mlp"] is None


def test_refuses_wrong_shapes_and_types(tmp_path):
    d = W.box_desc(p=1, n=2)
    with pytest.raises(ValueError):
        CK.save(tmp_path / "a.npz", d, np.zeros((d.n_elem + 1, 5, d.n_p)), 0.0, 0)
    with pytest.raises(ValueError):
        CK.save(tmp_path / "b.npz", d, np.zeros((d.n_elem, 5, d.n_p), dtype=np.float32), 0.0, 0)
    np.savez(tmp_path / "c.npz", format=np.int64(99))
    with pytest.raises(ValueError):
        CK.load(tmp_path / "c.npz")
