"""The radial 1D ensemble on the GPU (dg_radial_* through the C ABI) against the radial oracle.

Residual and exact Jv per variable to 1e-12 of the variable's largest oracle value, at p = 1 to 4
(the paper's 28-element p = 2 column and smaller ones), for columns with different sites, EUV
efficiencies and conductivity factors, with a ragged column count; columns are independent
(permuting the parameters permutes the results bit for bit); the DIRK(2,2) step of 30 s reaches
the oracle's step to the Newton tolerance; and the 16,384-column ensemble matches the oracle on
sampled columns."""
import numpy as np
import pytest

from oracle import radial as OR
from paper_2306_01085_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    from paper_2306_01085_gb300 import build as B
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    B.build()
    return torch


def _oracle(desc, u, params, t, v=None):
    C = OR.Coeffs(desc)
    mesh = OR.RadialMesh(desc, W.radial_nodes(desc))
    r = np.zeros_like(u)
    jv = np.zeros_like(u)
    for c in range(desc.n_col):
        r[..., c] = OR.residual(mesh, u[..., c], t, C, params[c])
        if v is not None:
            jv[..., c] = OR.jvp(mesh, u[..., c], v[..., c], t, C, params[c])
    return r, jv


def _err(got, ref):
    return np.abs(got - ref).max(axis=(1, 2, 3)) / np.abs(ref).max(axis=(1, 2, 3))


@pytest.mark.parametrize("p,n_elem,n_col", [(2, 28, 7), (1, 12, 5), (3, 10, 33), (4, 8, 37)])
def test_residual_and_jv_match_oracle(torch_cuda, p, n_elem, n_col):
    torch = torch_cuda
    from paper_2306_01085_gb300.dg import Radial
    d = W.radial_desc(n_col=n_col, n_elem=n_elem, p=p)
    params = W.radial_params(n_col, seed=31)
    u = W.radial_state(d, seed=5)
    v = W.unit_vector(41, u.shape)
    t = 7.3                                   # the Sun has moved: zenith angles differ per column
    r_ref, jv_ref = _oracle(d, u, params, t, v)
    rad = Radial(d, params, node_r=W.radial_nodes(d))
    ug, vg = torch.from_numpy(u).cuda(), torch.from_numpy(v).cuda()
    r = rad.residual(ug, t).cpu().numpy()
    r2 = rad.empty()
    jv = rad.jvp(ug, vg, t, r_out=r2).cpu().numpy()
    r2 = r2.cpu().numpy()
    rad.close()
    assert np.all(_err(r, r_ref) <= 1e-12), _err(r, r_ref)
    assert np.all(_err(jv, jv_ref) <= 1e-12), _err(jv, jv_ref)
    assert np.array_equal(r, r2)              # the fused pass gives the residual of the plain pass


def test_columns_are_independent(torch_cuda):
    """Permuting the columns' parameters and states permutes the results exactly."""
    torch = torch_cuda
    from paper_2306_01085_gb300.dg import Radial
    d = W.radial_desc(n_col=40, n_elem=28, p=2)
    params = W.radial_params(40, seed=8)
    u = W.radial_state(d, seed=9)
    perm = np.random.default_rng(2).permutation(40)
    a = Radial(d, params, node_r=W.radial_nodes(d))
    b = Radial(d, params[perm], node_r=W.radial_nodes(d))
    ra = a.residual(torch.from_numpy(u).cuda(), 3.0).cpu().numpy()
    rb = b.residual(torch.from_numpy(np.ascontiguousarray(u[..., perm])).cuda(), 3.0).cpu().numpy()
    a.close()
    b.close()
    assert np.array_equal(ra[..., perm], rb)


def test_library_mesh_matches_the_workload_mesh(torch_cuda):
    """The library's own geometric layers (no node radii given) give the same residual."""
    torch = torch_cuda
    from paper_2306_01085_gb300.dg import Radial
    d = W.radial_desc(n_col=4)
    params = W.radial_params(4)
    u = torch.from_numpy(W.radial_state(d)).cuda()
    a = Radial(d, params, node_r=W.radial_nodes(d))
    b = Radial(d, params)
    ra, rb = a.residual(u, 1.0).cpu().numpy(), b.residual(u, 1.0).cpu().numpy()
    a.close()
    b.close()
    assert np.all(_err(rb, ra) <= 1e-12)


@pytest.mark.parametrize("p,n_elem", [(2, 28), (4, 8)])
def test_dirk22_step_matches_oracle(torch_cuda, p, n_elem):
    """The paper's 1D time step (DIRK(2,2), 30 s) on the 28-element p = 2 column (and a p = 4
    column, whose band is 44 wide on each side): the ensemble's FP32-Jacobian Newton iteration and
    the oracle's exact Newton with a dense solve reach the same stage solutions, to the Newton
    tolerance."""
    torch = torch_cuda
    from paper_2306_01085_gb300.dg import Radial
    n_col = 3
    d = W.radial_desc(n_col=n_col, n_elem=n_elem, p=p)
    params = W.radial_params(n_col, seed=12)
    u = W.radial_state(d, seed=13)
    dt = 30.0 / W.shell_reference().t0
    C = OR.Coeffs(d)
    mesh = OR.RadialMesh(d, W.radial_nodes(d))
    ref = np.stack([OR.implicit_step(mesh, u[..., c], 0.0, dt, C, params[c], stages=2, tol=1e-12)[0]
                    for c in range(n_col)], axis=-1)
    rad = Radial(d, params, node_r=W.radial_nodes(d))
    ug = torch.from_numpy(u).cuda()
    st = rad.step(ug, 0.0, dt, stages=2, newton_rtol=1e-12, max_newton=30)
    got = ug.cpu().numpy()
    rad.close()
    assert st["status"] == 0
    change = np.abs(ref - u).max(axis=(0, 1, 2))
    assert np.all(change > 1e-6)
    err = np.abs(got - ref).max(axis=(0, 1, 2)) / change
    assert np.all(err <= 1e-8), err


def test_failed_step_leaves_the_state_unchanged(torch_cuda):
    """A Newton cap of one iteration reports DG_ENOTCONV and restores u (the fault is injected on
    the host through the iteration limit)."""
    torch = torch_cuda
    from paper_2306_01085_gb300.dg import Radial
    d = W.radial_desc(n_col=4)
    rad = Radial(d, W.radial_params(4), node_r=W.radial_nodes(d))
    u = torch.from_numpy(W.radial_state(d)).cuda()
    u0 = u.clone()
    st = rad.step(u, 0.0, 30.0 / W.shell_reference().t0, stages=2, newton_rtol=1e-14, max_newton=1, check=False)
    rad.close()
    assert st["rc"] == -4
    assert torch.equal(u, u0)


def test_large_ensemble_sampled_columns(torch_cuda):
    """The benchmark's 16,384-column ensemble: sampled columns' residual and Jv against the oracle
    (1e-12 per variable), and a DIRK(2,2) step that converges for every column."""
    torch = torch_cuda
    from paper_2306_01085_gb300.dg import Radial
    n_col = 16384
    d = W.radial_desc(n_col=n_col)
    params = W.radial_params(n_col)
    u = W.radial_state(d, seed=3)
    v = W.unit_vector(17, u.shape)
    rad = Radial(d, params, node_r=W.radial_nodes(d))
    ug, vg = torch.from_numpy(u).cuda(), torch.from_numpy(v).cuda()
    r = rad.empty()
    jv = rad.jvp(ug, vg, 11.0, r_out=r).cpu().numpy()
    r = r.cpu().numpy()
    cols = [0, 1, 4097, 8191, 12000, n_col - 1]
    ds = W.radial_desc(n_col=len(cols))
    r_ref, jv_ref = _oracle(ds, np.ascontiguousarray(u[..., cols]), params[cols], 11.0,
                            np.ascontiguousarray(v[..., cols]))
    assert np.all(_err(r[..., cols], r_ref) <= 1e-12)
    assert np.all(_err(jv[..., cols], jv_ref) <= 1e-12)
    st = rad.step(ug, 0.0, 30.0 / W.shell_reference().t0, stages=2, newton_rtol=1e-8)
    rad.close()
    assert st["status"] == 0 and st["max_ratio"] <= 1e-8
    assert torch.isfinite(ug).all()
