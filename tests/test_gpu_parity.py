"""FP64 parity of the CUDA path (through the C ABI) with the CPU oracle.

Bar: relative max-norm error per variable e_k = max|x_gpu - x_ref| / max|x_ref| <= 1e-12 for the
residual and the exact Jacobian-vector product. For the LDG gradient q the rounding of any FP64
evaluation is proportional to |u| / h (a variable with a large mean, such as sqrt(rho) T, has a
gradient far smaller than |u| / h), so its error is measured against
max(max|q_ref|, max|u| / h_min) per variable with the same 1e-12. Inputs are generated once from
the oracle's own nodes by the seeded workload module and handed to both sides unchanged.
"""
import numpy as np
import pytest

from oracle import dg as OD
from oracle import mesh as OM
from paper_2306_01085_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    from paper_2306_01085_gb300 import build as B
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    B.build()
    return torch


def rel_err_per_var(gpu, ref, var_axis):
    g = np.moveaxis(np.asarray(gpu), var_axis, 0).reshape(5, -1)
    r = np.moveaxis(np.asarray(ref), var_axis, 0).reshape(5, -1)
    return np.abs(g - r).max(1) / np.maximum(np.abs(r).max(1), 1e-300)


def grad_err_per_var(q, q_ref, u, om):
    """Error of a nodal gradient per variable against max(max|q_ref|, max|u| / h_min)."""
    h_min = float(((om.W[None, :] * om.detJ).sum(1)).min()) ** (1.0 / 3.0)
    err = np.abs(q - q_ref).max(axis=(0, 1, 3))
    scale = np.maximum(np.abs(q_ref).max(axis=(0, 1, 3)), np.abs(u).max(axis=(0, 2)) / h_min)
    return err / scale


def run_pair(torch, desc, seed=1, t=0.0, check_fd=True, interp="fp64"):
    from paper_2306_01085_gb300.dg import Mesh
    om = OM.OracleMesh(desc)
    u = W.state_for(desc, om.X, seed)
    v = W.unit_vector(seed + 100, u.shape)
    q_ref = OD.gradient(om, u)
    r_ref = OD.residual(om, u, q_ref, t)
    jv_ref = OD.jvp(om, u, v, t)
    m = Mesh(desc, nodes=om.X)
    m.set_interp(interp)
    ug = torch.from_numpy(u).cuda()
    vg = torch.from_numpy(v).cuda()
    q = m.gradient(ug)
    r = m.residual(ug, t=t)
    r2 = torch.empty_like(r)
    jv = m.jvp(ug, vg, t=t, r_out=r2)
    out = dict(q=grad_err_per_var(q.cpu().numpy(), q_ref, u, om), r=rel_err_per_var(r.cpu(), r_ref, 1),
               r_fused=rel_err_per_var(r2.cpu(), r_ref, 1), jv=rel_err_per_var(jv.cpu(), jv_ref, 1))
    out["x"] = float(np.abs(m.nodes().cpu().numpy() - om.X).max())
    if check_fd:
        jfd = m.jvp(ug, vg, t=t, mode="fd")
        out["jv_fd"] = rel_err_per_var(jfd.cpu(), jv_ref, 1)
    m.close()
    return out


def assert_parity(res, tol=TOL):
    assert res["x"] == 0.0, res
    for k in ("q", "r", "r_fused", "jv"):
        assert np.all(res[k] <= tol), (k, res[k])
    if "jv_fd" in res:
        # one-sided difference: truncation O(eps |v' H v|) with eps ~ 1e-8 (1 + |u|) / |v|
        assert np.all(res["jv_fd"] <= 1e-3), ("jv_fd", res["jv_fd"])


def test_box_4x4x4_p2_periodic(torch_cuda):
    """Periodic unit box 4x4x4, p = 2, Re = 100, Pr = 0.7, gravity along -z: one residual + one Jv."""
    assert_parity(run_pair(torch_cuda, W.box_desc(p=2, n=4), seed=1))


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_box_walls_ragged(torch_cuda, p):
    """3x3x3 box (27 elements: a ragged last CTA for every p), wall bottom, outflow top, mu ~ T^0.69."""
    d = W.box_desc(p=p, n=3, bc_lo=W.BC_WALL, bc_hi=W.BC_OUTFLOW, visc_exp=0.69, re=40.0)
    assert_parity(run_pair(torch_cuda, d, seed=3))


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_shell_small_with_rotation_and_heating(torch_cuda, p):
    """Cubed-sphere shell 6x3x3x2 (108 curved elements, panel edges with every orientation),
    rotation, radial gravity, sub-solar heating at t = 0.3, wall bottom / outflow top."""
    d = W.shell_desc(n=3, nr=2, p=p, euv=True)
    d.h_first = 0.0
    d.euv_r_peak = 0.5 * (d.r_inner + d.r_outer)
    d.euv_width = 0.25 * (d.r_outer - d.r_inner)
    assert_parity(run_pair(torch_cuda, d, seed=5, t=0.3))


def test_single_element_self_neighbour(torch_cuda):
    """One periodic element: every face is its own neighbour."""
    d = W.box_desc(p=2, n=1)
    assert_parity(run_pair(torch_cuda, d, seed=7))


def test_shell_16x8_p4_sampled_full_size(torch_cuda):
    """The 12,288-element p = 4 shell at full size, checked on sampled elements (bottom, top and
    interior layers, panel corners): the oracle computes r and Jv of those elements only."""
    torch = torch_cuda
    from paper_2306_01085_gb300.dg import Mesh
    desc = W.CONFIGS["shell16x8_p4"][0]()
    om = OM.OracleMesh(desc)
    u = W.state_for(desc, om.X, 2)
    v = W.unit_vector(102, u.shape)
    rng = np.random.default_rng(0)
    E = om.n_elem
    nz, n = desc.nz, desc.nx
    corners = [k + nz * (i + n * (j + n * P)) for P in range(6) for (i, j) in ((0, 0), (n - 1, n - 1))
               for k in (0, nz - 1)]
    sample = np.unique(np.concatenate([rng.choice(E, 24, replace=False), np.array(corners)]))
    r_ref = OD.residual(om, u, None, 0.0, elems=sample)
    jv_ref = OD.jvp(om, u, v, 0.0, elems=sample)
    m = Mesh(desc, nodes=om.X)
    ug = torch.from_numpy(u).cuda()
    vg = torch.from_numpy(v).cuda()
    r = torch.empty_like(ug)
    jv = m.jvp(ug, vg, t=0.0, r_out=r)
    e_r = rel_err_per_var(r.cpu().numpy()[sample], r_ref, 1)
    e_j = rel_err_per_var(jv.cpu().numpy()[sample], jv_ref, 1)
    m.close()
    assert np.all(e_r <= TOL) and np.all(e_j <= TOL), (e_r, e_j)


def test_mass_and_given_gradient(torch_cuda):
    torch = torch_cuda
    from paper_2306_01085_gb300.dg import Mesh
    d = W.shell_desc(n=2, nr=2, p=3)
    d.h_first = 0.0
    om = OM.OracleMesh(d)
    u = W.state_for(d, om.X, 9)
    v = W.unit_vector(19, u.shape)
    m = Mesh(d, nodes=om.X)
    ug = torch.from_numpy(u).cuda()
    mv = m.mass(torch.from_numpy(v).cuda()).cpu().numpy()
    assert np.all(rel_err_per_var(mv, OD.mass_apply(om, v), 1) <= TOL)
    # residual with the oracle's q passed in equals the oracle residual
    q_ref = OD.gradient(om, u)
    r = m.residual(ug, q=torch.from_numpy(q_ref).cuda()).cpu().numpy()
    assert np.all(rel_err_per_var(r, OD.residual(om, u, q_ref), 1) <= TOL)
    m.close()


def test_errors_are_reported(torch_cuda):
    from paper_2306_01085_gb300.dg import DgError, Mesh, lib
    d = W.box_desc(p=2, n=2)
    d.p = 5
    with pytest.raises(DgError, match="p must be"):
        Mesh(d)
    d = W.box_desc(p=2, n=2, bc_lo=W.BC_WALL, bc_hi=W.BC_PERIODIC)
    with pytest.raises(DgError, match="periodic"):
        Mesh(d)
    m = Mesh(W.box_desc(p=1, n=2))
    assert lib().dg_residual(m._h, None, None, 0.0, None, None) == -1
    m.close()


@pytest.mark.parametrize("name", ["box4_p2", "shell16x8_p4", "shell32x16_p2_euv"])
def test_library_mesh_generator_matches_workload_mesh(torch_cuda, name):
    """Without input nodes the library generates the workload mesh itself (Sec. 3.3 maps on the
    device); it agrees with the workload module's nodes to rounding of |x|."""
    from paper_2306_01085_gb300.dg import Mesh
    desc = W.CONFIGS[name][0]()
    ref = W.mesh_nodes(desc)
    m = Mesh(desc)
    x = m.nodes().cpu().numpy()
    m.close()
    assert np.abs(x - ref).max() <= 1e-14 * np.abs(ref).max()


# ---------------------------------------------------------------------------------------------
# The tensor-core interpolation (DG_INTERP_TC): nodes -> Gauss values and face traces as one dense
# contraction per element on tcgen05, FP64-accurate by digit slicing. Same bar against the oracle.
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_tc_interp_box_walls_ragged(torch_cuda, p):
    """27 elements: a partial last group of 6 (NC = 2) and 12 (NC = 1) elements for every p."""
    d = W.box_desc(p=p, n=3, bc_lo=W.BC_WALL, bc_hi=W.BC_OUTFLOW, visc_exp=0.69, re=40.0)
    assert_parity(run_pair(torch_cuda, d, seed=3, check_fd=False, interp="tc"))


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_tc_interp_shell_small(torch_cuda, p):
    d = W.shell_desc(n=3, nr=2, p=p, euv=True)
    d.h_first = 0.0
    d.euv_r_peak = 0.5 * (d.r_inner + d.r_outer)
    d.euv_width = 0.25 * (d.r_outer - d.r_inner)
    assert_parity(run_pair(torch_cuda, d, seed=5, t=0.3, check_fd=False, interp="tc"))


def test_tc_interp_single_element(torch_cuda):
    assert_parity(run_pair(torch_cuda, W.box_desc(p=4, n=1), seed=7, check_fd=False, interp="tc"))


def test_tc_interp_full_size(torch_cuda):
    """The 12,288-element p = 4 shell in the benchmark's launch configuration: the tensor-core
    path against the oracle on sampled elements (1e-12) and against the FP64 path everywhere
    (1e-13 per variable), residual and Jv."""
    torch = torch_cuda
    from paper_2306_01085_gb300.dg import Mesh
    desc = W.CONFIGS["shell16x8_p4"][0]()
    om = OM.OracleMesh(desc)
    u = W.state_for(desc, om.X, 4)
    v = W.unit_vector(104, u.shape)
    rng = np.random.default_rng(1)
    sample = np.unique(np.concatenate([rng.choice(om.n_elem, 12, replace=False), [0, om.n_elem - 1]]))
    r_ref = OD.residual(om, u, None, 0.0, elems=sample)
    jv_ref = OD.jvp(om, u, v, 0.0, elems=sample)
    m = Mesh(desc, nodes=om.X)
    ug = torch.from_numpy(u).cuda()
    vg = torch.from_numpy(v).cuda()
    out = {}
    for mode in ("fp64", "tc"):
        m.set_interp(mode)
        r = torch.empty_like(ug)
        jv = m.jvp(ug, vg, t=0.0, r_out=r)
        out[mode] = (r.cpu().numpy(), jv.cpu().numpy())
    m.close()
    r_tc, jv_tc = out["tc"]
    assert np.all(rel_err_per_var(r_tc[sample], r_ref, 1) <= TOL)
    assert np.all(rel_err_per_var(jv_tc[sample], jv_ref, 1) <= TOL)
    assert np.all(rel_err_per_var(r_tc, out["fp64"][0], 1) <= 1e-13)
    assert np.all(rel_err_per_var(jv_tc, out["fp64"][1], 1) <= 1e-13)


def test_tc_interp_propagates_nan(torch_cuda):
    """A NaN nodal value makes its element's Gauss values NaN, as in the FP64 passes: the residual's
    NaN pattern is the same in both modes (the solver's NaN checks see it)."""
    torch = torch_cuda
    from paper_2306_01085_gb300.dg import Mesh
    d = W.box_desc(p=3, n=3)
    m = Mesh(d)
    u = torch.from_numpy(W.state_for(d, m.nodes().cpu().numpy(), 2)).cuda()
    u[13, 4, 7] = float("nan")
    masks = []
    for mode in ("fp64", "tc"):
        m.set_interp(mode)
        masks.append(torch.isnan(m.residual(u)).cpu().numpy())
    m.close()
    assert masks[0].any() and np.array_equal(masks[0], masks[1])


def test_tc_interp_mode_is_validated(torch_cuda):
    from paper_2306_01085_gb300.dg import DgError, Mesh, lib
    m = Mesh(W.box_desc(p=2, n=2))
    assert lib().dg_mesh_set_interp(m._h, 7) == -1
    with pytest.raises(DgError):
        m.set_interp("bf16")
    m.close()


def test_tc_interp_in_the_implicit_step(torch_cuda):
    """The plain FP64 implicit step with the tensor-core interpolation (the Krylov solve's
    tangent-only interpolation writes the tangent planes) reaches the FP64-pass step to the Newton
    tolerance."""
    torch = torch_cuda
    from paper_2306_01085_gb300.dg import Mesh
    d = W.shell_desc(n=3, nr=2, p=2, euv=True)
    d.h_first = 0.0
    dt = 10.0 / W.shell_reference().t0
    m = Mesh(d)
    u0 = torch.from_numpy(W.state_for(d, m.nodes().cpu().numpy(), 6)).cuda()
    out = {}
    for mode in ("fp64", "tc"):
        m.set_interp(mode)
        u = u0.clone()
        st = m.implicit_step(u, 0.0, dt, stages=3, precond="bj", newton_rtol=1e-10, gmres_rtol=1e-6)
        assert st["status"] == 0
        out[mode] = u.cpu().numpy()
    m.close()
    change = np.abs(out["fp64"] - u0.cpu().numpy()).max()
    assert change > 1e-6
    assert np.abs(out["tc"] - out["fp64"]).max() <= 1e-8 * change
