"""GPU reduced-basis preconditioner, initial guess and inverse mass matrix against the oracle
(Sec. 3.2)."""
import numpy as np
import pytest

from oracle import dg as OD
from oracle import mesh as OM
from oracle import rb as RB
from oracle import solver as OS
from paper_2306_01085_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    from paper_2306_01085_gb300 import build as B
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    B.build()
    return torch


def _box():
    # three elements along each periodic direction keep the block-Jacobi blocks exact
    return W.box_desc(p=1, n=3, nz=2, bc_lo=W.BC_WALL, bc_hi=W.BC_OUTFLOW, visc_exp=0.69, re=30.0)


@pytest.mark.parametrize("case", ["box_p2", "shell_p3"])
def test_inverse_mass_matches_oracle(torch_cuda, case):
    torch = torch_cuda
    from paper_2306_01085_gb300.dg import Mesh
    d = W.CONFIGS["box4_p2"][0]() if case == "box_p2" else W.shell_desc(n=1, nr=2, p=3, euv=False)
    om = OM.OracleMesh(d)
    v = W.unit_vector(21, (om.n_elem, 5, om.Np))
    ref = np.linalg.solve(RB.mass_matrix(om), v.ravel()).reshape(v.shape)
    m = Mesh(d, nodes=om.X)
    got = m.mass_inverse(torch.from_numpy(v).cuda()).cpu().numpy()
    back = m.mass(m.mass_inverse(torch.from_numpy(v).cuda())).cpu().numpy()
    m.close()
    assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max()
    assert np.abs(back - v).max() <= 1e-12 * np.abs(v).max()


@pytest.fixture(scope="module")
def rb_problem():
    d = _box()
    om = OM.OracleMesh(d)
    U = W.state_for(d, om.X, 6)
    t, c = 0.1, 0.15
    n = U.size
    Wb = np.stack([W.unit_vector(30 + j, (n,)) for j in range(4)], axis=1)
    Wb[:, 3] += 0.5 * Wb[:, 0]                          # correlated columns
    Z = RB.stage_jacobian_times(om, U, t, c, Wb)
    return d, om, U, t, c, n, Wb, Z


@pytest.mark.parametrize("base", ["rb", "rb_bj"])
def test_rb_apply_against_oracle(torch_cuda, rb_problem, base):
    """J~^{-1} maps J_G w to w on the RB space, and matches the oracle's dense solve of J~ y = x.
    Over the FP64 mass base both hold to 1e-9. Over block-Jacobi the base is applied in FP32, so it
    is linear only up to FP32 rounding: P0^{-1}(Z a) and sum_j a_j P0^{-1} Z_j differ by a few
    eps_32 (6e-8), which the Woodbury correction carries into the result (bound 1e-5); against
    the oracle the FP32 block inverses bound the difference by 1e-6 times their condition."""
    torch = torch_cuda
    from paper_2306_01085_gb300.dg import Mesh
    d, om, U, t, c, n, Wb, Z = rb_problem
    m = Mesh(d, nodes=om.X)
    ug = torch.from_numpy(U).cuda()
    w = torch.from_numpy(np.ascontiguousarray(Wb.T).reshape((4,) + U.shape)).cuda()
    m.rb_load(w, ug, t, c, base=base)
    a = np.array([0.5, -1.0, 2.0, 0.25])
    y = m.precond_apply(base, torch.from_numpy((Z @ a).reshape(U.shape)).cuda()).cpu().numpy().ravel()
    assert np.abs(y - Wb @ a).max() <= (1e-9 if base == "rb" else 1e-5) * np.abs(Wb @ a).max()
    x = W.unit_vector(40, (n,))
    got = m.precond_apply(base, torch.from_numpy(x.reshape(U.shape)).cuda()).cpu().numpy().ravel()
    m.close()
    P0 = RB.mass_matrix(om) if base == "rb" else RB.block_jacobi_matrix(om, U, t, c)
    ref = np.linalg.solve(RB.approximate_jacobian(Wb, Z, P0), x)
    err = np.abs(got - ref).max() / np.abs(ref).max()
    if base == "rb":
        assert err <= 1e-9, err
    else:
        B = OS.diagonal_blocks(om, U, t, c)
        cond = np.linalg.cond(B).max()
        assert err <= 1e-6 * cond, (err, cond)


def test_rb_initial_guess_against_oracle(torch_cuda, rb_problem):
    torch = torch_cuda
    from paper_2306_01085_gb300.dg import Mesh
    d, om, U, t, c, n, Wb, Z = rb_problem
    m = Mesh(d, nodes=om.X)
    ug = torch.from_numpy(U).cuda()
    w = torch.from_numpy(np.ascontiguousarray(Wb.T).reshape((4,) + U.shape)).cuda()
    m.rb_load(w, ug, t, c, base="rb")
    b = W.unit_vector(41, (n,)) + Z @ np.array([1.0, 0.0, -2.0, 0.5])
    got = m.rb_initial_guess(torch.from_numpy(b.reshape(U.shape)).cuda()).cpu().numpy().ravel()
    m.rb_reset()
    with pytest.raises(Exception):
        m.rb_initial_guess(torch.from_numpy(b.reshape(U.shape)).cuda())
    m.close()
    ref = RB.initial_guess(Wb, Z, b)
    assert np.abs(got - ref).max() <= 1e-8 * np.abs(ref).max()


@pytest.mark.parametrize("base", ["rb", "rb_bj"])
def test_rb_implicit_steps_match_oracle(torch_cuda, base):
    """Two DIRK(2,2) steps with the RB preconditioner and initial guess reach the oracle's plain
    steps to 1e-9 at tight tolerances; the window carries over between the steps."""
    torch = torch_cuda
    from paper_2306_01085_gb300.dg import Mesh
    d = W.box_desc(p=1, n=2, bc_lo=W.BC_WALL, bc_hi=W.BC_OUTFLOW, visc_exp=0.69, re=30.0)
    om = OM.OracleMesh(d)
    u = W.state_for(d, om.X, 4)
    dt = 0.05
    ref = OS.implicit_step(om, u, 0.0, dt, stages=2, tol=1e-12, gmres_tol=1e-10, restart=40)
    ref = OS.implicit_step(om, ref, dt, dt, stages=2, tol=1e-12, gmres_tol=1e-10, restart=40)
    m = Mesh(d, nodes=om.X)
    ug = torch.from_numpy(u).cuda()
    kw = dict(stages=2, precond=base, newton_rtol=1e-12, gmres_rtol=1e-10, gmres_restart=40, max_restarts=20,
              rb_size=4)
    s1 = m.implicit_step(ug, 0.0, dt, **kw)
    s2 = m.implicit_step(ug, dt, dt, **kw)
    got = ug.cpu().numpy()
    m.close()
    assert s1["status"] == 0 and s2["status"] == 0
    assert np.abs(got - ref).max() <= 1e-9 * np.abs(ref).max(), np.abs(got - ref).max()
    print(f"\n{base}: GMRES per stage {s1['gmres']} then {s2['gmres']}")


def test_rb_over_block_jacobi_on_a_stratified_shell(torch_cuda):
    """DIRK(3,3) steps of 60 s on a stratified shell: block-Jacobi alone, with FP16 inverses, and
    the RB preconditioner over block-Jacobi reach the same states within the Newton tolerance."""
    torch = torch_cuda
    from paper_2306_01085_gb300.dg import Mesh
    d = W.shell_desc(n=3, nr=6, p=2, euv=True)
    m = Mesh(d)
    u0 = torch.from_numpy(W.state_for(d, m.nodes().cpu().numpy(), 8)).cuda()
    dt = 60.0 / W.shell_reference().t0
    out = {}
    for pc in ("bj", "rb_bj", "bj16"):
        u = u0.clone()
        m.rb_reset()
        sts = [m.implicit_step(u, k * dt, dt, stages=3, precond=pc) for k in range(2)]
        out[pc] = (sts, u.cpu().numpy())
    m.close()
    du = np.abs(out["bj"][1] - u0.cpu().numpy()).max(axis=(0, 2))
    print("\nGMRES per step", {pc: [sum(s["gmres"]) for s in out[pc][0]] for pc in out})
    for pc in ("rb_bj", "bj16"):
        diff = np.abs(out[pc][1] - out["bj"][1]).max(axis=(0, 2))
        assert np.all(diff <= 1e-4 * du), (pc, diff, du)
