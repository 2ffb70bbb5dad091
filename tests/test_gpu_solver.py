"""GPU implicit step, Newton-GMRES and block-Jacobi against the oracle (Sec. 3.1-3.2)."""
import numpy as np
import pytest

from oracle import dg as OD
from oracle import mesh as OM
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


def _walled_box(p=1, n=2):
    return W.box_desc(p=p, n=n, bc_lo=W.BC_WALL, bc_hi=W.BC_OUTFLOW, visc_exp=0.69, re=30.0)


@pytest.mark.parametrize("stages", [2, 3])
def test_dirk_tableau_matches_oracle(torch_cuda, stages):
    from paper_2306_01085_gb300 import dg as DG
    a, c = DG.dirk_tableau(stages)
    A, b, cc = OS.dirk_tableau(stages)
    assert np.abs(a - A).max() < 1e-14 and np.abs(c - cc).max() < 1e-14


@pytest.mark.parametrize("p", [2, 3, 4])
def test_block_jacobi_solve_inverts_the_assembled_blocks(torch_cuda, p):
    """dg_precond_apply (FP32 Gauss-Jordan inverses) against an FP64 solve of the same blocks: one
    CTA per block in shared memory at p = 2 (135^2), a cluster of CTAs sharing each block at p = 3
    (320^2, 2 CTAs) and p = 4 (625^2, 8 CTAs)."""
    torch = torch_cuda
    from paper_2306_01085_gb300.dg import Mesh
    d = W.shell_desc(n=2 if p == 2 else 1, nr=4 if p == 2 else 2, p=p, euv=True)
    d.h_first = 0.0                      # uniform layers keep the interpolated T positive
    m = Mesh(d)
    u = torch.from_numpy(W.state_for(d, m.nodes().cpu().numpy(), 4)).cuda()
    c = 0.8
    B = m.block_assemble(u, 0.2, c).cpu().numpy().astype(np.float64)
    m.precond_setup("bj", u, 0.2, c)
    x = W.unit_vector(5, tuple(u.shape))
    y = m.precond_apply("bj", torch.from_numpy(x).cuda()).cpu().numpy().reshape(m.n_elem, -1)
    m.close()
    ref = np.linalg.solve(B, x.reshape(m.n_elem, -1, 1))[..., 0]
    cond = np.linalg.cond(B).max()
    err = np.abs(y - ref).max() / np.abs(ref).max()
    assert err < 1e-6 * cond, (err, cond)


@pytest.mark.parametrize("p", [2, 3, 4])
def test_fp16_block_jacobi_is_the_fp32_inverse_rounded(torch_cuda, p):
    """DG_PC_BJ16 against DG_PC_BJ on the same FP32 inverses A: every stored entry carries at most
    2^-11 relative rounding (2^-25 c_j absolute in the subnormal range, c_j <= 2 max_i |A_ij|) and
    both sums of n terms in FP32 err by at most n 2^-24 (|A| |x|)_i, so
    |y16 - y32|_i <= (2^-11 + 2 n 2^-24) (|A| |x|)_i + 2^-24 sum_j max_i |A_ij| |x_j|,
    with 10 % slack for taking |A| from an FP64 inverse of the assembled block."""
    torch = torch_cuda
    from paper_2306_01085_gb300.dg import Mesh
    d = W.shell_desc(n=2 if p == 2 else 1, nr=4 if p == 2 else 2, p=p, euv=True)
    d.h_first = 0.0
    m = Mesh(d)
    u = torch.from_numpy(W.state_for(d, m.nodes().cpu().numpy(), 4)).cuda()
    c = 0.8
    B = m.block_assemble(u, 0.2, c).cpu().numpy().astype(np.float64)
    m.precond_setup("bj16", u, 0.2, c)
    x = W.unit_vector(5, tuple(u.shape))
    xg = torch.from_numpy(x).cuda()
    y16 = m.precond_apply("bj16", xg).cpu().numpy().reshape(m.n_elem, -1)
    y32 = m.precond_apply("bj", xg).cpu().numpy().reshape(m.n_elem, -1)
    m.precond_setup("bj", u, 0.2, c)                   # rebuilding FP32 only retires the FP16 copy
    with pytest.raises(Exception):
        m.precond_apply("bj16", xg)
    m.close()
    Ainv = np.abs(np.linalg.inv(B))
    xa = np.abs(x.reshape(m.n_elem, -1))
    ax = np.einsum("eij,ej->ei", Ainv, xa)
    cx = np.einsum("ej,ej->e", Ainv.max(axis=1), xa)[:, None]
    n = B.shape[1]
    bound = 1.1 * ((2.0 ** -11 + 2 * n * 2.0 ** -24) * ax + 2.0 ** -24 * cx)
    assert np.all(np.abs(y16 - y32) <= bound), np.abs(y16 - y32).max() / ax.max()
    assert np.abs(y16 - y32).max() > 0                 # the FP16 path is really a different path


@pytest.mark.parametrize("case", ["box_p1", "shell_p2"])
def test_block_assembly_matches_oracle_blocks(torch_cuda, case):
    """Assembled FP32 blocks against the oracle's FP64 brute-force blocks, entry by entry."""
    torch = torch_cuda
    from paper_2306_01085_gb300 import dg as DG
    if case == "box_p1":
        d = W.box_desc(p=1, n=3, nz=2, bc_lo=W.BC_WALL, bc_hi=W.BC_OUTFLOW, visc_exp=0.69, re=30.0)
    else:
        d = W.shell_desc(n=1, nr=2, p=2, euv=True)
        d.h_first = 0.0
    om = OM.OracleMesh(d)
    u = W.state_for(d, om.X, 6)
    c = 0.15
    B_ref = OS.diagonal_blocks(om, u, 0.1, c)
    m = DG.Mesh(d, nodes=om.X)
    B = m.block_assemble(torch.from_numpy(u).cuda(), 0.1, c).cpu().numpy().astype(np.float64)
    m.close()
    for e in range(om.n_elem):
        assert np.abs(B[e] - B_ref[e]).max() <= 2e-7 * np.abs(B_ref[e]).max(), e


@pytest.mark.parametrize("p,nr,elems", [(3, 2, [0, 1]), (4, 1, [0])])
def test_large_blocks_match_oracle_blocks_and_invert(torch_cuda, p, nr, elems):
    """The blocks of the p = 3 (320^2) and p = 4 (625^2) paths against the oracle's brute-force
    blocks on curved shell elements with a wall and an outflow face, entry by entry; and the
    block-Jacobi apply (Gauss-Jordan on a cluster of 2 or 8 CTAs sharing a block) against an FP64
    solve with the ORACLE's blocks, within 1e-6 x cond."""
    torch = torch_cuda
    from paper_2306_01085_gb300 import dg as DG
    d = W.shell_desc(n=1, nr=nr, p=p, euv=True)
    d.h_first = 0.0
    om = OM.OracleMesh(d)
    u = W.state_for(d, om.X, 6)
    c = 0.15
    B_ref = OS.diagonal_blocks(om, u, 0.1, c, elems=elems)
    m = DG.Mesh(d, nodes=om.X)
    ug = torch.from_numpy(u).cuda()
    B = m.block_assemble(ug, 0.1, c).cpu().numpy().astype(np.float64)
    m.precond_setup("bj", ug, 0.1, c)
    x = W.unit_vector(8, u.shape)
    y = m.precond_apply("bj", torch.from_numpy(x).cuda()).cpu().numpy().reshape(m.n_elem, -1)
    m.close()
    for k, e in enumerate(elems):
        assert np.abs(B[e] - B_ref[k]).max() <= 2e-7 * np.abs(B_ref[k]).max(), e
        ref = np.linalg.solve(B_ref[k], x[e].ravel())
        cond = np.linalg.cond(B_ref[k])
        assert np.abs(y[e] - ref).max() <= 1e-6 * cond * np.abs(ref).max(), (e, cond)


_SHELL_STEP = {}


def _oracle_shell_step(p):
    """The oracle's DIRK(3,3) step of 10 s on a 6x1x1x2 curved shell (p = 2 or 3) with rotation and
    EUV heating, Newton to 1e-11 (GMRES right-preconditioned by the element mass matrix, which
    changes only the iteration count)."""
    if p not in _SHELL_STEP:
        d = W.shell_desc(n=1, nr=2, p=p, euv=True)
        d.h_first = 0.0
        om = OM.OracleMesh(d)
        u = W.state_for(d, om.X, 4)
        dt = 10.0 / W.shell_reference().t0
        pb = lambda U, ti, daii: (lambda y: OD.mass_solve(om, y.reshape(U.shape)).ravel())
        ref = OS.implicit_step(om, u, 0.0, dt, stages=3, tol=1e-11, gmres_tol=1e-9, restart=60, precond_builder=pb)
        _SHELL_STEP[p] = (d, om, u, dt, ref)
    return _SHELL_STEP[p]


@pytest.mark.parametrize("p,precond,jv_prec", [(2, "bj", "f64"), (2, "bj16", "f32"), (3, "bj", "f64"),
                                               (3, "bj16", "f32")])
def test_shell_implicit_step_matches_oracle(torch_cuda, p, precond, jv_prec):
    """DIRK(3,3) on a curved shell at p = 2 and 3: the plain path (FP64 Jv, block-Jacobi with FP32
    inverses) and the mixed path (FP32 Jv and Gram-Schmidt arithmetic, FP16-stored inverses) both
    reach the oracle's step. Newton runs on the FP64 residual, so the precision of the Krylov solve
    changes the iteration counts, not the converged state."""
    torch = torch_cuda
    from paper_2306_01085_gb300.dg import Mesh
    d, om, u, dt, ref = _oracle_shell_step(p)
    m = Mesh(d, nodes=om.X)
    ug = torch.from_numpy(u).cuda()
    st = m.implicit_step(ug, 0.0, dt, stages=3, precond=precond, jv_prec=jv_prec, newton_rtol=1e-11,
                         gmres_rtol=1e-9, gmres_restart=60, max_restarts=20)
    got = ug.cpu().numpy()
    m.close()
    assert st["status"] == 0
    change = np.abs(ref - u).max()
    assert change > 1e-3                           # the step did something
    assert np.abs(got - ref).max() <= 1e-8 * change, np.abs(got - ref).max() / change


@pytest.mark.parametrize("stages", [2, 3])
def test_implicit_step_matches_oracle(torch_cuda, stages):
    """Tight tolerances: both reach the same DIRK step to ~1e-10."""
    torch = torch_cuda
    from paper_2306_01085_gb300.dg import Mesh
    d = _walled_box(p=1, n=2)
    om = OM.OracleMesh(d)
    u = W.state_for(d, om.X, 4)
    dt = 0.05
    ref = OS.implicit_step(om, u, 0.0, dt, stages=stages, tol=1e-12, gmres_tol=1e-10, restart=40)
    m = Mesh(d, nodes=om.X)
    ug = torch.from_numpy(u).cuda()
    st = m.implicit_step(ug, 0.0, dt, stages=stages, newton_rtol=1e-12, gmres_rtol=1e-10, gmres_restart=40,
                         max_restarts=20)
    got = ug.cpu().numpy()
    m.close()
    assert st["status"] == 0
    assert np.abs(got - ref).max() < 1e-9 * np.abs(ref).max(), np.abs(got - ref).max()
    assert np.abs(got - u).max() > 1e-6   # the step did something


def test_solver_variants_reach_the_same_state(torch_cuda):
    """On a stratified shell at dt = 60 s: block-Jacobi built once per step, rebuilt every Newton
    iteration, and with the paper's finite-difference Jv all reach the same DIRK(3,3) step within
    the Newton tolerance (1e-8)."""
    torch = torch_cuda
    from paper_2306_01085_gb300.dg import Mesh
    d = W.shell_desc(n=3, nr=6, p=2, euv=True)
    m = Mesh(d)
    u0 = torch.from_numpy(W.state_for(d, m.nodes().cpu().numpy(), 8)).cuda()
    dt = 60.0 / W.shell_reference().t0
    runs = {}
    for name, kw in {"step": dict(precond="bj"), "newton": dict(precond="bj", precond_refresh="newton"),
                     "fd": dict(precond="bj", jv_mode="fd")}.items():
        u = u0.clone()
        runs[name] = (m.implicit_step(u, 0.0, dt, stages=3, **kw), u.cpu().numpy())
    m.close()
    ref = runs["step"][1]
    du = np.abs(ref - u0.cpu().numpy()).max(axis=(0, 2))
    for name in ("newton", "fd"):
        diff = np.abs(runs[name][1] - ref).max(axis=(0, 2))
        assert np.all(diff <= 1e-4 * du + 1e-12), (name, diff, du)
    assert all(r[0]["status"] == 0 for r in runs.values())


def test_resume_from_checkpoint_is_bit_identical(torch_cuda, tmp_path):
    """Three DIRK(3,3) steps straight through, and two steps, a checkpoint, a new mesh built from
    the checkpoint's description and one more step: the final states are bit for bit the same
    (per-step block-Jacobi builds, FP32 inner Jv)."""
    torch = torch_cuda
    from paper_2306_01085_gb300 import checkpoint as CK
    from paper_2306_01085_gb300.dg import Mesh
    d = W.shell_desc(n=3, nr=4, p=2, euv=True)
    dt = 60.0 / W.shell_reference().t0
    kw = dict(stages=3, precond="bj16", jv_prec="f32")
    m = Mesh(d)
    u0 = torch.from_numpy(W.state_for(d, m.nodes().cpu().numpy(), 3)).cuda()
    straight = u0.clone()
    for k in range(3):
        m.implicit_step(straight, k * dt, dt, **kw)
    u = u0.clone()
    for k in range(2):
        m.implicit_step(u, k * dt, dt, **kw)
    CK.save(tmp_path / "run.npz", d, u, 2 * dt, 2)
    m.close()
    c = CK.load(tmp_path / "run.npz")
    m2 = Mesh(c["desc"])
    u2 = torch.from_numpy(c["u"]).cuda()
    m2.implicit_step(u2, c["t"], dt, **kw)
    m2.close()
    assert c["step"] == 2
    assert torch.equal(u2, straight)


def test_lagged_preconditioner_refresh(torch_cuda):
    """DG_REFRESH_LAGGED builds the FP16 block-Jacobi preconditioner on the first of every
    refresh_every steps and reuses it in between (no setup time on those steps); a change of dt or
    a failed step forces a build; every step still converges to the Newton tolerance, so the
    states follow the per-step builds to that tolerance."""
    torch = torch_cuda
    from paper_2306_01085_gb300.dg import DgError, Mesh
    d = W.shell_desc(n=3, nr=6, p=2, euv=True)
    m = Mesh(d)
    u0 = torch.from_numpy(W.state_for(d, m.nodes().cpu().numpy(), 8)).cuda()
    dt = 60.0 / W.shell_reference().t0
    kw = dict(stages=3, precond="bj16", jv_prec="f32", newton_rtol=1e-10, gmres_rtol=1e-4)
    u_ref, u_lag = u0.clone(), u0.clone()
    built = []
    for k in range(4):
        m.implicit_step(u_ref, k * dt, dt, **kw)
    for k in range(4):   # (the per-step builds above leave no lagged preconditioner: the first step builds)
        st = m.implicit_step(u_lag, k * dt, dt, precond_refresh="lagged", refresh_every=2, **kw)
        built.append(st["precond_ms"] > 0)
    assert built == [True, False, True, False], built
    du = np.abs(u_ref.cpu().numpy() - u0.cpu().numpy()).max(axis=(0, 2))
    diff = np.abs(u_lag.cpu().numpy() - u_ref.cpu().numpy()).max(axis=(0, 2))
    assert np.all(diff <= 1e-6 * du), (diff, du)
    # dt changes: build; then reuse
    st = m.implicit_step(u_lag, 4 * dt, 0.5 * dt, precond_refresh="lagged", refresh_every=3, **kw)
    assert st["precond_ms"] > 0
    st = m.implicit_step(u_lag, 4.5 * dt, 0.5 * dt, precond_refresh="lagged", refresh_every=3, **kw)
    assert st["precond_ms"] == 0
    # a failed step (Newton capped at one iteration) leaves the state and forces the next build
    before = u_lag.clone()
    st = m.implicit_step(u_lag, 5 * dt, 0.5 * dt, precond_refresh="lagged", refresh_every=3, check=False,
                         **dict(kw, newton_rtol=1e-14, max_newton=1))
    assert st["rc"] == -4 and torch.equal(u_lag, before)
    st = m.implicit_step(u_lag, 5 * dt, 0.5 * dt, precond_refresh="lagged", refresh_every=3, **kw)
    assert st["status"] == 0 and st["precond_ms"] > 0
    with pytest.raises(DgError):
        m.implicit_step(u_lag, 0.0, dt, precond_refresh="lagged", refresh_every=0, **kw)
    m.close()


@pytest.mark.parametrize("p", [2, 3])
@pytest.mark.parametrize("jv_prec", ["f64", "f32"])
def test_value_plane_once_per_solve_is_bit_identical(torch_cuda, jv_prec, p):
    """Forming the state's value plane once per Krylov solve and once per block assembly (the
    default) gives bit for bit the step of recomputing it in every operator application and every
    assembly sweep: same states, same iteration counts. The shell has wall and outflow boundaries,
    where the tangent trace reads the value plane."""
    torch = torch_cuda
    from paper_2306_01085_gb300.dg import Mesh
    d = W.shell_desc(n=2, nr=4, p=p, euv=True)
    d.h_first = 0.0
    m = Mesh(d)
    u0 = torch.from_numpy(W.state_for(d, m.nodes().cpu().numpy(), 8)).cuda()
    dt = (60.0 if p == 2 else 20.0) / W.shell_reference().t0
    out = {}
    for flags in (0, 1):
        u = u0.clone()
        st = m.implicit_step(u, 0.0, dt, stages=3, precond="bj", jv_prec=jv_prec, flags=flags)
        out[flags] = (st["gmres"], st["newton"], u.cpu().numpy())
    m.close()
    assert out[0][0] == out[1][0] and out[0][1] == out[1][1]
    assert np.array_equal(out[0][2], out[1][2])


def test_unpreconditioned_and_block_jacobi_agree(torch_cuda):
    """Unpreconditioned GMRES(30) stalls on this stratified shell once Newton has removed the
    smooth error, so the comparison is one backward-Euler stage of 2.2 s to a Newton tolerance of
    1e-5 (two Newton iterations); the block-Jacobi solve needs far fewer Krylov iterations and
    reaches the same state."""
    torch = torch_cuda
    from paper_2306_01085_gb300.dg import Mesh
    d = W.shell_desc(n=3, nr=6, p=2, euv=True)
    m = Mesh(d)
    u0 = torch.from_numpy(W.state_for(d, m.nodes().cpu().numpy(), 8)).cuda()
    dt = 2.2 / W.shell_reference().t0
    out = {}
    for pc in ("none", "bj"):
        u = u0.clone()
        out[pc] = (m.implicit_step(u, 0.0, dt, stages=1, precond=pc, newton_rtol=1e-5, max_restarts=60),
                   u.cpu().numpy())
    m.close()
    (s0, u_none), (s1, u_bj) = out["none"], out["bj"]
    du = np.abs(u_bj - u0.cpu().numpy()).max(axis=(0, 2))
    diff = np.abs(u_none - u_bj).max(axis=(0, 2))
    assert np.all(diff <= 5e-3 * du + 1e-12), (diff, du)
    assert sum(s1["gmres"]) * 10 < sum(s0["gmres"]), (s0, s1)


def test_failures_are_reported_not_hung(torch_cuda):
    """Host-side fault injection: a NaN in the state gives DG_ENAN; an iteration cap of one
    Newton iteration at a large step gives DG_ENOTCONV; the context stays usable."""
    torch = torch_cuda
    from paper_2306_01085_gb300.dg import Mesh
    d = _walled_box(p=1, n=2)
    m = Mesh(d)
    x = m.nodes().cpu().numpy()
    u = torch.from_numpy(W.state_for(d, x, 4)).cuda()
    bad = u.clone()
    bad[3, 1, 2] = float("nan")
    st = m.implicit_step(bad, 0.0, 0.05, check=False)
    assert st["rc"] == -5
    st = m.implicit_step(u.clone(), 0.0, 5.0, max_newton=1, check=False)
    assert st["rc"] == -4
    st = m.implicit_step(u.clone(), 0.0, 0.05, precond="bj")
    assert st["status"] == 0
    m.close()
