"""Reduced-precision variants against the FP64 oracle, and the mixed-precision implicit step.

FP32 storage and arithmetic: the error of r and J v is reported per
variable as max|x - x_ref| / max|x_ref| and held to 1e-4 (about 1700 eps_32). Two conditioning
factors multiply eps_32 = 2^-24: the cancellation between the volume, source and face terms of
the residual (printed as kappa; up to ~220 where pressure balances gravity), and the rounding of
the LDG gradient of a variable with a large mean (sqrt(rho) T), which grows like |u| / (h |grad u|)
and feeds the heat flux. Measured on GB300: box residual <= 1.7e-5, Jv <= 2.4e-7; p = 3 shell
residual <= 1.5e-5, Jv <= 6.6e-6.
"""
import numpy as np
import pytest

from oracle import dg as OD
from oracle import mesh as OM
from paper_2306_01085_gb300 import workloads as W

pytestmark = pytest.mark.gpu
EPS32 = 2.0 ** -24


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    from paper_2306_01085_gb300 import build as B
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    B.build()
    return torch


def _per_var(x, ref):
    g = np.moveaxis(x, 1, 0).reshape(5, -1)
    r = np.moveaxis(ref, 1, 0).reshape(5, -1)
    return np.abs(g - r).max(1) / np.abs(r).max(1)


def _cancellation(om, u, t):
    """kappa per variable: max over nodes of |volume flux term| + |source term| + |face term| of the
    residual (Eq. DGformulation b, each tested against the nodal basis), over max |r|."""
    from oracle import physics as P
    C = P.Coeffs(om.desc)
    q = OD.gradient(om, u)
    uG = np.moveaxis(np.einsum("gi,eci->ecg", om.phi, u), 0, 1)
    qG = np.moveaxis(np.einsum("gi,edci->edcg", om.phi, q), 0, 2)
    F = P.flux(uG, qG, C)
    s = P.source(uG, qG, np.moveaxis(om.xG, 1, 0), t, C)
    Wd = om.W[None, :] * om.detJ
    vol = np.einsum("eg,cdeg,egad,gai->eci", Wd, F, om.Jinv, om.dphi, optimize=True)
    src = np.einsum("eg,ceg,gi->eci", Wd, s, om.phi)
    fh = OD.face_fluxes(om, u, q, np.arange(om.n_elem), C)
    face = sum(np.abs(np.einsum("f,ecf,fi->eci", om.wF, fh[:, f], om.phiF[f])) for f in range(6))
    r = vol + src - sum(np.einsum("f,ecf,fi->eci", om.wF, fh[:, f], om.phiF[f]) for f in range(6))
    mag = (np.abs(vol) + np.abs(src) + face).max(axis=(0, 2))
    return mag / np.abs(r).max(axis=(0, 2))


@pytest.mark.parametrize("case", ["box4_p2", "shell_p3"])
def test_fp32_residual_and_jv_errors(torch_cuda, case):
    torch = torch_cuda
    from paper_2306_01085_gb300.dg import Mesh
    if case == "box4_p2":
        d = W.CONFIGS["box4_p2"][0]()
    else:
        d = W.shell_desc(n=3, nr=6, p=3, euv=True)
    om = OM.OracleMesh(d)
    u = W.state_for(d, om.X, 3)
    v = W.unit_vector(13, u.shape)
    r_ref = OD.residual(om, u, None, 0.1)
    jv_ref = OD.jvp(om, u, v, 0.1)
    m = Mesh(d, nodes=om.X)
    ug = torch.from_numpy(u).cuda()
    vg = torch.from_numpy(v).cuda()
    r32 = m.residual_f32(ug, t=0.1).cpu().numpy()
    r2 = torch.empty_like(ug)
    jv32 = m.jvp_f32(ug, vg, t=0.1, r_out=r2).cpu().numpy()
    m.close()
    e_r, e_j = _per_var(r32, r_ref), _per_var(jv32, jv_ref)
    e_r2 = _per_var(r2.cpu().numpy(), r_ref)
    print(f"\n{case}: FP32 residual rel. error per variable {e_r}\n{case}: FP32 Jv rel. error per variable {e_j}")
    # the residual of the fused tangent pass is an FP32 evaluation of the same quantity, rounded
    # differently: as accurate as the plain FP32 residual
    assert np.all(e_r2 <= 1.5 * e_r + 1e-9), (e_r2, e_r)
    kappa = _cancellation(om, u, 0.1)
    print(f"{case}: cancellation factor per variable {kappa}")
    assert np.all(e_r <= 1e-4), (e_r, kappa)
    assert np.all(e_j <= 1e-4), e_j
    assert np.all(e_r > 0)   # really FP32 (not the FP64 path)


def test_mixed_precision_step_matches_plain_step(torch_cuda):
    """FP32 inner Jv, FP32-assembled blocks and FP32 Gram-Schmidt arithmetic only change the Krylov
    iterations: the Newton residual is FP64, so the converged state equals the plain FP64 step to
    the Newton tolerance, and the GMRES iteration count stays within 10 % of the plain one."""
    torch = torch_cuda
    from paper_2306_01085_gb300.dg import Mesh
    d = W.shell_desc(n=3, nr=6, p=2, euv=True)
    m = Mesh(d)
    u0 = torch.from_numpy(W.state_for(d, m.nodes().cpu().numpy(), 8)).cuda()
    dt = 60.0 / W.shell_reference().t0
    res = {}
    for prec in ("f64", "f32"):
        u = u0.clone()
        res[prec] = (m.implicit_step(u, 0.0, dt, stages=3, precond="bj", jv_prec=prec), u.cpu().numpy())
    m.close()
    du = np.abs(res["f64"][1] - u0.cpu().numpy()).max(axis=(0, 2))
    diff = np.abs(res["f64"][1] - res["f32"][1]).max(axis=(0, 2))
    print("\nmixed vs plain:", diff / du, res["f64"][0]["gmres"], res["f32"][0]["gmres"])
    assert np.all(diff <= 1e-4 * du), (diff, du)
    g64, g32 = sum(res["f64"][0]["gmres"]), sum(res["f32"][0]["gmres"])
    assert abs(g32 - g64) <= 0.1 * g64, (g64, g32)


@pytest.mark.parametrize("case", ["box4_p2", "shell_p2_euv"])
def test_contraction_precision_modes(torch_cuda, case):
    """Basis contractions with bfloat16 / binary16 operands and FP32 accumulation (the arithmetic
    of a tensor-core MMA), with and without hi + lo splits, against the FP64 oracle. Reported per
    variable; held to what the arithmetic fixes: the FP32 mode is the FP32 variant bit for bit,
    one-term bfloat16 is at least as wrong as FP32, the fused pass's residual is as accurate as
    the plain one, and the three-product split recovers most of
    the lost digits (its operands carry 16 bits, so its error is at most 2^-7 of the one-term
    error plus the FP32 floor)."""
    torch = torch_cuda
    from paper_2306_01085_gb300.dg import Mesh
    if case == "box4_p2":
        d = W.CONFIGS["box4_p2"][0]()
    else:
        d = W.shell_desc(n=3, nr=6, p=2, euv=True)
    om = OM.OracleMesh(d)
    u = W.state_for(d, om.X, 3)
    v = W.unit_vector(13, u.shape)
    r_ref = OD.residual(om, u, None, 0.1)
    jv_ref = OD.jvp(om, u, v, 0.1)
    m = Mesh(d, nodes=om.X)
    ug = torch.from_numpy(u).cuda()
    vg = torch.from_numpy(v).cuda()
    r32 = m.residual_f32(ug, t=0.1).cpu().numpy()
    err = {}
    for mode in ("fp32", "bf16", "fp16", "bf16x3", "fp16x3"):
        r, _ = m.eval_precision(mode, ug, t=0.1)
        r2, jv = m.eval_precision(mode, ug, vg, t=0.1, r=torch.empty_like(ug))
        r, r2, jv = r.cpu().numpy(), r2.cpu().numpy(), jv.cpu().numpy()
        if mode == "fp32":
            assert np.array_equal(r, r32)
        with np.errstate(invalid="ignore"):
            err[mode] = (_per_var(r, r_ref), _per_var(jv, jv_ref))
            if mode == "fp32":   # the fused pass's residual: same accuracy, its own rounding
                assert np.all(_per_var(r2, r_ref) <= 1.5 * err[mode][0] + 1e-9)
        print(f"\n{case} {mode:7s} r {err[mode][0]}\n{case} {mode:7s} Jv {err[mode][1]}")
    m.close()
    for k in (0, 1):
        e32, e16, e3 = err["fp32"][k], err["bf16"][k], err["bf16x3"][k]
        assert np.all(np.isfinite(e16)) and np.all(np.isfinite(e3))
        assert e16.max() >= e32.max()
        assert np.all(e3 <= e16 / 128 + 4 * e32 + 1e-7), (e3, e16, e32)
