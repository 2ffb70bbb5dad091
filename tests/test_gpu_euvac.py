"""EUVAC heating (Sec. 2.2) on the GPU against the oracle: residual and exact Jv at 1e-12 per
variable, the heating actually active, the FP32 variant within its bound, and the descriptor check."""
import numpy as np
import pytest

from oracle import dg as OD
from oracle import mesh as OM
from paper_2306_01085_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    from paper_2306_01085_gb300 import build as B
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    B.build()
    return torch


def _err(gpu, ref):
    g = np.moveaxis(np.asarray(gpu), 1, 0).reshape(5, -1)
    r = np.moveaxis(np.asarray(ref), 1, 0).reshape(5, -1)
    return np.abs(g - r).max(1) / np.maximum(np.abs(r).max(1), 1e-300)


@pytest.mark.parametrize("p,day,t", [(2, 172.0, 0.0), (3, 80.0, 900.0), (1, 355.0, 2500.0)])
def test_euvac_residual_and_jv_match_oracle(torch_cuda, p, day, t):
    """Day side, terminator, lit night side and shadow all occur on a 6x2x2x3 shell; t is in
    nondimensional time units (the Sun moves by euv_omega_t t)."""
    torch = torch_cuda
    from paper_2306_01085_gb300.dg import Mesh
    d = W.shell_desc(n=2, nr=3, p=p, euvac=True, day=day)
    d.h_first = 0.0
    om = OM.OracleMesh(d)
    u = W.state_for(d, om.X, 5)
    v = W.unit_vector(77, u.shape)
    r_ref = OD.residual(om, u, None, t)
    jv_ref = OD.jvp(om, u, v, t)
    m = Mesh(d, nodes=om.X)
    ug, vg = torch.from_numpy(u).cuda(), torch.from_numpy(v).cuda()
    r = m.residual(ug, t=t).cpu().numpy()
    jv = m.jvp(ug, vg, t=t).cpu().numpy()
    r32 = m.residual_f32(ug, t=t).cpu().numpy()
    m.close()
    er, ej, e32 = _err(r, r_ref), _err(jv, jv_ref), _err(r32, r_ref)
    print(f"\np={p} day={day}: r {er}\n  Jv {ej}\n  FP32 r {e32}")
    assert np.all(er <= 1e-12) and np.all(ej <= 1e-12), (er, ej)
    assert np.all(e32 <= 1e-4)
    # the heating is really there: it changes the energy residual by more than the parity bar
    d0 = W.shell_desc(n=2, nr=3, p=p, euvac=False, day=day)
    d0.h_first = 0.0
    r0 = OD.residual(OM.OracleMesh(d0), u, None, t)
    assert np.abs(r0[:, 4] - r_ref[:, 4]).max() > 1e-6 * np.abs(r_ref[:, 4]).max()


def test_euvac_needs_reference_values(torch_cuda):
    from paper_2306_01085_gb300.dg import DgError, Mesh
    d = W.shell_desc(n=1, nr=2, p=1, euvac=True)
    d.ref_T0 = 0.0
    with pytest.raises(DgError):
        Mesh(d)
