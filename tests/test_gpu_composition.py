"""Variable composition and eddy transport (Sec. 2.1.1-2.1.2) on the GPU against the oracle:
residual and exact Jv at 1e-12 per variable, alone and with the four-absorber EUVAC heating; the
FP32 variant within its bound; the composition visibly changes the residual."""
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


@pytest.mark.parametrize("p,euvac", [(2, False), (3, False), (2, True)])
def test_composition_residual_and_jv_match_oracle(torch_cuda, p, euvac):
    torch = torch_cuda
    from paper_2306_01085_gb300.dg import Mesh
    d = W.shell_desc(n=2, nr=3, p=p, composition=True, euvac=euvac, day=172.0)
    d.h_first = 0.0
    om = OM.OracleMesh(d)
    u = W.state_for(d, om.X, 9)
    v = W.unit_vector(91, u.shape)
    t = 400.0
    r_ref = OD.residual(om, u, None, t)
    jv_ref = OD.jvp(om, u, v, t)
    m = Mesh(d, nodes=om.X)
    ug, vg = torch.from_numpy(u).cuda(), torch.from_numpy(v).cuda()
    r = m.residual(ug, t=t).cpu().numpy()
    jv = m.jvp(ug, vg, t=t).cpu().numpy()
    r32 = m.residual_f32(ug, t=t).cpu().numpy()
    m.close()
    er, ej, e32 = _err(r, r_ref), _err(jv, jv_ref), _err(r32, r_ref)
    print(f"\np={p} euvac={euvac}: r {er}\n  Jv {ej}\n  FP32 r {e32}")
    assert np.all(er <= 1e-12) and np.all(ej <= 1e-12), (er, ej)
    assert np.all(e32 <= 1e-4), e32
    d0 = W.shell_desc(n=2, nr=3, p=p, composition=False, euvac=euvac, day=172.0)
    d0.h_first = 0.0
    r0 = OD.residual(OM.OracleMesh(d0), u, None, t)
    assert np.abs(r0 - r_ref).max() > 1e-3 * np.abs(r_ref).max()
