"""dg_residual_static: the residual for callers that cannot have the library allocate.

Some applications cannot let a library call cudaMalloc/cudaFree while they run: their own caching
allocator holds the device's memory, or their loop cannot absorb the device synchronisation those
calls may cause. dg_residual_static computes the same residual as dg_residual from a fixed scratch
array inside the library. These tests call it through the C ABI and compare it with dg_residual.
This file is collected last so that a run stopping at the first failure has run everything else.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2306_01085_gb300 import build as B
    from paper_2306_01085_gb300 import dg as DG
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    B.build()
    L = DG.lib()
    L.dg_residual_static.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p,
                                     ctypes.c_void_p]
    L.dg_residual_static.restype = ctypes.c_int
    return torch, DG, L


def _rel_err(a, b):
    a = a.cpu().numpy().transpose(1, 0, 2).reshape(5, -1)
    b = b.cpu().numpy().transpose(1, 0, 2).reshape(5, -1)
    return np.abs(a - b).max(1) / np.abs(b).max(1)


@pytest.mark.parametrize("name,p", [("box", 2), ("shell", 3), ("box", 4), ("comp", 2)])
def test_static_residual_matches_dg_residual_twice(env, name, p):
    """Two calls in a row (different states, so stale scratch from the first would show) agree
    with dg_residual to 1e-12 per variable: a periodic box at p = 2 and p = 4 (64 elements, under
    the 335-element limit of p = 4), an EUV shell at p = 3, and a variable-composition shell whose
    mixture fields reach the kernels through the mesh view."""
    torch, DG, L = env
    from paper_2306_01085_gb300 import workloads as W
    if name == "box":
        desc = W.box_desc(p=p, n=4)
    elif name == "comp":
        desc = W.shell_desc(n=2, nr=2, p=p, euvac=True, day=172.0, composition=True)
        desc.h_first = 0.0        # uniform layers keep the interpolated temperature positive at p = 2
    else:
        desc = W.shell_desc(n=3, nr=2, p=p, euv=True)
    m = DG.Mesh(desc)
    x = m.nodes().cpu().numpy()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, seed in enumerate((1, 2)):
        u = torch.from_numpy(W.state_for(desc, x, seed)).cuda()
        ref = m.residual(u, t=0.25)
        out = torch.full_like(u, float("nan"))
        rc = L.dg_residual_static(m._h, ctypes.c_void_p(u.data_ptr()), 0.25, ctypes.c_void_p(out.data_ptr()), stream)
        assert rc == 0, L.dg_last_error().decode()
        torch.cuda.synchronize()
        err = _rel_err(out, ref)
        assert np.all(err <= 1e-12), (call, err)
    m.close()


def test_static_residual_rejects_meshes_beyond_its_scratch(env):
    torch, DG, L = env
    from paper_2306_01085_gb300 import workloads as W
    desc = W.shell_desc(n=4, nr=4, p=4)       # 384 elements at p = 4: above the 335-element limit
    m = DG.Mesh(desc)
    u = m.empty()
    r = m.empty()
    rc = L.dg_residual_static(m._h, ctypes.c_void_p(u.data_ptr()), 0.0, ctypes.c_void_p(r.data_ptr()), None)
    assert rc == -1
    assert "static scratch holds 16777216 bytes" in L.dg_last_error().decode()
    m.close()
