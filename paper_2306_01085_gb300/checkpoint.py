"""Checkpoint and resume of an implicit time integration.

The paper's runs write the solution at fixed intervals of simulated time (Sec. 4); a run that is
stopped resumes from the last such file. A checkpoint here is one `.npz` file holding:

  * the state u, FP64 [n_elem][5][n_p] (nodal, the library's layout);
  * the mesh description (every field of `workloads.MeshDesc`) and, when the mesh was built from
    input nodes, those nodes [n_elem][3][n_p];
  * the time t (nondimensional) and the step counter;
  * when the learned preconditioner is in use, its network size (hidden width, rank) and parameters.

Resuming continues the integration bit for bit when the preconditioner is built every step, stage
or Newton iteration: a step depends only on u, t, dt and the options. The lagged preconditioner and
the reduced basis carry state from one step to the next that is not saved; after a resume they
rebuild it, which changes iteration counts but not the converged states beyond the Newton tolerance.
"""
from __future__ import annotations

import dataclasses
import json

import numpy as np

from . import workloads as W

FORMAT = 1


def _host(a, dtype):
    arr = a.detach().cpu().numpy() if hasattr(a, "detach") else np.asarray(a)
    if arr.dtype != dtype:
        raise ValueError(f"checkpoint: expected {np.dtype(dtype).name} data, got {arr.dtype}")
    return np.ascontiguousarray(arr)


def save(path, desc: W.MeshDesc, u, t: float, step: int, nodes=None, mlp=None) -> None:
    """Write a checkpoint. u and nodes: torch tensors (any device) or numpy arrays, FP64;
    mlp: None or (hidden, rank, params) with params the FP32 parameter vector of
    `Mesh.mlp_params()`."""
    u = _host(u, np.float64)
    if u.ndim != 3 or u.shape[1] != 5 or u.shape[0] != desc.n_elem or u.shape[2] != desc.n_p:
        raise ValueError(f"checkpoint: u has shape {u.shape}, expected {(desc.n_elem, 5, desc.n_p)}")
    payload = {
        "format": np.int64(FORMAT),
        "desc": np.frombuffer(json.dumps(dataclasses.asdict(desc)).encode(), dtype=np.uint8),
        "u": u,
        "t": np.float64(t),
        "step": np.int64(step),
    }
    if nodes is not None:
        payload["nodes"] = _host(nodes, np.float64)
    if mlp is not None:
        hidden, rank, params = mlp
        payload["mlp_hidden"] = np.int64(hidden)
        payload["mlp_rank"] = np.int64(rank)
        payload["mlp_params"] = _host(params, np.float32)
    with open(path, "wb") as fh:
        np.savez(fh, **payload)


def load(path) -> dict:
    """Read a checkpoint: {"desc", "u", "t", "step", "nodes" (or None), "mlp" (None or
    (hidden, rank, params))}."""
    with np.load(path) as z:
        fmt = int(z["format"])
        if fmt != FORMAT:
            raise ValueError(f"checkpoint: format {fmt}, this reader knows {FORMAT}")
        fields = json.loads(bytes(z["desc"]).decode())
        desc = W.MeshDesc(**{k: tuple(v) if isinstance(v, list) else v for k, v in fields.items()})
        out = {"desc": desc, "u": z["u"].copy(), "t": float(z["t"]), "step": int(z["step"]),
               "nodes": z["nodes"].copy() if "nodes" in z.files else None, "mlp": None}
        if "mlp_params" in z.files:
            out["mlp"] = (int(z["mlp_hidden"]), int(z["mlp_rank"]), z["mlp_params"].copy())
    if out["u"].shape != (desc.n_elem, 5, desc.n_p):
        raise ValueError("checkpoint: state does not match the mesh description")
    return out
