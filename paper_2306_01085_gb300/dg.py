"""Thin Python binding of the C ABI in include/dg.h (argument marshalling only).

Every operation runs in the CUDA library libdg_gb300.so; there is no CPU path. Tensors are torch
CUDA float64 tensors in the layouts documented in include/dg.h; calls are ordered on torch's
current CUDA stream.
"""
from __future__ import annotations

import ctypes
import os
import re

from . import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libdg_gb300.so")
HEADER = os.path.join(HERE, "..", "include", "dg.h")

DG_JV_EXACT = 0
DG_JV_FD = 1
DG_INTERP_FP64 = 0
DG_INTERP_TC = 1


class DgMeshDesc(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32), ("p", ctypes.c_int32), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("nz", ctypes.c_int32), ("bc_lo", ctypes.c_int32), ("bc_hi", ctypes.c_int32),
        ("lx", ctypes.c_double), ("ly", ctypes.c_double), ("lz", ctypes.c_double),
        ("r_inner", ctypes.c_double), ("r_outer", ctypes.c_double), ("h_first", ctypes.c_double),
        ("gamma", ctypes.c_double), ("grashof", ctypes.c_double), ("prandtl", ctypes.c_double),
        ("mass", ctypes.c_double), ("visc_exp", ctypes.c_double), ("lambda0", ctypes.c_double),
        ("t_wall", ctypes.c_double), ("gravity_kind", ctypes.c_int32), ("euv", ctypes.c_int32),
        ("gvec", ctypes.c_double * 3), ("g_r0", ctypes.c_double), ("omega", ctypes.c_double * 3),
        ("froude", ctypes.c_double), ("euv_amp", ctypes.c_double), ("euv_sigma", ctypes.c_double),
        ("euv_r_peak", ctypes.c_double), ("euv_width", ctypes.c_double), ("euv_omega_t", ctypes.c_double),
        ("euv_day", ctypes.c_double), ("euv_f107", ctypes.c_double), ("euv_f107a", ctypes.c_double),
        ("euv_eff", ctypes.c_double), ("euv_dsun", ctypes.c_double), ("ref_T0", ctypes.c_double),
        ("ref_rho0", ctypes.c_double), ("ref_m", ctypes.c_double), ("ref_g0", ctypes.c_double),
        ("comp", ctypes.c_int32), ("reserved_comp", ctypes.c_int32), ("comp_a", ctypes.c_double * 6),
        ("comp_b", ctypes.c_double * 6), ("eddy_nu", ctypes.c_double), ("eddy_alpha", ctypes.c_double),
    ]


class DgSolverOpts(ctypes.Structure):
    _fields_ = [
        ("stages", ctypes.c_int32), ("gmres_restart", ctypes.c_int32), ("max_restarts", ctypes.c_int32),
        ("max_newton", ctypes.c_int32), ("precond", ctypes.c_int32), ("precond_refresh", ctypes.c_int32),
        ("jv_mode", ctypes.c_int32), ("jv_prec", ctypes.c_int32), ("newton_rtol", ctypes.c_double),
        ("gmres_rtol", ctypes.c_double), ("abs_floor", ctypes.c_double), ("rb_size", ctypes.c_int32),
        ("flags", ctypes.c_int32), ("refresh_every", ctypes.c_int32), ("reserved", ctypes.c_int32),
    ]


class DgStepStats(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int32), ("newton_iters", ctypes.c_int32 * 3), ("gmres_iters", ctypes.c_int32 * 3),
        ("n_hist", ctypes.c_int32), ("res_hist", ctypes.c_double * 64), ("wall_ms", ctypes.c_double),
        ("precond_ms", ctypes.c_double),
    ]


PC = {"none": 0, "bj": 1, "mlp": 2, "rb": 3, "rb_bj": 4, "bj16": 5}
REFRESH = {"step": 0, "stage": 1, "newton": 2, "lagged": 3}

_lib = None


def declared_functions():
    """Names of the functions declared in include/dg.h."""
    with open(HEADER) as fh:
        text = fh.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(dg_[a-z_0-9]+)\s*\(", text, flags=re.M)))


def lib():
    """Load libdg_gb300.so (raises if it was not built: the library has no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library missing at {LIB_PATH}; run paper_2306_01085_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, dp, i32, i64p, d = ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64), ctypes.c_double
    L.dg_last_error.restype = ctypes.c_char_p
    L.dg_mesh_create.argtypes = [ctypes.POINTER(DgMeshDesc), vp, ctypes.POINTER(vp)]
    L.dg_mesh_destroy.argtypes = [vp]
    L.dg_mesh_destroy.restype = None
    L.dg_mesh_sizes.argtypes = [vp, i64p, ctypes.POINTER(ctypes.c_int32), i64p]
    L.dg_mesh_nodes.argtypes = [vp, dp, vp]
    L.dg_mesh_set_interp.argtypes = [vp, i32]
    L.dg_gradient.argtypes = [vp, dp, dp, vp]
    L.dg_residual.argtypes = [vp, dp, dp, d, dp, vp]
    L.dg_jvp.argtypes = [vp, dp, dp, d, i32, d, dp, dp, vp]
    L.dg_mass_apply.argtypes = [vp, dp, dp, vp]
    L.dg_profile_start.argtypes = [vp, i32]
    L.dg_profile_stop.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32), i64p]
    L.dg_kernel_name.argtypes = [i32]
    L.dg_kernel_name.restype = ctypes.c_char_p
    L.dg_probe_fp64.argtypes = [ctypes.POINTER(ctypes.c_double)]
    L.dg_residual_f32.argtypes = [vp, dp, d, dp, vp]
    L.dg_jvp_f32.argtypes = [vp, dp, dp, d, dp, dp, vp]
    L.dg_mlp_init.argtypes = [vp, i32, i32, ctypes.c_int64, ctypes.c_uint64]
    L.dg_mlp_sizes.argtypes = [vp, i64p, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32), i64p]
    L.dg_mlp_params.argtypes = [vp, dp, dp, vp]
    L.dg_mlp_features.argtypes = [vp, dp, d, dp, dp, vp]
    L.dg_mlp_harvest.argtypes = [vp, dp, d, d, i32, i64p, vp]
    L.dg_mlp_loss_grad.argtypes = [vp, dp, dp, i32, ctypes.POINTER(ctypes.c_double), dp, vp]
    L.dg_mlp_train.argtypes = [vp, i32, i32, d, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), vp]
    L.dg_solver_opts_default.argtypes = [ctypes.POINTER(DgSolverOpts)]
    L.dg_solver_opts_default.restype = None
    L.dg_dirk_tableau.argtypes = [i32, dp, dp]
    L.dg_implicit_step.argtypes = [vp, dp, d, d, ctypes.POINTER(DgSolverOpts), ctypes.POINTER(DgStepStats), vp]
    L.dg_precond_setup.argtypes = [vp, i32, dp, d, d, vp]
    L.dg_precond_apply.argtypes = [vp, i32, dp, dp, vp]
    L.dg_block_assemble.argtypes = [vp, dp, d, d, dp, vp]
    L.dg_eval_precision.argtypes = [vp, i32, dp, dp, d, dp, dp, vp]
    L.dg_mass_inverse_apply.argtypes = [vp, dp, dp, vp]
    L.dg_rb_load.argtypes = [vp, dp, i32, dp, d, d, i32, vp]
    L.dg_rb_initial_guess.argtypes = [vp, dp, dp, vp]
    L.dg_rb_reset.argtypes = [vp]
    _lib = L
    return L


class DgError(RuntimeError):
    pass


def _check(rc):
    if rc != 0:
        raise DgError(f"dg error {rc}: {lib().dg_last_error().decode()}")


def to_c_desc(desc: W.MeshDesc) -> DgMeshDesc:
    c = DgMeshDesc()
    for name, _ in DgMeshDesc._fields_:
        if name == "reserved_comp":
            continue
        val = getattr(desc, name)
        if name in ("gvec", "omega", "comp_a", "comp_b"):
            getattr(c, name)[:] = [float(x) for x in val]
        else:
            setattr(c, name, val)
    return c


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t, shape=None, name="tensor"):
    import torch
    if t is None:
        return None
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise DgError(f"{name} must be a contiguous float64 CUDA tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise DgError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return ctypes.c_void_p(t.data_ptr())


class Mesh:
    """A library mesh: geometry, connectivity and workspace on the current CUDA device."""

    def __init__(self, desc: W.MeshDesc, nodes=None):
        """nodes: optional numpy array [n_elem][3][n_p] of node coordinates (the mesh as input);
        None lets the library generate the workload mesh from desc."""
        import numpy as np
        self.desc = desc
        self._c = to_c_desc(desc)
        h = ctypes.c_void_p()
        nptr = None
        if nodes is not None:
            self._nodes = np.ascontiguousarray(nodes, dtype=np.float64)
            if self._nodes.shape != (desc.n_elem, 3, desc.n_p):
                raise DgError(f"nodes has shape {self._nodes.shape}, expected {(desc.n_elem, 3, desc.n_p)}")
            nptr = ctypes.c_void_p(self._nodes.ctypes.data)
        _check(lib().dg_mesh_create(ctypes.byref(self._c), nptr, ctypes.byref(h)))
        self._nodes = None
        self._h = h
        ne, npe, nd = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int64()
        _check(lib().dg_mesh_sizes(h, ctypes.byref(ne), ctypes.byref(npe), ctypes.byref(nd)))
        self.n_elem, self.n_p, self.n_dof = ne.value, npe.value, nd.value
        self.u_shape = (self.n_elem, 5, self.n_p)
        self.q_shape = (self.n_elem, 3, 5, self.n_p)

    def close(self):
        if getattr(self, "_h", None):
            lib().dg_mesh_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def empty(self, shape=None):
        import torch
        return torch.empty(shape or self.u_shape, dtype=torch.float64, device="cuda")

    def set_interp(self, mode):
        """'fp64' (sum-factorised FP64 passes) or 'tc' (tensor-core contraction with FP64-accurate
        digit slicing) for the nodes -> Gauss values and face traces step of the FP64 paths."""
        modes = {"fp64": DG_INTERP_FP64, "tc": DG_INTERP_TC}
        if mode not in modes:
            raise DgError(f"unknown interpolation mode {mode!r}")
        _check(lib().dg_mesh_set_interp(self._h, modes[mode]))
        self.interp = mode

    def nodes(self):
        x = self.empty((self.n_elem, 3, self.n_p))
        _check(lib().dg_mesh_nodes(self._h, _ptr(x), _stream()))
        return x

    def gradient(self, u, out=None):
        q = out if out is not None else self.empty(self.q_shape)
        _check(lib().dg_gradient(self._h, _ptr(u, self.u_shape, "u"), _ptr(q, self.q_shape, "q"), _stream()))
        return q

    def residual(self, u, q=None, t=0.0, out=None):
        r = out if out is not None else self.empty()
        _check(lib().dg_residual(self._h, _ptr(u, self.u_shape, "u"), _ptr(q, self.q_shape, "q"), float(t),
                                 _ptr(r, self.u_shape, "r"), _stream()))
        return r

    def jvp(self, u, v, t=0.0, mode="exact", eps=0.0, out=None, r_out=None):
        jv = out if out is not None else self.empty()
        m = DG_JV_EXACT if mode == "exact" else DG_JV_FD
        _check(lib().dg_jvp(self._h, _ptr(u, self.u_shape, "u"), _ptr(v, self.u_shape, "v"), float(t), m,
                            float(eps), _ptr(jv, self.u_shape, "jv"), _ptr(r_out, self.u_shape, "r_out"),
                            _stream()))
        return jv

    def mass(self, v, out=None):
        mv = out if out is not None else self.empty()
        _check(lib().dg_mass_apply(self._h, _ptr(v, self.u_shape, "v"), _ptr(mv, self.u_shape, "mv"), _stream()))
        return mv

    def mass_inverse(self, v, out=None):
        mv = out if out is not None else self.empty()
        _check(lib().dg_mass_inverse_apply(self._h, _ptr(v, self.u_shape, "v"), _ptr(mv, self.u_shape, "mv"),
                                           _stream()))
        return mv

    # -- tracing ---------------------------------------------------------------------------
    def profile_start(self, capacity=4096):
        _check(lib().dg_profile_start(self._h, int(capacity)))

    def profile_stop(self, n_kinds=32):
        """Per kernel kind: (total device ms, launches) of the traced launches, and total launches."""
        ms = (ctypes.c_double * n_kinds)()
        cnt = (ctypes.c_int32 * n_kinds)()
        tot = ctypes.c_int64()
        _check(lib().dg_profile_stop(self._h, n_kinds, ms, cnt, ctypes.byref(tot)))
        out = {}
        for k in range(n_kinds):
            name = lib().dg_kernel_name(k).decode()
            if name and cnt[k]:
                out[name] = (ms[k], cnt[k])
        return out, tot.value


def probe_fp64():
    """Achieved FP64 FMA throughput of the device in TFLOP/s (library probe kernel)."""
    t = ctypes.c_double()
    _check(lib().dg_probe_fp64(ctypes.byref(t)))
    return t.value


def solver_opts(**kw):
    """dg_solver_opts with the library defaults, overridden by keyword (precond and
    precond_refresh accept the names of PC / REFRESH)."""
    o = DgSolverOpts()
    lib().dg_solver_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        if k == "precond" and isinstance(v, str):
            v = PC[v]
        if k == "precond_refresh" and isinstance(v, str):
            v = REFRESH[v]
        if k == "jv_mode" and isinstance(v, str):
            v = DG_JV_EXACT if v == "exact" else DG_JV_FD
        if k == "jv_prec" and isinstance(v, str):
            v = 1 if v == "f32" else 0
        setattr(o, k, v)
    return o


def dirk_tableau(stages):
    import numpy as np
    a = np.zeros(stages * stages)
    c = np.zeros(stages)
    _check(lib().dg_dirk_tableau(stages, a.ctypes.data_as(ctypes.c_void_p), c.ctypes.data_as(ctypes.c_void_p)))
    return a.reshape(stages, stages), c


def _stats_dict(st):
    return {"status": st.status, "newton": list(st.newton_iters), "gmres": list(st.gmres_iters),
            "res_hist": list(st.res_hist[: st.n_hist]), "wall_ms": st.wall_ms, "precond_ms": st.precond_ms}


def _mesh_implicit_step(self, u, t, dt, opts=None, check=True, **kw):
    """One DIRK step in place on u; returns the statistics (raises on failure when check)."""
    o = opts if opts is not None else solver_opts(**kw)
    st = DgStepStats()
    rc = lib().dg_implicit_step(self._h, _ptr(u, self.u_shape, "u"), float(t), float(dt), ctypes.byref(o),
                                ctypes.byref(st), _stream())
    if check:
        _check(rc)
    out = _stats_dict(st)
    out["rc"] = rc
    return out


def _mesh_precond_setup(self, kind, u, t, dt_aii):
    _check(lib().dg_precond_setup(self._h, PC[kind] if isinstance(kind, str) else kind,
                                  _ptr(u, self.u_shape, "u"), float(t), float(dt_aii), _stream()))


def _mesh_precond_apply(self, kind, x, out=None):
    y = out if out is not None else self.empty()
    _check(lib().dg_precond_apply(self._h, PC[kind] if isinstance(kind, str) else kind,
                                  _ptr(x, self.u_shape, "x"), _ptr(y, self.u_shape, "y"), _stream()))
    return y


def _mesh_block_assemble(self, u, t, dt_aii):
    """Exact diagonal blocks of J_G as a row-major FP32 tensor [n_elem][5 n_p][5 n_p]."""
    import torch
    nb = 5 * self.n_p
    out = torch.empty((self.n_elem, nb, nb), dtype=torch.float32, device="cuda")
    _check(lib().dg_block_assemble(self._h, _ptr(u, self.u_shape, "u"), float(t), float(dt_aii),
                                   ctypes.c_void_p(out.data_ptr()), _stream()))
    return out.transpose(1, 2)


Mesh.implicit_step = _mesh_implicit_step
Mesh.precond_setup = _mesh_precond_setup
Mesh.precond_apply = _mesh_precond_apply
Mesh.block_assemble = _mesh_block_assemble


def _mesh_residual_f32(self, u, t=0.0, out=None):
    """FP32 residual (FP64 in and out)."""
    r = out if out is not None else self.empty()
    _check(lib().dg_residual_f32(self._h, _ptr(u, self.u_shape, "u"), float(t), _ptr(r, self.u_shape, "r"), _stream()))
    return r


def _mesh_jvp_f32(self, u, v, t=0.0, out=None, r_out=None):
    """FP32 exact Jv (and residual when r_out is given)."""
    jv = out if out is not None else self.empty()
    _check(lib().dg_jvp_f32(self._h, _ptr(u, self.u_shape, "u"), _ptr(v, self.u_shape, "v"), float(t),
                            _ptr(jv, self.u_shape, "jv"), _ptr(r_out, self.u_shape, "r_out"), _stream()))
    return jv


Mesh.residual_f32 = _mesh_residual_f32
Mesh.jvp_f32 = _mesh_jvp_f32


# -- learned preconditioner -------------------------------------------------------------------
def _fptr(t, name):
    import torch
    if t is None:
        return None
    if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise DgError(f"{name} must be a contiguous float32 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _mesh_mlp_init(self, hidden=256, rank=16, max_samples=0, seed=7):
    _check(lib().dg_mlp_init(self._h, hidden, rank, int(max_samples), int(seed)))


def _mesh_mlp_sizes(self):
    npar, nin, nout, ns = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
    _check(lib().dg_mlp_sizes(self._h, ctypes.byref(npar), ctypes.byref(nin), ctypes.byref(nout), ctypes.byref(ns)))
    return {"n_params": npar.value, "n_in": nin.value, "n_out": nout.value, "n_samples": ns.value}


def _mesh_mlp_params(self, new=None):
    import torch
    out = torch.empty(self.mlp_sizes()["n_params"], dtype=torch.float32, device="cuda")
    _check(lib().dg_mlp_params(self._h, _fptr(out, "out"), _fptr(new, "in"), _stream()))
    return out


def _mesh_mlp_features(self, u, dt_aii):
    import torch
    sz = self.mlp_sizes()
    feat = torch.empty((self.n_elem, sz["n_in"]), dtype=torch.float32, device="cuda")
    sd = torch.empty((self.n_elem, self.n_p), dtype=torch.float32, device="cuda")
    _check(lib().dg_mlp_features(self._h, _ptr(u, self.u_shape, "u"), float(dt_aii), _fptr(feat, "feat"),
                                 _fptr(sd, "sdiag"), _stream()))
    return feat, sd


def _mesh_mlp_harvest(self, u, t, dt_aii, stride=1):
    n = ctypes.c_int64()
    _check(lib().dg_mlp_harvest(self._h, _ptr(u, self.u_shape, "u"), float(t), float(dt_aii), int(stride),
                                ctypes.byref(n), _stream()))
    return n.value


def _mesh_mlp_loss_grad(self, X, Bs):
    import torch
    g = torch.empty(self.mlp_sizes()["n_params"], dtype=torch.float32, device="cuda")
    L = ctypes.c_double()
    _check(lib().dg_mlp_loss_grad(self._h, _fptr(X, "X"), _fptr(Bs, "Bs"), int(X.shape[0]), ctypes.byref(L),
                                  _fptr(g, "grad"), _stream()))
    return L.value, g


def _mesh_mlp_train(self, epochs, batch=512, lr=1e-3):
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(lib().dg_mlp_train(self._h, int(epochs), int(batch), float(lr), ctypes.byref(a), ctypes.byref(b), _stream()))
    return a.value, b.value


Mesh.mlp_init = _mesh_mlp_init
Mesh.mlp_sizes = _mesh_mlp_sizes
Mesh.mlp_params = _mesh_mlp_params
Mesh.mlp_features = _mesh_mlp_features
Mesh.mlp_harvest = _mesh_mlp_harvest
Mesh.mlp_loss_grad = _mesh_mlp_loss_grad
Mesh.mlp_train = _mesh_mlp_train


CM = {"fp32": 0, "bf16": 1, "fp16": 2, "bf16x3": 3, "fp16x3": 4}


def _mesh_eval_precision(self, mode, u, v=None, t=0.0, r=None, jv=None):
    """Residual (v is None) or fused residual + exact Jv with the basis contractions in one of the
    modes of CM; returns (r, jv)."""
    if v is None and r is None:
        r = self.empty()
    if v is not None and jv is None:
        jv = self.empty()
    _check(lib().dg_eval_precision(self._h, CM[mode], _ptr(u, self.u_shape, "u"), _ptr(v, self.u_shape, "v"),
                                   float(t), _ptr(r, self.u_shape, "r"), _ptr(jv, self.u_shape, "jv"), _stream()))
    return r, jv


Mesh.eval_precision = _mesh_eval_precision


def _mesh_rb_load(self, w, u, t, dt_aii, base="rb"):
    """Replace the reduced basis by the rows of w ([r][n_elem][5][n_p] device FP64) and build the
    RB preconditioner at (u, t, dt_aii) over base "rb" (mass) or "rb_bj" (block-Jacobi)."""
    import torch
    r = int(w.shape[0]) if w is not None else 0
    if r and not (w.is_cuda and w.dtype == torch.float64 and w.is_contiguous()
                  and tuple(w.shape[1:]) == tuple(self.u_shape)):
        raise DgError("w must be a contiguous float64 CUDA tensor [r][n_elem][5][n_p]")
    _check(lib().dg_rb_load(self._h, ctypes.c_void_p(w.data_ptr()) if r else None, r, _ptr(u, self.u_shape, "u"),
                            float(t), float(dt_aii), PC[base], _stream()))


def _mesh_rb_initial_guess(self, b, out=None):
    x0 = out if out is not None else self.empty()
    _check(lib().dg_rb_initial_guess(self._h, _ptr(b, self.u_shape, "b"), _ptr(x0, self.u_shape, "x0"), _stream()))
    return x0


def _mesh_rb_reset(self):
    _check(lib().dg_rb_reset(self._h))


Mesh.rb_load = _mesh_rb_load
Mesh.rb_initial_guess = _mesh_rb_initial_guess
Mesh.rb_reset = _mesh_rb_reset


# ----------------------------------------------------------------------------------------------
# radial 1D ensemble (dg_radial_* in include/dg.h)
# ----------------------------------------------------------------------------------------------
class DgRadialDesc(ctypes.Structure):
    _fields_ = [
        ("p", ctypes.c_int32), ("n_elem", ctypes.c_int32), ("n_col", ctypes.c_int32), ("euv", ctypes.c_int32),
        ("bc_lo", ctypes.c_int32), ("bc_hi", ctypes.c_int32),
        ("r_inner", ctypes.c_double), ("r_outer", ctypes.c_double), ("h_first", ctypes.c_double),
        ("gamma", ctypes.c_double), ("grashof", ctypes.c_double), ("prandtl", ctypes.c_double),
        ("mass", ctypes.c_double), ("visc_exp", ctypes.c_double), ("lambda0", ctypes.c_double),
        ("t_wall", ctypes.c_double), ("g_r0", ctypes.c_double),
        ("euv_omega_t", ctypes.c_double), ("euv_day", ctypes.c_double), ("euv_f107", ctypes.c_double),
        ("euv_f107a", ctypes.c_double), ("euv_dsun", ctypes.c_double),
        ("ref_T0", ctypes.c_double), ("ref_rho0", ctypes.c_double), ("ref_m", ctypes.c_double),
        ("ref_g0", ctypes.c_double),
    ]


class DgRadialStats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("newton_iters", ctypes.c_int32 * 3), ("max_ratio", ctypes.c_double),
                ("wall_ms", ctypes.c_double)]


def _radial_lib():
    L = lib()
    if getattr(L, "_radial_ready", False):
        return L
    vp, dp, i32, d = ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_double
    i64p = ctypes.POINTER(ctypes.c_int64)
    L.dg_radial_create.argtypes = [ctypes.POINTER(DgRadialDesc), vp, vp, ctypes.POINTER(vp)]
    L.dg_radial_destroy.argtypes = [vp]
    L.dg_radial_destroy.restype = None
    L.dg_radial_sizes.argtypes = [vp, i64p, ctypes.POINTER(ctypes.c_int32), i64p]
    L.dg_radial_residual.argtypes = [vp, dp, d, dp, vp]
    L.dg_radial_jvp.argtypes = [vp, dp, dp, d, dp, dp, vp]
    L.dg_radial_step.argtypes = [vp, dp, d, d, i32, d, i32, ctypes.POINTER(DgRadialStats), vp]
    L.dg_radial_profile_start.argtypes = [vp, i32]
    L.dg_radial_profile_stop.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32),
                                         i64p]
    L.dg_radial_kernel_name.argtypes = [i32]
    L.dg_radial_kernel_name.restype = ctypes.c_char_p
    L._radial_ready = True
    return L


class Radial:
    """A library radial ensemble: n_col independent columns on one radial mesh (current device).
    State tensors are float64 [3][n_elem][p+1][n_col] (column index fastest)."""

    def __init__(self, desc: W.RadialDesc, params, node_r=None):
        """params: numpy [n_col][4] = (epsilon, alpha0, latitude, longitude); node_r: optional numpy
        [n_elem][p+1] node radii (None: the library's geometric layers)."""
        import numpy as np
        L = _radial_lib()
        self.desc = desc
        c = DgRadialDesc()
        for name, _ in DgRadialDesc._fields_:
            setattr(c, name, getattr(desc, name))
        self._c = c
        prm = np.ascontiguousarray(params, dtype=np.float64)
        if prm.shape != (desc.n_col, 4):
            raise DgError(f"params has shape {prm.shape}, expected {(desc.n_col, 4)}")
        nr = None
        if node_r is not None:
            nr = np.ascontiguousarray(node_r, dtype=np.float64)
            if nr.shape != (desc.n_elem, desc.p + 1):
                raise DgError(f"node_r has shape {nr.shape}, expected {(desc.n_elem, desc.p + 1)}")
        h = ctypes.c_void_p()
        _check(L.dg_radial_create(ctypes.byref(c), None if nr is None else ctypes.c_void_p(nr.ctypes.data),
                                  ctypes.c_void_p(prm.ctypes.data), ctypes.byref(h)))
        self._h = h
        nc, nn, nd = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int64()
        _check(L.dg_radial_sizes(h, ctypes.byref(nc), ctypes.byref(nn), ctypes.byref(nd)))
        self.n_col, self.n_node, self.n_dof = nc.value, nn.value, nd.value
        self.u_shape = (3, desc.n_elem, desc.p + 1, self.n_col)

    def close(self):
        if getattr(self, "_h", None):
            _radial_lib().dg_radial_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def empty(self):
        import torch
        return torch.empty(self.u_shape, dtype=torch.float64, device="cuda")

    def residual(self, u, t=0.0, out=None):
        out = self.empty() if out is None else out
        _check(_radial_lib().dg_radial_residual(self._h, _ptr(u, self.u_shape, "u"), float(t),
                                                _ptr(out, self.u_shape, "r"), _stream()))
        return out

    def jvp(self, u, v, t=0.0, out=None, r_out=None):
        out = self.empty() if out is None else out
        _check(_radial_lib().dg_radial_jvp(self._h, _ptr(u, self.u_shape, "u"), _ptr(v, self.u_shape, "v"), float(t),
                                           _ptr(out, self.u_shape, "jv"),
                                           None if r_out is None else _ptr(r_out, self.u_shape, "r_out"), _stream()))
        return out

    def step(self, u, t, dt, stages=2, newton_rtol=1e-8, max_newton=20, check=True):
        """One DIRK step in place on u; returns the statistics (raises on failure when check)."""
        st = DgRadialStats()
        rc = _radial_lib().dg_radial_step(self._h, _ptr(u, self.u_shape, "u"), float(t), float(dt), int(stages),
                                          float(newton_rtol), int(max_newton), ctypes.byref(st), _stream())
        if check:
            _check(rc)
        return {"rc": rc, "status": st.status, "newton": list(st.newton_iters), "max_ratio": st.max_ratio,
                "wall_ms": st.wall_ms}

    def profile_start(self, capacity=4096):
        _check(_radial_lib().dg_radial_profile_start(self._h, capacity))

    def profile_stop(self, n_kinds=16):
        L = _radial_lib()
        ms = (ctypes.c_double * n_kinds)()
        cnt = (ctypes.c_int32 * n_kinds)()
        tot = ctypes.c_int64()
        _check(L.dg_radial_profile_stop(self._h, n_kinds, ms, cnt, ctypes.byref(tot)))
        out = {}
        for k in range(n_kinds):
            name = L.dg_radial_kernel_name(k).decode()
            if name and cnt[k]:
                out[name] = (ms[k], cnt[k])
        return out, tot.value
