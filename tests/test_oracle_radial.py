"""Pins of the radial 1D oracle (oracle/radial.py), the spherically symmetric reading of the model
the paper runs in Sec. 4.3.

  * The 1D flux and source are the 3D oracle physics (pinned against the Navier-Stokes system,
    Eq. NS1) evaluated on symmetric fields: the 3D flux of every variable at a symmetric state is
    radial for the scalars and of the form F_rr r_hat r_hat + F_tt (I - r_hat r_hat) for the
    momentum, with the 1D values; the 3D source is radial with the 1D value (rotation off).
  * Free stream (uniform state at rest, no gravity or heating) gives r = 0 on the curved column: the
    tangential pressure term 2 F_tt / r balances the r^2-weighted flux exactly.
  * The isothermal hydrostatic column varrho = varrho0 + (m g_r0^2/T)(1/r - 1/r0) converges to
    rest at rate >= p under h-refinement.
  * The complex-step Jv matches central differences and is linear in v.
  * The DIRK(2,2) step converges at second order in dt.
Each pin fails on a planted mistake (dropped hoop term, wrong sign of the face term, first-order
tableau)."""
import math

import numpy as np
import pytest

from oracle import physics as P3
from oracle import radial as R
from paper_2306_01085_gb300 import workloads as W


def _desc(n_elem=6, p=2, euvac=True, h_first_km=2.5):
    return W.radial_desc(n_col=1, n_elem=n_elem, p=p, euvac=euvac, h_first_km=h_first_km)


def _mesh3d_desc(d):
    """A shell descriptor with the same physics, no rotation (the 3D oracle's coefficients)."""
    m = W.MeshDesc(kind=1, p=d.p, nx=1, ny=1, nz=1, r_inner=d.r_inner, r_outer=d.r_outer, gamma=d.gamma,
                   grashof=d.grashof, prandtl=d.prandtl, mass=d.mass, visc_exp=d.visc_exp, lambda0=d.lambda0,
                   t_wall=d.t_wall, gravity_kind=1, g_r0=d.g_r0, euv=d.euv, euv_omega_t=d.euv_omega_t,
                   euv_day=d.euv_day, euv_f107=d.euv_f107, euv_f107a=d.euv_f107a, euv_eff=0.3,
                   euv_dsun=d.euv_dsun, ref_T0=d.ref_T0, ref_rho0=d.ref_rho0, ref_m=d.ref_m, ref_g0=d.ref_g0)
    return m


def test_reduced_physics_is_the_3d_physics_on_symmetric_fields():
    d = _desc()
    C1 = R.Coeffs(d)
    C3 = P3.Coeffs(_mesh3d_desc(d))
    rng = np.random.default_rng(3)
    for trial in range(6):
        lat, lon = rng.uniform(-1.4, 1.4), rng.uniform(-3.1, 3.1)
        n = R._unit(lat, lon)
        r = d.r_inner + rng.uniform(0, d.r_outer - d.r_inner)
        u1 = np.array([rng.uniform(-11, 0), rng.normal() * 0.01, rng.uniform(0.01, 3.0)])
        q1 = rng.normal(size=4) * 0.05
        u3 = np.array([u1[0], u1[1] * n[0], u1[1] * n[1], u1[1] * n[2], u1[2]])
        q3 = np.zeros((3, 5))
        q3[:, 0] = q1[0] * n
        for c in range(3):
            for dd in range(3):
                q3[dd, 1 + c] = q1[1] * n[c] * n[dd] + q1[2] * ((c == dd) - n[c] * n[dd])
        q3[:, 4] = q1[3] * n
        x = r * n
        F1, Ftt = R.flux(u1, q1, r, C1, 1.0)
        F3 = P3.flux(u3, q3, C3, True, x)
        assert np.allclose(F3[0], F1[0] * n, rtol=1e-13, atol=1e-15 * abs(F1[0]) + 1e-300)
        assert np.allclose(F3[4], F1[2] * n, rtol=1e-12, atol=1e-13 * np.abs(F3[4]).max())
        Fm = F3[1:4]
        want = F1[1] * np.outer(n, n) + Ftt * (np.eye(3) - np.outer(n, n))
        assert np.abs(Fm - want).max() <= 1e-12 * np.abs(want).max()
        s1 = R.source(u1, q1, r, 0.37, C1, 1.0, 0.3, n)
        s3 = P3.source(u3, q3, x, 0.37, C3)
        assert abs(s3[0] - s1[0]) <= 1e-12 * abs(s1[0]) + 1e-300
        assert np.abs(s3[1:4] - s1[1] * n).max() <= 1e-12 * np.abs(s3[1:4]).max()
        assert abs(s3[4] - s1[2]) <= 1e-12 * abs(s1[2])


def test_conductivity_factor_scales_the_conduction_flux():
    d = _desc()
    C1 = R.Coeffs(d)
    u1 = np.array([-3.0, 0.002, 1.4])
    q1 = np.array([-0.3, 0.01, 0.001, 0.04])
    F_1, _ = R.flux(u1, q1, d.r_inner + 5.0, C1, 1.0)
    F_a, _ = R.flux(u1, q1, d.r_inner + 5.0, C1, 0.625)
    adv = u1[2] * u1[1] * math.exp(-0.5 * u1[0])
    assert abs((F_a[2] - adv) - 0.625 * (F_1[2] - adv)) < 1e-14 * abs(F_1[2])


def _free_stream(d):
    d.g_r0, d.euv = 0.0, 0
    C = R.Coeffs(d)
    mesh = R.RadialMesh(d, W.radial_nodes(d))
    u = np.zeros((3, d.n_elem, d.p + 1))
    u[0] = -2.0
    u[2] = math.exp(-1.0) * d.t_wall          # T = T_wall so the wall trace equals the state
    return mesh, u, C


@pytest.mark.parametrize("p", [1, 2, 3])
def test_free_stream_is_exact(p):
    d = _desc(p=p)
    mesh, u, C = _free_stream(d)
    r = R.residual(mesh, u, 0.0, C, (0.25, 1.0, 0.0, 0.0))
    pressure_scale = (mesh.rR.max() ** 2) * u[2].max() / d.gamma
    assert np.abs(r).max() <= 1e-13 * pressure_scale, np.abs(r).max() / pressure_scale


def test_free_stream_catches_a_dropped_hoop_term(monkeypatch):
    d = _desc(p=2)
    mesh, u, C = _free_stream(d)
    orig = R.flux
    monkeypatch.setattr(R, "flux", lambda *a, **k: (orig(*a, **k)[0], 0.0 * orig(*a, **k)[1]))
    r = R.residual(mesh, u, 0.0, C, (0.25, 1.0, 0.0, 0.0))
    pressure_scale = (mesh.rR.max() ** 2) * u[2].max() / d.gamma
    assert np.abs(r).max() > 1e-3 * pressure_scale


def _hydrostatic_rates(E_list, p, monkeypatch=None):
    errs = []
    for E in E_list:
        d = W.radial_desc(n_col=1, n_elem=E, p=p, euvac=False, h_first_km=0.0)
        d.r_outer = d.r_inner + 8.0
        C = R.Coeffs(d)
        mesh = R.RadialMesh(d, W.radial_nodes(d))
        r = W.radial_nodes(d)
        T = 1.0
        vr = (d.mass * d.g_r0 ** 2 / T) * (1.0 / r - 1.0 / d.r_inner)
        u = np.zeros((3, E, p + 1))
        u[0] = vr
        u[2] = np.exp(0.5 * vr) * T
        res = R.residual(mesh, u, 0.0, C, (0.25, 1.0, 0.0, 0.0))
        dudt = np.linalg.solve(mesh.M[None], res[..., None])[..., 0]
        errs.append(np.abs(dudt).max())
    return np.array(errs)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_isothermal_hydrostatic_column_converges(p):
    """du/dt = M^{-1} r of the exact isothermal column goes to zero at rate p (the interpolated
    exponential profile is not in the discrete space, as in the shell pin)."""
    errs = _hydrostatic_rates([8, 16, 32, 64], p)
    rates = np.log2(errs[:-1] / errs[1:])
    assert np.all(rates >= p - 0.2) and rates[-1] >= p - 0.05, (errs, rates)


def test_hydrostatic_pin_catches_a_face_term_sign(monkeypatch):
    orig = R.face_fluxes
    monkeypatch.setattr(R, "face_fluxes", lambda *a, **k: -orig(*a, **k))
    errs = _hydrostatic_rates([8, 16, 32], 2)
    assert errs[-1] > 1e-2


def test_complex_step_jv_against_central_differences():
    d = _desc(n_elem=8)
    C = R.Coeffs(d)
    mesh = R.RadialMesh(d, W.radial_nodes(d))
    u = W.radial_state(d)[..., 0]
    params = W.radial_params(1)[0]
    v = W.unit_vector(5, u.shape)
    w = W.unit_vector(6, u.shape)
    jv = R.jvp(mesh, u, v, 0.3, C, params)
    h = 1e-6
    fd = (R.residual(mesh, u + h * v, 0.3, C, params) - R.residual(mesh, u - h * v, 0.3, C, params)) / (2 * h)
    assert np.abs(fd - jv).max() <= 1e-8 * np.abs(jv).max()
    lin = R.jvp(mesh, u, 2.0 * v - 3.0 * w, 0.3, C, params)
    assert np.abs(lin - (2.0 * jv - 3.0 * R.jvp(mesh, u, w, 0.3, C, params))).max() <= 1e-12 * np.abs(lin).max()


def _step_error(stages_fn):
    d = _desc(n_elem=4, euvac=False)
    C = R.Coeffs(d)
    mesh = R.RadialMesh(d, W.radial_nodes(d))
    u0 = W.radial_state(d)[..., 0]
    params = (0.25, 1.0, 0.0, 0.0)
    T = 2.0

    def run(n):
        u = u0.copy()
        for k in range(n):
            u, _ = stages_fn(mesh, u, k * T / n, T / n, C, params)
        return u
    ref = run(64)
    return [np.abs(run(n) - ref).max() for n in (4, 8)]


def test_dirk22_step_is_second_order():
    e4, e8 = _step_error(lambda m, u, t, dt, C, p: R.implicit_step(m, u, t, dt, C, p, stages=2, tol=1e-12))
    assert 3.0 < e4 / e8 < 5.0, (e4, e8)


def test_order_pin_catches_backward_euler():
    e4, e8 = _step_error(lambda m, u, t, dt, C, p: R.implicit_step(m, u, t, dt, C, p, stages=1, tol=1e-12))
    assert e4 / e8 < 2.5, (e4, e8)
