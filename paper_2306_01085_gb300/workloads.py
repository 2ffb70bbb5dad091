"""Seeded synthetic workloads: mesh descriptors, physical constants, initial states, random vectors.

This module is the one place both the CUDA path and the CPU oracle take their inputs from. It holds
no arithmetic of the discretisation: no basis, quadrature, geometry, flux or residual. It only
states *which problem* is solved (the domain description, the nondimensional numbers of the model in
Sec. 2.4, the base atmosphere and the seeded perturbations) and draws random numbers. Since both
sides read what it computes, each of its computations is pinned on its own by
tests/test_workload_pins.py: the reference scales (hand values and algebraic identities of the
definitions), the hydrostatic state (a closed form and an independent ODE integration), the
cubed-sphere node map (layer radii, equal angles, cube-diagonal corners) and SplitMix64 (the
reference generator's published outputs).

State functions take node coordinates as an argument, so each side evaluates them on its own mesh
(the oracle on its nodes for parity tests; the benchmark on the library's nodes).

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) used as a counter-based generator: value(seed, i) = mix(seed + (i+1)*phi).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict

import numpy as np

# ----------------------------------------------------------------------------------------------
# SI constants of the thermosphere workloads (Sec. 2; reference values at the lower boundary, Sec. 2.4)
# ----------------------------------------------------------------------------------------------
EUV_GAUSS, EUV_EUVAC = 1, 2  # heating models: sub-solar Gaussian; EUVAC flux with Chapman depths
K_B = 1.380649e-23          # Boltzmann constant [J/K]
AMU = 1.66053906660e-27     # atomic mass unit [kg]
R_EARTH = 6371.0e3          # Earth radius [m]
G_SURFACE = 9.81            # surface gravity of the workloads, g = 9.81 (R_E / r)^2 [m/s^2]
OMEGA_EARTH = 7.292e-5      # rotation rate [rad/s]
GAMMA = 5.0 / 3.0           # ratio of specific heats (Sec. 2.1)

# boundary kinds (same integer codes as include/dg.h)
BC_PERIODIC = 0
BC_WALL = 1
BC_OUTFLOW = 2

KIND_BOX = 0
KIND_SHELL = 1


@dataclass
class MeshDesc:
    """Problem description handed to both the library (dg_mesh_desc) and the oracle.

    Box: [0,lx]x[0,ly]x[0,lz], nx*ny*nz hexahedra, periodic in x and y; the z ends carry
    bc_lo / bc_hi. Shell: cubed sphere, 6 panels of nx*nx elements, nz radial layers between
    r_inner and r_outer (nondimensional), first layer height h_first (geometric growth; <= 0 means
    uniform layers); bc_lo is the inner sphere, bc_hi the outer one.
    """
    kind: int = KIND_BOX
    p: int = 2
    nx: int = 4
    ny: int = 4
    nz: int = 4
    lx: float = 1.0
    ly: float = 1.0
    lz: float = 1.0
    r_inner: float = 0.0
    r_outer: float = 0.0
    h_first: float = 0.0
    bc_lo: int = BC_PERIODIC
    bc_hi: int = BC_PERIODIC
    # nondimensional physics (Eq. fluxSWNondimensional, Eq. nondimensional)
    gamma: float = GAMMA
    grashof: float = 100.0 ** 2 / GAMMA
    prandtl: float = 0.7
    mass: float = 1.0           # m* (molecular mass / m_O); c_v* = 1/m*
    visc_exp: float = 0.0       # mu* = kappa* = T*^visc_exp (0: constant)
    lambda0: float = 1.0        # sigma_c = lambda0 * I
    t_wall: float = 1.0         # isothermal wall temperature T*
    gravity_kind: int = 0       # 0: constant vector gvec; 1: radial, g* = -(g_r0/|r|)^2 r/|r|
    gvec: tuple = (0.0, 0.0, -1.0)
    g_r0: float = 0.0
    omega: tuple = (0.0, 0.0, 0.0)  # omega* (unit rotation axis times omega/omega_0)
    froude: float = 0.0
    euv: int = 0                # Gaussian sub-solar heating on/off
    euv_amp: float = 0.0        # peak heating, nondimensional (q H0 / (rho0 c_v0 T0 a0))
    euv_sigma: float = 0.0      # zenith-angle standard deviation [rad]
    euv_r_peak: float = 0.0     # radius of the heating peak (nondimensional)
    euv_width: float = 0.0      # vertical half width at half maximum (nondimensional)
    euv_omega_t: float = 0.0    # rotation angle of the sub-solar point per unit nondimensional time
    # EUVAC heating (euv = EUV_EUVAC, Sec. 2.2): solar and reference data
    euv_day: float = 80.0       # day of the year N_d (1 = January 1st)
    euv_f107: float = 150.0     # daily F10.7 index
    euv_f107a: float = 150.0    # its 81-day mean
    euv_eff: float = 0.25       # heating efficiency epsilon
    euv_dsun: float = 1.0       # Sun distance [astronomical units]
    ref_T0: float = 0.0         # reference temperature [K]
    ref_rho0: float = 0.0       # reference density [kg/m^3]
    ref_m: float = 0.0          # reference molecular mass [kg]
    ref_g0: float = 0.0         # reference gravity at the inner radius [m/s^2]
    # variable composition (Sec. 2.1.1-2.1.2): comp = 1 turns it on
    comp: int = 0
    comp_a: tuple = (0.0,) * 6  # chi_s = sum_j a_j^s exp(b_j^s |r|) for N2, O2, He (|r| nondimensional),
    comp_b: tuple = (0.0,) * 6  # row-major [species][j]; chi_O = 1 - the others
    eddy_nu: float = 200.0      # nu_eddy / nu_0
    eddy_alpha: float = 10.0    # alpha_eddy / alpha_0

    def as_dict(self):
        return asdict(self)

    @property
    def n_elem(self) -> int:
        if self.kind == KIND_BOX:
            return self.nx * self.ny * self.nz
        return 6 * self.nx * self.nx * self.nz

    @property
    def n_p(self) -> int:
        return (self.p + 1) ** 3

    @property
    def n_dof(self) -> int:
        return 5 * self.n_elem * self.n_p


@dataclass
class Reference:
    """Reference scales of Sec. 2.4 (lower-boundary values) for the shell workloads."""
    T0: float
    rho0: float
    m_O: float
    g0: float
    H0: float
    a0: float
    t0: float
    mu0: float
    kappa0: float
    Re: float
    Gr: float
    Pr: float
    Fr: float
    cv0: float


def shell_reference(T0=200.0, rho0=5.0e-7, h0=100.0e3) -> Reference:
    """Reference quantities at the lower boundary (Sec. 2.4).

    mu_0 and kappa_0 follow the nominal molecular laws of Sec. 2.2 evaluated in SI units for pure
    atomic oxygen at T0: mu_m = 6.5e-4 sqrt(T m / k), kappa_m = alpha_O T^0.69 with alpha_O = 5.6e-4.
    """
    m_O = 16.0 * AMU
    g0 = G_SURFACE * (R_EARTH / (R_EARTH + h0)) ** 2
    H0 = K_B * T0 / (m_O * g0)
    a0 = math.sqrt(GAMMA * K_B * T0 / m_O)
    mu0 = 6.5e-4 * math.sqrt(T0 * m_O / K_B)
    kappa0 = 5.6e-4 * T0 ** 0.69
    cv0 = K_B / ((GAMMA - 1.0) * m_O)
    cp0 = GAMMA * cv0
    Gr = g0 * H0 ** 3 / (mu0 / rho0) ** 2
    Re = rho0 * a0 * H0 / mu0
    Pr = mu0 * cp0 / kappa0
    Fr = math.sqrt(OMEGA_EARTH ** 2 * H0 / g0)
    return Reference(T0=T0, rho0=rho0, m_O=m_O, g0=g0, H0=H0, a0=a0, t0=H0 / a0, mu0=mu0,
                     kappa0=kappa0, Re=Re, Gr=Gr, Pr=Pr, Fr=Fr, cv0=cv0)


# ----------------------------------------------------------------------------------------------
# workload descriptors
# ----------------------------------------------------------------------------------------------
def box_desc(p=2, n=4, re=100.0, pr=0.7, bc_lo=BC_PERIODIC, bc_hi=BC_PERIODIC, gravity=1.0,
             visc_exp=0.0, nz=None, lz=1.0) -> MeshDesc:
    """Periodic unit box with constant gravity along -z (the 4x4x4, p=2 parity workload)."""
    return MeshDesc(kind=KIND_BOX, p=p, nx=n, ny=n, nz=n if nz is None else nz, lx=1.0, ly=1.0,
                    lz=lz, bc_lo=bc_lo, bc_hi=bc_hi, grashof=re * re / GAMMA, prandtl=pr,
                    visc_exp=visc_exp, gvec=(0.0, 0.0, -gravity))


def synthetic_composition(ref: Reference, r_inner: float):
    """Stand-in fit coefficients (a, b) [species N2, O2, He][j] for chi_s = sum_j a_j exp(b_j |r|), |r|
    nondimensional (the paper fits MSIS output, which is not available): N2 0.76 e^{-z/110 km} +
    0.02 e^{-z/30 km}, O2 0.19 e^{-z/75 km} + 0.01 e^{-z/25 km}, He 2e-6 e^{z/48 km}, z the height
    above the inner boundary; atomic oxygen takes the rest (0.02 at 100 km, 0.93 at 600 km)."""
    def term(frac, scale_km):
        b = (1.0 if scale_km < 0 else -1.0) * ref.H0 / (abs(scale_km) * 1e3)
        return frac * math.exp(-b * r_inner), b
    pairs = [(term(0.76, 110.0), term(0.02, 30.0)), (term(0.19, 75.0), term(0.01, 25.0)), (term(2e-6, -48.0), (0.0, 0.0))]
    a = tuple(p[j][0] for p in pairs for j in range(2))
    b = tuple(p[j][1] for p in pairs for j in range(2))
    return a, b


def shell_desc(n=16, nr=8, p=4, euv=False, rotation=True, h_first_km=2.5, ref: Reference | None = None,
               bc_lo=BC_WALL, bc_hi=BC_OUTFLOW, euvac=False, day=80.0, f107=150.0, f107a=150.0,
               composition=False) -> MeshDesc:
    """Cubed-sphere shell 100-600 km (Sec. 3.3) with the nondimensional numbers of Sec. 2.4."""
    ref = ref or shell_reference()
    H0 = ref.H0
    r_in = (R_EARTH + 100.0e3) / H0
    r_out = (R_EARTH + 600.0e3) / H0
    d = MeshDesc(kind=KIND_SHELL, p=p, nx=n, ny=n, nz=nr, r_inner=r_in, r_outer=r_out,
                 h_first=h_first_km * 1.0e3 / H0, bc_lo=bc_lo, bc_hi=bc_hi, grashof=ref.Gr,
                 prandtl=ref.Pr, mass=1.0, visc_exp=0.69, lambda0=1.0, t_wall=1.0,
                 gravity_kind=1, gvec=(0.0, 0.0, 0.0), g_r0=r_in,
                 omega=(0.0, 0.0, 1.0) if rotation else (0.0, 0.0, 0.0),
                 froude=ref.Fr if rotation else 0.0)
    if euv:
        d.euv = 1
        d.euv_amp = 1.0e-8 * H0 / (ref.rho0 * ref.cv0 * ref.T0 * ref.a0)
        d.euv_sigma = math.radians(60.0)
        d.euv_r_peak = (R_EARTH + 300.0e3) / H0
        d.euv_width = 50.0e3 / H0
        d.euv_omega_t = OMEGA_EARTH * ref.t0
    if euvac:
        d.euv = EUV_EUVAC
        d.euv_omega_t = OMEGA_EARTH * ref.t0
        d.euv_day, d.euv_f107, d.euv_f107a = day, f107, f107a
    d.ref_T0, d.ref_rho0, d.ref_m, d.ref_g0 = ref.T0, ref.rho0, ref.m_O, ref.g0
    if composition:
        d.comp = 1
        d.comp_a, d.comp_b = synthetic_composition(ref, r_in)
    return d


CONFIGS = {
    # name: (descriptor factory, human description)
    "box4_p2": (lambda: box_desc(p=2, n=4), "periodic unit box 4x4x4, p=2, Re=100, Pr=0.7"),
    "shell16x8_p4": (lambda: shell_desc(n=16, nr=8, p=4), "cubed-sphere shell 6x16x16x8, p=4"),
    "shell24x8_p2_euv": (lambda: shell_desc(n=24, nr=8, p=2, euv=True),
                         "cubed-sphere shell 6x24x24x8, p=2, EUV (small profiling case, 3.7M DOF)"),
    "shell32x16_p2_euv": (lambda: shell_desc(n=32, nr=16, p=2, euv=True),
                          "cubed-sphere shell 6x32x32x16, p=2, EUV"),
    "shell32x16_p2_euvac": (lambda: shell_desc(n=32, nr=16, p=2, euvac=True, day=172.0),
                            "cubed-sphere shell 6x32x32x16, p=2, EUVAC heating with Chapman depths, June solstice"),
    "shell32x16_p2_comp": (lambda: shell_desc(n=32, nr=16, p=2, euvac=True, day=172.0, composition=True),
                           "cubed-sphere shell 6x32x32x16, p=2, variable composition (O, N2, O2, He) with eddy "
                           "transport and four-absorber EUVAC heating, June solstice"),
    "shell48x16_p3_euv": (lambda: shell_desc(n=48, nr=16, p=3, euv=True),
                          "cubed-sphere shell 6x48x48x16, p=3, EUV"),
    "shell36x28_p3_euvac": (lambda: shell_desc(n=36, nr=28, p=3, euvac=True, day=79.0),
                            "cubed-sphere shell 6x36x36x28, p=3, EUVAC heating with Chapman depths, March "
                            "equinox (the paper's production mesh at k = 3: 217,728 elements, 69.7M DOF)"),
    "shell24x8_p3_euv": (lambda: shell_desc(n=24, nr=8, p=3, euv=True),
                         "cubed-sphere shell 6x24x24x8, p=3, EUV (small profiling case, 8.8M DOF)"),
    "shell8x4_p3_euv": (lambda: shell_desc(n=8, nr=4, p=3, euv=True),
                        "cubed-sphere shell 6x8x8x4, p=3, EUV (profiling case for the 320^2 block inversion, "
                        "1,536 blocks)"),
}



# ----------------------------------------------------------------------------------------------
# workload meshes (node coordinates of the isoparametric elements)
# ----------------------------------------------------------------------------------------------
PANELS = [
    ((1, 0, 0), (0, 1, 0), (0, 0, 1)),
    ((0, 1, 0), (-1, 0, 0), (0, 0, 1)),
    ((-1, 0, 0), (0, -1, 0), (0, 0, 1)),
    ((0, -1, 0), (1, 0, 0), (0, 0, 1)),
    ((0, 0, 1), (0, 1, 0), (-1, 0, 0)),
    ((0, 0, -1), (0, 1, 0), (1, 0, 0)),
]


def gll_points(n):
    """Gauss-Lobatto-Legendre points: -1, the roots of P'_{n-1}, +1 (where the nodes sit)."""
    c = np.zeros(n)
    c[n - 1] = 1.0
    inner = np.polynomial.legendre.legroots(np.polynomial.legendre.legder(c)) if n > 2 else np.array([])
    return np.concatenate([[-1.0], np.sort(np.real(inner)), [1.0]])


def radial_layers(r_in, r_out, nz, h_first):
    """Layer interfaces r_0 = r_in < ... < r_nz = r_out with heights h_first q^k (Sec. 3.3).

    The growth ratio q solves sum_{k<nz} h_first q^k = r_out - r_in (bisection); h_first <= 0 gives
    uniform layers.
    """
    total = r_out - r_in
    if h_first <= 0.0 or nz == 1:
        return r_in + total * np.arange(nz + 1) / nz
    def excess(q):
        return h_first * sum(q ** k for k in range(nz)) - total
    lo, hi = 1.0, 2.0
    if excess(lo) > 0:
        lo, hi = 1e-6, 1.0
    while excess(hi) < 0:
        hi *= 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if excess(mid) > 0:
            hi = mid
        else:
            lo = mid
    q = 0.5 * (lo + hi)
    r = r_in + np.concatenate([[0.0], np.cumsum(h_first * q ** np.arange(nz))])
    r[-1] = r_out
    return r


def mesh_nodes(desc):
    """GLL node positions X[e, d, i] of every element of the workload mesh (Sec. 3.3).

    box   element e = i + nx (j + ny k); nodes at x = (i + (1 + xi_a)/2) lx/nx, ...
    shell element e = k + nz (i + n (j + n P)) for panel P, angular cell (i, j), radial layer k;
          equiangular gnomonic panels: direction c_P + tan(alpha) a_P + tan(beta) b_P,
          normalised, alpha, beta in [-pi/4, pi/4], radius from the geometric layers.
    node  i = a + n b + n^2 c (a along xi_1, the fastest), n = p + 1, at the GLL points.
    """
    n = desc.p + 1
    xi = gll_points(n)
    c3, b3, a3 = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    ref = np.stack([xi[a3.ravel()], xi[b3.ravel()], xi[c3.ravel()]], axis=1)   # (n^3, 3)
    s = 0.5 * (1.0 + ref)              # in [0, 1]
    if desc.kind == 0:
        hx, hy, hz = desc.lx / desc.nx, desc.ly / desc.ny, desc.lz / desc.nz
        X = np.zeros((desc.n_elem, 3, n ** 3))
        for k in range(desc.nz):
            for j in range(desc.ny):
                for i in range(desc.nx):
                    e = i + desc.nx * (j + desc.ny * k)
                    X[e, 0] = (i + s[:, 0]) * hx
                    X[e, 1] = (j + s[:, 1]) * hy
                    X[e, 2] = (k + s[:, 2]) * hz
        return X
    nn, nz = desc.nx, desc.nz
    rl = radial_layers(desc.r_inner, desc.r_outer, nz, desc.h_first)
    d_ang = 0.5 * math.pi / nn
    X = np.zeros((desc.n_elem, 3, n ** 3))
    for P, (c, a, b) in enumerate(PANELS):
        c, a, b = np.array(c, float), np.array(a, float), np.array(b, float)
        for j in range(nn):
            for i in range(nn):
                alpha = -0.25 * math.pi + (i + s[:, 0]) * d_ang
                beta = -0.25 * math.pi + (j + s[:, 1]) * d_ang
                dirv = c[:, None] + np.tan(alpha)[None, :] * a[:, None] + np.tan(beta)[None, :] * b[:, None]
                dirv = dirv / np.sqrt((dirv ** 2).sum(0))[None, :]
                for k in range(nz):
                    e = k + nz * (i + nn * (j + nn * P))
                    r = rl[k] + s[:, 2] * (rl[k + 1] - rl[k])
                    X[e] = dirv * r[None, :]
    return X



# ----------------------------------------------------------------------------------------------
# SplitMix64 counter-based random numbers
# ----------------------------------------------------------------------------------------------
_PHI = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, idx: np.ndarray) -> np.ndarray:
    """SplitMix64 output for counters idx (uint64 arithmetic wraps modulo 2^64)."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (np.asarray(idx, dtype=np.uint64) + np.uint64(1)) * _PHI
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform01(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n doubles in [0,1) from counters offset..offset+n-1 (53 high bits)."""
    z = splitmix64(seed, np.arange(offset, offset + n, dtype=np.uint64))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n standard normals by Box-Muller from pairs of SplitMix64 uniforms."""
    m = (n + 1) // 2
    u1 = uniform01(seed, m, offset)
    u2 = uniform01(seed, m, offset + m)
    rad = np.sqrt(-2.0 * np.log1p(-u1))   # 1 - u1 in (0, 1]
    z = np.concatenate([rad * np.cos(2.0 * np.pi * u2), rad * np.sin(2.0 * np.pi * u2)])
    return z[:n]


def unit_vector(seed: int, shape) -> np.ndarray:
    """Seeded N(0,1) vector of the given shape normalised to unit 2-norm."""
    n = int(np.prod(shape))
    z = normal(seed, n)
    return (z / np.sqrt(np.dot(z, z))).reshape(shape)


def _wavevectors(kmax=3):
    ks = []
    for a in range(-kmax, kmax + 1):
        for b in range(-kmax, kmax + 1):
            for c in range(-kmax, kmax + 1):
                if 0 < a * a + b * b + c * c <= kmax * kmax:
                    ks.append((a, b, c))
    return np.array(ks, dtype=np.float64)


def fourier_field(seed: int, stream: int, xs: np.ndarray, kmax=3) -> np.ndarray:
    """Random Fourier sum over integer wavevectors 0 < |k|_2 <= kmax at points xs[..., 3].

    f(x) = sum_k a_k cos(2 pi k.x) + b_k sin(2 pi k.x), a, b ~ U(-1, 1), divided by its maximum
    modulus on the 32^3 lattice of one period (the unit cube), so the field has amplitude 1
    independently of the mesh. Periodic on the unit cube.
    """
    ks = _wavevectors(kmax)
    nk = ks.shape[0]
    ab = 2.0 * uniform01(seed, 2 * nk, offset=stream * 4096) - 1.0
    a, b = ab[:nk], ab[nk:]
    return _fourier_sum(ks, a, b, xs, kmax) / _fourier_max(ks, a, b, kmax)


def _fourier_max(ks, a, b, kmax, m=32):
    g = np.arange(m) / m
    lat = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    return float(np.abs(_fourier_sum(ks, a, b, lat, kmax)).max())


def _fourier_sum(ks, a, b, xs, kmax):
    nk = ks.shape[0]
    # exp(2 pi i k.x) as a product of per-axis powers of exp(2 pi i x_d)
    flat = xs.reshape(-1, 3)
    base = [np.exp(2j * np.pi * flat[:, d]) for d in range(3)]
    pw = []
    for d in range(3):
        tab = {0: np.ones(flat.shape[0], dtype=np.complex128)}
        for j in range(1, kmax + 1):
            tab[j] = tab[j - 1] * base[d]
            tab[-j] = np.conj(tab[j])
        pw.append(tab)
    f = np.zeros(flat.shape[0])
    for k in range(nk):
        k0, k1, k2 = (int(c) for c in ks[k])
        z = pw[0][k0] * pw[1][k1] * pw[2][k2]
        f += a[k] * z.real + b[k] * z.imag
    return f.reshape(xs.shape[:-1])


# ----------------------------------------------------------------------------------------------
# base atmospheres
# ----------------------------------------------------------------------------------------------
def bates_temperature(z_km):
    """Bates profile T(z) = 1000 - 800 exp(-0.02 (z - 100)) [K], z in km."""
    return 1000.0 - 800.0 * np.exp(-0.02 * (z_km - 100.0))


def workload_gravity(r_m):
    """Gravity of the shell workloads, g = 9.81 (R_E / r)^2 [m/s^2], r in m."""
    return G_SURFACE * (R_EARTH / r_m) ** 2


def bates_hydrostatic(r_m: np.ndarray, ref: Reference, p_points=16, temperature=None, gravity=None):
    """Density [kg/m^3] and temperature [K] of the Bates atmosphere in hydrostatic balance.

    ln p(r) = ln p0 - int_{R0}^{r} m g(s) / (k_B T(s)) ds with g = 9.81 (R_E/s)^2, integrated by
    composite Gauss-Legendre between consecutive distinct radii; rho = p m / (k_B T).
    temperature(z_km) and gravity(r_m) default to the Bates profile and workload_gravity.
    """
    temperature = temperature or bates_temperature
    gravity = gravity or workload_gravity
    R0 = R_EARTH + 100.0e3
    m = ref.m_O
    shape = r_m.shape
    rr = r_m.ravel()
    key = np.round(rr, 6)
    uniq, inv = np.unique(key, return_inverse=True)
    xg, wg = np.polynomial.legendre.leggauss(p_points)
    edges = np.concatenate([[R0], uniq])
    lo, hi = edges[:-1], edges[1:]
    s = 0.5 * (hi - lo)[:, None] * xg[None, :] + 0.5 * (hi + lo)[:, None]
    integrand = m * gravity(s) / (K_B * temperature((s - R_EARTH) / 1.0e3))
    seg = 0.5 * (hi - lo) * (integrand @ wg)
    lnp_rel = -np.cumsum(seg)
    T = temperature((uniq - R_EARTH) / 1.0e3)
    p0 = ref.rho0 * K_B * ref.T0 / m
    rho = p0 * np.exp(lnp_rel) * m / (K_B * T)
    return rho[inv].reshape(shape), T[inv].reshape(shape)


# ----------------------------------------------------------------------------------------------
# initial states on a node array x[N_e][3][N_p]
# ----------------------------------------------------------------------------------------------
def pack_state(rho, v, T):
    """u = (log rho*, sqrt(rho*) v*, sqrt(rho*) T*) in the layout [N_e][5][N_p] (Sec. 2.3)."""
    sr = np.sqrt(rho)
    return np.stack([np.log(rho), sr * v[0], sr * v[1], sr * v[2], sr * T], axis=1)


def box_state(x: np.ndarray, seed: int = 1, amp=0.01):
    """Uniform rho = T = 1, v = 0 plus seeded |k| <= 3 Fourier modes of amplitude amp."""
    xs = np.moveaxis(x, 1, -1)
    f = [fourier_field(seed, s, xs) for s in range(5)]
    rho = 1.0 + amp * f[0]
    T = 1.0 + amp * f[4]
    v = np.stack([amp * f[1], amp * f[2], amp * f[3]])
    return pack_state(rho, v, T)


def shell_state(x: np.ndarray, desc: MeshDesc, seed: int = 2, ref: Reference | None = None,
                t_amp=0.01, v_ms=10.0):
    """Bates + hydrostatic shell state, T x (1 + t_amp f), v = v_ms/a0 f_vec (f from the seeded
    Fourier construction in Cartesian coordinates divided by the outer radius)."""
    ref = ref or shell_reference()
    xs = np.moveaxis(x, 1, -1)
    r_nd = np.sqrt((xs ** 2).sum(-1))
    rho_d, T_d = bates_hydrostatic(r_nd * ref.H0, ref)
    unit = xs / desc.r_outer
    fT = fourier_field(seed, 0, unit)
    fv = [fourier_field(seed, s, unit) for s in (1, 2, 3)]
    T = T_d / ref.T0 * (1.0 + t_amp * fT)
    v = np.stack([v_ms / ref.a0 * f for f in fv])
    rho = rho_d / ref.rho0
    return pack_state(rho, v, T)


def isothermal_column(x: np.ndarray, T=1.0, g=1.0):
    """Hydrostatic isothermal column under constant gravity -g e_z: log rho = -g z / T, v = 0."""
    z = x[:, 2, :]
    rho = np.exp(-g * z / T)
    zeros = np.zeros_like(z)
    return pack_state(rho, np.stack([zeros, zeros, zeros]), T * np.ones_like(z))


def state_for(desc: MeshDesc, x: np.ndarray, seed: int):
    if desc.kind == KIND_BOX:
        return box_state(x, seed)
    return shell_state(x, desc, seed)


# ----------------------------------------------------------------------------------------------
# radial 1D ensemble (Sec. 4.3: 28 elements, p = 2, first element 2.5 km, geometric growth, 100-600 km)
# ----------------------------------------------------------------------------------------------
@dataclass
class RadialDesc:
    """An ensemble of independent radial columns on one shared radial mesh.

    Every column is the spherically symmetric thermosphere above one site (latitude, longitude) with
    its own EUV heating efficiency epsilon and conductivity factor alpha0 (kappa_m = alpha0 x the
    nominal law, Sec. 4.3); the physics numbers are those of the shell workloads (Sec. 2.4) with the
    EUVAC heating of Sec. 2.2 (euv = EUV_EUVAC) or none (euv = 0)."""
    p: int = 2
    n_elem: int = 28
    n_col: int = 1
    r_inner: float = 0.0
    r_outer: float = 0.0
    h_first: float = 0.0
    bc_lo: int = BC_WALL
    bc_hi: int = BC_OUTFLOW
    gamma: float = GAMMA
    grashof: float = 100.0 ** 2 / GAMMA
    prandtl: float = 0.7
    mass: float = 1.0
    visc_exp: float = 0.69
    lambda0: float = 1.0
    t_wall: float = 1.0
    g_r0: float = 0.0
    euv: int = EUV_EUVAC
    euv_omega_t: float = 0.0
    euv_day: float = 80.0
    euv_f107: float = 150.0
    euv_f107a: float = 150.0
    euv_eff: float = 0.25        # the nominal efficiency; a column's own epsilon replaces it
    euv_dsun: float = 1.0
    ref_T0: float = 0.0
    ref_rho0: float = 0.0
    ref_m: float = 0.0
    ref_g0: float = 0.0

    @property
    def n_node(self) -> int:
        return self.n_elem * (self.p + 1)

    @property
    def n_dof_col(self) -> int:
        return 3 * self.n_node

    @property
    def n_dof(self) -> int:
        return self.n_col * self.n_dof_col


def radial_desc(n_col=1, n_elem=28, p=2, h_first_km=2.5, euvac=True, ref: Reference | None = None,
                day=80.0, f107=150.0, f107a=150.0) -> RadialDesc:
    """The radial column mesh of the paper's 1D model: n_elem layers from 100 to 600 km with a first
    layer of h_first_km and geometric growth (Sec. 3.3 / 4.3)."""
    ref = ref or shell_reference()
    H0 = ref.H0
    r_in = (R_EARTH + 100.0e3) / H0
    return RadialDesc(p=p, n_elem=n_elem, n_col=n_col, r_inner=r_in, r_outer=(R_EARTH + 600.0e3) / H0,
                      h_first=h_first_km * 1.0e3 / H0, grashof=ref.Gr, prandtl=ref.Pr, g_r0=r_in,
                      euv=EUV_EUVAC if euvac else 0, euv_omega_t=OMEGA_EARTH * ref.t0, euv_day=day,
                      euv_f107=f107, euv_f107a=f107a, ref_T0=ref.T0, ref_rho0=ref.rho0, ref_m=ref.m_O,
                      ref_g0=ref.g0)


# the paper's parameter values (Sec. 4.3): epsilon and alpha0 grids
RADIAL_EPS = (0.2, 0.225, 0.25, 0.275, 0.3)
RADIAL_ALPHA0 = (0.5, 0.625, 0.75, 0.875, 1.0)


def radial_params(n_col: int, seed: int = 21) -> np.ndarray:
    """Per-column parameters [n_col][4] = (epsilon, alpha0, latitude, longitude) [-, -, rad, rad]:
    the 25 (epsilon, alpha0) pairs of the paper's grids in turn, at seeded sites uniform on the
    sphere (latitude asin(U(-1, 1)), longitude U(-pi, pi))."""
    k = np.arange(n_col)
    eps = np.array(RADIAL_EPS)[k % 5]
    alpha = np.array(RADIAL_ALPHA0)[(k // 5) % 5]
    u = uniform01(seed, 2 * n_col)
    lat = np.arcsin(2.0 * u[:n_col] - 1.0)
    lon = np.pi * (2.0 * u[n_col:] - 1.0)
    return np.stack([eps, alpha, lat, lon], axis=1)


def radial_nodes(desc: RadialDesc) -> np.ndarray:
    """Radii [n_elem][p+1] of the GLL nodes of the radial mesh (the layers of radial_layers)."""
    rl = radial_layers(desc.r_inner, desc.r_outer, desc.n_elem, desc.h_first)
    s = 0.5 * (1.0 + gll_points(desc.p + 1))
    return rl[:-1, None] + s[None, :] * (rl[1:] - rl[:-1])[:, None]


def radial_state(desc: RadialDesc, seed: int = 3, ref: Reference | None = None, t_amp=0.01, v_ms=5.0):
    """u [3][n_elem][p+1][n_col] = (log rho*, sqrt(rho*) v*, sqrt(rho*) T*) at the nodes: the Bates
    atmosphere in hydrostatic balance, T x (1 + t_amp f), radial wind v_ms f' [m/s], with f, f' seeded
    smooth profiles per column (sums of 4 sine modes of the height, amplitude 1)."""
    ref = ref or shell_reference()
    r = radial_nodes(desc)                                      # (E, N)
    rho_d, T_d = bates_hydrostatic(r * ref.H0, ref)
    s = (r - desc.r_inner) / (desc.r_outer - desc.r_inner)
    ab = 2.0 * uniform01(seed, 16 * desc.n_col).reshape(desc.n_col, 2, 4, 2) - 1.0
    modes = np.arange(1, 5)

    def profile(c, k):
        f = (ab[c, k, :, 0, None, None] * np.sin(np.pi * modes[:, None, None] * s[None])
             + ab[c, k, :, 1, None, None] * np.cos(np.pi * modes[:, None, None] * s[None])).sum(0)
        return f / max(1e-300, np.abs(f).max())

    u = np.zeros((3,) + r.shape + (desc.n_col,))
    for c in range(desc.n_col):
        T = T_d / ref.T0 * (1.0 + t_amp * profile(c, 0))
        v = v_ms / ref.a0 * profile(c, 1)
        rho = rho_d / ref.rho0
        sr = np.sqrt(rho)
        u[0, :, :, c] = np.log(rho)
        u[1, :, :, c] = sr * v
        u[2, :, :, c] = sr * T
    return u
