// Mesh creation (Sec. 3.3 cubed-sphere shells and boxes), face connectivity, and the C ABI
// entry points of the residual path.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>

#include "dg_euvac.h"
#include "dg_internal.cuh"
#include "dg_nvtx.h"
#include "dg_map.cuh"

namespace dg {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }
int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

#define DG_DISPATCH(m, call)                      \
  switch ((m)->n) {                               \
    case 2: return Driver<2>::call;               \
    case 3: return Driver<3>::call;               \
    case 4: return Driver<4>::call;               \
    case 5: return Driver<5>::call;               \
    default: return fail(DG_EINVAL, "unsupported degree"); \
  }

static int drv_geometry(dg_mesh* m, cudaStream_t s) { DG_DISPATCH(m, geometry(m, s)); }
static int drv_gradient(dg_mesh* m, const double* u, const double* v, cudaStream_t s, bool f32 = false,
                        bool tangent_only = false) {
  DG_DISPATCH(m, gradient(m, u, v, s, f32, tangent_only));
}
static int drv_residual(dg_mesh* m, const double* u, const double* v, double t, double* r, double* jv,
                        bool tan, cudaStream_t s, bool f32 = false, double stage_c = 0.0) {
  DG_DISPATCH(m, residual(m, u, v, t, r, jv, tan, s, f32, stage_c));
}
static int drv_q_to_nodal(dg_mesh* m, double* q, cudaStream_t s) { DG_DISPATCH(m, q_to_nodal(m, q, s)); }
static int drv_q_from_nodal(dg_mesh* m, const double* q, cudaStream_t s) { DG_DISPATCH(m, q_from_nodal(m, q, s)); }
static int drv_mass(dg_mesh* m, const double* v, double* mv, cudaStream_t s) { DG_DISPATCH(m, mass(m, v, mv, s)); }
static int drv_mixture(dg_mesh* m) { DG_DISPATCH(m, mixture(m)); }
static int drv_mass_inv(dg_mesh* m, const double* v, double* mv, cudaStream_t s) {
  DG_DISPATCH(m, mass_inv(m, v, mv, s));
}

// ------------------------------------------------------------------------------------------
// radial layers with geometric growth from the first-layer height (Sec. 3.3)
// ------------------------------------------------------------------------------------------
// Per-band coefficients of the EUVAC heating in the nondimensional variables (DG_EUV_EUVAC in
// dg.h). The absorbers' number densities are n_s = rho0 e^varrho w_s / m0 with w_s = chi_s / m_s*
// (or 1/m* for the single constituent), so with Phi_j = sum_s w_s phi_s^j and H = H0 H*,
// q* = q H0/(rho0 c_v0 T0 a0) = e^varrho sum_j B_j Phi_j exp(-tau_j), tau_j = cc e^varrho Phi_j H* Ch,
// B_j = eps I0_j (h c/lambda_j) H0 / (m0 c_v0 T0 a0) and cc = rho0 H0 / m0.
bool euvac_coefficients(const dg_mesh_desc& d, Phys& P) {
  if (!(d.ref_T0 > 0 && d.ref_rho0 > 0 && d.ref_m > 0 && d.ref_g0 > 0 && d.euv_dsun > 0 && d.g_r0 > 0 &&
        d.mass > 0 && d.gamma > 1))
    return false;
  const double kB = 1.380649e-23, h = 6.62607015e-34, c = 299792458.0;
  const double H0 = kB * d.ref_T0 / (d.ref_m * d.ref_g0);
  const double a0 = std::sqrt(d.gamma * kB * d.ref_T0 / d.ref_m);
  const double cv0 = kB / ((d.gamma - 1.0) * d.ref_m);
  const double fbar = 0.5 * (d.euv_f107 + d.euv_f107a);
  int n = 0;
  for (int j = 0; j < kEuvacRows && n < 40; ++j) {
    const EuvacRow& row = kEuvac[j];
    const double lambda = 0.5 * (row.lo + row.hi) * 1e-10;
    const double I0 = row.flux * 1e13 * std::max(0.8, 1.0 + row.a * (fbar - 80.0)) / (d.euv_dsun * d.euv_dsun);
    P.euvac_B[n] = d.euv_eff * I0 * (h * c / lambda) * H0 / (d.ref_m * cv0 * d.ref_T0 * a0);
    const double phis[4] = {row.phi_o, row.phi_n2, row.phi_o2, row.phi_he};   // O, N2, O2, He
    for (int s = 0; s < 4; ++s) P.euvac_phi[s][n] = phis[s] * 1e-22;
    ++n;
  }
  P.n_euvac = n;
  P.euvac_cc = d.ref_rho0 * H0 / d.ref_m;
  const double w = 2.0 * M_PI / 365.24;
  const double delta = std::asin(std::sin(-23.44 * M_PI / 180.0) *
                                 std::cos(w * (d.euv_day + 9.0) + 2.0 * 0.0167 * std::sin(w * (d.euv_day - 3.0))));
  P.sun_cd = std::cos(delta);
  P.sun_sd = std::sin(delta);
  P.g_r0 = d.g_r0;
  P.inv_m = 1.0 / d.mass;
  return true;
}

std::vector<double> radial_layers(double r_in, double r_out, int nz, double h1) {
  std::vector<double> r(nz + 1);
  const double total = r_out - r_in;
  if (h1 <= 0.0 || nz == 1) {
    for (int k = 0; k <= nz; ++k) r[k] = r_in + total * k / nz;
    r[nz] = r_out;
    return r;
  }
  auto sum = [&](double q) {
    double s = 0.0, t = 1.0;
    for (int k = 0; k < nz; ++k) {
      s += t;
      t *= q;
    }
    return h1 * s - total;
  };
  double lo = 1.0, hi = 2.0;
  if (sum(lo) > 0) { lo = 1e-6; hi = 1.0; }
  while (sum(hi) < 0) hi *= 2.0;
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    if (sum(mid) > 0) hi = mid; else lo = mid;
  }
  const double q = 0.5 * (lo + hi);
  double acc = r_in, h = h1;
  for (int k = 0; k < nz; ++k) {
    r[k] = acc;
    acc += h;
    h *= q;
  }
  r[nz] = r_out;
  return r;
}

__global__ void k_nodes(MapParams mp, long long E, int n, const double* __restrict__ xi, double* __restrict__ x) {
  const int np = n * n * n;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= E * np) return;
  const long long e = idx / np;
  const int i = (int)(idx % np);
  const int a = i % n, b = (i / n) % n, c = i / (n * n);
  double out[3];
  map_point(mp, e, xi[a], xi[b], xi[c], out);
  for (int d = 0; d < 3; ++d) x[(e * 3 + d) * np + i] = out[d];
}

// ------------------------------------------------------------------------------------------
// connectivity: faces matched by their centres (spatial hash), orientation from corners
// ------------------------------------------------------------------------------------------
namespace {

struct FaceKey {
  long long e;
  int f;
};

// reference coordinates of face corner (cs, ct) in {0,1}^2 of local face phi
void face_corner_ref(int phi, int cs, int ct, double out[3]) {
  const int axis = phi >> 1;
  const double side = (phi & 1) ? 1.0 : -1.0;
  const int s_ax = axis == 0 ? 1 : 0;
  const int t_ax = axis == 2 ? 1 : 2;
  out[axis] = side;
  out[s_ax] = cs ? 1.0 : -1.0;
  out[t_ax] = ct ? 1.0 : -1.0;
}

}  // namespace

static int build_connectivity(dg_mesh* m, const std::vector<double>& X, std::vector<int32_t>& nbr,
                              std::vector<int32_t>& nbr_fo, std::vector<int32_t>& face_e,
                              std::vector<int32_t>& face_f) {
  const dg_mesh_desc& d = m->desc;
  const long long E = m->E;
  const int n = m->n;
  const bool box = d.kind == DG_KIND_BOX;
  double per[3] = {0, 0, 0};
  if (box) {
    per[0] = d.lx;
    per[1] = d.ly;
    per[2] = (d.bc_lo == DG_BC_PERIODIC) ? d.lz : 0.0;
  }
  double extent = box ? std::max(d.lx, std::max(d.ly, d.lz)) : d.r_outer;
  const double tol = 1e-9 * extent;
  const double cell = 1e-5 * extent;
  auto wrap = [&](double* c) {
    for (int a = 0; a < 3; ++a)
      if (per[a] > 0) {
        c[a] = std::fmod(c[a], per[a]);
        if (c[a] < 0) c[a] += per[a];
        if (per[a] - c[a] < tol) c[a] = 0.0;
      }
  };
  auto wdist2 = [&](const double* a, const double* b) {
    double s = 0.0;
    for (int k = 0; k < 3; ++k) {
      double dd = a[k] - b[k];
      if (per[k] > 0) dd -= per[k] * std::round(dd / per[k]);
      s += dd * dd;
    }
    return s;
  };
  // corner nodes (the GLL nodes include the element corners) and centres of all faces
  const int np = n * n * n;
  std::vector<double> corners((size_t)E * 6 * 4 * 3), centres((size_t)E * 6 * 3), raw((size_t)E * 6 * 3);
  for (long long e = 0; e < E; ++e)
    for (int phi = 0; phi < 6; ++phi) {
      double cen[3] = {0, 0, 0};
      for (int k = 0; k < 4; ++k) {
        double ref[3];
        face_corner_ref(phi, k & 1, k >> 1, ref);
        const int ia = ref[0] > 0 ? n - 1 : 0, ib = ref[1] > 0 ? n - 1 : 0, ic = ref[2] > 0 ? n - 1 : 0;
        const int node = ia + n * (ib + n * ic);
        for (int a = 0; a < 3; ++a) {
          const double p = X[((size_t)e * 3 + a) * np + node];
          corners[((e * 6 + phi) * 4 + k) * 3 + a] = p;
          cen[a] += 0.25 * p;
        }
      }
      for (int a = 0; a < 3; ++a) raw[(e * 6 + phi) * 3 + a] = cen[a];
      wrap(cen);
      for (int a = 0; a < 3; ++a) centres[(e * 6 + phi) * 3 + a] = cen[a];
    }
  auto key_of = [&](long long ix, long long iy, long long iz) {
    return (unsigned long long)(ix * 73856093LL) ^ (unsigned long long)(iy * 19349663LL) ^
           (unsigned long long)(iz * 83492791LL);
  };
  std::unordered_map<unsigned long long, std::vector<long long>> grid;
  grid.reserve((size_t)E * 6);
  for (long long k = 0; k < E * 6; ++k) {
    const double* c = &centres[k * 3];
    grid[key_of((long long)std::floor(c[0] / cell), (long long)std::floor(c[1] / cell),
                (long long)std::floor(c[2] / cell))]
        .push_back(k);
  }
  nbr.assign((size_t)E * 6, 0);
  nbr_fo.assign((size_t)E * 6, 0);
  std::vector<long long> match((size_t)E * 6, -1);
  for (long long k = 0; k < E * 6; ++k) {
    if (match[k] >= 0) continue;
    const double* c = &centres[k * 3];
    const long long ix = (long long)std::floor(c[0] / cell), iy = (long long)std::floor(c[1] / cell),
                    iz = (long long)std::floor(c[2] / cell);
    long long found = -1;
    for (int dx = -1; dx <= 1 && found < 0; ++dx)
      for (int dy = -1; dy <= 1 && found < 0; ++dy)
        for (int dz = -1; dz <= 1 && found < 0; ++dz) {
          auto it = grid.find(key_of(ix + dx, iy + dy, iz + dz));
          if (it == grid.end()) continue;
          for (long long j : it->second)
            if (j != k && match[j] < 0 && wdist2(c, &centres[j * 3]) < tol * tol) {
              found = j;
              break;
            }
        }
    if (found >= 0) {
      match[k] = found;
      match[found] = k;
    }
  }
  // orientation codes and boundary kinds
  // the neighbour face is the own face moved by the exact translation between the two centres
  // (zero except across a periodic boundary), so corners are matched without wrapping
  auto corner_match = [&](long long k_own, int corner, long long k_oth) {
    const double* p = &corners[(k_own * 4 + corner) * 3];
    double q[3];
    for (int a = 0; a < 3; ++a) q[a] = p[a] + (raw[k_oth * 3 + a] - raw[k_own * 3 + a]);
    for (int j = 0; j < 4; ++j) {
      const double* c = &corners[(k_oth * 4 + j) * 3];
      double d2 = 0.0;
      for (int a = 0; a < 3; ++a) d2 += (c[a] - q[a]) * (c[a] - q[a]);
      if (d2 < tol * tol) return j;
    }
    return -1;
  };
  face_e.clear();
  face_f.clear();
  for (long long k = 0; k < E * 6; ++k) {
    const long long e = k / 6;
    const int phi = (int)(k % 6);
    if (match[k] >= 0) {
      const long long k2 = match[k];
      const int j00 = corner_match(k, 0, k2), j10 = corner_match(k, 1, k2), j01 = corner_match(k, 2, k2);
      if (j00 < 0 || j10 < 0 || j01 < 0) return fail(DG_EINVAL, "face corners do not match");
      const int s00 = j00 & 1, t00 = j00 >> 1, s10 = j10 & 1;
      const int swap = (s10 == s00) ? 1 : 0;
      const int o = swap | ((s00 ? 1 : 0) << 1) | ((t00 ? 1 : 0) << 2);
      // check the third corner against the orientation map
      const int m01 = orient_map(o, 0, n - 1, n);
      const int expect01 = ((m01 % n) ? 1 : 0) | (((m01 / n) ? 1 : 0) << 1);
      if (expect01 != j01) return fail(DG_EINVAL, "inconsistent face orientation");
      nbr[k] = (int32_t)(k2 / 6);
      nbr_fo[k] = (int32_t)((k2 % 6) | (o << 3));
      if (k < k2) {
        face_e.push_back((int32_t)e);
        face_f.push_back(phi);
      }
    } else {
      int bc;
      if (box) {
        const double z = centres[k * 3 + 2];
        if (per[2] > 0) return fail(DG_EINVAL, "unmatched face in a periodic box");
        bc = (std::fabs(z) < 1e-6 * extent) ? d.bc_lo : d.bc_hi;
      } else {
        double rr = 0.0;
        for (int j = 0; j < 4; ++j) {
          const double* p = &corners[(k * 4 + j) * 3];
          rr += 0.25 * std::sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
        }
        bc = (std::fabs(rr - d.r_inner) < std::fabs(rr - d.r_outer)) ? d.bc_lo : d.bc_hi;
      }
      if (bc != DG_BC_WALL && bc != DG_BC_OUTFLOW) return fail(DG_EINVAL, "boundary face without a wall/outflow kind");
      nbr[k] = -bc;
      nbr_fo[k] = 0;
      face_e.push_back((int32_t)e);
      face_f.push_back(phi);
    }
  }
  return DG_OK;
}

static void prof_release(dg_mesh* m) {
  Prof& p = m->prof;
  if (p.ev) {
    for (int i = 0; i < 2 * p.cap; ++i) cudaEventDestroy(p.ev[i]);
    delete[] p.ev;
    delete[] p.kind;
  }
  p = Prof();
}

static void free_mesh(dg_mesh* m) {
  prof_release(m);
  dg_solver_release(m);
  dg_mlp_release(m);
  dg::interp_tc_release(m);
  if (m->w32_base) cudaFree(m->w32_base);
  void* ptrs[] = {m->d_ops, m->x, m->geo, m->acc, m->xg, m->fgeo, m->mixg, m->mixf, m->nbr, m->nbr_fo, m->face_e,
                  m->face_f,
                  m->ws.ug, m->ws.uf, m->ws.qg, m->ws.qf, m->ws.fh, m->ws.tmp, m->ws.red, m->ws.qx};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (m->ws.red_host) cudaFreeHost(m->ws.red_host);
  delete m;
}

template <typename T>
static int dalloc(T** p, size_t count) {
  cudaError_t err = cudaMalloc((void**)p, sizeof(T) * (count ? count : 1));
  if (err != cudaSuccess) {
    *p = nullptr;
    return fail(DG_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(err));
  }
  return DG_OK;
}

}  // namespace dg

using namespace dg;

extern "C" const char* dg_last_error(void) { return g_last_error.c_str(); }

namespace dg {

__global__ void k_to_f32(long long n, const double* __restrict__ x, float* __restrict__ y) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}

int ensure_f32(dg_mesh* m) {
  if (m->w32_base) return DG_OK;
  const long long E = m->E, NP = m->np, NF = m->nf;
  const long long nmg = m->mixg ? E * 8 * NP : 0, nmf = m->mixf ? E * 12 * NF : 0;
  const long long sizes[12] = {2 * E * 5 * NP, 2 * E * 30 * NF, 2 * E * 15 * NP, 2 * E * 90 * NF, 2 * E * 30 * NF,
                               E * 90 * NF,    E * 10 * NP,     E * 24 * NF,     E * 3 * NP,      E * 3 * NP,
                               nmg,            nmf};
  long long total = 0;
  for (long long z : sizes) total += (z + 63) / 64 * 64;
  cudaError_t err = cudaMalloc(&m->w32_base, sizeof(float) * (size_t)total);
  if (err != cudaSuccess) {
    m->w32_base = nullptr;
    return fail(DG_ENOMEM, std::string("FP32 workspace: ") + cudaGetErrorString(err));
  }
  float* p[12];
  long long off = 0;
  for (int k = 0; k < 12; ++k) {
    p[k] = m->w32_base + off;
    off += (sizes[k] + 63) / 64 * 64;
  }
  m->w32 = WorkT<float>{p[0], p[1], p[2], p[3], p[4], p[5], p[6], p[7], p[8], p[9],
                        m->mixg ? p[10] : nullptr, m->mixf ? p[11] : nullptr};
  const double* src[6] = {m->geo, m->fgeo, m->acc, m->xg, m->mixg, m->mixf};
  for (int k = 0; k < 6; ++k) {
    if (!src[k]) continue;
    k_to_f32<<<1024, 256>>>(sizes[6 + k], src[k], p[6 + k]);
    err = cudaGetLastError();
    if (err != cudaSuccess) return fail(DG_ECUDA, std::string("k_to_f32: ") + cudaGetErrorString(err));
  }
  err = cudaDeviceSynchronize();
  if (err != cudaSuccess) return fail(DG_ECUDA, std::string("FP32 geometry: ") + cudaGetErrorString(err));
  return DG_OK;
}

}  // namespace dg

extern "C" int dg_mesh_create(const dg_mesh_desc* desc, const double* nodes, dg_mesh** out) {
  if (!desc || !out) return fail(DG_EINVAL, "dg_mesh_create: null argument");
  *out = nullptr;
  const dg_mesh_desc& d = *desc;
  if (d.p < 1 || d.p > 4) return fail(DG_EINVAL, "dg_mesh_create: p must be in 1..4");
  if (d.nx < 1 || d.nz < 1 || (d.kind == DG_KIND_BOX && d.ny < 1))
    return fail(DG_EINVAL, "dg_mesh_create: element counts must be positive");
  if (d.kind != DG_KIND_BOX && d.kind != DG_KIND_SHELL) return fail(DG_EINVAL, "dg_mesh_create: unknown kind");
  if ((d.bc_lo == DG_BC_PERIODIC) != (d.bc_hi == DG_BC_PERIODIC))
    return fail(DG_EINVAL, "dg_mesh_create: periodic z needs both ends periodic");
  if (d.kind == DG_KIND_SHELL && (d.bc_lo == DG_BC_PERIODIC || !(d.r_outer > d.r_inner) || d.r_inner <= 0))
    return fail(DG_EINVAL, "dg_mesh_create: shell needs r_outer > r_inner > 0 and wall/outflow boundaries");
  if (d.kind == DG_KIND_BOX && !(d.lx > 0 && d.ly > 0 && d.lz > 0))
    return fail(DG_EINVAL, "dg_mesh_create: box lengths must be positive");
  if (!(d.grashof > 0) || !(d.prandtl > 0) || !(d.mass > 0) || !(d.gamma > 1))
    return fail(DG_EINVAL, "dg_mesh_create: physical numbers out of range");

  dg_mesh* m = new dg_mesh();
  m->desc = d;
  m->n = d.p + 1;
  m->np = m->n * m->n * m->n;
  m->nf = m->n * m->n;
  m->E = (d.kind == DG_KIND_BOX) ? (long long)d.nx * d.ny * d.nz : 6LL * d.nx * d.nx * d.nz;
  m->ndof = 5 * m->E * m->np;
  cudaGetDevice(&m->device);
  build_ops(m->n, &m->ops);
  // physics coefficients of Eq. fluxSWNondimensional
  Phys& P = m->phys;
  P.gamma = d.gamma;
  P.c_mu = 1.0 / std::sqrt(d.gamma * d.grashof);
  P.c_k = std::sqrt(d.gamma / d.grashof) / d.prandtl;
  P.c_d = (d.gamma - 1.0) * std::sqrt(d.gamma / d.grashof);
  P.p_coef = 1.0 / (d.gamma * d.mass);
  P.cv = 1.0 / d.mass;
  P.visc_exp = d.visc_exp;
  P.lam = d.lambda0;
  P.t_wall = d.t_wall;
  for (int k = 0; k < 3; ++k) P.omega[k] = d.omega[k];
  P.cor = 2.0 * d.froude / std::sqrt(d.gamma);
  P.euv = d.euv;
  P.euv_amp = d.euv_amp;
  P.euv_inv2s2 = d.euv == DG_EUV_GAUSS ? 1.0 / (2.0 * d.euv_sigma * d.euv_sigma) : 0.0;
  P.euv_r_peak = d.euv_r_peak;
  P.euv_inv_w = d.euv == DG_EUV_GAUSS ? 1.0 / d.euv_width : 0.0;
  P.euv_omega_t = d.euv_omega_t;
  P.comp = d.comp;
  for (int k = 0; k < 6; ++k) {
    P.comp_a[k] = d.comp_a[k];
    P.comp_b[k] = d.comp_b[k];
  }
  P.eddy_nu = d.eddy_nu;
  P.eddy_alpha = d.eddy_alpha;
  P.inv_gamma = 1.0 / d.gamma;
  P.n_euvac = 0;
  if (d.euv == DG_EUV_EUVAC && !euvac_coefficients(d, P)) {
    delete m;
    return fail(DG_EINVAL, "dg_mesh_create: EUVAC heating needs positive reference values, g_r0 and Sun distance");
  }

  std::vector<double> layers = (d.kind == DG_KIND_SHELL) ? radial_layers(d.r_inner, d.r_outer, d.nz, d.h_first)
                                                         : std::vector<double>(2, 0.0);
  MapParams mp{d.kind, d.nx, d.ny, d.nz, d.lx, d.ly, d.lz, layers.data()};
  const long long E = m->E, NP = m->np, NF = m->nf;
  int rc = 0;
  rc |= dalloc(&m->x, E * 3 * NP);
  if (rc) { free_mesh(m); return DG_ENOMEM; }
  std::vector<double> X((size_t)E * 3 * NP);
  if (nodes) {
    std::memcpy(X.data(), nodes, sizeof(double) * X.size());
    cudaError_t e1 = cudaMemcpy(m->x, X.data(), sizeof(double) * X.size(), cudaMemcpyHostToDevice);
    if (e1 != cudaSuccess) { free_mesh(m); return fail(DG_ECUDA, std::string("node upload: ") + cudaGetErrorString(e1)); }
  } else {
    // nodes of the analytic map at the GLL points, on the device
    double* d_layers = nullptr;
    double* d_xi = nullptr;
    if (dalloc(&d_layers, layers.size()) || dalloc(&d_xi, MAXN)) {
      if (d_layers) cudaFree(d_layers);
      free_mesh(m);
      return DG_ENOMEM;
    }
    cudaError_t e1 = cudaMemcpy(d_layers, layers.data(), sizeof(double) * layers.size(), cudaMemcpyHostToDevice);
    if (e1 == cudaSuccess) e1 = cudaMemcpy(d_xi, m->ops.xi, sizeof(double) * MAXN, cudaMemcpyHostToDevice);
    MapParams mpd = mp;
    mpd.r_layers = d_layers;
    if (e1 == cudaSuccess) {
      k_nodes<<<(unsigned)((E * NP + 255) / 256), 256>>>(mpd, E, m->n, d_xi, m->x);
      e1 = cudaGetLastError();
    }
    if (e1 == cudaSuccess) e1 = cudaMemcpy(X.data(), m->x, sizeof(double) * X.size(), cudaMemcpyDeviceToHost);
    cudaFree(d_layers);
    cudaFree(d_xi);
    if (e1 != cudaSuccess) { free_mesh(m); return fail(DG_ECUDA, std::string("node kernel: ") + cudaGetErrorString(e1)); }
  }
  std::vector<int32_t> nbr, nbr_fo, face_e, face_f;
  rc = build_connectivity(m, X, nbr, nbr_fo, face_e, face_f);
  if (rc) { free_mesh(m); return rc; }
  m->nfaces = (long long)face_e.size();
  X.clear();
  X.shrink_to_fit();

  rc |= dalloc(&m->d_ops, 1);
  rc |= dalloc(&m->geo, E * 10 * NP);
  rc |= dalloc(&m->acc, E * 3 * NP);
  rc |= dalloc(&m->xg, E * 3 * NP);
  rc |= dalloc(&m->fgeo, E * 6 * 4 * NF);
  rc |= dalloc(&m->nbr, E * 6);
  rc |= dalloc(&m->nbr_fo, E * 6);
  rc |= dalloc(&m->face_e, m->nfaces);
  rc |= dalloc(&m->face_f, m->nfaces);
  rc |= dalloc(&m->ws.ug, 2 * E * 5 * NP);
  rc |= dalloc(&m->ws.uf, 2 * E * 30 * NF);
  rc |= dalloc(&m->ws.qg, 2 * E * 15 * NP);
  rc |= dalloc(&m->ws.qf, 2 * E * 90 * NF);
  rc |= dalloc(&m->ws.fh, 2 * E * 30 * NF);
  rc |= dalloc(&m->ws.tmp, 2 * m->ndof);
  rc |= dalloc(&m->ws.red, 1024);
  if (rc) { free_mesh(m); return DG_ENOMEM; }
  if (cudaMallocHost((void**)&m->ws.red_host, 1024 * sizeof(double)) != cudaSuccess) {
    free_mesh(m);
    return fail(DG_ENOMEM, "cudaMallocHost failed");
  }
  cudaError_t err = cudaSuccess;
  err = cudaMemcpy(m->d_ops, &m->ops, sizeof(Ops), cudaMemcpyHostToDevice);
  if (err == cudaSuccess) err = cudaMemcpy(m->nbr, nbr.data(), sizeof(int32_t) * nbr.size(), cudaMemcpyHostToDevice);
  if (err == cudaSuccess) err = cudaMemcpy(m->nbr_fo, nbr_fo.data(), sizeof(int32_t) * nbr_fo.size(), cudaMemcpyHostToDevice);
  if (err == cudaSuccess && m->nfaces)
    err = cudaMemcpy(m->face_e, face_e.data(), sizeof(int32_t) * face_e.size(), cudaMemcpyHostToDevice);
  if (err == cudaSuccess && m->nfaces)
    err = cudaMemcpy(m->face_f, face_f.data(), sizeof(int32_t) * face_f.size(), cudaMemcpyHostToDevice);
  if (err != cudaSuccess) {
    free_mesh(m);
    return fail(DG_ECUDA, std::string("dg_mesh_create upload: ") + cudaGetErrorString(err));
  }
  rc = drv_geometry(m, 0);
  if (rc == DG_OK && d.comp) {
    rc = dalloc(&m->mixg, E * 8 * NP) | dalloc(&m->mixf, E * 12 * NF);
    if (rc == DG_OK) rc = drv_mixture(m);
  }
  // the allocation-free residual's scratch array becomes resident here, where allocating is allowed
  if (rc == DG_OK) rc = static_scratch_address(m->device, &m->static_scratch);
  if (rc == DG_OK) err = cudaDeviceSynchronize();
  if (rc != DG_OK || err != cudaSuccess) {
    free_mesh(m);
    return rc ? rc : fail(DG_ECUDA, std::string("dg_mesh_create kernels: ") + cudaGetErrorString(err));
  }
  *out = m;
  return DG_OK;
}

extern "C" void dg_mesh_destroy(dg_mesh* mesh) {
  if (!mesh) return;
  cudaDeviceSynchronize();
  free_mesh(mesh);
}

extern "C" int dg_mesh_sizes(const dg_mesh* mesh, int64_t* n_elem, int32_t* n_p, int64_t* n_dof) {
  if (!mesh) return fail(DG_EINVAL, "dg_mesh_sizes: null mesh");
  if (n_elem) *n_elem = mesh->E;
  if (n_p) *n_p = mesh->np;
  if (n_dof) *n_dof = mesh->ndof;
  return DG_OK;
}

extern "C" int dg_mesh_nodes(const dg_mesh* mesh, double* x, void* stream) {
  if (!mesh || !x) return fail(DG_EINVAL, "dg_mesh_nodes: null argument");
  DG_CUDA_TRY(cudaMemcpyAsync(x, mesh->x, sizeof(double) * mesh->E * 3 * mesh->np, cudaMemcpyDeviceToDevice,
                              (cudaStream_t)stream));
  return DG_OK;
}

extern "C" int dg_mesh_set_interp(dg_mesh* mesh, int32_t mode) {
  if (!mesh) return fail(DG_EINVAL, "dg_mesh_set_interp: null mesh");
  if (mode != DG_INTERP_FP64 && mode != DG_INTERP_TC) return fail(DG_EINVAL, "dg_mesh_set_interp: unknown mode");
  if (mode == DG_INTERP_TC) {
    int dev = 0;
    DG_CUDA_TRY(cudaGetDevice(&dev));
    DG_CUDA_TRY(cudaSetDevice(mesh->device));
    const int rc = dg::interp_tc_prepare(mesh);
    cudaSetDevice(dev);
    if (rc) return rc;
  }
  mesh->interp_mode = mode;
  return DG_OK;
}

extern "C" int dg_gradient(dg_mesh* mesh, const double* u, double* q, void* stream) {
  dg::NvtxRange nvtx_range_("dg_gradient");
  if (!mesh || !u || !q) return fail(DG_EINVAL, "dg_gradient: null argument");
  cudaStream_t s = (cudaStream_t)stream;
  int rc = drv_gradient(mesh, u, nullptr, s);
  if (rc) return rc;
  return drv_q_to_nodal(mesh, q, s);
}

extern "C" int dg_residual(dg_mesh* mesh, const double* u, const double* q, double t, double* r, void* stream) {
  dg::NvtxRange nvtx_range_("dg_residual");
  if (!mesh || !u || !r) return fail(DG_EINVAL, "dg_residual: null argument");
  cudaStream_t s = (cudaStream_t)stream;
  int rc;
  if (q) {
    // interp of u (Gauss values and traces), then the given nodal q in Gauss space
    rc = drv_gradient(mesh, u, nullptr, s);   // fills U, UF (Q overwritten next)
    if (rc) return rc;
    rc = drv_q_from_nodal(mesh, q, s);
  } else {
    rc = drv_gradient(mesh, u, nullptr, s);
  }
  if (rc) return rc;
  return drv_residual(mesh, u, nullptr, t, r, nullptr, false, s);
}

namespace dg {

// out may alias x or y (each entry is read before it is written, by the same thread)
__global__ void k_axpby(long long n, double a, const double* x, double b, const double* y, double* out) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = a * x[i] + b * (y ? y[i] : 0.0);
}

// partial sums of squares (two vectors at once), fixed-size grid for a deterministic order
__global__ void k_sumsq2(long long n, const double* __restrict__ x, const double* __restrict__ y,
                         double* __restrict__ part) {
  __shared__ double sx[256], sy[256];
  double ax = 0.0, ay = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    ax = fma(x[i], x[i], ax);
    ay = fma(y[i], y[i], ay);
  }
  sx[threadIdx.x] = ax;
  sy[threadIdx.x] = ay;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (threadIdx.x < st) {
      sx[threadIdx.x] += sx[threadIdx.x + st];
      sy[threadIdx.x] += sy[threadIdx.x + st];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[blockIdx.x] = sx[0];
    part[256 + blockIdx.x] = sy[0];
  }
}

}  // namespace dg

extern "C" int dg_jvp(dg_mesh* mesh, const double* u, const double* v, double t, int32_t mode, double eps,
                      double* jv, double* r_out, void* stream) {
  dg::NvtxRange nvtx_range_("dg_jvp");
  if (!mesh || !u || !v || !jv) return fail(DG_EINVAL, "dg_jvp: null argument");
  cudaStream_t s = (cudaStream_t)stream;
  if (mode == DG_JV_EXACT) {
    int rc = drv_gradient(mesh, u, v, s);
    if (rc) return rc;
    return drv_residual(mesh, u, v, t, r_out, jv, true, s);
  }
  if (mode != DG_JV_FD) return fail(DG_EINVAL, "dg_jvp: unknown mode");
  const long long n = mesh->ndof;
  if (!(eps > 0.0)) {
    prof_begin(mesh, s, KK_BLAS);
    k_sumsq2<<<256, 256, 0, s>>>(n, u, v, mesh->ws.red);
    prof_end(mesh, s);
    DG_LAUNCH_CHECK("k_sumsq2");
    DG_CUDA_TRY(cudaMemcpyAsync(mesh->ws.red_host, mesh->ws.red, 512 * sizeof(double), cudaMemcpyDeviceToHost, s));
    DG_CUDA_TRY(cudaStreamSynchronize(s));
    double su = 0.0, sv = 0.0;
    for (int i = 0; i < 256; ++i) {
      su += mesh->ws.red_host[i];
      sv += mesh->ws.red_host[256 + i];
    }
    if (!(sv > 0.0)) return fail(DG_EINVAL, "dg_jvp: zero direction");
    eps = std::sqrt(2.220446049250313e-16) * (1.0 + std::sqrt(su)) / std::sqrt(sv);
  }
  double* r0 = r_out ? r_out : mesh->ws.tmp;
  double* up = mesh->ws.tmp + n;
  int rc = dg_residual(mesh, u, nullptr, t, r0, stream);
  if (rc) return rc;
  prof_begin(mesh, s, KK_BLAS);
  k_axpby<<<1024, 256, 0, s>>>(n, 1.0, u, eps, v, up);
  prof_end(mesh, s);
  DG_LAUNCH_CHECK("k_axpby");
  rc = dg_residual(mesh, up, nullptr, t, jv, stream);
  if (rc) return rc;
  prof_begin(mesh, s, KK_BLAS);
  k_axpby<<<1024, 256, 0, s>>>(n, 1.0 / eps, jv, -1.0 / eps, r0, jv);
  prof_end(mesh, s);
  DG_LAUNCH_CHECK("k_axpby");
  return DG_OK;
}

extern "C" int dg_mass_apply(dg_mesh* mesh, const double* v, double* mv, void* stream) {
  if (!mesh || !v || !mv) return fail(DG_EINVAL, "dg_mass_apply: null argument");
  return drv_mass(mesh, v, mv, (cudaStream_t)stream);
}

extern "C" int dg_mass_inverse_apply(dg_mesh* mesh, const double* v, double* mv, void* stream) {
  if (!mesh || !v || !mv) return fail(DG_EINVAL, "dg_mass_inverse_apply: null argument");
  return drv_mass_inv(mesh, v, mv, (cudaStream_t)stream);
}

static const char* kKernelNames[KK_COUNT] = {"k_interp", "k_grad", "k_faces", "k_volume", "k_tensor", "k_blas",
                                             "k_geometry", "k_lu", "k_precond_apply"};

extern "C" const char* dg_kernel_name(int32_t kind) {
  return (kind >= 0 && kind < KK_COUNT) ? kKernelNames[kind] : "";
}

extern "C" int dg_profile_start(dg_mesh* mesh, int32_t capacity) {
  if (!mesh || capacity < 1) return fail(DG_EINVAL, "dg_profile_start: bad argument");
  prof_release(mesh);
  Prof& p = mesh->prof;
  p.ev = new cudaEvent_t[2 * (size_t)capacity];
  p.kind = new int[capacity];
  for (int i = 0; i < 2 * capacity; ++i) {
    cudaError_t err = cudaEventCreate(&p.ev[i]);
    if (err != cudaSuccess) {
      p.cap = i / 2;
      for (int j = 2 * p.cap; j < i; ++j) cudaEventDestroy(p.ev[j]);
      prof_release(mesh);
      return fail(DG_ECUDA, std::string("cudaEventCreate: ") + cudaGetErrorString(err));
    }
  }
  p.cap = capacity;
  p.used = 0;
  p.launches = 0;
  p.on = true;
  return DG_OK;
}

extern "C" int dg_profile_stop(dg_mesh* mesh, int32_t n_kinds, double* ms, int32_t* count, int64_t* total) {
  if (!mesh) return fail(DG_EINVAL, "dg_profile_stop: null mesh");
  Prof& p = mesh->prof;
  for (int k = 0; k < n_kinds; ++k) {
    if (ms) ms[k] = 0.0;
    if (count) count[k] = 0;
  }
  int rc = DG_OK;
  for (int i = 0; i < p.used; ++i) {
    cudaError_t err = cudaEventSynchronize(p.ev[2 * i + 1]);
    float t = 0.0f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&t, p.ev[2 * i], p.ev[2 * i + 1]);
    if (err != cudaSuccess) {
      rc = fail(DG_ECUDA, std::string("dg_profile_stop: ") + cudaGetErrorString(err));
      break;
    }
    if (p.kind[i] < n_kinds) {
      if (ms) ms[p.kind[i]] += t;
      if (count) count[p.kind[i]] += 1;
    }
  }
  if (total) *total = p.launches;
  prof_release(mesh);
  return rc;
}

extern "C" int dg_residual_f32(dg_mesh* mesh, const double* u, double t, double* r, void* stream) {
  if (!mesh || !u || !r) return fail(DG_EINVAL, "dg_residual_f32: null argument");
  int rc = ensure_f32(mesh);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  rc = drv_gradient(mesh, u, nullptr, s, true);
  if (rc) return rc;
  return drv_residual(mesh, u, nullptr, t, r, nullptr, false, s, true);
}

extern "C" int dg_jvp_f32(dg_mesh* mesh, const double* u, const double* v, double t, double* jv, double* r_out,
                          void* stream) {
  if (!mesh || !u || !v || !jv) return fail(DG_EINVAL, "dg_jvp_f32: null argument");
  int rc = ensure_f32(mesh);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  rc = drv_gradient(mesh, u, v, s, true);
  if (rc) return rc;
  return drv_residual(mesh, u, v, t, r_out, jv, true, s, true);
}

int stage_jvp(dg_mesh* mesh, const double* u, const double* v, double t, double c, double* out, bool f32,
              cudaStream_t s, bool value_ready) {
  if (c == 0.0) return fail(DG_EINVAL, "stage operator needs dt a_ii != 0");
  if (f32) {
    int rc = ensure_f32(mesh);
    if (rc) return rc;
  }
  int rc = drv_gradient(mesh, u, v, s, f32, value_ready);
  if (rc) return rc;
  return drv_residual(mesh, u, v, t, nullptr, out, true, s, f32, c);
}

int stage_value_plane(dg_mesh* mesh, const double* u, bool f32, cudaStream_t s) {
  if (f32) {
    int rc = ensure_f32(mesh);
    if (rc) return rc;
  }
  return drv_gradient(mesh, u, nullptr, s, f32);
}

extern "C" int dg_eval_precision(dg_mesh* mesh, int32_t mode, const double* u, const double* v, double t, double* r,
                                 double* jv, void* stream) {
  if (!mesh || !u || (!r && !jv) || (v && !jv)) return fail(DG_EINVAL, "dg_eval_precision: bad argument");
  if (mode < DG_CM_FP32 || mode > DG_CM_FP16X3) return fail(DG_EINVAL, "dg_eval_precision: unknown mode");
  int rc = ensure_f32(mesh);
  if (rc) return rc;
  DG_DISPATCH(mesh, eval_cm(mesh, u, v, t, r, jv, mode, (cudaStream_t)stream));
}
