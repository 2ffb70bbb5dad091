// Internal declarations of the DG library: mesh storage, 1D operators, dual numbers, pointwise
// physics of the nondimensional thermosphere model (Eq. fluxSWNondimensional, Eq. LDG2).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/dg.h"

namespace dg {

constexpr int MAXN = 5;           // p <= 4

// --------------------------------------------------------------------------------------------
// error handling
// --------------------------------------------------------------------------------------------
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
#define DG_CUDA_TRY(expr)                                                                   \
  do {                                                                                      \
    cudaError_t err__ = (expr);                                                             \
    if (err__ != cudaSuccess)                                                               \
      return ::dg::fail(DG_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(err__));   \
  } while (0)
#define DG_LAUNCH_CHECK(name)                                                               \
  do {                                                                                      \
    cudaError_t err__ = cudaGetLastError();                                                 \
    if (err__ != cudaSuccess)                                                               \
      return ::dg::fail(DG_ECUDA, std::string(name) + ": " + cudaGetErrorString(err__));    \
  } while (0)

// --------------------------------------------------------------------------------------------
// 1D operators of the tensor basis (GLL nodal basis, Gauss quadrature), row-major [row][col]
// --------------------------------------------------------------------------------------------
struct Ops {
  double B[MAXN * MAXN];     // B[q][a]   = l^GLL_a(eta_q): nodes -> Gauss points
  double Binv[MAXN * MAXN];  // Binv[a][q] = l^Gauss_q(xi_a): Gauss points -> nodes
  double D[MAXN * MAXN];     // D[q][k]   = d l^Gauss_k / dx (eta_q): derivative on Gauss values
  double eL[MAXN], eR[MAXN]; // l^Gauss_k(-1), l^Gauss_k(+1): extrapolation to the faces
  double w[MAXN];            // Gauss weights
  double eta[MAXN];          // Gauss points
  double xi[MAXN];           // GLL nodes
};
void build_ops(int n, Ops* ops);   // host, defined in dg_ops.cu

// --------------------------------------------------------------------------------------------
// physics parameters (nondimensional, Sec. 2.4), passed by value to kernels
// --------------------------------------------------------------------------------------------
struct Phys {
  double gamma, c_mu, c_k, c_d, p_coef, cv, visc_exp, lam, t_wall;
  double omega[3];
  double cor;                     // 2 Fr / sqrt(gamma)
  int euv;
  double euv_amp, euv_inv2s2, euv_r_peak, euv_inv_w, euv_omega_t;
  // EUVAC: with Phi_j = sum_s w_s phi_s^j (w_s = chi_s / m_s*, or 1/m* on oxygen for a constant
  // composition), Q* = e^varrho sum_j B_j Phi_j exp(-tau_j), tau_j = euvac_cc e^varrho Phi_j H* Ch,
  // H* = T* r*^2 / (m* g_r0^2)
  int n_euvac;
  double euvac_B[40], euvac_phi[4][40], euvac_cc;
  double sun_cd, sun_sd, g_r0, inv_m;   // cos and sin of the declination, inner radius, 1/m*
  // variable composition (Sec. 2.1.1-2.1.2)
  int comp;
  double comp_a[6], comp_b[6], eddy_nu, eddy_alpha, inv_gamma;
};

// mixture properties at one point: c_v* = 1/m* and the conductivity factor sum_s x_s alpha_s/alpha_O
template <typename R>
struct Mix {
  R cv, kfac;
};

// --------------------------------------------------------------------------------------------
// mesh storage
// --------------------------------------------------------------------------------------------
struct Workspace {
  double* ug = nullptr;   // [2][E][5][Np]    Gauss values of u (and tangent)
  double* uf = nullptr;   // [2][E][6][5][Nf] face traces of u
  double* qg = nullptr;   // [2][E][3][5][Np] Gauss values of q
  double* qf = nullptr;   // [2][E][6][15][Nf] face traces of q
  double* fh = nullptr;   // [2][E][6][5][Nf] F_hat . (w n dS) per element face
  double* qx = nullptr;   // [E][6][15][Nf] cross gradient traces (block-diagonal tangent only)
  double* tmp = nullptr;  // [2][n_dof] scratch vectors (FD Jv, nodal q)
  double* red = nullptr;  // [1024] reduction partials
  double* red_host = nullptr;  // pinned host copy
};

}  // namespace dg

namespace dg {
enum KernelKind {
  KK_INTERP = 0, KK_GRAD, KK_FACES, KK_VOLUME, KK_TENSOR, KK_BLAS, KK_GEOMETRY, KK_LU, KK_PRECOND, KK_COUNT
};
struct Solver;
struct Mlp;
template <typename R>
struct WorkT {
  R *ug, *uf, *qg, *qf, *fh, *qx;
  const R *geo, *fgeo, *acc, *xg;
  const R *mixg, *mixf;   // variable composition at Gauss / face points (NULL without it)
};
// resident CTAs per device of a kernel at a launch shape, looked up once per mesh (the mesh fixes
// the device) and kernel instance
struct OccCache {
  static constexpr int CAP = 32;
  const void* fn[CAP] = {};
  size_t smem[CAP] = {};
  long long val[CAP] = {};
  int n = 0;
};
struct Prof {
  bool on = false;
  int cap = 0, used = 0;
  long long launches = 0;
  cudaEvent_t* ev = nullptr;
  int* kind = nullptr;
};
}  // namespace dg

struct dg_mesh {
  dg_mesh_desc desc;
  dg::Prof prof;
  dg::OccCache occ;
  int n, np, nf;           // points per direction, per element, per face
  int64_t E, ndof, nfaces;
  int device;
  dg::Phys phys;
  dg::Ops ops;
  dg::Ops* d_ops = nullptr;
  double* x = nullptr;     // [E][3][Np] node coordinates
  double* geo = nullptr;   // [E][10][Np]: G[a][d] = W detJ dxi_a/dx_d (9), W detJ (1)
  double* acc = nullptr;   // [E][3][Np]: static acceleration g/gamma - Fr^2/gamma w x (w x r)
  double* xg = nullptr;    // [E][3][Np]: Gauss point positions
  double* fgeo = nullptr;  // [E][6][4][Nf]: w n dS (3), w |n dS| (1), outward, own face order
  double* mixg = nullptr;  // [E][8][Np] variable composition at the Gauss points (desc.comp only)
  double* mixf = nullptr;  // [E][6][2][Nf] variable composition at the face points
  int32_t* nbr = nullptr;  // [E][6]: neighbour element, or -bc_kind for a boundary face
  int32_t* nbr_fo = nullptr; // [E][6]: neighbour local face | orientation << 3
  int32_t* face_e = nullptr; // [F] owner element of each face visited once by the face kernel
  int32_t* face_f = nullptr; // [F] owner local face
  dg::Workspace ws;
  dg::Solver* solver = nullptr;   // implicit-step storage, created on first use
  dg::WorkT<float> w32 = {};        // FP32 workspace and geometry, created on first FP32 call
  float* w32_base = nullptr;
  dg::Mlp* mlp = nullptr;           // learned preconditioner, created by dg_mlp_init
  double* static_scratch = nullptr; // device address of dg_residual_static's array on this device
  int interp_mode = DG_INTERP_FP64; // DG_INTERP_*: how the FP64 paths form Gauss values and traces
  uint16_t* tc_aslices = nullptr;   // tensor-core interpolation: operator digit slices (first use)
  int* tc_rowexp = nullptr;         //   their row exponents
  int* tc_err = nullptr;            //   set when a bounded wait of the kernel gave up
};

void dg_mlp_release(dg_mesh* m);

namespace dg {
int ensure_f32(dg_mesh* m);       // allocate and fill the FP32 workspace and geometry
// EUVAC band coefficients, Sun declination and Chapman constants of a description (false if the
// reference values needed are missing)
bool euvac_coefficients(const dg_mesh_desc& d, Phys& P);
// layer interfaces r_0 = r_in < ... < r_nz = r_out with heights h1 q^k (q solved by bisection so the
// layers fill the shell; h1 <= 0: uniform layers), Sec. 3.3
std::vector<double> radial_layers(double r_in, double r_out, int nz, double h1);
// device address of dg_residual_static's scratch array on the current device dev (looked up once
// per device; the lookup loads the module that holds the array)
int static_scratch_address(int dev, double** out);
// nodal -> Gauss values and face traces of NC planes (u, and v for NC = 2) on the tensor cores,
// FP64-accurate (dg_tc_interp.cu); ug / uf as k_interp's outputs, plane 0 at the given pointers
template <int N, int NC>
int interp_tc(dg_mesh* m, const double* u, const double* v, double* ug, double* uf, cudaStream_t s);
int interp_tc_prepare(dg_mesh* m);   // the operator's digit slices (allocates once per mesh)
void interp_tc_release(dg_mesh* m);
}
int mlp_setup(dg_mesh* mesh, const double* u, double dt_aii, cudaStream_t s);
// J_G v = M v - c J_r(u) v in one tangent pass (exact tangent; FP32 arithmetic when f32). With
// value_ready the workspace's value plane (Gauss values, traces and LDG gradient of u) was formed
// by stage_value_plane for this u and nothing has overwritten it since: only v's tangent is
// interpolated and differentiated.
int stage_jvp(dg_mesh* mesh, const double* u, const double* v, double t, double c, double* out, bool f32,
              cudaStream_t s, bool value_ready = false);
int stage_value_plane(dg_mesh* mesh, const double* u, bool f32, cudaStream_t s);
int mlp_apply(dg_mesh* mesh, const double* x, double* y, cudaStream_t s);

void dg_solver_release(dg_mesh* m);

namespace dg {

// tracing of kernel launches (dg_profile_start / dg_profile_stop)
inline void prof_begin(dg_mesh* m, cudaStream_t s, int kind) {
  Prof& p = m->prof;
  if (!p.on) return;
  if (p.used < p.cap) {
    cudaEventRecord(p.ev[2 * p.used], s);
    p.kind[p.used] = kind;
  }
}
inline void prof_end(dg_mesh* m, cudaStream_t s) {
  Prof& p = m->prof;
  if (!p.on) return;
  if (p.used < p.cap) {
    cudaEventRecord(p.ev[2 * p.used + 1], s);
    p.used++;
  }
  p.launches++;
}

// per-N kernel drivers (dg_kernels_N*.cu)
template <int N>
struct Driver {
  static int geometry(dg_mesh* m, cudaStream_t s);
  // f32: FP32 data and arithmetic; inputs and outputs stay FP64
  static int gradient(dg_mesh* m, const double* u, const double* v, cudaStream_t s, bool f32 = false,
                      bool tangent_only = false);
  static int residual(dg_mesh* m, const double* u, const double* v, double t, double* r, double* jv,
                      bool tangent, cudaStream_t s, bool f32 = false, double stage_c = 0.0);
  static int q_to_nodal(dg_mesh* m, double* q, cudaStream_t s);
  static int q_from_nodal(dg_mesh* m, const double* q, cudaStream_t s);
  static int mass(dg_mesh* m, const double* v, double* mv, cudaStream_t s, bool f32 = false);
  static int mass_inv(dg_mesh* m, const double* v, double* mv, cudaStream_t s);
  static int mixture(dg_mesh* m);
  // J_r probe restricted to each element's own diagonal block (exact, one column per element)
  static int jv_blockdiag(dg_mesh* m, const double* u, const double* probe, double t, double* jv, cudaStream_t s,
                          bool f32 = false, bool tangent_only = false);
  // FP32 residual (v == NULL) or fused residual + exact Jv with a contraction mode (CM_*)
  static int eval_cm(dg_mesh* m, const double* u, const double* v, double t, double* r, double* jv, int cm,
                     cudaStream_t s);
  template <int CM>
  static int eval_cm_t(dg_mesh* m, const double* u, const double* v, double t, double* r, double* jv, cudaStream_t s);
  template <typename R>
  static int gradient_p(dg_mesh* m, const double* u, const double* v, cudaStream_t s, bool tangent_only);
  template <typename R>
  static int residual_p(dg_mesh* m, double t, double* r, double* jv, bool tangent, cudaStream_t s, double stage_c);
  template <typename R>
  static int jv_blockdiag_p(dg_mesh* m, const double* u, const double* probe, double t, double* jv, cudaStream_t s,
                            bool tangent_only);
};

// orientation map of face point (is, it) to the neighbour's face point index
__host__ __device__ inline int orient_map(int o, int is, int it, int n) {
  int a = (o & 1) ? it : is;
  int b = (o & 1) ? is : it;
  if (o & 2) a = n - 1 - a;
  if (o & 4) b = n - 1 - b;
  return a + n * b;
}

// --------------------------------------------------------------------------------------------
// forward-mode dual numbers over a real type T: value and directional derivative
// --------------------------------------------------------------------------------------------
template <typename T>
struct DualT {
  T v, d;
};
using Dual = DualT<double>;
template <typename T> __host__ __device__ inline DualT<T> operator+(DualT<T> a, DualT<T> b) { return {a.v + b.v, a.d + b.d}; }
template <typename T> __host__ __device__ inline DualT<T> operator-(DualT<T> a, DualT<T> b) { return {a.v - b.v, a.d - b.d}; }
template <typename T> __host__ __device__ inline DualT<T> operator-(DualT<T> a) { return {-a.v, -a.d}; }
template <typename T> __host__ __device__ inline DualT<T> operator*(DualT<T> a, DualT<T> b) { return {a.v * b.v, a.v * b.d + a.d * b.v}; }
template <typename T> __host__ __device__ inline DualT<T> operator+(DualT<T> a, T b) { return {a.v + b, a.d}; }
template <typename T> __host__ __device__ inline DualT<T> operator+(T b, DualT<T> a) { return {a.v + b, a.d}; }
template <typename T> __host__ __device__ inline DualT<T> operator-(DualT<T> a, T b) { return {a.v - b, a.d}; }
template <typename T> __host__ __device__ inline DualT<T> operator-(T b, DualT<T> a) { return {b - a.v, -a.d}; }
template <typename T> __host__ __device__ inline DualT<T> operator*(DualT<T> a, T b) { return {a.v * b, a.d * b}; }
template <typename T> __host__ __device__ inline DualT<T> operator*(T b, DualT<T> a) { return {a.v * b, a.d * b}; }

template <typename S> struct RealOf { using type = S; };
template <typename T> struct RealOf<DualT<T>> { using type = T; };

__device__ inline double s_exp(double x) { return exp(x); }
__device__ inline float s_exp(float x) { return expf(x); }
template <typename T> __device__ inline DualT<T> s_exp(DualT<T> x) {
  const T e = s_exp(x.v);
  return {e, e * x.d};
}
__device__ inline double s_erfcx(double x) { return erfcx(x); }
__device__ inline float s_erfcx(float x) { return erfcxf(x); }
// d/dy erfcx(y) = 2 y erfcx(y) - 2/sqrt(pi)
template <typename T> __device__ inline DualT<T> s_erfcx(DualT<T> x) {
  const T e = s_erfcx(x.v);
  return {e, (T(2) * x.v * e - T(1.1283791670955126)) * x.d};
}
template <typename T> __device__ inline T s_inv(T x) { return T(1) / x; }
template <typename T> __device__ inline DualT<T> s_inv(DualT<T> x) {
  const T r = T(1) / x.v;
  return {r, -x.d * r * r};
}
__device__ inline double s_sqrt(double x) { return sqrt(x); }
__device__ inline float s_sqrt(float x) { return sqrtf(x); }
template <typename T> __device__ inline DualT<T> s_sqrt(DualT<T> x) {
  const T r = s_sqrt(x.v);
  return {r, x.d / (T(2) * r)};
}
__device__ inline double s_log(double x) { return log(x); }
__device__ inline float s_log(float x) { return logf(x); }
template <typename T> __device__ inline DualT<T> s_log(DualT<T> x) { return {s_log(x.v), x.d / x.v}; }
template <typename S> __device__ inline S s_zero() { return S{}; }
template <typename S> __device__ inline S s_const(typename RealOf<S>::type c);
template <> __device__ inline double s_const<double>(double c) { return c; }
template <> __device__ inline float s_const<float>(float c) { return c; }
template <> __device__ inline Dual s_const<Dual>(double c) { return {c, 0.0}; }
template <> __device__ inline DualT<float> s_const<DualT<float>>(float c) { return {c, 0.0f}; }

// physics parameters in the working precision
template <typename R>
struct PhysT {
  R gamma, c_mu, c_k, c_d, p_coef, cv, visc_exp, lam, t_wall;
  R omega[3];
  R cor;
  int euv;
  R euv_amp, euv_inv2s2, euv_r_peak, euv_inv_w, euv_omega_t;
  int n_euvac;
  R euvac_B[40], euvac_phi[4][40], euvac_cc;
  R sun_cd, sun_sd, g_r0, inv_m;
  int comp;
  R comp_a[6], comp_b[6], eddy_nu, eddy_alpha, inv_gamma;
};
template <typename R>
inline PhysT<R> phys_as(const Phys& P) {
  PhysT<R> q;
  q.gamma = (R)P.gamma; q.c_mu = (R)P.c_mu; q.c_k = (R)P.c_k; q.c_d = (R)P.c_d; q.p_coef = (R)P.p_coef;
  q.cv = (R)P.cv; q.visc_exp = (R)P.visc_exp; q.lam = (R)P.lam; q.t_wall = (R)P.t_wall;
  for (int k = 0; k < 3; ++k) q.omega[k] = (R)P.omega[k];
  q.cor = (R)P.cor; q.euv = P.euv; q.euv_amp = (R)P.euv_amp; q.euv_inv2s2 = (R)P.euv_inv2s2;
  q.euv_r_peak = (R)P.euv_r_peak; q.euv_inv_w = (R)P.euv_inv_w; q.euv_omega_t = (R)P.euv_omega_t;
  q.n_euvac = P.n_euvac;
  for (int j = 0; j < 40; ++j) {
    q.euvac_B[j] = (R)P.euvac_B[j];
    for (int s = 0; s < 4; ++s) q.euvac_phi[s][j] = (R)P.euvac_phi[s][j];
  }
  q.euvac_cc = (R)P.euvac_cc;
  q.sun_cd = (R)P.sun_cd; q.sun_sd = (R)P.sun_sd; q.g_r0 = (R)P.g_r0; q.inv_m = (R)P.inv_m;
  q.comp = P.comp;
  for (int k = 0; k < 6; ++k) {
    q.comp_a[k] = (R)P.comp_a[k];
    q.comp_b[k] = (R)P.comp_b[k];
  }
  q.eddy_nu = (R)P.eddy_nu; q.eddy_alpha = (R)P.eddy_alpha; q.inv_gamma = (R)P.inv_gamma;
  return q;
}

// --------------------------------------------------------------------------------------------
// pointwise physics (Eq. fluxSWNondimensional): flux F[c][d], source s[c]
//   u = (varrho, sqrt(rho) v, sqrt(rho) T), q[d][c] ~ d u_c / d x_d
// --------------------------------------------------------------------------------------------
template <typename S>
struct Prim {
  S isr, v[3], T, gv[3][3], gT[3], div, eps[3][3], mu, kappa;
};

template <typename S, typename R = typename RealOf<S>::type>
__device__ inline void transport(const PhysT<R>& P, const S& T, const S& isr, const Mix<R>& mx, S& mu, S& kappa) {
  if (P.comp) {
    // mu_m* = sqrt(T* m*), kappa_m* = kfac T*^0.69, plus the eddy offsets nu_e rho* and alpha_e rho* / m*
    const S rho = s_inv(isr * isr);   // e^varrho
    mu = s_sqrt(T * (R(1) / mx.cv)) + P.eddy_nu * rho;
    kappa = mx.kfac * s_exp(R(0.69) * s_log(T)) + (P.eddy_alpha * mx.cv) * rho;
  } else {
    mu = (P.visc_exp != R(0)) ? s_exp(P.visc_exp * s_log(T)) : s_const<S>(R(1));
    kappa = mu;
  }
}

template <typename S, typename R = typename RealOf<S>::type>
__device__ inline void primitives(const PhysT<R>& P, const S u[5], const S q[3][5], Prim<S>& w, const Mix<R>& mx) {
  w.isr = s_exp(R(-0.5) * u[0]);
  for (int m = 0; m < 3; ++m) w.v[m] = u[1 + m] * w.isr;
  w.T = u[4] * w.isr;
  for (int m = 0; m < 3; ++m)
    for (int d = 0; d < 3; ++d) w.gv[m][d] = w.isr * (q[d][1 + m] - R(0.5) * (u[1 + m] * q[d][0]));
  for (int d = 0; d < 3; ++d) w.gT[d] = w.isr * (q[d][4] - R(0.5) * (u[4] * q[d][0]));
  w.div = w.gv[0][0] + w.gv[1][1] + w.gv[2][2];
  for (int m = 0; m < 3; ++m)
    for (int d = 0; d < 3; ++d) w.eps[m][d] = w.gv[m][d] + w.gv[d][m];
  for (int m = 0; m < 3; ++m) w.eps[m][m] = w.eps[m][m] - R(2.0 / 3.0) * w.div;
  transport(P, w.T, w.isr, mx, w.mu, w.kappa);
}

// flux F(u, q) . n  (n: 3 reals), viscous terms optional
template <typename S, typename R = typename RealOf<S>::type>
__device__ inline void flux_dot_n(const PhysT<R>& P, const S u[5], const S q[3][5], const R n[3], bool viscous,
                                  S out[5], const Mix<R>& mx) {
  Prim<S> w;
  const R pc = P.comp ? mx.cv * P.inv_gamma : P.p_coef;   // 1/(gamma m*)
  if (viscous) {
    primitives(P, u, q, w, mx);
  } else {
    w.isr = s_exp(R(-0.5) * u[0]);
    for (int m = 0; m < 3; ++m) w.v[m] = u[1 + m] * w.isr;
  }
  S vn = w.v[0] * n[0] + w.v[1] * n[1] + w.v[2] * n[2];
  out[0] = u[0] * vn;
  for (int m = 0; m < 3; ++m) out[1 + m] = u[1 + m] * vn + (pc * n[m]) * u[4];
  out[4] = u[4] * vn;
  if (viscous) {
    S cm = (P.c_mu * w.mu) * w.isr;
    S ck = ((P.c_k / (P.comp ? mx.cv : P.cv)) * w.kappa) * w.isr;
    for (int m = 0; m < 3; ++m)
      out[1 + m] = out[1 + m] - cm * (w.eps[m][0] * n[0] + w.eps[m][1] * n[1] + w.eps[m][2] * n[2]);
    out[4] = out[4] - ck * (w.gT[0] * n[0] + w.gT[1] * n[1] + w.gT[2] * n[2]);
  }
}

// stabilisation diagonal sigma(u_hat) = lambda0 + sigma_d (Eq. LDG2)
template <typename S, typename R = typename RealOf<S>::type>
__device__ inline void sigma_diag(const PhysT<R>& P, const S uh[5], S sg[5], const Mix<R>& mx) {
  S isr = s_exp(R(-0.5) * uh[0]);
  S T = uh[4] * isr;
  S mu, kappa;
  transport(P, T, isr, mx, mu, kappa);
  S sm = P.lam + (P.c_mu * mu) * isr;
  sg[0] = s_const<S>(P.lam);
  sg[1] = sm;
  sg[2] = sm;
  sg[3] = sm;
  sg[4] = P.lam + ((P.c_k / (P.comp ? mx.cv : P.cv)) * kappa) * isr;
}

template <typename S, typename R = typename RealOf<S>::type>
__device__ inline void wall_trace(const PhysT<R>& P, const S u[5], S ub[5]) {
  ub[0] = u[0];
  ub[1] = s_zero<S>();
  ub[2] = s_zero<S>();
  ub[3] = s_zero<S>();
  ub[4] = s_exp(R(0.5) * u[0]) * P.t_wall;
}

}  // namespace dg
