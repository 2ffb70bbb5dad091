// Internal declarations of the DG library: mesh storage, 1D operators, dual numbers, pointwise
// physics of the nondimensional thermosphere model (Eq. fluxSWNondimensional, Eq. LDG2).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string>

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
  int32_t* nbr = nullptr;  // [E][6]: neighbour element, or -bc_kind for a boundary face
  int32_t* nbr_fo = nullptr; // [E][6]: neighbour local face | orientation << 3
  int32_t* face_e = nullptr; // [F] owner element of each face visited once by the face kernel
  int32_t* face_f = nullptr; // [F] owner local face
  dg::Workspace ws;
  dg::Solver* solver = nullptr;   // implicit-step storage, created on first use
};

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
  static int gradient(dg_mesh* m, const double* u, const double* v, cudaStream_t s);
  static int residual(dg_mesh* m, const double* u, const double* v, double t, double* r, double* jv,
                      bool tangent, cudaStream_t s);
  static int q_to_nodal(dg_mesh* m, double* q, cudaStream_t s);
  static int q_from_nodal(dg_mesh* m, const double* q, cudaStream_t s);
  static int mass(dg_mesh* m, const double* v, double* mv, cudaStream_t s);
  // J_r probe restricted to each element's own diagonal block (exact, one column per element)
  static int jv_blockdiag(dg_mesh* m, const double* u, const double* probe, double t, double* jv, cudaStream_t s);
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
// forward-mode dual numbers: value and directional derivative
// --------------------------------------------------------------------------------------------
struct Dual {
  double v, d;
};
__host__ __device__ inline Dual mk(double v, double d) { return Dual{v, d}; }
__host__ __device__ inline Dual operator+(Dual a, Dual b) { return Dual{a.v + b.v, a.d + b.d}; }
__host__ __device__ inline Dual operator-(Dual a, Dual b) { return Dual{a.v - b.v, a.d - b.d}; }
__host__ __device__ inline Dual operator-(Dual a) { return Dual{-a.v, -a.d}; }
__host__ __device__ inline Dual operator*(Dual a, Dual b) { return Dual{a.v * b.v, a.v * b.d + a.d * b.v}; }
__host__ __device__ inline Dual operator+(Dual a, double b) { return Dual{a.v + b, a.d}; }
__host__ __device__ inline Dual operator+(double b, Dual a) { return Dual{a.v + b, a.d}; }
__host__ __device__ inline Dual operator-(Dual a, double b) { return Dual{a.v - b, a.d}; }
__host__ __device__ inline Dual operator-(double b, Dual a) { return Dual{b - a.v, -a.d}; }
__host__ __device__ inline Dual operator*(Dual a, double b) { return Dual{a.v * b, a.d * b}; }
__host__ __device__ inline Dual operator*(double b, Dual a) { return Dual{a.v * b, a.d * b}; }

__device__ inline double s_exp(double x) { return exp(x); }
__device__ inline Dual s_exp(Dual x) {
  double e = exp(x.v);
  return Dual{e, e * x.d};
}
__device__ inline double s_log(double x) { return log(x); }
__device__ inline Dual s_log(Dual x) { return Dual{log(x.v), x.d / x.v}; }
__device__ inline double s_val(double x) { return x; }
__device__ inline double s_val(Dual x) { return x.v; }
template <typename S> __device__ inline S s_zero();
template <> __device__ inline double s_zero<double>() { return 0.0; }
template <> __device__ inline Dual s_zero<Dual>() { return Dual{0.0, 0.0}; }
template <typename S> __device__ inline S s_const(double c);
template <> __device__ inline double s_const<double>(double c) { return c; }
template <> __device__ inline Dual s_const<Dual>(double c) { return Dual{c, 0.0}; }

// --------------------------------------------------------------------------------------------
// pointwise physics (Eq. fluxSWNondimensional): flux F[c][d], source s[c]
//   u = (varrho, sqrt(rho) v, sqrt(rho) T), q[d][c] ~ d u_c / d x_d
// --------------------------------------------------------------------------------------------
template <typename S>
struct Prim {
  S isr, v[3], T, gv[3][3], gT[3], div, eps[3][3], mu;
};

template <typename S>
__device__ inline void primitives(const Phys& P, const S u[5], const S q[3][5], Prim<S>& w) {
  w.isr = s_exp(-0.5 * u[0]);
  for (int m = 0; m < 3; ++m) w.v[m] = u[1 + m] * w.isr;
  w.T = u[4] * w.isr;
  for (int m = 0; m < 3; ++m)
    for (int d = 0; d < 3; ++d) w.gv[m][d] = w.isr * (q[d][1 + m] - 0.5 * (u[1 + m] * q[d][0]));
  for (int d = 0; d < 3; ++d) w.gT[d] = w.isr * (q[d][4] - 0.5 * (u[4] * q[d][0]));
  w.div = w.gv[0][0] + w.gv[1][1] + w.gv[2][2];
  for (int m = 0; m < 3; ++m)
    for (int d = 0; d < 3; ++d) w.eps[m][d] = w.gv[m][d] + w.gv[d][m];
  for (int m = 0; m < 3; ++m) w.eps[m][m] = w.eps[m][m] - (2.0 / 3.0) * w.div;
  w.mu = (P.visc_exp != 0.0) ? s_exp(P.visc_exp * s_log(w.T)) : s_const<S>(1.0);
}

// flux F(u, q) . n  (n: 3 doubles), viscous terms optional
template <typename S>
__device__ inline void flux_dot_n(const Phys& P, const S u[5], const S q[3][5], const double n[3],
                                  bool viscous, S out[5]) {
  S isr = s_exp(-0.5 * u[0]);
  S v[3] = {u[1] * isr, u[2] * isr, u[3] * isr};
  S vn = v[0] * n[0] + v[1] * n[1] + v[2] * n[2];
  out[0] = u[0] * vn;
  for (int m = 0; m < 3; ++m) out[1 + m] = u[1 + m] * vn + (P.p_coef * n[m]) * u[4];
  out[4] = u[4] * vn;
  if (viscous) {
    Prim<S> w;
    primitives(P, u, q, w);
    S cm = (P.c_mu * w.mu) * w.isr;
    S ck = ((P.c_k / P.cv) * w.mu) * w.isr;
    for (int m = 0; m < 3; ++m)
      out[1 + m] = out[1 + m] - cm * (w.eps[m][0] * n[0] + w.eps[m][1] * n[1] + w.eps[m][2] * n[2]);
    out[4] = out[4] - ck * (w.gT[0] * n[0] + w.gT[1] * n[1] + w.gT[2] * n[2]);
  }
}

// stabilisation diagonal sigma(u_hat) = lambda0 + sigma_d (Eq. LDG2)
template <typename S>
__device__ inline void sigma_diag(const Phys& P, const S uh[5], S sg[5]) {
  S isr = s_exp(-0.5 * uh[0]);
  S T = uh[4] * isr;
  S mu = (P.visc_exp != 0.0) ? s_exp(P.visc_exp * s_log(T)) : s_const<S>(1.0);
  S sm = P.lam + (P.c_mu * mu) * isr;
  sg[0] = s_const<S>(P.lam);
  sg[1] = sm;
  sg[2] = sm;
  sg[3] = sm;
  sg[4] = P.lam + ((P.c_k / P.cv) * mu) * isr;
}

template <typename S>
__device__ inline void wall_trace(const Phys& P, const S u[5], S ub[5]) {
  ub[0] = u[0];
  ub[1] = s_zero<S>();
  ub[2] = s_zero<S>();
  ub[3] = s_zero<S>();
  ub[4] = s_exp(0.5 * u[0]) * P.t_wall;
}

}  // namespace dg
