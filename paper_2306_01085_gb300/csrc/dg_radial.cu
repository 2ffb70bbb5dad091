// Radial 1D ensemble (Sec. 4.3): the spherically symmetric restriction of the LDG discretisation
// for many independent columns at once, and their implicit DIRK steps.
//
// Per column, on elements [r_L, r_R] with (p+1) Gauss points r_g, weights w_g, J = (r_R - r_L)/2,
// W_g = w_g J r_g^2 (mass weights) and G_g = w_g r_g^2 (= W_g d xi/dr), in Gauss space (the values
// at the Gauss points of the degree-p fields; nodal GLL values map there by the square B):
//   gradient   q_j = [ -sum_g D_gj G_g U_g - 2 w_j J r_j U_j + r_R^2 u_hat_R eR_j - r_L^2 u_hat_L eL_j ] / W_j
//              for varrho, m = sqrt(rho) v_r and e = sqrt(rho) T, and Q_tt,j = m_j / r_j
//   residual   R_j = sum_g D_gj G_g F_r,g + W_j (s_j + [momentum] 2 F_tt,j / r_j)
//                    - r_R^2 F_hat_R eR_j + r_L^2 F_hat_L eL_j,        r_nodal = B^T R
// with D_gj = l'_j(xi_g) (Gauss Lagrange basis) and eL / eR its values at -1 / +1. These follow from
// the symmetric weak form term by term (the r^2 dr measure; div(p r_hat) = (r^2 p)'/r^2; the
// tangential part of the radial velocity's gradient), the same identities the shell kernels use.
//
// Kernels (one thread per (column, element) or (column, face); the column index is the fastest, so
// a warp reads 32 consecutive columns of one element: coalesced, and the element's geometry is a
// broadcast):
//   k_rgrad   nodal u (and tangent) -> Gauss values of q
//   k_rface   traces of u and q on both sides -> r_f^2 F_hat (Eq. LDG2) at every interface
//   k_rvol    pointwise flux and source, weak derivative, lifting, B^T -> nodal r (and J v)
// The implicit step assembles each column's stage Jacobian J_G = M - dt a_ii J_r in FP32 by
// colored probing (elements five apart share a probe: a perturbation reaches the residual of its
// own element and the two on each side, through the LDG gradient of the neighbours) and factors it
// by banded LU with partial pivoting, one thread per column; Newton iterates on the FP64 residual.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "dg_internal.cuh"
#include "dg_nvtx.h"

struct dg_radial;

namespace dg {
namespace rad {

constexpr int MAXN = 5;

// 1D operators (from build_ops) passed by value
template <typename R>
struct ROps {
  R B[MAXN * MAXN];   // B[g][i] = l^GLL_i(xi_g)
  R D[MAXN * MAXN];   // D[g][j] = l^Gauss_j'(xi_g)
  R eL[MAXN], eR[MAXN];
};

// physics numbers of the ensemble in the working precision
template <typename R>
struct RPhys {
  R gamma, c_mu, c_k, c_d, pc, cv, visc_exp, lam, t_wall, g_r0;
  int euv, bc_lo, bc_hi;
  int n_euvac;
  R B[40], phi[40], cc, sun_cd, sun_sd, omega_t, inv_m;   // EUVAC (oxygen), efficiency 1
};

// per element geometry: [E] rL, rR; [E][N] rg, W = w J r^2, G = w r^2, T2 = 2 w J r
template <typename R>
struct RGeo {
  const R *rL, *rR, *rg, *W, *G, *T2;
};

// per column parameters [5][n_col]: epsilon, alpha0, site unit vector
template <typename R>
struct RPrm {
  const R* p;
  long long nc;
  __device__ R eps(long long c) const { return p[c]; }
  __device__ R alpha(long long c) const { return p[nc + c]; }
  __device__ R site(int d, long long c) const { return p[(2 + d) * nc + c]; }
};

// ------------------------------------------------------------------------------------------------
// pointwise physics of the symmetric problem (the radial components of Eq. fluxSWNondimensional)
// ------------------------------------------------------------------------------------------------
template <typename S>
struct Prim1 {
  S isr, v, T, gvr, gvt, gT, div, er, et, mu, kap;
};

template <typename S, typename R>
__device__ __forceinline__ void prim1(const RPhys<R>& P, const S u[3], const S q[4], R alpha, Prim1<S>& w) {
  w.isr = s_exp(R(-0.5) * u[0]);
  w.v = u[1] * w.isr;
  w.T = u[2] * w.isr;
  w.gvr = w.isr * (q[1] - R(0.5) * (u[1] * q[0]));
  w.gvt = w.isr * q[2];
  w.gT = w.isr * (q[3] - R(0.5) * (u[2] * q[0]));
  w.div = w.gvr + R(2) * w.gvt;
  w.er = R(2) * w.gvr - R(2.0 / 3.0) * w.div;
  w.et = R(2) * w.gvt - R(2.0 / 3.0) * w.div;
  w.mu = (P.visc_exp != R(0)) ? s_exp(P.visc_exp * s_log(w.T)) : s_const<S>(R(1));
  w.kap = alpha * w.mu;
}

// radial fluxes F (varrho, F_rr, e) and the tangential momentum flux Ftt
template <typename S, typename R>
__device__ __forceinline__ void flux1(const RPhys<R>& P, const S u[3], const S q[4], R alpha, bool viscous, S F[3],
                                      S& Ftt) {
  Prim1<S> w;
  if (viscous) {
    prim1(P, u, q, alpha, w);
  } else {
    w.isr = s_exp(R(-0.5) * u[0]);
    w.v = u[1] * w.isr;
  }
  F[0] = u[0] * w.v;
  F[1] = u[1] * w.v + P.pc * u[2];
  Ftt = P.pc * u[2];
  F[2] = u[2] * w.v;
  if (viscous) {
    const S cm = (P.c_mu * w.mu) * w.isr;
    const S ck = ((P.c_k / P.cv) * w.kap) * w.isr;
    F[1] = F[1] - cm * w.er;
    Ftt = Ftt - cm * w.et;
    F[2] = F[2] - ck * w.gT;
  }
}

template <typename S, typename R>
__device__ __forceinline__ void sigma1(const RPhys<R>& P, const S uh[3], R alpha, S sg[3]) {
  const S isr = s_exp(R(-0.5) * uh[0]);
  const S T = uh[2] * isr;
  const S mu = (P.visc_exp != R(0)) ? s_exp(P.visc_exp * s_log(T)) : s_const<S>(R(1));
  sg[0] = s_const<S>(P.lam);
  sg[1] = P.lam + (P.c_mu * mu) * isr;
  sg[2] = P.lam + ((P.c_k / P.cv) * (alpha * mu)) * isr;
}

template <typename S, typename R>
__device__ __forceinline__ void wall1(const RPhys<R>& P, const S u[3], S ub[3]) {
  ub[0] = u[0];
  ub[1] = s_zero<S>();
  ub[2] = s_exp(R(0.5) * u[0]) * P.t_wall;
}

template <typename R> __device__ __forceinline__ R val_of(R x) { return x; }
template <typename R> __device__ __forceinline__ R val_of(DualT<R> x) { return x.v; }

// EUVAC heating q* (efficiency 1) at radius r above the site, Sec. 2.2 with Smith & Smith Chapman
// depths for the single absorber (oxygen); zero in the Earth's shadow. Bands whose optical depth
// exceeds 40 are skipped: their attenuated flux is below e^-40 (4e-18) of the band's own.
template <typename S, typename R>
__device__ __forceinline__ S heat1(const RPhys<R>& P, R r, const R site[3], R t, const S& isr, const S& T) {
  const R wt = P.omega_t * t;
  R cchi = site[0] * (-P.sun_cd * cos(wt)) + site[1] * (P.sun_cd * sin(wt)) + site[2] * P.sun_sd;
  cchi = fmin(R(1), fmax(R(-1), cchi));
  const R schi = sqrt(fmax(R(0), R(1) - cchi * cchi));
  if (!(cchi > R(0) || schi * r > P.g_r0)) return s_zero<S>();
  const S sr = s_inv(isr);
  const S er = sr * sr;                                   // e^varrho
  const S Hs = T * (r * r * P.inv_m / (P.g_r0 * P.g_r0)); // H* = T* r*^2 / (m* g_r0^2)
  const S rt = r * s_inv(Hs);
  const S ex = s_erfcx(s_sqrt(R(0.5) * rt) * fabs(cchi));
  const S base = s_sqrt(R(1.5707963267948966) * rt);
  S ch;
  if (cchi > R(0)) ch = base * ex;
  else ch = base * (R(2) * s_exp(rt * (R(1) - schi)) - ex);
  const S k = (P.cc * er) * Hs * ch;
  S qs = s_zero<S>();
  const R kv = val_of(k);
#pragma unroll 1
  for (int j = 0; j < P.n_euvac; ++j) {
    const R Phi = P.inv_m * P.phi[j];
    if (Phi * kv < R(40)) qs = qs + (P.B[j] * Phi) * s_exp(-Phi * k);
  }
  return er * qs;
}

// source (s_varrho, s_m + 2 F_tt / r, s_e) at a Gauss point
template <typename S, typename R>
__device__ __forceinline__ void source1(const RPhys<R>& P, const S u[3], const S q[4], R r, R alpha, R eps,
                                        const R site[3], R t, S F[3], S src[3]) {
  Prim1<S> w;
  prim1(P, u, q, alpha, w);
  const S cm = (P.c_mu * w.mu) * w.isr;
  const S ck = ((P.c_k / P.cv) * w.kap) * w.isr;
  const S Ftt = P.pc * u[2] - cm * w.et;
  F[0] = u[0] * w.v;
  F[1] = u[1] * w.v + P.pc * u[2] - cm * w.er;
  F[2] = u[2] * w.v - ck * w.gT;
  const R a_r = -(P.g_r0 / r) * (P.g_r0 / r) / P.gamma;
  src[0] = (u[0] - R(1)) * w.div;
  src[1] = s_inv(w.isr) * a_r + R(0.5) * (w.div * u[1]) - (R(0.5) * P.pc) * (u[2] * q[0]) + R(0.5) * (cm * w.er * q[0]) +
           (R(2) / r) * Ftt;
  S s2 = (R(1.5) - P.gamma) * (u[2] * w.div) + R(0.5) * (ck * w.gT * q[0]) +
         ((P.c_d / P.cv) * w.mu) * (w.isr * (w.er * w.gvr + R(2) * (w.et * w.gvt)));
  if (P.euv == DG_EUV_EUVAC) s2 = s2 + (eps * heat1<S, R>(P, r, site, t, w.isr, w.T)) * (R(1) / P.cv) * w.isr;
  src[2] = s2;
}

// ------------------------------------------------------------------------------------------------
// element kernels. Plane layout of the workspace (R): qg [NC][4][E][N][nc], fh [NC][3][E + 1][nc].
// PROBE (Jacobian assembly, NC = 2, R = float): the tangent of u is the probe (color, var a, node i)
// of blockIdx.y, 1 at (a, i) of every element k with k % 5 == color; tangent outputs go to the
// probe's own planes, and probe 0 also writes the value plane.
// ------------------------------------------------------------------------------------------------
template <typename S, int NC, typename R>
__device__ __forceinline__ S ldp(const R* p, long long plane) {
  if constexpr (NC == 1) return p[0];
  else return S{p[0], p[plane]};
}
template <typename R>
__device__ __forceinline__ void stp(R* p, long long, R v) { p[0] = v; }
template <typename R>
__device__ __forceinline__ void stp(R* p, long long plane, DualT<R> v) {
  p[0] = v.v;
  p[plane] = v.d;
}

struct Probe {
  int color, var, node;
  __device__ bool hit(int k, int c, int i) const { return (k % 5) == color && c == var && i == node; }
};
__device__ __forceinline__ Probe probe_of(int pidx, int N) {
  Probe p;
  p.color = pidx / (3 * N);
  p.var = (pidx / N) % 3;
  p.node = pidx % N;
  return p;
}

// nodal u of element k (value from u, tangent from v or the probe) in the working type
template <int N, int NC, bool PROBE, typename S, typename R>
__device__ __forceinline__ void load_u(const double* __restrict__ u, const double* __restrict__ v, int k, int E,
                                       long long col, long long nc, const Probe& pr, S out[3][N]) {
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const long long idx = (((long long)c * E + k) * N + i) * nc + col;
      if constexpr (NC == 1) {
        out[c][i] = (R)u[idx];
      } else if constexpr (PROBE) {
        out[c][i] = S{(R)u[idx], pr.hit(k, c, i) ? R(1) : R(0)};
      } else {
        out[c][i] = S{(R)u[idx], (R)v[idx]};
      }
    }
}

// one end node (i = 0: left, N - 1: right) of element k
template <int N, int NC, bool PROBE, typename S, typename R>
__device__ __forceinline__ void load_end(const double* __restrict__ u, const double* __restrict__ v, int k, int i,
                                         int E, long long col, long long nc, const Probe& pr, S out[3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const long long idx = (((long long)c * E + k) * N + i) * nc + col;
    if constexpr (NC == 1) out[c] = (R)u[idx];
    else if constexpr (PROBE) out[c] = S{(R)u[idx], pr.hit(k, c, i) ? R(1) : R(0)};
    else out[c] = S{(R)u[idx], (R)v[idx]};
  }
}

template <int N, int NC, bool PROBE, typename R>
__global__ void k_rgrad(int E, long long nc, ROps<R> O, RPhys<R> P, RGeo<R> g, const double* __restrict__ u,
                        const double* __restrict__ v, R* __restrict__ qg) {
  using S = typename std::conditional<NC == 2, DualT<R>, R>::type;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)E * nc) return;
  const int k = (int)(idx / nc);
  const long long col = idx % nc;
  const Probe pr = PROBE ? probe_of(blockIdx.y, N) : Probe{0, 0, 0};
  S un[3][N];
  load_u<N, NC, PROBE, S, R>(u, v, k, E, col, nc, pr, un);
  S U[3][N];
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int gq = 0; gq < N; ++gq) {
      S a = s_zero<S>();
#pragma unroll
      for (int i = 0; i < N; ++i) a = a + O.B[gq * N + i] * un[c][i];
      U[c][gq] = a;
    }
  // traces u_hat at both ends (Eq. LDG2; boundary traces at the column's ends)
  S uhL[3], uhR[3];
  if (k > 0) {
    S nb[3];
    load_end<N, NC, PROBE, S, R>(u, v, k - 1, N - 1, E, col, nc, pr, nb);
#pragma unroll
    for (int c = 0; c < 3; ++c) uhL[c] = R(0.5) * (un[c][0] + nb[c]);
  } else {
    const S own[3] = {un[0][0], un[1][0], un[2][0]};
    if (P.bc_lo == DG_BC_WALL) wall1(P, own, uhL);
    else for (int c = 0; c < 3; ++c) uhL[c] = own[c];
  }
  if (k < E - 1) {
    S nb[3];
    load_end<N, NC, PROBE, S, R>(u, v, k + 1, 0, E, col, nc, pr, nb);
#pragma unroll
    for (int c = 0; c < 3; ++c) uhR[c] = R(0.5) * (un[c][N - 1] + nb[c]);
  } else {
    const S own[3] = {un[0][N - 1], un[1][N - 1], un[2][N - 1]};
    if (P.bc_hi == DG_BC_WALL) wall1(P, own, uhR);
    else for (int c = 0; c < 3; ++c) uhR[c] = own[c];
  }
  const R rL = g.rL[k], rR = g.rR[k];
  const R rL2 = rL * rL, rR2 = rR * rR;
  R G[N], W[N], T2[N], rg[N];
#pragma unroll
  for (int j = 0; j < N; ++j) {
    G[j] = g.G[k * N + j];
    W[j] = g.W[k * N + j];
    T2[j] = g.T2[k * N + j];
    rg[j] = g.rg[k * N + j];
  }
  const long long plane = PROBE ? 0 : 4LL * E * N * nc;             // tangent plane offset
  R* qt = qg;
  if constexpr (PROBE) qt = qg + (long long)(1 + blockIdx.y) * 4 * E * N * nc;   // probe planes after the value
  const int qmap[3] = {0, 1, 3};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
#pragma unroll
    for (int j = 0; j < N; ++j) {
      S acc = (rR2 * O.eR[j]) * uhR[c] - (rL2 * O.eL[j]) * uhL[c] - T2[j] * U[c][j];
#pragma unroll
      for (int gq = 0; gq < N; ++gq) acc = acc - (O.D[gq * N + j] * G[gq]) * U[c][gq];
      const S qv = acc * (R(1) / W[j]);
      const long long o = (((long long)qmap[c] * E + k) * N + j) * nc + col;
      if constexpr (PROBE) {
        if (blockIdx.y == 0) qg[o] = qv.v;
        qt[o] = qv.d;
      } else {
        stp(qg + o, plane, qv);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < N; ++j) {
    const S qv = U[1][j] * (R(1) / rg[j]);
    const long long o = ((2LL * E + k) * N + j) * nc + col;
    if constexpr (PROBE) {
      if (blockIdx.y == 0) qg[o] = qv.v;
      qt[o] = qv.d;
    } else {
      stp(qg + o, plane, qv);
    }
  }
}

// q (4 components) extrapolated to one end of element k from its Gauss values
template <int N, int NC, typename S, typename R>
__device__ __forceinline__ void q_end(const R* __restrict__ qv, const R* __restrict__ qt, const R* e, int k, int E,
                                      long long col, long long nc, S out[4]) {
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    S a = s_zero<S>();
#pragma unroll
    for (int j = 0; j < N; ++j) {
      const long long o = (((long long)c * E + k) * N + j) * nc + col;
      if constexpr (NC == 1) a = a + e[j] * qv[o];
      else a = a + e[j] * S{qv[o], qt[o]};
    }
    out[c] = a;
  }
}

template <int N, int NC, bool PROBE, typename R>
__global__ void k_rface(int E, long long nc, ROps<R> O, RPhys<R> P, RGeo<R> g, RPrm<R> prm,
                        const double* __restrict__ u, const double* __restrict__ v, const R* __restrict__ qg,
                        R* __restrict__ fh) {
  using S = typename std::conditional<NC == 2, DualT<R>, R>::type;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)(E + 1) * nc) return;
  const int f = (int)(idx / nc);
  const long long col = idx % nc;
  const Probe pr = PROBE ? probe_of(blockIdx.y, N) : Probe{0, 0, 0};
  const R alpha = prm.alpha(col);
  const R* qv = qg;
  const R* qt = PROBE ? qg + (long long)(1 + blockIdx.y) * 4 * E * N * nc : qg + 4LL * E * N * nc;
  S Fh[3];
  S ua[3], ub[3], qa[4], qb[4];
  if (f > 0) {
    load_end<N, NC, PROBE, S, R>(u, v, f - 1, N - 1, E, col, nc, pr, ua);
    q_end<N, NC, S, R>(qv, qt, O.eR, f - 1, E, col, nc, qa);
  }
  if (f < E) {
    load_end<N, NC, PROBE, S, R>(u, v, f, 0, E, col, nc, pr, ub);
    q_end<N, NC, S, R>(qv, qt, O.eL, f, E, col, nc, qb);
  }
  if (f > 0 && f < E) {
    S Fa[3], Fb[3], uh[3], sg[3], t0, t1;
    flux1(P, ua, qa, alpha, true, Fa, t0);
    flux1(P, ub, qb, alpha, true, Fb, t1);
#pragma unroll
    for (int c = 0; c < 3; ++c) uh[c] = R(0.5) * (ua[c] + ub[c]);
    sigma1(P, uh, alpha, sg);
#pragma unroll
    for (int c = 0; c < 3; ++c) Fh[c] = R(0.5) * (Fa[c] + Fb[c]) + sg[c] * (R(0.5) * (ua[c] - ub[c]));
  } else {
    const bool bottom = f == 0;
    const S* uo = bottom ? ub : ua;
    const S* qo = bottom ? qb : qa;
    const int bc = bottom ? P.bc_lo : P.bc_hi;
    S t0;
    if (bc == DG_BC_WALL) {
      S ubd[3], F[3], sg[3];
      wall1(P, uo, ubd);
      flux1(P, ubd, qo, alpha, true, F, t0);
      sigma1(P, ubd, alpha, sg);
      // F_hat . n = F(u_b, q).n + sigma(u_b)(u - u_b) with n = -r_hat at the bottom, +r_hat at the top
#pragma unroll
      for (int c = 0; c < 3; ++c) Fh[c] = bottom ? F[c] - sg[c] * (uo[c] - ubd[c]) : F[c] + sg[c] * (uo[c] - ubd[c]);
    } else {
      flux1(P, uo, qo, alpha, false, Fh, t0);
    }
  }
  const R rf = (f < E) ? g.rL[f] : g.rR[E - 1];
  const R rf2 = rf * rf;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const long long o = ((long long)c * (E + 1) + f) * nc + col;
    const S val = rf2 * Fh[c];
    if constexpr (PROBE) {
      if (blockIdx.y == 0) fh[o] = val.v;
      fh[(long long)(1 + blockIdx.y) * 3 * (E + 1) * nc + o] = val.d;
    } else {
      stp(fh + o, 3LL * (E + 1) * nc, val);
    }
  }
}

// band storage of a column's n x n matrix (LAPACK gbtrf layout, leading dimension 2 kl + ku + 1):
// A[i][j] at row kl + ku + i - j of column j; entries [row][j][col] with the column index fastest
template <int N>
struct Band {
  static constexpr int KL = 9 * N - 1, KU = 9 * N - 1, LD = 2 * KL + KU + 1;
};

template <int N, int NC, bool PROBE, typename R>
__global__ void k_rvol(int E, long long nc, ROps<R> O, RPhys<R> P, RGeo<R> g, RPrm<R> prm, R t,
                       const double* __restrict__ u, const double* __restrict__ v, const R* __restrict__ qg,
                       const R* __restrict__ fh, double* __restrict__ r, double* __restrict__ jv, R stage_c,
                       float* __restrict__ band) {
  using S = typename std::conditional<NC == 2, DualT<R>, R>::type;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)E * nc) return;
  const int k = (int)(idx / nc);
  const long long col = idx % nc;
  const Probe pr = PROBE ? probe_of(blockIdx.y, N) : Probe{0, 0, 0};
  int kp = -1;   // PROBE: the perturbed element within reach of element k
  if constexpr (PROBE) {
    for (int d = -2; d <= 2; ++d)
      if (k + d >= 0 && k + d < E && ((k + d) % 5) == pr.color) kp = k + d;
    if (kp < 0) return;
  }
  const R alpha = prm.alpha(col), eps = prm.eps(col);
  const R site[3] = {prm.site(0, col), prm.site(1, col), prm.site(2, col)};
  const R* qv = qg;
  const R* qt = PROBE ? qg + (long long)(1 + blockIdx.y) * 4 * E * N * nc : qg + 4LL * E * N * nc;
  const R* fv = fh;
  const R* ft = PROBE ? fh + (long long)(1 + blockIdx.y) * 3 * (E + 1) * nc : fh + 3LL * (E + 1) * nc;
  S un[3][N];
  load_u<N, NC, PROBE, S, R>(u, v, k, E, col, nc, pr, un);
  S Rg[3][N];   // weak derivative accumulator per Gauss test function
  S Fw[3][N];   // G_g F_g
#pragma unroll
  for (int gq = 0; gq < N; ++gq) {
    S ug[3], qq[4];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      S a = s_zero<S>();
#pragma unroll
      for (int i = 0; i < N; ++i) a = a + O.B[gq * N + i] * un[c][i];
      ug[c] = a;
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const long long o = (((long long)c * E + k) * N + gq) * nc + col;
      if constexpr (NC == 1) qq[c] = qv[o];
      else qq[c] = S{qv[o], qt[o]};
    }
    const R rg = g.rg[k * N + gq];
    S F[3], src[3];
    source1<S, R>(P, ug, qq, rg, alpha, eps, site, t, F, src);
    const R Gg = g.G[k * N + gq], Wg = g.W[k * N + gq];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      Fw[c][gq] = Gg * F[c];
      Rg[c][gq] = Wg * src[c];
    }
  }
  S Fl[3], Fr[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const long long oL = ((long long)c * (E + 1) + k) * nc + col, oR = oL + nc;
    if constexpr (NC == 1) {
      Fl[c] = fv[oL];
      Fr[c] = fv[oR];
    } else {
      Fl[c] = S{fv[oL], ft[oL]};
      Fr[c] = S{fv[oR], ft[oR]};
    }
  }
  S Rn[3][N];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    S Rj[N];
#pragma unroll
    for (int j = 0; j < N; ++j) {
      S a = Rg[c][j] - O.eR[j] * Fr[c] + O.eL[j] * Fl[c];
#pragma unroll
      for (int gq = 0; gq < N; ++gq) a = a + O.D[gq * N + j] * Fw[c][gq];
      Rj[j] = a;
    }
#pragma unroll
    for (int i = 0; i < N; ++i) {
      S a = s_zero<S>();
#pragma unroll
      for (int j = 0; j < N; ++j) a = a + O.B[j * N + i] * Rj[j];
      Rn[c][i] = a;
    }
  }
  if constexpr (PROBE) {
    // column (kp, var, node) of J_G = M - stage_c J_r in the rows of element k
    constexpr int KL = Band<N>::KL, KU = Band<N>::KU;  // band offsets of the probe column
    const int n = 3 * N * E;
    const int jcol = kp * 3 * N + pr.var * N + pr.node;
    R Mcol[N];
#pragma unroll
    for (int i = 0; i < N; ++i) Mcol[i] = R(0);
    if (kp == k) {   // (B^T W B)[i][node]
#pragma unroll
      for (int i = 0; i < N; ++i) {
        R a = R(0);
#pragma unroll
        for (int gq = 0; gq < N; ++gq) a = a + O.B[gq * N + i] * g.W[k * N + gq] * O.B[gq * N + pr.node];
        Mcol[i] = a;
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const int row = k * 3 * N + c * N + i;
        const R val = ((kp == k && c == pr.var) ? Mcol[i] : R(0)) - stage_c * Rn[c][i].d;
        band[((long long)col * n + jcol) * Band<N>::LD + (KL + KU + row - jcol)] = (float)val;
      }
  } else {
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const long long o = (((long long)c * E + k) * N + i) * nc + col;
        if constexpr (NC == 1) {
          r[o] = (double)Rn[c][i];
        } else {
          if (r) r[o] = (double)Rn[c][i].v;
          jv[o] = (double)Rn[c][i].d;
        }
      }
  }
}

// ------------------------------------------------------------------------------------------------
// banded LU with partial pivoting (the unblocked LAPACK gbtf2 algorithm), one warp per column
// ------------------------------------------------------------------------------------------------
// Band storage per column (system) col, column-contiguous: entry (rb, j) of the LAPACK band at
// ab[(col n + j) LD + rb], i.e. matrix entry (j - KV + rb, j) with KV = KL + KU; ipiv[col n + j].
// The lanes take the rows j + i (i = lane + 32 r) of step j, so every load and store of a column is
// contiguous across the warp. The pivot column stays in registers from the search to the scaling;
// the columns to the right are updated in batches of RB_COLS, all of a batch's entries loaded
// before any is stored, and the row interchange of each column is a pair of shuffles. The
// arithmetic (pivot choice, scaling, x - l p per entry in the same order) is that of the
// one-thread-per-column algorithm.
constexpr int RB_COLS = 16;

template <int N>
__global__ void __launch_bounds__(128) k_rband_lu(int n, long long nc, float* __restrict__ ab, int* __restrict__ ipiv,
                                                  int* __restrict__ info) {
  constexpr int KL = Band<N>::KL, KU = Band<N>::KU, KV = KL + KU, LD = Band<N>::LD;
  constexpr int RP = (KL + 1 + 31) / 32;        // rows 0 .. KL of a step per lane
  const int lane = threadIdx.x & 31;
  const long long col = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (col >= nc) return;                        // whole warps
  float* A0 = ab + col * (long long)n * LD;
  int* pv = ipiv + col * (long long)n;
  int ju = 0;
  int bad = 0;
  for (int j = 0; j < n; ++j) {
    const int km = min(KL, n - 1 - j);
    float* Aj = A0 + (long long)j * LD + KV;     // Aj[i]: row j + i of column j
    float v[RP];
    float best = -1.0f;
    int bi = 0;
    bool nan = false;
#pragma unroll
    for (int r = 0; r < RP; ++r) {
      const int i = lane + 32 * r;
      v[r] = i <= km ? Aj[i] : 0.0f;
      const float a = fabsf(v[r]);
      nan |= i <= km && a != a;
      if (i <= km && a > best) {
        best = a;
        bi = i;
      }
    }
    for (int off = 16; off > 0; off >>= 1) {
      const float o = __shfl_xor_sync(0xffffffffu, best, off);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
      if (o > best || (o == best && oi < bi)) {
        best = o;
        bi = oi;
      }
    }
    nan = __any_sync(0xffffffffu, nan);
    const int jp = bi, jl = jp & 31, jr = jp >> 5;
    if (lane == 0) pv[j] = j + jp;
    if (nan || best == 0.0f || !isfinite(best)) {
      bad = 1;
      continue;
    }
    ju = max(ju, min(j + KU + jp, n - 1));
    // column j: rows 0 and jp interchanged, the pivot kept, the rest scaled by its reciprocal
    const float v0 = __shfl_sync(0xffffffffu, v[0], 0);
    float vp = 0.0f;
#pragma unroll
    for (int r = 0; r < RP; ++r) {
      const float t = __shfl_sync(0xffffffffu, v[r], jl);
      if (jr == r) vp = t;
    }
    const float inv = 1.0f / vp;
    float l[RP];
#pragma unroll
    for (int r = 0; r < RP; ++r) {
      const int i = lane + 32 * r;
      const float x = i == jp ? v0 : (i == 0 ? vp : v[r]);
      l[r] = i == 0 ? 0.0f : x * inv;
      if (i <= km) Aj[i] = i == 0 ? x : l[r];
    }
    // columns j + 1 .. ju
    for (int c0 = j + 1; c0 <= ju; c0 += RB_COLS) {
      float x[RB_COLS][RP];
#pragma unroll
      for (int q = 0; q < RB_COLS; ++q) {
        const int c = c0 + q;
        const float* Ac = A0 + (long long)c * LD + KV - (c - j);   // Ac[i]: row j + i of column c
#pragma unroll
        for (int r = 0; r < RP; ++r) {
          const int i = lane + 32 * r;
          x[q][r] = (c <= ju && i <= km) ? Ac[i] : 0.0f;
        }
      }
#pragma unroll
      for (int q = 0; q < RB_COLS; ++q) {
        const int c = c0 + q;
        if (c > ju) break;
        float xp = 0.0f;
#pragma unroll
        for (int r = 0; r < RP; ++r) {
          const float t = __shfl_sync(0xffffffffu, x[q][r], jl);
          if (jr == r) xp = t;
        }
        const float x0 = __shfl_sync(0xffffffffu, x[q][0], 0);
        // rows 0 and jp interchanged: the new row 0 (the multiplier's partner p) is the old row jp
#pragma unroll
        for (int r = 0; r < RP; ++r) {
          const int i = lane + 32 * r;
          if (i == 0) x[q][r] = xp;
          else if (i == jp) x[q][r] = x0;
        }
        const float pc = xp;
        if (pc != 0.0f) {
#pragma unroll
          for (int r = 0; r < RP; ++r) {
            const int i = lane + 32 * r;
            if (i >= 1) x[q][r] = x[q][r] - l[r] * pc;
          }
        }
      }
#pragma unroll
      for (int q = 0; q < RB_COLS; ++q) {
        const int c = c0 + q;
        float* Ac = A0 + (long long)c * LD + KV - (c - j);
#pragma unroll
        for (int r = 0; r < RP; ++r) {
          const int i = lane + 32 * r;
          if (c <= ju && i <= km) Ac[i] = x[q][r];
        }
      }
    }
    __syncwarp();
  }
  if (bad && lane == 0) atomicOr(info, 1);
}

// solve L U x = b in place on b (FP64 [n][nc] rows of the element-major ordering), FP32 products
// accumulated in float-float pairs (hi + lo, about 48 bits: the accuracy of the former FP64
// accumulation without the FP64 pipe, which issues 2 lanes per SM per cycle on this GPU); one warp
// per column with the column's b in shared memory ([warps][n] pairs). The band is read in blocks of
// SB_STEPS steps, the next block's loads issued before the current block is applied.
constexpr int SB_STEPS = 8;

// (hi, lo) -= p: Knuth's two-sum of hi and -p, the low parts added, then renormalised
__device__ __forceinline__ void ff_sub(float& hi, float& lo, float p) {
  const float s = hi - p;
  const float bb = s - hi;
  const float e = (hi - (s - bb)) + (-p - bb);
  const float t = e + lo;
  hi = s + t;
  lo = t - (hi - s);
}

template <int N>
__global__ void __launch_bounds__(128) k_rband_solve(int n, long long nc, const float* __restrict__ ab,
                                                     const int* __restrict__ ipiv, double* __restrict__ b) {
  constexpr int KL = Band<N>::KL, KU = Band<N>::KU, KV = KL + KU, LD = Band<N>::LD;
  constexpr int RPT = (KL + 31) / 32, RPB = (KV + 31) / 32;
  extern __shared__ float2 sb_all[];
  const int lane = threadIdx.x & 31;
  const long long col = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (col >= nc) return;                        // whole warps; no block barrier below
  float2* sb = sb_all + (size_t)(threadIdx.x >> 5) * n;
  for (int i = lane; i < n; i += 32) {
    const double x = b[(long long)i * nc + col];
    const float hi = (float)x;
    sb[i] = make_float2(hi, (float)(x - (double)hi));
  }
  const float* A0 = ab + col * (long long)n * LD;
  const int* pv = ipiv + col * (long long)n;
  // forward: L y = P b
  float a[SB_STEPS][RPT], an[SB_STEPS][RPT];
  int lp[SB_STEPS], lpn[SB_STEPS];
  auto load_lower = [&](int j0, float (&dst)[SB_STEPS][RPT], int (&pd)[SB_STEPS]) {
#pragma unroll
    for (int s = 0; s < SB_STEPS; ++s) {
      const int j = j0 + s;
      const int km = j < n ? min(KL, n - 1 - j) : -1;
#pragma unroll
      for (int r = 0; r < RPT; ++r) {
        const int i = 1 + lane + 32 * r;
        dst[s][r] = i <= km ? A0[(long long)j * LD + KV + i] : 0.0f;
      }
      pd[s] = j < n ? pv[j] : j;
    }
  };
  load_lower(0, a, lp);
  __syncwarp();
  for (int j0 = 0; j0 < n; j0 += SB_STEPS) {
    if (j0 + SB_STEPS < n) load_lower(j0 + SB_STEPS, an, lpn);
#pragma unroll
    for (int s = 0; s < SB_STEPS; ++s) {
      const int j = j0 + s;
      if (j >= n) break;
      const int km = min(KL, n - 1 - j);
      const int l = lp[s];
      if (l != j) {
        if (lane == 0) {
          const float2 t = sb[l];
          sb[l] = sb[j];
          sb[j] = t;
        }
        __syncwarp();
      }
      const float bj = sb[j].x;
#pragma unroll
      for (int r = 0; r < RPT; ++r) {
        const int i = 1 + lane + 32 * r;
        if (i <= km) {
          float2 y = sb[j + i];
          ff_sub(y.x, y.y, __fmul_rn(a[s][r], bj));   // the rounded product, never fused
          sb[j + i] = y;
        }
      }
      __syncwarp();
    }
#pragma unroll
    for (int s = 0; s < SB_STEPS; ++s) {
      lp[s] = lpn[s];
#pragma unroll
      for (int r = 0; r < RPT; ++r) a[s][r] = an[s][r];
    }
  }
  // backward: U x = y, steps j = n - 1 .. 0 in blocks
  float u[SB_STEPS][RPB], un[SB_STEPS][RPB], d[SB_STEPS], dn[SB_STEPS];
  auto load_upper = [&](int j0, float (&dst)[SB_STEPS][RPB], float (&dd)[SB_STEPS]) {
#pragma unroll
    for (int s = 0; s < SB_STEPS; ++s) {
      const int j = j0 - s;
      const int lm = j >= 0 ? min(j, KV) : -1;
#pragma unroll
      for (int r = 0; r < RPB; ++r) {
        const int i = 1 + lane + 32 * r;
        dst[s][r] = i <= lm ? A0[(long long)j * LD + KV - i] : 0.0f;
      }
      dd[s] = j >= 0 ? A0[(long long)j * LD + KV] : 1.0f;
    }
  };
  load_upper(n - 1, u, d);
  for (int j0 = n - 1; j0 >= 0; j0 -= SB_STEPS) {
    if (j0 - SB_STEPS >= 0) load_upper(j0 - SB_STEPS, un, dn);
#pragma unroll
    for (int s = 0; s < SB_STEPS; ++s) {
      const int j = j0 - s;
      if (j < 0) break;
      const int lm = min(j, KV);
      const float bj = sb[j].x / d[s];
      __syncwarp();                              // every lane has read sb[j]
      if (lane == 0) sb[j] = make_float2(bj, 0.0f);
#pragma unroll
      for (int r = 0; r < RPB; ++r) {
        const int i = 1 + lane + 32 * r;
        if (i <= lm) {
          float2 y = sb[j - i];
          ff_sub(y.x, y.y, __fmul_rn(u[s][r], bj));
          sb[j - i] = y;
        }
      }
      __syncwarp();
    }
#pragma unroll
    for (int s = 0; s < SB_STEPS; ++s) {
      d[s] = dn[s];
#pragma unroll
      for (int r = 0; r < RPB; ++r) u[s][r] = un[s][r];
    }
  }
  for (int i = lane; i < n; i += 32) b[(long long)i * nc + col] = (double)sb[i].x + (double)sb[i].y;
}

// ------------------------------------------------------------------------------------------------
// vector kernels of the Newton iteration (element-major unknown order for the band: row
// k 3N + c N + i; the state layout is [c][k][i][col])
// ------------------------------------------------------------------------------------------------
// out = M x (element mass matrices B^T W B per variable); x, out [3][E][N][nc]
template <int N>
__global__ void k_rmass(int E, long long nc, ROps<double> O, RGeo<double> g, const double* __restrict__ x,
                        double* __restrict__ out) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)E * nc * 3) return;
  const long long col = idx % nc;
  const int k = (int)((idx / nc) % E);
  const int c = (int)(idx / (nc * E));
  double xn[N], xg[N];
#pragma unroll
  for (int i = 0; i < N; ++i) xn[i] = x[(((long long)c * E + k) * N + i) * nc + col];
#pragma unroll
  for (int gq = 0; gq < N; ++gq) {
    double a = 0.0;
#pragma unroll
    for (int i = 0; i < N; ++i) a += O.B[gq * N + i] * xn[i];
    xg[gq] = a * g.W[k * N + gq];
  }
#pragma unroll
  for (int i = 0; i < N; ++i) {
    double a = 0.0;
#pragma unroll
    for (int gq = 0; gq < N; ++gq) a += O.B[gq * N + i] * xg[gq];
    out[(((long long)c * E + k) * N + i) * nc + col] = a;
  }
}

// G = M U - known - c r (in the band's element-major row order, [n][nc]) and per-column norms
// ||G||^2, ||M U||^2 (one thread per column)
template <int N>
__global__ void k_rstage(int E, long long nc, ROps<double> O, RGeo<double> g, const double* __restrict__ U,
                         const double* __restrict__ known, const double* __restrict__ r, double c,
                         double* __restrict__ G, double* __restrict__ norms) {
  const long long col = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= nc) return;
  double g2 = 0.0, m2 = 0.0;
  for (int k = 0; k < E; ++k)
    for (int v = 0; v < 3; ++v) {
      double xg[N];
#pragma unroll
      for (int gq = 0; gq < N; ++gq) {
        double a = 0.0;
#pragma unroll
        for (int i = 0; i < N; ++i) a += O.B[gq * N + i] * U[(((long long)v * E + k) * N + i) * nc + col];
        xg[gq] = a * g.W[k * N + gq];
      }
#pragma unroll
      for (int i = 0; i < N; ++i) {
        double mu = 0.0;
#pragma unroll
        for (int gq = 0; gq < N; ++gq) mu += O.B[gq * N + i] * xg[gq];
        const long long o = (((long long)v * E + k) * N + i) * nc + col;
        const double gv = mu - known[o] - c * r[o];
        G[((long long)(k * 3 + v) * N + i) * nc + col] = gv;
        g2 += gv * gv;
        m2 += mu * mu;
      }
    }
  norms[col] = sqrt(g2);
  norms[nc + col] = sqrt(m2);
}

// U -= delta (delta in the band's row order)
template <int N>
__global__ void k_rupdate(int E, long long nc, double* __restrict__ U, const double* __restrict__ delta) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 3LL * E * N * nc) return;
  const long long col = idx % nc;
  const int i = (int)((idx / nc) % N);
  const int k = (int)((idx / (nc * N)) % E);
  const int v = (int)(idx / (nc * N * E));
  U[idx] -= delta[((long long)(k * 3 + v) * N + i) * nc + col];
}

// known = M u_n + dt sum_j a_ij r(U_j) pieces: out = a x + b y
__global__ void k_raxpby(long long n, double a, const double* __restrict__ x, double b, const double* __restrict__ y,
                         double* __restrict__ out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = a * x[i] + b * y[i];
}

// largest ratio ||G|| / max(g0, tiny) over columns, counting columns below their absolute floor as 0
__global__ void k_rmaxratio(long long nc, const double* __restrict__ norms, const double* __restrict__ g0,
                            double* __restrict__ out) {
  __shared__ double red[256];
  double m = 0.0;
  for (long long c = threadIdx.x; c < nc; c += blockDim.x) {
    const double gn = norms[c], mu = norms[nc + c];
    double q = (gn <= 1e-14 * mu) ? 0.0 : gn / g0[c];
    if (!(q == q) || isinf(q)) q = INFINITY;
    m = fmax(m, q);
  }
  red[threadIdx.x] = m;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = red[0];
}

}  // namespace rad
}  // namespace dg

// --------------------------------------------------------------------------------------------------
// host side
// --------------------------------------------------------------------------------------------------
using namespace dg;
using namespace dg::rad;

enum { RK_GRAD = 0, RK_FACE, RK_VOL, RK_PROBE, RK_LU, RK_SOLVE, RK_VEC, RK_COUNT };
static const char* kRadialKernelNames[RK_COUNT] = {"k_rgrad", "k_rface", "k_rvol", "k_rprobe (grad+face+vol)",
                                                   "k_rband_lu", "k_rband_solve", "k_rvector"};

struct dg_radial {
  dg_radial_desc desc;
  int N, E, n;               // points per element, elements, unknowns per column (3 N E)
  long long nc;
  int device;
  ROps<double> ops64;
  ROps<float> ops32;
  RPhys<double> ph64;
  RPhys<float> ph32;
  double* geo64 = nullptr;   // rL [E], rR [E], rg, W, G, T2 [E][N]
  float* geo32 = nullptr;
  double* prm64 = nullptr;   // [5][nc]
  float* prm32 = nullptr;
  double* qg = nullptr;      // [2][4][E][N][nc]
  double* fh = nullptr;      // [2][3][E+1][nc]
  // implicit step
  float* qp = nullptr;       // [1 + probes][4][E][N][nc]
  float* fp = nullptr;       // [1 + probes][3][E+1][nc]
  float* band = nullptr;     // [nc][n][LD]: LAPACK band storage of each column's stage Jacobian
  int* ipiv = nullptr;       // [nc][n]
  int* info = nullptr;
  double *U0 = nullptr, *known = nullptr, *R1 = nullptr, *R2 = nullptr, *rr = nullptr, *G = nullptr;
  double *norms = nullptr, *g0 = nullptr, *ratio = nullptr, *ratio_h = nullptr;
  Prof prof;
};

namespace {

template <typename R>
RGeo<R> geo_view(const R* base, int E, int N) {
  RGeo<R> g;
  g.rL = base;
  g.rR = base + E;
  g.rg = base + 2 * E;
  g.W = g.rg + E * N;
  g.G = g.W + E * N;
  g.T2 = g.G + E * N;
  return g;
}

void rprof_begin(dg_radial* m, cudaStream_t s, int kind) {
  Prof& p = m->prof;
  if (!p.on) return;
  if (p.used < p.cap) {
    cudaEventRecord(p.ev[2 * p.used], s);
    p.kind[p.used] = kind;
  }
}
void rprof_end(dg_radial* m, cudaStream_t s) {
  Prof& p = m->prof;
  if (!p.on) return;
  if (p.used < p.cap) {
    cudaEventRecord(p.ev[2 * p.used + 1], s);
    p.used++;
  }
  p.launches++;
}

template <typename T>
int ralloc(T** p, long long count) {
  if (cudaMalloc((void**)p, sizeof(T) * (size_t)std::max(1LL, count)) != cudaSuccess) {
    cudaGetLastError();
    return fail(DG_ENOMEM, "dg_radial: cudaMalloc failed");
  }
  return DG_OK;
}

constexpr int kThreads = 128;
inline unsigned blocks_for(long long work) { return (unsigned)((work + kThreads - 1) / kThreads); }

// residual (and tangent) of every column in FP64
template <int N>
int residual_t(dg_radial* m, const double* u, const double* v, double t, double* r, double* jv, cudaStream_t s) {
  const int E = m->E;
  const long long nc = m->nc;
  const RGeo<double> g = geo_view<double>(m->geo64, E, N);
  const RPrm<double> prm{m->prm64, nc};
  const bool tan = v != nullptr;
  rprof_begin(m, s, RK_GRAD);
  if (tan) k_rgrad<N, 2, false, double><<<blocks_for((long long)E * nc), kThreads, 0, s>>>(E, nc, m->ops64, m->ph64, g, u, v, m->qg);
  else k_rgrad<N, 1, false, double><<<blocks_for((long long)E * nc), kThreads, 0, s>>>(E, nc, m->ops64, m->ph64, g, u, v, m->qg);
  rprof_end(m, s);
  DG_LAUNCH_CHECK("k_rgrad");
  rprof_begin(m, s, RK_FACE);
  if (tan) k_rface<N, 2, false, double><<<blocks_for((long long)(E + 1) * nc), kThreads, 0, s>>>(E, nc, m->ops64, m->ph64, g, prm, u, v, m->qg, m->fh);
  else k_rface<N, 1, false, double><<<blocks_for((long long)(E + 1) * nc), kThreads, 0, s>>>(E, nc, m->ops64, m->ph64, g, prm, u, v, m->qg, m->fh);
  rprof_end(m, s);
  DG_LAUNCH_CHECK("k_rface");
  rprof_begin(m, s, RK_VOL);
  if (tan)
    k_rvol<N, 2, false, double><<<blocks_for((long long)E * nc), kThreads, 0, s>>>(E, nc, m->ops64, m->ph64, g, prm, t, u, v, m->qg, m->fh, r, jv, 0.0, nullptr);
  else
    k_rvol<N, 1, false, double><<<blocks_for((long long)E * nc), kThreads, 0, s>>>(E, nc, m->ops64, m->ph64, g, prm, t, u, v, m->qg, m->fh, r, nullptr, 0.0, nullptr);
  rprof_end(m, s);
  DG_LAUNCH_CHECK("k_rvol");
  return DG_OK;
}

int residual_any(dg_radial* m, const double* u, const double* v, double t, double* r, double* jv, cudaStream_t s) {
  switch (m->N) {
    case 2: return residual_t<2>(m, u, v, t, r, jv, s);
    case 3: return residual_t<3>(m, u, v, t, r, jv, s);
    case 4: return residual_t<4>(m, u, v, t, r, jv, s);
    case 5: return residual_t<5>(m, u, v, t, r, jv, s);
    default: return fail(DG_EINVAL, "dg_radial: unsupported degree");
  }
}

// FP32 stage Jacobian J_G = M - c J_r(U) of every column by colored probing, then its banded LU
template <int N>
int jacobian_lu(dg_radial* m, const double* U, double t, double c, cudaStream_t s) {
  const int E = m->E, n = m->n;
  const long long nc = m->nc;
  constexpr int LD = Band<N>::LD;
  const int probes = 5 * 3 * N;
  const RGeo<float> g = geo_view<float>(m->geo32, E, N);
  const RPrm<float> prm{m->prm32, nc};
  DG_CUDA_TRY(cudaMemsetAsync(m->band, 0, sizeof(float) * (size_t)LD * n * nc, s));
  rprof_begin(m, s, RK_PROBE);
  dim3 gv(blocks_for((long long)E * nc), probes), gf(blocks_for((long long)(E + 1) * nc), probes);
  k_rgrad<N, 2, true, float><<<gv, kThreads, 0, s>>>(E, nc, m->ops32, m->ph32, g, U, nullptr, m->qp);
  k_rface<N, 2, true, float><<<gf, kThreads, 0, s>>>(E, nc, m->ops32, m->ph32, g, prm, U, nullptr, m->qp, m->fp);
  k_rvol<N, 2, true, float><<<gv, kThreads, 0, s>>>(E, nc, m->ops32, m->ph32, g, prm, (float)t, U, nullptr, m->qp, m->fp,
                                                   nullptr, nullptr, (float)c, m->band);
  rprof_end(m, s);
  DG_LAUNCH_CHECK("k_rprobe");
  DG_CUDA_TRY(cudaMemsetAsync(m->info, 0, sizeof(int), s));
  rprof_begin(m, s, RK_LU);
  k_rband_lu<N><<<blocks_for(32 * nc), kThreads, 0, s>>>(n, nc, m->band, m->ipiv, m->info);
  rprof_end(m, s);
  DG_LAUNCH_CHECK("k_rband_lu");
  return DG_OK;
}

template <int N>
int solve_t(dg_radial* m, double* b, cudaStream_t s) {
  rprof_begin(m, s, RK_SOLVE);
  const size_t smem = sizeof(float2) * (size_t)(kThreads / 32) * m->n;
  DG_CUDA_TRY(cudaFuncSetAttribute(k_rband_solve<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_rband_solve<N><<<blocks_for(32 * m->nc), kThreads, smem, s>>>(m->n, m->nc, m->band, m->ipiv, b);
  rprof_end(m, s);
  DG_LAUNCH_CHECK("k_rband_solve");
  return DG_OK;
}

template <int N>
int stage_norms(dg_radial* m, const double* U, const double* known, const double* r, double c, cudaStream_t s) {
  const RGeo<double> g = geo_view<double>(m->geo64, m->E, N);
  rprof_begin(m, s, RK_VEC);
  k_rstage<N><<<blocks_for(m->nc), kThreads, 0, s>>>(m->E, m->nc, m->ops64, g, U, known, r, c, m->G, m->norms);
  rprof_end(m, s);
  DG_LAUNCH_CHECK("k_rstage");
  return DG_OK;
}

template <int N>
int mass_t(dg_radial* m, const double* x, double* out, cudaStream_t s) {
  const RGeo<double> g = geo_view<double>(m->geo64, m->E, N);
  rprof_begin(m, s, RK_VEC);
  k_rmass<N><<<blocks_for(3LL * m->E * m->nc), kThreads, 0, s>>>(m->E, m->nc, m->ops64, g, x, out);
  rprof_end(m, s);
  DG_LAUNCH_CHECK("k_rmass");
  return DG_OK;
}

template <int N>
int update_t(dg_radial* m, double* U, cudaStream_t s) {
  rprof_begin(m, s, RK_VEC);
  k_rupdate<N><<<blocks_for(3LL * m->E * N * m->nc), kThreads, 0, s>>>(m->E, m->nc, U, m->G);
  rprof_end(m, s);
  DG_LAUNCH_CHECK("k_rupdate");
  return DG_OK;
}

int axpby(dg_radial* m, double a, const double* x, double b, const double* y, double* out, cudaStream_t s) {
  const long long n = (long long)m->n * m->nc;
  rprof_begin(m, s, RK_VEC);
  k_raxpby<<<blocks_for(n), kThreads, 0, s>>>(n, a, x, b, y, out);
  rprof_end(m, s);
  DG_LAUNCH_CHECK("k_raxpby");
  return DG_OK;
}

// max over columns of ||G|| / ||G0|| (0 for columns under the absolute floor), read by the host
int max_ratio(dg_radial* m, cudaStream_t s, double* out) {
  k_rmaxratio<<<1, 256, 0, s>>>(m->nc, m->norms, m->g0, m->ratio);
  DG_LAUNCH_CHECK("k_rmaxratio");
  DG_CUDA_TRY(cudaMemcpyAsync(m->ratio_h, m->ratio, sizeof(double), cudaMemcpyDeviceToHost, s));
  DG_CUDA_TRY(cudaStreamSynchronize(s));
  *out = m->ratio_h[0];
  return DG_OK;
}

template <int N>
int step_t(dg_radial* m, double* u, double t, double dt, int stages, double rtol, int max_newton,
           dg_radial_stats* st, cudaStream_t s) {
  double A[9], cc[3];
  int rc = dg_dirk_tableau(stages, A, cc);
  if (rc) return rc;
  const long long nd = (long long)m->n * m->nc;
  const size_t bytes = sizeof(double) * (size_t)nd;
  // U0 keeps u_n (restored on failure); known = M u_n + dt sum_{j<i} a_ij r(U_j)
  DG_CUDA_TRY(cudaMemcpyAsync(m->U0, u, bytes, cudaMemcpyDeviceToDevice, s));
  double* Rs[2] = {m->R1, m->R2};
  double last_ratio = 0.0;
  for (int i = 0; i < stages; ++i) {
    const double ti = t + cc[i] * dt, c = dt * A[i * stages + i];
    rc = mass_t<N>(m, m->U0, m->known, s);
    for (int j = 0; j < i && rc == DG_OK; ++j) rc = axpby(m, 1.0, m->known, dt * A[i * stages + j], Rs[j], m->known, s);
    if (rc) break;
    int it = 0;
    bool have_lu = false;
    for (;; ++it) {
      rc = residual_any(m, u, nullptr, ti, m->rr, nullptr, s);
      if (rc == DG_OK) rc = stage_norms<N>(m, u, m->known, m->rr, c, s);
      if (rc) break;
      if (it == 0) DG_CUDA_TRY(cudaMemcpyAsync(m->g0, m->norms, sizeof(double) * m->nc, cudaMemcpyDeviceToDevice, s));
      double ratio = 0.0;
      rc = max_ratio(m, s, &ratio);
      if (rc) break;
      if (!std::isfinite(ratio)) {
        rc = fail(DG_ENAN, "dg_radial_step: non-finite Newton residual");
        break;
      }
      last_ratio = ratio;
      if (ratio <= rtol) break;
      if (it >= max_newton) {
        rc = fail(DG_ENOTCONV, "dg_radial_step: Newton did not reach its tolerance (largest ratio " +
                                   std::to_string(ratio) + ")");
        break;
      }
      if (!have_lu) {   // the stage Jacobian at the stage's first iterate (FP32), factored once
        rc = jacobian_lu<N>(m, u, ti, c, s);
        if (rc) break;
        int info_h = 0;
        DG_CUDA_TRY(cudaMemcpyAsync(&info_h, m->info, sizeof(int), cudaMemcpyDeviceToHost, s));
        DG_CUDA_TRY(cudaStreamSynchronize(s));
        if (info_h) {
          rc = fail(DG_ENAN, "dg_radial_step: zero or non-finite pivot in a column's stage Jacobian");
          break;
        }
        have_lu = true;
      }
      rc = solve_t<N>(m, m->G, s);
      if (rc == DG_OK) rc = update_t<N>(m, u, s);
      if (rc) break;
    }
    if (st && i < 3) st->newton_iters[i] = it;
    if (rc) break;
    // r(U_i) for the next stages
    if (i + 1 < stages) {
      DG_CUDA_TRY(cudaMemcpyAsync(Rs[i], m->rr, bytes, cudaMemcpyDeviceToDevice, s));
    }
  }
  if (st) st->max_ratio = last_ratio;
  if (rc) cudaMemcpyAsync(u, m->U0, bytes, cudaMemcpyDeviceToDevice, s);
  return rc;
}

void release(dg_radial* m) {
  if (!m) return;
  void* ptrs[] = {m->geo64, m->geo32, m->prm64, m->prm32, m->qg, m->fh, m->qp, m->fp, m->band, m->ipiv, m->info,
                  m->U0, m->known, m->R1, m->R2, m->rr, m->G, m->norms, m->g0, m->ratio};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (m->ratio_h) cudaFreeHost(m->ratio_h);
  if (m->prof.ev) {
    for (int i = 0; i < 2 * m->prof.cap; ++i) cudaEventDestroy(m->prof.ev[i]);
    delete[] m->prof.ev;
    delete[] m->prof.kind;
  }
  delete m;
}

template <typename R>
RPhys<R> phys_cast(const RPhys<double>& P) {
  RPhys<R> q;
  q.gamma = (R)P.gamma; q.c_mu = (R)P.c_mu; q.c_k = (R)P.c_k; q.c_d = (R)P.c_d; q.pc = (R)P.pc; q.cv = (R)P.cv;
  q.visc_exp = (R)P.visc_exp; q.lam = (R)P.lam; q.t_wall = (R)P.t_wall; q.g_r0 = (R)P.g_r0;
  q.euv = P.euv; q.bc_lo = P.bc_lo; q.bc_hi = P.bc_hi; q.n_euvac = P.n_euvac;
  for (int j = 0; j < 40; ++j) {
    q.B[j] = (R)P.B[j];
    q.phi[j] = (R)P.phi[j];
  }
  q.cc = (R)P.cc; q.sun_cd = (R)P.sun_cd; q.sun_sd = (R)P.sun_sd; q.omega_t = (R)P.omega_t; q.inv_m = (R)P.inv_m;
  return q;
}

}  // namespace

extern "C" int dg_radial_create(const dg_radial_desc* desc, const double* node_r, const double* params,
                                dg_radial** out) {
  if (!desc || !params || !out) return fail(DG_EINVAL, "dg_radial_create: null argument");
  const dg_radial_desc& d = *desc;
  if (d.p < 1 || d.p > 4) return fail(DG_EINVAL, "dg_radial_create: p must be in 1..4");
  if (d.n_elem < 1 || d.n_col < 1) return fail(DG_EINVAL, "dg_radial_create: sizes must be positive");
  if ((long long)d.n_elem * 3 * (d.p + 1) > 6000)
    return fail(DG_EINVAL, "dg_radial_create: at most 6000 unknowns per variable set of a column (3 (p+1) n_elem)");
  if (!(d.r_inner > 0 && d.r_outer > d.r_inner)) return fail(DG_EINVAL, "dg_radial_create: need r_outer > r_inner > 0");
  if ((d.bc_lo != DG_BC_WALL && d.bc_lo != DG_BC_OUTFLOW) || (d.bc_hi != DG_BC_WALL && d.bc_hi != DG_BC_OUTFLOW))
    return fail(DG_EINVAL, "dg_radial_create: boundaries must be wall or outflow");
  if (d.euv != 0 && d.euv != DG_EUV_EUVAC) return fail(DG_EINVAL, "dg_radial_create: heating must be 0 or DG_EUV_EUVAC");
  if (!(d.gamma > 1 && d.grashof > 0 && d.prandtl > 0 && d.mass > 0))
    return fail(DG_EINVAL, "dg_radial_create: physical numbers out of range");
  for (int c = 0; c < d.n_col; ++c)
    if (!(params[4 * c + 1] > 0)) return fail(DG_EINVAL, "dg_radial_create: alpha0 must be positive");
  dg_radial* m = new dg_radial();
  m->desc = d;
  m->N = d.p + 1;
  m->E = d.n_elem;
  m->n = 3 * m->N * m->E;
  m->nc = d.n_col;
  cudaGetDevice(&m->device);
  const int N = m->N, E = m->E;
  Ops o;
  build_ops(N, &o);
  for (int i = 0; i < N * N; ++i) {
    m->ops64.B[i] = o.B[i];
    m->ops64.D[i] = o.D[i];
    m->ops32.B[i] = (float)o.B[i];
    m->ops32.D[i] = (float)o.D[i];
  }
  for (int i = 0; i < N; ++i) {
    m->ops64.eL[i] = o.eL[i];
    m->ops64.eR[i] = o.eR[i];
    m->ops32.eL[i] = (float)o.eL[i];
    m->ops32.eR[i] = (float)o.eR[i];
  }
  RPhys<double>& P = m->ph64;
  P.gamma = d.gamma;
  P.c_mu = 1.0 / std::sqrt(d.gamma * d.grashof);
  P.c_k = std::sqrt(d.gamma / d.grashof) / d.prandtl;
  P.c_d = (d.gamma - 1.0) * std::sqrt(d.gamma / d.grashof);
  P.pc = 1.0 / (d.gamma * d.mass);
  P.cv = 1.0 / d.mass;
  P.visc_exp = d.visc_exp;
  P.lam = d.lambda0;
  P.t_wall = d.t_wall;
  P.g_r0 = d.g_r0;
  P.euv = d.euv;
  P.bc_lo = d.bc_lo;
  P.bc_hi = d.bc_hi;
  P.n_euvac = 0;
  P.omega_t = d.euv_omega_t;
  P.inv_m = 1.0 / d.mass;
  P.cc = P.sun_cd = P.sun_sd = 0.0;
  if (d.euv == DG_EUV_EUVAC) {
    // the shell's EUVAC coefficients with efficiency 1 (each column scales by its own epsilon)
    dg_mesh_desc md;
    std::memset(&md, 0, sizeof(md));
    md.gamma = d.gamma;
    md.mass = d.mass;
    md.g_r0 = d.g_r0;
    md.euv_day = d.euv_day;
    md.euv_f107 = d.euv_f107;
    md.euv_f107a = d.euv_f107a;
    md.euv_eff = 1.0;
    md.euv_dsun = d.euv_dsun;
    md.ref_T0 = d.ref_T0;
    md.ref_rho0 = d.ref_rho0;
    md.ref_m = d.ref_m;
    md.ref_g0 = d.ref_g0;
    Phys full;
    std::memset(&full, 0, sizeof(full));
    if (!euvac_coefficients(md, full)) {
      delete m;
      return fail(DG_EINVAL, "dg_radial_create: EUVAC heating needs positive reference values, g_r0 and Sun distance");
    }
    P.n_euvac = full.n_euvac;
    for (int j = 0; j < 40; ++j) {
      P.B[j] = full.euvac_B[j];
      P.phi[j] = full.euvac_phi[0][j];
    }
    P.cc = full.euvac_cc;
    P.sun_cd = full.sun_cd;
    P.sun_sd = full.sun_sd;
  }
  m->ph32 = phys_cast<float>(P);
  // geometry: node radii -> element ends, Gauss radii and weights
  std::vector<double> nr((size_t)E * N);
  if (node_r) {
    std::copy(node_r, node_r + (size_t)E * N, nr.begin());
  } else {
    std::vector<double> rl = radial_layers(d.r_inner, d.r_outer, E, d.h_first);
    for (int k = 0; k < E; ++k)
      for (int i = 0; i < N; ++i) nr[k * N + i] = rl[k] + 0.5 * (1.0 + o.xi[i]) * (rl[k + 1] - rl[k]);
  }
  std::vector<double> geo((size_t)2 * E + 4 * E * N);
  for (int k = 0; k < E; ++k) {
    const double rL = nr[k * N], rR = nr[k * N + N - 1], J = 0.5 * (rR - rL);
    if (!(J > 0)) {
      delete m;
      return fail(DG_EINVAL, "dg_radial_create: node radii must increase within each element");
    }
    geo[k] = rL;
    geo[E + k] = rR;
    for (int gq = 0; gq < N; ++gq) {
      double rg = 0.0;
      for (int i = 0; i < N; ++i) rg += o.B[gq * N + i] * nr[k * N + i];
      const double w = o.w[gq];
      geo[2 * E + k * N + gq] = rg;
      geo[2 * E + E * N + k * N + gq] = w * J * rg * rg;
      geo[2 * E + 2 * E * N + k * N + gq] = w * rg * rg;
      geo[2 * E + 3 * E * N + k * N + gq] = 2.0 * w * J * rg;
    }
  }
  std::vector<float> geo32(geo.begin(), geo.end());
  const long long nc = m->nc;
  std::vector<double> prm((size_t)5 * nc);
  for (long long c = 0; c < nc; ++c) {
    const double lat = params[4 * c + 2], lon = params[4 * c + 3];
    prm[c] = params[4 * c];
    prm[nc + c] = params[4 * c + 1];
    prm[2 * nc + c] = std::cos(lat) * std::cos(lon);
    prm[3 * nc + c] = std::cos(lat) * std::sin(lon);
    prm[4 * nc + c] = std::sin(lat);
  }
  std::vector<float> prm32(prm.begin(), prm.end());
  const long long nd = (long long)m->n * nc;
  const int probes = 5 * 3 * N;
  const int LD = 2 * (9 * N - 1) + (9 * N - 1) + 1;
  int rc = 0;
  rc |= ralloc(&m->geo64, (long long)geo.size());
  rc |= ralloc(&m->geo32, (long long)geo.size());
  rc |= ralloc(&m->prm64, 5 * nc);
  rc |= ralloc(&m->prm32, 5 * nc);
  rc |= ralloc(&m->qg, 2LL * 4 * E * N * nc);
  rc |= ralloc(&m->fh, 2LL * 3 * (E + 1) * nc);
  rc |= ralloc(&m->qp, (1LL + probes) * 4 * E * N * nc);
  rc |= ralloc(&m->fp, (1LL + probes) * 3 * (E + 1) * nc);
  rc |= ralloc(&m->band, (long long)LD * m->n * nc);
  rc |= ralloc(&m->ipiv, (long long)m->n * nc);
  rc |= ralloc(&m->info, 1);
  rc |= ralloc(&m->U0, nd);
  rc |= ralloc(&m->known, nd);
  rc |= ralloc(&m->R1, nd);
  rc |= ralloc(&m->R2, nd);
  rc |= ralloc(&m->rr, nd);
  rc |= ralloc(&m->G, nd);
  rc |= ralloc(&m->norms, 2 * nc);
  rc |= ralloc(&m->g0, 2 * nc);
  rc |= ralloc(&m->ratio, 1);
  if (rc == DG_OK && cudaMallocHost((void**)&m->ratio_h, sizeof(double)) != cudaSuccess) rc = DG_ENOMEM;
  if (rc) {
    release(m);
    return fail(DG_ENOMEM, "dg_radial_create: device allocation failed");
  }
  cudaError_t err = cudaMemcpy(m->geo64, geo.data(), sizeof(double) * geo.size(), cudaMemcpyHostToDevice);
  if (err == cudaSuccess) err = cudaMemcpy(m->geo32, geo32.data(), sizeof(float) * geo32.size(), cudaMemcpyHostToDevice);
  if (err == cudaSuccess) err = cudaMemcpy(m->prm64, prm.data(), sizeof(double) * prm.size(), cudaMemcpyHostToDevice);
  if (err == cudaSuccess) err = cudaMemcpy(m->prm32, prm32.data(), sizeof(float) * prm32.size(), cudaMemcpyHostToDevice);
  if (err != cudaSuccess) {
    release(m);
    return fail(DG_ECUDA, std::string("dg_radial_create upload: ") + cudaGetErrorString(err));
  }
  *out = m;
  return DG_OK;
}

extern "C" void dg_radial_destroy(dg_radial* rad) {
  if (!rad) return;
  cudaDeviceSynchronize();
  release(rad);
}

extern "C" int dg_radial_sizes(const dg_radial* rad, int64_t* n_col, int32_t* n_node, int64_t* n_dof) {
  if (!rad) return fail(DG_EINVAL, "dg_radial_sizes: null handle");
  if (n_col) *n_col = rad->nc;
  if (n_node) *n_node = rad->E * rad->N;
  if (n_dof) *n_dof = (int64_t)rad->n * rad->nc;
  return DG_OK;
}

extern "C" int dg_radial_residual(dg_radial* rad, const double* u, double t, double* r, void* stream) {
  dg::NvtxRange nvtx_range_("dg_radial_residual");
  if (!rad || !u || !r) return fail(DG_EINVAL, "dg_radial_residual: null argument");
  return residual_any(rad, u, nullptr, t, r, nullptr, (cudaStream_t)stream);
}

extern "C" int dg_radial_jvp(dg_radial* rad, const double* u, const double* v, double t, double* jv, double* r_out,
                             void* stream) {
  dg::NvtxRange nvtx_range_("dg_radial_jvp");
  if (!rad || !u || !v || !jv) return fail(DG_EINVAL, "dg_radial_jvp: null argument");
  return residual_any(rad, u, v, t, r_out, jv, (cudaStream_t)stream);
}

extern "C" int dg_radial_step(dg_radial* rad, double* u, double t, double dt, int32_t stages, double newton_rtol,
                              int32_t max_newton, dg_radial_stats* stats, void* stream) {
  dg::NvtxRange nvtx_range_("dg_radial_step");
  if (!rad || !u) return fail(DG_EINVAL, "dg_radial_step: null argument");
  if (stages < 1 || stages > 3 || !(dt > 0) || !(newton_rtol > 0) || max_newton < 1)
    return fail(DG_EINVAL, "dg_radial_step: need 1 <= stages <= 3, dt > 0, newton_rtol > 0, max_newton >= 1");
  const auto t0 = std::chrono::steady_clock::now();
  if (stats) std::memset(stats, 0, sizeof(*stats));
  cudaStream_t s = (cudaStream_t)stream;
  int rc;
  switch (rad->N) {
    case 2: rc = step_t<2>(rad, u, t, dt, stages, newton_rtol, max_newton, stats, s); break;
    case 3: rc = step_t<3>(rad, u, t, dt, stages, newton_rtol, max_newton, stats, s); break;
    case 4: rc = step_t<4>(rad, u, t, dt, stages, newton_rtol, max_newton, stats, s); break;
    case 5: rc = step_t<5>(rad, u, t, dt, stages, newton_rtol, max_newton, stats, s); break;
    default: rc = fail(DG_EINVAL, "dg_radial_step: unsupported degree");
  }
  cudaStreamSynchronize(s);
  if (stats) {
    stats->status = rc;
    stats->wall_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  return rc;
}

extern "C" int dg_radial_profile_start(dg_radial* rad, int32_t capacity) {
  if (!rad || capacity < 1) return fail(DG_EINVAL, "dg_radial_profile_start: bad argument");
  Prof& p = rad->prof;
  if (p.ev) {
    for (int i = 0; i < 2 * p.cap; ++i) cudaEventDestroy(p.ev[i]);
    delete[] p.ev;
    delete[] p.kind;
  }
  p.cap = capacity;
  p.ev = new cudaEvent_t[2 * capacity];
  p.kind = new int[capacity];
  for (int i = 0; i < 2 * capacity; ++i) DG_CUDA_TRY(cudaEventCreate(&p.ev[i]));
  p.used = 0;
  p.launches = 0;
  p.on = true;
  return DG_OK;
}

extern "C" int dg_radial_profile_stop(dg_radial* rad, int32_t n_kinds, double* ms, int32_t* count, int64_t* total) {
  if (!rad) return fail(DG_EINVAL, "dg_radial_profile_stop: null handle");
  Prof& p = rad->prof;
  DG_CUDA_TRY(cudaDeviceSynchronize());
  for (int k = 0; k < n_kinds; ++k) {
    if (ms) ms[k] = 0.0;
    if (count) count[k] = 0;
  }
  for (int i = 0; i < p.used; ++i) {
    float t = 0.0f;
    DG_CUDA_TRY(cudaEventElapsedTime(&t, p.ev[2 * i], p.ev[2 * i + 1]));
    const int k = p.kind[i];
    if (k < n_kinds) {
      if (ms) ms[k] += t;
      if (count) count[k] += 1;
    }
  }
  if (total) *total = p.launches;
  p.on = false;
  return DG_OK;
}

extern "C" const char* dg_radial_kernel_name(int32_t kind) {
  return (kind >= 0 && kind < RK_COUNT) ? kRadialKernelNames[kind] : "";
}
