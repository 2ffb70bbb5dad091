// FP64 element and face kernels of the LDG residual, its exact tangent and the mass matrix.
//
// Representation. A degree-p field on an element is held by its values at the (p+1)^3 Gauss
// points ("Gauss space"). The ABI's nodal GLL coefficients map to Gauss space by B x B x B, with
// B[q][a] = l^GLL_a(eta_q) invertible. In Gauss space the operators of Eq. DGformulation reduce
// to exact sum-factorised 1D passes:
//   derivative along xi_a ............ D (Lagrange derivative on the Gauss points)
//   value on face xi_a = -1 / +1 ...... eL / eR (Lagrange extrapolation to the end points)
//   test-function weak derivative .... D^T;  face lifting ... eL / eR outer products
// and the element mass matrix is M = B^T W B with W = diag(w_g |J_g|), so
//   Gradient (Eq. DGformulation a):  Q_{d,c} = W^{-1} [ -sum_a D_a^T (G_{a d} U_c)
//                                                       + sum_faces e_face (w n_d dS) U_hat_c ]
//   Residual (Eq. DGformulation b):  r = B^T [ sum_a D_a^T (sum_d G_{a d} F_{c d}) + W s_c
//                                              - sum_faces e_face (F_hat . w n dS)_c ]
// with G_{a d} = w_g |J| d xi_a / d x_d (cofactor of the Jacobian). Each identity is exact
// (p-degree polynomials, the same quadrature), so these kernels compute the same discrete
// operator as a dense nodal implementation, up to rounding.
//
// Kernels (one CTA handles EPB elements, one thread per Gauss point; faces one thread per point):
//   k_interp   nodal u (and tangent v) -> Gauss values U, face traces UF
//   k_grad     U, UF (own + neighbour) -> Q in Gauss space, face traces QF
//   k_faces    UF, QF of both sides -> F_hat . (w n dS) for both element faces (Eq. LDG2)
//   k_volume   U, Q, F_hat -> pointwise F, s; projection; lifting; B^T -> nodal r (and J v)
// The exact Jacobian-vector product carries forward-mode dual numbers through every step.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <string>
#include <type_traits>

#include "dg_internal.cuh"

namespace dg {

template <int N>
struct Shape {
  static constexpr int NP = N * N * N;
  static constexpr int NF = N * N;
};

// elements per CTA by kernel footprint
template <int N, int NC>
struct Epb {
  static constexpr int value = (N == 2) ? 16 : (N == 3) ? 8 : (N == 4) ? (NC == 1 ? 4 : 2) : (NC == 1 ? 2 : 1);
};

template <int N>
__device__ __forceinline__ int pt_stride(int dir) {
  return dir == 0 ? 1 : (dir == 1 ? N : N * N);
}

// Contraction modes of the basis operators (the FP32 path only): CM_NATIVE multiplies in the
// working precision; CM_BF16 / CM_FP16 round both operands to bfloat16 / binary16 and accumulate
// in FP32 (the products of two such values are exact in FP32, as in a tensor-core MMA);
// CM_BF16X3 / CM_FP16X3 split each operand into hi + lo parts and keep three of the four products
// (hi*hi + hi*lo + lo*hi).
enum { CM_NATIVE = 0, CM_BF16 = 1, CM_FP16 = 2, CM_BF16X3 = 3, CM_FP16X3 = 4 };

template <int CM> __device__ __forceinline__ float cm_round(float v);
template <> __device__ __forceinline__ float cm_round<CM_BF16>(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }
template <> __device__ __forceinline__ float cm_round<CM_FP16>(float v) { return __half2float(__float2half_rn(v)); }

template <int CM, typename R>
__device__ __forceinline__ R cm_fma(R a, R x, R acc) {
  if constexpr (CM == CM_NATIVE) {
    return fma(a, x, acc);
  } else {
    constexpr int B = (CM == CM_BF16 || CM == CM_BF16X3) ? CM_BF16 : CM_FP16;
    const float ah = cm_round<B>(a), xh = cm_round<B>(x);
    if constexpr (CM == CM_BF16 || CM == CM_FP16) {
      return fmaf(ah, xh, acc);
    } else {
      const float al = cm_round<B>(a - ah), xl = cm_round<B>(x - xh);
      return fmaf(ah, xh, fmaf(ah, xl, fmaf(al, xh, acc)));
    }
  }
}

// 1D pass along `dir` at point g: sum_k A[i][k] in[.. k ..] (T = false) or A[k][i] (T = true)
template <int N, bool T, typename R, int CM = CM_NATIVE>
__device__ __forceinline__ R line(const R* __restrict__ A, const R* __restrict__ in, int g, int dir) {
  const int st = pt_stride<N>(dir);
  const int i = (g / st) % N;
  const int base = g - i * st;
  R acc = R(0);
#pragma unroll
  for (int k = 0; k < N; ++k) acc = cm_fma<CM>(T ? A[k * N + i] : A[i * N + k], in[base + k * st], acc);
  return acc;
}

// the same pass accumulated into acc (NEG: subtracted), one FMA chain
template <int N, bool T, bool NEG, typename R, int CM = CM_NATIVE>
__device__ __forceinline__ R line_fma(const R* __restrict__ A, const R* __restrict__ in, int g, int dir, R acc) {
  const int st = pt_stride<N>(dir);
  const int i = (g / st) % N;
  const int base = g - i * st;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const R a = T ? A[k * N + i] : A[i * N + k];
    acc = cm_fma<CM>(NEG ? -a : a, in[base + k * st], acc);
  }
  return acc;
}

// Gauss point index of (face phi, face point f, index k along the face normal)
template <int N>
__device__ __forceinline__ int face_vol_point(int phi, int f, int k) {
  const int axis = phi >> 1;
  const int is = f % N, it = f / N;
  int i0, i1, i2;
  if (axis == 0) { i0 = k; i1 = is; i2 = it; }
  else if (axis == 1) { i0 = is; i1 = k; i2 = it; }
  else { i0 = is; i1 = it; i2 = k; }
  return i0 + N * (i1 + N * i2);
}

// face point of volume point g on a face of the given axis
template <int N>
__device__ __forceinline__ int vol_face_point(int g, int axis) {
  const int i0 = g % N, i1 = (g / N) % N, i2 = g / (N * N);
  if (axis == 0) return i1 + N * i2;
  if (axis == 1) return i0 + N * i2;
  return i0 + N * i1;
}

template <int N>
__device__ __forceinline__ int axis_index(int g, int axis) {
  return axis == 0 ? g % N : (axis == 1 ? (g / N) % N : g / (N * N));
}

template <typename R>
struct SmemOpsT {
  R B[MAXN * MAXN], D[MAXN * MAXN], Binv[MAXN * MAXN], eL[MAXN], eR[MAXN];
};
using SmemOps = SmemOpsT<double>;

// the 1D operators (built in FP64 on the host) rounded to the working precision
template <int N, typename R>
__device__ __forceinline__ void load_ops(const Ops* __restrict__ o, SmemOpsT<R>& s) {
  for (int i = threadIdx.x; i < N * N; i += blockDim.x) {
    s.B[i] = (R)o->B[i];
    s.D[i] = (R)o->D[i];
    s.Binv[i] = (R)o->Binv[i];
  }
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    s.eL[i] = (R)o->eL[i];
    s.eR[i] = (R)o->eR[i];
  }
}


// --------------------------------------------------------------------------------------------
// k_interp: nodal -> Gauss values and face traces. NC = 1 (u) or 2 (u and tangent v).
// --------------------------------------------------------------------------------------------
template <int N, int NC, typename R, int CM = CM_NATIVE>
__global__ void k_interp(const double* __restrict__ u, const double* __restrict__ v, long long E,
                         const Ops* __restrict__ ops, R* __restrict__ ug, R* __restrict__ uf) {
  constexpr int NP = Shape<N>::NP, NF = Shape<N>::NF, C = 5 * NC, EPB = Epb<N, NC>::value;
  __shared__ SmemOpsT<R> so;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* smem = reinterpret_cast<R*>(smem_raw);
  R* b0 = smem;                            // [EPB][C][NP]
  R* b1 = smem + EPB * C * NP;             // [EPB][C][NP]
  load_ops<N, R>(ops, so);
  const long long e0 = (long long)blockIdx.x * EPB;
  for (int idx = threadIdx.x; idx < EPB * 5 * NP; idx += blockDim.x) {
    const int el = idx / (5 * NP), rem = idx % (5 * NP);
    const long long e = e0 + el;
    if (e < E) {
      b0[(el * C) * NP + rem] = (R)u[e * 5 * NP + rem];
      if (NC == 2) b0[(el * C + 5) * NP + rem] = (R)v[e * 5 * NP + rem];
    }
  }
  __syncthreads();
  const int el = threadIdx.x / NP, g = threadIdx.x % NP;
  const bool active = el < EPB;
  R* in = b0;
  R* out = b1;
#pragma unroll
  for (int dir = 0; dir < 3; ++dir) {
    if (active)
      for (int c = 0; c < C; ++c) out[(el * C + c) * NP + g] = line<N, false, R, CM>(so.B, in + (el * C + c) * NP, g, dir);
    __syncthreads();
    R* t = in;
    in = out;
    out = t;
  }
  // `in` holds Gauss values
  const long long plane_g = E * 5 * NP;
  for (int idx = threadIdx.x; idx < EPB * 5 * NP; idx += blockDim.x) {
    const int l = idx / (5 * NP), rem = idx % (5 * NP);
    const long long e = e0 + l;
    if (e < E) {
      ug[e * 5 * NP + rem] = in[(l * C) * NP + rem];
      if (NC == 2) ug[plane_g + e * 5 * NP + rem] = in[(l * C + 5) * NP + rem];
    }
  }
  // face traces. FP32: one face point per iteration, its N volume points found once (less index
  // arithmetic); FP64: the flat loop over (face, c, point), which spreads the FP64 work evenly.
  const long long plane_f = E * 6 * 5 * NF;
  if constexpr (sizeof(R) == 4) {
    for (int idx = threadIdx.x; idx < EPB * 6 * NF; idx += blockDim.x) {
      const int l = idx / (6 * NF), phi = (idx / NF) % 6, f = idx % NF;
      const long long e = e0 + l;
      if (e >= E) continue;
      const R* ev = (phi & 1) ? so.eR : so.eL;
      int vp[N];
#pragma unroll
      for (int k = 0; k < N; ++k) vp[k] = face_vol_point<N>(phi, f, k);
      for (int pl = 0; pl < NC; ++pl)
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          const R* src = in + (l * C + 5 * pl + c) * NP;
          R acc = R(0);
#pragma unroll
          for (int k = 0; k < N; ++k) acc = cm_fma<CM>(ev[k], src[vp[k]], acc);
          uf[pl * plane_f + e * 30 * NF + (phi * 5 + c) * NF + f] = acc;
        }
    }
  } else {
    for (int idx = threadIdx.x; idx < EPB * 6 * 5 * NF; idx += blockDim.x) {
      const int l = idx / (30 * NF), rem = idx % (30 * NF);
      const int phi = rem / (5 * NF), c = (rem / NF) % 5, f = rem % NF;
      const long long e = e0 + l;
      if (e >= E) continue;
      const R* ev = (phi & 1) ? so.eR : so.eL;
      for (int pl = 0; pl < NC; ++pl) {
        const R* src = in + (l * C + 5 * pl + c) * NP;
        R acc = R(0);
#pragma unroll
        for (int k = 0; k < N; ++k) acc = cm_fma<CM>(ev[k], src[face_vol_point<N>(phi, f, k)], acc);
        uf[pl * plane_f + e * 30 * NF + rem] = acc;
      }
    }
  }
}

// --------------------------------------------------------------------------------------------
// k_grad: LDG gradient in Gauss space (Eq. DGformulation a) and its face traces
// --------------------------------------------------------------------------------------------
// BLK (block-diagonal tangent, NC = 2): the tangent keeps only the element's own perturbation
// (u_hat picks up half of the own trace on interior faces) and qx receives, per face, the trace of
// the gradient tangent this element would get from its neighbour's perturbation across that face:
// kappa(f) (w n dS)(f) u_dot_nb(f) / 2 with kappa(f) = sum_k e_face[k]^2 / (w |J|)(g(f, k)).
// TO (tangent only, NC = 1): the value plane of ug, uf, qg, qf already holds the state's values
// (computed once for all the Jv of one Krylov solve, or for all the probes of one block assembly);
// only the tangent plane is formed, with the same arithmetic as the tangent of NC = 2, so the
// result is identical. The wall trace of the tangent reads the value plane's varrho trace.
template <int N, int NC, bool BLK, typename R, int CM = CM_NATIVE, bool TO = false>
__global__ void k_grad(long long E, const Ops* __restrict__ ops, PhysT<R> P, const R* __restrict__ geo,
                       const R* __restrict__ fgeo, const int* __restrict__ nbr,
                       const int* __restrict__ nbr_fo, const R* __restrict__ ug,
                       const R* __restrict__ uf, R* __restrict__ qg, R* __restrict__ qf,
                       R* __restrict__ qx) {
  static_assert(!TO || NC == 1, "tangent-only gradient works on one plane");
  constexpr int NP = Shape<N>::NP, NF = Shape<N>::NF, C = 5 * NC, EPB = Epb<N, NC>::value;
  __shared__ SmemOpsT<R> so;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* smem = reinterpret_cast<R*>(smem_raw);
  R* sU = smem;                             // [EPB][C][NP]
  R* sUh = sU + EPB * C * NP;               // [EPB][6][C][NF]   U_hat
  R* sN = sUh + EPB * 6 * C * NF;           // [EPB][6][3][NF]   w n dS
  R* sY = sN + EPB * 6 * 3 * NF;            // [EPB][9][NP]
  R* sQ = sY + EPB * 9 * NP;                // [EPB][3][C][NP]
  R* sL = sQ + EPB * 3 * C * NP;            // [EPB][6][3][NF]: (w n_d dS) u_hat_c of the current c
  load_ops<N, R>(ops, so);
  const long long e0 = (long long)blockIdx.x * EPB;
  const long long plane_g = E * 5 * NP, plane_f = E * 30 * NF;
  const long long og = TO ? plane_g : 0, of = TO ? plane_f : 0;   // TO: read the tangent plane
  for (int idx = threadIdx.x; idx < EPB * 5 * NP; idx += blockDim.x) {
    const int l = idx / (5 * NP), rem = idx % (5 * NP);
    const long long e = e0 + l;
    if (e < E)
      for (int pl = 0; pl < NC; ++pl) sU[(l * C + 5 * pl) * NP + rem] = ug[og + pl * plane_g + e * 5 * NP + rem];
  }
  // traces: u_hat on every face point (Eq. LDG2), and the face geometry
  for (int idx = threadIdx.x; idx < EPB * 6 * NF; idx += blockDim.x) {
    const int l = idx / (6 * NF), phi = (idx / NF) % 6, f = idx % NF;
    const long long e = e0 + l;
    if (e >= E) continue;
    const long long fbase = e * 30 * NF + phi * 5 * NF + f;
    for (int d = 0; d < 3; ++d) sN[((l * 6 + phi) * 3 + d) * NF + f] = fgeo[((e * 6 + phi) * 4 + d) * NF + f];
    const int nb = nbr[e * 6 + phi];
    R own[10], oth[10];
    for (int pl = 0; pl < NC; ++pl)
      for (int c = 0; c < 5; ++c) own[5 * pl + c] = uf[of + pl * plane_f + fbase + c * NF];
    R* dst = sUh + ((l * 6 + phi) * C) * NF + f;
    if (nb >= 0) {
      const int fo = nbr_fo[e * 6 + phi];
      const int f2 = orient_map(fo >> 3, f % N, f / N, N);
      const long long nbase = (long long)nb * 30 * NF + (fo & 7) * 5 * NF + f2;
      for (int pl = 0; pl < NC; ++pl)
        for (int c = 0; c < 5; ++c) oth[5 * pl + c] = uf[of + pl * plane_f + nbase + c * NF];
      if constexpr (BLK) {
        constexpr int T0 = TO ? 0 : 5;   // where the tangent sits in own / oth / dst
        for (int c = 0; c < 5; ++c) {
          if constexpr (!TO) dst[c * NF] = R(0.5) * (own[c] + oth[c]);
          dst[(T0 + c) * NF] = R(0.5) * own[T0 + c];
        }
        const R* ev = (phi & 1) ? so.eR : so.eL;
        R kappa = R(0);
        for (int k = 0; k < N; ++k) kappa += ev[k] * ev[k] / geo[e * 10 * NP + 9 * NP + face_vol_point<N>(phi, f, k)];
        R* xo = qx + (e * 6 + phi) * 15 * NF + f;
        for (int d = 0; d < 3; ++d) {
          const R kn = R(0.5) * kappa * fgeo[((e * 6 + phi) * 4 + d) * NF + f];
          for (int c = 0; c < 5; ++c) xo[(d * 5 + c) * NF] = kn * oth[T0 + c];
        }
      } else {
        for (int c = 0; c < C; ++c) dst[c * NF] = R(0.5) * (own[c] + oth[c]);
      }
    } else if (nb == -DG_BC_WALL) {
      if constexpr (BLK) {
        R* xo = qx + (e * 6 + phi) * 15 * NF + f;
        for (int k = 0; k < 15; ++k) xo[k * NF] = R(0);
      }
      if constexpr (TO) {
        const R sr = s_exp(R(0.5) * uf[fbase]);   // value plane's varrho trace
        dst[0] = own[0];
        dst[NF] = R(0);
        dst[2 * NF] = R(0);
        dst[3 * NF] = R(0);
        dst[4 * NF] = R(0.5) * sr * P.t_wall * own[0];
        continue;
      }
      const R sr = s_exp(R(0.5) * own[0]);
      dst[0] = own[0];
      dst[NF] = R(0);
      dst[2 * NF] = R(0);
      dst[3 * NF] = R(0);
      dst[4 * NF] = sr * P.t_wall;
      if (NC == 2) {
        dst[5 * NF] = own[5];
        dst[6 * NF] = R(0);
        dst[7 * NF] = R(0);
        dst[8 * NF] = R(0);
        dst[9 * NF] = R(0.5) * sr * P.t_wall * own[5];
      }
    } else {
      if constexpr (BLK) {
        R* xo = qx + (e * 6 + phi) * 15 * NF + f;
        for (int k = 0; k < 15; ++k) xo[k * NF] = R(0);
      }
      for (int c = 0; c < C; ++c) dst[c * NF] = own[c];
    }
  }
  __syncthreads();
  const int el = threadIdx.x / NP, g = threadIdx.x % NP;
  const bool active = el < EPB && (e0 + el) < E;
  R G[9], invW = R(0);
  if (active) {
    const R* gp = geo + (e0 + el) * 10 * NP + g;
    for (int k = 0; k < 9; ++k) G[k] = gp[k * NP];
    invW = R(1) / gp[9 * NP];
  }
  for (int c = 0; c < C; ++c) {
    if (active) {
      const R uc = sU[(el * C + c) * NP + g];
      for (int k = 0; k < 9; ++k) sY[(el * 9 + k) * NP + g] = G[k] * uc;
    }
    // (w n_d dS) u_hat_c once per face point, shared by the N volume points behind it
    for (int idx = threadIdx.x; idx < EPB * 6 * NF; idx += blockDim.x) {
      const int l = idx / (6 * NF), phi = (idx / NF) % 6, f = idx % NF;
      if (e0 + l < E) {
        const R uh = sUh[((l * 6 + phi) * C + c) * NF + f];
        for (int d = 0; d < 3; ++d) sL[((l * 6 + phi) * 3 + d) * NF + f] = sN[((l * 6 + phi) * 3 + d) * NF + f] * uh;
      }
    }
    __syncthreads();
    if (active) {
      // q_d = (sum over the 6 faces of e_face[i_axis] (w n_d dS) u_hat_c - D^T (G u_c)) / (w |J|)
      for (int d = 0; d < 3; ++d) {
        R acc = R(0);
#pragma unroll
        for (int phi = 0; phi < 6; ++phi) {
          const int axis = phi >> 1;
          const R coef = ((phi & 1) ? so.eR : so.eL)[axis_index<N>(g, axis)];
          acc = cm_fma<CM>(coef, sL[((el * 6 + phi) * 3 + d) * NF + vol_face_point<N>(g, axis)], acc);
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) acc = line_fma<N, true, true, R, CM>(so.D, sY + (el * 9 + a * 3 + d) * NP, g, a, acc);
        sQ[((el * 3 + d) * C + c) * NP + g] = acc * invW;
      }
    }
    __syncthreads();
  }
  // write Q (Gauss space): each thread its own point, the 15 (d, c) entries unrolled. For FP32 the
  // face traces go one face point per iteration with its N volume points found once (the kernel is
  // bound by instruction issue, much of it index arithmetic); the FP64 kernel is bound by the FP64
  // pipe, and there the flat loop over (face, d, c, point) keeps every thread equally busy.
  if (active) {
    const long long e = e0 + el;
    for (int pl = 0; pl < NC; ++pl)
#pragma unroll
      for (int dc = 0; dc < 15; ++dc)
        qg[(TO ? E * 15 * NP : 0) + pl * E * 15 * NP + e * 15 * NP + dc * NP + g] =
            sQ[((el * 3 + dc / 5) * C + 5 * pl + dc % 5) * NP + g];
  }
  if constexpr (sizeof(R) == 4) {
    for (int idx = threadIdx.x; idx < EPB * 6 * NF; idx += blockDim.x) {
      const int l = idx / (6 * NF), phi = (idx / NF) % 6, f = idx % NF;
      const long long e = e0 + l;
      if (e >= E) continue;
      const R* ev = (phi & 1) ? so.eR : so.eL;
      int vp[N];
#pragma unroll
      for (int k = 0; k < N; ++k) vp[k] = face_vol_point<N>(phi, f, k);
      for (int pl = 0; pl < NC; ++pl)
#pragma unroll
        for (int dc = 0; dc < 15; ++dc) {
          const R* src = sQ + ((l * 3 + dc / 5) * C + 5 * pl + dc % 5) * NP;
          R acc = R(0);
#pragma unroll
          for (int k = 0; k < N; ++k) acc = cm_fma<CM>(ev[k], src[vp[k]], acc);
          qf[(TO ? E * 90 * NF : 0) + pl * E * 90 * NF + e * 90 * NF + (phi * 15 + dc) * NF + f] = acc;
        }
    }
  } else {
    for (int idx = threadIdx.x; idx < EPB * 6 * 15 * NF; idx += blockDim.x) {
      const int l = idx / (90 * NF), rem = idx % (90 * NF);
      const int phi = rem / (15 * NF), dc = (rem / NF) % 15, f = rem % NF;
      const int d = dc / 5, c = dc % 5;
      const long long e = e0 + l;
      if (e >= E) continue;
      const R* ev = (phi & 1) ? so.eR : so.eL;
      for (int pl = 0; pl < NC; ++pl) {
        const R* src = sQ + ((l * 3 + d) * C + 5 * pl + c) * NP;
        R acc = R(0);
#pragma unroll
        for (int k = 0; k < N; ++k) acc = cm_fma<CM>(ev[k], src[face_vol_point<N>(phi, f, k)], acc);
        qf[(TO ? E * 90 * NF : 0) + pl * E * 90 * NF + e * 90 * NF + rem] = acc;
      }
    }
  }
}

// --------------------------------------------------------------------------------------------
// k_faces: numerical flux of Eq. LDG2 on every face, written for both element faces
// --------------------------------------------------------------------------------------------
template <typename S, int NC, typename R>
__device__ __forceinline__ S ld(const R* p, long long plane) {
  if constexpr (NC == 1) return p[0];
  else return S{p[0], p[plane]};
}
template <typename R>
__device__ __forceinline__ void st(R* p, long long, R v) { p[0] = v; }
template <typename R>
__device__ __forceinline__ void st(R* p, long long plane, DualT<R> v) {
  p[0] = v.v;
  p[plane] = v.d;
}

// interior numerical flux of Eq. LDG2 with the normal n = w n dS of the first side:
// F_hat . n = (F(u, q) + F(u2, q2)) . n / 2 + sigma(u_hat) (u - u_hat) |n|, u_hat = (u + u2) / 2
template <typename S, typename R = typename RealOf<S>::type>
__device__ __forceinline__ void face_flux_interior(const PhysT<R>& P, const S u[5], const S q[3][5], const S u2[5],
                                                   const S q2[3][5], const R n[3], R area, S out[5],
                                                   const Mix<R>& mx) {
  S f1[5], fn[5], uh[5], sg[5];
  flux_dot_n(P, u, q, n, true, f1, mx);
  flux_dot_n(P, u2, q2, n, true, fn, mx);
#pragma unroll
  for (int c = 0; c < 5; ++c) uh[c] = R(0.5) * (u[c] + u2[c]);
  sigma_diag(P, uh, sg, mx);
#pragma unroll
  for (int c = 0; c < 5; ++c) out[c] = R(0.5) * (f1[c] + fn[c]) + sg[c] * ((R(0.5) * area) * (u[c] - u2[c]));
}

// BLK (NC = 2): interior faces evaluate the tangent twice, once for each side's diagonal block:
// the own side carries its perturbation and the other side only the gradient it receives from it
// across this face (qx of the other element).
template <int N, int NC, bool BLK, typename R>
__global__ void k_faces(long long E, long long F, PhysT<R> P, const int* __restrict__ face_e,
                        const int* __restrict__ face_f, const int* __restrict__ nbr,
                        const int* __restrict__ nbr_fo, const R* __restrict__ fgeo,
                        const R* __restrict__ uf, const R* __restrict__ qf,
                        const R* __restrict__ qx, R* __restrict__ fh, const R* __restrict__ mixf) {
  using S = typename std::conditional<NC == 2, DualT<R>, R>::type;
  constexpr int NF = Shape<N>::NF;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= F * NF) return;
  const long long fi = idx / NF;
  const int f = (int)(idx % NF);
  const long long e = face_e[fi];
  const int phi = face_f[fi];
  Mix<R> mx{P.cv, R(1)};
  if (P.comp) {   // mixture at this face point: [E][6][2][NF] = (c_v*, conductivity factor)
    mx.cv = mixf[((e * 6 + phi) * 2) * NF + f];
    mx.kfac = mixf[((e * 6 + phi) * 2 + 1) * NF + f];
  }
  const long long plane_u = E * 30 * NF, plane_q = E * 90 * NF;
  const R* gp = fgeo + ((e * 6 + phi) * 4) * NF + f;
  const R n[3] = {gp[0], gp[NF], gp[2 * NF]};
  const R area = gp[3 * NF];
  S u[5], q[3][5];
  const long long ub = e * 30 * NF + phi * 5 * NF + f;
  const long long qb = e * 90 * NF + phi * 15 * NF + f;
#pragma unroll
  for (int c = 0; c < 5; ++c) u[c] = ld<S, NC, R>(uf + ub + c * NF, plane_u);
#pragma unroll
  for (int d = 0; d < 3; ++d)
#pragma unroll
    for (int c = 0; c < 5; ++c) q[d][c] = ld<S, NC, R>(qf + qb + (d * 5 + c) * NF, plane_q);
  const int nb = nbr[e * 6 + phi];
  S out[5];
  if (nb >= 0) {
    const int fo = nbr_fo[e * 6 + phi];
    const int phi2 = fo & 7;
    const int f2 = orient_map(fo >> 3, f % N, f / N, N);
    S u2[5], q2[3][5];
    const long long ub2 = (long long)nb * 30 * NF + phi2 * 5 * NF + f2;
    const long long qb2 = (long long)nb * 90 * NF + phi2 * 15 * NF + f2;
#pragma unroll
    for (int c = 0; c < 5; ++c) u2[c] = ld<S, NC, R>(uf + ub2 + c * NF, plane_u);
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int c = 0; c < 5; ++c) q2[d][c] = ld<S, NC, R>(qf + qb2 + (d * 5 + c) * NF, plane_q);
    const long long ob2 = (long long)nb * 30 * NF + phi2 * 5 * NF + f2;
    if constexpr (BLK) {
      // block of the own element: the neighbour side carries only the cross gradient tangent
      S ua[5], qa[3][5];
#pragma unroll
      for (int c = 0; c < 5; ++c) ua[c] = S{u2[c].v, R(0)};
#pragma unroll
      for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int c = 0; c < 5; ++c) qa[d][c] = S{q2[d][c].v, qx[((long long)nb * 6 + phi2) * 15 * NF + (d * 5 + c) * NF + f2]};
      face_flux_interior(P, u, q, ua, qa, n, area, out, mx);
      // block of the neighbour: the own side carries only its cross gradient tangent
      S ub[5], qb[3][5], outb[5];
#pragma unroll
      for (int c = 0; c < 5; ++c) ub[c] = S{u[c].v, R(0)};
#pragma unroll
      for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int c = 0; c < 5; ++c) qb[d][c] = S{q[d][c].v, qx[(e * 6 + phi) * 15 * NF + (d * 5 + c) * NF + f]};
      face_flux_interior(P, ub, qb, u2, q2, n, area, outb, mx);
#pragma unroll
      for (int c = 0; c < 5; ++c) st(fh + ob2 + c * NF, plane_u, -outb[c]);
    } else {
      face_flux_interior(P, u, q, u2, q2, n, area, out, mx);
#pragma unroll
      for (int c = 0; c < 5; ++c) st(fh + ob2 + c * NF, plane_u, -out[c]);
    }
  } else if (nb == -DG_BC_WALL) {
    S ubd[5], sg[5];
    wall_trace(P, u, ubd);
    flux_dot_n(P, ubd, q, n, true, out, mx);
    sigma_diag(P, ubd, sg, mx);
#pragma unroll
    for (int c = 0; c < 5; ++c) out[c] = out[c] + sg[c] * (area * (u[c] - ubd[c]));
  } else {
    flux_dot_n(P, u, q, n, false, out, mx);
  }
#pragma unroll
  for (int c = 0; c < 5; ++c) st(fh + ub + c * NF, plane_u, out[c]);
}

// --------------------------------------------------------------------------------------------
// k_volume: pointwise flux and source, projection, lifting of F_hat, B^T -> nodal r (and J v)
// --------------------------------------------------------------------------------------------
template <typename S, typename R = typename RealOf<S>::type>
__device__ __forceinline__ void volume_point(const PhysT<R>& P, const S u[5], const S q[3][5],
                                             const R G[9], R Wd, const R acc[3],
                                             const R* xg, R t, S Fref[3][5], S src[5], const R mg[8]) {
  // mg (variable composition): c_v*, grad c_v* (3), conductivity factor, mass fractions of N2, O2, He
  const Mix<R> mx{P.comp ? mg[0] : P.cv, P.comp ? mg[4] : R(1)};
  const R cvp = mx.cv;
  const R pcoef = P.comp ? cvp * P.inv_gamma : P.p_coef;   // 1/(gamma m*)
  Prim<S> w;
  primitives(P, u, q, w, mx);
  const S cm = (P.c_mu * w.mu) * w.isr;
  const S ck = ((P.c_k / cvp) * w.kappa) * w.isr;
  // reference-space fluxes Fref[a][c] = sum_d G[a][d] F[c][d], formed from the contractions of the
  // cofactor rows with v, grad T and the strain rows (F[c][d] = u_c v_d + p delta - viscous terms)
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const R g0 = G[a * 3 + 0], g1 = G[a * 3 + 1], g2 = G[a * 3 + 2];
    const S Gv = g0 * w.v[0] + g1 * w.v[1] + g2 * w.v[2];
    const S GgT = g0 * w.gT[0] + g1 * w.gT[1] + g2 * w.gT[2];
    Fref[a][0] = u[0] * Gv;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      const S Ge = g0 * w.eps[m][0] + g1 * w.eps[m][1] + g2 * w.eps[m][2];
      Fref[a][1 + m] = u[1 + m] * Gv + (pcoef * G[a * 3 + m]) * u[4] - cm * Ge;
    }
    Fref[a][4] = u[4] * Gv - ck * GgT;
  }
  // source terms
  const S sr = s_inv(w.isr);
  const S wxv[3] = {P.omega[1] * w.v[2] - P.omega[2] * w.v[1], P.omega[2] * w.v[0] - P.omega[0] * w.v[2],
                    P.omega[0] * w.v[1] - P.omega[1] * w.v[0]};
  src[0] = (u[0] - R(1)) * w.div;
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    const S a_m = acc[m] - P.cor * wxv[m];
    const S eg = w.eps[m][0] * q[0][0] + w.eps[m][1] * q[1][0] + w.eps[m][2] * q[2][0];
    src[1 + m] = sr * a_m + R(0.5) * (w.div * u[1 + m]) - (R(0.5) * pcoef) * (u[4] * q[m][0]) + R(0.5) * (cm * eg);
  }
  const S tg = w.gT[0] * q[0][0] + w.gT[1] * q[1][0] + w.gT[2] * q[2][0];
  S diss = s_zero<S>();
#pragma unroll
  for (int m = 0; m < 3; ++m)
#pragma unroll
    for (int d = 0; d < 3; ++d) diss = diss + w.eps[m][d] * w.gv[m][d];
  S s4 = (R(1.5) - P.gamma) * (u[4] * w.div) + R(0.5) * (ck * tg) + ((P.c_d / cvp) * w.mu) * (w.isr * diss);
  if (P.comp) {
    // -(1/c_v) (sqrt(rho) T v - c_kappa kappa / (sqrt(rho) c_v) grad T) . grad c_v
    const S vg = w.v[0] * mg[1] + w.v[1] * mg[2] + w.v[2] * mg[3];
    const S tgc = w.gT[0] * mg[1] + w.gT[1] * mg[2] + w.gT[2] * mg[3];
    s4 = s4 - (u[4] * vg - ck * tgc) * (R(1) / cvp);
  }
  if (P.euv == DG_EUV_GAUSS) {
    const R r = sqrt(xg[0] * xg[0] + xg[1] * xg[1] + xg[2] * xg[2]);
    const R sx = cos(P.euv_omega_t * t), sy = -sin(P.euv_omega_t * t);
    R cchi = (xg[0] * sx + xg[1] * sy) / r;
    cchi = fmin(R(1), fmax(R(-1), cchi));
    const R chi = acos(cchi);
    const R dz = (r - P.euv_r_peak) * P.euv_inv_w;
    const R Qh = P.euv_amp * s_exp(-chi * chi * P.euv_inv2s2) * s_exp(R(-0.6931471805599453) * dz * dz);
    s4 = s4 + (Qh / cvp) * w.isr;
  } else if (P.euv == DG_EUV_EUVAC) {
    // EUVAC photoabsorption with Smith & Smith Chapman depths (Sec. 2.2)
    const R r = sqrt(xg[0] * xg[0] + xg[1] * xg[1] + xg[2] * xg[2]);
    const R wt = P.euv_omega_t * t;
    R cchi = (xg[0] * (-P.sun_cd * cos(wt)) + xg[1] * (P.sun_cd * sin(wt)) + xg[2] * P.sun_sd) / r;
    cchi = fmin(R(1), fmax(R(-1), cchi));
    const R schi = sqrt(fmax(R(0), R(1) - cchi * cchi));
    if (cchi > R(0) || schi * r > P.g_r0) {          // not in the Earth's shadow
      const S er = sr * sr;                             // e^varrho
      const R minv = P.comp ? cvp : P.inv_m;            // 1/m*
      const S Hs = w.T * (r * r * minv / (P.g_r0 * P.g_r0));   // H* = T* r*^2 / (m* g_r0^2)
      const S rt = r * s_inv(Hs);                       // r~ = |r| / H
      const S ex = s_erfcx(s_sqrt(R(0.5) * rt) * fabs(cchi));
      const S base = s_sqrt(R(1.5707963267948966) * rt);
      S ch;
      if (cchi > R(0)) ch = base * ex;
      else ch = base * (R(2) * s_exp(rt * (R(1) - schi)) - ex);
      // species weights w_s = chi_s / m_s* (O, N2, O2, He), or 1/m* on oxygen alone
      R ws[4] = {P.inv_m, R(0), R(0), R(0)};
      if (P.comp) {
        ws[0] = (R(1) - mg[5] - mg[6] - mg[7]);
        ws[1] = mg[5] * R(16.0 / 28.0);
        ws[2] = mg[6] * R(16.0 / 32.0);
        ws[3] = mg[7] * R(16.0 / 4.0);
      }
      const S k = (P.euvac_cc * er) * Hs * ch;          // tau_j = Phi_j k
      S qs = s_zero<S>();
#pragma unroll 1
      for (int j = 0; j < P.n_euvac; ++j) {
        const R Phi = ws[0] * P.euvac_phi[0][j] + ws[1] * P.euvac_phi[1][j] + ws[2] * P.euvac_phi[2][j] +
                      ws[3] * P.euvac_phi[3][j];
        qs = qs + (P.euvac_B[j] * Phi) * s_exp(-Phi * k);
      }
      s4 = s4 + (er * qs) * (R(1) / cvp) * w.isr;
    }
  }
  src[4] = s4;
#pragma unroll
  for (int c = 0; c < 5; ++c) src[c] = src[c] * Wd;
}

// L2 prefetch hint for n consecutive elements from p, one 128-byte line per thread and iteration
template <typename R>
__device__ __forceinline__ void prefetch_l2(const R* p, long long n) {
  const char* c = reinterpret_cast<const char*>(p);
  const long long bytes = n * (long long)sizeof(R);
  for (long long off = threadIdx.x * 128LL; off < bytes; off += blockDim.x * 128LL)
    asm volatile("prefetch.global.L2 [%0];" ::"l"(c + off));
}

// stage_c != 0 (NC = 2): the tangent output is the DIRK stage operator J_G v = M v - stage_c J_r v,
// M v = B^T (W B v) being formed from the tangent's own Gauss values
// FP32: at least two CTAs per SM (four for the p = 3 Jv, where 128 registers suffice without spills), since
// the value + tangent physics would otherwise take enough registers to halve the resident warps of
// this latency-bound kernel (FP64 is bound by its pipe instead)
template <int N, int NC, typename R, int CM = CM_NATIVE>
__global__ void __launch_bounds__(Epb<N, NC>::value * Shape<N>::NP, sizeof(R) == 4 ? (N == 4 && NC == 2 ? 4 : 2) : 1)
k_volume(long long E, const Ops* __restrict__ ops, PhysT<R> P, R t,
                         const R* __restrict__ geo, const R* __restrict__ accg,
                         const R* __restrict__ xg, const R* __restrict__ ug,
                         const R* __restrict__ qg, const R* __restrict__ fh,
                         double* __restrict__ r, double* __restrict__ jv, R stage_c,
                         const R* __restrict__ mixg, long long ahead) {
  using S = typename std::conditional<NC == 2, DualT<R>, R>::type;
  constexpr int NP = Shape<N>::NP, NF = Shape<N>::NF, C = 5 * NC, EPB = Epb<N, NC>::value;
  __shared__ SmemOpsT<R> so;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* smem = reinterpret_cast<R*>(smem_raw);
  R* sF = smem;                             // [EPB][3][C][NP]
  R* sH = sF + EPB * 3 * C * NP;            // [EPB][6][C][NF]
  R* sR = sH + EPB * 6 * C * NF;            // [EPB][C][NP]
  R* sT = sR + EPB * C * NP;                // [EPB][C][NP]
  load_ops<N, R>(ops, so);
  const long long e0 = (long long)blockIdx.x * EPB;
  if constexpr (sizeof(R) == 4) {
    // FP32 is latency-bound on these loads: pull into L2 the records of the CTA `ahead` launches
    // later (one residency wave, so it starts about when this one ends)
    const long long eb = e0 + ahead * EPB;
    if (ahead > 0 && eb < E) {
      const long long ne = (E - eb < EPB) ? E - eb : EPB;
      for (int pl = 0; pl < NC; ++pl) {
        prefetch_l2(ug + pl * E * 5 * NP + eb * 5 * NP, ne * 5 * NP);
        prefetch_l2(qg + pl * E * 15 * NP + eb * 15 * NP, ne * 15 * NP);
        prefetch_l2(fh + pl * E * 30 * NF + eb * 30 * NF, ne * 30 * NF);
      }
      prefetch_l2(geo + eb * 10 * NP, ne * 10 * NP);
      prefetch_l2(accg + eb * 3 * NP, ne * 3 * NP);
      if (P.euv) prefetch_l2(xg + eb * 3 * NP, ne * 3 * NP);
      if (P.comp) prefetch_l2(mixg + eb * 8 * NP, ne * 8 * NP);
    }
  }
  const long long plane_f = E * 30 * NF;
  for (int idx = threadIdx.x; idx < EPB * 30 * NF; idx += blockDim.x) {
    const int l = idx / (30 * NF), rem = idx % (30 * NF);
    const long long e = e0 + l;
    if (e < E) {
      const int phi = rem / (5 * NF), c = (rem / NF) % 5, f = rem % NF;
      for (int pl = 0; pl < NC; ++pl)
        sH[((l * 6 + phi) * C + 5 * pl + c) * NF + f] = fh[pl * plane_f + e * 30 * NF + rem];
    }
  }
  const int el = threadIdx.x / NP, g = threadIdx.x % NP;
  const long long e = e0 + el;
  const bool active = el < EPB && e < E;
  S srcv[5];
  R wu[5] = {R(0), R(0), R(0), R(0), R(0)};   // W u_dot at this point (stage operator)
  if (active) {
    const long long plane_g = E * 5 * NP, plane_q = E * 15 * NP;
    S u[5], q[3][5];
#pragma unroll
    for (int c = 0; c < 5; ++c) u[c] = ld<S, NC, R>(ug + e * 5 * NP + c * NP + g, plane_g);
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int c = 0; c < 5; ++c) q[d][c] = ld<S, NC, R>(qg + e * 15 * NP + (d * 5 + c) * NP + g, plane_q);
    R G[9];
    const R* gp = geo + e * 10 * NP + g;
#pragma unroll
    for (int k = 0; k < 9; ++k) G[k] = gp[k * NP];
    const R Wd = gp[9 * NP];
    const R a3[3] = {accg[e * 3 * NP + g], accg[e * 3 * NP + NP + g], accg[e * 3 * NP + 2 * NP + g]};
    R x3[3] = {R(0), R(0), R(0)};
    if (P.euv) {
      x3[0] = xg[e * 3 * NP + g];
      x3[1] = xg[e * 3 * NP + NP + g];
      x3[2] = xg[e * 3 * NP + 2 * NP + g];
    }
    S Fref[3][5];
    R mg[8] = {R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0)};
    if (P.comp) {
#pragma unroll
      for (int k = 0; k < 8; ++k) mg[k] = mixg[(e * 8 + k) * NP + g];
    }
    volume_point<S>(P, u, q, G, Wd, a3, x3, t, Fref, srcv, mg);
    if constexpr (NC == 2) {
#pragma unroll
      for (int c = 0; c < 5; ++c) wu[c] = Wd * u[c].d;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        if constexpr (NC == 1) {
          sF[((el * 3 + a) * C + c) * NP + g] = Fref[a][c];
        } else {
          sF[((el * 3 + a) * C + c) * NP + g] = Fref[a][c].v;
          sF[((el * 3 + a) * C + 5 + c) * NP + g] = Fref[a][c].d;
        }
      }
  }
  __syncthreads();
  if (active) {
    for (int c = 0; c < C; ++c) {
      R acc;
      if constexpr (NC == 1) acc = srcv[c];
      else acc = (c < 5) ? srcv[c].v : srcv[c - 5].d;
#pragma unroll
      for (int a = 0; a < 3; ++a) acc = line_fma<N, true, false, R, CM>(so.D, sF + ((el * 3 + a) * C + c) * NP, g, a, acc);
#pragma unroll
      for (int phi = 0; phi < 6; ++phi) {
        const int axis = phi >> 1;
        const R coef = ((phi & 1) ? so.eR : so.eL)[axis_index<N>(g, axis)];
        acc = cm_fma<CM>(-coef, sH[((el * 6 + phi) * C + c) * NF + vol_face_point<N>(g, axis)], acc);
      }
      if (NC == 2 && c >= 5 && stage_c != R(0)) acc = wu[c - 5] - stage_c * acc;
      sR[(el * C + c) * NP + g] = acc;
    }
  }
  __syncthreads();
  R* in = sR;
  R* out = sT;
#pragma unroll
  for (int dir = 0; dir < 3; ++dir) {
    if (active)
      for (int c = 0; c < C; ++c) out[(el * C + c) * NP + g] = line<N, true, R, CM>(so.B, in + (el * C + c) * NP, g, dir);
    __syncthreads();
    R* tt = in;
    in = out;
    out = tt;
  }
  for (int idx = threadIdx.x; idx < EPB * 5 * NP; idx += blockDim.x) {
    const int l = idx / (5 * NP), rem = idx % (5 * NP);
    const long long ee = e0 + l;
    if (ee < E) {
      if (r) r[ee * 5 * NP + rem] = (double)in[(l * C) * NP + rem];
      if (NC == 2) jv[ee * 5 * NP + rem] = (double)in[(l * C + 5) * NP + rem];
    }
  }
}

// --------------------------------------------------------------------------------------------
// tensor transforms of nodal q and the mass matrix
// --------------------------------------------------------------------------------------------
// out = A x A x A in (T: A^T) for C components of EPB elements per CTA (one thread per point of
// each element), optional W-weighting and back-transform (mass matrix), optional face traces.
// Arithmetic in R (FP32 for the mass columns of FP32-assembled blocks); input and output FP64.
template <int N, bool T, int C, typename R = double>
__global__ void k_tensor(long long E, const Ops* __restrict__ ops, int which, const double* __restrict__ in_g,
                         double* __restrict__ out_g, const R* __restrict__ weight,
                         double* __restrict__ traces) {
  constexpr int NP = Shape<N>::NP, NF = Shape<N>::NF, EPB = Epb<N, 1>::value;
  __shared__ SmemOpsT<R> so;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* b0 = reinterpret_cast<R*>(smem_raw);   // [EPB][C][NP]
  R* b1 = b0 + EPB * C * NP;                // [EPB][C][NP]
  load_ops<N, R>(ops, so);
  const long long e0 = (long long)blockIdx.x * EPB;
  for (int idx = threadIdx.x; idx < EPB * C * NP; idx += blockDim.x) {
    const long long e = e0 + idx / (C * NP);
    if (e < E) b0[idx] = (R)in_g[e0 * C * NP + idx];
  }
  __syncthreads();
  const int el = threadIdx.x / NP, g = threadIdx.x % NP;
  const bool active = el < EPB && (e0 + el) < E;
  const R* A = (which == 0) ? so.B : so.Binv;
  R* in = b0;
  R* out = b1;
  for (int dir = 0; dir < 3; ++dir) {
    if (active)
      for (int c = 0; c < C; ++c) out[(el * C + c) * NP + g] = line<N, T>(A, in + (el * C + c) * NP, g, dir);
    __syncthreads();
    R* tt = in;
    in = out;
    out = tt;
  }
  if (weight) {
    // mass matrix: W-weighted Gauss values, then back with B^T
    if (active) {
      const R wd = weight[(e0 + el) * 10 * NP + 9 * NP + g];
      for (int c = 0; c < C; ++c) in[(el * C + c) * NP + g] *= wd;
    }
    __syncthreads();
    for (int dir = 0; dir < 3; ++dir) {
      if (active)
        for (int c = 0; c < C; ++c) out[(el * C + c) * NP + g] = line<N, true>(A, in + (el * C + c) * NP, g, dir);
      __syncthreads();
      R* tt = in;
      in = out;
      out = tt;
    }
  }
  for (int idx = threadIdx.x; idx < EPB * C * NP; idx += blockDim.x) {
    const long long e = e0 + idx / (C * NP);
    if (e < E) out_g[e0 * C * NP + idx] = (double)in[idx];
  }
  if (traces) {
    for (int idx = threadIdx.x; idx < EPB * 6 * C * NF; idx += blockDim.x) {
      const int l = idx / (6 * C * NF), rem = idx % (6 * C * NF);
      const long long e = e0 + l;
      if (e >= E) continue;
      const int phi = rem / (C * NF), c = (rem / NF) % C, f = rem % NF;
      const R* ev = (phi & 1) ? so.eR : so.eL;
      R acc = R(0);
      for (int k = 0; k < N; ++k) acc = fma(ev[k], in[(l * C + c) * NP + face_vol_point<N>(phi, f, k)], acc);
      traces[e * 6 * C * NF + rem] = (double)acc;
    }
  }
}

// variable composition (Sec. 2.1.1-2.1.2) at the Gauss and face points from the positions xg:
// mixg [E][8][NP] = (c_v*, grad c_v* (3), conductivity factor, chi_N2, chi_O2, chi_He),
// mixf [E][6][2][NF] = (c_v*, conductivity factor); face positions are the exact extrapolation of
// the Gauss-point positions (the map is a polynomial of degree p)
__device__ inline void mixture_at(const Phys& P, const double x[3], double out[8]) {
  const double r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  const double inv_ms[4] = {1.0, 16.0 / 28.0, 16.0 / 32.0, 16.0 / 4.0};      // m_O / m_s
  const double alpha[4] = {1.0, 3.6 / 5.6, 3.6 / 5.6, 1.0};                  // alpha_s / alpha_O
  double chi[4], dchi[4];
  chi[0] = 1.0;
  dchi[0] = 0.0;
  for (int s = 0; s < 3; ++s) {
    double c = 0.0, dc = 0.0;
    for (int j = 0; j < 2; ++j) {
      const double t = P.comp_a[2 * s + j] * exp(P.comp_b[2 * s + j] * r);
      c += t;
      dc += P.comp_b[2 * s + j] * t;
    }
    chi[1 + s] = c;
    dchi[1 + s] = dc;
    chi[0] -= c;
    dchi[0] -= dc;
  }
  double cv = 0.0, dcv = 0.0, ka = 0.0;
  for (int s = 0; s < 4; ++s) {
    cv += chi[s] * inv_ms[s];
    dcv += dchi[s] * inv_ms[s];
    ka += chi[s] * inv_ms[s] * alpha[s];
  }
  out[0] = cv;
  for (int d = 0; d < 3; ++d) out[1 + d] = dcv * x[d] / r;
  out[4] = ka / cv;
  out[5] = chi[1];
  out[6] = chi[2];
  out[7] = chi[3];
}

template <int N>
__global__ void k_mixture(long long E, const Ops* __restrict__ ops, Phys P, const double* __restrict__ xg,
                          double* __restrict__ mixg, double* __restrict__ mixf) {
  constexpr int NP = Shape<N>::NP, NF = Shape<N>::NF;
  const long long e = blockIdx.x;
  if (e >= E) return;
  for (int g = threadIdx.x; g < NP; g += blockDim.x) {
    const double x[3] = {xg[(e * 3 + 0) * NP + g], xg[(e * 3 + 1) * NP + g], xg[(e * 3 + 2) * NP + g]};
    double o[8];
    mixture_at(P, x, o);
    for (int k = 0; k < 8; ++k) mixg[(e * 8 + k) * NP + g] = o[k];
  }
  for (int idx = threadIdx.x; idx < 6 * NF; idx += blockDim.x) {
    const int phi = idx / NF, f = idx % NF;
    const double* ev = (phi & 1) ? ops->eR : ops->eL;
    double x[3] = {0.0, 0.0, 0.0};
    for (int d = 0; d < 3; ++d)
      for (int k = 0; k < N; ++k) x[d] = fma(ev[k], xg[(e * 3 + d) * NP + face_vol_point<N>(phi, f, k)], x[d]);
    double o[8];
    mixture_at(P, x, o);
    mixf[((e * 6 + phi) * 2) * NF + f] = o[0];
    mixf[((e * 6 + phi) * 2 + 1) * NF + f] = o[4];
  }
}

// M^{-1} v = B^{-1} (w |J|)^{-1} B^{-T} v for the 5 variables of EPB elements per CTA (the nodal
// mass matrix is B^T W B with B the square GLL-to-Gauss interpolation); in place allowed
template <int N>
__global__ void k_mass_inv(long long E, const Ops* __restrict__ ops, const double* in_g, double* out_g,
                           const double* __restrict__ geo) {
  constexpr int NP = Shape<N>::NP, EPB = Epb<N, 1>::value, C = 5;
  __shared__ SmemOps so;
  extern __shared__ double smem[];
  double* b0 = smem;                 // [EPB][C][NP]
  double* b1 = smem + EPB * C * NP;  // [EPB][C][NP]
  load_ops<N, double>(ops, so);
  const long long e0 = (long long)blockIdx.x * EPB;
  for (int idx = threadIdx.x; idx < EPB * C * NP; idx += blockDim.x) {
    const long long e = e0 + idx / (C * NP);
    if (e < E) b0[idx] = in_g[e0 * C * NP + idx];
  }
  __syncthreads();
  const int el = threadIdx.x / NP, g = threadIdx.x % NP;
  const bool active = el < EPB && (e0 + el) < E;
  double* in = b0;
  double* out = b1;
  for (int dir = 0; dir < 3; ++dir) {   // B^{-T}
    if (active)
      for (int c = 0; c < C; ++c) out[(el * C + c) * NP + g] = line<N, true>(so.Binv, in + (el * C + c) * NP, g, dir);
    __syncthreads();
    double* tt = in;
    in = out;
    out = tt;
  }
  if (active) {
    const double iw = 1.0 / geo[(e0 + el) * 10 * NP + 9 * NP + g];
    for (int c = 0; c < C; ++c) in[(el * C + c) * NP + g] *= iw;
  }
  __syncthreads();
  for (int dir = 0; dir < 3; ++dir) {   // B^{-1}
    if (active)
      for (int c = 0; c < C; ++c) out[(el * C + c) * NP + g] = line<N, false>(so.Binv, in + (el * C + c) * NP, g, dir);
    __syncthreads();
    double* tt = in;
    in = out;
    out = tt;
  }
  for (int idx = threadIdx.x; idx < EPB * C * NP; idx += blockDim.x) {
    const long long e = e0 + idx / (C * NP);
    if (e < E) out_g[e0 * C * NP + idx] = in[idx];
  }
}

// --------------------------------------------------------------------------------------------
// geometry at Gauss points and face points (isoparametric map of the node coordinates)
// --------------------------------------------------------------------------------------------
template <int N>
__global__ void k_geometry(long long E, const Ops* __restrict__ ops, Phys P, int gravity_kind,
                           double g0, double g1, double g2, double g_r0,
                           const double* __restrict__ x, double* __restrict__ geo,
                           double* __restrict__ accg, double* __restrict__ xg, double* __restrict__ fgeo) {
  constexpr int NP = Shape<N>::NP, NF = Shape<N>::NF;
  __shared__ SmemOps so;
  __shared__ double w1[MAXN];
  extern __shared__ double smem[];
  double* b0 = smem;           // [3][NP]
  double* b1 = b0 + 3 * NP;    // [3][NP]
  double* J = b1 + 3 * NP;     // [9][NP] J[d][a]
  load_ops<N, double>(ops, so);
  if (threadIdx.x < N) w1[threadIdx.x] = ops->w[threadIdx.x];
  const long long e = blockIdx.x;
  const int g = threadIdx.x;
  // positions relative to the element's first node: the Jacobian is unchanged (derivatives of the
  // basis sum to zero) and its rounding is relative to the element size instead of |x|
  for (int idx = threadIdx.x; idx < 3 * NP; idx += blockDim.x) {
    const int c = idx / NP;
    b0[idx] = x[e * 3 * NP + idx] - x[e * 3 * NP + c * NP];
  }
  __syncthreads();
  double* in = b0;
  double* out = b1;
  for (int dir = 0; dir < 3; ++dir) {
    if (g < NP)
      for (int c = 0; c < 3; ++c) out[c * NP + g] = line<N, false>(so.B, in + c * NP, g, dir);
    __syncthreads();
    double* tt = in;
    in = out;
    out = tt;
  }
  // in: Gauss point positions relative to the first node
  if (g < NP) {
    for (int d = 0; d < 3; ++d)
      for (int a = 0; a < 3; ++a) J[(d * 3 + a) * NP + g] = line<N, false>(so.D, in + d * NP, g, a);
  }
  __syncthreads();
  if (g < NP) {
    double j[3][3];
    for (int d = 0; d < 3; ++d)
      for (int a = 0; a < 3; ++a) j[d][a] = J[(d * 3 + a) * NP + g];
    // cofactors: cof[d][a] = d(det)/d j[d][a] = det * (J^{-1})[a][d]
    double cof[3][3];
    cof[0][0] = j[1][1] * j[2][2] - j[1][2] * j[2][1];
    cof[0][1] = j[1][2] * j[2][0] - j[1][0] * j[2][2];
    cof[0][2] = j[1][0] * j[2][1] - j[1][1] * j[2][0];
    cof[1][0] = j[0][2] * j[2][1] - j[0][1] * j[2][2];
    cof[1][1] = j[0][0] * j[2][2] - j[0][2] * j[2][0];
    cof[1][2] = j[0][1] * j[2][0] - j[0][0] * j[2][1];
    cof[2][0] = j[0][1] * j[1][2] - j[0][2] * j[1][1];
    cof[2][1] = j[0][2] * j[1][0] - j[0][0] * j[1][2];
    cof[2][2] = j[0][0] * j[1][1] - j[0][1] * j[1][0];
    const double det = j[0][0] * cof[0][0] + j[0][1] * cof[0][1] + j[0][2] * cof[0][2];
    const int i0 = g % N, i1 = (g / N) % N, i2 = g / (N * N);
    const double wq = w1[i0] * w1[i1] * w1[i2];
    double* gp = geo + e * 10 * NP + g;
    for (int a = 0; a < 3; ++a)
      for (int d = 0; d < 3; ++d) gp[(a * 3 + d) * NP] = wq * cof[d][a];
    gp[9 * NP] = wq * det;
    const double X[3] = {x[e * 3 * NP] + in[g], x[e * 3 * NP + NP] + in[NP + g], x[e * 3 * NP + 2 * NP] + in[2 * NP + g]};
    for (int d = 0; d < 3; ++d) xg[e * 3 * NP + d * NP + g] = X[d];
    double gv[3];
    if (gravity_kind == 0) {
      gv[0] = g0; gv[1] = g1; gv[2] = g2;
    } else {
      const double rr = sqrt(X[0] * X[0] + X[1] * X[1] + X[2] * X[2]);
      const double fac = -(g_r0 / rr) * (g_r0 / rr) / rr;
      for (int d = 0; d < 3; ++d) gv[d] = fac * X[d];
    }
    const double* w = P.omega;
    const double wx[3] = {w[1] * X[2] - w[2] * X[1], w[2] * X[0] - w[0] * X[2], w[0] * X[1] - w[1] * X[0]};
    const double wwx[3] = {w[1] * wx[2] - w[2] * wx[1], w[2] * wx[0] - w[0] * wx[2], w[0] * wx[1] - w[1] * wx[0]};
    const double cen = (P.cor * P.cor * 0.25);   // Fr^2 (cor = 2 Fr / sqrt(gamma))
    for (int d = 0; d < 3; ++d) accg[e * 3 * NP + d * NP + g] = gv[d] / P.gamma - cen * wwx[d];
  }
  // faces: extrapolate the tangential Jacobian columns, n dS = side * (J_{a+1} x J_{a+2})
  for (int idx = threadIdx.x; idx < 6 * NF; idx += blockDim.x) {
    const int phi = idx / NF, f = idx % NF;
    const int axis = phi >> 1;
    const double side = (phi & 1) ? 1.0 : -1.0;
    const double* ev = (phi & 1) ? so.eR : so.eL;
    const int a1 = (axis + 1) % 3, a2 = (axis + 2) % 3;
    double t1[3], t2[3];
    for (int d = 0; d < 3; ++d) {
      double s1 = 0.0, s2 = 0.0;
      for (int k = 0; k < N; ++k) {
        const int gg = face_vol_point<N>(phi, f, k);
        s1 = fma(ev[k], J[(d * 3 + a1) * NP + gg], s1);
        s2 = fma(ev[k], J[(d * 3 + a2) * NP + gg], s2);
      }
      t1[d] = s1;
      t2[d] = s2;
    }
    double nv[3] = {t1[1] * t2[2] - t1[2] * t2[1], t1[2] * t2[0] - t1[0] * t2[2], t1[0] * t2[1] - t1[1] * t2[0]};
    const int is = f % N, it = f / N;
    const double wf = w1[is] * w1[it];
    double* fp = fgeo + ((e * 6 + phi) * 4) * NF + f;
    double a2n = 0.0;
    for (int d = 0; d < 3; ++d) {
      fp[d * NF] = wf * side * nv[d];
      a2n += nv[d] * nv[d];
    }
    fp[3 * NF] = wf * sqrt(a2n);
  }
}

// --------------------------------------------------------------------------------------------
// Driver
// --------------------------------------------------------------------------------------------
template <int N, int NC, typename R>
struct Smem {
  static constexpr int NP = Shape<N>::NP, NF = Shape<N>::NF, C = 5 * NC, EPB = Epb<N, NC>::value;
  static constexpr size_t interp = sizeof(R) * (2 * EPB * C * NP);
  static constexpr size_t grad = sizeof(R) * (EPB * (C * NP + 6 * C * NF + 18 * NF + 9 * NP + 3 * C * NP + 18 * NF));
  static constexpr size_t volume = sizeof(R) * (EPB * (3 * C * NP + 6 * C * NF + 2 * C * NP));
};

template <typename R> inline WorkT<R> work_of(dg_mesh* m);
template <> inline WorkT<double> work_of<double>(dg_mesh* m) {
  return WorkT<double>{m->ws.ug, m->ws.uf, m->ws.qg, m->ws.qf, m->ws.fh, m->ws.qx, m->geo, m->fgeo, m->acc, m->xg,
                       m->mixg, m->mixf};
}
template <> inline WorkT<float> work_of<float>(dg_mesh* m) { return m->w32; }

template <typename K>
static int set_smem(K kernel, size_t bytes) {
  cudaError_t err = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (err != cudaSuccess) return fail(DG_ECUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(err));
  return DG_OK;
}

template <int N, int NC, typename R = double, int CM = CM_NATIVE>
static int run_interp(dg_mesh* m, const double* u, const double* v, cudaStream_t s) {
  constexpr int EPB = Epb<N, NC>::value, NP = Shape<N>::NP;
  if constexpr (std::is_same<R, double>::value && CM == CM_NATIVE)
    if (m->interp_mode == DG_INTERP_TC) return interp_tc<N, NC>(m, u, v, m->ws.ug, m->ws.uf, s);
  const size_t sm = Smem<N, NC, R>::interp;
  int rc = set_smem(k_interp<N, NC, R, CM>, sm);
  if (rc) return rc;
  const unsigned blocks = (unsigned)((m->E + EPB - 1) / EPB);
  const WorkT<R> w = work_of<R>(m);
  prof_begin(m, s, KK_INTERP);
  k_interp<N, NC, R, CM><<<blocks, EPB * NP, sm, s>>>(u, v, m->E, m->d_ops, w.ug, w.uf);
  prof_end(m, s);
  DG_LAUNCH_CHECK("k_interp");
  return DG_OK;
}

template <int N, int NC, bool BLK = false, typename R = double, int CM = CM_NATIVE, bool TO = false>
static int run_grad(dg_mesh* m, cudaStream_t s) {
  constexpr int EPB = Epb<N, NC>::value, NP = Shape<N>::NP;
  const size_t sm = Smem<N, NC, R>::grad;
  int rc = set_smem(k_grad<N, NC, BLK, R, CM, TO>, sm);
  if (rc) return rc;
  const unsigned blocks = (unsigned)((m->E + EPB - 1) / EPB);
  const WorkT<R> w = work_of<R>(m);
  prof_begin(m, s, KK_GRAD);
  k_grad<N, NC, BLK, R, CM, TO><<<blocks, EPB * NP, sm, s>>>(m->E, m->d_ops, phys_as<R>(m->phys), w.geo, w.fgeo,
                                                          m->nbr, m->nbr_fo, w.ug, w.uf, w.qg, w.qf, w.qx);
  prof_end(m, s);
  DG_LAUNCH_CHECK("k_grad");
  return DG_OK;
}

// the tangent plane of ug, uf (nodal v -> Gauss values and traces), with the NC = 1 kernel
template <int N, typename R>
static int run_interp_tangent(dg_mesh* m, const double* v, cudaStream_t s) {
  constexpr int EPB = Epb<N, 1>::value, NP = Shape<N>::NP, NF = Shape<N>::NF;
  if constexpr (std::is_same<R, double>::value)
    if (m->interp_mode == DG_INTERP_TC)
      return interp_tc<N, 1>(m, v, nullptr, m->ws.ug + m->E * 5 * NP, m->ws.uf + m->E * 30 * NF, s);
  const size_t sm = Smem<N, 1, R>::interp;
  int rc = set_smem(k_interp<N, 1, R, CM_NATIVE>, sm);
  if (rc) return rc;
  const unsigned blocks = (unsigned)((m->E + EPB - 1) / EPB);
  const WorkT<R> w = work_of<R>(m);
  prof_begin(m, s, KK_INTERP);
  k_interp<N, 1, R, CM_NATIVE><<<blocks, EPB * NP, sm, s>>>(v, nullptr, m->E, m->d_ops, w.ug + m->E * 5 * NP,
                                                             w.uf + m->E * 30 * NF);
  prof_end(m, s);
  DG_LAUNCH_CHECK("k_interp(tangent)");
  return DG_OK;
}

template <int N, int NC, bool BLK = false, typename R = double>
static int run_faces(dg_mesh* m, cudaStream_t s) {
  constexpr int NF = Shape<N>::NF;
  const long long work = m->nfaces * NF;
  const int threads = 128;
  const unsigned blocks = (unsigned)((work + threads - 1) / threads);
  const WorkT<R> w = work_of<R>(m);
  prof_begin(m, s, KK_FACES);
  k_faces<N, NC, BLK, R><<<blocks, threads, 0, s>>>(m->E, m->nfaces, phys_as<R>(m->phys), m->face_e, m->face_f,
                                                     m->nbr, m->nbr_fo, w.fgeo, w.uf, w.qf, w.qx, w.fh, w.mixf);
  prof_end(m, s);
  DG_LAUNCH_CHECK("k_faces");
  return DG_OK;
}

// resident CTAs of kernel fn on the mesh's device at this launch shape (0 if the query fails),
// cached in the mesh
inline long long resident_ctas(dg_mesh* m, const void* fn, int threads, size_t smem) {
  OccCache& c = m->occ;
  for (int i = 0; i < c.n; ++i)
    if (c.fn[i] == fn && c.smem[i] == smem) return c.val[i];
  int per_sm = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->device) != cudaSuccess) {
    cudaGetLastError();
    per_sm = sms = 0;
  }
  const long long v = (long long)per_sm * sms;
  if (c.n < OccCache::CAP) {
    c.fn[c.n] = fn;
    c.smem[c.n] = smem;
    c.val[c.n] = v;
    c.n++;
  }
  return v;
}

template <int N, int NC, typename R = double, int CM = CM_NATIVE>
static int run_volume(dg_mesh* m, double t, double* r, double* jv, cudaStream_t s, double stage_c = 0.0) {
  constexpr int EPB = Epb<N, NC>::value, NP = Shape<N>::NP;
  const size_t sm = Smem<N, NC, R>::volume;
  int rc = set_smem(k_volume<N, NC, R, CM>, sm);
  if (rc) return rc;
  const unsigned blocks = (unsigned)((m->E + EPB - 1) / EPB);
  const WorkT<R> w = work_of<R>(m);
  // CTAs resident at once (the prefetch distance of the FP32 kernel), per mesh and kernel instance
  const long long resident = resident_ctas(m, (const void*)k_volume<N, NC, R, CM>, EPB * NP, sm);
  prof_begin(m, s, KK_VOLUME);
  k_volume<N, NC, R, CM><<<blocks, EPB * NP, sm, s>>>(m->E, m->d_ops, phys_as<R>(m->phys), (R)t, w.geo, w.acc, w.xg,
                                                   w.ug, w.qg, w.fh, r, jv, (R)stage_c, w.mixg, resident);
  prof_end(m, s);
  DG_LAUNCH_CHECK("k_volume");
  return DG_OK;
}

template <int N>
int Driver<N>::geometry(dg_mesh* m, cudaStream_t s) {
  constexpr int NP = Shape<N>::NP;
  const size_t sm = sizeof(double) * 15 * NP;
  int rc = set_smem(k_geometry<N>, sm);
  if (rc) return rc;
  const dg_mesh_desc& d = m->desc;
  prof_begin(m, s, KK_GEOMETRY);
  k_geometry<N><<<(unsigned)m->E, NP < 32 ? 32 : NP, sm, s>>>(m->E, m->d_ops, m->phys, d.gravity_kind, d.gvec[0],
                                                            d.gvec[1], d.gvec[2], d.g_r0, m->x, m->geo, m->acc,
                                                            m->xg, m->fgeo);
  prof_end(m, s);
  DG_LAUNCH_CHECK("k_geometry");
  return DG_OK;
}

template <int N>
template <typename R>
int Driver<N>::gradient_p(dg_mesh* m, const double* u, const double* v, cudaStream_t s, bool tangent_only) {
  if (tangent_only) {   // u's value plane is in place: the tangent of v alone
    int rc = run_interp_tangent<N, R>(m, v, s);
    if (rc) return rc;
    return run_grad<N, 1, false, R, CM_NATIVE, true>(m, s);
  }
  int rc = v ? run_interp<N, 2, R>(m, u, v, s) : run_interp<N, 1, R>(m, u, nullptr, s);
  if (rc) return rc;
  return v ? run_grad<N, 2, false, R>(m, s) : run_grad<N, 1, false, R>(m, s);
}

template <int N>
template <typename R>
int Driver<N>::residual_p(dg_mesh* m, double t, double* r, double* jv, bool tangent, cudaStream_t s,
                          double stage_c) {
  int rc = tangent ? run_faces<N, 2, false, R>(m, s) : run_faces<N, 1, false, R>(m, s);
  if (rc) return rc;
  return tangent ? run_volume<N, 2, R>(m, t, r, jv, s, stage_c) : run_volume<N, 1, R>(m, t, r, nullptr, s);
}

template <int N>
int Driver<N>::gradient(dg_mesh* m, const double* u, const double* v, cudaStream_t s, bool f32, bool tangent_only) {
  return f32 ? gradient_p<float>(m, u, v, s, tangent_only) : gradient_p<double>(m, u, v, s, tangent_only);
}

template <int N>
int Driver<N>::residual(dg_mesh* m, const double* u, const double* v, double t, double* r, double* jv,
                        bool tangent, cudaStream_t s, bool f32, double stage_c) {
  (void)u;
  (void)v;
  return f32 ? residual_p<float>(m, t, r, jv, tangent, s, stage_c)
             : residual_p<double>(m, t, r, jv, tangent, s, stage_c);
}

template <int N>
template <typename R>
int Driver<N>::jv_blockdiag_p(dg_mesh* m, const double* u, const double* probe, double t, double* jv,
                              cudaStream_t s, bool tangent_only) {
  int rc;
  if (tangent_only) {   // u's value plane is in place
    rc = run_interp_tangent<N, R>(m, probe, s);
    if (rc) return rc;
    rc = run_grad<N, 1, true, R, CM_NATIVE, true>(m, s);
  } else {
    rc = run_interp<N, 2, R>(m, u, probe, s);
    if (rc) return rc;
    rc = run_grad<N, 2, true, R>(m, s);
  }
  if (rc) return rc;
  rc = run_faces<N, 2, true, R>(m, s);
  if (rc) return rc;
  return run_volume<N, 2, R>(m, t, nullptr, jv, s);
}

template <int N>
int Driver<N>::jv_blockdiag(dg_mesh* m, const double* u, const double* probe, double t, double* jv,
                            cudaStream_t s, bool f32, bool tangent_only) {
  return f32 ? jv_blockdiag_p<float>(m, u, probe, t, jv, s, tangent_only)
             : jv_blockdiag_p<double>(m, u, probe, t, jv, s, tangent_only);
}

template <int N>
template <int CM>
int Driver<N>::eval_cm_t(dg_mesh* m, const double* u, const double* v, double t, double* r, double* jv,
                         cudaStream_t s) {
  const bool tan = v != nullptr;
  int rc = tan ? run_interp<N, 2, float, CM>(m, u, v, s) : run_interp<N, 1, float, CM>(m, u, nullptr, s);
  if (rc) return rc;
  rc = tan ? run_grad<N, 2, false, float, CM>(m, s) : run_grad<N, 1, false, float, CM>(m, s);
  if (rc) return rc;
  rc = tan ? run_faces<N, 2, false, float>(m, s) : run_faces<N, 1, false, float>(m, s);
  if (rc) return rc;
  return tan ? run_volume<N, 2, float, CM>(m, t, r, jv, s) : run_volume<N, 1, float, CM>(m, t, r, nullptr, s);
}

template <int N>
int Driver<N>::eval_cm(dg_mesh* m, const double* u, const double* v, double t, double* r, double* jv, int cm,
                       cudaStream_t s) {
  switch (cm) {
    case CM_NATIVE: return eval_cm_t<CM_NATIVE>(m, u, v, t, r, jv, s);
    case CM_BF16: return eval_cm_t<CM_BF16>(m, u, v, t, r, jv, s);
    case CM_FP16: return eval_cm_t<CM_FP16>(m, u, v, t, r, jv, s);
    case CM_BF16X3: return eval_cm_t<CM_BF16X3>(m, u, v, t, r, jv, s);
    case CM_FP16X3: return eval_cm_t<CM_FP16X3>(m, u, v, t, r, jv, s);
    default: return fail(DG_EINVAL, "unknown contraction mode");
  }
}

template <int N>
int Driver<N>::q_to_nodal(dg_mesh* m, double* q, cudaStream_t s) {
  constexpr int NP = Shape<N>::NP;
  constexpr int EPB = Epb<N, 1>::value;
  const size_t sm = sizeof(double) * 2 * EPB * 15 * NP;
  int rc = set_smem(k_tensor<N, false, 15, double>, sm);
  if (rc) return rc;
  prof_begin(m, s, KK_TENSOR);
  k_tensor<N, false, 15, double><<<(unsigned)((m->E + EPB - 1) / EPB), EPB * NP, sm, s>>>(m->E, m->d_ops, 1, m->ws.qg, q,
                                                                                   nullptr, nullptr);
  prof_end(m, s);
  DG_LAUNCH_CHECK("k_tensor(q nodal)");
  return DG_OK;
}

template <int N>
int Driver<N>::q_from_nodal(dg_mesh* m, const double* q, cudaStream_t s) {
  constexpr int NP = Shape<N>::NP;
  constexpr int EPB = Epb<N, 1>::value;
  const size_t sm = sizeof(double) * 2 * EPB * 15 * NP;
  int rc = set_smem(k_tensor<N, false, 15, double>, sm);
  if (rc) return rc;
  prof_begin(m, s, KK_TENSOR);
  k_tensor<N, false, 15, double><<<(unsigned)((m->E + EPB - 1) / EPB), EPB * NP, sm, s>>>(m->E, m->d_ops, 0, q, m->ws.qg,
                                                                                   nullptr, m->ws.qf);
  prof_end(m, s);
  DG_LAUNCH_CHECK("k_tensor(q gauss)");
  return DG_OK;
}

template <int N>
int Driver<N>::mixture(dg_mesh* m) {
  k_mixture<N><<<(unsigned)m->E, 128>>>(m->E, m->d_ops, m->phys, m->xg, m->mixg, m->mixf);
  DG_LAUNCH_CHECK("k_mixture");
  return DG_OK;
}

template <int N>
int Driver<N>::mass_inv(dg_mesh* m, const double* v, double* mv, cudaStream_t s) {
  constexpr int NP = Shape<N>::NP;
  constexpr int EPB = Epb<N, 1>::value;
  const size_t sm = sizeof(double) * 2 * EPB * 5 * NP;
  int rc = set_smem(k_mass_inv<N>, sm);
  if (rc) return rc;
  prof_begin(m, s, KK_TENSOR);
  k_mass_inv<N><<<(unsigned)((m->E + EPB - 1) / EPB), EPB * NP, sm, s>>>(m->E, m->d_ops, v, mv, m->geo);
  prof_end(m, s);
  DG_LAUNCH_CHECK("k_mass_inv");
  return DG_OK;
}

template <int N>
int Driver<N>::mass(dg_mesh* m, const double* v, double* mv, cudaStream_t s, bool f32) {
  constexpr int NP = Shape<N>::NP;
  constexpr int EPB = Epb<N, 1>::value;
  const unsigned grid = (unsigned)((m->E + EPB - 1) / EPB);
  int rc;
  if (f32) {   // FP32 arithmetic on the FP32 geometry (ensure_f32 has run)
    if (!m->w32.geo) return fail(DG_EINVAL, "FP32 mass apply without the FP32 geometry");
    const size_t sm = sizeof(float) * 2 * EPB * 5 * NP;
    rc = set_smem(k_tensor<N, false, 5, float>, sm);
    if (rc) return rc;
    prof_begin(m, s, KK_TENSOR);
    k_tensor<N, false, 5, float><<<grid, EPB * NP, sm, s>>>(m->E, m->d_ops, 0, v, mv, m->w32.geo, nullptr);
  } else {
    const size_t sm = sizeof(double) * 2 * EPB * 5 * NP;
    rc = set_smem(k_tensor<N, false, 5, double>, sm);
    if (rc) return rc;
    prof_begin(m, s, KK_TENSOR);
    k_tensor<N, false, 5, double><<<grid, EPB * NP, sm, s>>>(m->E, m->d_ops, 0, v, mv, m->geo, nullptr);
  }
  prof_end(m, s);
  DG_LAUNCH_CHECK("k_tensor(mass)");
  return DG_OK;
}

}  // namespace dg
