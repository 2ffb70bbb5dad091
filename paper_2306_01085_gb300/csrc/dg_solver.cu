// Implicit DIRK step with Newton-GMRES (Sec. 3.1-3.2) and the block-Jacobi preconditioner.
//
// Stage i of the DIRK scheme (Alexander 1977) solves G(U) = M (U - u_n) - dt sum_{j<i} a_ij r(U_j)
// - dt a_ii r(U) = 0 by Newton's method (Eq. NewtonSolve); each Newton system J_G dU = -G with
// J_G = M - dt a_ii J_r is solved by right-preconditioned restarted GMRES whose only operator is
// the Jacobian-vector product. Arnoldi (classical Gram-Schmidt applied twice), the Hessenberg
// least-squares problem and every norm are FP64. The block-Jacobi preconditioner factors the exact
// element diagonal blocks of J_G in FP32 and applies their explicit inverses (batched in-place
// Gauss-Jordan with partial pivoting).
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_fp16.h>

#include "dg_bits.cuh"
#include "dg_internal.cuh"
#include "dg_nvtx.h"

namespace dg {

// ------------------------------------------------------------------------------------------
// DIRK tableaux from the order conditions (host)
// ------------------------------------------------------------------------------------------
// 2 stages: b = (1-g, g), c = (g, 1), order 2 requires g^2 - 2g + 1/2 = 0 -> g = 1 - 1/sqrt(2).
// 3 stages: stiffly accurate (last row of A = b), equal diagonal g; unknowns g, a21, b1, b2 solve
// b.1 = 1, b.c = 1/2, b.c^2 = 1/3, b.A.c = 1/6 (Newton's method from an L-stable starting point).
static int dirk_tableau(int stages, double A[3][3], double c[3]) {
  std::memset(A, 0, 9 * sizeof(double));
  if (stages == 1) {
    A[0][0] = 1.0;
    c[0] = 1.0;
    return DG_OK;
  }
  if (stages == 2) {
    const double g = 1.0 - 1.0 / std::sqrt(2.0);
    A[0][0] = g;
    A[1][0] = 1.0 - g;
    A[1][1] = g;
    c[0] = g;
    c[1] = 1.0;
    return DG_OK;
  }
  if (stages != 3) return fail(DG_EINVAL, "DIRK stages must be 1, 2 or 3");
  double x[4] = {0.44, 0.28, 1.2, -0.64};
  auto cond = [](const double* y, double* f) {
    const double g = y[0], a21 = y[1], b1 = y[2], b2 = y[3];
    const double c1 = g, c2 = a21 + g, c3 = 1.0;
    const double Ac[3] = {g * c1, a21 * c1 + g * c2, b1 * c1 + b2 * c2 + g * c3};
    f[0] = b1 + b2 + g - 1.0;
    f[1] = b1 * c1 + b2 * c2 + g * c3 - 0.5;
    f[2] = b1 * c1 * c1 + b2 * c2 * c2 + g * c3 * c3 - 1.0 / 3.0;
    f[3] = b1 * Ac[0] + b2 * Ac[1] + g * Ac[2] - 1.0 / 6.0;
  };
  for (int it = 0; it < 60; ++it) {
    double f[4], J[4][5];
    cond(x, f);
    for (int k = 0; k < 4; ++k) {
      double xp[4], xm[4], fp[4], fm[4];
      std::memcpy(xp, x, sizeof(x));
      std::memcpy(xm, x, sizeof(x));
      xp[k] += 1e-7;
      xm[k] -= 1e-7;
      cond(xp, fp);
      cond(xm, fm);
      for (int r = 0; r < 4; ++r) J[r][k] = (fp[r] - fm[r]) / 2e-7;
    }
    for (int r = 0; r < 4; ++r) J[r][4] = -f[r];
    for (int k = 0; k < 4; ++k) {  // Gaussian elimination with partial pivoting
      int p = k;
      for (int r = k + 1; r < 4; ++r)
        if (std::fabs(J[r][k]) > std::fabs(J[p][k])) p = r;
      for (int q = 0; q < 5; ++q) std::swap(J[k][q], J[p][q]);
      for (int r = k + 1; r < 4; ++r) {
        const double l = J[r][k] / J[k][k];
        for (int q = k; q < 5; ++q) J[r][q] -= l * J[k][q];
      }
    }
    double dx[4];
    for (int k = 3; k >= 0; --k) {
      double s = J[k][4];
      for (int q = k + 1; q < 4; ++q) s -= J[k][q] * dx[q];
      dx[k] = s / J[k][k];
    }
    double mx = 0.0;
    for (int k = 0; k < 4; ++k) {
      x[k] += dx[k];
      mx = std::fmax(mx, std::fabs(dx[k]));
    }
    if (mx < 1e-15) break;
  }
  const double g = x[0];
  A[0][0] = g;
  A[1][0] = x[1];
  A[1][1] = g;
  A[2][0] = x[2];
  A[2][1] = x[3];
  A[2][2] = g;
  c[0] = g;
  c[1] = x[1] + g;
  c[2] = 1.0;
  return DG_OK;
}

// ------------------------------------------------------------------------------------------
// vector kernels (FP64); reductions use a fixed grid and a fixed summation order
// ------------------------------------------------------------------------------------------
constexpr int RED_BLOCKS = 304;   // 2 x 152 SMs
constexpr int RED_THREADS = 256;
constexpr int MAXK = 64;          // largest restart + 1
constexpr int RB_MAX = 16;        // largest reduced basis

// out = a x + b y + c z; out may alias any input (each entry is read before it is written, by the
// same thread)
__global__ void k_lincomb(long long n, double a, const double* x, double b, const double* y, double c,
                          const double* z, double* out) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double v = a * x[i];
    if (y) v = fma(b, y[i], v);
    if (z) v = fma(c, z[i], v);
    out[i] = v;
  }
}

// out = x * (*scale_num) / sqrt(*scale_den)  (device-resident scalars)
__global__ void k_scale_dev(long long n, const double* x, const double* __restrict__ den, double* out) {
  __shared__ double s_sh;   // the scale formed once per block (an FP64 square root and division)
  if (threadIdx.x == 0) s_sh = 1.0 / sqrt(*den);
  __syncthreads();
  const double s = s_sh;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = x[i] * s;
}

// partial[j][block] = sum_i V_j[i] w[i] for j < k; partial[k][block] = sum_i w[i]^2.
// Vectors are taken 16 at a time (one pass over w per group) so the accumulators stay in
// registers; warp-shuffle and cross-warp reductions, fixed order.
constexpr int MDOT_G = 16;
__global__ void __launch_bounds__(RED_THREADS) k_mdot(long long n, int k, const double* __restrict__ V, long long ldv,
                                                     const double* __restrict__ w, double* __restrict__ partial) {
  __shared__ double red[RED_THREADS / 32][MDOT_G];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j0 = 0; j0 <= k; j0 += MDOT_G) {
    double acc[MDOT_G];
#pragma unroll
    for (int j = 0; j < MDOT_G; ++j) acc[j] = 0.0;
    // two elements per thread per pass keep twice the loads in flight
    const long long T = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += 2 * T) {
      const long long i2 = i + T;
      const bool ok2 = i2 < n;
      const double wa = w[i], wb = ok2 ? w[i2] : 0.0;
#pragma unroll
      for (int j = 0; j < MDOT_G; ++j) {
        const int jj = j0 + j;
        if (jj < k) {
          const double* Vj = V + jj * ldv;
          acc[j] = fma(Vj[i], wa, acc[j]);
          if (ok2) acc[j] = fma(Vj[i2], wb, acc[j]);
        } else if (jj == k) {
          acc[j] = fma(wa, wa, acc[j]);
          acc[j] = fma(wb, wb, acc[j]);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < MDOT_G; ++j) {
      double v = acc[j];
      for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
      if (lane == 0) red[warp][j] = v;
    }
    __syncthreads();
    if (threadIdx.x < MDOT_G && j0 + threadIdx.x <= k) {
      double v = 0.0;
      for (int q = 0; q < RED_THREADS / 32; ++q) v += red[q][threadIdx.x];
      partial[(j0 + threadIdx.x) * RED_BLOCKS + blockIdx.x] = v;
    }
    __syncthreads();
  }
}

// Fused Gram-Schmidt sweep: w <- w - sum_{j<k} h_j V_j, then (DOTS) partial[j][block] =
// sum_i V_j[i] w[i] for j < k, and partial[DOTS ? k : 0][block] = sum_i w[i]^2. V_j[i] is read
// from HBM once; the dot pass re-reads it right after the update (L1/L2 hits). KM >= k.
template <int KM, bool DOTS>
__global__ void __launch_bounds__(RED_THREADS, 2) k_update_dot(long long n, int k, const double* __restrict__ V,
                                                              long long ldv, const double* __restrict__ h,
                                                              double* __restrict__ w, double* __restrict__ partial) {
  constexpr int NA = DOTS ? KM + 1 : 1;
  __shared__ double hs[KM];
  __shared__ double red[RED_THREADS / 32][NA];
  if (threadIdx.x < k) hs[threadIdx.x] = h[threadIdx.x];
  __syncthreads();
  double acc[NA];
#pragma unroll
  for (int j = 0; j < NA; ++j) acc[j] = 0.0;
  const long long T = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += T) {
    double x = w[i];
#pragma unroll
    for (int j = 0; j < KM; ++j)
      if (j < k) x = fma(-hs[j], V[j * ldv + i], x);
    w[i] = x;
    if constexpr (DOTS) {
#pragma unroll
      for (int j = 0; j < KM; ++j)
        if (j < k) acc[j] = fma(V[j * ldv + i], x, acc[j]);
    }
    acc[NA - 1] = fma(x, x, acc[NA - 1]);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < NA; ++j) {
    double v = acc[j];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) red[warp][j] = v;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < NA; j += blockDim.x) {
    if (DOTS && j < KM && j >= k) continue;
    double v = 0.0;
    for (int q = 0; q < RED_THREADS / 32; ++q) v += red[q][j];
    const int row = DOTS ? (j == KM ? k : j) : 0;
    partial[row * RED_BLOCKS + blockIdx.x] = v;
  }
}

// The same two operations for a compile-time number of vectors K and 16-byte loads (n even, so
// every V_j starts on a 16-byte boundary): no predication, every load of an element issued
// back to back. partial rows as above.
template <int K>
__global__ void __launch_bounds__(RED_THREADS) k_mdot_k(long long n2, const double2* __restrict__ V, long long ldv2,
                                                       const double2* __restrict__ w, double* __restrict__ partial) {
  double acc[K + 1];
#pragma unroll
  for (int j = 0; j <= K; ++j) acc[j] = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += (long long)gridDim.x * blockDim.x) {
    const double2 x = w[i];
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const double2 v = V[j * ldv2 + i];
      acc[j] = fma(v.x, x.x, fma(v.y, x.y, acc[j]));
    }
    acc[K] = fma(x.x, x.x, fma(x.y, x.y, acc[K]));
  }
  __shared__ double red[RED_THREADS / 32][K + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j <= K; ++j) {
    double v = acc[j];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) red[warp][j] = v;
  }
  __syncthreads();
  for (int j = threadIdx.x; j <= K; j += blockDim.x) {
    double v = 0.0;
    for (int q = 0; q < RED_THREADS / 32; ++q) v += red[q][j];
    partial[j * RED_BLOCKS + blockIdx.x] = v;
  }
}

template <int K, bool DOTS>
__global__ void __launch_bounds__(RED_THREADS, 2) k_update_dot_k(long long n2, const double2* __restrict__ V,
                                                                long long ldv2, const double* __restrict__ h,
                                                                double2* __restrict__ w, double* __restrict__ partial) {
  // K <= 8: the element's V values stay in registers for the dots. K > 8: vector loops unrolled
  // by 8, the dot pass reads V again from L2 (ld.global.cg), and each thread's K dot accumulators
  // live in dynamic shared memory laid out [j][thread] (conflict-free), so nothing spills.
  constexpr bool SMALL = K <= 8;
  constexpr bool SACC = DOTS && !SMALL;
  constexpr int NR = (DOTS && SMALL) ? K + 1 : 1;   // register accumulators (last: |w|^2)
  extern __shared__ double sacc[];                  // SACC: [K][RED_THREADS]
  __shared__ double hs[K > 0 ? K : 1];
  if constexpr (K > 0)
    if (threadIdx.x < K) hs[threadIdx.x] = h[threadIdx.x];
  if constexpr (SACC)
    for (int j = 0; j < K; ++j) sacc[j * RED_THREADS + threadIdx.x] = 0.0;
  __syncthreads();
  double acc[NR];
#pragma unroll
  for (int j = 0; j < NR; ++j) acc[j] = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += (long long)gridDim.x * blockDim.x) {
    double2 x = w[i];
    if constexpr (SMALL) {
      double2 v[K > 0 ? K : 1];
#pragma unroll
      for (int j = 0; j < K; ++j) {
        v[j] = V[j * ldv2 + i];
        x.x = fma(-hs[j], v[j].x, x.x);
        x.y = fma(-hs[j], v[j].y, x.y);
      }
      w[i] = x;
      if constexpr (DOTS) {
#pragma unroll
        for (int j = 0; j < K; ++j) acc[j] = fma(v[j].x, x.x, fma(v[j].y, x.y, acc[j]));
      }
    } else {
#pragma unroll 8
      for (int j = 0; j < K; ++j) {
        const double2 vj = V[j * ldv2 + i];
        x.x = fma(-hs[j], vj.x, x.x);
        x.y = fma(-hs[j], vj.y, x.y);
      }
      w[i] = x;
      if constexpr (DOTS) {
#pragma unroll 8
        for (int j = 0; j < K; ++j) {
          const double2 vj = __ldcg(&V[j * ldv2 + i]);
          double& a = sacc[j * RED_THREADS + threadIdx.x];
          a = fma(vj.x, x.x, fma(vj.y, x.y, a));
        }
      }
    }
    acc[NR - 1] = fma(x.x, x.x, fma(x.y, x.y, acc[NR - 1]));
  }
  constexpr int NA = DOTS ? K + 1 : 1;
  __shared__ double red[RED_THREADS / 32][NA];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j = 0; j < NA; ++j) {
    double a;
    if constexpr (SACC) a = (j < K) ? sacc[j * RED_THREADS + threadIdx.x] : acc[0];
    else a = (NR == 1) ? acc[0] : acc[j < NR ? j : NR - 1];
    for (int off = 16; off > 0; off >>= 1) a += __shfl_down_sync(0xffffffffu, a, off);
    if (lane == 0) red[warp][j] = a;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < NA; j += blockDim.x) {
    double a = 0.0;
    for (int q = 0; q < RED_THREADS / 32; ++q) a += red[q][j];
    partial[j * RED_BLOCKS + blockIdx.x] = a;
  }
}

// FP32 Gram-Schmidt arithmetic on the FP64 basis (the mixed-precision solve, whose Jv is itself
// FP32), with the integer-pipe conversions to_f32 / to_f64 of dg_bits.cuh.

// k_mdot_k with FP32 products and per-thread FP32 sums (cross-thread sums in FP64); the |w|^2 row
// stays FP64.
template <int K>
__global__ void __launch_bounds__(RED_THREADS, 2) k_mdot_f32(long long n2, const double2* __restrict__ V, long long ldv2,
                                                         const double2* __restrict__ w, double* __restrict__ partial) {
  float acc[K];
#pragma unroll
  for (int j = 0; j < K; ++j) acc[j] = 0.0f;
  double nrm = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += (long long)gridDim.x * blockDim.x) {
    const double2 x = w[i];
    const float xx = to_f32(x.x), xy = to_f32(x.y);
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const double2 v = V[j * ldv2 + i];
      acc[j] = fmaf(to_f32(v.x), xx, fmaf(to_f32(v.y), xy, acc[j]));
    }
    nrm = fma(x.x, x.x, fma(x.y, x.y, nrm));
  }
  __shared__ double red[RED_THREADS / 32][K + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < K; ++j) {
    double v = to_f64(acc[j]);
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) red[warp][j] = v;
  }
  for (int off = 16; off > 0; off >>= 1) nrm += __shfl_down_sync(0xffffffffu, nrm, off);
  if (lane == 0) red[warp][K] = nrm;
  __syncthreads();
  for (int j = threadIdx.x; j <= K; j += blockDim.x) {
    double v = 0.0;
    for (int q = 0; q < RED_THREADS / 32; ++q) v += red[q][j];
    partial[j * RED_BLOCKS + blockIdx.x] = v;
  }
}

// k_update_dot_k with the correction sum_j h_j V_j formed in FP32 and subtracted from w in FP64
// (one FP64 add per entry), the element's truncated V values kept in registers for the FP32
// dots; |w|^2 in FP64. Partial rows as k_update_dot_k.
template <int K, bool DOTS>
__global__ void __launch_bounds__(RED_THREADS, 2) k_update_dot_f32(long long n2, const double2* __restrict__ V,
                                                                  long long ldv2, const double* __restrict__ h,
                                                                  double2* __restrict__ w, double* __restrict__ partial) {
  __shared__ float hs[K];
  if (threadIdx.x < K) hs[threadIdx.x] = to_f32(h[threadIdx.x]);
  __syncthreads();
  constexpr int NA = DOTS ? K : 1;
  constexpr bool CACHE = DOTS && K <= 24;   // the truncated V values stay in registers for the dots
  float acc[NA];
#pragma unroll
  for (int j = 0; j < NA; ++j) acc[j] = 0.0f;
  double nrm = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += (long long)gridDim.x * blockDim.x) {
    double2 x = w[i];
    float2 vf[CACHE ? K : 1];
    float cx = 0.0f, cy = 0.0f;
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const double2 v = V[j * ldv2 + i];
      const float2 f = make_float2(to_f32(v.x), to_f32(v.y));
      if constexpr (CACHE) vf[j] = f;
      cx = fmaf(hs[j], f.x, cx);
      cy = fmaf(hs[j], f.y, cy);
    }
    x.x -= to_f64(cx);
    x.y -= to_f64(cy);
    w[i] = x;
    if constexpr (DOTS) {
      const float xx = to_f32(x.x), xy = to_f32(x.y);
#pragma unroll
      for (int j = 0; j < K; ++j) {
        float2 f;
        if constexpr (CACHE) {
          f = vf[j];
        } else {   // the element was just read: an L2 hit
          const double2 v = __ldcg(&V[j * ldv2 + i]);
          f = make_float2(to_f32(v.x), to_f32(v.y));
        }
        acc[j] = fmaf(f.x, xx, fmaf(f.y, xy, acc[j]));
      }
    }
    nrm = fma(x.x, x.x, fma(x.y, x.y, nrm));
  }
  __shared__ double red[RED_THREADS / 32][NA + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if constexpr (DOTS) {
#pragma unroll
    for (int j = 0; j < K; ++j) {
      double a = to_f64(acc[j]);
      for (int off = 16; off > 0; off >>= 1) a += __shfl_down_sync(0xffffffffu, a, off);
      if (lane == 0) red[warp][j] = a;
    }
  }
  for (int off = 16; off > 0; off >>= 1) nrm += __shfl_down_sync(0xffffffffu, nrm, off);
  if (lane == 0) red[warp][NA] = nrm;
  __syncthreads();
  // DOTS: rows 0..K-1 the dots, row K |w|^2; otherwise row 0 |w|^2
  for (int j = threadIdx.x; j < (DOTS ? K + 1 : 1); j += blockDim.x) {
    const int src = DOTS ? j : NA;
    double a = 0.0;
    for (int q = 0; q < RED_THREADS / 32; ++q) a += red[q][src];
    partial[j * RED_BLOCKS + blockIdx.x] = a;
  }
}

// The same two sweeps on an FP32-stored basis (the mixed-precision solve keeps its Krylov vectors
// in FP32: the basis is read three times per Arnoldi step, and the projections are FP32 anyway).
template <int K>
__global__ void __launch_bounds__(RED_THREADS, 2) k_mdot_f32v(long long n2, const float2* __restrict__ V, long long ldv2,
                                                          const double2* __restrict__ w, double* __restrict__ partial) {
  float acc[K];
#pragma unroll
  for (int j = 0; j < K; ++j) acc[j] = 0.0f;
  double nrm = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += (long long)gridDim.x * blockDim.x) {
    const double2 x = w[i];
    const float xx = to_f32(x.x), xy = to_f32(x.y);
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const float2 v = V[j * ldv2 + i];
      acc[j] = fmaf(v.x, xx, fmaf(v.y, xy, acc[j]));
    }
    nrm = fma(x.x, x.x, fma(x.y, x.y, nrm));
  }
  __shared__ double red[RED_THREADS / 32][K + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < K; ++j) {
    double v = to_f64(acc[j]);
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) red[warp][j] = v;
  }
  for (int off = 16; off > 0; off >>= 1) nrm += __shfl_down_sync(0xffffffffu, nrm, off);
  if (lane == 0) red[warp][K] = nrm;
  __syncthreads();
  for (int j = threadIdx.x; j <= K; j += blockDim.x) {
    double v = 0.0;
    for (int q = 0; q < RED_THREADS / 32; ++q) v += red[q][j];
    partial[j * RED_BLOCKS + blockIdx.x] = v;
  }
}

template <int K, bool DOTS>
__global__ void __launch_bounds__(RED_THREADS, 2) k_update_dot_f32v(long long n2, const float2* __restrict__ V,
                                                                   long long ldv2, const double* __restrict__ h,
                                                                   double2* __restrict__ w, double* __restrict__ partial) {
  __shared__ float hs[K];
  if (threadIdx.x < K) hs[threadIdx.x] = to_f32(h[threadIdx.x]);
  __syncthreads();
  constexpr int NA = DOTS ? K : 1;
  constexpr bool CACHE = DOTS && K <= 24;
  float acc[NA];
#pragma unroll
  for (int j = 0; j < NA; ++j) acc[j] = 0.0f;
  double nrm = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += (long long)gridDim.x * blockDim.x) {
    double2 x = w[i];
    float2 vf[CACHE ? K : 1];
    float cx = 0.0f, cy = 0.0f;
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const float2 f = V[j * ldv2 + i];
      if constexpr (CACHE) vf[j] = f;
      cx = fmaf(hs[j], f.x, cx);
      cy = fmaf(hs[j], f.y, cy);
    }
    x.x -= to_f64(cx);
    x.y -= to_f64(cy);
    w[i] = x;
    if constexpr (DOTS) {
      const float xx = to_f32(x.x), xy = to_f32(x.y);
#pragma unroll
      for (int j = 0; j < K; ++j) {
        float2 f;
        if constexpr (CACHE) f = vf[j];
        else f = __ldcg(&V[j * ldv2 + i]);   // the element was just read: an L2 hit
        acc[j] = fmaf(f.x, xx, fmaf(f.y, xy, acc[j]));
      }
    }
    nrm = fma(x.x, x.x, fma(x.y, x.y, nrm));
  }
  __shared__ double red[RED_THREADS / 32][NA + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if constexpr (DOTS) {
#pragma unroll
    for (int j = 0; j < K; ++j) {
      double a = to_f64(acc[j]);
      for (int off = 16; off > 0; off >>= 1) a += __shfl_down_sync(0xffffffffu, a, off);
      if (lane == 0) red[warp][j] = a;
    }
  }
  for (int off = 16; off > 0; off >>= 1) nrm += __shfl_down_sync(0xffffffffu, nrm, off);
  if (lane == 0) red[warp][NA] = nrm;
  __syncthreads();
  for (int j = threadIdx.x; j < (DOTS ? K + 1 : 1); j += blockDim.x) {
    const int src = DOTS ? j : NA;
    double a = 0.0;
    for (int q = 0; q < RED_THREADS / 32; ++q) a += red[q][src];
    partial[j * RED_BLOCKS + blockIdx.x] = a;
  }
}

// out = a x in FP32 (a new basis vector), and the FP32 vector widened back to FP64
__global__ void k_scale_to_f32(long long n, const double* __restrict__ x, double a, const double* __restrict__ den,
                               float* __restrict__ out) {
  __shared__ float sf_sh;   // the scale formed once per block
  if (threadIdx.x == 0) sf_sh = den ? (float)(1.0 / sqrt(*den)) : (float)a;
  __syncthreads();
  const float sf = sf_sh;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = to_f32(x[i]) * sf;
}

__global__ void k_widen(long long n, const float* __restrict__ x, double* __restrict__ out) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = to_f64(x[i]);
}

// out = sum_j y[j] V_j (j < k) on the FP32 basis, FP32 sums widened to FP64
__global__ void k_combine_f32v(long long n, int k, const float* __restrict__ V, long long ldv,
                               const double* __restrict__ y, double* __restrict__ out) {
  __shared__ float ys[MAXK];
  if (threadIdx.x < k) ys[threadIdx.x] = (float)y[threadIdx.x];
  __syncthreads();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    float v = 0.0f;
    for (int j = 0; j < k; ++j) v = fmaf(ys[j], V[j * ldv + i], v);
    out[i] = to_f64(v);
  }
}

// out[j] = sum_b partial[j][b] (+= into out when accumulate); also out_sq = partial[k] sum
__global__ void k_mdot_finish(int k, const double* __restrict__ partial, double* __restrict__ out, int accumulate) {
  const int j = threadIdx.x;
  if (j > k) return;
  double s = 0.0;
  for (int b = 0; b < RED_BLOCKS; ++b) s += partial[j * RED_BLOCKS + b];
  out[j] = accumulate ? out[j] + s : s;
}

// w -= sum_j h[j] V_j for j < k
__global__ void k_maxpy(long long n, int k, const double* __restrict__ V, long long ldv,
                        const double* __restrict__ h, double* __restrict__ w) {
  __shared__ double hs[MAXK];
  if (threadIdx.x < k) hs[threadIdx.x] = h[threadIdx.x];
  __syncthreads();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double v = w[i];
    for (int j = 0; j < k; ++j) v = fma(-hs[j], V[j * ldv + i], v);
    w[i] = v;
  }
}

// t = C s for the r x r row-major matrix C (reduced-basis coefficients)
__global__ void k_small_matvec(int r, const double* __restrict__ C, const double* __restrict__ sv,
                               double* __restrict__ tv) {
  const int i = threadIdx.x;
  if (i >= r) return;
  double acc = 0.0;
  for (int j = 0; j < r; ++j) acc = fma(C[i * r + j], sv[j], acc);
  tv[i] = acc;
}

// out = sum_j y[j] V_j (j < k)
__global__ void k_combine(long long n, int k, const double* __restrict__ V, long long ldv,
                          const double* __restrict__ y, double* __restrict__ out) {
  __shared__ double ys[MAXK];
  if (threadIdx.x < k) ys[threadIdx.x] = y[threadIdx.x];
  __syncthreads();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double v = 0.0;
    for (int j = 0; j < k; ++j) v = fma(ys[j], V[j * ldv + i], v);
    out[i] = v;
  }
}

// ------------------------------------------------------------------------------------------
// block-Jacobi: probes, column scatter, FP32 batched LU (column-major blocks), solves
// ------------------------------------------------------------------------------------------
__global__ void k_probe(long long E, int n, int j, double* __restrict__ v) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < E * n; i += (long long)gridDim.x * blockDim.x)
    v[i] = ((int)(i % n) == j) ? 1.0 : 0.0;
}

// column j of every block: B[e][j][row] = mv[e][row] - c jv[e][row]
__global__ void k_scatter_col(long long E, int n, int j, double c, const double* __restrict__ mv,
                              const double* __restrict__ jv, float* __restrict__ blocks) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < E * n; i += (long long)gridDim.x * blockDim.x) {
    const long long e = i / n;
    const int row = (int)(i % n);
    blocks[(e * n + j) * (long long)n + row] = (float)(mv[i] - c * jv[i]);
  }
}

// Blocked Gauss-Jordan inversion in global memory, one CTA per block, for blocks too large for one
// CTA's shared memory. Only the current panel of B columns is staged, so two CTAs share an SM and one
// block's serial panel steps overlap another block's update. Row interchanges are not applied to
// the matrix: a permutation pi (logical row -> row in memory) records them, so a panel's pivoting
// costs no traffic in the other columns. Per panel:
//   1. the panel's rows are gathered through pi into registers (rows t, t + NT, t + 2 NT of thread
//      t) and the unblocked in-place steps run there: each step needs one block barrier, before
//      which the lane holding each warp's pivot candidate and the holder of row k publish their
//      rows in small double-buffered slots; after it every thread picks the pivot p, swaps pi[k]
//      and pi[p] (thread 0), and rewrites its own rows (rows k and p take the interchanged and
//      scaled values). The panel then holds the columns of the panel's transform
//      T = G_b P_b ... G_1 P_1, the identity outside the panel's columns, and is scattered back
//      through pi into the block and into shared memory in memory-row order;
//   2. T acts on every other column x as x <- x~ + P x_K (x_K the logical rows k0 .. k0 + b, x~ = x
//      with those rows zeroed): 64 columns at a time, x_K is gathered through pi into U and
//      C += P U runs as a tiled FP32 GEMM in memory-row order (4 x 4 register tiles, 16-byte shared
//      loads of P and U), the rows of x_K reading as zero.
// At the end every column is un-permuted through pi, and the columns are interchanged back in
// reverse pivot order, in strips of 32 rows read whole before they are written.
constexpr int GJG_B = 32;
constexpr int GJG_CH = 64;     // columns per update chunk

// The B steps of a full panel with the step index known at compile time: every row then needs one
// FMA per entry. Each warp's candidate lane publishes its row already scaled by the reciprocal of its
// pivot-column entry (r_j = x_j / x_c, r_c = 1 / x_c), the holder of row k publishes row k as it is;
// after the barrier, rows other than k and p take x_j - x_c r_j (x_c -> -x_c r_c), row k takes r and
// row p (the old row k) takes q_j - q_c r_j.
template <int B, int MRT, int NT>
__device__ __forceinline__ void gj_panel_full(float (&rv)[MRT][B], int n, int k0, float* __restrict__ slot,
                                              float (*wval)[NT / 32], int (*widx)[NT / 32], int* __restrict__ pv,
                                              int* __restrict__ pi, int* __restrict__ info) {
  constexpr int NWARP = NT / 32;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
#pragma unroll
  for (int c = 0; c < B; ++c) {
    const int kc = k0 + c, sb = c & 1;
    float best = -1.0f;
    int bi = n, bm = 0;
#pragma unroll
    for (int m = 0; m < MRT; ++m) {
      const int i = t + NT * m;
      if (i < n && i >= kc) {
        const float a = fabsf(rv[m][c]);
        if (a > best) { best = a; bi = i; bm = m; }
      }
    }
    float wb = best;
    int wi = bi;
    for (int off = 16; off > 0; off >>= 1) {
      const float o = __shfl_xor_sync(0xffffffffu, wb, off);
      const int oi = __shfl_xor_sync(0xffffffffu, wi, off);
      if (o > wb || (o == wb && oi < wi)) { wb = o; wi = oi; }
    }
    float* ws = slot + ((size_t)sb * (NWARP + 1) + warp) * B;
    float* ks = slot + ((size_t)sb * (NWARP + 1) + NWARP) * B;
    if (wi == bi && wi < n) {
#pragma unroll
      for (int m = 0; m < MRT; ++m)
        if (m == bm) {
          const float rinv = 1.0f / rv[m][c];
#pragma unroll
          for (int q = 0; q < B / 4; ++q) {
            float4 v;
            v.x = (4 * q + 0 == c) ? rinv : rv[m][4 * q + 0] * rinv;
            v.y = (4 * q + 1 == c) ? rinv : rv[m][4 * q + 1] * rinv;
            v.z = (4 * q + 2 == c) ? rinv : rv[m][4 * q + 2] * rinv;
            v.w = (4 * q + 3 == c) ? rinv : rv[m][4 * q + 3] * rinv;
            *reinterpret_cast<float4*>(ws + 4 * q) = v;
          }
        }
    }
#pragma unroll
    for (int m = 0; m < MRT; ++m)
      if (t + NT * m == kc)
#pragma unroll
        for (int q = 0; q < B / 4; ++q)
          *reinterpret_cast<float4*>(ks + 4 * q) =
              make_float4(rv[m][4 * q], rv[m][4 * q + 1], rv[m][4 * q + 2], rv[m][4 * q + 3]);
    if (lane == 0) { wval[sb][warp] = wb; widx[sb][warp] = wi; }
    __syncthreads();
    float pb = -1.0f;
    int p = kc, wq = 0;
    for (int q = 0; q < NWARP; ++q) {
      const float o = wval[sb][q];
      const int oi = widx[sb][q];
      if (o > pb || (o == pb && oi < p)) { pb = o; p = oi; wq = q; }
    }
    const bool ok = pb > 0.0f;
    if (!ok) p = kc;
    const float* r = slot + ((size_t)sb * (NWARP + 1) + wq) * B;   // the scaled pivot row
    if (t == 0) {
      pv[kc] = p;
      if (!ok) atomicExch(info, 1);
      const int a = pi[kc];
      pi[kc] = pi[p];
      pi[p] = a;
    }
#pragma unroll
    for (int q = 0; q < B / 4; ++q) {
      const float4 r4 = *reinterpret_cast<const float4*>(r + 4 * q);
      const float rq[4] = {r4.x, r4.y, r4.z, r4.w};
#pragma unroll
      for (int m = 0; m < MRT; ++m) {
        if (MRT > 1 && m > 0 && (t - lane) + NT * m >= n) continue;   // warp-uniform: no rows here
        const float f = rv[m][c];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int cc = 4 * q + u;
          if (cc == c) continue;
          rv[m][cc] = fmaf(-f, rq[u], rv[m][cc]);
        }
      }
    }
    const float rc = r[c];
#pragma unroll
    for (int m = 0; m < MRT; ++m) {
      const int i = t + NT * m;
      if (i == kc) {
#pragma unroll
        for (int cc = 0; cc < B; ++cc) rv[m][cc] = r[cc];
      } else if (i == p) {
        const float fq = ks[c];
#pragma unroll
        for (int cc = 0; cc < B; ++cc) rv[m][cc] = (cc == c) ? -fq * rc : fmaf(-fq, r[cc], ks[cc]);
      } else {
        rv[m][c] = -rv[m][c] * rc;
      }
    }
  }
}

template <int B, int MRT, int NT>
__global__ void __launch_bounds__(NT, 2) k_gj_global(long long E, int n, float* __restrict__ blocks,
                                                     int* __restrict__ piv, int* __restrict__ info) {
  constexpr int NWARP = NT / 32, CH = GJG_CH;
  const long long e = blockIdx.x;
  float* Ag = blocks + e * (long long)n * n;
  const int np = ((n + 3) & ~3) + 4;           // panel column stride (16-byte multiple)
  extern __shared__ __align__(16) float sgg[];
  float* P = sgg;                              // [B][np] the panel, memory-row order
  float* U = P + (size_t)B * np;               // [B][CH] gathered rows of a chunk
  float* slot = U + (size_t)B * CH;            // [2][NWARP + 1][B] candidate rows and row k
  int* pv = reinterpret_cast<int*>(slot + 2 * (NWARP + 1) * B);   // [n] pivot rows
  int* pi = pv + n;                            // [n] logical row -> memory row
  int* mask = pi + n;                          // [n] memory rows of the current panel's rows
  int* dest = mask + n;                        // [n] final column positions
  __shared__ float wval[2][NWARP];
  __shared__ int widx[2][NWARP];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  for (int i = t; i < n; i += NT) {
    pi[i] = i;
    mask[i] = 0;
  }
  __syncthreads();
  for (int k0 = 0; k0 < n; k0 += B) {
    const int b = min(B, n - k0);
    // 1. the panel's rows in registers
    float rv[MRT][B];
#pragma unroll
    for (int m = 0; m < MRT; ++m) {
      const int i = t + NT * m;
      const int src = i < n ? pi[i] : 0;
#pragma unroll
      for (int c = 0; c < B; ++c) rv[m][c] = (i < n && c < b) ? Ag[(long long)(k0 + c) * n + src] : 0.0f;
    }
    if (MRT == 1 && b == B) {
      gj_panel_full<B, MRT, NT>(rv, n, k0, slot, wval, widx, pv, pi, info);
    } else {
    float cv[MRT];                             // each own row's entry in the current pivot column
#pragma unroll
    for (int m = 0; m < MRT; ++m) cv[m] = rv[m][0];
    for (int c = 0; c < b; ++c) {
      const int kc = k0 + c, sb = c & 1;
      float best = -1.0f;
      int bi = n, bm = 0;
#pragma unroll
      for (int m = 0; m < MRT; ++m) {
        const int i = t + NT * m;
        if (i < n && i >= kc) {
          const float a = fabsf(cv[m]);
          if (a > best) { best = a; bi = i; bm = m; }
        }
      }
      float wb = best;
      int wi = bi;
      for (int off = 16; off > 0; off >>= 1) {
        const float o = __shfl_xor_sync(0xffffffffu, wb, off);
        const int oi = __shfl_xor_sync(0xffffffffu, wi, off);
        if (o > wb || (o == wb && oi < wi)) { wb = o; wi = oi; }
      }
      float* ws = slot + ((size_t)sb * (NWARP + 1) + warp) * B;
      float* ks = slot + ((size_t)sb * (NWARP + 1) + NWARP) * B;
      if (wi == bi && wi < n) {                // this lane holds the warp's candidate row
#pragma unroll
        for (int m = 0; m < MRT; ++m)
          if (m == bm)
#pragma unroll
            for (int cc = 0; cc < B; ++cc) ws[cc] = rv[m][cc];
      }
#pragma unroll
      for (int m = 0; m < MRT; ++m)
        if (t + NT * m == kc)
#pragma unroll
          for (int cc = 0; cc < B; ++cc) ks[cc] = rv[m][cc];
      if (lane == 0) { wval[sb][warp] = wb; widx[sb][warp] = wi; }
      __syncthreads();
      best = -1.0f;
      int p = kc, wq = 0;
      for (int q = 0; q < NWARP; ++q) {
        const float o = wval[sb][q];
        const int oi = widx[sb][q];
        if (o > best || (o == best && oi < p)) { best = o; p = oi; wq = q; }
      }
      const bool ok = best > 0.0f;
      if (!ok) p = kc;
      const float* R = ok ? slot + ((size_t)sb * (NWARP + 1) + wq) * B : ks;   // old row p
      if (t == 0) {
        pv[kc] = p;
        if (!ok) atomicExch(info, 1);
        const int a = pi[kc];
        pi[kc] = pi[p];
        pi[p] = a;
      }
      const float pinv = 1.0f / R[c];
      float cvn[MRT];
#pragma unroll
      for (int m = 0; m < MRT; ++m) cvn[m] = 0.0f;
      // every row: x <- x - x_c r with r = R / R_c, and x_c <- -x_c / R_c in the pivot column
#pragma unroll
      for (int cc = 0; cc < B; ++cc) {
        if (cc < b) {
          const float r = R[cc] * pinv;
#pragma unroll
          for (int m = 0; m < MRT; ++m) {
            const float v = (cc == c) ? -cv[m] * pinv : fmaf(-cv[m], r, rv[m][cc]);
            rv[m][cc] = v;
            if (cc == c + 1) cvn[m] = v;
          }
        }
      }
      // rows k and p after the interchange: row k is R scaled, row p is the old row k eliminated
#pragma unroll
      for (int m = 0; m < MRT; ++m) {
        const int i = t + NT * m;
        if (i == kc) {
#pragma unroll
          for (int cc = 0; cc < B; ++cc) {
            const float v = (cc == c) ? pinv : R[cc] * pinv;
            rv[m][cc] = v;
            if (cc == c + 1) cvn[m] = v;
          }
        } else if (i == p) {
          const float f = ks[c];
#pragma unroll
          for (int cc = 0; cc < B; ++cc) {
            const float v = (cc == c) ? -f * pinv : fmaf(-f, R[cc] * pinv, ks[cc]);
            rv[m][cc] = v;
            if (cc == c + 1) cvn[m] = v;
          }
        }
      }
#pragma unroll
      for (int m = 0; m < MRT; ++m) cv[m] = cvn[m];
    }
    }
    __syncthreads();                           // pi holds this panel's interchanges
    // the panel back into the block and into shared memory, at the rows' memory positions
#pragma unroll
    for (int m = 0; m < MRT; ++m) {
      const int i = t + NT * m;
      if (i < n) {
        const int dst = pi[i];
#pragma unroll
        for (int c = 0; c < B; ++c) {
          if (c < b) {
            Ag[(long long)(k0 + c) * n + dst] = rv[m][c];
            P[(size_t)c * np + dst] = rv[m][c];
          } else {
            P[(size_t)c * np + dst] = 0.0f;
          }
        }
      }
    }
    for (int c = t; c < b; c += NT) mask[pi[k0 + c]] = 1;
    __syncthreads();
    // 2. the other columns, 64 at a time
    const int ntrail = n - b;
    for (int j0 = 0; j0 < ntrail; j0 += CH) {
      const int nc = min(CH, ntrail - j0);
      for (int q = t; q < B * CH; q += NT) {
        const int c = q / CH, jc = q % CH;
        float v = 0.0f;
        if (c < b && jc < nc) {
          const int j = j0 + jc < k0 ? j0 + jc : j0 + jc + b;
          v = Ag[(long long)j * n + pi[k0 + c]];
        }
        U[q] = v;
      }
      __syncthreads();
      const int rt = (n + 3) / 4, ntile = rt * (CH / 4);
      for (int tile = t; tile < ntile; tile += NT) {
        const int r = tile % rt, sc = tile / rt;
        const int i0 = 4 * r, c0 = 4 * sc;
        if (c0 >= nc) continue;
        bool live[4];
#pragma unroll
        for (int qr = 0; qr < 4; ++qr) live[qr] = i0 + qr < n && !mask[i0 + qr];
        float acc[4][4];
#pragma unroll
        for (int qc = 0; qc < 4; ++qc) {
          const int jc = c0 + qc;
          const int j = j0 + jc < k0 ? j0 + jc : j0 + jc + b;
#pragma unroll
          for (int qr = 0; qr < 4; ++qr)
            acc[qc][qr] = (jc < nc && live[qr]) ? Ag[(long long)j * n + i0 + qr] : 0.0f;
        }
#pragma unroll 8
        for (int k = 0; k < B; ++k) {
          const float4 pk = *reinterpret_cast<const float4*>(P + (size_t)k * np + i0);
          const float4 uk = *reinterpret_cast<const float4*>(U + (size_t)k * CH + c0);
          const float pr[4] = {pk.x, pk.y, pk.z, pk.w};
          const float ur[4] = {uk.x, uk.y, uk.z, uk.w};
#pragma unroll
          for (int qc = 0; qc < 4; ++qc)
#pragma unroll
            for (int qr = 0; qr < 4; ++qr) acc[qc][qr] = fmaf(pr[qr], ur[qc], acc[qc][qr]);
        }
#pragma unroll
        for (int qc = 0; qc < 4; ++qc) {
          const int jc = c0 + qc;
          if (jc >= nc) continue;
          const int j = j0 + jc < k0 ? j0 + jc : j0 + jc + b;
#pragma unroll
          for (int qr = 0; qr < 4; ++qr)
            if (i0 + qr < n) Ag[(long long)j * n + i0 + qr] = acc[qc][qr];
        }
      }
      __syncthreads();
    }
    for (int c = t; c < b; c += NT) mask[pi[k0 + c]] = 0;
    __syncthreads();
  }
  // every column in logical row order, B columns at a time through shared memory
  float* colbuf = P;                           // [B][np]
  for (int j0 = 0; j0 < n; j0 += B) {
    const int w = min(B, n - j0);
    for (int q = t; q < w * n; q += NT) {
      const int jj = q / n, i = q - jj * n;
      colbuf[(size_t)jj * np + i] = Ag[(long long)(j0 + jj) * n + i];
    }
    __syncthreads();
    for (int q = t; q < w * n; q += NT) {
      const int jj = q / n, i = q - jj * n;
      Ag[(long long)(j0 + jj) * n + i] = colbuf[(size_t)jj * np + pi[i]];
    }
    __syncthreads();
  }
  // columns back in reverse pivot order: the composed interchange gives each column's final
  // position dest; the block is rewritten in strips of SR rows through shared memory, each strip
  // read whole before it is written (the strip, [n][SR], fits the panel buffer's B np floats)
  if (t == 0) {
    int* cur = mask;                           // (the mask is no longer needed)
    for (int i = 0; i < n; ++i) cur[i] = i;
    for (int k = n - 1; k >= 0; --k) {
      const int q = cur[k];
      cur[k] = cur[pv[k]];
      cur[pv[k]] = q;
    }
    for (int i = 0; i < n; ++i) dest[cur[i]] = i;
  }
  __syncthreads();
  constexpr int SR = B < 32 ? B : 32;
  float* strip = P;                            // [n][SR]
  for (int r0 = 0; r0 < n; r0 += SR) {
    const int rows = min(SR, n - r0);
    for (int q = t; q < n * SR; q += NT) {
      const int j = q / SR, rr = q % SR;
      if (rr < rows) strip[q] = Ag[(long long)j * n + r0 + rr];
    }
    __syncthreads();
    for (int q = t; q < n * SR; q += NT) {
      const int j = q / SR, rr = q % SR;
      if (rr < rows) Ag[(long long)dest[j] * n + r0 + rr] = strip[q];
    }
    __syncthreads();
  }
  for (int i = t; i < n; i += NT) piv[e * n + i] = pv[i];
}

// in-place Gauss-Jordan inversion with partial pivoting of one n x n column-major block per CTA
// (A[j n + i] = row i, column j). Step k: pick the pivot row in column k, interchange it with row
// k, scale row k by the reciprocal pivot (the pivot position takes the reciprocal itself) and
// eliminate column k from every other row (that column takes -a_ik / pivot). After n steps the
// columns are interchanged back in reverse pivot order, leaving A^{-1}.
template <bool SMEM>
__global__ void k_gj_inverse(long long E, int n, float* __restrict__ blocks, int* __restrict__ piv,
                             int* __restrict__ info) {
  extern __shared__ float sfr[];
  float* f = sfr;        // column k before the step
  float* r = sfr + n;    // scaled row k
  const long long e = blockIdx.x;
  float* Ag = blocks + e * (long long)n * n;
  float* A = SMEM ? sfr + 2 * n : Ag;   // the block itself, in shared memory when it fits
  if (SMEM) {
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) A[t] = Ag[t];
    __syncthreads();
  }
  int* pv = piv + e * n;
  __shared__ float sval[256];
  __shared__ int sidx[256];
  __shared__ int p_sh;
  for (int k = 0; k < n; ++k) {
    float best = -1.0f;
    int bi = k;
    for (int i = k + threadIdx.x; i < n; i += blockDim.x) {
      const float a = fabsf(A[(long long)k * n + i]);
      if (a > best) { best = a; bi = i; }
    }
    sval[threadIdx.x] = best;
    sidx[threadIdx.x] = bi;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
      if (threadIdx.x < st) {
        const float o = sval[threadIdx.x + st];
        const int oi = sidx[threadIdx.x + st];
        if (o > sval[threadIdx.x] || (o == sval[threadIdx.x] && oi < sidx[threadIdx.x])) {
          sval[threadIdx.x] = o;
          sidx[threadIdx.x] = oi;
        }
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      p_sh = sidx[0];
      pv[k] = p_sh;
      if (!(sval[0] > 0.0f)) atomicExch(info, 1);
    }
    __syncthreads();
    const int p = p_sh;
    if (p != k)
      for (int j = threadIdx.x; j < n; j += blockDim.x) {
        float* col = A + (long long)j * n;
        const float t = col[k];
        col[k] = col[p];
        col[p] = t;
      }
    __syncthreads();
    const float pinv = 1.0f / A[(long long)k * n + k];
    for (int i = threadIdx.x; i < n; i += blockDim.x) f[i] = A[(long long)k * n + i];
    for (int j = threadIdx.x; j < n; j += blockDim.x) r[j] = (j == k ? 1.0f : A[(long long)j * n + k]) * pinv;
    __syncthreads();
    // rank-1 elimination: columns by warp, rows by lane (coalesced, no index division)
    {
      const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
      for (int j = warp; j < n; j += nw) {
        float* col = A + (long long)j * n;
        const float rj = r[j];
        if (j == k) {
          for (int i = lane; i < n; i += 32) col[i] = (i == k) ? rj : -f[i] * rj;
        } else {
          for (int i = lane; i < n; i += 32) col[i] = (i == k) ? rj : fmaf(-f[i], rj, col[i]);
        }
      }
    }
    __syncthreads();
  }
  for (int k = n - 1; k >= 0; --k) {
    const int p = pv[k];
    if (p != k)
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const float t = A[(long long)k * n + i];
        A[(long long)k * n + i] = A[(long long)p * n + i];
        A[(long long)p * n + i] = t;
      }
    __syncthreads();
  }
  if (SMEM)
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) Ag[t] = A[t];
}

// y = B^{-1} x per element with the explicit FP32 inverse (column-major): coalesced over rows
__global__ void k_inv_apply(long long E, int n, const float* __restrict__ inv, const double* __restrict__ x,
                            double* __restrict__ y) {
  extern __shared__ float sx[];
  const long long e = blockIdx.x;
  const float* A = inv + e * (long long)n * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) sx[i] = (float)x[e * n + i];
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f, acc3 = 0.f;
    const float* a = A + i;
    int j = 0;
#pragma unroll 2
    for (; j + 3 < n; j += 4) {
      acc0 = fmaf(a[(long long)j * n], sx[j], acc0);
      acc1 = fmaf(a[(long long)(j + 1) * n], sx[j + 1], acc1);
      acc2 = fmaf(a[(long long)(j + 2) * n], sx[j + 2], acc2);
      acc3 = fmaf(a[(long long)(j + 3) * n], sx[j + 3], acc3);
    }
    for (; j < n; ++j) acc0 = fmaf(a[(long long)j * n], sx[j], acc0);
    y[e * n + i] = (double)((acc0 + acc1) + (acc2 + acc3));
  }
}

// FP16 copy of the FP32 inverses (DG_PC_BJ16): column j of an element's inverse is stored as
// B^{-1}[:, j] / c_j, c_j = 2^e the power of two just above the column's largest magnitude (the
// division is exact, only the FP16 rounding remains: 2^-11 relative down to 2^-14 c_j, 2^-25 c_j
// absolute below), in ld >= n halves with ld a multiple of 8 and zero padding rows. One warp per column.
__global__ void k_inv_to_half(long long ncol, int n, int ld, const float* __restrict__ inv, __half* __restrict__ H,
                              float* __restrict__ scale) {
  const long long col = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (col >= ncol) return;
  const float* a = inv + col * n;
  float mx = 0.0f;
  for (int i = lane; i < n; i += 32) mx = fmaxf(mx, fabsf(a[i]));
  for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  int ex = 0;
  if (mx > 0.0f) frexpf(mx, &ex);          // mx = f 2^ex, f in [0.5, 1)
  __half* h = H + col * ld;
  for (int i = lane; i < ld; i += 32) h[i] = __float2half_rn(i < n ? ldexpf(a[i], -ex) : 0.0f);
  if (lane == 0) scale[col] = ldexpf(1.0f, ex);
}

__device__ __forceinline__ void fma_half8(float* acc, const uint4& v, float xj) {
  const __half2* h = reinterpret_cast<const __half2*>(&v);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float2 f = __half22float2(h[k]);
    acc[2 * k] = fmaf(f.x, xj, acc[2 * k]);
    acc[2 * k + 1] = fmaf(f.y, xj, acc[2 * k + 1]);
  }
}

// y = B^{-1} x per element from the FP16 columns: y = sum_j H[:, j] (c_j x_j). Thread (rc, g) owns
// rows 8 rc .. 8 rc + 7 (one 16-byte streaming load per column) and the columns j = g (mod G); the
// G partial sums meet in shared memory. R = ld / 8 <= blockDim.x. x and y may alias.
__global__ void __launch_bounds__(256) k_inv_apply_h(long long E, int n, int ld, const __half* __restrict__ H,
                                                     const float* __restrict__ scale, const double* x, double* y) {
  extern __shared__ float sh[];
  const int R = ld >> 3;
  const int G = blockDim.x / R;
  float* sx = sh;            // [ld]
  float* part = sh + ld;     // [G][ld]
  const long long e = blockIdx.x;
  for (int i = threadIdx.x; i < n; i += blockDim.x) sx[i] = scale[e * n + i] * (float)x[e * n + i];
  __syncthreads();
  const int rc = threadIdx.x % R, g = threadIdx.x / R;
  if (g < G) {
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const uint4* Hc = reinterpret_cast<const uint4*>(H + e * (long long)n * ld) + rc;
    int j = g;
    for (; j + 3 * G < n; j += 4 * G) {
      const uint4 v0 = __ldcs(Hc + (long long)j * R);
      const uint4 v1 = __ldcs(Hc + (long long)(j + G) * R);
      const uint4 v2 = __ldcs(Hc + (long long)(j + 2 * G) * R);
      const uint4 v3 = __ldcs(Hc + (long long)(j + 3 * G) * R);
      fma_half8(acc, v0, sx[j]);
      fma_half8(acc, v1, sx[j + G]);
      fma_half8(acc, v2, sx[j + 2 * G]);
      fma_half8(acc, v3, sx[j + 3 * G]);
    }
    for (; j < n; j += G) fma_half8(acc, __ldcs(Hc + (long long)j * R), sx[j]);
#pragma unroll
    for (int q = 0; q < 8; ++q) part[g * ld + 8 * rc + q] = acc[q];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    float sum = 0.0f;
    for (int k = 0; k < G; ++k) sum += part[k * ld + i];
    y[e * n + i] = (double)sum;
  }
}

// ------------------------------------------------------------------------------------------
// solver storage
// ------------------------------------------------------------------------------------------
struct Solver {
  int restart = 0;
  long long n = 0;
  double* V = nullptr;      // [restart + 1][n]
  double* vec = nullptr;    // named work vectors below, [NV][n]
  double* partial = nullptr;
  double* hdev = nullptr;   // [2][MAXK]
  double* hhost = nullptr;  // pinned [2 MAXK + RB_MAX^2]
  double* probe = nullptr;  // [n]
  float* blocks = nullptr;  // [E][5Np][5Np]: assembled blocks, then (in place) their inverses
  int* piv = nullptr;
  int* info = nullptr;
  bool bj_ready = false;
  bool recompute_value = false;  // DG_OPT_RECOMPUTE_VALUE of the running implicit step
  __half* blocks_h = nullptr;  // [E][5Np][ld]: FP16 columns of the inverses (DG_PC_BJ16)
  float* hscale = nullptr;     // [E][5Np]: their power-of-two column scales
  int hld = 0;
  bool bj16_ready = false;
  // DG_REFRESH_LAGGED: what the current preconditioner was built for and how many steps it served
  bool lag_valid = false;
  int lag_kind = -1, lag_prec = -1, lag_steps = 0;
  double lag_caii = 0.0;
  // reduced basis (Sec. 3.2): ring of the last Newton updates, orthonormal basis W, Z = J_G W,
  // Y = P0^{-1} Z - W, C = (W^T P0^{-1} Z)^{-1} on the device, Gram Z^T Z on the host
  int rb_cap = 0, rb_count = 0, rb_head = 0, rb_r = 0, rb_kind = 0;
  bool rb_ready = false;
  double* rb_ring = nullptr;
  double* rb_W = nullptr;
  double* rb_Z = nullptr;
  double* rb_Y = nullptr;
  double* rb_C = nullptr;   // [RB_MAX * RB_MAX]
  double* rb_s = nullptr;   // [2 RB_MAX]
  std::vector<double> rb_gram;
  static constexpr int NV = 12;
  double* v(int i) { return vec + (long long)i * n; }
};

enum { VU = 0, VKNOWN, VR0, VR1, VR2, VG, VRES, VZ, VW, VDU, VTMP, VUN };

static void solver_free(Solver* S) {
  if (!S) return;
  void* ptrs[] = {S->V, S->vec, S->partial, S->hdev, S->probe, S->blocks, S->piv, S->info, S->blocks_h, S->hscale,
                  S->rb_ring, S->rb_W, S->rb_Z, S->rb_Y, S->rb_C, S->rb_s};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (S->hhost) cudaFreeHost(S->hhost);
  delete S;
}

}  // namespace dg

void dg_solver_release(dg_mesh* m) {
  dg::solver_free(m->solver);
  m->solver = nullptr;
}

namespace dg {

static int solver_get(dg_mesh* m, int restart, Solver** out) {
  if (restart < 1 || restart >= MAXK) return fail(DG_EINVAL, "gmres restart must be in 1..63");
  Solver* S = m->solver;
  if (S && S->restart >= restart) {
    *out = S;
    return DG_OK;
  }
  dg_solver_release(m);
  S = new Solver();
  S->restart = restart;
  S->n = m->ndof;
  cudaError_t err = cudaMalloc(&S->V, sizeof(double) * (size_t)(restart + 1) * S->n);
  if (err == cudaSuccess) err = cudaMalloc(&S->vec, sizeof(double) * (size_t)Solver::NV * S->n);
  if (err == cudaSuccess) err = cudaMalloc(&S->partial, sizeof(double) * RED_BLOCKS * MAXK);
  if (err == cudaSuccess) err = cudaMalloc(&S->hdev, sizeof(double) * 2 * MAXK);
  if (err == cudaSuccess) err = cudaMallocHost(&S->hhost, sizeof(double) * (2 * MAXK + RB_MAX * RB_MAX));
  if (err != cudaSuccess) {
    solver_free(S);
    return fail(DG_ENOMEM, std::string("solver storage: ") + cudaGetErrorString(err));
  }
  m->solver = S;
  *out = S;
  return DG_OK;
}

static int ensure_blocks(dg_mesh* m, Solver* S) {
  if (S->blocks) return DG_OK;
  const long long nb = 5LL * m->np;
  cudaError_t err = cudaMalloc(&S->blocks, sizeof(float) * (size_t)m->E * nb * nb);
  if (err == cudaSuccess) err = cudaMalloc(&S->piv, sizeof(int) * (size_t)m->E * nb);
  if (err == cudaSuccess) err = cudaMalloc(&S->info, sizeof(int));
  if (err == cudaSuccess) err = cudaMalloc(&S->probe, sizeof(double) * (size_t)m->ndof);
  if (err == cudaSuccess && !m->ws.qx) err = cudaMalloc(&m->ws.qx, sizeof(double) * (size_t)m->E * 90 * m->nf);
  if (err != cudaSuccess) return fail(DG_ENOMEM, std::string("block-Jacobi storage: ") + cudaGetErrorString(err));
  return DG_OK;
}

#define DG_DISPATCH_S(m, call)                                 \
  switch ((m)->n) {                                            \
    case 2: rc = Driver<2>::call; break;                       \
    case 3: rc = Driver<3>::call; break;                       \
    case 4: rc = Driver<4>::call; break;                       \
    case 5: rc = Driver<5>::call; break;                       \
    default: rc = fail(DG_EINVAL, "unsupported degree");       \
  }

static unsigned grid_for(long long n) {
  long long b = (n + 255) / 256;
  return (unsigned)(b < 4096 ? (b < 1 ? 1 : b) : 4096);
}

#define DG_K_CASES(X)                                                                                   \
  X(0) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15) X(16) X(17) X(18)    \
  X(19) X(20) X(21) X(22) X(23) X(24) X(25) X(26) X(27) X(28) X(29) X(30) X(31) X(32)
#define DG_K_CASES1(X)                                                                                  \
  X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15) X(16) X(17) X(18)         \
  X(19) X(20) X(21) X(22) X(23) X(24) X(25) X(26) X(27) X(28) X(29) X(30) X(31) X(32)

// partial rows 0..k-1 = V^T w, row k = |w|^2 (k vectors of length n, leading dimension n)
static void mdot(long long n, int k, const double* V, const double* w, double* partial, cudaStream_t s,
                 bool f32 = false) {
  if (f32 && n % 2 == 0 && k >= 1 && k <= 32) {
    const long long n2 = n / 2;
    const double2* V2 = reinterpret_cast<const double2*>(V);
    const double2* w2 = reinterpret_cast<const double2*>(w);
    switch (k) {
#define DG_MDF(K) \
  case K: k_mdot_f32<K><<<RED_BLOCKS, RED_THREADS, 0, s>>>(n2, V2, n2, w2, partial); return;
      DG_K_CASES1(DG_MDF)
#undef DG_MDF
    }
  }
  if (n % 2 == 0 && k <= 32) {
    const long long n2 = n / 2;
    const double2* V2 = reinterpret_cast<const double2*>(V);
    const double2* w2 = reinterpret_cast<const double2*>(w);
    switch (k) {
#define DG_MD(K) \
  case K: k_mdot_k<K><<<RED_BLOCKS, RED_THREADS, 0, s>>>(n2, V2, n2, w2, partial); return;
      DG_K_CASES(DG_MD)
#undef DG_MD
    }
  }
  k_mdot<<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, k, V, n, w, partial);
}

// w <- w - V h (k vectors); partial rows: DOTS ? (V^T w, |w|^2 at row k) : |w|^2 at row 0
static void update_dot(long long n, int k, const double* V, const double* h, double* w, double* partial, bool dots,
                       cudaStream_t s, bool f32 = false) {
  if (f32 && n % 2 == 0 && k >= 1 && k <= 32) {
    const long long n2 = n / 2;
    const double2* V2 = reinterpret_cast<const double2*>(V);
    double2* w2 = reinterpret_cast<double2*>(w);
    switch (k) {
#define DG_UDF(K)                                                                                 \
  case K:                                                                                         \
    if (dots) k_update_dot_f32<K, true><<<RED_BLOCKS, RED_THREADS, 0, s>>>(n2, V2, n2, h, w2, partial);  \
    else k_update_dot_f32<K, false><<<RED_BLOCKS, RED_THREADS, 0, s>>>(n2, V2, n2, h, w2, partial);      \
    return;
      DG_K_CASES1(DG_UDF)
#undef DG_UDF
    }
  }
  if (n % 2 == 0 && k >= 1 && k <= 32) {
    const long long n2 = n / 2;
    const double2* V2 = reinterpret_cast<const double2*>(V);
    double2* w2 = reinterpret_cast<double2*>(w);
    switch (k) {
#define DG_UDK(K)                                                                                            \
  case K:                                                                                                    \
    if (dots) {                                                                                              \
      const int sm = K > 8 ? (int)sizeof(double) * K * RED_THREADS : 0;                                      \
      static bool attr = false;                                                                              \
      if (!attr && sm > 0)                                                                                   \
        cudaFuncSetAttribute(k_update_dot_k<K, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);      \
      attr = true;                                                                                           \
      k_update_dot_k<K, true><<<RED_BLOCKS, RED_THREADS, sm, s>>>(n2, V2, n2, h, w2, partial);               \
    } else {                                                                                                 \
      k_update_dot_k<K, false><<<RED_BLOCKS, RED_THREADS, 0, s>>>(n2, V2, n2, h, w2, partial);               \
    }                                                                                                        \
    return;
      DG_K_CASES(DG_UDK)
#undef DG_UDK
    }
  }
#define DG_UD(KM)                                                                                        \
  do {                                                                                                   \
    if (dots) k_update_dot<KM, true><<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, k, V, n, h, w, partial);      \
    else k_update_dot<KM, false><<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, k, V, n, h, w, partial);          \
  } while (0)
  if (k <= 8) DG_UD(8);
  else if (k <= 16) DG_UD(16);
  else if (k <= 32) DG_UD(32);
  else DG_UD(64);
#undef DG_UD
}

// the two sweeps on the FP32 basis (k <= 32 vectors, n even)
static void mdot_f32v(long long n, int k, const float* V, const double* w, double* partial, cudaStream_t s) {
  const long long n2 = n / 2;
  const float2* V2 = reinterpret_cast<const float2*>(V);
  const double2* w2 = reinterpret_cast<const double2*>(w);
  switch (k) {
#define DG_MDV(K) \
  case K: k_mdot_f32v<K><<<RED_BLOCKS, RED_THREADS, 0, s>>>(n2, V2, n2, w2, partial); return;
    DG_K_CASES1(DG_MDV)
#undef DG_MDV
  }
}

static void update_dot_f32v(long long n, int k, const float* V, const double* h, double* w, double* partial, bool dots,
                            cudaStream_t s) {
  const long long n2 = n / 2;
  const float2* V2 = reinterpret_cast<const float2*>(V);
  double2* w2 = reinterpret_cast<double2*>(w);
  switch (k) {
#define DG_UDV(K)                                                                                    \
  case K:                                                                                            \
    if (dots) k_update_dot_f32v<K, true><<<RED_BLOCKS, RED_THREADS, 0, s>>>(n2, V2, n2, h, w2, partial);   \
    else k_update_dot_f32v<K, false><<<RED_BLOCKS, RED_THREADS, 0, s>>>(n2, V2, n2, h, w2, partial);       \
    return;
    DG_K_CASES1(DG_UDV)
#undef DG_UDV
  }
}

// J_G v = M v - c J_r(U) v
static int stage_matvec(dg_mesh* m, Solver* S, const double* U, double t, double c, int jv_mode, int jv_prec,
                        const double* v, double* out, cudaStream_t s, bool value_ready = false) {
  // exact tangent: one fused pass forms M v - c J_r v
  if (jv_mode == DG_JV_EXACT) return stage_jvp(m, U, v, t, c, out, jv_prec == DG_PREC_F32, s, value_ready);
  double* mv = S->v(VTMP);
  int rc = dg_mass_apply(m, v, mv, s);
  if (rc) return rc;
  rc = dg_jvp(m, U, v, t, jv_mode, 0.0, out, nullptr, s);
  if (rc) return rc;
  prof_begin(m, s, KK_BLAS);
  k_lincomb<<<grid_for(S->n), 256, 0, s>>>(S->n, 1.0, mv, -c, out, 0.0, nullptr, out);
  prof_end(m, s);
  DG_LAUNCH_CHECK("k_lincomb");
  return DG_OK;
}

// squared 2-norm on the device, read back (synchronises the stream)
static int norm2(dg_mesh* m, Solver* S, const double* x, double* out, cudaStream_t s) {
  prof_begin(m, s, KK_BLAS);
  mdot(S->n, 0, S->V, x, S->partial, s);
  k_mdot_finish<<<1, MAXK, 0, s>>>(0, S->partial, S->hdev, 0);
  prof_end(m, s);
  DG_LAUNCH_CHECK("k_mdot");
  DG_CUDA_TRY(cudaMemcpyAsync(S->hhost, S->hdev, sizeof(double), cudaMemcpyDeviceToHost, s));
  DG_CUDA_TRY(cudaStreamSynchronize(s));
  *out = std::sqrt(S->hhost[0]);
  return DG_OK;
}

// ------------------------------------------------------------------------------------------
// preconditioner
// ------------------------------------------------------------------------------------------
// exact diagonal blocks of J_G = M - c J_r(U), column j of every element per sweep, into dest
static int bj_assemble(dg_mesh* m, Solver* S, const double* U, double t, double c, float* dest, cudaStream_t s,
                       bool f32 = false) {
  int rc = ensure_blocks(m, S);
  if (rc) return rc;
  if (f32) {
    rc = ensure_f32(m);
    if (rc) return rc;
    if (!m->w32.qx) return fail(DG_EINVAL, "FP32 workspace without cross traces");
  }
  const int nb = 5 * m->np;
  double* jv = S->v(VW);
  double* mv = S->v(VTMP);
  // every probe linearises at the same U: its value plane is formed once and each sweep
  // differentiates the probe's tangent alone
  const bool once = !S->recompute_value;
  if (once) {
    rc = stage_value_plane(m, U, f32, s);
    if (rc) return rc;
  }
  for (int j = 0; j < nb; ++j) {
    prof_begin(m, s, KK_BLAS);
    k_probe<<<grid_for(S->n), 256, 0, s>>>(m->E, nb, j, S->probe);
    prof_end(m, s);
    DG_DISPATCH_S(m, jv_blockdiag(m, U, S->probe, t, jv, s, f32, once));
    if (rc) return rc;
    DG_DISPATCH_S(m, mass(m, S->probe, mv, s, f32));   // FP32 arithmetic for FP32 blocks
    if (rc) return rc;
    prof_begin(m, s, KK_BLAS);
    k_scatter_col<<<grid_for(S->n), 256, 0, s>>>(m->E, nb, j, c, mv, jv, dest);
    prof_end(m, s);
    DG_LAUNCH_CHECK("k_scatter_col");
  }
  return DG_OK;
}

static int bj_setup(dg_mesh* m, Solver* S, const double* U, double t, double c, cudaStream_t s, bool f32 = false,
                    bool half = false) {
  int rc = ensure_blocks(m, S);
  if (rc) return rc;
  const int nb = 5 * m->np;
  S->bj_ready = S->bj16_ready = false;
  if (half && !S->blocks_h) {
    S->hld = (nb + 7) / 8 * 8;
    cudaError_t err = cudaMalloc(&S->blocks_h, sizeof(__half) * (size_t)m->E * nb * S->hld);
    if (err == cudaSuccess) err = cudaMalloc(&S->hscale, sizeof(float) * (size_t)m->E * nb);
    if (err != cudaSuccess) return fail(DG_ENOMEM, std::string("FP16 block storage: ") + cudaGetErrorString(err));
  }
  DG_CUDA_TRY(cudaMemsetAsync(S->info, 0, sizeof(int), s));
  rc = bj_assemble(m, S, U, t, c, S->blocks, s, f32);
  if (rc) return rc;
  prof_begin(m, s, KK_LU);
  const size_t gj_smem = sizeof(float) * (2 * nb + (size_t)nb * nb);
  // blocked kernels: panel width B, MRT rows per thread, NT threads; the shared memory holds the
  // panel [B][np], a chunk of the other columns [B][GJG_CH], the pivot slots and four index arrays
  auto gj_blocked = [&](auto kern, int B, int NT) -> int {
    const int np = ((nb + 3) & ~3) + 4;
    const size_t smem = sizeof(float) * ((size_t)B * np + (size_t)B * GJG_CH + 2 * (NT / 32 + 1) * (size_t)B) +
                        sizeof(int) * 4 * (size_t)nb;
    DG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<(unsigned)m->E, NT, smem, s>>>(m->E, nb, S->blocks, S->piv, S->info);
    return DG_OK;
  };
  // panel widths measured per size: 16 for 135^2 (98,304 blocks: 56 ms against 68 ms at 32), 24
  // for 320^2 (221,184 blocks: 1.03 s against 1.17 s), 32 above
  if (nb > 64 && nb <= 160) {
    // one row per thread (160 threads): several blocks per SM overlap their panel steps
    rc = gj_blocked(k_gj_global<16, 1, 160>, 16, 160);
  } else if (gj_smem <= 200 * 1024) {
    cudaFuncSetAttribute(k_gj_inverse<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gj_smem);
    k_gj_inverse<true><<<(unsigned)m->E, 256, gj_smem, s>>>(m->E, nb, S->blocks, S->piv, S->info);
  } else if (nb <= 320) {
    // one row per thread (320 threads), the panel steps unrolled
    rc = gj_blocked(k_gj_global<24, 1, 320>, 24, 320);
  } else if (nb <= 640) {
    rc = gj_blocked(k_gj_global<GJG_B, 2, 320>, GJG_B, 320);   // two rows per thread
  } else if (nb <= 768) {
    rc = gj_blocked(k_gj_global<GJG_B, 3, 256>, GJG_B, 256);   // three rows per thread
  } else {
    k_gj_inverse<false><<<(unsigned)m->E, 256, sizeof(float) * 2 * nb, s>>>(m->E, nb, S->blocks, S->piv, S->info);
  }
  prof_end(m, s);
  if (rc) return rc;
  DG_LAUNCH_CHECK("k_gj_inverse");
  int info = 0;
  DG_CUDA_TRY(cudaMemcpyAsync(&info, S->info, sizeof(int), cudaMemcpyDeviceToHost, s));
  DG_CUDA_TRY(cudaStreamSynchronize(s));
  if (info) return fail(DG_ENAN, "block-Jacobi: a zero pivot in a diagonal block");
  S->bj_ready = true;
  if (half) {
    const long long ncol = m->E * (long long)nb;
    prof_begin(m, s, KK_LU);
    k_inv_to_half<<<(unsigned)((ncol + 7) / 8), 256, 0, s>>>(ncol, nb, S->hld, S->blocks, S->blocks_h, S->hscale);
    prof_end(m, s);
    DG_LAUNCH_CHECK("k_inv_to_half");
    S->bj16_ready = true;
  }
  return DG_OK;
}

// ------------------------------------------------------------------------------------------
// reduced-basis preconditioner and initial guess (Sec. 3.2)
// ------------------------------------------------------------------------------------------
static int ensure_rb(Solver* S, int cap) {
  if (cap < 1 || cap > RB_MAX) return fail(DG_EINVAL, "reduced basis size must be in 1..16");
  if (S->rb_ring && S->rb_cap >= cap) return DG_OK;
  double** bufs[] = {&S->rb_ring, &S->rb_W, &S->rb_Z, &S->rb_Y};
  for (double** b : bufs)
    if (*b) {
      cudaFree(*b);
      *b = nullptr;
    }
  S->rb_count = S->rb_head = S->rb_r = 0;
  S->rb_ready = false;
  cudaError_t err = cudaSuccess;
  for (double** b : bufs)
    if (err == cudaSuccess) err = cudaMalloc(b, sizeof(double) * (size_t)cap * S->n);
  if (err == cudaSuccess && !S->rb_C) err = cudaMalloc(&S->rb_C, sizeof(double) * RB_MAX * RB_MAX);
  if (err == cudaSuccess && !S->rb_s) err = cudaMalloc(&S->rb_s, sizeof(double) * 2 * RB_MAX);
  if (err != cudaSuccess) return fail(DG_ENOMEM, std::string("reduced-basis storage: ") + cudaGetErrorString(err));
  S->rb_cap = cap;
  return DG_OK;
}

static void rb_push(Solver* S, const double* du, cudaStream_t s) {
  cudaMemcpyAsync(S->rb_ring + (long long)S->rb_head * S->n, du, sizeof(double) * S->n, cudaMemcpyDeviceToDevice, s);
  S->rb_head = (S->rb_head + 1) % S->rb_cap;
  if (S->rb_count < S->rb_cap) ++S->rb_count;
}

// rows 0..k-1 of V^T x and |x|^2 into host out[0..k] (one synchronisation)
static int host_dots(dg_mesh* m, Solver* S, const double* V, int k, const double* x, double* out, cudaStream_t s) {
  prof_begin(m, s, KK_BLAS);
  mdot(S->n, k, V, x, S->partial, s);
  k_mdot_finish<<<1, MAXK, 0, s>>>(k, S->partial, S->hdev, 0);
  prof_end(m, s);
  DG_LAUNCH_CHECK("k_mdot");
  DG_CUDA_TRY(cudaMemcpyAsync(S->hhost, S->hdev, sizeof(double) * (k + 1), cudaMemcpyDeviceToHost, s));
  DG_CUDA_TRY(cudaStreamSynchronize(s));
  std::memcpy(out, S->hhost, sizeof(double) * (k + 1));
  return DG_OK;
}

// in-place inverse of an r x r row-major matrix (Gauss-Jordan, partial pivoting); false if singular
static bool small_inverse(std::vector<double>& A, int r) {
  std::vector<int> perm(r);
  for (int i = 0; i < r; ++i) perm[i] = i;
  double amax = 0.0;
  for (double v : A) amax = std::max(amax, std::fabs(v));
  if (!(amax > 0.0) || !std::isfinite(amax)) return false;
  for (int k = 0; k < r; ++k) {
    int p = k;
    for (int i = k + 1; i < r; ++i)
      if (std::fabs(A[i * r + k]) > std::fabs(A[p * r + k])) p = i;
    if (!(std::fabs(A[p * r + k]) > 1e-14 * amax)) return false;
    if (p != k) {
      for (int j = 0; j < r; ++j) std::swap(A[k * r + j], A[p * r + j]);
      std::swap(perm[k], perm[p]);
    }
    const double d = 1.0 / A[k * r + k];
    A[k * r + k] = 1.0;
    for (int j = 0; j < r; ++j) A[k * r + j] *= d;
    for (int i = 0; i < r; ++i) {
      if (i == k) continue;
      const double f = A[i * r + k];
      A[i * r + k] = 0.0;
      for (int j = 0; j < r; ++j) A[i * r + j] -= f * A[k * r + j];
    }
  }
  // columns come out permuted like the rows were: undo
  std::vector<double> B(A);
  for (int i = 0; i < r; ++i)
    for (int k = 0; k < r; ++k) A[i * r + perm[k]] = B[i * r + k];
  return true;
}

static int base_solve(dg_mesh* m, Solver* S, int kind, const double* x, double* y, cudaStream_t s);

// orthonormalise the window (newest first) into W; updates within 1e-10 of the span of the kept
// ones are dropped
static int rb_orthonormalise(dg_mesh* m, Solver* S, cudaStream_t s) {
  const long long n = S->n;
  int r = 0;
  std::vector<double> d(RB_MAX + 1);
  for (int q = 0; q < S->rb_count; ++q) {
    const int slot = ((S->rb_head - 1 - q) % S->rb_cap + S->rb_cap) % S->rb_cap;
    double* w = S->rb_W + (long long)r * n;
    DG_CUDA_TRY(cudaMemcpyAsync(w, S->rb_ring + (long long)slot * n, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    int rc = host_dots(m, S, S->rb_W, r, w, d.data(), s);   // h1 = W^T w and |w|^2
    if (rc) return rc;
    const double n0 = d[r];
    double nf = n0;
    if (r > 0) {   // h1 is in hdev[0..r-1]
      prof_begin(m, s, KK_BLAS);
      update_dot(n, r, S->rb_W, S->hdev, w, S->partial, true, s);
      k_mdot_finish<<<1, MAXK, 0, s>>>(r - 1, S->partial, S->hdev + MAXK, 0);
      update_dot(n, r, S->rb_W, S->hdev + MAXK, w, S->partial, false, s);
      k_mdot_finish<<<1, MAXK, 0, s>>>(0, S->partial, S->hdev + 2 * MAXK - 1, 0);
      prof_end(m, s);
      DG_LAUNCH_CHECK("rb orthonormalise");
      DG_CUDA_TRY(cudaMemcpyAsync(S->hhost, S->hdev + 2 * MAXK - 1, sizeof(double), cudaMemcpyDeviceToHost, s));
      DG_CUDA_TRY(cudaStreamSynchronize(s));
      nf = S->hhost[0];
    } else {
      S->hhost[0] = n0;
      DG_CUDA_TRY(cudaMemcpyAsync(S->hdev + 2 * MAXK - 1, S->hhost, sizeof(double), cudaMemcpyHostToDevice, s));
    }
    if (!std::isfinite(n0) || !std::isfinite(nf)) return fail(DG_ENAN, "reduced basis: non-finite Newton update");
    if (!(n0 > 0.0) || !(nf > 1e-20 * n0)) continue;
    prof_begin(m, s, KK_BLAS);
    k_scale_dev<<<grid_for(n), 256, 0, s>>>(n, w, S->hdev + 2 * MAXK - 1, w);
    prof_end(m, s);
    DG_LAUNCH_CHECK("k_scale_dev");
    ++r;
  }
  S->rb_r = r;
  return DG_OK;
}

// W, Z = J_G W, Y = P0^{-1} Z - W, C = (W^T P0^{-1} Z)^{-1} and Z^T Z at state U
static int rb_build(dg_mesh* m, Solver* S, int kind, const double* U, double t, double c, int jv_mode, int jv_prec,
                    cudaStream_t s);

static int rb_apply(dg_mesh* m, Solver* S, const double* x, double* y, cudaStream_t s) {
  if (!S->rb_ready) return fail(DG_EINVAL, "reduced-basis preconditioner used before it was built");
  int rc = base_solve(m, S, S->rb_kind, x, y, s);
  if (rc) return rc;
  const int r = S->rb_r;
  if (r == 0) return DG_OK;
  const long long n = S->n;
  prof_begin(m, s, KK_PRECOND);
  mdot(n, r, S->rb_W, y, S->partial, s);
  k_mdot_finish<<<1, MAXK, 0, s>>>(r - 1, S->partial, S->rb_s, 0);
  k_small_matvec<<<1, 32, 0, s>>>(r, S->rb_C, S->rb_s, S->rb_s + RB_MAX);
  k_maxpy<<<grid_for(n), 256, 0, s>>>(n, r, S->rb_Y, n, S->rb_s + RB_MAX, y);
  prof_end(m, s);
  DG_LAUNCH_CHECK("rb apply");
  return DG_OK;
}

// x0 = W a, a = argmin |b - Z a|, and r0 = b - Z a; false (nothing written) when the space is
// empty or the guess does not reduce |b|
static int rb_guess(dg_mesh* m, Solver* S, const double* b, double* x0, double* r0, bool* used, cudaStream_t s) {
  *used = false;
  const int r = S->rb_r;
  if (!S->rb_ready || r == 0) return DG_OK;
  const long long n = S->n;
  std::vector<double> g(r + 1);
  int rc = host_dots(m, S, S->rb_Z, r, b, g.data(), s);
  if (rc) return rc;
  const double bb = g[r];
  std::vector<double> Gi(S->rb_gram);
  if (!small_inverse(Gi, r)) return DG_OK;
  std::vector<double> a(r, 0.0);
  for (int i = 0; i < r; ++i)
    for (int j = 0; j < r; ++j) a[i] += Gi[i * r + j] * g[j];
  // |b - Z a|^2 = |b|^2 - 2 a^T g + a^T G a, checked on the device below
  std::memcpy(S->hhost, a.data(), sizeof(double) * r);
  DG_CUDA_TRY(cudaMemcpyAsync(S->rb_s, S->hhost, sizeof(double) * r, cudaMemcpyHostToDevice, s));
  DG_CUDA_TRY(cudaMemcpyAsync(r0, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  prof_begin(m, s, KK_BLAS);
  k_maxpy<<<grid_for(n), 256, 0, s>>>(n, r, S->rb_Z, n, S->rb_s, r0);
  prof_end(m, s);
  DG_LAUNCH_CHECK("k_maxpy");
  double rr = 0.0;
  rc = host_dots(m, S, S->rb_Z, 0, r0, &rr, s);
  if (rc) return rc;
  if (!std::isfinite(rr) || !(rr < bb)) return DG_OK;
  std::memcpy(S->hhost, a.data(), sizeof(double) * r);
  DG_CUDA_TRY(cudaMemcpyAsync(S->rb_s, S->hhost, sizeof(double) * r, cudaMemcpyHostToDevice, s));
  prof_begin(m, s, KK_BLAS);
  k_combine<<<grid_for(n), 256, 0, s>>>(n, r, S->rb_W, n, S->rb_s, x0);
  prof_end(m, s);
  DG_LAUNCH_CHECK("k_combine");
  *used = true;
  return DG_OK;
}

static int precond_apply(dg_mesh* m, Solver* S, int kind, const double* x, double* y, cudaStream_t s) {
  if (kind == DG_PC_NONE) {
    if (x != y) DG_CUDA_TRY(cudaMemcpyAsync(y, x, sizeof(double) * S->n, cudaMemcpyDeviceToDevice, s));
    return DG_OK;
  }
  if (kind == DG_PC_BJ) {
    if (!S->bj_ready) return fail(DG_EINVAL, "block-Jacobi preconditioner used before dg_precond_setup");
    const int nb = 5 * m->np;
    prof_begin(m, s, KK_PRECOND);
    k_inv_apply<<<(unsigned)m->E, nb <= 256 ? (nb + 31) / 32 * 32 : 256, sizeof(float) * nb, s>>>(m->E, nb, S->blocks, x, y);
    prof_end(m, s);
    DG_LAUNCH_CHECK("k_inv_apply");
    return DG_OK;
  }
  if (kind == DG_PC_BJ16) {
    if (!S->bj16_ready) return fail(DG_EINVAL, "FP16 block-Jacobi preconditioner used before dg_precond_setup");
    const int nb = 5 * m->np, R = S->hld / 8;
    if (R > 256) return fail(DG_EINVAL, "FP16 block-Jacobi: blocks larger than 2048");
    const int G = 256 / R;
    prof_begin(m, s, KK_PRECOND);
    k_inv_apply_h<<<(unsigned)m->E, 256, sizeof(float) * (size_t)S->hld * (1 + G), s>>>(m->E, nb, S->hld,
                                                                                      S->blocks_h, S->hscale, x, y);
    prof_end(m, s);
    DG_LAUNCH_CHECK("k_inv_apply_h");
    return DG_OK;
  }
  if (kind == DG_PC_MLP) {
    prof_begin(m, s, KK_PRECOND);
    const int rc = mlp_apply(m, x, y, s);
    prof_end(m, s);
    return rc;
  }
  if (kind == DG_PC_RB || kind == DG_PC_RB_BJ) {
    if (S->rb_ready && S->rb_kind != kind) return fail(DG_EINVAL, "reduced basis was built for the other base");
    return rb_apply(m, S, x, y, s);
  }
  return fail(DG_EINVAL, "unknown preconditioner kind");
}

// base of the reduced-basis preconditioner: M^{-1} (DG_PC_RB) or block-Jacobi (DG_PC_RB_BJ)
static int base_solve(dg_mesh* m, Solver* S, int kind, const double* x, double* y, cudaStream_t s) {
  if (kind == DG_PC_RB_BJ) return precond_apply(m, S, DG_PC_BJ, x, y, s);
  return dg_mass_inverse_apply(m, x, y, s);
}

static int rb_build(dg_mesh* m, Solver* S, int kind, const double* U, double t, double c, int jv_mode, int jv_prec,
                    cudaStream_t s) {
  const long long n = S->n;
  S->rb_ready = false;
  S->rb_kind = kind;
  int rc = rb_orthonormalise(m, S, s);
  if (rc) return rc;
  int r = S->rb_r;
  for (int j = 0; j < r; ++j) {
    double* Zj = S->rb_Z + (long long)j * n;
    double* Yj = S->rb_Y + (long long)j * n;
    rc = stage_matvec(m, S, U, t, c, jv_mode, jv_prec, S->rb_W + (long long)j * n, Zj, s);
    if (rc) return rc;
    rc = base_solve(m, S, kind, Zj, Yj, s);
    if (rc) return rc;
    prof_begin(m, s, KK_BLAS);
    k_lincomb<<<grid_for(n), 256, 0, s>>>(n, 1.0, Yj, -1.0, S->rb_W + (long long)j * n, 0.0, nullptr, Yj);
    prof_end(m, s);
    DG_LAUNCH_CHECK("k_lincomb");
  }
  std::vector<double> Cm((size_t)r * r), G((size_t)r * r), d(RB_MAX + 1);
  for (int j = 0; j < r; ++j) {
    rc = host_dots(m, S, S->rb_W, r, S->rb_Y + (long long)j * n, d.data(), s);   // W^T Y_j
    if (rc) return rc;
    for (int i = 0; i < r; ++i) Cm[i * r + j] = d[i] + (i == j ? 1.0 : 0.0);
    rc = host_dots(m, S, S->rb_Z, r, S->rb_Z + (long long)j * n, d.data(), s);   // Z^T Z_j
    if (rc) return rc;
    for (int i = 0; i < r; ++i) G[i * r + j] = d[i];
  }
  if (r > 0 && !small_inverse(Cm, r)) r = 0;   // singular reduced operator: base alone
  S->rb_r = r;
  S->rb_gram = G;
  if (r > 0) {
    std::memcpy(S->hhost, Cm.data(), sizeof(double) * r * r);
    DG_CUDA_TRY(cudaMemcpyAsync(S->rb_C, S->hhost, sizeof(double) * r * r, cudaMemcpyHostToDevice, s));
    DG_CUDA_TRY(cudaStreamSynchronize(s));
  }
  S->rb_ready = true;
  return DG_OK;
}

// (re)build the preconditioner of kind at state U
static int pc_setup(dg_mesh* m, Solver* S, int kind, const double* U, double t, double c, cudaStream_t s, bool f32) {
  dg::NvtxRange nvtx_range_("preconditioner setup");
  S->lag_valid = false;   // a lagged preconditioner is only reused as its own step built it
  if (kind == DG_PC_BJ || kind == DG_PC_RB_BJ) return bj_setup(m, S, U, t, c, s, f32);
  if (kind == DG_PC_BJ16) return bj_setup(m, S, U, t, c, s, f32, true);
  if (kind == DG_PC_MLP) return mlp_setup(m, U, c, s);
  return DG_OK;
}

// ------------------------------------------------------------------------------------------
// GMRES(restart), right preconditioned: solves J_G x = b to ||b - J_G x|| <= tol ||b||
// ------------------------------------------------------------------------------------------
// x0_given: x holds an initial guess and the work vector VRES already holds b - J_G x
static int gmres(dg_mesh* m, Solver* S, const dg_solver_opts& o, const double* U, double t, double c,
                 const double* b, double* x, int* iters, cudaStream_t s, bool x0_given = false) {
  dg::NvtxRange nvtx_range_("GMRES");
  const long long n = S->n;
  const int R = o.gmres_restart;
  double* V = S->V;
  double* w = S->v(VW);
  double* z = S->v(VZ);
  double* r = S->v(VRES);
  double bnorm = 0.0;
  int rc = norm2(m, S, b, &bnorm, s);
  if (rc) return rc;
  if (!std::isfinite(bnorm)) return fail(DG_ENAN, "GMRES: non-finite right-hand side");
  if (!x0_given || bnorm == 0.0) DG_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(double) * n, s));
  if (bnorm == 0.0) return DG_OK;
  // every operator application of this solve linearises at the same U: its value plane (Gauss
  // values, traces, LDG gradient) is formed once; the preconditioners do not touch the workspace
  bool vr = false;
  if (o.jv_mode == DG_JV_EXACT && !(o.flags & DG_OPT_RECOMPUTE_VALUE)) {
    rc = stage_value_plane(m, U, o.jv_prec == DG_PREC_F32, s);
    if (rc) return rc;
    vr = true;
  }
  std::vector<double> H((size_t)(R + 1) * R), cs(R), sn(R), g(R + 1), y(R);
  const bool f32gs = o.jv_prec == DG_PREC_F32;
  // the mixed-precision solve stores its Krylov basis in FP32 (in the same allocation)
  const bool f32basis = f32gs && n % 2 == 0 && R + 1 <= 32 && o.gmres_rtol >= 1e-6;
  float* Vf = reinterpret_cast<float*>(V);
  for (int cycle = 0; cycle < o.max_restarts; ++cycle) {
    // r = b - A x
    if (cycle == 0) {
      if (!x0_given) DG_CUDA_TRY(cudaMemcpyAsync(r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    } else {
      rc = stage_matvec(m, S, U, t, c, o.jv_mode, o.jv_prec, x, w, s, vr);
      if (rc) return rc;
      k_lincomb<<<grid_for(n), 256, 0, s>>>(n, 1.0, b, -1.0, w, 0.0, nullptr, r);
      DG_LAUNCH_CHECK("k_lincomb");
    }
    double beta = 0.0;
    rc = norm2(m, S, r, &beta, s);
    if (rc) return rc;
    if (!std::isfinite(beta)) return fail(DG_ENAN, "GMRES: non-finite residual");
    if (beta <= o.gmres_rtol * bnorm) return DG_OK;
    if (f32basis) k_scale_to_f32<<<grid_for(n), 256, 0, s>>>(n, r, 1.0 / beta, nullptr, Vf);
    else k_lincomb<<<grid_for(n), 256, 0, s>>>(n, 1.0 / beta, r, 0.0, nullptr, 0.0, nullptr, V);
    DG_LAUNCH_CHECK("k_lincomb");
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int kdone = 0;
    bool converged = false;
    for (int k = 0; k < R; ++k) {
      if (f32basis) {
        prof_begin(m, s, KK_BLAS);
        k_widen<<<grid_for(n), 256, 0, s>>>(n, Vf + (long long)k * n, S->v(VTMP));
        prof_end(m, s);
        DG_LAUNCH_CHECK("k_widen");
        rc = precond_apply(m, S, o.precond, S->v(VTMP), z, s);
      } else {
        rc = precond_apply(m, S, o.precond, V + (long long)k * n, z, s);
      }
      if (rc) return rc;
      rc = stage_matvec(m, S, U, t, c, o.jv_mode, o.jv_prec, z, w, s, vr);
      if (rc) return rc;
      // classical Gram-Schmidt twice; h and the norm stay on the device until one read-back. With
      // the FP32 Jv the projections are formed in FP32 arithmetic (orthogonality to ~1e-7, far
      // below the Krylov tolerance), the basis, the subtraction from w and the norms stay FP64.
      prof_begin(m, s, KK_BLAS);
      // h1 = V^T w; w -= V h1 fused with h2 = V^T w; w -= V h2 fused with |w|^2
      if (f32basis) {
        mdot_f32v(n, k + 1, Vf, w, S->partial, s);
        k_mdot_finish<<<1, MAXK, 0, s>>>(k, S->partial, S->hdev, 0);
        update_dot_f32v(n, k + 1, Vf, S->hdev, w, S->partial, true, s);
        k_mdot_finish<<<1, MAXK, 0, s>>>(k, S->partial, S->hdev + MAXK, 0);
        update_dot_f32v(n, k + 1, Vf, S->hdev + MAXK, w, S->partial, false, s);
        k_mdot_finish<<<1, MAXK, 0, s>>>(0, S->partial, S->hdev + MAXK + k + 1, 0);
        k_scale_to_f32<<<grid_for(n), 256, 0, s>>>(n, w, 0.0, S->hdev + MAXK + k + 1, Vf + (long long)(k + 1) * n);
      } else {
        mdot(n, k + 1, V, w, S->partial, s, f32gs);
        k_mdot_finish<<<1, MAXK, 0, s>>>(k, S->partial, S->hdev, 0);
        update_dot(n, k + 1, V, S->hdev, w, S->partial, true, s, f32gs);
        k_mdot_finish<<<1, MAXK, 0, s>>>(k, S->partial, S->hdev + MAXK, 0);
        update_dot(n, k + 1, V, S->hdev + MAXK, w, S->partial, false, s, f32gs);
        k_mdot_finish<<<1, MAXK, 0, s>>>(0, S->partial, S->hdev + MAXK + k + 1, 0);
        k_scale_dev<<<grid_for(n), 256, 0, s>>>(n, w, S->hdev + MAXK + k + 1, V + (long long)(k + 1) * n);
      }
      prof_end(m, s);
      DG_LAUNCH_CHECK("arnoldi");
      DG_CUDA_TRY(cudaMemcpyAsync(S->hhost, S->hdev, sizeof(double) * 2 * MAXK, cudaMemcpyDeviceToHost, s));
      DG_CUDA_TRY(cudaStreamSynchronize(s));
      double* Hk = &H[(size_t)k * (R + 1)];   // column k, rows 0..k+1
      for (int j = 0; j <= k; ++j) Hk[j] = S->hhost[j] + S->hhost[MAXK + j];
      Hk[k + 1] = std::sqrt(S->hhost[MAXK + k + 1]);
      for (int j = 0; j < k; ++j) {
        const double t1 = cs[j] * Hk[j] + sn[j] * Hk[j + 1];
        Hk[j + 1] = -sn[j] * Hk[j] + cs[j] * Hk[j + 1];
        Hk[j] = t1;
      }
      const double den = std::hypot(Hk[k], Hk[k + 1]);
      if (!std::isfinite(den)) return fail(DG_ENAN, "GMRES: non-finite Arnoldi coefficient");
      cs[k] = den > 0 ? Hk[k] / den : 1.0;
      sn[k] = den > 0 ? Hk[k + 1] / den : 0.0;
      Hk[k] = den;
      Hk[k + 1] = 0.0;
      g[k + 1] = -sn[k] * g[k];
      g[k] = cs[k] * g[k];
      ++*iters;
      kdone = k + 1;
      if (std::fabs(g[k + 1]) <= o.gmres_rtol * bnorm) {
        converged = true;
        break;
      }
    }
    for (int i = kdone - 1; i >= 0; --i) {
      double sum = g[i];
      for (int j = i + 1; j < kdone; ++j) sum -= H[(size_t)j * (R + 1) + i] * y[j];
      y[i] = sum / H[(size_t)i * (R + 1) + i];
    }
    std::memcpy(S->hhost, y.data(), sizeof(double) * kdone);
    DG_CUDA_TRY(cudaMemcpyAsync(S->hdev, S->hhost, sizeof(double) * kdone, cudaMemcpyHostToDevice, s));
    if (f32basis) k_combine_f32v<<<grid_for(n), 256, 0, s>>>(n, kdone, Vf, n, S->hdev, r);
    else k_combine<<<grid_for(n), 256, 0, s>>>(n, kdone, V, n, S->hdev, r);
    DG_LAUNCH_CHECK("k_combine");
    rc = precond_apply(m, S, o.precond, r, z, s);
    if (rc) return rc;
    k_lincomb<<<grid_for(n), 256, 0, s>>>(n, 1.0, x, 1.0, z, 0.0, nullptr, x);
    DG_LAUNCH_CHECK("k_lincomb");
    if (converged) return DG_OK;
  }
  return fail(DG_ENOTCONV, "GMRES did not reach its tolerance within max_restarts cycles");
}

}  // namespace dg

using namespace dg;

extern "C" void dg_solver_opts_default(dg_solver_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->stages = 3;
  o->gmres_restart = 30;
  o->max_restarts = 10;
  o->max_newton = 20;
  o->precond = DG_PC_NONE;
  o->precond_refresh = DG_REFRESH_STEP;
  o->jv_mode = DG_JV_EXACT;
  o->newton_rtol = 1e-8;
  o->gmres_rtol = 1e-3;
  o->abs_floor = 1e-14;
  o->rb_size = 8;
  o->refresh_every = 3;
}

extern "C" int dg_precond_setup(dg_mesh* mesh, int32_t kind, const double* u, double t, double dt_aii,
                                void* stream) {
  if (!mesh || !u) return fail(DG_EINVAL, "dg_precond_setup: null argument");
  Solver* S = nullptr;
  int rc = solver_get(mesh, mesh->solver ? mesh->solver->restart : 30, &S);
  if (rc) return rc;
  if (kind == DG_PC_NONE) return DG_OK;
  if (kind == DG_PC_BJ) return bj_setup(mesh, S, u, t, dt_aii, (cudaStream_t)stream);
  if (kind == DG_PC_BJ16) return bj_setup(mesh, S, u, t, dt_aii, (cudaStream_t)stream, false, true);
  if (kind == DG_PC_MLP) return mlp_setup(mesh, u, dt_aii, (cudaStream_t)stream);
  return fail(DG_EINVAL, "dg_precond_setup: unknown kind");
}

extern "C" int dg_precond_apply(dg_mesh* mesh, int32_t kind, const double* x, double* y, void* stream) {
  if (!mesh || !x || !y) return fail(DG_EINVAL, "dg_precond_apply: null argument");
  if (!mesh->solver) return fail(DG_EINVAL, "dg_precond_apply: no preconditioner was set up");
  return precond_apply(mesh, mesh->solver, kind, x, y, (cudaStream_t)stream);
}

extern "C" int dg_rb_load(dg_mesh* mesh, const double* w, int32_t r, const double* u, double t, double dt_aii,
                          int32_t base, void* stream) {
  if (!mesh || !u || (r > 0 && !w) || r < 0 || r > RB_MAX) return fail(DG_EINVAL, "dg_rb_load: bad argument");
  if (base != DG_PC_RB && base != DG_PC_RB_BJ) return fail(DG_EINVAL, "dg_rb_load: base must be DG_PC_RB or DG_PC_RB_BJ");
  Solver* S = nullptr;
  int rc = solver_get(mesh, mesh->solver ? mesh->solver->restart : 30, &S);
  if (rc) return rc;
  rc = ensure_rb(S, std::max(r, std::max(S->rb_cap, 1)));
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  S->rb_count = S->rb_head = 0;
  for (int j = 0; j < r; ++j) rb_push(S, w + (long long)j * S->n, s);
  if (base == DG_PC_RB_BJ) {
    rc = bj_setup(mesh, S, u, t, dt_aii, s);
    if (rc) return rc;
  }
  return rb_build(mesh, S, base, u, t, dt_aii, DG_JV_EXACT, DG_PREC_F64, s);
}

extern "C" int dg_rb_initial_guess(dg_mesh* mesh, const double* b, double* x0, void* stream) {
  if (!mesh || !b || !x0) return fail(DG_EINVAL, "dg_rb_initial_guess: null argument");
  Solver* S = mesh->solver;
  if (!S || !S->rb_ready) return fail(DG_EINVAL, "dg_rb_initial_guess: no reduced basis was built");
  cudaStream_t s = (cudaStream_t)stream;
  bool used = false;
  int rc = rb_guess(mesh, S, b, x0, S->v(VRES), &used, s);
  if (rc) return rc;
  if (!used) DG_CUDA_TRY(cudaMemsetAsync(x0, 0, sizeof(double) * S->n, s));
  DG_CUDA_TRY(cudaStreamSynchronize(s));
  return DG_OK;
}

extern "C" int dg_rb_reset(dg_mesh* mesh) {
  if (!mesh) return fail(DG_EINVAL, "dg_rb_reset: null argument");
  Solver* S = mesh->solver;
  if (S) {
    S->rb_count = S->rb_head = S->rb_r = 0;
    S->rb_ready = false;
  }
  return DG_OK;
}

extern "C" int dg_implicit_step(dg_mesh* mesh, double* u, double t, double dt, const dg_solver_opts* opts,
                                dg_step_stats* stats, void* stream) {
  dg::NvtxRange nvtx_range_("dg_implicit_step");
  if (!mesh || !u || !opts) return fail(DG_EINVAL, "dg_implicit_step: null argument");
  const dg_solver_opts o = *opts;
  cudaStream_t s = (cudaStream_t)stream;
  const auto t0 = std::chrono::steady_clock::now();
  double A[3][3], c[3];
  int rc = dirk_tableau(o.stages, A, c);
  if (rc) return rc;
  if (o.max_newton < 1 || o.max_restarts < 1) return fail(DG_EINVAL, "dg_implicit_step: bad limits");
  if (o.precond < DG_PC_NONE || o.precond > DG_PC_BJ16) return fail(DG_EINVAL, "dg_implicit_step: unknown precond");
  if (o.precond_refresh < DG_REFRESH_STEP || o.precond_refresh > DG_REFRESH_LAGGED ||
      (o.precond_refresh == DG_REFRESH_LAGGED && o.refresh_every < 1))
    return fail(DG_EINVAL, "dg_implicit_step: bad preconditioner refresh");
  const bool rb = o.precond == DG_PC_RB || o.precond == DG_PC_RB_BJ;
  Solver* S = nullptr;
  rc = solver_get(mesh, o.gmres_restart, &S);
  if (rc) return rc;
  if (rb) {
    rc = ensure_rb(S, o.rb_size);
    if (rc) return rc;
  }
  struct FlagScope {   // the flag holds for this step's block assemblies only
    Solver* S;
    ~FlagScope() { S->recompute_value = false; }
  } flag_scope{S};
  S->recompute_value = (o.flags & DG_OPT_RECOMPUTE_VALUE) != 0;
  dg_step_stats st;
  std::memset(&st, 0, sizeof(st));
  const long long n = S->n;
  double* U = S->v(VU);
  double* known = S->v(VKNOWN);
  double* G = S->v(VG);
  double* res = S->v(VRES);
  double* dU = S->v(VDU);
  double* un = S->v(VUN);
  double* R[3] = {S->v(VR0), S->v(VR1), S->v(VR2)};
  DG_CUDA_TRY(cudaMemcpyAsync(un, u, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  DG_CUDA_TRY(cudaMemcpyAsync(U, u, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  double* Mun = S->v(VTMP);
  auto finish = [&](int code) {
    if (code != DG_OK) S->lag_valid = false;   // a failed step rebuilds its preconditioner next time
    st.status = code;
    st.wall_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (stats) *stats = st;
    return code;
  };
  bool build_now = o.precond != DG_PC_NONE && o.precond_refresh == DG_REFRESH_STEP;
  if (o.precond != DG_PC_NONE && o.precond_refresh == DG_REFRESH_LAGGED) {
    build_now = !(S->lag_valid && S->lag_kind == o.precond && S->lag_prec == o.jv_prec &&
                  S->lag_caii == dt * A[0][0] && S->lag_steps < o.refresh_every);
    if (build_now) S->lag_valid = false;
    else ++S->lag_steps;
  }
  if (build_now) {
    const auto p0 = std::chrono::steady_clock::now();
    rc = pc_setup(mesh, S, o.precond, un, t + c[0] * dt, dt * A[0][0], s, o.jv_prec == DG_PREC_F32);
    st.precond_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - p0).count();
    if (rc) return finish(rc);
    if (o.precond_refresh == DG_REFRESH_LAGGED) {
      S->lag_valid = true;
      S->lag_kind = o.precond;
      S->lag_prec = o.jv_prec;
      S->lag_caii = dt * A[0][0];
      S->lag_steps = 1;
    }
  }
  for (int i = 0; i < o.stages; ++i) {
    dg::NvtxRange stage_range("DIRK stage");
    const double ti = t + c[i] * dt, ci = dt * A[i][i];
    // known = M u_n + dt sum_{j<i} a_ij R_j
    rc = dg_mass_apply(mesh, un, Mun, s);
    if (rc) return finish(rc);
    k_lincomb<<<grid_for(n), 256, 0, s>>>(n, 1.0, Mun, i > 0 ? dt * A[i][0] : 0.0, i > 0 ? R[0] : nullptr,
                                          i > 1 ? dt * A[i][1] : 0.0, i > 1 ? R[1] : nullptr, known);
    DG_LAUNCH_CHECK("k_lincomb");
    if (o.precond != DG_PC_NONE && o.precond_refresh == DG_REFRESH_STAGE) {
      const auto p0 = std::chrono::steady_clock::now();
      rc = pc_setup(mesh, S, o.precond, U, ti, ci, s, o.jv_prec == DG_PREC_F32);
      st.precond_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - p0).count();
      if (rc) return finish(rc);
    }
    double g0 = -1.0;
    bool done = false;
    for (int it = 0; it <= o.max_newton; ++it) {
      rc = dg_residual(mesh, U, nullptr, ti, res, s);
      if (rc) return finish(rc);
      rc = dg_mass_apply(mesh, U, G, s);
      if (rc) return finish(rc);
      double mun = 0.0;
      rc = norm2(mesh, S, G, &mun, s);
      if (rc) return finish(rc);
      k_lincomb<<<grid_for(n), 256, 0, s>>>(n, 1.0, G, -1.0, known, -ci, res, G);
      DG_LAUNCH_CHECK("k_lincomb");
      double gn = 0.0;
      rc = norm2(mesh, S, G, &gn, s);
      if (rc) return finish(rc);
      if (!std::isfinite(gn)) return finish(fail(DG_ENAN, "Newton: non-finite stage residual"));
      if (st.n_hist < DG_STATS_HIST) st.res_hist[st.n_hist++] = gn;
      if (g0 < 0) g0 = gn;
      if (gn <= o.newton_rtol * g0 || gn <= o.abs_floor * mun) {
        st.newton_iters[i] = it;
        done = true;
        break;
      }
      if (it == o.max_newton) break;
      if (o.precond != DG_PC_NONE && o.precond_refresh == DG_REFRESH_NEWTON) {
        const auto p0 = std::chrono::steady_clock::now();
        rc = pc_setup(mesh, S, o.precond, U, ti, ci, s, o.jv_prec == DG_PREC_F32);
        st.precond_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - p0).count();
        if (rc) return finish(rc);
      }
      // dU = -J_G^{-1} G
      k_lincomb<<<grid_for(n), 256, 0, s>>>(n, -1.0, G, 0.0, nullptr, 0.0, nullptr, G);
      DG_LAUNCH_CHECK("k_lincomb");
      bool x0 = false;
      if (rb) {   // reduced basis of the last Newton updates at the current iterate, and its guess
        const auto p0 = std::chrono::steady_clock::now();
        rc = rb_build(mesh, S, o.precond, U, ti, ci, o.jv_mode, o.jv_prec, s);
        if (!rc) rc = rb_guess(mesh, S, G, dU, S->v(VRES), &x0, s);
        st.precond_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - p0).count();
        if (rc) return finish(rc);
      }
      int gits = 0;
      rc = gmres(mesh, S, o, U, ti, ci, G, dU, &gits, s, x0);
      st.gmres_iters[i] += gits;
      if (rc) return finish(rc);
      if (rb) rb_push(S, dU, s);
      k_lincomb<<<grid_for(n), 256, 0, s>>>(n, 1.0, U, 1.0, dU, 0.0, nullptr, U);
      DG_LAUNCH_CHECK("k_lincomb");
    }
    if (!done) return finish(fail(DG_ENOTCONV, "Newton did not reach its tolerance"));
    if (i + 1 < o.stages) {
      rc = dg_residual(mesh, U, nullptr, ti, R[i], s);
      if (rc) return finish(rc);
    }
  }
  DG_CUDA_TRY(cudaMemcpyAsync(u, U, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  DG_CUDA_TRY(cudaStreamSynchronize(s));
  return finish(DG_OK);
}

extern "C" int dg_dirk_tableau(int32_t stages, double* a, double* c) {
  if (!a || !c) return fail(DG_EINVAL, "dg_dirk_tableau: null argument");
  double A[3][3], cc[3];
  int rc = dirk_tableau(stages, A, cc);
  if (rc) return rc;
  for (int i = 0; i < stages; ++i) {
    c[i] = cc[i];
    for (int j = 0; j < stages; ++j) a[i * stages + j] = A[i][j];
  }
  return DG_OK;
}

extern "C" int dg_block_assemble(dg_mesh* mesh, const double* u, double t, double dt_aii, float* out,
                                 void* stream) {
  if (!mesh || !u || !out) return fail(DG_EINVAL, "dg_block_assemble: null argument");
  Solver* S = nullptr;
  int rc = solver_get(mesh, mesh->solver ? mesh->solver->restart : 30, &S);
  if (rc) return rc;
  return bj_assemble(mesh, S, u, t, dt_aii, out, (cudaStream_t)stream);
}
