// Learned element preconditioner: features, network forward/backward, training and application.
//
// The paper has no learned component; this is the library's learned right preconditioner for
// the GMRES of Sec. 3.2. Per element e, with S_e the diagonal of the element mass matrix (one
// value per node, shared by the five variables) and Bs_e = S^{-1/2} B_e S^{-1/2} the scaled exact
// diagonal block of J_G, a two-hidden-layer SiLU network maps features x_e to
// D = 1 + o[:n], U = o[n : n + n r], V = o[n + n r :] (row-major n x r) and the preconditioner is
// P_e = S^{-1/2} (diag(D) + U V^T) S^{-1/2}. Training minimises
// L = mean_b || Bs_b (diag(D) + U V^T) - I ||_F^2 / n with Adam; the gradients are written out by
// hand (GEMM kernels for the layers, one CTA per sample for the loss). The loss measures P as a
// RIGHT inverse (|| Bs P - I ||) because GMRES applies it on the right.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "dg_internal.cuh"

namespace dg {

// ------------------------------------------------------------------------------------------
// FP32 tiled GEMM: C[m][n] = sum_k A(m,k) B(k,n) (+ beta C) (+ bias[n]); optional SiLU copy
// A(m,k) = TA ? A[k lda + m] : A[m lda + k];  B(k,n) = TB ? B[n ldb + k] : B[k ldb + n]
// ------------------------------------------------------------------------------------------
constexpr int GBM = 64, GBN = 64, GBK = 16;

template <bool TA, bool TB>
__global__ void __launch_bounds__(256) k_gemm(int M, int N, int K, const float* __restrict__ A, int lda,
                                              const float* __restrict__ B, int ldb, float* __restrict__ C, int ldc,
                                              float beta, const float* __restrict__ bias, float* __restrict__ H) {
  __shared__ float As[GBK][GBM + 4];
  __shared__ float Bs[GBK][GBN + 4];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += GBK) {
    for (int t = tid; t < GBK * GBM; t += 256) {
      int kk, mm;
      if (TA) { mm = t % GBM; kk = t / GBM; } else { kk = t % GBK; mm = t / GBK; }
      const int gm = m0 + mm, gk = k0 + kk;
      float v = 0.f;
      if (gm < M && gk < K) v = TA ? A[(long long)gk * lda + gm] : A[(long long)gm * lda + gk];
      As[kk][mm] = v;
    }
    for (int t = tid; t < GBK * GBN; t += 256) {
      int kk, nn;
      if (TB) { kk = t % GBK; nn = t / GBK; } else { nn = t % GBN; kk = t / GBN; }
      const int gn = n0 + nn, gk = k0 + kk;
      float v = 0.f;
      if (gn < N && gk < K) v = TB ? B[(long long)gn * ldb + gk] : B[(long long)gk * ldb + gn];
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GBK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gm = m0 + ty * 4 + i, gn = n0 + tx * 4 + j;
      if (gm < M && gn < N) {
        float v = acc[i][j];
        if (beta != 0.f) v += beta * C[(long long)gm * ldc + gn];
        if (bias) v += bias[gn];
        C[(long long)gm * ldc + gn] = v;
        if (H) H[(long long)gm * ldc + gn] = v / (1.f + expf(-v));
      }
    }
}

template <bool TA, bool TB>
static void gemm(cudaStream_t s, int M, int N, int K, const float* A, int lda, const float* B, int ldb, float* C,
                 int ldc, float beta = 0.f, const float* bias = nullptr, float* H = nullptr) {
  dim3 grid((N + GBN - 1) / GBN, (M + GBM - 1) / GBM);
  k_gemm<TA, TB><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, beta, bias, H);
}

// dz = dh * silu'(z) in place on dh
__global__ void k_silu_back(long long n, const float* __restrict__ z, float* __restrict__ dh) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float s = 1.f / (1.f + expf(-z[i]));
    dh[i] *= s * (1.f + z[i] * (1.f - s));
  }
}

// column sums of a [rows][cols] matrix (bias gradients), fixed order
__global__ void k_colsum(int rows, int cols, const float* __restrict__ X, float* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  float s = 0.f;
  for (int r = 0; r < rows; ++r) s += X[(long long)r * cols + c];
  out[c] = s;
}

// ------------------------------------------------------------------------------------------
// loss and output gradient, one CTA per sample, for P as a right inverse: R = Bs P - I (never
// stored), P = diag(D) + U V^T, G = scale Bs^T R:
//   W = Bs U (n x r);  R_ij = Bs_ij D_j + sum_k W_ik V_jk - delta_ij
//   dD_j = scale sum_i Bs_ij R_ij;  dV = scale R^T W;  Z = R V;  dU = scale Bs^T Z
// ------------------------------------------------------------------------------------------
constexpr int MLP_MAXR = 32;

__global__ void k_loss_grad(int nb, int n, int r, const float* __restrict__ out, const float* __restrict__ Bs,
                            float scale, float* __restrict__ dout, double* __restrict__ loss_part) {
  extern __shared__ float sm[];
  const int b = blockIdx.x;
  const int no = n + 2 * n * r;
  const float* o = out + (long long)b * no;
  const float* Bm = Bs + (long long)b * n * n;       // row-major
  float* D = sm;                                     // [n]
  float* U = D + n;                                  // [n][r]
  float* V = U + n * r;                              // [n][r]
  float* Wm = V + n * r;                             // [n][r]  Bs U
  float* Z = Wm + n * r;                             // [n][r]  R V
  __shared__ double red[256];
  for (int i = threadIdx.x; i < n; i += blockDim.x) D[i] = 1.f + o[i];
  for (int i = threadIdx.x; i < n * r; i += blockDim.x) {
    U[i] = o[n + i];
    V[i] = o[n + n * r + i];
  }
  __syncthreads();
  // W[i][k] = sum_j Bs_ij U_jk (threads over rows)
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    float acc[MLP_MAXR];
    for (int k = 0; k < r; ++k) acc[k] = 0.f;
    for (int j = 0; j < n; ++j) {
      const float bij = Bm[(long long)i * n + j];
      for (int k = 0; k < r; ++k) acc[k] = fmaf(bij, U[j * r + k], acc[k]);
    }
    for (int k = 0; k < r; ++k) Wm[i * r + k] = acc[k];
  }
  __syncthreads();
  // rows: loss and Z = R V
  double lsum = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    float z[MLP_MAXR];
    for (int k = 0; k < r; ++k) z[k] = 0.f;
    for (int j = 0; j < n; ++j) {
      float rij = Bm[(long long)i * n + j] * D[j] - (i == j ? 1.f : 0.f);
      for (int k = 0; k < r; ++k) rij = fmaf(Wm[i * r + k], V[j * r + k], rij);
      lsum += (double)rij * rij;
      for (int k = 0; k < r; ++k) z[k] = fmaf(rij, V[j * r + k], z[k]);
    }
    for (int k = 0; k < r; ++k) Z[i * r + k] = z[k];
  }
  __syncthreads();
  // columns: dD_j, dV_j = sum_i R_ij W_i, dU_j = sum_i Bs_ij Z_i
  float* g = dout + (long long)b * no;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    float dv[MLP_MAXR], du[MLP_MAXR];
    for (int k = 0; k < r; ++k) {
      dv[k] = 0.f;
      du[k] = 0.f;
    }
    float dd = 0.f;
    for (int i = 0; i < n; ++i) {
      const float bij = Bm[(long long)i * n + j];
      float rij = bij * D[j] - (i == j ? 1.f : 0.f);
      for (int k = 0; k < r; ++k) rij = fmaf(Wm[i * r + k], V[j * r + k], rij);
      dd = fmaf(bij, rij, dd);
      for (int k = 0; k < r; ++k) {
        dv[k] = fmaf(rij, Wm[i * r + k], dv[k]);
        du[k] = fmaf(bij, Z[i * r + k], du[k]);
      }
    }
    g[j] = scale * dd;
    for (int k = 0; k < r; ++k) {
      g[n + j * r + k] = scale * du[k];
      g[n + n * r + j * r + k] = scale * dv[k];
    }
  }
  red[threadIdx.x] = lsum;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) loss_part[b] = red[0];
}

__global__ void k_adam(long long n, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float c1, float c2, float eps) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// ------------------------------------------------------------------------------------------
// features and mass-diagonal scaling (one CTA per element, threads over nodes)
//   x = [varrho_i - mean, v_x, v_y, v_z, T_i / mean(T) - 1 (per node), mean(varrho)/10,
//        log mean(T), log(dt a_ii), log h_1, log h_2, log h_3]
//   S_i = sum_g (w |J|)_g phi_i(g)^2 (diagonal of the element mass matrix)
// ------------------------------------------------------------------------------------------
__global__ void k_features(long long E, int n, const double* __restrict__ u, const double* __restrict__ x,
                           const double* __restrict__ geo, const Ops* __restrict__ ops, double dt_aii,
                           float* __restrict__ feat, float* __restrict__ sdiag) {
  const int np = n * n * n;
  const long long e = blockIdx.x;
  const double* ue = u + e * 5 * np;
  const int nin = 5 * np + 6;
  float* f = feat + e * nin;
  __shared__ double s_r[256], s_t[256];
  double rsum = 0.0, tsum = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) {
    const double isr = exp(-0.5 * ue[i]);
    rsum += ue[i];
    tsum += ue[4 * np + i] * isr;
  }
  s_r[threadIdx.x] = rsum;
  s_t[threadIdx.x] = tsum;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) {
      s_r[threadIdx.x] += s_r[threadIdx.x + st];
      s_t[threadIdx.x] += s_t[threadIdx.x + st];
    }
    __syncthreads();
  }
  const double rmean = s_r[0] / np, tmean = s_t[0] / np;
  for (int i = threadIdx.x; i < np; i += blockDim.x) {
    const double isr = exp(-0.5 * ue[i]);
    f[i] = (float)(ue[i] - rmean);
    f[np + i] = (float)(ue[np + i] * isr);
    f[2 * np + i] = (float)(ue[2 * np + i] * isr);
    f[3 * np + i] = (float)(ue[3 * np + i] * isr);
    f[4 * np + i] = (float)(ue[4 * np + i] * isr / tmean - 1.0);
    // mass diagonal: sum over Gauss points of w|J| phi_i^2, phi_i(g) = B[g1][a] B[g2][b] B[g3][c]
    const int a = i % n, bb = (i / n) % n, c = i / (n * n);
    double s = 0.0;
    for (int g = 0; g < np; ++g) {
      const int g1 = g % n, g2 = (g / n) % n, g3 = g / (n * n);
      const double ph = ops->B[g1 * n + a] * ops->B[g2 * n + bb] * ops->B[g3 * n + c];
      s += geo[e * 10 * np + 9 * np + g] * ph * ph;
    }
    sdiag[e * np + i] = (float)s;
  }
  if (threadIdx.x == 0) {
    const double* xe = x + e * 3 * np;
    f[5 * np] = (float)(rmean / 10.0);
    f[5 * np + 1] = (float)log(tmean);
    f[5 * np + 2] = (float)log(dt_aii);
    const int corner[3] = {n - 1, (n - 1) * n, (n - 1) * n * n};
    for (int d = 0; d < 3; ++d) {
      double h2 = 0.0;
      for (int k = 0; k < 3; ++k) {
        const double dx = xe[k * np + corner[d]] - xe[k * np];
        h2 += dx * dx;
      }
      f[5 * np + 3 + d] = (float)(0.5 * log(h2));
    }
  }
}

// Bs[e][i][j] = block[e][j][i] / sqrt(S_i S_j) (row-major), node of DOF i = i mod np
__global__ void k_scale_blocks(long long E, int np, const float* __restrict__ blocks, const float* __restrict__ sdiag,
                               float* __restrict__ Bs) {
  const int nb = 5 * np;
  const long long e = blockIdx.x;
  const float* Bc = blocks + e * (long long)nb * nb;
  float* Bo = Bs + e * (long long)nb * nb;
  for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
    const int i = t / nb, j = t % nb;
    Bo[t] = Bc[(long long)j * nb + i] * rsqrtf(sdiag[e * np + i % np] * sdiag[e * np + j % np]);
  }
}

// y = S^{-1/2} (D * xs + U (V^T xs)), xs = S^{-1/2} x, per element (FP64 in and out)
__global__ void k_mlp_apply(long long E, int np, int r, const float* __restrict__ out, const float* __restrict__ sdiag,
                            const double* __restrict__ x, double* __restrict__ y) {
  extern __shared__ float sx[];
  __shared__ float tk[MLP_MAXR];
  const int nb = 5 * np, no = nb + 2 * nb * r;
  const long long e = blockIdx.x;
  const float* o = out + e * no;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) sx[i] = (float)x[e * nb + i] * rsqrtf(sdiag[e * np + i % np]);
  __syncthreads();
  // t_k = sum_i V[i][k] xs_i: one warp per k
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, nw = blockDim.x / 32;
  for (int k = warp; k < r; k += nw) {
    float acc = 0.f;
    for (int i = lane; i < nb; i += 32) acc = fmaf(o[nb + nb * r + i * r + k], sx[i], acc);
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if (lane == 0) tk[k] = acc;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    float v = (1.f + o[i]) * sx[i];
    for (int k = 0; k < r; ++k) v = fmaf(o[nb + i * r + k], tk[k], v);
    y[e * nb + i] = (double)(v * rsqrtf(sdiag[e * np + i % np]));
  }
}

// ------------------------------------------------------------------------------------------
// state
// ------------------------------------------------------------------------------------------
struct Mlp {
  int n_in = 0, hidden = 0, n = 0, rank = 0, n_out = 0;
  long long n_params = 0;
  float* params = nullptr;    // W1 b1 W2 b2 W3 b3
  float* grads = nullptr;
  float* adam_m = nullptr;
  float* adam_v = nullptr;
  long long adam_t = 0;
  // training set
  long long cap = 0, count = 0;
  float* X = nullptr;         // [cap][n_in]
  float* Bs = nullptr;        // [cap][n][n]
  // scratch for a batch and for inference
  int batch_cap = 0;
  float *z1 = nullptr, *h1 = nullptr, *z2 = nullptr, *h2 = nullptr, *o = nullptr, *dout = nullptr, *dh = nullptr;
  double* loss_part = nullptr;
  // inference outputs for every element
  float* feat = nullptr;      // [E][n_in]
  float* sdiag = nullptr;     // [E][np]
  float* outE = nullptr;      // [E][n_out]
  bool ready = false;
  float* W1() { return params; }
  float* b1() { return W1() + (long long)hidden * n_in; }
  float* W2() { return b1() + hidden; }
  float* b2() { return W2() + (long long)hidden * hidden; }
  float* W3() { return b2() + hidden; }
  float* b3() { return W3() + (long long)n_out * hidden; }
};

static void mlp_free(Mlp* M) {
  if (!M) return;
  void* p[] = {M->params, M->grads, M->adam_m, M->adam_v, M->X, M->Bs, M->z1, M->h1, M->z2, M->h2, M->o, M->dout,
               M->dh, M->loss_part, M->feat, M->sdiag, M->outE};
  for (void* q : p)
    if (q) cudaFree(q);
  delete M;
}

// SplitMix64 (Steele, Lea & Flood 2014) for the initial weights
static inline uint64_t splitmix(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

static int ensure_batch(Mlp* M, int batch) {
  if (M->batch_cap >= batch) return DG_OK;
  float** bufs[] = {&M->z1, &M->h1, &M->z2, &M->h2, &M->o, &M->dout, &M->dh};
  for (float** b : bufs)
    if (*b) { cudaFree(*b); *b = nullptr; }
  if (M->loss_part) cudaFree(M->loss_part);
  const size_t H = (size_t)batch * M->hidden, O = (size_t)batch * M->n_out;
  cudaError_t err = cudaMalloc(&M->z1, H * 4);
  if (err == cudaSuccess) err = cudaMalloc(&M->h1, H * 4);
  if (err == cudaSuccess) err = cudaMalloc(&M->z2, H * 4);
  if (err == cudaSuccess) err = cudaMalloc(&M->h2, H * 4);
  if (err == cudaSuccess) err = cudaMalloc(&M->o, O * 4);
  if (err == cudaSuccess) err = cudaMalloc(&M->dout, O * 4);
  if (err == cudaSuccess) err = cudaMalloc(&M->dh, (H > (size_t)batch * M->n_in ? H : (size_t)batch * M->n_in) * 4);
  if (err == cudaSuccess) err = cudaMalloc(&M->loss_part, sizeof(double) * batch);
  if (err != cudaSuccess) return fail(DG_ENOMEM, std::string("MLP batch storage: ") + cudaGetErrorString(err));
  M->batch_cap = batch;
  return DG_OK;
}

static int forward(Mlp* M, const float* X, int nb, float* out, cudaStream_t s) {
  gemm<false, true>(s, nb, M->hidden, M->n_in, X, M->n_in, M->W1(), M->n_in, M->z1, M->hidden, 0.f, M->b1(), M->h1);
  gemm<false, true>(s, nb, M->hidden, M->hidden, M->h1, M->hidden, M->W2(), M->hidden, M->z2, M->hidden, 0.f, M->b2(),
                    M->h2);
  gemm<false, true>(s, nb, M->n_out, M->hidden, M->h2, M->hidden, M->W3(), M->hidden, out, M->n_out, 0.f, M->b3(),
                    nullptr);
  DG_LAUNCH_CHECK("mlp forward");
  return DG_OK;
}

// loss over nb samples (X, Bs on the device) and parameter gradients into M->grads
static int loss_grad(Mlp* M, const float* X, const float* Bs, int nb, double* loss, cudaStream_t s) {
  int rc = ensure_batch(M, nb);
  if (rc) return rc;
  rc = forward(M, X, nb, M->o, s);
  if (rc) return rc;
  const size_t smem = sizeof(float) * (M->n + 4 * M->n * M->rank);
  if (smem > 200 * 1024) return fail(DG_EINVAL, "MLP block too large for the loss kernel");
  cudaFuncSetAttribute(k_loss_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const float scale = 2.f / ((float)nb * (float)M->n);
  k_loss_grad<<<nb, 256, smem, s>>>(nb, M->n, M->rank, M->o, Bs, scale, M->dout, M->loss_part);
  DG_LAUNCH_CHECK("k_loss_grad");
  const int H = M->hidden, I = M->n_in, O = M->n_out;
  float* gW1 = M->grads;
  float* gb1 = gW1 + (long long)H * I;
  float* gW2 = gb1 + H;
  float* gb2 = gW2 + (long long)H * H;
  float* gW3 = gb2 + H;
  float* gb3 = gW3 + (long long)O * H;
  // output layer
  gemm<true, false>(s, O, H, nb, M->dout, O, M->h2, H, gW3, H);
  k_colsum<<<(O + 255) / 256, 256, 0, s>>>(nb, O, M->dout, gb3);
  // dh2 = dout W3, dz2 = dh2 * silu'(z2)
  gemm<false, false>(s, nb, H, O, M->dout, O, M->W3(), H, M->dh, H);
  k_silu_back<<<1024, 256, 0, s>>>((long long)nb * H, M->z2, M->dh);
  gemm<true, false>(s, H, H, nb, M->dh, H, M->h1, H, gW2, H);
  k_colsum<<<(H + 255) / 256, 256, 0, s>>>(nb, H, M->dh, gb2);
  // dh1 = dz2 W2 (into z2's buffer, no longer needed), dz1 = dh1 * silu'(z1)
  gemm<false, false>(s, nb, H, H, M->dh, H, M->W2(), H, M->z2, H);
  k_silu_back<<<1024, 256, 0, s>>>((long long)nb * H, M->z1, M->z2);
  gemm<true, false>(s, H, I, nb, M->z2, H, X, I, gW1, I);
  k_colsum<<<(H + 255) / 256, 256, 0, s>>>(nb, H, M->z2, gb1);
  DG_LAUNCH_CHECK("mlp backward");
  if (loss) {
    std::vector<double> part(nb);
    DG_CUDA_TRY(cudaMemcpyAsync(part.data(), M->loss_part, sizeof(double) * nb, cudaMemcpyDeviceToHost, s));
    DG_CUDA_TRY(cudaStreamSynchronize(s));
    double L = 0.0;
    for (double v : part) L += v;
    *loss = L / ((double)nb * M->n);
  }
  return DG_OK;
}

}  // namespace dg

void dg_mlp_release(dg_mesh* m) {
  dg::mlp_free(m->mlp);
  m->mlp = nullptr;
}

using namespace dg;

extern "C" int dg_mlp_init(dg_mesh* mesh, int32_t hidden, int32_t rank, int64_t max_samples, uint64_t seed) {
  if (!mesh || hidden < 1 || rank < 1 || rank > MLP_MAXR || max_samples < 0)
    return fail(DG_EINVAL, "dg_mlp_init: bad argument");
  if (mesh->n > 4) return fail(DG_EINVAL, "dg_mlp_init: the learned preconditioner supports p <= 3");
  dg_mlp_release(mesh);
  Mlp* M = new Mlp();
  M->n = 5 * mesh->np;
  M->n_in = 5 * mesh->np + 6;
  M->hidden = hidden;
  M->rank = rank;
  M->n_out = M->n + 2 * M->n * rank;
  M->n_params = (long long)hidden * M->n_in + hidden + (long long)hidden * hidden + hidden +
                (long long)M->n_out * hidden + M->n_out;
  M->cap = max_samples;
  const long long E = mesh->E;
  cudaError_t err = cudaMalloc(&M->params, sizeof(float) * M->n_params);
  if (err == cudaSuccess) err = cudaMalloc(&M->grads, sizeof(float) * M->n_params);
  if (err == cudaSuccess) err = cudaMalloc(&M->adam_m, sizeof(float) * M->n_params);
  if (err == cudaSuccess) err = cudaMalloc(&M->adam_v, sizeof(float) * M->n_params);
  if (err == cudaSuccess && max_samples) err = cudaMalloc(&M->X, sizeof(float) * max_samples * M->n_in);
  if (err == cudaSuccess && max_samples) err = cudaMalloc(&M->Bs, sizeof(float) * max_samples * M->n * M->n);
  if (err == cudaSuccess) err = cudaMalloc(&M->feat, sizeof(float) * E * M->n_in);
  if (err == cudaSuccess) err = cudaMalloc(&M->sdiag, sizeof(float) * E * mesh->np);
  if (err == cudaSuccess) err = cudaMalloc(&M->outE, sizeof(float) * E * M->n_out);
  if (err != cudaSuccess) {
    mlp_free(M);
    return fail(DG_ENOMEM, std::string("dg_mlp_init: ") + cudaGetErrorString(err));
  }
  // initial weights: uniform(-a, a), a = sqrt(6 / fan_in) for the hidden layers (SiLU), 0.1 of that
  // for the output layer, zero biases (the initial preconditioner is close to the mass scaling)
  std::vector<float> h(M->n_params, 0.f);
  long long off = 0, idx = 0;
  auto fill = [&](long long count, int fan_in, float gain) {
    const float a = gain * std::sqrt(6.f / (float)fan_in);
    for (long long k = 0; k < count; ++k) {
      const double u01 = (double)(splitmix(seed, (uint64_t)idx++) >> 11) * (1.0 / 9007199254740992.0);
      h[off + k] = (float)((2.0 * u01 - 1.0) * a);
    }
    off += count;
  };
  fill((long long)hidden * M->n_in, M->n_in, 1.f);
  off += hidden;
  fill((long long)hidden * hidden, hidden, 1.f);
  off += hidden;
  fill((long long)M->n_out * hidden, hidden, 0.1f);
  err = cudaMemcpy(M->params, h.data(), sizeof(float) * M->n_params, cudaMemcpyHostToDevice);
  if (err == cudaSuccess) err = cudaMemset(M->adam_m, 0, sizeof(float) * M->n_params);
  if (err == cudaSuccess) err = cudaMemset(M->adam_v, 0, sizeof(float) * M->n_params);
  if (err != cudaSuccess) {
    mlp_free(M);
    return fail(DG_ECUDA, std::string("dg_mlp_init: ") + cudaGetErrorString(err));
  }
  mesh->mlp = M;
  return DG_OK;
}

extern "C" int dg_mlp_sizes(dg_mesh* mesh, int64_t* n_params, int32_t* n_in, int32_t* n_out, int64_t* n_samples) {
  if (!mesh || !mesh->mlp) return fail(DG_EINVAL, "dg_mlp_sizes: no network");
  if (n_params) *n_params = mesh->mlp->n_params;
  if (n_in) *n_in = mesh->mlp->n_in;
  if (n_out) *n_out = mesh->mlp->n_out;
  if (n_samples) *n_samples = mesh->mlp->count;
  return DG_OK;
}

extern "C" int dg_mlp_params(dg_mesh* mesh, float* out, const float* in, void* stream) {
  if (!mesh || !mesh->mlp) return fail(DG_EINVAL, "dg_mlp_params: no network");
  Mlp* M = mesh->mlp;
  cudaStream_t s = (cudaStream_t)stream;
  if (out) DG_CUDA_TRY(cudaMemcpyAsync(out, M->params, sizeof(float) * M->n_params, cudaMemcpyDeviceToDevice, s));
  if (in) {
    DG_CUDA_TRY(cudaMemcpyAsync(M->params, in, sizeof(float) * M->n_params, cudaMemcpyDeviceToDevice, s));
    M->ready = false;
  }
  return DG_OK;
}

// features (and mass diagonal) of every element at state u
static int mlp_features(dg_mesh* mesh, const double* u, double dt_aii, cudaStream_t s) {
  Mlp* M = mesh->mlp;
  k_features<<<(unsigned)mesh->E, 128, 0, s>>>(mesh->E, mesh->n, u, mesh->x, mesh->geo, mesh->d_ops, dt_aii, M->feat,
                                               M->sdiag);
  DG_LAUNCH_CHECK("k_features");
  return DG_OK;
}

extern "C" int dg_mlp_features(dg_mesh* mesh, const double* u, double dt_aii, float* feat, float* sdiag, void* stream) {
  if (!mesh || !mesh->mlp || !u) return fail(DG_EINVAL, "dg_mlp_features: bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  int rc = mlp_features(mesh, u, dt_aii, s);
  if (rc) return rc;
  Mlp* M = mesh->mlp;
  if (feat) DG_CUDA_TRY(cudaMemcpyAsync(feat, M->feat, sizeof(float) * mesh->E * M->n_in, cudaMemcpyDeviceToDevice, s));
  if (sdiag) DG_CUDA_TRY(cudaMemcpyAsync(sdiag, M->sdiag, sizeof(float) * mesh->E * mesh->np, cudaMemcpyDeviceToDevice, s));
  return DG_OK;
}

extern "C" int dg_mlp_harvest(dg_mesh* mesh, const double* u, double t, double dt_aii, int32_t stride,
                              int64_t* n_samples, void* stream) {
  if (!mesh || !mesh->mlp || !u || stride < 1) return fail(DG_EINVAL, "dg_mlp_harvest: bad argument");
  Mlp* M = mesh->mlp;
  cudaStream_t s = (cudaStream_t)stream;
  const long long E = mesh->E, nb = M->n;
  float* blocks = nullptr;
  DG_CUDA_TRY(cudaMalloc(&blocks, sizeof(float) * E * nb * nb));
  int rc = dg_block_assemble(mesh, u, t, dt_aii, blocks, stream);
  if (rc == DG_OK) rc = mlp_features(mesh, u, dt_aii, s);
  float* scaled = nullptr;
  if (rc == DG_OK && cudaMalloc(&scaled, sizeof(float) * E * nb * nb) != cudaSuccess) rc = fail(DG_ENOMEM, "harvest");
  if (rc == DG_OK) {
    k_scale_blocks<<<(unsigned)E, 256, 0, s>>>(E, mesh->np, blocks, M->sdiag, scaled);
    for (long long e = 0; e < E && M->count < M->cap; e += stride) {
      cudaMemcpyAsync(M->X + M->count * M->n_in, M->feat + e * M->n_in, sizeof(float) * M->n_in,
                      cudaMemcpyDeviceToDevice, s);
      cudaMemcpyAsync(M->Bs + M->count * nb * nb, scaled + e * nb * nb, sizeof(float) * nb * nb,
                      cudaMemcpyDeviceToDevice, s);
      M->count++;
    }
    cudaError_t err = cudaStreamSynchronize(s);
    if (err != cudaSuccess) rc = fail(DG_ECUDA, std::string("dg_mlp_harvest: ") + cudaGetErrorString(err));
  }
  cudaFree(blocks);
  if (scaled) cudaFree(scaled);
  if (n_samples) *n_samples = M->count;
  return rc;
}

extern "C" int dg_mlp_loss_grad(dg_mesh* mesh, const float* X, const float* Bs, int32_t nb, double* loss, float* grad,
                                void* stream) {
  if (!mesh || !mesh->mlp || !X || !Bs || nb < 1) return fail(DG_EINVAL, "dg_mlp_loss_grad: bad argument");
  Mlp* M = mesh->mlp;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = loss_grad(M, X, Bs, nb, loss, s);
  if (rc) return rc;
  if (grad) DG_CUDA_TRY(cudaMemcpyAsync(grad, M->grads, sizeof(float) * M->n_params, cudaMemcpyDeviceToDevice, s));
  return DG_OK;
}

extern "C" int dg_mlp_train(dg_mesh* mesh, int32_t epochs, int32_t batch, double lr, double* loss_first,
                            double* loss_last, void* stream) {
  if (!mesh || !mesh->mlp || epochs < 1 || batch < 1) return fail(DG_EINVAL, "dg_mlp_train: bad argument");
  Mlp* M = mesh->mlp;
  if (M->count < 1) return fail(DG_EINVAL, "dg_mlp_train: no harvested samples");
  cudaStream_t s = (cudaStream_t)stream;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  double first = -1.0, last = 0.0;
  for (int ep = 0; ep < epochs; ++ep) {
    double esum = 0.0;
    long long seen = 0;
    for (long long off = 0; off < M->count; off += batch) {
      const int nb = (int)((M->count - off < batch) ? (M->count - off) : batch);
      double L = 0.0;
      const bool want = (off + batch >= M->count) || ep == 0;
      int rc = loss_grad(M, M->X + off * M->n_in, M->Bs + off * (long long)M->n * M->n, nb, want ? &L : nullptr, s);
      if (rc) return rc;
      ++M->adam_t;
      const float c1 = 1.f - std::pow(b1, (float)M->adam_t), c2 = 1.f - std::pow(b2, (float)M->adam_t);
      k_adam<<<1024, 256, 0, s>>>(M->n_params, M->params, M->grads, M->adam_m, M->adam_v, (float)lr, b1, b2, c1, c2,
                                  eps);
      DG_LAUNCH_CHECK("k_adam");
      if (want) {
        esum += L * nb;
        seen += nb;
      }
    }
    if (ep == 0 && seen) first = esum / seen;
    if (seen) last = esum / seen;
  }
  M->ready = false;
  if (loss_first) *loss_first = first;
  if (loss_last) *loss_last = last;
  return DG_OK;
}

// inference for every element at state u: stores D, U, V (scaled) for dg_precond_apply
int mlp_setup(dg_mesh* mesh, const double* u, double dt_aii, cudaStream_t s) {
  Mlp* M = mesh->mlp;
  if (!M) return fail(DG_EINVAL, "learned preconditioner used before dg_mlp_init");
  int rc = mlp_features(mesh, u, dt_aii, s);
  if (rc) return rc;
  const int chunk = 8192;
  rc = ensure_batch(M, chunk);
  if (rc) return rc;
  for (long long e0 = 0; e0 < mesh->E; e0 += chunk) {
    const int nb = (int)((mesh->E - e0 < chunk) ? mesh->E - e0 : chunk);
    rc = forward(M, M->feat + e0 * M->n_in, nb, M->outE + e0 * M->n_out, s);
    if (rc) return rc;
  }
  M->ready = true;
  return DG_OK;
}

int mlp_apply(dg_mesh* mesh, const double* x, double* y, cudaStream_t s) {
  Mlp* M = mesh->mlp;
  if (!M || !M->ready) return fail(DG_EINVAL, "learned preconditioner used before dg_precond_setup");
  k_mlp_apply<<<(unsigned)mesh->E, 128, sizeof(float) * M->n, s>>>(mesh->E, mesh->np, M->rank, M->outE, M->sdiag, x, y);
  DG_LAUNCH_CHECK("k_mlp_apply");
  return DG_OK;
}
