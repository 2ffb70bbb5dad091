// FP64 fused multiply-add throughput probe: the ceiling of FP64-pipe-bound kernels.
#include "dg_internal.cuh"

namespace dg {

__global__ void k_fp64_fma(double* out, int iters, double a, double b) {
  double x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = threadIdx.x * 1e-3 + k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  out[(long long)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace dg

extern "C" int dg_probe_fp64(double* tflops) {
  using namespace dg;
  if (!tflops) return fail(DG_EINVAL, "dg_probe_fp64: null argument");
  int dev = 0, sms = 0;
  DG_CUDA_TRY(cudaGetDevice(&dev));
  DG_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 8, threads = 256, iters = 2048;
  double* out = nullptr;
  DG_CUDA_TRY(cudaMalloc(&out, sizeof(double) * blocks * threads));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_fp64_fma<<<blocks, threads>>>(out, iters, 0.999999, 1e-7);
  cudaEventRecord(e0);
  k_fp64_fma<<<blocks, threads>>>(out, iters, 0.999999, 1e-7);
  cudaEventRecord(e1);
  cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.0f;
  if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess) return fail(DG_ECUDA, std::string("dg_probe_fp64: ") + cudaGetErrorString(err));
  *tflops = 2.0 * 8.0 * iters * (double)blocks * threads / (ms * 1e-3) / 1e12;
  return DG_OK;
}
