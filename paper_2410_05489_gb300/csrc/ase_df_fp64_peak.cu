// FP64 FMA throughput microbenchmark (the denominator of the residual's roofline) and
// the check of the face kernel's own FP64 reciprocal / reciprocal square root.
// Eight independent FMA chains per thread, 8 CTAs of 256 threads per SM; the rate is
// FMA instructions per second (2 flops each).

#include <cuda_runtime.h>

#include "../../include/ase_df.h"
#include "ase_df_device.cuh"

namespace {

__global__ void recip_check_kernel(const double* x, double* out, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double v = x[i];
    out[4 * i + 0] = asedf::rcp_pos(v);
    out[4 * i + 1] = 1.0 / v;
    out[4 * i + 2] = asedf::rsqrt_pos(v);
    out[4 * i + 3] = rsqrt(v);
  }
}

__global__ void __launch_bounds__(256) dfma_chains(double* out, double a, double b, int iters) {
  double x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = 1.0 + 1e-3 * threadIdx.x + 0.1 * k;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
#pragma unroll
      for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
    }
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  if (s == 1234.5) out[0] = s;  // keeps the chains alive; never true for these inputs
}

}  // namespace

extern "C" ase_df_status ase_df_fp64_fma_rate(double* fma_per_s) {
  if (!fma_per_s) return ASE_DF_E_INVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return ASE_DF_E_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return ASE_DF_E_CUDA;
  double* d = nullptr;
  if (cudaMalloc(&d, sizeof(double)) != cudaSuccess) return ASE_DF_E_NOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int blocks = sms * 8, threads = 256, iters = 2048;
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {
    cudaEventRecord(e0, 0);
    dfma_chains<<<blocks, threads>>>(d, 0.9999, 1e-4, iters);
    cudaEventRecord(e1, 0);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;
  }
  cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(d);
  if (err != cudaSuccess) return ASE_DF_E_CUDA;
  const double n = (double)blocks * threads * iters * 4 * 8;
  *fma_per_s = n / (best * 1e-3);
  return ASE_DF_OK;
}

extern "C" ase_df_status ase_df_check_recip(const double* x, double* out, int64_t n, void* stream) {
  if (!x || !out || n < 0) return ASE_DF_E_INVAL;
  if (n == 0) return ASE_DF_OK;
  const long long blocks = (n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024;
  recip_check_kernel<<<(int)blocks, 256, 0, (cudaStream_t)stream>>>(x, out, (long long)n);
  return cudaGetLastError() == cudaSuccess ? ASE_DF_OK : ASE_DF_E_CUDA;
}
