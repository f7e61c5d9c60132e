// Measurement helper: FP64 FMA rate of the device from an in-register dependent-chain
// kernel (8 independent chains per thread, 2 blocks of 256 threads per SM).
#include <cuda_runtime.h>

#include "snap_internal.h"

namespace {

__global__ void k_fp64_rate(double *out, int iters, double s) {
  double a[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) a[c] = threadIdx.x * 1e-3 + c;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < 8; ++c) a[c] = fma(a[c], s, 0.5);
  }
  double r = 0.0;
#pragma unroll
  for (int c = 0; c < 8; ++c) r += a[c];
  if (r == 12345.678) out[threadIdx.x] = r;   // keeps the chains alive; never true
}

}  // namespace

extern "C" snap_status snap_measure_fp64_rate(int device, double *fma_per_s) {
  if (!fma_per_s) return SNAP_ERR_INVALID_ARG;
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess) return SNAP_ERR_CUDA;
  if (cudaSetDevice(device) != cudaSuccess) return SNAP_ERR_CUDA;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  double *d = nullptr;
  if (cudaMalloc(&d, 256 * sizeof(double)) != cudaSuccess) { cudaSetDevice(prev); return SNAP_ERR_CUDA; }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int iters = 4096, grid = 2 * sms, block = 256;
  k_fp64_rate<<<grid, block>>>(d, iters, 0.999);
  float best = 1e30f;
  for (int r = 0; r < 3; ++r) {
    cudaEventRecord(e0);
    k_fp64_rate<<<grid, block>>>(d, iters, 0.999);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(d);
  cudaSetDevice(prev);
  if (err != cudaSuccess) return SNAP_ERR_CUDA;
  *fma_per_s = (double)grid * block * iters * 8 / (best * 1e-3);
  return SNAP_OK;
}
