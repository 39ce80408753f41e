// Arithmetic-rate probe: the measured counterparts of the FMA-pipe peaks that the rooflines of
// the FP64 and double-float contractions divide by. Every thread runs eight independent FMA
// chains (enough to cover the pipe's latency), the grid fills every SM, and the rate is the FMA
// count over the CUDA-event time of the kernel.
#include <algorithm>

#include "handles.h"

namespace {

template <typename T>
__global__ void fma_chain_kernel(T* out, int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = (T)(threadIdx.x + k) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the chains live
}

}  // namespace

extern "C" int cc_probe_fma_rate(int device, int fp64, double* tflops) {
  if (!tflops) return CC_ERR_INVALID;
  *tflops = 0.0;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return CC_ERR_INVALID;
  }
  int sms = 0;
  if (cudaSetDevice(device) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    cudaGetLastError();
    return CC_ERR_CUDA;
  }
  const int threads = 256, blocks = sms * 8;
  const int iters = fp64 ? 4096 : 65536;
  void* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int status = CC_OK;
  float best = 1e30f;
  if (cudaMalloc(&out, (size_t)blocks * threads * 8) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    status = CC_ERR_CUDA;
  } else {
    for (int rep = 0; rep < 4 && status == CC_OK; ++rep) {  // the first launch is a warm-up
      cudaEventRecord(e0);
      if (fp64) fma_chain_kernel<double><<<blocks, threads>>>((double*)out, iters, 0.999999, 1e-7);
      else fma_chain_kernel<float><<<blocks, threads>>>((float*)out, iters, 0.999999f, 1e-7f);
      cudaEventRecord(e1);
      if (cudaEventSynchronize(e1) != cudaSuccess) status = CC_ERR_CUDA;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0 && ms > 0.f) best = std::min(best, ms);
    }
    if (status == CC_OK && cudaGetLastError() != cudaSuccess) status = CC_ERR_CUDA;
  }
  if (status == CC_OK) *tflops = 2.0 * 8.0 * (double)iters * blocks * threads / (best * 1e-3) / 1e12;
  cudaGetLastError();
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (out) cudaFree(out);
  return status;
}
