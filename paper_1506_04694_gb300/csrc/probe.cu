// Arithmetic-peak probe used as the roofline denominator of the ALU-bound
// kernels (the FP64 fields and solvers): a CUDA-event-timed kernel of
// independent fused multiply-add chains.  Not part of the method.
#include <cuda_runtime.h>

#include "../../include/mlmc.h"
#include "kernels.cuh"

namespace mlmc {

// Eight independent FMA chains per thread (enough to cover the pipeline's
// latency), `iters` rounds of the eight; x <- x a + b with a < 1 keeps every
// value bounded.  The sum is stored only under a condition that never holds
// for these inputs, so the compiler keeps the chains and nothing is written.
template <typename T>
__global__ void __launch_bounds__(256) fma_probe_kernel(T* out, int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = T(threadIdx.x + k) * T(1e-3);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  if (s == T(-1)) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
static int probe(int nsm, int iters, double* tflops, double* ms_out) {
  T* out = nullptr;
  if (cudaMalloc(&out, sizeof(T)) != cudaSuccess) return MLMC_ERR_NOMEM;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = MLMC_OK;
  const int threads = 256;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_probe_kernel<T>, threads, 0);
  const int blocks = nsm * (per_sm > 0 ? per_sm : 1);
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    rc = set_error(MLMC_ERR_CUDA, "mlmc_fma_peak: stream or event");
  } else {
    fma_probe_kernel<T><<<blocks, threads, 0, st>>>(out, iters / 8 + 1, T(0.9999999), T(1e-7));  // warm-up
    cudaEventRecord(e0, st);
    fma_probe_kernel<T><<<blocks, threads, 0, st>>>(out, iters, T(0.9999999), T(1e-7));
    cudaEventRecord(e1, st);
    float ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0.f) {
      rc = set_error(MLMC_ERR_CUDA, "mlmc_fma_peak: probe kernel");
    } else {
      const double flops = 2.0 * 8.0 * 4.0 * (double)iters * (double)blocks * threads;
      *tflops = flops / (ms * 1e-3) / 1e12;
      if (ms_out) *ms_out = ms;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  cudaFree(out);
  return rc;
}

}  // namespace mlmc

extern "C" int mlmc_fma_peak(int device, int fp64, int32_t iters, double* tflops, double* ms) {
  using namespace mlmc;
  if (!tflops || iters < 1) return set_error(MLMC_ERR_ARG, "mlmc_fma_peak: tflops required, iters >= 1");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return set_error(MLMC_ERR_NODEV, "no CUDA device");
  if (device < 0 || device >= ndev) return set_error(MLMC_ERR_ARG, "device index out of range");
  int prev = 0;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) return set_error(MLMC_ERR_NODEV, "cannot select the device");
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
  const int rc = fp64 ? probe<double>(nsm, iters, tflops, ms) : probe<float>(nsm, iters, tflops, ms);
  cudaSetDevice(prev);
  return rc;
}
