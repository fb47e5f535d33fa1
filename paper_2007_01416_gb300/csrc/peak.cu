// peak.cu -- measured throughput of the CUDA-core FMA pipes (FP64 and FP32),
// the denominator of the roofline of the arithmetic-bound ACAT step.
//
// Every thread runs ACC independent FMA chains for ITER iterations; the grid
// fills every SM with 8 CTAs of 256 threads. The chain operands depend on the
// thread index and the results are stored, so nothing folds away.
#include <cuda_runtime.h>

#include "acat_internal.h"

namespace {

constexpr int ACC = 8;

template <typename R>
__global__ void __launch_bounds__(256) k_fma_chain(R *out, R a, R b, int iters) {
  R acc[ACC];
#pragma unroll
  for (int k = 0; k < ACC; k++) acc[k] = (R)(threadIdx.x + k) * (R)1e-3;
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int k = 0; k < ACC; k++) acc[k] = fma(acc[k], a, b);
  }
  R s = 0;
#pragma unroll
  for (int k = 0; k < ACC; k++) s += acc[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename R>
double run(cudaStream_t st, int iters) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = sms * 8, block = 256;
  R *out = nullptr;
  if (cudaMalloc(&out, sizeof(R) * (size_t)grid * block) != cudaSuccess) return -1.0;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // a < 1 keeps the chains bounded
  k_fma_chain<R><<<grid, block, 0, st>>>(out, (R)0.999, (R)1e-4, iters / 8);  // warm-up
  cudaEventRecord(e0, st);
  k_fma_chain<R><<<grid, block, 0, st>>>(out, (R)0.999, (R)1e-4, iters);
  cudaEventRecord(e1, st);
  cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess || ms <= 0.f) return -1.0;
  const double flops = 2.0 * ACC * (double)iters * (double)grid * block;
  return flops / (ms * 1e-3);
}

}  // namespace

double acat_fma_peak_run(int precision, void *stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return precision == 0 ? run<double>(st, 1 << 12) : run<float>(st, 1 << 16);
}
