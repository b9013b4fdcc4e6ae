// FP64 FMA pipe throughput probe (measurement utility, not part of libwef):
// full-warp DFMA chains (8 independent accumulators per thread), 4 CTAs x 256
// threads per SM, CUDA-event timed; plus a half-warp run that shows whether idle
// lanes cost pipe slots.  Prints one JSON line.
#include <cuda_runtime.h>

#include <cstdio>

template <int ACTIVE>
__global__ void dfma_chain(double* out, int iters, double a, double b) {
  if ((threadIdx.x & 31) >= ACTIVE) return;
  double x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = threadIdx.x + j;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 8; ++r) {
#pragma unroll
      for (int j = 0; j < 8; ++j) x[j] = fma(x[j], a, b);
    }
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += x[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int ACTIVE>
static double run(int sms, double* buf, int iters) {
  const int blocks = sms * 4, threads = 256;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  dfma_chain<ACTIVE><<<blocks, threads>>>(buf, 8, 1.0000001, 1e-9);
  cudaEventRecord(e0);
  dfma_chain<ACTIVE><<<blocks, threads>>>(buf, iters, 1.0000001, 1e-9);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return 2.0 * 64.0 * iters * (double)blocks * threads * ACTIVE / 32.0 / (ms * 1e-3) / 1e12;
}

int main() {
  int sms = 0, clk = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, 0);
  double* buf = nullptr;
  if (cudaMalloc(&buf, (size_t)sms * 4 * 256 * sizeof(double)) != cudaSuccess) return 1;
  const double full = run<32>(sms, buf, 2000);
  const double half = run<16>(sms, buf, 2000);
  cudaError_t e = cudaDeviceSynchronize();
  cudaFree(buf);
  printf("{\"fp64_fma_tflops\": %.4f, \"half_warp_useful_tflops\": %.4f, \"sms\": %d, \"max_clock_mhz\": %.0f, \"status\": \"%s\"}\n",
         full, half, sms, clk / 1000.0, cudaGetErrorString(e));
  return e == cudaSuccess ? 0 : 1;
}
