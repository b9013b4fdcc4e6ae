// Radial-first contraction (the paper's Sec. 4.5.3 ordering, made dense):
//   A[k1,k3](q2) = sum_k2 Rt[k1,k2,k3] f[k2,q2]          FP32, CUDA cores
//   B[k1](q2,q3) = sum_k3 A[k1,k3](q2) f[k3,q3]           FP32, CUDA cores
//   Q[k1,q1]    += g_z B[k1](q2z,q3z)   over COO entries    FP64 (the angular reduction)
// followed by the Sec. 4.4 conservation projection.  On GB300 the FP64 pipe is the
// scarce unit; this ordering leaves it only 2K flops per Gaunt entry (2.0 MFLOP per
// cell at K=L=12 instead of 19.5 MFLOP for the angular-first coupling) and moves the
// dense K^3 / K^2 work to the FP32 pipe, which is ~60x faster.
//
// CTA = 32 cells x K warps (lane = cell, warp = k1).  A persistent grid pulls (shell,
// tile) items from a queue; each item accumulates the shell's Q[k1, q1] in FP64 and
// writes it once.  The accumulators live in tensor memory: with the register budget of
// several CTAs per SM where their columns fit in the SM's 512 (K = L = 12: 200 of a CTA's
// 256, two CTAs), else with one CTA per SM and the whole register file where two CTAs'
// accumulators do not fit in shared memory either (K = L = 16); in shared memory in between
// (K = 13 at Lmax = 16, and shapes whose columns round up past the SM's share).  This file
// holds the re-tiling kernel, the dispatch and the shared-memory instantiations;
// kernels_rf_tmem2.cu and kernels_rf_tmem.cu the tensor-memory ones.
#include <cuda_runtime.h>

#include <cstdlib>
#include <cstring>

#include "rf_kernel.cuh"
#include "wef_internal.hpp"

namespace wef {

namespace {

// f[ncells][K][NQ] (FP64) -> ftile32[tile][q][k][32] (FP32, round to nearest).
__global__ void tile_f32_kernel(const double* __restrict__ f, float* __restrict__ ft, int64_t ncells, int K, int NQ) {
  __shared__ double s[32][33];
  const int N = K * NQ;
  const int64_t tile = blockIdx.x;
  const int a0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int j = ty; j < 32; j += 8) {
    const int64_t cell = tile * 32 + j;
    const int a = a0 + tx;
    s[j][tx] = (cell < ncells && a < N) ? f[cell * N + a] : 0.0;
  }
  __syncthreads();
  for (int j = ty; j < 32; j += 8) {
    const int a = a0 + j;
    if (a < N) {
      const int k = a / NQ, q = a - k * NQ;
      ft[((tile * NQ + q) * K + k) * 32 + tx] = __double2float_rn(s[tx][j]);
    }
  }
}

}  // namespace

cudaError_t launch_tile_f32(const double* f, float* ftile32, int64_t ncells, int K, int NQ, cudaStream_t s) {
  const int64_t ntiles = (ncells + 31) / 32;
  const int N = K * NQ;
  tile_f32_kernel<<<dim3((unsigned)ntiles, (unsigned)((N + 31) / 32)), dim3(32, 8), 0, s>>>(f, ftile32, ncells, K, NQ);
  return cudaGetLastError();
}

// tensor-memory instantiations (kernels_rf_tmem.cu)
cudaError_t launch_rf_tmem(int K, const float* ftile32, int* queue, double* q, int64_t ncells, int NQ,
                           const DevRadial& r, const float* R32, int nsm, cudaStream_t s, cudaEvent_t ev0,
                           cudaEvent_t ev1, const RaggedView& rv, int64_t group_bytes);

cudaError_t launch_rf_tmem2(int K, const float* ftile32, int* queue, double* q, int64_t ncells, int NQ,
                            const DevRadial& r, const float* R32, int nsm, cudaStream_t s, cudaEvent_t ev0,
                            cudaEvent_t ev1, const RaggedView& rv, int64_t group_bytes);

// Tensor-memory accumulators with several CTAs per SM wherever their columns fit: the
// read-modify-writes of the accumulators then leave the L1/shared-memory pipe, which also
// carries the f loads (GB300, 16384 cells: K=L=12 429.4k against 390.2k cells/s with
// shared-memory accumulators, K=L=10 1.014M against 957k, K=L=8 4.16M against 3.85M).
// WEF_RF_ACCUMULATORS=smem keeps them in shared memory (for comparison).
static bool rf_use_tmem2(int K, int n1max) {
  static const bool off = [] {
    const char* v = std::getenv("WEF_RF_ACCUMULATORS");
    return v && std::strcmp(v, "smem") == 0;
  }();
  return !off && !rf_uses_tmem(K, n1max) && rf_ctas_per_sm(K) * rf_tmem_cols(K, n1max) <= 512;
}

cudaError_t prepare_rf(int K, int n1max) {
  if (K < 1 || K > 17) return cudaErrorInvalidValue;
  const size_t smem = (size_t)n1max * 32 * K * sizeof(double);
  if (rf_uses_tmem(K, n1max) || rf_use_tmem2(K, n1max)) return cudaSuccess;  // tensor-memory accumulators
  switch (K) {
#define WEF_RF(k) \
  case k:         \
    return rfk::prepare_rf_k<k, kRfAccSmem>(smem);
    WEF_RF(1) WEF_RF(2) WEF_RF(3) WEF_RF(4) WEF_RF(5) WEF_RF(6) WEF_RF(7) WEF_RF(8) WEF_RF(9) WEF_RF(10) WEF_RF(11)
    WEF_RF(12) WEF_RF(13) WEF_RF(14) WEF_RF(15) WEF_RF(16) WEF_RF(17)
#undef WEF_RF
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t launch_rf(int K, const double* f, float* ftile32, int* queue, double* q, int64_t ncells, int NQ,
                      const DevRadial& r, const float* R32, int nsm, cudaStream_t s, cudaEvent_t ev0,
                      cudaEvent_t ev1, int64_t group_bytes) {
  if (K < 1 || K > 17) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  const int64_t ntiles = (ncells + 31) / 32;
  const int N = K * NQ;
  tile_f32_kernel<<<dim3((unsigned)ntiles, (unsigned)((N + 31) / 32)), dim3(32, 8), 0, s>>>(f, ftile32, ncells, K, NQ);
  // shared-memory accumulators while two CTAs of them fit in the 228 KB of an SM (the
  // program was built for the same choice: its q2 block width depends on it)
  if (rf_uses_tmem(K, r.n1max))
    return launch_rf_tmem(K, ftile32, queue, q, ncells, NQ, r, R32, nsm, s, ev0, ev1, RaggedView(), group_bytes);
  if (rf_use_tmem2(K, r.n1max))
    return launch_rf_tmem2(K, ftile32, queue, q, ncells, NQ, r, R32, nsm, s, ev0, ev1, RaggedView(), group_bytes);
  switch (K) {
#define WEF_RF(k) \
  case k:         \
    return rfk::launch_rf_k<k, kRfAccSmem>(ftile32, queue, q, ncells, NQ, r, R32, nsm, s, ev0, ev1, RaggedView(), group_bytes);
    WEF_RF(1) WEF_RF(2) WEF_RF(3) WEF_RF(4) WEF_RF(5) WEF_RF(6) WEF_RF(7) WEF_RF(8) WEF_RF(9) WEF_RF(10) WEF_RF(11)
    WEF_RF(12) WEF_RF(13) WEF_RF(14) WEF_RF(15) WEF_RF(16) WEF_RF(17)
#undef WEF_RF
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t launch_rf_ragged(int K, const float* ftile32, int* queue, double* q, int64_t ncells_bound, int NQ,
                             const DevRadial& r, const float* R32, int nsm, const RaggedView& rv, cudaStream_t s) {
  if (K < 1 || K > 17) return cudaErrorInvalidValue;
  if (rf_uses_tmem(K, r.n1max))
    return launch_rf_tmem(K, ftile32, queue, q, ncells_bound, NQ, r, R32, nsm, s, nullptr, nullptr, rv, 0);
  if (rf_use_tmem2(K, r.n1max))
    return launch_rf_tmem2(K, ftile32, queue, q, ncells_bound, NQ, r, R32, nsm, s, nullptr, nullptr, rv, 0);
  switch (K) {
#define WEF_RF(k) \
  case k:         \
    return rfk::launch_rf_k<k, kRfAccSmem>(ftile32, queue, q, ncells_bound, NQ, r, R32, nsm, s, nullptr, nullptr, rv);
    WEF_RF(1) WEF_RF(2) WEF_RF(3) WEF_RF(4) WEF_RF(5) WEF_RF(6) WEF_RF(7) WEF_RF(8) WEF_RF(9) WEF_RF(10) WEF_RF(11)
    WEF_RF(12) WEF_RF(13) WEF_RF(14) WEF_RF(15) WEF_RF(16) WEF_RF(17)
#undef WEF_RF
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace wef
