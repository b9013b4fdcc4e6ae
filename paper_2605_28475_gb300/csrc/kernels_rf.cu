// Radial-first contraction (the paper's Sec. 4.5.3 ordering, made dense):
//   A[k1,k2](q3) = sum_k3 Rt[k1,k2,k3] f[k3,q3]          FP32, CUDA cores
//   B[k1](q2,q3) = sum_k2 A[k1,k2](q3) f[k2,q2]           FP32, CUDA cores
//   Q[k1,q1]    += g_z B[k1](q2z,q3z)   over COO entries    FP64 (the angular reduction)
// followed by the Sec. 4.4 conservation projection.  On GB300 the FP64 pipe is the
// scarce unit; this ordering leaves it only 2K flops per Gaunt entry (2.0 MFLOP per
// cell at K=L=12 instead of 19.5 MFLOP for the angular-first coupling) and moves the
// dense K^3 / K^2 work to the FP32 pipe, which is ~60x faster.
//
// CTA = 32 cells x K warps: warp = k1, lane = cell.  A persistent grid pulls
// (shell, tile) items from a queue, largest shells first; each item accumulates the
// shell's Q[k1, q1] in shared memory (FP64) and writes it once.
#include <cuda_runtime.h>

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

// Exact FP32 -> FP64 with 32-bit integer instructions (keeps the FP64 pipe free).
// FP32 subnormals flush to zero (below 1.2e-38).
__device__ __forceinline__ double f2d_exact(float x) {
  const uint32_t u = __float_as_uint(x);
  const uint32_t sign = u & 0x80000000u, e = (u >> 23) & 0xFFu, m = u & 0x7FFFFFu;
  uint32_t hi, lo;
  if (e == 0u) {
    hi = sign;
    lo = 0u;
  } else if (e == 0xFFu) {
    hi = sign | 0x7FF00000u | (m >> 3);
    lo = m << 29;
  } else {
    hi = sign | ((e + 896u) << 20) | (m >> 3);
    lo = m << 29;
  }
  return __hiloint2double((int)hi, (int)lo);
}

// q3 groups per register block (core values are reused this many times) and CTAs
// per SM: the kernel is latency-bound with one 13-warp CTA per SM, so blocks are
// sized to fit two CTAs (<= 78 registers per thread at K = 13).
template <int K>
__host__ __device__ constexpr int rf_chunk() {
  return K <= 9 ? 4 : 2;
}
template <int K>
__host__ __device__ constexpr int rf_min_blocks() {
  return K <= 13 ? 2 : 1;
}

template <int K>
__global__ void __launch_bounds__(32 * K, rf_min_blocks<K>()) rf_kernel(const float* __restrict__ ftile, double* __restrict__ qout,
                                                    int64_t ncells, int64_t ntiles, int NQ,
                                                    const int4* __restrict__ tasks, const int4* __restrict__ chans,
                                                    const int4* __restrict__ m3s, const int4* __restrict__ pairs,
                                                    const double2* __restrict__ pw, const int32_t* __restrict__ order,
                                                    int ntasks, const float* __restrict__ R32,
                                                    int* __restrict__ queue) {
  constexpr int kChunk = rf_chunk<K>();
  extern __shared__ double qacc[];  // [m1][k1][32]
  __shared__ int item_s;
  const int k1 = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t nitems = ntiles * ntasks;
  for (;;) {
    if (threadIdx.x == 0) item_s = atomicAdd(queue, 1);
    __syncthreads();
    const int64_t it = item_s;
    __syncthreads();
    if (it >= nitems) break;
    const int task = order[it / ntiles];
    const int64_t tile = it % ntiles;
    const int4 T = __ldg(tasks + task);  // q1_base, n1, chan_start, nchan
    const float* ft = ftile + tile * (int64_t)NQ * K * 32 + lane;
    double* acc = qacc + k1 * 32 + lane;
    for (int m = 0; m < T.y; ++m) acc[m * K * 32] = 0.0;
    for (int ch = T.z; ch < T.z + T.w; ++ch) {
      const int4 C = __ldg(chans + ch);  // sc, m3_start, n_m3
      const float* Rk = R32 + ((int64_t)C.x * K + k1) * K * K;  // Rt[k1][k2][k3]
      for (int m0 = 0; m0 < C.z; m0 += kChunk) {
        const int nj = C.z - m0 < kChunk ? C.z - m0 : kChunk;
        int4 M[kChunk];
        float fq[kChunk][K];
#pragma unroll
        for (int j = 0; j < kChunk; ++j) {
          M[j] = j < nj ? __ldg(m3s + C.y + m0 + j) : make_int4(0, 0, 0, 0);
#pragma unroll
          for (int k3 = 0; k3 < K; ++k3) fq[j][k3] = j < nj ? __ldg(ft + (M[j].x * K + k3) * 32) : 0.0f;
        }
        // stage 1: A[j][k2] = sum_k3 Rt[k1][k2][k3] f[k3][q3_j]
        float A[kChunk][K];
#pragma unroll
        for (int k2 = 0; k2 < K; ++k2) {
          float a[kChunk];
#pragma unroll
          for (int j = 0; j < kChunk; ++j) a[j] = 0.0f;
#pragma unroll
          for (int k3 = 0; k3 < K; ++k3) {
            const float r = __ldg(Rk + k2 * K + k3);
#pragma unroll
            for (int j = 0; j < kChunk; ++j) a[j] = fmaf(r, fq[j][k3], a[j]);
          }
#pragma unroll
          for (int j = 0; j < kChunk; ++j) A[j][k2] = a[j];
        }
        // stage 2 + FP64 reduction, pair by pair
#pragma unroll
        for (int j = 0; j < kChunk; ++j) {
          if (j >= nj) break;
          for (int p = M[j].y; p < M[j].y + M[j].z; ++p) {
            const int4 P = __ldg(pairs + p);  // q2, ne, q1a offset, q1b offset
            const double2 W = __ldg(pw + p);
            const float* f2 = ft + P.x * K * 32;
            float b0 = 0.0f, b1 = 0.0f;
#pragma unroll
            for (int k2 = 0; k2 < K; k2 += 2) {
              b0 = fmaf(A[j][k2], __ldg(f2 + k2 * 32), b0);
              if (k2 + 1 < K) b1 = fmaf(A[j][k2 + 1], __ldg(f2 + (k2 + 1) * 32), b1);
            }
            const double B = f2d_exact(b0 + b1);
            acc[P.z * K * 32] = fma(W.x, B, acc[P.z * K * 32]);
            if (P.y > 1) acc[P.w * K * 32] = fma(W.y, B, acc[P.w * K * 32]);
          }
        }
      }
    }
    const int64_t cell = tile * 32 + lane;
    if (cell < ncells) {
      double* qc = qout + cell * (int64_t)K * NQ + (int64_t)k1 * NQ + T.x;
      for (int m = 0; m < T.y; ++m) {
        const int q1 = T.x + m;
        double v = acc[m * K * 32];
        if ((k1 == 0 && q1 < 4) || (k1 == 1 && q1 == 0)) v = 0.0;  // conservation projection
        qc[m] = v;
      }
    }
    __syncthreads();
  }
}

template <int K>
cudaError_t launch_rf_k(const double* f, float* ftile32, int* queue, double* q, int64_t ncells, int NQ,
                        const DevRadial& r, const float* R32, int nsm, cudaStream_t s) {
  const int64_t ntiles = (ncells + 31) / 32;
  const size_t smem = (size_t)r.n1max * K * 32 * sizeof(double);
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(rf_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  const int N = K * NQ;
  tile_f32_kernel<<<dim3((unsigned)ntiles, (unsigned)((N + 31) / 32)), dim3(32, 8), 0, s>>>(f, ftile32, ncells, K, NQ);
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rf_kernel<K>, 32 * K, smem);
  if (per_sm < 1) per_sm = 1;
  const int64_t nitems = ntiles * r.ntasks;
  int64_t grid = (int64_t)nsm * per_sm;
  if (grid > nitems) grid = nitems;
  rf_kernel<K><<<(unsigned)grid, 32 * K, smem, s>>>(ftile32, q, ncells, ntiles, NQ, r.tasks, r.chans, r.m3s, r.pairs,
                                                    r.pw, r.order, r.ntasks, R32, queue);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_rf(int K, const double* f, float* ftile32, int* queue, double* q, int64_t ncells, int NQ,
                      const DevRadial& r, const float* R32, int nsm, cudaStream_t s) {
  switch (K) {
#define WEF_RF(k) \
  case k:         \
    return launch_rf_k<k>(f, ftile32, queue, q, ncells, NQ, r, R32, nsm, s);
    WEF_RF(1) WEF_RF(2) WEF_RF(3) WEF_RF(4) WEF_RF(5) WEF_RF(6) WEF_RF(7) WEF_RF(8) WEF_RF(9) WEF_RF(10) WEF_RF(11)
    WEF_RF(12) WEF_RF(13) WEF_RF(14) WEF_RF(15) WEF_RF(16) WEF_RF(17)
#undef WEF_RF
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace wef
