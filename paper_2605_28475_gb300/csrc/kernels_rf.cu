// Radial-first contraction (the paper's Sec. 4.5.3 ordering, made dense):
//   A[k1,k3](q2) = sum_k2 Rt[k1,k2,k3] f[k2,q2]          FP32, CUDA cores
//   B[k1](q2,q3) = sum_k3 A[k1,k3](q2) f[k3,q3]           FP32, CUDA cores
//   Q[k1,q1]    += g_z B[k1](q2z,q3z)   over COO entries    FP64 (the angular reduction)
// followed by the Sec. 4.4 conservation projection.  On GB300 the FP64 pipe is the
// scarce unit; this ordering leaves it only 2K flops per Gaunt entry (2.0 MFLOP per
// cell at K=L=12 instead of 19.5 MFLOP for the angular-first coupling) and moves the
// dense K^3 / K^2 work to the FP32 pipe, which is ~60x faster.
//
// CTA = 32 cells x ceil(K/2) warps (lane = cell, two k1 per warp).  A persistent grid
// pulls (shell, tile) items from a queue, largest shells first; each item accumulates
// the shell's Q[k1, q1] in shared memory (FP64) and writes it once.
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

// Thread mapping: lane = cell, warp w = the pair k1 = (2w, 2w + 1) (the second absent for
// odd K in the last warp).  Two k1 per thread halve the per-pair loads of f[:, q3] and of
// the pair records relative to one k1 per warp, which is what bounded the L1 pipe.
template <int K>
struct RfCfg {
  static constexpr int KW = (K + 1) / 2;         // warps per CTA
  static constexpr int KP4 = (K + 3) / 4 * 4;    // padded k2 (float4 core rows)
  static constexpr int J = K <= 9 ? 4 : (K <= 13 ? 2 : 1);  // q2 groups per register block
  // registers per thread that still let two CTAs share an SM (65536 / (2 * 32 * KW), in 8s)
  static constexpr int MAXREG = (65536 / (64 * KW)) / 8 * 8 > 255 ? 255 : (65536 / (64 * KW)) / 8 * 8;
};

// One symmetrised channel of one task: the channel's q2 groups in register blocks of J,
// stage 1 (core rows as float4, reused by the J groups), then stage 2 and the FP64 Gaunt
// reduction pair by pair.  TWO: this warp holds a second k1.
template <int K, bool TWO>
__device__ __forceinline__ void rf_channel(const int4 C, const float* __restrict__ ft, double2* __restrict__ acc,
                                           const int4* __restrict__ outer, const int4* __restrict__ pairs,
                                           const double2* __restrict__ pw, const float4* __restrict__ Ra) {
  using Cfg = RfCfg<K>;
  constexpr int J = Cfg::J, KP4 = Cfg::KP4, R4 = KP4 / 4;
  constexpr int ACC_STRIDE = Cfg::KW * 32;
  const float4* Rb = Ra + K * R4;  // next k1
  for (int m0 = 0; m0 < C.z; m0 += J) {
    const int nj = C.z - m0 < J ? C.z - m0 : J;
    int4 M[J];
    float fq[J][KP4];
#pragma unroll
    for (int j = 0; j < J; ++j) {
      M[j] = j < nj ? __ldg(outer + C.y + m0 + j) : make_int4(0, 0, 0, 0);
#pragma unroll
      for (int k2 = 0; k2 < KP4; ++k2) fq[j][k2] = (j < nj && k2 < K) ? __ldg(ft + (M[j].x * K + k2) * 32) : 0.0f;
    }
    // stage 1: A[j][t][k3] = sum_k2 Rt[k1_t][k2][k3] f[k2][q2_j]
    float A[J][TWO ? 2 : 1][K];
#pragma unroll
    for (int k3 = 0; k3 < K; ++k3) {
      float a0[J], a1[J];
#pragma unroll
      for (int j = 0; j < J; ++j) a0[j] = a1[j] = 0.0f;
#pragma unroll
      for (int c = 0; c < R4; ++c) {
        const float4 ra = __ldg(Ra + k3 * R4 + c);
#pragma unroll
        for (int j = 0; j < J; ++j) {
          a0[j] = fmaf(ra.x, fq[j][4 * c], a0[j]);
          a0[j] = fmaf(ra.y, fq[j][4 * c + 1], a0[j]);
          a0[j] = fmaf(ra.z, fq[j][4 * c + 2], a0[j]);
          a0[j] = fmaf(ra.w, fq[j][4 * c + 3], a0[j]);
        }
        if (TWO) {
          const float4 rb = __ldg(Rb + k3 * R4 + c);
#pragma unroll
          for (int j = 0; j < J; ++j) {
            a1[j] = fmaf(rb.x, fq[j][4 * c], a1[j]);
            a1[j] = fmaf(rb.y, fq[j][4 * c + 1], a1[j]);
            a1[j] = fmaf(rb.z, fq[j][4 * c + 2], a1[j]);
            a1[j] = fmaf(rb.w, fq[j][4 * c + 3], a1[j]);
          }
        }
      }
#pragma unroll
      for (int j = 0; j < J; ++j) {
        A[j][0][k3] = a0[j];
        if (TWO) A[j][TWO ? 1 : 0][k3] = a1[j];
      }
    }
    // stage 2 + FP64 reduction, pair by pair
#pragma unroll
    for (int j = 0; j < J; ++j) {
      if (j >= nj) break;
      for (int p = M[j].y; p < M[j].y + M[j].z; ++p) {
        const int4 P = __ldg(pairs + p);  // q3, ne, q1a offset, q1b offset
        const double2 W = __ldg(pw + p);
        const float* f3 = ft + P.x * K * 32;
        float b0 = 0.0f, b1 = 0.0f, c0 = 0.0f, c1 = 0.0f;
#pragma unroll
        for (int k3 = 0; k3 < K; ++k3) {
          const float x = __ldg(f3 + k3 * 32);
          if (k3 & 1) {
            b1 = fmaf(A[j][0][k3], x, b1);
            if (TWO) c1 = fmaf(A[j][TWO ? 1 : 0][k3], x, c1);
          } else {
            b0 = fmaf(A[j][0][k3], x, b0);
            if (TWO) c0 = fmaf(A[j][TWO ? 1 : 0][k3], x, c0);
          }
        }
        const double Ba = f2d_exact(b0 + b1);
        const double Bb = TWO ? f2d_exact(c0 + c1) : 0.0;
        double2* pa = acc + P.z * ACC_STRIDE;
        double2 v = *pa;
        v.x = fma(W.x, Ba, v.x);
        if (TWO) v.y = fma(W.x, Bb, v.y);
        *pa = v;
        if (P.y > 1) {
          double2* pb = acc + P.w * ACC_STRIDE;
          v = *pb;
          v.x = fma(W.y, Ba, v.x);
          if (TWO) v.y = fma(W.y, Bb, v.y);
          *pb = v;
        }
      }
    }
  }
}

template <int K>
__global__ void __launch_bounds__(32 * RfCfg<K>::KW) __maxnreg__(RfCfg<K>::MAXREG)
    rf_kernel(const float* __restrict__ ftile, double* __restrict__ qout, int64_t ncells, int64_t ntiles, int NQ,
              const int4* __restrict__ tasks, const int4* __restrict__ chans, const int4* __restrict__ outer,
              const int4* __restrict__ pairs, const double2* __restrict__ pw, const int32_t* __restrict__ order,
              int ntasks, const float* __restrict__ R32, int* __restrict__ queue) {
  using Cfg = RfCfg<K>;
  constexpr int ACC_STRIDE = Cfg::KW * 32, K1P = 2 * Cfg::KW;
  extern __shared__ double2 qacc[];  // [m1][w][32]: (k1 = 2w, k1 = 2w + 1)
  __shared__ int item_s;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int k1a = 2 * w;
  const bool two = k1a + 1 < K;
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
    double2* acc = qacc + w * 32 + lane;
    for (int m = 0; m < T.y; ++m) acc[m * ACC_STRIDE] = make_double2(0.0, 0.0);
    for (int ch = T.z; ch < T.z + T.w; ++ch) {
      const int4 C = __ldg(chans + ch);  // sc, outer_start, n_outer
      const float4* Ra = reinterpret_cast<const float4*>(R32 + ((int64_t)C.x * K1P + k1a) * K * Cfg::KP4);
      if (two)
        rf_channel<K, true>(C, ft, acc, outer, pairs, pw, Ra);
      else
        rf_channel<K, false>(C, ft, acc, outer, pairs, pw, Ra);
    }
    const int64_t cell = tile * 32 + lane;
    if (cell < ncells) {
      double* qc = qout + cell * (int64_t)K * NQ + (int64_t)k1a * NQ + T.x;
      for (int m = 0; m < T.y; ++m) {
        const int q1 = T.x + m;
        const double2 v = acc[m * ACC_STRIDE];
        // conservation projection: (k1 = 0, q1 = 0..3) and (k1 = 1, q1 = 0) are zero
        qc[m] = (k1a == 0 && q1 < 4) ? 0.0 : v.x;
        if (two) qc[NQ + m] = (k1a == 0 && q1 == 0) ? 0.0 : v.y;
      }
    }
    __syncthreads();
  }
}

template <int K>
cudaError_t launch_rf_k(const double* f, float* ftile32, int* queue, double* q, int64_t ncells, int NQ,
                        const DevRadial& r, const float* R32, int nsm, cudaStream_t s, cudaEvent_t ev0,
                        cudaEvent_t ev1) {
  constexpr int threads = 32 * RfCfg<K>::KW;
  const int64_t ntiles = (ncells + 31) / 32;
  const size_t smem = (size_t)r.n1max * threads * sizeof(double2);
  static size_t attr = 0;  // dynamic shared memory opted in so far for this instantiation
  if (smem > attr) {
    cudaError_t e = cudaFuncSetAttribute(rf_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = smem;
  }
  cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  const int N = K * NQ;
  tile_f32_kernel<<<dim3((unsigned)ntiles, (unsigned)((N + 31) / 32)), dim3(32, 8), 0, s>>>(f, ftile32, ncells, K, NQ);
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rf_kernel<K>, threads, smem);
  if (per_sm < 1) per_sm = 1;
  const int64_t nitems = ntiles * r.ntasks;
  int64_t grid = (int64_t)nsm * per_sm;
  if (grid > nitems) grid = nitems;
  if (ev0) cudaEventRecord(ev0, s);
  rf_kernel<K><<<(unsigned)grid, threads, smem, s>>>(ftile32, q, ncells, ntiles, NQ, r.tasks, r.chans, r.outer,
                                                     r.pairs, r.pw, r.order, r.ntasks, R32, queue);
  if (ev1) cudaEventRecord(ev1, s);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_rf(int K, const double* f, float* ftile32, int* queue, double* q, int64_t ncells, int NQ,
                      const DevRadial& r, const float* R32, int nsm, cudaStream_t s, cudaEvent_t ev0,
                      cudaEvent_t ev1) {
  switch (K) {
#define WEF_RF(k) \
  case k:         \
    return launch_rf_k<k>(f, ftile32, queue, q, ncells, NQ, r, R32, nsm, s, ev0, ev1);
    WEF_RF(1) WEF_RF(2) WEF_RF(3) WEF_RF(4) WEF_RF(5) WEF_RF(6) WEF_RF(7) WEF_RF(8) WEF_RF(9) WEF_RF(10) WEF_RF(11)
    WEF_RF(12) WEF_RF(13) WEF_RF(14) WEF_RF(15) WEF_RF(16) WEF_RF(17)
#undef WEF_RF
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace wef
