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
// tile) items from a queue, largest shells first; each item accumulates the shell's
// Q[k1, q1] in shared memory (FP64) and writes it once.
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

// Thread mapping: lane = cell, warp = radial row k1 (K warps per CTA).  Each warp walks the
// program on its own: per channel, per block of J q2 groups, stage 1 for the J groups
// (core rows as float4, reused by the J groups), then the union of the block's q3: f[:, q3]
// is loaded once and serves every q2 of the block it pairs with.
#ifndef WEF_RF_EARLY_ACC
#define WEF_RF_EARLY_ACC 0
#endif
template <int K>
struct RfCfg {
  static constexpr int KP4 = (K + 3) / 4 * 4;  // padded k2 (float4 core rows)
  static constexpr int J = rf_group_width(K);   // q2 groups per block (register budget)
  // Registers per thread that let two CTAs share an SM: each of the 4 sub-partitions has
  // 16384 registers and takes ceil(2 K / 4) of the two CTAs' warps.
  static constexpr int WARPS_PER_SMSP = (2 * K + 3) / 4;
  static constexpr int MAXREG_RAW = 16384 / (32 * WARPS_PER_SMSP) / 8 * 8;
  static constexpr int MAXREG = MAXREG_RAW > 255 ? 255 : MAXREG_RAW;
};

template <int K>
__global__ void __launch_bounds__(32 * K) __maxnreg__(RfCfg<K>::MAXREG)
    rf_kernel(const float* __restrict__ ftile, double* __restrict__ qout, int64_t ncells, int64_t ntiles, int NQ,
              const int4* __restrict__ tasks, const int4* __restrict__ chans, const int4* __restrict__ blocks,
              const int4* __restrict__ uents, const int4* __restrict__ pairs, const double2* __restrict__ pw,
              const int32_t* __restrict__ order, int ntasks, const float* __restrict__ R32, int* __restrict__ queue,
              int64_t group) {
  using Cfg = RfCfg<K>;
  constexpr int J = Cfg::J, KP4 = Cfg::KP4, R4 = KP4 / 4, S = K * 32;
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
    // Items run tile group by tile group (a group's FP32 tiles stay in L2 while all its
    // shells pass over them), largest shells first inside a group.
    const int64_t nfull = ntiles / group, full_items = nfull * group * ntasks;
    int task;
    int64_t tile;
    if (it < full_items) {
      const int64_t g = it / (group * ntasks), r = it - g * group * ntasks;
      task = order[r / group];
      tile = g * group + r % group;
    } else {
      const int64_t rem = ntiles - nfull * group, r = it - full_items;
      task = order[r / rem];
      tile = nfull * group + r % rem;
    }
    const int4 T = __ldg(tasks + task);  // q1_base, n1, chan_start, nchan
    const float* ft = ftile + tile * (int64_t)NQ * K * 32 + lane;
    double* acc = qacc + k1 * 32 + lane;
    for (int m = 0; m < T.y; ++m) acc[m * S] = 0.0;
    for (int ch = T.z; ch < T.z + T.w; ++ch) {
      const int4 C = __ldg(chans + ch);  // sc, blk_start, nblk
      const float4* Ra = reinterpret_cast<const float4*>(R32 + ((int64_t)C.x * K + k1) * K * KP4);  // [k3][k2]
      for (int b = C.y; b < C.y + C.z; ++b) {
        const int4 B0 = __ldg(blocks + 2 * b), B1 = __ldg(blocks + 2 * b + 1);  // {nj, u_start, nu}, q2s
        const int nj = B0.x;
        const int q2v[4] = {B1.x, B1.y, B1.z, B1.w};
        float fq[J][KP4];
#pragma unroll
        for (int j = 0; j < J; ++j)
#pragma unroll
          for (int k2 = 0; k2 < KP4; ++k2) fq[j][k2] = (j < nj && k2 < K) ? __ldg(ft + (q2v[j] * K + k2) * 32) : 0.0f;
        // stage 1: A[j][k3] = sum_k2 Rt[k1][k2][k3] f[k2][q2_j]
        float A[J][K];
#pragma unroll
        for (int k3 = 0; k3 < K; ++k3) {
          float a[J];
#pragma unroll
          for (int j = 0; j < J; ++j) a[j] = 0.0f;
#pragma unroll
          for (int c = 0; c < R4; ++c) {
            const float4 r = __ldg(Ra + k3 * R4 + c);
#pragma unroll
            for (int j = 0; j < J; ++j) {
              a[j] = fmaf(r.x, fq[j][4 * c], a[j]);
              a[j] = fmaf(r.y, fq[j][4 * c + 1], a[j]);
              a[j] = fmaf(r.z, fq[j][4 * c + 2], a[j]);
              a[j] = fmaf(r.w, fq[j][4 * c + 3], a[j]);
            }
          }
#pragma unroll
          for (int j = 0; j < J; ++j) A[j][k3] = a[j];
        }
        // stage 2 + FP64 reduction over the union of the block's q3
        for (int u = B0.y; u < B0.y + B0.z; ++u) {
          const int4 U = __ldg(uents + u);  // q3, mask, pair_start
          const float* f3 = ft + U.x * K * 32;
          // J = 1 (large K, tight registers): consume f[:, q3] as it arrives
          float x[J > 1 ? K : 1];
          if constexpr (J > 1) {
#pragma unroll
            for (int k3 = 0; k3 < K; ++k3) x[k3] = __ldg(f3 + k3 * 32);
          }
          int p = U.z;
#pragma unroll
          for (int j = 0; j < J; ++j) {
            if (!((U.y >> j) & 1)) continue;
#if WEF_RF_EARLY_ACC
            // record and accumulators first: their latency overlaps the dot product
            const int4 P = __ldg(pairs + p);  // ne, q1a offset, q1b offset
            const double2 W = __ldg(pw + p);
            ++p;
            const double a0 = acc[P.y * S];
            const double a1 = P.x > 1 ? acc[P.z * S] : 0.0;
#endif
            float b0 = 0.0f, b1 = 0.0f;
#pragma unroll
            for (int k3 = 0; k3 < K; ++k3) {
              const float xv = J > 1 ? x[J > 1 ? k3 : 0] : __ldg(f3 + k3 * 32);
              if (k3 & 1) b1 = fmaf(A[j][k3], xv, b1);
              else b0 = fmaf(A[j][k3], xv, b0);
            }
            const double Bv = f2d_exact(b0 + b1);
#if WEF_RF_EARLY_ACC
            acc[P.y * S] = fma(W.x, Bv, a0);
            if (P.x > 1) acc[P.z * S] = fma(W.y, Bv, a1);
#else
            const int4 P = __ldg(pairs + p);  // ne, q1a offset, q1b offset
            const double2 W = __ldg(pw + p);
            ++p;
            acc[P.y * S] = fma(W.x, Bv, acc[P.y * S]);
            if (P.x > 1) acc[P.z * S] = fma(W.y, Bv, acc[P.z * S]);
#endif
          }
        }
      }
    }
    const int64_t cell = tile * 32 + lane;
    if (cell < ncells) {
      double* qc = qout + cell * (int64_t)K * NQ + (int64_t)k1 * NQ + T.x;
      for (int m = 0; m < T.y; ++m) {
        const int q1 = T.x + m;
        // conservation projection: (k1 = 0, q1 = 0..3) and (k1 = 1, q1 = 0) are zero
        qc[m] = ((k1 == 0 && q1 < 4) || (k1 == 1 && q1 == 0)) ? 0.0 : acc[m * S];
      }
    }
    __syncthreads();
  }
}

template <int K>
cudaError_t launch_rf_k(const double* f, float* ftile32, int* queue, double* q, int64_t ncells, int NQ,
                        const DevRadial& r, const float* R32, int nsm, cudaStream_t s, cudaEvent_t ev0,
                        cudaEvent_t ev1) {
  constexpr int threads = 32 * K;
  const int64_t ntiles = (ncells + 31) / 32;
  const size_t smem = (size_t)r.n1max * threads * sizeof(double);
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
  // tile groups of ~48 MB of FP32 tiles (well inside the 126 MB L2)
  const int64_t tile_bytes = (int64_t)NQ * K * 32 * sizeof(float);
  int64_t group = (48LL << 20) / tile_bytes;
  if (group < 1) group = 1;
  if (group > ntiles) group = ntiles;
  rf_kernel<K><<<(unsigned)grid, threads, smem, s>>>(ftile32, q, ncells, ntiles, NQ, r.tasks, r.chans, r.blocks,
                                                     r.uents, r.pairs, r.pw, r.order, r.ntasks, R32, queue, group);
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
