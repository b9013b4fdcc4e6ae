// Radial-first contraction kernel (the paper's Sec. 4.5.3 ordering: both radial stages
// first, then the Gaunt reduction of Sec. 4.1-4.2 and the Sec. 4.4 projection), shared by
// the translation units that instantiate it with the FP64 accumulators in shared memory
// (kernels_rf.cu, which also holds the dispatch), in tensor memory with several CTAs per SM
// (kernels_rf_tmem2.cu) and in tensor memory with one CTA per SM (kernels_rf_tmem.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "wef_internal.hpp"

namespace wef {
namespace rfk {

// FP32 -> FP64 with 32-bit integer instructions (keeps the FP64 pipe free), scaled by
// 2^-896: moving the FP32 exponent and mantissa fields into the FP64 positions without
// re-biasing the exponent gives, for every finite x (zeros and subnormals included),
// exactly x * 2^-896 (FP32 exponent field e -> 2^(e-1023) instead of 2^(e-127); an FP32
// subnormal lands on the FP64 subnormal with the same ratio).  The radial-first program
// stores its Gaunt weights premultiplied by 2^896 (exact, |g| < 1), so the FP64 product
// g' * x' equals g * x exactly and the FMA rounds as it would on g * (double)x.
// Inf and NaN keep their meaning (rare branch).
__device__ __forceinline__ double f2d_scaled(float x) {
  const uint32_t u = __float_as_uint(x);
  if ((u & 0x7F800000u) == 0x7F800000u)
    return __hiloint2double((int)((u & 0x80000000u) | 0x7FF00000u | ((u & 0x7FFFFFu) >> 3)), (int)(u << 29));
  const uint32_t hi = (uint32_t)((int32_t)u >> 3) & 0x8FFFFFFFu;  // sign, then e and the top of m
  return __hiloint2double((int)hi, (int)(u << 29));
}

// c + a * b on a pair of FP32 values (two independent FMAs, each rounded once): one packed
// FP32x2 instruction, or two scalar ones (same results).
template <bool PACKED>
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  if constexpr (PACKED)
    return __ffma2_rn(a, b, c);
  else
    return make_float2(fmaf(a.x, b.x, c.x), fmaf(a.y, b.y, c.y));
}

// The shell's FP64 accumulators Q[k1 = warp][q1 offset m][cell = lane], in shared memory
// as [m][k1][32] doubles.
struct AccSmem {
  double* p;  // this thread's slot for m = 0
  __device__ __forceinline__ void zero(int n1, int S) const {
    for (int m = 0; m < n1; ++m) p[m * S] = 0.0;
  }
  __device__ __forceinline__ void add(int m, int S, double w, double b) const { p[m * S] = fma(w, b, p[m * S]); }
  // the two targets of a pair are distinct q1: both loads are issued before either update
  __device__ __forceinline__ void add2(int ma, int mb, int S, double wa, double wb, double b) const {
    const double a = p[ma * S], c = p[mb * S];
    p[ma * S] = fma(wa, b, a);
    p[mb * S] = fma(wb, b, c);
  }
  __device__ __forceinline__ double get(int m, int S) const { return p[m * S]; }
};

// In tensor memory: lane = cell within the warp's lane quadrant (warp % 4), two 32-bit
// columns per value; the warps of one quadrant use disjoint column ranges.  Accesses are
// warp-uniform (the program is), each read-modify-write waits for its load and store.
struct AccTmem {
  uint32_t base;  // TMEM address of m = 0 for this warp
  __device__ __forceinline__ void st(int m, double v) const {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1, %2};" ::"r"(base + 2u * m),
                 "r"(__double2loint(v)), "r"(__double2hiint(v))
                 : "memory");
  }
  __device__ __forceinline__ double ld(int m) const {
    int lo, hi;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%2];" : "=r"(lo), "=r"(hi) : "r"(base + 2u * m) : "memory");
    return __hiloint2double(hi, lo);
  }
  __device__ __forceinline__ static void wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
  __device__ __forceinline__ static void wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
  __device__ __forceinline__ void zero(int n1, int) const {
    for (int m = 0; m < n1; ++m) st(m, 0.0);
    wait_st();
  }
  __device__ __forceinline__ void add(int m, int, double w, double b) const {
    double a = ld(m);
    wait_ld();
    st(m, fma(w, b, a));
    wait_st();
  }
  __device__ __forceinline__ void add2(int ma, int mb, int, double wa, double wb, double b) const {
    double a = ld(ma), c = ld(mb);
    wait_ld();
    st(ma, fma(wa, b, a));
    st(mb, fma(wb, b, c));
    wait_st();
  }
  __device__ __forceinline__ double get(int m, int) const {
    double a = ld(m);
    wait_ld();
    return a;
  }
};
// Thread mapping: lane = cell, warp = radial row k1 (K warps per CTA).  Each warp walks the
// program on its own: per channel, per block of J q2 groups, stage 1 for the J groups
// (core rows as float4, reused by the J groups), then the union of the block's q3: f[:, q3]
// is loaded once and serves every q2 of the block it pairs with.  Both radial stages run
// as packed FP32x2 FMAs over k3 pairs: A is kept as KH float2 per q2 group, and each
// packed FMA advances the even-k3 and the odd-k3 partial sums of one dot product (the
// same two chains, in the same order, as scalar code with two accumulators).
template <int K>
struct RfCfg {
  static constexpr int KH = (K + 1) / 2;      // k3 pairs
  static constexpr int KP4 = (K + 3) / 4 * 4;  // padded k3 (float4 core rows)
  // packed FP32x2 FMAs up to K = 13; two scalar FMAs above (measured at K = 17, one CTA per
  // SM: 60.9k against 59.2k cells/s with packed ones)
  static constexpr bool PACKED = K <= 13;
  static constexpr int J = rf_group_width(K, false);  // q2 groups per block, shared-memory variant
  // CTAs per SM the register budget is sized for: about 32-36 resident warps where the
  // accumulators of a Kmax = Lmax shell let that many CTAs share the shared memory.  Each of
  // the 4 sub-partitions has 16384 registers and takes ceil(CTAS K / 4) of the warps.
  static constexpr int CTAS = rf_ctas_per_sm(K);
  static constexpr int WARPS_PER_SMSP = (CTAS * K + 3) / 4;
  static constexpr int MAXREG_RAW = 16384 / (32 * WARPS_PER_SMSP) / 8 * 8;
  static constexpr int MAXREG = MAXREG_RAW > 255 ? 255 : MAXREG_RAW;
  // The one-CTA-per-SM variant (rf_uses_tmem: K >= 15, or accumulators too large for two
  // CTAs) may use the whole register file.
  static constexpr int MAXREG_1CTA_RAW = 16384 / (32 * ((K + 3) / 4)) / 8 * 8;
  static constexpr int MAXREG_1CTA = MAXREG_1CTA_RAW > 255 ? 255 : MAXREG_1CTA_RAW;
};

template <int K, int ACC>
__global__ void __launch_bounds__(32 * K) __maxnreg__(ACC == kRfAccTmem ? RfCfg<K>::MAXREG_1CTA : RfCfg<K>::MAXREG)
    rf_kernel(const float* __restrict__ ftile, double* __restrict__ qout, int64_t ncells, int64_t ntiles, int NQ,
              const int4* __restrict__ tasks, const int4* __restrict__ chans, const int4* __restrict__ blocks,
              const int4* __restrict__ uents, const double2* __restrict__ pw,
              const int32_t* __restrict__ order, int ntasks, const float* __restrict__ R32, int* __restrict__ queue,
              int64_t group, int n1max, uint32_t tcols, RaggedView rv) {
  using Cfg = RfCfg<K>;
  constexpr bool TMEM = ACC != kRfAccSmem;
  constexpr int J = rf_group_width(K, ACC == kRfAccTmem), KH = Cfg::KH, R4 = Cfg::KP4 / 4, S = K * 32;
  __shared__ int item_s;
  const int k1 = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (rv.count) {  // one shape of a ragged batch: its size and tiles come from the device
    ncells = *rv.count;
    ntiles = (ncells + 31) / 32;
    ftile += *rv.tile_off;
    rv.cells += *rv.cells_off;
    if (group > ntiles) group = ntiles > 0 ? ntiles : 1;
  }
  const int64_t nitems = ntiles * ntasks;
  // Accumulators in tensor memory: warp k1 uses lane quadrant k1 % 4 and columns from
  // (k1 / 4) * 2 * n1max on; one allocation for the CTA's lifetime.  Otherwise in
  // shared memory.  The launcher sizes the grid so that the resident CTAs' columns fit in
  // the SM's 512; should the scheduler still place one more CTA on an SM, its allocation
  // waits only until a resident CTA (which waits on nothing) has drained the queue and
  // freed its columns.
  __shared__ uint32_t tbase_s;
  if constexpr (TMEM) {
    if (k1 == 0) {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                       (uint32_t)__cvta_generic_to_shared(&tbase_s)),
                   "r"(tcols)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  extern __shared__ double qacc[];  // [m1][k1][32] (shared-memory accumulators)
  using Acc = typename std::conditional<TMEM, AccTmem, AccSmem>::type;
  Acc acc;
  if constexpr (TMEM)
    acc = Acc{tbase_s + (((uint32_t)(k1 & 3) * 32u) << 16) + (uint32_t)(k1 >> 2) * 2u * (uint32_t)n1max};
  else
    acc = Acc{qacc + k1 * 32 + lane};
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
    acc.zero(T.y, S);
    for (int ch = T.z; ch < T.z + T.w; ++ch) {
      const int4 C = __ldg(chans + ch);  // sc, blk_start, nblk
      const float4* Ra = reinterpret_cast<const float4*>(R32 + ((int64_t)C.x * K + k1) * K * Cfg::KP4);  // [k2][k3]
      for (int b = C.y; b < C.y + C.z; ++b) {
        const int4 B0 = __ldg(blocks + 2 * b), B1 = __ldg(blocks + 2 * b + 1);  // {nj, u_start, nu}, q2s
        const int q2v[4] = {B1.x, B1.y, B1.z, B1.w};  // entries j >= nj are 0 (a valid row)
        // stage 1: A[j][k3] = sum_k2 Rt[k1][k2][k3] f[k2][q2_j], k2 ascending, one chain per (j, k3)
        float2 A2[J][KH];
#pragma unroll
        for (int j = 0; j < J; ++j)
#pragma unroll
          for (int i = 0; i < KH; ++i) A2[j][i] = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int k2 = 0; k2 < K; ++k2) {
          float2 fd[J];
#pragma unroll
          for (int j = 0; j < J; ++j) {
            const float v = __ldg(ft + (q2v[j] * K + k2) * 32);
            fd[j] = make_float2(v, v);
          }
#pragma unroll
          for (int c = 0; c < R4; ++c) {
            const float4 r = __ldg(Ra + k2 * R4 + c);
#pragma unroll
            for (int j = 0; j < J; ++j) {
              if (2 * c < KH) A2[j][2 * c] = fma2<Cfg::PACKED>(make_float2(r.x, r.y), fd[j], A2[j][2 * c]);
              if (2 * c + 1 < KH) A2[j][2 * c + 1] = fma2<Cfg::PACKED>(make_float2(r.z, r.w), fd[j], A2[j][2 * c + 1]);
            }
          }
        }
        // stage 2 + FP64 reduction over the union of the block's q3
        // the next union record is loaded one entry ahead, so that the loads of f[:, q3]
        // do not wait for their own record
        int4 Un = __ldg(uents + B0.y);
        for (int u = B0.y; u < B0.y + B0.z; ++u) {
          const int4 U = Un;  // q3 | mask << 16, pair_start, packed targets
          if (u + 1 < B0.y + B0.z) Un = __ldg(uents + u + 1);
          const int q3 = U.x & 0xFFFF, mask = U.x >> 16;
          const float* f3 = ft + q3 * K * 32;
          float2 xp[KH];
#pragma unroll
          for (int i = 0; i < KH; ++i) {
            xp[i].x = __ldg(f3 + (2 * i) * 32);
            xp[i].y = 2 * i + 1 < K ? __ldg(f3 + (2 * i + 1) * 32) : 0.0f;
          }
          int p = U.y;
#pragma unroll
          for (int j = 0; j < J; ++j) {
            if (!((mask >> j) & 1)) continue;
            float2 b = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int i = 0; i < KH; ++i) b = fma2<Cfg::PACKED>(A2[j][i], xp[i], b);
            const double Bv = f2d_scaled(b.x + b.y);
            const uint32_t T = ((uint32_t)(j < 2 ? U.z : U.w) >> (16 * (j & 1))) & 0xFFFFu;  // targets
            const double2 W = __ldg(pw + p);  // Gaunt weights x 2^896
            ++p;
            if (T & 0x8000u)
              acc.add2((int)(T & 0xFFu), (int)((T >> 8) & 0x7Fu), S, W.x, W.y, Bv);
            else
              acc.add((int)(T & 0xFFu), S, W.x, Bv);
          }
        }
      }
    }
    const int64_t cell = tile * 32 + lane;
    const bool store = cell < ncells;
    double* qc = qout + (store && rv.cells ? rv.cells[cell] : cell * (int64_t)K * NQ) + (int64_t)k1 * NQ + T.x;
    for (int m = 0; m < T.y; ++m) {
      const int q1 = T.x + m;
      const double v = acc.get(m, S);  // all lanes (tensor-memory loads are warp-wide)
      // conservation projection: (k1 = 0, q1 = 0..3) and (k1 = 1, q1 = 0) are zero
      if (store) qc[m] = ((k1 == 0 && q1 < 4) || (k1 == 1 && q1 == 0)) ? 0.0 : v;
    }
    __syncthreads();
  }
  if constexpr (TMEM) {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (k1 == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase_s), "r"(tcols) : "memory");
  }
}

// Shared-memory opt-in of one instantiation (so that later launches, possibly under
// stream capture, make no attribute calls).
template <int K, int ACC>
cudaError_t prepare_rf_k(size_t smem) {
  static std::atomic<size_t> attr[kMaxDevices];
  return smem > 0 ? smem_opt_in(rf_kernel<K, ACC>, smem, attr) : cudaSuccess;
}

// Launches the persistent radial-first kernel (the queue was reset and the FP32 tiles
// written by the caller).
// ncells: the cells of a one-shape call, or (rv.count set) an upper bound of the shape's
// cells in a ragged batch, which sizes the grid.
// group_bytes: FP32 tile bytes per L2 tile group (0: 24 MB).
template <int K, int ACC>
cudaError_t launch_rf_k(const float* ftile32, int* queue, double* q, int64_t ncells, int NQ, const DevRadial& r,
                        const float* R32, int nsm, cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1,
                        const RaggedView& rv = RaggedView(), int64_t group_bytes = 0) {
  constexpr int threads = 32 * K;
  constexpr bool TMEM = ACC != kRfAccSmem;
  const int64_t ntiles = (ncells + 31) / 32;
  const size_t smem = TMEM ? 0 : (size_t)r.n1max * threads * sizeof(double);
  uint32_t tcols = 0;
  if (TMEM) {
    // columns: ceil(K / 4) warps share a lane quadrant, 2 columns per FP64 accumulator
    tcols = (uint32_t)rf_tmem_cols(K, r.n1max);
    if (tcols > 512) return cudaErrorInvalidValue;
  }
  {
    cudaError_t e = prepare_rf_k<K, ACC>(smem);
    if (e != cudaSuccess) return e;
  }
  int per_sm = 1;
  if (TMEM) {
    per_sm = tmem_ctas_per_sm(rf_kernel<K, ACC>, threads, smem, (int)tcols);
  } else {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rf_kernel<K, ACC>, threads, smem);
    if (per_sm < 1) per_sm = 1;
  }
  const int64_t nitems = ntiles * r.ntasks;
  int64_t grid = (int64_t)nsm * per_sm;
  if (grid > nitems) grid = nitems;
  if (ev0) cudaEventRecord(ev0, s);
  // tile groups of ~24 MB of FP32 tiles: a group's tiles and the Q rows its items write
  // (twice the tiles' bytes, FP64) stay within the 126 MB L2.  Measured at K=L=12, 16384
  // cells: 485 MB of DRAM traffic per launch against 729 MB with 48 MB groups (432 MB
  // algorithmic), 0.9% faster.
  const int64_t tile_bytes = (int64_t)NQ * K * 32 * sizeof(float);
  int64_t group = (group_bytes > 0 ? group_bytes : (24LL << 20)) / tile_bytes;
  if (group < 1) group = 1;
  if (group > ntiles) group = ntiles;
  rf_kernel<K, ACC><<<(unsigned)grid, threads, smem, s>>>(ftile32, q, ncells, ntiles, NQ, r.tasks, r.chans, r.blocks,
                                                     r.uents, r.pw, r.order, r.ntasks, R32, queue, group,
                                                     r.n1max, tcols, rv);
  if (ev1) cudaEventRecord(ev1, s);
  return cudaGetLastError();
}

}  // namespace rfk
}  // namespace wef
