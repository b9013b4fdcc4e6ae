// Radial-first contraction with its first radial stage on the tcgen05 tensor cores
// (precision WEF_RADIAL_TC).  The paper's Sec. 4.5.3 ordering as in kernels_rf.cu:
//   A[k1,k3](q2) = sum_k2 Rt[k1,k2,k3] f[k2,q2]          tcgen05.mma, split TF32 (below)
//   B[k1](q2,q3) = sum_k3 A[k1,k3](q2) f[k3,q3]           FP32, CUDA cores
//   Q[k1,q1]    += g_z B[k1](q2z,q3z)   over COO entries    FP64 (the angular reduction)
// then the Sec. 4.4 conservation projection.
//
// Stage 1 is the only step with an operand shared by every cell: the channel's core
// Rt[k1][k2][k3].  Per q2 group of a block it is one MMA of M = 128 rows, N = 16 K columns
// and a reduction over k2 (padded to 16):
//   D[row = 32 quad + cell][n = 16 k1 + k3] = sum_k2 a[row][k2] b[k2][n],
//   a[32 quad + cell][k2] = f[k2][q2][cell]   (the 32 cells, repeated in all four lane
//                                              quadrants of tensor memory),
//   b[k2][16 k1 + k3]     = Rt[k1][k2][k3]     (zero for k3 >= K or k2 >= K).
// The warp of radial row k1 may read only the tensor-memory lanes of its quadrant
// (k1 % 4), hence the repetition: every warp finds its cells' A[k1][:] in its own lanes and
// keeps the lane = cell, warp = k1 mapping of the CUDA-core kernel for stage 2 and the FP64
// reduction.  The MMA's operands are split TF32 pairs x = x_hi + x_lo (each rounded to
// nearest), and D = a_lo b_hi + a_hi b_lo + a_hi b_hi is accumulated in FP32 on the tensor
// core: each product is correct to a few FP32 units in the last place (the dropped
// a_lo b_lo is below 2^-24 of it), against 2^-11 for a single TF32 product.
//
// Data: a (hi at columns [0, 16), lo at [16, 32)) and D (columns [32, 32 + 16 K)) in the
// CTA's tensor memory; the channel's b tiles (hi and lo, K-major core matrices, packed at
// core upload) are brought into shared memory by one bulk copy (TMA engine) per channel.
// Per group: the warps write a with tcgen05.st, a CTA barrier, one thread issues six
// MMAs (two k2 steps of 8 per product) and commits them to an mbarrier, every warp waits on
// it and reads its 16 columns with tcgen05.ld.  All waits are bounded; a wait that gives
// up sets the operator's status word and the CTA stops at its next barrier.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include "rf_kernel.cuh"
#include "tc_ptx.cuh"
#include "wef_internal.hpp"

namespace wef {

namespace {

template <int K>
struct RftCfg {
  static constexpr int NB = 16 * K;  // D columns: n = 16 k1 + k3
  static constexpr int DCOL = 32;    // D starts after a_hi [0, 16) and a_lo [16, 32)
  static constexpr int TCOLS = DCOL + NB <= 32 ? 32 : DCOL + NB <= 64 ? 64 : DCOL + NB <= 128 ? 128
                               : DCOL + NB <= 256 ? 256 : 512;
  static constexpr int BT = rft_b_tile_bytes(K);  // one b tile: NB rows x 16 k2 x 4 bytes
  static constexpr uint32_t IDESC = tc::instr_desc(2, 128, NB);
};

__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void tmem_st1(uint32_t taddr, uint32_t v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x1.b32 [%0], {%1};" ::"r"(taddr), "r"(v) : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// 2 KH consecutive 32-bit columns of this warp's 32 lanes (lane = cell) as KH pairs, in
// loads of 8, 4 and 2 columns, then one wait (results go straight to registers).
__device__ __forceinline__ void ld8(uint32_t a, float2& x0, float2& x1, float2& x2, float2& x3) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=f"(x0.x), "=f"(x0.y), "=f"(x1.x), "=f"(x1.y), "=f"(x2.x), "=f"(x2.y), "=f"(x3.x), "=f"(x3.y)
               : "r"(a)
               : "memory");
}
__device__ __forceinline__ void ld4(uint32_t a, float2& x0, float2& x1) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=f"(x0.x), "=f"(x0.y), "=f"(x1.x), "=f"(x1.y)
               : "r"(a)
               : "memory");
}
__device__ __forceinline__ void ld2(uint32_t a, float2& x0) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];" : "=f"(x0.x), "=f"(x0.y) : "r"(a) : "memory");
}
template <int KH>
__device__ __forceinline__ void tmem_ld_pairs(uint32_t a, float2 (&x)[KH]) {
  static_assert(KH >= 1 && KH <= 7, "up to 14 columns");
  constexpr int c8 = KH >= 4 ? 4 : 0, c4 = (KH - c8) >= 2 ? 2 : 0;
  if constexpr (c8 == 4) ld8(a, x[0], x[1], x[2], x[3]);
  if constexpr (c4 == 2) ld4(a + 2 * c8, x[c8], x[c8 + 1]);
  if constexpr (KH - c8 - c4 == 1) ld2(a + 2 * (c8 + c4), x[c8 + c4]);
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// D (tensor memory) += a (tensor memory) x b (shared-memory descriptor), TF32, FP32 accumulate.
__device__ __forceinline__ void mma_tf32_ts(uint32_t d, uint32_t a, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d),
      "r"(a), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}

// CTA = 32 cells x K warps (lane = cell, warp = k1), persistent over (shell, tile) items
// as rf_kernel; the shell's FP64 accumulators in shared memory after the b tiles.
template <int K>
__global__ void __launch_bounds__(32 * K) __maxnreg__(rfk::RfCfg<K>::MAXREG)
    rft_kernel(const float* __restrict__ ftile, double* __restrict__ qout, int64_t ncells, int64_t ntiles, int NQ,
               const int4* __restrict__ tasks, const int4* __restrict__ chans, const int4* __restrict__ blocks,
               const int4* __restrict__ uents, const double2* __restrict__ pw, const int32_t* __restrict__ order,
               int ntasks, const uint8_t* __restrict__ Bt, int* __restrict__ queue, int64_t group,
               int* __restrict__ status) {
  using Cfg = rfk::RfCfg<K>;
  using T = RftCfg<K>;
  constexpr int J = rf_group_width(K, false), KH = Cfg::KH, S = K * 32;
  extern __shared__ __align__(128) uint8_t smem[];
  uint8_t* sB = smem;                                    // b tiles: hi, then lo
  double* qacc = reinterpret_cast<double*>(smem + 2 * T::BT);  // [m1][k1][32]
  __shared__ uint64_t bar[2];  // [0]: the channel's b tiles landed; [1]: the group's MMAs done
  __shared__ uint32_t tbase_s;
  __shared__ int item_s;
  const int k1 = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar[0], 1);
    tc::mbar_init(&bar[1], 1);
    tc::fence_mbar_init();
  }
  if (k1 == 0) tc::tmem_alloc(&tbase_s, T::TCOLS);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  // the a columns k2 >= K (padding of the reduction) hold zeros, written once by the first
  // warp of each lane quadrant (warp k1 reaches the lanes of quadrant k1 % 4)
  if (k1 < 4) {
    const uint32_t tq = tbase_s + (((uint32_t)k1 * 32u) << 16);
    for (int k2 = K; k2 < 16; ++k2) {
      tmem_st1(tq + k2, 0u);
      tmem_st1(tq + 16 + k2, 0u);
    }
  }
  tmem_wait_st();
  const rfk::AccSmem acc{qacc + k1 * 32 + lane};
  const int64_t nitems = ntiles * ntasks;
  // CTA bookkeeping in one register (few registers are left beside stage 2): the parities of
  // the next b-tile copy and of the next MMA group, whether a wait of this thread gave up,
  // and (thread 0) whether a b-tile copy was issued and not yet waited for
  constexpr uint32_t kChPar = 1u, kGrPar = 2u, kFailed = 4u, kCopyPending = 8u;
  uint32_t st = 0u;
  for (;;) {
    if (threadIdx.x == 0) item_s = atomicAdd(queue, 1);
    __syncthreads();
    const int64_t it = item_s;
    const int stop0 = __syncthreads_or((st & kFailed) | (*(volatile int*)status != 0));
    if (it >= nitems || stop0) break;
    const int64_t nfull = ntiles / group, full_items = nfull * group * ntasks;
    int task;
    int64_t tile;
    if (it < full_items) {
      const int64_t g = it / (group * ntasks), rr = it - g * group * ntasks;
      task = order[rr / group];
      tile = g * group + rr % group;
    } else {
      const int64_t rem = ntiles - nfull * group, rr = it - full_items;
      task = order[rr / rem];
      tile = nfull * group + rr % rem;
    }
    const int4 Tk = __ldg(tasks + task);  // q1_base, n1, chan_start, nchan
    const float* ft = ftile + tile * (int64_t)NQ * K * 32 + lane;
    acc.zero(Tk.y, S);
    int stop = 0;
    for (int ch = Tk.z; ch < Tk.z + Tk.w && !stop; ++ch) {
      const int4 C = __ldg(chans + ch);  // sc, blk_start, nblk
      // the previous channel's MMAs have completed (every thread waited for each group)
      if (threadIdx.x == 0) {
        tc::mbar_expect_tx(&bar[0], 2 * T::BT);
        tc::bulk_g2s(sB, Bt + (size_t)C.x * 2 * T::BT, 2 * T::BT, &bar[0]);
        st |= kCopyPending;
      }
      for (int b = C.y; b < C.y + C.z && !stop; ++b) {
        const int4 B0 = __ldg(blocks + 2 * b), B1 = __ldg(blocks + 2 * b + 1);  // {nj, u_start, nu}, q2s
        float2 A2[J][KH];
#pragma unroll
        for (int j = 0; j < J; ++j) {
#pragma unroll
          for (int i = 0; i < KH; ++i) A2[j][i] = make_float2(0.0f, 0.0f);
          if (j >= B0.x || stop) continue;  // block-uniform
          const int q2 = j == 0 ? B1.x : j == 1 ? B1.y : j == 2 ? B1.z : B1.w;
          {
            // a = f[:, q2] of this tile's cells in this warp's lane quadrant, split TF32;
            // the nq warps of a quadrant share its K columns
            const int w = (int)(threadIdx.x >> 5), quad = w & 3, nq = (K - quad + 3) / 4;
            const uint32_t tq = tbase_s + (((uint32_t)quad * 32u) << 16);
            const float* fq = ft + q2 * K * 32;
            for (int k2 = w >> 2; k2 < K; k2 += nq) {
              const float v = __ldg(fq + k2 * 32);
              const uint32_t hi = tf32_rna(v);
              const uint32_t lo = tf32_rna(v - __uint_as_float(hi));
              tmem_st1(tq + k2, hi);
              tmem_st1(tq + 16 + k2, lo);
            }
          }
          tmem_wait_st();
          tc::tc_fence_before();
          stop = __syncthreads_or(st & kFailed);
          if (stop) continue;
          if (threadIdx.x == 0) {
            tc::tc_fence_after();
            bool ok = true;
            if (st & kCopyPending) {
              ok = tc::mbar_wait(&bar[0], st & kChPar);
              st = (st & ~kCopyPending) ^ kChPar;
            }
            if (ok) {
              const uint32_t tb = tbase_s, d = tb + T::DCOL, sBu = tc::smem_u32(sB);
              // small products first: a_lo b_hi, a_hi b_lo, then a_hi b_hi; k2 in steps of 8
#pragma unroll
              for (int t = 0; t < 3; ++t) {
                const uint32_t acol = t == 0 ? 16u : 0u;
                const uint32_t boff = t == 1 ? (uint32_t)T::BT : 0u;
#pragma unroll
                for (int kk = 0; kk < 2; ++kk)
                  mma_tf32_ts(d, tb + acol + 8u * kk, tc::smem_desc(sBu + boff + 256u * kk, 128, 512), T::IDESC,
                              (t > 0 || kk > 0) ? 1u : 0u);
              }
            } else {
              st |= kFailed;
            }
            tc::mma_commit(&bar[1]);  // arrives at once if nothing was issued
          }
          if (!tc::mbar_wait(&bar[1], (st & kGrPar) >> 1)) st |= kFailed;
          st ^= kGrPar;
          tc::tc_fence_after();
          tmem_ld_pairs<KH>(tbase_s + ((((uint32_t)(threadIdx.x >> 5) & 3u) * 32u) << 16) + T::DCOL +
                                16u * (threadIdx.x >> 5),
                            A2[j]);
          tc::tc_fence_before();
        }
        if (stop) break;
        // stage 2 + FP64 reduction over the union of the block's q3, as rf_kernel
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
            float2 bb = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int i = 0; i < KH; ++i) bb = rfk::fma2<Cfg::PACKED>(A2[j][i], xp[i], bb);
            const double Bv = rfk::f2d_scaled(bb.x + bb.y);
            const uint32_t Tg = ((uint32_t)(j < 2 ? U.z : U.w) >> (16 * (j & 1))) & 0xFFFFu;  // targets
            const double2 Wt = __ldg(pw + p);  // Gaunt weights x 2^896
            ++p;
            if (Tg & 0x8000u)
              acc.add2((int)(Tg & 0xFFu), (int)((Tg >> 8) & 0x7Fu), S, Wt.x, Wt.y, Bv);
            else
              acc.add((int)(Tg & 0xFFu), S, Wt.x, Bv);
          }
        }
      }
    }
    if (stop) {
      st |= kFailed;
      break;
    }
    const int64_t cell = tile * 32 + lane;
    if (cell < ncells) {
      double* qc = qout + cell * (int64_t)K * NQ + (int64_t)k1 * NQ + Tk.x;
      for (int m = 0; m < Tk.y; ++m) {
        const int q1 = Tk.x + m;
        const double v = acc.get(m, S);
        // conservation projection: (k1 = 0, q1 = 0..3) and (k1 = 1, q1 = 0) are zero
        qc[m] = ((k1 == 0 && q1 < 4) || (k1 == 1 && q1 == 0)) ? 0.0 : v;
      }
    }
    __syncthreads();
  }
  // teardown: nothing of this CTA may still use tensor memory or the b buffer (every
  // commit and copy was waited for, unless a wait gave up: then wait once more, bounded)
  if ((st & kFailed) && threadIdx.x == 0) atomicExch(status, 1);
  if (threadIdx.x == 0) {
    tc::mbar_wait(&bar[1], ((st & kGrPar) >> 1) ^ 1u);  // the last group's phase (completed, or none)
    if (st & kCopyPending) tc::mbar_wait(&bar[0], st & kChPar);
  }
  tc::tc_fence_before();
  __syncthreads();
  if (k1 == 0) tc::tmem_dealloc(tbase_s, T::TCOLS);
}

}  // namespace

}  // namespace wef

namespace wef {

namespace {

template <int K>
cudaError_t launch_rft_k(const float* ftile32, int* queue, double* q, int64_t ncells, int NQ, const DevRadial& r,
                         const uint8_t* Bt, int nsm, int* status, cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1,
                         int64_t group_bytes) {
  using T = RftCfg<K>;
  constexpr int threads = 32 * K;
  const int64_t ntiles = (ncells + 31) / 32;
  const size_t smem = 2 * (size_t)T::BT + (size_t)r.n1max * threads * sizeof(double);
  static std::atomic<size_t> attr[kMaxDevices];
  cudaError_t e = smem_opt_in(rft_kernel<K>, smem, attr);
  // two CTAs per SM need ~224 KB of shared memory: ask for the largest carve-out (the
  // default one holds a single CTA)
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(rft_kernel<K>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  const int per_sm = tmem_ctas_per_sm(rft_kernel<K>, threads, smem, T::TCOLS);
  const int64_t nitems = ntiles * r.ntasks;
  int64_t grid = (int64_t)nsm * per_sm;
  if (grid > nitems) grid = nitems;
  // L2 tile groups of ~24 MB of FP32 tiles, as the CUDA-core radial-first kernel
  const int64_t tile_bytes = (int64_t)NQ * K * 32 * sizeof(float);
  int64_t group = (group_bytes > 0 ? group_bytes : (24LL << 20)) / tile_bytes;
  if (group < 1) group = 1;
  if (group > ntiles) group = ntiles;
  if (ev0) cudaEventRecord(ev0, s);
  rft_kernel<K><<<(unsigned)grid, threads, smem, s>>>(ftile32, q, ncells, ntiles, NQ, r.tasks, r.chans, r.blocks,
                                                     r.uents, r.pw, r.order, r.ntasks, Bt, queue, group, status);
  if (ev1) cudaEventRecord(ev1, s);
  return cudaGetLastError();
}

// TF32 rounding to nearest (ties to even) of a double, on 11 significant bits.
float to_tf32(double x) {
  if (x == 0.0 || !std::isfinite(x)) return (float)x;
  int e = 0;
  const double m = std::frexp(x, &e);               // x = m 2^e, 0.5 <= |m| < 1
  return (float)std::ldexp(std::nearbyint(std::ldexp(m, 11)), e - 11);
}

}  // namespace

// b[k2][n = 16 k1 + k3] = Rt[k1][k2][k3] as split TF32 (hi tile, then lo tile), each tile
// K-major core matrices: element (n, k2) at (n / 8) 512 + (k2 / 4) 128 + (n % 8) 16 + (k2 % 4) 4.
void rft_pack_b_tiles(int K, const double* Rt, uint8_t* out) {
  const int bt = rft_b_tile_bytes(K);
  std::memset(out, 0, 2 * (size_t)bt);
  for (int k1 = 0; k1 < K; ++k1)
    for (int k2 = 0; k2 < K; ++k2)
      for (int k3 = 0; k3 < K; ++k3) {
        const int n = 16 * k1 + k3;
        const size_t off = (size_t)(n / 8) * 512 + (size_t)(k2 / 4) * 128 + (n % 8) * 16 + (k2 % 4) * 4;
        const double v = Rt[((size_t)k1 * K + k2) * K + k3];
        const float hi = to_tf32(v), lo = to_tf32(v - (double)hi);
        std::memcpy(out + off, &hi, 4);
        std::memcpy(out + bt + off, &lo, 4);
      }
}

cudaError_t launch_rft(int K, const double* f, float* ftile32, int* queue, double* q, int64_t ncells, int NQ,
                       const DevRadial& r, const uint8_t* Bt, int nsm, int* status, cudaStream_t s, cudaEvent_t ev0,
                       cudaEvent_t ev1, int64_t group_bytes) {
  if (!rft_supported(K) || !Bt) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(int), s);
  if (e == cudaSuccess) e = launch_tile_f32(f, ftile32, ncells, K, NQ, s);
  if (e != cudaSuccess) return e;
  switch (K) {
#define WEF_RFT(k) \
  case k:          \
    return launch_rft_k<k>(ftile32, queue, q, ncells, NQ, r, Bt, nsm, status, s, ev0, ev1, group_bytes);
    WEF_RFT(9) WEF_RFT(11) WEF_RFT(13)
#undef WEF_RFT
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace wef
