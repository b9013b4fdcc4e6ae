// Mixed-precision contraction on the 5th-generation tensor cores (tcgen05):
// FP64 angular coupling Phi (paper Sec. 4.5.4) -> rounded to BF16 or TF32 into a
// 128-row shared-memory tile -> tcgen05.mma against the symmetrised core tile of
// the channel (staged by the bulk-copy/TMA engine) -> FP32 accumulation in TMEM
// over all channels of the output shell -> FP64 epilogue with the Sec. 4.4
// conservation projection.
//
// A CTA works on tiles of 32 cells; warp w is the radial index k3 = w and the
// lane is the cell.  A task covers up to four q1 of one shell l1; the MMA row is
// (slot, cell) = 32 * slot + lane, its column k1, and the reduction index
// (k2, k3) = k2 * K + k3.  `run_tile` does all tasks [t0, t1) of one tile; the
// one-shape kernel calls it once, the ragged persistent kernel calls it for every
// work item it pulls from a device queue.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstring>

#include "phi.cuh"
#include "tc_ptx.cuh"
#include "wef_internal.hpp"

namespace wef {

namespace {

constexpr int kBarBytes = 1024;  // barriers and the TMEM address sit below the operand tiles

template <int K, bool TF32>
struct TcShape {
  static constexpr int ESZ = TF32 ? 4 : 2;
  static constexpr int KK = K * K;
  static constexpr int KSTEP = TF32 ? 8 : 16;                    // reduction elements per MMA
  static constexpr int KP = (KK + KSTEP - 1) / KSTEP * KSTEP;    // padded reduction length
  static constexpr int NN = K <= 16 ? 16 : 32;                   // MMA N (k1, padded)
  static constexpr int SBO = KP * ESZ * 8;                       // bytes between 8-row groups
  static constexpr int A_BYTES = 128 * KP * ESZ;
  static constexpr int B_BYTES = NN * KP * ESZ;
  static constexpr int NSTEP = KP / KSTEP;
  static constexpr int TMEM_COLS = 2 * NN <= 32 ? 32 : 2 * NN;   // two accumulators
  static constexpr int OFF_A = kBarBytes;
  static constexpr int OFF_B = OFF_A + A_BYTES;
  static constexpr int SMEM = OFF_B + 2 * B_BYTES;
};

template <int K>
__host__ __device__ constexpr int tc_warps() {
  return K < 4 ? 4 : K;
}

// FP64 -> TF32 / BF16 bit patterns with 32-bit integer instructions on the two
// halves of the double (the FP64 pipe, GB300's scarcest unit, would otherwise also
// execute the conversions).  Round to nearest even at the target mantissa width
// directly from the double; results below the FP32 normal range flush to a signed
// zero; overflow gives Inf; Inf/NaN are kept.
template <int MBITS>
__device__ __forceinline__ uint32_t d2f_bits(double x) {
  const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
  const uint32_t sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7FFu);
  const uint32_t mh = hi & 0xFFFFFu;  // top 20 of the 52 mantissa bits
  if (e == 0x7FF) return sign | 0x7F800000u | ((mh | lo) ? 0x00400000u : 0u);
  constexpr int drop = 20 - MBITS;     // bits of mh below the kept mantissa (lo is entirely below)
  uint32_t m = mh >> drop;
  const uint32_t rem = mh & ((1u << drop) - 1u), half = 1u << (drop - 1);
  const bool up = rem > half || (rem == half && (lo != 0u || (m & 1u)));
  int e32 = e - 1023 + 127;
  m += up ? 1u : 0u;
  if (m >> MBITS) {  // mantissa overflow into the exponent
    m = 0u;
    ++e32;
  }
  if (e == 0 || e32 <= 0) return sign;
  if (e32 >= 255) return sign | 0x7F800000u;
  return sign | ((uint32_t)e32 << 23) | (m << (23 - MBITS));
}

__device__ __forceinline__ uint32_t a_offset(int row, int k, int esz, int sbo) {
  return (uint32_t)((row >> 3) * sbo + ((k * esz) >> 4) * 128 + (row & 7) * 16 + ((k * esz) & 15));
}

// CTA-uniform bookkeeping, one copy per thread.
struct TcState {
  uint8_t* smem;
  uint64_t* tma_bar;  // [2]: B tile landed
  uint64_t* mma_bar;  // [2]: MMAs of a channel done
  uint32_t tmem;
  int g;              // channels issued so far by this CTA (selects buffers and barrier phases)
  int tma_issued;     // thread 0: channels whose B tile has been requested
  int tma_waited;     // thread 0: channels whose B tile has landed
  int failed;
};

__device__ void tc_setup(TcState& st, uint8_t* smem, int tmem_cols) {
  st.smem = smem;
  st.tma_bar = (uint64_t*)smem;
  st.mma_bar = st.tma_bar + 2;
  uint32_t* tmem_s = (uint32_t*)(st.mma_bar + 2);
  st.g = st.tma_issued = st.tma_waited = st.failed = 0;
  if (threadIdx.x == 0) {
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&st.tma_bar[b], 1);
      tc::mbar_init(&st.mma_bar[b], 1);
    }
    tc::fence_mbar_init();
  }
  if ((threadIdx.x >> 5) == 0) tc::tmem_alloc(tmem_s, tmem_cols);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  st.tmem = *tmem_s;
}

// Wait (bounded) for outstanding MMAs and bulk copies, then free TMEM.
__device__ void tc_teardown(TcState& st, int tmem_cols, int* status) {
  if (st.failed && threadIdx.x == 0) atomicExch(status, 1);
  if (threadIdx.x == 0) {
    if (st.g >= 1) tc::mbar_wait(&st.mma_bar[(st.g - 1) & 1], ((st.g - 1) >> 1) & 1);
    if (st.tma_issued > st.tma_waited) {
      const int gp = st.tma_issued - 1;
      tc::mbar_wait(&st.tma_bar[gp & 1], (gp >> 1) & 1);
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) tc::tmem_dealloc(st.tmem, tmem_cols);
}

// Epilogue of one task: TMEM accumulator -> FP64 -> projection -> Q (warps 0-3).
template <int K, bool TF32>
__device__ __forceinline__ void tc_epilogue(TcState& st, int last_g, int acc, int q1b, int nslots, double* qout,
                                            int64_t cell, int64_t ncells, int NQ) {
  using S = TcShape<K, TF32>;
  const int w = threadIdx.x >> 5;
  if (w >= 4) return;
  if (!tc::mbar_wait(&st.mma_bar[last_g & 1], (last_g >> 1) & 1)) st.failed = 1;
  tc::tc_fence_after();
  float v[16];
  const uint32_t ta = st.tmem + ((uint32_t)(32 * w) << 16) + acc * S::NN;
  tc::tmem_ld16(ta, v);
  const int q1 = q1b + w;
  const bool store = w < nslots && cell < ncells;
  double* qc = qout + cell * (int64_t)K * NQ + q1;
  if (store) {
#pragma unroll
    for (int k1 = 0; k1 < (K < 16 ? K : 16); ++k1) {
      double val = (double)v[k1];
      if ((k1 == 0 && q1 < 4) || (k1 == 1 && q1 == 0)) val = 0.0;  // conservation projection
      qc[(int64_t)k1 * NQ] = val;
    }
  }
  if constexpr (S::NN > 16) {
    tc::tmem_ld16(ta + 16, v);
    if (store) {
#pragma unroll
      for (int k1 = 16; k1 < K; ++k1) qc[(int64_t)k1 * NQ] = (double)v[k1 - 16];
    }
  }
  tc::tc_fence_before();
}

// All tasks [t0, t1) of one 32-cell tile.  ft = tile base of the re-tiled f;
// cell = this lane's cell index within its batch; qout = that batch's Q.
template <int K, bool TF32>
__device__ void run_tile(TcState& st, const double* __restrict__ ft, double* __restrict__ qout, int64_t cell,
                         int64_t ncells, int NQ, const int32_t* __restrict__ prog, const int4* __restrict__ groups,
                         const double2* __restrict__ gw, const int32_t* __restrict__ task_off, int t0, int t1,
                         const uint8_t* __restrict__ Btiles, int* __restrict__ status) {
  using S = TcShape<K, TF32>;
  const int tid = threadIdx.x;
  const int k3 = tid >> 5, lane = tid & 31;
  const bool active = k3 < K;  // extra warps (K < 4, or a wider persistent block) do no angular work
  uint8_t* sA = st.smem + S::OFF_A;
  uint8_t* sB = st.smem + S::OFF_B;
  const uint32_t sA_u = tc::smem_u32(sA), sB_u = tc::smem_u32(sB);
  constexpr uint32_t idesc = tc::instr_desc(TF32 ? 2 : 1, 128, S::NN);
  ft += lane;
  // zero the A tile: padding columns (k >= K*K) and unused rows stay zero.  The last
  // MMA that read A (channel g-1) has completed: every earlier call ended with an epilogue.
  for (int i = tid; i < S::A_BYTES / 16; i += blockDim.x) ((uint4*)sA)[i] = make_uint4(0, 0, 0, 0);
  tc::fence_proxy_async();
  __syncthreads();
  if (tid == 0 && t0 < t1) {
    const int32_t* p = prog + task_off[t0];
    const int b = st.g & 1;
    tc::mbar_expect_tx(&st.tma_bar[b], S::B_BYTES);
    tc::bulk_g2s(sB + b * S::B_BYTES, Btiles + (size_t)p[3] * S::B_BYTES, S::B_BYTES, &st.tma_bar[b]);
    st.tma_issued = st.g + 1;
  }
  int pend_g = -1, pend_q1 = 0, pend_slots = 0, pend_acc = 0;
  for (int t = t0; t < t1 && !st.failed; ++t) {
    const int32_t* p = prog + task_off[t];
    const int q1b = __ldg(p), nslots = __ldg(p + 1), nchan = __ldg(p + 2);
    p += 3;
    const int acc = (t - t0) & 1;
    // another CTA's bounded wait gave up: stop early (uniform: every thread reads the word)
    if (__syncthreads_or(*(volatile int*)status != 0)) {
      st.failed = 1;
      break;
    }
    for (int ci = 0; ci < nchan; ++ci) {
      int gs = __ldg(p + 1);
      int ngs[4];
#pragma unroll
      for (int s = 0; s < 4; ++s) ngs[s] = s < nslots ? __ldg(p + 2 + s) : 0;
      p += 2 + nslots;
      const int g = st.g;
      const int buf = g & 1;  // B tile buffer and MMA barrier of this channel
      for (int s = 0; s < nslots; ++s) {
        const int g0 = gs;
        gs += ngs[s];
        if (!active) continue;
        double Phi[K];
        phi_slice<K>(Phi, groups, gw, g0, ngs[s], ft, k3);
        if (s == 0 && g >= 1) {
          // the single A tile is read by MMA(g-1): wait for it before the first write
          if (!tc::mbar_wait(&st.mma_bar[(g - 1) & 1], ((g - 1) >> 1) & 1)) st.failed = 1;
        }
        const int row = s * 32 + lane;
#pragma unroll
        for (int k2 = 0; k2 < K; ++k2) {
          const uint32_t off = a_offset(row, k2 * K + k3, S::ESZ, S::SBO);
          if constexpr (TF32) {
            *(uint32_t*)(sA + off) = d2f_bits<10>(Phi[k2]);
          } else {
            *(uint16_t*)(sA + off) = (uint16_t)(d2f_bits<7>(Phi[k2]) >> 16);
          }
        }
      }
      if (ci == 0 && pend_g >= 0) {
        tc_epilogue<K, TF32>(st, pend_g, pend_acc, pend_q1, pend_slots, qout, cell, ncells, NQ);
        pend_g = -1;
      }
      tc::fence_proxy_async();
      st.failed = __syncthreads_or(st.failed);
      if (st.failed) break;
      if (tid == 0) {
        tc::tc_fence_after();
        const bool tma_ok = tc::mbar_wait(&st.tma_bar[buf], (g >> 1) & 1);
        if (tma_ok) st.tma_waited = g + 1;
        if (!tma_ok) {
          atomicExch(status, 1);
        } else {
          const uint32_t d = st.tmem + acc * S::NN;
#pragma unroll 1
          for (int k = 0; k < S::NSTEP; ++k) {
            const uint64_t ad = tc::smem_desc(sA_u + k * 256, 128, S::SBO);
            const uint64_t bd = tc::smem_desc(sB_u + buf * S::B_BYTES + k * 256, 128, S::SBO);
            tc::mma<TF32>(d, ad, bd, idesc, (ci > 0 || k > 0) ? 1u : 0u);
          }
          tc::mma_commit(&st.mma_bar[buf]);
          // prefetch the next channel's B tile into the other buffer once MMA(g-1) released it
          int nsc = -1;
          if (ci + 1 < nchan) {
            nsc = __ldg(p);
          } else if (t + 1 < t1) {
            nsc = prog[task_off[t + 1] + 3];
          }
          if (nsc >= 0) {
            const bool ok = g < 1 || tc::mbar_wait(&st.mma_bar[(g - 1) & 1], ((g - 1) >> 1) & 1);
            if (!ok) {
              atomicExch(status, 1);
            } else {
              tc::mbar_expect_tx(&st.tma_bar[buf ^ 1], S::B_BYTES);
              tc::bulk_g2s(sB + (buf ^ 1) * S::B_BYTES, Btiles + (size_t)nsc * S::B_BYTES, S::B_BYTES,
                           &st.tma_bar[buf ^ 1]);
              st.tma_issued = g + 2;
            }
          }
        }
      }
      st.g = g + 1;
    }
    pend_g = st.g - 1;
    pend_q1 = q1b;
    pend_slots = nslots;
    pend_acc = acc;
  }
  if (!st.failed && pend_g >= 0) tc_epilogue<K, TF32>(st, pend_g, pend_acc, pend_q1, pend_slots, qout, cell, ncells, NQ);
  st.failed = __syncthreads_or(st.failed);
}

template <int K, bool TF32>
__global__ void __launch_bounds__(32 * tc_warps<K>(), 1)
    tc_kernel(const double* __restrict__ ftile, double* __restrict__ qout, int64_t ncells, int NQ,
              const int32_t* __restrict__ prog, const int4* __restrict__ groups, const double2* __restrict__ gw,
              const int32_t* __restrict__ task_off, const int32_t* __restrict__ chunks,
              const uint8_t* __restrict__ Btiles, int* __restrict__ status) {
  using S = TcShape<K, TF32>;
  extern __shared__ __align__(1024) uint8_t smem[];
  TcState st;
  tc_setup(st, smem, S::TMEM_COLS);
  const int64_t tile = blockIdx.x;
  const int t0 = chunks[blockIdx.y], t1 = chunks[blockIdx.y + 1];
  run_tile<K, TF32>(st, ftile + tile * (int64_t)NQ * K * 32, qout, tile * 32 + (threadIdx.x & 31), ncells, NQ, prog,
                    groups, gw, task_off, t0, t1, Btiles, status);
  tc_teardown(st, S::TMEM_COLS, status);
}

// Ragged persistent kernel: CTAs pull work items (shape, tile, task range) from a
// device queue until it is empty.  Blocks are as wide as the largest K in the batch.
template <bool TF32>
__global__ void __launch_bounds__(32 * 17, 1)
    ragged_tc_kernel(const RaggedShape* __restrict__ shapes, const RaggedItem* __restrict__ items, int nitems,
                     int* __restrict__ queue, const double* __restrict__ ftile, double* __restrict__ qout,
                     int tmem_cols, int* __restrict__ status) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ int item_s;
  TcState st;
  tc_setup(st, smem, tmem_cols);
  for (;;) {
    if (threadIdx.x == 0) item_s = atomicAdd(queue, 1);
    __syncthreads();
    const int it = item_s;
    __syncthreads();
    if (it >= nitems || st.failed) break;
    const RaggedItem I = items[it];
    const RaggedShape& S = shapes[I.shape];
    const int64_t cell = (int64_t)I.tile * 32 + (threadIdx.x & 31);
    const double* ft = ftile + S.ftile_off + (int64_t)I.tile * S.NQ * S.K * 32;
    double* q = qout + S.q_off;
#define WEF_RAGGED_CASE(k)                                                                                      \
  case k:                                                                                                       \
    run_tile<k, TF32>(st, ft, q, cell, S.ncells, S.NQ, S.prog, S.groups, S.gw, S.task_off, I.t0, I.t1,            \
                      TF32 ? S.Btf32 : S.Bbf16, status);                                                        \
    break;
    switch (S.K) {
      WEF_RAGGED_CASE(2) WEF_RAGGED_CASE(3) WEF_RAGGED_CASE(4) WEF_RAGGED_CASE(5) WEF_RAGGED_CASE(6)
      WEF_RAGGED_CASE(7) WEF_RAGGED_CASE(8) WEF_RAGGED_CASE(9) WEF_RAGGED_CASE(10) WEF_RAGGED_CASE(11)
      WEF_RAGGED_CASE(12) WEF_RAGGED_CASE(13) WEF_RAGGED_CASE(14) WEF_RAGGED_CASE(15) WEF_RAGGED_CASE(16)
      WEF_RAGGED_CASE(17)
      default:
        st.failed = 1;
    }
#undef WEF_RAGGED_CASE
  }
  tc_teardown(st, tmem_cols, status);
}

template <int K, bool TF32>
cudaError_t launch_tc_k(const double* ftile, double* q, int64_t ncells, int NQ, const DevProgram& p,
                        const int32_t* chunks, int nchunks, const uint8_t* Btiles, int* status, cudaStream_t s) {
  using S = TcShape<K, TF32>;
  static_assert(S::SMEM <= 232448, "shared memory");
  const int64_t ntiles = (ncells + 31) / 32;
  static std::atomic<size_t> attr[kMaxDevices];
  cudaError_t e = smem_opt_in(tc_kernel<K, TF32>, (size_t)S::SMEM, attr);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)ntiles, (unsigned)nchunks);
  tc_kernel<K, TF32><<<grid, 32 * tc_warps<K>(), S::SMEM, s>>>(ftile, q, ncells, NQ, p.prog, p.groups, p.gw,
                                                              p.task_off, chunks, Btiles, status);
  return cudaGetLastError();
}

template <int K>
int smem_for(bool tf32) {
  return tf32 ? TcShape<K, true>::SMEM : TcShape<K, false>::SMEM;
}

}  // namespace

int tc_b_tile_bytes(int K, bool tf32) {
  const int esz = tf32 ? 4 : 2, kstep = tf32 ? 8 : 16;
  const int kp = (K * K + kstep - 1) / kstep * kstep;
  const int nn = K <= 16 ? 16 : 32;
  return nn * kp * esz;
}

int tc_smem_bytes(int K, bool tf32) {
  switch (K) {
#define WEF_S(k) \
  case k:        \
    return smem_for<k>(tf32);
    WEF_S(2) WEF_S(3) WEF_S(4) WEF_S(5) WEF_S(6) WEF_S(7) WEF_S(8) WEF_S(9) WEF_S(10) WEF_S(11) WEF_S(12) WEF_S(13)
    WEF_S(14) WEF_S(15) WEF_S(16) WEF_S(17)
#undef WEF_S
    default:
      return 0;
  }
}

// Host-side layout of one symmetrised core tile as the MMA's B operand:
// B[n = k1][k = k2*K + k3], K-major core matrices (8 rows x 16 bytes), zero padded.
void tc_pack_b_tile(int K, bool tf32, const double* Rt /* [k1][k2][k3] */, uint8_t* out) {
  const int esz = tf32 ? 4 : 2, kstep = tf32 ? 8 : 16;
  const int kp = (K * K + kstep - 1) / kstep * kstep;
  const int nn = K <= 16 ? 16 : 32;
  const int sbo = kp * esz * 8;
  std::memset(out, 0, (size_t)nn * kp * esz);
  for (int n = 0; n < K; ++n)
    for (int k = 0; k < K * K; ++k) {
      const size_t off = (size_t)(n / 8) * sbo + (size_t)(k * esz / 16) * 128 + (n % 8) * 16 + (k * esz) % 16;
      const double v = Rt[(size_t)n * K * K + k];
      if (tf32) {
        const float f = (float)v;
        uint32_t u;
        std::memcpy(&u, &f, 4);
        // round to nearest (ties away) at the TF32 mantissa width (10 bits)
        u = (u + 0x1000u) & 0xFFFFE000u;
        std::memcpy(out + off, &u, 4);
      } else {
        const __nv_bfloat16 b = __double2bfloat16(v);
        std::memcpy(out + off, &b, 2);
      }
    }
}

cudaError_t launch_tc(int K, bool tf32, const double* ftile, double* q, int64_t ncells, int NQ, const DevProgram& p,
                      const int32_t* chunks, int nchunks, const uint8_t* Btiles, int* status, cudaStream_t s) {
#define WEF_TC_CASE(k)                                                                                     \
  case k:                                                                                                  \
    return tf32 ? launch_tc_k<k, true>(ftile, q, ncells, NQ, p, chunks, nchunks, Btiles, status, s)        \
                : launch_tc_k<k, false>(ftile, q, ncells, NQ, p, chunks, nchunks, Btiles, status, s);
  switch (K) {
    WEF_TC_CASE(2) WEF_TC_CASE(3) WEF_TC_CASE(4) WEF_TC_CASE(5) WEF_TC_CASE(6) WEF_TC_CASE(7) WEF_TC_CASE(8)
    WEF_TC_CASE(9) WEF_TC_CASE(10) WEF_TC_CASE(11) WEF_TC_CASE(12) WEF_TC_CASE(13) WEF_TC_CASE(14) WEF_TC_CASE(15)
    WEF_TC_CASE(16) WEF_TC_CASE(17)
    default:
      return cudaErrorInvalidValue;
  }
#undef WEF_TC_CASE
}

cudaError_t prepare_ragged_tc() {
  // the largest dynamic size any shape needs (K = 17, TF32), within the opt-in limit
  // left after the kernel's static shared memory
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  for (int tf = 0; tf < 2 && e == cudaSuccess; ++tf) {
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, tf ? (const void*)ragged_tc_kernel<true> : (const void*)ragged_tc_kernel<false>);
    if (e != cudaSuccess) break;
    int need = 0;
    for (int k = 2; k <= 17; ++k) need = need > tc_smem_bytes(k, tf != 0) ? need : tc_smem_bytes(k, tf != 0);
    const int allowed = optin - (int)fa.sharedSizeBytes;
    if (need > allowed) return cudaErrorInvalidValue;
    e = cudaFuncSetAttribute(tf ? (const void*)ragged_tc_kernel<true> : (const void*)ragged_tc_kernel<false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, need);
  }
  return e;
}

cudaError_t launch_ragged_tc(bool tf32, int max_k, int nsm, const RaggedShape* shapes, const RaggedItem* items,
                             int nitems, int* queue, const double* ftile, double* q, int* status, cudaStream_t s) {
  int smem = 0, tmem_cols = 32;
  for (int k = 2; k <= max_k; ++k) smem = smem > tc_smem_bytes(k, tf32) ? smem : tc_smem_bytes(k, tf32);
  if (max_k > 16) tmem_cols = 64;
  const int warps = max_k < 4 ? 4 : max_k;
  cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  if (tf32)
    ragged_tc_kernel<true><<<nsm, 32 * warps, smem, s>>>(shapes, items, nitems, queue, ftile, q, tmem_cols, status);
  else
    ragged_tc_kernel<false><<<nsm, 32 * warps, smem, s>>>(shapes, items, nitems, queue, ftile, q, tmem_cols, status);
  return cudaGetLastError();
}

}  // namespace wef
