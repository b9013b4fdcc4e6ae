// Mixed-precision contraction on the 5th-generation tensor cores (tcgen05):
// FP64 angular coupling Phi (paper Sec. 4.5.4) -> rounded to BF16 or TF32 into a
// 128-row shared-memory tile -> tcgen05.mma against the symmetrised core tile of
// the channel (staged by the bulk-copy/TMA engine) -> FP32 accumulation in TMEM
// over all channels of the output shell -> FP64 epilogue with the Sec. 4.4
// conservation projection.
//
// CTA = 32 cells x K warps (warp = k3, lane = cell).  A task covers up to four
// q1 of one shell l1; the MMA row is (slot, cell) = 32 * slot + lane, its column
// k1, and the reduction index (k2, k3) = k2 * K + k3.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstring>

#include "tc_ptx.cuh"
#include "wef_internal.hpp"

namespace wef {

namespace {

template <int K, bool TF32>
struct TcShape {
  static constexpr int ESZ = TF32 ? 4 : 2;
  static constexpr int KK = K * K;
  static constexpr int KSTEP = TF32 ? 8 : 16;                    // reduction elements per MMA
  static constexpr int KP = (KK + KSTEP - 1) / KSTEP * KSTEP;    // padded reduction length
  static constexpr int NN = K <= 16 ? 16 : 32;                   // MMA N (k1, padded)
  static constexpr int SBO_A = KP * ESZ * 8;                     // bytes between 8-row groups
  static constexpr int A_BYTES = 128 * KP * ESZ;
  static constexpr int B_BYTES = NN * KP * ESZ;
  static constexpr int NSTEP = KP / KSTEP;
  static constexpr int TMEM_COLS = 2 * NN <= 32 ? 32 : 2 * NN;   // two accumulators
  static constexpr int OFF_B = A_BYTES;
  static constexpr int OFF_BAR = OFF_B + 2 * B_BYTES;
  static constexpr int SMEM = OFF_BAR + 64;
};

__device__ __forceinline__ uint32_t a_offset(int row, int k, int esz, int sbo) {
  return (uint32_t)((row >> 3) * sbo + ((k * esz) >> 4) * 128 + (row & 7) * 16 + ((k * esz) & 15));
}

template <int K>
__host__ __device__ constexpr int tc_warps() { return K < 4 ? 4 : K; }

template <int K, bool TF32>
__global__ void __launch_bounds__(32 * tc_warps<K>(), 1) tc_kernel(const double* __restrict__ ftile, double* __restrict__ qout,
                                                       int64_t ncells, int NQ, const int32_t* __restrict__ prog,
                                                       const double* __restrict__ progw,
                                                       const int32_t* __restrict__ task_off,
                                                       const int32_t* __restrict__ task_w,
                                                       const int32_t* __restrict__ chunks,
                                                       const uint8_t* __restrict__ Btiles, int* __restrict__ status) {
  using S = TcShape<K, TF32>;
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sA = smem;
  uint8_t* sB = smem + S::OFF_B;
  uint64_t* tma_bar = (uint64_t*)(smem + S::OFF_BAR);  // [2]
  uint64_t* mma_bar = tma_bar + 2;                      // [2]
  uint32_t* tmem_s = (uint32_t*)(mma_bar + 2);
  const int tid = threadIdx.x;
  const int k3 = tid >> 5, lane = tid & 31;
  const int64_t tile = blockIdx.x;
  const int t0 = chunks[blockIdx.y], t1 = chunks[blockIdx.y + 1];
  const double* ft = ftile + tile * (int64_t)NQ * K * 32 + lane;
  const int64_t cell = tile * 32 + lane;

  // zero the A tile once: padding columns (k >= K*K) and unused rows stay zero
  for (int i = tid; i < S::A_BYTES / 16; i += 32 * tc_warps<K>()) ((uint4*)sA)[i] = make_uint4(0, 0, 0, 0);
  // with K < 4 the block still has 4 warps so that every TMEM lane quarter is drained;
  // the extra warps do no angular work
  const bool active = k3 < K;
  if (tid == 0) {
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&tma_bar[b], 1);
      tc::mbar_init(&mma_bar[b], 1);
    }
    tc::fence_mbar_init();
  }
  if (k3 == 0) tc::tmem_alloc(tmem_s, S::TMEM_COLS);
  tc::fence_proxy_async();
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_s;
  constexpr uint32_t idesc = tc::instr_desc(TF32 ? 2 : 1, 128, S::NN);
  const uint32_t sA_u = tc::smem_u32(sA), sB_u = tc::smem_u32(sB);
  int failed = 0;
  int tma_issued = 0, tma_waited = 0;  // thread 0 only

  // global channel counter g over the CTA's tasks: A/B buffers and barrier phases
  int g = 0;
  int pend_task_slots = 0, pend_q1 = 0, pend_acc = 0, pend_g = -1;  // epilogue pending for the previous task
  // first B tile
  if (tid == 0 && t0 < t1) {
    const int32_t* p = prog + task_off[t0];
    if (p[2] > 0) {
      tc::mbar_expect_tx(&tma_bar[0], S::B_BYTES);
      tc::bulk_g2s(sB, Btiles + (size_t)p[3] * S::B_BYTES, S::B_BYTES, &tma_bar[0]);
      tma_issued = 1;
    }
  }
  for (int t = t0; t < t1 && !failed; ++t) {
    const int32_t* p = prog + task_off[t];
    const double* pw = progw + task_w[t];
    const int q1b = __ldg(p), nslots = __ldg(p + 1), nchan = __ldg(p + 2);
    p += 3;
    const int acc = (t - t0) & 1;
    // another CTA's bounded wait gave up: stop early (uniform: every thread reads the word)
    if (__syncthreads_or(*(volatile int*)status != 0)) {
      failed = 1;
      break;
    }
    for (int ci = 0; ci < nchan; ++ci) {
      const int sc = __ldg(p);
      int ngs[4];
#pragma unroll
      for (int s = 0; s < 4; ++s) ngs[s] = s < nslots ? __ldg(p + 1 + s) : 0;
      p += 1 + nslots;
      const int buf = g & 1;  // B tile buffer and MMA barrier of this channel
      for (int s = 0; s < nslots; ++s) {
        if (!active) {
          for (int gi = 0; gi < ngs[s]; ++gi) {
            const int ne = __ldg(p) >> 16;
            p += 1 + ne;
            pw += ne;
          }
          continue;
        }
        double Phi[K];
#pragma unroll
        for (int k = 0; k < K; ++k) Phi[k] = 0.0;
        for (int gi = 0; gi < ngs[s]; ++gi) {
          const int hdr = __ldg(p);
          const int q2 = hdr & 0xffff, ne = hdr >> 16;
          ++p;
          double h = 0.0;
          for (int e = 0; e < ne; ++e) h = fma(__ldg(pw + e), __ldg(ft + (__ldg(p + e) * K + k3) * 32), h);
          p += ne;
          pw += ne;
          const double* f2 = ft + q2 * K * 32;
          double fv[K];
#pragma unroll
          for (int k2 = 0; k2 < K; ++k2) fv[k2] = __ldg(f2 + k2 * 32);
#pragma unroll
          for (int k2 = 0; k2 < K; ++k2) Phi[k2] = fma(fv[k2], h, Phi[k2]);
        }
        if (s == 0 && g >= 1) {
          // the single A tile is read by MMA(g-1): wait for it before the first write
          if (!tc::mbar_wait(&mma_bar[(g - 1) & 1], ((g - 1) >> 1) & 1)) failed = 1;
        }
        const int row = s * 32 + lane;
#pragma unroll
        for (int k2 = 0; k2 < K; ++k2) {
          const uint32_t off = a_offset(row, k2 * K + k3, S::ESZ, S::SBO_A);
          if constexpr (TF32) {
            float v;
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(*(uint32_t*)&v) : "f"((float)Phi[k2]));
            *(float*)(sA + off) = v;
          } else {
            *(__nv_bfloat16*)(sA + off) = __double2bfloat16(Phi[k2]);
          }
        }
      }
      // epilogue of the previous task (warps 0-3), once its last MMA has completed
      if (ci == 0 && pend_g >= 0 && k3 < 4) {
        if (!tc::mbar_wait(&mma_bar[pend_g & 1], (pend_g >> 1) & 1)) failed = 1;
        tc::tc_fence_after();
        float v[16];
        tc::tmem_ld16(tmem + ((uint32_t)(32 * k3) << 16) + pend_acc * S::NN, v);
        const int q1 = pend_q1 + k3;
        if (k3 < pend_task_slots && cell < ncells) {
#pragma unroll
          for (int k1 = 0; k1 < K && k1 < 16; ++k1) {
            double val = (double)v[k1];
            if ((k1 == 0 && q1 < 4) || (k1 == 1 && q1 == 0)) val = 0.0;
            qout[cell * (int64_t)K * NQ + (int64_t)k1 * NQ + q1] = val;
          }
        }
        if constexpr (S::NN > 16) {
          tc::tmem_ld16(tmem + ((uint32_t)(32 * k3) << 16) + pend_acc * S::NN + 16, v);
          if (k3 < pend_task_slots && cell < ncells) {
#pragma unroll
            for (int k1 = 16; k1 < K; ++k1) qout[cell * (int64_t)K * NQ + (int64_t)k1 * NQ + q1] = (double)v[k1 - 16];
          }
        }
        tc::tc_fence_before();
      }
      if (ci == 0) pend_g = -1;
      tc::fence_proxy_async();
      failed = __syncthreads_or(failed);
      if (failed) break;
      if (tid == 0) {
        tc::tc_fence_after();
        const bool tma_ok = tc::mbar_wait(&tma_bar[buf], (g >> 1) & 1);
        if (tma_ok) tma_waited = g + 1;
        if (!tma_ok) {
          atomicExch(status, 1);
        } else {
          const uint32_t d = tmem + acc * S::NN;
#pragma unroll 1
          for (int st = 0; st < S::NSTEP; ++st) {
            const uint64_t ad = tc::smem_desc(sA_u + st * 256, 128, S::SBO_A);
            const uint64_t bd = tc::smem_desc(sB_u + buf * S::B_BYTES + st * 256, 128, S::SBO_A);
            tc::mma<TF32>(d, ad, bd, idesc, (ci > 0 || st > 0) ? 1u : 0u);
          }
          tc::mma_commit(&mma_bar[buf]);
          // prefetch the B tile of the next channel into the other buffer once MMA(g-1) released it
          int nsc = -1;
          if (ci + 1 < nchan) {
            nsc = __ldg(p);
          } else if (t + 1 < t1) {
            const int32_t* pn = prog + task_off[t + 1];
            if (pn[2] > 0) nsc = pn[3];
          }
          if (nsc >= 0) {
            bool ok = true;
            if (g >= 1) ok = tc::mbar_wait(&mma_bar[(g - 1) & 1], ((g - 1) >> 1) & 1);
            if (!ok) {
              atomicExch(status, 1);
            } else {
              tc::mbar_expect_tx(&tma_bar[buf ^ 1], S::B_BYTES);
              tc::bulk_g2s(sB + (buf ^ 1) * S::B_BYTES, Btiles + (size_t)nsc * S::B_BYTES, S::B_BYTES, &tma_bar[buf ^ 1]);
              tma_issued = g + 2;
            }
          }
        }
      }
      ++g;
    }
    pend_g = g - 1;
    pend_q1 = q1b;
    pend_task_slots = nslots;
    pend_acc = acc;
  }
  // epilogue of the last task
  if (!failed && pend_g >= 0 && k3 < 4) {
    if (tc::mbar_wait(&mma_bar[pend_g & 1], (pend_g >> 1) & 1)) {
      tc::tc_fence_after();
      float v[16];
      tc::tmem_ld16(tmem + ((uint32_t)(32 * k3) << 16) + pend_acc * S::NN, v);
      const int q1 = pend_q1 + k3;
      if (k3 < pend_task_slots && cell < ncells) {
#pragma unroll
        for (int k1 = 0; k1 < K && k1 < 16; ++k1) {
          double val = (double)v[k1];
          if ((k1 == 0 && q1 < 4) || (k1 == 1 && q1 == 0)) val = 0.0;
          qout[cell * (int64_t)K * NQ + (int64_t)k1 * NQ + q1] = val;
        }
      }
      if constexpr (S::NN > 16) {
        tc::tmem_ld16(tmem + ((uint32_t)(32 * k3) << 16) + pend_acc * S::NN + 16, v);
        if (k3 < pend_task_slots && cell < ncells) {
#pragma unroll
          for (int k1 = 16; k1 < K; ++k1) qout[cell * (int64_t)K * NQ + (int64_t)k1 * NQ + q1] = (double)v[k1 - 16];
        }
      }
    } else {
      failed = 1;
    }
  }
  if (failed && tid == 0) atomicExch(status, 1);
  // drain: wait (bounded) for outstanding MMAs and bulk copies before releasing TMEM
  if (tid == 0 && g >= 1) {
    tc::mbar_wait(&mma_bar[(g - 1) & 1], ((g - 1) >> 1) & 1);
  }
  if (tid == 0 && tma_issued > tma_waited) {
    // a bulk copy for channel tma_issued - 1 is still in flight (only after a failure)
    const int gp = tma_issued - 1;
    tc::mbar_wait(&tma_bar[gp & 1], (gp >> 1) & 1);
  }
  tc::tc_fence_before();
  __syncthreads();
  if (k3 == 0) tc::tmem_dealloc(tmem, S::TMEM_COLS);
}

template <int K, bool TF32>
cudaError_t launch_tc_k(const double* ftile, double* q, int64_t ncells, int NQ, const DevProgram& p,
                        const int32_t* chunks, int nchunks, const uint8_t* Btiles, int* status, cudaStream_t s) {
  using S = TcShape<K, TF32>;
  static_assert(S::SMEM <= 232448, "shared memory");
  const int64_t ntiles = (ncells + 31) / 32;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(tc_kernel<K, TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  dim3 grid((unsigned)ntiles, (unsigned)nchunks);
  tc_kernel<K, TF32><<<grid, 32 * tc_warps<K>(), S::SMEM, s>>>(ftile, q, ncells, NQ, p.prog, p.progw, p.task_off, p.task_w, chunks,
                                                  Btiles, status);
  return cudaGetLastError();
}

}  // namespace

int tc_b_tile_bytes(int K, bool tf32) {
  const int esz = tf32 ? 4 : 2, kstep = tf32 ? 8 : 16;
  const int kp = (K * K + kstep - 1) / kstep * kstep;
  const int nn = K <= 16 ? 16 : 32;
  return nn * kp * esz;
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

}  // namespace wef
