// Internal interfaces between the C ABI layer and the kernel launchers.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <exception>
#include <new>
#include <string>

#include "tables.hpp"
#include "../../include/wef.h"

#include <algorithm>
#include <atomic>

namespace wef {

// One of the four evaluation precisions of wef_precision.
inline bool valid_precision(wef_precision p) {
  return p == WEF_FP64 || p == WEF_MIXED_BF16 || p == WEF_MIXED_TF32 || p == WEF_RADIAL_FP32;
}
// The precisions of the one-shape evaluation (wef_evaluate and the calls built on it).
inline bool valid_eval_precision(wef_precision p) { return valid_precision(p) || p == WEF_RADIAL_TC; }
// Radial-first precisions: FP32 re-tiled f and a queue word in the workspace.
inline bool radial_first(wef_precision p) { return p == WEF_RADIAL_FP32 || p == WEF_RADIAL_TC; }

// Device copy of one Program (see tables.hpp).
struct DevProgram {
  const int32_t* prog = nullptr;
  const int4* groups = nullptr;
  const double2* gw = nullptr;
  const int32_t* task_off = nullptr;
  int ntasks = 0;
};

constexpr int kCellsPerTile = 32;

// Device copy of the radial-first program (see tables.hpp).
struct DevRadial {
  const int4* tasks = nullptr;
  const int4* chans = nullptr;
  const int4* blocks = nullptr;
  const int4* uents = nullptr;
  const double2* pw = nullptr;
  const int32_t* order = nullptr;
  int ntasks = 0;
  int n1max = 1;
};

// Where the cells of one shape of a ragged batch (wef_evaluate_ragged) are, as the
// evaluation kernels see it: all three pointers are device data written by the batch's
// set-up kernels on the stream, so nothing about the batch's composition is known on the
// host.  All null (the default): the cells are [0, ncells) of a one-shape call, contiguous
// in f and Q, with ncells known on the host.
struct RaggedView {
  const int* count = nullptr;          // cells of this shape
  const int64_t* tile_off = nullptr;   // start of this shape's re-tiled f, in elements of the tile buffer
  const int64_t* cells = nullptr;      // the batch's cell lists: offset (doubles) of a cell's values in f and Q
  const int64_t* cells_off = nullptr;  // start of this shape's list (count entries) in `cells`
};

// Opts a kernel in to `bytes` of dynamic shared memory on the current device, once per
// device and size (function attributes are per device).  `done` holds one entry per device.
constexpr int kMaxDevices = 64;
template <class Fn>
cudaError_t smem_opt_in(Fn fn, size_t bytes, std::atomic<size_t>* done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  if (done[dev].load(std::memory_order_relaxed) >= bytes) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) {
    size_t cur = done[dev].load(std::memory_order_relaxed);
    while (cur < bytes && !done[dev].compare_exchange_weak(cur, bytes)) {
    }
  }
  return e;
}

// CTAs per SM of a kernel that allocates `tcols` tensor-memory columns per CTA, from its
// registers, shared memory and threads and the SM's 512 columns.  (The runtime's occupancy
// query answers 1 for every kernel that uses tcgen05.alloc, whatever its resources; the
// allocation itself only waits while the SM's columns are taken.)
template <class Fn>
int tmem_ctas_per_sm(Fn fn, int threads, size_t dyn_smem, int tcols) {
  int dev = 0, regs_sm = 0, smem_sm = 0, reserved = 0, thr_sm = 0, blk_sm = 0;
  cudaFuncAttributes a{};
  if (cudaGetDevice(&dev) != cudaSuccess || cudaFuncGetAttributes(&a, fn) != cudaSuccess) return 1;
  cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
  cudaDeviceGetAttribute(&blk_sm, cudaDevAttrMaxBlocksPerMultiprocessor, dev);
  const int warps = (threads + 31) / 32;
  const long long regs_warp = ((long long)a.numRegs * 32 + 255) / 256 * 256;  // allocated per warp
  long long n = tcols > 0 ? 512 / tcols : blk_sm;
  if (regs_warp > 0) n = std::min(n, (long long)regs_sm / (regs_warp * warps));
  n = std::min(n, (long long)smem_sm / (long long)(a.sharedSizeBytes + dyn_smem + reserved));
  n = std::min(n, (long long)thr_sm / (warps * 32));
  if (blk_sm > 0) n = std::min(n, (long long)blk_sm);
  return n < 1 ? 1 : (int)n;
}

// Releases the cuBLAS handle of the dense baseline.
void destroy_cublas(void* handle);

// Radial-first FP32 core layout [sc][k1][k2][k3 -> KP4]: rows over k3 padded to whole float4s.
inline int rf_row_padded(int K) { return (K + 3) / 4 * 4; }

// Radial-first kernel attributes for operators of radial size K and largest shell n1max,
// set ahead of launches that may be captured in a graph.
cudaError_t prepare_rf(int K, int n1max);

// Radial-first evaluation: FP32 re-tiling of f, then the persistent radial-first
// kernel (queue reset here).  ftile32 and queue live in the caller's workspace.
// ev0/ev1 (may be null) are recorded around the contraction kernel alone.  group_bytes: FP32
// tile bytes per L2 tile group (0: the default, 24 MB).
cudaError_t launch_rf(int K, const double* f, float* ftile32, int* queue, double* q, int64_t ncells, int NQ,
                      const DevRadial& r, const float* R32, int nsm, cudaStream_t s, cudaEvent_t ev0 = nullptr,
                      cudaEvent_t ev1 = nullptr, int64_t group_bytes = 0);

// wef_evaluate with an explicit L2 tile-group size for the radial-first path (group_bytes,
// 0: the default; ignored by the other precisions): the same checks, errors and results.
wef_status evaluate_grouped(wef_op op, const double* f_dev, double* q_dev, int64_t ncells, wef_precision prec,
                            void* workspace, int64_t workspace_bytes, void* stream, int64_t group_bytes);

// The persistent radial-first kernel alone over one shape of a ragged batch: ftile32 is the
// base of the batch's FP32 tiles (the shape's start is *rv.tile_off), queue this shape's
// zeroed queue word, ncells_bound an upper bound of *rv.count (sizes the grid).
cudaError_t launch_rf_ragged(int K, const float* ftile32, int* queue, double* q, int64_t ncells_bound, int NQ,
                             const DevRadial& r, const float* R32, int nsm, const RaggedView& rv, cudaStream_t s);

// f[ncells][K][NQ] -> ftile[tile][q][k][32] (zero-padded tail cells).
cudaError_t launch_tile_f(const double* f, double* ftile, int64_t ncells, int K, int NQ, cudaStream_t s);

// FP64 angular coupling + FP64 radial contraction + conservation projection.
// chunks: device array of nchunks+1 task bounds.
cudaError_t launch_fp64(int K, const double* ftile, double* q, int64_t ncells, int NQ, const DevProgram& p,
                        const int32_t* chunks, int nchunks, const double* R64, cudaStream_t s,
                        const RaggedView& rv = RaggedView());

// Tensor-core path: bytes of one packed core tile (MMA B operand) and its packing.
// Radial-first evaluation with the first radial stage on the tensor cores
// (WEF_RADIAL_TC, kernels_rft.cu).  One symmetrised channel's MMA b operand is two tiles
// (TF32 hi, then lo) of 16 K rows n = 16 k1 + k3 by 16 k2, K-major core matrices.
WEF_HD constexpr int rft_b_tile_bytes(int K) { return 16 * K * 16 * 4; }
// Radial-function counts with a compiled kernel (the TF32 split of stage 1 needs a 16 K + 32
// column tensor-memory tile per CTA, two CTAs per SM).
inline bool rft_supported(int K) { return K == 9 || K == 11 || K == 13; }
void rft_pack_b_tiles(int K, const double* Rt /* [k1][k2][k3] */, uint8_t* out /* 2 rft_b_tile_bytes(K) */);
cudaError_t launch_rft(int K, const double* f, float* ftile32, int* queue, double* q, int64_t ncells, int NQ,
                       const DevRadial& r, const uint8_t* Bt, int nsm, int* status, cudaStream_t s, cudaEvent_t ev0,
                       cudaEvent_t ev1, int64_t group_bytes);
cudaError_t launch_tile_f32(const double* f, float* ftile32, int64_t ncells, int K, int NQ, cudaStream_t s);
int tc_b_tile_bytes(int K, bool tf32);
void tc_pack_b_tile(int K, bool tf32, const double* Rt /* [k1][k2][k3] */, uint8_t* out);

// FP64 angular coupling + BF16/TF32 tcgen05 radial contraction + FP64 projection.
// status: device int set to 1 if a bounded wait inside the kernel gave up.
cudaError_t launch_tc(int K, bool tf32, const double* ftile, double* q, int64_t ncells, int NQ, const DevProgram& p,
                      const int32_t* chunks, int nchunks, const uint8_t* Btiles, int* status, cudaStream_t s);

// One shape (operator) of a ragged batch, as the persistent kernel sees it.
// Offsets are in doubles from the bases passed to the kernels.
struct RaggedShape {
  int K, NQ;
  int64_t ncells;
  int64_t tile0;      // first tile of this shape in the batch's tile numbering
  int64_t f_off;      // first cell of this shape in f and Q
  int64_t ftile_off;  // this shape's re-tiled region in the workspace
  const int32_t* prog;
  const int4* groups;
  const double2* gw;
  const int32_t* task_off;
  const uint8_t* Bbf16;
  const uint8_t* Btf32;
  int64_t q_off;      // == f_off (same layout for Q)
};

// One work item: tasks [t0, t1) of tile `tile` of shape `shape`.
struct RaggedItem {
  int shape, tile, t0, t1;
};

int tc_smem_bytes(int K, bool tf32);

// Re-tile every shape's cells: grid over all tiles of the batch.
cudaError_t launch_ragged_tile_f(const RaggedShape* shapes, int nshapes, int64_t total_tiles, int max_n,
                                 const double* f, double* ftile, cudaStream_t s);

// Raise the persistent kernel's shared-memory limit (call once, outside stream capture).
cudaError_t prepare_ragged_tc();

// Persistent ragged contraction: nsm CTAs pull items from *queue (reset here).
cudaError_t launch_ragged_tc(bool tf32, int max_k, int nsm, const RaggedShape* shapes, const RaggedItem* items,
                             int nitems, int* queue, const double* ftile, double* q, int* status, cudaStream_t s);

// Record `msg` as this thread's last error (returned by wef_last_error) and return `s`.
wef_status set_error(wef_status s, const std::string& msg);

// Runs the body of a C entry point so that no C++ exception crosses the ABI: a failed
// host allocation becomes WEF_ENOMEM, any other exception WEF_EINVAL, with the message
// recorded when recording it is still possible.
template <class F>
wef_status guarded(const char* name, F&& body) {
  try {
    return body();
  } catch (const std::bad_alloc&) {
    try {
      return set_error(WEF_ENOMEM, std::string(name) + ": host allocation failed");
    } catch (...) {
      return WEF_ENOMEM;
    }
  } catch (const std::exception& e) {
    try {
      return set_error(WEF_EINVAL, std::string(name) + ": " + e.what());
    } catch (...) {
      return WEF_EINVAL;
    }
  } catch (...) {
    return WEF_EINVAL;
  }
}

std::string core_build(const Tables& T, double gamma, int pad_rad, int pad_ang, double* R);

}  // namespace wef
