// wef_evaluate_ragged: Q(f, f) for a batch of cells of several (Kmax, Lmax) operators in one
// call, with each cell's operator and position given per cell in device arrays (the bilinear
// form of Sec. 2.3, evaluated per cell by the contraction of Sec. 4.5 that the precision
// selects).  Nothing about the batch's composition is read back to the host: set-up kernels
// on the stream count the cells of each operator, lay out one list of cell offsets per
// operator and re-tile every operator's cells into its own 32-cell tiles; then each
// operator's contraction kernel runs over its tiles, reading its cell count from the device
// and writing each cell's Q at that cell's own offset.  The operators' contractions run on a
// small pool of streams forked from the caller's stream (one pool per caller stream and
// device, created at first use) and joined back to it.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <utility>
#include <string>
#include <vector>

#include "../../include/wef.h"
#include "operator.hpp"
#include "wef_internal.hpp"

using namespace wef;

namespace {

constexpr int kMaxOps = WEF_RAGGED_MAX_OPS;
constexpr int kForks = 4;

// Workspace header (bytes): counts, scatter cursors and queue words (int[kMaxOps] each),
// then list starts, first tiles and tile offsets (int64[kMaxOps + 1] each).
constexpr int64_t kOffCount = 0, kOffCursor = 128, kOffQueue = 256, kOffListBase = 512, kOffTileFirst = 1024,
                  kOffTileOff = 1536, kHeader = 2048;
static_assert(kMaxOps * 4 <= 128 && (kMaxOps + 1) * 8 <= 512, "header layout");

struct Shapes {
  int nops;
  int K[kMaxOps], NQ[kMaxOps];
};

int64_t align256(int64_t x) { return (x + 255) / 256 * 256; }

__global__ void ragged_count(const int32_t* __restrict__ shape_id, int64_t ncells, int nops, int* __restrict__ count) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ncells) return;
  const int s = shape_id[i];
  if (s >= 0 && s < nops) atomicAdd(count + s, 1);
}

// One thread: list starts, tile numbering and tile offsets (elements) from the counts.
__global__ void ragged_prefix(Shapes sh, const int* __restrict__ count, int64_t* __restrict__ list_base,
                              int64_t* __restrict__ tile_first, int64_t* __restrict__ tile_off) {
  int64_t lb = 0, tf = 0, to = 0;
  for (int s = 0; s < sh.nops; ++s) {
    list_base[s] = lb;
    tile_first[s] = tf;
    tile_off[s] = to;
    const int64_t nt = ((int64_t)count[s] + 31) / 32;
    lb += count[s];
    tf += nt;
    to += nt * 32 * (int64_t)sh.K[s] * sh.NQ[s];
  }
  list_base[sh.nops] = lb;
  tile_first[sh.nops] = tf;
  tile_off[sh.nops] = to;
}

// Each cell's offset into its operator's list (the order inside a list does not matter:
// every lane of a tile computes its own cell with the same arithmetic).
__global__ void ragged_scatter(const int32_t* __restrict__ shape_id, const int64_t* __restrict__ offset, int64_t ncells,
                               int nops, int* __restrict__ cursor, const int64_t* __restrict__ list_base,
                               int64_t* __restrict__ lists) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ncells) return;
  const int s = shape_id[i];
  if (s < 0 || s >= nops) return;
  const int slot = atomicAdd(cursor + s, 1);
  lists[list_base[s] + slot] = offset[i];
}

// tiles[tile_off[s] + ((tile * NQ + q) * K + k) * 32 + lane] = f[lists[s][tile * 32 + lane] + k * NQ + q]
// (zero for lanes past the operator's last cell).  grid (upper bound of all tiles,
// ceil(max N / 32)), block (32, 8).
template <class T>
__global__ void ragged_tile(Shapes sh, const double* __restrict__ f, const int* __restrict__ count,
                            const int64_t* __restrict__ list_base, const int64_t* __restrict__ tile_first,
                            const int64_t* __restrict__ tile_off, const int64_t* __restrict__ lists,
                            T* __restrict__ tiles) {
  __shared__ double buf[32][33];
  const int64_t gt = blockIdx.x;
  if (gt >= tile_first[sh.nops]) return;
  int s = 0;
  while (s + 1 < sh.nops && tile_first[s + 1] <= gt) ++s;
  const int K = sh.K[s], NQ = sh.NQ[s], N = K * NQ;
  const int a0 = blockIdx.y * 32;
  if (a0 >= N) return;
  const int64_t tile = gt - tile_first[s];
  const int64_t* list = lists + list_base[s];
  const int n = count[s];
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int j = ty; j < 32; j += 8) {
    const int64_t slot = tile * 32 + j;
    const int a = a0 + tx;
    buf[j][tx] = (slot < n && a < N) ? f[list[slot] + a] : 0.0;
  }
  __syncthreads();
  T* out = tiles + tile_off[s];
  for (int j = ty; j < 32; j += 8) {
    const int a = a0 + j;
    if (a < N) {
      const int k = a / NQ, q = a - k * NQ;
      out[((tile * NQ + q) * K + k) * 32 + tx] = (T)buf[tx][j];
    }
  }
}

// Forked streams for the operators' contractions: one pool per (device, caller stream), so
// that calls on different caller streams (a server's slots) overlap instead of queueing on
// shared forks; created by the first call with that stream on that device and kept until
// the process exits.  A lock keeps concurrent host threads from interleaving their uses of
// a pool's events.
struct ForkPool {
  bool ready = false;
  cudaStream_t fork[kForks] = {};
  cudaEvent_t ev[kForks + 1] = {};
};
constexpr int kMaxDev = 64;
constexpr size_t kMaxPools = 256;
std::mutex g_pool_mutex;
std::map<std::pair<int, cudaStream_t>, ForkPool> g_pools;

cudaError_t pool_setup(ForkPool& P) {
  if (P.ready) return cudaSuccess;
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < kForks && e == cudaSuccess; ++i) e = cudaStreamCreateWithFlags(&P.fork[i], cudaStreamNonBlocking);
  for (int i = 0; i <= kForks && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&P.ev[i], cudaEventDisableTiming);
  if (e == cudaSuccess) P.ready = true;
  return e;
}

// The pool of (dev, s); beyond kMaxPools caller streams, calls share the pool of the
// device's default stream.
ForkPool& pool_for(int dev, cudaStream_t s) {
  auto key = std::make_pair(dev, s);
  if (g_pools.size() >= kMaxPools && !g_pools.count(key)) key = std::make_pair(dev, (cudaStream_t) nullptr);
  return g_pools[key];
}

wef_status check_ops(const char* fn, const wef_op* ops, int nops, wef_precision prec, int* dev_out) {
  if (!ops || nops < 1 || nops > kMaxOps)
    return set_error(WEF_EINVAL, std::string(fn) + ": ops must hold 1 to " + std::to_string(kMaxOps) + " operators");
  if (prec != WEF_RADIAL_FP32 && prec != WEF_FP64)
    return set_error(WEF_EINVAL, std::string(fn) + ": ragged batches run WEF_RADIAL_FP32 or WEF_FP64 (plans run the "
                                                   "tensor-core paths)");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev)
    return set_error(WEF_ECUDA, std::string(fn) + ": no usable current device");
  for (int i = 0; i < nops; ++i) {
    if (!ops[i]) return set_error(WEF_EINVAL, std::string(fn) + ": NULL operator");
    if (!ops[i]->has_core) return set_error(WEF_ENOCORE, std::string(fn) + ": every operator needs an uploaded core");
    if (ops[i]->device != dev)
      return set_error(WEF_EINVAL, std::string(fn) + ": the current device is not the one an operator's core is on");
  }
  *dev_out = dev;
  return WEF_OK;
}

int64_t tile_bytes_bound(const wef_op* ops, int nops, int64_t ncells, wef_precision prec) {
  int64_t nmax = 1;
  for (int i = 0; i < nops; ++i) nmax = std::max<int64_t>(nmax, (int64_t)ops[i]->T.K * ops[i]->T.NQ);
  // sum over operators of ceil(count / 32) * 32 cells <= ncells + 31 * nops
  return (ncells + 31LL * nops) * nmax * (prec == WEF_FP64 ? 8 : 4);
}

}  // namespace

extern "C" {

wef_status wef_ragged_workspace_size(const wef_op* ops, int nops, int64_t ncells, wef_precision prec, int64_t* bytes) {
  return wef::guarded("wef_ragged_workspace_size", [&]() -> wef_status {
    if (!bytes || ncells < 0) return set_error(WEF_EINVAL, "wef_ragged_workspace_size: bad argument");
    if (!ops || nops < 1 || nops > kMaxOps)
      return set_error(WEF_EINVAL, "wef_ragged_workspace_size: ops must hold 1 to " + std::to_string(kMaxOps) +
                                       " operators");
    if (prec != WEF_RADIAL_FP32 && prec != WEF_FP64)
      return set_error(WEF_EINVAL, "wef_ragged_workspace_size: ragged batches run WEF_RADIAL_FP32 or WEF_FP64");
    for (int i = 0; i < nops; ++i)
      if (!ops[i]) return set_error(WEF_EINVAL, "wef_ragged_workspace_size: NULL operator");
    *bytes = kHeader + align256(ncells * 8) + align256(tile_bytes_bound(ops, nops, ncells, prec));
    return WEF_OK;
  });
}

wef_status wef_evaluate_ragged(const wef_op* ops, int nops, const int32_t* shape_id_dev, const int64_t* offset_dev,
                               const double* f_dev, double* q_dev, int64_t ncells, wef_precision prec,
                               void* workspace, int64_t ws_bytes, void* stream) {
  return wef::guarded("wef_evaluate_ragged", [&]() -> wef_status {
    int dev = 0;
    wef_status st = check_ops("wef_evaluate_ragged", ops, nops, prec, &dev);
    if (st != WEF_OK) return st;
    if (ncells < 0 || ncells > (int64_t)65535 * 32 * 1024)
      return set_error(WEF_EINVAL, "wef_evaluate_ragged: ncells out of range");
    if (ncells == 0) return WEF_OK;
    if (!shape_id_dev || !offset_dev || !f_dev || !q_dev || !workspace)
      return set_error(WEF_EINVAL, "wef_evaluate_ragged: NULL buffer");
    if (((uintptr_t)workspace & 255) != 0)
      return set_error(WEF_EINVAL, "wef_evaluate_ragged: workspace not 256-byte aligned");
    int64_t need = 0;
    st = wef_ragged_workspace_size(ops, nops, ncells, prec, &need);
    if (st != WEF_OK) return st;
    if (ws_bytes < need) return set_error(WEF_EINVAL, "wef_evaluate_ragged: workspace too small");
    for (int i = 0; i < nops; ++i)
      if (prec == WEF_RADIAL_FP32 && prepare_rf(ops[i]->T.K, ops[i]->T.rprog.n1max) != cudaSuccess)
        return set_error(WEF_ECUDA, "wef_evaluate_ragged: kernel attributes");
    cudaStream_t s = (cudaStream_t)stream;
    char* ws = (char*)workspace;
    int* count = (int*)(ws + kOffCount);
    int* cursor = (int*)(ws + kOffCursor);
    int* queue = (int*)(ws + kOffQueue);
    int64_t* list_base = (int64_t*)(ws + kOffListBase);
    int64_t* tile_first = (int64_t*)(ws + kOffTileFirst);
    int64_t* tile_off = (int64_t*)(ws + kOffTileOff);
    int64_t* lists = (int64_t*)(ws + kHeader);
    void* tiles = ws + kHeader + align256(ncells * 8);
    Shapes sh{};
    sh.nops = nops;
    int nmax = 1;
    for (int i = 0; i < nops; ++i) {
      sh.K[i] = ops[i]->T.K;
      sh.NQ[i] = ops[i]->T.NQ;
      nmax = std::max(nmax, sh.K[i] * sh.NQ[i]);
    }
    // set-up on the caller's stream: counts, list layout, lists, tiles
    cudaError_t e = cudaMemsetAsync(ws, 0, kOffListBase, s);
    const unsigned cgrid = (unsigned)((ncells + 255) / 256);
    if (e == cudaSuccess) {
      ragged_count<<<cgrid, 256, 0, s>>>(shape_id_dev, ncells, nops, count);
      ragged_prefix<<<1, 1, 0, s>>>(sh, count, list_base, tile_first, tile_off);
      ragged_scatter<<<cgrid, 256, 0, s>>>(shape_id_dev, offset_dev, ncells, nops, cursor, list_base, lists);
      const dim3 tgrid((unsigned)((ncells + 31) / 32 + nops), (unsigned)((nmax + 31) / 32));
      if (prec == WEF_FP64)
        ragged_tile<double><<<tgrid, dim3(32, 8), 0, s>>>(sh, f_dev, count, list_base, tile_first, tile_off, lists,
                                                          (double*)tiles);
      else
        ragged_tile<float><<<tgrid, dim3(32, 8), 0, s>>>(sh, f_dev, count, list_base, tile_first, tile_off, lists,
                                                         (float*)tiles);
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) return set_error(WEF_ECUDA, std::string("wef_evaluate_ragged: set-up: ") + cudaGetErrorString(e));
    // the operators' contractions on forked streams, most expensive per cell first
    std::vector<int> order(nops);
    for (int i = 0; i < nops; ++i) order[i] = i;
    auto cost = [&](int i) {
      const Tables& T = ops[i]->T;
      return prec == WEF_FP64 ? (double)T.K * T.K * T.K * T.n_sym_slices : T.rprog.fp64_flops + T.rprog.fp32_flops / 64.0;
    };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost(a) > cost(b); });
    std::lock_guard<std::mutex> lock(g_pool_mutex);
    ForkPool& P = pool_for(dev, s);
    e = pool_setup(P);
    if (e != cudaSuccess) return set_error(WEF_ECUDA, std::string("wef_evaluate_ragged: streams: ") + cudaGetErrorString(e));
    const int nf = std::min(kForks, nops);
    e = cudaEventRecord(P.ev[kForks], s);
    for (int i = 0; i < nf && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(P.fork[i], P.ev[kForks], 0);
    if (e != cudaSuccess) return set_error(WEF_ECUDA, std::string("wef_evaluate_ragged: fork: ") + cudaGetErrorString(e));
    cudaError_t le = cudaSuccess;
    for (int k = 0; k < nops && le == cudaSuccess; ++k) {
      const int i = order[k];
      wef_operator* op = ops[i];
      const RaggedView rv{count + i, tile_off + i, lists, list_base + i};
      cudaStream_t fs = P.fork[k % nf];
      if (prec == WEF_RADIAL_FP32) {
        const RadialProgram& RP = op->T.rprog;
        const DevRadial r{(const int4*)op->r_tasks, (const int4*)op->r_chans, (const int4*)op->r_blocks,
                          (const int4*)op->r_uents, (const double2*)op->r_pw, op->r_order,
                          (int)RP.task_cost.size(), RP.n1max};
        le = launch_rf_ragged(op->T.K, (const float*)tiles, queue + i, q_dev, ncells, op->T.NQ, r, op->d_R32, op->sms,
                              rv, fs);
      } else {
        const wef_operator::DevProg& D = op->dp[0];
        const int64_t ntiles = (ncells + 31) / 32;
        int idx = 0;
        while (idx + 1 < (int)D.chunk_n.size() && ntiles * D.chunk_n[idx] < 4LL * op->sms) ++idx;
        const DevProgram p{D.prog, (const int4*)D.groups, (const double2*)D.gw, D.off, op->T.prog1.ntasks()};
        le = launch_fp64(op->T.K, (const double*)tiles, q_dev, ncells, op->T.NQ, p, D.chunks + D.chunk_pos[idx],
                         D.chunk_n[idx], op->d_R64, fs, rv);
      }
    }
    // join every fork, also after a failed launch
    for (int i = 0; i < nf && e == cudaSuccess; ++i) {
      e = cudaEventRecord(P.ev[i], P.fork[i]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(s, P.ev[i], 0);
    }
    if (le != cudaSuccess)
      return set_error(WEF_ECUDA, std::string("wef_evaluate_ragged: contraction: ") + cudaGetErrorString(le));
    if (e != cudaSuccess) return set_error(WEF_ECUDA, std::string("wef_evaluate_ragged: join: ") + cudaGetErrorString(e));
    return WEF_OK;
  });
}

}  // extern "C"
