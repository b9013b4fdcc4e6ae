// Allocation-free variant of the FP64 evaluation (wef_evaluate_noalloc).
//
// Some callers cannot call cudaMalloc at the point where they evaluate the
// operator: a solver whose device memory is owned entirely by its own pool (or
// by another framework's caching allocator) and that must not grow the
// footprint behind that pool's back; code running in a host callback or a
// latency-critical loop, where cudaMalloc's implicit device-wide
// synchronisation is not allowed; tools that must not change the memory
// footprint after start-up.  For them the scratch that wef_evaluate takes as a
// caller-supplied workspace (the 32-cell re-tiled copy of f) lives here, in a
// file-scope device array of fixed size that every GPU loading this library
// keeps until the process exits.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/wef.h"
#include "wef_internal.hpp"

namespace {

// The scratch array; its size is WEF_NOALLOC_SCRATCH_BYTES.
static __device__ __align__(256) double g_noalloc_scratch[WEF_NOALLOC_SCRATCH_BYTES / sizeof(double)];

// Device address of g_noalloc_scratch per device, looked up once per device.
// In host code the array's name is only a host-side stand-in, never a device address.
constexpr int kMaxDevices = 128;
std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};

}  // namespace

extern "C" wef_status wef_evaluate_noalloc(wef_op op, const double* f_dev, double* q_dev, int64_t ncells,
                                           void* stream) {
  return wef::guarded("wef_evaluate_noalloc", [&]() -> wef_status {
  if (!op) return wef::set_error(WEF_EINVAL, "wef_evaluate_noalloc: op is NULL");
  if (ncells < 0) return wef::set_error(WEF_EINVAL, "wef_evaluate_noalloc: ncells < 0");
  int64_t need = 0;
  wef_status st = wef_workspace_size(op, ncells, WEF_FP64, &need);
  if (st != WEF_OK) return st;
  if (need > (int64_t)WEF_NOALLOC_SCRATCH_BYTES) {
    int64_t per_tile = 0;
    wef_workspace_size(op, 32, WEF_FP64, &per_tile);
    const int64_t max_cells = per_tile > 0 ? (int64_t)WEF_NOALLOC_SCRATCH_BYTES / per_tile * 32 : 0;
    return wef::set_error(WEF_EINVAL, "wef_evaluate_noalloc: ncells = " + std::to_string(ncells) +
                                          " exceeds the fixed scratch (at most " + std::to_string(max_cells) +
                                          " cells for this operator); use wef_evaluate with a workspace");
  }
  if (ncells == 0) return WEF_OK;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return wef::set_error(WEF_ECUDA, "wef_evaluate_noalloc: no usable current device");
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
      // set-up, once per device, with that device current.  This is also where CUDA's lazy
      // module loading brings in the module holding the array (its 16 MiB become resident,
      // with an implicit device synchronisation): a reason more to make the first call at set-up.
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p)
        return wef::set_error(WEF_ECUDA, std::string("wef_evaluate_noalloc: scratch set-up: ") + cudaGetErrorString(e));
      g_scratch_addr[dev] = p;
    }
    scratch = g_scratch_addr[dev];
  }
  // The re-tiling kernel overwrites every scratch byte it later reads (tail cells
  // are written as zeros), so nothing needs clearing between calls.
  return wef_evaluate(op, f_dev, q_dev, ncells, WEF_FP64, scratch, (int64_t)WEF_NOALLOC_SCRATCH_BYTES, stream);
  });
}
