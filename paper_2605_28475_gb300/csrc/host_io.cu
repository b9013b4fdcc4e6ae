// Evaluation from host memory: f is streamed to the device in chunks, evaluated and
// streamed back, with the copies of one chunk overlapping the evaluation of the next.
// Two staging slots for f and two for Q live in the caller's workspace; host-to-device
// and device-to-host copies run on two library streams, the evaluations on the caller's
// stream, ordered by events:
//   H2D(i) after eval(i-2) freed its f slot;  eval(i) after H2D(i) and D2H(i-2);
//   D2H(i) after eval(i).
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "../../include/wef.h"
#include "operator.hpp"
#include "wef_internal.hpp"

namespace {

int64_t al256(int64_t b) { return (b + 255) / 256 * 256; }

cudaError_t ensure_io(wef_operator* op) {
  if (op->io_ready) return cudaSuccess;
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaStreamCreateWithFlags(&op->io_stream[i], cudaStreamNonBlocking);
  for (int i = 0; i < 7 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&op->io_ev[i], cudaEventDisableTiming);
  if (e == cudaSuccess) op->io_ready = true;
  return e;
}

}  // namespace

extern "C" {

wef_status wef_host_workspace_size(wef_op op, int64_t chunk_cells, wef_precision prec, int64_t* bytes) {
  if (!op || !bytes || chunk_cells < 1) return wef::set_error(WEF_EINVAL, "wef_host_workspace_size: bad argument");
  int64_t n = 0, ev = 0;
  wef_status st = wef_sizes(op, &n, nullptr, nullptr, nullptr);
  if (st == WEF_OK) st = wef_workspace_size(op, chunk_cells, prec, &ev);
  if (st != WEF_OK) return st;
  *bytes = al256(ev) + 4 * al256(chunk_cells * n * (int64_t)sizeof(double));
  return WEF_OK;
}

wef_status wef_evaluate_host(wef_op op, const double* f_host, double* q_host, int64_t ncells, int64_t chunk_cells,
                             wef_precision prec, void* workspace, int64_t ws_bytes, void* stream) {
  if (!op || ncells < 0 || chunk_cells < 1) return wef::set_error(WEF_EINVAL, "wef_evaluate_host: bad argument");
  if (ncells == 0) return WEF_OK;
  if (!f_host || !q_host || !workspace) return wef::set_error(WEF_EINVAL, "wef_evaluate_host: NULL buffer");
  if (((uintptr_t)workspace & 255) != 0) return wef::set_error(WEF_EINVAL, "wef_evaluate_host: workspace not 256-byte aligned");
  int64_t need = 0, n = 0, ev = 0;
  wef_status st = wef_host_workspace_size(op, chunk_cells, prec, &need);
  if (st != WEF_OK) return st;
  if (ws_bytes < need) return wef::set_error(WEF_EINVAL, "wef_evaluate_host: workspace too small");
  wef_sizes(op, &n, nullptr, nullptr, nullptr);
  wef_workspace_size(op, chunk_cells, prec, &ev);
  cudaError_t e = ensure_io(op);
  if (e != cudaSuccess) return wef::set_error(WEF_ECUDA, std::string("wef_evaluate_host: ") + cudaGetErrorString(e));
  const int64_t slot = al256(chunk_cells * n * (int64_t)sizeof(double));
  char* base = (char*)workspace;
  void* ews = base;
  double* fs[2] = {(double*)(base + al256(ev)), (double*)(base + al256(ev) + slot)};
  double* qs[2] = {(double*)(base + al256(ev) + 2 * slot), (double*)(base + al256(ev) + 3 * slot)};
  cudaStream_t cs = (cudaStream_t)stream, h2d = op->io_stream[0], d2h = op->io_stream[1];
  cudaEvent_t* E = op->io_ev;  // [0,1] H2D done, [2,3] evaluation done, [4,5] D2H done, [6] entry
  // the copy streams start after everything already queued on the caller's stream
  e = cudaEventRecord(E[6], cs);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h2d, E[6], 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(d2h, E[6], 0);
  const int64_t nchunks = (ncells + chunk_cells - 1) / chunk_cells;
  for (int64_t i = 0; i < nchunks && e == cudaSuccess; ++i) {
    const int s = (int)(i & 1);
    const int64_t c0 = i * chunk_cells, nc = std::min(chunk_cells, ncells - c0);
    const size_t bytes = (size_t)(nc * n) * sizeof(double);
    if (i >= 2) e = cudaStreamWaitEvent(h2d, E[2 + s], 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(fs[s], f_host + c0 * n, bytes, cudaMemcpyHostToDevice, h2d);
    if (e == cudaSuccess) e = cudaEventRecord(E[s], h2d);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, E[s], 0);
    if (e == cudaSuccess && i >= 2) e = cudaStreamWaitEvent(cs, E[4 + s], 0);
    if (e != cudaSuccess) break;
    st = wef_evaluate(op, fs[s], qs[s], nc, prec, ews, ev, stream);
    if (st != WEF_OK) return st;
    e = cudaEventRecord(E[2 + s], cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(d2h, E[2 + s], 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(q_host + c0 * n, qs[s], bytes, cudaMemcpyDeviceToHost, d2h);
    if (e == cudaSuccess) e = cudaEventRecord(E[4 + s], d2h);
  }
  // the caller's stream completes with the last copies back
  for (int s = 0; s < 2 && e == cudaSuccess; ++s)
    if (nchunks > s) e = cudaStreamWaitEvent(cs, E[4 + ((nchunks - 1 - s) & 1)], 0);
  if (e != cudaSuccess) return wef::set_error(WEF_ECUDA, std::string("wef_evaluate_host: ") + cudaGetErrorString(e));
  return WEF_OK;
}

}  // extern "C"
