// GPU baselines for the factorised contraction (paper Sec. 4.5): the same Q(f, f)
// evaluated the two unfactorised ways the paper compares against, on the same GPU.
//  * naive COO (Sec. 4.5.2): for every non-zero Gaunt entry (q1, q2, q3, c) the full
//    K^3 radial sum  Q[k1,q1] += g * sum_{k2,k3} R_c[k1,k2,k3] f[k2,q2] f[k3,q3];
//  * dense tensor (Sec. 4.5.1): C[a1][a2][a3] assembled once on the device, then
//    Q_a1 = sum_{a2,a3} C[a1][a2][a3] f_a2 f_a3 for a batch as two cuBLAS FP64 GEMMs.
// Both work on the symmetrised entries (l2 <= l3; for l2 = l3 only q2 <= q3 with the
// diagonal weight halved) and the symmetrised core, which give the same Q.
#include <cublas_v2.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/wef.h"
#include "operator.hpp"
#include "wef_internal.hpp"

namespace {

struct SymEntry {
  int q2, q3, sc, pad;
};

// Symmetrised COO sorted by q1, with per-q1 offsets; uploaded on first use.
cudaError_t ensure_entries(wef_operator* op) {
  if (op->b_ent) return cudaSuccess;
  const Tables& T = op->T;
  std::vector<int> sym_of(T.chans.size(), -1);
  for (size_t s = 0; s < T.sym_chan.size(); ++s) sym_of[T.sym_chan[s]] = (int)s;
  std::vector<std::vector<std::pair<SymEntry, double>>> by_q1(T.NQ);
  for (size_t z = 0; z < T.g.size(); ++z) {
    const Channel& h = T.chans[T.c[z]];
    const int sc = sym_of[T.c[z]];
    if (sc < 0) continue;
    double w = T.g[z];
    if (h.l2 == h.l3) {
      if (T.q2[z] > T.q3[z]) continue;
      if (T.q2[z] == T.q3[z]) w *= 0.5;
    }
    by_q1[T.q1[z]].push_back({{T.q2[z], T.q3[z], sc, 0}, w});
  }
  std::vector<SymEntry> ent;
  std::vector<double> wt;
  std::vector<int32_t> off(1, 0);
  for (int q = 0; q < T.NQ; ++q) {
    for (const auto& p : by_q1[q]) {
      ent.push_back(p.first);
      wt.push_back(p.second);
    }
    off.push_back((int32_t)ent.size());
  }
  cudaError_t e = cudaMalloc((void**)&op->b_ent, std::max<size_t>(ent.size(), 1) * sizeof(SymEntry));
  if (e == cudaSuccess) e = cudaMalloc((void**)&op->b_w, std::max<size_t>(wt.size(), 1) * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void**)&op->b_off, off.size() * sizeof(int32_t));
  if (e == cudaSuccess && !ent.empty())
    e = cudaMemcpy(op->b_ent, ent.data(), ent.size() * sizeof(SymEntry), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !wt.empty()) e = cudaMemcpy(op->b_w, wt.data(), wt.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(op->b_off, off.data(), off.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
  op->b_nent = (int64_t)ent.size();
  if (e != cudaSuccess) op->release_baselines();
  return e;
}

// CTA = (32-cell tile, q1), warp = k1, lane = cell.  R64 layout [sc][k3][k1][k2].
__global__ void naive_coo_kernel(const double* __restrict__ ftile, double* __restrict__ q, int64_t ncells, int K, int NQ,
                                 const int4* __restrict__ ent, const double* __restrict__ wt,
                                 const int32_t* __restrict__ off, const double* __restrict__ R64) {
  const int k1 = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t tile = blockIdx.x;
  const int q1 = blockIdx.y;
  const double* ft = ftile + tile * (int64_t)NQ * K * 32 + lane;
  double acc = 0.0;
  for (int z = off[q1]; z < off[q1 + 1]; ++z) {
    const int4 E = __ldg(ent + z);  // q2, q3, sc
    const double* f2 = ft + (int64_t)E.x * K * 32;
    const double* f3 = ft + (int64_t)E.y * K * 32;
    const double* R = R64 + (int64_t)E.z * K * K * K + (int64_t)k1 * K;
    double s = 0.0;
    for (int k3 = 0; k3 < K; ++k3) {
      double t = 0.0;
      for (int k2 = 0; k2 < K; ++k2) t = fma(__ldg(R + (int64_t)k3 * K * K + k2), f2[k2 * 32], t);
      s = fma(t, f3[k3 * 32], s);
    }
    acc = fma(__ldg(wt + z), s, acc);
  }
  const int64_t cell = tile * 32 + lane;
  if (cell < ncells) {
    if ((k1 == 0 && q1 < 4) || (k1 == 1 && q1 == 0)) acc = 0.0;  // conservation projection
    q[cell * (int64_t)K * NQ + (int64_t)k1 * NQ + q1] = acc;
  }
}

// C[((k1 NQ + q1) N + (k2 NQ + q2)) N + (k3 NQ + q3)] = w * Rt[sc][k1][k2][k3] over all
// symmetrised entries (each (q1, q2, q3) occurs once, so plain stores suffice).
__global__ void dense_assemble_kernel(double* __restrict__ C, int K, int NQ, int64_t nent, const int4* __restrict__ ent,
                                      const double* __restrict__ wt, const int32_t* __restrict__ off,
                                      const double* __restrict__ R64) {
  const int64_t N = (int64_t)K * NQ, K3 = (int64_t)K * K * K;
  const int64_t total = nent * K3;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t z = i / K3;
    const int r = (int)(i - z * K3);
    const int k3 = r / (K * K), k1 = (r / K) % K, k2 = r % K;  // R64 order [k3][k1][k2]
    // q1 of entry z: last q with off[q] <= z
    int lo = 0, hi = NQ - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (off[mid] <= z) lo = mid; else hi = mid - 1;
    }
    const int4 E = ent[z];
    const int64_t a1 = (int64_t)k1 * NQ + lo, a2 = (int64_t)k2 * NQ + E.x, a3 = (int64_t)k3 * NQ + E.y;
    // conservation projection: the rows of the mass, momentum and energy outputs stay zero
    const bool invariant = (k1 == 0 && lo < 4) || (k1 == 1 && lo == 0);
    C[(a1 * N + a2) * N + a3] = invariant ? 0.0 : wt[z] * R64[(int64_t)E.z * K3 + r];
  }
}

cudaError_t ensure_cublas(wef_operator* op) {
  if (op->cublas) return cudaSuccess;
  cublasHandle_t h = nullptr;
  if (cublasCreate(&h) != CUBLAS_STATUS_SUCCESS) return cudaErrorUnknown;
  op->cublas = h;
  return cudaSuccess;
}

int64_t dense_n(const wef_operator* op) { return (int64_t)op->T.K * op->T.NQ; }

}  // namespace

void wef::destroy_cublas(void* handle) { cublasDestroy((cublasHandle_t)handle); }

extern "C" {

wef_status wef_naive_evaluate(wef_op op, const double* f_dev, double* q_dev, int64_t ncells, void* workspace,
                              int64_t ws_bytes, void* stream) {
  return wef::guarded("wef_naive_evaluate", [&]() -> wef_status {
    if (!op || ncells < 0) return wef::set_error(WEF_EINVAL, "wef_naive_evaluate: bad argument");
    if (ncells == 0) return WEF_OK;
    if (!f_dev || !q_dev || !workspace) return wef::set_error(WEF_EINVAL, "wef_naive_evaluate: NULL buffer");
    if (!op->has_core) return wef::set_error(WEF_ENOCORE, "wef_naive_evaluate: no core uploaded");
    if (((uintptr_t)workspace & 255) != 0)
      return wef::set_error(WEF_EINVAL, "wef_naive_evaluate: workspace not 256-byte aligned");
    int64_t need = 0;
    wef_workspace_size(op, ncells, WEF_FP64, &need);
    if (ws_bytes < need) return wef::set_error(WEF_EINVAL, "wef_naive_evaluate: workspace too small");
    if (ncells > (int64_t)65535 * 32 * 1024) return wef::set_error(WEF_EINVAL, "wef_naive_evaluate: ncells too large");
    cudaError_t e = ensure_entries(op);
    if (e != cudaSuccess) return wef::set_error(WEF_ECUDA, std::string("wef_naive_evaluate: ") + cudaGetErrorString(e));
    const int K = op->T.K, NQ = op->T.NQ;
    cudaStream_t s = (cudaStream_t)stream;
    double* ftile = (double*)workspace;
    e = wef::launch_tile_f(f_dev, ftile, ncells, K, NQ, s);
    if (e == cudaSuccess) {
      const int64_t ntiles = (ncells + 31) / 32;
      naive_coo_kernel<<<dim3((unsigned)ntiles, (unsigned)NQ), 32 * K, 0, s>>>(
          ftile, q_dev, ncells, K, NQ, (const int4*)op->b_ent, op->b_w, op->b_off, op->d_R64);
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) return wef::set_error(WEF_ECUDA, std::string("wef_naive_evaluate: ") + cudaGetErrorString(e));
    return WEF_OK;
  });
}

wef_status wef_dense_tensor_size(wef_op op, int64_t* bytes) {
  if (!op || !bytes) return wef::set_error(WEF_EINVAL, "wef_dense_tensor_size: bad argument");
  const int64_t N = dense_n(op);
  *bytes = N * N * N * (int64_t)sizeof(double);
  return WEF_OK;
}

wef_status wef_dense_assemble(wef_op op, double* C_dev, int64_t bytes, void* stream) {
  return wef::guarded("wef_dense_assemble", [&]() -> wef_status {
    if (!op || !C_dev) return wef::set_error(WEF_EINVAL, "wef_dense_assemble: bad argument");
    if (!op->has_core) return wef::set_error(WEF_ENOCORE, "wef_dense_assemble: no core uploaded");
    int64_t need = 0;
    wef_dense_tensor_size(op, &need);
    if (bytes < need) return wef::set_error(WEF_EINVAL, "wef_dense_assemble: buffer too small");
    cudaError_t e = ensure_entries(op);
    cudaStream_t s = (cudaStream_t)stream;
    if (e == cudaSuccess) e = cudaMemsetAsync(C_dev, 0, (size_t)need, s);
    if (e == cudaSuccess && op->b_nent > 0) {
      dense_assemble_kernel<<<op->sms * 8, 256, 0, s>>>(C_dev, op->T.K, op->T.NQ, op->b_nent, (const int4*)op->b_ent,
                                                         op->b_w, op->b_off, op->d_R64);
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) return wef::set_error(WEF_ECUDA, std::string("wef_dense_assemble: ") + cudaGetErrorString(e));
    return WEF_OK;
  });
}

wef_status wef_dense_workspace_size(wef_op op, int64_t ncells, int64_t* bytes) {
  if (!op || !bytes || ncells < 0) return wef::set_error(WEF_EINVAL, "wef_dense_workspace_size: bad argument");
  const int64_t N = dense_n(op);
  *bytes = N * N * std::min<int64_t>(std::max<int64_t>(ncells, 1), 256) * (int64_t)sizeof(double);
  return WEF_OK;
}

wef_status wef_dense_evaluate(wef_op op, const double* C_dev, const double* f_dev, double* q_dev, int64_t ncells,
                              void* workspace, int64_t ws_bytes, void* stream) {
  if (!op || ncells < 0) return wef::set_error(WEF_EINVAL, "wef_dense_evaluate: bad argument");
  if (ncells == 0) return WEF_OK;
  if (!C_dev || !f_dev || !q_dev || !workspace) return wef::set_error(WEF_EINVAL, "wef_dense_evaluate: NULL buffer");
  const int64_t N = dense_n(op);
  const int64_t chunk = ws_bytes / (N * N * (int64_t)sizeof(double));
  if (chunk < 1) return wef::set_error(WEF_EINVAL, "wef_dense_evaluate: workspace smaller than one cell (N^2 doubles)");
  if (ensure_cublas(op) != cudaSuccess) return wef::set_error(WEF_ECUDA, "wef_dense_evaluate: cublasCreate failed");
  cublasHandle_t h = (cublasHandle_t)op->cublas;
  if (cublasSetStream(h, (cudaStream_t)stream) != CUBLAS_STATUS_SUCCESS)
    return wef::set_error(WEF_ECUDA, "wef_dense_evaluate: cublasSetStream failed");
  double* Tm = (double*)workspace;
  const double one = 1.0, zero = 0.0;
  for (int64_t c0 = 0; c0 < ncells; c0 += chunk) {
    const int nc = (int)std::min<int64_t>(chunk, ncells - c0);
    const double* F = f_dev + c0 * N;
    // T[(a1 N + a2), cell] = sum_a3 C[a1][a2][a3] f[cell][a3]   (column-major views)
    cublasStatus_t st = cublasDgemm(h, CUBLAS_OP_T, CUBLAS_OP_N, (int)(N * N), nc, (int)N, &one, C_dev, (int)N, F,
                                    (int)N, &zero, Tm, (int)(N * N));
    // Q[cell][a1] = sum_a2 T[(a1 N + a2), cell] f[cell][a2]
    if (st == CUBLAS_STATUS_SUCCESS)
      st = cublasDgemmStridedBatched(h, CUBLAS_OP_T, CUBLAS_OP_N, (int)N, 1, (int)N, &one, Tm, (int)N, N * N, F, (int)N,
                                     N, &zero, q_dev + c0 * N, (int)N, N, nc);
    if (st != CUBLAS_STATUS_SUCCESS)
      return wef::set_error(WEF_ECUDA, "wef_dense_evaluate: cuBLAS status " + std::to_string((int)st));
  }
  return WEF_OK;
}

}  // extern "C"
