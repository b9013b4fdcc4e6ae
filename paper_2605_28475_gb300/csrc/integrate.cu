// Time integration and linearization on the device:
//  * wef_integrate: classical fourth-order Runge-Kutta for the spatially homogeneous
//    equation df/dt = Q(f, f) (paper Sec. 2.1; explicit RK time stepping as in Sec. 5.3.2),
//    in place, every cell independent;
//  * wef_linearized_apply: L d at a base state c0, L = dQ/dc |_{c0} (Sec. 5.3.1), from the
//    polarization identity of the bilinear form, L d = Q(c0 + d) - Q(c0) - Q(d).
// Both call wef_evaluate for Q and combine states with small FP64 kernels.
#include <cuda_runtime.h>

#include <string>

#include "../../include/wef.h"
#include "wef_internal.hpp"

namespace {

// out = x + a * y
__global__ void axpy_kernel(int64_t n, const double* __restrict__ x, double a, const double* __restrict__ y,
                            double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = fma(a, y[i], x[i]);
}

// y += h/6 (k1 + 2 k2 + 2 k3 + k4)
__global__ void rk4_update_kernel(int64_t n, double* __restrict__ y, double h6, const double* __restrict__ k1,
                                  const double* __restrict__ k2, const double* __restrict__ k3,
                                  const double* __restrict__ k4) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = fma(h6, (k1[i] + k4[i]) + 2.0 * (k2[i] + k3[i]), y[i]);
}

// out = p - q - r
__global__ void polar_kernel(int64_t n, const double* __restrict__ p, const double* __restrict__ q,
                             const double* __restrict__ r, double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (p[i] - q[i]) - r[i];
}

int grid_for(int64_t n) {
  int64_t g = (n + 255) / 256;
  return (int)(g < 152 * 8 ? (g < 1 ? 1 : g) : 152 * 8);
}

int64_t align256(int64_t b) { return (b + 255) / 256 * 256; }

}  // namespace

extern "C" {

wef_status wef_integrate_workspace_size(wef_op op, int64_t ncells, wef_precision prec, int64_t* bytes) {
  if (!op || !bytes || ncells < 0) return wef::set_error(WEF_EINVAL, "wef_integrate_workspace_size: bad argument");
  int64_t n = 0, ev = 0;
  wef_status st = wef_sizes(op, &n, nullptr, nullptr, nullptr);
  if (st == WEF_OK) st = wef_workspace_size(op, ncells, prec, &ev);
  if (st != WEF_OK) return st;
  *bytes = align256(ev) + 5 * align256(ncells * n * (int64_t)sizeof(double));
  return WEF_OK;
}

wef_status wef_integrate(wef_op op, double* f_dev, int64_t ncells, double dt, int nsteps, wef_precision prec,
                         void* workspace, int64_t ws_bytes, void* stream) {
  if (!op || ncells < 0 || nsteps < 0) return wef::set_error(WEF_EINVAL, "wef_integrate: bad argument");
  if (ncells == 0 || nsteps == 0) return WEF_OK;
  if (!f_dev || !workspace) return wef::set_error(WEF_EINVAL, "wef_integrate: NULL buffer");
  int64_t need = 0, n = 0, ev = 0;
  wef_status st0 = wef_integrate_workspace_size(op, ncells, prec, &need);
  if (st0 != WEF_OK) return st0;
  if (ws_bytes < need) return wef::set_error(WEF_EINVAL, "wef_integrate: workspace too small");
  wef_sizes(op, &n, nullptr, nullptr, nullptr);
  wef_workspace_size(op, ncells, prec, &ev);
  const int64_t len = ncells * n, sb = align256(len * (int64_t)sizeof(double));
  char* base = (char*)workspace;
  void* ews = base;
  double* k[4];
  for (int i = 0; i < 4; ++i) k[i] = (double*)(base + align256(ev) + i * sb);
  double* tmp = (double*)(base + align256(ev) + 4 * sb);
  cudaStream_t s = (cudaStream_t)stream;
  const int g = grid_for(len);
  for (int step = 0; step < nsteps; ++step) {
    wef_status st = wef_evaluate(op, f_dev, k[0], ncells, prec, ews, ev, stream);
    if (st != WEF_OK) return st;
    axpy_kernel<<<g, 256, 0, s>>>(len, f_dev, 0.5 * dt, k[0], tmp);
    if ((st = wef_evaluate(op, tmp, k[1], ncells, prec, ews, ev, stream)) != WEF_OK) return st;
    axpy_kernel<<<g, 256, 0, s>>>(len, f_dev, 0.5 * dt, k[1], tmp);
    if ((st = wef_evaluate(op, tmp, k[2], ncells, prec, ews, ev, stream)) != WEF_OK) return st;
    axpy_kernel<<<g, 256, 0, s>>>(len, f_dev, dt, k[2], tmp);
    if ((st = wef_evaluate(op, tmp, k[3], ncells, prec, ews, ev, stream)) != WEF_OK) return st;
    rk4_update_kernel<<<g, 256, 0, s>>>(len, f_dev, dt / 6.0, k[0], k[1], k[2], k[3]);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return wef::set_error(WEF_ECUDA, std::string("wef_integrate: ") + cudaGetErrorString(e));
  }
  return WEF_OK;
}

wef_status wef_linearized_apply(wef_op op, const double* c0_dev, const double* d_dev, double* out_dev, int64_t ncells,
                                wef_precision prec, void* workspace, int64_t ws_bytes, void* stream) {
  if (!op || ncells < 0) return wef::set_error(WEF_EINVAL, "wef_linearized_apply: bad argument");
  if (ncells == 0) return WEF_OK;
  if (!c0_dev || !d_dev || !out_dev || !workspace)
    return wef::set_error(WEF_EINVAL, "wef_linearized_apply: NULL buffer");
  int64_t need = 0, n = 0, ev = 0;
  wef_status st0 = wef_integrate_workspace_size(op, ncells, prec, &need);
  if (st0 != WEF_OK) return st0;
  if (ws_bytes < need) return wef::set_error(WEF_EINVAL, "wef_linearized_apply: workspace too small");
  wef_sizes(op, &n, nullptr, nullptr, nullptr);
  wef_workspace_size(op, ncells, prec, &ev);
  const int64_t len = ncells * n, sb = align256(len * (int64_t)sizeof(double));
  char* base = (char*)workspace;
  double* sum = (double*)(base + align256(ev));
  double* qs = (double*)(base + align256(ev) + sb);
  double* q0 = (double*)(base + align256(ev) + 2 * sb);
  double* qd = (double*)(base + align256(ev) + 3 * sb);
  cudaStream_t s = (cudaStream_t)stream;
  const int g = grid_for(len);
  axpy_kernel<<<g, 256, 0, s>>>(len, c0_dev, 1.0, d_dev, sum);
  wef_status st = wef_evaluate(op, sum, qs, ncells, prec, base, ev, stream);
  if (st == WEF_OK) st = wef_evaluate(op, c0_dev, q0, ncells, prec, base, ev, stream);
  if (st == WEF_OK) st = wef_evaluate(op, d_dev, qd, ncells, prec, base, ev, stream);
  if (st != WEF_OK) return st;
  polar_kernel<<<g, 256, 0, s>>>(len, qs, q0, qd, out_dev);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return wef::set_error(WEF_ECUDA, std::string("wef_linearized_apply: ") + cudaGetErrorString(e));
  return WEF_OK;
}

}  // extern "C"
