// FP64 kernels: cell-tile transpose and the plain FP64 angular-first contraction
// (paper Sec. 4.5.4; angular coupling Phi in FP64 followed by the radial
// contraction with the symmetrised core, plus the Sec. 4.4 conservation projection).
//
// Thread mapping of the contraction kernels: one CTA owns a tile of 32 cells;
// warp w is the radial index k3 = w (K warps), lane = cell.  Every lane of every
// warp does useful FP64 work (GB300's FP64 pipe saturates with a few full warps
// per SM and partially filled warps waste it), and the whole CTA walks the same
// warp-uniform instruction stream (the Program built on the host).
#include <cuda_runtime.h>

#include "phi.cuh"
#include "wef_internal.hpp"

namespace wef {

namespace {

// ftile[tile][q][k][32] = f[tile*32 + lane][k][q]; grid (ntiles, ceil(N/32)), block (32, 8).
__global__ void tile_f_kernel(const double* __restrict__ f, double* __restrict__ ftile, int64_t ncells, int K, int NQ) {
  __shared__ double s[32][33];
  const int N = K * NQ;
  const int64_t tile = blockIdx.x;
  const int a0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int j = ty; j < 32; j += 8) {
    const int64_t cell = tile * 32 + j;
    const int a = a0 + tx;
    s[j][tx] = (cell < ncells && a < N) ? f[cell * N + a] : 0.0;
  }
  __syncthreads();
  for (int j = ty; j < 32; j += 8) {
    const int a = a0 + j;
    if (a < N) {
      const int k = a / NQ, q = a - k * NQ;
      ftile[((tile * NQ + q) * K + k) * 32 + tx] = s[tx][j];
    }
  }
}

template <int K>
__global__ void __launch_bounds__(32 * K) fp64_kernel(const double* __restrict__ ftile, double* __restrict__ qout,
                                                      int64_t ncells, int NQ, const int32_t* __restrict__ prog,
                                                      const int4* __restrict__ groups, const double2* __restrict__ gw,
                                                      const int32_t* __restrict__ task_off,
                                                      const int32_t* __restrict__ chunks,
                                                      const double* __restrict__ R64, RaggedView rv) {
  extern __shared__ double red[];  // [k3][k1][32]
  const int k3 = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t tile = blockIdx.x;
  if (rv.count) {  // one shape of a ragged batch: the grid is an upper bound of its tiles
    ncells = *rv.count;
    if (tile * 32 >= ncells) return;
    ftile += *rv.tile_off;
    rv.cells += *rv.cells_off;
  }
  const int t0 = chunks[blockIdx.y], t1 = chunks[blockIdx.y + 1];
  const double* ft = ftile + tile * (int64_t)NQ * K * 32 + lane;
  const int64_t cell = tile * 32 + lane;
  double* qcell = qout + (cell < ncells && rv.cells ? rv.cells[cell] : cell * (int64_t)K * NQ);
  for (int t = t0; t < t1; ++t) {
    const int32_t* p = prog + task_off[t];
    const int q1 = __ldg(p);
    const int nchan = __ldg(p + 2);
    p += 3;
    double P[K];
#pragma unroll
    for (int k = 0; k < K; ++k) P[k] = 0.0;
    for (int ci = 0; ci < nchan; ++ci) {
      const int sc = __ldg(p), g0 = __ldg(p + 1), ng = __ldg(p + 2);
      p += 3;
      double Phi[K];
      phi_slice<K>(Phi, groups, gw, g0, ng, ft, k3);
      // radial contraction with the symmetrised core, layout R64[sc][k3][k1][k2]
      const double* Rs = R64 + ((int64_t)sc * K + k3) * K * K;
#pragma unroll
      for (int k1 = 0; k1 < K; ++k1) {
        double acc = P[k1];
#pragma unroll
        for (int k2 = 0; k2 < K; ++k2) acc = fma(__ldg(Rs + k1 * K + k2), Phi[k2], acc);
        P[k1] = acc;
      }
    }
    // sum the partial results over k3 (the warps) in a fixed order
#pragma unroll
    for (int k1 = 0; k1 < K; ++k1) red[(k3 * K + k1) * 32 + lane] = P[k1];
    __syncthreads();
    {
      const int k1 = k3;
      double s = 0.0;
#pragma unroll
      for (int j = 0; j < K; ++j) s += red[(j * K + k1) * 32 + lane];
      // conservation projection: mass (k=0,l=0), momentum (k=0,l=1), energy (k=1,l=0)
      if ((k1 == 0 && q1 < 4) || (k1 == 1 && q1 == 0)) s = 0.0;
      if (cell < ncells) qcell[(int64_t)k1 * NQ + q1] = s;
    }
    __syncthreads();
  }
}

// ncells: the cells of a one-shape call, or (rv.count set) an upper bound of the shape's
// cells in a ragged batch, which sizes the grid.
template <int K>
cudaError_t launch_fp64_k(const double* ftile, double* q, int64_t ncells, int NQ, const DevProgram& p,
                          const int32_t* chunks, int nchunks, const double* R64, cudaStream_t s,
                          const RaggedView& rv) {
  const int64_t ntiles = (ncells + 31) / 32;
  const size_t smem = (size_t)K * K * 32 * sizeof(double);
  static std::atomic<size_t> attr[kMaxDevices];
  cudaError_t e = smem_opt_in(fp64_kernel<K>, smem, attr);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)ntiles, (unsigned)nchunks);
  fp64_kernel<K><<<grid, 32 * K, smem, s>>>(ftile, q, ncells, NQ, p.prog, p.groups, p.gw, p.task_off, chunks, R64, rv);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_tile_f(const double* f, double* ftile, int64_t ncells, int K, int NQ, cudaStream_t s) {
  const int64_t ntiles = (ncells + 31) / 32;
  const int N = K * NQ;
  dim3 grid((unsigned)ntiles, (unsigned)((N + 31) / 32));
  tile_f_kernel<<<grid, dim3(32, 8), 0, s>>>(f, ftile, ncells, K, NQ);
  return cudaGetLastError();
}

cudaError_t launch_fp64(int K, const double* ftile, double* q, int64_t ncells, int NQ, const DevProgram& p,
                        const int32_t* chunks, int nchunks, const double* R64, cudaStream_t s, const RaggedView& rv) {
  switch (K) {
#define WEF_CASE(k) \
  case k:           \
    return launch_fp64_k<k>(ftile, q, ncells, NQ, p, chunks, nchunks, R64, s, rv);
    WEF_CASE(1) WEF_CASE(2) WEF_CASE(3) WEF_CASE(4) WEF_CASE(5) WEF_CASE(6) WEF_CASE(7) WEF_CASE(8) WEF_CASE(9)
    WEF_CASE(10) WEF_CASE(11) WEF_CASE(12) WEF_CASE(13) WEF_CASE(14) WEF_CASE(15) WEF_CASE(16) WEF_CASE(17)
#undef WEF_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace wef
