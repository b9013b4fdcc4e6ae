// FP64 angular coupling of one slice (paper Sec. 4.5.4):
//   Phi[k2] (column k3 of this thread) = sum over the slice's rank-1 groups of
//   f[k2][q2] * h,   h = sum over the group's one or two entries of g * f[k3][q3].
// Groups are 16-byte records {q2, ne, q3a, q3b} with a weight pair {ga, gb}, one
// vector load each; all loads of a group are independent of its FMAs' results, so
// the few warps per SM keep the FP64 pipe fed without software pipelining (which
// only raised register pressure).
#pragma once
#include <cstdint>

namespace wef {

template <int K>
__device__ __forceinline__ void phi_slice(double (&Phi)[K], const int4* __restrict__ grp, const double2* __restrict__ gw,
                                          int g0, int ng, const double* __restrict__ ft, int k3) {
#pragma unroll
  for (int k = 0; k < K; ++k) Phi[k] = 0.0;
  for (int i = 0; i < ng; ++i) {
    const int4 G = __ldg(grp + g0 + i);
    const double2 W = __ldg(gw + g0 + i);
    double h = W.x * __ldg(ft + (G.z * K + k3) * 32);
    if (G.y > 1) h = fma(W.y, __ldg(ft + (G.w * K + k3) * 32), h);
    const double* f2 = ft + G.x * K * 32;
#pragma unroll
    for (int k2 = 0; k2 < K; ++k2) Phi[k2] = fma(__ldg(f2 + k2 * 32), h, Phi[k2]);
  }
}

}  // namespace wef
