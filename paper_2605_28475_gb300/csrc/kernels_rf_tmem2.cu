// Radial-first kernel with its FP64 accumulators in tensor memory and the register budget
// of several CTAs per SM (the dispatch is in kernels_rf.cu).
#include <cuda_runtime.h>

#include "rf_kernel.cuh"
#include "wef_internal.hpp"

namespace wef {

cudaError_t launch_rf_tmem2(int K, const float* ftile32, int* queue, double* q, int64_t ncells, int NQ,
                           const DevRadial& r, const float* R32, int nsm, cudaStream_t s, cudaEvent_t ev0,
                           cudaEvent_t ev1, const RaggedView& rv, int64_t group_bytes) {
  switch (K) {
#define WEF_RF(k) \
  case k:         \
    return rfk::launch_rf_k<k, kRfAccTmem2>(ftile32, queue, q, ncells, NQ, r, R32, nsm, s, ev0, ev1, rv, group_bytes);
    WEF_RF(1) WEF_RF(2) WEF_RF(3) WEF_RF(4) WEF_RF(5) WEF_RF(6) WEF_RF(7) WEF_RF(8) WEF_RF(9) WEF_RF(10) WEF_RF(11)
    WEF_RF(12) WEF_RF(13) WEF_RF(14) WEF_RF(15) WEF_RF(16) WEF_RF(17)
#undef WEF_RF
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace wef
