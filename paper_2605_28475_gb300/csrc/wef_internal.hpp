// Internal interfaces between the C ABI layer and the kernel launchers.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "tables.hpp"

namespace wef {

// Device copy of one Program (see tables.hpp).
struct DevProgram {
  const int32_t* prog = nullptr;
  const double* progw = nullptr;
  const int32_t* task_off = nullptr;
  const int32_t* task_w = nullptr;
  int ntasks = 0;
};

constexpr int kCellsPerTile = 32;

// f[ncells][K][NQ] -> ftile[tile][q][k][32] (zero-padded tail cells).
cudaError_t launch_tile_f(const double* f, double* ftile, int64_t ncells, int K, int NQ, cudaStream_t s);

// FP64 angular coupling + FP64 radial contraction + conservation projection.
// chunks: device array of nchunks+1 task bounds.
cudaError_t launch_fp64(int K, const double* ftile, double* q, int64_t ncells, int NQ, const DevProgram& p,
                        const int32_t* chunks, int nchunks, const double* R64, cudaStream_t s);

// Tensor-core path: bytes of one packed core tile (MMA B operand) and its packing.
int tc_b_tile_bytes(int K, bool tf32);
void tc_pack_b_tile(int K, bool tf32, const double* Rt /* [k1][k2][k3] */, uint8_t* out);

// FP64 angular coupling + BF16/TF32 tcgen05 radial contraction + FP64 projection.
// status: device int set to 1 if a bounded wait inside the kernel gave up.
cudaError_t launch_tc(int K, bool tf32, const double* ftile, double* q, int64_t ncells, int NQ, const DevProgram& p,
                      const int32_t* chunks, int nchunks, const uint8_t* Btiles, int* status, cudaStream_t s);

std::string core_build(const Tables& T, double gamma, int pad_rad, int pad_ang, double* R);

}  // namespace wef
