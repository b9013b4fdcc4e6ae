// The operator object behind the opaque wef_op handle (shared by the C ABI files).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "tables.hpp"

using wef::Channel;
using wef::Program;
using wef::Tables;

struct wef_operator {
  Tables T;
  double gamma = 0.0;
  int device = 0;
  int sms = 1;
  // programs: [0] one q1 per task (FP64 path), [1] four q1 per task (tensor-core path)
  struct DevProg {
    int32_t *prog = nullptr, *off = nullptr, *chunks = nullptr, *groups = nullptr;
    double* gw = nullptr;
    std::vector<int> chunk_n, chunk_pos;  // chunk counts available and their offsets in `chunks`
  } dp[2];
  int* d_status = nullptr;  // set by kernels whose bounded waits gave up
  // radial-first program
  int32_t *r_tasks = nullptr, *r_chans = nullptr, *r_blocks = nullptr, *r_uents = nullptr, *r_order = nullptr;
  double* r_pw = nullptr;
  // core
  double* d_R64 = nullptr;      // symmetrised core [sc][k3][k1][k2]
  uint8_t* d_Bbf16 = nullptr;   // packed MMA B tiles, BF16
  uint8_t* d_Btf32 = nullptr;   // packed MMA B tiles, TF32
  float* d_R32 = nullptr;       // symmetrised core, FP32 [sc][k1][k2][KP4] (radial-first path)
  uint8_t* d_Brft = nullptr;    // split-TF32 b tiles of the tensor-core radial-first stage 1
  bool has_core = false;
  // tracing
  cudaEvent_t trace_start = nullptr, trace_stop = nullptr;
  // baselines (naive COO, dense tensor): symmetrised entries sorted by q1, cuBLAS handle
  void* b_ent = nullptr;
  double* b_w = nullptr;
  int32_t* b_off = nullptr;
  int64_t b_nent = 0;
  void* cublas = nullptr;
  // evaluation from host memory: copy streams and events, created on first use
  bool io_ready = false;
  cudaStream_t io_stream[2] = {nullptr, nullptr};
  cudaEvent_t io_ev[7] = {};

  void release_baselines() {
    cudaFree(b_ent);
    cudaFree(b_w);
    cudaFree(b_off);
    b_ent = nullptr;
    b_w = nullptr;
    b_off = nullptr;
    b_nent = 0;
  }

  void release_core() {
    cudaFree(d_R64);
    cudaFree(d_Bbf16);
    cudaFree(d_Btf32);
    cudaFree(d_R32);
    cudaFree(d_Brft);
    d_R32 = nullptr;
    d_Brft = nullptr;
    d_R64 = nullptr;
    d_Bbf16 = d_Btf32 = nullptr;
    has_core = false;
  }
  void release() {
    for (auto& d : dp) {
      cudaFree(d.prog);
      cudaFree(d.off);
      cudaFree(d.groups);
      cudaFree(d.chunks);
      cudaFree(d.gw);
      d = DevProg();
    }
    cudaFree(d_status);
    d_status = nullptr;
    for (int32_t** pp : {&r_tasks, &r_chans, &r_blocks, &r_uents, &r_order}) {
      cudaFree(*pp);
      *pp = nullptr;
    }
    cudaFree(r_pw);
    r_pw = nullptr;
    release_baselines();
    if (io_ready) {
      for (cudaStream_t& s : io_stream) cudaStreamDestroy(s);
      for (cudaEvent_t& e : io_ev) cudaEventDestroy(e);
      io_ready = false;
    }
    release_core();
  }
};
