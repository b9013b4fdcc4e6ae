// C ABI of the library (declared in include/wef.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "../../include/wef.h"
#include "operator.hpp"
#include "wef_internal.hpp"

using namespace wef;

namespace {

thread_local std::string g_err;

wef_status fail(wef_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

wef_status cuda_fail(cudaError_t e, const char* what) {
  return fail(WEF_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

template <class T>
cudaError_t upload(T** dst, const std::vector<T>& src) {
  *dst = nullptr;
  if (src.empty()) return cudaSuccess;
  cudaError_t e = cudaMalloc((void**)dst, src.size() * sizeof(T));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
}

}  // namespace

wef_status wef::set_error(wef_status s, const std::string& msg) { return fail(s, msg); }


namespace {

// Device-side set-up (programs, chunk tables) on the current device; done at the
// first call that needs the GPU so that host-only use (tables, core building)
// works on machines without one.
cudaError_t ensure_device(wef_operator* op) {
  if (op->d_status) return cudaSuccess;
  cudaError_t e = cudaGetDevice(&op->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&op->sms, cudaDevAttrMultiProcessorCount, op->device);
  for (int v = 0; v < 2 && e == cudaSuccess; ++v) {
    const Program& P = v == 0 ? op->T.prog1 : op->T.prog4;
    wef_operator::DevProg& D = op->dp[v];
    e = upload(&D.prog, P.prog);
    if (e == cudaSuccess) e = upload(&D.groups, P.groups);
    if (e == cudaSuccess) e = upload(&D.gw, P.gw);
    if (e == cudaSuccess) e = upload(&D.off, P.task_off);
    if (e == cudaSuccess) {
      std::vector<int32_t> all;
      D.chunk_n.clear();
      D.chunk_pos.clear();
      for (int n = 1; n <= P.ntasks(); n *= 2) {
        std::vector<int32_t> b = split_tasks(P.task_cost, n);
        D.chunk_n.push_back((int)b.size() - 1);
        D.chunk_pos.push_back((int)all.size());
        all.insert(all.end(), b.begin(), b.end());
      }
      e = upload(&D.chunks, all);
    }
  }
  const RadialProgram& RP = op->T.rprog;
  if (e == cudaSuccess) e = upload(&op->r_tasks, RP.tasks);
  if (e == cudaSuccess) e = upload(&op->r_chans, RP.chans);
  if (e == cudaSuccess) e = upload(&op->r_blocks, RP.blocks);
  if (e == cudaSuccess) e = upload(&op->r_uents, RP.uents);
  if (e == cudaSuccess) e = upload(&op->r_pw, RP.pw);
  if (e == cudaSuccess) e = upload(&op->r_order, RP.order);
  if (e == cudaSuccess) e = cudaMalloc((void**)&op->d_status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(op->d_status, 0, sizeof(int));
  if (e != cudaSuccess) op->release();
  return e;
}

}  // namespace

extern "C" {

const char* wef_last_error(void) { return g_err.c_str(); }

wef_status wef_create(int kmax, int lmax, double gamma, wef_op* out) {
  return wef::guarded("wef_create", [&]() -> wef_status {
    if (!out) return fail(WEF_EINVAL, "wef_create: out is NULL");
    *out = nullptr;
    if (kmax < 0 || kmax > WEF_MAX_KMAX || lmax < 0 || lmax > WEF_MAX_LMAX)
      return fail(WEF_ESHAPE, "wef_create: Kmax must be in [0,16] and Lmax in [0,20]");
    if (!(gamma >= 0.0 && gamma <= 2.0)) return fail(WEF_EINVAL, "wef_create: gamma must be in [0, 2]");
    std::unique_ptr<wef_operator> op(new (std::nothrow) wef_operator());
    if (!op) return fail(WEF_ENOMEM, "wef_create: host allocation failed");
    op->gamma = gamma;
    std::string err = build_tables(kmax, lmax, op->T);
    if (!err.empty()) return fail(WEF_ESHAPE, "wef_create: " + err);
    *out = op.release();
    return WEF_OK;
  });
}

wef_status wef_sizes(wef_op op, int64_t* n_per_cell, int64_t* n_channels, int64_t* n_gaunt, int64_t* core_len) {
  if (!op) return fail(WEF_EINVAL, "wef_sizes: op is NULL");
  const int64_t K = op->T.K;
  if (n_per_cell) *n_per_cell = K * op->T.NQ;
  if (n_channels) *n_channels = (int64_t)op->T.chans.size();
  if (n_gaunt) *n_gaunt = (int64_t)op->T.g.size();
  if (core_len) *core_len = (int64_t)op->T.chans.size() * K * K * K;
  return WEF_OK;
}

wef_status wef_gaunt_coo(wef_op op, int32_t* q1, int32_t* q2, int32_t* q3, int32_t* c, double* g) {
  if (!op) return fail(WEF_EINVAL, "wef_gaunt_coo: op is NULL");
  const size_t n = op->T.g.size();
  if (q1) std::memcpy(q1, op->T.q1.data(), n * sizeof(int32_t));
  if (q2) std::memcpy(q2, op->T.q2.data(), n * sizeof(int32_t));
  if (q3) std::memcpy(q3, op->T.q3.data(), n * sizeof(int32_t));
  if (c) std::memcpy(c, op->T.c.data(), n * sizeof(int32_t));
  if (g) std::memcpy(g, op->T.g.data(), n * sizeof(double));
  return WEF_OK;
}

wef_status wef_upload_core(wef_op op, const double* R_host, int64_t len, unsigned flags) {
  return wef::guarded("wef_upload_core", [&]() -> wef_status {
    if (!op || !R_host) return fail(WEF_EINVAL, "wef_upload_core: NULL argument");
    const Tables& T = op->T;
    const int K = T.K;
    const int64_t K3 = (int64_t)K * K * K;
    const int64_t NT = (int64_t)T.chans.size();
    if (len != NT * K3) return fail(WEF_ESHAPE, "wef_upload_core: len must be N_T*K^3");
    if (op->d_status) {
      int dev = -1;
      if (cudaGetDevice(&dev) != cudaSuccess || dev != op->device)
        return fail(WEF_EINVAL, "wef_upload_core: the current device is not the one the operator was set up on");
    }
    cudaError_t de = ensure_device(op);
    if (de != cudaSuccess) return cuda_fail(de, "wef_upload_core: device set-up");
    std::vector<double> R(R_host, R_host + len);
    if (flags & WEF_CORE_APPLY_NULLSPACE) {
      for (int64_t c = 0; c < NT; ++c) {
        const Channel& h = T.chans[c];
        double* Rc = &R[c * K3];
        if (h.l1 == 0) {
          std::fill(Rc, Rc + K * K, 0.0);                              // mass, k1 = 0
          if (K > 1) std::fill(Rc + K * K, Rc + 2 * K * K, 0.0);       // energy, k1 = 1
        }
        if (h.l1 == 1) std::fill(Rc, Rc + K * K, 0.0);                 // momentum, k1 = 0
        if (h.l1 == 0 && h.l2 == 0 && h.l3 == 0)
          for (int k1 = 0; k1 < K; ++k1) Rc[(int64_t)k1 * K * K] = 0.0;  // detailed balance
      }
    }
    // symmetrised core Rt[sc] = R[c] + R[c']^{T23}, FP64 layout [sc][k3][k1][k2]
    const int NS = (int)T.sym_chan.size();
    std::vector<double> R64((size_t)NS * K3);
    for (int s = 0; s < NS; ++s) {
      const double* A = &R[(int64_t)T.sym_chan[s] * K3];
      const double* B = &R[(int64_t)T.sym_partner[s] * K3];
      for (int k1 = 0; k1 < K; ++k1)
        for (int k2 = 0; k2 < K; ++k2)
          for (int k3 = 0; k3 < K; ++k3) {
            const double v = A[(k1 * K + k2) * K + k3] + B[(k1 * K + k3) * K + k2];
            R64[(((size_t)s * K + k3) * K + k1) * K + k2] = v;
          }
    }
    // packed tensor-core B tiles of Rt[sc][k1][k2][k3] (from the FP64 layout [sc][k3][k1][k2])
    std::vector<uint8_t> Bb, Bt;
    if (K <= 17) {
      const int nb = tc_b_tile_bytes(K, false), nt = tc_b_tile_bytes(K, true);
      Bb.resize((size_t)NS * nb);
      Bt.resize((size_t)NS * nt);
      std::vector<double> Rt((size_t)K3);
      for (int s = 0; s < NS; ++s) {
        for (int k1 = 0; k1 < K; ++k1)
          for (int k2 = 0; k2 < K; ++k2)
            for (int k3 = 0; k3 < K; ++k3)
              Rt[((size_t)k1 * K + k2) * K + k3] = R64[(((size_t)s * K + k3) * K + k1) * K + k2];
        tc_pack_b_tile(K, false, Rt.data(), &Bb[(size_t)s * nb]);
        tc_pack_b_tile(K, true, Rt.data(), &Bt[(size_t)s * nt]);
      }
    }
    // FP32 copy for the radial-first path, layout [sc][k1][k2][k3 -> KP4]: rows over k3 (the
    // index the first radial stage produces, two per packed FMA) padded with zeros to whole
    // float4s.
    const int KP4 = rf_row_padded(K);
    std::vector<float> R32((size_t)NS * K * K * KP4, 0.0f);
    for (int s = 0; s < NS; ++s)
      for (int k1 = 0; k1 < K; ++k1)
        for (int k2 = 0; k2 < K; ++k2)
          for (int k3 = 0; k3 < K; ++k3)
            R32[(((size_t)s * K + k1) * K + k2) * KP4 + k3] = (float)R64[(((size_t)s * K + k3) * K + k1) * K + k2];
    // split-TF32 b tiles of the tensor-core first radial stage (WEF_RADIAL_TC), per channel
    std::vector<uint8_t> Brft;
    if (rft_supported(K)) {
      const size_t nb = 2 * (size_t)rft_b_tile_bytes(K);
      Brft.resize((size_t)NS * nb);
      std::vector<double> Rt((size_t)K3);
      for (int s = 0; s < NS; ++s) {
        for (int k1 = 0; k1 < K; ++k1)
          for (int k2 = 0; k2 < K; ++k2)
            for (int k3 = 0; k3 < K; ++k3)
              Rt[((size_t)k1 * K + k2) * K + k3] = R64[(((size_t)s * K + k3) * K + k1) * K + k2];
        rft_pack_b_tiles(K, Rt.data(), &Brft[(size_t)s * nb]);
      }
    }
    op->release_core();
    cudaError_t e = upload(&op->d_R64, R64);
    if (e == cudaSuccess) e = upload(&op->d_R32, R32);
    if (e == cudaSuccess) e = upload(&op->d_Brft, Brft);
    if (e == cudaSuccess) e = upload(&op->d_Bbf16, Bb);
    if (e == cudaSuccess) e = upload(&op->d_Btf32, Bt);
    if (e != cudaSuccess) {
      op->release_core();
      return cuda_fail(e, "wef_upload_core");
    }
    op->has_core = true;
    return WEF_OK;
  });
}

wef_status wef_workspace_size(wef_op op, int64_t ncells, wef_precision prec, int64_t* bytes) {
  if (!op || !bytes || ncells < 0) return fail(WEF_EINVAL, "wef_workspace_size: bad argument");
  if (!valid_eval_precision(prec)) return fail(WEF_EINVAL, "wef_workspace_size: unknown precision");
  const int64_t ntiles = (ncells + 31) / 32;
  const int64_t tile_elems = ntiles * 32 * (int64_t)op->T.K * op->T.NQ;
  *bytes = tile_elems * (int64_t)sizeof(double);
  if (radial_first(prec) && ncells > 0) {
    // queue word (256 bytes) + FP32 re-tiled f
    const int64_t rb = 256 + (tile_elems * (int64_t)sizeof(float) + 255) / 256 * 256;
    if (rb > *bytes) *bytes = rb;
  }
  return WEF_OK;
}

wef_status wef_evaluate(wef_op op, const double* f_dev, double* q_dev, int64_t ncells, wef_precision prec,
                        void* workspace, int64_t workspace_bytes, void* stream) {
  return wef::evaluate_grouped(op, f_dev, q_dev, ncells, prec, workspace, workspace_bytes, stream, 0);
}

}  // extern "C"

wef_status wef::evaluate_grouped(wef_op op, const double* f_dev, double* q_dev, int64_t ncells, wef_precision prec,
                                 void* workspace, int64_t workspace_bytes, void* stream, int64_t group_bytes) {
  return wef::guarded("wef_evaluate", [&]() -> wef_status {
    if (!op) return fail(WEF_EINVAL, "wef_evaluate: op is NULL");
    if (!valid_eval_precision(prec)) return fail(WEF_EINVAL, "wef_evaluate: unknown precision");
    if (prec == WEF_RADIAL_TC && !rft_supported(op->T.K))
      return fail(WEF_EINVAL, "wef_evaluate: WEF_RADIAL_TC is compiled for Kmax = 8, 10 and 12 only");
    if (ncells < 0) return fail(WEF_EINVAL, "wef_evaluate: ncells < 0");
    if (ncells == 0) return WEF_OK;
    if (!f_dev || !q_dev || !workspace) return fail(WEF_EINVAL, "wef_evaluate: NULL buffer");
    if (!op->has_core) return fail(WEF_ENOCORE, "wef_evaluate: no core uploaded");
    if (((uintptr_t)workspace & 255) != 0) return fail(WEF_EINVAL, "wef_evaluate: workspace not 256-byte aligned");
    int64_t need = 0;
    if (wef_workspace_size(op, ncells, prec, &need) != WEF_OK) return WEF_EINVAL;
    if (workspace_bytes < need) return fail(WEF_EINVAL, "wef_evaluate: workspace too small");
    if (ncells > (int64_t)65535 * 32 * 1024) return fail(WEF_EINVAL, "wef_evaluate: ncells too large");
    {
      int dev = -1;
      if (cudaGetDevice(&dev) != cudaSuccess || dev != op->device)
        return fail(WEF_EINVAL, "wef_evaluate: the current device is not the one the core was uploaded on");
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int K = op->T.K, NQ = op->T.NQ;
    if (prec == WEF_RADIAL_FP32) {
      const RadialProgram& RP = op->T.rprog;
      DevRadial r{(const int4*)op->r_tasks, (const int4*)op->r_chans, (const int4*)op->r_blocks,
                  (const int4*)op->r_uents, (const double2*)op->r_pw, op->r_order,
                  (int)RP.task_cost.size(), RP.n1max};
      cudaError_t er = launch_rf(K, f_dev, (float*)((char*)workspace + 256), (int*)workspace, q_dev, ncells, NQ, r,
                                 op->d_R32, op->sms, s, op->trace_start, op->trace_stop, group_bytes);
      if (er != cudaSuccess) return cuda_fail(er, "wef_evaluate: radial-first kernels");
      return WEF_OK;
    }
    if (prec == WEF_RADIAL_TC) {
      const RadialProgram& RP = op->T.rprog;
      DevRadial r{(const int4*)op->r_tasks, (const int4*)op->r_chans, (const int4*)op->r_blocks,
                  (const int4*)op->r_uents, (const double2*)op->r_pw, op->r_order,
                  (int)RP.task_cost.size(), RP.n1max};
      cudaError_t er = launch_rft(K, f_dev, (float*)((char*)workspace + 256), (int*)workspace, q_dev, ncells, NQ, r,
                                  op->d_Brft, op->sms, op->d_status, s, op->trace_start, op->trace_stop, group_bytes);
      if (er != cudaSuccess) return cuda_fail(er, "wef_evaluate: radial-first tensor-core kernels");
      return WEF_OK;
    }
    double* ftile = (double*)workspace;
    cudaError_t e = launch_tile_f(f_dev, ftile, ncells, K, NQ, s);
    if (e != cudaSuccess) return cuda_fail(e, "wef_evaluate: tile kernel");
    // chunk count: enough CTAs for several waves of the GPU
    const int v = prec == WEF_FP64 ? 0 : 1;
    const wef_operator::DevProg& D = op->dp[v];
    const int64_t ntiles = (ncells + 31) / 32;
    const int64_t want = 4LL * op->sms;
    int idx = 0;
    while (idx + 1 < (int)D.chunk_n.size() && ntiles * D.chunk_n[idx] < want) ++idx;
    const Program& P = v == 0 ? op->T.prog1 : op->T.prog4;
    DevProgram p{D.prog, (const int4*)D.groups, (const double2*)D.gw, D.off, P.ntasks()};
    if (op->trace_start) cudaEventRecord(op->trace_start, s);
    if (prec == WEF_FP64)
      e = launch_fp64(K, ftile, q_dev, ncells, NQ, p, D.chunks + D.chunk_pos[idx], D.chunk_n[idx], op->d_R64, s);
    else
      e = launch_tc(K, prec == WEF_MIXED_TF32, ftile, q_dev, ncells, NQ, p, D.chunks + D.chunk_pos[idx], D.chunk_n[idx],
                    prec == WEF_MIXED_TF32 ? op->d_Btf32 : op->d_Bbf16, op->d_status, s);
    if (op->trace_stop) cudaEventRecord(op->trace_stop, s);
    if (e != cudaSuccess) return cuda_fail(e, "wef_evaluate: contraction kernel");
    return WEF_OK;
  });
}

extern "C" {

wef_status wef_core_build(wef_op op, int pad_rad, int pad_ang, double* R_out, int64_t len) {
  return wef::guarded("wef_core_build", [&]() -> wef_status {
    if (!op || !R_out) return fail(WEF_EINVAL, "wef_core_build: NULL argument");
    const int64_t K = op->T.K;
    if (len != (int64_t)op->T.chans.size() * K * K * K) return fail(WEF_ESHAPE, "wef_core_build: len must be N_T*K^3");
    if (pad_rad < 0 || pad_ang < 0 || pad_rad > 200 || pad_ang > 200) return fail(WEF_EINVAL, "wef_core_build: bad padding");
    std::string err = core_build(op->T, op->gamma, pad_rad, pad_ang, R_out);
    if (!err.empty()) return fail(WEF_EINVAL, "wef_core_build: " + err);
    return WEF_OK;
  });
}

wef_status wef_flops(wef_op op, wef_precision prec, double* fp64_flops_per_cell, double* tc_flops_per_cell) {
  if (!op) return fail(WEF_EINVAL, "wef_flops: op is NULL");
  if (!valid_eval_precision(prec)) return fail(WEF_EINVAL, "wef_flops: unknown precision");
  if (prec == WEF_RADIAL_FP32) {
    if (fp64_flops_per_cell) *fp64_flops_per_cell = op->T.rprog.fp64_flops;
    if (tc_flops_per_cell) *tc_flops_per_cell = op->T.rprog.fp32_flops;
    return WEF_OK;
  }
  if (prec == WEF_RADIAL_TC) {
    // tensor-core stage 1 as executed: per q2 group, three TF32 products of a 128-row tile
    // (the 32 cells four times) by 16 k2 by 16 K columns, i.e. per cell 4 x 3 x 2 x 16 x 16 K
    const int K = op->T.K;
    if (fp64_flops_per_cell) *fp64_flops_per_cell = op->T.rprog.fp64_flops;
    if (tc_flops_per_cell) *tc_flops_per_cell = (double)op->T.rprog.n_groups * 4.0 * 3.0 * 2.0 * 16.0 * 16.0 * K;
    return WEF_OK;
  }
  const Program& P = prec == WEF_FP64 ? op->T.prog1 : op->T.prog4;
  double f64 = 0.0;
  for (double c : P.task_cost) f64 += c;
  double tc = 0.0;
  if (prec != WEF_FP64) {
    // radial stage on the tensor cores: per task and channel, a 128-row tile times
    // the padded K^2 x N operand; per cell that is (128/32) rows per task and channel
    const int K = op->T.K;
    const int kpad = prec == WEF_MIXED_BF16 ? (K * K + 15) / 16 * 16 : (K * K + 7) / 8 * 8;
    const int npad = (K + 15) / 16 * 16;
    for (int t = 0; t < P.ntasks(); ++t) {
      const int nchan = P.prog[P.task_off[t] + 2];
      tc += 2.0 * 4.0 * kpad * npad * nchan;
    }
  }
  if (fp64_flops_per_cell) *fp64_flops_per_cell = f64;
  if (tc_flops_per_cell) *tc_flops_per_cell = tc;
  return WEF_OK;
}

wef_status wef_set_trace_events(wef_op op, void* ev_start, void* ev_stop) {
  if (!op) return fail(WEF_EINVAL, "wef_set_trace_events: op is NULL");
  op->trace_start = (cudaEvent_t)ev_start;
  op->trace_stop = (cudaEvent_t)ev_stop;
  return WEF_OK;
}

wef_status wef_device_status(wef_op op, int reset) {
  if (!op) return fail(WEF_EINVAL, "wef_device_status: op is NULL");
  if (!op->d_status) return WEF_OK;
  int h = 0;
  cudaError_t e = cudaMemcpy(&h, op->d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "wef_device_status");
  if (reset) cudaMemset(op->d_status, 0, sizeof(int));
  if (h != 0) return fail(WEF_ETIMEOUT, "a bounded device-side wait gave up in an earlier evaluation");
  return WEF_OK;
}

wef_status wef_destroy(wef_op op) {
  if (!op) return WEF_OK;
  if (op->cublas) wef::destroy_cublas(op->cublas);
  op->release();
  delete op;
  return WEF_OK;
}

}  // extern "C"
