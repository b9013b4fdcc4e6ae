// Ragged batches: one plan covers cells of several (Kmax, Lmax) operators laid out
// back to back in one buffer; it runs as one re-tiling launch plus one persistent
// tensor-core launch that pulls (shape, tile, task range) items from a device
// queue, optionally replayed from a captured CUDA graph.  Item granularity is
// picked by a timing autotuner whose choices can be cached in a file.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <memory>
#include <new>
#include <sstream>
#include <string>
#include <vector>

#include "../../include/wef.h"
#include "operator.hpp"
#include "wef_internal.hpp"

using namespace wef;

namespace {

// Every tile of every shape: ftile[shape region][tile][q][k][32] = f[shape cells][k][q].
__global__ void ragged_tile_f_kernel(const RaggedShape* __restrict__ shapes, int nshapes, const double* __restrict__ f,
                                     double* __restrict__ ftile) {
  __shared__ double s[32][33];
  __shared__ int sh;
  const int64_t gt = blockIdx.x;
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    int lo = 0, hi = nshapes - 1;  // last shape with tile0 <= gt
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (shapes[mid].tile0 <= gt) lo = mid; else hi = mid - 1;
    }
    sh = lo;
  }
  __syncthreads();
  const RaggedShape& S = shapes[sh];
  const int K = S.K, NQ = S.NQ, N = K * NQ;
  const int a0 = blockIdx.y * 32;
  if (a0 >= N) return;
  const int64_t tile = gt - S.tile0;
  const double* fs = f + S.f_off;
  double* ft = ftile + S.ftile_off;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int j = ty; j < 32; j += 8) {
    const int64_t cell = tile * 32 + j;
    const int a = a0 + tx;
    s[j][tx] = (cell < S.ncells && a < N) ? fs[cell * N + a] : 0.0;
  }
  __syncthreads();
  for (int j = ty; j < 32; j += 8) {
    const int a = a0 + j;
    if (a < N) {
      const int k = a / NQ, q = a - k * NQ;
      ft[((tile * NQ + q) * K + k) * 32 + tx] = s[tx][j];
    }
  }
}

}  // namespace

namespace wef {

cudaError_t launch_ragged_tile_f(const RaggedShape* shapes, int nshapes, int64_t total_tiles, int max_n,
                                 const double* f, double* ftile, cudaStream_t s) {
  dim3 grid((unsigned)total_tiles, (unsigned)((max_n + 31) / 32));
  ragged_tile_f_kernel<<<grid, dim3(32, 8), 0, s>>>(shapes, nshapes, f, ftile);
  return cudaGetLastError();
}

}  // namespace wef

struct wef_plan_s {
  std::vector<wef_op> ops;
  std::vector<int64_t> ncells;
  wef_precision prec = WEF_MIXED_TF32;
  int max_k = 2, max_n = 1, nsm = 1;
  int64_t total_tiles = 0, ws_bytes = 0, total_cells = 0;
  std::vector<RaggedShape> shapes;
  RaggedShape* d_shapes = nullptr;
  RaggedItem* d_items = nullptr;
  int nitems = 0, items_cap = 0, granularity = 1;
  int* d_queue = nullptr;
  int* d_status = nullptr;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t gexec = nullptr;
  const void *g_f = nullptr, *g_q = nullptr, *g_ws = nullptr;
  std::string key;
  // radial-first plans: one evaluation per shape, spread over `nfork` forked streams
  static constexpr int kMaxFork = 8;
  std::vector<int64_t> rf_ws_off, rf_ws_len;
  std::vector<int> rf_order;  // shapes by decreasing cost
  cudaStream_t fork[kMaxFork] = {};
  cudaEvent_t fork_ev[kMaxFork + 1] = {};
  int nfork = 4;
  int group_mb = 0;  // L2 tile-group size of the shapes' launches, MB (0: the default)

  void release() {
    for (auto& s : fork)
      if (s) cudaStreamDestroy(s), s = nullptr;
    for (auto& e : fork_ev)
      if (e) cudaEventDestroy(e), e = nullptr;
    cudaFree(d_shapes);
    cudaFree(d_items);
    cudaFree(d_queue);
    cudaFree(d_status);
    if (gexec) cudaGraphExecDestroy(gexec);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    d_shapes = nullptr;
    d_items = nullptr;
    d_queue = d_status = nullptr;
    gexec = nullptr;
    cap_stream = nullptr;
  }
};

namespace {

// Items for granularity g: each tile of each shape split into about g cost-balanced
// task ranges; longest items first.
std::vector<RaggedItem> make_items(const wef_plan_s& P, int g) {
  struct Costed {
    double c;
    RaggedItem it;
  };
  std::vector<Costed> v;
  for (size_t s = 0; s < P.ops.size(); ++s) {
    const Program& prog = P.ops[s]->T.prog4;
    std::vector<int32_t> b = split_tasks(prog.task_cost, g);
    const int64_t ntiles = (P.ncells[s] + 31) / 32;
    for (size_t j = 0; j + 1 < b.size(); ++j) {
      double c = 0.0;
      for (int t = b[j]; t < b[j + 1]; ++t) c += prog.task_cost[t];
      for (int64_t tile = 0; tile < ntiles; ++tile) v.push_back({c, {(int)s, (int)tile, b[j], b[j + 1]}});
    }
  }
  std::stable_sort(v.begin(), v.end(), [](const Costed& a, const Costed& b) { return a.c > b.c; });
  std::vector<RaggedItem> out(v.size());
  for (size_t i = 0; i < v.size(); ++i) out[i] = v[i].it;
  return out;
}

wef_status set_items(wef_plan_s* P, int g) {
  std::vector<RaggedItem> it = make_items(*P, g);
  if ((int)it.size() > P->items_cap) {
    cudaFree(P->d_items);
    P->d_items = nullptr;
    cudaError_t e = cudaMalloc((void**)&P->d_items, it.size() * sizeof(RaggedItem));
    if (e != cudaSuccess) return set_error(WEF_ENOMEM, "wef_plan: item buffer allocation failed");
    P->items_cap = (int)it.size();
  }
  cudaError_t e = cudaMemcpy(P->d_items, it.data(), it.size() * sizeof(RaggedItem), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return set_error(WEF_ECUDA, std::string("wef_plan: item upload: ") + cudaGetErrorString(e));
  P->nitems = (int)it.size();
  P->granularity = g;
  if (P->gexec) {  // captured graphs bake in the item count
    cudaGraphExecDestroy(P->gexec);
    P->gexec = nullptr;
  }
  return WEF_OK;
}

std::string cache_path() {
  const char* p = std::getenv("WEF_TUNE_CACHE");
  return p ? std::string(p) : std::string();
}

int cache_lookup(const std::string& key) {
  const std::string path = cache_path();
  if (path.empty()) return 0;
  std::ifstream in(path);
  std::string k;
  int g;
  int found = 0;
  while (in >> k >> g)
    if (k == key) found = g;
  return found;
}

void cache_store(const std::string& key, int g) {
  const std::string path = cache_path();
  if (path.empty()) return;
  std::ofstream out(path, std::ios::app);
  out << key << " " << g << "\n";
}

wef_status check_buffers(wef_plan_s* P, const double* f, double* q, void* ws, int64_t ws_bytes) {
  if (!f || !q || !ws) return set_error(WEF_EINVAL, "wef_plan: NULL buffer");
  if (((uintptr_t)ws & 255) != 0) return set_error(WEF_EINVAL, "wef_plan: workspace not 256-byte aligned");
  if (ws_bytes < P->ws_bytes) return set_error(WEF_EINVAL, "wef_plan: workspace too small");
  return WEF_OK;
}

// Radial-first plan: the shapes' evaluations, largest first, round-robin over the forked
// streams (fork from and join back to `s`, so the launch also captures into one graph).
wef_status plan_launch_rf(wef_plan_s* P, const double* f, double* q, void* ws, cudaStream_t s) {
  const int nf = std::max(1, std::min(P->nfork, wef_plan_s::kMaxFork));
  cudaError_t e = cudaEventRecord(P->fork_ev[wef_plan_s::kMaxFork], s);
  for (int i = 0; i < nf && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(P->fork[i], P->fork_ev[wef_plan_s::kMaxFork], 0);
  if (e != cudaSuccess) return set_error(WEF_ECUDA, std::string("wef_plan: fork: ") + cudaGetErrorString(e));
  int k = 0;
  wef_status st = WEF_OK;
  for (int si : P->rf_order) {
    const RaggedShape& S = P->shapes[si];
    if (S.ncells == 0) continue;
    st = evaluate_grouped(P->ops[si], f + S.f_off, q + S.q_off, S.ncells, WEF_RADIAL_FP32,
                          (char*)ws + P->rf_ws_off[si], P->rf_ws_len[si], P->fork[k % nf],
                          (int64_t)P->group_mb << 20);
    if (st != WEF_OK) break;
    ++k;
  }
  // join every fork even after a failure, so that a stream capture never ends with
  // unjoined work
  for (int i = 0; i < nf && e == cudaSuccess; ++i) {
    e = cudaEventRecord(P->fork_ev[i], P->fork[i]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, P->fork_ev[i], 0);
  }
  if (st != WEF_OK) return st;
  if (e != cudaSuccess) return set_error(WEF_ECUDA, std::string("wef_plan: join: ") + cudaGetErrorString(e));
  return WEF_OK;
}

wef_status plan_launch(wef_plan_s* P, const double* f, double* q, void* ws, cudaStream_t s) {
  if (P->total_cells == 0) return WEF_OK;
  if (P->prec == WEF_RADIAL_FP32) return plan_launch_rf(P, f, q, ws, s);
  cudaError_t e = launch_ragged_tile_f(P->d_shapes, (int)P->shapes.size(), P->total_tiles, P->max_n, f, (double*)ws, s);
  if (e == cudaSuccess)
    e = launch_ragged_tc(P->prec == WEF_MIXED_TF32, P->max_k, P->nsm, P->d_shapes, P->d_items, P->nitems, P->d_queue,
                         (const double*)ws, q, P->d_status, s);
  if (e != cudaSuccess) return set_error(WEF_ECUDA, std::string("wef_plan: launch: ") + cudaGetErrorString(e));
  return WEF_OK;
}

}  // namespace

extern "C" {

wef_status wef_plan_create(const wef_op* ops, const int64_t* ncells, int nops, wef_precision prec, int granularity,
                           wef_plan* out) {
  return wef::guarded("wef_plan_create", [&]() -> wef_status {
    if (!out || !ops || !ncells || nops <= 0) return set_error(WEF_EINVAL, "wef_plan_create: bad argument");
    *out = nullptr;
    const bool rf = prec == WEF_RADIAL_FP32;
    if (prec != WEF_MIXED_TF32 && prec != WEF_MIXED_BF16 && !rf)
      return set_error(WEF_EINVAL, "wef_plan_create: ragged plans run the tensor-core (BF16, TF32) or radial-first path");
    wef_plan_s* P = new (std::nothrow) wef_plan_s();
    if (!P) return set_error(WEF_ENOMEM, "wef_plan_create: host allocation failed");
    // owns the plan until it is handed out: every early return (and any exception)
    // releases its device resources
    std::unique_ptr<wef_plan_s, void (*)(wef_plan_s*)> hold(P, [](wef_plan_s* x) {
      x->release();
      delete x;
    });
    P->prec = prec;
    std::ostringstream key;
    key << (rf ? "rf32" : prec == WEF_MIXED_TF32 ? "tf32" : "bf16");
    int64_t tile0 = 0, fo = 0, wo = 0;
    for (int i = 0; i < nops; ++i) {
      wef_op op = ops[i];
      if (!op || ncells[i] < 0) {
        return set_error(WEF_EINVAL, "wef_plan_create: NULL operator or negative count");
      }
      if (!op->has_core || !op->d_Bbf16) {
        return set_error(WEF_ENOCORE, "wef_plan_create: every operator needs an uploaded core");
      }
      if (op->T.K < 2 && !rf) {
        return set_error(WEF_ESHAPE, "wef_plan_create: the tensor-core path needs Kmax >= 1");
      }
      RaggedShape S{};
      S.K = op->T.K;
      S.NQ = op->T.NQ;
      S.ncells = ncells[i];
      S.tile0 = tile0;
      S.f_off = fo;
      S.q_off = fo;
      S.ftile_off = wo;
      S.prog = op->dp[1].prog;
      S.groups = (const int4*)op->dp[1].groups;
      S.gw = (const double2*)op->dp[1].gw;
      S.task_off = op->dp[1].off;
      S.Bbf16 = op->d_Bbf16;
      S.Btf32 = op->d_Btf32;
      const int64_t nt = (ncells[i] + 31) / 32;
      const int64_t N = (int64_t)S.K * S.NQ;
      tile0 += nt;
      fo += ncells[i] * N;
      wo += nt * 32 * N;
      P->ops.push_back(op);
      P->ncells.push_back(ncells[i]);
      P->shapes.push_back(S);
      P->max_k = std::max(P->max_k, S.K);
      P->max_n = std::max(P->max_n, (int)N);
      P->total_cells += ncells[i];
      key << "_" << (S.K - 1) << "x" << op->T.lmax << "x" << ncells[i];
      P->nsm = op->sms;
    }
    P->total_tiles = tile0;
    P->ws_bytes = wo * (int64_t)sizeof(double);
    if (rf) {
      // one radial-first workspace per shape (they run concurrently), 256-byte aligned
      int64_t off = 0;
      std::vector<double> cost;
      for (size_t i = 0; i < P->ops.size(); ++i) {
        int64_t b = 0;
        wef_workspace_size(P->ops[i], P->ncells[i], WEF_RADIAL_FP32, &b);
        b = std::max<int64_t>((b + 255) / 256 * 256, 256);
        P->rf_ws_off.push_back(off);
        P->rf_ws_len.push_back(b);
        off += b;
        cost.push_back((double)P->ncells[i] * (P->ops[i]->T.rprog.fp64_flops + P->ops[i]->T.rprog.fp32_flops / 64.0));
        P->rf_order.push_back((int)i);
      }
      std::stable_sort(P->rf_order.begin(), P->rf_order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
      P->ws_bytes = off;
    }
    cudaDeviceProp prop;
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) key << "_" << prop.name;
    P->key = key.str();
    for (auto& ch : P->key)
      if (ch == ' ') ch = '-';
    cudaError_t e = cudaMalloc((void**)&P->d_shapes, P->shapes.size() * sizeof(RaggedShape));
    if (e == cudaSuccess)
      e = cudaMemcpy(P->d_shapes, P->shapes.data(), P->shapes.size() * sizeof(RaggedShape), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc((void**)&P->d_queue, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void**)&P->d_status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(P->d_status, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&P->cap_stream, cudaStreamNonBlocking);
    for (int i = 0; rf && i < wef_plan_s::kMaxFork && e == cudaSuccess; ++i)
      e = cudaStreamCreateWithFlags(&P->fork[i], cudaStreamNonBlocking);
    for (int i = 0; rf && i <= wef_plan_s::kMaxFork && e == cudaSuccess; ++i)
      e = cudaEventCreateWithFlags(&P->fork_ev[i], cudaEventDisableTiming);
    if (e != cudaSuccess) return set_error(WEF_ECUDA, std::string("wef_plan_create: ") + cudaGetErrorString(e));
    if (rf) {
      // the tuned quantity is the number of concurrent shape streams
      // tuned value: streams + 16 * tile-group MB (an explicit granularity gives the streams)
      const int v = granularity > 0 ? granularity : cache_lookup(P->key);
      const int nf = v % 16;
      P->nfork = nf > 0 ? std::min(nf, (int)wef_plan_s::kMaxFork) : 4;
      P->group_mb = granularity > 0 ? 0 : v / 16;
      P->granularity = P->nfork + 16 * P->group_mb;
      // kernel attributes of every shape now, outside any later stream capture
      for (size_t i = 0; i < P->ops.size() && e == cudaSuccess; ++i)
        e = prepare_rf(P->ops[i]->T.K, P->ops[i]->T.rprog.n1max);
      if (e != cudaSuccess) return set_error(WEF_ECUDA, std::string("wef_plan_create: ") + cudaGetErrorString(e));
      *out = hold.release();
      return WEF_OK;
    }
    // granularity: explicit, cached from an earlier autotune, or enough items for ~8 per SM
    int g = granularity;
    if (g <= 0) g = cache_lookup(P->key);
    if (g <= 0) {
      g = 1;
      while (g < 64 && (int64_t)P->total_tiles * g < 8LL * P->nsm) g *= 2;
    }
    wef_status st = set_items(P, g);
    if (st != WEF_OK) return st;
    // kernel attributes now, outside any later stream capture
    e = prepare_ragged_tc();
    if (e != cudaSuccess) return set_error(WEF_ECUDA, std::string("wef_plan_create: ") + cudaGetErrorString(e));
    *out = hold.release();
    return WEF_OK;
  });
}

wef_status wef_plan_workspace_size(wef_plan plan, int64_t* bytes) {
  if (!plan || !bytes) return set_error(WEF_EINVAL, "wef_plan_workspace_size: NULL argument");
  *bytes = plan->ws_bytes;
  return WEF_OK;
}

wef_status wef_plan_execute(wef_plan plan, const double* f_dev, double* q_dev, void* workspace, int64_t ws_bytes,
                            void* stream) {
  return wef::guarded("wef_plan_execute", [&]() -> wef_status {
    if (!plan) return set_error(WEF_EINVAL, "wef_plan_execute: plan is NULL");
    wef_status st = check_buffers(plan, f_dev, q_dev, workspace, ws_bytes);
    if (st != WEF_OK) return st;
    return plan_launch(plan, f_dev, q_dev, workspace, (cudaStream_t)stream);
  });
}

wef_status wef_plan_graph_launch(wef_plan plan, const double* f_dev, double* q_dev, void* workspace, int64_t ws_bytes,
                                 void* stream) {
  return wef::guarded("wef_plan_graph_launch", [&]() -> wef_status {
    if (!plan) return set_error(WEF_EINVAL, "wef_plan_graph_launch: plan is NULL");
    wef_status st = check_buffers(plan, f_dev, q_dev, workspace, ws_bytes);
    if (st != WEF_OK) return st;
    if (plan->total_cells == 0) return WEF_OK;
    if (plan->gexec && (plan->g_f != f_dev || plan->g_q != q_dev || plan->g_ws != workspace)) {
      cudaGraphExecDestroy(plan->gexec);
      plan->gexec = nullptr;
    }
    if (!plan->gexec) {
      // first call (or new buffers): capture the two launches on the plan's own stream
      cudaGraph_t graph = nullptr;
      cudaError_t e = cudaStreamBeginCapture(plan->cap_stream, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return set_error(WEF_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
      wef_status ls = plan_launch(plan, f_dev, q_dev, workspace, plan->cap_stream);
      e = cudaStreamEndCapture(plan->cap_stream, &graph);
      if (ls != WEF_OK) {
        if (graph) cudaGraphDestroy(graph);
        return ls;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&plan->gexec, graph, 0);
      if (graph) cudaGraphDestroy(graph);
      if (e != cudaSuccess) return set_error(WEF_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
      plan->g_f = f_dev;
      plan->g_q = q_dev;
      plan->g_ws = workspace;
    }
    cudaError_t e = cudaGraphLaunch(plan->gexec, (cudaStream_t)stream);
    if (e != cudaSuccess) return set_error(WEF_ECUDA, std::string("graph launch: ") + cudaGetErrorString(e));
    return WEF_OK;
  });
}

wef_status wef_plan_autotune(wef_plan plan, const double* f_dev, double* q_dev, void* workspace, int64_t ws_bytes,
                             void* stream, int* chosen) {
  return wef::guarded("wef_plan_autotune", [&]() -> wef_status {
    if (!plan) return set_error(WEF_EINVAL, "wef_plan_autotune: plan is NULL");
    wef_status st = check_buffers(plan, f_dev, q_dev, workspace, ws_bytes);
    if (st != WEF_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
      if (e0) cudaEventDestroy(e0);
      return set_error(WEF_ECUDA, std::string("wef_plan_autotune: ") + cudaGetErrorString(ce));
    }
    const bool rf = plan->prec == WEF_RADIAL_FP32;
    int best_g = plan->granularity;
    float best = 1e30f;
    int max_tasks = 1;
    for (wef_op op : plan->ops) max_tasks = std::max(max_tasks, op->T.prog4.ntasks());
    if (rf) max_tasks = wef_plan_s::kMaxFork;  // candidates: 1, 2, 4, 8 concurrent shape streams
    // candidates: granularities 1, 2, 4, ...; radial-first: 1, 2, 4, 8 streams, each with L2
    // tile groups of 12, 24 and 48 MB (encoded as streams + 16 * MB)
    std::vector<int> cand;
    for (int g = 1; g <= 64 && g <= max_tasks; g *= 2) {
      if (rf)
        for (int mb : {12, 24, 48}) cand.push_back(g + 16 * mb);
      else
        cand.push_back(g);
    }
    for (int g : cand) {
      if (rf) {
        plan->nfork = g % 16;
        plan->group_mb = g / 16;
        plan->granularity = g;
        if (plan->gexec) {
          cudaGraphExecDestroy(plan->gexec);
          plan->gexec = nullptr;
        }
      } else {
        st = set_items(plan, g);
      }
      if (st != WEF_OK) break;
      st = plan_launch(plan, f_dev, q_dev, workspace, s);  // warm-up
      if (st == WEF_OK) cudaEventRecord(e0, s);
      for (int r = 0; r < 2 && st == WEF_OK; ++r) st = plan_launch(plan, f_dev, q_dev, workspace, s);
      if (st != WEF_OK) break;
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        st = set_error(WEF_ECUDA, "wef_plan_autotune: timing failed");
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        best_g = g;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != WEF_OK) return st;
    if (rf) {
      plan->nfork = best_g % 16;
      plan->group_mb = best_g / 16;
      plan->granularity = best_g;
      if (plan->gexec) {
        cudaGraphExecDestroy(plan->gexec);
        plan->gexec = nullptr;
      }
    } else {
      st = set_items(plan, best_g);
      if (st != WEF_OK) return st;
    }
    cache_store(plan->key, best_g);
    if (chosen) *chosen = best_g;
    return WEF_OK;
  });
}

wef_status wef_plan_status(wef_plan plan, int reset) {
  if (!plan) return set_error(WEF_EINVAL, "wef_plan_status: plan is NULL");
  int h = 0;
  cudaError_t e = cudaMemcpy(&h, plan->d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return set_error(WEF_ECUDA, std::string("wef_plan_status: ") + cudaGetErrorString(e));
  if (reset) cudaMemset(plan->d_status, 0, sizeof(int));
  if (h) return set_error(WEF_ETIMEOUT, "a bounded device-side wait gave up in an earlier plan launch");
  return WEF_OK;
}

wef_status wef_plan_destroy(wef_plan plan) {
  if (!plan) return WEF_OK;
  plan->release();
  delete plan;
  return WEF_OK;
}

}  // extern "C"
