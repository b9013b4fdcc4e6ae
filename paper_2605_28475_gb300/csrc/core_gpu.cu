// Device assembly of the kinematic core R^{(c)}_{k1 k2 k3} (paper Sec. 4.3, Appendix
// A-B): the same singular quadrature as the host builder (same rules, point counts,
// paddings and Funk-Hecke reduction of the scattering sphere), in FP64 on the GPU.
//
//   R_c[k1,k2,k3] = (8 pi^2 / S_c) sum_r alpha_c[k1](r) R_{k2 l2}(v_r) R_{k3 l3}(w_r)
//
// over "radial points" r = (z, v, w).  For patch 1 a radial point collects the inner
// Duffy variable (v and w do not depend on it), alpha_c summing the angular points; for
// patch 2 every point is its own radial point.  Per angular point
//   alpha_c[k1] += W s2_c (a_c eps_{k1 l1}(V, u/2) - b_c R_{k1 l1}(v)),
//   a_c = sum_m G_c[m] Y_{l3 m}(w_hat) Y_{l1 m}(V_hat),  b_c = G_c[0] Y_{l3 0}(w_hat) Y_{l1 0}(z_hat)
// (gain through the sphere mean eps of Sec. 4.3, loss subtracted inside the integral).
// Kernel 1 tabulates eps, Y and R at the points of a chunk of z nodes (one warp per point,
// lane = l); kernel 2 runs one CTA per channel, thread = (k1, k2) holding the K values of
// k3 in registers, and accumulates the rank-1 terms in FP64.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/wef.h"
#include "core_quad.hpp"
#include "operator.hpp"
#include "wef_internal.hpp"

namespace {

constexpr int kMaxL1 = 21;  // Lmax <= 20
constexpr int kMaxK = 17;   // Kmax <= 16
constexpr int kNP = 64;     // patch-2 radial points per contraction step
constexpr int kNA = 128;    // patch-1 angular points per piece

// Point tables are component-major (component c of point p at [c * npoints + p]) so that
// the contraction's reads of one component over consecutive points are coalesced.
struct Geo {
  int K, L1, nz_chunk, Nx1, Nh1, Ny2, Nh2, nft;
  int DA, DR;        // components per angular / radial point
  int64_t na, nr;    // angular / radial points in the chunk (the component strides)
  int64_t na_zh;     // angular points per (z, half)
  int64_t nr_zh;     // radial points per (z, half)
  double gamma, pref;
};

// Device copies of the rules and constants.
struct Dev {
  const double *zz, *wz, *x1, *wx1, *h1, *wh1, *y2, *wy2, *h2, *wh2, *ftx, *ftw, *Nkl, *ylm_norm;
};

__device__ __forceinline__ double ipow(double x, int n) {
  double r = 1.0;
  for (int i = 0; i < n; ++i) r *= x;
  return r;
}

// Point geometry of angular point (patch, io, ih) at z, half.
struct Pt {
  double v, w, cb, y, W;
};

__device__ Pt point_geo(const Geo& g, const Dev& d, int iz, int half, int patch, int io, int ih) {
  const double z = d.zz[iz], sz = sqrt(z), sgn = half == 0 ? 1.0 : -1.0;
  Pt p;
  if (patch == 1) {
    const double xa = d.x1[io], x = sgn * xa, h = d.h1[ih], y = xa * h;
    const double sing = pow(xa, g.gamma) * pow(1.0 + (1.0 - xa * xa) * h * h, 0.5 * g.gamma);
    p.v = sz * (1.0 + x);
    p.w = sz * (1.0 - x);
    p.y = y;
    p.cb = 1.0 - 2.0 * y * y;
    p.W = d.wz[iz] * d.wx1[io] * d.wh1[ih] * xa * sing * exp(-z * xa * xa) * z * z * (1.0 - xa * xa) * (1.0 - xa * xa) * y *
          g.pref;
  } else {
    const double y = d.y2[io], h = d.h2[ih], xa = y * h, x = sgn * xa;
    const double sing = pow(y, g.gamma) * pow(1.0 + (1.0 - y * y) * h * h, 0.5 * g.gamma);
    p.v = sz * (1.0 + x);
    p.w = sz * (1.0 - x);
    p.y = y;
    p.cb = 1.0 - 2.0 * y * y;
    p.W = d.wz[iz] * d.wy2[io] * d.wh2[ih] * y * sing * exp(-z * xa * xa) * z * z * (1.0 - xa * xa) * (1.0 - xa * xa) * y *
          g.pref;
  }
  return p;
}

// Lane l: R_{k l}(r) for k < K into out[k] (normalised v^l L_k^{(l+1/2)}(v^2/2)).
__device__ __forceinline__ void radial_lane(const Geo& g, const Dev& d, int l, double r, double* out) {
  const double x = 0.5 * r * r, a = l + 0.5, rl = ipow(r, l);
  double l0 = 1.0, l1 = 1.0 + a - x;
  for (int k = 0; k < g.K; ++k) {
    double cur;
    if (k == 0) cur = 1.0;
    else if (k == 1) cur = l1;
    else {
      cur = ((2.0 * k - 1 + a - x) * l1 - (k - 1 + a) * l0) / k;
      l0 = l1;
      l1 = cur;
    }
    out[k] = d.Nkl[k * g.L1 + l] * rl * cur;
  }
}

// Lane l: cos-type real harmonics Y_{l m}(ct, azimuth 0), m = 0..l, into out[(l*L1 + m) * stride].
__device__ __forceinline__ void ylm_lane(const Geo& g, const Dev& d, int l, double ct, double* out, int64_t stride) {
  const double st = sqrt(fmax(0.0, 1.0 - ct * ct));
  double pmm = 1.0;
  for (int m = 0; m <= l; ++m) {
    if (m > 0) pmm *= (2.0 * m - 1.0) * st;
    double pprev = 0.0, p = pmm;
    for (int j = m + 1; j <= l; ++j) {
      double pn;
      if (j == m + 1) pn = (2.0 * m + 1.0) * ct * pmm;
      else pn = ((2.0 * j - 1.0) * ct * p - (j + m - 1.0) * pprev) / (j - m);
      pprev = p;
      p = pn;
    }
    out[(l * g.L1 + m) * stride] = d.ylm_norm[l * g.L1 + m] * p;
  }
}

// Kernel 1a: one warp per angular point of the chunk; components {W, eps[K][L1], Yv[L1][L1], Yw[L1][L1]}.
__global__ void angular_points_kernel(Geo g, Dev d, int iz0, double* __restrict__ A) {
  const int64_t gp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int l = threadIdx.x & 31;
  const int64_t total = (int64_t)g.nz_chunk * 2 * g.na_zh;
  if (gp >= total) return;
  const int64_t zh = gp / g.na_zh, loc = gp % g.na_zh;
  const int iz = iz0 + (int)(zh / 2), half = (int)(zh % 2);
  int patch, io, ih;
  if (loc < (int64_t)g.Nx1 * g.Nh1) {
    patch = 1;
    io = (int)(loc / g.Nh1);
    ih = (int)(loc % g.Nh1);
  } else {
    const int64_t r = loc - (int64_t)g.Nx1 * g.Nh1;
    patch = 2;
    io = (int)(r / g.Nh2);
    ih = (int)(r % g.Nh2);
  }
  const Pt p = point_geo(g, d, iz, half, patch, io, ih);
  double* rec = A + gp;  // component c at rec[c * na]
  const int64_t sa = g.na;
  const double sb = 2.0 * p.y * sqrt(fmax(0.0, 1.0 - p.y * p.y));
  const double Vx = 0.5 * p.w * sb, Vz = 0.5 * (p.v + p.w * p.cb);
  const double Vm = sqrt(Vx * Vx + Vz * Vz);
  const double u2 = p.v * p.v + p.w * p.w - 2.0 * p.v * p.w * p.cb;
  const double rho = 0.5 * sqrt(fmax(u2, 0.0));
  if (l == 0) rec[0] = p.W;
  if (l < g.L1) {
    // eps_{k l}(Vm, rho) = 1/2 int R_{kl}(r(t)) P_l((Vm + rho t) / r(t)) dt, Gauss-Legendre in t
    double eps[kMaxK], Rr[kMaxK];
    for (int k = 0; k < g.K; ++k) eps[k] = 0.0;
    for (int i = 0; i < g.nft; ++i) {
      const double t = d.ftx[i];
      const double r2 = Vm * Vm + rho * rho + 2.0 * Vm * rho * t;
      const double r = sqrt(fmax(r2, 0.0));
      const double ca = r > 0 ? (Vm + rho * t) / r : 1.0;
      double p0 = 1.0, p1 = ca, pl = 1.0;
      if (l == 1) pl = ca;
      for (int j = 2; j <= l; ++j) {
        pl = ((2.0 * j - 1.0) * ca * p1 - (j - 1.0) * p0) / j;
        p0 = p1;
        p1 = pl;
      }
      radial_lane(g, d, l, r, Rr);
      const double wt = 0.5 * d.ftw[i] * pl;
      for (int k = 0; k < g.K; ++k) eps[k] += wt * Rr[k];
    }
    for (int k = 0; k < g.K; ++k) rec[(1 + k * g.L1 + l) * sa] = eps[k];
    ylm_lane(g, d, l, Vm > 0 ? Vz / Vm : 1.0, rec + (1 + g.K * g.L1) * sa, sa);
    ylm_lane(g, d, l, p.cb, rec + (1 + g.K * g.L1 + g.L1 * g.L1) * sa, sa);
  }
}

// Kernel 1b: one warp per radial point; components {Rv[K][L1], Rw[K][L1]}.
__global__ void radial_points_kernel(Geo g, Dev d, int iz0, double* __restrict__ Rr) {
  const int64_t rp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int l = threadIdx.x & 31;
  const int64_t total = (int64_t)g.nz_chunk * 2 * g.nr_zh;
  if (rp >= total || l >= g.L1) return;
  const int64_t zh = rp / g.nr_zh, loc = rp % g.nr_zh;
  const int iz = iz0 + (int)(zh / 2), half = (int)(zh % 2);
  Pt p;
  if (loc < g.Nx1) {
    p = point_geo(g, d, iz, half, 1, (int)loc, 0);  // v, w do not depend on the inner variable
  } else {
    const int64_t r = loc - g.Nx1;
    p = point_geo(g, d, iz, half, 2, (int)(r / g.Nh2), (int)(r % g.Nh2));
  }
  double out[kMaxK];
  double* rec = Rr + rp;
  const int64_t sr = g.nr;
  radial_lane(g, d, l, p.v, out);
  for (int k = 0; k < g.K; ++k) rec[(k * g.L1 + l) * sr] = out[k];
  radial_lane(g, d, l, p.w, out);
  for (int k = 0; k < g.K; ++k) rec[(g.K * g.L1 + k * g.L1 + l) * sr] = out[k];
}

struct ChanDev {
  const int4* ch;        // {l1, l2, l3, Ghat_off}
  const double* Ghat;
  const double* s2;
  const double* fscale;  // 8 pi^2 / S_c
};

// a_c W and b_c W of angular point rec (component c at rec[c * na]).
__device__ __forceinline__ void ab_of(const Geo& g, const Dev& d, const double* rec, int l1, int l3, const double* G,
                                      double& aW, double& bW) {
  const int64_t sa = g.na;
  const double W = rec[0];
  const double* Yv = rec + (1 + g.K * g.L1) * sa;
  const double* Yw = Yv + g.L1 * g.L1 * sa;
  const int mm = l1 < l3 ? l1 : l3;
  double a = 0.0;
  for (int m = 0; m <= mm; ++m) a += G[m] * Yw[(l3 * g.L1 + m) * sa] * Yv[(l1 * g.L1 + m) * sa];
  aW = W * a;
  bW = W * G[0] * Yw[l3 * g.L1 * sa] * d.ylm_norm[l1 * g.L1];
}

// Kernel 2: S CTAs per channel, each over every S-th radial point of the chunk; thread
// (k1, k2) accumulates R_c[k1][k2][0..K) in registers (K is a template parameter) and adds
// its share to R atomically at the end (S is chosen so that the grid fills several waves).
template <int K>
__global__ void contract_kernel(Geo g, Dev d, ChanDev cd, const double* __restrict__ A, const double* __restrict__ Rr,
                                double* __restrict__ R, int nsplit) {
  __shared__ double aW[kNA], bW[kNA];
  __shared__ double alpha[kMaxK][kNP], rv2[kMaxK][kNP], rw3[kMaxK][kNP];
  const int c = blockIdx.x / nsplit, part = blockIdx.x % nsplit;
  const int4 ch = cd.ch[c];
  const int l1 = ch.x, l2 = ch.y, l3 = ch.z;
  const double* G = cd.Ghat + ch.w;
  const double s2 = cd.s2[c];
  const int L1 = g.L1, t = threadIdx.x;
  const bool own = t < K * K;
  const int k1 = t / K, k2 = t % K;
  double acc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) acc[k] = 0.0;
  const int64_t nzh = (int64_t)g.nz_chunk * 2, sa = g.na, sr = g.nr;
  for (int64_t zh = 0; zh < nzh; ++zh) {
    const double* Az = A + zh * g.na_zh;  // point p of this (z, half): Az + p, component c at + c * sa
    const double* Rz = Rr + zh * g.nr_zh;
    // patch 1: one radial point per outer node, alpha summed over the inner node
    for (int io = part; io < g.Nx1; io += nsplit) {
      const double* rrec = Rz + io;
      double al = 0.0;  // thread k < K: alpha[k]
      for (int h0 = 0; h0 < g.Nh1; h0 += kNA) {
        const int nh = min(kNA, g.Nh1 - h0);
        __syncthreads();
        for (int i = t; i < nh; i += blockDim.x)
          ab_of(g, d, Az + (int64_t)io * g.Nh1 + h0 + i, l1, l3, G, aW[i], bW[i]);
        __syncthreads();
        if (t < K) {
          const double rv = rrec[(t * L1 + l1) * sr];
          const double* eps = Az + (int64_t)io * g.Nh1 + h0 + (1 + t * L1 + l1) * sa;
          for (int i = 0; i < nh; ++i) al += aW[i] * eps[i] - bW[i] * rv;
        }
      }
      __syncthreads();
      if (t < K) {
        alpha[t][0] = s2 * al;
        rv2[t][0] = rrec[(t * L1 + l2) * sr];
        rw3[t][0] = rrec[(K * L1 + t * L1 + l3) * sr];
      }
      __syncthreads();
      if (own) {
        const double ab = alpha[k1][0] * rv2[k2][0];
#pragma unroll
        for (int k3 = 0; k3 < K; ++k3) acc[k3] = fma(ab, rw3[k3][0], acc[k3]);
      }
    }
    // patch 2: every point is a radial point
    const int64_t n2 = (int64_t)g.Ny2 * g.Nh2;
    for (int64_t p0 = (int64_t)part * kNP; p0 < n2; p0 += (int64_t)nsplit * kNP) {
      const int np = (int)min((int64_t)kNP, n2 - p0);
      __syncthreads();
      for (int i = t; i < np; i += blockDim.x)
        ab_of(g, d, Az + (int64_t)g.Nx1 * g.Nh1 + p0 + i, l1, l3, G, aW[i], bW[i]);
      __syncthreads();
      for (int i = t; i < K * np; i += blockDim.x) {
        const int k = i / np, j = i % np;  // consecutive threads: consecutive points (coalesced)
        const double* rec = Az + (int64_t)g.Nx1 * g.Nh1 + p0 + j;
        const double* rrec = Rz + (int64_t)g.Nx1 + p0 + j;
        alpha[k][j] = s2 * (aW[j] * rec[(1 + k * L1 + l1) * sa] - bW[j] * rrec[(k * L1 + l1) * sr]);
        rv2[k][j] = rrec[(k * L1 + l2) * sr];
        rw3[k][j] = rrec[(K * L1 + k * L1 + l3) * sr];
      }
      __syncthreads();
      if (own) {
        for (int j = 0; j < np; ++j) {
          const double ab = alpha[k1][j] * rv2[k2][j];
#pragma unroll
          for (int k3 = 0; k3 < K; ++k3) acc[k3] = fma(ab, rw3[k3][j], acc[k3]);
        }
      }
    }
  }
  if (own) {
    const double f = cd.fscale[c];
    double* out = R + (((int64_t)c * K + k1) * K + k2) * K;
#pragma unroll
    for (int k3 = 0; k3 < K; ++k3) atomicAdd(out + k3, f * acc[k3]);
  }
}

template <int K>
cudaError_t launch_contract_k(int NT, int threads, const Geo& g, const Dev& d, const ChanDev& cd, const double* A,
                              const double* Rr, double* R) {
  int dev = 0, sms = 1, per_sm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, contract_kernel<K>, threads, 0);
  const int slots = sms * (per_sm > 0 ? per_sm : 1);
  const int nsplit = std::max(1, (4 * slots + NT - 1) / NT);  // at least ~4 waves of CTAs
  contract_kernel<K><<<NT * nsplit, threads>>>(g, d, cd, A, Rr, R, nsplit);
  return cudaGetLastError();
}

cudaError_t launch_contract(int K, int NT, int threads, const Geo& g, const Dev& d, const ChanDev& cd, const double* A,
                            const double* Rr, double* R) {
  switch (K) {
#define WEF_CK(k) \
  case k:         \
    return launch_contract_k<k>(NT, threads, g, d, cd, A, Rr, R);
    WEF_CK(1) WEF_CK(2) WEF_CK(3) WEF_CK(4) WEF_CK(5) WEF_CK(6) WEF_CK(7) WEF_CK(8) WEF_CK(9) WEF_CK(10) WEF_CK(11)
    WEF_CK(12) WEF_CK(13) WEF_CK(14) WEF_CK(15) WEF_CK(16) WEF_CK(17)
#undef WEF_CK
    default:
      return cudaErrorInvalidValue;
  }
}

template <class T>
cudaError_t to_dev(T** dst, const std::vector<T>& v) {
  cudaError_t e = cudaMalloc((void**)dst, std::max<size_t>(v.size(), 1) * sizeof(T));
  if (e == cudaSuccess && !v.empty()) e = cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
  return e;
}

}  // namespace

extern "C" wef_status wef_core_build_device(wef_op op, int pad_rad, int pad_ang, double* R_out, int64_t len) {
  return wef::guarded("wef_core_build_device", [&]() -> wef_status {
    if (!op || !R_out) return wef::set_error(WEF_EINVAL, "wef_core_build_device: NULL argument");
    const int K = op->T.K, L1 = op->T.lmax + 1;
    if (len != (int64_t)op->T.chans.size() * K * K * K)
      return wef::set_error(WEF_ESHAPE, "wef_core_build_device: len must be N_T*K^3");
    if (pad_rad < 0 || pad_ang < 0 || pad_rad > 200 || pad_ang > 200)
      return wef::set_error(WEF_EINVAL, "wef_core_build_device: bad padding");
    if (K > kMaxK || L1 > kMaxL1) return wef::set_error(WEF_ESHAPE, "wef_core_build_device: Kmax <= 16, Lmax <= 20");
    wef::CoreQuad Q;
    std::string err = wef::core_quadrature(op->T, op->gamma, pad_rad, pad_ang, Q);
    if (!err.empty()) return wef::set_error(WEF_EINVAL, "wef_core_build_device: " + err);
    Geo g;
    g.K = K;
    g.L1 = L1;
    g.Nx1 = (int)Q.x1.size();
    g.Nh1 = (int)Q.h1.size();
    g.Ny2 = (int)Q.y2.size();
    g.Nh2 = (int)Q.h2.size();
    g.nft = (int)Q.ftx.size();
    g.DA = 1 + K * L1 + 2 * L1 * L1;
    g.DR = 2 * K * L1;
    g.na_zh = (int64_t)g.Nx1 * g.Nh1 + (int64_t)g.Ny2 * g.Nh2;
    g.nr_zh = (int64_t)g.Nx1 + (int64_t)g.Ny2 * g.Nh2;
    g.gamma = Q.gamma;
    g.pref = Q.pref;
    const int Nz = (int)Q.zz.size(), NT = Q.NT;
    // z nodes per chunk: point tables of about 1 GB at most
    const int64_t bytes_z = 2 * (g.na_zh * g.DA + g.nr_zh * g.DR) * (int64_t)sizeof(double);
    const int zc = (int)std::max<int64_t>(1, std::min<int64_t>(Nz, (int64_t)(1LL << 30) / bytes_z));
    std::vector<int32_t> chv;
    for (int c = 0; c < NT; ++c) {
      const wef::Channel& h = Q.ch[c];
      chv.insert(chv.end(), {h.l1, h.l2, h.l3, Q.Ghat_off[c]});
    }
    std::vector<double> fscale(NT);
    for (int c = 0; c < NT; ++c) fscale[c] = 8.0 * M_PI * M_PI / Q.S[c];
    std::vector<double*> bufs;
    auto dv = [&](const std::vector<double>& v, const double** p) {
      double* q = nullptr;
      cudaError_t e = to_dev(&q, v);
      bufs.push_back(q);
      *p = q;
      return e;
    };
    Dev d{};
    cudaError_t e = cudaSuccess;
    const std::vector<const std::vector<double>*> src = {&Q.zz, &Q.wz, &Q.x1, &Q.wx1, &Q.h1, &Q.wh1, &Q.y2,
                                                          &Q.wy2, &Q.h2, &Q.wh2, &Q.ftx, &Q.ftw, &Q.Nkl, &Q.ylm_norm};
    const double** dst[] = {&d.zz, &d.wz, &d.x1, &d.wx1, &d.h1, &d.wh1, &d.y2,
                            &d.wy2, &d.h2, &d.wh2, &d.ftx, &d.ftw, &d.Nkl, &d.ylm_norm};
    for (size_t i = 0; i < src.size() && e == cudaSuccess; ++i) e = dv(*src[i], dst[i]);
    ChanDev cd{};
    int32_t* dch = nullptr;
    double *A = nullptr, *Rr = nullptr, *Rd = nullptr;
    if (e == cudaSuccess) e = to_dev(&dch, chv);
    cd.ch = (const int4*)dch;
    if (e == cudaSuccess) e = dv(Q.Ghat, &cd.Ghat);
    if (e == cudaSuccess) e = dv(Q.s2, &cd.s2);
    if (e == cudaSuccess) e = dv(fscale, &cd.fscale);
    if (e == cudaSuccess) e = cudaMalloc((void**)&A, (size_t)zc * 2 * g.na_zh * g.DA * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void**)&Rr, (size_t)zc * 2 * g.nr_zh * g.DR * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void**)&Rd, (size_t)len * sizeof(double));
    if (e == cudaSuccess) e = cudaMemset(Rd, 0, (size_t)len * sizeof(double));
    const int threads2 = (K * K + 31) / 32 * 32;
    for (int iz0 = 0; iz0 < Nz && e == cudaSuccess; iz0 += zc) {
      g.nz_chunk = std::min(zc, Nz - iz0);
      const int64_t na = (int64_t)g.nz_chunk * 2 * g.na_zh, nr = (int64_t)g.nz_chunk * 2 * g.nr_zh;
      g.na = na;
      g.nr = nr;
      angular_points_kernel<<<(unsigned)((na * 32 + 255) / 256), 256>>>(g, d, iz0, A);
      radial_points_kernel<<<(unsigned)((nr * 32 + 255) / 256), 256>>>(g, d, iz0, Rr);
      e = cudaGetLastError();
      if (e == cudaSuccess) e = launch_contract(K, NT, threads2, g, d, cd, A, Rr, Rd);
    }
    if (e == cudaSuccess) e = cudaMemcpy(R_out, Rd, (size_t)len * sizeof(double), cudaMemcpyDeviceToHost);
    for (double* p : bufs) cudaFree(p);
    cudaFree(dch);
    cudaFree(A);
    cudaFree(Rr);
    cudaFree(Rd);
    if (e != cudaSuccess) return wef::set_error(WEF_ECUDA, std::string("wef_core_build_device: ") + cudaGetErrorString(e));
    return WEF_OK;
  });
}
