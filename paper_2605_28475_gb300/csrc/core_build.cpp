// Host-side kinematic core R^{(c)}_{k1 k2 k3} by singular quadrature
// (paper Sec. 3.2-3.3, Sec. 4.3, Appendix A-B), parallel over all host cores.
//
// Same 5D integral as the paper, organised for speed:
//  * the scattering sphere is not sampled: for an isotropic kernel the gain
//    term needs the mean of R_{k1 l1}(|v'|) Y_{l1 m}(v'_hat) over the sphere of
//    radius u/2 centred at V = (v+w)/2, which by the Funk-Hecke theorem is
//    Y_{l1 m}(V_hat) * eps_{k1 l1}(|V|, u/2),
//      eps_{kl}(V, rho) = 1/2 int_{-1}^{1} R_kl(r(t)) P_l((V + rho t)/r(t)) dt,
//      r(t)^2 = V^2 + rho^2 + 2 V rho t,
//    a polynomial of degree k + l in t, integrated exactly by Gauss-Legendre;
//  * coordinates, Duffy patches, point counts and paddings are those of
//    Sec. 4.3 / Appendix B (z = t^2/2 reading, see the oracle's core module);
//  * patch 1 is sum-factorised (inner Duffy variable first, Appendix A), patch 2
//    is accumulated point by point.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <thread>
#include <vector>

#include "core_quad.hpp"
#include "tables.hpp"

namespace wef {

namespace {

// Symmetric eigenproblem by cyclic Jacobi rotations (small matrices only).
void jacobi_eig(int n, std::vector<double>& A, std::vector<double>& V) {
  V.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += A[(size_t)p * n + q] * A[(size_t)p * n + q];
    if (off < 1e-300) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[(size_t)p * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        const double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
        const double theta = 0.5 * (aqq - app) / apq;
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {
          const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
          A[(size_t)k * n + p] = c * akp - s * akq;
          A[(size_t)k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {
          const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
          A[(size_t)p * n + k] = c * apk - s * aqk;
          A[(size_t)q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
          V[(size_t)k * n + p] = c * vkp - s * vkq;
          V[(size_t)k * n + q] = s * vkp + c * vkq;
        }
      }
  }
}

// Gauss-Legendre on [-1, 1]: Newton on P_n from cosine initial guesses.
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.resize(n);
  w.resize(n);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) {
        p1 = z;
        p0 = 1.0;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    // recompute derivative at the final node
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) {
      const double p2 = ((2.0 * k - 1) * z * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    if (n == 1) p0 = 1.0;
    dp = n * (z * p1 - p0) / (z * z - 1.0);
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// L_n^{(a)}(x) and its derivative by the three-term recurrence.
void laguerre_val(int n, double a, double x, double& Ln, double& dLn) {
  double l0 = 1.0, l1 = 1.0 + a - x;
  if (n == 0) {
    Ln = 1.0;
    dLn = 0.0;
    return;
  }
  for (int k = 1; k < n; ++k) {
    const double l2 = ((2.0 * k + 1 + a - x) * l1 - (k + a) * l0) / (k + 1);
    l0 = l1;
    l1 = l2;
  }
  Ln = l1;
  dLn = (n * l1 - (n + a) * l0) / x;
}

// Generalised Gauss-Laguerre (weight x^a e^-x): Golub-Welsch, then Newton polish
// and the weight formula w_i = Gamma(n+a+1) / (n! x_i L_n'(x_i)^2).
void gauss_laguerre(int n, double a, std::vector<double>& x, std::vector<double>& w) {
  std::vector<double> J((size_t)n * n, 0.0), V;
  for (int i = 0; i < n; ++i) J[(size_t)i * n + i] = 2.0 * i + a + 1.0;
  for (int i = 1; i < n; ++i) J[(size_t)i * n + i - 1] = J[(size_t)(i - 1) * n + i] = std::sqrt(i * (i + a));
  jacobi_eig(n, J, V);
  x.resize(n);
  w.resize(n);
  for (int i = 0; i < n; ++i) x[i] = J[(size_t)i * n + i];
  std::sort(x.begin(), x.end());
  const double lg = std::lgamma(n + a + 1.0) - std::lgamma(n + 1.0);
  for (int i = 0; i < n; ++i) {
    double L, dL;
    for (int it = 0; it < 4; ++it) {
      laguerre_val(n, a, x[i], L, dL);
      x[i] -= L / dL;
    }
    laguerre_val(n, a, x[i], L, dL);
    w[i] = std::exp(lg) / (x[i] * dL * dL);
  }
}

double radial_norm(int k, int l) {
  return std::exp(0.5 * ((1 - l) * std::log(2.0) + 1.5 * std::log(M_PI) + std::lgamma(k + 1.0) - std::lgamma(k + l + 1.5)));
}

struct Rule {
  std::vector<double> x, w;
};

Rule gl01(int n) {
  Rule r;
  gauss_legendre(n, r.x, r.w);
  for (int i = 0; i < n; ++i) {
    r.x[i] = 0.5 * (r.x[i] + 1.0);
    r.w[i] *= 0.5;
  }
  return r;
}

using Ctx = CoreQuad;

// cos-type real harmonics at a direction with polar cosine ct and azimuth 0:
// out[l*(L+1)+m], m = 0..l.
void ylm_azimuth0(const Ctx& C, double ct, double* out) {
  const int L = C.lmax;
  const double st = std::sqrt(std::max(0.0, 1.0 - ct * ct));
  double pmm = 1.0;
  for (int m = 0; m <= L; ++m) {
    if (m > 0) pmm *= (2.0 * m - 1.0) * st;
    double pprev = 0.0, p = pmm;
    for (int l = m; l <= L; ++l) {
      if (l == m + 1) {
        pprev = p;
        p = (2.0 * m + 1.0) * ct * pmm;
      } else if (l > m + 1) {
        const double pn = ((2.0 * l - 1.0) * ct * p - (l + m - 1.0) * pprev) / (l - m);
        pprev = p;
        p = pn;
      }
      out[l * (L + 1) + m] = C.ylm_norm[l * (L + 1) + m] * p;
    }
  }
}

// R_kl(v) for all k < K, l <= L: out[k*(L+1)+l].
void radial_all(const Ctx& C, double v, double* out) {
  const double x = 0.5 * v * v;
  for (int l = 0; l < C.L1; ++l) {
    const double a = l + 0.5, vl = std::pow(v, l);
    double l0 = 1.0, l1 = 1.0 + a - x;
    for (int k = 0; k < C.K; ++k) {
      double cur;
      if (k == 0) cur = 1.0;
      else if (k == 1) cur = l1;
      else {
        cur = ((2.0 * k - 1 + a - x) * l1 - (k - 1 + a) * l0) / k;
        l0 = l1;
        l1 = cur;
      }
      out[k * C.L1 + l] = C.Nkl[k * C.L1 + l] * vl * cur;
    }
  }
}

// eps_{kl}(Vm, rho) for all (k, l): out[k*(L+1)+l].
void sphere_mean(const Ctx& C, double Vm, double rho, double* out, double* scratch) {
  const int n = (int)C.ftx.size();
  std::fill(out, out + C.K * C.L1, 0.0);
  for (int i = 0; i < n; ++i) {
    const double t = C.ftx[i];
    const double r2 = Vm * Vm + rho * rho + 2.0 * Vm * rho * t;
    const double r = std::sqrt(std::max(r2, 0.0));
    const double ca = r > 0 ? (Vm + rho * t) / r : 1.0;
    radial_all(C, r, scratch);
    double p0 = 1.0, p1 = ca;
    const double wt = 0.5 * C.ftw[i];
    for (int l = 0; l < C.L1; ++l) {
      double pl;
      if (l == 0) pl = 1.0;
      else if (l == 1) pl = ca;
      else {
        pl = ((2.0 * l - 1.0) * ca * p1 - (l - 1.0) * p0) / l;
        p0 = p1;
        p1 = pl;
      }
      for (int k = 0; k < C.K; ++k) out[k * C.L1 + l] += wt * scratch[k * C.L1 + l] * pl;
    }
  }
}

// A^c_{k1} (without u^gamma and weights) at one point for all channels: A[c*K + k1].
void channel_terms(const Ctx& C, double v, double w, double cb, double y, double* A, double* buf) {
  const int L1 = C.L1, K = C.K;
  double* Yv = buf;                 // (L+1)^2 layout [l][m]
  double* Yw = Yv + L1 * L1;
  double* eps = Yw + L1 * L1;       // K*L1
  double* Rv = eps + K * L1;        // K*L1
  double* scr = Rv + K * L1;        // K*L1
  const double sb = 2.0 * y * std::sqrt(std::max(0.0, 1.0 - y * y));
  const double Vx = 0.5 * w * sb, Vz = 0.5 * (v + w * cb);
  const double Vm = std::sqrt(Vx * Vx + Vz * Vz);
  const double u2 = v * v + w * w - 2.0 * v * w * cb;
  const double rho = 0.5 * std::sqrt(std::max(u2, 0.0));
  ylm_azimuth0(C, Vm > 0 ? Vz / Vm : 1.0, Yv);
  ylm_azimuth0(C, cb, Yw);
  sphere_mean(C, Vm, rho, eps, scr);
  radial_all(C, v, Rv);
  for (int c = 0; c < C.NT; ++c) {
    const Channel& h = C.ch[c];
    const double* G = &C.Ghat[C.Ghat_off[c]];
    const int mm = std::min(h.l1, h.l3);
    double a = 0.0;
    for (int m = 0; m <= mm; ++m) a += G[m] * Yw[h.l3 * L1 + m] * Yv[h.l1 * L1 + m];
    const double b = G[0] * Yw[h.l3 * L1] * C.ylm_norm[h.l1 * L1];  // Y_{l1 0}(z_hat) = norm
    for (int k = 0; k < K; ++k) A[c * K + k] = C.s2[c] * (a * eps[k * L1 + h.l1] - b * Rv[k * L1 + h.l1]);
  }
}

}  // namespace

std::string core_quadrature(const Tables& T, double gamma, int pad_rad, int pad_ang, CoreQuad& C) {
  C = CoreQuad();
  C.kmax = T.kmax;
  C.lmax = T.lmax;
  C.K = T.K;
  C.L1 = T.lmax + 1;
  C.NT = (int)T.chans.size();
  C.gamma = gamma;
  C.ch = T.chans;
  C.Nkl.resize(C.K * C.L1);
  for (int k = 0; k < C.K; ++k)
    for (int l = 0; l < C.L1; ++l) C.Nkl[k * C.L1 + l] = radial_norm(k, l);
  C.ylm_norm.assign(C.L1 * C.L1, 0.0);
  for (int l = 0; l < C.L1; ++l)
    for (int m = 0; m <= l; ++m)
      C.ylm_norm[l * C.L1 + m] = std::sqrt((2.0 * l + 1) / (4.0 * M_PI) * std::exp(std::lgamma(l - m + 1.0) - std::lgamma(l + m + 1.0))) *
                                 (m > 0 ? std::sqrt(2.0) : 1.0);
  C.s2.resize(C.NT);
  C.Ghat_off.resize(C.NT);
  for (int c = 0; c < C.NT; ++c) {
    const Channel& h = C.ch[c];
    C.s2[c] = std::sqrt((2.0 * h.l2 + 1) / (4.0 * M_PI));
    C.Ghat_off[c] = (int)C.Ghat.size();
    for (int m = 0; m <= std::min(h.l1, h.l3); ++m) C.Ghat.push_back(real_gaunt(h.l1, m, h.l2, 0, h.l3, m));
  }
  // channel norms S_c = sum_m g^2 over all m-triples
  C.S.assign(C.NT, 0.0);
  for (size_t z = 0; z < T.g.size(); ++z) C.S[T.c[z]] += T.g[z] * T.g[z];
  gauss_legendre((C.kmax + C.lmax) / 2 + 2, C.ftx, C.ftw);
  // Table 2 / Appendix B point counts plus padding.
  const int kmax = C.kmax, lmax = C.lmax;
  const int Nz = (int)std::ceil((3.0 * kmax + 1.5 * lmax + 3.0) / 2.0) + pad_rad;
  const int Nx1 = 4 * kmax + 3 * lmax + 4 + pad_rad;
  const int Nh1 = kmax + (int)std::ceil(1.5 * lmax) + 1 + pad_ang;
  const int Ny2 = 4 * kmax + 3 * lmax + 4 + pad_ang;
  const int Nh2 = 3 * kmax + (int)std::floor(1.5 * lmax) + 3 + pad_rad;
  gauss_laguerre(Nz, 0.5 * gamma, C.zz, C.wz);
  Rule r;
  r = gl01(Nx1); C.x1 = r.x; C.wx1 = r.w;
  r = gl01(Nh1); C.h1 = r.x; C.wh1 = r.w;
  r = gl01(Ny2); C.y2 = r.x; C.wy2 = r.w;
  r = gl01(Nh2); C.h2 = r.x; C.wh2 = r.w;
  C.pref = std::pow(2.0, gamma) * 4.0 / std::pow(2.0 * M_PI, 3.0);
  return "";
}

// Returns "" on success.
std::string core_build(const Tables& T, double gamma, int pad_rad, int pad_ang, double* R) {
  CoreQuad C;
  std::string err = core_quadrature(T, gamma, pad_rad, pad_ang, C);
  if (!err.empty()) return err;
  const std::vector<double>& S = C.S;
  const std::vector<double>&zz = C.zz, &wz = C.wz;
  const int Nz = (int)zz.size(), Nx1 = (int)C.x1.size(), Nh1 = (int)C.h1.size(), Ny2 = (int)C.y2.size(),
            Nh2 = (int)C.h2.size();
  struct R01 {
    const std::vector<double>&x, &w;
  };
  const R01 rx1{C.x1, C.wx1}, rh1{C.h1, C.wh1}, ry2{C.y2, C.wy2}, rh2{C.h2, C.wh2};
  const int K = C.K, L1 = C.L1, NT = C.NT;
  const size_t RL = (size_t)NT * K * K * K;
  // work items: (z, outer node, patch, half)
  struct Item {
    int iz, io, patch, half;
  };
  std::vector<Item> items;
  for (int iz = 0; iz < Nz; ++iz)
    for (int half = 0; half < 2; ++half) {
      for (int i = 0; i < Nx1; ++i) items.push_back({iz, i, 1, half});
      for (int i = 0; i < Ny2; ++i) items.push_back({iz, i, 2, half});
    }
  // Deterministic reduction: item i is added, in item order, into partial sum i % kParts,
  // and the partial sums are added in a fixed order, so the core is bitwise the same for any
  // thread count and schedule (replicas built by ranks on the same kind of host agree exactly).
  constexpr unsigned kParts = 16;
  const unsigned nth = std::min(kParts, std::max(1u, std::thread::hardware_concurrency()));
  std::vector<std::vector<double>> acc(kParts);
  const double pref = C.pref;
  auto worker = [&](unsigned tid) {
    const int nbuf = 2 * L1 * L1 + 3 * K * L1;
    std::vector<double> buf(nbuf), A((size_t)NT * K), Abar((size_t)NT * K), Rv(K * L1), Rw(K * L1);
    const int maxh = std::max(Nh1, Nh2);
    std::vector<double> Ap((size_t)maxh * NT * K), Rvp((size_t)maxh * K * L1), Rwp((size_t)maxh * K * L1);
    for (unsigned part = tid; part < kParts; part += nth) {
      std::vector<double>& Racc = acc[part];
      Racc.assign(RL, 0.0);
      for (size_t it = part; it < items.size(); it += kParts) {
        const Item& I = items[it];
        const double z = zz[I.iz], sz = std::sqrt(z);
        const double sgn = I.half == 0 ? 1.0 : -1.0;
        if (I.patch == 1) {
          // outer x, inner h: y = x h; v, w fixed over the inner loop
          const double xa = rx1.x[I.io], x = sgn * xa;
          const double v = sz * (1.0 + x), w = sz * (1.0 - x);
          std::fill(Abar.begin(), Abar.end(), 0.0);
          for (int ih = 0; ih < Nh1; ++ih) {
            const double h = rh1.x[ih], y = xa * h;
            const double sing = std::pow(xa, gamma) * std::pow(1.0 + (1.0 - xa * xa) * h * h, 0.5 * gamma);
            const double W = wz[I.iz] * rx1.w[I.io] * rh1.w[ih] * xa * sing * std::exp(-z * xa * xa) * z * z *
                             (1.0 - xa * xa) * (1.0 - xa * xa) * y * pref;
            channel_terms(C, v, w, 1.0 - 2.0 * y * y, y, A.data(), buf.data());
            for (size_t j = 0; j < A.size(); ++j) Abar[j] += W * A[j];
          }
          radial_all(C, v, Rv.data());
          radial_all(C, w, Rw.data());
          for (int c = 0; c < NT; ++c) {
            const Channel& h = C.ch[c];
            double* Rc = &Racc[(size_t)c * K * K * K];
            for (int k1 = 0; k1 < K; ++k1) {
              const double a = Abar[c * K + k1];
              for (int k2 = 0; k2 < K; ++k2) {
                const double ab = a * Rv[k2 * L1 + h.l2];
                double* row = Rc + ((size_t)k1 * K + k2) * K;
                for (int k3 = 0; k3 < K; ++k3) row[k3] += ab * Rw[k3 * L1 + h.l3];
              }
            }
          }
        } else {
          // outer y, inner h: x = y h; v, w change with h
          const double y = ry2.x[I.io];
          for (int ih = 0; ih < Nh2; ++ih) {
            const double h = rh2.x[ih], xa = y * h, x = sgn * xa;
            const double v = sz * (1.0 + x), w = sz * (1.0 - x);
            const double sing = std::pow(y, gamma) * std::pow(1.0 + (1.0 - y * y) * h * h, 0.5 * gamma);
            const double W = wz[I.iz] * ry2.w[I.io] * rh2.w[ih] * y * sing * std::exp(-z * xa * xa) * z * z *
                             (1.0 - xa * xa) * (1.0 - xa * xa) * y * pref;
            channel_terms(C, v, w, 1.0 - 2.0 * y * y, y, &Ap[(size_t)ih * NT * K], buf.data());
            for (size_t j = 0; j < (size_t)NT * K; ++j) Ap[(size_t)ih * NT * K + j] *= W;
            radial_all(C, v, &Rvp[(size_t)ih * K * L1]);
            radial_all(C, w, &Rwp[(size_t)ih * K * L1]);
          }
          for (int c = 0; c < NT; ++c) {
            const Channel& hc = C.ch[c];
            double* Rc = &Racc[(size_t)c * K * K * K];
            for (int ih = 0; ih < Nh2; ++ih) {
              const double* a = &Ap[(size_t)ih * NT * K + (size_t)c * K];
              const double* rv = &Rvp[(size_t)ih * K * L1];
              const double* rw = &Rwp[(size_t)ih * K * L1];
              double wl3[32];
              for (int k3 = 0; k3 < K; ++k3) wl3[k3] = rw[k3 * L1 + hc.l3];
              for (int k1 = 0; k1 < K; ++k1) {
                const double a1 = a[k1];
                for (int k2 = 0; k2 < K; ++k2) {
                  const double ab = a1 * rv[k2 * L1 + hc.l2];
                  double* row = Rc + ((size_t)k1 * K + k2) * K;
                  for (int k3 = 0; k3 < K; ++k3) row[k3] += ab * wl3[k3];
                }
              }
            }
          }
        }
      }
    }
  };
  std::vector<std::thread> th;
  for (unsigned t = 0; t < nth; ++t) th.emplace_back(worker, t);
  for (auto& t : th) t.join();
  for (size_t j = 0; j < RL; ++j) {
    double s = 0.0;
    for (unsigned t = 0; t < kParts; ++t) s += acc[t][j];
    R[j] = s;
  }
  for (int c = 0; c < NT; ++c) {
    const double f = 8.0 * M_PI * M_PI / S[c];
    for (size_t j = 0; j < (size_t)K * K * K; ++j) R[(size_t)c * K * K * K + j] *= f;
  }
  return "";
}

}  // namespace wef
