// Host-side angular geometry: exact Wigner 3-j values, real Gaunt table in the
// COO order of Table 1, the symmetrised slices and the kernel programs.
#include "tables.hpp"

#include <algorithm>
#include <cmath>
#include <complex>
#include <limits>
#include <map>
#include <set>

namespace wef {

namespace {

// Pascal triangle up to n = 64 (C(64,32) < 2^63).
struct Binom {
  int64_t c[65][65];
  Binom() {
    for (int n = 0; n <= 64; ++n) {
      c[n][0] = c[n][n] = 1;
      for (int k = 1; k < n; ++k) c[n][k] = c[n - 1][k - 1] + c[n - 1][k];
    }
  }
  int64_t operator()(int n, int k) const { return (k < 0 || k > n || n < 0) ? 0 : c[n][k]; }
};
const Binom& binom() {
  static Binom b;
  return b;
}

const int kPrimes[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37, 41, 43, 47, 53, 59, 61, 67, 71, 73, 79, 83, 89, 97};

// exponent of p in n!
int fact_exp(int n, int p) {
  int e = 0;
  for (int64_t q = p; q <= n; q *= p) e += (int)(n / q);
  return e;
}

}  // namespace

// 3-j symbol from the Racah sum rewritten with binomials:
//   (j1 j2 j3; m1 m2 m3) = (-1)^{j1-j2-m3} P * S,
//   S = sum_k (-1)^k C(a,k) C(j3+m3, j1-m1-k) C(j3-m3, j2+m2-k),  a = j1+j2-j3  (exact, 128-bit)
//   P^2 = (j1-j2+j3)! (-j1+j2+j3)! (j1+m1)! (j1-m1)! (j2+m2)! (j2-m2)! / ((J+1)! a! (j3+m3)! (j3-m3)!)
// P is evaluated from the prime factorisation of P^2.
double wigner3j(int j1, int j2, int j3, int m1, int m2, int m3) {
  if (m1 + m2 + m3 != 0) return 0.0;
  if (j1 < 0 || j2 < 0 || j3 < 0) return 0.0;
  if (std::abs(m1) > j1 || std::abs(m2) > j2 || std::abs(m3) > j3) return 0.0;
  if (j3 > j1 + j2 || j3 < std::abs(j1 - j2)) return 0.0;
  const int J = j1 + j2 + j3;
  const int a = j1 + j2 - j3;
  const Binom& B = binom();
  __int128 S = 0;
  for (int k = 0; k <= a; ++k) {
    __int128 t = (__int128)B(a, k) * B(j3 + m3, j1 - m1 - k);
    t *= B(j3 - m3, j2 + m2 - k);
    S += (k & 1) ? -t : t;
  }
  if (S == 0) return 0.0;
  const int num[6] = {j1 - j2 + j3, -j1 + j2 + j3, j1 + m1, j1 - m1, j2 + m2, j2 - m2};
  const int den[4] = {J + 1, a, j3 + m3, j3 - m3};
  double P = 1.0;
  for (int p : kPrimes) {
    if (p > J + 1) break;
    int e = 0;
    for (int n : num) e += fact_exp(n, p);
    for (int n : den) e -= fact_exp(n, p);
    if (e != 0) P *= std::pow((double)p, 0.5 * e);
  }
  const double sgn = ((j1 - j2 - m3) & 1) ? -1.0 : 1.0;
  return sgn * P * (double)S;
}

namespace {

// 3j(l1 l2 l3; 0 0 0) for l <= 20, computed once per thread and triple.
double wigner3j_000(int l1, int l2, int l3) {
  constexpr int kL = 21;
  if (l1 >= kL || l2 >= kL || l3 >= kL) return wigner3j(l1, l2, l3, 0, 0, 0);
  thread_local std::vector<double> cache(kL * kL * kL, std::numeric_limits<double>::quiet_NaN());
  double& v = cache[(l1 * kL + l2) * kL + l3];
  if (std::isnan(v)) v = wigner3j(l1, l2, l3, 0, 0, 0);
  return v;
}

double complex_gaunt(int l1, int m1, int l2, int m2, int l3, int m3) {
  if (m1 + m2 + m3 != 0) return 0.0;
  const double t0 = wigner3j_000(l1, l2, l3);
  if (t0 == 0.0) return 0.0;
  return std::sqrt((2.0 * l1 + 1) * (2.0 * l2 + 1) * (2.0 * l3 + 1) / (4.0 * M_PI)) * t0 *
         wigner3j(l1, l2, l3, m1, m2, m3);
}

// Coefficients of the real harmonic Y_{l m} in the complex basis (Condon-Shortley
// complex harmonics Y_l^mu):  Y_{l,0} = Y_l^0;  for m > 0
// Y_{l,m} = ((-1)^m Y_l^m + Y_l^{-m}) / sqrt2;  for m < 0, mu = |m|,
// Y_{l,m} = -i ((-1)^mu Y_l^mu - Y_l^{-mu}) / sqrt2.
int real_to_complex(int m, int mu[2], std::complex<double> u[2]) {
  const double r = 1.0 / std::sqrt(2.0);
  if (m == 0) {
    mu[0] = 0;
    u[0] = 1.0;
    return 1;
  }
  const int a = std::abs(m);
  const double s = (a & 1) ? -1.0 : 1.0;
  mu[0] = a;
  mu[1] = -a;
  if (m > 0) {
    u[0] = s * r;
    u[1] = r;
  } else {
    u[0] = std::complex<double>(0.0, -s * r);
    u[1] = std::complex<double>(0.0, r);
  }
  return 2;
}

}  // namespace

double real_gaunt(int l1, int m1, int l2, int m2, int l3, int m3) {
  int mu1[2], mu2[2], mu3[2];
  std::complex<double> u1[2], u2[2], u3[2];
  const int n1 = real_to_complex(m1, mu1, u1), n2 = real_to_complex(m2, mu2, u2), n3 = real_to_complex(m3, mu3, u3);
  std::complex<double> acc = 0.0;
  // complex Gaunt values already computed in this call; G(-mu) = (-1)^(l1+l2+l3) G(mu)
  int seen_mu[8][2];
  double seen_g[8];
  int nseen = 0;
  const double parity = ((l1 + l2 + l3) & 1) ? -1.0 : 1.0;
  for (int a = 0; a < n1; ++a)
    for (int b = 0; b < n2; ++b)
      for (int c = 0; c < n3; ++c) {
        if (mu1[a] + mu2[b] + mu3[c] != 0) continue;
        double G = 0.0;
        bool found = false;
        for (int i = 0; i < nseen && !found; ++i)
          if (seen_mu[i][0] == -mu1[a] && seen_mu[i][1] == -mu2[b]) {
            G = parity * seen_g[i];
            found = true;
          }
        if (!found) {
          G = complex_gaunt(l1, mu1[a], l2, mu2[b], l3, mu3[c]);
          seen_mu[nseen][0] = mu1[a];
          seen_mu[nseen][1] = mu2[b];
          seen_g[nseen++] = G;
        }
        acc += u1[a] * u2[b] * u3[c] * G;
      }
  return acc.real();
}

namespace {

struct Entry {
  int q2, q3;
  double w;
};

// Append one task to a program.  ent[chan][slot] = that slice's entries sorted by (q2, q3).
std::string emit_task(Program& P, int q1_base, int nslots, int l1, const std::vector<int>& chans,
                      const std::vector<std::vector<std::vector<Entry>>>& ent, int K, bool radial_fp64) {
  P.task_off.push_back((int32_t)P.prog.size());
  P.task_l1.push_back(l1);
  P.prog.push_back(q1_base);
  P.prog.push_back(nslots);
  P.prog.push_back((int32_t)chans.size());
  double cost = 0.0;
  for (size_t ci = 0; ci < chans.size(); ++ci) {
    P.prog.push_back(chans[ci]);
    P.prog.push_back((int32_t)(P.groups.size() / 4));
    const size_t hdr = P.prog.size();
    for (int s = 0; s < nslots; ++s) P.prog.push_back(0);
    for (int s = 0; s < nslots; ++s) {
      const auto& e = ent[ci][s];
      int ng = 0;
      size_t i = 0;
      while (i < e.size()) {
        size_t j = i;
        while (j < e.size() && e[j].q2 == e[i].q2) ++j;
        const int ne = (int)(j - i);
        if (ne > 2) return "a rank-1 group with more than two entries";
        P.groups.push_back(e[i].q2);
        P.groups.push_back(ne);
        P.groups.push_back(e[i].q3);
        P.groups.push_back(ne > 1 ? e[i + 1].q3 : e[i].q3);
        P.gw.push_back(e[i].w);
        P.gw.push_back(ne > 1 ? e[i + 1].w : 0.0);
        cost += 2.0 * K * K + 2.0 * K * ne;
        ++ng;
        i = j;
      }
      P.prog[hdr + s] = ng;
      if (radial_fp64) cost += 2.0 * K * K * K;
    }
  }
  P.task_cost.push_back(cost);
  return "";
}

}  // namespace

// Split tasks [0, ntasks) into n contiguous chunks of about equal cost.
std::vector<int32_t> split_tasks(const std::vector<double>& cost, int n) {
  const int nt = (int)cost.size();
  n = std::max(1, std::min(n, nt));
  double total = 0.0;
  for (double c : cost) total += c;
  std::vector<int32_t> b(1, 0);
  double acc = 0.0;
  int t = 0;
  for (int i = 1; i < n; ++i) {
    const double target = total * i / n;
    while (t < nt && acc + 0.5 * cost[t] < target) acc += cost[t++];
    if (t <= b.back()) t = b.back() + 1;
    if (t > nt - (n - i)) t = nt - (n - i);
    b.push_back(t);
  }
  b.push_back(nt);
  return b;
}


std::string build_tables(int kmax, int lmax, Tables& t) {
  if (kmax < 0 || kmax > 16 || lmax < 0 || lmax > 20) return "Kmax must be in [0, 16] and Lmax in [0, 20]";
  t.kmax = kmax;
  t.lmax = lmax;
  t.K = kmax + 1;
  t.NQ = (lmax + 1) * (lmax + 1);
  const int L1 = lmax + 1;
  t.chan_of.assign(L1 * L1 * L1, -1);
  t.chans.clear();
  for (int l1 = 0; l1 <= lmax; ++l1)
    for (int l2 = 0; l2 <= lmax; ++l2)
      for (int l3 = std::abs(l1 - l2); l3 <= std::min(l1 + l2, lmax); ++l3)
        if (((l1 + l2 + l3) & 1) == 0) {
          t.chan_of[(l1 * L1 + l2) * L1 + l3] = (int)t.chans.size();
          t.chans.push_back({l1, l2, l3});
        }
  // COO in Table 1 order: q3 slowest, then q2, q1 fastest.
  std::vector<int> ql(t.NQ), qm(t.NQ);
  for (int q = 0; q < t.NQ; ++q) {
    ql[q] = lq(q);
    qm[q] = q - ql[q] * ql[q] - ql[q];
  }
  t.q1.clear(); t.q2.clear(); t.q3.clear(); t.c.clear(); t.g.clear();
  for (int c3 = 0; c3 < t.NQ; ++c3)
    for (int c2 = 0; c2 < t.NQ; ++c2)
      for (int c1 = 0; c1 < t.NQ; ++c1) {
        const int l1 = ql[c1], l2 = ql[c2], l3 = ql[c3];
        const int ch = t.chan_of[(l1 * L1 + l2) * L1 + l3];
        if (ch < 0) continue;
        const int a1 = std::abs(qm[c1]), a2 = std::abs(qm[c2]), a3 = std::abs(qm[c3]);
        if (a1 != a2 + a3 && a1 != std::abs(a2 - a3)) continue;
        const int nsin = (qm[c1] < 0) + (qm[c2] < 0) + (qm[c3] < 0);
        if (nsin & 1) continue;
        const double g = real_gaunt(l1, qm[c1], l2, qm[c2], l3, qm[c3]);
        if (std::fabs(g) < 1e-14) continue;
        t.q1.push_back(c1); t.q2.push_back(c2); t.q3.push_back(c3); t.c.push_back(ch); t.g.push_back(g);
      }
  // Symmetrised channels (l2 <= l3) and their slices.
  t.sym_chan.clear();
  t.sym_partner.clear();
  std::vector<int> sym_of(t.chans.size(), -1);
  for (size_t c = 0; c < t.chans.size(); ++c) {
    const Channel& ch = t.chans[c];
    if (ch.l2 <= ch.l3) {
      sym_of[c] = (int)t.sym_chan.size();
      t.sym_chan.push_back((int)c);
      t.sym_partner.push_back(t.chan_of[(ch.l1 * L1 + ch.l3) * L1 + ch.l2]);
    }
  }
  const int NS = (int)t.sym_chan.size();
  // entries per (sym channel, q1), sorted by (q2, q3)
  std::vector<std::vector<Entry>> sl((size_t)NS * t.NQ);
  for (size_t z = 0; z < t.g.size(); ++z) {
    const int sc = sym_of[t.c[z]];
    if (sc < 0) continue;
    const Channel& ch = t.chans[t.c[z]];
    double w = t.g[z];
    if (ch.l2 == ch.l3) {
      if (t.q2[z] > t.q3[z]) continue;
      if (t.q2[z] == t.q3[z]) w *= 0.5;
    }
    sl[(size_t)sc * t.NQ + t.q1[z]].push_back({t.q2[z], t.q3[z], w});
  }
  t.n_sym_entries = t.n_sym_groups = t.n_sym_slices = 0;
  for (auto& v : sl) {
    std::sort(v.begin(), v.end(), [](const Entry& a, const Entry& b) { return a.q2 != b.q2 ? a.q2 < b.q2 : a.q3 < b.q3; });
    if (!v.empty()) ++t.n_sym_slices;
    t.n_sym_entries += (int64_t)v.size();
    for (size_t i = 0; i < v.size(); ++i)
      if (i == 0 || v[i].q2 != v[i - 1].q2) ++t.n_sym_groups;
  }
  // Radial-first program: per shell, per channel, group the channel's entries by q2,
  // then by q3; each (q2, q3) pair feeds at most two q1 of the shell.  Blocks of J q2
  // groups list the union of their q3 with a membership mask.
  {
    RadialProgram& RP = t.rprog;
    RP = RadialProgram();
    const int K = t.K, J = rf_group_width(K, rf_uses_tmem(K, 2 * lmax + 1));
    RP.J = J;
    for (int l1 = 0; l1 <= lmax; ++l1) {
      const int q1b = l1 * l1, n1 = 2 * l1 + 1;
      RP.n1max = std::max(RP.n1max, n1);
      const int cs = (int)RP.chans.size() / 4;
      int nch = 0;
      double cost = 0.0;
      for (int sc = 0; sc < NS; ++sc) {
        if (t.chans[t.sym_chan[sc]].l1 != l1) continue;
        // q2 -> q3 -> list of (q1 offset, w)
        std::map<int, std::map<int, std::vector<std::pair<int, double>>>> byp;
        for (int m = 0; m < n1; ++m)
          for (const Entry& e : sl[(size_t)sc * t.NQ + q1b + m]) byp[e.q2][e.q3].push_back({m, e.w});
        if (byp.empty()) continue;
        // q2 groups ordered so that each block of J shares as many q3 as possible: greedily,
        // the pair of remaining groups sharing the most q3 (ties: the lowest q2), then the
        // J-2 groups sharing the most q3 with the block.
        std::vector<int> q2s;
        {
          std::vector<int> rest;
          std::map<int, std::vector<int>> q3of;  // q2 -> its q3, ascending
          for (const auto& kv : byp) {
            rest.push_back(kv.first);
            for (const auto& kq : kv.second) q3of[kv.first].push_back(kq.first);
          }
          auto n_shared = [&](int a, int b) {
            const std::vector<int>& x = q3of[a];
            const std::vector<int>& y = q3of[b];
            size_t n = 0;
            for (size_t i = 0, k = 0; i < x.size() && k < y.size();) {
              if (x[i] < y[k]) ++i;
              else if (y[k] < x[i]) ++k;
              else ++n, ++i, ++k;
            }
            return n;
          };
          while (!rest.empty()) {
            size_t sa = 0, sb = 0, best_pair = 0;
            bool pair = false;
            if (J > 1)
              for (size_t i = 0; i < rest.size(); ++i)
                for (size_t k = i + 1; k < rest.size(); ++k) {
                  const size_t n = n_shared(rest[i], rest[k]);
                  if (!pair || n > best_pair) {
                    best_pair = n;
                    sa = i;
                    sb = k;
                    pair = true;
                  }
                }
            std::set<int> uni;
            auto take = [&](size_t i) {
              for (const auto& kv : byp[rest[i]]) uni.insert(kv.first);
              q2s.push_back(rest[i]);
            };
            take(sa);
            if (pair) take(sb);
            if (pair) rest.erase(rest.begin() + (long)sb);  // sb > sa
            rest.erase(rest.begin() + (long)sa);
            for (int j = pair ? 2 : 1; j < J && !rest.empty(); ++j) {
              size_t best = 0, best_shared = 0;
              for (size_t i = 0; i < rest.size(); ++i) {
                size_t shared = 0;
                for (const auto& kv : byp[rest[i]]) shared += uni.count(kv.first);
                if (shared > best_shared) {
                  best_shared = shared;
                  best = i;
                }
              }
              for (const auto& kv : byp[rest[best]]) uni.insert(kv.first);
              q2s.push_back(rest[best]);
              rest.erase(rest.begin() + (long)best);
            }
          }
        }
        const int bs = (int)RP.blocks.size() / 8;
        int nblk = 0;
        for (size_t b0 = 0; b0 < q2s.size(); b0 += J) {
          const int nj = (int)std::min<size_t>(J, q2s.size() - b0);
          std::map<int, int> mask;  // q3 -> bits
          for (int j = 0; j < nj; ++j)
            for (const auto& kv : byp[q2s[b0 + j]]) mask[kv.first] |= 1 << j;
          RP.blocks.insert(RP.blocks.end(), {nj, (int32_t)(RP.uents.size() / 4), (int32_t)mask.size(), 0});
          for (int j = 0; j < 4; ++j) RP.blocks.push_back(j < nj ? q2s[b0 + j] : 0);
          for (const auto& mk : mask) {
            const int q3 = mk.first;
            const size_t u = RP.uents.size();
            RP.uents.insert(RP.uents.end(), {q3 | mk.second << 16, (int32_t)(RP.pw.size() / 2), 0, 0});
            for (int j = 0; j < nj; ++j) {
              if (!(mk.second >> j & 1)) continue;
              const auto& v = byp[q2s[b0 + j]][q3];
              if (v.size() > 2) return "a radial-first pair feeding more than two q1";
              if (n1 > 127) return "a shell too large for the radial-first target encoding";
              const int32_t T = v[0].first | (v.size() > 1 ? v[1].first : 0) << 8 | (v.size() > 1 ? 1 << 15 : 0);
              RP.uents[u + 2 + j / 2] = (int32_t)((uint32_t)RP.uents[u + 2 + j / 2] | (uint32_t)T << (16 * (j & 1)));
              RP.pw.push_back(std::ldexp(v[0].second, kRfWeightExp));
              RP.pw.push_back(v.size() > 1 ? std::ldexp(v[1].second, kRfWeightExp) : 0.0);
              cost += 2.0 * K * K + 2.0 * K * (double)v.size();
              RP.fp32_flops += 2.0 * K * K;
              RP.fp64_flops += 2.0 * K * (double)v.size();
            }
          }
          cost += 2.0 * K * K * K * nj;
          RP.fp32_flops += 2.0 * K * K * K * nj;
          RP.n_groups += nj;
          ++nblk;
        }
        RP.chans.insert(RP.chans.end(), {sc, bs, nblk, 0});
        ++nch;
      }
      RP.tasks.insert(RP.tasks.end(), {q1b, n1, cs, nch});
      RP.task_cost.push_back(cost);
    }
    RP.order.resize(RP.task_cost.size());
    for (size_t i = 0; i < RP.order.size(); ++i) RP.order[i] = (int32_t)i;
    std::stable_sort(RP.order.begin(), RP.order.end(),
                     [&](int a, int b) { return RP.task_cost[a] > RP.task_cost[b]; });
  }
  // Programs.
  for (int variant = 0; variant < 2; ++variant) {
    Program& P = variant == 0 ? t.prog1 : t.prog4;
    P = Program();
    P.nslots = variant == 0 ? 1 : 4;
    for (int l1 = 0; l1 <= lmax; ++l1) {
      std::vector<int> chans;
      for (int s = 0; s < NS; ++s)
        if (t.chans[t.sym_chan[s]].l1 == l1) chans.push_back(s);
      const int n1 = 2 * l1 + 1;
      for (int base = 0; base < n1; base += P.nslots) {
        const int ns = std::min(P.nslots, n1 - base);
        const int q1b = l1 * l1 + base;
        std::vector<std::vector<std::vector<Entry>>> ent(chans.size(), std::vector<std::vector<Entry>>(ns));
        for (size_t ci = 0; ci < chans.size(); ++ci)
          for (int s = 0; s < ns; ++s) ent[ci][s] = sl[(size_t)chans[ci] * t.NQ + q1b + s];
        std::string err = emit_task(P, q1b, ns, l1, chans, ent, t.K, variant == 0);
        if (!err.empty()) return err;
      }
    }
    P.task_off.push_back((int32_t)P.prog.size());
  }
  return "";
}

}  // namespace wef
