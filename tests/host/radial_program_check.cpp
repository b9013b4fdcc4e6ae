// Walk the radial-first program (blocks of q2 groups, union of q3) on the host:
// bounds, coverage and Q against the direct COO sum.
#include <cmath>
#include <cstdio>
#include <random>
#include <utility>
#include <vector>
#include "../../paper_2605_28475_gb300/csrc/tables.hpp"
using namespace wef;
int main() {
  int bad = 0;
  // every (Lmax, Kmax) of the grid, then the largest operators (tensor-memory placement)
  std::vector<std::pair<int, int>> shapes;
  for (int L : {0, 1, 2, 3, 4, 6, 8, 12}) for (int km : {0, 1, 4, 8, 12, 16}) shapes.push_back({L, km});
  for (int L : {16, 20}) shapes.push_back({L, 16});
  for (int L : {4, 8, 12}) for (int km : {13, 14, 15}) shapes.push_back({L, km});  // K = 14-16
  for (const auto& sh : shapes) {
    const int L = sh.first, km = sh.second;
    Tables T; std::string e = build_tables(km, L, T); if (!e.empty()) { printf("err %s\n", e.c_str()); return 1; }
    const int K = T.K, NQ = T.NQ, NS = (int)T.sym_chan.size(), NT = (int)T.chans.size();
    std::mt19937_64 rng(km * 100 + L); std::normal_distribution<double> nd;
    std::vector<double> R((size_t)NT * K * K * K), f((size_t)K * NQ);
    for (auto& x : R) x = nd(rng); for (auto& x : f) x = nd(rng);
    std::vector<double> Qref((size_t)K * NQ, 0.0);
    for (size_t z = 0; z < T.g.size(); ++z) for (int k1 = 0; k1 < K; ++k1) {
      double a = 0; for (int k2 = 0; k2 < K; ++k2) for (int k3 = 0; k3 < K; ++k3)
        a += R[(((size_t)T.c[z] * K + k1) * K + k2) * K + k3] * f[k2 * NQ + T.q2[z]] * f[k3 * NQ + T.q3[z]];
      Qref[k1 * NQ + T.q1[z]] += T.g[z] * a; }
    std::vector<double> Rt((size_t)NS * K * K * K);
    for (int s = 0; s < NS; ++s) for (int k1 = 0; k1 < K; ++k1) for (int k2 = 0; k2 < K; ++k2) for (int k3 = 0; k3 < K; ++k3)
      Rt[(((size_t)s * K + k1) * K + k2) * K + k3] = R[(((size_t)T.sym_chan[s] * K + k1) * K + k2) * K + k3] + R[(((size_t)T.sym_partner[s] * K + k1) * K + k3) * K + k2];
    const RadialProgram& P = T.rprog;
    const int J = P.J;
    if (J != rf_group_width(K, rf_uses_tmem(K, 2 * L + 1))) { bad++; printf("J\n"); }
    std::vector<double> Q((size_t)K * NQ, 0.0);
    std::vector<int> seen(NQ, 0);
    const int ntasks = (int)P.tasks.size() / 4, nch_all = (int)P.chans.size() / 4, nb_all = (int)P.blocks.size() / 8,
              nu_all = (int)P.uents.size() / 4, np_all = (int)P.pw.size() / 2;
    int64_t npairs_seen = 0;
    for (int oi = 0; oi < ntasks; ++oi) {
      const int t = P.order[oi];
      const int q1b = P.tasks[4*t], n1 = P.tasks[4*t+1], cs = P.tasks[4*t+2], nch = P.tasks[4*t+3];
      if (n1 > P.n1max || q1b + n1 > NQ) { bad++; printf("task bad\n"); }
      for (int m = 0; m < n1; ++m) seen[q1b + m]++;
      for (int ch = cs; ch < cs + nch; ++ch) {
        if (ch >= nch_all) { bad++; printf("chan idx\n"); continue; }
        const int sc = P.chans[4*ch], bs = P.chans[4*ch+1], nb = P.chans[4*ch+2];
        if (sc < 0 || sc >= NS) { bad++; printf("sc bad\n"); }
        for (int bi = bs; bi < bs + nb; ++bi) {
          if (bi >= nb_all) { bad++; printf("blk idx\n"); continue; }
          const int* B = &P.blocks[8 * bi];
          const int nj = B[0], us = B[1], nu = B[2];
          if (nj < 1 || nj > J) { bad++; printf("nj bad\n"); }
          std::vector<std::vector<double>> A(nj, std::vector<double>((size_t)K * K, 0.0));  // [j][k1*K+k3]
          for (int j = 0; j < nj; ++j) {
            const int q2 = B[4 + j];
            if (q2 < 0 || q2 >= NQ) { bad++; printf("q2 bad\n"); }
            for (int k1 = 0; k1 < K; ++k1) for (int k3 = 0; k3 < K; ++k3) for (int k2 = 0; k2 < K; ++k2)
              A[j][k1 * K + k3] += Rt[(((size_t)sc * K + k1) * K + k2) * K + k3] * f[k2 * NQ + q2];
          }
          for (int ui = us; ui < us + nu; ++ui) {
            if (ui >= nu_all) { bad++; printf("u idx\n"); continue; }
            const int q3 = P.uents[4*ui] & 0xFFFF, mask = P.uents[4*ui] >> 16;
            int p = P.uents[4*ui+1];
            if (q3 < 0 || q3 >= NQ || mask <= 0 || mask >= (1 << nj)) { bad++; printf("uent bad\n"); }
            for (int j = 0; j < nj; ++j) {
              if (!(mask >> j & 1)) continue;
              if (p >= np_all) { bad++; printf("pair idx\n"); break; }
              const uint32_t T = ((uint32_t)P.uents[4*ui + 2 + j / 2] >> (16 * (j & 1))) & 0xFFFFu;
              const int a = T & 0xFF, b = (T >> 8) & 0x7F, ne = (T >> 15) ? 2 : 1;
              if (ne < 1 || ne > 2 || a < 0 || a >= n1 || b < 0 || b >= n1) { bad++; printf("pair bad\n"); }
              for (int k1 = 0; k1 < K; ++k1) {
                double Bv = 0; for (int k3 = 0; k3 < K; ++k3) Bv += A[j][k1 * K + k3] * f[k3 * NQ + q3];
                Q[k1 * NQ + q1b + a] += std::ldexp(P.pw[2*p], -kRfWeightExp) * Bv;
                if (ne > 1) Q[k1 * NQ + q1b + b] += std::ldexp(P.pw[2*p+1], -kRfWeightExp) * Bv;
              }
              ++p; ++npairs_seen;
            }
          }
        }
      }
    }
    if (npairs_seen != np_all) { bad++; printf("pairs visited %lld of %d\n", (long long)npairs_seen, np_all); }
    for (int q = 0; q < NQ; ++q) if (seen[q] != 1) { bad++; printf("coverage\n"); }
    double err = 0, mx = 0; for (size_t i = 0; i < Q.size(); ++i) { err = fmax(err, fabs(Q[i] - Qref[i])); mx = fmax(mx, fabs(Qref[i])); }
    if (err > 1e-12 * fmax(mx, 1e-300)) { bad++; printf("K=%d L=%d rel err %g\n", K, L, err / mx); }
    if (L == 12 && km == 12) printf("L=12 K=13: J=%d groups %lld uents %d pairs %d fp64 %.2f MF fp32 %.2f MF\n", J, (long long)P.n_groups, nu_all, np_all, P.fp64_flops / 1e6, P.fp32_flops / 1e6);
  }
  printf("bad=%d\n", bad);
  return bad != 0;
}
