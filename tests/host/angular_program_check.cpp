// Walk the kernel programs on the host exactly as the kernels do; check bounds and evaluate Q.
#include <cstdio>
#include <cmath>
#include <random>
#include <utility>
#include <vector>
#include "../../paper_2605_28475_gb300/csrc/tables.hpp"
using namespace wef;
int main() {
  int bad = 0;
  // the grid, then the largest operator the library accepts (Kmax = 16, Lmax = 20)
  std::vector<std::pair<int, int>> shapes;
  for (int L : {0, 1, 2, 3, 4, 6, 8, 12, 16}) for (int km : {0, 1, 4, 12}) shapes.push_back({L, km});
  shapes.push_back({20, 16});
  for (const auto& sh : shapes) {
    const int L = sh.first, km = sh.second;
    Tables T; std::string e = build_tables(km, L, T); if (!e.empty()) { printf("err %s\n", e.c_str()); return 1; }
    const int K = T.K, NQ = T.NQ, NS = (int)T.sym_chan.size(), NT = (int)T.chans.size();
    std::mt19937_64 rng(km * 100 + L); std::normal_distribution<double> nd;
    std::vector<double> R((size_t)NT * K * K * K), f((size_t)K * NQ);
    for (auto& x : R) x = nd(rng); for (auto& x : f) x = nd(rng);
    // reference: direct COO sum (full discrete sum, Sec 4.5)
    std::vector<double> Qref((size_t)K * NQ, 0.0);
    for (size_t z = 0; z < T.g.size(); ++z) for (int k1 = 0; k1 < K; ++k1) {
      double a = 0; for (int k2 = 0; k2 < K; ++k2) for (int k3 = 0; k3 < K; ++k3)
        a += R[(((size_t)T.c[z] * K + k1) * K + k2) * K + k3] * f[k2 * NQ + T.q2[z]] * f[k3 * NQ + T.q3[z]];
      Qref[k1 * NQ + T.q1[z]] += T.g[z] * a; }
    // symmetrised core
    std::vector<double> Rt((size_t)NS * K * K * K);
    for (int s = 0; s < NS; ++s) for (int k1 = 0; k1 < K; ++k1) for (int k2 = 0; k2 < K; ++k2) for (int k3 = 0; k3 < K; ++k3)
      Rt[(((size_t)s * K + k1) * K + k2) * K + k3] = R[(((size_t)T.sym_chan[s] * K + k1) * K + k2) * K + k3] + R[(((size_t)T.sym_partner[s] * K + k1) * K + k3) * K + k2];
    for (int v = 0; v < 2; ++v) {
      const Program& P = v ? T.prog4 : T.prog1;
      const int ng_total = (int)P.groups.size() / 4;
      std::vector<double> Q((size_t)K * NQ, 0.0);
      std::vector<int> seen(NQ, 0);
      for (int t = 0; t < P.ntasks(); ++t) {
        const int32_t* p = P.prog.data() + P.task_off[t];
        int q1b = p[0], ns = p[1], nch = p[2]; p += 3;
        if (ns < 1 || ns > P.nslots || q1b < 0 || q1b + ns > NQ) { bad++; printf("task hdr bad\n"); }
        for (int s = 0; s < ns; ++s) seen[q1b + s]++;
        for (int ci = 0; ci < nch; ++ci) {
          int sc = p[0], gs = p[1]; const int32_t* ngs = p + 2; p += 2 + ns;
          if (sc < 0 || sc >= NS) { bad++; printf("sc bad\n"); }
          for (int s = 0; s < ns; ++s) {
            std::vector<double> Phi((size_t)K * K, 0.0);
            for (int gi = 0; gi < ngs[s]; ++gi, ++gs) {
              if (gs < 0 || gs >= ng_total) { bad++; printf("group index bad\n"); continue; }
              const int32_t* G = &P.groups[(size_t)gs * 4]; const double* W = &P.gw[(size_t)gs * 2];
              if (G[0] < 0 || G[0] >= NQ || G[2] < 0 || G[2] >= NQ || G[3] < 0 || G[3] >= NQ || G[1] < 1 || G[1] > 2) { bad++; printf("group bad\n"); }
              for (int k3 = 0; k3 < K; ++k3) {
                double h = W[0] * f[k3 * NQ + G[2]]; if (G[1] > 1) h += W[1] * f[k3 * NQ + G[3]];
                for (int k2 = 0; k2 < K; ++k2) Phi[k2 * K + k3] += f[k2 * NQ + G[0]] * h; }
            }
            for (int k1 = 0; k1 < K; ++k1) { double a = 0;
              for (int k = 0; k < K * K; ++k) a += Rt[((size_t)sc * K + k1) * K * K + k] * Phi[k];
              Q[k1 * NQ + q1b + s] += a; }
          }
        }
        if (p != P.prog.data() + P.task_off[t + 1]) { bad++; printf("task length mismatch\n"); }
      }
      for (int q = 0; q < NQ; ++q) if (seen[q] != 1) { bad++; printf("q1 coverage bad\n"); }
      double err = 0, mx = 0; for (size_t i = 0; i < Q.size(); ++i) { err = fmax(err, fabs(Q[i] - Qref[i])); mx = fmax(mx, fabs(Qref[i])); }
      if (err > 1e-12 * fmax(mx, 1e-300)) { bad++; printf("K=%d L=%d v=%d rel err %g\n", K, L, v, err / mx); }
    }
  }
  printf("bad=%d\n", bad);
  return bad != 0;
}
