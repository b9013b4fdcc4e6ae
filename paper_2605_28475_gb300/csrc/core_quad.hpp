// Quadrature set-up shared by the host and the device builders of the kinematic core
// (paper Sec. 4.3, Appendix A-B): point counts with padding, rules, and the per-channel
// constants of the Funk-Hecke reduced integrand.
#pragma once
#include <string>
#include <vector>

#include "tables.hpp"

namespace wef {

struct CoreQuad {
  int kmax = 0, lmax = 0, K = 0, L1 = 0, NT = 0;
  double gamma = 0.0;
  double pref = 0.0;                  // 2^gamma * 4 / (2 pi)^3
  std::vector<Channel> ch;            // paper order
  std::vector<double> Nkl;            // [k][l] radial normalisation
  std::vector<double> ylm_norm;       // [l][m], m >= 0, cos-type normalisation incl. sqrt2
  std::vector<double> Ghat;           // [c][m] = G[(l1 m),(l2 0),(l3 m)], m = 0..min(l1,l3)
  std::vector<int> Ghat_off;          // [c]
  std::vector<double> s2;             // [c] Y_{l2 0}(z_hat)
  std::vector<double> S;              // [c] channel norm sum_m g^2
  std::vector<double> ftx, ftw;       // Funk-Hecke Gauss-Legendre rule on [-1, 1]
  std::vector<double> zz, wz;         // generalised Gauss-Laguerre (weight z^{gamma/2} e^-z)
  std::vector<double> x1, wx1, h1, wh1;  // patch 1: outer x, inner h, Gauss-Legendre on [0, 1]
  std::vector<double> y2, wy2, h2, wh2;  // patch 2: outer y, inner h, Gauss-Legendre on [0, 1]
};

// Fills Q for the operator's tables; returns "" on success.
std::string core_quadrature(const Tables& T, double gamma, int pad_rad, int pad_ang, CoreQuad& Q);

}  // namespace wef
