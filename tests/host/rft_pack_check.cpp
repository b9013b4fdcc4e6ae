// Host check of the split-TF32 b tiles of the tensor-core first radial stage (WEF_RADIAL_TC),
// packed at core upload by wef::rft_pack_b_tiles: element (n = 16 k1 + k3, k2) of a tile at
// byte (n / 8) 512 + (k2 / 4) 128 + (n % 8) 16 + (k2 % 4) 4 (K-major core matrices of
// 8 rows x 16 bytes), hi tile then lo tile.  Checks, for random cores: every byte of both
// tiles is written by exactly one element of this map; hi and lo are TF32 values (the low 13
// bits of the FP32 pattern are zero); |v - hi| <= 2^-11 |v| and |v - hi - lo| <= 2^-22 |v|;
// zeros wherever k2 >= K or k3 >= K.  Prints "bad=<count>".
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <random>
#include <vector>

namespace wef {
void rft_pack_b_tiles(int K, const double* Rt, uint8_t* out);
}

int main() {
  std::mt19937_64 rng(7);
  std::normal_distribution<double> nd;
  std::uniform_real_distribution<double> ud(-3.0, 3.0);
  long bad = 0;
  for (int K : {9, 11, 13}) {
    std::vector<double> Rt((size_t)K * K * K);
    for (auto& x : Rt) x = nd(rng) * std::pow(10.0, ud(rng));
    const int bt = 16 * K * 16 * 4;
    std::vector<uint8_t> out(2 * (size_t)bt, 0xAB);
    wef::rft_pack_b_tiles(K, Rt.data(), out.data());
    std::vector<int> cover(bt, 0);
    for (int n = 0; n < 16 * K; ++n)
      for (int k2 = 0; k2 < 16; ++k2) {
        const size_t off = (size_t)(n / 8) * 512 + (size_t)(k2 / 4) * 128 + (n % 8) * 16 + (k2 % 4) * 4;
        if (off + 4 > (size_t)bt) { ++bad; continue; }
        for (int b = 0; b < 4; ++b) cover[off + b]++;
        float hi, lo;
        uint32_t uh, ul;
        std::memcpy(&hi, &out[off], 4);
        std::memcpy(&lo, &out[bt + off], 4);
        std::memcpy(&uh, &hi, 4);
        std::memcpy(&ul, &lo, 4);
        const int k1 = n / 16, k3 = n % 16;
        if (k2 >= K || k3 >= K) {
          if (hi != 0.0f || lo != 0.0f) ++bad;
          continue;
        }
        const double v = Rt[((size_t)k1 * K + k2) * K + k3];
        if ((uh & 0x1FFFu) || (ul & 0x1FFFu)) ++bad;                       // TF32 values
        if (std::fabs(v - (double)hi) > std::ldexp(std::fabs(v), -11)) ++bad;
        if (std::fabs(v - (double)hi - (double)lo) > std::ldexp(std::fabs(v), -22)) ++bad;
      }
    for (int i = 0; i < bt; ++i)
      if (cover[i] != 1) ++bad;  // the map covers each byte of a tile exactly once
  }
  std::printf("bad=%ld\n", bad);
  return bad == 0 ? 0 : 1;
}
