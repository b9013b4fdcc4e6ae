// Host-side angular geometry of the operator (paper Sec. 4.1, 4.2, 4.5.4, 4.6).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace wef {

struct Channel {
  int l1, l2, l3;
};

// Wigner 3-j symbol (j1 j2 j3; m1 m2 m3) for integer arguments, exact integer
// binomial sum times a prime-factorised square-root prefactor.
double wigner3j(int j1, int j2, int j3, int m1, int m2, int m3);

// Real Gaunt coefficient: integral over S^2 of Y_{l1 m1} Y_{l2 m2} Y_{l3 m3}
// for the real harmonics of the library (no Condon-Shortley phase, cos-type for
// m > 0, sin-type for m < 0), from complex Gaunt coefficients mapped by the
// unitary complex -> real transform (Sec. 4.1).
double real_gaunt(int l1, int m1, int l2, int m2, int l3, int m3);

// One evaluation "program": the instruction stream that the kernels walk.
// Tasks are groups of output rows (cell x q1); each task lists its channels, and
// per channel and per q1 slot a run of rank-1 groups.
//
// prog (int32 words), per task: [q1_base, nslots, nchan], then per channel
//   [sc, gstart, ngroups_slot0, ..., ngroups_slot{nslots-1}]
// where the slot groups are consecutive records of `groups` from index gstart.
// groups: 4 int32 per group {q2, ne, q3a, q3b} (ne in {1, 2}; q3b = q3a if ne = 1);
// gw: 2 doubles per group {weight a, weight b} (b = 0 if ne = 1).
struct Program {
  int nslots = 1;
  std::vector<int32_t> prog;
  std::vector<int32_t> groups;
  std::vector<double> gw;
  std::vector<int32_t> task_off;  // word offset of task t (size ntasks + 1)
  std::vector<double> task_cost;  // FP64 flops per cell of task t (for load balance)
  std::vector<int32_t> task_l1;
  int ntasks() const { return (int)task_cost.size(); }
};

#ifdef __CUDACC__
#define WEF_HD __host__ __device__
#else
#define WEF_HD
#endif

// Whether the radial-first kernel runs one CTA per SM with the whole register file (and its
// FP64 accumulators in tensor memory): from K = 15 on, where the register budget of two CTAs
// leaves room for one q2 group per block only (K = 17, Lmax = 8-12: 0.30-0.37 of the FP64
// peak with two CTAs), and wherever two CTAs' accumulators (largest shell, n1max targets)
// would not fit in an SM's shared memory.
WEF_HD constexpr bool rf_uses_tmem(int K, int n1max) {
  return K >= 15 || 2 * ((long long)n1max * 32 * K * 8 + 1024) > 228LL * 1024;
}
// Accumulator variants of the radial-first kernel (template argument ACC): shared memory with
// the register budget of rf_ctas_per_sm(K) CTAs per SM; tensor memory with one CTA per SM
// (rf_uses_tmem); tensor memory with the register budget of rf_ctas_per_sm(K) CTAs, whose
// columns (rf_tmem_cols each) fit in the SM's 512.
constexpr int kRfAccSmem = 0, kRfAccTmem = 1, kRfAccTmem2 = 2;
WEF_HD constexpr int rf_tmem_cols(int K, int n1max) {
  int need = (K + 3) / 4 * 2 * n1max, c = 32;
  while (c < need) c <<= 1;
  return c;
}
// q2 groups the radial-first kernel keeps in registers at once (rf_group_width): its
// register budget is that of two CTAs per SM, or of one (rf_uses_tmem).  Three groups at
// K = 12-14 (K = 14 keeps as many k3 pairs as K = 13) (measured at K = 13 with the next union record
// prefetched: 379.7k against 343.2k cells/s with two) and with tensor memory above K = 9
// (K = 17: 56.9k against 49.1k); four overflow the registers there.
// CTAs per SM the shared-memory variant's register budget is sized for: about 32-36
// warps for K <= 9 (measured at K = 9: 3.63M cells/s with 4 CTAs of 56 registers against
// 2.81M with 2 of 96); two from K = 10 on, where the tighter budget spills (-2 to -5%).
WEF_HD constexpr int rf_ctas_per_sm(int K) {
  return K <= 4 ? 8 : K == 5 ? 7 : K == 6 ? 6 : K == 7 ? 5 : K <= 9 ? 4 : 2;
}
WEF_HD constexpr int rf_group_width(int K, bool tmem) {
  return tmem ? (K <= 9 ? 4 : 3) : (K <= 4 ? 4 : K <= 11 ? 2 : K <= 14 ? 3 : 1);
}

// Radial-first program (paper Sec. 4.5.3 ordering with a dense two-stage radial
// contraction).  One task per output shell l1:
//   tasks:  {q1_base, n1, chan_start, nchan}
//   chans:  {sc, blk_start, nblk, 0}        symmetrised channel (l2 <= l3)
//   blocks: two int4 per block: {nj, u_start, nu, 0}, {q2_0, q2_1, q2_2, q2_3}: up to
//           J = rf_group_width(K, tmem) of the channel's q2 (the smaller shell), whose stage-1
//           products A(q2_j) are held together
//   uents:  {q3 | mask << 16, pair_start, T_0 | T_1 << 16, T_2 | T_3 << 16}: each q3 paired
//           with any q2 of the block, once; bit j of mask set if (q2_j, q3) is a pair, whose
//           targets are T_j = (q1a - q1_base) | (q1b - q1_base) << 8 | (ne == 2) << 15 and
//           whose weights pw[pair] = {ga, gb} * 2^kRfWeightExp (gb = 0 if ne = 1) follow from
//           pair_start in j order (the kernel widens its FP32 products to FP64 scaled by
//           2^-kRfWeightExp, see f2d_scaled in rf_kernel.cuh)
// order:  task indices by decreasing cost (the persistent kernel's schedule).
// Grouping by q2 makes stage 1 (2K^3 flops per q2 group) run over 4067 instead of 6125
// groups at K = L = 12; walking the union of the block's q3 loads each f[:, q3] once per
// block instead of once per pair (32707 instead of 56981 loads of K values for J = 2).
constexpr int kRfWeightExp = 896;  // radial-first weights are stored as g * 2^896
struct RadialProgram {
  std::vector<int32_t> tasks, chans, blocks, uents;
  std::vector<double> pw;
  std::vector<int32_t> order;
  std::vector<double> task_cost;  // FP64 + FP32 flops per cell, for the schedule
  double fp64_flops = 0.0, fp32_flops = 0.0;
  int n1max = 1, J = 1;
  int64_t n_groups = 0;  // q2 groups (stage-1 products) over all tasks
};

struct Tables {
  int kmax = 0, lmax = 0, K = 0, NQ = 0;
  std::vector<Channel> chans;        // paper order
  std::vector<int> chan_of;          // (l1*(L+1)+l2)*(L+1)+l3 -> c, or -1
  std::vector<int32_t> q1, q2, q3, c;  // COO, Table 1 order (q3 slowest, q1 fastest)
  std::vector<double> g;
  // symmetrised channel set used by the kernels: channels with l2 <= l3;
  // sym_partner[s] is the paper index of (l1, l3, l2)
  std::vector<int> sym_chan, sym_partner;
  Program prog1;  // one q1 per task (FP64 path)
  Program prog4;  // up to four q1 of one shell per task (tensor-core path, 128-row tiles)
  RadialProgram rprog;  // radial-first ordering
  int64_t n_sym_entries = 0, n_sym_groups = 0, n_sym_slices = 0;
};

// Split tasks [0, ntasks) into n contiguous chunks of about equal cost; returns n+1 bounds.
std::vector<int32_t> split_tasks(const std::vector<double>& cost, int n);

// Build everything; returns "" on success or an error message.
std::string build_tables(int kmax, int lmax, Tables& t);

inline int lq(int q) {
  int l = 0;
  while ((l + 1) * (l + 1) <= q) ++l;
  return l;
}

}  // namespace wef
