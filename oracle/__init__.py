"""Plain FP64 CPU oracle for the Wigner-Eckart factorized collision operator.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports this
package; only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may call it.  It shares no code with the CUDA path: it has
its own basis functions, its own real Gaunt table (computed by sphere
quadrature, not by Wigner 3-j formulas), its own kinematic-core quadrature
(the paper's 5D Duffy scheme with an explicit scattering-sphere rule) and a
dense Cartesian contraction.

Modules
-------
basis   radial Laguerre functions and real spherical harmonics (§2.2, §4.1)
gaunt   channel list, real Gaunt tensor and its COO table (§4.1, §4.2, §4.6)
dense   null-space / detailed-balance zeroing and the dense contraction
        Q_a = sum_bc C_abc f_b f_c with C = R * G (§2.3, §4.1, §4.4, §4.5.1)
core    the reduced kinematic core R by 5D singular quadrature
        (§3.2-3.3, §4.3, Appendix A, Appendix B)
angular_first
        the paper's factorised angular-first contraction (§4.5.4) in plain numpy,
        pinned to dense; a CPU comparison point for the bench

Parity status: every function here is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_*.py`` against closed forms or values printed in the paper
(Table 1, Table 3, Table 5, Table 6).  The core for any power law u^gamma (Maxwell,
VHS gamma=0.5, hard spheres) is also pinned entry by entry to an exact 8D evaluation of
the weak form in centre-of-mass and relative velocity at small (Kmax, Lmax).
"""
