"""Per-cell error of a result against the oracle, guarded against cancellation, and the
tolerances of the evaluation paths.

For every compared cell i (over the compared output rows a):

    e_i = max_a |Q_ia - Qo_ia| / max( max_a |Qo_ia| ,  EPS * max_a T_ia )

with T_ia = sum of |terms| of Qo_ia (the oracle's ``evaluate_rows_with_terms``): the size of
the terms whose sum is Q_ia.  A rounding error is proportional to T, not to Q, so a cell
whose Q cancels to below EPS of its terms is measured against that floor instead of against
its own tiny Q (the guard of the per-cell infinity norm).  The tests assert max_i e_i.

Tolerances: FP64 paths 1e-12.  A mixed path rounds the operands of its radial products
(f and the core, and for the angular-first paths the FP64 coupling Phi) to the unit
roundoff u of its format and sums short FP32 dot products, so its error is a small multiple
of u times the size of the terms; relative to the guarded norm that is (growth factor) * u.
The factor is stated per path and per kind of core: random stand-in cores (entries of one
scale, mild cancellation) and the physical hard-sphere core, whose cells near equilibrium
cancel strongly (Q(M, M) = 0) so that the same rounding is a larger fraction of Q.  Each
factor sits about 3-5x above the largest error measured on the seeded inputs of these tests
(GB300), so that a regression of that size fails.
"""
import numpy as np

EPS = 2.0 ** -10  # cancellation floor, relative to the largest sum of |terms| of the cell

UNIT_ROUNDOFF = {"fp64": 2.0 ** -53, "rf32": 2.0 ** -24, "rftc": 2.0 ** -24, "tf32": 2.0 ** -11, "bf16": 2.0 ** -8}
# growth factors (tolerance = factor * unit roundoff of the path's radial operands).
# Largest measured per-cell errors: random cores rf32 4.1e-7 (6.8 u, Kmax = 16, Lmax = 20),
# tf32 9.0e-4 (1.8 u), bf16 6.3e-3 (1.6 u); hard-sphere core at Kmax = Lmax = 12, 64
# two-Maxwellian cells: rf32 7.4e-7 (12 u), tf32 7.0e-3 (14 u), bf16 3.0e-2 (7.8 u).
# rftc (stage 1 on the tensor cores from split TF32 operands, three products per term, each
# within a few FP32 units of the exact product) is held to the bounds of rf32: measured 2.4-3.1 u
# on random cores at K = 9, 11, 13 against 1.9-2.3 u for rf32 on the same inputs.
GROWTH = {"rf32": 24.0, "rftc": 24.0, "tf32": 6.0, "bf16": 6.0}
GROWTH_PHYSICAL = {"rf32": 48.0, "rftc": 48.0, "tf32": 48.0, "bf16": 32.0}
FP64_TOL = 1e-12


def tolerance(prec, physical=False):
    """Bound of the per-cell guarded error of path `prec` (physical: the hard-sphere core)."""
    if prec == "fp64":
        return FP64_TOL
    return (GROWTH_PHYSICAL if physical else GROWTH)[prec] * UNIT_ROUNDOFF[prec]


def cell_errors(Q, Qo, T):
    """e_i for every cell: Q, Qo, T of shape [ncells, rows] (or [ncells, K, NQ])."""
    Q = np.asarray(Q, dtype=np.float64).reshape(len(Q), -1)
    Qo = np.asarray(Qo, dtype=np.float64).reshape(len(Qo), -1)
    T = np.asarray(T, dtype=np.float64).reshape(len(T), -1)
    num = np.max(np.abs(Q - Qo), axis=1)
    den = np.maximum(np.max(np.abs(Qo), axis=1), EPS * np.max(T, axis=1))
    return num / np.maximum(den, 1e-300)


def summary(e):
    e = np.asarray(e)
    return {"max": float(np.max(e)), "median": float(np.median(e)), "cells": int(e.size)}
