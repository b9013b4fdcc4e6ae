"""Dense Cartesian evaluation of the bilinear collision operator (§2.3, §4.5.1).

    Q_a1 = sum_{a2, a3} C_{a1 a2 a3} f_a2 f_a3,   a = (k, q),  flat index a = k*NQ + q

with the tensor assembled from the factorization of §4.1,

    C^{k1 k2 k3}_{q1 q2 q3} = R^{(c)}_{k1 k2 k3} * G_R[q1, q2, q3],   c = (l1, l2, l3).

R is stored as R[c, k1, k2, k3] (c in the order of ``gaunt.channels``).
The tensor is assembled one a1-slice at a time (an N x N matrix) because the
whole of C does not fit in memory beyond Lmax ~ 6; the quadratic form is then
f^T C_a1 f for every cell.  No symmetrisation, no reordering of the sum.
"""
import numpy as np

from . import basis, gaunt


def conservation_zeroing(R, lmax):
    """Null-space correction (§4.4.2) and detailed balance (§4.4.3) on a copy of R:

    * l1 = 0 channels: R[c][k1=0] = 0 (mass) and R[c][k1=1] = 0 (energy);
    * l1 = 1 channels: R[c][k1=0] = 0 (momentum);
    * channel (0,0,0): R[c][k1, 0, 0] = 0 for all k1 (Q(M, M) = 0)."""
    R = np.array(R, dtype=np.float64, copy=True)
    for c, (l1, l2, l3) in enumerate(gaunt.channels(lmax)):
        if l1 == 0:
            R[c, 0] = 0.0
            if R.shape[1] > 1:
                R[c, 1] = 0.0
        if l1 == 1:
            R[c, 0] = 0.0
        if (l1, l2, l3) == (0, 0, 0):
            R[c, :, 0, 0] = 0.0
    return R


class DenseOperator:
    """The dense tensor C of a (Kmax, Lmax) basis, built slice by slice from a
    core R[c, k1, k2, k3] and the oracle's own real Gaunt tensor."""

    def __init__(self, kmax, lmax, R, G=None):
        self.kmax, self.lmax = kmax, lmax
        self.K = kmax + 1
        self.NQ = (lmax + 1) ** 2
        self.N = self.K * self.NQ
        self.R = np.asarray(R, dtype=np.float64)
        assert self.R.shape == (len(gaunt.channels(lmax)), self.K, self.K, self.K)
        self.G = gaunt.gaunt_dense(lmax) if G is None else G
        cidx = gaunt.channel_index(lmax)
        lq = [basis.lm_of_q(q)[0] for q in range(self.NQ)]
        # For each q1: the nonzero (q2, q3) pairs of G[q1], their weights and channel.
        self.rows = []
        for q1 in range(self.NQ):
            q2, q3 = np.nonzero(self.G[q1])
            c = np.array([cidx[(lq[q1], lq[a], lq[b])] for a, b in zip(q2, q3)], dtype=np.int64)
            self.rows.append((q2, q3, c, self.G[q1, q2, q3]))

    def slice(self, a1):
        """C[a1, :, :] as a dense N x N matrix in the flat basis a = k*NQ + q."""
        K, NQ = self.K, self.NQ
        k1, q1 = divmod(a1, NQ)
        q2, q3, c, g = self.rows[q1]
        blk = np.zeros((NQ, NQ, K, K))  # [q2, q3, k2, k3]
        blk[q2, q3] = g[:, None, None] * self.R[c, k1]
        return blk.transpose(2, 0, 3, 1).reshape(self.N, self.N)

    def evaluate(self, f):
        """Q[cell, a1] = f[cell] . C[a1] . f[cell] for f of shape [ncells, N]."""
        f = np.asarray(f, dtype=np.float64).reshape(-1, self.N)
        Q = np.empty_like(f)
        for a1 in range(self.N):
            Q[:, a1] = np.einsum("ni,ni->n", f @ self.slice(a1), f)
        return Q

    def evaluate_rows(self, f, a1_list):
        """Q[cell, a1] for a subset of output indices (sampling at large sizes)."""
        f = np.asarray(f, dtype=np.float64).reshape(-1, self.N)
        return np.stack([np.einsum("ni,ni->n", f @ self.slice(a1), f) for a1 in a1_list], axis=1)

    def evaluate_rows_with_terms(self, f, a1_list=None):
        """Q[cell, a1] and T[cell, a1] = sum_{a2, a3} |C_{a1 a2 a3}| |f_a2| |f_a3| (the sum of
        the absolute values of the terms of Q_a1: the scale that bounds the rounding error
        of any summation order, against which cancellation in Q is measured) for the output
        rows `a1_list` (default: all N)."""
        f = np.asarray(f, dtype=np.float64).reshape(-1, self.N)
        fa = np.abs(f)
        rows = range(self.N) if a1_list is None else a1_list
        Q, T = [], []
        for a1 in rows:
            S = self.slice(a1)
            Q.append(np.einsum("ni,ni->n", f @ S, f))
            T.append(np.einsum("ni,ni->n", fa @ np.abs(S), fa))
        return np.stack(Q, axis=1), np.stack(T, axis=1)

    def linearized(self):
        """L[a1, a2] = C[a1, e0, a2] + C[a1, a2, e0] at c_000 = 1 (§5.3.1)."""
        L = np.empty((self.N, self.N))
        for a1 in range(self.N):
            S = self.slice(a1)
            L[a1] = S[0, :] + S[:, 0]
        return L


def evaluate(kmax, lmax, R, f, apply_conservation=True):
    """Convenience: Q(f, f) of the dense operator, with the §4.4 zeroing applied
    to R first unless `apply_conservation` is False."""
    if apply_conservation:
        R = conservation_zeroing(R, lmax)
    return DenseOperator(kmax, lmax, R).evaluate(f)
