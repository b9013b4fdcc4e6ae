"""The paper's own factorised evaluation on the CPU, plain numpy (TEST INFRASTRUCTURE and
a timed CPU comparison point; see the package docstring for who may import it).

Angular-first contraction of §4.5.4, written as the paper states it and vectorised over
cells only:

    Phi^{(c,q1)}_{k2 k3} = sum_{z in slice (c, q1)} g_z f_{k2, q2z} f_{k3, q3z}
    Q_{k1, q1}         += sum_{k2, k3} R^{(c)}_{k1 k2 k3} Phi^{(c,q1)}_{k2 k3}

over every non-empty slice (c, q1) of the oracle's own Gaunt COO table (§4.2), with the
§4.4 zeroing applied to R first.  No symmetrisation, no grouping: the same result as the
dense form of dense.py up to summation order, at O(N_G K^2 + N_S K^3) per cell.
"""
import numpy as np

from . import gaunt
from .dense import conservation_zeroing


def slices(lmax, G=None):
    """Non-empty slices (c, q1) -> (q2 array, q3 array, g array), in COO order."""
    q1, q2, q3, c, g = gaunt.coo(lmax, G)
    out = {}
    if q1.size == 0:
        return out
    order = np.lexsort((q1, c))
    c_s, q1_s = c[order], q1[order]
    bounds = np.flatnonzero(np.diff(c_s * (q1.max() + 1) + q1_s)) + 1
    for part in np.split(order, bounds):
        out[(int(c[part[0]]), int(q1[part[0]]))] = (q2[part], q3[part], g[part])
    return out


def evaluate(kmax, lmax, R, f, apply_conservation=True, sl=None):
    """Q(f, f) for f of shape [ncells, K, NQ] by the angular-first contraction."""
    f = np.asarray(f, dtype=np.float64)
    if apply_conservation:
        R = conservation_zeroing(R, lmax)
    if sl is None:
        sl = slices(lmax)
    Q = np.zeros_like(f)
    for (c, q1), (q2, q3, g) in sl.items():
        phi = np.einsum("z,nkz,nlz->nkl", g, f[:, :, q2], f[:, :, q3])  # [cells, k2, k3]
        Q[:, :, q1] += np.einsum("akl,nkl->na", R[c], phi)
    return Q
