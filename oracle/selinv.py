"""Selected inverse and marginal variances (oracle; test infrastructure).

The paper lists inverses among the standard tasks on arrowhead precision
matrices (Section I; INLA needs the marginal variances diag(A^{-1})).  This
module computes Sigma = (P A P^T)^{-1} on the filled tile map of L only --
the selected inverse -- from the identity Sigma L = L^{-T}:

  column block k of Sigma L = L^{-T} reads, for m >= k,
      Sigma_mk L_kk + sum_{j in S_k} Sigma_mj L_jk = [m == k] L_kk^{-T},
  with S_k = {j > k : (j, k) in L}.  Hence, for k = nt-1 down to 0,
      Sigma_mk = - sum_{j in S_k} Sigma_mj (L_jk L_kk^{-1})       (m in S_k),
      Sigma_kk = L_kk^{-T} L_kk^{-1} - sum_{j in S_k} Sigma_jk^T (L_jk L_kk^{-1}),
  where Sigma_mj with m, j in S_k lies on the filled map (the tile symbolic
  closure makes S_k a clique), read as Sigma_jm^T when m < j.

Matrix products and the triangular inverse are library primitives; the
recursion is the plain statement above, column by column.  The marginal
variances are diag(Sigma) returned to the original order (P^T).
"""
from __future__ import annotations

import numpy as np

from . import tiles as _tiles

__all__ = ["selected_inverse", "marginal_variances"]


def _tri_inv(lkk):
    """L_kk^{-1} of a lower-triangular tile (column substitution)."""
    b = lkk.shape[0]
    x = np.zeros_like(lkk)
    for c in range(b):
        e = np.zeros(b)
        e[c] = 1.0
        for i in range(b):
            x[i, c] = (e[i] - lkk[i, :i] @ x[:i, c]) / lkk[i, i]
    return x


def selected_inverse(L, tcolptr, trowidx):
    """Sigma on the tiles of L (dict {(I, J): tile}, I >= J)."""
    nt = tcolptr.size - 1
    S = {}

    def sig(m, j):
        return S[(m, j)] if m >= j else S[(j, m)].T

    for k in range(nt - 1, -1, -1):
        below = [int(i) for i in trowidx[tcolptr[k] + 1:tcolptr[k + 1]]]
        linv = _tri_inv(L[(k, k)])
        U = {j: L[(j, k)] @ linv for j in below}
        for m in below:
            acc = np.zeros((L[(m, k)].shape[0], L[(k, k)].shape[0]))
            for j in below:
                acc = acc + sig(m, j) @ U[j]
            S[(m, k)] = -acc
        d = linv.T @ linv
        for j in below:
            d = d - S[(j, k)].T @ U[j]
        S[(k, k)] = d
    return S


def marginal_variances(S, perm, n, T):
    """diag(A^{-1}) in the original order from the selected inverse."""
    nt = len({k for (i, k) in S if i == k})
    dims = _tiles.tile_dims(n, T)
    vp = np.concatenate([np.diag(S[(k, k)])[:dims[k]] for k in range(nt)])
    out = np.empty(n)
    out[perm] = vp
    return out
