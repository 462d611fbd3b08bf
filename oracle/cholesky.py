"""Left-looking sparse tile Cholesky, log-determinant and solves (oracle).

Algorithm 1 (Section II), restated in lower storage: the paper factors the
upper part, L = U^T, so its A_km (upper) is our L_mk (lower).  For tile
columns k = 0 .. nt-1:

    A_kk <- A_kk - sum_{n < k, (k,n) in L} L_kn L_kn^T          (SYRK)
    L_kk <- chol(A_kk)                                         (POTRF)
    for m > k with (m,k) in L:
        A_mk <- A_mk - sum_{n < k, (m,n),(k,n) in L} L_mn L_kn^T (GEMM)
        L_mk <- A_mk L_kk^{-T}                                 (TRSM)

Readings of the printed pseudocode: the GEMM loop bound "n < k-1" is read as
n < k (otherwise column k-1 would never update column k); the SYRK loop
takes only n < k; GEMM(A_nk^T, A_mn, A_km) in upper storage is
L_mk -= L_mn L_kn^T in lower storage.  All sums run over ascending n.

POTRF and TRSM are written out as textbook column Cholesky and column
substitution; the only library primitive is the matrix product of the GEMM
and SYRK steps.  Tiles keep their actual (ragged) sizes; nothing is padded.

A non-positive or NaN pivot stops the factorization and reports the global
permuted column (1-based, LAPACK "info" convention).

The log-determinant is 2 sum_i log L_ii (a plain definition; the paper lists
determinants among the standard arrowhead tasks, Section I) and the solve is
x = P^T L^{-T} L^{-1} P b.
"""
from __future__ import annotations

import math

import numpy as np

from . import tiles as _tiles

__all__ = ["scatter_tiles", "potrf_tile", "trsm_tile", "factorize", "logdet", "solve", "NotSPD",
           "factor_residual_tiles", "dense_factor"]


class NotSPD(Exception):
    def __init__(self, info):
        super().__init__(f"matrix is not positive definite (pivot at permuted column {info})")
        self.info = info


def scatter_tiles(m, perm, T, tcolptr, trowidx):
    """P A P^T cut into the tiles of the L map (zero-initialised, actual sizes).

    Section III.B: each element is mapped to its tile; a tile's untouched
    elements are zero.  Returns dict {(I, J): ndarray}.
    """
    n = m["n"]
    nt = tcolptr.size - 1
    dims = _tiles.tile_dims(n, T)
    out = {}
    for k in range(nt):
        for i in trowidx[tcolptr[k]:tcolptr[k + 1]]:
            out[(int(i), k)] = np.zeros((dims[int(i)], dims[k]))
    r, c = _tiles.permuted_lower_entries(n, m["colptr"], m["rowidx"], perm)
    ti, tj = r // T, c // T
    key = ti * nt + tj
    order = np.argsort(key, kind="stable")
    key_s = key[order]
    bounds = np.flatnonzero(np.diff(key_s)) + 1
    starts = np.concatenate([[0], bounds])
    ends = np.concatenate([bounds, [key_s.size]])
    vals = m["values"]
    for s, e in zip(starts, ends):
        idx = order[s:e]
        kk = int(key_s[s])
        t = out[(kk // nt, kk % nt)]
        t[r[idx] % T, c[idx] % T] = vals[idx]
    return out


def potrf_tile(a, col0):
    """Textbook column Cholesky of a symmetric tile (lower triangle is read)."""
    b = a.shape[0]
    l = np.zeros_like(a)
    for j in range(b):
        s = a[j, j] - np.dot(l[j, :j], l[j, :j])
        if not s > 0.0:
            raise NotSPD(col0 + j + 1)
        l[j, j] = math.sqrt(s)
        l[j + 1:, j] = (a[j + 1:, j] - l[j + 1:, :j] @ l[j, :j]) / l[j, j]
    return l


def trsm_tile(a, lkk):
    """X with X lkk^T = a, by substitution over the columns of X."""
    x = np.zeros_like(a)
    for j in range(lkk.shape[0]):
        x[:, j] = (a[:, j] - x[:, :j] @ lkk[j, :j]) / lkk[j, j]
    return x


def factorize(m, perm, T, tcolptr, trowidx):
    """Algorithm 1 on the tile map; returns dict {(I, J): L tile}."""
    nt = tcolptr.size - 1
    L = scatter_tiles(m, perm, T, tcolptr, trowidx)
    rows = _tiles.row_lists(nt, tcolptr, trowidx)
    rowsets = [set(r) for r in rows]
    for k in range(nt):
        akk = L[(k, k)]
        for n in rows[k]:
            if n < k:
                lkn = L[(k, n)]
                akk = akk - lkn @ lkn.T
        L[(k, k)] = potrf_tile(akk, k * T)
        for mm in trowidx[tcolptr[k] + 1:tcolptr[k + 1]]:
            mm = int(mm)
            amk = L[(mm, k)]
            for n in sorted(rowsets[mm] & rowsets[k]):
                if n < k:
                    amk = amk - L[(mm, n)] @ L[(k, n)].T
            L[(mm, k)] = trsm_tile(amk, L[(k, k)])
    return L


def logdet(L, nt):
    """2 sum_i log L_ii, summed exactly-rounded (math.fsum) in ascending i."""
    terms = []
    for k in range(nt):
        terms.extend(math.log(v) for v in np.diag(L[(k, k)]))
    return 2.0 * math.fsum(terms)


def solve(L, perm, T, tcolptr, trowidx, b):
    """x = P^T L^{-T} L^{-1} P b for b of shape (n,) or (n, nrhs)."""
    nt = tcolptr.size - 1
    b = np.asarray(b, dtype=np.float64)
    vec = b.ndim == 1
    bb = b.reshape(b.shape[0], -1)
    n = bb.shape[0]
    dims = _tiles.tile_dims(n, T)
    rows = _tiles.row_lists(nt, tcolptr, trowidx)
    pb = bb[perm, :]
    y = [pb[k * T:k * T + dims[k], :].copy() for k in range(nt)]
    for k in range(nt):  # forward: L y = P b
        for nn in rows[k]:
            if nn < k:
                y[k] = y[k] - L[(k, nn)] @ y[nn]
        lkk = L[(k, k)]
        for j in range(dims[k]):
            y[k][j, :] = (y[k][j, :] - lkk[j, :j] @ y[k][:j, :]) / lkk[j, j]
    x = y
    for k in range(nt - 1, -1, -1):  # backward: L^T x = y
        for mm in trowidx[tcolptr[k] + 1:tcolptr[k + 1]]:
            mm = int(mm)
            x[k] = x[k] - L[(mm, k)].T @ x[mm]
        lkk = L[(k, k)]
        for j in range(dims[k] - 1, -1, -1):
            x[k][j, :] = (x[k][j, :] - lkk[j + 1:, j] @ x[k][j + 1:, :]) / lkk[j, j]
    xp = np.concatenate(x, axis=0)
    out = np.empty_like(xp)
    out[perm, :] = xp
    return out[:, 0] if vec else out


def factor_residual_tiles(L, A, tcolptr, trowidx):
    """||L L^T - P A P^T||_F / ||P A P^T||_F evaluated tile by tile.

    (L L^T)_IJ = sum_n L_In L_Jn^T over the common tile columns n; both
    matrices vanish outside the (symmetric) tile map, so the sum over the
    lower tiles, with off-diagonal tiles counted twice, is exact.
    ``A`` is the dict returned by :func:`scatter_tiles`.
    """
    nt = tcolptr.size - 1
    rows = _tiles.row_lists(nt, tcolptr, trowidx)
    rowsets = [set(r) for r in rows]
    num = 0.0
    den = 0.0
    for k in range(nt):
        for i in trowidx[tcolptr[k]:tcolptr[k + 1]]:
            i = int(i)
            acc = np.zeros_like(A[(i, k)])
            for nn in sorted(rowsets[i] & rowsets[k]):
                acc = acc + L[(i, nn)] @ L[(k, nn)].T
            if i == k:
                e = np.tril(acc - A[(i, k)])
                a = np.tril(A[(i, k)])
                w = 2.0 - np.eye(acc.shape[0])
                num += float(np.sum(w * e * e))
                den += float(np.sum(w * a * a))
            else:
                e = acc - A[(i, k)]
                num += 2.0 * float(np.sum(e * e))
                den += 2.0 * float(np.sum(A[(i, k)] ** 2))
    return math.sqrt(num / den)


def dense_factor(L, n, T, tcolptr, trowidx):
    """Assemble the tiles of L into a dense lower-triangular array (small n)."""
    out = np.zeros((n, n))
    nt = tcolptr.size - 1
    for k in range(nt):
        for i in trowidx[tcolptr[k]:tcolptr[k + 1]]:
            i = int(i)
            t = L[(i, k)]
            out[i * T:i * T + t.shape[0], k * T:k * T + t.shape[1]] = t
    return np.tril(out)
