"""Tile map, tile-level symbolic factorization and flop count (oracle).

Section III.B (Compressed Tile Storage Format): the permuted matrix is cut
into fixed T x T tiles starting at index 0, independent of where the arrow
begins; a tile exists only if some stored element maps into it.  Diagonal
tiles always exist (every diagonal element is stored).  Only the lower
triangle is kept (the paper works on the upper part, which is its transpose).

Section II, step 2 (symbolic factorization) with Algorithm 1: the GEMM that
updates tile (m, k) from tiles (m, n) and (k, n) creates tile (m, k) if it
did not exist.  Reading: the symbolic factorization is the tile-level
elimination closure, taken in ascending column order:

    for k = 0 .. nt-1:  S_k = {m > k : tile (m, k) exists}
                         every pair m > j of S_k creates tile (m, j).

``neighbors(k)`` of Section II (m is a neighbour of k if tile (m, k) or
(k, m) is nonzero) is taken on this closed map.
"""
from __future__ import annotations

import numpy as np

__all__ = ["permuted_lower_entries", "tile_map", "symbolic_closure", "tile_csc", "row_lists",
           "neighbors", "task_flops", "tile_dims", "plan"]


def permuted_lower_entries(n, colptr, rowidx, perm):
    """(row, col) of every stored entry of P A P^T, flipped into the lower triangle."""
    inv = np.empty(n, dtype=np.int64)
    inv[perm] = np.arange(n, dtype=np.int64)
    cols = np.repeat(np.arange(n, dtype=np.int64), np.diff(colptr))
    r = inv[rowidx.astype(np.int64)]
    c = inv[cols]
    return np.maximum(r, c), np.minimum(r, c)


def tile_map(n, colptr, rowidx, perm, T):
    """Set of present tiles (I, J), I >= J, before symbolic fill."""
    nt = (n + T - 1) // T
    r, c = permuted_lower_entries(n, colptr, rowidx, perm)
    keys = np.unique((r // T) * nt + (c // T))
    present = {(int(k // nt), int(k % nt)) for k in keys}
    present.update((k, k) for k in range(nt))
    return nt, present


def symbolic_closure(nt, present):
    """Tile-level elimination closure; returns the list of row sets per column."""
    cols = [set() for _ in range(nt)]
    for (i, j) in present:
        if i > j:
            cols[j].add(i)
    for k in range(nt):
        s = sorted(cols[k])
        for a in range(len(s)):
            for b in range(a):
                cols[s[b]].add(s[a])  # tile (s[a], s[b]) with s[a] > s[b]
    return cols


def tile_csc(nt, cols):
    """Tile-CSC arrays of L: colptr[nt+1], rows (diagonal first, ascending)."""
    tcolptr = np.zeros(nt + 1, dtype=np.int64)
    rows = []
    for k in range(nt):
        rk = [k] + sorted(cols[k])
        rows.extend(rk)
        tcolptr[k + 1] = tcolptr[k] + len(rk)
    return tcolptr, np.array(rows, dtype=np.int32)


def row_lists(nt, tcolptr, trowidx):
    """For every tile row m, the ascending list of tile columns J with (m, J) in L."""
    rows = [[] for _ in range(nt)]
    for k in range(nt):
        for m in trowidx[tcolptr[k]:tcolptr[k + 1]]:
            rows[int(m)].append(k)
    return rows


def neighbors(nt, tcolptr, trowidx):
    """neighbors(k) of Section II on the filled map (both directions, k excluded)."""
    nb = [set() for _ in range(nt)]
    for k in range(nt):
        for m in trowidx[tcolptr[k]:tcolptr[k + 1]]:
            m = int(m)
            if m != k:
                nb[k].add(m)
                nb[m].add(k)
    return nb


def tile_dims(n, T):
    nt = (n + T - 1) // T
    return [min(T, n - I * T) for I in range(nt)]


def task_flops(n, T, tcolptr, trowidx):
    """Exact flop count of the tile tasks of Algorithm 1 on this map.

    POTRF of a b x b tile: b(b+1)(2b+1)/6 (= b^3/3 + b^2/2 + b/6);
    SYRK of a b x b tile with inner width w: w b (b+1);
    GEMM of an r x c output with inner width w: 2 r c w;
    TRSM of an r x b tile: r b^2.
    Tile sizes are the actual (ragged) dimensions.  Returns a dict of
    Python ints.
    """
    nt = tcolptr.size - 1
    dims = tile_dims(n, T)
    rows = row_lists(nt, tcolptr, trowidx)
    rowsets = [set(r) for r in rows]
    f = {"potrf": 0, "syrk": 0, "gemm": 0, "trsm": 0}
    for k in range(nt):
        b = dims[k]
        f["potrf"] += b * (b + 1) * (2 * b + 1) // 6
        for nn in rows[k]:
            if nn < k:
                f["syrk"] += dims[nn] * b * (b + 1)
        for m in trowidx[tcolptr[k] + 1:tcolptr[k + 1]]:
            m = int(m)
            f["trsm"] += dims[m] * b * b
            for nn in rowsets[m] & rowsets[k]:
                if nn < k:
                    f["gemm"] += 2 * dims[m] * b * dims[nn]
    f["total"] = f["potrf"] + f["syrk"] + f["gemm"] + f["trsm"]
    return f


def plan(n, colptr, rowidx, perm, T):
    """Tile map + closure for a given permutation: (nt, tcolptr, trowidx)."""
    nt, present = tile_map(n, colptr, rowidx, perm, T)
    cols = symbolic_closure(nt, present)
    tcolptr, trowidx = tile_csc(nt, cols)
    return nt, tcolptr, trowidx
