"""Partial Reverse Cuthill-McKee ordering of the arrowhead body (oracle).

Section III.A: RCM is applied to the body only, leaving the dense arrow rows
and columns in place at the end ("partial permutation"), and a permutation is
kept only if it reduces fill.

The paper does not fix RCM's tie-breaks, so this module uses the following
reading (the library implements the same reading independently):

* the graph is the off-diagonal pattern of the body block A[0:nb, 0:nb]
  (nb = n - n_arrow), made symmetric; arrow couplings are ignored;
* deg(v) = number of distinct body neighbours of v;
* connected components are handled in the order of their smallest vertex;
* the start vertex of a component is found by the George-Liu
  pseudo-peripheral search: start at the component's min-(degree, index)
  vertex r; build its BFS level structure; take x = the min-(degree, index)
  vertex of the last level; if x's level structure is strictly deeper,
  r <- x and repeat, otherwise stop with r;
* Cuthill-McKee: breadth-first from the start vertex, each dequeued vertex
  enqueueing its unvisited neighbours in ascending (degree, index) order;
* the component sequences are concatenated and the whole body sequence is
  reversed.

The result is ``perm`` with ``perm[new] = old``; arrow vertices map to
themselves.
"""
from __future__ import annotations

import numpy as np

__all__ = ["body_graph", "level_structure", "pseudo_peripheral", "cuthill_mckee", "partial_rcm",
           "identity_perm", "adaptable_nd"]


def identity_perm(n):
    return np.arange(n, dtype=np.int64)


def body_graph(n, colptr, rowidx, n_arrow):
    """Symmetric adjacency (CSR: indptr, indices sorted) of the body block."""
    nb = n - n_arrow
    cols = np.repeat(np.arange(n, dtype=np.int64), np.diff(colptr))
    rows = rowidx.astype(np.int64)
    keep = (rows != cols) & (rows < nb) & (cols < nb)
    r, c = rows[keep], cols[keep]
    src = np.concatenate([r, c])
    dst = np.concatenate([c, r])
    key = np.unique(src * max(nb, 1) + dst)  # removes duplicate edges
    src, dst = key // max(nb, 1), key % max(nb, 1)
    indptr = np.zeros(nb + 1, dtype=np.int64)
    np.cumsum(np.bincount(src, minlength=nb), out=indptr[1:])
    return indptr, dst.astype(np.int64)


def level_structure(indptr, indices, root):
    """Breadth-first levels from ``root``: list of arrays of vertices."""
    nb = indptr.size - 1
    seen = np.zeros(nb, dtype=bool)
    seen[root] = True
    levels = [np.array([root], dtype=np.int64)]
    while True:
        f = levels[-1]
        starts, ends = indptr[f], indptr[f + 1]
        lens = ends - starts
        if lens.sum() == 0:
            break
        offs = np.repeat(starts - np.concatenate([[0], np.cumsum(lens)[:-1]]), lens)
        nbrs = indices[np.arange(lens.sum()) + offs]
        nxt = np.unique(nbrs[~seen[nbrs]])
        if nxt.size == 0:
            break
        seen[nxt] = True
        levels.append(nxt)
    return levels


def _min_deg_index(vertices, deg):
    vertices = np.asarray(vertices)
    order = np.lexsort((vertices, deg[vertices]))  # by degree, then index
    return int(vertices[order[0]])


def pseudo_peripheral(indptr, indices, deg, component):
    """George-Liu pseudo-peripheral start vertex of one component."""
    r = _min_deg_index(component, deg)
    lv = level_structure(indptr, indices, r)
    while True:
        x = _min_deg_index(lv[-1], deg)
        lx = level_structure(indptr, indices, x)
        if len(lx) > len(lv):
            r, lv = x, lx
        else:
            return r


def cuthill_mckee(indptr, indices, deg, start, visited):
    """Cuthill-McKee sequence of the component of ``start`` (marks ``visited``)."""
    queue = [start]
    visited[start] = True
    head = 0
    while head < len(queue):
        v = queue[head]
        head += 1
        nb = indices[indptr[v]:indptr[v + 1]]
        nb = nb[~visited[nb]]
        if nb.size:
            nb = nb[np.lexsort((nb, deg[nb]))]
            visited[nb] = True
            queue.extend(int(u) for u in nb)
    return queue


def partial_rcm(n, colptr, rowidx, n_arrow):
    """Partial RCM permutation (perm[new] = old), arrow kept last."""
    nb = n - n_arrow
    indptr, indices = body_graph(n, colptr, rowidx, n_arrow)
    deg = np.diff(indptr)
    visited = np.zeros(nb, dtype=bool)
    seq = []
    for v in range(nb):
        if visited[v]:
            continue
        comp = np.concatenate(level_structure(indptr, indices, v))
        start = pseudo_peripheral(indptr, indices, deg, comp)
        seq.extend(cuthill_mckee(indptr, indices, deg, start, visited))
    body = np.array(seq[::-1], dtype=np.int64)
    return np.concatenate([body, np.arange(nb, n, dtype=np.int64)])


def adaptable_nd(n, colptr, rowidx, n_arrow, align=1):
    """One level of the adaptable nested dissection of Section III.A.

    The paper's recipe: take a separator as wide as the bandwidth and move it
    towards the end of the matrix, ahead of the arrow.  Reading used here:

    * the body [0, nb) is split at mid = (nb // 2) rounded down to a multiple
      of ``align`` (the tile size: a tile holding rows of both parts would join
      the two elimination chains again at the tile level); mid = 0 leaves the
      order unchanged;
    * the separator S = [mid, s_end) holds every row that some body column
      left of mid reaches: s_end = 1 + max{i : (i, j) stored, j < mid <= i < nb}
      (S is empty when nothing crosses mid);
    * new order: [0, mid), then [s_end, nb) reversed, then S, then the arrow.

    Reversing the second part makes both parts touch the separator with their
    last rows, so eliminating either part adds no fill between the separator
    and the part's interior, and the two parts are independent chains.
    """
    nb = n - n_arrow
    mid = (nb // 2) // align * align
    if nb < 2 or mid == 0:
        return identity_perm(n)
    cols = np.repeat(np.arange(n, dtype=np.int64), np.diff(colptr))
    rows = rowidx.astype(np.int64)
    cross = (cols < mid) & (rows >= mid) & (rows < nb)
    s_end = int(rows[cross].max()) + 1 if np.any(cross) else mid
    left = np.arange(0, mid, dtype=np.int64)
    right = np.arange(nb - 1, s_end - 1, -1, dtype=np.int64)
    sep = np.arange(mid, s_end, dtype=np.int64)
    return np.concatenate([left, right, sep, np.arange(nb, n, dtype=np.int64)])
