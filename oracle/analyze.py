"""Ordering choice + symbolic analysis (oracle).

Section III.A, closing rule: the fill is evaluated before and after an
ordering and the ordering is dropped if it does not improve.  Reading: the
quantity compared is the number of L tiles after the tile-level symbolic
factorization (tiles are what the method stores and computes on); the
permutation is kept only if it gives strictly fewer tiles.
"""
from __future__ import annotations

from . import ordering, tiles

ORDER_NONE, ORDER_RCM, ORDER_AUTO = 0, 1, 2

__all__ = ["analyze", "ORDER_NONE", "ORDER_RCM", "ORDER_AUTO"]


def analyze(m, T, order=ORDER_AUTO):
    """Return dict(perm, nt, tcolptr, trowidx, ordering_used)."""
    n, colptr, rowidx, na = m["n"], m["colptr"], m["rowidx"], m["n_arrow"]
    ident = ordering.identity_perm(n)
    if order == ORDER_NONE:
        cands = [(ORDER_NONE, ident)]
    elif order == ORDER_RCM:
        cands = [(ORDER_RCM, ordering.partial_rcm(n, colptr, rowidx, na))]
    else:
        cands = [(ORDER_NONE, ident), (ORDER_RCM, ordering.partial_rcm(n, colptr, rowidx, na))]
    best = None
    for used, perm in cands:
        nt, tcolptr, trowidx = tiles.plan(n, colptr, rowidx, perm, T)
        if best is None or trowidx.size < best["trowidx"].size:
            best = {"perm": perm, "nt": nt, "tcolptr": tcolptr, "trowidx": trowidx, "ordering_used": used}
    return best
