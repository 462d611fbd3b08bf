"""Ordering choice + symbolic analysis (oracle).

Section III.A, closing rule: the fill is evaluated before and after an
ordering and the ordering is dropped if it does not improve.  Reading: the
quantity compared is the number of L tiles after the tile-level symbolic
factorization (tiles are what the method stores and computes on); the
permutation is kept only if it gives strictly fewer tiles.  The adaptable
nested dissection is an explicit choice (it trades a little fill for two
independent elimination chains) and is not part of the automatic rule.
"""
from __future__ import annotations

from . import ordering, tiles

ORDER_NONE, ORDER_RCM, ORDER_AUTO, ORDER_ND = 0, 1, 2, 3

__all__ = ["analyze", "ORDER_NONE", "ORDER_RCM", "ORDER_AUTO", "ORDER_ND"]


def analyze(m, T, order=ORDER_AUTO):
    """Return dict(perm, nt, tcolptr, trowidx, ordering_used)."""
    n, colptr, rowidx, na = m["n"], m["colptr"], m["rowidx"], m["n_arrow"]
    ident = ordering.identity_perm(n)
    if order == ORDER_NONE:
        cands = [(ORDER_NONE, ident)]
    elif order == ORDER_RCM:
        cands = [(ORDER_RCM, ordering.partial_rcm(n, colptr, rowidx, na))]
    elif order == ORDER_ND:
        # chosen for parallelism, not fill (Section III.A: "when enough cores are available")
        cands = [(ORDER_ND, ordering.adaptable_nd(n, colptr, rowidx, na, align=T))]
    else:
        cands = [(ORDER_NONE, ident), (ORDER_RCM, ordering.partial_rcm(n, colptr, rowidx, na))]
    best = None
    for used, perm in cands:
        nt, tcolptr, trowidx = tiles.plan(n, colptr, rowidx, perm, T)
        if best is None or trowidx.size < best["trowidx"].size:
            best = {"perm": perm, "nt": nt, "tcolptr": tcolptr, "trowidx": trowidx, "ordering_used": used}
    return best
