"""Pins for the oracle's partial RCM (Section III.A) against hand-derived orderings.

Each expected permutation below was worked out by hand from the stated
reading (George-Liu start vertex, neighbours enqueued by ascending
(degree, index), whole body sequence reversed).
"""
import numpy as np
import pytest

from oracle import ordering
from paper_2501_02483_b300 import inputs


def _graph_matrix(nb, edges, n_arrow=0):
    """Lower CSC with the given body edges, a dominant diagonal and a dense arrow."""
    n = nb + n_arrow
    rows = [max(a, b) for a, b in edges] + list(range(n))
    cols = [min(a, b) for a, b in edges] + list(range(n))
    vals = [-1.0] * len(edges) + [10.0] * n
    for a in range(n_arrow):
        for j in range(nb + a):
            rows.append(nb + a)
            cols.append(j)
            vals.append(0.01)
    colptr, rowidx, values = inputs.coo_to_csc_lower(n, rows, cols, vals)
    return n, colptr, rowidx


def _rcm(nb, edges, n_arrow=0):
    n, colptr, rowidx = _graph_matrix(nb, edges, n_arrow)
    return ordering.partial_rcm(n, colptr, rowidx, n_arrow).tolist()


def test_path_graph_reverses():
    # start 0 (min degree, min index); 0's structure is not beaten by n-1's.
    n = 12
    assert _rcm(n, [(i, i + 1) for i in range(n - 1)]) == list(range(n - 1, -1, -1))


def test_path_graph_with_arrow_keeps_arrow_last():
    n = 9
    assert _rcm(n, [(i, i + 1) for i in range(n - 1)], n_arrow=3) == list(range(n - 1, -1, -1)) + [9, 10, 11]


def test_star_graph():
    # leaves 1..5 around centre 0: start 1; CM 1,0,2,3,4,5; reversed.
    assert _rcm(6, [(0, k) for k in range(1, 6)]) == [5, 4, 3, 2, 0, 1]


def test_grid_3x3():
    # v = 3x + y; CM from corner 0: 0,1,3,2,4,6,5,7,8 (2 before 4: lower degree).
    edges = []
    for x in range(3):
        for y in range(3):
            v = 3 * x + y
            if x + 1 < 3:
                edges.append((v, v + 3))
            if y + 1 < 3:
                edges.append((v, v + 1))
    assert _rcm(9, edges) == [8, 7, 5, 6, 4, 2, 3, 1, 0]


def test_two_components_in_order_of_smallest_vertex():
    # component {0,3,5}: CM 0,3,5; component {1,2,4}: CM 1,2,4.
    assert _rcm(6, [(0, 3), (3, 5), (1, 2), (2, 4)]) == [4, 2, 1, 5, 3, 0]


def test_pseudo_peripheral_search_moves_start():
    # path 1-2-3-4-5 with pendant 0 on 3: min-degree vertex 0 is not
    # peripheral; the search moves to 1 (depth 4 > 3) and stops there.
    assert _rcm(6, [(1, 2), (2, 3), (3, 4), (4, 5), (0, 3)]) == [5, 4, 0, 3, 2, 1]


def test_isolated_vertices():
    # no edges: every vertex is its own component, visited in index order.
    assert _rcm(5, []) == [4, 3, 2, 1, 0]


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_shuffled_path_recovers_bandwidth_one(seed):
    """A randomly relabelled path has an RCM ordering of bandwidth 1."""
    rng = np.random.default_rng(seed)
    n = 200
    lab = rng.permutation(n)
    edges = [(int(lab[i]), int(lab[i + 1])) for i in range(n - 1)]
    perm = np.array(_rcm(n, edges))
    inv = np.empty(n, dtype=int)
    inv[perm] = np.arange(n)
    bw = max(abs(int(inv[a]) - int(inv[b])) for a, b in edges)
    assert bw == 1


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_rcm_is_a_level_ordering(seed):
    """Unreversed, RCM visits each component in non-decreasing BFS level."""
    m = inputs.band_arrow(300, 4, 6, 0.4, seed)
    n, nb = m["n"], m["n"] - m["n_arrow"]
    perm = ordering.partial_rcm(n, m["colptr"], m["rowidx"], m["n_arrow"])
    assert sorted(perm.tolist()) == list(range(n))
    assert perm[nb:].tolist() == list(range(nb, n))
    seq = perm[:nb][::-1]
    indptr, indices = ordering.body_graph(n, m["colptr"], m["rowidx"], m["n_arrow"])
    # split seq into components: a new component starts where the vertex
    # has no neighbour earlier in the sequence
    pos = np.empty(nb, dtype=int)
    pos[seq] = np.arange(nb)
    start = 0
    for i in range(1, nb + 1):
        if i == nb or not np.any(pos[indices[indptr[seq[i]]:indptr[seq[i] + 1]]] < i):
            comp = seq[start:i]
            lv = ordering.level_structure(indptr, indices, int(comp[0]))
            level = {int(v): d for d, vs in enumerate(lv) for v in vs}
            assert sorted(level) == sorted(int(v) for v in comp)
            ls = [level[int(v)] for v in comp]
            assert ls == sorted(ls)
            start = i


def test_rcm_reduces_bandwidth_of_scrambled_band():
    rng = np.random.default_rng(5)
    m = inputs.band_arrow(400, 0, 5, 0.6, 7)
    lab = rng.permutation(400)
    cols = np.repeat(np.arange(400), np.diff(m["colptr"]))
    r, c = lab[m["rowidx"]], lab[cols]
    colptr, rowidx, values = inputs.coo_to_csc_lower(400, np.maximum(r, c), np.minimum(r, c), m["values"])
    perm = ordering.partial_rcm(400, colptr, rowidx, 0)
    inv = np.empty(400, dtype=int)
    inv[perm] = np.arange(400)
    cc = np.repeat(np.arange(400), np.diff(colptr))
    bw_before = int(np.max(np.abs(rowidx - cc)))
    bw_after = int(np.max(np.abs(inv[rowidx] - inv[cc])))
    assert bw_before > 100
    assert bw_after <= 15


def test_adaptable_nd_on_a_path():
    # path 0..9, mid = 5: separator {5} (column 4 reaches row 5); right part 9..6 reversed
    n, colptr, rowidx = _graph_matrix(10, [(i, i + 1) for i in range(9)], n_arrow=2)
    perm = ordering.adaptable_nd(n, colptr, rowidx, 2).tolist()
    assert perm == [0, 1, 2, 3, 4, 9, 8, 7, 6, 5, 10, 11]


def test_adaptable_nd_band_separator_width_and_independence():
    m = inputs.band_arrow(1000, 7, 12, 1.0, 0)  # full band of half-width 12
    perm = ordering.adaptable_nd(m["n"], m["colptr"], m["rowidx"], 7)
    assert sorted(perm.tolist()) == list(range(m["n"]))
    # separator = rows 500..511 (12 rows), just before the arrow
    assert perm[1000 - 12:1000].tolist() == list(range(500, 512))
    # no stored entry joins the two parts
    inv = np.empty(m["n"], dtype=int)
    inv[perm] = np.arange(m["n"])
    cols = np.repeat(np.arange(m["n"]), np.diff(m["colptr"]))
    r, c = inv[m["rowidx"]], inv[cols]
    body = (r < 1000 - 12) & (c < 1000 - 12)
    part = lambda x: x >= 500
    assert not np.any(body & (part(r) != part(c)))


def test_adaptable_nd_no_crossing_entries():
    # two disconnected blocks: nothing crosses mid, separator empty
    n, colptr, rowidx = _graph_matrix(8, [(0, 1), (1, 2), (2, 3), (4, 5), (5, 6), (6, 7)])
    assert ordering.adaptable_nd(n, colptr, rowidx, 0).tolist() == [0, 1, 2, 3, 7, 6, 5, 4]


def test_adaptable_nd_split_is_tile_aligned():
    # path 0..9 with tiles of 4: mid = 5 rounds down to 4, separator {4}
    n, colptr, rowidx = _graph_matrix(10, [(i, i + 1) for i in range(9)], n_arrow=2)
    assert ordering.adaptable_nd(n, colptr, rowidx, 2, align=4).tolist() == [0, 1, 2, 3, 9, 8, 7, 6, 5, 4, 10, 11]
    # a tile wider than half the body leaves the order unchanged
    assert ordering.adaptable_nd(n, colptr, rowidx, 2, align=8).tolist() == list(range(12))


def _tile_etree_leaves(m, perm, T):
    from oracle import tiles
    nt, present = tiles.tile_map(m["n"], m["colptr"], m["rowidx"], perm, T)
    tcp, tri = tiles.tile_csc(nt, tiles.symbolic_closure(nt, present))
    parent = [int(tri[tcp[k] + 1]) if tcp[k + 1] - tcp[k] > 1 else -1 for k in range(nt)]
    has_child = set(p for p in parent if p >= 0)
    return [k for k in range(nt) if k not in has_child]


def test_adaptable_nd_gives_two_tile_chains_only_when_aligned():
    # body of 1001 rows (mid = 500, not a multiple of 16): aligned at 16 the
    # tile elimination tree has two leaves (two independent chains); the
    # unaligned split puts rows of both parts into one tile and leaves one chain
    m = inputs.band_arrow(1001, 5, 20, 1.0, 1)
    T = 16
    aligned = ordering.adaptable_nd(m["n"], m["colptr"], m["rowidx"], 5, align=T)
    unaligned = ordering.adaptable_nd(m["n"], m["colptr"], m["rowidx"], 5, align=1)
    assert len(_tile_etree_leaves(m, aligned, T)) == 2
    assert len(_tile_etree_leaves(m, unaligned, T)) == 1
