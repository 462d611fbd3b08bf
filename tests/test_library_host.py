"""Host-side checks of libstiles.so (no GPU needed).

* the shared library loads and exports every function declared in
  include/stiles.h;
* stiles_analyze agrees bit-for-bit with the oracle's independent analysis:
  permutation, tile map and per-kernel flop counts;
* malformed input is rejected with STILES_ERR_INVALID.
"""
import os
import re

import numpy as np
import pytest

from oracle import analyze as oan
from oracle import ordering as oord
from oracle import tiles as otiles
from paper_2501_02483_b300 import build, inputs
from tests.golden import make_golden as golden
from paper_2501_02483_b300 import stiles as st

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build_library()
    st.lib()


def test_exports_every_declared_symbol():
    hdr = open(os.path.join(ROOT, "include", "stiles.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    names = sorted(set(re.findall(r"\b(stiles_[a-z0-9_]+)\s*\(", hdr)))
    assert len(names) >= 15
    L = st.lib()
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def _oracle_plan(m, T, order):
    p = oan.analyze(m, T, order)
    f = otiles.task_flops(m["n"], T, p["tcolptr"], p["trowidx"])
    return p, f


def _compare(m, T, order, **kw):
    p, f = _oracle_plan(m, T, order)
    plan = st.Plan.from_matrix(m, tile=T, ordering=order, **kw)
    info = plan.info()
    assert np.array_equal(plan.perm(), p["perm"])
    tc, tr = plan.tilemap()
    assert np.array_equal(tc, p["tcolptr"])
    assert np.array_equal(tr, p["trowidx"])
    assert info["ordering_used"] == p["ordering_used"]
    for k in ("potrf", "syrk", "gemm", "trsm", "total"):
        assert info["flops_" + k] == f[k], k
    plan.close()


CASES = [
    ("band", lambda s: inputs.band_arrow(300, 5, 12, 0.3, s)),
    ("wide", lambda s: inputs.band_arrow(500, 20, 60, 0.1, s)),
    ("noarrow", lambda s: inputs.band_arrow(257, 0, 9, 0.5, s)),
    ("diag", lambda s: inputs.diagonal_matrix(np.arange(1.0, 101.0), n_arrow=3)),
    ("kron", lambda s: inputs.kronecker_spatiotemporal(6, 0.8, 5, 1.0, 4, 0.1, s, nrhs=0)),
    ("arrowhead", lambda s: inputs.pure_arrowhead(200, 7, seed=s)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("T", [1, 3, 16, 32, 64, 100])
@pytest.mark.parametrize("order", [oan.ORDER_NONE, oan.ORDER_RCM, oan.ORDER_AUTO, oan.ORDER_ND])
def test_analyze_matches_oracle(name, make, T, order):
    _compare(make(T + 7 * order), T, order)


def _scrambled(n, hw, w, seed):
    rng = np.random.default_rng(seed)
    m = inputs.band_arrow(n, w, hw, 0.4, seed)
    lab = np.concatenate([rng.permutation(n), np.arange(n, n + w)])
    cols = np.repeat(np.arange(n + w), np.diff(m["colptr"]))
    r, c = lab[m["rowidx"]], lab[cols]
    colptr, rowidx, values = inputs.coo_to_csc_lower(n + w, np.maximum(r, c), np.minimum(r, c), m["values"])
    return {"n": n + w, "n_arrow": w, "colptr": colptr, "rowidx": rowidx, "values": values}


@pytest.mark.parametrize("seed", range(25))
def test_analyze_matches_oracle_random_scrambled(seed):
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(20, 400))
    hw = int(rng.integers(1, 20))
    w = int(rng.integers(0, 8))
    T = int(rng.choice([1, 2, 5, 8, 16, 32, 48]))
    order = int(rng.integers(0, 4))
    _compare(_scrambled(n, hw, w, seed), T, order)


def test_analyze_matches_oracle_medium_rcm():
    m = _scrambled(20_000, 40, 30, 77)
    _compare(m, 32, oan.ORDER_AUTO)


def test_analyze_large_config_identity_matches_oracle():
    m = inputs.config_large(0)
    nt, tc, tr = otiles.plan(m["n"], m["colptr"], m["rowidx"], np.arange(m["n"]), 32)
    plan = st.Plan.from_matrix(m, tile=32, ordering=st.ORDER_NONE)
    tc2, tr2 = plan.tilemap()
    assert np.array_equal(tc, tc2) and np.array_equal(tr, tr2)
    # the oracle's count at T = 32, written by tests/golden/make_golden.py
    assert plan.info()["flops_total"] == golden.load()["flops_total"]


def test_rcm_library_equals_oracle_on_hand_cases():
    # 3x3 grid: the hand-derived order of the oracle pins
    edges = []
    for x in range(3):
        for y in range(3):
            v = 3 * x + y
            if x + 1 < 3:
                edges.append((v, v + 3))
            if y + 1 < 3:
                edges.append((v, v + 1))
    rows = [max(a, b) for a, b in edges] + list(range(9))
    cols = [min(a, b) for a, b in edges] + list(range(9))
    colptr, rowidx, _ = inputs.coo_to_csc_lower(9, rows, cols, np.ones(len(rows)))
    plan = st.Plan(9, colptr, rowidx, 0, tile=2, ordering=st.ORDER_RCM)
    assert plan.perm().tolist() == [8, 7, 5, 6, 4, 2, 3, 1, 0]
    assert plan.perm().tolist() == oord.partial_rcm(9, colptr, rowidx, 0).tolist()


def _bad(colptr, rowidx, n, n_arrow=0, tile=32):
    with pytest.raises(st.StilesError) as e:
        st.Plan(n, np.array(colptr), np.array(rowidx), n_arrow, tile=tile)
    assert e.value.name == "INVALID"


def test_invalid_inputs_are_rejected():
    _bad([0, 1, 2], [0, 0], 2)          # column 1 lacks its diagonal (has row 0 < 1)
    _bad([0, 2, 3], [1, 0, 1], 2)       # column 0 starts with row 1 (diagonal missing)
    _bad([0, 3, 4, 5], [0, 2, 1, 1, 2], 3)  # rows of column 0 not ascending
    _bad([0, 2, 3], [0, 1, 1], 2, n_arrow=3)
    _bad([0, 2, 3], [0, 1, 1], 2, tile=0)
    _bad([0, 2, 3], [0, 5, 1], 2)       # row out of range


def test_plan_info_fields_are_consistent():
    m = inputs.config_small(0)
    plan = st.Plan.from_matrix(m, tile=64)
    info = plan.info()
    assert info["n"] == 2010 and info["nt"] == 32 and info["nnzt"] == 93
    assert info["block"] == 32 and info["nsub"] == 93 * 4
    assert info["factor_bytes"] == 93 * 64 * 64 * 8
    assert info["flops_total"] == 29714265


def test_analyze_large_config_nd_matches_oracle():
    m = inputs.config_large(0)
    p = oan.analyze(m, 16, oan.ORDER_ND)
    plan = st.Plan.from_matrix(m, tile=16, ordering=st.ORDER_ND)
    assert np.array_equal(plan.perm(), p["perm"])
    tc, tr = plan.tilemap()
    assert np.array_equal(tc, p["tcolptr"]) and np.array_equal(tr, p["trowidx"])


def test_task_order_is_topological_and_interleaves_nd_parts():
    """Tickets follow elimination-tree levels: with the adaptable ND the two
    halves' diagonal tasks alternate instead of running one after the other."""
    m = inputs.band_arrow(4000, 10, 20, 0.5, 2)
    plan = st.Plan.from_matrix(m, tile=16, ordering=st.ORDER_ND)
    tasks = plan.tasks(0)
    diag_cols = np.where(tasks[:, 0] == 4, tasks[:, 9], tasks[:, 3])[(tasks[:, 0] == 0) | (tasks[:, 0] == 4)]
    half = 2000 // 16
    first = diag_cols[:40]
    assert np.any(first < half) and np.any((first >= half) & (first < 2 * half))


def _selinv_graph_case(T, B, order):
    m = inputs.band_arrow(1000, 24, 40, 0.3, 5)  # n = 1024: no padding at T, B in {16, 32}
    plan = st.Plan.from_matrix(m, tile=T, block=B, ordering=order)
    return m, plan


@pytest.mark.parametrize("T,B,order", [(16, 16, st.ORDER_ND), (32, 16, st.ORDER_ND), (32, 32, st.ORDER_RCM),
                                       (16, 16, st.ORDER_NONE), (64, 16, st.ORDER_ND)])
def test_selected_inverse_graph_executes_to_the_dense_inverse(T, B, order):
    """Runs the selected inverse's host-built task graph in ticket order with
    numpy, with the semantics the persistent kernel implements:
      off-diagonal task (m, k): Sigma_mk = -(sum of its products S U + sum of its
        loaded X terms), then W(m, k) = Sigma_mk^T U_mk and X(m, c) = Sigma_mk^T U_mc
        for its X products;
      diagonal task k: Sigma_kk = L_kk^{-T} L_kk^{-1} - sum of its loaded W terms;
    and checks every Sigma sub-tile against the dense inverse of P A P^T.  Each
    operand's and each loaded term's guarding flag must belong to an earlier
    ticket, each term must be formed before it is loaded, and every sub-tile is
    produced once."""
    m, plan = _selinv_graph_case(T, B, order)
    n = m["n"]
    A = inputs.dense_from_csc(m)
    perm = plan.perm()
    Ap = A[np.ix_(perm, perm)]
    Lf = np.linalg.cholesky(Ap)
    Sig = np.linalg.inv(Ap)
    tc, tr = plan.tilemap()
    R = T // B
    nsb = n // B
    # sub-tile index -> (sub-row, sub-column), as the library numbers them
    where = {}
    for J in range(len(tc) - 1):
        for e in range(tc[J], tc[J + 1]):
            I = tr[e]
            for q in range(R):
                for p in range(R):
                    ii, jj = I * R + p, J * R + q
                    if ii >= jj and ii < nsb and jj < nsb:
                        where[e * R * R + q * R + p] = (ii, jj)
    blk = lambda M, ii, jj: M[ii * B:(ii + 1) * B, jj * B:(jj + 1) * B]
    tasks, pairs, loads, posts = plan.tasks(3), plan.tasks(4), plan.tasks(5), plan.tasks(6)[:, 0]
    outs = tasks[:, 0]
    assert len(np.unique(outs)) == len(outs) == len(where)
    mask = (1 << 30) - 1
    linv = {k: np.linalg.inv(blk(Lf, k, k)) for k in range(nsb)}
    U = lambda s: blk(Lf, *where[s]) @ linv[where[s][1]]
    # executing in ticket order, every operand must already be final and every
    # loaded term's flag must already hold its wanted value
    S, W, X = {}, {}, {}

    def loaded(lb, le):
        acc = np.zeros((B, B))
        for f, want, x in loads[lb:le]:
            f, want, x = int(f), int(want), int(x)
            assert f in S and want == 1
            acc += (W if (x >> 30) & 1 else X)[x & mask]
        return acc

    def products(pb, pe):
        acc = np.zeros((B, B))
        for sg, su in pairs[pb:pe]:
            s = S[int(sg) & mask]
            acc += (s.T if (int(sg) >> 30) & 1 else s) @ U(int(su))
        return acc

    for t, (out, kind, pb, pe, lb, le, xb, xe) in enumerate(tasks):
        out = int(out)
        ii, k = where[out]
        for sg, su in pairs[pb:pe]:
            assert where[int(su)][1] == k
        if kind >= 0:
            assert kind == k == ii and pe == pb and xe == xb
            v = linv[k].T @ linv[k] - loaded(lb, le)
        else:
            assert kind == -1
            v = -(loaded(lb, le) + products(pb, pe))
            W[out] = v.T @ U(out)
            for x in posts[xb:xe]:
                assert where[int(x)][0] == ii
                X[int(x)] = v.T @ U(int(x))
        S[out] = v
        assert np.allclose(v, blk(Sig, ii, k), rtol=1e-9, atol=1e-12 * np.abs(Sig).max())
    assert len(S) == len(where)


def test_selected_inverse_graph_interleaves_nd_halves():
    """Columns are ordered by elimination-tree depth, so the two nested-dissection
    halves' diagonal tasks alternate rather than one half waiting for the other."""
    m = inputs.band_arrow(4000, 10, 20, 0.5, 2)
    plan = st.Plan.from_matrix(m, tile=16, ordering=st.ORDER_ND)
    tasks = plan.tasks(3)
    cols = tasks[tasks[:, 1] >= 0, 1]
    assert len(cols) == -(-m["n"] // 16) and len(np.unique(cols)) == len(cols)
    half = 2000 // 16
    body = cols[cols < 4000 // 16]
    first = body[:40]
    assert np.any(first < half) and np.any((first >= half) & (first < 2 * half))


@pytest.mark.parametrize("T,order", [(16, st.ORDER_ND), (32, st.ORDER_RCM), (64, st.ORDER_AUTO)])
def test_fused_graph_adds_one_forward_task_per_block(T, order):
    """The factorization with the forward sweep folded in (host-built, checked for
    ticket order when built): the factor's tasks in their order, plus the forward
    solve graph's tasks, a forward block k being an OFF task with output nsub + k
    placed after the task that finishes L_kk."""
    m = inputs.band_arrow(3000, 24, 40, 0.4, 11, nrhs=2)
    plan = st.Plan.from_matrix(m, tile=T, ordering=order)
    inf = plan.info()
    nsub, nsb = inf["nsub"], -(-m["n"] // inf["block"])
    fac, fwd, fus = plan.tasks(0), plan.tasks(1), plan.tasks(7)
    assert len(fus) == len(fac) + len(fwd)
    is_fwd = (fus[:, 1] >= nsub) & (fus[:, 0] == 1)
    assert sorted(fus[is_fwd, 1] - nsub) == list(range(nsb))
    # factor tasks keep their relative order
    fac_rows = [tuple(r) for r in fac]
    kept = [tuple(r) for r, f in zip(fus, is_fwd) if not f and not (r[0] in (2, 3) and r[1] >= inf["nscratch"])]
    assert kept == fac_rows
    # each forward block follows the task that produces its diagonal sub-tile
    pos = {}
    for t, r in enumerate(fus):
        if r[0] in (0, 1, 4) and r[1] < nsub:
            pos[int(r[1])] = t
            if r[0] == 4:
                pos[int(r[8])] = t
    for t in np.where(is_fwd)[0]:
        assert pos[int(fus[t, 2])] < t


@pytest.mark.parametrize("n_body,n_arrow", [(7, 3), (0, 20), (300, 0)])
def test_fused_graph_small_and_degenerate(n_body, n_arrow):
    """One padded block, an arrow alone, a band alone: the merged graph still
    holds every factor task and one forward OFF task per block."""
    if n_body == 0:
        m = inputs.diagonal_matrix(np.arange(1.0, n_arrow + 1.0), n_arrow=n_arrow)
    else:
        m = inputs.band_arrow(n_body, n_arrow, 3, 0.5, 2)
    plan = st.Plan.from_matrix(m, tile=16)
    inf = plan.info()
    nsub, nsb = inf["nsub"], -(-m["n"] // inf["block"])
    fac, fwd, fus = plan.tasks(0), plan.tasks(1), plan.tasks(7)
    assert len(fus) == len(fac) + len(fwd)
    is_fwd = (fus[:, 1] >= nsub) & (fus[:, 0] == 1)
    assert sorted(fus[is_fwd, 1] - nsub) == list(range(nsb))


@pytest.mark.parametrize("order", [st.ORDER_NONE, st.ORDER_ND])
@pytest.mark.parametrize("which", [1, 2])
def test_sweep_tasks_split_into_leaves_keep_their_newest_inputs(which, order):
    """A sweep task with more inputs than a tree chunk (32 by default) sends only
    its older inputs to tree leaves and keeps at least its 8 newest itself; the
    leaves and the task's own list together name each input once.  "Newest" is
    by producer: every input a task keeps comes from a block task at or after
    the latest producer of any input in its leaves (also under nested
    dissection, where block index order is not producer order)."""
    m = inputs.band_arrow(6000, 100, 500, 0.2, 3)  # up to 31 band blocks + 7 arrow blocks per column at B = 16
    plan = st.Plan.from_matrix(m, tile=16, ordering=order)
    tasks = plan.tasks(which)
    pairs, parts = plan.tasks(which + 7), plan.tasks(which + 9)[:, 0]
    # rank of each block's producing task in ticket order, and the task writing each scratch block
    rank = {}
    for t in range(tasks.shape[0]):
        if tasks[t, 0] == 0:
            rank[int(tasks[t, 1])] = t
    writer = {int(tasks[t, 1]): t for t in range(tasks.shape[0]) if tasks[t, 0] in (2, 3)}

    def leaf_blocks(t):
        if tasks[t, 0] == 2:
            return [int(b) for b in pairs[tasks[t, 4]:tasks[t, 5], 1]]
        return [b for q in range(tasks[t, 6], tasks[t, 7]) for b in leaf_blocks(writer[int(parts[q])])]

    checked = 0
    for t in range(tasks.shape[0]):
        if tasks[t, 0] != 0 or tasks[t, 7] == tasks[t, 6]:
            continue
        own = [rank[int(b)] for b in pairs[tasks[t, 4]:tasks[t, 5], 1]]
        leaves = [rank[b] for q in range(tasks[t, 6], tasks[t, 7]) for b in leaf_blocks(writer[int(parts[q])])]
        assert min(own) >= max(leaves)
        checked += 1
    assert checked > 0
    final = tasks[:, 0] == 0
    own = tasks[:, 5] - tasks[:, 4]
    has_parts = tasks[:, 7] > tasks[:, 6]
    assert np.any(final & has_parts)
    assert np.all(own[final & has_parts] >= 8)
    assert np.all(own[final & ~has_parts] <= 32)
    leaves = tasks[tasks[:, 0] == 2]
    assert np.all(leaves[:, 5] - leaves[:, 4] <= 32)
    # every input once: the owners' and the leaves' pair counts add up to the sweep's pair total
    assert own[final].sum() + (leaves[:, 5] - leaves[:, 4]).sum() == tasks[:, 5].max()


@pytest.mark.parametrize("order", [st.ORDER_NONE, st.ORDER_ND])
@pytest.mark.parametrize("which", [1, 2])
def test_sweep_release_lists_and_ready_queue_model(which, order):
    """The release lists of a batched (ready-queue) sweep launch, read back from
    the library, against lists rebuilt here from the sweep's pairs and partial
    lists: each task counts its distinct producers, each producer lists each
    reader once.  Then the queue rule itself, modelled with 1-3 workers: a
    worker takes the next released task, which releases every reader whose
    last producer this was as it starts, and finishes once its producers have
    finished.  Every task must be released exactly once and finish (no worker
    waits on a task that can never run)."""
    m = inputs.band_arrow(6000, 100, 500, 0.2, 3)  # tree partials on the arrow rows
    plan = st.Plan.from_matrix(m, tile=16, ordering=order)
    tasks = plan.tasks(which)
    pairs, parts = plan.tasks(which + 7), plan.tasks(which + 9)[:, 0]
    base = 12 if which == 1 else 15
    cnt0, cptr, cons = (plan.tasks(base + k)[:, 0] for k in range(3))
    n = tasks.shape[0]
    assert cnt0.shape == (n,) and cptr.shape == (n + 1,) and cons.shape == (int(cptr[-1]),)
    final = {int(tasks[t, 1]): t for t in range(n) if tasks[t, 0] == 0}
    writer = {int(tasks[t, 1]): t for t in range(n) if tasks[t, 0] != 0}
    prods = []
    for t in range(n):
        ps = {final[int(b)] for b in pairs[tasks[t, 4]:tasks[t, 5], 1]}
        ps |= {writer[int(s)] for s in parts[tasks[t, 6]:tasks[t, 7]]}
        assert all(p < t for p in ps)  # producers precede their readers in the list
        prods.append(ps)
    assert [len(ps) for ps in prods] == list(cnt0)
    readers = [[] for _ in range(n)]
    for t, ps in enumerate(prods):
        for p in ps:
            readers[p].append(t)
    for p in range(n):
        got = list(cons[cptr[p]:cptr[p + 1]])
        assert sorted(got) == sorted(readers[p]) and len(set(got)) == len(got)
    assert np.any(tasks[:, 0] != 0)  # the case has tree partials

    for workers in (1, 2, 3):
        cnt = cnt0.copy()
        queue = [t for t in range(n) if cnt0[t] == 0]
        head, finished, busy = 0, set(), [None] * workers
        while len(finished) < n:
            progress = False
            for w in range(workers):
                t = busy[w]
                if t is not None and prods[t] <= finished:
                    finished.add(t)
                    busy[w] = None
                    progress = True
            for w in range(workers):
                if busy[w] is None and head < len(queue):
                    t = queue[head]
                    head += 1
                    busy[w] = t
                    for v in cons[cptr[t]:cptr[t + 1]]:
                        cnt[v] -= 1
                        if cnt[v] == 0:
                            queue.append(int(v))
                    progress = True
            assert progress, (workers, len(finished), n)
        assert sorted(queue) == list(range(n))
