"""Seeded synthetic block-arrowhead SPD matrices (inputs only).

This module builds the test and benchmark inputs that both the library and the
CPU oracle consume.  It holds none of the factorization's arithmetic: it only
draws random patterns and values and writes them as a lower-triangular CSC
matrix (diagonal included, rows sorted within each column).

The shapes follow the paper's workloads: a banded "body" of variable
bandwidth followed by a thin dense "arrow" of trailing rows/columns
(Section I, Section V.B and Table 2: arrow thickness 10..200, INLA
spatial/spatio-temporal precision matrices built from Kronecker products).
The paper's own matrices are not published, so these generators stand in for
them.

A matrix is returned as a dict::

    {"n": int, "n_arrow": int,
     "colptr": int64[n+1], "rowidx": int32[nnz], "values": float64[nnz],
     "rhs": float64[n, nrhs] (Fortran order) or None, "name": str}
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "coo_to_csc_lower",
    "band_arrow",
    "config_small",
    "config_large",
    "config_spatiotemporal",
    "kronecker_spatiotemporal",
    "ar1_precision",
    "grid_laplacian",
    "tridiag_matrix",
    "diagonal_matrix",
    "pure_arrowhead",
    "batch_sweep",
    "serving_stream",
    "serving_workload",
    "scaled",
    "dense_from_csc",
    "near_singular_arrowhead",
]


def coo_to_csc_lower(n, rows, cols, vals):
    """Assemble lower-triangular CSC from COO triplets with rows >= cols.

    Duplicates are not allowed (the generators never create them).
    """
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    assert rows.shape == cols.shape == vals.shape
    assert np.all(rows >= cols)
    order = np.lexsort((rows, cols))
    rows, cols, vals = rows[order], cols[order], vals[order]
    counts = np.bincount(cols, minlength=n)
    colptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=colptr[1:])
    return colptr, rows.astype(np.int32), vals


def _with_dominant_diagonal(n, rows, cols, vals, shift=1.0, extra_diag=None):
    """Append a diagonal equal to the absolute off-diagonal row sum + shift.

    The row sum runs over the full symmetric row (lower part of row i plus the
    column-i entries below the diagonal), so the matrix is strictly diagonally
    dominant with a positive diagonal, hence SPD.
    """
    absv = np.abs(vals)
    rowsum = np.bincount(rows, weights=absv, minlength=n) + np.bincount(cols, weights=absv, minlength=n)
    diag = rowsum + shift
    if extra_diag is not None:
        diag = diag + extra_diag
    idx = np.arange(n, dtype=np.int64)
    return (np.concatenate([rows, idx]), np.concatenate([cols, idx]), np.concatenate([vals, diag]))


def band_arrow(n_body, n_arrow, halfwidth, density, seed, nrhs=1, arrow_std=1.0, name="band_arrow",
               rng=None):
    """Variable-bandwidth band body plus a dense arrow, diagonally dominant.

    * body row i (< n_body) has lower half-width ``halfwidth[i]``; each entry
      (i, j) with i - halfwidth[i] <= j < i is present with probability
      ``density`` and drawn U(-1, 1);
    * every lower entry of the arrow rows n_body..n-1 (body columns and the
      arrow's own strictly-lower part) is present and drawn N(0, arrow_std^2);
    * the diagonal is the absolute off-diagonal row sum + 1;
    * ``nrhs`` right-hand sides are drawn N(0, 1).

    Random numbers are drawn in a fixed order from ``default_rng(seed)``:
    for offset d = 1, 2, ... a presence mask then the values of that offset,
    then the arrow values row by row, then the right-hand sides.
    """
    if rng is None:
        rng = np.random.default_rng(seed)
    n = n_body + n_arrow
    hw = np.broadcast_to(np.asarray(halfwidth, dtype=np.int64), (n_body,)) if n_body else np.zeros(0, np.int64)
    rows_l, cols_l, vals_l = [], [], []
    hmax = int(hw.max()) if n_body else 0
    for d in range(1, hmax + 1):
        i = np.arange(d, n_body, dtype=np.int64)
        i = i[hw[d:] >= d]
        if i.size == 0:
            continue
        keep = rng.random(i.size) < density
        i = i[keep]
        rows_l.append(i)
        cols_l.append(i - d)
        vals_l.append(rng.uniform(-1.0, 1.0, i.size))
    for a in range(n_arrow):
        r = n_body + a
        cols = np.arange(r, dtype=np.int64)
        rows_l.append(np.full(r, r, dtype=np.int64))
        cols_l.append(cols)
        vals_l.append(rng.normal(0.0, arrow_std, r))
    rows = np.concatenate(rows_l) if rows_l else np.zeros(0, np.int64)
    cols = np.concatenate(cols_l) if cols_l else np.zeros(0, np.int64)
    vals = np.concatenate(vals_l) if vals_l else np.zeros(0)
    rows, cols, vals = _with_dominant_diagonal(n, rows, cols, vals)
    colptr, rowidx, values = coo_to_csc_lower(n, rows, cols, vals)
    rhs = np.asfortranarray(rng.normal(0.0, 1.0, (n, nrhs))) if nrhs else None
    return {"n": n, "n_arrow": n_arrow, "colptr": colptr, "rowidx": rowidx, "values": values,
            "rhs": rhs, "name": name}


def config_small(seed=0):
    """The small single-matrix case: n = 2,000 body + 10 arrow, half-width 50,
    in-band density 0.3, tile 64, one right-hand side."""
    return band_arrow(2000, 10, 50, 0.3, seed, nrhs=1, name="band2000_hw50_arrow10")


def config_large(seed=0, n_body=200_000, n_arrow=100, nrhs=4):
    """The large single matrix: 200,000 body rows whose lower half-width is
    piecewise constant over 2,000-row segments, drawn uniformly from the
    integers 100..500 per segment; in-band density 0.2; 100 dense arrow
    rows; four right-hand sides.  The segment half-widths are the first draws."""
    rng = np.random.default_rng(seed)
    nseg = (n_body + 1999) // 2000
    seg_hw = rng.integers(100, 501, size=nseg)
    hw = np.repeat(seg_hw, 2000)[:n_body]
    m = band_arrow(n_body, n_arrow, hw, 0.2, seed, nrhs=nrhs, name=f"band{n_body}_hw100-500_arrow{n_arrow}",
                   rng=rng)
    m["segment_halfwidths"] = seg_hw
    return m


def ar1_precision(n_t, rho):
    """Dense precision matrix of a unit-variance stationary AR(1) process."""
    q = np.zeros((n_t, n_t))
    s = 1.0 / (1.0 - rho * rho)
    for t in range(n_t):
        q[t, t] = s * (1.0 + rho * rho) if 0 < t < n_t - 1 else s
        if t + 1 < n_t:
            q[t, t + 1] = q[t + 1, t] = -rho * s
    if n_t == 1:
        q[0, 0] = 1.0
    return q


def grid_laplacian(g):
    """Graph Laplacian D - W of the g x g 5-point grid, as a dense array."""
    n = g * g
    lap = np.zeros((n, n))
    for x in range(g):
        for y in range(g):
            v = x * g + y
            for dx, dy in ((1, 0), (0, 1)):
                xx, yy = x + dx, y + dy
                if xx < g and yy < g:
                    u = xx * g + yy
                    lap[v, u] = lap[u, v] = -1.0
                    lap[v, v] += 1.0
                    lap[u, u] += 1.0
    return lap


def kronecker_spatiotemporal(n_t=100, rho=0.9, g=45, kappa2=1.0, n_arrow=20, arrow_std=0.1, seed=0, nrhs=1):
    """INLA-like spatio-temporal precision Q_t (x) Q_s plus a fixed-effect arrow.

    Q_t is the AR(1) precision (n_t, rho); Q_s = (kappa2 I + L)^2 with L the
    Laplacian of a g x g 5-point grid.  The index is time-major (t * g^2 + s).
    Arrow: B (body x arrow) dense N(0, arrow_std^2); the arrow block D is
    diagonal with D_jj = sum_i |B_ij| + 1, and each body diagonal gets
    sum_j |B_ij| added, which keeps the matrix SPD.  With n_arrow = 0 the
    matrix is exactly Q_t (x) Q_s.
    """
    rng = np.random.default_rng(seed)
    qt = ar1_precision(n_t, rho)
    lap = grid_laplacian(g)
    m = kappa2 * np.eye(g * g) + lap
    qs = m @ m
    ns = g * g
    n_body = n_t * ns
    # lower entries of kron(qt, qs): blocks (t, t') with t >= t'
    srows, scols = np.nonzero(qs)
    svals = qs[srows, scols]
    rows_l, cols_l, vals_l = [], [], []
    for t in range(n_t):
        for tp in (t - 1, t):
            if tp < 0 or qt[t, tp] == 0.0:
                continue
            r = t * ns + srows
            c = tp * ns + scols
            v = qt[t, tp] * svals
            keep = r >= c if tp == t else np.ones(r.size, bool)
            rows_l.append(r[keep])
            cols_l.append(c[keep])
            vals_l.append(v[keep])
    rows = np.concatenate(rows_l).astype(np.int64)
    cols = np.concatenate(cols_l).astype(np.int64)
    vals = np.concatenate(vals_l)
    n = n_body + n_arrow
    if n_arrow:
        b = rng.normal(0.0, arrow_std, (n_arrow, n_body))
        ar_rows = np.repeat(np.arange(n_body, n, dtype=np.int64), n_body)
        ar_cols = np.tile(np.arange(n_body, dtype=np.int64), n_arrow)
        ab = np.abs(b)
        body_extra = ab.sum(axis=0)
        diag_idx = np.arange(n_body, dtype=np.int64)
        is_diag = rows == cols
        vals = vals.copy()
        # add sum_j |B_ij| to the body diagonal
        dpos = np.nonzero(is_diag)[0]
        vals[dpos] += body_extra[rows[dpos]]
        arrow_diag = ab.sum(axis=1) + 1.0
        rows = np.concatenate([rows, ar_rows, np.arange(n_body, n, dtype=np.int64)])
        cols = np.concatenate([cols, ar_cols, np.arange(n_body, n, dtype=np.int64)])
        vals = np.concatenate([vals, b.ravel(), arrow_diag])
        del diag_idx
    colptr, rowidx, values = coo_to_csc_lower(n, rows, cols, vals)
    rhs = np.asfortranarray(rng.normal(0.0, 1.0, (n, nrhs))) if nrhs else None
    return {"n": n, "n_arrow": n_arrow, "colptr": colptr, "rowidx": rowidx, "values": values,
            "rhs": rhs, "name": f"kron_ar1x{n_t}_grid{g}_k2{kappa2}_arrow{n_arrow}",
            "qt": qt, "qs": qs}


def config_spatiotemporal(seed=0, kappa2=1.0):
    """The spatio-temporal case: n_t = 100, rho = 0.9, 45 x 45 grid,
    20 fixed-effect arrow rows with N(0, 0.1^2) couplings."""
    return kronecker_spatiotemporal(100, 0.9, 45, kappa2, 20, 0.1, seed, nrhs=1)


def tridiag_matrix(n):
    """tridiag(-1, 2, -1), whose determinant is n + 1."""
    idx = np.arange(n, dtype=np.int64)
    rows = np.concatenate([idx, idx[1:]])
    cols = np.concatenate([idx, idx[:-1]])
    vals = np.concatenate([np.full(n, 2.0), np.full(n - 1, -1.0)])
    colptr, rowidx, values = coo_to_csc_lower(n, rows, cols, vals)
    return {"n": n, "n_arrow": 0, "colptr": colptr, "rowidx": rowidx, "values": values, "rhs": None,
            "name": f"tridiag{n}"}


def diagonal_matrix(d, n_arrow=0):
    d = np.asarray(d, dtype=np.float64)
    n = d.size
    idx = np.arange(n, dtype=np.int64)
    colptr, rowidx, values = coo_to_csc_lower(n, idx, idx, d)
    return {"n": n, "n_arrow": n_arrow, "colptr": colptr, "rowidx": rowidx, "values": values, "rhs": None,
            "name": f"diag{n}"}


def pure_arrowhead(n_body, n_arrow, seed=0):
    """Diagonal body d plus dense arrow B and dense corner D (SPD).

    Returns the matrix and its blocks (d, B of shape n_body x n_arrow, D) so a
    test can evaluate the Schur-complement determinant formula directly.
    """
    rng = np.random.default_rng(seed)
    d = rng.uniform(1.0, 3.0, n_body)
    b = rng.normal(0.0, 1.0, (n_body, n_arrow)) / math.sqrt(max(n_body, 1))
    c = rng.normal(0.0, 1.0, (n_arrow, n_arrow))
    dd = c @ c.T / max(n_arrow, 1) + np.eye(n_arrow) * (1.0 + (np.abs(b).sum(axis=0).max() if n_body else 0.0) ** 2)
    n = n_body + n_arrow
    rows, cols, vals = [np.arange(n_body)], [np.arange(n_body)], [d]
    ar = np.repeat(np.arange(n_body, n), n_body)
    ac = np.tile(np.arange(n_body), n_arrow)
    rows.append(ar)
    cols.append(ac)
    vals.append(b.T.ravel())
    ri, ci = np.tril_indices(n_arrow)
    rows.append(ri + n_body)
    cols.append(ci + n_body)
    vals.append(dd[ri, ci])
    colptr, rowidx, values = coo_to_csc_lower(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))
    return {"n": n, "n_arrow": n_arrow, "colptr": colptr, "rowidx": rowidx, "values": values, "rhs": None,
            "name": f"arrowhead{n_body}_{n_arrow}", "d": d, "B": b, "D": dd}


def scaled(m, theta):
    """The same matrix multiplied by theta (pattern unchanged)."""
    out = dict(m)
    out["values"] = m["values"] * theta
    out["name"] = f"{m['name']}_x{theta:g}"
    return out


def near_singular_arrowhead(n_body, n_arrow, eps_rel, seed=0):
    """Diagonal body d ~ U(1, 2), dense arrow B ~ N(0, 1), and an arrow block
    D = B^T diag(d)^{-1} B + eps_rel ||B^T diag(d)^{-1} B||_2 I, so the Schur
    complement of the body is eps_rel times its norm times the identity: an SPD
    matrix whose conditioning is set by eps_rel (a low-precision factor of it
    is a poor approximation when eps_rel is near the 16-bit rounding level)."""
    rng = np.random.default_rng(seed)
    d = rng.uniform(1.0, 2.0, n_body)
    B = rng.standard_normal((n_body, n_arrow))
    S = B.T @ (B / d[:, None])
    D = S + eps_rel * np.linalg.norm(S, 2) * np.eye(n_arrow)
    bi, bj = np.nonzero(np.ones((n_body, n_arrow)))
    di, dj = np.tril_indices(n_arrow)
    rows = np.concatenate([np.arange(n_body), n_body + bj, n_body + di])
    cols = np.concatenate([np.arange(n_body), bi, n_body + dj])
    vals = np.concatenate([d, B[bi, bj], D[di, dj]])
    colptr, rowidx, values = coo_to_csc_lower(n_body + n_arrow, rows, cols, vals)
    return {"n": n_body + n_arrow, "n_arrow": n_arrow, "colptr": colptr, "rowidx": rowidx, "values": values,
            "rhs": rng.standard_normal((n_body + n_arrow, 1)), "name": f"nearsing{n_body}_{n_arrow}_{eps_rel}"}


def batch_sweep(count=256, seed=0, n_lo=5_000, n_hi=50_000):
    """Hyperparameter-sweep batch: ``count`` matrices with n log-uniform in
    [n_lo, n_hi], half-width from {64, 128, 256}, arrow width U{0..50},
    values drawn as in the small case, and each whole matrix scaled by
    theta ~ U(0.5, 2).  Returns a list of matrices, each with its "theta"."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        h = int(rng.choice([64, 128, 256]))
        w = int(rng.integers(0, 51))
        theta = float(rng.uniform(0.5, 2.0))
        sub_seed = int(rng.integers(0, 2**31 - 1))
        n_body = max(n - w, 1)
        m = band_arrow(n_body, w, h, 0.3, sub_seed, nrhs=1, name=f"sweep{i}")
        m = scaled(m, theta)
        m["theta"] = theta
        out.append(m)
    return out


def serving_stream(count, rate=500.0, seed=0, n_lo=1_000, n_hi=200_000, resolve_frac=0.3):
    """Poisson request stream for the serving loop.

    Each request is a dict {"t": arrival time [s], "kind": "new"|"resolve",
    "n_body", "halfwidth", "n_arrow", "nrhs", "seed"}; a "resolve" request
    names no matrix (the server picks a resident factor uniformly with the
    request's ``pick`` number in [0, 1))."""
    rng = np.random.default_rng(seed)
    t = 0.0
    reqs = []
    for i in range(count):
        t += float(rng.exponential(1.0 / rate))
        kind = "resolve" if (i > 0 and rng.random() < resolve_frac) else "new"
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        h = int(rng.integers(32, 513))
        w = int(rng.integers(0, 101))
        nrhs = int(rng.integers(1, 17))
        reqs.append({"id": i, "t": t, "kind": kind, "n_body": max(n - w, 1), "halfwidth": h, "n_arrow": w,
                     "nrhs": nrhs, "seed": int(rng.integers(0, 2**31 - 1)), "pick": float(rng.random())})
    return reqs


def dense_from_csc(m):
    """Full symmetric dense array of a (small) lower CSC matrix."""
    n = m["n"]
    a = np.zeros((n, n))
    colptr, rowidx, values = m["colptr"], m["rowidx"], m["values"]
    cols = np.repeat(np.arange(n), np.diff(colptr))
    a[rowidx, cols] = values
    a[cols, rowidx] = values
    return a


def serving_workload(count, rate=500.0, seed=0, n_lo=1_000, n_hi=200_000, hw_lo=32, hw_hi=512, w_hi=100,
                     nrhs_hi=16, resolve_frac=0.3, pool=48, density=0.2, variants=0):
    """Request stream of the serving workload.

    Arrivals are Poisson with the given rate.  A pool of ``pool`` distinct
    patterns is drawn first (n log-uniform in [n_lo, n_hi], lower half-width
    uniform in [hw_lo, hw_hi], arrow uniform in [0, w_hi], in-band density
    ``density``); a new request takes one of them with all values scaled by a
    fresh theta ~ U(0.5, 2) (same structure, new values, as in a
    hyperparameter sweep); a re-solve request (probability ``resolve_frac``)
    names an earlier new request.  Every request carries nrhs ~ U{1..nrhs_hi}
    N(0,1) right-hand sides.  With ``variants`` > 0 each pattern has that many
    pre-drawn thetas and a new request picks one of them (bounds host memory on
    long streams; the matrices still differ from request to request in pattern
    or scale).  Returns (requests, arrivals) with requests as dicts {"id",
    "kind", "key", "matrix", "rhs", "target"}.
    """
    rng = np.random.default_rng(seed)
    shapes = []
    for k in range(pool):
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        h = int(rng.integers(hw_lo, hw_hi + 1))
        w = int(rng.integers(0, w_hi + 1))
        shapes.append(band_arrow(max(n - w, 1), w, min(h, max(n - w - 1, 1)), density, int(rng.integers(0, 2**31 - 1)),
                                 nrhs=0, name=f"serve{k}"))
    t = 0.0
    reqs, arrivals, news = [], [], []
    shared = {}
    for i in range(count):
        t += float(rng.exponential(1.0 / rate))
        nrhs = int(rng.integers(1, nrhs_hi + 1))
        if news and rng.random() < resolve_frac:
            tgt = news[int(rng.integers(0, len(news)))]
            n = reqs[tgt]["matrix"]["n"]
            reqs.append({"id": i, "kind": "resolve", "key": None, "matrix": None,
                         "rhs": np.asfortranarray(rng.normal(0.0, 1.0, (n, nrhs))), "target": tgt})
        else:
            k = int(rng.integers(0, pool))
            theta = float(rng.uniform(0.5, 2.0))
            base = shapes[k]
            if variants > 0:
                v = int(rng.integers(0, variants))
                mat = shared.get((k, v))
                if mat is None:
                    mat = shared[(k, v)] = scaled(base, 0.5 + 1.5 * (v + 0.5) / variants)
            else:
                mat = scaled(base, theta)
            reqs.append({"id": i, "kind": "new", "key": k, "matrix": mat,
                         "rhs": np.asfortranarray(rng.normal(0.0, 1.0, (base["n"], nrhs))), "target": None})
            news.append(i)
        arrivals.append(t)
    return reqs, arrivals
