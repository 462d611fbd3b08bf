"""Pins for the oracle's numeric factorization, log-determinant and solve.

Pins used (none re-runs the oracle's own formulas):
* dense LAPACK Cholesky / slogdet / solve of P A P^T, including the small
  configuration at full scale (n = 2,010);
* closed forms: diagonal matrices; pure arrowheads (Schur complement);
  tridiag(-1, 2, -1) (det = n + 1); Kronecker AR(1) x grid precision
  (spectra of the path-graph Laplacian);
* invariances: tile size, ordering, scaling by theta;
* non-SPD input reports the failing permuted column;
* planted mistakes in the oracle are caught by these pins.
"""
import math

import numpy as np
import pytest

from oracle import analyze as an
from oracle import cholesky as ch
from oracle import tiles
from paper_2501_02483_b300 import inputs


def _run(m, T, order=an.ORDER_NONE):
    p = an.analyze(m, T, order)
    L = ch.factorize(m, p["perm"], T, p["tcolptr"], p["trowidx"])
    return p, L


@pytest.fixture(scope="module")
def small():
    return inputs.config_small(0)


@pytest.mark.parametrize("order", [an.ORDER_NONE, an.ORDER_RCM])
def test_small_config_matches_lapack(small, order):
    m = small
    T = 64
    p, L = _run(m, T, order)
    a = inputs.dense_from_csc(m)
    perm = p["perm"]
    pa = a[np.ix_(perm, perm)]
    lref = np.linalg.cholesky(pa)
    ld = ch.dense_factor(L, m["n"], T, p["tcolptr"], p["trowidx"])
    assert np.max(np.abs(ld - lref)) <= 1e-12 * np.max(np.abs(lref))
    sign, ldref = np.linalg.slogdet(a)
    assert sign == 1.0
    assert abs(ch.logdet(L, p["nt"]) - ldref) <= 1e-12 * abs(ldref)
    x = ch.solve(L, perm, T, p["tcolptr"], p["trowidx"], m["rhs"])
    xref = np.linalg.solve(a, m["rhs"])
    assert np.max(np.abs(x - xref)) <= 1e-12 * np.max(np.abs(xref))
    at = ch.scatter_tiles(m, perm, T, p["tcolptr"], p["trowidx"])
    assert ch.factor_residual_tiles(L, at, p["tcolptr"], p["trowidx"]) <= 1e-15


def test_factor_residual_tiles_matches_dense(small):
    m = small
    T = 64
    p, L = _run(m, T)
    a = inputs.dense_from_csc(m)
    at = ch.scatter_tiles(m, p["perm"], T, p["tcolptr"], p["trowidx"])
    assert ch.factor_residual_tiles(L, at, p["tcolptr"], p["trowidx"]) <= 1e-15
    # perturb one tile: the tiled residual must equal the dense one
    rng = np.random.default_rng(0)
    L2 = dict(L)
    L2[(1, 0)] = L[(1, 0)] + 1e-6 * rng.normal(size=L[(1, 0)].shape)
    L2[(31, 3)] = L[(31, 3)] + 1e-7 * rng.normal(size=L[(31, 3)].shape)
    ld = ch.dense_factor(L2, m["n"], T, p["tcolptr"], p["trowidx"])
    perm = p["perm"]
    pa = a[np.ix_(perm, perm)]
    dense = np.linalg.norm(ld @ ld.T - pa) / np.linalg.norm(pa)
    tiled = ch.factor_residual_tiles(L2, at, p["tcolptr"], p["trowidx"])
    assert dense > 1e-9
    assert abs(dense - tiled) <= 1e-6 * dense


@pytest.mark.parametrize("T", [1, 7, 16, 64, 100, 2048])
def test_tile_size_invariance(T):
    m = inputs.band_arrow(300, 7, 20, 0.3, 11)
    a = inputs.dense_from_csc(m)
    p, L = _run(m, T)
    _, ldref = np.linalg.slogdet(a)
    assert abs(ch.logdet(L, p["nt"]) - ldref) <= 1e-12 * abs(ldref)
    b = np.random.default_rng(0).normal(size=(m["n"], 3))
    x = ch.solve(L, p["perm"], T, p["tcolptr"], p["trowidx"], b)
    assert np.linalg.norm(a @ x - b) <= 1e-13 * np.linalg.norm(b)


def test_diagonal_closed_form():
    d = np.random.default_rng(1).uniform(0.5, 4.0, 500)
    m = inputs.diagonal_matrix(d)
    p, L = _run(m, 32)
    assert abs(ch.logdet(L, p["nt"]) - math.fsum(np.log(d))) <= 1e-13 * abs(math.fsum(np.log(d)))
    b = np.arange(1.0, 501.0)
    x = ch.solve(L, p["perm"], 32, p["tcolptr"], p["trowidx"], b)
    assert np.allclose(x, b / d, rtol=1e-15, atol=0)


@pytest.mark.parametrize("nb,w,T", [(400, 5, 32), (1000, 20, 64), (97, 3, 16)])
def test_pure_arrowhead_schur_closed_form(nb, w, T):
    m = inputs.pure_arrowhead(nb, w, seed=nb)
    d, B, D = m["d"], m["B"], m["D"]
    schur = D - B.T @ (B / d[:, None])
    s, lds = np.linalg.slogdet(schur)
    assert s == 1.0
    expect = math.fsum(np.log(d)) + lds
    p, L = _run(m, T)
    assert abs(ch.logdet(L, p["nt"]) - expect) <= 1e-12 * abs(expect)


def test_tridiagonal_logdet_is_log_n_plus_1():
    n = 20_000
    m = inputs.tridiag_matrix(n)
    p, L = _run(m, 64)
    assert abs(ch.logdet(L, p["nt"]) - math.log(n + 1)) <= 1e-9 * math.log(n + 1)


@pytest.mark.parametrize("kappa2", [0.1, 1.0])
def test_kronecker_closed_form(kappa2):
    n_t, rho, g = 8, 0.9, 6
    m = inputs.kronecker_spatiotemporal(n_t, rho, g, kappa2, n_arrow=0, seed=0, nrhs=0)
    ns = g * g
    ld_qt = -(n_t - 1) * math.log(1.0 - rho * rho)
    lam = [2.0 - 2.0 * math.cos(math.pi * a / g) for a in range(g)]
    ld_qs = math.fsum(2.0 * math.log(kappa2 + la + lb) for la in lam for lb in lam)
    expect = ns * ld_qt + n_t * ld_qs
    for T in (8, 36, 50):
        p, L = _run(m, T, an.ORDER_AUTO)
        assert abs(ch.logdet(L, p["nt"]) - expect) <= 1e-11 * abs(expect)


def test_scaling_by_theta():
    m = inputs.band_arrow(500, 10, 30, 0.3, 4)
    theta = 1.7
    m2 = inputs.scaled(m, theta)
    p, L = _run(m, 32)
    p2, L2 = _run(m2, 32)
    ld, ld2 = ch.logdet(L, p["nt"]), ch.logdet(L2, p2["nt"])
    assert abs(ld2 - (ld + m["n"] * math.log(theta))) <= 1e-12 * abs(ld2)
    x = ch.solve(L, p["perm"], 32, p["tcolptr"], p["trowidx"], m["rhs"])
    x2 = ch.solve(L2, p2["perm"], 32, p2["tcolptr"], p2["trowidx"], m["rhs"])
    assert np.allclose(x2, x / theta, rtol=1e-12, atol=0)


def test_ordering_invariance_of_logdet():
    m = inputs.band_arrow(600, 8, 25, 0.3, 6)
    lds = []
    for order in (an.ORDER_NONE, an.ORDER_RCM, an.ORDER_AUTO):
        p, L = _run(m, 32, order)
        lds.append(ch.logdet(L, p["nt"]))
    assert max(lds) - min(lds) <= 1e-12 * abs(lds[0])


def test_not_spd_reports_permuted_column():
    d = np.ones(100)
    d[37] = -1.0
    m = inputs.diagonal_matrix(d)
    with pytest.raises(ch.NotSPD) as e:
        _run(m, 16)
    assert e.value.info == 38
    d[37] = np.nan
    with pytest.raises(ch.NotSPD) as e:
        _run(inputs.diagonal_matrix(d), 16)
    assert e.value.info == 38


def test_planted_mistake_dropped_latest_term_is_caught(small, monkeypatch):
    """Reading n < k-1 literally (the latest column never updates) must fail the pin."""
    real = tiles.row_lists

    def typo_rows(nt, tcolptr, trowidx):
        rows = real(nt, tcolptr, trowidx)
        return [r[:-2] + r[-1:] if len(r) >= 2 else r for r in rows]

    monkeypatch.setattr(ch._tiles, "row_lists", typo_rows)
    m = small
    try:
        p, L = _run(m, 64)
    except ch.NotSPD:
        return
    a = inputs.dense_from_csc(m)
    _, ldref = np.linalg.slogdet(a)
    assert abs(ch.logdet(L, p["nt"]) - ldref) > 1e-6 * abs(ldref)


def test_planted_mistake_transposed_trsm_is_caught(small, monkeypatch):
    def bad_trsm(a, lkk):
        return a @ np.linalg.inv(lkk)  # A L^{-1} instead of A L^{-T}

    monkeypatch.setattr(ch, "trsm_tile", bad_trsm)
    m = small
    a = inputs.dense_from_csc(m)
    try:
        p, L = _run(m, 64)
    except ch.NotSPD:
        return
    ld = ch.dense_factor(L, m["n"], 64, p["tcolptr"], p["trowidx"])
    assert np.linalg.norm(ld @ ld.T - a) / np.linalg.norm(a) > 1e-6
