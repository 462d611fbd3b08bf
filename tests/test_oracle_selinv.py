"""Pins for the oracle's selected inverse and marginal variances.

Pins used (none re-runs the oracle's recursion):
* the dense inverse of P A P^T (numpy LAPACK), tile by tile on the filled map,
  and its diagonal in the original order, for several tile sizes and orderings;
* closed forms: tridiag(-1, 2, -1), whose inverse is
  min(i, j) (n + 1 - max(i, j)) / (n + 1) (1-based), and the unit-variance
  AR(1) precision, whose inverse is rho^|i - j|;
* a planted mistake (the diagonal block's L_kk^{-T} L_kk^{-1} taken in the
  other order) fails the dense check.
"""
import numpy as np
import pytest

from oracle import analyze as an
from oracle import cholesky as ch
from oracle import selinv as si
from oracle import tiles
from paper_2501_02483_b300 import inputs


def _sigma(m, T, order):
    p = an.analyze(m, T, order)
    L = ch.factorize(m, p["perm"], T, p["tcolptr"], p["trowidx"])
    return p, L, si.selected_inverse(L, p["tcolptr"], p["trowidx"])


def _check_tiles(S, p, T, dense_inv):
    n = dense_inv.shape[0]
    perm = p["perm"]
    inv_p = dense_inv[np.ix_(perm, perm)]
    dims = tiles.tile_dims(n, T)
    worst = 0.0
    scale = np.abs(inv_p).max()
    for (i, k), t in S.items():
        ref = inv_p[i * T:i * T + dims[i], k * T:k * T + dims[k]]
        worst = max(worst, float(np.abs(t - ref).max()) / scale)
    return worst


@pytest.mark.parametrize("T,order", [(64, an.ORDER_AUTO), (16, an.ORDER_NONE), (48, an.ORDER_ND), (32, an.ORDER_RCM)])
def test_matches_dense_inverse_small_config(T, order):
    m = inputs.config_small(0)
    p, L, S = _sigma(m, T, order)
    inv = np.linalg.inv(inputs.dense_from_csc(m))
    assert _check_tiles(S, p, T, inv) <= 1e-12
    var = si.marginal_variances(S, p["perm"], m["n"], T)
    np.testing.assert_allclose(var, np.diag(inv), rtol=1e-12)
    # every tile of the filled map is present, and nothing else
    assert set(S) == set(L)


def test_ragged_arrowhead_matches_dense_inverse():
    m = inputs.band_arrow(437, 9, 23, 0.4, seed=5)
    p, L, S = _sigma(m, 16, an.ORDER_AUTO)
    inv = np.linalg.inv(inputs.dense_from_csc(m))
    assert _check_tiles(S, p, 16, inv) <= 1e-12
    np.testing.assert_allclose(si.marginal_variances(S, p["perm"], m["n"], 16), np.diag(inv), rtol=1e-12)


@pytest.mark.parametrize("n,T", [(300, 16), (257, 32)])
def test_tridiagonal_closed_form(n, T):
    m = inputs.tridiag_matrix(n)
    p, L, S = _sigma(m, T, an.ORDER_NONE)
    i = np.arange(1, n + 1)
    closed = np.minimum.outer(i, i) * (n + 1 - np.maximum.outer(i, i)) / (n + 1)
    assert _check_tiles(S, p, T, closed) <= 1e-13
    np.testing.assert_allclose(si.marginal_variances(S, p["perm"], n, T), i * (n + 1 - i) / (n + 1), rtol=1e-13)


def test_ar1_closed_form():
    n, rho = 200, 0.9
    q = inputs.ar1_precision(n, rho)
    r, c = np.nonzero(np.tril(q))
    colptr, rowidx, values = inputs.coo_to_csc_lower(n, r, c, q[r, c])
    m = {"n": n, "n_arrow": 0, "colptr": colptr, "rowidx": rowidx, "values": values}
    p, L, S = _sigma(m, 16, an.ORDER_NONE)
    idx = np.arange(n)
    closed = rho ** np.abs(idx[:, None] - idx[None, :])
    assert _check_tiles(S, p, 16, closed) <= 1e-12
    np.testing.assert_allclose(si.marginal_variances(S, p["perm"], n, 16), np.ones(n), rtol=1e-12)


def test_planted_mistake_is_caught():
    """The recursion with L_kk^{-1} L_kk^{-T} for the diagonal term (a plausible slip)."""
    m = inputs.config_small(0)
    p = an.analyze(m, 64, an.ORDER_AUTO)
    L = ch.factorize(m, p["perm"], 64, p["tcolptr"], p["trowidx"])
    tcolptr, trowidx = p["tcolptr"], p["trowidx"]
    nt = tcolptr.size - 1
    S = {}
    for k in range(nt - 1, -1, -1):
        below = [int(i) for i in trowidx[tcolptr[k] + 1:tcolptr[k + 1]]]
        linv = np.linalg.inv(L[(k, k)])
        U = {j: L[(j, k)] @ linv for j in below}
        for mm in below:
            acc = 0
            for j in below:
                acc = acc + (S[(mm, j)] if mm >= j else S[(j, mm)].T) @ U[j]
            S[(mm, k)] = -acc
        d = linv @ linv.T  # the slip
        for j in below:
            d = d - S[(j, k)].T @ U[j]
        S[(k, k)] = d
    inv = np.linalg.inv(inputs.dense_from_csc(m))
    assert _check_tiles(S, p, 64, inv) > 1e-6
