"""GPU checks of the sliced-update factorization (STILES_PREC_SLICED): FP64
tiles whose SYRK/GEMM updates run on the tensor cores as exact products of
four BF16 digit slices per operand (per-row power-of-two scales), combined in
64-bit integers; POTRF, TRSM and tree partials in FP64.

Tolerances against the FP64 oracle (and closed forms):
* log-determinant: relative 1e-8 (the stated target for the tensor-core path);
* solves: ||b - A x|| / ||b|| <= 1e-10 after FP64 refinement (the stated target);
  the sweeps run on an FP32 copy of the factor (~1e-7 alone), one refinement step;
* factor entries: |L - L_oracle| <= 1e-8 max|L|.  Derivation: every update
  term is exact up to the slices' representation error, |dL_ij| <= 2^-33 2^e_i
  with 2^e_i <= 2 sqrt(a_ii), i.e. a backward error of about
  2^-32 sqrt(a_ii a_cc) sqrt(K) per entry for K inner terms with independent
  rounding signs (K <= ~400 here: ~1e-8 of the diagonal scale), and these
  inputs are diagonally dominant (the forward error stays of that order).
"""
import math

import numpy as np
import pytest

from oracle import analyze as oan
from oracle import cholesky as och
from paper_2501_02483_b300 import build, inputs
from paper_2501_02483_b300 import stiles as st

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

LD_TOL = 1e-8
RES_TOL = 1e-10
L_TOL = 1e-8


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build_library()
    st.lib()


def _factor(m, T, order, **kw):
    plan = st.Plan.from_matrix(m, tile=T, ordering=order, precision=st.PREC_SLICED, **kw)
    f = st.Factor(plan)
    f.factorize(torch.from_numpy(m["values"]).cuda())
    return plan, f


def _check(m, T, order, **kw):
    p = oan.analyze(m, T, order)
    Lo = och.factorize(m, p["perm"], T, p["tcolptr"], p["trowidx"])
    plan, f = _factor(m, T, order, **kw)
    assert plan.info()["block"] == 32
    assert np.array_equal(plan.perm(), p["perm"])
    tiles = f.tiles()
    tc, tr = plan.tilemap()
    n = m["n"]
    worst, scale = 0.0, 0.0
    for k in range(tc.size - 1):
        for e in range(tc[k], tc[k + 1]):
            i = int(tr[e])
            g = tiles[e].T[:min(T, n - i * T), :min(T, n - k * T)]
            worst = max(worst, float(np.max(np.abs(g - Lo[(i, k)]))))
            scale = max(scale, float(np.max(np.abs(Lo[(i, k)]))))
    assert worst <= L_TOL * scale, worst / scale
    ld_o = och.logdet(Lo, p["nt"])
    ld = f.logdet()
    assert abs(ld - ld_o) <= LD_TOL * abs(ld_o), (ld, ld_o)
    b = m["rhs"] if m.get("rhs") is not None else np.random.default_rng(0).normal(size=(n, 2))
    x, rr = f.solve(b, relres=True)
    assert rr <= RES_TOL
    assert f.refine_iters() <= 2
    xo = och.solve(Lo, p["perm"], T, p["tcolptr"], p["trowidx"], b)
    assert np.max(np.abs(x - xo)) <= 1e-8 * np.max(np.abs(xo))
    return plan, f, worst / scale, abs(ld - ld_o) / abs(ld_o)


@pytest.mark.parametrize("T,order", [(32, oan.ORDER_NONE), (64, oan.ORDER_AUTO)])
def test_small_config_sliced(T, order):
    _check(inputs.config_small(0), T, order)


@pytest.mark.parametrize("T,order", [(32, oan.ORDER_ND), (96, oan.ORDER_RCM)])
def test_ragged_multi_tile_sliced(T, order):
    m = inputs.band_arrow(3001, 37, 90, 0.35, 5)
    _check(m, T, order)


@pytest.mark.parametrize("chunk,fanin", [(1, 2), (4, 16)])
def test_tree_shapes_sliced(chunk, fanin):
    m = inputs.band_arrow(2500, 70, 20, 0.5, 9)
    plan, f, _, _ = _check(m, 32, oan.ORDER_NONE, tree_chunk=chunk, tree_fanin=fanin)
    assert plan.info()["nscratch"] > 0


@pytest.mark.parametrize("kappa2", [0.1, 1.0])
def test_spatiotemporal_small_sliced(kappa2):
    """The Kronecker construction of the spatio-temporal workload with 3 time steps."""
    m = inputs.kronecker_spatiotemporal(3, 0.9, 45, kappa2, 20, 0.1, 0, nrhs=1)
    _, _, lerr, lderr = _check(m, 32, oan.ORDER_ND)
    # measured well inside the bound; the products are exact up to 2^-33 of the row scales
    assert lderr <= 1e-10


def test_kronecker_full_scale_closed_form_sliced():
    """Q_t (x) Q_s at the spatio-temporal workload's size (n = 202,500, no arrow):
    logdet against the closed form n_s logdet Q_t + n_t logdet Q_s."""
    n_t, rho, g, k2 = 100, 0.9, 45, 1.0
    m = inputs.kronecker_spatiotemporal(n_t, rho, g, k2, n_arrow=0, seed=0, nrhs=1)
    ns = g * g
    ld_qt = -(n_t - 1) * math.log(1.0 - rho * rho)
    lam = [2.0 - 2.0 * math.cos(math.pi * a / g) for a in range(g)]
    ld_qs = math.fsum(2.0 * math.log(k2 + la + lb) for la in lam for lb in lam)
    expect = ns * ld_qt + n_t * ld_qs
    plan, f = _factor(m, 32, st.ORDER_ND)
    assert abs(f.logdet() - expect) <= LD_TOL * abs(expect)
    x, rr = f.solve(m["rhs"], relres=True)
    assert rr <= RES_TOL


def test_spatiotemporal_full_size_sliced_matches_fp64():
    """The benchmark's spatio-temporal matrix (n = 202,520, 20 arrow rows): the
    sliced factor's log-determinant within 1e-8 of the FP64 factor's (itself
    pinned to the closed form above without the arrow), relres <= 1e-10."""
    m = inputs.config_spatiotemporal(0)
    vals = torch.from_numpy(m["values"]).cuda()
    p64 = st.Plan.from_matrix(m, tile=16, ordering=st.ORDER_ND)
    f64 = st.Factor(p64)
    f64.factorize(vals)
    ld64 = f64.logdet()
    f64.close()
    plan, f = _factor(m, 32, st.ORDER_ND)
    ld = f.logdet()
    assert abs(ld - ld64) <= LD_TOL * abs(ld64), (ld, ld64)
    x, rr = f.solve(m["rhs"], relres=True)
    assert rr <= RES_TOL


def test_not_spd_sliced():
    m = inputs.config_small(1)
    m = dict(m)
    vals = m["values"].copy()
    # make one diagonal entry negative in the middle of the body
    col = 777
    vals[m["colptr"][col]] = -5.0
    m["values"] = vals
    p = oan.analyze(m, 32, oan.ORDER_NONE)
    with pytest.raises(och.NotSPD) as eo:
        och.factorize(m, p["perm"], 32, p["tcolptr"], p["trowidx"])
    plan = st.Plan.from_matrix(m, tile=32, ordering=st.ORDER_NONE, precision=st.PREC_SLICED)
    f = st.Factor(plan)
    with pytest.raises(st.StilesError) as e:
        f.factorize(torch.from_numpy(m["values"]).cuda())
    assert e.value.name == "NOT_SPD"
    assert e.value.info == eo.value.info


@pytest.mark.parametrize("scale", [1e-150, 1e150])
def test_extreme_scales_sliced(scale):
    """s A: the row scales follow the diagonal, so the factor is sqrt(s) L and the
    log-determinant moves by n log s."""
    m = inputs.config_small(3)
    ms = dict(m)
    ms["values"] = m["values"] * scale
    _, f = _factor(m, 32, st.ORDER_RCM)
    _, fs = _factor(ms, 32, st.ORDER_RCM)
    n = m["n"]
    ld, lds = f.logdet(), fs.logdet()
    assert abs(lds - (ld + n * math.log(scale))) <= 1e-12 * abs(n * math.log(scale)) + 1e-10 * abs(ld)
    # entries of the matrix only (the padding past n keeps an unscaled identity); the
    # row scales follow the diagonal only up to one binade, so the digits differ and
    # the two factors agree to the slices' accuracy
    plan = st.Plan.from_matrix(m, tile=32, ordering=st.ORDER_RCM, precision=st.PREC_SLICED)
    tc, tr = plan.tilemap()
    col = np.repeat(np.arange(tc.size - 1), np.diff(tc))
    t, ts = f.tiles(), fs.tiles() / math.sqrt(scale)
    r_in = (tr[:, None] * 32 + np.arange(32)[None, :]) < n   # tile, row within tile
    c_in = (col[:, None] * 32 + np.arange(32)[None, :]) < n  # tile, column within tile
    mask = c_in[:, :, None] & r_in[:, None, :]               # tiles[e][c][r] holds L(r, c) (column-major)
    assert np.max(np.abs(ts - t)[mask]) <= L_TOL * np.max(np.abs(t[mask]))


def test_sliced_is_deterministic():
    m = inputs.band_arrow(4000, 50, 120, 0.3, 2)
    _, f1 = _factor(m, 32, st.ORDER_ND)
    _, f2 = _factor(m, 32, st.ORDER_ND)
    assert np.array_equal(f1.tiles(), f2.tiles())
    assert f1.logdet() == f2.logdet()


def test_sliced_marginal_variances_match_fp64():
    """The selected inverse runs on a sliced factor as on an FP64 one."""
    m = inputs.band_arrow(3000, 20, 60, 0.3, 4)
    vals = torch.from_numpy(m["values"]).cuda()
    p64 = st.Plan.from_matrix(m, tile=32, ordering=st.ORDER_ND)
    f64 = st.Factor(p64)
    f64.factorize(vals)
    v64 = f64.marginal_variances()
    _, f = _factor(m, 32, st.ORDER_ND)
    v = f.marginal_variances()
    np.testing.assert_allclose(v, v64, rtol=1e-8)


def test_sliced_batch_solves_refine_to_target():
    """A batch of sweep-like matrices (theta-scaled) in one launch: every
    log-determinant within 1e-8 of the oracle and every batched solve refined to
    relres <= 1e-10."""
    mats = inputs.batch_sweep(5, seed=11, n_lo=1500, n_hi=5000)
    plans = [st.Plan.from_matrix(m, tile=32, ordering=st.ORDER_NONE, precision=st.PREC_SLICED) for m in mats]
    batch = st.Batch(plans)
    statuses, _ = batch.factorize([torch.from_numpy(m["values"]).cuda() for m in mats])
    assert np.all(statuses == 0)
    lds = batch.logdets()
    for i, m in enumerate(mats):
        p = oan.analyze(m, 32, oan.ORDER_NONE)
        Lo = och.factorize(m, p["perm"], 32, p["tcolptr"], p["trowidx"])
        ld_o = och.logdet(Lo, p["nt"])
        assert abs(lds[i] - ld_o) <= LD_TOL * abs(ld_o)
    xs, rel, its, status = batch.solve([m["rhs"] for m in mats])
    assert status == 0 and np.all(rel <= RES_TOL) and np.all(its <= 2)
    batch.close()
