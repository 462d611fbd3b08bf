"""GPU parity of libstiles.so against the CPU oracle (FP64 path).

Tolerances (FP64, both sides backward stable; the GPU contracts to FMA and
sums the long arrow chains as a fixed-shape tree):
* factor entries: |L_gpu - L_oracle| <= 1e-11 * max|L| (derived as
  kappa * w * u with kappa <= ~10 for these diagonally dominant inputs,
  inner width w <= 2,100 and u = 1.1e-16, rounded up);
* ||L L^T - P A P^T||_F / ||A||_F <= 1e-13 (spec bound);
* log-determinant: relative 1e-12 against the oracle / closed form;
* solves: ||b - A x|| / ||b|| <= 1e-12 (target 1e-10) and x within 1e-10
  relative of the oracle's x.
"""
import math

import numpy as np
import pytest

from oracle import analyze as oan
from oracle import cholesky as och
from paper_2501_02483_b300 import build, inputs
from tests.golden import make_golden as golden
from paper_2501_02483_b300 import stiles as st

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build_library()
    st.lib()


def _oracle(m, T, order):
    p = oan.analyze(m, T, order)
    L = och.factorize(m, p["perm"], T, p["tcolptr"], p["trowidx"])
    return p, L


def _gpu(m, T, order, block=0, device_values=True, **kw):
    plan = st.Plan.from_matrix(m, tile=T, ordering=order, block=block, **kw)
    f = st.Factor(plan)
    vals = torch.from_numpy(m["values"]).cuda() if device_values else m["values"]
    f.factorize(vals)
    return plan, f


def _gpu_tiles_dict(plan, f, n):
    tiles = f.tiles()
    tc, tr = plan.tilemap()
    T = plan.info()["tile"]
    out = {}
    for k in range(tc.size - 1):
        for e in range(tc[k], tc[k + 1]):
            i = int(tr[e])
            ri = min(T, n - i * T)
            ck = min(T, n - k * T)
            out[(i, k)] = tiles[e].T[:ri, :ck]
    return out


def _compare_factor(m, T, order=oan.ORDER_AUTO, block=0, **kw):
    p, Lo = _oracle(m, T, order)
    plan, f = _gpu(m, T, order, block, **kw)
    assert np.array_equal(plan.perm(), p["perm"])
    Lg = _gpu_tiles_dict(plan, f, m["n"])
    assert set(Lg) == set(Lo)
    scale = max(float(np.max(np.abs(t))) for t in Lo.values())
    worst = max(float(np.max(np.abs(Lg[k] - Lo[k]))) if Lo[k].size else 0.0 for k in Lo)
    assert worst <= 1e-11 * scale, worst / scale
    at = och.scatter_tiles(m, p["perm"], T, p["tcolptr"], p["trowidx"])
    assert och.factor_residual_tiles(Lg, at, p["tcolptr"], p["trowidx"]) <= 1e-13
    ld_o = och.logdet(Lo, p["nt"])
    assert abs(f.logdet() - ld_o) <= 1e-12 * abs(ld_o)
    return p, Lo, plan, f


@pytest.mark.parametrize("T,block", [(64, 32), (64, 64), (32, 0), (16, 0), (64, 16)])
def test_small_config_factor_logdet_solve(T, block):
    m = inputs.config_small(0)
    p, Lo, plan, f = _compare_factor(m, T, oan.ORDER_AUTO, block)
    b = m["rhs"]
    xo = och.solve(Lo, p["perm"], T, p["tcolptr"], p["trowidx"], b)
    x, rr = f.solve(b, relres=True)
    assert rr <= 1e-12
    assert np.max(np.abs(x - xo)) <= 1e-10 * np.max(np.abs(xo))
    # device-resident right-hand sides give the same answer
    xd = f.solve(torch.from_numpy(np.asfortranarray(b)).cuda())
    assert np.max(np.abs(xd.cpu().numpy() - x)) <= 1e-13 * np.max(np.abs(x))


@pytest.mark.parametrize("n_body,w,hw,T,order", [
    (1017, 13, 40, 16, oan.ORDER_NONE),
    (1017, 13, 40, 48, oan.ORDER_RCM),
    (3001, 37, 90, 64, oan.ORDER_AUTO),
    (500, 0, 7, 32, oan.ORDER_NONE),
    (40, 3, 5, 16, oan.ORDER_NONE),
    (3001, 37, 90, 32, oan.ORDER_ND),
    (1017, 13, 40, 16, oan.ORDER_ND),
])
def test_ragged_multi_tile(n_body, w, hw, T, order):
    m = inputs.band_arrow(n_body, w, hw, 0.35, n_body + w)
    p, Lo, plan, f = _compare_factor(m, T, order)
    b = np.random.default_rng(1).normal(size=(m["n"], 5))
    x, rr = f.solve(b, relres=True)
    assert rr <= 1e-12


def test_scrambled_input_with_rcm():
    rng = np.random.default_rng(3)
    m = inputs.band_arrow(2000, 8, 20, 0.4, 5)
    n, nb = m["n"], 2000
    lab = np.concatenate([rng.permutation(nb), np.arange(nb, n)])
    cols = np.repeat(np.arange(n), np.diff(m["colptr"]))
    r, c = lab[m["rowidx"]], lab[cols]
    colptr, rowidx, values = inputs.coo_to_csc_lower(n, np.maximum(r, c), np.minimum(r, c), m["values"])
    ms = {"n": n, "n_arrow": 8, "colptr": colptr, "rowidx": rowidx, "values": values}
    p, Lo, plan, f = _compare_factor(ms, 32, oan.ORDER_AUTO)
    assert plan.info()["ordering_used"] == st.ORDER_RCM


@pytest.mark.parametrize("chunk,fanin", [(1, 2), (3, 2), (4, 16), (32, 16)])
def test_tree_reduction_shapes(chunk, fanin):
    """Long arrow chains split into multi-level trees give the oracle's factor."""
    m = inputs.band_arrow(1500, 40, 12, 0.5, 9)
    p, Lo, plan, f = _compare_factor(m, 16, oan.ORDER_NONE, tree_chunk=chunk, tree_fanin=fanin)
    assert plan.info()["nscratch"] > 0
    b = np.random.default_rng(2).normal(size=(m["n"], 3))
    x, rr = f.solve(b, relres=True)
    assert rr <= 1e-12


def test_pure_arrowhead_closed_form():
    m = inputs.pure_arrowhead(5000, 30, seed=4)
    d, B, D = m["d"], m["B"], m["D"]
    _, lds = np.linalg.slogdet(D - B.T @ (B / d[:, None]))
    expect = math.fsum(np.log(d)) + lds
    plan, f = _gpu(m, 32, oan.ORDER_NONE)
    assert abs(f.logdet() - expect) <= 1e-12 * abs(expect)


def test_tridiagonal_full_scale_closed_form():
    n = 200_000
    m = inputs.tridiag_matrix(n)
    plan, f = _gpu(m, 32, oan.ORDER_NONE)
    assert abs(f.logdet() - math.log(n + 1)) <= 1e-9 * math.log(n + 1)


def test_kronecker_full_scale_closed_form():
    """Q_t (x) Q_s at the spatio-temporal workload's size (n = 202,500, no arrow)."""
    n_t, rho, g, k2 = 100, 0.9, 45, 1.0
    m = inputs.kronecker_spatiotemporal(n_t, rho, g, k2, n_arrow=0, seed=0, nrhs=1)
    ns = g * g
    ld_qt = -(n_t - 1) * math.log(1.0 - rho * rho)
    lam = [2.0 - 2.0 * math.cos(math.pi * a / g) for a in range(g)]
    ld_qs = math.fsum(2.0 * math.log(k2 + la + lb) for la in lam for lb in lam)
    expect = ns * ld_qt + n_t * ld_qs
    plan, f = _gpu(m, 32, oan.ORDER_NONE)
    assert abs(f.logdet() - expect) <= 1e-10 * abs(expect)
    x, rr = f.solve(m["rhs"], relres=True)
    assert rr <= 1e-10


def test_scaling_pin_theta():
    m = inputs.config_small(0)
    theta = 1.37
    _, f1 = _gpu(m, 64, oan.ORDER_AUTO)
    _, f2 = _gpu(inputs.scaled(m, theta), 64, oan.ORDER_AUTO)
    ld1, ld2 = f1.logdet(), f2.logdet()
    assert abs(ld2 - (ld1 + m["n"] * math.log(theta))) <= 1e-12 * abs(ld2)
    x1 = f1.solve(m["rhs"])
    x2 = f2.solve(m["rhs"])
    assert np.max(np.abs(x2 - x1 / theta)) <= 1e-12 * np.max(np.abs(x1))


def test_not_spd_reports_first_bad_column():
    d = np.ones(300)
    d[137] = -2.0
    d[250] = -1.0
    m = inputs.diagonal_matrix(d)
    plan = st.Plan.from_matrix(m, tile=32)
    f = st.Factor(plan)
    with pytest.raises(st.StilesError) as e:
        f.factorize(m["values"])
    assert e.value.name == "NOT_SPD" and e.value.info == 138
    # a band matrix that loses definiteness mid-way: same column as the oracle
    mb = inputs.band_arrow(800, 5, 10, 0.5, 2)
    vals = mb["values"].copy()
    colptr = mb["colptr"]
    vals[colptr[400]] = 0.05  # shrink one diagonal (first entry of column 400 is its diagonal)
    mb2 = dict(mb, values=vals)
    with pytest.raises(och.NotSPD) as eo:
        _oracle(mb2, 32, oan.ORDER_NONE)
    plan2 = st.Plan.from_matrix(mb2, tile=32, ordering=st.ORDER_NONE)
    with pytest.raises(st.StilesError) as eg:
        st.Factor(plan2).factorize(mb2["values"])
    assert eg.value.name == "NOT_SPD" and eg.value.info == eo.value.info


def test_timeout_is_reported_and_context_survives():
    """A wait bound of one poll makes dependent tasks give up: the launch
    returns STILES_ERR_TIMEOUT and the device stays usable."""
    m = inputs.band_arrow(4000, 20, 60, 0.3, 1)
    plan = st.Plan.from_matrix(m, tile=32, spin_limit=1)
    f = st.Factor(plan)
    with pytest.raises(st.StilesError) as e:
        f.factorize(m["values"])
    assert e.value.name == "TIMEOUT"
    torch.cuda.synchronize()
    plan_ok, f_ok = _gpu(m, 32, oan.ORDER_AUTO)
    p, Lo = _oracle(m, 32, oan.ORDER_AUTO)
    assert abs(f_ok.logdet() - och.logdet(Lo, p["nt"])) <= 1e-12 * abs(och.logdet(Lo, p["nt"]))


def test_refactorize_in_place_and_determinism():
    m = inputs.band_arrow(3000, 30, 50, 0.3, 8)
    plan = st.Plan.from_matrix(m, tile=32, tree_chunk=4)
    f = st.Factor(plan)
    f.factorize(m["values"])
    t1 = f.tiles().copy()
    ld1 = f.logdet()
    f.factorize(torch.from_numpy(m["values"]).cuda())
    t2 = f.tiles()
    assert np.array_equal(t1, t2)
    assert f.logdet() == ld1


def test_nested_dissection_large_workload_logdet_and_solve():
    """Adaptable ND on the full 200,000-row workload: same log-determinant as the
    natural order (an invariant of the permutation) and a 1e-12 residual."""
    m = inputs.config_large(0)
    vals = torch.from_numpy(m["values"]).cuda()
    out = {}
    for order in (st.ORDER_NONE, st.ORDER_ND):
        plan = st.Plan.from_matrix(m, tile=16, ordering=order)
        f = st.Factor(plan)
        f.factorize(vals)
        x, rr = f.solve(m["rhs"], relres=True)
        assert rr <= 1e-12
        out[order] = f.logdet()
    ld0 = out[st.ORDER_NONE]
    assert abs(out[st.ORDER_ND] - ld0) <= 1e-12 * abs(ld0)
    # the oracle's value at T = 32 (natural order), written by tests/golden/make_golden.py
    assert abs(ld0 - golden.load()["logdet"]) <= 1e-12 * ld0


@pytest.mark.parametrize("scale", [1e-150, 1e150, 2.0 ** -1000])
def test_extreme_scales_factor_and_logdet(scale):
    """s A has factor sqrt(s) L and logdet logdet(A) + n log s: exercised at
    scales where products of two entries would leave the exponent range (the
    division-free POTRF equilibrates its tile by powers of two first), for the
    tile sizes with that POTRF (16, 32) and the reciprocal one (64)."""
    m = inputs.config_small(3)
    ms = dict(m)
    ms["values"] = m["values"] * scale
    for T in (16, 32, 64):
        plan, f = _gpu(m, T, st.ORDER_RCM, block=T, device_values=False)
        ld = f.logdet()
        plan_s, fs = _gpu(ms, T, st.ORDER_RCM, block=T, device_values=False)
        lds = fs.logdet()
        n = m["n"]
        assert abs(lds - (ld + n * math.log(scale))) <= 1e-12 * abs(n * math.log(scale)) + 1e-10 * abs(ld)
        # entries of the matrix only (the padding past n keeps an unscaled identity)
        Ls, L = _gpu_tiles_dict(plan_s, fs, n), _gpu_tiles_dict(plan, f, n)
        big = max(np.abs(t).max() for t in L.values())
        for key, t in L.items():
            np.testing.assert_allclose(Ls[key] / math.sqrt(scale), t, rtol=1e-12, atol=1e-12 * big)
